"""Armchair graphene nanoribbon tight-binding blocks, from atom coordinates.

Paper: one p orbital per carbon atom, honeycomb lattice with 0.142 nm C-C
distance, armchair edges, semi-infinite leads of the same width (text around
Fig. 1(a)).  The hopping value is not printed in the paper; the workloads use
t = -2.7 eV and on-site energy 0 for the pristine lattice.

Reading used throughout (the paper does not fix an orbital order): a slice is
one unit cell of length 3a holding 2N atoms (N dimer lines, rows j = 0..N-1 at
y = j * sqrt(3)/2 * a).  Even rows hold atoms at x = 0 and x = a, odd rows at
x = 1.5a and x = 2.5a.  Orbital index 2j + k, k = 0 for the left atom of the
row and k = 1 for the right one.  Bonds are found here by brute force: every
pair of atoms at distance a (within a cell for H00, between a cell and the next
one, shifted by 3a, for H01).
"""
from __future__ import annotations

import numpy as np


def cell_coordinates(N: int, a: float = 1.0) -> np.ndarray:
    """(2N, 2) array of (x, y) positions of one unit cell, orbital order 2j + k
    (the geometry of Fig. 1(a))."""
    xy = np.zeros((2 * N, 2))
    h = np.sqrt(3.0) / 2.0 * a
    for j in range(N):
        xs = (0.0, a) if j % 2 == 0 else (1.5 * a, 2.5 * a)
        for k in range(2):
            xy[2 * j + k] = (xs[k], j * h)
    return xy


def _bonds(xa: np.ndarray, xb: np.ndarray, a: float) -> np.ndarray:
    """Adjacency of atoms xa[i], xb[j] at the C-C distance a (nearest neighbours)."""
    d = np.linalg.norm(xa[:, None, :] - xb[None, :, :], axis=-1)
    return np.abs(d - a) < 1e-6 * a


def blocks(N: int, t: float = -2.7, a: float = 1.0):
    """Return (H00, H01): intra-cell and cell(n) -> cell(n+1) hopping blocks (2N x 2N, real).

    H_{n,n+1} = H01 and H_{n+1,n} = H01.T.  One p orbital per carbon atom and
    nearest-neighbour hopping (text around Fig. 1(a)).
    """
    xy = cell_coordinates(N, a)
    nxt = xy + np.array([3.0 * a, 0.0])
    H00 = t * _bonds(xy, xy, a).astype(np.float64)
    H01 = t * _bonds(xy, nxt, a).astype(np.float64)
    return H00, H01


def device_slices(N, L, t, eps, removed):
    """Per-slice blocks of the scattering region with removed atoms dropped.

    eps: [L, 2N] on-site energies (or None), removed: [L, 2N] uint8 (or None).
    Returns (Hd, V, keep): Hd[n] is the on-site block of slice n over its kept
    orbitals, V[n] = H_{n,n+1} between kept orbitals of slices n and n+1
    (n = 0..L-2), keep[n] the kept orbital indices.  (The scattering region of
    length L, Fig. 1(a).)
    """
    H00, H01 = blocks(N, t)
    M = 2 * N
    if eps is None:
        eps = np.zeros((L, M))
    if removed is None:
        removed = np.zeros((L, M), dtype=np.uint8)
    keep = [np.flatnonzero(removed[n] == 0) for n in range(L)]
    Hd = [H00[np.ix_(keep[n], keep[n])] + np.diag(eps[n, keep[n]]) for n in range(L)]
    V = [H01[np.ix_(keep[n], keep[n + 1])] for n in range(L - 1)]
    return Hd, V, keep


def full_hamiltonian(N, L, t, eps, removed):
    """Dense Hamiltonian of the L-slice scattering region (kept orbitals only). (The H of Eq. 1.)"""
    Hd, V, keep = device_slices(N, L, t, eps, removed)
    sizes = [len(k) for k in keep]
    off = np.concatenate([[0], np.cumsum(sizes)])
    H = np.zeros((off[-1], off[-1]))
    for n in range(L):
        H[off[n]:off[n + 1], off[n]:off[n + 1]] = Hd[n]
    for n in range(L - 1):
        H[off[n]:off[n + 1], off[n + 1]:off[n + 2]] = V[n]
        H[off[n + 1]:off[n + 2], off[n]:off[n + 1]] = V[n].T
    return H, off, keep
