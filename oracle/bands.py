"""Number of propagating channels of a pristine armchair ribbon at energy E.

Paper: an ideal ribbon's conductance is step-like, a multiple of 2e^2/h
(discussion of Fig. 3).  The multiple is the number of right-moving Bloch
states at E.  Two independent counts:

* ``channels_closed_form``: the armchair ribbon of N dimer lines separates into
  transverse modes p = 1..N with c_p = cos(p pi / (N + 1)); mode p carries one
  right-mover for |t| |1 + 2 c_p| < |E| < |t| (1 + 2 |c_p|)  (the standard
  nearest-neighbour armchair band edges).
* ``channels_band_structure``: diagonalise H(k) = H00 + H01 e^{ik} + H01^T e^{-ik}
  of the unit cell on a k grid and count, for every band, the sign changes of
  E_b(k) - E with positive slope.

``bloch_ldos`` is the local density of states of the infinite pristine ribbon
per orbital of a cell, from its Bloch states: every crossing k* of a band with
E contributes |psi_b(k*)_i|^2 / (2 pi |dE_b/dk|), the slope taken from the
Hellmann-Feynman form psi^dagger dH/dk psi.
"""
from __future__ import annotations

import numpy as np

from .lattice import blocks


def channels_closed_form(N: int, E: float, t: float = -2.7) -> int:
    """Right-moving channels at E from the closed-form armchair band edges (the
    step-like conductance of an ideal ribbon, discussion of Fig. 3).  A lower
    edge within 1e-12 |t| of |E| counts: the metallic mode of N = 3q + 2 has its
    edge at exactly 0, a linear band crossing that carries one channel at E = 0
    (rounding of the cosine puts the computed edge a few 1e-16 eV off 0)."""
    p = np.arange(1, N + 1)
    c = np.cos(p * np.pi / (N + 1))
    lo = abs(t) * np.abs(1.0 + 2.0 * c)
    hi = abs(t) * (1.0 + 2.0 * np.abs(c))
    return int(np.sum((lo <= abs(E) + 1e-12 * abs(t)) & (abs(E) < hi)))


def band_structure(N: int, nk: int = 2001, t: float = -2.7):
    """Bands E_b(k), k in [-pi, pi) (nk points), shape [nk, 2N] sorted per k
    (the band structure behind the conductance steps discussed with Fig. 3)."""
    H00, H01 = blocks(N, t)
    ks = np.linspace(-np.pi, np.pi, nk, endpoint=False)
    out = np.empty((nk, 2 * N))
    for i, k in enumerate(ks):
        Hk = H00 + H01 * np.exp(1j * k) + H01.T * np.exp(-1j * k)
        out[i] = np.linalg.eigvalsh(Hk)
    return ks, out


def channels_band_structure(N: int, E: float, nk: int = 2001, t: float = -2.7, bands=None) -> int:
    """Count right-moving crossings of E (periodic k grid)."""
    if bands is None:
        _, bands = band_structure(N, nk, t)
    d = bands - E
    d_next = np.roll(d, -1, axis=0)
    up = (d < 0) & (d_next >= 0)
    return int(np.sum(up))


def _hk(H00, H01, k):
    """Bloch Hamiltonian H(k) of the unit cell."""
    return H00 + H01 * np.exp(1j * k) + H01.T * np.exp(-1j * k)


def bloch_ldos(N: int, E: float, nk: int = 4001, t: float = -2.7) -> np.ndarray:
    """LDOS [2N] (states per eV per orbital) of the infinite pristine ribbon."""
    H00, H01 = blocks(N, t)
    ks, bands = band_structure(N, nk, t)
    ks = np.append(ks, np.pi)
    bands = np.vstack([bands, bands[:1]])
    rho = np.zeros(2 * N)
    for b in range(2 * N):
        d = bands[:, b] - E
        for i in np.nonzero(np.sign(d[:-1]) * np.sign(d[1:]) < 0)[0]:
            lo, hi = ks[i], ks[i + 1]
            flo = d[i]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                fm = np.linalg.eigvalsh(_hk(H00, H01, mid))[b] - E
                if np.sign(fm) == np.sign(flo):
                    lo, flo = mid, fm
                else:
                    hi = mid
            k = 0.5 * (lo + hi)
            w, U = np.linalg.eigh(_hk(H00, H01, k))
            psi = U[:, b]
            dH = 1j * H01 * np.exp(1j * k) - 1j * H01.T * np.exp(-1j * k)
            v = float(np.real(psi.conj() @ dH @ psi))
            rho += np.abs(psi) ** 2 / (2.0 * np.pi * abs(v))
    return rho
