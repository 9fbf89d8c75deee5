"""Seeded synthetic inputs for the armchair-nanoribbon RGF workloads.

This module is shared by the CPU oracle (``oracle/``), the tests and
``bench.py``.  It holds no arithmetic of the transport method itself: only
random draws (Anderson on-site energies, edge-roughness removal masks, random
chain parameters), energy grids and the descriptions of the standard workloads.

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: draw number ``i`` of stream ``seed`` is
``mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)`` (mod 2**64), where ``mix64`` is
the SplitMix64 output function.  A uniform double in [0, 1) is
``(bits >> 11) * 2**-53``.  The C library implements the same definition
independently (``rgf_generate_onsite``), so a ribbon described by seeds is the
same ribbon on both sides, bit for bit.

Draw indices for a ribbon of ``N`` dimer lines and ``L`` unit cells: the draw for
orbital ``o = 2*j + k`` (row ``j``, ``k = 0`` left atom, ``k = 1`` right atom) of
cell ``n`` is number ``n * 2N + o``.  Anderson energies use stream ``seed``:
``eps = W * (2u - 1)``.  Edge roughness uses stream ``edge_seed``: an atom of
row 0 or row N-1 is removed when ``u < p``; atoms of the other rows are never
drawn.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = 2.0 ** -53

# Physical constants of the standard workloads.
T_HOP = -2.7          # nearest-neighbour hopping, eV
A_CC = 0.142          # carbon-carbon distance, nm
ETA = 1e-8            # broadening, eV


def mix64(z):
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64(seed: int, index):
    """Draw(s) number ``index`` of the SplitMix64 stream ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN
    return mix64(state)


def uniform01(seed: int, index):
    """Uniform doubles in [0, 1) from draw(s) ``index`` of stream ``seed``."""
    bits = splitmix64(seed, index)
    return (bits >> np.uint64(11)).astype(np.float64) * _TWO_M53


def anderson_onsite(N: int, L: int, W: float, seed: int) -> np.ndarray:
    """On-site energies eps[L, 2N] i.i.d. uniform in [-W, W] eV."""
    M = 2 * N
    idx = np.arange(L * M, dtype=np.uint64)
    u = uniform01(seed, idx)
    return (W * (2.0 * u - 1.0)).reshape(L, M)


def edge_removed(N: int, L: int, p: float, seed: int) -> np.ndarray:
    """Removal mask removed[L, 2N] (uint8): outermost-row atoms dropped with prob. p."""
    M = 2 * N
    out = np.zeros((L, M), dtype=np.uint8)
    if p <= 0.0:
        return out
    rows = sorted({0, N - 1})
    orbs = np.array([2 * j + k for j in rows for k in (0, 1)], dtype=np.uint64)
    n = np.arange(L, dtype=np.uint64)[:, None]
    idx = n * np.uint64(M) + orbs[None, :]
    u = uniform01(seed, idx)
    out[:, orbs.astype(np.int64)] = (u < p).astype(np.uint8)
    return out


def energy_grid(lo: float, hi: float, K: int) -> np.ndarray:
    """K energies uniform in [lo, hi], endpoints included."""
    return np.linspace(lo, hi, K)


def derived_seed(seed: int, index: int) -> int:
    """An independent seed for sub-stream ``index`` of ``seed`` (one SplitMix64 draw)."""
    return int(splitmix64(seed, np.uint64(index)))


# ---------------------------------------------------------------------------
# Standard workloads, named by what they are.
# ---------------------------------------------------------------------------

def agnr245_energies() -> np.ndarray:
    """64 energies in [-0.5, 0.5] eV plus the five near the charge-neutrality point."""
    return np.concatenate([energy_grid(-0.5, 0.5, 64),
                           np.array([0.0, 1e-3, -1e-3, 5e-3, -5e-3])])


WORKLOADS = {
    # Pristine N=11 ribbon, 50 cells, 201 energies in [-1, 1] eV.
    "agnr11_L50_pristine": dict(N=11, L=50, W=0.0, seed=0, edge_p=0.0, edge_seed=0,
                                energies=lambda: energy_grid(-1.0, 1.0, 201)),
    # W = 30 nm ribbon (N=245, 490 orbitals per cell), 4000 cells (1.7 um),
    # Anderson disorder +-0.25 eV, 69 energies.
    "agnr245_L4000_anderson": dict(N=245, L=4000, W=0.25, seed=1, edge_p=0.0, edge_seed=0,
                                   energies=agnr245_energies),
    # Gradient workload: N=101, 500 cells, Anderson +-0.15 eV, 128 energies.
    "agnr101_L500_grad": dict(N=101, L=500, W=0.15, seed=4, edge_p=0.0, edge_seed=0,
                              energies=lambda: energy_grid(-0.8, 0.8, 128), ckpt_stride=23),
    # W = 123 nm ribbon (N=1001), 2000 cells, Anderson +-0.1 eV, edge p=0.02,
    # 256 energies; gradients at energies 16 + 32k, k = 0..7.
    "agnr1001_L2000": dict(N=1001, L=2000, W=0.1, seed=5, edge_p=0.02, edge_seed=55,
                           energies=lambda: energy_grid(-0.3, 0.3, 256),
                           grad_idx=[16 + 32 * k for k in range(8)]),
}


def batched_uneven_chains(n_chains: int = 2048, seed: int = 3):
    """Independent chains with N ~ U{51..401}, L ~ U{100..2000}, E ~ U[-1, 1] eV.

    Each chain carries Anderson disorder U[-0.1, 0.1] eV and edge roughness
    p = 0.05, with its own derived seeds.  Returns a list of dicts.
    """
    out = []
    for c in range(n_chains):
        u = uniform01(seed, np.arange(4 * c, 4 * c + 3, dtype=np.uint64))
        N = 51 + int(u[0] * 351)
        L = 100 + int(u[1] * 1901)
        E = -1.0 + 2.0 * float(u[2])
        out.append(dict(N=N, L=L, E=E, W=0.1, seed=derived_seed(seed, 2 * c + 100000),
                        edge_p=0.05, edge_seed=derived_seed(seed, 2 * c + 100001)))
    return out
