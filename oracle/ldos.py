"""Local density of states of the scattering region, rho_i(E) = -Im G_ii / pi.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper notes that the Green's function of Eq. 1 gives every quantity of
interest, the charge density among them; the local density of states is its
integrand over energy.  Its diagonal G_ii comes from the diagonal blocks of G,
each assembled by the Dyson equation (Eq. 3) with the bonds on both sides of
slice j cut (gradient.half_sweeps / gradient.diagonal_block):

    G_jj = (A_j - V_{j-1,j}^T gl_{j-1} V_{j-1,j} - V_{j,j+1} gr_{j+1} V_{j,j+1}^T)^-1

Removed atoms get rho = 0.
"""
from __future__ import annotations

import numpy as np

from .gradient import diagonal_block, half_sweeps


def ldos(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """rho_i(E) in states per eV per orbital, [L, 2N]. (From Eq. 1; Dyson-assembled diagonal
    blocks, Eq. 3.)"""
    h = half_sweeps(N, L, E, eta_device, eta_lead, t, eps, removed, sig)
    out = np.zeros((L, 2 * N))
    for j in range(L):
        out[j, h["keep"][j]] = -np.imag(np.diag(diagonal_block(h, j))) / np.pi
    return out
