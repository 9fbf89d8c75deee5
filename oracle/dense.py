"""The plain definition of the conductance, by dense inversion (small ribbons only).

Eq. 1: G = (E - H)^-1, with E -> E + i eta_device and the leads folded into H
as Sigma_L on the first slice and Sigma_R on the last.  Eq. 2: the conductance
in units of 2e^2/h is T = Tr[Gamma_L G_{1L} Gamma_R G_{1L}^dagger], with
Gamma = i(Sigma - Sigma^dagger).  (The paper writes Tr[Gamma_L G^a Gamma_R G^r];
the two agree because H is real symmetric, so G is complex symmetric.)
"""
from __future__ import annotations

import numpy as np

from .lattice import full_hamiltonian
from .leads import self_energies, broadening


def green_dense(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """Dense retarded G of the scattering region. Returns (G, off, keep, sigL, sigR). (Eq. 1.)"""
    H, off, keep = full_hamiltonian(N, L, t, eps, removed)
    if sig is None:
        sig = self_energies(N, E, eta_lead, t)
    sigL_full, sigR_full = sig
    sigL = sigL_full[np.ix_(keep[0], keep[0])]
    sigR = sigR_full[np.ix_(keep[-1], keep[-1])]
    A = (E + 1j * eta_device) * np.eye(H.shape[0]) - H
    A[off[0]:off[1], off[0]:off[1]] -= sigL
    A[off[L - 1]:off[L], off[L - 1]:off[L]] -= sigR
    G = np.linalg.inv(A)
    return G, off, keep, sigL, sigR


def transmission_dense(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """T of Eq. 2 from the dense G of Eq. 1."""
    G, off, keep, sigL, sigR = green_dense(N, L, E, eta_device, eta_lead, t, eps, removed, sig)
    G1L = G[off[0]:off[1], off[L - 1]:off[L]]
    gL, gR = broadening(sigL), broadening(sigR)
    return float(np.real(np.trace(gL @ G1L @ gR @ G1L.conj().T)))


def transmission_dense_paper_form(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None):
    """Eq. 2 exactly as printed: Tr[Gamma_L G^a Gamma_R G^r] with G^a = (G^r)^dagger."""
    G, off, keep, sigL, sigR = green_dense(N, L, E, eta_device, eta_lead, t, eps, removed)
    Ga = G.conj().T
    gL, gR = broadening(sigL), broadening(sigR)
    Ga_1L = Ga[off[0]:off[1], off[L - 1]:off[L]]
    Gr_L1 = G[off[L - 1]:off[L], off[0]:off[1]]
    return float(np.real(np.trace(gL @ Ga_1L @ gR @ Gr_L1)))
