"""Recursive Green's function sweep over unit-cell slices (Eqs. 4-5) and Eq. 2.

Eq. 4 reads G_jj = (1 - G0_jj S^l G_{j-1,j-1} S^r)^-1 G0_jj, with G0_jj the
Green's function of the isolated slice and S^l, S^r the couplings to the
previous slice.  Since (1 - G0 X)^-1 G0 = ((G0)^-1 - X)^-1 and
(G0_jj)^-1 = z - H_jj, the oracle uses the algebraically identical form

    g_1 = (z - H_11 - Sigma_L)^-1
    g_j = (z - H_jj - V_{j-1,j}^T g_{j-1} V_{j-1,j})^-1        (Eq. 4)
    P_1 = g_1,   P_j = P_{j-1} V_{j-1,j} g_j  ( = G_{1j} )        (Eq. 5)

with Sigma_R also subtracted on the last slice, so that P_L = G_{1L} of the
whole system.  It never inverts the isolated slice (singular at its
eigenvalues when eta_device = 0).  T = Tr[Gamma_L P_L Gamma_R P_L^dagger] (Eq. 2).
Removed atoms are dropped, so slices may be ragged.
"""
from __future__ import annotations

import numpy as np

from .lattice import device_slices
from .leads import self_energies, broadening


def _sigmas(N, E, eta_lead, t, keep, sig):
    """Lead self-energies restricted to the kept atoms of the end slices (text after Eqs. 4-5)."""
    if sig is None:
        sig = self_energies(N, E, eta_lead, t)
    sigL_full, sigR_full = sig
    return sigL_full[np.ix_(keep[0], keep[0])], sigR_full[np.ix_(keep[-1], keep[-1])]


def forward(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None,
            keep_history=False):
    """Left-to-right sweep. Returns dict with T, P (= G_1L), and optionally g[], P[] history. (Eqs.
    4-5, then Eq. 2.)"""
    Hd, V, keep = device_slices(N, L, t, eps, removed)
    sigL, sigR = _sigmas(N, E, eta_lead, t, keep, sig)
    z = E + 1j * eta_device
    gs, Ps = [], []
    g = None
    P = None
    for j in range(L):
        A = z * np.eye(len(keep[j])) - Hd[j]
        if j == 0:
            A = A - sigL
        else:
            A = A - V[j - 1].T @ g @ V[j - 1]
        if j == L - 1:
            A = A - sigR
        g = np.linalg.inv(A)
        P = g if j == 0 else P @ V[j - 1] @ g
        if keep_history:
            gs.append(g)
            Ps.append(P)
    gL, gR = broadening(sigL), broadening(sigR)
    T = float(np.real(np.trace(gL @ P @ gR @ P.conj().T)))
    out = dict(T=T, P=P, sigL=sigL, sigR=sigR, keep=keep, V=V)
    if keep_history:
        out.update(g=gs, Ps=Ps)
    return out


def transmission(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """T of Eq. 2 by the forward recursion of Eqs. 4-5."""
    return forward(N, L, E, eta_device, eta_lead, t, eps, removed, sig)["T"]


def transmission_right_to_left(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None,
                               sig=None):
    """The mirror sweep (from the right lead to the left): T_RL = Tr[Gamma_R G_L1 Gamma_L
    G_L1^dagger]."""
    Hd, V, keep = device_slices(N, L, t, eps, removed)
    sigL, sigR = _sigmas(N, E, eta_lead, t, keep, sig)
    z = E + 1j * eta_device
    g = None
    Q = None
    for j in range(L - 1, -1, -1):
        A = z * np.eye(len(keep[j])) - Hd[j]
        if j == L - 1:
            A = A - sigR
        else:
            A = A - V[j] @ g @ V[j].T
        if j == 0:
            A = A - sigL
        g = np.linalg.inv(A)
        Q = g if j == L - 1 else Q @ V[j].T @ g
    gL, gR = broadening(sigL), broadening(sigR)
    return float(np.real(np.trace(gR @ Q @ gL @ Q.conj().T)))
