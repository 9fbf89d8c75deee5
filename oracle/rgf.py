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


def transmission_modes(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None):
    """T of Eq. 2 by the recursion of Eqs. 4-5 with the lead-attached atoms of the
    end slices written in the leads' transverse-mode basis (oracle.modes).

    The recursion and the trace are those of ``forward``, in the basis rotated by
    R = U_even on the even-row left atoms of slice 1 and R' = U_odd on the
    odd-row right atoms of slice L (identity elsewhere), an orthogonal change of
    basis that leaves G_1L's blocks and T unchanged.  In that basis the lead
    self-energies are diagonal (w_p), so the first and last slice matrices are

        A~ = R^T (z - H_jj - V^T g V) R - diag(w)

    and the order-1/eta self-energies of the surface-state modes near E = 0
    never meet the order-1 entries of z - H_jj in one sum.  The corner block is
    carried with its rows in the left lead's mode basis, P~_j = U_even^T G_1j,
    and T = sum_pq gamma_p gamma'_q |(U_even^T G_1L U_odd)_pq|^2 with
    gamma = -2 Im w.  The lead-attached atoms of slices 1 and L must not be
    removed (ValueError otherwise).
    """
    from .modes import left_orbitals, mode_self_energies, mode_vectors, right_orbitals
    Hd, V, keep = device_slices(N, L, t, eps, removed)
    UL, UR = mode_vectors(N)
    KL, KR = UL.shape[0], UR.shape[0]
    w = mode_self_energies(N, E, eta_lead, t)
    gamL, gamR = -2.0 * w.imag, -2.0 * w[:KR].imag
    iL, iR = left_orbitals(N), right_orbitals(N)
    pos0 = np.searchsorted(keep[0], iL)
    posL = np.searchsorted(keep[-1], iR)
    if not (np.array_equal(keep[0][np.minimum(pos0, len(keep[0]) - 1)], iL) and
            np.array_equal(keep[-1][np.minimum(posL, len(keep[-1]) - 1)], iR)):
        raise ValueError("transmission_modes: a lead-attached atom of an end slice is removed")
    z = E + 1j * eta_device

    def rotation(n, blocks):
        R = np.eye(n)
        for pos, U in blocks:
            R[np.ix_(pos, pos)] = U
        return R

    g = P = None
    for j in range(L):
        n = len(keep[j])
        B = z * np.eye(n) - Hd[j]
        if j > 0:
            B = B - V[j - 1].T @ g @ V[j - 1]
        ends = []
        if j == 0:
            ends.append((pos0, UL, w))
        if j == L - 1:
            ends.append((posL, UR, w[:KR]))
        if not ends:
            g = np.linalg.inv(B)
            P = P @ V[j - 1] @ g
            continue
        R = rotation(n, [(pos, U) for pos, U, _ in ends])
        At = R.T @ B @ R
        for pos, _, wp in ends:
            At[pos, pos] -= wp
        gt = np.linalg.inv(At)                      # R^T g R
        if j == 0:
            P = (gt @ R.T)[pos0, :]                 # U_even^T G_11 (rows in mode basis)
        else:
            P = P @ V[j - 1] @ R @ gt               # columns of slice L in the rotated basis
        g = R @ gt @ R.T
    Pt = P[:, posL] if L > 1 else (gt[np.ix_(pos0, posL)])
    return float(np.sum(gamL[:, None] * gamR[None, :] * np.abs(Pt) ** 2))
