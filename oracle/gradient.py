"""dT/d eps_i for every on-site energy of the scattering region.

The paper does not differentiate; the derivative follows from Eq. 1 and
Eq. 2.  With A = z - H - Sigma and dA/d eps_i = -e_i e_i^T, dG = G e_i e_i^T G,
so for T = Tr[Gamma_L G_1L Gamma_R G_1L^dagger] (Gamma real symmetric here):

    dT/d eps_i = 2 Re[ G_{i,L} Gamma_R G_{1L}^dagger Gamma_L G_{1,i} ]

``closed_form`` evaluates this with the dense G (small ribbons only).
``adjoint`` is the reverse sweep of the recursion of ``rgf.forward``: with
X_bar = dT/dX (holomorphic part, dT = 2 Re Tr[X_bar^T dX]) and g_j symmetric,

    P_bar_L = Gamma_L conj(P_L) Gamma_R
    for j = L..1:
        g_bar_j = [V^T P_{j-1}^T P_bar_j  if j > 1]  + [P_bar_1 if j = 1]
                - [V_{j,j+1} A_bar_{j+1} V_{j,j+1}^T  if j < L]
        A_bar_j = -g_j g_bar_j g_j
        dT/d eps_{j,i} = -2 Re (A_bar_j)_ii
        P_bar_{j-1} = P_bar_j g_j V_{j-1,j}^T

``two_sided`` evaluates the closed form slice by slice without the dense G:
the blocks it needs follow from the Dyson equation (Eq. 3) with the bond
between slices j-1 and j (or j and j+1) cut,

    G_jj = (A_j - V_{j-1,j}^T gl_{j-1} V_{j-1,j} - V_{j,j+1} gr_{j+1} V_{j,j+1}^T)^-1
    G_{1j} = Pl_{j-1} V_{j-1,j} G_jj,        G_{jL} = G_jj V_{j,j+1} Qr_{j+1}

with gl, Pl = G_{1j} of the part left of the cut (the forward recursion of
Eqs. 4-5) and gr, Qr = G_{jL} of the part right of it (the same recursion run
from the right lead), A_j = z - H_jj (minus Sigma_L, Sigma_R on the end
slices).  It forms the blocks of the whole system's G directly instead of
propagating the cotangents through the half systems' Green's functions.
Near the poles of the half systems (E close to 0, where the ends of a cut
carry nearly bound states) the reverse sweep loses accuracy at isolated
sites (rounding amplified by the large g_j), while this form stays at the
dense closed form (tests/test_oracle.py).

Removed atoms get derivative 0.
"""
from __future__ import annotations

import numpy as np

from .dense import green_dense
from .lattice import device_slices
from .leads import broadening, self_energies
from .rgf import forward


def closed_form(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None):
    """dT/d eps_i = 2 Re[G_iL Gamma_R G_1L^dagger Gamma_L G_1i] with the dense G (from Eqs. 1-2)."""
    G, off, keep, sigL, sigR = green_dense(N, L, E, eta_device, eta_lead, t, eps, removed)
    gL, gR = broadening(sigL), broadening(sigR)
    first = slice(off[0], off[1])
    last = slice(off[L - 1], off[L])
    G1L = G[first, last]
    mid = gR @ G1L.conj().T @ gL          # K_L x K_1
    # dT/d eps_i = 2 Re sum_{a,b} G[i, last_a] mid[a, b] G[first_b, i]
    vals = 2.0 * np.real(np.einsum("ia,ab,bi->i", G[:, last], mid, G[first, :]))
    out = np.zeros((L, 2 * N))
    for n in range(L):
        out[n, keep[n]] = vals[off[n]:off[n + 1]]
    return out


def adjoint(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """Returns (T, dT/d eps [L, 2N]). Reverse sweep of the recursion of Eqs. 4-5 (from Eqs. 1-2)."""
    f = forward(N, L, E, eta_device, eta_lead, t, eps, removed, sig, keep_history=True)
    g, Ps, V, keep = f["g"], f["Ps"], f["V"], f["keep"]
    gL, gR = broadening(f["sigL"]), broadening(f["sigR"])
    Pbar = gL @ np.conj(Ps[-1]) @ gR
    out = np.zeros((L, 2 * N))
    Abar_next = None
    for j in range(L - 1, -1, -1):
        gbar = np.zeros_like(g[j])
        if j > 0:
            gbar += V[j - 1].T @ Ps[j - 1].T @ Pbar
        else:
            gbar += Pbar
        if j < L - 1:
            gbar -= V[j] @ Abar_next @ V[j].T
        Abar = -g[j] @ gbar @ g[j]
        out[j, keep[j]] = -2.0 * np.real(np.diag(Abar))
        if j > 0:
            Pbar = Pbar @ g[j] @ V[j - 1].T
        Abar_next = Abar
    return f["T"], out


def half_sweeps(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """The left- and right-connected recursions (Eqs. 4-5 from either lead).

    Returns a dict with the slice matrices A_j (z - H_jj, minus Sigma_L and
    Sigma_R on the end slices), the couplings V, the kept-atom lists, gl / Pl
    (G_jj and G_1j of slices 1..j), gr / Qr (G_jj and G_jL of slices j..L) and
    the lead self-energies restricted to the kept atoms."""
    Hd, V, keep = device_slices(N, L, t, eps, removed)
    if sig is None:
        sig = self_energies(N, E, eta_lead, t)
    sigL = sig[0][np.ix_(keep[0], keep[0])]
    sigR = sig[1][np.ix_(keep[-1], keep[-1])]
    z = E + 1j * eta_device
    A = [z * np.eye(len(keep[j])) - Hd[j] for j in range(L)]
    A[0] = A[0] - sigL
    A[L - 1] = A[L - 1] - sigR
    gl, Pl = [], []
    for j in range(L):
        Aj = A[j] if j == 0 else A[j] - V[j - 1].T @ gl[j - 1] @ V[j - 1]
        gl.append(np.linalg.inv(Aj))
        Pl.append(gl[j] if j == 0 else Pl[j - 1] @ V[j - 1] @ gl[j])
    gr, Qr = [None] * L, [None] * L
    for j in range(L - 1, -1, -1):
        Aj = A[j] if j == L - 1 else A[j] - V[j] @ gr[j + 1] @ V[j].T
        gr[j] = np.linalg.inv(Aj)
        Qr[j] = gr[j] if j == L - 1 else gr[j] @ V[j] @ Qr[j + 1]
    return dict(A=A, V=V, keep=keep, gl=gl, Pl=Pl, gr=gr, Qr=Qr, sigL=sigL, sigR=sigR)


def diagonal_block(h, j):
    """G_jj of the whole system: (A_j - V^T gl_{j-1} V - V gr_{j+1} V^T)^-1. (Dyson, Eq. 3.)"""
    A, V, gl, gr = h["A"], h["V"], h["gl"], h["gr"]
    L = len(A)
    Aj = A[j].copy()
    if j > 0:
        Aj -= V[j - 1].T @ gl[j - 1] @ V[j - 1]
    if j < L - 1:
        Aj -= V[j] @ gr[j + 1] @ V[j].T
    return np.linalg.inv(Aj)


def two_sided(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, sig=None):
    """Returns (T, dT/d eps [L, 2N]) from the closed form with the blocks of G
    assembled by the Dyson relations above (left- and right-connected sweeps).
    (Eqs. 1-3.)"""
    h = half_sweeps(N, L, E, eta_device, eta_lead, t, eps, removed, sig)
    V, keep, Pl, Qr = h["V"], h["keep"], h["Pl"], h["Qr"]
    G1L = Pl[L - 1]
    gL, gR = broadening(h["sigL"]), broadening(h["sigR"])
    T = float(np.real(np.trace(gL @ G1L @ gR @ G1L.conj().T)))
    mid = gR @ G1L.conj().T @ gL          # K_L x K_1
    out = np.zeros((L, 2 * N))
    for j in range(L):
        Gjj = diagonal_block(h, j)
        G1j = Gjj if j == 0 else Pl[j - 1] @ V[j - 1] @ Gjj
        GjL = Gjj if j == L - 1 else Gjj @ V[j] @ Qr[j + 1]
        out[j, keep[j]] = 2.0 * np.real(np.einsum("ia,ab,bi->i", GjL, mid, G1j))
    return T, out
