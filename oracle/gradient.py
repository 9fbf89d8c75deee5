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

Removed atoms get derivative 0.
"""
from __future__ import annotations

import numpy as np

from .dense import green_dense
from .leads import broadening
from .rgf import forward


def closed_form(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None):
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
    """Returns (T, dT/d eps [L, 2N])."""
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
