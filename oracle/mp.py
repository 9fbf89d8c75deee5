"""The unit-cell recursion (Eqs. 4-5) and Eq. 2 in arbitrary precision (mpmath).

Near the charge-neutrality point the problem is ill-conditioned: the
transverse cut of an armchair ribbon is a zigzag edge, so the surface Green's
function of each semi-infinite lead has an edge-state pole at E = 0 whose
weight only cancels at the last slice.  The paper reports the resulting
single-precision error near E = 0 (discussion of Fig. 3); at E = 0 exactly
with eta = 1e-8 eV even complex128 loses digits.  This module repeats the
decimation of ``leads`` and the recursion of ``rgf`` with ``dps`` decimal
digits, for small ribbons only, to pin what complex128 cannot.
"""
from __future__ import annotations

import mpmath as mpm
import numpy as np

from .lattice import blocks, device_slices


def _m(a):
    """mpmath matrix from a numpy array."""
    return mpm.matrix(np.asarray(a).tolist())


def _absmax(m):
    """Largest entry magnitude of an mpmath matrix."""
    return max(abs(m[i, j]) for i in range(m.rows) for j in range(m.cols))


def _surface(H00, a0, b0, z, tol):
    """Sancho-Rubio decimation in dps digits (text after Eqs. 4-5)."""
    M = H00.rows
    I = mpm.eye(M)
    eps_s, eps, al, be = H00.copy(), H00.copy(), a0.copy(), b0.copy()
    for _ in range(400):
        g = mpm.inverse(z * I - eps)
        agb = al * g * be
        bga = be * g * al
        eps_s += agb
        eps += agb + bga
        al = al * g * al
        be = be * g * be
        if _absmax(al) < tol and _absmax(be) < tol:
            return mpm.inverse(z * I - eps_s)
    raise RuntimeError("mp decimation did not converge")


def self_energies(N, E, eta, t=-2.7, dps=40):
    """Full-cell Sigma_L, Sigma_R (as complex128 arrays) from the decimation in dps digits."""
    with mpm.workdps(dps):
        tol = mpm.mpf(10) ** (-(dps - 5))
        H00n, H01n = blocks(N, t)
        H00, H01 = _m(H00n), _m(H01n)
        z = mpm.mpf(E) + 1j * mpm.mpf(eta)
        gR = _surface(H00, H01, H01.T, z, tol)
        gL = _surface(H00, H01.T, H01, z, tol)
        sR = H01 * gR * H01.T
        sL = H01.T * gL * H01
        conv = lambda m: np.array([[complex(m[i, j]) for j in range(m.cols)] for i in range(m.rows)])
        return conv(sL), conv(sR)


def transmission(N, L, E, eta_device, eta_lead, t=-2.7, eps=None, removed=None, dps=40):
    """T of Eq. 2 by the recursion of Eqs. 4-5 in dps digits."""
    with mpm.workdps(dps):
        tol = mpm.mpf(10) ** (-(dps - 5))
        H00n, H01n = blocks(N, t)
        H00, H01 = _m(H00n), _m(H01n)
        zl = mpm.mpf(E) + 1j * mpm.mpf(eta_lead)
        zd = mpm.mpf(E) + 1j * mpm.mpf(eta_device)
        gR = _surface(H00, H01, H01.T, zl, tol)
        gLs = _surface(H00, H01.T, H01, zl, tol)
        sigR_full = H01 * gR * H01.T
        sigL_full = H01.T * gLs * H01
        Hd, V, keep = device_slices(N, L, t, eps, removed)

        def sub(m, idx):
            return mpm.matrix([[m[int(i), int(j)] for j in idx] for i in idx])

        sigL = sub(sigL_full, keep[0])
        sigR = sub(sigR_full, keep[-1])
        g = P = None
        for j in range(L):
            K = len(keep[j])
            A = zd * mpm.eye(K) - _m(Hd[j])
            if j == 0:
                A -= sigL
            else:
                Vm = _m(V[j - 1])
                A -= Vm.T * g * Vm
            if j == L - 1:
                A -= sigR
            g = mpm.inverse(A)
            P = g if j == 0 else P * _m(V[j - 1]) * g
        gL = 1j * (sigL - sigL.H)
        gRb = 1j * (sigR - sigR.H)
        X = gL * P * gRb * P.H
        return float(mpm.re(sum(X[i, i] for i in range(X.rows))))
