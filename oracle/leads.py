"""Semi-infinite lead self-energies by Lopez Sancho-Rubio decimation.

The paper includes lead self-energies at the first and the last slice and
computes them from an eigenproblem on the CPU (text after Eqs. 4-5; step list
items 1-2).  The workloads fix decimation instead (M. P. Lopez Sancho, J. M.
Lopez Sancho, J. Rubio, J. Phys. F 15 (1985) 851).  Written here on whole
unit-cell blocks, as the method states it:

    init  eps_s = eps = H00, alpha = alpha0, beta = beta0
    loop  g = (z - eps)^-1
          eps_s += alpha g beta
          eps   += alpha g beta + beta g alpha
          alpha  = alpha g alpha
          beta   = beta  g beta
    until max|alpha|, max|beta| < tol
    surface Green's function g_s = (z - eps_s)^-1

Right lead (cells L+1, L+2, ... to the right of the device): alpha0 = H01,
beta0 = H01^T, and Sigma_R = H01 g_s H01^T acts on the last device slice.
Left lead (cells ..., -1, 0 to the left): alpha0 = H01^T, beta0 = H01, and
Sigma_L = H01^T g_s H01 acts on the first device slice.  Leads are pristine
(on-site 0).  z = E + i eta.
"""
from __future__ import annotations

import numpy as np

from .lattice import blocks


class NoConvergence(RuntimeError):
    pass


def surface_green(H00, alpha0, beta0, z, tol=1e-14, max_iter=200):
    """Sancho-Rubio surface Green's function. Returns (g_s, iterations). (The lead self-energies
    entering at the first and last slice, text after Eqs. 4-5.)"""
    M = H00.shape[0]
    I = np.eye(M)
    eps_s = H00.astype(np.complex128).copy()
    eps = H00.astype(np.complex128).copy()
    alpha = alpha0.astype(np.complex128).copy()
    beta = beta0.astype(np.complex128).copy()
    for it in range(1, max_iter + 1):
        g = np.linalg.inv(z * I - eps)
        agb = alpha @ g @ beta
        bga = beta @ g @ alpha
        eps_s = eps_s + agb
        eps = eps + agb + bga
        alpha = alpha @ g @ alpha
        beta = beta @ g @ beta
        if np.max(np.abs(alpha)) < tol and np.max(np.abs(beta)) < tol:
            return np.linalg.inv(z * I - eps_s), it
    raise NoConvergence(f"Sancho-Rubio did not converge in {max_iter} iterations (z={z})")


def fixed_point_residual(g_s, H00, alpha0, beta0, z):
    """Relative residual of the surface Dyson equation g = (z - H00 - alpha0 g beta0)^-1."""
    M = H00.shape[0]
    rhs = np.linalg.inv(z * np.eye(M) - H00 - alpha0 @ g_s @ beta0)
    return np.max(np.abs(g_s - rhs)) / np.max(np.abs(g_s))


def self_energies(N, E, eta, t=-2.7, tol=1e-14, max_iter=200, return_iters=False):
    """Full-cell (2N x 2N) Sigma_L and Sigma_R of pristine semi-infinite leads. (Text after Eqs.
    4-5.)"""
    H00, H01 = blocks(N, t)
    z = E + 1j * eta
    gR, itR = surface_green(H00, H01, H01.T, z, tol, max_iter)
    gL, itL = surface_green(H00, H01.T, H01, z, tol, max_iter)
    sigR = H01 @ gR @ H01.T
    sigL = H01.T @ gL @ H01
    if return_iters:
        return sigL, sigR, itL, itR
    return sigL, sigR


def broadening(sigma):
    """Gamma = i (Sigma - Sigma^dagger). (Eq. 2.)"""
    return 1j * (sigma - sigma.conj().T)
