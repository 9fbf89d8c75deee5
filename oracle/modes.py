"""Lead self-energies in the transverse-mode basis of the pristine armchair lead.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper includes the self-energies of the two semi-infinite leads at the
first and the last slice (text after Eqs. 4-5).  A pristine armchair lead
separates exactly into transverse modes.  With phi_p(j) = sin(p pi (j+1)/(N+1))
on the rows j = 0..N-1, the row-(j+-1) hopping maps phi_p on the even rows to
2 cos(p pi/(N+1)) phi_p on the odd rows, because phi_p(j-1) + phi_p(j+1) =
2 cos(p pi/(N+1)) phi_p(j) and phi_p(-1) = phi_p(N) = 0.  In the basis of the
normalised restricted vectors

    U_even[i, p-1] ~ phi_p(2i)      (i < ceil(N/2), the even-row atoms)
    U_odd [i, p-1] ~ phi_p(2i + 1)  (i < floor(N/2), the odd-row atoms)

each mode is a linear chain whose bonds alternate between t (two atoms of one
row) and tau_p = 2 t cos(p pi/(N+1)) (atoms of neighbouring rows).  Seen from
the device, the outermost lead atom of either lead (the odd-row right atom of
the left lead's last cell, the even-row left atom of the right lead's first
cell) starts its chain with a t bond, so both leads have the same surface
Green's function g_p, the fixed point of

    g = 1 / (z - t^2 / (z - tau^2 g)),   i.e.   tau^2 z g^2 - (z^2 + tau^2 - t^2) g + z = 0,

taken as the root with Im g < 0 (the other root is 1/(tau^2 g), whose
imaginary part has the opposite sign).  The device atoms bonded to the lead
feel Sigma = U diag(w) U^T with w_p = tau_p^2 g_p: on the even-row left atoms of
the first cell (Sigma_L, modes p = 1..ceil(N/2)) and on the odd-row right atoms
of the last cell (Sigma_R, p = 1..floor(N/2)); Gamma = U diag(-2 Im w) U^T.

This is the exact value that Sancho-Rubio decimation (``leads``) converges to,
reached by a closed form instead of an iteration.  Near E = 0 the modes with
|tau_p| > |t| carry a surface state of the zigzag-like transverse cut, and
w_p ~ 1/eta: the closed form keeps full relative accuracy there, where the
full-cell decimation in complex128 does not.
"""
from __future__ import annotations

import numpy as np


def mode_vectors(N: int):
    """(U_even [KL, KL], U_odd [KR, KR]): orthonormal restricted sine modes, columns
    p = 1..KL and p = 1..KR (KL = ceil(N/2), KR = floor(N/2))."""
    KL, KR = (N + 1) // 2, N // 2
    out = []
    for K, parity in ((KL, 0), (KR, 1)):
        i = np.arange(K)[:, None]
        p = np.arange(1, K + 1)[None, :]
        U = np.sin(np.pi * p * (2 * i + parity + 1) / (N + 1))
        U /= np.linalg.norm(U, axis=0, keepdims=True)
        out.append(U)
    return out[0], out[1]


def mode_hoppings(N: int, t: float = -2.7) -> np.ndarray:
    """tau_p = 2 t cos(p pi / (N+1)) for p = 1..ceil(N/2)."""
    KL = (N + 1) // 2
    return 2.0 * t * np.cos(np.pi * np.arange(1, KL + 1) / (N + 1))


def surface_green(z: complex, t: float, tau: float) -> complex:
    """Surface Green's function of the semi-infinite chain with bonds t, tau, t, tau, ...
    (on-site 0) at complex energy z with Im z > 0: the root of
    tau^2 z g^2 - (z^2 + tau^2 - t^2) g + z = 0 with Im g < 0."""
    if tau == 0.0:
        return 1.0 / (z - t * t / z)          # the chain ends after two atoms
    a = tau * tau * z
    b = -(z * z + (tau - t) * (tau + t))      # tau^2 - t^2 first: no cancellation against z^2
    c = z
    d = np.sqrt(b * b - 4.0 * a * c + 0j)
    # the root of larger magnitude without cancellation, the other by Vieta
    q = -0.5 * (b + d) if (np.conj(b) * d).real >= 0.0 else -0.5 * (b - d)
    g1, g2 = q / a, c / q
    return g1 if g1.imag < 0.0 else g2


def mode_self_energies(N: int, E: float, eta: float, t: float = -2.7) -> np.ndarray:
    """w_p = tau_p^2 g_p, p = 1..ceil(N/2) (the same for both leads)."""
    z = E + 1j * eta
    return np.array([tau * tau * surface_green(z, t, tau) for tau in mode_hoppings(N, t)])


def dyson_residual(N: int, E: float, eta: float, t: float = -2.7) -> float:
    """max_p |g_p - 1/(z - t^2/(z - tau_p^2 g_p))| / |g_p| of the closed-form roots."""
    z = E + 1j * eta
    r = 0.0
    for tau in mode_hoppings(N, t):
        g = surface_green(z, t, tau)
        rhs = 1.0 / (z - t * t / (z - tau * tau * g))
        r = max(r, abs(g - rhs) / abs(g))
    return r


def left_orbitals(N: int) -> np.ndarray:
    """Cell orbitals (2j + k order) of the even-row left atoms, the atoms Sigma_L acts on."""
    return np.array([4 * i for i in range((N + 1) // 2)])


def right_orbitals(N: int) -> np.ndarray:
    """Cell orbitals of the odd-row right atoms, the atoms Sigma_R acts on."""
    return np.array([4 * i + 3 for i in range(N // 2)])


def self_energies(N: int, E: float, eta: float, t: float = -2.7):
    """Full-cell (2N x 2N) Sigma_L, Sigma_R assembled from the modes."""
    UL, UR = mode_vectors(N)
    w = mode_self_energies(N, E, eta, t)
    KR = N // 2
    M = 2 * N
    sigL = np.zeros((M, M), dtype=np.complex128)
    sigR = np.zeros((M, M), dtype=np.complex128)
    iL, iR = left_orbitals(N), right_orbitals(N)
    sigL[np.ix_(iL, iL)] = UL @ np.diag(w) @ UL.T
    sigR[np.ix_(iR, iR)] = UR @ np.diag(w[:KR]) @ UR.T
    return sigL, sigR
