"""Sum-over-poles ("fully analytical") route to W^c and Sigma^c (test infrastructure).

THIS MODULE IS TEST INFRASTRUCTURE (same rule as gwc_oracle: only tests/, smoke()
and bench.py's CPU legs may use it). It is the independent route that pins the
contour-deformation oracle: it never forms Pi(z) or solves with eps(z).

Paper, Sec. "G0W0 approximation":
  * RPA excitations from the non-Hermitian Casida problem [[A, B], [-B, -A]] (X, Y) =
    Omega (X, Y) (Eq. rpa_casida) with A, B built from (ia|jb) (Eq. rpa_matrices);
  * transition moments rho^nu_mn = sum_ia (mn|ia)(X^nu + Y^nu)_ia (Eq. density_shifts);
  * W^c_mn(w) = sum_nu rho rho [1/(w - Omega + i eta) - 1/(w + Omega - i eta)] (Eq. W_spectral);
  * Sigma^c_n(w) = sum_{m,nu} rho^2 / (w - eps_m + (Omega - i eta) sgn(eps_F - eps_m)) (Eq. sigma_spectral).

Closed-shell singlet spin adaptation (the paper writes the spin-orbital form):
A = diag(Delta) + 2K, B = 2K with K_{ia,jb} = (ia|jb) = sum_P O^P_ia O^P_jb, and
rho^nu_mn = sqrt(2) sum_ia (mn|ia)(X+Y)^nu_ia with X^T X - Y^T Y = 1.
"""
from __future__ import annotations

import math

import numpy as np


def casida_sop(o_ov: np.ndarray, delta: np.ndarray):
    """Solve the full 2N x 2N Casida problem with a general eigensolver.

    Returns (Omega [N] ascending, XpY [N_ov][N]) normalised so that X^T X - Y^T Y = 1.
    Only for small N_ov (the matrix is built explicitly).
    """
    k = o_ov.T @ o_ov  # (ia|jb)
    a = np.diag(delta) + 2.0 * k
    b = 2.0 * k
    big = np.block([[a, b], [-b, -a]])
    vals, vecs = np.linalg.eig(big)
    vals = vals.real
    n = delta.size
    pos = np.argsort(vals)[n:]  # the N positive excitation energies
    om = vals[pos]
    x = vecs[:n, pos].real
    y = vecs[n:, pos].real
    norm = np.einsum("in,in->n", x, x) - np.einsum("in,in->n", y, y)
    s = 1.0 / np.sqrt(norm)
    return om, (x + y) * s[None, :]


def transition_moments(o_ov: np.ndarray, xpy: np.ndarray, o_vec: np.ndarray) -> np.ndarray:
    """rho^nu for one orbital pair mn with RI vector o_vec = O^.(m,n): sqrt(2) (mn|ia)(X+Y)."""
    return math.sqrt(2.0) * ((o_vec @ o_ov) @ xpy)


def w_sop(rho: np.ndarray, omega: np.ndarray, z: complex, eta_sign: bool = False, eta: float = 0.0) -> complex:
    """W^c(z) = sum_nu rho^2 [1/(z - Omega) - 1/(z + Omega)] evaluated at complex z.

    With eta_sign=True the time-ordered form of Eq. W_spectral is used at real z:
    rho^2 [1/(z - Omega + i eta) - 1/(z + Omega - i eta)].
    """
    if eta_sign:
        return complex(np.sum(rho**2 * (1.0 / (z - omega + 1j * eta) - 1.0 / (z + omega - 1j * eta))))
    return complex(np.sum(rho**2 * (1.0 / (z - omega) - 1.0 / (z + omega))))


def sigma_c_sop(eps, eps_f, rho_by_m, omega_nu, w, eta):
    """Eq. sigma_spectral for one state n: sum_{m,nu} rho_mn^2/(w - eps_m + (Omega - i eta) sgn(eps_F - eps_m)).

    rho_by_m: [n_states][N] transition moments rho^nu_{m n}.
    """
    tot = 0.0 + 0.0j
    for m in range(eps.size):
        sg = 1.0 if eps_f > eps[m] else -1.0
        tot += np.sum(rho_by_m[m] ** 2 / (w - eps[m] + (omega_nu - 1j * eta) * sg))
    return complex(tot)


def sigma_c_cd_closed_form(eps, eps_f, rho_by_m, omega_nu, w, eta):
    """The contour-deformation expression -I + R evaluated with the SOP W^c in closed form.

    With W^c(i xi) = -sum rho^2 2 Omega/(xi^2 + Omega^2) the imaginary-axis integral of
    Eq. cd_imaginary is exact: (1/pi) int_0^inf a/(a^2+xi^2) W^c(i xi) dxi =
    -sum_nu rho^2 sgn(a)/(|a| + Omega). The residue term uses W^c(|eps_m - w| + i eta) with the
    same analytic W^c. This differs from the CD oracle only by its quadrature error.
    """
    tot = 0.0 + 0.0j
    for m in range(eps.size):
        a = w - eps[m]
        r2 = rho_by_m[m] ** 2
        if a != 0.0:
            tot -= -np.sum(r2 * math.copysign(1.0, a) / (abs(a) + omega_nu))
        f = _prefactor(eps[m], w, eps_f)
        if f != 0.0:
            z = abs(eps[m] - w) + 1j * eta
            tot += f * np.sum(r2 * (1.0 / (z - omega_nu) - 1.0 / (z + omega_nu)))
    return complex(tot)


def _prefactor(eps_m, w, eps_f):
    def th(x):
        return 1.0 if x > 0 else (0.0 if x < 0 else 0.5)

    return -th(eps_f - eps_m) * th(eps_m - w) + th(eps_m - eps_f) * th(w - eps_m)
