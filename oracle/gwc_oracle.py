"""Plain FP64 CPU oracle for the G_dH W0 + cumulant hot path (test infrastructure).

THIS MODULE IS TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import it. The product library
never calls it, and it shares no code with the CUDA path (it imports numpy and
nothing of the package).

It follows the paper (arXiv 2412.17132, "GW plus cumulant approach for predicting
core-level shake-up satellites in large molecules") step by step, in its order
and notation, with numpy primitives (matmul, LU solve, FFT) as single steps.
Units are Hartree atomic units throughout.

Readings taken where the paper is silent (all listed in the design notes):
  * RI form of the polarizability (the paper only says its CD is RI based, Sec.
    "Self-energy evaluation"): Pi(z) = O diag(D(z)) O^T over occupied-virtual
    pairs, D_ia(z) = 2[1/(z - Delta_ia) - 1/(z + Delta_ia)] = 4 Delta/(z^2 - Delta^2)
    (closed shell, spin factor 2), eps(z) = 1 - Pi(z), and
    W^c_mn(z) = o_mn^T (eps(z)^-1 - 1) o_mn with o_mn = O^.(m,n).
  * eta enters the residue term as the analytic W^c evaluated at |eps_m - w| + i eta.
  * Theta(0) = 1/2 in the prefactors f_m; eps_F = midpoint of HOMO and LUMO.
  * Sigma^x runs over occupied m only.
  * The imaginary-axis integral uses a modified Gauss-Legendre grid
    xi = xi0 (1+x)/(1-x) with analytic subtraction of W^c(i0).
  * The G_dH W0 quasiparticle equation is solved by the secant method from eps_n; so is the
    plain G0W0 equation, whose several solutions are also listed by a sign-change scan of the
    equation on a frequency grid (linear interpolation, Z from the local slope).
  * v^xc defaults to Sigma^x (zero static shift) when not given.
"""
from __future__ import annotations

import copy
import math

import numpy as np

# ----------------------------------------------------------------------------------------
# Basic quantities
# ----------------------------------------------------------------------------------------


def fermi_level(eps: np.ndarray, n_occ: int) -> float:
    """eps_F: midpoint of HOMO and LUMO (the paper leaves it undefined, Sec. "G0W0 approximation")."""
    return 0.5 * (float(eps[n_occ - 1]) + float(eps[n_occ]))


def transition_energies(eps: np.ndarray, n_occ: int) -> np.ndarray:
    """Delta_ia = eps_a - eps_i, flattened i-major (the index order of O_ov)."""
    return (eps[None, n_occ:] - eps[:n_occ, None]).reshape(-1)


def d_factor(delta: np.ndarray, z: complex) -> np.ndarray:
    """Independent-particle response of one pair, spin-summed: 2[1/(z-Delta) - 1/(z+Delta)]."""
    z = complex(z)
    return 2.0 * (1.0 / (z - delta) - 1.0 / (z + delta))


def chi0(o_ov: np.ndarray, delta: np.ndarray, z: complex) -> np.ndarray:
    """RI polarizability Pi_PQ(z) = sum_ia O^P_ia D_ia(z) O^Q_ia (complex128 [n_aux][n_aux]).

    Built twice as a plain sum of two real products so that the imaginary axis
    (where D is real) gives an exactly real matrix.
    """
    d = d_factor(delta, z)
    re = (o_ov * d.real[None, :]) @ o_ov.T
    im = (o_ov * d.imag[None, :]) @ o_ov.T
    return re + 1j * im


def screened_wc(pi: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """W^c = b^T (eps^-1 - 1) b for each column b of rhs [n_aux][k]; eps = 1 - Pi (LU solve)."""
    n = pi.shape[0]
    eps_m = np.eye(n) - pi
    x = np.linalg.solve(eps_m, rhs.astype(eps_m.dtype))
    return np.einsum("pk,pk->k", rhs, x) - np.einsum("pk,pk->k", rhs, rhs)


# ----------------------------------------------------------------------------------------
# Frequency grids
# ----------------------------------------------------------------------------------------


def modified_gl_grid(n: int, xi0: float = 1.0):
    """Imaginary-axis nodes/weights: Gauss-Legendre on (-1,1) mapped by xi = xi0 (1+x)/(1-x).

    The paper uses a "modified Gauss-Legendre grid" with 200 points (Sec.
    "Computational Details") without giving the map; this rational map of (-1,1)
    onto (0, inf) is the reading used here. Weights: w = 2 xi0 w_GL / (1-x)^2.
    """
    x, w = np.polynomial.legendre.leggauss(n)
    xi = xi0 * (1.0 + x) / (1.0 - x)
    wt = 2.0 * xi0 * w / (1.0 - x) ** 2
    return xi, wt


def trapezoid_weights(omega: np.ndarray) -> np.ndarray:
    """Trapezoid weights of a (possibly non-uniform) ascending grid."""
    w = np.zeros_like(omega)
    if omega.size > 1:
        d = np.diff(omega)
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
    return w


# ----------------------------------------------------------------------------------------
# Self-energy by contour deformation (Sec. "Self-energy evaluation", Eqs. cd_terms,
# cd_imaginary, cd_residue, cd_prefactors)
# ----------------------------------------------------------------------------------------


def heaviside(x: float) -> float:
    """Theta with Theta(0) = 1/2."""
    return 1.0 if x > 0 else (0.0 if x < 0 else 0.5)


def residue_prefactor(eps_m: float, omega: float, eps_f: float) -> float:
    """f_m = -Theta(eps_F - eps_m) Theta(eps_m - w) + Theta(eps_m - eps_F) Theta(w - eps_m) (Eq. cd_prefactors)."""
    return -heaviside(eps_f - eps_m) * heaviside(eps_m - omega) + heaviside(eps_m - eps_f) * heaviside(omega - eps_m)


class System:
    """Inputs of one calculation (same layout as the library): see the synthetic generator."""

    def __init__(self, eps, n_occ, core_idx, o_ov, o_core, eta, n_im=32, xi0=1.0, vxc=None, eps_f=None):
        self.eps = np.asarray(eps, dtype=np.float64)
        self.n_occ = int(n_occ)
        self.core_idx = np.asarray(core_idx, dtype=np.int64)
        self.o_ov = np.asarray(o_ov, dtype=np.float64)
        self.o_core = np.asarray(o_core, dtype=np.float64)
        self.eta = float(eta)
        self.n_im = int(n_im)
        self.xi0 = float(xi0)
        self.vxc = None if vxc is None else np.asarray(vxc, dtype=np.float64)
        self.eps_f = fermi_level(self.eps, self.n_occ) if eps_f is None else float(eps_f)
        # orbital energies in G (the poles of the Green's function); the input energies unless an
        # eigenvalue-self-consistent scheme replaces them (see evgw0). W always uses self.eps.
        self.eps_g = self.eps
        self.delta = transition_energies(self.eps, self.n_occ)
        self.xi, self.w_xi = modified_gl_grid(self.n_im, self.xi0)
        self._w_im = None

    @classmethod
    def from_molecule(cls, mol, **kw):
        args = dict(n_im=mol.n_im, xi0=mol.xi0)
        args.update(kw)
        return cls(mol.eps, mol.n_occ, mol.core_idx, mol.o_ov, mol.o_core, mol.eta, **args)

    @property
    def n_states(self):
        return self.eps.shape[0]

    @property
    def n_core(self):
        return self.core_idx.shape[0]

    # -- W^c on the imaginary axis: all states m, all cores n ---------------------------
    def w_imag_table(self):
        """W^c_mn(i xi_k) for k = 0..n_im-1 and W^c_mn(i0): arrays [n_im][n_states][n_core], [n_states][n_core]."""
        if self._w_im is None:
            rhs = self.o_core.reshape(self.n_states * self.n_core, -1).T  # [n_aux][m*n_core + c]
            tab = np.empty((self.n_im, self.n_states, self.n_core))
            for k, xi in enumerate(self.xi):
                w = screened_wc(chi0(self.o_ov, self.delta, 1j * xi).real, rhs)
                tab[k] = w.reshape(self.n_states, self.n_core)
            w0 = screened_wc(chi0(self.o_ov, self.delta, 0.0).real, rhs).reshape(self.n_states, self.n_core)
            self._w_im = (tab, w0)
        return self._w_im

    def w_residue(self, m: int, x: float) -> np.ndarray:
        """W^c_{m,n}(x + i eta) for every core n (one dielectric solve, n_core right-hand sides)."""
        pi = chi0(self.o_ov, self.delta, complex(x, self.eta))
        return screened_wc(pi, self.o_core[m].T)  # rhs columns: O^.(m, n) for each core n

    # -- Imaginary-axis term I_n(w) (Eq. cd_imaginary) ---------------------------------
    def imag_axis_term(self, omega: float) -> np.ndarray:
        """I_n(w) for every core n.

        I_n(w) = (1/pi) sum_m int_0^inf dxi a_m/(a_m^2 + xi^2) W^c_mn(i xi), a_m = w - eps_m
        (Eq. cd_imaginary with the odd part of the integrand dropped since W^c(i xi) is even in
        xi and real), evaluated as quadrature of [W(i xi) - W(i0)] plus the exact integral
        (1/2) sgn(a) W(i0) of the subtracted part; the term is 0 at a = 0.
        """
        tab, w0 = self.w_imag_table()
        out = np.zeros(self.n_core)
        for m in range(self.n_states):
            a = omega - self.eps_g[m]
            if a == 0.0:
                continue
            kern = self.w_xi * a / (a * a + self.xi**2) / math.pi  # [n_im]
            out += kern @ (tab[:, m, :] - w0[m][None, :]) + 0.5 * math.copysign(1.0, a) * w0[m]
        return out

    # -- Residue term R_n(w) (Eq. cd_residue) ---------------------------------------------
    def residue_term(self, omega: float):
        """R_n(w) = sum_m f_m W^c_mn(|eps_m - w| + i eta) for every core n; also returns the
        per-m contributions so that decoupled forms can be read off."""
        out = np.zeros(self.n_core, dtype=np.complex128)
        per_m = {}
        for m in range(self.n_states):
            f = residue_prefactor(self.eps_g[m], omega, self.eps_f)
            if f == 0.0:
                continue
            w = self.w_residue(m, abs(self.eps_g[m] - omega))
            per_m[m] = (f, w)
            out += f * w
        return out, per_m

    # -- Sigma^c (Eq. cd_terms) -------------------------------------------------------------
    def sigma_c(self, omega: float):
        """Sigma^c_n(w) = -I_n(w) + R_n(w) (G0W0, CD) for every core n, plus the decoupled
        Im Sigma of Eq. cd_sigma_imaginary_decoupled: f_n Im W^c_nn(|eps_n - w| + i eta)."""
        r, per_m = self.residue_term(omega)
        sig = -self.imag_axis_term(omega) + r
        dec = np.zeros(self.n_core)
        for c, n in enumerate(self.core_idx):
            if int(n) in per_m:
                f, w = per_m[int(n)]
                dec[c] = f * w[c].imag
        return sig, dec

    def im_sigma_dec_group(self, omega: float, groups, cores=None) -> np.ndarray:
        """Decoupled Im Sigma with symmetry-equivalent cores (Sec. "Core-valence decoupling", Eq.
        sigma_spectral_decoupled_symmetric, in the residue form of Eq. cd_sigma_imaginary_decoupled):
        for core n the sum over the cores i of its group (groups[c] is the label of core c),
            Im Sigma^dec_n(w) = sum_{i in group(n)} f_i Im W^c_{i n}(|eps_i - w| + i eta),
        each member with its own prefactor f_i, its own residue frequency |eps_i - w| and the RI vector
        o_{in} = O^.(i, n) (one solve per member). A group of one member is the DIAG form. Returns [n_core];
        with `cores` (core indices) given, only those entries are computed and the others are 0."""
        groups = [int(g) for g in groups]
        out = np.zeros(self.n_core)
        todo = range(self.n_core) if cores is None else [int(c) for c in cores]
        for c in todo:
            for c2, i in enumerate(self.core_idx):
                if groups[c2] != groups[c]:
                    continue
                f = residue_prefactor(self.eps_g[i], omega, self.eps_f)
                if f == 0.0:
                    continue
                pi = chi0(self.o_ov, self.delta, complex(abs(self.eps_g[i] - omega), self.eta))
                w = screened_wc(pi, self.o_core[int(i), c][:, None])[0]
                out[c] += f * w.imag
        return out

    def sigma_c_grid(self, omegas: np.ndarray):
        """Sigma^c on a common absolute grid: complex [n_core][n_w] and decoupled Im [n_core][n_w]."""
        s = np.empty((self.n_core, omegas.size), dtype=np.complex128)
        d = np.empty((self.n_core, omegas.size))
        for j, w in enumerate(omegas):
            s[:, j], d[:, j] = self.sigma_c(float(w))
        return s, d

    def sigma_c_core(self, c: int, omega: float) -> complex:
        """Sigma^c of core c alone at w (the same formulas, one core's right-hand sides)."""
        return complex(self.sigma_c(omega)[0][c])

    def with_g_energies(self, eps_g, eps_f=None):
        """The same system with the orbital energies in G replaced by eps_g (W, the exchange and
        the RI data unchanged; the imaginary-axis W table is shared). eps_f: the Fermi level used in
        the residue prefactors, default the midpoint of the HOMO and LUMO of eps_g."""
        other = copy.copy(self)
        other.eps_g = np.asarray(eps_g, dtype=np.float64)
        other.eps_f = fermi_level(other.eps_g, self.n_occ) if eps_f is None else float(eps_f)
        self.w_imag_table()
        other._w_im = self._w_im
        return other

    # -- Exchange (Eq. sigma_x) -----------------------------------------------------------------
    def sigma_x(self) -> np.ndarray:
        """Sigma^x_n = -sum_{i occ} (n i | i n) = -sum_{i occ} sum_P (O^P_{n i})^2."""
        return -np.einsum("icp,icp->c", self.o_core[: self.n_occ], self.o_core[: self.n_occ])

    def v_xc(self) -> np.ndarray:
        return self.sigma_x() if self.vxc is None else self.vxc

    # -- Hedin shift and QP equation (Eqs. hedin_shift, hedin_sigma_spectral,
    #    quasiparticle_equation, QPGWC) ------------------------------------------------------
    def hedin_shift(self) -> np.ndarray:
        """dH_n = Re Sigma^c_n(eps_n) + Sigma^x_n - v^xc_n, evaluated core by core."""
        sx, vxc = self.sigma_x(), self.v_xc()
        out = np.empty(self.n_core)
        for c, n in enumerate(self.core_idx):
            out[c] = self.sigma_c_core(c, float(self.eps[n])).real + sx[c] - vxc[c]
        return out

    def qp_solve(self, tol=1e-7, max_iter=50, cores=None, mode="gdh"):
        """Solve eps = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n(eps - dH_n) by the secant method
        from eps_n (G_dH W0 QP equation). Returns (eps_qp, dH, iterations); with `cores` given
        only those cores are solved (the other entries are NaN / 0).

        mode "g0w0": the plain G0W0 QP equation of Eq. quasiparticle_equation, Sigma^c evaluated at
        eps itself (no shift); the same secant from eps_n, dH still reported."""
        sx, vxc = self.sigma_x(), self.v_xc()
        todo = range(self.n_core) if cores is None else list(cores)
        dh = np.full(self.n_core, np.nan)
        for c in todo:
            n = self.core_idx[c]
            dh[c] = self.sigma_c_core(c, float(self.eps[n])).real + sx[c] - vxc[c]
        eqp = np.full(self.n_core, np.nan)
        iters = np.zeros(self.n_core, dtype=np.int64)
        for c in todo:
            n = self.core_idx[c]
            e_n = float(self.eps[n])

            shift = 0.0 if mode == "g0w0" else dh[c]

            def g(e):
                return e_n + sx[c] - vxc[c] + self.sigma_c_core(c, e - shift).real - e

            x0 = e_n
            g0 = g(x0)
            x1 = x0 + g0
            it = 1
            while True:
                g1 = g(x1)
                it += 1
                if abs(g1) < tol or it >= max_iter:
                    break
                denom = g1 - g0
                x2 = x1 + g1 if denom == 0.0 else x1 - g1 * (x1 - x0) / denom
                x0, g0, x1 = x1, g1, x2
                if abs(x1 - x0) < tol:
                    g1 = g(x1)
                    it += 1
                    break
            eqp[c] = x1
            iters[c] = it
        return eqp, dh, iters


class NotConverged(RuntimeError):
    """An iteration stopped without meeting its tolerance (evgw0 with on_fail="raise")."""


def evgw0(system: "System", tol: float = 1e-8, max_iter: int = 100, on_fail: str = "return"):
    """Eigenvalue self-consistency in G with W fixed (evGW0; Sec. "GW for core-levels: beyond
    G0W0", Eq. ev_sigma_spectral): the orbital energies in G are replaced by the current QP
    energies of EVERY state while W keeps the RPA excitations of the input energies, so the
    system must list every state in core_idx (in state order) with o_core = O^P_{m,n} for all n.

    Reading of the iteration (the paper gives the scheme, not the update rule): starting from the
    input energies eps^(0) = eps, every state is updated at once,
        eps^(k+1)_n = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n[G(eps^(k))](eps^(k)_n),
    so that the first step is eps_n + dH_n (the Hedin shift of Eq. hedin_shift is the first
    iteration of evGW0), with eps_F the midpoint of the current QP HOMO and LUMO, until
    max_n |eps^(k+1)_n - eps^(k)_n| < tol. The scheme stops without converging when max_iter steps
    do not reach tol, or when an iterate moves a state across eps_F (an occupied QP energy at or above
    the midpoint of the QP HOMO and LUMO, or a virtual one below it: the occupations of G would no
    longer be the input's). Returns (eps_qp [n_states], iterations); on a stop without convergence it
    returns the last iterate and max_iter (or the steps done before the crossing), or raises
    NotConverged with on_fail="raise"."""
    n = system.n_states
    if system.n_core != n or np.any(system.core_idx != np.arange(n)):
        raise ValueError("evgw0 needs every state as a core (core_idx = 0..n_states-1)")
    sx, vxc = system.sigma_x(), system.v_xc()
    e = system.eps.copy()
    for it in range(1, max_iter + 1):
        ef = fermi_level(e, system.n_occ)
        if np.any(e[: system.n_occ] >= ef) or np.any(e[system.n_occ :] < ef):
            if on_fail == "raise":
                raise NotConverged(f"evGW0: QP energies crossed eps_F at iteration {it}")
            return e, it - 1
        s = system.with_g_energies(e)
        new = np.array([system.eps[c] + sx[c] - vxc[c] + s.sigma_c(float(e[c]))[0][c].real for c in range(n)])
        done = np.max(np.abs(new - e)) < tol
        e = new
        if done:
            return e, it
    if on_fail == "raise":
        raise NotConverged(f"evGW0 did not reach tol {tol} in {max_iter} steps")
    return e, max_iter


def g0w0_graphical_solutions(omega: np.ndarray, sigma_c: np.ndarray, eps_n: float, sigma_x: float, vxc: float):
    """All solutions of the plain G0W0 QP equation (Eq. quasiparticle_equation) on a grid — the
    "graphical solution" of Sec. "Satellites in the G0W0 approximation", which for core levels has
    several roots. With f(w) = eps_n + Sigma^x - v^xc + Re Sigma^c(w) - w on the ascending grid
    omega (sigma_c complex on the same grid): a grid point with f = 0 is a root; between points j
    and j+1 with f_j f_{j+1} < 0 the root is the linear interpolant
        w* = w_j - f_j (w_{j+1} - w_j) / (f_{j+1} - f_j),
    and its renormalisation factor is Z = 1 / (1 - dRe Sigma/dw) with the slope of Re Sigma^c over
    that interval (at a grid root: over the interval to its right, or to its left at the end).
    Returns a list of (w*, Z) in ascending w*."""
    w = np.asarray(omega, dtype=np.float64)
    rs = np.asarray(sigma_c).real.astype(np.float64)
    f = eps_n + sigma_x - vxc + rs - w
    out = []
    n = w.size
    for j in range(n):
        if f[j] == 0.0:
            k = j if j + 1 < n else j - 1
            slope = (rs[k + 1] - rs[k]) / (w[k + 1] - w[k])
            out.append((float(w[j]), float(1.0 / (1.0 - slope))))
        elif j + 1 < n and f[j] * f[j + 1] < 0.0:
            ws = w[j] - f[j] * (w[j + 1] - w[j]) / (f[j + 1] - f[j])
            slope = (rs[j + 1] - rs[j]) / (w[j + 1] - w[j])
            out.append((float(ws), float(1.0 / (1.0 - slope))))
    return out


# ----------------------------------------------------------------------------------------
# CD-WAC: W^c_mn(w) by analytic continuation (Sec. "Self-energy evaluation", Eq. pade_approximation)
# ----------------------------------------------------------------------------------------


def thiele_coefficients(zref: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Coefficients of the continued fraction C(z) = a_0/(1 + a_1(z - z_0)/(1 + a_2(z - z_1)/(1 + ...)))
    through the points (z_i, u_i) (Eq. pade_approximation; Thiele's interpolation, recursion of
    Vidberg and Serene, J. Low Temp. Phys. 29, 179 (1977)):
    g_0(z_i) = u_i,  g_p(z_i) = [g_{p-1}(z_{p-1}) - g_{p-1}(z_i)] / [(z_i - z_{p-1}) g_{p-1}(z_i)],  a_p = g_p(z_p)."""
    g = np.array(u, dtype=np.complex128)
    z = np.asarray(zref, dtype=np.complex128)
    a = np.empty(g.size, dtype=np.complex128)
    a[0] = g[0]
    for p in range(1, g.size):
        g[p:] = (g[p - 1] - g[p:]) / ((z[p:] - z[p - 1]) * g[p:])
        a[p] = g[p]
    return a


def thiele_eval(a: np.ndarray, zref: np.ndarray, z) -> np.ndarray:
    """C(z) of thiele_coefficients, evaluated from the innermost level outwards."""
    z = np.asarray(z, dtype=np.complex128)
    t = np.ones_like(z)
    for p in range(a.size - 1, 0, -1):
        t = 1.0 + a[p] * (z - zref[p - 1]) / t
    return a[0] / t


def wac_reference_points(eps, n_occ, core_idx, omegas, eps_f, n_core_ref=100, n_val_ref=100, wc_max_ev=40.0,
                         d_lower=0.08, d_upper=0.01):
    """Real reference frequencies x (W is sampled at x + i eta).

    Reading of the paper's parameters (Sec. "Computational Details": N_C = N_V = 100 points,
    w_C in [0, 40] eV for the core region, Delta_lower = 8 %, Delta_upper = 1 % for the valence
    region): N_C points uniform on [0, w_C^max]; N_V points uniform on [x_lo (1 - Delta_lower),
    x_hi (1 + Delta_upper)], where x_lo, x_hi bound |eps_m - w| over the non-core occupied states m
    with a nonzero residue prefactor on the requested frequencies.
    """
    cores = set(int(c) for c in core_idx)
    xs = [abs(eps[m] - w) for w in omegas for m in range(n_occ)
          if m not in cores and residue_prefactor(eps[m], w, eps_f) != 0.0]
    core_pts = np.linspace(0.0, wc_max_ev / 27.211386245988, n_core_ref)
    if not xs:
        return core_pts
    lo, hi = min(xs) * (1.0 - d_lower), max(xs) * (1.0 + d_upper)
    return np.concatenate([core_pts, np.linspace(lo, hi, n_val_ref)])


def sigma_c_wac(system, omegas, xref):
    """Sigma^c_n(w) = -I_n(w) + R_n(w) with R from the continued-fraction W^c_mn.

    Reference values: W^c_mn(i xi_k) (the imaginary-axis quadrature nodes and i0, real) and
    W^c_mn(x_l + i eta) at the real reference points; one fit per (occupied m, core n).
    Returns complex [n_core][n_w]."""
    s = system
    tab, w0 = s.w_imag_table()
    zim = np.concatenate([1j * s.xi, [0.0]])
    zre = xref + 1j * s.eta
    # W at the real references for every occupied m and core n: one build per reference frequency
    wre = np.empty((xref.size, s.n_occ, s.n_core), dtype=np.complex128)
    rhs = s.o_core[: s.n_occ].reshape(s.n_occ * s.n_core, -1).T
    for l, z in enumerate(zre):
        wre[l] = screened_wc(chi0(s.o_ov, s.delta, z), rhs).reshape(s.n_occ, s.n_core)
    zref = np.concatenate([zim, zre])
    coef = {}
    for m in range(s.n_occ):
        for c in range(s.n_core):
            u = np.concatenate([tab[:, m, c], [w0[m, c]], wre[:, m, c]])
            coef[(m, c)] = thiele_coefficients(zref, u)
    out = np.empty((s.n_core, len(omegas)), dtype=np.complex128)
    for j, w in enumerate(omegas):
        i_term = s.imag_axis_term(float(w))
        for c in range(s.n_core):
            r = 0.0 + 0.0j
            for m in range(s.n_states):
                f = residue_prefactor(s.eps[m], float(w), s.eps_f)
                if f == 0.0:
                    continue
                if m >= s.n_occ:
                    raise ValueError("CD-WAC here covers frequencies below the LUMO (occupied residues only)")
                r += f * thiele_eval(coef[(m, c)], zref, abs(s.eps[m] - w) + 1j * s.eta)
            out[c, j] = -i_term[c] + r
    return out


# ----------------------------------------------------------------------------------------
# G_dH W0 spectral function (Sec. "G0W0 approximation": Eqs. g_dyson, gw_full_propagator,
# A_definition, A_explicit_real_imaginary, with the shifted self-energy of Eq. hedin_sigma_spectral)
# ----------------------------------------------------------------------------------------


def gdh_spectrum(omega_common, sigma_c, eps_n, dh, sigma_x, vxc):
    """A^{G_dH W0}_n on the shifted grid w = w' + dH_n, from Sigma^c_n(w') on a common grid w'.

    G_n(w) = [w - eps_n + v^xc_n - Sigma^x_n - Sigma^c_n(w - dH_n)]^-1 and
    A_n(w) = (1/pi) |Im Sigma| / ([w - eps_n + v^xc_n - Re Sigma]^2 + [Im Sigma]^2).
    Returns (w [n_w], A [n_w]).
    """
    w = omega_common + dh
    re = w - eps_n + vxc - sigma_x - sigma_c.real
    im = sigma_c.imag
    return w, np.abs(im) / (re * re + im * im) / math.pi


# ----------------------------------------------------------------------------------------
# Cumulant and spectral function (Sec. "Numerical GW+C scheme": Eqs. landau_cumulant_truncated,
# cumulant_propagator_numerical_time, cumulant_propagator_convolution,
# cumulant_propagator_fourier, eq:AGWC)
# ----------------------------------------------------------------------------------------


def cumulant_ct(omega_rel: np.ndarray, beta: np.ndarray, t: np.ndarray) -> np.ndarray:
    """C~(t) = int dw beta(w)/w^2 (e^{-i w t} - 1), beta = |Im Sigma(w + eps_n)|/pi,
    by the trapezoid rule on the given relative grid; a node at w = 0 is skipped
    (its integrand has the finite limit -i t beta(0)/0 -> beta vanishes there)."""
    wq = trapezoid_weights(omega_rel)
    keep = omega_rel != 0.0
    c = (wq * beta)[keep] / omega_rel[keep] ** 2
    ph = np.exp(-1j * np.outer(t, omega_rel[keep]))
    return (ph - 1.0) @ c


def spectrum_from_cumulant(ct: np.ndarray, dt: float, eta: float, direct: bool = False):
    """A(w) on FFT bins from e^{C~(t)} (retarded, Eq. eq:AGWC).

    G^C(t) = -i Theta(t) e^{-i eps^QP t - eta t} e^{C~(t)}, so
    A(eps^QP + nu) = (1/pi) Re int_0^T e^{i nu t - eta t} e^{C~(t)} dt, discretised with
    t_k = k dt, weights 1/2 at k = 0 and 1 elsewhere, nu_j = 2 pi j/(n dt) (j wrapped to
    -n/2..n/2-1). One damped transform gives the paper's FFT followed by convolution
    with G^QP (convolution theorem). Returns (nu [n], A [n]) with nu ascending.
    """
    n = ct.size
    k = np.arange(n)
    g = np.exp(ct - eta * dt * k)
    g[0] *= 0.5
    if direct:
        x = dt * np.exp(2j * np.pi * np.outer(k, k) / n) @ g
    else:
        x = dt * n * np.fft.ifft(g)
    a = x.real / math.pi
    j = np.where(k < n // 2, k, k - n)
    nu = 2.0 * math.pi * j / (n * dt)
    order = np.argsort(nu, kind="stable")
    return nu[order], a[order]


def gwc_spectrum(omega_rel: np.ndarray, im_sigma: np.ndarray, eta: float, n_t: int, t_max: float, direct=False):
    """Whole cumulant step for one core: beta -> C~(t_k) -> A on bins nu relative to eps^QP."""
    beta = np.abs(im_sigma) / math.pi
    dt = t_max / n_t
    t = dt * np.arange(n_t)
    ct = cumulant_ct(omega_rel, beta, t)
    return spectrum_from_cumulant(ct, dt, eta, direct=direct)


def find_peaks(nu: np.ndarray, a: np.ndarray, rel_threshold=1e-3):
    """Local maxima of A above rel_threshold * max(A), refined by a 3-point parabola.

    Returns a list of (position, height) sorted by position (lower first).
    """
    amax = float(np.max(a))
    out = []
    for j in range(1, a.size - 1):
        if a[j] > a[j - 1] and a[j] >= a[j + 1] and a[j] > rel_threshold * amax:
            y0, y1, y2 = a[j - 1], a[j], a[j + 1]
            den = y0 - 2.0 * y1 + y2
            s = 0.0 if den == 0.0 else 0.5 * (y0 - y2) / den
            h = nu[j + 1] - nu[j]
            out.append((float(nu[j] + s * h), float(y1 - 0.25 * (y0 - y2) * s)))
    return out
