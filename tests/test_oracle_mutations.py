"""The oracle's pins catch plausible mistakes (CPU only).

Each test plants one mistake in the oracle (a flipped sign, a dropped term, a wrong weight or
threshold), on the CPU and for the duration of the test only, and checks that at least one pin
of tests/test_oracle_pins.py then fails. A pin that passed on a broken oracle would pin nothing.
"""
import math

import numpy as np
import pytest

import test_oracle_pins as P
from oracle import gwc_oracle as G
from oracle import sop as S
from paper_2412_17132_gb300 import synth


def _small_sop():
    # the data of the pins' small_sop fixture, built under the planted mistake
    m = synth.small(n_states=16, n_occ=4, n_core=1, n_aux=12, seed=5, n_high=2)
    s = G.System.from_molecule(m, n_im=32)
    om, xpy = S.casida_sop(s.o_ov, s.delta)
    rho = np.array([S.transition_moments(s.o_ov, xpy, s.o_core[mm, 0]) for mm in range(m.n_states)])
    return m, s, om, xpy, rho


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_pins_pass_on_the_unmodified_oracle():
    P.test_chi0_imaginary_axis_nsd(synth.tiny())
    P.test_w_ri_solve_equals_sum_over_poles(_small_sop(), 0.7j)
    P.test_sigma_continuous_at_residue_threshold(_small_sop())
    P.test_gl_grid_is_exact_for_lorentzian_kernel()
    P.test_sum_rule_is_one()
    P.test_cumulant_single_pole_is_exact()
    P.test_sigma_cd_converges_to_closed_form(_small_sop())


def test_flipped_sign_of_the_pair_response(monkeypatch):
    orig = G.d_factor
    monkeypatch.setattr(G, "d_factor", lambda delta, z: -orig(delta, z))
    _fails(P.test_chi0_imaginary_axis_nsd, synth.tiny())


def test_dropped_antiresonant_term(monkeypatch):
    monkeypatch.setattr(G, "d_factor", lambda delta, z: 2.0 / (complex(z) - delta))
    _fails(P.test_w_ri_solve_equals_sum_over_poles, _small_sop(), 0.7j)


def test_missing_spin_factor(monkeypatch):
    orig = G.d_factor
    monkeypatch.setattr(G, "d_factor", lambda delta, z: 0.5 * orig(delta, z))
    _fails(P.test_w_ri_solve_equals_sum_over_poles, _small_sop(), 2.5 + 1e-3j)


def test_bare_coulomb_part_left_in_w(monkeypatch):
    def wc_total(pi, rhs):  # b^T eps^-1 b instead of b^T (eps^-1 - 1) b
        x = np.linalg.solve(np.eye(pi.shape[0]) - pi, rhs.astype(complex))
        return np.einsum("pk,pk->k", rhs, x)

    monkeypatch.setattr(G, "screened_wc", wc_total)
    _fails(P.test_w_ri_solve_equals_sum_over_poles, _small_sop(), 0.7j)


def test_theta_of_zero_taken_as_one(monkeypatch):
    monkeypatch.setattr(G, "heaviside", lambda x: 1.0 if x >= 0 else 0.0)
    _fails(P.test_sigma_continuous_at_residue_threshold, _small_sop())


def test_imaginary_axis_term_with_the_wrong_sign(monkeypatch):
    orig = G.System.imag_axis_term
    monkeypatch.setattr(G.System, "imag_axis_term", lambda self, omega: -orig(self, omega))
    _fails(P.test_sigma_cd_converges_to_closed_form, _small_sop())


def test_grid_weights_without_the_jacobian_scale(monkeypatch):
    def grid(n, xi0=1.0):
        x, w = np.polynomial.legendre.leggauss(n)
        return xi0 * (1.0 + x) / (1.0 - x), w / (1.0 - x) ** 2  # 2 xi0 dropped

    monkeypatch.setattr(G, "modified_gl_grid", grid)
    _fails(P.test_gl_grid_is_exact_for_lorentzian_kernel)


def test_full_trapezoid_weight_at_t0(monkeypatch):
    def spectrum(ct, dt, eta, direct=False):  # weight 1 at k = 0 instead of 1/2
        n = ct.size
        k = np.arange(n)
        g = np.exp(ct - eta * dt * k)
        x = dt * n * np.fft.ifft(g)
        j = np.where(k < n // 2, k, k - n)
        nu = 2.0 * math.pi * j / (n * dt)
        order = np.argsort(nu, kind="stable")
        return nu[order], (x.real / math.pi)[order]

    monkeypatch.setattr(G, "spectrum_from_cumulant", spectrum)
    _fails(P.test_sum_rule_is_one)


def test_cumulant_phase_with_the_wrong_sign(monkeypatch):
    def ct(omega_rel, beta, t):  # e^{+i w t} instead of e^{-i w t}
        wq = G.trapezoid_weights(omega_rel)
        keep = omega_rel != 0.0
        c = (wq * beta)[keep] / omega_rel[keep] ** 2
        return (np.exp(1j * np.outer(t, omega_rel[keep])) - 1.0) @ c

    monkeypatch.setattr(G, "cumulant_ct", ct)
    _fails(P.test_cumulant_single_pole_is_exact)


def test_g_energies_ignored_in_the_imaginary_axis_term(monkeypatch):
    def imag_axis_term(self, omega):  # poles of G taken from the input energies, not eps_g
        tab, w0 = self.w_imag_table()
        out = np.zeros(self.n_core)
        for m in range(self.n_states):
            a = omega - self.eps[m]
            if a == 0.0:
                continue
            kern = self.w_xi * a / (a * a + self.xi**2) / math.pi
            out += kern @ (tab[:, m, :] - w0[m][None, :]) + 0.5 * math.copysign(1.0, a) * w0[m]
        return out

    monkeypatch.setattr(G.System, "imag_axis_term", imag_axis_term)
    _fails(P.test_sigma_invariant_under_a_common_shift_of_g_energies)


def test_g_energies_ignored_in_the_residues(monkeypatch):
    def residue_term(self, omega):  # residue positions and occupations from the input energies
        out = np.zeros(self.n_core, dtype=np.complex128)
        per_m = {}
        for m in range(self.n_states):
            f = G.residue_prefactor(self.eps[m], omega, self.eps_f)
            if f == 0.0:
                continue
            w = self.w_residue(m, abs(self.eps[m] - omega))
            per_m[m] = (f, w)
            out += f * w
        return out, per_m

    monkeypatch.setattr(G.System, "residue_term", residue_term)
    _fails(P.test_evgw0_sigma_matches_sum_over_poles_with_qp_energies)


def _group_variant(member_energy_of_n=False, diagonal_rhs=False, all_cores=False):
    """im_sigma_dec_group with one planted mistake: the residue frequency of every member taken from
    the core's own energy, the RI vector o_nn used for every member, or the sum over all cores."""

    def fn(self, omega, groups):
        out = np.zeros(self.n_core)
        for c, n in enumerate(self.core_idx):
            for c2, i in enumerate(self.core_idx):
                if not all_cores and groups[c2] != groups[c]:
                    continue
                e = self.eps_g[n] if member_energy_of_n else self.eps_g[i]
                f = G.residue_prefactor(e, omega, self.eps_f)
                if f == 0.0:
                    continue
                pi = G.chi0(self.o_ov, self.delta, complex(abs(e - omega), self.eta))
                rhs = self.o_core[int(n) if diagonal_rhs else int(i), c][:, None]
                out[c] += f * G.screened_wc(pi, rhs)[0].imag
        return out

    return fn


def test_group_members_at_the_cores_own_residue_frequency(monkeypatch):
    monkeypatch.setattr(G.System, "im_sigma_dec_group", _group_variant(member_energy_of_n=True))
    _fails(P.test_group_decoupling_uses_each_members_own_residue_frequency)


def test_group_members_with_the_diagonal_ri_vector(monkeypatch):
    monkeypatch.setattr(G.System, "im_sigma_dec_group", _group_variant(diagonal_rhs=True))
    _fails(P.test_group_decoupling_equals_sum_over_symmetry_equivalent_poles)


def test_group_sum_over_every_core(monkeypatch):
    monkeypatch.setattr(G.System, "im_sigma_dec_group", _group_variant(all_cores=True))
    _fails(P.test_group_decoupling_equals_sum_over_symmetry_equivalent_poles)


def test_group_pins_pass_on_the_unmodified_variant(monkeypatch):
    monkeypatch.setattr(G.System, "im_sigma_dec_group", _group_variant())
    P.test_group_decoupling_equals_sum_over_symmetry_equivalent_poles()
    P.test_group_decoupling_uses_each_members_own_residue_frequency()


def test_wac_core_window_left_in_ev(monkeypatch):
    orig = G.wac_reference_points

    def ref(*a, **kw):  # 40 taken as Ha: the eV -> Ha conversion dropped
        kw["wc_max_ev"] = 40.0 * 27.211386245988
        return orig(*a, **kw)

    monkeypatch.setattr(G, "wac_reference_points", ref)
    _fails(P.test_wac_reference_points_follow_the_printed_parameters)


def test_wac_valence_margins_swapped(monkeypatch):
    orig = G.wac_reference_points

    def ref(*a, **kw):  # 1 % below and 8 % above instead of 8 % below and 1 % above
        kw.update(d_lower=0.01, d_upper=0.08)
        return orig(*a, **kw)

    monkeypatch.setattr(G, "wac_reference_points", ref)
    _fails(P.test_wac_reference_points_follow_the_printed_parameters)


def test_continued_fraction_with_the_wrong_reference_point(monkeypatch):
    def ev(a, zref, z):  # level p paired with z_p instead of z_{p-1}
        z = np.asarray(z, dtype=np.complex128)
        t = np.ones_like(z)
        for p in range(a.size - 1, 0, -1):
            t = 1.0 + a[p] * (z - zref[min(p, zref.size - 1)]) / t
        return a[0] / t

    monkeypatch.setattr(G, "thiele_eval", ev)
    _fails(P.test_thiele_interpolates_and_reproduces_rational_functions)


def test_g0w0_renormalisation_with_the_slope_sign_flipped(monkeypatch):
    orig = G.g0w0_graphical_solutions

    def sols(*args):  # Z = 1/(1 + dRe Sigma/dw) instead of 1/(1 - dRe Sigma/dw)
        return [(x, 1.0 / (2.0 - 1.0 / z)) for x, z in orig(*args)]

    monkeypatch.setattr(G, "g0w0_graphical_solutions", sols)
    _fails(P.test_g0w0_graphical_solutions_single_pole_closed_form)


def test_beta_without_the_one_over_pi(monkeypatch):
    def spectrum(omega_rel, im_sigma, eta, n_t, t_max, direct=False):  # beta = |Im Sigma|, 1/pi dropped
        dt = t_max / n_t
        ct = G.cumulant_ct(omega_rel, np.abs(im_sigma), dt * np.arange(n_t))
        return G.spectrum_from_cumulant(ct, dt, eta, direct=direct)

    monkeypatch.setattr(G, "gwc_spectrum", spectrum)
    _fails(P.test_spectrum_poisson_closed_form, 0.5)


def test_exchange_summed_over_every_state(monkeypatch):
    monkeypatch.setattr(G.System, "sigma_x", lambda self: -np.einsum("icp,icp->c", self.o_core, self.o_core))
    _fails(P.test_sigma_x_brute_force)


def test_residue_prefactor_with_the_occupations_swapped(monkeypatch):
    orig = G.residue_prefactor
    monkeypatch.setattr(G, "residue_prefactor", lambda eps_m, omega, eps_f: -orig(eps_m, omega, eps_f))
    _fails(P.test_sigma_cd_matches_time_ordered_sop, _small_sop())


def test_pair_response_at_the_conjugate_frequency(monkeypatch):
    orig = G.d_factor
    monkeypatch.setattr(G, "d_factor", lambda delta, z: orig(delta, np.conj(complex(z))))
    _fails(P.test_w_ri_solve_equals_sum_over_poles, _small_sop(), 2.5 + 1e-3j)


def test_w_rebuilt_from_the_g_energies(monkeypatch):
    orig = G.System.with_g_energies

    def with_g(self, eps_g, eps_f=None):  # evGW instead of evGW0: W from the QP energies too
        other = orig(self, eps_g, eps_f)
        other.delta = G.transition_energies(other.eps_g, self.n_occ)
        other._w_im = None
        return other

    monkeypatch.setattr(G.System, "with_g_energies", with_g)
    _fails(P.test_evgw0_sigma_matches_sum_over_poles_with_qp_energies)


def test_trapezoid_endpoints_with_full_weight(monkeypatch):
    def weights(omega):  # interior rule at the ends too: w_0 = d_0 and w_{n-1} = d_{n-2}
        d = np.diff(omega)
        w = np.zeros_like(omega)
        w[:-1] += 0.5 * d
        w[1:] += 0.5 * d
        w[0] += 0.5 * d[0]
        w[-1] += 0.5 * d[-1]
        return w

    monkeypatch.setattr(G, "trapezoid_weights", weights)
    _fails(P.test_trapezoid_weights_integrate_linear_functions_exactly)


def test_near_pole_subtraction_without_its_sign(monkeypatch):
    def imag_axis_term(self, omega):  # + W(i0)/2 whatever the side of the pole, instead of sgn(a) W(i0)/2
        tab, w0 = self.w_imag_table()
        out = np.zeros(self.n_core)
        for m in range(self.n_states):
            a = omega - self.eps_g[m]
            if a == 0.0:
                continue
            kern = self.w_xi * a / (a * a + self.xi**2) / math.pi
            out += kern @ (tab[:, m, :] - w0[m][None, :]) + 0.5 * w0[m]
        return out

    monkeypatch.setattr(G.System, "imag_axis_term", imag_axis_term)
    _fails(P.test_sigma_cd_matches_time_ordered_sop, _small_sop())


def test_residue_frequency_without_its_absolute_value(monkeypatch):
    def residue_term(self, omega):  # W at (eps_m - w) + i eta, negative below the state
        out = np.zeros(self.n_core, dtype=np.complex128)
        per_m = {}
        for m in range(self.n_states):
            f = G.residue_prefactor(self.eps_g[m], omega, self.eps_f)
            if f == 0.0:
                continue
            w = self.w_residue(m, self.eps_g[m] - omega)
            per_m[m] = (f, w)
            out += f * w
        return out, per_m

    monkeypatch.setattr(G.System, "residue_term", residue_term)
    _fails(P.test_sigma_cd_matches_time_ordered_sop, _small_sop())


def test_group_members_with_the_cores_prefactor(monkeypatch):
    def grp(self, omega, groups, cores=None):  # f of core n for every member instead of each member's own f_i
        groups = [int(g) for g in groups]
        out = np.zeros(self.n_core)
        todo = range(self.n_core) if cores is None else [int(c) for c in cores]
        for c in todo:
            f = G.residue_prefactor(self.eps_g[self.core_idx[c]], omega, self.eps_f)
            for c2, i in enumerate(self.core_idx):
                if groups[c2] != groups[c] or f == 0.0:
                    continue
                pi = G.chi0(self.o_ov, self.delta, complex(abs(self.eps_g[i] - omega), self.eta))
                out[c] += f * G.screened_wc(pi, self.o_core[int(i), c][:, None])[0].imag
        return out

    monkeypatch.setattr(G.System, "im_sigma_dec_group", grp)
    _fails(P.test_group_decoupling_uses_each_members_own_prefactor)


def test_gdh_spectrum_without_the_static_part(monkeypatch):
    def gdh(omega_common, sigma_c, eps_n, dh, sigma_x, vxc):  # v^xc - Sigma^x left out of the denominator
        w = omega_common + dh
        re = w - eps_n - sigma_c.real
        im = sigma_c.imag
        return w, np.abs(im) / (re * re + im * im) / math.pi

    monkeypatch.setattr(G, "gdh_spectrum", gdh)
    _fails(P.test_gw_spectral_function_of_the_three_level_model, 0.2)


def test_evgw0_without_the_fermi_level_check(monkeypatch):
    def ev(system, tol=1e-8, max_iter=100, on_fail="return"):  # iterates on past a change of occupations
        n = system.n_states
        sx, vxc = system.sigma_x(), system.v_xc()
        e = system.eps.copy()
        for it in range(1, max_iter + 1):
            s = system.with_g_energies(e)
            new = np.array([system.eps[c] + sx[c] - vxc[c] + s.sigma_c(float(e[c]))[0][c].real for c in range(n)])
            done = np.max(np.abs(new - e)) < tol
            e = new
            if done:
                return e, it
        if on_fail == "raise":
            raise G.NotConverged("max_iter")
        return e, max_iter

    monkeypatch.setattr(G, "evgw0", ev)
    _fails(P.test_evgw0_stops_when_a_state_crosses_the_fermi_level)
