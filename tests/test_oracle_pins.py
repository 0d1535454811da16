"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form, an
independent algebraic route (the Casida sum over poles), an exact discrete identity, a
printed parameter set, or brute force. Citations name the paper's sections/equation labels.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import gwc_oracle as G
from oracle import sop as S
from paper_2412_17132_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EV = synth.HARTREE_EV


# ----------------------------------------------------------------------------------------
# Imaginary-axis grid (Sec. "Computational Details": modified Gauss-Legendre grid)
# ----------------------------------------------------------------------------------------


def test_gl_grid_is_exact_for_lorentzian_kernel():
    # int_0^inf dxi a/(a^2+xi^2) = pi/2 sgn(a); with xi0 = a the mapped integrand is 1/(1+x^2) on (-1,1)
    xi, w = G.modified_gl_grid(32, 1.0)
    assert abs(np.sum(w / (1.0 + xi**2)) - math.pi / 2) < 1e-14
    xi, w = G.modified_gl_grid(200, 1.0)
    for a in (0.05, 0.7, 3.0, 11.0):
        assert abs(np.sum(w * a / (a * a + xi**2)) - math.pi / 2) < 2e-4


# ----------------------------------------------------------------------------------------
# P1: chi0 on the imaginary axis is real symmetric negative semidefinite; ||Pi(i0)|| = 2
# ----------------------------------------------------------------------------------------


def test_chi0_imaginary_axis_nsd(tiny_mol):
    s = G.System.from_molecule(tiny_mol)
    for xi in (0.0, 0.1, 1.0, 7.5, 40.0):
        pi = G.chi0(s.o_ov, s.delta, 1j * xi)
        assert np.all(pi.imag == 0.0)
        p = pi.real
        assert np.max(np.abs(p - p.T)) <= 1e-15 * np.max(np.abs(p))
        ev = np.linalg.eigvalsh(p)
        assert ev[-1] <= 1e-12 * np.max(np.abs(ev))
    n0 = np.linalg.eigvalsh(-G.chi0(s.o_ov, s.delta, 0.0).real)[-1]
    assert abs(n0 - 2.0) < 1e-12


def test_chi0_brute_force_sum_over_pairs():
    # Pi_PQ(z) as the literal double loop over occupied i and virtual a with D = 2[1/(z-D)-1/(z+D)]
    m = synth.small(n_states=9, n_occ=3, n_aux=5, seed=11)
    s = G.System.from_molecule(m)
    z = 1.3 + 0.02j
    pi = G.chi0(s.o_ov, s.delta, z)
    ref = np.zeros((5, 5), dtype=complex)
    n_v = m.n_states - m.n_occ
    for i in range(m.n_occ):
        for a in range(n_v):
            dl = m.eps[m.n_occ + a] - m.eps[i]
            d = 2.0 / (z - dl) - 2.0 / (z + dl)
            col = m.o_ov[:, i * n_v + a]
            ref += d * np.outer(col, col)
    assert np.max(np.abs(pi - ref)) < 1e-14


# ----------------------------------------------------------------------------------------
# P2: contour deformation == sum over poles (Eqs. rpa_casida, density_shifts, W_spectral,
# sigma_spectral vs Eqs. cd_terms, cd_imaginary, cd_residue)
# ----------------------------------------------------------------------------------------


@pytest.fixture(scope="module")
def small_sop():
    m = synth.small(n_states=16, n_occ=4, n_core=1, n_aux=12, seed=5, n_high=2)
    s = G.System.from_molecule(m, n_im=32)
    om, xpy = S.casida_sop(s.o_ov, s.delta)
    rho = np.array([S.transition_moments(s.o_ov, xpy, s.o_core[mm, 0]) for mm in range(m.n_states)])
    return m, s, om, xpy, rho


def test_casida_energies_match_ri_form(small_sop):
    # Omega^2 = eig(Delta^2 + 4 Delta^1/2 K Delta^1/2): the symmetric reduction of the Casida problem
    m, s, om, _, _ = small_sop
    k = s.o_ov.T @ s.o_ov
    sq = np.sqrt(s.delta)
    c = np.diag(s.delta**2) + 4.0 * sq[:, None] * k * sq[None, :]
    ref = np.sqrt(np.linalg.eigvalsh(c))
    assert np.max(np.abs(np.sort(om) - ref)) < 1e-10 * ref.max()


@pytest.mark.parametrize("z", [0.37 + 0.01j, 2.5 + 1e-3j, 10.2 + 1e-3j, 0.7j, 15.0j, 0.0])
def test_w_ri_solve_equals_sum_over_poles(small_sop, z):
    m, s, om, _, rho = small_sop
    pi = G.chi0(s.o_ov, s.delta, z)
    w_ri = G.screened_wc(pi, s.o_core[:, 0, :].T)
    w_sp = np.array([S.w_sop(rho[mm], om, z) for mm in range(m.n_states)])
    assert np.max(np.abs(w_ri - w_sp)) <= 1e-10 * max(1e-3, np.max(np.abs(w_sp)))


def test_w_ri_equals_sop_on_tiny(tiny_mol):
    s = G.System.from_molecule(tiny_mol)
    om, xpy = S.casida_sop(s.o_ov, s.delta)
    for mm in (0, 3, 7, 30, 59):
        rho = S.transition_moments(s.o_ov, xpy, s.o_core[mm, 0])
        for z in (0.2 + 1e-3j, 9.9 + 1e-3j, 1.5j):
            w_ri = G.screened_wc(G.chi0(s.o_ov, s.delta, z), s.o_core[mm, 0][:, None])[0]
            w_sp = S.w_sop(rho, om, z)
            assert abs(w_ri - w_sp) <= 1e-9 * max(1e-4, abs(w_sp))


def test_sigma_cd_converges_to_closed_form(small_sop):
    # CD with quadrature vs the same CD expression with the exact imaginary-axis integral:
    # the only difference is quadrature error, which must shrink with more nodes.
    m, _, om, _, rho = small_sop
    eps_f = G.fermi_level(m.eps, m.n_occ)
    ws = [m.eps[0] - 0.9, m.eps[0] - 0.31, m.eps[0] + 0.05, m.eps[0]]
    errs = {}
    for n_im in (32, 200, 800):
        s = G.System.from_molecule(m, n_im=n_im)
        e = 0.0
        for w in ws:
            cd = s.sigma_c(float(w))[0][0]
            ref = S.sigma_c_cd_closed_form(m.eps, eps_f, rho, om, float(w), m.eta)
            e = max(e, abs(cd - ref))
        errs[n_im] = e
    assert errs[800] < errs[32]
    assert errs[800] < 1e-6
    assert errs[200] < 1e-4


def test_sigma_cd_matches_time_ordered_sop(small_sop):
    # Eq. sigma_spectral (time-ordered +-i eta per pole) vs CD: differ by the anti-resonant eta
    # placement, bounded by sum rho^2 eta/(x+Omega)^2, plus quadrature error.
    m, _, om, _, rho = small_sop
    s = G.System.from_molecule(m, n_im=800)
    eps_f = s.eps_f
    # below and at the core level (occupied residues), and above virtual levels (virtual residues; the
    # last one excites the lowest RPA pole through the residue of the lowest virtual state)
    for w in (m.eps[0] - 0.9, m.eps[0] - 0.31, m.eps[0] + 0.05, m.eps[m.n_occ] + 0.05, m.eps[m.n_occ + 2] + 0.3,
              m.eps[m.n_occ] + float(np.min(om))):
        cd = s.sigma_c(float(w))[0][0]
        sp = S.sigma_c_sop(m.eps, eps_f, rho, om, float(w), m.eta)
        bound = sum(np.sum(rho[mm] ** 2 * 2 * m.eta / (abs(m.eps[mm] - w) + om) ** 2) for mm in range(m.n_states))
        assert abs(cd - sp) <= bound + 1e-6


def test_im_sigma_only_from_residues(tiny_mol):
    # Eq. cd_sigma_imaginary: I_n is real, so Im Sigma^c = Im R_n
    s = G.System.from_molecule(tiny_mol)
    w = float(tiny_mol.omega[123])
    sig, _ = s.sigma_c(w)
    r, _ = s.residue_term(w)
    assert np.all(np.isreal(s.imag_axis_term(w)))
    assert abs(sig[0].imag - r[0].imag) == 0.0


def test_sigma_continuous_at_residue_threshold(small_sop):
    # Theta(0) = 1/2 makes Sigma^c continuous at w = eps_m (both one-sided limits agree)
    m, s, _, _, _ = small_sop
    e = float(m.eps[2])
    lo = s.sigma_c(e - 1e-9)[0][0]
    mid = s.sigma_c(e)[0][0]
    hi = s.sigma_c(e + 1e-9)[0][0]
    assert abs(lo - mid) < 1e-6 and abs(hi - mid) < 1e-6


# ----------------------------------------------------------------------------------------
# P4: the G_dH W0 QP solution is eps_n + dH_n (Eqs. hedin_shift, hedin_sigma_spectral, QPGWC)
# ----------------------------------------------------------------------------------------


def test_qp_lands_on_hedin_closed_form(tiny_mol):
    s = G.System.from_molecule(tiny_mol)
    eqp, dh, it = s.qp_solve()
    assert abs(eqp[0] - (tiny_mol.eps[0] + dh[0])) * EV < 1e-3
    assert it[0] < 50


def test_qp_closed_form_small_multi_core():
    m = synth.small(n_states=20, n_occ=5, n_core=2, n_aux=14, seed=9)
    s = G.System.from_molecule(m, n_im=16, vxc=np.array([-0.3, -0.25]))
    eqp, dh, _ = s.qp_solve()
    sx = s.sigma_x()
    for c in range(2):
        assert abs(eqp[c] - (m.eps[c] + dh[c])) * EV < 1e-3
        # dH contains the static part Sigma^x - v^xc
        assert abs(dh[c] - (s.sigma_c_core(c, float(m.eps[c])).real + sx[c] - s.vxc[c])) < 1e-12


# ----------------------------------------------------------------------------------------
# P3/P5/P6: cumulant spectrum (Eqs. landau_cumulant_truncated, cumulant_propagator_fourier,
# eq:AGWC; Poisson satellites of the minimal model)
# ----------------------------------------------------------------------------------------


def _single_pole_beta(n_w, omega_sat, mass):
    w = np.linspace(-1.2, 0.2, n_w)
    j = int(np.argmin(np.abs(w - (-omega_sat))))
    w = w - (w[j] + omega_sat)  # put node j exactly at -Omega
    wq = G.trapezoid_weights(w)
    im = np.zeros(n_w)
    im[j] = math.pi * mass / wq[j]
    return w, im


def test_cumulant_single_pole_is_exact():
    om = 0.5
    w, im = _single_pole_beta(301, om, 0.02)
    t = np.linspace(0, 300, 1001)
    ct = G.cumulant_ct(w, np.abs(im) / math.pi, t)
    gam = 0.02 / om**2
    ref = gam * (np.exp(1j * om * t) - 1.0)
    assert np.max(np.abs(ct - ref)) < 1e-13


def _poisson_closed_form(gam, om, eta, n, dt, qmax=60):
    # X_j = dt e^{-gam} sum_q gam^q/q! [sum_k r_q^k - 1/2], r_q = exp((i(nu_j + q Om) - eta) dt)
    k = np.arange(n)
    nu = 2 * math.pi * np.where(k < n // 2, k, k - n) / (n * dt)
    x = np.zeros(n, dtype=complex)
    for q in range(qmax):
        r = np.exp((1j * (nu + q * om) - eta) * dt)
        geo = (1.0 - r**n) / (1.0 - r) - 0.5
        x += gam**q / math.factorial(q) * geo
    x *= dt * math.exp(-gam)
    order = np.argsort(nu, kind="stable")
    return nu[order], x.real[order] / math.pi


@pytest.mark.parametrize("ratio", json.load(open(os.path.join(GOLDEN, "model_ratios.json")))["rho_over_omega"])
def test_spectrum_poisson_closed_form(ratio):
    om, eta, n, t_max = 0.5, 1e-3, 1 << 14, 2000.0
    gam = ratio**2
    w, im = _single_pole_beta(401, om, gam * om**2)
    nu, a = G.gwc_spectrum(w, im, eta, n, t_max)
    nu2, ref = _poisson_closed_form(gam, om, eta, n, t_max / n)
    assert np.max(np.abs(nu - nu2)) == 0.0
    assert np.max(np.abs(a - ref)) < 1e-9 * np.max(ref)


def test_spectrum_fft_equals_direct_dft():
    w, im = _single_pole_beta(101, 0.3, 0.01)
    nu, a = G.gwc_spectrum(w, im, 2e-3, 256, 300.0)
    nu2, a2 = G.gwc_spectrum(w, im, 2e-3, 256, 300.0, direct=True)
    assert np.max(np.abs(a - a2)) < 1e-12 * np.max(np.abs(a))


def test_sum_rule_is_one():
    # sum_j A_j dnu = Re e^{C~(0)} = 1 for any beta (discrete identity of the transform)
    rng = np.random.default_rng(4)
    w = np.linspace(-1.0, 0.2, 300)
    im = np.where(w < 0, rng.uniform(0, 0.05, w.size), 0.0)
    for n, t_max in ((4096, 500.0), (1 << 16, 2000.0)):
        nu, a = G.gwc_spectrum(w, im, 1e-3, n, t_max)
        assert abs(np.sum(a) * (nu[1] - nu[0]) - 1.0) < 1e-10


def test_poisson_positions_and_weights_ch4():
    # Table 1 CH4 cc-pVTZ: Omega = 13.91 eV, rho = 0.3352 eV -> gamma = (rho/Omega)^2 = 5.8e-4 (weak
    # coupling); satellites at eps^QP - k Omega with weights e^-g g^k/k! (minimal-model discussion)
    row = json.load(open(os.path.join(GOLDEN, "ch4_table1.json")))["rows"][0]
    om = row["Omega_sat1_eV"] / EV
    gam = (row["rho_c1s_c1s_eV"] / row["Omega_sat1_eV"]) ** 2
    assert abs(gam - 5.807e-4) < 1e-6
    eta, n, t_max = 1e-3, 1 << 19, 32000.0  # dnu = eta/5
    w, im = _single_pole_beta(801, om, gam * om**2)
    nu, a = G.gwc_spectrum(w, im, eta, n, t_max)
    peaks = G.find_peaks(nu, a, rel_threshold=1e-5)
    pos = sorted(p for p, _ in peaks)
    assert abs(pos[-1]) * EV < 0.01  # QP peak at eps^QP
    assert abs(pos[-2] + om) * EV < 0.01  # first satellite at eps^QP - Omega
    dnu = nu[1] - nu[0]
    for k in (0, 1):
        lo, hi = -k * om - 0.1, -k * om + 0.1
        win = (nu > lo) & (nu < hi)
        area = np.sum(a[win]) * dnu
        # mass of the Poisson series of Lorentzians (width eta) centred at -q Omega inside the window
        ref = sum(
            math.exp(-gam) * gam**q / math.factorial(q) * (math.atan((hi + q * om) / eta) - math.atan((lo + q * om) / eta)) / math.pi
            for q in range(6)
        )
        assert abs(area - ref) < 2e-3 * gam**k


# ----------------------------------------------------------------------------------------
# P8: three-level core-hole model (Sec. minimal model; Cederbaum et al.)
# ----------------------------------------------------------------------------------------


def three_level(omega, rho, eps_c=-10.0, eps_o=-0.5, eta=1e-3):
    dl = 0.9 * omega  # bare valence excitation eps_v - eps_o
    kappa = math.sqrt((omega**2 - dl**2) / (4 * dl))
    rt = math.sqrt(rho**2 * omega / (2 * kappa**2 * dl))
    eps = np.array([eps_c, eps_o, eps_o + dl])
    o_ov = np.array([[0.0, kappa]])  # (c,v) omitted (CVS), (o,v) = kappa
    o_core = np.array([[[rt]], [[0.0]], [[0.0]]])
    return G.System(eps, 2, [0], o_ov, o_core, eta, n_im=200), dl, kappa, rt


@pytest.mark.parametrize("ratio", [0.05, 0.5, 1.0])
def test_three_level_w_closed_form(ratio):
    om = 0.5
    s, dl, kappa, rt = three_level(om, ratio * om)
    big = math.sqrt(dl**2 + 4 * dl * kappa**2)
    assert abs(big - om) < 1e-14
    for z in (0.2 + 1e-3j, 0.5 + 1e-3j, 1.3j):
        w = G.screened_wc(G.chi0(s.o_ov, s.delta, z), s.o_core[0, 0][:, None])[0]
        ref = (ratio * om) ** 2 * 2 * om / (z * z - om * om)
        assert abs(w - ref) < 1e-12 * max(1.0, abs(ref))


def test_three_level_spectrum_is_poisson():
    om, ratio, eta = 0.5, 0.5, 1e-3
    s, _, _, _ = three_level(om, ratio * om, eta=eta)
    ec = float(s.eps[0])
    w_abs = np.linspace(ec - 1.0, ec + 0.1, 2201)
    dec = np.array([s.sigma_c(float(w))[1][0] for w in w_abs])
    eqp, dh, _ = s.qp_solve()
    nu, a = G.gwc_spectrum(w_abs - ec, dec, eta, 1 << 18, 25000.0)
    peaks = sorted(G.find_peaks(nu, a, rel_threshold=1e-4))
    pos = [p for p, _ in peaks]
    # QP peak at 0 (relative to eps^QP), satellites at -k Omega, k = 1, 2, 3
    for k in range(4):
        assert min(abs(p + k * om) for p in pos) * EV < 0.01
    # cumulant weight gamma = rho^2/Omega^2 (Lorentzian-broadened pole carries ~all the mass)
    beta = np.abs(dec) / math.pi
    wr = w_abs - ec
    wq = G.trapezoid_weights(wr)
    keep = wr != 0
    gam_num = np.sum((wq * beta)[keep] / wr[keep] ** 2)
    # closed-form Im W^c of the model on the same grid: rho^2 Im[2 Omega/((x + i eta)^2 - Omega^2)], x = -w
    x = -wr
    im_ref = np.where(x > 0, (ratio * om) ** 2 * (2 * om / ((x + 1j * eta) ** 2 - om**2)).imag, 0.0)
    gam_ref = np.sum((wq * np.abs(im_ref) / math.pi)[keep] / wr[keep] ** 2)
    assert abs(gam_num - gam_ref) < 1e-9 * gam_ref
    # and gamma -> rho^2/Omega^2 up to the finite-eta Lorentzian tails (relative O(eta/Omega log))
    assert abs(gam_num - ratio**2) < 0.03 * ratio**2
    assert abs(eqp[0] - (ec + dh[0])) * EV < 1e-3


# ----------------------------------------------------------------------------------------
# P7: first-order approximation (Eq. im_sigma_satellites) for weak, smooth coupling
# ----------------------------------------------------------------------------------------


def test_first_order_satellite_shape():
    # The quadrature grid must resolve the damping (d omega << eta), otherwise e^{C~} is a comb of
    # separate grid lines; here d omega = eta/10.
    eta = 1e-2
    w = np.linspace(-3.0, 0.0, 3001)
    gam_target = 2e-3
    beta = np.exp(-((w + 1.2) ** 2) / (2 * 0.25**2))
    wq = G.trapezoid_weights(w)
    keep = w != 0
    beta *= gam_target / np.sum((wq * beta)[keep] / w[keep] ** 2)
    nu, a = G.gwc_spectrum(w, math.pi * beta, eta, 1 << 15, 2500.0)  # e^{-eta t_max} negligible
    z = math.exp(-gam_target)
    sel = (nu > -2.0) & (nu < -0.6)
    # Z [delta(nu) + beta(nu)/nu^2], the delta broadened into the damping Lorentzian of width eta
    approx = z * (eta / math.pi / (nu[sel] ** 2 + eta**2) + np.interp(nu[sel], w, beta) / nu[sel] ** 2)
    # residual: second order (gamma) and the eta-Lorentzian smoothing of beta, ~1% here
    assert np.max(np.abs(a[sel] - approx)) < 0.015 * np.max(approx)


# ----------------------------------------------------------------------------------------
# P9: decoupling (Eqs. sigma_spectral_decoupled, cd_sigma_imaginary_decoupled)
# ----------------------------------------------------------------------------------------


def test_decoupling_exact_without_off_diagonal_moments():
    m = synth.small(n_states=18, n_occ=4, n_core=1, n_aux=10, seed=21)
    o_core = m.o_core.copy()
    o_core[1:, 0, :] = 0.0  # O^P_{m,c} = 0 for m != c
    s = G.System(m.eps, m.n_occ, m.core_idx, m.o_ov, o_core, m.eta, n_im=16)
    for w in np.linspace(m.eps[0] - 0.9, m.eps[0] + 0.1, 7):
        sig, dec = s.sigma_c(float(w))
        assert abs(sig[0].imag - dec[0]) <= 1e-15 * max(1.0, abs(dec[0]))


def test_correlation_satellites_appear_with_high_virtuals(tiny_mol):
    # with the 3-40 Ha virtuals the full Im Sigma carries structure the decoupled one lacks
    s = G.System.from_molecule(tiny_mol)
    ws = tiny_mol.omega[::20]
    full = np.array([s.sigma_c(float(w))[0][0].imag for w in ws])
    dec = np.array([s.sigma_c(float(w))[1][0] for w in ws])
    assert np.max(np.abs(full - dec)) > 1e-6


def mirrored_two_core_system(seed=41, n_states=14, n_occ=4, n_aux=10, eta=2e-3):
    """Two symmetry-equivalent 1s cores (states 0 and 1, degenerate) plus a third core (state 2).

    A full RI tensor O^P_mn (symmetric in m, n) is made invariant under the mirror that swaps the
    states 0 <-> 1 together with the auxiliary functions P <-> n_aux-1-P, so W^c_00 = W^c_11 and
    W^c_10 = W^c_01 at every z, while W^c_10 != W^c_00."""
    rng = np.random.default_rng(seed)
    eps = np.sort(np.concatenate([[-10.4, -10.4, -10.3], rng.uniform(-1.0, -0.25, n_occ - 3),
                                  rng.uniform(0.0, 3.0, n_states - n_occ - 2), [6.0, 25.0]]))
    o = rng.normal(0.0, 0.05, (n_aux, n_states, n_states))
    o = 0.5 * (o + o.transpose(0, 2, 1))
    perm = np.arange(n_states)
    perm[[0, 1]] = [1, 0]
    o = 0.5 * (o + o[::-1][:, perm][:, :, perm])
    o[:, :3, :] *= 3.0  # core-localised coefficients
    o[:, :, :3] *= 3.0
    o_ov = np.ascontiguousarray(o[:, :n_occ, n_occ:].reshape(n_aux, -1))
    o_core = np.ascontiguousarray(o[:, :, :3].transpose(1, 2, 0))  # [m][core][P]
    return eps, n_occ, np.array([0, 1, 2]), o_ov, o_core, eta


def _group_sop_reference(s, omega, groups, c):
    """sum over the group of core c and the RPA poles of rho_{i n}^2 eta / ((w - eps_i + Omega)^2 + eta^2)
    (Eq. sigma_spectral_decoupled_symmetric with the pole at eps_i - Omega), and the bound
    sum rho^2 eta / (|eps_i - w| + Omega)^2 on its difference from the residue form (the anti-resonant
    term that the residue form keeps and the time-ordered sum drops)."""
    om, xpy = S.casida_sop(s.o_ov, s.delta)
    ref, bound = 0.0, 0.0
    for c2, i in enumerate(s.core_idx):
        if groups[c2] != groups[c]:
            continue
        rho = S.transition_moments(s.o_ov, xpy, s.o_core[int(i), c])
        x = omega - s.eps[i]
        ref += float(np.sum(rho**2 * s.eta / ((x + om) ** 2 + s.eta**2)))
        bound += float(np.sum(rho**2 * s.eta / (abs(x) + om) ** 2))
    return ref, bound


def test_group_decoupling_equals_sum_over_symmetry_equivalent_poles():
    # Eq. sigma_spectral_decoupled_symmetric: the group form is the RPA pole sum over the group's
    # members, each with its own transition moments rho_{i n} and its own pole position eps_i - Omega
    eps, n_occ, core_idx, o_ov, o_core, eta = mirrored_two_core_system()
    s = G.System(eps, n_occ, core_idx, o_ov, o_core, eta, n_im=8)
    groups = [0, 0, 1]
    om, _ = S.casida_sop(s.o_ov, s.delta)
    ws = [eps[0] - om[0] - 0.3 * eta, eps[0] - om[3], eps[0] - 0.37, eps[0] + 0.01, eps[2] - om[1]]
    for w in ws:
        got = s.im_sigma_dec_group(float(w), groups)
        for c in range(3):
            ref, bound = _group_sop_reference(s, float(w), groups, c)
            assert abs(got[c] - ref) <= bound * (1.0 + 1e-9) + 1e-13, (w, c, got[c], ref, bound)
        # the two mirror images see the same group sum; the off-diagonal member contributes
        assert abs(got[0] - got[1]) <= 1e-12 * max(1e-12, abs(got[0]))
        diag = s.sigma_c(float(w))[1]
        assert abs(got[2] - diag[2]) <= 1e-14 * max(1.0, abs(diag[2]))  # a one-member group is DIAG


def test_group_decoupling_uses_each_members_own_residue_frequency():
    # non-degenerate members: the residue of member i sits at |eps_i - w| (checked against the pole sum)
    m = synth.small(n_states=16, n_occ=5, n_core=3, n_aux=9, seed=44, n_high=2)
    s = G.System.from_molecule(m, n_im=8)
    groups = [0, 0, 0]
    om, _ = S.casida_sop(s.o_ov, s.delta)
    for w in (m.eps[0] - om[0], m.eps[2] - om[0], m.eps[1] - om[2]):
        got = s.im_sigma_dec_group(float(w), groups)
        for c in range(3):
            ref, bound = _group_sop_reference(s, float(w), groups, c)
            assert abs(got[c] - ref) <= bound * (1.0 + 1e-9) + 1e-13, (w, c, got[c], ref, bound)
        # every member on its own resonance carries weight: the group sum is not the DIAG value
        assert np.max(np.abs(got - s.sigma_c(float(w))[1])) > 1e-3 * np.max(np.abs(got))


def two_members_apart_system(seed=61, n_states=14, n_occ=5, n_aux=9):
    """Two occupied cores (states 0 and 1) 1.4 Ha apart, one symmetry group; the lowest RPA pole lies
    below their separation. Returns (eps, n_occ, core_idx, o_ov, o_core, eta)."""
    rng = np.random.default_rng(seed)
    eps = np.sort(np.concatenate([[-10.4, -9.0], rng.uniform(-1.0, -0.25, n_occ - 2),
                                  rng.uniform(0.0, 3.0, n_states - n_occ)]))
    o = rng.normal(0.0, 0.05, (n_aux, n_states, n_states))
    o = 0.5 * (o + o.transpose(0, 2, 1))
    o[:, :2, :] *= 3.0
    o[:, :, :2] *= 3.0
    o_ov = np.ascontiguousarray(o[:, :n_occ, n_occ:].reshape(n_aux, -1))
    o_core = np.ascontiguousarray(o[:, :, :2].transpose(1, 2, 0))
    return eps, n_occ, np.array([0, 1]), o_ov, o_core, 1e-3


def test_group_decoupling_uses_each_members_own_prefactor():
    # members 1.4 Ha apart: at w = eps_0 + Omega_0 (above member 0, below member 1) member 0 has f_0 = 0 and
    # adds nothing, although its residue frequency |eps_0 - w| = Omega_0 sits on the lowest RPA pole; the
    # prefactor of core 1 (f_1 = -1) applied to it would add a Lorentzian peak of height rho^2/eta
    eps, n_occ, core_idx, o_ov, o_core, eta = two_members_apart_system()
    s = G.System(eps, n_occ, core_idx, o_ov, o_core, eta, n_im=8)
    om, _ = S.casida_sop(s.o_ov, s.delta)
    w = float(eps[0] + np.min(om))
    assert eps[0] < w < eps[1]
    got = s.im_sigma_dec_group(w, [0, 0])
    for c in range(2):
        ref, bound = _group_sop_reference(s, w, [0, 0], c)
        assert abs(got[c] - ref) <= bound * (1.0 + 1e-9) + 1e-13, (c, got[c], ref, bound)


# ----------------------------------------------------------------------------------------
# Exchange (Eq. sigma_x): brute force over (n i | i n) with (mn|kl) = sum_P O^P_mn O^P_kl
# ----------------------------------------------------------------------------------------


def test_trapezoid_weights_integrate_linear_functions_exactly():
    # the Landau integral's quadrature (Eq. landau_cumulant_truncated) on a non-uniform grid: exact for
    # a + b w, so the weights sum to the grid's length and their first moment is (w_max^2 - w_min^2)/2
    rng = np.random.default_rng(17)
    w = np.sort(rng.uniform(-1.3, 0.4, 57))
    wq = G.trapezoid_weights(w)
    lo, hi = w[0], w[-1]
    assert abs(np.sum(wq) - (hi - lo)) < 1e-14
    assert abs(np.sum(wq * (0.7 - 2.1 * w)) - (0.7 * (hi - lo) - 2.1 * (hi**2 - lo**2) / 2)) < 1e-13
    assert np.all(wq > 0)


def test_sigma_x_brute_force():
    m = synth.small(n_states=10, n_occ=4, n_core=2, n_aux=6, seed=2)
    s = G.System.from_molecule(m)
    for c in range(2):
        ref = 0.0
        for i in range(m.n_occ):
            ref -= sum(m.o_core[i, c, p] * m.o_core[i, c, p] for p in range(6))
        assert abs(s.sigma_x()[c] - ref) < 1e-14 * abs(ref)


def test_peak_finder_on_parabola():
    nu = np.linspace(-1, 1, 201)
    a = 1.0 - (nu - 0.0123) ** 2
    (p, h), = G.find_peaks(nu, a)
    assert abs(p - 0.0123) < 1e-12 and abs(h - 1.0) < 1e-12


# ----------------------------------------------------------------------------------------
# G_dH W0 spectral function (eqs gw_full_propagator, A_explicit_real_imaginary, hedin_sigma_spectral)
# ----------------------------------------------------------------------------------------


@pytest.mark.parametrize("static", [0.0, 0.2])
def test_gw_spectral_function_of_the_three_level_model(static):
    # With Sigma^c(w) = rho^2/(w - eps_c + Omega - i eta) (eq sigma_spectral for the model) and a static
    # part s = Sigma^x - v^xc, G has the two poles x (x = w - eps_c) with (x - s)(x + Omega) = rho^2,
    # x = (-(Omega - s) +- sqrt((Omega - s)^2 + 4 (s Omega + rho^2)))/2: one QP peak and one satellite
    # below it, with weights (x_+ + Omega)/(x_+ - x_-) and the rest. eta = 1e-3 makes the QP peak's width
    # Z rho^2 eta/(x_+ + Omega)^2 several grid steps wide, so that the sums over the grid hold its mass.
    om, rho, eta, ec = 0.5, 0.2, 1e-3, -10.0
    w = np.linspace(ec - 1.5, ec + 0.5, 200001)
    sig = rho**2 / (w - ec + om - 1j * eta)
    ww, a = G.gdh_spectrum(w, sig, ec, 0.0, -3.0, -3.0 - static)
    disc = math.sqrt((om - static) ** 2 + 4 * (static * om + rho * rho))
    xp, xm = (-(om - static) + disc) / 2, (-(om - static) - disc) / 2
    pk = sorted(p for p, h in G.find_peaks(ww - ec, a, 1e-3))
    assert len(pk) == 2
    assert abs(pk[1] - xp) < 2e-5 and abs(pk[0] - xm) < 2e-5
    dw = w[1] - w[0]
    wp = (xp + om) / (xp - xm)
    assert abs(np.sum(a[np.abs(ww - ec - xp) < 0.05]) * dw - wp) < 5e-3
    assert abs(np.sum(a) * dw - 1.0) < 5e-3


def test_gdh_qp_peak_sits_at_eps_plus_hedin_shift(tiny_mol):
    # the real part of the G_dH W0 denominator vanishes at w = eps_n + dH_n (eq QPGWC)
    s = G.System.from_molecule(tiny_mol)
    ec = float(tiny_mol.eps[0])
    dh = s.hedin_shift()[0]
    sig0 = s.sigma_c_core(0, ec)
    w, a = G.gdh_spectrum(np.array([ec]), np.array([sig0]), ec, dh, s.sigma_x()[0], s.v_xc()[0])
    re = w[0] - ec + s.v_xc()[0] - s.sigma_x()[0] - sig0.real
    assert abs(w[0] - (ec + dh)) < 1e-15 and abs(re) < 1e-12


# ----------------------------------------------------------------------------------------
# CD-WAC (Eq. pade_approximation): the continued fraction interpolates, reproduces rational
# functions exactly, and then gives the CD self-energy exactly
# ----------------------------------------------------------------------------------------


def test_thiele_interpolates_and_reproduces_rational_functions():
    rng = np.random.default_rng(3)
    z = rng.uniform(-2, 2, 12) + 1j * rng.uniform(0.1, 2, 12)
    u = rng.normal(size=12) + 1j * rng.normal(size=12)
    a = G.thiele_coefficients(z, u)
    assert np.max(np.abs(G.thiele_eval(a, z, z) - u)) < 1e-9 * np.max(np.abs(u))
    # W^c of three poles is a rational function of degree 6: 13 points determine it everywhere
    rho, om = np.array([0.3, 0.2, 0.1]), np.array([0.7, 1.9, 3.4])

    def w(zz):
        return np.sum(rho[:, None] ** 2 * 2 * om[:, None] / (np.asarray(zz)[None, :] ** 2 - om[:, None] ** 2), axis=0)

    zr = np.concatenate([1j * np.linspace(0.1, 5, 7), np.linspace(0.2, 4.0, 7) + 1e-3j])
    a = G.thiele_coefficients(zr, w(zr))
    zt = np.array([0.55 + 1e-3j, 2.7 + 1e-3j, 1.1j, 7.0 + 1e-3j])
    assert np.max(np.abs(G.thiele_eval(a, zr, zt) - w(zt))) < 1e-8 * np.max(np.abs(w(zt)))


def test_wac_reference_points_follow_the_printed_parameters():
    # Sec. "Computational Details": N_C = N_V = 100 real points; core region w_C in [0, 40] eV; valence
    # region from 8 % below to 1 % above the range of |eps_m - w| of the residues of the non-core
    # occupied states. Hand-built three-level case: core -10.4, valence -0.5, virtual 2.0 Ha,
    # eps_F = 0.75; at w = -10.5 and -10.0 the valence residue sits at x = 10.0 and 9.5 Ha.
    eps = np.array([-10.4, -0.5, 2.0])
    x = G.wac_reference_points(eps, 2, [0], [-10.5, -10.0], 0.75)
    assert x.size == 200
    core, val = x[:100], x[100:]
    assert core[0] == 0.0 and abs(core[-1] - 40.0 / 27.211386245988) < 1e-12  # 40 eV = 1.46998 Ha
    assert np.allclose(np.diff(core), core[-1] / 99, rtol=0, atol=1e-14)
    assert abs(val[0] - 9.5 * 0.92) < 1e-12 and abs(val[-1] - 10.0 * 1.01) < 1e-12
    assert np.allclose(np.diff(val), (10.1 - 8.74) / 99, rtol=0, atol=1e-13)
    # above the valence level no non-core occupied state has a residue: only the core region
    assert G.wac_reference_points(eps, 2, [0], [0.1], 0.75).size == 100
    # the core's own residue does not move the valence window
    x2 = G.wac_reference_points(eps, 2, [0], [-10.5, -10.0, -10.4], 0.75)
    assert np.array_equal(x2, x)


def test_cdwac_equals_cd_when_w_has_few_poles():
    # 2 occupied x 2 virtual states -> 4 RPA poles: W^c_mn is rational of degree 8, so the fit through
    # 33 + 20 reference points is exact and CD-WAC reproduces the CD self-energy
    m = synth.small(n_states=4, n_occ=2, n_core=1, n_aux=6, seed=13, n_high=1, n_omega=9)
    s = G.System.from_molecule(m, n_im=32)
    xref = G.wac_reference_points(m.eps, m.n_occ, m.core_idx, m.omega, s.eps_f, n_core_ref=10, n_val_ref=10)
    wac = G.sigma_c_wac(s, m.omega, xref)
    cd = np.array([s.sigma_c(float(w))[0] for w in m.omega]).T
    assert np.max(np.abs(wac - cd)) < 1e-7 * max(1.0, np.max(np.abs(cd)))


# ---- plain G0W0 QP equation: several solutions (Sec. "Satellites in the G0W0 approximation") -----
def test_g0w0_graphical_solutions_single_pole_closed_form():
    """Re Sigma(w) = rho^2 (w - p) / ((w - p)^2 + eta^2) (one pole, eta far below the grid step): the
    G0W0 equation eps + Re Sigma(w) = w has the two closed-form solutions
    w = [(eps + p) +- sqrt((eps - p)^2 + 4 rho^2)] / 2 with Z = 1 / (1 + rho^2 / (w - p)^2), whose Z sum
    to 1; the crossing of the pole itself comes out with Z < 0."""
    eps, p, rho2, eta = -10.0, -11.0, 0.1, 1e-6
    w = np.linspace(-12.0, -9.0, 30001)
    re = rho2 * (w - p) / ((w - p) ** 2 + eta ** 2)
    roots = G.g0w0_graphical_solutions(w, re + 0j, eps, 0.0, 0.0)
    phys = [(x, z) for x, z in roots if z > 0]
    assert len(phys) == 2 and len(roots) == 3
    s = math.sqrt((eps - p) ** 2 + 4 * rho2)
    exact = sorted([((eps + p) - s) / 2, ((eps + p) + s) / 2])
    for (x, z), xe in zip(phys, exact):
        ze = 1.0 / (1.0 + rho2 / (xe - p) ** 2)
        assert abs(x - xe) < 1e-7, (x, xe)
        assert abs(z - ze) < 5e-3 * ze, (z, ze)
    assert abs(sum(1.0 / (1.0 + rho2 / (xe - p) ** 2) for xe in exact) - 1.0) < 1e-12
    pole = [x for x, z in roots if z < 0]
    assert len(pole) == 1 and abs(pole[0] - p) < 2e-4


def test_g0w0_secant_root_is_a_graphical_solution():
    """The secant solution of the plain G0W0 equation satisfies it and lies within one grid step of
    a graphical solution with Z > 0 (a small system, 201-point grid around the core level)."""
    m = synth.small(n_states=20, n_occ=5, n_core=1, n_aux=14, seed=9)
    s = G.System.from_molecule(m)
    eqp, dh, it = s.qp_solve(mode="g0w0")
    sx, vxc = s.sigma_x(), s.v_xc()
    e_n = float(m.eps[m.core_idx[0]])
    resid = e_n + sx[0] - vxc[0] + s.sigma_c_core(0, float(eqp[0])).real - eqp[0]
    assert abs(resid) < 1e-6
    grid = np.linspace(min(e_n, eqp[0]) - 0.5, max(e_n, eqp[0]) + 0.5, 201)
    sig, _ = s.sigma_c_grid(grid)
    roots = G.g0w0_graphical_solutions(grid, sig[0], e_n, sx[0], vxc[0])
    step = grid[1] - grid[0]
    assert any(z > 0 and abs(x - eqp[0]) < step for x, z in roots), (eqp[0], roots)


# ----------------------------------------------------------------------------------------
# evGW0: QP energies of every state in G, W at the RPA level of the input energies
# (Sec. "GW for core-levels: beyond G0W0", Eqs. ev_sigma_spectral, hedin_shift)
# ----------------------------------------------------------------------------------------


def _all_state_system(seed=21, n_occ=3, n_virt=7, n_aux=8, scale=0.06, n_im=32):
    # every state is a "core" (its self-energy is computed): O^P_mn symmetric in m, n
    rng = np.random.default_rng(seed)
    eps = np.concatenate([np.sort(rng.uniform(-1.2, -0.3, n_occ)), np.sort(rng.uniform(0.1, 2.5, n_virt))])
    n = eps.size
    o = rng.normal(0.0, scale, (n_aux, n, n))
    o = 0.5 * (o + o.transpose(0, 2, 1))
    o_ov = o[:, :n_occ, n_occ:].reshape(n_aux, -1)
    o_core = np.ascontiguousarray(np.transpose(o, (1, 2, 0)))  # [m][n][P] = O^P_{m,n}
    return G.System(eps, n_occ, np.arange(n), o_ov, o_core, 1e-3, n_im=n_im)


def test_sigma_invariant_under_a_common_shift_of_g_energies():
    # CD depends on the poles of G only through w - eps~_m and the occupations: shifting every
    # eps~_m, eps_F and w by the same amount leaves Sigma^c unchanged (both terms, all states)
    s = _all_state_system()
    d = 0.37
    s2 = s.with_g_energies(s.eps + d, eps_f=s.eps_f + d)
    for w in (-0.95, -0.5, 0.05, 0.8, 1.7):
        a = s.sigma_c(w)[0]
        b = s2.sigma_c(w + d)[0]
        assert np.max(np.abs(a - b)) < 1e-10 * max(1.0, np.max(np.abs(a)))


def test_evgw0_sigma_matches_sum_over_poles_with_qp_energies():
    # Eq. ev_sigma_spectral: sum over m, nu of rho^2 / (w - eps~_m + (Omega - i eta) sgn(eps_F - eps~_m))
    # with Omega, rho from the Casida problem of the input energies; CD with G(eps~) must agree
    # within the anti-resonant eta bound (as for G0W0) plus quadrature error
    s = _all_state_system(n_im=800, scale=0.15)  # coupling strong enough that G(eps) instead of G(eps~) fails
    rng = np.random.default_rng(3)
    eps_t = s.eps + rng.uniform(-0.05, 0.05, s.n_states)
    st = s.with_g_energies(eps_t)
    om, xpy = S.casida_sop(s.o_ov, s.delta)
    for n in (0, 2, 3, 8):
        rho = np.array([S.transition_moments(s.o_ov, xpy, s.o_core[m, n]) for m in range(s.n_states)])
        for w in (eps_t[n] - 0.45, eps_t[n] + 0.2, eps_t[n]):
            cd = st.sigma_c(float(w))[0][n]
            sp = S.sigma_c_sop(eps_t, st.eps_f, rho, om, float(w), s.eta)
            bound = sum(np.sum(rho[m] ** 2 * 2 * s.eta / (abs(eps_t[m] - w) + om) ** 2) for m in range(s.n_states))
            assert abs(cd - sp) <= bound + 1e-6, (n, w, abs(cd - sp), bound)


def test_evgw0_first_iteration_is_the_hedin_shift():
    s = _all_state_system()
    e1, it = G.evgw0(s, max_iter=1)
    assert it == 1
    assert np.max(np.abs(e1 - (s.eps + s.hedin_shift()))) < 1e-12


def test_evgw0_converges_to_a_fixed_point():
    s = _all_state_system()
    e, it = G.evgw0(s, tol=1e-9)
    assert it < 100
    st = s.with_g_energies(e)
    sx, vxc = s.sigma_x(), s.v_xc()
    res = [e[n] - (s.eps[n] + sx[n] - vxc[n] + st.sigma_c(float(e[n]))[0][n].real) for n in range(s.n_states)]
    assert np.max(np.abs(res)) < 1e-7
    assert np.all(e[: s.n_occ] < st.eps_f) and np.all(e[s.n_occ :] > st.eps_f)  # occupations kept
    # not the G0W0 / Hedin-shift answer: the QP energies in G moved the result
    assert np.max(np.abs(e - (s.eps + s.hedin_shift()))) > 1e-6


def test_evgw0_rejects_a_core_only_system(tiny_mol):
    with pytest.raises(ValueError):
        G.evgw0(G.System.from_molecule(tiny_mol))


def test_evgw0_stops_when_a_state_crosses_the_fermi_level():
    # reading of the iteration: an iterate whose occupied QP energy reaches the midpoint of the QP HOMO
    # and LUMO ends the scheme without convergence (the occupations of G would change). A v^xc 1 Ha below
    # Sigma^x for the HOMO lifts its first iterate above the LUMO: the scheme returns that iterate after
    # one step, or raises NotConverged
    s0 = _all_state_system()
    v = s0.sigma_x().copy()
    v[s0.n_occ - 1] -= 1.0
    s = G.System(s0.eps, s0.n_occ, s0.core_idx, s0.o_ov, s0.o_core, s0.eta, n_im=s0.n_im, vxc=v)
    e1 = s.eps + s.hedin_shift()
    assert e1[s.n_occ - 1] > e1[s.n_occ]
    e, it = G.evgw0(s)
    assert it == 1 and np.max(np.abs(e - e1)) < 1e-12
    with pytest.raises(G.NotConverged):
        G.evgw0(s, on_fail="raise")
