"""The accuracy gates at the benzene size (300 states, six 1s cores, N_aux = 1100: nine 128-row tile rows,
eighteen 64-wide panels), the split-BF16 precision form against FP64 oracle values written by
tests/golden/make_benzene_golden.py (oracle only):
  * A(w) max-abs <= 1e-3 of the peak height (Sec. "Numerical GW+C scheme", eq:AGWC) for every core,
    the GPU spectrum from the GPU's decoupled Im Sigma against the oracle's spectrum from its own;
  * satellite positions <= 0.01 eV (every oracle peak above 2e-3 of the maximum has a GPU peak there);
  * the decoupled Im Sigma on the whole 800-point grid and the full Sigma^c at 16 grid points,
    elementwise, within tolerances derived from the chi0 rounding (see SIG_REL below).
"""
import json
import os

import numpy as np
import pytest

from oracle import gwc_oracle as G
from paper_2412_17132_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EV = synth.HARTREE_EV
GOLD = os.path.join(os.path.dirname(__file__), "golden", "benzene_oracle.json")

# Split-BF16 chi0 has a relative error u ~ 2e-6 (three BF16 products of 8-bit-mantissa parts, FP32
# accumulation in segments of 512 terms); W^c = b^T (eps^-1 - 1) b moves by about kappa u |W| with the
# condition number kappa of eps = 1 - Pi, largest near the RPA poles (the bottom of the window). Measured
# on a GB300 at this size: max |dSigma| / |Sigma| = 2.4e-4 (grid point 0, 25 eV below the cores; 1.5e-6
# at the points above the valence residues), an absolute floor of 3.6e-6 Ha there, and max
# |d Im Sigma_dec| = 1.7e-4 Ha against a peak |Im Sigma_dec| of 1.9 Ha. The bounds are 4x those: a
# kernel error above 0.1 % of Sigma anywhere on the grid fails them.
SIG_REL = 1e-3
SIG_ABS = 1.5e-5
DEC_ABS = 7e-4


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(GOLD):
        pytest.skip("no benzene oracle values")
    from paper_2412_17132_gb300 import gwc

    gwc.lib()
    with open(GOLD) as f:
        gold = json.load(f)
    mol = synth.benzene()
    ctx = gwc.Context.from_molecule(mol, prec="bf16x3")
    sig, dec, _ = ctx.sigma_core(mol.omega)
    w_rel = mol.omega[None, :] - mol.eps[mol.core_idx][:, None]
    a, nu = ctx.cumulant_spectrum(torch.as_tensor(np.ascontiguousarray(w_rel), device="cuda"), dec)
    ctx.sync()
    out = dict(mol=mol, gold=gold, sig=sig.cpu().numpy(), dec=dec.cpu().numpy(), a=a.cpu().numpy(),
               nu=nu.cpu().numpy(), w_rel=w_rel)
    ctx.close()
    return out


def test_decoupled_im_sigma_on_the_whole_grid(run):
    ref = np.array(run["gold"]["im_sigma_dec"])
    err = np.max(np.abs(run["dec"] - ref))
    print(f"max |d Im Sigma_dec| = {err:.3e} Ha (max |Im Sigma_dec| = {np.max(np.abs(ref)):.3e})")
    assert err <= DEC_ABS


def test_full_sigma_at_sixteen_points(run):
    g = run["gold"]
    for k, j in enumerate(g["sigma_idx"]):
        ref = np.array([complex(*v) for v in g["sigma_c"][k]])
        got = run["sig"][:, j, 0] + 1j * run["sig"][:, j, 1]
        err = np.abs(got - ref)
        print(f"grid point {j}: max |dSigma| = {np.max(err):.3e} Ha, max rel = {np.max(err / np.abs(ref)):.3e}")
        assert np.all(err <= SIG_REL * np.abs(ref) + SIG_ABS), (j, np.max(err))


def test_spectra_and_satellite_gates(run):
    mol, ref_dec = run["mol"], np.array(run["gold"]["im_sigma_dec"])
    for c in range(mol.n_core):
        nu_ref, a_ref = G.gwc_spectrum(run["w_rel"][c], ref_dec[c], mol.eta, mol.n_t, mol.t_max)
        assert np.max(np.abs(run["nu"] - nu_ref)) < 1e-12
        a = run["a"][c]
        gap = np.max(np.abs(a - a_ref)) / np.max(a_ref)
        print(f"core {c}: max |dA| / peak = {gap:.3e}")
        assert gap <= 1e-3
        pk = G.find_peaks(nu_ref, a_ref, 1e-3)
        pg = G.find_peaks(run["nu"], a, 1e-3)
        for p, h in pk:
            if h > 2e-3 * np.max(a_ref):
                assert min(abs(p - q) for q, _ in pg) * EV <= 0.01, (c, p)
