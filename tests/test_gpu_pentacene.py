"""The pentacene-sized precision form (N_states 1300, N_occ 73, 22 cores, N_aux 4500) against the
FP64 oracle on a subset (the oracle needs hours of CPU time at this size):
  * Hedin shifts dH_n = Re Sigma^c_n(eps_n) (+ Sigma^x - v^xc = 0 by default) of the cores stored in
    tests/golden/pentacene_oracle.json, written by tests/golden/make_pentacene_golden.py (oracle only);
    with the default v^xc the G_dH W0 QP energy is eps_n + dH_n (eq QPGWC), so this is the QP gate
    |dE| <= 1e-3 eV per core;
  * Sigma^c of all 22 cores at the stored grid frequencies, within the bf16x3 tolerance of the
    Sigma tests (2e-2 |Sigma| + 2e-3 Ha).
The inputs come from the device generator with the exact normalisation, equal to the host
generator's molecule to 1e-13 relative (tests/test_synth.py).
"""
import json
import os

import numpy as np
import pytest

from paper_2412_17132_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EV = synth.HARTREE_EV
GOLD = os.path.join(os.path.dirname(__file__), "golden", "pentacene_oracle.json")


@pytest.fixture(scope="module")
def gold():
    if not os.path.exists(GOLD):
        pytest.skip("no pentacene oracle values")
    with open(GOLD) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def ctx(gold):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17132_gb300 import gwc

    gwc.lib()
    mol = synth.pentacene_device()
    return mol, gwc.Context.from_molecule(mol, prec="bf16x3", qp_mode="hedin")


def test_pentacene_hedin_shifts_vs_oracle(gold, ctx):
    mol, c = ctx
    assert gold["cores"], "no core finished in the oracle file"
    e, dh, _ = c.qp_solve()
    c.sync()
    for core, ref, eps_n in zip(gold["cores"], gold["dH"], gold["eps"]):
        assert abs(float(dh[core]) - ref) * EV <= 1e-3, (core, float(dh[core]), ref)
        assert abs(float(e[core]) - (eps_n + ref)) * EV <= 1e-3


def test_pentacene_sigma_points_vs_oracle(gold, ctx):
    mol, c = ctx
    if not gold["points"]:
        pytest.skip("no grid point finished in the oracle file")
    for pt in gold["points"]:
        sig, _, _ = c.sigma_core(np.array([pt["omega"]]))
        c.sync()
        got = sig[:, 0, 0].cpu().numpy() + 1j * sig[:, 0, 1].cpu().numpy()
        ref = np.array([complex(a, b) for a, b in pt["sigma_c"]])
        assert np.all(np.abs(got - ref) <= 2e-2 * np.abs(ref) + 2e-3), np.max(np.abs(got - ref))


def test_pentacene_decoupled_im_sigma_vs_oracle(gold, ctx):
    """The decoupled Im Sigma the spectra start from (request mode, relative grid of 800 points over 30 eV),
    cores 0, 11 and 21 at the stored grid points, within the bound the benzene-sized gates use."""
    from test_gpu_benzene_gates import DEC_ABS

    d = gold.get("dec_rel")
    if not d or not d["values"]:
        pytest.skip("no decoupled values in the oracle file")
    mol, c = ctx
    grid = np.linspace(-25.0 / EV, 5.0 / EV, 800)
    c.request_plan(grid)
    c.set_qp_cores([0])
    c.request_step()
    im = c.request_results()[3].cpu().numpy()
    c.sync()
    c.set_qp_cores(None)
    for k, core in enumerate(d["cores"][: len(d["values"])]):
        err = np.max(np.abs(im[core, d["nu_idx"]] - np.array(d["values"][k])))
        assert err <= DEC_ABS, (core, err)
