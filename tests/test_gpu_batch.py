"""Request mode (decoupled spectra + QP as one capturable step), the batched CUDA-graph form and
the autotuner, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import gwc_oracle as G
from paper_2412_17132_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EV = synth.HARTREE_EV


@pytest.fixture(scope="module")
def gwc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17132_gb300 import gwc as g

    g.lib()
    return g


def _rel_grid(n=201, lo_ev=-25.0, hi_ev=5.0):
    return np.linspace(lo_ev / EV, hi_ev / EV, n)


def _request(gwc, mol, prec="bf16x3", qp_mode="hedin", n=201):
    ctx = gwc.Context.from_molecule(mol, prec=prec, qp_mode=qp_mode)
    ctx.request_plan(_rel_grid(n))
    ctx.request_step()
    res = [t.clone() for t in ctx.request_results()]
    ctx.sync()
    return ctx, res


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_request_step_matches_oracle(gwc, prec):
    mol = synth.small(n_states=40, n_occ=6, n_core=2, n_aux=90, seed=41)
    ctx, (eqp, dh, it, im, a, nu) = _request(gwc, mol, prec=prec)
    s = G.System.from_molecule(mol)
    w_rel = _rel_grid()
    tol = {"fp64": (0.0, 1e-9), "bf16x3": (2e-2, 2e-3)}[prec]
    for c in range(2):
        ec = float(mol.eps[c])
        ref = np.array([s.sigma_c(ec + w)[1][c] for w in w_rel])
        got = im[c].cpu().numpy()
        assert np.all(np.abs(got - ref) <= tol[0] * np.abs(ref) + tol[1]), np.max(np.abs(got - ref))
        # QP in closed form (eq QPGWC): eps_n + dH_n with dH_n = Re Sigma^c_n(eps_n) (v^xc = Sigma^x)
        dh_ref = s.sigma_c_core(c, ec).real
        assert abs(float(dh[c]) - dh_ref) * EV < (1e-9 if prec == "fp64" else 1e-3)
        assert abs(float(eqp[c]) - (ec + float(dh[c]))) < 1e-12
        # spectrum of the request equals the cumulant oracle applied to the same Im Sigma
        nu_ref, a_ref = G.gwc_spectrum(w_rel, got, mol.eta, mol.n_t, mol.t_max)
        assert np.max(np.abs(a[c].cpu().numpy() - a_ref)) < 1e-9 * np.max(a_ref)


def test_request_secant_agrees_with_closed_form(gwc):
    mol = synth.small(n_states=40, n_occ=6, n_core=2, n_aux=90, seed=43)
    _, (e_h, dh_h, _, _, _, _) = _request(gwc, mol, prec="fp64", qp_mode="hedin")
    _, (e_s, dh_s, it_s, _, _, _) = _request(gwc, mol, prec="fp64", qp_mode="secant")
    assert torch.allclose(dh_h, dh_s, rtol=0, atol=1e-12)
    assert float((e_h - e_s).abs().max()) * EV < 1e-3
    assert int(it_s.min()) >= 2


@pytest.mark.parametrize("grouped", [True, False])
def test_batch_graph_equals_individual_steps(gwc, grouped, monkeypatch):
    """Each molecule's result is the same alone and inside the batched graph (uneven sizes): the grouped
    form (persistent grouped chi0 and grouped factorisation launches over all molecules) and the graph of
    per-molecule steps (GWC_BATCH set)."""
    monkeypatch.setenv("GWC_BATCH", "grouped" if grouped else "per-molecule")
    if grouped:  # the grouped launch factors with the one-CTA tensor-core kernel; so do the steps it is compared to
        monkeypatch.setenv("GWC_FACTOR", "tc")
    mols = [synth.small(n_states=n, n_occ=max(2, n // 8), n_core=1 + (n % 2), n_aux=int(2.5 * n), seed=100 + n)
            for n in (24, 41, 57, 33)]
    alone = []
    for m in mols:
        ctx, res = _request(gwc, m)
        alone.append(res)
        ctx.close()
    ctxs = []
    for m in mols:
        c = gwc.Context.from_molecule(m, prec="bf16x3", qp_mode="hedin")
        c.request_plan(_rel_grid())
        ctxs.append(c)
    batch = gwc.Batch(ctxs)
    assert batch.grouped == grouped
    for rep in range(2):  # two launches of the same graph
        batch.launch()
        torch.cuda.synchronize()
        for c, ref in zip(ctxs, alone):
            got = c.request_results()
            torch.cuda.synchronize()
            for g, r in zip(got, ref):
                if g.dtype == torch.int32:
                    assert torch.equal(g, r)
                else:
                    assert float((g - r).abs().max()) <= 1e-12 * max(1.0, float(r.abs().max()))
    batch.close()
    for c in ctxs:
        c.sync()


def test_autotune_picks_a_valid_batch(gwc):
    mol = synth.small(n_states=40, n_occ=6, n_core=2, n_aux=90, seed=47)
    ctx = gwc.Context.from_molecule(mol, prec="bf16x3", qp_mode="hedin", batch=128)
    ctx.request_plan(_rel_grid())
    chosen = ctx.autotune()
    assert chosen in (16, 32, 64, 128)
    assert ctx.chi0_ctas() in (0, torch.cuda.get_device_properties(0).multi_processor_count)
    tile = ctx.chi0_tile()
    assert tile in (0, 1)
    ctx.request_step()
    ctx.sync()
    eq, dh, _, im, _, _ = [t.cpu().numpy() for t in ctx.request_results()]
    # the second context of the same shape bucket reuses the cached choice
    ctx2 = gwc.Context.from_molecule(mol, prec="bf16x3", qp_mode="hedin", batch=128)
    ctx2.request_plan(_rel_grid())
    assert ctx2.autotune() == chosen
    assert ctx2.chi0_tile() == tile and ctx2.chi0_ctas() == ctx.chi0_ctas()
    # the other tile shape gives the same step (both FP32-accurate; only the summation order differs)
    ctx3 = gwc.Context.from_molecule(mol, prec="bf16x3", qp_mode="hedin", batch=128, chi0_tile=1 - tile)
    assert ctx3.chi0_tile() == 1 - tile
    ctx3.request_plan(_rel_grid())
    ctx3.request_step()
    ctx3.sync()
    eq3, dh3, _, im3, _, _ = [t.cpu().numpy() for t in ctx3.request_results()]
    assert np.max(np.abs(dh3 - dh)) <= 1e-5 * max(1.0, np.max(np.abs(dh)))
    assert np.max(np.abs(im3 - im)) <= 1e-4 * np.max(np.abs(im))
    for c in (ctx, ctx2, ctx3):
        c.close()


def test_persistent_chi0_equals_one_cta_per_item(gwc):
    """The polarizability build as a persistent launch (one CTA per SM looping over the tile items, running
    barrier phases across items) gives the same matrices as one CTA per item, real and complex z."""
    mol = synth.small(n_states=60, n_occ=9, n_core=2, n_aux=300, seed=53)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    z = torch.tensor([[0.0, 0.6], [0.0, 0.0], [0.41, 1e-3], [3.3, 1e-3], [0.0, 5.0]], dtype=torch.float64, device="cuda")
    outs = []
    for ctas in (0, n_sm, 7):  # 7 CTAs: many items per CTA
        ctx = gwc.Context.from_molecule(mol, prec="bf16x3", chi0_ctas=ctas)
        outs.append(ctx.build_chi0(z))
        ctx.sync()
        ctx.close()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_grouped_batch_with_many_chunks(gwc, monkeypatch):
    """Small workspaces (16 frequencies per batch) give each molecule several residue chunks, and the grouped
    launches hold different numbers of molecules chunk by chunk; results as the molecules alone (both with the
    one-CTA tensor-core factorisation, the grouped launch's kernel)."""
    monkeypatch.setenv("GWC_FACTOR", "tc")
    mols = [synth.small(n_states=n, n_occ=max(2, n // 8), n_core=1 + (n % 3), n_aux=int(2.5 * n), seed=200 + n)
            for n in (36, 52, 29)]
    alone = []
    for m in mols:
        ctx, res = _request(gwc, m)
        alone.append(res)
        ctx.close()
    ctxs = []
    for m in mols:
        c = gwc.Context.from_molecule(m, prec="bf16x3", qp_mode="hedin", batch=16)
        c.request_plan(_rel_grid())
        ctxs.append(c)
    import os

    os.environ["GWC_BATCH"] = "grouped"
    try:
        batch = gwc.Batch(ctxs)
    finally:
        del os.environ["GWC_BATCH"]
    assert batch.grouped
    batch.launch()
    torch.cuda.synchronize()
    for c, ref in zip(ctxs, alone):
        got = c.request_results()
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            if g.dtype == torch.int32:
                assert torch.equal(g, r)
            else:
                assert float((g - r).abs().max()) <= 1e-12 * max(1.0, float(r.abs().max()))
        c.sync()
    batch.close()
