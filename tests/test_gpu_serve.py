"""Serving loop: results are the same alone and in the mix; admission respects the memory budget."""
import math

import numpy as np
import pytest

from paper_2412_17132_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EV = synth.HARTREE_EV


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17132_gb300 import gwc, serve as s

    gwc.lib()
    return s


def _requests(serve, sizes, arrival=0.0):
    reqs = []
    for rid, n in enumerate(sizes):
        n_occ = max(2, round(n / 18))
        n_core = max(1, round(0.3 * n_occ))

        def make(rid=rid, n=n, n_occ=n_occ, n_core=n_core):
            return synth.molecule_device(f"r{rid}", n, n_occ, n_core, int(round(2.5 * n)), seed=500 + rid, n_t=1 << 14)

        reqs.append(serve.Request(rid=rid, arrival=arrival, make=make, n_states=n))
    return reqs


GRID = np.linspace(-25.0 / EV, 5.0 / EV, 161)
# 20 requests of uneven size (log-uniform in [60, 160] states, seeded), as in the serving recipe's
# equality check of 20 requests alone and in the mix
SIZES = [int(round(math.exp(x))) for x in np.random.default_rng(7).uniform(math.log(60), math.log(160), 20)]


def test_results_same_alone_and_in_the_mix(serve):
    alone = {}
    srv1 = serve.SpectrumServer(GRID, budget_bytes=1 << 40, slots=1, n_t=1 << 14)
    for r in _requests(serve, SIZES):
        (d,) = srv1.run([r])
        assert d.status == 0
        alone[d.rid] = d
    srv = serve.SpectrumServer(GRID, budget_bytes=1 << 40, slots=8, n_t=1 << 14)
    done = srv.run(_requests(serve, SIZES))
    assert len(done) == len(SIZES)
    # at least two requests were on the GPU at the same time
    spans = sorted((d.admitted, d.finished) for d in done)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    for d in done:
        a = alone[d.rid]
        assert d.status == 0
        np.testing.assert_allclose(d.eps_qp, a.eps_qp, rtol=0, atol=1e-12)
        np.testing.assert_allclose(d.im_sigma, a.im_sigma, rtol=0, atol=1e-12)
        np.testing.assert_allclose(d.spectrum, a.spectrum, rtol=0, atol=1e-9 * np.max(np.abs(a.spectrum)))
        # the spectrum of each core integrates to one (sum rule of the damped transform)
        dnu = 2 * math.pi / 2000.0
        assert np.max(np.abs(d.spectrum.sum(axis=1) * dnu - 1.0)) < 1e-9


def test_admission_respects_the_memory_budget(serve):
    reqs = _requests(serve, [80, 80, 80])
    srv = serve.SpectrumServer(GRID, budget_bytes=1, slots=3, n_t=1 << 14)  # nothing fits next to another
    done = srv.run(reqs)
    spans = sorted((d.admitted, d.finished) for d in done)
    assert len(done) == 3
    assert all(spans[i + 1][0] >= spans[i][1] for i in range(2))  # strictly one at a time


def test_capacity_context_reloads_smaller_systems(serve):
    """A context created with sizes only (the capacity of a size class) runs requests of smaller molecules
    loaded with gwc_load, one after another, with the results of a context made for each molecule."""
    from paper_2412_17132_gb300 import gwc

    n_cap, n_occ_cap, n_aux_cap, n_core_cap = serve.recipe_sizes(150)
    cap = gwc.Context.with_capacity(n_cap, n_occ_cap, n_aux_cap, n_core_cap, prec="bf16x3", qp_mode="hedin", n_t=1 << 14)
    with pytest.raises(gwc.GwcError):
        cap.request_plan(GRID)  # no system loaded yet
    for rid, n in enumerate((120, 90, 150)):
        n_s, n_occ, n_aux, n_core = serve.recipe_sizes(n)
        mol = synth.molecule_device(f"c{rid}", n_s, n_occ, n_core, n_aux, seed=900 + rid, n_t=1 << 14)
        eps = torch.as_tensor(mol.eps, device="cuda")
        cap.load(eps, mol.o_ov, mol.o_core, core_idx=mol.core_idx, n_occ=mol.n_occ)
        cap.request_plan(GRID)
        cap.request_step()
        got = [t.cpu().numpy() for t in cap.request_results()]
        cap.sync()
        ref_ctx = gwc.Context(eps, mol.n_occ, mol.core_idx, mol.o_ov, mol.o_core, prec="bf16x3", qp_mode="hedin",
                              n_t=1 << 14)
        ref_ctx.request_plan(GRID)
        ref_ctx.request_step()
        ref = [t.cpu().numpy() for t in ref_ctx.request_results()]
        ref_ctx.sync()
        ref_ctx.close()
        for g, r in zip(got, ref):
            np.testing.assert_allclose(g, r, rtol=0, atol=1e-12 * max(1.0, float(np.max(np.abs(r)))))
    big = serve.recipe_sizes(200)
    mol = synth.molecule_device("big", big[0], big[1], big[3], big[2], seed=1, n_t=1 << 14)
    with pytest.raises(gwc.GwcError) as err:
        cap.load(torch.as_tensor(mol.eps, device="cuda"), mol.o_ov, mol.o_core, core_idx=mol.core_idx, n_occ=mol.n_occ)
    assert err.value.status == 1
    cap.close()


def test_server_reuses_resident_contexts(serve):
    sizes = [100, 130, 110, 140, 95, 120]
    srv = serve.SpectrumServer(GRID, budget_bytes=1 << 40, slots=2, n_t=1 << 14)
    reqs = []
    for rid, n in enumerate(sizes):
        n_s, n_occ, n_aux, n_core = serve.recipe_sizes(n)
        reqs.append(serve.Request(rid=rid, arrival=0.0, n_states=n,
                                  make=lambda rid=rid, n_s=n_s, n_occ=n_occ, n_aux=n_aux, n_core=n_core:
                                  synth.molecule_device(f"s{rid}", n_s, n_occ, n_core, n_aux, seed=700 + rid, n_t=1 << 14)))
    done = srv.run(reqs)
    assert len(done) == len(sizes) and all(d.status == 0 for d in done)
    assert srv.created <= 2 and srv.reused >= len(sizes) - 2  # one class, at most one context per slot
    srv.close()
