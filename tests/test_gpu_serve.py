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
