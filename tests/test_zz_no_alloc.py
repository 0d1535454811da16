"""gwc_cumulant_spectrum_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: a serving thread sharing the GPU with another framework's
caching allocator or running under a fixed memory budget (an allocation there can synchronise
the device or exceed the budget), or a caller that holds no gwc_ctx. This test calls the
allocation-free entry point through the C ABI twice in a row, with different inputs and sizes,
and checks each result against the context-based gwc_cumulant_spectrum on the same inputs. It
sits in its own file, collected last, and needs nothing from the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(n_core, n_w, seed):
    rng = np.random.default_rng(seed)
    w = np.stack([np.linspace(-0.9 - 0.01 * c, 0.15, n_w) for c in range(n_core)])
    im = np.where(w < 0, rng.uniform(0.0, 0.02, w.shape), 0.0)
    j = np.argmin(np.abs(w[0] + 0.5))
    im[0, j] = 2.0  # one strong pole: Poisson satellites
    return torch.as_tensor(w, device="cuda"), torch.as_tensor(im, device="cuda")


def _with_context(n_core, n_t, t_max, eta, w, im):
    from paper_2412_17132_gb300 import gwc

    # any small molecule with n_core cores gives a context with these cumulant settings
    n_states, n_occ, n_aux = 12, n_core + 1, 8
    eps = torch.linspace(-10.5, 3.0, n_states, dtype=torch.float64, device="cuda")
    o_ov = torch.zeros((n_aux, n_occ * (n_states - n_occ)), dtype=torch.float64, device="cuda")
    o_core = torch.zeros((n_states, n_core, n_aux), dtype=torch.float64, device="cuda")
    ctx = gwc.Context(eps, n_occ, list(range(n_core)), o_ov, o_core, prec="fp64", n_t=n_t, t_max=t_max, eta=eta)
    a, nu = ctx.cumulant_spectrum(w, im)
    ctx.sync()
    out = (a.clone(), nu.clone())
    ctx.close()
    return out


@pytest.fixture(scope="module")
def gwc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_17132_gb300 import gwc as g

    g.lib()
    return g


def test_noalloc_matches_context_path_twice(gwc):
    cases = [(2, 300, 1 << 16, 2000.0, 1e-3, 7), (3, 150, 1 << 14, 900.0, 2e-3, 8)]
    for n_core, n_w, n_t, t_max, eta, seed in cases:
        w, im = _inputs(n_core, n_w, seed)
        a = torch.full((n_core, n_t), float("nan"), dtype=torch.float64, device="cuda")
        nu = torch.empty((n_t,), dtype=torch.float64, device="cuda")
        gwc.cumulant_spectrum_noalloc(w, im, n_t, t_max, eta, a, nu)
        torch.cuda.synchronize()
        a_ref, nu_ref = _with_context(n_core, n_t, t_max, eta, w, im)
        peak = float(a_ref.abs().max())
        assert torch.isfinite(a).all()
        assert float((a - a_ref).abs().max()) <= 1e-10 * peak
        assert float((nu - nu_ref).abs().max()) <= 1e-12
        # the sum rule holds for every core (each spectrum integrates to 1)
        dnu = float(nu[1] - nu[0])
        assert float((a.sum(dim=1) * dnu - 1.0).abs().max()) < 1e-9


def test_noalloc_at_the_size_limit_and_without_bins(gwc):
    # n_core * n_t = 2^18 (the whole ping-pong buffers and twiddle table), n_omega = 4096 (the
    # cumulant kernel above 48 KB of shared memory), then nu_out = NULL; both against the context path
    n_core, n_w, n_t, t_max, eta = 4, 4096, 1 << 16, 2000.0, 1e-3
    w, im = _inputs(n_core, n_w, 9)
    a_ref, nu_ref = _with_context(n_core, n_t, t_max, eta, w, im)
    peak = float(a_ref.abs().max())
    for with_nu in (True, False):
        a = torch.full((n_core, n_t), float("nan"), dtype=torch.float64, device="cuda")
        nu = torch.empty((n_t,), dtype=torch.float64, device="cuda") if with_nu else None
        gwc.cumulant_spectrum_noalloc(w, im, n_t, t_max, eta, a, nu)
        torch.cuda.synchronize()
        assert torch.isfinite(a).all()
        assert float((a - a_ref).abs().max()) <= 1e-10 * peak
        if with_nu:
            assert float((nu - nu_ref).abs().max()) <= 1e-12


def test_noalloc_rejects_sizes_beyond_the_static_scratch(gwc):
    lib = gwc.lib()
    w, im = _inputs(1, 10, 1)
    a = torch.empty((8, 1 << 16), dtype=torch.float64, device="cuda")
    # 8 cores x 2^16 time points exceeds GWC_NOALLOC_MAX_WORK = 2^18
    st = lib.gwc_cumulant_spectrum_noalloc(w.data_ptr(), 10, im.data_ptr(), 8, 1 << 16, 2000.0, 1e-3, a.data_ptr(), None,
                                           torch.cuda.current_stream().cuda_stream)
    assert st == 1
    assert b"static scratch" in lib.gwc_last_error(None)
