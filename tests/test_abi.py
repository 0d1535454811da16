"""C-ABI checks that need no GPU: the library builds, loads, and exports what gwc.h declares;
host-side validation rejects bad arguments before any launch."""
import ctypes
import math
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gwc.h")


@pytest.fixture(scope="module")
def libgwc():
    from paper_2412_17132_gb300 import gwc

    if not os.path.exists(gwc.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("no nvcc to build libgwc.so")
        from paper_2412_17132_gb300 import _build

        _build.build()
    return gwc.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gwc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_paths_entry_points():
    names = declared_functions()
    for n in ("gwc_build_chi0", "gwc_screen", "gwc_sigma_core", "gwc_qp_solve", "gwc_cumulant_spectrum",
              "gwc_create", "gwc_destroy", "gwc_last_error", "gwc_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol(libgwc):
    for name in declared_functions():
        assert hasattr(libgwc, name), name


def test_abi_version_and_strings(libgwc):
    assert libgwc.gwc_abi_version() == 3
    assert libgwc.gwc_status_string(4) == b"singular dielectric matrix"


def test_default_options(libgwc):
    from paper_2412_17132_gb300 import gwc

    o = gwc.default_options()
    assert o.eta == 1e-3 and o.n_im == 32 and o.n_t == 1 << 16 and o.prec == gwc.PREC["bf16x3"]
    assert o.chi0_ctas == 0 and o.chi0_tile == 0


def _sys(n_states=20, n_occ=4, n_aux=10, n_core=1, core=None):
    from paper_2412_17132_gb300 import gwc

    core = np.zeros(n_core, dtype=np.int32) if core is None else np.asarray(core, dtype=np.int32)
    eps = np.linspace(-10, 5, n_states)
    o_ov = np.zeros((n_aux, n_occ * (n_states - n_occ)))
    o_core = np.zeros((n_states, n_core, n_aux))
    keep = (core, eps, o_ov, o_core)
    s = gwc.System(n_states, n_occ, n_aux, n_core, core.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), eps.ctypes.data,
                   o_ov.ctypes.data, o_core.ctypes.data, None, math.nan, 1)
    return s, keep


def test_workspace_bytes_host_only(libgwc):
    from paper_2412_17132_gb300 import gwc

    s, keep = _sys()
    o = gwc.default_options()
    b = ctypes.c_size_t()
    assert libgwc.gwc_workspace_bytes(ctypes.byref(s), ctypes.byref(o), 400, ctypes.byref(b)) == 0
    assert b.value > 20 * 10 * 8


@pytest.mark.parametrize(
    "kw",
    [dict(n_occ=0), dict(n_occ=20), dict(n_aux=0), dict(n_core=0), dict(n_core=21), dict(core=[20]), dict(core=[-1])],
)
def test_create_rejects_bad_sizes_without_gpu(libgwc, kw):
    from paper_2412_17132_gb300 import gwc

    s, keep = _sys(**kw)
    o = gwc.default_options()
    ctx = ctypes.c_void_p()
    st = libgwc.gwc_create(ctypes.byref(ctx), ctypes.byref(s), ctypes.byref(o), None)
    assert st == 1 and not ctx.value
    assert libgwc.gwc_last_error(None)


@pytest.mark.parametrize("field,val", [("eta", 0.0), ("n_im", 0), ("n_t", 1000), ("max_qp_iter", 1), ("prec", 9),
                                       ("chi0_ctas", -1), ("chi0_tile", 2), ("chi0_tile", -1)])
def test_create_rejects_bad_options_without_gpu(libgwc, field, val):
    from paper_2412_17132_gb300 import gwc

    s, keep = _sys()
    o = gwc.default_options()
    setattr(o, field, val)
    ctx = ctypes.c_void_p()
    assert libgwc.gwc_create(ctypes.byref(ctx), ctypes.byref(s), ctypes.byref(o), None) == 1


def test_null_context_calls_are_rejected(libgwc):
    assert libgwc.gwc_sigma_core(None, None, 0, None, None, None, None) == 1
    assert libgwc.gwc_qp_solve(None, None, None, None, None) == 1
    assert libgwc.gwc_cumulant_spectrum(None, None, 0, None, None, None, None) == 1
    assert libgwc.gwc_build_chi0(None, None, 0, None, None) == 1
    assert libgwc.gwc_screen(None, None, 0, None, 0, None, None) == 1
    assert libgwc.gwc_set_g_energies(None, None, 0.0, None) == 1
    it = ctypes.c_int(0)
    assert libgwc.gwc_evgw0(None, 1e-8, 10, None, ctypes.byref(it), None) == 1


@pytest.mark.parametrize(
    "n_core,n_omega,n_t",
    [(1, 100, 1 << 19), (2, 100, 1 << 18), (64, 2048, 4096), (1, 0, 1024), (1, 100, 1000), (0, 100, 1024)],
)
def test_noalloc_rejects_bad_sizes_without_gpu(libgwc, n_core, n_omega, n_t):
    # the limits of the static scratch (n_core n_t <= 2^18, n_core n_omega <= 2^16) and the shape
    # rules are checked before any CUDA call; the pointers are never touched on rejection
    buf = (ctypes.c_double * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    st = libgwc.gwc_cumulant_spectrum_noalloc(p, n_omega, p, n_core, n_t, 2000.0, 1e-3, p, p, None)
    assert st == 1
    assert libgwc.gwc_last_error(None)
