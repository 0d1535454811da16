"""Thin ctypes binding of libgwc (argument marshalling only).

Every step of the self-energy / QP / cumulant path runs in the CUDA kernels of
``libgwc.so``; this module only turns torch tensors and numpy arrays into the
pointers and sizes of the C ABI declared in ``include/gwc.h``. PyTorch provides
device memory and streams. There is no CPU fallback: if the library is missing the
import of the binding functions raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgwc.so")

PREC = {"fp64": 0, "bf16": 1, "bf16x3": 2, "fp32": 3, "bf16x3f64": 4}
DEC = {"none": 0, "diag": 1, "group": 2}
QP = {"secant": 0, "hedin": 1, "g0w0": 2}
STATUS = {
    0: "ok",
    1: "invalid argument",
    2: "out of memory",
    3: "CUDA error",
    4: "singular dielectric matrix",
    5: "QP iteration not converged",
    6: "device wait timed out",
    7: "unsupported",
}


class GwcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"gwc status {status} ({STATUS.get(status, '?')}): {message}")
        self.status = status


class System(ctypes.Structure):
    _fields_ = [
        ("n_states", ctypes.c_int),
        ("n_occ", ctypes.c_int),
        ("n_aux", ctypes.c_int),
        ("n_core", ctypes.c_int),
        ("core_idx", ctypes.POINTER(ctypes.c_int)),
        ("eps", ctypes.c_void_p),
        ("o_ov", ctypes.c_void_p),
        ("o_core", ctypes.c_void_p),
        ("vxc", ctypes.c_void_p),
        ("eps_f", ctypes.c_double),
        ("memory", ctypes.c_int),
    ]


ABI_VERSION = 3  # GWC_ABI_VERSION of the gwc.h these structures mirror


class Options(ctypes.Structure):
    _fields_ = [
        ("eta", ctypes.c_double),
        ("n_im", ctypes.c_int),
        ("xi0", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("dec", ctypes.c_int),
        ("group_of_core", ctypes.POINTER(ctypes.c_int)),
        ("n_t", ctypes.c_int),
        ("t_max", ctypes.c_double),
        ("max_qp_iter", ctypes.c_int),
        ("qp_tol", ctypes.c_double),
        ("batch", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("qp_mode", ctypes.c_int),
        ("wait_us", ctypes.c_int),
        ("chi0_ctas", ctypes.c_int),
        ("chi0_tile", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("chi0_builds", ctypes.c_longlong),
        ("chi0_flop", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
        ("factorizations", ctypes.c_longlong),
        ("chi0_launches", ctypes.c_longlong),
        ("chi0_ms", ctypes.c_double),
        ("factor_launches", ctypes.c_longlong),
        ("factor_ms", ctypes.c_double),
        ("factor_flop", ctypes.c_double),
        ("solve_launches", ctypes.c_longlong),
        ("solve_ms", ctypes.c_double),
    ]


_LIB = None

_SIGS = {
    "gwc_abi_version": (ctypes.c_int, []),
    "gwc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gwc_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "gwc_default_options": (ctypes.c_int, [ctypes.POINTER(Options)]),
    "gwc_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(System), ctypes.POINTER(Options), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "gwc_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(System), ctypes.POINTER(Options), ctypes.c_void_p]),
    "gwc_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(System), ctypes.c_void_p]),
    "gwc_build_chi0": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_screen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_sigma_core": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_qp_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_set_g_energies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "gwc_evgw0": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                 ctypes.c_void_p]),
    "gwc_cumulant_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "gwc_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "gwc_destroy": (None, [ctypes.c_void_p]),
    "gwc_sigma_core_wac": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_gdh_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_g0w0_solutions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_request_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "gwc_request_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_request_copy_results": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_void_p]),
    "gwc_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "gwc_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.c_void_p]),
    "gwc_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gwc_batch_destroy": (None, [ctypes.c_void_p]),
    "gwc_batch_is_grouped": (ctypes.c_int, [ctypes.c_void_p]),
    "gwc_batch_timings": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "gwc_get_options": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Options)]),
    "gwc_set_qp_cores": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "gwc_copy_out": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "gwc_cumulant_spectrum_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p]),
}


def lib():
    """Load libgwc.so (built in-tree by ``__graft_entry__.build()``); raise loudly if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgwc.so not found at {LIB_PATH}: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.gwc_abi_version() != ABI_VERSION:  # the structures below mirror this version's layout
            raise RuntimeError(f"libgwc.so has ABI {L.gwc_abi_version()}, this binding {ABI_VERSION}: rebuild it")
        _LIB = L
    return _LIB


def _check(status: int, ctx=None):
    if status != 0:
        msg = lib().gwc_last_error(ctx)
        raise GwcError(status, msg.decode() if msg else "")


def default_options() -> Options:
    o = Options()
    _check(lib().gwc_default_options(ctypes.byref(o)))
    return o


def _ptr(t) -> int:
    """Device/host address of a torch tensor or numpy array (must be contiguous)."""
    if t is None:
        return 0
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def cumulant_spectrum_noalloc(omega_rel, im_sigma, n_t, t_max, eta, a_out, nu_out=None, stream=None):
    """gwc_cumulant_spectrum_noalloc: no context and no allocation by the library; the caller
    passes device tensors omega_rel/im_sigma [n_core][n_omega] and a_out [n_core][n_t]."""
    n_core, n_w = int(omega_rel.shape[0]), int(omega_rel.shape[1])
    _check(lib().gwc_cumulant_spectrum_noalloc(_ptr(omega_rel), n_w, _ptr(im_sigma), n_core, int(n_t), float(t_max),
                                               float(eta), _ptr(a_out), _ptr(nu_out), _stream(stream)), None)
    return a_out, nu_out


class Batch:
    """Many contexts' request steps captured into one CUDA graph (gwc_batch_*)."""

    def __init__(self, contexts, stream=None):
        self._contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self._contexts))(*[c._ctx.value for c in self._contexts])
        self._b = ctypes.c_void_p()
        _check(lib().gwc_batch_create(ctypes.byref(self._b), arr, len(self._contexts), _stream(stream)), None)

    def launch(self, stream=None):
        _check(lib().gwc_batch_launch(self._b, _stream(stream)), None)

    @property
    def grouped(self) -> bool:
        return bool(lib().gwc_batch_is_grouped(self._b))

    def timings(self):
        """ms of the plans gwc_batch_create timed: per-molecule, grouped persistent, grouped per item (-1: not tried)."""
        t = (ctypes.c_float * 3)()
        _check(lib().gwc_batch_timings(self._b, t), None)
        return [float(v) for v in t]

    @property
    def chi0_shape(self) -> str:
        return {0: "per-molecule graph", 1: "pipelined, one CTA per item", 2: "sequential chunks, persistent"}[
            lib().gwc_batch_is_grouped(self._b)]

    def close(self):
        if self._b:
            lib().gwc_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One molecule resident on the current CUDA device (wraps ``gwc_ctx``).

    Inputs may be CUDA torch tensors (``memory='device'``) or numpy arrays
    (``memory='host'``; copied host->device by gwc_create).
    """

    def __init__(self, eps, n_occ, core_idx, o_ov, o_core, *, vxc=None, eps_f=math.nan, eta=1e-3, n_im=32, xi0=1.0,
                 prec="bf16x3", dec="diag", groups=None, n_t=1 << 16, t_max=2000.0, max_qp_iter=50, qp_tol=1e-7,
                 batch=0, profile=False, qp_mode="secant", wait_us=0, chi0_ctas=0, chi0_tile=0, stream=None):
        self._ctx = ctypes.c_void_p()
        host = isinstance(eps, np.ndarray)
        self._keep = []
        core = np.ascontiguousarray(np.asarray(core_idx, dtype=np.int32))
        self._keep.append(core)
        n_states = int(eps.shape[0])
        n_aux = int(o_ov.shape[0])
        self.n_states, self.n_occ, self.n_aux, self.n_core = n_states, int(n_occ), n_aux, int(core.shape[0])
        sysd = System(n_states, int(n_occ), n_aux, int(core.shape[0]), core.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      _ptr(eps), _ptr(o_ov), _ptr(o_core), _ptr(vxc), float(eps_f), 1 if host else 0)
        opt = default_options()
        opt.eta, opt.n_im, opt.xi0 = float(eta), int(n_im), float(xi0)
        opt.prec, opt.dec = PREC[prec], DEC[dec]
        if groups is not None:
            g = np.ascontiguousarray(np.asarray(groups, dtype=np.int32))
            self._keep.append(g)
            opt.group_of_core = g.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        opt.n_t, opt.t_max = int(n_t), float(t_max)
        opt.max_qp_iter, opt.qp_tol, opt.batch = int(max_qp_iter), float(qp_tol), int(batch)
        opt.profile = 1 if profile else 0
        opt.qp_mode = QP[qp_mode]
        opt.wait_us = int(wait_us)
        opt.chi0_ctas = int(chi0_ctas)
        opt.chi0_tile = int(chi0_tile)
        self.opt = opt
        self.prec = prec
        _check(lib().gwc_create(ctypes.byref(self._ctx), ctypes.byref(sysd), ctypes.byref(opt), _stream(stream)), None)

    @classmethod
    def with_capacity(cls, n_states, n_occ, n_aux, n_core, **kw):
        """A context allocated for a system of these sizes that holds no system yet: gwc_load (``load``) puts
        one in, of these sizes or smaller (serving slots)."""
        self = cls.__new__(cls)
        self._ctx = ctypes.c_void_p()
        self._keep = []
        self.n_states, self.n_occ, self.n_aux, self.n_core = int(n_states), int(n_occ), int(n_aux), int(n_core)
        self.capacity = (self.n_states, self.n_occ, self.n_aux, self.n_core)
        sysd = System(self.n_states, self.n_occ, self.n_aux, self.n_core, None, None, None, None, None, math.nan, 0)
        opt = default_options()
        for k, v in kw.items():
            if k in ("prec", "dec", "qp_mode"):
                v = {"prec": PREC, "dec": DEC, "qp_mode": QP}[k][v]
            if k == "stream":
                continue
            setattr(opt, k, v)
        self.opt = opt
        self.prec = kw.get("prec", "bf16x3")
        _check(lib().gwc_create(ctypes.byref(self._ctx), ctypes.byref(sysd), ctypes.byref(opt), _stream(kw.get("stream"))),
               None)
        return self

    @classmethod
    def from_molecule(cls, mol, device="cuda", host=False, **kw):
        import torch

        args = dict(eta=mol.eta, n_im=mol.n_im, xi0=mol.xi0, n_t=mol.n_t, t_max=mol.t_max)
        args.update(kw)
        if host:
            return cls(mol.eps, mol.n_occ, mol.core_idx, mol.o_ov, mol.o_core, **args)
        dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()  # noqa: E731
        return cls(dev(mol.eps), mol.n_occ, mol.core_idx, dev(mol.o_ov), dev(mol.o_core), **args)

    # -- entry points ---------------------------------------------------------------------
    def load(self, eps, o_ov, o_core, vxc=None, eps_f=math.nan, core_idx=None, n_occ=None, stream=None):
        """gwc_load: a system of the context's sizes, or a smaller one within its capacity (then give n_occ
        and core_idx; the sizes follow from the arrays)."""
        host = isinstance(eps, np.ndarray)
        n_states, n_aux = int(eps.shape[0]), int(o_ov.shape[0])
        n_occ = self.n_occ if n_occ is None else int(n_occ)
        core = np.ascontiguousarray(np.asarray(core_idx if core_idx is not None else range(self.n_core), dtype=np.int32))
        sysd = System(n_states, n_occ, n_aux, int(core.shape[0]), core.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      _ptr(eps), _ptr(o_ov), _ptr(o_core), _ptr(vxc), float(eps_f), 1 if host else 0)
        _check(lib().gwc_load(self._ctx, ctypes.byref(sysd), _stream(stream)), self._ctx)
        self.n_states, self.n_occ, self.n_aux, self.n_core = n_states, n_occ, n_aux, int(core.shape[0])

    def build_chi0(self, z, stream=None):
        import torch

        F = int(z.shape[0])
        out = torch.empty((F, self.n_aux, self.n_aux, 2), dtype=torch.float64, device=z.device)
        _check(lib().gwc_build_chi0(self._ctx, _ptr(z), F, _ptr(out), _stream(stream)), self._ctx)
        return out

    def screen(self, z, rhs, stream=None):
        import torch

        F, r = int(rhs.shape[0]), int(rhs.shape[1])
        out = torch.empty((F, r, 2), dtype=torch.float64, device=z.device)
        _check(lib().gwc_screen(self._ctx, _ptr(z), F, _ptr(rhs), r, _ptr(out), _stream(stream)), self._ctx)
        return out

    def sigma_core(self, omega, want_dec=True, stream=None, out=None):
        """omega: host numpy [n_w]; returns CUDA tensors (sigma [n_core][n_w][2], im_dec, sigma_x)."""
        import torch

        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        n_w = om.shape[0]
        if out is None:
            sig = torch.empty((self.n_core, n_w, 2), dtype=torch.float64, device="cuda")
            dec = torch.empty((self.n_core, n_w), dtype=torch.float64, device="cuda") if want_dec else None
            sx = torch.empty((self.n_core,), dtype=torch.float64, device="cuda")
        else:
            sig, dec, sx = out
        _check(lib().gwc_sigma_core(self._ctx, om.ctypes.data, n_w, _ptr(sig), _ptr(dec), _ptr(sx), _stream(stream)), self._ctx)
        return sig, dec, sx

    def set_g_energies(self, eps_g=None, eps_f=math.nan, stream=None):
        """Orbital energies in G for sigma_core (host array [n_states]); None returns to the input energies."""
        if eps_g is None:
            _check(lib().gwc_set_g_energies(self._ctx, None, math.nan, _stream(stream)), self._ctx)
            return
        e = np.ascontiguousarray(np.asarray(eps_g, dtype=np.float64))
        _check(lib().gwc_set_g_energies(self._ctx, e.ctypes.data, float(eps_f), _stream(stream)), self._ctx)

    def evgw0(self, tol=1e-8, max_iter=100, stream=None, out=None):
        """evGW0 QP energies of every state (the context must list every state as a core): a CUDA
        tensor [n_states] and the number of steps. With `out` given, the last iterate is there even
        when the call raises (GWC_ERR_NOT_CONVERGED)."""
        import torch

        e = torch.empty((self.n_states,), dtype=torch.float64, device="cuda") if out is None else out
        it = ctypes.c_int(0)
        _check(lib().gwc_evgw0(self._ctx, float(tol), int(max_iter), _ptr(e), ctypes.byref(it), _stream(stream)), self._ctx)
        return e, it.value

    def qp_solve(self, stream=None, out=None):
        import torch

        if out is None:
            e = torch.empty((self.n_core,), dtype=torch.float64, device="cuda")
            dh = torch.empty_like(e)
            it = torch.empty((self.n_core,), dtype=torch.int32, device="cuda")
        else:
            e, dh, it = out
        _check(lib().gwc_qp_solve(self._ctx, _ptr(e), _ptr(dh), _ptr(it), _stream(stream)), self._ctx)
        return e, dh, it

    def cumulant_spectrum(self, omega_rel, im_sigma, stream=None, out=None):
        import torch

        n_w = int(omega_rel.shape[-1])
        if out is None:
            a = torch.empty((self.n_core, self.opt.n_t), dtype=torch.float64, device="cuda")
            nu = torch.empty((self.opt.n_t,), dtype=torch.float64, device="cuda")
        else:
            a, nu = out
        _check(lib().gwc_cumulant_spectrum(self._ctx, _ptr(omega_rel), n_w, _ptr(im_sigma), _ptr(a), _ptr(nu), _stream(stream)),
               self._ctx)
        return a, nu

    def sigma_core_wac(self, omega, n_core_ref=100, n_val_ref=100, stream=None):
        """Sigma^c by CD-WAC on the host grid omega: CUDA tensors (sigma [n_core][n_w][2], decoupled Im)."""
        import torch

        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        sig = torch.empty((self.n_core, om.shape[0], 2), dtype=torch.float64, device="cuda")
        dec = torch.empty((self.n_core, om.shape[0]), dtype=torch.float64, device="cuda")
        _check(lib().gwc_sigma_core_wac(self._ctx, om.ctypes.data, om.shape[0], int(n_core_ref), int(n_val_ref), _ptr(sig),
                                        _ptr(dec), _stream(stream)), self._ctx)
        return sig, dec

    def gdh_spectrum(self, omega, sigma_c, dh, stream=None):
        """G_dH W0 spectral function on w' + dH_n from Sigma^c on the common grid omega (CUDA tensors)."""
        import torch

        nw = int(omega.shape[0])
        a = torch.empty((self.n_core, nw), dtype=torch.float64, device="cuda")
        w = torch.empty((self.n_core, nw), dtype=torch.float64, device="cuda")
        _check(lib().gwc_gdh_spectrum(self._ctx, _ptr(omega), nw, _ptr(sigma_c), _ptr(dh), _ptr(a), _ptr(w),
                                      _stream(stream)), self._ctx)
        return a, w

    def g0w0_solutions(self, omega, sigma_c, max_roots=32, stream=None):
        """All grid solutions of the plain G0W0 QP equation per core: (roots [n_core][max_roots][2] =
        (w, Z), counts [n_core]) from Sigma^c on the ascending grid omega (CUDA tensors)."""
        import torch

        nw = int(omega.shape[0])
        roots = torch.zeros((self.n_core, max_roots, 2), dtype=torch.float64, device="cuda")
        cnt = torch.zeros((self.n_core,), dtype=torch.int32, device="cuda")
        _check(lib().gwc_g0w0_solutions(self._ctx, _ptr(omega), nw, _ptr(sigma_c), max_roots, _ptr(roots), _ptr(cnt),
                                        _stream(stream)), self._ctx)
        return roots, cnt

    # -- request mode (decoupled spectra + QP as one capturable step) -------------------------
    def request_plan(self, omega_rel, stream=None):
        om = np.ascontiguousarray(np.asarray(omega_rel, dtype=np.float64))
        self.req_n_omega = int(om.shape[0])
        _check(lib().gwc_request_plan(self._ctx, om.ctypes.data, self.req_n_omega, _stream(stream)), self._ctx)

    def request_step(self, stream=None):
        _check(lib().gwc_request_step(self._ctx, _stream(stream)), self._ctx)

    def request_results(self, stream=None, out=None):
        """Copies the last step's results into CUDA tensors (eps_qp, dh, iters, im_sigma, a, nu)."""
        import torch

        nc, nw, nt = self.n_core, self.req_n_omega, self.opt.n_t
        if out is None:
            out = (torch.empty(nc, dtype=torch.float64, device="cuda"), torch.empty(nc, dtype=torch.float64, device="cuda"),
                   torch.empty(nc, dtype=torch.int32, device="cuda"), torch.empty((nc, nw), dtype=torch.float64, device="cuda"),
                   torch.empty((nc, nt), dtype=torch.float64, device="cuda"), torch.empty(nt, dtype=torch.float64, device="cuda"))
        _check(lib().gwc_request_copy_results(self._ctx, *[_ptr(t) for t in out], _stream(stream)), self._ctx)
        return out

    def set_qp_cores(self, cores=None, stream=None):
        """Cores (indices 0..n_core-1) whose QP energies qp_solve and the request step compute; None: all."""
        if cores is None:
            _check(lib().gwc_set_qp_cores(self._ctx, None, 0, _stream(stream)), self._ctx)
            return
        c = np.ascontiguousarray(np.asarray(cores, dtype=np.int32))
        _check(lib().gwc_set_qp_cores(self._ctx, c.ctypes.data, int(c.size), _stream(stream)), self._ctx)

    def copy_out(self, dst, src, stream=None):
        """gwc_copy_out: copies the device tensor src into dst (a pinned host tensor or a device tensor)."""
        nbytes = src.numel() * src.element_size()
        assert dst.numel() * dst.element_size() == nbytes
        _check(lib().gwc_copy_out(self._ctx, _ptr(dst), _ptr(src), nbytes, _stream(stream)), self._ctx)
        return dst

    def autotune(self, stream=None) -> int:
        c = ctypes.c_int()
        _check(lib().gwc_autotune(self._ctx, _stream(stream), ctypes.byref(c)), self._ctx)
        return c.value

    def chi0_ctas(self) -> int:
        """The context's polarizability launch shape (gwc_options.chi0_ctas) after gwc_autotune."""
        o = Options()
        _check(lib().gwc_get_options(self._ctx, ctypes.byref(o)), self._ctx)
        return o.chi0_ctas

    def chi0_tile(self) -> int:
        """The context's polarizability tile shape (gwc_options.chi0_tile: 0 256 x 128 CTA-pair tiles, 1 128 x 128
        one-CTA tiles) after gwc_autotune."""
        o = Options()
        _check(lib().gwc_get_options(self._ctx, ctypes.byref(o)), self._ctx)
        return o.chi0_tile

    def sync(self, stream=None):
        _check(lib().gwc_sync(self._ctx, _stream(stream)), self._ctx)

    def sync_status(self, stream=None) -> int:
        return int(lib().gwc_sync(self._ctx, _stream(stream)))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().gwc_get_stats(self._ctx, ctypes.byref(s)), self._ctx)
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def reset_stats(self):
        _check(lib().gwc_reset_stats(self._ctx), self._ctx)

    def close(self):
        if self._ctx:
            lib().gwc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
