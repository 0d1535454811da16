"""Serving loop: spectrum requests of uneven size admitted by HBM footprint and run concurrently.

A request is one molecule (orbital energies and RI coefficients) for which the caller wants the
decoupled GW+C spectra of all its 1s cores and their QP energies (the library's request mode,
`gwc_request_plan` / `gwc_request_step`). The server keeps a set of requests in flight, each on its
own CUDA stream with pinned host buffers for its results.

Contexts are resident and reused: requests fall into size classes (by N_states), and a context is
created once per class with the capacity of the class's largest molecule (`gwc_create` with sizes
only); every later request of that class, or of a smaller one, is loaded into an idle context with
`gwc_load` (its O^P_mn copied into the resident buffers, the dielectric workspace and W-table buffers
reused, no device allocation by the library), and the context goes back to the pool when the request
completes. A request is admitted in arrival order as soon as (a) a stream slot is free and (b) an
idle context fits it or a new one fits the HBM budget next to the contexts already resident (idle
contexts of other classes are released to make room); completed requests free their slot at once, so
new arrivals join while others are still on the GPU (continuous batching). Latency is measured from
arrival to the moment the results are in host memory.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import time
from collections import deque
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                      # seconds after the start of the run
    make: Callable[[], object]          # returns a synth.Molecule with device (or host) arrays
    n_states: int = 0
    footprint: int = 0
    admitted: float = math.nan
    finished: float = math.nan
    eps_qp: Optional[np.ndarray] = None
    im_sigma: Optional[np.ndarray] = None
    spectrum: Optional[np.ndarray] = None
    status: int = 0


def footprint_bytes(gwc, mol, n_omega, prec, batch, n_t):
    """Device bytes of one request: the context's workspace plus the caller-side inputs."""
    core = np.ascontiguousarray(np.asarray(mol.core_idx, dtype=np.int32))
    eps = np.ascontiguousarray(mol.eps)
    n_ov = mol.n_occ * (mol.n_states - mol.n_occ)
    sysd = gwc.System(mol.n_states, mol.n_occ, mol.n_aux, mol.n_core, core.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      eps.ctypes.data, 1, 1, None, math.nan, 1)
    opt = gwc.default_options()
    opt.prec, opt.batch, opt.n_t = gwc.PREC[prec], batch, n_t
    b = ctypes.c_size_t()
    gwc._check(gwc.lib().gwc_workspace_bytes(ctypes.byref(sysd), ctypes.byref(opt), n_omega, ctypes.byref(b)))
    return int(b.value) + 8 * (mol.n_aux * n_ov + mol.n_states * mol.n_core * mol.n_aux)


def recipe_sizes(n_states):
    """(n_states, n_occ, n_aux, n_core) of the serving recipe for a molecule of n_states orbitals."""
    n_occ = max(2, int(round(n_states / 18)))
    return n_states, n_occ, int(round(3.5 * n_states)), max(1, int(round(0.3 * n_occ)))


# size classes by N_states (upper bounds, log-spaced over the recipe's 100..1500)
SIZE_CLASSES = (150, 225, 340, 510, 770, 1150, 1500)


def size_class(n_states, classes=SIZE_CLASSES):
    for c in classes:
        if n_states <= c:
            return c
    return n_states


class SpectrumServer:
    def __init__(self, omega_rel, budget_bytes, slots=8, prec="bf16x3", qp_mode="hedin", batch=32, n_t=1 << 16,
                 t_max=2000.0, eta=1e-3, keep_results=True, classes=SIZE_CLASSES):
        import torch

        from paper_2412_17132_gb300 import gwc

        self.gwc = gwc
        self.torch = torch
        self.omega_rel = np.ascontiguousarray(np.asarray(omega_rel, dtype=np.float64))
        self.budget = int(budget_bytes)
        self.slots = [torch.cuda.Stream() for _ in range(slots)]
        self.prec, self.qp_mode, self.batch = prec, qp_mode, batch
        self.n_t, self.t_max, self.eta = n_t, t_max, eta
        self.keep = keep_results
        self.classes = tuple(classes)
        self.pool = []  # resident contexts: dicts with "cls", "ctx", "bytes", "busy"
        self.created = 0
        self.reused = 0

    def resident_bytes(self):
        return sum(e["bytes"] for e in self.pool)

    def _class_bytes(self, cls):
        n, n_occ, n_aux, n_core = recipe_sizes(cls)

        class _M:
            pass

        m = _M()
        m.n_states, m.n_occ, m.n_aux, m.n_core = n, n_occ, n_aux, n_core
        m.core_idx = np.arange(n_core, dtype=np.int32)
        m.eps = np.linspace(-10.4, 3.0, n)
        return footprint_bytes(self.gwc, m, len(self.omega_rel), self.prec, self.batch, self.n_t) - \
            8 * (n_aux * n_occ * (n - n_occ) + n * n_core * n_aux)

    def _acquire(self, req, input_bytes):
        """An idle resident context that fits the request (the smallest class that does), or a new one of the
        request's class if the budget allows (releasing idle contexts of other classes first); None if the
        request has to wait for memory."""
        cls = size_class(req.n_states, self.classes)
        idle = [e for e in self.pool if not e["busy"] and e["cls"] >= cls]
        if idle:
            e = min(idle, key=lambda e: e["cls"])
            if self.resident_bytes() + input_bytes <= self.budget or not any(x["busy"] for x in self.pool):
                e["busy"] = True
                self.reused += 1
                return e
        need = self._class_bytes(cls)
        while self.resident_bytes() + need + input_bytes > self.budget:
            free = [e for e in self.pool if not e["busy"]]
            if not free:
                break
            victim = max(free, key=lambda e: e["bytes"])
            victim["ctx"].close()
            self.pool.remove(victim)
        if self.resident_bytes() + need + input_bytes > self.budget and any(e["busy"] for e in self.pool):
            return None
        n, n_occ, n_aux, n_core = recipe_sizes(cls)
        ctx = self.gwc.Context.with_capacity(n, n_occ, n_aux, n_core, prec=self.prec, qp_mode=self.qp_mode,
                                             batch=self.batch, n_t=self.n_t, t_max=self.t_max, eta=self.eta)
        e = {"cls": cls, "ctx": ctx, "bytes": need, "busy": True}
        self.pool.append(e)
        self.created += 1
        return e

    def _start(self, req, entry, stream, now):
        torch = self.torch
        ctx = entry["ctx"]
        with torch.cuda.stream(stream):
            mol = req.make()
            req.n_states = mol.n_states
            eps = mol.eps if isinstance(mol.o_ov, np.ndarray) else torch.as_tensor(mol.eps, device="cuda")
            try:
                ctx.load(eps, mol.o_ov, mol.o_core, core_idx=mol.core_idx, n_occ=mol.n_occ, stream=stream)
            except self.gwc.GwcError:
                # sizes outside the class recipe: a context of this molecule's own sizes takes the slot
                ctx.close()
                ctx = self.gwc.Context(eps, mol.n_occ, mol.core_idx, mol.o_ov, mol.o_core, prec=self.prec,
                                       qp_mode=self.qp_mode, batch=self.batch, n_t=self.n_t, t_max=self.t_max,
                                       eta=self.eta, n_im=mol.n_im, xi0=mol.xi0, stream=stream)
                entry["ctx"] = ctx
            del mol, eps  # the context holds its own copies; the caller-side inputs can go
            ctx.request_plan(self.omega_rel, stream=stream)
            ctx.request_step(stream=stream)
            nc, nw = ctx.n_core, len(self.omega_rel)
            host = (torch.empty(nc, dtype=torch.float64).pin_memory(), torch.empty((nc, nw), dtype=torch.float64).pin_memory(),
                    torch.empty((nc, self.n_t), dtype=torch.float64).pin_memory())
            self.gwc._check(self.gwc.lib().gwc_request_copy_results(ctx._ctx, host[0].data_ptr(), None, None, host[1].data_ptr(),
                                                                     host[2].data_ptr(), None, stream.cuda_stream), ctx._ctx)
            ev = torch.cuda.Event()
            ev.record(stream)
        req.admitted = now
        return host, ev

    def close(self):
        for e in self.pool:
            e["ctx"].close()
        self.pool = []

    def run(self, requests: List[Request], time_limit: float = 3600.0):
        """Serves the requests (arrival times relative to the start); returns them completed."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        inflight = []  # (req, entry, host, ev, slot)
        free_slots = list(range(len(self.slots)))
        t0 = time.perf_counter()
        done = []
        while pending or inflight:
            now = time.perf_counter() - t0
            if now > time_limit:
                break
            progressed = False
            # completions
            for item in list(inflight):
                req, entry, host, ev, slot = item
                if ev.query():
                    req.status = entry["ctx"].sync_status(stream=self.slots[slot])
                    req.finished = time.perf_counter() - t0
                    if self.keep:
                        req.eps_qp = host[0].numpy().copy()
                        req.im_sigma = host[1].numpy().copy()
                        req.spectrum = host[2].numpy().copy()
                    entry["busy"] = False  # back to the pool, resident
                    inflight.remove(item)
                    free_slots.append(slot)
                    done.append(req)
                    progressed = True
            # admissions (arrival order; a request that does not fit waits for memory)
            while pending and pending[0].arrival <= now and free_slots:
                req = pending[0]
                if req.n_states == 0:
                    req.n_states = self._size(req)
                n, n_occ, n_aux, n_core = recipe_sizes(req.n_states)
                input_bytes = 8 * (n_aux * n_occ * (n - n_occ) + n * n_core * n_aux)
                entry = self._acquire(req, input_bytes)
                if entry is None:
                    break
                req.footprint = entry["bytes"]
                pending.popleft()
                slot = free_slots.pop(0)
                host, ev = self._start(req, entry, self.slots[slot], time.perf_counter() - t0)
                inflight.append((req, entry, host, ev, slot))
                progressed = True
            if not progressed:
                time.sleep(0.0005)
        return done

    @staticmethod
    def _size(req):
        # the request's size from the generator's recipe, without generating the arrays
        return serving_size(req.rid)


def poisson_arrivals(n, rate, seed=0):
    """Arrival times of n requests of a Poisson stream with the given mean rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def serving_size(request_id: int) -> int:
    """N_states of request `request_id` (log-uniform on [100, 1500], seed = request id)."""
    rng = np.random.default_rng(request_id)
    return int(round(math.exp(rng.uniform(math.log(100), math.log(1500)))))


def summarize(done: List[Request], makespan: float):
    lat = np.array([r.finished - r.arrival for r in done])
    n_spectra = sum(int(r.eps_qp.shape[0]) if r.eps_qp is not None else 0 for r in done)
    return {
        "completed": len(done),
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "requests_per_s": len(done) / makespan if makespan > 0 else None,
        "spectra_per_s": n_spectra / makespan if makespan > 0 else None,
        "failed": int(sum(1 for r in done if r.status != 0)),
    }
