"""Host logic of the serving loop on the CPU: admission in arrival order by device footprint and by
free stream slots, continuous admission as requests complete, and the latency summary. The GPU
work of a request is replaced by a fake context whose completion event fires after a set time."""
import math
import time

import numpy as np
import pytest

from paper_2412_17132_gb300 import serve


class _Ev:
    def __init__(self, t_done):
        self.t_done = t_done

    def query(self):
        return time.perf_counter() >= self.t_done


class _Ctx:
    def sync_status(self, stream=None):
        return 0

    def close(self):
        pass


class _FakeServer(serve.SpectrumServer):
    """The loop of SpectrumServer.run with the GPU parts replaced: every request gets its own resident
    "context" of its footprint (no reuse), admitted while the busy footprints fit the budget or nothing
    else runs; a request 'runs' for `work[rid]` seconds; every admission records the bytes and slots in
    use at that moment."""

    def __init__(self, budget, slots, work):
        self.budget, self.slots, self.keep = budget, [None] * slots, False
        self.work, self.log, self.inflight, self.pool = work, [], {}, []

    def _acquire(self, req, input_bytes):
        busy = sum(e["bytes"] for e in self.pool if e["busy"])
        if busy + req.footprint > self.budget and any(e["busy"] for e in self.pool):
            return None
        self.pool = [e for e in self.pool if e["busy"]]  # idle ones released
        e = {"busy": True, "ctx": _Ctx(), "bytes": req.footprint, "cls": 0}
        self.pool.append(e)
        return e

    def _start(self, req, entry, stream, now):
        req.admitted = now
        live = [r for r in self.inflight.values() if not (r.finished == r.finished)]  # not finished yet
        self.log.append((req.rid, now, sum(r.footprint for r in live) + req.footprint, len(live) + 1))
        self.inflight[req.rid] = req
        return (), _Ev(time.perf_counter() + self.work[req.rid])


def _reqs(sizes, arrivals):
    return [serve.Request(rid=i, arrival=a, make=None, n_states=100, footprint=f) for i, (f, a) in enumerate(zip(sizes, arrivals))]


def test_size_classes_and_recipe():
    assert serve.size_class(100) == 150 and serve.size_class(151) == 225 and serve.size_class(1500) == 1500
    for n in (100, 149, 150, 700, 1499):
        c = serve.size_class(n)
        a, b = serve.recipe_sizes(n), serve.recipe_sizes(c)
        # every size of the request fits the class's capacity (the context's buffers grow with each)
        assert all(x <= y for x, y in zip(a, b))
        n_ov = lambda s: s[1] * (s[0] - s[1])  # noqa: E731
        assert n_ov(a) <= n_ov(b) and a[2] * n_ov(a) <= b[2] * n_ov(b)


def test_admission_respects_budget_and_slots():
    sizes = [40, 30, 50, 20, 60, 10, 30]
    srv = _FakeServer(budget=100, slots=3, work={i: 0.03 for i in range(7)})
    done = srv.run(_reqs(sizes, [0.0] * 7))
    assert sorted(r.rid for r in done) == list(range(7))
    assert [rid for rid, *_ in srv.log] == list(range(7))  # arrival order
    for _, _, used, n in srv.log:
        assert used <= 100 and n <= 3


def test_request_larger_than_the_budget_runs_alone():
    srv = _FakeServer(budget=100, slots=4, work={0: 0.02, 1: 0.02, 2: 0.02})
    done = srv.run(_reqs([30, 250, 30], [0.0, 0.0, 0.0]))
    assert len(done) == 3
    big = next(r for r in done if r.rid == 1)
    others = [r for r in done if r.rid != 1]
    # the oversize request starts only after the one before it finished, and the next waits for it
    assert big.admitted >= others[0].finished
    assert others[1].admitted >= big.finished


def test_continuous_admission_overlaps_requests():
    # a late arrival joins while an earlier long request is still running
    srv = _FakeServer(budget=100, slots=2, work={0: 0.2, 1: 0.02})
    done = srv.run(_reqs([40, 40], [0.0, 0.05]))
    r0, r1 = sorted(done, key=lambda r: r.rid)
    assert r1.admitted < r0.finished
    assert r1.finished < r0.finished


def test_poisson_arrivals_and_sizes():
    a = serve.poisson_arrivals(4000, 20.0, seed=0)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 4000 - 1 / 20.0) < 0.005  # mean inter-arrival 50 ms
    n = np.array([serve.serving_size(i) for i in range(2000)])
    assert n.min() >= 100 and n.max() <= 1500
    assert abs(np.median(np.log(n)) - 0.5 * (math.log(100) + math.log(1500))) < 0.1  # log-uniform


def test_summary_percentiles():
    done = _reqs([1] * 4, [0.0, 1.0, 2.0, 3.0])
    for r, lat in zip(done, (1.0, 2.0, 3.0, 10.0)):
        r.finished = r.arrival + lat
        r.eps_qp = np.zeros(2)
    s = serve.summarize(done, makespan=13.0)
    assert s["completed"] == 4 and s["failed"] == 0
    assert s["p50_s"] == pytest.approx(2.5)
    assert s["requests_per_s"] == pytest.approx(4 / 13.0) and s["spectra_per_s"] == pytest.approx(8 / 13.0)
