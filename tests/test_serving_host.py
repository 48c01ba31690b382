"""Host logic of the serving loop, driven without a GPU by a stand-in solve: admission by
device footprint within the budget, at most `lanes` requests in flight, no request started
before it arrives, every request answered once, the latency summary, and the precision policy."""
import threading
import time

import numpy as np
import pytest

from paper_2509_13224_gb300 import FP64, MIXED_FP32
from paper_2509_13224_gb300.serving import Request, Server, footprint_bytes, summarize, synthetic_stream


class FakeSolve:
    """Sleeps a few ms per request and records what the scheduler had admitted meanwhile."""

    def __init__(self):
        self.srv = None
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.in_use_seen = []
        self.starts = {}

    def __call__(self, req, t0):
        start = time.perf_counter() - t0
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.in_use_seen.append(self.srv.in_use)
            self.starts[req.rid] = start
        time.sleep(0.002 + 0.004 * (req.n % 5) / 4)
        with self.lock:
            self.running -= 1
        end = time.perf_counter() - t0
        return {"rid": req.rid, "n": req.n, "p": req.p, "dofs": req.n ** 3, "arrival": req.arrival,
                "start": start, "end": end, "latency": end - req.arrival, "status": 0}


@pytest.mark.parametrize("lanes,budget_factor", [(4, 2.0), (3, 100.0), (1, 1.0)])
def test_admission_respects_lanes_and_budget(lanes, budget_factor):
    reqs = synthetic_stream(24, rate_hz=800.0, seed=5, n_lo=16, n_hi=64)
    need = [footprint_bytes(r.n, r.p) for r in reqs]
    budget = int(budget_factor * max(need))
    fake = FakeSolve()
    srv = Server(lanes=lanes, budget_bytes=budget, runner=fake)
    fake.srv = srv
    records, summ = srv.serve(reqs)
    assert sorted(r["rid"] for r in records) == list(range(len(reqs)))
    assert summ["ok"] == len(reqs) and summ["requests"] == len(reqs)
    assert fake.max_running <= lanes
    assert max(fake.in_use_seen) <= max(budget, max(need))
    assert srv.in_use == 0
    for r in reqs:
        assert fake.starts[r.rid] >= r.arrival - 1e-3
    if budget_factor < 2.5:
        # the budget admits at most two of the largest requests at once
        assert fake.max_running <= max(2, int(budget // min(need)))


def test_oversized_request_runs_alone():
    """A request larger than the whole budget is admitted once nothing else is in use."""
    reqs = [Request(k, {"kind": "box", "lx": 1, "ly": 1, "lz": 1}, 2, 8 + 40 * (k == 1), 1e-8,
                    arrival=0.0005 * k) for k in range(3)]
    budget = footprint_bytes(8, 2) + 1
    fake = FakeSolve()
    srv = Server(lanes=3, budget_bytes=budget, runner=fake)
    fake.srv = srv
    records, summ = srv.serve(reqs)
    assert summ["ok"] == 3
    assert fake.max_running == 1
    assert max(fake.in_use_seen) == footprint_bytes(48, 2)


def test_summary_percentiles_and_throughput():
    lat = np.arange(1, 101) * 1e-3
    recs = [{"status": 0, "latency": float(l), "dofs": 1000, "arrival": 0.01 * k, "end": 0.01 * k + float(l)}
            for k, l in enumerate(lat)]
    recs.append({"status": -4, "latency": 5.0, "dofs": 10 ** 9, "arrival": 0.0, "end": 9.0})
    s = summarize(recs, wall=2.0)
    assert s["requests"] == 101 and s["ok"] == 100
    assert abs(s["p50_ms"] - 50.5) < 1e-9 and abs(s["p99_ms"] - 99.01) < 1e-9
    span = max(r["end"] for r in recs[:100]) - min(r["arrival"] for r in recs[:100])
    assert abs(s["dofs_per_s"] - 100 * 1000 / span) < 1e-6


def test_precision_policy():
    srv = Server(lanes=1, budget_bytes=1, runner=lambda req, t0: None)
    loose = Request(0, {}, 2, 8, 1e-6)
    tight = Request(1, {}, 2, 8, 1e-8)
    forced = Request(2, {}, 2, 8, 1e-6, precision=FP64)
    assert srv._precision(loose) == MIXED_FP32 and srv._precision(tight) == FP64
    assert srv._precision(forced) == FP64
    srv.policy = "fp64"
    assert srv._precision(loose) == FP64
    srv.policy = "mixed"
    assert srv._precision(tight) == MIXED_FP32
