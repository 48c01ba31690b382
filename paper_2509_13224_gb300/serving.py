"""Serving loop for TT-IGA Poisson solves on one GPU (continuous batching).

Requests (geometry, degree, resolution, tolerance) arrive open-loop.  A
request is admitted as soon as a lane is free and its estimated device
footprint fits the memory budget; admitted requests run concurrently, one per
lane, each lane a host thread with its own library context and CUDA stream,
so their kernels overlap on the device.  Requests that arrive while others
run are admitted as lanes and memory free up.  Every request records its
arrival, start and finish times; the session reports p50/p99 latency and
DOFs/s.  Each solve's arithmetic is independent of the others (own context,
deterministic reductions), so a result is the same alone and in the mix.

All computation happens in libtt_iga.so; this module only schedules.
"""
import math
import queue
import threading
import time

import numpy as np

from . import (FP64, MIXED_FP32, MIXED_TF32, geom_desc, rhs_desc, solve_opts, tt_iga_assemble, tt_iga_ctx_create,
               tt_iga_ctx_destroy, tt_iga_ctx_set_sm_limit, tt_iga_geom_destroy, tt_iga_geometry, tt_iga_import_cores,
               tt_iga_l2_diff,
               tt_iga_solution_cores, tt_iga_solution_destroy, tt_iga_solve, tt_iga_system_destroy)


# The "auto" policy solves requests with a tolerance at or above this in mixed precision
# and tighter ones in FP64.
AUTO_MIXED_MIN_TOL = 1e-7


def footprint_bytes(n, p, rank=48, op_rank=24, rhs_rank=16):
    """Conservative device footprint of one solve: TT cores of K, F and u, AMEn interfaces,
    the fused-PCG work vectors and the cross fibre matrices (FP64 unless noted)."""
    m = n - 2
    b = 2 * p + 1
    q = (n - p) * (p + 1)
    k_cores = 3 * op_rank * op_rank * m * b
    f_cores = 3 * rhs_rank * rhs_rank * m
    u_cores = 3 * rank * rank * m
    local = rank * rank * m
    pcg = 5 * local + 2 * local * op_rank       # vectors + T1/T2
    cross = 6 * q * 96 + 64 * q * 96            # fibre matrices + QR work
    return 8 * (k_cores + f_cores + u_cores + pcg + cross) * 2 + (16 << 20)


class Request:
    def __init__(self, rid, geometry, p, n, tol, modes=(), arrival=0.0, precision=None, seed=0):
        self.rid, self.geometry, self.p, self.n, self.tol = rid, geometry, int(p), int(n), float(tol)
        self.modes = list(modes)
        self.arrival = float(arrival)
        self.precision = precision
        self.seed = int(seed)
        self.record = None


class Server:
    """lanes: concurrent solves; budget_bytes: device memory allowed for admitted requests."""

    def __init__(self, device=0, lanes=4, budget_bytes=None, precision_policy="auto", keep_cores=False,
                 cross_tol=1e-10, round_tol=1e-12, runner=None, mixed_precision=MIXED_FP32, sm_per_lane=-1):
        """runner: None (each request is solved by libtt_iga.so on the lane's context) or a
        callable runner(request, t0) -> record with the keys of _run_one, for driving the
        scheduler without a GPU.  mixed_precision: the precision mode of mixed requests
        (MIXED_FP32 or MIXED_TF32).  sm_per_lane: SM budget of each lane's local PCG kernels
        (-1: the SM count divided by the lanes, so concurrent requests' solves run side by side;
        0: the whole GPU)."""
        self.device = device
        self.lanes = int(lanes)
        self.runner = runner
        if budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(0.8 * free)
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.policy = precision_policy
        self.mixed = mixed_precision
        self.keep_cores = keep_cores
        self.cross_tol, self.round_tol = cross_tol, round_tol
        self.sm_per_lane = int(sm_per_lane)
        self._cv = threading.Condition()

    def _precision(self, req):
        if req.precision is not None:
            return req.precision
        if self.policy == "fp64":
            return FP64
        if self.policy == "mixed":
            return self.mixed
        return self.mixed if req.tol >= AUTO_MIXED_MIN_TOL else FP64

    def _run_one(self, ctx, req, t0):
        rec = {"rid": req.rid, "n": req.n, "p": req.p, "tol": req.tol, "dofs": req.n ** 3,
               "arrival": req.arrival}
        prec = self._precision(req)
        rec["precision"] = {FP64: "fp64", MIXED_FP32: "mixed_fp32", MIXED_TF32: "mixed_tf32"}[prec]
        rec["start"] = time.perf_counter() - t0
        g = s = u = None
        try:
            g = tt_iga_geometry(ctx, geom_desc(req.geometry, req.p, req.n, cross_tol=self.cross_tol, seed=req.seed))
            s = tt_iga_assemble(ctx, g, [rhs_desc(req.modes)], round_tol=self.round_tol)
            u, st = tt_iga_solve(ctx, s, solve_opts(tol=req.tol, precision=prec), allow_not_converged=True)
            rec.update({"status": 0 if st["converged"] else -4, "rel_residual": st["rel_residual"],
                        "ranks": st["ranks"], "sweeps": st["sweeps"]})
            if self.keep_cores:
                rec["cores"] = [c.copy() for c in tt_iga_solution_cores(ctx, u)]
        except Exception as exc:  # a failed request is reported, the server keeps running
            rec.update({"status": getattr(exc, "code", -3), "error": str(exc)})
        finally:
            if u is not None:
                tt_iga_solution_destroy(u)
            if s is not None:
                tt_iga_system_destroy(s)
            if g is not None:
                tt_iga_geom_destroy(g)
        rec["end"] = time.perf_counter() - t0
        rec["latency"] = rec["end"] - rec["arrival"]
        return rec

    def serve(self, requests, realtime=True):
        """Run an open-loop session; requests carry arrival times (s from the session start).
        Returns (records in completion order, summary dict)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        arrived = queue.Queue()
        records = []
        lock = threading.Lock()
        t0 = time.perf_counter()
        done_arriving = threading.Event()

        def arrivals():
            for r in pending:
                if realtime:
                    dt = r.arrival - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                arrived.put(r)
            done_arriving.set()

        waiting = []  # arrived but not admitted, FIFO

        def admit():
            """Next admissible request (FIFO, footprint within budget), or None."""
            with self._cv:
                while True:
                    while True:
                        try:
                            waiting.append(arrived.get_nowait())
                        except queue.Empty:
                            break
                    if waiting:
                        need = footprint_bytes(waiting[0].n, waiting[0].p)
                        if self.in_use + need <= self.budget or self.in_use == 0:
                            req = waiting.pop(0)
                            self.in_use += need
                            return req, need
                    elif done_arriving.is_set() and arrived.empty():
                        return None, 0
                    self._cv.wait(timeout=0.002)

        def lane():
            ctx = None
            if self.runner is None:
                import torch
                torch.cuda.set_device(self.device)
                ctx = tt_iga_ctx_create(None, self.device)
                share = self.sm_per_lane
                if share < 0:
                    sms = torch.cuda.get_device_properties(self.device).multi_processor_count
                    share = sms // self.lanes if self.lanes > 1 else 0
                tt_iga_ctx_set_sm_limit(ctx, share)
            try:
                while True:
                    req, need = admit()
                    if req is None:
                        return
                    rec = self._run_one(ctx, req, t0) if self.runner is None else self.runner(req, t0)
                    with self._cv:
                        self.in_use -= need
                        self._cv.notify_all()
                    with lock:
                        records.append(rec)
            finally:
                if ctx is not None:
                    tt_iga_ctx_destroy(ctx)

        ta = threading.Thread(target=arrivals, daemon=True)
        ta.start()
        threads = [threading.Thread(target=lane, daemon=True) for _ in range(self.lanes)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        ta.join()
        wall = time.perf_counter() - t0
        return records, summarize(records, wall)


def summarize(records, wall):
    ok = [r for r in records if r.get("status") == 0]
    lat = np.array([r["latency"] for r in ok]) if ok else np.array([math.nan])
    dofs = sum(r["dofs"] for r in ok)
    span = (max(r["end"] for r in ok) - min(r["arrival"] for r in ok)) if ok else math.nan
    return {"requests": len(records), "ok": len(ok), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "dofs_per_s": dofs / span if ok else 0.0,
            "wall_s": wall}


def summarize_by(records, key):
    """summarize() per value of records[key] (e.g. the requested tolerance), over the session's wall."""
    groups = {}
    for r in records:
        groups.setdefault(r.get(key), []).append(r)
    out = {}
    for k, recs in sorted(groups.items(), key=lambda kv: str(kv[0])):
        ok = [r for r in recs if r.get("status") == 0]
        lat = np.array([r["latency"] for r in ok]) if ok else np.array([math.nan])
        span = (max(r["end"] for r in ok) - min(r["arrival"] for r in ok)) if ok else math.nan
        out[str(k)] = {"requests": len(recs), "ok": len(ok), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                       "p99_ms": float(np.percentile(lat, 99) * 1e3),
                       "dofs_per_s": sum(r["dofs"] for r in ok) / span if ok else 0.0}
    return out


def accuracy_vs(requests, records, reference, device=0, cross_tol=1e-10, round_tol=1e-12):
    """Relative L2 difference of each request's solution in `records` from its solution in
    `reference` (both kept with keep_cores): the request's system is rebuilt, both solutions are
    imported from their cores and compared on the mapped domain (tt_iga_l2_diff).  Returns
    {"per_request": {rid: diff}, "max_by_tol": ..., "median_by_tol": ...}."""
    by_id = {r.rid: r for r in requests}
    ref = {r["rid"]: r for r in reference if r.get("status") == 0 and "cores" in r}
    ctx = tt_iga_ctx_create(None, device)
    per = {}
    try:
        for rec in records:
            rid = rec["rid"]
            if rec.get("status") != 0 or "cores" not in rec or rid not in ref:
                continue
            req = by_id[rid]
            g = tt_iga_geometry(ctx, geom_desc(req.geometry, req.p, req.n, cross_tol=cross_tol, seed=req.seed))
            s = tt_iga_assemble(ctx, g, [rhs_desc(req.modes)], round_tol=round_tol)
            u = tt_iga_import_cores(ctx, s, rec["cores"])
            v = tt_iga_import_cores(ctx, s, ref[rid]["cores"])
            try:
                per[rid] = tt_iga_l2_diff(ctx, g, u, v)
            finally:
                tt_iga_solution_destroy(u)
                tt_iga_solution_destroy(v)
                tt_iga_system_destroy(s)
                tt_iga_geom_destroy(g)
    finally:
        tt_iga_ctx_destroy(ctx)
    by_tol = {}
    for rid, e in per.items():
        by_tol.setdefault(str(by_id[rid].tol), []).append(e)
    return {"per_request": per, "compared": len(per),
            "max_by_tol": {k: float(max(v)) for k, v in by_tol.items()},
            "median_by_tol": {k: float(np.median(v)) for k, v in by_tol.items()}}


def synthetic_stream(count, rate_hz, seed, n_lo=32, n_hi=1024, tols=(1e-6, 1e-8)):
    """Open-loop request stream with geometry drawn as in the batched workload."""
    import synthetic
    times = synthetic.poisson_arrivals(rate_hz, count, seed)
    reqs = []
    g = synthetic.rng(seed + 1)
    for k in range(count):
        inst = synthetic.random_instance(seed * 100_000 + k, n_lo=n_lo, n_hi=n_hi)
        tol = float(tols[int(g.integers(0, len(tols)))])
        reqs.append(Request(k, inst["geometry"], inst["p"], inst["n"], tol, modes=inst["rhs"][0],
                            arrival=float(times[k]), seed=inst["seed"]))
    return reqs
