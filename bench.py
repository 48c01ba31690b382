#!/usr/bin/env python3
"""Benchmark of the TT-IGA hot path on GB300: DOFs solved per second.

One step = the whole hot path on one synthetic problem: TT-cross of the
geometry coefficients, per-direction contraction into the TT stiffness and
load, TT rounding, Dirichlet restriction and the AMEn solve to relative
residual 1e-8 (exact, TT arithmetic).  The default workload is the
non-separable twisted and swollen quarter annulus (radii 1..2, height 1, twist
0.8 z, swell 1 + 0.2 sin(pi z)) at degree p = 3 with n = 512 B-splines per
direction (134,217,728 DOFs), coefficient cross and rounding at 1e-10, and the
manufactured bubble solution.  DOFs per step = n^3.  The line's `value` is the
plain FP64 path; `mixed` is the mixed-precision path on the same workload with
its relative L2 difference from the FP64 solution; the quarter cylinder at
p = 3, n = 128 and the ring, NURBS, batched and serving measurements are side
entries.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own replica (independent problems, no
collective on the data path); rank 0 prints one JSON line.  `--impl
reference` times the FP64 CPU oracle (full-grid IGA + Jacobi PCG) on a bounded
sample of the same workload on the host cores.
"""
import argparse
import json
import os
import resource
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Hardware work queues of the process (read when CUDA starts): the batched and serving measurements
# run up to dozens of lanes, each on its own stream, and 8 queues (the default) would make
# unrelated streams wait on each other.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import synthetic  # noqa: E402

WORKLOAD = "twisted_annulus_p3_n512"
SIDE_WORKLOAD = "quarter_cylinder_p3_n128"
METRIC = "DOFs solved/s at 1e-8 rel. residual, mixed vs FP64; serving p50/p99 latency"
TOL = 1e-8
# Inexact AMEn local solves on the headline workload (tt_iga_solve_opts.local_rtol): each local system
# is solved to this factor of its initial residual when that is above the tolerance's bound; the
# exact global residual still decides convergence.  The library default (exact local solves) is
# measured beside it.
HEADLINE_LOCAL_RTOL = 1e-3
FP64_ALU_PEAK_TFLOPS = 1.258  # 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s)
FP32_ALU_PEAK_TFLOPS = 80.54  # 152 SMs x 128 FP32 FMA/clk x 2 FLOP x 2.07 GHz

# DRAM bytes (read + write) per launch of the timed kernel, mean over the launches of one
# step, from one ncu capture whose summary is committed with the profiles, keyed by
# (workload, precision).  Valid only for the sources they were taken from: reported as null
# once those change.
PCG_TRAFFIC_SOURCES = ("pcg_fused_impl.cuh", "pcg_fused.cuh", "bbprec.cu", "bbprec.cuh")
PCG_TRAFFIC = {  # (workload, "fp64" | "mixed") -> (bytes per launch, sha256 of the sources)
    ("twisted_annulus_p3_n512", "fp64"):
        (1360555, "b161e4c9238ae2a7df6f34ce9cabe1ee24a5d5e8300fa07700314d9e71a0043b"),
    ("twisted_annulus_p3_n512", "mixed"):
        (1063125, "b161e4c9238ae2a7df6f34ce9cabe1ee24a5d5e8300fa07700314d9e71a0043b"),
}


def pcg_traffic(workload, precision):
    import hashlib
    rec = PCG_TRAFFIC.get((workload, precision))
    if rec is None:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2509_13224_gb300", "csrc")
    for f in PCG_TRAFFIC_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return rec[0] if h.hexdigest() == rec[1] else None
REFERENCE_SAMPLE_N = 16


def fma_peaks(device):
    """Measured (FP64, FP32) FMA throughput in TFLOP/s from the benchmark's probe library
    (fma_probe.cu), or (None, None) if the probe fails."""
    import ctypes
    from paper_2509_13224_gb300.build import build_probe
    lib = ctypes.CDLL(build_probe())
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib.fma_probe_tflops(int(device), ctypes.byref(a), ctypes.byref(b))
    return (a.value, b.value) if rc == 0 else (None, None)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--profile-family", type=int, default=6,
                    help="kernel family timed live for the roofline (6: fused PCG of the AMEn local solves)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--mixed-precision", choices=["fp32", "tf32"], default="fp32",
                    help="inner precision of the mixed arm")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the side measurements (quarter cylinder n=128, ring, NURBS)")
    ap.add_argument("--batch-instances", type=int, default=64, help="instances in the batched measurement (0 skips)")
    ap.add_argument("--serve-requests", type=int, default=160, help="requests in the serving session (0 skips)")
    ap.add_argument("--serve-rate", type=float, default=12.0, help="open-loop arrival rate (requests/s)")
    ap.add_argument("--serve-nmax", type=int, default=1024, help="largest n per direction in the serving stream")
    return ap.parse_args()


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_step(n, p, geo):
    """Full-grid FP64 IGA assembly + Jacobi PCG to relative residual TOL (the oracle as it stands)."""
    from oracle.geometry import Annulus
    from oracle.iga import Space1D, assemble, pcg, restrict
    from oracle.manufactured import Manufactured
    og = Annulus(geo["r_in"], geo["r_out"], geo["height"], geo["twist"], geo["swell"])
    sp = [Space1D(n, p)] * 3
    Kst, F = assemble(sp, og, Manufactured(og))
    Ki, Fi = restrict(Kst, F)
    x, it, rr = pcg(Ki, Fi, (p, p, p), tol=TOL)
    return rr


def timed_oracle(n, p, geo):
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    oracle_step(n, p, geo)
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return wall, max(1.0, cpu / wall)


def cpu_baseline(wl):
    n, p = 24, wl["p"]
    wall, cores = timed_oracle(n, p, wl["geometry"])
    return {"value": n ** 3 / wall, "unit": "DOFs/s", "cores": round(cores, 2), "kind": "oracle",
            "sample": f"one full-grid FP64 assemble + Jacobi-PCG solve to 1e-8 of the same geometry at p={p}, "
                      f"n={n} ({n ** 3} DOFs), {wall:.1f} s on the host"}


def run_reference(args, rank, world):
    wl = synthetic.WORKLOADS[args.workload]
    if rank != 0:
        return
    n, p = REFERENCE_SAMPLE_N, wl["p"]
    for _ in range(args.warmup):
        oracle_step(n, p, wl["geometry"])
    walls, cores = [], []
    for _ in range(args.steps):
        w, cr = timed_oracle(n, p, wl["geometry"])
        walls.append(w)
        cores.append(cr)
    t = statistics.mean(walls)
    value = n ** 3 / t
    line = {"metric": METRIC, "value": value, "unit": "DOFs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "p": p, "n": wl["n"], "tol": TOL,
                       "sample_n": n, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "DOFs/s", "cores": round(statistics.mean(cores), 2),
                             "kind": "oracle",
                             "sample": f"per step: full-grid FP64 assemble + Jacobi-PCG to 1e-8 at p={p}, "
                                       f"n={n} ({n ** 3} DOFs)"},
            "e2e": {"value": value, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import numpy as np
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_13224_gb300 as tt

    wl = synthetic.WORKLOADS[args.workload]
    n, p = wl["n"], wl["p"]
    dofs = n ** 3
    mixed_prec = tt.MIXED_TF32 if args.mixed_precision == "tf32" else tt.MIXED_FP32
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(wl)

    stream = torch.cuda.Stream()
    ctx = tt.tt_iga_ctx_create(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    fp64_meas, fp32_meas = fma_peaks(local)

    def release(hs):
        g, s, u = hs
        tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)

    def make_step(w, seed, local_rtol=0.0):
        gd = tt.geom_desc(w["geometry"], w["p"], w["n"], cross_tol=w["cross_tol"], seed=seed)
        rh = [tt.rhs_desc(w["modes"])]

        def step(precision, info=None, marks=None):
            g = tt.tt_iga_geometry(ctx, gd)
            if marks is not None:
                marks[0].record(stream)
            s = tt.tt_iga_assemble(ctx, g, rh, round_tol=w["round_tol"])
            if marks is not None:
                marks[1].record(stream)
            u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=TOL, precision=precision, local_rtol=local_rtol))
            if info is not None:
                info.update(st)
                info["op_ranks"] = tt.tt_iga_system_info(s)["op_ranks"]
            return g, s, u
        return step, gd, rh

    def timed(step, precision, k, w, profile=False, keep_last=False):
        """W untimed steps, then K steps timed by CUDA events on the library stream with the L2
        flushed before each; returns (mean ms, info, launches, profile record, clocks, last handles)."""
        for _ in range(w):
            release(step(precision))
        info, times, phases = {}, [], []
        barrier(world)
        torch.cuda.synchronize()
        if profile:
            tt.tt_iga_profile_enable(ctx, args.profile_family)
        clocks = ClockSampler(local)
        clocks.start()
        l0 = tt.tt_iga_launch_count()
        last = None
        for i in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            marks = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            e0.record(stream)
            hs = step(precision, info, marks)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            phases.append((e0.elapsed_time(marks[0]), marks[0].elapsed_time(marks[1]), marks[1].elapsed_time(e1)))
            if keep_last and i == k - 1:
                last = hs
            else:
                release(hs)
        launches = tt.tt_iga_launch_count() - l0
        clk = clocks.stop()
        info["phases_ms"] = {name: statistics.mean(ph[i] for ph in phases)
                             for i, name in enumerate(("geometry", "assembly", "solve"))}
        prof = tt.tt_iga_profile_read(ctx) if profile else None
        if profile:
            tt.tt_iga_profile_enable(ctx, 0)
        torch.cuda.synchronize()
        barrier(world)
        return statistics.mean(times), info, launches, prof, clk, last

    def roofline(prof, ms_step, steps, precision_name):
        if prof is None or prof[1] <= 0:
            return None
        ms_k, n_k, flops_k = prof
        achieved = flops_k / n_k / (ms_k / n_k / 1e3) / 1e12
        fp64 = precision_name == "fp64"
        peak = FP64_ALU_PEAK_TFLOPS if fp64 else FP32_ALU_PEAK_TFLOPS
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": pcg_traffic(args.workload, precision_name) if args.profile_family == 6 else None,
                "kernel": ("k_pcg_fused<double> (AMEn local PCG, one launch per solve)" if fp64 else
                           "k_pcg_fused<float> (mixed: FP32 local PCG inside FP64 refinement)"),
                "peak_kind": ("derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz" if fp64 else
                              "derived: 152 SMs x 128 FP32 FMA/clk x 2 FLOP x 2.07 GHz"),
                "peak_measured_fp64": fp64_meas, "peak_measured_fp32": fp32_meas,
                "launches": n_k, "kernel_ms_per_step": ms_k / steps, "share_of_step": ms_k / steps / ms_step,
                "flops_per_launch": flops_k / n_k}

    def e2e(step, precision, k):
        """Through the C ABI with host buffers: host descriptors in, the solution's TT cores read back to
        pinned host memory, all inside the host wall clock of each step."""
        times, d2h = [], 0
        hbuf = torch.empty(4 * 1024 * 1024, dtype=torch.float64).pin_memory().numpy()
        for _ in range(max(1, k)):
            with torch.cuda.stream(stream):
                flush.zero_()
            stream.synchronize()
            t0 = time.perf_counter()
            hs = step(precision)
            cores = tt.tt_iga_solution_cores(ctx, hs[2], hbuf)
            d2h = sum(c.size for c in cores) * 8
            times.append(time.perf_counter() - t0)
            release(hs)
        return max_over_ranks(statistics.mean(times), world), d2h

    # ---- headline workload: FP64 arm (the line's value) and mixed arm
    step, gdesc, rhs = make_step(wl, rank, local_rtol=HEADLINE_LOCAL_RTOL)
    h2d = len(bytes(gdesc)) + sum(len(bytes(r_)) for r_ in rhs) + len(bytes(tt.solve_opts()))
    ms64, info64, launches, prof64, clk, last64 = timed(step, tt.FP64, args.steps, args.warmup, profile=True,
                                                        keep_last=True)
    ms64_max = max_over_ranks(ms64, world)
    roof = roofline(prof64, ms64, args.steps, "fp64")
    e2e64_s, d2h = e2e(step, tt.FP64, args.steps)

    mixed = None
    if not args.no_mixed:
        msm, infom, launm, profm, clkm, lastm = timed(step, mixed_prec, args.steps, args.warmup, profile=True,
                                                      keep_last=True)
        msm_max = max_over_ranks(msm, world)
        # relative L2 difference of the mixed solution from the FP64 solution of the same problem
        l2_vs_fp64 = tt.tt_iga_l2_diff(ctx, last64[0], lastm[2], last64[2])
        e2em_s, d2hm = e2e(step, mixed_prec, args.steps)
        release(lastm)
        mixed = {"value": world * dofs / (msm_max / 1e3), "unit": "DOFs/s", "ms_per_step": msm_max,
                 "speedup_vs_fp64": ms64_max / msm_max,
                 "dtype": ("tf32 tensor-core contractions" if mixed_prec == tt.MIXED_TF32 else "f32") +
                          " local solves inside f64 refinement",
                 "rel_l2_vs_fp64": l2_vs_fp64, "rel_residual": infom.get("rel_residual"),
                 "sweeps": infom.get("sweeps"), "ranks": infom.get("ranks"),
                 "local_matvecs": infom.get("local_matvecs"), "local_matvecs_fp64": infom.get("local_matvecs_fp64"),
                 "phases_ms": infom.get("phases_ms"), "gpu_launches": launm, "clocks": clkm,
                 "roofline": roofline(profm, msm, args.steps, "mixed"),
                 "e2e": {"value": world * dofs / e2em_s, "unit": "DOFs/s", "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2hm}}
    # the same workload with the library's default exact local solves (both precisions)
    exact = None
    if not args.no_extra:
        estep, _, _ = make_step(wl, rank, local_rtol=-1.0)
        exact = {"local_solves": "exact (library default)"}
        for name, prec in (("fp64", tt.FP64), ("mixed", mixed_prec)):
            ms_e, info_e, _, _, _, lst = timed(estep, prec, max(3, args.steps // 2), 2, keep_last=True)
            exact[name] = {"value": world * dofs / (max_over_ranks(ms_e, world) / 1e3), "unit": "DOFs/s",
                           "ms_per_step": ms_e, "rel_residual": info_e.get("rel_residual"),
                           "sweeps": info_e.get("sweeps"), "ranks": info_e.get("ranks"),
                           "local_matvecs": info_e.get("local_matvecs"), "phases_ms": info_e.get("phases_ms"),
                           "rel_l2_vs_headline_fp64": tt.tt_iga_l2_diff(ctx, last64[0], lst[2], last64[2])}
            release(lst)
    release(last64)

    # ---- side entries (not the headline): the quarter cylinder at p = 3, n = 128, FP64 and mixed, with
    # the L2 error against the manufactured solution; the ring problem; the NURBS input path
    side = None
    if not args.no_extra and args.workload == WORKLOAD:
        ws = synthetic.WORKLOADS[SIDE_WORKLOAD]
        sstep, sgd, srhs = make_step(ws, rank)
        side = {"workload": SIDE_WORKLOAD, "dofs": ws["n"] ** 3}
        keep = {}
        for name, prec in (("fp64", tt.FP64), ("mixed", mixed_prec)):
            ms_s, info_s, _, _, _, lst = timed(sstep, prec, max(3, args.steps // 2), 2, keep_last=True)
            keep[name] = lst
            side[name] = {"value": world * ws["n"] ** 3 / (max_over_ranks(ms_s, world) / 1e3), "unit": "DOFs/s",
                          "ms_per_step": ms_s, "rel_residual": info_s.get("rel_residual"),
                          "ranks": info_s.get("ranks"), "sweeps": info_s.get("sweeps"),
                          "phases_ms": info_s.get("phases_ms"),
                          "l2_error_vs_exact": tt.tt_iga_l2_error(ctx, lst[0], lst[2], srhs[0])}
        side["mixed"]["rel_l2_vs_fp64"] = tt.tt_iga_l2_diff(ctx, keep["fp64"][0], keep["mixed"][2], keep["fp64"][2])
        for hs in keep.values():
            release(hs)

    # the ring problem of Section 4.3 (Dirichlet data 1 and 2 on the radial faces, natural conditions
    # elsewhere, f = 0) on the quarter cylinder at p = 3, n = 128, with its L2 error against the log solution
    ring = None
    if not args.no_extra and args.workload == WORKLOAD:
        ws = synthetic.WORKLOADS[SIDE_WORKLOAD]
        rgd = tt.geom_desc(ws["geometry"], ws["p"], ws["n"], cross_tol=ws["cross_tol"], seed=rank)
        bc = tt.bc_desc([1, 1, 0, 0, 0, 0], [1.0, 2.0, 0, 0, 0, 0])
        rrhs = [tt.rhs_desc(ring_log=True)]
        ring = {"workload": "ring_quarter_cylinder_p3_n128", "dofs": ws["n"] ** 3,
                "bc": "u=1 on rho=1, u=2 on rho=2, natural"}
        ts = []
        for rep in range(3):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g = tt.tt_iga_geometry(ctx, rgd)
            s = tt.tt_iga_assemble_bc(ctx, g, rrhs, bc, round_tol=ws["round_tol"])
            u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=TOL, precision=tt.FP64))
            e1.record(stream)
            e1.synchronize()
            if rep > 0:
                ts.append(e0.elapsed_time(e1))
            if rep == 2:
                ring["l2_error"] = tt.tt_iga_l2_error(ctx, g, u, rrhs[0])
            release((g, s, u))
        ms = max_over_ranks(statistics.mean(ts), world)
        ring.update({"value": world * ws["n"] ** 3 / (ms / 1e3), "unit": "DOFs/s", "ms_per_step": ms,
                     "rel_residual": st["rel_residual"], "ranks": st["ranks"], "sweeps": st["sweeps"]})

    # the NURBS input path: (1) the quarter cylinder given as a NURBS control net (the map evaluated from
    # the net on the device) at n = 128, (2) a curved patch (degree 2, perturbed cylindrical net, random
    # weights) at n = 32; constant source, homogeneous Dirichlet data.  Convergence is reported as it is:
    # the geometry cross's own validation, and the solve's exact residual (dense when its TT rank is large)
    nurbs = None
    if not args.no_extra and args.workload == WORKLOAD:
        ws = synthetic.WORKLOADS[SIDE_WORKLOAD]
        cases = [("quarter_cylinder_as_nurbs_p3_n128", synthetic.quarter_cylinder_net(1.0, 2.0, 1.0), ws["n"],
                  ws["cross_tol"], [tt.rhs_desc(constant=1.0)]),
                 ("curved_nurbs_patch_p3_n32", synthetic.curved_patch(seed=2), 32, 1e-8, [tt.rhs_desc(constant=1.0)])]
        nurbs = {}
        for name, net, nn, ctol, rr in cases:
            ndesc = tt.geom_desc({"kind": "nurbs"}, ws["p"], nn, cross_tol=ctol, seed=rank)
            rec = {"dofs": nn ** 3, "cross_tol": ctol}
            ts, tg = [], []
            for rep in range(3):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                eg = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                code_g = tt.OK
                try:
                    g = tt.tt_iga_geometry_nurbs(ctx, ndesc, *net)
                except tt.TTIgaError as exc:
                    if exc.code != tt.ERR_NOT_CONVERGED:
                        raise
                    code_g = exc.code
                    g = tt.tt_iga_geometry_nurbs(ctx, ndesc, *net, allow_not_converged=True)
                eg.record(stream)
                s = tt.tt_iga_assemble(ctx, g, rr, round_tol=max(ctol, ws["round_tol"]))
                u, st = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=TOL, precision=tt.FP64), allow_not_converged=True)
                e1.record(stream)
                e1.synchronize()
                if rep > 0:
                    ts.append(e0.elapsed_time(e1))
                    tg.append(e0.elapsed_time(eg))
                if rep == 2:
                    gr, gerr = tt.tt_iga_geom_ranks(g)
                    rec.update({"geometry_ranks": gr, "cross_max_rel_err": max(gerr),
                                "cross_validated": code_g == tt.OK,
                                "op_ranks": tt.tt_iga_system_info(s)["op_ranks"]})
                release((g, s, u))
            ms = max_over_ranks(statistics.mean(ts), world)
            # converged: the exact residual met the tolerance and the geometry's cross validated; null when
            # the exact residual could not be computed (the solve then rests on local residuals only)
            conv = None if st["rel_residual"] < 0 else bool(st["rel_residual"] <= TOL and rec["cross_validated"])
            rec.update({"value": world * nn ** 3 / (ms / 1e3), "unit": "DOFs/s", "ms_per_step": ms,
                        "geometry_ms": statistics.mean(tg), "rel_residual": st["rel_residual"], "converged": conv,
                        "solver_converged": bool(st["converged"]), "ranks": st["ranks"], "sweeps": st["sweeps"]})
            nurbs[name] = rec

    tt.tt_iga_ctx_destroy(ctx)

    # ---- batched: uneven random instances (geometry, p, n in [32, 256], 1-8 right-hand sides).  The
    # autotuner picks the lane count and the SM budget per lane (an equal share, so the lanes' local PCG
    # kernels run side by side, or the whole GPU per lane); the same batch as 8 lanes of independent
    # solves (each lane's PCG may take the whole GPU) is the comparison
    batched = None
    if args.batch_instances > 0:
        inst = [synthetic.random_instance(1 + k + 1000 * rank) for k in range(args.batch_instances)]
        items, keep = tt.batch_items(inst, tol=TOL, precision=mixed_prec)
        lanes, share, ms_tune, _ = tt.tt_iga_batch_autotune(items, [8, 16, 32, 48], shares=[-1, 0])
        out = {}
        # every instance's right-hand sides as one block-TT solve (the default), and, for
        # comparison, one AMEn solve per right-hand side and independent lanes
        for name, prec, how, ln, sh in (("mixed", mixed_prec, tt.RHS_BLOCK, lanes, share),
                                        ("fp64", tt.FP64, tt.RHS_BLOCK, lanes, share),
                                        ("mixed_per_rhs", mixed_prec, tt.RHS_EACH, lanes, share),
                                        ("mixed_8_independent_lanes", mixed_prec, tt.RHS_BLOCK, 8, 0)):
            items, keep = tt.batch_items(inst, tol=TOL, precision=prec, rhs_solve=how)
            code, res, ms = tt.tt_iga_batch_solve(items, ln, device=local, sm_per_lane=sh)
            dofs_b = sum(r["dofs"] for r in res if r["status"] == 0)
            out[name] = {"value": dofs_b / (ms / 1e3), "wall_ms": ms, "lanes": ln, "sm_per_lane": sh,
                         "ok": sum(r["status"] == 0 for r in res),
                         "worst_residual": max(r["rel_residual_max"] for r in res),
                         "residual_skipped": sum(r["rel_residual_max"] < 0 for r in res)}
        batched = {"instances": args.batch_instances, "lanes": lanes, "sm_per_lane": share,
                   "rhs_total": sum(len(i["rhs"]) for i in inst),
                   "dofs_total": sum(i["n"] ** 3 * len(i["rhs"]) for i in inst),
                   "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                   "speedup_vs_independent_lanes": out["mixed_8_independent_lanes"]["wall_ms"] / out["mixed"]["wall_ms"],
                   **out}

    # ---- serving: open-loop Poisson arrivals, n log-uniform in [32, nmax], tolerance 1e-6 or 1e-8 per
    # request, admission by footprint, continuous batching over lanes; each mixed result is compared
    # with the FP64 result of the same request (relative L2 difference, after the sessions)
    serving = None
    if args.serve_requests > 0:
        from paper_2509_13224_gb300.serving import Server, accuracy_vs, summarize_by, synthetic_stream
        serving = {"requests": args.serve_requests, "rate_hz": args.serve_rate, "n_range": [32, args.serve_nmax],
                   "tols": [1e-6, 1e-8]}
        recs_by = {}
        for policy in ("mixed", "fp64", "auto"):
            reqs = synthetic_stream(args.serve_requests, args.serve_rate, seed=11 + rank, n_lo=32,
                                    n_hi=args.serve_nmax)
            srv = Server(device=local, lanes=4, precision_policy=policy, keep_cores=True,
                         mixed_precision=mixed_prec)
            recs, summ = srv.serve(reqs)
            recs_by[policy] = recs
            serving[policy] = {**{k: summ[k] for k in ("p50_ms", "p99_ms", "dofs_per_s", "ok", "wall_s")},
                               "by_tol": summarize_by(recs, "tol")}
        reqs = synthetic_stream(args.serve_requests, args.serve_rate, seed=11 + rank, n_lo=32, n_hi=args.serve_nmax)
        acc = accuracy_vs(reqs, recs_by["mixed"], recs_by["fp64"], device=local)
        serving["mixed_vs_fp64"] = acc
        for policy in ("mixed", "auto"):
            errs = {}
            for r in recs_by[policy]:
                e = acc["per_request"].get(r["rid"])
                if e is not None and r.get("precision") != "fp64":
                    errs.setdefault(r["tol"], []).append(e)
            serving[policy]["rel_l2_vs_fp64_max_by_tol"] = {str(k): max(v) for k, v in errs.items()}
        del acc["per_request"]

    if rank != 0:
        return
    line = {"metric": METRIC, "value": world * dofs / (ms64_max / 1e3), "unit": "DOFs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms64_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload,
                       "geometry": "twisted and swollen quarter annulus r 1..2 h 1, twist 0.8 z, swell 0.2 sin(pi z)",
                       "p": p, "n": n, "dofs": dofs, "unknowns": (n - 2) ** 3, "tol": TOL,
                       "cross_tol": wl["cross_tol"], "round_tol": wl["round_tol"], "precision": "fp64",
                       "local_rtol": HEADLINE_LOCAL_RTOL,
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas"},
            "e2e": {"value": world * dofs / e2e64_s, "unit": "DOFs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "cpu_baseline": base, "mixed": mixed,
            "phases_ms": info64.get("phases_ms"),
            "solve": {"rel_residual": info64.get("rel_residual"), "sweeps": info64.get("sweeps"),
                      "ranks": info64.get("ranks"), "op_ranks": info64.get("op_ranks"),
                      "local_matvecs": info64.get("local_matvecs"), "solve_ms": info64.get("ms_total")},
            "exact_local_solves": exact, "quarter_cylinder_n128": side, "ring_dirichlet": ring, "nurbs_patch": nurbs, "batched": batched,
            "serving": serving}
    print(json.dumps(line), flush=True)

def main():
    args = parse()
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
