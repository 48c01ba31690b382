"""Batched solves (many uneven instances, concurrent lanes) and the serving loop:
results do not depend on what else runs, and the session statistics are computed."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    return load_binding()


def _instances(count, seed0, n_lo=16, n_hi=40):
    out = []
    for k in range(count):
        inst = synthetic.random_instance(seed0 + k, n_lo=n_lo, n_hi=n_hi)
        inst["rhs"] = inst["rhs"][:3]
        out.append(inst)
    return out


def test_batch_is_independent_of_concurrency(tt):
    """With the same lanes (hence the same SM budget per lane) an instance gives the same bits alone
    and in the batch; one lane (the whole GPU per solve) converges as well."""
    inst = _instances(6, 100)
    items, keep = tt.batch_items(inst, tol=1e-8)
    code1, res1, ms1 = tt.tt_iga_batch_solve(items, lanes=1)
    code4, res4, ms4 = tt.tt_iga_batch_solve(items, lanes=4)
    assert code1 == tt.OK and code4 == tt.OK
    for k, (a, b, i) in enumerate(zip(res1, res4, inst)):
        assert a["status"] == 0 and b["status"] == 0
        assert a["rel_residual_max"] <= 1e-8 and b["rel_residual_max"] <= 1e-8
        assert a["dofs"] == i["n"] ** 3 * len(i["rhs"])
        one, keep1 = tt.batch_items([i], tol=1e-8)
        code, alone, _ = tt.tt_iga_batch_solve(one, lanes=4)
        assert code == tt.OK
        assert alone[0]["ranks"] == b["ranks"] and alone[0]["sweeps"] == b["sweeps"]
        assert alone[0]["rel_residual_max"] == b["rel_residual_max"], k


def test_batch_solutions_match_oracle(tt):
    """A handful of batch instances (uneven geometry, degree, size and right-hand sides), every
    right-hand side's solution against the oracle's full-grid FP64 solve."""
    from oracle.iga import Space1D, solve
    from oracle.manufactured import Manufactured
    from oracle.tt import tt_full
    from tests.gpu_util import oracle_geometry
    inst = _instances(4, 300, n_lo=10, n_hi=16)
    for i in inst:
        i["rhs"] = i["rhs"][:2]
    items, keep = tt.batch_items(inst, tol=1e-12, cross_tol=1e-13, round_tol=1e-13, cores_cap=1 << 18)
    code, res, _ = tt.tt_iga_batch_solve(items, lanes=3)
    assert code == tt.OK
    for k, (i, r) in enumerate(zip(inst, res)):
        sols = tt.batch_cores(keep[1][k], r, i["n"])
        assert len(sols) == len(i["rhs"])
        og = oracle_geometry(i["geometry"])
        sp = [Space1D(i["n"], i["p"])] * 3
        for cores, modes in zip(sols, i["rhs"]):
            uo, _ = solve(sp, og, Manufactured(og, modes), tol=1e-14)
            ref = uo[1:-1, 1:-1, 1:-1]
            got = tt_full(cores)
            assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), (k, i["n"], i["p"])


def test_batch_autotune_picks_a_candidate(tt):
    items, keep = tt.batch_items(_instances(4, 200), tol=1e-6, precision=tt.MIXED_FP32)
    best, share, ms, res = tt.tt_iga_batch_autotune(items, [1, 2, 4], shares=[-1, 0])
    assert best in (1, 2, 4) and share in (-1, 0) and ms > 0
    assert all(r["status"] == 0 for r in res)


def test_serving_same_result_alone_and_in_the_mix(tt):
    from oracle.tt import tt_full
    from paper_2509_13224_gb300.serving import Request, Server
    target = synthetic.random_instance(7, n_lo=24, n_hi=32)
    others = [synthetic.random_instance(50 + k, n_lo=16, n_hi=40) for k in range(7)]

    def req(inst, rid, arrival):
        return Request(rid, inst["geometry"], inst["p"], inst["n"], 1e-8, modes=inst["rhs"][0], arrival=arrival,
                       seed=inst["seed"])

    srv = Server(lanes=4, keep_cores=True)
    alone, _ = srv.serve([req(target, 0, 0.0)])
    mix = [req(target, 0, 0.002)] + [req(o, k + 1, 0.0005 * k) for k, o in enumerate(others)]
    mixed, summary = srv.serve(mix)
    a = [r for r in alone if r["rid"] == 0][0]
    b = [r for r in mixed if r["rid"] == 0][0]
    assert a["status"] == 0 and b["status"] == 0
    ua, ub = tt_full(a["cores"]), tt_full(b["cores"])
    assert np.max(np.abs(ua - ub)) <= 1e-12 * np.max(np.abs(ua))
    assert summary["ok"] == len(mix)
    assert summary["p99_ms"] >= summary["p50_ms"] > 0


def test_serving_admission_respects_budget(tt):
    from paper_2509_13224_gb300.serving import Server, footprint_bytes, synthetic_stream
    reqs = synthetic_stream(6, rate_hz=1000.0, seed=3, n_lo=16, n_hi=32)
    one = max(footprint_bytes(r.n, r.p) for r in reqs)
    srv = Server(lanes=4, budget_bytes=one)  # at most one request fits at a time
    recs, summary = srv.serve(reqs)
    assert summary["ok"] == len(reqs)
    spans = sorted((r["start"], r["end"]) for r in recs)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3  # no overlap when the budget admits one request
