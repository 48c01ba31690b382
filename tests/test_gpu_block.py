"""Several right-hand sides as one block-TT solve (AMEn of Section 4.1.2 on the block system
I (x) K with the right-hand-side index merged into one TT mode): the block operator and load
densified against their definition, and every sliced solution against its own plain solve and
the oracle."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import load_binding, oracle_geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    return load_binding()


@pytest.fixture(scope="module")
def ctx(tt):
    import torch
    c = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    yield c
    tt.tt_iga_ctx_destroy(c)


def _eval(tt, ctx, u, pts):
    import torch
    xi = torch.tensor(pts, dtype=torch.float64, device="cuda")
    out = torch.empty(len(pts), dtype=torch.float64, device="cuda")
    tt.tt_iga_eval(ctx, u, xi, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _modes(k):
    return synthetic.random_modes(100 + k, count=2)


def _oracle_solution(geo, n, p, modes):
    """Restricted full-grid FP64 solution of the oracle (flat, i1 fastest)."""
    from oracle.iga import Space1D, solve, to_flat
    from oracle.manufactured import Manufactured
    og = oracle_geometry(geo)
    u, _ = solve([Space1D(n, p)] * 3, og, Manufactured(og, modes), tol=1e-14)
    return to_flat(u[1:-1, 1:-1, 1:-1])


def _system(tt, ctx, geo, p, n, rhs, bc=None):
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-14, seed=7))
    if bc is None:
        s = tt.tt_iga_assemble(ctx, g, rhs, round_tol=1e-14)
    else:
        s = tt.tt_iga_assemble_bc(ctx, g, rhs, bc, round_tol=1e-14)
    return g, s


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_block_operator_and_load_are_the_stacked_definition(tt, ctx, mode):
    """With the right-hand-side index merged into mode d (index i_d + m_d k):
    K_b[(.., i_d + m_d k, ..), (.., j_d + m_d k', ..)] = delta_kk' K[(i1, i2, i3), (j1, j2, j3)] and
    block k of F_b is F_k / ||F_k||, on a ragged mesh with three right-hand sides."""
    nb = 3
    rhs = [tt.rhs_desc(_modes(k)) for k in range(nb)]
    g, s = _system(tt, ctx, synthetic.TWISTED_ANNULUS, 2, (7, 6, 5), rhs)
    b, scales = tt.tt_iga_system_stack(ctx, s, mode)
    try:
        m = tt.tt_iga_system_info(s)["modes"]
        mb = tt.tt_iga_system_info(b)["modes"]
        want = list(m)
        want[mode] *= nb
        assert mb == tuple(want) and tt.tt_iga_system_info(b)["n_rhs"] == 1
        K = tt.tt_iga_densify_operator(ctx, s)
        Kb = tt.tt_iga_densify_operator(ctx, b)
        F = [tt.tt_iga_densify_rhs(ctx, s, k) for k in range(nb)]
        Fb = tt.tt_iga_densify_rhs(ctx, b, 0)
    finally:
        tt.tt_iga_system_destroy(b)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    N = m[0] * m[1] * m[2]
    # index maps: plain g = i1 + m1 (i2 + m2 i3); block: the same with i_d -> i_d + m_d k and m_d -> nb m_d
    idx = np.meshgrid(np.arange(m[0]), np.arange(m[1]), np.arange(m[2]), indexing="ij")
    gp = (idx[0] + m[0] * (idx[1] + m[1] * idx[2])).ravel()
    ref = np.zeros((nb * N, nb * N))
    for k in range(nb):
        j = list(idx)
        j[mode] = j[mode] + m[mode] * k
        gb = (j[0] + mb[0] * (j[1] + mb[1] * j[2])).ravel()
        ref[np.ix_(gb, gb)] = K[np.ix_(gp, gp)]
        assert np.max(np.abs(Fb[gb] - F[k][gp] / scales[k])) < 1e-13
        assert abs(scales[k] - np.linalg.norm(F[k])) < 1e-12 * scales[k]
    assert np.array_equal(Kb, ref)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_block_solve_matches_plain_solves_and_oracle(tt, ctx, mode):
    from oracle.iga import Space1D, evaluate, solve
    from oracle.manufactured import Manufactured
    n, p, nb = 8, 2, 3
    geo = synthetic.QUARTER_CYLINDER
    rhs = [tt.rhs_desc(_modes(k)) for k in range(nb)]
    g, s = _system(tt, ctx, geo, p, n, rhs)
    tol = 1e-11
    sols, st, rr = tt.tt_iga_solve_block(ctx, s, tt.solve_opts(tol=tol), mode)
    x = np.linspace(0.0, 1.0, 5)
    pts = np.array([[a, b, c] for c in x for b in x for a in x])
    try:
        assert st["converged"]
        ub = [_eval(tt, ctx, u, pts) for u in sols]
        up = []
        for k in range(nb):
            u, stk = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=tol, rhs_index=k))
            up.append(_eval(tt, ctx, u, pts))
            tt.tt_iga_solution_destroy(u)
    finally:
        for u in sols:
            tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    assert all(0 <= r <= tol for r in rr), rr
    og = oracle_geometry(geo)
    sp = [Space1D(n, p)] * 3
    for k in range(nb):
        uo, _ = solve(sp, og, Manufactured(og, _modes(k)), tol=1e-14)
        ref = evaluate(sp, uo, x, x, x).transpose(2, 1, 0).ravel()
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(ub[k] - ref)) < 1e-9 * scale
        assert np.max(np.abs(ub[k] - up[k])) < 1e-9 * scale


def test_block_solve_keeps_the_boundary_data(tt, ctx):
    """Ring with Dirichlet data and a flux face: both right-hand sides carry the lift and the
    surface load; the slices equal the plain solves."""
    bc = tt.bc_desc([1, 0, 0, 0, 0, 0], [1.0, 0, 0, 0, 0, 0], [0, 0.5, 0, 0, 0, 0])
    rhs = [tt.rhs_desc(ring_log=True), tt.rhs_desc(constant=2.0)]
    g, s = _system(tt, ctx, synthetic.QUARTER_CYLINDER, 2, 9, rhs, bc)
    pts = synthetic.random_points(100, seed=21)
    sols, st, rr = tt.tt_iga_solve_block(ctx, s, tt.solve_opts(tol=1e-11))
    try:
        assert st["converged"] and max(rr) <= 1e-11
        ub = [_eval(tt, ctx, u, pts) for u in sols]
        l2 = tt.tt_iga_l2_error(ctx, g, sols[0], tt.rhs_desc(ring_log=True))
        up = []
        for k in range(2):
            u, _ = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-11, rhs_index=k))
            up.append(_eval(tt, ctx, u, pts))
            if k == 0:
                l2p = tt.tt_iga_l2_error(ctx, g, u, tt.rhs_desc(ring_log=True))
            tt.tt_iga_solution_destroy(u)
    finally:
        for u in sols:
            tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    for k in range(2):
        assert np.max(np.abs(ub[k] - up[k])) < 1e-9 * np.max(np.abs(up[k]))
    assert abs(l2 - l2p) <= 1e-6 * l2p


def test_block_handles_are_checked(tt, ctx):
    rhs = [tt.rhs_desc(_modes(k)) for k in range(2)]
    g, s = _system(tt, ctx, synthetic.QUARTER_CYLINDER, 2, 6, rhs)
    b, scales = tt.tt_iga_system_stack(ctx, s, 2)
    ub, _ = tt.tt_iga_solve(ctx, b, tt.solve_opts(tol=1e-10))
    try:
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_system_stack(ctx, b, 1)  # already a block system
        assert e.value.code == tt.ERR_ARG
        with pytest.raises(tt.TTIgaError) as e:
            tt.tt_iga_solution_unstack(ctx, ub, 2, 1.0)
        assert e.value.code == tt.ERR_ARG
        with pytest.raises(tt.TTIgaError) as e:
            _eval(tt, ctx, ub, np.full((4, 3), 0.5))
        assert e.value.code == tt.ERR_ARG
        u1 = tt.tt_iga_solution_unstack(ctx, ub, 1, scales[1])
        r = tt.tt_iga_residual(ctx, s, u1, 1)
        tt.tt_iga_solution_destroy(u1)
        assert r <= 1e-9
    finally:
        tt.tt_iga_solution_destroy(ub)
        tt.tt_iga_system_destroy(b)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)


def test_batch_block_and_per_rhs_both_meet_the_tolerance(tt):
    inst = [synthetic.random_instance(s, n_lo=12, n_hi=24) for s in (1, 2, 6)]
    assert all(len(i["rhs"]) >= 2 for i in inst)
    res = {}
    for how in (tt.RHS_BLOCK, tt.RHS_EACH):
        items, keep = tt.batch_items(inst, tol=1e-8, rhs_solve=how)
        code, r, ms = tt.tt_iga_batch_solve(items, lanes=2)
        assert code == tt.OK
        res[how] = r
    for a, b in zip(res[tt.RHS_BLOCK], res[tt.RHS_EACH]):
        assert a["status"] == b["status"] == 0 and a["dofs"] == b["dofs"]
        assert 0 <= a["rel_residual_max"] <= 1e-8 and 0 <= b["rel_residual_max"] <= 1e-8
    items, keep = tt.batch_items(inst[:1], rhs_solve=7)
    code, _, _ = tt.tt_iga_batch_solve(items, lanes=1)
    assert code == tt.ERR_ARG


def test_eight_right_hand_sides_in_one_block_solve(tt, ctx):
    """The batch limit of right-hand sides: every slice meets the tolerance and equals its plain solve."""
    n, p, nb = 7, 2, 8
    rhs = [tt.rhs_desc(_modes(k)) for k in range(nb)]
    g, s = _system(tt, ctx, synthetic.TWISTED_ANNULUS, p, n, rhs)
    pts = synthetic.random_points(64, seed=31)
    sols, st, rr = tt.tt_iga_solve_block(ctx, s, tt.solve_opts(tol=1e-11))
    try:
        assert st["converged"] and len(sols) == nb
        ub = [_eval(tt, ctx, u, pts) for u in sols]
        m = tt.tt_iga_system_info(s)["modes"]
        dense = [tt.tt_iga_densify_solution(ctx, u, m) for u in sols]
        up = []
        for k in range(nb):
            u, _ = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-11, rhs_index=k))
            up.append(_eval(tt, ctx, u, pts))
            tt.tt_iga_solution_destroy(u)
    finally:
        for u in sols:
            tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    assert all(0 <= r <= 1e-11 for r in rr), rr
    for k in range(nb):
        assert np.max(np.abs(ub[k] - up[k])) < 1e-8 * np.max(np.abs(up[k]))
    # and every slice against the oracle's full-grid solve of its own right-hand side
    for k in range(nb):
        ref = _oracle_solution(synthetic.TWISTED_ANNULUS, n, p, _modes(k))
        assert np.linalg.norm(dense[k] - ref) <= 1e-9 * np.linalg.norm(ref), k


def test_mixed_precision_block_solve(tt, ctx):
    """FP32 local solves inside FP64 refinement on the block system: every right-hand side meets
    1e-10 and agrees with its FP64 solve to the accuracy that residual allows."""
    n, p, nb = 9, 2, 3
    rhs = [tt.rhs_desc(_modes(k)) for k in range(nb)]
    g, s = _system(tt, ctx, synthetic.QUARTER_CYLINDER, p, n, rhs)
    pts = synthetic.random_points(64, seed=32)
    sols, st, rr = tt.tt_iga_solve_block(ctx, s, tt.solve_opts(tol=1e-10, precision=tt.MIXED_FP32))
    try:
        assert st["converged"] and st["local_matvecs"] > st["local_matvecs_fp64"]
        ub = [_eval(tt, ctx, u, pts) for u in sols]
        m = tt.tt_iga_system_info(s)["modes"]
        dense = [tt.tt_iga_densify_solution(ctx, u, m) for u in sols]
        up = []
        for k in range(nb):
            u, _ = tt.tt_iga_solve(ctx, s, tt.solve_opts(tol=1e-12, rhs_index=k))
            up.append(_eval(tt, ctx, u, pts))
            tt.tt_iga_solution_destroy(u)
    finally:
        for u in sols:
            tt.tt_iga_solution_destroy(u)
        tt.tt_iga_system_destroy(s)
        tt.tt_iga_geom_destroy(g)
    assert all(0 <= r <= 1e-10 for r in rr), rr
    for k in range(nb):
        assert np.max(np.abs(ub[k] - up[k])) < 1e-6 * np.max(np.abs(up[k]))
    for k in range(nb):
        ref = _oracle_solution(synthetic.QUARTER_CYLINDER, n, p, _modes(k))
        assert np.linalg.norm(dense[k] - ref) <= 1e-7 * np.linalg.norm(ref), k
