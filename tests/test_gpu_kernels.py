"""Kernel-level parity of the CUDA path against the oracle (tables, point evaluator, contraction,
QR / SVD / maxvol, TT rounding)."""
import numpy as np
import pytest

import synthetic
from tests.gpu_util import band_to_dense, load_binding, oracle_geometry

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


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("n,p", [(4, 1), (8, 2), (16, 3), (37, 3), (9, 4), (128, 3)])
def test_basis_tables_match_oracle(tt, ctx, n, p):
    import torch
    from oracle.iga import Space1D
    s = Space1D(n, p)
    Q = s.Q
    pts = torch.empty(Q, dtype=torch.float64, device="cuda")
    wts = torch.empty_like(pts)
    N = torch.empty(Q, p + 1, dtype=torch.float64, device="cuda")
    dN = torch.empty_like(N)
    tt.tt_iga_basis_tables(ctx, n, p, p + 1, pts, wts, N, dN)
    torch.cuda.synchronize()
    assert np.max(np.abs(pts.cpu().numpy() - s.flat_points())) < 1e-15
    assert np.max(np.abs(wts.cpu().numpy() - s.flat_weights())) < 1e-15
    # rounding of x is amplified by the 1/h knot-span divisions of Cox-de Boor: allow O(n eps)
    eps = np.finfo(np.float64).eps
    assert np.max(np.abs(N.cpu().numpy() - s.N.reshape(Q, p + 1))) < 4 * n * eps
    dref = s.dN.reshape(Q, p + 1)
    assert np.max(np.abs(dN.cpu().numpy() - dref)) < 8 * n * eps * max(1.0, np.max(np.abs(dref)))


@pytest.mark.parametrize("geo,modes", [
    (synthetic.TWISTED_ANNULUS, []),
    (synthetic.QUARTER_CYLINDER, [(0.2, (1.0, -2.0, 0.5), 0.3)]),
    ({"kind": "box", "lx": 1.0, "ly": 2.0, "lz": 0.5}, [(0.1, (0.5, 0.5, 2.0), 1.0)]),
])
def test_geometry_points_match_oracle(tt, ctx, geo, modes):
    import torch
    from oracle.geometry import coefficient_tensor
    from oracle.iga import Space1D
    from oracle.manufactured import Manufactured
    n, p = 10, 2
    g = tt.tt_iga_geometry(ctx, tt.geom_desc(geo, p, n, cross_tol=1e-12, seed=3))
    try:
        s = Space1D(n, p)
        Q = s.Q
        rng = np.random.default_rng(5)
        idx = rng.integers(0, Q, size=(400, 3)).astype(np.int32)
        idx[:8] = [[0, 0, 0], [Q - 1, Q - 1, Q - 1], [0, Q - 1, 0], [Q - 1, 0, Q - 1], [1, 2, 3], [0, 0, Q - 1],
                   [Q - 1, Q - 1, 0], [5, 0, 5]]
        out = torch.empty(len(idx), 8, dtype=torch.float64, device="cuda")
        rhs = tt.rhs_desc(modes)
        bad = tt.tt_iga_geom_points(ctx, g, rhs, _t(idx), out)
        assert bad == 0
        got = out.cpu().numpy()
    finally:
        tt.tt_iga_geom_destroy(g)
    og = oracle_geometry(geo)
    m = Manufactured(og, modes)
    x = s.flat_points()
    for t, (a, b, c) in enumerate(idx):
        X, J = og.map(x[[a]], x[[b]], x[[c]])
        detJ, R = coefficient_tensor(J)
        R = R[0, 0, 0]
        ref = [R[0, 0], R[0, 1], R[0, 2], R[1, 1], R[1, 2], R[2, 2], detJ[0, 0, 0]]
        scale = np.max(np.abs(R))
        assert np.max(np.abs(got[t, :6] - ref[:6])) < 1e-13 * scale, t
        assert abs(got[t, 6] - ref[6]) < 1e-13 * abs(ref[6])
        fj = m.f(X)[0, 0, 0] * detJ[0, 0, 0]
        assert abs(got[t, 7] - fj) < 1e-11 * max(1.0, abs(fj)), (t, got[t, 7], fj)


@pytest.mark.parametrize("n,p,r0,r1", [(12, 3, 3, 5), (9, 2, 1, 4), (20, 3, 6, 1), (5, 1, 2, 2)])
def test_stiffness_and_load_cores_match_definition(tt, ctx, n, p, r0, r1):
    import torch
    from oracle.iga import Space1D
    from oracle.tt import load_core, stiffness_core
    s = Space1D(n, p)
    Q = s.Q
    G = synthetic.rng(13 + n).standard_normal((r0, Q, r1))
    w = s.flat_weights()
    Nt, Dt = s.full_tables()  # [n, Q]
    wts, N, dN = _t(w), _t(s.N.reshape(Q, p + 1)), _t(s.dN.reshape(Q, p + 1))
    Gd = _t(G)
    for te in (0, 1):
        for tr in (0, 1):
            M = torch.empty(r0, n, 2 * p + 1, r1, dtype=torch.float64, device="cuda")
            tt.tt_iga_stiffness_core(ctx, n, p, p + 1, wts, N, dN, Gd, r0, r1, te, tr, M)
            torch.cuda.synchronize()
            ref = stiffness_core(G, w, Dt if te else Nt, Dt if tr else Nt)
            got = band_to_dense(M.cpu().numpy(), n, p)
            assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref)), (te, tr)
    F = torch.empty(r0, n, r1, dtype=torch.float64, device="cuda")
    tt.tt_iga_load_core(ctx, n, p, p + 1, wts, N, Gd, r0, r1, F)
    torch.cuda.synchronize()
    ref = load_core(G, w, Nt)
    assert np.max(np.abs(F.cpu().numpy() - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("m,n,k", [(1260, 18, 9), (10, 1134, 30), (10, 20, 1260), (4, 30, 504), (70, 70, 70),
                                   (300, 5, 2000), (3, 3, 100000), (129, 257, 33), (1, 1, 1), (64, 64, 0)])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_matches_numpy(tt, ctx, m, n, k, ta, tb):
    """Every tile shape (64x64, 128x16, 16x128, 32x32), split-K and both transposes."""
    import torch
    rng = np.random.default_rng(m * 7 + n * 3 + k + 11 * ta + 5 * tb)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C0 = rng.standard_normal((m, n))
    C = _t(C0.copy())
    tt.tt_iga_gemm_f64(ctx, ta, tb, 1.5, _t(A), _t(B), -0.5, C)
    ref = 1.5 * (A.T if ta else A) @ (B.T if tb else B) - 0.5 * C0
    assert np.max(np.abs(C.cpu().numpy() - ref)) <= 1e-13 * max(1.0, np.sqrt(k)) * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("m,k", [(1000, 37), (100000, 16), (5000, 128), (7, 20), (300, 1), (2048, 256),
                                 (14280, 4), (50000, 3)])
def test_qr(tt, ctx, m, k):
    """Tall panels, wide panels, m < k, and narrow panels whose upper tree level is one whole block."""
    import torch
    rng = np.random.default_rng(m + k)
    A = rng.standard_normal((m, k))
    if k >= 4:
        A[:, 3] = A[:, 1] * 2.0  # rank deficiency
        A[:, 2] = 0.0
    Ad = _t(A)
    Q = torch.empty(m, k, dtype=torch.float64, device="cuda")
    R = torch.empty(k, k, dtype=torch.float64, device="cuda")
    tt.tt_iga_qr(ctx, Ad, Q, R)
    torch.cuda.synchronize()
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    assert np.max(np.abs(np.tril(Rh, -1))) == 0.0
    assert np.max(np.abs(Qh @ Rh - A)) < 1e-13 * max(1.0, np.max(np.abs(A))) * np.sqrt(k)
    kk = min(m, k)
    G = Qh[:, :kk].T @ Qh[:, :kk]
    assert np.max(np.abs(G - np.eye(kk))) < 1e-13 * np.sqrt(m)
    if m < k:
        assert np.max(np.abs(Qh[:, m:])) == 0.0 and np.max(np.abs(Rh[m:])) == 0.0


@pytest.mark.parametrize("k", [1, 2, 7, 50, 129, 200])
def test_svd_small(tt, ctx, k):
    import torch
    rng = np.random.default_rng(k)
    A = rng.standard_normal((k, k)) * np.logspace(0, -12, k)[None, :]
    U = torch.empty(k, k, dtype=torch.float64, device="cuda")
    V = torch.empty_like(U)
    s = torch.empty(k, dtype=torch.float64, device="cuda")
    tt.tt_iga_svd_small(ctx, _t(A), U, s, V)
    torch.cuda.synchronize()
    Uh, sh, Vh = U.cpu().numpy(), s.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.diff(sh) <= 0)
    assert np.max(np.abs(sh - ref)) < 1e-14 * ref[0] * k
    assert np.max(np.abs((Uh * sh) @ Vh.T - A)) < 1e-14 * ref[0] * k
    # U is the accumulated rotation (orthonormal); V's columns have unit norm and are orthogonal
    # to the accuracy their singular value allows
    assert np.max(np.abs(Uh.T @ Uh - np.eye(k))) < 1e-13 * k
    G = Vh.T @ Vh
    assert np.max(np.abs(np.diag(G) - 1.0)) < 1e-13 * k
    big = sh >= 1e-6 * sh[0]
    assert np.max(np.abs(G[np.ix_(big, big)] - np.eye(int(big.sum())))) < 1e-9


@pytest.mark.parametrize("m,r", [(500, 10), (4000, 40), (64, 64), (100, 1)])
def test_maxvol(tt, ctx, m, r):
    import torch
    rng = np.random.default_rng(r)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    rows = torch.empty(r, dtype=torch.int32, device="cuda")
    B = torch.empty(m, r, dtype=torch.float64, device="cuda")
    tt.tt_iga_maxvol(ctx, _t(U), rows, B, delta=1e-2, maxit=200)
    torch.cuda.synchronize()
    I, Bh = rows.cpu().numpy(), B.cpu().numpy()
    assert len(set(I.tolist())) == r
    assert np.max(np.abs(Bh[I] - np.eye(r))) < 1e-10
    assert np.max(np.abs(Bh)) <= 1.0 + 1e-2 + 1e-10
    assert np.max(np.abs(Bh - U @ np.linalg.inv(U[I]))) < 1e-9


def _block_sum(tts, weights):
    """Cores of sum_k weights[k] * tts[k] as one TT with block-diagonal middle core."""
    r1 = sum(t[0].shape[2] for t in tts)
    r2 = sum(t[1].shape[2] for t in tts)
    n2 = tts[0][1].shape[1]
    G1 = np.concatenate([w * t[0] for t, w in zip(tts, weights)], axis=2)
    G2 = np.zeros((r1, n2, r2))
    a = b = 0
    for t in tts:
        G2[a:a + t[1].shape[0], :, b:b + t[1].shape[2]] = t[1]
        a += t[1].shape[0]
        b += t[1].shape[2]
    G3 = np.concatenate([t[2] for t in tts], axis=0)
    return [G1, G2, G3]


@pytest.mark.parametrize("dims,ranks,eps", [([9, 10, 11], [3, 4], 1e-13), ([30, 25, 20], [8, 6], 1e-10),
                                            ([12, 40, 7], [5, 7], 1e-6), ([200, 30, 50], [20, 12], 1e-12)])
def test_round_matches_tt_svd(tt, ctx, dims, ranks, eps):
    """X = 2a + b stored with the redundant ranks of a + b + a; rounding must drop them."""
    import torch
    from oracle.tt import tt_full, tt_svd
    a = synthetic.random_tt_cores(dims, ranks, seed=21)
    b = synthetic.random_tt_cores(dims, ranks, seed=22)
    cores = _block_sum([a, b, a], [1.0, 1.0, 1.0])
    X = 2.0 * tt_full(a) + tt_full(b)
    assert np.max(np.abs(tt_full(cores) - X)) < 1e-10 * np.max(np.abs(X))
    out, rr = tt.tt_iga_round(ctx, [_t(G) for G in cores], eps)
    torch.cuda.synchronize()
    Y = tt_full([c.cpu().numpy() for c in out])
    assert np.linalg.norm(Y - X) <= eps * np.linalg.norm(X) * 1.0001 + 1e-14 * np.linalg.norm(X)
    ref = tt_svd(X, eps)
    assert rr[1:3] == [ref[0].shape[2], ref[1].shape[2]]
    assert rr[1] <= 2 * ranks[0] and rr[2] <= 2 * ranks[1]


def test_fma_peaks_are_physical(tt):
    """The benchmark's throughput probe (its own library, not the solver's): FP64 within the
    GB300's nominal range, FP32 far above it."""
    import bench
    fp64, fp32 = bench.fma_peaks(0)
    assert 0.3 < fp64 < 5.0, fp64      # nominal FP64 about 1.25 TFLOP/s
    assert 20.0 < fp32 < 200.0, fp32   # 152 SMs x 128 FP32 FMA/clk x 2 x ~2 GHz is about 80
    assert fp32 > 10.0 * fp64


def _spd(rng, m):
    G = rng.standard_normal((m, m))
    return G @ G.T / m + np.eye(m)


@pytest.mark.parametrize("rl,rr,Rl,Rr,n,p", [(1, 1, 1, 1, 7, 2), (1, 2, 2, 3, 64, 3), (2, 3, 3, 2, 510, 3),
                                            (2, 2, 1, 2, 5, 3), (3, 2, 2, 2, 37, 2), (1, 4, 2, 2, 100, 4),
                                            (8, 1, 2, 1, 33, 1), (1, 2, 1, 1, 1024, 3)])
def test_blockband_solve_matches_dense(tt, ctx, rl, rr, Rl, Rr, n, p):
    """The block-band preconditioner of the AMEn local solves (odd-even reduction of the block-tridiagonal
    super-row form, FP32 factor) against a dense FP64 solve of the same SPD local matrix
    B = sum_{g,d} PhiL_g (x) A_gd (x) PhiR_d: super-row counts 1 (n <= p) to 342, padded tails, blocks of 1 to 8."""
    import torch
    rng = np.random.default_rng(n * 31 + rl * 7 + rr)
    PhiL = np.stack([_spd(rng, rl) for _ in range(Rl)], axis=1)  # [rl][Rl][rl]
    PhiR = np.stack([_spd(rng, rr) for _ in range(Rr)], axis=1)  # [rr][Rr][rr]
    A = np.zeros((Rl, n, 2 * p + 1, Rr))
    B = np.zeros((rl * n * rr, rl * n * rr))
    for g in range(Rl):
        for d in range(Rr):
            Mg = np.zeros((n, n))
            for o in range(1, p + 1):
                v = rng.uniform(-1.0, 1.0, n - o) if n > o else np.zeros(0)
                Mg += np.diag(v, o) + np.diag(v, -o)
            Mg += np.diag(np.abs(Mg).sum(axis=1) + rng.uniform(0.5, 1.5, n))  # diagonally dominant: SPD
            for i in range(n):
                for o in range(2 * p + 1):
                    j = i + o - p
                    if 0 <= j < n:
                        A[g, i, o, d] = Mg[i, j]
            B += np.kron(PhiL[:, g, :], np.kron(Mg, PhiR[:, d, :]))
    r = rng.standard_normal(rl * n * rr)
    ref = np.linalg.solve(B, r)
    z = torch.zeros(rl * n * rr, dtype=torch.float64, device="cuda")
    tt.tt_iga_blockband_solve(ctx, _t(PhiL), _t(A), _t(PhiR), _t(r), z)
    torch.cuda.synchronize()
    got = z.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_blockband_solve_rejects_large_blocks(tt, ctx):
    import torch
    z = torch.zeros(9 * 8, dtype=torch.float64, device="cuda")
    PhiL = torch.eye(3, dtype=torch.float64, device="cuda").reshape(3, 1, 3)
    A = torch.zeros(1, 8, 5, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(tt.TTIgaError) as e:
        tt.tt_iga_blockband_solve(ctx, PhiL, A, PhiL, z, z)  # m = 3 x 3 = 9 > 8
    assert e.value.code == tt.ERR_TOO_LARGE
