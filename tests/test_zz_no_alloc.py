"""The allocation-free SVD entry point (tt_iga_svd_small_noalloc) against the allocating one
(tt_iga_svd_small) and against numpy.

Some callers of this library cannot allocate device memory: a serving process that reserved all of
the GPU's memory for its own pools at start-up, or a plug-in that is handed only a stream and its
buffers.  For them the library keeps a fixed 1 MiB scratch array of its own, and this entry point
works from that array alone.  The file is collected last on purpose: it must pass in a fresh process
(where its first call performs the one-time lookup of the array's device address) and after the
other tests.
"""
import numpy as np
import pytest

from tests.gpu_util import load_binding

pytestmark = pytest.mark.gpu


def _matrix(k, seed):
    rng = np.random.default_rng(seed)
    # graded column scales: singular values over ten orders of magnitude
    return rng.standard_normal((k, k)) * np.logspace(0, -10, k)[None, :]


def test_noalloc_svd_matches_allocating_svd_and_numpy():
    import torch
    tt = load_binding()
    ctx = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    try:
        for k in (129, 7, 256):
            A = _matrix(k, seed=k)
            At = torch.as_tensor(A, device="cuda")
            ref = [torch.empty(k, k, dtype=torch.float64, device="cuda"),
                   torch.empty(k, dtype=torch.float64, device="cuda"),
                   torch.empty(k, k, dtype=torch.float64, device="cuda")]
            tt.tt_iga_svd_small(ctx, At, *ref)
            torch.cuda.synchronize()
            Ur, sr, Vr = (t.cpu().numpy() for t in ref)
            s_np = np.linalg.svd(A, compute_uv=False)
            tol = 1e-14 * sr[0] * k
            # two calls in a row: the shared array still holds the previous call's panels
            for rep in range(2):
                U = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
                s = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
                V = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
                info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
                code = tt.tt_iga_svd_small_noalloc(torch.cuda.current_stream(), At, U, s, V, info)
                assert code == tt.OK
                torch.cuda.synchronize()
                assert int(info.item()) == 0, (k, rep)
                Uh, sh, Vh = U.cpu().numpy(), s.cpu().numpy(), V.cpu().numpy()
                # against the allocating entry point
                assert np.max(np.abs(sh - sr)) <= tol, (k, rep)
                assert np.max(np.abs((Uh * sh) @ Vh.T - (Ur * sr) @ Vr.T)) <= tol, (k, rep)
                # against numpy and the definition
                assert np.all(np.diff(sh) <= 0.0), (k, rep)
                assert np.max(np.abs(sh - s_np)) <= tol, (k, rep)
                assert np.max(np.abs((Uh * sh) @ Vh.T - A)) <= tol, (k, rep)
                assert np.max(np.abs(Uh.T @ Uh - np.eye(k))) <= 1e-12, (k, rep)
                # columns of V belong to nonzero singular values; each has unit norm and they are
                # orthogonal to the accuracy their singular value allows
                G = Vh.T @ Vh
                assert np.max(np.abs(np.diag(G) - 1.0)) <= 1e-12, (k, rep)
                big = sh >= 1e-6 * sh[0]
                assert np.max(np.abs(G[np.ix_(big, big)] - np.eye(int(big.sum())))) <= 1e-10, (k, rep)
        # sizes beyond the fixed scratch are rejected before any launch
        out_s = torch.empty(8, dtype=torch.float64, device="cuda")
        big_m = torch.zeros(257, 257, dtype=torch.float64, device="cuda")
        assert tt.tt_iga_svd_small_noalloc(None, big_m, big_m, out_s, big_m) == tt.ERR_TOO_LARGE
    finally:
        tt.tt_iga_ctx_destroy(ctx)
