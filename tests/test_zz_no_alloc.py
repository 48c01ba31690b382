"""The allocation-free SVD entry point (tt_iga_svd_small_noalloc) gives the same factorisation as
tt_iga_svd_small.

It exists for callers that cannot allocate device memory -- code running while a stream is captured
into a CUDA graph, or a host that has reserved all device memory up front -- and works from a fixed
1 MiB scratch array inside the library.  This file is collected last on purpose; it must pass in a
fresh process (where its first call performs the one-time device set-up) and after the other tests.
"""
import numpy as np
import pytest

from tests.gpu_util import load_binding

pytestmark = pytest.mark.gpu


def _svd_pair(tt, k, seed):
    import torch
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((k, k)) * np.logspace(0, -10, k)[None, :]
    At = torch.as_tensor(A, device="cuda")
    outs = [torch.empty(k, k, dtype=torch.float64, device="cuda"), torch.empty(k, dtype=torch.float64, device="cuda"),
            torch.empty(k, k, dtype=torch.float64, device="cuda")]
    return A, At, outs


def test_noalloc_svd_matches_allocating_svd():
    import torch
    tt = load_binding()
    ctx = tt.tt_iga_ctx_create(torch.cuda.current_stream())
    try:
        for k in (129, 7, 256):  # two calls in a row per size, the array keeps the previous contents
            A, At, ref = _svd_pair(tt, k, seed=k)
            tt.tt_iga_svd_small(ctx, At, *ref)
            torch.cuda.synchronize()
            Ur, sr, Vr = (t.cpu().numpy() for t in ref)
            for rep in range(2):
                U = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
                s = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
                V = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
                code = tt.tt_iga_svd_small_noalloc(torch.cuda.current_stream(), At, U, s, V)
                assert code == tt.OK
                torch.cuda.synchronize()
                Uh, sh, Vh = U.cpu().numpy(), s.cpu().numpy(), V.cpu().numpy()
                tol = 1e-14 * sr[0] * k
                assert np.max(np.abs(sh - sr)) <= tol, (k, rep)
                assert np.max(np.abs((Uh * sh) @ Vh.T - A)) <= tol, (k, rep)
                assert np.max(np.abs((Uh * sh) @ Vh.T - (Ur * sr) @ Vr.T)) <= tol, (k, rep)
        # sizes beyond the fixed scratch are rejected before any launch
        A, At, out = _svd_pair(tt, 8, seed=1)
        big = torch.zeros(257, 257, dtype=torch.float64, device="cuda")
        assert tt.tt_iga_svd_small_noalloc(None, big, big, out[1], big) == tt.ERR_TOO_LARGE
    finally:
        tt.tt_iga_ctx_destroy(ctx)
