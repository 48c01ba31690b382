"""Tensor-train definitions used as plain references (oracle, Section 4).

TEST INFRASTRUCTURE ONLY.

* ``tt_full`` -- the TT format of Section 4.1.1: X(i1..id) = G1(1,i1,:) G2(:,i2,:) ... Gd(:,id,1).
* ``ttm_full`` -- the TT-matrix format: K(i, j) = M1(1,i1,j1,:) ... Md(:,id,jd,1),
  returned as a dense matrix with row/column index g = i1 + n1 (i2 + n2 i3 ...) (i1 fastest).
* ``tt_svd`` -- TT-SVD by successive truncated SVDs of the unfoldings
  (Oseledets 2011, the reference the paper cites for TT rounding), with the
  per-step threshold eps ||X||_F / sqrt(d-1).  Used to pin the ranks that
  TT rounding must reach.
* ``selector`` / ``stiffness_core`` / ``load_core`` -- Section 4.2.1 and 4.2.2:
  the per-direction contraction of a coefficient core with the univariate
  basis factors a_ij^(d), written as the sum over quadrature points.

Pins (tests/test_oracle_tt.py): rank-1 outer products are exact TT (the
"connection between tensor product and rank-1 TT" paragraph), TT-SVD error
bound, and the identity-map Kronecker structure of the assembled operator.
"""
import numpy as np


def tt_full(cores):
    """Dense tensor of a TT with cores G_k[r_{k-1}, n_k, r_k] (r_0 = r_d = 1)."""
    out = cores[0][0]  # [n1, r1]
    for G in cores[1:]:
        out = np.tensordot(out, G, axes=([-1], [0]))
    return out[..., 0]


def ttm_full(cores):
    """Dense matrix of a TT-matrix with cores M_k[r_{k-1}, n_k, n_k, r_k], i1 fastest."""
    out = cores[0][0]  # [i1, j1, r1]
    for M in cores[1:]:
        out = np.tensordot(out, M, axes=([-1], [0]))
    out = out[..., 0]  # [i1, j1, i2, j2, ..., id, jd]
    d = len(cores)
    rows = [2 * k for k in reversed(range(d))]
    cols = [2 * k + 1 for k in reversed(range(d))]
    out = out.transpose(rows + cols)
    N = int(np.prod([M.shape[1] for M in cores]))
    return out.reshape(N, N)


def tt_svd(X, eps):
    """TT-SVD of a dense tensor with relative accuracy eps; returns the list of cores."""
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    n = X.shape
    delta = eps * np.linalg.norm(X) / np.sqrt(max(d - 1, 1))
    cores = []
    r = 1
    C = X.reshape(n[0], -1)
    for k in range(d - 1):
        C = C.reshape(r * n[k], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tail[j] = ||s[j:]||
        rk = max(1, int(np.sum(tail > delta)))
        cores.append(U[:, :rk].reshape(r, n[k], rk))
        C = s[:rk, None] * Vt[:rk]
        r = rk
    cores.append(C.reshape(r, n[d - 1], 1))
    return cores


def selector(i, j, d):
    """The factor a_ij^(d) of Section 4.2.1 as (test factor, trial factor).

    'D' is the basis derivative N', 'N' the basis N.  d = i = j gives N'^T N'
    (the 'd' case), d not in {i, j} gives N^T N ('m'), d = i != j puts the
    derivative on the test index and d = j != i on the trial index (the two
    orientations of 'c').
    """
    test = "D" if d == i else "N"
    trial = "D" if d == j else "N"
    return test, trial


def stiffness_core(G, w, A, B):
    """M[alpha, a, b, beta] = sum_q w_q G[alpha, q, beta] A[a, q] B[b, q] (Section 4.2.1)."""
    return np.einsum("xqy,q,aq,bq->xaby", G, w, A, B)


def load_core(G, w, N):
    """F[alpha, a, beta] = sum_q w_q G[alpha, q, beta] N[a, q] (Section 4.2.2)."""
    return np.einsum("xqy,q,aq->xay", G, w, N)
