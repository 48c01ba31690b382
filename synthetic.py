"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module holds problem descriptors and random draws only: no step of the
TT-IGA method is computed here.  Every draw is a numpy PCG64 stream keyed by
an explicit seed.

Geometry descriptor (dict): kind ('annulus' or 'box'), r_in, r_out, height,
twist, swell (annulus), lx, ly, lz (box).
Right-hand-side descriptor: list of modes (a, (b1, b2, b3), c) modulating the
manufactured bubble by 1 + sum a sin(b . x + c).
"""
import math

import numpy as np

QUARTER_CYLINDER = {"kind": "annulus", "r_in": 1.0, "r_out": 2.0, "height": 1.0, "twist": 0.0, "swell": 0.0}
TWISTED_ANNULUS = {"kind": "annulus", "r_in": 1.0, "r_out": 2.0, "height": 1.0, "twist": 0.8, "swell": 0.2}
UNIT_BOX = {"kind": "box", "lx": 1.0, "ly": 1.0, "lz": 1.0}

# Named workloads.  Sizes are basis functions per direction (n) and degree (p).
WORKLOADS = {
    "quarter_cylinder_p2_n16": {"geometry": QUARTER_CYLINDER, "p": 2, "n": 16, "cross_tol": 1e-12,
                                "round_tol": 1e-12, "modes": []},
    "quarter_cylinder_p3_n128": {"geometry": QUARTER_CYLINDER, "p": 3, "n": 128, "cross_tol": 1e-12,
                                 "round_tol": 1e-12, "modes": [], "sweep": [16, 32, 64, 128]},
    "quarter_cylinder_p3_n64": {"geometry": QUARTER_CYLINDER, "p": 3, "n": 64, "cross_tol": 1e-12,
                                "round_tol": 1e-12, "modes": []},
    "twisted_annulus_p3_n512": {"geometry": TWISTED_ANNULUS, "p": 3, "n": 512, "cross_tol": 1e-10,
                                "round_tol": 1e-10, "modes": []},
}


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_tt_cores(dims, ranks, seed, scale=1.0):
    """Gaussian TT cores G_k[r_{k-1}, n_k, r_k] with r_0 = r_d = 1."""
    g = rng(seed)
    r = [1] + list(ranks) + [1]
    return [scale * g.standard_normal((r[k], dims[k], r[k + 1])) for k in range(len(dims))]


def random_modes(seed, count=None):
    """Random smooth modulation modes: |a| <= 0.3, |b| <= 3, c in [0, 2 pi)."""
    g = rng(seed)
    k = int(g.integers(1, 4)) if count is None else int(count)
    modes = []
    for _ in range(k):
        a = float(g.uniform(-0.3, 0.3))
        v = g.standard_normal(3)
        v = v / np.linalg.norm(v) * g.uniform(0.0, 3.0)
        c = float(g.uniform(0.0, 2.0 * math.pi))
        modes.append((a, tuple(float(t) for t in v), c))
    return modes


def random_instance(seed, n_lo=32, n_hi=256):
    """One instance of the batched workload (geometry, degree, size, right-hand sides)."""
    g = rng(1_000_003 * int(seed) + 17)
    r_in = float(g.uniform(0.5, 1.5))
    thick = float(g.uniform(0.5, 1.5))
    twist = float(g.uniform(0.0, 1.2))
    p = int(g.choice([2, 3]))
    n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
    n_rhs = int(g.integers(1, 9))
    geom = {"kind": "annulus", "r_in": r_in, "r_out": r_in + thick, "height": 1.0, "twist": twist, "swell": 0.0}
    rhs = [random_modes(10_000 * int(seed) + k) for k in range(n_rhs)]
    return {"seed": int(seed), "geometry": geom, "p": p, "n": n, "rhs": rhs}


def poisson_arrivals(rate_hz, count, seed):
    """Arrival times (s) of an open-loop Poisson request stream."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_hz, size=count))


def random_points(m, seed):
    """m parametric points in [0, 1]^3."""
    return rng(seed).uniform(0.0, 1.0, size=(m, 3))


def curved_patch(seed=2, counts=(4, 4, 3), jitter=0.05):
    """A curved single-patch NURBS volume for the NURBS-input tests: degree 2 in every
    direction, control points on a cylindrical grid (r in [1, 2], theta in [0, pi/2],
    z in [0, 1]) moved by Gaussian noise of size jitter, weights in [0.7, 1.3], one interior
    knot at 0.5 in the first two directions.  Returns (degrees, knots, ctrl[c1, c2, c3, 3],
    weights[c1, c2, c3])."""
    g = rng(seed)
    c1, c2, c3 = counts
    r = np.linspace(1.0, 2.0, c1)[:, None, None]
    t = np.linspace(0.0, 0.5 * math.pi, c2)[None, :, None]
    z = np.linspace(0.0, 1.0, c3)[None, None, :]
    ctrl = np.zeros((c1, c2, c3, 3))
    ctrl[..., 0] = r * np.cos(t) + 0 * z
    ctrl[..., 1] = r * np.sin(t) + 0 * z
    ctrl[..., 2] = 0 * r + 0 * t + z
    ctrl = ctrl + jitter * g.standard_normal(ctrl.shape)
    w = g.uniform(0.7, 1.3, (c1, c2, c3))

    def knots(c, inner):
        return [0.0, 0.0, 0.0] + inner + [1.0, 1.0, 1.0] if c == 3 + len(inner) else None

    kn = [knots(c1, [0.5]), knots(c2, [0.5]), knots(c3, [])]
    return (2, 2, 2), kn, ctrl, w


def quarter_cylinder_net(r_in=1.0, r_out=2.0, height=1.0):
    """The quarter cylinder as a NURBS control net (degrees (1, 2, 1)): radial control values
    r_in, r_out, the quarter circle (1,0), (1,1), (0,1) with weights 1, sqrt(2)/2, 1, axial 0 and
    height.  Returns (degrees, knots, ctrl[2, 3, 2, 3], weights[2, 3, 2])."""
    arc = [(1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
    warc = [1.0, math.sqrt(0.5), 1.0]
    ctrl = np.zeros((2, 3, 2, 3))
    w = np.zeros((2, 3, 2))
    for i, r in enumerate((r_in, r_out)):
        for j in range(3):
            for k, z in enumerate((0.0, height)):
                ctrl[i, j, k] = [r * arc[j][0], r * arc[j][1], z]
                w[i, j, k] = warc[j]
    knots = [[0.0, 0.0, 1.0, 1.0], [0.0, 0.0, 0.0, 1.0, 1.0, 1.0], [0.0, 0.0, 1.0, 1.0]]
    return (1, 2, 1), knots, ctrl, w
