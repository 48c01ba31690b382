"""Shared fixtures for the GPU tests: the built binding and one context on cuda:0."""
import numpy as np
import pytest


def load_binding():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2509_13224_gb300 as tt
    return tt


def oracle_geometry(geo):
    from oracle.geometry import Annulus, Box
    if geo["kind"] == "annulus":
        return Annulus(geo["r_in"], geo["r_out"], geo["height"], geo.get("twist", 0.0), geo.get("swell", 0.0))
    return Box(geo["lx"], geo["ly"], geo["lz"])


def band_to_dense(M, n, p):
    """[r0][n][2p+1][r1] band core -> dense [r0][n][n][r1] (index bookkeeping only)."""
    r0, _, b, r1 = M.shape
    D = np.zeros((r0, n, n, r1))
    for i in range(n):
        for o in range(b):
            j = i + o - p
            if 0 <= j < n:
                D[:, i, j, :] = M[:, i, o, :]
    return D
