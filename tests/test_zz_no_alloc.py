"""h2_matvec_noalloc: the matvec variant for callers that cannot allocate device memory.

It must give the same product as h2_matvec (within the 1e-12 relative tolerance of
the FP64 matvec tests) on two calls in a row, which share the library's fixed
device scratch, and reject sizes that do not fit that scratch.  Kept in a file of
its own that is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG

import factors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as h2
    h2.lib()
    c = W.SMALL_N32
    p, b = c["problem"], c["build"]
    op = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    ho = O.build(op, W.grid_coords(p.n), b.leaf, ADM_STRONG, b.eta, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                 b.adaptive, b.seed)[0]
    tree = h2.Tree(W.grid_coords(p.n), b.leaf, ADM_STRONG, b.eta)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(ho), keep_fp32=True)
    return h2, G, p.N


def _call(h2, G, X, Y, nrhs, mode):
    return h2.lib().h2_matvec_noalloc(G._h, X.data_ptr(), X.shape[1], Y.data_ptr(), Y.shape[1], nrhs, mode, None)


def test_noalloc_matches_matvec_on_two_calls(setup):
    h2, G, N = setup
    for nrhs, seed in ((7, 1), (7, 2)):
        X = torch.from_numpy(np.ascontiguousarray(W.rhs(N, nrhs, seed).T)).cuda()
        ref = torch.empty_like(X)
        G.matvec(X, ref, nrhs, h2.H2_FP64)
        out = torch.full_like(X, float("nan"))
        assert _call(h2, G, X, out, nrhs, h2.H2_FP64) == h2.H2_OK
        torch.cuda.synchronize()
        assert float((out - ref).norm() / ref.norm()) < 1e-12
    # FP32 mode against the FP32 h2_matvec
    X = torch.from_numpy(np.ascontiguousarray(W.rhs(N, 5, 3).T)).cuda().float()
    ref = torch.empty_like(X)
    G.matvec(X, ref, 5, h2.H2_FP32)
    out = torch.empty_like(X)
    assert _call(h2, G, X, out, 5, h2.H2_FP32) == h2.H2_OK
    torch.cuda.synchronize()
    assert float((out - ref).norm() / ref.norm()) < 1e-6


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    h2, G, N = setup
    X = torch.zeros((1, N), dtype=torch.float64, device="cuda")
    # nrhs large enough to need more than the fixed scratch; the check happens before any access
    st = h2.lib().h2_matvec_noalloc(G._h, X.data_ptr(), N, X.data_ptr(), N, 1_000_000, h2.H2_FP64, None)
    assert st == h2.H2_ERR_INVALID_ARG
    assert b"scratch" in h2.lib().h2_last_error()
