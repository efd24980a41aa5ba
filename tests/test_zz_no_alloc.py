"""h2_matvec_noalloc: the matvec variant for callers that cannot allocate device memory.

It must give the product of h2_matvec (within the tolerances of the matvec tests) on two
calls in a row, which share the library's fixed device scratch, and match the oracle's
four-stage product of the same factors element-wise; it must reject sizes that do not fit
that scratch and the tensor-core-only modes.  A handle with FP64 factors only, used with
no h2_matvec before, must work too (the scratch's address is looked up at handle
creation).  Kept in a file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG

import factors
from parity import assert_elementwise, leaf_index_sets

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
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(ho), keep_fp32=True, keep_bf16=True)
    return h2, G, p.N, ho


def _call(h2, G, X, Y, nrhs, mode):
    return h2.lib().h2_matvec_noalloc(G._h, X.data_ptr(), X.shape[1], Y.data_ptr(), Y.shape[1], nrhs, mode, None)


def test_noalloc_fp64_only_handle_before_any_matvec(setup):
    """A fresh handle with FP64 factors only, no h2_matvec before: the first call succeeds and
    equals the oracle's product (1e-12, element-wise)."""
    h2, G0, N, ho = setup
    tree = h2.Tree(W.grid_coords(32), 32, ADM_STRONG, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(ho))
    X = torch.from_numpy(np.ascontiguousarray(W.rhs(N, 3, 9).T)).cuda()
    out = torch.full_like(X, float("nan"))
    assert _call(h2, G, X, out, 3, h2.H2_FP64) == h2.H2_OK
    torch.cuda.synchronize()
    want = O.matvec(ho, X.cpu().numpy().T)
    assert_elementwise(out.cpu().numpy().T, want, leaf_index_sets(ho.tree), 1e-12, "FP64 first call")


@pytest.mark.parametrize("mode,nrhs,tol", [(0, 1, 1e-12), (0, 3, 1e-12), (0, 7, 1e-12), (0, 70, 1e-12),
                                           (1, 1, 1e-5), (1, 3, 1e-5), (1, 7, 1e-5), (1, 70, 1e-5),
                                           (3, 1, 2e-2), (3, 3, 2e-2), (3, 7, 2e-2), (3, 70, 2e-2)])
def test_noalloc_matches_oracle(setup, mode, nrhs, tol):
    """FP64 / FP32 / BF16 at nrhs 1 and 3 (the scatter path, which zeroes part of the scratch),
    7 (gather kernels) and 70 (at least half the transfer kernels' right-hand-side tile), two
    calls in a row, against the oracle's product of the same factors (BF16: of the BF16-rounded
    inputs), element-wise at the bounds of the matvec tests."""
    h2, G, N, ho = setup
    xdt = {0: torch.float64, 1: torch.float32, 3: torch.bfloat16}[mode]
    ydt = torch.float64 if mode == 0 else torch.float32
    for seed in (11, 12):
        X = torch.from_numpy(np.ascontiguousarray(W.rhs(N, nrhs, seed).T)).to("cuda", xdt)
        out = torch.full((nrhs, N), float("nan"), dtype=ydt, device="cuda")
        assert _call(h2, G, X, out, nrhs, mode) == h2.H2_OK
        torch.cuda.synchronize()
        want = O.matvec(ho, X.double().cpu().numpy().T)
        assert_elementwise(out.double().cpu().numpy().T, want, leaf_index_sets(ho.tree), tol, f"mode {mode}")


def test_noalloc_rejects_tensor_core_modes(setup):
    h2, G, N, ho = setup
    X = torch.zeros((64, N), dtype=torch.float32, device="cuda")
    Y = torch.zeros_like(X)
    for mode in (h2.H2_TF32, h2.H2_TF32X3):
        assert _call(h2, G, X, Y, 64, mode) == h2.H2_ERR_INVALID_ARG


def test_noalloc_matches_matvec_on_two_calls(setup):
    h2, G, N, ho = setup
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
    """The smallest rejected nrhs, with X and Y allocated at that size: a regression of the
    size check shows as a wrong status, not as an access beyond a buffer."""
    h2, G, N, ho = setup
    rows = int(sum(int(k.sum()) for k in ho.k)) * 2        # coefficient rows: x-hat and y-hat of every box
    nrhs = (32 << 20) // (rows * 8) + 1
    assert rows * nrhs * 8 > (32 << 20) >= rows * (nrhs - 1) * 8
    X = torch.zeros((nrhs, N), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    assert _call(h2, G, X, Y, nrhs - 1, h2.H2_FP64) == h2.H2_OK
    st = _call(h2, G, X, Y, nrhs, h2.H2_FP64)
    assert st == h2.H2_ERR_INVALID_ARG
    assert b"scratch" in h2.lib().h2_last_error()
