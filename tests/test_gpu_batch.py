"""Batching pattern: many Hessians of uneven sizes built in one call and applied in merged,
graph-captured launches.  The per-Hessian arithmetic is that of the single-Hessian path, so
the batched results must equal the individual ones (bit-for-bit where both use the same
kernels; 1e-12 relative where the single path uses the atomic small-nrhs scatter)."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as h2
    h2.lib()
    probs = [W.HeatProblem(n=n, m=max(1, (n * n) // k), kappa=kap, T=0.5, sigma=0.01, sensor_seed=900 + n)
             for n, k, kap in ((24, 9, 0.02), (31, 12, 0.01), (40, 7, 0.005), (48, 16, 0.03), (57, 10, 0.01))]
    ops = [h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed)) for p in probs]
    trees = [h2.Tree(W.grid_coords(p.n), 32, h2.H2_ADM_STRONG, 0.7) for p in probs]
    opts = h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=128, adaptive=1, seed=3, keep_fp32=1, keep_bf16=1)
    batched = h2.build_batched(ops, trees, 1e-6, opts)
    single = [h2.H2.build(op, t, 1e-6, opts) for op, t in zip(ops, trees)]
    return h2, probs, ops, trees, batched, single


def test_batched_build_equals_individual_builds(setup):
    h2, probs, ops, trees, batched, single = setup
    for b, s in zip(batched, single):
        sb, ss = b.stats(), s.stats()
        for k in ("samples", "range_probes", "proj_probes", "max_rank", "entries_D", "entries_S"):
            assert sb[k] == ss[k], k
        for xb, xs in zip(b.export(), s.export()):
            np.testing.assert_array_equal(xb, xs)


@pytest.mark.parametrize("mode,nrhs", [(0, 5), (0, 64), (1, 64), (1, 3)])
def test_batch_matvec_equals_individual(setup, mode, nrhs):
    h2, probs, ops, trees, batched, single = setup
    dt = torch.float64 if mode == h2.H2_FP64 else torch.float32
    Xs = [torch.from_numpy(np.ascontiguousarray(W.rhs(p.N, nrhs, 40 + i).T)).to("cuda", dt) for i, p in enumerate(probs)]
    Ys = [torch.full_like(x, float("nan")) for x in Xs]
    B = h2.Batch(batched)
    B.matvec(Xs, Ys, nrhs, mode)
    B.matvec(Xs, Ys, nrhs, mode)         # second call replays the captured graph
    torch.cuda.synchronize()
    assert B.tuned(nrhs, mode) in (8, 16, 32)
    for G, X, Y in zip(single, Xs, Ys):
        R = torch.empty_like(X)
        G.matvec(X, R, nrhs, mode)
        torch.cuda.synchronize()
        if nrhs > 4:
            assert torch.equal(R, Y)      # same gather kernels, same summation order
        else:
            tol = 1e-12 if mode == h2.H2_FP64 else 1e-5
            assert float((R - Y).norm() / R.norm()) < tol
    B.close()


def test_one_shot_batched_matvec_equals_batch(setup):
    h2, probs, ops, trees, batched, single = setup
    nrhs = 16
    Xs = [torch.from_numpy(np.ascontiguousarray(W.rhs(p.N, nrhs, 70 + i).T)).to("cuda", torch.float32)
          for i, p in enumerate(probs)]
    Y1 = [torch.empty_like(x) for x in Xs]
    Y2 = [torch.empty_like(x) for x in Xs]
    B = h2.Batch(batched)
    B.matvec(Xs, Y1, nrhs, h2.H2_FP32)
    h2.matvec_batched(batched, Xs, Y2, nrhs, h2.H2_FP32)
    torch.cuda.synchronize()
    for a, b in zip(Y1, Y2):
        assert torch.equal(a, b)      # same tuned tile candidates, same kernels, same order
    B.close()


@pytest.mark.parametrize("mode,nrhs", [(2, 64), (2, 130), (3, 64), (3, 130), (4, 64)])
def test_batch_tensor_core_matvec_equals_individual(setup, mode, nrhs):
    """TF32 / BF16 with nrhs >= 64: per-handle tensor-core phases between merged SIMT sweeps; the
    result equals each handle's own tensor-core matvec (same products, same summation order),
    also when the graph is replayed and when the buffers change (recaptured)."""
    h2, probs, ops, trees, batched, single = setup
    xdt = torch.bfloat16 if mode == h2.H2_BF16 else torch.float32
    B = h2.Batch(batched)
    for trial in range(2):
        Xs = [torch.from_numpy(np.ascontiguousarray(W.rhs(p.N, nrhs, 90 + i + 7 * trial).T)).to("cuda", xdt)
              for i, p in enumerate(probs)]
        Ys = [torch.full((nrhs, p.N), float("nan"), dtype=torch.float32, device="cuda") for p in probs]
        B.matvec(Xs, Ys, nrhs, mode)
        B.matvec(Xs, Ys, nrhs, mode)      # replay
        torch.cuda.synchronize()
        for G, X, Y in zip(single, Xs, Ys):
            R = torch.empty_like(Y)
            G.matvec(X, R, nrhs, mode)
            torch.cuda.synchronize()
            assert torch.equal(R, Y)
    B.close()
