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


@pytest.fixture(scope="module")
def oracle_batch():
    """Four uneven heat Hessians (n 64..96, leaf 64, strong 0.7, tol 1e-6) built in one batched
    call, and their oracle constructions."""
    import oracle as O
    from oracle.tree import ADM_STRONG

    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as h2
    h2.lib()
    probs = [W.HeatProblem(n=n, m=max(1, round(f * n * n)), kappa=kap, T=0.5, sigma=0.01, sensor_seed=700 + n)
             for n, f, kap in ((64, 0.06, 0.01), (72, 0.12, 0.03), (83, 0.08, 0.005), (96, 0.15, 0.02))]
    ops = [h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed)) for p in probs]
    trees = [h2.Tree(W.grid_coords(p.n), 64, h2.H2_ADM_STRONG, 0.7) for p in probs]
    opts = h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=256, adaptive=1, seed=7, keep_fp32=1)
    batched = h2.build_batched(ops, trees, 1e-6, opts)
    oracle = []
    for p in probs:
        op = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
        oracle.append((op,) + O.build(op, W.grid_coords(p.n), 64, ADM_STRONG, 0.7, 1e-6, 32, 32, 16, 256, True, 7))
    return h2, probs, batched, oracle


def test_batched_build_matches_oracle(oracle_batch):
    """Each batched construction takes the oracle's decisions (samples, probes per level, ranks
    of every box) and agrees with the oracle's H^2 in the 2-norm (power iteration on the
    difference) to within ten times the method's own sensitivity to rounding, measured here as
    the change of the oracle's construction (rank replay) when its operator products are
    perturbed by 1e-16 relative (see test_replay_sensitivity_adaptive_64), and at most 1e-9."""
    import oracle as O

    h2, probs, batched, oracle = oracle_batch
    for p, G, (op, ho, res) in zip(probs, batched, oracle):
        st = G.stats()
        L = st["levels"]
        assert st["samples"] == res.samples - res.norm_its
        assert abs(st["norm_est"] - res.norm_est) <= 1e-10 * res.norm_est
        for l in range(1, L + 1):
            assert st["range_probes"][l] == res.range_probes[l]
            assert st["proj_probes"][l] == res.proj_probes[l]
        rk = G.export()[0]
        o = 0
        for l in range(L + 1):
            np.testing.assert_array_equal(rk[o:o + (1 << l)], ho.k[l])
            o += 1 << l

        def gpu(v):
            vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
            yd = torch.empty_like(vd)
            G.matvec(vd, yd, 1)
            torch.cuda.synchronize()
            return yd.cpu().numpy()

        v0 = np.random.default_rng(3).standard_normal(p.N)
        d = O.power_norm(lambda v: gpu(v) - O.matvec(ho, v), p.N, v0) / res.norm_est
        e = O.power_norm(lambda v: gpu(v) - op(v), p.N, v0) / res.norm_est
        rng = np.random.default_rng(11)
        probes = [res.range_probes.get(l, 0) for l in range(L + 1)]
        hp, _ = O.replay_build(lambda X: op(X) * (1.0 + 1e-16 * rng.standard_normal(np.shape(X))),
                               W.grid_coords(p.n), 64, O.ADM_STRONG, 0.7, 1e-6, 32, 7, res.norm_est, probes, ho.k)
        sens = O.power_norm(lambda v: O.matvec(hp, v) - O.matvec(ho, v), p.N, v0) / res.norm_est
        print(f"n={p.n}: ||H2_batched - H2_oracle|| / ||H|| = {d:.1e} (oracle's own sensitivity {sens:.1e}), "
              f"||H - H2_batched|| / ||H|| = {e:.1e}")
        assert d <= min(max(1e-12, 10.0 * sens), 1e-9)
        assert e <= 1e-6


@pytest.mark.parametrize("mode,nrhs", [(0, 5), (0, 64), (1, 3), (1, 64)])
def test_batched_matvec_matches_oracle(oracle_batch, mode, nrhs):
    """The merged, graph-captured batched matvec of every handle against the oracle's four-stage
    product of the same (exported) factors, element-wise: FP64 1e-12, FP32 1e-5."""
    import oracle as O
    from oracle.tree import ADM_STRONG, ClusterTree, Partition

    import factors
    from parity import assert_elementwise, leaf_index_sets

    h2, probs, batched, oracle = oracle_batch
    dt = torch.float64 if mode == h2.H2_FP64 else torch.float32
    Xs = [W.rhs(p.N, nrhs, 300 + i) for i, p in enumerate(probs)]
    Xd = [torch.from_numpy(np.ascontiguousarray(x.T)).to("cuda", dt) for x in Xs]
    Yd = [torch.full_like(x, float("nan")) for x in Xd]
    B = h2.Batch(batched)
    B.matvec(Xd, Yd, nrhs, mode)
    B.matvec(Xd, Yd, nrhs, mode)         # replay of the captured graph
    torch.cuda.synchronize()
    for p, G, X, Y, (op, ho, res) in zip(probs, batched, Xs, Yd, oracle):
        g = factors.import_to_oracle(ho.tree, ho.part, *G.export())
        want = O.matvec(g, np.asarray(Xd[probs.index(p)].double().cpu().numpy().T))
        assert_elementwise(Y.double().cpu().numpy().T, want, leaf_index_sets(ho.tree),
                           1e-12 if mode == h2.H2_FP64 else 1e-5, f"n={p.n}")
    B.close()


def test_batched_certified_build_equals_individual_builds(setup):
    """Certified range bases through the batched construction: each Hessian equals its own
    certified construction, and spends fewer products than with the default bases."""
    h2, probs, ops, trees, batched, single = setup
    opts = h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=128, adaptive=1, seed=3, certified=1)
    cb = h2.build_batched(ops, trees, 1e-6, opts)
    cs = [h2.H2.build(op, t, 1e-6, opts) for op, t in zip(ops, trees)]
    fewer = 0
    for b, s, d in zip(cb, cs, single):
        sb, ss = b.stats(), s.stats()
        for k in ("samples", "range_probes", "proj_probes", "max_rank", "entries_D", "entries_S"):
            assert sb[k] == ss[k], k
        for xb, xs in zip(b.export(), s.export()):
            np.testing.assert_array_equal(xb, xs)
        assert sb["samples"] <= d.stats()["samples"]
        fewer += sb["samples"] < d.stats()["samples"]
    assert fewer > 0
    for G in cb + cs:
        G.close()
