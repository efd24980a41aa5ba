"""Learned ranks on the GPU: the rank model's kernels against the oracle MLP, the predicted
start counts in the construction against the oracle peeling, and the gain over plain
adaptive peeling on held-out heat Hessians.

Tolerances: the kernels compute in FP32 with FP32 master weights; the oracle in FP64 on the
same (float32-representable) parameters and inputs, with the same bfloat16 rounding of the
weights.  Loss and gradient: 1e-4 relative to the largest gradient entry (FP32
accumulation over a few hundred rows).  One Adam step: parameters to 1e-7 absolute (the
update is lr * m_hat / (sqrt(v_hat) + eps), lr = 1e-3).  Over many steps the FP32 and FP64
trajectories separate (Adam normalises tiny gradient differences), so longer training is
compared by its loss, not its parameters.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle import mlp
from oracle.tree import ADM_STRONG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h2():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as m
    m.lib()
    assert torch.cuda.is_available()
    return m


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, mlp.F)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * X[:, 3] ** 2 + 3.0).astype(np.float32)
    return X, t


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _model(h2, bf16, seed=3):
    m = h2.RankModel(seed=seed, bf16=bf16)
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(mlp.NPARAM) * 0.3).astype(np.float32)
    m.set(p, np.zeros(mlp.NPARAM, np.float32), np.zeros(mlp.NPARAM, np.float32), 0)
    return m, p


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("n", [1, 64, 300])
def test_loss_and_gradient_match_oracle(h2, bf16, n):
    m, p = _model(h2, bf16)
    X, t = _data(n, 5)
    loss, g = m.loss_grad(_dev(X), _dev(t))
    lo, go = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), bf16=bf16)
    assert abs(loss - lo) <= 1e-5 * lo
    scale = np.abs(go).max()
    assert np.abs(g - go).max() <= 1e-4 * scale


@pytest.mark.parametrize("bf16", [False, True])
def test_one_adam_step_matches_oracle(h2, bf16):
    m, p = _model(h2, bf16)
    X, t = _data(300, 6)
    idx = np.random.default_rng(1).integers(0, 300, 200).astype(np.int32)
    loss = torch.zeros(1, device="cuda")
    m.train(_dev(X), _dev(t), 1, 200, 1e-3, idx=_dev(idx), loss_out=loss)
    p1, m1, v1, step = m.get()
    assert step == 1
    p64 = p.astype(np.float64)
    lo, g = mlp.loss_and_grad(p64, X[idx].astype(np.float64), t[idx].astype(np.float64), bf16=bf16)
    pw, mw, vw = mlp.adam_step(p64, np.zeros_like(p64), np.zeros_like(p64), g, 1, lr=1e-3)
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    np.testing.assert_allclose(m1, mw, rtol=0, atol=1e-4 * np.abs(mw).max())
    np.testing.assert_allclose(v1, vw, rtol=0, atol=1e-4 * np.abs(vw).max())
    np.testing.assert_allclose(p1, pw, rtol=0, atol=1e-7)


def test_training_tracks_oracle(h2):
    """200 Adam steps (explicit minibatches, batch 96 = one full and one ragged chunk)."""
    m, p = _model(h2, True, seed=8)
    X, t = _data(400, 9)
    steps, batch, lr = 200, 96, 3e-3
    idx = np.random.default_rng(2).integers(0, 400, (steps, batch)).astype(np.int32)
    losses = torch.zeros(steps, device="cuda")
    m.train(_dev(X), _dev(t), steps, batch, lr, idx=_dev(idx), loss_out=losses)
    pg = m.get()[0]
    X64, t64 = X.astype(np.float64), t.astype(np.float64)
    po, mo, vo = p.astype(np.float64), np.zeros(mlp.NPARAM), np.zeros(mlp.NPARAM)
    l_or = []
    for s in range(steps):
        lo, g = mlp.loss_and_grad(po, X64[idx[s]], t64[idx[s]], bf16=True)
        l_or.append(lo)
        po, mo, vo = mlp.adam_step(po, mo, vo, g, s + 1, lr=lr)
    lg = losses.cpu().numpy()
    assert abs(lg[0] - l_or[0]) <= 1e-5 * l_or[0]
    full0 = mlp.loss_and_grad(p.astype(np.float64), X64, t64, bf16=True)[0]
    full_g = mlp.loss_and_grad(pg.astype(np.float64), X64, t64, bf16=True)[0]
    full_o = mlp.loss_and_grad(po, X64, t64, bf16=True)[0]
    assert full_o < 0.2 * full0 and full_g < 0.2 * full0
    assert abs(full_g - full_o) <= 0.1 * full_o


def test_predict_matches_oracle_forward(h2):
    for bf16 in (False, True):
        m, p = _model(h2, bf16, seed=4)
        X, _ = _data(1000, 10)              # 16 CTAs, ragged last one
        y = torch.empty(1000, device="cuda")
        m.predict(_dev(X), y)
        torch.cuda.synchronize()
        yo, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64), bf16=bf16)
        assert np.abs(y.cpu().numpy() - yo).max() <= 1e-5 * np.abs(yo).max()


def test_in_kernel_minibatches_are_deterministic(h2):
    X, t = _data(500, 11)
    Xd, td = _dev(X), _dev(t)
    outs = []
    for _ in range(2):
        m = h2.RankModel(seed=12, bf16=True)
        losses = torch.zeros(300, device="cuda")
        m.train(Xd, td, 300, 64, 3e-3, loss_out=losses)
        outs.append((m.get()[0], losses.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1][-20:].mean() < 0.3 * outs[0][1][:20].mean()


def test_bad_minibatch_index_is_reported(h2):
    m, _ = _model(h2, True)
    X, t = _data(50, 1)
    idx = np.zeros((2, 8), dtype=np.int32)
    idx[1, 3] = 50                           # out of range: the kernel skips the row and flags it
    m.train(_dev(X), _dev(t), 2, 8, 1e-3, idx=_dev(idx))
    with pytest.raises(h2.H2Error) as e:
        m.get()
    assert e.value.status == h2.H2_ERR_DEVICE_CHECK
    m.get()                                  # the flag is cleared once reported


def test_q_levels_match_oracle(h2):
    m, p = _model(h2, True, seed=14)
    p2 = p.copy()
    p2[-1] = 5.0                             # b3: predictions around 2^5
    m.set(p2)
    coords = W.grid_coords(40)
    tree = h2.Tree(coords, 32, ADM_STRONG, 0.7)
    q, y = m.q_levels(tree, 0.005, 0.1, 1e-6, pad=8, q_max=128)
    f = mlp.level_features(O.ClusterTree(coords, 32), 0.005, 0.1, 1e-6)
    yo, _ = mlp.forward(p2.astype(np.float64), f.astype(np.float32).astype(np.float64), bf16=True)
    assert np.abs(y - yo).max() <= 1e-5 * np.abs(yo).max()
    assert q[0] == 0
    for l in range(1, tree.L + 1):
        assert q[l] == mlp.q_start_from_prediction(float(y[l]), 8, 128)


def test_build_with_predicted_starts_matches_oracle(h2):
    """Start counts below and above the adaptive need: calls, probes, need and ranks equal the oracle's."""
    n, m_s = 32, 200
    mask = W.sensor_mask(n * n, m_s, 1001)
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    coords = W.grid_coords(n)
    _, ad = O.build(op, coords, 16, ADM_STRONG, 0.7, 1e-6, 32, 16, 8, 128, True, 7)
    L = max(ad.need.keys())
    ql = [0] * (L + 1)
    for l in range(1, L + 1):
        # alternate: too small by 8 (the first test fails), enough + 8 (passes at once)
        ql[l] = max(8, ad.need[l] - 8) if l % 2 else ad.need[l] + 8
    ho, res = O.build(op, coords, 16, ADM_STRONG, 0.7, 1e-6, 32, 16, 8, 128, True, 7, q_level=ql, q_test=8)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    tree = h2.Tree(coords, 16, ADM_STRONG, 0.7)
    opts = h2.default_opts(kmax=32, q0=16, b_inc=8, q_max=128, adaptive=1, seed=7, q_level=ql, q_test=8)
    G = h2.H2.build(gop, tree, 1e-6, opts)
    st = G.stats()
    assert st["samples"] == res.samples - res.norm_its
    # range calls, one projection call per level and the leaf pass
    assert st["op_calls"] == sum(res.range_calls.values()) + tree.L + 1
    for l in range(1, tree.L + 1):
        assert st["range_calls"][l] == res.range_calls[l]
        assert st["range_probes"][l] == res.range_probes[l]
        assert st["range_need"][l] == res.need[l]
        assert st["range_passed"][l] == res.passed[l]
        assert st["max_rank"][l] == int(ho.k[l].max())
    # both branches occur: a first test that fails (a second call) and one that passes at once
    assert any(res.range_calls[l] >= 2 for l in range(1, tree.L + 1) if res.passed[l] == 1)
    assert any(res.range_calls[l] == 1 and res.passed[l] == 1 for l in range(1, tree.L + 1))


# ---------------------------------------------------------------- gain over adaptive peeling

def _heat_set(h2, probs, leaf=64):
    out = []
    for p in probs:
        mask = W.sensor_mask(p.N, p.m, p.sensor_seed)
        out.append((p, h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, mask),
                    h2.Tree(W.grid_coords(p.n), leaf, ADM_STRONG, 0.7)))
    return out


def _gpu_err(h2, G, gop, N, its=30):
    """||H - H~||_2 / ||H||_2 by power iteration on the device."""
    def diff(v):
        a = torch.empty_like(v)
        b = torch.empty_like(v)
        gop.apply(v, a, 1)
        G.matvec(v, b, 1)
        return a - b
    def hv(v):
        a = torch.empty_like(v)
        gop.apply(v, a, 1)
        return a
    out = []
    for f in (diff, hv):
        v = torch.from_numpy(np.random.default_rng(3).standard_normal(N)).cuda()
        lam = 0.0
        for _ in range(its):
            v = v / torch.linalg.norm(v)
            w = f(v)
            lam = float(torch.linalg.norm(w))
            v = w
        out.append(lam)
    return out[0] / out[1]


def test_learned_start_saves_operator_calls(h2):
    """Train on adaptive builds of 32 heat Hessians (n 96..160), then build 6 held-out ones
    (n 112..160) with plain adaptive peeling (q0 32, b_inc 16) and from the predicted starts:
    fewer operator calls, no more samples, the same accuracy."""
    tol = 1e-6
    train = _heat_set(h2, W.batch_problems(32, seed=77, n_lo=96, n_hi=160))
    opts_fine = h2.default_opts(kmax=32, q0=16, b_inc=8, q_max=256)
    Gs = h2.build_batched([o for _, o, _ in train], [t for _, _, t in train], tol, opts_fine)
    feats, targ = [], []
    for (p, _, t), G in zip(train, Gs):
        f = h2.rank_features(t, p.kappa * p.T, p.m / p.N, tol)
        lv, tg = h2.rank_targets(G)
        feats.append(f[lv])
        targ += tg
    X = np.concatenate(feats).astype(np.float32)
    y = np.asarray(targ, dtype=np.float32)
    model = h2.RankModel(seed=1, bf16=True)
    p0 = model.get()[0]
    p0[-1] = float(y.mean())                 # start the output bias at the mean target
    model.set(p0)
    model.train(_dev(X), _dev(y), 3000, 64, 3e-3)
    loss, _ = model.loss_grad(_dev(X), _dev(y))
    print(f"rank model: {len(y)} rows, target range {y.min():.2f}..{y.max():.2f}, train loss {loss:.4f}")
    assert loss < 0.1                        # log2 units

    test = _heat_set(h2, W.batch_problems(6, seed=78, n_lo=112, n_hi=160))
    tot = {"ad": [0, 0, 0.0], "ml": [0, 0, 0.0]}
    for p, gop, t in test:
        Ga = h2.H2.build(gop, t, tol, h2.default_opts())
        q, _ = model.q_levels(t, p.kappa * p.T, p.m / p.N, tol, pad=8, q_max=256)
        Gm = h2.H2.build(gop, t, tol, h2.default_opts(q_level=q, q_test=8))
        sa, sm = Ga.stats(), Gm.stats()
        print(f"n={p.n} need(adaptive)={sa['range_need'][1:]} q_start={list(q[1:])} "
              f"calls {sa['op_calls']} -> {sm['op_calls']} samples {sa['samples']} -> {sm['samples']}")
        for key, G in (("ad", Ga), ("ml", Gm)):
            st = G.stats()
            tot[key][0] += st["op_calls"]
            tot[key][1] += st["samples"]
            tot[key][2] += st["t_peel"]
            assert _gpu_err(h2, G, gop, p.N) < 2 * tol
    print("adaptive calls/samples/t_peel", tot["ad"], "learned", tot["ml"])
    assert tot["ml"][0] <= tot["ad"][0]
    assert tot["ml"][1] <= 0.9 * tot["ad"][1]


def test_save_and_load_round_trip(h2, tmp_path):
    m, p = _model(h2, True, seed=21)
    X, t = _data(200, 3)
    m.train(_dev(X), _dev(t), 5, 32, 1e-3)
    path = str(tmp_path / "model.bin")
    m.save(path)
    m2 = h2.RankModel.load(path)
    a, b = m.get(), m2.get()
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
    assert a[3] == b[3] == 5
    y1 = torch.empty(200, device="cuda")
    y2 = torch.empty(200, device="cuda")
    m.predict(_dev(X), y1)
    m2.predict(_dev(X), y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
