"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (FP64): the matvec of a given H^2 and the Hessian operator are
deterministic products, compared at 1e-12 relative.  Matvec results are compared
element-wise (tests/parity.py): every right-hand side's relative 2-norm error and every
leaf block's largest error relative to its largest entry must be within the bound.  Exact-recovery inputs (planted structures) must be recovered to 1e-12.
The construction of an approximation is not unique: the sampled range bases of
the two implementations agree on the sampled range but differ in the directions
of its numerical null space (about 1e-10 ||H||), and the truncation at tau_basis
turns such differences into rotations of the basis vectors whose singular values
lie near tau_basis.  Sample counts, probes per level and ranks must therefore be
equal, and the two approximations must each be within tol of H and within tol of
each other in the relative 2-norm (power iteration, two significant digits).
Reduced-precision matvecs are compared with the FP64 oracle at the stated bounds:
FP32 storage 1e-5, BF16 storage and inputs 2e-2 (8-bit mantissa, FP32 accumulation).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

import factors
import planted
from parity import assert_elementwise, leaf_index_sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h2():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as m
    m.lib()
    assert torch.cuda.is_available()
    return m


def dev(x, dtype=torch.float64):
    """numpy (N x nrhs, column-major) -> device tensor laid out column-major (shape nrhs x N)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).to("cuda", dtype)


def host(t):
    return t.double().cpu().numpy().T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _heat_problem(n, m, seed, kappa=0.01):
    mask = W.sensor_mask(n * n, m, seed)
    return mask, O.HeatHessian(n, kappa, 0.5, 0.01, mask)


@pytest.mark.parametrize("n,nrhs", [(32, 5), (13, 3), (64, 1)])
def test_heat_operator_matches_oracle(h2, n, nrhs):
    mask, op = _heat_problem(n, max(1, n * n // 8), 3)
    X = W.rhs(n * n, nrhs, 4)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    Xd = dev(X)
    Yd = torch.empty_like(Xd)
    gop.apply(Xd, Yd, nrhs)
    torch.cuda.synchronize()
    assert rel(host(Yd), op(X)) < 1e-12


@pytest.mark.parametrize("N,nrhs", [(300, 7), (2100, 3), (64, 64)])
def test_dense_operator_gemm(h2, N, nrhs):
    rng = np.random.default_rng(N)
    A = rng.standard_normal((N, N))
    X = rng.standard_normal((N, nrhs))
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()   # column-major A
    dop = h2.DenseOperator(Ad)
    Xd, Yd = dev(X), torch.empty((nrhs, N), dtype=torch.float64, device="cuda")
    h2.lib().h2_dense_op_apply(dop.ctx, N, nrhs, Xd.data_ptr(), N, Yd.data_ptr(), N, 0)
    torch.cuda.synchronize()
    assert rel(host(Yd), A @ X) < 1e-13


def _oracle_h2(kind):
    if kind == "heat32_strong":
        c = W.SMALL_N32
        p, b = c["problem"], c["build"]
        mask, op = _heat_problem(p.n, p.m, p.sensor_seed)
        return O.build(op, W.grid_coords(p.n), b.leaf, ADM_STRONG, 0.7, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                       b.adaptive, b.seed)[0], p.n, b.leaf, ADM_STRONG
    if kind == "heat32_weak":
        c = W.SMALL_N32
        p, b = c["problem"], c["build"]
        mask, op = _heat_problem(p.n, p.m, p.sensor_seed)
        return O.build(op, W.grid_coords(p.n), b.leaf, ADM_WEAK, 0.7, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                       b.adaptive, b.seed)[0], p.n, b.leaf, ADM_WEAK
    if kind == "ragged":   # 37 x 37 grid: leaves of 42/43 points
        mask, op = _heat_problem(37, 150, 5)
        return O.build(op, W.grid_coords(37), 48, ADM_STRONG, 0.7, 1e-6, 24, 32, 16, 128, True, 3)[0], 37, 48, ADM_STRONG
    if kind == "weak_k48":   # HSS partition at a tight threshold: ranks above 32 (up to the cap 48)
        mask, op = _heat_problem(32, 200, 11)
        return O.build(op, W.grid_coords(32), 32, ADM_WEAK, 0.7, 1e-9, 48, 32, 16, 256, True, 3)[0], 32, 32, ADM_WEAK
    if kind == "tiny":     # no levels: a single dense block
        mask, op = _heat_problem(4, 5, 5)
        return O.build(op, W.grid_coords(4), 16, ADM_STRONG, 0.7, 1e-6, 8, 8, 8, 8, False, 3)[0], 4, 16, ADM_STRONG
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["heat32_strong", "heat32_weak", "ragged", "tiny"])
@pytest.mark.parametrize("nrhs", [1, 7, 33, 130])
def test_matvec_fp64_matches_oracle(h2, kind, nrhs):
    h, n, leaf, adm = _oracle_h2(kind)
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(h), keep_fp32=True, keep_bf16=True)
    X = W.rhs(n * n, nrhs, 9)
    want = O.matvec(h, X)
    Xd = dev(X)
    Yd = torch.full_like(Xd, float("nan"))
    G.matvec(Xd, Yd, nrhs, h2.H2_FP64)
    torch.cuda.synchronize()
    leaves = leaf_index_sets(h.tree)
    assert_elementwise(host(Yd), want, leaves, 1e-12, "FP64")
    # reduced precision against the FP64 oracle
    Y32 = torch.empty((nrhs, n * n), dtype=torch.float32, device="cuda")
    G.matvec(Xd.float(), Y32, nrhs, h2.H2_FP32)
    torch.cuda.synchronize()
    assert_elementwise(host(Y32), want, leaves, 1e-5, "FP32")
    Yb = torch.empty((nrhs, n * n), dtype=torch.float32, device="cuda")
    G.matvec(Xd.to(torch.bfloat16), Yb, nrhs, h2.H2_BF16)
    torch.cuda.synchronize()
    # BF16 inputs and storage: the reference is the oracle product of the BF16-rounded inputs
    want_b = O.matvec(h, host(Xd.to(torch.bfloat16)))
    assert_elementwise(host(Yb), want_b, leaves, 2e-2, "BF16")
    # export returns what was imported
    rk, U, E, S, D = G.export()
    r0, U0, E0, S0, D0 = factors.oracle_to_import(h)
    np.testing.assert_array_equal(rk, r0)
    for a, b in ((U, U0), (E, E0), (S, S0), (D, D0)):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("kind", ["heat32_strong", "heat32_weak", "ragged", "tiny", "weak_k48"])
@pytest.mark.parametrize("nrhs", [1, 7, 33, 130])
def test_matvec_compensated_fp32_matches_oracle(h2, kind, nrhs):
    """H2_FP32C: FP32 factor storage, every value carried as a float pair hi + lo.  The stored
    factors' rounding (2^-24 relative per entry) is the only reduced-precision step, so each
    stage's output errs by a few 2^-24 of the sum of its terms' magnitudes; bound 1e-6 relative
    (element-wise, per column and per leaf block) against the FP64 oracle's product of the
    FP64 factors, the accuracy the FP64 construction itself is built to."""
    h, n, leaf, adm = _oracle_h2(kind)
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(h), keep_fp32=True)
    X = W.rhs(n * n, nrhs, 19)
    want = O.matvec(h, X)
    Xd = dev(X)
    Yd = torch.full_like(Xd, float("nan"))
    G.matvec(Xd, Yd, nrhs, h2.H2_FP32C)
    torch.cuda.synchronize()
    c, b = assert_elementwise(host(Yd), want, leaf_index_sets(h.tree), 1e-6, "FP32C")
    print(f"FP32C {kind} nrhs {nrhs}: worst column {c:.1e}, worst leaf block {b:.1e}")


def test_matvec_compensated_fp32_host_buffers(h2):
    """H2_FP32C through h2_matvec_host: FP64 host X and Y, the same result as the device call."""
    h, n, leaf, adm = _oracle_h2("heat32_strong")
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(h), keep_fp32=True)
    X = W.rhs(n * n, 9, 21)
    Xh = np.ascontiguousarray(X.T)
    Yh = np.full_like(Xh, np.nan)
    G.matvec_host(Xh, Yh, 9, h2.H2_FP32C)
    Yd = torch.empty((9, n * n), dtype=torch.float64, device="cuda")
    G.matvec(dev(X), Yd, 9, h2.H2_FP32C)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Yh, Yd.cpu().numpy())
    assert_elementwise(Yh.T, O.matvec(h, X), leaf_index_sets(h.tree), 1e-6, "FP32C host")


@pytest.mark.parametrize("nrhs", [64, 130, 300])
def test_matvec_wide_transfer_blocks(h2, nrhs):
    """Ranks above 32 in the tree sweeps (transfer blocks up to 48 x 48) with many right-hand
    sides, FP64 and FP32, against the oracle's matvec of the same H^2."""
    h, n, leaf, adm = _oracle_h2("weak_k48")
    assert max(int(k.max()) for k in h.k) > 32
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(h), keep_fp32=True)
    X = W.rhs(n * n, nrhs, 13)
    want = O.matvec(h, X)
    Xd = dev(X)
    Yd = torch.full_like(Xd, float("nan"))
    G.matvec(Xd, Yd, nrhs, h2.H2_FP64)
    torch.cuda.synchronize()
    leaves = leaf_index_sets(h.tree)
    assert_elementwise(host(Yd), want, leaves, 1e-12, "FP64")
    Y32 = torch.full((nrhs, n * n), float("nan"), dtype=torch.float32, device="cuda")
    G.matvec(Xd.float(), Y32, nrhs, h2.H2_FP32)
    torch.cuda.synchronize()
    assert_elementwise(host(Y32), want, leaves, 1e-5, "FP32")


@pytest.mark.parametrize("kind", ["heat32_strong", "ragged", "heat64", "weak_k48"])
@pytest.mark.parametrize("nrhs", [64, 130])
def test_matvec_tensor_cores_match_oracle(h2, kind, nrhs):
    """nrhs >= 64 in BF16 / TF32 runs the near field on tcgen05 (FP32 accumulation in tensor memory).
    Bounds against the FP64 oracle, element-wise: BF16 2e-2 (8-bit mantissa), TF32 2e-3 (10-bit
    mantissa), split TF32 3e-5 (two TF32 parts of each operand, three products: the dropped lo*lo
    term and the rounding of the 13-bit remainder to TF32 leave about 2^-21 per product, and a
    column's error over up to ~1,500 terms grows like sqrt(K) 2^-21 ~ 2e-5; measured up to 1.3e-5).
    The BF16 and TF32 references are the oracle products of the rounded inputs (BF16 inputs; TF32
    rounds the FP32 inputs inside the kernel, so its reference is the unrounded input).  weak_k48
    has ranks in (32, 48]: couplings up to 48 x 48 run the three-stage 48 x 48 operand ring."""
    if kind == "heat64":
        mask, op = _heat_problem(64, 256, 1002)
        h = O.build(op, W.grid_coords(64), 64, ADM_STRONG, 0.7, 1e-6, 32, 32, 16, 256, True, 7)[0]
        n, leaf, adm = 64, 64, ADM_STRONG
    else:
        h, n, leaf, adm = _oracle_h2(kind)
    if kind == "weak_k48":
        assert max(int(k.max()) for k in h.k) > 32
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(h), keep_fp32=True, keep_bf16=True)
    X = W.rhs(n * n, nrhs, 21)
    want = O.matvec(h, X)
    leaves = leaf_index_sets(h.tree)
    Xd = dev(X)
    Yb = torch.full((nrhs, n * n), float("nan"), dtype=torch.float32, device="cuda")
    G.matvec(Xd.to(torch.bfloat16), Yb, nrhs, h2.H2_BF16)
    Yt = torch.full((nrhs, n * n), float("nan"), dtype=torch.float32, device="cuda")
    G.matvec(Xd.float(), Yt, nrhs, h2.H2_TF32)
    torch.cuda.synchronize()
    assert G.device_status() == h2.H2_OK
    want_b = O.matvec(h, host(Xd.to(torch.bfloat16)))
    assert_elementwise(host(Yb), want_b, leaves, 2e-2, "BF16")
    assert_elementwise(host(Yt), want, leaves, 2e-3, "TF32")
    # split TF32 (hi*hi + hi*lo + lo*hi): FP32-grade, about 22 significant bits per product
    Y3 = torch.full((nrhs, n * n), float("nan"), dtype=torch.float32, device="cuda")
    G.matvec(Xd.float(), Y3, nrhs, h2.H2_TF32X3)
    torch.cuda.synchronize()
    assert G.device_status() == h2.H2_OK
    assert_elementwise(host(Y3), want, leaves, 3e-5, "TF32X3")
    # same inputs through the SIMT path (nrhs <= 4 columns at a time) agree column by column
    Y4 = torch.empty((4, n * n), dtype=torch.float32, device="cuda")
    G.matvec(Xd[:4].float(), Y4, 4, h2.H2_FP32)
    torch.cuda.synchronize()
    assert_elementwise(host(Yt[:4]), host(Y4), leaves, 2e-3, "TF32 vs FP32")


def test_matvec_leading_dimensions_and_empty(h2):
    h, n, leaf, adm = _oracle_h2("heat32_strong")
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(h))
    N = n * n
    X = W.rhs(N, 4, 1)
    Xp = torch.zeros((4, N + 5), dtype=torch.float64, device="cuda")
    Xp[:, :N] = dev(X)
    Yp = torch.zeros((4, N + 3), dtype=torch.float64, device="cuda")
    G.matvec(Xp, Yp, 4, h2.H2_FP64, ldx=N + 5, ldy=N + 3)
    torch.cuda.synchronize()
    assert rel(host(Yp[:, :N]), O.matvec(h, X)) < 1e-12
    assert float(Yp[:, N:].abs().max()) == 0.0
    G.matvec(Xp, Yp, 0, h2.H2_FP64)          # nrhs = 0 is a no-op
    with pytest.raises(h2.H2Error):
        G.matvec(Xp, Yp, 4, h2.H2_FP64, ldx=N - 1)
    with pytest.raises(h2.H2Error):
        G.matvec(Xp.float(), Yp.float(), 4, h2.H2_FP32)   # FP32 copy not kept


def _gpu_build(h2, op_gpu, n, leaf, adm, tol, kmax, q0, b_inc, q_max, adaptive, seed, norm_est=0.0):
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    opts = h2.default_opts(kmax=kmax, q0=q0, b_inc=b_inc, q_max=q_max, adaptive=int(adaptive), seed=seed,
                           norm_est=norm_est)
    return h2.H2.build(op_gpu, tree, tol, opts)


def gpu_apply(h2, G, N):
    def f(v):
        vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
        yd = torch.empty_like(vd)
        G.matvec(vd, yd, 1)
        torch.cuda.synchronize()
        return yd.cpu().numpy()
    return f


def norm2_rel(apply_a, apply_b, N, ref_norm):
    """||A - B||_2 / ref_norm by power iteration (symmetric difference)."""
    v0 = np.random.default_rng(17).standard_normal(N)
    return O.power_norm(lambda v: apply_a(v) - apply_b(v), N, v0) / ref_norm


@pytest.mark.parametrize("which", ["low_rank", "block_diag", "hss", "strong"])
def test_build_exact_recovery_planted(h2, which):
    if which == "low_rank":
        n, leaf, adm, q0, kmax = 24, 16, ADM_STRONG, 32, 16
        A = planted.global_low_rank(n * n, 9, 1)
    else:
        n, leaf = 16, 8
        tree = ClusterTree(W.grid_coords(n), leaf)
        if which == "block_diag":
            adm, q0, kmax = ADM_WEAK, 32, 16
            A = planted.block_diagonal(tree, 2)
        elif which == "hss":
            adm, q0, kmax = ADM_WEAK, 8, 16
            A = planted.planted_h2(tree, Partition(tree, ADM_WEAK, 0.7), 4, 0, 3)
        else:
            adm, q0, kmax = ADM_STRONG, 16, 16
            A = planted.planted_h2(tree, Partition(tree, ADM_STRONG, 0.7), 3, 2, 4)
    N = n * n
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dop = h2.DenseOperator(Ad)
    # a fixed norm: the planted matrices are indefinite, where the power-iteration stop is rounding-sensitive
    nrm = float(np.linalg.norm(A, 2))
    G = _gpu_build(h2, dop, n, leaf, adm, 1e-6, kmax, q0, 16, 256, True, 5, norm_est=nrm)
    ho, res = O.build(O.DenseOperator(A), W.grid_coords(n), leaf, adm, 0.7, 1e-6, kmax, q0, 16, 256, True, 5,
                      norm_est=nrm)
    st = G.stats()
    X = W.rhs(N, 6, 2)
    Xd = dev(X)
    Yd = torch.empty_like(Xd)
    G.matvec(Xd, Yd, 6)
    torch.cuda.synchronize()
    assert rel(host(Yd), A @ X) < 1e-12
    assert st["samples"] == res.samples - res.norm_its
    for l in range(1, ho.tree.L + 1):
        assert st["max_rank"][l] == int(ho.k[l].max())
        assert st["range_probes"][l] == res.range_probes[l]


@pytest.mark.parametrize("adm", [ADM_STRONG, ADM_WEAK])
def test_build_heat_small_matches_oracle(h2, adm):
    c = W.SMALL_N32
    p, b = c["problem"], c["build"]
    mask, op = _heat_problem(p.n, p.m, p.sensor_seed)
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, mask)
    G = _gpu_build(h2, gop, p.n, b.leaf, adm, b.tol, b.kmax, b.q0, b.b_inc, b.q_max, b.adaptive, b.seed)
    ho, res = O.build(op, W.grid_coords(p.n), b.leaf, adm, 0.7, b.tol, b.kmax, b.q0, b.b_inc, b.q_max,
                      b.adaptive, b.seed)
    st = G.stats()
    assert st["samples"] == res.samples - res.norm_its
    assert abs(st["norm_est"] - res.norm_est) <= 1e-10 * res.norm_est
    for l in range(ho.tree.L + 1):
        assert st["max_rank"][l] == int(ho.k[l].max())
    nH = res.norm_est
    g = gpu_apply(h2, G, p.N)
    d = norm2_rel(g, lambda v: O.matvec(ho, v), p.N, nH)
    e_gpu = norm2_rel(g, op, p.N, nH)
    e_or = norm2_rel(lambda v: O.matvec(ho, v), op, p.N, nH)
    if adm == ADM_STRONG:
        assert st["tol_met"] == 1
        assert e_gpu < b.tol and e_or < b.tol and d < b.tol
    else:
        assert st["tol_met"] == 0      # rank cap 16 binds on the weak partition
        assert abs(e_gpu - e_or) < 0.05 * e_or


def test_build_heat_adaptive_matches_oracle(h2):
    """Adaptive probing at 64 x 64 (leaf 64, strong 0.7): per-level probe counts equal the oracle's."""
    n, m = 64, 256
    mask, op = _heat_problem(n, m, 1002)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    G = _gpu_build(h2, gop, n, 64, ADM_STRONG, 1e-6, 32, 32, 16, 256, True, 7)
    ho, res = O.build(op, W.grid_coords(n), 64, ADM_STRONG, 0.7, 1e-6, 32, 32, 16, 256, True, 7)
    st = G.stats()
    assert st["samples"] == res.samples - res.norm_its
    for l in range(1, ho.tree.L + 1):
        assert st["range_probes"][l] == res.range_probes[l]
        assert st["proj_probes"][l] == res.proj_probes[l]
        assert st["max_rank"][l] == int(ho.k[l].max())
    g = gpu_apply(h2, G, n * n)
    assert norm2_rel(g, op, n * n, res.norm_est) < 1e-6
    assert norm2_rel(g, lambda v: O.matvec(ho, v), n * n, res.norm_est) < 1e-6
    assert abs(st["norm_est"] - res.norm_est) <= 1e-10 * res.norm_est


def test_operator_failure_is_reported(h2):
    """An operator that fails on its third call aborts the build with OP_FAILED."""
    calls = {"n": 0}
    A = torch.eye(256, dtype=torch.float64, device="cuda")
    dop = h2.DenseOperator(A)

    def bad(X, ldx, Y, ldy, nrhs, stream):
        calls["n"] += 1
        if calls["n"] == 3:
            return 5
        return h2.lib().h2_dense_op_apply(dop.ctx, 256, nrhs, X, ldx, Y, ldy, stream)

    op = h2.PyOperator(256, bad)
    tree = h2.Tree(W.grid_coords(16), 8, ADM_STRONG, 0.7)
    with pytest.raises(h2.H2Error) as e:
        h2.H2.build(op, tree, 1e-6, h2.default_opts(norm_est=1.0))
    assert e.value.status == h2.H2_ERR_OP_FAILED


def test_nan_samples_are_reported(h2):
    N = 256
    A = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
    dop = h2.DenseOperator(A)
    tree = h2.Tree(W.grid_coords(16), 8, ADM_STRONG, 0.7)
    with pytest.raises(h2.H2Error) as e:
        h2.H2.build(dop, tree, 1e-6, h2.default_opts(norm_est=1.0))
    assert e.value.status == h2.H2_ERR_NAN


@pytest.mark.parametrize("mode,nrhs", [(0, 1), (1, 3), (1, 40), (3, 64)])
def test_repeated_matvec_graph_replay(h2, mode, nrhs):
    """Repeated calls with the same buffers are captured in a CUDA graph and replayed; the replay
    reads the buffers' current contents and equals a direct (profiled, uncaptured) launch."""
    ho, n, leaf, adm = _oracle_h2("ragged")
    tree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(tree, *factors.oracle_to_import(ho), keep_fp32=True, keep_bf16=True)
    N = n * n
    xdt = {0: torch.float64, 1: torch.float32, 3: torch.bfloat16}[mode]
    ydt = torch.float64 if mode == 0 else torch.float32
    X = torch.empty((nrhs, N), dtype=xdt, device="cuda")
    Y = torch.empty((nrhs, N), dtype=ydt, device="cuda")
    for call in range(4):
        X.copy_(dev(W.rhs(N, nrhs, 50 + call)).to(xdt))
        G.matvec(X, Y, nrhs, mode)            # direct, direct + capture, replay, replay
        torch.cuda.synchronize()
        R = torch.empty_like(Y)
        G.profile(True)                        # profiled calls always launch directly
        G.matvec(X, R, nrhs, mode)
        G.profile(False)
        torch.cuda.synchronize()
        G.profile_read()
        if nrhs > 4:
            assert torch.equal(R, Y)           # gather / tensor-core paths: fixed summation order
        else:
            tol = 1e-13 if mode == 0 else 1e-6   # atomics in the small-nrhs scatter
            assert float((R.double() - Y.double()).norm() / R.double().norm()) < tol


def test_allocation_failure_is_reported_without_leaks(h2):
    """A cap on the library's device memory makes a construction fail with H2_ERR_OOM part-way;
    every block it allocated is returned, and the next construction succeeds."""
    n = 64
    mask, op = _heat_problem(n, 256, 4)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    tree = h2.Tree(W.grid_coords(n), 64, ADM_STRONG, 0.7)
    # one full build first: the operator keeps its own workspaces (sized by the widest product)
    h2.H2.build(gop, tree, 1e-6, h2.default_opts()).close()
    torch.cuda.synchronize()
    before = h2.device_bytes()
    for extra in (1 << 16, 1 << 20, 8 << 20):
        h2.set_device_limit(before + extra)
        try:
            with pytest.raises(h2.H2Error) as e:
                h2.H2.build(gop, tree, 1e-6, h2.default_opts(global_rank=128 if extra == (8 << 20) else 0))
            assert e.value.status == h2.H2_ERR_OOM
        finally:
            h2.set_device_limit(0)
        assert h2.device_bytes() == before
    G = h2.H2.build(gop, tree, 1e-6, h2.default_opts())
    assert G.stats()["samples"] > 0
    G.close()
    assert h2.device_bytes() == before
