"""Plain CPU FP64 oracle of the H^2 Hessian construction and matvec.

TEST INFRASTRUCTURE.  This package is the slow, obviously-correct reference
that the CUDA library is checked against.  Only the tests, the smoke check
(`__graft_entry__.smoke`) and the benchmark's CPU-baseline leg may import it;
the library never does, and it shares no code with the library.  It is
written from the paper (arXiv 2003.10173): Section 3.1 (representation),
Section 3.2 (matvec, recompression, norms), Section 3.3 (construction from
Hessian-vector products), with numpy library primitives (QR, SVD, matmul)
as steps.
"""
from .h2 import (H2Matrix, assemble, basis_threshold, expand_dense, factor_arrays, frobenius_norm,
                 from_factor_arrays, matvec, power_norm, storage_entries)
from .heat import DenseOperator, HeatHessian, LowRankOperator
from .peel import PeelResult, TreeOperator, apply_pieces, global_lowrank, norm2_estimate, peel, psd_cholesky
from .tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition
from .update import compress_dense, far_columns, lowrank_update


def build(op, coords, leaf, adm, eta, tol, kmax, q0, b_inc, q_max, adaptive, seed, norm_est=None,
          q_level=None, q_test=8, global_rank=0, ranks=None, q_exact=None, certified=False):
    """Full construction: tree, partition, peeling, assembly.  Returns (h2, peel_result).
    ranks, q_exact: optional basis ranks and range-probe counts to replay (see assemble, peel).
    certified: range bases without the passing test's columns (see peel)."""
    tree = ClusterTree(coords, leaf)
    part = Partition(tree, adm, eta)
    res = peel(op, tree, tol, q0, b_inc, q_max, adaptive, seed, norm_est=norm_est, q_level=q_level,
               q_test=q_test, global_rank=global_rank, q_exact=q_exact, certified=certified)
    res.tau_basis = basis_threshold(tol, res.norm_est, 1 << tree.L)
    h = assemble(tree, part, res, res.tau_basis, kmax, ranks=ranks)
    return h, res


def replay_build(op, coords, leaf, adm, eta, tol, kmax, seed, norm_est, range_probes, ranks):
    """Rank replay: the construction with every decision of another run given as data.
    range_probes[l] > 0 is the number of range-pass probes of level l (0: identity range, no
    range pass); norm_est the 2-norm estimate used; ranks[l][b] the basis rank of box b of
    level l.  The peeling then runs with exactly these probe counts (no adaptive test) and
    the truncations keep exactly these ranks; everything else is the ordinary method."""
    return build(op, coords, leaf, adm, eta, tol, kmax, 1, 1, 1 << 30, False, seed, norm_est=norm_est,
                 ranks=ranks, q_exact=[int(q) for q in range_probes])
