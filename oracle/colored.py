"""Strong-structure coloured sampling (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Section 3.3 samples blocks of the matrix with patterned random probes, level by
level from coarse to fine, after removing what the coarser levels already
represent; one probe block serves several blocks at once as long as no other
block interferes with the rows that are read, and the sampling blocks may be
larger than the destination blocks (the weak structure of the paper's own
implementation, `peel.py`) or be the destination blocks themselves.  The number
of products per level is C_l k: C_l counts the probe blocks needed to sample all
blocks of level l without interference.  This module is the second choice: the
destination (strong-admissibility) far blocks of every level are sampled
directly, and interference is avoided by colouring.

Readings (the paper describes the structure in words only):

* Remaining blocks.  After the far blocks of the levels above l are removed, the
  residual has, at the box granularity of level l, nonzero blocks only on the
  pairs (t, s) that the partition visits at level l: the far blocks of level l
  and the inadmissible pairs that are split further.  V_l(t) lists them.
* Range pass.  Every lower far pair (t > s) of level l is sampled through probes
  on the rows of its column box s; the column boxes are coloured greedily in box
  order so that no row box t sees two boxes of one colour in V_l(t) (a
  distance-2 colouring of the visited pairs).  Colour c owns q probe columns
  [c q, (c + 1) q): Gaussian (stream `colored`, the level as key) on the rows of
  its boxes, zero elsewhere.  One product with all colours' columns gives
  Y[t, cols of colour(s)] = H[t, s] Omega[s] for every lower far pair, and
  Q_ts = the signed Q factor of that block (q fixed, below every box size).
* Projection pass.  The pairs are given probe slots greedily in (t, s) order:
  a pair may join a slot unless the slot already holds a pair with the same row
  box t, a pair whose row box t2 has s in V_l(t2), or a pair whose column box s2
  is in V_l(t).  Slot j owns q columns; its pairs put Q_ts on the rows of t.
  One product gives Z_ts = H[s, t] Q_ts on the rows of s, and the piece of the
  pair is H[t, s] ~ Q_ts Z_ts^T (H[s, t] ~ Z_ts Q_ts^T).
* Leaf pass.  The leaves are coloured the same way over the near pairs;
  colour c owns leaf_max columns holding identity blocks on its leaves.  After
  all pieces are removed, the near block (t, s) is read from the rows of t in
  the columns of colour(s); diagonal blocks are symmetrised.
* Assembly.  The result is the sampled approximation K (pieces and near
  blocks) in H^2 form: nested bases from truncated SVDs of the far block rows
  of K at the construction's basis threshold, couplings by projection
  (`update.compress_dense`, the definition written out).
"""
from __future__ import annotations

import numpy as np

from . import rng
from .h2 import basis_threshold
from .peel import TreeOperator, norm2_estimate, range_basis
from .tree import ClusterTree, Partition
from .update import compress_dense

STREAM_COLORED = rng.STREAM_COLORED


def visited_pairs(tree: ClusterTree, part: Partition):
    """V[l][t]: sorted boxes s such that the partition visits (t, s) at level l (a far block of
    level l, or an inadmissible pair that is split further or is a near block)."""
    V = [dict() for _ in range(tree.L + 1)]
    stack = [(0, 0, 0)]
    while stack:
        l, t, s = stack.pop()
        V[l].setdefault(t, set()).add(s)
        if part.admissible(l, t, s) or l == tree.L:
            continue
        for ct in (2 * t, 2 * t + 1):
            for cs in (2 * s, 2 * s + 1):
                stack.append((l + 1, ct, cs))
    return [{t: sorted(v) for t, v in d.items()} for d in V]


def color_boxes(Vl: dict, boxes) -> dict:
    """Greedy distance-2 colouring of the given boxes (in increasing order) over the visited
    pairs Vl: boxes s and s2 conflict when some t has both in Vl[t]."""
    color = {}
    for s in sorted(boxes):
        used = set()
        for t in Vl.get(s, ()):            # Vl is symmetric: s in Vl[t] <=> t in Vl[s]
            for s2 in Vl.get(t, ()):
                if s2 in color:
                    used.add(color[s2])
        c = 0
        while c in used:
            c += 1
        color[s] = c
    return color


def pair_slots(pairs, Vl: dict) -> list:
    """Greedy probe slots of the lower far pairs (in the given order) for the projection pass."""
    slots = []            # per slot: (row boxes, column boxes)
    out = []
    for t, s in pairs:
        Vt = set(Vl.get(t, ()))
        Vs = set(Vl.get(s, ()))
        j = 0
        while j < len(slots):
            T, S = slots[j]
            if t not in T and not (Vs & T) and not (Vt & S):
                break
            j += 1
        if j == len(slots):
            slots.append((set(), set()))
        slots[j][0].add(t)
        slots[j][1].add(s)
        out.append(j)
    return out


class ColoredPlan:
    def __init__(self, tree: ClusterTree, part: Partition, q: int):
        L = tree.L
        self.q = q
        self.V = visited_pairs(tree, part)
        self.pairs, self.color, self.slot, self.ncolors, self.nslots = [], [], [], [], []
        for l in range(L + 1):
            pl = sorted((int(t), int(s)) for t, s in part.far[l] if t > s)
            col = color_boxes(self.V[l], {s for _, s in pl})
            sl = pair_slots(pl, self.V[l])
            self.pairs.append(pl)
            self.color.append(col)
            self.slot.append(sl)
            self.ncolors.append(1 + max(col.values()) if col else 0)
            self.nslots.append(1 + max(sl) if sl else 0)
            for t, _ in pl:
                m = tree.rows(l, t).stop - tree.rows(l, t).start
                if m <= q:
                    raise ValueError("coloured sampling needs q below every box with far blocks")
        self.leaf_color = color_boxes(self.V[L], range(1 << L))
        self.nleafcolors = 1 + max(self.leaf_color.values())
        self.leaf_max = tree.leaf_max

    def range_probes(self, l):
        return self.ncolors[l] * self.q

    def proj_probes(self, l):
        return self.nslots[l] * self.q

    def samples(self):
        return sum(self.range_probes(l) + self.proj_probes(l) for l in range(len(self.pairs))) + \
            self.nleafcolors * self.leaf_max


def apply_colored(pieces, levels, tree: ClusterTree, X: np.ndarray) -> np.ndarray:
    """K X (tree order) for the pieces of the given levels: H[t, s] ~ Q Z^T and H[s, t] ~ Z Q^T."""
    out = np.zeros_like(X)
    for l in levels:
        for t, s, Q, Z in pieces.get(l, ()):
            rt, rs = tree.rows(l, t), tree.rows(l, s)
            out[rt] += Q @ (Z.T @ X[rs])
            out[rs] += Z @ (Q.T @ X[rt])
    return out


class ColoredResult:
    def __init__(self):
        self.pieces = {}
        self.D = {}
        self.samples = 0
        self.norm_est = 0.0
        self.norm_its = 0
        self.range_probes = {}
        self.proj_probes = {}


def peel_colored(op, tree: ClusterTree, part: Partition, tol: float, q: int, seed: int, norm_est=None,
                 plan: ColoredPlan | None = None) -> ColoredResult:
    """Pieces of every level and the near blocks by coloured sampling (see the module notes)."""
    N, L = tree.N, tree.L
    plan = plan or ColoredPlan(tree, part, q)
    opt = TreeOperator(op, tree)
    res = ColoredResult()
    if norm_est is None:
        res.norm_est, res.norm_its = norm2_estimate(opt, N, seed)
    else:
        res.norm_est = float(norm_est)
    samples0 = opt.samples
    for l in range(1, L + 1):
        pl = plan.pairs[l]
        if not pl:
            continue
        below = range(1, l)
        ncol, nsl = plan.ncolors[l], plan.nslots[l]
        # range pass
        Om = np.zeros((N, ncol * q))
        cols = np.arange(ncol * q, dtype=np.uint64)
        for s, c in plan.color[l].items():
            r = tree.rows(l, s)
            rr = np.arange(r.start, r.stop, dtype=np.uint64)[:, None]
            cc = cols[c * q:(c + 1) * q][None, :]
            Om[r, c * q:(c + 1) * q] = rng.gaussian(seed, STREAM_COLORED, l, rr, cc)
        Y = opt(Om) - apply_colored(res.pieces, below, tree, Om)
        Qs = []
        for t, s in pl:
            c = plan.color[l][s]
            Qs.append(range_basis(Y[tree.rows(l, t), c * q:(c + 1) * q]))
        # projection pass
        Psi = np.zeros((N, nsl * q))
        for (t, s), j, Q in zip(pl, plan.slot[l], Qs):
            Psi[tree.rows(l, t), j * q:(j + 1) * q] = Q
        Zf = opt(Psi) - apply_colored(res.pieces, below, tree, Psi)
        res.pieces[l] = [(t, s, Q, Zf[tree.rows(l, s), j * q:(j + 1) * q].copy())
                         for (t, s), j, Q in zip(pl, plan.slot[l], Qs)]
        res.range_probes[l] = ncol * q
        res.proj_probes[l] = nsl * q
    # leaf pass
    lm = tree.leaf_max
    nlc = plan.nleafcolors
    Om = np.zeros((N, nlc * lm))
    for s, c in plan.leaf_color.items():
        r = tree.rows(L, s)
        m = r.stop - r.start
        Om[r.start + np.arange(m), c * lm + np.arange(m)] = 1.0
    Y = opt(Om) - apply_colored(res.pieces, range(1, L + 1), tree, Om)
    for t, s in part.near:
        t, s = int(t), int(s)
        if t < s:
            continue
        rt, rs = tree.rows(L, t), tree.rows(L, s)
        c = plan.leaf_color[s]
        D = Y[rt, c * lm:c * lm + (rs.stop - rs.start)].copy()
        if t == s:
            D = 0.5 * (D + D.T)
        res.D[(t, s)] = D
    res.samples = opt.samples - samples0
    return res


def dense_from_colored(tree: ClusterTree, part: Partition, res: ColoredResult) -> np.ndarray:
    """The sampled approximation K (tree order): pieces on the far blocks, near blocks as read."""
    L = tree.L
    K = np.zeros((tree.N, tree.N))
    for l, pcs in res.pieces.items():
        for t, s, Q, Z in pcs:
            rt, rs = tree.rows(l, t), tree.rows(l, s)
            B = Q @ Z.T
            K[rt, rs] = B
            K[rs, rt] = B.T
    for (t, s), D in res.D.items():
        rt, rs = tree.rows(L, t), tree.rows(L, s)
        K[rt, rs] = D
        if t != s:
            K[rs, rt] = D.T
    return K


def build_colored(op, coords, leaf, adm, eta, tol, kmax, q, seed, norm_est=None, ranks=None):
    """Coloured-sampling construction: tree, partition, sampling, H^2 form of K.
    Returns (H2Matrix, ColoredResult, ColoredPlan)."""
    tree = ClusterTree(coords, leaf)
    part = Partition(tree, adm, eta)
    plan = ColoredPlan(tree, part, q)
    res = peel_colored(op, tree, part, tol, q, seed, norm_est=norm_est, plan=plan)
    tau = basis_threshold(tol, res.norm_est, 1 << tree.L)
    h = compress_dense(tree, part, dense_from_colored(tree, part, res), tau, kmax, ranks=ranks)
    return h, res, plan
