"""Cluster tree and block partition (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

* Cluster tree: KD-tree binary space partition of the mesh nodes; the node
  ordering it induces keeps spatially close nodes adjacent, which makes large
  blocks smooth (Section 4.2, Section 4.4).  Reading of the unstated rules: every
  box of a level is split while the largest box of that level exceeds the
  leaf size, so all leaves share one depth L; the split coordinate is the
  longer side of the box's bounding box (ties: x); points are ordered by
  (coordinate, original index) and the first floor(|t|/2) go to child 0.
* Admissibility (Section 2, Section 3.1, Table 1): WEAK admits every pair t != s
  (recursion from (root, root) then only reaches sibling pairs: the HSS
  partition); STRONG(eta) admits t != s with
  max(diam t, diam s) <= eta * dist(t, s) on axis-aligned bounding boxes.
* Block tree: recursion from (root, root); an admissible pair is a far
  (low-rank) block, an inadmissible leaf pair is a near (dense) block, and any
  other pair is split into its four child pairs (Section 3.1: dense blocks only
  at the leaf level).

Boxes are numbered per level, 0..2^l-1, in tree order (children of box i at
level l are boxes 2i and 2i+1 at level l+1).
"""
from __future__ import annotations

import math

import numpy as np

ADM_WEAK = 0
ADM_STRONG = 1


class ClusterTree:
    def __init__(self, coords: np.ndarray, leaf: int):
        coords = np.asarray(coords, dtype=np.float64)
        N, dim = coords.shape
        if N < 1 or leaf < 2:
            raise ValueError("need N >= 1 and leaf >= 2")
        self.N, self.dim, self.leaf = N, dim, leaf
        L = 0
        while -(-N // (1 << L)) > leaf:
            L += 1
        self.L = L
        perm = np.arange(N, dtype=np.int64)
        # starts[l][i], sizes[l][i]: range of box i of level l in tree order
        self.starts = [np.array([0], dtype=np.int64)]
        self.sizes = [np.array([N], dtype=np.int64)]
        for l in range(L):
            st, sz = self.starts[l], self.sizes[l]
            nst = np.empty(2 * len(st), dtype=np.int64)
            nsz = np.empty(2 * len(st), dtype=np.int64)
            for i in range(len(st)):
                a, m = int(st[i]), int(sz[i])
                idx = perm[a:a + m]
                pts = coords[idx]
                ext = pts.max(axis=0) - pts.min(axis=0)
                d = int(np.argmax(ext))            # first maximum: ties go to x
                order = np.lexsort((idx, pts[:, d]))  # by coordinate, then original index
                perm[a:a + m] = idx[order]
                h = m // 2
                nst[2 * i], nsz[2 * i] = a, h
                nst[2 * i + 1], nsz[2 * i + 1] = a + h, m - h
            self.starts.append(nst)
            self.sizes.append(nsz)
        self.perm = perm                           # tree position -> original index
        self.iperm = np.empty(N, dtype=np.int64)
        self.iperm[perm] = np.arange(N, dtype=np.int64)
        self.lo, self.hi = [], []
        for l in range(L + 1):
            lo = np.empty((len(self.starts[l]), dim))
            hi = np.empty((len(self.starts[l]), dim))
            for i, (a, m) in enumerate(zip(self.starts[l], self.sizes[l])):
                pts = coords[perm[a:a + m]]
                lo[i], hi[i] = pts.min(axis=0), pts.max(axis=0)
            self.lo.append(lo)
            self.hi.append(hi)

    def rows(self, level: int, box: int) -> slice:
        a = int(self.starts[level][box])
        return slice(a, a + int(self.sizes[level][box]))

    def diam(self, level: int, box: int) -> float:
        return float(np.linalg.norm(self.hi[level][box] - self.lo[level][box]))

    def dist(self, level: int, t: int, s: int) -> float:
        gap = np.maximum(0.0, np.maximum(self.lo[level][s] - self.hi[level][t],
                                         self.lo[level][t] - self.hi[level][s]))
        return float(np.linalg.norm(gap))

    @property
    def leaf_max(self) -> int:
        return int(self.sizes[self.L].max())


class Partition:
    """Far blocks per level and near (leaf) blocks, both triangles, sorted by (t, s)."""

    def __init__(self, tree: ClusterTree, adm: int, eta: float):
        self.tree, self.adm, self.eta = tree, adm, eta
        far = [[] for _ in range(tree.L + 1)]
        near = []
        stack = [(0, 0, 0)]
        while stack:
            l, t, s = stack.pop()
            if self.admissible(l, t, s):
                far[l].append((t, s))
            elif l == tree.L:
                near.append((t, s))
            else:
                for ct in (2 * t, 2 * t + 1):
                    for cs in (2 * s, 2 * s + 1):
                        stack.append((l + 1, ct, cs))
        self.far = [np.array(sorted(f), dtype=np.int64).reshape(-1, 2) for f in far]
        self.near = np.array(sorted(near), dtype=np.int64).reshape(-1, 2)
        # far_of[l][t]: column boxes s of the far blocks (t, s) of level l
        self.far_of = []
        for l, f in enumerate(self.far):
            d = {}
            for t, s in f:
                d.setdefault(int(t), []).append(int(s))
            self.far_of.append(d)

    def admissible(self, l: int, t: int, s: int) -> bool:
        if t == s:
            return False
        if self.adm == ADM_WEAK:
            return True
        tr = self.tree
        d = tr.dist(l, t, s)
        return max(tr.diam(l, t), tr.diam(l, s)) <= self.eta * d

    @staticmethod
    def pair_level(level: int, t: int, s: int) -> int:
        """Level of the sibling pair that contains block (t, s): one below the lowest common ancestor."""
        lvl = level
        while t != s:
            t >>= 1
            s >>= 1
            lvl -= 1
        return lvl + 1
