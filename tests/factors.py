"""Conversion of an oracle H^2 matrix into the flat factor layout of h2_import.

Layout (include/h2.h): ranks of every box (levels 0..L, 2^l boxes each); leaf
bases |t| x k_t; transfer matrices k_c x k_parent for every box c of levels
1..L; couplings of the lower far blocks per level in partition order; near
blocks with t >= s in partition order; all column-major FP64.
"""
import numpy as np


def oracle_to_import(h):
    tree, part = h.tree, h.part
    L = tree.L
    ranks = np.concatenate([np.asarray(h.k[l], dtype=np.int32) for l in range(L + 1)])
    U = [h.U[t].flatten(order="F") for t in range(1 << L)] if L >= 0 else []
    E = []
    for l in range(1, L + 1):
        for c in range(1 << l):
            if l == 1:
                kc = int(h.k[1][c])
                E.append(np.zeros(0))          # parent is the root, which has rank 0
                continue
            E.append(h.E[(l, c)].flatten(order="F"))
    S = []
    for l in range(1, L + 1):
        for t, s in part.far[l]:
            if t > s:
                S.append(h.S[(l, int(t), int(s))].flatten(order="F"))
    D = []
    for t, s in part.near:
        if t >= s:
            D.append(h.D[(int(t), int(s))].flatten(order="F"))
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0)
    return ranks, cat(U), cat(E), cat(S), cat(D)
