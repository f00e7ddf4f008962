"""Oracle: cluster tree, cuts, neighbour lists and interaction lists (Section 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3 defines the tree: level 0 is one box enclosing the domain; each box
is bisected along every dimension into 2^d children; empty boxes are dropped;
a box is split only while it holds more than m points.  Neighbours are boxes of
the same level whose closed boxes touch (up to 3^d, the box itself included);
the interaction list of a box is the set of children of its parent's neighbours
that are not its own neighbours (up to 6^d - 3^d boxes).

Readings where the paper is silent (Section 3 assumes a uniform distribution):
  * root box: the unit cube when all points lie in [0,1]^d (the paper's domain),
    otherwise the smallest cube anchored at the coordinate-wise minimum;
  * boxes are identified by integer coordinates on a 2^21 grid per dimension;
    a point on a split plane belongs to the upper child; the top face clamps;
  * points are ordered by Morton key, ties by original index (stable), so every
    index set I_tau is a contiguous range of the permuted order;
  * adaptive trees: the "cut" at level l holds the level-l boxes plus the leaves
    of coarser levels ("carried leaves").  A carried leaf is its own parent and
    its own only child.  Neighbours in a cut are boxes whose closed boxes touch,
    whatever their levels.  This keeps beta in int(alpha) <=> alpha in int(beta)
    and covers every matrix entry exactly once.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

QBITS = 21  # bits per coordinate of the integer grid


def root_cube(x: np.ndarray):
    """Root box (reading, see module docstring): returns (lo, side)."""
    n, d = x.shape
    if n == 0 or (x.min() >= 0.0 and x.max() <= 1.0):
        return np.zeros(d), 1.0
    lo = x.min(axis=0)
    side = float((x.max(axis=0) - lo).max())
    if not side > 0.0:
        side = 1.0
    return lo, side


def quantize(x: np.ndarray, lo: np.ndarray, side: float) -> np.ndarray:
    """Integer grid coordinates q = min(floor((x - lo)/side * 2^21), 2^21 - 1).

    Each operation is one correctly rounded FP64 operation (subtract, divide,
    exact power-of-two scale), so any IEEE implementation gets the same q.
    """
    t = (x - lo) / side
    q = np.floor(t * float(1 << QBITS))
    q = np.clip(q, 0, (1 << QBITS) - 1)
    return q.astype(np.int64)


def morton(q: np.ndarray) -> np.ndarray:
    """Morton key: bit b of coordinate t goes to bit b*d + t."""
    n, d = q.shape
    key = np.zeros(n, dtype=np.int64)
    for b in range(QBITS):
        for t in range(d):
            key |= ((q[:, t] >> b) & 1) << (b * d + t)
    return key


@dataclass
class Box:
    level: int
    index: int          # position within its level (Morton order)
    gid: int            # global id: level offset + index
    start: int          # I_tau = [start, end) in the permuted order
    end: int
    anchor: tuple       # integer box coordinates at its own level
    parent: int         # index of the parent within level-1 (-1 at the root)
    leaf: bool


@dataclass
class Tree:
    d: int
    n: int
    perm: np.ndarray         # perm[i] = original index of the i-th sorted point
    q: np.ndarray            # integer coordinates, sorted order
    levels: list             # levels[l] = list of Box
    cuts: list               # cuts[l] = list of (level, index) sorted by start
    cut_parent: list         # cut_parent[l][i] = index in cut l-1 (l >= 1)
    near: list               # near[l][i] = sorted list of cut-l indices
    inter: list              # inter[l][i] = sorted list of cut-l indices
    lo: np.ndarray
    side: float

    @property
    def L(self) -> int:
        return len(self.levels) - 1

    def box(self, l: int, i: int) -> Box:
        lev, idx = self.cuts[l][i]
        return self.levels[lev][idx]

    def rng(self, l: int, i: int):
        b = self.box(l, i)
        return b.start, b.end

    def n_boxes(self) -> int:
        return sum(len(v) for v in self.levels)


def build_levels(keys_sorted: np.ndarray, q_sorted: np.ndarray, d: int, m: int,
                 uniform_depth: int):
    """Recursive 2^d-ary subdivision (Section 3), on Morton-sorted points.

    A box is split iff it holds more than m points (adaptive), or iff its level
    is below uniform_depth (uniform mode).  Children are the non-empty runs of
    the next Morton prefix.  Splitting stops at the grid resolution.
    """
    n = keys_sorted.shape[0]
    levels = [[Box(0, 0, 0, 0, n, tuple([0] * d), -1, True)]]
    gid = 1
    l = 0
    while True:
        nxt = []
        shift = d * (QBITS - l - 1)
        for bi, b in enumerate(levels[l]):
            count = b.end - b.start
            split = (l < uniform_depth) if uniform_depth > 0 else (count > m)
            split = split and l < QBITS and count > 0
            if not split:
                b.leaf = True
                continue
            b.leaf = False
            pref = keys_sorted[b.start:b.end] >> shift
            cuts = np.flatnonzero(np.diff(pref)) + 1
            bounds = [0] + cuts.tolist() + [count]
            for s, e in zip(bounds[:-1], bounds[1:]):
                start = b.start + s
                anchor = tuple(int(v) for v in (q_sorted[start] >> (QBITS - l - 1)))
                nxt.append(Box(l + 1, len(nxt), gid, start, b.start + e, anchor, bi, True))
                gid += 1
        if not nxt:
            break
        levels.append(nxt)
        l += 1
    return levels


def touch(bt: Box, bs: Box, l: int) -> bool:
    """Closed boxes of two cut-l entries overlap ("overlapping boundaries")."""
    st, ss = l - bt.level, l - bs.level
    for t in range(len(bt.anchor)):
        lo_t, hi_t = bt.anchor[t] << st, ((bt.anchor[t] + 1) << st) - 1
        lo_s, hi_s = bs.anchor[t] << ss, ((bs.anchor[t] + 1) << ss) - 1
        if lo_t > hi_s + 1 or lo_s > hi_t + 1:
            return False
    return True


def build_tree(x: np.ndarray, leaf_size: int, uniform_depth: int = 0) -> Tree:
    """Cluster tree, cuts, neighbour lists and interaction lists (Section 3)."""
    x = np.asarray(x, dtype=np.float64)
    n, d = x.shape
    lo, side = root_cube(x)
    q = quantize(x, lo, side)
    key = morton(q)
    perm = np.argsort(key, kind="stable")
    ks, qs = key[perm], q[perm]
    levels = build_levels(ks, qs, d, leaf_size, uniform_depth)
    L = len(levels) - 1

    # cuts: level-l boxes plus carried leaves, ordered by their first point
    cuts, where = [], []
    for l in range(L + 1):
        ent = [(l, b.index) for b in levels[l]]
        for lev in range(l):
            ent += [(lev, b.index) for b in levels[lev] if b.leaf]
        ent.sort(key=lambda e: levels[e[0]][e[1]].start)
        cuts.append(ent)
        where.append({e: i for i, e in enumerate(ent)})

    cut_parent = [None]
    for l in range(1, L + 1):
        par = []
        for lev, idx in cuts[l]:
            b = levels[lev][idx]
            if lev == l:
                par.append(where[l - 1][(l - 1, b.parent)])
            else:
                par.append(where[l - 1][(lev, idx)])
        cut_parent.append(par)

    near = [[[0]]]
    inter = [[[]]]
    for l in range(1, L + 1):
        kids = [[] for _ in cuts[l - 1]]
        for i, p in enumerate(cut_parent[l]):
            kids[p].append(i)
        nl, il = [], []
        for i, (lev, idx) in enumerate(cuts[l]):
            bi = levels[lev][idx]
            cand = []
            for s in near[l - 1][cut_parent[l][i]]:
                cand += kids[s]
            nn, ii = [], []
            for j in sorted(cand):
                lj, xj = cuts[l][j]
                (nn if touch(bi, levels[lj][xj], l) else ii).append(j)
            nl.append(nn)
            il.append(ii)
        near.append(nl)
        inter.append(il)
    return Tree(d, n, perm, qs, levels, cuts, cut_parent, near, inter, lo, side)


def admissible_pairs(tree: Tree, l: int):
    """Admissible pairs of cut l: (alpha, beta) with beta in int(alpha),
    alpha in cut order, beta in cut order."""
    return [(a, b) for a in range(len(tree.cuts[l])) for b in tree.inter[l][a]]


def near_pairs(tree: Tree, l: int):
    """Inadmissible (neighbour) pairs of cut l (Section 4.1.3)."""
    return [(a, b) for a in range(len(tree.cuts[l])) for b in tree.near[l][a]]
