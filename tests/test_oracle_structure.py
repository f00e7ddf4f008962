"""Pins of the oracle's tree, lists, graph and colouring against what the paper fixes.

CPU only.  The worked 1D example (depth-3 tree over [0,1]) gives exact counts and
colour classes at every stage; the general bounds of Section 4.1.4 and the
coverage/symmetry invariants of the H^1 tessellation pin the rest.
"""
import itertools
import json
import os

import numpy as np
import pytest

import hm_workloads as W
from oracle import graph as og
from oracle import tree as ot

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def worked_tree():
    x = ((np.arange(64) + 0.5) / 64)[:, None]
    return ot.build_tree(x, 8, uniform_depth=3)


def classes(tree, l, col):
    return sorted(sorted((1 << tree.box(l, b).level) + tree.box(l, b).index
                         for b in col.active(c)) for c in range(col.n_colors))


def chromatic_number(nv, edges):
    adj = [set() for _ in range(nv)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    for k in range(1, nv + 1):
        col = [-1] * nv

        def bt(i):
            if i == nv:
                return True
            for c in range(k):
                if all(col[w] != c for w in adj[i]):
                    col[i] = c
                    if bt(i + 1):
                        return True
            col[i] = -1
            return False
        if bt(0):
            return k
    return nv


def test_worked_example_levels():
    g = json.load(open(os.path.join(GOLD, "worked_example_1d.json")))
    t = worked_tree()
    assert t.L == 3
    assert [len(c) for c in t.cuts] == [1, 2, 4, 8]
    blocks2 = [((1 << 2) + a, (1 << 2) + b) for a, b in ot.admissible_pairs(t, 2)]
    assert sorted(blocks2) == sorted(tuple(p) for p in g["level2_admissible_blocks"])
    for l, key in ((2, "level2"), (3, "level3")):
        pairs = ot.admissible_pairs(t, l)
        col = og.color_level(t, l)
        ref = g[key]
        assert len(pairs) == ref["blocks"]
        assert col.n_vertices == ref["vertices"]
        assert col.n_edges == ref["edges"]
        assert col.n_colors == ref["colors"]
        assert classes(t, l, col) == sorted(ref["classes"])
    ref = g["leaf"]
    col = og.color_leaf(t)
    assert len(ot.near_pairs(t, 3)) == ref["blocks"]
    assert (col.n_vertices, col.n_edges, col.n_colors) == (ref["vertices"], ref["edges"], ref["colors"])
    assert classes(t, 3, col) == sorted(ref["classes"])


def test_worked_example_chromatic_number():
    """DSatur's 6 colours at level 3 are optimal (brute force over 12 vertices)."""
    t = worked_tree()
    pairs = ot.admissible_pairs(t, 3)
    pv, vb, vS = og.constraint_vertices(pairs, lambda a: sorted(t.near[3][a] + t.inter[3][a]))
    edges = og.brute_force_edges(vb.tolist(), vS)
    assert len(edges) == 54
    assert chromatic_number(len(vb), edges) == 6


def test_shared_vertex_example():
    """A_{8,11} and A_{9,11} share one constraint set (Fig. graph_strong_1d_lvl3)."""
    t = worked_tree()
    pairs = ot.admissible_pairs(t, 3)
    col = og.color_level(t, 3)
    heap = {(8 + a, 8 + b): i for i, (a, b) in enumerate(pairs)}
    assert col.pair_vertex[heap[(8, 11)]] == col.pair_vertex[heap[(9, 11)]]
    assert col.pair_vertex[heap[(8, 10)]] != col.pair_vertex[heap[(9, 11)]]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_native_edges_match_definition(seed):
    """The C edge builder equals the O(V^2) definition on random constraint sets."""
    rng = np.random.default_rng(seed)
    nbox = 25
    pairs, zs = [], {}
    for a in range(nbox):
        S = sorted(set(rng.choice(nbox, size=rng.integers(2, 9), replace=False).tolist()) | {a})
        zs[a] = S
        for b in S:
            if b != a and rng.random() < 0.6:
                pairs.append((a, b))
    col = og.color_pairs(pairs, lambda a: zs[a], nbox)
    pv, vb, vS = og.constraint_vertices(pairs, lambda a: zs[a])
    edges = og.brute_force_edges(vb.tolist(), vS)
    assert col.n_edges == len(edges)
    for u, v in edges:
        assert col.vertex_color[u] != col.vertex_color[v]
    deg = np.zeros(len(vb), dtype=int)
    for u, v in edges:
        deg[u] += 1
        deg[v] += 1
    assert np.array_equal(deg, col.vertex_degree)


def dsatur_python(nv, edges):
    """Algorithm 2.3 in plain Python (tie-break: degree, then id)."""
    adj = [set() for _ in range(nv)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    color = [-1] * nv
    for _ in range(nv):
        best = None
        for v in range(nv):
            if color[v] >= 0:
                continue
            sat = len({color[w] for w in adj[v] if color[w] >= 0})
            key = (sat, len(adj[v]), -v)
            if best is None or key > best[0]:
                best = (key, v)
        v = best[1]
        used = {color[w] for w in adj[v]}
        c = 0
        while c in used:
            c += 1
        color[v] = c
    return color


def test_native_dsatur_matches_python():
    x = W.torus(1500, 7)
    t = ot.build_tree(x, 16)
    for l in range(2, t.L + 1):
        pairs = ot.admissible_pairs(t, l)
        if not pairs:
            continue
        zs = lambda a: sorted(t.near[l][a] + t.inter[l][a])
        col = og.color_pairs(pairs, zs, len(t.cuts[l]))
        if col.n_vertices > 400:
            continue
        pv, vb, vS = og.constraint_vertices(pairs, zs)
        ref = dsatur_python(len(vb), og.brute_force_edges(vb.tolist(), vS))
        assert col.vertex_color.tolist() == ref


def coverage(t):
    n2 = 0
    for l in range(2, t.L + 1):
        for a, b in ot.admissible_pairs(t, l):
            (a0, a1), (b0, b1) = t.rng(l, a), t.rng(l, b)
            n2 += (a1 - a0) * (b1 - b0)
    for a, b in ot.near_pairs(t, t.L):
        (a0, a1), (b0, b1) = t.rng(t.L, a), t.rng(t.L, b)
        n2 += (a1 - a0) * (b1 - b0)
    return n2


@pytest.mark.parametrize("name", ["line", "grid", "torus", "sphere", "cube3d"])
def test_coverage_and_symmetry(name):
    """Every entry of A is in exactly one admissible or leaf-neighbour block, and
    beta in int(alpha) <=> alpha in int(beta) (Section 3)."""
    rng = np.random.default_rng(3)
    x = {"line": W.line1d(700, 1), "grid": W.grid2d(24), "torus": W.torus(2500, 4),
         "sphere": W.sphere(2000, 5), "cube3d": rng.random((1800, 3))}[name]
    t = ot.build_tree(x, 20)
    assert coverage(t) == t.n * t.n
    cover = np.zeros((t.n, t.n), dtype=np.int8)
    for l in range(2, t.L + 1):
        for a, b in ot.admissible_pairs(t, l):
            (a0, a1), (b0, b1) = t.rng(l, a), t.rng(l, b)
            cover[a0:a1, b0:b1] += 1
    for a, b in ot.near_pairs(t, t.L):
        (a0, a1), (b0, b1) = t.rng(t.L, a), t.rng(t.L, b)
        cover[a0:a1, b0:b1] += 1
    assert cover.min() == 1 and cover.max() == 1
    for l in range(t.L + 1):
        for a in range(len(t.cuts[l])):
            for b in t.inter[l][a]:
                assert a in t.inter[l][b]
            for b in t.near[l][a]:
                assert a in t.near[l][b]
            assert a in t.near[l][a]
    assert sorted(t.perm.tolist()) == list(range(t.n))


@pytest.mark.parametrize("d,n_side", [(1, 256), (2, 32)])
def test_uniform_bounds(d, n_side):
    """Uniform grids: |near| <= 3^d, |int| <= 6^d - 3^d, chi <= 6^d, chi_leaf <= 3^d
    (Section 4.1.4, general test-matrix patterns)."""
    if d == 1:
        x = ((np.arange(n_side) + 0.5) / n_side)[:, None]
        t = ot.build_tree(x, 4)
    else:
        t = ot.build_tree(W.grid2d(n_side), 4)
    for l in range(t.L + 1):
        assert max(len(v) for v in t.near[l]) <= 3 ** d
        assert max(len(v) for v in t.inter[l]) <= 6 ** d - 3 ** d
    for l in range(2, t.L + 1):
        assert og.color_level(t, l).n_colors <= 6 ** d
    assert og.color_leaf(t).n_colors <= 3 ** d


def test_quantize_boundaries():
    """Reading: a point on a split plane goes to the upper child; 1.0 clamps."""
    x = np.array([[0.0], [0.5], [0.25], [1.0], [0.5 - 2.0 ** -30]])
    q = ot.quantize(x, np.zeros(1), 1.0)[:, 0]
    assert q.tolist() == [0, 1 << 20, 1 << 19, (1 << 21) - 1, (1 << 20) - 1]
    assert ot.morton(np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 0, 0]])).tolist() == [1, 2, 4, 9]


def test_root_cube():
    lo, side = ot.root_cube(np.array([[0.2, 0.9], [0.3, 0.1]]))
    assert side == 1.0 and lo.tolist() == [0.0, 0.0]
    lo, side = ot.root_cube(np.array([[-1.0, 0.0, 2.0], [1.0, 0.5, 2.5]]))
    assert lo.tolist() == [-1.0, 0.0, 2.0] and side == 2.0


def test_adaptive_split_rule():
    x = W.torus(3000, 9)
    t = ot.build_tree(x, 32)
    for l, lev in enumerate(t.levels):
        for b in lev:
            assert (b.end - b.start > 32) == (not b.leaf) or l == t.L
            assert b.end > b.start
    leaves = [t.box(t.L, i) for i in range(len(t.cuts[t.L]))]
    assert sum(b.end - b.start for b in leaves) == t.n
    assert all(b.leaf for b in leaves)
