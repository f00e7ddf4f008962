"""Pins of the oracle's uniform H^1 compression (Section 4.2) against what the paper fixes.

CPU only.  The worked 1D example's level-3 box graph (Figure
graph_strong_1d_lvl3_unif: 8 box vertices, 22 edges, 5 colours with the
printed fill colours and the 5 printed test matrices), the edge definition
brute-forced, DSatur against a plain-Python DSatur, the 5^d colour bound on
uniform grids, and exact recovery of random exact uniform H^1 matrices.
"""
import json
import os

import numpy as np
import pytest

import hm_workloads as W
from oracle import graph as og
from oracle import h1
from oracle import tree as ot

from test_oracle_structure import dsatur_python, worked_tree

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def heap(tree, l, b):
    box = tree.box(l, b)
    return (1 << box.level) + box.index


def test_worked_example_uniform_level3():
    ref = json.load(open(os.path.join(GOLD, "worked_example_1d.json")))["uniform_level3"]
    t = worked_tree()
    bc = og.color_boxes(t, 3)
    assert (len(bc.boxes), bc.n_edges, bc.n_colors) == (ref["vertices"], ref["edges"], ref["colors"])
    classes = sorted(sorted(heap(t, 3, int(b)) for b in bc.boxes[bc.color == c]) for c in range(bc.n_colors))
    assert classes == sorted(ref["classes"])
    rows = sorted(sorted(heap(t, 3, b) for b in bc.active(c)) for c in range(bc.n_colors))
    assert rows == sorted(ref["test_matrix_rows"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_box_edges_match_definition(seed):
    """The C builder of set constraints equals the O(V^2) definition."""
    x = np.random.default_rng(seed).random((1200, 3))
    t = ot.build_tree(x, 12)
    for l in range(2, t.L + 1):
        bc = og.color_boxes(t, l)
        if len(bc.boxes) < 2:
            continue
        gs = [t.inter[l][int(a)] for a in bc.boxes]
        zs = [t.near[l][int(a)] for a in bc.boxes]
        edges = og.brute_force_set_edges(gs, zs)
        assert bc.n_edges == len(edges), l
        deg = np.zeros(len(gs), dtype=int)
        for u, v in edges:
            assert bc.color[u] != bc.color[v]
            deg[u] += 1
            deg[v] += 1
        assert np.array_equal(deg, bc.degree)
        if len(gs) <= 300:
            assert bc.color.tolist() == dsatur_python(len(gs), edges), l


@pytest.mark.parametrize("d,n_side", [(1, 256), (2, 32)])
def test_uniform_colour_bound(d, n_side):
    """Uniform grids: the paper's pattern -- a box coloured by its grid
    coordinates modulo 5 (the 5^d shifts of the activation pattern of Section
    4.2.1) -- is a proper colouring of the box graph, so chi_unif <= 5^d.
    DSatur's own count stays within a few colours of it."""
    if d == 1:
        t = ot.build_tree(((np.arange(n_side) + 0.5) / n_side)[:, None], 4)
    else:
        t = ot.build_tree(W.grid2d(n_side), 4)
    for l in range(2, t.L + 1):
        bc = og.color_boxes(t, l)
        pattern = {}
        for a in bc.boxes:
            anchor = t.box(l, int(a)).anchor
            pattern[int(a)] = tuple(q % 5 for q in anchor)  # box coordinates at level l
        gs = [t.inter[l][int(a)] for a in bc.boxes]
        zs = [t.near[l][int(a)] for a in bc.boxes]
        for u, v in og.brute_force_set_edges(gs, zs):
            assert pattern[int(bc.boxes[u])] != pattern[int(bc.boxes[v])], (l, u, v)
        assert bc.n_colors <= 5 ** d + 2


def random_uniform_hmatrix(t, k, seed):
    """A = sum over admissible pairs of U_alpha S_ab V_beta^T (one orthonormal
    U and V per box and level, rank <= k) plus random dense near blocks: an
    exact uniform H^1 matrix on the tree."""
    rng = np.random.default_rng(seed)
    A = np.zeros((t.n, t.n))
    for l in range(2, t.L + 1):
        U, V = {}, {}
        for a in range(len(t.cuts[l])):
            a0, a1 = t.rng(l, a)
            kk = min(k, a1 - a0)
            U[a] = np.linalg.qr(rng.standard_normal((a1 - a0, kk)))[0]
            V[a] = np.linalg.qr(rng.standard_normal((a1 - a0, kk)))[0]
        for a, b in ot.admissible_pairs(t, l):
            a0, a1 = t.rng(l, a)
            b0, b1 = t.rng(l, b)
            A[a0:a1, b0:b1] = U[a] @ rng.standard_normal((U[a].shape[1], V[b].shape[1])) @ V[b].T
    for a, b in ot.near_pairs(t, t.L):
        a0, a1 = t.rng(t.L, a)
        b0, b1 = t.rng(t.L, b)
        A[a0:a1, b0:b1] = rng.standard_normal((a1 - a0, b1 - b0))
    return A


@pytest.mark.parametrize("geom,kw", [("torus", {"tol": 1e-10}), ("cube", {"rank": 6}), ("line", {"tol": 1e-10})])
def test_exact_uniform_hmatrix_recovered(geom, kw):
    """Sampling is exact when the block rows have rank <= r - p (Section 2.5):
    the compressed operator equals A to rounding, on adaptive trees with boxes
    smaller than r."""
    if geom == "torus":
        x = W.torus(1500, 12)
    elif geom == "cube":
        x = np.random.default_rng(3).random((1300, 3))
    else:
        x = W.line1d(900, 4)
    t = ot.build_tree(x, 24)
    A = random_uniform_hmatrix(t, 6, 21)
    H = h1.compress_uniform(t, h1.DenseOp(A), 16, seed=5, **kw)
    At = h1.apply_h1(H, np.eye(t.n))
    assert np.linalg.norm(At - A) <= 1e-12 * np.linalg.norm(A)
    assert getattr(H, "uniform", False)
    # one basis per box: every pair of a box shares its U (and of a column box its V)
    for l, lf in H.levels.items():
        U, V = H.bases[l]
        for (a, b), Ua, Vb in zip(lf.pairs, lf.U, lf.V):
            assert Ua is U[a] and Vb is V[b]


def test_uniform_compression_of_a_kernel_matrix():
    """1/(4 pi r) on a torus: with r large enough for the block rows' rank the
    uniform compression reaches the tolerance's order (dense 2-norm), and it
    stores fewer floats than the per-pair bases of Section 4.1 at the same r."""
    w = W.torus_laplace(n=2000, tol=1e-6, r=48)
    t = ot.build_tree(w.points, 32)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    A = op.dense()
    Hu = h1.compress_uniform(t, op, 48, tol=1e-6, seed=w.seed)
    Hn = h1.compress(t, op, 48, tol=1e-6, seed=w.seed)
    eu = np.linalg.norm(h1.apply_h1(Hu, np.eye(w.n)) - A, 2) / np.linalg.norm(A, 2)
    assert eu <= 1e-5, eu
    assert Hu.floats() < Hn.floats()
