"""Oracle: sampling constraints, incompatibility graph, DSatur (Sections 2.6, 4.1.2, 4.1.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For an admissible pair (alpha, beta) of cut l, eq. (h1constraints) asks for a
test matrix with Omega(I_beta) = G_beta and zeros on every other box of
near(alpha) u int(alpha).  The constraint set is therefore determined by the key
(beta, S_alpha) with S_alpha = near(alpha) u int(alpha); pairs with the same key
share one vertex (e.g. A_{8,11} and A_{9,11} in the worked example).  For the
leaf extraction (Section 4.1.3) the zero set is near(alpha) only.

Vertex ids follow the order of first occurrence, scanning alpha in cut order and
then beta in cut order.  Edges and DSatur live in graph.c (plain C).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graph.c")
_LIB = os.path.join(_HERE, "_graph_oracle.so")
_lib = None


def build_native(force: bool = False) -> str:
    """Compile graph.c into a shared library next to it (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _native():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_native())
        _lib.oracle_color.restype = ctypes.c_int
        _lib.oracle_color.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 3 + \
            [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return _lib


@dataclass
class Coloring:
    n_vertices: int
    n_colors: int
    n_edges: int
    pair_vertex: np.ndarray   # vertex id of every pair (pair order)
    vertex_beta: np.ndarray   # beta (cut index) of every vertex
    vertex_color: np.ndarray  # colour of every vertex
    vertex_degree: np.ndarray
    s_ptr: np.ndarray         # zero-set S of every vertex, CSR over cut indices
    s_idx: np.ndarray

    @property
    def pair_color(self) -> np.ndarray:
        return self.vertex_color[self.pair_vertex]

    def active(self, c: int) -> list:
        """Boxes beta that carry random (or identity) rows in colour c."""
        return sorted(set(self.vertex_beta[self.vertex_color == c].tolist()))


def constraint_vertices(pairs, zero_set):
    """Distinct constraint sets (Definition 4.1) in order of first occurrence.

    pairs: list of (alpha, beta); zero_set(alpha) -> sorted list of boxes.
    Returns (pair_vertex, vertex_beta, S list).
    """
    key_to_v = {}
    pair_vertex = np.empty(len(pairs), dtype=np.int64)
    vbeta, vS = [], []
    cache = {}
    for p, (a, b) in enumerate(pairs):
        if a not in cache:
            cache[a] = tuple(zero_set(a))
        key = (b, cache[a])
        v = key_to_v.get(key)
        if v is None:
            v = len(vbeta)
            key_to_v[key] = v
            vbeta.append(b)
            vS.append(cache[a])
        pair_vertex[p] = v
    return pair_vertex, np.array(vbeta, dtype=np.int64), vS


def color_pairs(pairs, zero_set, n_boxes: int) -> Coloring:
    """Build the incompatibility graph of the pairs' constraint sets and colour
    it with DSatur (Algorithm 2.3; tie-break: degree, then vertex id)."""
    pair_vertex, vbeta, vS = constraint_vertices(pairs, zero_set)
    nv = len(vbeta)
    s_ptr = np.zeros(nv + 1, dtype=np.int64)
    for v, S in enumerate(vS):
        s_ptr[v + 1] = s_ptr[v] + len(S)
    s_idx = np.array([g for S in vS for g in S], dtype=np.int32)
    beta32 = vbeta.astype(np.int32)
    color = np.empty(nv, dtype=np.int32)
    degree = np.empty(nv, dtype=np.int32)
    n_edges = ctypes.c_int64(0)
    lib = _native()
    nc = lib.oracle_color(nv, int(n_boxes), beta32.ctypes.data, s_ptr.ctypes.data,
                          s_idx.ctypes.data if nv else None, color.ctypes.data,
                          ctypes.addressof(n_edges), degree.ctypes.data)
    if nc < 0:
        raise MemoryError("oracle_color failed")
    return Coloring(nv, nc, int(n_edges.value), pair_vertex, vbeta,
                    color.astype(np.int64), degree.astype(np.int64), s_ptr, s_idx)


def color_level(tree, l: int) -> Coloring:
    """Colouring of the admissible pairs of cut l (Section 4.1.2)."""
    from .tree import admissible_pairs
    pairs = admissible_pairs(tree, l)
    zs = lambda a: sorted(tree.near[l][a] + tree.inter[l][a])
    return color_pairs(pairs, zs, len(tree.cuts[l]))


def color_leaf(tree) -> Coloring:
    """Colouring of the neighbour pairs of the leaf cut (Section 4.1.3)."""
    from .tree import near_pairs
    L = tree.L
    return color_pairs(near_pairs(tree, L), lambda a: tree.near[L][a], len(tree.cuts[L]))


def brute_force_edges(vbeta, vS):
    """Edges straight from the definition, O(V^2): for tiny graphs in tests."""
    edges = set()
    for u in range(len(vbeta)):
        for v in range(u + 1, len(vbeta)):
            if vbeta[u] != vbeta[v] and (vbeta[u] in vS[v] or vbeta[v] in vS[u]):
                edges.add((u, v))
    return edges


@dataclass
class BoxColoring:
    """Colouring of the box constraint sets of uniform H^1 sampling (Section 4.2)."""
    boxes: np.ndarray         # cut index of every vertex (boxes with a non-empty interaction list)
    n_colors: int
    n_edges: int
    color: np.ndarray         # colour of every vertex
    degree: np.ndarray
    inter: list               # int(alpha) of every vertex (sorted cut indices)

    def active(self, c: int) -> list:
        """Boxes that carry random rows in colour c: the union of int(alpha)
        over the boxes alpha of that colour (eq. unifh1constraints)."""
        out = set()
        for v in np.flatnonzero(self.color == c):
            out.update(self.inter[v])
        return sorted(out)


def color_boxes(tree, l: int) -> BoxColoring:
    """Uniform H^1, first sampling stage of cut l (Section 4.2): one vertex per
    box alpha with a non-empty interaction list, in cut order; it asks for
    G_beta on every beta in int(alpha) and zeros on near(alpha).  Two vertices
    conflict when one asks for random rows on a box the other asks to be zero;
    DSatur as for the pair graphs."""
    boxes = [a for a in range(len(tree.cuts[l])) if tree.inter[l][a]]
    nv = len(boxes)
    inter = [sorted(tree.inter[l][a]) for a in boxes]
    near = [sorted(tree.near[l][a]) for a in boxes]
    g_ptr = np.zeros(nv + 1, dtype=np.int64)
    z_ptr = np.zeros(nv + 1, dtype=np.int64)
    for v in range(nv):
        g_ptr[v + 1] = g_ptr[v] + len(inter[v])
        z_ptr[v + 1] = z_ptr[v] + len(near[v])
    g_idx = np.array([b for s in inter for b in s], dtype=np.int32)
    z_idx = np.array([b for s in near for b in s], dtype=np.int32)
    color = np.empty(nv, dtype=np.int32)
    degree = np.empty(nv, dtype=np.int32)
    n_edges = ctypes.c_int64(0)
    lib = _native()
    lib.oracle_color_sets.restype = ctypes.c_int
    lib.oracle_color_sets.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 7
    nc = lib.oracle_color_sets(nv, len(tree.cuts[l]), g_ptr.ctypes.data, g_idx.ctypes.data if nv else None,
                               z_ptr.ctypes.data, z_idx.ctypes.data if nv else None, color.ctypes.data,
                               ctypes.addressof(n_edges), degree.ctypes.data)
    if nc < 0:
        raise MemoryError("oracle_color_sets failed")
    return BoxColoring(np.array(boxes, dtype=np.int64), nc, int(n_edges.value), color.astype(np.int64),
                       degree.astype(np.int64), inter)


def brute_force_set_edges(gsets, zsets):
    """Edges of set constraints straight from the definition, O(V^2)."""
    edges = set()
    for u in range(len(gsets)):
        for v in range(u + 1, len(gsets)):
            if set(gsets[u]) & set(zsets[v]) or set(gsets[v]) & set(zsets[u]):
                edges.add((u, v))
    return edges
