"""Acceptance at full size: the 200,000-point torus job of the benchmark
(1/(4 pi |x - y|) on a torus, adaptive octree with leaves of at most 64 points,
tolerance 1e-6, r = 32; the stand-in for the paper's 3D-surface experiment,
Section 5.3), through the C ABI, against the CPU oracle.

* Structure (Section 3; Definition 4.1 and Algorithm 2.3): permutation, boxes
  of every level, cuts, neighbour and interaction lists, and the constraint
  vertices, degrees and colours of every admissible level and of the leaf
  level -- bit-exact.
* Black box (Algorithm 4.1, sampling step): the raw samples Y_l = A Omega_l and
  Z_l = A^* Psi_l of every level on seeded (row, colour) entries of the sample
  tiles, against the oracle's sampled-row product: <= 1e-12 relative in FP64,
  <= 1e-6 with the split-BF16 tensor-core black box.
* Level 2 (nothing to peel there, so Algorithm 2.1 applies to the raw samples
  of each block): the blocks U B V^T of seeded pairs against the oracle's
  per-block solve: equal ranks and <= 1e-10 relative in FP64, <= 1e-6 with the
  mixed-precision black box.
* Whole operator (Section 5): the FP64 and the mixed-precision compressions
  both meet the tolerance in the relative error E, their E agree to 1e-6, and
  the two compressed operators differ by <= 1e-6 relative in the spectral
  norm (E's norm; estimated by power iterations on the difference -- random
  vectors mostly excite the small singular values of a smoothing kernel, so
  they overstate a norm-relative difference).
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle import graph as og
from oracle import h1 as oh1
from oracle import tree as ot

from gpu_helpers import check_structure, factors, hm, i32, run_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP64, MIXED = 0, 1
TOL = {FP64: 1e-12, MIXED: 1e-6}       # raw samples
TOL_BLOCK = {FP64: 1e-10, MIXED: 1e-6}  # level-2 blocks


def job():
    return W.torus_laplace(n=200_000, tol=1e-6, r=32)


@pytest.fixture(scope="module")
def oracle_structure():
    w = job()
    t = ot.build_tree(w.points, w.leaf_size)
    cols = {l: og.color_level(t, l) for l in range(2, t.L + 1)}
    return w, t, cols, og.color_leaf(t)


def test_200k_structure_bitexact(oracle_structure):
    w, t, cols, leaf = oracle_structure
    m = hm()
    comp, _ = run_gpu(w, precision=MIXED, keep=False, compress=False)
    check_structure(comp, t)
    for l in list(range(2, t.L + 1)) + [m.HM_LEVEL_LEAF]:
        ref = leaf if l == m.HM_LEVEL_LEAF else cols[l]
        chi = comp.color(l)
        assert chi == ref.n_colors, l
        assert np.array_equal(i32(comp.export(m.HM_X_PAIR_VERTEX, l)), ref.pair_vertex), l
        assert np.array_equal(i32(comp.export(m.HM_X_VERTEX_BETA, l)), ref.vertex_beta), l
        assert np.array_equal(i32(comp.export(m.HM_X_VERTEX_DEGREE, l)), ref.vertex_degree), l
        assert np.array_equal(i32(comp.export(m.HM_X_VERTEX_COLOR, l)), ref.vertex_color), l
    comp.close()


def sampled_tile_entries(t, l, col, n_pairs, seed):
    """Seeded (row, colour) entries of the level-l sample tiles: one random row
    of I_alpha for each of n_pairs random pairs (alpha, beta), in the pair's colour."""
    pairs = ot.admissible_pairs(t, l)
    rng = np.random.default_rng(seed + l)
    pick = rng.choice(len(pairs), min(n_pairs, len(pairs)), replace=False)
    pc = col.pair_color
    rows, colors = [], []
    for p in pick:
        a0, a1 = t.rng(l, pairs[p][0])
        rows.append(int(rng.integers(a0, a1)))
        colors.append(int(pc[p]))
    return np.array(rows), np.array(colors)


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_200k_raw_samples_on_sampled_tile_rows(oracle_structure, precision):
    import torch
    w, t, cols, _ = oracle_structure
    m = hm()
    comp, _ = run_gpu(w, precision=precision, keep=False, compress=False)
    op = oh1.KernelOp(w.points[t.perm], w.kernel)
    buf = None
    for l in range(2, t.L + 1):
        chi = comp.color(l)
        if chi == 0:
            continue
        comp.sample(comp._op, l)
        GO, GP = oh1.gaussians(t, l, 0, w.r, w.seed), oh1.gaussians(t, l, 1, w.r, w.seed)
        rows, colors = sampled_tile_entries(t, l, cols[l], 48, w.seed)
        for what, G in ((m.HM_X_SAMPLE_Y, GO), (m.HM_X_SAMPLE_Z, GP)):
            need = chi * w.n * w.r
            if buf is None or buf.numel() < need:
                buf = torch.empty(need, dtype=torch.float64).pin_memory()
            comp.export_into(what, l, buf)
            S = buf[:need].numpy().reshape(chi, w.n, w.r)
            got = S[colors, rows, :]
            ref = oh1.sample_rows(op, t, l, cols[l], G, w.r, rows, colors)
            e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert e <= TOL[precision], (l, what, e)
            rowscale = np.linalg.norm(ref, axis=1, keepdims=True) + 1e-300
            assert np.max(np.abs(got - ref) / rowscale) <= 100 * TOL[precision], (l, what)
    comp.close()


@pytest.fixture(scope="module")
def compressions(oracle_structure):
    w, _, _, _ = oracle_structure
    out = {}
    for precision in (FP64, MIXED):
        comp, info = run_gpu(w, precision=precision, keep=False)
        out[precision] = (comp, info)
    yield out
    for comp, _ in out.values():
        comp.close()


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_200k_level2_blocks_match_oracle(oracle_structure, compressions, precision):
    w, t, cols, _ = oracle_structure
    comp, _ = compressions[precision]
    l, r = 2, w.r
    col = cols[l]
    pairs = ot.admissible_pairs(t, l)
    rng_a = [t.rng(l, a) for a, _ in pairs]
    rng_b = [t.rng(l, b) for _, b in pairs]
    ranks, fac = factors(comp, l, rng_a, rng_b)
    op = oh1.KernelOp(w.points[t.perm], w.kernel)
    GO, GP = oh1.gaussians(t, l, 0, r, w.seed), oh1.gaussians(t, l, 1, r, w.seed)
    pc = col.pair_color
    index = {pq: i for i, pq in enumerate(pairs)}
    rng = np.random.default_rng(w.seed)
    for p in rng.choice(len(pairs), 2, replace=False):
        a, b = pairs[p]
        (a0, a1), (b0, b1) = rng_a[p], rng_b[p]
        c, ct = pc[p], pc[index[(b, a)]]
        P = oh1.sample_rows(op, t, l, col, GO, r, np.arange(a0, a1), np.full(a1 - a0, c))
        Zt = oh1.sample_rows(op, t, l, col, GP, r, np.arange(b0, b1), np.full(b1 - b0, ct))
        cap = min(r - w.oversample, a1 - a0, b1 - b0)
        U = oh1.qr_trunc(P, 0, w.tol, cap)
        V = oh1.qr_trunc(Zt, 0, w.tol, cap)
        B = oh1.core(GP[a0:a1], P, GO[b0:b1], U, V)
        Ug, Bg, Vg = fac[p]
        if precision == FP64:
            assert tuple(ranks[p]) == (U.shape[1], V.shape[1]), p
        X = rng.standard_normal((b1 - b0, 4))
        ref = U @ (B @ (V.T @ X))
        got = Ug @ (Bg @ (Vg.T @ X))
        e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert e <= TOL_BLOCK[precision], (p, e, tuple(ranks[p]), (U.shape[1], V.shape[1]))


def test_200k_fp64_and_mixed_operators_agree(oracle_structure, compressions):
    import torch
    w, _, _, _ = oracle_structure
    c64, _ = compressions[FP64]
    cmx, info = compressions[MIXED]
    assert info.bb_tc_levels > 0, "the mixed compression did not use the tensor-core black box"
    e64 = c64.relerr(c64._op, 10)
    emx = cmx.relerr(cmx._op, 10)
    assert e64 <= w.tol and emx <= w.tol, (e64, emx)
    assert abs(emx - e64) <= 1e-6, (e64, emx)
    def spectral_norm(apply, iters=10):
        v = torch.from_numpy(np.random.default_rng(5).standard_normal(w.n)).cuda()
        v /= torch.linalg.norm(v)
        lam = 0.0
        for _ in range(iters):
            u = apply(apply(v, 0), 1)
            lam = float(torch.linalg.norm(u))
            v = u / lam
        return lam ** 0.5

    norm64 = spectral_norm(c64.apply)
    diff = spectral_norm(lambda v, trans: cmx.apply(v, trans) - c64.apply(v, trans))
    assert diff <= 1e-6 * norm64, (diff, norm64, diff / norm64)
