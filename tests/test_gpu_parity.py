"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tree, cuts, lists and colourings: bit-exact.  Gaussian test matrices: <= 4 ulp
(each side calls its own libm log/cos).  FP64 mode: peeled samples, compressed
blocks U B V^T, leaf blocks and the applied operator within 1e-10 relative
(the tolerance the design fixes for FP64).
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle import h1 as oh1
from oracle import tree as ot

from gpu_helpers import check_structure, f64, factors, hm, i32, oracle_op, run_gpu, samples

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def small_workloads():
    return {
        "line1d_dense": W.line1d_dense(),
        "grid2d_log_64": W.grid2d_log(n_side=64, rank=12),
        "torus_4k": W.torus_laplace(n=4000, tol=1e-8, r=16),
        "torus_ragged": W.Workload("torus_ragged", W.torus(2777, 17), W.K_LAPLACE3D, leaf_size=23, r=12,
                                   tol=1e-7, seed=99),
        "sphere_invr": W.Workload("sphere_invr_3k", W.sphere(3001, 5), W.K_INVR, leaf_size=40, r=16, rank=8,
                                  seed=7),
        "cube_exp": W.Workload("cube_exp", np.random.default_rng(4).random((2500, 3)), W.K_EXP, leaf_size=48,
                               r=16, tol=1e-9, seed=3),
    }


@pytest.mark.parametrize("name", list(small_workloads()))
def test_tree_and_lists_bitexact(name):
    w = small_workloads()[name]
    comp, _ = run_gpu(w, compress=False)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    check_structure(comp, t)
    comp.close()


@pytest.mark.parametrize("name", list(small_workloads()))
def test_colorings_bitexact(name):
    from oracle import graph as og
    m = hm()
    w = small_workloads()[name]
    comp, _ = run_gpu(w, compress=False)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    for l in list(range(2, t.L + 1)) + [m.HM_LEVEL_LEAF]:
        chi = comp.color(l)
        ref = og.color_leaf(t) if l == m.HM_LEVEL_LEAF else og.color_level(t, l)
        if len(ref.pair_vertex) == 0:
            assert chi == 0
            continue
        assert chi == ref.n_colors, f"level {l}"
        assert np.array_equal(i32(comp.export(m.HM_X_PAIR_VERTEX, l)), ref.pair_vertex)
        assert np.array_equal(i32(comp.export(m.HM_X_VERTEX_BETA, l)), ref.vertex_beta)
        assert np.array_equal(i32(comp.export(m.HM_X_VERTEX_DEGREE, l)), ref.vertex_degree)
        assert np.array_equal(i32(comp.export(m.HM_X_VERTEX_COLOR, l)), ref.vertex_color)
    comp.close()


def test_gaussians_within_4ulp():
    m = hm()
    w = small_workloads()["torus_ragged"]
    comp, _ = run_gpu(w, compress=False)
    t = ot.build_tree(w.points, w.leaf_size)
    for l in range(2, t.L + 1):
        comp.color(l)
        comp.sample(comp._op, l)
        g = f64(comp.export(m.HM_X_GAUSS, l)).reshape(2, w.n, w.r)
        for side in (0, 1):
            ref = oh1.gaussians(t, l, side, w.r, w.seed)
            ulp = np.abs(g[side] - ref) / np.spacing(np.maximum(np.abs(ref), 1e-300))
            assert ulp.max() <= 4, (l, side, ulp.max())
    comp.close()


@pytest.mark.parametrize("name", ["line1d_dense", "torus_ragged", "cube_exp"])
def test_raw_samples_match_black_box(name):
    """hm_sample: Y = A Omega_l, Z = A^* Psi_l before peeling."""
    from oracle import graph as og
    m = hm()
    w = small_workloads()[name]
    comp, _ = run_gpu(w, compress=False)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    op = oracle_op(w, t)
    for l in range(2, t.L + 1):
        chi = comp.color(l)
        if chi == 0:
            continue
        comp.sample(comp._op, l)
        col = og.color_level(t, l)
        GO, GP = oh1.gaussians(t, l, 0, w.r, w.seed), oh1.gaussians(t, l, 1, w.r, w.seed)
        Yr = op.apply(oh1.test_matrix(t, l, col, GO, w.r))
        Zr = op.apply_t(oh1.test_matrix(t, l, col, GP, w.r))
        Y = samples(comp, m.HM_X_SAMPLE_Y, l, w.n, chi, w.r)
        Z = samples(comp, m.HM_X_SAMPLE_Z, l, w.n, chi, w.r)
        assert np.linalg.norm(Y - Yr) <= 1e-12 * np.linalg.norm(Yr)
        assert np.linalg.norm(Z - Zr) <= 1e-12 * np.linalg.norm(Zr)
    comp.close()


def compare_compression(w, comp, tol=TOL64):
    """Peeled samples, blocks U B V^T, leaf blocks and apply against the oracle."""
    m = hm()
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    H = oh1.compress(t, oracle_op(w, t), w.r, rank=w.rank, tol=w.tol, seed=w.seed, keep_samples=True,
                      oversample=w.oversample)
    r = w.r
    worst = {}
    for l, lf in H.levels.items():
        if not lf.pairs:
            continue
        chi = lf.coloring.n_colors
        pc = lf.coloring.pair_color
        Y = samples(comp, m.HM_X_SAMPLE_Y, l, w.n, chi, r)
        Z = samples(comp, m.HM_X_SAMPLE_Z, l, w.n, chi, r)
        for i, ((a0, a1), c) in enumerate(zip(lf.rng_a, pc)):
            for got, ref in ((Y, lf.Y), (Z, lf.Z)):
                g, rf = got[a0:a1, c * r:(c + 1) * r], ref[a0:a1, c * r:(c + 1) * r]
                e = np.linalg.norm(g - rf) / max(np.linalg.norm(rf), 1e-300)
                worst["sample"] = max(worst.get("sample", 0.0), e)
        ranks, fac = factors(comp, l, lf.rng_a, lf.rng_b)
        ref_ranks = np.array([[u.shape[1], v.shape[1]] for u, v in zip(lf.U, lf.V)])
        assert np.array_equal(ranks, ref_ranks), f"ranks differ at level {l}"
        for (U, B, V), Ur, Br, Vr in zip(fac, lf.U, lf.B, lf.V):
            blk, ref = U @ B @ V.T, Ur @ Br @ Vr.T
            e = np.linalg.norm(blk - ref) / max(np.linalg.norm(ref), 1e-300)
            worst["block"] = max(worst.get("block", 0.0), e)
    D = f64(comp.export(m.HM_X_LEAF_D))
    off = 0
    num = den = 0.0
    for (a0, a1), (b0, b1), Dr in zip(H.leaf.rng_a, H.leaf.rng_b, H.leaf.D):
        sz = (a1 - a0) * (b1 - b0)
        num += np.sum((D[off:off + sz].reshape(a1 - a0, b1 - b0) - Dr) ** 2)
        den += np.sum(Dr ** 2)
        off += sz
    worst["leaf"] = np.sqrt(num / den)
    import torch
    x = np.random.default_rng(1).standard_normal((w.n, 2))
    for trans in (0, 1):
        y = comp.apply(torch.from_numpy(x).cuda(), trans=trans).cpu().numpy()
        yr = np.empty_like(x)
        yr[t.perm] = oh1.apply_h1(H, x[t.perm], transpose=bool(trans))
        worst[f"apply{trans}"] = np.linalg.norm(y - yr) / np.linalg.norm(yr)
    for k, v in worst.items():
        assert v <= tol, (k, v, worst)
    return H, worst


@pytest.mark.parametrize("name", list(small_workloads()))
def test_compress_fp64_matches_oracle(name):
    w = small_workloads()[name]
    comp, info = run_gpu(w)
    compare_compression(w, comp)
    comp.close()


def test_relative_error_matches_oracle():
    w = small_workloads()["torus_4k"]
    comp, _ = run_gpu(w, keep=False)
    e_gpu = comp.relerr(comp._op, 20)
    t = ot.build_tree(w.points, w.leaf_size)
    op = oracle_op(w, t)
    H = oh1.compress(t, op, w.r, tol=w.tol, seed=w.seed, oversample=w.oversample)
    e_ref = oh1.relative_error(H, op, 20, seed=w.seed + 1)
    assert abs(e_gpu - e_ref) <= 1e-6 * e_ref + 1e-15
    comp.close()


def test_exact_hmatrix_recovered_on_gpu():
    """A dense operator that is an exact rank-6 H^1 matrix on the tree is
    recovered to ~1e-12 (Section 2.5: sampling is exact when rank <= r)."""
    import torch
    from test_oracle_numerics import random_hmatrix
    x = W.torus(2000, 12)
    t = ot.build_tree(x, 24)
    A = random_hmatrix(t, 6, 21)
    Aorig = np.empty_like(A)
    Aorig[np.ix_(t.perm, t.perm)] = A
    w = W.Workload("hmat", x, W.K_LAPLACE3D, leaf_size=24, r=16, tol=1e-9, dense=Aorig, seed=5)
    comp, _ = run_gpu(w, keep=False)
    X = np.random.default_rng(3).standard_normal((w.n, 3))
    Y = comp.apply(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.linalg.norm(Y - Aorig @ X) <= 1e-12 * np.linalg.norm(Aorig @ X)
    comp.close()


def test_callback_operator_equals_builtin():
    """A user black box (torch matmul on raw device pointers) gives the same
    compression as the built-in dense operator."""
    import torch
    m = hm()
    w = W.line1d_dense(n=1024)
    A = torch.from_numpy(w.dense).cuda()
    calls = []

    def black_box(trans, xp, yp, s, stream):
        n = w.n
        X = torch.as_tensor(_DevArray(xp, (s, n))).t()
        Y = torch.as_tensor(_DevArray(yp, (s, n)))
        M = A.t() if trans else A
        Y.copy_((M @ X).t())
        calls.append(s)
        return 0

    comp = m.Compressor(m.Settings(d=1, leaf_size=64, r=w.r, rank=w.rank, uniform_depth=5, seed=w.seed))
    comp.tree_build(torch.from_numpy(w.points).cuda())
    comp.compress(m.callback_op(black_box))
    ref, _ = run_gpu(w, keep=False)
    X = torch.from_numpy(np.random.default_rng(0).standard_normal((w.n, 2))).cuda()
    y1, y2 = comp.apply(X), ref.apply(X)
    assert calls and torch.linalg.norm(y1 - y2) <= 1e-12 * torch.linalg.norm(y2)
    comp.close()
    ref.close()


class _DevArray:
    """A raw float64 device buffer seen through __cuda_array_interface__."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape, "typestr": "<f8",
                                         "version": 3, "strides": None}


def test_error_paths():
    import torch
    m = hm()
    comp = m.Compressor(m.Settings(d=3, leaf_size=16, r=8, rank=4))
    with pytest.raises(m.HMError) as ei:
        comp.color(2)
    assert ei.value.status == m.HM_ESTATE
    x = torch.from_numpy(W.torus(500, 1)).cuda()
    comp.tree_build(x)
    with pytest.raises(m.HMError) as ei:
        comp.apply(torch.zeros(500, dtype=torch.float64, device="cuda"))
    assert ei.value.status == m.HM_ESTATE
    with pytest.raises(m.HMError) as ei:
        comp.color(99)
    assert ei.value.status == m.HM_EINVAL
    # a failing black box surfaces as HM_EOP and the context stays usable
    with pytest.raises(m.HMError) as ei:
        comp.compress(m.callback_op(lambda *a: 3))
    assert ei.value.status == m.HM_EOP
    comp.compress(m.kernel_op(m.HM_K_LAPLACE3D))
    y = comp.apply(torch.ones(500, dtype=torch.float64, device="cuda"))
    assert torch.isfinite(y).all()
    comp.close()


def test_single_point_and_tiny_inputs():
    import torch
    m = hm()
    for n in (1, 2, 7):
        pts = np.random.default_rng(n).random((n, 3))
        comp = m.Compressor(m.Settings(d=3, leaf_size=4, r=4, rank=2))
        comp.tree_build(torch.from_numpy(pts).cuda())
        comp.compress(m.kernel_op(m.HM_K_EXP))
        x = np.ones(n)
        y = comp.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        A = oh1.kernel_eval(4, pts, pts)
        assert np.allclose(y, A @ x, rtol=1e-12, atol=1e-12)
        comp.close()
