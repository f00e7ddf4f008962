"""Uniform H^1 (Section 4.2) on the GPU against the oracle's compress_uniform.

* The box graph of every level (stage 1: box alpha asks for random rows on
  int(alpha) and zeros on near(alpha)) and its DSatur colouring: bit-exact.
* FP64: every admissible block U_a B_ab V_b^T, the ranks of the bases, the
  leaf blocks and the applied operator within 1e-10 of the oracle's; an exact
  uniform H^1 matrix is recovered to 1e-12.
* Split-BF16 tensor-core black box: the applied operator within 1e-6 of the
  oracle's (FP64) compression.
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle import graph as og
from oracle import h1 as oh1
from oracle import tree as ot

from gpu_helpers import f64, factors, hm, i32, oracle_op, run_gpu

pytestmark = pytest.mark.gpu

UNIFORM = 1
TOL64 = 1e-10


def workloads():
    return {
        "torus_3k": W.Workload("torus_u", W.torus(3000, 31), W.K_LAPLACE3D, leaf_size=32, r=32, tol=1e-7, seed=9),
        "cube_exp_rank": W.Workload("cube_u", np.random.default_rng(4).random((2500, 3)), W.K_EXP, leaf_size=40,
                                    r=24, rank=12, seed=3),
        "grid_log": W.Workload("grid_u", W.grid2d(48), W.K_LOG, leaf_size=24, r=32, tol=1e-8, seed=2),
        "sphere_ragged": W.Workload("sphere_u", W.sphere(2777, 5), W.K_INVR, leaf_size=23, r=24, tol=1e-6, seed=7,
                                    oversample=8),
    }


@pytest.mark.parametrize("name", list(workloads()))
def test_box_colorings_bitexact(name):
    m = hm()
    w = workloads()[name]
    comp, _ = run_gpu(w, compress=False, fmt=UNIFORM)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    for l in range(2, t.L + 1):
        chi = comp.color_boxes(l)
        ref = og.color_boxes(t, l)
        assert chi == ref.n_colors, l
        if len(ref.boxes) == 0:
            continue
        assert np.array_equal(i32(comp.export(m.HM_X_BOX_VERTEX_BOX, l)), ref.boxes), l
        assert np.array_equal(i32(comp.export(m.HM_X_BOX_DEGREE, l)), ref.degree), l
        assert np.array_equal(i32(comp.export(m.HM_X_BOX_COLOR, l)), ref.color), l
    comp.close()


def compare_uniform(w, comp, tol):
    import torch
    m = hm()
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    H = oh1.compress_uniform(t, oracle_op(w, t), w.r, rank=w.rank, tol=w.tol, seed=w.seed, oversample=w.oversample)
    worst = {}
    for l, lf in H.levels.items():
        if not lf.pairs:
            continue
        ranks, fac = factors(comp, l, lf.rng_a, lf.rng_b)
        if tol <= TOL64:
            ref_ranks = np.array([[u.shape[1], v.shape[1]] for u, v in zip(lf.U, lf.V)])
            assert np.array_equal(ranks, ref_ranks), f"ranks differ at level {l}"
        for (U, B, V), Ur, Br, Vr in zip(fac, lf.U, lf.B, lf.V):
            blk, ref = U @ B @ V.T, Ur @ Br @ Vr.T
            e = np.linalg.norm(blk - ref) / max(np.linalg.norm(ref), 1e-300)
            worst["block"] = max(worst.get("block", 0.0), e)
    x = np.random.default_rng(1).standard_normal((w.n, 2))
    for trans in (0, 1):
        y = comp.apply(torch.from_numpy(x).cuda(), trans=trans).cpu().numpy()
        yr = np.empty_like(x)
        yr[t.perm] = oh1.apply_h1(H, x[t.perm], transpose=bool(trans))
        worst[f"apply{trans}"] = np.linalg.norm(y - yr) / np.linalg.norm(yr)
    checked = worst if tol <= TOL64 else {k: v for k, v in worst.items() if k.startswith("apply")}
    for k, v in checked.items():
        assert v <= tol, (k, v, worst)
    return H


@pytest.mark.parametrize("name", list(workloads()))
def test_uniform_fp64_matches_oracle(name):
    w = workloads()[name]
    comp, info = run_gpu(w, keep=False, fmt=UNIFORM)
    H = compare_uniform(w, comp, TOL64)
    assert info.factor_floats == H.floats(), (info.factor_floats, H.floats())
    comp.close()


@pytest.mark.parametrize("name", ["torus_3k", "sphere_ragged"])
def test_uniform_mixed_matches_oracle(name):
    w = workloads()[name]
    comp, info = run_gpu(w, precision=1, keep=False, fmt=UNIFORM)
    assert info.bb_tc_levels > 0
    compare_uniform(w, comp, max(1e-6, w.tol))
    comp.close()


def test_exact_uniform_hmatrix_recovered_on_gpu():
    import torch
    from test_oracle_uniform import random_uniform_hmatrix
    x = W.torus(2000, 12)
    t = ot.build_tree(x, 24)
    A = random_uniform_hmatrix(t, 6, 21)
    Aorig = np.empty_like(A)
    Aorig[np.ix_(t.perm, t.perm)] = A
    w = W.Workload("uhmat", x, W.K_LAPLACE3D, leaf_size=24, r=16, tol=1e-10, dense=Aorig, seed=5)
    comp, _ = run_gpu(w, keep=False, fmt=UNIFORM)
    X = np.random.default_rng(3).standard_normal((w.n, 3))
    Y = comp.apply(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.linalg.norm(Y - Aorig @ X) <= 1e-12 * np.linalg.norm(Aorig @ X)
    comp.close()
