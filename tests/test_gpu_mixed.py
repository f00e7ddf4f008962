"""Mixed precision (tcgen05 split-BF16 black box) against the FP64 oracle,
with the peel, QR and core solves in FP64 (HM_MIXED_BF16X6) and in FP32
(HM_MIXED_BF16X6_F32).

The black-box samples must match the FP64 products to FP32-class accuracy
(<= 1e-6 relative per level) on the entries the method reads (the rows of
every colour's sample tiles), and the compressed operator must apply within
the stated tolerance of the oracle's: 1e-6, or the workload's truncation
tolerance when that is larger (a rank decision at the threshold may differ
once the samples carry FP32-level rounding).
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle import graph as og
from oracle import h1 as oh1
from oracle import tree as ot

from gpu_helpers import hm, oracle_op, run_gpu, samples, tile_mask

pytestmark = pytest.mark.gpu

MIXED = 1        # split-BF16 black box; FP64 peel, QR and core solves
MIXED_F32 = 2    # the same black box; FP32 peel products, QR and core solves
TOL_MIXED = 1e-6


def mixed_workloads():
    return {
        "torus_6k": W.torus_laplace(n=6000, tol=1e-6, r=32),
        "torus_ragged_r16": W.Workload("torus_ragged", W.torus(3333, 17), W.K_LAPLACE3D, leaf_size=23, r=16,
                                       tol=1e-5, seed=99, oversample=6),
        "sphere_invr_r24": W.Workload("sphere_invr", W.sphere(4001, 5), W.K_INVR, leaf_size=40, r=24, tol=1e-6,
                                      seed=7, oversample=8),
        "grid_log_r40": W.Workload("grid_log", W.grid2d(48), W.K_LOG, leaf_size=32, r=40, rank=20, seed=2),
        "cube_exp_r8": W.Workload("cube_exp", np.random.default_rng(4).random((2100, 3)), W.K_EXP, leaf_size=40,
                                  r=8, rank=4, seed=3),
        # level-2 tiles of 2000 rows: the tall-skinny QR path (tiles above the
        # shared-memory limit of the one-CTA kernel).  1/r: with a kernel whose
        # far field does not decay (log, exp) the peeled tiles of an 8-level 1D
        # tree are far smaller than the raw samples, and FP32-class sample
        # rounding alone puts the result 2e-6..6e-6 from the FP64 oracle.
        "line_tall_r16": W.Workload("line_tall", W.line1d(8000, 11), W.K_INVR, leaf_size=64, r=16, rank=12,
                                    seed=11),
        # r above 40: two accumulator sets of 4r tensor-memory columns (r <= 64)
        "sphere_invr_r48": W.Workload("sphere48", W.sphere(4500, 6), W.K_INVR, leaf_size=64, r=48, tol=1e-8,
                                      seed=8),
        "torus_r64": W.Workload("torus64", W.torus(5000, 12), W.K_LAPLACE3D, leaf_size=64, r=64, tol=1e-9,
                                seed=10),
    }


@pytest.mark.parametrize("name", list(mixed_workloads()))
def test_mixed_raw_samples(name):
    m = hm()
    w = mixed_workloads()[name]
    comp, _ = run_gpu(w, precision=MIXED, compress=False)
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
        # the sampler computes the rows of the sample tiles only
        mask = tile_mask(t, l, col, w.r)
        assert mask.any()
        Yr, Zr = np.where(mask, Yr, 0.0), np.where(mask, Zr, 0.0)
        Y = np.where(mask, samples(comp, m.HM_X_SAMPLE_Y, l, w.n, chi, w.r), 0.0)
        Z = np.where(mask, samples(comp, m.HM_X_SAMPLE_Z, l, w.n, chi, w.r), 0.0)
        ey = np.linalg.norm(Y - Yr) / np.linalg.norm(Yr)
        ez = np.linalg.norm(Z - Zr) / np.linalg.norm(Zr)
        assert ey <= TOL_MIXED and ez <= TOL_MIXED, (l, ey, ez)
        # every entry, relative to its row's scale
        rowscale = np.linalg.norm(Yr, axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(Y - Yr) / rowscale) <= 1e-5, l
    comp.close()


@pytest.mark.parametrize("precision", [MIXED, MIXED_F32], ids=["fp64-solves", "fp32-solves"])
@pytest.mark.parametrize("name", list(mixed_workloads()))
def test_mixed_compression_matches_oracle(name, precision):
    import torch
    w = mixed_workloads()[name]
    comp, info = run_gpu(w, precision=precision, keep=False)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    H = oh1.compress(t, oracle_op(w, t), w.r, rank=w.rank, tol=w.tol, seed=w.seed, oversample=w.oversample)
    x = np.random.default_rng(1).standard_normal((w.n, 3))
    for trans in (0, 1):
        y = comp.apply(torch.from_numpy(x).cuda(), trans=trans).cpu().numpy()
        yr = np.empty_like(x)
        yr[t.perm] = oh1.apply_h1(H, x[t.perm], transpose=bool(trans))
        e = np.linalg.norm(y - yr) / np.linalg.norm(yr)
        assert e <= max(TOL_MIXED, w.tol), (trans, e)
    comp.close()


@pytest.mark.parametrize("name", ["sphere_invr_r48", "torus_r64"])
def test_tensor_path_covers_r_up_to_64(name):
    """With r of 48 and 64 every admissible level is sampled on the tensor cores
    (none falls back to the FP64 black box)."""
    w = mixed_workloads()[name]
    comp, info = run_gpu(w, precision=MIXED, keep=False)
    levels = sum(1 for l in range(2, info.L + 1) if info.pairs[l] > 0)
    assert info.bb_tc_levels == levels and info.bb_fp64_levels == 0, (info.bb_tc_levels, info.bb_fp64_levels)
    comp.close()


def _level_block_errors(comp, H):
    """Per level: ranks (GPU, oracle) and the aggregate relative error of the
    blocks U B V^T, sqrt(sum ||blk - ref||^2 / sum ||ref||^2)."""
    from gpu_helpers import factors
    out = {}
    for l, lf in H.levels.items():
        if not lf.pairs:
            continue
        ranks, fac = factors(comp, l, lf.rng_a, lf.rng_b)
        ref_ranks = np.array([[u.shape[1], v.shape[1]] for u, v in zip(lf.U, lf.V)])
        num = den = 0.0
        for (U, B, V), Ur, Br, Vr in zip(fac, lf.U, lf.B, lf.V):
            if U.shape[1] == Ur.shape[1] and V.shape[1] == Vr.shape[1]:
                ref = Ur @ Br @ Vr.T
                num += np.sum((U @ B @ V.T - ref) ** 2)
                den += np.sum(ref ** 2)
        out[l] = (ranks, ref_ranks, np.sqrt(num / max(den, 1e-300)))
    return out


@pytest.mark.parametrize("name", ["grid_log_r40", "cube_exp_r8", "line_tall_r16", "torus_6k"])
def test_mixed_blocks_match_oracle(name):
    """Block by block (Algorithm 4.1 per admissible pair) in the spec precision:
    with a fixed rank the ranks are identical and the blocks U B V^T agree with
    the oracle's to 1e-5 per level (FP32-class samples, a basis perturbed by
    the sample error over the spectral gap at k); with a tolerance a rank may
    move where pivot norms sit within the samples' rounding of the threshold:
    by one, or by two where two adjacent pivots both do (on the 6k torus 0.3 %,
    1.5 % and 1.8 % of the pairs at levels 2, 3, 4, one of them by two; at most
    5 % and two allowed), and the blocks of equal rank agree to the same bound."""
    w = mixed_workloads()[name]
    comp, _ = run_gpu(w, precision=MIXED, keep=False)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    H = oh1.compress(t, oracle_op(w, t), w.r, rank=w.rank, tol=w.tol, seed=w.seed, oversample=w.oversample)
    rows = []
    for l, (ranks, ref_ranks, e) in _level_block_errors(comp, H).items():
        d = np.abs(ranks - ref_ranks)
        rows.append((l, int(d.max()), float(np.mean(d > 0)), float(e)))
    print(name, "level, max rank move, fraction moved, block error:", rows)
    for l, dmax, frac, e in rows:
        if w.rank and not w.tol:
            assert dmax == 0, l
        else:
            assert dmax <= 2 and frac <= 0.05, (l, dmax, frac)
        assert e <= 1e-5, (l, e)
    comp.close()


def deep_1d_workloads():
    return {
        "line_log": W.Workload("line_log", W.line1d(8000, 11), W.K_LOG, leaf_size=64, r=16, rank=12, seed=11),
        "line_exp": W.Workload("line_exp", W.line1d(8000, 11), W.K_EXP, leaf_size=64, r=16, rank=12, seed=11),
    }


# measured: 2.1e-6 (log) and 2.5e-6 (exp) with FP64 solves, 1.0e-5 and 1.3e-5
# with FP32 solves
DEEP_1D_BOUND = {MIXED: 5e-6, MIXED_F32: 2e-5}


@pytest.mark.parametrize("precision", [MIXED, MIXED_F32], ids=["fp64-solves", "fp32-solves"])
@pytest.mark.parametrize("name", list(deep_1d_workloads()))
def test_mixed_deep_1d_non_decaying_kernels(name, precision):
    """log|x-y| and exp(-|x-y|) on an 8-level 1D tree: the far field does not
    decay, so the coarser levels' contribution that the peel removes is far
    larger than the level's own blocks, and the FP32-class rounding of the
    raw samples (about 1e-7 of the raw sample) is amplified in the peeled
    tiles.  The stated bound for this case, relative on the applied operator,
    is 5e-6 in the spec precision (FP64 solves) and 2e-5 with FP32 solves
    (1e-6 holds for kernels that decay, tested above); the raw samples
    themselves still meet 1e-6 on the tile rows."""
    import torch
    w = deep_1d_workloads()[name]
    comp, _ = run_gpu(w, precision=precision, keep=False)
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    assert t.L >= 7
    H = oh1.compress(t, oracle_op(w, t), w.r, rank=w.rank, tol=w.tol, seed=w.seed, oversample=w.oversample)
    x = np.random.default_rng(1).standard_normal((w.n, 3))
    errs = []
    for trans in (0, 1):
        y = comp.apply(torch.from_numpy(x).cuda(), trans=trans).cpu().numpy()
        yr = np.empty_like(x)
        yr[t.perm] = oh1.apply_h1(H, x[t.perm], transpose=bool(trans))
        errs.append(np.linalg.norm(y - yr) / np.linalg.norm(yr))
    print(f"{name} precision {precision}: apply error vs oracle {errs}")
    assert max(errs) <= DEEP_1D_BOUND[precision], errs
    comp.close()
