"""H^2 (Section 4.3, Algorithm 4.2; nested apply of Algorithm 4.3) on the GPU
against the oracle's compress_h2 / apply_h2.

* FP64: the rank of every entry's column and row basis equals the oracle's, the
  singular values S^in and S^out agree to 1e-10 of the entry's largest, and the
  nested operator (both products) agrees to 1e-10; the stored float count is
  the oracle's exactly (long bases of the finest cut, short bases, cores, leaf
  blocks).  The sketches are written through the bases (G = U^T Gamma), so
  rounding-level differences in a basis cannot change them.
* An exact H^2 matrix is recovered to 1e-12.
* Split-BF16 tensor-core black box: the operator within max(1e-6, tol) of the
  oracle's FP64 compression.
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle import h1 as oh1
from oracle import h2 as oh2
from oracle import tree as ot

from gpu_helpers import f64, hm, i32, oracle_op, run_gpu

pytestmark = pytest.mark.gpu

H2 = 2
TOL64 = 1e-10


def workloads():
    return {
        "torus_3k": W.Workload("torus_h2", W.torus(3000, 31), W.K_LAPLACE3D, leaf_size=32, r=32, tol=1e-7, seed=9),
        "cube_exp_rank": W.Workload("cube_h2", np.random.default_rng(4).random((2500, 3)), W.K_EXP, leaf_size=40,
                                    r=24, rank=12, seed=3),
        "sphere_ragged": W.Workload("sphere_h2", W.sphere(2777, 5), W.K_INVR, leaf_size=23, r=24, tol=1e-6, seed=7,
                                    oversample=8),
        "clustered_cube": W.Workload("clustered_h2", np.random.default_rng(8).random((3000, 3)) ** 3, W.K_LAPLACE3D,
                                     leaf_size=24, r=32, tol=1e-8, seed=4),
    }


def oracle_h2(w):
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    H = oh2.compress_h2(t, oracle_op(w, t), w.r, rank=w.rank, tol=w.tol, seed=w.seed, oversample=w.oversample)
    return t, H


def apply_errors(w, comp, t, H):
    import torch
    x = np.random.default_rng(1).standard_normal((w.n, 2))
    out = []
    for trans in (0, 1):
        y = comp.apply(torch.from_numpy(x).cuda(), trans=trans).cpu().numpy()
        yr = np.empty_like(x)
        yr[t.perm] = oh2.apply_h2(H, x[t.perm], transpose=bool(trans))
        out.append(np.linalg.norm(y - yr) / np.linalg.norm(yr))
    return out


@pytest.mark.parametrize("name", list(workloads()))
def test_h2_fp64_matches_oracle(name):
    m = hm()
    w = workloads()[name]
    comp, info = run_gpu(w, keep=False, fmt=H2)
    t, H = oracle_h2(w)
    r = w.r
    for l in range(2, t.L + 1):
        if l not in H.bases:
            continue
        nc = len(t.cuts[l])
        U, V = H.bases[l]
        Sin, Sout = H.S[l]
        ks = i32(comp.export(m.HM_X_H2_RANKS, l)).reshape(2, nc)
        ref = np.array([[U[a].shape[1] if a in U else 0 for a in range(nc)],
                        [V[a].shape[1] if a in V else 0 for a in range(nc)]])
        assert np.array_equal(ks, ref), f"ranks differ at cut {l}"
        sig = f64(comp.export(m.HM_X_H2_SIGMA, l)).reshape(nc, 2, r)
        for side, S in ((0, Sin), (1, Sout)):
            for a, s_ref in S.items():
                k = len(s_ref)
                if k == 0:
                    continue
                assert np.max(np.abs(sig[a, side, :k] - s_ref)) <= TOL64 * s_ref[0], (l, side, a)
    e = apply_errors(w, comp, t, H)
    assert max(e) <= TOL64, e
    assert info.factor_floats == H.floats(), (info.factor_floats, H.floats())
    comp.close()


def test_h2_relative_error_matches_oracle():
    w = workloads()["torus_3k"]
    comp, _ = run_gpu(w, keep=False, fmt=H2)
    e_gpu = comp.relerr(comp._op, 20)
    t, H = oracle_h2(w)
    e_ref = oh1.relative_error(H, oracle_op(w, t), 20, seed=w.seed + 1)
    assert abs(e_gpu - e_ref) <= 1e-6 * e_ref + 1e-15, (e_gpu, e_ref)
    comp.close()


@pytest.mark.parametrize("name", ["torus_3k", "sphere_ragged"])
def test_h2_mixed_matches_oracle(name):
    w = workloads()[name]
    comp, info = run_gpu(w, precision=1, keep=False, fmt=H2)
    assert info.bb_tc_levels > 0
    t, H = oracle_h2(w)
    e = apply_errors(w, comp, t, H)
    assert max(e) <= max(1e-6, w.tol), e
    comp.close()


def test_exact_h2_matrix_recovered_on_gpu():
    import torch
    from test_oracle_h2 import random_h2matrix
    x = W.torus(2000, 12)
    t = ot.build_tree(x, 24)
    A = random_h2matrix(t, 6, 21)
    Aorig = np.empty_like(A)
    Aorig[np.ix_(t.perm, t.perm)] = A
    w = W.Workload("h2mat", x, W.K_LAPLACE3D, leaf_size=24, r=16, tol=1e-10, dense=Aorig, seed=5)
    comp, _ = run_gpu(w, keep=False, fmt=H2)
    X = np.random.default_rng(3).standard_normal((w.n, 3))
    for trans in (0, 1):
        Y = comp.apply(torch.from_numpy(X).cuda(), trans=trans).cpu().numpy()
        ref = (Aorig.T if trans else Aorig) @ X
        assert np.linalg.norm(Y - ref) <= 1e-12 * np.linalg.norm(ref), trans
    comp.close()


def test_h2_apply_noalloc_refused():
    import torch
    m = hm()
    w = workloads()["torus_3k"]
    comp, _ = run_gpu(w, keep=False, fmt=H2)
    x = torch.ones(w.n, dtype=torch.float64, device="cuda")
    with pytest.raises(m.HMError) as ei:
        comp.apply_noalloc(x)
    assert ei.value.status == m.HM_ENOTSUP
    comp.close()
