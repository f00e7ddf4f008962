"""Pins of the oracle's numerics: Philox, Gaussians, sampling, exact recovery,
truncation quality, apply and the error estimate.  CPU only.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import hm_workloads as W
from oracle import h1
from oracle import tree as ot
from oracle.philox import gaussian_block, philox4x32_10, uniform53

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = philox4x32_10([np.array([c]) for c in v[:4]], [np.array([k]) for k in v[4:6]])
        assert [int(o[0]) for o in out] == v[6:]


def test_uniform53_range_and_gaussian_moments():
    u = uniform53(np.array([0, 0xFFFFFFFF], dtype=np.uint64), np.array([0, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 2.0 ** -53 and u[1] == 1.0 - 2.0 ** -53
    g = gaussian_block(12345, 0, 3, 77, 4000, 50).ravel()
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.01
    assert abs(np.mean(g ** 4) - 3.0) < 0.06
    # counter keys: a different box, side or level gives different numbers
    a = gaussian_block(1, 0, 2, 5, 3, 4)
    assert not np.allclose(a, gaussian_block(1, 1, 2, 5, 3, 4))
    assert not np.allclose(a, gaussian_block(1, 0, 3, 5, 3, 4))
    assert not np.allclose(a, gaussian_block(1, 0, 2, 6, 3, 4))
    assert np.array_equal(a, gaussian_block(1, 0, 2, 5, 3, 4))
    # entry (i, j) does not depend on the block's shape
    assert np.array_equal(gaussian_block(1, 0, 2, 5, 8, 6)[:3, :4], a)


def test_kernel_values():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    K = h1.kernel_eval(2, x, x)
    assert K[0, 0] == 0.0 and K[0, 1] == pytest.approx(1.0 / (4 * math.pi))
    assert K[0, 2] == pytest.approx(1.0 / (8 * math.pi))
    assert h1.kernel_eval(1, x, x)[0, 2] == pytest.approx(math.log(2.0))
    assert h1.kernel_eval(3, x, x)[1, 0] == 1.0
    assert h1.kernel_eval(4, x, x)[0, 0] == 1.0


def random_hmatrix(t, k, seed):
    """An exact rank-k H^1 matrix on the tree: random U B V^T on every admissible
    pair and random dense leaf-neighbour blocks, assembled densely."""
    rng = np.random.default_rng(seed)
    A = np.zeros((t.n, t.n))
    for l in range(2, t.L + 1):
        for a, b in ot.admissible_pairs(t, l):
            (a0, a1), (b0, b1) = t.rng(l, a), t.rng(l, b)
            kk = min(k, a1 - a0, b1 - b0)
            A[a0:a1, b0:b1] = rng.standard_normal((a1 - a0, kk)) @ rng.standard_normal((kk, b1 - b0))
    for a, b in ot.near_pairs(t, t.L):
        (a0, a1), (b0, b1) = t.rng(t.L, a), t.rng(t.L, b)
        A[a0:a1, b0:b1] = rng.standard_normal((a1 - a0, b1 - b0))
    return A


@pytest.mark.parametrize("geom", ["line", "torus", "grid"])
def test_exact_recovery_of_rank_k_hmatrix(geom):
    """Randomized sampling is exact when every block has rank <= r (Sec. 2.5):
    the whole peeling pipeline must recover an exact H^1 matrix to ~1e-12."""
    if geom == "line":
        x = W.line1d(600, 3)
        t = ot.build_tree(x, 16, uniform_depth=5)
    elif geom == "torus":
        t = ot.build_tree(W.torus(1500, 4), 24)
    else:
        t = ot.build_tree(W.grid2d(32), 16)
    A = random_hmatrix(t, 6, 11)
    op = h1.DenseOp(A)
    for kw in ({"rank": 6}, {"tol": 1e-9}):
        H = h1.compress(t, op, r=16, seed=5, **kw)
        Ac = h1.apply_h1(H, np.eye(t.n))
        err = np.linalg.norm(Ac - A) / np.linalg.norm(A)
        assert err < 1e-12, (kw, err)
        if "tol" in kw:
            for lf in H.levels.values():
                for (a0, a1), (b0, b1), U, V in zip(lf.rng_a, lf.rng_b, lf.U, lf.V):
                    assert U.shape[1] == min(6, a1 - a0, b1 - b0)


def test_level2_samples_are_block_times_gaussian():
    """At level 2 nothing is peeled: Y(I_alpha, c) = A(I_alpha, I_beta) G_beta
    exactly (eq. h1testmatrices), for every admissible pair."""
    w = W.torus_laplace(n=1200)
    t = ot.build_tree(w.points, 32)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    A = op.dense()
    H = h1.compress(t, op, r=8, tol=1e-8, seed=w.seed, keep_samples=True, levels_only=True)
    lf = H.levels[2]
    G = h1.gaussians(t, 2, 0, 8, w.seed)
    pc = lf.coloring.pair_color
    for i, ((a0, a1), (b0, b1)) in enumerate(zip(lf.rng_a, lf.rng_b)):
        c = pc[i]
        ref = A[a0:a1, b0:b1] @ G[b0:b1]
        got = lf.Y[a0:a1, c * 8:(c + 1) * 8]
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_alg21_textbook_single_block():
    """Alg. 2.1 on one low-rank block equals a direct textbook computation:
    U spans qr(A G1), V spans qr(A^T G2), and U B V^T reproduces A."""
    rng = np.random.default_rng(0)
    A = rng.standard_normal((50, 5)) @ rng.standard_normal((5, 40))
    G1, G2 = rng.standard_normal((40, 9)), rng.standard_normal((50, 9))
    U = h1.qr_trunc(A @ G1, 5, 0.0, 9)
    V = h1.qr_trunc(A.T @ G2, 5, 0.0, 9)
    B = h1.core(G2, A @ G1, G1, U, V)
    assert np.linalg.norm(U @ B @ V.T - A) < 1e-12 * np.linalg.norm(A)
    Q = np.linalg.qr(A @ G1)[0]
    # same column space as the unpivoted textbook basis
    assert np.linalg.norm(Q @ (Q.T @ U) - U) < 1e-12
    assert np.allclose(U.T @ U, np.eye(5), atol=1e-13)


def test_qr_trunc_conventions():
    rng = np.random.default_rng(1)
    P = rng.standard_normal((30, 8)) @ np.diag([1, 1e-1, 1e-2, 1e-3, 1e-5, 1e-7, 1e-9, 1e-11])
    Q, R, piv = scipy.linalg.qr(P, mode="economic", pivoting=True)
    for tol, kexp in ((1e-4, None), (1e-6, None)):
        U = h1.qr_trunc(P, 0, tol, 8)
        d = np.abs(np.diag(R))
        assert U.shape[1] == int(np.sum(d > tol * d[0]))
        # R_jj >= 0 convention: U^T P has a non-negative pivoted diagonal
        Rk = U.T @ P[:, piv]
        assert np.all(np.diag(Rk)[:U.shape[1]] > 0)
    assert h1.qr_trunc(P, 3, 0.0, 8).shape == (30, 3)
    assert h1.qr_trunc(P[:2], 5, 0.0, 8).shape == (2, 2)
    assert h1.qr_trunc(np.zeros((5, 4)), 0, 1e-6, 4).shape == (5, 0)


def test_truncation_quality_against_dense_svd():
    """Eckart-Young (Sec. 2.3): each compressed level-2 block's error is within a
    modest factor of the optimal sigma_{k+1} (dense SVD at tiny N), with
    oversampling p = r - k = 10 (Sec. 2.5).  Level 2 is the only level whose
    samples carry no peeled coarse-level error; finer levels are pinned by the
    exact-recovery test instead."""
    w = W.torus_laplace(n=900)
    t = ot.build_tree(w.points, 24)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    A = op.dense()
    H = h1.compress(t, op, r=16, rank=6, seed=w.seed)
    worst = 0.0
    for lf in [H.levels[2]]:
        for (a0, a1), (b0, b1), U, B, V in zip(lf.rng_a, lf.rng_b, lf.U, lf.B, lf.V):
            blk = A[a0:a1, b0:b1]
            s = np.linalg.svd(blk, compute_uv=False)
            k = U.shape[1]
            if k >= len(s) or s[k] < 1e-14 * s[0]:
                continue
            worst = max(worst, np.linalg.norm(blk - U @ B @ V.T, 2) / s[k])
    assert 1.0 <= worst < 30.0


def test_apply_matches_assembled_and_adjoint():
    w = W.torus_laplace(n=1000)
    t = ot.build_tree(w.points, 24)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    H = h1.compress(t, op, r=24, tol=1e-6, seed=w.seed)
    Ac = np.zeros((t.n, t.n))
    for lf in H.levels.values():
        for (a0, a1), (b0, b1), U, B, V in zip(lf.rng_a, lf.rng_b, lf.U, lf.B, lf.V):
            Ac[a0:a1, b0:b1] += U @ B @ V.T
    for (a0, a1), (b0, b1), D in zip(H.leaf.rng_a, H.leaf.rng_b, H.leaf.D):
        Ac[a0:a1, b0:b1] += D
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((t.n, 3)), rng.standard_normal((t.n, 3))
    assert np.allclose(h1.apply_h1(H, x), Ac @ x, rtol=1e-12, atol=1e-12)
    assert np.allclose(h1.apply_h1(H, y, transpose=True), Ac.T @ y, rtol=1e-12, atol=1e-12)
    A = op.dense()
    E = h1.relative_error(H, op, iters=20)
    Ed = np.linalg.norm(Ac - A, 2) / np.linalg.norm(A, 2)
    assert E <= Ed * 1.0000001 and E > 0.5 * Ed
    assert Ed < 1e-5


def test_leaf_blocks_are_exact_kernel_blocks():
    """With exact coarser factors, the leaf step returns A(I_alpha, I_beta)."""
    t = ot.build_tree(W.torus(1200, 2), 24)
    A = random_hmatrix(t, 5, 3)
    H = h1.compress(t, h1.DenseOp(A), r=10, rank=5, seed=1)
    for (a0, a1), (b0, b1), D in zip(H.leaf.rng_a, H.leaf.rng_b, H.leaf.D):
        assert np.allclose(D, A[a0:a1, b0:b1], rtol=0, atol=1e-11)


def test_matvec_count_formula():
    """Number of applied columns = r * sum_l chi_l (both sides) + m_max * chi_leaf."""
    w = W.line1d_dense()
    t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
    H = h1.compress(t, h1.DenseOp(w.dense[t.perm][:, t.perm]), w.r, rank=w.rank, seed=w.seed)
    chis = [lf.coloring.n_colors for lf in H.levels.values()]
    assert H.matvec_cols == 2 * w.r * sum(chis) + H.leaf.m_max * H.leaf.coloring.n_colors
    assert all(c <= 6 for c in chis) and H.leaf.coloring.n_colors <= 3


def test_pivoted_qr_matches_lapack_without_near_ties():
    """The oracle's own Businger-Golub QR picks LAPACK's pivots and returns the
    same signed Q_k whenever no two column norms nearly tie."""
    rng = np.random.default_rng(0)
    for t in range(150):
        m, n = int(rng.integers(3, 40)), int(rng.integers(2, 20))
        P = rng.standard_normal((m, n)) @ np.diag(10.0 ** -rng.uniform(0, 8, n))
        Q, k = h1.pivoted_qr(P, min(m, n), 0, 1e-6)
        Q2, R2, piv = scipy.linalg.qr(P, mode="economic", pivoting=True)
        d = np.abs(np.diag(R2))
        k2 = int(np.sum(np.cumprod(d > 1e-6 * d[0])))
        assert k == k2
        assert np.allclose(Q, Q2[:, :k2] * np.where(np.diag(R2)[:k2] < 0, -1, 1), atol=1e-10)
        assert np.allclose(Q.T @ Q, np.eye(k), atol=1e-13)


def test_core_least_squares_equals_pseudo_inverse():
    rng = np.random.default_rng(5)
    Ga, Gb = rng.standard_normal((40, 12)), rng.standard_normal((30, 12))
    U = np.linalg.qr(rng.standard_normal((40, 7)))[0]
    V = np.linalg.qr(rng.standard_normal((30, 5)))[0]
    P = rng.standard_normal((40, 12))
    B = h1.core(Ga, P, Gb, U, V)
    ref = np.linalg.pinv(Ga.T @ U) @ (Ga.T @ P) @ np.linalg.pinv(V.T @ Gb)
    assert np.allclose(B, ref, rtol=1e-10, atol=1e-12)


def test_kernelop_rows_equals_dense_rows():
    """KernelOp.rows (the sampled-row product used at full size) equals the
    assembled matrix's rows times X, zero rows of X included, across chunks."""
    w = W.torus_laplace(n=900)
    op = h1.KernelOp(w.points, w.kernel, chunk_elems=5000)  # several chunks
    rng = np.random.default_rng(3)
    X = rng.standard_normal((w.n, 5))
    X[rng.random(w.n) < 0.6] = 0.0
    idx = np.sort(rng.choice(w.n, 77, replace=False))
    ref = op.dense()[idx] @ X
    assert np.allclose(op.rows(idx, X), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_sample_rows_equals_full_sample():
    """sample_rows gives the entries of Y_l = A Omega_l (Omega_l formed in full
    by test_matrix) for arbitrary (row, colour) pairs of every level."""
    from oracle import graph as og
    w = W.torus_laplace(n=1500)
    t = ot.build_tree(w.points, 24)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    rng = np.random.default_rng(8)
    r = 6
    for l in range(2, t.L + 1):
        col = og.color_level(t, l)
        if col.n_vertices == 0:
            continue
        G = h1.gaussians(t, l, 0, r, w.seed)
        Y = op.apply(h1.test_matrix(t, l, col, G, r))
        rows = rng.integers(0, w.n, 40)
        colors = rng.integers(0, col.n_colors, 40)
        got = h1.sample_rows(op, t, l, col, G, r, rows, colors)
        ref = np.stack([Y[i, c * r:(c + 1) * r] for i, c in zip(rows, colors)])
        assert np.allclose(got, ref, rtol=0, atol=1e-13 * max(np.abs(ref).max(), 1e-300)), l
