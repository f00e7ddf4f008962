"""Pins of the oracle's H^2 compression (Section 4.3, Algorithm 4.2) and of the
nested apply (Algorithm 4.3) against what the paper and the mathematics fix.

CPU only.  Exact recovery of random exact H^2 matrices (nested bases built
bottom-up on the tree): sampling is exact when every far field has rank <= r - p
(Section 2.5), and the nested bases can only hold the parents' ranges if the
samples are augmented by the parents' far fields (Section 4.3); the nested apply
of Algorithm 4.3 against the sum of expanded blocks; the truncated SVD against
its definition; a kernel matrix against its dense 2-norm.
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle import h1, h2
from oracle import tree as ot


def _children(t, l):
    ch = {}
    for a, p in enumerate(t.cut_parent[l]):
        ch.setdefault(p, []).append(a)
    return ch


def random_h2matrix(t, k, seed):
    """sum over admissible pairs of U_alpha S_ab V_beta^T plus random dense near
    blocks, with U and V nested (eq. nested_basis): orthonormal long bases on
    cut L, and on every coarser cut U_tau = diag(U_alpha) Ut_tau with a random
    orthonormal Ut_tau (rank <= k everywhere)."""
    rng = np.random.default_rng(seed)
    L = t.L
    bases = {}
    for l in range(L, 1, -1):
        U, V = {}, {}
        for side in (U, V):
            for a in range(len(t.cuts[l])):
                a0, a1 = t.rng(l, a)
                if l == L:
                    side[a] = np.linalg.qr(rng.standard_normal((a1 - a0, min(k, a1 - a0))))[0]
            if l < L:
                lower = bases[l + 1][0] if side is U else bases[l + 1][1]
                for tau, kids in _children(t, l + 1).items():
                    blocks = [lower[a] for a in kids]
                    D = np.zeros((sum(b.shape[0] for b in blocks), sum(b.shape[1] for b in blocks)))
                    i = j = 0
                    for b in blocks:
                        D[i:i + b.shape[0], j:j + b.shape[1]] = b
                        i += b.shape[0]
                        j += b.shape[1]
                    kk = min(k, D.shape[1])
                    side[tau] = D @ np.linalg.qr(rng.standard_normal((D.shape[1], kk)))[0]
        bases[l] = (U, V)
    A = np.zeros((t.n, t.n))
    for l in range(2, L + 1):
        U, V = bases[l]
        for a, b in ot.admissible_pairs(t, l):
            a0, a1 = t.rng(l, a)
            b0, b1 = t.rng(l, b)
            A[a0:a1, b0:b1] = U[a] @ rng.standard_normal((U[a].shape[1], V[b].shape[1])) @ V[b].T
    for a, b in ot.near_pairs(t, L):
        a0, a1 = t.rng(L, a)
        b0, b1 = t.rng(L, b)
        A[a0:a1, b0:b1] = rng.standard_normal((a1 - a0, b1 - b0))
    return A


def test_svd_trunc_definition():
    rng = np.random.default_rng(0)
    Q1 = np.linalg.qr(rng.standard_normal((40, 12)))[0]
    P = Q1 @ np.diag(10.0 ** -np.arange(12)) @ np.linalg.qr(rng.standard_normal((12, 12)))[0]
    U, s = h2.svd_trunc(P, 0, 3e-6, 12)
    W, sv, _ = np.linalg.svd(P)
    assert U.shape[1] == int(np.sum(sv > 3e-6 * sv[0])) == 6
    assert np.allclose(s, 10.0 ** -np.arange(6), rtol=1e-10)
    assert np.allclose(s, sv[:6], rtol=1e-12)
    assert np.allclose(U.T @ U, np.eye(6), atol=1e-13)
    # the same projector as the SVD's leading vectors, each signed by its largest entry
    assert np.allclose(U @ U.T, W[:, :6] @ W[:, :6].T, atol=1e-12)
    assert all(U[np.argmax(np.abs(U[:, j])), j] > 0 for j in range(6))
    U2, s2 = h2.svd_trunc(P, 4, 0.0, 12)
    assert U2.shape[1] == 4 and np.allclose(U2, U[:, :4], atol=1e-12)
    assert h2.svd_trunc(P, 0, 3e-6, 3)[0].shape[1] == 3      # the cap
    assert h2.svd_trunc(np.zeros((5, 3)), 0, 3e-6, 3)[0].shape[1] == 0


@pytest.mark.parametrize("geom,kw", [("torus", {"tol": 1e-10}), ("cube", {"rank": 6}), ("line", {"tol": 1e-10})])
def test_exact_h2_matrix_recovered(geom, kw):
    """The compressed operator equals an exact H^2 matrix to rounding; the
    nested apply (Algorithm 4.3) gives the same product as the expanded blocks."""
    if geom == "torus":
        x = W.torus(1500, 12)
    elif geom == "cube":
        x = np.random.default_rng(3).random((1300, 3)) ** 3   # clustered at a corner: a deep adaptive tree
    else:
        x = W.line1d(900, 4)
    t = ot.build_tree(x, 24)
    assert t.L >= 4
    A = random_h2matrix(t, 6, 21)
    H = h2.compress_h2(t, h1.DenseOp(A), 16, seed=5, **kw)
    I = np.eye(t.n)
    At = h2.apply_h2(H, I)
    assert np.linalg.norm(At - A) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(h2.apply_h2(H, I, transpose=True) - A.T) <= 1e-12 * np.linalg.norm(A)
    # short bases exist for every coarser cut that has a far field
    assert set(H.Ut) == set(range(2, t.L)) and set(H.Vt) == set(range(2, t.L))


def test_augmentation_is_needed():
    """Without the parents' far fields in the samples (the uniform H^1 bases of
    Section 4.2 nested as they are), the children's bases miss part of the
    parents' ranges and the nested operator is not exact: the augmentation of
    Section 4.3 is what makes eq. nested_basis hold."""
    x = W.torus(1500, 12)
    t = ot.build_tree(x, 24)
    A = random_h2matrix(t, 6, 21)
    H = h2.compress_h2(t, h1.DenseOp(A), 16, seed=5, tol=1e-10)
    # nested bases span the children's augmented ranges: each expanded U_tau
    # equals diag(U_alpha) Ut_tau exactly, and the long U_tau is reproduced
    Hu = h1.compress_uniform(t, h1.DenseOp(A), 16, seed=5, tol=1e-10)
    lost = 0.0
    for l in range(3, t.L + 1):
        Uc, _ = Hu.bases[l]
        Up, _ = Hu.bases[l - 1]
        for tau, kids in _children(t, l).items():
            if tau not in Up:
                continue
            t0 = t.rng(l - 1, tau)[0]
            for a in kids:
                a0, a1 = t.rng(l, a)
                blk = Up[tau][a0 - t0:a1 - t0]
                Ua = Uc.get(a, np.zeros((a1 - a0, 0)))
                lost = max(lost, np.linalg.norm(blk - Ua @ (Ua.T @ blk)) / max(np.linalg.norm(blk), 1e-300))
    assert lost > 1e-3          # uniform H^1 bases are not nested
    for l in range(3, t.L + 1):
        Uc, _ = H.bases[l]
        for tau, blocks in H.Ut[l - 1].items():
            for a, Ut in blocks:
                assert Ut.shape == (Uc[a].shape[1], H.bases[l - 1][0][tau].shape[1])


def test_nested_apply_equals_expanded_blocks():
    """Algorithm 4.3 (upward and downward passes through the short bases) and
    the plain sum of U B V^T blocks with the nested long bases are the same
    operator."""
    w = W.torus_laplace(n=2500, tol=1e-6, r=32)
    t = ot.build_tree(w.points, 32)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    H = h2.compress_h2(t, op, 32, tol=1e-6, seed=w.seed)
    X = np.random.default_rng(2).standard_normal((w.n, 3))
    for tr in (False, True):
        a = h2.apply_h2(H, X, transpose=tr)
        b = h1.apply_h1(H, X, transpose=tr)
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_h2_compression_of_a_kernel_matrix():
    """1/(4 pi r) on a torus at tol 1e-6: the H^2 operator reaches the
    tolerance's order in the dense 2-norm and stores fewer floats than the
    uniform H^1 operator of the same job."""
    w = W.torus_laplace(n=2000, tol=1e-6, r=48)
    t = ot.build_tree(w.points, 32)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    A = op.dense()
    H = h2.compress_h2(t, op, 48, tol=1e-6, seed=w.seed)
    Hu = h1.compress_uniform(t, op, 48, tol=1e-6, seed=w.seed)
    e = np.linalg.norm(h2.apply_h2(H, np.eye(w.n)) - A, 2) / np.linalg.norm(A, 2)
    assert e <= 1e-5, e
    assert H.floats() < Hu.floats()


def test_result_does_not_depend_on_singular_vector_signs(monkeypatch):
    """The augmentation and the stage-2 mixes are written through the bases
    themselves (G = U_tau^T Gamma_tau, M_a = U_a^T Gamma'_a), so flipping the
    sign of every singular vector leaves the compressed operator unchanged to
    rounding: rounding-level differences in a basis cannot change a sketch."""
    w = W.torus_laplace(n=2000, tol=1e-6, r=32)
    t = ot.build_tree(w.points, 32)
    op = h1.KernelOp(w.points[t.perm], w.kernel)
    X = np.random.default_rng(4).standard_normal((w.n, 2))
    H = h2.compress_h2(t, op, 32, tol=1e-6, seed=w.seed)
    ref = h2.apply_h2(H, X)
    base = h2.svd_trunc

    def flipped(P, rank, tol, cap):
        U, s = base(P, rank, tol, cap)
        return -U, s

    monkeypatch.setattr(h2, "svd_trunc", flipped)
    Hf = h2.compress_h2(t, op, 32, tol=1e-6, seed=w.seed)
    assert np.linalg.norm(h2.apply_h2(Hf, X) - ref) <= 1e-12 * np.linalg.norm(ref)
