"""Oracle: randomized compression of an H^2 matrix (Section 4.3, Algorithm 4.2
with the H^2 branches) and the apply of the nested representation (Algorithm
4.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 4.3 changes the uniform H^1 compression (Section 4.2; h1.compress_uniform)
in three ways, taken here in the paper's order, level by level l = 2..L:

  1. the basis of a box comes from a truncated SVD of its sample instead of a
     QR, and the singular values are kept (S^in for U, S^out for V);
  2. the sample of box alpha (parent tau in cut l-1) is augmented by a sketch
     of the parent's far field, U_tau(I_{tau,alpha}, :) S^in_tau G, so that
     U_alpha spans A(I_alpha, complement of the near field of alpha):
        [U_alpha, S^in_alpha] = svd(Y(I_alpha, :) + U_tau(I_{tau,alpha}, :) S^in_tau G, k)
     and likewise on the row side with the summed stage-2 tiles and
     V_tau(I_{tau,beta}, :) S^out_tau G';
  3. once the bases of cut l exist, every box tau of cut l-1 is nested: its
     short basis Ut_tau solves eq. nested_basis, U_tau = diag(U_alpha) Ut_tau
     over its children alpha; with orthonormal U_alpha the least-squares
     solution is Ut_tau(rows of alpha) = U_alpha^T U_tau(I_{tau,alpha}, :).
     The long U_tau is then replaced by its nested form, and so are the bases of
     the coarser cuts, whose nested forms run through it.

Readings of points where the paper is silent or inconsistent:
  * G_k is printed k x k, but it multiplies the k-column U_tau S_tau and is
    added to an r-column sample, so it is k_tau x r.  Reading: G = U_tau^T
    Gamma_tau, with Gamma_tau an |I_tau| x r Philox Gaussian (side SIDE_AUG_U
    for U and SIDE_AUG_V for V, level l, keyed by the parent box tau).  With
    orthonormal U_tau this G is exactly a k_tau x r standard Gaussian, and the
    augmentation U_tau S_tau U_tau^T Gamma_tau does not depend on the signs of
    the singular vectors or on the basis chosen inside a cluster of equal
    singular values, so two implementations that differ by rounding draw the
    same sketch.
  * The nesting step of Algorithm 4.2 is listed for "boxes alpha in level l",
    but eq. nested_basis expresses a box through its children; the text says
    it is done once the children's long bases exist.  Reading: after the
    bases of cut l, the boxes of cut l-1 are nested.  The sampling of level
    l + 1 therefore peels levels <= l-1 with nested bases and level l with
    its long bases (the order of Algorithm 4.2).
  * A box receives a basis when its sample (stage 1 of the box colouring) or
    its parent's basis is non-empty: on adaptive trees a box can have an empty
    interaction list and still a far field, which the nested chain needs.
  * svd(P, k): k = #{sigma_j > tol sigma_1} with a tolerance (k <= r - p,
    and <= rank when both are given), k = rank with a fixed rank; always
    k <= |I_alpha| and k <= r.  Each singular vector is signed so that its
    entry of largest magnitude (the first on ties) is positive.
  * The stage-2 tiles are summed with Gaussian mixes as in the uniform H^1
    oracle (h1.compress_uniform), for the same reason in the same basis-free
    form: M_a = U_a^T Gamma'_a, Gamma'_a an |I_a| x r Philox Gaussian (side
    SIDE_MIX_H2, level l, keyed by the box a).  B_ab = T_ab^T V_beta.
  * The leaf blocks are extracted as in Section 4.1.3, peeling every level.

Storage of the result: long bases of cut L, short bases (transfer matrices) of
cuts 2..L-1, the cores B of every admissible pair and the leaf blocks.
"""
from __future__ import annotations

import numpy as np

from . import graph as og
from . import tree as ot
from .h1 import H1Matrix, LevelFactors, SIDE_OMEGA, apply_levels, extract_leaf, gaussians
from .philox import gaussian_block

SIDE_AUG_U, SIDE_AUG_V, SIDE_MIX_H2 = 4, 5, 6


def svd_trunc(P: np.ndarray, rank: int, tol: float, cap: int):
    """Truncated SVD of a sample (reading in the module docstring): the first k
    left singular vectors, signed, and their singular values."""
    m, n = P.shape
    kmax = min(m, n, cap)
    if kmax == 0:
        return np.zeros((m, 0)), np.zeros(0)
    W, s, _ = np.linalg.svd(P, full_matrices=False)
    if rank > 0 and tol <= 0.0:
        k = min(rank, kmax)
    elif not (s[0] > 0.0):
        k = 0
    else:
        k = min(int(np.sum(s > tol * s[0])), kmax)
    U = W[:, :k].copy()
    for j in range(k):
        if U[int(np.argmax(np.abs(U[:, j]))), j] < 0.0:
            U[:, j] = -U[:, j]
    return U, s[:k].copy()


class H2Matrix(H1Matrix):
    """H.levels[l]: per-pair references to the (nested, expanded) bases and the
    cores, so h1.apply_h1 applies it; H.long: the long bases of cut L; H.Ut,
    H.Vt: the short bases of cuts 2..L-1, {tau: [(alpha, block)]}."""

    def floats(self) -> int:
        s = 0
        for l, lf in self.levels.items():
            s += sum(b.size for b in lf.B)
        U, V = self.long
        s += sum(u.size for u in U.values()) + sum(v.size for v in V.values())
        for tab in (self.Ut, self.Vt):
            for per in tab.values():
                for blocks in per.values():
                    s += sum(b.size for _, b in blocks)
        if self.leaf is not None:
            s += sum(d.size for d in self.leaf.D)
        return s


def _children(tree, l: int):
    """Entries of cut l grouped by their parent in cut l-1 (Morton order, so
    the children of tau tile I_tau in order)."""
    ch = {}
    for a, p in enumerate(tree.cut_parent[l]):
        ch.setdefault(p, []).append(a)
    return ch


def _nest(tree, l: int, Uprev: dict, U: dict):
    """Short bases of the boxes of cut l-1 from their children's long bases in
    cut l: Ut_tau(rows of alpha) = U_alpha^T U_tau(I_{tau,alpha}, :)."""
    short = {}
    for tau, kids in _children(tree, l).items():
        if tau not in Uprev or Uprev[tau].shape[1] == 0:
            continue
        t0 = tree.rng(l - 1, tau)[0]
        blocks = []
        for a in kids:
            a0, a1 = tree.rng(l, a)
            Ua = U.get(a, np.zeros((a1 - a0, 0)))
            blocks.append((a, Ua.T @ Uprev[tau][a0 - t0:a1 - t0]))
        short[tau] = blocks
    return short


def _expand(tree, l: int, U: dict, short: dict):
    """The bases of cut l-1 that the nested representation defines,
    diag(U_alpha) Ut_tau, from the (effective) bases U of cut l."""
    out = {}
    for tau, blocks in short.items():
        parts = []
        for a, Ut in blocks:
            a0, a1 = tree.rng(l, a)
            parts.append(U.get(a, np.zeros((a1 - a0, 0))) @ Ut)
        out[tau] = np.vstack(parts)
    return out


def _aug_gauss(tree, l: int, Bprev: dict, side: int, r: int, seed: int):
    """G_tau = B_tau^T Gamma_tau for every box tau of cut l-1 with a basis
    (reading in the module docstring)."""
    out = {}
    for tau, B in Bprev.items():
        if B.shape[1] == 0:
            continue
        t0, t1 = tree.rng(l - 1, tau)
        out[tau] = B.T @ gaussian_block(seed, side, l, tree.box(l - 1, tau).gid, t1 - t0, r)
    return out


def compress_h2(tree, op, r: int, rank: int = 0, tol: float = 0.0, seed: int = 0,
                levels_only: bool = False, oversample: int = 10) -> H2Matrix:
    """Randomized compression of an H^2 matrix (Section 4.3, Algorithm 4.2)."""
    if rank <= 0 and tol <= 0.0:
        raise ValueError("a tolerance or a rank is needed")
    kcap = (min(r - oversample, rank) if rank > 0 else r - oversample) if tol > 0.0 else r
    rank_fixed = 0 if tol > 0.0 else rank
    H = H2Matrix(tree, {}, None, r)
    H.h2 = True
    H.bases, H.S = {}, {}
    H.Ut, H.Vt = {}, {}
    L = tree.L
    for l in range(2, L + 1):
        nc = len(tree.cuts[l])
        pairs = ot.admissible_pairs(tree, l)
        lf = LevelFactors(l, pairs, [tree.rng(l, a) for a, _ in pairs], [tree.rng(l, b) for _, b in pairs])
        coarse = sorted(H.levels)
        Uprev, Vprev = H.bases.get(l - 1, ({}, {}))
        Sin_prev, Sout_prev = H.S.get(l - 1, ({}, {}))
        # stage 1: Y = A Omega - A^(l-1) Omega on the box colouring
        bcol = og.color_boxes(tree, l) if pairs else None
        Y = None
        if bcol is not None and len(bcol.boxes):
            GO = gaussians(tree, l, SIDE_OMEGA, r, seed)
            Om = np.zeros((tree.n, bcol.n_colors * r))
            for c in range(bcol.n_colors):
                for b in bcol.active(c):
                    s_, e_ = tree.rng(l, b)
                    Om[s_:e_, c * r:(c + 1) * r] = GO[s_:e_]
            Y = op.apply(Om) - apply_levels(H, coarse, Om)
            H.matvec_cols += Om.shape[1]
        vcolor = {int(a): int(bcol.color[v]) for v, a in enumerate(bcol.boxes)} if Y is not None else {}
        aug_u = _aug_gauss(tree, l, Uprev, SIDE_AUG_U, r, seed)
        aug_v = _aug_gauss(tree, l, Vprev, SIDE_AUG_V, r, seed)
        U, Sin = {}, {}
        for a in range(nc):
            a0, a1 = tree.rng(l, a)
            P = np.zeros((a1 - a0, r))
            if a in vcolor:
                c = vcolor[a]
                P += Y[a0:a1, c * r:(c + 1) * r]
            tau = tree.cut_parent[l][a]
            if tau in Uprev and Uprev[tau].shape[1] > 0:
                t0 = tree.rng(l - 1, tau)[0]
                P += Uprev[tau][a0 - t0:a1 - t0] @ (Sin_prev[tau][:, None] * aug_u[tau])
            if a in vcolor or (tau in Uprev and Uprev[tau].shape[1] > 0):
                U[a], Sin[a] = svd_trunc(P, rank_fixed, tol, kcap)
        # stage 2: Z = A^* Psi - A^(l-1)* Psi with Psi(I_alpha) = U_alpha on the pair colouring
        T, W = [], {}
        if pairs:
            kmax = max(1, max(U[a].shape[1] for a, _ in pairs))
            col = og.color_level(tree, l)
            Psi = np.zeros((tree.n, col.n_colors * kmax))
            for c in range(col.n_colors):
                for b in col.active(c):
                    s_, e_ = tree.rng(l, b)
                    Psi[s_:e_, c * kmax:c * kmax + U[b].shape[1]] = U[b]
            Z = op.apply_t(Psi) - apply_levels(H, coarse, Psi, transpose=True)
            H.matvec_cols += Psi.shape[1]
            pindex = {pq: i for i, pq in enumerate(pairs)}
            mix = {}
            for i, (a, b) in enumerate(pairs):
                b0, b1 = lf.rng_b[i]
                ct = col.pair_color[pindex[(b, a)]]
                Tab = Z[b0:b1, ct * kmax:ct * kmax + U[a].shape[1]]
                T.append(Tab)
                if a not in mix:
                    a0, a1 = tree.rng(l, a)
                    mix[a] = U[a].T @ gaussian_block(seed, SIDE_MIX_H2, l, tree.box(l, a).gid, a1 - a0, r)
                acc = W.setdefault(b, np.zeros((b1 - b0, r)))
                acc += Tab @ mix[a]
            lf.coloring = col
            lf.box_coloring = bcol
        V, Sout = {}, {}
        for b in range(nc):
            b0, b1 = tree.rng(l, b)
            tau = tree.cut_parent[l][b]
            has_parent = tau in Vprev and Vprev[tau].shape[1] > 0
            if b not in W and not has_parent:
                continue
            Wb = W.get(b, np.zeros((b1 - b0, r))).copy()
            if has_parent:
                t0 = tree.rng(l - 1, tau)[0]
                Wb += Vprev[tau][b0 - t0:b1 - t0] @ (Sout_prev[tau][:, None] * aug_v[tau])
            V[b], Sout[b] = svd_trunc(Wb, rank_fixed, tol, kcap)
        for i, (a, b) in enumerate(pairs):
            lf.U.append(U[a])
            lf.B.append(T[i].T @ V[b])
            lf.V.append(V[b])
        H.bases[l] = (U, V)
        H.S[l] = (Sin, Sout)
        H.levels[l] = lf
        # nest cut l-1 through its children's long bases (eq. nested_basis);
        # the coarser cuts' bases are the ones the nested chain now defines
        if l > 2:
            H.Ut[l - 1] = _nest(tree, l, Uprev, U)
            H.Vt[l - 1] = _nest(tree, l, Vprev, V)
            for j in range(l - 1, 1, -1):
                Uj, Vj = H.bases[j]
                Uj.update(_expand(tree, j + 1, H.bases[j + 1][0], H.Ut[j]))
                Vj.update(_expand(tree, j + 1, H.bases[j + 1][1], H.Vt[j]))
                lj = H.levels[j]
                lj.U = [Uj[a] for a, _ in lj.pairs]
                lj.V = [Vj[b] for _, b in lj.pairs]
    H.long = H.bases.get(L, ({}, {}))
    if levels_only:
        return H
    H.leaf = extract_leaf(H, op)
    return H


def apply_h2(H: H2Matrix, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """y = A~ x by Algorithm 4.3 with l = L (the whole admissible part) plus the
    leaf neighbour blocks: outgoing expansions from the long bases of cut L,
    the upward pass through the short bases, the cores at every level, the
    downward pass, and the long bases of cut L again."""
    tree = H.tree
    X = np.asarray(X, np.float64)
    out = np.zeros_like(X)
    L = tree.L
    if L >= 2 and H.levels:
        Uin, Vout = H.long
        Uts, Vts = H.Ut, H.Vt
        if transpose:
            Uin, Vout = Vout, Uin
            Uts, Vts = Vts, Uts
        # outgoing expansions of cut L, then upward through the short bases
        qh = {L: {}}
        for b, Vb in Vout.items():
            b0, b1 = tree.rng(L, b)
            qh[L][b] = Vb.T @ X[b0:b1]
        for l in range(L - 1, 1, -1):
            qh[l] = {}
            for tau, blocks in Vts.get(l, {}).items():
                acc = None
                for a, Vt in blocks:
                    if a in qh[l + 1]:
                        term = Vt.T @ qh[l + 1][a]
                        acc = term if acc is None else acc + term
                qh[l][tau] = acc if acc is not None else np.zeros((blocks[0][1].shape[1], X.shape[1]))
        # incoming expansions: cores at every level, downward through the short bases
        uh = {}
        for l in range(2, L + 1):
            uh[l] = {}
            lf = H.levels.get(l)
            if lf is not None:
                for (a, b), B in zip(lf.pairs, lf.B):
                    if transpose:
                        a, b, B = b, a, B.T
                    if B.size == 0:
                        continue
                    term = B @ qh[l][b]
                    uh[l][a] = uh[l][a] + term if a in uh[l] else term
            if l > 2:
                for tau, blocks in Uts.get(l - 1, {}).items():
                    if tau not in uh[l - 1]:
                        continue
                    for a, Ut in blocks:
                        term = Ut @ uh[l - 1][tau]
                        uh[l][a] = uh[l][a] + term if a in uh[l] else term
        for a, ua in uh[L].items():
            a0, a1 = tree.rng(L, a)
            out[a0:a1] += Uin[a] @ ua
    if H.leaf is not None:
        for (a0, a1), (b0, b1), D in zip(H.leaf.rng_a, H.leaf.rng_b, H.leaf.D):
            if not transpose:
                out[a0:a1] += D @ X[b0:b1]
            else:
                out[b0:b1] += D.T @ X[a0:a1]
    return out
