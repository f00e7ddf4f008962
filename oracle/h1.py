"""Oracle: randomized H^1 compression by peeling with graph-coloured test matrices.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Algorithm 4.1 (randomized compression of an H^1 matrix) level by level,
with the per-block factorisation of Algorithm 2.1 (two randomized samples), the
leaf extraction of Section 4.1.3, the apply of the compressed operator and the
relative-error estimate of Section 5.  All arithmetic is FP64 NumPy.  All index
sets refer to the Morton-permuted point order of oracle.tree.

Readings of points where the paper is silent, garbled or inconsistent:
  * Peel (Alg. 4.1 writes A^(l); Sec. 4.1.2 subtracts A^(2) at level 3): the
    samples of level l are Y = A Omega - A^(l-1) Omega, with A^(l-1) the sum of
    the factors of all levels 2..l-1; the leaf step subtracts levels 2..L.
  * qr(Y, k) (Sec. 2.4 "partial QR"): column-pivoted Householder QR with the
    column norms recomputed exactly at every step (so any two implementations
    pick the same pivots unless two norms tie to rounding); with a fixed rank k
    the first k columns of Q are kept; with a tolerance tau, k is the number of
    pivots with |R_jj| > tau |R_11|.  Always k <= min(|I_alpha|, |I_beta|) (the
    block's rank cannot exceed it) and, with a tolerance, k <= r - p so that the
    core's r x k solves keep p rows of oversampling (Sec. 2.5: p = 10 is often
    good).  Columns of Q are signed so that R_jj >= 0.
  * The pseudo-inverses of the core are least-squares solves through a
    Householder QR of the r x k factor (full column rank).
  * Core (eq. solveforb drops the transposes; Alg. 2.1 fixes them):
      B = (G_alpha^T U)^+ (G_alpha^T Y(I_alpha, c)) (V^T G_beta)^+,
    with G_alpha the Psi-side block of alpha and G_beta the Omega-side block of
    beta; A(I_alpha, I_beta) ~ U B V^T.
  * V of pair (alpha, beta) comes from Z(I_beta, c') where c' is the colour of
    the pair (beta, alpha): the rank structure is symmetric, so one colouring
    serves both Omega and Psi (Alg. 4.1 allows reusing the test matrices).
  * Leaf test matrices have m_max columns per colour, m_max = the largest leaf.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import graph as og
from . import tree as ot
from .philox import gaussian_block

SIDE_OMEGA, SIDE_PSI, SIDE_START, SIDE_MIX = 0, 1, 2, 3


# ----------------------------------------------------------------------------
# Black-box operators (Section 1: the user can apply A and A^* to tall thin
# matrices).  All act in the permuted point order.
# ----------------------------------------------------------------------------

def kernel_eval(kind: int, xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """K(x, y) for all pairs: log r, 1/(4 pi r), 1/r (zero where r = 0), exp(-r)."""
    diff = xa[:, None, :] - xb[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    pos = r > 0.0
    rs = np.where(pos, r, 1.0)
    if kind == 1:
        return np.where(pos, np.log(rs), 0.0)
    if kind == 2:
        return np.where(pos, 1.0 / (4.0 * math.pi * rs), 0.0)
    if kind == 3:
        return np.where(pos, 1.0 / rs, 0.0)
    if kind == 4:
        return np.exp(-r)
    raise ValueError(kind)


class KernelOp:
    """A(i, j) = K(x_i, x_j) evaluated on the fly (the matrix is symmetric)."""

    def __init__(self, x_sorted: np.ndarray, kind: int, chunk_elems: int = 1 << 23):
        self.x, self.kind, self.chunk = np.asarray(x_sorted, np.float64), kind, chunk_elems
        self.n = self.x.shape[0]

    def apply(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, np.float64)
        nz = np.flatnonzero(np.any(X != 0.0, axis=1))     # skip zero rows of X
        Y = np.zeros((self.n, X.shape[1]))
        if nz.size == 0:
            return Y
        rows = max(1, self.chunk // nz.size)
        for s in range(0, self.n, rows):
            e = min(self.n, s + rows)
            Y[s:e] = kernel_eval(self.kind, self.x[s:e], self.x[nz]) @ X[nz]
        return Y

    def apply_t(self, X):
        return self.apply(X)

    def rows(self, idx: np.ndarray, X: np.ndarray) -> np.ndarray:
        """(A X)(idx, :) only: used for sampled checks at full size."""
        nz = np.flatnonzero(np.any(X != 0.0, axis=1))
        out = np.zeros((len(idx), X.shape[1]))
        step = max(1, self.chunk // max(nz.size, 1))
        for s in range(0, len(idx), step):
            out[s:s + step] = kernel_eval(self.kind, self.x[idx[s:s + step]], self.x[nz]) @ X[nz]
        return out

    def dense(self) -> np.ndarray:
        return kernel_eval(self.kind, self.x, self.x)


class DenseOp:
    """A stored as a dense FP64 matrix (permuted order)."""

    def __init__(self, a_sorted: np.ndarray):
        self.a = np.asarray(a_sorted, np.float64)
        self.n = self.a.shape[0]

    def apply(self, X):
        return self.a @ X

    def apply_t(self, X):
        return self.a.T @ X

    def dense(self):
        return self.a


# ----------------------------------------------------------------------------
# Factor storage
# ----------------------------------------------------------------------------

@dataclass
class LevelFactors:
    level: int
    pairs: list                 # (alpha, beta) cut indices
    rng_a: list                 # (start, end) of I_alpha
    rng_b: list                 # (start, end) of I_beta
    U: list = field(default_factory=list)
    B: list = field(default_factory=list)
    V: list = field(default_factory=list)
    coloring: object = None
    Y: np.ndarray | None = None  # peeled samples (kept for parity checks)
    Z: np.ndarray | None = None


@dataclass
class LeafBlocks:
    pairs: list
    rng_a: list
    rng_b: list
    D: list
    coloring: object
    m_max: int
    Y: np.ndarray | None = None


@dataclass
class H1Matrix:
    tree: object
    levels: dict                # l -> LevelFactors
    leaf: LeafBlocks | None
    r: int
    matvec_cols: int = 0        # columns of Omega and Psi applied to A or A^*

    def floats(self) -> int:
        s = 0
        bases = getattr(self, "bases", None)
        for l, lf in self.levels.items():
            if bases and l in bases:  # uniform: one U and one V per box, a B per pair
                U, V = bases[l]
                s += sum(u.size for u in U.values()) + sum(v.size for v in V.values()) + sum(b.size for b in lf.B)
                continue
            s += sum(u.size for u in lf.U) + sum(b.size for b in lf.B) + sum(v.size for v in lf.V)
        if self.leaf is not None:
            s += sum(d.size for d in self.leaf.D)
        return s


def apply_levels(H: H1Matrix, levels, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """A^(l) X restricted to the given admissible levels: sum of U B V^T blocks
    (Section 4.1.2, level-truncated matrix)."""
    out = np.zeros_like(X, dtype=np.float64)
    for j in levels:
        lf = H.levels[j]
        for (a0, a1), (b0, b1), U, B, V in zip(lf.rng_a, lf.rng_b, lf.U, lf.B, lf.V):
            if not transpose:
                out[a0:a1] += U @ (B @ (V.T @ X[b0:b1]))
            else:
                out[b0:b1] += V @ (B.T @ (U.T @ X[a0:a1]))
    return out


def apply_h1(H: H1Matrix, X: np.ndarray, transpose: bool = False) -> np.ndarray:
    """y = A~ x: all admissible blocks plus the leaf neighbour blocks (permuted order)."""
    X = np.asarray(X, np.float64)
    out = apply_levels(H, sorted(H.levels), X, transpose)
    if H.leaf is not None:
        for (a0, a1), (b0, b1), D in zip(H.leaf.rng_a, H.leaf.rng_b, H.leaf.D):
            if not transpose:
                out[a0:a1] += D @ X[b0:b1]
            else:
                out[b0:b1] += D.T @ X[a0:a1]
    return out


# ----------------------------------------------------------------------------
# Per-block steps
# ----------------------------------------------------------------------------

def pivoted_qr(P: np.ndarray, kmax: int, rank: int, tol: float):
    """Column-pivoted Householder QR (Businger-Golub), steps in order: at step s
    the remaining column of largest norm (norms recomputed exactly over rows
    s.., lowest index on ties) is swapped to position s, and one Householder
    reflection zeroes it below the diagonal.  Stops after `rank` steps (fixed
    rank) or before the first pivot whose norm is <= tol times the first
    pivot's (tolerance), and never after kmax steps.
    Returns (Q_k with R_jj >= 0, k)."""
    A = np.array(P, dtype=np.float64, copy=True)
    m, n = A.shape
    vs, taus, betas = [], [], []
    n0 = 0.0
    k = 0
    for s in range(kmax):
        norms = np.sum(A[s:, s:] ** 2, axis=0)
        piv = s + int(np.argmax(norms))               # first maximum
        nv = float(np.sqrt(norms[piv - s]))
        if s == 0:
            n0 = nv
        if rank > 0:
            if s >= rank:
                break
        elif not (n0 > 0.0) or not (nv > tol * n0):
            break
        A[:, [s, piv]] = A[:, [piv, s]]
        x = A[s:, s].copy()
        nx = float(np.sqrt(np.sum(x * x)))
        v = x.copy()
        if nx == 0.0:
            tau, beta = 0.0, 0.0
            v[:] = 0.0
            v[0] = 1.0
        else:
            beta = -np.copysign(nx, x[0])
            tau = (beta - x[0]) / beta
            v[1:] = x[1:] / (x[0] - beta)
            v[0] = 1.0
        # apply H = I - tau v v^T to the trailing block
        w = v @ A[s:, s:]
        A[s:, s:] -= tau * np.outer(v, w)
        vs.append(v)
        taus.append(tau)
        betas.append(beta)
        k = s + 1
    # Q_k = H_0 ... H_{k-1} [I_k; 0], columns signed so that R_jj >= 0
    Q = np.zeros((m, k))
    Q[:k, :k] = np.eye(k)
    for s in range(k - 1, -1, -1):
        v, tau = vs[s], taus[s]
        Q[s:, :] -= tau * np.outer(v, v @ Q[s:, :])
    for j in range(k):
        if betas[j] < 0.0:
            Q[:, j] = -Q[:, j]
    return Q, k


def qr_trunc(P: np.ndarray, rank: int, tol: float, cap: int) -> np.ndarray:
    """qr(P, k) of Section 2.4 (reading in the module docstring); k <= cap."""
    m, n = P.shape
    kmax = min(m, n, cap)
    if kmax == 0:
        return np.zeros((m, 0))
    Q, _ = pivoted_qr(P, kmax, rank, tol)
    return Q


def core(Ga: np.ndarray, P: np.ndarray, Gb: np.ndarray, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """B = (Ga^T U)^+ (Ga^T P) (V^T Gb)^+  (Alg. 2.1, last step)."""
    M = Ga.T @ P
    S1 = Ga.T @ U
    S2 = Gb.T @ V
    if U.shape[1] == 0 or V.shape[1] == 0:
        return np.zeros((U.shape[1], V.shape[1]))
    T = lstsq_qr(S1, M)            # (Ga^T U)^+ M,            k_U x r
    return lstsq_qr(S2, T.T).T     # T (V^T Gb)^+ = (S2^+ T^T)^T, k_U x k_V


def lstsq_qr(S: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Least-squares solution of S X = R for S of full column rank, through a
    Householder QR of S and a triangular solve (S^+ R)."""
    Q, Rs = np.linalg.qr(S)
    return scipy.linalg.solve_triangular(Rs, Q.T @ R, lower=False)


def gaussians(tree, l: int, side: int, r: int, seed: int) -> np.ndarray:
    """G_beta for every box beta of cut l, stacked in permuted order (N x r)."""
    G = np.zeros((tree.n, r))
    for i in range(len(tree.cuts[l])):
        b = tree.box(l, i)
        G[b.start:b.end] = gaussian_block(seed, side, l, b.gid, b.end - b.start, r)
    return G


def test_matrix(tree, l: int, col: og.Coloring, G: np.ndarray, r: int) -> np.ndarray:
    """Omega_l: colour c has G_beta on the rows of every beta active in c (eq. neartestmatrices)."""
    Om = np.zeros((tree.n, col.n_colors * r))
    for c in range(col.n_colors):
        for b in col.active(c):
            s, e = tree.rng(l, b)
            Om[s:e, c * r:(c + 1) * r] = G[s:e]
    return Om


def sample_rows(op, tree, l: int, col: og.Coloring, G: np.ndarray, r: int, rows: np.ndarray,
                colors: np.ndarray) -> np.ndarray:
    """Selected entries of the raw sample Y_l = A Omega_l without forming Omega_l
    (used for sampled checks at full size): row k of the result is
    Y_l(rows[k], colors[k] r : (colors[k] + 1) r).  Colour c of Omega_l holds
    G_beta on the rows of every box beta active in c and zeros elsewhere
    (eq. neartestmatrices), so the product needs only those rows of A."""
    rows = np.asarray(rows, dtype=np.int64)
    colors = np.asarray(colors, dtype=np.int64)
    out = np.zeros((len(rows), r))
    for c in np.unique(colors):
        X = np.zeros((tree.n, r))
        for b in col.active(int(c)):
            s, e = tree.rng(l, b)
            X[s:e] = G[s:e]
        k = np.flatnonzero(colors == c)
        out[k] = op.rows(rows[k], X)
    return out


# ----------------------------------------------------------------------------
# Algorithm 4.1
# ----------------------------------------------------------------------------

def compress(tree, op, r: int, rank: int = 0, tol: float = 0.0, seed: int = 0,
             keep_samples: bool = False, levels_only: bool = False, oversample: int = 10) -> H1Matrix:
    """Randomized compression of an H^1 matrix (Algorithm 4.1)."""
    if (rank > 0) == (tol > 0.0):
        raise ValueError("exactly one of rank > 0 or tol > 0")
    kcap = r if rank > 0 else r - oversample
    H = H1Matrix(tree, {}, None, r)
    L = tree.L
    for l in range(2, L + 1):
        pairs = ot.admissible_pairs(tree, l)
        lf = LevelFactors(l, pairs, [tree.rng(l, a) for a, _ in pairs],
                          [tree.rng(l, b) for _, b in pairs])
        if not pairs:
            H.levels[l] = lf
            continue
        col = og.color_level(tree, l)
        lf.coloring = col
        GO = gaussians(tree, l, SIDE_OMEGA, r, seed)
        GP = gaussians(tree, l, SIDE_PSI, r, seed)
        Om = test_matrix(tree, l, col, GO, r)
        Ps = test_matrix(tree, l, col, GP, r)
        coarse = sorted(H.levels)
        Y = op.apply(Om) - apply_levels(H, coarse, Om)
        Z = op.apply_t(Ps) - apply_levels(H, coarse, Ps, transpose=True)
        H.matvec_cols += Om.shape[1] + Ps.shape[1]
        pcol = col.pair_color
        pindex = {pq: i for i, pq in enumerate(pairs)}
        for i, (a, b) in enumerate(pairs):
            (a0, a1), (b0, b1) = lf.rng_a[i], lf.rng_b[i]
            c = pcol[i]
            ct = pcol[pindex[(b, a)]]
            P = Y[a0:a1, c * r:(c + 1) * r]
            cap = min(kcap, a1 - a0, b1 - b0)    # rank(A(I_a, I_b)) <= min(|I_a|, |I_b|)
            U = qr_trunc(P, rank, tol, cap)
            V = qr_trunc(Z[b0:b1, ct * r:(ct + 1) * r], rank, tol, cap)
            B = core(GP[a0:a1], P, GO[b0:b1], U, V)
            lf.U.append(U)
            lf.B.append(B)
            lf.V.append(V)
        if keep_samples:
            lf.Y, lf.Z = Y, Z
        H.levels[l] = lf
    if levels_only:
        return H
    H.leaf = extract_leaf(H, op, keep_samples)
    return H


def compress_uniform(tree, op, r: int, rank: int = 0, tol: float = 0.0, seed: int = 0,
                     levels_only: bool = False, oversample: int = 10) -> H1Matrix:
    """Randomized compression of a uniform H^1 matrix (Section 4.2; Algorithm
    2.2's two stages applied to every box at once), level by level:

      1. colour the box constraint sets (graph.color_boxes: G_beta on int(alpha),
         zeros on near(alpha)); Y = A Omega - A^(l-1) Omega with Gaussian Omega;
         U_alpha = qr(Y(I_alpha, colour of alpha)): Algorithm 2.2 orthonormalizes
         the whole sample, all r = k + p columns (at most |I_alpha| and the
         sampled block's width), with no truncation;
      2. colour the pair constraint sets (the non-uniform graph) and fill the
         test matrices with the bases instead of Gaussians: Psi(I_alpha) =
         U_alpha; Z = A^* Psi - A^(l-1)* Psi, so the tile of the pair (beta,
         alpha) gives T_ab = Z(I_beta, :k_alpha) = A_ab^* U_alpha;
      3. V_beta = qr(sum over alpha in int(beta) of T_ab M_a, k), B_ab =
         T_ab^T V_beta.  Section 4.2 sums the T_ab themselves, which spans the
         row space of A(union of I_alpha, I_beta) when every U_alpha has r
         columns; on an adaptive tree a box smaller than r has a narrower
         basis and the plain sum can lose dimensions.  Reading: each term is
         first mixed by its own Gaussian k_alpha x r matrix M_a (Philox, side
         SIDE_MIX, keyed by the box alpha), a randomized sketch of the
         concatenation [T_a1 ... T_am] with r columns.  The truncation (fixed
         rank or tolerance, qr(Y, k) of Section 2.4) applies here, with the p
         columns of oversampling.

    A_ab ~ U_alpha B_ab V_beta^T.  The bases are shared by all pairs of a box;
    the per-pair lists of the result hold references to them, so apply_levels
    and the peel work unchanged.  Rank caps: k <= min(|I_beta|, rows of the
    sampled block) always, and k <= r - p with a tolerance (k <= rank too when
    both are given).  The leaf blocks are extracted as in Section 4.1.3."""
    if rank <= 0 and tol <= 0.0:
        raise ValueError("a tolerance or a rank is needed")
    kcap = (min(r - oversample, rank) if rank > 0 else r - oversample) if tol > 0.0 else r
    rank_fixed = 0 if tol > 0.0 else rank
    H = H1Matrix(tree, {}, None, r)
    H.uniform = True
    H.bases = {}
    L = tree.L
    for l in range(2, L + 1):
        pairs = ot.admissible_pairs(tree, l)
        lf = LevelFactors(l, pairs, [tree.rng(l, a) for a, _ in pairs], [tree.rng(l, b) for _, b in pairs])
        if not pairs:
            H.levels[l] = lf
            continue
        coarse = sorted(H.levels)
        # stage 1: column bases of every box
        bcol = og.color_boxes(tree, l)
        GO = gaussians(tree, l, SIDE_OMEGA, r, seed)
        Om = np.zeros((tree.n, bcol.n_colors * r))
        for c in range(bcol.n_colors):
            for b in bcol.active(c):
                s_, e_ = tree.rng(l, b)
                Om[s_:e_, c * r:(c + 1) * r] = GO[s_:e_]
        Y = op.apply(Om) - apply_levels(H, coarse, Om)
        H.matvec_cols += Om.shape[1]
        U = {}
        for v, a in enumerate(bcol.boxes):
            a = int(a)
            a0, a1 = tree.rng(l, a)
            c = int(bcol.color[v])
            width = sum(tree.rng(l, b)[1] - tree.rng(l, b)[0] for b in bcol.inter[v])
            kU = min(r, a1 - a0, width)
            U[a] = qr_trunc(Y[a0:a1, c * r:(c + 1) * r], kU, 0.0, kU)
        kmax = max(1, max(u.shape[1] for u in U.values()))
        # stage 2: A_ab^* U_alpha for every pair, from the pair colouring
        col = og.color_level(tree, l)
        Psi = np.zeros((tree.n, col.n_colors * kmax))
        for c in range(col.n_colors):
            for b in col.active(c):
                s_, e_ = tree.rng(l, b)
                Psi[s_:e_, c * kmax:c * kmax + U[b].shape[1]] = U[b]
        Z = op.apply_t(Psi) - apply_levels(H, coarse, Psi, transpose=True)
        H.matvec_cols += Psi.shape[1]
        pcol = col.pair_color
        pindex = {pq: i for i, pq in enumerate(pairs)}
        T = []
        W = {}
        mix = {}
        for i, (a, b) in enumerate(pairs):
            b0, b1 = lf.rng_b[i]
            ct = pcol[pindex[(b, a)]]             # Psi of the pair (b, a) holds U_a on I_a
            Tab = Z[b0:b1, ct * kmax:ct * kmax + U[a].shape[1]]
            T.append(Tab)
            if a not in mix:
                mix[a] = gaussian_block(seed, SIDE_MIX, l, tree.box(l, a).gid, U[a].shape[1], r)
            acc = W.setdefault(b, np.zeros((b1 - b0, r)))
            acc += Tab @ mix[a]
        V = {}
        for b, Wb in W.items():
            b0, b1 = tree.rng(l, b)
            rows = sum(tree.rng(l, a)[1] - tree.rng(l, a)[0] for a in tree.inter[l][b])
            V[b] = qr_trunc(Wb, rank_fixed, tol, min(kcap, b1 - b0, rows))
        for i, (a, b) in enumerate(pairs):
            lf.U.append(U[a])
            lf.B.append(T[i].T @ V[b])
            lf.V.append(V[b])
        lf.coloring = col
        lf.box_coloring = bcol
        H.bases[l] = (U, V)
        H.levels[l] = lf
    if levels_only:
        return H
    H.leaf = extract_leaf(H, op)
    return H


def extract_leaf(H: H1Matrix, op, keep_samples: bool = False) -> LeafBlocks:
    """Section 4.1.3: identity test matrices recover the leaf neighbour blocks."""
    tree = H.tree
    L = tree.L
    pairs = ot.near_pairs(tree, L)
    col = og.color_leaf(tree)
    m_max = max(tree.box(L, i).end - tree.box(L, i).start for i in range(len(tree.cuts[L])))
    Om = np.zeros((tree.n, col.n_colors * m_max))
    for c in range(col.n_colors):
        for b in col.active(c):
            s, e = tree.rng(L, b)
            Om[s:e, c * m_max:c * m_max + (e - s)] = np.eye(e - s)
    Y = op.apply(Om) - apply_levels(H, sorted(H.levels), Om)
    H.matvec_cols += Om.shape[1]
    pcol = col.pair_color
    rng_a = [tree.rng(L, a) for a, _ in pairs]
    rng_b = [tree.rng(L, b) for _, b in pairs]
    D = []
    for i, (a, b) in enumerate(pairs):
        (a0, a1), (b0, b1) = rng_a[i], rng_b[i]
        c = pcol[i]
        D.append(Y[a0:a1, c * m_max:c * m_max + (b1 - b0)].copy())
    return LeafBlocks(pairs, rng_a, rng_b, D, col, m_max, Y if keep_samples else None)


# ----------------------------------------------------------------------------
# Accuracy (Section 5): E = ||A_c - A|| / ||A|| by 20 power iterations
# ----------------------------------------------------------------------------

def power_norm(apply, apply_t, n: int, iters: int, seed: int) -> float:
    """Spectral norm by the power method on M^T M from a Philox Gaussian start."""
    v = gaussian_block(seed, SIDE_START, 0, 0, n, 1)[:, 0]
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = apply_t(apply(v[:, None]))[:, 0]
        lam = np.linalg.norm(w)
        if lam == 0.0:
            return 0.0
        v = w / lam
    return math.sqrt(lam)


def relative_error(H: H1Matrix, op, iters: int = 20, seed: int = 1) -> float:
    n = H.tree.n
    diff = lambda X: apply_h1(H, X) - op.apply(X)
    diff_t = lambda X: apply_h1(H, X, transpose=True) - op.apply_t(X)
    num = power_norm(diff, diff_t, n, iters, seed)
    den = power_norm(op.apply, op.apply_t, n, iters, seed)
    return num / den if den > 0 else 0.0
