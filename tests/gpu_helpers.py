"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and decode its exports into the oracle's shapes."""
import numpy as np

import hm_workloads as W


def hm():
    import paper_2205_03406_gb300 as m
    return m


def settings_for(w: W.Workload, precision: int = 0, keep: bool = True, fmt: int = 0):
    m = hm()
    return m.Settings(d=w.d, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, rank=w.rank, tol=w.tol,
                      uniform_depth=w.uniform_depth, precision=precision, keep_samples=keep, seed=w.seed,
                      format=fmt)


def op_for(w: W.Workload, dense_keep: list):
    """Built-in operator of a workload: stored dense matrix or kernel on the fly."""
    import torch
    m = hm()
    if w.dense is not None:
        # the library reads column-major: A's column-major storage is A.T row-major
        a = torch.from_numpy(np.ascontiguousarray(w.dense.T)).cuda()
        dense_keep.append(a)
        return m.dense_op(a)
    return m.kernel_op(w.kernel)


def run_gpu(w: W.Workload, precision: int = 0, keep: bool = True, compress: bool = True, fmt: int = 0):
    import torch
    m = hm()
    comp = m.Compressor(settings_for(w, precision, keep, fmt))
    comp.tree_build(torch.from_numpy(w.points).cuda())
    keepalive = []
    op = op_for(w, keepalive)
    info = comp.compress(op) if compress else None
    comp._op, comp._keep = op, keepalive
    return comp, info


def i32(b):
    return np.frombuffer(b, dtype=np.int32)


def f64(b):
    return np.frombuffer(b, dtype=np.float64)


def csr(b, nc):
    a = i32(b)
    ptr, idx = a[:nc + 1], a[nc + 1:]
    return [idx[ptr[i]:ptr[i + 1]].tolist() for i in range(nc)]


def samples(comp, what, level, n, chi, cols):
    """[chi][n][cols] colour-major -> N x (chi cols) like the oracle."""
    y = f64(comp.export(what, level)).reshape(chi, n, cols)
    return y.transpose(1, 0, 2).reshape(n, chi * cols)


def tile_mask(t, l, col, r):
    """Entries of the level-l samples that Algorithm 4.1 reads: colour c's
    columns on the rows I_alpha of every pair (alpha, beta) of colour c (the
    sample tiles Y(I_alpha, c), Section 4.1.2).  The tensor-core sampler
    computes only these rows; the rest of the sample buffer is unspecified."""
    from oracle import tree as ot
    mask = np.zeros((t.n, col.n_colors * r), dtype=bool)
    for (a, _), c in zip(ot.admissible_pairs(t, l), col.pair_color):
        s, e = t.rng(l, a)
        mask[s:e, c * r:(c + 1) * r] = True
    return mask


def factors(comp, level, rng_a, rng_b):
    """Per-pair (U, B, V) from the level's arenas."""
    m = hm()
    ranks = i32(comp.export(m.HM_X_PAIR_RANKS, level)).reshape(-1, 2)
    offs = np.frombuffer(comp.export(m.HM_X_FACTOR_OFFS, level), dtype=np.int64).reshape(-1, 3)
    arena = f64(comp.export(m.HM_X_FACTORS, level))
    # arena lengths: the largest block end (uniform H^1 shares one block among a box's pairs)
    nU = max(int(offs[p, 0] + (a1 - a0) * ranks[p, 0]) for p, (a0, a1) in enumerate(rng_a))
    nV = max(int(offs[p, 1] + (b1 - b0) * ranks[p, 1]) for p, (b0, b1) in enumerate(rng_b))
    U_ar, V_ar, B_ar = arena[:nU], arena[nU:nU + nV], arena[nU + nV:]
    out = []
    for p, ((a0, a1), (b0, b1)) in enumerate(zip(rng_a, rng_b)):
        ku, kv = ranks[p]
        U = U_ar[offs[p, 0]:offs[p, 0] + (a1 - a0) * ku].reshape(a1 - a0, ku)
        V = V_ar[offs[p, 1]:offs[p, 1] + (b1 - b0) * kv].reshape(b1 - b0, kv)
        B = B_ar[offs[p, 2]:offs[p, 2] + ku * kv].reshape(ku, kv)
        out.append((U, B, V))
    return ranks, out


def oracle_op(w: W.Workload, t):
    from oracle import h1
    if w.dense is not None:
        return h1.DenseOp(w.dense[t.perm][:, t.perm])
    return h1.KernelOp(w.points[t.perm], w.kernel)


def check_structure(comp, t):
    """Permutation, boxes of every level, cuts, neighbour and interaction lists:
    bit-exact against the oracle's tree."""
    m = hm()
    assert np.array_equal(i32(comp.export(m.HM_X_PERM)), t.perm)
    assert comp.info().L == t.L
    for l in range(t.L + 1):
        bx = i32(comp.export(m.HM_X_LEVEL_BOXES, l)).reshape(-1, 8)
        ref = np.array([[b.start, b.end, *(list(b.anchor) + [0] * (3 - t.d)), b.parent, int(b.leaf), b.gid]
                        for b in t.levels[l]])
        assert np.array_equal(bx, ref), f"level {l} boxes"
        cut = i32(comp.export(m.HM_X_CUT, l)).reshape(-1, 2)
        assert np.array_equal(cut, np.array(t.cuts[l])), f"cut {l}"
        nc = len(t.cuts[l])
        assert csr(comp.export(m.HM_X_NEAR, l), nc) == t.near[l], f"near {l}"
        assert csr(comp.export(m.HM_X_INTER, l), nc) == t.inter[l], f"inter {l}"
