// Test matrices and the black-box products Y = A Omega, Z = A^* Psi
// (Algorithm 4.1 sampling steps; eq. h1constraints, eq. neartestmatrices).
//
//  K6  Philox4x32-10 Gaussians: entry (i, j) of G_beta (side s, cut level l)
//      uses key = seed and counter (j, i, gid(beta), s << 8 | l); two 52-bit
//      uniforms and Box-Muller give one standard normal.  Keyed by box, so
//      G_beta is the same in every colour where beta is active.
//  K7  built-in operators, FP64: for colour c, Y(:, c) = sum over the active
//      boxes beta of K(:, I_beta) G_beta.  Zero tiles of Omega are never
//      touched; the kernel matrix is evaluated on the fly (or gathered from a
//      stored dense matrix).  For a symmetric kernel A^* = A, so one sweep
//      produces Y and Z from the same kernel tiles.
//  Leaf: Omega(I_beta, c m + t) = delta(t, row), so Y(i, c m + t) is the sum of
//      K(i, start_beta + t) over the active boxes beta.
//
// Sample layout: Y[c][i][j] = Y(i, c * cols + j), i in sorted (Morton) order.
#include "ctx.cuh"
#include "philox.cuh"

#include <cmath>

namespace hm {

__global__ void k_gauss(int64_t n, int r, const int *pt2ent, const int *ent, int level, unsigned long long seed,
                        double *GO, double *GP) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * r) return;
    const int64_t i = t / r;
    const int j = (int)(t - i * r);
    const int *e = ent + (int64_t)pt2ent[i] * ENT_FIELDS;
    const int row = (int)i - e[3];
    GO[t] = gauss(seed, 0, level, e[2], row, j);
    GP[t] = gauss(seed, 1, level, e[2], row, j);
}

Err make_gaussians(hm_ctx *c, int level) {
    const int r = c->cfg.r;
    const int64_t n = c->n;
    HM_TRY(ensure(c->GO, n * r * sizeof(double)));
    HM_TRY(ensure(c->GP, n * r * sizeof(double)));
    const Cut &cu = c->cuts[level];
    k_gauss<<<ceil_div(n * r, 256), 256, 0, c->st>>>(n, r, cu.pt2ent.as<int>(), cu.ent.as<int>(), level,
                                                     (unsigned long long)c->cfg.seed, c->GO.as<double>(),
                                                     c->GP.as<double>()); ::hm::count_launch();
    HM_LAUNCH("gauss");
    c->gauss_level = level;
    return ok();
}

// ---------------------------------------------------------------------------
// kernel functions (FP64)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double kfun64(int kind, double r2) {
    if (kind == HM_K_EXP) return exp(-sqrt(r2));
    if (r2 == 0.0) return 0.0;
    if (kind == HM_K_LOG) return 0.5 * log(r2);
    if (kind == HM_K_LAPLACE3D) return rsqrt(r2) * 0.079577471545947667884;  // 1/(4 pi)
    return rsqrt(r2);                                                       // HM_K_INVR
}

struct OpDev {
    int kind;             // HM_OP_KERNEL or HM_OP_DENSE
    int kernel;           // HM_K_*
    const double *xs;     // sorted points [n][3]
    const double *dense;  // original-order column-major
    const int *perm;
    int64_t n;
};

// entry (i, j) of A (trans = 0) or A^* (trans = 1), sorted indices
__device__ __forceinline__ double op_entry(const OpDev &o, int64_t i, int64_t j, int trans) {
    if (o.kind == HM_OP_DENSE) {
        const int64_t a = o.perm[trans ? j : i], b = o.perm[trans ? i : j];
        return o.dense[a + b * o.n];
    }
    const double dx = o.xs[i * 3] - o.xs[j * 3], dy = o.xs[i * 3 + 1] - o.xs[j * 3 + 1],
                 dz = o.xs[i * 3 + 2] - o.xs[j * 3 + 2];
    return kfun64(o.kernel, dx * dx + dy * dy + dz * dz);
}

// ---------------------------------------------------------------------------
// K7 FP64: OUT[c][i][0:NC] = sum_{j in rows(c)} A(i, j) G[j][0:NC]
//   grid (row tiles of 64, colours); 256 threads; thread = (row, column phase)
// ---------------------------------------------------------------------------

constexpr int TR = 64, TK = 16;

template <int MAXQ>
__global__ void __launch_bounds__(256) k_sample64(OpDev o, int trans, const int64_t *rows_ptr, const int *rows,
                                                  const double *G, int NC, double *out0, double *out1, int split) {
    __shared__ double Ks[TR][TK + 1];
    __shared__ double Gs[TK][4 * MAXQ];
    __shared__ int jr[TK];
    const int c = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * TR;
    const int tid = threadIdx.x, ri = tid >> 2, ph = tid & 3;
    const int64_t n = o.n;
    double acc[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) acc[q] = 0.0;
    const int64_t b0 = rows_ptr ? rows_ptr[c] : 0, b1 = rows_ptr ? rows_ptr[c + 1] : n;
    for (int64_t kb = b0; kb < b1; kb += TK) {
        const int kn = (int)((b1 - kb) < TK ? (b1 - kb) : TK);
        if (tid < TK) jr[tid] = (tid < kn) ? (rows ? rows[kb + tid] : (int)(kb + tid)) : -1;
        __syncthreads();
        for (int e = tid; e < TR * TK; e += 256) {
            const int a = e / TK, b = e % TK;
            const int64_t i = i0 + a;
            const int j = jr[b];
            Ks[a][b] = (i < n && j >= 0) ? op_entry(o, i, j, trans) : 0.0;
        }
        for (int e = tid; e < TK * NC; e += 256) {
            const int b = e / NC, q = e % NC;
            const int j = jr[b];
            Gs[b][q] = (j >= 0) ? G[(int64_t)j * NC + q] : 0.0;
        }
        __syncthreads();
        for (int b = 0; b < kn; ++b) {
            const double kij = Ks[ri][b];
#pragma unroll
            for (int q = 0; q < MAXQ; ++q) {
                const int col = q * 4 + ph;
                if (col < NC) acc[q] = fma(kij, Gs[b][col], acc[q]);
            }
        }
        __syncthreads();
    }
    const int64_t i = i0 + ri;
    if (i >= n) return;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        const int col = q * 4 + ph;
        if (col >= NC) continue;
        if (split && col >= split) out1[((int64_t)c * n + i) * split + (col - split)] = acc[q];
        else out0[((int64_t)c * n + i) * (split ? split : NC) + col] = acc[q];
    }
}

// leaf: OUT[c][i][t] = sum over active boxes beta of A(i, start_beta + t)
__global__ void __launch_bounds__(256) k_sample_leaf64(OpDev o, const int *act_ptr, const int *act_box,
                                                       const int *ent, int m, double *out) {
    const int c = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2);
    const int ph = threadIdx.x & 3, t0 = blockIdx.z * 64;  // columns [t0, t0 + 64)
    if (i >= o.n) return;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int a = act_ptr[c]; a < act_ptr[c + 1]; ++a) {
        const int *e = ent + (int64_t)act_box[a] * ENT_FIELDS;
        const int s = e[3], len = e[4] - e[3];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int t = t0 + q * 4 + ph;
            if (t < len && t < m) acc[q] += op_entry(o, i, s + t, 0);
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int t = t0 + q * 4 + ph;
        if (t < m) out[((int64_t)c * o.n + i) * m + t] = acc[q];
    }
}

// interleave [GO | GP] rows for the fused symmetric sweep
__global__ void k_interleave(const double *GO, const double *GP, int64_t n, int r, double *GG) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * r) return;
    const int64_t i = t / r;
    const int j = (int)(t - i * r);
    GG[i * 2 * r + j] = GO[t];
    GG[i * 2 * r + r + j] = GP[t];
}

template <int MAXQ>
static void launch_sample64(const OpDev &o, int trans, const int64_t *rp, const int *rows, const double *G, int NC,
                            double *o0, double *o1, int split, int chi, cudaStream_t st) {
    dim3 grid(ceil_div(o.n, TR), chi);
    k_sample64<MAXQ><<<grid, 256, 0, st>>>(o, trans, rp, rows, G, NC, o0, o1, split); ::hm::count_launch();
}

static Err run_sample64(const OpDev &o, int trans, const int64_t *rp, const int *rows, const double *G, int NC,
                        double *o0, double *o1, int split, int chi, cudaStream_t st) {
    if (chi == 0) return ok();
    if (NC <= 16) launch_sample64<4>(o, trans, rp, rows, G, NC, o0, o1, split, chi, st);
    else if (NC <= 32) launch_sample64<8>(o, trans, rp, rows, G, NC, o0, o1, split, chi, st);
    else if (NC <= 64) launch_sample64<16>(o, trans, rp, rows, G, NC, o0, o1, split, chi, st);
    else if (NC <= 128) launch_sample64<32>(o, trans, rp, rows, G, NC, o0, o1, split, chi, st);
    else return fail(HM_ENOTSUP, "sample: more than 128 columns per colour");
    HM_LAUNCH("sample64");
    return ok();
}

// ---------------------------------------------------------------------------
// user black box: dense Omega in original order, then back to colour-major
// ---------------------------------------------------------------------------

__global__ void k_build_omega(int64_t n, int chi, int cols, const int *pt2ent, const int *ent_cptr,
                              const int *ent_col, const double *G, int leaf, const int *ent, const int *perm,
                              double *Om) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = pt2ent[i];
    const int64_t orow = perm[i];
    for (int k = ent_cptr[e]; k < ent_cptr[e + 1]; ++k) {
        const int c = ent_col[k];
        if (leaf) {
            const int t = (int)i - ent[(int64_t)e * ENT_FIELDS + 3];
            Om[orow + n * ((int64_t)c * cols + t)] = 1.0;
        } else {
            for (int j = 0; j < cols; ++j) Om[orow + n * ((int64_t)c * cols + j)] = G[i * cols + j];
        }
    }
}

__global__ void k_gather_samples(int64_t n, int s, const int *perm, const double *Yd, double *Y, int cols) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * s) return;
    const int64_t col = t / n, i = t - col * n;
    const int64_t c = col / cols, j = col - c * cols;
    Y[(c * n + i) * cols + j] = Yd[perm[i] + n * col];
}

static Err sample_callback(hm_ctx *c, const hm_op *op, const Coloring &g, bool leaf, double *Y, double *Z) {
    const int64_t n = c->n;
    const int chi = g.n_colors, cols = g.m_cols;
    const int64_t s = (int64_t)chi * cols;
    const Cut &cu = c->cuts[g.level];
    HM_TRY(ensure(c->scratch_a, (size_t)n * s * sizeof(double)));
    HM_TRY(ensure(c->scratch_b, (size_t)n * s * sizeof(double)));
    double *Om = c->scratch_a.as<double>(), *Yd = c->scratch_b.as<double>();
    for (int side = 0; side < (leaf ? 1 : 2); ++side) {
        HM_CUDA(cudaMemsetAsync(Om, 0, (size_t)n * s * sizeof(double), c->st));
        k_build_omega<<<ceil_div(n, 256), 256, 0, c->st>>>(n, chi, cols, cu.pt2ent.as<int>(), g.ent_cptr.as<int>(),
                                                           g.ent_col.as<int>(),
                                                           side ? c->GP.as<double>() : c->GO.as<double>(), leaf,
                                                           cu.ent.as<int>(), c->perm.as<int>(), Om); ::hm::count_launch();
        HM_LAUNCH("build_omega");
        const int rc = op->apply(op->user, side, Om, Yd, s, (void *)c->st);
        if (rc != 0) return fail(HM_EOP, "black-box operator returned " + std::to_string(rc));
        HM_LAUNCH("user operator");
        k_gather_samples<<<ceil_div(n * s, 256), 256, 0, c->st>>>(n, (int)s, c->perm.as<int>(), Yd, side ? Z : Y,
                                                                  cols); ::hm::count_launch();
        HM_LAUNCH("gather_samples");
    }
    return ok();
}

// M_a (k_a x r) of box vertex v: entry (u, j) = gauss(seed, 3, level, gid(a), u, j)
__global__ void k_mix_gauss(const int *vbox, int64_t nv, const int *kbox, const int64_t *moff, const int *ent,
                            int level, int r, unsigned long long seed, double *M) {
    const int64_t v = blockIdx.x;
    if (v >= nv) return;
    const int gid = ent[(int64_t)vbox[v] * ENT_FIELDS + 2];
    for (int o = threadIdx.x; o < kbox[v] * r; o += blockDim.x)
        M[moff[v] + o] = gauss(seed, 3, level, gid, o / r, o % r);
}

Err make_mix(hm_ctx *c, int level, const int *vbox, int64_t nv, const int *kbox, const int64_t *moff, double *M) {
    if (nv == 0) return ok();
    k_mix_gauss<<<(unsigned)nv, 128, 0, c->st>>>(vbox, nv, kbox, moff, c->cuts[level].ent.as<int>(), level,
                                                  c->cfg.r, (unsigned long long)c->cfg.seed, M); ::hm::count_launch();
    HM_LAUNCH("mix_gauss");
    return ok();
}

static OpDev make_opdev(const hm_ctx *c, const hm_op *op) {
    OpDev o;
    o.kind = op->kind;
    o.kernel = op->kernel;
    o.xs = c->xs.as<double>();
    o.dense = op->dense_dev;
    o.perm = c->perm.as<int>();
    o.n = c->n;
    return o;
}

Err sample_level(hm_ctx *c, const hm_op *op, int level, bool leaf) {
    const int idx = leaf ? c->L + 1 : level;
    const Coloring &g = (!leaf && c->cur_tiles) ? *c->cur_tiles : c->colorings[idx];
    const int chi = g.n_colors, cols = g.m_cols;
    const int64_t n = c->n;
    Samples &S = c->cur;
    S.level = leaf ? HM_LEVEL_LEAF : level;
    S.chi = chi;
    S.cols = cols;
    const size_t bytes = (size_t)chi * n * cols * sizeof(double);
    HM_TRY(ensure(S.Y, bytes));
    if (!leaf) HM_TRY(ensure(S.Z, bytes));
    if (chi == 0) return ok();
    if (op->kind == HM_OP_CALLBACK) {
        c->bb_fp64_levels++;
        return sample_callback(c, op, g, leaf, S.Y.as<double>(), S.Z.as<double>());
    }
    if (op->kind != HM_OP_KERNEL && op->kind != HM_OP_DENSE) return fail(HM_EINVAL, "unknown operator kind");
    const OpDev o = make_opdev(c, op);
    const Cut &cu = c->cuts[g.level];
    if (leaf && c->cfg.precision != HM_FP64 && op->kind == HM_OP_KERNEL)
        return sample_leaf_mixed(c, op->kernel);  // FP32 kernel values, FP64 sums
    // from here on the black box runs in FP64 (or on tensor cores, counted there)
    if (leaf) {
        c->bb_fp64_levels++;
        dim3 grid(ceil_div(n, 64), chi, ceil_div(cols, 64));
        k_sample_leaf64<<<grid, 256, 0, c->st>>>(o, g.act_ptr.as<int>(), g.act_box.as<int>(), cu.ent.as<int>(), cols,
                                                 S.Y.as<double>()); ::hm::count_launch();
        HM_LAUNCH("sample_leaf64");
        return ok();
    }
    if (c->cfg.precision != HM_FP64 && op->kind == HM_OP_KERNEL && tc_supported(c)) {
        c->bb_tc_levels++;
        return sample_tc(c, level, op->kernel);
    }
    c->bb_fp64_levels++;
    const int64_t *rp = g.act_rows_ptr.as<int64_t>();
    const int *rows = g.act_rows.as<int>();
    if (op->kind == HM_OP_KERNEL) {
        // symmetric kernel: one sweep for [Y | Z]
        HM_TRY(ensure(c->scratch_c, (size_t)n * 2 * cols * sizeof(double)));
        k_interleave<<<ceil_div(n * cols, 256), 256, 0, c->st>>>(c->GO.as<double>(), c->GP.as<double>(), n, cols,
                                                                 c->scratch_c.as<double>()); ::hm::count_launch();
        HM_LAUNCH("interleave");
        return run_sample64(o, 0, rp, rows, c->scratch_c.as<double>(), 2 * cols, S.Y.as<double>(), S.Z.as<double>(),
                            cols, chi, c->st);
    }
    HM_TRY(run_sample64(o, 0, rp, rows, c->GO.as<double>(), cols, S.Y.as<double>(), nullptr, 0, chi, c->st));
    return run_sample64(o, 1, rp, rows, c->GP.as<double>(), cols, S.Z.as<double>(), nullptr, 0, chi, c->st);
}

// y = A x or A^* x (dense vectors, sorted order, row-major [n][nrhs]) with a built-in operator
Err op_apply_dense_vectors(hm_ctx *c, const hm_op *op, const double *x_sorted, double *y_sorted, int nrhs,
                           int trans) {
    const OpDev o = make_opdev(c, op);
    return run_sample64(o, trans, nullptr, nullptr, x_sorted, nrhs, y_sorted, nullptr, 0, 1, c->st);
}

}  // namespace hm
