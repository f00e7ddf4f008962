// Peeling for the mixed-precision mode (Section 4.1.2, Algorithm 4.1):
//     Y_l(I_alpha, c) -= sum over coarse pairs q of U_q(I_alpha) B_q V_q^T Omega_l(I_b, c)
// (and the transpose for Z).  The products of the coarse factors run in FP32
// from FP32 copies of U, V, B and of the level's Gaussians; the subtraction from
// the FP64 samples is FP64.  The FP32 products carry the same ~1e-7 relative
// rounding as the mixed-precision black-box samples they are subtracted from.
//
// One warp owns one (tile, chunk of 32 rows), lane = row, and walks every
// coarse level and pair with warp-level synchronisation only:
//   * the level-l boxes gamma inside the coarse pair's other box that are
//     active in the tile's colour c form a contiguous run of that colour's
//     sorted active-box list, found by two binary searches;
//   * W = sum of the precomputed X_{q,gamma} = F_q(I_gamma)^T G(I_gamma) over
//     them, T = B_q W (or B_q^T W), and acc(row) += F_q'(row, :) T;
//   * at the end the FP64 tile -= acc.
#include "ctx.cuh"

namespace hm {

namespace pm {

constexpr int WARPS = 4;  // warps per CTA

__global__ void k_to_f32(const double *in, float *out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// size of the X block of each coarse pair: k x cols per level-l box inside its box
__global__ void k_xsize(const int *pair_alpha, const int *pair_col, int64_t np, const int *entj, const int *pt2ent_l,
                        const int *kdim, int cols, int side, int64_t *xsz) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= np) return;
    const int box = side ? pair_alpha[q] : pair_col[q];
    const int *e = entj + (int64_t)box * ENT_FIELDS;
    xsz[q] = (int64_t)(pt2ent_l[e[4] - 1] + 1 - pt2ent_l[e[3]]) * kdim[q] * cols;
}

// X_{q,gamma} (k x cols, FP32): F_q(I_gamma)^T G(I_gamma), or the identity
// block's F rows at the leaf step; CTA (q, y) takes the gammas y, y + gridDim.y, ...
__global__ void k_peel_x32(const int *pair_alpha, const int *pair_col, const int *entj, const int *entl,
                           const int *pt2ent_l, const int *kdim, const int64_t *offF, const float *F, const float *G,
                           int cols, int identity, int side, const int64_t *xoff, float *X) {
    const int64_t q = blockIdx.x;
    const int k = kdim[q];
    if (k == 0) return;
    const int box = side ? pair_alpha[q] : pair_col[q];
    const int *e = entj + (int64_t)box * ENT_FIELDS;
    const int bstart = e[3];
    const int kb = pt2ent_l[e[3]], ke = pt2ent_l[e[4] - 1] + 1;
    const float *Fq = F + offF[q];
    float *Xq = X + xoff[q];
    for (int g = kb + blockIdx.y; g < ke; g += gridDim.y) {
        const int *eg = entl + (int64_t)g * ENT_FIELDS;
        const int s0 = eg[3], len = eg[4] - eg[3];
        float *xg = Xq + (int64_t)(g - kb) * k * cols;
        for (int o = threadIdx.x; o < k * cols; o += blockDim.x) {
            const int v = o / cols, t = o % cols;
            float acc = 0.0f;
            if (identity) {
                acc = (t < len) ? Fq[(int64_t)(s0 - bstart + t) * k + v] : 0.0f;
            } else {
                for (int i = 0; i < len; ++i)
                    acc = fmaf(Fq[(int64_t)(s0 - bstart + i) * k + v], G[(int64_t)(s0 + i) * cols + t], acc);
            }
            xg[o] = acc;
        }
    }
}

struct Coarse {
    const int *ent, *pt2ent, *int_ptr, *int_idx, *pairT;
    const int *kU, *kV;
    const int64_t *offU, *offV, *offB;
    const float *U, *V, *B;
    const int64_t *xoff;
    const float *X;
};

__device__ __forceinline__ int lower_bound(const int *a, int lo, int hi, int key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_item_count(const int *tile_alpha, const int *entl, int64_t ntiles, int64_t *cnt) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= ntiles) return;
    const int *e = entl + (int64_t)tile_alpha[p] * ENT_FIELDS;
    cnt[p] = (e[4] - e[3] + 31) / 32;
}

__global__ void k_item_fill(const int64_t *off, int64_t ntiles, int64_t *item_tile, int *item_row) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= ntiles) return;
    for (int64_t k = off[p]; k < off[p + 1]; ++k) {
        item_tile[k] = p;
        item_row[k] = (int)(k - off[p]) * 32;
    }
}

// MAXC: compile-time bound on the columns per colour (32 or 64)
template <int MAXC>
__global__ void __launch_bounds__(WARPS * 32) k_peel_warp(const Coarse *cl, int ncl, int side, const int *tile_alpha,
                                                         const int *tile_color, const int *entl,
                                                         const int *pt2ent_l, const int *act_ptr,
                                                         const int *act_box, const int64_t *item_tile,
                                                         const int *item_row, int64_t nitems, int cols, int kcap,
                                                         int64_t n, double *OUT) {
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * WARPS + warp;
    if (item >= nitems) return;  // the whole warp leaves together
    float *W = sm + (size_t)warp * 2 * kcap * MAXC;
    float *T = W + (size_t)kcap * MAXC;
    const int64_t p = item_tile[item];
    const int alpha = tile_alpha[p], c = tile_color[p];
    const int *ea = entl + (int64_t)alpha * ENT_FIELDS;
    const int sa = ea[3] + item_row[item];
    const int rows = min(32, ea[4] - sa);
    const bool live = lane < rows;
    float acc[MAXC];
#pragma unroll
    for (int j = 0; j < MAXC; ++j) acc[j] = 0.0f;
    const int a0 = act_ptr[c], a1 = act_ptr[c + 1];
    for (int lvl = 0; lvl < ncl; ++lvl) {
        const Coarse &C = cl[lvl];
        const int anc = C.pt2ent[sa];
        const int anc_start = C.ent[(int64_t)anc * ENT_FIELDS + 3];
        for (int t = C.int_ptr[anc]; t < C.int_ptr[anc + 1]; ++t) {
            const int q = side ? C.pairT[t] : t;
            const int kin = side ? C.kU[q] : C.kV[q];
            const int kout = side ? C.kV[q] : C.kU[q];
            if (kin == 0 || kout == 0) continue;
            const int *eo = C.ent + (int64_t)C.int_idx[t] * ENT_FIELDS;
            const int kb = pt2ent_l[eo[3]], ke = pt2ent_l[eo[4] - 1] + 1;
            const int lo = lower_bound(act_box, a0, a1, kb);
            const int hi = lower_bound(act_box, lo, a1, ke);
            if (lo == hi) continue;
            // W = sum of X_{q,gamma} over the active gammas (kin x cols)
            const float *Xq = C.X + C.xoff[q];
            for (int o = lane; o < kin * cols; o += 32) {
                float s = 0.0f;
                for (int g = lo; g < hi; ++g) s += Xq[(int64_t)(act_box[g] - kb) * kin * cols + o];
                W[(o / cols) * MAXC + o % cols] = s;
            }
            __syncwarp();
            // T = B W (Y side, B is kout x kin) or B^T W (Z side)
            const float *Bq = C.B + C.offB[q];
            for (int o = lane; o < kout * cols; o += 32) {
                const int u = o / cols, col = o % cols;
                float s = 0.0f;
                for (int v = 0; v < kin; ++v)
                    s = fmaf(side ? Bq[v * kout + u] : Bq[u * kin + v], W[v * MAXC + col], s);
                T[u * MAXC + col] = s;
            }
            __syncwarp();
            // acc(row) += F(row, :) T, F = U_q (Y side) or V_q (Z side), rows inside anc
            const float *F = side ? C.V + C.offV[q] : C.U + C.offU[q];
            const float *Fr = F + (int64_t)(sa - anc_start + lane) * kout;
            for (int u = 0; u < kout; ++u) {
                const float f = live ? Fr[u] : 0.0f;
                const float4 *tr = reinterpret_cast<const float4 *>(T + u * MAXC);
#pragma unroll
                for (int j4 = 0; j4 < MAXC / 4; ++j4) {
                    const float4 tv = tr[j4];
                    acc[4 * j4] = fmaf(f, tv.x, acc[4 * j4]);
                    acc[4 * j4 + 1] = fmaf(f, tv.y, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(f, tv.z, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(f, tv.w, acc[4 * j4 + 3]);
                }
            }
            __syncwarp();
        }
    }
    if (!live) return;
    double *out = OUT + ((int64_t)c * n + sa + lane) * cols;
#pragma unroll
    for (int j = 0; j < MAXC; ++j)
        if (j < cols) out[j] -= (double)acc[j];
}

}  // namespace pm

static Err f32_copy(DBuf &dst, const DBuf &src, int64_t count, cudaStream_t st) {
    HM_TRY(alloc(dst, std::max<int64_t>(count, 1) * sizeof(float)));
    if (count > 0) {
        pm::k_to_f32<<<ceil_div(count, 256), 256, 0, st>>>(src.as<double>(), dst.as<float>(), count);
        count_launch();
        HM_LAUNCH("to_f32");
    }
    return ok();
}

// FP32 copies of a level's factors, made once when a finer level first peels it
static Err factors_f32(Factors &f, cudaStream_t st) {
    if (f.U32.p) return ok();
    HM_TRY(f32_copy(f.U32, f.U, f.nU, st));
    HM_TRY(f32_copy(f.V32, f.V, f.nV, st));
    HM_TRY(f32_copy(f.B32, f.B, f.nB, st));
    return ok();
}

Err peel_level_mixed(hm_ctx *c, int level, bool leaf) {
    const int l = leaf ? c->L : level;
    const int idx = leaf ? c->L + 1 : level;
    const Coloring &g = c->colorings[idx];
    if (g.n_pairs == 0 || g.n_colors == 0) return ok();
    const int cols = g.m_cols;
    const int jmax = leaf ? c->L : level - 1;
    const Cut &cl = c->cuts[l];
    cudaStream_t st = c->st;
    const int r = c->cfg.r;
    const int64_t n = c->n;
    // FP32 Gaussians of this level (not used at the leaf: identity test matrices)
    DBuf G32[2];
    if (!leaf) {
        HM_TRY(f32_copy(G32[0], c->GO, n * r, st));
        HM_TRY(f32_copy(G32[1], c->GP, n * r, st));
    }
    // work items: 32-row chunks of every tile
    const int64_t ntiles = g.n_pairs;
    DBuf cnt, off, item_tile, item_row;
    HM_TRY(alloc(cnt, (ntiles + 1) * sizeof(int64_t)));
    HM_TRY(alloc(off, (ntiles + 1) * sizeof(int64_t)));
    pm::k_item_count<<<ceil_div(ntiles, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), cl.ent.as<int>(), ntiles,
                                                            cnt.as<int64_t>());
    count_launch();
    HM_LAUNCH("item_count");
    HM_TRY(scan_exclusive(cnt.as<int64_t>(), off.as<int64_t>(), ntiles, st));
    int64_t nitems = 0;
    HM_TRY(read_scalar(nitems, off.as<int64_t>() + ntiles, st));
    HM_TRY(alloc(item_tile, nitems * sizeof(int64_t)));
    HM_TRY(alloc(item_row, nitems * sizeof(int)));
    pm::k_item_fill<<<ceil_div(ntiles, 256), 256, 0, st>>>(off.as<int64_t>(), ntiles, item_tile.as<int64_t>(),
                                                           item_row.as<int>());
    count_launch();
    HM_LAUNCH("item_fill");

    for (int side = 0; side < (leaf ? 1 : 2); ++side) {
        std::vector<pm::Coarse> tab;
        std::vector<DBuf> xs, xoffs;
        for (int j = 2; j <= jmax; ++j) {
            if (j >= (int)c->factors.size() || !c->factors[j].done || c->factors[j].n_pairs == 0) continue;
            Factors &f = c->factors[j];
            const Coloring &gj = c->colorings[j];
            const Cut &cj = c->cuts[j];
            const int64_t np = f.n_pairs;
            HM_TRY(factors_f32(f, st));
            DBuf xsz, xo, X;
            HM_TRY(alloc(xsz, (np + 1) * sizeof(int64_t)));
            HM_TRY(alloc(xo, (np + 1) * sizeof(int64_t)));
            const int *kdim = side ? f.kU.as<int>() : f.kV.as<int>();
            pm::k_xsize<<<ceil_div(np, 256), 256, 0, st>>>(gj.pair_alpha.as<int>(), cj.int_idx.as<int>(), np,
                                                           cj.ent.as<int>(), cl.pt2ent.as<int>(), kdim, cols, side,
                                                           xsz.as<int64_t>());
            count_launch();
            HM_LAUNCH("xsize");
            HM_TRY(scan_exclusive(xsz.as<int64_t>(), xo.as<int64_t>(), np, st));
            int64_t xtot = 0;
            HM_TRY(read_scalar(xtot, xo.as<int64_t>() + np, st));
            HM_TRY(alloc(X, std::max<int64_t>(xtot, 1) * sizeof(float)));
            // CTAs per coarse pair: about one per level-l box inside the largest coarse box
            const int gy = std::min(256, std::max(1, cj.max_rows / std::max(1, std::min(cl.max_rows, 64))));
            pm::k_peel_x32<<<dim3((unsigned)np, gy), 128, 0, st>>>(gj.pair_alpha.as<int>(), cj.int_idx.as<int>(), cj.ent.as<int>(),
                                                     cl.ent.as<int>(), cl.pt2ent.as<int>(), kdim,
                                                     side ? f.offU.as<int64_t>() : f.offV.as<int64_t>(),
                                                     side ? f.U32.as<float>() : f.V32.as<float>(),
                                                     leaf ? nullptr : G32[side].as<float>(), cols, leaf ? 1 : 0, side,
                                                     xo.as<int64_t>(), X.as<float>());
            count_launch();
            HM_LAUNCH("peel_x32");
            pm::Coarse co;
            co.ent = cj.ent.as<int>();
            co.pt2ent = cj.pt2ent.as<int>();
            co.int_ptr = cj.int_ptr.as<int>();
            co.int_idx = cj.int_idx.as<int>();
            co.pairT = gj.pair_T.as<int>();
            co.kU = f.kU.as<int>();
            co.kV = f.kV.as<int>();
            co.offU = f.offU.as<int64_t>();
            co.offV = f.offV.as<int64_t>();
            co.offB = f.offB.as<int64_t>();
            co.U = f.U32.as<float>();
            co.V = f.V32.as<float>();
            co.B = f.B32.as<float>();
            co.xoff = xo.as<int64_t>();
            co.X = X.as<float>();
            tab.push_back(co);
            xs.push_back(std::move(X));
            xoffs.push_back(std::move(xo));
        }
        if (tab.empty()) continue;
        DBuf tabd;
        HM_TRY(alloc(tabd, tab.size() * sizeof(pm::Coarse)));
        HM_CUDA(cudaMemcpyAsync(tabd.p, tab.data(), tab.size() * sizeof(pm::Coarse), cudaMemcpyHostToDevice, st));
        double *OUT = side ? c->cur.Z.as<double>() : c->cur.Y.as<double>();
        const int grid = ceil_div(nitems, pm::WARPS);
        if (cols <= 32) {
            const size_t smem = (size_t)pm::WARPS * 2 * r * 32 * sizeof(float);
            HM_CUDA(cudaFuncSetAttribute(pm::k_peel_warp<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            pm::k_peel_warp<32><<<grid, pm::WARPS * 32, smem, st>>>(
                tabd.as<pm::Coarse>(), (int)tab.size(), side, g.pair_alpha.as<int>(), g.pair_color.as<int>(),
                cl.ent.as<int>(), cl.pt2ent.as<int>(), g.act_ptr.as<int>(), g.act_box.as<int>(), item_tile.as<int64_t>(),
                item_row.as<int>(), nitems, cols, r, n, OUT);
        } else {
            const size_t smem = (size_t)pm::WARPS * 2 * r * 64 * sizeof(float);
            HM_CUDA(cudaFuncSetAttribute(pm::k_peel_warp<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            pm::k_peel_warp<64><<<grid, pm::WARPS * 32, smem, st>>>(
                tabd.as<pm::Coarse>(), (int)tab.size(), side, g.pair_alpha.as<int>(), g.pair_color.as<int>(),
                cl.ent.as<int>(), cl.pt2ent.as<int>(), g.act_ptr.as<int>(), g.act_box.as<int>(), item_tile.as<int64_t>(),
                item_row.as<int>(), nitems, cols, r, n, OUT);
        }
        count_launch();
        HM_LAUNCH("peel_warp");
    }
    return ok();
}

}  // namespace hm
