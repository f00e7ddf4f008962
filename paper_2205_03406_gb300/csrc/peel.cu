// Peeling (Section 4.1.2, Algorithm 4.1): remove the contribution of the
// coarser levels already compressed from the samples of cut level l.  Colours
// of up to 64 columns (every admissible level, and leaves of up to 64 points)
// go to peel_mixed.cu, which forms T = B W once per (coarse pair, colour), in
// FP32 or FP64; this file holds that dispatch and the per-tile FP64 peel that
// serves wider leaf colours:
//     Y_l -= A^(l-1) Omega_l,   Z_l -= A^(l-1)* Psi_l,
// where A^(l-1) holds the factors U B V^T of every admissible pair of levels
// 2..l-1 (2..L for the leaf step).  Only the tiles that a pair of level l reads
// are peeled: the tile of pair p = (alpha, beta) is Y(I_alpha, colour of p),
// and the same rows and colour of Z serve the transposed pair.
//
// For a coarse pair q = (a, b) and a colour c, the test matrix restricted to
// I_b is the sum of G_gamma over the level-l boxes gamma inside b that are
// active in c, so
//     V_q^T Omega_l(I_b, c) = sum_{gamma in b, c active} V_q(I_gamma)^T G_gamma.
// Stage X computes the products X_{q,gamma} = V_q(I_gamma)^T G_gamma once per
// coarse level; stage U sums the matching ones per tile and applies B_q and the
// rows of U_q that belong to the tile.  One launch per coarse level keeps each
// tile owned by one CTA, so the result is deterministic.
#include "ctx.cuh"

namespace hm {

// X size of each coarse pair: k times cols times the number of level-l entries
// inside its column box (Y side: b_q) or its row box (Z side: a_q)
__global__ void k_desc_count(const int *pair_alpha, const int *pair_col, int64_t np, const int *entj,
                             const int *pt2ent_l, const int *kdim, int cols, int side, int64_t *xsz) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= np) return;
    const int box = side ? pair_alpha[q] : pair_col[q];
    const int *e = entj + (int64_t)box * ENT_FIELDS;
    const int kb = pt2ent_l[e[3]], ke = pt2ent_l[e[4] - 1] + 1;
    xsz[q] = (int64_t)(ke - kb) * kdim[q] * cols;
}

// X_{q,gamma} = F_q(I_gamma)^T G(I_gamma), F = V (Y side) or U (Z side);
// identity G at the leaf: X[v][t] = F(start_gamma + t, v) for t < |I_gamma|.
__global__ void k_peel_x(const int *pair_alpha, const int *pair_col, int64_t np, const int *entj, const int *entl,
                         const int *pt2ent_l, const int *kdim, const int64_t *offF, const double *F,
                         const double *G, int cols, int identity, int side, const int64_t *xoff, double *X) {
    const int64_t q = blockIdx.x;
    const int k = kdim[q];
    if (k == 0) return;
    const int box = side ? pair_alpha[q] : pair_col[q];
    const int *e = entj + (int64_t)box * ENT_FIELDS;
    const int bstart = e[3];
    const int kb = pt2ent_l[e[3]], ke = pt2ent_l[e[4] - 1] + 1;
    const double *Fq = F + offF[q];
    double *Xq = X + xoff[q];
    for (int g = kb; g < ke; ++g) {
        const int *eg = entl + (int64_t)g * ENT_FIELDS;
        const int s0 = eg[3], len = eg[4] - eg[3];
        double *xg = Xq + (int64_t)(g - kb) * k * cols;
        for (int o = threadIdx.x; o < k * cols; o += blockDim.x) {
            const int v = o / cols, t = o % cols;
            double acc = 0.0;
            if (identity) {
                acc = (t < len) ? Fq[(int64_t)(s0 - bstart + t) * k + v] : 0.0;
            } else {
                for (int i = 0; i < len; ++i)
                    acc = fma(Fq[(int64_t)(s0 - bstart + i) * k + v], G[(int64_t)(s0 + i) * cols + t], acc);
            }
            xg[o] = acc;
        }
    }
}

struct PeelLevel {
    // target cut l
    const int *entl, *pt2ent_l, *ent_cptr, *ent_col;
    // target pairs (tiles)
    const int *tile_alpha, *tile_color;
    int64_t ntiles;
    int cols;
    int kcap;   // largest k (= r): rows of the W and T scratch
    int64_t n;
    // coarse level j
    const int *entj, *pt2ent_j;
    const int *int_ptr_j, *int_idx_j, *pairT_j, *pair_alpha_j;
    const int *kU, *kV;
    const int64_t *offU, *offV, *offB;
    const double *U, *V, *B;
};

// One CTA per tile (alpha, c): rows I_alpha of Y[c] (side 0) or Z[c] (side 1).
// side 0: sum over q = (anc, b), b in int_j(anc): Y -= U_q(I_alpha) B_q W,
//         W = sum of X_{q,gamma} (V side) over gamma in b active in c;
// side 1: sum over q = (a, anc), a in int_j(anc): Z -= V_q(I_alpha) B_q^T W',
//         W' = sum of X'_{q,gamma} (U side) over gamma in a active in c.
__global__ void __launch_bounds__(128) k_peel_update(PeelLevel P, int side, const int64_t *xoff, const double *X,
                                                     double *OUT) {
    extern __shared__ double sm[];
    __shared__ int gl[128];
    __shared__ int wcnt[4];
    const int64_t tile = blockIdx.x;
    const int alpha = P.tile_alpha[tile], c = P.tile_color[tile];
    const int *ea = P.entl + (int64_t)alpha * ENT_FIELDS;
    const int sa = ea[3], ma = ea[4] - ea[3];
    const int cols = P.cols;
    double *W = sm;                // [r][cols]
    double *T = sm + P.kcap * cols;  // [r][cols]
    double *out = OUT + ((int64_t)c * P.n + sa) * cols;
    const int anc = P.pt2ent_j[sa];
    const int *eanc = P.entj + (int64_t)anc * ENT_FIELDS;
    for (int t = P.int_ptr_j[anc]; t < P.int_ptr_j[anc + 1]; ++t) {
        const int other = P.int_idx_j[t];                 // b (side 0) or a (side 1)
        const int q = side ? P.pairT_j[t] : t;            // pair (anc, b) or (a, anc)
        const int kin = side ? P.kU[q] : P.kV[q];         // rows of W
        const int kout = side ? P.kV[q] : P.kU[q];        // rows of T
        if (kin == 0 || kout == 0) continue;
        const int *eo = P.entj + (int64_t)other * ENT_FIELDS;
        const int kb = P.pt2ent_l[eo[3]], ke = P.pt2ent_l[eo[4] - 1] + 1;
        // W = sum of X_{q,gamma} over gamma in [kb, ke) active in colour c, in
        // increasing gamma, compacted 128 candidates at a time
        const double *Xq = X + xoff[q];
        for (int o = threadIdx.x; o < kin * cols; o += blockDim.x) W[o] = 0.0;
        int any = 0;
        for (int g0 = kb; g0 < ke; g0 += blockDim.x) {
            const int g = g0 + threadIdx.x;
            bool hit = false;
            if (g < ke)
                for (int u = P.ent_cptr[g]; u < P.ent_cptr[g + 1]; ++u) hit |= (P.ent_col[u] == c);
            const unsigned int bal = __ballot_sync(0xffffffffu, hit);
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            if (lane == 0) wcnt[w] = __popc(bal);
            __syncthreads();
            int base = 0;
            for (int u = 0; u < w; ++u) base += wcnt[u];
            if (hit) gl[base + __popc(bal & ((1u << lane) - 1))] = g - kb;
            const int ng = wcnt[0] + wcnt[1] + wcnt[2] + wcnt[3];
            __syncthreads();
            if (ng) {
                any = 1;
                for (int o = threadIdx.x; o < kin * cols; o += blockDim.x) {
                    double acc = W[o];
                    for (int u = 0; u < ng; ++u) acc += Xq[(int64_t)gl[u] * kin * cols + o];
                    W[o] = acc;
                }
            }
            __syncthreads();
        }
        if (!any) continue;
        // T = B W (side 0, B is kU x kV) or B^T W (side 1)
        const double *Bq = P.B + P.offB[q];
        for (int o = threadIdx.x; o < kout * cols; o += blockDim.x) {
            const int u = o / cols, col = o % cols;
            double acc = 0.0;
            for (int v = 0; v < kin; ++v) {
                const double bv = side ? Bq[(int64_t)v * kout + u] : Bq[(int64_t)u * kin + v];
                acc = fma(bv, W[v * cols + col], acc);
            }
            T[o] = acc;
        }
        __syncthreads();
        // OUT(I_alpha) -= F(rows of alpha) T, F = U_q (side 0) or V_q (side 1)
        const double *F = side ? (P.V + P.offV[q]) : (P.U + P.offU[q]);
        const int rowbox_start = eanc[3];           // anc holds the tile's rows on both sides
        const double *Fr = F + (int64_t)(sa - rowbox_start) * kout;
        for (int o = threadIdx.x; o < ma * cols; o += blockDim.x) {
            const int i = o / cols, col = o % cols;
            double acc = 0.0;
            for (int u = 0; u < kout; ++u) acc = fma(Fr[(int64_t)i * kout + u], T[u * cols + col], acc);
            out[(int64_t)i * cols + col] -= acc;
        }
        __syncthreads();
    }
}

Err peel_level(hm_ctx *c, int level, bool leaf) {
    const int l = leaf ? c->L : level;
    const int idx = leaf ? c->L + 1 : level;
    const Coloring &g = (!leaf && c->cur_tiles) ? *c->cur_tiles : c->colorings[idx];
    if (g.n_pairs == 0 || g.n_colors == 0) return ok();
    const int cols = g.m_cols;
    // up to 64 columns per colour: T = B W once per (coarse pair, colour) and a
    // register-tiled update (peel_mixed.cu), in FP32 or FP64; wider leaves: below
    if (cols <= 64) {
        if (c->cfg.precision == HM_MIXED_BF16X6_F32) return peel_level_mixed(c, level, leaf);
        if (c->cfg.precision == HM_MIXED_BF16X6) return peel_level_df(c, level, leaf);
        return peel_level_fp64(c, level, leaf);
    }
    const int jmax = leaf ? c->L : level - 1;
    const Cut &cl = c->cuts[l];
    cudaStream_t st = c->st;
    const size_t smem = 2 * (size_t)c->cfg.r * cols * sizeof(double);
    if (smem > 200 * 1024) return fail(HM_ENOTSUP, "peel: r x columns per colour too large");
    HM_TRY(allow_smem(k_peel_update, (size_t)((int)smem)));
    for (int j = 2; j <= jmax; ++j) {
        if (j >= (int)c->factors.size() || !c->factors[j].done || c->factors[j].n_pairs == 0) continue;
        const Factors &f = c->factors[j];
        const Coloring &gj = c->colorings[j];
        const Cut &cj = c->cuts[j];
        const int64_t np = f.n_pairs;
        for (int side = 0; side < (leaf ? 1 : 2); ++side) {
            HM_TRY(ensure(c->scratch_c, 2 * (np + 1) * sizeof(int64_t)));
            int64_t *xsz = c->scratch_c.as<int64_t>();
            int64_t *xoff = xsz + (np + 1);
            k_desc_count<<<ceil_div(np, 256), 256, 0, st>>>(gj.pair_alpha.as<int>(), cj.int_idx.as<int>(), np,
                                                            cj.ent.as<int>(), cl.pt2ent.as<int>(),
                                                            side ? f.kU.as<int>() : f.kV.as<int>(), cols, side,
                                                            xsz); ::hm::count_launch();
            HM_LAUNCH("desc_count");
            HM_TRY(scan_exclusive(xsz, xoff, np, st));
            int64_t xtot = 0;
            HM_TRY(read_scalar(xtot, xoff + np, st));
            HM_TRY(ensure(c->scratch_d, std::max<int64_t>(xtot, 1) * sizeof(double)));
            const double *G = side ? c->GP.as<double>() : c->GO.as<double>();
            k_peel_x<<<(int)np, 128, 0, st>>>(gj.pair_alpha.as<int>(), cj.int_idx.as<int>(), np, cj.ent.as<int>(),
                                              cl.ent.as<int>(), cl.pt2ent.as<int>(),
                                              side ? f.kU.as<int>() : f.kV.as<int>(),
                                              side ? f.offU.as<int64_t>() : f.offV.as<int64_t>(),
                                              side ? f.U.as<double>() : f.V.as<double>(), G, cols, leaf ? 1 : 0,
                                              side, xoff, c->scratch_d.as<double>()); ::hm::count_launch();
            HM_LAUNCH("peel_x");
            PeelLevel P;
            P.entl = cl.ent.as<int>();
            P.pt2ent_l = cl.pt2ent.as<int>();
            P.ent_cptr = g.ent_cptr.as<int>();
            P.ent_col = g.ent_col.as<int>();
            P.tile_alpha = g.pair_alpha.as<int>();
            P.tile_color = g.pair_color.as<int>();
            P.ntiles = g.n_pairs;
            P.cols = cols;
            P.kcap = c->cfg.r;
            P.n = c->n;
            P.entj = cj.ent.as<int>();
            P.pt2ent_j = cj.pt2ent.as<int>();
            P.int_ptr_j = cj.int_ptr.as<int>();
            P.int_idx_j = cj.int_idx.as<int>();
            P.pairT_j = gj.pair_T.as<int>();
            P.pair_alpha_j = gj.pair_alpha.as<int>();
            P.kU = f.kU.as<int>();
            P.kV = f.kV.as<int>();
            P.offU = f.offU.as<int64_t>();
            P.offV = f.offV.as<int64_t>();
            P.offB = f.offB.as<int64_t>();
            P.U = f.U.as<double>();
            P.V = f.V.as<double>();
            P.B = f.B.as<double>();
            double *OUT = side ? c->cur.Z.as<double>() : c->cur.Y.as<double>();
            k_peel_update<<<(int)g.n_pairs, 128, smem, st>>>(P, side, xoff, c->scratch_d.as<double>(), OUT); ::hm::count_launch();
            HM_LAUNCH("peel_update");
        }
    }
    return ok();
}

}  // namespace hm
