// Uniform H^1 compression of one level (Section 4.2, with Algorithm 2.2's two
// stages applied to every box at once):
//
//  stage 1  box colouring (colour.cu: box alpha asks for G on int(alpha) and
//           zeros on near(alpha)); Y = A Omega - A^(l-1) Omega on the tiles
//           Y(I_alpha, colour of alpha) (the sampler and the peel run on the
//           box colouring); U_alpha = the whole r-column sample basis
//           (pivoted QR, k = min(r, |I_alpha|, rows of int(alpha)));
//  stage 2  the pair colouring with the bases in place of Gaussians:
//           Psi(I_alpha) = U_alpha, Z = A^* Psi - A^(l-1)* Psi, so the tile of
//           the pair (beta, alpha) is T_ab = A_ab^* U_alpha on I_beta;
//           W_beta = sum over alpha in int(beta) of T_ab M_alpha with Gaussian
//           k_alpha x r mixes M_alpha (Philox side 3, keyed by the box);
//           V_beta = qr(W_beta, k) with the rank or tolerance rule;
//           B_ab = T_ab^T V_beta.
//
// The bases are stored once per box; the per-pair offsets of the factor arena
// point at them, so the peel of finer levels and the apply read the level as
// they read a per-pair one.  Every product here is FP64.
#include "ctx.cuh"

#include <algorithm>

namespace hm {

namespace un {

// rows of int(alpha) of every box vertex (the width of its sampled block row)
__global__ void k_width(const int *vbox, int64_t nv, const int *ent, const int *int_ptr, const int *int_idx,
                        int *width) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int a = vbox[v];
    int w = 0;
    for (int t = int_ptr[a]; t < int_ptr[a + 1]; ++t) {
        const int *e = ent + (int64_t)int_idx[t] * ENT_FIELDS;
        w += e[4] - e[3];
    }
    width[v] = w;
}

// stage-1 caps: min(r, width); the QR caps by |I_alpha| itself
__global__ void k_cap_u(const int *width, int64_t nv, int r, int *cap) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < nv) cap[v] = min(r, width[v]);
}

__global__ void k_box_sizes(const int *vbox, int64_t nv, const int *ent, const int *k, int r, int64_t *sz,
                            int64_t *msz) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int *e = ent + (int64_t)vbox[v] * ENT_FIELDS;
    sz[v] = (int64_t)(e[4] - e[3]) * k[v];
    if (msz) msz[v] = (int64_t)k[v] * r;
}

// copy the first k columns of a tile (layout [colour][n][r]) into the arena,
// and (fill != nullptr) the same rows into fill[n][r] with zeros beyond k
__global__ void k_pack_box(const int *vbox, const int *vcolor, const int *ent, int64_t n, int r, const int *k,
                           const int64_t *off, const double *src, double *dst, double *fill) {
    const int64_t v = blockIdx.x;
    const int *e = ent + (int64_t)vbox[v] * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3], kk = k[v];
    const double *T = src + ((int64_t)(vcolor ? vcolor[v] : 0) * n + s0) * r;
    for (int o = threadIdx.x; o < m * kk; o += blockDim.x) dst[off[v] + o] = T[(int64_t)(o / kk) * r + o % kk];
    if (fill)
        for (int o = threadIdx.x; o < m * r; o += blockDim.x) {
            const int i = o / r, j = o % r;
            fill[(int64_t)(s0 + i) * r + j] = j < kk ? T[(int64_t)i * r + j] : 0.0;
        }
}

// W_beta = sum over the entries t of int(beta) of Z[c_t](I_beta, 0:k_a) M_a,
// a = int_idx[t], c_t the colour of the pair (beta, a); into W[n][r].
// One CTA per box vertex beta; thread o owns entries (i, j) = (o / r, o % r).
__global__ void k_mix_sum(const int *vbox, int64_t nv, const int *ent, const int *int_ptr, const int *int_idx,
                          const int *pair_color, const int *vid, const int *kU, const int64_t *moff, const double *M,
                          const double *Z, int64_t n, int r, double *W) {
    const int64_t v = blockIdx.x;
    if (v >= nv) return;
    const int b = vbox[v];
    const int *e = ent + (int64_t)b * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3];
    for (int o = threadIdx.x; o < m * r; o += blockDim.x) {
        const int i = o / r, j = o % r;
        double acc = 0.0;
        for (int t = int_ptr[b]; t < int_ptr[b + 1]; ++t) {
            const int va = vid[int_idx[t]];
            const int ka = kU[va];
            const double *Zr = Z + ((int64_t)pair_color[t] * n + s0 + i) * r;
            const double *Ma = M + moff[va];
            for (int u = 0; u < ka; ++u) acc = fma(Zr[u], Ma[(int64_t)u * r + j], acc);
        }
        W[(int64_t)(s0 + i) * r + j] = acc;
    }
}

// factor tables of every pair p = (a, b): ranks, offsets into the per-box
// arenas, the size of B_p
__global__ void k_pair_factors(const int *pair_alpha, const int *pair_col, int64_t np, const int *vid, const int *kUb,
                               const int *kVb, const int64_t *offUb, const int64_t *offVb, int *kU, int *kV,
                               int64_t *offU, int64_t *offV, int64_t *szB) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int va = vid[pair_alpha[p]], vb = vid[pair_col[p]];
    kU[p] = kUb[va];
    kV[p] = kVb[vb];
    offU[p] = offUb[va];
    offV[p] = offVb[vb];
    szB[p] = (int64_t)kUb[va] * kVb[vb];
}

// B_p = T^T V_b, T = Z[c](I_b, 0:k_a) with c the colour of the transposed pair
// (b, a): k_a x k_b row-major.  One warp per pair.
__global__ void k_core_uniform(int64_t np, const int *pair_col, const int *pairT, const int *pair_color,
                               const int *ent, const int *kU, const int *kV, const int64_t *offV,
                               const int64_t *offB, const double *V, const double *Z, int64_t n, int r, double *B) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= np) return;
    const int ka = kU[p], kb = kV[p];
    if (ka == 0 || kb == 0) return;
    const int *e = ent + (int64_t)pair_col[p] * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3];
    const double *Zt = Z + ((int64_t)pair_color[pairT[p]] * n + s0) * r;
    const double *Vb = V + offV[p];
    for (int o = lane; o < ka * kb; o += 32) {
        const int u = o / kb, w = o % kb;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(Zt[(int64_t)i * r + u], Vb[(int64_t)i * kb + w], acc);
        B[offB[p] + o] = acc;
    }
}

}  // namespace un

// one level of the uniform H^1 compression; phase_secs[1..4] receive device
// time of the test matrices, black box, peel and bases (CUDA events)
Err uniform_level(hm_ctx *c, const hm_op *op, int l, double *phase_secs) {
    using namespace un;
    cudaStream_t st = c->st;
    Coloring &gb = c->box_colorings[l];
    Coloring &gp = c->colorings[l];
    const Cut &cu = c->cuts[l];
    const int r = c->cfg.r;
    const int64_t n = c->n;
    const int64_t nv = gb.n_vertices, np = gp.n_pairs;
    Factors &f = c->factors[l];
    f = Factors();
    f.n_pairs = np;
    if (np == 0 || nv == 0) {
        f.done = true;
        return ok();
    }
    struct Timer {
        cudaStream_t st;
        cudaEvent_t a = nullptr, b = nullptr;
        double *acc;
        explicit Timer(cudaStream_t s, double *x) : st(s), acc(x) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, st);
        }
        ~Timer() {
            cudaEventRecord(b, st);
            cudaEventSynchronize(b);
            float ms = 0.f;
            if (acc && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) *acc += ms * 1e-3;
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    };
    // box vertex of every cut entry
    DBuf vid, width, capu, kUb, kVb;
    HM_TRY(alloc(vid, (size_t)std::max(cu.nc, 1) * sizeof(int)));
    HM_CUDA(cudaMemsetAsync(vid.p, 0xff, (size_t)std::max(cu.nc, 1) * sizeof(int), st));
    {
        std::vector<int> hb;
        HM_TRY(to_host(hb, gb.pair_alpha.p, nv, st));
        std::vector<int> hv(cu.nc, -1);
        for (int64_t v = 0; v < nv; ++v) hv[hb[v]] = (int)v;
        HM_TRY(to_dev(vid, hv, st));
    }
    HM_TRY(alloc(width, nv * sizeof(int)));
    HM_TRY(alloc(capu, nv * sizeof(int)));
    HM_TRY(alloc(kUb, nv * sizeof(int)));
    HM_TRY(alloc(kVb, nv * sizeof(int)));
    k_width<<<ceil_div(nv, 128), 128, 0, st>>>(gb.pair_alpha.as<int>(), nv, cu.ent.as<int>(), cu.int_ptr.as<int>(),
                                               cu.int_idx.as<int>(), width.as<int>()); ::hm::count_launch();
    k_cap_u<<<ceil_div(nv, 128), 128, 0, st>>>(width.as<int>(), nv, r, capu.as<int>()); ::hm::count_launch();
    HM_LAUNCH("uniform widths");

    // ---- stage 1: Y on the box colouring, U = the sample bases
    {
        Timer tm(st, phase_secs ? phase_secs + 1 : nullptr);
        HM_TRY(make_gaussians(c, l));
    }
    c->cur_tiles = &gb;
    c->peel_sides = 1;
    Err e;
    {
        Timer tm(st, phase_secs ? phase_secs + 2 : nullptr);
        e = sample_level(c, op, l, false);
    }
    if (!e) {
        Timer tm(st, phase_secs ? phase_secs + 3 : nullptr);
        e = peel_level(c, l, false);
    }
    c->cur_tiles = nullptr;
    c->peel_sides = 3;
    HM_TRY(e);
    DBuf sz, offUb, msz, moff, M;
    {
        Timer tm(st, phase_secs ? phase_secs + 4 : nullptr);
        HM_TRY(qr_tiles_fp64(c, l, gb.pair_alpha.as<int>(), gb.pair_color.as<int>(), capu.as<int>(), nv,
                             cu.max_rows, c->cur.Y.as<double>(), r, r, 0.0, kUb.as<int>()));
        // U arena per box, and the stage-2 fill of Psi in place of the Gaussians of GP
        HM_TRY(alloc(sz, (nv + 1) * sizeof(int64_t)));
        HM_TRY(alloc(offUb, (nv + 1) * sizeof(int64_t)));
        HM_TRY(alloc(msz, (nv + 1) * sizeof(int64_t)));
        HM_TRY(alloc(moff, (nv + 1) * sizeof(int64_t)));
        k_box_sizes<<<ceil_div(nv, 128), 128, 0, st>>>(gb.pair_alpha.as<int>(), nv, cu.ent.as<int>(), kUb.as<int>(),
                                                       r, sz.as<int64_t>(), msz.as<int64_t>()); ::hm::count_launch();
        HM_TRY(scan_exclusive(sz.as<int64_t>(), offUb.as<int64_t>(), nv, st));
        HM_TRY(scan_exclusive(msz.as<int64_t>(), moff.as<int64_t>(), nv, st));
        HM_TRY(read_scalar(f.nU, offUb.as<int64_t>() + nv, st));
        int64_t nM = 0;
        HM_TRY(read_scalar(nM, moff.as<int64_t>() + nv, st));
        HM_TRY(alloc(f.U, std::max<int64_t>(f.nU, 1) * sizeof(double)));
        HM_CUDA(cudaMemsetAsync(c->GP.p, 0, (size_t)n * r * sizeof(double), st));
        k_pack_box<<<(unsigned)nv, 128, 0, st>>>(gb.pair_alpha.as<int>(), gb.pair_color.as<int>(), cu.ent.as<int>(),
                                                n, r, kUb.as<int>(), offUb.as<int64_t>(), c->cur.Y.as<double>(),
                                                f.U.as<double>(), c->GP.as<double>()); ::hm::count_launch();
        HM_LAUNCH("pack U");
        HM_TRY(alloc(M, std::max<int64_t>(nM, 1) * sizeof(double)));
        HM_TRY(make_mix(c, l, gb.pair_alpha.as<int>(), nv, kUb.as<int>(), moff.as<int64_t>(), M.as<double>()));
    }

    // ---- stage 2: Z = A^* Psi on the pair colouring, Psi filled with the bases
    c->peel_sides = 2;
    {
        Timer tm(st, phase_secs ? phase_secs + 2 : nullptr);
        e = sample_level(c, op, l, false);
    }
    if (!e) {
        Timer tm(st, phase_secs ? phase_secs + 3 : nullptr);
        e = peel_level(c, l, false);
    }
    c->peel_sides = 3;
    HM_TRY(e);
    Timer tb(st, phase_secs ? phase_secs + 4 : nullptr);
    // W_beta = sum of T_ab M_a (into Y's first colour block, free now; every
    // W tile is in colour 0), V = qr(W, k)
    double *W = c->cur.Y.as<double>();
    DBuf zero;
    HM_TRY(alloc(zero, nv * sizeof(int)));
    HM_CUDA(cudaMemsetAsync(zero.p, 0, nv * sizeof(int), st));
    k_mix_sum<<<(unsigned)nv, 128, 0, st>>>(gb.pair_alpha.as<int>(), nv, cu.ent.as<int>(), cu.int_ptr.as<int>(),
                                           cu.int_idx.as<int>(), gp.pair_color.as<int>(), vid.as<int>(),
                                           kUb.as<int>(), moff.as<int64_t>(), M.as<double>(), c->cur.Z.as<double>(),
                                           n, r, W); ::hm::count_launch();
    HM_LAUNCH("mix sum");
    HM_TRY(qr_tiles_fp64(c, l, gb.pair_alpha.as<int>(), zero.as<int>(), width.as<int>(), nv, cu.max_rows, W,
                         c->kcap, c->rank_fixed, c->tol, kVb.as<int>()));
    DBuf offVb;
    HM_TRY(alloc(offVb, (nv + 1) * sizeof(int64_t)));
    k_box_sizes<<<ceil_div(nv, 128), 128, 0, st>>>(gb.pair_alpha.as<int>(), nv, cu.ent.as<int>(), kVb.as<int>(), r,
                                                   sz.as<int64_t>(), nullptr); ::hm::count_launch();
    HM_TRY(scan_exclusive(sz.as<int64_t>(), offVb.as<int64_t>(), nv, st));
    HM_TRY(read_scalar(f.nV, offVb.as<int64_t>() + nv, st));
    HM_TRY(alloc(f.V, std::max<int64_t>(f.nV, 1) * sizeof(double)));
    k_pack_box<<<(unsigned)nv, 128, 0, st>>>(gb.pair_alpha.as<int>(), nullptr, cu.ent.as<int>(), n, r, kVb.as<int>(),
                                            offVb.as<int64_t>(), W, f.V.as<double>(), nullptr); ::hm::count_launch();
    HM_LAUNCH("pack V");
    HM_TRY(box_pairs_and_cores(c, l, vid.as<int>(), kUb.as<int>(), kVb.as<int>(), offUb.as<int64_t>(),
                               offVb.as<int64_t>()));
    f.done = true;
    return ok();
}

Err mix_sum(hm_ctx *c, int l, const int *vbox, int64_t nv, const int *vid, const int *kU, const int64_t *moff,
            const double *M, double *W) {
    if (nv == 0) return ok();
    const Cut &cu = c->cuts[l];
    un::k_mix_sum<<<(unsigned)nv, 128, 0, c->st>>>(vbox, nv, cu.ent.as<int>(), cu.int_ptr.as<int>(),
                                                   cu.int_idx.as<int>(), c->colorings[l].pair_color.as<int>(), vid,
                                                   kU, moff, M, c->cur.Z.as<double>(), c->n, c->cfg.r, W); ::hm::count_launch();
    HM_LAUNCH("mix sum");
    return ok();
}

Err box_pairs_and_cores(hm_ctx *c, int l, const int *vid, const int *kUb, const int *kVb, const int64_t *offUb,
                        const int64_t *offVb) {
    using namespace un;
    cudaStream_t st = c->st;
    const Coloring &gp = c->colorings[l];
    const Cut &cu = c->cuts[l];
    Factors &f = c->factors[l];
    const int64_t np = gp.n_pairs, n = c->n;
    const int r = c->cfg.r;
    HM_TRY(alloc(f.kU, np * sizeof(int)));
    HM_TRY(alloc(f.kV, np * sizeof(int)));
    HM_TRY(alloc(f.offU, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(f.offV, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(f.offB, (np + 1) * sizeof(int64_t)));
    DBuf szB;
    HM_TRY(alloc(szB, (np + 1) * sizeof(int64_t)));
    k_pair_factors<<<ceil_div(np, 256), 256, 0, st>>>(gp.pair_alpha.as<int>(), cu.int_idx.as<int>(), np, vid, kUb, kVb,
                                                      offUb, offVb, f.kU.as<int>(), f.kV.as<int>(),
                                                      f.offU.as<int64_t>(), f.offV.as<int64_t>(),
                                                      szB.as<int64_t>()); ::hm::count_launch();
    HM_LAUNCH("pair factors");
    HM_TRY(scan_exclusive(szB.as<int64_t>(), f.offB.as<int64_t>(), np, st));
    HM_TRY(read_scalar(f.nB, f.offB.as<int64_t>() + np, st));
    HM_TRY(alloc(f.B, std::max<int64_t>(f.nB, 1) * sizeof(double)));
    k_core_uniform<<<ceil_div(np * 32, 256), 256, 0, st>>>(np, cu.int_idx.as<int>(), gp.pair_T.as<int>(),
                                                           gp.pair_color.as<int>(), cu.ent.as<int>(), f.kU.as<int>(),
                                                           f.kV.as<int>(), f.offV.as<int64_t>(),
                                                           f.offB.as<int64_t>(), f.V.as<double>(),
                                                           c->cur.Z.as<double>(), n, r, f.B.as<double>()); ::hm::count_launch();
    HM_LAUNCH("core uniform");
    std::vector<int> hk;
    f.max_k = 0;
    HM_TRY(to_host(hk, f.kU.p, np, st));
    for (int v : hk) f.max_k = std::max(f.max_k, v);
    HM_TRY(to_host(hk, f.kV.p, np, st));
    for (int v : hk) f.max_k = std::max(f.max_k, v);
    return ok();
}

}  // namespace hm
