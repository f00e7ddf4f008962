// Apply of the compressed operator (Section 4.1.2 level-truncated product, the
// apply timed in Section 5):  y = sum_l sum_(a,b) U B V^T x(I_b) + sum_near D x(I_b)
// and the adjoint.  Vectors are row-major [n][nrhs] in sorted order.
//
//  stage 1: t_q = B_q (V_q^T x(I_b)) for every admissible pair of every level
//           (adjoint: t_q = B_q^T (U_q^T x(I_a)));
//  stage 2: one CTA per leaf owns its rows: y(I_alpha) = sum over levels j of
//           U_q(rows of alpha) t_q for the pairs q of alpha's level-j ancestor,
//           plus the neighbour blocks.  No atomics; deterministic.
#include "apply_kernels.cuh"

#include <algorithm>

namespace hm {

__global__ void k_permute(const double *in, double *out, const int *perm, int64_t n, int nrhs, int to_sorted) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * nrhs) return;
    const int64_t i = t / nrhs;
    const int j = (int)(t - i * nrhs);
    if (to_sorted) out[t] = in[perm[i] + n * j];  // in: column-major original order
    else out[perm[i] + n * j] = in[t];
}

Err permute_rows(hm_ctx *c, const double *in, double *out, int nrhs, bool to_sorted) {
    k_permute<<<ceil_div(c->n * nrhs, 256), 256, 0, c->st>>>(in, out, c->perm.as<int>(), c->n, nrhs, to_sorted); ::hm::count_launch();
    HM_LAUNCH("permute");
    return ok();
}

// t_q (kout x nrhs) = B^(T) (F^T x(I_box))
__global__ void k_apply_stage1(const int *pair_alpha, const int *pair_col, const int *ent, int64_t np,
                               const int *kU, const int *kV, const int64_t *offU, const int64_t *offV,
                               const int64_t *offB, const double *U, const double *V, const double *B,
                               const double *x, int nrhs, int trans, const int64_t *toff, double *tq) {
    extern __shared__ double s1[];  // kin x nrhs
    const int64_t q = blockIdx.x;
    const int ku = kU[q], kv = kV[q];
    if (ku == 0 || kv == 0) return;
    const int kin = trans ? ku : kv, kout = trans ? kv : ku;
    const int box = trans ? pair_alpha[q] : pair_col[q];
    const int *e = ent + (int64_t)box * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3];
    const double *F = trans ? U + offU[q] : V + offV[q];
    for (int o = threadIdx.x; o < kin * nrhs; o += blockDim.x) {
        const int v = o / nrhs, j = o % nrhs;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(F[(int64_t)i * kin + v], x[(int64_t)(s0 + i) * nrhs + j], acc);
        s1[o] = acc;
    }
    __syncthreads();
    const double *Bq = B + offB[q];
    for (int o = threadIdx.x; o < kout * nrhs; o += blockDim.x) {
        const int u = o / nrhs, j = o % nrhs;
        double acc = 0.0;
        for (int v = 0; v < kin; ++v) {
            const double b = trans ? Bq[(int64_t)v * kout + u] : Bq[(int64_t)u * kin + v];
            acc = fma(b, s1[v * nrhs + j], acc);
        }
        tq[toff[q] + o] = acc;
    }
}

__global__ void k_apply_stage2(const int *ent_leaf, int nleaf, const ApplyLevel *lv, int nlev, const int *near_ptr,
                               const int *near_idx, const int *leaf_pairT, const int64_t *offD, const double *D,
                               const double *x, int nrhs, int trans, double *y) {
    const int a = blockIdx.x;
    const int *ea = ent_leaf + (int64_t)a * ENT_FIELDS;
    const int sa = ea[3], ma = ea[4] - ea[3];
    for (int o = threadIdx.x; o < ma * nrhs; o += blockDim.x) {
        const int i = o / nrhs, j = o % nrhs;
        double acc = 0.0;
        for (int l = 0; l < nlev; ++l) {
            const ApplyLevel &L = lv[l];
            const int anc = L.pt2ent[sa];
            const int as = L.ent[(int64_t)anc * ENT_FIELDS + 3];
            for (int t = L.int_ptr[anc]; t < L.int_ptr[anc + 1]; ++t) {
                const int q = trans ? L.pairT[t] : t;
                const int ku = L.kU[q], kv = L.kV[q];
                if (ku == 0 || kv == 0) continue;
                const int kk = trans ? kv : ku;
                const double *F = trans ? L.V + L.offV[q] : L.U + L.offU[q];
                const double *tv = L.tq + L.toff[q];
                const double *Fr = F + (int64_t)(sa - as + i) * kk;
                for (int u = 0; u < kk; ++u) acc = fma(Fr[u], tv[u * nrhs + j], acc);
            }
        }
        for (int t = near_ptr[a]; t < near_ptr[a + 1]; ++t) {
            const int b = near_idx[t];
            const int *eb = ent_leaf + (int64_t)b * ENT_FIELDS;
            const int sb = eb[3], mb = eb[4] - eb[3];
            if (!trans) {
                const double *Dp = D + offD[t];  // |I_a| x |I_b|
                for (int u = 0; u < mb; ++u) acc = fma(Dp[(int64_t)i * mb + u], x[(int64_t)(sb + u) * nrhs + j], acc);
            } else {
                const double *Dp = D + offD[leaf_pairT[t]];  // block (b, a): |I_b| x |I_a|
                for (int u = 0; u < mb; ++u) acc = fma(Dp[(int64_t)u * ma + i], x[(int64_t)(sb + u) * nrhs + j], acc);
            }
        }
        y[(int64_t)(sa + i) * nrhs + j] = acc;
    }
}

__global__ void k_toff_sizes(const int *kU, const int *kV, int64_t np, int nrhs, int trans, int64_t *sz) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < np) sz[q] = (int64_t)(trans ? kV[q] : kU[q]) * nrhs;
}

Err apply_sorted(hm_ctx *c, const double *x, double *y, int nrhs, int trans) {
    cudaStream_t st = c->st;
    std::vector<ApplyLevel> lv;
    std::vector<DBuf> tq(c->L + 1), toff(c->L + 1);
    for (int l = 2; l <= c->L; ++l) {
        if (l >= (int)c->factors.size() || !c->factors[l].done || c->factors[l].n_pairs == 0) continue;
        const Factors &f = c->factors[l];
        const Coloring &g = c->colorings[l];
        const Cut &cu = c->cuts[l];
        const int64_t np = f.n_pairs;
        DBuf sz;
        HM_TRY(alloc(sz, (np + 1) * sizeof(int64_t)));
        HM_TRY(alloc(toff[l], (np + 1) * sizeof(int64_t)));
        k_toff_sizes<<<ceil_div(np, 256), 256, 0, st>>>(f.kU.as<int>(), f.kV.as<int>(), np, nrhs, trans,
                                                        sz.as<int64_t>()); ::hm::count_launch();
        HM_TRY(scan_exclusive(sz.as<int64_t>(), toff[l].as<int64_t>(), np, st));
        int64_t tot = 0;
        HM_TRY(read_scalar(tot, toff[l].as<int64_t>() + np, st));
        HM_TRY(alloc(tq[l], std::max<int64_t>(tot, 1) * sizeof(double)));
        const size_t smem = (size_t)std::max(f.max_k, 1) * nrhs * sizeof(double);
        if (smem > 200 * 1024) return fail(HM_ENOTSUP, "apply: too many right-hand sides");
        HM_CUDA(cudaFuncSetAttribute(k_apply_stage1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        k_apply_stage1<<<(int)np, 128, smem, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(), cu.ent.as<int>(), np,
                                                   f.kU.as<int>(), f.kV.as<int>(), f.offU.as<int64_t>(),
                                                   f.offV.as<int64_t>(), f.offB.as<int64_t>(), f.U.as<double>(),
                                                   f.V.as<double>(), f.B.as<double>(), x, nrhs, trans,
                                                   toff[l].as<int64_t>(), tq[l].as<double>()); ::hm::count_launch();
        HM_LAUNCH("apply_stage1");
        ApplyLevel a;
        a.pt2ent = cu.pt2ent.as<int>();
        a.ent = cu.ent.as<int>();
        a.int_ptr = cu.int_ptr.as<int>();
        a.int_idx = cu.int_idx.as<int>();
        a.pairT = g.pair_T.as<int>();
        a.kU = f.kU.as<int>();
        a.kV = f.kV.as<int>();
        a.offU = f.offU.as<int64_t>();
        a.offV = f.offV.as<int64_t>();
        a.U = f.U.as<double>();
        a.V = f.V.as<double>();
        a.toff = toff[l].as<int64_t>();
        a.tq = tq[l].as<double>();
        lv.push_back(a);
    }
    DBuf lvd;
    HM_TRY(alloc(lvd, std::max<size_t>(lv.size(), 1) * sizeof(ApplyLevel)));
    if (!lv.empty())
        HM_CUDA(cudaMemcpyAsync(lvd.p, lv.data(), lv.size() * sizeof(ApplyLevel), cudaMemcpyHostToDevice, st));
    const Cut &cl = c->cuts[c->L];
    const Coloring &gl = c->colorings[c->L + 1];
    k_apply_stage2<<<cl.nc, 128, 0, st>>>(cl.ent.as<int>(), cl.nc, lvd.as<ApplyLevel>(), (int)lv.size(),
                                          cl.near_ptr.as<int>(), cl.near_idx.as<int>(), gl.pair_T.as<int>(),
                                          c->leaf.offD.as<int64_t>(), c->leaf.D.as<double>(), x, nrhs, trans, y); ::hm::count_launch();
    HM_LAUNCH("apply_stage2");
    HM_CUDA(cudaStreamSynchronize(st));
    return ok();
}

}  // namespace hm
