// Apply of the compressed operator (Section 4.1.2 level-truncated product, the
// apply timed in Section 5):  y = sum_l sum_(a,b) U B V^T x(I_b) + sum_near D x(I_b)
// and the adjoint.  Vectors are row-major [n][nrhs] in sorted order; the
// right-hand sides are processed in blocks of APPLY_NB (grid dimension y).
//
// Every factor is read once per block of right-hand sides, so the apply is
// bound by HBM bandwidth (8 bytes per stored factor entry):
//  stage 1 (k_ap1): one CTA per pair q of a level; its warps take the rows of
//           the pair's column box (adjoint: row box) in turn, each lane one
//           column of the factor (whole rows are read coalesced), the warps'
//           sums are added in warp order and t_q = B_q s (adjoint B_q^T s);
//           on cuts of boxes of at most AP1W_MAX_ROWS rows one warp per pair
//           does the same (k_ap1w), 8 pairs per CTA;
//  stage 2 (k_ap2): one CTA per APPLY_ROWS-row chunk of a box of the cut,
//           thread i owning row i; for every pair of the box the chunk's rows
//           of U_q (adjoint V) -- contiguous in the arena -- and t_q are
//           copied into shared memory with cp.async while the previous pair
//           multiplies; y(rows) += U_q(rows) t_q;
//  near    (k_apnear): the same shape over the leaf cut's neighbour blocks
//           D (adjoint D^T), in column chunks of APPLY_UC.
// Each output row belongs to one CTA per launch and the levels run in order,
// so the result is deterministic.  The metadata (t offsets, items) is built
// once after the compression (build_apply_plan).
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

namespace {

constexpr int AP1_BATCH = 8;  // rows a stage-1 warp reads before it multiplies
constexpr int AP1W_BATCH = 4;  // rows per warp load batch in the warp-per-pair kernel
constexpr int AP1W_MAX_ROWS = 512;  // cuts whose boxes are at most this long: one warp per pair

__device__ __forceinline__ void cp8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace

// stage 1: s = F_q^T x(I_box) (F = V, box = column box; adjoint F = U, row
// box), t_q = B_q s (adjoint B_q^T s), for the right-hand sides j0 .. j0+nb-1.
// Lanes are packed so that FP64 issue slots do useful work: with kp the
// smallest of 8, 16, 32, 64 not below kin, lane l takes column l % kp of rows
// l / kp (mod 32 / kp) of each group of rows (kp = 64: columns l and l + 32);
// AP1_BATCH groups are read before the products, so their loads overlap.
template <int NW, int NB>
__global__ void __launch_bounds__(NW * 32) k_ap1(ApplyLevel L, const double *x, int nrhs, int trans, double *t) {
    __shared__ double sp[NW][64][NB];
    __shared__ double ss[64][NB];
    const int64_t q = blockIdx.x;
    const int j0 = blockIdx.y * NB, nb = min(NB, nrhs - j0);
    const int ku = L.kU[q], kv = L.kV[q];
    if (ku == 0 || kv == 0) return;  // no t_q: stage 2 skips the pair too
    const int kin = trans ? ku : kv, kout = trans ? kv : ku;
    const int box = trans ? L.pair_alpha[q] : L.int_idx[q];
    const int *e = L.ent + (int64_t)box * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3];
    const double *F = trans ? L.U + L.offU[q] : L.V + L.offV[q];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kp = kin <= 8 ? 8 : (kin <= 16 ? 16 : (kin <= 32 ? 32 : 64));
    const int rpi = kp >= 32 ? 1 : 32 / kp;            // rows per warp instruction
    const int v = kp == 64 ? lane : lane % kp, rsub = kp >= 32 ? 0 : lane / kp;
    const bool c0 = v < kin, c1 = kp == 64 && lane + 32 < kin;
    double a0[NB], a1[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) a0[j] = a1[j] = 0.0;
    const int step = rpi * NW;  // rows per pass of all warps
    for (int g0 = w * rpi; g0 < m; g0 += AP1_BATCH * step) {
        double f0[AP1_BATCH], f1[AP1_BATCH], xv[AP1_BATCH][NB];
#pragma unroll
        for (int b = 0; b < AP1_BATCH; ++b) {
            const int i = g0 + b * step + rsub;
            const bool in = i < m;
            const double *Fr = F + (int64_t)i * kin;
            f0[b] = (in && c0) ? Fr[v] : 0.0;
            f1[b] = (in && c1) ? Fr[lane + 32] : 0.0;
#pragma unroll
            for (int j = 0; j < NB; ++j) xv[b][j] = (in && j < nb) ? x[(int64_t)(s0 + i) * nrhs + j0 + j] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < AP1_BATCH; ++b)
#pragma unroll
            for (int j = 0; j < NB; ++j) a0[j] = fma(f0[b], xv[b][j], a0[j]);
        if (kp == 64)
#pragma unroll
            for (int b = 0; b < AP1_BATCH; ++b)
#pragma unroll
                for (int j = 0; j < NB; ++j) a1[j] = fma(f1[b], xv[b][j], a1[j]);
    }
    // lanes holding the same column (rsub = 0 .. rpi-1) are added in rsub order
#pragma unroll
    for (int j = 0; j < NB; ++j)
        for (int o = kp; o < 32; o <<= 1) a0[j] += __shfl_down_sync(0xffffffffu, a0[j], o);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (rsub == 0 && c0) sp[w][v][j] = a0[j];
        if (c1) sp[w][lane + 32][j] = a1[j];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < kin * NB; o += NW * 32) {
        const int vv = o / NB, j = o % NB;
        double acc = 0.0;
        for (int ww = 0; ww < NW; ++ww) acc += sp[ww][vv][j];
        ss[vv][j] = acc;
    }
    __syncthreads();
    const double *Bq = L.B + L.offB[q];
    double *tq = t + (trans ? L.toffV[q] : L.toffU[q]) * nrhs;
    for (int o = threadIdx.x; o < kout * nb; o += NW * 32) {
        const int u = o / nb, j = o % nb;
        double acc = 0.0;
        for (int vv = 0; vv < kin; ++vv)
            acc = fma(trans ? Bq[(int64_t)vv * kout + u] : Bq[(int64_t)u * kin + vv], ss[vv][j], acc);
        tq[(int64_t)u * nrhs + j0 + j] = acc;
    }
}

// stage 1 for cuts of small boxes: one warp per pair (8 pairs per CTA), the
// same lane packing as k_ap1; the column sums are reduced with shuffles and
// t_q = B_q s (adjoint B_q^T s) is formed by the same warp, lane u (and u + 32)
// owning output u, with s broadcast from the lanes that hold it.
template <int NB>
__global__ void __launch_bounds__(256, 2) k_ap1w(ApplyLevel L, int64_t np, const double *x, int nrhs, int trans,
                                              double *t) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (q >= np) return;
    const int j0 = blockIdx.y * NB, nb = min(NB, nrhs - j0);
    const int ku = L.kU[q], kv = L.kV[q];
    if (ku == 0 || kv == 0) return;
    const int kin = trans ? ku : kv, kout = trans ? kv : ku;
    const int box = trans ? L.pair_alpha[q] : L.int_idx[q];
    const int *e = L.ent + (int64_t)box * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3];
    const double *F = trans ? L.U + L.offU[q] : L.V + L.offV[q];
    const int kp = kin <= 8 ? 8 : (kin <= 16 ? 16 : (kin <= 32 ? 32 : 64));
    const int rpi = kp >= 32 ? 1 : 32 / kp;
    const int v = kp == 64 ? lane : lane % kp, rsub = kp >= 32 ? 0 : lane / kp;
    const bool c0 = v < kin, c1 = kp == 64 && lane + 32 < kin;
    double a0[NB], a1[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) a0[j] = a1[j] = 0.0;
    for (int g0 = rsub; g0 < m; g0 += AP1W_BATCH * rpi) {
        double f0[AP1W_BATCH], f1[AP1W_BATCH], xv[AP1W_BATCH][NB];
#pragma unroll
        for (int b = 0; b < AP1W_BATCH; ++b) {
            const int i = g0 + b * rpi;
            const bool in = i < m;
            const double *Fr = F + (int64_t)i * kin;
            f0[b] = (in && c0) ? Fr[v] : 0.0;
            f1[b] = (in && c1) ? Fr[lane + 32] : 0.0;
#pragma unroll
            for (int j = 0; j < NB; ++j) xv[b][j] = (in && j < nb) ? x[(int64_t)(s0 + i) * nrhs + j0 + j] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < AP1W_BATCH; ++b)
#pragma unroll
            for (int j = 0; j < NB; ++j) a0[j] = fma(f0[b], xv[b][j], a0[j]);
        if (kp == 64)
#pragma unroll
            for (int b = 0; b < AP1W_BATCH; ++b)
#pragma unroll
                for (int j = 0; j < NB; ++j) a1[j] = fma(f1[b], xv[b][j], a1[j]);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        for (int o = kp; o < 32; o <<= 1) a0[j] += __shfl_down_sync(0xffffffffu, a0[j], o);
    // lane vv < kp holds s[vv] (and s[vv + 32] when kp == 64)
    const double *Bq = L.B + L.offB[q];
    double *tq = t + (trans ? L.toffV[q] : L.toffU[q]) * nrhs;
    double acc0[NB], acc1[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc0[j] = acc1[j] = 0.0;
    const int u0 = lane, u1 = lane + 32;
    for (int vv = 0; vv < kin; ++vv) {
        double sv[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) sv[j] = __shfl_sync(0xffffffffu, vv < 32 ? a0[j] : a1[j], vv & 31);
        if (u0 < kout) {
            const double bv = trans ? Bq[(int64_t)vv * kout + u0] : Bq[(int64_t)u0 * kin + vv];
#pragma unroll
            for (int j = 0; j < NB; ++j) acc0[j] = fma(bv, sv[j], acc0[j]);
        }
        if (u1 < kout) {
            const double bv = trans ? Bq[(int64_t)vv * kout + u1] : Bq[(int64_t)u1 * kin + vv];
#pragma unroll
            for (int j = 0; j < NB; ++j) acc1[j] = fma(bv, sv[j], acc1[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j >= nb) break;
        if (u0 < kout) tq[(int64_t)u0 * nrhs + j0 + j] = acc0[j];
        if (u1 < kout) tq[(int64_t)u1 * nrhs + j0 + j] = acc1[j];
    }
}

// Sources of stage 2: for entry tt of a box's list, the rank k of the block
// (0: skip), its rows r0.. (row-major, leading dimension k) and its t (k x
// nrhs, leading dimension nrhs).
struct FactorRows {  // admissible pairs of a level: U_q t_q (adjoint V_q of the transposed pair)
    ApplyLevel L;
    const double *t;
    int trans;
    __device__ int first(int box) const { return L.int_ptr[box]; }
    __device__ int last(int box) const { return L.int_ptr[box + 1]; }
    __device__ int rank(int tt) const {
        const int q = trans ? L.pairT[tt] : tt;
        return (L.kU[q] == 0 || L.kV[q] == 0) ? 0 : (trans ? L.kV[q] : L.kU[q]);
    }
    __device__ const double *rows(int tt, int r0, int k) const {
        const int q = trans ? L.pairT[tt] : tt;
        return (trans ? L.V + L.offV[q] : L.U + L.offU[q]) + (int64_t)r0 * k;
    }
    __device__ const double *tvec(int tt, int nrhs) const {
        const int q = trans ? L.pairT[tt] : tt;
        return t + (trans ? L.toffV[q] : L.toffU[q]) * nrhs;
    }
};
struct NearRows {  // leaf neighbour blocks, forward: D_ab x(I_b)
    const int *ent, *near_ptr, *near_idx;
    const int64_t *offD;
    const double *D, *x;
    __device__ int first(int box) const { return near_ptr[box]; }
    __device__ int last(int box) const { return near_ptr[box + 1]; }
    __device__ int rank(int tt) const {
        const int *eb = ent + (int64_t)near_idx[tt] * ENT_FIELDS;
        return eb[4] - eb[3];
    }
    __device__ const double *rows(int tt, int r0, int k) const { return D + offD[tt] + (int64_t)r0 * k; }
    __device__ const double *tvec(int tt, int nrhs) const {
        return x + (int64_t)ent[(int64_t)near_idx[tt] * ENT_FIELDS + 3] * nrhs;
    }
};

// stage 2: y(rows of the item) += sum over the box's list of F(rows) t, the
// next entry's rows and t copied into the other shared-memory stage with
// cp.async while the current one multiplies.  ld: row stride in shared memory
// (odd, >= every k); every k <= 64.  A chunk of at most 16 (32) rows gives
// each row 4 (2) threads, which take every 4th (2nd) column and are added by
// shuffles, so that FP64 issue slots do useful work on short boxes.
template <int NB, class Src>
__global__ void __launch_bounds__(APPLY_ROWS) k_ap2(Src S, const int *ent, const int *items, int nrhs, int ld,
                                                     double *y) {
    extern __shared__ __align__(16) double sm2[];
    const int item = blockIdx.x;
    const int j0 = blockIdx.y * NB, nb = min(NB, nrhs - j0);
    const int box = items[2 * item], r0 = items[2 * item + 1];
    const int *e = ent + (int64_t)box * ENT_FIELDS;
    const int bs = e[3], rows = min(APPLY_ROWS, e[4] - e[3] - r0);
    const int tid = threadIdx.x;
    const int spr = rows <= 16 ? 4 : (rows <= 32 ? 2 : 1);  // threads per row
    const int row = tid / spr, part = tid % spr;
    const int t0 = S.first(box), t1 = S.last(box);
    // stage b: rows at sm2 + b APPLY_ROWS ld, t at sm2 + 2 APPLY_ROWS ld + b 64 NB
    double *const sT0 = sm2 + 2 * APPLY_ROWS * ld;
    auto issue = [&](int tt, int b) -> int {
        const int k = S.rank(tt);
        if (k > 0) {
            const double *F = S.rows(tt, r0, k), *tq = S.tvec(tt, nrhs);
            double *sF = sm2 + b * APPLY_ROWS * ld, *sT = sT0 + b * 64 * NB;
            for (int o = tid; o < rows * k; o += APPLY_ROWS) {
                const int i = o / k, u = o - i * k;
                cp8(&sF[i * ld + u], F + o);
            }
            for (int o = tid; o < k * nb; o += APPLY_ROWS) {
                const int u = o / nb, j = o - u * nb;
                cp8(&sT[u * NB + j], tq + (int64_t)u * nrhs + j0 + j);
            }
        }
        cp_commit();  // one group per entry, empty or not
        return k;
    };
    double acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = 0.0;
    int kcur = t0 < t1 ? issue(t0, 0) : 0;
    for (int tt = t0; tt < t1; ++tt) {
        const int s = tt - t0;
        int knext = 0;
        if (tt + 1 < t1) {
            knext = issue(tt + 1, (s + 1) & 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        if (row < rows && kcur > 0) {
            const double *f = sm2 + (s & 1) * APPLY_ROWS * ld + row * ld, *tv = sT0 + (s & 1) * 64 * NB;
            for (int u = part; u < kcur; u += spr) {
                const double fu = f[u];
#pragma unroll
                for (int j = 0; j < NB; ++j) acc[j] = fma(fu, j < nb ? tv[u * NB + j] : 0.0, acc[j]);
            }
        }
        __syncthreads();
        kcur = knext;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        for (int o = 1; o < spr; o <<= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
    if (part == 0 && row < rows && t1 > t0)
        for (int j = 0; j < nb; ++j) y[(int64_t)(bs + r0 + row) * nrhs + j0 + j] += acc[j];
}

// near field: y(rows) += sum over neighbours b of D_ab(rows, :) x(I_b) (adjoint
// D_ba(:, rows)^T x(I_b)), the neighbour's points in chunks of APPLY_UC
template <int NB>
__global__ void __launch_bounds__(APPLY_ROWS) k_apnear(const int *ent, const int *items, const int *near_ptr,
                                                        const int *near_idx, const int *pairT, const int64_t *offD,
                                                        const double *D, const double *x, int nrhs, int trans,
                                                        double *y) {
    __shared__ double sD[APPLY_UC][APPLY_ROWS + 1];  // (column, row) of the block chunk
    __shared__ double sx[APPLY_UC][NB];
    const int item = blockIdx.x;
    const int j0 = blockIdx.y * NB, nb = min(NB, nrhs - j0);
    const int a = items[2 * item], r0 = items[2 * item + 1];
    const int *ea = ent + (int64_t)a * ENT_FIELDS;
    const int sa = ea[3], ma = ea[4] - ea[3], rows = min(APPLY_ROWS, ma - r0);
    const int tid = threadIdx.x;
    double acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = 0.0;
    for (int tt = near_ptr[a]; tt < near_ptr[a + 1]; ++tt) {
        const int b = near_idx[tt];
        const int *eb = ent + (int64_t)b * ENT_FIELDS;
        const int sb = eb[3], mb = eb[4] - eb[3];
        // forward: D_ab is ma x mb row-major; adjoint: D_ba is mb x ma row-major
        const double *Dp = D + offD[trans ? pairT[tt] : tt];
        for (int u0 = 0; u0 < mb; u0 += APPLY_UC) {
            const int uc = min(APPLY_UC, mb - u0);
            __syncthreads();
            if (!trans) {
                for (int o = tid; o < rows * uc; o += APPLY_ROWS) {
                    const int i = o / uc, u = o - i * uc;
                    sD[u][i] = Dp[(int64_t)(r0 + i) * mb + u0 + u];
                }
            } else {
                for (int o = tid; o < uc * rows; o += APPLY_ROWS) {
                    const int u = o / rows, i = o - u * rows;
                    sD[u][i] = Dp[(int64_t)(u0 + u) * ma + r0 + i];
                }
            }
            for (int o = tid; o < uc * nb; o += APPLY_ROWS) {
                const int u = o / nb, j = o - u * nb;
                sx[u][j] = x[(int64_t)(sb + u0 + u) * nrhs + j0 + j];
            }
            __syncthreads();
            if (tid < rows)
                for (int u = 0; u < uc; ++u) {
                    const double d = sD[u][tid];
#pragma unroll
                    for (int j = 0; j < NB; ++j) acc[j] = fma(d, j < nb ? sx[u][j] : 0.0, acc[j]);
                }
        }
    }
    if (tid < rows)
        for (int j = 0; j < nb; ++j) y[(int64_t)(sa + r0 + tid) * nrhs + j0 + j] += acc[j];
}

// --- metadata ---------------------------------------------------------------

__global__ void k_toff_sizes(const int *kU, const int *kV, int64_t np, int trans, int64_t *sz) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < np) sz[q] = (kU[q] > 0 && kV[q] > 0) ? (int64_t)(trans ? kV[q] : kU[q]) : 0;
}

__global__ void k_ap_item_count(const int *ent, int nc, int64_t *cnt) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nc) return;
    const int *e = ent + (int64_t)b * ENT_FIELDS;
    cnt[b] = (e[4] - e[3] + APPLY_ROWS - 1) / APPLY_ROWS;
}

__global__ void k_ap_item_fill(const int64_t *off, int nc, int *items) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nc) return;
    for (int64_t k = off[b]; k < off[b + 1]; ++k) {
        items[2 * k] = b;
        items[2 * k + 1] = (int)(k - off[b]) * APPLY_ROWS;
    }
}

Err build_apply_plan(hm_ctx *c) {
    cudaStream_t st = c->st;
    ApplyPlan &P = c->plan;
    P = ApplyPlan();
    const int nl = c->L + 1;
    P.toffU.resize(nl);
    P.toffV.resize(nl);
    P.items.resize(nl);
    P.nitems.assign(nl, 0);
    P.maxk.assign(nl, 0);
    for (int l = std::min(2, c->L); l <= c->L; ++l) {
        const Cut &cu = c->cuts[l];
        // items of cut l (the leaf cut's also serve the near field, whatever L is)
        DBuf cnt, off;
        HM_TRY(alloc(cnt, ((size_t)cu.nc + 1) * sizeof(int64_t)));
        HM_TRY(alloc(off, ((size_t)cu.nc + 1) * sizeof(int64_t)));
        k_ap_item_count<<<ceil_div(cu.nc, 256), 256, 0, st>>>(cu.ent.as<int>(), cu.nc, cnt.as<int64_t>()); ::hm::count_launch();
        HM_LAUNCH("ap_item_count");
        HM_TRY(scan_exclusive(cnt.as<int64_t>(), off.as<int64_t>(), cu.nc, st));
        HM_TRY(read_scalar(P.nitems[l], off.as<int64_t>() + cu.nc, st));
        if (P.nitems[l] >= (1ll << 31)) return fail(HM_ENOTSUP, "apply: too many row chunks in one cut");
        HM_TRY(alloc(P.items[l], std::max<int64_t>(P.nitems[l], 1) * 2 * sizeof(int)));
        k_ap_item_fill<<<ceil_div(cu.nc, 256), 256, 0, st>>>(off.as<int64_t>(), cu.nc, P.items[l].as<int>()); ::hm::count_launch();
        HM_LAUNCH("ap_item_fill");
        if (l < 2 || l >= (int)c->factors.size() || !c->factors[l].done || c->factors[l].n_pairs == 0) continue;
        const Factors &f = c->factors[l];
        const int64_t np = f.n_pairs;
        P.maxk[l] = f.max_k;
        for (int trans = 0; trans < 2; ++trans) {
            DBuf &to = trans ? P.toffV[l] : P.toffU[l];
            DBuf sz;
            HM_TRY(alloc(sz, (np + 1) * sizeof(int64_t)));
            HM_TRY(alloc(to, (np + 1) * sizeof(int64_t)));
            k_toff_sizes<<<ceil_div(np, 256), 256, 0, st>>>(f.kU.as<int>(), f.kV.as<int>(), np, trans, sz.as<int64_t>()); ::hm::count_launch();
            HM_LAUNCH("toff_sizes");
            HM_TRY(scan_exclusive(sz.as<int64_t>(), to.as<int64_t>(), np, st));
            int64_t tot = 0;
            HM_TRY(read_scalar(tot, to.as<int64_t>() + np, st));
            P.t_max = std::max(P.t_max, tot);
        }
    }
    P.ready = true;
    return ok();
}

// --- apply ------------------------------------------------------------------

// stage 1 (16 warps per pair where boxes are long, else 4) and stage 2 of one level
template <int NB>
static Err launch_level(const ApplyLevel &a, int max_rows, int64_t np, const int *items, int64_t nitems, int ld,
                        const double *x, int nrhs, int trans, double *t, double *y, cudaStream_t st) {
    const unsigned nblk = (unsigned)ceil_div(nrhs, NB);
    if (max_rows > 1024) k_ap1<16, NB><<<dim3((unsigned)np, nblk), 512, 0, st>>>(a, x, nrhs, trans, t);
    else if (max_rows > AP1W_MAX_ROWS) k_ap1<4, NB><<<dim3((unsigned)np, nblk), 128, 0, st>>>(a, x, nrhs, trans, t);
    else k_ap1w<NB><<<dim3((unsigned)ceil_div(np, 8), nblk), 256, 0, st>>>(a, np, x, nrhs, trans, t);
    ::hm::count_launch();
    HM_LAUNCH("apply stage 1");
    const size_t smem = (2 * (size_t)APPLY_ROWS * ld + 2 * 64 * NB) * sizeof(double);
    HM_TRY(allow_smem(k_ap2<NB, FactorRows>, smem));
    if (nitems > 0) {
        FactorRows src{a, t, trans};
        k_ap2<NB, FactorRows><<<dim3((unsigned)nitems, nblk), APPLY_ROWS, smem, st>>>(src, a.ent, items, nrhs, ld, y);
        ::hm::count_launch();
        HM_LAUNCH("apply stage 2");
    }
    return ok();
}

Err apply_near(hm_ctx *c, const double *x, double *y, int nrhs, int trans) {
    cudaStream_t st = c->st;
    const ApplyPlan &P = c->plan;
    const int nb = nrhs >= 4 ? 4 : nrhs;
    const Cut &cl = c->cuts[c->L];
    const Coloring &gl = c->colorings[c->L + 1];
    if (c->leaf.done && c->leaf.n_pairs > 0 && P.nitems[c->L] > 0) {
        const dim3 grid((unsigned)P.nitems[c->L], (unsigned)ceil_div(nrhs, nb));
        const int m_max = c->leaf.m_max;
        if (!trans && m_max <= 64) {  // forward: the rows of D_ab are contiguous, like a factor's
            NearRows src{cl.ent.as<int>(), cl.near_ptr.as<int>(), cl.near_idx.as<int>(), c->leaf.offD.as<int64_t>(),
                         c->leaf.D.as<double>(), x};
            const int ld = std::max(1, m_max) | 1;
#define NEARF(NBV)                                                                                                 \
    do {                                                                                                           \
        const size_t smem = (2 * (size_t)APPLY_ROWS * ld + 2 * 64 * NBV) * sizeof(double);                         \
        HM_TRY(allow_smem(k_ap2<NBV, NearRows>, smem));                                                             \
        k_ap2<NBV, NearRows><<<grid, APPLY_ROWS, smem, st>>>(src, cl.ent.as<int>(), P.items[c->L].as<int>(), nrhs,  \
                                                             ld, y);                                              \
    } while (0)
            if (nb == 1) NEARF(1);
            else if (nb == 2) NEARF(2);
            else NEARF(4);
#undef NEARF
        } else {  // adjoint (columns of D_ba) or leaves above 64 points
#define NEAR(NBV)                                                                                                  \
    k_apnear<NBV><<<grid, APPLY_ROWS, 0, st>>>(cl.ent.as<int>(), P.items[c->L].as<int>(), cl.near_ptr.as<int>(),    \
                                               cl.near_idx.as<int>(), gl.pair_T.as<int>(), c->leaf.offD.as<int64_t>(), \
                                               c->leaf.D.as<double>(), x, nrhs, trans, y)
            if (nb == 1) NEAR(1);
            else if (nb == 2) NEAR(2);
            else NEAR(4);
#undef NEAR
        }
        ::hm::count_launch();
        HM_LAUNCH("apply near field");
    }
    return ok();
}


Err apply_sorted_into(hm_ctx *c, const double *x, double *y, int nrhs, int trans, double *t) {
    cudaStream_t st = c->st;
    const ApplyPlan &P = c->plan;
    if (!P.ready) return fail(HM_ESTATE, "apply: no apply plan (compress first)");
    if (c->cfg.format == HM_FORMAT_H2) return apply_h2_into(c, x, y, nrhs, trans, t);
    const int nb = nrhs >= 4 ? 4 : nrhs;  // right-hand sides per CTA: 1, 2 or 4
    HM_CUDA(cudaMemsetAsync(y, 0, (size_t)c->n * nrhs * sizeof(double), st));
    for (int l = 2; l <= c->L; ++l) {
        if (l >= (int)c->factors.size() || !c->factors[l].done || c->factors[l].n_pairs == 0) continue;
        const Factors &f = c->factors[l];
        const Coloring &g = c->colorings[l];
        const Cut &cu = c->cuts[l];
        ApplyLevel a;
        a.ent = cu.ent.as<int>();
        a.int_ptr = cu.int_ptr.as<int>();
        a.int_idx = cu.int_idx.as<int>();
        a.pair_alpha = g.pair_alpha.as<int>();
        a.pairT = g.pair_T.as<int>();
        a.kU = f.kU.as<int>();
        a.kV = f.kV.as<int>();
        a.offU = f.offU.as<int64_t>();
        a.offV = f.offV.as<int64_t>();
        a.offB = f.offB.as<int64_t>();
        a.U = f.U.as<double>();
        a.V = f.V.as<double>();
        a.B = f.B.as<double>();
        a.toffU = P.toffU[l].as<int64_t>();
        a.toffV = P.toffV[l].as<int64_t>();
        if (f.max_k > 64) return fail(HM_ENOTSUP, "apply: rank above 64");
        const int ld = std::max(1, P.maxk[l]) | 1;
        switch (nb) {
        case 1: HM_TRY(launch_level<1>(a, cu.max_rows, f.n_pairs, P.items[l].as<int>(), P.nitems[l], ld, x, nrhs, trans, t, y, st)); break;
        case 2: HM_TRY(launch_level<2>(a, cu.max_rows, f.n_pairs, P.items[l].as<int>(), P.nitems[l], ld, x, nrhs, trans, t, y, st)); break;
        default: HM_TRY(launch_level<4>(a, cu.max_rows, f.n_pairs, P.items[l].as<int>(), P.nitems[l], ld, x, nrhs, trans, t, y, st));
        }
    }
    return apply_near(c, x, y, nrhs, trans);
}

Err apply_sorted(hm_ctx *c, const double *x, double *y, int nrhs, int trans) {
    const int64_t per = c->cfg.format == HM_FORMAT_H2 ? h2_scratch_elems(c) : c->plan.t_max;
    HM_TRY(ensure(c->apply_t, (size_t)std::max<int64_t>(per, 1) * nrhs * sizeof(double)));
    return apply_sorted_into(c, x, y, nrhs, trans, c->apply_t.as<double>());
}

}  // namespace hm
