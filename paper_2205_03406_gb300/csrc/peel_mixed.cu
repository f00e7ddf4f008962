// Peeling for HM_MIXED_BF16X6_F32 (Section 4.1.2, Algorithm 4.1):
//     Y_l(I_alpha, c) -= sum over coarse pairs q of U_q(I_alpha) B_q V_q^T Omega_l(I_b, c)
// (and the transpose for Z).  The products of the coarse factors run in FP32
// from FP32 copies of U, V, B and of the level's Gaussians; the subtraction from
// the FP64 samples is FP64.  The FP32 products carry the same ~1e-7 relative
// rounding as the mixed-precision black-box samples they are subtracted from.
//
// For every coarse level j the subtraction splits into two products:
//   T_{q,c} = B_q W_{q,c},  W_{q,c} = sum over the level-l boxes gamma inside the
//   pair's other box that are active in colour c of X_{q,gamma} = F_q(I_gamma)^T G(I_gamma),
// computed ONCE per (coarse pair q, colour c) that some tile needs (k_peel_T),
// and the update of every tile (alpha, c) by sum over q of F'_q(I_alpha) T_{q,c},
// a register-tiled FP32 product over 64-row chunks (k_peel_gemm).  The (q, c)
// combinations a level needs are found through the (ancestor box A at level
// j, colour c) combinations of the tiles: the slots of T for (A, c) are
// contiguous, one per entry of A's interaction list, in list order.
//
// HM_MIXED_BF16X6 runs the same three products in double-float arithmetic
// (df.cuh: two FP32 words, about 48 significant bits, on the FP32 pipe, whose
// rate on this GPU is about 60 times the FP64 rate) from double-float copies of
// the factors and Gaussians, and subtracts the result from the FP64 samples in
// FP64.  Its update kernel (k_peel_gemm_df) reads compacted records of the live
// T slots (written by k_peel_T) and stages the next slot's F and T rows in
// shared memory with cp.async while the current one multiplies.  HM_FP64 runs
// the same compacted records and update kernel with FP64 elements.
#include "ctx.cuh"
#include "df.cuh"

#include <type_traits>

namespace hm {

namespace pm {

constexpr int WARPS = 4;  // warps per CTA

__global__ void k_to_f32(const double *in, float *out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

__global__ void k_to_df(const double *in, dfloat *out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = df_from(in[i]);
}

// a live T slot of (ancestor A, colour c) for the double-float update: the
// pair's factor offset in its arena, the first row of its T (kout rows of
// cols) in the compact T arena, and the rank of the factor
struct PeelRec {
    int64_t foff;
    int trow;
    int kout;
};

// size of the X block of each coarse pair: k x cols per level-l box inside its box
__global__ void k_xsize(const int *pair_alpha, const int *pair_col, int64_t np, const int *entj, const int *pt2ent_l,
                        const int *kdim, int cols, int side, int64_t *xsz) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= np) return;
    const int box = side ? pair_alpha[q] : pair_col[q];
    const int *e = entj + (int64_t)box * ENT_FIELDS;
    xsz[q] = (int64_t)(pt2ent_l[e[4] - 1] + 1 - pt2ent_l[e[3]]) * kdim[q] * cols;
}

// X_{q,gamma} (k x cols, type R): F_q(I_gamma)^T G(I_gamma), or the identity
// block's F rows at the leaf step; CTA (q, y) takes the gammas y, y + gridDim.y, ...
template <typename R>
__global__ void k_peel_xr(const int *pair_alpha, const int *pair_col, const int *entj, const int *entl,
                          const int *pt2ent_l, const int *kdim, const int64_t *offF, const R *F, const R *G,
                          int cols, int identity, int side, const int64_t *xoff, R *X) {
    const int64_t q = blockIdx.x;
    const int k = kdim[q];
    if (k == 0) return;
    const int box = side ? pair_alpha[q] : pair_col[q];
    const int *e = entj + (int64_t)box * ENT_FIELDS;
    const int bstart = e[3];
    const int kb = pt2ent_l[e[3]], ke = pt2ent_l[e[4] - 1] + 1;
    const R *Fq = F + offF[q];
    R *Xq = X + xoff[q];
    for (int g = kb + blockIdx.y; g < ke; g += gridDim.y) {
        const int *eg = entl + (int64_t)g * ENT_FIELDS;
        const int s0 = eg[3], len = eg[4] - eg[3];
        R *xg = Xq + (int64_t)(g - kb) * k * cols;
        for (int o = threadIdx.x; o < k * cols; o += blockDim.x) {
            const int v = o / cols, t = o % cols;
            R acc = R(0);
            if (identity) {
                acc = (t < len) ? Fq[(int64_t)(s0 - bstart + t) * k + v] : R(0);
            } else {
                for (int i = 0; i < len; ++i)
                    acc = mac(Fq[(int64_t)(s0 - bstart + i) * k + v], G[(int64_t)(s0 + i) * cols + t], acc);
            }
            xg[o] = acc;
        }
    }
}

template <typename R> struct CoarseT {
    const int *ent, *pt2ent, *int_ptr, *int_idx, *pairT;
    const int *kU, *kV;
    const int64_t *offU, *offV, *offB;
    const R *U, *V, *B;
    const int64_t *xoff;
    const R *X;
    const int64_t *base;        // [nc_j * chi + 1]: first T slot of (A, c)
    R *T;                       // [slots][kcap][cols]
    unsigned char *live;        // [slots]: T holds a nonzero product
};
using Coarse = CoarseT<float>;

__device__ __forceinline__ int lower_bound(const int *a, int lo, int hi, int key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// weight of (A, c): the length of A's interaction list if some tile (alpha, c)
// lies inside A (idempotent writes), else 0 from the memset
__global__ void k_anc_mark(const int *tile_alpha, const int *tile_color, int64_t ntiles, const int *entl,
                           const int *pt2ent_j, const int *int_ptr_j, int chi, int64_t *w) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= ntiles) return;
    const int A = pt2ent_j[entl[(int64_t)tile_alpha[p] * ENT_FIELDS + 3]];
    w[(int64_t)A * chi + tile_color[p]] = int_ptr_j[A + 1] - int_ptr_j[A];
}

// One warp per (A, c) combination of level j; for every entry t of A's
// interaction list: W = sum of X_{q,gamma} over the gammas of colour c in the
// other box, T[slot] = B W (Y side, B is kout x kin) or B^T W (Z side).
// With rec != nullptr (double-float mode) T is compact: only the live slots of
// (A, c) are stored, kout rows each from row trow[e] on, and the records
// rec[base[e] ..] (in list order) point at them; cnt[e] receives their number.
template <typename R>
__global__ void __launch_bounds__(WARPS * 32) k_peel_T(CoarseT<R> C, int64_t ncomb, int chi, int side, int cols,
                                                     int kcap, const int *pt2ent_l, const int *act_ptr,
                                                     const int *act_box, PeelRec *rec, int *cnt,
                                                     const int64_t *trow) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    R *sm = reinterpret_cast<R *>(sm_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * WARPS + warp;
    if (e >= ncomb) return;
    const int64_t s0 = C.base[e];
    if (C.base[e + 1] == s0) return;  // no tile needs (A, c)
    const int A = (int)(e / chi), c = (int)(e % chi);
    R *W = sm + (size_t)warp * kcap * cols;
    const int a0 = act_ptr[c], a1 = act_ptr[c + 1];
    const int t0 = C.int_ptr[A];
    int nlive = 0;
    int64_t row = rec ? trow[e] : 0;  // next free row of the compact T
    for (int t = t0; t < C.int_ptr[A + 1]; ++t) {
        const int64_t slot = s0 + (t - t0);
        const int q = side ? C.pairT[t] : t;
        const int kin = side ? C.kU[q] : C.kV[q];
        const int kout = side ? C.kV[q] : C.kU[q];
        int lo = 0, hi = 0;
        if (kin > 0 && kout > 0) {
            const int *eo = C.ent + (int64_t)C.int_idx[t] * ENT_FIELDS;
            const int kb = pt2ent_l[eo[3]], ke = pt2ent_l[eo[4] - 1] + 1;
            lo = lower_bound(act_box, a0, a1, kb);
            hi = lower_bound(act_box, lo, a1, ke);
            if (lo < hi) {
                const R *Xq = C.X + C.xoff[q];
                for (int o = lane; o < kin * cols; o += 32) {
                    R sacc = R(0);
                    for (int g = lo; g < hi; ++g) sacc = add(sacc, Xq[(int64_t)(act_box[g] - kb) * kin * cols + o]);
                    W[o] = sacc;
                }
                __syncwarp();
                const R *Bq = C.B + C.offB[q];
                R *To = rec ? C.T + row * cols : C.T + slot * kcap * cols;
                for (int o = lane; o < kout * cols; o += 32) {
                    const int u = o / cols, col = o % cols;
                    R sacc = R(0);
                    for (int v = 0; v < kin; ++v)
                        sacc = mac(side ? Bq[v * kout + u] : Bq[u * kin + v], W[v * cols + col], sacc);
                    To[o] = sacc;
                }
                __syncwarp();
            }
        }
        const bool live = kin > 0 && kout > 0 && lo < hi;  // the same in every lane
        if (lane == 0) {
            if (C.live) C.live[slot] = live ? 1 : 0;
            if (rec && live) rec[s0 + nlive] = PeelRec{side ? C.offV[q] : C.offU[q], (int)row, kout};
        }
        nlive += live ? 1 : 0;
        if (live) row += kout;
    }
    if (rec && lane == 0) cnt[e] = nlive;
}

// Size of the compact T of every (A, c) (double-float mode): the sum of kout
// over its live slots (the liveness rule of k_peel_T), one thread per (A, c).
template <typename R>
__global__ void k_peel_rows(CoarseT<R> C, int64_t ncomb, int chi, int side, const int *pt2ent_l,
                            const int *act_ptr, const int *act_box, int64_t *rows) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ncomb) return;
    int64_t tot = 0;
    if (C.base[e + 1] > C.base[e]) {
        const int A = (int)(e / chi), c = (int)(e % chi);
        const int a0 = act_ptr[c], a1 = act_ptr[c + 1];
        for (int t = C.int_ptr[A]; t < C.int_ptr[A + 1]; ++t) {
            const int q = side ? C.pairT[t] : t;
            const int kin = side ? C.kU[q] : C.kV[q], kout = side ? C.kV[q] : C.kU[q];
            if (kin == 0 || kout == 0) continue;
            const int *eo = C.ent + (int64_t)C.int_idx[t] * ENT_FIELDS;
            const int kb = pt2ent_l[eo[3]], ke = pt2ent_l[eo[4] - 1] + 1;
            const int lo = lower_bound(act_box, a0, a1, kb);
            if (lo < a1 && act_box[lo] < ke) tot += kout;
        }
    }
    rows[e] = tot;
}

// work items of the update: chunks of gr rows of every tile
__global__ void k_item_count(const int *tile_alpha, const int *entl, int64_t ntiles, int gr, int64_t *cnt) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= ntiles) return;
    const int *e = entl + (int64_t)tile_alpha[p] * ENT_FIELDS;
    cnt[p] = (e[4] - e[3] + gr - 1) / gr;
}

__global__ void k_item_fill(const int64_t *off, int64_t ntiles, int gr, int64_t *item_tile, int *item_row) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= ntiles) return;
    for (int64_t k = off[p]; k < off[p + 1]; ++k) {
        item_tile[k] = p;
        item_row[k] = (int)(k - off[p]) * gr;
    }
}

// One CTA of 128 threads per 64-row chunk of a tile (alpha, c): for every
// coarse level and every entry of the ancestor's interaction list with a live
// T slot, acc += F'(rows, 0:kout) T (kout x cols), staged through shared
// memory (F' transposed, leading dimension 68); thread (rg, cg) owns rows
// 4rg..4rg+3 and columns cg*CW..cg*CW+CW-1 (CW = MAXC / 8).  At the end the
// FP64 tile -= acc.  MAXC (32 or 64) bounds the columns, KMAX = 64 the ranks.
constexpr int GEMM_ROWS = 64, GEMM_LDF = 68, KMAX = 64;

template <int MAXC>
__global__ void __launch_bounds__(128) k_peel_gemm(const Coarse *cl, int ncl, int side, int chi,
                                                   const int *tile_alpha, const int *tile_color, const int *entl,
                                                   const int64_t *item_tile, const int *item_row, int64_t nitems,
                                                   int cols, int kcap, int64_t n, double *OUT) {
    constexpr int CW = MAXC / 8;
    __shared__ __align__(16) float Fs[KMAX * GEMM_LDF];
    __shared__ __align__(16) float Ts[KMAX * MAXC];
    const int64_t item = blockIdx.x;
    if (item >= nitems) return;
    const int tid = threadIdx.x, rg = tid >> 3, cg = tid & 7;
    const int64_t p = item_tile[item];
    const int alpha = tile_alpha[p], c = tile_color[p];
    const int *ea = entl + (int64_t)alpha * ENT_FIELDS;
    const int sa = ea[3] + item_row[item];
    const int rows = min(GEMM_ROWS, ea[4] - sa);
    float acc[4][CW];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[i][j] = 0.0f;
    for (int lvl = 0; lvl < ncl; ++lvl) {
        const Coarse &C = cl[lvl];
        const int A = C.pt2ent[sa];
        const int anc_start = C.ent[(int64_t)A * ENT_FIELDS + 3];
        const int t0 = C.int_ptr[A], t1 = C.int_ptr[A + 1];
        const int64_t s0 = C.base[(int64_t)A * chi + c];
        for (int t = t0; t < t1; ++t) {
            const int64_t slot = s0 + (t - t0);
            if (!C.live[slot]) continue;  // uniform over the CTA
            const int q = side ? C.pairT[t] : t;
            const int kout = side ? C.kV[q] : C.kU[q];
            const float *F = (side ? C.V + C.offV[q] : C.U + C.offU[q]) + (int64_t)(sa - anc_start) * kout;
            const float *Tq = C.T + slot * kcap * cols;
            __syncthreads();  // the previous step's reads of Fs / Ts are done
            for (int o = tid; o < GEMM_ROWS * kout; o += 128) {
                const int row = o / kout, u = o % kout;
                Fs[u * GEMM_LDF + row] = row < rows ? F[o] : 0.0f;
            }
            for (int o = tid; o < kout * cols; o += 128) Ts[(o / cols) * MAXC + o % cols] = Tq[o];
            if (cols < MAXC)
                for (int o = tid; o < kout * (MAXC - cols); o += 128)
                    Ts[(o / (MAXC - cols)) * MAXC + cols + o % (MAXC - cols)] = 0.0f;
            __syncthreads();
            for (int u = 0; u < kout; ++u) {
                const float4 f = *reinterpret_cast<const float4 *>(&Fs[u * GEMM_LDF + rg * 4]);
                float tv[CW];
#pragma unroll
                for (int j4 = 0; j4 < CW / 4; ++j4) {
                    const float4 x = *reinterpret_cast<const float4 *>(&Ts[u * MAXC + cg * CW + 4 * j4]);
                    tv[4 * j4] = x.x;
                    tv[4 * j4 + 1] = x.y;
                    tv[4 * j4 + 2] = x.z;
                    tv[4 * j4 + 3] = x.w;
                }
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    acc[0][j] = fmaf(f.x, tv[j], acc[0][j]);
                    acc[1][j] = fmaf(f.y, tv[j], acc[1][j]);
                    acc[2][j] = fmaf(f.z, tv[j], acc[2][j]);
                    acc[3][j] = fmaf(f.w, tv[j], acc[3][j]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = rg * 4 + i;
        if (row >= rows) continue;
        double *out = OUT + ((int64_t)c * n + sa + row) * cols;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const int col = cg * CW + j;
            if (col < cols) out[col] -= (double)acc[i][j];
        }
    }
}

// rows per work item of the compact update, and the leading dimension of its
// staged F' rows
constexpr int GEMM64_ROWS = 32, GEMM64_LDF = 36;

// ---------------------------------------------------------------------------
// Compact update: double-float elements (HM_MIXED_BF16X6) or FP64 elements
// (HM_FP64), E.  One CTA of 128 threads per 32-row
// chunk of a tile (alpha, c): the steps are the live T slots of the chunk's
// ancestors at every coarse level (the records k_peel_T compacted), each a
// product F'(rows, 0:kout) T (kout x cols).  Step s + 1's F rows (row-major, a
// flat copy) and T are copied into the other shared-memory stage with
// cp.async while step s multiplies; thread (rg, cg) owns rows 4 rg .. 4 rg + 3 and columns
// cg CW .. cg CW + CW - 1 (CW = MAXC / 16) in accumulators of type E, and the
// FP64 tile -= the accumulated value at the end.  macs (optional) receives the
// multiply-adds of the valid rows and columns.
// ---------------------------------------------------------------------------

template <typename E> struct CoarseC {
    const int *ent, *pt2ent;
    const int64_t *base;   // [nc_j * chi + 1]: first record of (A, c)
    const int *cnt;        // [nc_j * chi]: live records of (A, c)
    const PeelRec *rec;
    const E *F;            // U (Y side) or V (Z side) arena
    const E *T;            // compact T rows
};
using CoarseDF = CoarseC<dfloat>;

constexpr int DF_MAXLV = MAX_LEVELS;

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int MAXC, typename E>
__global__ void __launch_bounds__(128) k_peel_gemm_df(const CoarseC<E> *cl, int ncl, int chi, const int *tile_alpha,
                                                      const int *tile_color, const int *entl, const int64_t *item_tile,
                                                      const int *item_row, int64_t nitems, int cols, int kcap,
                                                      int64_t n, double *OUT, unsigned long long *macs) {
    constexpr int CW = MAXC / 16;
    constexpr int LDF = GEMM64_LDF;
    extern __shared__ __align__(16) unsigned char smdf_raw[];
    E *Fs = reinterpret_cast<E *>(smdf_raw);  // [2][kcap][LDF]: F' transposed
    E *Ts = Fs + 2 * kcap * LDF;               // [2][kcap][MAXC]
    __shared__ int lv_first[DF_MAXLV + 1], lv_n[DF_MAXLV], lv_rowoff[DF_MAXLV];
    __shared__ int64_t lv_s0[DF_MAXLV];
    const int64_t item = blockIdx.x;
    if (item >= nitems) return;
    const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
    const int64_t p = item_tile[item];
    const int alpha = tile_alpha[p], c = tile_color[p];
    const int *ea = entl + (int64_t)alpha * ENT_FIELDS;
    const int sa = ea[3] + item_row[item];
    const int rows = min(GEMM64_ROWS, ea[4] - sa);
    if (tid < ncl) {  // ancestor of the chunk at coarse level tid: its records
        const CoarseC<E> &C = cl[tid];
        const int A = C.pt2ent[sa];
        const int64_t e = (int64_t)A * chi + c;
        lv_s0[tid] = C.base[e];
        lv_n[tid] = C.cnt[e];
        lv_rowoff[tid] = sa - C.ent[(int64_t)A * ENT_FIELDS + 3];
    }
    __syncthreads();
    if (tid == 0) {
        lv_first[0] = 0;
        for (int l = 0; l < ncl; ++l) lv_first[l + 1] = lv_first[l] + lv_n[l];
    }
    __syncthreads();
    const int S = lv_first[ncl];
    // stage the F rows (row-major, leading dimension kout: one flat copy) and
    // T of step s into buffer b; returns the step's rank
    auto issue = [&](int s, int b) -> int {
        int lv = 0;
        while (s >= lv_first[lv + 1]) ++lv;
        const CoarseC<E> &C = cl[lv];
        const PeelRec rc = C.rec[lv_s0[lv] + (s - lv_first[lv])];
        const int kout = rc.kout;
        const E *F = C.F + rc.foff + (int64_t)lv_rowoff[lv] * kout;
        const E *T = C.T + (int64_t)rc.trow * cols;
        E *fs = Fs + b * kcap * LDF, *ts = Ts + b * kcap * MAXC;
        const int nf = rows * kout;
        for (int o = tid; o < GEMM64_ROWS * kout; o += 128) {
            if (o < nf) cp_async8(&fs[o], F + o);
            else fs[o] = E(0);
        }
        for (int o = tid; o < kout * MAXC; o += 128) {
            const int u = o / MAXC, col = o - u * MAXC;
            if (col < cols) cp_async8(&ts[o], T + (int64_t)u * cols + col);
            else ts[o] = E(0);
        }
        cp_async_commit();
        return kout;
    };
    E acc[4][CW];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[i][j] = E(0);
    unsigned long long nmac = 0;
    int kcur = S > 0 ? issue(0, 0) : 0;
    for (int s = 0; s < S; ++s) {
        int knext = 0;
        if (s + 1 < S) {
            knext = issue(s + 1, (s + 1) & 1);  // that stage was last read in step s - 1
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const E *fs = Fs + (s & 1) * kcap * LDF + rg * 4 * kcur, *ts = Ts + (s & 1) * kcap * MAXC;
        // warps whose rows all lie past the chunk's last row skip the products
        for (int u = 0; u < (rg * 4 < rows ? kcur : 0); ++u) {
            const E fv[4] = {fs[u], fs[kcur + u], fs[2 * kcur + u], fs[3 * kcur + u]};
            E tv[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) tv[j] = ts[u * MAXC + cg * CW + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < CW; ++j) acc[i][j] = mac(fv[i], tv[j], acc[i][j]);
        }
        nmac += (unsigned long long)rows * kcur * cols;
        __syncthreads();  // stage s & 1 is refilled in step s + 1
        kcur = knext;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = rg * 4 + i;
        if (row >= rows) continue;
        double *out = OUT + ((int64_t)c * n + sa + row) * cols;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            const int col = cg * CW + j;
            if (col < cols) out[col] -= widen(acc[i][j], 0.0);
        }
    }
    if (macs && tid == 0 && nmac) atomicAdd(macs, nmac);
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

static Err df_copy(DBuf &dst, const DBuf &src, int64_t count, cudaStream_t st) {
    HM_TRY(alloc(dst, std::max<int64_t>(count, 1) * sizeof(dfloat)));
    if (count > 0) {
        pm::k_to_df<<<ceil_div(count, 256), 256, 0, st>>>(src.as<double>(), dst.as<dfloat>(), count);
        count_launch();
        HM_LAUNCH("to_df");
    }
    return ok();
}

// double-float copies of a level's factors, made once when a finer level first peels it
static Err factors_df(Factors &f, cudaStream_t st) {
    if (f.U2.p) return ok();
    HM_TRY(df_copy(f.U2, f.U, f.nU, st));
    HM_TRY(df_copy(f.V2, f.V, f.nV, st));
    HM_TRY(df_copy(f.B2, f.B, f.nB, st));
    return ok();
}

// the double-float update of one side, timed by CUDA events (hm_info.seconds_peel_update)
// the compact update (double-float, or FP64 in the FP64 mode), timed by CUDA
// events and counting its multiply-adds
template <typename E>
static Err launch_update_c(hm_ctx *c, const pm::CoarseC<E> *tab, int ntab, int chi, const Coloring &g, const Cut &cl,
                           const DBuf &item_tile, const DBuf &item_row, int64_t nitems, int cols, int r, double *OUT) {
    cudaStream_t st = c->st;
    const int maxc = cols <= 32 ? 32 : 64;
    const size_t smem = 2 * (size_t)r * (pm::GEMM64_LDF + maxc) * sizeof(E);
    if (smem > 220 * 1024) return fail(HM_ENOTSUP, "peel: r x columns per colour too large");
    HM_TRY(ensure(c->peel_macs, sizeof(unsigned long long)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HM_CUDA(cudaEventCreate(&e0));
    HM_CUDA(cudaEventCreate(&e1));
    c->ev_update.push_back({e0, e1});
    HM_CUDA(cudaEventRecord(e0, st));
    auto *macs = c->peel_macs.as<unsigned long long>();
    if (maxc == 32) {
        HM_TRY(allow_smem(pm::k_peel_gemm_df<32, E>, smem));
        pm::k_peel_gemm_df<32, E><<<(unsigned)nitems, 128, smem, st>>>(
            tab, ntab, chi, g.pair_alpha.as<int>(), g.pair_color.as<int>(), cl.ent.as<int>(), item_tile.as<int64_t>(),
            item_row.as<int>(), nitems, cols, r, c->n, OUT, macs);
    } else {
        HM_TRY(allow_smem(pm::k_peel_gemm_df<64, E>, smem));
        pm::k_peel_gemm_df<64, E><<<(unsigned)nitems, 128, smem, st>>>(
            tab, ntab, chi, g.pair_alpha.as<int>(), g.pair_color.as<int>(), cl.ent.as<int>(), item_tile.as<int64_t>(),
            item_row.as<int>(), nitems, cols, r, c->n, OUT, macs);
    }
    count_launch();
    HM_LAUNCH("peel_gemm_compact");
    HM_CUDA(cudaEventRecord(e1, st));
    return ok();
}

static Err launch_update(const pm::CoarseT<float> *tab, int ntab, int side, int chi, const Coloring &g,
                         const Cut &cl, const DBuf &item_tile, const DBuf &item_row, int64_t nitems, int cols, int r,
                         int64_t n, double *OUT, cudaStream_t st) {
    if (cols <= 32)
        pm::k_peel_gemm<32><<<(unsigned)nitems, 128, 0, st>>>(tab, ntab, side, chi, g.pair_alpha.as<int>(),
                                                              g.pair_color.as<int>(), cl.ent.as<int>(),
                                                              item_tile.as<int64_t>(), item_row.as<int>(), nitems,
                                                              cols, r, n, OUT);
    else
        pm::k_peel_gemm<64><<<(unsigned)nitems, 128, 0, st>>>(tab, ntab, side, chi, g.pair_alpha.as<int>(),
                                                              g.pair_color.as<int>(), cl.ent.as<int>(),
                                                              item_tile.as<int64_t>(), item_row.as<int>(), nitems,
                                                              cols, r, n, OUT);
    count_launch();
    HM_LAUNCH("peel_gemm");
    return ok();
}

// the factors and Gaussians the peel of type R reads: FP32 copies for float,
// the FP64 arrays themselves for double
template <typename R> struct PeelData;
template <> struct PeelData<float> {
    static Err factors(Factors &f, cudaStream_t st) { return factors_f32(f, st); }
    static const float *U(const Factors &f) { return f.U32.as<float>(); }
    static const float *V(const Factors &f) { return f.V32.as<float>(); }
    static const float *B(const Factors &f) { return f.B32.as<float>(); }
    static Err gauss(hm_ctx *c, DBuf *G32, const float **G) {
        HM_TRY(f32_copy(G32[0], c->GO, c->n * c->cfg.r, c->st));
        HM_TRY(f32_copy(G32[1], c->GP, c->n * c->cfg.r, c->st));
        G[0] = G32[0].as<float>();
        G[1] = G32[1].as<float>();
        return ok();
    }
    static constexpr int rows = 64;  // rows per update chunk
};
template <> struct PeelData<double> {
    static Err factors(Factors &, cudaStream_t) { return ok(); }
    static const double *U(const Factors &f) { return f.U.as<double>(); }
    static const double *V(const Factors &f) { return f.V.as<double>(); }
    static const double *B(const Factors &f) { return f.B.as<double>(); }
    static Err gauss(hm_ctx *c, DBuf *, const double **G) {
        G[0] = c->GO.as<double>();
        G[1] = c->GP.as<double>();
        return ok();
    }
    static constexpr int rows = pm::GEMM64_ROWS;
};

template <> struct PeelData<dfloat> {
    static Err factors(Factors &f, cudaStream_t st) { return factors_df(f, st); }
    static const dfloat *U(const Factors &f) { return f.U2.as<dfloat>(); }
    static const dfloat *V(const Factors &f) { return f.V2.as<dfloat>(); }
    static const dfloat *B(const Factors &f) { return f.B2.as<dfloat>(); }
    static Err gauss(hm_ctx *c, DBuf *G2, const dfloat **G) {
        HM_TRY(df_copy(G2[0], c->GO, c->n * c->cfg.r, c->st));
        HM_TRY(df_copy(G2[1], c->GP, c->n * c->cfg.r, c->st));
        G[0] = G2[0].as<dfloat>();
        G[1] = G2[1].as<dfloat>();
        return ok();
    }
    static constexpr int rows = pm::GEMM64_ROWS;
};

template <typename R> static Err peel_level_t(hm_ctx *c, int level, bool leaf) {
    using PD = PeelData<R>;
    // compacted T records and the record-driven update: double-float (spec
    // precision) and FP64; the FP32-solve mode keeps the dense slot table
    constexpr bool kDF = std::is_same<R, dfloat>::value || std::is_same<R, double>::value;
    const int l = leaf ? c->L : level;
    const int idx = leaf ? c->L + 1 : level;
    const Coloring &g = (!leaf && c->cur_tiles) ? *c->cur_tiles : c->colorings[idx];
    if (g.n_pairs == 0 || g.n_colors == 0) return ok();
    const int cols = g.m_cols;
    const int jmax = leaf ? c->L : level - 1;
    const Cut &cl = c->cuts[l];
    cudaStream_t st = c->st;
    const int r = c->cfg.r;
    const int64_t n = c->n;
    // Gaussians of this level (not used at the leaf: identity test matrices)
    DBuf G32[2];
    const R *Gl[2] = {nullptr, nullptr};
    if (!leaf) HM_TRY(PD::gauss(c, G32, Gl));
    // work items: chunks of PD::rows rows of every tile
    const int64_t ntiles = g.n_pairs;
    const int chi = g.n_colors;
    DBuf cnt, off, item_tile, item_row;
    HM_TRY(alloc(cnt, (ntiles + 1) * sizeof(int64_t)));
    HM_TRY(alloc(off, (ntiles + 1) * sizeof(int64_t)));
    pm::k_item_count<<<ceil_div(ntiles, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), cl.ent.as<int>(), ntiles,
                                                            PD::rows, cnt.as<int64_t>());
    count_launch();
    HM_LAUNCH("item_count");
    HM_TRY(scan_exclusive(cnt.as<int64_t>(), off.as<int64_t>(), ntiles, st));
    int64_t nitems = 0;
    HM_TRY(read_scalar(nitems, off.as<int64_t>() + ntiles, st));
    HM_TRY(alloc(item_tile, nitems * sizeof(int64_t)));
    HM_TRY(alloc(item_row, nitems * sizeof(int)));
    pm::k_item_fill<<<ceil_div(ntiles, 256), 256, 0, st>>>(off.as<int64_t>(), ntiles, PD::rows,
                                                           item_tile.as<int64_t>(), item_row.as<int>());
    count_launch();
    HM_LAUNCH("item_fill");

    // coarse levels with factors, and their (ancestor, colour) slot tables
    // (the same for both sides)
    std::vector<int> js;
    for (int j = 2; j <= jmax; ++j)
        if (j < (int)c->factors.size() && c->factors[j].done && c->factors[j].n_pairs > 0) js.push_back(j);
    if (js.empty()) return ok();
    std::vector<DBuf> bases(js.size());
    std::vector<int64_t> nslots(js.size(), 0);
    for (size_t i = 0; i < js.size(); ++i) {
        const Cut &cj = c->cuts[js[i]];
        const int64_t ncomb = (int64_t)cj.nc * chi;
        DBuf w;
        HM_TRY(alloc(w, (ncomb + 1) * sizeof(int64_t)));
        HM_CUDA(cudaMemsetAsync(w.p, 0, (ncomb + 1) * sizeof(int64_t), st));
        pm::k_anc_mark<<<ceil_div(ntiles, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), g.pair_color.as<int>(), ntiles,
                                                              cl.ent.as<int>(), cj.pt2ent.as<int>(),
                                                              cj.int_ptr.as<int>(), chi, w.as<int64_t>());
        count_launch();
        HM_LAUNCH("anc_mark");
        HM_TRY(alloc(bases[i], (ncomb + 1) * sizeof(int64_t)));
        HM_TRY(scan_exclusive(w.as<int64_t>(), bases[i].as<int64_t>(), ncomb, st));
        HM_TRY(read_scalar(nslots[i], bases[i].as<int64_t>() + ncomb, st));
    }

    for (int side = 0; side < (leaf ? 1 : 2); ++side) {
        if (!leaf && !(c->peel_sides & (1 << side))) continue;  // uniform H^1 peels one side per stage
        std::vector<pm::CoarseT<R>> tab;
        std::vector<pm::CoarseC<R>> dtab;
        std::vector<DBuf> keep;  // X, offsets, T, live flags and records of every coarse level
        for (size_t i = 0; i < js.size(); ++i) {
            const int j = js[i];
            Factors &f = c->factors[j];
            const Coloring &gj = c->colorings[j];
            const Cut &cj = c->cuts[j];
            const int64_t np = f.n_pairs;
            HM_TRY(PD::factors(f, st));
            DBuf xsz, xo, X, T, live;
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
            HM_TRY(alloc(X, std::max<int64_t>(xtot, 1) * sizeof(R)));
            // CTAs per coarse pair: about one per level-l box inside the largest coarse box
            const int gy = std::min(256, std::max(1, cj.max_rows / std::max(1, std::min(cl.max_rows, 64))));
            pm::k_peel_xr<R><<<dim3((unsigned)np, gy), 128, 0, st>>>(
                gj.pair_alpha.as<int>(), cj.int_idx.as<int>(), cj.ent.as<int>(), cl.ent.as<int>(),
                cl.pt2ent.as<int>(), kdim, side ? f.offU.as<int64_t>() : f.offV.as<int64_t>(),
                side ? PD::U(f) : PD::V(f), leaf ? nullptr : Gl[side], cols, leaf ? 1 : 0, side, xo.as<int64_t>(),
                X.as<R>());
            count_launch();
            HM_LAUNCH("peel_x");
            pm::CoarseT<R> co;
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
            co.U = PD::U(f);
            co.V = PD::V(f);
            co.B = PD::B(f);
            co.xoff = xo.as<int64_t>();
            co.X = X.as<R>();
            co.base = bases[i].as<int64_t>();
            co.live = nullptr;
            const int64_t ncomb = (int64_t)cj.nc * chi;
            DBuf recb, cntb, trow;
            if (kDF) {
                // compact T: kout rows per live slot only
                if (nslots[i] >= (1ll << 31)) return fail(HM_ENOTSUP, "peel: more than 2^31 T slots in one level");
                DBuf rows;
                HM_TRY(alloc(rows, (ncomb + 1) * sizeof(int64_t)));
                HM_TRY(alloc(trow, (ncomb + 1) * sizeof(int64_t)));
                pm::k_peel_rows<R><<<ceil_div(ncomb, 128), 128, 0, st>>>(co, ncomb, chi, side, cl.pt2ent.as<int>(),
                                                                          g.act_ptr.as<int>(), g.act_box.as<int>(),
                                                                          rows.as<int64_t>());
                count_launch();
                HM_LAUNCH("peel_rows");
                HM_TRY(scan_exclusive(rows.as<int64_t>(), trow.as<int64_t>(), ncomb, st));
                int64_t trows = 0;
                HM_TRY(read_scalar(trows, trow.as<int64_t>() + ncomb, st));
                if (trows >= (1ll << 31)) return fail(HM_ENOTSUP, "peel: more than 2^31 rows of T in one level");
                HM_TRY(alloc(T, std::max<int64_t>(trows, 1) * cols * sizeof(R)));
                HM_TRY(alloc(recb, std::max<int64_t>(nslots[i], 1) * sizeof(pm::PeelRec)));
                HM_TRY(alloc(cntb, std::max<int64_t>(ncomb, 1) * sizeof(int)));
                HM_CUDA(cudaMemsetAsync(cntb.p, 0, std::max<int64_t>(ncomb, 1) * sizeof(int), st));
            } else {
                HM_TRY(alloc(T, std::max<int64_t>(nslots[i], 1) * r * cols * sizeof(R)));
                HM_TRY(alloc(live, std::max<int64_t>(nslots[i], 1)));
                co.live = live.as<unsigned char>();
            }
            co.T = T.as<R>();
            if (nslots[i] > 0) {
                const size_t smem = (size_t)pm::WARPS * r * cols * sizeof(R);
                HM_TRY(allow_smem(pm::k_peel_T<R>, (size_t)((int)smem)));
                pm::k_peel_T<R><<<ceil_div(ncomb, pm::WARPS), pm::WARPS * 32, smem, st>>>(
                    co, ncomb, chi, side, cols, r, cl.pt2ent.as<int>(), g.act_ptr.as<int>(), g.act_box.as<int>(),
                    kDF ? recb.as<pm::PeelRec>() : nullptr, kDF ? cntb.as<int>() : nullptr,
                    kDF ? trow.as<int64_t>() : nullptr);
                count_launch();
                HM_LAUNCH("peel_T");
            }
            if (kDF) {
                pm::CoarseC<R> d;
                d.ent = cj.ent.as<int>();
                d.pt2ent = cj.pt2ent.as<int>();
                d.base = bases[i].as<int64_t>();
                d.cnt = cntb.as<int>();
                d.rec = recb.as<pm::PeelRec>();
                d.F = side ? PD::V(f) : PD::U(f);
                d.T = T.template as<R>();
                dtab.push_back(d);
                keep.push_back(std::move(recb));
                keep.push_back(std::move(cntb));
                keep.push_back(std::move(trow));
            }
            tab.push_back(co);
            keep.push_back(std::move(X));
            keep.push_back(std::move(xo));
            keep.push_back(std::move(T));
            keep.push_back(std::move(live));
        }
        double *OUT = side ? c->cur.Z.as<double>() : c->cur.Y.as<double>();
        DBuf tabd;
        if constexpr (kDF) {
            HM_TRY(alloc(tabd, dtab.size() * sizeof(pm::CoarseC<R>)));
            HM_CUDA(cudaMemcpyAsync(tabd.p, dtab.data(), dtab.size() * sizeof(pm::CoarseC<R>), cudaMemcpyHostToDevice,
                                    st));
            if (nitems > 0)
                HM_TRY(launch_update_c<R>(c, tabd.as<pm::CoarseC<R>>(), (int)dtab.size(), chi, g, cl, item_tile,
                                          item_row, nitems, cols, r, OUT));
        } else {
            HM_TRY(alloc(tabd, tab.size() * sizeof(pm::CoarseT<R>)));
            HM_CUDA(cudaMemcpyAsync(tabd.p, tab.data(), tab.size() * sizeof(pm::CoarseT<R>), cudaMemcpyHostToDevice,
                                    st));
            if (nitems > 0)
                HM_TRY(launch_update(tabd.as<pm::CoarseT<R>>(), (int)tab.size(), side, chi, g, cl, item_tile,
                                     item_row, nitems, cols, r, n, OUT, st));
        }
    }
    return ok();
}

Err peel_level_mixed(hm_ctx *c, int level, bool leaf) { return peel_level_t<float>(c, level, leaf); }
Err peel_level_fp64(hm_ctx *c, int level, bool leaf) { return peel_level_t<double>(c, level, leaf); }
Err peel_level_df(hm_ctx *c, int level, bool leaf) { return peel_level_t<dfloat>(c, level, leaf); }

}  // namespace hm
