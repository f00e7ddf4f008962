// Per-pair bases and cores of one level (Algorithm 2.1 applied to every
// admissible block, Algorithm 4.1), and the leaf blocks (Section 4.1.3).
//
//  K9   U_{alpha,beta} = qr(Y(I_alpha, c), k): column-pivoted Householder QR of
//       the peeled sample tile, in place, one CTA per tile.  Pivot = the column
//       of largest remaining norm (norms recomputed exactly each step, lowest
//       index on ties); k is fixed, or the number of pivots whose norm exceeds
//       tol times the first; the explicit Q columns are signed so that
//       R_jj >= 0.  The same kernel factors every Z tile; V of pair
//       (alpha, beta) is the Q of the Z tile of the pair (beta, alpha).
//       FP64 mode: one warp per tile up to 256 rows, one CTA per larger tile.
//       HM_MIXED_BF16X6_F32: FP32 in shared memory, one CTA per tile up to
//       QR32_MAX_ROWS rows (FP64 CTA kernel beyond).
//  K10  B = (G_alpha^T U)^+ (G_alpha^T Y(I_alpha, c)) (V^T G_beta)^+ with
//       G_alpha the Psi-side block of alpha and G_beta the Omega-side block of
//       beta: the three r x k products over the boxes' rows by row-split CTAs
//       (k_gram), then Householder QR of the two r x k matrices and triangular
//       solves in shared memory (one warp per pair).
//  K11  D_{alpha,beta} = Y_leaf(I_alpha, c m_max + [0, |I_beta|)).
#include "ctx.cuh"
#include "df.cuh"

#include <algorithm>

namespace hm {

// Row-split Gram products of the core solve, one CTA per (pair, chunk of
// GRAM_CHUNK rows):  out[chunk][p] (r x r slot, row-major, first kf columns)
//   = sum over the chunk's rows i of G(s0 + i, :)^T F_p(i, :),
// G the level's Gaussians [n][r], s0 the first row of box[p], F_p the pair's
// block: the peeled Y tile of colour color[p] (kdim == nullptr, kf = r) or the
// packed factor at offF[p] with kf = kdim[p] columns.  A chunk beyond the box
// writes zeros; the consumer adds the chunks in order.  T is the type of the
// products and of the sums over 32-row blocks, TA that of the sums over the
// blocks and of the output: double-float and double in the HM_MIXED_BF16X6
// mode (products of about 48 bits on the FP32 pipe, 2^-44 relative per
// product: FP64-class for samples with FP32-class rounding, and five times
// the throughput of GB300's FP64 pipe), float and float in the
// HM_MIXED_BF16X6_F32 mode, double and double in FP64.
constexpr int GRAM_CHUNK = 1024;

template <typename T, typename TA>
__global__ void __launch_bounds__(256) k_gram(const int *box, const int *ent, int64_t np, int r, const double *G,
                                              const double *F, const int *color, int64_t n, const int64_t *offF,
                                              const int *kdim, TA *out) {
    __shared__ T gs[32][64], fs[32][64];
    const int64_t p = blockIdx.x;
    const int *e = ent + (int64_t)box[p] * ENT_FIELDS;
    const int s0 = e[3], m = e[4] - e[3];
    int kf;
    const double *Fp;
    if (kdim) {
        kf = kdim[p];
        Fp = F + offF[p];
    } else {
        kf = r;
        Fp = F + ((int64_t)color[p] * n + s0) * r;
    }
    const int i_begin = blockIdx.y * GRAM_CHUNK, i_end = min(m, i_begin + GRAM_CHUNK);
    TA acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = TA(0);
    for (int i0 = i_begin; i0 < i_end; i0 += 32) {
        const int mm = min(32, i_end - i0);
        for (int o = threadIdx.x; o < 32 * r; o += 256) {
            const int i = o / r, j = o % r;
            gs[i][j] = (i < mm) ? from_f64<T>(G[(int64_t)(s0 + i0 + i) * r + j]) : T(0);
        }
        for (int o = threadIdx.x; o < 32 * kf; o += 256) {
            const int i = o / kf, j = o % kf;
            fs[i][j] = (i < mm) ? from_f64<T>(Fp[(int64_t)(i0 + i) * kf + j]) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int o = threadIdx.x + q * 256;
            if (o < r * kf) {
                const int a = o / kf, b = o % kf;
                T sacc = T(0);  // the 32-row block in T, added to the TA sum
                for (int i = 0; i < mm; ++i) sacc = mac(gs[i][a], fs[i][b], sacc);
                acc[q] += widen(sacc, TA(0));
            }
        }
        __syncthreads();
    }
    TA *o_ = out + ((int64_t)blockIdx.y * np + p) * r * r;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int o = threadIdx.x + q * 256;
        if (o < r * kf) o_[(o / kf) * r + o % kf] = acc[q];
    }
}

constexpr int QR_WARP_ROWS_DECL = 256;
constexpr int QR32_MAX_ROWS = 1600;  // FP32 shared-memory QR: at most this many rows

// Column-pivoted Householder QR of one tile (m x r, row-major), in place;
// on exit the first k columns hold Q_k with R_jj >= 0.
__global__ void __launch_bounds__(256) k_qr_tiles(const int *tile_alpha, const int *tile_beta, const int *tile_color,
                                                  const int *ent, int64_t n, int r, int cap, int rank, double tol,
                                                  double *Ybase, int *kout, int min_rows,
                                                  const int *tile_cap = nullptr) {
    // thread (w, lane) owns columns lane and lane + 32 on the rows w, w + 8, ...:
    // every pass reads whole 256-byte rows.  One FMA per element and step in
    // the update, which also sums the squares of the updated trailing columns:
    // the exact norms of the next step, without a separate pass.
    __shared__ double red[8][64];
    __shared__ double nrm[64], wv[64], tau[64], beta[64];
    __shared__ int sh_piv, sh_stop;
    __shared__ double sh_scale, sh_n0;
    const int64_t p = blockIdx.x;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = e[4] - e[3];
    if (m <= min_rows) return;  // a warp or shared-memory kernel factors this tile
    double *A = Ybase + ((int64_t)tile_color[p] * n + e[3]) * r;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int *eb = ent + (int64_t)tile_beta[p] * ENT_FIELDS;
    // the block A(I_alpha, I_beta) has rank <= min(|I_alpha|, |I_beta|)
    const int kmax = min(min(min(m, eb[4] - eb[3]), min(r, cap)), tile_cap ? tile_cap[p] : r);
    // norms of step 0
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        double acc = 0.0;
        if (j < r)
            for (int i = w; i < m; i += 8) acc = fma(A[(int64_t)i * r + j], A[(int64_t)i * r + j], acc);
        red[w][j] = acc;
    }
    __syncthreads();
    if (tid < r) {
        double t = 0.0;
        for (int u = 0; u < 8; ++u) t += red[u][tid];
        nrm[tid] = t;
    }
    __syncthreads();
    int k = 0;
    for (int s = 0; s < kmax; ++s) {
        if (tid == 0) {
            int piv = s;
            for (int j = s + 1; j < r; ++j)
                if (nrm[j] > nrm[piv]) piv = j;  // largest norm, lowest column on ties
            const double nv = sqrt(nrm[piv]);
            if (s == 0) sh_n0 = nv;
            int stop = 0;
            if (rank > 0) stop = (s >= rank);
            else stop = !(sh_n0 > 0.0) || !(nv > tol * sh_n0);
            sh_piv = piv;
            sh_stop = stop;
            if (!stop && piv != s) {  // the norms move with their columns
                const double t = nrm[s];
                nrm[s] = nrm[piv];
                nrm[piv] = t;
            }
        }
        __syncthreads();
        if (sh_stop) break;
        const int piv = sh_piv;
        if (piv != s)
            for (int i = tid; i < m; i += blockDim.x) {
                const double a = A[(int64_t)i * r + s];
                A[(int64_t)i * r + s] = A[(int64_t)i * r + piv];
                A[(int64_t)i * r + piv] = a;
            }
        __syncthreads();
        if (tid == 0) {
            const double x0 = A[(int64_t)s * r + s];
            const double nx = sqrt(nrm[s]);
            if (nx == 0.0) {
                tau[s] = 0.0;
                beta[s] = 0.0;
                sh_scale = 0.0;
            } else {
                const double b = -copysign(nx, x0);
                tau[s] = (b - x0) / b;
                beta[s] = b;
                sh_scale = 1.0 / (x0 - b);
                A[(int64_t)s * r + s] = b;
            }
        }
        __syncthreads();
        const double sc = sh_scale, ts = tau[s];
        for (int i = s + 1 + tid; i < m; i += blockDim.x) A[(int64_t)i * r + s] *= sc;
        __syncthreads();
        // H = I - tau v v^T, v = [1; A(s+1:m, s)]: w_j = A(s, j) + v(s+1:)^T A(s+1:, j)
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            double acc = 0.0;
            if (j > s && j < r)
                for (int i = s + 1 + w; i < m; i += 8) acc = fma(A[(int64_t)i * r + s], A[(int64_t)i * r + j], acc);
            red[w][j] = acc;
        }
        __syncthreads();
        if (tid > s && tid < r) {
            double t = A[(int64_t)s * r + tid];
            for (int u = 0; u < 8; ++u) t += red[u][tid];
            const double tw = ts * t;
            wv[tid] = tw;
            A[(int64_t)s * r + tid] -= tw;
        }
        __syncthreads();
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            double acc = 0.0;
            if (j > s && j < r) {
                const double tw = wv[j];
                for (int i = s + 1 + w; i < m; i += 8) {
                    const double a = fma(-tw, A[(int64_t)i * r + s], A[(int64_t)i * r + j]);
                    A[(int64_t)i * r + j] = a;
                    acc = fma(a, a, acc);
                }
            }
            red[w][j] = acc;
        }
        __syncthreads();
        if (tid > s && tid < r) {  // norms over rows s+1.. for the next step
            double t = 0.0;
            for (int u = 0; u < 8; ++u) t += red[u][tid];
            nrm[tid] = t;
        }
        __syncthreads();
        k = s + 1;
    }
    // explicit Q_k (backward accumulation of the reflectors)
    for (int j = k - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (j < k - 1) {
            for (int h = 0; h < 2; ++h) {
                const int t = lane + 32 * h;
                double acc = 0.0;
                if (t > j && t < k)
                    for (int i = j + 1 + w; i < m; i += 8) acc = fma(A[(int64_t)i * r + j], A[(int64_t)i * r + t], acc);
                red[w][t] = acc;
            }
            __syncthreads();
            if (tid > j && tid < k) {
                double x = A[(int64_t)j * r + tid];
                for (int u = 0; u < 8; ++u) x += red[u][tid];
                const double tw = tj * x;
                wv[tid] = tw;
                A[(int64_t)j * r + tid] -= tw;
            }
            __syncthreads();
            for (int h = 0; h < 2; ++h) {
                const int t = lane + 32 * h;
                if (t > j && t < k) {
                    const double tw = wv[t];
                    for (int i = j + 1 + w; i < m; i += 8)
                        A[(int64_t)i * r + t] = fma(-tw, A[(int64_t)i * r + j], A[(int64_t)i * r + t]);
                }
            }
            __syncthreads();
        }
        for (int i = tid; i < m; i += blockDim.x) {
            double v;
            if (i < j) v = 0.0;
            else if (i == j) v = 1.0 - tj;
            else v = -tj * A[(int64_t)i * r + j];
            A[(int64_t)i * r + j] = v;
        }
        __syncthreads();
    }
    // R_jj >= 0
    for (int i = w; i < m; i += 8)
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            if (j < k && beta[j] < 0.0) A[(int64_t)i * r + j] = -A[(int64_t)i * r + j];
        }
    if (tid == 0) kout[p] = k;
}

// The same pivoted QR for tiles of at most QR_WARP_ROWS rows: one warp per
// tile, lane j owns columns j and j + 32; for a fixed row the lanes touch
// consecutive columns (coalesced), and the Householder vector's entry is a
// broadcast load.  No block barriers.
constexpr int QR_WARP_ROWS = QR_WARP_ROWS_DECL;

__global__ void __launch_bounds__(128) k_qr_warp(const int *tile_alpha, const int *tile_beta, const int *tile_color,
                                                 const int *ent, int64_t n, int r, int cap, int rank, double tol,
                                                 double *Ybase, int *kout, int64_t ntiles,
                                                 const int *tile_cap = nullptr) {
    __shared__ double s_tau[4][64], s_beta[4][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * 4 + warp;
    if (p >= ntiles) return;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = e[4] - e[3];
    if (m > QR_WARP_ROWS) return;  // the block kernel factors this tile
    double *A = Ybase + ((int64_t)tile_color[p] * n + e[3]) * r;
    const int *eb = ent + (int64_t)tile_beta[p] * ENT_FIELDS;
    const int kmax = min(min(min(m, eb[4] - eb[3]), min(r, cap)), tile_cap ? tile_cap[p] : r);
    double *tau = s_tau[warp], *beta = s_beta[warp];
    const int c0 = lane, c1 = lane + 32;
    double n0 = 0.0;
    int k = 0;
    // exact norms of the lane's columns over rows s..m-1: a pass for step 0, then
    // summed by the update of each step over the rows it leaves
    double a0 = 0.0, a1 = 0.0;
    for (int i = 0; i < m; ++i) {
        if (c0 < r) a0 = fma(A[(int64_t)i * r + c0], A[(int64_t)i * r + c0], a0);
        if (c1 < r) a1 = fma(A[(int64_t)i * r + c1], A[(int64_t)i * r + c1], a1);
    }
    for (int s = 0; s < kmax; ++s) {
        double best = -1.0;
        int bj = 1 << 30;
        if (c0 < r && c0 >= s) { best = a0; bj = c0; }
        if (c1 < r && c1 >= s && (a1 > best || bj == (1 << 30))) { best = a1; bj = c1; }
        for (int o = 16; o > 0; o >>= 1) {  // largest norm, lowest column on ties
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        const double nv = sqrt(best);
        if (s == 0) n0 = nv;
        const bool stop = rank > 0 ? (s >= rank) : (!(n0 > 0.0) || !(nv > tol * n0));
        if (stop) break;
        const int piv = bj;
        if (piv != s) {
            for (int i = lane; i < m; i += 32) {
                const double t = A[(int64_t)i * r + s];
                A[(int64_t)i * r + s] = A[(int64_t)i * r + piv];
                A[(int64_t)i * r + piv] = t;
            }
            // the norm of column s moves to column piv
            const double ns = __shfl_sync(0xffffffffu, s < 32 ? a0 : a1, s & 31);
            if (lane == (piv & 31)) {
                if (piv < 32) a0 = ns;
                else a1 = ns;
            }
        }
        __syncwarp();
        const double x0 = A[(int64_t)s * r + s];
        double t = 0.0, b = 0.0, sc = 0.0;
        if (nv > 0.0) {
            b = -copysign(nv, x0);
            t = (b - x0) / b;
            sc = 1.0 / (x0 - b);
        }
        for (int i = s + 1 + lane; i < m; i += 32) A[(int64_t)i * r + s] *= sc;
        __syncwarp();
        if (lane == 0) {
            tau[s] = t;
            beta[s] = b;
            if (nv > 0.0) A[(int64_t)s * r + s] = b;
        }
        for (int h = 0; h < 2; ++h) {
            const int j = h ? c1 : c0;
            if (j <= s || j >= r) continue;
            double wj = A[(int64_t)s * r + j];
            for (int i = s + 1; i < m; ++i) wj = fma(A[(int64_t)i * r + s], A[(int64_t)i * r + j], wj);
            const double tw = t * wj;
            A[(int64_t)s * r + j] -= tw;
            double acc = 0.0;
            for (int i = s + 1; i < m; ++i) {
                const double a = fma(-tw, A[(int64_t)i * r + s], A[(int64_t)i * r + j]);
                A[(int64_t)i * r + j] = a;
                acc = fma(a, a, acc);
            }
            if (h) a1 = acc;
            else a0 = acc;
        }
        __syncwarp();
        k = s + 1;
    }
    // explicit Q_k, backward accumulation of the reflectors
    for (int j = k - 1; j >= 0; --j) {
        const double tj = tau[j];
        for (int h = 0; h < 2; ++h) {
            const int c = h ? c1 : c0;
            if (c <= j || c >= k) continue;
            double w = A[(int64_t)j * r + c];
            for (int i = j + 1; i < m; ++i) w = fma(A[(int64_t)i * r + j], A[(int64_t)i * r + c], w);
            const double tw = tj * w;
            A[(int64_t)j * r + c] -= tw;
            for (int i = j + 1; i < m; ++i) A[(int64_t)i * r + c] = fma(-tw, A[(int64_t)i * r + j], A[(int64_t)i * r + c]);
        }
        __syncwarp();
        for (int i = lane; i < m; i += 32) {
            double v;
            if (i < j) v = 0.0;
            else if (i == j) v = 1.0 - tj;
            else v = -tj * A[(int64_t)i * r + j];
            A[(int64_t)i * r + j] = v;
        }
        __syncwarp();
    }
    for (int h = 0; h < 2; ++h) {  // R_jj >= 0
        const int c = h ? c1 : c0;
        if (c < k && beta[c] < 0.0)
            for (int i = 0; i < m; ++i) A[(int64_t)i * r + c] = -A[(int64_t)i * r + c];
    }
    if (lane == 0) kout[p] = k;
}

// ---------------------------------------------------------------------------
// HM_MIXED_BF16X6_F32: FP32 QR with the tile in shared memory (the samples it
// factors carry FP32-level rounding already).  The CTA's threads (128 or 512) work on
// column t % RP (RP = 32 for r <= 32, else 64) and on the rows i = t / RP
// (mod blockDim / RP) in the column passes; partial sums over the row groups are
// added in group order.
// ---------------------------------------------------------------------------

// sum over the rows i >= i0 of a(i, j) b(i, j') for the thread's column, added
// over the row groups: the result for column t (t < r) is returned to thread t
template <typename T>
__device__ __forceinline__ void col_dots(const T *qa, int m, int r, int i0, int ca, int cb_lo, int cb_hi,
                                         bool square, T (*red)[64], T *out) {
    const int t = threadIdx.x, RP = r <= 32 ? 32 : 64, NG = (int)blockDim.x / RP, cj = t % RP, grp = t / RP;
    T a = T(0);
    if (cj >= cb_lo && cj < cb_hi) {
        if (square)
            for (int i = i0 + grp; i < m; i += NG) a = fma(qa[i * r + cj], qa[i * r + cj], a);
        else
            for (int i = i0 + grp; i < m; i += NG) a = fma(qa[i * r + ca], qa[i * r + cj], a);
    }
    red[grp][cj] = a;
    __syncthreads();
    if (t < r) {
        T v = T(0);
        for (int g = 0; g < NG; ++g) v += red[g][t];
        out[t] = v;
    }
    __syncthreads();
}

// A(i, j) -= tau v_i w_j for i >= s, j in (s, jhi); v_s = 1, v_i = A(i, s) below
template <typename T>
__device__ __forceinline__ void reflect(T *qa, int m, int r, int s, int jhi, T ts, const T *wv) {
    const int t = threadIdx.x, RP = r <= 32 ? 32 : 64, NG = (int)blockDim.x / RP, cj = t % RP, grp = t / RP;
    if (cj > s && cj < jhi) {
        const T w = ts * wv[cj];
        for (int i = s + grp; i < m; i += NG) {
            const T vi = (i == s) ? T(1) : qa[i * r + s];
            qa[i * r + cj] -= vi * w;
        }
    }
    __syncthreads();
}

// Column-pivoted Householder QR of the m x r shared tile qa (ld r), at most
// kmax steps, stopping by the rank or tolerance rule; on return columns
// 0..k-1 hold Q_k with R_jj >= 0, and every thread returns k.
template <typename T>
__device__ int qr_pivoted_smem(T *qa, int m, int r, int kmax, int rank, double tol) {
    __shared__ T red[16][64], nrm[64], wv[64], tau[64], beta[64];
    __shared__ T sh_sc;
    __shared__ int sh_piv, sh_stop;
    const int t = threadIdx.x;
    T n0 = T(0);
    int k = 0;
    for (int s = 0; s < kmax; ++s) {
        col_dots(qa, m, r, s, 0, s, r, true, red, nrm);  // exact norms of the trailing columns
        if (t == 0) {
            T best = T(-1);
            int piv = s;
            for (int j = s; j < r; ++j)
                if (nrm[j] > best) {  // largest norm, lowest column on ties
                    best = nrm[j];
                    piv = j;
                }
            const T nv = sqrt(best);
            if (s == 0) n0 = nv;
            const int stop = rank > 0 ? (s >= rank) : (!(n0 > T(0)) || !((double)nv > tol * (double)n0));
            sh_stop = stop;
            sh_piv = piv;
            if (!stop) {
                const T x0 = qa[s * r + piv];
                T tt = T(0), b = T(0), sc = T(0);
                if (nv > T(0)) {
                    b = -copysign(nv, x0);
                    tt = (b - x0) / b;
                    sc = T(1) / (x0 - b);
                }
                tau[s] = tt;
                beta[s] = b;
                sh_sc = sc;
            }
        }
        __syncthreads();
        if (sh_stop) break;
        const int piv = sh_piv;
        const T sc = sh_sc, ts = tau[s], bs = beta[s];
        // swap columns s and piv, scale the reflector, set R_ss
        for (int i = t; i < m; i += blockDim.x) {
            T vs = qa[i * r + s];
            if (piv != s) {
                const T vp = qa[i * r + piv];
                qa[i * r + piv] = vs;
                vs = vp;
            }
            if (i > s) vs *= sc;
            else if (i == s && bs != T(0)) vs = bs;
            qa[i * r + s] = vs;
        }
        __syncthreads();
        // w_j = A(s, j) + sum_{i > s} v_i A(i, j), then A(i, j) -= tau v_i w_j
        col_dots(qa, m, r, s + 1, s, s + 1, r, false, red, wv);
        if (t > s && t < r) wv[t] += qa[s * r + t];
        __syncthreads();
        reflect(qa, m, r, s, r, ts, wv);
        k = s + 1;
    }
    // explicit Q_k, backward accumulation of the reflectors
    for (int j = k - 1; j >= 0; --j) {
        const T tj = tau[j];
        if (j < k - 1) {
            col_dots(qa, m, r, j + 1, j, j + 1, k, false, red, wv);
            if (t > j && t < k) wv[t] += qa[j * r + t];
            __syncthreads();
            reflect(qa, m, r, j, k, tj, wv);
        }
        for (int i = t; i < m; i += blockDim.x) {
            T v;
            if (i < j) v = T(0);
            else if (i == j) v = T(1) - tj;
            else v = -tj * qa[i * r + j];
            qa[i * r + j] = v;
        }
        __syncthreads();
    }
    for (int o = t; o < m * k; o += blockDim.x) {  // R_jj >= 0
        const int j = o % k;
        if (beta[j] < T(0)) qa[(o / k) * r + j] = -qa[(o / k) * r + j];
    }
    __syncthreads();
    return k;
}

// One CTA per tile of min_rows < m <= max_rows rows; Q_k back to the FP64 tile.
template <typename T>
__global__ void __launch_bounds__(512) k_qr_smem(const int *tile_alpha, const int *tile_beta, const int *tile_color,
                                              const int *ent, int64_t n, int r, int cap, int rank, double tol,
                                              double *Ybase, int *kout, int min_rows, int max_rows,
                                              const int *tile_cap = nullptr) {
    extern __shared__ __align__(16) unsigned char qa_raw[];
    T *qa = reinterpret_cast<T *>(qa_raw);  // m x r, leading dimension r
    const int64_t p = blockIdx.x;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = e[4] - e[3];
    if (m <= min_rows || m > max_rows) return;  // another launch factors this tile
    double *Ag = Ybase + ((int64_t)tile_color[p] * n + e[3]) * r;
    const int *eb = ent + (int64_t)tile_beta[p] * ENT_FIELDS;
    const int kmax = min(min(min(m, eb[4] - eb[3]), min(r, cap)), tile_cap ? tile_cap[p] : r);
    for (int o = threadIdx.x; o < m * r; o += blockDim.x) qa[o] = (T)Ag[o];
    __syncthreads();
    const int k = qr_pivoted_smem<T>(qa, m, r, kmax, rank, tol);
    for (int o = threadIdx.x; o < m * k; o += blockDim.x) Ag[(int64_t)(o / k) * r + o % k] = (double)qa[(o / k) * r + o % k];
    if (threadIdx.x == 0) kout[p] = k;
}

// ---------------------------------------------------------------------------
// HM_MIXED_BF16X6_F32, tall tiles: FP32 tall-skinny QR.  A tile of m rows is cut
// into nb balanced blocks of at most TS_ROWS rows (blocks of tiles above the
// shared-memory limit only).  (1) every block: unpivoted Householder QR,
// A_b = Q_b R_b, the reflectors written over the block, R_b into the stack;
// (2) every tile: the column-pivoted QR of the stacked R_b (nb r x r) -- the
// column norms, hence the pivots, the rank and R, are those of the tile --
// giving Q_S; (3) every block: U_b = Q_b Q_S(block rows, 0:k).
// ---------------------------------------------------------------------------

__global__ void k_ts_count(const int *tile_alpha, const int *ent, int64_t np, int min_rows, int max_rows, int brows,
                           int64_t *cnt) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = e[4] - e[3];
    cnt[p] = (m > min_rows && m <= max_rows) ? (m + brows - 1) / brows : 0;
}

__global__ void k_ts_fill(const int *tile_alpha, const int *ent, const int64_t *off, int64_t np, int64_t *blk_tile,
                          int *blk_row0, int *blk_rows) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int nb = (int)(off[p + 1] - off[p]);
    if (nb == 0) return;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = e[4] - e[3], per = (m + nb - 1) / nb;
    for (int b = 0; b < nb; ++b) {
        blk_tile[off[p] + b] = p;
        blk_row0[off[p] + b] = b * per;
        blk_rows[off[p] + b] = min(per, m - b * per);
    }
}

// (1) unpivoted QR of one block; R_b (r x r, zero below the diagonal) into
// the stack at [blk][r][r], the reflectors over the block, tau at [blk][r]
template <typename T>
__global__ void __launch_bounds__(512) k_ts_block(const int *tile_alpha, const int *tile_color, const int *ent,
                                                  int64_t n, int r, double *Ybase, const int64_t *blk_tile,
                                                  const int *blk_row0, const int *blk_rows, T *Rstack, T *taus) {
    extern __shared__ __align__(16) unsigned char ts_raw[];
    T *qa = reinterpret_cast<T *>(ts_raw);
    __shared__ T red[16][64], nrm[64], wv[64];
    const int64_t blk = blockIdx.x;
    const int64_t p = blk_tile[blk];
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = blk_rows[blk], t = threadIdx.x;
    double *Ag = Ybase + ((int64_t)tile_color[p] * n + e[3] + blk_row0[blk]) * r;
    for (int o = t; o < m * r; o += blockDim.x) qa[o] = (T)Ag[o];
    __syncthreads();
    const int steps = min(m, r);
    for (int s = 0; s < steps; ++s) {
        col_dots(qa, m, r, s, 0, s, s + 1, true, red, nrm);
        const T nv = sqrt(nrm[s]), x0 = qa[s * r + s];
        T ts = T(0), b = T(0), sc = T(0);
        if (nv > T(0)) {
            b = -copysign(nv, x0);
            ts = (b - x0) / b;
            sc = T(1) / (x0 - b);
        }
        for (int i = s + 1 + t; i < m; i += blockDim.x) qa[i * r + s] *= sc;
        __syncthreads();
        if (t == 0) {
            taus[blk * r + s] = ts;
            if (nv > T(0)) qa[s * r + s] = b;
        }
        col_dots(qa, m, r, s + 1, s, s + 1, r, false, red, wv);
        if (t > s && t < r) wv[t] += qa[s * r + t];
        __syncthreads();
        reflect(qa, m, r, s, r, ts, wv);
    }
    for (int s = steps + t; s < r; s += blockDim.x) taus[blk * r + s] = T(0);
    T *R = Rstack + blk * r * r;
    for (int o = t; o < r * r; o += blockDim.x) {
        const int i = o / r, j = o % r;
        R[o] = (i <= j && i < m) ? qa[i * r + j] : T(0);
    }
    for (int o = t; o < m * r; o += blockDim.x) Ag[o] = (double)qa[o];
}

// (2) pivoted QR of the stacked R_b of one tile, in place in the stack
template <typename T>
__global__ void __launch_bounds__(512) k_ts_top(const int *tile_alpha, const int *tile_beta, const int *ent,
                                                int64_t np, int r, int cap, int rank, double tol, const int64_t *off,
                                                T *Rstack, int *kout, const int *tile_cap = nullptr) {
    extern __shared__ __align__(16) unsigned char ts_raw[];
    T *qa = reinterpret_cast<T *>(ts_raw);
    const int64_t p = blockIdx.x;
    const int nb = (int)(off[p + 1] - off[p]);
    if (nb == 0) return;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS, *eb = ent + (int64_t)tile_beta[p] * ENT_FIELDS;
    const int m = e[4] - e[3], ms = nb * r;
    const int kmax = min(min(min(m, eb[4] - eb[3]), min(r, cap)), tile_cap ? tile_cap[p] : r);
    T *S = Rstack + off[p] * r * r;
    for (int o = threadIdx.x; o < ms * r; o += blockDim.x) qa[o] = S[o];
    __syncthreads();
    const int k = qr_pivoted_smem<T>(qa, ms, r, kmax, rank, tol);
    for (int o = threadIdx.x; o < ms * r; o += blockDim.x) S[o] = qa[o];
    if (threadIdx.x == 0) kout[p] = k;
}

// (3) U_b = Q_b [Q_S(block rows, 0:k); 0] into the block's rows, columns 0..k-1
template <typename T>
__global__ void __launch_bounds__(512) k_ts_form(const int *tile_alpha, const int *tile_color, const int *ent,
                                                 int64_t n, int r, double *Ybase, const int64_t *blk_tile,
                                                 const int *blk_row0, const int *blk_rows, const T *Rstack,
                                                 const T *taus, const int *kout) {
    extern __shared__ __align__(16) unsigned char ts_raw[];
    T *qa = reinterpret_cast<T *>(ts_raw);  // reflectors m x r, then X m x k (ld r)
    __shared__ T red[16][64], wv[64];
    const int64_t blk = blockIdx.x;
    const int64_t p = blk_tile[blk];
    const int k = kout[p];
    if (k == 0) return;
    const int *e = ent + (int64_t)tile_alpha[p] * ENT_FIELDS;
    const int m = blk_rows[blk], t = threadIdx.x;
    double *Ag = Ybase + ((int64_t)tile_color[p] * n + e[3] + blk_row0[blk]) * r;
    T *X = qa + m * r;
    const T *QS = Rstack + blk * r * r;  // this block's r rows of Q_S
    for (int o = t; o < m * r; o += blockDim.x) {
        const int i = o / r, j = o % r;
        qa[o] = (T)Ag[o];
        X[o] = (j < k && i < r) ? QS[i * r + j] : T(0);
    }
    __syncthreads();
    const int steps = min(m, r);
    for (int s = steps - 1; s >= 0; --s) {
        const T ts = taus[blk * r + s];
        // w_c = X(s, c) + sum_{i > s} v_i X(i, c); X(i, c) -= tau v_i w_c
        const int RP = r <= 32 ? 32 : 64, NG = (int)blockDim.x / RP, cj = t % RP, grp = t / RP;
        T a = T(0);
        if (cj < k)
            for (int i = s + 1 + grp; i < m; i += NG) a = fma(qa[i * r + s], X[i * r + cj], a);
        red[grp][cj] = a;
        __syncthreads();
        if (t < k) {
            T w = X[s * r + t];
            for (int g = 0; g < NG; ++g) w += red[g][t];
            wv[t] = ts * w;
        }
        __syncthreads();
        if (cj < k)
            for (int i = s + grp; i < m; i += NG) {
                const T vi = (i == s) ? T(1) : qa[i * r + s];
                X[i * r + cj] -= vi * wv[cj];
            }
        __syncthreads();
    }
    for (int o = t; o < m * k; o += blockDim.x) Ag[(int64_t)(o / k) * r + o % k] = (double)X[(o / k) * r + o % k];
}

__global__ void k_factor_sizes(const int *pair_alpha, const int *pair_col, const int *pairT, const int *kY,
                               const int *kZ, const int *ent, int64_t np, int *kU, int *kV, int64_t *sU, int64_t *sV,
                               int64_t *sB) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int *ea = ent + (int64_t)pair_alpha[p] * ENT_FIELDS, *eb = ent + (int64_t)pair_col[p] * ENT_FIELDS;
    const int ku = kY[p], kv = kZ[pairT[p]];
    kU[p] = ku;
    kV[p] = kv;
    sU[p] = (int64_t)(ea[4] - ea[3]) * ku;
    sV[p] = (int64_t)(eb[4] - eb[3]) * kv;
    sB[p] = (int64_t)ku * kv;
}

__global__ void k_pack(const int *pair_alpha, const int *pair_col, const int *pair_color, const int *pairT,
                       const int *ent, int64_t n, int r, const int *kU, const int *kV, const int64_t *offU,
                       const int64_t *offV, const double *Y, const double *Z, double *U, double *V) {
    const int64_t p = blockIdx.x;
    const int *ea = ent + (int64_t)pair_alpha[p] * ENT_FIELDS, *eb = ent + (int64_t)pair_col[p] * ENT_FIELDS;
    const int ma = ea[4] - ea[3], mb = eb[4] - eb[3], ku = kU[p], kv = kV[p];
    const double *Yt = Y + ((int64_t)pair_color[p] * n + ea[3]) * r;
    const int pt = pairT[p];
    const double *Zt = Z + ((int64_t)pair_color[pt] * n + eb[3]) * r;
    for (int o = threadIdx.x; o < ma * ku; o += blockDim.x) U[offU[p] + o] = Yt[(int64_t)(o / ku) * r + o % ku];
    for (int o = threadIdx.x; o < mb * kv; o += blockDim.x) V[offV[p] + o] = Zt[(int64_t)(o / kv) * r + o % kv];
}

// --- warp-level small dense helpers (row-major, leading dimension ld) -------

// Householder QR of A (m x k), R in the upper triangle, v below (v0 = 1).
template <typename T> __device__ void warp_house_qr(T *A, int m, int k, int ld, T *tau) {
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < k; ++s) {
        T ss = T(0);
        for (int i = s + lane; i < m; i += 32) ss = fma(A[i * ld + s], A[i * ld + s], ss);
        ss = warp_sum(ss);
        const T x0 = A[s * ld + s], nx = sqrt(ss);
        T t = T(0), b = T(0), sc = T(0);
        if (nx > T(0)) {
            b = -copysign(nx, x0);
            t = (b - x0) / b;
            sc = T(1) / (x0 - b);
        }
        __syncwarp();
        for (int i = s + 1 + lane; i < m; i += 32) A[i * ld + s] *= sc;
        if (lane == 0) {
            tau[s] = t;
            if (nx > T(0)) A[s * ld + s] = b;
        }
        __syncwarp();
        for (int j = s + 1 + lane; j < k; j += 32) {
            T wv = A[s * ld + j];
            for (int i = s + 1; i < m; ++i) wv = fma(A[i * ld + s], A[i * ld + j], wv);
            A[s * ld + j] -= t * wv;
            for (int i = s + 1; i < m; ++i) A[i * ld + j] -= t * A[i * ld + s] * wv;
        }
        __syncwarp();
    }
}

// X (m x nc) := Q^T X for the reflectors stored in A (m x k)
template <typename T>
__device__ void warp_apply_qt(const T *A, int m, int k, int lda, const T *tau, T *X, int nc, int ldx) {
    const int lane = threadIdx.x & 31;
    for (int s = 0; s < k; ++s) {
        const T t = tau[s];
        for (int j = lane; j < nc; j += 32) {
            T wv = X[s * ldx + j];
            for (int i = s + 1; i < m; ++i) wv = fma(A[i * lda + s], X[i * ldx + j], wv);
            X[s * ldx + j] -= t * wv;
            for (int i = s + 1; i < m; ++i) X[i * ldx + j] -= t * A[i * lda + s] * wv;
        }
        __syncwarp();
    }
}

// X (k x nc) := R^{-1} X, R the k x k upper triangle of A
template <typename T> __device__ void warp_back_solve(const T *A, int k, int lda, T *X, int nc, int ldx) {
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < nc; j += 32)
        for (int i = k - 1; i >= 0; --i) {
            T v = X[i * ldx + j];
            for (int t = i + 1; t < k; ++t) v -= A[i * lda + t] * X[t * ldx + j];
            X[i * ldx + j] = v / A[i * lda + i];
        }
    __syncwarp();
}

// one warp per pair, up to four pairs per CTA: B = (GP_a^T U)^+ M (GO_b^T V)^{+T}.
// M = GP_a^T P, S1 = GP_a^T U and S2 = GO_b^T V arrive as nsplit row-chunk
// partial products (k_gram); the warp adds them in chunk order into shared
// memory, where S1, S2 and X^T have leading dimension kc (the largest k) and
// M leading dimension r.
constexpr int CORE_WARPS = 4;

template <typename T, typename TP>
__device__ __forceinline__ T sum_chunks(const TP *part, int nsplit, int64_t np, int64_t p, int r, int idx) {
    T s = T(0);
    for (int c = 0; c < nsplit; ++c) s += part[((int64_t)c * np + p) * r * r + idx];
    return s;
}

// T: compute type of the solves; TP: type of the partial products
template <typename T, typename TP>
__global__ void __launch_bounds__(128) k_core(int r, int kc, int64_t np, int nsplit, const int *kU, const int *kV,
                                              const int64_t *offB, const TP *Mpart, const TP *S1part,
                                              const TP *S2part, double *B) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *sm = reinterpret_cast<T *>(sm_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * nwarps + warp;
    if (p >= np) return;
    const int ku = kU[p], kv = kV[p];
    if (ku == 0 || kv == 0) return;
    T *S1 = sm + (size_t)warp * (3 * r * kc + r + r * r);  // r x ku  (ld kc)
    T *S2 = S1 + r * kc;                                    // r x kv
    T *X = S2 + r * kc;                                     // r x ku: X^T
    T *tau = X + r * kc;                                    // r
    T *Mx = tau + r;                                        // r x r (ld r)
    for (int o = lane; o < r * ku; o += 32)
        S1[(o / ku) * kc + o % ku] = sum_chunks<T>(S1part, nsplit, np, p, r, (o / ku) * r + o % ku);
    for (int o = lane; o < r * kv; o += 32)
        S2[(o / kv) * kc + o % kv] = sum_chunks<T>(S2part, nsplit, np, p, r, (o / kv) * r + o % kv);
    for (int o = lane; o < r * r; o += 32) Mx[o] = sum_chunks<T>(Mpart, nsplit, np, p, r, o);
    __syncwarp();
    // X = R1^{-1} (Q1^T M)(0:ku, :)
    warp_house_qr(S1, r, ku, kc, tau);
    warp_apply_qt(S1, r, ku, kc, tau, Mx, r, r);
    warp_back_solve(S1, ku, kc, Mx, r, r);
    // B^T = R2^{-1} (Q2^T X^T)(0:kv, :)
    for (int o = lane; o < r * ku; o += 32) {
        const int a = o / ku, u = o % ku;
        X[a * kc + u] = Mx[u * r + a];
    }
    __syncwarp();
    warp_house_qr(S2, r, kv, kc, tau);
    warp_apply_qt(S2, r, kv, kc, tau, X, ku, kc);
    warp_back_solve(S2, kv, kc, X, ku, kc);
    double *Bp = B + offB[p];
    for (int o = lane; o < ku * kv; o += 32) {
        const int u = o / kv, v = o % kv;
        Bp[o] = (double)X[v * kc + u];
    }
}

template <typename T, typename TA>
static void launch_gram(unsigned np, int nsplit, cudaStream_t st, const int *box, const int *ent, int r,
                        const double *G, const double *F, const int *color, int64_t n, const int64_t *offF,
                        const int *kdim, void *out) {
    k_gram<T, TA><<<dim3(np, nsplit), 256, 0, st>>>(box, ent, (int64_t)np, r, G, F, color, n, offF, kdim,
                                                   static_cast<TA *>(out));
    ::hm::count_launch();
}

// the Gram products' arithmetic of the context's precision mode
using GramLaunch = void (*)(unsigned, int, cudaStream_t, const int *, const int *, int, const double *, const double *,
                            const int *, int64_t, const int64_t *, const int *, void *);
static GramLaunch gram_launcher(const hm_ctx *c) {
    if (c->cfg.precision == HM_MIXED_BF16X6_F32) return launch_gram<float, float>;
    if (c->cfg.precision == HM_MIXED_BF16X6) return launch_gram<dfloat, double>;
    return launch_gram<double, double>;
}


template <typename T, typename TP>
static Err launch_core(int64_t np, int nsplit, int r, int kc, cudaStream_t st, const int *kU, const int *kV,
                       const int64_t *offB, const void *Mpart, const void *S1part, const void *S2part, double *B) {
    const size_t per_warp = (3 * (size_t)r * kc + r + (size_t)r * r) * sizeof(T);
    const int core_warps = (int)std::min<size_t>(CORE_WARPS, (200 * 1024) / per_warp);
    if (core_warps < 1) return fail(HM_ENOTSUP, "cores: r x k too large for shared memory");
    const size_t smem = (size_t)core_warps * per_warp;
    HM_TRY(allow_smem(k_core<T, TP>, smem));
    k_core<T, TP><<<ceil_div(np, core_warps), core_warps * 32, smem, st>>>(
        r, kc, np, nsplit, kU, kV, offB, static_cast<const TP *>(Mpart), static_cast<const TP *>(S1part),
        static_cast<const TP *>(S2part), B);
    ::hm::count_launch();
    return ok();
}

// the three tall-skinny QR launches of one side (block QRs, pivoted QR of each
// tile's stacked R, composition of Q) in element type T
template <typename T>
static void launch_ts(const int *tile_box, const int *tile_beta, const int *tile_color, const int *tile_cap,
                      const int *ent, int64_t n, int r, int cap, int rank, double tol, double *Y, int *kk, int64_t np,
                      int64_t nblk, int nb_top, int ts_rows, const DBuf &ts_off, const DBuf &blk_tile,
                      const DBuf &blk_row0, const DBuf &blk_rows, DBuf &rstack, DBuf &taus, cudaStream_t st) {
    k_ts_block<T><<<(unsigned)nblk, 512, (size_t)ts_rows * r * sizeof(T), st>>>(
        tile_box, tile_color, ent, n, r, Y, blk_tile.as<int64_t>(), blk_row0.as<int>(), blk_rows.as<int>(),
        rstack.as<T>(), taus.as<T>()); ::hm::count_launch();
    k_ts_top<T><<<(unsigned)np, 512, (size_t)nb_top * r * r * sizeof(T), st>>>(
        tile_box, tile_beta, ent, np, r, cap, rank, tol, ts_off.as<int64_t>(), rstack.as<T>(), kk, tile_cap); ::hm::count_launch();
    k_ts_form<T><<<(unsigned)nblk, 512, (size_t)2 * ts_rows * r * sizeof(T), st>>>(
        tile_box, tile_color, ent, n, r, Y, blk_tile.as<int64_t>(), blk_row0.as<int>(), blk_rows.as<int>(),
        rstack.as<T>(), taus.as<T>(), kk); ::hm::count_launch();
}

Err qr_tiles_fp64(hm_ctx *c, int level, const int *tile_box, const int *tile_color, const int *tile_cap, int64_t nt,
                  int max_rows, double *base, int cap, int rank, double tol, int *kout) {
    if (nt == 0) return ok();
    cudaStream_t st = c->st;
    const int r = c->cfg.r;
    const int64_t n = c->n;
    const int *ent = c->cuts[level].ent.as<int>();
    const int qr64_rows = (200 * 1024) / (8 * r);
    // the box is its own partner (tile_beta = tile_box): the caps come from tile_cap
    k_qr_warp<<<ceil_div(nt, 4), 128, 0, st>>>(tile_box, tile_box, tile_color, ent, n, r, cap, rank, tol, base, kout,
                                               nt, tile_cap); ::hm::count_launch();
    if (max_rows > QR_WARP_ROWS) {
        const size_t smem = (size_t)std::min(qr64_rows, max_rows) * r * sizeof(double);
        HM_TRY(allow_smem(k_qr_smem<double>, (size_t)((int)smem)));
        k_qr_smem<double><<<(unsigned)nt, 512, smem, st>>>(tile_box, tile_box, tile_color, ent, n, r, cap, rank, tol,
                                                           base, kout, QR_WARP_ROWS, qr64_rows, tile_cap); ::hm::count_launch();
    }
    // taller tiles: the FP64 tall-skinny QR up to ts_max rows (each tile read
    // once; these QRs run to full width, r columns, so the tall-skinny blocks
    // add little FP64 work), the streaming block kernel beyond
    const int ts_rows = (200 * 1024) / (16 * r) / 32 * 32, ts_max = (200 * 1024) / (8 * r * r) * ts_rows;
    if (max_rows > qr64_rows && ts_max > qr64_rows) {
        DBuf ts_cnt, ts_off, blk_tile, blk_row0, blk_rows, rstack, taus;
        int64_t nblk = 0;
        HM_TRY(alloc(ts_cnt, (nt + 1) * sizeof(int64_t)));
        HM_TRY(alloc(ts_off, (nt + 1) * sizeof(int64_t)));
        k_ts_count<<<ceil_div(nt, 256), 256, 0, st>>>(tile_box, ent, nt, qr64_rows, ts_max, ts_rows,
                                                      ts_cnt.as<int64_t>()); ::hm::count_launch();
        HM_TRY(scan_exclusive(ts_cnt.as<int64_t>(), ts_off.as<int64_t>(), nt, st));
        HM_TRY(read_scalar(nblk, ts_off.as<int64_t>() + nt, st));
        if (nblk > 0) {
            HM_TRY(alloc(blk_tile, nblk * sizeof(int64_t)));
            HM_TRY(alloc(blk_row0, nblk * sizeof(int)));
            HM_TRY(alloc(blk_rows, nblk * sizeof(int)));
            HM_TRY(alloc(rstack, (size_t)nblk * r * r * sizeof(double)));
            HM_TRY(alloc(taus, (size_t)nblk * r * sizeof(double)));
            k_ts_fill<<<ceil_div(nt, 256), 256, 0, st>>>(tile_box, ent, ts_off.as<int64_t>(), nt,
                                                         blk_tile.as<int64_t>(), blk_row0.as<int>(),
                                                         blk_rows.as<int>()); ::hm::count_launch();
            const int nb_top = ceil_div(std::min(max_rows, ts_max), ts_rows);
            HM_TRY(allow_smem(k_ts_block<double>, (size_t)ts_rows * r * sizeof(double)));
            HM_TRY(allow_smem(k_ts_top<double>, (size_t)nb_top * r * r * sizeof(double)));
            HM_TRY(allow_smem(k_ts_form<double>, (size_t)2 * ts_rows * r * sizeof(double)));
            launch_ts<double>(tile_box, tile_box, tile_color, tile_cap, ent, n, r, cap, rank, tol, base, kout, nt,
                              nblk, nb_top, ts_rows, ts_off, blk_tile, blk_row0, blk_rows, rstack, taus, st);
        }
    }
    if (max_rows > std::max(qr64_rows, ts_max))
        k_qr_tiles<<<(unsigned)nt, 256, 0, st>>>(tile_box, tile_box, tile_color, ent, n, r, cap, rank, tol, base, kout,
                                                 std::max(qr64_rows, ts_max), tile_cap); ::hm::count_launch();
    HM_LAUNCH("qr_tiles_fp64");
    return ok();
}

Err bases_and_cores(hm_ctx *c, int level) {
    cudaStream_t st = c->st;
    Coloring &g = c->colorings[level];
    if ((int)c->factors.size() < c->L + 1) c->factors.resize(c->L + 1);
    Factors &f = c->factors[level];
    f = Factors();
    f.n_pairs = g.n_pairs;
    const int64_t np = g.n_pairs;
    const int r = c->cfg.r;
    const int64_t n = c->n;
    const Cut &cu = c->cuts[level];
    if (np == 0) {
        f.done = true;
        return ok();
    }
    // M = G_alpha^T P for every pair (tile p is read only by pair p), before the
    // tiles are factored in place
    if (r > 64) return fail(HM_ENOTSUP, "cores: r > 64");
    // HM_MIXED_BF16X6_F32: the three products and the solves in FP32 (P, U and V
    // carry FP32-class rounding already); FP64 otherwise.  The products are
    // summed over 32-row blocks first: one running FP32 sum over a 1024-row
    // chunk raised the compression error at 200k points from 5.1e-7 to 6.5e-7.
    const bool core32 = c->cfg.precision == HM_MIXED_BF16X6_F32;
    const size_t elem = core32 ? sizeof(float) : sizeof(double);
    const int nsplit = std::max(1, ceil_div(cu.max_rows, GRAM_CHUNK));
    const size_t part_elems = (size_t)nsplit * np * r * r;
    HM_TRY(ensure(c->scratch_a, part_elems * elem));
    gram_launcher(c)((unsigned)np, nsplit, st, g.pair_alpha.as<int>(),
                                                         cu.ent.as<int>(), r, c->GP.as<double>(),
                                                         c->cur.Y.as<double>(), g.pair_color.as<int>(), n, nullptr,
                                                         nullptr, c->scratch_a.p);
    HM_LAUNCH("gram M");
    // QR of every Y tile and every Z tile
    DBuf kY, kZ;
    HM_TRY(alloc(kY, np * sizeof(int)));
    HM_TRY(alloc(kZ, np * sizeof(int)));
    const int cap = c->kcap;  // r (fixed rank), or r - p and the rank cap (tolerance)
    // HM_MIXED_BF16X6_F32: tiles up to qr32_rows rows by the FP32 shared-memory
    // kernel, tiles up to ts_max rows by the FP32 tall-skinny QR, larger ones
    // by the FP64 block kernel.  FP64 modes: the warp kernel up to QR_WARP_ROWS
    // rows, the FP64 shared-memory kernel up to qr64_rows (200 KB of tile), the
    // block kernel beyond.  Tall-skinny blocks: the block and its composed Q
    // fit 200 KB of shared memory; the stacked R of a tile does too.
    const bool mixed = c->cfg.precision == HM_MIXED_BF16X6_F32;
    const int esz = mixed ? (int)sizeof(float) : (int)sizeof(double);
    const int qr32_rows = mixed ? std::min(QR32_MAX_ROWS, (200 * 1024) / (4 * r)) : 0;
    const int qr64_rows = mixed ? 0 : (200 * 1024) / (8 * r);
    const int ts_rows = (200 * 1024) / (2 * esz * r) / 32 * 32;  // rows per tall-skinny block
    // FP64 modes keep the direct pivoted QR on their tall tiles: the tall-skinny
    // blocks factor all r columns and form Q from r reflectors, about twice the
    // FP64 work of a pivoted QR that stops at k, which costs more on this GPU's
    // FP64 pipe than the tile re-reads it saves (measured on the 200k torus)
    const int ts_max = mixed ? (200 * 1024) / (esz * r * r) * ts_rows : 0;
    const int ts_min = mixed ? qr32_rows : std::max(QR_WARP_ROWS, qr64_rows);
    const int small_rows = std::max(ts_min, ts_max);
    const size_t qr32_smem = (size_t)std::max(1, std::min(qr32_rows, cu.max_rows)) * r * sizeof(float);
    const size_t qr64_smem = (size_t)std::max(1, std::min(qr64_rows, cu.max_rows)) * r * sizeof(double);
    if (mixed)
        HM_TRY(allow_smem(k_qr_smem<float>, (size_t)((int)qr32_smem)));
    else if (cu.max_rows > QR_WARP_ROWS)
        HM_TRY(allow_smem(k_qr_smem<double>, (size_t)((int)qr64_smem)));
    // tall-skinny blocks (the same for the Y and the Z tiles)
    DBuf ts_cnt, ts_off, blk_tile, blk_row0, blk_rows, rstack, taus;
    int64_t nblk = 0;
    int nb_top = 0;
    if (cu.max_rows > ts_min && ts_max > ts_min) {
        HM_TRY(alloc(ts_cnt, (np + 1) * sizeof(int64_t)));
        HM_TRY(alloc(ts_off, (np + 1) * sizeof(int64_t)));
        k_ts_count<<<ceil_div(np, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), cu.ent.as<int>(), np, ts_min, ts_max,
                                                      ts_rows, ts_cnt.as<int64_t>()); ::hm::count_launch();
        HM_TRY(scan_exclusive(ts_cnt.as<int64_t>(), ts_off.as<int64_t>(), np, st));
        HM_TRY(read_scalar(nblk, ts_off.as<int64_t>() + np, st));
        if (nblk > 0) {
            HM_TRY(alloc(blk_tile, nblk * sizeof(int64_t)));
            HM_TRY(alloc(blk_row0, nblk * sizeof(int)));
            HM_TRY(alloc(blk_rows, nblk * sizeof(int)));
            HM_TRY(alloc(rstack, (size_t)nblk * r * r * esz));
            HM_TRY(alloc(taus, (size_t)nblk * r * esz));
            k_ts_fill<<<ceil_div(np, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), cu.ent.as<int>(), ts_off.as<int64_t>(),
                                                         np, blk_tile.as<int64_t>(), blk_row0.as<int>(),
                                                         blk_rows.as<int>()); ::hm::count_launch();
            HM_LAUNCH("ts_fill");
            nb_top = ceil_div(std::min(cu.max_rows, ts_max), ts_rows);
            if (mixed) {
                HM_TRY(allow_smem(k_ts_block<float>, (size_t)ts_rows * r * esz));
                HM_TRY(allow_smem(k_ts_top<float>, (size_t)nb_top * r * r * esz));
                HM_TRY(allow_smem(k_ts_form<float>, (size_t)2 * ts_rows * r * esz));
            } else {
                HM_TRY(allow_smem(k_ts_block<double>, (size_t)ts_rows * r * esz));
                HM_TRY(allow_smem(k_ts_top<double>, (size_t)nb_top * r * r * esz));
                HM_TRY(allow_smem(k_ts_form<double>, (size_t)2 * ts_rows * r * esz));
            }
        }
    }
    for (int side = 0; side < 2; ++side) {
        double *T = side ? c->cur.Z.as<double>() : c->cur.Y.as<double>();
        int *kk = side ? kZ.as<int>() : kY.as<int>();
        if (cu.max_rows > small_rows) {
            k_qr_tiles<<<(int)np, 256, 0, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(), g.pair_color.as<int>(),
                                                cu.ent.as<int>(), n, r, cap, c->rank_fixed, c->tol, T, kk,
                                                small_rows); ::hm::count_launch();
        }
        if (nblk > 0) {
            (mixed ? launch_ts<float> : launch_ts<double>)(
                g.pair_alpha.as<int>(), cu.int_idx.as<int>(), g.pair_color.as<int>(), nullptr, cu.ent.as<int>(), n,
                r, cap, c->rank_fixed, c->tol, T, kk, np, nblk, nb_top, ts_rows, ts_off, blk_tile, blk_row0,
                blk_rows, rstack, taus, st);
            HM_LAUNCH("tall-skinny qr");
        }
        if (mixed) {
            // tiles up to 256 rows with 128 threads, taller ones with 512
            k_qr_smem<float><<<(int)np, 128, qr32_smem, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(),
                                                    g.pair_color.as<int>(), cu.ent.as<int>(), n, r, cap, c->rank_fixed,
                                                    c->tol, T, kk, 0, std::min(256, qr32_rows)); ::hm::count_launch();
            if (cu.max_rows > 256 && qr32_rows > 256) {
                k_qr_smem<float><<<(int)np, 512, qr32_smem, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(),
                                                        g.pair_color.as<int>(), cu.ent.as<int>(), n, r, cap,
                                                        c->rank_fixed, c->tol, T, kk, 256, qr32_rows); ::hm::count_launch();
            }
        } else {
            k_qr_warp<<<ceil_div(np, 4), 128, 0, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(),
                                                       g.pair_color.as<int>(), cu.ent.as<int>(), n, r, cap,
                                                       c->rank_fixed, c->tol, T, kk, np); ::hm::count_launch();
            if (cu.max_rows > QR_WARP_ROWS && qr64_rows > QR_WARP_ROWS) {
                k_qr_smem<double><<<(int)np, 512, qr64_smem, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(),
                                                                   g.pair_color.as<int>(), cu.ent.as<int>(), n, r,
                                                                   cap, c->rank_fixed, c->tol, T, kk, QR_WARP_ROWS,
                                                                   qr64_rows); ::hm::count_launch();
            }
        }
    }
    HM_LAUNCH("qr_tiles");
    HM_TRY(alloc(f.kU, np * sizeof(int)));
    HM_TRY(alloc(f.kV, np * sizeof(int)));
    DBuf sz;
    HM_TRY(alloc(sz, 3 * (np + 1) * sizeof(int64_t)));
    int64_t *sU = sz.as<int64_t>(), *sV = sU + (np + 1), *sB = sV + (np + 1);
    k_factor_sizes<<<ceil_div(np, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(),
                                                      g.pair_T.as<int>(), kY.as<int>(), kZ.as<int>(), cu.ent.as<int>(),
                                                      np, f.kU.as<int>(), f.kV.as<int>(), sU, sV, sB); ::hm::count_launch();
    HM_LAUNCH("factor_sizes");
    HM_TRY(alloc(f.offU, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(f.offV, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(f.offB, (np + 1) * sizeof(int64_t)));
    HM_TRY(scan_exclusive(sU, f.offU.as<int64_t>(), np, st));
    HM_TRY(scan_exclusive(sV, f.offV.as<int64_t>(), np, st));
    HM_TRY(scan_exclusive(sB, f.offB.as<int64_t>(), np, st));
    HM_TRY(read_scalar(f.nU, f.offU.as<int64_t>() + np, st));
    HM_TRY(read_scalar(f.nV, f.offV.as<int64_t>() + np, st));
    HM_TRY(read_scalar(f.nB, f.offB.as<int64_t>() + np, st));
    HM_TRY(alloc(f.U, std::max<int64_t>(f.nU, 1) * sizeof(double)));
    HM_TRY(alloc(f.V, std::max<int64_t>(f.nV, 1) * sizeof(double)));
    HM_TRY(alloc(f.B, std::max<int64_t>(f.nB, 1) * sizeof(double)));
    k_pack<<<(int)np, 128, 0, st>>>(g.pair_alpha.as<int>(), cu.int_idx.as<int>(), g.pair_color.as<int>(),
                                    g.pair_T.as<int>(), cu.ent.as<int>(), n, r, f.kU.as<int>(), f.kV.as<int>(),
                                    f.offU.as<int64_t>(), f.offV.as<int64_t>(), c->cur.Y.as<double>(),
                                    c->cur.Z.as<double>(), f.U.as<double>(), f.V.as<double>()); ::hm::count_launch();
    HM_LAUNCH("pack");
    const int kc = std::max(1, std::min(r, cap));
    // S1 = G_alpha^T U (Psi side) and S2 = G_beta^T V (Omega side)
    DBuf spart;
    HM_TRY(alloc(spart, 2 * part_elems * elem));
    void *S1part = spart.p;
    void *S2part = static_cast<unsigned char *>(spart.p) + part_elems * elem;
    gram_launcher(c)((unsigned)np, nsplit, st, g.pair_alpha.as<int>(),
                                                         cu.ent.as<int>(), r, c->GP.as<double>(), f.U.as<double>(),
                                                         nullptr, n, f.offU.as<int64_t>(), f.kU.as<int>(), S1part);
    gram_launcher(c)((unsigned)np, nsplit, st, cu.int_idx.as<int>(),
                                                         cu.ent.as<int>(), r, c->GO.as<double>(), f.V.as<double>(),
                                                         nullptr, n, f.offV.as<int64_t>(), f.kV.as<int>(), S2part);
    HM_LAUNCH("gram S");
    HM_TRY((core32 ? launch_core<float, float> : launch_core<double, double>)(np, nsplit, r, kc, st, f.kU.as<int>(), f.kV.as<int>(),
                                                               f.offB.as<int64_t>(), c->scratch_a.p, S1part, S2part,
                                                               f.B.as<double>()));
    HM_LAUNCH("core");
    std::vector<int> hk;
    HM_TRY(to_host(hk, f.kU.p, np, st));
    f.max_k = 0;
    for (int v : hk) f.max_k = std::max(f.max_k, v);
    HM_TRY(to_host(hk, f.kV.p, np, st));
    for (int v : hk) f.max_k = std::max(f.max_k, v);
    f.done = true;
    return ok();
}

// ---------------------------------------------------------------------------
// K11 leaf blocks
// ---------------------------------------------------------------------------

__global__ void k_leaf_sizes(const int *pair_alpha, const int *pair_col, const int *ent, int64_t np, int64_t *sz) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int *ea = ent + (int64_t)pair_alpha[p] * ENT_FIELDS, *eb = ent + (int64_t)pair_col[p] * ENT_FIELDS;
    sz[p] = (int64_t)(ea[4] - ea[3]) * (eb[4] - eb[3]);
}

__global__ void k_leaf_extract(const int *pair_alpha, const int *pair_col, const int *pair_color, const int *ent,
                               int64_t n, int m, const int64_t *off, const double *Y, double *D) {
    const int64_t p = blockIdx.x;
    const int *ea = ent + (int64_t)pair_alpha[p] * ENT_FIELDS, *eb = ent + (int64_t)pair_col[p] * ENT_FIELDS;
    const int ma = ea[4] - ea[3], mb = eb[4] - eb[3];
    const double *Yt = Y + ((int64_t)pair_color[p] * n + ea[3]) * m;
    for (int o = threadIdx.x; o < ma * mb; o += blockDim.x) D[off[p] + o] = Yt[(int64_t)(o / mb) * m + o % mb];
}

Err extract_leaf(hm_ctx *c) {
    cudaStream_t st = c->st;
    const Coloring &g = c->colorings[c->L + 1];
    const Cut &cu = c->cuts[c->L];
    Leaf &lf = c->leaf;
    lf = Leaf();
    lf.n_pairs = g.n_pairs;
    lf.m_max = g.m_cols;
    const int64_t np = g.n_pairs;
    DBuf sz;
    HM_TRY(alloc(sz, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(lf.offD, (np + 1) * sizeof(int64_t)));
    k_leaf_sizes<<<ceil_div(np, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), cu.near_idx.as<int>(), cu.ent.as<int>(), np,
                                                    sz.as<int64_t>()); ::hm::count_launch();
    HM_LAUNCH("leaf_sizes");
    HM_TRY(scan_exclusive(sz.as<int64_t>(), lf.offD.as<int64_t>(), np, st));
    HM_TRY(read_scalar(lf.nD, lf.offD.as<int64_t>() + np, st));
    HM_TRY(alloc(lf.D, std::max<int64_t>(lf.nD, 1) * sizeof(double)));
    k_leaf_extract<<<(int)np, 128, 0, st>>>(g.pair_alpha.as<int>(), cu.near_idx.as<int>(), g.pair_color.as<int>(),
                                            cu.ent.as<int>(), c->n, g.m_cols, lf.offD.as<int64_t>(),
                                            c->cur.Y.as<double>(), lf.D.as<double>()); ::hm::count_launch();
    HM_LAUNCH("leaf_extract");
    lf.done = true;
    return ok();
}

}  // namespace hm
