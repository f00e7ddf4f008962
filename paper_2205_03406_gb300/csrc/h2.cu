// H^2 compression (Section 4.3, Algorithm 4.2) and the apply of the nested
// representation (Algorithm 4.3).
//
// Per cut l = 2..L, on top of the two stages of the uniform H^1 compression
// (uniform.cu):
//   stage 1  Y = A Omega - A^(l-1) Omega on the box colouring; the sample of
//            every entry a, P_a = Y(I_a, colour of a) (zero without one), is
//            augmented by the far field of its parent t in cut l-1:
//                P_a += U_t(I_{t,a}, :) diag(S^in_t) G_t,   G_t = U_t^T Gamma_t,
//            with Gamma_t an |I_t| x r Philox Gaussian (side 4, level l, box t);
//            [U_a, S^in_a] = svd(P_a, k);
//   stage 2  Psi(I_a) = U_a on the pair colouring, Z = A^* Psi - A^(l-1)* Psi;
//            W_b = sum over a in int(b) of Z(I_b, colour of (b, a))[:, 0:k_a] M_a,
//            M_a = U_a^T Gamma'_a (side 6), plus V_t(I_{t,b}, :) diag(S^out_t)
//            V_t^T Gamma''_t (side 5); [V_b, S^out_b] = svd(W_b, k);
//            B_ab = Z(I_b, ...)^T V_b;
//   nesting  the short bases of cut l-1, U~_t(rows of a) = U_a^T U_t(I_{t,a}, :)
//            (eq. nested_basis with orthonormal U_a), then the bases of every
//            coarser cut are re-expanded through the chain, diag(U_a) U~_t, so
//            that the peel of the next level subtracts the nested operator.
//
// svd(P, k): column-pivoted QR P = Q R (basis.cu), R = Q^T P, one-sided Jacobi
// on the columns of R (Hestenes: R X = W Sigma), U = Q W(:, 0:k), each column
// signed so that its entry of largest magnitude is positive.  k follows the
// rank or tolerance rule on the singular values (k <= |I_a|, r, and the cap).
// Every product here is FP64.
//
// After the leaf blocks, only the long bases of cut L, the short bases, the
// cores and the leaf blocks are kept; the apply runs the upward pass
// (outgoing expansions), the cores of every level, the downward pass
// (incoming expansions) and the near field.
#include "ctx.cuh"
#include "philox.cuh"

#include <algorithm>

namespace hm {

namespace h2k {

constexpr int SIDE_AUG_U = 4, SIDE_AUG_V = 5, SIDE_MIX = 6;
constexpr int JAC_THREADS = 512;
constexpr int JAC_SWEEPS = 40;
constexpr int MAXR = 64;

// Gamma[i][j] = gauss(seed, side, key_level, gid(entry of i), row of i in it, j)
__global__ void k_gamma(int64_t n, int r, const int *pt2ent, const int *ent, int key_level, int side,
                        unsigned long long seed, double *out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n * r) return;
    const int64_t i = t / r;
    const int j = (int)(t - i * r);
    const int *e = ent + (int64_t)pt2ent[i] * ENT_FIELDS;
    out[t] = gauss(seed, side, key_level, e[2], (int)(i - e[3]), j);
}

// G_e = B_e^T Gamma(I_e, :) (k_e x r) for every entry e with k_e > 0
__global__ void k_proj(int nc, const int *ent, const int *k, const int64_t *eoff, const double *B, const double *Gam,
                       int r, const int64_t *goff, double *G) {
    const int e = blockIdx.x;
    if (e >= nc) return;
    const int ke = k[e];
    if (ke == 0) return;
    const int *en = ent + (int64_t)e * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const double *Be = B + eoff[e];
    for (int o = threadIdx.x; o < ke * r; o += blockDim.x) {
        const int u = o / r, j = o - u * r;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(Be[(int64_t)i * ke + u], Gam[(int64_t)(s0 + i) * r + j], acc);
        G[goff[e] + o] = acc;
    }
}

// P(I_a, :) = Y[colour of a](I_a, :) for the box vertices a (P is zero elsewhere)
__global__ void k_gather(const int *vbox, const int *vcolor, int64_t nv, const int *ent, const double *Y, int64_t n,
                         int r, double *P) {
    const int64_t v = blockIdx.x;
    if (v >= nv) return;
    const int *en = ent + (int64_t)vbox[v] * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const double *T = Y + ((int64_t)vcolor[v] * n + s0) * r;
    for (int o = threadIdx.x; o < m * r; o += blockDim.x) P[(int64_t)s0 * r + o] = T[o];
}

// P(I_a, :) += B_t(I_{t,a}, :) diag(S_t) G_t for the parent t of a (k_t > 0)
__global__ void k_augment(int nc, const int *ent, const int *parent, const int *ent_p, const int *kp,
                          const int64_t *eoffp, const double *Bp, const double *Sp, int sidx, const int64_t *goffp,
                          const double *Gp, int r, double *P) {
    const int a = blockIdx.x;
    if (a >= nc) return;
    const int t = parent[a];
    const int kt = kp[t];
    if (kt == 0) return;
    const int *en = ent + (int64_t)a * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const int i0 = s0 - ent_p[(int64_t)t * ENT_FIELDS + 3];
    const double *Bt = Bp + eoffp[t] + (int64_t)i0 * kt;
    const double *St = Sp + ((int64_t)t * 2 + sidx) * r;
    const double *Gt = Gp + goffp[t];
    for (int o = threadIdx.x; o < m * r; o += blockDim.x) {
        const int i = o / r, j = o - i * r;
        double acc = P[(int64_t)s0 * r + o];
        for (int u = 0; u < kt; ++u) acc = fma(Bt[(int64_t)i * kt + u], St[u] * Gt[(int64_t)u * r + j], acc);
        P[(int64_t)s0 * r + o] = acc;
    }
}

// R_p = Q^T P on tile p (kq_p x r, rows kq_p.. zero), Q in Pq's first kq_p columns
__global__ void k_rmat(int64_t nt, const int *tiles, const int *ent, const int *kq, const double *Q, const double *P,
                       int r, double *R) {
    const int64_t p = blockIdx.x;
    if (p >= nt) return;
    const int *en = ent + (int64_t)tiles[p] * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const int k = kq[p];
    double *Rp = R + p * r * r;
    for (int o = threadIdx.x; o < r * r; o += blockDim.x) {
        const int u = o / r, j = o - u * r;
        double acc = 0.0;
        if (u < k)
            for (int i = 0; i < m; ++i)
                acc = fma(Q[(int64_t)(s0 + i) * r + u], P[(int64_t)(s0 + i) * r + j], acc);
        Rp[o] = acc;
    }
}

// One-sided Jacobi SVD of R_p (kq rows, r columns) in shared memory: cyclic
// sweeps in round-robin order (r/2 disjoint column pairs per round, one warp
// each) rotate every pair whose inner product exceeds thresh sqrt(a b) (pairs
// with a negligible column excepted) until a sweep rotates none (at most
// JAC_SWEEPS).  Then sigma_j = |column j|, sorted
// in decreasing order (lower index first on ties); W_p(:, q) = column / sigma
// (zero where sigma is 0); k by the rank or tolerance rule.
__global__ void __launch_bounds__(JAC_THREADS) k_jacobi(int64_t nt, const int *tiles, const int *ent, const int *kq,
                                                       int r, int cap, int rank, double tol, const double *R,
                                                       double *W, double *sig, int *kout) {
    __shared__ double A[MAXR * MAXR];  // column j at A[j * MAXR + u]
    __shared__ double nrm[MAXR];
    __shared__ int order[MAXR];
    __shared__ int rotated;
    const int64_t p = blockIdx.x;
    if (p >= nt) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    const int kr = kq[p];
    const int *en = ent + (int64_t)tiles[p] * ENT_FIELDS;
    const int m = en[4] - en[3];
    const double *Rp = R + p * r * r;
    for (int o = tid; o < r * MAXR; o += blockDim.x) {
        const int j = o / MAXR, u = o - j * MAXR;
        A[j * MAXR + u] = u < kr ? Rp[(int64_t)u * r + j] : 0.0;
    }
    __syncthreads();
    const int rr = r + (r & 1);  // a padding column when r is odd
    // a pair is orthogonal once |a_p . a_q| <= thresh |a_p| |a_q| with thresh
    // above the rounding of a kr-term dot product; a column whose squared norm
    // is below 1e-30 of |R|_F^2 (invariant under the rotations) lies far below
    // any truncation and is not rotated
    const double thresh = 4e-16 * (double)(kr > 0 ? kr : 1);
    if (tid < 32) {
        double f = 0.0;
        for (int o = tid; o < r * kr; o += 32) {
            const double v = A[(o / kr) * MAXR + o % kr];
            f = fma(v, v, f);
        }
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (tid == 0) nrm[0] = f;
    }
    __syncthreads();
    const double negligible = 1e-30 * nrm[0];
    __syncthreads();
    for (int sweep = 0; sweep < JAC_SWEEPS; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < rr - 1; ++round) {
            for (int q = warp; q < rr / 2; q += nw) {
                // circle method: position 0 fixed, positions 1..rr-1 rotate
                const int pa = q == 0 ? 0 : 1 + (q - 1 + round) % (rr - 1);
                const int pb = 1 + (rr - 2 - q + round) % (rr - 1);
                if (pa >= r || pb >= r) continue;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int u = lane; u < kr; u += 32) {
                    const double x = A[pa * MAXR + u], y = A[pb * MAXR + u];
                    a = fma(x, x, a);
                    b = fma(y, y, b);
                    g = fma(x, y, g);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (!(a > negligible && b > negligible) || !(fabs(g) > thresh * sqrt(a * b))) continue;
                const double zeta = (b - a) / (2.0 * g);
                double t;
                if (fabs(zeta) > 1e150) t = 0.5 / zeta;
                else t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int u = lane; u < kr; u += 32) {
                    const double x = A[pa * MAXR + u], y = A[pb * MAXR + u];
                    A[pa * MAXR + u] = cs * x - sn * y;
                    A[pb * MAXR + u] = sn * x + cs * y;
                }
                if (lane == 0) rotated = 1;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    for (int j = tid; j < r; j += blockDim.x) {
        double a = 0.0;
        for (int u = 0; u < kr; ++u) a = fma(A[j * MAXR + u], A[j * MAXR + u], a);
        nrm[j] = sqrt(a);
    }
    __syncthreads();
    for (int j = tid; j < r; j += blockDim.x) {
        int pos = 0;
        for (int i = 0; i < r; ++i) pos += (nrm[i] > nrm[j] || (nrm[i] == nrm[j] && i < j)) ? 1 : 0;
        order[pos] = j;
    }
    __syncthreads();
    const int kmax = min(min(kr, m), min(r, cap));
    int k;
    if (rank > 0) {
        k = min(rank, kmax);
    } else if (!(nrm[order[0]] > 0.0)) {
        k = 0;
    } else {
        int cnt = 0;
        for (int q = 0; q < r; ++q) cnt += nrm[order[q]] > tol * nrm[order[0]] ? 1 : 0;
        k = min(cnt, kmax);
    }
    double *Wp = W + p * r * r;  // W_p(u, q) at u * r + q
    for (int o = tid; o < r * r; o += blockDim.x) {
        const int u = o / r, q = o - u * r;
        const int j = order[q];
        const double sg = nrm[j];
        Wp[o] = (u < kr && q < k && sg > 0.0) ? A[j * MAXR + u] / sg : 0.0;
    }
    for (int q = tid; q < r; q += blockDim.x) sig[p * r + q] = nrm[order[q]];
    if (tid == 0) kout[p] = k;
}

// per entry: its k (0 for entries that are not tiles) and |I_e| k_e
__global__ void k_scatter_k(int64_t nt, const int *tiles, const int *kt, const int *ent, int *ek, int64_t *sz) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nt) return;
    const int e = tiles[p];
    const int *en = ent + (int64_t)e * ENT_FIELDS;
    ek[e] = kt[p];
    sz[e] = (int64_t)(en[4] - en[3]) * kt[p];
}

// U_e = Q W_p(:, 0:k) into the arena, every column signed so that its entry of
// largest magnitude (the first on ties) is positive; S[e][sidx] = sigma(0:k)
__global__ void k_rotate(int64_t nt, const int *tiles, const int *ent, const int *kq, const int *kt, const double *Q,
                         int r, const double *W, const double *sig, const int64_t *eoff, double *U, double *S,
                         int sidx) {
    const int64_t p = blockIdx.x;
    if (p >= nt) return;
    const int e = tiles[p];
    const int *en = ent + (int64_t)e * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const int k = kt[p], kr = kq[p];
    const double *Wp = W + p * r * r;
    double *Ue = U + eoff[e];
    for (int o = threadIdx.x; o < m * k; o += blockDim.x) {
        const int i = o / k, q = o - i * k;
        double acc = 0.0;
        for (int u = 0; u < kr; ++u) acc = fma(Q[(int64_t)(s0 + i) * r + u], Wp[u * r + q], acc);
        Ue[o] = acc;
    }
    for (int q = threadIdx.x; q < k; q += blockDim.x) S[((int64_t)e * 2 + sidx) * r + q] = sig[p * r + q];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < k; q += nw) {
        double best = -1.0;
        int bi = 1 << 30;
        for (int i = lane; i < m; i += 32) {
            const double v = fabs(Ue[(int64_t)i * k + q]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const bool flip = bi < m && Ue[(int64_t)bi * k + q] < 0.0;
        __syncwarp();
        if (flip)
            for (int i = lane; i < m; i += 32) Ue[(int64_t)i * k + q] = -Ue[(int64_t)i * k + q];
    }
}

// Psi(I_e, :) = [U_e 0] for every entry with a basis
__global__ void k_fill(int nc, const int *ent, const int *k, const int64_t *eoff, const double *U, int r, double *G) {
    const int e = blockIdx.x;
    if (e >= nc) return;
    const int ke = k[e];
    if (ke == 0) return;
    const int *en = ent + (int64_t)e * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    for (int o = threadIdx.x; o < m * r; o += blockDim.x) {
        const int i = o / r, j = o - i * r;
        G[(int64_t)s0 * r + o] = j < ke ? U[eoff[e] + (int64_t)i * ke + j] : 0.0;
    }
}

// sizes of the short blocks: child a of cut l, parent t: k_a x k_t
__global__ void k_short_sizes(int nc, const int *parent, const int *kc, const int *kp, int64_t *sz) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < nc) sz[a] = (int64_t)kc[a] * kp[parent[a]];
}

// T[a] = U_a^T U_t(I_{t,a}, :) (k_a x k_t), the short basis block of child a
__global__ void k_nest(int nc, const int *ent, const int *parent, const int *ent_p, const int *kp,
                       const int64_t *eoffp, const double *Bp, const int *kc, const int64_t *eoffc, const double *Bc,
                       const int64_t *offT, double *T) {
    const int a = blockIdx.x;
    if (a >= nc) return;
    const int t = parent[a];
    const int kt = kp[t], ka = kc[a];
    if (kt == 0 || ka == 0) return;
    const int *en = ent + (int64_t)a * ENT_FIELDS;
    const int m = en[4] - en[3];
    const int i0 = en[3] - ent_p[(int64_t)t * ENT_FIELDS + 3];
    const double *Ba = Bc + eoffc[a];
    const double *Bt = Bp + eoffp[t] + (int64_t)i0 * kt;
    for (int o = threadIdx.x; o < ka * kt; o += blockDim.x) {
        const int u = o / kt, w = o - u * kt;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(Ba[(int64_t)i * ka + u], Bt[(int64_t)i * kt + w], acc);
        T[offT[a] + o] = acc;
    }
}

// the nested basis of the parent on the rows of child a: B_t(I_{t,a}, :) = B_a T[a]
__global__ void k_expand(int nc, const int *ent, const int *parent, const int *ent_p, const int *kp,
                         const int64_t *eoffp, double *Bp, const int *kc, const int64_t *eoffc, const double *Bc,
                         const int64_t *offT, const double *T) {
    const int a = blockIdx.x;
    if (a >= nc) return;
    const int t = parent[a];
    const int kt = kp[t], ka = kc[a];
    if (kt == 0) return;
    const int *en = ent + (int64_t)a * ENT_FIELDS;
    const int m = en[4] - en[3];
    const int i0 = en[3] - ent_p[(int64_t)t * ENT_FIELDS + 3];
    double *Bt = Bp + eoffp[t] + (int64_t)i0 * kt;
    const double *Ba = Bc + eoffc[a];
    for (int o = threadIdx.x; o < m * kt; o += blockDim.x) {
        const int i = o / kt, w = o - i * kt;
        double acc = 0.0;
        for (int u = 0; u < ka; ++u) acc = fma(Ba[(int64_t)i * ka + u], T[offT[a] + (int64_t)u * kt + w], acc);
        Bt[o] = acc;
    }
}

__global__ void k_kr_sizes(int nc, const int *k, int r, int64_t *sz) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nc) sz[e] = (int64_t)k[e] * r;
}

__global__ void k_iota(int nc, int *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nc) out[e] = e;
}

__global__ void k_k_sizes(int nc, const int *k, int64_t *sz) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nc) sz[e] = k[e];
}

// ---- apply (Algorithm 4.3); expansions are [sum of k][nrhs] per level ----

// outgoing expansions of the finest cut: q_e = B_e^T x(I_e)
__global__ void k_ap_out(int nc, const int *ent, const int *k, const int64_t *eoff, const double *B, const double *x,
                         int nrhs, const int64_t *qoff, double *q) {
    const int e = blockIdx.x;
    if (e >= nc) return;
    const int ke = k[e];
    if (ke == 0) return;
    const int *en = ent + (int64_t)e * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const double *Be = B + eoff[e];
    for (int o = threadIdx.x; o < ke * nrhs; o += blockDim.x) {
        const int u = o / nrhs, j = o - u * nrhs;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(Be[(int64_t)i * ke + u], x[(int64_t)(s0 + i) * nrhs + j], acc);
        q[qoff[e] * nrhs + o] = acc;
    }
}

// upward pass: q_t = sum over the children a of t of T[a]^T q_a
__global__ void k_ap_up(int nc, const int *kp, const int64_t *qoffp, double *qp, const int *kid_begin,
                        const int *kid_end, const int *kc, const int64_t *qoffc, const double *qc, const int64_t *offT,
                        const double *T, int nrhs) {
    const int t = blockIdx.x;
    if (t >= nc) return;
    const int kt = kp[t];
    if (kt == 0) return;
    for (int o = threadIdx.x; o < kt * nrhs; o += blockDim.x) {
        const int w = o / nrhs, j = o - w * nrhs;
        double acc = 0.0;
        for (int a = kid_begin[t]; a < kid_end[t]; ++a) {
            const int ka = kc[a];
            const double *Ta = T + offT[a];
            for (int u = 0; u < ka; ++u) acc = fma(Ta[(int64_t)u * kt + w], qc[(qoffc[a] + u) * nrhs + j], acc);
        }
        qp[qoffp[t] * nrhs + o] = acc;
    }
}

// cores: u_e = sum over b in int(e) of B_(e,b) q_b (trans: B_(b,e)^T q_b)
__global__ void k_ap_far(int nc, const int *int_ptr, const int *int_idx, const int *pairT, const int *pkU,
                         const int *pkV, const int64_t *offB, const double *B, int trans, const int64_t *qoff,
                         const double *q, const int *kout, const int64_t *uoff, double *u, int nrhs) {
    const int e = blockIdx.x;
    if (e >= nc) return;
    const int ke = kout[e];
    for (int o = threadIdx.x; o < ke * nrhs; o += blockDim.x) {
        const int a = o / nrhs, j = o - a * nrhs;
        double acc = 0.0;
        for (int t = int_ptr[e]; t < int_ptr[e + 1]; ++t) {
            const int b = int_idx[t];
            const double *qb = q + qoff[b] * nrhs + j;
            if (!trans) {
                const int kv = pkV[t];
                const double *Bp = B + offB[t] + (int64_t)a * kv;
                for (int w = 0; w < kv; ++w) acc = fma(Bp[w], qb[(int64_t)w * nrhs], acc);
            } else {
                const int p = pairT[t];
                const int ku = pkU[p], kv = pkV[p];
                const double *Bp = B + offB[p] + a;
                for (int w = 0; w < ku; ++w) acc = fma(Bp[(int64_t)w * kv], qb[(int64_t)w * nrhs], acc);
            }
        }
        u[uoff[e] * nrhs + o] = acc;
    }
}

// downward pass: u_a += T[a] u_t for the parent t of a
__global__ void k_ap_down(int nc, const int *parent, const int *kc, const int64_t *uoffc, double *uc, const int *kp,
                          const int64_t *uoffp, const double *up, const int64_t *offT, const double *T, int nrhs) {
    const int a = blockIdx.x;
    if (a >= nc) return;
    const int t = parent[a];
    const int kt = kp[t], ka = kc[a];
    if (kt == 0 || ka == 0) return;
    const double *Ta = T + offT[a];
    for (int o = threadIdx.x; o < ka * nrhs; o += blockDim.x) {
        const int v = o / nrhs, j = o - v * nrhs;
        double acc = 0.0;
        for (int w = 0; w < kt; ++w) acc = fma(Ta[(int64_t)v * kt + w], up[(uoffp[t] + w) * nrhs + j], acc);
        uc[uoffc[a] * nrhs + o] += acc;
    }
}

// incoming expansions of the finest cut: y(I_e) += B_e u_e
__global__ void k_ap_in(int nc, const int *ent, const int *k, const int64_t *eoff, const double *B,
                        const int64_t *uoff, const double *u, int nrhs, double *y) {
    const int e = blockIdx.x;
    if (e >= nc) return;
    const int ke = k[e];
    if (ke == 0) return;
    const int *en = ent + (int64_t)e * ENT_FIELDS;
    const int s0 = en[3], m = en[4] - en[3];
    const double *Be = B + eoff[e];
    for (int o = threadIdx.x; o < m * nrhs; o += blockDim.x) {
        const int i = o / nrhs, j = o - i * nrhs;
        double acc = 0.0;
        for (int a = 0; a < ke; ++a) acc = fma(Be[(int64_t)i * ke + a], u[(uoff[e] + a) * nrhs + j], acc);
        y[(int64_t)(s0 + i) * nrhs + j] += acc;
    }
}

}  // namespace h2k


namespace {

using namespace h2k;

// G_e = B_e^T Gamma(I_e, :) for the entries of cut cl, Gamma drawn per entry of
// cut cl with (side, key_level); goff = offsets of the k_e x r blocks
Err project_gauss(hm_ctx *c, int cl, int key_level, int side, const DBuf &ek, const DBuf &eoff, const DBuf &B,
                  DBuf &goff, DBuf &G) {
    cudaStream_t st = c->st;
    const Cut &cu = c->cuts[cl];
    const int r = c->cfg.r, nc = cu.nc;
    const int64_t n = c->n;
    DBuf Gam, sz;
    HM_TRY(alloc(Gam, (size_t)n * r * sizeof(double)));
    k_gamma<<<ceil_div(n * r, 256), 256, 0, st>>>(n, r, cu.pt2ent.as<int>(), cu.ent.as<int>(), key_level, side,
                                                  (unsigned long long)c->cfg.seed, Gam.as<double>()); ::hm::count_launch();
    HM_TRY(alloc(sz, ((size_t)nc + 1) * sizeof(int64_t)));
    HM_TRY(alloc(goff, ((size_t)nc + 1) * sizeof(int64_t)));
    k_kr_sizes<<<ceil_div(nc, 256), 256, 0, st>>>(nc, ek.as<int>(), r, sz.as<int64_t>()); ::hm::count_launch();
    HM_TRY(scan_exclusive(sz.as<int64_t>(), goff.as<int64_t>(), nc, st));
    int64_t tot = 0;
    HM_TRY(read_scalar(tot, goff.as<int64_t>() + nc, st));
    HM_TRY(alloc(G, (size_t)std::max<int64_t>(tot, 1) * sizeof(double)));
    k_proj<<<(unsigned)nc, 128, 0, st>>>(nc, cu.ent.as<int>(), ek.as<int>(), eoff.as<int64_t>(), B.as<double>(),
                                         Gam.as<double>(), r, goff.as<int64_t>(), G.as<double>()); ::hm::count_launch();
    HM_LAUNCH("H2 sketch projection");
    return ok();
}

// [U_e, S_e] = svd(P(I_e, :), k) for the entries htiles of cut l: per-entry
// ranks ek (0 elsewhere), offsets eoff, bases in arena, singular values into
// eS[e][sidx]
Err svd_tiles(hm_ctx *c, int l, const std::vector<int> &htiles, const double *P, int sidx, DBuf &ek, DBuf &eoff,
              DBuf &arena, int64_t &narena, DBuf &eS) {
    cudaStream_t st = c->st;
    const Cut &cu = c->cuts[l];
    const int nc = cu.nc, r = c->cfg.r;
    const int64_t n = c->n, nt = (int64_t)htiles.size();
    DBuf sz, tiles, zeros, Pq, kq, R, W, sig, kt;
    HM_TRY(alloc(ek, (size_t)nc * sizeof(int)));
    HM_CUDA(cudaMemsetAsync(ek.p, 0, (size_t)nc * sizeof(int), st));
    HM_TRY(alloc(eoff, ((size_t)nc + 1) * sizeof(int64_t)));
    HM_TRY(alloc(sz, ((size_t)nc + 1) * sizeof(int64_t)));
    HM_CUDA(cudaMemsetAsync(sz.p, 0, ((size_t)nc + 1) * sizeof(int64_t), st));
    if (nt > 0) {
        HM_TRY(to_dev(tiles, htiles, st));
        HM_TRY(alloc(zeros, (size_t)nt * sizeof(int)));
        HM_CUDA(cudaMemsetAsync(zeros.p, 0, (size_t)nt * sizeof(int), st));
        HM_TRY(alloc(Pq, (size_t)n * r * sizeof(double)));
        HM_CUDA(cudaMemcpyAsync(Pq.p, P, (size_t)n * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
        HM_TRY(alloc(kq, (size_t)nt * sizeof(int)));
        // Q: pivoted QR without truncation (k = min(|I_e|, r))
        HM_TRY(qr_tiles_fp64(c, l, tiles.as<int>(), zeros.as<int>(), nullptr, nt, cu.max_rows, Pq.as<double>(), r, r,
                             0.0, kq.as<int>()));
        HM_TRY(alloc(R, (size_t)nt * r * r * sizeof(double)));
        k_rmat<<<(unsigned)nt, 256, 0, st>>>(nt, tiles.as<int>(), cu.ent.as<int>(), kq.as<int>(), Pq.as<double>(), P, r,
                                             R.as<double>()); ::hm::count_launch();
        HM_TRY(alloc(W, (size_t)nt * r * r * sizeof(double)));
        HM_TRY(alloc(sig, (size_t)nt * r * sizeof(double)));
        HM_TRY(alloc(kt, (size_t)nt * sizeof(int)));
        k_jacobi<<<(unsigned)nt, JAC_THREADS, 0, st>>>(nt, tiles.as<int>(), cu.ent.as<int>(), kq.as<int>(), r, c->kcap,
                                                       c->rank_fixed, c->tol, R.as<double>(), W.as<double>(),
                                                       sig.as<double>(), kt.as<int>()); ::hm::count_launch();
        k_scatter_k<<<ceil_div(nt, 256), 256, 0, st>>>(nt, tiles.as<int>(), kt.as<int>(), cu.ent.as<int>(),
                                                        ek.as<int>(), sz.as<int64_t>()); ::hm::count_launch();
        HM_LAUNCH("H2 svd");
    }
    HM_TRY(scan_exclusive(sz.as<int64_t>(), eoff.as<int64_t>(), nc, st));
    HM_TRY(read_scalar(narena, eoff.as<int64_t>() + nc, st));
    HM_TRY(alloc(arena, (size_t)std::max<int64_t>(narena, 1) * sizeof(double)));
    if (nt > 0) {
        k_rotate<<<(unsigned)nt, 256, 0, st>>>(nt, tiles.as<int>(), cu.ent.as<int>(), kq.as<int>(), kt.as<int>(),
                                               Pq.as<double>(), r, W.as<double>(), sig.as<double>(),
                                               eoff.as<int64_t>(), arena.as<double>(), eS.as<double>(), sidx); ::hm::count_launch();
        HM_LAUNCH("H2 bases");
    }
    return ok();
}

// short bases of cut l-1 from the long bases of cut l, then the bases of cuts
// l-1 .. 2 re-expanded through the nested chain
Err nest_and_expand(hm_ctx *c, int l) {
    cudaStream_t st = c->st;
    Factors &f = c->factors[l];
    Factors &fp = c->factors[l - 1];
    const Cut &cu = c->cuts[l];
    const int nc = cu.nc;
    for (int side = 0; side < 2; ++side) {
        const DBuf &kc = side ? f.ekV : f.ekU, &kp = side ? fp.ekV : fp.ekU;
        const DBuf &oc = side ? f.eoffV : f.eoffU, &op = side ? fp.eoffV : fp.eoffU;
        const DBuf &Bc = side ? f.V : f.U, &Bp = side ? fp.V : fp.U;
        DBuf &offT = side ? fp.offVt : fp.offUt;
        DBuf &T = side ? fp.Vt : fp.Ut;
        int64_t &nT = side ? fp.nVt : fp.nUt;
        DBuf sz;
        HM_TRY(alloc(sz, ((size_t)nc + 1) * sizeof(int64_t)));
        HM_TRY(alloc(offT, ((size_t)nc + 1) * sizeof(int64_t)));
        k_short_sizes<<<ceil_div(nc, 256), 256, 0, st>>>(nc, cu.parent.as<int>(), kc.as<int>(), kp.as<int>(),
                                                         sz.as<int64_t>()); ::hm::count_launch();
        HM_TRY(scan_exclusive(sz.as<int64_t>(), offT.as<int64_t>(), nc, st));
        HM_TRY(read_scalar(nT, offT.as<int64_t>() + nc, st));
        HM_TRY(alloc(T, (size_t)std::max<int64_t>(nT, 1) * sizeof(double)));
        k_nest<<<(unsigned)nc, 128, 0, st>>>(nc, cu.ent.as<int>(), cu.parent.as<int>(), c->cuts[l - 1].ent.as<int>(),
                                             kp.as<int>(), op.as<int64_t>(), Bp.as<double>(), kc.as<int>(),
                                             oc.as<int64_t>(), Bc.as<double>(), offT.as<int64_t>(), T.as<double>()); ::hm::count_launch();
        HM_LAUNCH("H2 nest");
    }
    for (int j = l - 1; j >= 2; --j) {
        Factors &fj = c->factors[j], &fc = c->factors[j + 1];
        if (!fj.has_bases || !fc.has_bases) break;
        const Cut &cc = c->cuts[j + 1];
        for (int side = 0; side < 2; ++side) {
            k_expand<<<(unsigned)cc.nc, 128, 0, st>>>(
                cc.nc, cc.ent.as<int>(), cc.parent.as<int>(), c->cuts[j].ent.as<int>(),
                (side ? fj.ekV : fj.ekU).as<int>(), (side ? fj.eoffV : fj.eoffU).as<int64_t>(),
                (side ? fj.V : fj.U).as<double>(), (side ? fc.ekV : fc.ekU).as<int>(),
                (side ? fc.eoffV : fc.eoffU).as<int64_t>(), (side ? fc.V : fc.U).as<double>(),
                (side ? fj.offVt : fj.offUt).as<int64_t>(), (side ? fj.Vt : fj.Ut).as<double>()); ::hm::count_launch();
        }
        HM_LAUNCH("H2 expand");
        // the peel's reduced-precision copies of these bases are stale now
        fj.U2.release();
        fj.V2.release();
        fj.U32.release();
        fj.V32.release();
    }
    return ok();
}

// device time of a region on a stream, added to *acc (CUDA events)
struct PhaseTimer {
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    double *acc;
    PhaseTimer(cudaStream_t s, double *x) : st(s), acc(x) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
    }
    ~PhaseTimer() {
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        if (acc && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) *acc += ms * 1e-3;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

Err h2_level(hm_ctx *c, const hm_op *op, int l, double *phase_secs) {
    using namespace h2k;
    cudaStream_t st = c->st;
    const Cut &cu = c->cuts[l];
    const int nc = cu.nc, r = c->cfg.r;
    const int64_t n = c->n;
    if (r > MAXR) return fail(HM_ENOTSUP, "H^2: r above 64");
    Coloring &gp = c->colorings[l];
    Coloring &gb = c->box_colorings[l];
    const int64_t np = gp.n_pairs;
    const int64_t nv = (np > 0 && gp.n_colors > 0 && gb.done) ? gb.n_vertices : 0;
    if (np > 0 && nv == 0) return fail(HM_ESTATE, "H^2: level has pairs but no box colouring");
    Factors &f = c->factors[l];
    f = Factors();
    f.n_pairs = np;
    f.nc = nc;
    const bool has_prev = l > 2 && c->factors[l - 1].has_bases;
    Factors *fp = has_prev ? &c->factors[l - 1] : nullptr;
    auto ph = [&](int k) { return phase_secs ? phase_secs + k : nullptr; };

    // entries that get a column basis (a sample, or a parent's far field) and a row basis
    std::vector<int> hvbox, hpar, hkpU, hkpV;
    std::vector<char> vert((size_t)nc, 0);
    if (nv > 0) {
        HM_TRY(to_host(hvbox, gb.pair_alpha.p, nv, st));
        for (int b : hvbox) vert[b] = 1;
    }
    if (has_prev) {
        HM_TRY(to_host(hpar, cu.parent.p, nc, st));
        HM_TRY(to_host(hkpU, fp->ekU.p, fp->nc, st));
        HM_TRY(to_host(hkpV, fp->ekV.p, fp->nc, st));
    }
    std::vector<int> tU, tV;
    for (int e = 0; e < nc; ++e) {
        if (vert[e] || (has_prev && hkpU[hpar[e]] > 0)) tU.push_back(e);
        if (vert[e] || (has_prev && hkpV[hpar[e]] > 0)) tV.push_back(e);
    }
    DBuf P, Wb, ident;
    HM_TRY(alloc(P, (size_t)n * r * sizeof(double)));
    HM_CUDA(cudaMemsetAsync(P.p, 0, (size_t)n * r * sizeof(double), st));
    HM_TRY(alloc(ident, (size_t)std::max(nc, 1) * sizeof(int)));
    k_iota<<<ceil_div(nc, 256), 256, 0, st>>>(nc, ident.as<int>()); ::hm::count_launch();

    // ---- stage 1: Y on the box colouring
    if (nv > 0) {
        {
            PhaseTimer tm(st, ph(1));
            HM_TRY(make_gaussians(c, l));
        }
        c->cur_tiles = &gb;
        c->peel_sides = 1;
        Err e;
        {
            PhaseTimer tm(st, ph(2));
            e = sample_level(c, op, l, false);
        }
        if (!e) {
            PhaseTimer tm(st, ph(3));
            e = peel_level(c, l, false);
        }
        c->cur_tiles = nullptr;
        c->peel_sides = 3;
        HM_TRY(e);
        k_gather<<<(unsigned)nv, 128, 0, st>>>(gb.pair_alpha.as<int>(), gb.pair_color.as<int>(), nv, cu.ent.as<int>(),
                                               c->cur.Y.as<double>(), n, r, P.as<double>()); ::hm::count_launch();
        HM_LAUNCH("H2 gather");
    }
    HM_TRY(alloc(f.eS, (size_t)std::max(nc, 1) * 2 * r * sizeof(double)));
    HM_CUDA(cudaMemsetAsync(f.eS.p, 0, (size_t)std::max(nc, 1) * 2 * r * sizeof(double), st));
    {
        PhaseTimer tm(st, ph(4));
        if (has_prev) {  // the parents' far fields
            DBuf goff, G;
            HM_TRY(project_gauss(c, l - 1, l, SIDE_AUG_U, fp->ekU, fp->eoffU, fp->U, goff, G));
            k_augment<<<(unsigned)nc, 128, 0, st>>>(nc, cu.ent.as<int>(), cu.parent.as<int>(),
                                                    c->cuts[l - 1].ent.as<int>(), fp->ekU.as<int>(),
                                                    fp->eoffU.as<int64_t>(), fp->U.as<double>(), fp->eS.as<double>(), 0,
                                                    goff.as<int64_t>(), G.as<double>(), r, P.as<double>()); ::hm::count_launch();
            HM_LAUNCH("H2 augment U");
        }
        HM_TRY(svd_tiles(c, l, tU, P.as<double>(), 0, f.ekU, f.eoffU, f.U, f.nU, f.eS));
    }
    P.release();

    // ---- stage 2: Z = A^* Psi on the pair colouring, Psi filled with the bases
    HM_TRY(alloc(Wb, (size_t)n * r * sizeof(double)));
    HM_CUDA(cudaMemsetAsync(Wb.p, 0, (size_t)n * r * sizeof(double), st));
    if (nv > 0) {
        HM_CUDA(cudaMemsetAsync(c->GP.p, 0, (size_t)n * r * sizeof(double), st));
        k_fill<<<(unsigned)nc, 128, 0, st>>>(nc, cu.ent.as<int>(), f.ekU.as<int>(), f.eoffU.as<int64_t>(),
                                             f.U.as<double>(), r, c->GP.as<double>()); ::hm::count_launch();
        HM_LAUNCH("H2 fill Psi");
        c->peel_sides = 2;
        Err e;
        {
            PhaseTimer tm(st, ph(2));
            e = sample_level(c, op, l, false);
        }
        if (!e) {
            PhaseTimer tm(st, ph(3));
            e = peel_level(c, l, false);
        }
        c->peel_sides = 3;
        HM_TRY(e);
        PhaseTimer tm(st, ph(4));
        DBuf moff, M;
        HM_TRY(project_gauss(c, l, l, SIDE_MIX, f.ekU, f.eoffU, f.U, moff, M));
        HM_TRY(mix_sum(c, l, gb.pair_alpha.as<int>(), nv, ident.as<int>(), f.ekU.as<int>(), moff.as<int64_t>(),
                       M.as<double>(), Wb.as<double>()));
    }
    {
        PhaseTimer tm(st, ph(4));
        if (has_prev) {
            DBuf goff, G;
            HM_TRY(project_gauss(c, l - 1, l, SIDE_AUG_V, fp->ekV, fp->eoffV, fp->V, goff, G));
            k_augment<<<(unsigned)nc, 128, 0, st>>>(nc, cu.ent.as<int>(), cu.parent.as<int>(),
                                                    c->cuts[l - 1].ent.as<int>(), fp->ekV.as<int>(),
                                                    fp->eoffV.as<int64_t>(), fp->V.as<double>(), fp->eS.as<double>(), 1,
                                                    goff.as<int64_t>(), G.as<double>(), r, Wb.as<double>()); ::hm::count_launch();
            HM_LAUNCH("H2 augment V");
        }
        HM_TRY(svd_tiles(c, l, tV, Wb.as<double>(), 1, f.ekV, f.eoffV, f.V, f.nV, f.eS));
        Wb.release();
        if (np > 0)
            HM_TRY(box_pairs_and_cores(c, l, ident.as<int>(), f.ekU.as<int>(), f.ekV.as<int>(),
                                       f.eoffU.as<int64_t>(), f.eoffV.as<int64_t>()));
        f.has_bases = true;
        f.done = true;
        if (has_prev) HM_TRY(nest_and_expand(c, l));
    }
    return ok();
}

// the finest cut that holds bases (its long bases are kept), or -1
static int h2_top(const hm_ctx *c) {
    for (int l = c->L; l >= 2; --l)
        if (l < (int)c->factors.size() && c->factors[l].has_bases) return l;
    return -1;
}

Err h2_finish(hm_ctx *c) {
    using namespace h2k;
    cudaStream_t st = c->st;
    const int top = h2_top(c);
    for (int l = 2; l <= c->L && l < (int)c->factors.size(); ++l) {
        Factors &f = c->factors[l];
        if (!f.has_bases) continue;
        for (int side = 0; side < 2; ++side) {
            DBuf sz;
            DBuf &ep = side ? f.epV : f.epU;
            HM_TRY(alloc(sz, ((size_t)f.nc + 1) * sizeof(int64_t)));
            HM_TRY(alloc(ep, ((size_t)f.nc + 1) * sizeof(int64_t)));
            k_k_sizes<<<ceil_div(f.nc, 256), 256, 0, st>>>(f.nc, (side ? f.ekV : f.ekU).as<int>(), sz.as<int64_t>()); ::hm::count_launch();
            HM_TRY(scan_exclusive(sz.as<int64_t>(), ep.as<int64_t>(), f.nc, st));
            HM_TRY(read_scalar(side ? f.sumkV : f.sumkU, ep.as<int64_t>() + f.nc, st));
        }
        if (l < top) {  // the nested chain replaces the long bases of the coarser cuts
            f.U.release();
            f.V.release();
            f.U2.release();
            f.V2.release();
            f.U32.release();
            f.V32.release();
            f.nU = f.nV = 0;
        }
    }
    return ok();
}

int64_t h2_scratch_elems(const hm_ctx *c) {
    int64_t s = 0;
    for (int l = 2; l <= c->L && l < (int)c->factors.size(); ++l)
        if (c->factors[l].has_bases) s += c->factors[l].sumkU + c->factors[l].sumkV;
    return s;
}

Err apply_h2_into(hm_ctx *c, const double *x, double *y, int nrhs, int trans, double *t) {
    using namespace h2k;
    cudaStream_t st = c->st;
    HM_CUDA(cudaMemsetAsync(y, 0, (size_t)c->n * nrhs * sizeof(double), st));
    const int top = h2_top(c);
    if (top >= 2) {
        const int64_t tot = h2_scratch_elems(c);
        HM_CUDA(cudaMemsetAsync(t, 0, (size_t)std::max<int64_t>(tot, 1) * nrhs * sizeof(double), st));
        // per level: outgoing expansions (k of the row side, or of the column side
        // with trans) then incoming ones
        std::vector<double *> qb(c->L + 1, nullptr), ub(c->L + 1, nullptr);
        int64_t off = 0;
        for (int l = 2; l <= top; ++l) {
            const Factors &f = c->factors[l];
            if (!f.has_bases) continue;
            qb[l] = t + off * nrhs;
            off += trans ? f.sumkU : f.sumkV;
            ub[l] = t + off * nrhs;
            off += trans ? f.sumkV : f.sumkU;
        }
        auto kout = [&](const Factors &f) { return (trans ? f.ekU : f.ekV).as<int>(); };  // outgoing side
        auto kin = [&](const Factors &f) { return (trans ? f.ekV : f.ekU).as<int>(); };   // incoming side
        auto pout = [&](const Factors &f) { return (trans ? f.epU : f.epV).as<int64_t>(); };
        auto pin = [&](const Factors &f) { return (trans ? f.epV : f.epU).as<int64_t>(); };
        const Factors &ft = c->factors[top];
        const Cut &ct = c->cuts[top];
        k_ap_out<<<(unsigned)ct.nc, 128, 0, st>>>(ct.nc, ct.ent.as<int>(), kout(ft), (trans ? ft.eoffU : ft.eoffV).as<int64_t>(),
                                                  (trans ? ft.U : ft.V).as<double>(), x, nrhs, pout(ft), qb[top]); ::hm::count_launch();
        for (int l = top - 1; l >= 2; --l) {
            const Factors &f = c->factors[l], &fc = c->factors[l + 1];
            if (!f.has_bases || !fc.has_bases) continue;
            const Cut &cu = c->cuts[l];
            k_ap_up<<<(unsigned)cu.nc, 128, 0, st>>>(cu.nc, kout(f), pout(f), qb[l], cu.kid_begin.as<int>(),
                                                     cu.kid_end.as<int>(), kout(fc), pout(fc), qb[l + 1],
                                                     (trans ? f.offUt : f.offVt).as<int64_t>(),
                                                     (trans ? f.Ut : f.Vt).as<double>(), nrhs); ::hm::count_launch();
        }
        for (int l = 2; l <= top; ++l) {
            const Factors &f = c->factors[l];
            if (!f.has_bases || f.n_pairs == 0) continue;
            const Cut &cu = c->cuts[l];
            const Coloring &g = c->colorings[l];
            k_ap_far<<<(unsigned)cu.nc, 128, 0, st>>>(cu.nc, cu.int_ptr.as<int>(), cu.int_idx.as<int>(),
                                                      g.pair_T.as<int>(), f.kU.as<int>(), f.kV.as<int>(),
                                                      f.offB.as<int64_t>(), f.B.as<double>(), trans, pout(f), qb[l],
                                                      kin(f), pin(f), ub[l], nrhs); ::hm::count_launch();
        }
        for (int l = 3; l <= top; ++l) {
            const Factors &f = c->factors[l], &fp = c->factors[l - 1];
            if (!f.has_bases || !fp.has_bases) continue;
            const Cut &cu = c->cuts[l];
            k_ap_down<<<(unsigned)cu.nc, 128, 0, st>>>(cu.nc, cu.parent.as<int>(), kin(f), pin(f), ub[l], kin(fp),
                                                       pin(fp), ub[l - 1], (trans ? fp.offVt : fp.offUt).as<int64_t>(),
                                                       (trans ? fp.Vt : fp.Ut).as<double>(), nrhs); ::hm::count_launch();
        }
        k_ap_in<<<(unsigned)ct.nc, 128, 0, st>>>(ct.nc, ct.ent.as<int>(), kin(ft), (trans ? ft.eoffV : ft.eoffU).as<int64_t>(),
                                                 (trans ? ft.V : ft.U).as<double>(), pin(ft), ub[top], nrhs, y); ::hm::count_launch();
        HM_LAUNCH("H2 apply");
    }
    return apply_near(c, x, y, nrhs, trans);
}

}  // namespace hm
