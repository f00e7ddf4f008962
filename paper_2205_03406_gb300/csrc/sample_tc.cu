// Mixed-precision black-box contraction on the 5th-generation tensor cores
// (tcgen05, sm_103a): for colour c and a block of 128 of its output rows (the
// rows of its sample tiles, Section 4.1.2),
//     [Y | Z](rows, c) = sum_{j in rows(c)} K(x_i, x_j) [G^Omega_j | G^Psi_j],
// the sampling step of Algorithm 4.1 with the kernel matrix evaluated on the fly.
//
// Precision (both mixed modes): K is evaluated in FP32 from double-float point
// coordinates (x = hi + lo, both FP32), so differences of nearby points keep
// FP32 accuracy; K and G are split into three BF16 pieces (h + m + l carries
// 24 bits) and the six products hh, hm, mh, hl, mm, lh accumulate in FP32 in
// tensor memory, in two accumulators: hh, and the five lower-order products
// together (each at most 2^-8 of hh, so their FP32 rounding is about 2^-32 of
// the total); every four chunks the producers add them into double-float
// registers, and the epilogue writes FP64.  Two accumulator sets of 4r columns
// fit the 512 columns of tensor memory for r <= 64.
//
// Per level a pack kernel writes, for every colour, chunks of 64 active rows
// in the exact shared-memory image the tensor core reads: the three BF16
// pieces of [G^Omega | G^Psi]^T (K-major, 128-byte swizzle) followed by the
// chunk's double-float coordinates.  The main kernel (one CTA per 128 output
// rows of a colour) streams chunks through two shared-memory stages:
//   - one thread of the TMA warp issues cp.async.bulk copies of the next chunk,
//   - sixteen producer warps evaluate the 128 x 64 kernel tile with packed
//     FP32x2 arithmetic, split it and store it swizzled, then arrive on an
//     mbarrier,
//   - one thread of the MMA warp issues tcgen05.mma (M = 128, K = 16 per
//     instruction, five instructions per K step: A_h x [B_h B_m] into
//     hh | rest, then A_h x B_l, A_m x B_h, A_m x B_m, A_l x B_h into rest)
//     and tcgen05.commit frees the stage,
//   - the producers read the accumulators with tcgen05.ld (promotion and
//     epilogue).
// Every mbarrier wait is bounded; on expiry a status word is set and the CTA
// drains and frees its tensor memory before returning.
#include "ctx.cuh"

#include <cuda_bf16.h>

#include <atomic>
#include <cmath>
#include <cstdlib>

namespace hm {

namespace tc {

constexpr int KC = 64;          // rows j per chunk (one 128-byte row of BF16)
constexpr int TM = 128;         // rows i per tile (MMA M)
constexpr int NPROD = 512;      // producer threads (16 warps)
constexpr int PWARPS = NPROD / 32;
constexpr int NTHREADS = NPROD + 64;  // + MMA warp (16) + TMA warp (17)
constexpr int A_PIECE = TM * 128;        // bytes of one A piece (16 KB)
constexpr int COORD_BYTES = KC * 32;     // 64 entries x 8 floats
constexpr unsigned long long WAIT_NS = 4000000000ull;  // 4 s per wait (Params.wait_ns)
constexpr unsigned long long STALL_WAIT_NS = 1000000ull;  // 1 ms in an injected stall

__host__ __device__ constexpr int b_bytes(int r) { return 3 * 2 * r * 128; }
__host__ __device__ constexpr int chunk_bytes(int r) { return b_bytes(r) + COORD_BYTES; }
__host__ __device__ constexpr int stage_bytes(int r) {
    return ((3 * A_PIECE + chunk_bytes(r)) + 1023) / 1024 * 1024;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and *status set) when the phase does not complete
// within limit_ns or another thread has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *status,
                                          unsigned long long limit_ns, bool abortable = true) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 1023) == 0) {
            if (abortable && *status) return false;
            if (gtime() - t0 > limit_ns) {
                *status = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float *v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// kernel value up to the constant factor applied in the epilogue
template <int KIND> __device__ __forceinline__ float kval(float r2) {
    if (KIND == HM_K_EXP) return exp2f(-sqrtf(r2) * 1.4426950408889634f);
    float v;
    if (KIND == HM_K_LOG) v = __log2f(r2);
    else v = rsqrtf(r2);
    return r2 > 0.0f ? v : 0.0f;
}

// packed FP32 pairs (f32x2): element 0 in the low word
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// BF16 pair (element 0 in the low half) and its exact FP32 values
__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint64_t bf2f(uint32_t h) {
    return pk2(__uint_as_float(h << 16), __uint_as_float(h & 0xFFFF0000u));
}

__host__ __device__ constexpr double kscale(int kind) {
    return kind == HM_K_LAPLACE3D ? 0.079577471545947667884 : (kind == HM_K_LOG ? 0.34657359027997265471 : 1.0);
}

struct Params {
    const float4 *xdf;         // sorted points, double-float: [n][2] = (hi xyz, lo xyz)
    int64_t n;
    int r;
    const int64_t *chunk_off;  // per colour: first chunk (chi + 1)
    const int64_t *rows_ptr;   // per colour: active rows offset (chi + 1)
    const unsigned char *pack; // packed chunks
    double *Y, *Z;             // [chi][n][r]
    int *status;
    // output rows: CTA b computes rows out_rows[item_base[b] + m], m < 128, of
    // colour item_color[b] (the rows of that colour's sample tiles)
    const int *out_rows;
    const int64_t *out_ptr;    // per colour (chi + 1)
    const int64_t *item_base;
    const int *item_color;
    unsigned long long wait_ns;  // limit of every mbarrier wait
    int withhold;              // fault injection: the TMA warp issues no copy, so the
                               // pipeline's waits run out (set by the host only)
};

constexpr int SEG = 4;      // chunks accumulated in tensor memory before promotion
constexpr int MAXR = 64;    // largest r (two sets of 4r accumulator columns in 512)

// exact FP32 -> FP64 with integer operations (normal numbers; zero and
// subnormals map to a signed zero), keeping the conversion off the FP64 pipe
__device__ __forceinline__ double f2d(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint64_t sgn = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sgn);
    return __longlong_as_double((long long)(sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// hi + lo += v, error-free (Knuth two-sum on the high part)
__device__ __forceinline__ void dfadd(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += err;
}

// MH: the largest r / 2 of the instantiation (accumulator columns per producer thread)
template <int KIND, int MH>
__global__ void __launch_bounds__(NTHREADS, 1) k_sample_tc(Params P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full_a[2], full_b[2], empty[2], seg_done[2], set_free[2], accum;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float4 cbuf[2][2 * KC];  // double-float coordinates of chunks q, q+1
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int r = P.r;
    const int SB = stage_bytes(r);
    const int CB = chunk_bytes(r);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = P.item_color[blockIdx.x];
    const int64_t obase = P.item_base[blockIdx.x];
    const int nvalid = (int)min((int64_t)TM, P.out_ptr[c + 1] - obase);
    const int64_t nrows = P.rows_ptr[c + 1] - P.rows_ptr[c];
    const int nchunks = (int)((nrows + KC - 1) / KC);
    const int nseg = (nchunks + SEG - 1) / SEG;
    const unsigned char *gpack = P.pack + (size_t)P.chunk_off[c] * CB;
    volatile int *status = P.status;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full_a[s], NPROD);
            mbar_init(&full_b[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&seg_done[s], 1);
            mbar_init(&set_free[s], NPROD);
        }
        mbar_init(&accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == PWARPS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (warp < PWARPS) {
        // ------------------------------------------------------------ producers
        // rows 16 (warp % 8) + lane % 8 + 8 u (u = 0, 1), columns 8 ck .. 8 ck + 7
        // (the 16-byte chunk ck = 4 (warp / 8) + lane / 8 of the 128-byte row),
        // in column pairs.  The 8 lanes of a quarter-warp store 8 rows of one
        // chunk: with the 128-byte swizzle they hit 8 distinct bank groups.
        const int ck = 4 * (warp >> 3) + (lane >> 3);
        uint64_t RH[2][3], RL[2][3];  // double-float row coordinates, each duplicated in a pair
        int mrow[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            mrow[u] = 16 * (warp & 7) + (lane & 7) + 8 * u;
            float4 h = make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f), l = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mrow[u] < nvalid) {  // padding rows sit far away: K ~ 0 there
                const int64_t i = P.out_rows[obase + mrow[u]];
                h = P.xdf[2 * i];
                l = P.xdf[2 * i + 1];
            }
            RH[u][0] = pk2(h.x, h.x); RH[u][1] = pk2(h.y, h.y); RH[u][2] = pk2(h.z, h.z);
            RL[u][0] = pk2(l.x, l.x); RL[u][1] = pk2(l.y, l.y); RL[u][2] = pk2(l.z, l.z);
        }
        // promotion: this thread owns TMEM lane quarter (warp & 3) and the
        // columns [sub r/2, sub r/2 + r/2), sub = warp / 4, of the 2r outputs
        // (Y: columns 0..r-1, Z: r..2r-1)
        const int quarter = warp & 3, sub = warp >> 2, hr = r >> 1;
        const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(sub * hr);
        const float scale = (float)kscale(KIND);
        float acc_hi[MH], acc_lo[MH];
#pragma unroll
        for (int k = 0; k < MH; ++k) acc_hi[k] = acc_lo[k] = 0.0f;
        int promoted = 0;
        auto promote = [&](int sg) -> bool {
            const int set = sg & 1;
            // tcgen05.ld is warp-collective: the whole warp goes on or stops together
            const bool done = mbar_wait(&seg_done[set], (uint32_t)(sg >> 1) & 1, status, P.wait_ns, false);
            if (!__all_sync(0xffffffffu, done)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = trow + (uint32_t)(set * 4 * r);
#pragma unroll
            for (int g = 0; g < MH / 4; ++g) {
                if (4 * g >= hr) break;
                float hh[4], lo[4];
                tmem_ld4(base + 4 * g, hh);
                tmem_ld4(base + 2 * r + 4 * g, lo);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    dfadd(acc_hi[4 * g + k], acc_lo[4 * g + k], hh[k] * scale);
                    acc_lo[4 * g + k] = fmaf(lo[k], scale, acc_lo[4 * g + k]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&set_free[set]);
            return true;
        };
        // coordinates: 2 KB per chunk, 4 bytes per producer thread, prefetched
        // one chunk ahead into cbuf (producers sync on named barrier 1)
        const float *gcoord = reinterpret_cast<const float *>(gpack + b_bytes(r));
        float cnext = 0.f;
        if (nchunks > 0) reinterpret_cast<float *>(cbuf[0])[tid] = gcoord[tid];
        asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
        // every producer runs every named barrier; after an error it only
        // skips the work, so no warp can be left waiting at bar.sync
        for (int q = 0; q < nchunks; ++q) {
            const int s = q & 1;
            const uint32_t u = (uint32_t)(q >> 1);
            if (q + 1 < nchunks) cnext = reinterpret_cast<const float *>(gpack + (size_t)(q + 1) * CB + b_bytes(r))[tid];
            if (ok && q >= 2) ok = mbar_wait(&empty[s], (u - 1) & 1, status, P.wait_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                unsigned char *st = smem + s * SB;
                // column pair (ck, e2): 16-byte slots ((3 e2 + j) 8 + ck), j = 0..2:
                // (hx hx' hy hy'), (hz hz' lx lx'), (ly ly' lz lz') -- the 4 chunks a
                // warp reads sit in consecutive slots
                const ulonglong2 *cp = reinterpret_cast<const ulonglong2 *>(cbuf[q & 1]);
                uint64_t kv[2][4];  // K of the thread's 2 rows x 4 column pairs
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    const ulonglong2 q0 = cp[(3 * e2) * 8 + ck], q1 = cp[(3 * e2 + 1) * 8 + ck],
                                     q2 = cp[(3 * e2 + 2) * 8 + ck];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const uint64_t dx = add2(sub2(RH[u][0], q0.x), sub2(RL[u][0], q1.y));
                        const uint64_t dy = add2(sub2(RH[u][1], q0.y), sub2(RL[u][1], q2.x));
                        const uint64_t dz = add2(sub2(RH[u][2], q1.x), sub2(RL[u][2], q2.y));
                        const uint64_t r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                        float a0, a1;
                        up2(r2, a0, a1);
                        kv[u][e2] = pk2(kval<KIND>(a0), kval<KIND>(a1));
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int m = mrow[u];
                    uint32_t ph[4], pm[4], pl[4];
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        // three-piece BF16 split of the pair: v = h + m + l
                        const uint64_t v = kv[u][e2];
                        float v0, v1;
                        up2(v, v0, v1);
                        ph[e2] = bf2(v0, v1);
                        const uint64_t rr = sub2(v, bf2f(ph[e2]));
                        float r0, r1;
                        up2(rr, r0, r1);
                        pm[e2] = bf2(r0, r1);
                        const uint64_t ll = sub2(rr, bf2f(pm[e2]));
                        float l0, l1;
                        up2(ll, l0, l1);
                        pl[e2] = bf2(l0, l1);
                    }
                    const int off = (m >> 3) * 1024 + (m & 7) * 128 + ((ck ^ (m & 7)) << 4);
                    *reinterpret_cast<uint4 *>(st + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                    *reinterpret_cast<uint4 *>(st + A_PIECE + off) = make_uint4(pm[0], pm[1], pm[2], pm[3]);
                    *reinterpret_cast<uint4 *>(st + 2 * A_PIECE + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&full_a[s]);
                // promote the previous segment once the next one has started
                if (q % SEG == 0 && q > 0) {
                    ok = promote(promoted);
                    ++promoted;
                }
            }
            if (q + 1 < nchunks) reinterpret_cast<float *>(cbuf[(q + 1) & 1])[tid] = cnext;
            asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
        }
        if (ok)
            while (promoted < nseg && ok) {
                ok = promote(promoted);
                ++promoted;
            }
        // epilogue: row 32 quarter + lane, its r/2 columns
        const int mo = 32 * quarter + lane;
        if (ok && *status == 0 && mo < nvalid) {
            const int64_t i = P.out_rows[obase + mo];
            double *dst = ((sub >> 1) ? P.Z : P.Y) + ((int64_t)c * P.n + i) * r + (sub & 1) * hr;
#pragma unroll
            for (int k = 0; k < MH; k += 2) {
                if (k >= hr) break;
                *reinterpret_cast<double2 *>(dst + k) =
                    make_double2(f2d(acc_hi[k]) + f2d(acc_lo[k]), f2d(acc_hi[k + 1]) + f2d(acc_lo[k + 1]));
            }
        }
    } else if (warp == PWARPS + 1) {
        // ------------------------------------------------------------ TMA issuer
        if (lane == 0) {
            int issued = 0;
            for (int q = 0; q < nchunks && ok && !P.withhold; ++q) {
                const int s = q & 1;
                if (q >= 2) ok = mbar_wait(&empty[s], ((uint32_t)(q >> 1) - 1) & 1, status, P.wait_ns);
                if (!ok) break;
                mbar_expect_tx(&full_b[s], b_bytes(r));
                bulk_g2s(smem + s * SB + 3 * A_PIECE, gpack + (size_t)q * CB, b_bytes(r), &full_b[s]);
                issued = q + 1;
            }
            // never leave a bulk copy in flight: wait for the last two issued
            for (int k = (issued > 2 ? issued - 2 : 0); k < issued; ++k)
                mbar_wait(&full_b[k & 1], (uint32_t)(k >> 1) & 1, status, P.wait_ns, false);
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        const uint32_t id4 = idesc_bf16(4 * r), id2 = idesc_bf16(2 * r);
        for (int q = 0; q < nchunks && ok; ++q) {
            const int s = q & 1;
            const uint32_t u = (uint32_t)(q >> 1);
            const int sg = q / SEG, set = sg & 1;
            const bool first = (q % SEG) == 0;
            // the accumulator set is free once the producers promoted segment sg - 2
            if (first && sg >= 2) ok = mbar_wait(&set_free[set], (uint32_t)((sg >> 1) - 1) & 1, status, P.wait_ns);
            if (ok) ok = mbar_wait(&full_a[s], u & 1, status, P.wait_ns) && mbar_wait(&full_b[s], u & 1, status, P.wait_ns);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * SB);
            const uint64_t ah = sw128_desc(sa), am = sw128_desc(sa + A_PIECE), al = sw128_desc(sa + 2 * A_PIECE);
            // B pieces: 2r rows each (128 bytes a row), B_m and B_l at multiples of 1024 bytes
            const uint32_t sb = sa + 3 * A_PIECE;
            const uint64_t bh = sw128_desc(sb), bm = sw128_desc(sb + 2 * r * 128), bl = sw128_desc(sb + 4 * r * 128);
            const uint32_t d = tmem + (uint32_t)(set * 4 * r), dl = d + 2 * r;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 2);  // 32 bytes per K step, in 16-byte units
                // A_h x [B_h B_m] -> hh | hm (the first product of a segment starts the
                // set), then hl, mh, mm, lh onto the low-order accumulator
                mma_bf16(d, ah + adv, bh + adv, id4, (first && kk == 0) ? 0u : 1u);
                mma_bf16(dl, ah + adv, bl + adv, id2, 1u);
                mma_bf16(dl, am + adv, bh + adv, id2, 1u);
                mma_bf16(dl, am + adv, bm + adv, id2, 1u);
                mma_bf16(dl, al + adv, bh + adv, id2, 1u);
            }
            mma_commit(&empty[s]);
            if ((q % SEG) == SEG - 1 || q == nchunks - 1) mma_commit(&seg_done[set]);
        }
        // every MMA of this CTA has completed before tensor memory is freed
        mma_commit(&accum);
        mbar_wait(&accum, 0, status, P.wait_ns, false);
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == PWARPS) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// ---------------------------------------------------------------------------
// pack: chunk g of colour c holds rows j_{64q .. 64q+63} of rows(c)
// ---------------------------------------------------------------------------

// B image: row n' = piece * 2r + n (n < r: G^Omega column n, else G^Psi
// column n - r), 64 BF16 of consecutive j per row, 128-byte swizzle.
__global__ void k_pack_b(const int64_t *chunk_color_first, int chi, const int64_t *rows_ptr, const int *rows,
                         const double *GO, const double *GP, int r, int64_t nchunks_total, unsigned char *pack) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int ncol = 2 * r;
    if (t >= nchunks_total * ncol * 8) return;
    const int64_t g = t / (ncol * 8);
    const int rem = (int)(t - g * ncol * 8);
    const int n = rem / 8, kg = rem % 8;
    // colour of chunk g (chi is small: linear search)
    int c = 0;
    while (c + 1 < chi && chunk_color_first[c + 1] <= g) ++c;
    const int64_t q = g - chunk_color_first[c];
    const int64_t r0 = rows_ptr[c], r1 = rows_ptr[c + 1];
    __align__(16) __nv_bfloat16 ph[8], pm[8], pl[8];
    for (int e = 0; e < 8; ++e) {
        const int64_t idx = r0 + q * KC + kg * 8 + e;
        double v = 0.0;
        if (idx < r1) {
            const int j = rows[idx];
            v = (n < r) ? GO[(int64_t)j * r + n] : GP[(int64_t)j * r + (n - r)];
        }
        const __nv_bfloat16 h = __double2bfloat16(v);
        const double r1d = v - (double)__bfloat162float(h);
        const __nv_bfloat16 m = __double2bfloat16(r1d);
        const double r2d = r1d - (double)__bfloat162float(m);
        ph[e] = h;
        pm[e] = m;
        pl[e] = __double2bfloat16(r2d);
    }
    unsigned char *base = pack + (size_t)g * chunk_bytes(r);
    for (int piece = 0; piece < 3; ++piece) {
        const int row = piece * ncol + n;
        const int off = (row >> 3) * 1024 + (row & 7) * 128 + ((kg ^ (row & 7)) << 4);
        const __nv_bfloat16 *src = piece == 0 ? ph : (piece == 1 ? pm : pl);
        *reinterpret_cast<uint4 *>(base + off) = *reinterpret_cast<const uint4 *>(src);
    }
}

// coordinates: entry k = (x_hi, y_hi, z_hi, pad, x_lo, y_lo, z_lo, pad)
__global__ void k_pack_coords(const int64_t *chunk_color_first, int chi, const int64_t *rows_ptr, const int *rows,
                              const float4 *xdf, int r, int64_t nchunks_total, unsigned char *pack) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nchunks_total * KC) return;
    const int64_t g = t / KC;
    const int k = (int)(t - g * KC);
    int c = 0;
    while (c + 1 < chi && chunk_color_first[c + 1] <= g) ++c;
    const int64_t idx = rows_ptr[c] + (g - chunk_color_first[c]) * KC + k;
    float4 h = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f), l = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx < rows_ptr[c + 1]) {  // padding entries sit far away (and their G rows are zero)
        const int j = rows[idx];
        h = xdf[2 * (int64_t)j];
        l = xdf[2 * (int64_t)j + 1];
    }
    // column k = 8 ck + 2 e2 + o (o = 0, 1): element o of the pair (ck, e2), whose
    // three 16-byte slots ((3 e2 + j) 8 + ck), j = 0..2, hold (hx hx' hy hy'),
    // (hz hz' lx lx'), (ly ly' lz lz'); 1536 of the 2048 bytes are used
    const int ck = k >> 3, e2 = (k & 7) >> 1, o = k & 1;
    float *base = reinterpret_cast<float *>(pack + (size_t)g * chunk_bytes(r) + b_bytes(r));
    float *s0 = base + 4 * ((3 * e2) * 8 + ck) + o, *s1 = base + 4 * ((3 * e2 + 1) * 8 + ck) + o,
          *s2 = base + 4 * ((3 * e2 + 2) * 8 + ck) + o;
    s0[0] = h.x;
    s0[2] = h.y;
    s1[0] = h.z;
    s1[2] = l.x;
    s2[0] = l.y;
    s2[2] = l.z;
}

// leaf black box, FP32 kernel values from double-float coordinates, FP64 output:
// Y(i, c m + t) = sum over active boxes beta of K(i, start_beta + t), for the
// output rows i of colour c only (the rows of its leaf tiles): CTA (b, z)
// takes 64 of them from out_rows[item_base[b]], colour item_color[b], and
// the columns t in [64 z, 64 z + 64)
template <int KIND>
__global__ void __launch_bounds__(256) k_sample_leaf32(const float4 *xdf, int64_t n, const int *act_ptr,
                                                       const int *act_box, const int *ent, int m,
                                                       const int *out_rows, const int64_t *out_ptr,
                                                       const int *item_color, const int64_t *item_base,
                                                       double *out) {
    const int c = item_color[blockIdx.x];
    const int64_t oi = item_base[blockIdx.x] + (threadIdx.x >> 2);
    const int ph = threadIdx.x & 3, t0 = blockIdx.y * 64;
    if (oi >= out_ptr[c + 1]) return;
    const int64_t i = out_rows[oi];
    const float4 ih = xdf[2 * i], il = xdf[2 * i + 1];
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    for (int a = act_ptr[c]; a < act_ptr[c + 1]; ++a) {
        const int *e = ent + (int64_t)act_box[a] * ENT_FIELDS;
        const int s = e[3], len = e[4] - e[3];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int t = t0 + q * 4 + ph;
            if (t < len && t < m) {
                const int64_t j = s + t;
                const float4 jh = xdf[2 * j], jl = xdf[2 * j + 1];
                const float dx = (ih.x - jh.x) + (il.x - jl.x);
                const float dy = (ih.y - jh.y) + (il.y - jl.y);
                const float dz = (ih.z - jh.z) + (il.z - jl.z);
                acc[q] += kval<KIND>(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            }
        }
    }
    const double scale = kscale(KIND);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int t = t0 + q * 4 + ph;
        if (t < m) out[((int64_t)c * n + i) * m + t] = (double)acc[q] * scale;
    }
}

__global__ void k_make_xdf(const double *xs, int64_t n, float4 *xdf) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
        const double x = xs[i * 3 + d];
        h[d] = (float)x;
        l[d] = (float)(x - (double)h[d]);
    }
    xdf[2 * i] = make_float4(h[0], h[1], h[2], 0.f);
    xdf[2 * i + 1] = make_float4(l[0], l[1], l[2], 0.f);
}

}  // namespace tc

// double-float copy of the sorted points (x = hi + lo, both FP32), made once
static Err make_xdf(hm_ctx *c) {
    if (c->xdf.p) return ok();
    HM_TRY(alloc(c->xdf, (size_t)c->n * 2 * sizeof(float4)));
    tc::k_make_xdf<<<ceil_div(c->n, 256), 256, 0, c->st>>>(c->xs.as<double>(), c->n, c->xdf.as<float4>()); ::hm::count_launch();
    HM_LAUNCH("make_xdf");
    return ok();
}

// Fault injection for the failure-detection tests: with HM_FAULT_TC_STALL_AFTER=k
// in the environment when the library is loaded, the tensor-core sampler
// launch after k normal ones withholds its copies and waits at most 1 ms, so
// that its waits expire and the call returns HM_ETIMEOUT; it fires once.
static std::atomic<long long> g_tc_stall_countdown{[] {
    const char *s = getenv("HM_FAULT_TC_STALL_AFTER");
    return s && *s ? atoll(s) : -1ll;
}()};
static bool tc_stall_now() {
    if (g_tc_stall_countdown.load(std::memory_order_relaxed) < 0) return false;
    return g_tc_stall_countdown.fetch_sub(1, std::memory_order_relaxed) == 0;
}

bool tc_supported(const hm_ctx *c) {
    const int r = c->cfg.r;
    return r % 8 == 0 && r >= 8 && r <= tc::MAXR;
}

Err sample_tc(hm_ctx *c, int level, int kernel) {
    using namespace tc;
    cudaStream_t st = c->st;
    const Coloring &g = c->cur_tiles ? *c->cur_tiles : c->colorings[level];
    const int chi = g.n_colors, r = c->cfg.r;
    const int64_t n = c->n;
    HM_TRY(make_xdf(c));  // the pack and main kernels read the double-float points
    // chunk table per colour
    std::vector<int64_t> rp;
    HM_TRY(to_host(rp, g.act_rows_ptr.p, chi + 1, st));
    std::vector<int64_t> cf(chi + 1, 0);
    for (int k = 0; k < chi; ++k) cf[k + 1] = cf[k] + (rp[k + 1] - rp[k] + KC - 1) / KC;
    const int64_t total = cf[chi];
    DBuf cfd;
    HM_TRY(to_dev(cfd, cf, st));
    HM_TRY(ensure(c->scratch_b, (size_t)std::max<int64_t>(total, 1) * chunk_bytes(r)));
    HM_TRY(ensure(c->scratch_c, sizeof(int)));
    HM_CUDA(cudaMemsetAsync(c->scratch_c.p, 0, sizeof(int), st));
    if (total > 0) {
        k_pack_b<<<ceil_div(total * 2 * r * 8, 256), 256, 0, st>>>(
            cfd.as<int64_t>(), chi, g.act_rows_ptr.as<int64_t>(), g.act_rows.as<int>(), c->GO.as<double>(),
            c->GP.as<double>(), r, total, c->scratch_b.as<unsigned char>()); ::hm::count_launch();
        k_pack_coords<<<ceil_div(total * KC, 256), 256, 0, st>>>(cfd.as<int64_t>(), chi,
                                                                  g.act_rows_ptr.as<int64_t>(), g.act_rows.as<int>(),
                                                                  c->xdf.as<float4>(), r, total,
                                                                  c->scratch_b.as<unsigned char>()); ::hm::count_launch();
        HM_LAUNCH("pack");
    }
    // one CTA per 128 output rows of a colour
    std::vector<int> icol;
    std::vector<int64_t> ibase;
    if ((int)g.h_out_rows_ptr.size() == chi + 1)
        for (int k = 0; k < chi; ++k)
            for (int64_t b = g.h_out_rows_ptr[k]; b < g.h_out_rows_ptr[k + 1]; b += TM) {
                icol.push_back(k);
                ibase.push_back(b);
                c->tc_evals += std::min<int64_t>(TM, g.h_out_rows_ptr[k + 1] - b) * (rp[k + 1] - rp[k]);
            }
    if (icol.empty()) return ok();
    DBuf icold, ibased;
    HM_TRY(to_dev(icold, icol, st));
    HM_TRY(to_dev(ibased, ibase, st));
    Params P;
    P.xdf = c->xdf.as<float4>();
    P.n = n;
    P.r = r;
    P.chunk_off = cfd.as<int64_t>();
    P.rows_ptr = g.act_rows_ptr.as<int64_t>();
    P.pack = c->scratch_b.as<unsigned char>();
    P.Y = c->cur.Y.as<double>();
    P.Z = c->cur.Z.as<double>();
    P.status = c->scratch_c.as<int>();
    P.out_rows = g.out_rows.as<int>();
    P.out_ptr = g.out_rows_ptr.as<int64_t>();
    P.item_base = ibased.as<int64_t>();
    P.item_color = icold.as<int>();
    P.withhold = tc_stall_now() ? 1 : 0;
    P.wait_ns = P.withhold ? STALL_WAIT_NS : WAIT_NS;
    const int smem = 2 * stage_bytes(r) + 1024;
    const unsigned grid = (unsigned)icol.size();
    cudaEvent_t e0, e1;
    HM_CUDA(cudaEventCreate(&e0));
    HM_CUDA(cudaEventCreate(&e1));
    HM_CUDA(cudaEventRecord(e0, st));
    switch (kernel) {
#define LAUNCH(K)                                                                                       \
    case K:                                                                                             \
        if (r <= 40) {                                                                                  \
            HM_TRY(allow_smem(k_sample_tc<K, 20>, (size_t)smem));                                      \
            k_sample_tc<K, 20><<<grid, NTHREADS, smem, st>>>(P);                                       \
        } else {                                                                                        \
            HM_TRY(allow_smem(k_sample_tc<K, 32>, (size_t)smem));                                      \
            k_sample_tc<K, 32><<<grid, NTHREADS, smem, st>>>(P);                                       \
        }                                                                                               \
        ::hm::count_launch();                                                                           \
        break;
        LAUNCH(HM_K_LOG)
        LAUNCH(HM_K_LAPLACE3D)
        LAUNCH(HM_K_INVR)
        LAUNCH(HM_K_EXP)
#undef LAUNCH
    default: return fail(HM_EINVAL, "sample_tc: unknown kernel");
    }
    HM_LAUNCH("sample_tc");
    HM_CUDA(cudaEventRecord(e1, st));
    int status = 0;
    HM_TRY(read_scalar(status, c->scratch_c.p, st));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) c->t_tc += ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status) return fail(HM_ETIMEOUT, "sample_tc: a pipeline wait expired");
    return ok();
}

Err sample_leaf_mixed(hm_ctx *c, int kernel) {
    using namespace tc;
    const Coloring &g = c->colorings[c->L + 1];
    const Cut &cu = c->cuts[c->L];
    const int chi = g.n_colors, m = g.m_cols;
    const int64_t n = c->n;
    cudaStream_t st = c->st;
    HM_TRY(make_xdf(c));
    // one CTA per 64 output rows of a colour (and 64 columns)
    std::vector<int> icol;
    std::vector<int64_t> ibase;
    if ((int)g.h_out_rows_ptr.size() == chi + 1)
        for (int k = 0; k < chi; ++k)
            for (int64_t b = g.h_out_rows_ptr[k]; b < g.h_out_rows_ptr[k + 1]; b += 64) {
                icol.push_back(k);
                ibase.push_back(b);
            }
    if (icol.empty()) return ok();
    DBuf icold, ibased;
    HM_TRY(to_dev(icold, icol, st));
    HM_TRY(to_dev(ibased, ibase, st));
    dim3 grid((unsigned)icol.size(), ceil_div(m, 64));
    switch (kernel) {
#define LAUNCH(K)                                                                                              \
    case K:                                                                                                    \
        k_sample_leaf32<K><<<grid, 256, 0, st>>>(c->xdf.as<float4>(), n, g.act_ptr.as<int>(), g.act_box.as<int>(), \
                                                 cu.ent.as<int>(), m, g.out_rows.as<int>(),                     \
                                                 g.out_rows_ptr.as<int64_t>(), icold.as<int>(),                 \
                                                 ibased.as<int64_t>(), c->cur.Y.as<double>());                  \
        ::hm::count_launch();                                                                                  \
        break;
        LAUNCH(HM_K_LOG)
        LAUNCH(HM_K_LAPLACE3D)
        LAUNCH(HM_K_INVR)
        LAUNCH(HM_K_EXP)
#undef LAUNCH
    default: return fail(HM_EINVAL, "sample_leaf_mixed: unknown kernel");
    }
    HM_LAUNCH("sample_leaf32");
    return ok();
}

}  // namespace hm
