// Philox4x32-10 (Salmon et al., SC'11) standard normals, shared by the
// modules that draw test matrices: entry (row, j) of the Gaussian of box gid
// (side s, cut level l) uses key = seed and counter (j, row, gid, s << 8 | l);
// two 52-bit uniforms and Box-Muller give one standard normal.
#pragma once

#include <cmath>
#include <cstdint>

namespace hm {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const unsigned int M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += W0;
            k.y += W1;
        }
        const unsigned int hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const unsigned int hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double uniform52(unsigned int lo, unsigned int hi) {
    const unsigned long long x = ((unsigned long long)hi << 32) | lo;
    return __dmul_rn(__dadd_rn((double)(x >> 12), 0.5), 0x1.0p-52);
}

__device__ __forceinline__ double gauss(unsigned long long seed, int side, int level, int gid, int row, int j) {
    const uint4 ctr = make_uint4((unsigned)j, (unsigned)row, (unsigned)gid, ((unsigned)side << 8) | (unsigned)level);
    const uint4 o = philox4x32_10(ctr, make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
    const double u1 = uniform52(o.x, o.y), u2 = uniform52(o.z, o.w);
    return __dmul_rn(sqrt(__dmul_rn(-2.0, log(u1))), cos(__dmul_rn(2.0 * M_PI, u2)));
}

}  // namespace hm
