// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the uniform streams.
//
// Stream of one task: key = (seed mod 2^32, seed div 2^32), counter =
// (block, iteration, evaluation counter, task).  Uniform number u = s*D + d
// (sample s, dimension d) is word u mod 4 of block u div 4 in FP32, the value
// x 2^-32 in [0, 1) (its VEGAS increment and fraction follow exactly from the
// 64-bit product x nb), and words 2(u mod 2), 2(u mod 2)+1 of block u div 2
// in FP64, mapped to (((x0 >> 6) 2^26 + (x1 >> 6)) + 1/2) 2^-52 (exactly
// representable), so any implementation of the same definition draws the
// same points.
#pragma once

#include <cstdint>

namespace best {

struct PhiloxKey {
    uint32_t k[2 * 10];     // round keys k_r = k_0 + r * Weyl, precomputed
};

__host__ __device__ inline PhiloxKey philox_key(uint64_t seed) {
    PhiloxKey key;
    uint32_t k0 = static_cast<uint32_t>(seed);
    uint32_t k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        key.k[2 * r] = k0;
        key.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return key;
}

// Ten rounds: (c0, c2) are multiplied by the round multipliers; the high
// halves are mixed with the other words and the round key.
template <typename Keys>
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              const Keys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
        const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

__device__ __forceinline__ float uniform_f32(uint32_t x) {
    return static_cast<float>(x) * 2.3283064365386963e-10f;                  // x 2^-32 (rounded to FP32)
}

__device__ __forceinline__ double uniform_f64(uint32_t x0, uint32_t x1) {
    const uint64_t k = (static_cast<uint64_t>(x0 >> 6) << 26) | static_cast<uint64_t>(x1 >> 6);
    return (static_cast<double>(k) + 0.5) * 2.220446049250313080847e-16;       // 2^-52
}

// Number of uniforms per Philox block and the smallest sample group whose
// uniforms fill whole blocks, for D dimensions.
template <int D, bool F32>
struct StreamShape {
    static constexpr int kPerBlock = F32 ? 4 : 2;
    static constexpr int gcd_(int a, int b) { return b == 0 ? a : gcd_(b, a % b); }
    static constexpr int kGroup = kPerBlock / gcd_(D, kPerBlock);
    static constexpr int kUniforms = kGroup * D;
    static constexpr int kBlocks = kUniforms / kPerBlock;
};

// Fills u[0 .. G*D) with the uniforms of sample group g of one task stream.
// rk: the 20 round keys (pass the kernel-parameter array so that they are
// read from the constant bank rather than held in registers).
template <int D, bool F32, typename R, typename Keys>
__device__ __forceinline__ void group_uniforms(R* u, int64_t g, uint32_t itn, uint32_t call,
                                               uint32_t task, const Keys& rk) {
    using S = StreamShape<D, F32>;
    const uint64_t b0 = static_cast<uint64_t>(g) * S::kBlocks;
#pragma unroll
    for (int j = 0; j < S::kBlocks; ++j) {
        uint32_t c0 = static_cast<uint32_t>(b0 + j), c1 = itn, c2 = call, c3 = task;
        philox4x32_10(c0, c1, c2, c3, rk);
        if constexpr (F32) {
            u[4 * j + 0] = static_cast<R>(uniform_f32(c0));
            u[4 * j + 1] = static_cast<R>(uniform_f32(c1));
            u[4 * j + 2] = static_cast<R>(uniform_f32(c2));
            u[4 * j + 3] = static_cast<R>(uniform_f32(c3));
        } else {
            u[2 * j + 0] = static_cast<R>(uniform_f64(c0, c1));
            u[2 * j + 1] = static_cast<R>(uniform_f64(c2, c3));
        }
    }
}

// Raw 32-bit words of sample group g (FP32 stream: one word per uniform).
template <int D, typename Keys>
__device__ __forceinline__ void group_words(uint32_t* w, uint32_t g, uint32_t itn, uint32_t call,
                                            uint32_t task, const Keys& rk) {
    using S = StreamShape<D, true>;
    const uint32_t b0 = g * S::kBlocks;            // counter word 0 is the block index mod 2^32
#pragma unroll
    for (int j = 0; j < S::kBlocks; ++j) {
        uint32_t c0 = b0 + j, c1 = itn, c2 = call, c3 = task;
        philox4x32_10(c0, c1, c2, c3, rk);
        w[4 * j + 0] = c0;
        w[4 * j + 1] = c1;
        w[4 * j + 2] = c2;
        w[4 * j + 3] = c3;
    }
}

}  // namespace best
