// Device helpers shared by the rank proposer (tp_sketch.cu) and the batched randomized SVT
// stages (tp_sketch_svt.cu): the counter-based hash that draws the random test matrices,
// warp reductions and the load of a Fourier-slice entry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tp {
namespace sk {

// 32-bit finaliser of MurmurHash3 (a published bijective mixing function).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// Hash of (seed, slice, row, column group); two bits per column of the group draw the signs.
__device__ __forceinline__ uint32_t omega_hash(uint32_t seed, uint32_t slice, uint32_t r,
                                               uint32_t c0) {
    return mix32(seed ^ mix32(slice * 0x9e3779b9u ^ mix32(r * 0x632be5abu + c0)));
}

// Entry of a random test matrix from two hash bits: +-1 on real slices, (+-1 +- i)/sqrt(2)
// otherwise (unit modulus either way).
__device__ __forceinline__ float2 omega_entry(uint32_t bits, bool real) {
    const float a = (bits & 1u) ? 1.f : -1.f, b = (bits & 2u) ? 1.f : -1.f;
    return real ? make_float2(a, 0.f) : make_float2(a * 0.70710678f, b * 0.70710678f);
}

// Entry (r, c) of the test matrix of slice `slice` (one hash per row and 16 columns).
__device__ __forceinline__ float2 omega(uint32_t seed, uint32_t slice, uint32_t r, uint32_t c,
                                        bool real) {
    const uint32_t c0 = c & ~15u;
    return omega_entry(omega_hash(seed, slice, r, c0) >> (2 * (c - c0)), real);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Entry of a Fourier slice; the real slices of Eq. 8 are read with a zero imaginary part.
__device__ __forceinline__ float2 ld_a(const float2* A, int64_t idx, bool real) {
    float2 v = A[idx];
    if (real) v.y = 0.f;
    return v;
}

}  // namespace sk
}  // namespace tp
