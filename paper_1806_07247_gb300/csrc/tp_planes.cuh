// Writes one spectrum value into the BF16x3 operand planes of the tensor-core slice GEMM
// (layouts PLANE_LEFT / PLANE_RIGHT of tp_internal.cuh).  Shared by the forward DFT, which can
// write the planes directly, and by the kernel that fills them from a complex spectrum.
#pragma once

#include <cuda_bf16.h>

#include "tp_internal.cuh"

namespace tp {

// x = hi + lo with hi = bf16(x) and lo = bf16(x - hi), both rounded to nearest even; the split
// of -x is the negated split of x.
__device__ __forceinline__ void bf16_split(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// Tube p = r + rows * q of the operand (left: r = m, q = k; right: r = k, q = n); `other` is
// the operand's other size (K for the left operand, N for the right one).
struct PlaneCursor {
    int64_t q = 0, r = 0, other = 0;
};

__device__ __forceinline__ PlaneCursor plane_cursor(const FftJob& J, int64_t p) {
    PlaneCursor c;
    c.q = p / J.plane_rows;
    c.r = p - c.q * J.plane_rows;
    c.other = J.P / J.plane_rows;
    return c;
}

// Frequency z of one tube, written by its own thread: four (left) or eight (right) 2-byte
// stores, each warp-coalesced along the rows.
__device__ __forceinline__ void store_plane_value(const FftJob& J, PlaneCursor c, int z, float2 v) {
    const int64_t pitch = J.plane_pitch;
    const int64_t other = c.other;
    uint16_t rh, rl, ih, il;
    bf16_split(v.x, rh, rl);
    bf16_split(v.y, ih, il);
    if (J.plane_kind == PLANE_LEFT) {
        const int64_t re = ((int64_t)(2 * z) * other + c.q) * pitch + c.r;
        const int64_t im = re + other * pitch;
        J.plane_hi[re] = rh;
        J.plane_lo[re] = rl;
        J.plane_hi[im] = ih;
        J.plane_lo[im] = il;
    } else {
        const int64_t rows = 2 * other;
        const int64_t a = ((int64_t)(2 * z) * rows + 2 * c.q) * pitch + c.r;  // part 0, row 2n
        const int64_t b = a + rows * pitch;                                     // part 1, row 2n
        J.plane_hi[a] = rh;
        J.plane_lo[a] = rl;
        J.plane_hi[a + pitch] = ih;
        J.plane_lo[a + pitch] = il;
        J.plane_hi[b] = ih ^ 0x8000u;  // -Im
        J.plane_lo[b] = il ^ 0x8000u;
        J.plane_hi[b + pitch] = rh;
        J.plane_lo[b + pitch] = rl;
    }
}

}  // namespace tp
