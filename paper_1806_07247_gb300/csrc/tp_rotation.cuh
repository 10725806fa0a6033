// Jacobi rotation arithmetic shared by the slice SVD kernels.
#pragma once

#include <cuda_runtime.h>

namespace tp {

// 1/sqrt(x) and 1/x from the hardware approximations plus one Newton step (about 1 ulp).
__device__ __forceinline__ float rsqrt_nr(float x) {
    const float r = rsqrtf(x);
    return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ float rcp_nr(float x) {
    const float r = __fdividef(1.f, x);
    return r * fmaf(-x, r, 2.f);
}

// Cosine and sine of the Jacobi rotation with tangent t (|t| <= 1): c = 1/sqrt(1 + t^2),
// s = c t.  c^2 + s^2 = 1 must hold to about an ulp with no bias, because every column is
// rotated some n * sweeps times and a biased norm drift accumulates into the singular
// values.  1 + t^2 is therefore kept exactly as qh + ql (error-free product and Fast2Sum),
// and the hardware reciprocal square root gets one Newton step whose residual
// 1 - (qh + ql) r^2 is evaluated with the exact product qh r = h + hl.  The _rn intrinsics
// keep the compiler from fusing or reassociating these steps.
__device__ __forceinline__ void rotation_cs(float t, float& c, float& s) {
    const float hi = __fmul_rn(t, t);
    const float lo = fmaf(t, t, -hi);
    const float qh = __fadd_rn(1.f, hi);
    const float ql = __fadd_rn(__fadd_rn(__fsub_rn(1.f, qh), hi), lo);
    const float r = rsqrtf(qh);
    const float h = __fmul_rn(qh, r);
    const float hl = fmaf(qh, r, -h);
    const float rho = __fsub_rn(fmaf(-h, r, 1.f), r * fmaf(ql, r, hl));
    c = fmaf(0.5f * r, rho, r);
    s = __fmul_rn(c, t);
}


// Rotation of a complex column pair (p, q) from alpha = |g_p|^2, beta = |g_q|^2 and
// gamma = g_p^H g_q (gr + i gi), ag2 = |gamma|^2 > 0: the unitary 2 x 2 map
// g_p <- c g_p - s conj(e) g_q, g_q <- s e g_p + c g_q with e = gamma/|gamma| makes the pair
// orthogonal.  Returns c and (sr, si) = s e.
__device__ __forceinline__ void jacobi_rotation(float al, float be, float gr, float gi, float ag2,
                                                float& c, float& sr, float& si) {
    const float inv_ag = rsqrt_nr(ag2);
    const float zeta = 0.5f * (be - al) * inv_ag;
    const float az = fabsf(zeta);
    float t;
    if (az > 1e8f) {
        t = 0.5f * rcp_nr(az);
    } else {
        const float q = fmaf(zeta, zeta, 1.f);
        t = rcp_nr(az + q * rsqrt_nr(q));
    }
    t = copysignf(t, zeta);
    float s;
    rotation_cs(t, c, s);
    sr = s * (gr * inv_ag);
    si = s * (gi * inv_ag);
}

}  // namespace tp
