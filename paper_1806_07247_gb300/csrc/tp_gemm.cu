// Slice GEMMs of the t-product (Algorithm 1, step 2; Eq. 10): Cbar^(k) = Abar^(k) Bbar^(k)
// for the independent Fourier slices k < ceil((n3+1)/2).
//
// This file holds the plain FP32 path: complex interleaved operands, column-major slices,
// 64 x 64 complex output tile per 256-thread CTA, K staged 16 at a time in shared memory,
// a 4 x 4 complex register tile per thread (64 FFMA per 8 shared loads).
#include "tp_internal.cuh"

namespace tp {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kThreads = 256;

__global__ void __launch_bounds__(kThreads) cgemm_fp32_kernel(
    const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C, int M,
    int N, int K, int64_t sA, int64_t sB, int64_t sC) {
    __shared__ float2 As[kBK][kBM];
    __shared__ float2 Bs[kBK][kBN + 1];
    const int z = blockIdx.z;
    A += sA * z;
    B += sB * z;
    C += sC * z;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

    float cr[4][4], ci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0.f;

    for (int k0 = 0; k0 < K; k0 += kBK) {
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            int idx = tid + kThreads * it;
            int kk = idx / kBM, mm = idx % kBM;
            float2 v = make_float2(0.f, 0.f);
            if (m0 + mm < M && k0 + kk < K) v = __ldg(A + (m0 + mm) + (int64_t)M * (k0 + kk));
            As[kk][mm] = v;
        }
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            int idx = tid + kThreads * it;
            int nn = idx / kBK, kk = idx % kBK;
            float2 v = make_float2(0.f, 0.f);
            if (k0 + kk < K && n0 + nn < N) v = __ldg(B + (k0 + kk) + (int64_t)K * (n0 + nn));
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cr[i][j] = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, cr[i][j]));
                    ci[i][j] = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, ci[i][j]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + tx + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + ty + 16 * j;
            if (n < N) C[m + (int64_t)M * n] = make_float2(cr[i][j], ci[i][j]);
        }
    }
}

}  // namespace

cudaError_t launch_cgemm_fp32(const float2* A, const float2* B, float2* C, int M, int N, int K,
                              int64_t sA, int64_t sB, int64_t sC, int nslices, cudaStream_t s) {
    if (M <= 0 || N <= 0 || nslices <= 0) return cudaSuccess;
    dim3 grid((M + kBM - 1) / kBM, (N + kBN - 1) / kBN, nslices);
    cgemm_fp32_kernel<<<grid, kThreads, 0, s>>>(A, B, C, M, N, K, sA, sB, sC);
    return cudaGetLastError();
}

}  // namespace tp
