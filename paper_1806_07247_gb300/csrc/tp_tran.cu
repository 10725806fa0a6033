// Conjugate tensor transpose of a real tensor (Def. 2.2): every frontal slice is
// transposed and slices 1..n3-1 are taken in reverse order, so output slice k is the
// transpose of input slice (n3 - k) mod n3.  Pure data movement through shared memory, reads
// and writes coalesced.  When n1 and n2 are multiples of 4 and both tensors are 16-byte
// aligned, a CTA moves a 64 x 64 tile of one slice with float4 loads and stores (each thread
// keeps four 16-byte loads in flight; the tile has one padding column against bank
// conflicts); otherwise 32 x 32 tiles with scalar accesses.
#include "tp_internal.cuh"

namespace tp {

namespace {

constexpr int kTile = 32, kRows = 8;

__global__ void __launch_bounds__(kTile * kRows) tran_kernel(const float* __restrict__ A,
                                                             float* __restrict__ AT, int64_t n1,
                                                             int64_t n2, int64_t n3,
                                                             int64_t tiles_i) {
    __shared__ float tile[kTile][kTile + 1];
    const int64_t bx = blockIdx.x % tiles_i, by = blockIdx.x / tiles_i;
    for (int64_t k = blockIdx.y; k < n3; k += gridDim.y) {
        const int64_t ks = (k == 0) ? 0 : n3 - k;
        const float* src = A + n1 * n2 * ks;
        float* dst = AT + n1 * n2 * k;
        const int64_t i0 = bx * kTile, j0 = by * kTile;
        // read A(i, j) with i fastest
        for (int r = threadIdx.y; r < kTile; r += kRows) {
            int64_t i = i0 + threadIdx.x, j = j0 + r;
            if (i < n1 && j < n2) tile[r][threadIdx.x] = __ldg(src + i + n1 * j);
        }
        __syncthreads();
        // write AT(j, i) = A(i, j) with j fastest (AT is n2 x n1)
        for (int r = threadIdx.y; r < kTile; r += kRows) {
            int64_t j = j0 + threadIdx.x, i = i0 + r;
            if (i < n1 && j < n2) dst[j + n2 * i] = tile[threadIdx.x][r];
        }
        __syncthreads();
    }
}

constexpr int kVT = 64;  // tile edge of the float4 path

__global__ void __launch_bounds__(256) tran_vec_kernel(const float* __restrict__ A,
                                                       float* __restrict__ AT, int64_t n1,
                                                       int64_t n2, int64_t n3, int64_t tiles_i) {
    __shared__ float tile[kVT][kVT + 1];
    const int64_t bx = blockIdx.x % tiles_i, by = blockIdx.x / tiles_i;
    const int64_t k = blockIdx.y;
    const int64_t ks = (k == 0) ? 0 : n3 - k;
    const float* src = A + n1 * n2 * ks;
    float* dst = AT + n1 * n2 * k;
    const int64_t i0 = bx * kVT, j0 = by * kVT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 float4 x 16 rows
    // read A(i..i+3, j): float4 along i (n1 % 4 == 0, so a float4 is all in or all out)
    float4 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + 4 * tx, j = j0 + ty + 16 * r;
        v[r] = (i < n1 && j < n2) ? __ldg(reinterpret_cast<const float4*>(src + i + n1 * j))
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float* t = &tile[ty + 16 * r][4 * tx];
        t[0] = v[r].x;
        t[1] = v[r].y;
        t[2] = v[r].z;
        t[3] = v[r].w;
    }
    __syncthreads();
    // write AT(j..j+3, i) = A(i, j..j+3): float4 along j
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int il = ty + 16 * r;
        const int64_t j = j0 + 4 * tx, i = i0 + il;
        if (i < n1 && j < n2) {
            const float4 o = make_float4(tile[4 * tx][il], tile[4 * tx + 1][il], tile[4 * tx + 2][il],
                                         tile[4 * tx + 3][il]);
            *reinterpret_cast<float4*>(dst + j + n2 * i) = o;
        }
    }
}

}  // namespace

cudaError_t launch_tran(const float* A, float* AT, int64_t n1, int64_t n2, int64_t n3,
                        cudaStream_t s) {
    if (n1 <= 0 || n2 <= 0 || n3 <= 0) return cudaSuccess;
    const bool vec = n1 % 4 == 0 && n2 % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(AT) & 15u) == 0 && n3 <= 65535;
    if (vec) {
        const int64_t ti = (n1 + kVT - 1) / kVT, tj = (n2 + kVT - 1) / kVT;
        if (ti * tj > 0x7fffffffLL) return cudaErrorInvalidValue;
        tran_vec_kernel<<<dim3((unsigned)(ti * tj), (unsigned)n3), 256, 0, s>>>(A, AT, n1, n2, n3, ti);
        return cudaGetLastError();
    }
    int64_t ti = (n1 + kTile - 1) / kTile, tj = (n2 + kTile - 1) / kTile;
    int64_t tiles = ti * tj;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int gy = (int)(n3 < 65535 ? n3 : 65535);
    dim3 grid((unsigned)tiles, gy);
    tran_kernel<<<grid, dim3(kTile, kRows), 0, s>>>(A, AT, n1, n2, n3, ti);
    return cudaGetLastError();
}

}  // namespace tp
