// Conjugate tensor transpose of a real tensor (Def. 2.2): every frontal slice is
// transposed and slices 1..n3-1 are taken in reverse order, so output slice k is the
// transpose of input slice (n3 - k) mod n3.  Pure data movement: 32 x 32 tiles through
// shared memory (one padded column against bank conflicts), reads and writes coalesced.
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

}  // namespace

cudaError_t launch_tran(const float* A, float* AT, int64_t n1, int64_t n2, int64_t n3,
                        cudaStream_t s) {
    if (n1 <= 0 || n2 <= 0 || n3 <= 0) return cudaSuccess;
    int64_t ti = (n1 + kTile - 1) / kTile, tj = (n2 + kTile - 1) / kTile;
    int64_t tiles = ti * tj;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int gy = (int)(n3 < 65535 ? n3 : 65535);
    dim3 grid((unsigned)tiles, gy);
    tran_kernel<<<grid, dim3(kTile, kRows), 0, s>>>(A, AT, n1, n2, n3, ti);
    return cudaGetLastError();
}

}  // namespace tp
