// Per-slice dense factorisations of the Fourier slices: the inverse of Def. 2.4 and the QR
// factorisation behind Thm. 2.4.  One CTA owns one independent slice Abar^(k) (k < h), the
// same unit of work as the SVD kernels; the tube DFTs around it are those of tp_fft.cu.
//
// tinv_kernel  Gauss-Jordan elimination with partial pivoting, in place: at step k the
//              pivot row is scaled and every other row is reduced, and the eliminated
//              column stores the matching column of the inverse, so no augmented identity
//              is needed.  The row exchanges are undone on the columns at the end, in
//              reverse order.  8 n^3 real flops per slice.
// tqr_kernel   Householder QR: reflector k maps column k of the trailing block onto
//              beta e_1 with beta = -phase(a_kk) ||x||; its vector is the column itself
//              below the diagonal plus one head element.  Q is accumulated backwards from
//              the identity.  Finally row i of R and column i of Q are rotated by the phase
//              of R(i, i) so that the diagonal of R is real and non-negative, which makes
//              the factors unique for slices of full rank.  The real slices (Eq. 8) stay real:
//              every reflector of a real column is real.
//
// The whole slice (and Q) sits in shared memory when it fits; larger slices are worked on in
// place in global memory (the spectrum buffer), one CTA each, L2-resident.
#include <algorithm>

#include "tp_internal.cuh"

namespace tp {

namespace {

constexpr float kEps = 1.1920929e-07f;  // 2^-23, FP32 unit roundoff x 2

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cjmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float abs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// 1 / z with the operands scaled by max(|re|, |im|) first, so |z|^2 cannot overflow.
__device__ __forceinline__ float2 crcp(float2 z) {
    const float m = fmaxf(fabsf(z.x), fabsf(z.y));
    const float r = 1.0f / m;
    const float2 u = make_float2(z.x * r, z.y * r);
    const float d = 1.0f / abs2(u);
    return make_float2(u.x * d * r, -u.y * d * r);
}

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread receives the total.  `red` holds 32 floats.
__device__ __forceinline__ float block_sum(float v, float* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();  // a previous call may still be reading red
    if (l == 0) red[w] = v;
    __syncthreads();
    return warp_sum(l < nw ? red[l] : 0.0f);
}

// Maximum over the block; every thread receives it.
__device__ __forceinline__ float block_max(float v, float* red) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float t = l < nw ? red[l] : 0.0f;
    for (int o = 16; o; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

// Largest value and its index over the block (the smaller index on ties).
__device__ __forceinline__ void argmax_step(float& v, int& i, float ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}
__device__ __forceinline__ void block_argmax(float& v, int& idx, float* red, int* redi) {
    for (int o = 16; o; o >>= 1)
        argmax_step(v, idx, __shfl_xor_sync(0xffffffffu, v, o), __shfl_xor_sync(0xffffffffu, idx, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) {
        red[w] = v;
        redi[w] = idx;
    }
    __syncthreads();
    v = l < nw ? red[l] : -1.0f;
    idx = l < nw ? redi[l] : 0x7fffffff;
    for (int o = 16; o; o >>= 1)
        argmax_step(v, idx, __shfl_xor_sync(0xffffffffu, v, o), __shfl_xor_sync(0xffffffffu, idx, o));
}

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// ---------------------------------------------------------------------------------------
// Slice inverse.  Shared memory: [n*n matrix if in_smem][rowk n][rowold n][colk n]
// [perm n ints][reduction 32 floats + 32 ints].
// ---------------------------------------------------------------------------------------
// R: rows per lane, n <= 32 R.
template <int R>
__global__ void __launch_bounds__(512, 1) tinv_kernel(const LaJob* __restrict__ jobs, int in_smem,
                                                    uint32_t* status) {
    extern __shared__ float4 la_smem[];
    const LaJob J = jobs[blockIdx.x];
    const int n = J.n1;
    const size_t nn = (size_t)n * n;
    float2* base = reinterpret_cast<float2*>(la_smem);
    float2* M = in_smem ? base : J.A;
    float2* rowk = base + (in_smem ? nn : 0);
    float2* rowold = rowk + n;
    float2* colk = rowold + n;
    int* perm = reinterpret_cast<int*>(colk + n);
    float* red = reinterpret_cast<float*>(perm + n);
    int* redi = reinterpret_cast<int*>(red + 32);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    float amax2 = 0.0f;
    for (size_t e = tid; e < nn; e += nt) {
        const float2 v = J.A[e];
        if (in_smem) M[e] = v;
        amax2 = fmaxf(amax2, abs2(v));
    }
    amax2 = block_max(amax2, red);  // also publishes the shared-memory copy
    // A pivot at or below n * 2^-23 of the slice's largest entry means the slice is singular
    // to FP32 working precision.
    const float thr = (float)n * kEps;
    const float thr2 = thr * thr * amax2;
    bool singular = false;
    for (int k = 0; k < n; ++k) {
        float pv = -1.0f;
        int p = 0x7fffffff;
        for (int i = k + tid; i < n; i += nt) argmax_step(pv, p, abs2(M[i + (size_t)n * k]), i);
        block_argmax(pv, p, red, redi);
        if (!(pv > thr2)) {  // also catches NaN and Inf
            singular = true;
            break;
        }
        if (tid == 0) perm[k] = p;
        // read-only pass over M: scaled pivot row, old row k, column k after the exchange
        const float2 inv = crcp(M[p + (size_t)n * k]);
        for (int j = tid; j < n; j += nt) {
            rowk[j] = (j == k) ? inv : cmul(M[p + (size_t)n * j], inv);
            rowold[j] = M[k + (size_t)n * j];
        }
        for (int i = tid; i < n; i += nt) {
            const int src = (i == p) ? k : (i == k ? p : i);
            colk[i] = M[src + (size_t)n * k];
        }
        __syncthreads();
        // Every element is written by the thread that reads it.  Lane `lane` owns rows
        // lane + 32 m; their multipliers f_i (column k after the exchange) stay in registers.
        float2 f[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int i = lane + 32 * m;
            f[m] = i < n ? colk[i] : make_float2(0.f, 0.f);
        }
        for (int j = warp; j < n; j += nw) {
            const float2 r = rowk[j], ro = rowold[j];
            float2* col = M + (size_t)n * j;
            if (j == k) {  // the pivot column becomes -f_i / pivot (r = 1 / pivot here)
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const int i = lane + 32 * m;
                    if (i < n)
                        col[i] = (i == k) ? r
                                          : make_float2(-fmaf(f[m].x, r.x, -f[m].y * r.y),
                                                        -fmaf(f[m].x, r.y, f[m].y * r.x));
                }
            } else {  // a_ij <- a'_ij - f_i r_j, row k <- r, row p takes the old row k
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const int i = lane + 32 * m;
                    if (i < n) {
                        float2 a = col[i];
                        if (i == p) a = ro;
                        const float2 v = make_float2(fmaf(-f[m].x, r.x, fmaf(f[m].y, r.y, a.x)),
                                                     fmaf(-f[m].x, r.y, fmaf(-f[m].y, r.x, a.y)));
                        col[i] = (i == k) ? r : v;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (singular) {
        const float qnan = __int_as_float(0x7fc00000);
        for (size_t e = tid; e < nn; e += nt) J.R[e] = make_float2(qnan, qnan);
        if (tid == 0 && status) atomicOr(status, 2u);
        return;
    }
    // undo the row exchanges on the columns, last exchange first
    for (int k = n - 1; k >= 0; --k) {
        const int p = perm[k];
        if (p != k) {
            for (int i = tid; i < n; i += nt) {
                const float2 a = M[i + (size_t)n * k];
                M[i + (size_t)n * k] = M[i + (size_t)n * p];
                M[i + (size_t)n * p] = a;
            }
            __syncthreads();
        }
    }
    if (in_smem)
        for (size_t e = tid; e < nn; e += nt) J.R[e] = M[e];
}

// ---------------------------------------------------------------------------------------
// Slice QR.  Shared memory: [A n1*n2, Q n1*qcols if in_smem][vhead nref][dph m]
// [vscale nref floats][reduction 32 floats].
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) tqr_kernel(const LaJob* __restrict__ jobs, int in_smem) {
    extern __shared__ float4 la_smem[];
    const LaJob J = jobs[blockIdx.x];
    const int n1 = J.n1, n2 = J.n2, qc = J.qcols, rr = J.rrows;
    const int m = min(n1, n2), nref = min(n1 - 1, n2);
    const size_t na = (size_t)n1 * n2, nq = (size_t)n1 * qc;
    float2* base = reinterpret_cast<float2*>(la_smem);
    float2* M = in_smem ? base : J.A;
    float2* Qm = in_smem ? base + na : J.Q;
    float2* vhead = base + (in_smem ? na + nq : 0);
    float2* dph = vhead + max(nref, 1);
    float* vscale = reinterpret_cast<float*>(dph + m);
    float* red = vscale + max(nref, 1);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    if (in_smem)
        for (size_t e = tid; e < na; e += nt) M[e] = J.A[e];
    __syncthreads();

    for (int k = 0; k < nref; ++k) {
        const float2 a = M[k + (size_t)n1 * k];
        float s = 0.0f;
        for (int i = k + 1 + tid; i < n1; i += nt) s += abs2(M[i + (size_t)n1 * k]);
        s = block_sum(s, red);  // its barriers order every read of a before the write below
        if (s == 0.0f) {        // nothing below the diagonal: no reflector
            if (tid == 0) vscale[k] = 0.0f;
            continue;
        }
        const float absa = sqrtf(abs2(a));
        const float nrm = sqrtf(fmaf(absa, absa, s));
        const float2 ph = absa > 0.0f ? make_float2(a.x / absa, a.y / absa) : make_float2(1.0f, 0.0f);
        const float2 v0 = make_float2(ph.x * (absa + nrm), ph.y * (absa + nrm));
        const float scale = 1.0f / (nrm * (nrm + absa));  // H = I - scale v v^H
        if (tid == 0) {
            vhead[k] = v0;
            vscale[k] = scale;
        }
        const float2* v = M + (size_t)n1 * k;  // v(i) = M(i, k) for i > k
        for (int j = k + 1 + warp; j < n2; j += nw) {
            float2* col = M + (size_t)n1 * j;
            float2 w = lane == 0 ? cjmul(v0, col[k]) : make_float2(0.0f, 0.0f);
            for (int i = k + 1 + lane; i < n1; i += 32) {
                const float2 t = cjmul(v[i], col[i]);
                w.x += t.x;
                w.y += t.y;
            }
            w.x = warp_sum(w.x) * scale;
            w.y = warp_sum(w.y) * scale;
            if (lane == 0) {
                const float2 t = cmul(v0, w);
                col[k] = make_float2(col[k].x - t.x, col[k].y - t.y);
            }
            for (int i = k + 1 + lane; i < n1; i += 32) {
                const float2 t = cmul(v[i], w);
                col[i] = make_float2(col[i].x - t.x, col[i].y - t.y);
            }
        }
        if (tid == 0) M[k + (size_t)n1 * k] = make_float2(-ph.x * nrm, -ph.y * nrm);
        __syncthreads();
    }

    // Q = H_0 H_1 ... H_{nref-1} I(:, 0:qc), applied right to left; H_k leaves columns j < k
    for (int j = warp; j < qc; j += nw)
        for (int i = lane; i < n1; i += 32)
            Qm[i + (size_t)n1 * j] = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
    __syncthreads();
    for (int k = nref - 1; k >= 0; --k) {
        const float scale = vscale[k];
        if (scale == 0.0f) continue;
        const float2 v0 = vhead[k];
        const float2* v = M + (size_t)n1 * k;
        for (int j = k + warp; j < qc; j += nw) {
            float2* col = Qm + (size_t)n1 * j;
            float2 w = lane == 0 ? cjmul(v0, col[k]) : make_float2(0.0f, 0.0f);
            for (int i = k + 1 + lane; i < n1; i += 32) {
                const float2 t = cjmul(v[i], col[i]);
                w.x += t.x;
                w.y += t.y;
            }
            w.x = warp_sum(w.x) * scale;
            w.y = warp_sum(w.y) * scale;
            if (lane == 0) {
                const float2 t = cmul(v0, w);
                col[k] = make_float2(col[k].x - t.x, col[k].y - t.y);
            }
            for (int i = k + 1 + lane; i < n1; i += 32) {
                const float2 t = cmul(v[i], w);
                col[i] = make_float2(col[i].x - t.x, col[i].y - t.y);
            }
        }
        __syncthreads();
    }

    // phases of the diagonal of R
    for (int i = tid; i < m; i += nt) {
        const float2 d = M[i + (size_t)n1 * i];
        const float ad = sqrtf(abs2(d));
        dph[i] = ad > 0.0f ? make_float2(d.x / ad, d.y / ad) : make_float2(1.0f, 0.0f);
    }
    __syncthreads();
    for (int j = warp; j < n2; j += nw) {
        for (int i = lane; i < rr; i += 32) {
            float2 r = make_float2(0.0f, 0.0f);
            if (i < m && i <= j) {
                const float2 x = M[i + (size_t)n1 * j];
                r = (i == j) ? make_float2(sqrtf(abs2(x)), 0.0f) : cjmul(dph[i], x);
            }
            J.R[i + (size_t)rr * j] = r;
        }
    }
    for (int j = warp; j < qc; j += nw) {
        const float2 ph = j < m ? dph[j] : make_float2(1.0f, 0.0f);
        for (int i = lane; i < n1; i += 32) J.Q[i + (size_t)n1 * j] = cmul(Qm[i + (size_t)n1 * j], ph);
    }
}

int la_threads(int n1, int n2) { return max(n1, n2) > 64 ? 512 : 256; }

cudaError_t set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t tinv_smem_bytes(int n, bool in_smem) {
    return align16((in_smem ? sizeof(float2) * (size_t)n * n : 0) + sizeof(float2) * 3 * (size_t)n +
                   sizeof(int) * (size_t)n + 64 * sizeof(float));
}

size_t tqr_smem_bytes(int n1, int n2, int qcols, bool in_smem) {
    const size_t m = (size_t)std::min(n1, n2), nref = (size_t)std::max(std::min(n1 - 1, n2), 1);
    return align16((in_smem ? sizeof(float2) * ((size_t)n1 * n2 + (size_t)n1 * qcols) : 0) +
                   sizeof(float2) * (nref + m) + sizeof(float) * nref + 32 * sizeof(float));
}

cudaError_t launch_tinv(const LaJob* d_jobs, int njobs, int n, uint32_t* status, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const bool in_smem = tinv_smem_bytes(n, true) <= kLaSmemLimit;
    const size_t smem = tinv_smem_bytes(n, in_smem);
    const int rows = (n + 31) / 32;
#define TP_TINV_LAUNCH(R)                                                                      \
    do {                                                                                       \
        cudaError_t e = set_smem(reinterpret_cast<const void*>(tinv_kernel<R>), smem);          \
        if (e != cudaSuccess) return e;                                                        \
        tinv_kernel<R><<<njobs, la_threads(n, n), smem, s>>>(d_jobs, in_smem ? 1 : 0, status); \
    } while (0)
    if (rows <= 1) TP_TINV_LAUNCH(1);
    else if (rows <= 2) TP_TINV_LAUNCH(2);
    else if (rows <= 4) TP_TINV_LAUNCH(4);
    else if (rows <= 8) TP_TINV_LAUNCH(8);
    else TP_TINV_LAUNCH(16);
#undef TP_TINV_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_tqr(const LaJob* d_jobs, int njobs, int n1, int n2, int qcols, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const bool in_smem = tqr_smem_bytes(n1, n2, qcols, true) <= kLaSmemLimit;
    const size_t smem = tqr_smem_bytes(n1, n2, qcols, in_smem);
    cudaError_t e = set_smem(reinterpret_cast<const void*>(tqr_kernel), smem);
    if (e != cudaSuccess) return e;
    tqr_kernel<<<njobs, la_threads(n1, n2), smem, s>>>(d_jobs, in_smem ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace tp
