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
// Register-resident slice inverse for n <= 32 RM.  Lane l of warp w holds rows l + 32 m
// (m < RM) of columns w + W c (c < CW) in registers for the whole elimination, so a step reads
// and writes no matrix element in memory.  The rows are not exchanged: step k takes as pivot
// the largest |a_ik| among the rows not yet used (physical row p_k), scales row p_k and reduces
// every other row, as the kernel above does after its exchange.  Regarding the matrix as the
// map y = A x, each such step swaps the roles of x_k and y_(p_k), so after n steps the element
// at (p_k, j) is element (k, p_j) of the inverse; the final store applies that permutation.
// One barrier per step: the warp that owns column k chooses the pivot and publishes the
// column (double-buffered), and each warp takes row p_k of its own columns from lane p_k mod 32
// by shuffles.
// ---------------------------------------------------------------------------------------
template <int RM, int W, int CW>
__global__ void __launch_bounds__(32 * W) tinv_reg_kernel(const LaJob* __restrict__ jobs,
                                                          uint32_t* status) {
    static_assert(32 * RM == W * CW, "the register tile is square");
    constexpr int NC = 32 * RM;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ float2 colk[2][NC];
    __shared__ int pivot[2];
    __shared__ int perm[NC], iperm[NC];
    __shared__ float red[W];
    const LaJob J = jobs[blockIdx.x];
    const int n = J.n1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float2 M[RM][CW];
    float amax2 = 0.0f;
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int m = 0; m < RM; ++m) {
            const int i = lane + 32 * m, j = warp + W * c;
            M[m][c] = (i < n && j < n) ? J.A[i + (size_t)n * j] : make_float2(0.0f, 0.0f);
            amax2 = fmaxf(amax2, abs2(M[m][c]));
        }
    for (int o = 16; o; o >>= 1) amax2 = fmaxf(amax2, __shfl_xor_sync(kFull, amax2, o));
    if (lane == 0) red[warp] = amax2;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < W; ++w) amax2 = fmaxf(amax2, red[w]);
    // the singularity threshold of the kernel above
    const float thr = (float)n * kEps;
    const float thr2 = thr * thr * amax2;
    uint32_t avail = 0;  // bit m: row lane + 32 m can still be a pivot
#pragma unroll
    for (int m = 0; m < RM; ++m)
        if (lane + 32 * m < n) avail |= 1u << m;

    bool singular = false;
    for (int k = 0; k < n; ++k) {
        const int b = k & 1;
        const int wk = k % W, ck = k / W;
        if (warp == wk) {  // owner of column k: publish it and choose the pivot
            float pv = -1.0f;
            int p = 0x7fffffff;
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (c == ck) {
#pragma unroll
                    for (int m = 0; m < RM; ++m) {
                        colk[b][lane + 32 * m] = M[m][c];
                        if ((avail >> m) & 1u) argmax_step(pv, p, abs2(M[m][c]), lane + 32 * m);
                    }
                }
            for (int o = 16; o; o >>= 1)
                argmax_step(pv, p, __shfl_xor_sync(kFull, pv, o), __shfl_xor_sync(kFull, p, o));
            if (lane == 0) pivot[b] = pv > thr2 ? p : -1;  // also catches NaN and Inf
        }
        __syncthreads();
        const int p = pivot[b];
        if (p < 0) {
            singular = true;
            break;
        }
        if (threadIdx.x == 0) perm[k] = p;
        const float2 inv = crcp(colk[b][p]);
        const int lp = p & 31, mp = p >> 5;
        // the scaled pivot row on this warp's columns; 1 / pivot in column k
        float2 r[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) r[c] = M[0][c];
#pragma unroll
        for (int m = 1; m < RM; ++m)
            if (m == mp) {
#pragma unroll
                for (int c = 0; c < CW; ++c) r[c] = M[m][c];
            }
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const float2 x = make_float2(__shfl_sync(kFull, r[c].x, lp), __shfl_sync(kFull, r[c].y, lp));
            r[c] = cmul(x, inv);
        }
        if (warp == wk) {  // column k: a_ik <- 0 before the update, so it ends at -f_i / pivot
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (c == ck) {
                    r[c] = inv;
#pragma unroll
                    for (int m = 0; m < RM; ++m) M[m][c] = make_float2(0.0f, 0.0f);
                }
        }
#pragma unroll
        for (int m = 0; m < RM; ++m) {
            const float2 f = colk[b][lane + 32 * m];
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                const float2 a = M[m][c];
                M[m][c] = make_float2(fmaf(-f.x, r[c].x, fmaf(f.y, r[c].y, a.x)),
                                      fmaf(-f.x, r[c].y, fmaf(-f.y, r[c].x, a.y)));
            }
        }
        if (lane == lp) {  // the pivot row itself becomes the scaled row
#pragma unroll
            for (int m = 0; m < RM; ++m)
                if (m == mp) {
#pragma unroll
                    for (int c = 0; c < CW; ++c) M[m][c] = r[c];
                }
            avail &= ~(1u << mp);
        }
    }
    if (singular) {
        const float qnan = __int_as_float(0x7fc00000);
        for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) J.R[e] = make_float2(qnan, qnan);
        if (threadIdx.x == 0 && status) atomicOr(status, 2u);
        return;
    }
    __syncthreads();  // perm complete
    for (int t = threadIdx.x; t < n; t += blockDim.x) iperm[perm[t]] = t;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int j = warp + W * c;
        if (j >= n) continue;
        const size_t col = (size_t)n * perm[j];
#pragma unroll
        for (int m = 0; m < RM; ++m) {
            const int i = lane + 32 * m;
            if (i < n) J.R[iperm[i] + col] = M[m][c];
        }
    }
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

// ---------------------------------------------------------------------------------------
// Register-resident slice QR for n1 <= 32 RM and n2, qcols <= 16 CW, 16 warps (the launcher
// takes it for 32 x 128, 64 x 64 and 128 x 64 tiles, which keep the tile in registers).  The layout of
// tinv_reg_kernel: lane l of warp w holds rows l + 32 m of columns w + 16 c, first of the
// slice and then of Q.  Step k: the warp that owns column k forms reflector k from its
// registers (a warp sum for the norm) and publishes it to shared memory, where every reflector
// stays; after one barrier each warp applies it to its own columns j > k (a warp sum per
// column for w = v^H a_j).  Q = H_0 ... H_(nref-1) I(:, 0:qcols) is then formed column by
// column with no barrier at all, each warp applying the stored reflectors to its own columns
// of the identity, last reflector first.  Shared memory: [V max(nref, 1) x 32 RM]
// [diagonal phases 32 RM][scales max(nref, 1) floats].
// ---------------------------------------------------------------------------------------
constexpr int kQrWarps = 16;

template <int RM, int CW>
__global__ void __launch_bounds__(32 * kQrWarps) tqr_reg_kernel(const LaJob* __restrict__ jobs) {
    constexpr int W = kQrWarps, NR = 32 * RM;
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ float4 la_smem[];
    const LaJob J = jobs[blockIdx.x];
    const int n1 = J.n1, n2 = J.n2, qc = J.qcols, rr = J.rrows;
    const int m = min(n1, n2), nref = min(n1 - 1, n2);
    float2* V = reinterpret_cast<float2*>(la_smem);
    float2* dph = V + (size_t)max(nref, 1) * NR;
    float* vscale = reinterpret_cast<float*>(dph + NR);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float2 M[RM][CW];
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) {
            const int i = lane + 32 * mm, j = warp + W * c;
            M[mm][c] = (i < n1 && j < n2) ? J.A[i + (size_t)n1 * j] : make_float2(0.0f, 0.0f);
        }

    for (int k = 0; k < nref; ++k) {
        const int wk = k % W, ck = k / W;
        float2* vk = V + (size_t)k * NR;
        if (warp == wk) {  // owner of column k: reflector k
            float2 x[RM];
#pragma unroll
            for (int mm = 0; mm < RM; ++mm) x[mm] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (c == ck) {
#pragma unroll
                    for (int mm = 0; mm < RM; ++mm) x[mm] = M[mm][c];
                }
            float s = 0.0f;
            float2 a = x[0];
#pragma unroll
            for (int mm = 0; mm < RM; ++mm) {
                if (lane + 32 * mm > k) s += abs2(x[mm]);
                if (mm == (k >> 5)) a = x[mm];
            }
            s = warp_sum(s);
            a = make_float2(__shfl_sync(kFull, a.x, k & 31), __shfl_sync(kFull, a.y, k & 31));
            float scale = 0.0f;  // s == 0: nothing below the diagonal, no reflector
            if (s != 0.0f) {
                const float absa = sqrtf(abs2(a));
                const float nrm = sqrtf(fmaf(absa, absa, s));
                const float2 ph = absa > 0.0f ? make_float2(a.x / absa, a.y / absa) : make_float2(1.0f, 0.0f);
                scale = 1.0f / (nrm * (nrm + absa));  // H = I - scale v v^H
                const float2 v0 = make_float2(ph.x * (absa + nrm), ph.y * (absa + nrm));
#pragma unroll
                for (int mm = 0; mm < RM; ++mm) {
                    const int i = lane + 32 * mm;
                    vk[i] = i > k ? x[mm] : (i == k ? v0 : make_float2(0.0f, 0.0f));
                }
                if (lane == (k & 31)) {  // the diagonal becomes beta = -phase(a) ||x||
#pragma unroll
                    for (int c = 0; c < CW; ++c)
                        if (c == ck) {
#pragma unroll
                            for (int mm = 0; mm < RM; ++mm)
                                if (mm == (k >> 5)) M[mm][c] = make_float2(-ph.x * nrm, -ph.y * nrm);
                        }
                }
            }
            if (lane == 0) vscale[k] = scale;
        }
        __syncthreads();
        const float scale = vscale[k];
        if (scale == 0.0f) continue;
        float2 v[RM];
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) v[mm] = vk[lane + 32 * mm];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const int j = warp + W * c;
            if (j <= k || j >= n2) continue;
            float2 w = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int mm = 0; mm < RM; ++mm) {
                const float2 t = cjmul(v[mm], M[mm][c]);
                w.x += t.x;
                w.y += t.y;
            }
            w.x = warp_sum(w.x) * scale;
            w.y = warp_sum(w.y) * scale;
#pragma unroll
            for (int mm = 0; mm < RM; ++mm) {
                const float2 t = cmul(v[mm], w);
                M[mm][c] = make_float2(M[mm][c].x - t.x, M[mm][c].y - t.y);
            }
        }
    }

    // phases of the diagonal of R, then R with row i rotated by conj(phase_i)
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int j = warp + W * c;
#pragma unroll
        for (int mm = 0; mm < RM; ++mm)
            if (j < m && lane + 32 * mm == j) {
                const float2 d = M[mm][c];
                const float ad = sqrtf(abs2(d));
                dph[j] = ad > 0.0f ? make_float2(d.x / ad, d.y / ad) : make_float2(1.0f, 0.0f);
            }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int j = warp + W * c;
        if (j >= n2) continue;
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) {
            const int i = lane + 32 * mm;
            if (i >= rr) continue;
            float2 r = make_float2(0.0f, 0.0f);
            if (i < m && i <= j) {
                const float2 x = M[mm][c];
                r = (i == j) ? make_float2(sqrtf(abs2(x)), 0.0f) : cjmul(dph[i], x);
            }
            J.R[i + (size_t)rr * j] = r;
        }
    }

    // Q: the reflectors, last first, on this warp's columns of the identity; H_k leaves
    // column j < k unchanged
    float2 Q[RM][CW];
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int mm = 0; mm < RM; ++mm)
            Q[mm][c] = make_float2(lane + 32 * mm == warp + W * c ? 1.0f : 0.0f, 0.0f);
    for (int k = nref - 1; k >= 0; --k) {
        const float scale = vscale[k];
        if (scale == 0.0f) continue;
        const float2* vk = V + (size_t)k * NR;
        float2 v[RM];
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) v[mm] = vk[lane + 32 * mm];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const int j = warp + W * c;
            if (j < k || j >= qc) continue;
            float2 w = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int mm = 0; mm < RM; ++mm) {
                const float2 t = cjmul(v[mm], Q[mm][c]);
                w.x += t.x;
                w.y += t.y;
            }
            w.x = warp_sum(w.x) * scale;
            w.y = warp_sum(w.y) * scale;
#pragma unroll
            for (int mm = 0; mm < RM; ++mm) {
                const float2 t = cmul(v[mm], w);
                Q[mm][c] = make_float2(Q[mm][c].x - t.x, Q[mm][c].y - t.y);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int j = warp + W * c;
        if (j >= qc) continue;
        const float2 ph = j < m ? dph[j] : make_float2(1.0f, 0.0f);
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) {
            const int i = lane + 32 * mm;
            if (i < n1) J.Q[i + (size_t)n1 * j] = cmul(Q[mm][c], ph);
        }
    }
}

size_t tqr_reg_smem_bytes(int n1, int n2) {
    const size_t nr = n1 <= 32 ? 32 : (n1 <= 64 ? 64 : 128);
    const size_t nref = (size_t)std::max(std::min(n1 - 1, n2), 1);
    return align16(sizeof(float2) * (nref * nr + nr) + sizeof(float) * nref);
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
    if (n <= 128) {  // register-resident: 32 x 32, 64 x 64 or 128 x 128 tile
        if (n <= 32) tinv_reg_kernel<1, 8, 4><<<njobs, 256, 0, s>>>(d_jobs, status);
        else if (n <= 64) tinv_reg_kernel<2, 8, 8><<<njobs, 256, 0, s>>>(d_jobs, status);
        else tinv_reg_kernel<4, 16, 8><<<njobs, 512, 0, s>>>(d_jobs, status);
        return cudaGetLastError();
    }
    const bool in_smem = tinv_smem_bytes(n, true) <= kLaSmemLimit;
    const size_t smem = tinv_smem_bytes(n, in_smem);
    const int rows = (n + 31) / 32;
#define TP_TINV_LAUNCH(R)                                                                      \
    do {                                                                                       \
        cudaError_t e = set_smem(reinterpret_cast<const void*>(tinv_kernel<R>), smem);          \
        if (e != cudaSuccess) return e;                                                        \
        tinv_kernel<R><<<njobs, la_threads(n, n), smem, s>>>(d_jobs, in_smem ? 1 : 0, status); \
    } while (0)
    if (rows <= 8) TP_TINV_LAUNCH(8);  // n > 128 here
    else TP_TINV_LAUNCH(16);
#undef TP_TINV_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_tqr(const LaJob* d_jobs, int njobs, int n1, int n2, int qcols, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const int cols = std::max(n2, qcols);
    // register-resident where the tile fits the registers: 32 x 128, 64 x 64 or 128 x 64
    if ((n1 <= 32 && cols <= 128) || (n1 <= 128 && cols <= 64)) {
        const size_t smem = tqr_reg_smem_bytes(n1, n2);
#define TP_TQR_REG(RM, CW)                                                                   \
    do {                                                                                     \
        cudaError_t e = set_smem(reinterpret_cast<const void*>(tqr_reg_kernel<RM, CW>), smem); \
        if (e != cudaSuccess) return e;                                                      \
        tqr_reg_kernel<RM, CW><<<njobs, 32 * kQrWarps, smem, s>>>(d_jobs);                   \
    } while (0)
#define TP_TQR_REG_COLS(RM)                     \
    do {                                        \
        if (cols <= 32) TP_TQR_REG(RM, 2);      \
        else TP_TQR_REG(RM, 4);                 \
    } while (0)
        if (n1 <= 32) {
            if (cols <= 64) TP_TQR_REG_COLS(1);
            else TP_TQR_REG(1, 8);
        } else if (n1 <= 64) {
            TP_TQR_REG_COLS(2);
        } else {
            TP_TQR_REG_COLS(4);
        }
#undef TP_TQR_REG_COLS
#undef TP_TQR_REG
        return cudaGetLastError();
    }
    const bool in_smem = tqr_smem_bytes(n1, n2, qcols, true) <= kLaSmemLimit;
    const size_t smem = tqr_smem_bytes(n1, n2, qcols, in_smem);
    cudaError_t e = set_smem(reinterpret_cast<const void*>(tqr_kernel), smem);
    if (e != cudaSuccess) return e;
    tqr_kernel<<<njobs, la_threads(n1, n2), smem, s>>>(d_jobs, in_smem ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace tp
