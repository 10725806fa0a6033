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
// Slices up to 128 wide are factorised in registers (tinv_reg_kernel, tqr_reg_kernel: one
// barrier per pivot or reflector, the pivot search or next reflector formed ahead by the warp
// that owns the next column).  For wider slices the whole slice (and Q) sits in shared memory
// when it fits (tinv_kernel, tqr_kernel); larger ones are worked on in place in global memory
// (the spectrum buffer), one CTA each, L2-resident.
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
//
// One barrier per step.  The warp that owns column k + 1 updates that column first, publishes
// it (double-buffered) with its pivot row and 1 / pivot, and only then updates its other
// columns, so the pivot search overlaps the other warps' updates.  Each warp takes row p_k of
// its own columns from lane p_k mod 32 by shuffles.  With g_i = a_ik / pivot the update is
// a_ij -= g_i a_(p_k) j on every row; column k is zeroed first and row p_k enters with
// a = 0 and g = -1 / pivot, which leaves -g_i in column k and the scaled pivot row in row p_k.
// ---------------------------------------------------------------------------------------
// p ? a : b through a PTX select the optimiser cannot see into: a chain of these over a
// register array stays a chain of selects instead of becoming an indexed access to a copy of
// the array in local memory.
__device__ __forceinline__ float sel(bool p, float a, float b) {
    float r;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\tselp.f32 %0, %1, %2, q;\n\t}"
        : "=f"(r) : "f"(a), "f"(b), "r"((unsigned)p));
    return r;
}
__device__ __forceinline__ float2 sel(bool p, float2 a, float2 b) {
    return make_float2(sel(p, a.x, b.x), sel(p, a.y, b.y));
}

// Row MI of the register tile (a compile-time index, chosen by a switch on the uniform row):
// its values on this warp's columns from lane lp, and its reset for the pivot row.
template <int MI, int RM, int CW>
__device__ __forceinline__ void row_from_lane(const float2 (&M)[RM][CW], float2 (&x)[CW], int lp) {
#pragma unroll
    for (int c = 0; c < CW; ++c)
        x[c] = make_float2(__shfl_sync(0xffffffffu, M[MI][c].x, lp), __shfl_sync(0xffffffffu, M[MI][c].y, lp));
}
template <int MI, int RM, int CW>
__device__ __forceinline__ void pivot_row_reset(float2 (&M)[RM][CW], float2 (&g)[RM], float2 inv) {
#pragma unroll
    for (int c = 0; c < CW; ++c) M[MI][c] = make_float2(0.0f, 0.0f);
    g[MI] = make_float2(-inv.x, -inv.y);
}

// Runs BODY(C) for the compile-time C in [0, 8) equal to the warp-uniform value v, so that the
// register tile is indexed by constants only.
#define TP_STATIC_SWITCH8(v, BODY)         \
    switch (v) {                           \
        case 0: BODY(0) break;             \
        case 1: BODY(1) break;             \
        case 2: BODY(2) break;             \
        case 3: BODY(3) break;             \
        case 4: BODY(4) break;             \
        case 5: BODY(5) break;             \
        case 6: BODY(6) break;             \
        case 7: BODY(7) break;             \
        default: break;                    \
    }

// Column CC of this warp: published to col_out with its pivot row among the available rows
// (-1 when the pivot is at or below the threshold) and 1 / pivot.  The arg-max is two warp
// reductions: the largest |a|^2 (its bit pattern, which orders non-negative floats; NaN counts
// as 0) and then the smallest row holding it.  Warp-level.
template <int CC, int RM, int CW>
__device__ __forceinline__ void tinv_publish(const float2 (&M)[RM][CW], uint32_t avail, float thr2,
                                             float2* col_out, int* pivot_out, float2* inv_out) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned best = 0u;
    int bi = 0x7fffffff;
#pragma unroll
    for (int m = 0; m < RM; ++m) {
        const float2 v = M[m][CC];
        col_out[lane + 32 * m] = v;
        const float a2 = abs2(v);
        const unsigned bits = (((avail >> m) & 1u) && a2 == a2) ? __float_as_uint(a2) : 0u;
        if (bits > best) {
            best = bits;
            bi = lane + 32 * m;
        }
    }
    const unsigned mx = __reduce_max_sync(kFull, best);
    const int p = (int)__reduce_min_sync(kFull, best == mx ? (unsigned)bi : 0xffffffffu);
    const float pv = __uint_as_float(mx);
    float2 a = M[0][CC];
#pragma unroll
    for (int m = 1; m < RM; ++m) a = sel(m == (p >> 5), M[m][CC], a);
    a = make_float2(__shfl_sync(kFull, a.x, p & 31), __shfl_sync(kFull, a.y, p & 31));
    if (lane == 0) {
        const bool ok = pv > thr2;
        *pivot_out = ok ? p : -1;
        *inv_out = ok ? crcp(a) : make_float2(0.0f, 0.0f);
    }
}

// a_ij -= g_i x_j on column c of the tile
template <int RM, int CW>
__device__ __forceinline__ void tinv_update(float2 (&M)[RM][CW], const float2 (&g)[RM], float2 xc, int c) {
#pragma unroll
    for (int m = 0; m < RM; ++m) {
        const float2 a = M[m][c];
        M[m][c] = make_float2(fmaf(-g[m].x, xc.x, fmaf(g[m].y, xc.y, a.x)),
                              fmaf(-g[m].x, xc.y, fmaf(-g[m].y, xc.x, a.y)));
    }
}
template <int CSKIP, int RM, int CW>
__device__ __forceinline__ void tinv_update_all_but(float2 (&M)[RM][CW], const float2 (&g)[RM],
                                                    const float2 (&x)[CW]) {
#pragma unroll
    for (int c = 0; c < CW; ++c)
        if (c != CSKIP) tinv_update(M, g, x[c], c);
}

template <int RM, int W, int CW>
__global__ void __launch_bounds__(32 * W) tinv_reg_kernel(const LaJob* __restrict__ jobs,
                                                          uint32_t* status) {
    static_assert(32 * RM == W * CW, "the register tile is square");
    constexpr int NC = 32 * RM;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ float2 colk[2][NC];
    __shared__ float2 pinv[2];
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

    if (warp == 0) tinv_publish<0>(M, avail, thr2, colk[0], &pivot[0], &pinv[0]);
    bool singular = false;
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        const int b = k & 1;
        const int p = pivot[b];
        if (p < 0) {
            singular = true;
            break;
        }
        if (threadIdx.x == 0) perm[k] = p;
        const float2 inv = pinv[b];
        const int lp = p & 31, mp = p >> 5;
        // row p of this warp's columns
        float2 x[CW];
#define TP_ROW(C) if constexpr (C < RM) row_from_lane<C>(M, x, lp);
        TP_STATIC_SWITCH8(mp, TP_ROW)
#undef TP_ROW
        float2 g[RM];
#pragma unroll
        for (int m = 0; m < RM; ++m) g[m] = cmul(colk[b][lane + 32 * m], inv);
        const int wk = k % W, ck = k / W;
        if (warp == wk) {  // column k: zero, and a unit entry in row p
#define TP_UNIT_COL(C)                                                 \
    if constexpr (C < CW) {                                            \
        x[C] = make_float2(1.0f, 0.0f);                                \
        _Pragma("unroll") for (int m = 0; m < RM; ++m) M[m][C] = make_float2(0.0f, 0.0f); \
    }
            TP_STATIC_SWITCH8(ck, TP_UNIT_COL)
#undef TP_UNIT_COL
        }
        if (lane == lp) {  // row p: a = 0, g = -1 / pivot
#define TP_RESET(C) if constexpr (C < RM) pivot_row_reset<C>(M, g, inv);
            TP_STATIC_SWITCH8(mp, TP_RESET)
#undef TP_RESET
            avail &= ~(1u << mp);
        }
        if (k + 1 < n && warp == (k + 1) % W) {
            // look-ahead: column k + 1 first, then its pivot, then the other columns
#define TP_AHEAD(C)                                                                      \
    if constexpr (C < CW) {                                                              \
        tinv_update(M, g, x[C], C);                                                      \
        tinv_publish<C>(M, avail, thr2, colk[b ^ 1], &pivot[b ^ 1], &pinv[b ^ 1]);       \
        tinv_update_all_but<C>(M, g, x);                                                 \
    }
            TP_STATIC_SWITCH8((k + 1) / W, TP_AHEAD)
#undef TP_AHEAD
        } else {
            tinv_update_all_but<-1>(M, g, x);
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
// takes it for 32 x 128, 64 x 64 and 128 x 64 tiles, which keep the tile in registers).  The
// layout of tinv_reg_kernel: lane l of warp w holds rows l + 32 m of columns w + 16 c, first
// of the slice and then of Q.  Step k: reflector k is in shared memory, where every reflector
// stays; after one barrier each warp applies it to its own columns j > k, the w = v^H a_j of
// all its columns summed over the warp together (warp_sum_all).  The warp that owns column
// k + 1 updates that column first, forms and publishes reflector k + 1 (a warp sum for the
// norm) and applies reflector k to its other columns only in the next step, so that the next
// reflector is ready when the others arrive.
// Q = H_0 ... H_(nref-1) I(:, 0:qcols) is then formed with no barrier at all, each warp
// applying the stored reflectors, last first, to its own columns of the identity.
// Shared memory: [V max(nref, 1) x 32 RM][diagonal phases 32 RM][scales max(nref, 1) floats].
// ---------------------------------------------------------------------------------------
constexpr int kQrWarps = 16;

// Sums each of the NV values of every lane over the warp; every lane receives all NV sums.
// Recursive halving over the values padded to a power of two P (in each round a lane keeps one
// half of its values, summed with its partner's copy of that half), plain butterflies for the
// remaining lane bits, then a gather: about 2 P + 5 - log2 P shuffles instead of 5 NV.
template <int NV>
__device__ __forceinline__ void warp_sum_all(float (&v)[NV]) {
    static_assert(NV >= 1 && NV <= 32, "up to 32 values");
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int P = NV > 16 ? 32 : NV > 8 ? 16 : NV > 4 ? 8 : NV > 2 ? 4 : NV > 1 ? 2 : 1;
    constexpr int R = P == 32 ? 5 : P == 16 ? 4 : P == 8 ? 3 : P == 4 ? 2 : P == 2 ? 1 : 0;
    const int lane = threadIdx.x & 31;
    float u[P];
#pragma unroll
    for (int i = 0; i < P; ++i) u[i] = i < NV ? v[i] : 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int o = 16 >> r, half = P >> (r + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? u[i] : u[i + half];
            const float keep = upper ? u[i + half] : u[i];
            u[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    float s = u[0];
#pragma unroll
    for (int o = 16 >> R; o >= 1; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    // lane L now holds the sum of value sum_r [L & (16 >> r)] (P >> (r + 1))
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        int src = 0;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (i & (P >> (r + 1))) src |= 16 >> r;
        v[i] = __shfl_sync(kFull, s, src);
    }
}

// Reflector kk of the QR from column CC of this warp, which is column kk: V_kk (zero above
// row kk), its scale (0 when nothing lies below the diagonal: no reflector) and beta on the
// diagonal.  have_hint: s_hint and a_hint already hold the squared norm below the diagonal and
// the diagonal element (qr_apply_one), else they are summed here.  Warp-level.
template <int CC, int RM, int CW>
__device__ __forceinline__ void qr_reflector(float2 (&M)[RM][CW], int kk, float2* vk, float* scale_out,
                                             bool have_hint, float s_hint, float2 a_hint) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float2 x[RM];
#pragma unroll
    for (int mm = 0; mm < RM; ++mm) x[mm] = M[mm][CC];
    float s = s_hint;
    float2 a = a_hint;
    if (!have_hint) {
        s = 0.0f;
        a = x[0];
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) {
            if (lane + 32 * mm > kk) s += abs2(x[mm]);
            if (mm > 0) a = sel(mm == (kk >> 5), x[mm], a);
        }
        s = warp_sum(s);
        a = make_float2(__shfl_sync(kFull, a.x, kk & 31), __shfl_sync(kFull, a.y, kk & 31));
    }
    float scale = 0.0f;
    if (s != 0.0f) {
        const float absa = sqrtf(abs2(a));
        const float nrm = sqrtf(fmaf(absa, absa, s));
        const float ra = __frcp_rn(absa);
        const float2 ph = absa > 0.0f ? make_float2(a.x * ra, a.y * ra) : make_float2(1.0f, 0.0f);
        scale = __frcp_rn(nrm * (nrm + absa));  // H = I - scale v v^H
        const float2 v0 = make_float2(ph.x * (absa + nrm), ph.y * (absa + nrm));
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) {
            const int i = lane + 32 * mm;
            vk[i] = i > kk ? x[mm] : (i == kk ? v0 : make_float2(0.0f, 0.0f));
        }
        const float2 beta = make_float2(-ph.x * nrm, -ph.y * nrm);  // the new diagonal
#pragma unroll
        for (int mm = 0; mm < RM; ++mm)
            M[mm][CC] = sel(mm == (kk >> 5) && lane == (kk & 31), beta, M[mm][CC]);
    }
    if (lane == 0) *scale_out = scale;
}

// T <- (I - v v^H mask_c) T on the columns c >= CLO of the tile; mask_c = 0 leaves column c
// as is.  Rows below 32 MLO are skipped, where v is zero.
template <int CLO, int MLO, int RM, int CW>
__device__ __forceinline__ void qr_apply(float2 (&T)[RM][CW], const float2 (&v)[RM], const float (&mask)[CW]) {
    constexpr int NC = CW - CLO;
    float w[2 * NC];
#pragma unroll
    for (int c = CLO; c < CW; ++c) {
        float wr = 0.0f, wi = 0.0f;
#pragma unroll
        for (int mm = MLO; mm < RM; ++mm) {
            wr = fmaf(v[mm].x, T[mm][c].x, fmaf(v[mm].y, T[mm][c].y, wr));
            wi = fmaf(v[mm].x, T[mm][c].y, fmaf(-v[mm].y, T[mm][c].x, wi));
        }
        w[2 * (c - CLO)] = wr;
        w[2 * (c - CLO) + 1] = wi;
    }
    warp_sum_all<2 * NC>(w);
#pragma unroll
    for (int c = CLO; c < CW; ++c) {
        const float wx = w[2 * (c - CLO)] * mask[c], wy = w[2 * (c - CLO) + 1] * mask[c];
#pragma unroll
        for (int mm = MLO; mm < RM; ++mm) {
            const float2 t = T[mm][c];
            T[mm][c] = make_float2(fmaf(-v[mm].x, wx, fmaf(v[mm].y, wy, t.x)),
                                   fmaf(-v[mm].x, wy, fmaf(-v[mm].y, wx, t.y)));
        }
    }
}

// Reflector k touches neither the columns c < k / 16 of any warp (done in the factorisation, or
// left unchanged in Q) nor the rows below 32 (k / 32), where it is zero.
#define TP_QR_APPLY(C)                                                                  \
    if constexpr (C < CW) qr_apply<C, (C / 2 < RM ? C / 2 : RM - 1)>(T_, v, mask);

// Reflector k (scale != 0) on column c alone, which is column k + 1, with its own warp sums.
// The same sums give the squared norm t of rows >= k, which the unitary reflector keeps, so the
// squared norm below the next diagonal is t - |y_k|^2 - |y_(k+1)|^2 with y the updated column
// (y_(k+1) is returned in a).  Returns whether that difference kept at least a quarter of t,
// i.e. lost at most two bits to cancellation; otherwise the caller sums it again.
template <int RM, int CW>
__device__ __forceinline__ bool qr_apply_one(float2 (&T)[RM][CW], const float2 (&v)[RM], float scale,
                                             int c, int k, float& s, float2& a) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float wr = 0.0f, wi = 0.0f, t = 0.0f;
#pragma unroll
    for (int mm = 0; mm < RM; ++mm) {
        wr = fmaf(v[mm].x, T[mm][c].x, fmaf(v[mm].y, T[mm][c].y, wr));
        wi = fmaf(v[mm].x, T[mm][c].y, fmaf(-v[mm].y, T[mm][c].x, wi));
        if (lane + 32 * mm >= k) t += abs2(T[mm][c]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        wr += __shfl_xor_sync(kFull, wr, o);
        wi += __shfl_xor_sync(kFull, wi, o);
        t += __shfl_xor_sync(kFull, t, o);
    }
    const float wx = wr * scale, wy = wi * scale;
#pragma unroll
    for (int mm = 0; mm < RM; ++mm) {
        const float2 u = T[mm][c];
        T[mm][c] = make_float2(fmaf(-v[mm].x, wx, fmaf(v[mm].y, wy, u.x)),
                               fmaf(-v[mm].x, wy, fmaf(-v[mm].y, wx, u.y)));
    }
    float2 yk = T[0][c], yk1 = T[0][c];
#pragma unroll
    for (int mm = 1; mm < RM; ++mm) {
        yk = sel(mm == (k >> 5), T[mm][c], yk);
        yk1 = sel(mm == ((k + 1) >> 5), T[mm][c], yk1);
    }
    yk = make_float2(__shfl_sync(kFull, yk.x, k & 31), __shfl_sync(kFull, yk.y, k & 31));
    a = make_float2(__shfl_sync(kFull, yk1.x, (k + 1) & 31), __shfl_sync(kFull, yk1.y, (k + 1) & 31));
    s = t - abs2(yk) - abs2(a);
    return s >= 0.25f * t;
}

template <int RM, int CW>
__global__ void __launch_bounds__(32 * kQrWarps) tqr_reg_kernel(const LaJob* __restrict__ jobs) {
    constexpr int W = kQrWarps, NR = 32 * RM;
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

    if (nref > 0 && warp == 0) qr_reflector<0>(M, 0, V, &vscale[0], false, 0.0f, make_float2(0.0f, 0.0f));
    // The warp that forms reflector k + 1 in step k leaves reflector k on its other columns
    // for step k + 1 (kd), so that its path to the barrier is the look-ahead alone.
    int kd = -1;
    for (int k = 0; k < nref; ++k) {
        __syncthreads();
        if (kd >= 0) {  // the deferred reflector first: columns j > kd except kd + 1
            const float sd = vscale[kd];
            if (sd != 0.0f) {
                float2 v[RM];
#pragma unroll
                for (int mm = 0; mm < RM; ++mm) v[mm] = V[(size_t)kd * NR + lane + 32 * mm];
                float mask[CW];
                bool any = false;
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    const int j = warp + W * c;
                    const bool on = j > kd + 1 && j < n2;
                    mask[c] = on ? sd : 0.0f;
                    any |= on;
                }
                if (any) {
                    auto& T_ = M;
                    TP_STATIC_SWITCH8(kd >> 4, TP_QR_APPLY)
                }
            }
            kd = -1;
        }
        const float scale = vscale[k];
        float2 v[RM];
#pragma unroll
        for (int mm = 0; mm < RM; ++mm)
            v[mm] = scale != 0.0f ? V[(size_t)k * NR + lane + 32 * mm] : make_float2(0.0f, 0.0f);
        if (k + 1 < nref && warp == (k + 1) % W) {  // look-ahead: column k + 1, reflector k + 1
#define TP_AHEAD(C)                                                                   \
    if constexpr (C < CW) {                                                           \
        float sh = 0.0f;                                                              \
        float2 ah = make_float2(0.0f, 0.0f);                                          \
        const bool hint = scale != 0.0f && qr_apply_one(M, v, scale, C, k, sh, ah);   \
        qr_reflector<C>(M, k + 1, V + (size_t)(k + 1) * NR, &vscale[k + 1], hint, sh, ah); \
    }
            TP_STATIC_SWITCH8((k + 1) / W, TP_AHEAD)
#undef TP_AHEAD
            kd = k;
            continue;
        }
        if (scale == 0.0f) continue;
        float mask[CW];
        bool any = false;
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const int j = warp + W * c;
            const bool on = j > k && j < n2;
            mask[c] = on ? scale : 0.0f;
            any |= on;
        }
        if (any) {
            auto& T_ = M;
            TP_STATIC_SWITCH8(k >> 4, TP_QR_APPLY)
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
        if (scale == 0.0f || warp + W * (CW - 1) < k) continue;
        float2 v[RM];
#pragma unroll
        for (int mm = 0; mm < RM; ++mm) v[mm] = V[(size_t)k * NR + lane + 32 * mm];
        float mask[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const int j = warp + W * c;
            mask[c] = (j >= k && j < qc) ? scale : 0.0f;
        }
        auto& T_ = Q;
        TP_STATIC_SWITCH8(k >> 4, TP_QR_APPLY)
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
