// Learned-rank randomized singular value thresholding of the Fourier slices: the fast path
// of prox_tnn (Algorithm 3, step 2) for slices whose number of singular values above tau is
// small, with the full one-sided Jacobi SVD (tp_svd.cu) as fallback and accuracy reference.
//
// Per slice A (n1 x n2 complex, column-major, in place in the half spectrum):
//   1. a tiny MLP (12 -> 64 -> 64 -> 1, ReLU) reads cheap sketch features -- log ||A||_F / tau,
//      the diagonal of the QR factor of an 8-column sketch A Omega_8 over tau, log n1, log n2,
//      log min(n1, n2) -- and predicts k = #{sigma > tau}; the sketch width is l = k + 4;
//   2. randomized range finder: Y = A Omega (Omega n2 x l, random +-1 / (+-1 +- i)/sqrt 2
//      from a counter-based hash), q power iterations (Z = A^H Q, Y = A Z), each followed by
//      shifted CholeskyQR3 orthonormalisation, Q = orth(Y) (rank revealing: columns that
//      are dependent to working precision become zero columns);
//   3. small SVD: Z = A^H Q (n2 x l) = B^H; one-sided Jacobi over the whole CTA turns Z into
//      D = Z V with orthogonal columns, sigma_j = ||d_j||, so
//      A ~ Q Z^H = (Q V) diag(sigma) (D / sigma)^H;
//   4. acceptance: (a) the smallest of the l computed singular values is below tau (else the
//      rank was underestimated); (b) every kept triplet (u, sigma, r) has
//      ||A r - sigma u|| (sigma - tau) / sigma <= rtol * sigma_max, its weight in W; (c) two
//      power iterations on the deflated matrix
//      A - U_k S_k R_k^H estimate its norm below 0.8 tau (no singular value above tau missed);
//   5. W = sum_{sigma_j > tau} (sigma_j - tau) u_j r_j^H written over A.
// A slice that fails a check keeps A untouched and is flagged; the Jacobi SVT kernel then
// processes exactly the flagged slices.  The MLP is trained with hand-written kernels on
// (features, #{sigma > tau}) pairs produced by the plain Jacobi path.
#include <math.h>

#include <mutex>
#include <vector>

#include "tp_internal.cuh"
#include "tp_rotation.cuh"

namespace tp {

namespace {

constexpr int kT = 256;   // threads per CTA of the feature and training kernels
constexpr int kTS = 256;  // threads per CTA of the sketch kernel
constexpr int kLMax = kSketchMaxL;
constexpr int kD = kProposerInputs;
constexpr int kH = 64;
constexpr int kW1 = 0, kB1 = kW1 + kH * kD, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kH, kMean = kB3 + 1, kStd = kMean + kD, kNParams = kMean;
static_assert(kStd + kD == kProposerFloats, "proposer layout");

// Per-device proposer: weights, biases and the feature standardisation.
__device__ float g_proposer[kProposerFloats];

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

// Entry (r, c) of the random test matrix of slice `slice`: +-1 on real slices,
// (+-1 +- i)/sqrt(2) otherwise.
__device__ __forceinline__ float2 omega(uint32_t seed, uint32_t slice, uint32_t r, uint32_t c,
                                        bool real) {
    const uint32_t h = mix32(seed ^ mix32(slice * 0x9e3779b9u ^ mix32(r * 0x632be5abu + c)));
    const float a = (h & 1u) ? 1.f : -1.f, b = (h & 2u) ? 1.f : -1.f;
    return real ? make_float2(a, 0.f) : make_float2(a * 0.70710678f, b * 0.70710678f);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ float block_sum(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < kT / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

__device__ __forceinline__ float2 ld_a(const float2* A, int64_t idx, bool real) {
    float2 v = A[idx];
    if (real) v.y = 0.f;
    return v;
}

// Y (n1 x l, ld n1) = A X (X: n2 x l, ld n2, shared).  A work item is one row of Y and a
// chunk of 4 of its columns; all threads of the CTA share the items.
__device__ void mult_a(const float2* __restrict__ A, int n1, int n2, bool real, const float2* X,
                       float2* Y, int l) {
    const int nch = (l + 3) >> 2;
    for (int t = threadIdx.x; t < n1 * nch; t += (int)blockDim.x) {
        const int i = t % n1, j0 = (t / n1) * 4;
        const int jn = min(4, l - j0);
        float2 acc[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[jj] = make_float2(0.f, 0.f);
        const float2* x = X + (size_t)n2 * j0;
#pragma unroll 4
        for (int c = 0; c < n2; ++c) {
            const float2 a = ld_a(A, i + (int64_t)n1 * c, real);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                if (jj < jn) {
                    const float2 xv = x[c + (size_t)n2 * jj];
                    acc[jj].x = fmaf(a.x, xv.x, fmaf(-a.y, xv.y, acc[jj].x));
                    acc[jj].y = fmaf(a.x, xv.y, fmaf(a.y, xv.x, acc[jj].y));
                }
            }
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
            if (jj < jn) Y[i + (size_t)n1 * (j0 + jj)] = acc[jj];
    }
}

// Z (n2 x l, ld n2) = A^H Y (Y: n1 x l, ld n1, shared).  A work item is one column of A, a
// chunk of 4 columns of Y and (when items are fewer than threads) a range of rows; partial
// sums over row ranges meet in Z through shared-memory atomics.
__device__ void mult_ah(const float2* __restrict__ A, int n1, int n2, bool real, const float2* Y,
                        float2* Z, int l) {
    const int nch = (l + 3) >> 2;
    const int items = n2 * nch;
    const int parts = max(1, min((int)blockDim.x / max(items, 1), 8));
    const int span = (n1 + parts - 1) / parts;
    if (parts > 1) {
        for (int t = threadIdx.x; t < n2 * l; t += (int)blockDim.x) Z[t] = make_float2(0.f, 0.f);
        __syncthreads();
    }
    for (int t = threadIdx.x; t < items * parts; t += (int)blockDim.x) {
        const int c = t % n2, rest = t / n2, ch = rest % nch, pr = rest / nch;
        const int j0 = ch * 4, jn = min(4, l - j0);
        const int i0 = pr * span, i1 = min(n1, i0 + span);
        float2 acc[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[jj] = make_float2(0.f, 0.f);
        const float2* y = Y + (size_t)n1 * j0;
#pragma unroll 4
        for (int i = i0; i < i1; ++i) {
            const float2 a = ld_a(A, i + (int64_t)n1 * c, real);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                if (jj < jn) {
                    const float2 yv = y[i + (size_t)n1 * jj];
                    acc[jj].x = fmaf(a.x, yv.x, fmaf(a.y, yv.y, acc[jj].x));  // conj(a) y
                    acc[jj].y = fmaf(a.x, yv.y, fmaf(-a.y, yv.x, acc[jj].y));
                }
            }
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            if (jj < jn) {
                float2* z = Z + c + (size_t)n2 * (j0 + jj);
                if (parts == 1) {
                    *z = acc[jj];
                } else {
                    atomicAdd(&z->x, acc[jj].x);
                    atomicAdd(&z->y, acc[jj].y);
                }
            }
        }
    }
    __syncthreads();
}

// G (l x l, column-major, full Hermitian) = Y^H Y for Y n x l (ld n).
__device__ void gram(const float2* Y, int n, int l, float2* G) {
    for (int t = threadIdx.x; t < l * l; t += (int)blockDim.x) {
        const int a = t % l, b = t / l;
        if (a > b) continue;
        const float2* ya = Y + (size_t)n * a;
        const float2* yb = Y + (size_t)n * b;
        float gr = 0.f, gi = 0.f;
#pragma unroll 4
        for (int e = 0; e < n; ++e) {
            const float2 u = ya[e], v = yb[e];
            gr = fmaf(u.x, v.x, fmaf(u.y, v.y, gr));  // conj(u) v
            gi = fmaf(u.x, v.y, fmaf(-u.y, v.x, gi));
        }
        G[a + l * b] = make_float2(gr, gi);
        G[b + l * a] = make_float2(gr, -gi);
    }
    __syncthreads();
}

// C (l x l, upper triangular) with C^H (G + shift I) C = I, i.e. C = R^-1 for the Cholesky
// factor R^H R = G + shift I: Gram-Schmidt of the unit vectors e_0..e_{l-1} in the
// (G + shift I) inner product, each normalised vector projected out of all later ones at
// once.  G is overwritten by M = (G + shift I) C, kept current column by column, so that
// every step needs only dot products of length l: warp 0 normalises c_j (and m_j), then one
// half-warp per later column k forms h = m_j^H c_k and updates c_k -= h c_j, m_k -= h m_j.
// Rank revealing: a column whose squared norm after the projections, c_j^H m_j, is at most
// drop_tol times its squared norm before them (G_jj + shift) lies in the span of the earlier
// columns to working precision; it is dropped (c_j = m_j = 0), so Y C gets a zero column
// there instead of a normalised rounding error.  Returns false (uniformly) only if a norm is
// not a number.
__device__ bool chol_inv_narrow(float2* G, float2* C, int l, float shift, float drop_tol,
                                int* s_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < l * l; t += kTS) {
        const bool d = (t % l) == (t / l);
        C[t] = make_float2(d ? 1.f : 0.f, 0.f);
        if (d) G[t].x += shift;
    }
    __syncthreads();
    // squared column norms before the projections (warp 0, lane j: column j)
    const float dreg = (warp == 0 && lane < l) ? G[lane + l * lane].x : 0.f;
    const int hw = tid >> 4, hl = tid & 15;  // 16 half-warps; rows hl and hl + 16
    for (int j = 0; j < l; ++j) {
        if (warp == 0) {
            const float2 cj = lane <= j ? C[lane + l * j] : make_float2(0.f, 0.f);
            const float2 mj = lane < l ? G[lane + l * j] : make_float2(0.f, 0.f);
            const float p = warp_sum(fmaf(cj.x, mj.x, cj.y * mj.y));  // c_j^H m_j (real)
            const float dj = __shfl_sync(0xffffffffu, dreg, j);
            const bool keep = p > drop_tol * dj;
            const float inv = keep ? 1.f / sqrtf(p) : 0.f;
            if (lane <= j) C[lane + l * j] = make_float2(cj.x * inv, cj.y * inv);
            if (lane < l) G[lane + l * j] = make_float2(mj.x * inv, mj.y * inv);
            if (lane == 0) *s_flag = (p == p) ? 0 : 1;
        }
        __syncthreads();
        if (*s_flag) return false;
        for (int kb = j + 1; kb < l; kb += kTS / 16) {  // uniform over each warp
            const int k = kb + hw;
            const bool act = k < l;
            float hr = 0.f, hi = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = hl + 16 * h;
                if (act && m <= k) {
                    const float2 mm = G[m + l * j], c = C[m + l * k];
                    hr = fmaf(mm.x, c.x, fmaf(mm.y, c.y, hr));  // conj(m_j) c_k
                    hi = fmaf(mm.x, c.y, fmaf(-mm.y, c.x, hi));
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                hr += __shfl_xor_sync(0xffffffffu, hr, o);
                hi += __shfl_xor_sync(0xffffffffu, hi, o);
            }
            if (act) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int m = hl + 16 * h;
                    if (m <= j) {
                        const float2 cj = C[m + l * j];
                        float2 c = C[m + l * k];
                        c.x -= fmaf(hr, cj.x, -hi * cj.y);
                        c.y -= fmaf(hr, cj.y, hi * cj.x);
                        C[m + l * k] = c;
                    }
                    if (m < l) {
                        const float2 mj = G[m + l * j];
                        float2 mk = G[m + l * k];
                        mk.x -= fmaf(hr, mj.x, -hi * mj.y);
                        mk.y -= fmaf(hr, mj.y, hi * mj.x);
                        G[m + l * k] = mk;
                    }
                }
            }
        }
        __syncthreads();
    }
    return true;
}

__device__ bool chol_inv_wide(float2* G, float2* C, int l, float shift, float drop_tol,
                              int* s_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int t = tid; t < l * l; t += kTS) {
        const bool d = (t % l) == (t / l);
        C[t] = make_float2(d ? 1.f : 0.f, 0.f);
        if (d) G[t].x += shift;
    }
    __syncthreads();
    static_assert(kLMax <= 64, "two squared norms per lane");
    const float dreg0 = (warp == 0 && lane < l) ? G[lane + l * lane].x : 0.f;
    const float dreg1 = (warp == 0 && lane + 32 < l) ? G[lane + 32 + l * (lane + 32)].x : 0.f;
    constexpr int kRowSets = (kLMax + 15) / 16;  // rows hl + 16 h of a half-warp, h < kRowSets
    const int hw = tid >> 4, hl = tid & 15;       // 16 half-warps
    for (int j = 0; j < l; ++j) {
        if (warp == 0) {
            float p = 0.f;
            for (int m = lane; m <= j; m += 32) {
                const float2 cj = C[m + l * j], mj = G[m + l * j];
                p = fmaf(cj.x, mj.x, fmaf(cj.y, mj.y, p));  // c_j^H m_j (real)
            }
            p = warp_sum(p);
            const float d0 = __shfl_sync(0xffffffffu, dreg0, j & 31);
            const float d1 = __shfl_sync(0xffffffffu, dreg1, j & 31);
            const bool keep = p > drop_tol * (j < 32 ? d0 : d1);
            const float inv = keep ? 1.f / sqrtf(p) : 0.f;
            for (int m = lane; m < l; m += 32) {
                if (m <= j) { C[m + l * j].x *= inv; C[m + l * j].y *= inv; }
                G[m + l * j].x *= inv;
                G[m + l * j].y *= inv;
            }
            if (lane == 0) *s_flag = (p == p) ? 0 : 1;
        }
        __syncthreads();
        if (*s_flag) return false;
        for (int kb = j + 1; kb < l; kb += kTS / 16) {  // uniform over each warp
            const int k = kb + hw;
            const bool act = k < l;
            float hr = 0.f, hi = 0.f;
#pragma unroll
            for (int h = 0; h < kRowSets; ++h) {
                const int m = hl + 16 * h;
                if (act && m <= k) {
                    const float2 mm = G[m + l * j], c = C[m + l * k];
                    hr = fmaf(mm.x, c.x, fmaf(mm.y, c.y, hr));  // conj(m_j) c_k
                    hi = fmaf(mm.x, c.y, fmaf(-mm.y, c.x, hi));
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                hr += __shfl_xor_sync(0xffffffffu, hr, o);
                hi += __shfl_xor_sync(0xffffffffu, hi, o);
            }
            if (act) {
#pragma unroll
                for (int h = 0; h < kRowSets; ++h) {
                    const int m = hl + 16 * h;
                    if (m <= j) {
                        const float2 cj = C[m + l * j];
                        float2 c = C[m + l * k];
                        c.x -= fmaf(hr, cj.x, -hi * cj.y);
                        c.y -= fmaf(hr, cj.y, hi * cj.x);
                        C[m + l * k] = c;
                    }
                    if (m < l) {
                        const float2 mj = G[m + l * j];
                        float2 mk = G[m + l * k];
                        mk.x -= fmaf(hr, mj.x, -hi * mj.y);
                        mk.y -= fmaf(hr, mj.y, hi * mj.x);
                        G[m + l * k] = mk;
                    }
                }
            }
        }
        __syncthreads();
    }
    return true;
}

// The Cholesky inverse above: rows of a column in one lane of warp 0 and of each half-warp
// (WIDE = false, l <= 32), or in several (WIDE = true, l <= kLMax).
template <bool WIDE>
__device__ __forceinline__ bool chol_inv(float2* G, float2* C, int l, float shift, float drop_tol,
                                         int* s_flag) {
    if constexpr (WIDE) return chol_inv_wide(G, C, l, shift, drop_tol, s_flag);
    else return chol_inv_narrow(G, C, l, shift, drop_tol, s_flag);
}

// Yout (n x l) = Yin C for an upper triangular C (l x l); items of one row and 4 columns.
__device__ void mult_upper(const float2* Yin, const float2* C, float2* Yout, int n, int l) {
    const int nq = (l + 3) >> 2;
    for (int t = threadIdx.x; t < n * nq; t += kTS) {
        const int e = t % n, k0 = (t / n) * 4;
        const int kn = min(4, l - k0);
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int m = 0; m < k0 + kn; ++m) {
            const float2 y = Yin[e + (size_t)n * m];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q < kn) {
                    const float2 c = C[m + l * (k0 + q)];  // zero below the diagonal
                    acc[q].x = fmaf(y.x, c.x, fmaf(-y.y, c.y, acc[q].x));
                    acc[q].y = fmaf(y.x, c.y, fmaf(y.y, c.x, acc[q].y));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < kn) Yout[e + (size_t)n * (k0 + q)] = acc[q];
    }
    __syncthreads();
}

// Shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa): the l columns of
// Y (n x l, ld n) are orthonormalised by three passes of Y <- Y R^-1 with R^H R the Cholesky
// factorisation of the Gram matrix, the first pass shifted by 11 (n l + l (l + 1)) u ||Y||_F^2
// (u = 2^-24) so that it cannot break down.  The passes alternate between Y and the scratch
// S (both n x l); returns the buffer that holds the result, or nullptr if a norm was not a
// number (the slice then goes to the Jacobi path).
// When Y has fewer than l numerically independent columns (a sketch wider than the slice's
// rank, whose remaining singular values sit below FP32 resolution relative to the largest),
// a plain pass finds columns that lie in the span of the earlier ones to within
// 8 n u of their norm (the rounding of an n-term Gram entry) and drops them: the result
// has orthonormal columns and zero columns, and the zero columns stay zero through the
// power iterations and come out as singular values 0 (not kept).  Check (c) still rejects
// the sketch if a dropped direction carried a singular value above tau.
template <bool WIDE>
__device__ float2* orth3(float2* Y, float2* S, int n, int l, float2* G, float2* C, int* s_flag,
                         int passes = 3) {
    float2* cur = Y;
    float2* oth = S;
    for (int pass = 0; pass < passes; ++pass) {
        gram(cur, n, l, G);
        float shift = 0.f;
        if (pass == 0) {
            float tr = 0.f;
            for (int j = 0; j < l; ++j) tr += G[j + l * j].x;
            shift = 11.f * (float)(n * l + l * (l + 1)) * 5.9604645e-08f * tr;
        }
        if (!chol_inv<WIDE>(G, C, l, shift, 8.f * (float)n * 5.9604645e-08f, s_flag))
            return nullptr;
        mult_upper(cur, C, oth, n, l);
        float2* t = cur;
        cur = oth;
        oth = t;
    }
    return cur;
}

// Eigen-decomposition G = V diag(lambda) V^H of the l x l (l <= 32) Hermitian G by the whole
// CTA: parallel two-sided Jacobi over the round-robin tournament.  Each round first forms the
// rotations of its P pairs (one thread per pair), then applies all of them at once: every
// 2 x 2 block of G (rows of pair i, columns of pair j) becomes J_i^H G_ij J_j and V <- V J.
// Rows and columns of different pairs are disjoint, so the blocks are independent.  G ends
// diagonal up to the tolerance.  `rot` (4 kLMax floats) and `pq` (kLMax ints) are scratch.
// Returns false without convergence in 30 sweeps.
__device__ bool eigh_cta(float2* G, float2* V, int l, float4* rot, int2* pq) {
    const int tid = threadIdx.x;
    for (int t = tid; t < l * l; t += kTS) V[t] = make_float2((t % l) == (t / l) ? 1.f : 0.f, 0.f);
    __syncthreads();
    if (l < 2) return true;
    const int Np = l + (l & 1), P = Np / 2;
    const float tol = 8.f * 1.1920928955078125e-07f, tol2 = tol * tol;
    for (int sweep = 0; sweep < 30; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < Np - 1; ++r) {
            if (tid < P) {
                int a, b;
                if (tid == 0) { a = Np - 1; b = r; }
                else { a = (r + tid) % (Np - 1); b = (r - tid + Np - 1) % (Np - 1); }
                const int p = min(a, b), q = max(a, b);  // q == l only for the odd-l dummy
                float c = 1.f, sr = 0.f, si = 0.f, f = 0.f;
                if (q < l) {
                    const float al = G[p + l * p].x, be = G[q + l * q].x;
                    const float2 g = G[p + l * q];
                    const float ag2 = fmaf(g.x, g.x, g.y * g.y);
                    if (ag2 > (tol2 * fabsf(al)) * fabsf(be) && ag2 > 0.f) {
                        jacobi_rotation(al, be, g.x, g.y, ag2, c, sr, si);
                        f = 1.f;
                        rotated = 1;
                    }
                }
                rot[tid] = make_float4(c, sr, si, f);
                pq[tid] = make_int2(p, q < l ? q : -1);
            }
            __syncthreads();
            for (int t = tid; t < P * P + l * P; t += kTS) {
                if (t < P * P) {
                    const int i = t % P, j = t / P;
                    const float4 ri = rot[i], rj = rot[j];
                    if (ri.w == 0.f && rj.w == 0.f) continue;
                    const int2 a = pq[i], b = pq[j];
                    // block [[x0, x1], [y0, y1]]: rows (a.x, a.y), columns (b.x, b.y)
                    const float2 z = make_float2(0.f, 0.f);
                    float2 x0 = G[a.x + l * b.x];
                    float2 x1 = b.y >= 0 ? G[a.x + l * b.y] : z;
                    float2 y0 = a.y >= 0 ? G[a.y + l * b.x] : z;
                    float2 y1 = (a.y >= 0 && b.y >= 0) ? G[a.y + l * b.y] : z;
                    // rows: g_p <- c g_p - w g_q, g_q <- conj(w) g_p + c g_q   (w = sr + i si)
                    const float c = ri.x, sr = ri.y, si = ri.z;
                    float2 n0 = make_float2(fmaf(c, x0.x, -fmaf(sr, y0.x, -si * y0.y)),
                                            fmaf(c, x0.y, -fmaf(sr, y0.y, si * y0.x)));
                    float2 m0 = make_float2(fmaf(sr, x0.x, fmaf(si, x0.y, c * y0.x)),
                                            fmaf(sr, x0.y, fmaf(-si, x0.x, c * y0.y)));
                    float2 n1 = make_float2(fmaf(c, x1.x, -fmaf(sr, y1.x, -si * y1.y)),
                                            fmaf(c, x1.y, -fmaf(sr, y1.y, si * y1.x)));
                    float2 m1 = make_float2(fmaf(sr, x1.x, fmaf(si, x1.y, c * y1.x)),
                                            fmaf(sr, x1.y, fmaf(-si, x1.x, c * y1.y)));
                    // columns: g_p <- c g_p - conj(w) g_q, g_q <- w g_p + c g_q
                    const float d = rj.x, tr = rj.y, ti = rj.z;
                    x0 = make_float2(fmaf(d, n0.x, fmaf(-tr, n1.x, -ti * n1.y)),
                                     fmaf(d, n0.y, fmaf(-tr, n1.y, ti * n1.x)));
                    x1 = make_float2(fmaf(tr, n0.x, fmaf(-ti, n0.y, d * n1.x)),
                                     fmaf(tr, n0.y, fmaf(ti, n0.x, d * n1.y)));
                    y0 = make_float2(fmaf(d, m0.x, fmaf(-tr, m1.x, -ti * m1.y)),
                                     fmaf(d, m0.y, fmaf(-tr, m1.y, ti * m1.x)));
                    y1 = make_float2(fmaf(tr, m0.x, fmaf(-ti, m0.y, d * m1.x)),
                                     fmaf(tr, m0.y, fmaf(ti, m0.x, d * m1.y)));
                    G[a.x + l * b.x] = x0;
                    if (b.y >= 0) G[a.x + l * b.y] = x1;
                    if (a.y >= 0) G[a.y + l * b.x] = y0;
                    if (a.y >= 0 && b.y >= 0) G[a.y + l * b.y] = y1;
                } else {
                    const int u = t - P * P, k = u % l, j = u / l;
                    const float4 rj = rot[j];
                    if (rj.w == 0.f) continue;
                    const int2 b = pq[j];
                    const float d = rj.x, tr = rj.y, ti = rj.z;
                    const float2 x = V[k + l * b.x], y = V[k + l * b.y];
                    V[k + l * b.x] = make_float2(fmaf(d, x.x, fmaf(-tr, y.x, -ti * y.y)),
                                                 fmaf(d, x.y, fmaf(-tr, y.y, ti * y.x)));
                    V[k + l * b.y] = make_float2(fmaf(tr, x.x, fmaf(-ti, x.y, d * y.x)),
                                                 fmaf(tr, x.y, fmaf(ti, x.x, d * y.y)));
                }
            }
            __syncthreads();
        }
        if (!__syncthreads_or(rotated)) return true;
    }
    return false;
}

// y (n1) = A x (x: n2, shared); partial sums over column ranges meet through shared atomics.
__device__ void matvec_a(const float2* __restrict__ A, int n1, int n2, bool real, const float2* x,
                         float2* y) {
    const int parts = max(1, min(kTS / n1, 8));
    const int span = (n2 + parts - 1) / parts;
    for (int i = threadIdx.x; i < n1; i += kTS) y[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int t = threadIdx.x; t < n1 * parts; t += kTS) {
        const int i = t % n1, pr = t / n1;
        const int c0 = pr * span, c1 = min(n2, c0 + span);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const float2 a = ld_a(A, i + (int64_t)n1 * c, real), v = x[c];
            acc.x = fmaf(a.x, v.x, fmaf(-a.y, v.y, acc.x));
            acc.y = fmaf(a.x, v.y, fmaf(a.y, v.x, acc.y));
        }
        if (parts == 1) {
            y[i] = acc;
        } else {
            atomicAdd(&y[i].x, acc.x);
            atomicAdd(&y[i].y, acc.y);
        }
    }
    __syncthreads();
}

// x (n2) = A^H y (y: n1, shared); one warp per column of A (coalesced), lanes over its rows.
__device__ void matvec_ah(const float2* __restrict__ A, int n1, int n2, bool real, const float2* y,
                          float2* x) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < n2; c += kTS / 32) {
        float dr = 0.f, di = 0.f;
        for (int i = lane; i < n1; i += 32) {
            const float2 a = ld_a(A, i + (int64_t)n1 * c, real), v = y[i];
            dr = fmaf(a.x, v.x, fmaf(a.y, v.y, dr));  // conj(a) v
            di = fmaf(a.x, v.y, fmaf(-a.y, v.x, di));
        }
        dr = warp_sum(dr);
        di = warp_sum(di);
        if (lane == 0) x[c] = make_float2(dr, di);
    }
    __syncthreads();
}

// D = Z V over Z (n2 x l, l > 32) by rows: a warp per row, lanes over columns lane and lane + 32.
__device__ __forceinline__ void zv_wide(float2* bz, const float2* V, int n2, int l) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = warp; e < n2; e += kTS / 32) {
        float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = lane + 32 * h;
            if (col < l) {
                for (int m = 0; m < l; ++m) {
                    const float2 z = bz[e + (size_t)n2 * m], v = V[m + (size_t)l * col];
                    acc[h].x = fmaf(z.x, v.x, fmaf(-z.y, v.y, acc[h].x));
                    acc[h].y = fmaf(z.x, v.y, fmaf(z.y, v.x, acc[h].y));
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < l) bz[e + (size_t)n2 * (lane + 32 * h)] = acc[h];
    }
}

// Shared state of one CTA of the sketch kernel besides the dynamic buffers.
struct SketchShared {
    int flag, item;
    int keep[kLMax];  // sigma_j > tau, decided in FP64
    float worst[kTS / 32];
    float4 rot[kLMax / 2];
    int2 pq[kLMax / 2];
};

// The whole sketch SVT of one slice (steps 2-5 of the file comment) by the calling CTA.
// RETRY: the slice comes from a retry list and takes its extra power iterations from
// P.extra_power (a first attempt uses P.power_iters alone, a block-uniform loop bound).
template <bool RETRY, bool WIDE>
__device__ void sketch_one(const SvdJob* __restrict__ jobs, int job, const SketchParams& P,
                           float4* smem4, SketchShared& sh) {
    int& s_flag = sh.flag;
    float* s_worst = sh.worst;
    float4* s_rot = sh.rot;
    int2* s_pq = sh.pq;
    const SvdJob J = jobs[job];
    const int n1 = J.n1, n2 = J.n2, nm = max(n1, n2);
    const bool real = J.real_slice != 0;
    const int l = P.ell[job];
    // power iterations: a first attempt reads the launch parameter wherever it needs it
    const int q_retry = RETRY ? P.power_iters + P.extra_power[job] : 0;
#define TP_SKETCH_Q (RETRY ? q_retry : P.power_iters)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tall buffers in the global scratch when the launch has one: always in the global class
    // (its shared memory holds only the small arrays), and in a retry round only for the
    // slices that do not fit the round's shared memory (the others keep the faster
    // shared-memory buffers)
    const bool global_bufs = WIDE && P.gscratch != nullptr &&
                             (!RETRY || sketch_smem_need(n1, n2, l) > (size_t)P.smem_bytes);
    if (l <= 0 || l >= min(n1, n2) || l > (WIDE ? kLMax : kNarrowL) ||
        (global_bufs ? (sketch_small_need(n1, n2, l) > (size_t)P.smem_bytes ||
                        (int64_t)3 * nm * l > P.gstride)
                     : sketch_smem_need(n1, n2, l) > (size_t)P.smem_bytes)) {
        if (tid == 0) P.flag[job] = 1;
        return;
    }
    // three max(n1, n2) x l buffers: in shared memory, or in this CTA's global scratch
    float2* B0 = global_bufs ? P.gscratch + (int64_t)blockIdx.x * P.gstride
                             : reinterpret_cast<float2*>(smem4);
    float2* B1 = B0 + (size_t)nm * l;
    float2* B2 = B1 + (size_t)nm * l;
    float2* V = global_bufs ? reinterpret_cast<float2*>(smem4) : B2 + (size_t)nm * l;  // l x l
    float2* G = V + (size_t)l * l;                  // l x l
    float2* C = G + (size_t)l * l;                  // l x l
    float2* xv = C + (size_t)l * l;                 // n2
    float2* yv = xv + n2;                           // n1
    float2* coef = yv + n1;                         // 2 kLMax
    float* sig = reinterpret_cast<float*>(coef + 2 * kLMax);
    float* fac = sig + kLMax;
    const float2* A = J.A;

    // 2. range finder with power iterations; shifted CholeskyQR orthonormalisations of two
    // passes (shifted, then plain: after the shifted pass the basis is well conditioned, so one
    // plain pass leaves it orthonormal to working accuracy, which check (b) confirms).  bq holds
    // the current Q (n1 x l), bz the current Z (n2 x l), bs is scratch.
    float2* bq = B0;
    float2* bz = B1;
    float2* bs = B2;
    // Omega (n2 x l): one hash per row and group of 16 columns, two bits per entry
    for (int t = tid; t < n2 * ((l + 15) >> 4); t += kTS) {
        const int rr = t % n2, c0 = (t / n2) * 16;
        const uint32_t h = mix32(P.seed ^ mix32((uint32_t)job * 0x9e3779b9u ^
                                                mix32((uint32_t)rr * 0x632be5abu + (uint32_t)c0)));
        for (int c = c0; c < min(l, c0 + 16); ++c) {
            const uint32_t b = h >> (2 * (c - c0));
            const float a = (b & 1u) ? 1.f : -1.f, bb = (b & 2u) ? 1.f : -1.f;
            bs[rr + (size_t)n2 * c] = real ? make_float2(a, 0.f)
                                           : make_float2(a * 0.70710678f, bb * 0.70710678f);
        }
    }
    __syncthreads();
    mult_a(A, n1, n2, real, bs, bq, l);
    __syncthreads();
    float2* r = orth3<WIDE>(bq, bs, n1, l, G, C, &s_flag, TP_SKETCH_Q > 0 ? 2 : 3);
    bool ok = r != nullptr;
    if (ok && r != bq) { bs = bq; bq = r; }
    for (int it = 0; ok && it < TP_SKETCH_Q; ++it) {
        mult_ah(A, n1, n2, real, bq, bz, l);
        r = orth3<WIDE>(bz, bs, n2, l, G, C, &s_flag, 2);
        ok = r != nullptr;
        if (!ok) break;
        if (r != bz) { bs = bz; bz = r; }
        mult_a(A, n1, n2, real, bz, bq, l);
        __syncthreads();
        r = orth3<WIDE>(bq, bs, n1, l, G, C, &s_flag, 2);
        ok = r != nullptr;
        if (ok && r != bq) { bs = bq; bq = r; }
    }
    // 3. Z = A^H Q = B^H; one-sided Jacobi Z V = D with orthogonal columns, sigma_j = ||d_j||,
    // so A ~ Q Z^H = (Q V) diag(sigma) (D / sigma)^H
    if (ok) {
        mult_ah(A, n1, n2, real, bq, bz, l);
        gram(bz, n2, l, G);
        ok = eigh_cta(G, V, l, s_rot, s_pq);
    }
    if (ok && !WIDE) {  // D = Z V over Z, by rows (a warp per row, lanes over columns)
        for (int e = warp; e < n2; e += kTS / 32) {
            float2 acc = make_float2(0.f, 0.f);
            if (lane < l) {
                for (int m = 0; m < l; ++m) {
                    const float2 z = bz[e + (size_t)n2 * m], v = V[m + (size_t)l * lane];
                    acc.x = fmaf(z.x, v.x, fmaf(-z.y, v.y, acc.x));
                    acc.y = fmaf(z.x, v.y, fmaf(z.y, v.x, acc.y));
                }
            }
            __syncwarp();
            if (lane < l) bz[e + (size_t)n2 * lane] = acc;
        }
        __syncthreads();
    } else if (ok) {  // the same with up to kLMax columns
        zv_wide(bz, V, n2, l);
        __syncthreads();
    }
    float smax = 0.f;
    int k = 0;

    float2* U = bs;  // n1 x l
    float2* R = bz;  // n2 x l: D, then D / sigma on the kept columns
    float2* T = bq;  // n1 x l: A R for the residuals (Q is dead once U is formed)
    if (ok) {
        // sigma_j = ||d_j||; the kept set {sigma_j > tau} in FP64, a sigma within 1e-6 relative of
        // tau first recomputed as ||d_j|| accumulated in FP64
        for (int j = warp; j < l; j += kTS / 32) {
            float sacc = 0.f;
            for (int e = lane; e < n2; e += 32) {
                const float2 d = R[e + (size_t)n2 * j];
                sacc = fmaf(d.x, d.x, fmaf(d.y, d.y, sacc));
            }
            sacc = warp_sum(sacc);
            const float sj = sqrtf(sacc);
            double sd = sj;
            if (fabs(sd - J.tau) <= 1e-6 * J.tau) {
                double s2 = 0.0;
                for (int e = lane; e < n2; e += 32) {
                    const float2 d = R[e + (size_t)n2 * j];
                    s2 = fma((double)d.x, (double)d.x, fma((double)d.y, (double)d.y, s2));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                sd = sqrt(s2);
            }
            if (lane == 0) {
                sig[j] = sj;
                sh.keep[j] = sd > J.tau ? 1 : 0;
            }
        }
        // U = Q V
        for (int t = tid; t < n1 * l; t += kTS) {
            const int i = t % n1, j = t / n1;
            float2 acc = make_float2(0.f, 0.f);
            for (int m = 0; m < l; ++m) {
                const float2 q = bq[i + (size_t)n1 * m], v = V[m + (size_t)l * j];
                acc.x = fmaf(q.x, v.x, fmaf(-q.y, v.y, acc.x));
                acc.y = fmaf(q.x, v.y, fmaf(q.y, v.x, acc.y));
            }
            U[t] = acc;
        }
        __syncthreads();
        // 4(a): the sketch must reach below tau (some computed sigma is not kept)
        for (int j = 0; j < l; ++j) {
            smax = fmaxf(smax, sig[j]);
            k += sh.keep[j];
        }
        ok = k < l;
        if (!ok) {  // the rank was underestimated
            if (tid == 0) P.flag[job] = 3;
            return;
        }
    }
    if (ok) {
        for (int j = tid; j < l; j += kTS) fac[j] = sh.keep[j] ? 1.f / sig[j] : 0.f;
        __syncthreads();
        for (int t = tid; t < n2 * l; t += kTS) {
            const float f = fac[t / n2];
            R[t].x *= f;
            R[t].y *= f;
        }
        __syncthreads();
        // 4(b): residuals of the kept triplets, T = A R in one pass
        mult_a(A, n1, n2, real, R, T, l);
        __syncthreads();
        float worst = 0.f;
        for (int j = warp; j < l; j += kTS / 32) {
            if (!sh.keep[j]) continue;
            float sacc = 0.f;
            for (int e = lane; e < n1; e += 32) {
                const float2 a = T[e + (size_t)n1 * j], u = U[e + (size_t)n1 * j];
                const float dx = a.x - sig[j] * u.x, dy = a.y - sig[j] * u.y;
                sacc = fmaf(dx, dx, fmaf(dy, dy, sacc));
            }
            sacc = warp_sum(sacc);
            worst = fmaxf(worst, sqrtf(sacc) * (float)(((double)sig[j] - J.tau) / sig[j]));
        }
        if (lane == 0) s_worst[warp] = worst;
        __syncthreads();
        worst = 0.f;
        for (int w = 0; w < kTS / 32; ++w) worst = fmaxf(worst, s_worst[w]);
        // the FP32 rounding of the residual product grows like sqrt(max(n1, n2)) u, so the
        // tolerance grows with it past 100 rows
        ok = worst <= P.resid_tol * fmaxf(1.f, sqrtf((float)nm * 0.01f)) * smax;
    }
    if (ok) {
        // 4(c): norm of A - U_k S_k R_k^H by two power iterations from a random start
        for (int c = tid; c < n2; c += kTS) xv[c] = omega(P.seed ^ 0x5bd1e995u, job, c, 0, real);
        __syncthreads();
        float est = 0.f;
        for (int it = 0; it < 2; ++it) {
            // normalise x (every warp reduces the same shared vector)
            float nx = 0.f;
            for (int c = lane; c < n2; c += 32) nx = fmaf(xv[c].x, xv[c].x, fmaf(xv[c].y, xv[c].y, nx));
            nx = warp_sum(nx);
            const float inx = nx > 0.f ? rsqrtf(nx) : 0.f;
            __syncthreads();
            for (int c = tid; c < n2; c += kTS) { xv[c].x *= inx; xv[c].y *= inx; }
            __syncthreads();
            // coef_j = sigma_j (r_j^H x)   (r_j = 0 for the columns that are not kept)
            for (int j = warp; j < l; j += kTS / 32) {
                float dr = 0.f, di = 0.f;
                for (int c = lane; c < n2; c += 32) {
                    const float2 rr = R[c + (size_t)n2 * j], x = xv[c];
                    dr = fmaf(rr.x, x.x, fmaf(rr.y, x.y, dr));
                    di = fmaf(rr.x, x.y, fmaf(-rr.y, x.x, di));
                }
                dr = warp_sum(dr);
                di = warp_sum(di);
                if (lane == 0) coef[j] = make_float2(sig[j] * dr, sig[j] * di);
            }
            // y = A x - U coef
            matvec_a(A, n1, n2, real, xv, yv);
            for (int i = tid; i < n1; i += kTS) {
                float2 acc = yv[i];
                for (int j = 0; j < l; ++j) {
                    const float2 u = U[i + (size_t)n1 * j], d = coef[j];
                    acc.x -= fmaf(u.x, d.x, -u.y * d.y);
                    acc.y -= fmaf(u.x, d.y, u.y * d.x);
                }
                yv[i] = acc;
            }
            __syncthreads();
            // coef_j = sigma_j (u_j^H y) for the kept columns
            for (int j = warp; j < l; j += kTS / 32) {
                float dr = 0.f, di = 0.f;
                for (int i = lane; i < n1; i += 32) {
                    const float2 u = U[i + (size_t)n1 * j], y = yv[i];
                    dr = fmaf(u.x, y.x, fmaf(u.y, y.y, dr));
                    di = fmaf(u.x, y.y, fmaf(-u.y, y.x, di));
                }
                dr = warp_sum(dr);
                di = warp_sum(di);
                const float w = fac[j] > 0.f ? sig[j] : 0.f;
                if (lane == 0) coef[j + kLMax] = make_float2(w * dr, w * di);
            }
            // x = A^H y - R coef
            matvec_ah(A, n1, n2, real, yv, xv);
            for (int c = tid; c < n2; c += kTS) {
                float2 acc = xv[c];
                for (int j = 0; j < l; ++j) {
                    const float2 rr = R[c + (size_t)n2 * j], d = coef[j + kLMax];
                    acc.x -= fmaf(rr.x, d.x, -rr.y * d.y);
                    acc.y -= fmaf(rr.x, d.y, rr.y * d.x);
                }
                xv[c] = acc;
            }
            __syncthreads();
            float nx2 = 0.f;
            for (int c = lane; c < n2; c += 32) nx2 = fmaf(xv[c].x, xv[c].x, fmaf(xv[c].y, xv[c].y, nx2));
            nx2 = warp_sum(nx2);
            est = sqrtf(sqrtf(nx2));  // ||E^H E x||^(1/2) with ||x|| = 1
        }
        ok = (double)est < 0.8 * J.tau;
    }
    if (!ok) {
        if (tid == 0) P.flag[job] = 1;
        return;
#undef TP_SKETCH_Q
    }
    // 5. W = sum_{sigma_j > tau} (sigma_j - tau) u_j r_j^H over A
    for (int j = tid; j < l; j += kTS)
        fac[j] = sh.keep[j] ? (float)((double)sig[j] - J.tau) : 0.f;
    __syncthreads();
    // scale the kept columns of U by sigma - tau (the others by 0) once
    for (int t = tid; t < n1 * l; t += kTS) {
        const float f = fac[t / n1];
        U[t].x *= f;
        U[t].y *= f;
    }
    __syncthreads();
    // 2 x 2 output tiles: rows (i, i + 1), columns (c, c + 1)
    const int h1 = (n1 + 1) >> 1, h2 = (n2 + 1) >> 1;
    for (int t = tid; t < h1 * h2; t += kTS) {
        const int i = 2 * (t % h1), c = 2 * (t / h1);
        const bool i1 = i + 1 < n1, c1 = c + 1 < n2;
        float2 a00 = make_float2(0.f, 0.f), a10 = a00, a01 = a00, a11 = a00;
        for (int j = 0; j < l; ++j) {
            if (fac[j] == 0.f) continue;
            const float2 u0 = U[i + (size_t)n1 * j], u1 = i1 ? U[i + 1 + (size_t)n1 * j] : u0;
            const float2 r0 = R[c + (size_t)n2 * j], r1 = c1 ? R[c + 1 + (size_t)n2 * j] : r0;
            // u conj(r)
            a00.x = fmaf(u0.x, r0.x, fmaf(u0.y, r0.y, a00.x));
            a00.y = fmaf(u0.y, r0.x, fmaf(-u0.x, r0.y, a00.y));
            a10.x = fmaf(u1.x, r0.x, fmaf(u1.y, r0.y, a10.x));
            a10.y = fmaf(u1.y, r0.x, fmaf(-u1.x, r0.y, a10.y));
            a01.x = fmaf(u0.x, r1.x, fmaf(u0.y, r1.y, a01.x));
            a01.y = fmaf(u0.y, r1.x, fmaf(-u0.x, r1.y, a01.y));
            a11.x = fmaf(u1.x, r1.x, fmaf(u1.y, r1.y, a11.x));
            a11.y = fmaf(u1.y, r1.x, fmaf(-u1.x, r1.y, a11.y));
        }
        if (real) a00.y = a10.y = a01.y = a11.y = 0.f;
        float2* w0 = J.W + i + (size_t)n1 * c;
        w0[0] = a00;
        if (i1) w0[1] = a10;
        if (c1) {
            w0[n1] = a01;
            if (i1) w0[n1 + 1] = a11;
        }
    }
    if (tid == 0) {
        P.flag[job] = 0;
        if (P.count) P.count[job] = k;
    }
}

// One slice per CTA (P.queue_next == nullptr, CTA b takes P.order[b]), or a persistent grid
// that takes slices P.order[i] from a work counter until the queue of *P.queue_len is empty;
// the queue is ordered largest slice first, so the tail is made of small slices.
// WIDE: widths up to kLMax (the global-scratch class and the retry rounds); otherwise up to
// kNarrowL, with the leaner code of one lane per column.
template <bool RETRY, bool WIDE>
__global__ void __launch_bounds__(kTS, 4) sketch_svt_kernel(const SvdJob* __restrict__ jobs,
                                                           SketchParams P) {
    extern __shared__ float4 smem4[];
    __shared__ SketchShared sh;
    if (!P.queue_next) {
        sketch_one<RETRY, WIDE>(jobs, P.order ? P.order[blockIdx.x] : (int)blockIdx.x, P, smem4, sh);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(P.queue_next, 1);
        __syncthreads();
        const int item = sh.item;
        if (item >= *P.queue_len) break;
        const int job = P.order[item];
        if (job >= 0 && job < P.njobs) {
            // a retry round holds slices of every width: those within the narrow limit whose
            // buffers fit the round's shared memory take the leaner narrow code (block-uniform:
            // every thread reads the same slice)
            if constexpr (RETRY && WIDE) {
                const int l = P.ell[job];
                if (l <= kNarrowL &&
                    sketch_smem_need(jobs[job].n1, jobs[job].n2, l) <= (size_t)P.smem_bytes)
                    sketch_one<RETRY, false>(jobs, job, P, smem4, sh);
                else
                    sketch_one<RETRY, WIDE>(jobs, job, P, smem4, sh);
            } else {
                sketch_one<RETRY, WIDE>(jobs, job, P, smem4, sh);
            }
        }
        __syncthreads();  // the CTA is done with this slice's shared state
    }
}

// Sorts the slices into the sketch kernel's queues: class c holds the slices whose shared
// memory need at their proposed width is at most caps[c] (and above caps[c - 1]), in the
// order of `sorted` (largest first).  Slices without a usable width, or too large for every
// class, are flagged for the Jacobi path here.  One CTA of 1024 threads; stable compaction by
// warp ballots and per-class running offsets.  queues: ncls lists of n entries; counts: per
// class (length, work counter).
__global__ void __launch_bounds__(1024) sketch_bin_kernel(const SvdJob* __restrict__ jobs,
                                                          const int32_t* __restrict__ sorted,
                                                          int n, const int32_t* __restrict__ ell,
                                                          int32_t* __restrict__ flag,
                                                          SketchCaps caps, int32_t* queues,
                                                          int32_t* counts) {
    __shared__ int wsum[32][kSketchClasses];
    __shared__ int base[kSketchClasses];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncls = caps.n;
    if (tid < ncls) base[tid] = 0;
    __syncthreads();
    for (int chunk = 0; chunk < n; chunk += 1024) {
        const int idx = chunk + tid;
        int c = -1, job = -1;
        if (idx < n) {
            job = sorted[idx];
            const SvdJob& J = jobs[job];
            const int l = ell[job];
            if (l > 0 && l < min(J.n1, J.n2) && l <= kLMax) {
                const size_t need = sketch_smem_need(J.n1, J.n2, l);
                if (l > kNarrowL) {
                    c = ncls - 1;  // the wide kernel runs only in the last class
                } else {
                    for (int q = 0; q < ncls; ++q)
                        if (need <= caps.bytes[q]) { c = q; break; }
                }
            }
            if (c < 0) flag[job] = 1;
        }
        int mypos = 0;
        for (int q = 0; q < ncls; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, c == q);
            if (c == q) mypos = __popc(m & ((1u << lane) - 1u));
            if (lane == 0) wsum[warp][q] = __popc(m);
        }
        __syncthreads();
        if (tid < ncls) {
            int run = base[tid];
            for (int w = 0; w < 32; ++w) {
                const int t = wsum[w][tid];
                wsum[w][tid] = run;
                run += t;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (c >= 0) queues[(size_t)c * n + wsum[warp][c] + mypos] = job;
        __syncthreads();
    }
    if (tid < ncls) {
        counts[2 * tid] = base[tid];
        counts[2 * tid + 1] = 0;
    }
}

// Features of each slice for the proposer (see the file comment); one CTA per slice.
__global__ void __launch_bounds__(kT) features_kernel(const SvdJob* __restrict__ jobs,
                                                      float* __restrict__ feat, uint32_t seed) {
    extern __shared__ float4 smem4[];
    const int job = blockIdx.x;
    const SvdJob J = jobs[job];
    const int n1 = J.n1, n2 = J.n2, tid = threadIdx.x;
    const bool real = J.real_slice != 0;
    constexpr int S = 8;
    float2* X = reinterpret_cast<float2*>(smem4);  // n2 x S
    float2* Y = X + (size_t)n2 * S;                // n1 x S
    float2* coef = Y + (size_t)n1 * S;
    float* red = reinterpret_cast<float*>(coef + S);
    float* dg = red + 32;
    const float2* A = J.A;
    float fr = 0.f;
    for (int64_t t = tid; t < (int64_t)n1 * n2; t += kT) {
        const float2 a = ld_a(A, t, real);
        fr = fmaf(a.x, a.x, fmaf(a.y, a.y, fr));
    }
    fr = block_sum(fr, red);
    for (int t = tid; t < n2 * S; t += kT) X[t] = omega(seed, job, t % n2, t / n2, real);
    __syncthreads();
    const int l = min(S, n2);
    mult_a(A, n1, n2, real, X, Y, l);
    __syncthreads();
    // modified Gram-Schmidt: |R_jj| = norm of column j after removing the previous ones
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = 0; j < l; ++j) {
        float2* y = Y + n1 * j;
        for (int i = warp; i < j; i += kT / 32) {
            const float2* q = Y + n1 * i;
            float dr = 0.f, di = 0.f;
            for (int e = lane; e < n1; e += 32) {
                dr = fmaf(q[e].x, y[e].x, fmaf(q[e].y, y[e].y, dr));
                di = fmaf(q[e].x, y[e].y, fmaf(-q[e].y, y[e].x, di));
            }
            dr = warp_sum(dr);
            di = warp_sum(di);
            if (lane == 0) coef[i] = make_float2(dr, di);
        }
        __syncthreads();
        for (int e = tid; e < n1; e += kT) {
            float2 v = y[e];
            for (int i = 0; i < j; ++i) {
                const float2 q = Y[e + n1 * i], d = coef[i];
                v.x -= fmaf(d.x, q.x, -d.y * q.y);
                v.y -= fmaf(d.x, q.y, d.y * q.x);
            }
            y[e] = v;
        }
        __syncthreads();
        float nn = 0.f;
        for (int e = tid; e < n1; e += kT) nn = fmaf(y[e].x, y[e].x, fmaf(y[e].y, y[e].y, nn));
        nn = block_sum(nn, red);
        const float rjj = sqrtf(nn);
        if (tid == 0) dg[j] = rjj;
        const float inv = rjj > 0.f ? 1.f / rjj : 0.f;
        for (int e = tid; e < n1; e += kT) { y[e].x *= inv; y[e].y *= inv; }
        __syncthreads();
    }
    if (tid == 0) {
        const float itau = J.tau > 0.0 ? (float)(1.0 / J.tau) : 1e30f;
        float d[S];
        for (int j = 0; j < S; ++j) d[j] = j < l ? dg[j] : 0.f;
        for (int a = 0; a < S; ++a)  // sort decreasing
            for (int b = a + 1; b < S; ++b)
                if (d[b] > d[a]) { const float t = d[a]; d[a] = d[b]; d[b] = t; }
        float* f = feat + (size_t)job * kD;
        f[0] = logf(sqrtf(fr) * itau + 1e-6f);
        for (int j = 0; j < S; ++j) f[1 + j] = logf(d[j] * itau + 1e-6f);
        f[9] = logf((float)n1);
        f[10] = logf((float)n2);
        f[11] = logf((float)min(n1, n2));
    }
}

// Proposer inference: one thread per slice, ell = clamp(ceil(k_hat) + 4).  The CTA stages the
// parameters in shared memory (every thread reads the same weight at the same time, a
// broadcast); the first hidden layer stays in registers.
constexpr int kInferT = 64;
__global__ void __launch_bounds__(kInferT) mlp_infer_kernel(const float* __restrict__ feat,
                                                            const SvdJob* __restrict__ jobs, int n,
                                                            int32_t* __restrict__ ell) {
    __shared__ float w[kProposerFloats];
    for (int t = threadIdx.x; t < kProposerFloats; t += kInferT) w[t] = g_proposer[t];
    __syncthreads();
    const int s = blockIdx.x * kInferT + threadIdx.x;
    if (s >= n) return;
    float x[kD];
#pragma unroll
    for (int d = 0; d < kD; ++d) x[d] = (feat[(size_t)s * kD + d] - w[kMean + d]) / w[kStd + d];
    float h1[kH];
#pragma unroll
    for (int a = 0; a < kH; ++a) {
        float v = w[kB1 + a];
#pragma unroll
        for (int d = 0; d < kD; ++d) v = fmaf(w[kW1 + a * kD + d], x[d], v);
        h1[a] = fmaxf(v, 0.f);
    }
    float out = w[kB3];
    for (int a = 0; a < kH; ++a) {
        float v = w[kB2 + a];
#pragma unroll
        for (int b = 0; b < kH; ++b) v = fmaf(w[kW2 + a * kH + b], h1[b], v);
        out = fmaf(w[kW3 + a], fmaxf(v, 0.f), out);
    }
    const int r = min(jobs[s].n1, jobs[s].n2);
    int l = (int)ceilf(fmaxf(out, 0.f)) + 4;
    l = min(l, kLMax);
    ell[s] = (l >= r) ? 0 : l;  // 0: sketching cannot help, full Jacobi
}

// Training: per-sample forward/backward of the squared error, gradients summed in shared
// memory per CTA and then into `grad`; `loss` accumulates the summed squared error.
__global__ void __launch_bounds__(kT) mlp_grad_kernel(const float* __restrict__ X,
                                                      const float* __restrict__ y, int n,
                                                      const float* __restrict__ w,
                                                      float* __restrict__ grad, float* loss) {
    __shared__ float g[kNParams];
    __shared__ float sl;
    for (int t = threadIdx.x; t < kNParams; t += kT) g[t] = 0.f;
    if (threadIdx.x == 0) sl = 0.f;
    __syncthreads();
    const int s = blockIdx.x * kT + threadIdx.x;
    if (s < n) {
        float x[kD];
#pragma unroll
        for (int d = 0; d < kD; ++d) x[d] = X[(size_t)s * kD + d];
        float h1[kH], h2[kH];
        for (int a = 0; a < kH; ++a) {
            float v = w[kB1 + a];
#pragma unroll
            for (int d = 0; d < kD; ++d) v = fmaf(w[kW1 + a * kD + d], x[d], v);
            h1[a] = fmaxf(v, 0.f);
        }
        float out = w[kB3];
        for (int a = 0; a < kH; ++a) {
            float v = w[kB2 + a];
            for (int b = 0; b < kH; ++b) v = fmaf(w[kW2 + a * kH + b], h1[b], v);
            h2[a] = fmaxf(v, 0.f);
            out = fmaf(w[kW3 + a], h2[a], out);
        }
        const float diff = out - y[s];
        atomicAdd(&sl, diff * diff);
        const float dout = 2.f * diff / (float)n;
        atomicAdd(&g[kB3], dout);
        float dh1[kH];
#pragma unroll
        for (int b = 0; b < kH; ++b) dh1[b] = 0.f;
        for (int a = 0; a < kH; ++a) {
            atomicAdd(&g[kW3 + a], dout * h2[a]);
            const float dh2 = h2[a] > 0.f ? dout * w[kW3 + a] : 0.f;
            if (dh2 != 0.f) {
                atomicAdd(&g[kB2 + a], dh2);
                for (int b = 0; b < kH; ++b) {
                    if (h1[b] > 0.f) atomicAdd(&g[kW2 + a * kH + b], dh2 * h1[b]);
                    dh1[b] = fmaf(dh2, w[kW2 + a * kH + b], dh1[b]);
                }
            }
        }
        for (int b = 0; b < kH; ++b) {
            if (h1[b] <= 0.f) continue;
            atomicAdd(&g[kB1 + b], dh1[b]);
#pragma unroll
            for (int d = 0; d < kD; ++d) atomicAdd(&g[kW1 + b * kD + d], dh1[b] * x[d]);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kNParams; t += kT)
        if (g[t] != 0.f) atomicAdd(&grad[t], g[t]);
    if (threadIdx.x == 0) atomicAdd(loss, sl);
}

// Adam update of the proposer parameters; zeroes the gradient for the next step.
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int step, float lr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kNParams) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[t];
    const float mt = b1 * m[t] + (1.f - b1) * g, vt = b2 * v[t] + (1.f - b2) * g * g;
    m[t] = mt;
    v[t] = vt;
    const float mh = mt / (1.f - powf(b1, (float)step)), vh = vt / (1.f - powf(b2, (float)step));
    w[t] -= lr * mh / (sqrtf(vh) + eps);
    grad[t] = 0.f;
}

std::mutex g_prop_mutex;
bool g_prop_ready[128] = {};

}  // namespace

size_t features_smem_bytes(int n1, int n2) {
    return sizeof(float2) * ((size_t)n2 * 8 + (size_t)n1 * 8 + 8) + sizeof(float) * (32 + 8) + 64;
}

cudaError_t launch_features(const SvdJob* jobs, int njobs, int max_n1, int max_n2, float* feat,
                            uint32_t seed, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const size_t smem = features_smem_bytes(max_n1, max_n2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    features_kernel<<<njobs, kT, smem, s>>>(jobs, feat, seed);
    return cudaGetLastError();
}

cudaError_t launch_proposer(const float* feat, const SvdJob* jobs, int njobs, int32_t* ell,
                            cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    mlp_infer_kernel<<<(njobs + kInferT - 1) / kInferT, kInferT, 0, s>>>(feat, jobs, njobs, ell);
    return cudaGetLastError();
}

// Between sketch rounds: every slice that failed (flag 1 or 3) and has min(n1, n2) >=
// min_dim (its Jacobi SVD would cost much more than another sketch) is queued for another
// attempt -- with two more power iterations if its sketch reached below tau (flag 1), or half
// again as wide (at least 4 columns more, at most kLMax) if the rank was underestimated
// (flag 3) -- when the attempt fits the retry launch (shared memory `smem`, and with gstride > 0
// the tall buffers in a global scratch slot of gstride complex values); it is marked 2
// (pending).  Any other failed slice is marked 4 (left to the Jacobi path).
__global__ void __launch_bounds__(1024) sketch_collect_kernel(const SvdJob* __restrict__ jobs,
                                                              int n, int32_t* __restrict__ flag,
                                                              int32_t* __restrict__ ell,
                                                              int32_t* __restrict__ extra,
                                                              int min_dim, int smem, int64_t gstride,
                                                              int32_t* list, int32_t* len) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int f = flag[j];
        if (f != 1 && f != 3) continue;
        const int n1 = jobs[j].n1, n2 = jobs[j].n2, l = ell[j];
        const int64_t nm = max(n1, n2);
        auto fits = [&](int lw) {
            return gstride > 0 ? (sketch_small_need(n1, n2, lw) <= (size_t)smem &&
                                  3 * nm * lw <= gstride)
                               : sketch_smem_need(n1, n2, lw) <= (size_t)smem;
        };
        bool again = min(n1, n2) >= min_dim;
        if (again && f == 1) {
            again = fits(l);
            if (again) extra[j] += 2;
        } else if (again) {
            const int lw = min(min(kLMax, min(n1, n2) - 1), max(l + 4, l + l / 2));
            again = lw > l && fits(lw);
            if (again) ell[j] = lw;
        }
        flag[j] = again ? 2 : 4;
        if (again) list[atomicAdd(len, 1)] = j;
    }
}

cudaError_t launch_sketch_collect(const SvdJob* jobs, int n, int32_t* flag, int32_t* ell,
                                  int32_t* extra, int min_dim, int smem, int64_t gstride,
                                  int32_t* list, int32_t* len, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    sketch_collect_kernel<<<1, 1024, 0, s>>>(jobs, n, flag, ell, extra, min_dim, smem, gstride, list,
                                             len);
    return cudaGetLastError();
}

__global__ void flags01_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = in[j] != 0 ? 1 : 0;
}

cudaError_t launch_flags01(const int32_t* flags, int32_t* out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    flags01_kernel<<<(n + 255) / 256, 256, 0, s>>>(flags, out, n);
    return cudaGetLastError();
}

cudaError_t launch_sketch_bin(const SvdJob* jobs, const int32_t* sorted, int n, const int32_t* ell,
                              int32_t* flag, const SketchCaps& caps, int32_t* queues,
                              int32_t* counts, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    sketch_bin_kernel<<<1, 1024, 0, s>>>(jobs, sorted, n, ell, flag, caps, queues, counts);
    return cudaGetLastError();
}

// Both instantiations have the same resources; the first stands for them.
int sketch_blocks_per_sm(size_t smem) {
    for (const void* fn : {reinterpret_cast<const void*>(sketch_svt_kernel<false, false>),
                           reinterpret_cast<const void*>(sketch_svt_kernel<false, true>),
                           reinterpret_cast<const void*>(sketch_svt_kernel<true, true>)})
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
            return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sketch_svt_kernel<false, true>, kTS, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_sketch_svt(const SvdJob* jobs, int ncta, size_t smem, const SketchParams& p,
                              cudaStream_t s) {
    if (ncta <= 0) return cudaSuccess;
    const void* fn = p.retry_launch ? reinterpret_cast<const void*>(sketch_svt_kernel<true, true>)
                     : p.wide       ? reinterpret_cast<const void*>(sketch_svt_kernel<false, true>)
                                    : reinterpret_cast<const void*>(sketch_svt_kernel<false, false>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (p.retry_launch) sketch_svt_kernel<true, true><<<ncta, kTS, smem, s>>>(jobs, p);
    else if (p.wide) sketch_svt_kernel<false, true><<<ncta, kTS, smem, s>>>(jobs, p);
    else sketch_svt_kernel<false, false><<<ncta, kTS, smem, s>>>(jobs, p);
    return cudaGetLastError();
}

bool proposer_ready() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return false;
    std::lock_guard<std::mutex> lock(g_prop_mutex);
    return g_prop_ready[dev];
}

cudaError_t proposer_set(const float* host) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    e = cudaMemcpyToSymbol(g_proposer, host, sizeof(float) * kProposerFloats);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_prop_mutex);
    g_prop_ready[dev] = true;
    return cudaSuccess;
}

cudaError_t proposer_get(float* host) {
    return cudaMemcpyFromSymbol(host, g_proposer, sizeof(float) * kProposerFloats);
}

// Fit the proposer to (feat, count) pairs resident on the device: standardise the features
// (statistics computed on the host), Xavier-style initialisation from `seed`, `steps` full-
// batch Adam steps of the squared error.  Returns the final mean squared error in *mse.
cudaError_t proposer_fit(const float* d_feat, const int32_t* d_count, int n, int steps, float lr,
                         uint64_t seed, float* scratch, double* mse, cudaStream_t s) {
    if (n <= 0) return cudaErrorInvalidValue;
    std::vector<float> f((size_t)n * kD);
    std::vector<int32_t> c(n);
    cudaError_t e = cudaMemcpyAsync(f.data(), d_feat, sizeof(float) * f.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.data(), d_count, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    std::vector<float> w(kProposerFloats, 0.f);
    for (int d = 0; d < kD; ++d) {
        double m = 0, v = 0;
        for (int i = 0; i < n; ++i) m += f[(size_t)i * kD + d];
        m /= n;
        for (int i = 0; i < n; ++i) {
            const double t = f[(size_t)i * kD + d] - m;
            v += t * t;
        }
        v = sqrt(v / n);
        w[kMean + d] = (float)m;
        w[kStd + d] = (float)(v > 1e-6 ? v : 1.0);
    }
    std::vector<float> xs((size_t)n * kD), ys(n);
    for (int i = 0; i < n; ++i) {
        for (int d = 0; d < kD; ++d)
            xs[(size_t)i * kD + d] = (f[(size_t)i * kD + d] - w[kMean + d]) / w[kStd + d];
        ys[i] = (float)c[i];
    }
    uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto uni = [&]() {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return ((st >> 40) & 0xFFFFFF) / 16777216.0 * 2.0 - 1.0;
    };
    for (int i = 0; i < kH * kD; ++i) w[kW1 + i] = (float)(uni() * sqrt(6.0 / (kD + kH)));
    for (int i = 0; i < kH * kH; ++i) w[kW2 + i] = (float)(uni() * sqrt(6.0 / (2 * kH)));
    for (int i = 0; i < kH; ++i) w[kW3 + i] = (float)(uni() * sqrt(6.0 / (kH + 1)));
    for (int i = 0; i < kH; ++i) w[kB1 + i] = w[kB2 + i] = 0.01f;
    double mean_y = 0;
    for (int i = 0; i < n; ++i) mean_y += ys[i];
    w[kB3] = (float)(mean_y / n);
    // scratch: X (n*kD), y (n), params, grad, m, v, loss
    float* dX = scratch;
    float* dy = dX + (size_t)n * kD;
    float* dw = dy + n;
    float* dg = dw + kProposerFloats;
    float* dm = dg + kProposerFloats;
    float* dv = dm + kProposerFloats;
    float* dl = dv + kProposerFloats;
    e = cudaMemcpyAsync(dX, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, ys.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w.data(), sizeof(float) * kProposerFloats, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dg, 0, sizeof(float) * (3 * kProposerFloats + 1), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const int blocks = (n + kT - 1) / kT;
    for (int it = 1; it <= steps; ++it) {
        if (it == steps) cudaMemsetAsync(dl, 0, sizeof(float), s);
        mlp_grad_kernel<<<blocks, kT, 0, s>>>(dX, dy, n, dw, dg, dl);
        adam_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(dw, dg, dm, dv, it, lr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float hl = 0.f;
    e = cudaMemcpyAsync(w.data(), dw, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, dl, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (mse) *mse = hl / n;
    return proposer_set(w.data());
}

size_t proposer_fit_scratch_floats(int n) { return (size_t)n * (kD + 1) + 4 * kProposerFloats + 1; }

}  // namespace tp
