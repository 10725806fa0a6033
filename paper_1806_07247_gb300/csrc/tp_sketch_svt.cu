// Learned-rank randomized singular value thresholding of the Fourier slices: the fast path
// of prox_tnn (Algorithm 3, step 2; the result is Eq. 21's W = U (S - tau)_+ V^* on every slice
// it accepts) for slices whose number of singular values above tau is small. The full
// one-sided Jacobi SVD (tp_svd.cu) is the fallback and the accuracy reference.
//
// Per slice A (n1 x n2 complex, column-major, in place in the half spectrum) and sketch
// width l (k + 4 for the proposer's k = #{sigma > tau}):
//   1. range finder: Y = A Omega (Omega n2 x l, entries +-1 or (+-1 +- i)/sqrt 2 from a
//      counter-based hash), Q = orth(Y); q power iterations Z = orth(A^H Q), Q = orth(A Z);
//      every orth is a shifted CholeskyQR pass followed by a plain one;
//   2. small SVD: Z = A^H Q (= B^H for B = Q^H A); the l x l Gram G = Z^H Z is diagonalised by
//      two-sided Jacobi, G = V diag V^H, so Z V = D has orthogonal columns, sigma_j = ||d_j||
//      and A ~ Q Z^H = (Q V) diag(sigma) (D / sigma)^H: U = Q V, R = D / sigma;
//   3. acceptance: (a) the smallest computed sigma is below tau (else the rank was
//      underestimated); (b) every kept triplet has ||A r - sigma u|| (sigma - tau) / sigma <=
//      rtol sigma_max; (c) two power iterations on A - U_k S_k R_k^H from a random start
//      estimate its norm below 0.8 tau;
//   4. W = sum_{sigma_j > tau} (sigma_j - tau) u_j r_j^H written over A.
// The kept set {sigma_j > tau} is decided in FP64; a sigma within 1e-6 relative of tau is first
// recomputed as ||d_j|| accumulated in FP64.
//
// Execution: every step above is its own kernel over the list of slices of a round, so each
// launch has thousands of independent slices in flight -- the products with A are passes over
// the spectrum at memory speed, and the latency-bound l x l work (Cholesky inverses, Jacobi
// rounds) of many slices overlaps on every SM.  A slice that fails a check is flagged and later
// stages skip it; the collect kernel queues some failed slices for a retry round (more power
// iterations, or a wider sketch), every other failed slice goes to the Jacobi path.
//
// Per-slice flag values: 0 finished here, 1 failed (Jacobi), 2 in progress, 3 rank
// underestimated, 4 left to Jacobi after a failed retry.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "tp_internal.cuh"
#include "tp_rotation.cuh"
#include "tp_sketch.cuh"

namespace tp {

namespace {

using sk::ld_a;
using sk::warp_sum;

constexpr int kLMax = kSketchMaxL;
constexpr int kPT = 256;               // threads of the product and write kernels
constexpr int kST = 128;               // threads of the per-slice small-matrix kernels
constexpr int kXsBytes = 32 * 1024;    // A X: staged rows of the right-hand matrix X
constexpr int kXsBytesAH = 8 * 1024;   // A^H X: staged rows of X ...
constexpr int kAtBytes = 32 * 1024;    // ... and the transposed tile of A
constexpr int kYsBytes = 12 * 1024;    // Gram: staged rows of the tall matrix
constexpr int kAccCplx = 2048;         // split-K accumulation tile (complex values)
constexpr uint32_t kOmegaSeed = 0x9e3779b9u, kDeflSeed = 0x9e3779b9u ^ 0x5bd1e995u;

enum : int { FLAG_DONE = 0, FLAG_FAIL = 1, FLAG_RUN = 2, FLAG_LOW = 3, FLAG_LEFT = 4 };

struct StageArgs {
    const SketchJob* jobs;
    const int32_t* list;     // slice indices of the round
    const int32_t* len_d;    // device list length (nullptr: len_h)
    int len_h;
    int32_t* ell;            // per slice: sketch width
    int32_t* flag;
    int32_t* count;          // per slice: #{sigma > tau} on success (optional)
    const int32_t* extra;    // per slice: extra power iterations of a retry
    int power_iters;
    int stage;               // power-iteration index of this launch, -1 outside the loop
    float resid_tol;
};

// Work item `item` of the round, or -1 when the slice does not take part in this launch.
// Thread 0 decides and the CTA reads the answer from shared memory (uniform control flow).
__device__ __forceinline__ int stage_slice(const StageArgs& a, int item, int* s_job) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int j = a.list[item];
        if (j >= 0 && a.flag[j] != FLAG_RUN) j = -1;
        if (j >= 0 && a.stage >= 0 && a.stage >= a.power_iters + a.extra[j]) j = -1;
        *s_job = j;
    }
    __syncthreads();
    return *s_job;
}

__device__ __forceinline__ int list_len(const StageArgs& a) {
    return a.len_d ? *a.len_d : a.len_h;
}

// Split of a K loop over S thread groups for `items` outputs of W columns: the fewest rounds
// of kPT threads times K / S, plus a small cost per split level; parts meet in a shared tile of
// kAccCplx complex values.
__device__ __forceinline__ int choose_split(int items, int W, int K) {
    int best = 1;
    float bc = 3.4e38f;
    for (int S = 1; S <= 8; S *= 2) {
        if (S > 1 && items * W > kAccCplx) break;
        const int rounds = (items * S + kPT - 1) / kPT;
        const float cost = (float)rounds * ((float)K / (float)S + 6.f) + (S > 1 ? 10.f : 0.f);
        if (cost < bc) { bc = cost; best = S; }
    }
    return best;
}

// Columns per thread of a product with ncols columns: the W in {4, 8, 12, 16} with the least
// work, W per column block plus a fixed cost per block (the reloads of A).
__device__ __forceinline__ int choose_width(int ncols) {
    int best = 4, bc = 1 << 30;
    for (int W = 4; W <= 16; W += 4) {
        const int c = ((ncols + W - 1) / W) * (W + 3);
        if (c < bc) { bc = c; best = W; }
    }
    return best;
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 x) {  // acc += a x
    acc.x = fmaf(a.x, x.x, fmaf(-a.y, x.y, acc.x));
    acc.y = fmaf(a.x, x.y, fmaf(a.y, x.x, acc.y));
}
__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 x) {  // acc += conj(a) x
    acc.x = fmaf(a.x, x.x, fmaf(a.y, x.y, acc.x));
    acc.y = fmaf(a.x, x.y, fmaf(-a.y, x.x, acc.y));
}

// Sources of the right-hand matrix X of a product with A.
enum : int { SRC_OMEGA = 0, SRC_Z = 1, SRC_RX = 2, SRC_Q = 3 };

// Stages rows [k0, k0 + kc) of X (K x ncols) into Xs as rows of ld complex values (zero padded).
__device__ void stage_x(float2* Xs, int ld, int k0, int kc, int ncols, int src, const SketchJob& J,
                        int job, int l) {
    const bool real = J.real_slice != 0;
    const int K = (src == SRC_Q) ? J.n1 : J.n2;
    if (src == SRC_OMEGA) {
        const int ng = (ncols + 15) >> 4;
        for (int t = threadIdx.x; t < kc * ng; t += blockDim.x) {
            const int r = k0 + t % kc, g = t / kc;
            const uint32_t h = sk::omega_hash(kOmegaSeed, (uint32_t)job, (uint32_t)r, 16u * g);
            for (int c = 16 * g; c < min(ncols, 16 * g + 16); ++c)
                Xs[(r - k0) * ld + c] = sk::omega_entry(h >> (2 * (c - 16 * g)), real);
        }
        const int pad = ld - ncols;
        for (int t = threadIdx.x; t < kc * pad; t += blockDim.x)
            Xs[(t / pad) * ld + ncols + t % pad] = make_float2(0.f, 0.f);
        return;
    }
    const float2* X = (src == SRC_Q) ? J.Q : J.Z;
    for (int t = threadIdx.x; t < kc * ld; t += blockDim.x) {
        const int r = t % kc, c = t / kc;  // coalesced along the column of X
        float2 v = make_float2(0.f, 0.f);
        if (c < l) {
            v = X[(k0 + r) + (size_t)K * c];
        } else if (src == SRC_RX && c == l) {
            v = sk::omega(kDeflSeed, (uint32_t)job, (uint32_t)(k0 + r), 0u, real);
        }
        Xs[r * ld + c] = v;
    }
}

// Products with A for every slice of a round, one CTA per slice at a time:
//   AH = false: Y (n1 x ncols) = A X into Q, X from Omega (SRC_OMEGA), Z (SRC_Z) or [R x]
//               (SRC_RX, giving T = A [R x]);
//   AH = true:  Z (n2 x l) = A^H Q.
// A thread owns one output row and W columns (a register tile) over a part of the K range
// (parts meet in a shared-memory tile); X is staged in shared memory in chunks of rows, read as
// float4 pairs.  For A X consecutive threads read consecutive rows of a column of A (coalesced
// loads).  For A^H X the rows k0..k0+kc of A are first staged transposed (coalesced down each
// column of A, stored with an odd stride so that threads of consecutive columns read distinct
// banks).
template <bool AH, int W>
__device__ void mult_slice(const SketchJob& J, int job, int l, int src, float2* Xs, float2* At,
                           float2* acc_tile, int xs_cap, int at_cap) {
    const int n1 = J.n1, n2 = J.n2;
    const bool real = J.real_slice != 0;
    const int ncols = (src == SRC_RX) ? l + 1 : l;
    const int rows = AH ? n2 : n1, K = AH ? n1 : n2;
    const int nch = (ncols + W - 1) / W, ld = W * nch;
    int kcap = max(2, xs_cap / ld);
    if (AH) kcap = min(kcap, max(2, at_cap / n2 - 1));
    const int items = rows * nch;
    const int S = choose_split(items, W, K);
    const int total = items * S;
    float2* out = AH ? J.Z : J.Q;  // A [R x] goes to Q too: Q is dead once U = Q V is formed
    if (S > 1) {
        for (int t = threadIdx.x; t < items * W; t += kPT) acc_tile[t] = make_float2(0.f, 0.f);
    }
    const int nchunks = (K + kcap - 1) / kcap;
    for (int base = 0; base < total; base += kPT) {
        const int t = base + threadIdx.x;
        const bool act = t < total;
        const int it = act ? t % items : 0, p = act ? t / items : 0;
        const int r = it % rows, jc = it / rows;
        float2 acc[W];
#pragma unroll
        for (int q = 0; q < W; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int ch = 0; ch < nchunks; ++ch) {
            const int k0 = ch * kcap, kc = min(kcap, K - k0);
            if (nchunks > 1 || base == 0) {
                __syncthreads();
                stage_x(Xs, ld, k0, kc, ncols, AH ? SRC_Q : src, J, job, l);
                if (AH) {  // At[c * (kc | 1) + i] = A(k0 + i, c)
                    const int kp = kc | 1;
                    for (int u = threadIdx.x; u < kc * n2; u += kPT) {
                        const int i = u % kc, c = u / kc;
                        At[c * kp + i] = ld_a(J.A, (k0 + i) + (int64_t)n1 * c, real);
                    }
                }
                __syncthreads();
            }
            if (!act) continue;
            const float4* x4 = reinterpret_cast<const float4*>(Xs) + (W * jc) / 2;
            const float2* col = AH ? At + r * (kc | 1) : nullptr;
#pragma unroll 4
            for (int k = p; k < kc; k += S) {
                // parts interleave over k; A X: rows of a thread group are consecutive in A
                const float2 av = AH ? col[k] : ld_a(J.A, r + (int64_t)n1 * (k0 + k), real);
                const float4* xr = x4 + (k * ld) / 2;
#pragma unroll
                for (int q = 0; q < W / 2; ++q) {
                    const float4 xv = xr[q];
                    if (AH) {
                        cmac_conj(acc[2 * q], av, make_float2(xv.x, xv.y));
                        cmac_conj(acc[2 * q + 1], av, make_float2(xv.z, xv.w));
                    } else {
                        cmac(acc[2 * q], av, make_float2(xv.x, xv.y));
                        cmac(acc[2 * q + 1], av, make_float2(xv.z, xv.w));
                    }
                }
            }
        }
        if (!act) continue;
        if (S == 1) {
#pragma unroll
            for (int q = 0; q < W; ++q)
                if (W * jc + q < ncols) out[r + (size_t)rows * (W * jc + q)] = acc[q];
        } else {
#pragma unroll
            for (int q = 0; q < W; ++q) {
                atomicAdd(&acc_tile[W * it + q].x, acc[q].x);
                atomicAdd(&acc_tile[W * it + q].y, acc[q].y);
            }
        }
    }
    if (S > 1) {
        __syncthreads();
        for (int t = threadIdx.x; t < items * W; t += kPT) {
            const int it = t / W, q = t % W;
            const int r = it % rows, c = W * (it / rows) + q;
            if (c < ncols) out[r + (size_t)rows * c] = acc_tile[t];
        }
    }
}

template <bool AH>
__global__ void __launch_bounds__(kPT, 2) sk_mult_kernel(StageArgs a, int src) {
    extern __shared__ float4 smem4[];
    __shared__ int s_job;
    constexpr int xs_cap = (AH ? kXsBytesAH : kXsBytes) / (int)sizeof(float2);
    constexpr int at_cap = kAtBytes / (int)sizeof(float2);
    float2* Xs = reinterpret_cast<float2*>(smem4);
    float2* At = Xs + xs_cap;  // A^H X only
    float2* acc_tile = At + (AH ? at_cap : 0);
    const int n = list_len(a);
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
        const int job = stage_slice(a, item, &s_job);
        if (job < 0) continue;
        const SketchJob J = a.jobs[job];
        const int l = a.ell[job];
        switch (choose_width((src == SRC_RX) ? l + 1 : l)) {
            case 4: mult_slice<AH, 4>(J, job, l, src, Xs, At, acc_tile, xs_cap, at_cap); break;
            case 8: mult_slice<AH, 8>(J, job, l, src, Xs, At, acc_tile, xs_cap, at_cap); break;
            case 12: mult_slice<AH, 12>(J, job, l, src, Xs, At, acc_tile, xs_cap, at_cap); break;
            default: mult_slice<AH, 16>(J, job, l, src, Xs, At, acc_tile, xs_cap, at_cap); break;
        }
    }
}

// ----------------------------------------------------------------------------- small matrices
// G (l x l, column-major, full Hermitian, shared) = Y^H Y for Y n x l (ld n, global).  Rows
// of Y are staged in chunks (coalesced down each column, stored row-major with an odd stride)
// and every thread accumulates the entries i <= j it owns (at most kPairs of them) over the
// chunk: threads of a warp read one staged row at different columns.
constexpr int kPairs = (kLMax * (kLMax + 1) / 2 + kST - 1) / kST;
__device__ void gram_global(const float2* __restrict__ Y, int n, int l, float2* G, float2* Ys) {
    const int np = l * (l + 1) / 2;
    const int lp = l | 1;
    const int kr = max(1, (kYsBytes / (int)sizeof(float2)) / lp);
    int pi[kPairs], pj[kPairs];
    float2 acc[kPairs];
#pragma unroll
    for (int u = 0; u < kPairs; ++u) {
        const int p = threadIdx.x + u * kST;
        int j = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
        while (j * (j + 1) / 2 > p) --j;
        while ((j + 1) * (j + 2) / 2 <= p) ++j;
        pj[u] = p < np ? j : 0;
        pi[u] = p < np ? p - j * (j + 1) / 2 : 0;
        acc[u] = make_float2(0.f, 0.f);
    }
    for (int e0 = 0; e0 < n; e0 += kr) {
        const int rows = min(kr, n - e0);
        __syncthreads();
        for (int t = threadIdx.x; t < rows * l; t += blockDim.x) {
            const int r = t % rows, c = t / rows;
            Ys[r * lp + c] = Y[(e0 + r) + (size_t)n * c];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPairs; ++u) {
            if (threadIdx.x + u * kST >= np) break;
            const float2* ya = Ys + pi[u];
            const float2* yb = Ys + pj[u];
            float gr = acc[u].x, gi = acc[u].y;
#pragma unroll 4
            for (int r = 0; r < rows; ++r) {
                const float2 x = ya[r * lp], y = yb[r * lp];
                gr = fmaf(x.x, y.x, fmaf(x.y, y.y, gr));  // conj(x) y
                gi = fmaf(x.x, y.y, fmaf(-x.y, y.x, gi));
            }
            acc[u] = make_float2(gr, gi);
        }
    }
#pragma unroll
    for (int u = 0; u < kPairs; ++u) {
        if (threadIdx.x + u * kST >= np) break;
        G[pi[u] + l * pj[u]] = acc[u];
        G[pj[u] + l * pi[u]] = make_float2(acc[u].x, -acc[u].y);
    }
    __syncthreads();
}

// C (l x l, upper triangular) with C^H (G + shift I) C = I, i.e. C = R^-1 for the Cholesky
// factor R^H R = G + shift I: Gram-Schmidt of the unit vectors e_0..e_{l-1} in the
// (G + shift I) inner product.  G is overwritten by M = (G + shift I) C, kept current column
// by column, so every step needs only dot products of length l: warp 0 normalises c_j (and
// m_j), then one half-warp per later column k forms h = m_j^H c_k and updates c_k -= h c_j,
// m_k -= h m_j.  Returns false (uniformly) if a norm is not positive (breakdown).
__device__ bool chol_inv(float2* G, float2* C, int l, float shift, int* s_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = blockDim.x;
    for (int t = tid; t < l * l; t += T) {
        const bool d = (t % l) == (t / l);
        C[t] = make_float2(d ? 1.f : 0.f, 0.f);
        if (d) G[t].x += shift;
    }
    __syncthreads();
    const int hw = tid >> 4, hl = tid & 15, nhw = T >> 4;
    for (int j = 0; j < l; ++j) {
        if (warp == 0) {
            float p = 0.f;
            for (int m = lane; m <= j; m += 32) {
                const float2 cj = C[m + l * j], mj = G[m + l * j];
                p = fmaf(cj.x, mj.x, fmaf(cj.y, mj.y, p));  // c_j^H m_j (real)
            }
            p = warp_sum(p);
            const bool ok = p > 0.f;
            const float inv = ok ? rsqrt_nr(p) : 0.f;
            for (int m = lane; m < l; m += 32) {
                if (m <= j) { C[m + l * j].x *= inv; C[m + l * j].y *= inv; }
                G[m + l * j].x *= inv;
                G[m + l * j].y *= inv;
            }
            if (lane == 0) *s_flag = ok ? 0 : 1;
        }
        __syncthreads();
        if (*s_flag) return false;
        for (int kb = j + 1; kb < l; kb += nhw) {  // uniform over each warp
            const int k = kb + hw;
            const bool act = k < l;
            float hr = 0.f, hi = 0.f;
            for (int m = hl; m <= (act ? k : -1); m += 16) {
                const float2 mm = G[m + l * j], c = C[m + l * k];
                hr = fmaf(mm.x, c.x, fmaf(mm.y, c.y, hr));  // conj(m_j) c_k
                hi = fmaf(mm.x, c.y, fmaf(-mm.y, c.x, hi));
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                hr += __shfl_xor_sync(0xffffffffu, hr, o);
                hi += __shfl_xor_sync(0xffffffffu, hi, o);
            }
            if (act) {
                for (int m = hl; m < l; m += 16) {
                    if (m <= j) {
                        const float2 cj = C[m + l * j];
                        float2 c = C[m + l * k];
                        c.x -= fmaf(hr, cj.x, -hi * cj.y);
                        c.y -= fmaf(hr, cj.y, hi * cj.x);
                        C[m + l * k] = c;
                    }
                    const float2 mj = G[m + l * j];
                    float2 mk = G[m + l * k];
                    mk.x -= fmaf(hr, mj.x, -hi * mj.y);
                    mk.y -= fmaf(hr, mj.y, hi * mj.x);
                    G[m + l * k] = mk;
                }
            }
        }
        __syncthreads();
    }
    return true;
}

// Yout (n x l, global) = Yin C (global) for an upper triangular C (l x l, shared): a thread
// owns one row and 4 columns.
__device__ void mult_upper_global(const float2* __restrict__ Yin, const float2* C,
                                  float2* __restrict__ Yout, int n, int l) {
    const int nq = (l + 3) >> 2;
    for (int t = threadIdx.x; t < n * nq; t += blockDim.x) {
        const int e = t % n, k0 = (t / n) * 4;
        const int kn = min(4, l - k0);
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int m = 0; m < k0 + kn; ++m) {
            const float2 y = Yin[e + (size_t)n * m];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < kn) cmac(acc[q], y, C[m + l * (k0 + q)]);  // C is zero below the diagonal
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < kn) Yout[e + (size_t)n * (k0 + q)] = acc[q];
    }
    __syncthreads();
}

struct SmallShared {
    int job, flag;
    float red[kST / 32];
    float4 rot[kLMax / 2];
    int2 pq[kLMax / 2];
};

// Shifted CholeskyQR (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa) of the l columns of
// Q (which = 0, n1 x l) or Z (which = 1, n2 x l): a pass Y <- Y R^-1 with R^H R the Cholesky
// factorisation of Y^H Y + shift I, the shift 11 (n l + l (l + 1)) u ||Y||_F^2 (u = 2^-24) so
// that the pass cannot break down, then a plain pass, which leaves the (now well
// conditioned) basis orthonormal to working accuracy.  The passes go through S and back.
__global__ void __launch_bounds__(kST) sk_orth_kernel(StageArgs a, int which) {
    extern __shared__ float4 smem4[];
    __shared__ SmallShared sh;
    float2* G = reinterpret_cast<float2*>(smem4);
    float2* C = G + kLMax * kLMax;
    float2* Ys = C + kLMax * kLMax;
    const int nlist = list_len(a);
    for (int item = blockIdx.x; item < nlist; item += gridDim.x) {
        const int job = stage_slice(a, item, &sh.job);
        if (job < 0) continue;
        const SketchJob J = a.jobs[job];
        const int l = a.ell[job];
        const int n = which ? J.n2 : J.n1;
        float2* Y = which ? J.Z : J.Q;
        float2* S = J.S;
        bool ok = true;
        for (int pass = 0; pass < 2 && ok; ++pass) {
            float2* src = pass == 0 ? Y : S;
            float2* dst = pass == 0 ? S : Y;
            gram_global(src, n, l, G, Ys);
            float shift = 0.f;
            if (pass == 0) {
                float tr = 0.f;
                for (int j = 0; j < l; ++j) tr += G[j + l * j].x;
                shift = 11.f * (float)(n * l + l * (l + 1)) * 5.9604645e-08f * tr;
            }
            ok = chol_inv(G, C, l, shift, &sh.flag);
            if (ok) mult_upper_global(src, C, dst, n, l);
        }
        if (!ok && threadIdx.x == 0) a.flag[job] = FLAG_FAIL;
    }
}

// Eigen-decomposition G = V diag(lambda) V^H of the l x l (l <= kLMax) Hermitian G by the
// CTA: parallel two-sided Jacobi over the round-robin tournament.  Each round first forms the
// rotations of its P pairs (one thread per pair), then applies all of them at once: every
// 2 x 2 block of G (rows of pair i, columns of pair j) becomes J_i^H G_ij J_j and V <- V J.
// Rows and columns of different pairs are disjoint, so the blocks are independent.  Returns
// false without convergence in 30 sweeps.
__device__ bool eigh_cta(float2* G, float2* V, int l, float4* rot, int2* pq) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int t = tid; t < l * l; t += T) V[t] = make_float2((t % l) == (t / l) ? 1.f : 0.f, 0.f);
    __syncthreads();
    if (l < 2) return true;
    const int Np = l + (l & 1), P = Np / 2;
    const float tol = 8.f * 1.1920928955078125e-07f, tol2 = tol * tol;
    for (int sweep = 0; sweep < 30; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < Np - 1; ++r) {
            if (tid < P) {
                int pa, pb;
                if (tid == 0) { pa = Np - 1; pb = r; }
                else { pa = (r + tid) % (Np - 1); pb = (r - tid + Np - 1) % (Np - 1); }
                const int p = min(pa, pb), q = max(pa, pb);  // q == l only for the odd-l dummy
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
            for (int t = tid; t < P * P + l * P; t += T) {
                if (t < P * P) {
                    const int i = t % P, j = t / P;
                    const float4 ri = rot[i], rj = rot[j];
                    if (ri.w == 0.f && rj.w == 0.f) continue;
                    const int2 ra = pq[i], rb = pq[j];
                    // block [[x0, x1], [y0, y1]]: rows (ra.x, ra.y), columns (rb.x, rb.y)
                    const float2 z = make_float2(0.f, 0.f);
                    float2 x0 = G[ra.x + l * rb.x];
                    float2 x1 = rb.y >= 0 ? G[ra.x + l * rb.y] : z;
                    float2 y0 = ra.y >= 0 ? G[ra.y + l * rb.x] : z;
                    float2 y1 = (ra.y >= 0 && rb.y >= 0) ? G[ra.y + l * rb.y] : z;
                    // rows: g_p <- c g_p - w g_q, g_q <- conj(w) g_p + c g_q   (w = sr + i si)
                    const float c = ri.x, sr = ri.y, si = ri.z;
                    const float2 n0 = make_float2(fmaf(c, x0.x, -fmaf(sr, y0.x, -si * y0.y)),
                                                  fmaf(c, x0.y, -fmaf(sr, y0.y, si * y0.x)));
                    const float2 m0 = make_float2(fmaf(sr, x0.x, fmaf(si, x0.y, c * y0.x)),
                                                  fmaf(sr, x0.y, fmaf(-si, x0.x, c * y0.y)));
                    const float2 n1 = make_float2(fmaf(c, x1.x, -fmaf(sr, y1.x, -si * y1.y)),
                                                  fmaf(c, x1.y, -fmaf(sr, y1.y, si * y1.x)));
                    const float2 m1 = make_float2(fmaf(sr, x1.x, fmaf(si, x1.y, c * y1.x)),
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
                    G[ra.x + l * rb.x] = x0;
                    if (rb.y >= 0) G[ra.x + l * rb.y] = x1;
                    if (ra.y >= 0) G[ra.y + l * rb.x] = y0;
                    if (ra.y >= 0 && rb.y >= 0) G[ra.y + l * rb.y] = y1;
                } else {
                    const int u = t - P * P, k = u % l, j = u / l;
                    const float4 rj = rot[j];
                    if (rj.w == 0.f) continue;
                    const int2 rb = pq[j];
                    const float d = rj.x, tr = rj.y, ti = rj.z;
                    const float2 x = V[k + l * rb.x], y = V[k + l * rb.y];
                    V[k + l * rb.x] = make_float2(fmaf(d, x.x, fmaf(-tr, y.x, -ti * y.y)),
                                                  fmaf(d, x.y, fmaf(-tr, y.y, ti * y.x)));
                    V[k + l * rb.y] = make_float2(fmaf(tr, x.x, fmaf(-ti, x.y, d * y.x)),
                                                  fmaf(tr, x.y, fmaf(ti, x.x, d * y.y)));
                }
            }
            __syncthreads();
        }
        if (!__syncthreads_or(rotated)) return true;
    }
    return false;
}

// Yout (n x l, global, ld n) = Yin (global, ld n) V (l x l, shared): a thread owns a row and
// 4 columns.
__device__ void mult_small_global(const float2* __restrict__ Yin, const float2* V,
                                  float2* __restrict__ Yout, int n, int l) {
    const int nq = (l + 3) >> 2;
    for (int t = threadIdx.x; t < n * nq; t += blockDim.x) {
        const int e = t % n, k0 = (t / n) * 4;
        const int kn = min(4, l - k0);
        float2 acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int m = 0; m < l; ++m) {
            const float2 y = Yin[e + (size_t)n * m];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < kn) cmac(acc[q], y, V[m + l * (k0 + q)]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < kn) Yout[e + (size_t)n * (k0 + q)] = acc[q];
    }
    __syncthreads();
}

// Step 2 and check (a): G = Z^H Z, its eigenvectors V, D = Z V (into S), sigma_j = ||d_j||
// (near tau: accumulated in FP64), the kept set, R = D / sigma on the kept columns and 0
// elsewhere (into Z), U = Q V (into S, after D is consumed).
__global__ void __launch_bounds__(kST) sk_small_svd_kernel(StageArgs a) {
    extern __shared__ float4 smem4[];
    __shared__ SmallShared sh;
    float2* G = reinterpret_cast<float2*>(smem4);
    float2* V = G + kLMax * kLMax;
    float2* Ys = V + kLMax * kLMax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nlist = list_len(a);
    for (int item = blockIdx.x; item < nlist; item += gridDim.x) {
        const int job = stage_slice(a, item, &sh.job);
        if (job < 0) continue;
        const SketchJob J = a.jobs[job];
        const int l = a.ell[job], n1 = J.n1, n2 = J.n2;
        gram_global(J.Z, n2, l, G, Ys);
        const bool ok = eigh_cta(G, V, l, sh.rot, sh.pq);
        if (!ok) {
            if (tid == 0) a.flag[job] = FLAG_FAIL;
            continue;
        }
        mult_small_global(J.Z, V, J.S, n2, l);  // D
        // sigma_j = ||d_j||; the kept set in FP64, near tau from an FP64 norm
        for (int j = warp; j < l; j += kST / 32) {
            const float2* d = J.S + (size_t)n2 * j;
            float s = 0.f;
            for (int e = lane; e < n2; e += 32) s = fmaf(d[e].x, d[e].x, fmaf(d[e].y, d[e].y, s));
            s = warp_sum(s);
            const float sj = sqrtf(s);
            double sd = sj;
            if (fabs(sd - J.tau) <= 1e-6 * J.tau) {
                double s2 = 0.0;
                for (int e = lane; e < n2; e += 32)
                    s2 = fma((double)d[e].x, (double)d[e].x, fma((double)d[e].y, (double)d[e].y, s2));
                sd = sqrt(sk::warp_sum_d(s2));
            }
            if (lane == 0) {
                J.sig[j] = sj;
                J.keep[j] = sd > J.tau ? 1 : 0;
            }
        }
        __syncthreads();
        int kept = 0;
        for (int j = 0; j < l; ++j) kept += J.keep[j];
        if (kept == l) {  // no computed sigma below tau: the rank was underestimated
            if (tid == 0) a.flag[job] = FLAG_LOW;
            continue;
        }
        // R = D / sigma on the kept columns (0 elsewhere), D read from S
        for (int t = tid; t < n2 * l; t += kST) {
            const int j = t / n2;
            const float f = J.keep[j] ? 1.f / J.sig[j] : 0.f;
            const float2 d = J.S[t];
            J.Z[t] = make_float2(d.x * f, d.y * f);
        }
        __syncthreads();
        mult_small_global(J.Q, V, J.S, n1, l);  // U
    }
}

// Checks (b) and (c) from T = A [R x] (in Q; column l is A x for the random start x):
// residuals ||A r_j - sigma_j u_j|| (sigma_j - tau) / sigma_j of the kept triplets against
// rtol sigma_max, then two power iterations on E = A - U_k S_k R_k^H; flag 0 when both pass.
__global__ void __launch_bounds__(kST, 6) sk_check_kernel(StageArgs a) {
    extern __shared__ float4 smem4[];
    __shared__ SmallShared sh;
    __shared__ float2 coef[kLMax];
    __shared__ float s_norm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nlist = list_len(a);
    for (int item = blockIdx.x; item < nlist; item += gridDim.x) {
        const int job = stage_slice(a, item, &sh.job);
        if (job < 0) continue;
        const SketchJob J = a.jobs[job];
        const int l = a.ell[job], n1 = J.n1, n2 = J.n2;
        const bool real = J.real_slice != 0;
        float2* xv = reinterpret_cast<float2*>(smem4);  // n2
        float2* yv = xv + n2;                            // n1
        const float2* T = J.Q;                           // n1 x (l + 1)
        const float2* U = J.S;                           // n1 x l
        const float2* R = J.Z;                           // n2 x l
        float smax = 0.f;
        int k = 0;
        for (int j = 0; j < l; ++j) {
            smax = fmaxf(smax, J.sig[j]);
            k += J.keep[j];
        }
        // (b) residuals of the kept triplets
        float worst = 0.f;
        for (int j = warp; j < l; j += kST / 32) {
            if (!J.keep[j]) continue;
            const float sj = J.sig[j];
            float s = 0.f;
            for (int e = lane; e < n1; e += 32) {
                const float2 t = T[e + (size_t)n1 * j], u = U[e + (size_t)n1 * j];
                const float dx = t.x - sj * u.x, dy = t.y - sj * u.y;
                s = fmaf(dx, dx, fmaf(dy, dy, s));
            }
            s = warp_sum(s);
            worst = fmaxf(worst, sqrtf(s) * (float)(((double)sj - J.tau) / sj));
        }
        if (lane == 0) sh.red[warp] = worst;
        __syncthreads();
        worst = 0.f;
        for (int w = 0; w < kST / 32; ++w) worst = fmaxf(worst, sh.red[w]);
        if (!(worst <= a.resid_tol * smax)) {
            if (tid == 0) a.flag[job] = FLAG_FAIL;
            continue;
        }
        // (c) x = x0 / ||x0||; A x is column l of T
        float nx = 0.f;
        for (int c = tid; c < n2; c += kST) {
            const float2 v = sk::omega(kDeflSeed, (uint32_t)job, (uint32_t)c, 0u, real);
            xv[c] = v;
            nx = fmaf(v.x, v.x, fmaf(v.y, v.y, nx));
        }
        nx = warp_sum(nx);
        if (lane == 0) sh.red[warp] = nx;
        __syncthreads();
        if (tid == 0) {
            float s = 0.f;
            for (int w = 0; w < kST / 32; ++w) s += sh.red[w];
            s_norm = s > 0.f ? rsqrtf(s) : 0.f;
        }
        __syncthreads();
        float est = 0.f;
        for (int iter = 0; iter < 2; ++iter) {
            const float inx = s_norm;
            for (int c = tid; c < n2; c += kST) { xv[c].x *= inx; xv[c].y *= inx; }
            __syncthreads();
            // coef_j = sigma_j (r_j^H x)   (r_j = 0 on the columns that are not kept)
            for (int j = warp; j < l; j += kST / 32) {
                float dr = 0.f, di = 0.f;
                for (int c = lane; c < n2; c += 32) {
                    const float2 rr = R[c + (size_t)n2 * j], x = xv[c];
                    dr = fmaf(rr.x, x.x, fmaf(rr.y, x.y, dr));
                    di = fmaf(rr.x, x.y, fmaf(-rr.y, x.x, di));
                }
                dr = warp_sum(dr);
                di = warp_sum(di);
                if (lane == 0) coef[j] = make_float2(J.sig[j] * dr, J.sig[j] * di);
            }
            __syncthreads();
            // y = A x - U coef   (A x from T on the first iteration)
            for (int i = tid; i < n1; i += kST) {
                float2 acc = make_float2(0.f, 0.f);
                if (iter == 0) {
                    const float2 t = T[i + (size_t)n1 * l];
                    acc = make_float2(t.x * inx, t.y * inx);
                } else {
                    for (int c = 0; c < n2; ++c) cmac(acc, ld_a(J.A, i + (int64_t)n1 * c, real), xv[c]);
                }
                for (int j = 0; j < l; ++j) {
                    const float2 u = U[i + (size_t)n1 * j], d = coef[j];
                    acc.x -= fmaf(u.x, d.x, -u.y * d.y);
                    acc.y -= fmaf(u.x, d.y, u.y * d.x);
                }
                yv[i] = acc;
            }
            __syncthreads();
            // coef_j = sigma_j (u_j^H y) on the kept columns
            for (int j = warp; j < l; j += kST / 32) {
                float dr = 0.f, di = 0.f;
                for (int i = lane; i < n1; i += 32) {
                    const float2 u = U[i + (size_t)n1 * j], y = yv[i];
                    dr = fmaf(u.x, y.x, fmaf(u.y, y.y, dr));
                    di = fmaf(u.x, y.y, fmaf(-u.y, y.x, di));
                }
                dr = warp_sum(dr);
                di = warp_sum(di);
                const float w = J.keep[j] ? J.sig[j] : 0.f;
                if (lane == 0) coef[j] = make_float2(w * dr, w * di);
            }
            __syncthreads();
            // x = A^H y (a warp per column of A, coalesced, lanes over its rows) ...
            for (int c = warp; c < n2; c += kST / 32) {
                float dr = 0.f, di = 0.f;
                for (int i = lane; i < n1; i += 32) {
                    const float2 av = ld_a(J.A, i + (int64_t)n1 * c, real), y = yv[i];
                    dr = fmaf(av.x, y.x, fmaf(av.y, y.y, dr));
                    di = fmaf(av.x, y.y, fmaf(-av.y, y.x, di));
                }
                dr = warp_sum(dr);
                di = warp_sum(di);
                if (lane == 0) xv[c] = make_float2(dr, di);
            }
            __syncthreads();
            // ... - R coef (threads over the rows of R: coalesced, independent loads)
            for (int c = tid; c < n2; c += kST) {
                float2 acc = xv[c];
                for (int j = 0; j < l; ++j) {
                    const float2 rr = R[c + (size_t)n2 * j], d = coef[j];
                    acc.x -= fmaf(rr.x, d.x, -rr.y * d.y);
                    acc.y -= fmaf(rr.x, d.y, rr.y * d.x);
                }
                xv[c] = acc;
            }
            __syncthreads();
            float s = 0.f;
            for (int c = tid; c < n2; c += kST) s = fmaf(xv[c].x, xv[c].x, fmaf(xv[c].y, xv[c].y, s));
            s = warp_sum(s);
            if (lane == 0) sh.red[warp] = s;
            __syncthreads();
            if (tid == 0) {
                float t = 0.f;
                for (int w = 0; w < kST / 32; ++w) t += sh.red[w];
                s_norm = t > 0.f ? rsqrtf(t) : 0.f;
                sh.red[0] = sqrtf(sqrtf(t));  // ||E^H E x||^(1/2) with ||x|| = 1
            }
            __syncthreads();
            est = sh.red[0];
            __syncthreads();
        }
        if (tid == 0) {
            const bool pass = (double)est < 0.8 * J.tau;
            a.flag[job] = pass ? FLAG_DONE : FLAG_FAIL;
            if (pass && a.count) a.count[job] = k;
        }
    }
}

// Step 4 on the accepted slices: W = sum_{kept j} (sigma_j - tau) u_j r_j^H over the slice, in
// 2 x 2 output tiles (rows i, i + 1; columns c, c + 1).
__global__ void __launch_bounds__(kPT) sk_write_kernel(StageArgs a) {
    __shared__ int s_job;
    __shared__ float fac[kLMax];
    const int nlist = list_len(a);
    for (int item = blockIdx.x; item < nlist; item += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int j = a.list[item];
            s_job = (j >= 0 && a.flag[j] == FLAG_DONE) ? j : -1;
        }
        __syncthreads();
        const int job = s_job;
        if (job < 0) continue;
        const SketchJob J = a.jobs[job];
        const int l = a.ell[job], n1 = J.n1, n2 = J.n2;
        const bool real = J.real_slice != 0;
        for (int j = threadIdx.x; j < l; j += kPT)
            fac[j] = J.keep[j] ? (float)((double)J.sig[j] - J.tau) : 0.f;
        __syncthreads();
        const float2* U = J.S;
        const float2* R = J.Z;
        const int h1 = (n1 + 1) >> 1, h2 = (n2 + 1) >> 1;
        for (int t = threadIdx.x; t < h1 * h2; t += kPT) {
            const int i = 2 * (t % h1), c = 2 * (t / h1);
            const bool i1 = i + 1 < n1, c1 = c + 1 < n2;
            float2 a00 = make_float2(0.f, 0.f), a10 = a00, a01 = a00, a11 = a00;
            for (int j = 0; j < l; ++j) {
                const float f = fac[j];
                if (f == 0.f) continue;
                float2 u0 = U[i + (size_t)n1 * j], u1 = i1 ? U[i + 1 + (size_t)n1 * j] : u0;
                u0.x *= f; u0.y *= f; u1.x *= f; u1.y *= f;
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
    }
}

// Start of the first round: slices with a usable width are marked in progress, the others go
// to the Jacobi path; no extra power iterations yet.
__global__ void sk_init_kernel(const SketchJob* __restrict__ jobs, int n, const int32_t* ell,
                               int32_t* flag, int32_t* extra) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const SketchJob& J = jobs[j];
    const int l = ell[j];
    const bool ok = l > 0 && l < min(J.n1, J.n2) && l <= J.lcap && l <= kLMax;
    flag[j] = ok ? FLAG_RUN : FLAG_FAIL;
    extra[j] = 0;
}

// Between rounds: every slice that failed (flag 1 or 3) and has min(n1, n2) >= min_dim (its
// Jacobi SVD would cost much more than another sketch) is queued for another attempt -- with
// two more power iterations if its sketch reached below tau (flag 1), or 4 columns wider if
// the rank was underestimated (flag 3) and the wider sketch fits its buffers; it is marked in
// progress.  Any other failed slice is marked 4 (left to the Jacobi path).
__global__ void __launch_bounds__(1024) sk_collect_kernel(const SketchJob* __restrict__ jobs,
                                                          int n, int32_t* __restrict__ flag,
                                                          int32_t* __restrict__ ell,
                                                          int32_t* __restrict__ extra, int min_dim,
                                                          int32_t* list, int32_t* len) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int f = flag[j];
        if (f != FLAG_FAIL && f != FLAG_LOW) continue;
        const SketchJob& J = jobs[j];
        const int l = ell[j];
        bool again = min(J.n1, J.n2) >= min_dim && l > 0;
        if (again && f == FLAG_FAIL) {
            extra[j] += 2;
        } else if (again) {
            again = l + 4 < min(J.n1, J.n2) && l + 4 <= min(kLMax, J.lcap);
            if (again) ell[j] = l + 4;
        }
        flag[j] = again ? FLAG_RUN : FLAG_LEFT;
        if (again) list[atomicAdd(len, 1)] = j;
    }
}

constexpr size_t kMultSmem = kXsBytes + (size_t)kAccCplx * sizeof(float2);
constexpr size_t kMultSmemAH = kXsBytesAH + kAtBytes + (size_t)kAccCplx * sizeof(float2);
constexpr size_t kSmallSmem = 2 * (size_t)kLMax * kLMax * sizeof(float2) + kYsBytes;
// sk_check_kernel: the vectors x (n2) and y (n1), at most 2 * TP_MAX_SVD_DIM complex values
constexpr size_t kCheckSmem = 2 * (size_t)TP_MAX_SVD_DIM * sizeof(float2);

struct Occupancy {
    int mult_a = 0, mult_ah = 0, orth = 0, svd = 0, check = 0, write = 0;
};
std::mutex g_occ_mutex;
Occupancy g_occ[128];
bool g_occ_ready[128] = {};

cudaError_t occupancy(Occupancy* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_occ_mutex);
    if (!g_occ_ready[dev]) {
        Occupancy o;
        struct K { const void* fn; size_t smem; int threads; int* dst; };
        const K ks[] = {
            {reinterpret_cast<const void*>(sk_mult_kernel<false>), kMultSmem, kPT, &o.mult_a},
            {reinterpret_cast<const void*>(sk_mult_kernel<true>), kMultSmemAH, kPT, &o.mult_ah},
            {reinterpret_cast<const void*>(sk_orth_kernel), kSmallSmem, kST, &o.orth},
            {reinterpret_cast<const void*>(sk_small_svd_kernel), kSmallSmem, kST, &o.svd},
            {reinterpret_cast<const void*>(sk_check_kernel), kCheckSmem, kST, &o.check},
            {reinterpret_cast<const void*>(sk_write_kernel), 0, kPT, &o.write}};
        for (const K& k : ks) {
            // opt in for every kernel: dynamic plus static shared memory may pass 48 KB
            e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(k.dst, k.fn, k.threads, k.smem);
            if (e != cudaSuccess) return e;
            if (*k.dst < 1) return cudaErrorInvalidConfiguration;
        }
        g_occ[dev] = o;
        g_occ_ready[dev] = true;
    }
    *out = g_occ[dev];
    return cudaSuccess;
}

}  // namespace

size_t sketch_job_floats(int n1, int n2) {
    const int lcap = sketch_lcap(n1, n2);
    if (lcap <= 0) return 0;
    const size_t m = n1 > n2 ? n1 : n2;
    // Q n1 x (lcap + 1), Z n2 x lcap, S m x (lcap + 1) complex; sig and keep lcap each
    const size_t cplx = (size_t)n1 * (lcap + 1) + (size_t)n2 * lcap + m * (lcap + 1);
    return ((2 * cplx + 2 * (size_t)lcap) + 63) & ~(size_t)63;  // 256-byte multiples
}

cudaError_t run_sketch_svt(const SketchJob* jobs, int n, const int32_t* order, int32_t* ell,
                           int32_t* flag, int32_t* count, int32_t* extra, int32_t* retry_lists,
                           int32_t* retry_len, int sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    Occupancy occ;
    cudaError_t e = occupancy(&occ);
    if (e != cudaSuccess) return e;
    sk_init_kernel<<<(n + 255) / 256, 256, 0, s>>>(jobs, n, ell, flag, extra);
    e = cudaMemsetAsync(retry_len, 0, sizeof(int32_t) * kSketchRetryRounds, s);
    if (e != cudaSuccess) return e;
    StageArgs a;
    a.jobs = jobs;
    a.ell = ell;
    a.flag = flag;
    a.count = count;
    a.extra = extra;
    a.power_iters = 1;
    a.resid_tol = 1e-5f;
    auto grid = [&](int per_sm) { return std::max(1, std::min(n, sms * per_sm)); };
    auto mult = [&](bool ah, int src, int stage) {
        a.stage = stage;
        if (ah) sk_mult_kernel<true><<<grid(occ.mult_ah), kPT, kMultSmemAH, s>>>(a, src);
        else sk_mult_kernel<false><<<grid(occ.mult_a), kPT, kMultSmem, s>>>(a, src);
    };
    auto orth = [&](int which, int stage) {
        a.stage = stage;
        sk_orth_kernel<<<grid(occ.orth), kST, kSmallSmem, s>>>(a, which);
    };
    for (int round = 0; round <= kSketchRetryRounds; ++round) {
        if (round == 0) {
            a.list = order;
            a.len_d = nullptr;
            a.len_h = n;
        } else {
            int32_t* list = retry_lists + (size_t)((round - 1) & 1) * n;
            sk_collect_kernel<<<1, 1024, 0, s>>>(jobs, n, flag, ell, extra, kSketchRetryMinDim, list,
                                                 retry_len + (round - 1));
            a.list = list;
            a.len_d = retry_len + (round - 1);
        }
        const int qmax = a.power_iters + 2 * round;  // a retry adds two power iterations
        mult(false, SRC_OMEGA, -1);
        orth(0, -1);
        for (int it = 0; it < qmax; ++it) {
            mult(true, SRC_Q, it);
            orth(1, it);
            mult(false, SRC_Z, it);
            orth(0, it);
        }
        mult(true, SRC_Q, -1);
        a.stage = -1;
        sk_small_svd_kernel<<<grid(occ.svd), kST, kSmallSmem, s>>>(a);
        mult(false, SRC_RX, -1);
        sk_check_kernel<<<grid(occ.check), kST, kCheckSmem, s>>>(a);
        sk_write_kernel<<<grid(occ.write), kPT, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int sketch_stage_launches(int power_iters) {
    int total = 1;  // init
    for (int round = 0; round <= kSketchRetryRounds; ++round)
        total += (round > 0 ? 1 : 0) + 7 + 4 * (power_iters + 2 * round);
    return total;
}

}  // namespace tp
