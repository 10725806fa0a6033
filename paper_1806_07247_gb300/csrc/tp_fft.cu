// Mode-3 tube DFTs (section 2.2): the forward real DFT that keeps the ceil((n3+1)/2)
// independent frequencies (Lemma 2.1, Eq. 8) and the inverse DFT that implies the
// conjugate mirror of the remaining frequencies and scales by 1/n3 (F^-1 = F^*/n, Eq. 1).
//
// Data layout.  A tensor of n1*n2 = P tubes and n3 samples is column-major, so sample t
// of tube p is at x[p + P*t]: consecutive tubes are consecutive in memory.  A CTA takes
// TP consecutive tubes, stages all their samples in shared memory with coalesced (float4
// where the alignment allows) loads, and each thread then produces 4 consecutive tubes
// x 4 frequencies per pass, reading the samples as float4 and the twiddles as warp
// broadcasts.  Outputs are written back coalesced, frequency-major (X[p + P*k]).
//
// Twiddles.  w(n, m) = exp(2*pi*i*m/n) for 0 <= m < n and every n <= TP_MAX_N3 are
// computed once per device on the host in FP64 (quarter points exact) and kept in a
// static device table; the exponent (k*t) mod n3 is advanced by integer addition.
//
// This direct form serves n3 > 64; a launch whose tubes all have the same power-of-two
// n3 <= 64 uses the register FFT kernels further below, and any other launch with n3 <= 64
// the register-resident mixed-radix FFT kernels after them (a direct paired DFT for the odd
// prime lengths 37..61).  The power-of-two kernels can also write the forward spectrum
// straight into the BF16 hi/lo operand planes of the tensor-core slice GEMM
// (FftJob::plane_kind), so that the t-product's BF16x3 path needs no separate split pass.
#include <math.h>

#include <mutex>
#include <vector>

#include "tp_internal.cuh"
#include "tp_planes.cuh"

namespace tp {

namespace {

constexpr int kFftThreads = 256;
constexpr int64_t kTwiddleCount = (int64_t)TP_MAX_N3 * (TP_MAX_N3 + 1) / 2;

// Table for length n starts at n*(n-1)/2.
__device__ float2 g_twiddle[kTwiddleCount];

__host__ __device__ inline int64_t tw_offset(int n) { return (int64_t)n * (n - 1) / 2; }

int tubes_per_cta(int max_n3) {
    if (max_n3 <= 128) return 128;
    if (max_n3 <= 256) return 64;
    return 32;
}

size_t fft_smem_bytes(int max_n3, bool inverse) {
    int tp = tubes_per_cta(max_n3);
    int rows = inverse ? free_slices(max_n3) : max_n3;
    size_t elem = inverse ? sizeof(float2) : sizeof(float);
    return (size_t)rows * tp * elem + (size_t)max_n3 * sizeof(float2);
}

// The job of CTA b: the last job whose tile_begin <= b (tile_begin increases with the job
// index, job 0 starts at 0).  Each warp searches with 32 probes per round (two rounds up to
// 1,024 jobs) instead of a binary search's chain of dependent loads; every lane of the warp
// must call it.
__device__ inline int find_job(const FftJob* jobs, int njobs, int b) {
    const int lane = threadIdx.x & 31;
    int lo = 0, end = njobs;
    while (end - lo > 1) {
        const int step = (end - lo + 31) / 32;
        const int j = lo + lane * step;
        const bool le = j < end && __ldg(&jobs[j].tile_begin) <= b;  // true in lane 0
        const unsigned m = __ballot_sync(0xffffffffu, le);
        lo += (31 - __clz(m)) * step;
        end = min(end, lo + step);
    }
    return lo;
}

// Forward: X[p, k] = sum_t x[p, t] * exp(-2 pi i k t / n3), k < h.
template <bool VEC>
__global__ void __launch_bounds__(kFftThreads) rfft_kernel(const FftJob* __restrict__ jobs,
                                                           int njobs, int TP) {
    extern __shared__ float4 smem4[];
    const FftJob J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int n3 = J.n3, h = free_slices(n3);
    const int64_t P = J.P;
    const int64_t p0 = (int64_t)(blockIdx.x - J.tile_begin) * TP;
    const int G = TP / 4;  // groups of 4 tubes
    float* xs = reinterpret_cast<float*>(smem4);
    float2* tw = reinterpret_cast<float2*>(xs + (size_t)n3 * TP);
    const float2* gtw = g_twiddle + tw_offset(n3);
    const int tid = threadIdx.x;

    for (int i = tid; i < n3; i += kFftThreads) tw[i] = gtw[i];
    if (VEC) {
        float4* xs4 = reinterpret_cast<float4*>(xs);
        for (int idx = tid; idx < n3 * G; idx += kFftThreads) {
            int t = idx / G, g = idx - t * G;
            int64_t p = p0 + 4 * g;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < P) v = __ldg(reinterpret_cast<const float4*>(J.x + p + P * t));
            xs4[idx] = v;
        }
    } else {
        for (int idx = tid; idx < n3 * TP; idx += kFftThreads) {
            int t = idx / TP, j = idx - t * TP;
            int64_t p = p0 + j;
            xs[idx] = (p < P) ? __ldg(J.x + p + P * t) : 0.f;
        }
    }
    __syncthreads();

    const int g = tid % G, f = tid / G, F = kFftThreads / G;
    const float4* xs4 = reinterpret_cast<const float4*>(xs);
    const int64_t pg = p0 + 4 * g;
    for (int base = f; base < h; base += 4 * F) {
        int k[4], e[4];
        float ar[4][4], ai[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kq = base + q * F;
            k[q] = (kq < h) ? kq : 0;
            e[q] = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) ar[q][i] = ai[q][i] = 0.f;
        }
        // samples t and n3 - t paired: x_t e^{-i th k t} + x_{n3-t} e^{+i th k t}
        //   = (x_t + x_{n3-t}) cos(th k t) - i (x_t - x_{n3-t}) sin(th k t)
        {
            const float4 x0 = xs4[g];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ar[q][0] = x0.x; ar[q][1] = x0.y; ar[q][2] = x0.z; ar[q][3] = x0.w;
            }
            if ((n3 & 1) == 0) {  // x_{n3/2} e^{-i pi k} = (-1)^k x_{n3/2}
                const float4 xm = xs4[(n3 / 2) * G + g];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float sg = (k[q] & 1) ? -1.f : 1.f;
                    ar[q][0] = fmaf(sg, xm.x, ar[q][0]); ar[q][1] = fmaf(sg, xm.y, ar[q][1]);
                    ar[q][2] = fmaf(sg, xm.z, ar[q][2]); ar[q][3] = fmaf(sg, xm.w, ar[q][3]);
                }
            }
        }
        for (int t = 1; 2 * t < n3; ++t) {
            const float4 a = xs4[t * G + g], b = xs4[(n3 - t) * G + g];
            const float4 sv = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
            const float4 dv = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                e[q] += k[q];
                if (e[q] >= n3) e[q] -= n3;
                const float2 w = tw[e[q]];
                ar[q][0] = fmaf(sv.x, w.x, ar[q][0]); ai[q][0] = fmaf(-dv.x, w.y, ai[q][0]);
                ar[q][1] = fmaf(sv.y, w.x, ar[q][1]); ai[q][1] = fmaf(-dv.y, w.y, ai[q][1]);
                ar[q][2] = fmaf(sv.z, w.x, ar[q][2]); ai[q][2] = fmaf(-dv.z, w.y, ai[q][2]);
                ar[q][3] = fmaf(sv.w, w.x, ar[q][3]); ai[q][3] = fmaf(-dv.w, w.y, ai[q][3]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kq = base + q * F;
            if (kq >= h) continue;
            if (is_real_slice(kq, n3)) {
#pragma unroll
                for (int i = 0; i < 4; ++i) ai[q][i] = 0.f;
            }
            float2* dst = J.X + pg + P * kq;
            if (VEC) {
                if (pg < P) {
                    reinterpret_cast<float4*>(dst)[0] = make_float4(ar[q][0], ai[q][0], ar[q][1], ai[q][1]);
                    reinterpret_cast<float4*>(dst)[1] = make_float4(ar[q][2], ai[q][2], ar[q][3], ai[q][3]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (pg + i < P) dst[i] = make_float2(ar[q][i], ai[q][i]);
            }
        }
    }
}

// Inverse: x[p, t] = (1/n3) sum_{k<n3} X[p, k] exp(2 pi i k t / n3) with X[n3-k] = conj(X[k]),
// i.e. (1/n3) [Re X0 + 2 sum_{0<k<n3/2} Re(X_k e^{i theta}) + (even n3) Re X_{n3/2} (-1)^t].
template <bool VEC>
__global__ void __launch_bounds__(kFftThreads) irfft_kernel(const FftJob* __restrict__ jobs,
                                                            int njobs, int TP) {
    extern __shared__ float4 smem4[];
    const FftJob J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int n3 = J.n3, h = free_slices(n3);
    const int64_t P = J.P;
    const int64_t p0 = (int64_t)(blockIdx.x - J.tile_begin) * TP;
    const int G = TP / 4;
    float2* Xs = reinterpret_cast<float2*>(smem4);
    float2* tw = Xs + (size_t)h * TP;
    const float2* gtw = g_twiddle + tw_offset(n3);
    const int tid = threadIdx.x;
    const float inv_n = 1.0f / (float)n3;

    for (int i = tid; i < n3; i += kFftThreads) tw[i] = gtw[i];
    // Stage the half spectrum, pre-scaled by its weight (1 or 2) / n3; the imaginary
    // parts of the real slices are dropped.
    for (int idx = tid; idx < h * G; idx += kFftThreads) {
        int k = idx / G, gg = idx - k * G;
        int64_t p = p0 + 4 * gg;
        float wk = is_real_slice(k, n3) ? inv_n : 2.f * inv_n;
        float wi = is_real_slice(k, n3) ? 0.f : wk;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        const float2* src = J.X + p + P * k;
        if (VEC) {
            if (p < P) {
                a = __ldg(reinterpret_cast<const float4*>(src));
                b = __ldg(reinterpret_cast<const float4*>(src) + 1);
            }
        } else {
            float2 v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                v[i] = (p + i < P) ? __ldg(src + i) : make_float2(0.f, 0.f);
            a = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
            b = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
        }
        a.x *= wk; a.y *= wi; a.z *= wk; a.w *= wi;
        b.x *= wk; b.y *= wi; b.z *= wk; b.w *= wi;
        float4* d = reinterpret_cast<float4*>(Xs + (size_t)k * TP + 4 * gg);
        d[0] = a;
        d[1] = b;
    }
    __syncthreads();

    // outputs t and n3 - t paired: with the weighted X_k = Xr + i Xi,
    //   x_t = sum_k (Xr cos - Xi sin),  x_{n3-t} = sum_k (Xr cos + Xi sin)   (angle th k t)
    const int g = tid % G, f = tid / G, F = kFftThreads / G;
    const int64_t pg = p0 + 4 * g;
    float* xout = const_cast<float*>(J.x);
    const int half = n3 / 2;  // t = 0..half produce every output
    for (int base = f; base <= half; base += 4 * F) {
        int tt[4], e[4];
        float ca[4][4], sb[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int tq = base + q * F;
            tt[q] = (tq <= half) ? tq : 0;
            e[q] = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) ca[q][i] = sb[q][i] = 0.f;
        }
        for (int k = 0; k < h; ++k) {
            const float4* row = reinterpret_cast<const float4*>(Xs + (size_t)k * TP + 4 * g);
            float4 a = row[0], b = row[1];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 w = tw[e[q]];
                e[q] += tt[q];
                if (e[q] >= n3) e[q] -= n3;
                ca[q][0] = fmaf(a.x, w.x, ca[q][0]); sb[q][0] = fmaf(a.y, w.y, sb[q][0]);
                ca[q][1] = fmaf(a.z, w.x, ca[q][1]); sb[q][1] = fmaf(a.w, w.y, sb[q][1]);
                ca[q][2] = fmaf(b.x, w.x, ca[q][2]); sb[q][2] = fmaf(b.y, w.y, sb[q][2]);
                ca[q][3] = fmaf(b.z, w.x, ca[q][3]); sb[q][3] = fmaf(b.w, w.y, sb[q][3]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int tq = base + q * F;
            if (tq > half) continue;
#pragma unroll
            for (int m = 0; m < 2; ++m) {  // m = 0: t, m = 1: n3 - t
                const int tout = m == 0 ? tq : n3 - tq;
                if (m == 1 && (tq == 0 || 2 * tq == n3)) continue;
                const float sg = m == 0 ? -1.f : 1.f;
                float o[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) o[i] = fmaf(sg, sb[q][i], ca[q][i]);
                float* dst = xout + pg + P * tout;
                if (VEC) {
                    if (pg < P) *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (pg + i < P) dst[i] = o[i];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Power-of-two n3 <= 64: one thread per tube, the tube in registers.  The real DFT of
// length n3 = 2N is one complex FFT of length N on z[t] = x[2t] + i x[2t+1] (radix-2,
// decimation in time, fully unrolled) followed by the split of Z into the DFTs of the even
// and odd samples: X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[N-k]) / 2,
// O = (Z[k] - conj Z[N-k]) / (2i), W = exp(-2 pi i / n3).  The inverse runs the same steps
// backwards.  Twiddles are exp(2 pi i m / 64) from a constant table, indexed by
// compile-time constants.  Loads and stores are coalesced across the threads of a warp
// (consecutive tubes), so the kernels move each byte once.
// ---------------------------------------------------------------------------------------
__constant__ float2 c_tw64[64];

__host__ __device__ constexpr int bit_reverse(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

__host__ __device__ constexpr int log2_pow2(int n) {
    int b = 0;
    while ((1 << b) < n) ++b;
    return b;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// In-place complex FFT of length N (power of two <= 32) on data already in bit-reversed
// order, unnormalised; INV selects exp(+2 pi i ...) kernels.  Every index is a compile-time
// constant after unrolling, so z stays in registers.
template <int N, bool INV>
__device__ __forceinline__ void cfft_bitrev_regs(float2 (&z)[N]) {
    constexpr int B = log2_pow2(N);
#pragma unroll
    for (int st = 0; st < B; ++st) {
        const int m = 2 << st;
#pragma unroll
        for (int k = 0; k < N; k += m) {
#pragma unroll
            for (int j = 0; j < m / 2; ++j) {
                float2 w = c_tw64[(64 / m) * j];
                if (!INV) w.y = -w.y;
                const float2 t = cmul(w, z[k + j + m / 2]);
                const float2 u = z[k + j];
                z[k + j] = make_float2(u.x + t.x, u.y + t.y);
                z[k + j + m / 2] = make_float2(u.x - t.x, u.y - t.y);
            }
        }
    }
}

// PLANES: the jobs write the BF16x3 operand planes instead of X (FftJob::plane_kind); that
// instantiation is held to 128 registers so that two CTAs still fit on an SM.
template <int N3, bool PLANES>
__global__ void __launch_bounds__(256, PLANES ? 2 : 1)
    rfft_reg_kernel(const FftJob* __restrict__ jobs, int njobs) {
    constexpr int N = N3 / 2;
    const FftJob J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int64_t p = (int64_t)(blockIdx.x - J.tile_begin) * 256 + threadIdx.x;
    if (p >= J.P) return;
    const int64_t P = J.P;
    constexpr int B = log2_pow2(N);
    float2 z[N];  // z[t] = x[2t] + i x[2t+1], stored at bit_reverse(t)
#pragma unroll
    for (int t = 0; t < N; ++t)
        z[bit_reverse(t, B)] =
            make_float2(__ldg(J.x + p + P * (2 * t)), __ldg(J.x + p + P * (2 * t + 1)));
    cfft_bitrev_regs<N, false>(z);
    const PlaneCursor pc = PLANES ? plane_cursor(J, p) : PlaneCursor{};
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        const float2 zk = z[k % N], zc = z[(N - k) % N];
        const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
        const float2 o = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
        float2 w = c_tw64[(64 / N3) * k % 64];
        w.y = -w.y;
        if (k == N) w = make_float2(-1.f, 0.f);
        float2 X = make_float2(e.x + (w.x * o.x - w.y * o.y), e.y + (w.x * o.y + w.y * o.x));
        if (k == 0 || k == N) X.y = 0.f;
        if constexpr (PLANES) store_plane_value(J, pc, k, X);
        else J.X[p + P * k] = X;
    }
}

template <int N3>
__global__ void __launch_bounds__(256) irfft_reg_kernel(const FftJob* __restrict__ jobs, int njobs) {
    constexpr int N = N3 / 2;
    const FftJob J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int64_t p = (int64_t)(blockIdx.x - J.tile_begin) * 256 + threadIdx.x;
    if (p >= J.P) return;
    const int64_t P = J.P;
    float2 X[N + 1];
#pragma unroll
    for (int k = 0; k <= N; ++k) X[k] = __ldg(J.X + p + P * k);
    X[0].y = 0.f;  // the real slices of Eq. 8
    X[N].y = 0.f;
    constexpr int B = log2_pow2(N);
    float2 z[N];  // Z[k] = E[k] + i O[k], stored at bit_reverse(k)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const float2 xk = X[k], xc = X[N - k];
        const float2 e = make_float2(0.5f * (xk.x + xc.x), 0.5f * (xk.y - xc.y));
        const float2 d = make_float2(0.5f * (xk.x - xc.x), 0.5f * (xk.y + xc.y));
        const float2 w = c_tw64[(64 / N3) * k];   // exp(+2 pi i k / n3)
        const float2 o = cmul(d, w);
        z[bit_reverse(k, B)] = make_float2(e.x - o.y, e.y + o.x);
    }
    cfft_bitrev_regs<N, true>(z);
    const float s = 1.f / (float)N;
    float* xo = const_cast<float*>(J.x);
#pragma unroll
    for (int t = 0; t < N; ++t) {
        xo[p + P * (2 * t)] = z[t].x * s;
        xo[p + P * (2 * t + 1)] = z[t].y * s;
    }
}

bool reg_fft_size(int n3) { return n3 >= 2 && n3 <= 64 && (n3 & (n3 - 1)) == 0; }

// ---------------------------------------------------------------------------------------
// Odd prime n3 in 37..61 (launches whose tubes differ in n3, see the mixed-radix kernels
// below for the other lengths): one thread per tube, the tube in registers, the real DFT by
// its definition.  Samples t and n3 - t are
// paired: Re X[k] = x0 + sum_t (x_t + x_{n3-t}) cos(2 pi k t / n3),
// Im X[k] = -sum_t (x_t - x_{n3-t}) sin(2 pi k t / n3), and the inverse pairs the same way.
// The twiddles come from a row table: row k of length n3 holds exp(2 pi i k t / n3) for
// t = 1..H (H = (n3 - 1) / 2, padded to an even count), so the unrolled inner loop reads them
// two at a time (16-byte loads, the same address across the warp) at fixed offsets from one
// row pointer and needs no index arithmetic.  The table is symmetric in k and t, so the
// inverse reads row t for its sum over k.
// A CTA's tubes belong to one job, so the switch on n3 is uniform.
// ---------------------------------------------------------------------------------------
constexpr int kSmallN3 = 64;
__constant__ float2 c_twall[kSmallN3 * (kSmallN3 + 1) / 2];  // length n at n (n - 1) / 2

__host__ __device__ constexpr int prime_row_len(int n) { return ((n - 1) / 2 + 1) & ~1; }
// Offset of the rows of prime length n (37 <= n <= 61) in g_prime_rows; -1 for other n.
__host__ __device__ constexpr int prime_rows_offset(int n) {
    constexpr int primes[7] = {37, 41, 43, 47, 53, 59, 61};
    int off = 0;
    for (int i = 0; i < 7; ++i) {
        if (primes[i] == n) return off;
        off += (primes[i] / 2 + 1) * prime_row_len(primes[i]);
    }
    return -1;
}
constexpr int kPrimeRowsTotal = prime_rows_offset(61) + 31 * prime_row_len(61);
__device__ __align__(16) float2 g_prime_rows[kPrimeRowsTotal];

template <int N>
__device__ __forceinline__ void rdft_small(const float* __restrict__ x, int64_t P, float2* X) {
    constexpr int H = (N - 1) / 2;  // pairs (t, N - t), 1 <= t <= H
    constexpr int L = prime_row_len(N);
    static_assert(N == 1 || prime_rows_offset(N) >= 0, "row table");
    float s[L + 1], d[L + 1];  // entries H + 1 .. L are zero padding
    const float x0 = __ldg(x);
#pragma unroll
    for (int t = 1; t <= L; ++t) {
        if (t <= H) {
            const float a = __ldg(x + P * t), b = __ldg(x + P * (N - t));
            s[t] = a + b;
            d[t] = a - b;
        } else {
            s[t] = d[t] = 0.f;
        }
    }
    if constexpr (N > 1) {
        const float4* rows = reinterpret_cast<const float4*>(g_prime_rows + prime_rows_offset(N));
#pragma unroll 1
        for (int k = 0; k <= N / 2; ++k) {  // rolled: the body stays small in the instruction cache
            const float4* row = rows + k * (L / 2);
            float re = x0, im = 0.f;
#pragma unroll
            for (int u = 0; u < L / 2; ++u) {
                const float4 w = __ldg(row + u);  // t = 2u + 1 and 2u + 2
                re = fmaf(s[2 * u + 1], w.x, re);
                im = fmaf(-d[2 * u + 1], w.y, im);
                re = fmaf(s[2 * u + 2], w.z, re);
                im = fmaf(-d[2 * u + 2], w.w, im);
            }
            if (k == 0) im = 0.f;
            X[P * k] = make_float2(re, im);
        }
    } else {
        X[0] = make_float2(x0, 0.f);
    }
}

template <int N>
__device__ __forceinline__ void irdft_small(const float2* __restrict__ X, int64_t P, float* x) {
    constexpr int H = (N - 1) / 2;  // frequencies 1..H appear twice (k and N - k)
    constexpr int L = prime_row_len(N);
    float re[L + 1], im[L + 1];
    const float r0 = __ldg(X).x;
#pragma unroll
    for (int k = 1; k <= L; ++k) {
        if (k <= H) {
            const float2 v = __ldg(X + P * k);
            re[k] = 2.f * v.x;
            im[k] = 2.f * v.y;
        } else {
            re[k] = im[k] = 0.f;
        }
    }
    const float sc = 1.f / (float)N;
    if constexpr (N > 1) {
        const float4* rows = reinterpret_cast<const float4*>(g_prime_rows + prime_rows_offset(N));
#pragma unroll 1
        for (int t = 0; t <= N / 2; ++t) {
            const float4* row = rows + t * (L / 2);
            float a = r0, b = 0.f;
#pragma unroll
            for (int u = 0; u < L / 2; ++u) {
                const float4 w = __ldg(row + u);  // k = 2u + 1 and 2u + 2
                a = fmaf(re[2 * u + 1], w.x, a);
                b = fmaf(im[2 * u + 1], w.y, b);
                a = fmaf(re[2 * u + 2], w.z, a);
                b = fmaf(im[2 * u + 2], w.w, b);
            }
            x[P * t] = (a - b) * sc;
            if (t > 0) x[P * (N - t)] = (a + b) * sc;
        }
    } else {
        x[0] = r0 * sc;
    }
}

// ---------------------------------------------------------------------------------------
// Mixed-radix FFTs for the other n3 <= 64, one compile-time plan per length.  A complex DFT of
// length M is split by its smallest prime factor R (decimation in time: R sub-DFTs of length
// M / R, twiddles, then R-point DFTs), down to prime lengths, which are computed from their
// definition with the symmetric pairing of samples t and P - t and of frequencies k and P - k
// (about (P - 1)^2 real multiply-adds).  Every index and twiddle index is a compile-time
// constant, so the data stay in registers and each twiddle is an operand read from the
// constant bank (c_twall holds exp(2 pi i m / n) for every n <= 64).
//   Even n3:  one tube per thread, z[t] = x[2t] + i x[2t+1], a complex FFT of length n3 / 2 and
//             the split X[k] = E[k] + W^k O[k] (the inverse runs these steps backwards).
//   Odd n3 that is composite or <= 31:  one tube per thread, a complex FFT of length n3 on
//             x + 0i (two tubes packed as x_a + i x_b would halve the work, but rounding
//             errors of one tube would then reach the other: a zero tube beside a non-zero one
//             would no longer come out exactly zero).
//   Odd primes 37..61: the direct paired DFT above (fully unrolled code for those lengths
//             would not fit the instruction cache).
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

enum : int { SMALL_DIRECT = 0, SMALL_EVEN = 1, SMALL_ODD = 2 };
// How a tube of length n3 <= 64 is transformed (see above).
__host__ __device__ constexpr int small_kind(int n3) {
    return (n3 >= 2 && n3 % 2 == 0) ? SMALL_EVEN
           : (n3 >= 3 && (n3 <= 31 || smallest_factor(n3) != n3)) ? SMALL_ODD
                                                                  : SMALL_DIRECT;
}

// exp(S 2 pi i m / N) for S = +1 or -1 (m a compile-time constant after unrolling).
template <int N, int S>
__device__ __forceinline__ float2 twc(int m) {
    const float2 w = c_twall[N * (N - 1) / 2 + ((m % N) + N) % N];
    return S > 0 ? w : make_float2(w.x, -w.y);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// In-place DFT of prime length P: X[k] = sum_t z[t] exp(S 2 pi i k t / P).
template <int P, int S>
__device__ __forceinline__ void dft_prime(float2 (&z)[P]) {
    if constexpr (P == 2) {
        const float2 a = z[0], b = z[1];
        z[0] = cadd(a, b);
        z[1] = csub(a, b);
    } else if constexpr (P > 2) {
        constexpr int H = (P - 1) / 2;
        float2 sp[H + 1], sm[H + 1];
        const float2 z0 = z[0];
        float2 sum = z0;
#pragma unroll
        for (int t = 1; t <= H; ++t) {
            sp[t] = cadd(z[t], z[P - t]);
            sm[t] = csub(z[t], z[P - t]);
            sum = cadd(sum, sp[t]);
        }
        z[0] = sum;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            float2 a = z0, b = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 1; t <= H; ++t) {
                const float2 w = twc<P, 1>(k * t);  // (cos, sin) of 2 pi k t / P
                a.x = fmaf(sp[t].x, w.x, a.x);
                a.y = fmaf(sp[t].y, w.x, a.y);
                b.x = fmaf(sm[t].x, w.y, b.x);
                b.y = fmaf(sm[t].y, w.y, b.y);
            }
            // X[k] = a + S i b,  X[P - k] = a - S i b
            if (S > 0) {
                z[k] = make_float2(a.x - b.y, a.y + b.x);
                z[P - k] = make_float2(a.x + b.y, a.y - b.x);
            } else {
                z[k] = make_float2(a.x + b.y, a.y - b.x);
                z[P - k] = make_float2(a.x - b.y, a.y + b.x);
            }
        }
    }
}

// In-place DFT of length M (natural order in and out), split by the smallest prime factor.
template <int M, int S>
__device__ __forceinline__ void cfft(float2 (&z)[M]) {
    constexpr int R = smallest_factor(M);
    if constexpr (M == 1) {
    } else if constexpr (R == M) {
        dft_prime<M, S>(z);
    } else {
        constexpr int Q = M / R;
        float2 sub[R][Q];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < Q; ++q) sub[r][q] = z[r + R * q];
#pragma unroll
        for (int r = 0; r < R; ++r) cfft<Q, S>(sub[r]);
        // X[k + Q s] = sum_r exp(S 2 pi i r s / R) (exp(S 2 pi i r k / M) Sub_r[k])
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            float2 t[R];
            t[0] = sub[0][k];
#pragma unroll
            for (int r = 1; r < R; ++r) t[r] = cmul(sub[r][k], twc<M, S>(r * k));
            dft_prime<R, S>(t);
#pragma unroll
            for (int q = 0; q < R; ++q) z[k + Q * q] = t[q];
        }
    }
}

// Even N: real DFT of one tube through a complex FFT of length N / 2.
template <int N>
__device__ __forceinline__ void rfft_even(const float* __restrict__ x, int64_t P, float2* X) {
    constexpr int M = N / 2;
    float2 z[M];
#pragma unroll
    for (int t = 0; t < M; ++t) z[t] = make_float2(__ldg(x + P * (2 * t)), __ldg(x + P * (2 * t + 1)));
    cfft<M, -1>(z);
#pragma unroll
    for (int k = 0; k <= M; ++k) {
        const float2 zk = z[k % M], zc = z[(M - k) % M];
        const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y - zc.y));
        const float2 o = make_float2(0.5f * (zk.y + zc.y), -0.5f * (zk.x - zc.x));
        const float2 w = twc<N, -1>(k);
        float2 Xk = make_float2(e.x + (w.x * o.x - w.y * o.y), e.y + (w.x * o.y + w.y * o.x));
        if (k == 0 || k == M) Xk.y = 0.f;
        X[P * k] = Xk;
    }
}

template <int N>
__device__ __forceinline__ void irfft_even(const float2* __restrict__ X, int64_t P, float* x) {
    constexpr int M = N / 2;
    float2 Xv[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) Xv[k] = __ldg(X + P * k);
    Xv[0].y = 0.f;  // the real slices of Eq. 8
    Xv[M].y = 0.f;
    float2 z[M];  // Z[k] = E[k] + i O[k]
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float2 xk = Xv[k], xc = Xv[M - k];
        const float2 e = make_float2(0.5f * (xk.x + xc.x), 0.5f * (xk.y - xc.y));
        const float2 d = make_float2(0.5f * (xk.x - xc.x), 0.5f * (xk.y + xc.y));
        const float2 o = cmul(d, twc<N, 1>(k));
        z[k] = make_float2(e.x - o.y, e.y + o.x);
    }
    cfft<M, 1>(z);
    const float s = 1.f / (float)M;
#pragma unroll
    for (int t = 0; t < M; ++t) {
        x[P * (2 * t)] = z[t].x * s;
        x[P * (2 * t + 1)] = z[t].y * s;
    }
}

// Odd N: real DFT of one tube through a complex FFT of length N on x + 0i.
template <int N>
__device__ __forceinline__ void rfft_odd(const float* __restrict__ x, int64_t P, float2* X) {
    float2 z[N];
#pragma unroll
    for (int t = 0; t < N; ++t) z[t] = make_float2(__ldg(x + P * t), 0.f);
    cfft<N, -1>(z);
#pragma unroll
    for (int k = 0; k <= N / 2; ++k) {
        float2 v = z[k];
        if (k == 0) v.y = 0.f;
        X[P * k] = v;
    }
}

// Inverse: the full spectrum from the half (Z[N - k] = conj Z[k]), a complex FFT, the real part.
template <int N>
__device__ __forceinline__ void irfft_odd(const float2* __restrict__ X, int64_t P, float* x) {
    float2 z[N];
#pragma unroll
    for (int k = 0; k <= N / 2; ++k) {
        float2 v = __ldg(X + P * k);
        if (k == 0) v.y = 0.f;
        z[k] = v;
        if (k > 0) z[N - k] = make_float2(v.x, -v.y);
    }
    cfft<N, 1>(z);
    const float s = 1.f / (float)N;
#pragma unroll
    for (int t = 0; t < N; ++t) x[P * t] = z[t].x * s;
}

// Register class of the transforms of length n3 <= 64 (ptxas, sm_103a): '0' needs at most 64
// registers, '1' at most 128, '2' more.  Each class runs in its own kernel instantiation whose
// launch bounds give it 4, 2 or 1 CTAs of 256 threads per SM.
// Bit n3 - 1 of kClassAtLeast1 / kClass2: class >= 1 / class 2.
constexpr unsigned long long kClassAtLeast1 = 0xfffffff500000000ull, kClass2 = 0x0ull;
__host__ __device__ constexpr int small_class(int n3) {
    return (int)((kClassAtLeast1 >> (n3 - 1)) & 1ull) + (int)((kClass2 >> (n3 - 1)) & 1ull);
}

// Tubes per CTA of the kernels below (one per thread).
__host__ __device__ constexpr int small_tubes_per_cta(int) { return 256; }

template <int N, int CLS>
__device__ __forceinline__ void rfft_small_one(const FftJob& J, int64_t p0) {
    const int64_t P = J.P;
    if constexpr (small_class(N) == CLS) {
        const int64_t p = p0 + threadIdx.x;
        if (p >= P) return;
        if constexpr (small_kind(N) == SMALL_EVEN) rfft_even<N>(J.x + p, P, J.X + p);
        else if constexpr (small_kind(N) == SMALL_ODD) rfft_odd<N>(J.x + p, P, J.X + p);
        else rdft_small<N>(J.x + p, P, J.X + p);
    }
}

template <int N, int CLS>
__device__ __forceinline__ void irfft_small_one(const FftJob& J, int64_t p0) {
    const int64_t P = J.P;
    float* x = const_cast<float*>(J.x);
    if constexpr (small_class(N) == CLS) {
        const int64_t p = p0 + threadIdx.x;
        if (p >= P) return;
        if constexpr (small_kind(N) == SMALL_EVEN) irfft_even<N>(J.X + p, P, x + p);
        else if constexpr (small_kind(N) == SMALL_ODD) irfft_odd<N>(J.X + p, P, x + p);
        else irdft_small<N>(J.X + p, P, x + p);
    }
}

#define TP_SMALL_CASES(M) \
    M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) \
    M(17) M(18) M(19) M(20) M(21) M(22) M(23) M(24) M(25) M(26) M(27) M(28) M(29) M(30) \
    M(31) M(32) M(33) M(34) M(35) M(36) M(37) M(38) M(39) M(40) M(41) M(42) M(43) M(44) \
    M(45) M(46) M(47) M(48) M(49) M(50) M(51) M(52) M(53) M(54) M(55) M(56) M(57) M(58) \
    M(59) M(60) M(61) M(62) M(63) M(64)

// A CTA's tubes belong to one job, so the switch on n3 is uniform.  A launch holds the jobs of
// one register class CLS only.
template <int CLS>
__global__ void __launch_bounds__(256, CLS == 0 ? 4 : (CLS == 1 ? 2 : 1))
    rfft_small_kernel(const FftJob* __restrict__ jobs, int njobs) {
    const FftJob J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int64_t p0 = (int64_t)(blockIdx.x - J.tile_begin) * small_tubes_per_cta(J.n3);
    switch (J.n3) {
#define TP_FWD(n) case n: rfft_small_one<n, CLS>(J, p0); break;
        TP_SMALL_CASES(TP_FWD)
#undef TP_FWD
        default: break;
    }
}

template <int CLS>
__global__ void __launch_bounds__(256, CLS == 0 ? 4 : (CLS == 1 ? 2 : 1))
    irfft_small_kernel(const FftJob* __restrict__ jobs, int njobs) {
    const FftJob J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int64_t p0 = (int64_t)(blockIdx.x - J.tile_begin) * small_tubes_per_cta(J.n3);
    switch (J.n3) {
#define TP_INV(n) case n: irfft_small_one<n, CLS>(J, p0); break;
        TP_SMALL_CASES(TP_INV)
#undef TP_INV
        default: break;
    }
}

template <bool INV>
cudaError_t launch_small(const FftJob* d_jobs, int njobs, int tiles, int cls, cudaStream_t s) {
    switch (cls) {
        case 0:
            if (INV) irfft_small_kernel<0><<<tiles, 256, 0, s>>>(d_jobs, njobs);
            else rfft_small_kernel<0><<<tiles, 256, 0, s>>>(d_jobs, njobs);
            break;
        case 1:
            if (INV) irfft_small_kernel<1><<<tiles, 256, 0, s>>>(d_jobs, njobs);
            else rfft_small_kernel<1><<<tiles, 256, 0, s>>>(d_jobs, njobs);
            break;
        case 2:
            if (INV) irfft_small_kernel<2><<<tiles, 256, 0, s>>>(d_jobs, njobs);
            else rfft_small_kernel<2><<<tiles, 256, 0, s>>>(d_jobs, njobs);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

std::mutex g_tw_mutex;
bool g_tw_ready[128] = {};

}  // namespace

cudaError_t ensure_twiddles() {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_tw_mutex);
    if (g_tw_ready[dev]) return cudaSuccess;
    static std::vector<float2> host;
    if (host.empty()) {
        host.resize((size_t)kTwiddleCount);
        for (int n = 1; n <= TP_MAX_N3; ++n) {
            float2* row = host.data() + tw_offset(n);
            for (int m = 0; m < n; ++m) {
                double c, s;
                if (m == 0) { c = 1.0; s = 0.0; }
                else if (2 * m == n) { c = -1.0; s = 0.0; }
                else if (4 * m == n) { c = 0.0; s = 1.0; }
                else if (4 * m == 3 * n) { c = 0.0; s = -1.0; }
                else {
                    double a = 2.0 * M_PI * (double)m / (double)n;
                    c = cos(a);
                    s = sin(a);
                }
                row[m] = make_float2((float)c, (float)s);
            }
        }
    }
    err = cudaMemcpyToSymbol(g_twiddle, host.data(), sizeof(float2) * host.size());
    if (err != cudaSuccess) return err;
    err = cudaMemcpyToSymbol(c_tw64, host.data() + tw_offset(64), sizeof(float2) * 64);
    if (err != cudaSuccess) return err;
    err = cudaMemcpyToSymbol(c_twall, host.data(),
                             sizeof(float2) * (size_t)kSmallN3 * (kSmallN3 + 1) / 2);
    if (err != cudaSuccess) return err;
    {
        // rows of the direct prime-length DFTs: entry (k, t) = w(n, k t mod n), zero padding
        std::vector<float2> rows((size_t)kPrimeRowsTotal, make_float2(0.f, 0.f));
        for (int n : {37, 41, 43, 47, 53, 59, 61}) {
            const int L = prime_row_len(n), H = (n - 1) / 2;
            float2* base = rows.data() + prime_rows_offset(n);
            for (int k = 0; k <= n / 2; ++k)
                for (int t = 1; t <= H; ++t)
                    base[(size_t)k * L + (t - 1)] = host[(size_t)tw_offset(n) + (size_t)((k * t) % n)];
        }
        err = cudaMemcpyToSymbol(g_prime_rows, rows.data(), sizeof(float2) * rows.size());
        if (err != cudaSuccess) return err;
    }
    // the largest dynamic shared memory any launch of these kernels asks for
    const int fwd = (int)fft_smem_bytes(TP_MAX_N3, false), inv = (int)fft_smem_bytes(TP_MAX_N3, true);
    int mf = fwd, mi = inv;
    for (int n = 1; n <= TP_MAX_N3; ++n) {
        mf = mf > (int)fft_smem_bytes(n, false) ? mf : (int)fft_smem_bytes(n, false);
        mi = mi > (int)fft_smem_bytes(n, true) ? mi : (int)fft_smem_bytes(n, true);
    }
    cudaError_t e1 = cudaFuncSetAttribute(rfft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mf);
    cudaError_t e2 = cudaFuncSetAttribute(rfft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mf);
    cudaError_t e3 = cudaFuncSetAttribute(irfft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mi);
    cudaError_t e4 = cudaFuncSetAttribute(irfft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mi);
    for (cudaError_t e : {e1, e2, e3, e4})
        if (e != cudaSuccess) return e;
    g_tw_ready[dev] = true;
    return cudaSuccess;
}

int fft_tiles(int64_t P, int max_n3, int uniform_n3, int n3) {
    const int tp = reg_fft_size(uniform_n3) ? 256
                   : max_n3 <= kSmallN3    ? small_tubes_per_cta(n3)
                                           : tubes_per_cta(max_n3);
    return (int)((P + tp - 1) / tp);
}

template <bool INV>
cudaError_t launch_reg(const FftJob* d_jobs, int njobs, int tiles, int n3, bool planes,
                       cudaStream_t s) {
    switch (n3) {
#define TP_REG_CASE(n)                                                                 \
    case n:                                                                            \
        if (INV) irfft_reg_kernel<n><<<tiles, 256, 0, s>>>(d_jobs, njobs);             \
        else if (planes) rfft_reg_kernel<n, true><<<tiles, 256, 0, s>>>(d_jobs, njobs); \
        else rfft_reg_kernel<n, false><<<tiles, 256, 0, s>>>(d_jobs, njobs);           \
        break;
        TP_REG_CASE(2) TP_REG_CASE(4) TP_REG_CASE(8) TP_REG_CASE(16) TP_REG_CASE(32)
        TP_REG_CASE(64)
#undef TP_REG_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool fft_writes_planes(int n3) { return reg_fft_size(n3); }

bool fft_small_path(int max_n3, int uniform_n3) {
    return !reg_fft_size(uniform_n3) && max_n3 <= kSmallN3;
}

int fft_small_class(int n3) { return (n3 >= 1 && n3 <= kSmallN3) ? small_class(n3) : 0; }

cudaError_t launch_rfft(const FftJob* d_jobs, int njobs, int total_tiles, int max_n3,
                        int uniform_n3, bool vec_ok, cudaStream_t s, int small_cls, bool planes) {
    if (total_tiles <= 0) return cudaSuccess;
    if (planes && !reg_fft_size(uniform_n3)) return cudaErrorInvalidValue;
    if (reg_fft_size(uniform_n3))
        return launch_reg<false>(d_jobs, njobs, total_tiles, uniform_n3, planes, s);
    if (max_n3 <= kSmallN3) {
        const int cls = small_cls >= 0 ? small_cls : fft_small_class(uniform_n3);
        return launch_small<false>(d_jobs, njobs, total_tiles, cls, s);
    }
    int tp = tubes_per_cta(max_n3);
    size_t smem = fft_smem_bytes(max_n3, false);
    if (vec_ok) rfft_kernel<true><<<total_tiles, kFftThreads, smem, s>>>(d_jobs, njobs, tp);
    else rfft_kernel<false><<<total_tiles, kFftThreads, smem, s>>>(d_jobs, njobs, tp);
    return cudaGetLastError();
}

cudaError_t launch_irfft(const FftJob* d_jobs, int njobs, int total_tiles, int max_n3,
                         int uniform_n3, bool vec_ok, cudaStream_t s, int small_cls) {
    if (total_tiles <= 0) return cudaSuccess;
    if (reg_fft_size(uniform_n3))
        return launch_reg<true>(d_jobs, njobs, total_tiles, uniform_n3, false, s);
    if (max_n3 <= kSmallN3) {
        const int cls = small_cls >= 0 ? small_cls : fft_small_class(uniform_n3);
        return launch_small<true>(d_jobs, njobs, total_tiles, cls, s);
    }
    int tp = tubes_per_cta(max_n3);
    size_t smem = fft_smem_bytes(max_n3, true);
    if (vec_ok) irfft_kernel<true><<<total_tiles, kFftThreads, smem, s>>>(d_jobs, njobs, tp);
    else irfft_kernel<false><<<total_tiles, kFftThreads, smem, s>>>(d_jobs, njobs, tp);
    return cudaGetLastError();
}

}  // namespace tp
