// Per-slice SVDs of the Fourier slices (Algorithm 2 step 2, Algorithm 3 step 2, Eq. 14):
// one CTA per slice runs a one-sided (Hestenes) Jacobi SVD and then one of three
// epilogues:
//   SVD_SIGMA  singular values only, sorted decreasing (tnn, tsn, tubal rank);
//   SVD_PROX   singular value thresholding W = U (S - tau)_+ V^* (Algorithm 3);
//   SVD_FULL   U, S and V (Algorithm 2), with the unitary factors completed to the
//              requested number of columns.
//
// Orientation.  The slice A (n1 x n2, column-major) is worked on as G = A when n1 >= n2
// and as G = A^H otherwise, so G is m x n with n = min(n1, n2) columns of length
// m = max(n1, n2).  Jacobi rotations from the right make the columns of G V orthogonal:
// G V = B with b_j = sigma_j u_j.
//
// Rotation of a column pair (p, q), with alpha = |g_p|^2, beta = |g_q|^2 and
// gamma = g_p^H g_q = |gamma| e (|e| = 1): the pair is rotated when
// |gamma| > tol * sqrt(alpha beta).  With zeta = (beta - alpha) / (2 |gamma|),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t:
//   g_p <- c g_p - s conj(e) g_q,   g_q <- s e g_p + c g_q,
// a unitary 2 x 2 map that makes the new pair orthogonal (the real Jacobi rotation
// applied after taking the phase of gamma out of g_q).  On the real slices of Eq. 8
// gamma is real, e = +-1, and the arithmetic stays real.
//
// Parallel order.  Each sweep is the round-robin tournament over n (rounded up to even)
// columns: n' - 1 rounds of n'/2 disjoint pairs.  A pair is handled by a group of LP
// lanes (LP = 8, 16 or 32 by column length, so that each lane holds several elements);
// a warp carries 32/LP pairs at once and the CTA is sized to the pairs of a round.  The
// group holds its two columns in registers (up to 2*MAXE2 elements per lane) between the dot
// products and the update, reduces within the group with xor shuffles, and forms the
// rotation with refined reciprocal square roots (rotation_cs keeps c^2 + s^2 = 1 to an ulp,
// which is what bounds the singular value error; computing c and s in FP64 is no better).  A sweep with no rotation ends the
// iteration.
//
// Working storage.  G lives in shared memory when it fits, otherwise in a global scratch
// area of the slice; its columns are zero-padded to 2*LP*e2 entries so that each lane owns
// e2 float4 pairs (8 lanes of a quarter-warp read 128 contiguous bytes: no bank conflicts,
// no bounds tests in the rotation loop).  SVD_FULL accumulates V in global scratch.
//
// The SVT epilogue needs no V: u_j = b_j / sigma_j and v_j^* = b_j^* A_G / sigma_j^2,
// so W_G = sum_{sigma_j > tau} ((sigma_j - tau) / sigma_j) (1/sigma_j^2) b_j (b_j^* g_c)
// column by column, re-reading the original column g_c of the slice.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "tp_internal.cuh"
#include "tp_rotation.cuh"

namespace tp {

namespace {

constexpr int kMaxThreads = 512;
constexpr float kEps = 1.1920928955078125e-07f;  // 2^-23

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float block_sum(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

// Largest key (ties to the smaller index) over the block; returns the index.
__device__ __forceinline__ int block_argmax(float key, int idx, float* redf, int* redi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float k2 = __shfl_xor_sync(0xffffffffu, key, o);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
    }
    __syncthreads();
    if (lane == 0) { redf[warp] = key; redi[warp] = idx; }
    __syncthreads();
    float bk = redf[0];
    int bi = redi[0];
    for (int w = 1; w < nw; ++w)
        if (redf[w] > bk || (redf[w] == bk && redi[w] < bi)) { bk = redf[w]; bi = redi[w]; }
    return bi;
}

// Sum over the aligned group of LP lanes holding one column pair.
template <int LP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = LP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of four values over the aligned LP-lane group (LP >= 8), returned in every lane:
// the first two xor steps exchange halves of the set, so log2(LP) + 5 shuffles replace
// the 4 log2(LP) of four separate reductions.
template <int LP>
__device__ __forceinline__ void group_sum4(float& v0, float& v1, float& v2, float& v3,
                                           int sub, int lane) {
    const bool h1 = (sub & (LP / 2)) != 0;
    float k0 = h1 ? v2 : v0, k1 = h1 ? v3 : v1;
    const float s0 = h1 ? v0 : v2, s1 = h1 ? v1 : v3;
    k0 += __shfl_xor_sync(0xffffffffu, s0, LP / 2);
    k1 += __shfl_xor_sync(0xffffffffu, s1, LP / 2);
    const bool h2 = (sub & (LP / 4)) != 0;
    float k = h2 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h2 ? k0 : k1, LP / 4);
#pragma unroll
    for (int o = LP / 8; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    // lane with (h1, h2) = (a, b) now holds the total of value 2a + b
    const int base = lane - sub;
    v0 = __shfl_sync(0xffffffffu, k, base);
    v1 = __shfl_sync(0xffffffffu, k, base + LP / 4);
    v2 = __shfl_sync(0xffffffffu, k, base + LP / 2);
    v3 = __shfl_sync(0xffffffffu, k, base + LP / 2 + LP / 4);
}

// One Jacobi rotation of columns gp, gq by the LP-lane group whose lane index within the
// group is `sub`; for SVD_FULL also of the accumulated V columns vp, vq (length nv).
// Columns are zero-padded to 2*LP*e2 complex entries, so lane `sub` owns the float4 pairs
// sub + LP*i, i < e2, with no bounds test (zero rows stay zero under rotation).  Every lane
// of the warp must call this (the reductions use the full warp mask); inactive groups read
// column 0 and discard the result.  Returns true if the pair was rotated.
template <int LP, int MAXE2, bool WITH_V>
__device__ __forceinline__ bool jacobi_pair(float2* gp, float2* gq, int e2, int sub, int lane,
                                            float tol2, bool active, float2* vp, float2* vq,
                                            int nv, bool fp64_rot) {
    float4* p4 = reinterpret_cast<float4*>(gp);
    float4* q4 = reinterpret_cast<float4*>(gq);
    float4 xp[MAXE2], xq[MAXE2];
    float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
    for (int i = 0; i < MAXE2; ++i) {
        if (i < e2) {
            const float4 a = p4[sub + LP * i], b = q4[sub + LP * i];
            xp[i] = a;
            xq[i] = b;
            al = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, al))));
            be = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, be))));
            gr = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, gr))));
            gi = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, gi))));
        }
    }
    group_sum4<LP>(al, be, gr, gi, sub, lane);
    const float ag2 = fmaf(gr, gr, gi * gi);
    // |gamma| > tol sqrt(alpha beta), squared; a test within a factor 2 of the threshold (or
    // with the threshold below the FP32 normal range) is decided again in FP64
    const float thr = (tol2 * al) * be;
    bool rot = ag2 > thr;
    if ((ag2 > 0.5f * thr && ag2 < 2.f * thr) || thr < 1.17549435e-38f) {
        const double agd = fma((double)gr, (double)gr, (double)gi * (double)gi);
        rot = agd > ((double)tol2 * (double)al) * (double)be;
    }
    if (!active || !rot) return false;
    float c, sr, si;  // s e = (sr, si); s conj(e) = (sr, -si)
    if (fp64_rot) {
        // zeta, t, c, s and the phase e = gamma / |gamma| in FP64 from the FP32 dot products
        const double dgr = gr, dgi = gi;
        const double ag = sqrt(fma(dgr, dgr, dgi * dgi));
        const double zeta = 0.5 * ((double)be - (double)al) / ag;
        const double az = fabs(zeta);
        const double t = copysign(1.0 / (az + sqrt(fma(zeta, zeta, 1.0))), zeta);
        const double cd = 1.0 / sqrt(fma(t, t, 1.0));
        const double sd = cd * t;
        c = (float)cd;
        sr = (float)(sd * (dgr / ag));
        si = (float)(sd * (dgi / ag));
    } else {
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
    // g_p <- c g_p - s conj(e) g_q,  g_q <- s e g_p + c g_q
#pragma unroll
    for (int i = 0; i < MAXE2; ++i) {
        if (i < e2) {
            const float4 a = xp[i], b = xq[i];
            float4 np, nq;
            np.x = fmaf(c, a.x, fmaf(-sr, b.x, -si * b.y));
            np.y = fmaf(c, a.y, fmaf(-sr, b.y, si * b.x));
            np.z = fmaf(c, a.z, fmaf(-sr, b.z, -si * b.w));
            np.w = fmaf(c, a.w, fmaf(-sr, b.w, si * b.z));
            nq.x = fmaf(sr, a.x, fmaf(-si, a.y, c * b.x));
            nq.y = fmaf(sr, a.y, fmaf(si, a.x, c * b.y));
            nq.z = fmaf(sr, a.z, fmaf(-si, a.w, c * b.z));
            nq.w = fmaf(sr, a.w, fmaf(si, a.z, c * b.w));
            p4[sub + LP * i] = np;
            q4[sub + LP * i] = nq;
        }
    }
    if (WITH_V) {
        for (int e = sub; e < nv; e += LP) {
            const float2 a = vp[e], b = vq[e];
            vp[e] = make_float2(fmaf(c, a.x, fmaf(-sr, b.x, -si * b.y)),
                                fmaf(c, a.y, fmaf(-sr, b.y, si * b.x)));
            vq[e] = make_float2(fmaf(sr, a.x, fmaf(-si, a.y, c * b.x)),
                                fmaf(sr, a.y, fmaf(si, a.x, c * b.y)));
        }
    }
    return true;
}

// Shared-memory bytes for the small per-slice arrays that follow G.
__host__ __device__ inline int aux_bytes(int m, int n) {
    int b = 6 * n * 4 + 64 * 4;  // sig, perm, kept, ratio, invs, flag + reductions
    b += (m + 1) * 4 + m * (8 + 8 + 4);  // FULL: rn (padded to even), vtmp, dcoef, valid
    return (b + 15) & ~15;
}

// Column stride of G in complex entries: m rounded up to whole float4 pairs of every lane
// of a group (zero rows pad the tail).
__host__ __device__ inline int col_e2(int m, int lp) { return (m + 2 * lp - 1) / (2 * lp); }
__host__ __device__ inline int col_ld(int m, int lp) { return 2 * lp * col_e2(m, lp); }

template <int MODE, int LP, int MAXE2, bool SMEM>
__global__ void __launch_bounds__(MAXE2 >= 8 ? 512 : 1024, 1)
    svd_kernel(const SvdJob* __restrict__ jobs, SvdParams prm) {
    constexpr int MAXE = 2 * MAXE2;  // complex elements per lane in the scalar phases
    extern __shared__ float4 smem4[];
    __shared__ int s_rot, s_cnt;
    const SvdJob J = jobs[blockIdx.x];
    if (J.skip && *J.skip == 0) return;  // slice finished by the sketch path
    const int n1 = J.n1, n2 = J.n2;
    const bool tr = n1 < n2;
    const int m = tr ? n2 : n1, n = tr ? n1 : n2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int T = blockDim.x;
    const bool real = J.real_slice != 0;
    constexpr int SPW = 32 / LP;             // pairs (or columns) a warp carries at once
    const int grp = lane / LP, sub = lane % LP;
    const int slots = nw * SPW;
    const int slot = warp * SPW + grp;

    const int e2 = col_e2(m, LP);
    const int ld = col_ld(m, LP);
    float2* G = SMEM ? reinterpret_cast<float2*>(smem4) : J.work;
    char* auxp = reinterpret_cast<char*>(smem4) + (SMEM ? (size_t)n * ld * sizeof(float2) : 0);
    float* sig = reinterpret_cast<float*>(auxp);
    int* perm = reinterpret_cast<int*>(sig + n);
    int* kept = perm + n;
    float* ratio = reinterpret_cast<float*>(kept + n);
    float* invs = ratio + n;
    int* flag = reinterpret_cast<int*>(invs + n);
    float* redf = reinterpret_cast<float*>(flag + n);
    int* redi = reinterpret_cast<int*>(redf + 32);
    float* rn = reinterpret_cast<float*>(redi + 32);
    float2* vtmp = reinterpret_cast<float2*>(rn + m + (m & 1));
    float2* dco = vtmp + m;
    int* valid = reinterpret_cast<int*>(dco + m);

    float2* VG = nullptr;
    if (MODE == SVD_FULL) VG = SMEM ? J.work : J.work + (size_t)n * ld;

    // ---- load G (= A or A^H), zero rows m..ld-1 --------------------------------
    if (ld > m) {
        const int pad = ld - m;
        for (int idx = tid; idx < n * pad; idx += T) {
            const int c = idx / pad, e = m + (idx - c * pad);
            G[(size_t)c * ld + e] = make_float2(0.f, 0.f);
        }
    }
    if (!tr) {
        for (int idx = tid; idx < m * n; idx += T) {
            const int c = idx / m, e = idx - c * m;
            float2 v = J.A[e + (int64_t)n1 * c];
            if (real) v.y = 0.f;
            G[(size_t)c * ld + e] = v;
        }
    } else {
        for (int idx = tid; idx < m * n; idx += T) {
            const int e = idx / n1, c = idx - e * n1;  // A(c, e), contiguous in idx
            float2 v = J.A[idx];
            v.y = real ? 0.f : -v.y;
            G[(size_t)c * ld + e] = v;
        }
    }
    if (MODE == SVD_FULL) {
        for (int idx = tid; idx < n * n; idx += T) {
            const int c = idx / n, e = idx - c * n;
            VG[idx] = make_float2(e == c ? 1.f : 0.f, 0.f);
        }
    }
    __syncthreads();

    // ---- Jacobi sweeps ----------------------------------------------------------
    const float tol = prm.tol > 0.f ? prm.tol : 8.f * kEps;
    const float tol2 = tol * tol;
    const int N = n + (n & 1);
    // Unchanged pairs are not revisited: every pair meets once per sweep, in the same round,
    // so a pair whose two columns were not rotated since its previous visit (N - 1 rounds
    // earlier) still passes the test it passed then, on the same data; skipping it gives the
    // same result bit for bit.  last[c] is the round of column c's last rotation (-1: never;
    // the `perm` array, unused until the epilogue).
    int* last = perm;
    for (int c = tid; c < n; c += T) last[c] = -1;
    int sweeps = 0, round = 0;
    bool converged = n < 2;
    while (!converged && sweeps < prm.max_sweeps) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r, ++round) {
            for (int base = 0; base < N / 2; base += slots) {  // uniform over the block
                const int pi = base + slot;
                int a = 0, b = 0;
                if (pi == 0) { a = N - 1; b = r; }
                else { a = (r + pi) % (N - 1); b = (r - pi + N - 1) % (N - 1); }
                bool active = pi < N / 2 && a < n && b < n;
                const int p = active ? min(a, b) : 0, q = active ? max(a, b) : 0;
                if (active && sweeps > 0) {
                    const int prev = round - (N - 1);
                    active = last[p] >= prev || last[q] >= prev;
                }
                if (!__any_sync(0xffffffffu, active)) continue;  // the warp's pairs all skip
                bool did = jacobi_pair<LP, MAXE2, MODE == SVD_FULL>(
                    G + (size_t)p * ld, G + (size_t)q * ld, e2, sub, lane, tol2, active,
                    MODE == SVD_FULL ? VG + (size_t)p * n : nullptr,
                    MODE == SVD_FULL ? VG + (size_t)q * n : nullptr, n, prm.fp64_rotation != 0);
                if (did && sub == 0) {
                    s_rot = 1;
                    last[p] = round;
                    last[q] = round;
                }
            }
            __syncthreads();
        }
        ++sweeps;
        converged = (s_rot == 0);
        __syncthreads();
    }
    if (tid == 0) {
        if (!converged) atomicOr(prm.status, 1u);
        if (prm.sweeps_out && J.sweeps_index >= 0) prm.sweeps_out[J.sweeps_index] = sweeps;
    }

    // ---- column norms: sigma_j = ||b_j|| ----------------------------------------
    for (int cb = 0; cb < n; cb += slots) {  // uniform over the block
        const int c = cb + slot;
        float s = 0.f;
        if (c < n) {
            const float2* g = G + (size_t)c * ld;
            for (int e = sub; e < m; e += LP) s = fmaf(g[e].x, g[e].x, fmaf(g[e].y, g[e].y, s));
        }
        s = group_sum<LP>(s);
        if (c < n && sub == 0) sig[c] = sqrtf(s);
    }
    __syncthreads();

    if (MODE == SVD_SIGMA || MODE == SVD_FULL) {
        // rank sort, decreasing (ties by column index)
        for (int c = tid; c < n; c += T) {
            const float v = sig[c];
            int rank = 0;
            for (int j = 0; j < n; ++j) {
                const float w = sig[j];
                rank += (w > v) || (w == v && j < c);
            }
            perm[rank] = c;
            J.sigma[rank] = v;
        }
        __syncthreads();
    }

    if (MODE == SVD_PROX) {
        // kept set {sigma_j > tau} in column order (ballot compaction); the comparison is in
        // FP64, and a sigma within 1e-6 relative of tau is first recomputed as the column norm
        // accumulated in FP64 (the FP32 norm's rounding could put it on the wrong side)
        int any_near = 0;
        for (int c = tid; c < n; c += T) {
            const double sd = (double)sig[c];
            const int f = sd > J.tau;
            flag[c] = f;
            any_near |= fabs(sd - J.tau) <= 1e-6 * J.tau;
            if (f) {
                ratio[c] = (float)((sd - J.tau) / sd);
                invs[c] = 1.f / sig[c];
            }
        }
        if (__syncthreads_or(any_near)) {
            for (int cb = 0; cb < n; cb += slots) {  // uniform over the block
                const int c = cb + slot;
                const bool near = c < n && fabs((double)sig[c] - J.tau) <= 1e-6 * J.tau;
                double s2 = 0.0;
                if (near) {
                    const float2* g = G + (size_t)c * ld;
                    for (int e = sub; e < m; e += LP)
                        s2 = fma((double)g[e].x, (double)g[e].x, fma((double)g[e].y, (double)g[e].y, s2));
                }
#pragma unroll
                for (int o = LP / 2; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                if (near && sub == 0) {
                    const double sd = sqrt(s2);
                    const int f = sd > J.tau;
                    flag[c] = f;
                    if (f) {
                        ratio[c] = (float)((sd - J.tau) / sd);
                        invs[c] = (float)(1.0 / sd);
                    }
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
            int cnt = 0;
            for (int base = 0; base < n; base += 32) {
                const int c = base + lane;
                const int f = (c < n) ? flag[c] : 0;
                const unsigned mask = __ballot_sync(0xffffffffu, f);
                if (f) kept[cnt + __popc(mask & ((1u << lane) - 1u))] = c;
                cnt += __popc(mask);
            }
            if (lane == 0) {
                s_cnt = cnt;
                if (J.count_out) *J.count_out = cnt;
            }
        }
        __syncthreads();
        const int cnt = s_cnt;
        // W_G(:, c) = sum_k ratio_k invs_k^2 b_k (b_k^H g_c), g_c re-read from the slice
        for (int cb = 0; cb < n; cb += slots) {  // uniform over the block
            const int c = cb + slot;
            const bool act = c < n;
            float2 a[MAXE], w[MAXE];
#pragma unroll
            for (int i = 0; i < MAXE; ++i) {
                const int e = sub + LP * i;
                float2 v = make_float2(0.f, 0.f);
                if (act && e < m) {
                    v = tr ? J.A[c + (int64_t)n1 * e] : J.A[e + (int64_t)n1 * c];
                    if (tr) v.y = -v.y;
                    if (real) v.y = 0.f;
                }
                a[i] = v;
                w[i] = make_float2(0.f, 0.f);
            }
            for (int kk = 0; kk < cnt; ++kk) {
                const int j = kept[kk];
                const float2* b = G + (size_t)j * ld;
                float dr = 0.f, di = 0.f;
#pragma unroll
                for (int i = 0; i < MAXE; ++i) {
                    const int e = sub + LP * i;
                    if (e < m) {
                        const float2 bv = b[e];
                        dr = fmaf(bv.x, a[i].x, fmaf(bv.y, a[i].y, dr));
                        di = fmaf(bv.x, a[i].y, fmaf(-bv.y, a[i].x, di));
                    }
                }
                dr = group_sum<LP>(dr);
                di = group_sum<LP>(di);
                const float sc = ratio[j] * invs[j] * invs[j];
                dr *= sc;
                di *= sc;
#pragma unroll
                for (int i = 0; i < MAXE; ++i) {
                    const int e = sub + LP * i;
                    if (e < m) {
                        const float2 bv = b[e];
                        w[i].x = fmaf(dr, bv.x, fmaf(-di, bv.y, w[i].x));
                        w[i].y = fmaf(dr, bv.y, fmaf(di, bv.x, w[i].y));
                    }
                }
            }
            if (act) {
#pragma unroll
                for (int i = 0; i < MAXE; ++i) {
                    const int e = sub + LP * i;
                    if (e < m) {
                        float2 v = w[i];
                        if (real) v.y = 0.f;
                        if (tr) J.W[c + (int64_t)n1 * e] = make_float2(v.x, -v.y);
                        else J.W[e + (int64_t)n1 * c] = v;
                    }
                }
            }
        }
    }

    if (MODE == SVD_FULL) {
        // V side: the accumulated V_G, columns in decreasing-sigma order (n x n).
        float2* Vd = tr ? J.W : J.Vout;
        for (int idx = tid; idx < n * n; idx += T) {
            const int j = idx / n, e = idx - j * n;
            Vd[idx] = VG[e + (size_t)n * perm[j]];
        }
        // B side: b_j / sigma_j (m x nb), completed to an orthonormal set.
        float2* Bd = tr ? J.Vout : J.W;
        const int nb = tr ? J.vcols : J.ucols;
        const float smax = (n > 0) ? sig[perm[0]] : 0.f;
        const float zero_thr = fmaxf(smax * 1e-30f, 1e-30f);
        for (int j = tid; j < nb; j += T) valid[j] = (j < n) && (sig[perm[j]] > zero_thr);
        for (int idx = tid; idx < m * min(n, nb); idx += T) {
            const int j = idx / m, e = idx - j * m;
            const int c = perm[j];
            const float sv = sig[c];
            float2 v = make_float2(0.f, 0.f);
            if (sv > zero_thr) {
                const float inv = 1.f / sv;
                v = G[(size_t)c * ld + e];
                v.x *= inv;
                v.y *= inv;
            }
            Bd[e + (size_t)m * j] = v;
        }
        __syncthreads();
        for (int i = tid; i < m; i += T) {
            float s = 0.f;
            for (int j = 0; j < nb; ++j)
                if (valid[j]) {
                    const float2 u = Bd[i + (size_t)m * j];
                    s = fmaf(u.x, u.x, fmaf(u.y, u.y, s));
                }
            rn[i] = s;
        }
        __syncthreads();
        for (int slot = 0; slot < nb; ++slot) {
            if (valid[slot]) continue;
            // the standard basis vector least represented by the current columns
            float key = -1.f;
            int idx = 0x7fffffff;
            for (int i = tid; i < m; i += T) {
                const float k = 1.f - rn[i];
                if (k > key || (k == key && i < idx)) { key = k; idx = i; }
            }
            const int istar = block_argmax(key, idx, redf, redi);
            // v = e_i* - sum_j u_j conj(u_j[i*])
            for (int e = tid; e < m; e += T) {
                float vr = (e == istar) ? 1.f : 0.f, vi = 0.f;
                for (int j = 0; j < nb; ++j) {
                    if (!valid[j]) continue;
                    const float2 u = Bd[e + (size_t)m * j];
                    const float2 ui = Bd[istar + (size_t)m * j];
                    // u * conj(ui)
                    vr -= fmaf(u.x, ui.x, u.y * ui.y);
                    vi -= fmaf(u.y, ui.x, -u.x * ui.y);
                }
                vtmp[e] = make_float2(vr, real ? 0.f : vi);
            }
            __syncthreads();
            // second Gram-Schmidt pass: d_j = u_j^H v, v -= sum_j d_j u_j
            for (int j = warp; j < nb; j += nw) {
                float dr = 0.f, di = 0.f;
                if (valid[j]) {
                    for (int e = lane; e < m; e += 32) {
                        const float2 u = Bd[e + (size_t)m * j], v = vtmp[e];
                        dr = fmaf(u.x, v.x, fmaf(u.y, v.y, dr));
                        di = fmaf(u.x, v.y, fmaf(-u.y, v.x, di));
                    }
                    dr = warp_sum(dr);
                    di = warp_sum(di);
                }
                if (lane == 0) dco[j] = make_float2(dr, di);
            }
            __syncthreads();
            float ss = 0.f;
            for (int e = tid; e < m; e += T) {
                float2 v = vtmp[e];
                for (int j = 0; j < nb; ++j) {
                    if (!valid[j]) continue;
                    const float2 u = Bd[e + (size_t)m * j], d = dco[j];
                    v.x -= fmaf(d.x, u.x, -d.y * u.y);
                    v.y -= fmaf(d.x, u.y, d.y * u.x);
                }
                if (real) v.y = 0.f;
                vtmp[e] = v;
                ss = fmaf(v.x, v.x, fmaf(v.y, v.y, ss));
            }
            const float nrm2 = block_sum(ss, redf);
            const float inv = nrm2 > 0.f ? 1.f / sqrtf(nrm2) : 0.f;
            for (int e = tid; e < m; e += T) {
                float2 v = vtmp[e];
                v.x *= inv;
                v.y *= inv;
                Bd[e + (size_t)m * slot] = v;
                rn[e] += fmaf(v.x, v.x, v.y * v.y);
            }
            if (tid == 0) valid[slot] = 1;
            __syncthreads();
        }
    }
}

template <int MODE, int LP, int MAXE2, bool SMEM>
cudaError_t launch_one(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    auto k = svd_kernel<MODE, LP, MAXE2, SMEM>;
    if (L.smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L.smem_bytes);
        if (e != cudaSuccess) return e;
    }
    k<<<L.njobs, L.threads, L.smem_bytes, s>>>(L.jobs, p);
    return cudaGetLastError();
}

template <int MODE, bool SMEM>
cudaError_t launch_cfg(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    switch (L.lp * 100 + L.maxe) {
        case 802: return launch_one<MODE, 8, 2, SMEM>(L, p, s);
        case 804: return launch_one<MODE, 8, 4, SMEM>(L, p, s);
        case 808: return launch_one<MODE, 8, 8, SMEM>(L, p, s);
        case 1602: return launch_one<MODE, 16, 2, SMEM>(L, p, s);
        case 1604: return launch_one<MODE, 16, 4, SMEM>(L, p, s);
        case 1608: return launch_one<MODE, 16, 8, SMEM>(L, p, s);
        case 3202: return launch_one<MODE, 32, 2, SMEM>(L, p, s);
        case 3204: return launch_one<MODE, 32, 4, SMEM>(L, p, s);
        case 3208: return launch_one<MODE, 32, 8, SMEM>(L, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t launch_mode(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    return L.in_smem ? launch_cfg<MODE, true>(L, p, s) : launch_cfg<MODE, false>(L, p, s);
}

// Reductions over the decreasing singular values sigma[k * r + i] of the h directly
// computed slices of one tensor; slice k stands for itself and, when 0 < k and 2k != n3,
// for its mirror n3 - k as well (Eq. 8), so it is weighted 2.
__global__ void sigma_reduce_kernel(const float* __restrict__ sigma, int h, int r, int n3,
                                    double tol, int64_t rank_scale, double* out_tnn,
                                    double* out_tsn, int64_t* out_rank, double* s_out) {
    __shared__ double red[256];
    __shared__ double s0;
    const int tid = threadIdx.x;
    const double inv_n3 = 1.0 / (double)n3;
    double part = 0.0, mx = 0.0;
    for (int i = tid; i < r; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < h; ++k) {
            const double w = (k == 0 || 2 * k == n3) ? 1.0 : 2.0;
            s += w * (double)sigma[(size_t)k * r + i];
        }
        s *= inv_n3;  // S(i, i, 0) of Eq. 14
        if (s_out) s_out[i] = s;
        if (i == 0) s0 = s;
        part += s;
    }
    for (int k = tid; k < h; k += blockDim.x) mx = fmax(mx, (double)sigma[(size_t)k * r]);
    red[tid] = part;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const double total = red[0];
    __syncthreads();
    red[tid] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
        __syncthreads();
    }
    const double smx = red[0];
    __syncthreads();
    if (out_rank) {
        const double S0 = (r > 0) ? s0 : 0.0;
        const double t = tol >= 0.0 ? tol : (double)rank_scale * 1.1920928955078125e-07 * S0;
        int cnt = 0;
        for (int i = tid; i < r; i += blockDim.x) {
            double s = 0.0;
            for (int k = 0; k < h; ++k) {
                const double w = (k == 0 || 2 * k == n3) ? 1.0 : 2.0;
                s += w * (double)sigma[(size_t)k * r + i];
            }
            cnt += (s * inv_n3 > t);
        }
        red[tid] = (double)cnt;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0) *out_rank = (int64_t)red[0];
    }
    if (tid == 0) {
        if (out_tnn) *out_tnn = total;
        if (out_tsn) *out_tsn = (r > 0 && h > 0) ? smx : 0.0;
    }
}

__global__ void diag_spectrum_kernel(const float* __restrict__ sigma, int h, int r,
                                     float2* __restrict__ Sb) {
    const int64_t total = (int64_t)h * r;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x)
        Sb[idx] = make_float2(sigma[idx], 0.f);  // tube i, frequency k at i + r*k
}

__global__ void diag_scatter_kernel(const float* __restrict__ tubes, int r, int n3,
                                    float* __restrict__ S, int64_t nS1, int64_t nS2) {
    const int64_t total = (int64_t)r * n3;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx / r, i = idx - t * r;
        S[i + nS1 * i + nS1 * nS2 * t] = tubes[idx];
    }
}

}  // namespace

bool jacobi_shape_valid(const JacobiShape& sh) {
    return sh.target_e2 >= 1 && sh.target_e2 <= 8 && sh.max_warps >= 2 && sh.max_warps <= 32 &&
           (sh.split == 0 || sh.split == 1);
}

namespace {
// Per-device shape, packed as target_e2 | max_warps << 8 | split << 16 (0 = default).
std::atomic<uint32_t> g_shape[128];

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return -1;
    return dev;
}
}  // namespace

JacobiShape jacobi_shape_current() {
    JacobiShape sh;
    const int dev = current_device();
    if (dev < 0) return sh;
    const uint32_t v = g_shape[dev].load(std::memory_order_relaxed);
    if (v == 0) return sh;
    sh.target_e2 = (int)(v & 0xff);
    sh.max_warps = (int)((v >> 8) & 0xff);
    sh.split = (int)((v >> 16) & 0xff);
    return sh;
}

void jacobi_shape_store(const JacobiShape& sh) {
    const int dev = current_device();
    if (dev < 0) return;
    const uint32_t v = (uint32_t)sh.target_e2 | ((uint32_t)sh.max_warps << 8) |
                       ((uint32_t)sh.split << 16);
    g_shape[dev].store(v, std::memory_order_relaxed);
}

bool svd_plan(int n1, int n2, int mode, SvdConfig* cfg, const JacobiShape* shape) {
    const JacobiShape sh = shape ? *shape : JacobiShape();
    const int m = n1 > n2 ? n1 : n2, n = n1 > n2 ? n2 : n1;
    if (m > TP_MAX_SVD_DIM || n < 0 || m < 1) return false;
    // lanes per column pair: little zero padding, about target_e2 float4 pairs per lane
    int lp = 32;
    double best = 1e30;
    for (int cand : {8, 16, 32}) {
        const int e2 = col_e2(m, cand);
        if (e2 > 8) continue;
        const double score =
            (double)(col_ld(m, cand) - m) / m + 0.03 * fabs(e2 - (double)sh.target_e2);
        if (score < best) { best = score; lp = cand; }
    }
    const int e2 = col_e2(m, lp);
    const int maxe2 = e2 <= 2 ? 2 : (e2 <= 4 ? 4 : 8);
    cfg->lp = lp;
    cfg->maxe = maxe2;
    const int ld = col_ld(m, lp);
    const int aux = aux_bytes(m, n);
    const int64_t gbytes = (int64_t)n * ld * sizeof(float2);
    const int64_t limit = 227 * 1024 - 1024;  // static shared + margin
    const bool sm = gbytes + aux <= limit;
    cfg->in_smem = sm;
    cfg->smem_bytes = sm ? (int)(gbytes + aux) : aux;
    // pair slots: the pairs of a round split evenly over as few passes as the warp cap allows
    // (the kernels' launch bounds: 512 threads with 8 float4 pairs per lane, else 1024)
    const int pairs = (n + 1) / 2, spw = 32 / lp;
    const int wmax = std::min(sh.max_warps, maxe2 >= 8 ? 16 : 32);
    const int passes = (pairs + wmax * spw - 1) / (wmax * spw);
    int warps = (pairs + passes * spw - 1) / (passes * spw);
    warps = warps < 2 ? 2 : warps;
    cfg->threads = 32 * warps;
    cfg->group = sh.split ? cfg->threads : 0;
    int64_t w = 0;
    if (!sm) w += (int64_t)n * ld;
    if (mode == SVD_FULL) w += (int64_t)n * n;
    cfg->work_elems = (w + 31) & ~(int64_t)31;  // keeps every slice's scratch 256-byte aligned
    return true;
}

cudaError_t launch_svd(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    if (L.njobs <= 0) return cudaSuccess;
    switch (p.mode) {
        case SVD_SIGMA: return launch_mode<SVD_SIGMA>(L, p, s);
        case SVD_PROX: return launch_mode<SVD_PROX>(L, p, s);
        case SVD_FULL: return launch_mode<SVD_FULL>(L, p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sigma_reduce(const float* sigma, int h, int r, int n3, int kind, double tol,
                                int64_t rank_scale, double* out_d, int64_t* out_i, double* s_out,
                                cudaStream_t s) {
    double* tnn = kind == 0 ? out_d : nullptr;
    double* tsn = kind == 1 ? out_d : nullptr;
    int64_t* rk = kind == 2 ? out_i : nullptr;
    double* so = kind == 2 ? s_out : nullptr;
    sigma_reduce_kernel<<<1, 256, 0, s>>>(sigma, h, r, n3, tol, rank_scale, tnn, tsn, rk, so);
    return cudaGetLastError();
}

cudaError_t launch_diag_spectrum(const float* sigma, int h, int r, float2* Sb, cudaStream_t s) {
    const int64_t total = (int64_t)h * r;
    if (total <= 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    diag_spectrum_kernel<<<blocks, 256, 0, s>>>(sigma, h, r, Sb);
    return cudaGetLastError();
}

cudaError_t launch_diag_scatter(const float* tubes, int r, int n3, float* S, int64_t nS1,
                                int64_t nS2, cudaStream_t s) {
    const int64_t total = (int64_t)r * n3;
    if (total <= 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    diag_scatter_kernel<<<blocks, 256, 0, s>>>(tubes, r, n3, S, nS1, nS2);
    return cudaGetLastError();
}

}  // namespace tp
