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
// columns: n' - 1 rounds of n'/2 disjoint pairs; pairs of a round go to different warps,
// a warp holds its two columns in registers (MAXE elements per lane) between the dot
// products and the update.  A sweep with no rotation ends the iteration.
//
// Working storage.  G lives in shared memory (row stride m rounded up to odd, which keeps
// the 64-bit accesses of a warp free of bank conflicts) when it fits, otherwise in a
// global scratch area of the slice.  SVD_FULL accumulates V in global scratch.
//
// The SVT epilogue needs no V: u_j = b_j / sigma_j and v_j^* = b_j^* A_G / sigma_j^2,
// so W_G = sum_{sigma_j > tau} ((sigma_j - tau) / sigma_j) (1/sigma_j^2) b_j (b_j^* g_c)
// column by column, re-reading the original column g_c of the slice.
#include <math.h>

#include "tp_internal.cuh"

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

// One Jacobi rotation of columns gp, gq (length m) and, for SVD_FULL, of the
// accumulated V columns vp, vq (length nv).  Returns true if the pair was rotated.
template <int MAXE, bool WITH_V>
__device__ __forceinline__ bool jacobi_pair(float2* gp, float2* gq, int m, int lane, float tol,
                                            float2* vp, float2* vq, int nv) {
    float2 xp[MAXE], xq[MAXE];
    float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
    for (int i = 0; i < MAXE; ++i) {
        const int e = lane + 32 * i;
        if (e < m) {
            xp[i] = gp[e];
            xq[i] = gq[e];
        } else {
            xp[i] = make_float2(0.f, 0.f);
            xq[i] = make_float2(0.f, 0.f);
        }
        al = fmaf(xp[i].x, xp[i].x, fmaf(xp[i].y, xp[i].y, al));
        be = fmaf(xq[i].x, xq[i].x, fmaf(xq[i].y, xq[i].y, be));
        gr = fmaf(xp[i].x, xq[i].x, fmaf(xp[i].y, xq[i].y, gr));
        gi = fmaf(xp[i].x, xq[i].y, fmaf(-xp[i].y, xq[i].x, gi));
    }
    al = warp_sum(al);
    be = warp_sum(be);
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    const float ag = sqrtf(fmaf(gr, gr, gi * gi));
    if (!(ag > tol * sqrtf(al) * sqrtf(be))) return false;
    const float zeta = (be - al) / (2.f * ag);
    const float az = fabsf(zeta);
    float t = (az > 1e8f) ? 0.5f / az : 1.f / (az + sqrtf(fmaf(zeta, zeta, 1.f)));
    t = copysignf(t, zeta);
    const float c = 1.f / sqrtf(fmaf(t, t, 1.f));
    const float s = c * t;
    const float er = gr / ag, ei = gi / ag;
#pragma unroll
    for (int i = 0; i < MAXE; ++i) {
        const int e = lane + 32 * i;
        if (e < m) {
            const float2 a = xp[i], b = xq[i];
            const float cbx = fmaf(er, b.x, ei * b.y), cby = fmaf(er, b.y, -ei * b.x);  // conj(e) b
            const float eax = fmaf(er, a.x, -ei * a.y), eay = fmaf(er, a.y, ei * a.x);  // e a
            gp[e] = make_float2(fmaf(c, a.x, -s * cbx), fmaf(c, a.y, -s * cby));
            gq[e] = make_float2(fmaf(s, eax, c * b.x), fmaf(s, eay, c * b.y));
        }
    }
    if (WITH_V) {
        for (int e = lane; e < nv; e += 32) {
            const float2 a = vp[e], b = vq[e];
            const float cbx = fmaf(er, b.x, ei * b.y), cby = fmaf(er, b.y, -ei * b.x);
            const float eax = fmaf(er, a.x, -ei * a.y), eay = fmaf(er, a.y, ei * a.x);
            vp[e] = make_float2(fmaf(c, a.x, -s * cbx), fmaf(c, a.y, -s * cby));
            vq[e] = make_float2(fmaf(s, eax, c * b.x), fmaf(s, eay, c * b.y));
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

__host__ __device__ inline int odd_ld(int m) { return m | 1; }

template <int MODE, int MAXE, bool SMEM>
__global__ void __launch_bounds__(kMaxThreads, 1) svd_kernel(const SvdJob* __restrict__ jobs,
                                                              SvdParams prm) {
    extern __shared__ float4 smem4[];
    __shared__ int s_rot, s_cnt;
    const SvdJob J = jobs[blockIdx.x];
    const int n1 = J.n1, n2 = J.n2;
    const bool tr = n1 < n2;
    const int m = tr ? n2 : n1, n = tr ? n1 : n2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int T = blockDim.x;
    const bool real = J.real_slice != 0;

    const int ld = SMEM ? odd_ld(m) : m;
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
    if (MODE == SVD_FULL) VG = SMEM ? J.work : J.work + (size_t)m * n;

    // ---- load G (= A or A^H) -------------------------------------------------
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
    const float tol = prm.tol > 0.f ? prm.tol : fmaxf(8.f, sqrtf((float)m)) * kEps;
    const int N = n + (n & 1);
    int sweeps = 0;
    bool converged = n < 2;
    while (!converged && sweeps < prm.max_sweeps) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < N - 1; ++r) {
            for (int pi = warp; pi < N / 2; pi += nw) {
                int a, b;
                if (pi == 0) { a = N - 1; b = r; }
                else { a = (r + pi) % (N - 1); b = (r - pi + N - 1) % (N - 1); }
                if (a >= n || b >= n) continue;
                const int p = min(a, b), q = max(a, b);
                bool did = jacobi_pair<MAXE, MODE == SVD_FULL>(
                    G + (size_t)p * ld, G + (size_t)q * ld, m, lane, tol,
                    MODE == SVD_FULL ? VG + (size_t)p * n : nullptr,
                    MODE == SVD_FULL ? VG + (size_t)q * n : nullptr, n);
                if (did && lane == 0) s_rot = 1;
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
    for (int c = warp; c < n; c += nw) {
        const float2* g = G + (size_t)c * ld;
        float s = 0.f;
        for (int e = lane; e < m; e += 32) s = fmaf(g[e].x, g[e].x, fmaf(g[e].y, g[e].y, s));
        s = warp_sum(s);
        if (lane == 0) sig[c] = sqrtf(s);
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
        // kept set {sigma_j > tau}, decided in FP64, in column order (ballot compaction)
        for (int c = tid; c < n; c += T) {
            const double sd = (double)sig[c];
            const int f = sd > J.tau;
            flag[c] = f;
            if (f) {
                ratio[c] = (float)((sd - J.tau) / sd);
                invs[c] = 1.f / sig[c];
            }
        }
        __syncthreads();
        if (warp == 0) {
            int cnt = 0;
            for (int base = 0; base < n; base += 32) {
                const int c = base + lane;
                const int f = (c < n) ? flag[c] : 0;
                const unsigned mask = __ballot_sync(0xffffffffu, f);
                if (f) kept[cnt + __popc(mask & ((1u << lane) - 1u))] = c;
                cnt += __popc(mask);
            }
            if (lane == 0) s_cnt = cnt;
        }
        __syncthreads();
        const int cnt = s_cnt;
        // W_G(:, c) = sum_k ratio_k invs_k^2 b_k (b_k^H g_c), g_c re-read from the slice
        for (int c = warp; c < n; c += nw) {
            float2 a[MAXE], w[MAXE];
#pragma unroll
            for (int i = 0; i < MAXE; ++i) {
                const int e = lane + 32 * i;
                float2 v = make_float2(0.f, 0.f);
                if (e < m) {
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
                    const int e = lane + 32 * i;
                    if (e < m) {
                        const float2 bv = b[e];
                        dr = fmaf(bv.x, a[i].x, fmaf(bv.y, a[i].y, dr));
                        di = fmaf(bv.x, a[i].y, fmaf(-bv.y, a[i].x, di));
                    }
                }
                dr = warp_sum(dr);
                di = warp_sum(di);
                const float sc = ratio[j] * invs[j] * invs[j];
                dr *= sc;
                di *= sc;
#pragma unroll
                for (int i = 0; i < MAXE; ++i) {
                    const int e = lane + 32 * i;
                    if (e < m) {
                        const float2 bv = b[e];
                        w[i].x = fmaf(dr, bv.x, fmaf(-di, bv.y, w[i].x));
                        w[i].y = fmaf(dr, bv.y, fmaf(di, bv.x, w[i].y));
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < MAXE; ++i) {
                const int e = lane + 32 * i;
                if (e < m) {
                    float2 v = w[i];
                    if (real) v.y = 0.f;
                    if (tr) J.W[c + (int64_t)n1 * e] = make_float2(v.x, -v.y);
                    else J.W[e + (int64_t)n1 * c] = v;
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

template <int MODE, int MAXE, bool SMEM>
cudaError_t launch_one(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    auto k = svd_kernel<MODE, MAXE, SMEM>;
    if (L.smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L.smem_bytes);
        if (e != cudaSuccess) return e;
    }
    k<<<L.njobs, L.threads, L.smem_bytes, s>>>(L.jobs, p);
    return cudaGetLastError();
}

template <int MODE, bool SMEM>
cudaError_t launch_maxe(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    switch (L.maxe) {
        case 1: return launch_one<MODE, 1, SMEM>(L, p, s);
        case 2: return launch_one<MODE, 2, SMEM>(L, p, s);
        case 3: return launch_one<MODE, 3, SMEM>(L, p, s);
        case 4: return launch_one<MODE, 4, SMEM>(L, p, s);
        case 5: return launch_one<MODE, 5, SMEM>(L, p, s);
        case 8: return launch_one<MODE, 8, SMEM>(L, p, s);
        case 16: return launch_one<MODE, 16, SMEM>(L, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int MODE>
cudaError_t launch_mode(const SvdLaunch& L, const SvdParams& p, cudaStream_t s) {
    return L.in_smem ? launch_maxe<MODE, true>(L, p, s) : launch_maxe<MODE, false>(L, p, s);
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

bool svd_plan(int n1, int n2, int mode, int* maxe, bool* in_smem, int* smem_bytes, int* threads,
              int64_t* work_elems) {
    const int m = n1 > n2 ? n1 : n2, n = n1 > n2 ? n2 : n1;
    if (m > TP_MAX_SVD_DIM || n < 0) return false;
    const int need = (m + 31) / 32;
    int e = need <= 5 ? (need < 1 ? 1 : need) : (need <= 8 ? 8 : 16);
    *maxe = e;
    const int aux = aux_bytes(m, n);
    const int64_t gbytes = (int64_t)n * odd_ld(m) * sizeof(float2);
    const int64_t limit = 227 * 1024 - 1024;  // static shared + margin
    const bool sm = gbytes + aux <= limit;
    *in_smem = sm;
    *smem_bytes = sm ? (int)(gbytes + aux) : aux;
    const int pairs = (n + 1) / 2;
    *threads = pairs >= 24 ? 512 : (pairs >= 8 ? 256 : 128);
    if (e >= 8 && *threads > 256) *threads = 256;
    int64_t w = 0;
    if (!sm) w += (int64_t)m * n;
    if (mode == SVD_FULL) w += (int64_t)n * n;
    *work_elems = w;
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
