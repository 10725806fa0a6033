// The learned rank proposer of the learned prox_tnn path (not in the paper): for each Fourier
// slice A (n1 x n2 complex, in place in the half spectrum) a tiny MLP (12 -> 64 -> 64 -> 1,
// ReLU) reads cheap sketch features -- log ||A||_F / tau, the diagonal of the QR factor of an
// 8-column sketch A Omega_8 over tau, log n1, log n2, log min(n1, n2) -- and predicts
// k = #{sigma > tau}, the number of singular values Algorithm 3 keeps; the randomized SVT
// (tp_sketch_svt.cu) then sketches the slice with width l = k + 4.  The MLP is trained with
// hand-written forward/backward and Adam kernels on (features, #{sigma > tau}) pairs that the
// plain Jacobi path produces.
#include <math.h>

#include <mutex>
#include <vector>

#include "tp_internal.cuh"
#include "tp_rotation.cuh"
#include "tp_sketch.cuh"

namespace tp {

namespace {

constexpr int kT = 256;   // threads per CTA of the feature and training kernels
constexpr int kLMax = kSketchMaxL;
constexpr int kD = kProposerInputs;
constexpr int kH = 64;
constexpr int kW1 = 0, kB1 = kW1 + kH * kD, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kH, kMean = kB3 + 1, kStd = kMean + kD, kNParams = kMean;
static_assert(kStd + kD == kProposerFloats, "proposer layout");

// Per-device proposer: weights, biases and the feature standardisation.
__device__ float g_proposer[kProposerFloats];

using sk::ld_a;
using sk::omega;
using sk::warp_sum;

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

// Proposer inference: one thread per slice, ell = clamp(ceil(k_hat) + 4).
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

__global__ void flags01_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = in[j] != 0 ? 1 : 0;
}

cudaError_t launch_flags01(const int32_t* flags, int32_t* out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    flags01_kernel<<<(n + 255) / 256, 256, 0, s>>>(flags, out, n);
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
