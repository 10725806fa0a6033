// Internal declarations shared by the translation units of libtp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tp.h"

namespace tp {

// Number of Fourier slices computed directly: ceil((n3+1)/2) = floor(n3/2)+1
// (Algorithms 1-3); slices k >= h are conjugate mirrors of slice n3-k (Eq. 8).
inline __host__ __device__ int free_slices(int n3) { return n3 / 2 + 1; }

// Slice 0 and, for even n3, slice n3/2 are real matrices (Eq. 8).
inline __host__ __device__ bool is_real_slice(int k, int n3) {
    return k == 0 || (2 * k == n3);
}

// ---------------------------------------------------------------------------
// Tube DFTs (tp_fft.cu)
// ---------------------------------------------------------------------------
// One tensor's tubes: x is P tubes x n3 samples (tube p, sample t at x[p + P*t]),
// X is P tubes x h complex frequencies (X[p + P*k]).
struct FftJob {
    const float* x = nullptr;  // rfft: input; irfft: output (written)
    float2* X = nullptr;       // rfft: output; irfft: input
    int64_t P = 0;             // tubes (n1*n2)
    int32_t n3 = 0;
    int32_t tile_begin = 0;    // first CTA of this job in the launch
    // Forward DFT only, power-of-two n3 <= 64: with plane_kind != 0 the spectrum is written,
    // instead of to X, as the BF16 hi/lo operand planes of the tensor-core slice GEMM
    // (PLANE_LEFT / PLANE_RIGHT below; plane_rows = M or K, plane_pitch = the row pitch).
    uint16_t* plane_hi = nullptr;
    uint16_t* plane_lo = nullptr;
    int64_t plane_pitch = 0;
    int32_t plane_kind = 0;
    int32_t plane_rows = 0;
};

// BF16x3 operand planes of the tensor-core slice GEMM C_z = A_z B_z (A_z M x K, B_z K x N,
// complex), each value x stored as hi = bf16(x) and lo = bf16(x - hi) in two planes of the
// same layout.  Rows have `pitch` elements (a multiple of 8, so that every row starts on a
// 16-byte boundary); nothing beyond M or K is ever read, the GEMM's tensor maps zero-fill.
//   PLANE_LEFT  (A, MN-major):  Re A_z(m, k) at ((2z + 0) K + k) pitch + m,
//                               Im A_z(m, k) at ((2z + 1) K + k) pitch + m.
//   PLANE_RIGHT (B, K-major, the rows of the real form [Br -Bi; Bi Br] interleaved so that
//                output columns 2n and 2n+1 are Re and Im of C(:, n)):
//                               part 0, rows 2n / 2n+1:  Re B_z(k, n) / Im B_z(k, n),
//                               part 1, rows 2n / 2n+1: -Im B_z(k, n) / Re B_z(k, n),
//                               at ((2z + part) 2N + row) pitch + k.
enum : int32_t { PLANE_NONE = 0, PLANE_LEFT = 1, PLANE_RIGHT = 2 };

// Fills the per-device twiddle table on first use; returns cudaSuccess or the error.
cudaError_t ensure_twiddles();

// Forward real DFT of every tube, frequencies 0..h-1 (unnormalised, Eq. 2).  uniform_n3 is
// the common n3 of all jobs of the launch, or 0 when they differ.  On the small-n3 path
// (fft_small_path) a launch holds jobs of one register class (fft_small_class), given as
// small_cls (-1: the class of uniform_n3).
// `planes`: the jobs write BF16x3 operand planes (plane_kind != 0); the launch must then
// satisfy fft_writes_planes(uniform_n3).
cudaError_t launch_rfft(const FftJob* d_jobs, int njobs, int total_tiles, int max_n3,
                        int uniform_n3, bool vec_ok, cudaStream_t s, int small_cls = -1,
                        bool planes = false);
// Inverse DFT from the half spectrum with the conjugate mirror implied, scaled by 1/n3.
cudaError_t launch_irfft(const FftJob* d_jobs, int njobs, int total_tiles, int max_n3,
                         int uniform_n3, bool vec_ok, cudaStream_t s, int small_cls = -1);
// True when a forward DFT of tubes of length n3 (all of one length) can write the BF16x3
// operand planes itself (FftJob::plane_kind).
bool fft_writes_planes(int n3);
// True when launches over jobs with these lengths use the per-length kernels for n3 <= 64.
bool fft_small_path(int max_n3, int uniform_n3);
// Register class (0, 1, 2) of the per-length kernel of n3 <= 64.
int fft_small_class(int n3);
// CTAs one job of length n3 needs (tubes per CTA depend on the kernel the launch uses).
int fft_tiles(int64_t P, int max_n3, int uniform_n3, int n3);

// ---------------------------------------------------------------------------
// Slice GEMMs (tp_gemm.cu): C_k = A_k B_k for k < nslices, complex, column-major.
// ---------------------------------------------------------------------------
cudaError_t launch_cgemm_fp32(const float2* A, const float2* B, float2* C, int M, int N, int K,
                              int64_t sA, int64_t sB, int64_t sC, int nslices, cudaStream_t s);

// Tensor-core path (tp_gemm_tc.cu): split-precision planes (bytes below, in `planes`) and the
// tcgen05 GEMM; `err` (device, zeroed by the caller) receives a non-zero bit on a timeout.
int64_t cgemm_tc_plane_bytes(int M, int N, int K, int nslices, int precision);
cudaError_t launch_cgemm_tc(const float2* A, const float2* B, float2* C, int M, int N, int K,
                            int nslices, int precision, void* planes, uint32_t* err,
                            cudaStream_t s);
// BF16x3 path on the operand planes above.  `planes` holds, in order, A's hi and lo planes
// (bf16_left_plane_elems each) and B's hi and lo planes (bf16_right_plane_elems each).
// bf16_planes_from_spectrum fills them from complex spectra A (M x K x nslices) and B
// (K x N x nslices) when the forward DFT has not written them itself.  n3 marks the real
// slices (0 and n3 / 2), whose second K half is zero and is skipped.
int64_t bf16_plane_pitch(int rows);
int64_t bf16_left_plane_elems(int M, int K, int nslices);
int64_t bf16_right_plane_elems(int N, int K, int nslices);
cudaError_t bf16_planes_from_spectrum(const float2* A, const float2* B, int M, int N, int K,
                                      int nslices, void* planes, cudaStream_t s);
cudaError_t launch_cgemm_bf16x3(const void* planes, float2* C, int M, int N, int K, int nslices,
                                int n3, uint32_t* err, cudaStream_t s);

// ---------------------------------------------------------------------------
// Slice SVDs (tp_svd.cu)
// ---------------------------------------------------------------------------
enum SvdMode : int32_t { SVD_SIGMA = 0, SVD_PROX = 1, SVD_FULL = 2 };

// Every field has a default so that a record built field by field (on the host or on the
// device) never carries an indeterminate pointer.
struct SvdJob {
    const float2* A = nullptr;   // Fourier slice, n1 x n2, column-major, ld n1
    float2* W = nullptr;         // PROX: output slice (may equal A); FULL: Ubar (n1 x ucols)
    float2* Vout = nullptr;      // FULL: Vbar slice (n2 x vcols)
    float2* work = nullptr;      // global scratch: FULL needs n*n (V_G); big slices need m*n (G)
    float* sigma = nullptr;      // min(n1,n2) singular values, decreasing (SIGMA, FULL)
    int32_t n1 = 0, n2 = 0;
    int32_t real_slice = 0;      // 1 for the real slices of Eq. 8
    int32_t ucols = 0, vcols = 0;  // FULL: columns of U and V to produce
    int32_t sweeps_index = -1;   // index into sweeps_out, or -1
    double tau = 0.0;            // PROX threshold
    const int32_t* skip = nullptr;  // if set and *skip == 0 the slice is already done (sketch)
    int32_t* count_out = nullptr;   // PROX: receives #{sigma > tau} if set
};

struct SvdLaunch {
    const SvdJob* jobs;  // device array
    int njobs;
    int lp;              // lanes per column pair (8, 16, 32)
    int maxe;            // elements per lane: m <= lp*maxe
    bool in_smem;        // working matrix in shared memory
    int smem_bytes;
    int threads;
};

// Launch configuration of one slice size (see svd_plan).
struct SvdConfig {
    int lp, maxe, smem_bytes, threads;
    bool in_smem;
    int64_t work_elems;  // global scratch elements (float2) per slice
    int group = 0;       // > 0: slices launch only with slices of the same group (CTA size)
};

// CTA shape policy of the Jacobi kernel (tp_jacobi_shape of tp.h): lanes per column pair are
// picked so that each lane holds about `target_e2` float4 pairs, the CTA has at most
// `max_warps` warps (the pairs of a round are spread over passes of that many warps), and
// with `split` set, slices whose CTA sizes differ are launched separately instead of sharing
// the largest CTA of their kernel instantiation.  The default reproduces the fixed choice.
struct JacobiShape {
    int target_e2 = 5;
    int max_warps = 32;
    int split = 0;
};
bool jacobi_shape_valid(const JacobiShape& sh);
// The current device's shape (the default until tp_jacobi_shape_set / tp_autotune_jacobi).
JacobiShape jacobi_shape_current();
void jacobi_shape_store(const JacobiShape& sh);

struct SvdParams {
    int mode;
    int max_sweeps;
    float tol;           // <= 0: default per slice
    int32_t* sweeps_out; // device, may be null
    uint32_t* status;    // device status word (bit 0: not converged)
    int fp64_rotation = 0;  // 1: rotation parameters in FP64 (tp_options.jacobi_fp64)
};

// Checks a tp_options record as every entry point does (TP_OK or TP_ERR_INVALID_ARG).
tp_status validate_options(const tp_options* o);

// Which launch configuration a slice of size n1 x n2 needs under `shape` (NULL: default).
bool svd_plan(int n1, int n2, int mode, SvdConfig* cfg, const JacobiShape* shape = nullptr);
cudaError_t launch_svd(const SvdLaunch& L, const SvdParams& p, cudaStream_t s);

// Reductions over the sorted singular values of one tensor (tnn, tsn, tubal rank).
cudaError_t launch_sigma_reduce(const float* sigma, int h, int r, int n3, int kind, double tol,
                                int64_t rank_scale, double* out_d, int64_t* out_i, double* s_out,
                                cudaStream_t s);
// S(i, i, t) tubes from the singular values: S is nS1 x nS2 x n3 (zeroed by the caller).
cudaError_t launch_diag_spectrum(const float* sigma, int h, int r, float2* Sbar_diag,
                                 cudaStream_t s);
cudaError_t launch_diag_scatter(const float* tubes, int r, int n3, float* S, int64_t nS1,
                                int64_t nS2, cudaStream_t s);

// ---------------------------------------------------------------------------
// Learned-rank randomized SVT (tp_sketch.cu)
// ---------------------------------------------------------------------------
constexpr int kSketchMaxL = 48;        // widest sketch
constexpr int kNarrowL = 32;           // widest sketch of the shared-memory classes
constexpr int kProposerInputs = 12;    // features per slice
constexpr int kProposerFloats = TP_PROPOSER_FLOATS;

struct SketchParams {
    const int32_t* order = nullptr;  // CTA (or queue position) -> job index (nullptr: identity)
    const int32_t* queue_len = nullptr;  // persistent mode: number of entries of `order`
    int32_t* queue_next = nullptr;       // persistent mode: work counter (zero at launch)
    int32_t* ell;         // per job: sketch width (0: go to the full Jacobi SVD); a wider
                          // retry raises it
    int32_t* flag;        // per job: 0 = W written by the sketch path, 1 = needs Jacobi
    int32_t* count;       // per job: #{sigma > tau} on success (optional)
    uint32_t seed;
    int power_iters;
    int njobs = 0;                   // jobs in the launch's job array (bounds queue entries)
    int32_t* extra_power = nullptr;  // per job: extra power iterations of a retry
    int retry_launch = 0;            // 1: `order` is a retry list (per-slice power iterations)
    float resid_tol;
    int smem_bytes;       // dynamic shared memory of the launch
    int wide = 0;                // 1: widths up to kSketchMaxL (the last class; retries are wide)
    float2* gscratch = nullptr;  // if set: the three tall buffers of CTA b at gscratch + b * gstride
    int64_t gstride = 0;         // (complex values), the rest in shared memory
};

// Shared memory of the sketch of one slice without its three max(n1, n2) x l buffers.
__host__ __device__ inline size_t sketch_small_need(int n1, int n2, int l) {
    return sizeof(float2) * ((size_t)3 * l * l + (size_t)n1 + n2 + 2 * kSketchMaxL) +
           sizeof(float) * (2 * kSketchMaxL) + 64;
}
// ... and with them.
__host__ __device__ inline size_t sketch_smem_need(int n1, int n2, int l) {
    const size_t nm = n1 > n2 ? n1 : n2;
    return sizeof(float2) * 3 * nm * l + sketch_small_need(n1, n2, l);
}
// Retry rounds of the sketch path (each: collect the failed slices, sketch them again).
constexpr int kSketchRetryRounds = 4;
// Size classes of the sketch kernel's queues: shared memory bytes per CTA, increasing.
// Classes 0..3 hold everything in shared memory; the last class keeps the three tall buffers
// in global memory (slices larger than the largest shared-memory class).
constexpr int kSketchClasses = 5;
constexpr uint32_t kSketchSmemCap = 220 * 1024;  // the largest shared-memory class
struct SketchCaps {
    int n;
    uint32_t bytes[kSketchClasses];
};
// Bins the slices (in the order of `sorted`) into one queue per class; see tp_sketch.cu.
cudaError_t launch_sketch_bin(const SvdJob* jobs, const int32_t* sorted, int n, const int32_t* ell,
                              int32_t* flag, const SketchCaps& caps, int32_t* queues,
                              int32_t* counts, cudaStream_t s);
// Queues the failed slices worth another sketch (see tp_sketch.cu) into `list`.
cudaError_t launch_sketch_collect(const SvdJob* jobs, int n, int32_t* flag, int32_t* ell,
                                  int32_t* extra, int min_dim, int smem, int64_t gstride,
                                  int32_t* list, int32_t* len, cudaStream_t s);
// out[j] = (flags[j] != 0): the per-slice fallback flags as 0 / 1.
cudaError_t launch_flags01(const int32_t* flags, int32_t* out, int n, cudaStream_t s);
// Resident CTAs of the sketch kernel per SM at this dynamic shared memory (0 on error).
int sketch_blocks_per_sm(size_t smem);
size_t features_smem_bytes(int n1, int n2);
cudaError_t launch_features(const SvdJob* jobs, int njobs, int max_n1, int max_n2, float* feat,
                            uint32_t seed, cudaStream_t s);
cudaError_t launch_proposer(const float* feat, const SvdJob* jobs, int njobs, int32_t* ell,
                            cudaStream_t s);
cudaError_t launch_sketch_svt(const SvdJob* jobs, int ncta, size_t smem, const SketchParams& p,
                              cudaStream_t s);
bool proposer_ready();
cudaError_t proposer_set(const float* host);
cudaError_t proposer_get(float* host);
cudaError_t proposer_fit(const float* d_feat, const int32_t* d_count, int n, int steps, float lr,
                         uint64_t seed, float* scratch, double* mse, cudaStream_t s);
size_t proposer_fit_scratch_floats(int n);

// ---------------------------------------------------------------------------
// Transpose (tp_tran.cu)
// ---------------------------------------------------------------------------
// Per-slice factorisations (tp_slice_la.cu): one CTA per independent Fourier slice.
// ---------------------------------------------------------------------------
struct LaJob {
    float2* A = nullptr;  // slice (column-major, leading dimension n1); overwritten
    float2* Q = nullptr;  // tqr: Q (n1 x qcols, leading dimension n1)
    float2* R = nullptr;  // tqr: R (rrows x n2, leading dimension rrows); tinv: the inverse
                          // (must equal A)
    int32_t n1 = 0, n2 = 0, qcols = 0, rrows = 0;
};

// Shared memory one CTA may use; larger slices work in global memory.
constexpr size_t kLaSmemLimit = 227 * 1024;

// Inverse of every n x n slice (Def. 2.4); a singular slice is filled with NaN and sets bit 2
// of *status.
cudaError_t launch_tinv(const LaJob* d_jobs, int njobs, int n, uint32_t* status, cudaStream_t s);
// QR of every n1 x n2 slice with the diagonal of R real and non-negative (Thm. 2.4).
cudaError_t launch_tqr(const LaJob* d_jobs, int njobs, int n1, int n2, int qcols, cudaStream_t s);

// ---------------------------------------------------------------------------
cudaError_t launch_tran(const float* A, float* AT, int64_t n1, int64_t n2, int64_t n3,
                        cudaStream_t s);

}  // namespace tp
