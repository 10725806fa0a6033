/*
 * tp.h -- C ABI of the GB300 t-product library (libtp).
 *
 * The operations are those of Lu, "Tensor-Tensor Product Toolbox" (2018), on real
 * third-order tensors, computed by the Fourier-domain method the paper describes:
 * a real DFT along every mode-3 tube that keeps the ceil((n3+1)/2) independent
 * frontal slices (Lemma 2.1, Eq. 8), one batched kernel over those slices (a
 * complex GEMM, a one-sided Jacobi SVD with one of several epilogues), and the
 * inverse DFT with the mirrored slices implied (Algorithms 1-3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.    A tensor A of size n1 x n2 x n3 is an array of n1*n2*n3 float32 values,
 *            column-major: entry A(i, j, k) (0-based) is at A[i + n1*j + n1*n2*k]
 *            (the paper's Matlab indexing, section 2.1).
 * Memory.    Every tensor or scalar pointer is a DEVICE pointer of the current CUDA
 *            device, owned by the caller; the library never frees or keeps it.
 *            Tensor pointers need 4-byte alignment; 16-byte alignment enables the
 *            vectorised paths.
 * Stream.    `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *            enqueued on it and the call returns without waiting, unless
 *            tp_options.sync is set (the default), in which case the call waits for
 *            the stream and reports device-side non-convergence.
 * Workspace. The library allocates its temporary buffers with the stream-ordered
 *            allocator (cudaMallocAsync / cudaFreeAsync on `stream`) and keeps a
 *            per-device table of DFT twiddles in static device memory, filled on the
 *            first call on each device: make that first call before any stream
 *            capture.
 * Empty.     A dimension equal to 0 is a valid empty tensor: the call writes nothing
 *            (scalar results are 0) and returns TP_OK.
 * Errors.    Arguments are checked before anything is enqueued. A negative dimension,
 *            a NULL pointer for a non-empty tensor, a negative or NaN tau or an
 *            invalid option gives TP_ERR_INVALID_ARG; inconsistent shapes give
 *            TP_ERR_SHAPE; sizes beyond the documented limits give
 *            TP_ERR_UNSUPPORTED; a failing allocation gives TP_ERR_NO_MEMORY; a CUDA
 *            launch error gives TP_ERR_CUDA. No call aborts, traps or prints.
 * Aliasing.  Inputs and outputs must not overlap, except in tp_prox_tnn, where
 *            X == Y (fully in place) is allowed.
 * Limits.    n3 <= TP_MAX_N3. For the per-slice factorisations (SVD, inverse, QR),
 *            max(n1, n2) <= TP_MAX_SVD_DIM.
 *            All counts fit in int64_t; a single tensor has fewer than 2^31 entries
 *            per frontal slice.
 */
#ifndef TP_H
#define TP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TP_MAX_N3 1024
#define TP_MAX_SVD_DIM 512

typedef enum tp_status {
    TP_OK = 0,
    TP_ERR_INVALID_ARG = 1,
    TP_ERR_SHAPE = 2,
    TP_ERR_NO_MEMORY = 3,
    TP_ERR_CUDA = 4,
    TP_ERR_NOT_CONVERGED = 5, /* a Jacobi SVD hit max_sweeps; outputs are still written */
    TP_ERR_UNSUPPORTED = 6,
    TP_ERR_SINGULAR = 7 /* tp_tinv: a Fourier slice is singular to FP32 working precision */
} tp_status;

/* Arithmetic of the tprod slice GEMMs (Algorithm 1, step 2). */
typedef enum tp_precision {
    TP_PREC_FP32 = 0,   /* plain FP32 FFMA */
    TP_PREC_3XTF32 = 1, /* tensor cores: split-TF32, three products, FP32 accumulation */
    TP_PREC_BF16X3 = 2  /* tensor cores: split-BF16, three products, FP32 accumulation */
} tp_precision;

typedef struct tp_options {
    int32_t precision;   /* tp_precision, used by tp_tprod (default TP_PREC_FP32) */
    int32_t econ;        /* tp_tsvd: 0 = full shapes of Thm. 2.2, 1 = economy shapes */
    int32_t max_sweeps;  /* Jacobi sweep cap per slice (default 30, range 1..1000; 0 = 30) */
    int32_t sync;        /* 1 (default): wait for the stream before returning and report
                            TP_ERR_NOT_CONVERGED; 0: fully asynchronous */
    double jacobi_tol;   /* rotate a column pair when |a_p^H a_q| > tol*||a_p||*||a_q||;
                            <= 0 selects 8 * 2^-23 */
    int32_t* sweeps_out; /* optional DEVICE array, one int per directly computed Fourier
                            slice (tensor-major, slice-minor): Jacobi sweeps used */
    void* const* stage_events; /* optional HOST array of TP_STAGE_EVENTS cudaEvent_t recorded
                            on `stream` for timing: [0] before the tube DFT, [1] after it,
                            [2] after the rank proposer, [3] after the sketch SVT, [4] after
                            the Jacobi / GEMM slice kernels, [5] after the inverse DFT (or final
                            reduction). Stages an operation does not run are recorded at the
                            same point as the stage before them. */
    int32_t method;      /* prox_tnn slice SVT: TP_METHOD_JACOBI (default) or TP_METHOD_LEARNED */
    int32_t* slice_flags_out; /* optional DEVICE array, one int per directly computed slice
                            (same indexing as sweeps_out): with TP_METHOD_LEARNED, 0 if the
                            sketch path finished the slice, 1 if it fell back to Jacobi */
    int32_t* sketch_width_out; /* optional DEVICE array, same indexing: the sketch width of
                            the slice's last attempt (the proposer's choice, wider after a
                            retry for an underestimated rank; 0: the slice went straight to
                            Jacobi) */
    int32_t host_parts;  /* tp_prox_tnn_batched_host: parts the batch is cut into, 1 or 2
                            (0 = 2, the default). Two parts overlap a call's copies with its
                            own kernels; one part leaves that overlap to a caller that issues
                            consecutive calls on alternating streams (their copies then overlap
                            each other's kernels, with no per-part kernel tails) */
    int32_t* counts_out; /* optional DEVICE array, same indexing as sweeps_out (prox_tnn and
                            its batched forms): #{sigma > tau} of the slice, the count of
                            Algorithm 3's kept singular values. A singular value within 1e-6
                            relative of tau is re-decided from its column norm accumulated in
                            FP64 */
    int32_t jacobi_fp64; /* 0 (default): Jacobi rotation parameters in compensated FP32;
                            1: rotation angle, cosine and sine in FP64 from the FP32 dot
                            products (GB300's FP64 rate is about 1/64 of FP32: slower, for
                            accuracy studies). Either way the convergence test of a pair whose
                            FP32 test is within a factor 2 of the tolerance is re-done in FP64 */
} tp_options;

#define TP_STAGE_EVENTS 6

/*
 * Slice SVT methods of prox_tnn (Algorithm 3, step 2).
 * TP_METHOD_JACOBI:  one-sided Jacobi SVD of every slice (the plain FP32 path).
 * TP_METHOD_LEARNED: not in the paper. A trained proposer (tp_proposer_train) predicts
 *   k = #{sigma > tau} of each slice from cheap sketch features; a randomized range finder of
 *   width k + 4 with one power iteration and a small Jacobi SVD gives the top singular
 *   triplets; the slice is accepted only if the smallest computed singular value is below
 *   tau, the kept triplets' residuals ||A r - sigma u|| (times their weight (sigma - tau)/sigma
 *   in the result) are below 1e-5 sigma_max (times sqrt(max(n1, n2) / 100) above 100 rows, the
 *   growth of the product's FP32 rounding) and the
 *   deflated matrix's norm is estimated below 0.8 tau. A slice with min(n1, n2) >= 96 that
 *   fails is sketched again (up to four times) with two more power iterations, or half again
 *   as wide (at least 4 columns more, at most 48) if the rank was underestimated; every other
 *   failed slice is recomputed by the Jacobi path. Widths up to 48; slices whose sketch
 *   buffers exceed shared memory keep them in a global scratch area of the call. Error target
 *   1e-4 relative (Frobenius) against the exact prox. A call of at least 16 slices per SM runs
 *   its sketch size classes on library streams forked from `stream` and joined back (shared
 *   by the calls on a device, like those of the Jacobi launch groups).
 */
#define TP_METHOD_JACOBI 0
#define TP_METHOD_LEARNED 1

/* Fill *opts with the defaults used when a NULL options pointer is passed. */
void tp_options_default(tp_options* opts);

/* Human-readable name of a status code (static string). */
const char* tp_status_string(tp_status status);

/* Name of the last CUDA error this thread's library calls met ("cudaSuccess" if none);
   a static string, for diagnosing TP_ERR_CUDA. */
const char* tp_last_error_string(void);

/*
 * t-product C = A * B (Def. 2.1, Eq. 9), computed as Algorithm 1: DFT of the tubes
 * of A and B, Cbar^(k) = Abar^(k) Bbar^(k) for the ceil((n3+1)/2) independent slices,
 * inverse DFT with the conjugate mirror implied.
 *   A: n1 x n2 x n3 (in), B: n2 x l x n3 (in), C: n1 x l x n3 (out).
 * opts->precision selects the slice-GEMM arithmetic.
 */
tp_status tp_tprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2,
                   int64_t l, int64_t n3, const tp_options* opts, void* stream);

/*
 * Conjugate tensor transpose (Def. 2.2) of a real tensor: AT(j, i, 0) = A(i, j, 0)
 * and AT(j, i, k) = A(i, j, n3 - k) for 0 < k < n3.
 *   A: n1 x n2 x n3 (in), AT: n2 x n1 x n3 (out).
 */
tp_status tp_tran(const float* A, float* AT, int64_t n1, int64_t n2, int64_t n3,
                  void* stream);

/*
 * t-SVD A = U * S * V^* (Thm. 2.2) by Algorithm 2: one-sided Jacobi SVD of each of the
 * ceil((n3+1)/2) independent Fourier slices (real arithmetic on the real slices 0 and
 * n3/2, so U and V come out real), the other slices implied as conjugate mirrors.
 *   Full (opts->econ == 0): U n1 x n1 x n3, S n1 x n2 x n3, V n2 x n2 x n3.
 *   Economy (opts->econ == 1): U n1 x r x n3, S r x r x n3, V n2 x r x n3,
 *   r = min(n1, n2).
 * S is f-diagonal with S(:, :, 0) decreasing (Eq. 13). U and V are unique only up to
 * the usual phase and repeated-singular-value freedom.
 */
tp_status tp_tsvd(const float* A, float* U, float* S, float* V, int64_t n1, int64_t n2,
                  int64_t n3, const tp_options* opts, void* stream);

/*
 * Tensor nuclear norm (Def. 2.9 with Eq. 14): out[0] = (1/n3) * sum over all n3 Fourier
 * slices of the sum of their singular values. `out` is a device double.
 */
tp_status tp_tnn(const float* A, double* out, int64_t n1, int64_t n2, int64_t n3,
                 const tp_options* opts, void* stream);

/*
 * Tensor spectral norm (Def. 2.8, Eq. 17): out[0] = ||bcirc(A)|| = the largest singular
 * value over the Fourier slices. `out` is a device double.
 */
tp_status tp_tsn(const float* A, double* out, int64_t n1, int64_t n2, int64_t n3,
                 const tp_options* opts, void* stream);

/*
 * Tensor tubal rank (Def. 2.7, Eq. 16): out[0] = #{i : S(i, i, 0) > tol}, with
 * S(i, i, 0) = (1/n3) sum_k sigma_i(Abar^(k)) (Eq. 14). tol < 0 selects
 * max(n1, n2) * 2^-23 * S(0, 0, 0). If s_out is not NULL it receives the
 * min(n1, n2) tensor singular values S(i, i, 0) (device doubles).
 */
tp_status tp_tubalrank(const float* A, int64_t* out, double* s_out, int64_t n1, int64_t n2,
                       int64_t n3, double tol, const tp_options* opts, void* stream);

/*
 * Proximal operator of the tensor nuclear norm (Eq. 19), X = U * S_tau * V^* (Thm. 2.3),
 * computed by Algorithm 3: singular value thresholding at tau of each independent
 * Fourier slice, the mirrored slices implied, inverse DFT.
 *   Y, X: n1 x n2 x n3. tau >= 0 (tau = 0 returns Y up to rounding). X == Y allowed.
 */
tp_status tp_prox_tnn(const float* Y, float* X, int64_t n1, int64_t n2, int64_t n3,
                      double tau, const tp_options* opts, void* stream);

/*
 * Tensor inverse (Def. 2.4): B with A * B = B * A = I (Def. 2.3). By Eq. 10 the Fourier
 * slices of B are the inverses of those of A, so each of the ceil((n3+1)/2) independent
 * slices is inverted by Gauss-Jordan elimination with partial pivoting (FP32; real arithmetic
 * on the real slices), and B is their inverse DFT with the mirror implied.
 *   A, B: n x n x n3 (n1 == n2 == n, else TP_ERR_SHAPE); n <= TP_MAX_SVD_DIM.
 * A slice whose pivot at some step is at most n * 2^-23 times the largest magnitude in that
 * slice is singular: the whole of B is then NaN and, with opts->sync, the call returns
 * TP_ERR_SINGULAR (asynchronous calls report nothing). B must not overlap A.
 */
tp_status tp_tinv(const float* A, float* B, int64_t n1, int64_t n2, int64_t n3,
                  const tp_options* opts, void* stream);

/*
 * t-QR A = Q * R (Thm. 2.4): Q orthogonal (Def. 2.5), R f-upper triangular (every frontal
 * slice upper triangular). The paper states the factorisation without an algorithm; it is
 * computed as Algorithm 2 computes the t-SVD: a Householder QR of each independent Fourier
 * slice (real arithmetic on the real slices), the mirrored slices implied, inverse DFT.
 * Every Fourier slice of R has a real non-negative diagonal, so Q and R are unique where
 * every slice has full rank (for the first min(n1, n2) columns of Q).
 *   Full (opts->econ == 0): Q n1 x n1 x n3, R n1 x n2 x n3.
 *   Economy (opts->econ == 1): Q n1 x r x n3, R r x n2 x n3, r = min(n1, n2).
 * max(n1, n2) <= TP_MAX_SVD_DIM. Q and R must not overlap A or each other.
 */
tp_status tp_tqr(const float* A, float* Q, float* R, int64_t n1, int64_t n2, int64_t n3,
                 const tp_options* opts, void* stream);

/*
 * The rank proposer of TP_METHOD_LEARNED (not in the paper): an MLP 12 -> 64 -> 64 -> 1 (ReLU,
 * FP32) per device. Its parameters are TP_PROPOSER_FLOATS floats laid out as
 * W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3, feature mean[12], feature std[12].
 *
 * tp_proposer_train: runs the plain Jacobi prox path on the given tensors (outputs are not
 *   written) to label every directly computed slice with #{sigma > tau}, computes the slice
 *   features, and fits the MLP with `steps` full-batch Adam steps (learning rate lr, weights
 *   initialised from `seed`) on the device with the library's own kernels. The fitted
 *   proposer becomes the current device's; *mse_out (host, optional) receives the final
 *   mean squared error in counts^2. Synchronous.
 * tp_proposer_get / tp_proposer_set: copy the current device's parameters out to / in from
 *   a HOST array of TP_PROPOSER_FLOATS floats (to save and restore a trained proposer).
 *   tp_proposer_get returns TP_ERR_INVALID_ARG if no proposer was trained or set.
 */
#define TP_PROPOSER_FLOATS (64 * 12 + 64 + 64 * 64 + 64 + 64 + 1 + 2 * 12)

/* One tensor of a batched call. */
typedef struct tp_tensor_desc {
    const float* in; /* device, n1 x n2 x n3 */
    float* out;      /* device, n1 x n2 x n3; may equal `in` */
    int64_t n1, n2, n3;
    double tau;
} tp_tensor_desc;

/*
 * tp_prox_tnn on `count` independent tensors of any sizes, as three launches over all
 * of them (one DFT launch, slice SVT launches grouped by slice size, one inverse-DFT
 * launch) on one stream. `descs` is a HOST array. Each tensor obeys tp_prox_tnn's rules;
 * tensors must not overlap one another. sweeps_out (if set) is indexed by the
 * concatenation, in descriptor order, of each tensor's ceil((n3+1)/2) slices.
 */
tp_status tp_prox_tnn_batched(const tp_tensor_desc* descs, int64_t count,
                              const tp_options* opts, void* stream);

/*
 * tp_prox_tnn_batched on tensors in HOST memory: descs[t].in / .out are host pointers (in may
 * equal out). The library copies the batch into one device buffer and runs the batched prox
 * on it in place in up to opts->host_parts (default 2) parts of at least 16 MiB each (cut at
 * tensor boundaries). Each
 * part is copied in, computed and copied back on its own: the copy in of part c+1 and the
 * copy back of part c-1 overlap part c's kernels. The parts' kernels run in order on one
 * library-owned compute stream per device and the copies on two more library-owned streams;
 * all of it is ordered after earlier work on `stream` and before later work on it by events.
 * Calls issued on different streams overlap one another's copies and kernels: the library's
 * stream-ordered allocations never make one caller stream wait for another. Runs of tensors that are contiguous in host memory
 * move with one copy each. The host buffers should be page-locked (cudaHostAlloc /
 * cudaHostRegister) for the copies to overlap; pageable memory works but serialises. Device
 * memory: the batch once plus the batched prox workspace of every part. With
 * opts->sync == 0 the host buffers must stay valid and untouched until `stream` reaches the
 * end of the call. stage_events [0] is recorded before the first copy and [1]..[5] after the
 * last; sweeps_out and the other per-slice outputs are device arrays indexed as in
 * tp_prox_tnn_batched. Arguments are validated as there.
 */
tp_status tp_prox_tnn_batched_host(const tp_tensor_desc* descs, int64_t count,
                                   const tp_options* opts, void* stream);

/*
 * Replayable batched prox (not in the paper): tp_prox_plan_create records the whole launch
 * sequence of tp_prox_tnn_batched on `descs` (DFT, slice SVT launches, inverse DFT; plain or
 * learned per opts->method) into a CUDA graph, with the job tables uploaded from page-locked
 * copies the plan owns; tp_prox_plan_run replays it on `stream` with no host-side planning,
 * allocation or table upload. The tensors are those of `descs` at creation: their contents
 * may change between runs, their addresses and shapes may not. The learned method reads the
 * device's current proposer at every run (it must exist at creation). opts->sync applies to
 * every run (TP_ERR_NOT_CONVERGED reported as in tp_prox_tnn_batched); stage_events must be
 * NULL. Workspace comes from the graph's own stream-ordered allocations at every replay.
 * Destroy a plan only when no run of it is pending.
 */
typedef struct tp_prox_plan tp_prox_plan;
tp_status tp_prox_plan_create(const tp_tensor_desc* descs, int64_t count, const tp_options* opts,
                              tp_prox_plan** plan);
tp_status tp_prox_plan_run(tp_prox_plan* plan, void* stream);
tp_status tp_prox_plan_destroy(tp_prox_plan* plan);

tp_status tp_proposer_train(const tp_tensor_desc* descs, int64_t count, int32_t steps, double lr,
                            uint64_t seed, double* mse_out, void* stream);
tp_status tp_proposer_get(float* host_params);
tp_status tp_proposer_set(const float* host_params);

/*
 * CTA shape of the one-sided Jacobi kernel (not in the paper; the method is Algorithm 3,
 * step 2, or the singular values of Eq. 14 and 17). The kernel runs one CTA per Fourier
 * slice; each column pair of a sweep round is rotated by a group of 8, 16 or 32 lanes, and a
 * round's n/2 disjoint pairs are spread over the CTA's warps in as few passes as its warp
 * count allows. A shape sets:
 *   target_lane_pairs: lanes per pair are chosen so that each lane holds about this many
 *     float4 pairs of the two columns, balanced against zero padding (1..8; default 5);
 *   max_warps: warps per CTA at most (2..32; default 32; 16 when a lane holds more than
 *     4 pairs, the kernel's register limit);
 *   split_launches: 1 launches slices whose CTA sizes differ separately; 0 (default) launches
 *     all slices of one kernel instantiation together at the largest CTA size among them.
 *     With TP_METHOD_LEARNED the Jacobi launches (only the slices the sketch path rejects)
 *     are never split.
 * With several launches, the Jacobi method runs the first on `stream` and the others on
 * library streams forked from it and joined back before the call's next step (the library
 * creates these streams once per device; concurrent calls on one device share them).
 * The current device's shape applies to the Jacobi launches of tp_prox_tnn, tp_prox_tnn_batched,
 * tp_prox_tnn_batched_host, plans created while it is set, tp_proposer_train, tp_tnn, tp_tsn
 * and tp_tubalrank; tp_tsvd and tp_prox_tnn_noalloc always use the default. Results under
 * different shapes differ only by rounding order.
 *
 * tp_jacobi_shape_get / tp_jacobi_shape_set: read or replace the current device's shape (HOST
 *   struct; set(NULL) restores the default; an out-of-range field gives TP_ERR_INVALID_ARG).
 *   Not safe to call while another host thread launches work on the same device.
 * tp_autotune_jacobi: the autotuner. It computes the Fourier slices of `descs` (the tensors are
 *   read, never written; rules of tp_prox_tnn_batched) and times the batched prox's Jacobi
 *   launches on them under 18 candidate shapes (target_lane_pairs 3, 5, 7 x max_warps 8, 16,
 *   32 x split_launches 0, 1), each once untimed and then `reps` (1..100) times with CUDA events
 *   on `stream`, and makes the fastest the current device's shape (the default wins ties).
 *   *chosen (HOST, required) receives it; ms_out (HOST, optional, 2 doubles) receives the
 *   default shape's and the chosen shape's time per pass over the batch in milliseconds.
 *   Synchronous. Device memory: the batch's half spectra twice plus the Jacobi workspace.
 *   A batch without any non-empty tensor gives TP_ERR_INVALID_ARG.
 */
typedef struct tp_jacobi_shape {
    int32_t target_lane_pairs;
    int32_t max_warps;
    int32_t split_launches;
} tp_jacobi_shape;
tp_status tp_jacobi_shape_get(tp_jacobi_shape* shape);
tp_status tp_jacobi_shape_set(const tp_jacobi_shape* shape);
tp_status tp_autotune_jacobi(const tp_tensor_desc* descs, int64_t count, int32_t reps,
                             tp_jacobi_shape* chosen, double* ms_out, void* stream);

/*
 * tp_prox_tnn without any device allocation. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run -- for instance code
 * that must not trigger the implicit synchronisation or the latency of an allocator call
 * inside a time-critical loop, or a process whose device memory is handed out by another
 * framework's allocator so that the library may not obtain any of its own.
 *
 * It computes exactly what tp_prox_tnn computes with TP_METHOD_JACOBI, with the same kernels,
 * but all scratch (the half spectrum, the per-slice job records and the status word) lives in
 * one file-scope static device array of TP_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that
 * loads the library holds until the process exits. With h = n3/2 + 1 and R(x) = x rounded up
 * to a multiple of 256, a tensor fits when
 *   R(512 + h * TP_NOALLOC_JOB_BYTES) + R(8 * n1 * n2 * h) + R(8 * W * h) <= 16 MiB,
 * where W = 0 when a slice's working matrix fits in shared memory (min(n1,n2) * ld complex
 * values, ld = max(n1,n2) rounded up to a multiple of 16, 32 or 64, below about 226 KB) and
 * W = min(n1,n2) * ld rounded up to a multiple of 32 otherwise. Larger tensors are rejected
 * with TP_ERR_UNSUPPORTED before anything is enqueued. The call never calls cudaMalloc,
 * cudaFree or any allocating routine.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * and fills the twiddle table, with that device current; make it before any stream capture.
 * All calls share the one array and it keeps the last call's contents (the status word is
 * cleared at the start of every call): calls that overlap on the GPU -- on different
 * streams, or from several host threads without ordering -- race and must not be issued.
 * Arguments, errors and aliasing (X == Y allowed) are those of tp_prox_tnn. Options are
 * checked as there; in addition method must be TP_METHOD_JACOBI and stage_events,
 * slice_flags_out and sketch_width_out must be NULL (TP_ERR_INVALID_ARG otherwise).
 * sweeps_out and counts_out (h entries each) are written; precision, econ and host_parts
 * have no effect.
 */
#define TP_NOALLOC_SCRATCH_BYTES (16u << 20)
#define TP_NOALLOC_JOB_BYTES 128
tp_status tp_prox_tnn_noalloc(const float* Y, float* X, int64_t n1, int64_t n2, int64_t n3,
                              double tau, const tp_options* opts, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TP_H */
