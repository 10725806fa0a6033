// tp_prox_tnn_noalloc: the prox_tnn pipeline (tube DFT -> slice SVT -> inverse DFT) with all
// of its scratch in one fixed, statically sized device array instead of the stream-ordered
// allocator, for callers that cannot allocate device memory during a call.
//
// The array below is a file-scope __device__ symbol: every GPU that loads the library holds
// TP_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code cannot use the symbol
// name as a device address, so the first call on each device (with that device current)
// looks the address up once with cudaGetSymbolAddress and caches it; later calls reuse it.
// Make that first call before any stream capture.
//
// Scratch layout (offsets in bytes): [0, 256) status word, [256, 512) the two DFT job
// records, then room for TP_NOALLOC_JOB_BYTES per slice of SVD job records (rounded up to
// 256), then the half spectrum (and, for slices that do not fit in shared memory, their
// working matrices).  The job records are written
// by a small kernel, so a call issues no host-to-device copy either.  Every call reuses the
// same array and it keeps the previous call's contents: the status word is cleared at the
// start of each call, everything else is fully rewritten before it is read.  Two calls
// that overlap on the GPU (different streams, or different host threads without ordering)
// race on the array.
#include <mutex>

#include "tp_internal.cuh"

namespace tp {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TP_NOALLOC_SCRATCH_BYTES];

constexpr size_t kStatusOff = 0;
constexpr size_t kFftOff = 256;
constexpr size_t kSvdOff = 512;
static_assert(sizeof(SvdJob) <= TP_NOALLOC_JOB_BYTES, "job record budget of tp.h");
static_assert(2 * sizeof(FftJob) <= kSvdOff - kFftOff, "DFT job records");

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

std::mutex g_mutex;
void* g_base[128] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}

// Fills the two DFT job records and the h SVD job records inside the scratch array.
__global__ void noalloc_jobs_kernel(FftJob* fft, SvdJob* svd, const float* Y, float* X,
                                    float2* spec, float2* work, int64_t work_elems, int n1,
                                    int n2, int n3, double tau, int with_sweeps,
                                    int32_t* counts_out) {
    const int64_t P = (int64_t)n1 * n2;
    const int h = free_slices(n3);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        FftJob f;  // every field from its default (the array keeps the previous call's bytes)
        f.x = Y;
        f.X = spec;
        f.P = P;
        f.n3 = n3;
        f.tile_begin = 0;
        fft[0] = f;
        f.x = X;
        fft[1] = f;
    }
    if (k < h) {
        SvdJob j;
        j.A = spec + P * k;
        j.W = spec + P * k;
        j.Vout = nullptr;
        j.work = work ? work + work_elems * k : nullptr;
        j.sigma = nullptr;
        j.n1 = n1;
        j.n2 = n2;
        j.real_slice = is_real_slice(k, n3) ? 1 : 0;
        j.ucols = 0;
        j.vcols = 0;
        j.sweeps_index = with_sweeps ? k : -1;
        j.tau = tau;
        j.skip = nullptr;
        j.count_out = counts_out ? counts_out + k : nullptr;
        svd[k] = j;
    }
}

}  // namespace

}  // namespace tp

using namespace tp;

extern "C" tp_status tp_prox_tnn_noalloc(const float* Y, float* X, int64_t n1, int64_t n2,
                                         int64_t n3, double tau, const tp_options* opts,
                                         void* stream) {
    tp_options o;
    tp_options_default(&o);
    if (opts) o = *opts;
    // the options every entry point checks, then those this path cannot honour: it runs the
    // Jacobi SVT only and records no stage events or sketch outputs
    if (validate_options(&o) != TP_OK) return TP_ERR_INVALID_ARG;
    if (o.method != TP_METHOD_JACOBI || o.stage_events || o.slice_flags_out || o.sketch_width_out)
        return TP_ERR_INVALID_ARG;
    if (n1 < 0 || n2 < 0 || n3 < 0 || tau != tau || tau < 0.0) return TP_ERR_INVALID_ARG;
    if (n3 > TP_MAX_N3 || n1 > TP_MAX_SVD_DIM || n2 > TP_MAX_SVD_DIM) return TP_ERR_UNSUPPORTED;
    if (n1 == 0 || n2 == 0 || n3 == 0) return TP_OK;
    if (!Y || !X) return TP_ERR_INVALID_ARG;

    const int h = free_slices((int)n3);
    const int64_t P = n1 * n2;
    SvdConfig cfg;
    if (!svd_plan((int)n1, (int)n2, SVD_PROX, &cfg)) return TP_ERR_UNSUPPORTED;
    // sizes must fit the fixed array; reject anything larger before touching the GPU
    const size_t spec_off = round256(kSvdOff + (size_t)TP_NOALLOC_JOB_BYTES * h);
    const size_t spec_bytes = round256(sizeof(float2) * (size_t)(P * h));
    const size_t work_bytes = round256(sizeof(float2) * (size_t)(cfg.work_elems * h));
    if (spec_off + spec_bytes + work_bytes > (size_t)TP_NOALLOC_SCRATCH_BYTES)
        return TP_ERR_UNSUPPORTED;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* basep = nullptr;
    if (scratch_base(&basep) != cudaSuccess) return TP_ERR_CUDA;
    if (ensure_twiddles() != cudaSuccess) return TP_ERR_CUDA;
    unsigned char* base = static_cast<unsigned char*>(basep);
    uint32_t* status = reinterpret_cast<uint32_t*>(base + kStatusOff);
    FftJob* fft = reinterpret_cast<FftJob*>(base + kFftOff);
    SvdJob* svd = reinterpret_cast<SvdJob*>(base + kSvdOff);
    float2* spec = reinterpret_cast<float2*>(base + spec_off);
    float2* work = cfg.work_elems > 0 ? reinterpret_cast<float2*>(base + spec_off + spec_bytes)
                                      : nullptr;

    if (cudaMemsetAsync(status, 0, sizeof(uint32_t), s) != cudaSuccess) return TP_ERR_CUDA;
    noalloc_jobs_kernel<<<(h + 127) / 128, 128, 0, s>>>(fft, svd, Y, X, spec, work, cfg.work_elems,
                                                        (int)n1, (int)n2, (int)n3, tau,
                                                        o.sweeps_out ? 1 : 0, o.counts_out);
    if (cudaGetLastError() != cudaSuccess) return TP_ERR_CUDA;
    const bool vec = (P % 4 == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15u) == 0) &&
                     ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
    const int tiles = fft_tiles(P, (int)n3, (int)n3, (int)n3);
    if (launch_rfft(fft, 1, tiles, (int)n3, (int)n3, vec, s) != cudaSuccess) return TP_ERR_CUDA;
    SvdLaunch L;
    L.jobs = svd;
    L.njobs = h;
    L.lp = cfg.lp;
    L.maxe = cfg.maxe;
    L.in_smem = cfg.in_smem;
    L.smem_bytes = cfg.smem_bytes;
    L.threads = cfg.threads;
    SvdParams p;
    p.mode = SVD_PROX;
    p.max_sweeps = o.max_sweeps == 0 ? 30 : o.max_sweeps;
    p.tol = (float)o.jacobi_tol;
    p.sweeps_out = o.sweeps_out;
    p.status = status;
    p.fp64_rotation = o.jacobi_fp64;
    if (launch_svd(L, p, s) != cudaSuccess) return TP_ERR_CUDA;
    if (launch_irfft(fft + 1, 1, tiles, (int)n3, (int)n3, vec, s) != cudaSuccess) return TP_ERR_CUDA;
    if (!o.sync) return TP_OK;
    uint32_t hstatus = 0;
    if (cudaMemcpyAsync(&hstatus, status, sizeof(hstatus), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TP_ERR_CUDA;
    return (hstatus & 1u) ? TP_ERR_NOT_CONVERGED : TP_OK;
}
