// extern "C" entry points of libtp: argument checks, workspace planning and the launch
// sequence of each operation (DFT of the tubes -> per-slice kernel -> inverse DFT).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "tp_internal.cuh"

using namespace tp;

namespace {

thread_local cudaError_t t_last_error = cudaSuccess;

tp_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TP_OK;
    t_last_error = e;
    if (e == cudaErrorMemoryAllocation) return TP_ERR_NO_MEMORY;
    return TP_ERR_CUDA;
}

#define TP_TRY(expr)                              \
    do {                                          \
        tp_status _st = (expr);                   \
        if (_st != TP_OK) return _st;             \
    } while (0)
#define TP_CUDA(expr) TP_TRY(from_cuda(expr))

std::mutex g_pool_mutex;
bool g_pool_ready[128] = {};

// 1: let cudaMallocAsync reuse a block freed on another stream by making the allocating stream
// wait for that stream (the pool's default); 0: never add such a wait (the pool maps new memory
// instead), so that calls issued on different streams stay independent.
#ifndef TP_POOL_INTERNAL_DEPS
#define TP_POOL_INTERNAL_DEPS 0
#endif

// Keep freed stream-ordered allocations in this process's default pool for reuse.
cudaError_t ensure_pool() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (g_pool_ready[dev]) return cudaSuccess;
    cudaMemPool_t pool;
    e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e != cudaSuccess) return e;
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    int deps = TP_POOL_INTERNAL_DEPS;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &deps);
    if (e != cudaSuccess) return e;
    g_pool_ready[dev] = true;
    return cudaSuccess;
}

int g_sms[128] = {};

// Number of SMs of the current device (cached).
tp_status sm_count(int* out) {
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return TP_ERR_CUDA;
    if (!g_sms[dev]) TP_CUDA(cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev));
    *out = g_sms[dev];
    return TP_OK;
}

tp_status prepare() {
    TP_CUDA(ensure_pool());
    TP_CUDA(ensure_twiddles());
    return TP_OK;
}

// One stream-ordered workspace per call, carved into 256-byte aligned pieces.
struct Workspace {
    cudaStream_t s;
    char* base = nullptr;
    size_t size = 0, used = 0;
    explicit Workspace(cudaStream_t st) : s(st) {}
    ~Workspace() {
        if (base) cudaFreeAsync(base, s);
    }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
    tp_status reserve(size_t bytes) {
        size = bytes;
        if (bytes == 0) return TP_OK;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s);
        if (e != cudaSuccess) {
            base = nullptr;
            cudaGetLastError();
            return from_cuda(e);
        }
        return TP_OK;
    }
    // Carve `count` elements; an over-run (a sizing bug) is recorded, not written through.
    template <class T>
    T* take(size_t count) {
        size_t b = round(count * sizeof(T));
        if (used + b > size) {
            overflow = true;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + used);
        used += b;
        return p;
    }
    bool overflow = false;
    tp_status check() const { return overflow ? TP_ERR_CUDA : TP_OK; }
};

struct Opts {
    int precision = TP_PREC_FP32, econ = 0, max_sweeps = 30, sync = 1;
    double jacobi_tol = 0.0;
    int32_t* sweeps_out = nullptr;
    void* const* events = nullptr;
    int method = TP_METHOD_JACOBI;
    int32_t* slice_flags_out = nullptr;
    int32_t* sketch_width_out = nullptr;
    int host_parts = 2;
    int32_t* counts_out = nullptr;
    int jacobi_fp64 = 0;
    // Record stage boundary i (0..3) on the stream when the caller asked for it.
    tp_status mark(int i, cudaStream_t s) const {
        if (!events || !events[i]) return TP_OK;
        return from_cuda(cudaEventRecord(static_cast<cudaEvent_t>(events[i]), s));
    }
    // Record stages i..j (inclusive) at this point.
    tp_status marks(int i, int j, cudaStream_t s) const {
        for (int k = i; k <= j; ++k) {
            tp_status st = mark(k, s);
            if (st != TP_OK) return st;
        }
        return TP_OK;
    }
};

tp_status resolve(const tp_options* o, Opts* r) {
    *r = Opts();
    if (!o) return TP_OK;
    if (o->precision < TP_PREC_FP32 || o->precision > TP_PREC_BF16X3) return TP_ERR_INVALID_ARG;
    if (o->econ != 0 && o->econ != 1) return TP_ERR_INVALID_ARG;
    if (o->max_sweeps < 0 || o->max_sweeps > 1000) return TP_ERR_INVALID_ARG;
    if (o->sync != 0 && o->sync != 1) return TP_ERR_INVALID_ARG;
    if (isnan(o->jacobi_tol) || o->jacobi_tol >= 1.0) return TP_ERR_INVALID_ARG;
    r->precision = o->precision;
    r->econ = o->econ;
    r->max_sweeps = o->max_sweeps == 0 ? 30 : o->max_sweeps;
    r->sync = o->sync;
    r->jacobi_tol = o->jacobi_tol;
    r->sweeps_out = o->sweeps_out;
    r->events = o->stage_events;
    if (o->method != TP_METHOD_JACOBI && o->method != TP_METHOD_LEARNED) return TP_ERR_INVALID_ARG;
    r->method = o->method;
    r->slice_flags_out = o->slice_flags_out;
    r->sketch_width_out = o->sketch_width_out;
    if (o->host_parts < 0 || o->host_parts > 2) return TP_ERR_INVALID_ARG;
    r->host_parts = o->host_parts == 0 ? 2 : o->host_parts;
    if (o->jacobi_fp64 != 0 && o->jacobi_fp64 != 1) return TP_ERR_INVALID_ARG;
    r->jacobi_fp64 = o->jacobi_fp64;
    r->counts_out = o->counts_out;
    return TP_OK;
}

}  // namespace

namespace tp {
tp_status validate_options(const tp_options* o) {
    Opts r;
    return resolve(o, &r);
}
}  // namespace tp

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

tp_status check_dims(int64_t n1, int64_t n2, int64_t n3) {
    if (n1 < 0 || n2 < 0 || n3 < 0) return TP_ERR_INVALID_ARG;
    if (n3 > TP_MAX_N3) return TP_ERR_UNSUPPORTED;
    if (n1 * n2 >= ((int64_t)1 << 31)) return TP_ERR_UNSUPPORTED;
    return TP_OK;
}

// Upload a host array into the workspace (pageable copy; the source may be freed on return).
// Page-locked host copies of the tables a captured call uploads: a CUDA graph's copy nodes
// read their source at every replay, so the source must live as long as the graph.
struct HostArena {
    std::vector<void*> blocks;
    ~HostArena() {
        for (void* b : blocks) cudaFreeHost(b);
    }
};
thread_local HostArena* t_arena = nullptr;  // set while a plan's launch sequence is captured

// Page-locked staging for the job tables of ordinary calls.  A copy from pageable memory
// waits for a driver staging buffer, i.e. for the stream to drain the work queued before
// it, which would tie every call's host-side planning to the GPU finishing the previous
// call.  Each upload takes a free page-locked block, copies the table into it and records an
// event after its copy; the block is free again once that event has completed.
struct StageBlock {
    char* p = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool busy = false;
};
std::mutex g_stage_mutex;
std::vector<StageBlock> g_stage[128];

tp_status stage_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return TP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    std::vector<StageBlock>& pool = g_stage[dev];
    StageBlock* pick = nullptr;
    for (StageBlock& b : pool) {
        if (b.busy && cudaEventQuery(b.done) == cudaSuccess) b.busy = false;
        if (!b.busy && b.cap >= bytes && (!pick || b.cap < pick->cap)) pick = &b;
    }
    if (!pick) {
        StageBlock b;
        b.cap = std::max<size_t>(bytes, (size_t)256 << 10);
        TP_CUDA(cudaMallocHost(reinterpret_cast<void**>(&b.p), b.cap));
        TP_CUDA(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
        pool.push_back(b);
        pick = &pool.back();
    }
    memcpy(pick->p, src, bytes);
    TP_CUDA(cudaMemcpyAsync(dst, pick->p, bytes, cudaMemcpyHostToDevice, s));
    TP_CUDA(cudaEventRecord(pick->done, s));
    pick->busy = true;
    return TP_OK;
}

template <class T>
tp_status upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (src.empty()) return TP_OK;
    const size_t bytes = sizeof(T) * src.size();
    if (t_arena) {  // captured: the copy's source must outlive the graph
        void* h = nullptr;
        TP_CUDA(cudaMallocHost(&h, bytes));
        t_arena->blocks.push_back(h);
        memcpy(h, src.data(), bytes);
        return from_cuda(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, s));
    }
    return stage_copy(dst, src.data(), bytes, s);
}

tp_status finish(uint32_t* d_status, const Opts& o, cudaStream_t s) {
    TP_CUDA(cudaGetLastError());
    if (!o.sync) return TP_OK;
    uint32_t h = 0;
    if (d_status) TP_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    if (h & 2u) return TP_ERR_SINGULAR;
    return (h & 1u) ? TP_ERR_NOT_CONVERGED : TP_OK;
}

// Events of one call, destroyed when it returns (the driver releases them once
// the recorded work completes).
struct CallEvents {
    std::vector<cudaEvent_t> ev;
    tp_status create(size_t n) {
        ev.assign(n, nullptr);
        for (auto& e : ev) TP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return TP_OK;
    }
    ~CallEvents() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// Per-device streams on which the launch groups of one SVD batch after the first run beside it
// (created once, never destroyed).
constexpr int kGroupStreams = 3;
std::mutex g_group_mutex;
cudaStream_t g_group_streams[128][kGroupStreams] = {};

tp_status group_streams(cudaStream_t* out) {
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return TP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_group_mutex);
    for (int i = 0; i < kGroupStreams; ++i) {
        if (!g_group_streams[dev][i])
            TP_CUDA(cudaStreamCreateWithFlags(&g_group_streams[dev][i], cudaStreamNonBlocking));
        out[i] = g_group_streams[dev][i];
    }
    return TP_OK;
}

// Group per-slice SVD jobs by kernel instantiation and launch each group.
struct SvdBatch {
    struct Item {
        SvdJob job{};
        SvdConfig cfg{};
        int64_t cost = 0;
    };
    std::vector<Item> items;

    SvdJob* d_jobs = nullptr;

    tp_status launch(Workspace& ws, int mode, const Opts& o, uint32_t* d_status, cudaStream_t s) {
        if (items.empty()) return TP_OK;
        TP_TRY(upload_jobs(ws, s));
        return run(mode, o, d_status, s);
    }

    int64_t key(const Item& a) const {
        return (int64_t)a.cfg.group * 10000000 + (a.cfg.in_smem ? 0 : 1000000) +
               a.cfg.lp * 100 + a.cfg.maxe;
    }

    // Sort the jobs into launch groups (largest first within a group) and upload them.
    tp_status upload_jobs(Workspace& ws, cudaStream_t s) {
        if (items.empty()) return TP_OK;
        std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& b) {
            if (key(a) != key(b)) return key(a) < key(b);
            return a.cost > b.cost;
        });
        std::vector<SvdJob> jobs(items.size());
        for (size_t i = 0; i < items.size(); ++i) jobs[i] = items[i].job;
        d_jobs = ws.take<SvdJob>(jobs.size());
        TP_TRY(ws.check());
        return upload(d_jobs, jobs, s);
    }

    // One launch per group of uploaded jobs.
    tp_status run(int mode, const Opts& o, uint32_t* d_status, cudaStream_t s) const {
        if (items.empty()) return TP_OK;
        SvdParams p;
        p.mode = mode;
        p.max_sweeps = o.max_sweeps;
        p.tol = (float)o.jacobi_tol;
        p.sweeps_out = o.sweeps_out;
        p.status = d_status;
        p.fp64_rotation = o.jacobi_fp64;
        std::vector<SvdLaunch> launches;
        size_t i = 0;
        while (i < items.size()) {
            size_t j = i;
            int smem = 0, threads = 0;
            while (j < items.size() && key(items[j]) == key(items[i])) {
                smem = std::max(smem, items[j].cfg.smem_bytes);
                threads = std::max(threads, items[j].cfg.threads);
                ++j;
            }
            SvdLaunch L;
            L.jobs = d_jobs + i;
            L.njobs = (int)(j - i);
            L.lp = items[i].cfg.lp;
            L.maxe = items[i].cfg.maxe;
            L.in_smem = items[i].cfg.in_smem;
            L.smem_bytes = smem;
            L.threads = threads;
            launches.push_back(L);
            i = j;
        }
        // One group, or the learned method's fallback (its groups hold only the few slices the
        // sketch path rejected): in order on the caller's stream.  Otherwise the first group on
        // the caller's stream and the others on group streams that fork from it and join back,
        // so that one group's tail overlaps the others.  (The group streams are shared by all
        // calls on a device, so concurrent callers would also wait on each other's groups.)
        if (launches.size() == 1 || o.method == TP_METHOD_LEARNED) {
            for (const SvdLaunch& L : launches) TP_CUDA(launch_svd(L, p, s));
            return TP_OK;
        }
        cudaStream_t gs[kGroupStreams];
        TP_TRY(group_streams(gs));
        const int nside = (int)std::min<size_t>(launches.size() - 1, kGroupStreams);
        CallEvents ev;
        TP_TRY(ev.create(1 + (size_t)nside));
        TP_CUDA(cudaEventRecord(ev.ev[0], s));
        for (int k = 0; k < nside; ++k) TP_CUDA(cudaStreamWaitEvent(gs[k], ev.ev[0], 0));
        for (size_t g = 0; g < launches.size(); ++g)
            TP_CUDA(launch_svd(launches[g], p, g == 0 ? s : gs[(g - 1) % nside]));
        for (int k = 0; k < nside; ++k) {
            TP_CUDA(cudaEventRecord(ev.ev[1 + k], gs[k]));
            TP_CUDA(cudaStreamWaitEvent(s, ev.ev[1 + k], 0));
        }
        return TP_OK;
    }
};

struct FftBatch {
    std::vector<FftJob> jobs;
    int max_n3 = 1;
    int uniform_n3 = -1;  // common n3 of all jobs, 0 once two differ
    bool vec = true;
    bool planes = false;  // the jobs write BF16x3 operand planes (all of them, add_planes)
    void add(const float* x, float2* X, int64_t P, int n3) {
        if (P <= 0 || n3 <= 0) return;
        FftJob j{};
        j.x = x;
        j.X = X;
        j.P = P;
        j.n3 = n3;
        j.tile_begin = 0;
        jobs.push_back(j);
        max_n3 = std::max(max_n3, n3);
        uniform_n3 = (uniform_n3 == -1 || uniform_n3 == n3) ? n3 : 0;
        vec = vec && (P % 4 == 0) && aligned16(x) && aligned16(X);
    }
    // Forward DFT whose output is the BF16x3 operand planes (kind PLANE_LEFT / PLANE_RIGHT,
    // rows M or K) instead of a complex spectrum; n3 must satisfy fft_writes_planes.
    void add_planes(const float* x, int64_t P, int n3, int kind, int rows, int64_t pitch,
                    uint16_t* hi, uint16_t* lo) {
        if (P <= 0 || n3 <= 0) return;
        FftJob j{};
        j.x = x;
        j.P = P;
        j.n3 = n3;
        j.plane_kind = kind;
        j.plane_rows = rows;
        j.plane_pitch = pitch;
        j.plane_hi = hi;
        j.plane_lo = lo;
        jobs.push_back(j);
        planes = true;
        max_n3 = std::max(max_n3, n3);
        uniform_n3 = (uniform_n3 == -1 || uniform_n3 == n3) ? n3 : 0;
        vec = vec && (P % 4 == 0) && aligned16(x);
    }
    tp_status launch(Workspace& ws, bool inverse, cudaStream_t s) {
        if (jobs.empty()) return TP_OK;
        // the per-length kernels for n3 <= 64 run one launch per register class: jobs are
        // grouped by class and each group's tiles count from 0
        const bool small = fft_small_path(max_n3, uniform_n3);
        if (small)
            std::stable_sort(jobs.begin(), jobs.end(), [](const FftJob& a, const FftJob& b) {
                return fft_small_class(a.n3) < fft_small_class(b.n3);
            });
        std::vector<int64_t> group_tiles;
        std::vector<size_t> group_first;
        int64_t tiles = 0;
        for (size_t i = 0; i < jobs.size(); ++i) {
            if (i == 0 || (small && fft_small_class(jobs[i].n3) != fft_small_class(jobs[i - 1].n3))) {
                group_first.push_back(i);
                group_tiles.push_back(0);
                tiles = 0;
            }
            jobs[i].tile_begin = (int32_t)tiles;
            tiles += fft_tiles(jobs[i].P, max_n3, uniform_n3, jobs[i].n3);
            if (tiles > 0x7fffffffLL) return TP_ERR_UNSUPPORTED;
            group_tiles.back() = tiles;
        }
        group_first.push_back(jobs.size());
        FftJob* d = ws.take<FftJob>(jobs.size());
        TP_TRY(ws.check());
        TP_TRY(upload(d, jobs, s));
        for (size_t g = 0; g + 1 < group_first.size(); ++g) {
            const size_t a = group_first[g], n = group_first[g + 1] - a;
            const int cls = small ? fft_small_class(jobs[a].n3) : -1;
            cudaError_t e =
                inverse ? launch_irfft(d + a, (int)n, (int)group_tiles[g], max_n3, uniform_n3, vec, s, cls)
                        : launch_rfft(d + a, (int)n, (int)group_tiles[g], max_n3, uniform_n3, vec, s, cls,
                                      planes);
            if (e != cudaSuccess) return from_cuda(e);
        }
        return TP_OK;
    }
};

size_t cbytes(int64_t count) { return Workspace::round((size_t)count * sizeof(float2)); }

// Batched prox over validated descriptors.  With TP_METHOD_LEARNED the slices first go
// through features -> proposer -> sketch SVT; the Jacobi launches then skip the slices the
// sketch path accepted.  With `train` set (proposer training) the Jacobi path labels every
// slice with its count, features are kept, and no output tensor is written.
struct ProxCapture {
    int steps = 300;
    float lr = 3e-3f;
    uint64_t seed = 0;
    double mse = 0.0;
    int64_t slices = 0;
};

// ext_status: a caller-owned (zeroed) status word shared by several calls; the call then
// neither clears it nor reads it back.
tp_status prox_batched(const tp_tensor_desc* d, int64_t count, const Opts& o, cudaStream_t s,
                       ProxCapture* train = nullptr, uint32_t* ext_status = nullptr) {
    const bool learned = (o.method == TP_METHOD_LEARNED) && !train;
    const bool need_feat = learned || train;
    size_t bytes = Workspace::round(sizeof(uint32_t));
    int64_t slices = 0;
    std::vector<SvdConfig> cfg(count);
    std::vector<int64_t> work(count, 0);
    JacobiShape shape = jacobi_shape_current();
    // the learned method's Jacobi launches hold only the slices the sketch path rejects: one
    // launch per instantiation, never split by CTA size (splitting would only add launches)
    if (o.method == TP_METHOD_LEARNED) shape.split = 0;
    int64_t nfft = 0;
    int max_n1 = 1, max_n2 = 1;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t n1 = d[t].n1, n2 = d[t].n2, n3 = d[t].n3;
        if (n1 == 0 || n2 == 0 || n3 == 0) continue;
        const int h = free_slices((int)n3);
        if (!svd_plan((int)n1, (int)n2, SVD_PROX, &cfg[t], &shape)) return TP_ERR_UNSUPPORTED;
        work[t] = cfg[t].work_elems;
        bytes += cbytes(n1 * n2 * h);
        if (work[t] > 0) bytes += cbytes(work[t] * h);
        slices += h;
        ++nfft;
        max_n1 = std::max<int>(max_n1, (int)n1);
        max_n2 = std::max<int>(max_n2, (int)n2);

    }
    if (nfft == 0) return TP_OK;
    bytes += 2 * Workspace::round(sizeof(FftJob) * (nfft + 1));
    bytes += Workspace::round(sizeof(SvdJob) * (slices + 1));
    if (need_feat) {
        bytes += Workspace::round(sizeof(SvdJob) * (slices + 1));        // natural-order jobs
        bytes += Workspace::round(sizeof(float) * kProposerInputs * slices);
        bytes += 4 * Workspace::round(sizeof(int32_t) * slices);  // ell, flags, counts, order
        bytes += Workspace::round(sizeof(int32_t) * kSketchClasses * slices);  // sketch queues
        bytes += Workspace::round(sizeof(int32_t) * 2 * kSketchClasses);       // queue counters
        bytes += 3 * Workspace::round(sizeof(int32_t) * slices);  // extra power its, 2 retry lists
        bytes += Workspace::round(sizeof(int32_t) * 2 * kSketchRetryRounds);  // retry counters
    }
    // sketch class 4 (tall buffers in global memory): one scratch slot per CTA of its launch,
    // sized for the largest slice whose widest possible sketch misses the shared-memory classes
    int sms_ws = 0;
    TP_TRY(sm_count(&sms_ws));
    int64_t g_stride = 0;
    size_t g_small = 0;
    if (learned) {
        for (int64_t t = 0; t < count; ++t) {
            const int n1 = (int)d[t].n1, n2 = (int)d[t].n2;
            if (n1 == 0 || n2 == 0 || d[t].n3 == 0) continue;
            const int lcap = std::min(kSketchMaxL, std::min(n1, n2) - 1);
            if (lcap <= 0 || (lcap <= kNarrowL && sketch_smem_need(n1, n2, lcap) <= kSketchSmemCap))
                continue;
            g_stride = std::max<int64_t>(g_stride, (int64_t)3 * std::max(n1, n2) * lcap);
            g_small = std::max(g_small, sketch_small_need(n1, n2, lcap));
        }
        g_stride = (g_stride + 31) & ~(int64_t)31;
        if (g_stride > 0) bytes += Workspace::round(sizeof(float2) * (size_t)g_stride * sms_ws);
    }
    if (train) bytes += Workspace::round(sizeof(float) * proposer_fit_scratch_floats((int)slices));
    Workspace ws(s);
    TP_TRY(ws.reserve(bytes));
    uint32_t* d_status = ws.take<uint32_t>(1);
    TP_TRY(ws.check());
    if (ext_status)
        d_status = ext_status;
    else
        TP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    float* feat = nullptr;
    int32_t *ell = nullptr, *flags = nullptr, *counts = nullptr, *d_order = nullptr;
    int32_t *d_queues = nullptr, *d_qcount = nullptr;
    int32_t *d_extra = nullptr, *d_retry = nullptr, *d_rcount = nullptr;
    SvdJob* d_nat = nullptr;
    if (need_feat) {
        d_nat = ws.take<SvdJob>(slices);
        feat = ws.take<float>((size_t)kProposerInputs * slices);
        ell = ws.take<int32_t>(slices);
        flags = ws.take<int32_t>(slices);
        counts = ws.take<int32_t>(slices);
        d_order = ws.take<int32_t>(slices);
        d_queues = ws.take<int32_t>((size_t)kSketchClasses * slices);
        d_qcount = ws.take<int32_t>(2 * kSketchClasses);
        d_extra = ws.take<int32_t>(slices);
        d_retry = ws.take<int32_t>(2 * (size_t)slices);
        d_rcount = ws.take<int32_t>(2 * kSketchRetryRounds);
        TP_TRY(ws.check());
    }
    FftBatch fwd, inv;
    SvdBatch svd;
    std::vector<SvdJob> natural;
    int64_t sidx = 0;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t n1 = d[t].n1, n2 = d[t].n2, n3 = d[t].n3;
        if (n1 == 0 || n2 == 0 || n3 == 0) continue;
        const int h = free_slices((int)n3);
        const int64_t P = n1 * n2;
        float2* spec = ws.take<float2>(P * h);
        float2* wk = work[t] > 0 ? ws.take<float2>(work[t] * h) : nullptr;
        fwd.add(d[t].in, spec, P, (int)n3);
        inv.add(d[t].out, spec, P, (int)n3);
        for (int k = 0; k < h; ++k) {
            SvdBatch::Item it{};
            SvdJob& j = it.job;
            j.A = spec + P * k;
            j.W = spec + P * k;
            j.Vout = nullptr;
            j.work = wk ? wk + work[t] * k : nullptr;
            j.sigma = nullptr;
            j.n1 = (int)n1;
            j.n2 = (int)n2;
            j.real_slice = is_real_slice(k, (int)n3) ? 1 : 0;
            j.ucols = j.vcols = 0;
            j.sweeps_index = (int32_t)sidx;
            j.tau = d[t].tau;
            j.skip = learned ? flags + sidx : nullptr;
            j.count_out = train ? counts + sidx : (o.counts_out ? o.counts_out + sidx : nullptr);
            if (need_feat) natural.push_back(j);
            it.cfg = cfg[t];
            const int64_t m = std::max(n1, n2), n = std::min(n1, n2);
            it.cost = m * n * n;
            svd.items.push_back(it);
            ++sidx;
        }
    }
    TP_TRY(ws.check());
    TP_TRY(o.mark(0, s));
    TP_TRY(fwd.launch(ws, false, s));
    TP_TRY(o.mark(1, s));
    if (need_feat) {
        TP_TRY(upload(d_nat, natural, s));
        TP_CUDA(launch_features(d_nat, (int)slices, max_n1, max_n2, feat, 0x2545f491u, s));
    }
    if (!learned) TP_TRY(o.marks(2, 3, s));
    if (learned) {
        TP_CUDA(launch_proposer(feat, d_nat, (int)slices, ell, s));
        TP_TRY(o.mark(2, s));
        // Sketch queues: the slices, largest first, binned on the device by the shared memory
        // their proposed width needs (4, 3, 2 and 1 CTAs of the sketch kernel per SM); one
        // persistent launch per class works through its queue.  Slices too large for every
        // class (or without a usable width) are flagged for the Jacobi path by the binning.
        std::vector<int32_t> sorted(slices);
        for (int64_t j = 0; j < slices; ++j) sorted[j] = (int32_t)j;
        std::stable_sort(sorted.begin(), sorted.end(), [&](int32_t a, int32_t b) {
            return (int64_t)natural[a].n1 * natural[a].n2 > (int64_t)natural[b].n1 * natural[b].n2;
        });
        TP_TRY(upload(d_order, sorted, s));
        SketchCaps caps;
        caps.n = kSketchClasses;
        caps.bytes[0] = 55 * 1024;
        caps.bytes[1] = 74 * 1024;
        caps.bytes[2] = 112 * 1024;
        caps.bytes[3] = kSketchSmemCap;
        caps.bytes[4] = 0xffffffffu;  // the rest: tall buffers in global scratch
        float2* gscratch = g_stride > 0 ? ws.take<float2>((size_t)g_stride * sms_ws) : nullptr;
        TP_TRY(ws.check());
        TP_CUDA(launch_sketch_bin(d_nat, d_order, (int)slices, ell, flags, caps, d_queues, d_qcount,
                                  s));
        int sms = 0;
        TP_TRY(sm_count(&sms));
        // retries: two rounds over lists of the slices that failed a check but are worth
        // another attempt (more power iterations or a wider sketch), in the largest class
        constexpr int kRetryRounds = kSketchRetryRounds;
        constexpr int kRetryMinDim = 96;
        const size_t retry_smem = caps.bytes[3];
        TP_CUDA(cudaMemsetAsync(d_extra, 0, sizeof(int32_t) * slices, s));
        TP_CUDA(cudaMemsetAsync(d_rcount, 0, sizeof(int32_t) * 2 * kRetryRounds, s));
        auto base = [&]() {
            SketchParams sp;
            sp.ell = ell;
            sp.flag = flags;
            sp.count = o.counts_out ? o.counts_out : counts;
            sp.njobs = (int)slices;
            sp.seed = 0x9e3779b9u;
            sp.power_iters = 1;
            sp.extra_power = d_extra;
            sp.resid_tol = 1e-5f;
            return sp;
        };
        // the class launches are independent (each takes its own queue).  With many slices
        // (several per resident CTA of every SM) class 0 runs on the caller's stream and the
        // others on group streams forked from it, so that one class's tail overlaps the next
        // classes; the retry rounds wait for all of them.  A call of few, large slices keeps
        // them in order: there concurrent classes only compete for the same SMs.
        const bool fork_classes = slices >= (int64_t)16 * sms;
        cudaStream_t cls_streams[kGroupStreams] = {};
        CallEvents cls_ev;
        if (fork_classes) {
            TP_TRY(group_streams(cls_streams));
            TP_TRY(cls_ev.create(1 + kGroupStreams));
            TP_CUDA(cudaEventRecord(cls_ev.ev[0], s));
            for (int k = 0; k < kGroupStreams; ++k)
                TP_CUDA(cudaStreamWaitEvent(cls_streams[k], cls_ev.ev[0], 0));
        }
        for (int c = 0; c < caps.n; ++c) {
            const cudaStream_t cst =
                (c == 0 || !fork_classes) ? s : cls_streams[(c - 1) % kGroupStreams];
            const bool global_class = c == caps.n - 1;
            // the global-scratch class: its shared part, one CTA per SM (one scratch slot each);
            // empty unless some slice can need it (then a one-CTA launch finds its queue empty)
            const size_t smem = global_class ? (g_stride > 0 ? g_small : (size_t)1024) : caps.bytes[c];
            const int per_sm = sketch_blocks_per_sm(smem);
            if (per_sm <= 0) return TP_ERR_CUDA;
            SketchParams sp = base();
            sp.order = d_queues + (size_t)c * slices;
            sp.queue_len = d_qcount + 2 * c;
            sp.queue_next = d_qcount + 2 * c + 1;
            sp.smem_bytes = (int)smem;
            int64_t grid = std::min<int64_t>(slices, (int64_t)sms * per_sm);
            if (global_class) {
                sp.wide = 1;
                sp.gscratch = gscratch;
                sp.gstride = g_stride;
                grid = g_stride > 0 ? std::min<int64_t>(slices, sms_ws) : 1;
            }
            TP_CUDA(launch_sketch_svt(d_nat, (int)grid, smem, sp, cst));
        }
        for (int k = 0; fork_classes && k < kGroupStreams; ++k) {
            TP_CUDA(cudaEventRecord(cls_ev.ev[1 + k], cls_streams[k]));
            TP_CUDA(cudaStreamWaitEvent(s, cls_ev.ev[1 + k], 0));
        }
        const int retry_per_sm = sketch_blocks_per_sm(retry_smem);
        if (retry_per_sm <= 0) return TP_ERR_CUDA;
        for (int round = 0; round < kRetryRounds; ++round) {
            int32_t* list = d_retry + (size_t)(round & 1) * slices;
            TP_CUDA(launch_sketch_collect(d_nat, (int)slices, flags, ell, d_extra, kRetryMinDim,
                                          (int)retry_smem, g_stride, list, d_rcount + 2 * round,
                                          s));
            SketchParams sp = base();
            sp.retry_launch = 1;
            sp.order = list;
            sp.queue_len = d_rcount + 2 * round;       // round r: length, then work counter
            sp.queue_next = d_rcount + 2 * round + 1;
            sp.smem_bytes = (int)retry_smem;
            int64_t grid = std::min<int64_t>(slices, (int64_t)sms * retry_per_sm);
            if (g_stride > 0) {
                sp.gscratch = gscratch;
                sp.gstride = g_stride;
                grid = std::min<int64_t>(slices, sms_ws);
            }
            TP_CUDA(launch_sketch_svt(d_nat, (int)grid, retry_smem, sp, s));
        }
        TP_TRY(o.mark(3, s));
        if (o.slice_flags_out)
            TP_CUDA(launch_flags01(flags, o.slice_flags_out, (int)slices, s));
        if (o.sketch_width_out)
            TP_CUDA(cudaMemcpyAsync(o.sketch_width_out, ell, sizeof(int32_t) * slices,
                                    cudaMemcpyDeviceToDevice, s));
    }
    TP_TRY(svd.launch(ws, SVD_PROX, o, d_status, s));
    TP_TRY(o.mark(4, s));
    if (train) {
        float* scratch = ws.take<float>(proposer_fit_scratch_floats((int)slices));
        TP_TRY(ws.check());
        const tp_status fs = finish(d_status, o, s);
        if (fs != TP_OK && fs != TP_ERR_NOT_CONVERGED) return fs;
        train->slices = slices;
        TP_CUDA(proposer_fit(feat, counts, (int)slices, train->steps, train->lr, train->seed,
                             scratch, &train->mse, s));
        return TP_OK;
    }
    TP_TRY(inv.launch(ws, true, s));
    TP_TRY(o.mark(5, s));
    return finish(d_status, o, s);
}

// Singular values of all free slices of one tensor, sorted decreasing, then one reduction.
tp_status sigma_op(const float* A, int64_t n1, int64_t n2, int64_t n3, int kind, double tol,
                   double* out_d, int64_t* out_i, double* s_out, const Opts& o, cudaStream_t s) {
    const int h = free_slices((int)n3);
    const int64_t r = std::min(n1, n2), P = n1 * n2;
    SvdConfig cfg;
    const JacobiShape shape = jacobi_shape_current();
    if (!svd_plan((int)n1, (int)n2, SVD_SIGMA, &cfg, &shape)) return TP_ERR_UNSUPPORTED;
    const int64_t work = cfg.work_elems;
    size_t bytes = Workspace::round(4) + cbytes(P * h) + (work ? cbytes(work * h) : 0) +
                   Workspace::round(sizeof(float) * r * h) + 2 * Workspace::round(sizeof(FftJob)) +
                   Workspace::round(sizeof(SvdJob) * h);
    Workspace ws(s);
    TP_TRY(ws.reserve(bytes));
    uint32_t* d_status = ws.take<uint32_t>(1);
    TP_TRY(ws.check());
    TP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    float2* spec = ws.take<float2>(P * h);
    float2* wk = work ? ws.take<float2>(work * h) : nullptr;
    float* sig = ws.take<float>(r * h);
    FftBatch fwd;
    fwd.add(A, spec, P, (int)n3);
    SvdBatch svd;
    for (int k = 0; k < h; ++k) {
        SvdBatch::Item it{};
        SvdJob& j = it.job;
        j.A = spec + P * k;
        j.W = nullptr;
        j.Vout = nullptr;
        j.work = wk ? wk + work * k : nullptr;
        j.sigma = sig + r * k;
        j.n1 = (int)n1;
        j.n2 = (int)n2;
        j.real_slice = is_real_slice(k, (int)n3) ? 1 : 0;
        j.ucols = j.vcols = 0;
        j.sweeps_index = k;
        j.tau = 0.0;
        it.cfg = cfg;
        it.cost = 0;
        svd.items.push_back(it);
    }
    TP_TRY(o.mark(0, s));
    TP_TRY(fwd.launch(ws, false, s));
    TP_TRY(o.marks(1, 3, s));
    TP_TRY(svd.launch(ws, SVD_SIGMA, o, d_status, s));
    TP_TRY(o.mark(4, s));
    TP_TRY(ws.check());
    TP_CUDA(launch_sigma_reduce(sig, h, (int)r, (int)n3, kind, tol, std::max(n1, n2), out_d, out_i,
                                s_out, s));
    TP_TRY(o.mark(5, s));
    return finish(d_status, o, s);
}

// Per-device streams of the host-buffer entry point (created once, never destroyed): the two
// copy directions and TP_HOST_COMPUTE_STREAMS compute streams; part c of a batch computes on
// stream c mod TP_HOST_COMPUTE_STREAMS.  With one compute stream the parts' kernels run in
// order while the copies overlap them.  With one stream per part, part 0 runs at the highest
// stream priority and each later part one level lower, so that later parts' blocks fill the
// SMs the earlier ones leave idle -- but the persistent sketch launches that need a whole SM's
// shared memory then wait for the other part's blocks to drain every SM, once per launch.
#ifndef TP_HOST_COMPUTE_STREAMS
#define TP_HOST_COMPUTE_STREAMS 1
#endif
constexpr int kHostParts = 2;  // most parts a host-buffer call is cut into (tp_options.host_parts)
constexpr int kHostComputeStreams = TP_HOST_COMPUTE_STREAMS;
static_assert(kHostComputeStreams >= 1 && kHostComputeStreams <= kHostParts, "compute streams");
struct SideStreams {
    cudaStream_t h2d = nullptr, d2h = nullptr, comp[kHostComputeStreams] = {};
};
std::mutex g_side_mutex;
SideStreams g_side[128];

tp_status side_streams(SideStreams* out) {
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return TP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_side_mutex);
    SideStreams& c = g_side[dev];
    if (!c.h2d) TP_CUDA(cudaStreamCreateWithFlags(&c.h2d, cudaStreamNonBlocking));
    if (!c.d2h) TP_CUDA(cudaStreamCreateWithFlags(&c.d2h, cudaStreamNonBlocking));
    if (!c.comp[0]) {
        int least = 0, greatest = 0;
        TP_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        for (int p = 0; p < kHostComputeStreams; ++p)
            TP_CUDA(cudaStreamCreateWithPriority(&c.comp[p], cudaStreamNonBlocking,
                                                 std::min(least, greatest + p)));
    }
    *out = c;
    return TP_OK;
}


// Copies [first, last) of a chunk between host and device, one cudaMemcpyAsync per run of
// tensors that are contiguous on both sides.
tp_status copy_runs(const tp_tensor_desc* d, const std::vector<int64_t>& bytes,
                    const std::vector<char*>& dev, int64_t first, int64_t last, bool to_device,
                    cudaStream_t st) {
    int64_t t = first;
    while (t < last) {
        if (bytes[t] == 0) {
            ++t;
            continue;
        }
        const char* h0 = to_device ? static_cast<const char*>(static_cast<const void*>(d[t].in))
                                   : static_cast<const char*>(static_cast<void*>(d[t].out));
        char* dv0 = dev[t];
        int64_t run = bytes[t], u = t + 1;
        while (u < last && bytes[u] > 0) {
            const char* hu = to_device ? static_cast<const char*>(static_cast<const void*>(d[u].in))
                                       : static_cast<const char*>(static_cast<void*>(d[u].out));
            if (hu != h0 + run || dev[u] != dv0 + run) break;
            run += bytes[u];
            ++u;
        }
        if (to_device)
            TP_CUDA(cudaMemcpyAsync(dv0, h0, (size_t)run, cudaMemcpyHostToDevice, st));
        else
            TP_CUDA(cudaMemcpyAsync(const_cast<char*>(h0), dv0, (size_t)run, cudaMemcpyDeviceToHost, st));
        t = u;
    }
    return TP_OK;
}

}  // namespace

extern "C" {

void tp_options_default(tp_options* opts) {
    if (!opts) return;
    opts->precision = TP_PREC_FP32;
    opts->econ = 0;
    opts->max_sweeps = 30;
    opts->sync = 1;
    opts->jacobi_tol = 0.0;
    opts->sweeps_out = nullptr;
    opts->stage_events = nullptr;
    opts->method = TP_METHOD_JACOBI;
    opts->slice_flags_out = nullptr;
    opts->sketch_width_out = nullptr;
    opts->host_parts = 2;
    opts->counts_out = nullptr;
    opts->jacobi_fp64 = 0;
}

const char* tp_last_error_string(void) {
    return t_last_error == cudaSuccess ? "cudaSuccess" : cudaGetErrorName(t_last_error);
}

const char* tp_status_string(tp_status status) {
    switch (status) {
        case TP_OK: return "TP_OK";
        case TP_ERR_INVALID_ARG: return "TP_ERR_INVALID_ARG";
        case TP_ERR_SHAPE: return "TP_ERR_SHAPE";
        case TP_ERR_NO_MEMORY: return "TP_ERR_NO_MEMORY";
        case TP_ERR_CUDA: return "TP_ERR_CUDA";
        case TP_ERR_NOT_CONVERGED: return "TP_ERR_NOT_CONVERGED";
        case TP_ERR_UNSUPPORTED: return "TP_ERR_UNSUPPORTED";
        case TP_ERR_SINGULAR: return "TP_ERR_SINGULAR";
        default: return "TP_ERR_UNKNOWN";
    }
}

tp_status tp_tprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t l,
                   int64_t n3, const tp_options* opts, void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_dims(n1, n2, n3));
    TP_TRY(check_dims(n2, l, n3));
    TP_TRY(check_dims(n1, l, n3));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n1 == 0 || l == 0 || n3 == 0) return TP_OK;
    if (!C) return TP_ERR_INVALID_ARG;
    if (n2 > 0 && (!A || !B)) return TP_ERR_INVALID_ARG;
    TP_TRY(prepare());
    if (n2 == 0) {
        TP_CUDA(cudaMemsetAsync(C, 0, sizeof(float) * n1 * l * n3, s));
        return finish(nullptr, o, s);
    }
    const int h = free_slices((int)n3);
    const int64_t PA = n1 * n2, PB = n2 * l, PC = n1 * l;
    const bool tc = o.precision != TP_PREC_FP32;
    // BF16x3: the operands go to the tensor cores as BF16 hi/lo planes; for power-of-two
    // n3 <= 64 the forward DFT writes them itself and no complex spectrum of A or B exists
    const bool bf = o.precision == TP_PREC_BF16X3;
    const bool direct_planes = bf && fft_writes_planes((int)n3);
    const int64_t la = bf ? bf16_left_plane_elems((int)n1, (int)n2, h) : 0;
    const int64_t lb = bf ? bf16_right_plane_elems((int)l, (int)n2, h) : 0;
    const int64_t plane_bytes =
        bf ? 2 * (int64_t)sizeof(uint16_t) * (la + lb)
           : tc ? cgemm_tc_plane_bytes((int)n1, (int)l, (int)n2, h, o.precision) : 0;
    const int64_t spec_a = direct_planes ? 0 : PA * h, spec_b = direct_planes ? 0 : PB * h;
    Workspace ws(s);
    TP_TRY(ws.reserve(cbytes(spec_a) + cbytes(spec_b) + cbytes(PC * h) +
                      2 * Workspace::round(sizeof(FftJob) * 3) + Workspace::round(4) +
                      Workspace::round((size_t)plane_bytes)));
    float2* Ab = spec_a ? ws.take<float2>(spec_a) : nullptr;
    float2* Bb = spec_b ? ws.take<float2>(spec_b) : nullptr;
    float2* Cb = ws.take<float2>(PC * h);
    uint32_t* d_err = ws.take<uint32_t>(1);
    void* planes = tc ? static_cast<void*>(ws.take<char>((size_t)plane_bytes)) : nullptr;
    TP_TRY(ws.check());
    if (tc) TP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s));
    FftBatch fwd, inv;
    if (direct_planes) {
        uint16_t* pl = static_cast<uint16_t*>(planes);
        fwd.add_planes(A, PA, (int)n3, PLANE_LEFT, (int)n1, bf16_plane_pitch((int)n1), pl, pl + la);
        fwd.add_planes(B, PB, (int)n3, PLANE_RIGHT, (int)n2, bf16_plane_pitch((int)n2),
                       pl + 2 * la, pl + 2 * la + lb);
    } else {
        fwd.add(A, Ab, PA, (int)n3);
        fwd.add(B, Bb, PB, (int)n3);
    }
    TP_TRY(o.mark(0, s));
    TP_TRY(fwd.launch(ws, false, s));
    TP_TRY(o.marks(1, 3, s));
    TP_TRY(ws.check());
    if (bf) {
        if (!direct_planes)
            TP_CUDA(bf16_planes_from_spectrum(Ab, Bb, (int)n1, (int)l, (int)n2, h, planes, s));
        TP_CUDA(launch_cgemm_bf16x3(planes, Cb, (int)n1, (int)l, (int)n2, h, (int)n3, d_err, s));
    } else if (tc) {
        TP_CUDA(launch_cgemm_tc(Ab, Bb, Cb, (int)n1, (int)l, (int)n2, h, o.precision, planes, d_err, s));
    } else {
        TP_CUDA(launch_cgemm_fp32(Ab, Bb, Cb, (int)n1, (int)l, (int)n2, PA, PB, PC, h, s));
    }
    TP_TRY(o.mark(4, s));
    inv.add(C, Cb, PC, (int)n3);
    TP_TRY(inv.launch(ws, true, s));
    TP_TRY(o.mark(5, s));
    if (!tc) return finish(nullptr, o, s);
    TP_TRY(finish(nullptr, o, s));
    if (o.sync) {
        uint32_t herr = 0;
        TP_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
        if (herr) return TP_ERR_CUDA;
    }
    return TP_OK;
}

tp_status tp_tran(const float* A, float* AT, int64_t n1, int64_t n2, int64_t n3, void* stream) {
    TP_TRY(check_dims(n1, n2, n3));
    if (n1 == 0 || n2 == 0 || n3 == 0) return TP_OK;
    if (!A || !AT) return TP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TP_CUDA(launch_tran(A, AT, n1, n2, n3, s));
    return TP_OK;
}

tp_status tp_tsvd(const float* A, float* U, float* S, float* V, int64_t n1, int64_t n2,
                  int64_t n3, const tp_options* opts, void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_dims(n1, n2, n3));
    if (n1 == 0 || n2 == 0 || n3 == 0) return TP_OK;
    if (!A || !U || !S || !V) return TP_ERR_INVALID_ARG;
    const int64_t r = std::min(n1, n2);
    const int64_t ucols = o.econ ? r : n1, vcols = o.econ ? r : n2;
    const int64_t sS1 = o.econ ? r : n1, sS2 = o.econ ? r : n2;
    if (n1 * ucols >= ((int64_t)1 << 31) || n2 * vcols >= ((int64_t)1 << 31))
        return TP_ERR_UNSUPPORTED;
    SvdConfig cfg;
    if (!svd_plan((int)n1, (int)n2, SVD_FULL, &cfg)) return TP_ERR_UNSUPPORTED;
    const int64_t work = cfg.work_elems;
    TP_TRY(prepare());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int h = free_slices((int)n3);
    const int64_t P = n1 * n2, PU = n1 * ucols, PV = n2 * vcols;
    Workspace ws(s);
    TP_TRY(ws.reserve(Workspace::round(4) + cbytes(P * h) + cbytes(work * h) + cbytes(PU * h) +
                      cbytes(PV * h) + cbytes(r * h) + Workspace::round(sizeof(float) * r * h) +
                      Workspace::round(sizeof(float) * r * n3) +
                      2 * Workspace::round(sizeof(FftJob) * 4) +
                      Workspace::round(sizeof(SvdJob) * h)));
    uint32_t* d_status = ws.take<uint32_t>(1);
    TP_TRY(ws.check());
    TP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    float2* spec = ws.take<float2>(P * h);
    float2* wk = ws.take<float2>(work * h);
    float2* Ub = ws.take<float2>(PU * h);
    float2* Vb = ws.take<float2>(PV * h);
    float2* Sb = ws.take<float2>(r * h);
    float* sig = ws.take<float>(r * h);
    float* tubes = ws.take<float>(r * n3);
    FftBatch fwd;
    fwd.add(A, spec, P, (int)n3);
    TP_TRY(fwd.launch(ws, false, s));
    SvdBatch svd;
    for (int k = 0; k < h; ++k) {
        SvdBatch::Item it{};
        SvdJob& j = it.job;
        j.A = spec + P * k;
        j.W = Ub + PU * k;
        j.Vout = Vb + PV * k;
        j.work = wk + work * k;
        j.sigma = sig + r * k;
        j.n1 = (int)n1;
        j.n2 = (int)n2;
        j.real_slice = is_real_slice(k, (int)n3) ? 1 : 0;
        j.ucols = (int)ucols;
        j.vcols = (int)vcols;
        j.sweeps_index = k;
        j.tau = 0.0;
        it.cfg = cfg;
        it.cost = 0;
        svd.items.push_back(it);
    }
    TP_TRY(svd.launch(ws, SVD_FULL, o, d_status, s));
    TP_TRY(ws.check());
    TP_CUDA(launch_diag_spectrum(sig, h, (int)r, Sb, s));
    TP_CUDA(cudaMemsetAsync(S, 0, sizeof(float) * sS1 * sS2 * n3, s));
    FftBatch inv;
    inv.add(U, Ub, PU, (int)n3);
    inv.add(V, Vb, PV, (int)n3);
    inv.add(tubes, Sb, r, (int)n3);
    TP_TRY(inv.launch(ws, true, s));
    TP_CUDA(launch_diag_scatter(tubes, (int)r, (int)n3, S, sS1, sS2, s));
    return finish(d_status, o, s);
}

tp_status tp_tinv(const float* A, float* B, int64_t n1, int64_t n2, int64_t n3,
                  const tp_options* opts, void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_dims(n1, n2, n3));
    if (n1 != n2) return TP_ERR_SHAPE;
    if (n1 > TP_MAX_SVD_DIM) return TP_ERR_UNSUPPORTED;
    if (n1 == 0 || n3 == 0) return TP_OK;
    if (!A || !B) return TP_ERR_INVALID_ARG;
    TP_TRY(prepare());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int h = free_slices((int)n3);
    const int64_t P = n1 * n1;
    Workspace ws(s);
    TP_TRY(ws.reserve(Workspace::round(4) + cbytes(P * h) + 2 * Workspace::round(sizeof(FftJob) * 2) +
                      Workspace::round(sizeof(LaJob) * h)));
    uint32_t* d_status = ws.take<uint32_t>(1);
    TP_TRY(ws.check());
    TP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    float2* spec = ws.take<float2>(P * h);
    LaJob* d_jobs = ws.take<LaJob>(h);
    TP_TRY(ws.check());
    std::vector<LaJob> jobs(h);
    for (int k = 0; k < h; ++k) {
        jobs[k].A = jobs[k].R = spec + P * k;
        jobs[k].n1 = jobs[k].n2 = (int)n1;
    }
    TP_TRY(upload(d_jobs, jobs, s));
    TP_TRY(o.mark(0, s));
    FftBatch fwd;
    fwd.add(A, spec, P, (int)n3);
    TP_TRY(fwd.launch(ws, false, s));
    TP_TRY(o.marks(1, 3, s));
    TP_CUDA(launch_tinv(d_jobs, h, (int)n1, d_status, s));
    TP_TRY(o.mark(4, s));
    FftBatch inv;
    inv.add(B, spec, P, (int)n3);
    TP_TRY(inv.launch(ws, true, s));
    TP_TRY(o.mark(5, s));
    return finish(d_status, o, s);
}

tp_status tp_tqr(const float* A, float* Q, float* R, int64_t n1, int64_t n2, int64_t n3,
                 const tp_options* opts, void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_dims(n1, n2, n3));
    if (std::max(n1, n2) > TP_MAX_SVD_DIM) return TP_ERR_UNSUPPORTED;
    if (n1 == 0 || n2 == 0 || n3 == 0) return TP_OK;
    if (!A || !Q || !R) return TP_ERR_INVALID_ARG;
    TP_TRY(prepare());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t m = std::min(n1, n2);
    const int64_t qc = o.econ ? m : n1, rr = o.econ ? m : n1;
    const int h = free_slices((int)n3);
    const int64_t P = n1 * n2, PQ = n1 * qc, PR = rr * n2;
    Workspace ws(s);
    TP_TRY(ws.reserve(cbytes(P * h) + cbytes(PQ * h) + cbytes(PR * h) +
                      Workspace::round(sizeof(FftJob) * 2) + Workspace::round(sizeof(FftJob) * 3) +
                      Workspace::round(sizeof(LaJob) * h)));
    float2* spec = ws.take<float2>(P * h);
    float2* Qb = ws.take<float2>(PQ * h);
    float2* Rb = ws.take<float2>(PR * h);
    LaJob* d_jobs = ws.take<LaJob>(h);
    TP_TRY(ws.check());
    std::vector<LaJob> jobs(h);
    for (int k = 0; k < h; ++k) {
        jobs[k].A = spec + P * k;
        jobs[k].Q = Qb + PQ * k;
        jobs[k].R = Rb + PR * k;
        jobs[k].n1 = (int)n1;
        jobs[k].n2 = (int)n2;
        jobs[k].qcols = (int)qc;
        jobs[k].rrows = (int)rr;
    }
    TP_TRY(upload(d_jobs, jobs, s));
    TP_TRY(o.mark(0, s));
    FftBatch fwd;
    fwd.add(A, spec, P, (int)n3);
    TP_TRY(fwd.launch(ws, false, s));
    TP_TRY(o.marks(1, 3, s));
    TP_CUDA(launch_tqr(d_jobs, h, (int)n1, (int)n2, (int)qc, s));
    TP_TRY(o.mark(4, s));
    FftBatch inv;
    inv.add(Q, Qb, PQ, (int)n3);
    inv.add(R, Rb, PR, (int)n3);
    TP_TRY(inv.launch(ws, true, s));
    TP_TRY(o.mark(5, s));
    return finish(nullptr, o, s);
}

static tp_status scalar_op(const float* A, double* out, int64_t n1, int64_t n2, int64_t n3,
                           const tp_options* opts, void* stream, int kind) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_dims(n1, n2, n3));
    if (!out) return TP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n1 == 0 || n2 == 0 || n3 == 0) {
        TP_TRY(prepare());
        TP_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
        return finish(nullptr, o, s);
    }
    if (!A) return TP_ERR_INVALID_ARG;
    TP_TRY(prepare());
    return sigma_op(A, n1, n2, n3, kind, 0.0, out, nullptr, nullptr, o, s);
}

tp_status tp_tnn(const float* A, double* out, int64_t n1, int64_t n2, int64_t n3,
                 const tp_options* opts, void* stream) {
    return scalar_op(A, out, n1, n2, n3, opts, stream, 0);
}

tp_status tp_tsn(const float* A, double* out, int64_t n1, int64_t n2, int64_t n3,
                 const tp_options* opts, void* stream) {
    return scalar_op(A, out, n1, n2, n3, opts, stream, 1);
}

tp_status tp_tubalrank(const float* A, int64_t* out, double* s_out, int64_t n1, int64_t n2,
                       int64_t n3, double tol, const tp_options* opts, void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_dims(n1, n2, n3));
    if (!out || isnan(tol)) return TP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TP_TRY(prepare());
    if (n1 == 0 || n2 == 0 || n3 == 0) {
        TP_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return finish(nullptr, o, s);
    }
    if (!A) return TP_ERR_INVALID_ARG;
    return sigma_op(A, n1, n2, n3, 2, tol, nullptr, out, s_out, o, s);
}

tp_status tp_prox_tnn(const float* Y, float* X, int64_t n1, int64_t n2, int64_t n3, double tau,
                      const tp_options* opts, void* stream) {
    tp_tensor_desc d;
    d.in = Y;
    d.out = X;
    d.n1 = n1;
    d.n2 = n2;
    d.n3 = n3;
    d.tau = tau;
    return tp_prox_tnn_batched(&d, 1, opts, stream);
}

static tp_status check_descs(const tp_tensor_desc* descs, int64_t count) {
    if (count < 0 || (count > 0 && !descs)) return TP_ERR_INVALID_ARG;
    for (int64_t t = 0; t < count; ++t) {
        const tp_tensor_desc& d = descs[t];
        TP_TRY(check_dims(d.n1, d.n2, d.n3));
        if (isnan(d.tau) || d.tau < 0.0) return TP_ERR_INVALID_ARG;
        if (d.n1 == 0 || d.n2 == 0 || d.n3 == 0) continue;
        if (!d.in) return TP_ERR_INVALID_ARG;
        if (std::max(d.n1, d.n2) > TP_MAX_SVD_DIM) return TP_ERR_UNSUPPORTED;
    }
    return TP_OK;
}

struct tp_prox_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t* d_status = nullptr;
    HostArena arena;
    int sync = 1;
    ~tp_prox_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (d_status) cudaFree(d_status);
    }
};

tp_status tp_prox_plan_create(const tp_tensor_desc* descs, int64_t count, const tp_options* opts,
                              tp_prox_plan** plan) {
    if (!plan) return TP_ERR_INVALID_ARG;
    *plan = nullptr;
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_descs(descs, count));
    for (int64_t t = 0; t < count; ++t)
        if (descs[t].n1 > 0 && descs[t].n2 > 0 && descs[t].n3 > 0 && !descs[t].out)
            return TP_ERR_INVALID_ARG;
    if (o.events) return TP_ERR_INVALID_ARG;  // stage events cannot be replayed
    TP_TRY(prepare());
    if (o.method == TP_METHOD_LEARNED && !proposer_ready()) return TP_ERR_INVALID_ARG;
    std::unique_ptr<tp_prox_plan> p(new tp_prox_plan());
    p->sync = o.sync;
    TP_CUDA(cudaMalloc(&p->d_status, sizeof(uint32_t)));
    cudaStream_t cap = nullptr;
    TP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    Opts oc = o;
    oc.sync = 0;
    tp_status st = from_cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    if (st == TP_OK) {
        t_arena = &p->arena;
        st = from_cuda(cudaMemsetAsync(p->d_status, 0, sizeof(uint32_t), cap));
        if (st == TP_OK) st = prox_batched(descs, count, oc, cap, nullptr, p->d_status);
        t_arena = nullptr;
        cudaGraph_t g = nullptr;
        const tp_status end = from_cuda(cudaStreamEndCapture(cap, &g));
        p->graph = g;
        if (st == TP_OK) st = end;
    }
    if (st == TP_OK) st = from_cuda(cudaGraphInstantiate(&p->exec, p->graph, 0));
    cudaStreamDestroy(cap);
    if (st != TP_OK) return st;
    *plan = p.release();
    return TP_OK;
}

tp_status tp_prox_plan_run(tp_prox_plan* plan, void* stream) {
    if (!plan || !plan->exec) return TP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TP_CUDA(cudaGraphLaunch(plan->exec, s));
    if (!plan->sync) return TP_OK;
    uint32_t h = 0;
    TP_CUDA(cudaMemcpyAsync(&h, plan->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    return (h & 1u) ? TP_ERR_NOT_CONVERGED : TP_OK;
}

tp_status tp_prox_plan_destroy(tp_prox_plan* plan) {
    delete plan;
    return TP_OK;
}

tp_status tp_proposer_train(const tp_tensor_desc* descs, int64_t count, int32_t steps, double lr,
                            uint64_t seed, double* mse_out, void* stream) {
    TP_TRY(check_descs(descs, count));
    if (steps < 1 || steps > 100000 || !(lr > 0.0) || lr > 1.0) return TP_ERR_INVALID_ARG;
    int64_t slices = 0;
    for (int64_t t = 0; t < count; ++t)
        if (descs[t].n1 > 0 && descs[t].n2 > 0 && descs[t].n3 > 0) slices += free_slices((int)descs[t].n3);
    if (slices == 0 || slices > (1 << 24)) return TP_ERR_INVALID_ARG;
    TP_TRY(prepare());
    Opts o;
    o.sync = 1;
    ProxCapture cap;
    cap.steps = steps;
    cap.lr = (float)lr;
    cap.seed = seed;
    tp_status st = prox_batched(descs, count, o, static_cast<cudaStream_t>(stream), &cap);
    if (st != TP_OK && st != TP_ERR_NOT_CONVERGED) return st;
    if (mse_out) *mse_out = cap.mse;
    return TP_OK;
}

tp_status tp_proposer_get(float* host_params) {
    if (!host_params) return TP_ERR_INVALID_ARG;
    if (!proposer_ready()) return TP_ERR_INVALID_ARG;
    TP_CUDA(proposer_get(host_params));
    return TP_OK;
}

tp_status tp_proposer_set(const float* host_params) {
    if (!host_params) return TP_ERR_INVALID_ARG;
    for (int i = 0; i < kProposerFloats; ++i)
        if (!isfinite(host_params[i])) return TP_ERR_INVALID_ARG;
    TP_CUDA(proposer_set(host_params));
    return TP_OK;
}

static tp_status shape_in(const tp_jacobi_shape* in, JacobiShape* out) {
    out->target_e2 = in->target_lane_pairs;
    out->max_warps = in->max_warps;
    out->split = in->split_launches;
    return jacobi_shape_valid(*out) ? TP_OK : TP_ERR_INVALID_ARG;
}

static void shape_out(const JacobiShape& in, tp_jacobi_shape* out) {
    out->target_lane_pairs = in.target_e2;
    out->max_warps = in.max_warps;
    out->split_launches = in.split;
}

tp_status tp_jacobi_shape_get(tp_jacobi_shape* shape) {
    if (!shape) return TP_ERR_INVALID_ARG;
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    shape_out(jacobi_shape_current(), shape);
    return TP_OK;
}

tp_status tp_jacobi_shape_set(const tp_jacobi_shape* shape) {
    JacobiShape sh;
    if (shape) TP_TRY(shape_in(shape, &sh));
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    jacobi_shape_store(sh);
    return TP_OK;
}

// Times the batched Jacobi prox launches on the batch's own Fourier slices under every
// candidate shape and keeps the fastest.  The slices are computed once; each candidate reads
// them and writes its thresholded slices to a second buffer, so every candidate sees the
// same input.
tp_status tp_autotune_jacobi(const tp_tensor_desc* descs, int64_t count, int32_t reps,
                             tp_jacobi_shape* chosen, double* ms_out, void* stream) {
    TP_TRY(check_descs(descs, count));
    if (reps < 1 || reps > 100 || !chosen) return TP_ERR_INVALID_ARG;
    int64_t slices = 0, nfft = 0;
    size_t spec_bytes = 0;
    for (int64_t t = 0; t < count; ++t) {
        const tp_tensor_desc& d = descs[t];
        if (d.n1 == 0 || d.n2 == 0 || d.n3 == 0) continue;
        const int h = free_slices((int)d.n3);
        spec_bytes += cbytes(d.n1 * d.n2 * h);
        slices += h;
        ++nfft;
    }
    if (slices == 0) return TP_ERR_INVALID_ARG;
    TP_TRY(prepare());
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    Workspace ws(s);
    TP_TRY(ws.reserve(Workspace::round(sizeof(uint32_t)) + 2 * spec_bytes +
                      Workspace::round(sizeof(FftJob) * (nfft + 1))));
    uint32_t* d_status = ws.take<uint32_t>(1);
    std::vector<float2*> spec(count, nullptr), outs(count, nullptr);
    FftBatch fwd;
    for (int64_t t = 0; t < count; ++t) {
        const tp_tensor_desc& d = descs[t];
        if (d.n1 == 0 || d.n2 == 0 || d.n3 == 0) continue;
        const int64_t P = d.n1 * d.n2;
        const int h = free_slices((int)d.n3);
        spec[t] = ws.take<float2>(P * h);
        outs[t] = ws.take<float2>(P * h);
        fwd.add(d.in, spec[t], P, (int)d.n3);
    }
    TP_TRY(ws.check());
    TP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    TP_TRY(fwd.launch(ws, false, s));

    std::vector<JacobiShape> cands;
    cands.push_back(JacobiShape());  // the default first: it wins ties
    for (int split : {0, 1})
        for (int e2 : {3, 5, 7})
            for (int w : {8, 16, 32}) {
                JacobiShape c;
                c.target_e2 = e2;
                c.max_warps = w;
                c.split = split;
                if (c.target_e2 == 5 && c.max_warps == 32 && c.split == 0) continue;
                cands.push_back(c);
            }

    struct Ev {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Ev() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    TP_CUDA(cudaEventCreate(&ev.a));
    TP_CUDA(cudaEventCreate(&ev.b));
    Opts o;  // default sweep cap and tolerance, no per-slice outputs
    double best_ms = 0.0, default_ms = 0.0;
    size_t best = 0;
    for (size_t c = 0; c < cands.size(); ++c) {
        SvdBatch svd;
        std::vector<SvdConfig> cfg(count);
        size_t bytes = Workspace::round(sizeof(SvdJob) * (slices + 1));
        for (int64_t t = 0; t < count; ++t) {
            const tp_tensor_desc& d = descs[t];
            if (!spec[t]) continue;
            if (!svd_plan((int)d.n1, (int)d.n2, SVD_PROX, &cfg[t], &cands[c]))
                return TP_ERR_UNSUPPORTED;
            if (cfg[t].work_elems > 0) bytes += cbytes(cfg[t].work_elems * free_slices((int)d.n3));
        }
        Workspace cw(s);
        TP_TRY(cw.reserve(bytes));
        for (int64_t t = 0; t < count; ++t) {
            const tp_tensor_desc& d = descs[t];
            if (!spec[t]) continue;
            const int h = free_slices((int)d.n3);
            const int64_t P = d.n1 * d.n2;
            float2* wk = cfg[t].work_elems > 0 ? cw.take<float2>(cfg[t].work_elems * h) : nullptr;
            for (int k = 0; k < h; ++k) {
                SvdBatch::Item it{};
                SvdJob& j = it.job;
                j.A = spec[t] + P * k;
                j.W = outs[t] + P * k;
                j.work = wk ? wk + cfg[t].work_elems * k : nullptr;
                j.n1 = (int)d.n1;
                j.n2 = (int)d.n2;
                j.real_slice = is_real_slice(k, (int)d.n3) ? 1 : 0;
                j.tau = d.tau;
                it.cfg = cfg[t];
                const int64_t m = std::max(d.n1, d.n2), n = std::min(d.n1, d.n2);
                it.cost = m * n * n;
                svd.items.push_back(it);
            }
        }
        TP_TRY(cw.check());
        TP_TRY(svd.upload_jobs(cw, s));
        TP_TRY(svd.run(SVD_PROX, o, d_status, s));  // untimed: first launch of each kernel
        TP_CUDA(cudaEventRecord(ev.a, s));
        for (int r = 0; r < reps; ++r) TP_TRY(svd.run(SVD_PROX, o, d_status, s));
        TP_CUDA(cudaEventRecord(ev.b, s));
        TP_CUDA(cudaEventSynchronize(ev.b));
        float ms = 0.f;
        TP_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
        const double per = (double)ms / reps;
        if (c == 0) default_ms = best_ms = per;
        else if (per < best_ms) {
            best_ms = per;
            best = c;
        }
    }
    TP_CUDA(cudaStreamSynchronize(s));
    jacobi_shape_store(cands[best]);
    shape_out(cands[best], chosen);
    if (ms_out) {
        ms_out[0] = default_ms;
        ms_out[1] = best_ms;
    }
    return TP_OK;
}

tp_status tp_prox_tnn_batched(const tp_tensor_desc* descs, int64_t count, const tp_options* opts,
                              void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    if (count < 0 || (count > 0 && !descs)) return TP_ERR_INVALID_ARG;
    for (int64_t t = 0; t < count; ++t) {
        const tp_tensor_desc& d = descs[t];
        TP_TRY(check_dims(d.n1, d.n2, d.n3));
        if (isnan(d.tau) || d.tau < 0.0) return TP_ERR_INVALID_ARG;
        if (d.n1 == 0 || d.n2 == 0 || d.n3 == 0) continue;
        if (!d.in || !d.out) return TP_ERR_INVALID_ARG;
        if (std::max(d.n1, d.n2) > TP_MAX_SVD_DIM) return TP_ERR_UNSUPPORTED;
    }
    if (count == 0) return TP_OK;
    TP_TRY(prepare());
    if (o.method == TP_METHOD_LEARNED && !proposer_ready()) return TP_ERR_INVALID_ARG;
    return prox_batched(descs, count, o, static_cast<cudaStream_t>(stream));
}

tp_status tp_prox_tnn_batched_host(const tp_tensor_desc* descs, int64_t count,
                                   const tp_options* opts, void* stream) {
    Opts o;
    TP_TRY(resolve(opts, &o));
    TP_TRY(check_descs(descs, count));
    for (int64_t t = 0; t < count; ++t)
        if (descs[t].n1 > 0 && descs[t].n2 > 0 && descs[t].n3 > 0 && !descs[t].out)
            return TP_ERR_INVALID_ARG;
    if (count == 0) return TP_OK;
    TP_TRY(prepare());
    if (o.method == TP_METHOD_LEARNED && !proposer_ready()) return TP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SideStreams ss;
    TP_TRY(side_streams(&ss));

    // The batch is cut, at tensor boundaries, into up to o.host_parts parts of at least 16 MiB.
    // Part c runs on side compute stream c once its host-to-device copy has landed and is
    // copied back as soon as its kernels are done: the copy of part c+1 and the copy back of
    // part c-1 overlap part c's kernels.
    const int kParts = std::min(o.host_parts, kHostParts);
    std::vector<int64_t> bytes(count), slices(count);
    int64_t total = 0;
    for (int64_t t = 0; t < count; ++t) {
        const tp_tensor_desc& d = descs[t];
        const bool empty = d.n1 == 0 || d.n2 == 0 || d.n3 == 0;
        bytes[t] = empty ? 0 : (int64_t)sizeof(float) * d.n1 * d.n2 * d.n3;
        slices[t] = empty ? 0 : free_slices((int)d.n3);
        total += bytes[t];
    }
    if (total == 0) return TP_OK;
    const int64_t target = std::max<int64_t>(total / kParts, 16 << 20);
    std::vector<int64_t> cut{0};
    std::vector<int64_t> off(count, 0);  // device offset of each tensor in the batch buffer
    int64_t acc = 0, cur = 0;
    for (int64_t t = 0; t < count; ++t) {
        if (bytes[t] > 0) {
            // keep the host pointer's alignment (mod 256) so that tensors contiguous in host
            // memory stay contiguous on the device and one copy moves a whole run
            const bool follows = t > 0 && bytes[t - 1] > 0 &&
                                 reinterpret_cast<const char*>(descs[t].in) ==
                                     reinterpret_cast<const char*>(descs[t - 1].in) + bytes[t - 1];
            const int64_t a = (int64_t)(reinterpret_cast<uintptr_t>(descs[t].in) & 255u);
            off[t] = follows ? cur : ((cur + 255) & ~(int64_t)255) + a;
            cur = off[t] + bytes[t];
            acc += bytes[t];
        }
        if ((acc >= target && (int)cut.size() < kParts) || t + 1 == count) {
            cut.push_back(t + 1);
            acc = 0;
        }
    }
    const int nparts = (int)cut.size() - 1;
    const size_t slab = Workspace::round((size_t)cur + 256);
    Workspace ws(s);
    TP_TRY(ws.reserve(Workspace::round(4) + slab));
    uint32_t* d_status = ws.take<uint32_t>(1);
    char* buf = ws.take<char>(slab);
    TP_TRY(ws.check());
    TP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    CallEvents ce;  // [0] start, [1 + c] copied in, [1 + nparts + c] computed, [last] copied back
    TP_TRY(ce.create(2 + 2 * (size_t)nparts));
    cudaEvent_t ev_start = ce.ev[0], ev_back = ce.ev.back();
    TP_TRY(o.mark(0, s));
    TP_CUDA(cudaEventRecord(ev_start, s));
    TP_CUDA(cudaStreamWaitEvent(ss.h2d, ev_start, 0));
    TP_CUDA(cudaStreamWaitEvent(ss.d2h, ev_start, 0));

    std::vector<char*> dev(count, nullptr);
    for (int64_t t = 0; t < count; ++t) dev[t] = buf + off[t];
    std::vector<tp_tensor_desc> part;
    int64_t slice_base = 0;
    for (int c = 0; c < nparts; ++c) {
        const int64_t first = cut[c], last = cut[c + 1];
        cudaStream_t cs = ss.comp[c % kHostComputeStreams];
        cudaEvent_t ev_in = ce.ev[1 + c], ev_done = ce.ev[1 + nparts + c];
        TP_TRY(copy_runs(descs, bytes, dev, first, last, true, ss.h2d));
        TP_CUDA(cudaEventRecord(ev_in, ss.h2d));
        TP_CUDA(cudaStreamWaitEvent(cs, ev_in, 0));  // ev_in follows ev_start
        part.clear();
        int64_t part_slices = 0;
        for (int64_t t = first; t < last; ++t) {
            tp_tensor_desc d = descs[t];
            d.in = reinterpret_cast<const float*>(dev[t]);
            d.out = reinterpret_cast<float*>(dev[t]);
            part.push_back(d);
            part_slices += slices[t];
        }
        Opts oc = o;
        oc.sync = 0;
        oc.events = nullptr;
        oc.sweeps_out = o.sweeps_out ? o.sweeps_out + slice_base : nullptr;
        oc.slice_flags_out = o.slice_flags_out ? o.slice_flags_out + slice_base : nullptr;
        oc.sketch_width_out = o.sketch_width_out ? o.sketch_width_out + slice_base : nullptr;
        oc.counts_out = o.counts_out ? o.counts_out + slice_base : nullptr;
        TP_TRY(prox_batched(part.data(), (int64_t)part.size(), oc, cs, nullptr, d_status));
        slice_base += part_slices;
        TP_CUDA(cudaEventRecord(ev_done, cs));
        TP_CUDA(cudaStreamWaitEvent(ss.d2h, ev_done, 0));
        TP_TRY(copy_runs(descs, bytes, dev, first, last, false, ss.d2h));
    }
    // every part's kernels precede its copy back, so this one event covers all side streams
    TP_CUDA(cudaEventRecord(ev_back, ss.d2h));
    TP_CUDA(cudaStreamWaitEvent(s, ev_back, 0));
    TP_TRY(o.marks(1, 5, s));
    return finish(d_status, o, s);
}

}  // extern "C"
