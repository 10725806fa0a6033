// Tensor-core slice GEMMs of the t-product (Algorithm 1, step 2): Cbar^(k) = Abar^(k) Bbar^(k)
// on the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory, operands
// staged by TMA), in split precision with FP32 accumulation:
//   BF16x3:  x = x_hi + x_lo with x_hi = bf16(x), x_lo = bf16(x - x_hi);
//            a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi  (kind::f16, bf16 inputs)
//   3xTF32:  the same with tf32 halves (kind::tf32).
//
// Complex to real.  With A' = [Ar | Ai] (M x 2K) and, for every output column n, the two rows
// [Br(:,n) ; -Bi(:,n)] and [Bi(:,n) ; Br(:,n)] of B' (2N x 2K, K-major), the real product
// A' B'^T has Cr(m,n) in column 2n and Ci(m,n) in column 2n+1: one real GEMM of
// M x 2N x 2K carries the 8 M N K flops of the complex product, and the accumulator's
// adjacent columns are the (re, im) pair the epilogue stores as one float2.
//
// Data path.  Split kernels turn the complex FP32 spectra into hi/lo planes in the K-major,
// zero-padded layout the MMA reads (A transposed through shared memory, B row-interleaved as
// above).  The GEMM CTA (128 threads) owns a 128 x 256 accumulator tile (128 rows of C by
// 128 complex columns) in 256 TMEM columns; one lane of warp 0 streams 128-byte-wide K blocks
// of the four operand tiles with TMA (128B swizzle) into a two-stage ring, one lane of warp 1
// issues three MMAs per K step and commits each stage back to the producer, and all four
// warps then read the accumulator (tcgen05.ld, 32 lanes each) and store C.  Every mbarrier
// wait is bounded: on timeout the kernel records an error bit, stops, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "tp_internal.cuh"
#include "tp_planes.cuh"

namespace tp {

namespace {

constexpr int kBM = 128;                  // rows of C per CTA (UMMA M)
constexpr int kBN = 256;                  // accumulator columns per CTA (UMMA N): 128 complex
constexpr int kRowBytes = 128;            // one K block of a row: a 128-byte swizzle span
constexpr int kTileA = kBM * kRowBytes;   // 16 KB
constexpr int kTileB = kBN * kRowBytes;   // 32 KB
constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;
constexpr int kStages = 2;
constexpr int kThreads = 128;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitLimit = 2000000000LL;  // clock cycles (about 1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Wait for the phase with the given parity to complete; false after kWaitLimit cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitLimit) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored with the 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (the tile base is 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(const void* tile) {
    const uint64_t a = smem_u32(tile);
    uint64_t d = (a >> 4) & 0x3FFFull;        // start address
    d |= 1ull << 16;                          // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
    d |= 1ull << 46;                          // descriptor version
    d |= 2ull << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of the given format, both K-major,
// N = kBN, M = kBM.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kBN >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    if (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc(2)), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc(1)), "r"(accumulate));
    }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                     "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------------------
// Split kernels: complex FP32 spectra -> hi/lo planes, K-major, zero-padded.
// ---------------------------------------------------------------------------------------
template <bool TF32>
struct Split;

template <>
struct Split<false> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ void run(float x, T& hi, T& lo) {
        hi = __float2bfloat16_rn(x);
        lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
};

template <>
struct Split<true> {
    using T = float;
    static __device__ __forceinline__ void run(float x, T& hi, T& lo) {
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        hi = __uint_as_float(h);
        lo = x - hi;
    }
};

// A' planes: row m of slice z is [Ar(m, 0..Kp) | Ai(m, 0..Kp)]; input Abar column-major M x K.
template <bool TF32>
__global__ void __launch_bounds__(256) split_a_kernel(const float2* __restrict__ Ab,
                                                      typename Split<TF32>::T* __restrict__ hi,
                                                      typename Split<TF32>::T* __restrict__ lo,
                                                      int M, int K, int Mp, int Kp) {
    __shared__ float2 tile[32][33];
    const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 32, z = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float2* src = Ab + (int64_t)z * M * K;
    for (int r = ty; r < 32; r += 8) {
        const int kk = k0 + r, m = m0 + tx;
        tile[r][tx] = (m < M && kk < K) ? src[m + (int64_t)M * kk] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int64_t plane = (int64_t)Mp * 2 * Kp;
    for (int r = ty; r < 32; r += 8) {
        const int m = m0 + r, kk = k0 + tx;
        const float2 v = tile[tx][r];
        const int64_t row = (int64_t)z * plane + (int64_t)m * 2 * Kp;
        typename Split<TF32>::T h, l;
        Split<TF32>::run(v.x, h, l);
        hi[row + kk] = h;
        lo[row + kk] = l;
        Split<TF32>::run(v.y, h, l);
        hi[row + Kp + kk] = h;
        lo[row + Kp + kk] = l;
    }
}

// B' planes: rows 2n and 2n+1 of slice z are [Br(:,n) | -Bi(:,n)] and [Bi(:,n) | Br(:,n)];
// input Bbar column-major K x N (already K-major).
template <bool TF32>
__global__ void __launch_bounds__(256) split_b_kernel(const float2* __restrict__ Bb,
                                                      typename Split<TF32>::T* __restrict__ hi,
                                                      typename Split<TF32>::T* __restrict__ lo,
                                                      int K, int N, int Kp, int Np) {
    const int kk = blockIdx.x * 32 + threadIdx.x, n = blockIdx.y * 8 + threadIdx.y,
              z = blockIdx.z;
    if (kk >= Kp || n >= Np) return;
    const float2 v = (kk < K && n < N) ? Bb[(int64_t)z * K * N + kk + (int64_t)K * n]
                                       : make_float2(0.f, 0.f);
    const int64_t plane = (int64_t)2 * Np * 2 * Kp;
    const int64_t r0 = (int64_t)z * plane + (int64_t)(2 * n) * 2 * Kp;
    const int64_t r1 = r0 + 2 * Kp;
    typename Split<TF32>::T h, l;
    Split<TF32>::run(v.x, h, l);
    hi[r0 + kk] = h;
    lo[r0 + kk] = l;
    hi[r1 + Kp + kk] = h;
    lo[r1 + Kp + kk] = l;
    Split<TF32>::run(-v.y, h, l);
    hi[r0 + Kp + kk] = h;
    lo[r0 + Kp + kk] = l;
    Split<TF32>::run(v.y, h, l);
    hi[r1 + kk] = h;
    lo[r1 + kk] = l;
}

// ---------------------------------------------------------------------------------------
// The GEMM: grid (Mp/128, 2Np/256, slices), 128 threads, one 128 x 256 FP32 accumulator.
// ---------------------------------------------------------------------------------------
template <bool TF32>
__global__ void __launch_bounds__(kThreads, 1) cgemm_tc_kernel(
    const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
    float2* __restrict__ C, int M, int N, int64_t sC, int nkb, uint32_t* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    constexpr int kElemsPerRow = kRowBytes / (TF32 ? 4 : 2);  // K elements per K block
    constexpr int kSteps = TF32 ? 4 : 4;                      // MMAs of K = 32 bytes per block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, nt = blockIdx.y, z = blockIdx.z;
    // a CTA that timed out already: the rest of the grid does no work
    if (*reinterpret_cast<volatile uint32_t*>(err) != 0u) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the four operand tiles of each K block
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kStages, j = kb / kStages;
            if (j > 0 && !mbar_wait(&empty[s], (j - 1) & 1)) {
                atomicOr(err, 2u);
                break;
            }
            unsigned char* st = smem + s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            const int kc = kb * kElemsPerRow;
            tma_load_3d(st, &mAh, &full[s], kc, mt * kBM, z);
            tma_load_3d(st + kTileA, &mAl, &full[s], kc, mt * kBM, z);
            tma_load_3d(st + 2 * kTileA, &mBh, &full[s], kc, nt * kBN, z);
            tma_load_3d(st + 2 * kTileA + kTileB, &mBl, &full[s], kc, nt * kBN, z);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issue: hi*hi + hi*lo + lo*hi per K step, one commit per stage
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kStages, j = kb / kStages;
            if (!mbar_wait(&full[s], j & 1)) {
                atomicOr(err, 2u);
                break;
            }
            fence_after_sync();
            unsigned char* st = smem + s * kStageBytes;
            const uint64_t ah = sw128_desc(st), al = sw128_desc(st + kTileA);
            const uint64_t bh = sw128_desc(st + 2 * kTileA), bl = sw128_desc(st + 2 * kTileA + kTileB);
#pragma unroll
            for (int kk = 0; kk < kSteps; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 32 bytes per MMA K step
                umma<TF32>(tmem, ah + adv, bh + adv, (kb | kk) != 0);
                umma<TF32>(tmem, ah + adv, bl + adv, 1u);
                umma<TF32>(tmem, al + adv, bh + adv, 1u);
            }
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    __syncwarp();

    // epilogue: each warp reads its 32 TMEM lanes (rows) and stores (re, im) column pairs
    // tcgen05.ld is warp-collective: the whole warp proceeds only if every lane saw completion
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0));
    fence_after_sync();
    if (ok) {
        const int row = mt * kBM + warp * 32 + lane;
        float2* Cz = C + sC * z;
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int n = nt * (kBN / 2) + c0 / 2 + q;
                    if (n < N) Cz[row + (int64_t)M * n] = make_float2(v[2 * q], v[2 * q + 1]);
                }
            }
        }
    } else if (lane == 0) {
        atomicOr(err, 4u);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// BF16x3 on the operand planes of tp_internal.cuh (PLANE_LEFT / PLANE_RIGHT), which the
// forward DFT writes directly for power-of-two n3 <= 64.  A is read MN-major (m contiguous,
// as the DFT lays out the spectrum), B K-major; 4-D tensor maps [slice][part][row][col]
// zero-fill the M, N and K tails, so the planes carry no padding.  One K block is 64
// elements (128 bytes); the K loop runs over part 0 (Re A against the rows [Br; Bi]) and then
// part 1 (Im A against [-Bi; Br]).  On the real slices (0 and n3 / 2) Im A is zero and the
// loop stops after part 0.  The kernel is persistent, with two accumulators (below).
// ---------------------------------------------------------------------------------------
constexpr int kHalfA = 64 * kRowBytes;  // 64 k rows of one 64-element half of M: 8 KB

// Shared-memory descriptor of an MN-major tile with the 128-byte swizzle: a 128-byte row holds
// 64 consecutive m of one k, groups of 8 rows (8 k) are 1024 bytes apart (stride byte
// offset) and the second 64 m start kHalfA bytes after the first (leading byte offset).
__device__ __forceinline__ uint64_t sw128_mn_desc(const void* tile) {
    const uint64_t a = smem_u32(tile);
    uint64_t d = (a >> 4) & 0x3FFFull;
    d |= (uint64_t)(kHalfA >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// bf16 x bf16 -> FP32, A MN-major (transpose-A bit), B K-major, M = kBM, N = kBN.
__device__ __forceinline__ void umma_bf16_mn(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc(1) | (1u << 15)), "r"(acc));
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
        "r"(c3)
        : "memory");
}

constexpr int kPThreads = 256;         // 8 warps: TMA, MMA, two idle, four for the epilogue
constexpr uint32_t kPTmemCols = 512;   // two 256-column accumulators

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent: min(tiles, SMs) CTAs, CTA b taking tiles b, b + gridDim.x, ... of the
// (m tile, n tile, slice) grid, m tile fastest.  Lane 0 of warp 0 streams the K blocks of all
// its tiles through the two-stage ring; lane 0 of warp 1 issues the MMAs of tile i into
// accumulator i % 2 (TMEM columns 256 (i % 2) ..), once the epilogue has drained the tile
// two before; warps 4..7 (TMEM lanes 32 (w - 4) ..) drain each finished accumulator to C and
// release it.  So the epilogue of one tile overlaps the main loop of the next.  nk =
// ceil(K/64) K blocks per part; zr1 = n3 / 2 for even n3 (the second real slice), else -1.
// Every wait is bounded: a role that times out records an error bit and stops, and the
// roles waiting on it time out in turn.
__global__ void __launch_bounds__(kPThreads, 1) cgemm_bf16x3_kernel(
    const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
    float2* __restrict__ C, int M, int N, int64_t sC, int nk, int zr1, int mtiles, int ntiles,
    int tiles, uint32_t* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;  // accumulator b filled (MMA commit)
    uint64_t* acce = accf + 2;         // accumulator b drained (four epilogue warps)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (*reinterpret_cast<volatile uint32_t*>(err) != 0u) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kPTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    auto slice_of = [&](int t) { return t / (mtiles * ntiles); };

    if (warp == 0 && lane == 0) {
        int g = 0;  // K blocks issued by this CTA so far (ring position)
        bool bad = false;
        for (int t = blockIdx.x; t < tiles && !bad; t += gridDim.x) {
            const int mt = t % mtiles, nt = (t / mtiles) % ntiles, z = slice_of(t);
            const int nkb = (z == 0 || z == zr1) ? nk : 2 * nk;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = g % kStages, j = g / kStages;
                if (j > 0 && !mbar_wait(&empty[s], (j - 1) & 1)) {
                    atomicOr(err, 2u);
                    bad = true;
                    break;
                }
                unsigned char* st = smem + s * kStageBytes;
                mbar_expect_tx(&full[s], kStageBytes);
                const int part = kb >= nk ? 1 : 0;
                const int k0 = (kb - part * nk) * 64;
                const int m0 = mt * kBM;
                tma_load_4d(st, &mAh, &full[s], m0, k0, part, z);
                tma_load_4d(st + kHalfA, &mAh, &full[s], m0 + 64, k0, part, z);
                tma_load_4d(st + kTileA, &mAl, &full[s], m0, k0, part, z);
                tma_load_4d(st + kTileA + kHalfA, &mAl, &full[s], m0 + 64, k0, part, z);
                tma_load_4d(st + 2 * kTileA, &mBh, &full[s], k0, nt * kBN, part, z);
                tma_load_4d(st + 2 * kTileA + kTileB, &mBl, &full[s], k0, nt * kBN, part, z);
            }
        }
    } else if (warp == 1 && lane == 0) {
        int g = 0, i = 0;
        bool bad = false;
        for (int t = blockIdx.x; t < tiles && !bad; t += gridDim.x, ++i) {
            const int z = slice_of(t);
            const int nkb = (z == 0 || z == zr1) ? nk : 2 * nk;
            const int b = i & 1;
            if (i >= 2 && !mbar_wait(&acce[b], ((i >> 1) - 1) & 1)) {
                atomicOr(err, 2u);
                break;
            }
            fence_after_sync();
            const uint32_t acc = tmem + (uint32_t)(b * kBN);
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const int s = g % kStages, j = g / kStages;
                if (!mbar_wait(&full[s], j & 1)) {
                    atomicOr(err, 2u);
                    bad = true;
                    break;
                }
                fence_after_sync();
                unsigned char* st = smem + s * kStageBytes;
                const uint64_t ah = sw128_mn_desc(st), al = sw128_mn_desc(st + kTileA);
                const uint64_t bh = sw128_desc(st + 2 * kTileA), bl = sw128_desc(st + 2 * kTileA + kTileB);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t aadv = (uint64_t)(kk * 16 * kRowBytes) >> 4;  // 16 k rows
                    const uint64_t badv = (uint64_t)(kk * 32) >> 4;              // 16 k elements
                    umma_bf16_mn(acc, ah + aadv, bh + badv, (kb | kk) != 0);
                    umma_bf16_mn(acc, ah + aadv, bl + badv, 1u);
                    umma_bf16_mn(acc, al + aadv, bh + badv, 1u);
                }
                umma_commit(&empty[s]);
            }
            if (bad) break;
            umma_commit(&accf[b]);
        }
    } else if (warp >= 4) {
        const int q = warp - 4;  // TMEM lanes 32 q .. 32 q + 31 = rows of the tile
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const int mt = t % mtiles, nt = (t / mtiles) % ntiles, z = slice_of(t);
            const int b = i & 1;
            // tcgen05.ld is warp-collective: the whole warp proceeds only if every lane saw it
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&accf[b], (i >> 1) & 1));
            if (!ok) {
                if (lane == 0) atomicOr(err, 4u);
                break;
            }
            fence_after_sync();
            const int row = mt * kBM + q * 32 + lane;
            float2* Cz = C + sC * z;
#pragma unroll 1
            for (int c0 = 0; c0 < kBN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kBN + c0), v);
                if (row < M) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int n = nt * (kBN / 2) + c0 / 2 + k;
                        if (n < N) Cz[row + (int64_t)M * n] = make_float2(v[2 * k], v[2 * k + 1]);
                    }
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
    }
    __syncwarp();
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kPTmemCols)
                     : "memory");
    }
}

// Fills the planes of one operand from its complex spectrum X (P tubes x nslices).
__global__ void __launch_bounds__(256) planes_from_spectrum_kernel(const float2* __restrict__ X,
                                                                   FftJob J, int nslices) {
    const int64_t total = J.P * nslices;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(i / J.P);
        const int64_t p = i - (int64_t)z * J.P;
        store_plane_value(J, plane_cursor(J, p), z, __ldg(X + i));
    }
}

// ---------------------------------------------------------------------------------------
// Host side: tensor maps and launches.
// ---------------------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 3-D map over [slices][rows][row_elems] with a box of one 128-byte K block x box_rows rows.
bool make_map(CUtensorMap* map, void* base, bool tf32, int64_t row_elems, int64_t rows,
              int64_t slices, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int64_t esz = tf32 ? 4 : 2;
    cuuint64_t dims[3] = {(cuuint64_t)row_elems, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)(row_elems * esz), (cuuint64_t)(row_elems * esz * rows)};
    cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                    base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <bool TF32>
cudaError_t run_tc(const float2* Ab, const float2* Bb, float2* Cb, int M, int N, int K,
                   int nslices, void* planes, uint32_t* err, cudaStream_t s) {
    using T = typename Split<TF32>::T;
    const int Mp = (M + kBM - 1) / kBM * kBM;
    const int Np = (N + 127) / 128 * 128;
    const int kb = TF32 ? 32 : 64;  // K elements per 128-byte block
    const int Kp = (K + kb - 1) / kb * kb;
    T* base = static_cast<T*>(planes);
    const int64_t pa = (int64_t)Mp * 2 * Kp * nslices, pb = (int64_t)2 * Np * 2 * Kp * nslices;
    T *ahi = base, *alo = base + pa, *bhi = base + 2 * pa, *blo = base + 2 * pa + pb;
    split_a_kernel<TF32><<<dim3(Kp / 32, Mp / 32, nslices), dim3(32, 8), 0, s>>>(Ab, ahi, alo, M, K,
                                                                                 Mp, Kp);
    split_b_kernel<TF32><<<dim3(Kp / 32, Np / 8, nslices), dim3(32, 8), 0, s>>>(Bb, bhi, blo, K, N,
                                                                                Kp, Np);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap mah, mal, mbh, mbl;
    if (!make_map(&mah, ahi, TF32, 2 * Kp, Mp, nslices, kBM) ||
        !make_map(&mal, alo, TF32, 2 * Kp, Mp, nslices, kBM) ||
        !make_map(&mbh, bhi, TF32, 2 * Kp, 2 * Np, nslices, kBN) ||
        !make_map(&mbl, blo, TF32, 2 * Kp, 2 * Np, nslices, kBN))
        return cudaErrorInvalidValue;
    auto k = cgemm_tc_kernel<TF32>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    const int nkb = 2 * Kp / kb;
    k<<<dim3(Mp / kBM, 2 * Np / kBN, nslices), kThreads, kSmemBytes, s>>>(
        mah, mal, mbh, mbl, Cb, M, N, (int64_t)M * N, nkb, err);
    return cudaGetLastError();
}

// 4-D map over [slices][parts][rows][cols] of bf16 with row pitch `pitch` elements and a
// box of 64 columns (128 bytes) x box_rows rows; elements beyond cols or rows read as zero.
bool make_map4(CUtensorMap* map, void* base, int64_t cols, int64_t rows, int64_t pitch,
               int64_t slices, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, 2, (cuuint64_t)slices};
    cuuint64_t strides[3] = {(cuuint64_t)(pitch * 2), (cuuint64_t)(pitch * 2 * rows),
                             (cuuint64_t)(pitch * 2 * rows * 2)};
    cuuint32_t box[4] = {64, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

int64_t bf16_plane_pitch(int rows) { return ((int64_t)rows + 7) / 8 * 8; }

int64_t bf16_left_plane_elems(int M, int K, int nslices) {
    return bf16_plane_pitch(M) * 2 * (int64_t)K * nslices;
}

int64_t bf16_right_plane_elems(int N, int K, int nslices) {
    return bf16_plane_pitch(K) * 2 * (2 * (int64_t)N) * nslices;
}

cudaError_t bf16_planes_from_spectrum(const float2* A, const float2* B, int M, int N, int K,
                                      int nslices, void* planes, cudaStream_t s) {
    uint16_t* base = static_cast<uint16_t*>(planes);
    const int64_t la = bf16_left_plane_elems(M, K, nslices), lb = bf16_right_plane_elems(N, K, nslices);
    FftJob ja{}, jb{};
    ja.P = (int64_t)M * K;
    ja.plane_kind = PLANE_LEFT;
    ja.plane_rows = M;
    ja.plane_pitch = bf16_plane_pitch(M);
    ja.plane_hi = base;
    ja.plane_lo = base + la;
    jb.P = (int64_t)K * N;
    jb.plane_kind = PLANE_RIGHT;
    jb.plane_rows = K;
    jb.plane_pitch = bf16_plane_pitch(K);
    jb.plane_hi = base + 2 * la;
    jb.plane_lo = base + 2 * la + lb;
    int sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = 8 * sms;
    planes_from_spectrum_kernel<<<grid, 256, 0, s>>>(A, ja, nslices);
    planes_from_spectrum_kernel<<<grid, 256, 0, s>>>(B, jb, nslices);
    return cudaGetLastError();
}

cudaError_t launch_cgemm_bf16x3(const void* planes, float2* C, int M, int N, int K, int nslices,
                                int n3, uint32_t* err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0 || nslices <= 0) return cudaSuccess;
    uint16_t* base = static_cast<uint16_t*>(const_cast<void*>(planes));
    const int64_t la = bf16_left_plane_elems(M, K, nslices), lb = bf16_right_plane_elems(N, K, nslices);
    const int64_t pa = bf16_plane_pitch(M), pb = bf16_plane_pitch(K);
    CUtensorMap mah, mal, mbh, mbl;
    if (!make_map4(&mah, base, M, K, pa, nslices, 64) ||
        !make_map4(&mal, base + la, M, K, pa, nslices, 64) ||
        !make_map4(&mbh, base + 2 * la, K, 2 * (int64_t)N, pb, nslices, kBN) ||
        !make_map4(&mbl, base + 2 * la + lb, K, 2 * (int64_t)N, pb, nslices, kBN))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(cgemm_bf16x3_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    const int nk = (K + 63) / 64;
    const int zr1 = (n3 % 2 == 0) ? n3 / 2 : -1;
    const int mtiles = (M + kBM - 1) / kBM, ntiles = (int)((2 * (int64_t)N + kBN - 1) / kBN);
    const int64_t tiles = (int64_t)mtiles * ntiles * nslices;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(tiles, sms);
    cgemm_bf16x3_kernel<<<grid, kPThreads, kSmemBytes, s>>>(
        mah, mal, mbh, mbl, C, M, N, (int64_t)M * N, nk, zr1, mtiles, ntiles, (int)tiles, err);
    return cudaGetLastError();
}

int64_t cgemm_tc_plane_bytes(int M, int N, int K, int nslices, int precision) {
    const bool tf32 = precision == TP_PREC_3XTF32;
    const int64_t esz = tf32 ? 4 : 2;
    const int64_t Mp = (M + kBM - 1) / kBM * kBM, Np = (N + 127) / 128 * 128;
    const int64_t kb = tf32 ? 32 : 64;
    const int64_t Kp = (K + kb - 1) / kb * kb;
    return esz * 2 * ((int64_t)Mp * 2 * Kp + 2 * Np * 2 * Kp) * nslices;
}

cudaError_t launch_cgemm_tc(const float2* A, const float2* B, float2* C, int M, int N, int K,
                            int nslices, int precision, void* planes, uint32_t* err,
                            cudaStream_t s) {
    if (M <= 0 || N <= 0 || nslices <= 0) return cudaSuccess;
    if (precision == TP_PREC_3XTF32)
        return run_tc<true>(A, B, C, M, N, K, nslices, planes, err, s);
    return run_tc<false>(A, B, C, M, N, K, nslices, planes, err, s);
}

}  // namespace tp
