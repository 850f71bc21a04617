// lv_internal.cuh -- shared declarations of the CUDA implementation.
//
// Device data layout (all in HBM):
//   graph   off   int32[n+1]   row offsets (arcs < 2^31 because 2m < 2^31, w >= 1)
//           arcs  int2[A]      {col, w} interleaved, so one 8-byte load brings
//                              both halves of an arc and rows stream as 16-byte
//                              vectors
//   vertex  k     int32[n]     weighted degree (Sec. 2), < 2m < 2^31
//           loop  int32[n]     self-loop weight (0 if none)
//           C     int32[n]     community label; labels are vertex ids of G_p
//   community comm u64[n]      packed {a_C (low 32 bits), |C| (high 32 bits)};
//                              one 8-byte gather serves the gain (a_C) and the
//                              singlet rule (|C|), and one 64-bit atomicAdd
//                              moves a vertex's degree and count together
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "lv.h"

namespace lv {

constexpr int kEmpty = -1;           // empty hash slot (labels are >= 0)
// Sweep bins: 0..5 = groups of G = 1, 2, 4, 8, 16, 32 lanes per vertex,
// 6 = a quarter CTA (4 warps) per vertex, 7 = one CTA per vertex, 8 = hubs
// (several CTAs per vertex).
constexpr int kGroupBins = 6;
constexpr int kBins = 9;
constexpr int kBinSkip = kBins;      // isolated vertices (no arcs)
constexpr int kBinQuad = 6;
constexpr int kBinCta = 7;
constexpr int kBinHub = 8;
constexpr int kQuadMaxArcs = 1024;   // quarter-CTA vertices have at most this many arcs
constexpr int kLaneArcsLimit = 8;    // a group of G lanes takes <= G * lane_arcs arcs
constexpr int kWarpMaxLimit = 256;   // warp table holds 2x this
constexpr int kCtaMaxLimit = 4096;   // CTA-bin table holds 2x this (64 KB)
constexpr int kGroupTableInts = 512;  // per warp: every group's table slots
constexpr int kWarpSlots = 2 * kWarpMaxLimit;
constexpr int kCtaSlots = 2 * kCtaMaxLimit;

// ------------------------------------------------------------------ errors
void set_cuda_error(cudaError_t e, const char *what, const char *file, int line);

#define LV_CUDA(x)                                                       \
    do {                                                                 \
        cudaError_t e_ = (x);                                            \
        if (e_ != cudaSuccess) {                                         \
            ::lv::set_cuda_error(e_, #x, __FILE__, __LINE__);            \
            return e_ == cudaErrorMemoryAllocation ? LV_ERR_OOM : LV_ERR_CUDA; \
        }                                                                \
    } while (0)

#define LV_TRY(x)                         \
    do {                                  \
        lv_status s_ = (x);               \
        if (s_ != LV_OK) return s_;       \
    } while (0)

// every kernel launch is followed by this check, which also counts it (the
// counter is process-wide; a serving thread launches beside the caller's)
extern std::atomic<unsigned long long> g_kernel_launches;
#define LV_LAUNCH_CHECK()                 \
    do {                                  \
        ++::lv::g_kernel_launches;        \
        LV_CUDA(cudaGetLastError());      \
    } while (0)

// ------------------------------------------------------------------ memory
// Stream-ordered allocation from a library-owned pool (kept cached between
// calls, so repeated runs do not return memory to the driver).
lv_status dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

template <typename T>
lv_status dalloc_n(T **p, size_t count, cudaStream_t s) {
    return dalloc(reinterpret_cast<void **>(p), count * sizeof(T) + 16, s);
}

// ------------------------------------------------------------------ graph
struct DGraph {
    int32_t n = 0;
    int32_t A = 0;
    int32_t *off = nullptr;   // n+1
    int2 *arcs = nullptr;     // A
};

// ----------------------------------------------------------- device utils
__device__ __forceinline__ unsigned hash32(int c) {
    return (unsigned)c * 0x9E3779B1u;  // Fibonacci hashing (Knuth 6.4)
}

__device__ __forceinline__ int comm_a(unsigned long long v) { return (int)(unsigned)v; }
__device__ __forceinline__ int comm_size(unsigned long long v) { return (int)(v >> 32); }
__device__ __forceinline__ unsigned long long comm_pack(int a, int sz) {
    return ((unsigned long long)(unsigned)sz << 32) | (unsigned)a;
}
// delta that adds (+k, +1) / removes (-k, -1) a vertex of degree k
__device__ __forceinline__ unsigned long long comm_join(int k) {
    return (1ull << 32) + (unsigned long long)(unsigned)k;
}
__device__ __forceinline__ unsigned long long comm_leave(int k) {
    return (unsigned long long)(-(long long)((1ll << 32) + (long long)k));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a 256-thread block; result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum_256(T v, T *smem8) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem8[w] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) r += smem8[i];
    return r;
}

// Warp-wide segmented add: lane l holds (key, v); equal keys occupy
// contiguous lanes.  Each run's sum of v is added to out[key] by one atomic.
// Lanes with valid == false take no part.
__device__ __forceinline__ void warp_run_add(int key, unsigned long long v, bool valid,
                                             unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int k = valid ? key : -1 - lane;
    if (!valid) v = 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long vu = __shfl_up_sync(0xffffffffu, v, o);
        const int ku = __shfl_up_sync(0xffffffffu, k, o);
        if (lane >= o && ku == k) v += vu;
    }
    const int kn = __shfl_down_sync(0xffffffffu, k, 1);
    if (valid && v && (lane == 31 || kn != k)) atomicAdd(&out[key], v);
}

// splitmix64 output function (Steele, Lea, Flood 2014): colouring priority
__device__ __forceinline__ unsigned long long prio_hash(unsigned long long x) {
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
// pi(u) > pi(v) with pi(v) = (h(v ^ seed), v) compared lexicographically
__device__ __forceinline__ bool prio_greater(unsigned long long hu, int u, unsigned long long hv,
                                             int v) {
    return hu > hv || (hu == hv && u > v);
}

// ------------------------------------------------------------ grid barrier
// Barrier across all blocks of a cooperative (co-resident) launch.  One
// 64-bit word holds the arrivals (bits 0..47, monotonic: the k-th barrier of
// a launch completes when they reach k * gridDim.x) and error flags (bits
// 48..63).  Callers clear the word before every launch, and each block keeps
// its own count of barriers passed, so arriving is one fire-and-forget
// release add and waiting polls the word with acquire loads, which see the
// error flags in the same load.  The wait is bounded: a block that waits
// longer than the limit raises flag 1 and gets false, as does every block
// that sees a flag raised; callers then return, so a fault cannot hang the
// device.
struct alignas(8) GridBarrier {
    unsigned long long word;
};
constexpr int kBarrierFlagShift = 48;
constexpr unsigned long long kBarrierCountMask = (1ull << kBarrierFlagShift) - 1;
constexpr unsigned long long kBarrierSpinLimit = 1ull << 27;  // x ~20-100 ns sleeps

__host__ __device__ __forceinline__ int barrier_flags(const GridBarrier &b) {
    return (int)(b.word >> kBarrierFlagShift);
}

// raise error flag(s) `f` (1: a wait expired; others are the caller's)
__device__ __forceinline__ void barrier_raise(GridBarrier *gb, int f) {
    atomicOr(&gb->word, (unsigned long long)f << kBarrierFlagShift);
}

__device__ __forceinline__ void red_release_add_i32(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_acq_rel_add_i32(int *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ int ld_acquire_i32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// `passed` counts the barriers this block has completed in this launch
// (start it at 0; only thread 0's copy is used)
__device__ __forceinline__ bool grid_sync(GridBarrier *gb, unsigned &passed) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (unsigned long long)(++passed) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&gb->word) : "memory");
        unsigned long long spins = 0;
        for (;;) {
            unsigned long long w;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(&gb->word) : "memory");
            if (w >> kBarrierFlagShift) {
                ok = 0;
                break;
            }
            if ((w & kBarrierCountMask) >= target) break;
            if (++spins > kBarrierSpinLimit) {
                ok = 0;
                barrier_raise(gb, 1);
                break;
            }
            __nanosleep(20);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ----------------------------------------------------------------- tracing
// Builds with -DLV_TRACE record %globaltimer stamps at the stage boundaries
// of the persistent kernels into a device buffer (read back by a profiling
// driver); in normal builds the buffer pointer is null and the calls vanish.
struct TraceBuf {
    unsigned long long *buf = nullptr;
    unsigned int *n = nullptr;
};
#ifdef LV_TRACE
#define LV_TRACE_ON 1
#else
#define LV_TRACE_ON 0
#endif
TraceBuf trace_buffer();  // the process-wide buffer (null unless LV_TRACE)
#ifndef LV_TRACE_CAP
#define LV_TRACE_CAP (1u << 20)
#endif
constexpr unsigned kTraceCap = LV_TRACE_CAP;  // 64-bit words
// host side: record {0xA << 32 | tag, device time, val} on stream s when it
// gets there (profiling builds; nothing otherwise)
#ifdef LV_TRACE
void trace_stamp(cudaStream_t s, unsigned tag, unsigned long long val = 0);
#else
inline void trace_stamp(cudaStream_t, unsigned, unsigned long long = 0) {}
#endif
__device__ __forceinline__ unsigned long long gtimer() {
#ifdef LV_TRACE
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
#else
    return 0;
#endif
}
__device__ __forceinline__ void trace4(const TraceBuf &tb, unsigned long long a,
                                       unsigned long long b, unsigned long long c,
                                       unsigned long long d) {
#ifdef LV_TRACE
    const unsigned i = atomicAdd(tb.n, 4u);
    if (i + 4 <= kTraceCap) {
        tb.buf[i] = a;
        tb.buf[i + 1] = b;
        tb.buf[i + 2] = c;
        tb.buf[i + 3] = d;
    }
#else
    (void)tb; (void)a; (void)b; (void)c; (void)d;
#endif
}

// ------------------------------------------------------------- primitives
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total (in == out allowed).
lv_status scan_excl_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);

// Stable LSD radix sort on the low `nbits` bits of the keys, values carried.
// Sorted data ends in (keys, vals); (keys_alt, vals_alt) are scratch of the same size.
lv_status radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                         int n, int nbits, cudaStream_t s);
lv_status radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                         int n, int nbits, cudaStream_t s);

inline int bits_for(uint64_t maxval) {  // bits needed to represent values <= maxval
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

inline int grid_for(int64_t work, int per_block, int max_blocks) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

extern int g_num_sms;  // set once per process from the current device

}  // namespace lv
