// lv_prims.cu -- error state, device memory pool, prefix scan and radix sort.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lv_internal.cuh"

namespace lv {

int g_num_sms = 0;
static TraceBuf g_trace;
TraceBuf trace_buffer() {
#ifdef LV_TRACE
    if (!g_trace.buf) {
        cudaMalloc(&g_trace.buf, sizeof(unsigned long long) * kTraceCap);
        cudaMalloc(&g_trace.n, sizeof(unsigned int));
        cudaMemset(g_trace.n, 0, sizeof(unsigned int));
    }
#endif
    return g_trace;
}
std::atomic<unsigned long long> g_kernel_launches{0};

// --------------------------------------------------------------- errors
static thread_local char t_last_error[512] = "";

void set_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    std::snprintf(t_last_error, sizeof t_last_error, "%s: %s (%s:%d)", cudaGetErrorString(e),
                  what, file, line);
}

// ------------------------------------------------------------------ pool
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];
static bool g_pool_init[64];

static lv_status pool_for_current(cudaMemPool_t *out) {
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return LV_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_init[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        LV_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
        uint64_t thresh = UINT64_MAX;
        LV_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thresh));
        int nsm = 0;
        LV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        g_num_sms = nsm;
        g_pool_init[dev] = true;
    }
    *out = g_pools[dev];
    return LV_OK;
}

lv_status dalloc(void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    LV_TRY(pool_for_current(&pool));
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMallocFromPoolAsync", __FILE__, __LINE__);
        cudaGetLastError();
        *p = nullptr;
        return LV_ERR_OOM;
    }
    return LV_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ------------------------------------------------------------------ scan
namespace {
constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

// exclusive scan over a 256-thread block; *total gets the block sum
__device__ __forceinline__ int block_excl_scan_256(int v, int *total) {
    __shared__ int warp_tot[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int wofs = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int t = warp_tot[i];
        if (i < w) wofs += t;
        tot += t;
    }
    __syncthreads();
    *total = tot;
    return wofs + x - v;
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const int32_t *__restrict__ in,
                                                                 int64_t n, int32_t *bsum) {
    __shared__ int red[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j * kScanBlock + threadIdx.x;
        if (i < n) s += in[i];
    }
    s = block_sum_256(s, red);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanBlock) scan_tile_kernel(const int32_t *in, int32_t *out,
                                                               int64_t n, const int32_t *boff,
                                                               int64_t nblocks) {
    __shared__ int sm[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = j * kScanBlock + threadIdx.x;
        sm[idx] = (base + idx < n) ? in[base + idx] : 0;
    }
    __syncthreads();
    int loc[kScanItems];
    int t = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        loc[j] = sm[threadIdx.x * kScanItems + j];
        t += loc[j];
    }
    int total = 0;
    int run = block_excl_scan_256(t, &total) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        sm[threadIdx.x * kScanItems + j] = run;
        run += loc[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int idx = j * kScanBlock + threadIdx.x;
        if (base + idx < n) out[base + idx] = sm[idx];
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) out[n] = boff ? boff[nblocks] : total;
}
}  // namespace

lv_status scan_excl_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        LV_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return LV_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        scan_tile_kernel<<<1, kScanBlock, 0, s>>>(in, out, n, nullptr, 1);
        LV_LAUNCH_CHECK();
        return LV_OK;
    }
    int32_t *bsum = nullptr;
    LV_TRY(dalloc_n(&bsum, nb + 1, s));
    scan_reduce_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, bsum);
    LV_LAUNCH_CHECK();
    lv_status st = scan_excl_i32(bsum, bsum, nb, s);
    if (st == LV_OK) {
        scan_tile_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, bsum, nb);
        ++g_kernel_launches;
        if (cudaGetLastError() != cudaSuccess) st = LV_ERR_CUDA;
    }
    dfree(bsum, s);
    return st;
}

// ------------------------------------------------------------ radix sort
// LSD radix sort, 8-bit digits.  Per pass: a per-tile digit histogram, an
// exclusive scan of the histograms in digit-major order, and a stable
// scatter.  Within a tile, each warp ranks its 512 items in order (match_any
// groups the lanes that share a digit) and warps are combined by a per-digit
// prefix over the warps, so equal keys keep their input order.
namespace {
constexpr int kRsBlock = 256;
constexpr int kRsRounds = 16;
constexpr int kRsWarpItems = 32 * kRsRounds;
constexpr int kRsTile = 8 * kRsWarpItems;  // 4096

template <typename K>
__global__ void __launch_bounds__(kRsBlock) rs_hist_kernel(const K *__restrict__ keys, int n,
                                                           int shift, int32_t *hist, int ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kRsTile;
    const int end = min(base + kRsTile, n);
    for (int i = base + threadIdx.x; i < end; i += kRsBlock)
        atomicAdd(&h[(int)((keys[i] >> shift) & 255u)], 1);
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kRsBlock) rs_scatter_kernel(const K *__restrict__ kin,
                                                              const uint32_t *__restrict__ vin,
                                                              K *kout, uint32_t *vout, int n,
                                                              int shift,
                                                              const int32_t *__restrict__ hoff,
                                                              int ntiles) {
    __shared__ int wcnt[8][256];
    __shared__ int goff[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = 0; i < 8; ++i) wcnt[i][threadIdx.x] = 0;
    goff[threadIdx.x] = hoff[threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const int base = blockIdx.x * kRsTile + w * kRsWarpItems;
    const unsigned lt = (1u << lane) - 1u;
    K kr[kRsRounds];
    uint32_t vr[kRsRounds];
    int rk[kRsRounds];
    int dg[kRsRounds];
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int idx = base + r * 32 + lane;
        const bool valid = idx < n;
        kr[r] = valid ? kin[idx] : (K)0;
        vr[r] = valid ? vin[idx] : 0u;
        const int d = valid ? (int)((kr[r] >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = (valid ? wcnt[w][d] : 0);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rk[r] = before + __popc(peers & lt);
        dg[r] = d;
    }
    __syncthreads();
    {
        int run = 0;
        for (int i = 0; i < 8; ++i) {
            const int t = wcnt[i][threadIdx.x];
            wcnt[i][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int d = dg[r];
        if (d < 256) {
            const int pos = goff[d] + wcnt[w][d] + rk[r];
            kout[pos] = kr[r];
            vout[pos] = vr[r];
        }
    }
}

template <typename K>
lv_status radix_sort_impl(K *keys, uint32_t *vals, K *kalt, uint32_t *valt, int n, int nbits,
                          cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return LV_OK;
    const int ntiles = (n + kRsTile - 1) / kRsTile;
    int32_t *hist = nullptr;
    LV_TRY(dalloc_n(&hist, (size_t)256 * ntiles + 1, s));
    K *ks = keys, *kd = kalt;
    uint32_t *vs = vals, *vd = valt;
    lv_status st = LV_OK;
    for (int shift = 0; shift < nbits && st == LV_OK; shift += 8) {
        rs_hist_kernel<K><<<ntiles, kRsBlock, 0, s>>>(ks, n, shift, hist, ntiles);
        ++g_kernel_launches;
        if (cudaGetLastError() != cudaSuccess) { st = LV_ERR_CUDA; break; }
        st = scan_excl_i32(hist, hist, (int64_t)256 * ntiles, s);
        if (st != LV_OK) break;
        rs_scatter_kernel<K><<<ntiles, kRsBlock, 0, s>>>(ks, vs, kd, vd, n, shift, hist, ntiles);
        ++g_kernel_launches;
        if (cudaGetLastError() != cudaSuccess) { st = LV_ERR_CUDA; break; }
        K *tk = ks; ks = kd; kd = tk;
        uint32_t *tv = vs; vs = vd; vd = tv;
    }
    if (st == LV_OK && ks != keys) {
        cudaError_t e1 = cudaMemcpyAsync(keys, ks, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(vals, vs, (size_t)n * sizeof(uint32_t),
                                         cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = LV_ERR_CUDA;
    }
    dfree(hist, s);
    return st;
}
}  // namespace

lv_status radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                         int n, int nbits, cudaStream_t s) {
    return radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, nbits, s);
}
lv_status radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                         int n, int nbits, cudaStream_t s) {
    return radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, nbits > 32 ? 32 : nbits, s);
}

}  // namespace lv

extern "C" const char *lv_last_error(void) { return lv::t_last_error; }

namespace lv {
namespace {
// The grid barrier's wait (arrive with a release add on the one-word
// barrier, poll it with acquire loads, give up after `limit` polls and raise
// flag 1; see grid_sync) with block 0 never arriving.
__global__ void wait_check_kernel(GridBarrier *bar, unsigned long long limit) {
    if (blockIdx.x == 0) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long target = gridDim.x;  // the first barrier of the launch
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(&bar->word) : "memory");
        for (unsigned long long spins = 0;;) {
            unsigned long long w;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(&bar->word) : "memory");
            if (w >> kBarrierFlagShift) break;
            if ((w & kBarrierCountMask) >= target) break;
            if (++spins > limit) {
                barrier_raise(bar, 1);
                break;
            }
            __nanosleep(20);
        }
    }
    __syncthreads();
}
}  // namespace
}  // namespace lv

extern "C" lv_status lv_check_bounded_wait(int32_t polls) {
    using namespace lv;
    if (polls < 1 || polls > (1 << 24)) return LV_ERR_ARG;
    GridBarrier *bar = nullptr;
    LV_CUDA(cudaMalloc(&bar, sizeof(GridBarrier)));
    lv_status st = LV_OK;
    GridBarrier h;
    if (cudaMemset(bar, 0, sizeof(GridBarrier)) != cudaSuccess) st = LV_ERR_CUDA;
    if (st == LV_OK) {
        wait_check_kernel<<<4, 32>>>(bar, (unsigned long long)polls);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(&h, bar, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LV_ERR_CUDA;
    }
    cudaFree(bar);
    if (st != LV_OK) return st;
    return (barrier_flags(h) & 1) ? LV_ERR_TIMEOUT : LV_ERR_STATE;
}

#ifdef LV_TRACE
namespace lv {
namespace {
__global__ void trace_stamp_kernel(TraceBuf tb, unsigned tag, unsigned long long val) {
    trace4(tb, 0xA00000000ull | tag, gtimer(), val, 0);
}
}  // namespace
void trace_stamp(cudaStream_t s, unsigned tag, unsigned long long val) {
    trace_stamp_kernel<<<1, 1, 0, s>>>(trace_buffer(), tag, val);
}
}  // namespace lv
// profiling builds only: read and reset the stage timestamps
extern "C" int lv_trace_read(unsigned long long *out, int max) {
    lv::TraceBuf tb = lv::trace_buffer();
    unsigned int n = 0;
    cudaDeviceSynchronize();
    cudaMemcpy(&n, tb.n, sizeof n, cudaMemcpyDeviceToHost);
    if (n > lv::kTraceCap) n = lv::kTraceCap;
    if ((int)n > max) n = (unsigned)max;
    cudaMemcpy(out, tb.buf, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    return (int)n;
}
extern "C" void lv_trace_reset(void) {
    lv::TraceBuf tb = lv::trace_buffer();
    cudaDeviceSynchronize();
    cudaMemset(tb.n, 0, sizeof(unsigned int));
    cudaMemset(tb.buf, 0, sizeof(unsigned long long) * lv::kTraceCap);
}
extern "C" void lv_trace_read_region(unsigned long long *out, int offset, int count) {
    lv::TraceBuf tb = lv::trace_buffer();
    cudaDeviceSynchronize();
    cudaMemcpy(out, tb.buf + offset, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
}
#endif
