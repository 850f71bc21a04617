// lv_noalloc.cu -- modularity of a given labelling without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// modularity value: services that hand the whole device to a fixed-size
// memory pool at start-up and forbid further cudaMalloc calls (a second
// allocator would fail or fragment the pool), and hosts that must keep a
// strict, pre-computed device-memory budget.  lv_modularity_noalloc serves
// them: its only scratch is a file-scope __device__ array of fixed size that
// exists from the moment the library is loaded, so the call performs no
// cudaMalloc, no cudaFree and no allocating library call.  It waits for its
// stream (cudaStreamSynchronize) before it returns the numerator.
//
// Scratch layout (u64): [0, kNoAllocMaxN) community degrees a_c, then the
// accumulators 2m, sum of intra-community weights, sum of a_c^2 and an error
// flag.  Every call clears what it uses, so earlier contents do not matter,
// but all calls share the array: calls whose GPU work overlaps (different
// streams, or different host threads on the same device) race and must be
// serialised by the caller.
#include <cstring>
#include <mutex>

#include "lv_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxN = 1 << 20;  // largest n accepted
constexpr int kAcc = 64;                   // accumulator words after the a_c array
enum { kTwoM = 0, kEin = 1, kA2 = 2, kErr = 3 };

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocMaxN + kAcc];

// per-device address of the scratch array, looked up once per device (the
// first call on a device, under that device's once-flag).  The cached address
// belongs to the device's primary context: after cudaDeviceReset it is stale.
constexpr int kMaxDevices = 64;
unsigned long long *g_scratch_ptr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];

__global__ void noalloc_clear_kernel(unsigned long long *scr, int n) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        scr[c] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x < kAcc) scr[kNoAllocMaxN + threadIdx.x] = 0ull;
}

// one warp per row: k_i, a_{C(i)} += k_i, intra-community weight (Eq. 3, with
// a self-loop counted once as intra-community weight)
__global__ void __launch_bounds__(256) noalloc_rows_kernel(int n, const int64_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ col,
                                                           const int32_t *__restrict__ w,
                                                           const int32_t *__restrict__ labels,
                                                           unsigned long long *scr) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    unsigned long long k_acc = 0, e_acc = 0;
    int bad = 0;
    for (int64_t i = blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += nw) {
        const int ci = labels[i];
        if (ci < 0 || ci >= n) {
            bad = 1;
            continue;  // warp-uniform: every lane read the same label
        }
        long long k = 0, e = 0;
        for (int64_t a = rowptr[i] + lane; a < rowptr[i + 1]; a += 32) {
            const int j = col[a];
            const int wt = w[a];
            k += wt;
            if (j >= 0 && j < n) {
                if (labels[j] == ci) e += wt;
            } else {
                bad = 1;
            }
        }
        k = lv::warp_sum(k);
        e = lv::warp_sum(e);
        if (lane == 0) {
            atomicAdd(&scr[ci], (unsigned long long)k);
            k_acc += (unsigned long long)k;
            e_acc += (unsigned long long)e;
        }
    }
    if (lane == 0) {
        if (k_acc) atomicAdd(&scr[kNoAllocMaxN + kTwoM], k_acc);
        if (e_acc) atomicAdd(&scr[kNoAllocMaxN + kEin], e_acc);
    }
    if (bad) atomicOr(&scr[kNoAllocMaxN + kErr], 1ull);
}

__global__ void __launch_bounds__(256) noalloc_a2_kernel(int n, unsigned long long *scr) {
    __shared__ long long red[8];
    long long acc = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const long long a = (long long)scr[c];
        acc += a * a;
    }
    acc = lv::block_sum_256(acc, red);
    if (threadIdx.x == 0 && acc) atomicAdd(&scr[kNoAllocMaxN + kA2], (unsigned long long)acc);
}

}  // namespace

extern "C" lv_status lv_modularity_noalloc(int64_t n, const int64_t *rowptr, const int32_t *col,
                                           const int32_t *w, const int32_t *labels,
                                           int64_t *num_hi, uint64_t *num_lo, int64_t *den,
                                           void *cuda_stream) {
    if (n <= 0 || !rowptr || !col || !w || !labels || !num_hi || !num_lo || !den)
        return LV_ERR_ARG;
    if (n > kNoAllocMaxN) return LV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LV_ERR_ARG;
    // one-time set-up on this device: the host-side name of the array is not
    // a device address, so look the address up with the device current
    std::call_once(g_scratch_once[dev], [dev] {
        void *p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
    });
    LV_CUDA(g_scratch_err[dev]);
    if (!g_scratch_ptr[dev]) return LV_ERR_CUDA;
    unsigned long long *scr = g_scratch_ptr[dev];
    int nsm = 0;
    LV_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int ni = (int)n;
    noalloc_clear_kernel<<<nsm * 4, 256, 0, s>>>(scr, ni);
    LV_CUDA(cudaGetLastError());
    noalloc_rows_kernel<<<nsm * 16, 256, 0, s>>>(ni, rowptr, col, w, labels, scr);
    LV_CUDA(cudaGetLastError());
    noalloc_a2_kernel<<<nsm * 4, 256, 0, s>>>(ni, scr);
    LV_CUDA(cudaGetLastError());
    unsigned long long acc[4];
    LV_CUDA(cudaMemcpyAsync(acc, scr + kNoAllocMaxN, sizeof acc, cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    if (acc[kErr]) return LV_ERR_ARG;
    const long long two_m = (long long)acc[kTwoM];
    if (two_m == 0) return LV_ERR_EMPTY;
    if (two_m >= (1ll << 31)) return LV_ERR_OVERFLOW;
    // N = 2m * sum e_{i->C(i)} - sum a_C^2; |N| <= (2m)^2 < 2^62
    const long long N = two_m * (long long)acc[kEin] - (long long)acc[kA2];
    *num_hi = N < 0 ? -1 : 0;
    *num_lo = (uint64_t)N;
    *den = two_m * two_m;
    return LV_OK;
}
