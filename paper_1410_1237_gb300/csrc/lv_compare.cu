// lv_compare.cu -- qualitative comparison of two partitions (Sec. 5).
//
// The paper classifies every unordered vertex pair (TP: together in both
// partitions, FP: together only in p, FN: only in s, TN: apart in both) and
// notes that this takes time quadratic in n.  The counts follow from the
// contingency table instead: after sorting the (s, p) label pairs, a run of c
// equal pairs holds C(c, 2) pairs together in both (TP); runs of equal s
// labels (contiguous after the same sort) give the pairs together in s, and
// runs of a sort of the p labels alone those together in p.  So
// FP = together_in_p - TP, FN = together_in_s - TP and TN = C(n, 2) minus the
// three.  All counts are exact 64-bit integers (C(n, 2) < 2^61).
#include <algorithm>
#include <cstring>

#include "lv_ops.cuh"

namespace lv {
namespace {

int grid_n(int64_t items) { return grid_for(items, 256, g_num_sms * 16); }

__global__ void label_max_kernel(int n, const int32_t *__restrict__ s, const int32_t *__restrict__ p,
                                 unsigned *mx) {
    unsigned ms = 0, mp = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ms = max(ms, (unsigned)s[i]);
        mp = max(mp, (unsigned)p[i]);
    }
    ms = max(ms, __reduce_max_sync(0xffffffffu, ms));
    mp = max(mp, __reduce_max_sync(0xffffffffu, mp));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&mx[0], ms);
        atomicMax(&mx[1], mp);
    }
}

// key = s << bp | p (labels read as unsigned), and p alone
__global__ void pair_keys_kernel(int n, const int32_t *__restrict__ s, const int32_t *__restrict__ p,
                                 int bp, uint64_t *keys, uint32_t *pkeys, uint32_t *zeros) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        keys[i] = ((uint64_t)(uint32_t)s[i] << bp) | (uint32_t)p[i];
        pkeys[i] = (uint32_t)p[i];
        zeros[i] = 0u;
    }
}

// head[i] = 1 where (key[i] >> shift) starts a run of equal values
template <typename K>
__global__ void run_heads_kernel(int n, const K *__restrict__ keys, int shift, int32_t *head) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        head[i] = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift)) ? 1 : 0;
}

__global__ void run_starts_kernel(int n, const int32_t *__restrict__ head, const int32_t *__restrict__ idx,
                                  int32_t *starts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (head[i]) starts[idx[i]] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) starts[idx[n]] = n;
}

// out += sum over runs of C(length, 2)
__global__ void run_pairs_kernel(int runs, const int32_t *__restrict__ starts,
                                 unsigned long long *out) {
    unsigned long long acc = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < runs; r += gridDim.x * blockDim.x) {
        const unsigned long long c = (unsigned long long)(starts[r + 1] - starts[r]);
        acc += c * (c - 1) / 2;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// pairs within runs of equal (keys >> shift); keys sorted so that runs are contiguous
template <typename K>
lv_status pairs_in_runs(int n, const K *keys, int shift, int32_t *head, int32_t *starts,
                        unsigned long long *out, int *pinned, cudaStream_t s) {
    run_heads_kernel<K><<<grid_n(n), 256, 0, s>>>(n, keys, shift, head);
    LV_LAUNCH_CHECK();
    int32_t *idx = starts + n + 2;  // second half of the scratch
    LV_TRY(scan_excl_i32(head, idx, n, s));
    run_starts_kernel<<<grid_n(n), 256, 0, s>>>(n, head, idx, starts);
    LV_LAUNCH_CHECK();
    LV_CUDA(cudaMemcpyAsync(pinned, idx + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const int runs = pinned[0];
    run_pairs_kernel<<<grid_n(runs), 256, 0, s>>>(runs, starts, out);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

}  // namespace
}  // namespace lv

using namespace lv;

extern "C" lv_status lv_compare_partitions(int64_t n, const int32_t *labels_s,
                                           const int32_t *labels_p, int ptrs_on_device,
                                           lv_partition_compare *out, void *cuda_stream) {
    if (!out || n < 0 || n > 0x7ffffffell || (n > 0 && (!labels_s || !labels_p))) return LV_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    out->sp = out->se = out->oq = out->rand = 1.0;
    if (n < 2) return LV_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    LV_TRY(ensure_setup(s));
    struct Bufs {
        cudaStream_t s;
        int32_t *ls = nullptr, *lp = nullptr, *head = nullptr, *starts = nullptr;
        uint64_t *keys = nullptr, *keys_alt = nullptr;
        uint32_t *pk = nullptr, *pk_alt = nullptr, *z = nullptr, *z_alt = nullptr;
        unsigned long long *cnt = nullptr;
        unsigned *mx = nullptr;
        int *pinned = nullptr;
        ~Bufs() {
            dfree(ls, s);
            dfree(lp, s);
            dfree(head, s);
            dfree(starts, s);
            dfree(keys, s);
            dfree(keys_alt, s);
            dfree(pk, s);
            dfree(pk_alt, s);
            dfree(z, s);
            dfree(z_alt, s);
            dfree(cnt, s);
            dfree(mx, s);
            if (pinned) {
                cudaStreamSynchronize(s);
                cudaFreeHost(pinned);
            }
        }
    } b;
    b.s = s;
    const int N = (int)n;
    if (cudaMallocHost((void **)&b.pinned, 64 * sizeof(int)) != cudaSuccess) return LV_ERR_OOM;
    const int32_t *ds = labels_s, *dp = labels_p;
    if (!ptrs_on_device) {
        LV_TRY(dalloc_n(&b.ls, (size_t)N, s));
        LV_TRY(dalloc_n(&b.lp, (size_t)N, s));
        LV_CUDA(cudaMemcpyAsync(b.ls, labels_s, sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
        LV_CUDA(cudaMemcpyAsync(b.lp, labels_p, sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
        ds = b.ls;
        dp = b.lp;
    }
    LV_TRY(dalloc_n(&b.mx, 2, s));
    LV_TRY(dalloc_n(&b.cnt, 3, s));
    LV_CUDA(cudaMemsetAsync(b.mx, 0, 2 * sizeof(unsigned), s));
    LV_CUDA(cudaMemsetAsync(b.cnt, 0, 3 * sizeof(unsigned long long), s));
    label_max_kernel<<<grid_n(N), 256, 0, s>>>(N, ds, dp, b.mx);
    LV_LAUNCH_CHECK();
    unsigned mxh[2];
    LV_CUDA(cudaMemcpyAsync(b.pinned, b.mx, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    std::memcpy(mxh, b.pinned, sizeof mxh);
    const int bs = std::max(1, bits_for(mxh[0])), bp = std::max(1, bits_for(mxh[1]));
    LV_TRY(dalloc_n(&b.keys, (size_t)N, s));
    LV_TRY(dalloc_n(&b.keys_alt, (size_t)N, s));
    LV_TRY(dalloc_n(&b.pk, (size_t)N, s));
    LV_TRY(dalloc_n(&b.pk_alt, (size_t)N, s));
    LV_TRY(dalloc_n(&b.z, (size_t)N, s));
    LV_TRY(dalloc_n(&b.z_alt, (size_t)N, s));
    LV_TRY(dalloc_n(&b.head, (size_t)N + 1, s));
    LV_TRY(dalloc_n(&b.starts, 2 * (size_t)N + 4, s));
    pair_keys_kernel<<<grid_n(N), 256, 0, s>>>(N, ds, dp, bp, b.keys, b.pk, b.z);
    LV_LAUNCH_CHECK();
    LV_TRY(radix_sort_u64(b.keys, b.z, b.keys_alt, b.z_alt, N, bs + bp, s));
    LV_TRY(pairs_in_runs<uint64_t>(N, b.keys, 0, b.head, b.starts, b.cnt + 0, b.pinned, s));   // TP
    LV_TRY(pairs_in_runs<uint64_t>(N, b.keys, bp, b.head, b.starts, b.cnt + 1, b.pinned, s));  // in s
    LV_TRY(radix_sort_u32(b.pk, b.z, b.pk_alt, b.z_alt, N, bp, s));
    LV_TRY(pairs_in_runs<uint32_t>(N, b.pk, 0, b.head, b.starts, b.cnt + 2, b.pinned, s));     // in p
    unsigned long long c[3];
    LV_CUDA(cudaMemcpyAsync(b.pinned, b.cnt, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    std::memcpy(c, b.pinned, sizeof c);
    const uint64_t total = (uint64_t)N * (uint64_t)(N - 1) / 2;
    out->tp = c[0];
    out->fn = c[1] - c[0];
    out->fp = c[2] - c[0];
    out->tn = total - out->tp - out->fp - out->fn;
    auto ratio = [](uint64_t a, uint64_t d) { return d ? (double)a / (double)d : 1.0; };
    out->sp = ratio(out->tp, out->tp + out->fp);
    out->se = ratio(out->tp, out->tp + out->fn);
    out->oq = ratio(out->tp, out->tp + out->fp + out->fn);
    out->rand = ratio(out->tp + out->tn, total);
    return LV_OK;
}
