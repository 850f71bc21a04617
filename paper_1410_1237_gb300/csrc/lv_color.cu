// lv_color.cu -- distance-1 colouring (Sec. 4.2) and the per-phase vertex order.
//
// Colouring: Jones-Plassmann with a hash priority pi(v) = (h(v ^ seed), v).
// Every vertex counts its higher-priority neighbours; a vertex whose count
// reaches zero takes the smallest colour not used by those neighbours, then
// decrements the counts of its lower-priority neighbours.  The result equals
// greedy colouring in decreasing priority order, whatever the timing, because
// a vertex's colour depends only on its higher-priority neighbours' colours.
// Rounds are launched in batches with device-side counts so the host only
// synchronises once per batch.
//
// Vertex order: a stable radix sort of (colour, degree bin) keys, so each
// colour class is split into the group / warp / CTA / hub bins of the sweep,
// ascending vertex id inside each bucket.
#include "lv_ops.cuh"

namespace lv {
namespace {

constexpr int kJpBatch = 8;
constexpr int kMexWindow = 1024;  // colours examined per pass of the mex search

__global__ void __launch_bounds__(256) jp_init_kernel(DGraph g, unsigned long long seed,
                                                      int32_t *cnt, int32_t *color, int32_t *list,
                                                      int32_t *list_count) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t vv = blockIdx.x * 8 + (threadIdx.x >> 5); vv < g.n; vv += nw) {
        const int v = (int)vv;
        const unsigned long long hv = prio_hash((unsigned long long)v ^ seed);
        const int beg = g.off[v], end = g.off[v + 1];
        int c = 0;
        for (int e = beg + lane; e < end; e += 32) {
            const int u = g.arcs[e].x;
            if (u != v && prio_greater(prio_hash((unsigned long long)u ^ seed), u, hv, v)) ++c;
        }
        c = warp_sum(c);
        if (lane == 0) {
            cnt[v] = c;
            color[v] = -1;
            if (c == 0) list[atomicAdd(list_count, 1)] = v;
        }
    }
}

// one warp per ready vertex
__global__ void __launch_bounds__(256) jp_round_kernel(DGraph g, unsigned long long seed,
                                                       int32_t *cnt, int32_t *color,
                                                       const int32_t *__restrict__ list_in,
                                                       const int32_t *count_in, int32_t *list_out,
                                                       int32_t *count_out, int32_t *max_color) {
    __shared__ unsigned bm_all[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned *bm = bm_all[wib];
    const unsigned lt = (1u << lane) - 1u;
    const int nin = *count_in;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t t = blockIdx.x * 8 + wib; t < nin; t += nw) {
        const int v = list_in[t];
        const unsigned long long hv = prio_hash((unsigned long long)v ^ seed);
        const int beg = g.off[v], end = g.off[v + 1];
        // smallest colour not used by a higher-priority neighbour
        int mex = -1;
        for (int base = 0; mex < 0; base += kMexWindow) {
            bm[lane] = 0u;
            __syncwarp();
            for (int e = beg + lane; e < end; e += 32) {
                const int u = g.arcs[e].x;
                if (u != v && prio_greater(prio_hash((unsigned long long)u ^ seed), u, hv, v)) {
                    const int c = color[u] - base;
                    if (c >= 0 && c < kMexWindow) atomicOr(&bm[c >> 5], 1u << (c & 31));
                }
            }
            __syncwarp();
            const unsigned word = bm[lane];
            const unsigned notfull = __ballot_sync(0xffffffffu, word != 0xffffffffu);
            if (notfull) {
                const int f = __ffs(notfull) - 1;
                const unsigned wf = __shfl_sync(0xffffffffu, word, f);
                mex = base + 32 * f + __ffs(~wf) - 1;
            }
            __syncwarp();
        }
        if (lane == 0) {
            color[v] = mex;
            atomicMax(max_color, mex);
        }
        // release lower-priority neighbours
        for (int b0 = beg; b0 < end; b0 += 32) {
            const int e = b0 + lane;
            bool ready = false;
            int u = -1;
            if (e < end) {
                u = g.arcs[e].x;
                if (u != v && prio_greater(hv, v, prio_hash((unsigned long long)u ^ seed), u))
                    ready = (atomicSub(&cnt[u], 1) == 1);
            }
            const unsigned br = __ballot_sync(0xffffffffu, ready);
            if (br) {
                int basepos = 0;
                if (lane == 0) basepos = atomicAdd(count_out, __popc(br));
                basepos = __shfl_sync(0xffffffffu, basepos, 0);
                if (ready) list_out[basepos + __popc(br & lt)] = u;
            }
        }
    }
}

__global__ void jp_carry_kernel(int32_t *counts) {
    // move the last round's output count to slot 0, clear the others
    const int last = counts[kJpBatch];
    __syncthreads();
    if (threadIdx.x == 0) counts[0] = last;
    if (threadIdx.x >= 1 && threadIdx.x <= kJpBatch) counts[threadIdx.x] = 0;
}

// ------------------------------------------------------------ bucketing
__global__ void bucket_key_kernel(DGraph g, const int32_t *__restrict__ color, BinLimits lim,
                                  uint32_t *keys, uint32_t *vals) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        const int deg = g.off[v + 1] - g.off[v];
        int bin;
        if (deg == 0) bin = kBinSkip;
        else if (deg <= lim.small_max) bin = 0;
        else if (deg <= lim.warp_max) bin = 1;
        else if (deg <= lim.cta_max) bin = 2;
        else bin = 3;
        const int cls = color ? color[v] : 0;
        keys[v] = (uint32_t)(cls * (kBins + 1) + bin);
        vals[v] = (uint32_t)v;
    }
}

__global__ void bucket_count_kernel(const uint32_t *__restrict__ keys, int n, int32_t *counts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // count run heads only: one atomic per bucket boundary
        const uint32_t k = keys[i];
        if (i == n - 1 || keys[i + 1] != k) atomicAdd(&counts[k], i + 1);
        if (i > 0 && keys[i - 1] != k) atomicAdd(&counts[k], -i);
    }
}

__device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// hub hash-table size at each position of the order (0 for non-hubs)
__global__ void hub_size_kernel(DGraph g, const int32_t *__restrict__ order, int cta_max,
                                int32_t *tsize) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += gridDim.x * blockDim.x) {
        const int v = order[p];
        const int deg = g.off[v + 1] - g.off[v];
        tsize[p] = deg > cta_max ? next_pow2(2 * deg) : 0;
    }
}

}  // namespace

lv_status jp_color(const DGraph &g, uint64_t seed, int32_t *color, int32_t *num_colors,
                   int *pinned, cudaStream_t s) {
    const int n = g.n;
    int32_t *cnt = nullptr, *lists = nullptr, *counts = nullptr, *maxc = nullptr;
    LV_TRY(dalloc_n(&cnt, (size_t)n, s));
    LV_TRY(dalloc_n(&lists, 2 * (size_t)n, s));
    LV_TRY(dalloc_n(&counts, kJpBatch + 1, s));
    LV_TRY(dalloc_n(&maxc, 1, s));
    LV_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (kJpBatch + 1), s));
    LV_CUDA(cudaMemsetAsync(maxc, 0, sizeof(int32_t), s));
    const int grid_init = grid_for(n, 8, g_num_sms * 16);
    jp_init_kernel<<<grid_init, 256, 0, s>>>(g, seed, cnt, color, lists, counts);
    LV_LAUNCH_CHECK();
    const int grid_round = g_num_sms * 8;
    int cur = 0;  // list holding counts[0]'s vertices
    int64_t rounds = 0;
    for (;;) {
        for (int r = 0; r < kJpBatch; ++r) {
            const int li = (cur + r) & 1;
            jp_round_kernel<<<grid_round, 256, 0, s>>>(g, seed, cnt, color, lists + (size_t)li * n,
                                                       counts + r, lists + (size_t)(li ^ 1) * n,
                                                       counts + r + 1, maxc);
            LV_LAUNCH_CHECK();
        }
        rounds += kJpBatch;
        cur = (cur + kJpBatch) & 1;
        LV_CUDA(cudaMemcpyAsync(pinned, counts + kJpBatch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        jp_carry_kernel<<<1, 32, 0, s>>>(counts);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaStreamSynchronize(s));
        if (pinned[0] == 0) break;
        if (rounds > (int64_t)n + kJpBatch) return LV_ERR_STATE;  // cannot happen: each round colours >= 1
    }
    LV_CUDA(cudaMemcpyAsync(pinned, maxc, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    *num_colors = pinned[0] + 1;
    dfree(cnt, s);
    dfree(lists, s);
    dfree(counts, s);
    dfree(maxc, s);
    return LV_OK;
}

lv_status bucket_vertices(const DGraph &g, const int32_t *color, int32_t classes,
                          const BinLimits &lim, Buckets *b, int *pinned, cudaStream_t s) {
    const int n = g.n;
    const int nb = classes * (kBins + 1);
    b->classes = classes;
    uint32_t *keys = nullptr, *keys_alt = nullptr, *vals_alt = nullptr;
    LV_TRY(dalloc_n(&keys, (size_t)n, s));
    LV_TRY(dalloc_n(&keys_alt, (size_t)n, s));
    LV_TRY(dalloc_n(&vals_alt, (size_t)n, s));
    LV_TRY(dalloc_n(&b->order, (size_t)n, s));
    LV_TRY(dalloc_n(&b->bucket_off, (size_t)nb + 1, s));
    const int grid = grid_for(n, 256, g_num_sms * 16);
    bucket_key_kernel<<<grid, 256, 0, s>>>(g, color, lim, keys, reinterpret_cast<uint32_t *>(b->order));
    LV_LAUNCH_CHECK();
    LV_TRY(radix_sort_u32(keys, reinterpret_cast<uint32_t *>(b->order), keys_alt, vals_alt, n,
                          bits_for((uint64_t)nb - 1), s));
    LV_CUDA(cudaMemsetAsync(b->bucket_off, 0, sizeof(int32_t) * ((size_t)nb + 1), s));
    bucket_count_kernel<<<grid, 256, 0, s>>>(keys, n, b->bucket_off);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(b->bucket_off, b->bucket_off, nb, s));
    b->host_off = new int32_t[(size_t)nb + 1];
    LV_CUDA(cudaMemcpyAsync(b->host_off, b->bucket_off, sizeof(int32_t) * ((size_t)nb + 1),
                            cudaMemcpyDeviceToHost, s));
    // hub tables
    LV_TRY(dalloc_n(&b->hub_off, (size_t)n + 1, s));
    hub_size_kernel<<<grid, 256, 0, s>>>(g, b->order, lim.cta_max, b->hub_off);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(b->hub_off, b->hub_off, n, s));
    LV_CUDA(cudaMemcpyAsync(pinned, b->hub_off + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    b->hub_slots = pinned[0];
    if (b->hub_slots > 0) LV_TRY(dalloc_n(&b->hub_table, (size_t)b->hub_slots, s));
    dfree(keys, s);
    dfree(keys_alt, s);
    dfree(vals_alt, s);
    return LV_OK;
}

void free_buckets(Buckets &b, cudaStream_t s) {
    dfree(b.order, s);
    dfree(b.bucket_off, s);
    dfree(b.hub_off, s);
    dfree(b.hub_table, s);
    delete[] b.host_off;
    b = Buckets();
}

}  // namespace lv
