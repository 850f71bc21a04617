// lv_color.cu -- distance-1 colouring (Sec. 4.2) and the per-phase vertex order.
//
// Colouring: Jones-Plassmann with a hash priority pi(v) = (h(v ^ seed), v).
// Every vertex counts its higher-priority neighbours; a vertex whose count
// reaches zero takes the smallest colour not used by those neighbours, then
// decrements the counts of its lower-priority neighbours.  The result equals
// greedy colouring in decreasing priority order, whatever the timing, because
// a vertex's colour depends only on its higher-priority neighbours' colours.
// On power-law graphs the priority DAG is deep (hundreds to thousands of
// rounds), so all rounds run inside one cooperative launch separated by a
// bounded grid barrier; a ready vertex of high degree is handled by a whole
// CTA, the others by one warp each.
//
// Vertex order: a stable radix sort of (colour, degree bin) keys, so each
// colour class is split into the group / warp / CTA / hub bins of the sweep,
// ascending vertex id inside each bucket.
#include "lv_ops.cuh"

namespace lv {
namespace {

constexpr int kJpBlock = 1024;       // threads per block of the persistent kernel
constexpr int kJpWarps = kJpBlock / 32;
constexpr int kJpBigDegree = 512;    // vertices with at least this many arcs use a whole CTA
constexpr int kMexWindow = 1024;     // colours examined per pass of the mex search

struct JpState {
    int32_t *cnt;          // higher-priority neighbours not yet coloured
    int32_t *color;
    int32_t *small_list[2];
    int32_t *big_list[2];
    int32_t *counts;       // ring of 3 x {small, big} list lengths
    int32_t *max_color;
    GridBarrier *bar;
    int *err;
};

__device__ __forceinline__ int degree_of(const DGraph &g, int u) { return g.off[u + 1] - g.off[u]; }

// append u to the next round's small or big list; warp-aggregated
__device__ __forceinline__ void push_ready(const DGraph &g, const JpState &st, int32_t *cnt_next,
                                           int nxt_list, bool ready, int u) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const bool big = ready && degree_of(g, u) >= kJpBigDegree;
    const unsigned bs = __ballot_sync(0xffffffffu, ready && !big);
    const unsigned bb = __ballot_sync(0xffffffffu, big);
    int ps = 0, pb = 0;
    if (lane == 0) {
        if (bs) ps = atomicAdd(&cnt_next[0], __popc(bs));
        if (bb) pb = atomicAdd(&cnt_next[1], __popc(bb));
    }
    ps = __shfl_sync(0xffffffffu, ps, 0);
    pb = __shfl_sync(0xffffffffu, pb, 0);
    if (ready && !big) st.small_list[nxt_list][ps + __popc(bs & lt)] = u;
    if (big) st.big_list[nxt_list][pb + __popc(bb & lt)] = u;
}

// mark the colours of v's higher-priority neighbours that fall in
// [base, base + kMexWindow); arcs e = first, first + step, ...
__device__ __forceinline__ void mark_window(const DGraph &g, unsigned long long seed, int v,
                                            unsigned long long hv, const int32_t *color, int beg,
                                            int end, int first, int step, int base, unsigned *bm) {
    for (int e = beg + first; e < end; e += step) {
        const int u = g.arcs[e].x;
        if (u != v && prio_greater(prio_hash((unsigned long long)u ^ seed), u, hv, v)) {
            const int c = __ldcg(&color[u]) - base;
            if (c >= 0 && c < kMexWindow) atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
    }
}

// one warp colours v and releases its lower-priority neighbours
__device__ void jp_small(const DGraph &g, unsigned long long seed, const JpState &st, int v,
                         int32_t *cnt_next, int nxt_list, unsigned *bm) {
    const int lane = threadIdx.x & 31;
    const unsigned long long hv = prio_hash((unsigned long long)v ^ seed);
    const int beg = g.off[v], end = g.off[v + 1];
    int mex = -1;
    for (int base = 0; mex < 0; base += kMexWindow) {
        bm[lane] = 0u;
        __syncwarp();
        mark_window(g, seed, v, hv, st.color, beg, end, lane, 32, base, bm);
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
        __stcg(&st.color[v], mex);
        atomicMax(st.max_color, mex);
    }
    for (int b0 = beg; b0 < end; b0 += 32) {
        const int e = b0 + lane;
        bool ready = false;
        int u = 0;
        if (e < end) {
            u = g.arcs[e].x;
            if (u != v && prio_greater(hv, v, prio_hash((unsigned long long)u ^ seed), u))
                ready = (atomicSub(&st.cnt[u], 1) == 1);
        }
        push_ready(g, st, cnt_next, nxt_list, ready, u);
    }
}

// one CTA colours a high-degree v
__device__ void jp_big(const DGraph &g, unsigned long long seed, const JpState &st, int v,
                       int32_t *cnt_next, int nxt_list, unsigned *bm, int *s_mex) {
    const unsigned long long hv = prio_hash((unsigned long long)v ^ seed);
    const int beg = g.off[v], end = g.off[v + 1];
    for (int base = 0;; base += kMexWindow) {
        if (threadIdx.x < 32) bm[threadIdx.x] = 0u;
        __syncthreads();
        mark_window(g, seed, v, hv, st.color, beg, end, threadIdx.x, kJpBlock, base, bm);
        __syncthreads();
        if (threadIdx.x < 32) {
            const unsigned word = bm[threadIdx.x];
            const unsigned notfull = __ballot_sync(0xffffffffu, word != 0xffffffffu);
            if (threadIdx.x == 0) {
                if (notfull) {
                    const int f = __ffs(notfull) - 1;
                    *s_mex = base + 32 * f + __ffs(~bm[f]) - 1;
                } else {
                    *s_mex = -1;
                }
            }
        }
        __syncthreads();
        if (*s_mex >= 0) break;
    }
    if (threadIdx.x == 0) {
        __stcg(&st.color[v], *s_mex);
        atomicMax(st.max_color, *s_mex);
    }
    for (int b0 = beg; b0 < end; b0 += kJpBlock) {
        const int e = b0 + (int)threadIdx.x;
        bool ready = false;
        int u = 0;
        if (e < end) {
            u = g.arcs[e].x;
            if (u != v && prio_greater(hv, v, prio_hash((unsigned long long)u ^ seed), u))
                ready = (atomicSub(&st.cnt[u], 1) == 1);
        }
        push_ready(g, st, cnt_next, nxt_list, ready, u);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) jp_init_kernel(DGraph g, unsigned long long seed, JpState st) {
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
            st.cnt[v] = c;
            st.color[v] = -1;
        }
        // round 0 lists (ring slot 0)
        push_ready(g, st, st.counts, 0, lane == 0 && c == 0, v);
    }
}

// All rounds of Jones-Plassmann in one cooperative launch; rounds are
// separated by a bounded grid barrier.
__global__ void __launch_bounds__(kJpBlock) jp_persistent_kernel(DGraph g, unsigned long long seed,
                                                                 JpState st) {
    __shared__ unsigned bm_warp[kJpWarps][32];
    __shared__ unsigned bm_cta[32];
    __shared__ int s_mex;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kJpWarps + wib;
    const int nwarps = gridDim.x * kJpWarps;
    for (int r = 0;; ++r) {
        const int cur = r % 3, nxt = (r + 1) % 3, clr = (r + 2) % 3;
        if (blockIdx.x == 0 && threadIdx.x < 2) st.counts[2 * clr + threadIdx.x] = 0;
        const int n_small = __ldcg(&st.counts[2 * cur]);
        const int n_big = __ldcg(&st.counts[2 * cur + 1]);
        const int in_list = r & 1, out_list = (r + 1) & 1;
        int32_t *cnt_next = st.counts + 2 * nxt;
        for (int t = blockIdx.x; t < n_big; t += gridDim.x)
            jp_big(g, seed, st, __ldcg(&st.big_list[in_list][t]), cnt_next, out_list, bm_cta, &s_mex);
        for (int t = gw; t < n_small; t += nwarps)
            jp_small(g, seed, st, __ldcg(&st.small_list[in_list][t]), cnt_next, out_list,
                     bm_warp[wib]);
        if (!grid_sync(st.bar, st.err)) return;
        if (__ldcg(&cnt_next[0]) + __ldcg(&cnt_next[1]) == 0) return;
        if (r > g.n) {  // every round colours at least one vertex
            if (threadIdx.x == 0) atomicExch(st.err, 2);
            return;
        }
    }
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

// hub hash-table size and arc-chunk count at each position of the order
// (0 for non-hubs)
__global__ void hub_size_kernel(DGraph g, const int32_t *__restrict__ order, int cta_max,
                                int32_t *tsize, int32_t *nchunks) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += gridDim.x * blockDim.x) {
        const int v = order[p];
        const int deg = g.off[v + 1] - g.off[v];
        const bool hub = deg > cta_max;
        tsize[p] = hub ? next_pow2(2 * deg) : 0;
        nchunks[p] = hub ? (deg + kHubChunk - 1) / kHubChunk : 0;
    }
}

__global__ void fill_empty_kernel(int2 *tab, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        tab[i] = make_int2(kEmpty, 0);
}

__global__ void gather_at_kernel(const int32_t *__restrict__ vals, const int32_t *__restrict__ idx,
                                 int m, int32_t *out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x)
        out[q] = vals[idx[q]];
}

}  // namespace

lv_status jp_color(const DGraph &g, uint64_t seed, int32_t *color, int32_t *num_colors,
                   int *pinned, cudaStream_t s) {
    const int n = g.n;
    JpState st;
    st.color = color;
    LV_TRY(dalloc_n(&st.cnt, (size_t)n, s));
    LV_TRY(dalloc_n(&st.small_list[0], (size_t)n, s));
    LV_TRY(dalloc_n(&st.small_list[1], (size_t)n, s));
    LV_TRY(dalloc_n(&st.big_list[0], (size_t)n, s));
    LV_TRY(dalloc_n(&st.big_list[1], (size_t)n, s));
    int32_t *small_state = nullptr;  // counts[6], max_color, err, barrier
    LV_TRY(dalloc_n(&small_state, 16, s));
    LV_CUDA(cudaMemsetAsync(small_state, 0, 16 * sizeof(int32_t), s));
    st.counts = small_state;
    st.max_color = small_state + 6;
    st.err = small_state + 7;
    st.bar = reinterpret_cast<GridBarrier *>(small_state + 8);
    jp_init_kernel<<<grid_for(n, 8, g_num_sms * 16), 256, 0, s>>>(g, seed, st);
    LV_LAUNCH_CHECK();
    static int blocks_per_sm = 0;
    if (!blocks_per_sm) {
        LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, jp_persistent_kernel,
                                                              kJpBlock, 0));
        if (blocks_per_sm < 1) return LV_ERR_CUDA;
    }
    unsigned long long seed_arg = seed;
    DGraph garg = g;
    void *args[] = {&garg, &seed_arg, &st};
    LV_CUDA(cudaLaunchCooperativeKernel((void *)jp_persistent_kernel, dim3(g_num_sms * blocks_per_sm),
                                        dim3(kJpBlock), args, 0, s));
    LV_LAUNCH_CHECK();
    LV_CUDA(cudaMemcpyAsync(pinned, small_state + 6, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    if (pinned[1] == 1) return LV_ERR_TIMEOUT;
    if (pinned[1] != 0) return LV_ERR_STATE;
    *num_colors = pinned[0] + 1;
    dfree(st.cnt, s);
    dfree(st.small_list[0], s);
    dfree(st.small_list[1], s);
    dfree(st.big_list[0], s);
    dfree(st.big_list[1], s);
    dfree(small_state, s);
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
    // hub tables: slots, occupied lists, arc chunks
    int32_t *chunk_at = nullptr;
    LV_TRY(dalloc_n(&b->hub_off, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&b->hub_chunk_off, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&chunk_at, (size_t)nb + 1, s));
    hub_size_kernel<<<grid, 256, 0, s>>>(g, b->order, lim.cta_max, b->hub_off, b->hub_chunk_off);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(b->hub_off, b->hub_off, n, s));
    LV_TRY(scan_excl_i32(b->hub_chunk_off, b->hub_chunk_off, n, s));
    gather_at_kernel<<<grid_for(nb + 1, 256, 1024), 256, 0, s>>>(b->hub_chunk_off, b->bucket_off,
                                                               nb + 1, chunk_at);
    LV_LAUNCH_CHECK();
    b->host_chunk = new int32_t[(size_t)nb + 1];
    LV_CUDA(cudaMemcpyAsync(b->host_chunk, chunk_at, sizeof(int32_t) * ((size_t)nb + 1),
                            cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(pinned, b->hub_off + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    dfree(chunk_at, s);
    b->hub_slots = pinned[0];
    if (b->hub_slots > 0) {
        LV_TRY(dalloc_n(&b->hub_table, (size_t)b->hub_slots, s));
        LV_TRY(dalloc_n(&b->hub_occ, (size_t)b->hub_slots, s));
        LV_TRY(dalloc_n(&b->hub_cnt, (size_t)n, s));
        LV_CUDA(cudaMemsetAsync(b->hub_cnt, 0, sizeof(int32_t) * (size_t)n, s));
        fill_empty_kernel<<<grid_for(b->hub_slots, 256, g_num_sms * 8), 256, 0, s>>>(b->hub_table,
                                                                                   b->hub_slots);
        LV_LAUNCH_CHECK();
    }
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
    dfree(b.hub_occ, s);
    dfree(b.hub_cnt, s);
    dfree(b.hub_chunk_off, s);
    delete[] b.host_off;
    delete[] b.host_chunk;
    b = Buckets();
}

}  // namespace lv
