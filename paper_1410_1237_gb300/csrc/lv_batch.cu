// lv_batch.cu -- batched runs: many independent graphs behind one handle.
//
// The graphs are held as one disjoint union (vertices numbered graph after
// graph, gid[v] = graph of v).  Vertex following, the sweep and the rebuild
// never cross a graph boundary, so they run on the union unchanged; what is
// per graph is the arithmetic of the gain (each graph's own 2m), the
// modularity terms (summed per graph inside the sweep) and the control of
// Algorithm 1 and Sec. 4.4 (iteration and phase stopping), which the host
// replays per graph exactly as the single-graph driver does:
//   - each batched sweep covers the vertices of graphs still iterating in
//     the current phase; the sweep that proposes iteration t's moves also
//     yields N(C^{t-1}) per graph (fused modularity), the host runs every
//     graph's stopping test and applies the moves only of graphs that go on;
//   - phases are taken in lock step: when no graph iterates any more, one
//     renumber / compose / coarsen pass serves all graphs.  A graph whose
//     phase loop has stopped rides along with the identity partition (its
//     coarse graph is rebuilt from its final communities and never swept),
//     so its labels do not change any more.
// Renumbering ranks communities by id, so graphs stay contiguous and ordered
// in every coarse union and local ids are union ids minus the graph's start.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lv_ops.cuh"

using namespace lv;

namespace {

// gid[v] = g with gptr[g] <= v < gptr[g+1] (gptr strictly increasing)
__global__ void graph_of_kernel(int32_t n, int32_t G, const int32_t *__restrict__ gptr,
                                int32_t *gid) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int a = 0, b = G;  // gptr[a] <= v < gptr[b]
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (gptr[mid] <= v) a = mid; else b = mid;
        }
        gid[v] = a;
    }
}

// every arc of row i must stay inside graph gid[i]; one warp per row
__global__ void __launch_bounds__(256) cross_check_kernel(DGraph g, const int32_t *__restrict__ gid,
                                                          const int32_t *__restrict__ gptr,
                                                          int *bad) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * 8;
    for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < g.n; i += nw) {
        const int gi = gid[i];
        const int lo = gptr[gi], hi = gptr[gi + 1];
        bool ok = true;
        for (int e = g.off[i] + lane; e < g.off[i + 1]; e += 32) {
            const int c = g.arcs[e].x;
            ok = ok && c >= lo && c < hi;
        }
        if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicExch(bad, 1);
    }
}

// Per-graph sums over vertices of graphs with active[g] != 0 (all graphs
// when active is null): sum_k (2m), sum_loop and sum_k2.  Any output may be
// null.  Vertices of a graph are consecutive, so whole warps form runs.
__global__ void __launch_bounds__(256) graph_sums_kernel(int32_t n, const int32_t *__restrict__ gid,
                                                         const int32_t *__restrict__ k,
                                                         const int32_t *__restrict__ loop,
                                                         const uint8_t *__restrict__ active,
                                                         unsigned long long *sum_k,
                                                         unsigned long long *sum_loop,
                                                         unsigned long long *sum_k2) {
    const int nr = (n + 31) & ~31;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nr; v += gridDim.x * blockDim.x) {
        const bool in = v < n;
        const int g = in ? gid[v] : 0;
        const bool on = in && (!active || active[g]);
        const long long kv = on ? k[v] : 0;
        const long long lv = on ? loop[v] : 0;
        if (sum_k) warp_run_add(g, (unsigned long long)kv, on, sum_k);
        if (sum_loop) warp_run_add(g, (unsigned long long)lv, on, sum_loop);
        if (sum_k2) warp_run_add(g, (unsigned long long)(kv * kv), on, sum_k2);
    }
}

// gid_new[to[v]] = gid[v], to[v] = idx[C[v]] (or idx[v] when C is null);
// all writers of one target write the same graph
__global__ void gid_scatter_kernel(int32_t n, const int32_t *__restrict__ gid,
                                   const int32_t *__restrict__ C, const int32_t *__restrict__ idx,
                                   int32_t *gid_new) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        gid_new[idx[C ? C[v] : v]] = gid[v];
}

// gptr from a non-decreasing gid: gptr[g] = first vertex of g, gptr[G] = n
__global__ void gptr_kernel(int32_t n, int32_t G, const int32_t *__restrict__ gid, int32_t *gptr) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (v == 0 || gid[v] != gid[v - 1]) gptr[gid[v]] = v;
        if (v == 0) gptr[G] = n;
    }
}

// out[g] = arr[gptr[g]] for g <= G (arc offsets, or new ids, at graph starts)
__global__ void gather_at_kernel(int32_t G, const int32_t *__restrict__ gptr,
                                 const int32_t *__restrict__ arr, int32_t *out) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
        out[g] = arr[gptr[g]];
}

// apply the listed moves of graphs whose apply flag is set
__global__ void apply_batch_kernel(int32_t *C, unsigned long long *comm,
                                   const int4 *__restrict__ moves, const int32_t *__restrict__ count,
                                   const int32_t *__restrict__ gid,
                                   const uint8_t *__restrict__ apply) {
    const int cnt = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int4 m = moves[t];
        if (!apply[gid[m.x]]) continue;
        C[m.x] = m.z;
        atomicAdd(&comm[m.y], comm_leave(m.w));
        atomicAdd(&comm[m.z], comm_join(m.w));
    }
}

// union labels -> labels local to each graph
__global__ void localize_kernel(int32_t n, const int32_t *__restrict__ gid,
                                const int32_t *__restrict__ gstart, int32_t *labels) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        labels[v] -= gstart[gid[v]];
}

// Compaction of the group bins (degree bins 0..5, positions [lo, hi) of
// the bucketed order): vertices of graphs that stopped iterating are dropped,
// so later sweeps of a phase hand out items over live vertices only.  The
// kept vertices are packed at the END of [lo, hi) (CTA-bin and hub positions
// after hi keep their places and their per-position hub arrays).
__global__ void keep_flags_kernel(const int32_t *__restrict__ order, int lo, int hi,
                                  const int32_t *__restrict__ gid,
                                  const uint8_t *__restrict__ active, int32_t *flag) {
    for (int p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x)
        flag[p - lo] = active[gid[order[p]]] ? 1 : 0;
}

__global__ void compact_kernel(const int32_t *__restrict__ order, int lo, int hi,
                               const int32_t *__restrict__ pos, int32_t *out) {
    const int base = hi - pos[hi - lo];
    for (int p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x)
        if (pos[p - lo + 1] != pos[p - lo]) out[base + pos[p - lo]] = order[p];
}

// bucket offsets of the compacted list (class 0): group-bin starts move,
// the rest is copied
__global__ void compact_offsets_kernel(const int32_t *__restrict__ bo, const int32_t *__restrict__ pos,
                                       int32_t *bo_c) {
    const int t = threadIdx.x;
    const int lo = bo[0], hi = bo[kBinCta];
    if (t <= kBins) bo_c[t] = t <= kBinCta ? hi - pos[hi - lo] + pos[bo[t] - lo] : bo[t];
}

int grid_n(int64_t items) { return grid_for(items, 256, g_num_sms * 16); }

}  // namespace

struct lv_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t G = 0;
    int64_t n = 0, A = 0;
    DGraph in;
    int32_t *k_in = nullptr, *loop_in = nullptr;
    int32_t *gid_in = nullptr;       // device, n
    int32_t *gptr_in = nullptr;      // device, G+1
    long long *two_m_dev = nullptr;  // device, G
    std::vector<int32_t> gptr;       // host, G+1
    std::vector<int64_t> arcs;       // host, per graph
    std::vector<long long> two_m;    // host, per graph
    // pinned host scratch: 3G u64 per-graph sums, 2(G+1) int32, IterStats
    unsigned long long *pin_u64 = nullptr;
    int32_t *pin_i32 = nullptr;
    IterStats *pin_stats = nullptr;
    uint8_t *pin_flags = nullptr;    // G
    int *pinned = nullptr;           // 64 ints for the shared helpers
    void *pin_block = nullptr;
    // results of the last run
    bool have_run = false;
    std::vector<int32_t *> labels;   // per batch phase: device int32[n], local ids
    std::vector<std::vector<lv_phase_info>> info;  // per graph, per phase
    std::vector<lv_batch_sweep> sweeps;
    // bins chosen by measurement per phase index (autotune), kept across runs
    std::vector<BinLimits> tuned;
    std::vector<char> tuned_ok;
    lv_stats stats;
    Timer timer;

    void clear_results() {
        for (auto p : labels) dfree(p, stream);
        labels.clear();
        info.clear();
        sweeps.clear();
        std::memset(&stats, 0, sizeof stats);
        timer.clear();
        have_run = false;
    }
};

namespace {

lv_status alloc_pinned(lv_batch *b) {
    const size_t G = (size_t)b->G;
    const size_t bytes = 8 * (3 * G) + 4 * (2 * (G + 1)) + sizeof(IterStats) + G + 64 * 4 + 256;
    if (cudaMallocHost(&b->pin_block, bytes) != cudaSuccess) return LV_ERR_OOM;
    char *p = static_cast<char *>(b->pin_block);
    b->pin_u64 = reinterpret_cast<unsigned long long *>(p);
    p += 8 * 3 * G;
    b->pin_stats = reinterpret_cast<IterStats *>(p);
    p += (sizeof(IterStats) + 15) & ~size_t(15);
    b->pinned = reinterpret_cast<int *>(p);
    p += 64 * 4;
    b->pin_i32 = reinterpret_cast<int32_t *>(p);
    p += 4 * 2 * (G + 1);
    b->pin_flags = reinterpret_cast<uint8_t *>(p);
    return LV_OK;
}

// Checks the union against the batch contract and fills gid, gptr, 2m and
// per-graph arc counts.
lv_status batch_setup(lv_batch *b) {
    cudaStream_t s = b->stream;
    const int32_t G = b->G;
    LV_TRY(dalloc_n(&b->gid_in, (size_t)b->n, s));
    LV_TRY(dalloc_n(&b->gptr_in, (size_t)G + 1, s));
    LV_TRY(dalloc_n(&b->two_m_dev, (size_t)G, s));
    LV_CUDA(cudaMemcpyAsync(b->gptr_in, b->gptr.data(), sizeof(int32_t) * ((size_t)G + 1),
                            cudaMemcpyHostToDevice, s));
    graph_of_kernel<<<grid_n(b->n), 256, 0, s>>>((int32_t)b->n, G, b->gptr_in, b->gid_in);
    LV_LAUNCH_CHECK();
    int *bad = nullptr;
    unsigned long long *sk = nullptr;
    int32_t *starts = nullptr;
    LV_TRY(dalloc_n(&bad, 1, s));
    LV_TRY(dalloc_n(&sk, (size_t)G, s));
    LV_TRY(dalloc_n(&starts, (size_t)G + 1, s));
    LV_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    LV_CUDA(cudaMemsetAsync(sk, 0, sizeof(unsigned long long) * G, s));
    cross_check_kernel<<<grid_for(b->n, 8, g_num_sms * 16), 256, 0, s>>>(b->in, b->gid_in,
                                                                          b->gptr_in, bad);
    LV_LAUNCH_CHECK();
    graph_sums_kernel<<<grid_n(b->n), 256, 0, s>>>((int32_t)b->n, b->gid_in, b->k_in, b->loop_in,
                                                   nullptr, sk, nullptr, nullptr);
    LV_LAUNCH_CHECK();
    gather_at_kernel<<<grid_n(G + 1), 256, 0, s>>>(G, b->gptr_in, b->in.off, starts);
    LV_LAUNCH_CHECK();
    LV_CUDA(cudaMemcpyAsync(b->pinned, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(b->pin_u64, sk, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(b->pin_i32, starts, sizeof(int32_t) * ((size_t)G + 1),
                            cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    dfree(bad, s);
    dfree(sk, s);
    dfree(starts, s);
    if (b->pinned[0]) return LV_ERR_ARG;
    b->two_m.assign(G, 0);
    b->arcs.assign(G, 0);
    lv_status st = LV_OK;
    for (int32_t g = 0; g < G; ++g) {
        const unsigned long long tm = b->pin_u64[g];
        if (tm >= (1ull << 31) && st == LV_OK) st = LV_ERR_OVERFLOW;
        b->two_m[g] = (long long)tm;
        b->arcs[g] = (int64_t)b->pin_i32[g + 1] - b->pin_i32[g];
    }
    if (st != LV_OK) return st;
    for (int32_t g = 0; g < G; ++g)
        if (b->two_m[g] == 0) return LV_ERR_EMPTY;
    LV_CUDA(cudaMemcpyAsync(b->two_m_dev, b->two_m.data(), sizeof(long long) * G,
                            cudaMemcpyHostToDevice, s));
    LV_CUDA(cudaStreamSynchronize(s));
    return LV_OK;
}

}  // namespace

extern "C" {

lv_status lv_batch_create(lv_batch **out, int32_t n_graphs, const int64_t *gptr,
                          const int64_t *rowptr, const int32_t *col, const int32_t *w,
                          int ptrs_on_device, void *cuda_stream) {
    if (!out) return LV_ERR_ARG;
    *out = nullptr;
    if (n_graphs < 1 || !gptr || !rowptr) return LV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    LV_TRY(ensure_setup(s));
    std::vector<int64_t> gp((size_t)n_graphs + 1);
    if (ptrs_on_device) {
        LV_CUDA(cudaMemcpyAsync(gp.data(), gptr, sizeof(int64_t) * gp.size(), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
    } else {
        std::memcpy(gp.data(), gptr, sizeof(int64_t) * gp.size());
    }
    if (gp[0] != 0) return LV_ERR_ARG;
    for (int32_t g = 0; g < n_graphs; ++g)
        if (gp[g + 1] <= gp[g]) return LV_ERR_ARG;
    const int64_t n = gp[n_graphs];
    if (n > 0x7ffffffell) return LV_ERR_ARG;

    const int64_t *d_rowptr = rowptr;
    const int32_t *d_col = col, *d_w = w;
    int64_t *st_rowptr = nullptr;
    int32_t *st_col = nullptr, *st_w = nullptr;
    if (!ptrs_on_device) {
        const int64_t A = rowptr[n];
        LV_TRY(dalloc_n(&st_rowptr, (size_t)n + 1, s));
        LV_CUDA(cudaMemcpyAsync(st_rowptr, rowptr, sizeof(int64_t) * ((size_t)n + 1),
                                cudaMemcpyHostToDevice, s));
        d_rowptr = st_rowptr;
        if (A > 0 && A <= 0x7fffffffll) {
            if (!col || !w) return LV_ERR_ARG;
            LV_TRY(dalloc_n(&st_col, (size_t)A, s));
            LV_TRY(dalloc_n(&st_w, (size_t)A, s));
            LV_CUDA(cudaMemcpyAsync(st_col, col, sizeof(int32_t) * (size_t)A, cudaMemcpyHostToDevice, s));
            LV_CUDA(cudaMemcpyAsync(st_w, w, sizeof(int32_t) * (size_t)A, cudaMemcpyHostToDevice, s));
        }
        d_col = st_col;
        d_w = st_w;
    }
    lv_batch *b = new lv_batch();
    b->stream = s;
    b->timer.s = s;
    cudaGetDevice(&b->device);
    b->G = n_graphs;
    b->n = n;
    b->gptr.resize(gp.size());
    for (size_t g = 0; g < gp.size(); ++g) b->gptr[g] = (int32_t)gp[g];
    lv_status st = alloc_pinned(b);
    int64_t total_2m = 0;
    if (st == LV_OK)
        st = validate_and_build(n, d_rowptr, d_col, d_w, &b->in, &b->k_in, &b->loop_in, &total_2m,
                                b->pinned, s, /*limit_two_m=*/false);
    dfree(st_rowptr, s);
    dfree(st_col, s);
    dfree(st_w, s);
    if (st == LV_OK) {
        b->A = b->in.A;
        st = batch_setup(b);
    }
    if (st != LV_OK) {
        cudaStreamSynchronize(s);
        lv_batch_destroy(b);
        return st;
    }
    *out = b;
    return LV_OK;
}

void lv_batch_destroy(lv_batch *b) {
    if (!b) return;
    b->clear_results();
    free_graph(b->in, b->stream);
    dfree(b->k_in, b->stream);
    dfree(b->loop_in, b->stream);
    dfree(b->gid_in, b->stream);
    dfree(b->gptr_in, b->stream);
    dfree(b->two_m_dev, b->stream);
    cudaStreamSynchronize(b->stream);
    if (b->pin_block) cudaFreeHost(b->pin_block);
    delete b;
}

lv_status lv_batch_num_graphs(const lv_batch *b, int32_t *out) {
    if (!b || !out) return LV_ERR_ARG;
    *out = b->G;
    return LV_OK;
}

}  // extern "C"

namespace {

// control state of one graph (the single-graph driver's locals, per graph)
struct GState {
    bool done = false;     // its phase loop has stopped
    bool running = false;  // still iterating in the current phase
    int step = 0;          // sweeps of the current phase
    bool have_np = false;
    int64_t n_p = 0;
    int64_t N_start = 0, N_end = 0;
    int32_t iters = 0;
};

// The fixed part of a batched iteration (clearing the counters and the
// persistent sweep launch) as an instantiated CUDA graph: captured at the
// first sweep of a phase and again when the vertex list moves to the
// compacted buffer, replayed by every other iteration.  If the capture is
// refused the iterations are issued directly.
struct SweepGraph {
    cudaGraphExec_t exec = nullptr;
    const int32_t *order = nullptr, *bo = nullptr;
    bool disabled = false;
    int captures = 0;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        order = bo = nullptr;
    }
    ~SweepGraph() { reset(); }
};

// device buffers of one run, released on every exit path
struct RunBufs {
    cudaStream_t s = nullptr;
    DGraph g;                  // current phase graph when owned
    bool own_g = false;
    int32_t *k = nullptr, *loop = nullptr, *gid = nullptr;  // owned per-phase arrays
    int32_t *map = nullptr;    // original vertex -> vertex of the phase graph
    int32_t *gbuf[2] = {nullptr, nullptr};  // graph starts: current / next
    int32_t *tmp = nullptr;    // G+1 scratch
    int32_t *newid = nullptr;
    unsigned long long *gsum = nullptr;  // 3G per-graph sums
    uint8_t *flags = nullptr;  // G: graph iterates (sweep) / applies its moves
    PhaseState ps;
    Buckets b;
    bool have_b = false;
    int32_t *order_c = nullptr, *bo_c = nullptr, *pos = nullptr;  // compacted vertex list
    SweepGraph sg;
    ~RunBufs() {
        sg.reset();
        dfree(order_c, s);
        dfree(bo_c, s);
        dfree(pos, s);
        if (own_g) free_graph(g, s);
        dfree(k, s);
        dfree(loop, s);
        dfree(gid, s);
        dfree(map, s);
        dfree(gbuf[0], s);
        dfree(gbuf[1], s);
        dfree(tmp, s);
        dfree(newid, s);
        dfree(gsum, s);
        dfree(flags, s);
        dfree(ps.C, s);
        dfree(ps.comm[0], s);
        dfree(ps.moves[0], s);
        dfree(ps.stats, s);
        dfree(ps.move_count, s);
        dfree(ps.act, s);
        if (have_b) free_buckets(b, s);
    }
};

lv_status batch_run_impl(lv_batch *h, const lv_params &P) {
    cudaStream_t s = h->stream;
    BinLimits lim;
    if (P.bin_lane_arcs) lim.lane_arcs = P.bin_lane_arcs;
    if (P.bin_warp_max) lim.warp_max = P.bin_warp_max;
    if (P.bin_cta_max) lim.cta_max = P.bin_cta_max;
    if (lim.lane_arcs < 1 || lim.lane_arcs > kLaneArcsLimit || lim.warp_max < 1 ||
        lim.warp_max > kWarpMaxLimit || lim.cta_max <= lim.warp_max || lim.cta_max > kCtaMaxLimit)
        return LV_ERR_ARG;
    if (P.max_iters < 1 || P.max_phases < 1 || !(P.theta_low >= -1e300) ||
        !(P.theta_high >= 0.0))
        return LV_ERR_ARG;
    const int32_t G = h->G;
    const int32_t n_orig = (int32_t)h->n;
    const double theta = P.theta_low;  // batched phases are uncoloured
    h->timer.on = P.collect_timing != 0;
    const unsigned long long launches0 = g_kernel_launches;
    const int ev_run0 = h->timer.mark();
    h->info.assign(G, std::vector<lv_phase_info>());

    RunBufs r;
    r.s = s;
    LV_TRY(dalloc_n(&r.map, (size_t)n_orig, s));
    LV_TRY(dalloc_n(&r.gbuf[0], (size_t)G + 1, s));
    LV_TRY(dalloc_n(&r.gbuf[1], (size_t)G + 1, s));
    LV_TRY(dalloc_n(&r.tmp, (size_t)G + 1, s));
    LV_TRY(dalloc_n(&r.gsum, 3 * (size_t)G, s));
    LV_TRY(dalloc_n(&r.flags, (size_t)G, s));
    int cur = 0;  // r.gbuf[cur] holds the graph starts of the phase graph

    // ---- vertex following on the union (Sec. 4.3; never crosses graphs)
    DGraph Gp = h->in;
    const int32_t *k = h->k_in, *loop = h->loop_in, *gid = h->gid_in;
    const int ev_vf0 = h->timer.mark();
    if (P.vertex_following) {
        DGraph G2;
        LV_TRY(vertex_following(Gp, h->loop_in, &G2, r.map, h->pinned, s));
        r.g = G2;
        r.own_g = true;
        Gp = G2;
        LV_TRY(dalloc_n(&r.k, (size_t)Gp.n, s));
        LV_TRY(dalloc_n(&r.loop, (size_t)Gp.n, s));
        LV_TRY(compute_degrees(Gp, r.k, r.loop, s));
        LV_TRY(dalloc_n(&r.gid, (size_t)Gp.n, s));
        gid_scatter_kernel<<<grid_n(n_orig), 256, 0, s>>>(n_orig, h->gid_in, nullptr, r.map, r.gid);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemsetAsync(r.gbuf[0], 0xff, sizeof(int32_t) * ((size_t)G + 1), s));
        gptr_kernel<<<grid_n(Gp.n), 256, 0, s>>>(Gp.n, G, r.gid, r.gbuf[0]);
        LV_LAUNCH_CHECK();
        k = r.k;
        loop = r.loop;
        gid = r.gid;
    } else {
        LV_TRY(iota(n_orig, r.map, s));
        LV_CUDA(cudaMemcpyAsync(r.gbuf[0], h->gptr_in, sizeof(int32_t) * ((size_t)G + 1),
                                cudaMemcpyDeviceToDevice, s));
    }
    const int ev_vf1 = h->timer.mark();
    h->stats.vf_n = Gp.n;
    std::vector<int32_t> gp((size_t)G + 1);
    LV_CUDA(cudaMemcpyAsync(h->pin_i32, r.gbuf[0], sizeof(int32_t) * ((size_t)G + 1),
                            cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    std::memcpy(gp.data(), h->pin_i32, sizeof(int32_t) * gp.size());
    for (int32_t g = 0; g < G; ++g) {
        if (gp[g] < 0 || gp[g + 1] <= gp[g]) return LV_ERR_CUDA;  // cannot happen: m_g > 0
        if (P.coloring && (int64_t)(gp[g + 1] - gp[g]) >= P.color_cutoff) return LV_ERR_ARG;
    }

    // per-vertex state, sized for the phase-0 union
    const int nmax = Gp.n;
    PhaseState &ps = r.ps;
    LV_TRY(dalloc_n(&ps.C, (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.comm[0], (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.moves[0], (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.stats, 1, s));
    LV_TRY(dalloc_n(&r.newid, (size_t)nmax + 1, s));
    LV_TRY(dalloc_n(&r.order_c, (size_t)nmax, s));
    LV_TRY(dalloc_n(&r.bo_c, (size_t)kBins + 2, s));
    LV_TRY(dalloc_n(&r.pos, (size_t)nmax + 1, s));
    LV_TRY(dalloc_n(&ps.act, 1, s));
    LV_TRY(dalloc_n(&ps.move_count, 4, s));
    LV_CUDA(cudaMemsetAsync(ps.act, 0, sizeof(int32_t), s));
    ps.bar = &ps.stats->bar;
    ps.bar_err = &ps.stats->bar_err;
    ps.coloured = false;
    ps.n_act = 1;
    ps.two_m = 0;
    ps.two_m_g = h->two_m_dev;
    ps.active_g = r.flags;
    ps.g_ein = r.gsum;
    ps.g_a2 = r.gsum + G;
    ps.g_moved = r.gsum + 2 * (size_t)G;

    std::vector<GState> gs((size_t)G);
    std::vector<int64_t> garcs((size_t)G);
    double ms_iter = 0.0, ms_rebuild = 0.0;
    const size_t gsum_bytes = sizeof(unsigned long long) * 3 * (size_t)G;
    std::vector<int> ev_iter, ev_reb;  // event index pairs per phase
    std::vector<int> ev_sweep;         // event index pairs per sweep

    for (int32_t p = 0; p < P.max_phases; ++p) {
        const int32_t *gptr = r.gbuf[cur];
        int32_t *gstart = r.gbuf[cur ^ 1];
        // per-graph arc counts of the phase graph
        gather_at_kernel<<<grid_n(G + 1), 256, 0, s>>>(G, gptr, Gp.off, r.tmp);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(h->pin_i32, r.tmp, sizeof(int32_t) * ((size_t)G + 1),
                                cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        for (int32_t g = 0; g < G; ++g) garcs[g] = (int64_t)h->pin_i32[g + 1] - h->pin_i32[g];

        // ---- initial state and N_start of every graph in the phase
        ps.g = Gp;
        ps.k = k;
        ps.loop = loop;
        ps.gid = gid;
        const int ev_i0 = h->timer.mark();
        LV_TRY(init_phase(ps, s));
        int n_running = 0;
        for (int32_t g = 0; g < G; ++g) {
            GState &t = gs[g];
            t.running = !t.done;
            t.step = 0;
            t.have_np = false;
            t.n_p = 0;
            t.iters = 0;
            h->pin_flags[g] = t.running ? 1 : 0;
            n_running += t.running ? 1 : 0;
        }
        LV_CUDA(cudaMemcpyAsync(r.flags, h->pin_flags, (size_t)G, cudaMemcpyHostToDevice, s));
        LV_CUDA(cudaMemsetAsync(r.gsum, 0, gsum_bytes, s));
        graph_sums_kernel<<<grid_n(Gp.n), 256, 0, s>>>(Gp.n, gid, k, loop, r.flags, nullptr,
                                                       r.gsum, r.gsum + G);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(h->pin_u64, r.gsum, sizeof(unsigned long long) * 2 * (size_t)G,
                                cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        for (int32_t g = 0; g < G; ++g)
            if (gs[g].running)
                gs[g].N_start = h->two_m[g] * (int64_t)h->pin_u64[g] - (int64_t)h->pin_u64[G + g];

        // ---- degree bins (measured once per phase index when autotuning)
        BinLimits plim = lim;
        if (P.autotune && Gp.A >= kTuneMinArcs) {
            if ((int32_t)h->tuned.size() <= p || !h->tuned_ok[p]) {
                BinLimits best = lim;
                LV_TRY(tune_bins(ps, lim, r.gsum, gsum_bytes, &best, h->pinned, s));
                if ((int32_t)h->tuned.size() <= p) {
                    h->tuned.resize(p + 1);
                    h->tuned_ok.resize(p + 1, 0);
                }
                h->tuned[p] = best;
                h->tuned_ok[p] = 1;
            }
            plim = h->tuned[p];
        }
        r.have_b = true;
        LV_TRY(bucket_vertices(Gp, nullptr, 1, plim, &r.b, h->pinned, s));

        // ---- batched iterations (Alg. 1 per graph, fused modularity)
        r.sg.reset();  // new phase graph: recapture
        int32_t sweep_no = 0;
        Buckets bl = r.b;  // the vertex list the sweeps walk (compacted as graphs stop)
        const int glo = r.b.host_off[0], ghi = r.b.host_off[kBinCta];
        int64_t listed = 0;  // vertices of the graphs in the list
        for (int32_t g = 0; g < G; ++g)
            if (gs[g].running) listed += gp[g + 1] - gp[g];
        while (n_running > 0) {
            lv_batch_sweep rec;
            std::memset(&rec, 0, sizeof rec);
            rec.phase = p;
            rec.sweep = ++sweep_no;
            rec.graphs = n_running;
            for (int32_t g = 0; g < G; ++g)
                if (gs[g].running) {
                    rec.vertices += gp[g + 1] - gp[g];
                    rec.arcs += garcs[g];
                }
            auto enqueue = [&]() -> lv_status {
                LV_CUDA(cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s));
                LV_CUDA(cudaMemsetAsync(ps.move_count, 0, 3 * sizeof(int32_t), s));
                LV_CUDA(cudaMemsetAsync(r.gsum, 0, gsum_bytes, s));
                return sweep_iteration(ps, bl, s);
            };
            SweepGraph &sg = r.sg;
            if (P.graph_capture && !sg.disabled &&
                (!sg.exec || sg.order != bl.order || sg.bo != bl.bucket_off)) {
                sg.reset();
                const unsigned long long l0 = g_kernel_launches;
                cudaGraph_t graph = nullptr;
                bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    const lv_status est = enqueue();
                    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
                    ok = est == LV_OK && ce == cudaSuccess && graph &&
                         cudaGraphInstantiate(&sg.exec, graph, 0) == cudaSuccess;
                    if (graph) cudaGraphDestroy(graph);
                }
                g_kernel_launches = l0;
                if (ok) {
                    sg.order = bl.order;
                    sg.bo = bl.bucket_off;
                    ++sg.captures;
                } else {
                    cudaGetLastError();
                    sg.reset();
                    sg.disabled = true;
                }
            }
            ev_sweep.push_back(h->timer.mark());
            if (sg.exec) {
                LV_CUDA(cudaGraphLaunch(sg.exec, s));
                ++g_kernel_launches;
                ++h->stats.graph_launches;
            } else {
                LV_TRY(enqueue());
            }
            ev_sweep.push_back(h->timer.mark());
            ++h->stats.sweep_launches;
            LV_CUDA(cudaMemcpyAsync(h->pin_stats, ps.stats, sizeof(IterStats), cudaMemcpyDeviceToHost, s));
            LV_CUDA(cudaMemcpyAsync(h->pin_u64, r.gsum, gsum_bytes, cudaMemcpyDeviceToHost, s));
            LV_CUDA(cudaStreamSynchronize(s));
            if (h->pin_stats->bar_err) return LV_ERR_TIMEOUT;
            if (h->pin_stats->err) return LV_ERR_HASH;
            for (int32_t g = 0; g < G; ++g) {
                GState &t = gs[g];
                if (!t.running) continue;
                const int step = ++t.step;
                // N(C^{step-1}) of this graph, read by the sweep under the labels it used
                const int64_t N_prev =
                    h->two_m[g] * (int64_t)h->pin_u64[g] - (int64_t)h->pin_u64[G + g];
                const int64_t moved = (int64_t)h->pin_u64[2 * (size_t)G + g];
                rec.moved += moved;
                bool fin = false;
                if (step == 1) {
                    if (moved == 0) {
                        t.iters = 1;
                        fin = true;
                    }
                } else {
                    const int tt = step - 1;
                    if ((t.have_np && gain_below(N_prev, t.n_p, theta)) || tt >= P.max_iters) {
                        t.iters = tt;
                        fin = true;
                    } else {
                        t.n_p = N_prev;
                        t.have_np = true;
                        if (moved == 0) {
                            t.iters = step;
                            fin = true;
                        }
                    }
                }
                if (fin) {
                    t.N_end = N_prev;
                    t.running = false;
                    h->pin_flags[g] = 0;
                    --n_running;
                }
            }
            h->sweeps.push_back(rec);
            if (n_running > 0) {
                // graphs that go on apply their moves and are swept again
                LV_CUDA(cudaMemcpyAsync(r.flags, h->pin_flags, (size_t)G, cudaMemcpyHostToDevice, s));
                apply_batch_kernel<<<g_num_sms * 4, 256, 0, s>>>(ps.C, ps.comm[0], ps.moves[0],
                                                                  ps.move_count, gid, r.flags);
                LV_LAUNCH_CHECK();
                int64_t live_v = 0;
                for (int32_t g = 0; g < G; ++g)
                    if (gs[g].running) live_v += gp[g + 1] - gp[g];
                if (ghi > glo && live_v * 4 < listed * 3) {
                    // drop stopped graphs from the group bins (from the full list)
                    keep_flags_kernel<<<grid_n(ghi - glo), 256, 0, s>>>(r.b.order, glo, ghi, gid,
                                                                         r.flags, r.pos);
                    LV_LAUNCH_CHECK();
                    LV_TRY(scan_excl_i32(r.pos, r.pos, ghi - glo, s));
                    compact_kernel<<<grid_n(ghi - glo), 256, 0, s>>>(r.b.order, glo, ghi, r.pos,
                                                                     r.order_c);
                    LV_LAUNCH_CHECK();
                    if (bl.order != r.order_c) {  // first compaction: CTA, hub and skip bins
                        const int tail = r.b.host_off[kBins + 1] - ghi;
                        if (tail > 0)
                            LV_CUDA(cudaMemcpyAsync(r.order_c + ghi, r.b.order + ghi,
                                                    sizeof(int32_t) * (size_t)tail,
                                                    cudaMemcpyDeviceToDevice, s));
                        LV_CUDA(cudaMemcpyAsync(r.bo_c + kBins + 1, r.b.bucket_off + kBins + 1,
                                                sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                    }
                    compact_offsets_kernel<<<1, 32, 0, s>>>(r.b.bucket_off, r.pos, r.bo_c);
                    LV_LAUNCH_CHECK();
                    bl.order = r.order_c;
                    bl.bucket_off = r.bo_c;
                    listed = live_v;
                }
            }
        }
        const int ev_i1 = h->timer.mark();

        // ---- rebuild (Sec. 4.5) of all graphs at once
        const int ev_r0 = h->timer.mark();
        LV_TRY(renumber(Gp.n, ps.comm[0], r.newid, s));
        gather_at_kernel<<<grid_n(G + 1), 256, 0, s>>>(G, gptr, r.newid, gstart);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(h->pin_i32, gstart, sizeof(int32_t) * ((size_t)G + 1),
                                cudaMemcpyDeviceToHost, s));
        int32_t *lab = nullptr;
        LV_TRY(dalloc_n(&lab, (size_t)n_orig, s));
        h->labels.push_back(lab);
        LV_TRY(compose_labels(n_orig, r.map, ps.C, r.newid, lab, s));
        localize_kernel<<<grid_n(n_orig), 256, 0, s>>>(n_orig, h->gid_in, gstart, lab);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaStreamSynchronize(s));
        const int32_t n_next = h->pin_i32[G];
        bool all_done = true;
        for (int32_t g = 0; g < G; ++g) {
            GState &t = gs[g];
            if (t.done) continue;
            lv_phase_info in;
            std::memset(&in, 0, sizeof in);
            in.n = gp[g + 1] - gp[g];
            in.arcs = garcs[g];
            in.n_next = (int64_t)h->pin_i32[g + 1] - h->pin_i32[g];
            in.two_m = h->two_m[g];
            in.N_start = t.N_start;
            in.N_end = t.N_end;
            in.q = (double)t.N_end / ((double)h->two_m[g] * (double)h->two_m[g]);
            in.theta = theta;
            in.iterations = t.iters;
            in.ms_color = in.ms_iterate = in.ms_rebuild = -1.0;
            h->info[g].push_back(in);
            if (in.n_next == in.n || gain_below(t.N_end, t.N_start, P.theta_low) ||
                p + 1 >= P.max_phases)
                t.done = true;
            all_done = all_done && t.done;
        }
        for (int32_t g = 0; g <= G; ++g) gp[g] = h->pin_i32[g];  // starts in the coarse union
        if (!all_done) {
            DGraph G2;
            LV_TRY(coarsen(Gp, ps.C, r.newid, n_next, &G2, h->pinned, s));
            int32_t *k2 = nullptr, *l2 = nullptr, *gid2 = nullptr;
            LV_TRY(dalloc_n(&k2, (size_t)G2.n, s));
            LV_TRY(dalloc_n(&l2, (size_t)G2.n, s));
            LV_TRY(dalloc_n(&gid2, (size_t)G2.n, s));
            gid_scatter_kernel<<<grid_n(Gp.n), 256, 0, s>>>(Gp.n, gid, ps.C, r.newid, gid2);
            LV_LAUNCH_CHECK();
            LV_TRY(compute_degrees(G2, k2, l2, s));
            if (r.own_g) free_graph(r.g, s);
            dfree(r.k, s);
            dfree(r.loop, s);
            dfree(r.gid, s);
            r.g = G2;
            r.own_g = true;
            Gp = G2;
            k = r.k = k2;
            loop = r.loop = l2;
            gid = r.gid = gid2;
            cur ^= 1;
        }
        const int ev_r1 = h->timer.mark();
        free_buckets(r.b, s);
        r.b = Buckets();
        r.have_b = false;
        ev_iter.push_back(ev_i0);
        ev_iter.push_back(ev_i1);
        ev_reb.push_back(ev_r0);
        ev_reb.push_back(ev_r1);
        if (all_done) break;
    }
    const int ev_run1 = h->timer.mark();
    LV_CUDA(cudaStreamSynchronize(s));

    // totals, as lv_run would report them summed over the graphs
    h->stats.num_phases = 0;
    h->stats.total_iterations = 0;
    h->stats.edge_visits = 0;
    for (int32_t g = 0; g < G; ++g) {
        h->stats.num_phases = std::max(h->stats.num_phases, (int32_t)h->info[g].size());
        for (const auto &in : h->info[g]) {
            h->stats.total_iterations += in.iterations;
            h->stats.edge_visits += (int64_t)in.iterations * in.arcs;
        }
    }
    for (size_t q = 0; q + 1 < ev_iter.size(); q += 2) {
        ms_iter += h->timer.ms(ev_iter[q], ev_iter[q + 1]);
        ms_rebuild += h->timer.ms(ev_reb[q], ev_reb[q + 1]);
    }
    for (size_t q = 0; q < h->sweeps.size(); ++q)
        h->sweeps[q].ms = h->timer.ms(ev_sweep[2 * q], ev_sweep[2 * q + 1]);
    h->stats.ms_total = h->timer.ms(ev_run0, ev_run1);
    h->stats.ms_vf = h->timer.ms(ev_vf0, ev_vf1);
    h->stats.ms_color = h->timer.on ? 0.0 : -1.0;
    h->stats.ms_iterate = h->timer.on ? ms_iter : -1.0;
    h->stats.ms_rebuild = h->timer.on ? ms_rebuild : -1.0;
    h->stats.kernel_launches = (int64_t)(g_kernel_launches - launches0);
    h->timer.clear();
    return LV_OK;
}

}  // namespace

extern "C" {

lv_status lv_batch_run(lv_batch *b, const lv_params *p) {
    if (!b) return LV_ERR_ARG;
    lv_params P;
    if (p) P = *p;
    else lv_params_default(&P);
    b->clear_results();
    const lv_status st = batch_run_impl(b, P);
    if (st != LV_OK) {
        cudaStreamSynchronize(b->stream);
        b->clear_results();
        return st;
    }
    b->have_run = true;
    return LV_OK;
}

lv_status lv_batch_get_labels(const lv_batch *b, int32_t graph, int32_t phase, int32_t *out,
                              int ptr_on_device) {
    if (!b || !out || graph < -1 || graph >= b->G) return LV_ERR_ARG;
    if (!b->have_run || b->labels.empty()) return LV_ERR_STATE;
    const int32_t nb = (int32_t)b->labels.size();
    int32_t q;
    if (graph >= 0) {
        const int32_t np = (int32_t)b->info[graph].size();
        q = phase == -1 ? np - 1 : phase;
        if (q < 0 || q >= np) return LV_ERR_STATE;
    } else {
        q = phase == -1 ? nb - 1 : phase;
        if (q < 0 || q >= nb) return LV_ERR_STATE;
    }
    const int32_t lo = graph >= 0 ? b->gptr[graph] : 0;
    const int32_t cnt = graph >= 0 ? b->gptr[graph + 1] - lo : (int32_t)b->n;
    LV_CUDA(cudaMemcpyAsync(out, b->labels[q] + lo, sizeof(int32_t) * (size_t)cnt,
                            ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            b->stream));
    LV_CUDA(cudaStreamSynchronize(b->stream));
    return LV_OK;
}

lv_status lv_batch_get_graph_info(const lv_batch *b, int32_t graph, lv_batch_graph_info *out) {
    if (!b || !out || graph < 0 || graph >= b->G) return LV_ERR_ARG;
    if (!b->have_run) return LV_ERR_STATE;
    const auto &ph = b->info[graph];
    std::memset(out, 0, sizeof *out);
    out->n = b->gptr[graph + 1] - b->gptr[graph];
    out->arcs = b->arcs[graph];
    out->two_m = b->two_m[graph];
    out->num_phases = (int32_t)ph.size();
    for (const auto &in : ph) out->iterations += in.iterations;
    if (!ph.empty()) {
        out->n_final = ph.back().n_next;
        out->N_final = ph.back().N_end;
        out->q = ph.back().q;
    }
    return LV_OK;
}

lv_status lv_batch_get_phase_info(const lv_batch *b, int32_t graph, int32_t phase,
                                  lv_phase_info *out) {
    if (!b || !out || graph < 0 || graph >= b->G) return LV_ERR_ARG;
    if (!b->have_run) return LV_ERR_STATE;
    const auto &ph = b->info[graph];
    const int32_t q = phase == -1 ? (int32_t)ph.size() - 1 : phase;
    if (q < 0 || q >= (int32_t)ph.size()) return LV_ERR_STATE;
    *out = ph[q];
    return LV_OK;
}

lv_status lv_batch_get_num_sweeps(const lv_batch *b, int64_t *count) {
    if (!b || !count) return LV_ERR_ARG;
    if (!b->have_run) return LV_ERR_STATE;
    *count = (int64_t)b->sweeps.size();
    return LV_OK;
}

lv_status lv_batch_get_sweeps(const lv_batch *b, lv_batch_sweep *out, int64_t count) {
    if (!b || (!out && count > 0) || count < 0) return LV_ERR_ARG;
    if (!b->have_run) return LV_ERR_STATE;
    const size_t c = std::min((size_t)count, b->sweeps.size());
    if (c) std::memcpy(out, b->sweeps.data(), c * sizeof(lv_batch_sweep));
    return LV_OK;
}

lv_status lv_batch_get_stats(const lv_batch *b, lv_stats *out) {
    if (!b || !out) return LV_ERR_ARG;
    if (!b->have_run) return LV_ERR_STATE;
    *out = b->stats;
    return LV_OK;
}

}  // extern "C"
