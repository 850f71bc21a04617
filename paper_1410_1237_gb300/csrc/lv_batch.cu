// lv_batch.cu -- batched runs: many independent graphs behind one handle.
//
// A batch validates the disjoint union of its graphs once (lv_batch_create);
// each run hands the union to the multi-graph engine (lv_engine.cu), which
// takes every graph through its own phases with batched sweeps, and records
// per graph what lv_run records for it alone.  Graphs leave the engine when
// their phase loop stops, so later phases sweep and rebuild only the graphs
// still running.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lv_engine.cuh"

using namespace lv;

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
    LV_TRY(graph_of((int32_t)b->n, G, b->gptr_in, b->gid_in, s));
    int *bad = nullptr;
    unsigned long long *sk = nullptr;
    int32_t *starts = nullptr;
    LV_TRY(dalloc_n(&bad, 1, s));
    LV_TRY(dalloc_n(&sk, (size_t)G, s));
    LV_TRY(dalloc_n(&starts, (size_t)G + 1, s));
    LV_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    LV_CUDA(cudaMemsetAsync(sk, 0, sizeof(unsigned long long) * G, s));
    LV_TRY(cross_check(b->in, b->gid_in, b->gptr_in, bad, s));
    LV_TRY(graph_sums((int32_t)b->n, b->gid_in, b->k_in, b->loop_in, nullptr, sk, nullptr, nullptr, s));
    LV_TRY(gather_at(G, b->gptr_in, b->in.off, starts, s));
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

lv_status batch_run_impl(lv_batch *h, const lv_params &P) {
    cudaStream_t s = h->stream;
    BinLimits lim;
    if (P.bin_lane_arcs) lim.lane_arcs = P.bin_lane_arcs;
    if (P.bin_warp_max) lim.warp_max = P.bin_warp_max;
    if (P.bin_cta_max) lim.cta_max = P.bin_cta_max;
    lim.blocks_per_sm = P.sweep_blocks_per_sm;
    lim.hub_factor = P.hub_slots_per_arc;
    lim.sms = P.persistent_sms;
    if (lim.lane_arcs < 1 || lim.lane_arcs > kLaneArcsLimit || lim.warp_max < 1 ||
        lim.warp_max > kWarpMaxLimit || lim.cta_max <= lim.warp_max || lim.cta_max > kCtaMaxLimit ||
        !valid_shape(lim))
        return LV_ERR_ARG;
    if (P.max_iters < 1 || P.max_phases < 1 || !(P.theta_low >= -1e300) ||
        !(P.theta_high >= 0.0))
        return LV_ERR_ARG;
    const int32_t G = h->G;
    const int32_t n_orig = (int32_t)h->n;
    h->timer.on = P.collect_timing != 0;
    const unsigned long long launches0 = g_kernel_launches;
    const int ev_run0 = h->timer.mark();
    h->info.assign(G, std::vector<lv_phase_info>());

    Engine e;
    e.s = s;
    e.P = P;
    e.lim = lim;
    e.pinned = h->pinned;
    e.timer = &h->timer;
    e.tuned = &h->tuned;
    e.tuned_ok = &h->tuned_ok;

    // ---- vertex following of every graph and the engine's union
    const int ev_vf0 = h->timer.mark();
    NewGraphs ng;
    ng.g = h->in;
    ng.k = h->k_in;
    ng.loop = h->loop_in;
    ng.gptr = h->gptr;
    ng.two_m = h->two_m;
    ng.tags.resize(G);
    for (int32_t q = 0; q < G; ++q) ng.tags[q] = q;
    LV_TRY(e.append(ng));
    const int ev_vf1 = h->timer.mark();
    h->stats.vf_n = e.g.n;
    if (P.coloring)
        for (int32_t q = 0; q < G; ++q)
            if ((int64_t)(e.gp[q + 1] - e.gp[q]) >= P.color_cutoff) return LV_ERR_ARG;

    // labels of every graph after each phase (final ones for graphs that left)
    int32_t *cur = nullptr, *dst_off = nullptr;
    struct Free {
        cudaStream_t s;
        int32_t **a, **b;
        ~Free() {
            dfree(*a, s);
            dfree(*b, s);
        }
    } fr{s, &cur, &dst_off};
    LV_TRY(dalloc_n(&cur, (size_t)n_orig, s));
    LV_TRY(dalloc_n(&dst_off, (size_t)G, s));
    std::vector<int32_t> off_h((size_t)G);
    std::vector<Finished> fin;
    while (e.num_graphs() > 0) {
        LV_TRY(e.phase_run());
        // engine position q holds batch graph tag; its original vertices move
        // from the engine's order to the batch's
        const int32_t Gq = e.num_graphs();
        for (int32_t q = 0; q < Gq; ++q)
            off_h[q] = h->gptr[e.graphs[q].tag] - e.optr[q];
        LV_CUDA(cudaMemcpyAsync(dst_off, off_h.data(), sizeof(int32_t) * Gq, cudaMemcpyHostToDevice, s));
        LV_TRY(scatter_blocks((int32_t)e.n_orig, e.gid_orig, dst_off, e.labels, cur, s));
        int32_t *snap = nullptr;
        LV_TRY(dalloc_n(&snap, (size_t)n_orig, s));
        h->labels.push_back(snap);
        LV_CUDA(cudaMemcpyAsync(snap, cur, sizeof(int32_t) * (size_t)n_orig, cudaMemcpyDeviceToDevice, s));
        LV_CUDA(cudaStreamSynchronize(s));  // off_h is read by the copy above
        for (int32_t q = 0; q < Gq; ++q) h->info[e.graphs[q].tag] = e.graphs[q].info;
        fin.clear();
        LV_TRY(e.phase_end(fin));
    }
    const int ev_run1 = h->timer.mark();
    LV_CUDA(cudaStreamSynchronize(s));

    // totals, as lv_run would report them summed over the graphs
    h->sweeps = e.sweeps;
    h->stats.sweep_launches = e.sweep_launches;
    h->stats.graph_launches = e.graph_launches;
    h->stats.num_phases = 0;
    h->stats.total_iterations = 0;
    h->stats.edge_visits = 0;
    for (int32_t q = 0; q < G; ++q) {
        h->stats.num_phases = std::max(h->stats.num_phases, (int32_t)h->info[q].size());
        for (const auto &in : h->info[q]) {
            h->stats.total_iterations += in.iterations;
            h->stats.edge_visits += (int64_t)in.iterations * in.arcs;
        }
    }
    double ms_iter = 0.0, ms_rebuild = 0.0;
    for (size_t q = 0; q + 1 < e.ev_iter.size(); q += 2) ms_iter += h->timer.ms(e.ev_iter[q], e.ev_iter[q + 1]);
    for (size_t q = 0; q + 1 < e.ev_reb.size(); q += 2) ms_rebuild += h->timer.ms(e.ev_reb[q], e.ev_reb[q + 1]);
    for (size_t q = 0; q < h->sweeps.size() && 2 * q + 1 < e.ev_sweep.size(); ++q)
        h->sweeps[q].ms = h->timer.ms(e.ev_sweep[2 * q], e.ev_sweep[2 * q + 1]);
    if (!h->timer.on)
        for (auto &sw : h->sweeps) sw.ms = -1.0;
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
    if (P.vf_recursive) return LV_ERR_ARG;  // single-graph runs only
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

lv_status lv_batch_get_tuning(const lv_batch *b, int32_t round, int32_t *out) {
    if (!b || !out) return LV_ERR_ARG;
    if (round < 0 || round >= (int32_t)b->tuned.size() || !b->tuned_ok[round])
        return LV_ERR_STATE;
    const BinLimits &t = b->tuned[round];
    out[0] = t.lane_arcs;
    out[1] = t.warp_max;
    out[2] = t.cta_max;
    out[3] = t.blocks_per_sm;
    out[4] = t.hub_factor;
    return LV_OK;
}

}  // extern "C"
