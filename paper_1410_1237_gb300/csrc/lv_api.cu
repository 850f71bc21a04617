// lv_api.cu -- the C ABI (include/lv.h) and the host driver of a run.
//
// Driver (Sec. 4.4): vertex following once, then phases.  A phase colours its
// graph when colouring is on, the graph has at least color_cutoff vertices
// and no earlier coloured phase gained less than theta_high (Sec. 5.1); it
// then iterates Algorithm 1's while-loop and rebuilds the coarse graph.
//
// Uncoloured phases (Jacobi sweeps): the sweep that proposes the moves of
// iteration t also accumulates sum_i e_{i->C(i)} under the labels it reads,
// i.e. the modularity of iteration t-1 (the paper's "pre-aggregation" of the
// modularity terms into the gain loop, Sec. 4.5).  So the stopping test of
// iteration t-1 is evaluated after sweep t and before its moves are applied;
// when it stops, sweep t's proposals are discarded.  One extra sweep per
// phase replaces a separate modularity pass per iteration.
//
// Coloured phases: vertices of one class are pairwise non-adjacent, so when
// a class's movers are applied, sum_i e_{i->C(i)} changes by exactly
// 2 (e_{i->new} - e_{i->old}) per mover; the sweep accumulates that change and
// the numerator is updated exactly after each iteration.
//
// Stopping tests use the signed net gain: (N_C - N_P) < theta |N_P|, on the
// exact numerators converted to double once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "lv_ops.cuh"

using namespace lv;

namespace {

struct PhaseRec {
    lv_phase_info info;
    int32_t *labels = nullptr;  // device, n_orig
    DGraph graph;               // kept copy (keep_graphs)
    int32_t *colors = nullptr;  // kept copy (keep_graphs, coloured phases)
};

std::once_flag g_setup_once;
lv_status g_setup_status = LV_OK;

}  // namespace

lv_status lv::ensure_setup(cudaStream_t s) {
    std::call_once(g_setup_once, [&] {
        void *p = nullptr;
        g_setup_status = dalloc(&p, 16, s);  // creates the pool, reads the SM count
        if (g_setup_status == LV_OK) {
            dfree(p, s);
            g_setup_status = sweep_setup();
        }
    });
    return g_setup_status;
}

struct lv_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0, A = 0, two_m = 0;
    DGraph in;
    int32_t *k_in = nullptr, *loop_in = nullptr;
    int *pinned = nullptr;  // 64 ints of pinned host memory for readbacks
    bool have_run = false;
    std::vector<PhaseRec> phases;
    std::vector<lv_iter_stat> iters;
    lv_stats stats;
    int32_t *vf_map = nullptr;
    Timer timer;
    // bins chosen by measurement per phase index (autotune), kept across runs
    std::vector<BinLimits> tuned;
    std::vector<char> tuned_ok;

    void clear_results() {
        for (auto &p : phases) {
            dfree(p.labels, stream);
            free_graph(p.graph, stream);
            dfree(p.colors, stream);
        }
        phases.clear();
        iters.clear();
        std::memset(&stats, 0, sizeof stats);
        timer.clear();
        have_run = false;
    }
};

extern "C" {

void lv_params_default(lv_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->vertex_following = 1;
    p->coloring = 1;
    p->theta_low = 1e-6;
    p->theta_high = 1e-2;
    p->color_cutoff = 100000;
    p->max_iters = 10000;
    p->max_phases = 64;
    p->color_seed = 0x5EED;
    p->graph_capture = 1;
}

const char *lv_status_string(lv_status s) {
    switch (s) {
    case LV_OK: return "ok";
    case LV_ERR_ARG: return "invalid argument or malformed CSR";
    case LV_ERR_NOT_SYMMETRIC: return "CSR is not symmetric";
    case LV_ERR_WEIGHT: return "weight < 1";
    case LV_ERR_DUPLICATE: return "duplicate column in a row";
    case LV_ERR_OVERFLOW: return "2m >= 2^31 or too many arcs";
    case LV_ERR_EMPTY: return "graph has no edges (m = 0)";
    case LV_ERR_CUDA: return "CUDA error";
    case LV_ERR_OOM: return "device out of memory";
    case LV_ERR_TIMEOUT: return "bounded device wait expired";
    case LV_ERR_STATE: return "no such result (run first / phase out of range)";
    case LV_ERR_HASH: return "hash table probe bound exceeded";
    }
    return "unknown status";
}

lv_status lv_graph_create(lv_graph **out, int64_t n, const int64_t *rowptr, const int32_t *col,
                          const int32_t *w, int ptrs_on_device, void *cuda_stream) {
    if (!out) return LV_ERR_ARG;
    *out = nullptr;
    if (n < 0 || n > 0x7ffffffell || !rowptr) return LV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    LV_TRY(ensure_setup(s));
    const int64_t *d_rowptr = rowptr;
    const int32_t *d_col = col, *d_w = w;
    int64_t *st_rowptr = nullptr;
    int32_t *st_col = nullptr, *st_w = nullptr;
    if (!ptrs_on_device) {
        // stage host arrays on the device; validation runs there
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
    lv_graph *g = new lv_graph();
    g->stream = s;
    cudaGetDevice(&g->device);
    if (cudaMallocHost((void **)&g->pinned, 64 * sizeof(int)) != cudaSuccess) {
        delete g;
        return LV_ERR_OOM;
    }
    g->timer.s = s;
    lv_status st = validate_and_build(n, d_rowptr, d_col, d_w, &g->in, &g->k_in, &g->loop_in,
                                      &g->two_m, g->pinned, s);
    dfree(st_rowptr, s);
    dfree(st_col, s);
    dfree(st_w, s);
    if (st != LV_OK) {
        cudaStreamSynchronize(s);
        cudaFreeHost(g->pinned);
        delete g;
        return st;
    }
    g->n = n;
    g->A = g->in.A;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        lv_graph_destroy(g);
        return LV_ERR_CUDA;
    }
    *out = g;
    return LV_OK;
}

void lv_graph_destroy(lv_graph *g) {
    if (!g) return;
    g->clear_results();
    free_graph(g->in, g->stream);
    dfree(g->k_in, g->stream);
    dfree(g->loop_in, g->stream);
    dfree(g->vf_map, g->stream);
    cudaStreamSynchronize(g->stream);
    if (g->pinned) cudaFreeHost(g->pinned);
    delete g;
}

}  // extern "C"

namespace {

struct IterResult {
    int32_t iters = 0;
    int64_t N = 0;
};

lv_status read_stats(lv_graph *h, const PhaseState &ps, IterStats *hs) {
    LV_CUDA(cudaMemcpyAsync(h->pinned, ps.stats, sizeof(IterStats), cudaMemcpyDeviceToHost, h->stream));
    LV_CUDA(cudaStreamSynchronize(h->stream));
    std::memcpy(hs, h->pinned, sizeof(IterStats));
    if (barrier_flags(hs->bar)) return LV_ERR_TIMEOUT;
    if (hs->err) return LV_ERR_HASH;
    return LV_OK;
}

struct IterRecord {
    lv_iter_stat st;
    int ev0 = -1, ev1 = -1;
};

// Uncoloured phase: fused Jacobi sweeps (see the file comment).
lv_status iterate_jacobi(lv_graph *h, PhaseState &ps, const Buckets &b, const BinLimits &lim,
                         double theta, bool abs_mode, int32_t max_iters, int phase,
                         std::vector<IterRecord> &recs, IterResult *out) {
    cudaStream_t s = h->stream;
    bool have_np = false;
    int64_t n_p = 0;
    int64_t moved_prev = 0;
    int ev_prev0 = -1, ev_prev1 = -1;
    auto record = [&](int t, int64_t moved, int64_t N, int e0, int e1) {
        IterRecord r;
        r.st.phase = phase;
        r.st.iter = t;
        r.st.color_steps = 1;
        r.st.moved = moved;
        r.st.N = N;
        r.st.arcs = ps.g.A;
        r.st.ms = -1.0;
        r.ev0 = e0;
        r.ev1 = e1;
        recs.push_back(r);
    };
    for (int step = 1;; ++step) {
        LV_CUDA(cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s));
        LV_CUDA(cudaMemsetAsync(ps.move_count, 0, 3 * sizeof(int32_t), s));
        const int e0 = h->timer.mark();
        LV_TRY(sweep_iteration(ps, b, s));
        ++h->stats.sweep_launches;
        const int e1 = h->timer.mark();
        IterStats hs;
        LV_TRY(read_stats(h, ps, &hs));
        const int64_t N_prev = ps.two_m * (int64_t)hs.sum_ein - (int64_t)hs.sum_a2;  // N(C^{step-1})
        const int64_t moved = hs.moved;
        if (step == 1) {
            if (moved == 0) {
                record(1, 0, N_prev, e0, e1);
                out->iters = 1;
                out->N = N_prev;
                return LV_OK;
            }
        } else {
            const int t = step - 1;
            record(t, moved_prev, N_prev, ev_prev0, ev_prev1);
            if ((have_np && gain_below(N_prev, n_p, theta, abs_mode)) || t >= max_iters) {
                out->iters = t;
                out->N = N_prev;
                return LV_OK;
            }
            n_p = N_prev;
            have_np = true;
            if (moved == 0) {
                record(step, 0, N_prev, e0, e1);
                out->iters = step;
                out->N = N_prev;
                return LV_OK;
            }
        }
        LV_TRY(apply_moves(ps, s));
        moved_prev = moved;
        ev_prev0 = e0;
        ev_prev1 = e1;
    }
}

// Coloured phase: classes in ascending colour, moves applied after each class.
lv_status iterate_colored(lv_graph *h, PhaseState &ps, const Buckets &b, const BinLimits &lim,
                          double theta, bool abs_mode, int32_t max_iters, int phase,
                          int64_t sum_loops, std::vector<IterRecord> &recs, IterResult *out) {
    cudaStream_t s = h->stream;
    bool have_np = false;
    int64_t n_p = 0;
    int64_t sum_ein = sum_loops;
    for (int t = 1;; ++t) {
        LV_CUDA(cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s));
        LV_CUDA(cudaMemsetAsync(ps.move_count, 0, 3 * sizeof(int32_t) * (size_t)ps.n_act, s));
        const int e0 = h->timer.mark();
        LV_TRY(sweep_iteration(ps, b, s));
        ++h->stats.sweep_launches;
        const int e1 = h->timer.mark();
        IterStats hs;
        LV_TRY(read_stats(h, ps, &hs));
        sum_ein += (int64_t)hs.delta_ein;
        const int64_t N = ps.two_m * sum_ein - (int64_t)hs.sum_a2;
        IterRecord r;
        r.st.phase = phase;
        r.st.iter = t;
        r.st.color_steps = (int32_t)ps.n_act;
        r.st.moved = hs.moved;
        r.st.N = N;
        r.st.arcs = ps.g.A;
        r.st.ms = -1.0;
        r.ev0 = e0;
        r.ev1 = e1;
        recs.push_back(r);
        if (hs.moved == 0 || (have_np && gain_below(N, n_p, theta, abs_mode)) || t >= max_iters) {
            out->iters = t;
            out->N = N;
            return LV_OK;
        }
        n_p = N;
        have_np = true;
    }
}

lv_status copy_graph(const DGraph &src, DGraph *dst, cudaStream_t s) {
    dst->n = src.n;
    dst->A = src.A;
    LV_TRY(dalloc_n(&dst->off, (size_t)src.n + 1, s));
    LV_TRY(dalloc_n(&dst->arcs, (size_t)src.A, s));
    LV_CUDA(cudaMemcpyAsync(dst->off, src.off, sizeof(int32_t) * ((size_t)src.n + 1),
                            cudaMemcpyDeviceToDevice, s));
    if (src.A)
        LV_CUDA(cudaMemcpyAsync(dst->arcs, src.arcs, sizeof(int2) * (size_t)src.A,
                                cudaMemcpyDeviceToDevice, s));
    return LV_OK;
}

lv_status run_impl(lv_graph *h, const lv_params &P) {
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
        !(P.theta_high >= 0.0) || P.color_order < 0 || P.color_order > 1)
        return LV_ERR_ARG;
    h->timer.on = P.collect_timing != 0;
    const unsigned long long launches0 = g_kernel_launches;
    const int ev_run0 = h->timer.mark();
    const int32_t n_orig = (int32_t)h->n;
    if (!h->vf_map) LV_TRY(dalloc_n(&h->vf_map, (size_t)n_orig, s));

    // ---- step 1: vertex following (once, Sec. 4.4)
    DGraph G = h->in;
    bool own_g = false;
    const int32_t *k = h->k_in, *loop = h->loop_in;
    int32_t *k_own = nullptr, *loop_own = nullptr;
    const int ev_vf0 = h->timer.mark();
    if (P.vertex_following) {
        DGraph G2;
        LV_TRY(vertex_following(G, h->loop_in, &G2, h->vf_map, h->pinned, s));
        if (P.vf_recursive) {
            int32_t vf_rounds = 0;
            const lv_status st_vf = vf_recursive(&G2, h->two_m, h->vf_map, n_orig, h->pinned,
                                                 &vf_rounds, s);
            if (st_vf != LV_OK) {
                free_graph(G2, s);
                return st_vf;
            }
        }
        G = G2;
        own_g = true;
        LV_TRY(dalloc_n(&k_own, (size_t)G.n, s));
        LV_TRY(dalloc_n(&loop_own, (size_t)G.n, s));
        LV_TRY(compute_degrees(G, k_own, loop_own, s));
        k = k_own;
        loop = loop_own;
    } else {
        LV_TRY(iota(n_orig, h->vf_map, s));
    }
    const int ev_vf1 = h->timer.mark();
    h->stats.vf_n = G.n;

    int32_t *map = nullptr;
    LV_TRY(dalloc_n(&map, (size_t)n_orig, s));
    LV_CUDA(cudaMemcpyAsync(map, h->vf_map, sizeof(int32_t) * (size_t)n_orig,
                            cudaMemcpyDeviceToDevice, s));

    // per-vertex state, sized for the largest (first) phase graph
    const int nmax = G.n;
    PhaseState ps;
    int32_t *newid = nullptr, *color = nullptr;
    LV_TRY(dalloc_n(&ps.C, (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.comm[0], (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.comm[1], (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.moves[0], (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.moves[1], (size_t)nmax, s));
    LV_TRY(dalloc_n(&ps.stats, 1, s));
    ps.bar = &ps.stats->bar;
    LV_TRY(dalloc_n(&newid, (size_t)nmax + 1, s));
    LV_TRY(dalloc_n(&color, (size_t)nmax, s));
    ps.two_m = h->two_m;

    std::vector<IterRecord> recs;
    struct PhaseEvents {
        int c0, c1, i0, i1, r0, r1;
    };
    std::vector<PhaseEvents> phase_events;
    bool colour_stopped = false;
    int32_t coloured_phases = 0;
    lv_status st = LV_OK;
    for (int32_t p = 0; p < P.max_phases; ++p) {
        // persistent kernels of a small phase graph run on fewer SMs: fewer
        // barrier arrivals and claims, and the graph's work still fills them
        const int phase_sms = P.persistent_sms > 0 ? std::min(P.persistent_sms, auto_sms(G.A))
                                                   : auto_sms(G.A);
        PhaseRec rec;
        std::memset(&rec.info, 0, sizeof rec.info);
        lv_phase_info &info = rec.info;
        info.n = G.n;
        info.arcs = G.A;
        info.two_m = h->two_m;
        const bool colour_on = P.coloring && !colour_stopped && (int64_t)G.n >= P.color_cutoff &&
                               (P.color_phases <= 0 || coloured_phases < P.color_phases);
        coloured_phases += colour_on ? 1 : 0;
        const double theta = (colour_on && P.theta_high > 0.0) ? P.theta_high : P.theta_low;
        info.colored = colour_on ? 1 : 0;
        info.theta = theta;

        // ---- colouring and vertex order
        const int ev_c0 = h->timer.mark();
        int32_t K = 1;
        int32_t rounds = 0;
        if (colour_on)
            LV_TRY(jp_color(G, P.color_seed + (uint64_t)p, P.color_order == 0, color, &K, &rounds,
                            h->pinned, s, phase_sms));
        info.color_rounds = rounds;
        info.num_colors = colour_on ? K : 0;
        BinLimits plim = lim;
        plim.sms = phase_sms;
        if (P.autotune && !colour_on && (int64_t)G.A >= kTuneMinArcs) {
            if ((int32_t)h->tuned.size() <= p || !h->tuned_ok[p]) {
                // time candidate bins on the phase's initial state (a scratch
                // phase state over the run's buffers; the phase starts afresh)
                PhaseState tp = ps;
                tp.g = G;
                tp.k = k;
                tp.loop = loop;
                tp.coloured = false;
                tp.n_act = 1;
                tp.act = nullptr;
                tp.move_count = nullptr;
                BinLimits best = lim;
                lv_status ts = dalloc_n(&tp.act, 1, s);
                if (ts == LV_OK) ts = dalloc_n(&tp.move_count, 4, s);
                if (ts == LV_OK && cudaMemsetAsync(tp.act, 0, sizeof(int32_t), s) != cudaSuccess)
                    ts = LV_ERR_CUDA;
                if (ts == LV_OK) ts = init_phase(tp, s);
                if (ts == LV_OK) ts = tune_bins(tp, lim, nullptr, 0, &best, h->pinned, s);
                dfree(tp.act, s);
                dfree(tp.move_count, s);
                LV_TRY(ts);
                if ((int32_t)h->tuned.size() <= p) {
                    h->tuned.resize(p + 1);
                    h->tuned_ok.resize(p + 1, 0);
                }
                h->tuned[p] = best;
                h->tuned_ok[p] = 1;
            }
            plim = h->tuned[p];
            plim.sms = phase_sms;
        }
        Buckets b;
        LV_TRY(bucket_vertices(G, colour_on ? color : nullptr, K, plim, &b, h->pinned, s));
        const int ev_c1 = h->timer.mark();
        if (P.keep_graphs) {
            LV_TRY(copy_graph(G, &rec.graph, s));
            if (colour_on) {
                LV_TRY(dalloc_n(&rec.colors, (size_t)G.n, s));
                LV_CUDA(cudaMemcpyAsync(rec.colors, color, sizeof(int32_t) * (size_t)G.n,
                                        cudaMemcpyDeviceToDevice, s));
            }
        }

        // ---- iterations (Alg. 1)
        ps.g = G;
        ps.k = k;
        ps.loop = loop;
        ps.coloured = colour_on;
        {
            // classes holding at least one vertex with arcs, in ascending colour
            std::vector<int32_t> act;
            for (int c = 0; c < K; ++c)
                if (b.host_off[c * (kBins + 1) + kBins] > b.host_off[c * (kBins + 1)]) act.push_back(c);
            if (act.empty()) act.push_back(0);
            ps.n_act = (int)act.size();
            LV_TRY(dalloc_n(&ps.act, act.size(), s));
            LV_CUDA(cudaMemcpyAsync(ps.act, act.data(), sizeof(int32_t) * act.size(),
                                    cudaMemcpyHostToDevice, s));
        }
        LV_TRY(dalloc_n(&ps.move_count, 3 * (size_t)ps.n_act + 1, s));
        const int ev_i0 = h->timer.mark();
        LV_TRY(init_phase(ps, s));
        IterStats hs0;
        LV_TRY(read_stats(h, ps, &hs0));
        info.N_start = ps.two_m * (int64_t)hs0.sum_ein - (int64_t)hs0.sum_a2;
        IterResult ir;
        if (colour_on)
            st = iterate_colored(h, ps, b, lim, theta, P.abs_threshold != 0, P.max_iters, p,
                                 (int64_t)hs0.sum_ein, recs, &ir);
        else
            st = iterate_jacobi(h, ps, b, lim, theta, P.abs_threshold != 0, P.max_iters, p, recs,
                                &ir);
        if (st != LV_OK) return st;
        const int ev_i1 = h->timer.mark();
        info.iterations = ir.iters;
        info.N_end = ir.N;
        info.q = (double)ir.N / (double)(h->two_m * h->two_m);

        // ---- rebuild (Sec. 4.5): renumber, labels, coarse graph
        const int ev_r0 = h->timer.mark();
        LV_TRY(renumber(G.n, current_comm(ps), newid, s));
        LV_CUDA(cudaMemcpyAsync(h->pinned, newid + G.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        const int32_t n_next = h->pinned[0];
        info.n_next = n_next;
        LV_TRY(dalloc_n(&rec.labels, (size_t)n_orig, s));
        LV_TRY(compose_labels(n_orig, map, ps.C, newid, rec.labels, s));

        bool stop = false;
        if (n_next == G.n) stop = true;
        else if (colour_on) {
            if (P.theta_high > 0.0 &&
                gain_below(info.N_end, info.N_start, P.theta_high, P.abs_threshold != 0))
                colour_stopped = true;
        } else if (gain_below(info.N_end, info.N_start, P.theta_low, P.abs_threshold != 0)) {
            stop = true;
        }
        if (p + 1 >= P.max_phases) stop = true;
        if (!stop) {
            DGraph G2;
            LV_TRY(coarsen(G, ps.C, newid, n_next, &G2, h->pinned, s));
            int32_t *k2 = nullptr, *l2 = nullptr;
            LV_TRY(dalloc_n(&k2, (size_t)G2.n, s));
            LV_TRY(dalloc_n(&l2, (size_t)G2.n, s));
            LV_TRY(compute_degrees(G2, k2, l2, s));
            if (own_g) free_graph(G, s);
            dfree(k_own, s);
            dfree(loop_own, s);
            G = G2;
            own_g = true;
            k = k_own = k2;
            loop = loop_own = l2;
        }
        const int ev_r1 = h->timer.mark();
        LV_CUDA(cudaStreamSynchronize(s));  // the host copy of act must outlive its transfer
        dfree(ps.move_count, s);
        ps.move_count = nullptr;
        dfree(ps.act, s);
        ps.act = nullptr;
        free_buckets(b, s);
        info.ms_color = -1.0;
        info.ms_iterate = -1.0;
        info.ms_rebuild = -1.0;
        h->phases.push_back(rec);
        phase_events.push_back({ev_c0, ev_c1, ev_i0, ev_i1, ev_r0, ev_r1});
        if (stop) break;
    }
    const int ev_run1 = h->timer.mark();
    LV_CUDA(cudaStreamSynchronize(s));

    // totals
    h->stats.num_phases = (int32_t)h->phases.size();
    h->stats.total_iterations = 0;
    h->stats.edge_visits = 0;
    for (auto &r : recs) {
        r.st.ms = h->timer.ms(r.ev0, r.ev1);
        h->iters.push_back(r.st);
        h->stats.total_iterations++;
        h->stats.edge_visits += r.st.arcs;
    }
    h->stats.ms_total = h->timer.ms(ev_run0, ev_run1);
    h->stats.kernel_launches = (int64_t)(g_kernel_launches - launches0);
    h->stats.ms_vf = h->timer.ms(ev_vf0, ev_vf1);
    for (size_t q = 0; q < h->phases.size(); ++q) {
        const PhaseEvents &pe = phase_events[q];
        h->phases[q].info.ms_color = h->timer.ms(pe.c0, pe.c1);
        h->phases[q].info.ms_iterate = h->timer.ms(pe.i0, pe.i1);
        h->phases[q].info.ms_rebuild = h->timer.ms(pe.r0, pe.r1);
    }
    double mc = 0, mi = 0, mr = 0;
    for (auto &ph : h->phases) {
        mc += ph.info.ms_color;
        mi += ph.info.ms_iterate;
        mr += ph.info.ms_rebuild;
    }
    h->stats.ms_color = h->timer.on ? mc : -1.0;
    h->stats.ms_iterate = h->timer.on ? mi : -1.0;
    h->stats.ms_rebuild = h->timer.on ? mr : -1.0;

    if (own_g) free_graph(G, s);
    dfree(k_own, s);
    dfree(loop_own, s);
    dfree(map, s);
    dfree(ps.C, s);
    dfree(ps.comm[0], s);
    dfree(ps.comm[1], s);
    dfree(ps.moves[0], s);
    dfree(ps.moves[1], s);
    dfree(ps.stats, s);
    dfree(newid, s);
    dfree(color, s);
    LV_CUDA(cudaStreamSynchronize(s));
    h->timer.clear();
    return st;
}

const PhaseRec *phase_at(const lv_graph *g, int32_t phase) {
    if (!g || !g->have_run || g->phases.empty()) return nullptr;
    if (phase == -1) phase = (int32_t)g->phases.size() - 1;
    if (phase < 0 || phase >= (int32_t)g->phases.size()) return nullptr;
    return &g->phases[phase];
}

}  // namespace

extern "C" {

lv_status lv_run(lv_graph *g, const lv_params *p) {
    if (!g) return LV_ERR_ARG;
    lv_params P;
    if (p) P = *p;
    else lv_params_default(&P);
    g->clear_results();
    lv_status st = run_impl(g, P);
    if (st != LV_OK) {
        cudaStreamSynchronize(g->stream);
        g->clear_results();
        return st;
    }
    g->have_run = true;
    return LV_OK;
}

lv_status lv_num_phases(const lv_graph *g, int32_t *out) {
    if (!g || !out) return LV_ERR_ARG;
    if (!g->have_run) return LV_ERR_STATE;
    *out = (int32_t)g->phases.size();
    return LV_OK;
}

lv_status lv_get_labels(const lv_graph *g, int32_t phase, int32_t *out, int ptr_on_device) {
    if (!g || !out) return LV_ERR_ARG;
    const PhaseRec *r = phase_at(g, phase);
    if (!r) return LV_ERR_STATE;
    LV_CUDA(cudaMemcpyAsync(out, r->labels, sizeof(int32_t) * (size_t)g->n,
                            ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            g->stream));
    LV_CUDA(cudaStreamSynchronize(g->stream));
    return LV_OK;
}

lv_status lv_get_modularity(const lv_graph *g, int32_t phase, double *q, int64_t *num_hi,
                            uint64_t *num_lo, int64_t *den) {
    if (!g) return LV_ERR_ARG;
    const PhaseRec *r = phase_at(g, phase);
    if (!r) return LV_ERR_STATE;
    if (q) *q = r->info.q;
    if (num_hi) *num_hi = r->info.N_end < 0 ? -1 : 0;
    if (num_lo) *num_lo = (uint64_t)r->info.N_end;
    if (den) *den = g->two_m * g->two_m;
    return LV_OK;
}

lv_status lv_get_phase_info(const lv_graph *g, int32_t phase, lv_phase_info *out) {
    if (!g || !out) return LV_ERR_ARG;
    const PhaseRec *r = phase_at(g, phase);
    if (!r) return LV_ERR_STATE;
    *out = r->info;
    return LV_OK;
}

lv_status lv_get_num_iterations(const lv_graph *g, int64_t *count) {
    if (!g || !count) return LV_ERR_ARG;
    if (!g->have_run) return LV_ERR_STATE;
    *count = (int64_t)g->iters.size();
    return LV_OK;
}

lv_status lv_get_iteration_stats(const lv_graph *g, lv_iter_stat *out, int64_t count) {
    if (!g || (!out && count > 0) || count < 0) return LV_ERR_ARG;
    if (!g->have_run) return LV_ERR_STATE;
    const int64_t n = count < (int64_t)g->iters.size() ? count : (int64_t)g->iters.size();
    for (int64_t i = 0; i < n; ++i) out[i] = g->iters[i];
    return LV_OK;
}

lv_status lv_get_stats(const lv_graph *g, lv_stats *out) {
    if (!g || !out) return LV_ERR_ARG;
    if (!g->have_run) return LV_ERR_STATE;
    *out = g->stats;
    return LV_OK;
}

lv_status lv_get_tuning(const lv_graph *g, int32_t phase, int32_t *out) {
    if (!g || !out) return LV_ERR_ARG;
    if (phase < 0 || phase >= (int32_t)g->tuned.size() || !g->tuned_ok[phase]) return LV_ERR_STATE;
    const BinLimits &t = g->tuned[phase];
    out[0] = t.lane_arcs;
    out[1] = t.warp_max;
    out[2] = t.cta_max;
    out[3] = t.blocks_per_sm;
    out[4] = t.hub_factor;
    return LV_OK;
}

lv_status lv_get_vf_map(const lv_graph *g, int32_t *out, int ptr_on_device) {
    if (!g || !out) return LV_ERR_ARG;
    if (!g->have_run) return LV_ERR_STATE;
    LV_CUDA(cudaMemcpyAsync(out, g->vf_map, sizeof(int32_t) * (size_t)g->n,
                            ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            g->stream));
    LV_CUDA(cudaStreamSynchronize(g->stream));
    return LV_OK;
}

lv_status lv_get_phase_graph(const lv_graph *g, int32_t phase, int64_t *n, int64_t *arcs,
                             int64_t *rowptr, int32_t *col, int32_t *w, int ptrs_on_device) {
    if (!g) return LV_ERR_ARG;
    const PhaseRec *r = phase_at(g, phase);
    if (!r || !r->graph.off) return LV_ERR_STATE;
    if (n) *n = r->graph.n;
    if (arcs) *arcs = r->graph.A;
    if (!rowptr && !col && !w) return LV_OK;
    std::vector<int32_t> off((size_t)r->graph.n + 1);
    std::vector<int2> a((size_t)r->graph.A);
    LV_CUDA(cudaMemcpyAsync(off.data(), r->graph.off, sizeof(int32_t) * off.size(),
                            cudaMemcpyDeviceToHost, g->stream));
    if (!a.empty())
        LV_CUDA(cudaMemcpyAsync(a.data(), r->graph.arcs, sizeof(int2) * a.size(),
                                cudaMemcpyDeviceToHost, g->stream));
    LV_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<int64_t> rp(off.begin(), off.end());
    std::vector<int32_t> c(a.size()), ww(a.size());
    for (size_t e = 0; e < a.size(); ++e) {
        c[e] = a[e].x;
        ww[e] = a[e].y;
    }
    const cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    if (rowptr) LV_CUDA(cudaMemcpy(rowptr, rp.data(), sizeof(int64_t) * rp.size(), kind));
    if (col && !c.empty()) LV_CUDA(cudaMemcpy(col, c.data(), sizeof(int32_t) * c.size(), kind));
    if (w && !ww.empty()) LV_CUDA(cudaMemcpy(w, ww.data(), sizeof(int32_t) * ww.size(), kind));
    return LV_OK;
}

lv_status lv_get_phase_colors(const lv_graph *g, int32_t phase, int32_t *out, int ptr_on_device) {
    if (!g || !out) return LV_ERR_ARG;
    const PhaseRec *r = phase_at(g, phase);
    if (!r || !r->colors) return LV_ERR_STATE;
    LV_CUDA(cudaMemcpyAsync(out, r->colors, sizeof(int32_t) * (size_t)r->info.n,
                            ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            g->stream));
    LV_CUDA(cudaStreamSynchronize(g->stream));
    return LV_OK;
}

}  // extern "C"
