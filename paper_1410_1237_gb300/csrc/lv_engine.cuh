// lv_engine.cuh -- the multi-graph engine behind batched runs and serving.
//
// The engine holds a set of resident graphs as one disjoint union (vertices
// numbered graph after graph, gid[v] = position of v's graph) together with
// the union of their original vertices (map[u] = vertex of the phase graph
// holding original vertex u).  One phase takes every resident graph
// through one phase of Algorithm 1 with its own 2m and stopping tests
// (batched sweeps over the graphs still iterating, fused modularity per
// graph), then one renumber / compose / coarsen pass over the union; graphs
// whose phase loop stops leave the union (phase_run, then phase_end) and are
// reported with their final labels.  append() adds validated graphs (vertex
// following applied) at a phase boundary, so new graphs join the sweeps of
// those already running.
// Every graph follows exactly the control of the single-graph driver, so
// its results do not depend on the other graphs.
#pragma once

#include <vector>

#include "lv_ops.cuh"

namespace lv {

// control state and records of one resident graph
struct EngineGraph {
    int64_t tag = 0;          // caller's id (batch index, request id)
    int32_t n_orig = 0;       // vertices of the input graph
    long long two_m = 0;
    std::vector<lv_phase_info> info;  // one record per finished phase
    // the current phase (the single-graph driver's locals)
    bool running = false;
    bool stop = false;        // its phase loop ends after the current phase
    int step = 0;
    bool have_np = false;
    int64_t n_p = 0, N_start = 0, N_end = 0;
    int32_t iters = 0;
    int64_t n = 0, arcs = 0;  // its current phase graph
};

// New graphs for append(): a validated union on the device, owned by the
// caller until append() returns (the engine copies what it keeps).
struct NewGraphs {
    DGraph g;
    const int32_t *k = nullptr, *loop = nullptr;
    std::vector<int32_t> gptr;       // host, vertex starts (G+1)
    std::vector<long long> two_m;    // host, per graph
    std::vector<int64_t> tags;       // host, per graph
};

// New graphs after vertex following, ready to join an engine (device memory
// owned here; made on any stream, complete when prepare_graphs returns).
struct Prepared {
    cudaStream_t s = nullptr;
    NewGraphs ng;               // ng.g, ng.k, ng.loop are owned when own_input
    bool own_input = false;
    DGraph vf;                  // the graphs after vertex following (owned when own_vf)
    bool own_vf = false;
    int32_t *vmap = nullptr;    // original vertex -> vertex of vf
    std::vector<int32_t> vgp;   // starts of the graphs in vf
    void release();
    ~Prepared() { release(); }
};
// Vertex following (when P.vertex_following) of a validated union.
lv_status prepare_graphs(const NewGraphs &ng, const lv_params &P, int *pinned, cudaStream_t s,
                         Prepared *out);

// a graph that left the engine after phase()
struct Finished {
    EngineGraph rec;
    int32_t lab_off = 0;  // its labels start at labels[lab_off] of phase()'s label output
};

// helpers shared with the batch and server entry points
lv_status graph_of(int32_t n, int32_t G, const int32_t *gptr, int32_t *gid, cudaStream_t s);
lv_status cross_check(const DGraph &g, const int32_t *gid, const int32_t *gptr, int *bad,
                      cudaStream_t s);
lv_status graph_sums(int32_t n, const int32_t *gid, const int32_t *k, const int32_t *loop,
                     const uint8_t *active, unsigned long long *sum_k, unsigned long long *sum_loop,
                     unsigned long long *sum_k2, cudaStream_t s);
lv_status gather_at(int32_t G, const int32_t *idx, const int32_t *arr, int32_t *out, cudaStream_t s);
// dst[u + dst_off[gid[u]]] = src[u] for u < n
lv_status scatter_blocks(int32_t n, const int32_t *gid, const int32_t *dst_off, const int32_t *src,
                         int32_t *dst, cudaStream_t s);

// The fixed part of a batched iteration (clearing the counters and the
// persistent sweep launch) as an instantiated CUDA graph: captured at the
// first sweep of a phase and again when the vertex list moves to the
// compacted buffer, replayed by every other iteration.  If the capture is
// refused the iterations are issued directly.
struct SweepGraph {
    cudaGraphExec_t exec = nullptr;
    const int32_t *order = nullptr, *bo = nullptr;
    bool disabled = false;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        order = bo = nullptr;
    }
    ~SweepGraph() { reset(); }
};

struct Engine {
    cudaStream_t s = nullptr;
    lv_params P;
    BinLimits lim;
    int *pinned = nullptr;   // 64 pinned ints, owned by the caller
    Timer *timer = nullptr;  // optional
    std::vector<BinLimits> *tuned = nullptr;  // autotune cache by phase round (optional)
    std::vector<char> *tuned_ok = nullptr;

    // the union of resident graphs (device, owned)
    DGraph g;
    int32_t *k = nullptr, *loop = nullptr, *gid = nullptr;
    int32_t *gptr_d = nullptr;       // G+1
    long long *two_m_d = nullptr;    // G
    std::vector<int32_t> gp;         // host copy of the vertex starts
    // the union of their original vertices (device, owned)
    int64_t n_orig = 0;
    int32_t *map = nullptr, *gid_orig = nullptr;
    std::vector<int32_t> optr;       // host, original-vertex starts (G+1)
    std::vector<EngineGraph> graphs; // by position
    int32_t round = 0;               // phases run by this engine

    // statistics
    std::vector<lv_batch_sweep> sweeps;
    std::vector<int> ev_sweep;       // timer event pairs per sweep
    std::vector<int> ev_iter, ev_reb;
    int64_t sweep_launches = 0, graph_launches = 0;

    int32_t num_graphs() const { return (int32_t)graphs.size(); }
    // Vertex following (when on) and append to the union (between phases).
    lv_status append(const NewGraphs &ng);
    // Append sets of graphs prepared by prepare_graphs (between phases; one
    // copy of the union for all of them).
    lv_status append_prepared(const std::vector<const Prepared *> &prs);
    // One phase for every resident graph, up to and including the labels:
    // afterwards `labels` (device, n_orig entries in the current
    // original-vertex order: graph at position g owns [optr[g], optr[g+1]))
    // holds every graph's labels after the phase, numbered per graph; each
    // record has the phase appended and `stop` set when its phase loop ends.
    lv_status phase_run();
    int32_t *labels = nullptr;
    // Coarse graphs of the graphs that go on become the new union; the
    // others leave the engine and are returned (their labels at lab_off of
    // `labels`, which stays valid until the next phase_run or release).
    lv_status phase_end(std::vector<Finished> &finished);
    void release();
    ~Engine() { release(); }

  private:
    // pinned host scratch for the per-iteration readback, sized for `pin_cap` graphs
    void *pin_block = nullptr;
    size_t pin_cap = 0;
    unsigned long long *pin_u64 = nullptr;  // 3 per graph
    IterStats *pin_stats = nullptr;
    uint8_t *pin_flags = nullptr;           // 1 per graph
    lv_status ensure_pinned(size_t graphs);
    SweepGraph sg;
    // between phase_run and phase_end
    PhaseState ps;
    int32_t *newid = nullptr;
    std::vector<int32_t> gstart;  // host: starts of the graphs in the coarse numbering
    int32_t n_next = 0;
    void free_phase();
    // the union from blocks of several sources: graphs `keep` of (src,
    // map_src, starts src_gp), then every graph of each prepared set
    lv_status assemble(const DGraph &src, const int32_t *map_src, const std::vector<int32_t> &src_gp,
                       const std::vector<int> &keep, const std::vector<const Prepared *> &news);
};

}  // namespace lv
