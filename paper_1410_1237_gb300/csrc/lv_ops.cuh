// lv_ops.cuh -- host-side entry points of the kernel translation units.
#pragma once

#include <vector>

#include "lv_internal.cuh"

namespace lv {

// lv_graph.cu ------------------------------------------------------------
lv_status severity_to_status(int sev);
// Validate a device-resident CSR (Sec. 2 contract) and build the internal
// graph plus k (weighted degree) and loop (self-loop weight).  limit_two_m =
// false skips the 2m < 2^31 test (a batch checks each of its graphs instead).
lv_status validate_and_build(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const int32_t *w, DGraph *out, int32_t **k, int32_t **loop,
                             int64_t *two_m, int *scratch_pinned, cudaStream_t s,
                             bool limit_two_m = true);
lv_status compute_degrees(const DGraph &g, int32_t *k, int32_t *loop, cudaStream_t s);
lv_status iota(int32_t n, int32_t *out, cudaStream_t s);
// Vertex following (Sec. 4.3); allocates *out; map[v] = vertex of v in *out.
lv_status vertex_following(const DGraph &g, const int32_t *loop, DGraph *out, int32_t *map,
                           int *scratch_pinned, cudaStream_t s);
void free_graph(DGraph &g, cudaStream_t s);
// Recursive single-neighbour merge after vertex following (R23, the closing
// paragraph of Sec. 4.3): rounds that merge every single-neighbour vertex
// passing Lemma 3's bound (k_i^2 > 2m l_i) into its neighbour, until none
// passes.  Replaces *G (owned) by the merged graph and composes map
// (n_orig entries); *rounds = merging rounds.
lv_status vf_recursive(DGraph *G, int64_t two_m, int32_t *map, int32_t n_orig, int *pinned,
                       int32_t *rounds, cudaStream_t s);

// lv_color.cu ------------------------------------------------------------
// Jones-Plassmann distance-1 colouring with priority (d(v), h(v ^ seed), v),
// d(v) = neighbours other than v (degree_first), else (h(v ^ seed), v).
lv_status jp_color(const DGraph &g, uint64_t seed, bool degree_first, int32_t *color,
                   int32_t *num_colors, int32_t *rounds, int *scratch_pinned, cudaStream_t s,
                   int sms = 0);

// Vertex order of a phase: vertices grouped by (colour class, degree bin),
// ascending id inside a group.  order[n], bucket_off[(classes*(kBins+1))+1]
// (device) and the same offsets on the host.
struct Buckets {
    int32_t classes = 1;
    int32_t *order = nullptr;        // device, n
    int32_t *bucket_off = nullptr;   // device
    int32_t *hub_off = nullptr;      // device, n+1: hub hash-table offset per position
    int64_t hub_slots = 0;           // total hub table slots
    int2 *hub_table = nullptr;       // device, {label, weight}, kept empty between uses
    int32_t *hub_occ = nullptr;      // device, occupied-slot list per hub (same offsets)
    int32_t *hub_cnt = nullptr;      // device, n: occupied count per position
    int32_t *hub_chunk_off = nullptr;  // device, n+1: first arc chunk of each position
    int32_t *hub_chunk_at = nullptr;   // device: hub_chunk_off at every bucket boundary
    // device, per class: log2 of the class's hub arc chunk in units of
    // kHubChunk (null: every class uses kHubChunk)
    uint8_t *hub_shift = nullptr;
    void *hub_part = nullptr;          // device: partial best per hub chunk
    int32_t *hub_done = nullptr;       // device, n: finished decide chunks per position
    int32_t *host_off = nullptr;     // host copy of bucket_off
    int32_t *host_chunk = nullptr;   // host: hub_chunk_off at every bucket boundary
    int hub_factor = 2;              // hub table slots per arc (next power of two)
    int blocks_per_sm = 0;           // sweep blocks per SM (0 = as many as fit)
    int sms = 0;                     // SMs of the sweep's grid (0 = all)
};
#ifndef LV_HUB_CHUNK
#define LV_HUB_CHUNK 1024
#endif
constexpr int kHubChunk = LV_HUB_CHUNK;  // arcs (and occupied slots) per block item of a hub
// a colour class whose hubs have more than this many kHubChunk chunks per
// block of the sweep grid has its hubs cut into chunks of 2 kHubChunk
#ifndef LV_HUB_WIDE_AT
#define LV_HUB_WIDE_AT 1
#endif
// a hub's global table has the next power of two >= this many slots per arc:
// 4 in coloured sweeps (shorter probe chains on the latency-bound path), 2 in
// one-class sweeps (batches and serving, where memory is budgeted)
__host__ __device__ constexpr int hub_table_factor(bool coloured) { return coloured ? 4 : 2; }
struct BinLimits {
    // the best fixed set on the R-MAT, Chung-Lu and planted-batch workloads
    int lane_arcs = 8, warp_max = 256, cta_max = 4096;
    // hub table slots per arc (0 = hub_table_factor of the mode) and sweep
    // blocks per SM (0 = as many as fit); the autotuner may set both
    int hub_factor = 0, blocks_per_sm = 0;
    // SMs the persistent kernels run on (0 = all): concurrent solves of
    // small graphs can share the GPU
    int sms = 0;
};
// SMs of the persistent kernels for a phase graph of `arcs` arcs when the
// caller leaves it open: one per kAutoArcsPerSm arcs, at least kAutoMinSms
// (all SMs from 152 * kAutoArcsPerSm arcs on)
#ifndef LV_AUTO_ARCS_PER_SM
#define LV_AUTO_ARCS_PER_SM (1 << 16)
#endif
constexpr int64_t kAutoArcsPerSm = LV_AUTO_ARCS_PER_SM;
constexpr int kAutoMinSms = 16;
inline int auto_sms(int64_t arcs) {
    const int64_t want = (arcs + kAutoArcsPerSm - 1) / kAutoArcsPerSm;
    return (int)(want < kAutoMinSms ? kAutoMinSms : (want > (1 << 20) ? (1 << 20) : want));
}
// sweep blocks per SM 0..2 and hub table slots per arc 0 (the mode's default),
// 2, 4 or 8
inline bool valid_shape(const BinLimits &l) {
    return l.blocks_per_sm >= 0 && l.blocks_per_sm <= 2 && l.sms >= 0 &&
           (l.hub_factor == 0 || l.hub_factor == 2 || l.hub_factor == 4 || l.hub_factor == 8);
}
lv_status bucket_vertices(const DGraph &g, const int32_t *color, int32_t classes,
                          const BinLimits &lim, Buckets *b, int *scratch_pinned, cudaStream_t s);
void free_buckets(Buckets &b, cudaStream_t s);

// lv_sweep.cu ------------------------------------------------------------
struct IterStats {
    unsigned long long sum_ein;    // sum over swept vertices of e_{i->C(i)} incl. self-loop
    unsigned long long delta_ein;  // sum over movers of 2 (e_{i->new} - e_{i->old})
    unsigned long long sum_a2;     // sum over communities of a_C^2
    int moved;
    int err;                       // a hash probe bound was exceeded
    int max_occ;                   // largest distinct-label count of a hub this sweep
    int pad;
    GridBarrier bar;               // barrier of the persistent sweep (reset with the stats)
};
struct PhaseState {
    DGraph g;
    const int32_t *k = nullptr;
    const int32_t *loop = nullptr;
    int32_t *C = nullptr;
    unsigned long long *comm[2] = {nullptr, nullptr};  // {a_C, |C|}; two buffers when coloured
    int4 *moves[2] = {nullptr, nullptr};               // {i, old, new, k_i}
    int32_t *move_count = nullptr;  // per active class: moves, block / warp work counters; + carry
    int32_t *act = nullptr;         // device: active classes (those with arcs)
    int n_act = 0;
    bool coloured = false;
    long long g_total = 0;          // classes swept so far in the phase (buffer parity)
    IterStats *stats = nullptr;
    GridBarrier *bar = nullptr;   // &stats->bar
    long long two_m = 0;
    // batched runs over a disjoint union of graphs (all null otherwise): the
    // sweep skips graphs whose active flag is 0 and sums the modularity terms
    // and moves per graph instead of into stats
    const int32_t *gid = nullptr;          // graph of each vertex
    const long long *two_m_g = nullptr;    // 2m of each graph
    const uint8_t *active_g = nullptr;     // graphs still iterating in this phase
    unsigned long long *g_ein = nullptr;   // per graph: sum of e_{i->C(i)} incl. loops
    unsigned long long *g_a2 = nullptr;    // per graph: sum of a_C^2 after the sweep
    unsigned long long *g_moved = nullptr; // per graph: moves proposed
};
// C = identity, comm = (k, 1) (both buffers when coloured); stats->sum_ein =
// sum of loops, stats->sum_a2 = sum of k^2; move counters cleared
lv_status init_phase(PhaseState &ps, cudaStream_t s);
// One cooperative launch sweeping all active classes.  Coloured phases apply
// each class's moves before the next class (double-buffered community state);
// uncoloured phases leave the moves in ps.moves[0] / move_count[0].  Adds
// sum_ein, delta_ein, moved and the sum of a_C^2 (after the sweep) to stats.
lv_status sweep_iteration(PhaseState &ps, const Buckets &b, cudaStream_t s);
// uncoloured phases: apply the listed moves
lv_status apply_moves(PhaseState &ps, cudaStream_t s);
// the community-state buffer holding the current state
unsigned long long *current_comm(const PhaseState &ps);
size_t hub_part_bytes();
// blocks of the sweep's cooperative grid for buckets b (after sweep_setup)
int sweep_grid(const Buckets &b);

// lv_tune.cu -------------------------------------------------------------
// Time one sweep of the (uncoloured) phase state per candidate bin set and
// return the fastest in *best; `first` is tried first.  `zero` (may be null)
// is cleared before each sweep with the statistics.  Leaves ps's community
// state untouched; its move list and statistics hold the last candidate's.
lv_status tune_bins(PhaseState &ps, const BinLimits &first, void *zero, size_t zero_bytes,
                    BinLimits *best, int *pinned, cudaStream_t s);
constexpr int64_t kTuneMinArcs = int64_t(1) << 22;  // phases smaller than this keep their bins

// lv_rebuild.cu ----------------------------------------------------------
// newid[c] = rank of c among non-empty communities (n+1 entries, newid[n] = count)
lv_status renumber(int32_t n, const unsigned long long *comm, int32_t *newid, cudaStream_t s);
// map[v] = newid[C[map[v]]] for every original vertex; labels = copy of the new map
lv_status compose_labels(int32_t n_orig, int32_t *map, const int32_t *C, const int32_t *newid,
                         int32_t *labels, cudaStream_t s);
// Coarse graph of Sec. 4.5 (i)-(iii); allocates *out
lv_status coarsen(const DGraph &g, const int32_t *C, const int32_t *newid, int32_t n_next,
                  DGraph *out, int *scratch_pinned, cudaStream_t s);

}  // namespace lv

namespace lv {
lv_status sweep_setup();  // one-time kernel attributes (large dynamic shared memory)
// process-wide setup (memory pool, SM count, kernel attributes), run once
lv_status ensure_setup(cudaStream_t s);

// Signed relative stopping test of Sec. 4.1 on exact numerators:
// (N_C - N_P) < theta |N_P|, converted to double once; abs_mode takes
// |N_C - N_P| (the form printed in Alg. 1, a variant).
inline bool gain_below(int64_t Nc, int64_t Np, double theta, bool abs_mode = false) {
    int64_t d = Nc - Np;
    if (abs_mode && d < 0) d = -d;
    const int64_t b = Np < 0 ? -Np : Np;
    return (double)d < theta * (double)b;
}

// CUDA events on one stream, recorded on demand (timing switched on per run).
struct Timer {
    bool on = false;
    cudaStream_t s = nullptr;
    std::vector<cudaEvent_t> ev;
    int mark() {  // returns an index, or -1 when timing is off
        if (!on) return -1;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        cudaEventRecord(e, s);
        ev.push_back(e);
        return (int)ev.size() - 1;
    }
    double ms(int a, int b) const {
        if (a < 0 || b < 0) return -1.0;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) return -1.0;
        return (double)t;
    }
    void clear() {
        for (auto e : ev) cudaEventDestroy(e);
        ev.clear();
    }
};
}  // namespace lv
