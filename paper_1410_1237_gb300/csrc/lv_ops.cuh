// lv_ops.cuh -- host-side entry points of the kernel translation units.
#pragma once

#include "lv_internal.cuh"

namespace lv {

// lv_graph.cu ------------------------------------------------------------
lv_status severity_to_status(int sev);
// Validate a device-resident CSR (Sec. 2 contract) and build the internal
// graph plus k (weighted degree) and loop (self-loop weight).
lv_status validate_and_build(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const int32_t *w, DGraph *out, int32_t **k, int32_t **loop,
                             int64_t *two_m, int *scratch_pinned, cudaStream_t s);
lv_status compute_degrees(const DGraph &g, int32_t *k, int32_t *loop, cudaStream_t s);
lv_status iota(int32_t n, int32_t *out, cudaStream_t s);
// Vertex following (Sec. 4.3); allocates *out; map[v] = vertex of v in *out.
lv_status vertex_following(const DGraph &g, const int32_t *loop, DGraph *out, int32_t *map,
                           int *scratch_pinned, cudaStream_t s);
void free_graph(DGraph &g, cudaStream_t s);

// lv_color.cu ------------------------------------------------------------
// Jones-Plassmann distance-1 colouring with priority (h(v ^ seed), v).
lv_status jp_color(const DGraph &g, uint64_t seed, int32_t *color, int32_t *num_colors,
                   int *scratch_pinned, cudaStream_t s);

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
    int32_t *host_off = nullptr;     // host copy of bucket_off
    int32_t *host_chunk = nullptr;   // host: hub_chunk_off at every bucket boundary
};
constexpr int kHubChunk = 4096;      // arcs per block of the hub accumulate kernel
struct BinLimits {
    int small_max = 16, warp_max = 128, cta_max = 4096;
};
lv_status bucket_vertices(const DGraph &g, const int32_t *color, int32_t classes,
                          const BinLimits &lim, Buckets *b, int *scratch_pinned, cudaStream_t s);
void free_buckets(Buckets &b, cudaStream_t s);

// lv_sweep.cu ------------------------------------------------------------
struct IterStats {
    unsigned long long sum_ein;    // sum over swept vertices of e_{i->C(i)} incl. self-loop
    unsigned long long delta_ein;  // sum over movers of 2 (e_{i->new} - e_{i->old})
    unsigned long long sum_a2;     // sum over communities of a_C^2
    int moved;
    int err;
};
struct PhaseState {
    DGraph g;
    const int32_t *k = nullptr;
    const int32_t *loop = nullptr;
    int32_t *C = nullptr;
    unsigned long long *comm = nullptr;
    int2 *moves = nullptr;
    int32_t *move_count = nullptr;  // one slot per colour class
    IterStats *stats = nullptr;
    long long two_m = 0;
};
// C = identity, comm = (k, 1); stats->sum_ein = sum of loops, stats->sum_a2 = sum k^2
lv_status init_phase(PhaseState &ps, cudaStream_t s);
// sweep every bin of class `cls`; appends moves to ps.moves / move_count[cls]
lv_status sweep_class(PhaseState &ps, const Buckets &b, int cls, const BinLimits &lim,
                      int64_t *launches, cudaStream_t s);
lv_status apply_moves(PhaseState &ps, int cls, cudaStream_t s);
lv_status sum_a2(PhaseState &ps, cudaStream_t s);

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
}  // namespace lv
