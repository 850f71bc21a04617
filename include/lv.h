/*
 * lv.h -- C ABI of the GB300 parallel-Louvain library (liblv.so).
 *
 * The library runs the parallel Louvain community-detection method of Lu,
 * Halappanavar and Kalyanaraman, "Parallel Heuristics for Scalable Community
 * Detection" (arXiv 1410.1237), on one CUDA GPU: vertex following (Sec. 4.3),
 * distance-1 colouring (Sec. 4.2), phases of parallel sweeps with the
 * minimum-label heuristics (Algorithm 1, Sec. 4.1), the modularity of Eq. 3,
 * and the coarse-graph rebuild between phases (Sec. 4.4 step 4, Sec. 4.5).
 *
 * Arithmetic is exact: weights are integers, gains are compared as
 * 2m*e_{i->C} - k_i*a_C in 64-bit integers (Eq. 4 scaled by (2m)^2/2) and
 * modularity is carried as the integer numerator N = (2m)^2 Q; the only
 * floating-point operations are the threshold tests and the final Q = N /
 * (2m)^2.  Results are deterministic: the same input and parameters give
 * the same labels on every run and launch configuration.
 *
 * Conventions for every entry point:
 *   - Every function returns lv_status; nothing throws across the ABI.
 *   - Pointers flagged "on device" are CUDA device pointers; otherwise host.
 *   - The caller keeps ownership of every buffer it passes.  Input arrays
 *     are copied during lv_graph_create and may be freed when it returns.
 *     Output arrays are caller-allocated.
 *   - Calls on one handle must not run concurrently; distinct handles are
 *     independent.  All GPU work of a handle is ordered on the stream given
 *     at creation, and each entry point returns after that work completes.
 *   - On LV_ERR_CUDA the handle's state is undefined; destroy it.
 */
#ifndef LV_H_
#define LV_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lv_graph lv_graph; /* opaque, owned by the library */

typedef enum {
    LV_OK = 0,
    LV_ERR_ARG = -1,           /* bad argument, rowptr not non-decreasing from 0,
                                  column out of range or columns not ascending */
    LV_ERR_NOT_SYMMETRIC = -2, /* (i,j,w) stored without (j,i,w) */
    LV_ERR_WEIGHT = -3,        /* a weight < 1 (Sec. 2: weights are positive) */
    LV_ERR_DUPLICATE = -4,     /* a column repeated in a row (Sec. 2: no multi-edges) */
    LV_ERR_OVERFLOW = -5,      /* 2m >= 2^31, or more than 2^31-1 stored arcs */
    LV_ERR_EMPTY = -6,         /* m == 0 */
    LV_ERR_CUDA = -7,          /* a CUDA call failed; see lv_last_error() */
    LV_ERR_OOM = -8,           /* device allocation failed */
    LV_ERR_TIMEOUT = -9,       /* a bounded device wait gave up */
    LV_ERR_STATE = -10,        /* no run yet, or phase index out of range */
    LV_ERR_HASH = -11          /* a hash table probe exceeded its bound (internal) */
} lv_status;

/* Heuristic switches and threshold schedule of Sec. 5.1 (variant
 * "baseline+VF+Color"), plus guards the paper leaves implicit. */
typedef struct {
    int32_t vertex_following; /* 0/1: merge single-degree vertices once, before phase 0 (Sec. 4.3) */
    int32_t coloring;         /* 0/1: sweep one distance-1 colour class at a time (Sec. 4.2) */
    double theta_low;         /* threshold of uncoloured phases, 1e-6 in Sec. 5.1 */
    double theta_high;        /* threshold of coloured phases, 1e-2 in Sec. 5.1; 0 = use theta_low */
    int64_t color_cutoff;     /* colour only phases whose graph has >= this many vertices (100,000) */
    int32_t max_iters;        /* guard: iterations per phase (default 10,000) */
    int32_t max_phases;       /* guard: phases (default 64) */
    uint64_t color_seed;      /* seed of the colouring priority hash; phase p uses seed + p */
    int32_t collect_timing;   /* 0/1: record CUDA-event times per stage and per iteration */
    int32_t keep_graphs;      /* 0/1: keep every phase graph and colouring for inspection */
    /* Degree bins of the sweep (0 = default); results do not depend on them.
     * A vertex of degree d <= bin_warp_max is swept by the smallest group of
     * G = 1, 2, ..., 32 lanes with d <= G * bin_lane_arcs (else 32 lanes);
     * d <= bin_cta_max by a quarter CTA (4 warps) up to 1,024 arcs, else by
     * one CTA; larger (hubs) by several CTAs. */
    int32_t bin_lane_arcs;    /* 1..8, default 8 */
    int32_t bin_warp_max;     /* 1..256, default 256 */
    int32_t bin_cta_max;      /* bin_warp_max+1 .. 4096, default 4096 */
    /* 0/1: choose the bins of each uncoloured phase with >= 2^22 arcs by
     * timing one sweep per candidate set (the sweep of an uncoloured phase
     * changes no community state, so results do not change).  The choice is
     * kept per phase index in the handle and reused by later runs; the bin_*
     * fields then only seed the first candidate. */
    int32_t autotune;
    /* 0/1: batched runs replay each phase's sweep launch (with the clearing
     * of its counters) from a captured CUDA graph; default 1.  Ignored on the
     * legacy default stream (NULL), which cannot be captured. */
    int32_t graph_capture;
    /* Variants of the Sec. 5 experiments: colour at most this many phases
     * (0 = no limit, 1 = the first phase only), and */
    int32_t color_phases;
    /* 0/1: every threshold test uses |N_C - N_P| < theta |N_P|, the form
     * printed in Alg. 1, instead of the signed net gain (default 0; the
     * absolute form can cycle between two labellings until max_iters). */
    int32_t abs_threshold;
    /* 0/1: after vertex following, merge single-neighbour vertices (one
     * neighbour j plus an optional self-loop l) into their neighbour, round
     * after round, while Lemma 3's bound (Eq. eqnClaimIItemp, taken at the
     * largest community degree C(j) can have) guarantees the move: k_i^2 >
     * 2m l_i with k_i = w(i,j) + l_i.  The extension sketched at the end of
     * Sec. 4.3 (default 0; single-graph runs and the server's second lane;
     * lv_batch_run returns LV_ERR_ARG). */
    int32_t vf_recursive;
    /* Colouring priority (Sec. 4.2 leaves the colouring order to the
     * implementation): 0 = largest number of neighbours first, ties by the
     * seeded hash, then by id (default: fewer colour classes, so fewer
     * class steps per iteration); 1 = the seeded hash alone, then id. */
    int32_t color_order;
    /* Sweep launch shape (0 = default; results never depend on them; the
     * autotuner may choose others for uncoloured phases): persistent sweep
     * blocks per SM, 1 or 2 (default: as many as fit, 2), and hub hash-table
     * slots per arc, 2, 4 or 8 (default 4 in coloured phases, 2 otherwise). */
    int32_t sweep_blocks_per_sm;
    int32_t hub_slots_per_arc;
    /* Most SMs the persistent kernels (sweep, colouring) of a single-graph
     * run use: 0 = all.  A phase graph of A arcs uses about A / 65,536 SMs
     * (at least 16) within that bound: fewer blocks make cheaper grid
     * barriers on small graphs, and solves of small graphs on different
     * streams run side by side (the server's single-graph lane uses it). */
    int32_t persistent_sms;
} lv_params;

/* Per-phase record.  N values are exact modularity numerators: Q = N/(2m)^2. */
typedef struct {
    int64_t n;          /* vertices of the phase graph G_p */
    int64_t arcs;       /* stored arcs of G_p (each edge twice, each self-loop once) */
    int64_t n_next;     /* non-empty communities = vertices of G_{p+1} */
    int64_t two_m;      /* 2m (the same for every phase) */
    int64_t N_start;    /* numerator of the singleton partition of G_p */
    int64_t N_end;      /* numerator after the phase's last iteration */
    double q;           /* N_end / (2m)^2 */
    double theta;       /* threshold used by the phase */
    int32_t colored;    /* 1 if the phase swept colour classes */
    int32_t num_colors; /* colour classes (0 if not coloured) */
    int32_t iterations; /* iterations of Alg. 1's while-loop */
    int32_t color_rounds; /* Jones-Plassmann rounds after the degree core (coloured first,
                             without rounds); 0 if not coloured */
    double ms_color;    /* CUDA-event times (collect_timing), else -1 */
    double ms_iterate;
    double ms_rebuild;
} lv_phase_info;

/* Per-iteration record. */
typedef struct {
    int32_t phase;
    int32_t iter;        /* 1-based iteration within the phase */
    int32_t color_steps; /* colour classes swept (1 when uncoloured) */
    int32_t reserved;
    int64_t moved;       /* vertices that changed community */
    int64_t N;           /* modularity numerator after the iteration */
    int64_t arcs;        /* arcs scanned by the iteration's sweep */
    double ms;           /* CUDA-event time of the iteration (collect_timing), else -1 */
} lv_iter_stat;

/* Whole-run totals. */
typedef struct {
    int32_t num_phases;
    int32_t total_iterations;
    int64_t edge_visits;   /* sum over iterations of the arcs scanned */
    int64_t vf_n;          /* vertices after vertex following (n if off) */
    int64_t sweep_launches;
    double ms_total;       /* CUDA-event times (collect_timing), else -1 */
    double ms_vf;
    double ms_color;
    double ms_iterate;
    double ms_rebuild;
    int64_t kernel_launches; /* CUDA kernels this run launched (a graph replay counts 1) */
    int64_t graph_launches;  /* CUDA graph replays among them */
} lv_stats;

/* Fill *p with the defaults of Sec. 5.1: VF on, colouring on, theta_low 1e-6,
 * theta_high 1e-2, cutoff 100,000 vertices, max_iters 10,000, max_phases 64;
 * default bins, no autotuning, graph capture on. */
void lv_params_default(lv_params *p);

/* Create a handle from a symmetric CSR with integer weights (Sec. 2: an
 * undirected graph, positive weights, self-loops allowed, no multi-edges).
 *   n        vertices, 0 <= n < 2^31 - 1
 *   rowptr   int64[n+1], rowptr[0] = 0, non-decreasing
 *   col      int32[rowptr[n]], ascending within each row, each in [0, n)
 *   w        int32[rowptr[n]], each >= 1; (i,j,w) stored iff (j,i,w) stored;
 *            a self-loop (i,i,w) is stored once in row i and counts once in k_i
 *   ptrs_on_device  0: the three arrays are host memory; 1: device memory
 *   cuda_stream     cudaStream_t (NULL = legacy default stream) for all work
 * Requires 2m = sum of all stored weights < 2^31.  The input is validated on
 * the device; when it breaks several rules the first of ARG, DUPLICATE,
 * WEIGHT, NOT_SYMMETRIC, OVERFLOW, EMPTY is returned and *out is NULL. */
lv_status lv_graph_create(lv_graph **out, int64_t n, const int64_t *rowptr, const int32_t *col,
                          const int32_t *w, int ptrs_on_device, void *cuda_stream);

/* Run the whole method (Sec. 4.4 steps 1-4) with parameters *p (NULL =
 * defaults).  Replaces the results of any earlier run on the handle.  Phase
 * control: phase p is coloured when coloring && n_p >= color_cutoff and no
 * earlier coloured phase gained less than theta_high; the iteration loop of a
 * phase stops when nothing moved, when (N_C - N_P) < theta |N_P| after the
 * second iteration, or at max_iters; phases stop when nothing merged, when an
 * uncoloured phase gained less than theta_low relative to its singleton start,
 * or at max_phases. */
lv_status lv_run(lv_graph *g, const lv_params *p);

/* Number of recorded phases of the last run. */
lv_status lv_num_phases(const lv_graph *g, int32_t *out);

/* Community of every ORIGINAL vertex after phase `phase` (-1 = last phase):
 * int32[n] written to `out` (host, or device when ptr_on_device = 1).
 * Communities are numbered 0..n_next-1 in ascending order of their label in
 * the phase graph. */
lv_status lv_get_labels(const lv_graph *g, int32_t phase, int32_t *out, int ptr_on_device);

/* Modularity after phase `phase` (-1 = last): q = N/(2m)^2 (Eq. 3), and the
 * exact numerator as a 128-bit two's-complement value (num_hi:num_lo) with
 * den = (2m)^2.  Any output pointer may be NULL. */
lv_status lv_get_modularity(const lv_graph *g, int32_t phase, double *q, int64_t *num_hi,
                            uint64_t *num_lo, int64_t *den);

/* Per-phase record (phase -1 = last). */
lv_status lv_get_phase_info(const lv_graph *g, int32_t phase, lv_phase_info *out);

/* Per-iteration records of the last run: count, then copy up to `count`. */
lv_status lv_get_num_iterations(const lv_graph *g, int64_t *count);
lv_status lv_get_iteration_stats(const lv_graph *g, lv_iter_stat *out, int64_t count);

/* Whole-run totals of the last run. */
lv_status lv_get_stats(const lv_graph *g, lv_stats *out);

/* The sweep configuration the autotuner chose for phase `phase` (runs with
 * autotune = 1; kept in the handle across runs): out = int32[5] host array
 * {lane_arcs, warp_max, cta_max, sweep blocks per SM (0 = as many as fit),
 * hub table slots per arc (0 = the default: 4 coloured, 2 otherwise)}.
 * LV_ERR_STATE when that phase was not tuned (coloured, or < 2^22 arcs). */
lv_status lv_get_tuning(const lv_graph *g, int32_t phase, int32_t *out);

/* Map of vertex following: int32[n] giving each original vertex's vertex in
 * the phase-0 graph (identity when vertex following is off). */
lv_status lv_get_vf_map(const lv_graph *g, int32_t *out, int ptr_on_device);

/* Phase graph G_p of the last run (requires keep_graphs = 1): first call
 * with NULL arrays to read n and arcs, then with int64[n+1], int32[arcs] x 2. */
lv_status lv_get_phase_graph(const lv_graph *g, int32_t phase, int64_t *n, int64_t *arcs,
                             int64_t *rowptr, int32_t *col, int32_t *w, int ptrs_on_device);

/* Colour of each vertex of G_p (requires keep_graphs = 1 and a coloured
 * phase): int32[n_p]. */
lv_status lv_get_phase_colors(const lv_graph *g, int32_t phase, int32_t *out, int ptr_on_device);

/* Qualitative comparison of two partitions of the same n vertices (Sec. 5):
 * over all unordered vertex pairs, TP = same community in both, FP = same
 * only in p, FN = same only in s, TN = different in both; SP = TP/(TP+FP),
 * SE = TP/(TP+FN), OQ = TP/(TP+FP+FN), Rand = (TP+TN)/(n(n-1)/2) (a ratio
 * whose denominator is 0 is 1).  Computed from the contingency table of the
 * two labellings (sort by label pairs), not pair by pair. */
typedef struct {
    uint64_t tp, fp, fn, tn;
    double sp, se, oq, rand;
} lv_partition_compare;

/*   n            vertices, 0 <= n < 2^31
 *   labels_s/p   int32[n], any values (equal values = same community)
 *   ptrs_on_device  0: host arrays, 1: device arrays
 *   cuda_stream  the stream for the work; the call returns after it */
lv_status lv_compare_partitions(int64_t n, const int32_t *labels_s, const int32_t *labels_p,
                                int ptrs_on_device, lv_partition_compare *out, void *cuda_stream);

/* Modularity numerator of a caller-given labelling, computed without any
 * device allocation.  (This entry point has no counterpart in the paper; it
 * serves callers that cannot allocate device memory where they need it:
 * services that reserve all device memory in a fixed pool at start-up and
 * forbid further cudaMalloc calls, hosts with a strict pre-computed memory
 * budget.)
 *   n, rowptr, col, w  a CSR meeting the lv_graph_create contract, all four
 *                      arrays in DEVICE memory; 1 <= n <= 1,048,576
 *   labels             int32[n] on the device, each in [0, n)
 *   num_hi:num_lo      out (host): N as a 128-bit two's-complement value
 *   den                out (host): (2m)^2, so that Q = N / den (Eq. 3)
 *   cuda_stream        cudaStream_t for the work; the call waits for this
 *                      stream (cudaStreamSynchronize) before it returns
 * Scratch is a fixed 8 MB array of device memory that exists once the library
 * is loaded (on every device the process uses, until exit).  The first call
 * on a device looks up that array's address (once per device, thread-safe);
 * make that first call before any stream capture.  The address is not looked
 * up again, so it does not survive cudaDeviceReset.  All calls share the
 * array and each one clears what it uses first, so calls whose GPU work
 * overlaps race: serialise them.
 * Returns LV_ERR_ARG for n outside [1, 2^20], a label or column out of
 * range, or a NULL pointer (checked before any GPU work);
 * LV_ERR_EMPTY / LV_ERR_OVERFLOW as lv_graph_create. */
lv_status lv_modularity_noalloc(int64_t n, const int64_t *rowptr, const int32_t *col,
                                const int32_t *w, const int32_t *labels, int64_t *num_hi,
                                uint64_t *num_lo, int64_t *den, void *cuda_stream);

/* Check of the bounded device waits (every grid barrier and wait of the
 * persistent kernels gives up after a bounded number of polls, raises an
 * error flag and returns, so a fault cannot hang the GPU): launches four
 * blocks on the current device whose block 0 never arrives at their grid
 * barrier; the other three give up after `polls` polls of the barrier word
 * and raise the wait flag.  Returns LV_ERR_TIMEOUT when they did (the
 * expected result; the device stays usable), LV_ERR_STATE if the barrier
 * completed anyway, LV_ERR_ARG for polls outside [1, 2^24], LV_ERR_CUDA on
 * a CUDA error.  Synchronises the current device's default stream. */
lv_status lv_check_bounded_wait(int32_t polls);

/* Static description of a status code. */
const char *lv_status_string(lv_status s);

/* Text of the last CUDA error seen by this thread (empty if none). */
const char *lv_last_error(void);

/* Release the handle and all its device memory (NULL is a no-op). */
void lv_graph_destroy(lv_graph *g);

/* ---------------------------------------------------------------- batches
 * A batch holds many independent graphs and runs the method on all of them
 * at once: each sweep is one persistent launch over the vertices of every
 * graph still iterating, and each rebuild one pass over all graphs.  Every
 * graph follows exactly the phase and iteration control of lv_run (its own
 * 2m, thresholds and stopping tests), so its labels, numerators and
 * iteration counts are those lv_run gives for it alone.  Graphs that finish
 * early are skipped by later sweeps.  Colouring is not batched: lv_batch_run
 * returns LV_ERR_ARG when colouring is on and a graph has at least
 * color_cutoff vertices after vertex following (run such graphs alone). */
typedef struct lv_batch lv_batch; /* opaque, owned by the library */

/* Per-graph record of a batched run. */
typedef struct {
    int64_t n;          /* vertices of the graph */
    int64_t arcs;       /* stored arcs */
    int64_t two_m;      /* 2m of the graph */
    int64_t n_final;    /* communities after its last phase */
    int64_t N_final;    /* modularity numerator after its last phase */
    double q;           /* N_final / (2m)^2 */
    int32_t num_phases; /* phases it ran */
    int32_t iterations; /* iterations over all its phases */
} lv_batch_graph_info;

/* Record of one batched sweep (one persistent launch over the graphs still
 * iterating in the phase). */
typedef struct {
    int32_t phase;
    int32_t sweep;      /* 1-based within the phase */
    int32_t graphs;     /* graphs swept */
    int32_t reserved;
    int64_t vertices;   /* vertices of the swept graphs */
    int64_t arcs;       /* arcs of the swept graphs */
    int64_t moved;      /* moves proposed */
    double ms;          /* CUDA-event time of the sweep (collect_timing), else -1 */
} lv_batch_sweep;

/* Create a batch: the disjoint union of n_graphs graphs as ONE CSR whose
 * vertices are numbered graph after graph.
 *   n_graphs  >= 1
 *   gptr      int64[n_graphs+1]: graph g owns vertices [gptr[g], gptr[g+1]);
 *             gptr[0] = 0, strictly increasing (every graph has a vertex),
 *             gptr[n_graphs] = n < 2^31 - 1
 *   rowptr, col, w  the union CSR under the lv_graph_create contract, with
 *             union vertex ids; every arc must stay inside its graph
 *   ptrs_on_device  applies to gptr, rowptr, col and w alike
 * Each graph needs 2m_g < 2^31 (LV_ERR_OVERFLOW) and m_g > 0 (LV_ERR_EMPTY);
 * the union needs fewer than 2^31 stored arcs.  An arc between two graphs
 * or a malformed gptr gives LV_ERR_ARG.  Other errors as lv_graph_create. */
lv_status lv_batch_create(lv_batch **out, int32_t n_graphs, const int64_t *gptr,
                          const int64_t *rowptr, const int32_t *col, const int32_t *w,
                          int ptrs_on_device, void *cuda_stream);

/* Run every graph of the batch with parameters *p (NULL = defaults); the
 * bin limits apply to all graphs.  Replaces the results of an earlier run. */
lv_status lv_batch_run(lv_batch *b, const lv_params *p);

/* Number of graphs in the batch. */
lv_status lv_batch_num_graphs(const lv_batch *b, int32_t *out);

/* Labels after phase `phase` of the last run, numbered per graph from 0 as
 * lv_get_labels numbers them for the graph alone.
 *   graph >= 0: int32[n_g] of that graph; phase -1 = its last phase, else a
 *               phase it ran (LV_ERR_STATE otherwise)
 *   graph = -1: int32[n] of all graphs in union order; phase -1 = each
 *               graph's last phase, else phase p of the graphs that ran it
 *               and the final labels of those that had stopped before p
 *               (p < the largest phase count)
 * `out` is host memory, or device memory when ptr_on_device = 1. */
lv_status lv_batch_get_labels(const lv_batch *b, int32_t graph, int32_t phase, int32_t *out,
                              int ptr_on_device);

/* Per-graph summary, and per-graph phase record (phase -1 = its last). */
lv_status lv_batch_get_graph_info(const lv_batch *b, int32_t graph, lv_batch_graph_info *out);
lv_status lv_batch_get_phase_info(const lv_batch *b, int32_t graph, int32_t phase,
                                  lv_phase_info *out);

/* Whole-batch totals: num_phases = largest phase count; total_iterations
 * and edge_visits = the sums over graphs of what lv_run reports for each;
 * vf_n = vertices of the union after vertex following; sweep_launches =
 * batched sweeps; times (collect_timing) and kernel launches of the run. */
lv_status lv_batch_get_stats(const lv_batch *b, lv_stats *out);

/* The sweep configuration the autotuner chose for batched phase round
 * `round` (autotune = 1; as lv_get_tuning).  LV_ERR_STATE when that round
 * was not tuned. */
lv_status lv_batch_get_tuning(const lv_batch *b, int32_t round, int32_t *out);

/* Batched sweep records of the last run: count, then copy up to `count`. */
lv_status lv_batch_get_num_sweeps(const lv_batch *b, int64_t *count);
lv_status lv_batch_get_sweeps(const lv_batch *b, lv_batch_sweep *out, int64_t count);

/* Release the batch and its device memory (NULL is a no-op). */
void lv_batch_destroy(lv_batch *b);

/* ---------------------------------------------------------------- serving
 * A server runs community detection for a stream of requests on one GPU
 * with continuous batching.  An admission thread takes queued requests
 * (first come, first served) while the estimated device footprint of the
 * requests in flight stays within the memory budget and the slot limit, and
 * uploads, validates and vertex-follows them on its own stream; a worker
 * thread joins them to its running multi-graph engine at its next phase
 * boundary, runs one batched phase of every resident request (their sweeps
 * share launches), and completes the requests whose phase loop stopped.
 * That is lane 0, for requests with fewer than 2^22 stored arcs that would
 * not colour any phase.  Lane 1 (its own worker and stream) solves the other
 * requests (large ones, and those with colouring on and at least
 * color_cutoff vertices) one at a time with the single-graph driver, so small
 * requests never wait for the iterations of large ones.   A
 * request's CSR and labels stay on the device across its phases.  Each
 * request gets exactly what lv_run gives for it alone with the same
 * parameters, whatever else is resident. */
typedef struct lv_server lv_server; /* opaque, owned by the library */

typedef struct {
    int64_t mem_budget_bytes; /* resident requests' estimated device bytes (48 per
                                 stored arc + 64 per vertex); 0 = 120 GB.  A request
                                 larger than the budget is admitted alone. */
    int32_t max_graphs;       /* resident requests at most; 0 = 65,536 */
    int32_t reserved;
    lv_params params;         /* for every request (all heuristics allowed) */
} lv_server_config;

/* Outcome of one request (times in ms since lv_server_create, host clock). */
typedef struct {
    int32_t status;      /* LV_OK, or the validation error of its CSR */
    int32_t num_phases;
    int32_t iterations;  /* over all its phases */
    int32_t reserved;
    int64_t n, arcs, two_m, n_final;
    int64_t N_final;     /* modularity numerator after its last phase */
    double q;            /* N_final / (2m)^2 */
    double t_submit_ms, t_admit_ms, t_done_ms;
} lv_server_result_info;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    int64_t rounds;       /* batched phases run */
    int64_t sweeps;       /* batched sweeps */
    int64_t peak_graphs;  /* most requests resident at once */
    int64_t peak_bytes;   /* largest estimated resident footprint */
    int64_t kernel_launches; /* CUDA kernels the worker launched (a graph replay counts 1) */
    double ms_admit;      /* admission thread: uploading, validating and vertex following */
    double ms_append;     /* worker thread: joining prepared requests to the engine */
    double ms_iterate;    /* ... batched iterations up to the labels */
    double ms_rebuild;    /* ... coarse graphs and departures */
    double ms_results;    /* ... copying finished requests' labels to the host */
} lv_server_stats;

/* Start a server on the current device.  cuda_stream: the stream of lane 0
 * (NULL = a stream the server creates; lane 1 and admission always use their
 * own).  LV_ERR_ARG for a NULL config or invalid parameters. */
lv_status lv_server_create(lv_server **out, const lv_server_config *cfg, void *cuda_stream);

/* Queue a request: a CSR under the lv_graph_create contract in HOST memory,
 * copied before the call returns.  *request_id receives its id (>= 0).  The
 * CSR is validated on admission; an invalid one completes with its error. */
lv_status lv_server_submit(lv_server *srv, int64_t n, const int64_t *rowptr, const int32_t *col,
                           const int32_t *w, int64_t *request_id);

/* Wait up to timeout_s seconds (< 0: forever) for a request; *done = 1 when
 * it completed.  LV_ERR_ARG for an unknown id. */
lv_status lv_server_wait(lv_server *srv, int64_t request_id, double timeout_s, int32_t *done);

/* Result of a completed request: labels int32[n] in host memory (may be
 * NULL), numbered per graph as lv_get_labels numbers the final phase, and
 * its record.  LV_ERR_STATE while it is not done; the request's own error
 * status when its CSR was invalid. */
lv_status lv_server_result(lv_server *srv, int64_t request_id, int32_t *labels,
                           lv_server_result_info *info);

/* Forget a completed request (frees its stored labels). */
lv_status lv_server_release(lv_server *srv, int64_t request_id);

lv_status lv_server_get_stats(lv_server *srv, lv_server_stats *out);

/* Stop the worker after its current phase and free everything; requests not
 * completed are dropped (NULL is a no-op). */
void lv_server_destroy(lv_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* LV_H_ */
