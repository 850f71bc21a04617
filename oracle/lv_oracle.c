/*
 * lv_oracle.c -- plain serial CPU oracle of the parallel Louvain method of
 * Lu, Halappanavar, Kalyanaraman, "Parallel Heuristics for Scalable
 * Community Detection" (arXiv 1410.1237).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that
 * the CUDA library is compared against.  Only the test suite, the smoke
 * check and the bench's CPU-baseline leg may build, load or run it; the
 * product path never does.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * It is written to be checked by eye against the paper, not to be fast:
 *   - every quantity is recomputed from its definition where that is cheap
 *     enough (modularity is re-evaluated from scratch after every iteration,
 *     Eq. 3);
 *   - gains are evaluated in exact 128-bit integer arithmetic (Eq. 4 scaled
 *     by (2m)^2/2, so no rounding can decide a move);
 *   - the iteration is the synchronous form of Algorithm 1: every vertex of
 *     the current colour class decides from the state at the start of the
 *     class, then all decided moves are applied together.
 *
 * Readings of points the paper leaves open (each is also used by the CUDA
 * path, and listed with its justification in the design notes):
 *   R1  a self-loop is stored once in its row and counted once in k_i and in
 *       e_{i->C(i)}; a coarse self-loop is the sum over directed intra arcs.
 *   R2  vertex following adds 2*w(i,j) to the survivor's self-loop, which
 *       keeps m and Q exact.
 *   R3  when both ends of an edge have degree one, the smaller id merges
 *       into the larger.
 *   R4  staying has gain 0; self-loops are excluded from e_{i->C}.
 *   R5  a vertex moves only on a strictly positive best gain; ties between
 *       equal gains go to the smallest community label.
 *   R6  Jacobi within a colour class, classes in ascending colour order.
 *   R7  the singlet rule is judged on the class-start state and a blocked
 *       vertex stays.
 *   R9  the loop stops when the net gain is below the threshold relative
 *       to the previous value: (double)(N_C - N_P) < theta * (double)|N_P|
 *       on exact numerators (signed: a negative gain stops it).
 *   R11 colouring = greedy distance-1 colouring in decreasing priority
 *       (degree, hash, id) -- the fixed point of Jones-Plassmann with that
 *       priority; optionally (hash, id) alone.
 *   R12 colour phases use theta_high; once a coloured phase gains less than
 *       theta_high colouring stops for good; uncoloured phases use theta_low.
 *   R13 phases stop when nothing merged or an uncoloured phase gains less
 *       than theta_low relative to its singleton start (same signed test).
 *
 * Parity unpinned: the colouring priority (R11) and the guards
 * max_iters / max_phases are choices of these readings; no printed example
 * fixes them.  The threshold and phase-control semantics (R9, R12, R13) are
 * readings too; the tests check the recorded numerators of whole runs
 * against the rules as stated above, not against a printed value.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef __int128 i128;

/* status codes of the library boundary (same numeric values) */
enum {
    ORC_OK = 0,
    ORC_ERR_ARG = -1,
    ORC_ERR_NOT_SYMMETRIC = -2,
    ORC_ERR_WEIGHT = -3,
    ORC_ERR_DUPLICATE = -4,
    ORC_ERR_OVERFLOW = -5,
    ORC_ERR_EMPTY = -6,
    ORC_ERR_OOM = -8,
    ORC_ERR_STATE = -10
};

typedef struct {
    int32_t vertex_following; /* VF preprocessing, Sec. 4.3 */
    int32_t coloring;         /* distance-1 colouring, Sec. 4.2 */
    double theta_low;         /* final threshold, 1e-6 in Sec. 5.1 */
    double theta_high;        /* colour-phase threshold, 1e-2 in Sec. 5.1; 0 = none */
    int64_t color_cutoff;     /* colour only phases with at least this many vertices */
    int32_t max_iters;        /* guard on iterations per phase */
    int32_t max_phases;       /* guard on phases */
    uint64_t color_seed;      /* priority hash seed; phase p uses seed + p */
    int32_t trace;            /* keep phase graphs, colourings, per-iteration labels */
    int32_t color_phases;     /* colour at most this many phases (0 = no limit; 1 = only the
                                 first phase, the variant of the Sec. 5 experiments) */
    int32_t abs_threshold;    /* 1: every threshold test uses |N_C - N_P| (the form printed
                                 in Alg. 1) instead of the signed net gain of R9 */
    int32_t vf_recursive;     /* 1: after vertex following, merge single-neighbour vertices
                                 round by round while Lemma 3's bound guarantees the move
                                 (R23; the closing paragraph of Sec. 4.3) */
    int32_t color_order;      /* colouring priority (R11): 0 = largest degree first, hash
                                 tie-break; 1 = hash only */
} orc_params;

typedef struct {
    int64_t n, arcs;
    int64_t *rowptr;
    int32_t *col, *w;
} orc_graph;

typedef struct {
    int64_t n, arcs, n_next;
    int32_t colored, num_colors, iterations;
    double theta;
    i128 N_start, N_end;
    int64_t two_m;
    double seconds;      /* wall time of this phase's iteration loop */
    int32_t *labels;     /* n_orig: community of every original vertex after this phase */
    orc_graph *graph;    /* trace: the phase's input graph */
    int32_t *colors;     /* trace: colours (NULL when not coloured) */
    int32_t **iter_labels; /* trace: labels of G_p after each iteration */
} orc_phase;

typedef struct {
    int32_t phase, iter;
    int64_t moved;
    i128 N;
    double seconds;
} orc_iter;

typedef struct {
    int64_t n_orig;
    int64_t two_m;
    int32_t num_phases;
    orc_phase *ph;
    int32_t cap_ph;
    orc_iter *it;
    int64_t num_iters, cap_it;
    int32_t *vf_map;       /* n_orig -> vertex of G_0 */
    int64_t vf_n;          /* vertices after VF */
    double seconds_total;
} orc_result;

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* ------------------------------------------------------------ graphs */
static orc_graph *graph_alloc(int64_t n, int64_t arcs) {
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    if (!g) return NULL;
    g->n = n;
    g->arcs = arcs;
    g->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->col = (int32_t *)malloc((size_t)(arcs ? arcs : 1) * sizeof(int32_t));
    g->w = (int32_t *)malloc((size_t)(arcs ? arcs : 1) * sizeof(int32_t));
    if (!g->rowptr || !g->col || !g->w) {
        free(g->rowptr); free(g->col); free(g->w); free(g);
        return NULL;
    }
    return g;
}
static void graph_free(orc_graph *g) {
    if (!g) return;
    free(g->rowptr); free(g->col); free(g->w); free(g);
}
static orc_graph *graph_copy_in(int64_t n, const int64_t *rowptr, const int32_t *col,
                                const int32_t *w) {
    orc_graph *g = graph_alloc(n, rowptr[n]);
    if (!g) return NULL;
    memcpy(g->rowptr, rowptr, ((size_t)n + 1) * sizeof(int64_t));
    memcpy(g->col, col, (size_t)g->arcs * sizeof(int32_t));
    memcpy(g->w, w, (size_t)g->arcs * sizeof(int32_t));
    return g;
}

/* ------------------------------------------------------- validation */
/* Input contract of the problem statement (Sec. 2): undirected graph,
 * positive weights, self-loops allowed, no multi-edges.  Stored as a
 * symmetric CSR with ascending columns.  When several violations are
 * present the most severe one is reported, in the order
 * ARG > DUPLICATE > WEIGHT > NOT_SYMMETRIC > OVERFLOW > EMPTY. */
static int severity(int s) {
    switch (s) {
    case ORC_ERR_ARG: return 6;
    case ORC_ERR_DUPLICATE: return 5;
    case ORC_ERR_WEIGHT: return 4;
    case ORC_ERR_NOT_SYMMETRIC: return 3;
    case ORC_ERR_OVERFLOW: return 2;
    case ORC_ERR_EMPTY: return 1;
    default: return 0;
    }
}
static int worse(int a, int b) { return severity(b) > severity(a) ? b : a; }

/* is (i, j, w) stored?  row j is searched by bisection (rows are sorted) */
static int has_arc(const int64_t *rowptr, const int32_t *col, const int32_t *w, int32_t i,
                   int32_t j, int32_t wt) {
    int64_t lo = rowptr[j], hi = rowptr[j + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < i) lo = mid + 1; else hi = mid;
    }
    return lo < rowptr[j + 1] && col[lo] == i && w[lo] == wt;
}

int orc_validate(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                 int64_t *two_m_out) {
    if (two_m_out) *two_m_out = 0;
    if (n < 0 || n > (int64_t)INT32_MAX - 1 || !rowptr) return ORC_ERR_ARG;
    if (rowptr[0] != 0) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) return ORC_ERR_ARG;
    if (rowptr[n] > (int64_t)INT32_MAX) return ORC_ERR_OVERFLOW;
    int st = ORC_OK;
    int64_t two_m = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            if (col[e] < 0 || col[e] >= n) { st = worse(st, ORC_ERR_ARG); continue; }
            if (e > rowptr[i]) {
                if (col[e] == col[e - 1]) st = worse(st, ORC_ERR_DUPLICATE);
                else if (col[e] < col[e - 1]) st = worse(st, ORC_ERR_ARG);
            }
            if (w[e] < 1) st = worse(st, ORC_ERR_WEIGHT);
            else two_m += w[e];
        }
    }
    if (severity(st) < severity(ORC_ERR_NOT_SYMMETRIC)) {
        for (int64_t i = 0; i < n && st == ORC_OK; ++i)
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
                if (col[e] != i && !has_arc(rowptr, col, w, (int32_t)i, col[e], w[e])) {
                    st = ORC_ERR_NOT_SYMMETRIC;
                    break;
                }
    }
    if (st != ORC_OK) return st;
    if (two_m >= ((int64_t)1 << 31)) return ORC_ERR_OVERFLOW;
    if (two_m == 0) return ORC_ERR_EMPTY;
    if (two_m_out) *two_m_out = two_m;
    return ORC_OK;
}

/* ----------------------------------------------------- definitions */
/* weighted degree k_i = sum of w(i,j) over the row of i (Sec. 2);
 * a self-loop is counted once (R1) */
static int64_t degrees(const orc_graph *g, int64_t *k) {
    int64_t two_m = 0;
    for (int64_t i = 0; i < g->n; ++i) {
        int64_t s = 0;
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) s += g->w[e];
        k[i] = s;
        two_m += s;
    }
    return two_m;
}

/* Modularity numerator from scratch, Eq. 3 scaled by (2m)^2:
 *   N = 2m * sum_i e_{i->C(i)} - sum_C a_C^2,   Q = N / (2m)^2
 * with e_{i->C} of Eq. 1 (self-loops included, they are intra-community)
 * and a_C of Eq. 2. */
static i128 modularity_num(const orc_graph *g, const int32_t *C, int64_t *two_m_out) {
    const int64_t n = g->n;
    int64_t *k = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *a = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    const int64_t two_m = degrees(g, k);
    for (int64_t i = 0; i < n; ++i) a[C[i]] += k[i];
    i128 ein = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e)
            if (C[g->col[e]] == C[i]) ein += g->w[e];
    i128 a2 = 0;
    for (int64_t c = 0; c < n; ++c) a2 += (i128)a[c] * a[c];
    free(k);
    free(a);
    if (two_m_out) *two_m_out = two_m;
    return (i128)two_m * ein - a2;
}

static void split128(i128 x, int64_t *hi, uint64_t *lo) {
    *hi = (int64_t)(x >> 64);
    *lo = (uint64_t)x;
}

/* labels must lie in [0, n) */
int orc_modularity(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                   const int32_t *labels, int64_t *num_hi, uint64_t *num_lo, int64_t *two_m) {
    orc_graph g = {n, rowptr[n], (int64_t *)rowptr, (int32_t *)col, (int32_t *)w};
    for (int64_t i = 0; i < n; ++i)
        if (labels[i] < 0 || labels[i] >= n) return ORC_ERR_ARG;
    i128 N = modularity_num(&g, labels, two_m);
    split128(N, num_hi, num_lo);
    return ORC_OK;
}

/* Gain of moving vertex i alone from C(i) to community c, Eq. 4 scaled by
 * (2m)^2 / 2 (R4):
 *   G = (2m e_{i->c} - k_i a_c) - (2m e_{i->C(i)\{i}} - k_i (a_{C(i)} - k_i))
 * with self-loops excluded from both e terms.  All sums from scratch. */
int orc_gain(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
             const int32_t *labels, int32_t i, int32_t c, int64_t *g_hi, uint64_t *g_lo) {
    orc_graph g = {n, rowptr[n], (int64_t *)rowptr, (int32_t *)col, (int32_t *)w};
    if (i < 0 || i >= n || c < 0 || c >= n) return ORC_ERR_ARG;
    int64_t *k = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    const int64_t two_m = degrees(&g, k);
    int64_t a_c = 0, a_old = 0, e_c = 0, e_old = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (labels[v] == c) a_c += k[v];
        if (labels[v] == labels[i]) a_old += k[v];
    }
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        if (col[e] == i) continue;
        if (labels[col[e]] == c) e_c += w[e];
        if (labels[col[e]] == labels[i]) e_old += w[e];
    }
    const i128 G = ((i128)two_m * e_c - (i128)k[i] * a_c) -
                   ((i128)two_m * e_old - (i128)k[i] * (a_old - k[i]));
    free(k);
    split128(G, g_hi, g_lo);
    return ORC_OK;
}

/* ------------------------------------------------- vertex following */
/* Sec. 4.3 and step 1 of Sec. 4.4.  D = vertices whose only incident edge is
 * (i, j) with j != i.  Each i in D is removed into j, except that of two
 * mutually single-degree vertices only the smaller id is removed (R3).  The
 * survivor gets self-loop weight 2*w(i,j) per removed vertex (R2).
 * Survivors are renumbered in ascending original id; map[v] is the new id of
 * v (or of the vertex v was merged into). */
static orc_graph *vertex_following(const orc_graph *g, int32_t *map) {
    const int64_t n = g->n;
    char *deg1 = (char *)calloc((size_t)(n ? n : 1), 1);
    char *removed = (char *)calloc((size_t)(n ? n : 1), 1);
    int32_t *target = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t *extra = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    int32_t *newid = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i)
        deg1[i] = (g->rowptr[i + 1] - g->rowptr[i] == 1) && g->col[g->rowptr[i]] != i;
    for (int64_t i = 0; i < n; ++i) {
        if (!deg1[i]) continue;
        int32_t j = g->col[g->rowptr[i]];
        if (deg1[j] && j < i) continue; /* i is the larger end of an isolated edge */
        removed[i] = 1;
        target[i] = j;
        extra[j] += 2 * (int64_t)g->w[g->rowptr[i]];
    }
    int64_t nn = 0;
    for (int64_t i = 0; i < n; ++i) newid[i] = removed[i] ? -1 : (int32_t)nn++;
    /* count the new rows */
    int64_t arcs = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (removed[i]) continue;
        int has_loop = 0;
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
            if (g->col[e] == i) has_loop = 1;
            else if (!removed[g->col[e]]) arcs++;
        }
        if (has_loop || extra[i] > 0) arcs++;
    }
    orc_graph *h = graph_alloc(nn, arcs);
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (removed[i]) continue;
        const int64_t row_start = o;
        int64_t loop_w = extra[i];
        int has_loop = extra[i] > 0;
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
            int32_t j = g->col[e];
            if (j == i) { loop_w += g->w[e]; has_loop = 1; }
            else if (!removed[j]) { h->col[o] = newid[j]; h->w[o] = g->w[e]; o++; }
        }
        if (has_loop) {
            /* insert the self-loop at its sorted position */
            int64_t p = o;
            while (p > row_start && h->col[p - 1] > newid[i]) {
                h->col[p] = h->col[p - 1];
                h->w[p] = h->w[p - 1];
                p--;
            }
            h->col[p] = newid[i];
            h->w[p] = (int32_t)loop_w;
            o++;
        }
        h->rowptr[newid[i] + 1] = o;
    }
    for (int64_t v = 0; v < n; ++v) map[v] = removed[v] ? newid[target[v]] : newid[v];
    free(deg1); free(removed); free(target); free(extra); free(newid);
    return h;
}

/* ----------------------------------------------------------- colouring */
/* Priority of the colouring (R11): pi(v) = (d(v), h(v xor seed), v),
 * compared lexicographically, where d(v) is the number of neighbours of v
 * other than v itself (largest degree first, Welsh and Powell 1967) and h is
 * the SplitMix64 output mixing function (Steele, Lea, Flood 2014).  With
 * order = 1 the degree is left out: pi(v) = (h(v xor seed), v). */
static uint64_t prio_hash(uint64_t x) {
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}
typedef struct { int64_t d; uint64_t h; int32_t v; } prio_t;
static int cmp_prio_desc(const void *a, const void *b) {
    const prio_t *x = (const prio_t *)a, *y = (const prio_t *)b;
    if (x->d != y->d) return x->d < y->d ? 1 : -1;
    if (x->h != y->h) return x->h < y->h ? 1 : -1;
    return (x->v < y->v) - (x->v > y->v);
}

/* Greedy distance-1 colouring visiting vertices in decreasing priority; each
 * takes the smallest colour not used by an already coloured neighbour.
 * Self-loops are ignored.  Returns the number of colours. */
static int32_t greedy_color(const orc_graph *g, uint64_t seed, int order, int32_t *color) {
    const int64_t n = g->n;
    prio_t *ord = (prio_t *)malloc((size_t)(n ? n : 1) * sizeof(prio_t));
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = 0;
        for (int64_t e = g->rowptr[v]; e < g->rowptr[v + 1]; ++e) d += g->col[e] != v;
        ord[v].d = order == 1 ? 0 : d;
        ord[v].h = prio_hash((uint64_t)v ^ seed);
        ord[v].v = (int32_t)v;
        color[v] = -1;
    }
    qsort(ord, (size_t)n, sizeof(prio_t), cmp_prio_desc);
    int64_t *stamp = (int64_t *)malloc(((size_t)n + 2) * sizeof(int64_t));
    for (int64_t c = 0; c < n + 2; ++c) stamp[c] = -1;
    int32_t ncol = 0;
    for (int64_t t = 0; t < n; ++t) {
        const int32_t v = ord[t].v;
        for (int64_t e = g->rowptr[v]; e < g->rowptr[v + 1]; ++e) {
            int32_t u = g->col[e];
            if (u != v && color[u] >= 0) stamp[color[u]] = v;
        }
        int32_t c = 0;
        while (stamp[c] == v) c++;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(ord);
    free(stamp);
    return ncol;
}

int32_t orc_color(int64_t n, const int64_t *rowptr, const int32_t *col, uint64_t seed,
                  int32_t order, int32_t *color) {
    orc_graph g = {n, rowptr[n], (int64_t *)rowptr, (int32_t *)col, NULL};
    return greedy_color(&g, seed, order, color);
}

/* ------------------------------------------------------------- sweep */
/* One colour class of one iteration (Alg. 1 while-loop body, Sec. 4.1 rules).
 * Every vertex of S decides from the current state; the decided moves are
 * applied together afterwards (R6).  Returns the number of moves. */
typedef struct {
    int64_t *e;      /* e_{i->c} accumulator, indexed by community */
    char *seen;
    int32_t *touched;
    int32_t *mv_v, *mv_c;
} sweep_scratch;

static int64_t sweep_class(const orc_graph *g, const int32_t *S, int64_t ns, int32_t *C,
                           int64_t *a, int64_t *size, const int64_t *k, int64_t two_m,
                           sweep_scratch *sc) {
    int64_t nmoves = 0;
    for (int64_t t = 0; t < ns; ++t) {
        const int32_t i = S[t];
        const int32_t ci = C[i];
        const int64_t ki = k[i];
        /* neighbouring communities and e_{i->c}, Eq. 1 (self-loop excluded, R4) */
        int64_t nt = 0;
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
            const int32_t j = g->col[e];
            if (j == i) continue;
            const int32_t c = C[j];
            if (!sc->seen[c]) { sc->seen[c] = 1; sc->touched[nt++] = c; }
            sc->e[c] += g->w[e];
        }
        const int64_t e_old = sc->e[ci];
        const i128 s_old = (i128)two_m * e_old - (i128)ki * (a[ci] - ki);
        int32_t best = ci;
        i128 bestG = 0;
        for (int64_t q = 0; q < nt; ++q) {
            const int32_t c = sc->touched[q];
            if (c == ci) continue;
            const i128 G = ((i128)two_m * sc->e[c] - (i128)ki * a[c]) - s_old;
            /* maximum gain; equal gains -> minimum label (Sec. 4.1) */
            if (G > bestG || (G == bestG && c < best)) { best = c; bestG = G; }
        }
        for (int64_t q = 0; q < nt; ++q) { sc->e[sc->touched[q]] = 0; sc->seen[sc->touched[q]] = 0; }
        if (bestG > 0) {
            /* singlet minimum-label rule (Sec. 4.1), judged on the class-start state (R7) */
            if (size[ci] == 1 && size[best] == 1 && best > ci) continue;
            sc->mv_v[nmoves] = i;
            sc->mv_c[nmoves] = best;
            nmoves++;
        }
    }
    for (int64_t t = 0; t < nmoves; ++t) {
        const int32_t i = sc->mv_v[t], c = sc->mv_c[t];
        a[C[i]] -= k[i];
        size[C[i]] -= 1;
        a[c] += k[i];
        size[c] += 1;
        C[i] = c;
    }
    return nmoves;
}

/* Timing sample (for the bench's host-core baseline only): from the
 * singleton partition of the given graph, the oracle's own sweep_class over
 * the `count` vertices first, first+1, ... as one class of an uncoloured
 * first iteration.  Reports the moves, the arcs those vertices scan and the
 * wall time of the sweep alone (set-up excluded).  No other oracle result
 * depends on this entry point. */
int orc_sweep_sample(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                     int64_t first, int64_t count, int64_t *moves, int64_t *visits,
                     double *seconds) {
    if (n <= 0 || first < 0 || count < 0 || first + count > n) return ORC_ERR_ARG;
    orc_graph G = {n, rowptr[n], (int64_t *)rowptr, (int32_t *)col, (int32_t *)w};
    int64_t *k = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *a = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *size = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *C = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *S = (int32_t *)malloc((size_t)(count ? count : 1) * sizeof(int32_t));
    sweep_scratch sc;
    sc.e = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    sc.seen = (char *)calloc((size_t)n, 1);
    sc.touched = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    sc.mv_v = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    sc.mv_c = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!k || !a || !size || !C || !S || !sc.e || !sc.seen || !sc.touched || !sc.mv_v ||
        !sc.mv_c) {
        free(k); free(a); free(size); free(C); free(S);
        free(sc.e); free(sc.seen); free(sc.touched); free(sc.mv_v); free(sc.mv_c);
        return ORC_ERR_OOM;
    }
    const int64_t two_m = degrees(&G, k);
    for (int64_t i = 0; i < n; ++i) { C[i] = (int32_t)i; a[i] = k[i]; size[i] = 1; }
    int64_t vis = 0;
    for (int64_t t = 0; t < count; ++t) {
        S[t] = (int32_t)(first + t);
        vis += rowptr[first + t + 1] - rowptr[first + t];
    }
    const double t0 = now_s();
    *moves = sweep_class(&G, S, count, C, a, size, k, two_m, &sc);
    *seconds = now_s() - t0;
    *visits = vis;
    free(k); free(a); free(size); free(C); free(S);
    free(sc.e); free(sc.seen); free(sc.touched); free(sc.mv_v); free(sc.mv_c);
    return ORC_OK;
}

/* ------------------------------------------------------------- rebuild */
/* Coarse graph of Sec. 4.4 step 4 / Sec. 4.5 (i)-(iii): vertex c' per
 * non-empty community (renumbered in ascending old label), and for every
 * stored arc (u, v, w) the arc (c'(u), c'(v), w); equal pairs are summed.
 * A community's self-loop is therefore the sum over its directed intra arcs
 * (R1). */
typedef struct { int32_t u, v, w; } arc_t;
static int cmp_arc(const void *a, const void *b) {
    const arc_t *x = (const arc_t *)a, *y = (const arc_t *)b;
    if (x->u != y->u) return (x->u > y->u) - (x->u < y->u);
    return (x->v > y->v) - (x->v < y->v);
}
static orc_graph *rebuild(const orc_graph *g, const int32_t *C, const int32_t *newid,
                          int64_t n_next) {
    const int64_t A = g->arcs;
    arc_t *t = (arc_t *)malloc((size_t)(A ? A : 1) * sizeof(arc_t));
    for (int64_t u = 0; u < g->n; ++u)
        for (int64_t e = g->rowptr[u]; e < g->rowptr[u + 1]; ++e) {
            t[e].u = newid[C[u]];
            t[e].v = newid[C[g->col[e]]];
            t[e].w = g->w[e];
        }
    qsort(t, (size_t)A, sizeof(arc_t), cmp_arc);
    int64_t nu = 0;
    for (int64_t e = 0; e < A; ++e)
        if (e == 0 || t[e].u != t[e - 1].u || t[e].v != t[e - 1].v) nu++;
    orc_graph *h = graph_alloc(n_next, nu);
    int64_t o = -1;
    for (int64_t e = 0; e < A; ++e) {
        if (e == 0 || t[e].u != t[e - 1].u || t[e].v != t[e - 1].v) {
            o++;
            h->col[o] = t[e].v;
            h->w[o] = 0;
            h->rowptr[t[e].u + 1]++;
        }
        h->w[o] += t[e].w;
    }
    for (int64_t c = 0; c < n_next; ++c) h->rowptr[c + 1] += h->rowptr[c];
    free(t);
    return h;
}

/* ------------------------------------- recursive single-neighbour VF */
/* The extension sketched at the end of Sec. 4.3 (R23).  A single-neighbour
 * vertex i has exactly one neighbour j != i and an optional self-loop of
 * weight l.  With k_i = w(i,j) + l, the lower bound of Eq. (eqnClaimIItemp)
 * on the gain of moving i into C(j), taken at the largest community degree
 * C(j) can have without i (a_C(j) <= 2m - k_i), is
 *     w(i,j)/m - 2 k_i (2m - k_i) / (2m)^2,
 * which is positive iff 2m w(i,j) > k_i (2m - k_i), i.e. iff
 * k_i^2 > 2m l.  A vertex passing this test joins C(j) whatever the rest of
 * the partition is, so it is merged into j before the phases start, as
 * plain vertex following does with single-degree vertices (l = 0 always
 * passes).  Rounds: every vertex of the current graph is tested at once; of
 * two single-neighbour vertices adjacent to each other only the smaller id
 * merges (R3); the merged graph is the coarse graph of that partition (a
 * survivor's loop becomes its old loop + the merged loops + 2 w(i,j), R1,
 * R2) with survivors renumbered ascending; rounds repeat until no vertex
 * passes.  Takes ownership of G; map (n_orig entries) is composed. */
static orc_graph *vf_recursive_rounds(orc_graph *G, int32_t *map, int64_t n_orig) {
    int64_t two_m = 0;
    for (int64_t e = 0; e < G->arcs; ++e) two_m += G->w[e];
    for (;;) {
        const int64_t n = G->n;
        int32_t *target = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
        int64_t merges = 0;
        for (int64_t i = 0; i < n; ++i) {
            target[i] = -1;
            int64_t nb = 0, loop = 0, wij = 0;
            int32_t j = -1;
            for (int64_t e = G->rowptr[i]; e < G->rowptr[i + 1]; ++e) {
                if (G->col[e] == i) loop += G->w[e];
                else { nb++; j = G->col[e]; wij = G->w[e]; }
            }
            if (nb != 1) continue;
            const int64_t k = wij + loop;
            if ((i128)k * k > (i128)two_m * loop) target[i] = j;
        }
        int32_t *C = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
        for (int64_t i = 0; i < n; ++i) {
            const int32_t j = target[i];
            /* of two single-neighbour vertices passing towards each other,
             * the smaller merges into the larger */
            const int merge = j >= 0 && !(target[j] == (int32_t)i && j < i);
            C[i] = merge ? j : (int32_t)i;
            merges += merge;
        }
        free(target);
        if (merges == 0) {
            free(C);
            return G;
        }
        int32_t *newid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        int64_t nn = 0;
        for (int64_t i = 0; i < n; ++i) newid[i] = C[i] == i ? (int32_t)nn++ : -1;
        orc_graph *H = rebuild(G, C, newid, nn);
        for (int64_t v = 0; v < n_orig; ++v) map[v] = newid[C[map[v]]];
        free(C);
        free(newid);
        graph_free(G);
        G = H;
    }
}

int orc_rebuild(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                const int32_t *labels, orc_graph **out) {
    orc_graph g = {n, rowptr[n], (int64_t *)rowptr, (int32_t *)col, (int32_t *)w};
    int32_t *newid = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    char *used = (char *)calloc((size_t)(n ? n : 1), 1);
    for (int64_t i = 0; i < n; ++i) {
        if (labels[i] < 0 || labels[i] >= n) { free(newid); free(used); return ORC_ERR_ARG; }
        used[labels[i]] = 1;
    }
    int64_t nn = 0;
    for (int64_t c = 0; c < n; ++c) newid[c] = used[c] ? (int32_t)nn++ : -1;
    *out = rebuild(&g, labels, newid, nn);
    free(newid);
    free(used);
    return ORC_OK;
}

int orc_vertex_following(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                         int32_t *map, orc_graph **out) {
    orc_graph g = {n, rowptr[n], (int64_t *)rowptr, (int32_t *)col, (int32_t *)w};
    *out = vertex_following(&g, map);
    return ORC_OK;
}

void orc_graph_size(const orc_graph *g, int64_t *n, int64_t *arcs) { *n = g->n; *arcs = g->arcs; }
void orc_graph_copy(const orc_graph *g, int64_t *rowptr, int32_t *col, int32_t *w) {
    memcpy(rowptr, g->rowptr, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(col, g->col, (size_t)g->arcs * sizeof(int32_t));
    memcpy(w, g->w, (size_t)g->arcs * sizeof(int32_t));
}
void orc_graph_free(orc_graph *g) { graph_free(g); }

/* --------------------------------------------------------------- driver */
static orc_phase *new_phase(orc_result *r) {
    if (r->num_phases == r->cap_ph) {
        r->cap_ph = r->cap_ph ? 2 * r->cap_ph : 16;
        r->ph = (orc_phase *)realloc(r->ph, (size_t)r->cap_ph * sizeof(orc_phase));
    }
    orc_phase *p = &r->ph[r->num_phases++];
    memset(p, 0, sizeof(*p));
    return p;
}
static void push_iter(orc_result *r, int32_t phase, int32_t iter, int64_t moved, i128 N,
                      double secs) {
    if (r->num_iters == r->cap_it) {
        r->cap_it = r->cap_it ? 2 * r->cap_it : 64;
        r->it = (orc_iter *)realloc(r->it, (size_t)r->cap_it * sizeof(orc_iter));
    }
    orc_iter *t = &r->it[r->num_iters++];
    t->phase = phase; t->iter = iter; t->moved = moved; t->N = N; t->seconds = secs;
}

static int64_t abs64(int64_t x) { return x < 0 ? -x : x; }

/* Stopping test (R9): the net gain N_C - N_P, signed, below theta relative to
 * |N_P|, on exact numerators.  Alg. 1 prints the relative form; Sec. 4.1
 * (last paragraph) relies on a minimum net gain to continue, so a negative
 * gain stops the loop.  |N| < 2^62, so both differences fit in int64. */
static int gain_below(i128 Nc, i128 Np, double theta, int abs_mode) {
    int64_t d = (int64_t)(Nc - Np);
    if (abs_mode) d = abs64(d);  /* the printed form of Alg. 1 (variant) */
    const int64_t b = abs64((int64_t)Np);
    return (double)d < theta * (double)b;
}

void orc_free(orc_result *r);

int orc_run(int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
            const orc_params *prm, orc_result **out) {
    *out = NULL;
    int64_t two_m_in = 0;
    int st = orc_validate(n, rowptr, col, w, &two_m_in);
    if (st != ORC_OK) return st;
    const double t_start = now_s();
    orc_result *r = (orc_result *)calloc(1, sizeof(orc_result));
    r->n_orig = n;
    r->two_m = two_m_in;
    int32_t *map = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    orc_graph *G;
    if (prm->vertex_following) {
        G = vertex_following(&(orc_graph){n, rowptr[n], (int64_t *)rowptr, (int32_t *)col,
                                          (int32_t *)w}, map);
    } else {
        G = graph_copy_in(n, rowptr, col, w);
        for (int64_t v = 0; v < n; ++v) map[v] = (int32_t)v;
    }
    if (prm->vertex_following && prm->vf_recursive) G = vf_recursive_rounds(G, map, n);
    r->vf_map = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    memcpy(r->vf_map, map, (size_t)n * sizeof(int32_t));
    r->vf_n = G->n;

    int colour_stopped = 0, coloured_phases = 0;
    for (int32_t p = 0; p < prm->max_phases; ++p) {
        const int64_t np = G->n;
        orc_phase *ph = new_phase(r);
        ph->n = np;
        ph->arcs = G->arcs;
        const int colour_on = prm->coloring && !colour_stopped && np >= prm->color_cutoff &&
                              (prm->color_phases <= 0 || coloured_phases < prm->color_phases);
        coloured_phases += colour_on;
        const double theta = (colour_on && prm->theta_high > 0.0) ? prm->theta_high
                                                                  : prm->theta_low;
        ph->colored = colour_on;
        ph->theta = theta;

        /* colour classes (Sec. 4.2): ascending colour, ascending id within a class */
        int32_t *order = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
        int64_t *cls_off;
        int32_t K = 1;
        int32_t *color = NULL;
        if (colour_on) {
            color = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
            K = greedy_color(G, prm->color_seed + (uint64_t)p, prm->color_order, color);
            cls_off = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
            for (int64_t v = 0; v < np; ++v) cls_off[color[v] + 1]++;
            for (int32_t c = 0; c < K; ++c) cls_off[c + 1] += cls_off[c];
            int64_t *fill = (int64_t *)malloc((size_t)K * sizeof(int64_t));
            for (int32_t c = 0; c < K; ++c) fill[c] = cls_off[c];
            for (int64_t v = 0; v < np; ++v) order[fill[color[v]]++] = (int32_t)v;
            free(fill);
        } else {
            cls_off = (int64_t *)calloc(2, sizeof(int64_t));
            cls_off[1] = np;
            for (int64_t v = 0; v < np; ++v) order[v] = (int32_t)v;
        }
        ph->num_colors = colour_on ? K : 0;
        if (prm->trace) {
            ph->graph = graph_copy_in(G->n, G->rowptr, G->col, G->w);
            if (colour_on) {
                ph->colors = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
                memcpy(ph->colors, color, (size_t)np * sizeof(int32_t));
            }
        }

        /* initialisation of Alg. 1: C(i) = {i}, a_i = k_i */
        int64_t *k = (int64_t *)malloc((size_t)(np ? np : 1) * sizeof(int64_t));
        int64_t *a = (int64_t *)malloc((size_t)(np ? np : 1) * sizeof(int64_t));
        int64_t *size = (int64_t *)malloc((size_t)(np ? np : 1) * sizeof(int64_t));
        int32_t *C = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
        const int64_t two_m = degrees(G, k);
        ph->two_m = two_m;
        for (int64_t i = 0; i < np; ++i) { C[i] = (int32_t)i; a[i] = k[i]; size[i] = 1; }
        ph->N_start = modularity_num(G, C, NULL);

        sweep_scratch sc;
        sc.e = (int64_t *)calloc((size_t)(np ? np : 1), sizeof(int64_t));
        sc.seen = (char *)calloc((size_t)(np ? np : 1), 1);
        sc.touched = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
        sc.mv_v = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
        sc.mv_c = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));

        /* the while-loop of Alg. 1 with the stopping rules R9, R10 */
        int32_t iter = 0;
        int have_NP = 0;
        i128 N_P = 0, N_C = ph->N_start;
        const double t0 = now_s();
        int32_t **itl = NULL;
        int32_t itl_cap = 0;
        for (;;) {
            const double ti = now_s();
            int64_t moved = 0;
            for (int32_t c = 0; c < K; ++c)
                moved += sweep_class(G, order + cls_off[c], cls_off[c + 1] - cls_off[c], C, a,
                                     size, k, two_m, &sc);
            iter++;
            N_C = modularity_num(G, C, NULL);
            push_iter(r, p, iter, moved, N_C, now_s() - ti);
            if (prm->trace) {
                if (iter > itl_cap) {
                    itl_cap = itl_cap ? 2 * itl_cap : 16;
                    itl = (int32_t **)realloc(itl, (size_t)itl_cap * sizeof(int32_t *));
                }
                itl[iter - 1] = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
                memcpy(itl[iter - 1], C, (size_t)np * sizeof(int32_t));
            }
            if (moved == 0) break;
            if (have_NP && gain_below(N_C, N_P, theta, prm->abs_threshold)) break;
            if (iter >= prm->max_iters) break;
            N_P = N_C;
            have_NP = 1;
        }
        ph->seconds = now_s() - t0;
        ph->iterations = iter;
        ph->iter_labels = itl;
        ph->N_end = N_C;

        /* renumber non-empty communities in ascending label (Sec. 4.5 i) */
        int32_t *newid = (int32_t *)malloc((size_t)(np ? np : 1) * sizeof(int32_t));
        int64_t nn = 0;
        for (int64_t c = 0; c < np; ++c) newid[c] = size[c] > 0 ? (int32_t)nn++ : -1;
        ph->n_next = nn;
        for (int64_t v = 0; v < n; ++v) map[v] = newid[C[map[v]]];
        ph->labels = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
        memcpy(ph->labels, map, (size_t)n * sizeof(int32_t));

        /* phase control (R12, R13) */
        int stop = 0;
        if (nn == np) stop = 1;
        else if (colour_on) {
            if (prm->theta_high > 0.0 &&
                gain_below(N_C, ph->N_start, prm->theta_high, prm->abs_threshold))
                colour_stopped = 1;
        } else if (gain_below(N_C, ph->N_start, prm->theta_low, prm->abs_threshold)) {
            stop = 1;
        }
        if (p + 1 >= prm->max_phases) stop = 1;
        orc_graph *H = stop ? NULL : rebuild(G, C, newid, nn);

        free(order); free(cls_off); free(color); free(k); free(a); free(size); free(C);
        free(sc.e); free(sc.seen); free(sc.touched); free(sc.mv_v); free(sc.mv_c);
        free(newid);
        graph_free(G);
        G = H;
        if (stop) break;
    }
    graph_free(G);
    free(map);
    r->seconds_total = now_s() - t_start;
    *out = r;
    return ORC_OK;
}

/* ------------------------------------------------------------ accessors */
int32_t orc_num_phases(const orc_result *r) { return r->num_phases; }
int64_t orc_two_m(const orc_result *r) { return r->two_m; }
int64_t orc_vf_n(const orc_result *r) { return r->vf_n; }
double orc_seconds_total(const orc_result *r) { return r->seconds_total; }
void orc_vf_map(const orc_result *r, int32_t *out) {
    memcpy(out, r->vf_map, (size_t)r->n_orig * sizeof(int32_t));
}

/* ints: n, arcs, n_next, colored, num_colors, iterations, two_m
 * nums: N_start hi/lo, N_end hi/lo;  dbl: theta, seconds */
int orc_phase_info(const orc_result *r, int32_t p, int64_t *ints, int64_t *num_hi,
                   uint64_t *num_lo, double *dbl) {
    if (p < 0 || p >= r->num_phases) return ORC_ERR_STATE;
    const orc_phase *ph = &r->ph[p];
    ints[0] = ph->n; ints[1] = ph->arcs; ints[2] = ph->n_next; ints[3] = ph->colored;
    ints[4] = ph->num_colors; ints[5] = ph->iterations; ints[6] = ph->two_m;
    split128(ph->N_start, &num_hi[0], &num_lo[0]);
    split128(ph->N_end, &num_hi[1], &num_lo[1]);
    dbl[0] = ph->theta;
    dbl[1] = ph->seconds;
    return ORC_OK;
}
int orc_phase_labels(const orc_result *r, int32_t p, int32_t *out) {
    if (p < 0 || p >= r->num_phases) return ORC_ERR_STATE;
    memcpy(out, r->ph[p].labels, (size_t)r->n_orig * sizeof(int32_t));
    return ORC_OK;
}
const orc_graph *orc_phase_graph(const orc_result *r, int32_t p) {
    if (p < 0 || p >= r->num_phases) return NULL;
    return r->ph[p].graph;
}
int orc_phase_colors(const orc_result *r, int32_t p, int32_t *out) {
    if (p < 0 || p >= r->num_phases || !r->ph[p].colors) return ORC_ERR_STATE;
    memcpy(out, r->ph[p].colors, (size_t)r->ph[p].n * sizeof(int32_t));
    return ORC_OK;
}
int orc_phase_iter_labels(const orc_result *r, int32_t p, int32_t it, int32_t *out) {
    if (p < 0 || p >= r->num_phases || !r->ph[p].iter_labels || it < 0 ||
        it >= r->ph[p].iterations)
        return ORC_ERR_STATE;
    memcpy(out, r->ph[p].iter_labels[it], (size_t)r->ph[p].n * sizeof(int32_t));
    return ORC_OK;
}
int64_t orc_num_iters(const orc_result *r) { return r->num_iters; }
/* per record: phase, iter, moved, N hi, N lo (as bits), seconds (as bits) */
void orc_iters(const orc_result *r, int64_t *phase_iter_moved, int64_t *num_hi, uint64_t *num_lo,
               double *secs) {
    for (int64_t t = 0; t < r->num_iters; ++t) {
        phase_iter_moved[3 * t] = r->it[t].phase;
        phase_iter_moved[3 * t + 1] = r->it[t].iter;
        phase_iter_moved[3 * t + 2] = r->it[t].moved;
        split128(r->it[t].N, &num_hi[t], &num_lo[t]);
        secs[t] = r->it[t].seconds;
    }
}
void orc_free(orc_result *r) {
    if (!r) return;
    for (int32_t p = 0; p < r->num_phases; ++p) {
        orc_phase *ph = &r->ph[p];
        free(ph->labels);
        graph_free(ph->graph);
        free(ph->colors);
        if (ph->iter_labels) {
            for (int32_t t = 0; t < ph->iterations; ++t) free(ph->iter_labels[t]);
            free(ph->iter_labels);
        }
    }
    free(r->ph);
    free(r->it);
    free(r->vf_map);
    free(r);
}


/* ------------------------------------------------------------------------
 * Qualitative comparison of two partitions (Sec. 5): every unordered pair
 * {u, v} of the n vertices is a true positive (same community in both s and
 * p), a false positive (same only in p), a false negative (same only in s)
 * or a true negative (different in both).  Plain definition: all n(n-1)/2
 * pairs are examined.  out = {TP, FP, FN, TN}.
 * ---------------------------------------------------------------------- */
int orc_compare(int64_t n, const int32_t *s, const int32_t *p, uint64_t *out) {
    if (n < 0 || !out || (n > 0 && (!s || !p))) return ORC_ERR_ARG;
    uint64_t tp = 0, fp = 0, fn = 0, tn = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t v = u + 1; v < n; ++v) {
            const int same_s = s[u] == s[v], same_p = p[u] == p[v];
            if (same_s && same_p) ++tp;
            else if (same_p) ++fp;
            else if (same_s) ++fn;
            else ++tn;
        }
    out[0] = tp;
    out[1] = fp;
    out[2] = fn;
    out[3] = tn;
    return ORC_OK;
}
