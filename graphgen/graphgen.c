/*
 * graphgen.c -- seeded synthetic graph generators (input side only).
 *
 * This file produces the symmetric CSR inputs that both the CUDA library and
 * the serial oracle consume.  It contains none of the community-detection
 * arithmetic: it only draws edges and assembles a validated CSR (rows sorted
 * ascending, duplicates merged, every undirected edge stored in both rows).
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) seeds xoshiro256**
 * (Blackman, Vigna, "Scrambled linear pseudorandom number generators",
 * 2018).  Work is split into fixed-size chunks, each with its own stream
 * derived from (seed, chunk index), so the output does not depend on the
 * number of OpenMP threads.
 *
 * Generators (the paper's real inputs are not available; these are
 * stand-ins with the same kinds of structure):
 *   gg_planted  planted partition, edges drawn by geometric skipping
 *               (Batagelj, Brandes, "Efficient generation of large random
 *               networks", Phys. Rev. E 71, 2005)
 *   gg_rmat     R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004), duplicate
 *               draws merged into integer weights
 *   gg_chunglu  Chung-Lu expected-degree graph with a power-law weight
 *               sequence, plus a layer of pendant (degree-1) vertices
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t xo_next(xo256 *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}
static void xo_seed(xo256 *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed;
    uint64_t k = sm64_next(&x) ^ (stream * 0xD1B54A32D192ED03ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&k);
}
static inline double xo_unif(xo256 *r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }
static inline uint64_t xo_below(xo256 *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)xo_next(r) * n) >> 64);
}

/* ------------------------------------------------------------ edge list */
typedef struct { int32_t u, v, w; } gg_edge;

typedef struct {
    int64_t n;
    int64_t arcs;
    int64_t *rowptr;
    int32_t *col;
    int32_t *w;
    /* generator statistics */
    int64_t draws, self_draws, dup_merged;
} gg_graph;

enum { MERGE_SUM = 0, MERGE_MAX = 1 };

/* Ascending sort of 64-bit keys: insertion sort for short runs, otherwise
 * quicksort with a three-way partition (rows of R-MAT hubs repeat keys
 * often) recursing into the smaller side, so the stack stays O(log n). */
static void sort_u64(uint64_t *x, int64_t n) {
    while (n > 24) {
        const uint64_t p0 = x[0], p1 = x[n / 2], p2 = x[n - 1];
        const uint64_t piv = p0 < p1 ? (p1 < p2 ? p1 : (p0 < p2 ? p2 : p0))
                                     : (p0 < p2 ? p0 : (p1 < p2 ? p2 : p1));
        int64_t lt = 0, i = 0, gt = n; /* [0,lt) < piv, [lt,i) == piv, [gt,n) > piv */
        while (i < gt) {
            const uint64_t v = x[i];
            if (v < piv) { x[i] = x[lt]; x[lt] = v; ++lt; ++i; }
            else if (v > piv) { --gt; x[i] = x[gt]; x[gt] = v; }
            else ++i;
        }
        if (lt < n - gt) { sort_u64(x, lt); x += gt; n -= gt; }
        else { sort_u64(x + gt, n - gt); n = lt; }
    }
    for (int64_t i = 1; i < n; ++i) {
        const uint64_t v = x[i];
        int64_t j = i;
        while (j > 0 && x[j - 1] > v) { x[j] = x[j - 1]; --j; }
        x[j] = v;
    }
}

/* Assemble a symmetric CSR from undirected edges.  Edges with u < 0 are
 * skipped; a self-loop (u == v) is stored once in its row.  Duplicate (u,v)
 * entries are merged by summing (MERGE_SUM) or by taking the maximum weight
 * (MERGE_MAX). */
static gg_graph *build_csr(int64_t n, const gg_edge *e, int64_t ne, int mode) {
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    g->n = n;
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) { free(g); return NULL; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; ++i) {
        if (e[i].u < 0) continue;
#pragma omp atomic
        cnt[e[i].u]++;
        if (e[i].u != e[i].v) {
#pragma omp atomic
            cnt[e[i].v]++;
        }
    }
    int64_t *off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    off[0] = 0;
    for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + cnt[i];
    const int64_t total = off[n];
    uint64_t *packed = (uint64_t *)malloc((size_t)(total ? total : 1) * sizeof(uint64_t));
    for (int64_t i = 0; i < n; ++i) cnt[i] = off[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; ++i) {
        int32_t u = e[i].u, v = e[i].v;
        if (u < 0) continue;
        uint64_t wv = (uint32_t)e[i].w;
        int64_t p;
#pragma omp atomic capture
        p = cnt[u]++;
        packed[p] = ((uint64_t)(uint32_t)v << 32) | wv;
        if (u != v) {
#pragma omp atomic capture
            p = cnt[v]++;
            packed[p] = ((uint64_t)(uint32_t)u << 32) | wv;
        }
    }
    /* sort each row, merge duplicates in place, record the new length */
    int64_t *newlen = cnt; /* reuse */
    int64_t dups = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : dups)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t *r = packed + off[i];
        int64_t d = off[i + 1] - off[i];
        if (d > 1) sort_u64(r, d);
        int64_t o = 0;
        for (int64_t k = 0; k < d; ++k) {
            uint32_t c = (uint32_t)(r[k] >> 32), wk = (uint32_t)r[k];
            if (o > 0 && (uint32_t)(r[o - 1] >> 32) == c) {
                uint32_t wp = (uint32_t)r[o - 1];
                uint32_t wn = (mode == MERGE_SUM) ? wp + wk : (wk > wp ? wk : wp);
                r[o - 1] = ((uint64_t)c << 32) | wn;
                dups++;
            } else {
                r[o++] = r[k];
            }
        }
        newlen[i] = o;
    }
    g->dup_merged = dups;
    g->rowptr = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) g->rowptr[i + 1] = g->rowptr[i] + newlen[i];
    g->arcs = g->rowptr[n];
    g->col = (int32_t *)malloc((size_t)(g->arcs ? g->arcs : 1) * sizeof(int32_t));
    g->w = (int32_t *)malloc((size_t)(g->arcs ? g->arcs : 1) * sizeof(int32_t));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t *r = packed + off[i];
        int64_t o = g->rowptr[i];
        for (int64_t k = 0; k < newlen[i]; ++k) {
            g->col[o + k] = (int32_t)(uint32_t)(r[k] >> 32);
            g->w[o + k] = (int32_t)(uint32_t)r[k];
        }
    }
    free(packed);
    free(off);
    free(cnt);
    return g;
}

/* Threads of the OpenMP regions that the calling thread starts (0 = the
 * default).  Lets several host threads generate graphs side by side without
 * oversubscribing the cores; the output never depends on it. */
void gg_set_threads(int32_t t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------ accessors */
void gg_size(const gg_graph *g, int64_t *n, int64_t *arcs) { *n = g->n; *arcs = g->arcs; }
void gg_stats(const gg_graph *g, int64_t *draws, int64_t *self_draws, int64_t *dup_merged) {
    *draws = g->draws; *self_draws = g->self_draws; *dup_merged = g->dup_merged;
}
void gg_copy(const gg_graph *g, int64_t *rowptr, int32_t *col, int32_t *w) {
    memcpy(rowptr, g->rowptr, ((size_t)g->n + 1) * sizeof(int64_t));
    if (g->arcs) {
        memcpy(col, g->col, (size_t)g->arcs * sizeof(int32_t));
        memcpy(w, g->w, (size_t)g->arcs * sizeof(int32_t));
    }
}
void gg_free(gg_graph *g) {
    if (!g) return;
    free(g->rowptr); free(g->col); free(g->w); free(g);
}

/* Build a CSR from a caller-provided undirected edge list (u[i], v[i], w[i]);
 * duplicates are summed.  Used for hand-made test graphs. */
gg_graph *gg_from_edges(int64_t n, int64_t ne, const int32_t *u, const int32_t *v, const int32_t *w) {
    gg_edge *e = (gg_edge *)malloc((size_t)(ne ? ne : 1) * sizeof(gg_edge));
    for (int64_t i = 0; i < ne; ++i) { e[i].u = u[i]; e[i].v = v[i]; e[i].w = w[i]; }
    gg_graph *g = build_csr(n, e, ne, MERGE_SUM);
    free(e);
    return g;
}

/* --------------------------------------------------- planted partition */
/* n vertices in `blocks` contiguous blocks of near-equal size (the first
 * n % blocks blocks get one extra vertex).  Each unordered pair i < j is an
 * edge independently with probability p_in (same block) or p_out.  Weights
 * are uniform integers in [wmin, wmax]. */
typedef struct { gg_edge *e; int64_t n, cap; } ebuf;
static void eb_push(ebuf *b, int32_t u, int32_t v, int32_t w) {
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 1024;
        b->e = (gg_edge *)realloc(b->e, (size_t)b->cap * sizeof(gg_edge));
    }
    b->e[b->n].u = u; b->e[b->n].v = v; b->e[b->n].w = w; b->n++;
}
/* append every j in [lo, hi) independently with probability p */
static void skip_range(ebuf *b, xo256 *r, int32_t i, int64_t lo, int64_t hi, double p,
                       int32_t wmin, int32_t wmax) {
    if (p <= 0.0 || lo >= hi) return;
    const uint64_t wr = (uint64_t)(wmax - wmin + 1);
    if (p >= 1.0) {
        for (int64_t j = lo; j < hi; ++j) eb_push(b, i, (int32_t)j, wmin + (int32_t)xo_below(r, wr));
        return;
    }
    const double lq = log(1.0 - p);
    int64_t j = lo - 1;
    for (;;) {
        double u = xo_unif(r);
        double s = floor(log(1.0 - u) / lq);
        if (s > (double)(hi - j)) break;
        j += 1 + (int64_t)s;
        if (j >= hi) break;
        eb_push(b, i, (int32_t)j, wmin + (int32_t)xo_below(r, wr));
    }
}

gg_graph *gg_planted(int64_t n, int32_t blocks, double p_in, double p_out, int32_t wmin,
                     int32_t wmax, uint64_t seed) {
    if (n <= 0 || blocks <= 0 || blocks > n || wmin < 1 || wmax < wmin) return NULL;
    const int64_t base = n / blocks, extra = n % blocks;
    /* block end for vertex i */
    const int64_t CH = 256; /* vertices per stream chunk */
    const int64_t nch = (n + CH - 1) / CH;
    ebuf *bufs = (ebuf *)calloc((size_t)nch, sizeof(ebuf));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < nch; ++c) {
        xo256 r;
        xo_seed(&r, seed, (uint64_t)c);
        for (int64_t i = c * CH; i < (c + 1) * CH && i < n; ++i) {
            /* block index of i */
            int64_t bi;
            if (i < extra * (base + 1)) bi = i / (base + 1);
            else bi = extra + (i - extra * (base + 1)) / base;
            int64_t bend = (bi < extra) ? (bi + 1) * (base + 1)
                                        : extra * (base + 1) + (bi - extra + 1) * base;
            skip_range(&bufs[c], &r, (int32_t)i, i + 1, bend, p_in, wmin, wmax);
            skip_range(&bufs[c], &r, (int32_t)i, bend, n, p_out, wmin, wmax);
        }
    }
    int64_t ne = 0;
    for (int64_t c = 0; c < nch; ++c) ne += bufs[c].n;
    gg_edge *e = (gg_edge *)malloc((size_t)(ne ? ne : 1) * sizeof(gg_edge));
    int64_t o = 0;
    for (int64_t c = 0; c < nch; ++c) {
        if (bufs[c].n) memcpy(e + o, bufs[c].e, (size_t)bufs[c].n * sizeof(gg_edge));
        o += bufs[c].n;
        free(bufs[c].e);
    }
    free(bufs);
    gg_graph *g = build_csr(n, e, ne, MERGE_SUM);
    if (g) g->draws = ne;
    free(e);
    return g;
}

/* ----------------------------------------------------------------- R-MAT */
/* 2^scale vertices, `draws` edge draws with quadrant probabilities
 * (a, b, c, 1-a-b-c).  Self draws are dropped, each draw is stored as the
 * undirected edge (min, max) with weight 1, and duplicate draws are merged
 * with their multiplicity as the weight. */
gg_graph *gg_rmat(int32_t scale, int64_t draws, double a, double b, double c, uint64_t seed) {
    if (scale < 1 || scale > 30 || draws < 0) return NULL;
    const int64_t n = (int64_t)1 << scale;
    gg_edge *e = (gg_edge *)malloc((size_t)(draws ? draws : 1) * sizeof(gg_edge));
    const int64_t CH = 1 << 16;
    const int64_t nch = (draws + CH - 1) / CH;
    int64_t selfd = 0;
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : selfd)
    for (int64_t ch = 0; ch < nch; ++ch) {
        xo256 r;
        xo_seed(&r, seed, (uint64_t)ch);
        for (int64_t d = ch * CH; d < (ch + 1) * CH && d < draws; ++d) {
            uint32_t u = 0, v = 0;
            for (int l = 0; l < scale; ++l) {
                /* quadrant a = (0,0), b = (0,1), c = (1,0), d = (1,1) */
                const double x = xo_unif(&r);
                const uint32_t bu = x >= ab;
                const uint32_t bv = (uint32_t)((x >= a) & (x < ab)) | (uint32_t)(x >= abc);
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            if (u == v) { e[d].u = -1; e[d].v = -1; e[d].w = 0; selfd++; continue; }
            e[d].u = (int32_t)(u < v ? u : v);
            e[d].v = (int32_t)(u < v ? v : u);
            e[d].w = 1;
        }
    }
    gg_graph *g = build_csr(n, e, draws, MERGE_SUM);
    if (g) { g->draws = draws; g->self_draws = selfd; }
    free(e);
    return g;
}

/* -------------------------------------------------------------- Chung-Lu */
/* Vose alias table over nonnegative weights x[0..k). */
typedef struct { double *prob; int32_t *alias; int64_t k; } alias_t;
static void alias_build(alias_t *t, const double *x, int64_t k) {
    t->k = k;
    t->prob = (double *)malloc((size_t)k * sizeof(double));
    t->alias = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    double sum = 0.0;
    for (int64_t i = 0; i < k; ++i) sum += x[i];
    int32_t *small = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    int32_t *large = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < k; ++i) {
        t->prob[i] = x[i] * (double)k / sum;
        if (t->prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns], l = large[--nl];
        t->alias[s] = l;
        t->prob[l] = (t->prob[l] + t->prob[s]) - 1.0;
        if (t->prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int32_t l = large[--nl]; t->prob[l] = 1.0; t->alias[l] = l; }
    while (ns > 0) { int32_t s = small[--ns]; t->prob[s] = 1.0; t->alias[s] = s; }
    free(small);
    free(large);
}
static inline int32_t alias_draw(const alias_t *t, xo256 *r) {
    int32_t i = (int32_t)xo_below(r, (uint64_t)t->k);
    return (xo_unif(r) < t->prob[i]) ? i : t->alias[i];
}

/* approximate sum_{i<N} (i + i0)^-beta by the midpoint integral */
static double zsum(double N, double i0, double beta) {
    double e = 1.0 - beta;
    return (pow(N - 0.5 + i0, e) - pow(i0 - 0.5, e)) / e;
}

/* n vertices: floor(core_frac * n) core vertices carry weights
 * x_i = (i + i0)^(-1/(gamma-1)), i0 chosen so the heaviest core vertex has
 * expected degree about dmax.  `edges` undirected edges are targeted in
 * total: one per pendant vertex (joined to a core vertex drawn in
 * proportion to x) and the rest as core-core draws with both ends drawn in
 * proportion to x.  Self draws and duplicate core edges are dropped (weight
 * 1).  Vertex ids are finally shuffled by a seeded random permutation so
 * hubs and pendant vertices are spread over the id range. */
gg_graph *gg_chunglu(int64_t n, double gamma, double core_frac, int64_t edges, double dmax,
                     uint64_t seed) {
    if (n < 4 || gamma <= 1.0 || core_frac <= 0.0 || core_frac > 1.0) return NULL;
    const int64_t ncore = (int64_t)floor(core_frac * (double)n);
    const int64_t npend = n - ncore;
    int64_t D = edges - npend;
    if (D < 0) D = 0;
    const double beta = 1.0 / (gamma - 1.0);
    /* bisection on i0: expected degree of vertex 0 = 2D i0^-beta / X(i0) */
    double lo = 0.75, hi = (double)ncore * 4.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double d0 = 2.0 * (double)D * pow(mid, -beta) / zsum((double)ncore, mid, beta);
        if (d0 > dmax) lo = mid; else hi = mid;
    }
    const double i0 = 0.5 * (lo + hi);
    double *x = (double *)malloc((size_t)ncore * sizeof(double));
    for (int64_t i = 0; i < ncore; ++i) x[i] = pow((double)i + i0, -beta);
    alias_t at;
    alias_build(&at, x, ncore);
    free(x);

    const int64_t ne = D + npend;
    gg_edge *e = (gg_edge *)malloc((size_t)(ne ? ne : 1) * sizeof(gg_edge));
    const int64_t CH = 1 << 16;
    const int64_t nch = (ne + CH - 1) / CH;
    int64_t selfd = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : selfd)
    for (int64_t ch = 0; ch < nch; ++ch) {
        xo256 r;
        xo_seed(&r, seed, (uint64_t)ch);
        for (int64_t d = ch * CH; d < (ch + 1) * CH && d < ne; ++d) {
            if (d < D) {
                int32_t u = alias_draw(&at, &r), v = alias_draw(&at, &r);
                if (u == v) { e[d].u = -1; e[d].v = -1; e[d].w = 0; selfd++; continue; }
                e[d].u = u < v ? u : v;
                e[d].v = u < v ? v : u;
            } else {
                int32_t p = (int32_t)(ncore + (d - D));
                int32_t t = alias_draw(&at, &r);
                e[d].u = t;
                e[d].v = p;
            }
            e[d].w = 1;
        }
    }
    free(at.prob);
    free(at.alias);
    /* seeded permutation of vertex ids (Fisher-Yates, one stream) */
    int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    {
        xo256 r;
        xo_seed(&r, seed, 0xFFFFFFFFFFFFULL);
        for (int64_t i = n - 1; i > 0; --i) {
            int64_t j = (int64_t)xo_below(&r, (uint64_t)(i + 1));
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t d = 0; d < ne; ++d) {
        if (e[d].u < 0) continue;
        e[d].u = perm[e[d].u];
        e[d].v = perm[e[d].v];
    }
    free(perm);
    gg_graph *g = build_csr(n, e, ne, MERGE_MAX);
    if (g) { g->draws = ne; g->self_draws = selfd; }
    free(e);
    return g;
}
