// lv_sweep.cu -- the vertex sweep of one iteration (Algorithm 1, Sec. 4.1).
//
// For every vertex i of a colour class (or of the whole graph):
//   e[c]   = sum of w(i,j) over neighbours j != i with C(j) = c     (Eq. 1)
//   s(c)   = 2m e[c] - k_i a_c                                        (Eq. 4 x (2m)^2/2)
//   s_old  = 2m e[C(i)] - k_i (a_{C(i)} - k_i)
//   best   = argmax over c != C(i) of s(c), ties to the smaller label (Eq. 5)
//   move   iff s(best) - s_old > 0 and not (|C(i)| = |best| = 1 and best > C(i))
// All products are below 2^62 (2m < 2^31), so int64 holds them exactly and
// every decision is exact.  All vertices of a class decide from the state at
// the start of the class.
//
// One cooperative launch sweeps every class of an iteration.  Per class:
//   stage A  block items: hub arc chunks (global tables) and CTA-bin vertices
//            (shared-memory table); warp items: 32/G vertices of G lanes each,
//            G = 1..32 chosen per vertex so each lane holds a few arcs.  In a
//            coloured sweep whose hub chunks each get a block, a hub's chunk
//            blocks wait for one another (bounded), evaluate the table slots
//            each claimed, and the last to finish decides the hub's move
//   [otherwise, with hubs: barrier, stage B: per hub, blocks evaluate chunks
//    of its occupied slots; the last one to finish combines them and decides]
//   barrier
// Coloured phases keep the community state {a_C, |C|} in two buffers.  Class
// g reads X[g % 2] and writes X[(g + 1) % 2], which before class g holds the
// state of class g - 1's start: class g replays class g - 1's moves into it
// and its own movers add their deltas there directly.  Labels are updated in
// place (a class is an independent set, so no vertex of the class reads the
// label of another).  One barrier per class suffices (two with hubs whose
// chunks outnumber the blocks).
// Uncoloured phases sweep the whole graph from X[0] and leave the moves in a
// list for the host (the stopping test decides whether they are applied).
//
// Labels and community state change between classes, so they are read with
// L2-only loads (L1 is not coherent across SMs); the graph is read normally.
// Every loop keeps up to 4 independent loads in flight per thread.
//
// Hash tables are open-addressing (linear probing) keyed by community label
// and sized to the next power of two >= 2 * degree (4 * degree for hubs in
// coloured sweeps), so the load factor is <= 1/2 and every probe sequence ends; a probe count above the table size is
// an internal error (LV_ERR_HASH), never a hang.  Grid barriers wait a bounded
// time and report LV_ERR_TIMEOUT.
#include <algorithm>
#include <climits>

#include "lv_ops.cuh"

namespace lv {
namespace {

constexpr int kSwBlock = 512;
constexpr int kSwWarps = kSwBlock / 32;
// Dynamic shared memory: every table key lives in the first half, every
// value in the second, whatever the item kind (warp w's group tables use keys
// [w*kGroupTableInts, (w+1)*kGroupTableInts) and the same range of values; a
// CTA-bin vertex or a hub chunk uses the block's whole key and value halves).
// The halves are cleared once at kernel start, and every item leaves the
// slots it used empty again (key kEmpty, value 0) before the next item, so no
// item clears or scans a table it did not fill.
constexpr int kSwSmemInts = 2 * kCtaSlots;
constexpr int kU = 4;                                  // loads in flight per thread
constexpr int kCtaArcs = kCtaMaxLimit / kSwBlock;      // arcs per thread of a CTA-bin vertex
constexpr int kQuadThreads = kSwBlock / 4;             // a quarter CTA: 4 warps
constexpr int kQuadArcs = kQuadMaxArcs / kQuadThreads; // arcs per thread of a quarter-CTA vertex
constexpr int kQuadSlots = kCtaSlots / 4;              // its table: 2x the arcs
static_assert(kQuadSlots >= 2 * kQuadMaxArcs, "quarter-CTA table must fit");
static_assert(kSwWarps * kGroupTableInts == kCtaSlots, "warp tables tile the key half");
static_assert(2 * kWarpMaxLimit <= kGroupTableInts, "warp table must fit");
static_assert(kCtaArcs * kSwBlock == kCtaMaxLimit, "CTA-bin arcs split evenly");

struct HubPart {
    long long s;
    int c, z, e, eo;
};

struct Sweep {
    const int32_t *__restrict__ off;
    const int2 *__restrict__ arcs;
    const int32_t *__restrict__ k;
    const int32_t *__restrict__ loop;
    int32_t *C;
    unsigned long long *comm0, *comm1;
    int4 *moves0, *moves1;
    // [0, n_act): moves per class; [n_act, 2 n_act): block-item counters;
    // [2 n_act, 3 n_act): warp-item counters; [3 n_act]: moves of the last
    // class of the previous launch
    int32_t *move_count;
    IterStats *stats;
    const int32_t *__restrict__ order;
    const int32_t *__restrict__ bucket_off;
    const int32_t *__restrict__ chunk_at;
    int2 *hub_table;
    const int32_t *__restrict__ hub_off;
    int32_t *hub_occ;
    int32_t *hub_cnt;
    const int32_t *__restrict__ hub_chunk_off;
    HubPart *hub_part;
    int32_t *hub_done;
    const int32_t *__restrict__ act;  // active classes (colour indexes)
    int n_act;
    long long g0;  // classes swept in this phase before this launch
    int coloured;
    int hub_factor;  // hub table slots per arc (next power of two)
    const uint8_t *__restrict__ hub_shift;  // per class: hub arc chunk = kHubChunk << shift
    int n;
    long long two_m;
    GridBarrier *bar;
    TraceBuf tb;
    // batched runs (disjoint union of graphs); gid == nullptr otherwise
    const int32_t *__restrict__ gid;       // graph of each vertex
    const long long *__restrict__ two_m_g; // 2m of each graph
    const uint8_t *__restrict__ active_g;  // graphs still iterating
    unsigned long long *g_ein;             // per graph: sum of e_{i->C(i)} incl. loops
    unsigned long long *g_a2;              // per graph: sum of a_C^2
    unsigned long long *g_moved;           // per graph: moves
};

// 2m of the graph holding vertex i
__device__ __forceinline__ long long tm_of(const Sweep &s, int i) {
    return s.gid ? s.two_m_g[s.gid[i]] : s.two_m;
}
// false for vertices of batched graphs that stopped iterating
__device__ __forceinline__ bool live(const Sweep &s, int i) {
    return !s.gid || s.active_g[s.gid[i]];
}
// modularity terms of one decided vertex, for block items
__device__ __forceinline__ void add_terms(const Sweep &s, struct Acc &acc, int i, int ein, bool mv);

// per-class view: read buffer, write buffer, move list and its counter
struct Cls {
    const unsigned long long *xr;
    unsigned long long *xw;
    int4 *mw;
    int32_t *cnt;
    int coloured;
};

struct Acc {
    long long ein = 0, dein = 0;
    int moved = 0, err = 0;
};

__device__ __forceinline__ void add_terms(const Sweep &s, Acc &acc, int i, int ein, bool mv) {
    if (s.gid) {
        const int g = s.gid[i];
        if (ein) atomicAdd(&s.g_ein[g], (unsigned long long)ein);
        if (mv) atomicAdd(&s.g_moved[g], 1ull);
    } else {
        acc.ein += ein;
        acc.moved += mv ? 1 : 0;
    }
}

__device__ __forceinline__ int ldC(const Sweep &s, int j) { return __ldcg(&s.C[j]); }

__device__ __forceinline__ int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// insert (c, w) into a shared-memory table of `mask + 1` slots whose slot h
// lives at key[h * ST] / val[h * ST] (ST = 32 interleaves one table per lane
// so that the lanes of a warp never collide on a bank)
template <int ST>
__device__ __forceinline__ bool smem_insert(int *key, int *val, unsigned mask, int c, int w) {
    unsigned h = hash32(c) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int cur = ((volatile int *)key)[h * ST];
        if (cur == c) {
            atomicAdd(&val[h * ST], w);
            return true;
        }
        if (cur == kEmpty) {
            const int prev = atomicCAS(&key[h * ST], kEmpty, c);
            if (prev == kEmpty || prev == c) {
                atomicAdd(&val[h * ST], w);
                return true;
            }
        }
        h = (h + 1) & mask;
    }
    return false;
}

// as smem_insert, but every probe is a compare-and-swap (no read first: a
// shared-memory CAS costs about a load, and one branch level less measured
// +18% on the batched sweep); `own` receives the slot when this call
// created the key (exactly one inserter creates each distinct label's
// slot), else -1
template <int ST>
__device__ __forceinline__ bool smem_insert_own(int *key, int *val, unsigned mask, int c, int w,
                                                int &own) {
    unsigned h = hash32(c) & mask;
    own = -1;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int prev = atomicCAS(&key[h * ST], kEmpty, c);
        if (prev == kEmpty || prev == c) {
            if (prev == kEmpty) own = (int)h;
            atomicAdd(&val[h * ST], w);
            return true;
        }
        h = (h + 1) & mask;
    }
    return false;
}

// Per-thread arcs of one vertex: up to NA arcs e = first + u * step < end,
// all loads and label gathers in flight at once, inserted into a
// shared-memory table; own[u] is the slot arc u's label created (or -1).
// After the table is complete (a barrier), owner_eval evaluates each owned
// slot -- every distinct label exactly once over the threads -- with all its
// community gathers in flight, and clears the slot.
template <int ST, int NA>
__device__ __forceinline__ void insert_owned(const Sweep &s, int i, int first, int end, int step,
                                             int *key, int *val, unsigned mask, int (&own)[NA],
                                             Acc &acc) {
    int2 a[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
        const int e = first + u * step;
        a[u] = e < end ? s.arcs[e] : make_int2(i, 0);
    }
#pragma unroll
    for (int u = 0; u < NA; ++u) a[u].x = a[u].x != i ? ldC(s, a[u].x) : kEmpty;
#pragma unroll
    for (int u = 0; u < NA; ++u) {
        own[u] = -1;
        if (a[u].x != kEmpty && !smem_insert_own<ST>(key, val, mask, a[u].x, a[u].y, own[u]))
            acc.err = 1;
    }
}

// insert the arcs e = first, first + step, ... < end of vertex i into a
// shared-memory table, U arcs (and their label gathers) at a time
template <int ST, int U = kU>
__device__ __forceinline__ void insert_arcs(const Sweep &s, int i, int first, int end, int step,
                                            int *key, int *val, unsigned mask, Acc &acc) {
    for (int e0 = first; e0 < end; e0 += U * step) {
        int2 a[U];
        int c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * step;
            a[u] = e < end ? s.arcs[e] : make_int2(i, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = a[u].x != i ? ldC(s, a[u].x) : kEmpty;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c[u] != kEmpty && !smem_insert<ST>(key, val, mask, c[u], a[u].y)) acc.err = 1;
    }
}

// best candidate so far: maximum s, then minimum label
struct Best {
    long long s;
    int c;
    int size;
    int e;
};
__device__ __forceinline__ void best_init(Best &b) {
    b.s = LLONG_MIN;
    b.c = INT_MAX;
    b.size = 0;
    b.e = 0;
}
__device__ __forceinline__ void best_take(Best &b, long long s, int c, int size, int e) {
    if (s > b.s || (s == b.s && c < b.c)) {
        b.s = s;
        b.c = c;
        b.size = size;
        b.e = e;
    }
}
__device__ __forceinline__ void best_shfl_xor(Best &b, int o) {
    const long long s = __shfl_xor_sync(0xffffffffu, b.s, o);
    const int c = __shfl_xor_sync(0xffffffffu, b.c, o);
    const int z = __shfl_xor_sync(0xffffffffu, b.size, o);
    const int e = __shfl_xor_sync(0xffffffffu, b.e, o);
    best_take(b, s, c, z, e);
}

// evaluate (and clear) the table slots this thread created (own[u] >= 0):
// the label is read back from the slot, the weight to the vertex's own
// community goes to e_old (its slot has exactly one owner)
template <int ST, int NA>
__device__ __forceinline__ void owner_eval(const Cls &cc, int *key, int *val, const int (&own)[NA],
                                           int ci, int ki, long long tm, Best &b, int &e_old) {
    int lab[NA];
    unsigned long long cm[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) lab[u] = own[u] >= 0 ? key[own[u] * ST] : kEmpty;
#pragma unroll
    for (int u = 0; u < NA; ++u)
        cm[u] = (lab[u] != kEmpty && lab[u] != ci) ? __ldcg(&cc.xr[lab[u]]) : 0ull;
#pragma unroll
    for (int u = 0; u < NA; ++u) {
        if (lab[u] == kEmpty) continue;
        const int v = val[own[u] * ST];
        key[own[u] * ST] = kEmpty;
        val[own[u] * ST] = 0;
        if (lab[u] == ci) {
            e_old = v;
            continue;
        }
        best_take(b, tm * (long long)v - (long long)ki * comm_a(cm[u]), lab[u], comm_size(cm[u]), v);
    }
}

// decision for vertex i given the reduced candidate; true on a move.  ein
// receives e_{i->C(i)} including the self-loop (the vertex's modularity term).
// cmi = the vertex's own community state and lp its self-loop, loaded by the
// caller together with its other per-vertex data (one round trip less).
__device__ __forceinline__ bool decide(int ci, int ki, unsigned long long cmi, int lp, long long tm,
                                       const Best &b, int e_old, Acc &acc, int &ein) {
    const long long s_old = tm * (long long)e_old - (long long)ki * (comm_a(cmi) - ki);
    ein = e_old + lp;
    if (b.c == INT_MAX) return false;
    if (b.s - s_old <= 0) return false;
    if (comm_size(cmi) == 1 && b.size == 1 && b.c > ci) return false;  // singlet rule
    acc.dein += 2ll * ((long long)b.e - e_old);
    return true;
}

// record a decided move at list position pos; coloured phases apply it now
// (label in place, community deltas into the write buffer)
__device__ __forceinline__ void commit(const Sweep &s, const Cls &cc, int pos, int i, int ci,
                                       int nc, int ki) {
    cc.mw[pos] = make_int4(i, ci, nc, ki);
    if (cc.coloured) {
        __stcg(&s.C[i], nc);
        atomicAdd(&cc.xw[ci], comm_leave(ki));
        atomicAdd(&cc.xw[nc], comm_join(ki));
    }
}

// block-wide reduction of (Best, e_old) over kSwWarps warps; result in thread 0
struct BlockRed {
    long long s[kSwWarps];
    int c[kSwWarps], z[kSwWarps], e[kSwWarps], eo[kSwWarps];
};
__device__ __forceinline__ void block_best(Best &b, int &e_old, BlockRed &r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_old += __shfl_xor_sync(0xffffffffu, e_old, o);
        best_shfl_xor(b, o);
    }
    if (lane == 0) {
        r.s[w] = b.s;
        r.c[w] = b.c;
        r.z[w] = b.size;
        r.e[w] = b.e;
        r.eo[w] = e_old;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        best_init(b);
        e_old = 0;
        for (int q = 0; q < kSwWarps; ++q) {
            best_take(b, r.s[q], r.c[q], r.z[q], r.e[q]);
            e_old += r.eo[q];
        }
    }
}

// ------------------------------------------------ group items (1..32 lanes)
// One warp sweeps 32/G vertices verts[base + lane/G] with G lanes each.  The
// NG = 32/G tables of a warp are interleaved (slot s of group q at s*NG + q),
// so the lanes of a warp clear and probe distinct banks.
template <int G>
__device__ void warp_group_sweep(const Sweep &s, const Cls &cc, const int32_t *verts, int nverts,
                                 int base, int *kreg, int *vreg, Acc &acc) {
    constexpr int NG = 32 / G;
    constexpr int ST = NG;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    int *key = kreg + lane / G;
    int *val = vreg + lane / G;
    const unsigned lt = (1u << lane) - 1u;
    const int vi = base + lane / G;
    bool valid = vi < nverts;
    int i = 0, beg = 0, end = 0, ci = 0, ki = 0, lp = 0;
    long long tm = 0;
    unsigned long long cmi = 0;
    unsigned mask = 0;
    if (valid) {
        i = verts[vi];
        valid = live(s, i);
    }
    if (valid) {
        tm = tm_of(s, i);
        beg = s.off[i];
        end = s.off[i + 1];
        ci = ldC(s, i);
        ki = s.k[i];
        if (gl == 0) {
            lp = s.loop[i];
            cmi = __ldcg(&cc.xr[ci]);
        }
        const int h = pow2_at_least(2 * (end - beg));
        mask = (unsigned)((h < 4 ? 4 : h) - 1);
        if (end - beg > G * kLaneArcsLimit) {  // bins never give a group more
            acc.err = 1;
            end = beg;
        }
    }
    // all of a lane's arcs (at most kLaneArcsLimit) and labels in flight at once
    int own[kLaneArcsLimit];
    insert_owned<ST, kLaneArcsLimit>(s, i, beg + gl, end, G, key, val, mask, own, acc);
    __syncwarp();
    Best b;
    best_init(b);
    int e_old = 0;
    owner_eval<ST, kLaneArcsLimit>(cc, key, val, own, ci, ki, tm, b, e_old);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        e_old += __shfl_xor_sync(0xffffffffu, e_old, o);
        best_shfl_xor(b, o);
    }
    bool mv = false;
    int ein = 0;
    const bool leader = valid && gl == 0;
    if (leader) mv = decide(ci, ki, cmi, lp, tm, b, e_old, acc, ein);
    const unsigned bm = __ballot_sync(0xffffffffu, mv);
    if (bm) {
        int pos = 0;
        if (lane == 0) pos = atomicAdd(cc.cnt, __popc(bm));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (mv) commit(s, cc, pos + __popc(bm & lt), i, ci, b.c, ki);
    }
    if (s.gid) {
        // per-graph terms, merged over the warp's leaders of one graph; their
        // ein sum is at most that graph's 2m < 2^31, so it fits 32 bits
        const int g = leader ? s.gid[i] : -1 - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, g);
        const unsigned se = __reduce_add_sync(peers, (unsigned)ein);
        const int nm = __popc(peers & bm);
        if (leader && lane == __ffs(peers) - 1) {
            if (se) atomicAdd(&s.g_ein[g], (unsigned long long)se);
            if (nm) atomicAdd(&s.g_moved[g], (unsigned long long)nm);
        }
    } else if (leader) {
        acc.ein += ein;
        acc.moved += mv ? 1 : 0;
    }
    __syncwarp();  // every owned slot is clear before the next item inserts
}

// ------------------------------------------------------------ block items
// CTA-bin vertex: the whole block, table in shared memory.
__device__ void block_vertex_sweep(const Sweep &s, const Cls &cc, int i, int *dyn, BlockRed &red,
                                   Acc &acc) {
    if (!live(s, i)) return;  // block-uniform
    const long long tm = tm_of(s, i);
    const int beg = s.off[i];
    int end = s.off[i + 1];
    const int ci = ldC(s, i), ki = s.k[i];
    unsigned long long cmi = 0;
    int lp = 0;
    if (threadIdx.x == 0) {
        cmi = __ldcg(&cc.xr[ci]);
        lp = s.loop[i];
    }
    const unsigned mask = (unsigned)pow2_at_least(2 * (end - beg)) - 1u;
    if (end - beg > kCtaMaxLimit) {  // bins never give a CTA more (block-uniform)
        acc.err = 1;
        end = beg;
    }
    int *key = dyn;
    int *val = dyn + kCtaSlots;
    int own[kCtaArcs];
    insert_owned<1, kCtaArcs>(s, i, beg + threadIdx.x, end, kSwBlock, key, val, mask, own, acc);
    __syncthreads();
    Best b;
    best_init(b);
    int e_old = 0;
    owner_eval<1, kCtaArcs>(cc, key, val, own, ci, ki, tm, b, e_old);
    block_best(b, e_old, red);
    if (threadIdx.x == 0) {
        int ein = 0;
        const bool mv = decide(ci, ki, cmi, lp, tm, b, e_old, acc, ein);
        if (mv) commit(s, cc, atomicAdd(cc.cnt, 1), i, ci, b.c, ki);
        add_terms(s, acc, i, ein, mv);
    }
    __syncthreads();
}

// Quarter-CTA vertices (warp_max < arcs <= 1,024): four per block item, each
// swept by 4 warps with its own quarter of the shared-memory table and a
// named barrier of its own, so a block has four vertices in flight instead
// of one.  Group-uniform control flow: every thread of a group reaches its
// barriers.
__device__ __forceinline__ void quad_sync(int grp) {
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(kQuadThreads) : "memory");
}
__device__ void quad_vertex_sweep(const Sweep &s, const Cls &cc, const int32_t *verts, int nq,
                                  int qi, int *dyn, BlockRed &red, Acc &acc) {
    const int grp = threadIdx.x / kQuadThreads, t = threadIdx.x % kQuadThreads;
    const int lane = threadIdx.x & 31, wig = t >> 5;
    const int vi = qi * 4 + grp;
    bool valid = vi < nq;
    int i = 0;
    if (valid) {
        i = verts[vi];
        valid = live(s, i);
    }
    int beg = 0, end = 0, ci = 0, ki = 0, lp = 0;
    long long tm = 0;
    unsigned long long cmi = 0;
    unsigned mask = 0;
    if (valid) {
        tm = tm_of(s, i);
        beg = s.off[i];
        end = s.off[i + 1];
        ci = ldC(s, i);
        ki = s.k[i];
        if (t == 0) {
            cmi = __ldcg(&cc.xr[ci]);
            lp = s.loop[i];
        }
        mask = (unsigned)pow2_at_least(2 * (end - beg)) - 1u;
        if (end - beg > kQuadMaxArcs) {  // bins never give a quarter CTA more
            acc.err = 1;
            end = beg;
        }
    }
    int *key = dyn + grp * kQuadSlots;
    int *val = dyn + kCtaSlots + grp * kQuadSlots;
    int own[kQuadArcs];
    insert_owned<1, kQuadArcs>(s, i, beg + t, end, kQuadThreads, key, val, mask, own, acc);
    quad_sync(grp);
    Best b;
    best_init(b);
    int e_old = 0;
    owner_eval<1, kQuadArcs>(cc, key, val, own, ci, ki, tm, b, e_old);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_old += __shfl_xor_sync(0xffffffffu, e_old, o);
        best_shfl_xor(b, o);
    }
    const int slot = grp * 4 + wig;
    if (lane == 0) {
        red.s[slot] = b.s;
        red.c[slot] = b.c;
        red.z[slot] = b.size;
        red.e[slot] = b.e;
        red.eo[slot] = e_old;
    }
    quad_sync(grp);
    if (t == 0 && valid) {
        best_init(b);
        e_old = 0;
        for (int q = grp * 4; q < grp * 4 + 4; ++q) {
            best_take(b, red.s[q], red.c[q], red.z[q], red.e[q]);
            e_old += red.eo[q];
        }
        int ein = 0;
        const bool mv = decide(ci, ki, cmi, lp, tm, b, e_old, acc, ein);
        if (mv) commit(s, cc, atomicAdd(cc.cnt, 1), i, ci, b.c, ki);
        add_terms(s, acc, i, ein, mv);
    }
}

// position of the hub owning arc chunk `chunk` in bucket [lo, lo + cnt)
__device__ __forceinline__ int hub_of_chunk(const Sweep &s, int lo, int cnt, int chunk) {
    const int32_t *co = s.hub_chunk_off + lo;  // co[cnt] > chunk >= co[0]
    int a = 0, b = cnt;
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (co[mid] <= chunk) a = mid; else b = mid;
    }
    return a;
}

// Hub arc chunk: CHS arcs of one hub (kHubChunk, or twice that in classes
// whose hubs have more chunks than the grid has blocks) are first summed per
// label in a
// shared-memory table of the block, then each distinct label is added to the
// hub's global table once (so a popular label costs one global atomic per
// chunk, not one per warp).  Global first probes are compare-and-swaps issued
// for all of a thread's labels at once; collisions fall back to linear
// probing.
//
// With `par` (every chunk of the class's hubs has a block of its own), the
// blocks of a hub then wait for all of its chunks (a bounded wait on the
// hub's arrival counter), each evaluates the slots it claimed (at most
// CHS, one pass) and stores a partial best, and the last to finish
// combines the partials and decides: no grid barrier, and the evaluation is
// spread over the hub's blocks.  Chunks are handed out before any other item
// of the class and a block holding one claims nothing else until it is done,
// so every block waited for is running.  Otherwise claimed slots are
// appended to the hub's occupied list (one counter update per warp) for the
// evaluation after a grid barrier.
constexpr int kHubWide = 2 * kHubChunk;  // the wider chunk
static_assert(2 * kHubWide <= kCtaSlots, "hub chunk table fits the key half");
__device__ void hub_combine(const Sweep &s, const Cls &cc, int p, int first, int nch, int i, int ci,
                            int ki, unsigned long long cmi, int lp, long long tm, BlockRed &red,
                            Acc &acc);
template <int CHS>
__device__ void hub_chunk(const Sweep &s, const Cls &cc, int lo, int cnt, int chunk, int *dyn,
                          BlockRed &red, Acc &acc, bool par) {
    constexpr int kHubSmemSlots = 2 * CHS;  // power of two, >= 2x the distinct labels
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31;
    const int a = hub_of_chunk(s, lo, cnt, chunk);
    const int p = lo + a;
    const int i = s.order[p];
    if (!live(s, i)) return;  // block-uniform
    const int beg = s.off[i], end = s.off[i + 1];
    const unsigned mask = (unsigned)pow2_at_least(s.hub_factor * (end - beg)) - 1u;
    int2 *tab = s.hub_table + s.hub_off[p];
    const int first = s.hub_chunk_off[p], nch = s.hub_chunk_off[p + 1] - first;
    // the hub's own terms, loaded ahead of the arcs (used after the wait)
    const long long tm = tm_of(s, i);
    const int ci = ldC(s, i), ki = s.k[i], lp = s.loop[i];
    const unsigned long long cmi = __ldcg(&cc.xr[ci]);
    const int start = beg + (chunk - first) * CHS;
    const int stop = min(end, start + CHS);
    int *key = dyn, *val = dyn + kCtaSlots;  // both empty on entry
    insert_arcs<1>(s, i, start + threadIdx.x, stop, kSwBlock, key, val, kHubSmemSlots - 1, acc);
    __syncthreads();
    constexpr int kHubPer = kHubSmemSlots / kSwBlock;  // table slots per thread
    static_assert(kHubPer * kSwBlock == kHubSmemSlots, "one pass over the chunk's table");
    int claimed[kHubPer];
    {
        int cl[kHubPer], sum[kHubPer];
        unsigned hslot[kHubPer];
        int prev[kHubPer];
#pragma unroll
        for (int u = 0; u < kHubPer; ++u) {
            cl[u] = key[threadIdx.x + u * kSwBlock];
            sum[u] = val[threadIdx.x + u * kSwBlock];
            key[threadIdx.x + u * kSwBlock] = kEmpty;  // each thread clears the slots it read
            val[threadIdx.x + u * kSwBlock] = 0;
            hslot[u] = hash32(cl[u]) & mask;
            prev[u] = cl[u] != kEmpty ? atomicCAS(&tab[hslot[u]].x, kEmpty, cl[u]) : 0;
        }
#pragma unroll
        for (int u = 0; u < kHubPer; ++u) {
            claimed[u] = -1;
            if (cl[u] == kEmpty) continue;
            const int c = cl[u];
            unsigned h = hslot[u];
            bool done = prev[u] == kEmpty || prev[u] == c;
            if (prev[u] == kEmpty) claimed[u] = (int)h;
            for (unsigned probe = 1; probe <= mask && !done; ++probe) {
                h = (h + 1) & mask;
                const int pv = atomicCAS(&tab[h].x, kEmpty, c);
                if (pv == kEmpty) claimed[u] = (int)h;
                done = pv == kEmpty || pv == c;
            }
            if (done) atomicAdd(&tab[h].y, sum[u]);
            else acc.err = 1;
        }
    }
    if (!par) {  // one occupied-list reservation per warp for all its claims
        int32_t *occ = s.hub_occ + s.hub_off[p];
        int mine = 0;
#pragma unroll
        for (int u = 0; u < kHubPer; ++u) mine += claimed[u] >= 0 ? 1 : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            int base = 0;
            if (lane == 31) base = atomicAdd(s.hub_cnt + p, total);
            base = __shfl_sync(0xffffffffu, base, 31) + incl - mine;
#pragma unroll
            for (int u = 0; u < kHubPer; ++u)
                if (claimed[u] >= 0) __stcg(&occ[base++], claimed[u]);
        }
        return;
    }
    // wait until every chunk of the hub has added its labels
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add_i32(&s.hub_done[p], 1);
        int ok = 1;
        for (unsigned long long spins = 0; ld_acquire_i32(&s.hub_done[p]) < nch;) {
            if (++spins > kBarrierSpinLimit) {
                ok = 0;
                barrier_raise(s.bar, 1);
                break;
            }
            __nanosleep(20);
        }
        s_flag = ok;
    }
    __syncthreads();
    if (!s_flag) return;
    Best b;
    best_init(b);
    int e_old = 0;
    {
        int2 kv[kHubPer];
        unsigned long long cm[kHubPer];
#pragma unroll
        for (int u = 0; u < kHubPer; ++u) kv[u] = claimed[u] >= 0 ? __ldcg(&tab[claimed[u]]) : make_int2(kEmpty, 0);
#pragma unroll
        for (int u = 0; u < kHubPer; ++u) {
            if (claimed[u] >= 0) __stcg(&tab[claimed[u]], make_int2(kEmpty, 0));
            cm[u] = (kv[u].x != kEmpty && kv[u].x != ci) ? __ldcg(&cc.xr[kv[u].x]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kHubPer; ++u) {
            if (kv[u].x == kEmpty) continue;
            if (kv[u].x == ci) {
                e_old = kv[u].y;
                continue;
            }
            best_take(b, tm * (long long)kv[u].y - (long long)ki * comm_a(cm[u]), kv[u].x,
                      comm_size(cm[u]), kv[u].y);
        }
    }
    block_best(b, e_old, red);
    if (threadIdx.x == 0) {
        HubPart hp;
        hp.s = b.s;
        hp.c = b.c;
        hp.z = b.size;
        hp.e = b.e;
        hp.eo = e_old;
        s.hub_part[chunk] = hp;
        s_flag = atom_acq_rel_add_i32(&s.hub_done[p], 1) == 2 * nch - 1;
    }
    __syncthreads();
    if (s_flag)  // block-uniform: the last block combines the partials
        hub_combine(s, cc, p, first, nch, i, ci, ki, cmi, lp, tm, red, acc);
    __syncthreads();
}

// Evaluates (and resets) the hub table slots listed in occ[t0, t1): the best
// candidate and the weight to the hub's own community, per thread.
__device__ __forceinline__ void hub_eval(const Sweep &s, const Cls &cc, int2 *tab, const int32_t *occ,
                                         int t0, int t1, int ci, int ki, long long tm, Best &b,
                                         int &e_old) {
    for (int q0 = t0 + threadIdx.x; q0 < t1; q0 += kU * kSwBlock) {
        int hh[kU];
        int2 kv[kU];
        unsigned long long cm[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int q = q0 + u * kSwBlock;
            hh[u] = q < t1 ? __ldcg(&occ[q]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) kv[u] = hh[u] >= 0 ? __ldcg(&tab[hh[u]]) : make_int2(kEmpty, 0);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (hh[u] >= 0) __stcg(&tab[hh[u]], make_int2(kEmpty, 0));
            cm[u] = (kv[u].x != kEmpty && kv[u].x != ci) ? __ldcg(&cc.xr[kv[u].x]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (kv[u].x == kEmpty) continue;
            if (kv[u].x == ci) {
                e_old = kv[u].y;
                continue;
            }
            best_take(b, tm * (long long)kv[u].y - (long long)ki * comm_a(cm[u]), kv[u].x,
                      comm_size(cm[u]), kv[u].y);
        }
    }
}

// Combines the partial bests of a hub's nch chunks (its counter is reset)
// and decides the hub's move; the whole block takes part, thread 0 decides.
__device__ void hub_combine(const Sweep &s, const Cls &cc, int p, int first, int nch, int i, int ci,
                            int ki, unsigned long long cmi, int lp, long long tm, BlockRed &red,
                            Acc &acc) {
    Best t;
    best_init(t);
    int eo = 0;
    for (int q = first + threadIdx.x; q < first + nch; q += kSwBlock) {
        const HubPart *hq = &s.hub_part[q];
        best_take(t, __ldcg(&hq->s), __ldcg(&hq->c), __ldcg(&hq->z), __ldcg(&hq->e));
        eo += __ldcg(&hq->eo);
    }
    block_best(t, eo, red);
    if (threadIdx.x == 0) {
        __stcg(&s.hub_done[p], 0);
        int ein = 0;
        const bool mv = decide(ci, ki, cmi, lp, tm, t, eo, acc, ein);
        if (mv) commit(s, cc, atomicAdd(cc.cnt, 1), i, ci, t.c, ki);
        add_terms(s, acc, i, ein, mv);
    }
}

// Hub decision, one block per chunk of the occupied list: evaluates its
// slots (resetting them to empty) and stores a partial best; the last block
// of the hub to finish (counted with a fenced atomic, no waiting) combines
// the partials and decides.
__device__ void hub_decide_chunk(const Sweep &s, const Cls &cc, int lo, int cnt, int chunk, int chs,
                                 BlockRed &red, Acc &acc) {
    __shared__ int s_last;
    const int a = hub_of_chunk(s, lo, cnt, chunk);
    const int p = lo + a;
    const int first = s.hub_chunk_off[p], nch = s.hub_chunk_off[p + 1] - first;
    const int i = s.order[p];
    if (!live(s, i)) return;  // block-uniform; its chunks inserted nothing
    const long long tm = tm_of(s, i);
    const int ci = ldC(s, i), ki = s.k[i];
    int2 *tab = s.hub_table + s.hub_off[p];
    const int32_t *occ = s.hub_occ + s.hub_off[p];
    const int n_occ = __ldcg(&s.hub_cnt[p]);
    const int t0 = (chunk - first) * chs, t1 = min(n_occ, t0 + chs);
    Best b;
    best_init(b);
    int e_old = 0;
    hub_eval(s, cc, tab, occ, t0, t1, ci, ki, tm, b, e_old);
    block_best(b, e_old, red);
    if (threadIdx.x == 0) {
        HubPart hp;
        hp.s = b.s;
        hp.c = b.c;
        hp.z = b.size;
        hp.e = b.e;
        hp.eo = e_old;
        s.hub_part[chunk] = hp;
        __threadfence();
        s_last = (atomicAdd(&s.hub_done[p], 1) == nch - 1);
    }
    __syncthreads();
    if (s_last) {  // block-uniform: the last block combines the partials in parallel
        __threadfence();
        if (threadIdx.x == 0) {
            __stcg(&s.hub_cnt[p], 0);
            atomicMax(&s.stats->max_occ, n_occ);
        }
        hub_combine(s, cc, p, first, nch, i, ci, ki, __ldcg(&cc.xr[ci]), s.loop[i], tm, red, acc);
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T block_sum_sw(T v, T *sm) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kSwWarps; ++q) r += sm[q];
    return r;
}

// ------------------------------------------------------------ the kernel
__global__ void __launch_bounds__(kSwBlock, 2) sweep_persistent_kernel(Sweep s) {
    extern __shared__ int dyn[];
    __shared__ BlockRed red;
    __shared__ long long sml[kSwWarps];
    __shared__ int s_item;
    Acc acc;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *kreg = dyn + wib * kGroupTableInts;
    int *vreg = dyn + kCtaSlots + wib * kGroupTableInts;
    for (int t = threadIdx.x; t < kCtaSlots; t += kSwBlock) {
        dyn[t] = kEmpty;
        dyn[kCtaSlots + t] = 0;
    }
    __syncthreads();
    const int gthread = blockIdx.x * kSwBlock + threadIdx.x;
    const int nthreads = gridDim.x * kSwBlock;
    unsigned bar_passed = 0;
    for (int q = 0; q < s.n_act; ++q) {
        const int c = s.act[q];
        const long long g = s.g0 + q;
        Cls cc;
        cc.coloured = s.coloured;
        cc.xr = s.coloured && (g & 1) ? s.comm1 : s.comm0;
        cc.xw = s.coloured && (g & 1) ? s.comm0 : s.comm1;
        cc.mw = s.coloured && (g & 1) ? s.moves1 : s.moves0;
        cc.cnt = s.move_count + q;
        if (LV_TRACE_ON && blockIdx.x == 0 && threadIdx.x == 0)
            trace4(s.tb, 0x600000000ull | (unsigned)q, (unsigned long long)g, gtimer(), 0);
        if (s.coloured) {
            // bring the write buffer up to date with the previous class's moves
            const int4 *mp = (g & 1) ? s.moves0 : s.moves1;
            const int np = __ldcg(&s.move_count[q == 0 ? 3 * s.n_act : q - 1]);
            for (int t = gthread; t < np; t += nthreads) {
                const int4 m = __ldcg(&mp[t]);
                atomicAdd(&cc.xw[m.y], comm_leave(m.w));
                atomicAdd(&cc.xw[m.z], comm_join(m.w));
            }
        }
        const int32_t *bo = s.bucket_off + c * (kBins + 1);
        const int b_quad = bo[kBinQuad];
        const int b_cta = bo[kBinCta], b_hub = bo[kBinHub], b_end = bo[kBins];
        const int n_quad = b_cta - b_quad, n_qitems = (n_quad + 3) >> 2;
        const int32_t *ca = s.chunk_at + c * (kBins + 1);
        const int chunk0 = ca[kBinHub], nchunks = ca[kBins] - ca[kBinHub];
        const int n_cta = b_hub - b_cta, n_hub = b_end - b_hub;
        const bool wide = s.hub_shift && s.hub_shift[c];
        // in coloured sweeps hubs are decided by their chunk blocks (no grid
        // barrier) when every chunk gets a block of its own; otherwise (and
        // in a one-class sweep, which has its barrier anyway) many blocks
        // evaluate them after a barrier
        const bool hub_par = s.coloured && n_hub > 0 && nchunks <= (int)gridDim.x;
        // block items, handed out by a class counter (the next index is
        // fetched while the current item runs)
        const int n_bitems = nchunks + n_cta + n_qitems;
        if (n_bitems > 0) {
            int32_t *bctr = s.move_count + s.n_act + q;
            if (threadIdx.x == 0) s_item = atomicAdd(bctr, 1);
            __syncthreads();
            int it = s_item;
            while (it < n_bitems) {
                // a block holding a chunk that waits for its hub claims
                // nothing else meanwhile
                const bool wait_item = hub_par && it < nchunks;
                int nxt = 0;
                if (threadIdx.x == 0 && !wait_item) nxt = atomicAdd(bctr, 1);
#ifdef LV_TRACE
                const unsigned long long ti0 = gtimer();
#endif
                if (it < nchunks) {
                    if (wide) hub_chunk<kHubWide>(s, cc, b_hub, n_hub, chunk0 + it, dyn, red, acc, hub_par);
                    else hub_chunk<kHubChunk>(s, cc, b_hub, n_hub, chunk0 + it, dyn, red, acc, hub_par);
                }
                else if (it < nchunks + n_cta)
                    block_vertex_sweep(s, cc, s.order[b_cta + it - nchunks], dyn, red, acc);
                else
                    quad_vertex_sweep(s, cc, s.order + b_quad, n_quad, it - nchunks - n_cta, dyn,
                                      red, acc);
                __syncthreads();
#ifdef LV_TRACE
                if (threadIdx.x == 0 && blockIdx.x < 64) {
                    const int vv =
                        it < nchunks || it >= nchunks + n_cta ? -1 : s.order[b_cta + it - nchunks];
                    const int dd = vv < 0 ? kHubChunk : s.off[vv + 1] - s.off[vv];
                    trace4(s.tb, 0x700000000ull | (unsigned)(it < nchunks ? 0 : 1),
                           (unsigned long long)g, (unsigned long long)dd, gtimer() - ti0);
                }
#endif
                if (threadIdx.x == 0) s_item = wait_item ? atomicAdd(bctr, 1) : nxt;
                __syncthreads();
                it = s_item;
            }
        }
        __syncthreads();
        // warp items: 32/G vertices of group bin log2(G), largest groups first
        int item_end[kGroupBins];
        {
            int acc_items = 0;
            for (int gb = kGroupBins - 1; gb >= 0; --gb) {
                acc_items += (bo[gb + 1] - bo[gb] + (32 >> gb) - 1) >> (5 - gb);
                item_end[gb] = acc_items;
            }
        }
        // items are claimed `claim` at a time (about 8 claims per warp), so
        // the class counter sees few atomics even with millions of items
        int32_t *wctr = s.move_count + 2 * s.n_act + q;
        const int claim = max(1, item_end[0] / (gridDim.x * kSwWarps * 8));
        if (LV_TRACE_ON && blockIdx.x == 0 && threadIdx.x == 0)
            trace4(s.tb, 0x900000000ull | (unsigned)q, (unsigned long long)g,
                   (unsigned long long)n_hub | ((unsigned long long)nchunks << 20) |
                       ((unsigned long long)hub_par << 40),
                   (unsigned long long)n_cta | ((unsigned long long)item_end[0] << 32));
        int it = 0;
        if (item_end[0] > 0) {
            if (lane == 0) it = atomicAdd(wctr, claim);
            it = __shfl_sync(0xffffffffu, it, 0);
        }
        while (it < item_end[0]) {
          int nxt = 0;
          if (lane == 0) nxt = atomicAdd(wctr, claim);
          const int it_stop = min(it + claim, item_end[0]);
          for (; it < it_stop; ++it) {
            int gb = kGroupBins - 1;
            while (it >= item_end[gb]) --gb;
            const int first = gb == kGroupBins - 1 ? 0 : item_end[gb + 1];
            const int lo = bo[gb], cnt = bo[gb + 1] - bo[gb];
            const int base = (it - first) << (5 - gb);
#ifdef LV_TRACE
            const unsigned long long tw0 = gtimer();
#endif
            switch (gb) {
            case 5: warp_group_sweep<32>(s, cc, s.order + lo, cnt, base, kreg, vreg, acc); break;
            case 4: warp_group_sweep<16>(s, cc, s.order + lo, cnt, base, kreg, vreg, acc); break;
            case 3: warp_group_sweep<8>(s, cc, s.order + lo, cnt, base, kreg, vreg, acc); break;
            case 2: warp_group_sweep<4>(s, cc, s.order + lo, cnt, base, kreg, vreg, acc); break;
            case 1: warp_group_sweep<2>(s, cc, s.order + lo, cnt, base, kreg, vreg, acc); break;
            default: warp_group_sweep<1>(s, cc, s.order + lo, cnt, base, kreg, vreg, acc); break;
            }
#ifdef LV_TRACE
            if (lane == 0 && blockIdx.x < 16)
                trace4(s.tb, 0x800000000ull | (unsigned)gb, (unsigned long long)g, 0, gtimer() - tw0);
#endif
          }
          it = __shfl_sync(0xffffffffu, nxt, 0);
        }
#ifdef LV_TRACE
        __syncthreads();
        if (threadIdx.x == 0 && g < (long long)(kTraceCap / 4))
            atomicMax(&s.tb.buf[kTraceCap / 2 + 2 * g], gtimer());
#endif
        if (n_hub > 0 && !hub_par) {
            if (!grid_sync(s.bar, bar_passed)) return;
            for (int it = blockIdx.x; it < nchunks; it += gridDim.x)
                hub_decide_chunk(s, cc, b_hub, n_hub, chunk0 + it, wide ? kHubWide : kHubChunk,
                                 red, acc);
#ifdef LV_TRACE
            __syncthreads();
#endif
        }
#ifdef LV_TRACE
        if (threadIdx.x == 0 && g < (long long)(kTraceCap / 4))
            atomicMax(&s.tb.buf[kTraceCap / 2 + 2 * g + 1], gtimer());
#endif
        if (s.coloured || q + 1 < s.n_act)
            if (!grid_sync(s.bar, bar_passed)) return;
    }
    if (s.coloured && blockIdx.x == 0 && threadIdx.x == 0 && s.n_act > 0)
        s.move_count[3 * s.n_act] = __ldcg(&s.move_count[s.n_act - 1]);  // carry for the next launch
    // sum of a_C^2 over all communities of the state the sweep leaves
    const unsigned long long *xf =
        s.coloured && ((s.g0 + s.n_act) & 1) ? s.comm1 : s.comm0;
    long long a2 = 0;
    if (s.gid) {  // per graph: communities of a graph are consecutive ids
        const int nr = (s.n + 31) & ~31;  // whole warps take part in the runs
        for (int c = gthread; c < nr; c += nthreads) {
            const bool in = c < s.n;
            const int g = in ? s.gid[c] : 0;
            const bool v = in && s.active_g[g];
            const long long x = v ? comm_a(__ldcg(&xf[c])) : 0;
            warp_run_add(g, (unsigned long long)(x * x), v, s.g_a2);
        }
    } else {
        for (int c = gthread; c < s.n; c += nthreads) {
            const long long x = comm_a(__ldcg(&xf[c]));
            a2 += x * x;
        }
    }
    const long long t_ein = block_sum_sw(acc.ein, sml);
    const long long t_dein = block_sum_sw(acc.dein, sml);
    const long long t_a2 = block_sum_sw(a2, sml);
    const long long t_mv = block_sum_sw((long long)acc.moved, sml);
    const long long t_err = block_sum_sw((long long)acc.err, sml);
    if (threadIdx.x == 0) {
        if (t_ein) atomicAdd(&s.stats->sum_ein, (unsigned long long)t_ein);
        if (t_dein) atomicAdd(&s.stats->delta_ein, (unsigned long long)t_dein);
        if (t_a2) atomicAdd(&s.stats->sum_a2, (unsigned long long)t_a2);
        if (t_mv) atomicAdd(&s.stats->moved, (int)t_mv);
        if (t_err) atomicOr(&s.stats->err, 1);
    }
}

// ------------------------------------------------------------ apply, init
// uncoloured phases: apply the listed moves (after the stopping test)
__global__ void apply_moves_kernel(int32_t *C, unsigned long long *comm,
                                   const int4 *__restrict__ moves,
                                   const int32_t *__restrict__ count) {
    const int cnt = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int4 m = moves[t];
        C[m.x] = m.z;
        atomicAdd(&comm[m.y], comm_leave(m.w));
        atomicAdd(&comm[m.z], comm_join(m.w));
    }
}

__global__ void __launch_bounds__(256) init_phase_kernel(int n, const int32_t *__restrict__ k,
                                                         const int32_t *__restrict__ loop,
                                                         int32_t *C, unsigned long long *comm0,
                                                         unsigned long long *comm1,
                                                         IterStats *stats) {
    __shared__ long long red[8];
    long long sl = 0, sk = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ki = k[i];
        C[i] = i;
        comm0[i] = comm_pack(ki, 1);
        if (comm1) comm1[i] = comm_pack(ki, 1);
        sl += loop[i];
        sk += (long long)ki * ki;
    }
    sl = block_sum_256(sl, red);
    sk = block_sum_256(sk, red);
    if (threadIdx.x == 0) {
        if (sl) atomicAdd(&stats->sum_ein, (unsigned long long)sl);
        if (sk) atomicAdd(&stats->sum_a2, (unsigned long long)sk);
    }
}

int g_sweep_blocks_per_sm = 0;

}  // namespace

lv_status sweep_setup() {
    const int smem = kSwSmemInts * (int)sizeof(int);
    LV_CUDA(cudaFuncSetAttribute(sweep_persistent_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_sweep_blocks_per_sm,
                                                          sweep_persistent_kernel, kSwBlock, smem));
    if (g_sweep_blocks_per_sm < 1) return LV_ERR_CUDA;
    return LV_OK;
}

size_t hub_part_bytes() { return sizeof(HubPart); }

int sweep_grid(const Buckets &b) {
    const int fit = g_sweep_blocks_per_sm > 0 ? g_sweep_blocks_per_sm : 1;
    const int bps = b.blocks_per_sm > 0 ? std::min(b.blocks_per_sm, fit) : fit;
    return (b.sms > 0 && b.sms < g_num_sms ? b.sms : g_num_sms) * bps;
}

lv_status init_phase(PhaseState &ps, cudaStream_t s) {
    LV_CUDA(cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s));
    LV_CUDA(cudaMemsetAsync(ps.move_count, 0, sizeof(int32_t) * (3 * (size_t)ps.n_act + 1), s));
    ps.g_total = 0;
    init_phase_kernel<<<grid_for(ps.g.n, 256, g_num_sms * 8), 256, 0, s>>>(
        ps.g.n, ps.k, ps.loop, ps.C, ps.comm[0], ps.coloured ? ps.comm[1] : nullptr, ps.stats);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status sweep_iteration(PhaseState &ps, const Buckets &b, cudaStream_t s) {
    Sweep a;
    a.off = ps.g.off;
    a.arcs = ps.g.arcs;
    a.k = ps.k;
    a.loop = ps.loop;
    a.C = ps.C;
    a.comm0 = ps.comm[0];
    a.comm1 = ps.comm[1];
    a.moves0 = ps.moves[0];
    a.moves1 = ps.moves[1];
    a.move_count = ps.move_count;
    a.stats = ps.stats;
    a.order = b.order;
    a.bucket_off = b.bucket_off;
    a.chunk_at = b.hub_chunk_at;
    a.hub_table = b.hub_table;
    a.hub_off = b.hub_off;
    a.hub_occ = b.hub_occ;
    a.hub_cnt = b.hub_cnt;
    a.hub_chunk_off = b.hub_chunk_off;
    a.hub_part = reinterpret_cast<HubPart *>(b.hub_part);
    a.hub_done = b.hub_done;
    a.act = ps.act;
    a.n_act = ps.n_act;
    a.g0 = ps.g_total;
    a.coloured = ps.coloured ? 1 : 0;
    a.hub_factor = b.hub_factor;
    a.hub_shift = b.hub_shift;
    a.n = ps.g.n;
    a.two_m = ps.two_m;
    a.bar = ps.bar;
    a.tb = trace_buffer();
    a.gid = ps.gid;
    a.two_m_g = ps.two_m_g;
    a.active_g = ps.active_g;
    a.g_ein = ps.g_ein;
    a.g_a2 = ps.g_a2;
    a.g_moved = ps.g_moved;
    // cooperative launch (all blocks co-resident, as the grid barrier needs);
    // the launch-attribute form is also valid inside a stream capture
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sweep_grid(b));
    cfg.blockDim = dim3(kSwBlock);
    cfg.dynamicSmemBytes = kSwSmemInts * sizeof(int);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LV_CUDA(cudaLaunchKernelEx(&cfg, sweep_persistent_kernel, a));
    LV_LAUNCH_CHECK();
    if (ps.coloured) ps.g_total += ps.n_act;
    return LV_OK;
}

unsigned long long *current_comm(const PhaseState &ps) {
    return ps.coloured ? ps.comm[ps.g_total & 1] : ps.comm[0];
}

lv_status apply_moves(PhaseState &ps, cudaStream_t s) {
    apply_moves_kernel<<<g_num_sms * 4, 256, 0, s>>>(ps.C, ps.comm[0], ps.moves[0], ps.move_count);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

}  // namespace lv
