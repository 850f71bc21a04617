// lv_color.cu -- distance-1 colouring (Sec. 4.2) and the per-phase vertex order.
//
// Colouring: Jones-Plassmann with the priority pi(v) = (d(v), h(v ^ seed), v)
// -- d(v) the neighbours of v other than v, largest first, then a hash -- or
// (h(v ^ seed), v) alone.  A first pass marks, per arc, whether the
// neighbour has the higher priority (one bit per arc, read beside the arc in
// every round).  Every vertex counts its higher-priority neighbours; a vertex whose count
// reaches zero takes the smallest colour not used by those neighbours, then
// decrements the counts of its lower-priority neighbours.  The result equals
// greedy colouring in decreasing priority order, whatever the timing, because
// a vertex's colour depends only on its higher-priority neighbours' colours.
// On power-law graphs the priority DAG is deep (1,500 to 3,500 levels on the
// R-MAT and Chung-Lu inputs), and almost all of its depth lies among the
// largest vertices.  With the degree first in the priority, the vertices of
// degree >= T form a prefix of the priority order (their higher-priority
// neighbours are all among them): this core is coloured first without rounds
// (sorted by priority, each vertex waiting for its earlier neighbours; the
// top of it on one thread-block cluster with the colours in distributed
// shared memory, the rest on the grid), and the other vertices in rounds,
// all inside one cooperative launch separated by a bounded grid barrier
// (about 20-30 rounds on those inputs).  Ready vertices are handled by size:
// small (< 256 arcs) one warp each; big (< 4,096 arcs) one block each; huge
// ones are split over the blocks left over, which mark a shared global colour
// bitmap; the last of them to finish computes the colour; tiny ones (at
// most 32 arcs, so a colour below 33) take 8 lanes each, 4 to a warp, and
// find their colour in a 64-bit mask held in registers.
//
// Vertex order: a stable radix sort of (colour, degree bin) keys, so each
// colour class is split into the group / warp / CTA / hub bins of the sweep,
// ascending vertex id inside each bucket.  Bins: groups of 1..32 lanes per
// vertex (about lane_arcs arcs per lane), quarter CTA (up to 1,024 arcs), CTA,
// hub (several CTAs).
#include <climits>
#include <cstring>
#include <vector>

#include "lv_ops.cuh"

namespace lv {
namespace {

constexpr int kJpBlock = 1024;       // threads per block of the persistent kernel
constexpr int kJpWarps = kJpBlock / 32;
constexpr int kJpBig = 256;          // arcs: from here a vertex uses a whole block
constexpr int kJpHuge = 4096;        // arcs: from here a vertex is split over blocks
constexpr int kMexWindow = 1024;     // colours examined per pass of the mex search
constexpr int kJpSmallU = 8;         // 32-arc chunks in flight per warp: a small vertex in one pass
constexpr int kJpTiny = 32;          // arcs: up to here a vertex uses 8 lanes (4 per warp)
constexpr int kJpTinyLanes = 8;
constexpr int kJpTinyPerWarp = 32 / kJpTinyLanes;
constexpr int kJpKinds = 4;          // small, big, huge, tiny

// device state; the ring of list lengths has 3 slots of {small, big, huge, tiny}.
// A list entry is {v, off[v], off[v + 1], 0}: whoever queues a vertex has
// its row bounds already, so the round that colours it starts at its arcs.
struct JpState {
    int32_t *cnt;          // higher-priority neighbours not yet processed
    int32_t *color;
    int4 *list[kJpKinds][2];  // [kind][round parity]
    int32_t *counts;       // [3 ring slots][kJpKinds kinds]
    int32_t *max_color;
    unsigned *huge_bm;     // 32-word first-window bitmap per slot of the huge list
    int32_t *huge_done;    // finished parts per slot of the huge list
    GridBarrier *bar;      // flag 1: a wait expired; flag 2: more rounds than vertices
    int32_t *rounds;
    const unsigned *hb;    // bit e: arc e leads to a higher-priority neighbour
    TraceBuf tb;
};

// is the neighbour of arc e of higher priority than the row's vertex
__device__ __forceinline__ bool higher_arc(const JpState &st, int e) {
    return (__ldg(&st.hb[e >> 5]) >> (e & 31)) & 1u;
}

// Block-local staging of the next round's ready vertices: pushes reserve
// room with shared-memory atomics, and the block appends each kind's staged
// entries to the global list with one global atomic per kind when it
// flushes (mid-round when a kind is half full, and before the round's
// barrier).  A push that does not fit goes straight to the global list.
// Without it, every warp's push was a global atomic on the same four
// counters, which serialised the rounds that release 10^5 vertices.
constexpr int kJpWB = 32;  // entries per warp and kind (small, tiny)
struct JpStage {
    int n[kJpWarps][2];
    int4 q[kJpWarps][2][kJpWB];
};

// append u (arcs [beg, end)) to the next round's list of its kind;
// warp-aggregated, through the block's stage when one is given
__device__ __forceinline__ void push_ready(const JpState &st, int32_t *cnt_next, int nxt_list,
                                           bool ready, int u, int beg, int end,
                                           JpStage *stg = nullptr) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int kind = 0;
    if (ready) {
        const int d = end - beg;
        kind = d >= kJpHuge ? 2 : (d >= kJpBig ? 1 : (d <= kJpTiny ? 3 : 0));
    }
#pragma unroll
    for (int k = 0; k < kJpKinds; ++k) {
        const bool mine = ready && kind == k;
        const unsigned bm = __ballot_sync(0xffffffffu, mine);
        if (bm) {
            const int c = __popc(bm);
            const int slot = k == 0 ? 0 : (k == 3 ? 1 : -1);
            if (stg && slot >= 0) {  // the warp's own buffer, written out when full
                const int w = threadIdx.x >> 5;
                int n0 = ((volatile int *)stg->n[w])[slot];
                if (n0 + c > kJpWB) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&cnt_next[k], n0);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    for (int t = lane; t < n0; t += 32)
                        st.list[k][nxt_list][base + t] = stg->q[w][slot][t];
                    n0 = 0;
                    __syncwarp();
                }
                if (mine) stg->q[w][slot][n0 + __popc(bm & lt)] = make_int4(u, beg, end, 0);
                __syncwarp();
                if (lane == 0) stg->n[w][slot] = n0 + c;
                __syncwarp();
                continue;
            }
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&cnt_next[k], c);
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (mine) st.list[k][nxt_list][pos + __popc(bm & lt)] = make_int4(u, beg, end, 0);
        }
    }
}

// One pass over arcs [e0, e1) of v by `nw` warps (this warp has rank
// `wrank`): the colour of every higher-priority neighbour is marked in the
// first window [0, kMexWindow) of bm (shared or global memory), and every
// lower-priority neighbour's count is decremented (and the neighbour queued
// for the next round when it reaches zero).  The two kinds of arcs are
// disjoint, so one pass serves both.  The row bounds of a lower-priority
// neighbour are loaded beside its decrement, for the queue entry.
template <int kU>  // chunks of 32 arcs in flight per warp
__device__ void jp_pass(const DGraph &g, const JpState &st, int v, int e0, int e1, int wrank,
                        int nw, unsigned *bm, int32_t *cnt_next, int nxt_list, JpStage *stg) {
    const int lane = threadIdx.x & 31;
    const int stride = nw * 32;
    for (int b0 = e0 + wrank * 32; b0 < e1; b0 += kU * stride) {
        int uu[kU];
        bool higher[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = b0 + u * stride + lane;
            uu[u] = e < e1 ? g.arcs[e].x : v;
            higher[u] = e < e1 && higher_arc(st, e);
        }
        int res[kU], ob[kU], oe[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            ob[u] = oe[u] = 0;
            if (uu[u] == v) res[u] = 0;
            else if (higher[u]) res[u] = __ldcg(&st.color[uu[u]]);
            else {
                res[u] = atomicSub(&st.cnt[uu[u]], 1);
                ob[u] = g.off[uu[u]];
                oe[u] = g.off[uu[u] + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (uu[u] != v && higher[u] && (unsigned)res[u] < (unsigned)kMexWindow)
                atomicOr(&bm[res[u] >> 5], 1u << (res[u] & 31));
            push_ready(st, cnt_next, nxt_list, uu[u] != v && !higher[u] && res[u] == 1, uu[u], ob[u],
                       oe[u], stg);
        }
    }
}

// Smallest colour of v not in the window bitmap whose word l is held by lane
// l; windows above the first are searched by mark-only passes of this warp
// over v's whole row (needs >= kMexWindow colours among v's higher-priority
// neighbours).
__device__ int warp_mex(const DGraph &g, const JpState &st, int v, unsigned word0,
                        unsigned *scratch32) {
    const int lane = threadIdx.x & 31;
    unsigned word = word0;
    const int beg = g.off[v], end = g.off[v + 1];
    for (int base = 0;; base += kMexWindow) {
        const unsigned notfull = __ballot_sync(0xffffffffu, word != 0xffffffffu);
        if (notfull) {
            const int f = __ffs(notfull) - 1;
            const unsigned wf = __shfl_sync(0xffffffffu, word, f);
            return base + 32 * f + __ffs(~wf) - 1;
        }
        const int nb = base + kMexWindow;
        scratch32[lane] = 0u;
        __syncwarp();
        for (int e = beg + lane; e < end; e += 32) {
            const int u = g.arcs[e].x;
            if (u != v && higher_arc(st, e)) {
                const int c = __ldcg(&st.color[u]) - nb;
                if (c >= 0 && c < kMexWindow) atomicOr(&scratch32[c >> 5], 1u << (c & 31));
            }
        }
        __syncwarp();
        word = scratch32[lane];
        __syncwarp();
    }
}

// the largest colour is kept per thread (`top`) and added to max_color once
// per warp when the kernel ends: one global atomic per vertex on a single
// word serialised the rounds that colour 10^5 vertices
__device__ __forceinline__ void set_color(const JpState &st, int v, int mex, int &top) {
    __stcg(&st.color[v], mex);
    top = max(top, mex);
}
__device__ __forceinline__ void flush_max(const JpState &st, int top) {
    const int t = __reduce_max_sync(0xffffffffu, top);
    if ((threadIdx.x & 31) == 0 && t >= 0) atomicMax(st.max_color, t);
}

// Tiny vertices (at most kJpTiny arcs), 32 / LANES per warp with LANES
// lanes each: every lane holds up to kJpTiny / LANES arcs, all loads in
// flight at once.  A tiny vertex has at most 32 higher-priority neighbours,
// so its colour is below 33: the colours of those neighbours go into a
// 64-bit mask in registers, OR-reduced over the group, and the colour is its
// lowest clear bit.  Lower-priority neighbours are released as in jp_pass.
// Every lane of the warp calls this (t >= n marks an empty group).
template <int LANES>
__device__ void jp_tiny_warp(const DGraph &g, const JpState &st, const int4 *list, int t, int n,
                             int32_t *cnt_next, int nxt_list, JpStage *stg, int &top) {
    constexpr int kA = kJpTiny / LANES;
    const int lane = threadIdx.x & 31, gl = lane & (LANES - 1);
    const bool has = t < n;
    const int4 it = has ? __ldcg(&list[t]) : make_int4(-1, 0, 0, 0);
    const int v = it.x;
    int uu[kA];
    bool higher[kA];
#pragma unroll
    for (int a = 0; a < kA; ++a) {
        const int e = it.y + gl + a * LANES;
        const bool in = has && e < it.z;
        uu[a] = in ? g.arcs[e].x : v;
        higher[a] = in && higher_arc(st, e);
    }
    int res[kA], ob[kA], oe[kA];
#pragma unroll
    for (int a = 0; a < kA; ++a) {
        ob[a] = oe[a] = 0;
        if (uu[a] == v) res[a] = 0;
        else if (higher[a]) res[a] = __ldcg(&st.color[uu[a]]);
        else {
            res[a] = atomicSub(&st.cnt[uu[a]], 1);
            ob[a] = g.off[uu[a]];
            oe[a] = g.off[uu[a] + 1];
        }
    }
    unsigned long long mask = 0ull;
#pragma unroll
    for (int a = 0; a < kA; ++a) {
        if (uu[a] != v && higher[a] && (unsigned)res[a] < 64u) mask |= 1ull << res[a];
        push_ready(st, cnt_next, nxt_list, uu[a] != v && !higher[a] && res[a] == 1, uu[a], ob[a],
                   oe[a], stg);
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    const int mex = __ffsll((long long)~mask) - 1;
    if (has && gl == 0) set_color(st, v, mex, top);
}

// d(v) = neighbours of v other than v itself (rows are sorted, so the
// self-loop is found by bisection)
__global__ void nbdeg_kernel(DGraph g, int32_t *d) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        int lo = g.off[v], hi = g.off[v + 1];
        const int len = hi - lo;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (g.arcs[mid].x < v) lo = mid + 1; else hi = mid;
        }
        d[v] = len - (lo < g.off[v + 1] && g.arcs[lo].x == v ? 1 : 0);
    }
}

// Priority pi(v) = (d(v), h(v ^ seed), v) compared lexicographically (R11;
// d = nullptr leaves the degree out).  One warp per vertex: the bit of every
// arc whose neighbour has the higher priority (hb, cleared before) and the
// count of such neighbours (outside the core of degree >= core_t, for a
// vertex outside it).
__global__ void __launch_bounds__(256) jp_init_kernel(DGraph g, unsigned long long seed,
                                                      const int32_t *__restrict__ d, int core_t,
                                                      unsigned *hb, JpState st) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t vv = blockIdx.x * 8 + (threadIdx.x >> 5); vv < g.n; vv += nw) {
        const int v = (int)vv;
        const unsigned long long hv = prio_hash((unsigned long long)v ^ seed);
        const int dv = d ? d[v] : 0;
        const int beg = g.off[v], end = g.off[v + 1];
        int c = 0, c_out = 0;  // higher-priority neighbours: all, outside the core
        for (int e0 = beg; e0 < end; e0 += 32) {
            const int e = e0 + lane;
            bool hi = false, out = false;
            if (e < end) {
                const int u = g.arcs[e].x;
                if (u != v) {
                    const int du = d ? d[u] : 0;
                    hi = du > dv ||
                         (du == dv &&
                          prio_greater(prio_hash((unsigned long long)u ^ seed), u, hv, v));
                    out = hi && du < core_t;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, hi);
            c += __popc(m);
            c_out += __popc(__ballot_sync(0xffffffffu, out));
            if (lane == 0 && m) {  // the 32 arcs from e0 span two words at most
                const int sh = e0 & 31;
                atomicOr(&hb[e0 >> 5], m << sh);
                if (sh && (m >> (32 - sh))) atomicOr(&hb[(e0 >> 5) + 1], m >> (32 - sh));
            }
        }
        // a core vertex keeps its full count (the length of its list of
        // higher-priority neighbours) and is coloured by the core pass
        const bool core = dv >= core_t;
        if (lane == 0) {
            st.cnt[v] = core ? c : c_out;
            st.color[v] = -1;
        }
    }
}

// Round 0: the vertices outside the core with no higher-priority neighbour
// outside it, listed by kind.  Each block counts its range's vertices per
// kind in shared memory (one atomic per warp and kind) and reserves room
// with one global atomic per kind; queuing them from jp_init_kernel cost a
// global atomic per warp on the same four counters, millions of them on a
// skewed graph.
constexpr int kR0PerThread = 8;
__global__ void __launch_bounds__(256) jp_round0_kernel(DGraph g, const int32_t *__restrict__ d,
                                                        int core_t, JpState st) {
    __shared__ int cnt[kJpKinds], base[kJpKinds];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    constexpr int kSpan = 256 * kR0PerThread;
    for (int64_t b0 = (int64_t)blockIdx.x * kSpan; b0 < g.n; b0 += (int64_t)gridDim.x * kSpan) {
        if (threadIdx.x < kJpKinds) cnt[threadIdx.x] = 0;
        __syncthreads();
        int kind[kR0PerThread], pos[kR0PerThread];
#pragma unroll
        for (int q = 0; q < kR0PerThread; ++q) {
            const int64_t vv = b0 + q * 256 + threadIdx.x;
            kind[q] = -1;
            if (vv < g.n) {
                const int v = (int)vv;
                const bool core = (d ? d[v] : 0) >= core_t;
                if (!core && __ldcg(&st.cnt[v]) == 0) {
                    const int deg = g.off[v + 1] - g.off[v];
                    kind[q] = deg >= kJpHuge ? 2 : (deg >= kJpBig ? 1 : (deg <= kJpTiny ? 3 : 0));
                }
            }
#pragma unroll
            for (int k = 0; k < kJpKinds; ++k) {
                const unsigned m = __ballot_sync(0xffffffffu, kind[q] == k);
                if (!m) continue;
                int p0 = 0;
                if (lane == 0) p0 = atomicAdd(&cnt[k], __popc(m));
                p0 = __shfl_sync(0xffffffffu, p0, 0);
                if (kind[q] == k) pos[q] = p0 + __popc(m & lt);
            }
        }
        __syncthreads();
        if (threadIdx.x < kJpKinds)
            base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&st.counts[threadIdx.x], cnt[threadIdx.x]) : 0;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kR0PerThread; ++q) {
            if (kind[q] < 0) continue;
            const int v = (int)(b0 + q * 256 + threadIdx.x);
            st.list[kind[q]][0][base[kind[q]] + pos[q]] = make_int4(v, g.off[v], g.off[v + 1], 0);
        }
        __syncthreads();
    }
}

// All rounds of Jones-Plassmann in one cooperative launch.  Round r colours
// the vertices queued in round r - 1, in units of one block each:
//   huge  split over P blocks each, which mark a global bitmap and release
//         lower-priority neighbours; the last of the P to finish (a
//         per-vertex arrival counter) turns the bitmap into the colour
//   big   one block each (mark, release, colour)
//   small one warp each, 32 to a block
// Huge vertices get the blocks that big and small ones leave (P >= 1), so
// a block takes one unit per round unless the units outnumber the blocks.
// A grid barrier ends the round; the vertices released in round r are
// coloured in round r + 1, after the colours they depend on have been
// written.
__global__ void __launch_bounds__(kJpBlock) jp_persistent_kernel(DGraph g, JpState st) {
    extern __shared__ int4 jp_dyn[];
    JpStage *stg = reinterpret_cast<JpStage *>(jp_dyn);
    __shared__ int s_abort;
    if (threadIdx.x < kJpWarps * 2) (&stg->n[0][0])[threadIdx.x] = 0;
    if (threadIdx.x == 0) {  // the core pass failed: its colours are incomplete
        unsigned long long w;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(&st.bar->word) : "memory");
        s_abort = (w >> kBarrierFlagShift) != 0;
    }
    __syncthreads();
    if (s_abort) return;
    __shared__ unsigned bm_warp[kJpWarps][32];
    __shared__ unsigned bm_cta[32];
    __shared__ int s_last_part;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned bar_passed = 0;
    int top = -1;  // largest colour this thread set
    int n_small = __ldcg(&st.counts[0]), n_big = __ldcg(&st.counts[1]),
        n_huge = __ldcg(&st.counts[2]), n_tiny = __ldcg(&st.counts[3]);
    for (int r = 0;; ++r) {
        const int nxt = (r + 1) % 3, clr = (r + 2) % 3;
        if (blockIdx.x == 0 && threadIdx.x < kJpKinds) st.counts[kJpKinds * clr + threadIdx.x] = 0;
        const int in_list = r & 1, out_list = (r + 1) & 1;
        int32_t *cnt_next = st.counts + kJpKinds * nxt;
        const unsigned long long tr0 = LV_TRACE_ON ? gtimer() : 0;
        const int small_units = (n_small + kJpWarps - 1) / kJpWarps;
        constexpr int tiny_per_unit = kJpWarps * kJpTinyPerWarp;
        const int tiny_units = (n_tiny + tiny_per_unit - 1) / tiny_per_unit;
        const int P = n_huge > 0
                          ? max(1, ((int)gridDim.x - n_big - small_units - tiny_units) / n_huge)
                          : 0;
        const int huge_units = n_huge * P;
        const int units = huge_units + n_big + small_units + tiny_units;
        // heavy rounds stage their pushes in the block; light ones (the long
        // tail of the priority DAG) push straight to the global lists
        JpStage *rs = stg;
        for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
            if (unit < huge_units) {
                const int t = unit % n_huge, part = unit / n_huge;
                const int4 it = __ldcg(&st.list[2][in_list][t]);
                const int v = it.x;
                const int L = (it.z - it.y + P - 1) / P;
                const int e0 = it.y + part * L, e1 = min(it.z, e0 + L);
                unsigned *gbm = st.huge_bm + (size_t)t * 32;
                jp_pass<4>(g, st, v, e0, e1, wib, kJpWarps, gbm, cnt_next, out_list, rs);
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) s_last_part = atomicAdd(&st.huge_done[t], 1) == P - 1;
                __syncthreads();
                if (s_last_part && wib == 0) {
                    __threadfence();
                    const unsigned w0 = __ldcg(&gbm[lane]);
                    __stcg(&gbm[lane], 0u);
                    const int mex = warp_mex(g, st, v, w0, bm_warp[0]);
                    if (lane == 0) {
                        set_color(st, v, mex, top);
                        st.huge_done[t] = 0;
                    }
                }
                __syncthreads();
            } else if (unit < huge_units + n_big) {
                const int4 it = __ldcg(&st.list[1][in_list][unit - huge_units]);
                const int v = it.x;
                if (threadIdx.x < 32) bm_cta[threadIdx.x] = 0u;
                __syncthreads();
                jp_pass<4>(g, st, v, it.y, it.z, wib, kJpWarps, bm_cta, cnt_next, out_list, rs);
                __syncthreads();
                if (wib == 0) {
                    const int mex = warp_mex(g, st, v, bm_cta[lane], bm_warp[0]);
                    if (lane == 0) set_color(st, v, mex, top);
                }
                __syncthreads();
            } else if (unit >= huge_units + n_big + small_units) {
                const int u0 = (unit - huge_units - n_big - small_units) * tiny_per_unit;
                jp_tiny_warp<kJpTinyLanes>(g, st, st.list[3][in_list],
                                           u0 + wib * kJpTinyPerWarp + lane / kJpTinyLanes,
                                           n_tiny, cnt_next, out_list, rs, top);
            } else {
                const int t = (unit - huge_units - n_big) * kJpWarps + wib;
                if (t < n_small) {
                    const int4 it = __ldcg(&st.list[0][in_list][t]);
                    const int v = it.x;
                    unsigned *bm = bm_warp[wib];
                    bm[lane] = 0u;
                    __syncwarp();
                    jp_pass<kJpSmallU>(g, st, v, it.y, it.z, 0, 1, bm, cnt_next, out_list, rs);
                    __syncwarp();
                    const unsigned w0 = bm[lane];
                    __syncwarp();
                    const int mex = warp_mex(g, st, v, w0, bm);
                    if (lane == 0) set_color(st, v, mex, top);
                    __syncwarp();
                }
            }
        }
        for (int slot = 0; slot < 2; ++slot) {  // the warp's last entries of the round
            const int k = slot ? 3 : 0;
            const int n0 = stg->n[wib][slot];
            if (n0) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&cnt_next[k], n0);
                base = __shfl_sync(0xffffffffu, base, 0);
                for (int t = lane; t < n0; t += 32) st.list[k][out_list][base + t] = stg->q[wib][slot][t];
                __syncwarp();
                if (lane == 0) stg->n[wib][slot] = 0;
                __syncwarp();
            }
        }
        const unsigned long long tr1 = LV_TRACE_ON ? gtimer() : 0;
        if (LV_TRACE_ON && threadIdx.x == 0 && blockIdx.x < 8)
            trace4(st.tb, 0x100000000ull | (unsigned)r, (unsigned long long)blockIdx.x, tr0, tr1);
        if (!grid_sync(st.bar, bar_passed)) {
            flush_max(st, top);
            return;
        }
        if (LV_TRACE_ON && blockIdx.x == 0 && threadIdx.x == 0)
            trace4(st.tb, 0x200000000ull | (unsigned)r,
                   ((unsigned long long)n_small << 32) | (unsigned)n_tiny, gtimer(),
                   ((unsigned long long)n_big << 32) | (unsigned)n_huge);
        n_small = __ldcg(&cnt_next[0]);
        n_big = __ldcg(&cnt_next[1]);
        n_huge = __ldcg(&cnt_next[2]);
        n_tiny = __ldcg(&cnt_next[3]);
        if (n_small + n_big + n_huge + n_tiny == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *st.rounds = r + 1;
            flush_max(st, top);
            return;
        }
        if (r > g.n) {  // every round colours at least one vertex
            if (threadIdx.x == 0) barrier_raise(st.bar, 2);
            return;
        }
    }
}

// ------------------------------------------------------------ bucketing
__global__ void bucket_key_kernel(DGraph g, const int32_t *__restrict__ color, BinLimits lim,
                                  uint32_t *keys, uint32_t *vals) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        const int deg = g.off[v + 1] - g.off[v];
        int bin;
        if (deg == 0) bin = kBinSkip;
        else if (deg <= lim.warp_max) {
            bin = 0;  // smallest group of G = 2^bin lanes with deg <= G * lane_arcs
            while (bin < kGroupBins - 1 && deg > (1 << bin) * lim.lane_arcs) ++bin;
        } else if (deg <= lim.cta_max && deg <= kQuadMaxArcs) bin = kBinQuad;
        else if (deg <= lim.cta_max) bin = kBinCta;
        else bin = kBinHub;
        const int cls = color ? color[v] : 0;
        keys[v] = (uint32_t)(cls * (kBins + 1) + bin);
        vals[v] = (uint32_t)v;
    }
}

__global__ void bucket_count_kernel(const uint32_t *__restrict__ keys, int n, int32_t *counts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // count run heads only: one atomic per bucket boundary
        const uint32_t k = keys[i];
        if (i == n - 1 || keys[i + 1] != k) atomicAdd(&counts[k], i + 1);
        if (i > 0 && keys[i - 1] != k) atomicAdd(&counts[k], -i);
    }
}

__device__ __forceinline__ int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// hub hash-table size and arc-chunk count at each position of the order
// (0 for non-hubs); the chunk is kHubChunk << shift[class] (keys: the sorted
// bucket keys; shift may be null)
__global__ void hub_size_kernel(DGraph g, const int32_t *__restrict__ order, int cta_max, int factor,
                                const uint32_t *__restrict__ keys,
                                const uint8_t *__restrict__ shift, int32_t *tsize,
                                int32_t *nchunks) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += gridDim.x * blockDim.x) {
        const int v = order[p];
        const int deg = g.off[v + 1] - g.off[v];
        const bool hub = deg > cta_max;
        const int chunk = kHubChunk << (shift && hub ? shift[keys[p] / (kBins + 1)] : 0);
        tsize[p] = hub ? next_pow2(factor * deg) : 0;
        nchunks[p] = hub ? (deg + chunk - 1) / chunk : 0;
    }
}

__global__ void fill_empty_kernel(int2 *tab, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        tab[i] = make_int2(kEmpty, 0);
}

__global__ void gather_at_kernel(const int32_t *__restrict__ vals, const int32_t *__restrict__ idx,
                                 int m, int32_t *out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x)
        out[q] = vals[idx[q]];
}

// ------------------------------------------------------------------ core
// With the largest-degree-first priority the vertices of degree >= T form
// a prefix of the priority order, so every higher-priority neighbour of
// such a vertex is one of them too.  This core (T the smallest power of two
// >= 64 that leaves at most kCoreMax vertices in it) holds the long
// priority chains of a skewed graph: hubs adjacent to hubs, one or a few
// ready per round, each round costing a grid barrier.  It is coloured first
// by one launch without rounds: its vertices are sorted by priority, warp w
// of the W in the grid takes ranks w, w + W, ..., and colours each vertex
// with the smallest colour that none of its higher-priority neighbours has,
// waiting (bounded) for those not coloured yet.  Those all have smaller
// ranks, the smallest unfinished rank never waits and every warp is resident
// (a cooperative launch), so the waits end.  The colour a vertex gets is
// the one a Jones-Plassmann round gives it, as both are the smallest colour
// absent from its higher-priority neighbours; the rounds then colour the
// rest, the core's colours already in place.
constexpr int kCoreMinLog = 6;                    // T >= 64
constexpr int kCoreMax = 1 << 20;                 // vertices in the core at most
constexpr int kCoreBlock = 512;
constexpr int kCoreWarps = kCoreBlock / 32;
constexpr int kCoreU = 4;                         // 32-entry chunks in flight per warp
constexpr unsigned kCoreSpinLimit = 1u << 22;     // polls of one colour, x >= 32 ns sleeps

__device__ __forceinline__ int ld_relaxed_i32(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_i32(int32_t *p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// vertices per bin floor(log2 d) for d >= 2^kCoreMinLog
__global__ void core_hist_kernel(const int32_t *__restrict__ d, int n, int32_t *hist) {
    __shared__ int h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int x = d[v];
        if (x >= (1 << kCoreMinLog)) atomicAdd(&h[31 - __clz(x)], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// the core's vertices with the hash part of their priority, inverted so
// that an ascending sort puts the higher priority first
__global__ void core_collect_kernel(const int32_t *__restrict__ d, int n, int core_t,
                                    unsigned long long seed, uint64_t *keys, uint32_t *vals,
                                    int32_t *count) {
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int v0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
        const int v = v0 + lane;
        const bool in = v < n && d[v] >= core_t;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (!m) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0) + __popc(m & ((1u << lane) - 1u));
        if (in) {
            keys[base] = ~prio_hash((unsigned long long)v ^ seed);
            vals[base] = (uint32_t)v;
        }
    }
}

// second sort key: the degree, inverted
__global__ void core_dkey_kernel(const uint32_t *__restrict__ vals, const int32_t *__restrict__ d,
                                 int k, uint32_t *keys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        keys[i] = ~(uint32_t)d[vals[i]];
}

// rank_of[order[r]] = r
__global__ void core_rank_kernel(const int32_t *__restrict__ order, int k, int32_t *rank_of) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x)
        rank_of[order[r]] = r;
}

// the ranks of the higher-priority neighbours of each core vertex, in rank
// order (one warp per vertex, a lane per 32-arc word of the priority bits;
// only the arcs whose bit is set are read)
__global__ void core_lists_kernel(DGraph g, const int32_t *__restrict__ order, int k,
                                  const int32_t *__restrict__ hoff,
                                  const unsigned *__restrict__ hb,
                                  const int32_t *__restrict__ rank_of, int32_t *hcol) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < k; r += nw) {
        const int v = order[r];
        const int beg = g.off[v], end = g.off[v + 1];
        int pos = hoff[r];
        if (end <= beg) continue;
        const int wlast = (end - 1) >> 5;
        for (int w0 = beg >> 5; w0 <= wlast; w0 += 32) {
            const int w = w0 + lane;
            unsigned bits = 0u;
            if (w <= wlast) {
                const int lo = max(beg - 32 * w, 0), hi = min(end - 32 * w, 32);
                const unsigned mhi = hi == 32 ? 0xffffffffu : (1u << hi) - 1u;
                bits = __ldg(&hb[w]) & mhi & ~((1u << lo) - 1u);
            }
            const int c = __popc(bits);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int p = pos + incl - c;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                hcol[p++] = rank_of[g.arcs[32 * w + b].x];
            }
            pos += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// colour of *p once it is written (>= 0), or -1 when the wait expires or
// another warp has raised an error
__device__ int core_wait(const int32_t *p, GridBarrier *bar) {
    for (unsigned spins = 1;; ++spins) {
        __nanosleep(32);
        const int c = ld_relaxed_i32(p);
        if (c >= 0) return c;
        if (spins >= kCoreSpinLimit) return -1;
        if ((spins & 255u) == 0u) {
            unsigned long long w;
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(&bar->word) : "memory");
            if (w >> kBarrierFlagShift) return -1;
        }
    }
}

// smallest colour absent from the list [e0, e1) (all coloured) whose first
// window is held in word0 (word l in lane l), as warp_mex does for a row
__device__ int core_mex(const int32_t *__restrict__ hcol, int e0, int e1, const int32_t *color,
                        unsigned word0, unsigned *scratch32) {
    const int lane = threadIdx.x & 31;
    unsigned word = word0;
    for (int base = 0;; base += kMexWindow) {
        const unsigned notfull = __ballot_sync(0xffffffffu, word != 0xffffffffu);
        if (notfull) {
            const int f = __ffs(notfull) - 1;
            const unsigned wf = __shfl_sync(0xffffffffu, word, f);
            return base + 32 * f + __ffs(~wf) - 1;
        }
        const int nb = base + kMexWindow;
        scratch32[lane] = 0u;
        __syncwarp();
        for (int e = e0 + lane; e < e1; e += 32) {
            const int c = ld_relaxed_i32(&color[hcol[e]]) - nb;
            if (c >= 0 && c < kMexWindow) atomicOr(&scratch32[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        word = scratch32[lane];
        __syncwarp();
    }
}

// The top of the core (ranks [0, r1), r1 <= kTopMax with at most kTopEntries
// list entries) on one thread-block cluster: the deepest priority chains
// run through the largest hubs, and there a colour reaches the warps
// waiting for it through shared memory: every block of the cluster keeps
// all of the top's colours, and the warp that colours a rank stores the
// colour into each block's copy (distributed shared memory), so a wait is a
// poll of the block's own shared memory.  Warp w of the cluster's W takes
// ranks w, w + W, ...; colours also go to rc (by rank) and to the vertex.
// Blocks do not return early (a failing warp stops working and flags the
// error), and a cluster barrier at the end keeps every block's shared
// memory alive until the last store into it.
constexpr int kTopThreads = 1024;
constexpr int kTopWarps = kTopThreads / 32;
constexpr int kTopMax = 40960;                     // ranks at most
constexpr int kTopEntries = 1 << 24;               // list entries at most
constexpr int kTopU = 8;                           // 32-entry chunks in flight per warp
constexpr unsigned kTopSpinLimit = 1u << 24;       // polls of one colour, x >= 20 ns sleeps
constexpr int kTopMaxCluster = 16;
constexpr int kTopPend = 256;                      // ranks a warp sets aside to wait for

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_blocks() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// *p of block `cta` of the cluster (p: this block's copy) = v
__device__ __forceinline__ void st_cluster_i32(const int *p, unsigned cta, int v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(cta));
    asm volatile("st.relaxed.cluster.shared::cluster.b32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_cluster_local_i32(const int *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    int v;
    asm volatile("ld.relaxed.cluster.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

// smallest colour absent from the ranks listed in [e0, e1) (all coloured,
// colours in this block's shared memory) whose first window is in word0
__device__ int core_mex_smem(const int32_t *__restrict__ hcol, int e0, int e1, const int *sc,
                             unsigned word0, unsigned *scratch32) {
    const int lane = threadIdx.x & 31;
    unsigned word = word0;
    for (int base = 0;; base += kMexWindow) {
        const unsigned notfull = __ballot_sync(0xffffffffu, word != 0xffffffffu);
        if (notfull) {
            const int f = __ffs(notfull) - 1;
            const unsigned wf = __shfl_sync(0xffffffffu, word, f);
            return base + 32 * f + __ffs(~wf) - 1;
        }
        const int nb = base + kMexWindow;
        scratch32[lane] = 0u;
        __syncwarp();
        for (int e = e0 + lane; e < e1; e += 32) {
            const int c = ld_cluster_local_i32(&sc[hcol[e]]) - nb;
            if (c >= 0 && c < kMexWindow) atomicOr(&scratch32[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        word = scratch32[lane];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kTopThreads) jp_core_top_kernel(
    const int32_t *__restrict__ order, const int32_t *__restrict__ hoff,
    const int32_t *__restrict__ hcol, int k, int32_t *rc, int32_t *r1_out, JpState st) {
    extern __shared__ int sc[];  // colours of ranks [0, r1)
    __shared__ unsigned bm[kTopWarps][32];
    __shared__ int pend[kTopWarps][kTopPend];
    __shared__ int s_r1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned crank = cluster_rank(), nblocks = cluster_blocks();
    if (threadIdx.x == 0) {  // largest r1 <= min(k, kTopMax) with hoff[r1] <= kTopEntries
        int lo = 0, hi = min(k, kTopMax);
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (hoff[mid] <= kTopEntries) lo = mid; else hi = mid - 1;
        }
        s_r1 = lo;
        if (crank == 0) *r1_out = lo;
    }
    __syncthreads();
    const int r1 = s_r1;
    for (int i = threadIdx.x; i < r1; i += kTopThreads) sc[i] = -1;
    cluster_barrier();  // every copy initialised before the first remote store
    const int nw = (int)nblocks * kTopWarps;
    int top = -1;
    bool fail = false;
    for (int r = (int)crank * kTopWarps + wib; r < r1 && !fail; r += nw) {
        const int e0 = hoff[r], e1 = hoff[r + 1];
        bm[wib][lane] = 0u;
        __syncwarp();
        // pass 1: the ranks already coloured are marked, the others set
        // aside; pass 2 polls those together, so that once the last of them
        // is coloured only shared-memory work is left (the chain of waits
        // runs through that step)
        int npend = 0;
        for (int b = e0; b < e1 && !fail; b += 32 * kTopU) {
            int x[kTopU];
#pragma unroll
            for (int q = 0; q < kTopU; ++q) {
                const int e = b + q * 32 + lane;
                x[q] = e < e1 ? __ldg(&hcol[e]) : -1;
            }
            bool bad = false;
#pragma unroll
            for (int q = 0; q < kTopU; ++q) {
                if (x[q] >= r) {  // not an earlier rank: the lists are inconsistent
                    bad = true;
                    x[q] = -1;
                }
                const int c = x[q] >= 0 ? ld_cluster_local_i32(&sc[x[q]]) : 0;
                const bool wait = x[q] >= 0 && c < 0;
                const unsigned m = __ballot_sync(0xffffffffu, wait);
                bool parked = false;
                if (m && npend + __popc(m) <= kTopPend) {
                    if (wait) pend[wib][npend + __popc(m & ((1u << lane) - 1u))] = x[q];
                    npend += __popc(m);
                    parked = wait;
                }
                int cc = c;
                for (unsigned spins = 1; wait && !parked && cc < 0; ++spins) {  // no room: wait now
                    if (spins > kTopSpinLimit) break;
                    __nanosleep(20);
                    cc = ld_cluster_local_i32(&sc[x[q]]);
                }
                if (x[q] < 0 || parked) continue;
                if (cc < 0) bad = true;
                else if (cc < kMexWindow) atomicOr(&bm[wib][cc >> 5], 1u << (cc & 31));
            }
            fail = __any_sync(0xffffffffu, bad);
        }
        __syncwarp();
        for (unsigned spins = 1; npend > 0 && !fail; ++spins) {
            bool left = false;
            for (int t = lane; t < npend; t += 32) {
                const int x = pend[wib][t];
                if (x < 0) continue;
                const int c = ld_cluster_local_i32(&sc[x]);
                if (c < 0) {
                    left = true;
                    continue;
                }
                if (c < kMexWindow) atomicOr(&bm[wib][c >> 5], 1u << (c & 31));
                pend[wib][t] = -1;
            }
            if (!__any_sync(0xffffffffu, left)) break;
            bool stop = spins > kTopSpinLimit;
            if ((spins & 255u) == 0u) {
                unsigned long long w = 0;
                if (lane == 0)
                    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
                                 : "=l"(w) : "l"(&st.bar->word) : "memory");
                stop |= (__shfl_sync(0xffffffffu, w, 0) >> kBarrierFlagShift) != 0;
            }
            fail = stop;
            if (!stop) __nanosleep(20);
        }
        if (fail) {  // warp-uniform: stop, flag the error
            if (lane == 0) barrier_raise(st.bar, 1);
            break;
        }
        __syncwarp();
        const unsigned w0 = bm[wib][lane];
        __syncwarp();
        const int mex = core_mex_smem(hcol, e0, e1, sc, w0, bm[wib]);
        if (lane < (int)nblocks) st_cluster_i32(&sc[r], (unsigned)lane, mex);
        if (lane == 0) {
            rc[r] = mex;
            __stcg(&st.color[order[r]], mex);
        }
        if (LV_TRACE_ON && lane == 0 && (r & 15) == 0)
            trace4(st.tb, 0xB00000000ull, (unsigned long long)r, gtimer(),
                   (unsigned long long)(e1 - e0));
        top = max(top, mex);
        __syncwarp();
    }
    if (lane == 0 && top >= 0) atomicMax(st.max_color, top);
    cluster_barrier();  // no block leaves while stores into its copy may follow
}

// The rest of the core, ranks [r1, k), on the whole grid: warp w of the W
// takes ranks r1 + w, r1 + w + W, ...; colours are read from and written to
// rc (by rank) in L2.
__global__ void __launch_bounds__(kCoreBlock) jp_core_kernel(const int32_t *__restrict__ order,
                                                             const int32_t *__restrict__ hoff,
                                                             const int32_t *__restrict__ hcol,
                                                             int k, int32_t *rc,
                                                             const int32_t *__restrict__ r1_in,
                                                             JpState st) {
    __shared__ unsigned bm[kCoreWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = gridDim.x * kCoreWarps;
    const int r1 = *r1_in;
    int top = -1;
    for (int r = r1 + blockIdx.x * kCoreWarps + wib; r < k; r += nw) {
        const int e0 = hoff[r], e1 = hoff[r + 1];
        bm[wib][lane] = 0u;
        __syncwarp();
        bool fail = false;
        for (int b = e0; b < e1; b += 32 * kCoreU) {
            int u[kCoreU], c[kCoreU];
#pragma unroll
            for (int q = 0; q < kCoreU; ++q) {
                const int e = b + q * 32 + lane;
                u[q] = e < e1 ? __ldg(&hcol[e]) : -1;
            }
#pragma unroll
            for (int q = 0; q < kCoreU; ++q) {  // a rank not below r: inconsistent lists
                if (u[q] >= r) fail = true;
                if (u[q] >= r) u[q] = -1;
            }
#pragma unroll
            for (int q = 0; q < kCoreU; ++q) c[q] = u[q] >= 0 ? ld_relaxed_i32(&rc[u[q]]) : 0;
#pragma unroll
            for (int q = 0; q < kCoreU; ++q) {
                if (u[q] < 0) continue;
                if (c[q] < 0) c[q] = core_wait(&rc[u[q]], st.bar);
                if (c[q] < 0) fail = true;
                else if (c[q] < kMexWindow) atomicOr(&bm[wib][c[q] >> 5], 1u << (c[q] & 31));
            }
            if (__any_sync(0xffffffffu, fail)) break;
        }
        if (__any_sync(0xffffffffu, fail)) {  // warp-uniform: give up, flag the error
            if (lane == 0) barrier_raise(st.bar, 1);
            return;
        }
        __syncwarp();
        const unsigned w0 = bm[wib][lane];
        __syncwarp();
        const int mex = core_mex(hcol, e0, e1, rc, w0, bm[wib]);
        if (lane == 0) {
            st_relaxed_i32(&rc[r], mex);
            __stcg(&st.color[order[r]], mex);
        }
        if (LV_TRACE_ON && lane == 0 && (r & 15) == 0)
            trace4(st.tb, 0xB00000000ull, (unsigned long long)r, gtimer(),
                   (unsigned long long)(e1 - e0));
        top = max(top, mex);
        __syncwarp();
    }
    if (lane == 0 && top >= 0) atomicMax(st.max_color, top);
}

// Colours the core of degree >= core_t (k vertices): sorts it by priority
// (degree, then hash; distinct vertices have distinct hashes), lists each
// vertex's higher-priority neighbours (their number is st.cnt) and runs the
// core kernel on `sms` SMs (0 = all).
lv_status core_pass(const DGraph &g, uint64_t seed, const int32_t *d, int k, int core_t,
                    const JpState &st, int *pinned, cudaStream_t s, int sms) {
    uint64_t *keys = nullptr, *keys_alt = nullptr;
    uint32_t *vals = nullptr, *vals_alt = nullptr, *dkeys = nullptr, *dkeys_alt = nullptr;
    int32_t *count = nullptr, *hoff = nullptr, *hcol = nullptr, *rank_of = nullptr, *rc = nullptr;
    int32_t *r1 = nullptr;
    LV_TRY(dalloc_n(&keys, (size_t)k, s));
    LV_TRY(dalloc_n(&keys_alt, (size_t)k, s));
    LV_TRY(dalloc_n(&vals, (size_t)k, s));
    LV_TRY(dalloc_n(&vals_alt, (size_t)k, s));
    LV_TRY(dalloc_n(&dkeys, (size_t)k, s));
    LV_TRY(dalloc_n(&dkeys_alt, (size_t)k, s));
    LV_TRY(dalloc_n(&count, 1, s));
    LV_TRY(dalloc_n(&hoff, (size_t)k + 1, s));
    LV_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t), s));
    core_collect_kernel<<<grid_for(g.n, 256, g_num_sms * 8), 256, 0, s>>>(d, g.n, core_t, seed, keys,
                                                                         vals, count);
    LV_LAUNCH_CHECK();
    LV_TRY(radix_sort_u64(keys, vals, keys_alt, vals_alt, k, 64, s));
    core_dkey_kernel<<<grid_for(k, 256, g_num_sms * 4), 256, 0, s>>>(vals, d, k, dkeys);
    LV_LAUNCH_CHECK();
    LV_TRY(radix_sort_u32(dkeys, vals, dkeys_alt, vals_alt, k, 32, s));
    trace_stamp(s, 4);
    const int32_t *order = reinterpret_cast<const int32_t *>(vals);
    gather_at_kernel<<<grid_for(k, 256, g_num_sms * 4), 256, 0, s>>>(st.cnt, order, k, hoff);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(hoff, hoff, k, s));
    LV_CUDA(cudaMemcpyAsync(pinned, hoff + k, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const int total = pinned[0];
    LV_TRY(dalloc_n(&hcol, (size_t)total + 1, s));
    LV_TRY(dalloc_n(&rank_of, (size_t)g.n, s));
    LV_TRY(dalloc_n(&rc, (size_t)k, s));
    LV_TRY(dalloc_n(&r1, 1, s));
    LV_CUDA(cudaMemsetAsync(rc, 0xff, sizeof(int32_t) * (size_t)k, s));  // -1: not coloured
    core_rank_kernel<<<grid_for(k, 256, g_num_sms * 4), 256, 0, s>>>(order, k, rank_of);
    LV_LAUNCH_CHECK();
    trace_stamp(s, 5);
    core_lists_kernel<<<grid_for(k, 8, g_num_sms * 16), 256, 0, s>>>(g, order, k, hoff, st.hb,
                                                                     rank_of, hcol);
    LV_LAUNCH_CHECK();
    trace_stamp(s, 6);
    static int core_bps = 0, top_cluster = 0;
    const int top_smem = kTopMax * (int)sizeof(int);
    if (!core_bps) {
        LV_CUDA(cudaFuncSetAttribute(jp_core_top_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     top_smem));
        LV_CUDA(cudaFuncSetAttribute(jp_core_top_kernel,
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        // the largest cluster (up to kTopMaxCluster blocks) that fits
        for (int c = kTopMaxCluster; c >= 1 && !top_cluster; c >>= 1) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(c);
            q.blockDim = dim3(kTopThreads);
            q.dynamicSmemBytes = top_smem;
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = c;
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            q.attrs = qa;
            q.numAttrs = 1;
            int fit = 0;
            if (cudaOccupancyMaxActiveClusters(&fit, jp_core_top_kernel, &q) == cudaSuccess && fit >= 1)
                top_cluster = c;
            else
                cudaGetLastError();
        }
        if (!top_cluster) return LV_ERR_CUDA;
        LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&core_bps, jp_core_kernel,
                                                              kCoreBlock, 0));
        if (core_bps < 1) return LV_ERR_CUDA;
    }
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(top_cluster);
        cfg.blockDim = dim3(kTopThreads);
        cfg.dynamicSmemBytes = top_smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = top_cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const int32_t *hoff_t = hoff, *hcol_t = hcol;
        LV_CUDA(cudaLaunchKernelEx(&cfg, jp_core_top_kernel, order, hoff_t, hcol_t, k, rc, r1, st));
        LV_LAUNCH_CHECK();
    }
    trace_stamp(s, 13);
    const int grid = (sms > 0 && sms < g_num_sms ? sms : g_num_sms) * core_bps;
    JpState sarg = st;
    const int32_t *hoff_c = hoff, *hcol_c = hcol, *r1_c = r1;
    int32_t *rc_c = rc;
    int karg = k;
    void *args[] = {&order, &hoff_c, &hcol_c, &karg, &rc_c, &r1_c, &sarg};
    LV_CUDA(cudaLaunchCooperativeKernel((void *)jp_core_kernel, dim3(grid), dim3(kCoreBlock), args,
                                        0, s));
    LV_LAUNCH_CHECK();
    dfree(keys, s);
    dfree(keys_alt, s);
    dfree(vals, s);
    dfree(vals_alt, s);
    dfree(dkeys, s);
    dfree(dkeys_alt, s);
    dfree(count, s);
    dfree(hoff, s);
    dfree(hcol, s);
    dfree(rank_of, s);
    dfree(rc, s);
    dfree(r1, s);
    return LV_OK;
}

}  // namespace

lv_status jp_color(const DGraph &g, uint64_t seed, bool degree_first, int32_t *color,
                   int32_t *num_colors, int32_t *rounds, int *pinned, cudaStream_t s, int sms) {
    const int n = g.n;
    JpState st;
    st.color = color;
    st.tb = trace_buffer();
    // higher-priority bit of every arc, and the degrees of the priority
    const size_t words = (size_t)g.A / 32 + 2;
    unsigned *hb = nullptr;
    int32_t *d = nullptr;
    LV_TRY(dalloc_n(&hb, words, s));
    LV_CUDA(cudaMemsetAsync(hb, 0, sizeof(unsigned) * words, s));
    if (degree_first) {
        LV_TRY(dalloc_n(&d, (size_t)n, s));
        nbdeg_kernel<<<grid_for(n, 256, g_num_sms * 16), 256, 0, s>>>(g, d);
        LV_LAUNCH_CHECK();
    }
    st.hb = hb;
    LV_TRY(dalloc_n(&st.cnt, (size_t)n, s));
    for (int k = 0; k < kJpKinds; ++k)
        for (int p = 0; p < 2; ++p) LV_TRY(dalloc_n(&st.list[k][p], (size_t)n, s));
    const size_t max_huge = (size_t)g.A / kJpHuge + 1;  // each has >= kJpHuge arcs
    LV_TRY(dalloc_n(&st.huge_bm, 32 * max_huge, s));
    LV_CUDA(cudaMemsetAsync(st.huge_bm, 0, sizeof(unsigned) * 32 * max_huge, s));
    LV_TRY(dalloc_n(&st.huge_done, max_huge, s));
    LV_CUDA(cudaMemsetAsync(st.huge_done, 0, sizeof(int32_t) * max_huge, s));
    // counts[3 * kJpKinds = 12], max_color, barrier (2 words at byte 56,
    // 8-byte aligned), rounds
    static_assert(3 * kJpKinds == 12, "state layout");
    int32_t *small_state = nullptr;
    LV_TRY(dalloc_n(&small_state, 20, s));
    LV_CUDA(cudaMemsetAsync(small_state, 0, 20 * sizeof(int32_t), s));
    st.counts = small_state;
    st.max_color = small_state + 13;
    st.bar = reinterpret_cast<GridBarrier *>(small_state + 14);
    st.rounds = small_state + 16;
    // the core: the smallest T = 2^b >= 64 with at most kCoreMax vertices of
    // degree >= T (none without the degree in the priority)
    int core_t = INT_MAX, core_k = 0;
    trace_stamp(s, 1);
    if (degree_first) {
        int32_t *hist = nullptr;
        LV_TRY(dalloc_n(&hist, 32, s));
        LV_CUDA(cudaMemsetAsync(hist, 0, 32 * sizeof(int32_t), s));
        core_hist_kernel<<<grid_for(n, 256, g_num_sms * 8), 256, 0, s>>>(d, n, hist);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(pinned, hist, 32 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        dfree(hist, s);
        int64_t above = 0;  // vertices of degree >= 2^b, b descending
        int64_t at_least[33] = {};
        for (int b = 31; b >= 0; --b) at_least[b] = above += pinned[b];
        for (int b = kCoreMinLog; b < 31; ++b)
            if (at_least[b] <= kCoreMax) {
                if (at_least[b] > 0) {
                    core_t = 1 << b;
                    core_k = (int)at_least[b];
                }
                break;
            }
    }
    trace_stamp(s, 2);
    jp_init_kernel<<<grid_for(n, 8, g_num_sms * 16), 256, 0, s>>>(g, seed, d, core_t, hb, st);
    LV_LAUNCH_CHECK();
    jp_round0_kernel<<<grid_for(n, 256 * kR0PerThread, g_num_sms * 8), 256, 0, s>>>(g, d, core_t,
                                                                                     st);
    LV_LAUNCH_CHECK();
    trace_stamp(s, 3);
    if (core_k > 0) LV_TRY(core_pass(g, seed, d, core_k, core_t, st, pinned, s, sms));
    trace_stamp(s, 7);
    static int blocks_per_sm = 0;
    const int stage_bytes = (int)sizeof(JpStage);
    if (!blocks_per_sm) {
        LV_CUDA(cudaFuncSetAttribute(jp_persistent_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, stage_bytes));
        LV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, jp_persistent_kernel,
                                                              kJpBlock, stage_bytes));
        if (blocks_per_sm < 1) return LV_ERR_CUDA;
    }
    DGraph garg = g;
    void *args[] = {&garg, &st};
    // one block per SM: a second one per SM only adds barrier arrivals
    const int grid = sms > 0 && sms < g_num_sms ? sms : g_num_sms;
    LV_CUDA(cudaLaunchCooperativeKernel((void *)jp_persistent_kernel, dim3(grid),
                                        dim3(kJpBlock), args, stage_bytes, s));
    LV_LAUNCH_CHECK();
    trace_stamp(s, 8);
    LV_CUDA(cudaMemcpyAsync(pinned, small_state + 13, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            s));
    LV_CUDA(cudaStreamSynchronize(s));
    GridBarrier bar;
    std::memcpy(&bar, pinned + 1, sizeof bar);
    if (barrier_flags(bar) & 1) return LV_ERR_TIMEOUT;
    if (barrier_flags(bar) != 0) return LV_ERR_STATE;
    *num_colors = pinned[0] + 1;
    *rounds = pinned[3];
    dfree(st.cnt, s);
    for (int k = 0; k < kJpKinds; ++k)
        for (int p = 0; p < 2; ++p) dfree(st.list[k][p], s);
    dfree(st.huge_bm, s);
    dfree(st.huge_done, s);
    dfree(small_state, s);
    dfree(hb, s);
    dfree(d, s);
    return LV_OK;
}

lv_status bucket_vertices(const DGraph &g, const int32_t *color, int32_t classes,
                          const BinLimits &lim, Buckets *b, int *pinned, cudaStream_t s) {
    const int n = g.n;
    const int nb = classes * (kBins + 1);
    b->classes = classes;
    trace_stamp(s, 9);
    uint32_t *keys = nullptr, *keys_alt = nullptr, *vals_alt = nullptr;
    LV_TRY(dalloc_n(&keys, (size_t)n, s));
    LV_TRY(dalloc_n(&keys_alt, (size_t)n, s));
    LV_TRY(dalloc_n(&vals_alt, (size_t)n, s));
    LV_TRY(dalloc_n(&b->order, (size_t)n, s));
    LV_TRY(dalloc_n(&b->bucket_off, (size_t)nb + 1, s));
    const int grid = grid_for(n, 256, g_num_sms * 16);
    bucket_key_kernel<<<grid, 256, 0, s>>>(g, color, lim, keys, reinterpret_cast<uint32_t *>(b->order));
    LV_LAUNCH_CHECK();
    LV_TRY(radix_sort_u32(keys, reinterpret_cast<uint32_t *>(b->order), keys_alt, vals_alt, n,
                          bits_for((uint64_t)nb - 1), s));
    LV_CUDA(cudaMemsetAsync(b->bucket_off, 0, sizeof(int32_t) * ((size_t)nb + 1), s));
    bucket_count_kernel<<<grid, 256, 0, s>>>(keys, n, b->bucket_off);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(b->bucket_off, b->bucket_off, nb, s));
    b->host_off = new int32_t[(size_t)nb + 1];
    LV_CUDA(cudaMemcpyAsync(b->host_off, b->bucket_off, sizeof(int32_t) * ((size_t)nb + 1),
                            cudaMemcpyDeviceToHost, s));
    // hub tables: slots, occupied lists, arc chunks
    LV_TRY(dalloc_n(&b->hub_off, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&b->hub_chunk_off, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&b->hub_chunk_at, (size_t)nb + 1, s));
    int32_t *chunk_at = b->hub_chunk_at;
    b->hub_factor = lim.hub_factor > 0 ? lim.hub_factor : hub_table_factor(color != nullptr);
    b->blocks_per_sm = lim.blocks_per_sm;
    b->sms = lim.sms;
    b->host_chunk = new int32_t[(size_t)nb + 1];
    auto size_hubs = [&]() -> lv_status {
        hub_size_kernel<<<grid, 256, 0, s>>>(g, b->order, lim.cta_max, b->hub_factor, keys,
                                             b->hub_shift, b->hub_off, b->hub_chunk_off);
        LV_LAUNCH_CHECK();
        LV_TRY(scan_excl_i32(b->hub_off, b->hub_off, n, s));
        LV_TRY(scan_excl_i32(b->hub_chunk_off, b->hub_chunk_off, n, s));
        gather_at_kernel<<<grid_for(nb + 1, 256, 1024), 256, 0, s>>>(
            b->hub_chunk_off, b->bucket_off, nb + 1, chunk_at);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(b->host_chunk, chunk_at, sizeof(int32_t) * ((size_t)nb + 1),
                                cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaMemcpyAsync(pinned, b->hub_off + n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                s));
        LV_CUDA(cudaStreamSynchronize(s));
        return LV_OK;
    };
    trace_stamp(s, 10);
    LV_TRY(size_hubs());
    trace_stamp(s, 11);
    // classes whose hubs have more chunks than the sweep grid has blocks take
    // chunks twice as long: half the block items and global-table merges
    {
        const int gsz = sweep_grid(*b);
        std::vector<uint8_t> wide((size_t)classes, 0);
        bool any = false;
        for (int c = 0; c < classes; ++c) {
            const size_t h = (size_t)c * (kBins + 1) + kBinHub;
            const int nch = b->host_chunk[h + 1] - b->host_chunk[h];
            if (nch > LV_HUB_WIDE_AT * gsz) wide[c] = 1, any = true;
        }
        if (any) {
            LV_TRY(dalloc_n(&b->hub_shift, (size_t)classes, s));
            LV_CUDA(cudaMemcpyAsync(b->hub_shift, wide.data(), (size_t)classes,
                                    cudaMemcpyHostToDevice, s));
            LV_TRY(size_hubs());
        }
    }
    b->hub_slots = pinned[0];
    if (b->hub_slots > 0) {
        LV_TRY(dalloc_n(&b->hub_table, (size_t)b->hub_slots, s));
        LV_TRY(dalloc_n(&b->hub_occ, (size_t)b->hub_slots, s));
        LV_TRY(dalloc_n(&b->hub_cnt, (size_t)n, s));
        LV_CUDA(cudaMemsetAsync(b->hub_cnt, 0, sizeof(int32_t) * (size_t)n, s));
        LV_TRY(dalloc_n(&b->hub_done, (size_t)n, s));
        LV_CUDA(cudaMemsetAsync(b->hub_done, 0, sizeof(int32_t) * (size_t)n, s));
        LV_TRY(dalloc(&b->hub_part, hub_part_bytes() * (b->host_chunk[nb] + 1), s));
        fill_empty_kernel<<<grid_for(b->hub_slots, 256, g_num_sms * 8), 256, 0, s>>>(b->hub_table,
                                                                                   b->hub_slots);
        LV_LAUNCH_CHECK();
    }
    dfree(keys, s);
    dfree(keys_alt, s);
    dfree(vals_alt, s);
    trace_stamp(s, 12);
    return LV_OK;
}

void free_buckets(Buckets &b, cudaStream_t s) {
    dfree(b.order, s);
    dfree(b.bucket_off, s);
    dfree(b.hub_off, s);
    dfree(b.hub_table, s);
    dfree(b.hub_occ, s);
    dfree(b.hub_cnt, s);
    dfree(b.hub_chunk_off, s);
    dfree(b.hub_chunk_at, s);
    dfree(b.hub_shift, s);
    dfree(b.hub_part, s);
    dfree(b.hub_done, s);
    delete[] b.host_off;
    delete[] b.host_chunk;
    b = Buckets();
}

}  // namespace lv
