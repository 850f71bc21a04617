// lv_rebuild.cu -- graph rebuild between phases (Sec. 4.4 step 4, Sec. 4.5).
//
// (i)  non-empty communities are renumbered by an exclusive scan of
//      (|C| > 0) in ascending label order (the paper's "prefix computation");
// (ii) every stored arc (u, v, w) becomes (c'(u), c'(v), w) with
//      c' = newid[C(.)]; the arcs are radix-sorted by the 64-bit key
//      c'(u) * 2^b + c'(v) and equal keys are summed (segmented reduce), so
//      a community's self-loop is the sum over its directed intra arcs and
//      each coarse row lists its neighbours in ascending order.
// All sums are integer, so the coarse graph is identical on every run.
#include <algorithm>

#include "lv_ops.cuh"

namespace lv {
namespace {

__global__ void nonempty_kernel(int n, const unsigned long long *__restrict__ comm, int32_t *flag) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        flag[c] = comm_size(comm[c]) > 0 ? 1 : 0;
}

__global__ void compose_kernel(int n_orig, int32_t *map, const int32_t *__restrict__ C,
                               const int32_t *__restrict__ newid, int32_t *labels) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n_orig; v += gridDim.x * blockDim.x) {
        const int x = newid[C[map[v]]];
        map[v] = x;
        labels[v] = x;
    }
}

__global__ void cmap_kernel(int n, const int32_t *__restrict__ C, const int32_t *__restrict__ newid,
                            uint32_t *cm) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        cm[v] = (uint32_t)newid[C[v]];
}

__global__ void heads_kernel(const uint64_t *__restrict__ keys, int A, int32_t *head) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < A; e += gridDim.x * blockDim.x)
        head[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// ---------------------------------------------------------------- grouped
// Coarse rows from the members of each community (the same coarse graph as
// the sort of all arcs, which is kept for communities with many arcs):
// vertices are grouped by coarse id (a radix sort of n keys instead of A),
// then each community's arcs (its members' rows, concatenated) are summed
// per neighbouring community in a shared-memory table, the distinct
// neighbours are ranked (ascending) and written to the community's slice of a
// scratch array, and a scan of the distinct counts packs the rows.
constexpr int kGrpWarps = 8;          // warps per block of the grouped kernels
constexpr int kGrpWarpArcs = 256;     // communities with at most this many arcs: one warp
constexpr int kGrpWarpSlots = 512;    // its table (power of two, 2x the arcs)
constexpr int kGrpBlockArcs = 1024;   // at most this many: one block (larger: the sort)
constexpr int kGrpBlockSlots = 2048;
constexpr int kGrpBlockThreads = 512;
// larger communities up to kGrpBigArcs arcs: one block walks the members'
// rows into a table of kGrpBigSlots; a community with more than
// kGrpBigDistinct distinct neighbouring communities, or more arcs (one block
// would be the critical path of the whole rebuild), takes the sort instead
constexpr int kGrpBigSlots = 4096;
constexpr int kGrpBigDistinct = kGrpBigSlots / 2;
constexpr int kGrpBigThreads = 512;
constexpr int kGrpBigArcs = 1 << 16;
constexpr int kGrpBigChunk = 2048;  // arcs per step of a large community

__global__ void group_starts_kernel(int n, const uint32_t *__restrict__ cm_sorted, int n_next,
                                    int32_t *gs) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (j == 0 || cm_sorted[j] != cm_sorted[j - 1]) gs[cm_sorted[j]] = j;
        if (j == 0) gs[n_next] = n;
    }
}

__global__ void member_deg_kernel(int n, const uint32_t *__restrict__ vo, const int32_t *__restrict__ off,
                                  int32_t *deg) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int u = (int)vo[j];
        deg[j] = off[u + 1] - off[u];
    }
}

// class of each community: 0 warp, 1 block, 2 sort; flags of classes 1 and 2
__global__ void group_class_kernel(int n_next, const int32_t *__restrict__ ga, int32_t *f_mid,
                                   int32_t *f_big, int32_t *big_arcs) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_next; c += gridDim.x * blockDim.x) {
        const int na = ga[c + 1] - ga[c];
        f_mid[c] = na > kGrpWarpArcs && na <= kGrpBlockArcs ? 1 : 0;
        f_big[c] = na > kGrpBlockArcs ? 1 : 0;
        big_arcs[c] = na > kGrpBlockArcs ? na : 0;
    }
}

__global__ void list_kernel(int n, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                            int32_t *list) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        if (flag[c]) list[pos[c]] = c;
}

// the k-th arc (0-based) of community c's concatenated member rows
__device__ __forceinline__ int2 group_arc(const DGraph &g, const uint32_t *__restrict__ vo,
                                          const int32_t *__restrict__ apos, int m0, int m1, int a0,
                                          int k) {
    int lo = m0, hi = m1;  // apos[lo] <= a0 + k < apos[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (apos[mid] <= a0 + k) lo = mid; else hi = mid;
    }
    const int u = (int)vo[lo];
    return g.arcs[g.off[u] + (a0 + k - apos[lo])];
}

// communities with at most kGrpWarpArcs arcs, one warp each
__global__ void __launch_bounds__(kGrpWarps * 32) group_warp_kernel(
    DGraph g, int n_next, const int32_t *__restrict__ gs, const int32_t *__restrict__ ga,
    const int32_t *__restrict__ apos, const uint32_t *__restrict__ vo, const uint32_t *__restrict__ cm,
    int2 *tmp, int32_t *cnt, int *err) {
    __shared__ int key[kGrpWarps][kGrpWarpSlots];
    __shared__ int val[kGrpWarps][kGrpWarpSlots];
    constexpr int kPer = kGrpWarpSlots / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *K = key[w], *V = val[w];
    const unsigned lt = (1u << lane) - 1u;
    for (int c = blockIdx.x * kGrpWarps + w; c < n_next; c += gridDim.x * kGrpWarps) {
        const int a0 = ga[c], na = ga[c + 1] - a0;
        if (na > kGrpWarpArcs) continue;  // warp-uniform
        const int m0 = gs[c], m1 = gs[c + 1];
        for (int sl = lane; sl < kGrpWarpSlots; sl += 32) {
            K[sl] = kEmpty;
            V[sl] = 0;
        }
        __syncwarp();
        for (int k = lane; k < na; k += 32) {
            const int2 a = group_arc(g, vo, apos, m0, m1, a0, k);
            unsigned h = hash32((int)cm[a.x]) & (kGrpWarpSlots - 1);
            const int cv = (int)cm[a.x];
            bool done = false;
            for (int probe = 0; probe < kGrpWarpSlots && !done; ++probe) {
                const int prev = atomicCAS(&K[h], kEmpty, cv);
                if (prev == kEmpty || prev == cv) {
                    atomicAdd(&V[h], a.y);
                    done = true;
                }
                h = (h + 1) & (kGrpWarpSlots - 1);
            }
            if (!done) atomicExch(err, 1);
        }
        __syncwarp();
        // pack the occupied slots to the front of the table
        int kr[kPer], vr[kPer], d = 0;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            kr[t] = K[t * 32 + lane];
            vr[t] = V[t * 32 + lane];
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const unsigned bm = __ballot_sync(0xffffffffu, kr[t] != kEmpty);
            if (kr[t] != kEmpty) {
                K[d + __popc(bm & lt)] = kr[t];
                V[d + __popc(bm & lt)] = vr[t];
            }
            d += __popc(bm);
        }
        __syncwarp();
        // rank (ascending neighbour) and write the row into c's slice
        for (int x = lane; x < d; x += 32) {
            const int kx = K[x];
            int r = 0;
            for (int y = 0; y < d; ++y) r += K[y] < kx ? 1 : 0;
            tmp[a0 + r] = make_int2(kx, V[x]);
        }
        if (lane == 0) cnt[c] = d;
        __syncwarp();
    }
}

// communities with kGrpWarpArcs < arcs <= kGrpBlockArcs, one block each
__global__ void __launch_bounds__(kGrpBlockThreads) group_block_kernel(
    DGraph g, int n_list, const int32_t *__restrict__ list, const int32_t *__restrict__ gs,
    const int32_t *__restrict__ ga, const int32_t *__restrict__ apos, const uint32_t *__restrict__ vo,
    const uint32_t *__restrict__ cm, int2 *tmp, int32_t *cnt, int *err) {
    __shared__ int K[kGrpBlockSlots], V[kGrpBlockSlots];
    __shared__ int s_d;
    constexpr int kPer = kGrpBlockSlots / kGrpBlockThreads;
    for (int li = blockIdx.x; li < n_list; li += gridDim.x) {
        const int c = list[li];
        const int a0 = ga[c], na = ga[c + 1] - a0;
        const int m0 = gs[c], m1 = gs[c + 1];
        for (int sl = threadIdx.x; sl < kGrpBlockSlots; sl += kGrpBlockThreads) {
            K[sl] = kEmpty;
            V[sl] = 0;
        }
        if (threadIdx.x == 0) s_d = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < na; k += kGrpBlockThreads) {
            const int2 a = group_arc(g, vo, apos, m0, m1, a0, k);
            const int cv = (int)cm[a.x];
            unsigned h = hash32(cv) & (kGrpBlockSlots - 1);
            bool done = false;
            for (int probe = 0; probe < kGrpBlockSlots && !done; ++probe) {
                const int prev = atomicCAS(&K[h], kEmpty, cv);
                if (prev == kEmpty || prev == cv) {
                    atomicAdd(&V[h], a.y);
                    done = true;
                }
                h = (h + 1) & (kGrpBlockSlots - 1);
            }
            if (!done) atomicExch(err, 1);
        }
        __syncthreads();
        int kr[kPer], vr[kPer];
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            kr[t] = K[t * kGrpBlockThreads + threadIdx.x];
            vr[t] = V[t * kGrpBlockThreads + threadIdx.x];
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kPer; ++t)
            if (kr[t] != kEmpty) {
                const int at = atomicAdd(&s_d, 1);  // order is fixed by the ranking below
                K[at] = kr[t];
                V[at] = vr[t];
            }
        __syncthreads();
        const int d = s_d;
        for (int x = threadIdx.x; x < d; x += kGrpBlockThreads) {
            const int kx = K[x];
            int r = 0;
            for (int y = 0; y < d; ++y) r += K[y] < kx ? 1 : 0;
            tmp[a0 + r] = make_int2(kx, V[x]);
        }
        if (threadIdx.x == 0) cnt[c] = d;
        __syncthreads();
    }
}

// communities with kGrpBlockArcs < arcs <= kGrpBigArcs, one block each: warps take
// member rows, lanes their arcs; each arc's neighbouring community is summed
// in a shared-memory table.  When the distinct neighbours stay within
// kGrpBigDistinct they are sorted ascending (bitonic, in shared memory) and
// written to the community's slice of tmp; otherwise fail[c] = 1 and the
// community goes to the sort of its arcs.
__global__ void __launch_bounds__(kGrpBigThreads) group_big_kernel(
    DGraph g, int n_list, const int32_t *__restrict__ list, const int32_t *__restrict__ gs,
    const int32_t *__restrict__ ga, const int32_t *__restrict__ apos,
    const uint32_t *__restrict__ vo, const uint32_t *__restrict__ cm, int2 *tmp, int32_t *cnt,
    int32_t *fail) {
    // the table (keys, then values) and, once its entries are in registers,
    // the sort buffer of up to kGrpBigDistinct packed (key, value) pairs
    __shared__ unsigned long long KV[kGrpBigSlots];
    __shared__ int mo[kGrpBigChunk + 1];  // arc starts of the chunk's members
    __shared__ int s_d, s_over, s_mlo, s_nm;
    int *K = reinterpret_cast<int *>(KV), *V = K + kGrpBigSlots;
    unsigned long long *S = KV;
    static_assert(2 * kGrpBigSlots * sizeof(int) == sizeof(KV) && kGrpBigDistinct <= kGrpBigSlots,
                  "table and sort buffer share the array");
    constexpr int kPer = kGrpBigSlots / kGrpBigThreads;
    for (int li = blockIdx.x; li < n_list; li += gridDim.x) {
        const int c = list[li];
        const int a0 = ga[c], m0 = gs[c], m1 = gs[c + 1];
        if (ga[c + 1] - a0 > kGrpBigArcs) {  // block-uniform
            if (threadIdx.x == 0) fail[c] = 1;
            continue;
        }
        for (int sl = threadIdx.x; sl < kGrpBigSlots; sl += kGrpBigThreads) {
            K[sl] = kEmpty;
            V[sl] = 0;
        }
        if (threadIdx.x == 0) {
            s_d = 0;
            s_over = 0;
        }
        __syncthreads();
        // the community's arcs in chunks of kGrpBigChunk, one thread per arc:
        // its member by a search of the chunk's members' arc starts in
        // shared memory (a warp per member row idled on rows of a few arcs)
        const int a1 = ga[c + 1];
        for (int p0 = a0; p0 < a1; p0 += kGrpBigChunk) {
            const int p1 = min(a1, p0 + kGrpBigChunk);
            if (threadIdx.x < 2) {  // members holding positions p0 and p1 - 1
                const int p = threadIdx.x ? p1 - 1 : p0;
                int l = m0, h = m1;  // apos[l] <= p < apos[h]
                while (h - l > 1) {
                    const int mid = (l + h) >> 1;
                    if (apos[mid] <= p) l = mid; else h = mid;
                }
                if (threadIdx.x) s_nm = l; else s_mlo = l;
            }
            __syncthreads();
            const int mlo = s_mlo, nm = s_nm + 1 - s_mlo;
            const bool local = nm <= kGrpBigChunk;  // else members without arcs
            if (local)
                for (int t = threadIdx.x; t <= nm; t += kGrpBigThreads) mo[t] = apos[mlo + t];
            __syncthreads();
            for (int p = p0 + (int)threadIdx.x; p < p1; p += kGrpBigThreads) {
                int2 a;
                if (local) {
                    int l = 0, h = nm;  // mo[l] <= p < mo[h]
                    while (h - l > 1) {
                        const int mid = (l + h) >> 1;
                        if (mo[mid] <= p) l = mid; else h = mid;
                    }
                    const int u = (int)vo[mlo + l];
                    a = g.arcs[g.off[u] + (p - mo[l])];
                } else {
                    a = group_arc(g, vo, apos, m0, m1, a0, p - a0);
                }
                const int cv = (int)cm[a.x];
                unsigned h = hash32(cv) & (kGrpBigSlots - 1);
                bool done = false;
                for (int probe = 0; probe < kGrpBigSlots && !done; ++probe) {
                    const int prev = atomicCAS(&K[h], kEmpty, cv);
                    if (prev == kEmpty || prev == cv) {
                        atomicAdd(&V[h], a.y);
                        if (prev == kEmpty && atomicAdd(&s_d, 1) >= kGrpBigDistinct)
                            s_over = 1;
                        done = true;
                    }
                    h = (h + 1) & (kGrpBigSlots - 1);
                }
                if (!done) s_over = 1;
            }
            __syncthreads();
            if (s_over) break;  // block-uniform after the barrier
        }
        __syncthreads();
        if (s_over) {  // block-uniform
            if (threadIdx.x == 0) fail[c] = 1;
            __syncthreads();
            continue;
        }
        const int d = s_d;
        int kr[kPer], vr[kPer];
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            kr[t] = K[t * kGrpBigThreads + threadIdx.x];
            vr[t] = V[t * kGrpBigThreads + threadIdx.x];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_d = 0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kPer; ++t)
            if (kr[t] != kEmpty) {
                const int at = atomicAdd(&s_d, 1);  // the sort below fixes the order
                S[at] = ((unsigned long long)(unsigned)kr[t] << 32) | (unsigned)vr[t];
            }
        int P = 1;
        while (P < d) P <<= 1;
        for (int x = d + threadIdx.x; x < P; x += kGrpBigThreads) S[x] = ~0ull;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int x = threadIdx.x; x < P; x += kGrpBigThreads) {
                    const int y = x ^ j;
                    if (y > x) {
                        const unsigned long long sx = S[x], sy = S[y];
                        if ((sx > sy) == ((x & k) == 0)) {
                            S[x] = sy;
                            S[y] = sx;
                        }
                    }
                }
                __syncthreads();
            }
        for (int x = threadIdx.x; x < d; x += kGrpBigThreads)
            tmp[a0 + x] = make_int2((int)(S[x] >> 32), (int)(unsigned)S[x]);
        if (threadIdx.x == 0) cnt[c] = d;
        __syncthreads();
    }
}

// arcs of the communities that failed the block path (0 for the others)
__global__ void fail_arcs_kernel(int n_next, const int32_t *__restrict__ ga,
                                 const int32_t *__restrict__ fail, int32_t *fail_arcs) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_next; c += gridDim.x * blockDim.x)
        fail_arcs[c] = fail[c] ? ga[c + 1] - ga[c] : 0;
}

// Communities left to the sort: their arcs as keys (c << b | c(v)) with
// weights, pre-summed per block.  A block takes a chunk of kAggArcs
// consecutive arcs of one community (chunks numbered over the listed
// communities: coff holds the first chunk of each, coff[n_list] the total),
// finds the members holding the chunk's first and last arcs, loads those
// members' arc starts into shared memory and maps each arc to its member by
// a search there (not over all of the community's members in global
// memory).  It sums equal keys in a shared-memory table and appends each
// distinct key once (at a position reserved with one atomic per block), so
// the sort sees the distinct (community, neighbour) pairs of each chunk
// instead of every arc.
constexpr int kAggArcs = 4096;
constexpr int kAggSlots = 2 * kAggArcs;
constexpr int kAggThreads = 512;
constexpr size_t kAggSmem = kAggSlots * 2 * sizeof(unsigned) + (kAggArcs + 1) * sizeof(int);

// chunks of kAggArcs arcs of each listed community
__global__ void agg_chunks_kernel(int n_list, const int32_t *__restrict__ list,
                                  const int32_t *__restrict__ ga, int32_t *chunks) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_list; i += gridDim.x * blockDim.x) {
        const int c = list[i];
        chunks[i] = (ga[c + 1] - ga[c] + kAggArcs - 1) / kAggArcs;
    }
}

__global__ void __launch_bounds__(kAggThreads) group_keys_kernel(
    DGraph g, int n_list, const int32_t *__restrict__ list, const int32_t *__restrict__ coff,
    const int32_t *__restrict__ gs, const int32_t *__restrict__ ga,
    const int32_t *__restrict__ apos, const uint32_t *__restrict__ vo, const uint32_t *__restrict__ cm,
    int b, uint64_t *keys, uint32_t *vals, int32_t *n_out, int *err) {
    // a chunk's arcs all belong to one community, so the table keys are the
    // neighbours' communities alone (32 bits); the 64-bit key is formed on
    // the way out
    extern __shared__ unsigned agg[];
    unsigned *K = agg;
    unsigned *V = agg + kAggSlots;
    int *mo = reinterpret_cast<int *>(V + kAggSlots);  // arc starts of the chunk's members
    __shared__ int s_cnt, s_base, s_c, s_p0, s_p1, s_m0, s_nm;
    constexpr int kPer = kAggSlots / kAggThreads;
    constexpr unsigned kNone = ~0u;  // community ids are below 2^31
    const int n_chunks = coff[n_list];
    for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_list;  // coff[lo] <= chunk < coff[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (coff[mid] <= chunk) lo = mid; else hi = mid;
            }
            const int c = list[lo], a0 = ga[c];
            const int p0 = a0 + (chunk - coff[lo]) * kAggArcs;
            const int p1 = min(ga[c + 1], p0 + kAggArcs);
            // members holding arc positions p0 and p1 - 1 (apos[m] <= p < apos[m + 1])
            int m[2];
            for (int q = 0; q < 2; ++q) {
                const int p = q ? p1 - 1 : p0;
                int l = gs[c], h = gs[c + 1];
                while (h - l > 1) {
                    const int mid = (l + h) >> 1;
                    if (apos[mid] <= p) l = mid; else h = mid;
                }
                m[q] = l;
            }
            s_c = c;
            s_p0 = p0;
            s_p1 = p1;
            s_m0 = m[0];
            s_nm = m[1] + 1 - m[0];
            s_cnt = 0;
        }
        __syncthreads();
        const int c = s_c, p0 = s_p0, p1 = s_p1, m0 = s_m0, nm = s_nm;
        // table: the next power of two >= 2x the chunk's arcs (a short last
        // chunk clears and scans only that much)
        int tsz = kAggThreads;
        while (tsz < 2 * (p1 - p0)) tsz <<= 1;
        const unsigned tmask = (unsigned)tsz - 1u;
        for (int sl = threadIdx.x; sl < tsz; sl += kAggThreads) {
            K[sl] = kNone;
            V[sl] = 0u;
        }
        const bool local = nm <= kAggArcs;  // else members without arcs: search globally
        if (local)
            for (int t = threadIdx.x; t <= nm; t += kAggThreads) mo[t] = apos[m0 + t];
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += kAggThreads) {
            int2 a;
            if (local) {
                int lo = 0, hi = nm;  // mo[lo] <= p < mo[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (mo[mid] <= p) lo = mid; else hi = mid;
                }
                const int u = (int)vo[m0 + lo];
                a = g.arcs[g.off[u] + (p - mo[lo])];
            } else {
                a = group_arc(g, vo, apos, gs[c], gs[c + 1], ga[c], p - ga[c]);
            }
            const unsigned key = cm[a.x];
            unsigned h = hash32((int)key) & tmask;
            bool done = false;
            for (int probe = 0; probe < tsz && !done; ++probe) {
                const unsigned prev = atomicCAS(&K[h], kNone, key);
                if (prev == kNone || prev == key) {
                    atomicAdd(&V[h], (unsigned)a.y);
                    done = true;
                }
                h = (h + 1) & tmask;
            }
            if (!done) atomicExch(err, 1);  // cannot happen: 2x the slots of the keys
        }
        __syncthreads();
        const int per = tsz / kAggThreads;
        int mine = 0;
#pragma unroll
        for (int t = 0; t < kPer; ++t)
            if (t < per) mine += K[t * kAggThreads + threadIdx.x] != kNone ? 1 : 0;
        const int off = mine ? atomicAdd(&s_cnt, mine) : 0;
        __syncthreads();
        if (threadIdx.x == 0) s_base = atomicAdd(n_out, s_cnt);
        __syncthreads();
        int o = s_base + off;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int sl = t * kAggThreads + threadIdx.x;
            if (t < per && K[sl] != kNone) {
                keys[o] = ((unsigned long long)c << b) | K[sl];
                vals[o] = V[sl];
                ++o;
            }
        }
        __syncthreads();
    }
}

// first and one-past-last position of each community's keys in the sorted
// key array
__global__ void key_bounds_kernel(const uint64_t *__restrict__ keys, int n, int b,
                                  int32_t *cstart, int32_t *cend) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int c = (int)(keys[e] >> b);
        if (e == 0 || (int)(keys[e - 1] >> b) != c) cstart[c] = e;
        if (e == n - 1 || (int)(keys[e + 1] >> b) != c) cend[c] = e + 1;
    }
}

// sorted keys of the large communities: distinct (c, c(v)) summed into c's
// slice at its rank (heads counted from the community's first sorted key)
__global__ void __launch_bounds__(256) group_emit_kernel(const uint64_t *__restrict__ keys,
                                                         const uint32_t *__restrict__ vals,
                                                         const int32_t *__restrict__ head,
                                                         const int32_t *__restrict__ pos,
                                                         const int32_t *__restrict__ cstart,
                                                         const int32_t *__restrict__ ga, int AL, int b,
                                                         int2 *tmp) {
    const int lane = threadIdx.x & 31;
    const uint64_t lowmask = (1ull << b) - 1ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < AL; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < AL;
        int slot = -1 - lane;
        int w = 0;
        if (valid) {
            const uint64_t k = keys[e];
            const int c = (int)(k >> b);
            const int h = head[e];
            slot = ga[c] + (pos[e] + h - 1 - pos[cstart[c]]);
            w = (int)vals[e];
            if (h) tmp[slot].x = (int)(k & lowmask);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ws = __shfl_up_sync(0xffffffffu, w, o);
            const int ss = __shfl_up_sync(0xffffffffu, slot, o);
            if (lane >= o && ss == slot) w += ws;
        }
        const int snext = __shfl_down_sync(0xffffffffu, slot, 1);
        if (valid && (lane == 31 || snext != slot)) atomicAdd(&tmp[slot].y, w);
    }
}

__global__ void group_big_count_kernel(int n_list, const int32_t *__restrict__ list,
                                       const int32_t *__restrict__ cstart,
                                       const int32_t *__restrict__ cend,
                                       const int32_t *__restrict__ pos, int32_t *cnt) {
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < n_list; li += gridDim.x * blockDim.x) {
        const int c = list[li];
        cnt[c] = pos[cend[c]] - pos[cstart[c]];
    }
}

// pack: row c = tmp[ga[c], ga[c] + cnt[c]) at off[c]; one warp per community
// A block per chunk of kPackArcs coarse arcs: the rows the chunk touches
// are found by two searches of off, their starts loaded into shared memory,
// and each arc's row by a search there (a global search when the chunk
// touches more rows than that, i.e. many empty rows).  So a community with
// 10^5 distinct neighbours is not copied by one warp, and a batch of small
// ones does not search all of off per arc.
constexpr int kPackArcs = 4096;
__global__ void __launch_bounds__(512) group_pack_kernel(int n_next, const int32_t *__restrict__ ga,
                                                         const int32_t *__restrict__ off, int A,
                                                         const int2 *__restrict__ tmp, int2 *arcs) {
    __shared__ int so[kPackArcs + 1], sg[kPackArcs];
    __shared__ int s_c0, s_nc;
    for (int64_t e0 = (int64_t)blockIdx.x * kPackArcs; e0 < A; e0 += (int64_t)gridDim.x * kPackArcs) {
        const int e1 = (int)min((int64_t)A, e0 + kPackArcs);
        if (threadIdx.x < 2) {  // rows of the chunk's first and last arcs
            const int e = threadIdx.x ? e1 - 1 : (int)e0;
            int lo = 0, hi = n_next;  // off[lo] <= e < off[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (off[mid] <= e) lo = mid; else hi = mid;
            }
            if (threadIdx.x) s_nc = lo; else s_c0 = lo;
        }
        __syncthreads();
        const int c0 = s_c0, nc = s_nc - s_c0 + 1;
        const bool local = nc <= kPackArcs;
        if (local)
            for (int t = threadIdx.x; t <= nc; t += blockDim.x) {
                so[t] = off[c0 + t];
                if (t < nc) sg[t] = ga[c0 + t];
            }
        __syncthreads();
        for (int e = (int)e0 + threadIdx.x; e < e1; e += blockDim.x) {
            int lo, hi;
            if (local) {
                lo = 0, hi = nc;  // so[lo] <= e < so[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (so[mid] <= e) lo = mid; else hi = mid;
                }
                arcs[e] = tmp[sg[lo] + (e - so[lo])];
            } else {
                lo = 0, hi = n_next;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (off[mid] <= e) lo = mid; else hi = mid;
                }
                arcs[e] = tmp[ga[lo] + (e - off[lo])];
            }
        }
        __syncthreads();
    }
}

// device scratch freed (stream-ordered) when the set goes out of scope
struct ScratchSet {
    static constexpr int kMax = 32;
    cudaStream_t s = nullptr;
    void *p[kMax] = {};
    int k = 0;
    template <typename T>
    lv_status get(T **x, size_t count) {
        if (k >= kMax) return LV_ERR_STATE;  // more buffers than the set holds
        LV_TRY(dalloc_n(x, count, s));
        p[k++] = *x;
        return LV_OK;
    }
    ~ScratchSet() {
        for (int i = 0; i < k; ++i) dfree(p[i], s);
    }
};

__global__ void gather_idx_kernel(int G, const int32_t *__restrict__ idx,
                                  const int32_t *__restrict__ arr, int32_t *out) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
        out[g] = arr[idx[g]];
}

}  // namespace

static int grid_items(int64_t items) { return grid_for(items, 256, g_num_sms * 16); }

lv_status renumber(int32_t n, const unsigned long long *comm, int32_t *newid, cudaStream_t s) {
    nonempty_kernel<<<grid_items(n), 256, 0, s>>>(n, comm, newid);
    LV_LAUNCH_CHECK();
    return scan_excl_i32(newid, newid, n, s);
}

lv_status compose_labels(int32_t n_orig, int32_t *map, const int32_t *C, const int32_t *newid,
                         int32_t *labels, cudaStream_t s) {
    compose_kernel<<<grid_items(n_orig), 256, 0, s>>>(n_orig, map, C, newid, labels);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status coarsen(const DGraph &g, const int32_t *C, const int32_t *newid, int32_t n_next,
                  DGraph *out, int *pinned, cudaStream_t s) {
    const int n = g.n, A = g.A;
    const int b = std::max(1, bits_for((uint64_t)(n_next > 0 ? n_next - 1 : 0)));
    ScratchSet t;
    t.s = s;
    uint32_t *cm, *cms, *cm_alt, *vo, *vo_alt;
    int32_t *gs, *deg, *apos, *ga, *cnt, *f_mid, *f_big, *big_arcs, *pmid, *pbig, *lpos, *lists;
    int2 *tmp;
    int *err;
    LV_TRY(t.get(&cm, (size_t)n));
    LV_TRY(t.get(&cms, (size_t)n));
    LV_TRY(t.get(&cm_alt, (size_t)n));
    LV_TRY(t.get(&vo, (size_t)n));
    LV_TRY(t.get(&vo_alt, (size_t)n));
    LV_TRY(t.get(&gs, (size_t)n_next + 1));
    LV_TRY(t.get(&deg, (size_t)n));
    LV_TRY(t.get(&apos, (size_t)n + 1));
    LV_TRY(t.get(&ga, (size_t)n_next + 1));
    LV_TRY(t.get(&cnt, (size_t)n_next + 1));
    LV_TRY(t.get(&f_mid, (size_t)n_next + 1));
    LV_TRY(t.get(&f_big, (size_t)n_next + 1));
    LV_TRY(t.get(&big_arcs, (size_t)n_next + 1));
    LV_TRY(t.get(&pmid, (size_t)n_next + 1));
    LV_TRY(t.get(&pbig, (size_t)n_next + 1));
    LV_TRY(t.get(&lpos, (size_t)n_next + 1));
    LV_TRY(t.get(&lists, 2 * (size_t)n_next + 2));
    LV_TRY(t.get(&tmp, (size_t)std::max(A, 1)));
    LV_TRY(t.get(&err, 1));
    LV_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    LV_CUDA(cudaMemsetAsync(tmp, 0, sizeof(int2) * (size_t)A, s));
    trace_stamp(s, 20);
    // vertices grouped by coarse id (ascending id inside a group)
    cmap_kernel<<<grid_items(n), 256, 0, s>>>(n, C, newid, cm);
    LV_LAUNCH_CHECK();
    LV_CUDA(cudaMemcpyAsync(cms, cm, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    LV_TRY(iota(n, reinterpret_cast<int32_t *>(vo), s));
    LV_TRY(radix_sort_u32(cms, vo, cm_alt, vo_alt, n, b, s));
    group_starts_kernel<<<grid_items(n), 256, 0, s>>>(n, cms, n_next, gs);
    LV_LAUNCH_CHECK();
    member_deg_kernel<<<grid_items(n), 256, 0, s>>>(n, vo, g.off, deg);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(deg, apos, n, s));
    gather_idx_kernel<<<grid_items(n_next + 1), 256, 0, s>>>(n_next, gs, apos, ga);
    LV_LAUNCH_CHECK();
    // size classes
    group_class_kernel<<<grid_items(n_next), 256, 0, s>>>(n_next, ga, f_mid, f_big, big_arcs);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(f_mid, pmid, n_next, s));
    LV_TRY(scan_excl_i32(f_big, pbig, n_next, s));
    int32_t *list_mid = lists, *list_big = lists + n_next + 1;
    list_kernel<<<grid_items(n_next), 256, 0, s>>>(n_next, f_mid, pmid, list_mid);
    LV_LAUNCH_CHECK();
    list_kernel<<<grid_items(n_next), 256, 0, s>>>(n_next, f_big, pbig, list_big);
    LV_LAUNCH_CHECK();
    LV_CUDA(cudaMemcpyAsync(pinned, pmid + n_next, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(pinned + 1, pbig + n_next, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const int n_mid = pinned[0];
    int n_big = pinned[1], AL = 0;
    trace_stamp(s, 21, (unsigned long long)n_mid << 32 | (unsigned)n_big);
    // small and medium communities
    group_warp_kernel<<<grid_for(n_next, kGrpWarps, g_num_sms * 16), kGrpWarps * 32, 0, s>>>(
        g, n_next, gs, ga, apos, vo, cm, tmp, cnt, err);
    LV_LAUNCH_CHECK();
    trace_stamp(s, 22);
    if (n_mid > 0) {
        group_block_kernel<<<std::min(n_mid, g_num_sms * 4), kGrpBlockThreads, 0, s>>>(
            g, n_mid, list_mid, gs, ga, apos, vo, cm, tmp, cnt, err);
        LV_LAUNCH_CHECK();
    }
    // large communities: one block each while their distinct neighbours fit
    // its table; the others sort their arcs by (community, neighbour)
    if (n_big > 0) {
        trace_stamp(s, 23);
        int32_t *fail = f_big;  // reused: one flag per community
        LV_CUDA(cudaMemsetAsync(fail, 0, sizeof(int32_t) * ((size_t)n_next + 1), s));
        group_big_kernel<<<std::min(n_big, g_num_sms * 4), kGrpBigThreads, 0, s>>>(
            g, n_big, list_big, gs, ga, apos, vo, cm, tmp, cnt, fail);
        LV_LAUNCH_CHECK();
        trace_stamp(s, 24);
        fail_arcs_kernel<<<grid_items(n_next), 256, 0, s>>>(n_next, ga, fail, big_arcs);
        LV_LAUNCH_CHECK();
        LV_TRY(scan_excl_i32(fail, pbig, n_next, s));
        LV_TRY(scan_excl_i32(big_arcs, lpos, n_next, s));
        list_kernel<<<grid_items(n_next), 256, 0, s>>>(n_next, fail, pbig, list_big);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(pinned, pbig + n_next, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaMemcpyAsync(pinned + 1, lpos + n_next, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                s));
        LV_CUDA(cudaStreamSynchronize(s));
        n_big = pinned[0];
        AL = pinned[1];
        trace_stamp(s, 25, (unsigned long long)n_big << 32 | (unsigned)AL);
    }
    if (n_big > 0) {
        uint64_t *keys, *keys_alt;
        uint32_t *vals, *vals_alt;
        int32_t *head, *pos;
        LV_TRY(t.get(&keys, (size_t)AL));
        LV_TRY(t.get(&keys_alt, (size_t)AL));
        LV_TRY(t.get(&vals, (size_t)AL));
        LV_TRY(t.get(&vals_alt, (size_t)AL));
        int32_t *coff;  // first chunk of each listed community; coff[n_big] = all chunks
        LV_TRY(t.get(&coff, (size_t)n_big + 1));
        agg_chunks_kernel<<<grid_items(n_big), 256, 0, s>>>(n_big, list_big, ga, coff);
        LV_LAUNCH_CHECK();
        LV_TRY(scan_excl_i32(coff, coff, n_big, s));
        int32_t *n_keys;
        LV_TRY(t.get(&n_keys, 1));
        LV_CUDA(cudaMemsetAsync(n_keys, 0, sizeof(int32_t), s));
        static bool agg_attr = false;
        if (!agg_attr) {
            LV_CUDA(cudaFuncSetAttribute(group_keys_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kAggSmem));
            agg_attr = true;
        }
        group_keys_kernel<<<grid_for((int64_t)AL + (int64_t)n_big * kAggArcs, kAggArcs,
                                     g_num_sms * 2),
                            kAggThreads, kAggSmem, s>>>(g, n_big, list_big, coff, gs, ga, apos, vo,
                                                        cm, b, keys, vals, n_keys, err);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(pinned, n_keys, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        const int NK = pinned[0];
        trace_stamp(s, 26, (unsigned)NK);
        LV_TRY(radix_sort_u64(keys, vals, keys_alt, vals_alt, NK, 2 * b, s));
        trace_stamp(s, 27);
        int32_t *cstart, *cend;
        LV_TRY(t.get(&cstart, (size_t)n_next + 1));
        LV_TRY(t.get(&cend, (size_t)n_next + 1));
        LV_TRY(t.get(&head, (size_t)NK));
        LV_TRY(t.get(&pos, (size_t)NK + 1));
        heads_kernel<<<grid_items(NK), 256, 0, s>>>(keys, NK, head);
        LV_LAUNCH_CHECK();
        key_bounds_kernel<<<grid_items(NK), 256, 0, s>>>(keys, NK, b, cstart, cend);
        LV_LAUNCH_CHECK();
        LV_TRY(scan_excl_i32(head, pos, NK, s));
        group_emit_kernel<<<grid_items(NK), 256, 0, s>>>(keys, vals, head, pos, cstart, ga, NK, b,
                                                         tmp);
        LV_LAUNCH_CHECK();
        group_big_count_kernel<<<grid_items(n_big), 256, 0, s>>>(n_big, list_big, cstart, cend,
                                                                 pos, cnt);
        LV_LAUNCH_CHECK();
    }
    trace_stamp(s, 28);
    // pack the rows
    DGraph h;
    h.n = n_next;
    LV_TRY(dalloc_n(&h.off, (size_t)n_next + 1, s));
    LV_TRY(scan_excl_i32(cnt, h.off, n_next, s));
    LV_CUDA(cudaMemcpyAsync(pinned, h.off + n_next, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(pinned + 1, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    if (pinned[1]) {
        dfree(h.off, s);
        return LV_ERR_HASH;
    }
    h.A = pinned[0];
    LV_TRY(dalloc_n(&h.arcs, (size_t)std::max(h.A, 1), s));
    group_pack_kernel<<<grid_for(h.A, kPackArcs, g_num_sms * 4), 512, 0, s>>>(n_next, ga, h.off,
                                                                              h.A, tmp, h.arcs);
    LV_LAUNCH_CHECK();
    trace_stamp(s, 29, (unsigned)h.A);
    *out = h;
    return LV_OK;
}

}  // namespace lv
