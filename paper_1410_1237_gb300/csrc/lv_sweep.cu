// lv_sweep.cu -- the vertex sweep of one iteration (Algorithm 1, Sec. 4.1).
//
// For every vertex i of the current colour class (or of the whole graph):
//   e[c]   = sum of w(i,j) over neighbours j != i with C(j) = c     (Eq. 1)
//   s(c)   = 2m e[c] - k_i a_c                                        (Eq. 4 x (2m)^2/2)
//   s_old  = 2m e[C(i)] - k_i (a_{C(i)} - k_i)
//   best   = argmax over c != C(i) of s(c), ties to the smaller label (Eq. 5)
//   move   iff s(best) - s_old > 0 and not (|C(i)| = |best| = 1 and best > C(i))
// All products are below 2^62 (2m < 2^31), so int64 holds them exactly and
// every decision is exact.  The sweep reads a snapshot: moves are appended
// to a list and applied by a second kernel after the sweep, so all vertices
// of a class decide from the state at the start of the class.
//
// Vertices are binned by degree:
//   bin 0  8 lanes per vertex, hash table of <= 64 slots in shared memory
//   bin 1  one warp per vertex, <= 512 slots in shared memory
//   bin 2  one CTA per vertex, <= 8192 slots (64 KB) in shared memory
//   bin 3  hubs: a table in global memory, filled by several CTAs per
//          vertex (chunks of kHubChunk arcs) and evaluated by one CTA
// Tables are open-addressing (linear probing) keyed by community label and
// sized to the next power of two >= 2 * degree, so the load factor is <= 1/2
// and every probe sequence ends; a probe count above the table size is an
// internal error (LV_ERR_HASH), never a hang.
#include <climits>

#include "lv_ops.cuh"

namespace lv {
namespace {

struct SweepArgs {
    const int32_t *__restrict__ off;
    const int2 *__restrict__ arcs;
    const int32_t *__restrict__ k;
    const int32_t *__restrict__ loop;
    const int32_t *__restrict__ C;
    const unsigned long long *__restrict__ comm;
    long long two_m;
    int2 *moves;
    int32_t *move_count;
    IterStats *stats;
    const int32_t *__restrict__ verts;  // vertices of this (class, bin)
    int nverts;
    int2 *hub_table;
    const int32_t *__restrict__ hub_off;  // table offset per position of `verts`
    int32_t *hub_occ;                     // occupied-slot lists (same offsets)
    int32_t *hub_cnt;                     // occupied count per position of `verts`
    const int32_t *__restrict__ hub_chunk_off;  // first arc chunk per position of `verts`
};

__device__ __forceinline__ int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// insert (c, w) into a shared-memory table of `mask + 1` slots
__device__ __forceinline__ bool smem_insert(int *key, int *val, unsigned mask, int c, int w) {
    unsigned h = hash32(c) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int cur = ((volatile int *)key)[h];
        if (cur == c) {
            atomicAdd(&val[h], w);
            return true;
        }
        if (cur == kEmpty) {
            const int prev = atomicCAS(&key[h], kEmpty, c);
            if (prev == kEmpty || prev == c) {
                atomicAdd(&val[h], w);
                return true;
            }
        }
        h = (h + 1) & mask;
    }
    return false;
}

// the same in a global-memory table of int2 {key, val}
__device__ __forceinline__ bool gmem_insert(int2 *tab, unsigned mask, int c, int w) {
    unsigned h = hash32(c) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        int *kp = &tab[h].x;
        const int cur = *((volatile int *)kp);
        if (cur == c) {
            atomicAdd(&tab[h].y, w);
            return true;
        }
        if (cur == kEmpty) {
            const int prev = atomicCAS(kp, kEmpty, c);
            if (prev == kEmpty || prev == c) {
                atomicAdd(&tab[h].y, w);
                return true;
            }
        }
        h = (h + 1) & mask;
    }
    return false;
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

// evaluate one table slot
__device__ __forceinline__ void eval_slot(const SweepArgs &a, int c, int e, int ci, int ki, Best &b,
                                          int &e_old) {
    if (c == kEmpty) return;
    if (c == ci) {
        e_old = e;
        return;
    }
    const unsigned long long cm = a.comm[c];
    best_take(b, a.two_m * (long long)e - (long long)ki * comm_a(cm), c, comm_size(cm), e);
}

// decision for vertex i given the reduced candidate; returns true on a move
__device__ __forceinline__ bool decide(const SweepArgs &a, int i, int ci, int ki, const Best &b,
                                       int e_old, long long &ein, long long &dein) {
    const unsigned long long cmi = a.comm[ci];
    const long long s_old = a.two_m * (long long)e_old - (long long)ki * (comm_a(cmi) - ki);
    ein += (long long)e_old + a.loop[i];
    if (b.c == INT_MAX) return false;
    const long long gain = b.s - s_old;
    if (gain <= 0) return false;
    if (comm_size(cmi) == 1 && b.size == 1 && b.c > ci) return false;  // singlet rule
    dein += 2ll * ((long long)b.e - e_old);
    return true;
}

__device__ __forceinline__ void flush_stats(const SweepArgs &a, long long ein, long long dein,
                                            int moved, int err) {
    __shared__ long long red[8];
    __shared__ int redi[8];
    const long long t1 = block_sum_256(ein, red);
    const long long t2 = block_sum_256(dein, red);
    const int t3 = block_sum_256(moved, redi);
    const int t4 = block_sum_256(err, redi);
    if (threadIdx.x == 0) {
        if (t1) atomicAdd(&a.stats->sum_ein, (unsigned long long)t1);
        if (t2) atomicAdd(&a.stats->delta_ein, (unsigned long long)t2);
        if (t3) atomicAdd(&a.stats->moved, t3);
        if (t4) atomicOr(&a.stats->err, 1);
    }
}

// ---------------------------------------------------------------- bins 0/1
// G lanes per vertex, up to SLOTS table slots per group.  The loop over
// vertices advances a whole warp at a time, so shuffles see full warps.
template <int G, int SLOTS>
__global__ void __launch_bounds__(256) sweep_group_kernel(SweepArgs a) {
    constexpr int GPB = 256 / G;  // groups per block
    constexpr int GPW = 32 / G;   // groups per warp
    __shared__ int skey[GPB * SLOTS];
    __shared__ int sval[GPB * SLOTS];
    const int lane = threadIdx.x & 31;
    const int gl = threadIdx.x & (G - 1);
    const int gib = threadIdx.x / G;
    int *key = skey + gib * SLOTS;
    int *val = sval + gib * SLOTS;
    const unsigned lt = (1u << lane) - 1u;
    long long ein = 0, dein = 0;
    int moved = 0, err = 0;
    const int wid = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * 8;
    for (int base = wid * GPW; base < a.nverts; base += nwarps * GPW) {
        const int vi = base + lane / G;
        const bool valid = vi < a.nverts;
        int i = 0, beg = 0, end = 0, ci = 0, ki = 0;
        unsigned mask = 0;
        if (valid) {
            i = a.verts[vi];
            beg = a.off[i];
            end = a.off[i + 1];
            ci = a.C[i];
            ki = a.k[i];
            const int h = pow2_at_least(2 * (end - beg));
            mask = (unsigned)((h < 8 ? 8 : h) - 1);
        }
        for (int sl = gl; sl <= (int)mask; sl += G) {
            key[sl] = kEmpty;
            val[sl] = 0;
        }
        __syncwarp();
        for (int e = beg + gl; e < end; e += G) {
            const int2 arc = a.arcs[e];
            if (arc.x != i && !smem_insert(key, val, mask, a.C[arc.x], arc.y)) err = 1;
        }
        __syncwarp();
        Best b;
        best_init(b);
        int e_old = 0;
        if (valid)
            for (int sl = gl; sl <= (int)mask; sl += G) eval_slot(a, key[sl], val[sl], ci, ki, b, e_old);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            e_old += __shfl_xor_sync(0xffffffffu, e_old, o);
            best_shfl_xor(b, o);
        }
        bool mv = false;
        if (valid && gl == 0) mv = decide(a, i, ci, ki, b, e_old, ein, dein);
        const unsigned bm = __ballot_sync(0xffffffffu, mv);
        if (bm) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(a.move_count, __popc(bm));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (mv) a.moves[pos + __popc(bm & lt)] = make_int2(i, b.c);
            moved += mv ? 1 : 0;
        }
        __syncwarp();
    }
    flush_stats(a, ein, dein, moved, err);
}

// ---------------------------------------------------------------- bins 2/3
// One 256-thread CTA per vertex.  GLOBAL = false: table in dynamic shared
// memory; GLOBAL = true: table in a per-vertex slice of global memory.
template <bool GLOBAL>
__global__ void __launch_bounds__(256) sweep_cta_kernel(SweepArgs a) {
    extern __shared__ int dyn[];
    __shared__ long long rs[8];
    __shared__ int rc[8], rz[8], re[8], reo[8];
    __shared__ int s_mv;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long ein = 0, dein = 0;
    int moved = 0, err = 0;
    for (int vi = blockIdx.x; vi < a.nverts; vi += gridDim.x) {
        const int i = a.verts[vi];
        const int beg = a.off[i], end = a.off[i + 1];
        const int ci = a.C[i], ki = a.k[i];
        const unsigned mask = (unsigned)pow2_at_least(2 * (end - beg)) - 1u;
        int *key = dyn;
        int *val = dyn + kCtaSlots;
        int2 *tab = GLOBAL ? a.hub_table + a.hub_off[vi] : nullptr;
        for (int sl = threadIdx.x; sl <= (int)mask; sl += 256) {
            if (GLOBAL) tab[sl] = make_int2(kEmpty, 0);
            else {
                key[sl] = kEmpty;
                val[sl] = 0;
            }
        }
        __syncthreads();
        for (int e = beg + threadIdx.x; e < end; e += 256) {
            const int2 arc = a.arcs[e];
            if (arc.x == i) continue;
            const int c = a.C[arc.x];
            const bool ok = GLOBAL ? gmem_insert(tab, mask, c, arc.y)
                                   : smem_insert(key, val, mask, c, arc.y);
            if (!ok) err = 1;
        }
        __syncthreads();
        Best b;
        best_init(b);
        int e_old = 0;
        for (int sl = threadIdx.x; sl <= (int)mask; sl += 256) {
            if (GLOBAL) {
                const int2 kv = tab[sl];
                eval_slot(a, kv.x, kv.y, ci, ki, b, e_old);
            } else {
                eval_slot(a, key[sl], val[sl], ci, ki, b, e_old);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e_old += __shfl_xor_sync(0xffffffffu, e_old, o);
            best_shfl_xor(b, o);
        }
        if (lane == 0) {
            rs[w] = b.s;
            rc[w] = b.c;
            rz[w] = b.size;
            re[w] = b.e;
            reo[w] = e_old;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Best t;
            best_init(t);
            int eo = 0;
            for (int q = 0; q < 8; ++q) {
                best_take(t, rs[q], rc[q], rz[q], re[q]);
                eo += reo[q];
            }
            const bool mv = decide(a, i, ci, ki, t, eo, ein, dein);
            if (mv) {
                const int pos = atomicAdd(a.move_count, 1);
                a.moves[pos] = make_int2(i, t.c);
                ++moved;
            }
        }
        __syncthreads();
    }
    (void)s_mv;
    flush_stats(a, ein, dein, moved, err);
}

// ------------------------------------------------------------------ hubs
// Hub vertices (degree above the CTA bin) are split into chunks of kHubChunk
// arcs.  hub_accum: one block per chunk inserts its arcs into the hub's
// global table, after merging equal labels within each warp; a thread that
// claims an empty slot appends the slot to the hub's occupied list.
// hub_decide: one block per hub evaluates only the occupied slots, resets
// them to empty (so the table is clean for the next use) and decides.
__global__ void __launch_bounds__(256) hub_accum_kernel(SweepArgs a) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int chunk = a.hub_chunk_off[0] + (int)blockIdx.x;
    // position p of the hub owning this chunk: last p with hub_chunk_off[p] <= chunk
    int lo = 0, hi = a.nverts;  // hub_chunk_off[nverts] > chunk
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.hub_chunk_off[mid] <= chunk) lo = mid; else hi = mid;
    }
    const int p = lo;
    const int i = a.verts[p];
    const int beg = a.off[i], end = a.off[i + 1];
    const unsigned mask = (unsigned)pow2_at_least(2 * (end - beg)) - 1u;
    int2 *tab = a.hub_table + a.hub_off[p];
    int32_t *occ = a.hub_occ + a.hub_off[p];
    int32_t *occ_cnt = a.hub_cnt + p;
    const int start = beg + (chunk - a.hub_chunk_off[p]) * kHubChunk;
    const int stop = min(end, start + kHubChunk);
    int err = 0;
    for (int base = start + w * 32; base < stop; base += 256) {
        const int e = base + lane;
        bool valid = e < stop;
        int c = 0, wt = 0;
        if (valid) {
            const int2 arc = a.arcs[e];
            valid = arc.x != i;
            if (valid) {
                c = a.C[arc.x];
                wt = arc.y;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, valid ? c : -1 - lane);
        const int sum = __reduce_add_sync(peers, wt);
        if (valid && lane == __ffs(peers) - 1) {
            unsigned h = hash32(c) & mask;
            bool done = false;
            for (unsigned probe = 0; probe <= mask; ++probe) {
                int *kp = &tab[h].x;
                const int cur = *((volatile int *)kp);
                if (cur == c) {
                    atomicAdd(&tab[h].y, sum);
                    done = true;
                    break;
                }
                if (cur == kEmpty) {
                    const int prev = atomicCAS(kp, kEmpty, c);
                    if (prev == kEmpty) occ[atomicAdd(occ_cnt, 1)] = (int)h;
                    if (prev == kEmpty || prev == c) {
                        atomicAdd(&tab[h].y, sum);
                        done = true;
                        break;
                    }
                }
                h = (h + 1) & mask;
            }
            if (!done) err = 1;
        }
    }
    if (err) atomicOr(&a.stats->err, 1);
}

__global__ void __launch_bounds__(1024) hub_decide_kernel(SweepArgs a) {
    __shared__ long long rs[32];
    __shared__ int rc[32], rz[32], re[32], reo[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x;
    const int i = a.verts[p];
    const int ci = a.C[i], ki = a.k[i];
    int2 *tab = a.hub_table + a.hub_off[p];
    const int32_t *occ = a.hub_occ + a.hub_off[p];
    const int cnt = a.hub_cnt[p];
    Best b;
    best_init(b);
    int e_old = 0;
    for (int t = threadIdx.x; t < cnt; t += 1024) {
        const int h = occ[t];
        const int2 kv = tab[h];
        tab[h] = make_int2(kEmpty, 0);
        eval_slot(a, kv.x, kv.y, ci, ki, b, e_old);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_old += __shfl_xor_sync(0xffffffffu, e_old, o);
        best_shfl_xor(b, o);
    }
    if (lane == 0) {
        rs[w] = b.s;
        rc[w] = b.c;
        rz[w] = b.size;
        re[w] = b.e;
        reo[w] = e_old;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Best t;
        best_init(t);
        int eo = 0;
        for (int q = 0; q < 32; ++q) {
            best_take(t, rs[q], rc[q], rz[q], re[q]);
            eo += reo[q];
        }
        a.hub_cnt[p] = 0;
        long long ein = 0, dein = 0;
        if (decide(a, i, ci, ki, t, eo, ein, dein)) {
            const int pos = atomicAdd(a.move_count, 1);
            a.moves[pos] = make_int2(i, t.c);
            atomicAdd(&a.stats->moved, 1);
        }
        if (ein) atomicAdd(&a.stats->sum_ein, (unsigned long long)ein);
        if (dein) atomicAdd(&a.stats->delta_ein, (unsigned long long)dein);
    }
}

// ------------------------------------------------------------ apply, a^2
__global__ void apply_moves_kernel(int32_t *C, unsigned long long *comm,
                                   const int32_t *__restrict__ k, const int2 *__restrict__ moves,
                                   const int32_t *__restrict__ count) {
    const int cnt = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int2 mv = moves[t];
        const int old = C[mv.x];
        const int ki = k[mv.x];
        C[mv.x] = mv.y;
        atomicAdd(&comm[old], comm_leave(ki));
        atomicAdd(&comm[mv.y], comm_join(ki));
    }
}

__global__ void __launch_bounds__(256) sum_a2_kernel(const unsigned long long *__restrict__ comm,
                                                     int n, unsigned long long *out) {
    __shared__ long long red[8];
    long long acc = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const long long x = comm_a(comm[c]);
        acc += x * x;
    }
    acc = block_sum_256(acc, red);
    if (threadIdx.x == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

__global__ void __launch_bounds__(256) init_phase_kernel(int n, const int32_t *__restrict__ k,
                                                         const int32_t *__restrict__ loop,
                                                         int32_t *C, unsigned long long *comm,
                                                         IterStats *stats) {
    __shared__ long long red[8];
    long long sl = 0, sk = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ki = k[i];
        C[i] = i;
        comm[i] = comm_pack(ki, 1);
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

}  // namespace

lv_status init_phase(PhaseState &ps, cudaStream_t s) {
    LV_CUDA(cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s));
    init_phase_kernel<<<grid_for(ps.g.n, 256, g_num_sms * 8), 256, 0, s>>>(
        ps.g.n, ps.k, ps.loop, ps.C, ps.comm, ps.stats);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status sweep_class(PhaseState &ps, const Buckets &b, int cls, const BinLimits &lim,
                      int64_t *launches, cudaStream_t s) {
    (void)lim;
    SweepArgs a;
    a.off = ps.g.off;
    a.arcs = ps.g.arcs;
    a.k = ps.k;
    a.loop = ps.loop;
    a.C = ps.C;
    a.comm = ps.comm;
    a.two_m = ps.two_m;
    a.moves = ps.moves;
    a.move_count = ps.move_count + cls;
    a.stats = ps.stats;
    a.hub_table = b.hub_table;
    a.hub_occ = b.hub_occ;
    for (int bin = 0; bin < kBins; ++bin) {
        const int lo = b.host_off[cls * (kBins + 1) + bin];
        const int hi = b.host_off[cls * (kBins + 1) + bin + 1];
        const int cnt = hi - lo;
        if (cnt <= 0) continue;
        a.verts = b.order + lo;
        a.nverts = cnt;
        a.hub_off = b.hub_off + lo;
        switch (bin) {
        case 0:
            sweep_group_kernel<kGroupLanes, kGroupSlots>
                <<<grid_for(cnt, 256 / kGroupLanes, g_num_sms * 8), 256, 0, s>>>(a);
            break;
        case 1:
            sweep_group_kernel<32, kWarpSlots><<<grid_for(cnt, 8, g_num_sms * 8), 256, 0, s>>>(a);
            break;
        case 2:
            sweep_cta_kernel<false>
                <<<grid_for(cnt, 1, g_num_sms * 3), 256, 2 * kCtaSlots * sizeof(int), s>>>(a);
            break;
        default: {
            const int bq = cls * (kBins + 1) + bin;
            const int nchunks = b.host_chunk[bq + 1] - b.host_chunk[bq];
            a.hub_chunk_off = b.hub_chunk_off + lo;
            a.hub_cnt = b.hub_cnt + lo;
            hub_accum_kernel<<<nchunks, 256, 0, s>>>(a);
            LV_LAUNCH_CHECK();
            hub_decide_kernel<<<cnt, 1024, 0, s>>>(a);
            break;
        }
        }
        LV_LAUNCH_CHECK();
        ++*launches;
    }
    return LV_OK;
}

lv_status apply_moves(PhaseState &ps, int cls, cudaStream_t s) {
    apply_moves_kernel<<<g_num_sms * 4, 256, 0, s>>>(ps.C, ps.comm, ps.k, ps.moves,
                                                    ps.move_count + cls);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status sum_a2(PhaseState &ps, cudaStream_t s) {
    sum_a2_kernel<<<grid_for(ps.g.n, 256, g_num_sms * 4), 256, 0, s>>>(ps.comm, ps.g.n,
                                                                      &ps.stats->sum_a2);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status sweep_setup() {
    LV_CUDA(cudaFuncSetAttribute(sweep_cta_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * kCtaSlots * (int)sizeof(int)));
    return LV_OK;
}

}  // namespace lv
