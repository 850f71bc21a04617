// lv_graph.cu -- input validation, weighted degrees, vertex following.
//
// Validation follows the problem statement of Sec. 2 (positive weights,
// self-loops allowed, no multi-edges, undirected => symmetric storage).
// Vertex following is the preprocessing of Sec. 4.3 / Sec. 4.4 step 1:
// every single-degree vertex is merged into its only neighbour once, before
// the first phase.
#include "lv_ops.cuh"

namespace lv {

// severity ranks; the most severe violation found is reported
__device__ __forceinline__ void raise_sev(int *sev, int rank) { atomicMax(sev, rank); }
constexpr int kSevArg = 6, kSevDup = 5, kSevWeight = 4, kSevSym = 3;

lv_status severity_to_status(int sev) {
    switch (sev) {
    case kSevArg: return LV_ERR_ARG;
    case kSevDup: return LV_ERR_DUPLICATE;
    case kSevWeight: return LV_ERR_WEIGHT;
    case kSevSym: return LV_ERR_NOT_SYMMETRIC;
    default: return LV_OK;
    }
}

namespace {

__global__ void rowptr_check_kernel(const int64_t *__restrict__ rowptr, int64_t n, int *sev) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (rowptr[i + 1] < rowptr[i]) raise_sev(sev, kSevArg);
}

__global__ void convert_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ w, int32_t n, int32_t A,
                               int32_t *off, int2 *arcs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += stride)
        off[i] = (int32_t)rowptr[i];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A; e += stride)
        arcs[e] = make_int2(col[e], w[e]);
}

// row of every arc (one warp per row)
__global__ void __launch_bounds__(256) row_of_kernel(DGraph g, int32_t *row_of) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t i = blockIdx.x * 8 + (threadIdx.x >> 5); i < g.n; i += nw) {
        const int beg = g.off[i], end = g.off[i + 1];
        for (int e = beg + lane; e < end; e += 32) row_of[e] = (int32_t)i;
    }
}

// one thread per arc: column range, ascending order without duplicates,
// positive weight; 64-bit weighted degrees k64 (zeroed by the caller; runs
// of equal rows within a warp, one atomic per run), self-loop weights; 2m
__global__ void __launch_bounds__(256) arc_check_kernel(DGraph g, const int32_t *__restrict__ row_of,
                                                        int *sev, unsigned long long *k64,
                                                        int32_t *loop, unsigned long long *two_m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t a_pad = ((int64_t)g.A + 31) & ~31ll;  // whole warps take part in the runs
    long long acc = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a_pad; e += stride) {
        const bool in = e < g.A;
        int r = 0;
        int2 a = make_int2(0, 0);
        if (in) {
            r = row_of[e];
            a = g.arcs[e];
            if (a.x < 0 || a.x >= g.n) raise_sev(sev, kSevArg);
            if (a.y < 1) raise_sev(sev, kSevWeight);
            if (e > 0 && row_of[e - 1] == r) {
                const int prev = g.arcs[e - 1].x;
                if (a.x == prev) raise_sev(sev, kSevDup);
                else if (a.x < prev) raise_sev(sev, kSevArg);
            }
            if (a.x == r) loop[r] = a.y;
            acc += a.y;
        }
        warp_run_add(r, (unsigned long long)(unsigned)a.y, in && a.y > 0, k64);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(two_m, (unsigned long long)acc);
}

// k = k64, saturated at 2^31 - 1 (a larger degree fails the 2m < 2^31 test)
__global__ void degree_store_kernel(int32_t n, const unsigned long long *__restrict__ k64, int32_t *k) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        k[i] = k64[i] > 0x7fffffffull ? 0x7fffffff : (int32_t)k64[i];
}

// Symmetry, one thread per non-loop arc.  Of the two arcs of a pair {i, j},
// the one stored in the longer row (ties: the larger row id) looks for its
// mirror, with the same weight, by bisection of the shorter row; the other
// is only counted.  Rows hold no duplicates, so the mirrors of the searching
// arcs are distinct counted arcs; when every search succeeds and the two
// counts agree, every arc has its mirror.
__global__ void __launch_bounds__(256) mirror_kernel(DGraph g, const int32_t *__restrict__ row_of,
                                                     int *sev, unsigned long long *counts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    long long searched = 0, counted = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.A; e += stride) {
        const int i = row_of[e];
        const int2 a = g.arcs[e];
        const int j = a.x;
        if (j == i) continue;
        const int di = g.off[i + 1] - g.off[i];
        int lo = g.off[j], hi = g.off[j + 1];
        const int dj = hi - lo;
        if (dj < di || (dj == di && j < i)) {
            ++searched;
            const int hend = hi;
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if (g.arcs[mid].x < i) lo = mid + 1; else hi = mid;
            }
            if (lo >= hend || g.arcs[lo].x != i || g.arcs[lo].y != a.y) raise_sev(sev, kSevSym);
        } else {
            ++counted;
        }
    }
    searched = warp_sum(searched);
    counted = warp_sum(counted);
    if ((threadIdx.x & 31) == 0) {
        if (searched) atomicAdd(&counts[0], (unsigned long long)searched);
        if (counted) atomicAdd(&counts[1], (unsigned long long)counted);
    }
}

constexpr int kBigRow = 1024;

// rows of at least kBigRow arcs (optionally only kept ones), appended to list
__global__ void big_rows_kernel(DGraph g, const int32_t *__restrict__ keep, int32_t *list,
                                int32_t *count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x)
        if (g.off[i + 1] - g.off[i] >= kBigRow && (!keep || keep[i])) list[atomicAdd(count, 1)] = i;
}

// one warp per row: weighted degree k_i and self-loop weight (R1: once)
__global__ void __launch_bounds__(256) degree_kernel(DGraph g, int32_t *k, int32_t *loop) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t i = blockIdx.x * 8 + (threadIdx.x >> 5); i < g.n; i += nw) {
        const int beg = g.off[i], end = g.off[i + 1];
        int s = 0, lp = 0;
        for (int e = beg + lane; e < end; e += 32) {
            const int2 a = g.arcs[e];
            s += a.y;
            if (a.x == i) lp = a.y;
        }
        s = warp_sum(s);
        lp = warp_sum(lp);
        if (lane == 0) {
            k[i] = s;
            loop[i] = lp;
        }
    }
}

// ------------------------------------------------------ vertex following
// single-degree: exactly one stored arc and it is not a self-loop
__global__ void vf_mark_kernel(DGraph g, uint8_t *d1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        const int beg = g.off[i];
        d1[i] = (g.off[i + 1] - beg == 1) && (g.arcs[beg].x != i);
    }
}

// removal decision; the survivor gets self-loop weight 2*w(i,j) (R2); of two
// mutually single-degree vertices the smaller id is removed (R3)
__global__ void vf_decide_kernel(DGraph g, const uint8_t *__restrict__ d1, int32_t *keep,
                                 int32_t *target, int32_t *extra, int32_t *nrem) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        int kp = 1;
        if (d1[i]) {
            const int2 a = g.arcs[g.off[i]];
            const int j = a.x;
            if (!(d1[j] && j < i)) {
                kp = 0;
                target[i] = j;
                atomicAdd(&extra[j], 2 * a.y);
                atomicAdd(&nrem[j], 1);
            }
        }
        keep[i] = kp;
    }
}

__global__ void vf_rowlen_kernel(DGraph g, const int32_t *__restrict__ keep,
                                 const int32_t *__restrict__ newid, const int32_t *__restrict__ loop,
                                 const int32_t *__restrict__ extra, const int32_t *__restrict__ nrem,
                                 int32_t *rowlen) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        if (!keep[i]) continue;
        const int deg = g.off[i + 1] - g.off[i];
        rowlen[newid[i]] = deg - nrem[i] + ((loop[i] == 0 && extra[i] > 0) ? 1 : 0);
    }
}

// Kept rows of at most kVfSmallRow arcs, four per warp with kVfLanes lanes
// each (rows of this size fill a warp's lanes poorly): as vf_fill_kernel,
// with the warp's ballots cut to the group's bits.
constexpr int kVfLanes = 8;
constexpr int kVfSmallRow = 64;
__global__ void __launch_bounds__(256) vf_fill_small_kernel(DGraph g, const int32_t *__restrict__ nid,
                                                            const int32_t *__restrict__ loop,
                                                            const int32_t *__restrict__ extra,
                                                            const int32_t *__restrict__ off2,
                                                            int2 *arcs2) {
    constexpr int kGroups = 32 / kVfLanes;
    const int lane = threadIdx.x & 31, grp = lane / kVfLanes, gl = lane % kVfLanes;
    const unsigned gshift = grp * kVfLanes, gbits = (1u << kVfLanes) - 1u;
    const unsigned lt = (1u << gl) - 1u;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t w = blockIdx.x * 8 + (threadIdx.x >> 5); w * kGroups < g.n; w += nw) {
        const int64_t ii = w * kGroups + grp;
        const int i = (int)ii;
        int beg = 0, end = 0;
        bool row = ii < g.n;
        if (row) {
            beg = g.off[i];
            end = g.off[i + 1];
            row = nid[i] >= 0 && end - beg <= kVfSmallRow;
        }
        if (!row) end = beg;
        const int ni = row ? nid[i] : 0;
        const int ex = row ? extra[i] : 0;
        bool pending = row && loop[i] == 0 && ex > 0;  // self-loop to insert
        int run = row ? off2[ni] : 0;
        int sh = 0;  // 1 once the inserted loop precedes the current arcs
        const int nch = __reduce_max_sync(0xffffffffu, (end - beg + kVfLanes - 1) / kVfLanes);
        for (int t = 0; t < nch; ++t) {
            const int e = beg + t * kVfLanes + gl;
            const bool valid = e < end;
            const int2 a = valid ? g.arcs[e] : make_int2(-1, 0);
            const int nv = valid && a.x != i ? nid[a.x] : -1;  // new id, -1: removed
            const bool kp = valid && (a.x == i || nv >= 0);
            const unsigned bk = (__ballot_sync(0xffffffffu, kp) >> gshift) & gbits;
            const unsigned bgt =
                (__ballot_sync(0xffffffffu, pending && kp && a.x > i) >> gshift) & gbits;
            int lsh = sh;
            if (bgt) {  // group-uniform: only a pending group has bits here
                const int f = __ffs(bgt) - 1;
                if (gl == 0) arcs2[run + __popc(bk & ((1u << f) - 1u))] = make_int2(ni, ex);
                if (gl >= f) lsh = 1;
                pending = false;
                sh = 1;
            }
            if (kp) {
                const int pos = run + __popc(bk & lt) + lsh;
                arcs2[pos] = (a.x == i) ? make_int2(ni, a.y + ex) : make_int2(nv, a.y);
            }
            run += __popc(bk);
        }
        if (pending && gl == 0) arcs2[run + sh] = make_int2(ni, ex);
    }
}

// one warp per kept row of kVfSmallRow < arcs < kBigRow: drop arcs to
// removed vertices, renumber, add the merged weight to the self-loop
// (inserting it at its sorted place if absent)
__global__ void __launch_bounds__(256) vf_fill_kernel(DGraph g, const int32_t *__restrict__ nid,
                                                      const int32_t *__restrict__ loop,
                                                      const int32_t *__restrict__ extra,
                                                      const int32_t *__restrict__ off2,
                                                      int2 *arcs2) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t ii = blockIdx.x * 8 + (threadIdx.x >> 5); ii < g.n; ii += nw) {
        const int i = (int)ii;
        const int len = g.off[i + 1] - g.off[i];
        const int ni = nid[i];
        if (ni < 0 || len >= kBigRow || len <= kVfSmallRow) continue;  // warp-uniform
        const int ex = extra[i];
        bool pending = (loop[i] == 0 && ex > 0);  // self-loop to insert
        int run = off2[ni];
        int sh = 0;  // 1 once the inserted loop precedes the current arcs
        const int beg = g.off[i], end = g.off[i + 1];
        for (int base0 = beg; base0 < end; base0 += 64) {
            // two 32-arc chunks' loads in flight, then each chunk in order
            int2 a2[2];
            int nv2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = base0 + 32 * h + lane;
                a2[h] = e < end ? g.arcs[e] : make_int2(-1, 0);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)  // new id, -1: removed
                nv2[h] = a2[h].x >= 0 && a2[h].x != i ? nid[a2[h].x] : -1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int base = base0 + 32 * h;
                if (base >= end) break;  // warp-uniform
                const bool valid = base + lane < end;
                const int2 a = a2[h];
                const int nv = nv2[h];
                const bool kp = valid && (a.x == i || nv >= 0);
                const unsigned bk = __ballot_sync(0xffffffffu, kp);
                int lsh = sh;
                if (pending) {
                    const unsigned bgt = __ballot_sync(0xffffffffu, kp && a.x > i);
                    if (bgt) {
                        const int f = __ffs(bgt) - 1;
                        if (lane == 0)
                            arcs2[run + __popc(bk & ((1u << f) - 1u))] = make_int2(ni, ex);
                        if (lane >= f) lsh = 1;
                        pending = false;
                        sh = 1;
                    }
                }
                if (kp) {
                    const int pos = run + __popc(bk & lt) + lsh;
                    arcs2[pos] = (a.x == i) ? make_int2(ni, a.y + ex) : make_int2(nv, a.y);
                }
                run += __popc(bk);
            }
        }
        if (pending && lane == 0) arcs2[run + sh] = make_int2(ni, ex);
    }
}

// the same for kept rows of at least kBigRow arcs, one 1024-thread block each:
// positions come from a block-wide prefix over the kept flags of each chunk
__global__ void __launch_bounds__(1024) vf_fill_big_kernel(DGraph g, const int32_t *__restrict__ nid,
                                                           const int32_t *__restrict__ list,
                                                           const int32_t *__restrict__ count,
                                                           const int32_t *__restrict__ loop,
                                                           const int32_t *__restrict__ extra,
                                                           const int32_t *__restrict__ off2,
                                                           int2 *arcs2) {
    __shared__ int s_wcnt[32], s_wpre[32], s_tot, s_first;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nbig = *count;
    for (int t = blockIdx.x; t < nbig; t += gridDim.x) {
        const int i = list[t];
        const int beg = g.off[i], end = g.off[i + 1];
        const int ni = nid[i];
        const int ex = extra[i];
        bool pending = (loop[i] == 0 && ex > 0);
        int run = off2[ni];
        int sh = 0;
        for (int base = beg; base < end; base += 1024) {
            const int e = base + (int)threadIdx.x;
            const bool valid = e < end;
            const int2 a = valid ? g.arcs[e] : make_int2(-1, 0);
            const int nv = valid && a.x != i ? nid[a.x] : -1;  // new id, -1: removed
            const bool kp = valid && (a.x == i || nv >= 0);
            const unsigned wb = __ballot_sync(0xffffffffu, kp);
            if (lane == 0) s_wcnt[w] = __popc(wb);
            if (threadIdx.x == 0) s_first = 1 << 30;
            __syncthreads();
            if (w == 0) {
                int x = s_wcnt[lane], incl = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                s_wpre[lane] = incl - x;
                if (lane == 31) s_tot = incl;
            }
            if (pending && kp && a.x > i) atomicMin(&s_first, (int)threadIdx.x);
            __syncthreads();
            const int rank = s_wpre[w] + __popc(wb & lt);
            int lsh = sh;
            if (pending && s_first < (1 << 30)) {
                if ((int)threadIdx.x == s_first) arcs2[run + rank] = make_int2(ni, ex);
                if ((int)threadIdx.x >= s_first) lsh = 1;
            }
            if (kp) arcs2[run + rank + lsh] =
                (a.x == i) ? make_int2(ni, a.y + ex) : make_int2(nv, a.y);
            if (pending && s_first < (1 << 30)) {
                pending = false;
                sh = 1;
            }
            run += s_tot;
            __syncthreads();
        }
        if (pending && threadIdx.x == 0) arcs2[run + sh] = make_int2(ni, ex);
        __syncthreads();
    }
}

// nid[v] = new id of v, -1 if v is removed
__global__ void vf_nid_kernel(int32_t n, const int32_t *__restrict__ keep,
                              const int32_t *__restrict__ newid, int32_t *nid) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        nid[v] = keep[v] ? newid[v] : -1;
}

__global__ void vf_map_kernel(int32_t n, const int32_t *__restrict__ keep,
                              const int32_t *__restrict__ newid, const int32_t *__restrict__ target,
                              int32_t *map) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        map[v] = keep[v] ? newid[v] : newid[target[v]];
}

__global__ void iota_kernel(int32_t n, int32_t *out) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = v;
}

// ------------------------------------------- recursive single-neighbour VF
// Target of each vertex in one round of the recursive merge: a vertex with
// exactly one neighbour j != i (row of one arc, or two arcs one of which is
// its self-loop l) passes when k_i^2 > 2m l with k_i = w(i,j) + l -- the
// bound of Lemma 3's Eq. (eqnClaimIItemp) taken at a_C(j) = 2m - k_i, exact
// in 64-bit integers (k_i <= 2m < 2^31).  Otherwise the target is -1.
__global__ void sn_target_kernel(DGraph g, long long two_m, int32_t *target) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
        const int b = g.off[i], len = g.off[i + 1] - b;
        int t = -1;
        if (len == 1 || len == 2) {
            const int2 a0 = g.arcs[b];
            const int2 a1 = len == 2 ? g.arcs[b + 1] : make_int2(i, 0);
            // rows hold no duplicates: a row of two arcs is single-neighbour
            // only when one of them is the self-loop
            const bool one = len == 1 ? a0.x != i : (a0.x == i) != (a1.x == i);
            if (one) {
                const int2 nb = a0.x != i ? a0 : a1;
                const long long l = a0.x == i ? a0.y : (len == 2 && a1.x == i ? a1.y : 0);
                const long long k = (long long)nb.y + l;
                if (k * k > two_m * l) t = nb.x;
            }
        }
        target[i] = t;
    }
}

// C[i] = the vertex i merges into (itself if it stays); of two vertices
// passing towards each other the smaller merges (R3); keep[i] = survivor
__global__ void sn_resolve_kernel(int n, const int32_t *__restrict__ target, int32_t *C,
                                  int32_t *keep) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = target[i];
        const bool merge = t >= 0 && !(target[t] == i && t < i);
        C[i] = merge ? t : i;
        keep[i] = merge ? 0 : 1;
    }
}

}  // namespace

static int grid_rows(int64_t rows) { return grid_for(rows, 8, g_num_sms * 16); }
static int grid_items(int64_t items) { return grid_for(items, 256, g_num_sms * 16); }

lv_status validate_and_build(int64_t n, const int64_t *rowptr, const int32_t *col,
                             const int32_t *w, DGraph *out, int32_t **k_out, int32_t **loop_out,
                             int64_t *two_m_out, int *scratch_pinned, cudaStream_t s,
                             bool limit_two_m) {
    *out = DGraph();
    *k_out = nullptr;
    *loop_out = nullptr;
    if (n < 0 || n > 0x7ffffffell) return LV_ERR_ARG;
    int64_t ends[2];
    LV_CUDA(cudaMemcpyAsync(&ends[0], rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(&ends[1], rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0) return LV_ERR_ARG;
    int *dsev = nullptr;
    unsigned long long *d2m = nullptr;
    LV_TRY(dalloc_n(&dsev, 1, s));
    LV_TRY(dalloc_n(&d2m, 1, s));
    LV_CUDA(cudaMemsetAsync(dsev, 0, sizeof(int), s));
    LV_CUDA(cudaMemsetAsync(d2m, 0, sizeof(unsigned long long), s));
    if (n > 0) {
        rowptr_check_kernel<<<grid_items(n), 256, 0, s>>>(rowptr, n, dsev);
        LV_LAUNCH_CHECK();
    }
    LV_CUDA(cudaMemcpyAsync(scratch_pinned, dsev, sizeof(int), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    lv_status st = LV_OK;
    if (scratch_pinned[0] != 0 || ends[1] < 0) st = LV_ERR_ARG;
    else if (ends[1] > 0x7fffffffll) st = LV_ERR_OVERFLOW;
    if (st != LV_OK) {
        dfree(dsev, s);
        dfree(d2m, s);
        return st;
    }
    DGraph g;
    g.n = (int32_t)n;
    g.A = (int32_t)ends[1];
    LV_TRY(dalloc_n(&g.off, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&g.arcs, (size_t)g.A, s));
    int32_t *k = nullptr, *loop = nullptr;
    LV_TRY(dalloc_n(&k, (size_t)n, s));
    LV_TRY(dalloc_n(&loop, (size_t)n, s));
    convert_kernel<<<grid_items((int64_t)g.A + n + 1), 256, 0, s>>>(rowptr, col, w, g.n, g.A,
                                                                    g.off, g.arcs);
    LV_LAUNCH_CHECK();
    unsigned long long *k64 = nullptr;
    if (n > 0) {
        LV_TRY(dalloc_n(&k64, (size_t)n, s));
        LV_CUDA(cudaMemsetAsync(k64, 0, sizeof(unsigned long long) * (size_t)n, s));
        LV_CUDA(cudaMemsetAsync(loop, 0, sizeof(int32_t) * (size_t)n, s));
    }
    // counts[0..1]: searching / counted arcs of the symmetry test
    unsigned long long *counts = nullptr;
    LV_TRY(dalloc_n(&counts, 2, s));
    LV_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s));
    if (g.A > 0) {
        int32_t *row_of = nullptr;
        LV_TRY(dalloc_n(&row_of, (size_t)g.A, s));
        row_of_kernel<<<grid_rows(n), 256, 0, s>>>(g, row_of);
        LV_LAUNCH_CHECK();
        arc_check_kernel<<<grid_items(g.A), 256, 0, s>>>(g, row_of, dsev, k64, loop, d2m);
        LV_LAUNCH_CHECK();
        LV_CUDA(cudaMemcpyAsync(scratch_pinned, dsev, sizeof(int), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        if (scratch_pinned[0] < kSevSym) {  // columns in range and rows sorted: bisection is safe
            mirror_kernel<<<grid_items(g.A), 256, 0, s>>>(g, row_of, dsev, counts);
            LV_LAUNCH_CHECK();
        }
        dfree(row_of, s);
    }
    if (n > 0) {
        degree_store_kernel<<<grid_items(n), 256, 0, s>>>(g.n, k64, k);
        LV_LAUNCH_CHECK();
        dfree(k64, s);
    }
    unsigned long long tm = 0, cnt[2] = {0, 0};
    LV_CUDA(cudaMemcpyAsync(scratch_pinned, dsev, sizeof(int), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(&tm, d2m, sizeof(tm), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaMemcpyAsync(cnt, counts, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    dfree(counts, s);
    if (cnt[0] != cnt[1] && scratch_pinned[0] < kSevSym) scratch_pinned[0] = kSevSym;
    st = severity_to_status(scratch_pinned[0]);
    if (st == LV_OK) {
        if (limit_two_m && tm >= (1ull << 31)) st = LV_ERR_OVERFLOW;
        else if (tm == 0) st = LV_ERR_EMPTY;
    }
    dfree(dsev, s);
    dfree(d2m, s);
    if (st != LV_OK) {
        dfree(g.off, s);
        dfree(g.arcs, s);
        dfree(k, s);
        dfree(loop, s);
        return st;
    }
    *out = g;
    *k_out = k;
    *loop_out = loop;
    *two_m_out = (int64_t)tm;
    return LV_OK;
}

lv_status compute_degrees(const DGraph &g, int32_t *k, int32_t *loop, cudaStream_t s) {
    if (g.n == 0) return LV_OK;
    degree_kernel<<<grid_rows(g.n), 256, 0, s>>>(g, k, loop);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status iota(int32_t n, int32_t *out, cudaStream_t s) {
    if (n == 0) return LV_OK;
    iota_kernel<<<grid_items(n), 256, 0, s>>>(n, out);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status vertex_following(const DGraph &g, const int32_t *loop, DGraph *out, int32_t *map,
                           int *scratch_pinned, cudaStream_t s) {
    const int n = g.n;
    uint8_t *d1 = nullptr;
    int32_t *keep = nullptr, *target = nullptr, *extra = nullptr, *nrem = nullptr,
            *newid = nullptr, *rowlen = nullptr;
    LV_TRY(dalloc_n(&d1, (size_t)n, s));
    LV_TRY(dalloc_n(&keep, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&target, (size_t)n, s));
    LV_TRY(dalloc_n(&extra, (size_t)n, s));
    LV_TRY(dalloc_n(&nrem, (size_t)n, s));
    LV_TRY(dalloc_n(&newid, (size_t)n + 1, s));
    LV_CUDA(cudaMemsetAsync(extra, 0, sizeof(int32_t) * n, s));
    LV_CUDA(cudaMemsetAsync(nrem, 0, sizeof(int32_t) * n, s));
    vf_mark_kernel<<<grid_items(n), 256, 0, s>>>(g, d1);
    LV_LAUNCH_CHECK();
    vf_decide_kernel<<<grid_items(n), 256, 0, s>>>(g, d1, keep, target, extra, nrem);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(keep, newid, n, s));
    LV_CUDA(cudaMemcpyAsync(scratch_pinned, newid + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    const int n2 = scratch_pinned[0];
    LV_TRY(dalloc_n(&rowlen, (size_t)n2 + 1, s));
    DGraph h;
    h.n = n2;
    LV_TRY(dalloc_n(&h.off, (size_t)n2 + 1, s));
    vf_rowlen_kernel<<<grid_items(n), 256, 0, s>>>(g, keep, newid, loop, extra, nrem, rowlen);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(rowlen, h.off, n2, s));
    LV_CUDA(cudaMemcpyAsync(scratch_pinned, h.off + n2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    h.A = scratch_pinned[0];
    LV_TRY(dalloc_n(&h.arcs, (size_t)h.A, s));
    // new id of every vertex, -1 for the removed: one gather per arc
    int32_t *nid = nullptr;
    LV_TRY(dalloc_n(&nid, (size_t)n, s));
    vf_nid_kernel<<<grid_items(n), 256, 0, s>>>(n, keep, newid, nid);
    LV_LAUNCH_CHECK();
    vf_fill_small_kernel<<<grid_rows((n + 3) / 4), 256, 0, s>>>(g, nid, loop, extra, h.off, h.arcs);
    LV_LAUNCH_CHECK();
    vf_fill_kernel<<<grid_rows(n), 256, 0, s>>>(g, nid, loop, extra, h.off, h.arcs);
    LV_LAUNCH_CHECK();
    int32_t *big = nullptr;
    LV_TRY(dalloc_n(&big, (size_t)g.A / kBigRow + 2, s));
    LV_CUDA(cudaMemsetAsync(big, 0, sizeof(int32_t), s));
    big_rows_kernel<<<grid_items(n), 256, 0, s>>>(g, keep, big + 1, big);
    LV_LAUNCH_CHECK();
    vf_fill_big_kernel<<<g_num_sms * 2, 1024, 0, s>>>(g, nid, big + 1, big, loop, extra, h.off,
                                                      h.arcs);
    LV_LAUNCH_CHECK();
    dfree(big, s);
    vf_map_kernel<<<grid_items(n), 256, 0, s>>>(n, keep, newid, target, map);
    LV_LAUNCH_CHECK();
    dfree(nid, s);
    dfree(d1, s);
    dfree(keep, s);
    dfree(target, s);
    dfree(extra, s);
    dfree(nrem, s);
    dfree(newid, s);
    dfree(rowlen, s);
    *out = h;
    return LV_OK;
}

lv_status vf_recursive(DGraph *G, int64_t two_m, int32_t *map, int32_t n_orig, int *pinned,
                       int32_t *rounds, cudaStream_t s) {
    *rounds = 0;
    for (;;) {
        const int n = G->n;
        int32_t *target = nullptr, *C = nullptr, *newid = nullptr, *scratch = nullptr;
        LV_TRY(dalloc_n(&target, (size_t)n, s));
        LV_TRY(dalloc_n(&C, (size_t)n, s));
        LV_TRY(dalloc_n(&newid, (size_t)n + 1, s));
        sn_target_kernel<<<grid_items(n), 256, 0, s>>>(*G, (long long)two_m, target);
        LV_LAUNCH_CHECK();
        sn_resolve_kernel<<<grid_items(n), 256, 0, s>>>(n, target, C, newid);
        LV_LAUNCH_CHECK();
        LV_TRY(scan_excl_i32(newid, newid, n, s));
        LV_CUDA(cudaMemcpyAsync(pinned, newid + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        const int32_t n_next = pinned[0];
        lv_status st = LV_OK;
        if (n_next < n) {
            DGraph H;
            st = coarsen(*G, C, newid, n_next, &H, pinned, s);
            if (st == LV_OK) st = dalloc_n(&scratch, (size_t)n_orig, s);
            if (st == LV_OK) st = compose_labels(n_orig, map, C, newid, scratch, s);
            if (st == LV_OK) {
                free_graph(*G, s);
                *G = H;
                ++*rounds;
            }
        }
        dfree(target, s);
        dfree(C, s);
        dfree(newid, s);
        dfree(scratch, s);
        if (st != LV_OK) return st;
        if (n_next == n) return LV_OK;
    }
}

void free_graph(DGraph &g, cudaStream_t s) {
    dfree(g.off, s);
    dfree(g.arcs, s);
    g = DGraph();
}

}  // namespace lv
