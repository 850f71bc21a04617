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

// one warp per row: key = c'(u) << b | c'(v), value = w
__global__ void __launch_bounds__(256) arc_keys_kernel(DGraph g, const uint32_t *__restrict__ cm,
                                                       int b, uint64_t *keys, uint32_t *vals) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t u = blockIdx.x * 8 + (threadIdx.x >> 5); u < g.n; u += nw) {
        const uint64_t hi = (uint64_t)cm[u] << b;
        const int beg = g.off[u], end = g.off[u + 1];
        for (int e = beg + lane; e < end; e += 32) {
            const int2 a = g.arcs[e];
            keys[e] = hi | cm[a.x];
            vals[e] = (uint32_t)a.y;
        }
    }
}

__global__ void heads_kernel(const uint64_t *__restrict__ keys, int A, int32_t *head) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < A; e += gridDim.x * blockDim.x)
        head[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// seg(e) = pos[e] + head[e] - 1; weights summed per segment with a warp
// segmented scan first (segments are contiguous), then one atomic per piece
__global__ void __launch_bounds__(256) emit_kernel(const uint64_t *__restrict__ keys,
                                                   const uint32_t *__restrict__ vals,
                                                   const int32_t *__restrict__ head,
                                                   const int32_t *__restrict__ pos, int A, int b,
                                                   int2 *arcs2, int32_t *rowcnt) {
    const int lane = threadIdx.x & 31;
    const uint64_t lowmask = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < A; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool valid = e < A;
        int seg = -1 - lane;  // distinct per invalid lane
        int w = 0;
        if (valid) {
            const int h = head[e];
            seg = pos[e] + h - 1;
            w = (int)vals[e];
            if (h) {
                const uint64_t k = keys[e];
                arcs2[seg].x = (int)(k & lowmask);
                atomicAdd(&rowcnt[(int)(k >> b)], 1);
            }
        }
        // inclusive segmented scan of w within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ws = __shfl_up_sync(0xffffffffu, w, o);
            const int ss = __shfl_up_sync(0xffffffffu, seg, o);
            if (lane >= o && ss == seg) w += ws;
        }
        const int snext = __shfl_down_sync(0xffffffffu, seg, 1);
        if (valid && (lane == 31 || snext != seg)) atomicAdd(&arcs2[seg].y, w);
    }
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
    const int A = g.A;
    const int b = bits_for((uint64_t)(n_next > 0 ? n_next - 1 : 0));
    uint32_t *cm = nullptr;
    uint64_t *keys = nullptr, *keys_alt = nullptr;
    uint32_t *vals = nullptr, *vals_alt = nullptr;
    int32_t *head = nullptr, *pos = nullptr, *rowcnt = nullptr;
    LV_TRY(dalloc_n(&cm, (size_t)g.n, s));
    LV_TRY(dalloc_n(&keys, (size_t)A, s));
    LV_TRY(dalloc_n(&keys_alt, (size_t)A, s));
    LV_TRY(dalloc_n(&vals, (size_t)A, s));
    LV_TRY(dalloc_n(&vals_alt, (size_t)A, s));
    cmap_kernel<<<grid_items(g.n), 256, 0, s>>>(g.n, C, newid, cm);
    LV_LAUNCH_CHECK();
    arc_keys_kernel<<<grid_for(g.n, 8, g_num_sms * 16), 256, 0, s>>>(g, cm, b, keys, vals);
    LV_LAUNCH_CHECK();
    LV_TRY(radix_sort_u64(keys, vals, keys_alt, vals_alt, A, 2 * b, s));
    dfree(keys_alt, s);
    dfree(vals_alt, s);
    dfree(cm, s);
    LV_TRY(dalloc_n(&head, (size_t)A, s));
    LV_TRY(dalloc_n(&pos, (size_t)A + 1, s));
    heads_kernel<<<grid_items(A), 256, 0, s>>>(keys, A, head);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(head, pos, A, s));
    LV_CUDA(cudaMemcpyAsync(pinned, pos + A, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    DGraph h;
    h.n = n_next;
    h.A = pinned[0];
    LV_TRY(dalloc_n(&h.off, (size_t)n_next + 1, s));
    LV_TRY(dalloc_n(&h.arcs, (size_t)h.A, s));
    LV_TRY(dalloc_n(&rowcnt, (size_t)n_next + 1, s));
    LV_CUDA(cudaMemsetAsync(h.arcs, 0, sizeof(int2) * (size_t)h.A, s));
    LV_CUDA(cudaMemsetAsync(rowcnt, 0, sizeof(int32_t) * ((size_t)n_next + 1), s));
    emit_kernel<<<grid_items(A), 256, 0, s>>>(keys, vals, head, pos, A, b, h.arcs, rowcnt);
    LV_LAUNCH_CHECK();
    LV_TRY(scan_excl_i32(rowcnt, h.off, n_next, s));
    dfree(keys, s);
    dfree(vals, s);
    dfree(head, s);
    dfree(pos, s);
    dfree(rowcnt, s);
    *out = h;
    return LV_OK;
}

}  // namespace lv
