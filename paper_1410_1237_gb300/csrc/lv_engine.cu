// lv_engine.cu -- the multi-graph engine (see lv_engine.cuh).
//
// Per graph, the engine replays the single-graph driver's control exactly:
//   - each batched sweep covers the vertices of graphs still iterating in
//     the current phase; the sweep that proposes iteration t's moves also
//     yields N(C^{t-1}) per graph (fused modularity), the host runs every
//     graph's stopping test and applies the moves only of graphs that go on;
//   - when no graph iterates any more, one renumber / compose / coarsen pass
//     serves all graphs, and each graph's phase-loop test decides whether its
//     coarse graph stays in the union.
// Renumbering ranks communities by id, so graphs stay contiguous and ordered
// in every coarse union and local ids are union ids minus the graph's start.
#include <algorithm>
#include <cstring>

#include "lv_engine.cuh"

namespace lv {

namespace {

int grid_n(int64_t items) { return grid_for(items, 256, g_num_sms * 16); }

// gid[v] = g with gptr[g] <= v < gptr[g+1] (gptr strictly increasing)
__global__ void graph_of_kernel(int32_t n, int32_t G, const int32_t *__restrict__ gptr,
                                int32_t *gid) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int a = 0, b = G;  // gptr[a] <= v < gptr[b]
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (gptr[mid] <= v) a = mid; else b = mid;
        }
        gid[v] = a;
    }
}

// every arc of row i must stay inside graph gid[i]; one warp per row
__global__ void __launch_bounds__(256) cross_check_kernel(DGraph g, const int32_t *__restrict__ gid,
                                                          const int32_t *__restrict__ gptr,
                                                          int *bad) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * 8;
    for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < g.n; i += nw) {
        const int gi = gid[i];
        const int lo = gptr[gi], hi = gptr[gi + 1];
        bool ok = true;
        for (int e = g.off[i] + lane; e < g.off[i + 1]; e += 32) {
            const int c = g.arcs[e].x;
            ok = ok && c >= lo && c < hi;
        }
        if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicExch(bad, 1);
    }
}

// Per-graph sums over vertices of graphs with active[g] != 0 (all graphs
// when active is null): sum_k (2m), sum_loop and sum_k2.  Any output may be
// null.  Vertices of a graph are consecutive, so whole warps form runs.
__global__ void __launch_bounds__(256) graph_sums_kernel(int32_t n, const int32_t *__restrict__ gid,
                                                         const int32_t *__restrict__ k,
                                                         const int32_t *__restrict__ loop,
                                                         const uint8_t *__restrict__ active,
                                                         unsigned long long *sum_k,
                                                         unsigned long long *sum_loop,
                                                         unsigned long long *sum_k2) {
    const int nr = (n + 31) & ~31;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nr; v += gridDim.x * blockDim.x) {
        const bool in = v < n;
        const int g = in ? gid[v] : 0;
        const bool on = in && (!active || active[g]);
        const long long kv = on ? k[v] : 0;
        const long long lv = on ? loop[v] : 0;
        if (sum_k) warp_run_add(g, (unsigned long long)kv, on, sum_k);
        if (sum_loop) warp_run_add(g, (unsigned long long)lv, on, sum_loop);
        if (sum_k2) warp_run_add(g, (unsigned long long)(kv * kv), on, sum_k2);
    }
}

// gid_new[idx[C[v]]] = gid[v] (idx[v] when C is null); all writers of one
// target write the same graph
__global__ void gid_scatter_kernel(int32_t n, const int32_t *__restrict__ gid,
                                   const int32_t *__restrict__ C, const int32_t *__restrict__ idx,
                                   int32_t *gid_new) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        gid_new[idx[C ? C[v] : v]] = gid[v];
}

// gptr from a non-decreasing gid: gptr[g] = first vertex of g, gptr[G] = n
__global__ void gptr_kernel(int32_t n, int32_t G, const int32_t *__restrict__ gid, int32_t *gptr) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (v == 0 || gid[v] != gid[v - 1]) gptr[gid[v]] = v;
        if (v == 0) gptr[G] = n;
    }
}

// out[g] = arr[idx[g]] for g <= G (arc offsets, or new ids, at graph starts)
__global__ void gather_at_kernel(int32_t G, const int32_t *__restrict__ idx,
                                 const int32_t *__restrict__ arr, int32_t *out) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x)
        out[g] = arr[idx[g]];
}

// apply the listed moves of graphs whose apply flag is set
__global__ void apply_batch_kernel(int32_t *C, unsigned long long *comm,
                                   const int4 *__restrict__ moves, const int32_t *__restrict__ count,
                                   const int32_t *__restrict__ gid,
                                   const uint8_t *__restrict__ apply) {
    const int cnt = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int4 m = moves[t];
        if (!apply[gid[m.x]]) continue;
        C[m.x] = m.z;
        atomicAdd(&comm[m.y], comm_leave(m.w));
        atomicAdd(&comm[m.z], comm_join(m.w));
    }
}

// union labels -> labels local to each graph
__global__ void localize_kernel(int32_t n, const int32_t *__restrict__ gid,
                                const int32_t *__restrict__ gstart, int32_t *labels) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        labels[v] -= gstart[gid[v]];
}

// Compaction of the group bins (degree bins 0..5, positions [lo, hi) of
// the bucketed order): vertices of graphs that stopped iterating are dropped,
// so later sweeps of a phase hand out items over live vertices only.  The
// kept vertices are packed at the END of [lo, hi) (CTA-bin and hub positions
// after hi keep their places and their per-position hub arrays).
__global__ void keep_flags_kernel(const int32_t *__restrict__ order, int lo, int hi,
                                  const int32_t *__restrict__ gid,
                                  const uint8_t *__restrict__ active, int32_t *flag) {
    for (int p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x)
        flag[p - lo] = active[gid[order[p]]] ? 1 : 0;
}

__global__ void compact_kernel(const int32_t *__restrict__ order, int lo, int hi,
                               const int32_t *__restrict__ pos, int32_t *out) {
    const int base = hi - pos[hi - lo];
    for (int p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x)
        if (pos[p - lo + 1] != pos[p - lo]) out[base + pos[p - lo]] = order[p];
}

// bucket offsets of the compacted list (class 0): group-bin starts move,
// the rest is copied
__global__ void compact_offsets_kernel(const int32_t *__restrict__ bo, const int32_t *__restrict__ pos,
                                       int32_t *bo_c) {
    const int t = threadIdx.x;
    const int lo = bo[0], hi = bo[kBinCta];
    if (t <= kBins) bo_c[t] = t <= kBinCta ? hi - pos[hi - lo] + pos[bo[t] - lo] : bo[t];
}

// dst[u + dst_off[gid[u]]] = src[u]: per-graph blocks moved by per-graph offsets
__global__ void scatter_blocks_kernel(int32_t n, const int32_t *__restrict__ gid,
                                      const int32_t *__restrict__ dst_off,
                                      const int32_t *__restrict__ src, int32_t *dst) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        dst[u + dst_off[gid[u]]] = src[u];
}

// one output graph of assemble(): vertex, arc and original-vertex blocks of
// a source union and their places in the new union
struct Blk {
    int src;          // 0: current union, 1 + j: j-th set of new graphs
    int v0, nv, dv0;  // vertices
    int a0, na, da0;  // arcs
    int o0, no, do0;  // original vertices
};

// Rows (offsets shifted to the new arc start), arcs (columns shifted to the
// new vertex start), graph ids, and the original-vertex map (shifted like the
// columns).  Work items are parts of output graphs: part p of block b covers
// the p-th of `parts[b]` equal slices of each of its three ranges, so a large
// graph is copied by many CTAs.  Sources are indexed by Blk::src.
__global__ void __launch_bounds__(512) assemble_kernel(int nitems, const int2 *__restrict__ items,
                                                       const Blk *__restrict__ blk,
                                                       const int32_t *const *__restrict__ offs,
                                                       const int2 *const *__restrict__ arcss,
                                                       const int32_t *const *__restrict__ maps,
                                                       int32_t *off_out, int2 *arcs_out,
                                                       int32_t *gid_out, int32_t *map_out,
                                                       int32_t *gid_orig_out) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 item = items[it];  // {block, part | parts << 16}
        const int b = item.x, part = item.y & 0xffff, parts = item.y >> 16;
        const Blk B = blk[b];
        const int32_t *off = offs[B.src];
        const int2 *arcs = arcss[B.src];
        const int32_t *mp = maps[B.src];
        const int dv = B.dv0 - B.v0, da = B.da0 - B.a0;
        const int lv = (B.nv + parts - 1) / parts, la = (B.na + parts - 1) / parts,
                  lo = (B.no + parts - 1) / parts;
        for (int i = part * lv + threadIdx.x; i < min(B.nv, (part + 1) * lv); i += blockDim.x) {
            off_out[B.dv0 + i] = off[B.v0 + i] + da;
            gid_out[B.dv0 + i] = b;
        }
        for (int e = part * la + threadIdx.x; e < min(B.na, (part + 1) * la); e += blockDim.x) {
            int2 a = arcs[B.a0 + e];
            a.x += dv;
            arcs_out[B.da0 + e] = a;
        }
        for (int u = part * lo + threadIdx.x; u < min(B.no, (part + 1) * lo); u += blockDim.x) {
            map_out[B.do0 + u] = mp[B.o0 + u] + dv;
            gid_orig_out[B.do0 + u] = b;
        }
    }
}

}  // namespace

// ------------------------------------------------------- shared helpers
lv_status graph_of(int32_t n, int32_t G, const int32_t *gptr, int32_t *gid, cudaStream_t s) {
    if (n <= 0) return LV_OK;
    graph_of_kernel<<<grid_n(n), 256, 0, s>>>(n, G, gptr, gid);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status cross_check(const DGraph &g, const int32_t *gid, const int32_t *gptr, int *bad,
                      cudaStream_t s) {
    if (g.n <= 0) return LV_OK;
    cross_check_kernel<<<grid_for(g.n, 8, g_num_sms * 16), 256, 0, s>>>(g, gid, gptr, bad);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status graph_sums(int32_t n, const int32_t *gid, const int32_t *k, const int32_t *loop,
                     const uint8_t *active, unsigned long long *sum_k, unsigned long long *sum_loop,
                     unsigned long long *sum_k2, cudaStream_t s) {
    if (n <= 0) return LV_OK;
    graph_sums_kernel<<<grid_n(n), 256, 0, s>>>(n, gid, k, loop, active, sum_k, sum_loop, sum_k2);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status gather_at(int32_t G, const int32_t *idx, const int32_t *arr, int32_t *out, cudaStream_t s) {
    gather_at_kernel<<<grid_n(G + 1), 256, 0, s>>>(G, idx, arr, out);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

lv_status scatter_blocks(int32_t n, const int32_t *gid, const int32_t *dst_off, const int32_t *src,
                         int32_t *dst, cudaStream_t s) {
    if (n <= 0) return LV_OK;
    scatter_blocks_kernel<<<grid_n(n), 256, 0, s>>>(n, gid, dst_off, src, dst);
    LV_LAUNCH_CHECK();
    return LV_OK;
}

}  // namespace lv

namespace lv {

// ---------------------------------------------------------------- engine
void Engine::free_phase() {
    dfree(ps.C, s);
    dfree(ps.comm[0], s);
    dfree(ps.moves[0], s);
    dfree(ps.stats, s);
    dfree(ps.act, s);
    dfree(ps.move_count, s);
    ps = PhaseState();
    dfree(newid, s);
    newid = nullptr;
}

void Engine::release() {
    free_phase();
    sg.reset();
    dfree(labels, s);
    labels = nullptr;
    free_graph(g, s);
    dfree(k, s);
    dfree(loop, s);
    dfree(gid, s);
    dfree(gptr_d, s);
    dfree(two_m_d, s);
    dfree(map, s);
    dfree(gid_orig, s);
    k = loop = gid = gptr_d = map = gid_orig = nullptr;
    two_m_d = nullptr;
    graphs.clear();
    gp.clear();
    optr.clear();
    n_orig = 0;
    if (pin_block) {
        cudaStreamSynchronize(s);
        cudaFreeHost(pin_block);
    }
    pin_block = nullptr;
    pin_cap = 0;
}

lv_status Engine::ensure_pinned(size_t G) {
    if (G <= pin_cap && pin_block) return LV_OK;
    const size_t cap = std::max<size_t>(G, 2 * pin_cap);
    if (pin_block) {
        LV_CUDA(cudaStreamSynchronize(s));
        cudaFreeHost(pin_block);
        pin_block = nullptr;
    }
    const size_t bytes = 8 * 3 * cap + ((sizeof(IterStats) + 15) & ~size_t(15)) + cap + 64;
    if (cudaMallocHost(&pin_block, bytes) != cudaSuccess) {
        pin_block = nullptr;
        pin_cap = 0;
        return LV_ERR_OOM;
    }
    char *p = static_cast<char *>(pin_block);
    pin_u64 = reinterpret_cast<unsigned long long *>(p);
    p += 8 * 3 * cap;
    pin_stats = reinterpret_cast<IterStats *>(p);
    p += (sizeof(IterStats) + 15) & ~size_t(15);
    pin_flags = reinterpret_cast<uint8_t *>(p);
    pin_cap = cap;
    return LV_OK;
}

// arc offsets of a union at its graph starts (host)
static lv_status arc_starts(const DGraph &u, const std::vector<int32_t> &starts,
                            std::vector<int32_t> *out, cudaStream_t s) {
    const int32_t G = (int32_t)starts.size() - 1;
    out->assign(starts.size(), 0);
    if (G < 1) return LV_OK;
    int32_t *d = nullptr;
    LV_TRY(dalloc_n(&d, 2 * starts.size(), s));
    LV_CUDA(cudaMemcpyAsync(d, starts.data(), sizeof(int32_t) * starts.size(), cudaMemcpyHostToDevice, s));
    LV_TRY(gather_at(G, d, u.off, d + starts.size(), s));
    LV_CUDA(cudaMemcpyAsync(out->data(), d + starts.size(), sizeof(int32_t) * starts.size(),
                            cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    dfree(d, s);
    return LV_OK;
}

lv_status Engine::assemble(const DGraph &src, const int32_t *map_src,
                           const std::vector<int32_t> &src_gp, const std::vector<int> &keep,
                           const std::vector<const Prepared *> &news) {
    std::vector<int32_t> sa;
    if (!keep.empty()) LV_TRY(arc_starts(src, src_gp, &sa, s));
    std::vector<std::vector<int32_t>> na(news.size());
    for (size_t j = 0; j < news.size(); ++j) LV_TRY(arc_starts(news[j]->vf, news[j]->vgp, &na[j], s));
    std::vector<Blk> blk;
    std::vector<EngineGraph> recs;
    std::vector<int32_t> ngp(1, 0), nop(1, 0);
    int64_t dv = 0, da = 0, dor = 0;
    auto add = [&](Blk b) {
        b.dv0 = (int)dv;
        b.da0 = (int)da;
        b.do0 = (int)dor;
        dv += b.nv;
        da += b.na;
        dor += b.no;
        blk.push_back(b);
        ngp.push_back((int32_t)dv);
        nop.push_back((int32_t)dor);
    };
    for (int gi : keep) {
        Blk b;
        b.src = 0;
        b.v0 = src_gp[gi];
        b.nv = src_gp[gi + 1] - src_gp[gi];
        b.a0 = sa[gi];
        b.na = sa[gi + 1] - sa[gi];
        b.o0 = optr[gi];
        b.no = optr[gi + 1] - optr[gi];
        add(b);
        recs.push_back(graphs[gi]);
    }
    for (size_t j = 0; j < news.size(); ++j) {
        const Prepared &pr = *news[j];
        const int32_t Gn = (int32_t)pr.vgp.size() - 1;
        for (int32_t q = 0; q < Gn; ++q) {
            Blk b;
            b.src = 1 + (int)j;
            b.v0 = pr.vgp[q];
            b.nv = pr.vgp[q + 1] - pr.vgp[q];
            b.a0 = na[j][q];
            b.na = na[j][q + 1] - na[j][q];
            b.o0 = pr.ng.gptr[q];
            b.no = pr.ng.gptr[q + 1] - pr.ng.gptr[q];
            add(b);
            EngineGraph r;
            r.tag = pr.ng.tags[q];
            r.n_orig = b.no;
            r.two_m = pr.ng.two_m[q];
            recs.push_back(r);
        }
    }
    if (dv > 0x7ffffffell || da > 0x7fffffffll || dor > 0x7ffffffell) return LV_ERR_OVERFLOW;
    const int nb = (int)blk.size();
    const int nsrc = 1 + (int)news.size();
    std::vector<const void *> ptrs(3 * (size_t)nsrc);
    ptrs[0] = src.off;
    ptrs[nsrc] = src.arcs;
    ptrs[2 * nsrc] = map_src;
    for (size_t j = 0; j < news.size(); ++j) {
        ptrs[1 + j] = news[j]->vf.off;
        ptrs[nsrc + 1 + j] = news[j]->vf.arcs;
        ptrs[2 * nsrc + 1 + j] = news[j]->vmap;
    }
    DGraph out;
    out.n = (int32_t)dv;
    out.A = (int32_t)da;
    int32_t *gid2 = nullptr, *map2 = nullptr, *gido2 = nullptr, *gptr2 = nullptr;
    long long *tm2 = nullptr;
    Blk *dblk = nullptr;
    const void **dptr = nullptr;
    LV_TRY(dalloc_n(&out.off, (size_t)out.n + 1, s));
    LV_TRY(dalloc_n(&out.arcs, (size_t)out.A, s));
    LV_TRY(dalloc_n(&gid2, (size_t)out.n, s));
    LV_TRY(dalloc_n(&map2, (size_t)dor, s));
    LV_TRY(dalloc_n(&gido2, (size_t)dor, s));
    LV_TRY(dalloc_n(&gptr2, (size_t)nb + 1, s));
    LV_TRY(dalloc_n(&tm2, (size_t)std::max(nb, 1), s));
    LV_TRY(dalloc_n(&dblk, (size_t)std::max(nb, 1), s));
    LV_TRY(dalloc_n(&dptr, ptrs.size(), s));
    std::vector<long long> tmh(nb);
    for (int b = 0; b < nb; ++b) tmh[b] = recs[b].two_m;
    // parts of at most 64K elements per range (and at most 65535 parts)
    std::vector<int2> items;
    for (int b = 0; b < nb; ++b) {
        const int64_t len = std::max({(int64_t)blk[b].nv, (int64_t)blk[b].na, (int64_t)blk[b].no});
        const int parts = (int)std::min<int64_t>(65535, std::max<int64_t>(1, (len + 65535) >> 16));
        for (int p = 0; p < parts; ++p) items.push_back(make_int2(b, p | (parts << 16)));
    }
    int2 *ditems = nullptr;
    LV_TRY(dalloc_n(&ditems, std::max<size_t>(items.size(), 1), s));
    if (nb > 0) {
        LV_CUDA(cudaMemcpyAsync(ditems, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, s));
        LV_CUDA(cudaMemcpyAsync(dblk, blk.data(), sizeof(Blk) * nb, cudaMemcpyHostToDevice, s));
        LV_CUDA(cudaMemcpyAsync(tm2, tmh.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice, s));
        LV_CUDA(cudaMemcpyAsync(gptr2, ngp.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, s));
        LV_CUDA(cudaMemcpyAsync(dptr, ptrs.data(), sizeof(void *) * ptrs.size(), cudaMemcpyHostToDevice, s));
        assemble_kernel<<<(int)std::min<size_t>(items.size(), (size_t)g_num_sms * 4), 512, 0, s>>>(
            (int)items.size(), ditems, dblk, reinterpret_cast<const int32_t *const *>(dptr),
            reinterpret_cast<const int2 *const *>(dptr + nsrc),
            reinterpret_cast<const int32_t *const *>(dptr + 2 * nsrc), out.off, out.arcs, gid2, map2,
            gido2);
        LV_LAUNCH_CHECK();
    }
    const int32_t A_out = out.A;
    LV_CUDA(cudaMemcpyAsync(out.off + out.n, &A_out, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int32_t *k2 = nullptr, *l2 = nullptr;
    LV_TRY(dalloc_n(&k2, (size_t)out.n, s));
    LV_TRY(dalloc_n(&l2, (size_t)out.n, s));
    LV_TRY(compute_degrees(out, k2, l2, s));
    LV_CUDA(cudaStreamSynchronize(s));  // host vectors above are read by the copies
    dfree(dblk, s);
    dfree(dptr, s);
    dfree(ditems, s);
    // the new union replaces the old one
    free_graph(g, s);
    dfree(k, s);
    dfree(loop, s);
    dfree(gid, s);
    dfree(gptr_d, s);
    dfree(two_m_d, s);
    dfree(map, s);
    dfree(gid_orig, s);
    g = out;
    k = k2;
    loop = l2;
    gid = gid2;
    gptr_d = gptr2;
    two_m_d = tm2;
    map = map2;
    gid_orig = gido2;
    gp = ngp;
    optr = nop;
    n_orig = dor;
    graphs.swap(recs);
    return LV_OK;
}

void Prepared::release() {
    if (own_vf) free_graph(vf, s);
    own_vf = false;
    vf = DGraph();
    dfree(vmap, s);
    vmap = nullptr;
    if (own_input) {
        free_graph(ng.g, s);
        dfree(const_cast<int32_t *>(ng.k), s);
        dfree(const_cast<int32_t *>(ng.loop), s);
        ng.g = DGraph();
        ng.k = ng.loop = nullptr;
    }
    own_input = false;
}

lv_status prepare_graphs(const NewGraphs &ng, const lv_params &P, int *pinned, cudaStream_t s,
                         Prepared *out) {
    out->s = s;
    out->ng.gptr = ng.gptr;
    out->ng.two_m = ng.two_m;
    out->ng.tags = ng.tags;
    const int32_t Gn = (int32_t)ng.gptr.size() - 1;
    if (Gn < 1) return LV_OK;
    const int32_t n_new = ng.gptr[Gn];
    out->vf = ng.g;
    out->vgp = ng.gptr;
    LV_TRY(dalloc_n(&out->vmap, (size_t)n_new, s));
    if (!P.vertex_following) {
        LV_TRY(iota(n_new, out->vmap, s));
        LV_CUDA(cudaStreamSynchronize(s));
        return LV_OK;
    }
    // vertex following on the new union (Sec. 4.3; never crosses graphs)
    DGraph vf;
    LV_TRY(vertex_following(ng.g, ng.loop, &vf, out->vmap, pinned, s));
    out->vf = vf;
    out->own_vf = true;
    int32_t *gptr_n = nullptr, *gid_n = nullptr, *gid_vf = nullptr;
    struct Tmp {
        cudaStream_t s;
        int32_t **a, **b, **c;
        ~Tmp() {
            dfree(*a, s);
            dfree(*b, s);
            dfree(*c, s);
        }
    } tmp{s, &gptr_n, &gid_n, &gid_vf};
    LV_TRY(dalloc_n(&gptr_n, 2 * ((size_t)Gn + 1), s));
    LV_TRY(dalloc_n(&gid_n, (size_t)n_new, s));
    LV_TRY(dalloc_n(&gid_vf, (size_t)std::max(vf.n, 1), s));
    LV_CUDA(cudaMemcpyAsync(gptr_n, ng.gptr.data(), sizeof(int32_t) * (Gn + 1), cudaMemcpyHostToDevice, s));
    LV_TRY(graph_of(n_new, Gn, gptr_n, gid_n, s));
    gid_scatter_kernel<<<grid_n(n_new), 256, 0, s>>>(n_new, gid_n, nullptr, out->vmap, gid_vf);
    LV_LAUNCH_CHECK();
    int32_t *vgp_d = gptr_n + Gn + 1;
    LV_CUDA(cudaMemsetAsync(vgp_d, 0xff, sizeof(int32_t) * ((size_t)Gn + 1), s));
    if (vf.n > 0) {
        gptr_kernel<<<grid_n(vf.n), 256, 0, s>>>(vf.n, Gn, gid_vf, vgp_d);
        LV_LAUNCH_CHECK();
    }
    LV_CUDA(cudaMemcpyAsync(out->vgp.data(), vgp_d, sizeof(int32_t) * (Gn + 1), cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    for (int32_t j = 0; j < Gn; ++j)
        if (out->vgp[j] < 0 || out->vgp[j + 1] <= out->vgp[j]) return LV_ERR_CUDA;  // each keeps a vertex
    return LV_OK;
}

lv_status Engine::append_prepared(const std::vector<const Prepared *> &prs) {
    std::vector<const Prepared *> news;
    for (const Prepared *p : prs)
        if (p && p->vgp.size() >= 2) news.push_back(p);
    if (news.empty()) return LV_OK;
    std::vector<int> keep(graphs.size());
    for (size_t i = 0; i < keep.size(); ++i) keep[i] = (int)i;
    return assemble(g, map, gp, keep, news);
}

lv_status Engine::append(const NewGraphs &ng) {
    Prepared pr;
    LV_TRY(prepare_graphs(ng, P, pinned, s, &pr));
    return append_prepared({&pr});
}

}  // namespace lv

namespace lv {

lv_status Engine::phase_run() {
    const int32_t G = num_graphs();
    dfree(labels, s);
    labels = nullptr;
    free_phase();
    if (G == 0) return LV_OK;
    const double theta = P.theta_low;  // engine phases are uncoloured
    const int32_t rnd = round++;
    LV_TRY(ensure_pinned((size_t)G));
    const size_t gsum_bytes = sizeof(unsigned long long) * 3 * (size_t)G;
    // per-graph sizes of the phase graphs
    std::vector<int32_t> ga;
    LV_TRY(arc_starts(g, gp, &ga, s));
    for (int32_t q = 0; q < G; ++q) {
        graphs[q].n = gp[q + 1] - gp[q];
        graphs[q].arcs = ga[q + 1] - ga[q];
    }

    // phase state over the union
    const int32_t n = g.n;
    ps.g = g;
    ps.k = k;
    ps.loop = loop;
    ps.gid = gid;
    ps.two_m_g = two_m_d;
    ps.coloured = false;
    ps.n_act = 1;
    ps.two_m = 0;
    LV_TRY(dalloc_n(&ps.C, (size_t)n, s));
    LV_TRY(dalloc_n(&ps.comm[0], (size_t)n, s));
    LV_TRY(dalloc_n(&ps.moves[0], (size_t)n, s));
    LV_TRY(dalloc_n(&ps.stats, 1, s));
    LV_TRY(dalloc_n(&ps.act, 1, s));
    LV_TRY(dalloc_n(&ps.move_count, 4, s));
    LV_TRY(dalloc_n(&newid, (size_t)n + 1, s));
    ps.bar = &ps.stats->bar;
    LV_CUDA(cudaMemsetAsync(ps.act, 0, sizeof(int32_t), s));
    // per-phase scratch, freed below
    struct Scratch {
        cudaStream_t s;
        unsigned long long *gsum = nullptr;
        uint8_t *flags = nullptr;
        int32_t *order_c = nullptr, *bo_c = nullptr, *pos = nullptr, *tmp = nullptr;
        Buckets b;
        bool have_b = false;
        ~Scratch() {
            dfree(gsum, s);
            dfree(flags, s);
            dfree(order_c, s);
            dfree(bo_c, s);
            dfree(pos, s);
            dfree(tmp, s);
            if (have_b) free_buckets(b, s);
        }
    } sc;
    sc.s = s;
    LV_TRY(dalloc_n(&sc.gsum, 3 * (size_t)G, s));
    LV_TRY(dalloc_n(&sc.flags, (size_t)G, s));
    LV_TRY(dalloc_n(&sc.order_c, (size_t)n, s));
    LV_TRY(dalloc_n(&sc.bo_c, (size_t)kBins + 2, s));
    LV_TRY(dalloc_n(&sc.pos, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&sc.tmp, (size_t)G + 1, s));
    ps.active_g = sc.flags;
    ps.g_ein = sc.gsum;
    ps.g_a2 = sc.gsum + G;
    ps.g_moved = sc.gsum + 2 * (size_t)G;

    // ---- initial state and N_start of every graph
    const int ev_i0 = timer ? timer->mark() : -1;
    LV_TRY(init_phase(ps, s));
    for (int32_t q = 0; q < G; ++q) {
        EngineGraph &t = graphs[q];
        t.running = true;
        t.stop = false;
        t.step = 0;
        t.have_np = false;
        t.n_p = 0;
        t.iters = 0;
        pin_flags[q] = 1;
    }
    int n_running = G;
    LV_CUDA(cudaMemcpyAsync(sc.flags, pin_flags, (size_t)G, cudaMemcpyHostToDevice, s));
    LV_CUDA(cudaMemsetAsync(sc.gsum, 0, gsum_bytes, s));
    LV_TRY(graph_sums(n, gid, k, loop, sc.flags, nullptr, sc.gsum, sc.gsum + G, s));
    LV_CUDA(cudaMemcpyAsync(pin_u64, sc.gsum, sizeof(unsigned long long) * 2 * (size_t)G,
                            cudaMemcpyDeviceToHost, s));
    LV_CUDA(cudaStreamSynchronize(s));
    for (int32_t q = 0; q < G; ++q)
        graphs[q].N_start = graphs[q].two_m * (int64_t)pin_u64[q] - (int64_t)pin_u64[G + q];

    // ---- degree bins (measured once per round when autotuning)
    BinLimits plim = lim;
    if (P.autotune && tuned && tuned_ok && g.A >= kTuneMinArcs) {
        if ((int32_t)tuned->size() <= rnd || !(*tuned_ok)[rnd]) {
            BinLimits best = lim;
            LV_TRY(tune_bins(ps, lim, sc.gsum, gsum_bytes, &best, pinned, s));
            if ((int32_t)tuned->size() <= rnd) {
                tuned->resize(rnd + 1);
                tuned_ok->resize(rnd + 1, 0);
            }
            (*tuned)[rnd] = best;
            (*tuned_ok)[rnd] = 1;
        }
        plim = (*tuned)[rnd];
    }
    sc.have_b = true;
    LV_TRY(bucket_vertices(g, nullptr, 1, plim, &sc.b, pinned, s));

    // ---- batched iterations (Alg. 1 per graph, fused modularity)
    sg.reset();  // new phase graph: recapture
    int32_t sweep_no = 0;
    Buckets bl = sc.b;  // the vertex list the sweeps walk (compacted as graphs stop)
    const int glo = sc.b.host_off[0], ghi = sc.b.host_off[kBinCta];
    int64_t listed = n;  // vertices of the graphs in the list
    while (n_running > 0) {
        lv_batch_sweep rec;
        std::memset(&rec, 0, sizeof rec);
        rec.phase = rnd;
        rec.sweep = ++sweep_no;
        rec.graphs = n_running;
        for (int32_t q = 0; q < G; ++q)
            if (graphs[q].running) {
                rec.vertices += graphs[q].n;
                rec.arcs += graphs[q].arcs;
            }
        auto enqueue = [&]() -> lv_status {
            LV_CUDA(cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s));
            LV_CUDA(cudaMemsetAsync(ps.move_count, 0, 3 * sizeof(int32_t), s));
            LV_CUDA(cudaMemsetAsync(sc.gsum, 0, gsum_bytes, s));
            return sweep_iteration(ps, bl, s);
        };
        if (P.graph_capture && !sg.disabled &&
            (!sg.exec || sg.order != bl.order || sg.bo != bl.bucket_off)) {
            sg.reset();
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const lv_status est = enqueue();
                if (est == LV_OK) g_kernel_launches.fetch_sub(1);  // captured, not launched
                const cudaError_t ce = cudaStreamEndCapture(s, &graph);
                ok = est == LV_OK && ce == cudaSuccess && graph &&
                     cudaGraphInstantiate(&sg.exec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
            }
            if (ok) {
                sg.order = bl.order;
                sg.bo = bl.bucket_off;
            } else {
                cudaGetLastError();
                sg.reset();
                sg.disabled = true;
            }
        }
        if (timer) ev_sweep.push_back(timer->mark());
        if (sg.exec) {
            LV_CUDA(cudaGraphLaunch(sg.exec, s));
            ++g_kernel_launches;
            ++graph_launches;
        } else {
            LV_TRY(enqueue());
        }
        if (timer) ev_sweep.push_back(timer->mark());
        ++sweep_launches;
        LV_CUDA(cudaMemcpyAsync(pin_stats, ps.stats, sizeof(IterStats), cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaMemcpyAsync(pin_u64, sc.gsum, gsum_bytes, cudaMemcpyDeviceToHost, s));
        LV_CUDA(cudaStreamSynchronize(s));
        if (barrier_flags(pin_stats->bar)) return LV_ERR_TIMEOUT;
        if (pin_stats->err) return LV_ERR_HASH;
        for (int32_t q = 0; q < G; ++q) {
            EngineGraph &t = graphs[q];
            if (!t.running) continue;
            const int step = ++t.step;
            // N(C^{step-1}) of this graph, read by the sweep under the labels it used
            const int64_t N_prev = t.two_m * (int64_t)pin_u64[q] - (int64_t)pin_u64[G + q];
            const int64_t moved = (int64_t)pin_u64[2 * (size_t)G + q];
            rec.moved += moved;
            bool fin = false;
            if (step == 1) {
                if (moved == 0) {
                    t.iters = 1;
                    fin = true;
                }
            } else {
                const int tt = step - 1;
                if ((t.have_np && gain_below(N_prev, t.n_p, theta, P.abs_threshold != 0)) ||
                    tt >= P.max_iters) {
                    t.iters = tt;
                    fin = true;
                } else {
                    t.n_p = N_prev;
                    t.have_np = true;
                    if (moved == 0) {
                        t.iters = step;
                        fin = true;
                    }
                }
            }
            if (fin) {
                t.N_end = N_prev;
                t.running = false;
                pin_flags[q] = 0;
                --n_running;
            }
        }
        sweeps.push_back(rec);
        if (n_running > 0) {
            // graphs that go on apply their moves and are swept again
            LV_CUDA(cudaMemcpyAsync(sc.flags, pin_flags, (size_t)G, cudaMemcpyHostToDevice, s));
            apply_batch_kernel<<<g_num_sms * 4, 256, 0, s>>>(ps.C, ps.comm[0], ps.moves[0],
                                                              ps.move_count, gid, sc.flags);
            LV_LAUNCH_CHECK();
            int64_t live_v = 0;
            for (int32_t q = 0; q < G; ++q)
                if (graphs[q].running) live_v += graphs[q].n;
            if (ghi > glo && live_v * 4 < listed * 3) {
                // drop stopped graphs from the group bins (from the full list)
                keep_flags_kernel<<<grid_n(ghi - glo), 256, 0, s>>>(sc.b.order, glo, ghi, gid,
                                                                     sc.flags, sc.pos);
                LV_LAUNCH_CHECK();
                LV_TRY(scan_excl_i32(sc.pos, sc.pos, ghi - glo, s));
                compact_kernel<<<grid_n(ghi - glo), 256, 0, s>>>(sc.b.order, glo, ghi, sc.pos,
                                                                 sc.order_c);
                LV_LAUNCH_CHECK();
                if (bl.order != sc.order_c) {  // first compaction: CTA, hub and skip bins
                    const int tail = sc.b.host_off[kBins + 1] - ghi;
                    if (tail > 0)
                        LV_CUDA(cudaMemcpyAsync(sc.order_c + ghi, sc.b.order + ghi,
                                                sizeof(int32_t) * (size_t)tail,
                                                cudaMemcpyDeviceToDevice, s));
                    LV_CUDA(cudaMemcpyAsync(sc.bo_c + kBins + 1, sc.b.bucket_off + kBins + 1,
                                            sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                }
                compact_offsets_kernel<<<1, 32, 0, s>>>(sc.b.bucket_off, sc.pos, sc.bo_c);
                LV_LAUNCH_CHECK();
                bl.order = sc.order_c;
                bl.bucket_off = sc.bo_c;
                listed = live_v;
            }
        }
    }
    sg.reset();  // it refers to this phase's buffers
    const int ev_i1 = timer ? timer->mark() : -1;

    // ---- renumber and labels of every graph (Sec. 4.5)
    const int ev_r0 = timer ? timer->mark() : -1;
    LV_TRY(renumber(n, ps.comm[0], newid, s));
    LV_TRY(gather_at(G, gptr_d, newid, sc.tmp, s));
    gstart.assign((size_t)G + 1, 0);
    LV_CUDA(cudaMemcpyAsync(gstart.data(), sc.tmp, sizeof(int32_t) * ((size_t)G + 1),
                            cudaMemcpyDeviceToHost, s));
    LV_TRY(dalloc_n(&labels, (size_t)std::max<int64_t>(n_orig, 1), s));
    LV_TRY(compose_labels((int32_t)n_orig, map, ps.C, newid, labels, s));
    if (n_orig > 0) {
        localize_kernel<<<grid_n(n_orig), 256, 0, s>>>((int32_t)n_orig, gid_orig, sc.tmp, labels);
        LV_LAUNCH_CHECK();
    }
    LV_CUDA(cudaStreamSynchronize(s));
    n_next = gstart[G];
    for (int32_t q = 0; q < G; ++q) {
        EngineGraph &t = graphs[q];
        lv_phase_info in;
        std::memset(&in, 0, sizeof in);
        in.n = t.n;
        in.arcs = t.arcs;
        in.n_next = (int64_t)gstart[q + 1] - gstart[q];
        in.two_m = t.two_m;
        in.N_start = t.N_start;
        in.N_end = t.N_end;
        in.q = (double)t.N_end / ((double)t.two_m * (double)t.two_m);
        in.theta = theta;
        in.iterations = t.iters;
        in.ms_color = in.ms_iterate = in.ms_rebuild = -1.0;
        t.info.push_back(in);
        t.stop = in.n_next == in.n ||
                 gain_below(t.N_end, t.N_start, P.theta_low, P.abs_threshold != 0) ||
                 (int32_t)t.info.size() >= P.max_phases;
    }
    if (timer) {
        ev_iter.push_back(ev_i0);
        ev_iter.push_back(ev_i1);
        ev_reb.push_back(ev_r0);
    }
    return LV_OK;
}

lv_status Engine::phase_end(std::vector<Finished> &finished) {
    const int32_t G = num_graphs();
    if (G == 0 || !newid) return LV_OK;
    std::vector<int> keep;
    for (int32_t q = 0; q < G; ++q) {
        if (graphs[q].stop) {
            Finished f;
            f.rec = graphs[q];
            f.lab_off = optr[q];
            finished.push_back(f);
        } else {
            keep.push_back(q);
        }
    }
    lv_status st = LV_OK;
    if (keep.empty()) {
        // every graph is done: the union goes away (labels stay for the caller)
        free_graph(g, s);
        dfree(k, s);
        dfree(loop, s);
        dfree(gid, s);
        dfree(gptr_d, s);
        dfree(two_m_d, s);
        dfree(map, s);
        dfree(gid_orig, s);
        k = loop = gid = gptr_d = map = gid_orig = nullptr;
        two_m_d = nullptr;
        graphs.clear();
        gp.clear();
        optr.clear();
        n_orig = 0;
    } else {
        DGraph G2;
        st = coarsen(g, ps.C, newid, n_next, &G2, pinned, s);
        if (st == LV_OK && (int32_t)keep.size() == G) {
            // every graph goes on: the coarse union is the new union
            int32_t *gid2 = nullptr, *k2 = nullptr, *l2 = nullptr;
            st = dalloc_n(&gid2, (size_t)G2.n, s);
            if (st == LV_OK) st = dalloc_n(&k2, (size_t)G2.n, s);
            if (st == LV_OK) st = dalloc_n(&l2, (size_t)G2.n, s);
            if (st == LV_OK) {
                gid_scatter_kernel<<<grid_n(g.n), 256, 0, s>>>(g.n, gid, ps.C, newid, gid2);
                st = cudaGetLastError() == cudaSuccess ? LV_OK : LV_ERR_CUDA;
                ++g_kernel_launches;
            }
            if (st == LV_OK) st = compute_degrees(G2, k2, l2, s);
            if (st == LV_OK &&
                cudaMemcpyAsync(gptr_d, gstart.data(), sizeof(int32_t) * ((size_t)G + 1),
                                cudaMemcpyHostToDevice, s) != cudaSuccess)
                st = LV_ERR_CUDA;
            if (st == LV_OK && cudaStreamSynchronize(s) != cudaSuccess) st = LV_ERR_CUDA;
            if (st == LV_OK) {
                free_graph(g, s);
                dfree(k, s);
                dfree(loop, s);
                dfree(gid, s);
                g = G2;
                k = k2;
                loop = l2;
                gid = gid2;
                gp = gstart;
            } else {
                free_graph(G2, s);
                dfree(gid2, s);
                dfree(k2, s);
                dfree(l2, s);
            }
        } else if (st == LV_OK) {
            // graphs that stopped leave: the kept coarse graphs are packed
            st = assemble(G2, map, gstart, keep, {});
            free_graph(G2, s);
        }
    }
    if (timer) ev_reb.push_back(timer->mark());
    free_phase();
    return st;
}

}  // namespace lv
