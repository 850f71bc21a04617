// lv_tune.cu -- choice of the sweep's degree bins, blocks per SM and hub table
// size by measurement.
//
// The bins decide how many lanes (or CTAs) sweep a vertex and how large its
// hash table is; the blocks per SM and the hub tables' slots per arc decide
// the launch shape and the probe chains.  None of them changes a decision,
// so any set is correct and the best one depends on the degree distribution
// and the hardware.  In an
// uncoloured phase a sweep only reads the labels and the community state and
// writes its move list and statistics (the moves are applied by a separate
// step), so candidate sets can be timed on the live phase state and the run
// continues unchanged.
#include "lv_ops.cuh"

namespace lv {

namespace {
// bin sets tried after the caller's (lane_arcs, warp_max, cta_max)
constexpr int kCands[][3] = {{4, 128, 4096}, {8, 256, 1024}, {2, 128, 4096}};
}  // namespace

// Times one sweep of the phase state with the limits `lim` (bucketing not
// timed).  *has_hubs reports whether the buckets hold hub vertices.
static lv_status time_sweep(PhaseState &ps, const BinLimits &lim, void *zero, size_t zero_bytes,
                            int reps, cudaEvent_t e0, cudaEvent_t e1, float *ms, bool *has_hubs,
                            int *pinned, cudaStream_t s) {
    Buckets b;
    lv_status st = bucket_vertices(ps.g, nullptr, 1, lim, &b, pinned, s);
    *has_hubs = b.hub_slots > 0;
    for (int rep = 0; rep < reps && st == LV_OK; ++rep) {
        if (cudaMemsetAsync(ps.stats, 0, sizeof(IterStats), s) != cudaSuccess ||
            cudaMemsetAsync(ps.move_count, 0, 3 * sizeof(int32_t), s) != cudaSuccess ||
            (zero && cudaMemsetAsync(zero, 0, zero_bytes, s) != cudaSuccess) ||
            cudaEventRecord(e0, s) != cudaSuccess) {
            st = LV_ERR_CUDA;
            break;
        }
        st = sweep_iteration(ps, b, s);
        if (st != LV_OK) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            st = LV_ERR_CUDA;
    }
    if (st == LV_OK) {
        IterStats hs;
        if (cudaMemcpy(&hs, ps.stats, sizeof hs, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LV_ERR_CUDA;
        else if (barrier_flags(hs.bar))
            st = LV_ERR_TIMEOUT;
        else if (hs.err)
            st = LV_ERR_HASH;
    }
    free_buckets(b, s);
    return st;
}

// Coordinate search: the bin sets first, then, with the best bins, one
// sweep block per SM instead of two, then (when the phase has hubs) hub
// tables of 4 slots per arc instead of 2.  Six timed sweeps at most.
lv_status tune_bins(PhaseState &ps, const BinLimits &first, void *zero, size_t zero_bytes,
                    BinLimits *best, int *pinned, cudaStream_t s) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LV_CUDA(cudaEventCreate(&e0));
    LV_CUDA(cudaEventCreate(&e1));
    // a sweep first warms L2 and the TLBs, unless its arcs alone (8 B each)
    // are twice the 129 MB L2: then one timed sweep per candidate suffices
    const int reps = (int64_t)ps.g.A * 8 >= (int64_t)2 * 129 * 1000 * 1000 ? 1 : 2;
    float best_ms = 0.f, ms = 0.f;
    bool hubs = false, h = false;
    *best = first;
    lv_status st = time_sweep(ps, first, zero, zero_bytes, reps, e0, e1, &best_ms, &hubs, pinned, s);
    for (const auto &c : kCands) {
        if (st != LV_OK) break;
        BinLimits lim = first;
        lim.lane_arcs = c[0];
        lim.warp_max = c[1];
        lim.cta_max = c[2];
        if (lim.lane_arcs == first.lane_arcs && lim.warp_max == first.warp_max &&
            lim.cta_max == first.cta_max)
            continue;
        st = time_sweep(ps, lim, zero, zero_bytes, reps, e0, e1, &ms, &h, pinned, s);
        if (st == LV_OK && ms < best_ms) {
            best_ms = ms;
            *best = lim;
            hubs = h;
        }
    }
    if (st == LV_OK && best->blocks_per_sm != 1) {
        BinLimits lim = *best;
        lim.blocks_per_sm = 1;
        st = time_sweep(ps, lim, zero, zero_bytes, reps, e0, e1, &ms, &h, pinned, s);
        if (st == LV_OK && ms < best_ms) {
            best_ms = ms;
            *best = lim;
        }
    }
    if (st == LV_OK && hubs && best->hub_factor != 4) {
        BinLimits lim = *best;
        lim.hub_factor = 4;
        st = time_sweep(ps, lim, zero, zero_bytes, reps, e0, e1, &ms, &h, pinned, s);
        if (st == LV_OK && ms < best_ms) {
            best_ms = ms;
            *best = lim;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace lv
