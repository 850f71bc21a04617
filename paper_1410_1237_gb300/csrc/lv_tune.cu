// lv_tune.cu -- choice of the sweep's degree bins by measurement.
//
// The bins decide how many lanes (or CTAs) sweep a vertex and how large its
// hash table is; they never change a decision, so any set is correct and the
// best one depends on the degree distribution and the hardware.  In an
// uncoloured phase a sweep only reads the labels and the community state and
// writes its move list and statistics (the moves are applied by a separate
// step), so candidate sets can be timed on the live phase state and the run
// continues unchanged.
#include "lv_ops.cuh"

namespace lv {

namespace {
// candidate (lane_arcs, warp_max, cta_max); the caller's set is tried first
constexpr int kCands[][3] = {{4, 128, 4096}, {8, 128, 4096}, {8, 256, 4096},
                             {2, 128, 4096}, {8, 256, 1024}, {4, 256, 2048}};
}  // namespace

lv_status tune_bins(PhaseState &ps, const BinLimits &first, void *zero, size_t zero_bytes,
                    BinLimits *best, int *pinned, cudaStream_t s) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LV_CUDA(cudaEventCreate(&e0));
    LV_CUDA(cudaEventCreate(&e1));
    float best_ms = 0.f;
    bool have = false;
    lv_status st = LV_OK;
    const int ncand = 1 + (int)(sizeof(kCands) / sizeof(kCands[0]));
    // a sweep first warms L2 and the TLBs, unless its arcs alone (8 B each)
    // are twice the 129 MB L2: then one timed sweep per candidate suffices
    const int reps = (int64_t)ps.g.A * 8 >= (int64_t)2 * 129 * 1000 * 1000 ? 1 : 2;
    for (int c = 0; c < ncand && st == LV_OK; ++c) {
        BinLimits lim = first;
        if (c > 0) {
            lim.lane_arcs = kCands[c - 1][0];
            lim.warp_max = kCands[c - 1][1];
            lim.cta_max = kCands[c - 1][2];
            if (lim.lane_arcs == first.lane_arcs && lim.warp_max == first.warp_max &&
                lim.cta_max == first.cta_max)
                continue;
        }
        Buckets b;
        st = bucket_vertices(ps.g, nullptr, 1, lim, &b, pinned, s);
        float ms = 0.f;
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
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
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
        if (st == LV_OK && (!have || ms < best_ms)) {
            best_ms = ms;
            *best = lim;
            have = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace lv
