// lv_server.cu -- serving with continuous batching (lv.h, "serving").
//
// Requests are queued by lv_server_submit (host copies of their CSRs).  An
// admission thread and two lane workers share the device.  Lane 0 (small
// requests) loops over rounds:
//   1. admission: queued requests, first come first served, while the
//      resident requests' estimated footprint stays within the budget and
//      the slot limit; the admitted CSRs are concatenated into one union,
//      validated on the device and appended to the engine (vertex following
//      included), so they join the requests already running;
//   2. one batched phase of every resident request (lv_engine.cu);
//   3. requests whose phase loop stopped leave the engine: their labels are
//      copied to the host and their waiters are woken.
// Lane 1 solves large requests, and those that would colour a phase, one at
// a time with the single-graph driver.  Every request is computed exactly as
// lv_run computes it alone, so results do not depend on what else is resident.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lv_engine.cuh"

using namespace lv;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kBytesPerArc = 48;     // CSR, coarse rebuild and sort scratch
constexpr int64_t kBytesPerVertex = 64;  // per-vertex state, map and labels
constexpr int64_t kDefaultBudget = 120ll << 30;
constexpr int32_t kDefaultMaxGraphs = 65536;
constexpr int64_t kLaneSplitArcs = int64_t(1) << 22;  // requests at least this large use lane 1
constexpr int kPlainWorkers = 4;

struct Request {
    int64_t id = 0;
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col, w;
    int64_t est = 0;  // estimated device bytes while resident
    bool done = false;
    lv_server_result_info info;
    std::vector<int32_t> labels;
};

// requests taken from the queue, validated and vertex-followed by the
// admission thread, waiting for the next phase boundary of the worker
struct Ready {
    std::unique_ptr<Prepared> pr;
    std::vector<std::shared_ptr<Request>> reqs;
};

// Host-to-device upload through two pinned staging buffers: a chunk is
// copied into one buffer while the other's transfer runs.  Pinned transfers
// are asynchronous DMA, so a large upload by the admission thread never
// holds up the worker's own small copies.
struct PinnedRing {
    static constexpr size_t kChunk = size_t(32) << 20;
    char *buf[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int next = 0;
    lv_status init() {
        for (int i = 0; i < 2; ++i) {
            if (cudaMallocHost((void **)&buf[i], kChunk) != cudaSuccess) return LV_ERR_OOM;
            if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) return LV_ERR_CUDA;
        }
        return LV_OK;
    }
    void destroy() {
        for (int i = 0; i < 2; ++i) {
            if (ev[i]) cudaEventSynchronize(ev[i]);
            if (buf[i]) cudaFreeHost(buf[i]);
            if (ev[i]) cudaEventDestroy(ev[i]);
            buf[i] = nullptr;
            ev[i] = nullptr;
        }
    }
    lv_status h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
        const char *p = static_cast<const char *>(src);
        char *d = static_cast<char *>(dst);
        while (bytes > 0) {
            const size_t c = bytes < kChunk ? bytes : kChunk;
            LV_CUDA(cudaEventSynchronize(ev[next]));  // its previous transfer is done
            std::memcpy(buf[next], p, c);
            LV_CUDA(cudaMemcpyAsync(d, buf[next], c, cudaMemcpyHostToDevice, s));
            LV_CUDA(cudaEventRecord(ev[next], s));
            next ^= 1;
            p += c;
            d += c;
            bytes -= c;
        }
        return LV_OK;
    }
};

}  // namespace

struct lv_server {
    int device = 0;
    lv_server_config cfg;
    BinLimits lim;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_done, cv_adm;
    std::deque<std::shared_ptr<Request>> queue;
    // Two lanes, each a worker thread with its own stream.  Lane 0 batches
    // the requests with fewer than kLaneSplitArcs arcs in a multi-graph
    // engine (continuous batching at phase boundaries).  Lane 1 solves large
    // requests, and those that would colour a phase (colouring on and at
    // least color_cutoff vertices), one at a time with the single-graph
    // driver.  A small request never waits for a large one's iterations, and
    // the lanes' launches interleave on the device.
    struct Lane {
        cudaStream_t stream = nullptr;
        bool own_stream = false;
        int *pinned = nullptr;
        std::condition_variable cv_work;
        std::deque<Ready> ready;  // lane 0: admitted and prepared, not yet in the engine
        std::deque<std::shared_ptr<Request>> plain;  // lane 1: admitted, solved one at a time
        std::thread worker;
        int64_t rounds = 0, sweeps = 0;
    } lanes[2];
    // lane 1 runs kPlainWorkers solves at a time, each on its own stream
    // (lanes[1].stream is the first), each solve's persistent kernels on at
    // most half the SMs (fewer for small graphs), so that several of them
    // share the device: four solves of 3-5 M arcs ran in 30 ms side by side
    // against 85 ms one after another on the whole GPU.
    cudaStream_t plain_streams[kPlainWorkers] = {};
    std::thread plain_workers[kPlainWorkers];
    int64_t inflight = 0;     // admitted and not completed
    std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;  // until released
    int64_t next_id = 0;
    bool stop = false;
    lv_server_stats stats;
    int64_t resident_bytes = 0;
    int64_t resident_n = 0, resident_a = 0;  // input vertices and arcs of resident requests
    cudaStream_t adm_stream = nullptr;  // admission thread's stream
    int *adm_pinned = nullptr;
    PinnedRing ring;                    // admission thread's upload staging
    std::thread admitter;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

namespace {

// a thread's stream and pinned scratch
struct Ctx {
    cudaStream_t s;
    int *pinned;
    const lv_params *P;
    PinnedRing *ring;  // may be null (plain copies)
};

// Upload one CSR (or a union of several) and validate it on the device.
struct Staged {
    cudaStream_t s = nullptr;
    DGraph g;
    int32_t *k = nullptr, *loop = nullptr;
    int64_t two_m = 0;
    ~Staged() {
        free_graph(g, s);
        dfree(k, s);
        dfree(loop, s);
    }
};

lv_status stage(const Ctx &c, int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                bool limit_two_m, Staged *out) {
    cudaStream_t s = c.s;
    out->s = s;
    const int64_t A = rowptr[n];
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr, *d_w = nullptr;
    lv_status st = dalloc_n(&d_rp, (size_t)n + 1, s);
    if (st == LV_OK) st = dalloc_n(&d_col, (size_t)std::max<int64_t>(A, 1), s);
    if (st == LV_OK) st = dalloc_n(&d_w, (size_t)std::max<int64_t>(A, 1), s);
    if (st == LV_OK &&
        (cudaMemcpyAsync(d_rp, rowptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s) !=
             cudaSuccess ||
         (A > 0 && cudaMemcpyAsync(d_col, col, sizeof(int32_t) * (size_t)A, cudaMemcpyHostToDevice, s) !=
                       cudaSuccess) ||
         (A > 0 && cudaMemcpyAsync(d_w, w, sizeof(int32_t) * (size_t)A, cudaMemcpyHostToDevice, s) !=
                       cudaSuccess)))
        st = LV_ERR_CUDA;
    if (st == LV_OK)
        st = validate_and_build(n, d_rp, d_col, d_w, &out->g, &out->k, &out->loop, &out->two_m,
                                c.pinned, s, limit_two_m);
    dfree(d_rp, s);
    dfree(d_col, s);
    dfree(d_w, s);
    return st;
}

// Union of admitted CSRs uploaded graph by graph: row offsets are shifted by
// the graph's first arc and columns by its first vertex on the device.
__device__ __forceinline__ int block_of(const int32_t *starts, int G, int x) {
    int a = 0, b = G;  // last a with starts[a] <= x
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (starts[mid] <= x) a = mid; else b = mid;
    }
    return a;
}

__global__ void shift_union_kernel(int32_t n, int32_t A, int32_t G, const int32_t *__restrict__ gptr,
                                   const int32_t *__restrict__ astart, int64_t *rp, int32_t *col) {
    const int stride = gridDim.x * blockDim.x;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        rp[v] += astart[block_of(gptr, G, v)];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < A; e += stride)
        col[e] += gptr[block_of(astart, G, e)];
}

lv_status stage_union(const Ctx &c, const std::vector<std::shared_ptr<Request>> &good,
                      std::vector<int32_t> *gptr, Staged *out) {
    cudaStream_t s = c.s;
    out->s = s;
    const int32_t G = (int32_t)good.size();
    int64_t n = 0, A = 0;
    gptr->assign((size_t)G + 1, 0);
    std::vector<int32_t> astart((size_t)G + 1, 0);
    for (int32_t q = 0; q < G; ++q) {
        n += good[q]->n;
        A += (int64_t)good[q]->col.size();
        (*gptr)[q + 1] = (int32_t)n;
        astart[q + 1] = (int32_t)A;
    }
    int64_t *rp = nullptr;
    int32_t *col = nullptr, *w = nullptr, *gd = nullptr;
    struct Tmp {
        cudaStream_t s;
        int64_t **rp;
        int32_t **col, **w, **gd;
        ~Tmp() {
            dfree(*rp, s);
            dfree(*col, s);
            dfree(*w, s);
            dfree(*gd, s);
        }
    } tmp{s, &rp, &col, &w, &gd};
    LV_TRY(dalloc_n(&rp, (size_t)n + 1, s));
    LV_TRY(dalloc_n(&col, (size_t)std::max<int64_t>(A, 1), s));
    LV_TRY(dalloc_n(&w, (size_t)std::max<int64_t>(A, 1), s));
    LV_TRY(dalloc_n(&gd, 2 * ((size_t)G + 1), s));
    auto up = [&](void *dst, const void *src, size_t bytes) -> lv_status {
        if (c.ring) return c.ring->h2d(dst, src, bytes, s);
        LV_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return LV_OK;
    };
    for (int32_t q = 0; q < G; ++q) {
        const Request &r = *good[q];
        const size_t a = r.col.size();
        LV_TRY(up(rp + (*gptr)[q], r.rowptr.data(), sizeof(int64_t) * (size_t)r.n));
        if (a) {
            LV_TRY(up(col + astart[q], r.col.data(), sizeof(int32_t) * a));
            LV_TRY(up(w + astart[q], r.w.data(), sizeof(int32_t) * a));
        }
    }
    LV_TRY(up(rp + n, &A, sizeof(int64_t)));
    LV_TRY(up(gd, gptr->data(), sizeof(int32_t) * ((size_t)G + 1)));
    LV_TRY(up(gd + G + 1, astart.data(), sizeof(int32_t) * ((size_t)G + 1)));
    shift_union_kernel<<<grid_for(std::max<int64_t>(n, A), 256, g_num_sms * 16), 256, 0, s>>>(
        (int32_t)n, (int32_t)A, G, gd, gd + G + 1, rp, col);
    LV_LAUNCH_CHECK();
    return validate_and_build(n, rp, col, w, &out->g, &out->k, &out->loop, &out->two_m, c.pinned, s,
                              false);
}

// rowptr of a request must start at 0, not decrease and fit int32 arc counts
bool rowptr_ok(const Request &r) {
    if (r.rowptr.empty() || r.rowptr[0] != 0) return false;
    for (int64_t i = 0; i < r.n; ++i)
        if (r.rowptr[i + 1] < r.rowptr[i]) return false;
    return r.rowptr[r.n] == (int64_t)r.col.size() && r.rowptr[r.n] <= 0x7fffffffll;
}

// Validates the admitted requests as one union and appends them; a request
// whose CSR is invalid is completed with its error (found by validating the
// requests one by one when the union fails).
lv_status admit(const Ctx &c, std::vector<std::shared_ptr<Request>> &adm,
                std::vector<std::shared_ptr<Request>> &failed, std::unique_ptr<Prepared> *out,
                std::vector<std::shared_ptr<Request>> *joined) {
    cudaStream_t s = c.s;
    std::vector<std::shared_ptr<Request>> good;
    for (auto &r : adm) {
        if (!rowptr_ok(*r) || r->n < 1) {
            r->info.status = r->n < 1 ? LV_ERR_EMPTY : LV_ERR_ARG;
            failed.push_back(r);
        } else {
            good.push_back(r);
        }
    }
    for (int attempt = 0; attempt < 2 && !good.empty(); ++attempt) {
        int64_t n = 0, A = 0;
        for (auto &r : good) {
            n += r->n;
            A += (int64_t)r->col.size();
        }
        if (n > 0x7ffffffell || A > 0x7fffffffll) return LV_ERR_OVERFLOW;  // admission keeps below
        std::vector<int32_t> gptr;
        Staged U;
        lv_status st = stage_union(c, good, &gptr, &U);
        std::vector<long long> two_m(good.size(), 0);
        if (st == LV_OK) {
            // per-graph checks: arcs stay inside their graph, 0 < 2m < 2^31
            const int32_t G = (int32_t)good.size();
            int32_t *gp_d = nullptr, *gid = nullptr;
            int *bad = nullptr;
            unsigned long long *sk = nullptr;
            lv_status s2 = dalloc_n(&gp_d, (size_t)G + 1, s);
            if (s2 == LV_OK) s2 = dalloc_n(&gid, (size_t)n, s);
            if (s2 == LV_OK) s2 = dalloc_n(&bad, 1, s);
            if (s2 == LV_OK) s2 = dalloc_n(&sk, (size_t)G, s);
            std::vector<unsigned long long> skh((size_t)G);
            int badh = 0;
            if (s2 == LV_OK &&
                (cudaMemcpyAsync(gp_d, gptr.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s) !=
                     cudaSuccess ||
                 cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess ||
                 cudaMemsetAsync(sk, 0, sizeof(unsigned long long) * G, s) != cudaSuccess))
                s2 = LV_ERR_CUDA;
            if (s2 == LV_OK) s2 = graph_of((int32_t)n, G, gp_d, gid, s);
            if (s2 == LV_OK) s2 = cross_check(U.g, gid, gp_d, bad, s);
            if (s2 == LV_OK) s2 = graph_sums((int32_t)n, gid, U.k, U.loop, nullptr, sk, nullptr, nullptr, s);
            if (s2 == LV_OK &&
                (cudaMemcpyAsync(skh.data(), sk, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess ||
                 cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaStreamSynchronize(s) != cudaSuccess))
                s2 = LV_ERR_CUDA;
            dfree(gp_d, s);
            dfree(gid, s);
            dfree(bad, s);
            dfree(sk, s);
            if (s2 == LV_ERR_CUDA || s2 == LV_ERR_OOM) return s2;
            st = s2;
            if (st == LV_OK && badh) st = LV_ERR_ARG;
            for (int32_t q = 0; st == LV_OK && q < G; ++q) {
                if (skh[q] == 0 || skh[q] >= (1ull << 31)) st = LV_ERR_ARG;
                two_m[q] = (long long)skh[q];
            }
        }
        if (st == LV_ERR_CUDA || st == LV_ERR_OOM) return st;
        if (st == LV_OK) {
            NewGraphs ng;
            ng.g = U.g;
            ng.k = U.k;
            ng.loop = U.loop;
            ng.gptr = gptr;
            ng.two_m = two_m;
            for (auto &r : good) ng.tags.push_back(r->id);
            for (auto &r : good) {
                r->info.n = r->n;
                r->info.arcs = (int64_t)r->col.size();
            }
            std::unique_ptr<Prepared> pr(new Prepared());
            LV_TRY(prepare_graphs(ng, *c.P, c.pinned, s, pr.get()));
            if (!pr->own_vf) {  // the engine copies the staged union itself
                pr->ng.g = U.g;
                pr->ng.k = U.k;
                pr->ng.loop = U.loop;
                pr->own_input = true;
                U.g = DGraph();
                U.k = U.loop = nullptr;
            }
            for (size_t q = 0; q < good.size(); ++q) good[q]->info.two_m = two_m[q];
            *out = std::move(pr);
            *joined = good;
            return LV_OK;
        }
        // the union failed: find the invalid requests one by one
        std::vector<std::shared_ptr<Request>> keep;
        for (auto &r : good) {
            Staged one;
            const lv_status s1 = stage(c, r->n, r->rowptr.data(), r->col.data(), r->w.data(), true, &one);
            if (s1 == LV_ERR_CUDA || s1 == LV_ERR_OOM) return s1;
            if (s1 != LV_OK) {
                r->info.status = s1;
                failed.push_back(r);
            } else {
                keep.push_back(r);
            }
        }
        good.swap(keep);
    }
    for (auto &r : good) {  // could not be appended (cannot happen for valid requests)
        r->info.status = LV_ERR_ARG;
        failed.push_back(r);
    }
    return LV_OK;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// completion under S->mu: the request leaves the budget and its waiters wake
void complete_locked(lv_server *S, Request &r, double t) {
    r.done = true;
    r.info.t_done_ms = t;
    S->resident_bytes -= r.est;
    S->resident_n -= r.n;
    S->resident_a -= (int64_t)r.col.size();
    --S->inflight;
    if (r.info.status == LV_OK) ++S->stats.completed;
    else ++S->stats.failed;
}

// lane 1 takes large requests, those that would colour a phase, and every
// request when recursive vertex following is on (single-graph runs only)
bool plain_lane(const lv_server *S, const Request &r) {
    return (int64_t)r.col.size() >= kLaneSplitArcs ||
           (S->cfg.params.coloring && r.n >= S->cfg.params.color_cutoff) ||
           S->cfg.params.vf_recursive;
}

// Lane 1: one request at a time through the single-graph entry points.
void plain_worker_main(lv_server *S, int wi) {
    cudaSetDevice(S->device);
    lv_server::Lane &L = S->lanes[1];
    cudaStream_t stream = S->plain_streams[wi];
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            L.cv_work.wait(lk, [&] { return S->stop || !L.plain.empty(); });
            if (S->stop) break;
            r = L.plain.front();
            L.plain.pop_front();
        }
        const Clock::time_point c0 = Clock::now();
        lv_graph *h = nullptr;
        lv_status st = rowptr_ok(*r) ? lv_graph_create(&h, r->n, r->rowptr.data(), r->col.data(),
                                                       r->w.data(), 0, stream)
                                     : LV_ERR_ARG;
        lv_params prm = S->cfg.params;
        const int half = std::max(1, g_num_sms / 2);
        prm.persistent_sms = prm.persistent_sms > 0 ? std::min(prm.persistent_sms, half) : half;
        if (st == LV_OK) st = lv_run(h, &prm);
        if (st == LV_OK) {
            r->labels.resize((size_t)r->n);
            st = lv_get_labels(h, -1, r->labels.data(), 0);
        }
        int32_t np = 0;
        if (st == LV_OK) st = lv_num_phases(h, &np);
        if (st == LV_OK) {
            r->info.num_phases = np;
            r->info.iterations = 0;
            for (int32_t p = 0; p < np && st == LV_OK; ++p) {
                lv_phase_info in;
                st = lv_get_phase_info(h, p, &in);
                r->info.iterations += in.iterations;
                if (p == np - 1) {
                    r->info.n_final = in.n_next;
                    r->info.N_final = in.N_end;
                    r->info.q = in.q;
                    r->info.two_m = in.two_m;
                }
            }
            lv_stats ls;
            if (st == LV_OK && lv_get_stats(h, &ls) == LV_OK) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->stats.kernel_launches += ls.kernel_launches;
                S->stats.sweeps += ls.sweep_launches;
            }
        }
        lv_graph_destroy(h);
        const Clock::time_point c1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->info.status = st;
            ++L.rounds;
            S->stats.rounds = S->lanes[0].rounds + S->lanes[1].rounds;
            S->stats.ms_iterate += ms_between(c0, c1);
            complete_locked(S, *r, S->now_ms());
        }
        S->cv_done.notify_all();
        S->cv_adm.notify_all();
    }
}

// Admission thread: takes queued requests first come first served while the
// budget, the slots and int32 ids allow, then uploads, validates and
// vertex-follows them on its own stream, so this work overlaps the worker's
// phases; the result joins the engine at the worker's next phase boundary.
void admitter_main(lv_server *S) {
    cudaSetDevice(S->device);
    const Ctx c{S->adm_stream, S->adm_pinned, &S->cfg.params, &S->ring};
    const int64_t budget = S->cfg.mem_budget_bytes > 0 ? S->cfg.mem_budget_bytes : kDefaultBudget;
    const int64_t maxg = S->cfg.max_graphs > 0 ? S->cfg.max_graphs : kDefaultMaxGraphs;
    for (;;) {
        std::vector<std::shared_ptr<Request>> adm;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto admissible = [&] {
                if (S->queue.empty()) return false;
                const Request &r = *S->queue.front();
                if (S->inflight >= maxg) return false;
                if (S->inflight > 0 && S->resident_bytes + r.est > budget) return false;
                return S->resident_n + r.n <= 0x7ffffffell &&
                       S->resident_a + (int64_t)r.col.size() <= 0x7fffffffll;
            };
            S->cv_adm.wait(lk, [&] { return S->stop || admissible(); });
            if (S->stop) break;
            while (admissible()) {
                std::shared_ptr<Request> r = S->queue.front();
                S->queue.pop_front();
                S->resident_bytes += r->est;
                S->resident_n += r->n;
                S->resident_a += (int64_t)r->col.size();
                ++S->inflight;
                adm.push_back(r);
            }
            const double t = S->now_ms();
            for (auto &r : adm) r->info.t_admit_ms = t;
            S->stats.admitted += (int64_t)adm.size();
        }
        {
            std::vector<std::shared_ptr<Request>> to_plain;
            for (auto &r : adm)
                if (plain_lane(S, *r)) to_plain.push_back(r);
            if (!to_plain.empty()) {
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto &r : to_plain) S->lanes[1].plain.push_back(r);
            }
            if (!to_plain.empty()) S->lanes[1].cv_work.notify_all();
        }
        do {  // the rest joins lane 0's engine
            const int ln = 0;
            std::vector<std::shared_ptr<Request>> group;
            for (auto &r : adm)
                if (!plain_lane(S, *r)) group.push_back(r);
            if (group.empty()) break;
            const Clock::time_point c0 = Clock::now();
            std::vector<std::shared_ptr<Request>> failed, joined;
            std::unique_ptr<Prepared> pr;
            const lv_status st = admit(c, group, failed, &pr, &joined);
            const Clock::time_point c1 = Clock::now();
            {
                std::lock_guard<std::mutex> lk(S->mu);
                const double t = S->now_ms();
                S->stats.ms_admit += ms_between(c0, c1);
                if (st != LV_OK) {  // a device failure ends the whole admitted group
                    for (auto &r : group) {
                        if (r->done) continue;
                        if (r->info.status == LV_OK) r->info.status = st;
                        complete_locked(S, *r, t);
                    }
                } else {
                    for (auto &r : failed) complete_locked(S, *r, t);
                    if (pr && !joined.empty()) {
                        Ready rd;
                        rd.pr = std::move(pr);
                        rd.reqs = joined;
                        S->lanes[ln].ready.push_back(std::move(rd));
                    }
                }
            }
            S->lanes[ln].cv_work.notify_all();
            S->cv_done.notify_all();
            S->cv_adm.notify_all();
        } while (false);
    }
}

// Worker thread: appends what the admission thread prepared, runs one
// batched phase of every resident request and completes those that finish.
void worker_main(lv_server *S, int ln) {
    cudaSetDevice(S->device);
    lv_server::Lane &L = S->lanes[ln];
    Engine e;
    e.s = L.stream;
    e.P = S->cfg.params;
    e.lim = S->lim;
    e.pinned = L.pinned;
    std::unordered_map<int64_t, std::shared_ptr<Request>> resident;
    for (;;) {
        std::vector<Ready> take;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            L.cv_work.wait(lk, [&] { return S->stop || !L.ready.empty() || e.num_graphs() > 0; });
            if (S->stop) break;
            while (!L.ready.empty()) {
                take.push_back(std::move(L.ready.front()));
                L.ready.pop_front();
            }
        }
        const unsigned long long launches0 = g_kernel_launches.load();
        lv_status st = LV_OK;
        const Clock::time_point c0 = Clock::now();
        std::vector<std::shared_ptr<Request>> lost;  // taken but not appended
        if (!take.empty()) {  // everything prepared since the last boundary joins in one copy
            std::vector<const Prepared *> prs;
            for (auto &rd : take) prs.push_back(rd.pr.get());
            st = e.append_prepared(prs);
            for (auto &rd : take) {
                for (auto &r : rd.reqs) {
                    if (st == LV_OK) resident[r->id] = r;
                    else lost.push_back(r);
                }
                rd.pr.reset();
            }
        }
        const Clock::time_point c1 = Clock::now();
        Clock::time_point c2 = c1, c3 = c1, c4 = c1;
        std::vector<Finished> fin;
        if (st == LV_OK && e.num_graphs() > 0) {
            st = e.phase_run();
            c2 = Clock::now();
            if (st == LV_OK) st = e.phase_end(fin);
            c3 = Clock::now();
            for (auto &f : fin) {  // labels of the requests that finished
                auto it = resident.find(f.rec.tag);
                if (it == resident.end()) continue;
                Request &r = *it->second;
                r.labels.resize((size_t)r.n);
                if (st == LV_OK &&
                    cudaMemcpyAsync(r.labels.data(), e.labels + f.lab_off, sizeof(int32_t) * (size_t)r.n,
                                    cudaMemcpyDeviceToHost, L.stream) != cudaSuccess)
                    st = LV_ERR_CUDA;
                r.info.num_phases = (int32_t)f.rec.info.size();
                r.info.iterations = 0;
                for (const auto &in : f.rec.info) r.info.iterations += in.iterations;
                if (!f.rec.info.empty()) {
                    r.info.n_final = f.rec.info.back().n_next;
                    r.info.N_final = f.rec.info.back().N_end;
                    r.info.q = f.rec.info.back().q;
                }
            }
            if (st == LV_OK && cudaStreamSynchronize(L.stream) != cudaSuccess) st = LV_ERR_CUDA;
            c4 = Clock::now();
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double t = S->now_ms();
            for (auto &r : lost) {
                r->info.status = st;
                complete_locked(S, *r, t);
            }
            if (st != LV_OK) {
                // a device failure ends every resident request with its status
                for (auto &kv : resident) {
                    kv.second->info.status = st;
                    complete_locked(S, *kv.second, t);
                }
                resident.clear();
                e.release();
            } else {
                for (auto &f : fin) {
                    auto it = resident.find(f.rec.tag);
                    if (it == resident.end()) continue;
                    complete_locked(S, *it->second, t);
                    resident.erase(it);
                }
            }
            if (!fin.empty() || e.num_graphs() > 0) ++L.rounds;
            S->stats.sweeps += e.sweep_launches - L.sweeps;
            L.sweeps = e.sweep_launches;
            S->stats.rounds = S->lanes[0].rounds + S->lanes[1].rounds;
            S->stats.peak_graphs = std::max<int64_t>(S->stats.peak_graphs, (int64_t)resident.size());
            S->stats.peak_bytes = std::max<int64_t>(S->stats.peak_bytes, S->resident_bytes);
            S->stats.kernel_launches += (int64_t)(g_kernel_launches.load() - launches0);
            S->stats.ms_append += ms_between(c0, c1);
            S->stats.ms_iterate += ms_between(c1, c2);
            S->stats.ms_rebuild += ms_between(c2, c3);
            S->stats.ms_results += ms_between(c3, c4);
        }
        S->cv_done.notify_all();
        S->cv_adm.notify_all();
    }
    e.release();
}

}  // namespace

extern "C" {

lv_status lv_server_create(lv_server **out, const lv_server_config *cfg, void *cuda_stream) {
    if (!out) return LV_ERR_ARG;
    *out = nullptr;
    if (!cfg) return LV_ERR_ARG;
    const lv_params &P = cfg->params;
    BinLimits lim;
    if (P.bin_lane_arcs) lim.lane_arcs = P.bin_lane_arcs;
    if (P.bin_warp_max) lim.warp_max = P.bin_warp_max;
    if (P.bin_cta_max) lim.cta_max = P.bin_cta_max;
    lim.blocks_per_sm = P.sweep_blocks_per_sm;
    lim.hub_factor = P.hub_slots_per_arc;
    lim.sms = P.persistent_sms;
    if (lim.lane_arcs < 1 || lim.lane_arcs > kLaneArcsLimit || lim.warp_max < 1 ||
        lim.warp_max > kWarpMaxLimit || lim.cta_max <= lim.warp_max || lim.cta_max > kCtaMaxLimit ||
        !valid_shape(lim) ||
        P.max_iters < 1 || P.max_phases < 1 || !(P.theta_low >= -1e300) || cfg->max_graphs < 0 ||
        cfg->mem_budget_bytes < 0)
        return LV_ERR_ARG;
    lv_server *S = new lv_server();
    S->cfg = *cfg;
    S->lim = lim;
    S->t0 = Clock::now();
    std::memset(&S->stats, 0, sizeof S->stats);
    cudaGetDevice(&S->device);
    lv_status st = LV_OK;
    for (int ln = 0; ln < 2 && st == LV_OK; ++ln) {
        lv_server::Lane &L = S->lanes[ln];
        L.stream = ln == 0 ? (cudaStream_t)cuda_stream : nullptr;
        if (!L.stream) {
            if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess) st = LV_ERR_CUDA;
            else L.own_stream = true;
        }
        if (st == LV_OK && cudaMallocHost((void **)&L.pinned, 64 * sizeof(int)) != cudaSuccess)
            st = LV_ERR_OOM;
    }
    S->plain_streams[0] = S->lanes[1].stream;
    for (int i = 1; i < kPlainWorkers && st == LV_OK; ++i)
        if (cudaStreamCreateWithFlags(&S->plain_streams[i], cudaStreamNonBlocking) != cudaSuccess)
            st = LV_ERR_CUDA;
    if (st == LV_OK) st = ensure_setup(S->lanes[0].stream);
    if (st == LV_OK && cudaMallocHost((void **)&S->adm_pinned, 64 * sizeof(int)) != cudaSuccess)
        st = LV_ERR_OOM;
    if (st == LV_OK && cudaStreamCreateWithFlags(&S->adm_stream, cudaStreamNonBlocking) != cudaSuccess)
        st = LV_ERR_CUDA;
    if (st == LV_OK) st = S->ring.init();
    if (st != LV_OK) {
        S->ring.destroy();
        for (auto &L : S->lanes) {
            if (L.pinned) cudaFreeHost(L.pinned);
            if (L.own_stream) cudaStreamDestroy(L.stream);
        }
        for (int i = 1; i < kPlainWorkers; ++i)
            if (S->plain_streams[i]) cudaStreamDestroy(S->plain_streams[i]);
        if (S->adm_pinned) cudaFreeHost(S->adm_pinned);
        if (S->adm_stream) cudaStreamDestroy(S->adm_stream);
        delete S;
        return st;
    }
    S->lanes[0].worker = std::thread(worker_main, S, 0);
    for (int i = 0; i < kPlainWorkers; ++i) S->plain_workers[i] = std::thread(plain_worker_main, S, i);
    S->admitter = std::thread(admitter_main, S);
    *out = S;
    return LV_OK;
}

lv_status lv_server_submit(lv_server *S, int64_t n, const int64_t *rowptr, const int32_t *col,
                           const int32_t *w, int64_t *request_id) {
    if (!S || !rowptr || !request_id || n < 0 || n > 0x7ffffffell) return LV_ERR_ARG;
    const int64_t A = rowptr[n];
    if (A < 0 || A > 0x7fffffffll || (A > 0 && (!col || !w))) return LV_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->n = n;
    r->rowptr.assign(rowptr, rowptr + n + 1);
    r->col.assign(col, col + A);
    r->w.assign(w, w + A);
    r->est = kBytesPerArc * A + kBytesPerVertex * n;
    std::memset(&r->info, 0, sizeof r->info);
    r->info.n = n;
    r->info.arcs = A;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->info.t_submit_ms = S->now_ms();
        S->reqs[r->id] = r;
        S->queue.push_back(r);
        ++S->stats.submitted;
        *request_id = r->id;
    }
    S->cv_adm.notify_one();
    return LV_OK;
}

lv_status lv_server_wait(lv_server *S, int64_t id, double timeout_s, int32_t *done) {
    if (!S || !done) return LV_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LV_ERR_ARG;
    std::shared_ptr<Request> r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s < 0) S->cv_done.wait(lk, pred);
    else S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
    *done = r->done ? 1 : 0;
    return LV_OK;
}

lv_status lv_server_result(lv_server *S, int64_t id, int32_t *labels, lv_server_result_info *info) {
    if (!S) return LV_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LV_ERR_ARG;
    const Request &r = *it->second;
    if (!r.done) return LV_ERR_STATE;
    if (info) *info = r.info;
    if (r.info.status != LV_OK) return (lv_status)r.info.status;
    if (labels && r.n > 0) std::memcpy(labels, r.labels.data(), sizeof(int32_t) * (size_t)r.n);
    return LV_OK;
}

lv_status lv_server_release(lv_server *S, int64_t id) {
    if (!S) return LV_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return LV_ERR_ARG;
    if (!it->second->done) return LV_ERR_STATE;
    S->reqs.erase(it);
    return LV_OK;
}

lv_status lv_server_get_stats(lv_server *S, lv_server_stats *out) {
    if (!S || !out) return LV_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return LV_OK;
}

void lv_server_destroy(lv_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    for (auto &L : S->lanes) L.cv_work.notify_all();
    S->cv_adm.notify_all();
    if (S->admitter.joinable()) S->admitter.join();
    for (auto &L : S->lanes)
        if (L.worker.joinable()) L.worker.join();
    for (auto &t : S->plain_workers)
        if (t.joinable()) t.join();
    for (auto &L : S->lanes) {
        L.ready.clear();  // prepared graphs never appended
        L.plain.clear();
    }
    cudaStreamSynchronize(S->adm_stream);
    S->ring.destroy();
    for (int i = 1; i < kPlainWorkers; ++i) {
        cudaStreamSynchronize(S->plain_streams[i]);
        cudaStreamDestroy(S->plain_streams[i]);
    }
    for (auto &L : S->lanes) {
        cudaStreamSynchronize(L.stream);
        if (L.pinned) cudaFreeHost(L.pinned);
        if (L.own_stream) cudaStreamDestroy(L.stream);
    }
    if (S->adm_pinned) cudaFreeHost(S->adm_pinned);
    cudaStreamDestroy(S->adm_stream);
    delete S;
}

}  // extern "C"
