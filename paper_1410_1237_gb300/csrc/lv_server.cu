// lv_server.cu -- serving with continuous batching (lv.h, "serving").
//
// Requests are queued by lv_server_submit (host copies of their CSRs).  One
// worker thread owns the device work and loops over rounds:
//   1. admission: queued requests, first come first served, while the
//      resident requests' estimated footprint stays within the budget and
//      the slot limit; the admitted CSRs are concatenated into one union,
//      validated on the device and appended to the engine (vertex following
//      included), so they join the requests already running;
//   2. one batched phase of every resident request (lv_engine.cu);
//   3. requests whose phase loop stopped leave the engine: their labels are
//      copied to the host and their waiters are woken.
// Every request is computed exactly as lv_run computes it alone, so results
// do not depend on what else is resident.
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

}  // namespace

struct lv_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lv_server_config cfg;
    BinLimits lim;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;  // until released
    int64_t next_id = 0;
    bool stop = false;
    lv_server_stats stats;
    int64_t resident_bytes = 0;
    int64_t resident_n = 0, resident_a = 0;  // input vertices and arcs of resident requests
    int *pinned = nullptr;
    std::thread worker;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

namespace {

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

lv_status stage(lv_server *S, int64_t n, const int64_t *rowptr, const int32_t *col, const int32_t *w,
                bool limit_two_m, Staged *out) {
    cudaStream_t s = S->stream;
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
                                S->pinned, s, limit_two_m);
    dfree(d_rp, s);
    dfree(d_col, s);
    dfree(d_w, s);
    return st;
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
lv_status admit(lv_server *S, Engine &e, std::vector<std::shared_ptr<Request>> &adm,
                std::vector<std::shared_ptr<Request>> &failed) {
    cudaStream_t s = S->stream;
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
        // host union: columns shifted by each request's vertex start
        int64_t n = 0, A = 0;
        for (auto &r : good) {
            n += r->n;
            A += (int64_t)r->col.size();
        }
        if (n > 0x7ffffffell || A > 0x7fffffffll) return LV_ERR_OVERFLOW;  // admission keeps below
        std::vector<int64_t> rp((size_t)n + 1);
        std::vector<int32_t> col((size_t)A), w((size_t)A);
        std::vector<int32_t> gptr(good.size() + 1, 0);
        int64_t v0 = 0, a0 = 0;
        for (size_t q = 0; q < good.size(); ++q) {
            const Request &r = *good[q];
            for (int64_t i = 0; i < r.n; ++i) rp[v0 + i] = r.rowptr[i] + a0;
            for (size_t e2 = 0; e2 < r.col.size(); ++e2) {
                col[a0 + e2] = (int32_t)(r.col[e2] + v0);
                w[a0 + e2] = r.w[e2];
            }
            v0 += r.n;
            a0 += (int64_t)r.col.size();
            gptr[q + 1] = (int32_t)v0;
        }
        rp[n] = A;
        Staged U;
        lv_status st = stage(S, n, rp.data(), col.data(), w.data(), false, &U);
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
            LV_TRY(e.append(ng));
            for (size_t q = 0; q < good.size(); ++q) good[q]->info.two_m = two_m[q];
            return LV_OK;
        }
        // the union failed: find the invalid requests one by one
        std::vector<std::shared_ptr<Request>> keep;
        for (auto &r : good) {
            Staged one;
            const lv_status s1 = stage(S, r->n, r->rowptr.data(), r->col.data(), r->w.data(), true, &one);
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

void worker_main(lv_server *S) {
    cudaSetDevice(S->device);
    Engine e;
    e.s = S->stream;
    e.P = S->cfg.params;
    e.lim = S->lim;
    e.pinned = S->pinned;
    std::unordered_map<int64_t, std::shared_ptr<Request>> resident;
    for (;;) {
        std::vector<std::shared_ptr<Request>> adm;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || e.num_graphs() > 0; });
            if (S->stop) break;
            const int64_t budget =
                S->cfg.mem_budget_bytes > 0 ? S->cfg.mem_budget_bytes : kDefaultBudget;
            const int64_t maxg = S->cfg.max_graphs > 0 ? S->cfg.max_graphs : kDefaultMaxGraphs;
            int64_t adm_n = 0, adm_a = 0;  // the admitted union must fit int32 ids
            while (!S->queue.empty()) {
                const std::shared_ptr<Request> &r = S->queue.front();
                const int64_t cnt = (int64_t)resident.size() + (int64_t)adm.size();
                if (cnt >= maxg) break;
                if (cnt > 0 && S->resident_bytes + r->est > budget) break;
                const int64_t ra = (int64_t)r->col.size();
                if (S->resident_n + adm_n + r->n > 0x7ffffffell ||
                    S->resident_a + adm_a + ra > 0x7fffffffll)
                    break;
                S->resident_bytes += r->est;
                adm_n += r->n;
                adm_a += ra;
                adm.push_back(r);
                S->queue.pop_front();
            }
            S->resident_n += adm_n;
            S->resident_a += adm_a;
            const double t = S->now_ms();
            for (auto &r : adm) r->info.t_admit_ms = t;
            S->stats.admitted += (int64_t)adm.size();
        }
        std::vector<std::shared_ptr<Request>> failed;
        lv_status st = LV_OK;
        if (!adm.empty()) {
            st = admit(S, e, adm, failed);
            for (auto &r : adm)
                if (r->info.status == LV_OK) resident[r->id] = r;
        }
        std::vector<Finished> fin;
        if (st == LV_OK && e.num_graphs() > 0) {
            st = e.phase_run();
            if (st == LV_OK) st = e.phase_end(fin);
            for (auto &f : fin) {  // labels of the requests that finished
                auto it = resident.find(f.rec.tag);
                if (it == resident.end()) continue;
                Request &r = *it->second;
                r.labels.resize((size_t)r.n);
                if (st == LV_OK &&
                    cudaMemcpyAsync(r.labels.data(), e.labels + f.lab_off, sizeof(int32_t) * (size_t)r.n,
                                    cudaMemcpyDeviceToHost, S->stream) != cudaSuccess)
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
            if (st == LV_OK && cudaStreamSynchronize(S->stream) != cudaSuccess) st = LV_ERR_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double t = S->now_ms();
            auto complete = [&](Request &r) {
                r.done = true;
                r.info.t_done_ms = t;
                S->resident_bytes -= r.est;
                S->resident_n -= r.n;
                S->resident_a -= (int64_t)r.col.size();
                if (r.info.status == LV_OK) ++S->stats.completed;
                else ++S->stats.failed;
            };
            for (auto &r : failed) complete(*r);
            if (st != LV_OK) {
                // a device failure ends every resident request with its status
                for (auto &kv : resident) {
                    kv.second->info.status = st;
                    complete(*kv.second);
                }
                resident.clear();
                e.release();
            } else {
                for (auto &f : fin) {
                    auto it = resident.find(f.rec.tag);
                    if (it == resident.end()) continue;
                    complete(*it->second);
                    resident.erase(it);
                }
            }
            if (!fin.empty() || e.num_graphs() > 0) ++S->stats.rounds;
            S->stats.sweeps = e.sweep_launches;
            S->stats.peak_graphs = std::max<int64_t>(S->stats.peak_graphs, (int64_t)resident.size());
            S->stats.peak_bytes = std::max<int64_t>(S->stats.peak_bytes, S->resident_bytes);
        }
        S->cv_done.notify_all();
    }
    e.release();
}

}  // namespace

extern "C" {

lv_status lv_server_create(lv_server **out, const lv_server_config *cfg, void *cuda_stream) {
    if (!out) return LV_ERR_ARG;
    *out = nullptr;
    if (!cfg || cfg->params.coloring) return LV_ERR_ARG;
    const lv_params &P = cfg->params;
    BinLimits lim;
    if (P.bin_lane_arcs) lim.lane_arcs = P.bin_lane_arcs;
    if (P.bin_warp_max) lim.warp_max = P.bin_warp_max;
    if (P.bin_cta_max) lim.cta_max = P.bin_cta_max;
    if (lim.lane_arcs < 1 || lim.lane_arcs > kLaneArcsLimit || lim.warp_max < 1 ||
        lim.warp_max > kWarpMaxLimit || lim.cta_max <= lim.warp_max || lim.cta_max > kCtaMaxLimit ||
        P.max_iters < 1 || P.max_phases < 1 || !(P.theta_low >= -1e300) || cfg->max_graphs < 0 ||
        cfg->mem_budget_bytes < 0)
        return LV_ERR_ARG;
    lv_server *S = new lv_server();
    S->cfg = *cfg;
    S->lim = lim;
    S->t0 = Clock::now();
    std::memset(&S->stats, 0, sizeof S->stats);
    cudaGetDevice(&S->device);
    S->stream = (cudaStream_t)cuda_stream;
    if (!S->stream) {
        if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete S;
            return LV_ERR_CUDA;
        }
        S->own_stream = true;
    }
    lv_status st = ensure_setup(S->stream);
    if (st == LV_OK && cudaMallocHost((void **)&S->pinned, 64 * sizeof(int)) != cudaSuccess)
        st = LV_ERR_OOM;
    if (st != LV_OK) {
        if (S->own_stream) cudaStreamDestroy(S->stream);
        delete S;
        return st;
    }
    S->worker = std::thread(worker_main, S);
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
    S->cv_work.notify_one();
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
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaStreamSynchronize(S->stream);
    if (S->pinned) cudaFreeHost(S->pinned);
    if (S->own_stream) cudaStreamDestroy(S->stream);
    delete S;
}

}  // extern "C"
