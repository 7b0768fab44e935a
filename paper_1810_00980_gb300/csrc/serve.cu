// Serving loop: resident graphs, a thread-safe ticket queue, and n_streams
// scheduler threads that each form a batch from whatever is queued (same
// graph, admitted while its estimated scratch footprint fits the budget),
// run it on their own stream with run_batch, and publish the results.  While
// one batch is on the GPU the other schedulers admit newly arrived queries,
// so batches overlap on the device (continuous batching).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tm_internal.cuh"

namespace {

enum TicketState { kQueued = 0, kRunning = 1, kDone = 2 };

struct Ticket {
    int32_t gid = 0;
    tm_query q{};
    int state = kQueued;
    int status = TM_PENDING;
    int64_t footprint = 0;
    uint64_t cls = 0;     // query class (graph, motif, delta, mode, c, p, b, q rule)
    double pred = 0.0;    // predicted work (first edges + candidates read)
    tm_result r{};
};

uint64_t class_key(int32_t gid, const tm_query& q) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    auto mixin = [&](uint64_t v) { h = tmo::sm64_mix(h ^ (v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2))); };
    mixin((uint64_t)gid);
    mixin((uint64_t)(uintptr_t)q.motif);
    mixin((uint64_t)q.delta);
    mixin((uint64_t)q.mode);
    if (q.mode == TM_MODE_ESTIMATE) {
        mixin((uint64_t)q.c);
        mixin((uint64_t)(int64_t)(q.p * 1e6));
        mixin((uint64_t)q.b);
        mixin((uint64_t)q.q_mode);
    }
    return h;
}

}  // namespace

struct tm_server {
    tm_serve_cfg cfg{};
    int device = 0;
    std::vector<const tm_graph*> graphs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::deque<uint64_t> done_q;     // finished tickets in completion order (for wait_any)
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<std::thread> workers;
    int64_t in_use = 0;
    bool stopping = false;
    uint64_t next_id = 1;
    std::unordered_map<uint64_t, double> work_ema;   // learned work per query class
};

namespace {

constexpr double kWorkFloor = 2e8;   // predicted work always admitted into one batch

// Upper estimate of the scratch a query needs inside run_batch.
int64_t footprint(const tm_graph* g, const tm_query& q) {
    int64_t per_first = 4 + 8 + 8 + 8;
    int64_t per_win = 8 * 7 + 4 * 3 + 8 + 8 * 7;
    if (q.mode != TM_MODE_ESTIMATE) return g->m * per_first + per_win + 4096;
    int64_t cd = (int64_t)q.c * q.delta;
    if (cd <= 0) return 4096;
    int64_t J = 1 + (g->t_max + cd - 1) / cd;
    double frac = q.q_mode == TM_Q_UNIFORM ? q.p : 1.0;
    double first = (double)q.b * (double)g->m * std::min(1.0, 2.0 * frac + 1.0 / (double)J);
    int64_t wt = q.delta + 1 <= ((int64_t)1 << 22) ? 16 * (q.delta + 1) : 0;
    return (int64_t)first * per_first + (int64_t)q.b * J * per_win + wt + 4096;
}

void worker_main(tm_server* S) {
    cudaSetDevice(S->device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    std::vector<uint64_t> ids;
    std::vector<tm_query> qs;
    std::vector<tm_result> rs;
    for (;;) {
        int32_t gid = -1;
        int64_t fp_total = 0;
        double work = 0.0, budget = 0.0;
        ids.clear();
        qs.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (!S->queue.empty()) {
                    // admit in arrival order: the oldest query's graph, while memory fits
                    for (auto it = S->queue.begin(); it != S->queue.end() && (int)ids.size() < S->cfg.max_batch;) {
                        Ticket& T = S->tickets[*it];
                        if (gid >= 0 && T.gid != gid) { ++it; continue; }
                        if (T.footprint > S->cfg.mem_budget_bytes) {
                            T.state = kDone;
                            T.status = TM_EADMIT;
                            std::memset(&T.r, 0, sizeof(T.r));
                            T.r.status = TM_EADMIT;
                            S->done_q.push_back(*it);
                            it = S->queue.erase(it);
                            S->cv_done.notify_all();
                            continue;
                        }
                        if (S->in_use + fp_total + T.footprint > S->cfg.mem_budget_bytes) break;
                        // the oldest query always goes; later ones join while the batch's
                        // predicted work stays within twice the oldest's (and a floor), so a
                        // heavy query does not hold many light ones back
                        if (!ids.empty() && work + T.pred > budget) { ++it; continue; }
                        if (ids.empty()) budget = std::max(2.0 * T.pred, kWorkFloor);
                        work += T.pred;
                        gid = T.gid;
                        fp_total += T.footprint;
                        T.state = kRunning;
                        ids.push_back(*it);
                        qs.push_back(T.q);
                        it = S->queue.erase(it);
                    }
                    if (!ids.empty()) break;
                }
                if (S->stopping && S->queue.empty()) break;
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
            if (ids.empty()) break;  // stopping and drained
            S->in_use += fp_total;
        }
        rs.assign(qs.size(), tm_result{});
        int rc = tmo::run_batch(S->graphs[(size_t)gid], qs.data(), (int)qs.size(), rs.data(), st, nullptr);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= fp_total;
            for (size_t i = 0; i < ids.size(); i++) {
                auto it = S->tickets.find(ids[i]);
                if (it == S->tickets.end()) continue;
                Ticket& T = it->second;
                T.state = kDone;
                T.r = rs[i];
                if (rs[i].status == TM_OK) {
                    double w = (double)rs[i].first_edges + (double)rs[i].cand_edges + (double)rs[i].inst_read;
                    auto e = S->work_ema.find(T.cls);
                    if (e == S->work_ema.end()) S->work_ema.emplace(T.cls, w);
                    else e->second = 0.5 * e->second + 0.5 * w;
                }
                if (rc != TM_OK && rs[i].status == TM_OK && rc != TM_EINVAL && rc != TM_EOVERFLOW) {
                    T.r.status = rc;  // batch-level failure (CUDA, memory)
                }
                T.status = T.r.status;
                S->done_q.push_back(ids[i]);
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    if (st) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
}

}  // namespace

extern "C" {

int tm_serve_create(const tm_serve_cfg* cfg, tm_server** out) {
    if (!out) { tmo::set_error("out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    tm_server* S = new (std::nothrow) tm_server();
    if (!S) { tmo::set_error("host allocation failed"); return TM_ENOMEM; }
    if (cfg) S->cfg = *cfg;
    if (S->cfg.mem_budget_bytes <= 0) S->cfg.mem_budget_bytes = (int64_t)4 << 30;
    if (S->cfg.max_batch <= 0) S->cfg.max_batch = 256;
    if (S->cfg.n_streams <= 0) S->cfg.n_streams = 2;
    if (S->cfg.n_streams > 4) S->cfg.n_streams = 4;
    cudaGetDevice(&S->device);
    try {
        for (int i = 0; i < S->cfg.n_streams; i++) S->workers.emplace_back(worker_main, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stopping = true;
        }
        S->cv_work.notify_all();
        for (auto& t : S->workers) t.join();
        delete S;
        tmo::set_error("could not start scheduler threads");
        return TM_ENOMEM;
    }
    *out = S;
    return TM_OK;
}

int tm_serve_attach_graph(tm_server* S, const tm_graph* g, int32_t* graph_id) {
    if (!S || !g || !graph_id) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    S->graphs.push_back(g);
    *graph_id = (int32_t)S->graphs.size() - 1;
    return TM_OK;
}

int tm_serve_submit(tm_server* S, int32_t graph_id, const tm_query* q, uint64_t* ticket) {
    if (!S || !q || !ticket || !q->motif) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) { tmo::set_error("server is shutting down"); return TM_ESHUTDOWN; }
    if (graph_id < 0 || graph_id >= (int32_t)S->graphs.size()) { tmo::set_error("unknown graph id"); return TM_ENOTFOUND; }
    uint64_t id = S->next_id++;
    Ticket T;
    T.gid = graph_id;
    T.q = *q;
    T.footprint = footprint(S->graphs[(size_t)graph_id], *q);
    T.cls = class_key(graph_id, *q);
    auto e = S->work_ema.find(T.cls);
    // unseen classes are assumed heavy (four reads per edge of the graph) until measured
    T.pred = e != S->work_ema.end() ? e->second : 4.0 * (double)S->graphs[(size_t)graph_id]->m;
    S->tickets.emplace(id, T);
    S->queue.push_back(id);
    *ticket = id;
    S->cv_work.notify_one();
    return TM_OK;
}

int tm_serve_poll(tm_server* S, uint64_t ticket, tm_result* r) {
    if (!S || !r) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return TM_ENOTFOUND;
    if (it->second.state != kDone) return TM_PENDING;
    *r = it->second.r;
    int s = it->second.status;
    S->tickets.erase(it);
    return s;
}

int tm_serve_wait(tm_server* S, uint64_t ticket, int64_t timeout_ms, tm_result* r) {
    if (!S || !r) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return TM_ENOTFOUND;
        if (it->second.state == kDone) {
            *r = it->second.r;
            int s = it->second.status;
            S->tickets.erase(it);
            return s;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = S->tickets.find(ticket);
            if (it2 != S->tickets.end() && it2->second.state == kDone) continue;
            return TM_ETIMEOUT;
        }
    }
}

int tm_serve_wait_any(tm_server* S, int64_t timeout_ms, uint64_t* ticket, tm_result* r) {
    if (!S || !ticket || !r) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        while (!S->done_q.empty()) {
            uint64_t id = S->done_q.front();
            S->done_q.pop_front();
            auto it = S->tickets.find(id);
            if (it == S->tickets.end() || it->second.state != kDone) continue;  // already collected
            *ticket = id;
            *r = it->second.r;
            int st = it->second.status;
            S->tickets.erase(it);
            return st;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->done_q.empty())
            return TM_ETIMEOUT;
    }
}

int tm_serve_cancel(tm_server* S, uint64_t ticket) {
    if (!S) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return TM_ENOTFOUND;
    if (it->second.state != kQueued) return TM_PENDING;  // already running or done
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
        if (*q == ticket) { S->queue.erase(q); break; }
    it->second.state = kDone;
    it->second.status = TM_ECANCELLED;
    std::memset(&it->second.r, 0, sizeof(tm_result));
    it->second.r.status = TM_ECANCELLED;
    S->done_q.push_back(ticket);
    S->cv_done.notify_all();
    return TM_OK;
}

void tm_serve_destroy(tm_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
}

}  // extern "C"
