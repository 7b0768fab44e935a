// C ABI entry points that are not graph loading or serving: errors, motif
// compilation, single queries, batches, tuning and the autotuner.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tm_internal.cuh"

namespace tmo {

namespace {
thread_local std::string g_last_error;

cudaStream_t thread_stream() {
    thread_local cudaStream_t s = nullptr;
    if (!s) {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    }
    return s;
}

std::mutex g_tune_mu;
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::atomic<int64_t> g_launches{0};
tm_profile g_prof{};
}  // namespace

bool profiling() { return g_prof_on.load(std::memory_order_relaxed); }

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void store_profile_batch(double windows_ms, double level2_ms, double match_ms, double fold_ms,
                         double batch_ms, int64_t match_items, int64_t first_edges, double sizing_ms,
                         double scan_ms, double ride_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.ride_ms = ride_ms;
    g_prof.sizing_ms = sizing_ms;
    g_prof.scan_ms = scan_ms;
    g_prof.windows_ms = windows_ms;
    g_prof.level2_ms = level2_ms;
    g_prof.match_ms = match_ms;
    g_prof.fold_ms = fold_ms;
    g_prof.batch_ms = batch_ms;
    g_prof.match_items = match_items;
    g_prof.first_edges = first_edges;
}

void store_profile_ride_records(int64_t n) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.ride_records = n;
}

void store_profile_graph(double graph_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.graph_ms = graph_ms;
}

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_status(cudaError_t e, const char* what, const char* file, int line) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                    std::to_string(line) + ")";
    set_error(m);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return TM_ENOMEM;
    }
    return TM_ECUDA;
}

}  // namespace tmo

using namespace tmo;

extern "C" {

const char* tm_strerror(int s) {
    switch (s) {
        case TM_OK: return "ok";
        case TM_EINVAL: return "invalid argument";
        case TM_EUNSORTED: return "timestamps not sorted";
        case TM_ERANGE: return "node id out of range";
        case TM_ENOMEM: return "out of memory";
        case TM_EADMIT: return "query can never be admitted";
        case TM_ETIMEOUT: return "timed out";
        case TM_ESTACK: return "matcher stack exhausted";
        case TM_EOVERFLOW: return "count overflow";
        case TM_ECUDA: return "CUDA error";
        case TM_PENDING: return "pending";
        case TM_ENOTFOUND: return "not found";
        case TM_ECANCELLED: return "cancelled";
        case TM_ESHUTDOWN: return "server shutting down";
        default: return "unknown status";
    }
}

const char* tm_last_error(void) { return g_last_error.c_str(); }

const char* tm_version(void) { return "libtmotif 0.1 sm_103a"; }

int tm_motif_compile(const int32_t* msrc, const int32_t* mdst, int32_t l, tm_motif** out) {
    if (!out) { set_error("out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    if (!msrc || !mdst) { set_error("NULL motif arrays"); return TM_EINVAL; }
    if (l < 1 || l > TM_L_MAX) { set_error("l outside [1, TM_L_MAX]"); return TM_EINVAL; }
    std::vector<int32_t> names;
    auto label = [&](int32_t x) {
        for (size_t i = 0; i < names.size(); i++)
            if (names[i] == x) return (int)i;
        names.push_back(x);
        return (int)names.size() - 1;
    };
    tm_motif m;
    std::memset(&m, 0, sizeof(m));
    m.l = l;
    int bound = 0;  // labels 0..bound-1 seen in earlier edges
    for (int i = 0; i < l; i++) {
        if (msrc[i] == mdst[i]) { set_error("motif self-loop"); return TM_EINVAL; }
        int a = label(msrc[i]);
        int b = label(mdst[i]);
        if ((int)names.size() > TM_K_MAX) { set_error("more than TM_K_MAX motif nodes"); return TM_EINVAL; }
        m.mu[i] = a;
        m.mv[i] = b;
        LevelPlan& P = m.lv[i];
        bool ub = a < bound, vb = b < bound;
        P.view = (ub && vb) ? kPair : ub ? kOut : vb ? kIn : kAll;
        P.su = (int8_t)a;
        P.sv = (int8_t)b;
        P.bind_u = ub ? 0 : 1;
        P.bind_v = vb ? 0 : 1;
        P.nb = (int8_t)bound;
        bound = (int)names.size();
    }
    m.k = (int)names.size();
    tm_motif* r = new (std::nothrow) tm_motif(m);
    if (!r) { set_error("host allocation failed"); return TM_ENOMEM; }
    *out = r;
    return TM_OK;
}

void tm_motif_free(tm_motif* m) { delete m; }

int tm_count_exact(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count) {
    if (!g || !m || !count) { set_error("NULL argument"); return TM_EINVAL; }
    tm_query q;
    std::memset(&q, 0, sizeof(q));
    q.motif = m;
    q.delta = delta;
    q.mode = TM_MODE_EXACT;
    tm_result r;
    int s = run_batch(g, &q, 1, &r, thread_stream(), nullptr);
    if (s != TM_OK) return s;
    *count = r.count;
    return TM_OK;
}

int tm_count_exact_plain(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count) {
    return count_plain(g, m, delta, count);
}

int tm_estimate(const tm_graph* g, const tm_motif* m, int64_t delta, int32_t c, double p,
                uint64_t seed, double* estimate) {
    if (!g || !m || !estimate) { set_error("NULL argument"); return TM_EINVAL; }
    tm_query q;
    std::memset(&q, 0, sizeof(q));
    q.motif = m;
    q.delta = delta;
    q.mode = TM_MODE_ESTIMATE;
    q.c = c;
    q.p = p;
    q.seed = seed;
    q.b = 1;
    q.q_mode = TM_Q_UNIFORM;
    tm_result r;
    int s = run_batch(g, &q, 1, &r, thread_stream(), nullptr);
    if (s != TM_OK) return s;
    *estimate = r.estimate;
    return TM_OK;
}

int tm_estimate_windows(const tm_graph* g, const tm_motif* m, int64_t delta, int32_t c, double p,
                        uint64_t seed, int32_t k, int32_t all_windows, tm_window_rec* out,
                        int64_t cap, int64_t* n_out, int64_t* shift) {
    if (!g || !m || !n_out || !shift || (cap > 0 && !out) || k < 0) { set_error("bad argument"); return TM_EINVAL; }
    tm_query q;
    std::memset(&q, 0, sizeof(q));
    q.motif = m;
    q.delta = delta;
    q.mode = TM_MODE_ESTIMATE;
    q.c = c;
    q.p = p;
    q.seed = seed;
    q.b = k + 1;
    q.q_mode = TM_Q_UNIFORM;
    tm_result r;
    BatchOut dbg;
    dbg.query = 0;
    dbg.k = k;
    dbg.all_windows = all_windows != 0;
    dbg.recs = out;
    dbg.cap = cap;
    int s = run_batch(g, &q, 1, &r, thread_stream(), &dbg);
    if (s != TM_OK) return s;
    *n_out = dbg.n_out;
    *shift = dbg.shift;
    return TM_OK;
}

int tm_run_batch(const tm_graph* g, const tm_query* queries, int32_t n_queries, tm_result* results,
                 void* stream) {
    return run_batch(g, queries, n_queries, results, (cudaStream_t)stream, nullptr);
}

int tm_get_tuning(tm_tuning* out) {
    if (!out) { set_error("NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const Tuning& t = tuning();
    out->block_threads = t.block_threads;
    out->blocks_per_sm = t.blocks_per_sm;
    out->chunk_items = t.chunk_items;
    out->enum_threshold = t.enum_threshold;
    return TM_OK;
}

int tm_set_tuning(const tm_tuning* in) {
    if (!in) { set_error("NULL argument"); return TM_EINVAL; }
    if (in->block_threads && (in->block_threads % 32 || in->block_threads < 32 || in->block_threads > 256)) {
        set_error("block_threads must be a multiple of 32 in [32, 256]");
        return TM_EINVAL;
    }
    if (in->blocks_per_sm < 0 || in->blocks_per_sm > 32) { set_error("blocks_per_sm outside [0, 32]"); return TM_EINVAL; }
    if (in->chunk_items && (in->chunk_items % 32 || in->chunk_items < 32)) {
        set_error("chunk_items must be a positive multiple of 32");
        return TM_EINVAL;
    }
    if (in->enum_threshold < 0) { set_error("enum_threshold < 0"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    Tuning& t = tuning();
    if (in->block_threads) t.block_threads = in->block_threads;
    if (in->blocks_per_sm) t.blocks_per_sm = in->blocks_per_sm;
    if (in->chunk_items) t.chunk_items = in->chunk_items;
    if (in->enum_threshold) t.enum_threshold = in->enum_threshold;
    return TM_OK;
}

int tm_autotune(const tm_graph* g, const tm_query* queries, int32_t n_queries, tm_tuning* best) {
    if (!g || !queries || n_queries <= 0 || !best) { set_error("bad argument"); return TM_EINVAL; }
    const int bts[] = {128, 256};
    const int bpss[] = {4, 6, 8, 12};
    const int chunks[] = {256, 1024, 4096};
    // the range threshold only matters for exact queries whose last edge has one bound
    // endpoint (two-edge motifs, or deeper ones closing on a node view)
    bool thr_matters = false;
    for (int i = 0; i < n_queries; i++) {
        const tm_motif* m = queries[i].motif;
        if (m && queries[i].mode == TM_MODE_EXACT && m->l >= 2 && m->lv[m->l - 1].view != kPair) thr_matters = true;
    }
    const int thr_all[] = {32, 128};
    const int n_thr = thr_matters ? 2 : 1;
    std::vector<tm_result> res((size_t)n_queries);
    cudaStream_t st = thread_stream();
    cudaEvent_t e0, e1;
    TM_CUDA(cudaEventCreate(&e0));
    TM_CUDA(cudaEventCreate(&e1));
    Tuning saved = tuning();
    Tuning bestt = saved;
    float best_ms = 1e30f;
    int rc = TM_OK;
    // warm-up once with the current tuning
    rc = run_batch(g, queries, n_queries, res.data(), st, nullptr);
    for (int bt : bts)
        for (int bps : bpss)
            for (int ch : chunks)
                for (int ti = 0; ti < n_thr; ti++) {
                    if (rc != TM_OK) break;
                    Tuning t;
                    t.block_threads = bt;
                    t.blocks_per_sm = bps;
                    t.chunk_items = ch;
                    t.enum_threshold = thr_matters ? thr_all[ti] : saved.enum_threshold;
                    {
                        std::lock_guard<std::mutex> lk(g_tune_mu);
                        tuning() = t;
                    }
                    // the median of three whole batches (one slow outlier does not pick a tuning)
                    float ms3[3] = {1e30f, 1e30f, 1e30f};
                    for (int rep = 0; rep < 3 && rc == TM_OK; rep++) {
                        cudaEventRecord(e0, st);
                        rc = run_batch(g, queries, n_queries, res.data(), st, nullptr);
                        cudaEventRecord(e1, st);
                        cudaEventSynchronize(e1);
                        cudaEventElapsedTime(&ms3[rep], e0, e1);
                    }
                    std::sort(ms3, ms3 + 3);
                    if (rc == TM_OK && ms3[1] < best_ms) {
                        best_ms = ms3[1];
                        bestt = t;
                    }
                }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tuning() = rc == TM_OK ? bestt : saved;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != TM_OK) return rc;
    best->block_threads = bestt.block_threads;
    best->blocks_per_sm = bestt.blocks_per_sm;
    best->chunk_items = bestt.chunk_items;
    best->enum_threshold = bestt.enum_threshold;
    return TM_OK;
}

int tm_check_status(uint32_t* word, int32_t clear) {
    if (!word) { set_error("NULL argument"); return TM_EINVAL; }
#ifndef TM_CHECKED
    *word = 0;
    set_error("bounds checks are not compiled into this build");
    return TM_EINVAL;
#else
    unsigned a = 0, b = 0, c = 0;
    TM_TRY(check_word_match(&a, clear != 0));
    TM_TRY(check_word_graph(&b, clear != 0));
    TM_TRY(check_word_prims(&c, clear != 0));
    *word = a | b | c;
    return TM_OK;
#endif
}

int tm_check_selftest(void) { return check_selftest(); }

int tm_profile_enable(int32_t on) {
    g_prof_on.store(on != 0);
    return TM_OK;
}

int tm_release_cached_memory(void) { return pool_trim(); }

int tm_profile_last(tm_profile* out) {
    if (!out) { set_error("NULL argument"); return TM_EINVAL; }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    *out = g_prof;
    out->launches = g_launches.load();
    return TM_OK;
}

}  // extern "C"
