// Streaming evaluation of a batch over a time-sorted edge list held in host memory.
//
// The sampling framework needs, for one window, only the edges inside it, so windows can
// be taken chronologically while edges stream in (the streaming remark that follows the
// choice of q_j in Section 4).  Here the edge list is cut into chronological segments of
// a bounded number of edges; each segment is copied to the device (the copy of segment
// i+1 overlaps the matching of segment i), built into a graph, and given the windows of
// every estimate query that lie wholly inside it and the first edges of every exact query
// whose delta-span lies inside it.  Each window and each first edge is taken in exactly
// one segment, so the per-shift sums -- exact integers for counts and Q64 weights -- add
// up to those of the whole graph; the results are those of tm_run_batch on the whole
// graph (bit-identical for counts and uniform-q estimates).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "tm_internal.cuh"

namespace tmo {
namespace {

constexpr int64_t kNoEnd = INT64_MAX;

struct QState {
    bool live = false;     // accepted and not finished
    bool exact = false;
    int64_t cd = 0, delta = 0, J = 0;
    int32_t b = 1;
    int64_t smin = 0, smax = 0;   // extreme shifts over the b repetitions
    int64_t j_next = 0;           // estimate: windows 1 .. j_next of every shift are done
    int64_t own_next = 0;         // exact: first edges with global time < own_next are done
    std::vector<ShiftSums> acc;   // per shift
};

// one segment: edges [ea, eb) of the list, complete for global times [.., B]
struct Seg {
    int64_t ea = 0, eb = 0, B = 0;
    bool last = false;
    std::vector<SegSpec> spec;    // per query (J = 0 / empty own range: nothing here)
    std::vector<int> qidx;        // queries with work in this segment
    std::vector<int64_t> j_hi, own_hi;
};

// the work of every live query inside edges [ea, eb); false if none can progress
bool plan_segment(const int64_t* t, int64_t m, int64_t tmin, int64_t tmax, int64_t ea, int64_t eb,
                  std::vector<QState>& qs, Seg& sg) {
    sg.ea = ea;
    sg.eb = eb;
    sg.last = eb >= m;
    sg.B = sg.last ? tmax : (t[eb] - tmin) - 1;
    int64_t t_off = ea < m ? t[ea] - tmin : 0;
    size_t nq = qs.size();
    sg.spec.assign(nq, SegSpec{});
    sg.qidx.clear();
    sg.j_hi.assign(nq, 0);
    sg.own_hi.assign(nq, 0);
    for (size_t i = 0; i < nq; i++) {
        QState& Q = qs[i];
        if (!Q.live) continue;
        SegSpec& S = sg.spec[i];
        S.t_off = t_off;
        S.m_total = m;
        if (Q.exact) {
            int64_t hi = sg.last ? kNoEnd : sg.B - Q.delta + 1;   // instances starting before hi end by B
            sg.own_hi[i] = std::max(hi, Q.own_next);
            if (sg.own_hi[i] > Q.own_next) {
                S.own_lo = Q.own_next - t_off;
                S.own_hi = sg.own_hi[i] == kNoEnd ? kNoEnd : sg.own_hi[i] - t_off;
                sg.qidx.push_back((int)i);
            }
        } else {
            // window j (1-based) of shift s spans [s + (j-1) cd, s + j cd - 1]
            int64_t jh = sg.last ? Q.J : std::min(Q.J, (sg.B + 1 - Q.smax) / Q.cd);
            sg.j_hi[i] = std::max(jh, Q.j_next);
            if (sg.j_hi[i] > Q.j_next) {
                S.j_lo = Q.j_next;
                S.J = sg.j_hi[i] - Q.j_next;
                sg.qidx.push_back((int)i);
            }
        }
    }
    return !sg.qidx.empty();
}

// the first edge the next segment needs, once this segment's work is done
int64_t next_start(const int64_t* t, int64_t m, int64_t tmin, const std::vector<QState>& qs) {
    int64_t A = kNoEnd;
    for (const QState& Q : qs) {
        if (!Q.live) continue;
        A = std::min(A, Q.exact ? Q.own_next : Q.smin + Q.j_next * Q.cd);
    }
    if (A == kNoEnd) return m;
    A = std::max<int64_t>(A, 0);
    return std::lower_bound(t, t + m, tmin + A) - t;
}

// edges [ea, eb') with eb' <= ea + E cut between two distinct times (or every edge of
// time t[ea] when they alone exceed E)
int64_t cut_end(const int64_t* t, int64_t m, int64_t ea, int64_t E) {
    int64_t eb = std::min(m, ea + E);
    if (eb >= m) return m;
    while (eb > ea && t[eb - 1] == t[eb]) eb--;
    if (eb == ea) eb = std::upper_bound(t, t + m, t[ea]) - t;
    return eb;
}

struct DevBuf {
    int32_t* src = nullptr;
    int32_t* dst = nullptr;
    int64_t* t = nullptr;
    int64_t cap = 0;
};

struct Staging {
    int32_t* src = nullptr;
    int32_t* dst = nullptr;
    int64_t* t = nullptr;
    int64_t cap = 0;
};

int grow_dev(DevBuf& d, int64_t n) {
    if (n <= d.cap) return TM_OK;
    cudaFree(d.src); cudaFree(d.dst); cudaFree(d.t);
    d = DevBuf{};
    TM_CUDA(cudaMalloc(&d.src, 4 * (size_t)n));
    TM_CUDA(cudaMalloc(&d.dst, 4 * (size_t)n));
    TM_CUDA(cudaMalloc(&d.t, 8 * (size_t)n));
    d.cap = n;
    return TM_OK;
}

int grow_host(Staging& h, int64_t n) {
    if (n <= h.cap) return TM_OK;
    cudaFreeHost(h.src); cudaFreeHost(h.dst); cudaFreeHost(h.t);
    h = Staging{};
    TM_CUDA(cudaMallocHost(&h.src, 4 * (size_t)n));
    TM_CUDA(cudaMallocHost(&h.dst, 4 * (size_t)n));
    TM_CUDA(cudaMallocHost(&h.t, 8 * (size_t)n));
    h.cap = n;
    return TM_OK;
}

bool is_pinned(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace
}  // namespace tmo

extern "C" int tm_stream_run(const int32_t* src, const int32_t* dst, const int64_t* t, int64_t m,
                             int32_t n_nodes, const tm_query* queries, int32_t n_queries,
                             int64_t segment_edges, tm_result* results, tm_stream_stats* stats) {
    using namespace tmo;
    auto wall0 = std::chrono::steady_clock::now();
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_queries < 0 || (n_queries > 0 && (!queries || !results))) { set_error("NULL argument"); return TM_EINVAL; }
    if (m < 0 || m >= ((int64_t)1 << 31) - 1) { set_error("m outside [0, 2^31-1)"); return TM_EINVAL; }
    if (m > 0 && (!src || !dst || !t)) { set_error("NULL edge array"); return TM_EINVAL; }
    if (n_nodes < 1) { set_error("n_nodes must be given (>= 1)"); return TM_EINVAL; }
    if (segment_edges < 1) { set_error("segment_edges < 1"); return TM_EINVAL; }
    if (n_queries == 0) return TM_OK;
    for (int64_t i = 1; i < m; i++)
        if (t[i] < t[i - 1]) { set_error("timestamps not sorted"); return TM_EUNSORTED; }
    const int64_t tmin = m > 0 ? t[0] : 0;
    const int64_t tmax = m > 0 ? t[m - 1] - tmin : 0;

    // queries: checked against the whole list, as tm_run_batch would
    std::vector<QState> qs((size_t)n_queries);
    int first_err = TM_OK;
    for (int i = 0; i < n_queries; i++) {
        const tm_query& q = queries[i];
        std::memset(&results[i], 0, sizeof(tm_result));
        std::string why;
        int s = check_query(tmax, q, why);
        if (s == TM_OK && q.mode == TM_MODE_ESTIMATE && q.q_mode == TM_Q_AUTO) {
            s = TM_EINVAL;   // the pilot would need the whole graph
            why = "TM_Q_AUTO needs tm_run_batch";
        }
        if (s != TM_OK) {
            results[i].status = s;
            if (first_err == TM_OK) { first_err = s; set_error("query " + std::to_string(i) + ": " + why); }
            continue;
        }
        QState& Q = qs[(size_t)i];
        Q.live = true;
        Q.exact = q.mode == TM_MODE_EXACT;
        Q.delta = q.delta;
        if (Q.exact) {
            Q.b = 1;
        } else {
            Q.b = q.b;
            Q.cd = (int64_t)q.c * q.delta;
            Q.J = 1 + (tmax + Q.cd - 1) / Q.cd;
            Q.smin = 0;
            Q.smax = -Q.cd;
            for (int k = 0; k < Q.b; k++) {
                int64_t sk = -(int64_t)(draw(q.seed, (uint64_t)k, 0) % (uint64_t)Q.cd);
                Q.smin = std::min(Q.smin, sk);
                Q.smax = std::max(Q.smax, sk);
            }
        }
        Q.acc.assign((size_t)Q.b, ShiftSums{});
    }

    cudaStream_t st = nullptr, cp = nullptr;
    DevBuf dev[2];
    Staging stg[2];
    int rc = TM_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        if (rc == TM_OK && e != cudaSuccess) rc = cuda_status(e, what, __FILE__, __LINE__);
    };
    fail(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    fail(cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking), "copy stream");
    const bool pinned = m > 0 && is_pinned(src) && is_pinned(dst) && is_pinned(t);
    int64_t E = segment_edges;
    double wait_ms = 0.0;
    int64_t n_seg = 0, copied = 0, max_seg = 0;

    // copy edges [ea, eb) into buffer slot b: through pinned staging unless the caller's
    // arrays are pinned; runs on its own thread so that it overlaps the matching
    int device = 0;
    fail(cudaGetDevice(&device), "device");
    auto copy_in = [&](int b, int64_t ea, int64_t eb, int* out_rc) {
        int64_t n = eb - ea;
        cudaSetDevice(device);
        int r = grow_dev(dev[b], std::max<int64_t>(n, 1));
        const int32_t* hs = src + ea;
        const int32_t* hd = dst + ea;
        const int64_t* ht = t + ea;
        if (r == TM_OK && !pinned) {
            r = grow_host(stg[b], std::max<int64_t>(n, 1));
            if (r == TM_OK && n > 0) {
                std::memcpy(stg[b].src, hs, 4 * (size_t)n);
                std::memcpy(stg[b].dst, hd, 4 * (size_t)n);
                std::memcpy(stg[b].t, ht, 8 * (size_t)n);
                hs = stg[b].src; hd = stg[b].dst; ht = stg[b].t;
            }
        }
        cudaError_t e = cudaSuccess;
        if (r == TM_OK && n > 0) {
            e = cudaMemcpyAsync(dev[b].src, hs, 4 * (size_t)n, cudaMemcpyHostToDevice, cp);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dev[b].dst, hd, 4 * (size_t)n, cudaMemcpyHostToDevice, cp);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dev[b].t, ht, 8 * (size_t)n, cudaMemcpyHostToDevice, cp);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cp);
            if (e != cudaSuccess) r = cuda_status(e, "segment copy", __FILE__, __LINE__);
        }
        *out_rc = r;
    };

    // first segment
    Seg cur, nxt;
    int64_t ea = 0;
    bool have = false;
    if (rc == TM_OK) {
        for (;;) {
            int64_t eb = cut_end(t, m, ea, E);
            if (plan_segment(t, m, tmin, tmax, ea, eb, qs, cur)) { have = true; break; }
            if (eb >= m) break;
            E *= 2;   // a window or a delta-span holds more edges than the budget
        }
    }
    int cur_rc = TM_OK;
    if (have) copy_in(0, cur.ea, cur.eb, &cur_rc);
    if (cur_rc != TM_OK) rc = cur_rc;
    int slot = 0;
    std::vector<tm_query> sq;
    std::vector<SegSpec> sspec;
    std::vector<tm_result> sres;
    std::vector<ShiftSums> ssum;
    while (rc == TM_OK && have) {
        // commit this segment's progress, then plan and start copying the next one
        for (int i : cur.qidx) {
            QState& Q = qs[(size_t)i];
            if (Q.exact) Q.own_next = cur.own_hi[(size_t)i];
            else Q.j_next = cur.j_hi[(size_t)i];
        }
        for (QState& Q : qs)
            if (Q.live && ((Q.exact && Q.own_next == kNoEnd) || (!Q.exact && Q.j_next >= Q.J))) Q.live = false;
        if (cur.last)
            for (QState& Q : qs) Q.live = false;
        bool have_next = false;
        int64_t na = next_start(t, m, tmin, qs);
        if (na < m || std::any_of(qs.begin(), qs.end(), [](const QState& Q) { return Q.live; })) {
            int64_t En = segment_edges;
            for (;;) {
                int64_t eb = cut_end(t, m, na, En);
                if (plan_segment(t, m, tmin, tmax, na, eb, qs, nxt)) { have_next = true; break; }
                if (eb >= m) break;
                En *= 2;
            }
        }
        int next_rc = TM_OK;
        std::thread pre;
        if (have_next) pre = std::thread(copy_in, slot ^ 1, nxt.ea, nxt.eb, &next_rc);

        // this segment: graph, then one batch of the queries with work in it
        tm_graph* g = nullptr;
        int64_t n = cur.eb - cur.ea;
        rc = tm_graph_load_device(dev[slot].src, dev[slot].dst, dev[slot].t, n, n_nodes, st, &g);
        if (rc == TM_OK) {
            size_t k = cur.qidx.size();
            sq.resize(k);
            sspec.resize(k);
            sres.assign(k, tm_result{});
            int64_t ns = 0;
            for (size_t x = 0; x < k; x++) {
                int i = cur.qidx[x];
                sq[x] = queries[i];
                sspec[x] = cur.spec[(size_t)i];
                ns += qs[(size_t)i].b;
            }
            ssum.assign((size_t)ns, ShiftSums{});
            BatchOut bo;
            bo.seg = sspec.data();
            bo.sums = ssum.data();
            rc = run_batch(g, sq.data(), (int)k, sres.data(), st, &bo);
            int64_t base = 0;
            for (size_t x = 0; x < k && rc == TM_OK; x++) {
                QState& Q = qs[(size_t)cur.qidx[x]];
                for (int kk = 0; kk < Q.b; kk++) add_shift_sums(Q.acc[(size_t)kk], ssum[(size_t)(base + kk)]);
                base += Q.b;
            }
            tm_graph_free(g);
        }
        n_seg++;
        copied += n;
        max_seg = std::max(max_seg, n);
        auto w0 = std::chrono::steady_clock::now();
        if (pre.joinable()) pre.join();
        wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
        if (rc == TM_OK && next_rc != TM_OK) rc = next_rc;
        if (!have_next) break;
        std::swap(cur, nxt);
        slot ^= 1;
    }

    // results, folded as the fold kernels fold one batch
    if (rc == TM_OK) {
        for (int i = 0; i < n_queries; i++) {
            if (results[i].status != TM_OK) continue;
            const QState& Q = qs[(size_t)i];
            const tm_query& q = queries[i];
            tm_result& r = results[i];
            unsigned long long cnt = 0, first = 0, cand = 0, last = 0, inst = 0, kept = 0;
            double zsum = 0.0, vsum = 0.0, wmean = 0.0, wm2 = 0.0;
            bool overflow = false;
            for (int k = 0; k < Q.b; k++) {
                const ShiftSums& S = Q.acc[(size_t)k];
                cnt += S.count; first += S.first; cand += S.cand; last += S.last; inst += S.inst; kept += S.kept;
                if (S.whi >= (1ull << 63) || S.count >= (1ull << 63)) overflow = true;
                double Wd = (double)S.whi + (double)S.wlo * 0x1.0p-64;
                double zk = q.q_mode == TM_Q_EDGES ? S.zq : Wd / q.p;
                zsum += zk;
                vsum += S.vq;
                double dz = zk - wmean;
                wmean += dz / (k + 1);
                wm2 += dz * (zk - wmean);
            }
            r.status = overflow ? TM_EOVERFLOW : TM_OK;
            r.count = (int64_t)cnt;
            if (Q.exact) {
                r.estimate = (double)cnt;
                r.windows = 1;
                r.windows_kept = 1;
                r.p_used = 1.0;
            } else {
                r.estimate = zsum / Q.b;
                r.windows = (int64_t)Q.b * Q.J;
                r.windows_kept = (int64_t)kept;
                r.var_hat = vsum / Q.b;
                r.shift_var = Q.b >= 2 ? wm2 / (Q.b - 1) : 0.0;
                r.p_used = q.p;
            }
            r.first_edges = (int64_t)first;
            r.cand_edges = (int64_t)cand;
            r.last_ranges = (int64_t)last;
            r.inst_read = (int64_t)inst;
            if (overflow && first_err == TM_OK) { first_err = TM_EOVERFLOW; set_error("count or weight >= 2^63"); }
        }
    }
    if (st) cudaStreamDestroy(st);
    if (cp) cudaStreamDestroy(cp);
    for (int b = 0; b < 2; b++) {
        cudaFree(dev[b].src); cudaFree(dev[b].dst); cudaFree(dev[b].t);
        cudaFreeHost(stg[b].src); cudaFreeHost(stg[b].dst); cudaFreeHost(stg[b].t);
    }
    if (stats) {
        stats->segments = n_seg;
        stats->edges_copied = copied;
        stats->max_segment_edges = max_seg;
        stats->copy_wait_ms = wait_ms;
        stats->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    }
    if (rc != TM_OK) return rc;
    return first_err;
}
