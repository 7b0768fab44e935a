// The estimator's hot path (Algorithm 1 around the exact counter A of
// Section 4), one batch of queries at a time:
//
//   k_wtab     per estimate query, the weights 1/p_{M'} = c delta / (c delta - Delta)
//              (Eq. 2) for every duration Delta in [0, delta], in unsigned Q64
//              fixed point, so that window sums are exact integer sums.
//   k_windows  one thread per window I_j of Eq. 1 of every shift of every
//              query: shift s and keep decision U_j < q_j (Algorithm 1), and
//              T_j as an edge range [lo, hi) found by binary search on time.
//   k_level2   one thread per first edge of every kept window: the range of
//              candidates for the second motif edge (time in (t_1, t_1 + delta],
//              clamped to the window) in the adjacency view the motif needs.
//   k_match    persistent warps over equal chunks of the concatenated
//              second-edge candidates (the work queue); deeper motif edges are
//              expanded warp-cooperatively (range lengths scanned across the
//              warp, each lane takes one candidate, owner found by shuffles);
//              in exact mode the last motif edge is counted by range length.
//   k_fold_shift, k_fold_final
//              per query, shift and slice of windows the partial sums, then per
//              query: Z_k = sum_j W_j / q_j per shift and the mean over shifts
//              (Algorithm 1's return value).
#include <algorithm>
#include <atomic>
#include <limits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "tm_internal.cuh"

namespace tmo {

Tuning& tuning() {
    static Tuning t;
    return t;
}

// Records the deferred-rider buffer of a batch holds: grows to the largest count a batch has
// needed (tm_set_ride_capacity sets it)
std::atomic<int64_t>& ride_capacity() {
    static std::atomic<int64_t> cap{(int64_t)1 << 23};
    return cap;
}

namespace {

constexpr int64_t kInf = INT64_MAX;
constexpr int64_t kWtabMax = (int64_t)1 << 22;   // largest delta+1 given a weight table
constexpr double kFullScanP = 0.25;              // keep rate from which windows enumerate by node
constexpr int64_t kRevMinLen = 8;                // shortest second-edge range worth closing from the other side

// per-window accumulator fields
enum { A_COUNT = 0, A_WLO, A_WHI, A_FIRST, A_CAND, A_LAST, A_INST, A_X0, A_X1, A_X2, A_N };

struct WinDev {
    int64_t* lo;      // first edges of the window: positions [lo, hi) of the query's order
    int64_t* hi;
    int64_t* tlo;     // T_j = edges [tlo, thi) of the time-sorted list
    int64_t* thi;
    int64_t* tend;    // last admissible time (window end), kInf for exact
    int64_t* start;   // a_j
    int64_t* j;       // window index (1-based; 0 for exact)
    int32_t* q;       // query
    int32_t* k;       // shift index
    int32_t* kept;
    double* qj;       // q_j
    int64_t* nfirst;  // hi - lo if kept else 0
    int64_t* fbase;   // exclusive scan of nfirst
    unsigned long long* acc;  // [NW][A_N]
};

// What the matcher needs of a first edge that has items, in one record that k_level2 writes
// (32 bytes with 32-bit times): each item starts from one load instead of a chain through
// the window table, the plan and the edge arrays.
template <typename TT>
struct FRec {
    int32_t s1, d1;   // the first edge's nodes
    int32_t win;      // its window slot
    int32_t q;        // its query
    TT t1;            // its time
    TT thi;           // last time an instance starting there may use (clamped to TT's range,
                      // which holds every edge time)
    int64_t lo2;      // start of its items in their view (negative: closing-side items)
};
static_assert(sizeof(FRec<int32_t>) == 32 && sizeof(FRec<int64_t>) == 40, "first-edge record layout");

// Instances of an exact query that its riders and smaller spans still have to weigh, deferred
// by k_match to k_ride (so the matcher's hot loop carries none of their chains of loads): the
// closing entries [x, x + n) of pair_t after time tc, or, for n < 0, -n instances whose last
// edge is at time x.
template <typename TT>
struct RideRec {
    int64_t x;
    TT t1;       // the instances' first-edge time
    TT tc;       // range records: the time after which the closing entries lie
    int32_t q;   // the exact query
    int32_t n;
};
static_assert(sizeof(RideRec<int32_t>) == 24 && sizeof(RideRec<int64_t>) == 32, "rider record layout");

template <typename TT>
struct MatchArgs {
    GraphDevT<TT> G;
    const QPlan* plans;
    int nq;
    WinDev W;
    int64_t NW;
    int64_t F;
    const int64_t* d_F;    // if set, the first-edge count is read here on the device
    const FRec<TT>* rec;   // [F] record of each first edge with items
    const int64_t* excl;   // [F] exclusive scan of the range lengths
    const int64_t* hs_a;   // [F] closing pair range start (queries whose last edge is fixed by the first)
    const int64_t* hs_hi;  // [F] closing pair range end
    const int64_t* d_W2;   // total second-edge candidates
    unsigned long long* counter;
    int64_t chunk;
    int enum_threshold;
    const int32_t* blockwin = nullptr;  // [ceil(F/32)] window of first edge 32 b (null: searched)
    const int64_t* chunkf = nullptr;    // [nchunkf] first edge of work item i * chunk (null: searched)
    int64_t nchunkf = 0;
    RideRec<TT>* rrec = nullptr;        // [rcap] deferred rider / smaller-span work (see RideRec)
    unsigned long long* rcount = nullptr;   // records appended (counts past rcap: the batch reruns)
    int64_t rcap = 0;
};

// ----------------------------------------------------------------- helpers
template <int K>
__device__ __forceinline__ int32_t phi_get(const int32_t (&phi)[K], int idx) {
    int32_t v = phi[0];
#pragma unroll
    for (int i = 1; i < K; i++)
        if (idx == i) v = phi[i];
    return v;
}
template <int K>
__device__ __forceinline__ void phi_set(int32_t (&phi)[K], int idx, int32_t v) {
#pragma unroll
    for (int i = 0; i < K; i++)
        if (idx == i) phi[i] = v;
}
template <int K>
__device__ __forceinline__ bool phi_has(const int32_t (&phi)[K], int nb, int32_t v) {
    bool r = false;
#pragma unroll
    for (int i = 0; i < K; i++) r |= (i < nb) & (phi[i] == v);
    return r;
}

// first index in [lo, hi) with a[idx] > v, by exponential then binary search
// from lo: about 2 log2(answer - lo) probes, cheap when the answer is near lo
template <typename T>
__device__ __forceinline__ int64_t gallop_ub(const T* __restrict__ a, int64_t lo, int64_t hi,
                                             int64_t v) {
    int64_t cur = lo, step = 1;
    while (cur < hi && (int64_t)__ldg(a + cur) <= v) {
        lo = cur + 1;
        cur += step;
        step <<= 1;
    }
    if (cur > hi) cur = hi;
    return upper_bound_i64(a, lo, cur, v);
}

// time-sorted entries of the (u -> v) pair: [a, b) of pair_t, through the
// open-addressing hash of static edges (probe chains end at an empty slot)
template <typename TT>
__device__ __forceinline__ int64_t pair_count(const GraphDevT<TT>& G, int32_t u, int32_t v, int64_t tprev,
                                              int64_t thi) {
    int64_t a, b;
    if (thi <= tprev || !pair_segment(G, u, v, a, b)) return 0;
    int64_t lo = upper_bound_i64(G.pair_t, a, b, tprev);
    int64_t hi = gallop_ub(G.pair_t, lo, b, thi);
    return hi - lo;
}

// the same entries as a range [lo, hi) of pair_t (empty: lo == hi)
template <typename TT>
__device__ __forceinline__ void pair_range(const GraphDevT<TT>& G, int32_t u, int32_t v, int64_t tprev,
                                           int64_t thi, int64_t& lo, int64_t& hi) {
    int64_t a, b;
    lo = hi = 0;
    if (thi <= tprev || !pair_segment(G, u, v, a, b)) return;
    lo = upper_bound_i64(G.pair_t, a, b, tprev);
    hi = gallop_ub(G.pair_t, lo, b, thi);
}

// candidates of motif edge P given the bound nodes: entries [lo, lo+len) of
// the view's time array with time in (tprev, thi]
template <typename TT, int K>
__device__ __forceinline__ void level_range(const GraphDevT<TT>& G, const LevelPlan& P,
                                            const int32_t (&phi)[K], int64_t tprev, int64_t thi,
                                            int64_t& lo, int64_t& len) {
    const TT* ta;
    int64_t a, b;
    lo = 0;
    len = 0;
    if (thi <= tprev) return;
    if (P.view == kPair) {
        ta = G.pair_t;
        if (!pair_segment(G, phi_get(phi, P.su), phi_get(phi, P.sv), a, b)) return;
    } else if (P.view == kOut) {
        int32_t u = (int32_t)TM_CHK_IDX(phi_get(phi, P.su), G.n, kChkNode);
        ta = G.out_t; a = __ldg(G.out_off + u); b = __ldg(G.out_off + u + 1);
    } else if (P.view == kIn) {
        int32_t v = (int32_t)TM_CHK_IDX(phi_get(phi, P.sv), G.n, kChkNode);
        ta = G.in_t; a = __ldg(G.in_off + v); b = __ldg(G.in_off + v + 1);
    } else {
        ta = G.t; a = 0; b = G.m;
    }
    lo = upper_bound_i64(ta, a, b, tprev);
    len = gallop_ub(ta, lo, b, thi) - lo;
}

// read candidate c of the view; returns its (src, dst, time)
template <typename TT, int K>
__device__ __forceinline__ void read_cand(const GraphDevT<TT>& G, const LevelPlan& P,
                                          const int32_t (&phi)[K], int64_t c, int32_t& s,
                                          int32_t& d, int64_t& tc) {
    if (P.view == kPair) {
        s = phi_get(phi, P.su); d = phi_get(phi, P.sv); tc = __ldg(G.pair_t + c);
    } else if (P.view == kOut) {
        s = phi_get(phi, P.su); d = __ldg(G.out_nbr + c); tc = __ldg(G.out_t + c);
    } else if (P.view == kIn) {
        s = __ldg(G.in_nbr + c); d = phi_get(phi, P.sv); tc = __ldg(G.in_t + c);
    } else {
        s = __ldg(G.src + c); d = __ldg(G.dst + c); tc = __ldg(G.t + c);
    }
}

// the first edge at position e of the order the query enumerates first edges in
template <typename TT>
__device__ __forceinline__ void first_edge(const GraphDevT<TT>& G, int order, int64_t e, int32_t& s,
                                           int32_t& d, int64_t& t) {
    if (order == kOrdOut) {
        s = __ldg(G.out_src + e); d = __ldg(G.out_nbr + e); t = __ldg(G.out_t + e);
    } else if (order == kOrdIn) {
        s = __ldg(G.in_nbr + e); d = __ldg(G.in_dst + e); t = __ldg(G.in_t + e);
    } else if (order == kOrdPair) {
        // the pair view is grouped by source at the same positions as the out view
        s = __ldg(G.out_src + e); d = __ldg(G.pair_dst + __ldg(G.pair_pid + e)); t = __ldg(G.pair_t + e);
    } else {
        s = __ldg(G.src + e); d = __ldg(G.dst + e); t = __ldg(G.t + e);
    }
}

// injectivity of the node map (Def. 2.2 item 1) for a candidate, and binding
template <int K>
__device__ __forceinline__ bool check_bind(const LevelPlan& P, int32_t (&phi)[K], int32_t s,
                                           int32_t d) {
    if (s == d) return false;
    if (P.bind_u && phi_has(phi, P.nb, s)) return false;
    if (P.bind_v && phi_has(phi, P.nb, d)) return false;
    if (P.bind_u) phi_set(phi, P.su, s);
    if (P.bind_v) phi_set(phi, P.sv, d);
    return true;
}

// exact count of the last motif edge's candidates in (tprev, thi] when one
// endpoint is new: the range length minus the entries whose new endpoint is
// already bound (those are exactly the pair segments to bound nodes)
template <typename TT, int K>
__device__ __forceinline__ int64_t last_count_subtract(const GraphDevT<TT>& G, const LevelPlan& P,
                                                       const int32_t (&phi)[K], int64_t len,
                                                       int64_t tprev, int64_t thi) {
    int64_t excl = 0;
    if (P.view == kOut) {
        int32_t u = phi_get(phi, P.su);
#pragma unroll
        for (int i = 0; i < K; i++)
            if (i < P.nb) excl += pair_count(G, u, phi[i], tprev, thi);
    } else {
        int32_t v = phi_get(phi, P.sv);
#pragma unroll
        for (int i = 0; i < K; i++)
            if (i < P.nb) excl += pair_count(G, phi[i], v, tprev, thi);
    }
    return len - excl;
}

// Per-lane accumulator of one window.  The count and the 128-bit weight, touched on every
// instance, live in registers; the other fields (work counters, counts of the spans that
// ride along) live in this thread's slots of shared memory (field-major, stride = block
// size), which keeps them out of the register budget of the matcher kernels.
constexpr int A_NREG = 3;   // A_COUNT, A_WLO, A_WHI
struct Acc {
    int64_t win;
    unsigned long long f[A_NREG];
    unsigned long long* x;   // this thread's first shared-memory slot
    int xs;                  // slot stride (threads per block)
    __device__ __forceinline__ unsigned long long& s(int i) { return x[(i - A_NREG) * xs]; }
    __device__ __forceinline__ unsigned long long get(int i) { return i < A_NREG ? f[i] : s(i); }
};

// dynamic shared memory of k_level2 / k_match: the staged plans, then the accumulator slots
__host__ __device__ __forceinline__ size_t acc_smem_offset(int nq) {
    size_t b = nq <= 64 ? sizeof(QPlan) * (size_t)nq : 0;   // kSmemPlans
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ void acc_init(Acc& a, unsigned char* smem, int nq) {
    a.x = reinterpret_cast<unsigned long long*>(smem + acc_smem_offset(nq)) + threadIdx.x;
    a.xs = blockDim.x;
    a.win = -1;
}

__device__ __forceinline__ void acc_zero(Acc& a) {
#pragma unroll
    for (int i = 0; i < A_NREG; i++) a.f[i] = 0;
#pragma unroll
    for (int i = A_NREG; i < A_N; i++) a.s(i) = 0;
}

__device__ __forceinline__ void atomic_add_u128(unsigned long long* lo_hi, unsigned long long lo,
                                                unsigned long long hi) {
    if (lo) {
        unsigned long long old = atomicAdd(lo_hi, lo);
        if (old + lo < old) hi += 1;
    }
    if (hi) atomicAdd(lo_hi + 1, hi);
}

__device__ __forceinline__ void acc_flush_lane(Acc& a, unsigned long long* acc) {
    if (a.win < 0) return;
    unsigned long long* p = acc + a.win * A_N;
    if (a.f[A_COUNT]) atomicAdd(p + A_COUNT, a.f[A_COUNT]);
    atomic_add_u128(p + A_WLO, a.f[A_WLO], a.f[A_WHI]);
#pragma unroll
    for (int i = A_FIRST; i < A_N; i++) {
        unsigned long long v = a.s(i);
        if (v) atomicAdd(p + i, v);
    }
    acc_zero(a);
}

// warp-uniform flush: one set of atomics when every lane holds the same window
__device__ __forceinline__ void acc_flush_warp(Acc& a, unsigned long long* acc) {
    int64_t w0 = __shfl_sync(kFull, a.win, 0);
    if (__all_sync(kFull, a.win == w0 || a.win < 0) && w0 >= 0) {
        // reduce: Q64 weights carried as 128-bit via (lo, hi) with carries
        unsigned long long lo = a.f[A_WLO], hi = a.f[A_WHI];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long lo2 = __shfl_xor_sync(kFull, lo, o);
            unsigned long long hi2 = __shfl_xor_sync(kFull, hi, o);
            unsigned long long s = lo + lo2;
            hi = hi + hi2 + (s < lo ? 1ull : 0ull);
            lo = s;
        }
        unsigned long long* p = acc + w0 * A_N;
#pragma unroll
        for (int i = 0; i < A_N; i++) {
            if (i == A_WLO || i == A_WHI) continue;
            unsigned long long v = a.get(i);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(p + i, v);
        }
        if ((threadIdx.x & 31) == 0) atomic_add_u128(p + A_WLO, lo, hi);
        acc_zero(a);
    } else {
        acc_flush_lane(a, acc);
    }
}

__device__ __forceinline__ void acc_switch(Acc& a, int64_t win, unsigned long long* acc) {
    if (a.win != win) {
        acc_flush_lane(a, acc);
        a.win = win;
    }
}

// c delta / (c delta - dur) in Q64 by long division (64 fraction bits, rounded down)
__device__ __forceinline__ void q64_weight(int64_t cd, int64_t dur, unsigned long long& wi,
                                        unsigned long long& wf) {
    unsigned long long D = (unsigned long long)(cd - dur);
    unsigned long long N = (unsigned long long)cd;
    wi = N / D;
    unsigned long long r = N - wi * D;
    wf = 0;
    for (int i = 0; i < 64; i++) {
        r <<= 1;
        wf <<= 1;
        if (r >= D) { r -= D; wf |= 1; }
    }
}

__device__ __forceinline__ void add_weight(Acc& a, const QPlan& Q, int64_t dur) {
    unsigned long long wi, wf;
    if (Q.wtab) {
        const ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2*>(Q.wtab) + dur);   // one 16-byte load
        wi = e.x;
        wf = e.y;
    } else {
        q64_weight(Q.cd, dur, wi, wf);
    }
    unsigned long long s = a.f[A_WLO] + wf;
    a.f[A_WHI] += wi + (s < wf ? 1ull : 0ull);
    a.f[A_WLO] = s;
}

// exact queries counted alongside at smaller spans: cnt instances whose last edge is at t3
__device__ __forceinline__ void add_sub_at(Acc& a, const QPlan& Q, int64_t t1, int64_t t3,
                                           unsigned long long cnt) {
#pragma unroll
    for (int i = 0; i < kMaxSub; i++)
        if (i < Q.nsub && t3 - t1 <= Q.dsub[i]) a.s(A_X0 + i) += cnt;
}

// ... and the instances closed by entries (tc, t1 + dsub_i] of a time-sorted range [lo, hi)
// whose entries after tc start at lo
template <typename TT>
__device__ __forceinline__ void add_sub_range(Acc& a, const QPlan& Q, const TT* __restrict__ ta, int64_t lo,
                                              int64_t hi, int64_t t1) {
#pragma unroll
    for (int i = 0; i < kMaxSub; i++)
        if (i < Q.nsub) a.s(A_X0 + i) += gallop_ub(ta, lo, hi, t1 + Q.dsub[i]) - lo;
}

// ---- estimates riding along with an exact query (QPlan::nride / riding).  An instance with
// first edge at t1 and last edge at t3 counts for rider R's shift k when the window of t1 is
// kept and holds t3, and t3 - t1 <= R.delta; it adds R's Q64 weight to that window's sums.
// Inlined: out of line, every call saved and restored the matcher's live registers, which
// cost more than the extra registers inlining takes.
// x / d for x >= 0, d > 0: one 32-bit division when both fit in 32 bits (times of a graph
// whose span fits in 31 bits, and spans c delta below 2^32), else the 64-bit one
__device__ __forceinline__ int64_t div_nonneg(int64_t x, int64_t d) {
    if ((((unsigned long long)x | (unsigned long long)d) >> 32) == 0) return (int64_t)((uint32_t)x / (uint32_t)d);
    return x / d;
}

__device__ __forceinline__ void ride_window(const QPlan& R, int k, int64_t t1, int64_t& w, int64_t& thi) {
    int64_t s = __ldg(R.shifts + k);
    int64_t j = div_nonneg(t1 - s, R.cd);   // 0-based window of t1
    w = R.win_base + (int64_t)k * R.J + j;
    thi = min(t1 + R.delta, s + (j + 1) * R.cd - 1);
}

// Rider sums go through a per-block table in shared memory keyed by window (when c delta is
// long, a handful of windows take most instances, and the same few global words would
// otherwise be hit by every SM; when it is short, a block's records still reach thousands of
// windows), flushed to the global sums when the block ends.  A window takes a free slot among
// kRideProbe from its hash; one that finds them all taken adds to the global sums.  The table
// sits at the end of k_ride's dynamic shared memory.
constexpr int kRideTab = 512;
constexpr int kRideProbe = 4;
constexpr unsigned long long kTabFree = ~0ull;
constexpr unsigned long long kInstKey = 1ull << 62;   // key flag: an exact query's entries-read counter
struct RideTab {
    unsigned long long key[kRideTab];   // window index (with kInstKey: the A_INST counter of that
                                        // window), kTabFree when unused
    unsigned long long cnt[kRideTab];
    unsigned long long lo[kRideTab];    // the Q64 weight sum: lo word, then the integer part
    unsigned long long hi[kRideTab];
};
__device__ __forceinline__ RideTab* ride_tab() {
    extern __shared__ __align__(16) unsigned char smem_plans[];
    uint32_t n;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
    return reinterpret_cast<RideTab*>(smem_plans + n - sizeof(RideTab));
}

// cnt instances with Q64 weight sum (lo, hi) into rider window w: the block's table when the
// window has (or takes) its slot there, else the global sums
__device__ __forceinline__ void ride_add(unsigned long long* acc, int64_t w, unsigned long long cnt,
                                         unsigned long long lo, unsigned long long hi) {
    if (!cnt) return;
    RideTab* tab = ride_tab();
    const unsigned long long h = sm64_mix((unsigned long long)w);
#pragma unroll
    for (int pr = 0; pr < kRideProbe; pr++) {
        const int sl = (int)((h + (unsigned long long)pr) & (kRideTab - 1));
        unsigned long long key = *(volatile unsigned long long*)&tab->key[sl];
        if (key == kTabFree) {
            unsigned long long old = atomicCAS(&tab->key[sl], kTabFree, (unsigned long long)w);
            key = old == kTabFree ? (unsigned long long)w : old;
        }
        if (key == (unsigned long long)w) {
            atomicAdd(&tab->cnt[sl], cnt);
            unsigned long long old = atomicAdd(&tab->lo[sl], lo);
            if (old + lo < old) hi += 1;
            if (hi) atomicAdd(&tab->hi[sl], hi);
            return;
        }
    }
    if ((unsigned long long)w & kInstKey) {
        atomicAdd(acc + ((unsigned long long)w & ~kInstKey) * A_N + A_INST, cnt);
        return;
    }
    unsigned long long* p = acc + w * A_N;
    atomicAdd(p + A_COUNT, cnt);
    atomic_add_u128(p + A_WLO, lo, hi);
}

__device__ __forceinline__ void ride_weight(const QPlan& R, int64_t dur, unsigned long long n,
                                            unsigned long long& lo, unsigned long long& hi) {
    unsigned long long wi, wf;
    if (R.wtab) {
        const ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2*>(R.wtab) + dur);   // one 16-byte load
        wi = e.x;
        wf = e.y;
    } else {
        q64_weight(R.cd, dur, wi, wf);
    }
    lo = wf * n;
    hi = wi * n + __umul64hi(wf, n);
}

// cnt instances closed by the edge at t3
__device__ __forceinline__ void ride_at(const QPlan* __restrict__ PL, const QPlan& Q, const int32_t* __restrict__ kept,
                                     unsigned long long* acc, int64_t t1, int64_t t3, unsigned long long cnt) {
    for (int r = 0; r < Q.nride; r++) {
        const QPlan& R = PL[Q.ride_q[r]];
        if (t3 - t1 > R.delta) continue;
        const bool all_kept = R.q_mode == TM_Q_UNIFORM && R.p >= 1.0;   // no keep flag to read
        for (int k = 0; k < R.b; k++) {
            int64_t w, thi;
            ride_window(R, k, t1, w, thi);
            if (t3 > thi || !(all_kept || kept[w])) continue;
            unsigned long long lo, hi;
            ride_weight(R, t3 - t1, cnt, lo, hi);
            ride_add(acc, w, cnt, lo, hi);
        }
    }
}

// one instance per closing entry of the time-sorted range [lo, hi) (entries after tc); the most
// entries read for one rider shift count as the exact query's last-edge entries read one by one
template <typename TT>
__device__ __forceinline__ void ride_range(const QPlan* __restrict__ PL, const QPlan& Q,
                                        const int32_t* __restrict__ kept, unsigned long long* acc,
                                        const TT* __restrict__ ta, int64_t clo, int64_t chi, int64_t t1,
                                        int64_t tc) {
    unsigned long long nread = 0;
    for (int r = 0; r < Q.nride; r++) {
        const QPlan& R = PL[Q.ride_q[r]];
        if (t1 + R.delta <= tc) continue;   // no closing edge after tc fits the span
        const bool all_kept = R.q_mode == TM_Q_UNIFORM && R.p >= 1.0;   // no keep flag to read
        for (int k = 0; k < R.b; k++) {
            int64_t w, thi;
            ride_window(R, k, t1, w, thi);
            if (thi <= tc || !(all_kept || kept[w])) continue;
            unsigned long long cnt = 0, wl = 0, wh = 0;
            for (int64_t x = clo; x < chi; x++) {
                int64_t t3 = (int64_t)ta[x];
                if (t3 > thi) break;   // times increase
                unsigned long long l, h;
                ride_weight(R, t3 - t1, 1, l, h);
                unsigned long long y = wl + l;
                wh += h + (y < wl ? 1ull : 0ull);
                wl = y;
                cnt++;
            }
            ride_add(acc, w, cnt, wl, wh);
            nread = max(nread, cnt);
        }
    }
    if (nread) ride_add(acc, (int64_t)(kInstKey | (unsigned long long)Q.win_base), nread, 0, 0);
}

// n instances of duration dur at once: n * (wi + wf 2^-64), exactly as n single adds
__device__ __forceinline__ void add_weight_n(Acc& a, const QPlan& Q, int64_t dur, unsigned long long n) {
    unsigned long long wi, wf;
    if (Q.wtab) {
        const ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2*>(Q.wtab) + dur);   // one 16-byte load
        wi = e.x;
        wf = e.y;
    } else {
        q64_weight(Q.cd, dur, wi, wf);
    }
    unsigned long long lo = wf * n, hi = __umul64hi(wf, n);
    unsigned long long s = a.f[A_WLO] + lo;
    a.f[A_WHI] += wi * n + hi + (s < lo ? 1ull : 0ull);
    a.f[A_WLO] = s;
}

__device__ __forceinline__ int64_t warp_incl_scan64(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Query plans staged in shared memory when the batch is small enough (every
// item reads its plan; the block copies them once).
constexpr int kSmemPlans = 64;

__device__ __forceinline__ const QPlan* stage_plans(const QPlan* gplans, int nq, unsigned char* smem) {
    if (nq > kSmemPlans) return gplans;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(gplans);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(smem);
    int words = nq * (int)(sizeof(QPlan) / 8);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    return reinterpret_cast<const QPlan*>(smem);
}

static_assert(kSmemPlans == 64, "acc_smem_offset assumes 64 staged plans at most");

// dynamic shared memory of k_level2 / k_match: plans, then the accumulator slots, then (k_match
// of a batch with riders) the rider table
size_t match_smem_bytes(int nq, int threads, bool ride_tab = false) {
    return acc_smem_offset(nq) + (size_t)(A_N - A_NREG) * 8 * (size_t)threads + (ride_tab ? sizeof(RideTab) : 0);
}

// ----------------------------------------------------------------- kernels
__global__ void k_wtab(uint64_t* __restrict__ tab, int64_t delta, int64_t cd) {
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d <= delta;
         d += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long D = (unsigned long long)(cd - d);
        if (D == 0) {  // duration c*delta (c = 1) never fits inside a window of c*delta ticks
            tab[2 * d] = 0;
            tab[2 * d + 1] = 0;
            continue;
        }
        unsigned long long N = (unsigned long long)cd;
        unsigned long long wi = N / D, r = N - wi * D, wf = 0;
        for (int i = 0; i < 64; i++) {
            r <<= 1;
            wf <<= 1;
            if (r >= D) { r -= D; wf |= 1; }
        }
        tab[2 * d] = wi;
        tab[2 * d + 1] = wf;
    }
}

template <typename TT>
__global__ void k_windows(GraphDevT<TT> G, const QPlan* __restrict__ plans, int nq, WinDev W, int64_t NW) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < NW;
         w += (int64_t)gridDim.x * blockDim.x) {
        int lo_q = 0, hi_q = nq;
        while (hi_q - lo_q > 1) {
            int mid = (lo_q + hi_q) >> 1;
            if (plans[mid].win_base <= w) lo_q = mid; else hi_q = mid;
        }
        const QPlan& Q = plans[lo_q];
        int64_t r = w - Q.win_base;
        int64_t lo, hi, tend, start, j;
        int32_t k, kept;
        double qj;
        if (Q.mode == TM_MODE_EXACT) {
            k = 0; j = 0; start = 0; lo = 0; hi = G.m; tend = kInf; kept = 1; qj = 1.0;
            W.tlo[w] = 0;
            W.thi[w] = G.m;
        } else if (Q.wclamp) {
            // every window kept: one slot per shift over every edge; start holds the shift
            k = (int32_t)r;
            j = 0; lo = 0; hi = G.m; tend = kInf; kept = 1; qj = 1.0;
            start = -(int64_t)(draw(Q.seed, (uint64_t)k, 0) % (uint64_t)Q.cd) - Q.t_off;
            W.tlo[w] = 0;
            W.thi[w] = G.m;
        } else {
            k = (int32_t)(r / Q.J);
            j = Q.j_lo + r % Q.J + 1;
            uint64_t h0 = draw(Q.seed, (uint64_t)k, 0);
            int64_t s = -(int64_t)(h0 % (uint64_t)Q.cd);
            start = s + (j - 1) * Q.cd - Q.t_off;
            tend = start + Q.cd - 1;
            lo = lower_bound_i64(G.t, 0, G.m, start);
            hi = upper_bound_i64(G.t, lo, G.m, tend);
            W.tlo[w] = lo;
            W.thi[w] = hi;
            if (Q.full) {
                // this window's node-grouped positions, partitioned per shift into perm
                const int64_t* off = Q.woff + (int64_t)k * (Q.J + 1);
                int64_t base = (int64_t)k * G.m;
                int64_t a = off[j - 1], b = off[j];
                lo = base + a;
                hi = base + b;
            }
            if (Q.q_mode == TM_Q_EDGES) {
                qj = Q.m_total > 0 ? Q.p * (double)(hi - lo) / (double)Q.m_total : 0.0;
                if (qj > 1.0) qj = 1.0;
            } else {
                qj = Q.p;
            }
            double u = (double)(draw(Q.seed, (uint64_t)k, (uint64_t)j) >> 11) * 0x1.0p-53;
            kept = u < qj ? 1 : 0;
        }
        W.lo[w] = lo; W.hi[w] = hi; W.tend[w] = tend; W.start[w] = start; W.j[w] = j;
        W.q[w] = lo_q; W.k[w] = k; W.kept[w] = kept; W.qj[w] = qj;
        W.nfirst[w] = (kept && !Q.riding) ? hi - lo : 0;   // riders take no first edges
    }
}

// window index (0-based) of every position of a node-grouped view for shift s
template <typename TT>
__global__ void k_winkey(const TT* __restrict__ tv, int64_t m, int64_t s, int64_t cd,
                         uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = (uint32_t)(((int64_t)tv[i] - s) / cd);
        val[i] = (uint32_t)i;
    }
}

__global__ void k_woff(const uint32_t* __restrict__ keys, int64_t m, int64_t nkeys, int64_t* __restrict__ off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t prev = i == 0 ? -1 : (int64_t)keys[i - 1];
        int64_t cur = i == m ? nkeys : (int64_t)keys[i];
        for (int64_t v = prev + 1; v <= cur; v++) off[v] = i;
    }
}

// last time an instance starting at t1 may use: t1 + delta, clamped to the window's end (for
// a query whose windows are all kept, the end of t1's own window)
__device__ __forceinline__ int64_t first_thi(const QPlan& Q, const WinDev& W, int64_t win, int64_t t1) {
    int64_t tend = W.tend[win];
    if (Q.wclamp) {
        int64_t s = W.start[win];
        tend = s + (div_nonneg(t1 - s, Q.cd) + 1) * Q.cd - 1;
    }
    return min(t1 + Q.delta, tend);
}

// window of first edge 32 b for every block b of 32 first edges: one search each,
// run at full occupancy instead of on the critical path of k_level2's warps
__global__ void k_blockwin(const int64_t* __restrict__ fbase, int64_t NW, int64_t Fh,
                           const int64_t* __restrict__ d_F, int32_t* __restrict__ bw) {
    const int64_t F = d_F ? *d_F : Fh;
    int64_t nb = (F + 31) >> 5;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = b << 5, lo = 0, hi = NW;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (__ldg(fbase + mid) <= x) lo = mid; else hi = mid;
        }
        bw[b] = (int32_t)lo;
    }
}

// first edge of work item i * chunk (the start of k_match's i-th chunk), for the first
// cap chunks and the one after the last
__global__ void k_chunkf(const int64_t* __restrict__ excl, int64_t Fh, const int64_t* __restrict__ d_F,
                         const int64_t* __restrict__ d_W2, int64_t chunk, int64_t cap,
                         int64_t* __restrict__ cf) {
    const int64_t F = d_F ? *d_F : Fh;
    int64_t n = min(cap, (*d_W2 + chunk - 1) / chunk + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        cf[i] = upper_bound_i64(excl, 0, F, i * chunk) - 1;
}

// one warp-uniform grid-stride loop over first edges f
template <typename TT>
__global__ void __launch_bounds__(256, 8) k_level2(MatchArgs<TT> A, FRec<TT>* __restrict__ rec,
                                                int32_t* __restrict__ len2, int64_t* __restrict__ hs_a,
                                                int64_t* __restrict__ hs_hi) {
    const GraphDevT<TT>& G = A.G;
    extern __shared__ __align__(16) unsigned char smem_plans[];
    const QPlan* PL = stage_plans(A.plans, A.nq, smem_plans);
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Acc acc;
    acc_init(acc, smem_plans, A.nq);
    acc_zero(acc);
    const int64_t F = A.d_F ? *A.d_F : A.F;
    for (int64_t base = warp * 32; base < F; base += nwarps * 32) {
        int64_t f = base + lane;
        bool valid = f < F;
        int64_t wi = -1;
        // window of the warp's first edge (precomputed per 32 first edges, else one binary
        // search); lanes past its end gallop forward from it
        int64_t w0 = 0;
        if (A.blockwin) {
            w0 = __ldg(A.blockwin + (base >> 5));
        } else {
            if (lane == 0) {
                int64_t lo = 0, hi = A.NW;
                while (hi - lo > 1) {
                    int64_t mid = (lo + hi) >> 1;
                    if (__ldg(A.W.fbase + mid) <= base) lo = mid; else hi = mid;
                }
                w0 = lo;
            }
            w0 = __shfl_sync(kFull, w0, 0);
        }
        if (valid) {
            if (f < __ldg(A.W.fbase + w0) + __ldg(A.W.nfirst + w0)) {
                wi = w0;
            } else {
                int64_t lo = w0, hi = A.NW;   // last window whose fbase <= f
                for (int64_t step = 1;; step <<= 1) {
                    int64_t nx = lo + step;
                    if (nx >= A.NW) break;
                    if (__ldg(A.W.fbase + nx) > f) { hi = nx; break; }
                    lo = nx;
                }
                while (hi - lo > 1) {
                    int64_t mid = (lo + hi) >> 1;
                    if (__ldg(A.W.fbase + mid) <= f) lo = mid; else hi = mid;
                }
                wi = lo;
            }
        }
        // flush when any lane changes window
        if (__any_sync(kFull, valid && acc.win != wi)) {
            acc_flush_warp(acc, A.W.acc);
            if (valid) acc.win = wi;
        }
        if (!valid) continue;
        wi = TM_CHK_IDX(wi, A.NW, kChkWindow);
        const QPlan& Q = PL[TM_CHK_IDX(A.W.q[wi], A.nq, kChkWindow)];
        int64_t e1 = A.W.lo[wi] + (f - A.W.fbase[wi]);
        if (Q.full) e1 = __ldg(Q.perm + TM_CHK_IDX(e1, (int64_t)Q.b * G.m, kChkView));
        e1 = TM_CHK_IDX(e1, G.m, kChkView);
        int32_t s1, d1;
        int64_t t1;
        first_edge(G, Q.order, e1, s1, d1, t1);
        s1 = (int32_t)TM_CHK_IDX(s1, G.n, kChkNode);
        d1 = (int32_t)TM_CHK_IDX(d1, G.n, kChkNode);
        int64_t thi = first_thi(Q, A.W, wi, t1);
        int64_t len = 0, lo = 0, ha = 0, hh = 0;
        // a segment of a streamed graph owns the exact queries' first edges in [own_lo, own_hi)
        bool owned = t1 >= Q.own_lo && t1 < Q.own_hi;
        if (owned) acc.s(A_FIRST) += 1;
        if (owned && s1 != d1) {
            if (Q.l == 1) {
                acc.f[A_COUNT] += 1;
                if (Q.mode == TM_MODE_ESTIMATE) add_weight(acc, Q, 0);
            } else if (Q.ex23) {
                // two-node motif (Algorithm 2): for a last edge j in (t1, thi] the middle
                // edges are those of the middle pair with time in (t1, t_j), a difference of
                // two counts; exact counts sum it over j in O(1) from the prefix tables.
                // The last edges' range comes first: most first edges have none.
                const bool mid_rev = Q.ex23 & kEx23MidRev, last_rev = Q.ex23 & kEx23LastRev;
                int64_t pa = 0, pb = 0, own_ub = 0, ra = 0, rb = 0, rev_ub = 0;
                bool have_own = false, have_rev = false;
                auto own_side = [&]() {
                    if (Q.order == kOrdPair) {
                        int32_t pid = __ldg(G.pair_pid + e1);
                        pa = __ldg(G.pair_off + pid);
                        pb = __ldg(G.pair_off + pid + 1);
                        own_ub = gallop_ub(G.pair_t, e1 + 1, pb, t1);
                    } else {
                        pair_segment(G, s1, d1, pa, pb, false);   // e1 is one of the pair's edges
                        own_ub = upper_bound_i64(G.pair_t, pa, pb, t1);
                    }
                    have_own = true;
                };
                auto rev_side = [&]() {
                    if (pair_segment(G, d1, s1, ra, rb)) rev_ub = upper_bound_i64(G.pair_t, ra, rb, t1);
                    have_rev = true;
                };
                if (last_rev) rev_side(); else own_side();
                ha = last_rev ? rev_ub : own_ub;
                hh = thi > t1 ? gallop_ub(G.pair_t, ha, last_rev ? rb : pb, thi) : ha;
                if (hh > ha) {
                    if (mid_rev && !have_rev) rev_side();
                    if (!mid_rev && !have_own) own_side();
                    int64_t le2 = mid_rev ? rev_ub - ra : own_ub - pa;   // middle-pair edges at or before t1
                    if (Q.mode == TM_MODE_EXACT) {
                        const int64_t* S = mid_rev == last_rev ? G.ex_own : G.ex_rev;
                        int64_t sa = __ldg(S + ha);
                        acc.f[A_COUNT] += (unsigned long long)((__ldg(S + hh) - sa) - (hh - ha) * le2);
                        acc.s(A_LAST) += 1;
                        for (int i = 0; i < Q.nsub; i++) {   // exact queries at smaller spans
                            int64_t hi = gallop_ub(G.pair_t, ha, hh, t1 + Q.dsub[i]);
                            acc.s(A_X0 + i) += (unsigned long long)((__ldg(S + hi) - sa) - (hi - ha) * le2);
                        }
                        if (Q.nride) {
                            // estimates riding along need the last edges one by one, up to the
                            // latest end of a kept rider window holding t1
                            int64_t thr = t1;
                            for (int r = 0; r < Q.nride; r++) {
                                const QPlan& R = PL[Q.ride_q[r]];
                                const bool all_kept = R.q_mode == TM_Q_UNIFORM && R.p >= 1.0;
                                for (int k = 0; k < R.b; k++) {
                                    int64_t w, th;
                                    ride_window(R, k, t1, w, th);
                                    if (all_kept || A.W.kept[w]) thr = max(thr, th);
                                }
                            }
                            if (thr > t1) {
                                len = gallop_ub(G.pair_t, ha, hh, thr) - ha;   // items for the riders only
                                hh = le2;
                                acc.s(A_INST) += (unsigned long long)len;   // last edges read one by one
                            }
                        }
                    } else {
                        len = hh - ha;   // items: the last edges; k_match reads ha and le2
                        hh = le2;
                    }
                }
            } else {
                int32_t phi[2] = {s1, d1};
                const LevelPlan P = Q.lv[1];
                bool have_h = false;
                if (Q.hoist) {
                    // the closing pair is fixed by the first edge: find its range first, so
                    // first edges with no closing edge skip every other search
                    if (Q.order == kOrdPair) {
                        // the first edge's own pair: its entries after e1 up to thi
                        int64_t pend = __ldg(G.pair_off + __ldg(G.pair_pid + e1) + 1);
                        ha = gallop_ub(G.pair_t, e1 + 1, pend, t1);
                        hh = thi > t1 ? gallop_ub(G.pair_t, ha, pend, thi) : ha;
                    } else {
                        const LevelPlan L = Q.lv[Q.l - 1];
                        int64_t a0, b0;
                        if (thi > t1 && pair_segment(G, phi_get(phi, L.su), phi_get(phi, L.sv), a0, b0)) {
                            ha = upper_bound_i64(G.pair_t, a0, b0, t1);
                            hh = gallop_ub(G.pair_t, ha, b0, thi);
                        }
                    }
                    have_h = true;
                }
                if (have_h && hh == ha) {
                    len = 0;   // no closing edge in time: nothing else to look up
                } else if (Q.order == kOrdOut && P.view == kOut && P.su == 0) {
                    // e1 is entry e1 of out(s1): its candidates start right after it
                    int64_t b = __ldg(G.out_off + s1 + 1);
                    lo = gallop_ub(G.out_t, e1 + 1, b, t1);
                    len = thi > t1 ? gallop_ub(G.out_t, lo, b, thi) - lo : 0;
                } else if (Q.order == kOrdIn && P.view == kIn && P.sv == 1) {
                    int64_t b = __ldg(G.in_off + d1 + 1);
                    lo = gallop_ub(G.in_t, e1 + 1, b, t1);
                    len = thi > t1 ? gallop_ub(G.in_t, lo, b, thi) - lo : 0;
                } else {
                    level_range(G, P, phi, t1, thi, lo, len);
                }
                if (Q.rev && len > kRevMinLen) {
                    // candidates of the last edge given only its first-edge node (worth a
                    // search only when the second-edge range is long)
                    const LevelPlan L = Q.lv[2];
                    bool x_src = L.su == 2;
                    int32_t bn = x_src ? phi_get(phi, L.sv) : phi_get(phi, L.su);
                    const TT* ta = x_src ? G.in_t : G.out_t;
                    const int64_t* off = x_src ? G.in_off : G.out_off;
                    int64_t a = __ldg(off + bn), b = __ldg(off + bn + 1);
                    int64_t rlo = upper_bound_i64(ta, a, b, t1);
                    int64_t rlen = gallop_ub(ta, rlo, b, thi) - rlo;
                    if (rlen == 0) {
                        len = 0;                 // nothing can close an instance
                    } else if (rlen < len) {
                        lo = -1 - rlo;           // negative: items are last-edge candidates
                        len = rlen;
                    }
                }
                if (Q.hoist && len > 0) {
                    if (hh == ha) {
                        len = 0;                 // no closing edge in time: no instance starts here
                    } else if (Q.hrev && hh - ha < len) {
                        // fewer closing edges than second-edge candidates: the closing
                        // edges become the items; keep the second-edge range for counting
                        int64_t end1 = lo + len;
                        lo = -1 - lo;
                        len = hh - ha;
                        hh = end1;
                    }
                }
                if (Q.l == 2 && Q.mode == TM_MODE_EXACT) {
                    if (P.view == kPair) {
                        acc.f[A_COUNT] += len;
                        acc.s(A_LAST) += 1;
                        len = 0;
                    } else if (len > A.enum_threshold && P.view != kAll) {
                        acc.f[A_COUNT] += last_count_subtract(G, P, phi, len, t1, thi);
                        acc.s(A_LAST) += 1;
                        len = 0;
                    }
                }
            }
        }
        // (closing-side items, lo < 0, are checked where k_match decodes them)
        TM_CHK(len <= 0 || lo < 0 || lo + len <= G.m, kChkRange);
        len2[f] = (int32_t)len;   // a range inside one view: below 2^31
        if (len > 0) {            // the matcher reads these only for first edges with items
            FRec<TT> r;
            r.s1 = s1;
            r.d1 = d1;
            r.win = (int32_t)wi;
            r.q = A.W.q[wi];
            r.t1 = (TT)t1;
            r.thi = (TT)min(thi, (int64_t)std::numeric_limits<TT>::max());
            r.lo2 = lo;
            rec[f] = r;
            if (hs_a) {
                hs_a[f] = ha;
                hs_hi[f] = hh;
            }
        }
    }
    acc_flush_warp(acc, A.W.acc);
}

// Warp-cooperative expansion of motif edge D (0-based) for the 32 partial
// instances held by the lanes (valid ones have edges 0..D-1 matched).
// (ha, hh): the closing pair range when the query fixed it at the first edge.
template <typename TT, int D, int LMAX, int KMAX>
__device__ void expand(const MatchArgs<TT>& A, const QPlan* __restrict__ PL, bool valid, int32_t q, int64_t win,
                       int32_t (&phi)[KMAX], int64_t t1, int64_t tprev, int64_t thi, int64_t ha,
                       int64_t hh, Acc& acc) {
    const GraphDevT<TT>& G = A.G;
    int lane = threadIdx.x & 31;
    int64_t lo = 0, len = 0;
    int dir = 0;   // 1: this lane's candidates are the last edge's (two-sided closing)
    if (valid) {
        const QPlan& Q = PL[q];
        const LevelPlan P = Q.lv[D];
        if (D == Q.l - 1 && Q.hoist) {
            lo = upper_bound_i64(G.pair_t, ha, hh, tprev);
            len = hh - lo;
        } else {
            level_range(G, P, phi, tprev, thi, lo, len);
        }
        if constexpr (D + 2 <= LMAX) {
            if (D == Q.l - 2 && Q.rev2 && len > 0) {
                // edge D binds one new node x and the last edge joins x to a bound
                // node: take whichever side has fewer candidates in (tprev, thi]
                const LevelPlan L = Q.lv[Q.l - 1];
                int xl = P.bind_u ? P.su : P.sv;
                bool x_src = L.su == xl;
                int32_t bn = x_src ? phi_get(phi, L.sv) : phi_get(phi, L.su);
                const TT* ta = x_src ? G.in_t : G.out_t;
                const int64_t* off = x_src ? G.in_off : G.out_off;
                int64_t a = __ldg(off + bn), b = __ldg(off + bn + 1);
                int64_t rlo = upper_bound_i64(ta, a, b, tprev);
                int64_t rlen = gallop_ub(ta, rlo, b, thi) - rlo;
                if (rlen == 0) {
                    len = 0;
                } else if (rlen < len) {
                    lo = rlo;
                    len = rlen;
                    dir = 1;
                }
            }
        }
        if (D == Q.l - 1) {
            acc_switch(acc, win, A.W.acc);
            acc.s(A_LAST) += 1;
            if (Q.mode == TM_MODE_EXACT) {
                if (P.view == kPair) {
                    acc.f[A_COUNT] += len;
                    len = 0;
                } else if (len > A.enum_threshold && P.view != kAll) {
                    acc.f[A_COUNT] += last_count_subtract(G, P, phi, len, tprev, thi);
                    len = 0;
                }
            }
        }
    }
    int64_t incl = warp_incl_scan64(len);
    int64_t total = __shfl_sync(kFull, incl, 31);
    int64_t mystart = incl - len;
    for (int64_t base = 0; base < total; base += 32) {
        int64_t x = base + lane;
        bool has = x < total;
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            int64_t v = __shfl_sync(kFull, incl, o + step - 1);
            if (v <= x) o += step;
        }
        if (!has) o = 0;
        int32_t oq = __shfl_sync(kFull, q, o);
        int64_t ow = __shfl_sync(kFull, win, o);
        int64_t olo = __shfl_sync(kFull, lo, o);
        int64_t ost = __shfl_sync(kFull, mystart, o);
        int64_t ot1 = __shfl_sync(kFull, t1, o);
        int64_t othi = __shfl_sync(kFull, thi, o);
        int64_t oha = __shfl_sync(kFull, ha, o);
        int64_t ohh = __shfl_sync(kFull, hh, o);
        int odir = 0;
        int64_t otp = 0;
        if constexpr (D + 2 <= LMAX) {
            odir = __shfl_sync(kFull, dir, o);
            otp = __shfl_sync(kFull, tprev, o);
        }
        int32_t ophi[KMAX];
#pragma unroll
        for (int i = 0; i < KMAX; i++) ophi[i] = __shfl_sync(kFull, phi[i], o);
        bool ok = false, deeper = false;
        int64_t tc = 0;
        if (has) {
            const QPlan& Q = PL[oq];
            const LevelPlan P = Q.lv[D];
            acc_switch(acc, ow, A.W.acc);
            if (odir) {
                // last-edge candidate (x, t_l): count the edge-D candidates in (tprev, t_l)
                const LevelPlan L = Q.lv[Q.l - 1];
                int xl = P.bind_u ? P.su : P.sv;
                bool x_src = L.su == xl;
                int64_t c = TM_CHK_IDX(olo + (x - ost), G.m, kChkView);
                int32_t xv = x_src ? __ldg(G.in_nbr + c) : __ldg(G.out_nbr + c);
                int64_t tl = x_src ? __ldg(G.in_t + c) : __ldg(G.out_t + c);
                acc.s(A_CAND) += 1;
                if (!phi_has(ophi, P.nb, xv)) {
                    int32_t mu = P.bind_u ? xv : phi_get(ophi, P.su);
                    int32_t mv = P.bind_v ? xv : phi_get(ophi, P.sv);
                    int64_t cnt = pair_count(G, mu, mv, otp, tl - 1);
                    acc.s(A_LAST) += 1;
                    if (cnt) {
                        acc.f[A_COUNT] += cnt;
                        if (Q.mode == TM_MODE_ESTIMATE) add_weight_n(acc, Q, tl - ot1, (unsigned long long)cnt);
                    }
                }
            } else {
                int32_t s, d;
                read_cand(G, P, ophi, TM_CHK_IDX(olo + (x - ost), G.m, kChkView), s, d, tc);
                ok = check_bind(P, ophi, s, d);
                if (D == Q.l - 1) {
                    acc.s(A_INST) += 1;
                    if (ok) {
                        acc.f[A_COUNT] += 1;
                        if (Q.mode == TM_MODE_ESTIMATE) add_weight(acc, Q, tc - ot1);
                    }
                } else {
                    acc.s(A_CAND) += 1;
                    deeper = ok;
                    if constexpr (D + 2 <= LMAX) {
                        const LevelPlan L = Q.lv[Q.l - 1];
                        if (ok && D == Q.l - 2 && Q.mode == TM_MODE_EXACT && L.view == kPair && !Q.hoist) {
                            // close here: the last edge counted by range length
                            acc.f[A_COUNT] += pair_count(G, phi_get(ophi, L.su), phi_get(ophi, L.sv), tc, othi);
                            acc.s(A_LAST) += 1;
                            deeper = false;
                        }
                    }
                }
            }
        }
        if constexpr (D + 1 < LMAX) {
            if (__any_sync(kFull, deeper))
                expand<TT, D + 1, LMAX, KMAX>(A, PL, deeper, oq, ow, ophi, ot1, tc, othi, oha, ohh, acc);
        }
    }
}

// OCC: resident 256-thread blocks per SM the register allocation must allow
// (three-edge motifs: 4 without spills, 6 with spilled registers; four-edge motifs: 1 leaves
// the compiler 118 registers, 4 caps them at 64 with spills -- the autotuner picks)
// EXPAND = false leaves out the warp-cooperative expansion of deeper motif edges, for batches
// whose items all end at their second edge (every query exact with the last edge between two
// bound nodes, two-node, riding along, or of at most two edges): the code the hot loop does
// not run still takes registers, and without it the 3-cycle enumeration of the benchmark
// batch runs 1.50 -> 1.32 ms
template <typename TT, int LMAX, int KMAX, int OCC = (LMAX <= 3 ? 4 : 1), bool EXPAND = true>
__global__ void __launch_bounds__(256, OCC) k_match(MatchArgs<TT> A) {
    const GraphDevT<TT>& G = A.G;
    extern __shared__ __align__(16) unsigned char smem_plans[];
    const QPlan* PL = stage_plans(A.plans, A.nq, smem_plans);
    int lane = threadIdx.x & 31;
    int64_t W2 = *A.d_W2;
    const int64_t F = A.d_F ? *A.d_F : A.F;
    Acc acc;
    acc_init(acc, smem_plans, A.nq);
    acc_zero(acc);
    for (;;) {
        unsigned long long c0u = 0;
        if (lane == 0) c0u = atomicAdd(A.counter, (unsigned long long)A.chunk);
        int64_t c0 = (int64_t)__shfl_sync(kFull, c0u, 0);
        if (c0 >= W2) break;
        int64_t c1 = min(c0 + A.chunk, W2);
        int64_t fb = 0, fe = 0;
        int64_t ci = c0 / A.chunk;
        if (A.chunkf && ci + 1 < A.nchunkf) {
            // first edges of this chunk's first item and of the next chunk's (a bound on
            // the last item's: first edges in between have no items below c1)
            fb = __ldg(A.chunkf + ci);
            fe = __ldg(A.chunkf + ci + 1);
        } else {
            if (lane < 2) {
                int64_t key = lane == 0 ? c0 : c1 - 1;
                fb = upper_bound_i64(A.excl, 0, F, key) - 1;
            }
            fe = __shfl_sync(kFull, fb, 1);
            fb = __shfl_sync(kFull, fb, 0);
        }
        int64_t fcur = fb;   // first edge of the round's first item
        for (int64_t base = c0; base < c1; base += 32) {
            int64_t w = base + lane;
            bool valid = w < c1;
            // first edges fcur .. fcur+31 in registers; each lane finds its item's
            // first edge among them by a shuffle search (falls back past them)
            int64_t ex = (fcur + lane <= fe) ? __ldg(A.excl + fcur + lane) : INT64_MAX;
            int k = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                int64_t v = __shfl_sync(kFull, ex, k + step - 1);
                if (v <= w) k += step;
            }
            int64_t last32 = __shfl_sync(kFull, ex, 31);
            int64_t fw = fcur + k - 1;
            if (valid && last32 <= w) fw = upper_bound_i64(A.excl, fcur + 31, fe + 1, w) - 1;
            fcur = __shfl_sync(kFull, fw, 31);
            int32_t q = 0;
            int64_t win = -1, t1 = 0, thi = 0, tc = 0, ha = 0, hh = 0;
            int32_t phi[KMAX];
#pragma unroll
            for (int i = 0; i < KMAX; i++) phi[i] = -1;
            bool deeper = false;
            int64_t rx = 0;   // this item's deferred rider / smaller-span record (rn != 0)
            int32_t rn = 0;
            if (valid) {
                int64_t f = TM_CHK_IDX(fw, F, kChkQueue);
                const FRec<TT> r = A.rec[f];
                win = TM_CHK_IDX(r.win, A.NW, kChkWindow);
                q = (int32_t)TM_CHK_IDX(r.q, A.nq, kChkWindow);
                const QPlan& Q = PL[q];
                phi[0] = r.s1;
                phi[1] = r.d1;
                t1 = (int64_t)r.t1;
                thi = (int64_t)r.thi;
                int64_t l2 = r.lo2;
                if (Q.ex23) {
                    // two-node motif: item = last edge j; its middle edges number
                    // (middle-pair edges before t_j) - (those at or before t1)
                    const bool mid_rev = Q.ex23 & kEx23MidRev, last_rev = Q.ex23 & kEx23LastRev;
                    const int64_t* S = mid_rev == last_rev ? G.ex_own : G.ex_rev;
                    int64_t j = TM_CHK_IDX(A.hs_a[f] + (w - A.excl[f]), G.m, kChkView);
                    int64_t t3 = __ldg(G.pair_t + j);
                    int64_t cnt = (__ldg(S + j + 1) - __ldg(S + j)) - A.hs_hi[f];
                    if (Q.mode == TM_MODE_EXACT) {
                        // the query's own count came from the tables: the items are its riders'
                        if (cnt > 0 && Q.nride) { rx = t3; rn = -(int32_t)cnt; }
                    } else {
                        acc_switch(acc, win, A.W.acc);
                        acc.s(A_CAND) += 1;
                        acc.s(A_LAST) += 1;
                        if (cnt > 0) {
                            acc.f[A_COUNT] += cnt;
                            add_weight_n(acc, Q, t3 - t1, (unsigned long long)cnt);
                        }
                    }
                } else if (l2 < 0 && Q.hoist) {
                    // closing edge e3 of the first edge's pair: count the valid second
                    // edges with time in (t1, t3)
                    const LevelPlan L = Q.lv[2];
                    const LevelPlan M1 = Q.lv[1];
                    int64_t lo1 = -1 - l2, end1 = A.hs_hi[f], ha0 = A.hs_a[f];
                    int64_t p3 = TM_CHK_IDX(ha0 + (w - A.excl[f]), G.m, kChkView);
                    int64_t t3 = __ldg(G.pair_t + p3);
                    acc_switch(acc, win, A.W.acc);
                    acc.s(A_CAND) += 1;
                    acc.s(A_LAST) += 1;
                    const TT* t1v = M1.view == kPair ? G.pair_t : M1.view == kOut ? G.out_t : G.in_t;
                    int64_t cnt = upper_bound_i64(t1v, lo1, end1, t3 - 1) - lo1;
                    if (M1.view != kPair) {
                        // second edges whose new node would be a first-edge node are invalid
                        int32_t bn = M1.view == kOut ? phi_get(phi, M1.su) : phi_get(phi, M1.sv);
                        int32_t hu = phi_get(phi, L.su), hv = phi_get(phi, L.sv);
#pragma unroll
                        for (int y = 0; y < 2; y++) {
                            int32_t xs = M1.view == kOut ? bn : phi[y];
                            int32_t xd = M1.view == kOut ? phi[y] : bn;
                            if (xs == hu && xd == hv) cnt -= lower_bound_i64(G.pair_t, ha0, p3, t3) - ha0;
                            else if (xs != xd || G.loops) cnt -= pair_count(G, xs, xd, t1, t3 - 1);
                        }
                    }
                    if (cnt) {
                        acc.f[A_COUNT] += cnt;
                        if (Q.mode == TM_MODE_ESTIMATE) add_weight_n(acc, Q, t3 - t1, (unsigned long long)cnt);
                        if (Q.nsub | Q.nride) { rx = t3; rn = -(int32_t)cnt; }
                    }
                } else {
                // Two item kinds end in a count of one pair's entries in a time range: a
                // closing-edge candidate e3 = (x, t3) counts second edges in (t1, t3); a
                // second-edge candidate of an exact three-edge query counts closing edges in
                // (tc, thi].  Their pair lookups go through one call site, so that a warp
                // holding both kinds waits on one chain of dependent loads, not two.
                int kind = 0;   // 1: closing-edge candidate, 2: second edge closed by range
                int32_t pu = 0, pv = 0;
                int64_t plo = 0, pthi = 0, t3 = 0;
                bool ok = false;
                acc_switch(acc, win, A.W.acc);
                acc.s(A_CAND) += 1;
                if (l2 < 0) {
                    const LevelPlan L = Q.lv[2];
                    const LevelPlan M1 = Q.lv[1];
                    int64_t c = TM_CHK_IDX((-1 - l2) + (w - A.excl[f]), G.m, kChkView);
                    bool x_src = L.su == 2;
                    int32_t x = x_src ? __ldg(G.in_nbr + c) : __ldg(G.out_nbr + c);
                    t3 = x_src ? __ldg(G.in_t + c) : __ldg(G.out_t + c);
                    if (x != phi[0] && x != phi[1]) {
                        kind = 1;
                        pu = M1.su == 2 ? x : phi_get(phi, M1.su);
                        pv = M1.sv == 2 ? x : phi_get(phi, M1.sv);
                        plo = t1;
                        pthi = t3 - 1;
                    }
                } else {
                    const LevelPlan P = Q.lv[1];
                    int32_t s, d;
                    read_cand(G, P, phi, TM_CHK_IDX(l2 + (w - A.excl[f]), G.m, kChkView), s, d, tc);
                    ok = check_bind(P, phi, s, d);
                    if (Q.hoist) {
                        ha = A.hs_a[f];
                        hh = A.hs_hi[f];
                    }
                    const LevelPlan L = Q.lv[2];
                    if (Q.l == 2) {
                        acc.s(A_CAND) -= 1;
                        acc.s(A_INST) += 1;
                        if (ok) {
                            acc.f[A_COUNT] += 1;
                            if (Q.mode == TM_MODE_ESTIMATE) add_weight(acc, Q, tc - t1);
                        }
                    } else if (ok && Q.l == 3 && Q.mode == TM_MODE_EXACT && L.view == kPair) {
                        kind = 2;
                        pu = phi_get(phi, L.su);
                        pv = phi_get(phi, L.sv);
                        plo = tc;
                        pthi = thi;
                    } else {
                        deeper = ok;
                    }
                }
                // the pair lookup: the hoisted closing range is already known
                int64_t clo = 0, chi = 0;
                if (kind == 2 && Q.hoist) {
                    clo = upper_bound_i64(G.pair_t, ha, hh, tc);
                    chi = hh;
                } else if (kind) {
                    pair_range(G, pu, pv, plo, pthi, clo, chi);
                }
                if (kind == 1) {
                    int64_t cnt = chi - clo;
                    acc.s(A_LAST) += 1;
                    if (cnt) {
                        acc.f[A_COUNT] += cnt;
                        if (Q.mode == TM_MODE_ESTIMATE) add_weight_n(acc, Q, t3 - t1, (unsigned long long)cnt);
                        if (Q.nsub | Q.nride) { rx = t3; rn = -(int32_t)cnt; }
                    }
                } else if (kind == 2) {
                    // close the instance here: the last edge is counted by range length
                    acc.f[A_COUNT] += chi - clo;
                    acc.s(A_LAST) += 1;
                    if ((Q.nsub | Q.nride) && chi > clo) { rx = clo; rn = (int32_t)(chi - clo); }
                }
                }
            }
            // the round's deferred records, appended with one atomic per warp
            const unsigned rm = __ballot_sync(kFull, rn != 0);
            if (rm) {
                unsigned long long rb = 0;
                if (lane == 0) rb = atomicAdd(A.rcount, (unsigned long long)__popc(rm));
                rb = __shfl_sync(kFull, rb, 0) + __popc(rm & ((1u << lane) - 1u));
                if (rn && (int64_t)rb < A.rcap) {
                    RideRec<TT> rr;
                    rr.x = rx;
                    rr.t1 = (TT)t1;
                    rr.tc = (TT)tc;
                    rr.q = q;
                    rr.n = rn;
                    A.rrec[rb] = rr;
                }
            }
            if constexpr (EXPAND) {
                if (__any_sync(kFull, deeper))
                    expand<TT, 2, LMAX, KMAX>(A, PL, deeper, q, win, phi, t1, tc, thi, ha, hh, acc);
            } else {
                TM_CHK(!deeper, kChkQueue);   // the host's choice of EXPAND = false must hold
            }
        }
        acc_flush_warp(acc, A.W.acc);
    }
    acc_flush_warp(acc, A.W.acc);
}

// Rider sums of one warp of k_ride records that all belong to exact query Q: every lane weighs
// its own record per rider and shift, and when the lanes with instances share one window (the
// usual case: neighbouring records come from the same first edges) their sums are added once,
// by one lane, instead of 32 times to the same shared-memory slot.
template <typename TT>
__device__ __forceinline__ void ride_warp(const QPlan* __restrict__ PL, const QPlan& Q,
                                          const int32_t* __restrict__ kept, unsigned long long* acc,
                                          const TT* __restrict__ ta, bool valid, const RideRec<TT>& r) {
    const int lane = threadIdx.x & 31;
    const int64_t t1 = (int64_t)r.t1, tc = (int64_t)r.tc;
    const bool at = r.n < 0;
    unsigned long long nread = 0;
    for (int rr = 0; rr < Q.nride; rr++) {
        const QPlan& R = PL[Q.ride_q[rr]];
        const bool all_kept = R.q_mode == TM_Q_UNIFORM && R.p >= 1.0;   // no keep flag to read
        for (int k = 0; k < R.b; k++) {
            unsigned long long cnt = 0, wl = 0, wh = 0;
            int64_t w = -1;
            if (valid) {
                int64_t thi;
                ride_window(R, k, t1, w, thi);
                if (at) {
                    const int64_t t3 = r.x;   // -n instances closed at t3
                    if (t3 - t1 <= R.delta && t3 <= thi && (all_kept || kept[w])) {
                        cnt = (unsigned long long)(-(int64_t)r.n);
                        ride_weight(R, t3 - t1, cnt, wl, wh);
                    }
                } else if (t1 + R.delta > tc && thi > tc && (all_kept || kept[w])) {
                    for (int64_t x = r.x; x < r.x + r.n; x++) {
                        const int64_t t3 = (int64_t)ta[x];
                        if (t3 > thi) break;   // times increase
                        unsigned long long l, h;
                        ride_weight(R, t3 - t1, 1, l, h);
                        const unsigned long long y = wl + l;
                        wh += h + (y < wl ? 1ull : 0ull);
                        wl = y;
                        cnt++;
                    }
                    nread = max(nread, cnt);
                }
            }
            const unsigned hm = __ballot_sync(kFull, cnt != 0);
            if (!hm) continue;
            const int first = __ffs(hm) - 1;
            const int64_t w0 = __shfl_sync(kFull, w, first);
            if (__all_sync(kFull, cnt == 0 || w == w0)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    cnt += __shfl_xor_sync(kFull, cnt, o);
                    const unsigned long long l2 = __shfl_xor_sync(kFull, wl, o);
                    const unsigned long long h2 = __shfl_xor_sync(kFull, wh, o);
                    const unsigned long long y = wl + l2;
                    wh = wh + h2 + (y < wl ? 1ull : 0ull);
                    wl = y;
                }
                if (lane == first) ride_add(acc, w0, cnt, wl, wh);
            } else if (cnt) {
                ride_add(acc, w, cnt, wl, wh);
            }
        }
    }
    // entries read one by one: per record the most any rider shift read, summed over the warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nread += __shfl_xor_sync(kFull, nread, o);
    if (lane == 0 && nread) ride_add(acc, (int64_t)(kInstKey | (unsigned long long)Q.win_base), nread, 0, 0);
}

// The deferred half of the exact queries that carry riders or smaller spans: one thread per
// record of k_match (grid-stride, every lane busy), adding the smaller spans' counts to the
// query's window and each rider's weighted instances to the rider's kept windows, exactly as
// the matcher would have on the spot (integer sums: the order does not matter).
template <typename TT>
__global__ void __launch_bounds__(256) k_ride(MatchArgs<TT> A) {
    const GraphDevT<TT>& G = A.G;
    extern __shared__ __align__(16) unsigned char smem_plans[];
    const QPlan* PL = stage_plans(A.plans, A.nq, smem_plans);
    Acc acc;
    acc_init(acc, smem_plans, A.nq);
    acc_zero(acc);
    RideTab* tab = ride_tab();
    for (int i = threadIdx.x; i < kRideTab; i += blockDim.x) {
        tab->key[i] = kTabFree;
        tab->cnt[i] = tab->lo[i] = tab->hi[i] = 0;
    }
    __syncthreads();
    const int64_t nrec = min((int64_t)*A.rcount, A.rcap);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps step together, so that the accumulator flushes see every lane
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t end = (nrec + 31) / 32 * 32;
    for (int64_t i = start; i < end; i += stride) {
        const bool valid = i < nrec;
        RideRec<TT> r = {};
        int64_t win = -1;
        int32_t q = -1;
        if (valid) {
            r = A.rrec[i];
            q = (int32_t)TM_CHK_IDX(r.q, A.nq, kChkWindow);
            win = PL[q].win_base;
        }
        if (__any_sync(kFull, valid && acc.win != win)) {
            acc_flush_warp(acc, A.W.acc);
            if (valid) acc.win = win;
        }
        if (valid) {
            const QPlan& Q = PL[q];
            const int64_t t1 = (int64_t)r.t1;
            if (r.n < 0) {
                // (a two-node query's smaller spans were counted from the pair tables in k_level2;
                // its records are for the riders only)
                if (Q.nsub && !Q.ex23) add_sub_at(acc, Q, t1, r.x, (unsigned long long)(-(int64_t)r.n));
            } else {
                r.x = TM_CHK_IDX(r.x, G.m, kChkView);
                TM_CHK(r.x + r.n <= G.m, kChkRange);
#ifdef TM_CHECKED
                if (r.x + r.n > G.m) r.n = 0;
#endif
                if (Q.nsub) add_sub_range(acc, Q, G.pair_t, r.x, r.x + r.n, t1);
            }
        }
        // riders: warp by warp when the warp's records belong to one query (the valid lanes are
        // a prefix of the warp, so lane 0 holds one), else lane by lane
        const int32_t q0 = __shfl_sync(kFull, q, 0);
        const bool uniform = __all_sync(kFull, !valid || q == q0);
        if (uniform && q0 >= 0) {
            if (PL[q0].nride) ride_warp(PL, PL[q0], A.W.kept, A.W.acc, G.pair_t, valid, r);
        } else if (!uniform && valid && PL[q].nride) {
            const QPlan& Q = PL[q];
            if (r.n < 0) ride_at(PL, Q, A.W.kept, A.W.acc, (int64_t)r.t1, r.x, (unsigned long long)(-(int64_t)r.n));
            else ride_range(PL, Q, A.W.kept, A.W.acc, G.pair_t, r.x, r.x + r.n, (int64_t)r.t1, (int64_t)r.tc);
        }
    }
    acc_flush_warp(acc, A.W.acc);
    __syncthreads();
    for (int i = threadIdx.x; i < kRideTab; i += blockDim.x) {
        const unsigned long long key = tab->key[i];
        if (key == kTabFree) continue;
        if (key & kInstKey) {
            atomicAdd(A.W.acc + (key & ~kInstKey) * A_N + A_INST, tab->cnt[i]);
            continue;
        }
        unsigned long long* p = A.W.acc + (int64_t)key * A_N;
        if (tab->cnt[i]) atomicAdd(p + A_COUNT, tab->cnt[i]);
        atomic_add_u128(p + A_WLO, tab->lo[i], tab->hi[i]);
    }
}

// Windows of one shift that a block of k_fold_shift sums: a query's shifts are cut into
// fold_slices(J) slices of whole windows, a function of the query alone, so that its
// result does not depend on the batch it runs in.
constexpr int kFoldThreads = 256;
constexpr int kFoldMaxSlices = 32;
__host__ __device__ inline int fold_slices(int64_t nwin) {
    int64_t s = (nwin + 8 * kFoldThreads - 1) / (8 * kFoldThreads);
    return (int)(s < 1 ? 1 : (s > kFoldMaxSlices ? kFoldMaxSlices : s));
}

// Fold, first half: block (query, shift k, slice) sums the kept windows of its slice —
// counts and work counters as integers, the Q64 weight sum W_j as a 128-bit integer, and
// the doubles sum_j W_j / q_j (the shift's Z_k when q_j varies, Algorithm 1) and
// sum_j W_j^2 (1 - q_j) / q_j^2 (Lemma 4.4) — into part[part_base + k * slices + slice].
// The grid's y extent is capped at the hardware limit; a block then also takes the shifts
// k + gridDim.y, k + 2 gridDim.y, ... (a loop that is uniform across the block).
__global__ void __launch_bounds__(kFoldThreads) k_fold_shift(const QPlan* __restrict__ plans, WinDev W,
                                                             ShiftSums* __restrict__ part) {
    const QPlan& Q = plans[blockIdx.x];
    const int sl = blockIdx.z;
    const int nsh = Q.l <= 0 ? 0 : (Q.mode == TM_MODE_EXACT ? 1 : Q.b);
    const int64_t nwin = Q.mode == TM_MODE_EXACT ? 1 : Q.J;
    const int ns = fold_slices(nwin);
    if (sl >= ns) return;
    __shared__ ShiftSums sh[kFoldThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = blockIdx.y; k < nsh; k += gridDim.y) {
        unsigned long long c[6] = {0, 0, 0, 0, 0, 0};   // count, first, cand, last, inst, kept
        unsigned long long wlo = 0, whi = 0;
        double zq = 0.0, vq = 0.0;
        for (int64_t r = (int64_t)sl * kFoldThreads + threadIdx.x; r < nwin; r += (int64_t)ns * kFoldThreads) {
            int64_t w = Q.win_base + (int64_t)k * nwin + r;
            if (!W.kept[w]) continue;
            const unsigned long long* a = W.acc + w * A_N;
            c[0] += a[A_COUNT];
            c[1] += a[A_FIRST];
            c[2] += a[A_CAND];
            c[3] += a[A_LAST];
            c[4] += a[A_INST];
            c[5] += 1;
            unsigned long long x = wlo + a[A_WLO];
            whi += a[A_WHI] + (x < wlo ? 1ull : 0ull);
            wlo = x;
            double y = (double)a[A_WHI] + (double)a[A_WLO] * 0x1.0p-64;
            double qj = W.qj[w];
            if (Q.q_mode == TM_Q_EDGES) zq += y / qj;
            vq += y * y * (1.0 - qj) / (qj * qj);
        }
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int i = 0; i < 6; i++) c[i] += __shfl_xor_sync(kFull, c[i], o);
            unsigned long long l2 = __shfl_xor_sync(kFull, wlo, o);
            unsigned long long h2 = __shfl_xor_sync(kFull, whi, o);
            unsigned long long x = wlo + l2;
            whi = whi + h2 + (x < wlo ? 1ull : 0ull);
            wlo = x;
            zq += __shfl_xor_sync(kFull, zq, o);
            vq += __shfl_xor_sync(kFull, vq, o);
        }
        if (lane == 0) {
            ShiftSums& o = sh[wid];
            o.count = c[0]; o.first = c[1]; o.cand = c[2]; o.last = c[3]; o.inst = c[4]; o.kept = c[5];
            o.wlo = wlo; o.whi = whi; o.zq = zq; o.vq = vq;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ShiftSums t = sh[0];
            for (int ww = 1; ww < kFoldThreads / 32; ww++) add_shift_sums(t, sh[ww]);
            part[Q.part_base + (int64_t)k * ns + sl] = t;
        }
        __syncthreads();   // sh is written again by the next shift
    }
}

// Fold, second half: one thread per query adds its slices in order, then its shifts in
// order: Z_k, their mean (the estimate of Algorithm 1), the mean variance estimate and
// the spread of the Z_k (Welford).
__global__ void k_fold_final(const QPlan* __restrict__ plans, int nq, WinDev W, const ShiftSums* __restrict__ part,
                             tm_result* __restrict__ res, ShiftSums* __restrict__ sums,
                             unsigned long long* __restrict__ subc) {
    int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    const QPlan& Q = plans[qi];
    const int nsh = Q.l <= 0 ? 0 : (Q.mode == TM_MODE_EXACT ? 1 : Q.b);
    const int ns = fold_slices(Q.mode == TM_MODE_EXACT ? 1 : Q.J);
    double zsum = 0.0, vsum = 0.0, wmean = 0.0, wm2 = 0.0;
    ShiftSums tot = {};
    int overflow = 0;
    for (int k = 0; k < nsh; k++) {
        const ShiftSums* pk = part + Q.part_base + (int64_t)k * ns;
        ShiftSums u = pk[0];
        for (int x = 1; x < ns; x++) add_shift_sums(u, pk[x]);
        if (sums) sums[Q.sum_base + k] = u;
        if (u.whi >= (1ull << 63) || u.count >= (1ull << 63)) overflow = 1;
        add_shift_sums(tot, u);
        double Wd = (double)u.whi + (double)u.wlo * 0x1.0p-64;
        double zk = Q.q_mode == TM_Q_EDGES ? u.zq : Wd / Q.p;
        zsum += zk;
        vsum += u.vq;
        double dz = zk - wmean;
        wmean += dz / (k + 1);
        wm2 += dz * (zk - wmean);
    }
    if (subc) {
        // counts of the exact queries at smaller spans (one window: the whole graph)
        const unsigned long long* a = W.acc + Q.win_base * A_N;
        for (int i = 0; i < kMaxSub; i++) subc[qi * kMaxSub + i] = (Q.l > 0 && i < Q.nsub) ? a[A_X0 + i] : 0;
    }
    tm_result r;
    memset(&r, 0, sizeof(r));
    r.status = Q.l <= 0 ? -1 : (overflow ? TM_EOVERFLOW : TM_OK);
    r.count = (int64_t)tot.count;
    if (Q.mode == TM_MODE_EXACT) {
        r.estimate = (double)tot.count;
        r.windows = 1;
        r.windows_kept = 1;
        r.var_hat = 0.0;
        r.p_used = 1.0;
    } else {
        r.estimate = nsh ? zsum / nsh : 0.0;
        r.windows = (int64_t)nsh * (Q.wclamp ? Q.J_all : Q.J);
        r.windows_kept = Q.wclamp ? (int64_t)nsh * Q.J_all : (int64_t)tot.kept;
        r.var_hat = nsh ? vsum / nsh : 0.0;
        r.shift_var = nsh >= 2 ? wm2 / (nsh - 1) : 0.0;
        r.p_used = Q.p;
    }
    r.first_edges = (int64_t)tot.first;
    r.cand_edges = (int64_t)tot.cand;
    r.last_ranges = (int64_t)tot.last;
    r.inst_read = (int64_t)tot.inst;
    res[qi] = r;
}

// the fold's partial records: part_base of every plan (a query's shifts times its slices,
// one after another); returns the total and, through smax, the most slices of a query
int64_t fold_parts(std::vector<QPlan>& hp, int& smax) {
    int64_t n = 0;
    smax = 1;
    for (QPlan& P : hp) {
        P.part_base = n;
        if (P.l <= 0) continue;
        int ns = fold_slices(P.mode == TM_MODE_EXACT ? 1 : P.J);
        smax = std::max(smax, ns);
        n += (int64_t)(P.mode == TM_MODE_EXACT ? 1 : P.b) * ns;
    }
    return std::max<int64_t>(n, 1);
}

constexpr int kMaxGridY = 65535;

// both halves of the fold on st
void launch_fold(const QPlan* dplans, int nq, int bmax, int smax, const WinDev& W, ShiftSums* part,
                 tm_result* dres, ShiftSums* sums, unsigned long long* subc, cudaStream_t st) {
    unsigned gy = (unsigned)std::min(std::max(bmax, 1), kMaxGridY);
    k_fold_shift<<<dim3((unsigned)nq, gy, (unsigned)smax), kFoldThreads, 0, st>>>(dplans, W, part);
    k_fold_final<<<(unsigned)((nq + 63) / 64), 64, 0, st>>>(dplans, nq, W, part, dres, sums, subc);
    count_launch(2);
}

// the persistent matcher for a batch whose deepest motif has lmax edges on kmax nodes: the
// instantiation whose register budget fits the tuning's blocks per SM
// a lane can go deeper than its second edge: a query of three or more edges, not two-node, not
// riding along, that is an estimate (it reads its last edges one by one), has four or more
// edges, or ends on an edge with a new node
bool plan_expands(const QPlan& P) {
    if (P.l < 3 || P.riding || P.ex23) return false;
    return P.l >= 4 || P.mode != TM_MODE_EXACT || P.lv[P.l - 1].view != kPair;
}

template <typename TT>
void launch_match(const MatchArgs<TT>& A, int lmax, int kmax, const Tuning& tu, int nsm, cudaStream_t st,
                  bool expand) {
    const int bps = tu.blocks_per_sm, bt = tu.block_threads;
    const unsigned gm = (unsigned)(nsm * bps);
    const size_t sm = match_smem_bytes(A.nq, bt);
    if (lmax <= 3 && kmax <= 4 && !expand) {
        if (bps >= 6) k_match<TT, 3, 4, 6, false><<<gm, bt, sm, st>>>(A);
        else k_match<TT, 3, 4, 4, false><<<gm, bt, sm, st>>>(A);
    } else if (lmax <= 3 && kmax <= 4 && bps >= 6) k_match<TT, 3, 4, 6><<<gm, bt, sm, st>>>(A);
    else if (lmax <= 3 && kmax <= 4) k_match<TT, 3, 4><<<gm, bt, sm, st>>>(A);
    else if (lmax <= 4 && kmax <= 4 && bps >= 4) k_match<TT, 4, 4, 4><<<gm, bt, sm, st>>>(A);
    else if (lmax <= 4 && kmax <= 4) k_match<TT, 4, 4><<<gm, bt, sm, st>>>(A);
    else if (lmax <= 4) k_match<TT, 4, TM_K_MAX><<<gm, bt, sm, st>>>(A);
    else k_match<TT, TM_L_MAX, TM_K_MAX><<<gm, bt, sm, st>>>(A);
    count_launch();
}

// ------------------------------------------------------- plain baseline K10
template <typename TT, int D, int LMAX>
__device__ int64_t plain_dfs(const GraphDevT<TT>& G, const QPlan& Q, int32_t (&phi)[TM_K_MAX],
                             int64_t tprev, int64_t thi) {
    const LevelPlan P = Q.lv[D];
    int64_t lo, len;
    level_range(G, P, phi, tprev, thi, lo, len);
    if (D == Q.l - 1 && P.view == kPair) return len;
    int64_t c = 0;
    for (int64_t i = 0; i < len; i++) {
        int32_t s, d;
        int64_t tc;
        int32_t nphi[TM_K_MAX];
#pragma unroll
        for (int z = 0; z < TM_K_MAX; z++) nphi[z] = phi[z];
        read_cand(G, P, nphi, lo + i, s, d, tc);
        if (!check_bind(P, nphi, s, d)) continue;
        if (D == Q.l - 1) {
            c += 1;
        } else if constexpr (D + 1 < LMAX) {
            c += plain_dfs<TT, D + 1, LMAX>(G, Q, nphi, tc, thi);
        }
    }
    return c;
}

template <typename TT>
__global__ void k_plain(GraphDevT<TT> G, const QPlan* __restrict__ plan, unsigned long long* out) {
    const QPlan& Q = *plan;
    unsigned long long c = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < G.m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t s1 = G.src[e], d1 = G.dst[e];
        if (s1 == d1) continue;
        if (Q.l == 1) { c += 1; continue; }
        int32_t phi[TM_K_MAX];
#pragma unroll
        for (int i = 0; i < TM_K_MAX; i++) phi[i] = -1;
        phi[0] = s1;
        phi[1] = d1;
        int64_t t1 = (int64_t)G.t[e];
        c += (unsigned long long)plain_dfs<TT, 1, TM_L_MAX>(G, Q, phi, t1, t1 + Q.delta);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// --------------------------------------------------------------- host side
size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int validate_query_t(int64_t t_max, const tm_query& q, std::string& why) {
    if (!q.motif) { why = "motif is NULL"; return TM_EINVAL; }
    if (q.delta < 0) { why = "delta < 0"; return TM_EINVAL; }
    if (q.delta >= ((int64_t)1 << 61)) { why = "delta >= 2^61"; return TM_EINVAL; }
    if (q.mode != TM_MODE_EXACT && q.mode != TM_MODE_ESTIMATE) { why = "bad mode"; return TM_EINVAL; }
    if (q.mode == TM_MODE_ESTIMATE) {
        if (q.delta < 1) { why = "estimate needs delta >= 1"; return TM_EINVAL; }
        if (q.c < 1) { why = "c < 1"; return TM_EINVAL; }
        if (q.b < 1 || q.b > (1 << 20)) { why = "b outside [1, 2^20]"; return TM_EINVAL; }
        if (q.q_mode != TM_Q_UNIFORM && q.q_mode != TM_Q_EDGES && q.q_mode != TM_Q_AUTO) {
            why = "bad q_mode";
            return TM_EINVAL;
        }
        if (q.q_mode == TM_Q_AUTO && !(q.p > 0.0 && q.p < 1.0)) { why = "target error outside (0, 1)"; return TM_EINVAL; }
        if (q.q_mode == TM_Q_UNIFORM && !(q.p > 0.0 && q.p <= 1.0)) { why = "p outside (0, 1]"; return TM_EINVAL; }
        if (q.q_mode == TM_Q_EDGES && !(q.p > 0.0 && std::isfinite(q.p))) { why = "r must be > 0"; return TM_EINVAL; }
        __int128 cd = (__int128)q.c * q.delta;
        if (cd >= ((__int128)1 << 61)) { why = "c*delta >= 2^61"; return TM_EINVAL; }
        int64_t J = 1 + (t_max + (int64_t)cd - 1) / (int64_t)cd;
        if ((__int128)J * q.b > ((__int128)1 << 31)) { why = "too many windows (b * J > 2^31)"; return TM_EINVAL; }
    }
    return TM_OK;
}

int validate_query(const tm_graph* g, const tm_query& q, std::string& why) {
    return validate_query_t(g->t_max, q, why);
}

void fill_plan(QPlan& P, const tm_query& q, const tm_graph* g) {
    std::memset(&P, 0, sizeof(P));
    P.own_lo = INT64_MIN;
    P.own_hi = INT64_MAX;
    P.m_total = g->m;
    const tm_motif* m = q.motif;
    P.l = m->l;
    P.k = m->k;
    P.mode = q.mode;
    P.delta = q.delta;
    for (int i = 0; i < TM_L_MAX; i++) P.lv[i] = m->lv[i];
    P.order = kOrdTime;
    P.hoist = 0;
    P.rev = 0;
    if (m->l >= 3) {
        const LevelPlan& L = m->lv[m->l - 1];
        P.hoist = (L.view == kPair && L.su <= 1 && L.sv <= 1) ? 1 : 0;
    }
    P.hrev = 0;
    if (m->l == 3 && P.hoist) {
        const LevelPlan& L1 = m->lv[1];
        bool one_new = (L1.view == kOut || L1.view == kIn) && (L1.bind_u + L1.bind_v == 1);
        P.hrev = (L1.view == kPair || one_new) ? 1 : 0;
    }
    P.rev2 = 0;
    if (m->l >= 4) {
        const LevelPlan& LD = m->lv[m->l - 2];
        const LevelPlan& L = m->lv[m->l - 1];
        bool one_new = (LD.view == kOut || LD.view == kIn) && (LD.bind_u + LD.bind_v == 1);
        int xl = LD.bind_u ? LD.su : LD.sv;
        bool closes_x = L.view == kPair && ((L.su == xl && L.sv < LD.nb) || (L.sv == xl && L.su < LD.nb));
        P.rev2 = (one_new && closes_x) ? 1 : 0;
    }
    if (m->l == 3) {
        const LevelPlan& L1 = m->lv[1];
        const LevelPlan& L2 = m->lv[2];
        bool one_new = (L1.view == kOut || L1.view == kIn) && (L1.bind_u + L1.bind_v == 1);
        bool closes_x = L2.view == kPair && ((L2.su == 2 && L2.sv <= 1) || (L2.sv == 2 && L2.su <= 1));
        P.rev = (one_new && closes_x) ? 1 : 0;
    }
    // two nodes, three edges (Algorithm 2's motif family): counted from the pair tables
    P.ex23 = 0;
    if (m->k == 2 && m->l == 3 && m->lv[1].su != m->lv[1].sv && m->lv[2].su != m->lv[2].sv) {
        P.ex23 = kEx23On | (m->lv[1].su == 1 ? kEx23MidRev : 0) | (m->lv[2].su == 1 ? kEx23LastRev : 0);
        P.hoist = P.hrev = P.rev = P.rev2 = 0;
    }
    // when the closing edge repeats the first edge's pair, first edges go in pair order:
    // the closing range then starts right after the first edge's own position
    bool own_pair = (P.hoist && m->lv[m->l - 1].su == 0 && m->lv[m->l - 1].sv == 1) || P.ex23;
    if (q.mode == TM_MODE_EXACT) {
        P.b = 1; P.cd = 0; P.J = 1; P.p = 1.0; P.q_mode = TM_Q_UNIFORM;
        // exact queries take first edges grouped by the node their second edge hangs off
        if (m->l >= 2) {
            const LevelPlan& L1 = m->lv[1];
            if (L1.view == kOut) P.order = L1.su == 0 ? kOrdOut : kOrdIn;
            else if (L1.view == kIn) P.order = L1.sv == 1 ? kOrdIn : kOrdOut;
            else if (L1.view == kPair) P.order = L1.su == 0 ? kOrdOut : kOrdIn;
            if (own_pair) P.order = kOrdPair;
        }
    } else {
        P.b = q.b;
        P.cd = (int64_t)q.c * q.delta;
        P.J = 1 + (g->t_max + P.cd - 1) / P.cd;
        P.p = q.p;
        P.seed = q.seed;
        P.q_mode = q.q_mode;
        // most windows kept: enumerate each window's first edges grouped by node
        // (positions of the node-grouped view partitioned by window) instead of in time order
        // (only for windows large enough to hold, on average, an edge per node: smaller
        // windows gain no locality from it and would pay for the partition)
        if (q.q_mode == TM_Q_UNIFORM && q.p >= kFullScanP && m->l >= 2 && g->m > 0 &&
            P.J < (int64_t)1 << 31 && g->m / P.J >= (int64_t)g->n && q.p < 1.0) {
            const LevelPlan& L1 = m->lv[1];
            int ord = kOrdTime;
            if (L1.view == kOut) ord = L1.su == 0 ? kOrdOut : kOrdIn;
            else if (L1.view == kIn) ord = L1.sv == 1 ? kOrdIn : kOrdOut;
            else if (L1.view == kPair) ord = L1.su == 0 ? kOrdOut : kOrdIn;
            if (own_pair) ord = kOrdPair;
            if (ord != kOrdTime) {
                P.order = ord;
                P.full = 1;
            }
        }
        // every window kept: Z_k is the sum of all window weights, so each first edge of the
        // whole graph (in node order, as exact queries take them) is clamped to its own window
        // and one accumulator per shift holds the sum (the integer sum is the same whatever
        // the grouping; run_batch keeps this only when no per-window detail is asked for)
        if (q.q_mode == TM_Q_UNIFORM && q.p == 1.0 && m->l >= 2) {
            const LevelPlan& L1 = m->lv[1];
            int ord = kOrdTime;
            if (L1.view == kOut) ord = L1.su == 0 ? kOrdOut : kOrdIn;
            else if (L1.view == kIn) ord = L1.sv == 1 ? kOrdIn : kOrdOut;
            else if (L1.view == kPair) ord = L1.su == 0 ? kOrdOut : kOrdIn;
            if (own_pair) ord = kOrdPair;
            if (ord != kOrdTime) {
                P.order = ord;
                P.wclamp = 1;
                P.J_all = P.J;
                P.J = 1;
            }
        }
    }
}

// back to one slot per window (time-ordered first edges) for callers that need the windows
void undo_wclamp(QPlan& P) {
    if (!P.wclamp) return;
    P.wclamp = 0;
    P.J = P.J_all;
    P.order = kOrdTime;
}

}  // namespace

int check_query(int64_t t_max, const tm_query& q, std::string& why) { return validate_query_t(t_max, q, why); }

// the two-node tables the batch's two-node queries read: own when the middle and the last
// edge are on the same pair, rev otherwise
template <typename TT>
int ex_tables_for(const tm_graph* g, const std::vector<QPlan>& hp, cudaStream_t st, GraphDevT<TT>& G) {
    bool need_own = false, need_rev = false;
    for (const QPlan& P : hp) {
        if (!P.ex23) continue;
        bool same = ((P.ex23 & kEx23MidRev) != 0) == ((P.ex23 & kEx23LastRev) != 0);
        need_own |= same;
        need_rev |= !same;
    }
    if (!need_own && !need_rev) return TM_OK;
    return ensure_ex_tables(const_cast<tm_graph*>(g), st, need_own, need_rev, &G.ex_own, &G.ex_rev);
}

// per-first-edge scratch of one batch: window, second-level range start and length, the
// exclusive scan of the lengths, the hoisted closing ranges, and the block-window and
// chunk-start tables
size_t per_first_scratch_bytes(int64_t F, bool hoist, size_t rec_bytes) {
    size_t Fs = (size_t)std::max<int64_t>(F, 1);
    size_t nbw = Fs / 32 + 1, ncf = Fs / 4 + 2;
    return a256(rec_bytes * Fs) + a256(4 * Fs) + (hoist ? 3 : 1) * a256(8 * Fs) + a256(4 * nbw) + a256(8 * ncf);
}
constexpr size_t kBoundScratchBytes = (size_t)2 << 30;


template <typename TT>
int run_batch_t(const tm_graph* g, const tm_query* qs, int nq, tm_result* res, cudaStream_t st,
                BatchOut* dbg) {
    if (!g || (!qs && nq > 0) || (!res && nq > 0) || nq < 0) { set_error("NULL argument"); return TM_EINVAL; }
    if (nq == 0) return TM_OK;
    const Tuning tu = tuning();
    std::vector<QPlan> hp((size_t)nq);
    std::vector<int> qstat((size_t)nq, TM_OK);
    int first_err = TM_OK;
    int64_t NW = 0, n_sums = 0, F_ub = 0;
    int lmax = 1, kmax = 2;
    bool any_hoist = false, any_full = false;
    size_t wtab_bytes = 0, full_bytes = 0;
    for (int i = 0; i < nq; i++) {
        std::string why;
        int s = validate_query(g, qs[i], why);
        if (s != TM_OK) {
            qstat[(size_t)i] = s;
            if (first_err == TM_OK) { first_err = s; set_error("query " + std::to_string(i) + ": " + why); }
            std::memset(&hp[(size_t)i], 0, sizeof(QPlan));
            hp[(size_t)i].l = 0;
            hp[(size_t)i].J = 0;
            hp[(size_t)i].win_base = NW;
            continue;
        }
        fill_plan(hp[(size_t)i], qs[i], g);
        if (dbg && (dbg->seg || dbg->query >= 0)) undo_wclamp(hp[(size_t)i]);   // per-window detail asked for
        if (dbg && dbg->seg) {
            // a segment of a streamed graph: the windows and first edges it owns
            QPlan& P = hp[(size_t)i];
            const SegSpec& S = dbg->seg[i];
            P.t_off = S.t_off;
            P.m_total = S.m_total;
            P.full = 0;
            if (P.mode == TM_MODE_ESTIMATE) {
                P.order = kOrdTime;
                P.j_lo = S.j_lo;
                P.J = S.J;
            } else {
                P.own_lo = S.own_lo;
                P.own_hi = S.own_hi;
            }
        }
        if (dbg && dbg->nsub && hp[(size_t)i].mode == TM_MODE_EXACT) {
            QPlan& P = hp[(size_t)i];
            P.nsub = std::min(dbg->nsub[i], (int32_t)kMaxSub);
            for (int x = 0; x < P.nsub; x++) P.dsub[x] = dbg->sub_delta[(size_t)i * kMaxSub + x];
        }
        if (dbg && dbg->ride_q && hp[(size_t)i].mode == TM_MODE_EXACT) {
            QPlan& P = hp[(size_t)i];
            for (int x = 0; x < kMaxRide; x++)
                if (dbg->ride_q[(size_t)i * kMaxRide + x] >= 0) P.ride_q[P.nride++] = dbg->ride_q[(size_t)i * kMaxRide + x];
        }
        if (dbg && dbg->riding && dbg->riding[i] && hp[(size_t)i].mode == TM_MODE_ESTIMATE) {
            QPlan& P = hp[(size_t)i];
            undo_wclamp(P);   // its instances arrive per window
            P.riding = 1;
            P.full = 0;
            P.order = kOrdTime;
        }
        hp[(size_t)i].win_base = NW;
        hp[(size_t)i].sum_base = n_sums;
        if (!hp[(size_t)i].riding)   // at most m first edges per exact query and per shift
            F_ub += hp[(size_t)i].mode == TM_MODE_EXACT ? g->m : (int64_t)hp[(size_t)i].b * g->m;
        n_sums += hp[(size_t)i].mode == TM_MODE_EXACT ? 1 : hp[(size_t)i].b;
        NW += hp[(size_t)i].mode == TM_MODE_EXACT ? 1 : hp[(size_t)i].J * hp[(size_t)i].b;
        lmax = std::max(lmax, hp[(size_t)i].l);
        kmax = std::max(kmax, hp[(size_t)i].k);
        any_hoist |= hp[(size_t)i].hoist != 0 || hp[(size_t)i].ex23 != 0;
        if (hp[(size_t)i].mode == TM_MODE_ESTIMATE && hp[(size_t)i].delta + 1 <= kWtabMax)
            wtab_bytes += a256(16 * (size_t)(hp[(size_t)i].delta + 1));
        if (hp[(size_t)i].full) {
            any_full = true;
            full_bytes += a256(4 * (size_t)hp[(size_t)i].b * (size_t)g->m) +
                          a256(8 * (size_t)hp[(size_t)i].b * (size_t)(hp[(size_t)i].J + 1));
        }
    }
    // exact queries with riders or smaller spans leave that work to k_ride in records; the
    // record buffer holds as many as the largest batch so far needed (a batch that needs more
    // runs again with room for all of them)
    bool any_share = false;
    for (const QPlan& P : hp) any_share |= P.nsub > 0 || P.nride > 0;
    const int64_t rcap = any_share ? ride_capacity().load() : 0;
    const size_t rrec_bytes = any_share ? a256(sizeof(RideRec<TT>) * (size_t)rcap) : 0;
    // window origins of the riding estimates' shifts, read per instance on the device
    std::vector<int64_t> h_shifts;
    for (const QPlan& P : hp)
        if (P.riding)
            for (int k = 0; k < P.b; k++)
                h_shifts.push_back(-(int64_t)(draw(P.seed, (uint64_t)k, 0) % (uint64_t)P.cd) - P.t_off);
    // ---- scratch layout
    int smax = 1;
    const int64_t n_parts = fold_parts(hp, smax);
    int bmax = 1;
    for (const QPlan& P : hp) bmax = std::max(bmax, P.b);
    size_t NWs = (size_t)std::max<int64_t>(NW, 1);
    size_t Ms = (size_t)std::max<int64_t>(g->m, 1);
    size_t sz = a256(sizeof(QPlan) * (size_t)nq) + a256(sizeof(tm_result) * (size_t)nq) + wtab_bytes +
                9 * a256(8 * NWs) + 3 * a256(4 * NWs) + a256(8 * NWs) + a256(8 * A_N * NWs) + 4 * 256 +
                full_bytes + (any_full ? 3 * a256(4 * Ms) : 0) +
                a256(sizeof(ShiftSums) * (size_t)std::max<int64_t>(n_sums, 1)) +
                a256(sizeof(ShiftSums) * (size_t)n_parts) +
                a256(8 * kMaxSub * (size_t)nq) + a256(8 * std::max<size_t>(h_shifts.size(), 1));
    char* sb = nullptr;
    TM_CUDA(cudaMallocAsync((void**)&sb, sz, st));
    char* p = sb;
    auto take = [&](size_t bytes) { char* r = p; p += a256(bytes); return (void*)r; };
    QPlan* dplans = (QPlan*)take(sizeof(QPlan) * (size_t)nq);
    tm_result* dres = (tm_result*)take(sizeof(tm_result) * (size_t)nq);
    for (int i = 0; i < nq; i++) {
        QPlan& P = hp[(size_t)i];
        if (P.l > 0 && P.mode == TM_MODE_ESTIMATE && P.delta + 1 <= kWtabMax) {
            P.wtab = (const uint64_t*)take(16 * (size_t)(P.delta + 1));
        }
        if (P.full) {
            P.perm = (const int32_t*)take(4 * (size_t)P.b * (size_t)g->m);
            P.woff = (const int64_t*)take(8 * (size_t)P.b * (size_t)(P.J + 1));
        }
    }
    uint32_t* pk_key = any_full ? (uint32_t*)take(4 * Ms) : nullptr;
    uint32_t* pk_ktmp = any_full ? (uint32_t*)take(4 * Ms) : nullptr;
    uint32_t* pk_vtmp = any_full ? (uint32_t*)take(4 * Ms) : nullptr;
    WinDev W;
    W.lo = (int64_t*)take(8 * NWs);
    W.hi = (int64_t*)take(8 * NWs);
    W.tlo = (int64_t*)take(8 * NWs);
    W.thi = (int64_t*)take(8 * NWs);
    W.tend = (int64_t*)take(8 * NWs);
    W.start = (int64_t*)take(8 * NWs);
    W.j = (int64_t*)take(8 * NWs);
    W.nfirst = (int64_t*)take(8 * NWs);
    W.fbase = (int64_t*)take(8 * NWs);
    W.q = (int32_t*)take(4 * NWs);
    W.k = (int32_t*)take(4 * NWs);
    W.kept = (int32_t*)take(4 * NWs);
    W.qj = (double*)take(8 * NWs);
    W.acc = (unsigned long long*)take(8 * A_N * NWs);
    int64_t* dF = (int64_t*)take(8);
    int64_t* dW2 = (int64_t*)take(8);
    unsigned long long* dctr = (unsigned long long*)take(8);
    unsigned long long* drcount = (unsigned long long*)take(8);
    ShiftSums* dsums = (ShiftSums*)take(sizeof(ShiftSums) * (size_t)std::max<int64_t>(n_sums, 1));
    ShiftSums* dpart = (ShiftSums*)take(sizeof(ShiftSums) * (size_t)n_parts);
    unsigned long long* dsubc = (unsigned long long*)take(8 * kMaxSub * (size_t)nq);
    int64_t* dshifts = (int64_t*)take(8 * std::max<size_t>(h_shifts.size(), 1));
    for (size_t i = 0, o = 0; i < (size_t)nq; i++)
        if (hp[i].riding) {
            hp[i].shifts = dshifts + o;
            o += (size_t)hp[i].b;
        }

    int rc = TM_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        if (rc == TM_OK && e != cudaSuccess) rc = cuda_status(e, what, __FILE__, __LINE__);
    };
    PhaseEvents pe(profiling());
    NvtxPhases nv;
    nv.next("tm_windows");
    auto wall0 = std::chrono::steady_clock::now();
    int ev_w0 = pe.mark(st), ev_w1 = -1, ev_l0 = -1, ev_l1 = -1, ev_l2 = -1, ev_m1 = -1, ev_r1 = -1, ev_f1 = -1;
    int64_t hW2 = 0;
    unsigned long long h_rcount = 0;
    fail(cudaMemcpyAsync(dplans, hp.data(), sizeof(QPlan) * (size_t)nq, cudaMemcpyHostToDevice, st), "plans");
    if (!h_shifts.empty())
        fail(cudaMemcpyAsync(dshifts, h_shifts.data(), 8 * h_shifts.size(), cudaMemcpyHostToDevice, st), "shifts");
    fail(cudaMemsetAsync(W.acc, 0, 8 * A_N * NWs, st), "acc");
    fail(cudaMemsetAsync(dctr, 0, 8, st), "counter");
    fail(cudaMemsetAsync(drcount, 0, 8, st), "record counter");
    for (int i = 0; i < nq && rc == TM_OK; i++) {
        const QPlan& P = hp[(size_t)i];
        if (P.wtab) {
            int64_t n = P.delta + 1;
            unsigned gr = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
            k_wtab<<<gr, 256, 0, st>>>((uint64_t*)P.wtab, P.delta, P.cd); count_launch();
            fail(cudaGetLastError(), "k_wtab");
        }
    }
    GraphDevT<TT> G = typed<TT>(g->dev);
    if (rc == TM_OK) rc = ex_tables_for(g, hp, st, G);
    int nsm = sm_count();
    // dense-sampling queries: per shift, node-grouped view positions stably partitioned by window
    for (int i = 0; i < nq && rc == TM_OK; i++) {
        const QPlan& P = hp[(size_t)i];
        if (!P.full || g->m == 0) continue;
        const TT* tv = P.order == kOrdOut ? G.out_t : P.order == kOrdIn ? G.in_t : G.pair_t;
        int bits = 0;
        while (bits < 31 && ((int64_t)1 << bits) < P.J) bits++;
        for (int k = 0; k < P.b && rc == TM_OK; k++) {
            int64_t sft = -(int64_t)(draw(P.seed, (uint64_t)k, 0) % (uint64_t)P.cd);
            uint32_t* vals = (uint32_t*)(P.perm + (size_t)k * (size_t)g->m);
            unsigned gr = (unsigned)std::min<int64_t>((g->m + 255) / 256, (int64_t)nsm * 8);
            k_winkey<TT><<<gr, 256, 0, st>>>(tv, g->m, sft, P.cd, pk_key, vals); count_launch();
            fail(cudaGetLastError(), "k_winkey");
            if (rc == TM_OK) rc = radix_sort_pairs(pk_key, vals, pk_ktmp, pk_vtmp, g->m, bits, st);
            if (rc == TM_OK) {
                k_woff<<<(unsigned)std::min<int64_t>((g->m + 256) / 256, (int64_t)nsm * 8), 256, 0, st>>>(
                    pk_key, g->m, P.J, (int64_t*)(P.woff + (size_t)k * (size_t)(P.J + 1)));
                count_launch();
                fail(cudaGetLastError(), "k_woff");
            }
        }
    }
    if (rc == TM_OK && NW > 0) {
        unsigned gr = (unsigned)std::min<int64_t>((NW + 255) / 256, (int64_t)nsm * 16);
        k_windows<TT><<<gr, 256, 0, st>>>(G, dplans, nq, W, NW); count_launch();
        fail(cudaGetLastError(), "k_windows");
    }
    if (rc == TM_OK) rc = scan_exclusive_i64(W.nfirst, W.fbase, NW, dF, st);
    // The per-first-edge scratch is sized for the bound on F when that fits in
    // kBoundScratchBytes, and the kernels read F on the device: no host round trip
    // between the window partition and the matcher.  Otherwise F is read back first.
    const bool bounded = F_ub > 0 && per_first_scratch_bytes(F_ub, any_hoist, sizeof(FRec<TT>)) <= kBoundScratchBytes;
    int64_t F = 0;
    ev_w1 = pe.mark(st);
    nv.next("tm_sizing");
    if (rc == TM_OK && !bounded) {
        fail(cudaMemcpyAsync(&F, dF, 8, cudaMemcpyDeviceToHost, st), "F readback");
        fail(cudaStreamSynchronize(st), "sync F");
    }
    const int64_t Fa = bounded ? F_ub : F;   // first edges the scratch holds
    ScratchLease fb;
    if (rc == TM_OK && Fa > 0) {
        size_t Fs = (size_t)Fa;
        size_t nbw = Fs / 32 + 1, ncf = Fs / 4 + 2;
        rc = scratch_acquire(per_first_scratch_bytes(Fa, any_hoist, sizeof(FRec<TT>)) + rrec_bytes, st, fb);
        if (rc == TM_OK) {
            char* q2 = (char*)fb.p;
            auto take2 = [&](size_t bytes) { char* r = q2; q2 += a256(bytes); return (void*)r; };
            FRec<TT>* rec = (FRec<TT>*)take2(sizeof(FRec<TT>) * Fs);
            int64_t* excl = (int64_t*)take2(8 * Fs);   // exclusive scan of the range lengths
            int32_t* len32 = (int32_t*)take2(4 * Fs);
            int64_t* hs_a = any_hoist ? (int64_t*)take2(8 * Fs) : nullptr;
            int64_t* hs_hi = any_hoist ? (int64_t*)take2(8 * Fs) : nullptr;
            int32_t* bwin = (int32_t*)take2(4 * nbw);
            int64_t* cf = (int64_t*)take2(8 * ncf);
            RideRec<TT>* rrec = any_share ? (RideRec<TT>*)take2(sizeof(RideRec<TT>) * (size_t)rcap) : nullptr;
            MatchArgs<TT> A;
            const int64_t* d_Fk = bounded ? dF : nullptr;
            A.G = G; A.plans = dplans; A.nq = nq; A.W = W; A.NW = NW; A.F = Fa; A.d_F = d_Fk;
            A.rec = rec; A.excl = excl; A.hs_a = hs_a; A.hs_hi = hs_hi;
            A.d_W2 = dW2; A.counter = dctr;
            A.enum_threshold = tu.enum_threshold;
            A.chunk = tu.chunk_items;
            A.blockwin = bwin; A.chunkf = cf; A.nchunkf = (int64_t)ncf;
            A.rrec = rrec;
            A.rcount = drcount;
            A.rcap = rcap;
            int64_t gl2 = std::min<int64_t>((Fa + 255) / 256, (int64_t)nsm * 8);
            k_blockwin<<<(unsigned)std::min<int64_t>(((int64_t)nbw + 255) / 256, (int64_t)nsm * 8), 256, 0, st>>>(
                W.fbase, NW, Fa, d_Fk, bwin);
            count_launch();
            ev_l0 = pe.mark(st);
            nv.next("tm_level2");
            k_level2<TT><<<(unsigned)std::max<int64_t>(gl2, 1), 256, match_smem_bytes(A.nq, 256), st>>>(A, rec, len32, hs_a, hs_hi); count_launch();
            fail(cudaGetLastError(), "k_level2");
            ev_l2 = pe.mark(st);
            nv.next("tm_scan");
            if (rc == TM_OK) rc = scan_lengths(len32, excl, Fa, d_Fk, dW2, nullptr, 0, st);
            if (rc == TM_OK) {
                k_chunkf<<<(unsigned)std::min<int64_t>(((int64_t)ncf + 255) / 256, (int64_t)nsm * 8), 256, 0, st>>>(
                    excl, Fa, d_Fk, dW2, A.chunk, (int64_t)ncf, cf);
                count_launch();
                fail(cudaGetLastError(), "k_chunkf");
            }
            ev_l1 = pe.mark(st);
            nv.next("tm_match");
            if (rc == TM_OK) {
                launch_match<TT>(A, lmax, kmax, tu, nsm, st,
                                 std::any_of(hp.begin(), hp.end(), [](const QPlan& P) { return plan_expands(P); }));
                fail(cudaGetLastError(), "k_match");
                ev_m1 = pe.mark(st);
                if (any_share && rc == TM_OK) {
                    nv.next("tm_ride");
                    k_ride<TT><<<(unsigned)(nsm * 8), 256, match_smem_bytes(A.nq, 256, true), st>>>(A);
                    count_launch();
                    fail(cudaGetLastError(), "k_ride");
                    ev_r1 = pe.mark(st);
                }
                if (pe.on) fail(cudaMemcpyAsync(&hW2, dW2, 8, cudaMemcpyDeviceToHost, st), "W2");
                if (pe.on && bounded) fail(cudaMemcpyAsync(&F, dF, 8, cudaMemcpyDeviceToHost, st), "F");
            }
        }
    }
    if (rc == TM_OK) {
        int ev_f0 = pe.mark(st);
        nv.next("tm_fold");
        launch_fold(dplans, nq, bmax, smax, W, dpart, dres, dbg && dbg->sums ? dsums : nullptr,
                    dbg && dbg->sub_count ? dsubc : nullptr, st);
        fail(cudaGetLastError(), "fold");
        ev_f1 = pe.mark(st);
        nv.next(nullptr);
        if (ev_m1 < 0) ev_m1 = ev_f0;
        if (ev_r1 < 0) ev_r1 = ev_m1;
    }
    if (rc == TM_OK && any_share) fail(cudaMemcpyAsync(&h_rcount, drcount, 8, cudaMemcpyDeviceToHost, st), "records");
    if (rc == TM_OK) fail(cudaMemcpyAsync(res, dres, sizeof(tm_result) * (size_t)nq, cudaMemcpyDeviceToHost, st), "results");
    if (rc == TM_OK && dbg && dbg->sub_count)
        fail(cudaMemcpyAsync(dbg->sub_count, dsubc, 8 * kMaxSub * (size_t)nq, cudaMemcpyDeviceToHost, st),
             "span counts");
    if (rc == TM_OK && dbg && dbg->sums && n_sums > 0) {
        std::memset(dbg->sums, 0, sizeof(ShiftSums) * (size_t)n_sums);   // rejected queries write none
        fail(cudaMemcpyAsync(dbg->sums, dsums, sizeof(ShiftSums) * (size_t)n_sums, cudaMemcpyDeviceToHost, st),
             "shift sums");
    }
    // optional window readback for one query
    std::vector<int64_t> h_lo, h_hi, h_start, h_j;
    std::vector<int32_t> h_k, h_kept;
    std::vector<double> h_qj;
    std::vector<unsigned long long> h_acc;
    int64_t dq_base = 0, dq_n = 0;
    if (rc == TM_OK && dbg && dbg->query >= 0 && dbg->query < nq && hp[(size_t)dbg->query].l > 0) {
        const QPlan& P = hp[(size_t)dbg->query];
        dq_n = P.mode == TM_MODE_EXACT ? 1 : P.J;
        dq_base = P.win_base + (P.mode == TM_MODE_EXACT ? 0 : (int64_t)dbg->k * P.J);
        if (dbg->k < 0 || dbg->k >= P.b) dq_n = 0;
        size_t n = (size_t)dq_n;
        h_lo.resize(n); h_hi.resize(n); h_start.resize(n); h_j.resize(n);
        h_k.resize(n); h_kept.resize(n); h_qj.resize(n); h_acc.resize(n * A_N);
        if (n) {
            fail(cudaMemcpyAsync(h_lo.data(), W.tlo + dq_base, 8 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_hi.data(), W.thi + dq_base, 8 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_start.data(), W.start + dq_base, 8 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_j.data(), W.j + dq_base, 8 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_k.data(), W.k + dq_base, 4 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_kept.data(), W.kept + dq_base, 4 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_qj.data(), W.qj + dq_base, 8 * n, cudaMemcpyDeviceToHost, st), "dbg");
            fail(cudaMemcpyAsync(h_acc.data(), W.acc + dq_base * A_N, 8 * A_N * n, cudaMemcpyDeviceToHost, st), "dbg");
        }
    }
    cudaError_t se = cudaStreamSynchronize(st);
    fail(se, "batch sync");
    if (pe.on && rc == TM_OK) {
        double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
        store_profile_batch(pe.ms(ev_w0, ev_w1), pe.ms(ev_l0, ev_l2), ev_l1 >= 0 ? pe.ms(ev_l1, ev_m1) : 0.0,
                            pe.ms(ev_m1 >= 0 && ev_l1 >= 0 ? ev_r1 : ev_f1, ev_f1), wall, hW2, F,
                            ev_l0 >= 0 ? pe.ms(ev_w1, ev_l0) : 0.0, ev_l1 >= 0 ? pe.ms(ev_l2, ev_l1) : 0.0,
                            ev_l1 >= 0 ? pe.ms(ev_m1, ev_r1) : 0.0);
    }
    if (pe.on && rc == TM_OK) store_profile_ride_records((int64_t)h_rcount);
    scratch_release(fb, st);
    cudaFreeAsync(sb, st);
    if (rc != TM_OK) return rc;
    if ((int64_t)h_rcount > rcap) {
        // more deferred records than the buffer held: run again with room for all of them
        int64_t want = (int64_t)h_rcount + (int64_t)(h_rcount >> 3) + 1024;
        int64_t cur = ride_capacity().load();
        while (cur < want && !ride_capacity().compare_exchange_weak(cur, want)) {}
        return run_batch_t<TT>(g, qs, nq, res, st, dbg);
    }
    if (dbg && dq_n > 0) {
        const QPlan& P = hp[(size_t)dbg->query];
        int64_t n_out = 0;
        for (int64_t i = 0; i < dq_n; i++) {
            if (!dbg->all_windows && !h_kept[(size_t)i]) continue;
            if (n_out < dbg->cap && dbg->recs) {
                tm_window_rec& r = dbg->recs[n_out];
                r.k = h_k[(size_t)i];
                r.kept = h_kept[(size_t)i];
                r.j = h_j[(size_t)i];
                r.start = h_start[(size_t)i];
                r.lo = h_lo[(size_t)i];
                r.hi = h_hi[(size_t)i];
                r.count = (int64_t)h_acc[(size_t)i * A_N + A_COUNT];
                r.w_int = h_acc[(size_t)i * A_N + A_WHI];
                r.w_frac = h_acc[(size_t)i * A_N + A_WLO];
                r.q = h_qj[(size_t)i];
            }
            n_out++;
        }
        dbg->n_out = n_out;
        dbg->shift = P.mode == TM_MODE_EXACT ? 0 : -(int64_t)(draw(P.seed, (uint64_t)dbg->k, 0) % (uint64_t)P.cd);
    }
    for (int i = 0; i < nq; i++) {
        if (qstat[(size_t)i] != TM_OK) {
            std::memset(&res[i], 0, sizeof(tm_result));
            res[i].status = qstat[(size_t)i];
        } else if (res[i].status != TM_OK && first_err == TM_OK) {
            first_err = res[i].status;
            set_error("query " + std::to_string(i) + ": count or weight sum overflowed 2^63");
        }
    }
    return first_err;
}

namespace {

int run_batch_typed(const tm_graph* g, const tm_query* qs, int nq, tm_result* res, cudaStream_t st,
                    BatchOut* dbg) {
    if (g && g->dev.tbytes == 4) return run_batch_t<int32_t>(g, qs, nq, res, st, dbg);
    return run_batch_t<int64_t>(g, qs, nq, res, st, dbg);
}

// exact three-edge queries whose last edge joins two bound nodes: a query of the same
// motif at a smaller span counts a subset of the same enumeration (the instances whose
// duration is within its span), so it rides along with the largest span's query
bool same_motif(const tm_motif* a, const tm_motif* b) {
    if (a == b) return true;
    if (a->l != b->l || a->k != b->k) return false;
    return std::memcmp(a->lv, b->lv, sizeof(LevelPlan) * (size_t)a->l) == 0;
}

int run_batch_once(const tm_graph* g, const tm_query* qs, int nq, tm_result* res, cudaStream_t st,
                   BatchOut* dbg) {
    if (dbg || !g || !qs || !res || nq < 2) return run_batch_typed(g, qs, nq, res, st, dbg);
    std::vector<int> lead((size_t)nq, -1), slot((size_t)nq, -1);   // span members: their leader
    std::vector<std::vector<int>> groups;
    for (int i = 0; i < nq; i++) {
        const tm_query& q = qs[i];
        std::string why;
        if (q.mode != TM_MODE_EXACT || !q.motif || q.motif->l != 3 || q.motif->lv[2].view != kPair) continue;
        if (validate_query(g, q, why) != TM_OK) continue;
        bool placed = false;
        for (auto& gr : groups)
            if ((int)gr.size() < 1 + kMaxSub && same_motif(qs[gr[0]].motif, q.motif)) {
                gr.push_back(i);
                placed = true;
                break;
            }
        if (!placed) groups.push_back({i});
    }
    bool any = false;
    std::vector<int> heads;   // exact queries that do their own enumeration
    for (auto& gr : groups) {
        int L = gr[0];
        for (int i : gr)
            if (qs[i].delta > qs[L].delta) L = i;
        heads.push_back(L);
        if (gr.size() < 2) continue;
        any = true;
        int k = 0;
        for (int i : gr)
            if (i != L) { lead[(size_t)i] = L; slot[(size_t)i] = k++; }
    }
    // estimates of the same three-edge motif with a span no larger than an exact query's ride
    // along with it: each instance that query enumerates also adds its weight to the window of
    // an estimate when it lies inside one of its kept windows and within its span, so the
    // estimate needs no enumeration of its own (its windows and fold stay its own)
    std::vector<int> host((size_t)nq, -1);    // estimate -> its exact head
    std::vector<int> nrid((size_t)nq, 0);
    for (int i = 0; i < nq; i++) {
        const tm_query& q = qs[i];
        std::string why;
        if (q.mode != TM_MODE_ESTIMATE || (q.q_mode != TM_Q_UNIFORM && q.q_mode != TM_Q_EDGES)) continue;
        if (!q.motif || q.motif->l != 3 || q.motif->lv[2].view != kPair) continue;
        if (validate_query(g, q, why) != TM_OK) continue;
        for (int L : heads)
            if (nrid[(size_t)L] < kMaxRide && qs[L].delta >= q.delta && same_motif(qs[L].motif, q.motif)) {
                host[(size_t)i] = L;
                nrid[(size_t)L]++;
                any = true;
                break;
            }
    }
    if (!any) return run_batch_typed(g, qs, nq, res, st, nullptr);
    // the batch without the span members, each head carrying its members' spans and riders
    std::vector<tm_query> qc;
    std::vector<int> pos((size_t)nq, -1);
    for (int i = 0; i < nq; i++)
        if (lead[(size_t)i] < 0) { pos[(size_t)i] = (int)qc.size(); qc.push_back(qs[i]); }
    int nc = (int)qc.size();
    std::vector<int32_t> riding((size_t)nc, 0), ride_q((size_t)nc * kMaxRide, -1), fill((size_t)nc, 0);
    for (int i = 0; i < nq; i++) {
        if (host[(size_t)i] < 0) continue;
        int c = pos[(size_t)i], h = pos[(size_t)host[(size_t)i]];
        riding[(size_t)c] = 1;
        ride_q[(size_t)h * kMaxRide + fill[(size_t)h]++] = c;
    }
    std::vector<int32_t> nsub((size_t)nc, 0);
    std::vector<int64_t> sd((size_t)nc * kMaxSub, 0);
    for (int i = 0; i < nq; i++) {
        if (lead[(size_t)i] < 0) continue;
        int c = pos[(size_t)lead[(size_t)i]];
        sd[(size_t)c * kMaxSub + slot[(size_t)i]] = qs[i].delta;
        nsub[(size_t)c] = std::max(nsub[(size_t)c], slot[(size_t)i] + 1);
    }
    std::vector<tm_result> rc_res((size_t)nc);
    std::vector<unsigned long long> sc((size_t)nc * kMaxSub, 0);
    BatchOut bo;
    bo.nsub = nsub.data();
    bo.sub_delta = sd.data();
    bo.sub_count = sc.data();
    bo.riding = riding.data();
    bo.ride_q = ride_q.data();
    int rc = run_batch_typed(g, qc.data(), nc, rc_res.data(), st, &bo);
    for (int i = 0; i < nq; i++) {
        if (lead[(size_t)i] < 0) {
            res[i] = rc_res[(size_t)pos[(size_t)i]];
            continue;
        }
        int c = pos[(size_t)lead[(size_t)i]];
        tm_result r = rc_res[(size_t)c];   // status of the shared enumeration
        r.count = (int64_t)sc[(size_t)c * kMaxSub + slot[(size_t)i]];
        r.estimate = (double)r.count;
        r.first_edges = r.cand_edges = r.last_ranges = r.inst_read = 0;   // the work is the leader's
        res[i] = r;
    }
    return rc;
}

// TM_Q_AUTO: p from a pilot estimate (see tm.h): the smallest p whose sampling standard
// deviation of the b-shift mean, predicted from the pilot's Var[Z | s] estimate (Lemma 4.4),
// is within target * Z0 / z
double auto_p(const tm_result& pilot, double target, int32_t b) {
    const double z = 1.96, p0 = TM_AUTO_PILOT_P;
    double z0 = pilot.estimate;
    double s2 = pilot.var_hat * p0 / (1.0 - p0);   // estimates sum_j Y_j^2
    if (!(z0 > 0.0)) return 1.0;
    if (!(s2 > 0.0)) return p0;
    double r = (double)b * (target * z0 / z) * (target * z0 / z) / s2;
    double p = 1.0 / (1.0 + r);
    return std::min(1.0, std::max(p0, p));
}

}  // namespace

int run_batch(const tm_graph* g, const tm_query* qs, int nq, tm_result* res, cudaStream_t st,
              BatchOut* dbg) {
    bool any_auto = false;
    for (int i = 0; qs && i < nq; i++)
        any_auto |= qs[i].mode == TM_MODE_ESTIMATE && qs[i].q_mode == TM_Q_AUTO;
    if (!any_auto) return run_batch_once(g, qs, nq, res, st, dbg);
    if (!g || !res) { set_error("NULL argument"); return TM_EINVAL; }
    if (dbg && (dbg->seg || dbg->query >= 0)) { set_error("TM_Q_AUTO needs the whole graph"); return TM_EINVAL; }
    // pilot batch: the auto queries at p0 (valid ones only; the rest is checked below)
    std::vector<tm_query> pq;
    std::vector<int> pidx;
    for (int i = 0; i < nq; i++) {
        if (qs[i].mode != TM_MODE_ESTIMATE || qs[i].q_mode != TM_Q_AUTO) continue;
        std::string why;
        if (validate_query(g, qs[i], why) != TM_OK) continue;
        tm_query q = qs[i];
        q.q_mode = TM_Q_UNIFORM;
        q.p = TM_AUTO_PILOT_P;
        q.seed = qs[i].seed ^ TM_AUTO_PILOT_SEED_XOR;
        pq.push_back(q);
        pidx.push_back(i);
    }
    std::vector<tm_result> pr(pq.size());
    std::vector<tm_query> fq(qs, qs + nq);
    if (!pq.empty()) {
        int rc = run_batch_once(g, pq.data(), (int)pq.size(), pr.data(), st, nullptr);
        if (rc != TM_OK) return rc;
        for (size_t x = 0; x < pq.size(); x++) {
            tm_query& q = fq[(size_t)pidx[x]];
            q.p = auto_p(pr[x], qs[pidx[x]].p, q.b);
            q.q_mode = TM_Q_UNIFORM;
        }
    }
    return run_batch_once(g, fq.data(), nq, res, st, dbg);
}

template <typename TT>
int count_plain_t(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count) {
    if (!g || !m || !count) { set_error("NULL argument"); return TM_EINVAL; }
    if (delta < 0 || delta >= ((int64_t)1 << 61)) { set_error("delta outside [0, 2^61)"); return TM_EINVAL; }
    tm_query q;
    std::memset(&q, 0, sizeof(q));
    q.motif = m;
    q.delta = delta;
    q.mode = TM_MODE_EXACT;
    QPlan P;
    fill_plan(P, q, g);
    cudaStream_t st;
    TM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    char* sb = nullptr;
    int rc = TM_OK;
    static_assert(sizeof(QPlan) <= 512, "the plan and the counter share a 768-byte block");
    cudaError_t e = cudaMallocAsync((void**)&sb, 768, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sb, &P, sizeof(P), cudaMemcpyHostToDevice, st);
    unsigned long long* dc = (unsigned long long*)(sb + 512);
    if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, 8, st);
    if (e == cudaSuccess && g->m > 0) {
        int nsm = sm_count();
        unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((g->m + 255) / 256, (int64_t)nsm * 8));
        k_plain<TT><<<gr, 256, 0, st>>>(typed<TT>(g->dev), (const QPlan*)sb, dc); count_launch();
        e = cudaGetLastError();
    }
    unsigned long long hc = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, dc, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_status(e, "tm_count_exact_plain", __FILE__, __LINE__);
    if (sb) cudaFreeAsync(sb, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc == TM_OK) {
        if (hc >= (1ull << 63)) { set_error("count overflowed 2^63"); return TM_EOVERFLOW; }
        *count = (int64_t)hc;
    }
    return rc;
}

int count_plain(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count) {
    if (g && g->dev.tbytes == 4) return count_plain_t<int32_t>(g, m, delta, count);
    return count_plain_t<int64_t>(g, m, delta, count);
}

TM_DEFINE_CHECK_WORD(check_word_match)

#ifdef TM_CHECKED
namespace {
// one out-of-range index (n for an array of n elements) through the checked accessor: the
// check records it and the read goes to element 0
__global__ void k_check_selftest(const int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = a[TM_CHK_IDX(n, n, kChkSelf)];
}
}  // namespace

int check_selftest() {
    int64_t* d = nullptr;
    TM_CUDA(cudaMalloc(&d, 2 * sizeof(int64_t)));
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int64_t));
    if (e == cudaSuccess) {
        k_check_selftest<<<1, 32>>>(d, 1, d + 1);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(e, "tm_check_selftest", __FILE__, __LINE__);
    return TM_OK;
}
#else
int check_selftest() {
    set_error("bounds checks are not compiled into this build");
    return TM_EINVAL;
}
#endif

}  // namespace tmo

// ---------------------------------------------------------------------------
// Exact count without any allocation (tm_count_exact_noalloc).
//
// For callers that may not allocate device memory while answering a query:
// the same kernels as the batched exact count, with every scratch buffer
// (query plan, window descriptor and accumulators, per-first-edge ranges and
// their scan, the work-queue counter, the result) carved out of one static
// device array that the library carries for at most TM_NOALLOC_MAX_EDGES
// edges.  Host code may not use the array's name as a device address, so the
// address is resolved once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t na_a256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int64_t kNaMaxEdges = TM_NOALLOC_MAX_EDGES;
constexpr int64_t kNaWsElems = 2 * ((kNaMaxEdges + 2047) / 2048);
constexpr size_t kNaWinBytes = 13 * 256 + na_a256(8 * tmo::A_N);
constexpr size_t kNaRecBytes = 40;   // the first-edge record with 64-bit times (the larger one)
constexpr size_t kNaBytes = na_a256(sizeof(tmo::QPlan)) + na_a256(sizeof(tm_result)) + kNaWinBytes +
                            3 * 256 + na_a256(kNaRecBytes * kNaMaxEdges) + 2 * na_a256(8 * kNaMaxEdges) +
                            na_a256(8 * kNaWsElems);
static_assert(kNaBytes == TM_NOALLOC_SCRATCH_BYTES, "tm.h states the scratch size");
constexpr int kNaMaxDevices = 64;

std::mutex g_na_mu;
unsigned char* g_na_base[kNaMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

namespace tmo {
namespace {

int na_status(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA;
}

// device address of the static scratch on the current device (resolved once per device)
int na_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_status(e);
    if (dev < 0 || dev >= kNaMaxDevices) return TM_EINVAL;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return na_status(e);
        g_na_base[dev] = (unsigned char*)p;
    }
    *out = g_na_base[dev];
    return TM_OK;
}

template <typename TT>
int count_exact_noalloc_t(const tm_graph* g, const tm_motif* m, int64_t delta, cudaStream_t st,
                          int64_t* count) {
    if (!g || !m || !count) return TM_EINVAL;
    if (delta < 0 || delta >= ((int64_t)1 << 61)) return TM_EINVAL;
    if (g->m > kNaMaxEdges) return TM_EINVAL;
    unsigned char* base = nullptr;
    int rc = na_scratch(&base);
    if (rc != TM_OK) return rc;
    // the array is resolved for the current device, and the kernels run there: the graph
    // must live on that device too
    int cur = -1;
    cudaError_t ce = cudaGetDevice(&cur);
    if (ce != cudaSuccess) return na_status(ce);
    if (cur != g->device) return TM_EINVAL;
    unsigned char* p = base;
    auto take = [&](size_t bytes) { unsigned char* r = p; p += na_a256(bytes); return (void*)r; };
    QPlan* dplan = (QPlan*)take(sizeof(QPlan));
    tm_result* dres = (tm_result*)take(sizeof(tm_result));
    WinDev W;
    W.lo = (int64_t*)take(8);
    W.hi = (int64_t*)take(8);
    W.tlo = (int64_t*)take(8);
    W.thi = (int64_t*)take(8);
    W.tend = (int64_t*)take(8);
    W.start = (int64_t*)take(8);
    W.j = (int64_t*)take(8);
    W.nfirst = (int64_t*)take(8);
    W.fbase = (int64_t*)take(8);
    W.q = (int32_t*)take(4);
    W.k = (int32_t*)take(4);
    W.kept = (int32_t*)take(4);
    W.qj = (double*)take(8);
    W.acc = (unsigned long long*)take(8 * A_N);
    int64_t* dF = (int64_t*)take(8);
    int64_t* dW2 = (int64_t*)take(8);
    unsigned long long* dctr = (unsigned long long*)take(8);
    static_assert(sizeof(FRec<TT>) <= kNaRecBytes, "record size of the static scratch");
    FRec<TT>* rec = (FRec<TT>*)take(kNaRecBytes * (size_t)kNaMaxEdges);
    int64_t* len2 = (int64_t*)take(8 * (size_t)kNaMaxEdges);
    int64_t* excl = (int64_t*)take(8 * (size_t)kNaMaxEdges);
    int64_t* ws = (int64_t*)take(8 * (size_t)kNaWsElems);
    if ((size_t)(p - base) > kNaBytes) return TM_EINVAL;   // layout and array size disagree

    tm_query q;
    std::memset(&q, 0, sizeof(q));
    q.motif = m;
    q.delta = delta;
    q.mode = TM_MODE_EXACT;
    QPlan P;
    fill_plan(P, q, g);
    P.win_base = 0;
    P.hoist = 0;   // no per-first-edge closing ranges: keeps the scratch at its stated size
    P.ex23 = 0;    // nor the two-node tables (an allocation)
    // every call starts from zeroed accumulators and queue counter
    cudaError_t e = cudaMemcpyAsync(dplan, &P, sizeof(P), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(W.acc, 0, 8 * A_N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dctr, 0, 8, st);
    if (e != cudaSuccess) return na_status(e);
    GraphDevT<TT> G = typed<TT>(g->dev);
    k_windows<TT><<<1, 32, 0, st>>>(G, dplan, 1, W, 1); count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_status(e);
    rc = scan_exclusive_i64_ws(W.nfirst, W.fbase, 1, dF, ws, kNaWsElems, st);
    if (rc != TM_OK) return rc;
    int64_t F = g->m;   // one window holding every edge
    if (F > 0) {
        const Tuning tu = tuning();
        MatchArgs<TT> A;
        A.G = G; A.plans = dplan; A.nq = 1; A.W = W; A.NW = 1; A.F = F; A.d_F = nullptr;
        A.rec = rec; A.excl = excl; A.d_W2 = dW2; A.counter = dctr;
        A.hs_a = nullptr; A.hs_hi = nullptr;
        A.enum_threshold = tu.enum_threshold;
        A.chunk = tu.chunk_items;
        int nsm = sm_count();
        int64_t gl2 = std::min<int64_t>((F + 255) / 256, (int64_t)nsm * 8);
        k_level2<TT><<<(unsigned)std::max<int64_t>(gl2, 1), 256, match_smem_bytes(A.nq, 256), st>>>(A, rec, (int32_t*)len2, nullptr, nullptr);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return na_status(e);
        // the 32-bit lengths fill the first half of their 8-byte-per-edge region; the scan's
        // workspace takes the second half
        rc = scan_lengths((const int32_t*)len2, excl, F, nullptr, dW2, len2 + kNaMaxEdges / 2, kNaMaxEdges / 2, st);
        if (rc != TM_OK) return rc;
        launch_match<TT>(A, P.l, std::max(P.k, 2), tu, nsm, st, plan_expands(P));
        e = cudaGetLastError();
        if (e != cudaSuccess) return na_status(e);
    }
    // the scan workspace is free again: it holds the fold's one partial record
    launch_fold(dplan, 1, 1, 1, W, (ShiftSums*)ws, dres, nullptr, nullptr, st);
    e = cudaGetLastError();
    tm_result hres;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hres, dres, sizeof(hres), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_status(e);
    if (hres.status != TM_OK) return hres.status;
    *count = hres.count;
    return TM_OK;
}

int count_exact_noalloc(const tm_graph* g, const tm_motif* m, int64_t delta, cudaStream_t st,
                        int64_t* count) {
    if (g && g->dev.tbytes == 4) return count_exact_noalloc_t<int32_t>(g, m, delta, st, count);
    return count_exact_noalloc_t<int64_t>(g, m, delta, st, count);
}

}  // namespace
}  // namespace tmo

extern "C" int tm_count_exact_noalloc(const tm_graph* g, const tm_motif* m, int64_t delta, void* stream,
                                      int64_t* count) {
    return tmo::count_exact_noalloc(g, m, delta, (cudaStream_t)stream, count);
}

// ---------------------------------------------------------------------------
// Prepared batches: the run_batch launch sequence captured once in a CUDA
// graph, with every size read on the device (first-edge count, candidate
// count) and scratch sized for the worst case, so a replay never waits on the
// host.
// ---------------------------------------------------------------------------
struct tm_batch {
    const tm_graph* g = nullptr;
    int nq = 0;
    std::vector<int> qstat;
    int first_err = TM_OK;
    void* scratch = nullptr;
    tm_result* h_res = nullptr;       // pinned: the graph's last node copies results here
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n_kernels = 0;
};

namespace tmo {
namespace {

void batch_release(tm_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) {
        cudaStreamSynchronize(b->cap);
        cudaStreamDestroy(b->cap);
    }
    if (b->scratch) cudaFree(b->scratch);
    if (b->h_res) cudaFreeHost(b->h_res);
    delete b;
}

template <typename TT>
int batch_create_t(const tm_graph* g, const tm_query* qs, int nq, tm_batch** out) {
    if (!out) { set_error("out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    if (!g || !qs || nq <= 0) { set_error("bad argument"); return TM_EINVAL; }
    tm_batch* b = new (std::nothrow) tm_batch();
    if (!b) { set_error("host allocation failed"); return TM_ENOMEM; }
    b->g = g;
    b->nq = nq;
    b->qstat.assign((size_t)nq, TM_OK);
    std::vector<QPlan> hp((size_t)nq);
    int64_t NW = 0, Fmax = 0, n_sums = 0;
    int lmax = 1, kmax = 2, bmax = 1;
    bool any_hoist = false;
    size_t wtab_bytes = 0;
    for (int i = 0; i < nq; i++) {
        std::string why;
        int s = validate_query(g, qs[i], why);
        if (s == TM_OK && qs[i].mode == TM_MODE_ESTIMATE && qs[i].q_mode == TM_Q_AUTO) {
            s = TM_EINVAL;   // p is chosen on the host from a pilot run: not a fixed sequence
            why = "TM_Q_AUTO needs tm_run_batch";
        }
        QPlan& P = hp[(size_t)i];
        if (s != TM_OK) {
            b->qstat[(size_t)i] = s;
            if (b->first_err == TM_OK) { b->first_err = s; set_error("query " + std::to_string(i) + ": " + why); }
            std::memset(&P, 0, sizeof(QPlan));
            P.win_base = NW;
            continue;
        }
        fill_plan(P, qs[i], g);
        undo_wclamp(P);
        P.full = 0;
        if (P.mode == TM_MODE_ESTIMATE) P.order = kOrdTime;
        P.win_base = NW;
        P.sum_base = n_sums;
        n_sums += P.mode == TM_MODE_EXACT ? 1 : P.b;
        bmax = std::max(bmax, P.b);
        NW += P.mode == TM_MODE_EXACT ? 1 : P.J * P.b;
        Fmax += P.mode == TM_MODE_EXACT ? g->m : (int64_t)P.b * g->m;
        lmax = std::max(lmax, P.l);
        kmax = std::max(kmax, P.k);
        any_hoist |= P.hoist != 0 || P.ex23 != 0;
        if (P.mode == TM_MODE_ESTIMATE && P.delta + 1 <= kWtabMax) wtab_bytes += a256(16 * (size_t)(P.delta + 1));
    }
    int smax = 1;
    const int64_t n_parts = fold_parts(hp, smax);
    size_t NWs = (size_t)std::max<int64_t>(NW, 1), Fs = (size_t)std::max<int64_t>(Fmax, 1);
    int64_t ws1 = 2 * ((NW + 2047) / 2048) + 2;
    int64_t ws2 = scan_dn_ws_elems(Fmax) + 2;
    size_t sz = a256(sizeof(QPlan) * (size_t)nq) + a256(sizeof(tm_result) * (size_t)nq) + wtab_bytes +
                9 * a256(8 * NWs) + 3 * a256(4 * NWs) + a256(8 * NWs) + a256(8 * A_N * NWs) + 3 * 256 +
                a256(sizeof(FRec<TT>) * Fs) + (any_hoist ? 3 : 1) * a256(8 * Fs) + a256(8 * (size_t)ws1) +
                a256(8 * (size_t)ws2) +
                a256(4 * (Fs / 32 + 1)) + a256(8 * (Fs / 4 + 2)) + a256(4 * Fs) +
                a256(sizeof(ShiftSums) * (size_t)n_parts);
    cudaError_t e = cudaMalloc(&b->scratch, sz);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_res, sizeof(tm_result) * (size_t)nq);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int rc = cuda_status(e, "tm_batch_create", __FILE__, __LINE__);
        batch_release(b);
        return rc;
    }
    char* p = (char*)b->scratch;
    auto take = [&](size_t bytes) { char* r = p; p += a256(bytes); return (void*)r; };
    QPlan* dplans = (QPlan*)take(sizeof(QPlan) * (size_t)nq);
    tm_result* dres = (tm_result*)take(sizeof(tm_result) * (size_t)nq);
    for (int i = 0; i < nq; i++) {
        QPlan& P = hp[(size_t)i];
        if (P.l > 0 && P.mode == TM_MODE_ESTIMATE && P.delta + 1 <= kWtabMax)
            P.wtab = (const uint64_t*)take(16 * (size_t)(P.delta + 1));
    }
    WinDev W;
    W.lo = (int64_t*)take(8 * NWs);
    W.hi = (int64_t*)take(8 * NWs);
    W.tlo = (int64_t*)take(8 * NWs);
    W.thi = (int64_t*)take(8 * NWs);
    W.tend = (int64_t*)take(8 * NWs);
    W.start = (int64_t*)take(8 * NWs);
    W.j = (int64_t*)take(8 * NWs);
    W.nfirst = (int64_t*)take(8 * NWs);
    W.fbase = (int64_t*)take(8 * NWs);
    W.q = (int32_t*)take(4 * NWs);
    W.k = (int32_t*)take(4 * NWs);
    W.kept = (int32_t*)take(4 * NWs);
    W.qj = (double*)take(8 * NWs);
    W.acc = (unsigned long long*)take(8 * A_N * NWs);
    int64_t* dF = (int64_t*)take(8);
    int64_t* dW2 = (int64_t*)take(8);
    unsigned long long* dctr = (unsigned long long*)take(8);
    FRec<TT>* rec = (FRec<TT>*)take(sizeof(FRec<TT>) * Fs);
    int64_t* excl = (int64_t*)take(8 * Fs);
    int32_t* len32 = (int32_t*)take(4 * Fs);
    int64_t* hs_a = any_hoist ? (int64_t*)take(8 * Fs) : nullptr;
    int64_t* hs_hi = any_hoist ? (int64_t*)take(8 * Fs) : nullptr;
    int64_t* wsp1 = (int64_t*)take(8 * (size_t)ws1);
    int64_t* wsp2 = (int64_t*)take(8 * (size_t)ws2);
    size_t nbw = Fs / 32 + 1, ncf = Fs / 4 + 2;
    int32_t* bwin = (int32_t*)take(4 * nbw);
    int64_t* cf = (int64_t*)take(8 * ncf);
    ShiftSums* dpart = (ShiftSums*)take(sizeof(ShiftSums) * (size_t)n_parts);

    cudaStream_t st = b->cap;
    int rc = TM_OK;
    auto fail = [&](cudaError_t ee, const char* what) {
        if (rc == TM_OK && ee != cudaSuccess) rc = cuda_status(ee, what, __FILE__, __LINE__);
    };
    // once: plans and weight tables
    fail(cudaMemcpyAsync(dplans, hp.data(), sizeof(QPlan) * (size_t)nq, cudaMemcpyHostToDevice, st), "plans");
    for (int i = 0; i < nq && rc == TM_OK; i++) {
        const QPlan& P = hp[(size_t)i];
        if (P.wtab) {
            int64_t n = P.delta + 1;
            k_wtab<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>((uint64_t*)P.wtab, P.delta, P.cd);
            count_launch();
            fail(cudaGetLastError(), "k_wtab");
        }
    }
    fail(cudaStreamSynchronize(st), "batch setup");
    if (rc != TM_OK) { batch_release(b); return rc; }

    // captured sequence
    const Tuning tu = tuning();
    int nsm = sm_count();
    GraphDevT<TT> G = typed<TT>(g->dev);
    if (rc == TM_OK) rc = ex_tables_for(g, hp, st, G);
    if (rc != TM_OK) { batch_release(b); return rc; }
    tm_profile pr0;
    tm_profile_last(&pr0);
    fail(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    fail(cudaMemsetAsync(W.acc, 0, 8 * A_N * NWs, st), "acc");
    fail(cudaMemsetAsync(dctr, 0, 8, st), "counter");
    if (rc == TM_OK && NW > 0) {
        unsigned gr = (unsigned)std::min<int64_t>((NW + 255) / 256, (int64_t)nsm * 16);
        k_windows<TT><<<gr, 256, 0, st>>>(G, dplans, nq, W, NW); count_launch();
        fail(cudaGetLastError(), "k_windows");
    }
    if (rc == TM_OK) rc = scan_exclusive_i64_ws(W.nfirst, W.fbase, NW, dF, wsp1, ws1, st);
    if (rc == TM_OK && Fmax > 0) {
        MatchArgs<TT> A;
        A.G = G; A.plans = dplans; A.nq = nq; A.W = W; A.NW = NW; A.F = Fmax; A.d_F = dF;
        A.rec = rec; A.excl = excl; A.hs_a = hs_a; A.hs_hi = hs_hi;
        A.d_W2 = dW2; A.counter = dctr;
        A.enum_threshold = tu.enum_threshold;
        A.chunk = tu.chunk_items;
        A.blockwin = bwin; A.chunkf = cf; A.nchunkf = (int64_t)ncf;
        int64_t gl2 = std::min<int64_t>((Fmax + 255) / 256, (int64_t)nsm * 8);
        k_blockwin<<<(unsigned)std::min<int64_t>(((int64_t)nbw + 255) / 256, (int64_t)nsm * 8), 256, 0, st>>>(
            W.fbase, NW, Fmax, dF, bwin);
        count_launch();
        k_level2<TT><<<(unsigned)std::max<int64_t>(gl2, 1), 256, match_smem_bytes(A.nq, 256), st>>>(A, rec, len32, hs_a, hs_hi); count_launch();
        fail(cudaGetLastError(), "k_level2");
        if (rc == TM_OK) rc = scan_lengths(len32, excl, Fmax, dF, dW2, wsp2, ws2, st);
        if (rc == TM_OK) {
            k_chunkf<<<(unsigned)std::min<int64_t>(((int64_t)ncf + 255) / 256, (int64_t)nsm * 8), 256, 0, st>>>(
                excl, Fmax, dF, dW2, A.chunk, (int64_t)ncf, cf);
            count_launch();
            fail(cudaGetLastError(), "k_chunkf");
        }
        if (rc == TM_OK) {
            launch_match<TT>(A, lmax, kmax, tu, nsm, st,
                             std::any_of(hp.begin(), hp.end(), [](const QPlan& P) { return plan_expands(P); }));
            fail(cudaGetLastError(), "k_match");
        }
    }
    if (rc == TM_OK) {
        launch_fold(dplans, nq, bmax, smax, W, dpart, dres, nullptr, nullptr, st);
        fail(cudaGetLastError(), "fold");
    }
    fail(cudaMemcpyAsync(b->h_res, dres, sizeof(tm_result) * (size_t)nq, cudaMemcpyDeviceToHost, st), "results");
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(st, &graph);
    fail(ee, "end capture");
    b->graph = graph;
    if (rc == TM_OK) fail(cudaGraphInstantiate(&b->exec, graph, 0), "instantiate");
    tm_profile pr1;
    tm_profile_last(&pr1);
    b->n_kernels = (int)(pr1.launches - pr0.launches);
    count_launch(-b->n_kernels);   // capture launched nothing; replays are counted
    if (rc != TM_OK) {
        cudaGetLastError();
        batch_release(b);
        return rc;
    }
    *out = b;
    return TM_OK;
}

int batch_create(const tm_graph* g, const tm_query* qs, int nq, tm_batch** out) {
    if (g && g->dev.tbytes == 4) return batch_create_t<int32_t>(g, qs, nq, out);
    return batch_create_t<int64_t>(g, qs, nq, out);
}

}  // namespace
}  // namespace tmo

extern "C" {

int tm_batch_create(const tm_graph* g, const tm_query* queries, int32_t n_queries, tm_batch** out) {
    return tmo::batch_create(g, queries, n_queries, out);
}

int tm_batch_launch(tm_batch* b, void* stream) {
    if (!b || !b->exec) { tmo::set_error("bad batch"); return TM_EINVAL; }
    TM_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    tmo::count_launch(b->n_kernels);
    return TM_OK;
}

int tm_batch_results(tm_batch* b, void* stream, tm_result* results) {
    if (!b || !results) { tmo::set_error("bad argument"); return TM_EINVAL; }
    TM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int first = b->first_err;
    for (int i = 0; i < b->nq; i++) {
        results[i] = b->h_res[i];
        if (b->qstat[(size_t)i] != TM_OK) {
            std::memset(&results[i], 0, sizeof(tm_result));
            results[i].status = b->qstat[(size_t)i];
        } else if (results[i].status != TM_OK && first == TM_OK) {
            first = results[i].status;
            tmo::set_error("query " + std::to_string(i) + ": count or weight sum overflowed 2^63");
        }
    }
    return first;
}

void tm_batch_free(tm_batch* b) { tmo::batch_release(b); }

int tm_set_ride_capacity(int64_t records) {
    if (records < 1 || records > ((int64_t)1 << 36)) {
        tmo::set_error("ride capacity outside [1, 2^36] records");
        return TM_EINVAL;
    }
    tmo::ride_capacity().store(records);
    return TM_OK;
}

}  // extern "C"
