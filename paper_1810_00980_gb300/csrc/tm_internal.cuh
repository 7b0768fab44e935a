// Internal declarations of libtmotif (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/tm.h"

namespace tmo {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// ----------------------------------------------------------------------------
// bounds-checked build
// ----------------------------------------------------------------------------
// Compiled with -DTM_CHECKED (libtmotif_checked.so), the indices the kernels derive from data
// (work items, first edges, candidates, windows, pair segments, sort positions) are checked
// against the sizes of the arrays they index.  A failed check sets its bit in the
// translation unit's device error word and the access goes to element 0 instead, so the
// kernel never touches memory outside its arrays and runs to the end; the host reads and
// clears the words with tm_check_status.  Without TM_CHECKED the checks compile to nothing.
enum CheckBit : unsigned {
    kChkQueue = 1u,     // work item / first edge beyond the batch's counts
    kChkWindow = 2u,    // window slot or query index beyond the batch's tables
    kChkView = 4u,      // position beyond an adjacency view (m entries)
    kChkNode = 8u,      // node id beyond n (offsets arrays hold n + 1 entries)
    kChkRange = 16u,    // a candidate or pair range not inside [0, m]
    kChkSort = 32u,     // a sort or scan output position beyond its array
    kChkSelf = 64u,     // the self-test's deliberate out-of-range index
};
#ifdef TM_CHECKED
static __device__ unsigned int g_tm_check_word;   // one per translation unit
__device__ __forceinline__ int64_t chk_idx(int64_t i, int64_t n, unsigned bit) {
    if ((unsigned long long)i >= (unsigned long long)n) {
        atomicOr(&g_tm_check_word, bit);
        return 0;
    }
    return i;
}
#define TM_CHK_IDX(i, n, bit) ::tmo::chk_idx((int64_t)(i), (int64_t)(n), (bit))
#define TM_CHK(cond, bit) \
    do { if (!(cond)) atomicOr(&::tmo::g_tm_check_word, (bit)); } while (0)
// the translation unit's error word, read (and cleared) from the host
#define TM_DEFINE_CHECK_WORD(fn)                                                             \
    int fn(unsigned* w, bool clear) {                                                        \
        if (cudaMemcpyFromSymbol(w, ::tmo::g_tm_check_word, sizeof(unsigned)) != cudaSuccess) \
            return TM_ECUDA;                                                                 \
        unsigned z = 0;                                                                      \
        if (clear && cudaMemcpyToSymbol(::tmo::g_tm_check_word, &z, sizeof(unsigned)) != cudaSuccess) \
            return TM_ECUDA;                                                                 \
        return TM_OK;                                                                        \
    }
#else
#define TM_CHK_IDX(i, n, bit) (i)
#define TM_CHK(cond, bit) do {} while (0)
#define TM_DEFINE_CHECK_WORD(fn) \
    int fn(unsigned* w, bool) { *w = 0; return TM_OK; }
#endif
int check_word_match(unsigned* w, bool clear);
int check_word_graph(unsigned* w, bool clear);
int check_word_prims(unsigned* w, bool clear);
int check_selftest();

// ----------------------------------------------------------------------------
// error plumbing
// ----------------------------------------------------------------------------
void set_error(const std::string& msg);
int cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define TM_CUDA(call)                                                             \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) return ::tmo::cuda_status(_e, #call, __FILE__, __LINE__); \
    } while (0)

#define TM_TRY(call)                   \
    do {                               \
        int _s = (call);               \
        if (_s != TM_OK) return _s;    \
    } while (0)

// ----------------------------------------------------------------------------
// device graph: edges sorted by time plus three time-sorted adjacency views
// ----------------------------------------------------------------------------
// Type-erased device graph: the time arrays hold int32 when every normalised
// time fits (tbytes = 4), else int64 (tbytes = 8).
struct GraphDev {
    int64_t m;
    int32_t n;
    int32_t tbytes;         // 4 or 8: element size of t, out_t, in_t, pair_t
    int64_t P;              // distinct (src, dst) pairs
    const int32_t* src;     // [m]
    const int32_t* dst;     // [m]
    const void* t;          // [m] normalised, non-decreasing
    const int64_t* out_off; // [n+1]
    const int32_t* out_nbr; // [m] destination
    const void* out_t;      // [m]
    const int64_t* in_off;  // [n+1]
    const int32_t* in_nbr;  // [m] source
    const void* in_t;       // [m]
    const int64_t* pk_off;  // [n+1] pair index range of each source
    const int32_t* pair_dst;// [P]
    const int64_t* pair_off;// [P+1]
    const void* pair_t;     // [m]
    const int32_t* out_src; // [m] source of each out-view entry (the sort key)
    const int32_t* in_dst;  // [m] destination of each in-view entry
    const int32_t* pair_pid;// [m] pair index of each pair-view entry
    const unsigned long long* hslots;  // [2*(hmask+1)]: key, then (length << 32 | begin) of the pair's segment
    unsigned long long hmask;          // hash capacity - 1 (power of two)
    // pair filter: two bits per pair in one 32-bit word; a lookup whose two bits are not both
    // set has no pair (most lookups of absent pairs end in this L2-resident array)
    const uint32_t* pfilt;             // [pfmask+1] or null
    unsigned long long pfmask;         // words - 1 (power of two)
    int32_t loops;          // 1 if some edge has src == dst
};

// The same graph with its time arrays typed (TT = int32_t or int64_t).
template <typename TT>
struct GraphDevT {
    int64_t m;
    int32_t n;
    int64_t P;
    const int32_t* src;
    const int32_t* dst;
    const TT* t;
    const int64_t* out_off;
    const int32_t* out_nbr;
    const TT* out_t;
    const int64_t* in_off;
    const int32_t* in_nbr;
    const TT* in_t;
    const int64_t* pk_off;
    const int32_t* pair_dst;
    const int64_t* pair_off;
    const TT* pair_t;
    const int32_t* out_src;
    const int32_t* in_dst;
    const int32_t* pair_pid;
    const unsigned long long* hslots;
    unsigned long long hmask;
    const uint32_t* pfilt;
    unsigned long long pfmask;
    int32_t loops;
    // two-node tables (set by the batch that needs them): over pair-view positions e,
    // exclusive prefix sums of the number of edges of e's own pair (ex_own) and of its
    // reverse pair (ex_rev) with time < t_e
    const int64_t* ex_own;  // [m+1] or null
    const int64_t* ex_rev;  // [m+1] or null
};

template <typename TT>
inline GraphDevT<TT> typed(const GraphDev& g) {
    GraphDevT<TT> r;
    r.m = g.m; r.n = g.n; r.P = g.P;
    r.src = g.src; r.dst = g.dst; r.t = (const TT*)g.t;
    r.out_off = g.out_off; r.out_nbr = g.out_nbr; r.out_t = (const TT*)g.out_t;
    r.in_off = g.in_off; r.in_nbr = g.in_nbr; r.in_t = (const TT*)g.in_t;
    r.pk_off = g.pk_off; r.pair_dst = g.pair_dst; r.pair_off = g.pair_off; r.pair_t = (const TT*)g.pair_t;
    r.out_src = g.out_src; r.in_dst = g.in_dst; r.pair_pid = g.pair_pid;
    r.hslots = g.hslots; r.hmask = g.hmask; r.loops = g.loops;
    r.pfilt = g.pfilt; r.pfmask = g.pfmask;
    r.ex_own = nullptr; r.ex_rev = nullptr;
    return r;
}

constexpr unsigned long long kHashEmpty = ~0ull;

}  // namespace tmo

struct tm_graph {
    int device;
    int64_t m;
    int32_t n;
    int64_t P;
    int64_t t_min;
    int64_t t_max;          // normalised
    int64_t bytes;
    void* block;            // one device allocation holding every array
    void* hash_block;       // the (src, dst) -> pair index hash table
    void* ex_own_block;     // the two-node tables ([m+1] each), built on first use (or null)
    void* ex_rev_block;
    tmo::GraphDev dev;
};

namespace tmo {

// ----------------------------------------------------------------------------
// motif plans
// ----------------------------------------------------------------------------
enum View : int8_t { kPair = 0, kOut = 1, kIn = 2, kAll = 3 };

struct LevelPlan {
    int8_t view;    // which adjacency view lists the candidates of this motif edge
    int8_t su, sv;  // motif node labels of u_i, v_i
    int8_t bind_u;  // u_i is first seen at this edge
    int8_t bind_v;  // v_i is first seen at this edge
    int8_t nb;      // labels 0..nb-1 are bound before this edge
    int8_t pad[2];
};

}  // namespace tmo

struct tm_motif {
    int32_t l, k;
    int32_t mu[TM_L_MAX];
    int32_t mv[TM_L_MAX];
    tmo::LevelPlan lv[TM_L_MAX];
};

namespace tmo {

// order in which a query enumerates first edges: by time (windows), or grouped
// by source / destination (positions of the out / in view) for exact queries
enum FirstOrder : int32_t { kOrdTime = 0, kOrdOut = 1, kOrdIn = 2, kOrdPair = 3 };

// QPlan::ex23 bits: a motif on two nodes with three edges, (u,v) first; the middle and
// the last edge each either repeat (u,v) or reverse it (v,u)
enum Ex23Bits : int32_t { kEx23On = 1, kEx23MidRev = 2, kEx23LastRev = 4 };

struct QPlan {
    int32_t l, k;
    int32_t mode;        // TM_MODE_*
    int32_t b;
    int32_t q_mode;
    int32_t order;       // FirstOrder
    int32_t hoist;       // 1: the last motif edge joins the first edge's two nodes
    int32_t rev;         // 1: three edges, the second binds one new node x and the last
                         //    joins x to a first-edge node: instances can be closed from
                         //    either the second or the last edge's candidates
    int32_t rev2;        // 1: four or more edges, and the same holds for the last two
    int32_t full;        // 1: windows enumerate node-grouped positions through perm
    int32_t hrev;        // 1: three edges, closing pair fixed by the first edge, and the second
                         //    edge either joins the first edge's nodes or adds one node: the
                         //    closing pair's entries can be the items instead
    int32_t ex23;        // kEx23*: two-node three-edge motif counted from the pair tables
    const int32_t* perm; // [b*m] per shift: view positions stably partitioned by window
    const int64_t* woff; // [b*(J+1)] per shift: start of each window's positions in perm
    int64_t delta;
    int64_t cd;          // c * delta (estimate), 0 for exact
    int64_t J;           // windows per shift (estimate), 1 for exact
    int64_t win_base;    // first window slot of this query
    double p;
    uint64_t seed;
    const uint64_t* wtab;// [2*(delta+1)] Q64 weights c delta / (c delta - Delta), or null
    // a segment of a streamed graph (defaults: the whole graph)
    int64_t t_off;       // window time origin minus the graph's time origin
    int64_t j_lo;        // windows j_lo+1 .. j_lo+J of every shift are processed
    int64_t own_lo;      // exact queries: first edges with time in [own_lo, own_hi)
    int64_t own_hi;
    int64_t m_total;     // |T| in q_j = r |T_j| / |T|
    int64_t sum_base;    // first per-shift sums slot of this query
    int64_t part_base;   // first partial record of the fold (shifts x slices) of this query
    // exact three-edge queries of the same motif at smaller spans, counted in the same
    // enumeration (spans dsub[0..nsub) < delta; their counts go to the A_X* accumulators)
    int32_t nsub;
    // estimate with every window kept (uniform p = 1): first edges of the whole graph in node
    // order, each clamped to its own window ((t1 - s) / cd), one accumulator slot per shift
    int32_t wclamp;
    int64_t dsub[3];
    int64_t J_all;       // wclamp: the windows per shift (J is then 1 slot)
    // estimates of the same motif riding along with this exact query: every instance this
    // query enumerates is also added, with the rider's weight, to the rider's window when it
    // lies inside a kept window of the rider and within the rider's span
    int32_t nride;
    int32_t riding;      // 1: this estimate rides along with an exact query (no first edges)
    int32_t ride_q[6];   // plan indices of the riders
    const int64_t* shifts;   // riding estimates: [b] window origins -(shift draw mod cd) - t_off
    LevelPlan lv[TM_L_MAX];
};
constexpr int kMaxSub = 3;
constexpr int kMaxRide = 6;

struct Tuning {
    int block_threads = 256;
    int blocks_per_sm = 4;
    int chunk_items = 256;
    int enum_threshold = 48;
};
Tuning& tuning();
std::atomic<int64_t>& ride_capacity();

// one query's part of a segment of a streamed graph
struct SegSpec {
    int64_t t_off;           // global time of the segment graph's time 0
    int64_t j_lo, J;         // estimate: windows j_lo+1 .. j_lo+J of every shift
    int64_t own_lo, own_hi;  // exact: first edges with (segment) time in [own_lo, own_hi)
    int64_t m_total;         // edges of the whole graph
};

// one shift's sums over the windows a batch processed (additive across segments)
struct ShiftSums {
    unsigned long long count, wlo, whi, first, cand, last, inst, kept;
    double zq, vq;
};
// a += b (the weight sum as one 128-bit integer)
__host__ __device__ inline void add_shift_sums(ShiftSums& a, const ShiftSums& b) {
    unsigned long long lo = a.wlo + b.wlo;
    a.whi += b.whi + (lo < a.wlo ? 1ull : 0ull);
    a.wlo = lo;
    a.count += b.count; a.first += b.first; a.cand += b.cand; a.last += b.last;
    a.inst += b.inst; a.kept += b.kept; a.zq += b.zq; a.vq += b.vq;
}

struct BatchOut {                 // optional per-window readback for one query
    int query = -1;
    int32_t k = 0;
    bool all_windows = false;
    tm_window_rec* recs = nullptr;
    int64_t cap = 0;
    int64_t n_out = 0;
    int64_t shift = 0;
    const SegSpec* seg = nullptr; // per query, or null (whole graph)
    ShiftSums* sums = nullptr;    // host: per query, per shift (exact: one), or null
    const int32_t* riding = nullptr;          // per query: 1 if it rides along (no first edges)
    const int32_t* ride_q = nullptr;          // per query: [kMaxRide] plan indices of its riders, -1 unused
    const int32_t* nsub = nullptr;            // per query: spans counted alongside (exact)
    const int64_t* sub_delta = nullptr;       // [nq][kMaxSub]
    unsigned long long* sub_count = nullptr;  // host out: [nq][kMaxSub]
};

int run_batch(const tm_graph* g, const tm_query* qs, int nq, tm_result* res,
              cudaStream_t st, BatchOut* dbg);
int count_plain(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count);
// query checks of tm_run_batch against a graph whose normalised times end at t_max
int check_query(int64_t t_max, const tm_query& q, std::string& why);

// primitives (prims.cu)
int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total,
                       cudaStream_t st);
int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                     int64_t n, int bits, cudaStream_t st);
// the same with 64-bit values; the sorted arrays end in (keys, vals) or (keys_tmp, vals_tmp),
// returned through kres / vres (no copy back)
int radix_sort_kv64(uint32_t* keys, uint64_t* vals, uint32_t* keys_tmp, uint64_t* vals_tmp, int64_t n,
                    int bits, cudaStream_t st, uint32_t** kres, uint64_t** vres);
// exclusive scan with the tile sums in caller workspace (2 * ceil(n/2048) int64, n <= 2048^2)
int scan_exclusive_i64_ws(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total,
                          int64_t* ws, int64_t ws_elems, cudaStream_t st);

// exclusive scan of the first *d_n (<= n_max) elements, the count read on the
// device; workspace of scan_dn_ws_elems(n_max) int64 (no allocation, capturable)
int64_t scan_dn_ws_elems(int64_t n_max);
// exclusive scan of 32-bit lengths into 64-bit offsets (the first *d_n, or n_max when d_n is
// null); workspace scan_dn_ws_elems(n_max), or null to allocate it on the stream
int scan_lengths(const int32_t* in, int64_t* out, int64_t n_max, const int64_t* d_n, int64_t* d_total,
                 int64_t* ws, int64_t ws_elems, cudaStream_t st);
int scan_exclusive_i64_dn(const int64_t* in, int64_t* out, int64_t n_max, const int64_t* d_n,
                          int64_t* d_total, int64_t* ws, int64_t ws_elems, cudaStream_t st);

int sm_count();
// the graph's two-node tables (own, rev: [m+1] each) that are asked for, each built on
// the first call that needs it (thread-safe; synchronises the stream when it builds);
// null for an empty graph or when not asked for
int ensure_ex_tables(tm_graph* g, cudaStream_t st, bool need_own, bool need_rev, const int64_t** own,
                     const int64_t** rev);
// device memory pool (prims.cu): raise the default pool's release threshold once
// per device; pool_free returns a stream-ordered block on an internal stream
int pool_prepare(int dev);
void pool_free(void* p, int dev);
int pool_trim();   // also frees the scratch arenas that no call holds
// scratch of one call, leased from a per-device grow-only arena (slot >= 0) or, when every
// arena is held, a pool block (slot < 0); usable on st from acquire to release
struct ScratchLease {
    void* p = nullptr;
    int slot = -1;
    int dev = 0;
};
int scratch_acquire(size_t bytes, cudaStream_t st, ScratchLease& L);
void scratch_release(ScratchLease& L, cudaStream_t st);

// profiling (abi.cu): phase events of the last batch / graph build, launch counter
bool profiling();
void store_profile_batch(double windows_ms, double level2_ms, double match_ms, double fold_ms,
                         double batch_ms, int64_t match_items, int64_t first_edges, double sizing_ms,
                         double scan_ms, double ride_ms = 0.0);
void store_profile_graph(double graph_ms);
void store_profile_ride_records(int64_t n);
void count_launch(int n = 1);

// NVTX ranges naming the host-side phases of a call (graph build, window partition, second-edge
// ranges, matcher, fold), one after another, so that a profiler can select them (for example
// ncu --nvtx --nvtx-include "tm_match/"); without a tool attached each call costs a branch
struct NvtxPhases {
    nvtxRangeId_t id = 0;
    bool open = false;
    void next(const char* name) {
        if (open) nvtxRangeEnd(id);
        open = name != nullptr;
        if (open) id = nvtxRangeStartA(name);
    }
    ~NvtxPhases() { next(nullptr); }
};

// CUDA events on a stream, created only while profiling is on
struct PhaseEvents {
    static constexpr int kMax = 12;
    cudaEvent_t ev[kMax];
    int n = 0;
    bool on = false;
    explicit PhaseEvents(bool enable) : on(enable) {
        if (on)
            for (int i = 0; i < kMax; i++)
                if (cudaEventCreate(&ev[i]) != cudaSuccess) on = false;
    }
    ~PhaseEvents() {
        if (on)
            for (int i = 0; i < kMax; i++) cudaEventDestroy(ev[i]);
    }
    int mark(cudaStream_t st) {
        if (!on || n >= kMax) return -1;
        cudaEventRecord(ev[n], st);
        return n++;
    }
    double ms(int a, int b) const {
        if (!on || a < 0 || b < 0) return 0.0;
        float x = 0.f;
        cudaEventElapsedTime(&x, ev[a], ev[b]);
        return (double)x;
    }
};

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------
// first index p in [lo, hi) with a[p] > v (a sorted non-decreasingly; any integer element type)
template <typename T>
__device__ __forceinline__ int64_t upper_bound_i64(const T* __restrict__ a, int64_t lo, int64_t hi,
                                                   int64_t v) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)__ldg(a + mid) <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// first index p in [lo, hi) with a[p] >= v
template <typename T>
__device__ __forceinline__ int64_t lower_bound_i64(const T* __restrict__ a, int64_t lo, int64_t hi,
                                                   int64_t v) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t lo,
                                                   int64_t hi, int32_t v) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// SplitMix64 (Steele, Lea & Flood 2014): output n (n >= 1) of the generator
// seeded with s is mix(s + n * 0x9E3779B97F4A7C15).
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_output(uint64_t seed, uint64_t n) {
    return sm64_mix(seed + n * 0x9E3779B97F4A7C15ull);
}
// draw n of repetition k of a query seeded with `seed`
__host__ __device__ __forceinline__ uint64_t draw(uint64_t seed, uint64_t k, uint64_t n) {
    return sm64_output(sm64_output(seed, k + 1), n + 1);
}

// the time-sorted segment [a, b) of pair (u, v) in the pair view, by one hash lookup
// (after the pair filter, which answers most lookups of absent pairs from L2)
template <typename TT>
__device__ __forceinline__ bool pair_segment(const GraphDevT<TT>& G, int32_t u, int32_t v, int64_t& a,
                                             int64_t& b, bool filter = true) {
    unsigned long long key = ((unsigned long long)(uint32_t)u << 32) | (uint32_t)v;
    unsigned long long h0 = sm64_mix(key);
    if (filter && G.pfilt) {   // callers that know the pair exists skip the filter
        uint32_t w = __ldg(G.pfilt + ((h0 >> 32) & G.pfmask));
        if (!((w >> (h0 & 31)) & (w >> ((h0 >> 5) & 31)) & 1u)) {
            a = b = 0;
            return false;
        }
    }
    unsigned long long h = h0 & G.hmask;
    for (unsigned long long it = 0; it <= G.hmask; it++) {
        ulonglong2 sl = __ldg(reinterpret_cast<const ulonglong2*>(G.hslots) + h);
        if (sl.x == key) {
            a = (int64_t)(uint32_t)sl.y;
            b = a + (int64_t)(sl.y >> 32);
            TM_CHK(b <= G.m, kChkRange);
#ifdef TM_CHECKED
            if (b > G.m) a = b = 0;   // an empty segment instead of one beyond the view
#endif
            return true;
        }
        unsigned long long k = sl.x;
        if (k == kHashEmpty) break;
        h = (h + 1) & G.hmask;
    }
    a = b = 0;
    return false;
}

}  // namespace tmo
