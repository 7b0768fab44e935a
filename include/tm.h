/*
 * tm.h -- C ABI of libtmotif: delta-temporal motif counting and the
 * interval-sampling estimator on one GB300 (sm_103a).
 *
 * Paper: P. Liu, A. R. Benson, M. Charikar, "A sampling framework for
 * counting temporal motifs", WSDM 2019 (arXiv:1810.00980).
 *
 * Conventions for every call
 *   - Returns an int status: TM_OK (0) or one of the TM_E* codes below.
 *     tm_strerror() names a code; tm_last_error() gives the calling thread's
 *     last detailed message.  No C++ exception crosses this boundary.
 *   - Host pointers are caller-owned and only read during the call unless a
 *     call says otherwise.  Device pointers ("d_" prefix) must be CUDA device
 *     memory on the current device.
 *   - Handles (tm_graph, tm_motif, tm_server) are library-owned; free them
 *     with the matching *_free / *_destroy call.  A graph must outlive every
 *     query and server that uses it.  Graphs and motifs are read-only after
 *     creation, so concurrent queries on them are safe.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.
 *   - Timestamps are int64 and must be sorted non-decreasingly.  Node ids
 *     are int32 in [0, n_nodes).
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TM_OK 0
#define TM_EINVAL 1      /* bad argument: NULL, l<1, l>TM_L_MAX, k>TM_K_MAX, motif self-loop,
                            delta<0, c<1, p outside (0,1], estimate with delta=0, c*delta overflow */
#define TM_EUNSORTED 2   /* timestamps not sorted non-decreasingly */
#define TM_ERANGE 3      /* node id outside [0, n_nodes) */
#define TM_ENOMEM 4      /* device or host allocation failed */
#define TM_EADMIT 5      /* server: query footprint can never fit the admission budget */
#define TM_ETIMEOUT 6    /* a bounded wait expired */
#define TM_ESTACK 7      /* reserved: matcher stack exhausted */
#define TM_EOVERFLOW 8   /* a count or weight sum reached 2^63 */
#define TM_ECUDA 9       /* CUDA runtime error (see tm_last_error) */
#define TM_PENDING 10    /* server: ticket not finished yet */
#define TM_ENOTFOUND 11  /* server: unknown ticket or graph id */
#define TM_ECANCELLED 12 /* server: ticket cancelled */
#define TM_ESHUTDOWN 13  /* server: shutting down */

#define TM_L_MAX 8       /* most motif edges */
#define TM_K_MAX 8       /* most motif nodes */

#define TM_MODE_EXACT 0
#define TM_MODE_ESTIMATE 1

#define TM_Q_UNIFORM 0   /* q_j = p for every window */
#define TM_Q_EDGES 1     /* q_j = min(1, r |T_j| / |T|) with r = the query's p field (Eq. 9) */
/* TM_Q_AUTO: uniform q_j = p with p chosen for a target relative error (the query's p field,
 * in (0, 1)) at 95 % confidence (z = 1.96).  A pilot estimate with p0 = TM_AUTO_PILOT_P and
 * the same c and b (seed ^ TM_AUTO_PILOT_SEED_XOR) gives Z0 and var_hat0; since var_hat is
 * unbiased for Var[Z | s] = sum_j Y_j^2 (1 - p)/p (Lemma 4.4), S2 = var_hat0 p0 / (1 - p0)
 * estimates sum_j Y_j^2, and the smallest p with z sqrt(S2 (1 - p) / (p b)) <= target Z0 is
 *   p = 1 / (1 + b (target Z0 / z)^2 / S2), clamped to [p0, 1] (p = 1 when Z0 = 0).
 * The shift variance (Lemma 4.2) is not part of this target.  The query then runs with that
 * p and its own seed; results.p_used reports it.  tm_run_batch and the server only (a
 * prepared batch or a stream rejects it with TM_EINVAL). */
#define TM_Q_AUTO 2
#define TM_AUTO_PILOT_P 0.05
#define TM_AUTO_PILOT_SEED_XOR 0xA5A5A5A5A5A5A5A5ull

typedef struct tm_graph tm_graph;
typedef struct tm_motif tm_motif;
typedef struct tm_server tm_server;

typedef struct {
    int64_t m;            /* temporal edges */
    int32_t n_nodes;
    int32_t pad0;
    int64_t n_pairs;      /* static edges (distinct ordered pairs), Section 2 */
    int64_t t_min;        /* smallest timestamp; stored times are t - t_min */
    int64_t t_max;        /* largest normalised timestamp */
    int64_t device_bytes; /* device memory held by the graph */
} tm_graph_info;

/* One window I_j of Eq. 1 as seen by the estimator (Algorithm 1). */
typedef struct {
    int32_t k;            /* repetition (shift) index, 0-based */
    int32_t kept;         /* 1 if Uniform(0,1) < q_j */
    int64_t j;            /* window index, 1-based */
    int64_t start;        /* a_j = s + (j-1) c delta (normalised time); end = start + c delta - 1 */
    int64_t lo, hi;       /* T_j = edges [lo, hi) of the time-sorted edge list */
    int64_t count;        /* exact number of instances inside I_j (0 if not kept) */
    uint64_t w_int;       /* W_j = w(I_j) of Eq. 3 in unsigned fixed point: */
    uint64_t w_frac;      /*   W_j ~= w_int + w_frac * 2^-64 (each term rounded down) */
    double q;             /* q_j used for the keep decision */
} tm_window_rec;

typedef struct {
    const tm_motif* motif;
    int64_t delta;        /* time span delta (Def. 2.2) */
    int32_t mode;         /* TM_MODE_EXACT or TM_MODE_ESTIMATE */
    int32_t c;            /* window width factor: windows are c*delta ticks wide (Eq. 1) */
    double p;             /* TM_Q_UNIFORM: keep probability; TM_Q_EDGES: the constant r;
                             TM_Q_AUTO: the target relative error */
    uint64_t seed;        /* random draws of Algorithm 1 (SplitMix64, see tm_estimate) */
    int32_t b;            /* number of shifts averaged (Algorithm 1 outer loop), >= 1 */
    int32_t q_mode;       /* TM_Q_UNIFORM, TM_Q_EDGES or TM_Q_AUTO */
} tm_query;

typedef struct {
    int32_t status;       /* TM_OK or an error for this query */
    int32_t pad0;
    int64_t count;        /* exact: C_M; estimate: instances found inside kept windows */
    double estimate;      /* exact: (double)count; estimate: mean over shifts of Z_k */
    int64_t windows;      /* windows considered (exact: 1) */
    int64_t windows_kept;
    int64_t first_edges;  /* first-edge candidates scanned (E_first) */
    int64_t cand_edges;   /* adjacency entries read at intermediate levels (N_cand) */
    int64_t last_ranges;  /* partial instances closed at the last motif edge (N_last) */
    int64_t inst_read;    /* last-edge entries read one by one (estimate mode) */
    double var_hat;       /* estimate: unbiased estimate of Var[Z | s] averaged over shifts
                             (Lemma 4.4: sum_j Q_j Y_j^2 (1-q_j)/q_j^2); exact: 0 */
    double shift_var;     /* estimate with b >= 2: sample variance of the b per-shift Z_k (an
                             unbiased estimate of Var[Z_k], shift variance included), so
                             estimate +- 1.96 sqrt(shift_var / b) is a 95 % interval; else 0 */
    double p_used;        /* estimate: the p (or r) the windows were kept with; exact: 1 */
} tm_result;

/* ---- errors -------------------------------------------------------------- */
const char* tm_strerror(int status);
const char* tm_last_error(void);
const char* tm_version(void);

/* ---- graphs ----------------------------------------------------------------
 * Temporal graph T of Section 2: m tuples (src[i], dst[i], t[i]).  Repeated
 * (src, dst) pairs and equal timestamps are allowed.  The library copies the
 * edges, subtracts t_min (Algorithm 1 assumes times start at 0) and builds,
 * on the device, three time-sorted adjacency views: by source, by
 * destination, and by (source, destination) pair (the static edges of
 * Section 2).
 *   n_nodes: number of node ids, or -1 to use max id + 1.
 * Errors: TM_EINVAL (NULL with m>0, m<0, m >= 2^31), TM_EUNSORTED, TM_ERANGE,
 * TM_ENOMEM, TM_ECUDA.  On error *out is left NULL.
 */
int tm_graph_load(const int32_t* src, const int32_t* dst, const int64_t* t, int64_t m,
                  int32_t n_nodes, tm_graph** out);
/* Same from device arrays, ordered on `stream`; returns after the build. */
int tm_graph_load_device(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_t,
                         int64_t m, int32_t n_nodes, void* stream, tm_graph** out);
void tm_graph_free(tm_graph* g);
int tm_graph_get_info(const tm_graph* g, tm_graph_info* info);

/* ---- motifs ----------------------------------------------------------------
 * Temporal motif of Def. 2.1 as its ordered edge list (u_1,v_1)..(u_l,v_l):
 * msrc[i] -> mdst[i], i < l.  Labels are any int32; they are renumbered in
 * order of first appearance, so k = number of distinct labels.
 * Errors: TM_EINVAL (NULL, l<1, l>TM_L_MAX, k>TM_K_MAX, msrc[i]==mdst[i]).
 */
int tm_motif_compile(const int32_t* msrc, const int32_t* mdst, int32_t l, tm_motif** out);
void tm_motif_free(tm_motif* m);

/* ---- queries ---------------------------------------------------------------
 * tm_count_exact: C_M, the number of delta-instances (Def. 2.2: l distinct
 * edges in strictly increasing time order, t_l - t_1 <= delta, a node map
 * that is injective both ways).  Synchronous.  TM_EOVERFLOW if C_M >= 2^63.
 */
int tm_count_exact(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count);

/* The same count by the plain one-thread-per-first-edge kernel (no batching,
 * no load balancing); a baseline for the batched matcher.  Synchronous. */
int tm_count_exact_plain(const tm_graph* g, const tm_motif* m, int64_t delta, int64_t* count);

/* tm_estimate: Algorithm 1 with one shift (b = 1) and uniform q_j = p.
 * Shift s = -(h0 mod c*delta) and keep draws U_j = (h_j >> 11) 2^-53, window
 * kept iff U_j < p, where h_n is output n+1 of SplitMix64 seeded with output
 * k+1 of SplitMix64 seeded with `seed` (k = 0 here).  Returns
 * Z = sum over kept windows j of sum_i count_i / ((1 - Delta_i/(c delta)) p).
 * Requires delta >= 1, c >= 1, 0 < p <= 1.  Synchronous. */
int tm_estimate(const tm_graph* g, const tm_motif* m, int64_t delta, int32_t c, double p,
                uint64_t seed, double* estimate);

/* Per-window detail of repetition k of one estimate (parity and debugging):
 * writes up to `cap` records for the kept windows (all windows if
 * all_windows != 0) in increasing j, sets *n_out to the number available and
 * *shift to s.  Synchronous. */
int tm_estimate_windows(const tm_graph* g, const tm_motif* m, int64_t delta, int32_t c,
                        double p, uint64_t seed, int32_t k, int32_t all_windows,
                        tm_window_rec* out, int64_t cap, int64_t* n_out, int64_t* shift);

/* Batched form: every window of every query in one partition + one
 * persistent matcher launch, ordered on `stream`.  results[i] receives query
 * i's result.  The call returns once the results are on the host.  Per-query
 * problems set results[i].status and make the call return the first one. */
int tm_run_batch(const tm_graph* g, const tm_query* queries, int32_t n_queries,
                 tm_result* results, void* stream);

/* ---- exact count without allocation ------------------------------------------
 * The paper has no counterpart to this call; it exists for deployments.
 *
 * tm_count_exact_noalloc returns the same C_M as tm_count_exact, for callers
 * that may not allocate device memory while they answer queries: a process
 * whose device memory is reserved up front by another allocator (for example
 * a framework's caching allocator that owns the whole GPU, or a fixed memory
 * budget), or latency-critical code that forbids allocation after start-up
 * because cudaMalloc/cudaFree can block and synchronise the device.  It calls
 * no cudaMalloc, cudaFree or other allocating routine.  Its scratch is one
 * static device array compiled into the library, TM_NOALLOC_SCRATCH_BYTES
 * (about 14.7 MB) on every GPU that loads the library, held until the process
 * exits.
 *   g       graph with at most TM_NOALLOC_MAX_EDGES edges (else TM_EINVAL), loaded on
 *           the current device (else TM_EINVAL: the array used is the current device's).
 *   stream  cudaStream_t as void* (NULL: legacy default stream); the work is
 *           ordered on it and the call returns once *count is on the host.
 *   count   host pointer receiving C_M.
 * The first call on a device resolves the array's device address with
 * cudaGetSymbolAddress (which can load the library's device code); make that
 * first call before any stream capture.  Every call uses the same array and
 * leaves its contents behind (each call clears what must start at zero), so
 * calls that overlap on the GPU -- on different streams or threads -- race;
 * serialise them.  Errors: TM_EINVAL, TM_ENOMEM, TM_ECUDA, TM_EOVERFLOW;
 * tm_last_error is not updated. */
#define TM_NOALLOC_MAX_EDGES 262144
#define TM_NOALLOC_SCRATCH_BYTES 14687232
int tm_count_exact_noalloc(const tm_graph* g, const tm_motif* m, int64_t delta, void* stream,
                           int64_t* count);

/* ---- streaming (graphs held in host memory) -------------------------------------
 * The sampling framework needs only the edges of one window at a time, so windows can
 * be processed chronologically as the edges stream in (Section 4, the remark on
 * streaming after the choice of q_j).  tm_stream_run evaluates a batch of queries over
 * a time-sorted edge list in HOST memory without ever holding the whole graph on the
 * device: the list is cut into chronological segments of about `segment_edges` edges
 * (cut between distinct times; consecutive segments overlap by up to max(delta, 2 c
 * delta) of time), each segment is copied to the device -- the copy of the next
 * segment overlaps the matching of the current one -- and built into a graph; each
 * estimate window is counted in the one segment that holds it whole, and each exact
 * query's first edge in the one segment that holds its delta-span.  A segment grows
 * past `segment_edges` when a single window or span holds more edges.
 *   src, dst, t   host arrays of m edges, t sorted non-decreasingly (pinned memory is
 *                 copied directly; pageable memory through pinned staging buffers)
 *   n_nodes       node ids must lie in [0, n_nodes)
 *   queries       as tm_run_batch; results[i] is identical to tm_run_batch's on the
 *                 whole graph for counts and uniform-q estimates (the per-shift Q64
 *                 weight sums add exactly); TM_Q_EDGES estimates and var_hat agree to
 *                 rounding (their per-window terms are summed in another order)
 *   stats         optional (NULL allowed)
 * Synchronous.  Device memory: about 2 x 16 B x segment_edges of input buffers plus one
 * segment graph and its batch scratch.  Errors as tm_graph_load and tm_run_batch. */
typedef struct tm_stream_stats {
    int64_t segments;          /* segment graphs built */
    int64_t edges_copied;      /* edges copied to the device (overlaps counted again) */
    int64_t max_segment_edges; /* largest segment */
    double wall_ms;            /* the whole call */
    double copy_wait_ms;       /* time spent waiting for a segment's copy after matching */
} tm_stream_stats;
int tm_stream_run(const int32_t* src, const int32_t* dst, const int64_t* t, int64_t m, int32_t n_nodes,
                  const tm_query* queries, int32_t n_queries, int64_t segment_edges, tm_result* results,
                  tm_stream_stats* stats);

/* ---- prepared batches (CUDA graph) ----------------------------------------------
 * A fixed set of queries on one graph, prepared once and launched many times:
 * plans and weight tables are built at creation, scratch is sized for the worst
 * case (every window of every shift kept), and the launch sequence -- window
 * partition, first-edge scan, second-edge ranges, persistent matcher, fold,
 * result copy -- is captured in one CUDA graph whose replay needs no host
 * synchronisation.  Results are identical to tm_run_batch on the same queries.
 *   tm_batch_create   captures on a private stream; TM_ENOMEM if the worst-case
 *                     scratch does not fit.  The graph and motifs must outlive it.
 *   tm_batch_launch   enqueues one replay on `stream` (asynchronous).
 *   tm_batch_results  waits for `stream`, then copies the last replay's results.
 * One replay at a time per batch: replays on different streams share scratch. */
typedef struct tm_batch tm_batch;
int tm_batch_create(const tm_graph* g, const tm_query* queries, int32_t n_queries, tm_batch** out);
int tm_batch_launch(tm_batch* b, void* stream);
int tm_batch_results(tm_batch* b, void* stream, tm_result* results);
void tm_batch_free(tm_batch* b);

/* ---- tuning ----------------------------------------------------------------
 * Matcher launch parameters.  0 keeps the current value.  The autotuner
 * (tm_autotune) writes these after timing candidates on a graph. */
typedef struct {
    int32_t block_threads;     /* threads per block of the matcher (multiple of 32) */
    int32_t blocks_per_sm;     /* persistent blocks per SM */
    int32_t chunk_items;       /* level-2 items a warp takes per queue grab (multiple of 32) */
    int32_t enum_threshold;    /* last-level ranges longer than this are counted by
                                  subtraction instead of being read entry by entry */
} tm_tuning;
int tm_get_tuning(tm_tuning* out);
int tm_set_tuning(const tm_tuning* in);
/* No counterpart in the paper: the matcher leaves the work of an exact query's riders (the
 * estimates riding along with it) and smaller spans to a second kernel, as one record per group
 * of instances, in a device buffer taken from the batch scratch.  `records` (1 .. 2^36) sets how
 * many records the next batches make room for (default 2^23: 192 MB with 32-bit times, 256 MB
 * with 64-bit times).  A batch that needs more runs a second time with room for all of them and
 * raises the capacity to that, so the setting changes only memory and time, never a result.
 * Returns TM_EINVAL outside that range. */
int tm_set_ride_capacity(int64_t records);
/* Time candidate tunings on `queries` over g (results discarded) and keep the
 * fastest; *best receives it.  Candidates: 128 or 256 threads, 4, 6, 8 or 12
 * blocks per SM, chunks of 256, 1024 or 4096 items, and (only when the batch
 * has an exact query whose last edge is counted on a node view) thresholds 32
 * and 128; each is timed as the median of three whole batches.  Synchronous. */
int tm_autotune(const tm_graph* g, const tm_query* queries, int32_t n_queries, tm_tuning* best);

/* ---- profiling ----------------------------------------------------------------
 * When enabled, every batch and graph build records CUDA events around its
 * phases on the stream it runs on; tm_profile_last returns the durations of
 * the most recent ones (any thread).  `launches` counts every kernel launch
 * the library has made since it was loaded (enabled or not). */
typedef struct {
    double graph_ms;        /* last graph build: validation through the last view */
    double windows_ms;      /* last batch: weight tables + window partition + first-edge scan */
    double level2_ms;       /* second-edge ranges of every first edge (k_level2) */
    double match_ms;        /* the persistent matcher launch */
    double fold_ms;         /* per-query combination */
    double batch_ms;        /* whole batch, first launch to results on the host */
    int64_t match_items;    /* second-edge candidates the matcher processed */
    int64_t first_edges;    /* first edges the batch scanned */
    int64_t launches;       /* kernel launches since load */
    double sizing_ms;       /* last batch: first-edge count to the host, per-edge scratch,
                               window-of-block index (between windows_ms and level2_ms) */
    double scan_ms;         /* last batch: scan of the range lengths, chunk index */
    double ride_ms;         /* last batch: the deferred pass of riders and smaller spans (k_ride),
                               after the matcher; 0 when no exact query carried any */
    int64_t ride_records;   /* last batch: records the matcher left to that pass */
} tm_profile;
int tm_profile_enable(int32_t on);
/* Return device memory that freed graphs and batch scratch left in the library's
 * stream-ordered pool (kept mapped for reuse) to the device, with the grow-only scratch
 * buffers (up to four per device, each as large as the largest graph build or batch
 * scratch it served) that no running call holds.  Synchronises the device. */
int tm_release_cached_memory(void);
int tm_profile_last(tm_profile* out);

/* ---- bounds-checked build ------------------------------------------------------
 * The paper has no counterpart: this is a debugging aid.  The library is also built as
 * libtmotif_checked.so (compiled with TM_CHECKED), where every index the kernels derive
 * from data -- work items, first edges, adjacency candidates, windows, query indices,
 * node ids into the offset arrays, pair segments, sort and offset positions -- is
 * checked against the size of the array it indexes.  A failed check sets one bit of a
 * device error word and redirects the access to element 0 of that array (no access
 * outside it, no trap), so the call completes and its results are unreliable.
 *   tm_check_status   *word = the OR of the bits set since the last clear:
 *                     1 work item or first edge, 2 window or query, 4 view position,
 *                     8 node id, 16 candidate or pair range, 32 sort or offset position,
 *                     64 the self-test; clear != 0 resets them.  Synchronous.
 *   tm_check_selftest runs one deliberately out-of-range index (one past a one-element
 *                     device array) through the check, which reads element 0 and sets
 *                     bit 64, so that a test can see the mechanism work.
 * In the ordinary build both return TM_EINVAL (*word = 0). */
int tm_check_status(uint32_t* word, int32_t clear);
int tm_check_selftest(void);

/* ---- serving -----------------------------------------------------------------
 * A server keeps graphs resident, accepts queries from any thread, and runs
 * them in continuous batches: queries that arrive while a batch is on the GPU
 * are admitted into the next one as device memory frees up (admission by the
 * query's estimated footprint against `mem_budget_bytes`), and batches run
 * on `n_streams` streams so their device work overlaps. */
typedef struct {
    int64_t mem_budget_bytes;  /* scratch admitted at once; 0 = 4 GiB */
    int32_t max_batch;         /* most queries in one batch; 0 = 256 */
    int32_t n_streams;         /* concurrent batches, 1..4; 0 = 2 */
} tm_serve_cfg;

int tm_serve_create(const tm_serve_cfg* cfg, tm_server** out);
/* The server does not own the graph; it must stay alive until the server is destroyed. */
int tm_serve_attach_graph(tm_server* s, const tm_graph* g, int32_t* graph_id);
/* Queue one query; *ticket identifies it.  Thread-safe. */
int tm_serve_submit(tm_server* s, int32_t graph_id, const tm_query* q, uint64_t* ticket);
/* TM_PENDING until the ticket finishes; then its final status with *r
 * filled, after which the ticket is forgotten (a later poll: TM_ENOTFOUND). */
int tm_serve_poll(tm_server* s, uint64_t ticket, tm_result* r);
/* Block until the ticket finishes (then as tm_serve_poll) or timeout_ms
 * passes (TM_ETIMEOUT; the ticket stays valid). */
int tm_serve_wait(tm_server* s, uint64_t ticket, int64_t timeout_ms, tm_result* r);
/* Block until any ticket finishes -- tickets come back in completion order --
 * or timeout_ms passes (TM_ETIMEOUT).  Sets *ticket and *r, returns the
 * ticket's final status and forgets it (as tm_serve_poll). */
int tm_serve_wait_any(tm_server* s, int64_t timeout_ms, uint64_t* ticket, tm_result* r);
/* Cancel a ticket that has not started: it finishes with TM_ECANCELLED.
 * TM_PENDING if it is already running or done. */
int tm_serve_cancel(tm_server* s, uint64_t ticket);
/* Drain the queue, stop the scheduler and free everything. */
void tm_serve_destroy(tm_server* s);

#ifdef __cplusplus
}
#endif

#endif /* TM_H */
