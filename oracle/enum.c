/*
 * CPU oracle for delta-temporal motif counting -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  It shares nothing with the CUDA library: no headers,
 * no helpers, no tables.
 *
 * What it computes (Liu, Benson & Charikar, "A sampling framework for
 * counting temporal motifs", Section 2):
 *   Def. 2.2  a time-ordered sequence of l distinct temporal edges
 *             (w_i, x_i, t_i) is a delta-instance of the motif
 *             (u_1,v_1),...,(u_l,v_l) when one node map sends u_i -> w_i and
 *             v_i -> x_i for every i, distinct motif nodes to distinct graph
 *             nodes, and t_l - t_1 <= delta.
 *   Def. 2.3  its duration is t_l - t_1, with t_1 < t_2 < ... < t_l.
 *   Section 4 intro: the exact counter returns count-duration pairs
 *             {(count_i, Delta_i)}; here that is a histogram hist[Delta].
 *
 * Readings where the paper is silent: timestamps must increase strictly
 * (equal times never share an instance); the node map is injective both
 * ways; an edge whose two endpoints coincide can never match a motif edge
 * (motifs have no self-loops).
 *
 * Method: for every candidate first edge, extend a partial instance one motif
 * edge at a time in time order.  The candidates for motif edge i are the
 * edges with time in (t_{i-1}, min(t_1 + delta, window end)].  When an
 * endpoint of motif edge i is already mapped, only that graph node's
 * outgoing (or incoming) edge list is scanned, which enumerates exactly the
 * same sequences as scanning all edges and rejecting the ones whose
 * endpoint differs.  Each completed sequence adds one to hist[t_l - t_1].
 *
 * Restricting edges to a window [w_lo, w_hi] gives the exact count on the
 * subgraph T_j of Algorithm 1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_MAXK 64

typedef struct {
    /* graph, time-sorted */
    const int32_t *src, *dst;
    const int64_t *t;
    int64_t m;
    int32_t n;
    /* per-node edge lists (edge indices in increasing index = time order) */
    const int64_t *out_beg, *out_e, *in_beg, *in_e;
    /* motif */
    const int32_t *mu, *mv;
    int l, k;
    int64_t delta, w_lo, w_hi;
} or_problem;

typedef struct {
    const or_problem *P;
    int64_t f_lo, f_hi, f_step_start, f_stride; /* first edges f_lo + f_step_start + r*f_stride */
    int64_t *hist;            /* length delta+1, may be NULL */
    int64_t count;
    int64_t visited;          /* partial instances extended (work measure) */
    int32_t phi[OR_MAXK];     /* motif node -> graph node, -1 if unmapped */
} or_worker;

static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

/* first position p in idx[lo, hi) whose edge time is > tv (idx lists are time-sorted) */
static int64_t first_after(const int64_t *t, const int64_t *idx, int64_t lo, int64_t hi, int64_t tv)
{
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t e = idx ? idx[mid] : mid;
        if (t[e] <= tv) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int node_is_mapped(const or_worker *W, int32_t g)
{
    for (int a = 0; a < W->P->k; a++)
        if (W->phi[a] == g) return 1;
    return 0;
}

static void extend(or_worker *W, int i, int64_t t1, int64_t tprev)
{
    const or_problem *P = W->P;
    if (i == P->l) {
        W->count++;
        if (W->hist) W->hist[tprev - t1]++;
        return;
    }
    W->visited++;
    int a = P->mu[i], b = P->mv[i];
    int64_t upper = min64(t1 + P->delta, P->w_hi);
    const int64_t *idx;
    int64_t lo, hi;
    if (W->phi[a] >= 0) {
        idx = P->out_e; lo = P->out_beg[W->phi[a]]; hi = P->out_beg[W->phi[a] + 1];
    } else if (W->phi[b] >= 0) {
        idx = P->in_e; lo = P->in_beg[W->phi[b]]; hi = P->in_beg[W->phi[b] + 1];
    } else {
        idx = NULL; lo = 0; hi = P->m;
    }
    for (int64_t p = first_after(P->t, idx, lo, hi, tprev); p < hi; p++) {
        int64_t e = idx ? idx[p] : p;
        int64_t te = P->t[e];
        if (te > upper) break;
        int32_t ws = P->src[e], xd = P->dst[e];
        if (ws == xd) continue;
        int new_a = 0, new_b = 0;
        if (W->phi[a] >= 0) { if (W->phi[a] != ws) continue; }
        else { if (node_is_mapped(W, ws)) continue; new_a = 1; }
        if (W->phi[b] >= 0) { if (W->phi[b] != xd) continue; }
        else { if (node_is_mapped(W, xd)) continue; new_b = 1; }
        if (new_a) W->phi[a] = ws;
        if (new_b) W->phi[b] = xd;
        extend(W, i + 1, t1, te);
        if (new_a) W->phi[a] = -1;
        if (new_b) W->phi[b] = -1;
    }
}

static void *run_worker(void *arg)
{
    or_worker *W = (or_worker *)arg;
    const or_problem *P = W->P;
    for (int a = 0; a < OR_MAXK; a++) W->phi[a] = -1;
    for (int64_t f = W->f_lo + W->f_step_start; f < W->f_hi; f += W->f_stride) {
        int64_t t1 = P->t[f];
        if (t1 < P->w_lo || t1 > P->w_hi) continue;
        int32_t ws = P->src[f], xd = P->dst[f];
        if (ws == xd) continue;
        int a = P->mu[0], b = P->mv[0];
        W->phi[a] = ws;
        W->phi[b] = xd;
        extend(W, 1, t1, t1);
        W->phi[a] = -1;
        W->phi[b] = -1;
    }
    return NULL;
}

/*
 * Count delta-instances of the motif (mu[i] -> mv[i], i < l, labels 0..k-1)
 * among edges with time in [w_lo, w_hi], taking as first edge only indices
 * in [f_lo, f_hi).  hist (length delta+1, may be NULL) receives the
 * duration histogram.  visited (may be NULL) receives the number of partial
 * instances extended.  Returns the count, or -1 on bad arguments.
 */
int64_t oracle_count(const int32_t *src, const int32_t *dst, const int64_t *t, int64_t m,
                     int32_t n_nodes, const int32_t *mu, const int32_t *mv, int32_t l,
                     int64_t delta, int64_t w_lo, int64_t w_hi, int64_t f_lo, int64_t f_hi,
                     int64_t *hist, int64_t *visited, int32_t n_threads)
{
    if (l < 1 || delta < 0 || m < 0 || n_nodes < 0) return -1;
    int k = 0;
    for (int i = 0; i < l; i++) {
        if (mu[i] < 0 || mv[i] < 0 || mu[i] >= OR_MAXK || mv[i] >= OR_MAXK || mu[i] == mv[i]) return -1;
        if (mu[i] + 1 > k) k = mu[i] + 1;
        if (mv[i] + 1 > k) k = mv[i] + 1;
    }
    if (f_lo < 0) f_lo = 0;
    if (f_hi > m) f_hi = m;
    if (n_threads < 1) n_threads = 1;

    /* per-node edge lists by plain bucketing in index order */
    int64_t *out_beg = calloc((size_t)n_nodes + 1, sizeof(int64_t));
    int64_t *in_beg = calloc((size_t)n_nodes + 1, sizeof(int64_t));
    int64_t *out_e = malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
    int64_t *in_e = malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
    int64_t *fill = calloc((size_t)n_nodes + 1, sizeof(int64_t));
    if (!out_beg || !in_beg || !out_e || !in_e || !fill) return -2;
    for (int64_t e = 0; e < m; e++) {
        if (src[e] < 0 || src[e] >= n_nodes || dst[e] < 0 || dst[e] >= n_nodes) return -1;
        out_beg[src[e] + 1]++;
        in_beg[dst[e] + 1]++;
    }
    for (int32_t v = 0; v < n_nodes; v++) { out_beg[v + 1] += out_beg[v]; in_beg[v + 1] += in_beg[v]; }
    for (int64_t e = 0; e < m; e++) out_e[out_beg[src[e]] + fill[src[e]]++] = e;
    memset(fill, 0, sizeof(int64_t) * ((size_t)n_nodes + 1));
    for (int64_t e = 0; e < m; e++) in_e[in_beg[dst[e]] + fill[dst[e]]++] = e;
    free(fill);

    or_problem P = {src, dst, t, m, n_nodes, out_beg, out_e, in_beg, in_e, mu, mv, l, k,
                    delta, w_lo, w_hi};
    or_worker *W = calloc((size_t)n_threads, sizeof(or_worker));
    pthread_t *th = calloc((size_t)n_threads, sizeof(pthread_t));
    for (int i = 0; i < n_threads; i++) {
        W[i].P = &P;
        W[i].f_lo = f_lo; W[i].f_hi = f_hi; W[i].f_step_start = i; W[i].f_stride = n_threads;
        W[i].hist = hist ? calloc((size_t)delta + 1, sizeof(int64_t)) : NULL;
    }
    if (n_threads == 1) run_worker(&W[0]);
    else {
        for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, run_worker, &W[i]);
        for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    }
    int64_t total = 0, vis = 0;
    for (int i = 0; i < n_threads; i++) {
        total += W[i].count;
        vis += W[i].visited;
        if (hist) {
            for (int64_t d = 0; d <= delta; d++) hist[d] += W[i].hist[d];
            free(W[i].hist);
        }
    }
    if (visited) *visited = vis;
    free(W); free(th);
    free(out_beg); free(in_beg); free(out_e); free(in_e);
    return total;
}
