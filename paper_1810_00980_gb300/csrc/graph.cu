// Graph ingest and adjacency build (temporal graph T and its static graph G,
// Section 2).  Everything after the input copy runs on the device: validation,
// normalisation t' = t - t_min (Algorithm 1 assumes times start at 0), three
// stable radix sorts that leave every adjacency segment in time order, and
// segment offsets found from the sorted keys.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "tm_internal.cuh"

namespace tmo {
namespace {

constexpr int kThreads = 256;

unsigned grid_for(int64_t n, int per_sm = 8) {
    int64_t g = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// flags[0]: unsorted, flags[1]: id out of range (n_nodes given) or negative,
// flags[2]: max node id
__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const int64_t* __restrict__ t, int64_t m, int32_t n_nodes,
                           int32_t* __restrict__ flags) {
    int32_t mx = -1;
    int bad_sort = 0, bad_id = 0, loop = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = src[i], d = dst[i];
        if (s < 0 || d < 0 || (n_nodes >= 0 && (s >= n_nodes || d >= n_nodes))) bad_id = 1;
        mx = max(mx, max(s, d));
        loop |= s == d;
        if (i > 0 && t[i] < t[i - 1]) bad_sort = 1;
    }
    if (__any_sync(kFull, bad_sort) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1);
    if (__any_sync(kFull, bad_id) && (threadIdx.x & 31) == 0) atomicOr(&flags[1], 1);
    if (__any_sync(kFull, loop) && (threadIdx.x & 31) == 0) atomicOr(&flags[3], 1);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&flags[2], mx);
}

template <typename TT>
__global__ void k_ingest(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                         const int64_t* __restrict__ t, int64_t m, int64_t tmin,
                         int32_t* __restrict__ gs, int32_t* __restrict__ gd, TT* __restrict__ gt,
                         uint32_t* __restrict__ key_src, uint32_t* __restrict__ key_dst,
                         uint32_t* __restrict__ iota_a, uint32_t* __restrict__ iota_b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = src[i], d = dst[i];
        gs[i] = s;
        gd[i] = d;
        gt[i] = (TT)(t[i] - tmin);
        key_src[i] = (uint32_t)s;
        key_dst[i] = (uint32_t)d;
        iota_a[i] = (uint32_t)i;
        iota_b[i] = (uint32_t)i;
    }
}

// off[v] = first position whose sorted key is >= v, for v in [0, n]
__global__ void k_offsets(const uint32_t* __restrict__ keys, int64_t m, int32_t n,
                          int64_t* __restrict__ off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t prev = i == 0 ? -1 : (int64_t)keys[i - 1];
        int64_t cur = i == m ? (int64_t)n : (int64_t)keys[i];
        for (int64_t v = prev + 1; v <= cur; v++) off[TM_CHK_IDX(v, (int64_t)n + 1, kChkNode)] = i;
    }
}

// out_nbr/out_t (or in_*) gathered through the sort permutation
template <typename TT>
__global__ void k_gather_view(const uint32_t* __restrict__ perm, const int32_t* __restrict__ other,
                              const TT* __restrict__ t, int64_t m, int32_t* __restrict__ nbr,
                              TT* __restrict__ tv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = perm[i];
        nbr[i] = other[e];
        tv[i] = t[e];
    }
}

// pair view: positions sorted by (src, dst, time); head flag where the pair changes
template <typename TT>
__global__ void k_pair_heads(const uint32_t* __restrict__ perm, const int32_t* __restrict__ src,
                             const int32_t* __restrict__ dst, const TT* __restrict__ t,
                             int64_t m, int64_t* __restrict__ head, TT* __restrict__ pair_t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = perm[i];
        pair_t[i] = t[e];
        int64_t h = 1;
        if (i > 0) {
            uint32_t f = perm[i - 1];
            h = (src[e] != src[f] || dst[e] != dst[f]) ? 1 : 0;
        }
        head[i] = h;
    }
}

// ---- views for 32-bit times: each sort carries its payload (the other endpoint and the
// time packed in 64 bits) instead of an edge index, so no view is gathered through a
// permutation (random reads of the edge arrays) after the sort
__global__ void k_ingest_kv(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            const int64_t* __restrict__ t, int64_t m, int64_t tmin,
                            int32_t* __restrict__ gs, int32_t* __restrict__ gd, int32_t* __restrict__ gt,
                            uint32_t* __restrict__ key_src, uint32_t* __restrict__ key_dst,
                            uint64_t* __restrict__ pay_out, uint64_t* __restrict__ pay_in) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = src[i], d = dst[i];
        uint32_t tt = (uint32_t)(t[i] - tmin);
        gs[i] = s;
        gd[i] = d;
        gt[i] = (int32_t)tt;
        key_src[i] = (uint32_t)s;
        key_dst[i] = (uint32_t)d;
        pay_out[i] = (uint64_t)(uint32_t)d | ((uint64_t)tt << 32);
        pay_in[i] = (uint64_t)(uint32_t)s | ((uint64_t)tt << 32);
    }
}

// a sorted view's neighbour and time arrays from its payload
__global__ void k_split_view(const uint64_t* __restrict__ pay, int64_t m, int32_t* __restrict__ nbr,
                             int32_t* __restrict__ tv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t v = pay[i];
        nbr[i] = (int32_t)(uint32_t)v;
        tv[i] = (int32_t)(uint32_t)(v >> 32);
    }
}

// the in view as sort input for the pair view: key = source, payload = destination | time
__global__ void k_pair_keys(const int32_t* __restrict__ in_nbr, const uint32_t* __restrict__ in_dst,
                            const int32_t* __restrict__ in_t, int64_t m, uint32_t* __restrict__ key,
                            uint64_t* __restrict__ pay) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = (uint32_t)in_nbr[i];
        pay[i] = (uint64_t)in_dst[i] | ((uint64_t)(uint32_t)in_t[i] << 32);
    }
}

// pair view from (source, destination | time) sorted by source: times, head flags
__global__ void k_pair_heads_kv(const uint32_t* __restrict__ key, const uint64_t* __restrict__ pay,
                                int64_t m, int64_t* __restrict__ head, int32_t* __restrict__ pair_t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t v = pay[i];
        pair_t[i] = (int32_t)(uint32_t)(v >> 32);
        head[i] = (i == 0 || key[i] != key[i - 1] || (uint32_t)v != (uint32_t)pay[i - 1]) ? 1 : 0;
    }
}

__global__ void k_pair_index_kv(const uint32_t* __restrict__ key, const uint64_t* __restrict__ pay,
                                const int64_t* __restrict__ head, const int64_t* __restrict__ pid_excl,
                                int64_t m, int32_t* __restrict__ pair_dst, int64_t* __restrict__ pair_off,
                                int32_t* __restrict__ pair_src) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (head[i]) {
            int64_t p = pid_excl[i];
            pair_dst[p] = (int32_t)(uint32_t)pay[i];
            pair_off[p] = i;
            pair_src[p] = (int32_t)key[i];
        }
    }
}

// pid_excl[i] = number of heads before i; a head at i starts pair pid_excl[i]
__global__ void k_pair_index(const uint32_t* __restrict__ perm, const int32_t* __restrict__ dst,
                             const int64_t* __restrict__ head, const int64_t* __restrict__ pid_excl,
                             int64_t m, int32_t* __restrict__ pair_dst, int64_t* __restrict__ pair_off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (head[i]) {
            int64_t p = pid_excl[i];
            pair_dst[p] = dst[perm[i]];
            pair_off[p] = i;
        }
    }
}

// Open-addressing hash of the static edges: key (src << 32 | dst) -> the pair's
// time-sorted segment of pair_t, stored in the slot as (begin, length) so that a
// lookup is one 16-byte load.  Capacity is a power of two >= 2 P, so every probe
// chain ends at an empty slot.
__global__ void k_hash_insert(const int32_t* __restrict__ pair_src, const int32_t* __restrict__ pair_dst,
                              const int64_t* __restrict__ pair_off, int64_t P,
                              unsigned long long* __restrict__ slots, unsigned long long mask,
                              uint32_t* __restrict__ filt, unsigned long long fmask) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = ((unsigned long long)(uint32_t)pair_src[p] << 32) | (uint32_t)pair_dst[p];
        unsigned long long seg = ((unsigned long long)(uint32_t)(pair_off[p + 1] - pair_off[p]) << 32) |
                                 (uint32_t)pair_off[p];
        unsigned long long h0 = sm64_mix(key);
        atomicOr(filt + ((h0 >> 32) & fmask), (1u << (h0 & 31)) | (1u << ((h0 >> 5) & 31)));
        unsigned long long h = h0 & mask;
        for (unsigned long long it = 0; it <= mask; it++) {
            unsigned long long prev = atomicCAS(&slots[2 * h], kHashEmpty, key);
            if (prev == kHashEmpty) {
                slots[2 * h + 1] = seg;
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__global__ void k_pair_src(const uint32_t* __restrict__ perm, const int32_t* __restrict__ src,
                           const int64_t* __restrict__ head, const int64_t* __restrict__ pid_excl,
                           int64_t m, int32_t* __restrict__ pair_src) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        if (head[i]) pair_src[pid_excl[i]] = src[perm[i]];
}

// pair index of every pair-view position: heads up to and including it, minus one
__global__ void k_pair_pid(const int64_t* __restrict__ head, const int64_t* __restrict__ pid_excl, int64_t m,
                           int32_t* __restrict__ pair_pid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        pair_pid[i] = (int32_t)(pid_excl[i] + head[i] - 1);
}

__global__ void k_pair_tail(int64_t* __restrict__ pair_off, const int64_t* __restrict__ P, int64_t m) {
    pair_off[*P] = m;
}

// pk_off[u] = pair index of the first pair whose source is >= u
__global__ void k_pk_off(const int64_t* __restrict__ out_off, const int64_t* __restrict__ head,
                         const int64_t* __restrict__ pid_excl, const int64_t* __restrict__ P,
                         int64_t m, int32_t n, int64_t* __restrict__ pk_off) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t pos = out_off[u];
        pk_off[u] = pos >= m ? *P : pid_excl[pos];
    }
}

int bits_for(int32_t n) {
    int b = 0;
    while (b < 31 && ((int64_t)1 << b) < (int64_t)n) b++;
    return b;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// A second stream of the calling thread on device dev, with two events, for the in-view sort
// that runs beside the out-view sort (null when it cannot be created: the sorts then share st)
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream* side_stream(int dev) {
    constexpr int kDevs = 64;
    thread_local SideStream ss[kDevs];
    if (dev < 0 || dev >= kDevs) return nullptr;
    SideStream& x = ss[dev];
    if (!x.s) {
        if (cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            x.s = nullptr;
            return nullptr;
        }
    }
    return &x;
}

int build_graph(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_t, int64_t m,
                int32_t n_nodes, cudaStream_t st, tm_graph** out) {
    if (!out) { set_error("out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    if (m < 0 || m >= ((int64_t)1 << 31) - 1) { set_error("m outside [0, 2^31-1)"); return TM_EINVAL; }
    if (m > 0 && (!d_src || !d_dst || !d_t)) { set_error("NULL edge array"); return TM_EINVAL; }
    if (n_nodes < -1) { set_error("n_nodes < -1"); return TM_EINVAL; }

    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    PhaseEvents pe(profiling());
    NvtxPhases nv;
    nv.next("tm_graph_build");
    int ev0 = pe.mark(st);
    int64_t tmin = 0, tmax = 0;
    int32_t loops = 0;
    int32_t n = n_nodes < 0 ? 0 : n_nodes;
    if (m > 0) {
        int32_t* flags = nullptr;
        TM_CUDA(cudaMallocAsync((void**)&flags, 4 * sizeof(int32_t), st));
        int32_t init[4] = {0, 0, -1, 0};
        TM_CUDA(cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, st));
        k_validate<<<grid_for(m), kThreads, 0, st>>>(d_src, d_dst, d_t, m, n_nodes, flags); count_launch();
        TM_CUDA(cudaGetLastError());
        int32_t hf[4];
        int64_t tt[2];
        TM_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaMemcpyAsync(&tt[0], d_t, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaMemcpyAsync(&tt[1], d_t + (m - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TM_CUDA(cudaStreamSynchronize(st));
        cudaFreeAsync(flags, st);
        if (hf[0]) { set_error("timestamps are not sorted non-decreasingly"); return TM_EUNSORTED; }
        if (hf[1]) { set_error("node id outside [0, n_nodes)"); return TM_ERANGE; }
        tmin = tt[0];
        tmax = tt[1] - tt[0];
        if (tt[1] < tt[0] || tmax >= ((int64_t)1 << 61)) { set_error("time span >= 2^61"); return TM_EINVAL; }
        if (n_nodes < 0) n = hf[2] + 1;
        loops = hf[3];
    }

    // ---- one allocation for the resident graph
    size_t nN = (size_t)n + 1, M = (size_t)m;
    // time arrays hold int32 when every normalised time fits, else int64
    const int tb = tmax <= (int64_t)INT32_MAX ? 4 : 8;
    size_t sz_i32m = align256(4 * M), sz_i64m = align256(8 * M), sz_off = align256(8 * nN);
    size_t sz_tm = align256((size_t)tb * M);
    size_t total = 2 * sz_i32m + sz_tm          // src, dst, t
                 + sz_off + sz_i32m + sz_tm     // out view
                 + sz_off + sz_i32m + sz_tm     // in view
                 + sz_off + sz_i32m + align256(8 * (M + 1)) + sz_tm   // pair view (P <= m)
                 + 3 * sz_i32m;                                          // view keys, pair index
    tm_graph* g = new (std::nothrow) tm_graph();
    if (!g) { set_error("host allocation failed"); return TM_ENOMEM; }
    g->device = dev;
    g->m = m;
    g->n = n;
    g->t_min = tmin;
    g->t_max = tmax;
    g->bytes = (int64_t)total;
    pool_prepare(dev);
    cudaError_t e = cudaMallocAsync(&g->block, total, st);
    if (e != cudaSuccess) {
        delete g;
        return cuda_status(e, "cudaMalloc(graph)", __FILE__, __LINE__);
    }
    char* p = (char*)g->block;
    auto take = [&](size_t bytes) { char* r = p; p += bytes; return (void*)r; };
    int32_t* gs = (int32_t*)take(sz_i32m);
    int32_t* gd = (int32_t*)take(sz_i32m);
    void* gt = take(sz_tm);
    int64_t* out_off = (int64_t*)take(sz_off);
    int32_t* out_nbr = (int32_t*)take(sz_i32m);
    void* out_t = take(sz_tm);
    int64_t* in_off = (int64_t*)take(sz_off);
    int32_t* in_nbr = (int32_t*)take(sz_i32m);
    void* in_t = take(sz_tm);
    int64_t* pk_off = (int64_t*)take(sz_off);
    int32_t* pair_dst = (int32_t*)take(sz_i32m);
    int64_t* pair_off = (int64_t*)take(align256(8 * (M + 1)));
    void* pair_t = take(sz_tm);
    int32_t* out_src = (int32_t*)take(sz_i32m);
    int32_t* in_dst = (int32_t*)take(sz_i32m);
    int32_t* pair_pid = (int32_t*)take(sz_i32m);

    GraphDev& G = g->dev;
    G.m = m; G.n = n; G.tbytes = tb; G.loops = loops;
    G.src = gs; G.dst = gd; G.t = gt;
    G.out_off = out_off; G.out_nbr = out_nbr; G.out_t = out_t;
    G.in_off = in_off; G.in_nbr = in_nbr; G.in_t = in_t;
    G.pk_off = pk_off; G.pair_dst = pair_dst; G.pair_off = pair_off; G.pair_t = pair_t;
    G.out_src = out_src; G.in_dst = in_dst; G.pair_pid = pair_pid;
    G.hslots = nullptr; G.hmask = 0;
    G.pfilt = nullptr; G.pfmask = 0;
    g->hash_block = nullptr;
    g->ex_own_block = nullptr;
    g->ex_rev_block = nullptr;

    int rc = TM_OK;
    if (m == 0) {
        TM_CUDA(cudaMemsetAsync(out_off, 0, 8 * nN, st));
        TM_CUDA(cudaMemsetAsync(in_off, 0, 8 * nN, st));
        TM_CUDA(cudaMemsetAsync(pk_off, 0, 8 * nN, st));
        TM_CUDA(cudaMemsetAsync(pair_off, 0, 8, st));
        TM_CUDA(cudaStreamSynchronize(st));
        g->P = 0;
        G.P = 0;
        *out = g;
        return TM_OK;
    }

    // ---- scratch: keys/values for three sorts (double-buffered) + pair scan
    uint32_t *ks, *kd, *va, *vb, *kt, *vt;
    int64_t *head, *pid, *dP;
    // index path: 6 u32 + 2 i64 per edge; payload path (32-bit times): 3 u32 + 3 u64
    // (the payload path takes a fourth key and value array when the in-view sort runs on a side
    // stream beside the out-view sort)
    SideStream* side = tb == 4 ? side_stream(dev) : nullptr;
    const int kv = side ? 4 : 3;
    size_t scratch = std::max(6 * align256(4 * M) + 2 * sz_i64m, kv * align256(4 * M) + kv * sz_i64m) + 256;
    ScratchLease lease;
    int lrc = scratch_acquire(scratch, st, lease);
    if (lrc != TM_OK) {
        cudaStreamSynchronize(st);
        pool_free(g->block, dev);
        delete g;
        return lrc;
    }
    char* q = (char*)lease.p;
    auto takes = [&](size_t bytes) { char* r = q; q += align256(bytes); return (void*)r; };
    ks = (uint32_t*)takes(4 * M);
    kd = (uint32_t*)takes(4 * M);
    va = (uint32_t*)takes(4 * M);
    vb = (uint32_t*)takes(4 * M);
    kt = (uint32_t*)takes(4 * M);
    vt = (uint32_t*)takes(4 * M);
    head = (int64_t*)takes(8 * M);
    pid = (int64_t*)takes(8 * M);
    dP = (int64_t*)((char*)lease.p + scratch - 256);

    int bits = bits_for(n);
    unsigned gr = grid_for(m);
    // the launches below that move timestamps, for the chosen element type
    auto typed_launch = [&](auto tag, int which, const uint32_t* perm, const int32_t* other, int32_t* nbr,
                            void* tv) {
        using TT = decltype(tag);
        if (which == 0)
            k_ingest<TT><<<gr, kThreads, 0, st>>>(d_src, d_dst, d_t, m, tmin, gs, gd, (TT*)gt, ks, kd, va, vb);
        else if (which == 1)
            k_gather_view<TT><<<gr, kThreads, 0, st>>>(perm, other, (const TT*)gt, m, nbr, (TT*)tv);
        else
            k_pair_heads<TT><<<gr, kThreads, 0, st>>>(perm, gs, gd, (const TT*)gt, m, head, (TT*)tv);
        count_launch();
    };
    auto tlaunch = [&](int which, const uint32_t* perm, const int32_t* other, int32_t* nbr, void* tv) {
        if (tb == 4) typed_launch(int32_t{}, which, perm, other, nbr, tv);
        else typed_launch(int64_t{}, which, perm, other, nbr, tv);
    };
    uint32_t* psrc = nullptr;   // pair sources (the hash keys), in pair order
    if (tb == 4) {
        // payload path: scratch laid out as three u32 and three u64 arrays
        char* q2 = (char*)lease.p;
        auto take2 = [&](size_t bytes) { char* r = q2; q2 += align256(bytes); return (void*)r; };
        uint32_t* k0 = (uint32_t*)take2(4 * M);
        uint32_t* k1 = (uint32_t*)take2(4 * M);
        uint32_t* k2 = (uint32_t*)take2(4 * M);
        uint32_t* k3 = side ? (uint32_t*)take2(4 * M) : k0;
        uint64_t* p0 = (uint64_t*)take2(8 * M);
        uint64_t* p1 = (uint64_t*)take2(8 * M);
        uint64_t* p2 = (uint64_t*)take2(8 * M);
        uint64_t* p3 = side ? (uint64_t*)take2(8 * M) : p0;
        uint32_t* kr = nullptr;
        uint64_t* pr = nullptr;
        k_ingest_kv<<<gr, kThreads, 0, st>>>(d_src, d_dst, d_t, m, tmin, gs, gd, (int32_t*)gt, k0, k1, p0, p1);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        // in view: (destination; source | time) stably sorted by destination -- on the side
        // stream when there is one, beside the out view's sort
        cudaStream_t sin = side ? side->s : st;
        if (rc == TM_OK && side && (cudaEventRecord(side->fork, st) != cudaSuccess ||
                                    cudaStreamWaitEvent(sin, side->fork, 0) != cudaSuccess))
            rc = TM_ECUDA;
        uint32_t* kr_in = nullptr;
        uint64_t* pr_in = nullptr;
        auto in_view = [&]() {
            if (rc == TM_OK) rc = radix_sort_kv64(k1, p1, k3, p3, m, bits, sin, &kr_in, &pr_in);
            if (rc == TM_OK) {
                k_offsets<<<grid_for(m + 1), kThreads, 0, sin>>>(kr_in, m, n, in_off); count_launch();
                k_split_view<<<gr, kThreads, 0, sin>>>(pr_in, m, in_nbr, (int32_t*)in_t); count_launch();
                if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
                if (rc == TM_OK && cudaMemcpyAsync(in_dst, kr_in, 4 * M, cudaMemcpyDeviceToDevice, sin) != cudaSuccess)
                    rc = TM_ECUDA;
            }
            if (side && cudaEventRecord(side->join, sin) != cudaSuccess && rc == TM_OK) rc = TM_ECUDA;
        };
        if (side) in_view();
        // out view: (source; destination | time) stably sorted by source
        if (rc == TM_OK) rc = radix_sort_kv64(k0, p0, k2, p2, m, bits, st, &kr, &pr);
        if (rc == TM_OK) {
            k_offsets<<<grid_for(m + 1), kThreads, 0, st>>>(kr, m, n, out_off); count_launch();
            k_split_view<<<gr, kThreads, 0, st>>>(pr, m, out_nbr, (int32_t*)out_t); count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
            if (rc == TM_OK && cudaMemcpyAsync(out_src, kr, 4 * M, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                rc = TM_ECUDA;
        }
        if (side) {
            // the pair view needs the in view, and reuses the in-view sort's arrays
            if (cudaStreamWaitEvent(st, side->join, 0) != cudaSuccess && rc == TM_OK) rc = TM_ECUDA;
        } else {
            in_view();   // after the out view, in its arrays (k0 / p0 are free again)
        }
        // pair view: the in view stably re-sorted by source = (source, destination, time)
        if (rc == TM_OK) {
            k_pair_keys<<<gr, kThreads, 0, st>>>(in_nbr, (const uint32_t*)in_dst, (const int32_t*)in_t, m, k2, p2);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
        if (rc == TM_OK) rc = radix_sort_kv64(k2, p2, k0, p0, m, bits, st, &kr, &pr);
        // heads and pair indices in the u64 arrays the sort left free; sources in a free u32 one
        int64_t* hd = (int64_t*)p1;
        int64_t* pd = (int64_t*)(pr == p2 ? p0 : p2);
        psrc = kr == k2 ? k0 : k2;
        if (rc == TM_OK) {
            k_pair_heads_kv<<<gr, kThreads, 0, st>>>(kr, pr, m, hd, (int32_t*)pair_t); count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
        if (rc == TM_OK) rc = scan_exclusive_i64(hd, pd, m, dP, st);
        if (rc == TM_OK) {
            k_pair_index_kv<<<gr, kThreads, 0, st>>>(kr, pr, hd, pd, m, pair_dst, pair_off, (int32_t*)psrc);
            count_launch();
            k_pair_tail<<<1, 1, 0, st>>>(pair_off, dP, m); count_launch();
            k_pk_off<<<grid_for((int64_t)n + 1), kThreads, 0, st>>>(out_off, hd, pd, dP, m, n, pk_off); count_launch();
            k_pair_pid<<<gr, kThreads, 0, st>>>(hd, pd, m, pair_pid); count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
    } else {
        tlaunch(0, nullptr, nullptr, nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        // out view: edges stably sorted by source (time order kept inside a source)
        if (rc == TM_OK) rc = radix_sort_pairs(ks, va, kt, vt, m, bits, st);
        if (rc == TM_OK) {
            k_offsets<<<grid_for(m + 1), kThreads, 0, st>>>(ks, m, n, out_off); count_launch();
            tlaunch(1, va, gd, out_nbr, out_t);
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
            if (rc == TM_OK && cudaMemcpyAsync(out_src, ks, 4 * M, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                rc = TM_ECUDA;
        }
        // in view: stably sorted by destination
        if (rc == TM_OK) rc = radix_sort_pairs(kd, vb, kt, vt, m, bits, st);
        if (rc == TM_OK) {
            k_offsets<<<grid_for(m + 1), kThreads, 0, st>>>(kd, m, n, in_off); count_launch();
            tlaunch(1, vb, gs, in_nbr, in_t);
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
            if (rc == TM_OK && cudaMemcpyAsync(in_dst, kd, 4 * M, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                rc = TM_ECUDA;
        }
        // pair view: the in-view order stably re-sorted by source = (src, dst, time)
        if (rc == TM_OK) {
            tlaunch(1, vb, gs, (int32_t*)ks, head);   // sources in in-view order; times go to scratch
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
        if (rc == TM_OK) rc = radix_sort_pairs(ks, vb, kt, vt, m, bits, st);
        if (rc == TM_OK) {
            tlaunch(2, vb, nullptr, nullptr, pair_t);
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
        if (rc == TM_OK) rc = scan_exclusive_i64(head, pid, m, dP, st);
        if (rc == TM_OK) {
            k_pair_index<<<gr, kThreads, 0, st>>>(vb, gd, head, pid, m, pair_dst, pair_off); count_launch();
            k_pair_tail<<<1, 1, 0, st>>>(pair_off, dP, m); count_launch();
            k_pk_off<<<grid_for((int64_t)n + 1), kThreads, 0, st>>>(out_off, head, pid, dP, m, n, pk_off); count_launch();
            k_pair_src<<<gr, kThreads, 0, st>>>(vb, gs, head, pid, m, (int32_t*)kt); count_launch();
            psrc = kt;
            k_pair_pid<<<gr, kThreads, 0, st>>>(head, pid, m, pair_pid); count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
    }
    int64_t P = 0;
    if (rc == TM_OK) {
        e = cudaMemcpyAsync(&P, dP, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_status(e, "graph build", __FILE__, __LINE__);
    }
    // pair hash: capacity the next power of two >= 2 P; then the pair filter: 8 bits per pair
    // (a power of two of 32-bit words), at most 32 MB so that it stays in L2
    if (rc == TM_OK) {
        unsigned long long cap = 2;
        while (cap < 2ull * (unsigned long long)P) cap <<= 1;
        unsigned long long fw = 1;
        while (fw < ((unsigned long long)P + 3) / 4 && fw < (1ull << 23)) fw <<= 1;
        e = cudaMallocAsync(&g->hash_block, 16 * cap + 4 * fw, st);
        if (e != cudaSuccess) rc = cuda_status(e, "cudaMalloc(pair hash)", __FILE__, __LINE__);
        if (rc == TM_OK) {
            g->bytes += (int64_t)(16 * cap + 4 * fw);
            G.hslots = (const unsigned long long*)g->hash_block;
            G.hmask = cap - 1;
            uint32_t* filt = (uint32_t*)((char*)g->hash_block + 16 * cap);
            G.pfilt = filt;
            G.pfmask = fw - 1;
            e = cudaMemsetAsync(g->hash_block, 0xff, 16 * cap, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(filt, 0, 4 * fw, st);
            if (e == cudaSuccess) {
                k_hash_insert<<<grid_for(P), kThreads, 0, st>>>((const int32_t*)psrc, pair_dst, pair_off, P,
                                                               (unsigned long long*)g->hash_block, cap - 1,
                                                               filt, fw - 1);
                count_launch();
                e = cudaGetLastError();
            }
            int ev1 = pe.mark(st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_status(e, "pair hash build", __FILE__, __LINE__);
            if (rc == TM_OK && pe.on) store_profile_graph(pe.ms(ev0, ev1));
        }
    }
    scratch_release(lease, st);
    if (rc != TM_OK) {
        cudaStreamSynchronize(st);
        pool_free(g->block, dev);
        pool_free(g->hash_block, dev);
        delete g;
        return rc;
    }
    g->P = P;
    G.P = P;
    *out = g;
    return TM_OK;
}

// Two-node tables.  For pair-view position e of pair (u, v) at time t_e:
//   own[e] = number of (u, v) edges with time < t_e, rev[e] = number of (v, u) edges with
//   time < t_e;
// each then turned into exclusive prefix sums over all positions.  The source of pair-view
// position e is out_src[e]: both views group the edges by source in the same ranges.
template <typename TT>
__global__ void k_ex_rank(GraphDevT<TT> G, int reverse, int64_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < G.m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t pid = G.pair_pid[e];
        int64_t te = (int64_t)G.pair_t[e];
        if (!reverse) {
            int64_t pa = G.pair_off[pid];
            int64_t r = e - pa;
            if (e > pa && (int64_t)G.pair_t[e - 1] == te) r = lower_bound_i64(G.pair_t, pa, e, te) - pa;
            out[e] = r;
        } else {
            int32_t u = G.out_src[e], v = G.pair_dst[pid];
            int64_t ra, rb;
            out[e] = pair_segment(G, v, u, ra, rb) ? lower_bound_i64(G.pair_t, ra, rb, te) - ra : 0;
        }
    }
}

std::mutex g_ex_mu;

int build_ex_table(tm_graph* g, int reverse, cudaStream_t st, void** blk_out) {
    size_t n1 = (size_t)g->m + 1;
    void* blk = nullptr;
    TM_CUDA(cudaMallocAsync(&blk, align256(8 * n1), st));
    int64_t* a = (int64_t*)blk;
    int rc = TM_OK;
    cudaError_t e = cudaMemsetAsync(a + g->m, 0, 8, st);
    if (e == cudaSuccess) {
        if (g->dev.tbytes == 4) k_ex_rank<int32_t><<<grid_for(g->m), kThreads, 0, st>>>(typed<int32_t>(g->dev), reverse, a);
        else k_ex_rank<int64_t><<<grid_for(g->m), kThreads, 0, st>>>(typed<int64_t>(g->dev), reverse, a);
        count_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = cuda_status(e, "two-node table", __FILE__, __LINE__);
    if (rc == TM_OK) rc = scan_exclusive_i64(a, a, (int64_t)n1, nullptr, st);
    if (rc == TM_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_status(e, "two-node table", __FILE__, __LINE__);
    }
    if (rc != TM_OK) {
        cudaStreamSynchronize(st);
        pool_free(blk, g->device);
        return rc;
    }
    g->bytes += (int64_t)align256(8 * n1);
    *blk_out = blk;
    return TM_OK;
}

}  // namespace

int ensure_ex_tables(tm_graph* g, cudaStream_t st, bool need_own, bool need_rev, const int64_t** own,
                     const int64_t** rev) {
    std::lock_guard<std::mutex> lk(g_ex_mu);
    *own = *rev = nullptr;
    if (g->m == 0) return TM_OK;
    int rc = TM_OK;
    if (need_own && !g->ex_own_block) rc = build_ex_table(g, 0, st, &g->ex_own_block);
    if (rc == TM_OK && need_rev && !g->ex_rev_block) rc = build_ex_table(g, 1, st, &g->ex_rev_block);
    if (rc != TM_OK) return rc;
    if (need_own) *own = (const int64_t*)g->ex_own_block;
    if (need_rev) *rev = (const int64_t*)g->ex_rev_block;
    return TM_OK;
}

}  // namespace tmo

extern "C" {

int tm_graph_load_device(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_t, int64_t m,
                         int32_t n_nodes, void* stream, tm_graph** out) {
    return tmo::build_graph(d_src, d_dst, d_t, m, n_nodes, (cudaStream_t)stream, out);
}

int tm_graph_load(const int32_t* src, const int32_t* dst, const int64_t* t, int64_t m,
                  int32_t n_nodes, tm_graph** out) {
    if (!out) { tmo::set_error("out is NULL"); return TM_EINVAL; }
    *out = nullptr;
    if (m < 0 || m >= ((int64_t)1 << 31) - 1) { tmo::set_error("m outside [0, 2^31-1)"); return TM_EINVAL; }
    if (m > 0 && (!src || !dst || !t)) { tmo::set_error("NULL edge array"); return TM_EINVAL; }
    cudaStream_t st;
    TM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    size_t M = (size_t)(m > 0 ? m : 1);
    tmo::ScratchLease lease;   // the three staged arrays
    int rc = tmo::scratch_acquire(2 * tmo::align256(4 * M) + 8 * M, st, lease);
    if (rc != TM_OK) {
        cudaStreamDestroy(st);
        return rc;
    }
    int32_t* ds = (int32_t*)lease.p;
    int32_t* dd = (int32_t*)((char*)lease.p + tmo::align256(4 * M));
    int64_t* dt = (int64_t*)((char*)lease.p + 2 * tmo::align256(4 * M));
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(ds, src, 4 * (size_t)m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(dd, dst, 4 * (size_t)m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(dt, t, 8 * (size_t)m, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = tmo::cuda_status(e, "tm_graph_load copy", __FILE__, __LINE__);
    if (rc == TM_OK) rc = tmo::build_graph(ds, dd, dt, m, n_nodes, st, out);
    tmo::scratch_release(lease, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}

void tm_graph_free(tm_graph* g) {
    if (!g) return;
    tmo::pool_free(g->block, g->device);
    tmo::pool_free(g->hash_block, g->device);
    tmo::pool_free(g->ex_own_block, g->device);
    tmo::pool_free(g->ex_rev_block, g->device);
    delete g;
}

int tm_graph_get_info(const tm_graph* g, tm_graph_info* info) {
    if (!g || !info) { tmo::set_error("NULL argument"); return TM_EINVAL; }
    std::memset(info, 0, sizeof(*info));
    info->m = g->m;
    info->n_nodes = g->n;
    info->n_pairs = g->P;
    info->t_min = g->t_min;
    info->t_max = g->t_max;
    info->device_bytes = g->bytes;
    return TM_OK;
}

}  // extern "C"

namespace tmo {
TM_DEFINE_CHECK_WORD(check_word_graph)
}  // namespace tmo
