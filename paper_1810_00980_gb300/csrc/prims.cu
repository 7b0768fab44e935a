// Device primitives: exclusive scan of int64 and a stable LSD radix sort of
// (uint32 key, uint32 value) pairs.  Neither waits on other blocks: the scan
// is reduce-then-scan over tiles, the sort is histogram / scan / scatter per
// digit, so no launch can spin.
#include <mutex>
#include <vector>

#include "tm_internal.cuh"

namespace tmo {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* smem, int64_t* total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) smem[w] = inc;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int64_t s = lane < nw ? smem[lane] : 0;
        int64_t si = warp_incl_scan(s);
        if (lane < nw) smem[lane] = si - s;
        if (lane == nw - 1) smem[32] = si;
    }
    __syncthreads();
    int64_t r = inc - v + smem[w];
    *total = smem[32];
    __syncthreads();
    return r;
}

// Each block scans one tile (exclusive), writes the tile total to sums[tile].
// (in may equal out: every thread reads its items before any thread writes)
__global__ void k_scan_tiles(const int64_t* in, int64_t* out, int64_t n, int64_t* __restrict__ sums) {
    // the tile passes through shared memory (padded: no bank conflicts) so that loads and
    // stores are coalesced
    __shared__ int64_t smem[33];
    __shared__ int64_t tile[kScanTile + kScanTile / 16];
    int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = t0 + i;
        tile[i + (i >> 4)] = idx < n ? in[idx] : 0;
    }
    __syncthreads();
    int b = threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = tile[b + i + ((b + i) >> 4)];
        loc += v[i];
    }
    int64_t total;
    int64_t run = block_excl_scan(loc, smem, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        tile[b + i + ((b + i) >> 4)] = run;
        run += v[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = t0 + i;
        if (idx < n) out[idx] = tile[i + (i >> 4)];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// 32-bit lengths -> 64-bit exclusive offsets, reduce-then-scan (each length read twice, each
// offset written once): per-tile sums first (tiles at or past the count, read on the device
// when d_n is given, sum to 0) ...
__global__ void k_len_reduce(const int32_t* __restrict__ in, int64_t n_max, const int64_t* __restrict__ d_n,
                             int64_t* __restrict__ sums) {
    __shared__ int64_t smem[33];
    int64_t n = d_n ? min(*d_n, n_max) : n_max;
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t loc = 0;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) loc += in[idx];
    }
    int64_t total;
    block_excl_scan(loc, smem, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// ... then each tile's exclusive scan plus the tile's offset; the tile passes through shared
// memory so that both the 32-bit loads and the 64-bit stores are coalesced
__global__ void k_len_scan(const int32_t* __restrict__ in, int64_t* __restrict__ out, int64_t n_max,
                           const int64_t* __restrict__ d_n, const int64_t* __restrict__ offs) {
    __shared__ int64_t smem[33];
    __shared__ int64_t tile[kScanTile + kScanTile / 16];   // one pad word per 16: no bank conflicts
    int64_t n = d_n ? min(*d_n, n_max) : n_max;
    int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    if (t0 >= n) return;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = t0 + i;
        tile[i + (i >> 4)] = idx < n ? (int64_t)in[idx] : 0;
    }
    __syncthreads();
    int b = threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = tile[b + i + ((b + i) >> 4)];
        loc += v[i];
    }
    int64_t total;
    int64_t run = block_excl_scan(loc, smem, &total) + offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        tile[b + i + ((b + i) >> 4)] = run;
        run += v[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = t0 + i;
        if (idx < n) out[idx] = tile[i + (i >> 4)];
    }
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t add = offs[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

__global__ void k_scan_small(const int64_t* in, int64_t* out, int64_t n, int64_t* __restrict__ d_total) {
    // single block, n <= kScanTile
    __shared__ int64_t smem[33];
    int64_t base = (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        loc += v[i];
    }
    int64_t total;
    int64_t run = block_excl_scan(loc, smem, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == 0 && d_total) *d_total = total;
}

__global__ void k_set_i64(int64_t* p, int64_t v) { *p = v; }

// the same scans for an element count held in device memory (*d_n <= n_max);
// tiles past *d_n contribute nothing and write nothing
__global__ void k_scan_tiles_dn(const int64_t* in, int64_t* out, const int64_t* __restrict__ d_n,
                                int64_t* __restrict__ sums) {
    __shared__ int64_t smem[33];
    int64_t n = *d_n;
    if ((int64_t)blockIdx.x * kScanTile >= n) {
        if (threadIdx.x == 0) sums[blockIdx.x] = 0;
        return;
    }
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        loc += v[i];
    }
    int64_t total;
    int64_t run = block_excl_scan(loc, smem, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add_dn(int64_t* __restrict__ out, const int64_t* __restrict__ d_n,
                              const int64_t* __restrict__ offs) {
    int64_t n = *d_n;
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) return;
    int64_t add = offs[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

__global__ void k_scan_small_dn(const int64_t* in, int64_t* out, const int64_t* __restrict__ d_n,
                                int64_t* __restrict__ d_total) {
    __shared__ int64_t smem[33];
    int64_t n = *d_n;
    int64_t base = (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        loc += v[i];
    }
    int64_t total;
    int64_t run = block_excl_scan(loc, smem, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == 0 && d_total) *d_total = total;
}

// ------------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                       // per lane
constexpr int kSortTile = kSortThreads * kSortItems; // 4096
constexpr int kMaxDigitBits = 10;

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int db,
                             int32_t* __restrict__ hist, int64_t ntiles) {
    __shared__ int32_t h[1 << kMaxDigitBits];
    int nd = 1 << db;
    for (int i = threadIdx.x; i < nd; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    uint32_t mask = (uint32_t)nd - 1;
    for (int i = threadIdx.x; i < kSortTile; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & mask], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += blockDim.x) hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

// Stable scatter of one tile: warp w owns items [w*512, w*512+512) of the
// tile, taken 32 at a time in index order; ranks among equal digits come from
// __match_any_sync and per-warp running counters, then warps are offset by
// the counts of lower warps.  The tile is first reordered by digit in shared
// memory, so that neighbouring threads write neighbouring addresses of one
// digit's output run (coalesced) instead of scattering single words.
// Dynamic shared memory: kSortTile keys and values, per-warp digit counters,
// and per-digit tile starts and output bases (sort_smem_bytes(db)).
template <typename V>
__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint32_t* __restrict__ kin, const V* __restrict__ vin,
                uint32_t* __restrict__ kout, V* __restrict__ vout, int64_t n, int shift,
                int db, const int64_t* __restrict__ offs, int64_t ntiles) {
    extern __shared__ __align__(16) unsigned char sm_sort[];
    int nd = 1 << db;
    uint32_t* skey = (uint32_t*)sm_sort;                        // [kSortTile]
    V* sval = (V*)(skey + kSortTile);                           // [kSortTile]
    int64_t* gbase = (int64_t*)(sval + kSortTile);              // [nd] output index of tile slot 0 of digit d
    int32_t* cnt = (int32_t*)(gbase + nd);                      // [kSortWarps][nd]
    int32_t* tds = cnt + kSortWarps * nd;                       // [nd] tile start of digit d
    uint32_t mask = (uint32_t)nd - 1;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = lane; i < nd; i += 32) cnt[w * nd + i] = 0;
    __syncwarp();
    int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    int64_t base = tbase + (int64_t)w * (kSortItems * 32);
    uint32_t key[kSortItems];
    int32_t rank[kSortItems];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        int64_t idx = base + r * 32 + lane;
        bool ok = idx < n;
        key[r] = ok ? kin[idx] : 0u;
        uint32_t d = ok ? ((key[r] >> shift) & mask) : 0xffffffffu;
        unsigned peers = __match_any_sync(kFull, d);
        int before = __popc(peers & lt);
        int32_t c0 = ok ? cnt[w * nd + d] : 0;
        rank[r] = c0 + before;
        __syncwarp();
        int leader = 31 - __clz(peers);
        if (ok && lane == leader) cnt[w * nd + d] = c0 + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets inside the digit, the digit's total in tds (scanned below)
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        int32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ww++) {
            int32_t c = cnt[ww * nd + d];
            cnt[ww * nd + d] = run;
            run += c;
        }
        tds[d] = run;
    }
    __syncthreads();
    if (w == 0) {   // exclusive scan of the digit totals (nd <= 1024: 32 per lane at most)
        int per = (nd + 31) / 32;
        int32_t sum = 0;
        for (int i = 0; i < per; i++) {
            int d = lane * per + i;
            if (d < nd) sum += tds[d];
        }
        int32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        int32_t run = inc - sum;
        for (int i = 0; i < per; i++) {
            int d = lane * per + i;
            if (d < nd) {
                int32_t c = tds[d];
                tds[d] = run;
                run += c;
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x)
        gbase[d] = offs[(int64_t)d * ntiles + blockIdx.x] - tds[d];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            uint32_t d = (key[r] >> shift) & mask;
            int32_t lp = tds[d] + cnt[w * nd + d] + rank[r];
            skey[lp] = key[r];
            sval[lp] = vin[idx];   // values are read here, not held through the ranking
        }
    }
    __syncthreads();
    int64_t tn = min((int64_t)kSortTile, n - tbase);
    for (int i = threadIdx.x; i < tn; i += blockDim.x) {
        uint32_t k = skey[i];
        int64_t pos = TM_CHK_IDX(gbase[(k >> shift) & mask] + i, n, kChkSort);
        kout[pos] = k;
        vout[pos] = sval[i];
    }
}

template <typename V>
size_t sort_smem_bytes(int db) {
    size_t nd = (size_t)1 << db;
    return (4 + sizeof(V)) * (size_t)kSortTile + 8 * nd + 4 * nd * (kSortWarps + 1);
}

// LSD radix sort of (u32 key, V value) by the low `bits` bits of the key, stable; the
// sorted arrays end in whichever of (keys, vals) / (keys_tmp, vals_tmp) the last pass
// wrote, returned through kres / vres
template <typename V>
int radix_sort_t(uint32_t* keys, V* vals, uint32_t* keys_tmp, V* vals_tmp, int64_t n, int bits,
                 cudaStream_t st, uint32_t** kres, V** vres) {
    *kres = keys;
    *vres = vals;
    if (n <= 1 || bits <= 0) return TM_OK;
    int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    int db = (bits + passes - 1) / passes;
    {
        // the scatter's dynamic shared memory can exceed the 48 KB default: allow the
        // largest digit width once per device and value type
        static std::mutex mu;
        static bool done[64] = {};
        int dev = 0;
        TM_CUDA(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !done[dev]) {
            TM_CUDA(cudaFuncSetAttribute(k_radix_scatter<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sort_smem_bytes<V>(kMaxDigitBits)));
            done[dev] = true;
        }
    }
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    int64_t nh = ((int64_t)1 << db) * ntiles;
    int32_t* hist = nullptr;
    int64_t* offs = nullptr;
    TM_CUDA(cudaMallocAsync((void**)&hist, sizeof(int32_t) * (size_t)nh, st));
    TM_CUDA(cudaMallocAsync((void**)&offs, sizeof(int64_t) * (size_t)nh * 2, st));
    int64_t* hist64 = offs + nh;
    uint32_t *ka = keys, *kb = keys_tmp;
    V *va = vals, *vb = vals_tmp;
    int rc = TM_OK;
    for (int p = 0; p < passes && rc == TM_OK; p++) {
        int shift = p * db;
        int width = (shift + db > bits) ? bits - shift : db;
        k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(ka, n, shift, width, hist, ntiles); count_launch();
        int64_t nhp = ((int64_t)1 << width) * ntiles;
        rc = scan_lengths(hist, offs, nhp, nullptr, nullptr, nh >= 8 ? hist64 : nullptr, nh, st);
        if (rc != TM_OK) break;
        k_radix_scatter<V><<<(unsigned)ntiles, kSortThreads, sort_smem_bytes<V>(width), st>>>(
            ka, va, kb, vb, n, shift, width, offs, ntiles);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) { rc = TM_ECUDA; break; }
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    cudaFreeAsync(hist, st);
    cudaFreeAsync(offs, st);
    if (rc != TM_OK) set_error("radix sort launch failed");
    *kres = ka;
    *vres = va;
    return rc;
}

}  // namespace

int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total,
                       cudaStream_t st) {
    if (n <= 0) {
        if (d_total) {
            k_set_i64<<<1, 1, 0, st>>>(d_total, 0); count_launch();
            TM_CUDA(cudaGetLastError());
        }
        return TM_OK;
    }
    if (n <= kScanTile) {
        k_scan_small<<<1, kScanThreads, 0, st>>>(in, out, n, d_total); count_launch();
        TM_CUDA(cudaGetLastError());
        return TM_OK;
    }
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t* sums = nullptr;
    TM_CUDA(cudaMallocAsync((void**)&sums, sizeof(int64_t) * (size_t)ntiles * 2, st));
    int64_t* soffs = sums + ntiles;
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, sums); count_launch();
    int s1 = cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
    if (s1 == TM_OK) s1 = scan_exclusive_i64(sums, soffs, ntiles, d_total, st);
    if (s1 == TM_OK) {
        k_scan_add<<<(unsigned)ntiles, kScanThreads, 0, st>>>(out, n, soffs); count_launch();
        if (cudaGetLastError() != cudaSuccess) s1 = TM_ECUDA;
    }
    cudaFreeAsync(sums, st);
    if (s1 != TM_OK) set_error("scan launch failed");
    return s1;
}

int scan_exclusive_i64_ws(const int64_t* in, int64_t* out, int64_t n, int64_t* d_total,
                          int64_t* ws, int64_t ws_elems, cudaStream_t st) {
    // Same result as scan_exclusive_i64, with the per-tile sums in the
    // caller's workspace `ws` instead of a stream-ordered allocation.
    if (n <= 0) {
        if (d_total) {
            k_set_i64<<<1, 1, 0, st>>>(d_total, 0); count_launch();
            TM_CUDA(cudaGetLastError());
        }
        return TM_OK;
    }
    if (n <= kScanTile) {
        k_scan_small<<<1, kScanThreads, 0, st>>>(in, out, n, d_total); count_launch();
        TM_CUDA(cudaGetLastError());
        return TM_OK;
    }
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanTile || 2 * ntiles > ws_elems) return TM_EINVAL;
    int64_t* sums = ws;
    int64_t* soffs = ws + ntiles;
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, sums); count_launch();
    k_scan_small<<<1, kScanThreads, 0, st>>>(sums, soffs, ntiles, d_total); count_launch();
    k_scan_add<<<(unsigned)ntiles, kScanThreads, 0, st>>>(out, n, soffs); count_launch();
    TM_CUDA(cudaGetLastError());
    return TM_OK;
}

int scan_lengths(const int32_t* in, int64_t* out, int64_t n_max, const int64_t* d_n, int64_t* d_total,
                 int64_t* ws, int64_t ws_elems, cudaStream_t st) {
    if (n_max <= 0) {
        if (d_total) {
            k_set_i64<<<1, 1, 0, st>>>(d_total, 0); count_launch();
            TM_CUDA(cudaGetLastError());
        }
        return TM_OK;
    }
    int64_t ntiles = (n_max + kScanTile - 1) / kScanTile;
    int64_t need = 2 * ntiles + 2 * ((ntiles + kScanTile - 1) / kScanTile) + 2;
    int64_t* own = nullptr;
    if (!ws) {
        TM_CUDA(cudaMallocAsync((void**)&own, sizeof(int64_t) * (size_t)need, st));
        ws = own;
        ws_elems = need;
    }
    int rc = TM_OK;
    if (ws_elems < need || ntiles > (int64_t)kScanTile * kScanTile) rc = TM_EINVAL;   // caller's workspace too small
    if (rc == TM_OK) {
        int64_t* sums = ws;
        int64_t* soffs = ws + ntiles;
        k_len_reduce<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n_max, d_n, sums); count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        if (rc == TM_OK) rc = scan_exclusive_i64_ws(sums, soffs, ntiles, d_total, ws + 2 * ntiles, need - 2 * ntiles, st);
        if (rc == TM_OK) {
            k_len_scan<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n_max, d_n, soffs); count_launch();
            if (cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
        }
    }
    if (own) cudaFreeAsync(own, st);
    if (rc != TM_OK) set_error("length scan failed");
    return rc;
}

int64_t scan_dn_ws_elems(int64_t n_max) {
    if (n_max <= kScanTile) return 0;
    int64_t ntiles = (n_max + kScanTile - 1) / kScanTile;
    return 2 * ntiles + 2 * ((ntiles + kScanTile - 1) / kScanTile) + 2;
}

int scan_exclusive_i64_dn(const int64_t* in, int64_t* out, int64_t n_max, const int64_t* d_n,
                          int64_t* d_total, int64_t* ws, int64_t ws_elems, cudaStream_t st) {
    if (n_max <= 0) {
        if (d_total) {
            k_set_i64<<<1, 1, 0, st>>>(d_total, 0); count_launch();
            TM_CUDA(cudaGetLastError());
        }
        return TM_OK;
    }
    if (n_max <= kScanTile) {
        k_scan_small_dn<<<1, kScanThreads, 0, st>>>(in, out, d_n, d_total); count_launch();
        TM_CUDA(cudaGetLastError());
        return TM_OK;
    }
    int64_t ntiles = (n_max + kScanTile - 1) / kScanTile;
    if (ws_elems < scan_dn_ws_elems(n_max)) return TM_EINVAL;
    int64_t* sums = ws;
    int64_t* soffs = ws + ntiles;
    int64_t* inner = ws + 2 * ntiles;
    k_scan_tiles_dn<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, d_n, sums); count_launch();
    TM_CUDA(cudaGetLastError());
    int rc = scan_exclusive_i64_ws(sums, soffs, ntiles, d_total, inner, ws_elems - 2 * ntiles, st);
    if (rc != TM_OK) return rc;
    k_scan_add_dn<<<(unsigned)ntiles, kScanThreads, 0, st>>>(out, d_n, soffs); count_launch();
    TM_CUDA(cudaGetLastError());
    return TM_OK;
}

int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                     int64_t n, int bits, cudaStream_t st) {
    // Sorts (keys, vals) stably by the low `bits` bits of keys; the result ends
    // in keys/vals.  bits <= 32.
    uint32_t *kr, *vr;
    int rc = radix_sort_t<uint32_t>(keys, vals, keys_tmp, vals_tmp, n, bits, st, &kr, &vr);
    if (rc == TM_OK && kr != keys) {
        TM_CUDA(cudaMemcpyAsync(keys, kr, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        TM_CUDA(cudaMemcpyAsync(vals, vr, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    }
    return rc;
}

int radix_sort_kv64(uint32_t* keys, uint64_t* vals, uint32_t* keys_tmp, uint64_t* vals_tmp, int64_t n,
                    int bits, cudaStream_t st, uint32_t** kres, uint64_t** vres) {
    return radix_sort_t<uint64_t>(keys, vals, keys_tmp, vals_tmp, n, bits, st, kres, vres);
}

namespace {
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};
cudaStream_t g_free_stream[64] = {};
}  // namespace

int pool_prepare(int dev) {
    if (dev < 0 || dev >= 64) return TM_OK;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_ready[dev]) return TM_OK;
    // keep freed blocks of the device's default pool mapped, so that graphs and
    // batch scratch that come and go reuse memory instead of remapping it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaStreamCreateWithFlags(&g_free_stream[dev], cudaStreamNonBlocking);
    cudaGetLastError();
    g_pool_ready[dev] = true;
    return TM_OK;
}

void pool_free(void* p, int dev) {
    if (!p) return;
    cudaStream_t s = (dev >= 0 && dev < 64) ? g_free_stream[dev] : nullptr;
    if (s) cudaFreeAsync(p, s);
    else cudaFree(p);
}

// Scratch arenas.  A large request to the stream-ordered pool costs about 0.3 ms of host
// time even when the pool keeps its memory (the device idles meanwhile), so the scratch
// of graph builds and batches comes from a few grow-only buffers per device instead.  A
// buffer is leased to one call at a time; the stream of the next lease waits on the event
// that the last holder recorded on its own stream at release.  A request that finds no
// free buffer is served by the pool.
namespace {
constexpr int kArenas = 4;
struct Arena {
    void* p = nullptr;
    size_t cap = 0;
    bool held = false;
    cudaEvent_t ev = nullptr;
    bool ev_set = false;
};
Arena g_arena[64][kArenas];
}  // namespace

int scratch_acquire(size_t bytes, cudaStream_t st, ScratchLease& L) {
    L = ScratchLease();
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    L.dev = dev;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        int fit = -1, grow = -1;
        for (int i = 0; i < kArenas; i++) {
            const Arena& A = g_arena[dev][i];
            if (A.held) continue;
            if (A.cap >= bytes && (fit < 0 || A.cap < g_arena[dev][fit].cap)) fit = i;
            if (grow < 0 || A.cap > g_arena[dev][grow].cap) grow = i;
        }
        int i = fit >= 0 ? fit : grow;
        if (i >= 0) {
            Arena& A = g_arena[dev][i];
            cudaError_t e = cudaSuccess;
            if (!A.ev) e = cudaEventCreateWithFlags(&A.ev, cudaEventDisableTiming);
            if (e == cudaSuccess && A.ev_set) e = cudaStreamWaitEvent(st, A.ev, 0);
            if (e == cudaSuccess && A.cap < bytes) {
                if (A.p) cudaFreeAsync(A.p, st);
                A.p = nullptr;
                A.cap = 0;
                e = cudaMallocAsync(&A.p, bytes, st);
                if (e == cudaSuccess) A.cap = bytes;
                else A.p = nullptr;
            }
            if (e == cudaSuccess) {
                A.held = true;
                L.p = A.p;
                L.slot = i;
                return TM_OK;
            }
            cudaGetLastError();   // fall through to a pool block
        }
    }
    TM_CUDA(cudaMallocAsync(&L.p, bytes, st));
    return TM_OK;
}

void scratch_release(ScratchLease& L, cudaStream_t st) {
    if (!L.p) return;
    if (L.slot < 0) {
        cudaFreeAsync(L.p, st);
    } else {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        Arena& A = g_arena[L.dev][L.slot];
        A.ev_set = cudaEventRecord(A.ev, st) == cudaSuccess;
        if (!A.ev_set) cudaGetLastError();
        A.held = false;
    }
    L = ScratchLease();
}

int pool_trim() {
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    TM_CUDA(cudaDeviceSynchronize());
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        for (int i = 0; i < kArenas; i++) {
            Arena& A = g_arena[dev][i];
            if (A.held || !A.p) continue;
            TM_CUDA(cudaFree(A.p));
            A.p = nullptr;
            A.cap = 0;
            A.ev_set = false;
        }
    }
    cudaMemPool_t pool;
    TM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    TM_CUDA(cudaMemPoolTrimTo(pool, 0));
    return TM_OK;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace tmo

namespace tmo {
TM_DEFINE_CHECK_WORD(check_word_prims)
}  // namespace tmo
