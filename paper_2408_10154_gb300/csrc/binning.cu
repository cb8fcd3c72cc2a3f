// binning.cu -- tile binning: exclusive scan of tiles-touched counts,
// duplicate emission with 64-bit (tile << 32 | depth bits) keys, stable LSD
// radix sort over the needed key bits, per-tile [start, end) ranges.
//
// All sizes that depend on the data (the number of duplicates) live on the
// device, so the whole sequence can be captured in a CUDA graph: grids are
// sized for the capacity and blocks past the live count exit early.
// HBM-bound throughout: the sort moves 8 B key + 4 B value in and out per
// duplicate per 8-bit pass.
#include "gs_internal.cuh"

namespace {

using namespace gsk;

// ---------------------------------------------------------------- scan
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(const uint32_t *in, size_t n, uint32_t *partials)
{
    __shared__ uint32_t s[kScanThreads / 32];
    const size_t base = (size_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanTile / kScanThreads; ++k) {
        const size_t i = base + (size_t)k * kScanThreads + threadIdx.x;
        if (i < n)
            acc += in[i];
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0)
        s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < kScanThreads / 32 ? s[threadIdx.x] : 0u;
        v = warp_sum(v);
        if (threadIdx.x == 0)
            partials[blockIdx.x] = v;
    }
}

// single block: exclusive scan of the partials in place; total (uint64
// saturated to 0xffffffff) to *total
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *partials, size_t np, uint32_t *total)
{
    __shared__ uint32_t s_warp[33];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    for (size_t c = 0; c < np; c += 1024) {
        const size_t i = c + threadIdx.x;
        const uint32_t x = i < np ? partials[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan<1024>(x, s_warp, tot);
        const unsigned long long carry = s_carry;
        if (i < np) {
            const unsigned long long v = carry + ex;
            partials[i] = v > 0xffffffffull ? 0xffffffffu : (uint32_t)v;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total)
        *total = s_carry > 0xffffffffull ? 0xffffffffu : (uint32_t)s_carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *in, size_t n, const uint32_t *partials,
                                                            uint32_t *out)
{
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    constexpr int K = kScanTile / kScanThreads;
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * K;  // blocked arrangement
    uint32_t v[K];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        sum += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<kScanThreads>(sum, s_warp, tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (base + k < n)
            out[base + k] = ex;
        ex += v[k];
    }
}

// ---------------------------------------------------------------- emission
// Block b owns records [b*kScanTile, (b+1)*kScanTile): it re-scans their
// counts locally, then emits its duplicates dup-parallel (thread j handles
// the block's j-th duplicate), so that a Gaussian touching many tiles does
// not stall a warp.
__global__ void __launch_bounds__(kScanThreads) k_emit(const gsl::BinArgs a, const uint32_t *blk_base)
{
    __shared__ uint32_t s_off[kScanTile + 1];
    __shared__ uint32_t s_t0[kScanTile];   // global tile of the rect corner
    __shared__ uint32_t s_geo[kScanTile];  // rect width | TX << 16
    __shared__ uint32_t s_z[kScanTile];
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    __shared__ int s_vp[2];
    constexpr int K = kScanTile / kScanThreads;
    const uint32_t rbase = blockIdx.x * kScanTile;
    if (threadIdx.x == 0) {
        // vp of the first record of this block (records of a vp are contiguous)
        int lo = 0, hi = a.n_vps - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.vps[mid].rec_base <= rbase) lo = mid; else hi = mid - 1;
        }
        s_vp[0] = lo;
    }
    __syncthreads();
    uint32_t c[K];
    uint32_t sum = 0;
    const int first = threadIdx.x * K;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t r = rbase + first + k;
        c[k] = r < a.n_records ? (uint32_t)a.counts[r] : 0u;
        sum += c[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan<kScanThreads>(sum, s_warp, tot);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int lr = first + k;
        const uint32_t r = rbase + lr;
        s_off[lr] = ex;
        ex += c[k];
        if (c[k]) {
            int vp = s_vp[0];
            while (vp + 1 < a.n_vps && a.vps[vp + 1].rec_base <= r)
                ++vp;
            const VpDesc &d = a.vps[vp];
            const float4 q1 = a.rec[3 * (size_t)r + 1];
            const float4 q2 = a.rec[3 * (size_t)r + 2];
            const uint32_t rx = __float_as_uint(q1.w), ry = __float_as_uint(q2.w);
            const uint32_t x0 = rx & 0xffffu, x1 = rx >> 16, y0 = ry & 0xffffu;
            s_t0[lr] = d.tile_base + y0 * (uint32_t)d.TX + x0;
            s_geo[lr] = (x1 - x0) | ((uint32_t)d.TX << 16);
            s_z[lr] = __float_as_uint(q1.z);
        }
    }
    if (threadIdx.x == 0)
        s_off[kScanTile] = tot;
    __syncthreads();
    const uint32_t gbase = blk_base[blockIdx.x];
    for (uint32_t j = threadIdx.x; j < tot; j += blockDim.x) {
        // last record with s_off <= j (upper bound - 1)
        int lo = 0, hi = kScanTile - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const uint32_t local = j - s_off[lo];
        const uint32_t geo = s_geo[lo];
        const uint32_t w = geo & 0xffffu, TX = geo >> 16;
        const uint32_t tile = s_t0[lo] + (local / w) * TX + local % w;
        const uint64_t pos = (uint64_t)gbase + j;
        if (pos < a.capacity) {
            a.keys[0][pos] = ((uint64_t)tile << 32) | s_z[lo];
            a.vals[0][pos] = rbase + (uint32_t)lo;
        }
    }
    if (threadIdx.x == 0 && (uint64_t)gbase + tot > a.capacity && tot > 0)
        atomicOr(a.flags, kFlagCapacity);
}

// ---------------------------------------------------------------- radix sort
__device__ __forceinline__ uint32_t div_up_d(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint32_t live_count(const uint32_t *n_dups, uint32_t cap)
{
    const uint32_t n = *n_dups;
    return n < cap ? n : cap;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const K *keys, const uint32_t *n_dups, uint32_t cap,
                                                          int shift, uint32_t *hist, uint32_t nblk)
{
    __shared__ uint32_t h[kSortThreads / 32][256];
    const int warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kSortThreads / 32) * 256; k += blockDim.x)
        (&h[0][0])[k] = 0;
    __syncthreads();
    const uint32_t n = live_count(n_dups, cap);
    const uint32_t base = blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortKPT; ++k) {
        const uint32_t i = base + k * kSortThreads + threadIdx.x;
        const uint32_t d = i < n ? (uint32_t)(keys[i] >> shift) & 0xffu : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < 256u && (uint32_t)(__ffs(peers) - 1) == (threadIdx.x & 31u))
            atomicAdd(&h[warp][d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w)
        s += h[w][threadIdx.x];
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = s;
}

// Stable scatter: warp w ranks the block's keys [w*256, w*256+256) in 8
// rounds of 32 consecutive keys (match_any finds equal digits), so ranks
// follow input order within the block; digit-major scanned histograms give
// the block's base per digit.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const K *kin, const uint32_t *vin,
                                                             const uint32_t *n_dups, uint32_t cap, int shift,
                                                             const uint32_t *hist_scanned, uint32_t nblk,
                                                             K *kout, uint32_t *vout)
{
    __shared__ uint32_t cnt[kSortThreads / 32][256];
    __shared__ uint32_t s_base[256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < (kSortThreads / 32) * 256; k += blockDim.x)
        (&cnt[0][0])[k] = 0;
    s_base[threadIdx.x] = hist_scanned[(size_t)threadIdx.x * nblk + blockIdx.x];
    __syncthreads();
    const uint32_t n = live_count(n_dups, cap);
    const uint32_t base = blockIdx.x * kSortTile + warp * (32 * kSortKPT);
    const unsigned lt = lanemask_lt();
    K key[kSortKPT];
    uint32_t val[kSortKPT], off[kSortKPT], dig[kSortKPT];
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : K(0);
        val[r] = valid ? vin[i] : 0u;
        const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & 0xffu : 256u;
        dig[r] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        uint32_t o = 0;
        if (valid)
            o = cnt[warp][d] + rank;
        off[r] = o;
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane)
            cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for each digit (thread = digit)
    {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t c = cnt[w][threadIdx.x];
            cnt[w][threadIdx.x] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        if (dig[r] < 256u) {
            const uint32_t pos = s_base[dig[r]] + cnt[warp][dig[r]] + off[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---------------------------------------------------------------- ranges
// tile of a key: the high word of a 64-bit (tile << 32 | depth) key, or a
// 32-bit tile key itself
__device__ __forceinline__ uint32_t tile_of(uint64_t k) { return (uint32_t)(k >> 32); }
__device__ __forceinline__ uint32_t tile_of(uint32_t k) { return k; }

template <typename K>
__global__ void k_ranges(const K *keys, const uint32_t *n_dups, uint32_t cap, uint2 *ranges)
{
    const uint32_t n = live_count(n_dups, cap);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint32_t t = tile_of(keys[i]);
    if (i == 0 || tile_of(keys[i - 1]) != t)
        ranges[t].x = i;
    if (i == n - 1 || tile_of(keys[i + 1]) != t)
        ranges[t].y = i + 1;
}

// ---------------------------------------------------------------- two-stage binning
// Stage 1 sorts the visible records by depth (stable, ties by record
// index); stage 2 emits their duplicates in that order with 32-bit tile
// keys and sorts them stably by tile.  The per-tile order is (depth bits,
// record index), the same as a stable sort of (tile << 32 | depth) keys
// emitted in record order, with 4-byte keys and 2 tile passes instead of 6
// passes over 8-byte keys.

// visible records per block of kScanTile records
__global__ void __launch_bounds__(kScanThreads) k_vis_partials(const int32_t *counts, uint32_t n, uint32_t *partials)
{
    __shared__ uint32_t s[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanTile / kScanThreads; ++k) {
        const uint32_t i = base + k * kScanThreads + threadIdx.x;
        acc += (i < n && counts[i] > 0) ? 1u : 0u;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0)
        s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < kScanThreads / 32 ? s[threadIdx.x] : 0u;
        v = warp_sum(v);
        if (threadIdx.x == 0)
            partials[blockIdx.x] = v;
    }
}

// compacts the visible records (record order) with their depth bits
__global__ void __launch_bounds__(kScanThreads) k_vis_compact(const int32_t *counts, const float4 *rec, uint32_t n,
                                                             const uint32_t *blk_base, uint32_t *dkeys, uint32_t *dvals)
{
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    constexpr int K = kScanTile / kScanThreads;
    const uint32_t first = blockIdx.x * kScanTile + threadIdx.x * K;
    uint32_t f[K], sum = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        f[k] = (first + k < n && counts[first + k] > 0) ? 1u : 0u;
        sum += f[k];
    }
    uint32_t tot;
    uint32_t pos = block_excl_scan<kScanThreads>(sum, s_warp, tot) + blk_base[blockIdx.x];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (f[k]) {
            const uint32_t r = first + k;
            dkeys[pos] = __float_as_uint(rec[3 * (size_t)r + 1].z);
            dvals[pos] = r;
            ++pos;
        }
    }
}

// tile count of each depth-sorted visible record (0 past the live count)
__global__ void k_sorted_counts(const int32_t *counts, const uint32_t *dvals, const uint32_t *n_vis, uint32_t n,
                                uint32_t *out)
{
    const uint32_t nv = live_count(n_vis, n);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = i < nv ? (uint32_t)counts[dvals[i]] : 0u;
}

// largest i in [0, n) with a[i] <= t, for non-decreasing a with a[0] <= t:
// a 32-ary search by one warp (each round narrows the range 32-fold)
__device__ __forceinline__ uint32_t warp_last_le(const uint32_t *a, uint32_t n, uint32_t t)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = n;
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t p = lo + lane * step;
        const unsigned m = __ballot_sync(0xffffffffu, p < hi && a[p] <= t) | 1u;
        const uint32_t nlo = lo + (uint32_t)(31 - __clz(m)) * step;
        hi = min(nlo + step, hi);
        lo = nlo;
    }
    const uint32_t p = lo + lane;
    const unsigned m = __ballot_sync(0xffffffffu, p < hi && a[p] <= t) | 1u;
    return lo + (uint32_t)(31 - __clz(m));
}

// Emits the duplicates [b*kScanTile, (b+1)*kScanTile) of the depth-sorted
// visible records (offsets = exclusive scan of their tile counts) with
// 32-bit tile keys.  Work is split by duplicates, not by records, so the
// few near-camera splats covering thousands of tiles (all at the front of
// the depth order) do not serialise one block.  A block touches at most
// kScanTile records because every visible record has at least one tile.
__global__ void __launch_bounds__(kScanThreads) k_emit_balanced(const gsl::BinArgs a, const uint32_t *dvals,
                                                               const uint32_t *offs, uint32_t *tkeys, uint32_t *vals)
{
    __shared__ uint32_t s_off[kScanTile];
    __shared__ uint32_t s_t0[kScanTile];
    __shared__ uint32_t s_geo[kScanTile];
    __shared__ uint32_t s_rec[kScanTile];
    __shared__ uint32_t s_r[2];
    const uint32_t total = *a.n_dups;
    if (blockIdx.x == 0 && threadIdx.x == 0 && total > a.capacity)
        atomicOr(a.flags, kFlagCapacity);
    const uint32_t nd = total < a.capacity ? total : a.capacity;
    const uint32_t b0 = blockIdx.x * kScanTile;
    if (b0 >= nd)
        return;
    const uint32_t b1 = min(b0 + (uint32_t)kScanTile, nd);
    const uint32_t nv = live_count(a.n_vis, a.n_records);
    if (nv == 0)
        return;
    if (threadIdx.x < 64) {
        const uint32_t r = warp_last_le(offs, nv, threadIdx.x < 32 ? b0 : b1 - 1);
        if ((threadIdx.x & 31) == 0)
            s_r[threadIdx.x >> 5] = r;
    }
    __syncthreads();
    const uint32_t r0 = s_r[0];
    if (s_r[1] < r0 || s_r[1] - r0 >= (uint32_t)kScanTile)
        return;  // offsets not monotone (a saturated count): nothing sound to emit
    const uint32_t nr = s_r[1] - r0 + 1;
    for (uint32_t k = threadIdx.x; k < nr; k += blockDim.x) {
        const uint32_t r = dvals[r0 + k];
        // keyframe of record r: the last vp whose records start at or before r
        int lo = 0, hi = a.n_vps - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.vps[mid].rec_base <= r) lo = mid; else hi = mid - 1;
        }
        const gsk::VpDesc &d = a.vps[lo];
        const uint32_t rx = __float_as_uint(a.rec[3 * (size_t)r + 1].w);
        const uint32_t ry = __float_as_uint(a.rec[3 * (size_t)r + 2].w);
        const uint32_t x0 = rx & 0xffffu, x1 = rx >> 16, y0 = ry & 0xffffu;
        s_off[k] = offs[r0 + k];
        s_t0[k] = d.tile_base + y0 * (uint32_t)d.TX + x0;
        s_geo[k] = (x1 - x0) | ((uint32_t)d.TX << 16);
        s_rec[k] = r;
    }
    __syncthreads();
    for (uint32_t j = b0 + threadIdx.x; j < b1; j += blockDim.x) {
        uint32_t lo = 0, hi = nr - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const uint32_t local = j - s_off[lo];
        const uint32_t geo = s_geo[lo];
        const uint32_t w = geo & 0xffffu, TX = geo >> 16;
        tkeys[j] = s_t0[lo] + (local / w) * TX + local % w;
        vals[j] = s_rec[lo];
    }
}

// 64-bit (tile << 32 | depth bits) keys of a tile-sorted list (for gs_bin)
__global__ void k_keys64(const uint32_t *tkeys, const uint32_t *vals, const float4 *rec, const uint32_t *n_dups,
                         uint32_t cap, uint64_t *keys)
{
    const uint32_t n = live_count(n_dups, cap);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        keys[i] = ((uint64_t)tkeys[i] << 32) | __float_as_uint(rec[3 * (size_t)vals[i] + 1].z);
}

inline uint32_t div_up(size_t a, size_t b) { return (uint32_t)((a + b - 1) / b); }

// ------------------------------------------------------------ one-sweep sort
// status word of (tile, digit): 2 flag bits (1 = aggregate of this tile
// only, 2 = inclusive prefix over tiles 0..t) and a 62-bit count
constexpr unsigned long long kOsAgg = 1ull << 62, kOsPrefix = 2ull << 62, kOsCount = (1ull << 62) - 1;
constexpr int kOsMaxPasses = 4;
constexpr long kOsSpinLimit = 1l << 20;  // well under a second of L2 round trips, then give up
constexpr int kOsWindow = 16;            // predecessor status words read per look-back step

struct OsLayout {
    uint32_t *counters;             // [passes] dynamic tile ids
    uint32_t *ghist;                // [passes][256] global digit counts
    uint32_t *gbase;                // [passes][256] their exclusive scan
    unsigned long long *status;     // [passes][tiles][256]
    size_t zero_bytes;              // bytes from counters through status to clear
};

OsLayout os_layout(uint8_t *base, uint32_t tiles)
{
    OsLayout L;
    L.counters = (uint32_t *)base;                                   // 64 B
    L.ghist = (uint32_t *)(base + 64);                               // 4 KB
    L.gbase = L.ghist + kOsMaxPasses * 256;                          // 4 KB
    L.status = (unsigned long long *)(base + 64 + 2 * 4 * kOsMaxPasses * 256);
    L.zero_bytes = 64 + 2 * 4 * kOsMaxPasses * 256 + sizeof(unsigned long long) * kOsMaxPasses * 256 * (size_t)tiles;
    return L;
}

// per-digit counts of every pass, over all live keys (grid-stride, warp-
// aggregated shared atomics, one global atomic per block and digit)
// digit mask of pass p over the low `bits` key bits (the last pass may be narrower)
__host__ __device__ __forceinline__ uint32_t os_digit_mask(int bits, int p)
{
    const int left = bits - 8 * p;
    return left >= 8 ? 0xffu : (1u << left) - 1u;
}

__global__ void __launch_bounds__(kSortThreads) k_os_hist(const uint32_t *keys, const uint32_t *n_dev, uint32_t cap,
                                                          int passes, int bits, uint32_t *ghist)
{
    __shared__ uint32_t h[kOsMaxPasses][256];
    for (int k = threadIdx.x; k < kOsMaxPasses * 256; k += blockDim.x)
        (&h[0][0])[k] = 0;
    __syncthreads();
    const uint32_t n = live_count(n_dev, cap);
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? keys[i] : 0u;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? (key >> (8 * p)) & os_digit_mask(bits, p) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && (uint32_t)(__ffs(peers) - 1) == lane)
                atomicAdd(&h[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < passes * 256; k += blockDim.x) {
        const uint32_t v = (&h[0][0])[k];
        if (v)
            atomicAdd(&ghist[k], v);
    }
}

// exclusive scan of each pass's 256 digit counts (one CTA of 256 threads)
__global__ void __launch_bounds__(256) k_os_scan(const uint32_t *ghist, int passes, uint32_t *gbase)
{
    __shared__ uint32_t s_warp[256 / 32 + 1];
    for (int p = 0; p < passes; ++p) {
        uint32_t tot;
        const uint32_t ex = block_excl_scan<256>(ghist[p * 256 + threadIdx.x], s_warp, tot);
        gbase[p * 256 + threadIdx.x] = ex;
    }
}

__device__ __forceinline__ unsigned long long os_load(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// One pass: rank the tile's keys stably (as k_rs_scatter), publish the
// tile's digit counts, look back for the prefix of the earlier tiles, and
// scatter to the digit's global base + that prefix + the local rank.
__global__ void __launch_bounds__(kSortThreads) k_os_pass(const uint32_t *kin, const uint32_t *vin,
                                                          const uint32_t *n_dev, uint32_t cap, int shift,
                                                          uint32_t dmask, const uint32_t *gbase,
                                                          unsigned long long *status,
                                                          uint32_t *counter, uint32_t *kout, uint32_t *vout,
                                                          int *flags)
{
    __shared__ uint32_t cnt[kSortThreads / 32][256];
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0)
        s_tile = atomicAdd(counter, 1u);
    for (int k = threadIdx.x; k < (kSortThreads / 32) * 256; k += blockDim.x)
        (&cnt[0][0])[k] = 0;
    __syncthreads();
    const uint32_t n = live_count(n_dev, cap);
    const uint32_t tile = s_tile;
    if (tile >= div_up_d(n, kSortTile))
        return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = tile * kSortTile + warp * (32 * kSortKPT);
    const unsigned lt = lanemask_lt();
    uint32_t key[kSortKPT], val[kSortKPT], off[kSortKPT], dig[kSortKPT];
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        const uint32_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0u;
        val[r] = valid ? vin[i] : 0u;
        const uint32_t d = valid ? (key[r] >> shift) & dmask : 256u;
        dig[r] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        uint32_t o = 0;
        if (valid)
            o = cnt[warp][d] + rank;
        off[r] = o;
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane)
            cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread = digit: prefix over warps, the tile's total, then the look-back
    {
        const uint32_t d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = tot;
            tot += c;
        }
        unsigned long long *mine = status + (size_t)tile * 256 + d;
        unsigned long long excl = 0;
        if (tile == 0) {
            atomicExch(mine, kOsPrefix | (unsigned long long)tot);
        } else {
            atomicExch(mine, kOsAgg | (unsigned long long)tot);
            // walk back kOsWindow tiles per step (independent loads in
            // flight): add aggregates up to the first inclusive prefix; stop
            // at a tile that has not published yet and re-read from there
            long spins = 0;
            long j = (long)tile - 1;
            bool found = false;
            while (!found && j >= 0) {
                unsigned long long v[kOsWindow];
#pragma unroll
                for (int w = 0; w < kOsWindow; ++w)
                    v[w] = (j - w >= 0) ? os_load(status + (size_t)(j - w) * 256 + d) : kOsPrefix;
                int w = 0;
                for (; w < kOsWindow; ++w) {
                    const unsigned long long f = v[w] & ~kOsCount;
                    if (f == 0)
                        break;  // not published yet
                    excl += v[w] & kOsCount;
                    if (f == kOsPrefix) {
                        found = true;
                        break;
                    }
                }
                if (found)
                    break;
                j -= w;
                if (w == 0 && ++spins > kOsSpinLimit) {  // an earlier tile never published: give up
                    atomicOr(flags, kFlagTimeout);
                    break;
                }
            }
            atomicExch(mine, kOsPrefix | (excl + tot));
        }
        s_base[d] = gbase[d] + (uint32_t)excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortKPT; ++r) {
        if (dig[r] < 256u) {
            const uint32_t pos = s_base[dig[r]] + cnt[warp][dig[r]] + off[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ------------------------------------------------------------ tile schedule
// bucket of a list length: 0 holds the longest (top bit 31), 32 the empty
__device__ __forceinline__ uint32_t len_bucket(const uint2 r) { return (uint32_t)__clz((int)(r.y - r.x)); }

__global__ void k_order_hist(const uint2 *ranges, uint32_t n, uint32_t *counts)
{
    __shared__ uint32_t h[33];
    if (threadIdx.x < 33)
        h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n)
        atomicAdd(&h[len_bucket(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x])
        atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

// exclusive scan of the 33 bucket counts into the cursors (one warp)
__global__ void k_order_scan(const uint32_t *counts, uint32_t *cursors)
{
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int b = 0; b < 33; ++b) {
            cursors[b] = s;
            s += counts[b];
        }
    }
}

__global__ void k_order_scatter(const uint2 *ranges, uint32_t n, uint32_t *cursors, uint32_t *order)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n)
        order[atomicAdd(&cursors[len_bucket(ranges[t])], 1u)] = t;
}

// stable LSD radix sort of (key, value) over `bits` low key bits, 8 per pass;
// returns the buffer index holding the result
template <typename K>
int radix_sort(K *keys[2], uint32_t *vals[2], const uint32_t *n_dev, uint32_t cap, int bits, uint32_t *hist,
               uint32_t *hist_partials, cudaStream_t s)
{
    const uint32_t sb = div_up(cap ? cap : 1, kSortTile);
    const size_t hn = (size_t)256 * sb;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<K><<<sb, kSortThreads, 0, s>>>(keys[cur], n_dev, cap, shift, hist, sb);
        gsl::scan_excl(hist, hist, hn, hist_partials, nullptr, s);
        k_rs_scatter<K><<<sb, kSortThreads, 0, s>>>(keys[cur], vals[cur], n_dev, cap, shift, hist, sb, keys[cur ^ 1],
                                                    vals[cur ^ 1]);
        gsl::g_launches += 2;
        cur ^= 1;
    }
    return cur;
}

}  // namespace

namespace gsl {

size_t scan_partials(size_t n) { return div_up(n, kScanTile) + 1; }

size_t sort_hist_entries(uint32_t capacity) { return (size_t)256 * div_up(capacity ? capacity : 1, kSortTile); }

void scan_excl(const uint32_t *in, uint32_t *out, size_t n, uint32_t *partials, uint32_t *total, cudaStream_t s)
{
    const uint32_t nb = div_up(n ? n : 1, kScanTile);
    k_scan_partials<<<nb, kScanThreads, 0, s>>>(in, n, partials);
    k_scan_top<<<1, 1024, 0, s>>>(partials, nb, total);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, n, partials, out);
    g_launches += 3;
}

void bin_count(const BinArgs &a, cudaStream_t s)
{
    const uint32_t nb = div_up(a.n_records ? a.n_records : 1, kScanTile);
    k_scan_partials<<<nb, kScanThreads, 0, s>>>((const uint32_t *)a.counts, a.n_records, a.partials);
    k_scan_top<<<1, 1024, 0, s>>>(a.partials, nb, a.n_dups);
    g_launches += 2;
}

void tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, uint32_t *counters, cudaStream_t s)
{
    if (n_tiles == 0)
        return;
    cudaMemsetAsync(counters, 0, 64 * sizeof(uint32_t), s);
    k_order_hist<<<div_up(n_tiles, 256), 256, 0, s>>>(ranges, n_tiles, counters);
    k_order_scan<<<1, 32, 0, s>>>(counters, counters + 64);
    k_order_scatter<<<div_up(n_tiles, 256), 256, 0, s>>>(ranges, n_tiles, counters + 64, order);
    g_launches += 3;
}

size_t onesweep_scratch_bytes(uint32_t cap, int bits)
{
    (void)bits;
    return os_layout(nullptr, div_up(cap ? cap : 1, kSortTile)).zero_bytes;
}

int onesweep_u32(uint32_t *keys[2], uint32_t *vals[2], const uint32_t *n_dev, uint32_t cap, int bits,
                 uint8_t *scratch, int *flags, cudaStream_t s, bool withhold_first_tile)
{
    const int passes = (bits + 7) / 8;
    if (passes <= 0)
        return 0;
    const uint32_t tiles = div_up(cap ? cap : 1, kSortTile);
    const OsLayout L = os_layout(scratch, tiles);
    // clear the ids, histograms and the status words of the passes used
    cudaMemsetAsync(scratch, 0, (size_t)((uint8_t *)L.status - scratch) + sizeof(unsigned long long) * 256 *
                                    (size_t)tiles * passes, s);
    if (withhold_first_tile) {
        // self-test of the bounded wait: tile ids of the first pass start at
        // 1, so tile 0 never publishes and every later tile gives up
        static const uint32_t one = 1;
        cudaMemcpyAsync(L.counters, &one, sizeof one, cudaMemcpyHostToDevice, s);
    }
    const uint32_t hb = std::min<uint32_t>(tiles, 4 * 152);
    k_os_hist<<<hb, kSortThreads, 0, s>>>(keys[0], n_dev, cap, passes, bits, L.ghist);
    k_os_scan<<<1, 256, 0, s>>>(L.ghist, passes, L.gbase);
    g_launches += 2;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        k_os_pass<<<tiles, kSortThreads, 0, s>>>(keys[cur], vals[cur], n_dev, cap, 8 * p, os_digit_mask(bits, p),
                                                 L.gbase + 256 * p,
                                                 L.status + (size_t)p * tiles * 256, L.counters + p,
                                                 keys[cur ^ 1], vals[cur ^ 1], flags);
        ++g_launches;
        cur ^= 1;
    }
    return cur;
}

int sort_u32(uint32_t *keys[2], uint32_t *vals[2], const uint32_t *n_dev, uint32_t cap, int bits, uint32_t *hist,
             uint32_t *hist_partials, cudaStream_t s)
{
    return radix_sort<uint32_t>(keys, vals, n_dev, cap, bits, hist, hist_partials, s);
}

int bin2(const BinArgs &a, cudaStream_t s)
{
    const uint32_t R = a.n_records;
    const uint32_t nb = div_up(R ? R : 1, kScanTile);
    k_vis_partials<<<nb, kScanThreads, 0, s>>>(a.counts, R, a.partials);
    k_scan_top<<<1, 1024, 0, s>>>(a.partials, nb, a.n_vis);
    k_vis_compact<<<nb, kScanThreads, 0, s>>>(a.counts, a.rec, R, a.partials, a.dkeys[0], a.dvals[0]);
    g_launches += 3;
    uint32_t *dk[2] = {a.dkeys[0], a.dkeys[1]}, *dv[2] = {a.dvals[0], a.dvals[1]};
    const int dc = a.os_scratch ? onesweep_u32(dk, dv, a.n_vis, R, 32, a.os_scratch, a.flags, s)
                                : radix_sort<uint32_t>(dk, dv, a.n_vis, R, 32, a.hist, a.hist_partials, s);
    // tile counts in depth order and their exclusive scan (total = n_dups),
    // in the depth-key buffers the sort no longer needs
    uint32_t *cnt = dk[dc], *offs = dk[dc ^ 1];
    k_sorted_counts<<<div_up(R ? R : 1, 256), 256, 0, s>>>(a.counts, dv[dc], a.n_vis, R, cnt);
    ++g_launches;
    scan_excl(cnt, offs, R, a.partials, a.n_dups, s);
    k_emit_balanced<<<div_up(a.capacity ? a.capacity : 1, kScanTile), kScanThreads, 0, s>>>(a, dv[dc], offs,
                                                                                          a.tkeys[0], a.vals[0]);
    ++g_launches;
    uint32_t *tk[2] = {a.tkeys[0], a.tkeys[1]}, *tv[2] = {a.vals[0], a.vals[1]};
    const int tc = a.os_scratch
                       ? onesweep_u32(tk, tv, a.n_dups, a.capacity, a.key_bits - 32, a.os_scratch, a.flags, s)
                       : radix_sort<uint32_t>(tk, tv, a.n_dups, a.capacity, a.key_bits - 32, a.hist, a.hist_partials,
                                              s);
    cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)a.n_tiles, s);
    k_ranges<uint32_t><<<div_up(a.capacity ? a.capacity : 1, 256), 256, 0, s>>>(tk[tc], a.n_dups, a.capacity,
                                                                                a.ranges);
    ++g_launches;
    return tc;
}

void keys64(const BinArgs &a, int cur, uint64_t *out, cudaStream_t s)
{
    k_keys64<<<div_up(a.capacity ? a.capacity : 1, 256), 256, 0, s>>>(a.tkeys[cur], a.vals[cur], a.rec, a.n_dups,
                                                                      a.capacity, out);
    ++g_launches;
}

int bin(const BinArgs &a, cudaStream_t s)
{
    bin_count(a, s);
    const uint32_t nb = div_up(a.n_records ? a.n_records : 1, kScanTile);
    k_emit<<<nb, kScanThreads, 0, s>>>(a, a.partials);
    ++g_launches;
    const uint32_t sb = div_up(a.capacity ? a.capacity : 1, kSortTile);
    const size_t hn = (size_t)256 * sb;
    int cur = 0;
    for (int shift = 0; shift < a.key_bits; shift += 8) {
        k_rs_hist<<<sb, kSortThreads, 0, s>>>(a.keys[cur], a.n_dups, a.capacity, shift, a.hist, sb);
        scan_excl(a.hist, a.hist, hn, a.hist_partials, nullptr, s);
        k_rs_scatter<<<sb, kSortThreads, 0, s>>>(a.keys[cur], a.vals[cur], a.n_dups, a.capacity, shift, a.hist, sb,
                                                 a.keys[cur ^ 1], a.vals[cur ^ 1]);
        g_launches += 2;
        cur ^= 1;
    }
    cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)a.n_tiles, s);
    k_ranges<<<div_up(a.capacity ? a.capacity : 1, 256), 256, 0, s>>>(a.keys[cur], a.n_dups, a.capacity, a.ranges);
    ++g_launches;
    return cur;
}

}  // namespace gsl
