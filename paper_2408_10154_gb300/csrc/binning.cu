// binning.cu -- tile lists: for every tile, the records whose tile
// rectangle covers it, ordered by (depth bits, record index).
//
// Segmented build (the context paths and gs_bin): per-keyframe 2-D
// difference grids of the records' rectangles give every tile's list length
// and start without sorting the duplicates; records are placed into their
// tiles through per-tile atomic cursors and each short list is then sorted
// on its own (registers, shared memory, or global memory for the rare long
// list).  One-stage route (gs_render_noalloc): exclusive scan of the
// tiles-touched counts, emission of 64-bit (tile << 32 | depth bits) keys,
// stable LSD radix sort, per-tile ranges.  Also the one-sweep LSD radix sort
// of 32-bit keys (gs_sort_u32) and the longest-first tile schedule.
//
// All sizes that depend on the data live on the device, so every sequence
// can be captured in a CUDA graph: grids are sized for the capacity and
// blocks past the live count exit early.
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
// tile of a 64-bit (tile << 32 | depth) key
__device__ __forceinline__ uint32_t tile_of(uint64_t k) { return (uint32_t)(k >> 32); }

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

// --------------------------------------------------------- segmented build
// Tile lists without a global sort: every record adds its tile rectangle to
// its keyframe's 2-D difference grid, whose prefix sums give each tile's
// list length and start; records are then placed into their tiles' lists
// through per-tile atomic cursors (in no particular order), and each list is
// sorted on its own by (depth bits, record index) -- the order of a stable
// depth sort of the records, as the key is unique.

// keyframe of record r: the last vp whose records start at or before r
__device__ __forceinline__ int vp_of_record(const VpDesc *vps, int n_vps, uint32_t r)
{
    int lo = 0, hi = n_vps - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vps[mid].rec_base <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

struct SegRect {
    uint32_t x0, x1, y0, y1;
};

__device__ __forceinline__ SegRect seg_rect(const float4 *rec, uint32_t r)
{
    const uint32_t rx = __float_as_uint(rec[3 * (size_t)r + 1].w);
    const uint32_t ry = __float_as_uint(rec[3 * (size_t)r + 2].w);
    return SegRect{rx & 0xffffu, rx >> 16, ry & 0xffffu, ry >> 16};
}

// a record takes part when its rectangle lies in its keyframe's tile grid
// and matches its count (records from the projection always do; gs_bin's
// caller-supplied ones are checked here, the same way in every kernel)
__device__ __forceinline__ bool seg_valid(const SegRect &q, const VpDesc &d, int count)
{
    return q.x0 < q.x1 && q.x1 <= (uint32_t)d.TX && q.y0 < q.y1 && q.y1 <= (uint32_t)d.TY &&
           (uint32_t)count == (q.x1 - q.x0) * (q.y1 - q.y0);
}

constexpr int kSegThreads = 256;

// One thread per record (gs_bin: records supplied by the caller; the
// context paths do this inside the projection): a valid visible record adds
// its rectangle to its keyframe's difference grid (+1 at (y0, x0) and
// (y1, x1), -1 mod 2^32 at (y0, x1) and (y1, x0));
// every record writes its entry (size 0 when not taking part).
__global__ void __launch_bounds__(kSegThreads) k_seg_collect(const gsl::BinArgs a)
{
    const uint32_t r = blockIdx.x * kSegThreads + threadIdx.x;
    if (r >= a.n_records)
        return;
    const int c = a.counts[r];
    const int vp = c > 0 ? vp_of_record(a.vps, a.n_vps, r) : 0;
    const VpDesc &d = a.vps[vp];
    const SegRect q = c > 0 ? seg_rect(a.rec, r) : SegRect{0, 0, 0, 0};
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    if (c > 0 && seg_valid(q, d, c)) {
        const uint32_t w1 = (uint32_t)d.TX + 1;
        uint32_t *g = a.seg_diff + d.diff_base;
        atomicAdd(g + q.y0 * w1 + q.x0, 1u);
        atomicAdd(g + q.y1 * w1 + q.x1, 1u);
        atomicAdd(g + q.y0 * w1 + q.x1, 0xffffffffu);
        atomicAdd(g + q.y1 * w1 + q.x0, 0xffffffffu);
        e = make_uint4(__float_as_uint(a.rec[3 * (size_t)r + 1].z), d.tile_base + q.y0 * (uint32_t)d.TX + q.x0,
                       (q.x1 - q.x0) | ((q.y1 - q.y0) << 16), (uint32_t)d.TX);
    }
    a.seg_list[r] = e;
}

constexpr int kSegTileThreads = 512;

// inclusive block scan of one value per thread (kSegTileThreads threads)
__device__ __forceinline__ unsigned long long block_incl_scan(unsigned long long v, unsigned long long *s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    if (lane == 31)
        s_w[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < kSegTileThreads / 32 ? s_w[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += u;
        }
        if (lane < kSegTileThreads / 32)
            s_w[lane] = x;
    }
    __syncthreads();
    const unsigned long long r = v + (warp ? s_w[warp - 1] : 0ull);
    __syncthreads();
    return r;
}

// One CTA per keyframe: 2-D prefix sums of its difference grid (rows, then
// columns) turn it into the tile counts, written back in place, and the
// keyframe's duplicate total goes to seg_hdr[1 + v].  SMEM: the TY x TX
// counting cells are summed in shared memory (dynamic, a.seg_max_cells
// words); otherwise in place in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(kSegTileThreads) k_seg_count(const gsl::BinArgs a)
{
    extern __shared__ uint32_t s_grid[];
    __shared__ unsigned long long s_w[kSegTileThreads / 32];
    const int v = blockIdx.x;
    const VpDesc &d = a.vps[v];
    const int TX = d.TX, TY = d.TY, w1 = TX + 1;
    uint32_t *g = a.seg_diff + d.diff_base;
    const uint32_t nt = (uint32_t)TX * (uint32_t)TY;
    uint32_t *c = SMEM ? s_grid : g;
    const int pitch = SMEM ? TX : w1;
    if (SMEM) {
        for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x)
            s_grid[i] = g[(size_t)(i / (uint32_t)TX) * w1 + i % (uint32_t)TX];
        __syncthreads();
    }
    for (int y = threadIdx.x; y < TY; y += blockDim.x) {
        uint32_t acc = 0;
        uint32_t *row = c + (size_t)y * pitch;
        for (int x = 0; x < TX; ++x) {
            acc += row[x];
            row[x] = acc;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < TX; x += blockDim.x) {
        uint32_t acc = 0;
        for (int y = 0; y < TY; ++y) {
            acc += c[(size_t)y * pitch + x];
            c[(size_t)y * pitch + x] = acc;
        }
    }
    __syncthreads();
    unsigned long long sum = 0;
    for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x) {
        const uint32_t y = i / (uint32_t)TX, x = i % (uint32_t)TX;
        const uint32_t n = c[(size_t)y * pitch + x];
        if (SMEM)
            g[(size_t)y * w1 + x] = n;
        sum += n;
    }
    const unsigned long long tot = block_incl_scan(sum, s_w);
    if (threadIdx.x == kSegTileThreads - 1)
        a.seg_hdr[1 + v] = tot;
}

// One CTA per keyframe: an exclusive scan of its tile counts in tile order,
// offset by the totals of the earlier keyframes, gives each tile's start.
// Writes the ranges ((0, 0) when empty; clipped to the capacity), the
// placement cursors, and (CTA 0) the duplicate total and the capacity flag.
__global__ void __launch_bounds__(kSegTileThreads) k_seg_ranges(const gsl::BinArgs a)
{
    __shared__ unsigned long long s_w[kSegTileThreads / 32];
    __shared__ unsigned long long s_base;
    const int v = blockIdx.x;
    const VpDesc &d = a.vps[v];
    const int TX = d.TX, w1 = TX + 1;
    const uint32_t *g = a.seg_diff + d.diff_base;
    const unsigned long long *tot = a.seg_hdr + 1;
    unsigned long long before = 0, all = 0;
    for (int k = threadIdx.x; k < a.n_vps; k += blockDim.x) {
        const unsigned long long t = tot[k];
        before += k < v ? t : 0ull;
        all += t;
    }
    const unsigned long long base = block_incl_scan(before, s_w);
    const unsigned long long grand = block_incl_scan(all, s_w);
    if (threadIdx.x == kSegTileThreads - 1) {
        s_base = base;
        if (v == 0) {
            *a.n_dups = grand < 0xffffffffull ? (uint32_t)grand : 0xffffffffu;
            if (grand > a.capacity)
                atomicOr(a.flags, kFlagCapacity);
        }
    }
    __syncthreads();
    // each thread scans a contiguous run of tiles; one block scan joins the runs
    const uint32_t nt = (uint32_t)TX * (uint32_t)d.TY;
    const uint32_t per = (nt + kSegTileThreads - 1) / kSegTileThreads;
    const uint32_t l0 = min(threadIdx.x * per, nt), l1 = min(l0 + per, nt);
    auto cell = [&](uint32_t lt) { return g[(size_t)(lt / (uint32_t)TX) * w1 + lt % (uint32_t)TX]; };
    unsigned long long run = 0;
    for (uint32_t lt = l0; lt < l1; ++lt)
        run += cell(lt);
    unsigned long long st = s_base + block_incl_scan(run, s_w) - run;
    const unsigned long long cap = a.capacity;
    for (uint32_t lt = l0; lt < l1; ++lt) {
        const uint32_t n = cell(lt);
        const unsigned long long en = st + n;
        const uint32_t t = d.tile_base + lt;
        // (0, 0) for an empty tile
        a.ranges[t] = n ? make_uint2((uint32_t)(st < cap ? st : cap), (uint32_t)(en < cap ? en : cap))
                        : make_uint2(0u, 0u);
        a.seg_cursor[t] = (uint32_t)(st < cap ? st : cap);
        st = en;
    }
}

constexpr uint32_t kSegSmall = 4;  // tiles of a record placed by its own thread; more: by the whole warp
constexpr int kSegPerThread = 2;    // records per thread (more cursor atomics in flight per warp)
constexpr int kSegRounds = 8;       // a large record: rounds of 32 tiles whose atomics are in flight together

// kSegPerThread records per thread (kSegThreads apart, so each load is
// coalesced): a visible one writes (depth bits, record) into the lists of
// the tiles of its rectangle (from its seg_list entry) at positions taken
// from the tiles' cursors, all cursor atomics of the thread in flight
// before its stores.  Records with more than kSegSmall tiles are spread over
// the lanes of their warp, one record at a time, so a splat covering
// thousands of tiles does not serialise one thread, kSegRounds rounds of 32
// tiles with all their atomics in flight before the stores (a record over a
// whole 1200x680 frame is 101 rounds: one atomic round trip each made it
// the kernel's critical path).  Positions at or past the capacity are
// dropped (the capacity flag is already set).
__global__ void __launch_bounds__(kSegThreads) k_seg_place(const gsl::BinArgs a)
{
    const int lane = threadIdx.x & 31;
    uint32_t cnt[kSegPerThread], t0[kSegPerThread], w[kSegPerThread], tx[kSegPerThread], zb[kSegPerThread],
        rr[kSegPerThread];
#pragma unroll
    for (int q = 0; q < kSegPerThread; ++q) {
        const uint32_t r = (blockIdx.x * kSegPerThread + q) * kSegThreads + threadIdx.x;
        rr[q] = r;
        cnt[q] = 0;
        t0[q] = 0;
        w[q] = 1;
        tx[q] = 0;
        zb[q] = 0;
        if (r < a.n_records) {
            const uint4 e = a.seg_list[r];
            if (e.z) {
                zb[q] = e.x;
                t0[q] = e.y;
                w[q] = e.z & 0xffffu;
                cnt[q] = w[q] * (e.z >> 16);
                tx[q] = e.w;
            }
        }
    }
    uint32_t pos[kSegPerThread][kSegSmall];
#pragma unroll
    for (int q = 0; q < kSegPerThread; ++q) {
        if (cnt[q] > kSegSmall)
            continue;
        uint32_t col = 0, row = t0[q];
#pragma unroll
        for (uint32_t k = 0; k < kSegSmall; ++k) {
            if (k < cnt[q]) {
                pos[q][k] = atomicAdd(a.seg_cursor + row + col, 1u);
                if (++col == w[q]) {
                    col = 0;
                    row += tx[q];
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kSegPerThread; ++q) {
        if (cnt[q] > kSegSmall)
            continue;
#pragma unroll
        for (uint32_t k = 0; k < kSegSmall; ++k) {
            if (k < cnt[q] && pos[q][k] < a.capacity) {
                a.tkeys[0][pos[q][k]] = zb[q];
                a.vals[0][pos[q][k]] = rr[q];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kSegPerThread; ++q) {
        unsigned m = __ballot_sync(0xffffffffu, cnt[q] > kSegSmall);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t c = __shfl_sync(0xffffffffu, cnt[q], src), b = __shfl_sync(0xffffffffu, t0[q], src);
            const uint32_t ww = __shfl_sync(0xffffffffu, w[q], src), tt = __shfl_sync(0xffffffffu, tx[q], src);
            const uint32_t z = __shfl_sync(0xffffffffu, zb[q], src), r = __shfl_sync(0xffffffffu, rr[q], src);
            for (uint32_t k0 = 0; k0 < c; k0 += 32 * kSegRounds) {
                uint32_t pos[kSegRounds];
#pragma unroll
                for (int u = 0; u < kSegRounds; ++u) {
                    const uint32_t k = k0 + 32 * u + lane;
                    if (k < c)
                        pos[u] = atomicAdd(a.seg_cursor + b + (k / ww) * tt + k % ww, 1u);
                }
#pragma unroll
                for (int u = 0; u < kSegRounds; ++u) {
                    const uint32_t k = k0 + 32 * u + lane;
                    if (k < c && pos[u] < a.capacity) {
                        a.tkeys[0][pos[u]] = z;
                        a.vals[0][pos[u]] = r;
                    }
                }
            }
        }
    }
}

// Ascending bitonic sort with "flip" merges: merging two sorted halves of a
// block of size k compares element i of the block with element k - 1 - i,
// after which every element of the lower half is at most every element of
// the upper one and each half is bitonic; half-cleaners at distances
// k/4, ..., 1 then sort each half.  Only ascending compare-exchanges occur,
// so positions past the list end act as +infinity and their exchanges can
// be skipped.

// 32 keys, one per lane (lanes past the list hold ~0)
__device__ __forceinline__ unsigned long long warp_bitonic32(unsigned long long x, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
        {
            // the lower position keeps the smaller key, the upper the larger
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, k - 1);
            const bool lower = (lane & (k >> 1)) == 0;
            x = (y < x) == lower ? y : x;
        }
#pragma unroll
        for (int j = k >> 2; j >= 1; j >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
            const bool lower = (lane & j) == 0;
            x = (y < x) == lower ? y : x;
        }
    }
    return x;
}

// 32 K keys in registers, element k * 32 + lane in slot k of its lane
// (positions past the list hold ~0): the same network, with exchanges at
// distances below 32 done by shuffles and at 32 and above inside a lane.
template <int K>
__device__ __forceinline__ void warp_bitonic_reg(unsigned long long (&x)[K], int lane)
{
    // the lower position keeps the smaller key, the upper the larger
    auto pick = [](unsigned long long u, unsigned long long v, bool lower) { return (v < u) == lower ? v : u; };
#pragma unroll
    for (int size = 2; size <= 32 * K; size <<= 1) {
        if (size <= 32) {
            const bool lower = (lane & (size >> 1)) == 0;
#pragma unroll
            for (int k = 0; k < K; ++k)
                x[k] = pick(x[k], __shfl_xor_sync(0xffffffffu, x[k], size - 1), lower);
        } else {
            // partner of k * 32 + lane: slot k ^ (size / 32 - 1) of lane ^ 31
            unsigned long long y[K];
#pragma unroll
            for (int k = 0; k < K; ++k)
                y[k] = __shfl_xor_sync(0xffffffffu, x[k ^ (size / 32 - 1)], 31);
#pragma unroll
            for (int k = 0; k < K; ++k)
                x[k] = pick(x[k], y[k], (k & (size / 64)) == 0);
        }
#pragma unroll
        for (int j = size >> 2; j >= 1; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if ((k & (j / 32)) == 0) {
                        const unsigned long long u = x[k], v = x[k | (j / 32)];
                        const bool sw = v < u;
                        x[k] = sw ? v : u;
                        x[k | (j / 32)] = sw ? u : v;
                    }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int k = 0; k < K; ++k)
                    x[k] = pick(x[k], __shfl_xor_sync(0xffffffffu, x[k], j), lower);
            }
        }
    }
}

template <int K>
__device__ __forceinline__ void sort_list_reg(const uint32_t *keys, uint32_t *vals, uint32_t n, int lane)
{
    unsigned long long x[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t e = (uint32_t)(k * 32 + lane);
        x[k] = e < n ? (((unsigned long long)keys[e] << 32) | vals[e]) : ~0ull;
    }
    warp_bitonic_reg<K>(x, lane);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t e = (uint32_t)(k * 32 + lane);
        if (e < n)
            vals[e] = (uint32_t)x[k];
    }
}

__device__ __forceinline__ void cex(unsigned long long *s, int i, int p)
{
    const unsigned long long u = s[i], v = s[p];
    if (u > v) {
        s[i] = v;
        s[p] = u;
    }
}

constexpr int kSegSortWarps = 8;
constexpr int kSegSortCap = 512;  // longest list sorted by one warp in shared memory

// One warp per tile: lists of up to 256 entries are sorted in registers (up
// to 8 per lane), up to kSegSortCap in shared memory (padded with ~0 to a
// power of two);
// longer lists are queued for k_seg_sort_big.  The sorted record indices
// replace the tile's values in place.
__global__ void __launch_bounds__(kSegSortWarps * 32) k_seg_sort(const gsl::BinArgs a)
{
    __shared__ unsigned long long s_k[kSegSortWarps][kSegSortCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t t = blockIdx.x * kSegSortWarps + warp;
    if (t >= a.n_tiles)
        return;
    const uint2 rg = a.ranges[t];
    const uint32_t n = rg.y - rg.x;
    if (n <= 1)
        return;
    const uint32_t *keys = a.tkeys[0] + rg.x;
    uint32_t *vals = a.vals[0] + rg.x;
    if (n <= 32) {
        unsigned long long x = ~0ull;
        if ((uint32_t)lane < n)
            x = ((unsigned long long)keys[lane] << 32) | vals[lane];
        x = warp_bitonic32(x, lane);
        if ((uint32_t)lane < n)
            vals[lane] = (uint32_t)x;
        return;
    }
    if (n <= 64) {
        sort_list_reg<2>(keys, vals, n, lane);
        return;
    }
    if (n <= 128) {
        sort_list_reg<4>(keys, vals, n, lane);
        return;
    }
    if (n <= 256) {
        sort_list_reg<8>(keys, vals, n, lane);
        return;
    }
    if (n > (uint32_t)kSegSortCap) {
        if (lane == 0)
            a.seg_big[atomicAdd(a.seg_hdr, 1ull)] = t;
        return;
    }
    int N = 512;
    while ((uint32_t)N < n)
        N <<= 1;
    unsigned long long *sk = s_k[warp];
    for (int i = lane; i < N; i += 32)
        sk[i] = (uint32_t)i < n ? (((unsigned long long)keys[i] << 32) | vals[i]) : ~0ull;
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1) {
        const int h = k >> 1;
        for (int q = lane; q < (N >> 1); q += 32) {
            const int i = (q / h) * k + (q & (h - 1));
            cex(sk, i, i + k - 1 - 2 * (q & (h - 1)));
        }
        __syncwarp();
        for (int j = k >> 2; j >= 1; j >>= 1) {
            for (int q = lane; q < (N >> 1); q += 32) {
                const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                cex(sk, i, i | j);
            }
            __syncwarp();
        }
    }
    for (int i = lane; (uint32_t)i < n; i += 32)
        vals[i] = (uint32_t)sk[i];
}

// 64-bit (tile << 32 | depth bits) keys of the segmented lists, one warp per tile (for gs_bin)
__global__ void __launch_bounds__(256) k_seg_keys64(const gsl::BinArgs a, uint64_t *keys)
{
    const uint32_t t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= a.n_tiles)
        return;
    const uint2 rg = a.ranges[t];
    for (uint32_t i = rg.x + (threadIdx.x & 31); i < rg.y; i += 32)
        keys[i] = ((uint64_t)t << 32) | __float_as_uint(a.rec[3 * (size_t)a.vals[0][i] + 1].z);
}

// Lists longer than kSegSortCap (none on typical views; a splat-dense tile
// close to the camera): one CTA per queued tile, the same network over the
// list in global memory, (key, value) pairs exchanged in place, then the
// values kept.  Slow per element but only ever reached by a few tiles.
__global__ void __launch_bounds__(1024) k_seg_sort_big(const gsl::BinArgs a)
{
    const unsigned long long nb = a.seg_hdr[0];
    for (unsigned long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint2 rg = a.ranges[a.seg_big[b]];
        const uint32_t n = rg.y - rg.x;
        uint32_t *keys = a.tkeys[0] + rg.x;
        uint32_t *vals = a.vals[0] + rg.x;
        uint64_t N = 1;
        while (N < n)
            N <<= 1;
        auto ce = [&](uint64_t i, uint64_t p) {
            if (p >= n)
                return;  // +infinity past the end
            const unsigned long long u = ((unsigned long long)keys[i] << 32) | vals[i];
            const unsigned long long v = ((unsigned long long)keys[p] << 32) | vals[p];
            if (u > v) {
                keys[i] = (uint32_t)(v >> 32);
                vals[i] = (uint32_t)v;
                keys[p] = (uint32_t)(u >> 32);
                vals[p] = (uint32_t)u;
            }
        };
        for (uint64_t k = 2; k <= N; k <<= 1) {
            const uint64_t h = k >> 1;
            for (uint64_t q = threadIdx.x; q < (N >> 1); q += blockDim.x) {
                const uint64_t i = (q / h) * k + (q & (h - 1));
                ce(i, i + k - 1 - 2 * (q & (h - 1)));
            }
            __syncthreads();
            for (uint64_t j = k >> 2; j >= 1; j >>= 1) {
                for (uint64_t q = threadIdx.x; q < (N >> 1); q += blockDim.x) {
                    const uint64_t i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                    ce(i, i | j);
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
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

size_t seg_zero_bytes(int n_vps, uint64_t n_diff)
{
    return sizeof(unsigned long long) * (1 + (size_t)n_vps) + sizeof(uint32_t) * (size_t)n_diff;
}

int bin_seg(const BinArgs &a, cudaStream_t s)
{
    if (!a.seg_counted)
        cudaMemsetAsync(a.seg_hdr, 0, a.seg_zero_bytes, s);
    if (a.n_vps == 0) {
        cudaMemsetAsync(a.n_dups, 0, sizeof(uint32_t), s);
        return 0;
    }
    if (a.n_records && !a.seg_counted) {
        k_seg_collect<<<div_up(a.n_records, kSegThreads), kSegThreads, 0, s>>>(a);
        ++g_launches;
    }
    if (a.seg_max_cells * sizeof(uint32_t) <= 40 * 1024)
        k_seg_count<true><<<a.n_vps, kSegTileThreads, a.seg_max_cells * sizeof(uint32_t), s>>>(a);
    else
        k_seg_count<false><<<a.n_vps, kSegTileThreads, 0, s>>>(a);
    k_seg_ranges<<<a.n_vps, kSegTileThreads, 0, s>>>(a);
    g_launches += 2;
    if (a.n_records) {
        k_seg_place<<<div_up(a.n_records, kSegThreads * kSegPerThread), kSegThreads, 0, s>>>(a);
        ++g_launches;
    }
    if (a.n_tiles) {
        k_seg_sort<<<div_up(a.n_tiles, kSegSortWarps), kSegSortWarps * 32, 0, s>>>(a);
        k_seg_sort_big<<<152, 1024, 0, s>>>(a);
        g_launches += 2;
    }
    return 0;
}

void seg_keys64(const BinArgs &a, uint64_t *out, cudaStream_t s)
{
    if (a.n_tiles == 0)
        return;
    k_seg_keys64<<<div_up(a.n_tiles, 8), 256, 0, s>>>(a, out);
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
