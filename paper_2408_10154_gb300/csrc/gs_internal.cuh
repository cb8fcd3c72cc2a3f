// gs_internal.cuh -- device-side data layout and helpers shared by the
// kernels of libgsreg (sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsreg.h"

namespace gsk {

constexpr int kTile = GS_TILE;        // 16x16 pixels per tile, one CTA each
constexpr int kTilePix = kTile * kTile;
constexpr int kScanTile = 2048;       // items per block in scans and emission
constexpr int kScanThreads = 256;
constexpr int kSortThreads = 256;
constexpr int kSortKPT = 8;           // keys per thread in a radix pass
constexpr int kSortTile = kSortThreads * kSortKPT;
constexpr int kMaxVpPerGroup = 64;    // keyframes sharing one projection pass

// device status word bits
enum : int { kFlagNonFinite = 1, kFlagCapacity = 2, kFlagTimeout = 4 };

// One view-problem: a moving submap seen by one keyframe camera, with its
// own pose, Adam state and (in registration) target images.
struct VpDesc {
    const float4 *means, *scales, *quats, *rgb;
    const float *logits;
    int n;                 // Gaussians of the moving submap
    int W, H, TX, TY;      // image and tile grid
    float fx, fy, cx, cy;
    float w2c[12];         // world -> camera
    uint32_t rec_base;     // first record index
    uint32_t tile_base;    // first global tile id
    uint32_t diff_base;    // first cell of its (TY + 1) x (TX + 1) tile difference grid
    int64_t pix_base;      // first pixel in concatenated per-pixel arrays
    const float *t_rgb;    // registration targets [3][H][W] (or null)
    const float *t_depth;  // [H][W]
    int group;             // projection group
    int set;               // Gaussian set (centroid slot)
    int problem;           // registration problem (fusion)
    int reverse;           // 1: keyframe of P localised in Q (estimate is inverted)
    int iters;             // pose updates of this keyframe's problem (0: the call's count); once
                           // taken, the pose is frozen and later iterations only re-measure the loss
    float lr_rot, lr_trans;  // Adam learning rates of this keyframe's problem
    int loss_kind;         // 0: registration L1 means; 1: tracking loss (Eq. 2, masks of Supp. A)
    float lambda_c;        // tracking loss colour weight
    int exposure;          // 1: the registration loss compares e^a I^ + b (Supp. B) and fits (a, b)
    float lr_exposure;
    float inv3hw, invhw;   // 1 / (3 W H) and 1 / (W H) in FP32 (the L1 means), set on the host
};

// A projection group: vps that share one Gaussian set and are projected by
// the same thread per Gaussian.
struct GroupDesc {
    int vp_first, vp_count;
    int n;
    uint32_t blk_base;     // first block of this group in the projection grid
};

// ------------------------------------------------------------------------
// FP32 decision arithmetic.  These helpers spell out every rounding step
// (round-to-nearest, fused multiply-add only where written) so that every
// integer outcome -- culls, tile rectangles, depth bits, skipped and
// stopping contributors -- is reproducible bit for bit.
// ------------------------------------------------------------------------
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// e^x: Cody-Waite reduction k = round(x log2 e), r = x - k ln2 (two-part
// ln2), degree-6 Taylor polynomial of e^r, exact scaling by 2^k; argument
// clamped to [-80, 80].
__device__ __forceinline__ float exp_ct_core(float x);
__device__ __forceinline__ float exp_ct(float x) { return exp_ct_core(fminf(fmaxf(x, -80.0f), 80.0f)); }
// the same function for x <= 0 (or NaN, which the lower clamp maps to -80
// either way): the upper clamp is a no-op there and is left out
__device__ __forceinline__ float exp_ct_nonpos(float x) { return exp_ct_core(fmaxf(x, -80.0f)); }
__device__ __forceinline__ float exp_ct_core(float x)
{
    const float magic = 12582912.0f;  // 1.5 * 2^23
    const float t = __fmaf_rn(x, 1.4426950408889634f, magic);
    const float kf = __fsub_rn(t, magic);
    float r = __fmaf_rn(kf, -0.693145751953125f, x);
    r = __fmaf_rn(kf, -1.428606820309417e-06f, r);
    float p = 1.3888888888888889e-03f;       // 1/720
    p = __fmaf_rn(p, r, 8.3333333333333333e-03f);  // 1/120
    p = __fmaf_rn(p, r, 4.1666666666666667e-02f);  // 1/24
    p = __fmaf_rn(p, r, 1.6666666666666667e-01f);  // 1/6
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    // p * 2^k with k = kf: t = 1.5 * 2^23 + k holds k in its low mantissa
    // bits (|k| <= 116 here), and the bit pattern of 1.5 * 2^23 (0x4B400000)
    // is 0 in its low 9 bits, so bits(t) << 23 = k << 23 (mod 2^32).  p lies
    // in [0.7, 1.5) and p 2^k stays a normal number, so adding k to p's
    // exponent field is the exact product __fmul_rn(p, 2^k), bit for bit.
    return __int_as_float(__float_as_int(p) + (int)((uint32_t)__float_as_int(t) << 23));
}

// ln x for a positive normal x (the tight tile lists' threshold): x = m 2^e
// with m in [sqrt(1/2), sqrt(2)), ln m = 2 artanh(s) with s = (m - 1) /
// (m + 1), |s| <= 0.1716, by the odd series 2 (s + s^3/3 + ... + s^9/9)
// (first omitted term below 2e-10), plus e ln 2.  A fixed FP32 operation
// sequence (no library logarithm), so the oracle takes the same value.
__device__ __forceinline__ float log_ct(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421354f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = 0.222222222f;              // 2/9
    p = __fmaf_rn(p, s2, 0.285714286f);  // 2/7
    p = __fmaf_rn(p, s2, 0.4f);          // 2/5
    p = __fmaf_rn(p, s2, 0.666666667f);  // 2/3
    p = __fmaf_rn(p, s2, 2.0f);
    return __fmaf_rn((float)e, 0.693147181f, __fmul_rn(s, p));
}

// hi + lo += bhi + blo without losing the rounding error of the high parts
// (Knuth's TwoSum: e is exactly the error of hi + bhi); FP32 only -- the
// FP64 pipe of this part is a small fraction of its FP32 rate.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float bhi, float blo)
{
    const float s = hi + bhi;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (bhi - bp);
    hi = s;
    lo = lo + blo + e;
}

// M = V o T (3x4 row-major) in FP32
__device__ __forceinline__ void compose_ct(const float *V, const float *T, float *M)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float v0 = V[4 * i], v1 = V[4 * i + 1], v2 = V[4 * i + 2];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            M[4 * i + j] = fma_rn(v2, T[8 + j], fma_rn(v1, T[4 + j], mul_rn(v0, T[j])));
        M[4 * i + 3] = fma_rn(v2, T[11], fma_rn(v1, T[7], fma_rn(v0, T[3], V[4 * i + 3])));
    }
}

// ------------------------------------------------------------------------
// small utilities
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// exclusive block scan of one uint32 per thread (blockDim.x = BLOCK)
template <int BLOCK>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *s_warp, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += y;
    }
    if (lane == 31)
        s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < BLOCK / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += y;
        }
        if (lane < BLOCK / 32)
            s_warp[lane] = wi - w;
        if (lane == BLOCK / 32 - 1)
            s_warp[BLOCK / 32] = wi;
    }
    __syncthreads();
    total = s_warp[BLOCK / 32];
    const uint32_t r = s_warp[warp] + inc - x;
    __syncthreads();
    return r;
}

}  // namespace gsk

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files; all enqueue on `s`)
// ---------------------------------------------------------------------------
namespace gsl {

// kernels launched (or captured) by this library since load; each launch
// site adds one
extern long long g_launches;

struct ProjectArgs {
    const gsk::VpDesc *vps;
    const gsk::GroupDesc *groups;
    int n_groups;
    uint32_t n_blocks;
    const float *pose32;      // [vp][12]
    float z_near, dilation;
    int smooth;
    float4 *rec;               // [records][3] main record (AoS, 48 B)
    float4 *aux;               // [records][2] auxiliary (may be null)
    int32_t *counts;          // tiles touched per record (null: not written; the segmented
                              // lists read the seg_list entries instead)
    int *flags;
    // tight lists: shrink each rectangle to the tiles that meet the
    // axis-aligned box of the record's alpha-threshold ellipse (exponent >=
    // ln(alpha_min / o) - 0.06, box widened by 0.1 % + 0.01 px; nearly
    // singular conics keep the 3-sigma rectangle; see tighten in
    // project.cu).  The dropped (tile, record) pairs fail the alpha test at
    // every pixel of the tile, so the compositing is unchanged; the lists
    // (and list positions such as `last`) are shorter.
    int tight;
    float alpha_min;          // the threshold of the tight rectangles
    // segmented tile lists (null: not built here): clears seg_hdr/seg_diff
    // (seg_zero_bytes), then every visible record adds its rectangle to its
    // keyframe's difference grid, and every record writes its seg_list
    // entry (see BinArgs)
    unsigned long long *seg_hdr;
    uint32_t *seg_diff;
    size_t seg_zero_bytes;
    uint4 *seg_list;
};
void project(const ProjectArgs &a, cudaStream_t s);

// exclusive scan of n uint32 (n host-known); partials sized scan_partials(n)
size_t scan_partials(size_t n);
void scan_excl(const uint32_t *in, uint32_t *out, size_t n, uint32_t *partials, uint32_t *total,
               cudaStream_t s);

struct BinArgs {
    const gsk::VpDesc *vps;
    int n_vps;
    const int32_t *counts;
    const float4 *rec;         // [records][3]
    uint32_t n_records;
    uint32_t *partials;       // scan_partials(n_records)
    uint32_t *n_dups;         // device scalar out (may exceed capacity)
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint32_t capacity;
    uint32_t *hist;           // 256 * sort blocks(capacity)
    uint32_t *hist_partials;  // scan_partials(256 * sort blocks)
    int key_bits;             // bits of (tile << 32 | depth) to sort
    uint2 *ranges;            // [total tiles]
    uint32_t n_tiles;
    int *flags;
    uint32_t *tkeys[2];             // [capacity] segmented build: depth bits of the placed entries (tkeys[0])
    // segmented build (bin_seg): seg_hdr[0] counts the tiles queued for the
    // long-list sort, seg_hdr[1 + v] holds keyframe v's duplicate total, and
    // the difference grids (VpDesc::diff_base) follow in the same allocation
    // of seg_zero_bytes, cleared at the start of every build.  seg_list: per
    // record {depth bits, first tile, width | height << 16, tiles per row}
    // (size 0: not visible).  seg_counted: the projection has already
    // cleared, counted and written the entries (ProjectArgs::seg_*);
    // otherwise bin_seg does it from rec / counts.
    unsigned long long *seg_hdr;
    uint32_t *seg_diff;
    size_t seg_zero_bytes;
    uint4 *seg_list;     // [n_records]
    int seg_counted;
    uint32_t *seg_cursor;  // [n_tiles] placement cursors
    uint32_t *seg_big;     // [n_tiles] tiles whose lists exceed the warp sort
    uint32_t seg_max_cells;  // largest TX * TY over the keyframes
};
// emits, sorts and ranges; returns which buffer holds the sorted result
int bin(const BinArgs &a, cudaStream_t s);
// the same lists by the segmented build: per-tile counts from 2-D
// difference grids of the records' tile rectangles, atomic placement, and a
// sort of each tile's list by (depth bits, record); sorted values in vals[0]
// (the return value), the ranges written directly, n_dups set
int bin_seg(const BinArgs &a, cudaStream_t s);
size_t seg_zero_bytes(int n_vps, uint64_t n_diff);
// 64-bit (tile << 32 | depth bits) keys of the lists bin_seg built
void seg_keys64(const BinArgs &a, uint64_t *out, cudaStream_t s);
// Tile schedule for the compositing kernels: tiles ordered by decreasing
// list length (bucketed by the position of the length's top bit; order
// within a bucket arbitrary), so the longest tiles start first and do not
// form the tail of a launch.  counters: 128 uint32 of scratch.
void tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, uint32_t *counters, cudaStream_t s);

// One-sweep LSD radix sort of 32-bit keys (8-bit digits): one histogram
// kernel for every digit, one scan of the digit counts, one scatter per
// pass whose CTAs find their digit offsets by decoupled look-back (dynamic
// tile ids; every wait bounded, a timeout sets kFlagTimeout).  Same stable
// order as radix_sort.  Returns the buffer index holding the result.
size_t onesweep_scratch_bytes(uint32_t cap, int bits);
int onesweep_u32(uint32_t *keys[2], uint32_t *vals[2], const uint32_t *n_dev, uint32_t cap, int bits,
                 uint8_t *scratch, int *flags, cudaStream_t s, bool withhold_first_tile = false);
void bin_count(const BinArgs &a, cudaStream_t s);  // scan only: n_dups
size_t sort_hist_entries(uint32_t capacity);

struct RasterArgs {
    const gsk::VpDesc *vps;
    const uint32_t *tile_vp;  // [tiles] vp of each tile
    uint32_t n_tiles;
    const uint2 *ranges;
    const uint32_t *vals;
    const float4 *rec;        // [records][3]
    const float4 *aux;        // [records][2]
    float alpha_min, alpha_max, t_min, skip_below;
    float bg[3];
    // per-pixel state
    float *t_final;
    int32_t *last;
    uint8_t *code;            // registration: sign code of the loss gradient
    // render outputs (render mode)
    float *out_rgb, *out_depth, *out_alpha;
    // cotangents (backward, render mode)
    const float *d_rgb, *d_depth, *d_alpha;
    // registration / backward outputs
    float *tile_loss;         // [tiles]
    unsigned long long *tile_pairs;  // [2][tiles] += sum of `last`, pairs passing the alpha test
                                     // (count_contrib only); statistics, may be null
    const uint32_t *tile_order;      // CTA -> tile schedule (longest lists first), or null = natural
    uint32_t *queue;                 // registration: work-queue word of the persistent kernels (zeroed
                                     // before each launch), or null = one CTA per tile
    int exposure;                    // some keyframe compensates exposure (forward variant)
    int count_contrib;               // count the pairs that pass the alpha test (forward variant)
    float2 *tile_twist;       // [tiles][6] camera-frame twist as FP32 (hi, lo) pairs (value hi + lo)
    const double *c_cam;      // [vp][3] pivot in camera frame
    float *dup_grads;         // [dups][10] screen-space partials (full mode)
    // tracking-loss keyframes (loss_kind 1): the forward writes the FP32
    // depth error (+inf without input depth) and the colour L1 per pixel;
    // the backward scales the loss signs by the per-pixel mask weight
    float *trk_err, *trk_col;
    const float *trk_w;
    // exposure compensation: [vp][2] gain e^a and offset b; [tiles][2]
    // partial dL/da, dL/db written by the forward
    const float *expo32;
    float *tile_expo;
};
void forward(const RasterArgs &a, bool registration, cudaStream_t s);
void raster_init();  // one-time kernel attributes (before any graph capture)
void backward(const RasterArgs &a, bool registration, bool full, cudaStream_t s);
// Registration forward and adjoint fused per tile (the registration loss
// only: no keyframe may use the tracking loss); the same values as
// forward(a, true) followed by backward(a, true, false), without the
// per-pixel T_final, last and code stores.
void forward_backward(const RasterArgs &a, cudaStream_t s);

// Tracking loss (Eq. 2, masks of Supp. A) of the tracking keyframes of a
// plan: per keyframe the lower median of the valid depth errors (radix
// select), then per pixel the mask weight M_in * alpha^3 and per tile the
// loss (overwriting the tile's registration loss).
struct TrackArgs {
    const gsk::VpDesc *vps;
    const uint32_t *tile_vp;
    uint32_t n_tiles;
    const int *track_vps;     // [n_track] vp indices with loss_kind 1
    int n_track;
    const float *t_final;     // [pix]
    const float *err, *col;   // [pix] from the forward (or k_track_prep)
    float *med;               // [vp] median depth error
    int *n_valid;             // [vp] pixels with input depth
    float *w;                 // [pix] out: M_in * alpha^3
    float *tile_loss;         // [tiles] out
    // standalone gs_track_loss: cotangents and the inlier mask (may be null)
    const float *rgb, *depth;
    float *d_rgb, *d_depth;
    uint8_t *inlier;
};
void track_loss(const TrackArgs &a, cudaStream_t s);
// err / col of rendered images (standalone gs_track_loss)
void track_prep(const TrackArgs &a, const float *rgb, const float *depth, float *err, float *col, cudaStream_t s);

// One submap of a batched rigid update (map adjustment after pose-graph
// optimisation, Eq. 8/9): blocks [blk_base, blk_base + ceil(n / 256)).
struct MapDesc {
    const float4 *means, *quats;
    float4 *out_means, *out_quats;
    int64_t n;
    unsigned blk_base;
    double T[12];
};
void transform_batch(const MapDesc *maps, int n_maps, unsigned blocks, cudaStream_t s);

// Overlap ratio of two submaps (loop filter): moved means of P, exact
// nearest neighbours both ways, reciprocal pairs and those within tau.
struct OverlapArgs {
    const float4 *p, *q;      // means [np], [nq]
    int np, nq;
    const float *T32;         // [12] device, T_{P->Q} rounded to FP32
    float4 *pt;               // [np] scratch: T p
    int32_t *nn_pq, *nn_qp;   // [np], [nq] out
    float *d2;                // [np] out: squared distance to the nearest of Q
    float tau2;               // tau * tau (FP32)
    unsigned long long *counts;  // [2] out: |K|, pairs of K within tau
};
void overlap(const OverlapArgs &a, cudaStream_t s);

// Uniform grid for exact nearest-neighbour search: cell of x is
// floor((x - o) * inv_s) per axis (FP32, clamped to the grid), cells
// numbered x-fastest.  margin bounds how far a cell boundary computed this
// way can sit from o + k s (FP32 rounding of coordinates within the box).
struct NNGrid {
    float ox, oy, oz, s, inv_s, margin;
    int nx, ny, nz;
};
// Scratch of one grid search (targets nt, queries na):
//   cell [nt], start [cells + 1], cursor [cells], spts [nt], sidx [nt],
//   list [na], n_list [1]
struct NNScratch {
    uint32_t *cell, *start, *cursor, *partials;
    float4 *spts;
    int32_t *sidx, *list;
    uint32_t *n_list;
};
// moved means pt = T p and the bounding box of pt and q as ordered-int
// min x, y, z, max x, y, z in bbox[6]
void overlap_moved_bbox(const OverlapArgs &a, uint32_t *bbox, cudaStream_t s);
// exact nearest neighbour in targets B of every query in A (FP32 squared
// distance, ties to the smaller index): a grid search that stops once no
// unsearched cell can hold a nearer target, and the brute-force sweep for
// the queries whose search would run past kNNMaxRing rings
// the grid of the targets B: their cells, per-cell starts, and the targets
// (sidx: their indices) in cell order
void nn_grid_build(const float4 *B, int nb, const NNGrid &g, const NNScratch &sc, cudaStream_t s);
// the search of every query of A in the grid of B built into sc; thread t
// takes query order[t] when order is given (a permutation of 0..na-1)
void nn_grid_search(const float4 *A, int na, const int32_t *order, const float4 *B, int nb, const NNGrid &g,
                    const NNScratch &sc, int32_t *nn, float *d2, cudaStream_t s);
// |K| and the pairs within tau from the nearest neighbours both ways
void overlap_count(const OverlapArgs &a, cudaStream_t s);

struct PoseArgs {
    const gsk::VpDesc *vps;
    int n_vps;
    const float2 *tile_twist;  // [tiles][6] (hi, lo)
    const float *tile_loss;    // [tiles]
    double *pose64;            // [vp][12]
    float *pose32;             // [vp][12]
    double *adam;              // [vp][13]
    double *pivot;             // [vp][3] world
    double *c_cam;             // [vp][3]
    const double *centroid;    // [set][3]
    double *loss;              // [vp] last loss
    double *grad;              // [vp][6] last world gradient (may be null)
    double *expo;              // [vp][7] exposure a, b and Adam state (m_a, m_b, v_a, v_b, steps)
    float *expo32;             // [vp][2] gain e^a, offset b for the forward
    const float *tile_expo;    // [tiles][2]
    float lr_rot, lr_trans, beta1, beta2, eps, lr_final;
    int iters;
    int update;                // 0: only reduce loss / gradient
};
void pose_update(const PoseArgs &a, cudaStream_t s);
// gain e^a and offset b (floats) from the FP64 exposure state [vp][7]
void exposure_floats(const double *expo, float *expo32, int n_vps, cudaStream_t s);
// per-keyframe sum of the tile losses (FP64, fixed order)
void loss_reduce(const gsk::VpDesc *vps, int n_vps, const float *tile_loss, double *loss_out, cudaStream_t s);
void pose_init(const PoseArgs &a, cudaStream_t s);
void centroids(const gsk::VpDesc *vps, const int *set_vp, int n_sets, double *centroid, cudaStream_t s);

struct FuseArgs {
    const double *pose64;      // [vp][12]
    const double *eps;         // [vp]
    const int32_t *reverse;    // [vp]
    const int32_t *prob_first, *prob_count;  // [problems]
    int n_problems;
    double *T_out;             // [problems][12]
    double *conf;              // [problems]
    double *est_out;           // [vp][12] estimates of T_{P->Q} (may be null)
};
void fuse(const FuseArgs &a, cudaStream_t s);

void pose_step_raw(int n, double *pose, double *state, const double *grad, const double *pivot, int k, int iters,
                   float lr_rot, float lr_trans, float b1, float b2, float eps, float lr_final, cudaStream_t s);
void loss(const gsk::VpDesc *vps, int n_vps, uint32_t n_tiles, const uint32_t *tile_vp, const float *rgb,
          const float *depth, double *loss, float *d_rgb, float *d_depth, float *tile_loss, cudaStream_t s);
void transform(const float4 *means, const float4 *quats, int64_t n, const double *T, float4 *out_means,
               float4 *out_quats, cudaStream_t s);

// stable LSD radix sort of 32-bit keys with 32-bit values over `bits` low
// bits (device-side count); returns the buffer index of the result
int sort_u32(uint32_t *keys[2], uint32_t *vals[2], const uint32_t *n_dev, uint32_t cap, int bits, uint32_t *hist,
             uint32_t *hist_partials, cudaStream_t s);

// adjoint to every Gaussian parameter of one submap seen by n_vps cameras
struct ParamArgs {
    const gsk::VpDesc *vps;
    int n_vps;
    int n;                    // Gaussians
    const float4 *rec, *aux;  // records of the forward
    const float *pose32;      // [vp][12]
    const float *dup_grads;   // [dups][10] screen gradients, tile-sorted order
    const uint32_t *rpos;     // dup positions grouped by record (filled by param_grads)
    const uint2 *rec_ranges;  // [records] (filled by param_grads)
    const float4 *quats, *scales;
    const float *logits;
    float *g_means, *g_scales, *g_quats, *g_logits, *g_rgb;  // outputs (any may be null)
};
void param_grads(const ParamArgs &a, const uint32_t *sorted_recs, const uint32_t *n_dups, uint32_t cap,
                 uint32_t *rkeys[2], uint32_t *rpos[2], int rec_bits, uint32_t *hist, uint32_t *hist_partials,
                 uint2 *rec_ranges, uint32_t n_records, cudaStream_t s);


}  // namespace gsl
