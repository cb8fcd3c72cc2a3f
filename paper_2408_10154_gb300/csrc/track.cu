// track.cu -- the frame-to-model tracking loss (Eq. 2 with the alpha^3 and
// inlier masks of Supp. A) for the tracking keyframes of a plan:
//   k_track_median  one CTA per tracking keyframe: the lower median of the
//                   FP32 depth errors of the pixels with input depth, by a
//                   three-pass radix select over the float's bits (11 + 11 +
//                   10; non-negative floats order as their bit patterns);
//   k_track_loss    one CTA per tile: inlier test e <= 50 * median (FP32),
//                   weight M_in * alpha^3, the tile's loss summed in a fixed
//                   order, and for the standalone entry the cotangents and
//                   the inlier mask.
// The inlier decisions use the FP32 values the oracle's mirror uses, so they
// are reproduced exactly; the weights and the loss are values.
#include "gs_internal.cuh"

namespace {

using namespace gsk;

constexpr uint32_t kInfBits = 0x7f800000u;  // +inf marks a pixel without input depth
constexpr int kMedThreads = 1024;
constexpr int kMedBins = 2048;

__global__ void __launch_bounds__(kMedThreads) k_track_median(const gsl::TrackArgs a)
{
    __shared__ uint32_t hist[kMedBins];
    __shared__ uint32_t s_scan[kMedThreads / 32 + 1];
    __shared__ uint32_t s_sel[2];
    const int vp = a.track_vps[blockIdx.x];
    const VpDesc &d = a.vps[vp];
    const int64_t n = (int64_t)d.W * d.H;
    const float *v = a.err + d.pix_base;
    const int shifts[3] = {21, 10, 0};
    const uint32_t widths[3] = {0x7ffu, 0x7ffu, 0x3ffu};
    uint32_t prefix = 0, mask = 0, k = 0, m = 0;
    for (int pass = 0; pass < 3; ++pass) {
        for (int b = threadIdx.x; b < kMedBins; b += kMedThreads)
            hist[b] = 0;
        __syncthreads();
        for (int64_t base = 0; base < n; base += kMedThreads) {
            const int64_t i = base + threadIdx.x;
            uint32_t dgt = kMedBins;  // not counted
            if (i < n) {
                const uint32_t bits = __float_as_uint(v[i]);
                if (bits < kInfBits && (bits & mask) == prefix)
                    dgt = (bits >> shifts[pass]) & widths[pass];
            }
            const unsigned peers = __match_any_sync(0xffffffffu, dgt);
            if (dgt < (uint32_t)kMedBins && (uint32_t)(__ffs(peers) - 1) == (threadIdx.x & 31u))
                atomicAdd(&hist[dgt], (uint32_t)__popc(peers));
        }
        __syncthreads();
        // exclusive scan of the bins (thread t owns bins 2t and 2t + 1) and
        // the bin holding rank k
        const uint32_t h0 = hist[2 * threadIdx.x], h1 = hist[2 * threadIdx.x + 1];
        uint32_t tot;
        const uint32_t ex = block_excl_scan<kMedThreads>(h0 + h1, s_scan, tot);
        if (pass == 0) {
            m = tot;
            if (m == 0)
                break;
            k = (m - 1) / 2;
        }
        if (k >= ex && k < ex + h0) {
            s_sel[0] = 2 * threadIdx.x;
            s_sel[1] = k - ex;
        } else if (k >= ex + h0 && k < ex + h0 + h1) {
            s_sel[0] = 2 * threadIdx.x + 1;
            s_sel[1] = k - ex - h0;
        }
        __syncthreads();
        prefix |= s_sel[0] << shifts[pass];
        mask |= widths[pass] << shifts[pass];
        k = s_sel[1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.med[vp] = m > 0 ? __uint_as_float(prefix) : 0.0f;
        a.n_valid[vp] = (int)m;
    }
}

__global__ void __launch_bounds__(256) k_track_loss(const gsl::TrackArgs a)
{
    __shared__ float s_red[8];
    const uint32_t t = blockIdx.x;
    const int vp = (int)a.tile_vp[t];
    const VpDesc &d = a.vps[vp];
    if (d.loss_kind != 1)
        return;
    const uint32_t lt = t - d.tile_base;
    const int px = (int)(lt % (uint32_t)d.TX) * kTile + (threadIdx.x & 15);
    const int py = (int)(lt / (uint32_t)d.TX) * kTile + (threadIdx.x >> 4);
    float l = 0.0f;
    if (px < d.W && py < d.H) {
        const int64_t HW = (int64_t)d.W * d.H, off = (int64_t)py * d.W + px, pix = d.pix_base + off;
        const float e = a.err[pix];
        const float thr = 50.0f * a.med[vp];
        const bool in = a.n_valid[vp] > 0 && __float_as_uint(e) < kInfBits && e <= thr;
        const float al = 1.0f - a.t_final[pix];
        const float w = in ? al * al * al : 0.0f;
        if (in)
            l = w * (d.lambda_c * a.col[pix] + (1.0f - d.lambda_c) * e);
        if (a.w)
            a.w[pix] = w;
        if (a.inlier)
            a.inlier[pix] = in ? 1 : 0;
        auto sg = [](float x) -> float { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); };
        if (a.d_rgb)
            for (int ch = 0; ch < 3; ++ch) {
                const int64_t q = 3 * d.pix_base + ch * HW + off;
                a.d_rgb[q] = w * d.lambda_c * sg(a.rgb[q] - d.t_rgb[ch * HW + off]);
            }
        if (a.d_depth)
            a.d_depth[pix] = w * (1.0f - d.lambda_c) * sg(a.depth[pix] - d.t_depth[off]);
    }
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w)
            s += s_red[w];
        a.tile_loss[t] = s;
    }
}

// depth error and colour L1 of rendered images (tracking keyframes)
__global__ void k_track_prep(const gsl::TrackArgs a, const float *rgb, const float *depth, float *err, float *col)
{
    const uint32_t t = blockIdx.x;
    const VpDesc &d = a.vps[a.tile_vp[t]];
    if (d.loss_kind != 1)
        return;
    const uint32_t lt = t - d.tile_base;
    const int px = (int)(lt % (uint32_t)d.TX) * kTile + (threadIdx.x & 15);
    const int py = (int)(lt / (uint32_t)d.TX) * kTile + (threadIdx.x >> 4);
    if (px >= d.W || py >= d.H)
        return;
    const int64_t HW = (int64_t)d.W * d.H, off = (int64_t)py * d.W + px, pix = d.pix_base + off;
    const float ed = depth[pix] - d.t_depth[off];
    err[pix] = d.t_depth[off] > 0.0f ? fabsf(ed) : __uint_as_float(kInfBits);
    float c = 0.0f;
    for (int ch = 0; ch < 3; ++ch)
        c += fabsf(rgb[3 * d.pix_base + ch * HW + off] - d.t_rgb[ch * HW + off]);
    col[pix] = c;
}

}  // namespace

namespace gsl {

void track_loss(const TrackArgs &a, cudaStream_t s)
{
    if (a.n_track <= 0 || a.n_tiles == 0)
        return;
    k_track_median<<<a.n_track, kMedThreads, 0, s>>>(a);
    k_track_loss<<<a.n_tiles, 256, 0, s>>>(a);
    g_launches += 2;
}

void track_prep(const TrackArgs &a, const float *rgb, const float *depth, float *err, float *col, cudaStream_t s)
{
    if (a.n_tiles == 0)
        return;
    k_track_prep<<<a.n_tiles, 256, 0, s>>>(a, rgb, depth, err, col);
    ++g_launches;
}

}  // namespace gsl
