// raster.cu -- front-to-back compositing (forward) and back-to-front adjoint
// (backward) of the tiled 3D Gaussian splatting renderer.
//
// Forward: one CTA of 128 threads per 16x16 tile, two pixels per thread
// (same column, 4 rows apart; each warp on an 8x8 patch), both walked with
// packed f32x2 operations.  The tile's depth-sorted list is staged through
// shared memory 256 records at a time, each warp iterates only the records
// that can reach alpha_min in its patch, and the CTA stops once every pixel
// is opaque (transmittance would drop below t_min).  In registration mode
// it fuses the loss: it reads the keyframe's colour and depth
// (exposure-compensated colour if asked), accumulates the tile's L1 loss and
// stores a 1-byte sign code of dL/dpixel next to the final transmittance and
// the last-contributor index.  Nothing else per pixel is saved; the adjoint
// recomputes alpha and recovers transmittance by division.
//
// Adjoint: 128 threads per tile, two pixels per thread (8x8 warp patches),
// both walked with packed operations.  Per (pixel, Gaussian)
// screen-space gradients are summed over each warp with shuffles, over the
// tile's warps in shared memory (fixed order), chained through the
// projection into a camera-frame twist per Gaussian, accumulated per thread
// in FP32 with Kahan compensation and reduced per tile by TwoSum butterflies
// to FP32 (hi, lo) pairs -- no global atomics, bit-reproducible.
//
// Registration iterations (the registration loss) run both in one CTA per
// tile (k_fwdbwd): the adjoint walks the forward's pixels from registers
// and, for lists of at most 256 entries, the forward's staging.
#include <float.h>

#include <algorithm>
#include <type_traits>

#include "gs_internal.cuh"

namespace {

using namespace gsk;

// Warp-level cull of a staged record against the warp's pixel patch.  The
// record can only pass the alpha test (alpha >= alpha_min) where its exact
// exponent is at least tau = ln(alpha_min / o), i.e. inside the ellipse
// q(d) = A dx^2 + 2 B dx dy + C dy^2 <= -2 tau about (u, v) (A = -2 ca,
// B = -cb, C = -2 cc).  Over the rectangle [xa, xb] x [ya, yb] of the
// patch's pixel samples the smallest q is 0 when (u, v) lies inside it;
// otherwise it sits on a side that faces (u, v) (q falls along the segment
// from any point of the rectangle to the centre, and that segment leaves
// the rectangle through such a side), where it is the minimum of a 1-D
// quadratic clamped to the side.  The record is dropped for the warp only
// when that minimum exceeds -2 tau, with margins that cover the FP32
// evaluation of the exponent and of this test (tau lowered by 0.06, the
// bound raised by 0.2 % + 0.02; conics with |B| > 0.999 sqrt(AC), where the
// FP32 exponent loses that accuracy, are never dropped).  A dropped pair
// would have failed the alpha test, so every result is unchanged; the cull
// only removes iterations (most of a tile's list misses a given patch).
// NaN anywhere keeps the record.  pcut = ln(alpha_min / o) - 0.05, the
// record's exponent cutoff (see stage_cutoff).
__device__ __forceinline__ bool patch_may_hit(const float4 &q0, float cc, float pcut, float xa, float xb, float ya,
                                              float yb)
{
    const float A = -2.0f * q0.z, B = -q0.w, C = -2.0f * cc;
    const float tau = pcut - 0.01f;
    if (tau >= 0.0f)
        return false;  // o < alpha_min e^-0.06: no pixel can reach alpha_min
    if (!(A > 0.0f) || !(C > 0.0f) || !(B * B <= 0.998f * (A * C)))
        return true;
    const float u = q0.x, v = q0.y;
    const bool lo_x = u < xa, hi_x = u > xb, lo_y = v < ya, hi_y = v > yb;
    if (!(lo_x || hi_x || lo_y || hi_y))
        return true;  // centre inside the patch (or NaN)
    float m = __int_as_float(0x7f800000);
    if (lo_x || hi_x) {
        const float dx = (lo_x ? xa : xb) - u;
        const float dy = fminf(fmaxf(-B * dx / C, ya - v), yb - v);
        m = fmaf(fmaf(C, dy, 2.0f * B * dx), dy, A * dx * dx);
    }
    if (lo_y || hi_y) {
        const float dy = (lo_y ? ya : yb) - v;
        const float dx = fminf(fmaxf(-B * dy / A, xa - u), xb - u);
        m = fminf(m, fmaf(fmaf(A, dx, 2.0f * B * dy), dx, C * dy * dy));
    }
    return !(m > fmaf(-2.0f * tau, 1.002f, 0.02f));
}

// The second float4 of a staged record, {cc, o, z, cutoff}: the tile
// rectangle it carries in HBM is not needed once the lists are built, and
// its slot takes the record's exponent cutoff ln(alpha_min / o) - 0.05
// (ln(alpha_min) - 0.05 - ln o; __logf's error is far inside the 0.05
// margin).  A pair whose exponent is below it has alpha = o e^x <
// alpha_min e^-0.05 and fails the alpha test, so skipping it before e^x
// changes no decision.  Without an alpha test (smooth mode) the cutoff is
// the plain skip_below (-3e38), which skips nothing.
__device__ __forceinline__ float4 stage_cutoff(float4 q1, const gsl::RasterArgs &a)
{
    q1.w = a.alpha_min > 0.0f ? a.skip_below - __logf(q1.y) : a.skip_below;
    return q1;
}

// Whether the exponent ca dx^2 + cb dx dy + cc dy^2 of a record, as the
// walks evaluate it in FP32 (h = ca dx + (cb dy), ky = cc dy, h dx + (ky dy),
// each product and sum rounded once), is <= 0 at every pixel, so that its
// pairs need no positive-exponent test.  The form is negative definite with
// smallest eigenvalue magnitude mu >= det / tr >= det / S (det = ca cc -
// cb^2 / 4, S = |ca| + |cb| + |cc|), and the rounding moves the computed
// value by at most 2.01 u S (dx^2 + dy^2) (u = 2^-24) plus subnormal
// terms far below mu (dx^2 + dy^2): a nonzero offset is at least 2^-26 px.
// det >= 1e-6 S^2 (after det's own rounding, <= 3u S^2) and |ca|, |cc| >
// 1e-12 leave a wide margin.  NaN or infinite coefficients fail the test.
__device__ __forceinline__ bool conic_safe(float ca, float cb, float cc)
{
    const float S = fabsf(ca) + fabsf(cb) + fabsf(cc);
    const float det = ca * cc - 0.25f * cb * cb;
    return ca < -1e-12f && cc < -1e-12f && det >= 1e-6f * (S * S);
}

// ---------------------------------------------------------------------------
// Packed pixel pairs.  In the registration forward and adjoint a thread
// walks two pixels (same column, rows r and r + 4) with one f32x2 operation
// per step: add/sub/mul/fma.rn.f32x2 round each of the two lanes exactly as
// the scalar .rn operation does, and issue once for both.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;  // {lo, hi} = {pixel 0, pixel 1}
__device__ __forceinline__ f32x2 x2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void x2_split(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 bc2(float v) { return x2(v, v); }

// A record's values, each broadcast to both lanes ({v, v} pairs), for the
// packed walks: {u, v}, {ca, cb}, {cc, o} (-o in the adjoint), {z, r}, {g, b}.
// Built from the staged float4s as they are loaded (staging the pairs
// themselves, 80 B a record, measured slower: more shared-memory loads).
struct RecX2 {
    ulonglong2 uv, ab, co, zr, gb;
};

// the two pixels' adjoint walk state: T, -Q and the loss gradient per pixel
struct PixAdj2 {
    f32x2 pxf, pyf, T, nQ, gr, gg, gb, gd;
    f32x2 ga_tf;  // render mode: the alpha cotangent times T_final
    int last0, last1;
};

// g . S of the background behind every Gaussian of a pixel (the colour
// behind starts at T_final bg): the adjoint walk's first Q
__device__ __forceinline__ float q_background(float gr, float gg, float gb, const float bg[3], float Tf)
{
    return (gr * bg[0] + gg * bg[1] + gb * bg[2]) * Tf;
}

// the contract exponential (exp_ct_nonpos) of both lanes of x
__device__ __forceinline__ void exp_ct_nonpos_x2(float x0, float x1, float &e0, float &e1)
{
    const f32x2 xc = x2(fmaxf(x0, -80.0f), fmaxf(x1, -80.0f));
    const f32x2 magic = bc2(12582912.0f);
    const f32x2 t = fma2(xc, bc2(1.4426950408889634f), magic);
    const f32x2 kf = sub2(t, magic);
    f32x2 r = fma2(kf, bc2(-0.693145751953125f), xc);
    r = fma2(kf, bc2(-1.428606820309417e-06f), r);
    f32x2 p = fma2(bc2(1.3888888888888889e-03f), r, bc2(8.3333333333333333e-03f));
    p = fma2(p, r, bc2(4.1666666666666667e-02f));
    p = fma2(p, r, bc2(1.6666666666666667e-01f));
    p = fma2(p, r, bc2(0.5f));
    p = fma2(p, r, bc2(1.0f));
    p = fma2(p, r, bc2(1.0f));
    float pl, ph, tl, th;
    x2_split(p, pl, ph);
    x2_split(t, tl, th);
    e0 = __int_as_float(__float_as_int(pl) + (int)((uint32_t)__float_as_int(tl) << 23));
    e1 = __int_as_float(__float_as_int(ph) + (int)((uint32_t)__float_as_int(th) << 23));
}

// exponent of a staged record (u, v, ca, cb, cc) at both pixel samples, the
// contract's FP32 sequence per lane: dx = u - px, dy = v - py, h = ca dx +
// (cb dy), ky = cc dy, power = h dx + (ky dy); h and ky are the gradient's
// intermediates
__device__ __forceinline__ f32x2 exponent_x2(const RecX2 &R, f32x2 pxf, f32x2 pyf, f32x2 &dx, f32x2 &h, f32x2 &ky)
{
    dx = sub2(R.uv.x, pxf);
    const f32x2 dy = sub2(R.uv.y, pyf);
    h = fma2(R.ab.x, dx, mul2(R.ab.y, dy));
    ky = mul2(R.co.x, dy);
    return fma2(h, dx, mul2(ky, dy));
}

// forward variants (registration mode): exposure compensation, and the
// count of pairs that pass the alpha test (statistics runs only: the counter
// costs the common variant a register)
constexpr int kFwdExposure = 1, kFwdCount = 2;

// ---------------------------------------------------------------------------
// Forward, two pixels per thread: 128 threads per 16x16 tile, warp w on the
// 8x8 quadrant (w & 1, w >> 1), lane -> column lane & 7, rows lane >> 3 and
// + 4 (the adjoint's layout), both pixels of a thread walked with packed
// operations.  A pixel's early exits and its stop are masks: a pair that
// fails the alpha test, or that would take T below t_min (the pixel is then
// done), enters the sums with weight 0 and leaves T and `last` as they are,
// so every output is the one-pixel walk's.  Records are staged 256 at a
// time (two per thread) with the exponent cutoff in the tile rectangle's
// slot (stage_cutoff); only the warp cull uses it: a pair below it fails the
// alpha test.
// ---------------------------------------------------------------------------
constexpr int kFwdThreads = 128, kFwdBatch = 256;

// Adjoint layout: kBwdPPT pixels per thread, each warp on a kBwdPatchW x 8
// patch of its tile (lane -> column lane % kBwdPatchW, rows lane /
// kBwdPatchW + k * kBwdRowStep for k < kBwdPPT).
constexpr int kBwdPPT = 2;
constexpr int kBwd2Threads = kTilePix / kBwdPPT;
constexpr int kBwd2Warps = kBwd2Threads / 32;
constexpr int kBwdPatchW = kBwdPPT == 2 ? 8 : 16;
constexpr int kBwdRowStep = 32 / kBwdPatchW;
constexpr int kBwd2Chunk = 64;
// a row of per-record warp sums in shared memory: one float more than the
// chunk, so that the lanes storing one record's sums of different values
// (rows k * warps + warp, 65 floats apart) hit different banks
constexpr int kBwdSlotRow = kBwd2Chunk + 1;
constexpr int kBwd2MinBlocks = kBwdPPT == 2 ? 8 : 12;
static_assert(kBwdPPT * kBwdRowStep == 8 && kTile % kBwdPatchW == 0, "warp patches of 8 rows tile the 16x16 tile");

// the adjoint half of the fused registration tile (defined with the adjoint)
__device__ __forceinline__ void fused_adjoint(const gsl::RasterArgs &a, uint32_t t, const VpDesc &d, uint2 rg,
                                              float4 *s0, float4 *s1, float4 *s2, const uint32_t *s_v,
                                              uint8_t *s_selw, float xa, float ya, PixAdj2 &P2, int maxl,
                                              int wmaxl, const float *cc, bool fgen);

template <bool REG, int X, bool FUSED = false>
__device__ __forceinline__ void fwd_tile(const gsl::RasterArgs &a, const uint32_t t)
{
    static_assert(REG || !FUSED, "only the registration forward is fused with the adjoint");
    __shared__ float4 s0[kFwdBatch], s1[kFwdBatch], s2[kFwdBatch];
    __shared__ uint32_t s_v[FUSED ? kFwdBatch : 1];  // fused: the staged records' indices
    __shared__ uint8_t s_sel[4][kFwdBatch];
    __shared__ float s_red[4], s_ea[4], s_eb[4];
    __shared__ int s_pairs[4], s_contrib[4];
    const uint32_t vp = a.tile_vp[t];
    const uint2 rg = a.ranges[t];
    uint32_t v0[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
        v0[r] = rg.x + threadIdx.x + r * kFwdThreads < rg.y ? a.vals[rg.x + threadIdx.x + r * kFwdThreads] : 0u;
    const VpDesc &d = a.vps[vp];
    auto stage = [&](int slot, uint32_t v) {
        const float4 *R = a.rec + 3 * (size_t)v;
        s0[slot] = R[0];
        const float4 q1 = R[1];
        s1[slot] = stage_cutoff(q1, a);
        float4 q2 = R[2];
        if (FUSED) {
            // the adjoint's -o in the slot of the tile rows, which compositing
            // does not read
            q2.w = -q1.y;
            s_v[slot] = v;
        }
        s2[slot] = q2;
    };
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if (rg.x + threadIdx.x + r * kFwdThreads < rg.y)
            stage(threadIdx.x + r * kFwdThreads, v0[r]);
    const uint32_t lt = t - d.tile_base;
    const int tx = (int)(lt % (uint32_t)d.TX), ty = (int)(lt / (uint32_t)d.TX);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = tx * kTile + (warp & 1) * 8, wy = ty * kTile + (warp >> 1) * 8;
    const int px = wx + (lane & 7), py0 = wy + (lane >> 3), py1 = py0 + 4;
    const bool in0 = px < d.W && py0 < d.H, in1 = px < d.W && py1 < d.H;
    const f32x2 pxf = bc2((float)px + 0.5f), pyf = x2((float)py0 + 0.5f, (float)py1 + 0.5f);
    const float xa = (float)wx + 0.5f, ya = (float)wy + 0.5f;
    const bool cull = a.alpha_min > 0.0f;
    // fused: the keyframe's camera-frame pivot as floats, read early
    float pivot = 0.0f;
    if (FUSED && threadIdx.x < 3 && a.c_cam)
        pivot = (float)a.c_cam[3 * vp + threadIdx.x];
    f32x2 T = bc2(1.0f), C0 = bc2(0.0f), C1 = bc2(0.0f), C2 = bc2(0.0f), D = bc2(0.0f);
    int last0 = 0, last1 = 0, nc = 0;
    bool done0 = !in0, done1 = !in1;
    // whether the batch needs the general walk: it holds a record whose
    // opacity exceeds alpha_max (only those can reach the clamp: x = o e with
    // e <= 1 for every exponent <= 0) or whose exponent could round above 0
    bool gen = false;
    for (uint32_t b = rg.x; b < rg.y; b += kFwdBatch) {
        if (b != rg.x) {
            if (__syncthreads_count(done0 && done1) == kFwdThreads)
                break;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t idx = b + threadIdx.x + r * kFwdThreads;
                if (idx < rg.y)
                    stage(threadIdx.x + r * kFwdThreads, a.vals[idx]);
            }
        }
        {
            bool hot = false;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int sl = threadIdx.x + r * kFwdThreads;
                if (b + sl < rg.y) {
                    const float4 t0 = s0[sl], t1 = s1[sl];
                    hot |= t1.y > a.alpha_max || !conic_safe(t0.z, t0.w, t1.x);
                }
            }
            gen = __syncthreads_or(hot) != 0;
        }
        const int cnt = (int)min((uint32_t)kFwdBatch, rg.y - b);
        int nsel = 0;
        if (!__all_sync(0xffffffffu, done0 && done1)) {
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                const int j = j0 + lane;
                bool keep = false;
                if (j < cnt) {
                    const float4 t1 = s1[j];
                    keep = !cull || patch_may_hit(s0[j], t1.x, t1.w, xa, xa + 7.0f, ya, ya + 7.0f);
                }
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep)
                    s_sel[warp][nsel + __popc(m & lanemask_lt())] = (uint8_t)j;
                nsel += __popc(m);
            }
            __syncwarp();
        }
        // The walk is warp-uniform: every lane iterates until all of the
        // warp's pixels are done (a done pixel's pairs are masked), so that
        // the votes below see all 32 lanes.
        if (!__all_sync(0xffffffffu, done0 && done1)) {
            const int base = (int)(b - rg.x) + 1;
            // two copies of the walk: the general one, and for a batch that
            // can reach neither the clamp nor a positive exponent one without
            // those tests
            auto walk = [&](auto gen_tag) {
            constexpr bool GEN = decltype(gen_tag)::value;
            for (int k = 0; k < nsel; ++k) {
                const int j = s_sel[warp][k];
                const float4 q0 = s0[j], q1 = s1[j], q2 = s2[j];
                RecX2 R;
                R.uv = make_ulonglong2(bc2(q0.x), bc2(q0.y));
                R.ab = make_ulonglong2(bc2(q0.z), bc2(q0.w));
                R.co = make_ulonglong2(bc2(q1.x), bc2(q1.y));
                R.zr = make_ulonglong2(bc2(q1.z), bc2(q2.x));
                R.gb = make_ulonglong2(bc2(q2.y), bc2(q2.z));
                f32x2 dx, h, ky;
                float p0, p1, e0, e1;
                x2_split(exponent_x2(R, pxf, pyf, dx, h, ky), p0, p1);
                exp_ct_nonpos_x2(p0, p1, e0, e1);
                float x0, x1;
                x2_split(mul2(R.co.y, x2(e0, e1)), x0, x1);
                const float al0 = GEN ? fminf(x0, a.alpha_max) : x0, al1 = GEN ? fminf(x1, a.alpha_max) : x1;
                const bool ok0 = !done0 && (!GEN || !(p0 > 0.0f)) && !(al0 < a.alpha_min);
                const bool ok1 = !done1 && (!GEN || !(p1 > 0.0f)) && !(al1 < a.alpha_min);
                const f32x2 al = x2(ok0 ? al0 : 0.0f, ok1 ? al1 : 0.0f);
                const f32x2 tn = mul2(T, sub2(bc2(1.0f), al));  // T itself where al = 0
                float tn0, tn1;
                x2_split(tn, tn0, tn1);
                // (a pair that fails leaves tn = T >= t_min: no ok test needed)
                const bool st0 = tn0 < a.t_min, st1 = tn1 < a.t_min;
                if (!__any_sync(0xffffffffu, st0 || st1)) {
                    // no pixel of the warp stops here (the common case)
                    const f32x2 w = mul2(al, T);
                    C0 = fma2(R.zr.y, w, C0);
                    C1 = fma2(R.gb.x, w, C1);
                    C2 = fma2(R.gb.y, w, C2);
                    D = fma2(R.zr.x, w, D);
                    T = tn;
                    last0 = ok0 ? base + j : last0;
                    last1 = ok1 ? base + j : last1;
                    if (X & kFwdCount)
                        nc += (int)ok0 + (int)ok1;
                    continue;
                }
                // a stopping pixel is done: its pair adds nothing, T stays
                const bool c0 = ok0 && !st0, c1 = ok1 && !st1;
                done0 |= st0;
                done1 |= st1;
                const f32x2 w = mul2(x2(c0 ? al0 : 0.0f, c1 ? al1 : 0.0f), T);
                C0 = fma2(R.zr.y, w, C0);
                C1 = fma2(R.gb.x, w, C1);
                C2 = fma2(R.gb.y, w, C2);
                D = fma2(R.zr.x, w, D);
                float T0, T1;
                x2_split(T, T0, T1);
                T = x2(c0 ? tn0 : T0, c1 ? tn1 : T1);
                last0 = c0 ? base + j : last0;
                last1 = c1 ? base + j : last1;
                if (X & kFwdCount)
                    nc += (int)c0 + (int)c1;
                if (__all_sync(0xffffffffu, done0 && done1))
                    break;
            }
            };
            if (gen)
                walk(std::true_type{});
            else
                walk(std::false_type{});
        }
    }
    float Tk[2], C0k[2], C1k[2], C2k[2], Dk[2];
    x2_split(T, Tk[0], Tk[1]);
    x2_split(C0, C0k[0], C0k[1]);
    x2_split(C1, C1k[0], C1k[1]);
    x2_split(C2, C2k[0], C2k[1]);
    x2_split(D, Dk[0], Dk[1]);
    const int lastk[2] = {last0, last1};
    const bool ink[2] = {in0, in1};
    const int pyk[2] = {py0, py1};
    const int64_t HW = (int64_t)d.W * d.H;
    if (!REG) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!ink[k])
                continue;
            const int64_t off = (int64_t)pyk[k] * d.W + px;
            const int64_t pix = d.pix_base + off;
            if (a.out_rgb) {
                float *rgb = a.out_rgb + 3 * d.pix_base;
                rgb[off] = fmaf(Tk[k], a.bg[0], C0k[k]);
                rgb[HW + off] = fmaf(Tk[k], a.bg[1], C1k[k]);
                rgb[2 * HW + off] = fmaf(Tk[k], a.bg[2], C2k[k]);
            }
            if (a.out_depth)
                a.out_depth[pix] = Dk[k];
            if (a.out_alpha)
                a.out_alpha[pix] = 1.0f - Tk[k];
            if (a.t_final)
                a.t_final[pix] = Tk[k];
            if (a.last)
                a.last[pix] = lastk[k];
        }
        return;
    }
    // registration: fused L1 colour + L1 depth loss and its sign code, per pixel
    constexpr bool EXPO = (X & kFwdExposure) != 0;
    const bool expo = EXPO && d.exposure;
    const float gain = expo ? a.expo32[2 * vp] : 1.0f;
    const float off_b = expo ? a.expo32[2 * vp + 1] : 0.0f;
    float lsum = 0.0f, ga = 0.0f, gb = 0.0f;
    // fused: the loss gradient's signs per pixel (the sign code's values)
    float sgk[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!ink[k])
            continue;
        const int64_t off = (int64_t)pyk[k] * d.W + px;
        const int64_t pix = d.pix_base + off;
        const float r0 = fmaf(Tk[k], a.bg[0], C0k[k]), r1 = fmaf(Tk[k], a.bg[1], C1k[k]),
                    r2 = fmaf(Tk[k], a.bg[2], C2k[k]);
        float o0 = r0, o1 = r1, o2 = r2;
        if (expo) {
            // exposure-compensated colour e^a I^ + b (Supp. B)
            o0 = fmaf(gain, r0, off_b);
            o1 = fmaf(gain, r1, off_b);
            o2 = fmaf(gain, r2, off_b);
        }
        const float e0 = o0 - d.t_rgb[off], e1 = o1 - d.t_rgb[HW + off], e2 = o2 - d.t_rgb[2 * HW + off];
        const float ed = Dk[k] - d.t_depth[off];
        const float inv3 = d.inv3hw, inv1 = d.invhw;
        lsum += (fabsf(e0) + fabsf(e1) + fabsf(e2)) * inv3 + fabsf(ed) * inv1;
        auto sg = [](float e) -> uint32_t { return e > 0.0f ? 1u : (e < 0.0f ? 2u : 0u); };
        if (FUSED) {
            auto sf = [](float e) -> float { return e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f); };
            sgk[k][0] = sf(e0);
            sgk[k][1] = sf(e1);
            sgk[k][2] = sf(e2);
            sgk[k][3] = sf(ed);
        } else {
            a.code[pix] = (uint8_t)(sg(e0) | (sg(e1) << 2) | (sg(e2) << 4) | (sg(ed) << 6));
        }
        if (expo) {
            // dL/da = sum_c dL/dI'_c e^a I^_c, dL/db = sum_c dL/dI'_c
            auto sf = [](float e) -> float { return e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f); };
            const float s0 = sf(e0), s1 = sf(e1), s2 = sf(e2);
            ga += inv3 * gain * (s0 * r0 + s1 * r1 + s2 * r2);
            gb += inv3 * (s0 + s1 + s2);
        }
        if (FUSED)
            continue;
        a.t_final[pix] = Tk[k];
        a.last[pix] = lastk[k];
        if (d.loss_kind == 1) {
            // tracking loss: depth error (+inf without input depth) and colour L1 for its masks
            a.trk_err[pix] = d.t_depth[off] > 0.0f ? fabsf(ed) : __uint_as_float(0x7f800000u);
            a.trk_col[pix] = fabsf(e0) + fabsf(e1) + fabsf(e2);
        }
    }
    lsum = warp_sum(lsum);
    const int wl = warp_sum(last0 + last1);
    if (expo) {
        ga = warp_sum(ga);
        gb = warp_sum(gb);
    }
    int wc = 0;
    if (X & kFwdCount)
        wc = warp_sum(nc);
    // fused: the warps' last contributors and the pivot behind the same barrier
    __shared__ int s_maxl[FUSED ? 4 : 1];
    __shared__ float s_cc[3];
    int wmaxl = 0;
    if (FUSED) {
        wmaxl = max(last0, last1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            wmaxl = max(wmaxl, __shfl_xor_sync(0xffffffffu, wmaxl, o));
        if (lane == 0)
            s_maxl[warp] = wmaxl;
        if (threadIdx.x < 3)
            s_cc[threadIdx.x] = pivot;
        // the adjoint's warp-sum slots, zeroed behind the same barrier
        extern __shared__ float4 s_dyn[];
        static_assert(6 * kBwd2Warps * kBwdSlotRow % 4 == 0, "slots zeroed as float4");
        for (int k = threadIdx.x; k < 6 * kBwd2Warps * kBwdSlotRow / 4; k += kBwd2Threads)
            s_dyn[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (lane == 0) {
        s_red[warp] = lsum;
        s_pairs[warp] = wl;
        s_contrib[warp] = wc;
        s_ea[warp] = ga;
        s_eb[warp] = gb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sl = 0.0f, sa = 0.0f, sb = 0.0f;
        unsigned long long np = 0, ncs = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            sl += s_red[w];
            np += (unsigned long long)s_pairs[w];
            ncs += (unsigned long long)s_contrib[w];
            sa += s_ea[w];
            sb += s_eb[w];
        }
        a.tile_loss[t] = sl;
        if (expo) {
            a.tile_expo[2 * (size_t)t] = sa;
            a.tile_expo[2 * (size_t)t + 1] = sb;
        }
        if (a.tile_pairs) {
            atomicAdd(&a.tile_pairs[t], np);
            if (X & kFwdCount)
                atomicAdd(&a.tile_pairs[a.n_tiles + t], ncs);
        }
    }
    if constexpr (FUSED) {
        // the adjoint's state from this thread's own two pixels, as
        // pix_adj_init derives it from the stored T_final, last and code
        int maxl = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            maxl = max(maxl, s_maxl[w]);
        const float cc[3] = {s_cc[0], s_cc[1], s_cc[2]};
        const float inv3 = expo ? d.inv3hw * gain : d.inv3hw, inv1 = d.invhw;
        float g[2][4], q[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            g[k][0] = sgk[k][0] * inv3;
            g[k][1] = sgk[k][1] * inv3;
            g[k][2] = sgk[k][2] * inv3;
            g[k][3] = sgk[k][3] * inv1;
            q[k] = q_background(g[k][0], g[k][1], g[k][2], a.bg, Tk[k]);
        }
        PixAdj2 P2;
        P2.pxf = pxf;
        P2.pyf = pyf;
        P2.T = T;
        P2.nQ = x2(-q[0], -q[1]);
        P2.gr = x2(g[0][0], g[1][0]);
        P2.gg = x2(g[0][1], g[1][1]);
        P2.gb = x2(g[0][2], g[1][2]);
        P2.gd = x2(g[0][3], g[1][3]);
        P2.last0 = last0;
        P2.last1 = last1;
        fused_adjoint(a, t, d, rg, s0, s1, s2, s_v, s_sel[warp], xa, ya, P2, maxl, wmaxl, cc, gen);
    }
}

// One CTA per tile (the grid covers every tile; tile_order, when given,
// maps CTA -> tile).
template <bool REG, int X>
__global__ void __launch_bounds__(kFwdThreads, 8) k_forward(const gsl::RasterArgs a)
{
    fwd_tile<REG, X>(a, a.tile_order ? a.tile_order[blockIdx.x] : blockIdx.x);
}


// Persistent form: a grid of a few CTAs per SM, each CTA pulling the next
// tile (in tile_order, or natural order) from the work queue a.queue (one
// atomic per tile, zeroed before the launch) until every tile is taken.
// Tiles of every keyframe problem of a batch share one queue.  Thread 0
// claims the next queue position as a tile starts and publishes it only
// when the tile ends, so the atomic's round trip overlaps the tile's work;
// the barrier before publishing also ends every thread's use of the
// previous tile's shared memory (the tile's own barriers order the read of
// s_next before its next write).
template <typename Tile>
__device__ __forceinline__ void run_queue(const gsl::RasterArgs &a, Tile &&tile)
{
    __shared__ uint32_t s_next;
    uint32_t claimed = threadIdx.x == 0 ? atomicAdd(a.queue, 1u) : 0u;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_next = claimed;
        __syncthreads();
        const uint32_t i = s_next;
        if (i >= a.n_tiles)
            return;
        if (threadIdx.x == 0)
            claimed = atomicAdd(a.queue, 1u);
        tile(a.tile_order ? a.tile_order[i] : i);
    }
}

template <int X>
__global__ void __launch_bounds__(kFwdThreads, 8) k_forward_q(const gsl::RasterArgs a)
{
    run_queue(a, [&](uint32_t t) { fwd_tile<true, X>(a, t); });
}

// Warp sums of N (8 or 16) values per lane.  Each exchange over a lane bit
// halves the values a lane carries (it keeps the half its partner sends
// away), so log2(N) halving steps plus log2(32/N) plain butterflies need
// N - 1 + log2(32/N) shuffles instead of 5 N.  On return lane l holds the
// full sum of value index l / (32 / N).  Values NV..N-1 are zero padding:
// in the first exchange the lanes that keep such an index would add two
// zeros, so that step adds v[i] of both partners instead (no selects); the
// lanes keeping index i + h >= NV then carry a sum that only ever meets
// other padding indices, and their results are not used.
template <int N, int NV = N>
__device__ __forceinline__ float warp_sum_transpose(float (&v)[N], int lane)
{
    int bit = 16;
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2) {
        const bool up = (lane & bit) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            if (h == N / 2 && i + h >= NV) {
                v[i] = v[i] + __shfl_xor_sync(0xffffffffu, v[i], bit);
                continue;
            }
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
        bit >>= 1;
    }
    float s = v[0];
#pragma unroll
    for (int o = 32 / N / 2; o >= 1; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}


// Six running FP32 sums of one thread with Kahan compensation (the lost
// low-order part is carried in c; the true sum is s - c), kept in shared
// memory as [2 k + (0: s, 1: c)][thread]: they are touched once per record
// at the end of a chunk, and in registers they would stay live across the
// whole pixel walk.  STRIDE: the columns of the block's [12][STRIDE] array.
template <int STRIDE>
struct Twist6T {
    float *base;  // the thread's column
    __device__ __forceinline__ float &s(int k) const { return base[(2 * k) * STRIDE]; }
    __device__ __forceinline__ float &c(int k) const { return base[(2 * k + 1) * STRIDE]; }
    __device__ __forceinline__ void zero() const
    {
#pragma unroll
        for (int k = 0; k < 6; ++k)
            s(k) = c(k) = 0.0f;
    }
    __device__ __forceinline__ void add(int k, float v) const
    {
        const float sk = s(k), y = v - c(k);
        const float t = sk + y;
        c(k) = (t - sk) - y;
        s(k) = t;
    }
};
using Twist6 = Twist6T<kBwd2Threads>;

// The tile's twist: each of the first nw warps (the ones whose threads
// accumulated anything) reduces its lanes' compensated sums with TwoSum
// butterflies, and threads 0..5 join those warps' (hi, lo) pairs the same
// way in a fixed order and store them.  Leaving out the warps that hold
// only zeros changes no bit: a TwoSum of (0, 0) leaves a pair as it is.
// (No FP64 here: the FP64 pipe is a small fraction of the FP32 one, and
// FP64 work in every warp kept it busy and lengthened every CTA's tail.)
template <int WARPS, typename Tw>
__device__ __forceinline__ void store_tile_twist(const Tw &tw, int nw, float (*s_tw)[6][2], float2 *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < nw) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float hi = tw.s(k), lo = -tw.c(k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float bh = __shfl_xor_sync(0xffffffffu, hi, o), bl = __shfl_xor_sync(0xffffffffu, lo, o);
                two_sum_add(hi, lo, bh, bl);
            }
            if (lane == 0) {
                s_tw[warp][k][0] = hi;
                s_tw[warp][k][1] = lo;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float hi = 0.0f, lo = 0.0f;
        if (nw > 0) {
            hi = s_tw[0][threadIdx.x][0];
            lo = s_tw[0][threadIdx.x][1];
        }
#pragma unroll
        for (int w = 1; w < WARPS; ++w)
            if (w < nw)
                two_sum_add(hi, lo, s_tw[w][threadIdx.x][0], s_tw[w][threadIdx.x][1]);
        out[threadIdx.x] = make_float2(hi, lo);
    }
}

// d(screen params) of one (tile, Gaussian) -> camera-frame twist (w, v)
// about cc (camera frame), added to tw.  G = {dL/du, dL/dv,
// 2 dL/dSigma2D_00, 2 dL/dSigma2D_01, 2 dL/dSigma2D_11, dL/dz, ...} (the 2D
// covariance is the dilated one; dilation is constant).
template <typename Tw>
__device__ __forceinline__ void chain_twist(const float *G, const float4 &q1, const float4 &x0, const float4 &x1,
                                            float fx, float fy, const float *cc, const Tw &tw)
{
    using S = float;
    const S mx = x0.x, my = x0.y, mz = q1.z;
    const S S00 = x0.z, S01 = x0.w, S02 = x1.x, S11 = x1.y, S12 = x1.z, S22 = x1.w;
    // dL/dSigma2D = [[gp, gq], [gq, gs]]
    const S gp = S(0.5) * S(G[2]), gq = S(0.5) * S(G[3]), gs = S(0.5) * S(G[4]);
    const S iz = S(1) / mz, iz2 = iz * iz;
    const S j00 = fx * iz, j11 = fy * iz, j02 = -fx * mx * iz2, j12 = -fy * my * iz2;
    // G2 J (2x3)
    const S r00 = gp * j00, r01 = gq * j11, r02 = gp * j02 + gq * j12;
    const S r10 = gq * j00, r11 = gs * j11, r12 = gq * j02 + gs * j12;
    // dL/dSigma_cam = J^T G2 J
    const S c00 = j00 * r00, c01 = j00 * r01, c02 = j00 * r02;
    const S c11 = j11 * r11, c12 = j11 * r12, c22 = j02 * r02 + j12 * r12;
    // dL/dJ = 2 G2 J Sigma_cam (entries used)
    const S dJ00 = S(2) * (r00 * S00 + r01 * S01 + r02 * S02);
    const S dJ02 = S(2) * (r00 * S02 + r01 * S12 + r02 * S22);
    const S dJ11 = S(2) * (r10 * S01 + r11 * S11 + r12 * S12);
    const S dJ12 = S(2) * (r10 * S02 + r11 * S12 + r12 * S22);
    const S du = G[0], dv = G[1], dz = G[5];
    const S gx = du * fx * iz - dJ02 * fx * iz2;
    const S gy = dv * fy * iz - dJ12 * fy * iz2;
    const S gz = -du * fx * mx * iz2 - dv * fy * my * iz2 + dz - dJ00 * fx * iz2 - dJ11 * fy * iz2 +
                 S(2) * iz2 * iz * (dJ02 * fx * mx + dJ12 * fy * my);
    // 2 vee(Gc S - S Gc)
    const S k21 = (c02 * S01 + c12 * S11 + c22 * S12) - (S02 * c01 + S12 * c11 + S22 * c12);
    const S k02 = (c00 * S02 + c01 * S12 + c02 * S22) - (S00 * c02 + S01 * c12 + S02 * c22);
    const S k10 = (c01 * S00 + c11 * S01 + c12 * S02) - (S01 * c00 + S11 * c01 + S12 * c02);
    const S rx = mx - cc[0], ry = my - cc[1], rz = mz - cc[2];
    tw.add(0, ry * gz - rz * gy + S(2) * k21);
    tw.add(1, rz * gx - rx * gz + S(2) * k02);
    tw.add(2, rx * gy - ry * gx + S(2) * k10);
    tw.add(3, gx);
    tw.add(4, gy);
    tw.add(5, gz);
}


// ---------------------------------------------------------------------------
// Adjoint with two pixels per thread: 128 threads per 16x16 tile, warp w
// owns the 8x8 quadrant (w & 1, w >> 1) (lane -> column lane & 7, rows
// lane >> 3 and +4): the squarest patch of 64 pixels, which the fewest
// records reach.
// Each staged record is evaluated for both pixels in one chain of packed
// operations (pix_adj_x2) and their gradients are added before the warp
// reduction, which therefore covers 64 pixels.
// ---------------------------------------------------------------------------
// Per-pixel state of the back-to-front walk (as read from the forward's
// outputs; the walk carries it packed, PixAdj2).  g = (gr, gg, gb, gd) is the
// loss gradient w.r.t. the pixel's colour and depth, constant along the
// walk, so the colour behind the current Gaussian enters dL/dalpha only
// through Q = g . S, S = sum over the Gaussians behind (and the background)
// of colour x alpha x transmittance: dL/dalpha_i = T_i (g . c_i) -
// Q / (1 - alpha_i), then Q += (g . c_i) alpha_i T_i.  (One scalar instead
// of the four normalised colours behind, and seven operations per pair
// instead of seventeen.)
struct PixAdj {
    float pxf, pyf, T, Tf, Q, gr, gg, gb, gd, ga_tf;
    int last;
};

template <bool REG>
__device__ __forceinline__ void pix_adj_init(PixAdj &P, const VpDesc &d, const gsl::RasterArgs &a, int px, int py,
                                             const float bg[3], float gain)
{
    P.pxf = (float)px + 0.5f;
    P.pyf = (float)py + 0.5f;
    P.Tf = 1.0f;
    P.gr = P.gg = P.gb = P.gd = 0.0f;
    float ga = 0.0f;
    P.last = 0;
    if (px < d.W && py < d.H) {
        const int64_t HW = (int64_t)d.W * d.H;
        const int64_t off = (int64_t)py * d.W + px;
        const int64_t pix = d.pix_base + off;
        P.Tf = a.t_final[pix];
        P.last = a.last[pix];
        if (REG) {
            const uint32_t c = a.code[pix];
            auto dec = [](uint32_t v) -> float { return v == 1u ? 1.0f : (v == 2u ? -1.0f : 0.0f); };
            // registration: means over 3HW and HW; tracking: mask weight x lambda_c, x (1 - lambda_c)
            float inv3 = d.inv3hw, inv1 = d.invhw;
            if (d.loss_kind == 1) {
                const float w = a.trk_w[pix];
                inv3 = w * d.lambda_c;
                inv1 = w * (1.0f - d.lambda_c);
            }
            if (d.exposure)
                inv3 *= gain;  // the raw render's colour cotangent is e^a times the compensated one
            P.gr = dec(c & 3u) * inv3;
            P.gg = dec((c >> 2) & 3u) * inv3;
            P.gb = dec((c >> 4) & 3u) * inv3;
            P.gd = dec((c >> 6) & 3u) * inv1;
        } else {
            if (a.d_rgb) {
                const float *dr = a.d_rgb + 3 * d.pix_base;
                P.gr = dr[off];
                P.gg = dr[HW + off];
                P.gb = dr[2 * HW + off];
            }
            if (a.d_depth)
                P.gd = a.d_depth[pix];
            if (a.d_alpha)
                ga = a.d_alpha[pix];
        }
    }
    P.T = P.Tf;
    P.Q = q_background(P.gr, P.gg, P.gb, bg, P.Tf);  // the background behind everything (depth 0)
    P.ga_tf = ga * P.Tf;
}


// Both pixels of one (thread, Gaussian) pair of the adjoint: the
// contract's decisions (the alpha test decides alone: the exponent cutoff
// only ever skips pairs that fail it), the transmittance recovery, the
// colour-behind update and the negated screen-space gradient, summed over
// the two pixels in a one-pixel walk's order (pixel 0's term first), into
// ng.  The pair's early exits are masks: a pair that fails a test enters
// every sum with weight 0 (so every value is the one-pixel walk's, up to the
// sign of zero sums).  ALPHA: the alpha image has a cotangent (render mode).
// FULL: also the opacity and colour gradients (ng[6..9]).  Returns whether
// either pixel contributed.
template <bool ALPHA, bool FULL, bool GEN = true>
__device__ __forceinline__ bool pix_adj_x2(PixAdj2 &P, int jj, const RecX2 &R, float amax, float namax,
                                           float namin, float (&ng)[FULL ? 10 : 6])
{
    f32x2 dx, h, ky;
    const f32x2 power = exponent_x2(R, P.pxf, P.pyf, dx, h, ky);
    float p0, p1, e0, e1;
    x2_split(power, p0, p1);
    exp_ct_nonpos_x2(p0, p1, e0, e1);
    // -x = (-o) e; clamped: x > alpha_max; -alpha; the alpha test
    float nx0, nx1;
    x2_split(mul2(R.co.y, x2(e0, e1)), nx0, nx1);
    const bool cl0 = GEN && nx0 < namax, cl1 = GEN && nx1 < namax;
    const float na0 = GEN ? fmaxf(nx0, namax) : nx0, na1 = GEN ? fmaxf(nx1, namax) : nx1;
    const bool live0 = jj < P.last0 && (!GEN || !(p0 > 0.0f)) && !(na0 > namin);
    const bool live1 = jj < P.last1 && (!GEN || !(p1 > 0.0f)) && !(na1 > namin);
    const f32x2 nal = x2(live0 ? na0 : 0.0f, live1 ? na1 : 0.0f);
    const f32x2 nag = GEN ? x2(live0 && !cl0 ? na0 : 0.0f, live1 && !cl1 ? na1 : 0.0f) : nal;
    // 1 - alpha, its reciprocal, T_i = T / (1 - alpha)
    float om0, om1;
    x2_split(add2(bc2(1.0f), nal), om0, om1);
    const f32x2 rom = x2(__fdividef(1.0f, om0), __fdividef(1.0f, om1));
    const f32x2 Ti = mul2(P.T, rom);
    const f32x2 gcc = fma2(P.gd, R.zr.x, fma2(P.gb, R.gb.y, fma2(P.gg, R.gb.x, mul2(P.gr, R.zr.y))));
    f32x2 dal = fma2(Ti, gcc, mul2(P.nQ, rom));
    if (ALPHA)
        dal = fma2(P.ga_tf, rom, dal);
    const f32x2 nwgt = mul2(nal, Ti);
    P.nQ = fma2(gcc, nwgt, P.nQ);
    const f32x2 ndp = mul2(dal, nag);
    const f32x2 gu = fma2(R.ab.x, dx, h);
    const f32x2 gv = fma2(R.ab.y, dx, add2(ky, ky));
    float a0, a1, b0, b1, u0, u1, v0, v1, d0, d1, w0, w1;
    x2_split(mul2(ndp, gu), a0, a1);
    x2_split(mul2(ndp, gv), b0, b1);
    x2_split(gu, u0, u1);
    x2_split(gv, v0, v1);
    x2_split(P.gd, d0, d1);
    x2_split(nwgt, w0, w1);
    ng[0] = a0 + a1;
    ng[1] = b0 + b1;
    ng[2] = fmaf(a1, u1, a0 * u0);
    ng[3] = fmaf(a1, v1, a0 * v0);
    ng[4] = fmaf(b1, v1, b0 * v0);
    ng[5] = fmaf(d1, w1, d0 * w0);
    if constexpr (FULL) {
        // -(dal e) over the live, unclamped pixels; -(g_c wgt) over the live ones
        const float ne0 = live0 && !cl0 ? -e0 : 0.0f, ne1 = live1 && !cl1 ? -e1 : 0.0f;
        float l0, l1, r0, r1, g0, g1, c0, c1;
        x2_split(dal, l0, l1);
        x2_split(P.gr, r0, r1);
        x2_split(P.gg, g0, g1);
        x2_split(P.gb, c0, c1);
        ng[6] = fmaf(l1, ne1, l0 * ne0);
        ng[7] = fmaf(r1, w1, r0 * w0);
        ng[8] = fmaf(g1, w1, g0 * w0);
        ng[9] = fmaf(c1, w1, c0 * w0);
    }
    P.T = Ti;
    return live0 || live1;
}

static_assert(kBwd2Chunk <= kBwd2Threads && kBwd2Chunk % 32 == 0, "one thread stages one record");

// One tile of the adjoint (all kBwd2Threads threads of the CTA take part).
template <bool REG, bool FULL>
__device__ __forceinline__ void bwd_tile(const gsl::RasterArgs &a, const uint32_t t)
{
    constexpr int NG = FULL ? 10 : 6;
    extern __shared__ float4 s_dyn[];  // declared float4: 16-byte aligned for the float4 zeroing
    float *const s_slots = reinterpret_cast<float *>(s_dyn);  // [NG][warps][kBwdSlotRow]
    __shared__ float4 s0[kBwd2Chunk], s1[kBwd2Chunk], s2[kBwd2Chunk];
    __shared__ float4 s_x0[kBwd2Chunk], s_x1[kBwd2Chunk];  // the records' camera-frame mean and covariance
    // both pixels of a thread are walked with packed operations (the
    // record's values broadcast to both lanes as loaded; o staged negated)
    constexpr bool PK = kBwdPPT == 2;
    static_assert(PK, "the adjoint walks two pixels per thread");
    __shared__ uint8_t s_sel[kBwd2Warps][kBwd2Chunk];  // per warp: chunk positions that may hit its rows
    __shared__ int s_maxl[kBwd2Warps];
    __shared__ float s_tw[kBwd2Warps][6][2];
    const int vp = (int)a.tile_vp[t];
    const VpDesc &d = a.vps[vp];
    const uint32_t lt = t - d.tile_base;
    const int tx = (int)(lt % (uint32_t)d.TX), ty = (int)(lt / (uint32_t)d.TX);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kPatchesX = kTile / kBwdPatchW;
    const int wx = tx * kTile + (warp % kPatchesX) * kBwdPatchW, wy = ty * kTile + (warp / kPatchesX) * 8;
    const int px = wx + lane % kBwdPatchW;
    const int py0 = wy + lane / kBwdPatchW;
    // the warp's pixel samples: a kBwdPatchW x 8 patch
    const float xa = (float)wx + 0.5f, xb = xa + (float)(kBwdPatchW - 1);
    const float ya = (float)wy + 0.5f, yb = ya + 7.0f;
    const bool cull = a.alpha_min > 0.0f;
    const uint2 rg = a.ranges[t];
    // staging of one record of a chunk (thread i, chunk position i)
    auto stage = [&](uint32_t r) {
        const float4 *R = a.rec + 3 * (size_t)r;
        s0[threadIdx.x] = R[0];
        float4 q1 = stage_cutoff(R[1], a);
        if (PK)
            q1.y = -q1.y;
        s1[threadIdx.x] = q1;
        s2[threadIdx.x] = R[2];
        if (a.tile_twist) {
            // the camera-frame mean and covariance, staged with the record
            // (not read after the walk) so that these loads overlap
            s_x0[threadIdx.x] = a.aux[2 * (size_t)r];
            s_x1[threadIdx.x] = a.aux[2 * (size_t)r + 1];
        }
    };
    // The walk's first chunk ends at the tile's last contributor, known only
    // after the barrier below.  It is staged before it on the guess that the
    // list's last entry contributes (checked after the barrier; a wrong guess
    // stages the chunk again), so that its loads overlap the pixel state's.
    const int n_list = (int)(rg.y - rg.x);
    const int lo_guess = max(n_list - kBwd2Chunk, 0);
    const bool guess_row = (int)threadIdx.x < n_list - lo_guess;
    const uint32_t r_guess = guess_row ? a.vals[rg.x + lo_guess + threadIdx.x] : 0u;
    // the keyframe's camera-frame pivot as floats, read with the pixel state
    // so that the two loads overlap, and shared behind the same barrier
    __shared__ float s_cc[3];
    float pivot = 0.0f;
    if (threadIdx.x < 3 && a.c_cam)
        pivot = (float)a.c_cam[3 * vp + threadIdx.x];
    PixAdj P[kBwdPPT];
    const float gain = (REG && d.exposure) ? a.expo32[2 * vp] : 1.0f;
#pragma unroll
    for (int k = 0; k < kBwdPPT; ++k)
        pix_adj_init<REG>(P[k], d, a, px, py0 + k * kBwdRowStep, a.bg, gain);
    PixAdj2 P2;
    if constexpr (PK) {
        P2.pxf = bc2(P[0].pxf);
        P2.pyf = x2(P[0].pyf, P[1].pyf);
        P2.T = x2(P[0].T, P[1].T);
        P2.nQ = x2(-P[0].Q, -P[1].Q);
        P2.gr = x2(P[0].gr, P[1].gr);
        P2.gg = x2(P[0].gg, P[1].gg);
        P2.gb = x2(P[0].gb, P[1].gb);
        P2.gd = x2(P[0].gd, P[1].gd);
        P2.ga_tf = x2(P[0].ga_tf, P[1].ga_tf);
        P2.last0 = P[0].last;
        P2.last1 = P[1].last;
    }
    if (guess_row)
        stage(r_guess);
    int ml = P[0].last;
#pragma unroll
    for (int k = 1; k < kBwdPPT; ++k)
        ml = max(ml, P[k].last);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        ml = max(ml, __shfl_xor_sync(0xffffffffu, ml, o));
    if (lane == 0)
        s_maxl[warp] = ml;
    if (threadIdx.x < 3)
        s_cc[threadIdx.x] = pivot;
    __syncthreads();
    int maxl = 0;
#pragma unroll
    for (int w = 0; w < kBwd2Warps; ++w)
        maxl = max(maxl, s_maxl[w]);
    const float cc[3] = {s_cc[0], s_cc[1], s_cc[2]};
    // one thread per record of a chunk runs chain_twist, so only threads
    // below the largest chunk (min(maxl, chunk)) ever hold twist sums
    __shared__ float s_acc[12][kBwd2Threads];
    const Twist6 tw{&s_acc[0][threadIdx.x]};
    if ((int)threadIdx.x < kBwd2Chunk)
        tw.zero();
    const int twist_warps = (min(maxl, kBwd2Chunk) + 31) / 32;
    // the warp sums' slots start zeroed; the epilogue thread of chunk
    // position i zeroes column i again after reading it, and no other column
    // is ever written
    static_assert(NG * kBwd2Warps * kBwdSlotRow % 4 == 0, "slots zeroed as float4");
    for (int k = threadIdx.x; k < NG * kBwd2Warps * kBwdSlotRow / 4; k += kBwd2Threads)
        s_dyn[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int hi = maxl; hi > 0; hi -= kBwd2Chunk) {
        const int lo = max(hi - kBwd2Chunk, 0), cnt = hi - lo;
        // Thread i stages chunk position i, which only its own epilogue of the
        // previous chunk read, and every warp's walk of that chunk ended at
        // its closing barrier: one barrier per chunk fewer than restaging
        // behind a barrier of its own.  hi == n_list only for a first chunk
        // the guess staged already.
        if (hi != n_list && (int)threadIdx.x < cnt)
            stage(a.vals[rg.x + lo + threadIdx.x]);
        // whether the chunk needs the general walk (a record whose opacity
        // exceeds alpha_max or whose exponent could round above 0; each
        // thread reads back the slot it staged, o staged negated)
        bool hot = false;
        if ((int)threadIdx.x < cnt) {
            const float4 t0 = s0[threadIdx.x], t1 = s1[threadIdx.x];
            hot = t1.y < -a.alpha_max || !conic_safe(t0.z, t0.w, t1.x);
        }
        const bool gen = __syncthreads_or(hot) != 0;
        // this warp's pixels never reach past wl: skip the list tail
        const int wl = min(s_maxl[warp] - lo, cnt);
        int nsel = 0;
        for (int j0 = 0; j0 < wl; j0 += 32) {
            const int j = j0 + lane;
            bool keep = false;
            if (j < wl) {
                const float4 t1 = s1[j];  // one 16-byte load for cc and the cutoff
                keep = !cull || patch_may_hit(s0[j], t1.x, t1.w, xa, xb, ya, yb);
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep)
                s_sel[warp][nsel + __popc(m & lanemask_lt())] = (uint8_t)j;
            nsel += __popc(m);
        }
        __syncwarp();
        auto walk = [&](auto gen_tag) {
        constexpr bool GEN = decltype(gen_tag)::value;
        for (int k = nsel - 1; k >= 0; --k) {
            const int j = s_sel[warp][k];
            float g[NG];
            const float4 q0 = s0[j], q1 = s1[j], q2 = s2[j];
            RecX2 R;
            R.uv = make_ulonglong2(bc2(q0.x), bc2(q0.y));
            R.ab = make_ulonglong2(bc2(q0.z), bc2(q0.w));
            R.co = make_ulonglong2(bc2(q1.x), bc2(q1.y));
            R.zr = make_ulonglong2(bc2(q1.z), bc2(q2.x));
            R.gb = make_ulonglong2(bc2(q2.y), bc2(q2.z));
            const bool contrib =
                pix_adj_x2<!REG, FULL, GEN>(P2, lo + j, R, a.alpha_max, -a.alpha_max, -a.alpha_min, g);
            if (__any_sync(0xffffffffu, contrib)) {
                constexpr int NP = NG <= 8 ? 8 : 16;
                float v[NP];
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    v[k] = k < NG ? g[k] : 0.0f;
                const float sum = warp_sum_transpose<NP, NG>(v, lane);
                constexpr int L = 32 / NP;
                const int k = lane / L;
                if ((lane % L) == 0 && k < NG)
                    s_slots[(k * kBwd2Warps + warp) * kBwdSlotRow + j] = sum;
            }
        }
        };
        if (gen)
            walk(std::true_type{});
        else
            walk(std::false_type{});
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            float G[NG];
            bool any = false;
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                float s = -0.0f;
#pragma unroll
                for (int w = 0; w < kBwd2Warps; ++w) {
                    float &slot = s_slots[(k * kBwd2Warps + w) * kBwdSlotRow + threadIdx.x];
                    s += slot;
                    slot = 0.0f;
                }
                G[k] = -s;  // the packed walk sums the negated gradient
                any |= s != 0.0f;
            }
            if (FULL) {
                float *dst = a.dup_grads + (size_t)(rg.x + lo + threadIdx.x) * 10;
#pragma unroll
                for (int k = 0; k < NG; ++k)
                    dst[k] = G[k];
            }
            if (any && a.tile_twist)
                chain_twist(G, s1[threadIdx.x], s_x0[threadIdx.x], s_x1[threadIdx.x], d.fx, d.fy, cc, tw);
        }
    }
    if (!a.tile_twist)
        return;
    store_tile_twist<kBwd2Warps>(tw, twist_warps, s_tw, a.tile_twist + (size_t)t * 6);
}

template <bool REG, bool FULL>
__global__ void __launch_bounds__(kBwd2Threads, kBwd2MinBlocks) k_backward2(const gsl::RasterArgs a)
{
    bwd_tile<REG, FULL>(a, a.tile_order ? a.tile_order[blockIdx.x] : blockIdx.x);
}

// persistent form of the adjoint (see k_forward_q)
template <bool REG, bool FULL>
__global__ void __launch_bounds__(kBwd2Threads, kBwd2MinBlocks) k_backward2_q(const gsl::RasterArgs a)
{
    run_queue(a, [&](uint32_t t) { bwd_tile<REG, FULL>(a, t); });
}

// The adjoint half of the fused registration tile (k_fwdbwd): the walk of
// bwd_tile's packed registration path on the forward's pixels and staging.
// A list the forward staged whole (n_list <= kFwdBatch) is walked from
// there, chunk position j at list position lo + j; a longer one is
// restaged chunk by chunk into the first kBwd2Chunk slots.  Only the
// records' camera-frame mean and covariance are loaded per chunk.
__device__ __forceinline__ void fused_adjoint(const gsl::RasterArgs &a, uint32_t t, const VpDesc &d, uint2 rg,
                                              float4 *s0, float4 *s1, float4 *s2, const uint32_t *s_v,
                                              uint8_t *s_selw, float xa, float ya, PixAdj2 &P2, int maxl,
                                              int wmaxl, const float *cc, bool fgen)
{
    constexpr int NG = 6;
    extern __shared__ float4 s_dyn[];
    float *const s_slots = reinterpret_cast<float *>(s_dyn);  // [NG][warps][kBwdSlotRow]
    __shared__ float4 s_x0[kBwd2Chunk], s_x1[kBwd2Chunk];
    __shared__ float s_acc[12][kBwd2Chunk];
    __shared__ float s_tw[kBwd2Warps][6][2];
    static_assert(kFwdThreads == kBwd2Threads && kBwd2Chunk <= kFwdBatch, "the fused tile shares the layout");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Twist6T<kBwd2Chunk> tw{&s_acc[0][threadIdx.x % kBwd2Chunk]};  // used by threads < kBwd2Chunk only
    if ((int)threadIdx.x < kBwd2Chunk)
        tw.zero();  // each thread's own column: no barrier needed
    // (the slots were zeroed before the forward's last barrier)
    const int n_list = (int)(rg.y - rg.x);
    const bool whole = n_list <= kFwdBatch;
    const bool cull = a.alpha_min > 0.0f;
    const int twist_warps = (min(maxl, kBwd2Chunk) + 31) / 32;
    for (int hi = maxl; hi > 0; hi -= kBwd2Chunk) {
        const int lo = max(hi - kBwd2Chunk, 0), cnt = hi - lo;
        const int sb = whole ? lo : 0;  // staging slot of chunk position 0
        // thread i stages chunk position i (as in bwd_tile: only its own
        // epilogue of the previous chunk read that slot)
        if ((int)threadIdx.x < cnt) {
            uint32_t r;
            if (whole) {
                r = s_v[lo + threadIdx.x];
            } else {
                r = a.vals[rg.x + lo + threadIdx.x];
                const float4 *R = a.rec + 3 * (size_t)r;
                s0[threadIdx.x] = R[0];
                const float4 q1 = R[1];
                s1[threadIdx.x] = stage_cutoff(q1, a);
                float4 q2 = R[2];
                q2.w = -q1.y;
                s2[threadIdx.x] = q2;
            }
            if (a.tile_twist) {
                s_x0[threadIdx.x] = a.aux[2 * (size_t)r];
                s_x1[threadIdx.x] = a.aux[2 * (size_t)r + 1];
            }
        }
        // The first chunk of a list walked from the forward's staging needs
        // no barrier: the walk reads that staging and the zeroed slots, both
        // ordered by the forward's last barrier, and the means and
        // covariances staged here are read only by the thread that staged
        // them (in the epilogue).  Any later chunk follows an epilogue that
        // re-zeroed slot columns the walk writes, and restaged records are
        // read by every warp.
        // whether the chunk needs the general walk (as in the forward; a
        // list walked from the forward's staging takes the forward's flag)
        bool gen = fgen;
        if (!(whole && hi == maxl)) {
            bool hot = false;
            if (!whole && (int)threadIdx.x < cnt) {
                const float4 t0 = s0[threadIdx.x], t1 = s1[threadIdx.x];
                hot = t1.y > a.alpha_max || !conic_safe(t0.z, t0.w, t1.x);
            }
            const bool any_hot = __syncthreads_or(hot) != 0;
            if (!whole)
                gen = any_hot;
        }
        const int wl = min(wmaxl - lo, cnt);
        int nsel = 0;
        for (int j0 = 0; j0 < wl; j0 += 32) {
            const int j = j0 + lane;
            bool keep = false;
            if (j < wl) {
                const float4 t1 = s1[sb + j];
                keep = !cull || patch_may_hit(s0[sb + j], t1.x, t1.w, xa, xa + 7.0f, ya, ya + 7.0f);
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep)
                s_selw[nsel + __popc(m & lanemask_lt())] = (uint8_t)j;
            nsel += __popc(m);
        }
        __syncwarp();
        auto walk = [&](auto gen_tag) {
        constexpr bool GEN = decltype(gen_tag)::value;
        for (int k = nsel - 1; k >= 0; --k) {
            const int j = s_selw[k];
            float g[NG];
            const float4 q0 = s0[sb + j], q1 = s1[sb + j], q2 = s2[sb + j];
            RecX2 R;
            R.uv = make_ulonglong2(bc2(q0.x), bc2(q0.y));
            R.ab = make_ulonglong2(bc2(q0.z), bc2(q0.w));
            R.co = make_ulonglong2(bc2(q1.x), bc2(q2.w));
            R.zr = make_ulonglong2(bc2(q1.z), bc2(q2.x));
            R.gb = make_ulonglong2(bc2(q2.y), bc2(q2.z));
            const bool contrib =
                pix_adj_x2<false, false, GEN>(P2, lo + j, R, a.alpha_max, -a.alpha_max, -a.alpha_min, g);
            if (__any_sync(0xffffffffu, contrib)) {
                float v[8];
#pragma unroll
                for (int k2 = 0; k2 < 8; ++k2)
                    v[k2] = k2 < NG ? g[k2] : 0.0f;
                const float sum = warp_sum_transpose<8, NG>(v, lane);
                const int kk = lane / 4;
                if ((lane % 4) == 0 && kk < NG)
                    s_slots[(kk * kBwd2Warps + warp) * kBwdSlotRow + j] = sum;
            }
        }
        };
        if (gen)
            walk(std::true_type{});
        else
            walk(std::false_type{});
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            float G[NG];
            bool any = false;
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                float s = -0.0f;
#pragma unroll
                for (int w = 0; w < kBwd2Warps; ++w) {
                    float &slot = s_slots[(k * kBwd2Warps + w) * kBwdSlotRow + threadIdx.x];
                    s += slot;
                    slot = 0.0f;
                }
                G[k] = -s;  // the packed walk sums the negated gradient
                any |= s != 0.0f;
            }
            if (any && a.tile_twist)
                chain_twist(G, s1[sb + threadIdx.x], s_x0[threadIdx.x], s_x1[threadIdx.x], d.fx, d.fy, cc, tw);
        }
    }
    if (a.tile_twist)
        store_tile_twist<kBwd2Warps>(tw, twist_warps, s_tw, a.tile_twist + (size_t)t * 6);
}

// The registration forward and adjoint of one tile in one CTA (the
// registration loss of Sec. 3.2; not the tracking loss, whose per-keyframe
// median needs every tile's forward first).  A thread holds the same two
// pixels in both halves, so T_final, `last` and the loss signs stay in
// registers instead of a round trip through HBM, and the adjoint needs no
// set-up of its own (descriptor, pixel state, pivot, first chunk): one
// launch in place of the forward and the adjoint, with the same values
// bit for bit (the same operations in the same order).
template <int X>
__global__ void __launch_bounds__(kFwdThreads, 8) k_fwdbwd(const gsl::RasterArgs a)
{
    fwd_tile<true, X, true>(a, a.tile_order ? a.tile_order[blockIdx.x] : blockIdx.x);
}

template <int X>
__global__ void __launch_bounds__(kFwdThreads, 8) k_fwdbwd_q(const gsl::RasterArgs a)
{
    run_queue(a, [&](uint32_t t) { fwd_tile<true, X, true>(a, t); });
}

template <bool REG, bool FULL>
constexpr size_t bwd2_smem()
{
    return (size_t)(FULL ? 10 : 6) * kBwd2Warps * kBwdSlotRow * sizeof(float);
}

// CTAs of the persistent kernels: as many as can be resident at once
// (occupancy x SMs), found once by raster_init
int g_fwd_q_ctas = 0, g_bwd_q_ctas = 0, g_fb_q_ctas = 0;

// (a one-pixel-per-thread adjoint with 256-thread CTAs measured 2.00 ms
// against 1.43 ms for this one on the room workload)
template <bool REG, bool FULL>
void launch_backward(const gsl::RasterArgs &a, cudaStream_t s)
{
    if constexpr (REG && !FULL) {
        if (a.queue && g_bwd_q_ctas > 0) {
            cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
            k_backward2_q<REG, FULL><<<(unsigned)std::min<uint32_t>(a.n_tiles, g_bwd_q_ctas), kBwd2Threads,
                                       bwd2_smem<REG, FULL>(), s>>>(a);
            ++gsl::g_launches;
            return;
        }
    }
    k_backward2<REG, FULL><<<a.n_tiles, kBwd2Threads, bwd2_smem<REG, FULL>(), s>>>(a);
    ++gsl::g_launches;
}

template <int X>
void launch_fwdbwd(const gsl::RasterArgs &a, cudaStream_t s)
{
    constexpr size_t smem = bwd2_smem<true, false>();
    if (a.queue && g_fb_q_ctas > 0) {
        cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
        k_fwdbwd_q<X><<<(unsigned)std::min<uint32_t>(a.n_tiles, g_fb_q_ctas), kFwdThreads, smem, s>>>(a);
    } else {
        k_fwdbwd<X><<<a.n_tiles, kFwdThreads, smem, s>>>(a);
    }
}

template <int X>
void launch_forward_reg(const gsl::RasterArgs &a, cudaStream_t s)
{
    if (a.queue && g_fwd_q_ctas > 0) {
        cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
        k_forward_q<X><<<(unsigned)std::min<uint32_t>(a.n_tiles, g_fwd_q_ctas), kFwdThreads, 0, s>>>(a);
    } else {
        k_forward<true, X><<<a.n_tiles, kFwdThreads, 0, s>>>(a);
    }
}

}  // namespace

namespace gsl {

void raster_init()
{
    cudaFuncSetAttribute(k_backward2<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwd2_smem<true, false>());
    cudaFuncSetAttribute(k_backward2<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwd2_smem<false, false>());
    cudaFuncSetAttribute(k_backward2<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwd2_smem<false, true>());
    cudaFuncSetAttribute(k_backward2_q<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwd2_smem<true, false>());
    int dev = 0, sms = 0, f = 0, b = 0, fb = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f, k_forward_q<0>, kFwdThreads, 0) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward2_q<true, false>, kBwd2Threads,
                                                      bwd2_smem<true, false>()) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fb, k_fwdbwd_q<0>, kFwdThreads, bwd2_smem<true, false>()) ==
            cudaSuccess) {
        g_fwd_q_ctas = std::max(f, 1) * sms;
        g_bwd_q_ctas = std::max(b, 1) * sms;
        g_fb_q_ctas = std::max(fb, 1) * sms;
    }
    cudaGetLastError();
}

void forward(const RasterArgs &a, bool registration, cudaStream_t s)
{
    if (a.n_tiles == 0)
        return;
    // (one pixel per thread with scalar operations, 256-thread CTAs on 8x4
    // warp patches: 0.551 against 0.447 ms on the room workload; without
    // packed operations two pixels per thread had measured slower, 0.82
    // against 0.76 ms, as the early stop favours one pixel per thread)
    if (!registration)
        k_forward<false, 0><<<a.n_tiles, kFwdThreads, 0, s>>>(a);
    else if (a.exposure && a.count_contrib)
        launch_forward_reg<kFwdExposure | kFwdCount>(a, s);
    else if (a.exposure)
        launch_forward_reg<kFwdExposure>(a, s);
    else if (a.count_contrib)
        launch_forward_reg<kFwdCount>(a, s);
    else
        launch_forward_reg<0>(a, s);
    ++g_launches;
}

void backward(const RasterArgs &a, bool registration, bool full, cudaStream_t s)
{
    if (a.n_tiles == 0)
        return;
    if (registration)
        launch_backward<true, false>(a, s);
    else if (full)
        launch_backward<false, true>(a, s);
    else
        launch_backward<false, false>(a, s);
}

void forward_backward(const RasterArgs &a, cudaStream_t s)
{
    if (a.n_tiles == 0)
        return;
    if (a.exposure && a.count_contrib)
        launch_fwdbwd<kFwdExposure | kFwdCount>(a, s);
    else if (a.exposure)
        launch_fwdbwd<kFwdExposure>(a, s);
    else if (a.count_contrib)
        launch_fwdbwd<kFwdCount>(a, s);
    else
        launch_fwdbwd<0>(a, s);
    ++g_launches;
}

}  // namespace gsl
