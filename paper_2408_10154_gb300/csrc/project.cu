// project.cu -- pose transform + EWA projection of moving submaps.
//
// One thread per Gaussian of a projection group loads the Gaussian once
// (float4 SoA loads, coalesced); the group's (keyframe, Gaussian) pairs in
// front of the camera are then projected by the warp's lanes in turn (the
// rigid transform of Eq. 8/9 composed with the keyframe's world -> camera
// transform), one record per visible pair.  56 B read per Gaussian per
// pass, 48 B record + 32 B auxiliary written per visible (keyframe,
// Gaussian), 16 B list entry per pair.
//
// Every value that decides an integer outcome follows a fixed FP32
// operation sequence (see gs_internal.cuh): camera-space mean, quaternion
// normalisation, scales e^s, camera-space covariance A A^T with
// A = M_R R(q) diag(e^s), the Jacobian J, the dilated 2D covariance, its
// determinant and conic, the 3-sigma radius, the pixel mean and the tile
// rectangle.
#include "gs_internal.cuh"

namespace {

using namespace gsk;

// Tight tile rectangle (contract step 7b, see ProjectArgs::tight): the
// tiles of the 3-sigma rectangle [x0, x1) x [y0, y1) whose pixel centres can
// reach the record's alpha threshold.  Such a pixel lies in the ellipse
// d^T Q d <= -2 tau (Q = [[A, B], [B, C]], A = -2 ca, B = -cb, C = -2 cc;
// tau = ln(alpha_min) - ln(o) - 0.06 with the contract's log_ct), whose
// axis-aligned box about (u, v) has half-sizes sqrt(-2 tau C / det),
// sqrt(-2 tau A / det) (det = AC - B^2), widened by 0.1 % + 0.01 px; tile t
// meets it when its centres [16 t + 0.5, 16 t + 15.5] meet the box.  An
// opacity below alpha_min e^-0.06 empties the rectangle; nearly singular
// conics (B^2 > 0.998 AC), whose FP32 exponent is less accurate than the
// margins, keep the 3-sigma rectangle.  Every step is a fixed FP32
// operation, mirrored by the oracle, so both sides build the same lists.
// the reciprocal of the tile size, a power of two: x * kInvTile is x / 16
// correctly rounded
constexpr float kInvTile = 1.0f / (float)kTile;
static_assert(kTile == 16, "kInvTile is exact for a power-of-two tile");

__device__ __forceinline__ void tighten(float ca, float cb, float cc, float o, float u, float v, float alpha_min,
                                        int TX, int TY, int &x0, int &x1, int &y0, int &y1)
{
    const float tau = sub_rn(sub_rn(log_ct(alpha_min), log_ct(o)), 0.06f);
    if (!(tau < 0.0f)) {
        x1 = x0;
        return;
    }
    const float A = mul_rn(-2.0f, ca), B = -cb, C = mul_rn(-2.0f, cc);
    const float AC = mul_rn(A, C), BB = mul_rn(B, B);
    const float det = sub_rn(AC, BB);
    if (!(det > 0.0f) || !(BB <= mul_rn(0.998f, AC)))
        return;
    const float s = __fdiv_rn(mul_rn(-2.0f, tau), det);
    const float ex = fma_rn(__fsqrt_rn(mul_rn(s, C)), 1.001f, 0.01f);
    const float ey = fma_rn(__fsqrt_rn(mul_rn(s, A)), 1.001f, 0.01f);
    if (!(ex >= 0.0f) || !(ey >= 0.0f))
        return;
    const float iB = kInvTile;
    const float tx0 = fminf(fmaxf(ceilf(mul_rn(sub_rn(sub_rn(u, ex), 15.5f), iB)), 0.0f), (float)TX);
    const float tx1 = fminf(fmaxf(add_rn(floorf(mul_rn(sub_rn(add_rn(u, ex), 0.5f), iB)), 1.0f), 0.0f), (float)TX);
    const float ty0 = fminf(fmaxf(ceilf(mul_rn(sub_rn(sub_rn(v, ey), 15.5f), iB)), 0.0f), (float)TY);
    const float ty1 = fminf(fmaxf(add_rn(floorf(mul_rn(sub_rn(add_rn(v, ey), 0.5f), iB)), 1.0f), 0.0f), (float)TY);
    x0 = max(x0, (int)tx0);
    x1 = min(x1, (int)tx1);
    y0 = max(y0, (int)ty0);
    y1 = min(y1, (int)ty1);
}

// Segmented lists: a visible record (count > 0) adds +1 at (y0, x0) and
// (y1, x1) and -1 (mod 2^32) at (y0, x1) and (y1, x0) of its keyframe's
// (TY + 1) x (TX + 1) difference grid, whose 2-D prefix sum is the tile
// count; every record writes its entry {depth bits, first tile, width |
// height << 16, tiles per row} (size 0 when not visible).
__device__ __forceinline__ void seg_note(const gsl::ProjectArgs &a, const int *geo, uint32_t rec, float z, int count,
                                         int x0, int x1, int y0, int y1)
{
    const bool vis = count > 0;
    const int TX = geo[0];
    if (vis) {
        const uint32_t w1 = (uint32_t)TX + 1;
        uint32_t *g = a.seg_diff + (uint32_t)geo[4];
        atomicAdd(g + (uint32_t)y0 * w1 + (uint32_t)x0, 1u);
        atomicAdd(g + (uint32_t)y1 * w1 + (uint32_t)x1, 1u);
        atomicAdd(g + (uint32_t)y0 * w1 + (uint32_t)x1, 0xffffffffu);
        atomicAdd(g + (uint32_t)y1 * w1 + (uint32_t)x0, 0xffffffffu);
    }
    a.seg_list[rec] = vis ? make_uint4(__float_as_uint(z),
                                           (uint32_t)geo[3] + (uint32_t)y0 * (uint32_t)TX + (uint32_t)x0,
                                           (uint32_t)(x1 - x0) | ((uint32_t)(y1 - y0) << 16), (uint32_t)TX)
                              : make_uint4(0u, 0u, 0u, 0u);
}

// One (keyframe, Gaussian) pair: camera-space mean, covariance, the
// dilated 2D covariance, conic, radius, pixel mean and tile rectangle (all
// the contract's FP32 sequence), the record and its list entry.
__device__ __forceinline__ void project_pair(const gsl::ProjectArgs &a, const float *M, const float *cam,
                                             const int *geo, uint32_t i, const float4 &mu, const float (&Rq)[3][3],
                                             const float (&sig)[3], float opa, const float4 &col, bool qok)
{
    const uint32_t rec = (uint32_t)geo[2] + i;
    const float x = fma_rn(M[2], mu.z, fma_rn(M[1], mu.y, fma_rn(M[0], mu.x, M[3])));
    const float y = fma_rn(M[6], mu.z, fma_rn(M[5], mu.y, fma_rn(M[4], mu.x, M[7])));
    const float z = fma_rn(M[10], mu.z, fma_rn(M[9], mu.y, fma_rn(M[8], mu.x, M[11])));
    int count = 0;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    if (z > a.z_near && qok) {
        float A[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float b = fma_rn(M[4 * r + 2], Rq[2][c], fma_rn(M[4 * r + 1], Rq[1][c], mul_rn(M[4 * r], Rq[0][c])));
                A[r][c] = mul_rn(b, sig[c]);
            }
        float S[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = r; c < 3; ++c)
                S[r][c] = fma_rn(A[r][2], A[c][2], fma_rn(A[r][1], A[c][1], mul_rn(A[r][0], A[c][0])));
        const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
        const float iz = __fdiv_rn(1.0f, z);
        const float tx = mul_rn(x, iz), ty = mul_rn(y, iz);
        const float j00 = mul_rn(fx, iz), j11 = mul_rn(fy, iz);
        const float j02 = -mul_rn(j00, tx), j12 = -mul_rn(j11, ty);
        const float r00 = fma_rn(j00, S[0][0], mul_rn(j02, S[0][2]));
        const float r01 = fma_rn(j00, S[0][1], mul_rn(j02, S[1][2]));
        const float r02 = fma_rn(j00, S[0][2], mul_rn(j02, S[2][2]));
        const float r11 = fma_rn(j11, S[1][1], mul_rn(j12, S[1][2]));
        const float r12 = fma_rn(j11, S[1][2], mul_rn(j12, S[2][2]));
        const float ea = add_rn(fma_rn(r00, j00, mul_rn(r02, j02)), a.dilation);
        const float eb = fma_rn(r01, j11, mul_rn(r02, j12));
        const float ec = add_rn(fma_rn(r11, j11, mul_rn(r12, j12)), a.dilation);
        const float det = fma_rn(ea, ec, -mul_rn(eb, eb));
        if (det > 0.0f) {
            const float idet = __fdiv_rn(1.0f, det);
            const float ca = mul_rn(-0.5f, mul_rn(ec, idet));
            const float cb = mul_rn(eb, idet);
            const float cc = mul_rn(-0.5f, mul_rn(ea, idet));
            const float mid = mul_rn(0.5f, add_rn(ea, ec));
            const float disc = fmaxf(0.1f, fma_rn(mid, mid, -det));
            const float lam = add_rn(mid, __fsqrt_rn(disc));
            const float rf = ceilf(mul_rn(3.0f, __fsqrt_rn(lam)));
            const float u = fma_rn(fx, tx, cx);
            const float vv = fma_rn(fy, ty, cy);
            if (rf < 1.0e7f && fabsf(u) < 1.0e7f && fabsf(vv) < 1.0e7f) {
                const int TX = geo[0], TY = geo[1];
                if (a.smooth) {
                    x0 = 0; x1 = TX; y0 = 0; y1 = TY;
                } else {
                    // x / 16 as x * (1/16): the same correctly rounded
                    // value (a power of two), without a division
                    const float iB = kInvTile;
                    const float fx0 = floorf(mul_rn(sub_rn(u, rf), iB));
                    const float fx1 = add_rn(floorf(mul_rn(add_rn(u, rf), iB)), 1.0f);
                    const float fy0 = floorf(mul_rn(sub_rn(vv, rf), iB));
                    const float fy1 = add_rn(floorf(mul_rn(add_rn(vv, rf), iB)), 1.0f);
                    x0 = (int)fminf(fmaxf(fx0, 0.0f), (float)TX);
                    x1 = (int)fminf(fmaxf(fx1, 0.0f), (float)TX);
                    y0 = (int)fminf(fmaxf(fy0, 0.0f), (float)TY);
                    y1 = (int)fminf(fmaxf(fy1, 0.0f), (float)TY);
                    if (a.tight)
                        tighten(ca, cb, cc, opa, u, vv, a.alpha_min, TX, TY, x0, x1, y0, y1);
                }
                if (x0 < x1 && y0 < y1) {
                    count = (x1 - x0) * (y1 - y0);
                    float4 *R = a.rec + 3 * (size_t)rec;
                    R[0] = make_float4(u, vv, ca, cb);
                    R[1] = make_float4(cc, opa, z, __uint_as_float((uint32_t)x0 | ((uint32_t)x1 << 16)));
                    R[2] = make_float4(col.x, col.y, col.z, __uint_as_float((uint32_t)y0 | ((uint32_t)y1 << 16)));
                    if (a.aux) {
                        a.aux[2 * (size_t)rec] = make_float4(x, y, S[0][0], S[0][1]);
                        a.aux[2 * (size_t)rec + 1] = make_float4(S[0][2], S[1][1], S[1][2], S[2][2]);
                    }
                }
            }
        }
    }
    if (a.counts)
        a.counts[rec] = count;
    if (a.seg_hdr)
        seg_note(a, geo, rec, z, count, x0, x1, y0, y1);
}

// keyframes per compaction round of a warp (its queue holds 32 per keyframe)
constexpr int kProjRound = 8;

// One thread per Gaussian of a group loads it and derives its
// view-independent part (R(q), e^s, opacity) once.  Of the group's
// (keyframe, Gaussian) pairs only those in front of the camera go on to the
// projection, and most of the rest of them then miss the image, so a
// thread that looped over its own keyframes would leave most lanes of its
// warp idle on every keyframe.  Instead each warp keeps its 32 Gaussians'
// view-independent parts in shared memory and, kProjRound keyframes at a
// time, queues the pairs in front of the camera (ballot compaction) and
// projects them 32 at a time on all of its lanes.  A pair behind the near
// plane writes its empty list entry in the first pass.  Every value is
// computed by the same operations as in a per-thread loop.
__global__ void __launch_bounds__(256) k_project(const gsl::ProjectArgs a)
{
    // locate the group of this block (groups are few; linear scan)
    int gi = 0;
    while (gi + 1 < a.n_groups && blockIdx.x >= a.groups[gi + 1].blk_base)
        ++gi;
    const GroupDesc G = a.groups[gi];
    __shared__ float sM[kMaxVpPerGroup][12];
    __shared__ float sCam[kMaxVpPerGroup][4];  // fx, fy, cx, cy
    __shared__ int sGeo[kMaxVpPerGroup][6];    // TX, TY, rec_base, tile_base, diff_base, unused
    // per warp and lane: mu (4), Rq (9), e^s (3), opacity, colour (3), q ok
    constexpr int kF = 21;
    __shared__ float sG[8][kF][32];
    __shared__ uint16_t sQ[8][kProjRound * 32];
    for (int v = threadIdx.x; v < G.vp_count; v += blockDim.x) {
        const int vp = G.vp_first + v;
        const VpDesc &d = a.vps[vp];
        float P[12], V[12], M[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            P[k] = a.pose32[12 * vp + k];
            V[k] = d.w2c[k];
        }
        compose_ct(V, P, M);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            sM[v][k] = M[k];
        sCam[v][0] = d.fx;
        sCam[v][1] = d.fy;
        sCam[v][2] = d.cx;
        sCam[v][3] = d.cy;
        sGeo[v][0] = d.TX;
        sGeo[v][1] = d.TY;
        sGeo[v][2] = (int)d.rec_base;
        sGeo[v][3] = (int)d.tile_base;
        sGeo[v][4] = (int)d.diff_base;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = (int)(blockIdx.x - G.blk_base) * blockDim.x + threadIdx.x;
    const int i_warp = i - lane;  // the warp's first Gaussian
    if (i_warp >= G.n)
        return;  // the whole warp is past the group (warp-uniform)
    const bool mine = i < G.n;
    float4 mu = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    bool qok = false;
    if (mine) {
        const VpDesc &d0 = a.vps[G.vp_first];
        mu = __ldg(d0.means + i);
        const float4 sc = __ldg(d0.scales + i);
        const float4 q = __ldg(d0.quats + i);
        const float logit = __ldg(d0.logits + i);
        const float4 col = __ldg(d0.rgb + i);
        const bool finite = isfinite(mu.x) && isfinite(mu.y) && isfinite(mu.z) && isfinite(sc.x) &&
                            isfinite(sc.y) && isfinite(sc.z) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) &&
                            isfinite(q.w) && isfinite(logit);
        if (!finite)
            atomicOr(a.flags, kFlagNonFinite);
        // view-independent part: R(q), e^s, opacity
        const float n2 = fma_rn(q.x, q.x, fma_rn(q.y, q.y, fma_rn(q.z, q.z, mul_rn(q.w, q.w))));
        qok = n2 > 0.0f;
        const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
        const float qw = mul_rn(q.x, inv), qx = mul_rn(q.y, inv), qy = mul_rn(q.z, inv), qz = mul_rn(q.w, inv);
        const float xx = mul_rn(qx, qx), yy = mul_rn(qy, qy), zz = mul_rn(qz, qz);
        const float xy = mul_rn(qx, qy), xz = mul_rn(qx, qz), yz = mul_rn(qy, qz);
        const float wx = mul_rn(qw, qx), wy = mul_rn(qw, qy), wz = mul_rn(qw, qz);
        float *g = &sG[warp][0][lane];
        g[0 * 32] = mu.x;
        g[1 * 32] = mu.y;
        g[2 * 32] = mu.z;
        g[3 * 32] = sub_rn(1.0f, mul_rn(2.0f, add_rn(yy, zz)));
        g[4 * 32] = mul_rn(2.0f, sub_rn(xy, wz));
        g[5 * 32] = mul_rn(2.0f, add_rn(xz, wy));
        g[6 * 32] = mul_rn(2.0f, add_rn(xy, wz));
        g[7 * 32] = sub_rn(1.0f, mul_rn(2.0f, add_rn(xx, zz)));
        g[8 * 32] = mul_rn(2.0f, sub_rn(yz, wx));
        g[9 * 32] = mul_rn(2.0f, sub_rn(xz, wy));
        g[10 * 32] = mul_rn(2.0f, add_rn(yz, wx));
        g[11 * 32] = sub_rn(1.0f, mul_rn(2.0f, add_rn(xx, yy)));
        g[12 * 32] = exp_ct(sc.x);
        g[13 * 32] = exp_ct(sc.y);
        g[14 * 32] = exp_ct(sc.z);
        g[15 * 32] = __fdiv_rn(1.0f, add_rn(1.0f, exp_ct(-logit)));
        g[16 * 32] = col.x;
        g[17 * 32] = col.y;
        g[18 * 32] = col.z;
        g[19 * 32] = qok ? 1.0f : 0.0f;
    }
    __syncwarp();
    for (int vb = 0; vb < G.vp_count; vb += kProjRound) {
        const int ve = min(vb + kProjRound, G.vp_count);
        int qn = 0;
        for (int v = vb; v < ve; ++v) {
            bool front = false;
            if (mine) {
                const float *M = sM[v];
                const float z = fma_rn(M[10], mu.z, fma_rn(M[9], mu.y, fma_rn(M[8], mu.x, M[11])));
                front = z > a.z_near && qok;
                if (!front) {
                    // behind the near plane: no record, an empty list entry
                    const uint32_t rec = (uint32_t)sGeo[v][2] + (uint32_t)i;
                    if (a.counts)
                        a.counts[rec] = 0;
                    if (a.seg_hdr)
                        seg_note(a, sGeo[v], rec, z, 0, 0, 0, 0, 0);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, front);
            if (front)
                sQ[warp][qn + __popc(m & lanemask_lt())] = (uint16_t)(((v - vb) << 5) | lane);
            qn += __popc(m);
        }
        __syncwarp();
        for (int q0 = 0; q0 < qn; q0 += 32) {
            if (q0 + lane < qn) {
                const int e = sQ[warp][q0 + lane];
                const int v = vb + (e >> 5), src = e & 31;
                const float *g = &sG[warp][0][src];
                const float4 m4 = make_float4(g[0], g[32], g[64], 0.0f);
                const float Rq[3][3] = {{g[3 * 32], g[4 * 32], g[5 * 32]},
                                        {g[6 * 32], g[7 * 32], g[8 * 32]},
                                        {g[9 * 32], g[10 * 32], g[11 * 32]}};
                const float sig[3] = {g[12 * 32], g[13 * 32], g[14 * 32]};
                const float4 c4 = make_float4(g[16 * 32], g[17 * 32], g[18 * 32], 0.0f);
                project_pair(a, sM[v], sCam[v], sGeo[v], (uint32_t)(i_warp + src), m4, Rq, sig, g[15 * 32], c4,
                             g[19 * 32] != 0.0f);
            }
        }
        __syncwarp();
    }
}

}  // namespace

namespace gsl {

void project(const ProjectArgs &a, cudaStream_t s)
{
    if (a.seg_hdr)
        cudaMemsetAsync(a.seg_hdr, 0, a.seg_zero_bytes, s);
    if (a.n_blocks == 0)
        return;
    k_project<<<a.n_blocks, 256, 0, s>>>(a);
    ++g_launches;
}

}  // namespace gsl
