// params.cu -- the adjoint to every Gaussian parameter (the optional output
// of gs_render_backward): per-duplicate screen gradients are grouped by
// record (a radix sort of the duplicates by record index), then one thread
// per Gaussian sums its records over the cameras in camera order and
// chains the result through the projection, the rigid transform
// (Eq. 8/9) and the scale / rotation / opacity parameterisation.  Fixed
// summation order, no atomics.
#include "gs_internal.cuh"

namespace {

using namespace gsk;

__global__ void k_iota_copy(const uint32_t *src, const uint32_t *n_dev, uint32_t cap, uint32_t *keys,
                            uint32_t *pos)
{
    const uint32_t n = min(*n_dev, cap);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        keys[i] = src[i];
        pos[i] = i;
    }
}

// ranges of equal keys in a sorted key array (key = record index)
__global__ void k_key_ranges(const uint32_t *keys, const uint32_t *n_dev, uint32_t cap, uint2 *ranges)
{
    const uint32_t n = min(*n_dev, cap);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint32_t k = keys[i];
    if (i == 0 || keys[i - 1] != k)
        ranges[k].x = i;
    if (i == n - 1 || keys[i + 1] != k)
        ranges[k].y = i + 1;
}

__global__ void __launch_bounds__(128) k_param_grads(const gsl::ParamArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n)
        return;
    // object-frame accumulators over cameras
    float gmu[3] = {0, 0, 0}, GS[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dop = 0.0f, drgb[3] = {0, 0, 0};
    for (int c = 0; c < a.n_vps; ++c) {
        const VpDesc &d = a.vps[c];
        const uint32_t r = d.rec_base + (uint32_t)i;
        const uint2 seg = a.rec_ranges[r];
        if (seg.y <= seg.x)
            continue;
        float G[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (uint32_t p = seg.x; p < seg.y; ++p) {
            const float *src = a.dup_grads + (size_t)a.rpos[p] * 10;
#pragma unroll
            for (int k = 0; k < 10; ++k)
                G[k] += src[k];
        }
        const float4 q1 = a.rec[3 * (size_t)r + 1];
        const float4 x0 = a.aux[2 * (size_t)r], x1 = a.aux[2 * (size_t)r + 1];
        const float fx = d.fx, fy = d.fy;
        const float mx = x0.x, my = x0.y, mz = q1.z;
        const float S00 = x0.z, S01 = x0.w, S02 = x1.x, S11 = x1.y, S12 = x1.z, S22 = x1.w;
        // screen -> camera frame (the same chain as the pose adjoint)
        const float gp = 0.5f * G[2], gq = 0.5f * G[3], gs = 0.5f * G[4];
        const float iz = 1.0f / mz, iz2 = iz * iz;
        const float j00 = fx * iz, j11 = fy * iz, j02 = -fx * mx * iz2, j12 = -fy * my * iz2;
        const float r00 = gp * j00, r01 = gq * j11, r02 = gp * j02 + gq * j12;
        const float r10 = gq * j00, r11 = gs * j11, r12 = gq * j02 + gs * j12;
        const float Gc[3][3] = {{j00 * r00, j00 * r01, j00 * r02},
                                {j00 * r01, j11 * r11, j11 * r12},
                                {j00 * r02, j11 * r12, j02 * r02 + j12 * r12}};
        const float dJ00 = 2.0f * (r00 * S00 + r01 * S01 + r02 * S02);
        const float dJ02 = 2.0f * (r00 * S02 + r01 * S12 + r02 * S22);
        const float dJ11 = 2.0f * (r10 * S01 + r11 * S11 + r12 * S12);
        const float dJ12 = 2.0f * (r10 * S02 + r11 * S12 + r12 * S22);
        const float du = G[0], dv = G[1], dz = G[5];
        const float gm[3] = {du * fx * iz - dJ02 * fx * iz2, dv * fy * iz - dJ12 * fy * iz2,
                             -du * fx * mx * iz2 - dv * fy * my * iz2 + dz - dJ00 * fx * iz2 - dJ11 * fy * iz2 +
                                 2.0f * iz2 * iz * (dJ02 * fx * mx + dJ12 * fy * my)};
        // camera-from-object rotation M = V_R T_R of this camera and pose
        float M[3][3];
        const float *P = a.pose32 + 12 * c;
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                M[u][v] = d.w2c[4 * u] * P[v] + d.w2c[4 * u + 1] * P[4 + v] + d.w2c[4 * u + 2] * P[8 + v];
        // object frame: g_mu = M^T g_m, G_Sigma = M^T Gc M
        float T1[3][3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            gmu[u] += M[0][u] * gm[0] + M[1][u] * gm[1] + M[2][u] * gm[2];
#pragma unroll
            for (int v = 0; v < 3; ++v)
                T1[u][v] = Gc[u][0] * M[0][v] + Gc[u][1] * M[1][v] + Gc[u][2] * M[2][v];
        }
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                GS[u][v] += M[0][u] * T1[0][v] + M[1][u] * T1[1][v] + M[2][u] * T1[2][v];
        dop += G[6];
        drgb[0] += G[7];
        drgb[1] += G[8];
        drgb[2] += G[9];
    }
    // Sigma = R(q) S^2 R(q)^T with S = diag(e^s); o = sigmoid(logit)
    const float4 q = a.quats[i], sc = a.scales[i];
    const float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    const float ql = sqrtf(n2), iq = 1.0f / ql;
    const float w = q.x * iq, x = q.y * iq, y = q.z * iq, z = q.w * iq;
    const float R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                           {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                           {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    const float sg2[3] = {expf(2.0f * sc.x), expf(2.0f * sc.y), expf(2.0f * sc.z)};
    // dL/ds_k = 2 sigma_k^2 (R^T G R)_kk ;  dL/dR = 2 G R S^2
    float GR[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v)
            GR[u][v] = GS[u][0] * R[0][v] + GS[u][1] * R[1][v] + GS[u][2] * R[2][v];
    float ds[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        ds[k] = 2.0f * sg2[k] * (R[0][k] * GR[0][k] + R[1][k] * GR[1][k] + R[2][k] * GR[2][k]);
    float dR[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v)
            dR[u][v] = 2.0f * GR[u][v] * sg2[v];
    // partial derivatives of R(q_hat) w.r.t. (w, x, y, z)
    const float gw = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    const float gx = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                          w * dR[2][1] - 2 * x * dR[2][2]);
    const float gy = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                          z * dR[2][1] - 2 * y * dR[2][2]);
    const float gz = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1] +
                          y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    // through q_hat = q / |q|
    const float dot = w * gw + x * gx + y * gy + z * gz;
    const float4 dq = make_float4((gw - w * dot) * iq, (gx - x * dot) * iq, (gy - y * dot) * iq, (gz - z * dot) * iq);
    const float o = 1.0f / (1.0f + expf(-a.logits[i]));
    if (a.g_means)
        reinterpret_cast<float4 *>(a.g_means)[i] = make_float4(gmu[0], gmu[1], gmu[2], 0.0f);
    if (a.g_scales)
        reinterpret_cast<float4 *>(a.g_scales)[i] = make_float4(ds[0], ds[1], ds[2], 0.0f);
    if (a.g_quats)
        reinterpret_cast<float4 *>(a.g_quats)[i] = dq;
    if (a.g_logits)
        a.g_logits[i] = dop * o * (1.0f - o);
    if (a.g_rgb)
        reinterpret_cast<float4 *>(a.g_rgb)[i] = make_float4(drgb[0], drgb[1], drgb[2], 0.0f);
}

inline uint32_t div_up(size_t a, size_t b) { return (uint32_t)((a + b - 1) / b); }

}  // namespace

namespace gsl {

void param_grads(const ParamArgs &a, const uint32_t *sorted_recs, const uint32_t *n_dups, uint32_t cap,
                 uint32_t *rkeys[2], uint32_t *rpos[2], int rec_bits, uint32_t *hist, uint32_t *hist_partials,
                 uint2 *rec_ranges, uint32_t n_records, cudaStream_t s)
{
    k_iota_copy<<<div_up(cap ? cap : 1, 256), 256, 0, s>>>(sorted_recs, n_dups, cap, rkeys[0], rpos[0]);
    ++g_launches;
    const int c = sort_u32(rkeys, rpos, n_dups, cap, rec_bits, hist, hist_partials, s);
    cudaMemsetAsync(rec_ranges, 0, sizeof(uint2) * (size_t)(n_records ? n_records : 1), s);
    k_key_ranges<<<div_up(cap ? cap : 1, 256), 256, 0, s>>>(rkeys[c], n_dups, cap, rec_ranges);
    ParamArgs b = a;
    b.rpos = rpos[c];
    b.rec_ranges = rec_ranges;
    if (a.n > 0)
        k_param_grads<<<div_up((size_t)a.n, 128), 128, 0, s>>>(b);
    g_launches += 2;
}

}  // namespace gsl
