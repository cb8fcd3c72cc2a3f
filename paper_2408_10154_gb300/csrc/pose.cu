// pose.cu -- per-keyframe reductions and the on-device registration step:
// tile twists -> 6-vector per keyframe (FP32 TwoSum pairs in a fixed
// order, one FP64 value per component),
// Adam on the twist with a cosine-decayed learning rate, exponential-map
// pose update about the moving submap's centroid (Sec. 3.2; learning rates
// Supp. B), the standalone L1 loss, the Eq. 7 fusion and the Eq. 8/9 rigid
// transform of a submap.  Latency-bound tiny kernels, FP64 state.
#include "gs_internal.cuh"

namespace {

using namespace gsk;

__device__ void so3_exp(const double *w, double R[3][3])
{
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        double sn, cs;
        sincos(th, &sn, &cs);
        a = sn / th;
        b = (1.0 - cs) / th2;
    }
    const double K[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double k2 = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
            R[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + b * k2;
        }
}

// b^n for a step count n >= 1 (binary powering: a few multiplies instead of
// a general pow, whose FP64 log/exp chain is long on this part)
__device__ __forceinline__ double pow_count(double b, double n)
{
    unsigned long long m = (unsigned long long)n;
    double r = 1.0, x = b;
    while (m) {
        if (m & 1ull)
            r *= x;
        x *= x;
        m >>= 1;
    }
    return r;
}

// Adam step of twist component i (0..2 rotation, 3..5 translation) with
// gradient gi: updates its moments st[i], st[6 + i] and returns the step
// xi_i.  k = iteration index in [0, iters) of the learning-rate schedule;
// t = steps taken including this one (bias correction).
__device__ double adam_component(double *st, int i, double gi, double t, int k, int iters, float lr_rot,
                                 float lr_trans, float b1f, float b2f, float epsf, float lr_final)
{
    const double kPi = 3.14159265358979323846;
    const double b1 = b1f, b2 = b2f, eps = epsf, f = lr_final;
    const double sched = f + (1.0 - f) * 0.5 * (1.0 + cos(kPi * (double)k / (double)iters));
    st[i] = b1 * st[i] + (1.0 - b1) * gi;
    st[6 + i] = b2 * st[6 + i] + (1.0 - b2) * gi * gi;
    const double mh = st[i] / (1.0 - pow_count(b1, t));
    const double vh = st[6 + i] / (1.0 - pow_count(b2, t));
    const double lr = (i < 3 ? (double)lr_rot : (double)lr_trans) * sched;
    return -lr * mh / (sqrt(vh) + eps);
}

// Pose update by the step xi about pivot c:
// R <- exp(-s_w) R, t <- exp(-s_w)(t - c) + c - s_v (xi carries the signs).
__device__ void exp_update(double *pose, const double *xi, const double *c)
{
    double dR[3][3];
    so3_exp(xi, dR);
    double R[3][3], tt[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            R[i][j] = pose[4 * i + j];
        tt[i] = pose[4 * i + 3];
    }
    const double rel[3] = {tt[0] - c[0], tt[1] - c[1], tt[2] - c[2]};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            pose[4 * i + j] = dR[i][0] * R[0][j] + dR[i][1] * R[1][j] + dR[i][2] * R[2][j];
        pose[4 * i + 3] = dR[i][0] * rel[0] + dR[i][1] * rel[1] + dR[i][2] * rel[2] + c[i] + xi[3 + i];
    }
}

// Adam step on the twist g (about pivot c) and the pose update, serially;
// st[12] counts the steps taken
__device__ void adam_exp_update(double *pose, double *st, const double *g, const double *c, int k, int iters,
                                float lr_rot, float lr_trans, float b1f, float b2f, float epsf, float lr_final)
{
    const double t = st[12] + 1.0;
    double xi[6];
    for (int i = 0; i < 6; ++i)
        xi[i] = adam_component(st, i, g[i], t, k, iters, lr_rot, lr_trans, b1f, b2f, epsf, lr_final);
    st[12] = t;
    exp_update(pose, xi, c);
}

// pivot = R mu_bar + t (world) and its camera-frame image for keyframe d
__device__ void pivots_of(const VpDesc &d, const double *pose, const double *mbar, double *piv, double *ccam)
{
    for (int i = 0; i < 3; ++i)
        piv[i] = pose[4 * i] * mbar[0] + pose[4 * i + 1] * mbar[1] + pose[4 * i + 2] * mbar[2] + pose[4 * i + 3];
    for (int i = 0; i < 3; ++i)
        ccam[i] = (double)d.w2c[4 * i] * piv[0] + (double)d.w2c[4 * i + 1] * piv[1] + (double)d.w2c[4 * i + 2] * piv[2] +
                  (double)d.w2c[4 * i + 3];
}

// mean of each Gaussian set's means (one 1024-thread block per set): FP32
// TwoSum pairs per thread (two interleaved chains), TwoSum butterflies and a
// fixed-order TwoSum of the warps, one FP64 division (FP64 sums over 10^5
// means were latency-bound on the slow FP64 pipe)
constexpr int kCentroidThreads = 1024;

__global__ void __launch_bounds__(kCentroidThreads) k_centroid(const VpDesc *vps, const int *set_vp, double *centroid)
{
    __shared__ float s[kCentroidThreads / 32][3][2];
    const VpDesc &d = vps[set_vp[blockIdx.x]];
    float hs[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}}, ls[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    int i = threadIdx.x;
    for (; i + kCentroidThreads < d.n; i += 2 * kCentroidThreads) {
        const float4 m0 = d.means[i], m1 = d.means[i + kCentroidThreads];
        two_sum_add(hs[0][0], ls[0][0], m0.x, 0.0f);
        two_sum_add(hs[0][1], ls[0][1], m0.y, 0.0f);
        two_sum_add(hs[0][2], ls[0][2], m0.z, 0.0f);
        two_sum_add(hs[1][0], ls[1][0], m1.x, 0.0f);
        two_sum_add(hs[1][1], ls[1][1], m1.y, 0.0f);
        two_sum_add(hs[1][2], ls[1][2], m1.z, 0.0f);
    }
    if (i < d.n) {
        const float4 m0 = d.means[i];
        two_sum_add(hs[0][0], ls[0][0], m0.x, 0.0f);
        two_sum_add(hs[0][1], ls[0][1], m0.y, 0.0f);
        two_sum_add(hs[0][2], ls[0][2], m0.z, 0.0f);
    }
    for (int k = 0; k < 3; ++k) {
        float h = hs[0][k], l = ls[0][k];
        two_sum_add(h, l, hs[1][k], ls[1][k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, h, o), bl = __shfl_xor_sync(0xffffffffu, l, o);
            two_sum_add(h, l, bh, bl);
        }
        if ((threadIdx.x & 31) == 0) {
            s[threadIdx.x >> 5][k][0] = h;
            s[threadIdx.x >> 5][k][1] = l;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float h = s[0][threadIdx.x][0], l = s[0][threadIdx.x][1];
        for (int w = 1; w < kCentroidThreads / 32; ++w)
            two_sum_add(h, l, s[w][threadIdx.x][0], s[w][threadIdx.x][1]);
        centroid[3 * blockIdx.x + threadIdx.x] = d.n > 0 ? ((double)h + (double)l) / d.n : 0.0;
    }
}

__global__ void k_pose_init(const gsl::PoseArgs a)
{
    const int vp = blockIdx.x * blockDim.x + threadIdx.x;
    if (vp >= a.n_vps)
        return;
    const VpDesc &d = a.vps[vp];
    double *P = a.pose64 + 12 * vp;
    for (int k = 0; k < 12; ++k) {
        P[k] = (k % 5 == 0) ? 1.0 : 0.0;
        a.pose32[12 * vp + k] = (float)P[k];
    }
    for (int k = 0; k < 13; ++k)
        a.adam[13 * vp + k] = 0.0;
    pivots_of(d, P, a.centroid + 3 * d.set, a.pivot + 3 * vp, a.c_cam + 3 * vp);
    if (a.expo) {
        for (int k = 0; k < 7; ++k)
            a.expo[7 * vp + k] = 0.0;
        a.expo32[2 * vp] = 1.0f;
        a.expo32[2 * vp + 1] = 0.0f;
    }
}

// Adam step on the exposure (a, b) with the pose's moments and schedule
// (iteration k of iters); e = a, b, m_a, m_b, v_a, v_b, steps taken
__device__ void exposure_step(double *e, const double *g, int k, int iters, float lr, float b1f, float b2f, float epsf,
                              float lr_final)
{
    const double kPi = 3.14159265358979323846;
    const double b1 = b1f, b2 = b2f, eps = epsf, f = lr_final;
    const double t = e[6] + 1.0;
    e[6] = t;
    const double sched = f + (1.0 - f) * 0.5 * (1.0 + cos(kPi * (double)k / (double)iters));
    for (int i = 0; i < 2; ++i) {
        e[2 + i] = b1 * e[2 + i] + (1.0 - b1) * g[i];
        e[4 + i] = b2 * e[4 + i] + (1.0 - b2) * g[i] * g[i];
        const double mh = e[2 + i] / (1.0 - pow(b1, t));
        const double vh = e[4 + i] / (1.0 - pow(b2, t));
        e[i] -= (double)lr * sched * mh / (sqrt(vh) + eps);
    }
}

// 1024 threads per block: a keyframe's 3,225 tile pairs (1200x680) are
// about three loads deep per thread (256 threads waited on thirteen).
constexpr int kPoseThreads = 1024, kPoseWarps = kPoseThreads / 32;

// one block per keyframe: reduce the tile twists and losses in a fixed
// order, rotate the twist to the world frame, then (update) take the step.
// The step's FP64 work runs on warp 0: Adam on the six twist components in
// parallel (one lane each -- serially, their pow/sqrt chains dominated the
// update, the FP64 pipe being a small fraction of the FP32 one), then the
// exponential-map update, the exposure step and the pivots on lane 0.
__global__ void __launch_bounds__(kPoseThreads) k_pose_update(const gsl::PoseArgs a)
{
    __shared__ float s[kPoseWarps][9][2];
    __shared__ double s_tot[9], s_g[6], s_xi[6];
    const int vp = blockIdx.x;
    const VpDesc &d = a.vps[vp];
    const uint32_t nt = (uint32_t)d.TX * d.TY;
    const bool expo = d.exposure && a.tile_expo && a.expo;
    // (hi, lo) FP32 pairs summed by TwoSum in a fixed order (per thread,
    // then butterflies, then the warps); one FP64 value per component
    float hs[9], ls[9];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        hs[i] = ls[i] = 0.0f;
#pragma unroll 4
    for (uint32_t k = threadIdx.x; k < nt; k += blockDim.x) {
        const size_t t = d.tile_base + k;
        if (a.tile_twist)
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const float2 v = a.tile_twist[t * 6 + i];
                two_sum_add(hs[i], ls[i], v.x, v.y);
            }
        two_sum_add(hs[6], ls[6], a.tile_loss[t], 0.0f);
        if (expo) {
            two_sum_add(hs[7], ls[7], a.tile_expo[2 * t], 0.0f);
            two_sum_add(hs[8], ls[8], a.tile_expo[2 * t + 1], 0.0f);
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, hs[i], o), bl = __shfl_xor_sync(0xffffffffu, ls[i], o);
            two_sum_add(hs[i], ls[i], bh, bl);
        }
        if ((threadIdx.x & 31) == 0) {
            s[threadIdx.x >> 5][i][0] = hs[i];
            s[threadIdx.x >> 5][i][1] = ls[i];
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32)
        return;
    const int lane = threadIdx.x;
    if (lane < 9) {
        float h = s[0][lane][0], l = s[0][lane][1];
        for (int w = 1; w < kPoseWarps; ++w)
            two_sum_add(h, l, s[w][lane][0], s[w][lane][1]);
        s_tot[lane] = (double)h + (double)l;
    }
    __syncwarp();
    double tot[9];
    for (int i = 0; i < 9; ++i)
        tot[i] = s_tot[i];
    if (lane == 0)
        a.loss[vp] = tot[6];
    if (!a.tile_twist)
        return;
    // camera frame -> world frame: w = Rv^T w_c, v = Rv^T v_c
    if (lane < 6) {
        const int r = lane % 3, o = lane < 3 ? 0 : 3;
        const double gi =
            (double)d.w2c[r] * tot[o] + (double)d.w2c[4 + r] * tot[o + 1] + (double)d.w2c[8 + r] * tot[o + 2];
        s_g[lane] = gi;
        if (a.grad)
            a.grad[6 * vp + lane] = gi;
    }
    if (!a.update)
        return;  // (pose and optimiser state may be absent: gradient-only callers)
    const int iters = d.iters > 0 ? d.iters : a.iters;
    double *st = a.adam + 13 * vp;
    const int k = (int)st[12];
    if (k >= iters)
        return;
    const double t = st[12] + 1.0;
    if (lane < 6)
        s_xi[lane] = adam_component(st, lane, s_g[lane], t, k, iters, d.lr_rot, d.lr_trans, a.beta1, a.beta2,
                                    a.eps, a.lr_final);
    __syncwarp();
    if (lane != 0)
        return;
    st[12] = t;
    double *P = a.pose64 + 12 * vp;
    exp_update(P, s_xi, a.pivot + 3 * vp);
    if (expo) {
        double *e = a.expo + 7 * vp;
        exposure_step(e, tot + 7, k, iters, d.lr_exposure, a.beta1, a.beta2, a.eps, a.lr_final);
        a.expo32[2 * vp] = (float)exp(e[0]);
        a.expo32[2 * vp + 1] = (float)e[1];
    }
    for (int q = 0; q < 12; ++q)
        a.pose32[12 * vp + q] = (float)P[q];
    pivots_of(d, P, a.centroid + 3 * d.set, a.pivot + 3 * vp, a.c_cam + 3 * vp);
}

__global__ void k_expo32(const double *expo, float *expo32, int n)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        expo32[2 * v] = (float)exp(expo[7 * v]);
        expo32[2 * v + 1] = (float)expo[7 * v + 1];
    }
}

__global__ void k_pose_step(int n, double *pose, double *state, const double *grad, const double *pivot, int k,
                            int iters, float lr_rot, float lr_trans, float b1, float b2, float eps, float lr_final)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    adam_exp_update(pose + 12 * i, state + 13 * i, grad + 6 * i, pivot + 3 * i, k, iters, lr_rot, lr_trans, b1, b2,
                    eps, lr_final);
}

// ---------------------------------------------------------------- fusion
__device__ void jacobi4(double A[4][4], double V[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q)
                off += A[p][q] * A[p][q];
        if (off < 1e-60)
            break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (fabs(A[p][q]) < 1e-300)
                    continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < 4; ++k) {  // A <- J^T A J
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
}

// T^-1 of a 3x4 rigid map
__device__ void rigid_inverse(const double *T, double *Ti)
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            Ti[4 * i + j] = T[4 * j + i];
        Ti[4 * i + 3] = -(T[i] * T[3] + T[4 + i] * T[7] + T[8 + i] * T[11]);
    }
}

// one thread per problem: weighted chordal L2 mean of the rotations (the
// quaternion maximising tr(R^T sum w_i R_i), i.e. the top eigenvector of
// Horn's symmetric 4x4 matrix) and weighted mean of the translations
__global__ void k_fuse(const gsl::FuseArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_problems)
        return;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, ts[3] = {0, 0, 0}, wsum = 0.0;
    const int first = a.prob_first[p], count = a.prob_count[p];
    for (int e = first; e < first + count; ++e) {
        double T[12];
        const double *src = a.pose64 + 12 * e;
        if (a.reverse[e])
            rigid_inverse(src, T);
        else
            for (int k = 0; k < 12; ++k)
                T[k] = src[k];
        if (a.est_out)
            for (int k = 0; k < 12; ++k)
                a.est_out[12 * e + k] = T[k];
        const double w = 1.0 / fmax(a.eps[e], 1e-12);
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j)
                M[i][j] += w * T[4 * i + j];
            ts[i] += w * T[4 * i + 3];
        }
        wsum += w;
    }
    double K[4][4] = {
        {M[0][0] + M[1][1] + M[2][2], M[2][1] - M[1][2], M[0][2] - M[2][0], M[1][0] - M[0][1]},
        {M[2][1] - M[1][2], M[0][0] - M[1][1] - M[2][2], M[0][1] + M[1][0], M[0][2] + M[2][0]},
        {M[0][2] - M[2][0], M[0][1] + M[1][0], -M[0][0] + M[1][1] - M[2][2], M[1][2] + M[2][1]},
        {M[1][0] - M[0][1], M[0][2] + M[2][0], M[1][2] + M[2][1], -M[0][0] - M[1][1] + M[2][2]}};
    double V[4][4];
    jacobi4(K, V);
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (K[i][i] > K[best][best])
            best = i;
    double w = V[0][best], x = V[1][best], y = V[2][best], z = V[3][best];
    const double nq = sqrt(w * w + x * x + y * y + z * z);
    w /= nq; x /= nq; y /= nq; z /= nq;
    double *T = a.T_out + 12 * p;
    T[0] = 1 - 2 * (y * y + z * z); T[1] = 2 * (x * y - w * z); T[2] = 2 * (x * z + w * y);
    T[4] = 2 * (x * y + w * z); T[5] = 1 - 2 * (x * x + z * z); T[6] = 2 * (y * z - w * x);
    T[8] = 2 * (x * z - w * y); T[9] = 2 * (y * z + w * x); T[10] = 1 - 2 * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        T[4 * i + 3] = wsum > 0 ? ts[i] / wsum : 0.0;
    a.conf[p] = count > 0 ? wsum / count : 0.0;
}

// ---------------------------------------------------------------- loss
__global__ void __launch_bounds__(256) k_loss_tiles(const VpDesc *vps, const uint32_t *tile_vp, const float *rgb,
                                                    const float *depth, float *d_rgb, float *d_depth,
                                                    float *tile_loss)
{
    __shared__ float s_red[8];
    const uint32_t t = blockIdx.x;
    const VpDesc &d = vps[tile_vp[t]];
    const uint32_t lt = t - d.tile_base;
    const int px = (int)(lt % (uint32_t)d.TX) * kTile + (threadIdx.x & 15);
    const int py = (int)(lt / (uint32_t)d.TX) * kTile + (threadIdx.x >> 4);
    float l = 0.0f;
    if (px < d.W && py < d.H) {
        const int64_t HW = (int64_t)d.W * d.H, off = (int64_t)py * d.W + px;
        const float inv3 = d.inv3hw, inv1 = d.invhw;
        auto sg = [](float e) -> float { return e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f); };
        for (int ch = 0; ch < 3; ++ch) {
            const float e = rgb[3 * d.pix_base + ch * HW + off] - d.t_rgb[ch * HW + off];
            l += fabsf(e) * inv3;
            if (d_rgb)
                d_rgb[3 * d.pix_base + ch * HW + off] = sg(e) * inv3;
        }
        const float e = depth[d.pix_base + off] - d.t_depth[off];
        l += fabsf(e) * inv1;
        if (d_depth)
            d_depth[d.pix_base + off] = sg(e) * inv1;
    }
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w)
            s += s_red[w];
        tile_loss[t] = s;
    }
}

// ---------------------------------------------------------------- Eq. 8/9
struct Rigid {
    double T[12];
};

// mu <- R mu + t and q <- q_R (x) q of one Gaussian (FP64 arithmetic)
__device__ __forceinline__ void rigid_apply(const double *T, const float4 m, const float4 q, float4 &om, float4 &oq)
{
    // quaternion of R (largest-pivot branch), w >= 0
    const double tr = T[0] + T[5] + T[10];
    double qw, qx, qy, qz;
    if (tr > 0) {
        const double s = sqrt(tr + 1.0) * 2;
        qw = 0.25 * s; qx = (T[9] - T[6]) / s; qy = (T[2] - T[8]) / s; qz = (T[4] - T[1]) / s;
    } else if (T[0] > T[5] && T[0] > T[10]) {
        const double s = sqrt(1.0 + T[0] - T[5] - T[10]) * 2;
        qw = (T[9] - T[6]) / s; qx = 0.25 * s; qy = (T[1] + T[4]) / s; qz = (T[2] + T[8]) / s;
    } else if (T[5] > T[10]) {
        const double s = sqrt(1.0 + T[5] - T[0] - T[10]) * 2;
        qw = (T[2] - T[8]) / s; qx = (T[1] + T[4]) / s; qy = 0.25 * s; qz = (T[6] + T[9]) / s;
    } else {
        const double s = sqrt(1.0 + T[10] - T[0] - T[5]) * 2;
        qw = (T[4] - T[1]) / s; qx = (T[2] + T[8]) / s; qy = (T[6] + T[9]) / s; qz = 0.25 * s;
    }
    float4 r;
    r.x = (float)(T[0] * m.x + T[1] * m.y + T[2] * m.z + T[3]);
    r.y = (float)(T[4] * m.x + T[5] * m.y + T[6] * m.z + T[7]);
    r.z = (float)(T[8] * m.x + T[9] * m.y + T[10] * m.z + T[11]);
    r.w = 0.0f;
    // q_R (x) q
    float4 p;
    p.x = (float)(qw * q.x - qx * q.y - qy * q.z - qz * q.w);
    p.y = (float)(qw * q.y + qx * q.x + qy * q.w - qz * q.z);
    p.z = (float)(qw * q.z - qx * q.w + qy * q.x + qz * q.y);
    p.w = (float)(qw * q.w + qx * q.z - qy * q.y + qz * q.x);
    om = r;
    oq = p;
}

__global__ void k_transform(const float4 *means, const float4 *quats, int64_t n, const Rigid rt, float4 *om,
                            float4 *oq)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float4 a, b;
    rigid_apply(rt.T, means[i], quats[i], a, b);
    om[i] = a;
    oq[i] = b;
}

// many submaps, each with its own T: blocks [blk_base, next blk_base) of map k
__global__ void k_transform_batch(const gsl::MapDesc *maps, int n_maps)
{
    int lo = 0, hi = n_maps - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (maps[mid].blk_base <= blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const gsl::MapDesc &m = maps[lo];
    const int64_t i = (int64_t)(blockIdx.x - m.blk_base) * blockDim.x + threadIdx.x;
    if (i >= m.n)
        return;
    float4 a, b;
    rigid_apply(m.T, m.means[i], m.quats[i], a, b);
    m.out_means[i] = a;
    m.out_quats[i] = b;
}

}  // namespace

namespace gsl {

void centroids(const VpDesc *vps, const int *set_vp, int n_sets, double *centroid, cudaStream_t s)
{
    if (n_sets > 0) {
        k_centroid<<<n_sets, kCentroidThreads, 0, s>>>(vps, set_vp, centroid);
        ++g_launches;
    }
}

void pose_init(const PoseArgs &a, cudaStream_t s)
{
    if (a.n_vps > 0) {
        k_pose_init<<<(a.n_vps + 127) / 128, 128, 0, s>>>(a);
        ++g_launches;
    }
}

void pose_update(const PoseArgs &a, cudaStream_t s)
{
    if (a.n_vps > 0) {
        k_pose_update<<<a.n_vps, kPoseThreads, 0, s>>>(a);
        ++g_launches;
    }
}

void pose_step_raw(int n, double *pose, double *state, const double *grad, const double *pivot, int k, int iters,
                   float lr_rot, float lr_trans, float b1, float b2, float eps, float lr_final, cudaStream_t s)
{
    if (n > 0) {
        k_pose_step<<<(n + 127) / 128, 128, 0, s>>>(n, pose, state, grad, pivot, k, iters, lr_rot, lr_trans, b1, b2,
                                                    eps, lr_final);
        ++g_launches;
    }
}

void fuse(const FuseArgs &a, cudaStream_t s)
{
    if (a.n_problems > 0) {
        k_fuse<<<(a.n_problems + 63) / 64, 64, 0, s>>>(a);
        ++g_launches;
    }
}

void loss(const VpDesc *vps, int n_vps, uint32_t n_tiles, const uint32_t *tile_vp, const float *rgb,
          const float *depth, double *loss_out, float *d_rgb, float *d_depth, float *tile_loss, cudaStream_t s)
{
    if (n_tiles == 0)
        return;
    k_loss_tiles<<<n_tiles, 256, 0, s>>>(vps, tile_vp, rgb, depth, d_rgb, d_depth, tile_loss);
    PoseArgs a{};
    a.vps = vps;
    a.n_vps = n_vps;
    a.tile_loss = tile_loss;
    a.loss = loss_out;
    k_pose_update<<<n_vps, kPoseThreads, 0, s>>>(a);
    g_launches += 2;
}

void exposure_floats(const double *expo, float *expo32, int n_vps, cudaStream_t s)
{
    if (n_vps <= 0)
        return;
    k_expo32<<<(n_vps + 127) / 128, 128, 0, s>>>(expo, expo32, n_vps);
    ++g_launches;
}

void loss_reduce(const VpDesc *vps, int n_vps, const float *tile_loss, double *loss_out, cudaStream_t s)
{
    if (n_vps <= 0)
        return;
    PoseArgs a{};
    a.vps = vps;
    a.n_vps = n_vps;
    a.tile_loss = tile_loss;
    a.loss = loss_out;
    k_pose_update<<<n_vps, kPoseThreads, 0, s>>>(a);
    ++g_launches;
}

void transform(const float4 *means, const float4 *quats, int64_t n, const double *T, float4 *out_means,
               float4 *out_quats, cudaStream_t s)
{
    if (n <= 0)
        return;
    Rigid r;
    for (int k = 0; k < 12; ++k)
        r.T[k] = T[k];
    k_transform<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(means, quats, n, r, out_means, out_quats);
    ++g_launches;
}

void transform_batch(const MapDesc *maps, int n_maps, unsigned blocks, cudaStream_t s)
{
    if (n_maps <= 0 || blocks == 0)
        return;
    k_transform_batch<<<blocks, 256, 0, s>>>(maps, n_maps);
    ++g_launches;
}

}  // namespace gsl
