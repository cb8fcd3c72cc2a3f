// overlap.cu -- the overlap ratio of two submaps under an estimated
// T_{P->Q} (the supplement's loop filter): P's means are moved by T, each
// moved mean finds its closest mean of Q and each mean of Q its closest
// moved mean of P (exact nearest neighbours: FP32 squared distances
// dx = b - a per axis, fma(dz, dz, fma(dy, dy, dx * dx)), ties to the
// smaller index), the reciprocal pairs form the putative correspondences K,
// and OR = |{(p, q) in K : |T p - q|^2 < tau^2}| / |K|.
//
// k_nn is a brute-force sweep: targets staged through shared memory 2048 at
// a time (one broadcast load per target per warp), four queries per thread;
// FP32-ALU bound at ~9 operations per (query, target) pair.
#include "gs_internal.cuh"

namespace {

constexpr int kNNThreads = 256;
constexpr int kNNQ = 4;        // queries per thread
constexpr int kNNChunk = 2048; // targets per shared-memory stage (32 KB)

__global__ void k_rigid32(const float4 *p, int n, const float *T, float4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 v = p[i];
    float r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        r[k] = __fmaf_rn(T[4 * k + 2], v.z, __fmaf_rn(T[4 * k + 1], v.y, __fmaf_rn(T[4 * k], v.x, T[4 * k + 3])));
    out[i] = make_float4(r[0], r[1], r[2], 0.0f);
}

__global__ void __launch_bounds__(kNNThreads) k_nn(const float4 *A, int na, const float4 *B, int nb, int32_t *nn,
                                                   float *d2)
{
    __shared__ float4 sb[kNNChunk];
    const int base = blockIdx.x * kNNThreads * kNNQ + threadIdx.x;
    float ax[kNNQ], ay[kNNQ], az[kNNQ], best[kNNQ];
    int bi[kNNQ];
#pragma unroll
    for (int q = 0; q < kNNQ; ++q) {
        const int i = base + q * kNNThreads;
        const float4 a = i < na ? A[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        ax[q] = a.x;
        ay[q] = a.y;
        az[q] = a.z;
        best[q] = __int_as_float(0x7f800000);
        bi[q] = -1;
    }
    for (int c0 = 0; c0 < nb; c0 += kNNChunk) {
        const int cnt = min(kNNChunk, nb - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNNThreads)
            sb[k] = B[c0 + k];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float4 b = sb[j];
#pragma unroll
            for (int q = 0; q < kNNQ; ++q) {
                const float dx = __fsub_rn(b.x, ax[q]), dy = __fsub_rn(b.y, ay[q]), dz = __fsub_rn(b.z, az[q]);
                const float d = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                if (d < best[q]) {  // strict: the first (smallest) index keeps a tie
                    best[q] = d;
                    bi[q] = c0 + j;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kNNQ; ++q) {
        const int i = base + q * kNNThreads;
        if (i < na) {
            nn[i] = bi[q];
            if (d2)
                d2[i] = best[q];
        }
    }
}

// |K| and the pairs of K within tau (counts[0], counts[1])
__global__ void k_reciprocal(const int32_t *nn_pq, const float *d2, int np, const int32_t *nn_qp, float tau2,
                             unsigned long long *counts)
{
    __shared__ unsigned s_k[8], s_in[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned k = 0, in = 0;
    if (i < np) {
        const int32_t j = nn_pq[i];
        if (j >= 0 && nn_qp[j] == i) {
            k = 1;
            in = d2[i] < tau2 ? 1u : 0u;
        }
    }
    k = __reduce_add_sync(0xffffffffu, k);
    in = __reduce_add_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0) {
        s_k[threadIdx.x >> 5] = k;
        s_in[threadIdx.x >> 5] = in;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_k[w];
            b += s_in[w];
        }
        if (a)
            atomicAdd(&counts[0], a);
        if (b)
            atomicAdd(&counts[1], b);
    }
}

inline unsigned div_up(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

namespace gsl {

void overlap(const OverlapArgs &a, cudaStream_t s)
{
    if (a.np > 0) {
        k_rigid32<<<div_up(a.np, 256), 256, 0, s>>>(a.p, a.np, a.T32, a.pt);
        k_nn<<<div_up(a.np, kNNThreads * kNNQ), kNNThreads, 0, s>>>(a.pt, a.np, a.q, a.nq, a.nn_pq, a.d2);
        g_launches += 2;
    }
    if (a.nq > 0) {
        k_nn<<<div_up(a.nq, kNNThreads * kNNQ), kNNThreads, 0, s>>>(a.q, a.nq, a.pt, a.np, a.nn_qp, nullptr);
        ++g_launches;
    }
    cudaMemsetAsync(a.counts, 0, 2 * sizeof(unsigned long long), s);
    if (a.np > 0) {
        k_reciprocal<<<div_up(a.np, 256), 256, 0, s>>>(a.nn_pq, a.d2, a.np, a.nn_qp, a.tau2, a.counts);
        ++g_launches;
    }
}

}  // namespace gsl
