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
//
// k_nn_grid searches a uniform grid over the targets instead: each query
// scans the shells of cells at Chebyshev distance r = 0, 1, 2, ... around
// its cell and stops after shell r once its best squared distance is below
// (r s - margin)^2 (1 - 1e-6): a target outside the searched block lies at
// least r s - margin away (cell boundaries are computed in FP32 within the
// box), and its FP32 squared distance exceeds the best, so the result is
// the brute-force argmin.  Queries that would need more than kNNMaxRing
// shells go to the brute-force sweep.
#include <algorithm>

#include "gs_internal.cuh"

namespace {

constexpr int kNNMaxRing = 6;

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

// brute-force nearest neighbours of the queries listed in list[0 .. *n_list)
__global__ void __launch_bounds__(kNNThreads) k_nn_list(const float4 *A, const int32_t *list,
                                                        const uint32_t *n_list, const float4 *B, int nb, int32_t *nn,
                                                        float *d2)
{
    __shared__ float4 sb[kNNChunk];
    const uint32_t nl = *n_list;
    const uint32_t base = blockIdx.x * kNNThreads * kNNQ;
    if (base >= nl)
        return;
    float ax[kNNQ], ay[kNNQ], az[kNNQ], best[kNNQ];
    int bi[kNNQ];
#pragma unroll
    for (int q = 0; q < kNNQ; ++q) {
        const uint32_t i = base + q * kNNThreads + threadIdx.x;
        const float4 a = i < nl ? A[list[i]] : make_float4(0.f, 0.f, 0.f, 0.f);
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
                if (d < best[q]) {
                    best[q] = d;
                    bi[q] = c0 + j;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kNNQ; ++q) {
        const uint32_t i = base + q * kNNThreads + threadIdx.x;
        if (i < nl) {
            nn[list[i]] = bi[q];
            if (d2)
                d2[list[i]] = best[q];
        }
    }
}

// float <-> order-preserving uint (for atomic min / max of floats)
__device__ __forceinline__ uint32_t f2o(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_bbox(const float4 *a, int na, const float4 *b, int nb, uint32_t *mm)
{
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += gridDim.x * blockDim.x) {
        const float4 v = i < na ? a[i] : b[i - na];
        const uint32_t c[3] = {f2o(v.x), f2o(v.y), f2o(v.z)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = min(lo[k], c[k]);
            hi[k] = max(hi[k], c[k]);
        }
    }
    // warp, then block (shared memory), then one atomic per block and bound
    // (an atomic per warp serialised ~10^4 of them on six addresses)
    __shared__ uint32_t s_mm[6][8];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
        hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
    }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            s_mm[k][threadIdx.x >> 5] = lo[k];
            s_mm[3 + k][threadIdx.x >> 5] = hi[k];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        uint32_t m = s_mm[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            m = k < 3 ? min(m, s_mm[k][w]) : max(m, s_mm[k][w]);
        if (k < 3)
            atomicMin(&mm[k], m);
        else
            atomicMax(&mm[k], m);
    }
}

__device__ __forceinline__ int cell_axis(float x, float o, float inv_s, int n)
{
    const float t = floorf(__fmul_rn(__fsub_rn(x, o), inv_s));
    return (int)fminf(fmaxf(t, 0.0f), (float)(n - 1));
}

__global__ void k_cell_count(const float4 *pts, int n, const gsl::NNGrid g, uint32_t *cell, uint32_t *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 p = pts[i];
    const uint32_t c = (uint32_t)cell_axis(p.x, g.ox, g.inv_s, g.nx) +
                       (uint32_t)g.nx * ((uint32_t)cell_axis(p.y, g.oy, g.inv_s, g.ny) +
                                         (uint32_t)g.ny * (uint32_t)cell_axis(p.z, g.oz, g.inv_s, g.nz));
    cell[i] = c;
    atomicAdd(&cnt[c], 1u);
}

// targets bucketed by cell (order within a cell arbitrary: ties are broken by index)
__global__ void k_cell_scatter(const float4 *pts, int n, const uint32_t *cell, uint32_t *cursor, float4 *spts,
                               int32_t *sidx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint32_t pos = atomicAdd(&cursor[cell[i]], 1u);
    spts[pos] = pts[i];
    sidx[pos] = i;
}

__global__ void __launch_bounds__(256) k_nn_grid(const float4 *A, int na, const int32_t *order, const gsl::NNGrid g,
                                                 const uint32_t *start, const float4 *spts, const int32_t *sidx,
                                                 int32_t *nn, float *d2, int32_t *list, uint32_t *n_list)
{
    // thread t takes query order[t] (the queries in cell order: neighbouring
    // lanes search the same cells) or query t
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na)
        return;
    const int i = order ? order[t] : t;
    const float4 a = A[i];
    const int cx = cell_axis(a.x, g.ox, g.inv_s, g.nx), cy = cell_axis(a.y, g.oy, g.inv_s, g.ny),
              cz = cell_axis(a.z, g.oz, g.inv_s, g.nz);
    float best = __int_as_float(0x7f800000);
    int bi = -1;
    auto scan_cell = [&](int x, int y, int z) {
        const uint32_t c = (uint32_t)x + (uint32_t)g.nx * ((uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
        for (uint32_t j = start[c]; j < start[c + 1]; ++j) {
            const float4 b = spts[j];
            const float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y), dz = __fsub_rn(b.z, a.z);
            const float d = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            const int idx = sidx[j];
            if (d < best || (d == best && idx < bi)) {
                best = d;
                bi = idx;
            }
        }
    };
    for (int r = 0;; ++r) {
        // the shell of cells at Chebyshev distance r (clipped to the grid)
        for (int dz = -r; dz <= r; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.nz)
                continue;
            const bool zface = (dz == -r || dz == r);
            for (int dy = -r; dy <= r; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.ny)
                    continue;
                const bool face = zface || dy == -r || dy == r;
                const int step = face ? 1 : 2 * r;  // inside the shell only dx = -r and +r
                for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
                    const int x = cx + dx;
                    if (x >= 0 && x < g.nx)
                        scan_cell(x, y, z);
                }
            }
        }
        const bool covered = cx - r <= 0 && cx + r >= g.nx - 1 && cy - r <= 0 && cy + r >= g.ny - 1 &&
                             cz - r <= 0 && cz + r >= g.nz - 1;
        const float lb = (float)r * g.s - g.margin;
        if (covered || (lb > 0.0f && best < lb * lb * (1.0f - 1e-6f)))
            break;
        if (r >= kNNMaxRing) {
            list[atomicAdd(n_list, 1u)] = i;  // far from every target: the brute-force sweep
            return;
        }
    }
    nn[i] = bi;
    if (d2)
        d2[i] = best;
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

void overlap_moved_bbox(const OverlapArgs &a, uint32_t *bbox, cudaStream_t s)
{
    static const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    cudaMemcpyAsync(bbox, init, sizeof init, cudaMemcpyHostToDevice, s);
    if (a.np > 0) {
        k_rigid32<<<div_up(a.np, 256), 256, 0, s>>>(a.p, a.np, a.T32, a.pt);
        ++g_launches;
    }
    if (a.np + a.nq > 0) {
        k_bbox<<<std::min<unsigned>(div_up(a.np + a.nq, 256), 2 * 152), 256, 0, s>>>(a.pt, a.np, a.q, a.nq, bbox);
        ++g_launches;
    }
}

void nn_grid_build(const float4 *B, int nb, const NNGrid &g, const NNScratch &sc, cudaStream_t s)
{
    const size_t cells = (size_t)g.nx * g.ny * g.nz;
    cudaMemsetAsync(sc.start, 0, sizeof(uint32_t) * (cells + 1), s);
    if (nb > 0) {
        k_cell_count<<<div_up(nb, 256), 256, 0, s>>>(B, nb, g, sc.cell, sc.start);
        ++g_launches;
    }
    scan_excl(sc.start, sc.start, cells + 1, sc.partials, nullptr, s);
    cudaMemcpyAsync(sc.cursor, sc.start, sizeof(uint32_t) * cells, cudaMemcpyDeviceToDevice, s);
    if (nb > 0) {
        k_cell_scatter<<<div_up(nb, 256), 256, 0, s>>>(B, nb, sc.cell, sc.cursor, sc.spts, sc.sidx);
        ++g_launches;
    }
}

void nn_grid_search(const float4 *A, int na, const int32_t *order, const float4 *B, int nb, const NNGrid &g,
                    const NNScratch &sc, int32_t *nn, float *d2, cudaStream_t s)
{
    if (na <= 0)
        return;
    cudaMemsetAsync(sc.n_list, 0, sizeof(uint32_t), s);
    k_nn_grid<<<div_up(na, 256), 256, 0, s>>>(A, na, order, g, sc.start, sc.spts, sc.sidx, nn, d2, sc.list,
                                             sc.n_list);
    k_nn_list<<<div_up(na, kNNThreads * kNNQ), kNNThreads, 0, s>>>(A, sc.list, sc.n_list, B, nb, nn, d2);
    g_launches += 2;
}

void overlap_count(const OverlapArgs &a, cudaStream_t s)
{
    cudaMemsetAsync(a.counts, 0, 2 * sizeof(unsigned long long), s);
    if (a.np > 0) {
        k_reciprocal<<<div_up(a.np, 256), 256, 0, s>>>(a.nn_pq, a.d2, a.np, a.nn_qp, a.tau2, a.counts);
        ++g_launches;
    }
}

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
