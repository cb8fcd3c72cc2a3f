// api.cu -- the C ABI of include/gsreg.h: context and scratch arena,
// argument checks, and the orchestration of the kernels behind each entry
// point, including the CUDA-graph-replayed registration loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "gs_internal.cuh"

namespace {

enum Slot {
    S_VPS, S_GROUPS, S_TILEVP, S_POSE32, S_REC, S_AUX, S_COUNTS, S_PARTIALS, S_NDUPS, S_K0, S_V0, S_V1,
    S_HIST, S_HISTP, S_RANGES, S_FLAGS, S_TF, S_LAST, S_CODE, S_TLOSS, S_TTWIST, S_POSE64, S_ADAM, S_PIVOT,
    S_CCAM, S_CENT, S_LOSS, S_SETVP, S_REV, S_PFIRST, S_PCOUNT, S_TOUT, S_CONF, S_EST, S_GRAD, S_DUPG,
    S_PAIRS, S_RK0, S_RK1, S_RP0, S_RP1, S_RRANGES, S_TERR, S_TCOL, S_TW,
    S_TMED, S_TNV, S_TVPS, S_EXPO, S_EXPO32, S_TEXPO, S_OPT, S_ONN1, S_ONN2, S_OD2, S_OT, S_OCNT, S_MAPS, S_OS, S_ORDER, S_ORDC, S_SK, S_SV, S_SN, S_OBOX, S_GCELL, S_GSTART, S_GCUR, S_GPART, S_GPTS, S_GIDX, S_GLIST, S_GNL, S_GCELL2, S_GSTART2, S_GCUR2, S_GPART2, S_GPTS2, S_GIDX2, S_GLIST2, S_GNL2, S_SEGZ, S_SEGCUR, S_SEGBIG, S_SEGLIST, S_PROBE, S_QUEUE, S_COUNT
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

constexpr int kPhases = 5;  // project, bin, forward, backward, update

}  // namespace

namespace gsl {
long long g_launches = 0;
}

struct gs_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    std::string err;
    Buf bufs[S_COUNT];
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    gs_stats_t stats{};
    cudaEvent_t tev[kPhases + 1] = {};  // phase boundaries recorded in the captured iteration
    std::vector<cudaEvent_t> pool;      // per-iteration copies of the boundaries
    // autotuner: tile schedule chosen per plan shape (tiles, keyframes, records)
    std::map<std::tuple<uint64_t, size_t, uint64_t>, int> schedule;
    int64_t tuned = 0;  // trial runs made
    // largest tile-duplicate count seen at the initial poses per plan shape
    // (sizes the lists of the asynchronous registration calls)
    std::map<std::tuple<uint64_t, size_t, uint64_t>, uint32_t> dups_seen;
};

namespace {

using gsk::GroupDesc;
using gsk::VpDesc;

gs_status_t fail(gs_ctx *c, gs_status_t st, const std::string &msg)
{
    if (c)
        c->err = msg;
    return st;
}

#define GS_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, GS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

#define GS_TRY(expr)                   \
    do {                               \
        gs_status_t s_ = (expr);       \
        if (s_ != GS_OK)               \
            return s_;                 \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

// scratch buffer of at least `bytes` for `slot` (grown, never shrunk)
gs_status_t ws(gs_ctx *ctx, int slot, size_t bytes, void **out)
{
    Buf &b = ctx->bufs[slot];
    if (bytes == 0)
        bytes = 16;
    if (b.bytes >= bytes) {
        *out = b.p;
        return GS_OK;
    }
    size_t want = ((bytes + bytes / 4) + 255) & ~(size_t)255;
    if (ctx->used - b.bytes + want > ctx->budget) {
        want = (bytes + 255) & ~(size_t)255;
        if (ctx->used - b.bytes + want > ctx->budget)
            return fail(ctx, GS_ERR_OOM, "scratch of " + std::to_string(bytes) + " bytes exceeds the context budget");
    }
    if (b.p) {
        cudaFree(b.p);  // synchronises the device: no kernel still uses it
        ctx->used -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(ctx, GS_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    b.bytes = want;
    ctx->used += want;
    *out = b.p;
    return GS_OK;
}

template <typename T>
gs_status_t wsT(gs_ctx *ctx, int slot, size_t count, T **out)
{
    void *p = nullptr;
    GS_TRY(ws(ctx, slot, count * sizeof(T), &p));
    *out = (T *)p;
    return GS_OK;
}

template <typename T>
gs_status_t upload(gs_ctx *ctx, int slot, const std::vector<T> &v, T **out, cudaStream_t s)
{
    GS_TRY(wsT(ctx, slot, v.size(), out));
    if (!v.empty())
        GS_CUDA(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return GS_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

gs_status_t check_gaussians(gs_ctx *ctx, const gs_gaussians_t *g, const char *what)
{
    if (!g)
        return fail(ctx, GS_ERR_INVALID_ARG, std::string(what) + ": null submap");
    if (g->n < 0 || g->n >= (int64_t)1 << 31)
        return fail(ctx, GS_ERR_INVALID_ARG, std::string(what) + ": n out of range");
    if (g->n == 0)
        return GS_OK;
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->rgb)
        return fail(ctx, GS_ERR_INVALID_ARG, std::string(what) + ": null array");
    if (!aligned16(g->means) || !aligned16(g->log_scales) || !aligned16(g->quats) || !aligned16(g->rgb))
        return fail(ctx, GS_ERR_INVALID_ARG, std::string(what) + ": float4 arrays must be 16-byte aligned");
    return GS_OK;
}

gs_status_t check_camera(gs_ctx *ctx, const gs_camera_t &c)
{
    if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768)
        return fail(ctx, GS_ERR_INVALID_ARG, "camera size out of range [1, 32768]");
    if (!(c.fx > 0) || !(c.fy > 0) || !std::isfinite(c.fx) || !std::isfinite(c.fy) || !std::isfinite(c.cx) ||
        !std::isfinite(c.cy))
        return fail(ctx, GS_ERR_INVALID_ARG, "camera intrinsics must be finite with fx, fy > 0");
    for (float v : c.world_to_cam)
        if (!std::isfinite(v))
            return fail(ctx, GS_ERR_INVALID_ARG, "camera extrinsics must be finite");
    return GS_OK;
}

gs_status_t check_options(gs_ctx *ctx, const gs_options_t *o)
{
    if (!o)
        return fail(ctx, GS_ERR_INVALID_ARG, "null options");
    if (o->tile != GS_TILE)
        return fail(ctx, GS_ERR_INVALID_ARG, "options.tile must be GS_TILE (16)");
    if (!(o->alpha_max > 0 && o->alpha_max <= 1) || !(o->alpha_min >= 0) || !(o->t_min >= 0) ||
        !(o->dilation >= 0) || !std::isfinite(o->z_near))
        return fail(ctx, GS_ERR_INVALID_ARG, "options out of range");
    if ((o->tracking_loss != 0 && o->tracking_loss != 1) || !(o->lambda_c >= 0 && o->lambda_c <= 1))
        return fail(ctx, GS_ERR_INVALID_ARG, "tracking_loss must be 0 or 1 and lambda_c in [0, 1]");
    if (o->tile_schedule < 0 || o->tile_schedule > 4)
        return fail(ctx, GS_ERR_INVALID_ARG, "tile_schedule must be 0 (autotune) or 1..4");
    if (o->tight_lists != 0 && o->tight_lists != 1)
        return fail(ctx, GS_ERR_INVALID_ARG, "tight_lists must be 0 or 1");
    if (!(o->list_headroom > 0.0f) || !(o->list_headroom <= 64.0f))
        return fail(ctx, GS_ERR_INVALID_ARG, "list_headroom must be in (0, 64]");
    if (o->fuse_compositing != 0 && o->fuse_compositing != 1)
        return fail(ctx, GS_ERR_INVALID_ARG, "fuse_compositing must be 0 or 1");
    if ((o->exposure != 0 && o->exposure != 1) || !(o->lr_exposure >= 0) || !std::isfinite(o->lr_exposure) ||
        (o->exposure && o->tracking_loss))
        return fail(ctx, GS_ERR_INVALID_ARG,
                    "exposure must be 0 or 1 with a finite lr_exposure >= 0, and applies to the registration loss only");
    return GS_OK;
}

// the tiles / records / pixels of a list of keyframes
struct Plan {
    std::vector<VpDesc> vps;
    std::vector<GroupDesc> groups;
    std::vector<uint32_t> tile_vp;
    std::vector<int> set_vp;  // a vp of each Gaussian set
    uint64_t n_records = 0, n_tiles = 0, n_diff = 0;
    int64_t n_pix = 0;
    uint32_t proj_blocks = 0;
};

void add_vp(Plan &P, const gs_gaussians_t *g, const gs_camera_t &c, int set, int problem, int reverse,
            const float *trgb, const float *tdepth)
{
    VpDesc d{};
    d.means = (const float4 *)g->means;
    d.scales = (const float4 *)g->log_scales;
    d.quats = (const float4 *)g->quats;
    d.rgb = (const float4 *)g->rgb;
    d.logits = g->opacity_logits;
    d.n = (int)g->n;
    d.W = c.width;
    d.H = c.height;
    d.TX = (c.width + GS_TILE - 1) / GS_TILE;
    d.TY = (c.height + GS_TILE - 1) / GS_TILE;
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    std::memcpy(d.w2c, c.world_to_cam, sizeof d.w2c);
    d.rec_base = (uint32_t)P.n_records;
    d.tile_base = (uint32_t)P.n_tiles;
    d.diff_base = (uint32_t)P.n_diff;
    d.pix_base = P.n_pix;
    // the loss means' FP32 factors, rounded as the kernels would round them
    const int64_t HW = (int64_t)c.width * c.height;
    d.inv3hw = 1.0f / (3.0f * (float)HW);
    d.invhw = 1.0f / (float)HW;
    d.t_rgb = trgb;
    d.t_depth = tdepth;
    d.set = set;
    d.problem = problem;
    d.reverse = reverse;
    const int vp = (int)P.vps.size();
    for (int k = 0; k < d.TX * d.TY; ++k)
        P.tile_vp.push_back((uint32_t)vp);
    P.n_records += (uint64_t)d.n;
    P.n_tiles += (uint64_t)d.TX * d.TY;
    P.n_diff += (uint64_t)(d.TX + 1) * (d.TY + 1);
    P.n_pix += (int64_t)c.width * c.height;
    if ((int)P.set_vp.size() <= set)
        P.set_vp.resize(set + 1, vp);
    P.vps.push_back(d);
}

// groups: runs of consecutive vps that share a Gaussian set, <= kMaxVpPerGroup
gs_status_t finalize(gs_ctx *ctx, Plan &P)
{
    if (P.n_records >= 0xffffffffull || P.n_tiles >= 0xffffffffull || P.n_diff >= 0xffffffffull)
        return fail(ctx, GS_ERR_INVALID_ARG, "too many records or tiles for 32-bit indices");
    P.groups.clear();
    uint32_t blocks = 0;
    for (int v = 0; v < (int)P.vps.size();) {
        int e = v + 1;
        while (e < (int)P.vps.size() && e - v < gsk::kMaxVpPerGroup && P.vps[e].means == P.vps[v].means &&
               P.vps[e].n == P.vps[v].n)
            ++e;
        GroupDesc G{};
        G.vp_first = v;
        G.vp_count = e - v;
        G.n = P.vps[v].n;
        G.blk_base = blocks;
        for (int k = v; k < e; ++k)
            P.vps[k].group = (int)P.groups.size();
        P.groups.push_back(G);
        blocks += (uint32_t)((G.n + 255) / 256);
        v = e;
    }
    P.proj_blocks = blocks;
    return GS_OK;
}

int tile_bits(uint64_t n_tiles)
{
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < n_tiles)
        ++b;
    return b;
}

float skip_threshold(const gs_options_t *o)
{
    // exponents below ln(alpha_min) - 0.05 cannot reach alpha_min (o <= 1):
    // skipping them without evaluating e^x leaves every decision unchanged
    return o->alpha_min > 0 ? logf(o->alpha_min) - 0.05f : -3.0e38f;
}

// device copies of a plan's tables
struct DevPlan {
    VpDesc *vps = nullptr;
    GroupDesc *groups = nullptr;
    uint32_t *tile_vp = nullptr;
    int *set_vp = nullptr;
};

gs_status_t upload_plan(gs_ctx *ctx, const Plan &P, DevPlan &D, cudaStream_t s)
{
    GS_TRY(upload(ctx, S_VPS, P.vps, &D.vps, s));
    GS_TRY(upload(ctx, S_GROUPS, P.groups, &D.groups, s));
    GS_TRY(upload(ctx, S_TILEVP, P.tile_vp, &D.tile_vp, s));
    GS_TRY(upload(ctx, S_SETVP, P.set_vp, &D.set_vp, s));
    return GS_OK;
}

// scratch of the projection + binning pipeline
struct Pipe {
    float4 *rec = nullptr, *aux = nullptr;
    int32_t *counts = nullptr;
    uint32_t *partials = nullptr, *ndups = nullptr;
    uint64_t *keys[2] = {nullptr, nullptr};
    uint32_t *vals[2] = {nullptr, nullptr};
    uint32_t *hist = nullptr, *histp = nullptr;
    uint2 *ranges = nullptr;
    int *flags = nullptr;
    uint32_t cap = 0;
    uint32_t *tkeys[2] = {nullptr, nullptr};
    uint64_t n_records = 0;
    // segmented build
    unsigned long long *seg_hdr = nullptr;
    uint32_t *seg_diff = nullptr, *seg_cursor = nullptr, *seg_big = nullptr;
    uint4 *seg_list = nullptr;
    size_t seg_zero = 0;
};

// Binning routes.  The context-based entry points and gs_bin use the
// segmented build (per-tile counts from difference grids of the records'
// tile rectangles, atomic placement, a sort of each short tile list): no
// global sort at all.  gs_render_noalloc keeps the one-stage route (one
// radix sort of 64-bit (tile, depth) keys), which needs less scratch; both
// yield the same lists, which the tests cross-check.

// scratch of the segmented build: cleared header + difference grids,
// visible-record list, cursors, long-list queue
gs_status_t alloc_seg(gs_ctx *ctx, const Plan &P, Pipe &p)
{
    const size_t T = P.n_tiles ? P.n_tiles : 1, R = P.n_records ? P.n_records : 1;
    p.seg_zero = gsl::seg_zero_bytes((int)P.vps.size(), P.n_diff);
    uint8_t *z = nullptr;
    GS_TRY(wsT(ctx, S_SEGZ, p.seg_zero, &z));
    p.seg_hdr = (unsigned long long *)z;
    p.seg_diff = (uint32_t *)(p.seg_hdr + 1 + P.vps.size());
    GS_TRY(wsT(ctx, S_SEGLIST, R, &p.seg_list));
    GS_TRY(wsT(ctx, S_SEGCUR, T, &p.seg_cursor));
    GS_TRY(wsT(ctx, S_SEGBIG, T, &p.seg_big));
    return GS_OK;
}

gs_status_t alloc_pipe(gs_ctx *ctx, const Plan &P, bool aux, Pipe &p)
{
    const size_t R = P.n_records ? P.n_records : 1;
    GS_TRY(wsT(ctx, S_REC, 3 * R, &p.rec));
    if (aux)
        GS_TRY(wsT(ctx, S_AUX, 2 * R, &p.aux));
    GS_TRY(wsT(ctx, S_COUNTS, R, &p.counts));
    GS_TRY(wsT(ctx, S_PARTIALS, gsl::scan_partials(R), &p.partials));
    GS_TRY(wsT(ctx, S_NDUPS, 4, &p.ndups));
    GS_TRY(wsT(ctx, S_RANGES, P.n_tiles ? P.n_tiles : 1, &p.ranges));
    GS_TRY(wsT(ctx, S_FLAGS, 4, &p.flags));
    GS_TRY(alloc_seg(ctx, P, p));
    p.n_records = R;
    return GS_OK;
}

gs_status_t alloc_sort(gs_ctx *ctx, uint64_t want, Pipe &p)
{
    if (want > 0xfff00000ull)
        return fail(ctx, GS_ERR_CAPACITY, "more than 2^32 tile duplicates");
    const uint32_t cap = (uint32_t)std::max<uint64_t>(want, 1024);
    GS_TRY(wsT(ctx, S_K0, cap, &p.tkeys[0]));
    GS_TRY(wsT(ctx, S_V0, cap, &p.vals[0]));
    GS_TRY(wsT(ctx, S_V1, cap, &p.vals[1]));
    const size_t hn = gsl::sort_hist_entries((uint32_t)std::max<uint64_t>(cap, p.n_records));
    GS_TRY(wsT(ctx, S_HIST, hn, &p.hist));
    GS_TRY(wsT(ctx, S_HISTP, gsl::scan_partials(hn), &p.histp));
    p.cap = cap;
    return GS_OK;
}

int run_bin(const gsl::BinArgs &b, cudaStream_t s) { return gsl::bin_seg(b, s); }

// counts = false: the per-record tile counts are not written (the
// segmented lists read the records' seg_list entries; only the scan for the
// duplicate total at the initial poses reads the counts)
gsl::ProjectArgs project_args(const Plan &P, const DevPlan &D, const Pipe &p, const float *pose32,
                              const gs_options_t *o, bool counts = true)
{
    gsl::ProjectArgs a{};
    a.vps = D.vps;
    a.groups = D.groups;
    a.n_groups = (int)P.groups.size();
    a.n_blocks = P.proj_blocks;
    a.pose32 = pose32;
    a.z_near = o->z_near;
    a.dilation = o->dilation;
    a.smooth = o->smooth;
    a.rec = p.rec;
    a.aux = p.aux;
    a.counts = counts ? p.counts : nullptr;
    a.flags = p.flags;
    // tight lists need a normal alpha_min (the contract's logarithm)
    a.tight = o->tight_lists != 0 && o->alpha_min >= FLT_MIN && !o->smooth;
    a.alpha_min = o->alpha_min;
    // the projection counts and lists for the segmented build (run_bin follows every projection here)
    a.seg_hdr = p.seg_hdr;
    a.seg_diff = p.seg_diff;
    a.seg_zero_bytes = p.seg_zero;
    a.seg_list = p.seg_list;
    return a;
}

gsl::BinArgs bin_args(const Plan &P, const DevPlan &D, const Pipe &p)
{
    gsl::BinArgs b{};
    b.vps = D.vps;
    b.n_vps = (int)P.vps.size();
    b.counts = p.counts;
    b.rec = p.rec;
    b.n_records = (uint32_t)P.n_records;
    b.partials = p.partials;
    b.n_dups = p.ndups;
    b.keys[0] = p.keys[0];
    b.keys[1] = p.keys[1];
    b.vals[0] = p.vals[0];
    b.vals[1] = p.vals[1];
    b.capacity = p.cap;
    b.hist = p.hist;
    b.hist_partials = p.histp;
    b.key_bits = 32 + tile_bits(P.n_tiles);
    b.ranges = p.ranges;
    b.n_tiles = (uint32_t)P.n_tiles;
    b.flags = p.flags;
    b.tkeys[0] = p.tkeys[0];
    b.seg_hdr = p.seg_hdr;
    b.seg_diff = p.seg_diff;
    b.seg_zero_bytes = p.seg_zero;
    b.seg_cursor = p.seg_cursor;
    b.seg_big = p.seg_big;
    b.seg_list = p.seg_list;
    b.seg_counted = 1;
    for (const VpDesc &d : P.vps)
        b.seg_max_cells = std::max(b.seg_max_cells, (uint32_t)(d.TX * d.TY));
    return b;
}

gsl::RasterArgs raster_args(const Plan &P, const DevPlan &D, const Pipe &p, int cur, const gs_options_t *o)
{
    gsl::RasterArgs r{};
    r.vps = D.vps;
    r.tile_vp = D.tile_vp;
    r.n_tiles = (uint32_t)P.n_tiles;
    r.ranges = p.ranges;
    r.vals = p.vals[cur];
    r.rec = p.rec;
    r.aux = p.aux;
    r.alpha_min = o->alpha_min;
    r.alpha_max = o->alpha_max;
    r.t_min = o->t_min;
    r.skip_below = skip_threshold(o);
    r.bg[0] = o->bg[0];
    r.bg[1] = o->bg[1];
    r.bg[2] = o->bg[2];
    return r;
}

// project + count duplicates (synchronises) + size the sort + emit/sort/range
gs_status_t project_and_bin(gs_ctx *ctx, const Plan &P, const DevPlan &D, Pipe &p, const float *pose32,
                            const gs_options_t *o, cudaStream_t s, int *cur, uint32_t *n_dups_out)
{
    GS_CUDA(cudaMemsetAsync(p.flags, 0, sizeof(int), s));
    gsl::project(project_args(P, D, p, pose32, o), s);
    gsl::BinArgs b = bin_args(P, D, p);
    gsl::bin_count(b, s);
    uint32_t nd = 0;
    GS_CUDA(cudaMemcpyAsync(&nd, p.ndups, sizeof nd, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (nd == 0xffffffffu)
        return fail(ctx, GS_ERR_CAPACITY, "more than 2^32 tile duplicates");
    if (p.cap < nd || !p.tkeys[0])
        GS_TRY(alloc_sort(ctx, nd, p));
    b = bin_args(P, D, p);
    *cur = run_bin(b, s);
    if (n_dups_out)
        *n_dups_out = nd;
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t read_flags(gs_ctx *ctx, const Pipe &p, cudaStream_t s, int *flags)
{
    GS_CUDA(cudaMemcpyAsync(flags, p.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    return GS_OK;
}

gs_status_t check_common(gs_ctx *ctx, const gs_gaussians_t *g, const gs_camera_t *cams, int n_cams,
                         const gs_options_t *o)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, o));
    GS_TRY(check_gaussians(ctx, g, "submap"));
    if (n_cams < 0 || (n_cams > 0 && !cams))
        return fail(ctx, GS_ERR_INVALID_ARG, "bad camera list");
    for (int c = 0; c < n_cams; ++c)
        GS_TRY(check_camera(ctx, cams[c]));
    return GS_OK;
}

Plan plan_for(const gs_gaussians_t *g, const gs_camera_t *cams, int n_cams)
{
    Plan P;
    for (int c = 0; c < n_cams; ++c)
        add_vp(P, g, cams[c], 0, 0, 0, nullptr, nullptr);
    return P;
}

// pivots (world, float [n][3]) -> camera frame for each vp
__global__ void k_cam_pivots(const VpDesc *vps, int n, const float *piv, double *ccam)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n)
        return;
    const VpDesc &d = vps[v];
    const double c[3] = {piv ? piv[3 * v] : 0.0, piv ? piv[3 * v + 1] : 0.0, piv ? piv[3 * v + 2] : 0.0};
    for (int i = 0; i < 3; ++i)
        ccam[3 * v + i] = (double)d.w2c[4 * i] * c[0] + (double)d.w2c[4 * i + 1] * c[1] +
                          (double)d.w2c[4 * i + 2] * c[2] + (double)d.w2c[4 * i + 3];
}

__global__ void k_to_float(const double *in, float *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = (float)in[i];
}

// FP32 peak probe: each thread runs 8 independent FMA chains for `iters`
// rounds (enough independent work per warp to hide the FMA latency), and
// writes one value so the chains are not removed.  PACKED: the chains are
// pairs (fma.rn.f32x2, two FMAs per instruction), as the compositing
// kernels issue them.
constexpr int kProbeChains = 8;
template <bool PACKED>
__global__ void __launch_bounds__(256) k_fma_probe(float *sink, int iters, float a, float b)
{
    float s = 0.0f;
    if constexpr (PACKED) {
        unsigned long long x[kProbeChains / 2], ab, bb;
        asm("mov.b64 %0, {%1, %1};" : "=l"(ab) : "f"(a));
        asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
#pragma unroll
        for (int k = 0; k < kProbeChains / 2; ++k)
            asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"((float)(threadIdx.x + 2 * k)), "f"((float)(threadIdx.x + 2 * k + 1)));
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains / 2; ++k)
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(ab), "l"(bb));
        }
#pragma unroll
        for (int k = 0; k < kProbeChains / 2; ++k) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
            s += lo + hi;
        }
    } else {
        float x[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k)
            x[k] = (float)(threadIdx.x + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k)
                x[k] = fmaf(x[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k)
            s += x[k];
    }
    if (s == 1.2345f)  // never true for the arguments used: keeps the store conditional
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The keyframe problems of one registration problem (Sec. 3.2): keyframes
// of P are localised in Q (Q moves; the estimate is inverted), keyframes of
// Q in P (P moves).  Each moving submap is one Gaussian set.
void add_problem(Plan &P, const gs_gaussians_t *src, const gs_gaussians_t *tgt, const gs_view_t *sv, int ns,
                 const gs_view_t *tv, int nt, int problem, int &sets, const gs_options_t *o)
{
    const size_t v0 = P.vps.size();
    if (ns > 0) {
        const int set = sets++;
        for (int k = 0; k < ns; ++k)
            add_vp(P, tgt, sv[k].cam, set, problem, 1, sv[k].rgb, sv[k].depth);
    }
    if (nt > 0) {
        const int set = sets++;
        for (int k = 0; k < nt; ++k)
            add_vp(P, src, tv[k].cam, set, problem, 0, tv[k].rgb, tv[k].depth);
    }
    for (size_t v = v0; v < P.vps.size(); ++v) {
        P.vps[v].lr_rot = o->lr_rot;
        P.vps[v].lr_trans = o->lr_trans;
        P.vps[v].loss_kind = o->tracking_loss ? 1 : 0;
        P.vps[v].lambda_c = o->lambda_c;
        P.vps[v].exposure = o->exposure ? 1 : 0;
        P.vps[v].lr_exposure = o->lr_exposure;
    }
}

bool any_exposure(const Plan &P)
{
    for (const VpDesc &d : P.vps)
        if (d.exposure)
            return true;
    return false;
}

// exposure state [vp][7] (FP64), gains / offsets [vp][2] and the forward's
// per-tile partial gradients [tiles][2]
gs_status_t alloc_exposure(gs_ctx *ctx, const Plan &P, gsl::PoseArgs &pa, gsl::RasterArgs &r)
{
    const size_t nv = std::max<size_t>(P.vps.size(), 1), ntl = (size_t)std::max<uint64_t>(P.n_tiles, 1);
    float *e32 = nullptr, *te = nullptr;
    GS_TRY(wsT(ctx, S_EXPO, 7 * nv, &pa.expo));
    GS_TRY(wsT(ctx, S_EXPO32, 2 * nv, &e32));
    GS_TRY(wsT(ctx, S_TEXPO, 2 * ntl, &te));
    pa.expo32 = e32;
    pa.tile_expo = te;
    r.expo32 = e32;
    r.tile_expo = te;
    return GS_OK;
}

// per-pixel and per-keyframe scratch of the tracking loss, if the plan has
// tracking keyframes (else ta.n_track = 0 and nothing is allocated)
gs_status_t alloc_track(gs_ctx *ctx, const Plan &P, const DevPlan &D, gsl::RasterArgs &r, gsl::TrackArgs &ta,
                        float *tloss, cudaStream_t s)
{
    ta = gsl::TrackArgs{};
    std::vector<int> tv;
    for (int v = 0; v < (int)P.vps.size(); ++v)
        if (P.vps[v].loss_kind == 1)
            tv.push_back(v);
    if (tv.empty())
        return GS_OK;
    const size_t npix = (size_t)std::max<int64_t>(P.n_pix, 1), nv = P.vps.size();
    int *tvd = nullptr;
    GS_TRY(wsT(ctx, S_TERR, npix, &r.trk_err));
    GS_TRY(wsT(ctx, S_TCOL, npix, &r.trk_col));
    float *w = nullptr;
    GS_TRY(wsT(ctx, S_TW, npix, &w));
    r.trk_w = w;
    GS_TRY(wsT(ctx, S_TMED, nv, &ta.med));
    GS_TRY(wsT(ctx, S_TNV, nv, &ta.n_valid));
    GS_TRY(upload(ctx, S_TVPS, tv, &tvd, s));
    ta.vps = D.vps;
    ta.tile_vp = D.tile_vp;
    ta.n_tiles = (uint32_t)P.n_tiles;
    ta.track_vps = tvd;
    ta.n_track = (int)tv.size();
    ta.t_final = r.t_final;
    ta.err = r.trk_err;
    ta.col = r.trk_col;
    ta.w = w;
    ta.tile_loss = tloss;
    return GS_OK;
}

gs_status_t check_views(gs_ctx *ctx, const gs_view_t *v, int n)
{
    if (n < 0 || (n > 0 && !v))
        return fail(ctx, GS_ERR_INVALID_ARG, "bad keyframe list");
    for (int k = 0; k < n; ++k) {
        GS_TRY(check_camera(ctx, v[k].cam));
        if (!v[k].rgb || !v[k].depth)
            return fail(ctx, GS_ERR_INVALID_ARG, "null keyframe image");
    }
    return GS_OK;
}

gs_status_t check_problem(gs_ctx *ctx, const gs_problem_t &q)
{
    GS_TRY(check_gaussians(ctx, &q.src, "src"));
    GS_TRY(check_gaussians(ctx, &q.tgt, "tgt"));
    if (q.n_src_views + q.n_tgt_views <= 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "a problem without keyframes");
    GS_TRY(check_views(ctx, q.src_views, q.n_src_views));
    GS_TRY(check_views(ctx, q.tgt_views, q.n_tgt_views));
    return GS_OK;
}

// device outputs of the asynchronous registration calls
struct AsyncOut {
    double *T = nullptr, *conf = nullptr, *eps = nullptr, *est = nullptr;
    int32_t *status = nullptr;
};

gs_status_t run_registration(gs_ctx *ctx, Plan &P, int n_problems, const gs_options_t *opt, int iters,
                             cudaStream_t s, double *T_out, double *conf_out, double *eps_out, double *est_out,
                             const AsyncOut *ao = nullptr, double *grad_out = nullptr);

}  // namespace

// ===========================================================================
// exported entry points
// ===========================================================================
extern "C" {

void gs_default_options(gs_options_t *o)
{
    if (!o)
        return;
    std::memset(o, 0, sizeof *o);
    o->tile = GS_TILE;
    o->z_near = 0.2f;
    o->dilation = 0.3f;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->t_min = 1e-4f;
    o->smooth = 0;
    o->lr_rot = 0.015f;
    o->lr_trans = 0.005f;
    o->beta1 = 0.8f;
    o->beta2 = 0.99f;
    o->adam_eps = 1e-8f;
    o->tracking_loss = 0;
    o->lambda_c = 0.6f;
    o->exposure = 0;
    o->lr_exposure = 0.1f;
    o->tile_schedule = 0;
    o->tight_lists = 1;
    o->list_headroom = 1.5f;
    o->fuse_compositing = 1;
    o->lr_final = 0.001f;
}

gs_status_t gs_ctx_create(int device, size_t budget, gs_ctx_t **out)
{
    if (!out)
        return GS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return GS_ERR_INVALID_ARG;
    }
    gs_ctx *ctx = new gs_ctx();
    ctx->device = device;
    ctx->budget = budget ? budget : ((size_t)16 << 30);
    DeviceGuard dg(device);
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return GS_ERR_CUDA;
    }
    gsl::raster_init();
    *out = ctx;
    return GS_OK;
}

gs_status_t gs_ctx_destroy(gs_ctx_t *ctx)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    for (Buf &b : ctx->bufs)
        if (b.p)
            cudaFree(b.p);
    for (cudaEvent_t e : ctx->tev)
        if (e)
            cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->pool)
        cudaEventDestroy(e);
    if (ctx->cap)
        cudaStreamDestroy(ctx->cap);
    delete ctx;
    return GS_OK;
}

const char *gs_last_error(const gs_ctx_t *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t gs_ctx_bytes(const gs_ctx_t *ctx) { return ctx ? ctx->used : 0; }

gs_status_t gs_ctx_stats(const gs_ctx_t *ctx, gs_stats_t *out)
{
    if (!ctx || !out)
        return GS_ERR_INVALID_ARG;
    *out = ctx->stats;
    return GS_OK;
}

int gs_abi_sizes(size_t *out, int n)
{
    const size_t s[7] = {sizeof(gs_gaussians_t), sizeof(gs_camera_t),  sizeof(gs_view_t),           sizeof(gs_options_t),
                         sizeof(gs_stats_t),     sizeof(gs_gaussian_grads_t), sizeof(gs_problem_t)};
    int k = 0;
    for (; out && k < n && k < 7; ++k)
        out[k] = s[k];
    return k;
}

gs_status_t gs_project(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams,
                       int n_cams, const gs_options_t *opt, float *records, float *aux, int32_t *counts,
                       gs_stream_t stream)
{
    GS_TRY(check_common(ctx, g, cams, n_cams, opt));
    if (!poses || !records || !counts || !aligned16(records) || (aux && !aligned16(aux)))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_project: null or unaligned output");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Plan P = plan_for(g, cams, n_cams);
    GS_TRY(finalize(ctx, P));
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    Pipe p;
    p.rec = (float4 *)records;
    p.aux = (float4 *)aux;
    p.counts = counts;
    GS_TRY(wsT(ctx, S_FLAGS, 4, &p.flags));
    GS_CUDA(cudaMemsetAsync(p.flags, 0, sizeof(int), s));
    gsl::project(project_args(P, D, p, poses, opt), s);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t gs_bin(gs_ctx_t *ctx, const float *records, const int32_t *counts, const gs_camera_t *cams,
                   int n_cams, int64_t n, uint64_t *keys, uint32_t *vals, int64_t capacity, uint32_t *ranges,
                   int64_t *n_dups, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (!records || !counts || !ranges || !n_dups || n < 0 || n_cams < 0 || (n_cams > 0 && !cams) ||
        capacity < 0 || !aligned16(records))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_bin: bad arguments");
    for (int c = 0; c < n_cams; ++c)
        GS_TRY(check_camera(ctx, cams[c]));
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gs_gaussians_t g{};
    g.n = n;
    Plan P = plan_for(&g, cams, n_cams);
    GS_TRY(finalize(ctx, P));
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    Pipe p;
    p.rec = (float4 *)records;
    p.counts = (int32_t *)counts;
    GS_TRY(wsT(ctx, S_PARTIALS, gsl::scan_partials(P.n_records ? P.n_records : 1), &p.partials));
    GS_TRY(wsT(ctx, S_NDUPS, 4, &p.ndups));
    GS_TRY(wsT(ctx, S_FLAGS, 4, &p.flags));
    GS_CUDA(cudaMemsetAsync(p.flags, 0, sizeof(int), s));
    p.ranges = (uint2 *)ranges;
    const size_t R = P.n_records ? P.n_records : 1;
    p.n_records = R;
    GS_TRY(alloc_seg(ctx, P, p));
    gsl::BinArgs b = bin_args(P, D, p);
    gsl::bin_count(b, s);
    uint32_t nd = 0;
    GS_CUDA(cudaMemcpyAsync(&nd, p.ndups, sizeof nd, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    *n_dups = nd;
    if ((int64_t)nd > capacity || nd == 0xffffffffu)
        return fail(ctx, GS_ERR_CAPACITY, "gs_bin: " + std::to_string(nd) + " duplicates exceed capacity");
    GS_TRY(alloc_sort(ctx, nd, p));
    b = bin_args(P, D, p);
    b.seg_counted = 0;  // the caller's records: collect them here
    const int cur = gsl::bin_seg(b, s);
    if (nd > 0) {
        gsl::seg_keys64(b, keys, s);
        GS_CUDA(cudaMemcpyAsync(vals, p.vals[cur], sizeof(uint32_t) * nd, cudaMemcpyDeviceToDevice, s));
    }
    GS_CUDA(cudaGetLastError());
    int flags = 0;
    GS_TRY(read_flags(ctx, p, s, &flags));
    if (flags & gsk::kFlagTimeout)
        return fail(ctx, GS_ERR_TIMEOUT, "a sort pass gave up waiting for an earlier tile");
    return GS_OK;
}

gs_status_t gs_render(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams,
                      int n_cams, const gs_options_t *opt, float *rgb, float *depth, float *alpha, float *t_final,
                      int32_t *last, gs_stream_t stream)
{
    GS_TRY(check_common(ctx, g, cams, n_cams, opt));
    if (!poses)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_render: null poses");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Plan P = plan_for(g, cams, n_cams);
    GS_TRY(finalize(ctx, P));
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    Pipe p;
    GS_TRY(alloc_pipe(ctx, P, false, p));
    int cur = 0;
    uint32_t nd = 0;
    const long long l0 = gsl::g_launches;
    GS_TRY(project_and_bin(ctx, P, D, p, poses, opt, s, &cur, &nd));
    gsl::RasterArgs r = raster_args(P, D, p, cur, opt);
    r.out_rgb = rgb;
    r.out_depth = depth;
    r.out_alpha = alpha;
    r.t_final = t_final;
    r.last = last;
    gsl::forward(r, false, s);
    GS_CUDA(cudaGetLastError());
    ctx->stats = gs_stats_t{};
    ctx->stats.kernel_launches = gsl::g_launches - l0;
    ctx->stats.n_dups = nd;
    ctx->stats.n_pixels = P.n_pix;
    int flags = 0;
    GS_TRY(read_flags(ctx, p, s, &flags));
    if (flags & gsk::kFlagNonFinite)
        return fail(ctx, GS_ERR_NONFINITE, "non-finite Gaussian parameter");
    if (flags & gsk::kFlagTimeout)
        return fail(ctx, GS_ERR_TIMEOUT, "a sort pass gave up waiting for an earlier tile");
    return GS_OK;
}

}  // extern "C"

namespace {

// The adjoint of one forward pass whose projection (p.rec, p.aux), tile
// lists (p.vals[cur], p.ranges, p.ndups, capacity p.cap) and per-pixel state
// (t_final, last) are in place: screen-space adjoint per tile, the pose
// twist per camera, and optionally every Gaussian parameter.
gs_status_t backward_core(gs_ctx *ctx, const Plan &P, const DevPlan &D, Pipe &p, int cur, const gs_gaussians_t *g,
                          const float *poses, const gs_options_t *opt, const float *t_final, const int32_t *last,
                          const float *d_rgb, const float *d_depth, const float *d_alpha, const float *pivots,
                          float *pose_grad, const gs_gaussian_grads_t *grads, bool full, cudaStream_t s)
{
    gsl::RasterArgs r = raster_args(P, D, p, cur, opt);
    r.t_final = (float *)t_final;
    r.last = (int32_t *)last;
    r.d_rgb = d_rgb;
    r.d_depth = d_depth;
    r.d_alpha = d_alpha;
    const int nv = (int)P.vps.size();
    double *ccam = nullptr, *grad = nullptr, *lossd = nullptr;
    float *tloss = nullptr;
    GS_TRY(wsT(ctx, S_CCAM, 3 * (size_t)std::max(nv, 1), &ccam));
    GS_TRY(wsT(ctx, S_GRAD, 6 * (size_t)std::max(nv, 1), &grad));
    GS_TRY(wsT(ctx, S_LOSS, (size_t)std::max(nv, 1), &lossd));
    GS_TRY(wsT(ctx, S_TTWIST, 6 * (size_t)std::max<uint64_t>(P.n_tiles, 1), &r.tile_twist));
    GS_TRY(wsT(ctx, S_TLOSS, (size_t)std::max<uint64_t>(P.n_tiles, 1), &tloss));
    GS_CUDA(cudaMemsetAsync(tloss, 0, sizeof(float) * std::max<uint64_t>(P.n_tiles, 1), s));
    if (nv > 0) {
        k_cam_pivots<<<(nv + 63) / 64, 64, 0, s>>>(D.vps, nv, pivots, ccam);
        ++gsl::g_launches;
    }
    r.c_cam = ccam;
    if (full)
        GS_TRY(wsT(ctx, S_DUPG, 10 * (size_t)p.cap, &r.dup_grads));
    gsl::backward(r, false, full, s);
    if (full) {
        // group the duplicates by record, then chain per Gaussian
        uint32_t *rk[2] = {nullptr, nullptr}, *rp[2] = {nullptr, nullptr};
        uint2 *rr = nullptr;
        GS_TRY(wsT(ctx, S_RK0, p.cap, &rk[0]));
        GS_TRY(wsT(ctx, S_RK1, p.cap, &rk[1]));
        GS_TRY(wsT(ctx, S_RP0, p.cap, &rp[0]));
        GS_TRY(wsT(ctx, S_RP1, p.cap, &rp[1]));
        GS_TRY(wsT(ctx, S_RRANGES, (size_t)std::max<uint64_t>(P.n_records, 1), &rr));
        gsl::ParamArgs pa{};
        pa.vps = D.vps;
        pa.n_vps = nv;
        pa.n = (int)g->n;
        pa.rec = p.rec;
        pa.aux = p.aux;
        pa.pose32 = poses;
        pa.dup_grads = r.dup_grads;
        pa.quats = (const float4 *)g->quats;
        pa.scales = (const float4 *)g->log_scales;
        pa.logits = g->opacity_logits;
        pa.g_means = grads->means;
        pa.g_scales = grads->log_scales;
        pa.g_quats = grads->quats;
        pa.g_logits = grads->opacity_logits;
        pa.g_rgb = grads->rgb;
        gsl::param_grads(pa, p.vals[cur], p.ndups, p.cap, rk, rp, tile_bits(P.n_records), p.hist, p.histp, rr,
                         (uint32_t)P.n_records, s);
    }
    gsl::PoseArgs a{};
    a.vps = D.vps;
    a.n_vps = nv;
    a.tile_twist = r.tile_twist;
    a.tile_loss = tloss;
    a.loss = lossd;
    a.grad = grad;
    a.update = 0;
    gsl::pose_update(a, s);
    if (pose_grad && nv > 0) {
        k_to_float<<<(6 * nv + 255) / 256, 256, 0, s>>>(grad, pose_grad, 6 * nv);
        ++gsl::g_launches;
    }
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

bool wants_params(const gs_gaussian_grads_t *grads)
{
    return grads && (grads->means || grads->log_scales || grads->quats || grads->opacity_logits || grads->rgb);
}

gs_status_t check_grads(gs_ctx *ctx, const gs_gaussian_grads_t *grads)
{
    if (wants_params(grads) &&
        ((grads->means && !aligned16(grads->means)) || (grads->log_scales && !aligned16(grads->log_scales)) ||
         (grads->quats && !aligned16(grads->quats)) || (grads->rgb && !aligned16(grads->rgb))))
        return fail(ctx, GS_ERR_INVALID_ARG, "gradient float4 arrays must be 16-byte aligned");
    return GS_OK;
}

}  // namespace

extern "C" {

gs_status_t gs_render_backward(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses,
                               const gs_camera_t *cams, int n_cams, const gs_options_t *opt,
                               const float *t_final, const int32_t *last, const float *d_rgb,
                               const float *d_depth, const float *d_alpha, const float *pivots, float *pose_grad,
                               const gs_gaussian_grads_t *grads, gs_stream_t stream)
{
    GS_TRY(check_common(ctx, g, cams, n_cams, opt));
    if (!poses || !t_final || !last)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_backward: null poses or forward state");
    GS_TRY(check_grads(ctx, grads));
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Plan P = plan_for(g, cams, n_cams);
    GS_TRY(finalize(ctx, P));
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    Pipe p;
    GS_TRY(alloc_pipe(ctx, P, true, p));
    int cur = 0;
    GS_TRY(project_and_bin(ctx, P, D, p, poses, opt, s, &cur, nullptr));
    GS_TRY(backward_core(ctx, P, D, p, cur, g, poses, opt, t_final, last, d_rgb, d_depth, d_alpha, pivots, pose_grad,
                         grads, wants_params(grads), s));
    int flags = 0;
    GS_TRY(read_flags(ctx, p, s, &flags));
    if (flags & gsk::kFlagTimeout)
        return fail(ctx, GS_ERR_TIMEOUT, "a sort pass gave up waiting for an earlier tile");
    return GS_OK;
}

}  // extern "C"

// A forward pass kept for its adjoint: the plan (host), and in two
// stream-ordered device blocks the plan tables, the pose copy, the records
// and their auxiliary camera-frame mean and covariance, the counts, tile
// ranges, the duplicate count, per-pixel final transmittance and last
// contributor (block 1, sized from the plan), and the sorted tile lists
// (block 2, sized after counting).
struct gs_saved {
    int device = 0;
    Plan P;
    DevPlan D;
    gs_gaussians_t g{};
    gs_options_t opt{};
    void *blk[2] = {nullptr, nullptr};
    float *pose32 = nullptr, *t_final = nullptr;
    float4 *rec = nullptr, *aux = nullptr;
    int32_t *counts = nullptr, *last = nullptr;
    uint2 *ranges = nullptr;
    uint32_t *vals = nullptr, *ndups = nullptr;
    uint32_t cap = 0;
};

namespace {

// byte offsets of 256-aligned pieces in one block
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = off;
        off += ((bytes ? bytes : 1) + 255) & ~(size_t)255;
        return o;
    }
};

}  // namespace

extern "C" {

gs_status_t gs_render_saved(gs_ctx_t *ctx, const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams,
                            int n_cams, const gs_options_t *opt, float *rgb, float *depth, float *alpha,
                            gs_saved_t **saved, gs_stream_t stream)
{
    GS_TRY(check_common(ctx, g, cams, n_cams, opt));
    if (!poses || !saved)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_saved: null poses or saved");
    *saved = nullptr;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gs_saved *sv = new gs_saved();
    sv->device = ctx->device;
    sv->g = *g;
    sv->opt = *opt;
    sv->P = plan_for(g, cams, n_cams);
    Plan &P = sv->P;
    const gs_status_t fs = finalize(ctx, P);
    if (fs != GS_OK) {
        delete sv;
        return fs;
    }
    const size_t nv = P.vps.size(), R = std::max<uint64_t>(P.n_records, 1), T = std::max<uint64_t>(P.n_tiles, 1),
                 px = (size_t)std::max<int64_t>(P.n_pix, 1);
    Layout L;
    const size_t o_vps = L.take(sizeof(VpDesc) * nv), o_grp = L.take(sizeof(GroupDesc) * P.groups.size()),
                 o_tvp = L.take(sizeof(uint32_t) * P.tile_vp.size()), o_pose = L.take(sizeof(float) * 12 * nv),
                 o_rec = L.take(sizeof(float4) * 3 * R), o_aux = L.take(sizeof(float4) * 2 * R),
                 o_cnt = L.take(sizeof(int32_t) * R), o_rng = L.take(sizeof(uint2) * T),
                 o_nd = L.take(sizeof(uint32_t) * 4), o_tf = L.take(sizeof(float) * px),
                 o_last = L.take(sizeof(int32_t) * px);
    auto cleanup = [&](gs_status_t st) {
        for (void *b : sv->blk)
            if (b)
                cudaFreeAsync(b, s);
        delete sv;
        return st;
    };
    if (cudaMallocAsync(&sv->blk[0], L.off, s) != cudaSuccess) {
        cudaGetLastError();
        sv->blk[0] = nullptr;
        return cleanup(fail(ctx, GS_ERR_OOM, "gs_render_saved: cudaMallocAsync failed"));
    }
    char *b0 = (char *)sv->blk[0];
    sv->D.vps = (VpDesc *)(b0 + o_vps);
    sv->D.groups = (GroupDesc *)(b0 + o_grp);
    sv->D.tile_vp = (uint32_t *)(b0 + o_tvp);
    sv->pose32 = (float *)(b0 + o_pose);
    sv->rec = (float4 *)(b0 + o_rec);
    sv->aux = (float4 *)(b0 + o_aux);
    sv->counts = (int32_t *)(b0 + o_cnt);
    sv->ranges = (uint2 *)(b0 + o_rng);
    sv->ndups = (uint32_t *)(b0 + o_nd);
    sv->t_final = (float *)(b0 + o_tf);
    sv->last = (int32_t *)(b0 + o_last);
    auto copy = [&](void *dst, const void *src, size_t bytes, cudaMemcpyKind k) {
        return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, k, s) == cudaSuccess;
    };
    if (!copy(sv->D.vps, P.vps.data(), sizeof(VpDesc) * nv, cudaMemcpyHostToDevice) ||
        !copy(sv->D.groups, P.groups.data(), sizeof(GroupDesc) * P.groups.size(), cudaMemcpyHostToDevice) ||
        !copy(sv->D.tile_vp, P.tile_vp.data(), sizeof(uint32_t) * P.tile_vp.size(), cudaMemcpyHostToDevice) ||
        !copy(sv->pose32, poses, sizeof(float) * 12 * nv, cudaMemcpyDeviceToDevice))
        return cleanup(fail(ctx, GS_ERR_CUDA, "gs_render_saved: copy of the plan"));
    // projection into the saved block, list building scratch in the arena
    Pipe p;
    p.rec = sv->rec;
    p.aux = sv->aux;
    p.counts = sv->counts;
    p.ranges = sv->ranges;
    p.ndups = sv->ndups;
    p.n_records = R;
    gs_status_t st = wsT(ctx, S_PARTIALS, gsl::scan_partials(R), &p.partials);
    if (st == GS_OK)
        st = wsT(ctx, S_FLAGS, 4, &p.flags);
    if (st == GS_OK)
        st = alloc_seg(ctx, P, p);
    if (st != GS_OK)
        return cleanup(st);
    if (cudaMemsetAsync(p.flags, 0, sizeof(int), s) != cudaSuccess)
        return cleanup(fail(ctx, GS_ERR_CUDA, "gs_render_saved: memset"));
    gsl::project(project_args(P, sv->D, p, sv->pose32, opt), s);
    gsl::BinArgs b = bin_args(P, sv->D, p);
    gsl::bin_count(b, s);
    uint32_t nd = 0;
    if (cudaMemcpyAsync(&nd, p.ndups, sizeof nd, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cleanup(fail(ctx, GS_ERR_CUDA, "gs_render_saved: duplicate count"));
    if (nd == 0xffffffffu)
        return cleanup(fail(ctx, GS_ERR_CAPACITY, "more than 2^32 tile duplicates"));
    st = alloc_sort(ctx, nd, p);
    if (st != GS_OK)
        return cleanup(st);
    if (cudaMallocAsync(&sv->blk[1], sizeof(uint32_t) * (size_t)p.cap, s) != cudaSuccess) {
        cudaGetLastError();
        sv->blk[1] = nullptr;
        return cleanup(fail(ctx, GS_ERR_OOM, "gs_render_saved: cudaMallocAsync failed"));
    }
    sv->vals = (uint32_t *)sv->blk[1];
    sv->cap = p.cap;
    p.vals[0] = sv->vals;  // the sorted lists land in the saved block
    b = bin_args(P, sv->D, p);
    const int cur = run_bin(b, s);
    gsl::RasterArgs r = raster_args(P, sv->D, p, cur, opt);
    r.out_rgb = rgb;
    r.out_depth = depth;
    r.out_alpha = alpha;
    r.t_final = sv->t_final;
    r.last = sv->last;
    gsl::forward(r, false, s);
    if (cudaGetLastError() != cudaSuccess)
        return cleanup(fail(ctx, GS_ERR_CUDA, "gs_render_saved: launch"));
    int flags = 0;
    st = read_flags(ctx, p, s, &flags);
    if (st != GS_OK)
        return cleanup(st);
    if (flags & gsk::kFlagNonFinite)
        return cleanup(fail(ctx, GS_ERR_NONFINITE, "non-finite Gaussian parameter"));
    ctx->stats = gs_stats_t{};
    ctx->stats.n_dups = nd;
    ctx->stats.n_pixels = P.n_pix;
    *saved = sv;
    return GS_OK;
}

gs_status_t gs_saved_outputs(const gs_saved_t *saved, float **t_final, int32_t **last)
{
    if (!saved)
        return GS_ERR_INVALID_ARG;
    if (t_final)
        *t_final = saved->t_final;
    if (last)
        *last = saved->last;
    return GS_OK;
}

gs_status_t gs_render_backward_saved(gs_ctx_t *ctx, const gs_saved_t *saved, const float *d_rgb,
                                     const float *d_depth, const float *d_alpha, const float *pivots,
                                     float *pose_grad, const gs_gaussian_grads_t *grads, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (!saved || saved->device != ctx->device)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_backward_saved: no saved forward of this context's device");
    GS_TRY(check_grads(ctx, grads));
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const Plan &P = saved->P;
    Pipe p;
    p.rec = saved->rec;
    p.aux = saved->aux;
    p.counts = saved->counts;
    p.ranges = saved->ranges;
    p.vals[0] = saved->vals;
    p.ndups = saved->ndups;
    p.cap = saved->cap;
    p.n_records = std::max<uint64_t>(P.n_records, 1);
    const bool full = wants_params(grads);
    if (full) {
        const size_t hn = gsl::sort_hist_entries((uint32_t)std::max<uint64_t>(p.cap, p.n_records));
        GS_TRY(wsT(ctx, S_HIST, hn, &p.hist));
        GS_TRY(wsT(ctx, S_HISTP, gsl::scan_partials(hn), &p.histp));
    }
    return backward_core(ctx, P, saved->D, p, 0, &saved->g, saved->pose32, &saved->opt, saved->t_final,
                         saved->last, d_rgb, d_depth, d_alpha, pivots, pose_grad, grads, full, s);
}

gs_status_t gs_saved_destroy(gs_saved_t *saved, gs_stream_t stream)
{
    if (!saved)
        return GS_ERR_INVALID_ARG;
    DeviceGuard dg(saved->device);
    for (void *b : saved->blk)
        if (b)
            cudaFreeAsync(b, (cudaStream_t)stream);
    delete saved;
    return GS_OK;
}

gs_status_t gs_loss(gs_ctx_t *ctx, const gs_camera_t *cams, int n_cams, const float *rgb, const float *depth,
                    const float *t_rgb, const float *t_depth, double *loss, float *d_rgb, float *d_depth,
                    gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (n_cams < 0 || (n_cams > 0 && (!cams || !rgb || !depth || !t_rgb || !t_depth || !loss)))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_loss: bad arguments");
    for (int c = 0; c < n_cams; ++c)
        GS_TRY(check_camera(ctx, cams[c]));
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gs_gaussians_t g{};
    Plan P;
    int64_t pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        add_vp(P, &g, cams[c], 0, 0, 0, t_rgb + 3 * pix, t_depth + pix);
        pix += (int64_t)cams[c].width * cams[c].height;
    }
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    float *tloss = nullptr;
    GS_TRY(wsT(ctx, S_TLOSS, (size_t)std::max<uint64_t>(P.n_tiles, 1), &tloss));
    gsl::loss(D.vps, (int)P.vps.size(), (uint32_t)P.n_tiles, D.tile_vp, rgb, depth, loss, d_rgb, d_depth, tloss, s);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t gs_track_loss(gs_ctx_t *ctx, const gs_camera_t *cams, int n_cams, const float *rgb, const float *depth,
                          const float *t_final, const float *t_rgb, const float *t_depth, float lambda_c,
                          double *loss, float *d_rgb, float *d_depth, uint8_t *inlier, float *median,
                          gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (n_cams < 0 || (n_cams > 0 && (!cams || !rgb || !depth || !t_final || !t_rgb || !t_depth || !loss)) ||
        !(lambda_c >= 0.0f && lambda_c <= 1.0f))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_track_loss: bad arguments");
    for (int c = 0; c < n_cams; ++c)
        GS_TRY(check_camera(ctx, cams[c]));
    if (n_cams == 0)
        return GS_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gs_gaussians_t g{};
    Plan P;
    int64_t pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        add_vp(P, &g, cams[c], 0, 0, 0, t_rgb + 3 * pix, t_depth + pix);
        P.vps.back().loss_kind = 1;
        P.vps.back().lambda_c = lambda_c;
        pix += (int64_t)cams[c].width * cams[c].height;
    }
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    float *tloss = nullptr;
    GS_TRY(wsT(ctx, S_TLOSS, (size_t)std::max<uint64_t>(P.n_tiles, 1), &tloss));
    gsl::RasterArgs r{};
    r.t_final = const_cast<float *>(t_final);
    gsl::TrackArgs ta;
    GS_TRY(alloc_track(ctx, P, D, r, ta, tloss, s));
    ta.rgb = rgb;
    ta.depth = depth;
    ta.d_rgb = d_rgb;
    ta.d_depth = d_depth;
    ta.inlier = inlier;
    gsl::track_prep(ta, rgb, depth, r.trk_err, r.trk_col, s);
    gsl::track_loss(ta, s);
    gsl::loss_reduce(D.vps, (int)P.vps.size(), tloss, loss, s);
    if (median)
        GS_CUDA(cudaMemcpyAsync(median, ta.med, sizeof(float) * (size_t)n_cams, cudaMemcpyDeviceToDevice, s));
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t gs_overlap_ratio(gs_ctx_t *ctx, const gs_gaussians_t *p, const gs_gaussians_t *q, const double *T_host,
                             float tau, double *ratio, int64_t *n_corr, int32_t *nn_pq, int32_t *nn_qp,
                             gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_gaussians(ctx, p, "P"));
    GS_TRY(check_gaussians(ctx, q, "Q"));
    if (!T_host || !ratio || !(tau >= 0.0f) || !std::isfinite(tau))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_overlap_ratio: bad arguments");
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(T_host[k]))
            return fail(ctx, GS_ERR_INVALID_ARG, "gs_overlap_ratio: non-finite transform");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)p->n, nq = (size_t)q->n;
    gsl::OverlapArgs a{};
    a.p = (const float4 *)p->means;
    a.q = (const float4 *)q->means;
    a.np = (int)np;
    a.nq = (int)nq;
    std::vector<float> T32(12);
    for (int k = 0; k < 12; ++k)
        T32[k] = (float)T_host[k];
    float *Td = nullptr;
    GS_TRY(upload(ctx, S_OT, T32, &Td, s));
    a.T32 = Td;
    GS_TRY(wsT(ctx, S_OPT, std::max<size_t>(np, 1), &a.pt));
    if (nn_pq)
        a.nn_pq = nn_pq;
    else
        GS_TRY(wsT(ctx, S_ONN1, std::max<size_t>(np, 1), &a.nn_pq));
    if (nn_qp)
        a.nn_qp = nn_qp;
    else
        GS_TRY(wsT(ctx, S_ONN2, std::max<size_t>(nq, 1), &a.nn_qp));
    GS_TRY(wsT(ctx, S_OD2, std::max<size_t>(np, 1), &a.d2));
    GS_TRY(wsT(ctx, S_OCNT, 2, &a.counts));
    a.tau2 = tau * tau;
    if (np < 64 || nq < 64) {
        gsl::overlap(a, s);  // brute force
    } else {
        // uniform grid over the box of both point sets (read back once)
        uint32_t *bbox = nullptr;
        GS_TRY(wsT(ctx, S_OBOX, 6, &bbox));
        gsl::overlap_moved_bbox(a, bbox, s);
        uint32_t mm[6];
        GS_CUDA(cudaMemcpyAsync(mm, bbox, sizeof mm, cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaStreamSynchronize(s));
        auto o2f = [](uint32_t u) {
            const uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
            float f;
            std::memcpy(&f, &b, sizeof f);
            return (double)f;
        };
        double lo[3], ext[3], emax = 0.0;
        for (int k = 0; k < 3; ++k) {
            lo[k] = o2f(mm[k]);
            ext[k] = o2f(mm[3 + k]) - lo[k];
            if (!std::isfinite(lo[k]) || !std::isfinite(ext[k]))
                return fail(ctx, GS_ERR_NONFINITE, "gs_overlap_ratio: non-finite mean");
            emax = std::max(emax, ext[k]);
        }
        const double pad = 1e-3 * emax + 1e-6;
        double vol = 1.0;
        for (int k = 0; k < 3; ++k) {
            lo[k] -= pad;
            ext[k] = std::max(ext[k] + 2.0 * pad, 1e-3 * emax + 1e-6);
            vol *= ext[k];
        }
        // about two cells per target, at most 2^22 cells and 2048 per axis
        double cell = std::cbrt(vol / (2.0 * (double)std::max(np, nq)));
        cell = std::max(cell, (emax + 2.0 * pad) / 2048.0);
        int dims[3];
        for (;;) {
            size_t cells = 1;
            for (int k = 0; k < 3; ++k) {
                dims[k] = std::max(1, (int)std::ceil(ext[k] / cell));
                cells *= (size_t)dims[k];
            }
            if (cells <= ((size_t)1 << 22))
                break;
            cell *= 1.26;
        }
        gsl::NNGrid g{};
        g.ox = (float)lo[0];
        g.oy = (float)lo[1];
        g.oz = (float)lo[2];
        g.s = (float)cell;
        g.inv_s = 1.0f / g.s;
        g.nx = dims[0];
        g.ny = dims[1];
        g.nz = dims[2];
        double amax = 0.0;  // largest coordinate magnitude in the box
        for (int k = 0; k < 3; ++k)
            amax = std::max(amax, std::max(std::fabs(lo[k]), std::fabs(lo[k] + ext[k])));
        g.margin = (float)(4e-6 * (emax + amax) + 1e-7);
        const size_t cells = (size_t)dims[0] * dims[1] * dims[2], nmax = std::max(np, nq);
        // one grid per set; each set's points in cell order are then the
        // query order of its search in the other set's grid (neighbouring
        // threads search the same cells)
        gsl::NNScratch sq{}, sp{};
        const int sl[2][8] = {{S_GCELL, S_GSTART, S_GCUR, S_GPART, S_GPTS, S_GIDX, S_GLIST, S_GNL},
                              {S_GCELL2, S_GSTART2, S_GCUR2, S_GPART2, S_GPTS2, S_GIDX2, S_GLIST2, S_GNL2}};
        gsl::NNScratch *scs[2] = {&sq, &sp};
        for (int k = 0; k < 2; ++k) {
            gsl::NNScratch &sc = *scs[k];
            GS_TRY(wsT(ctx, sl[k][0], nmax, &sc.cell));
            GS_TRY(wsT(ctx, sl[k][1], cells + 1, &sc.start));
            GS_TRY(wsT(ctx, sl[k][2], cells, &sc.cursor));
            GS_TRY(wsT(ctx, sl[k][3], gsl::scan_partials(cells + 1), &sc.partials));
            GS_TRY(wsT(ctx, sl[k][4], nmax, &sc.spts));
            GS_TRY(wsT(ctx, sl[k][5], nmax, &sc.sidx));
            GS_TRY(wsT(ctx, sl[k][6], nmax, &sc.list));
            GS_TRY(wsT(ctx, sl[k][7], 1, &sc.n_list));
        }
        gsl::nn_grid_build(a.q, (int)nq, g, sq, s);
        gsl::nn_grid_build(a.pt, (int)np, g, sp, s);
        gsl::nn_grid_search(a.pt, (int)np, sp.sidx, a.q, (int)nq, g, sq, a.nn_pq, a.d2, s);
        gsl::nn_grid_search(a.q, (int)nq, sq.sidx, a.pt, (int)np, g, sp, a.nn_qp, nullptr, s);
        gsl::overlap_count(a, s);
    }
    unsigned long long c[2] = {0, 0};
    GS_CUDA(cudaMemcpyAsync(c, a.counts, sizeof c, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    *ratio = c[0] ? (double)c[1] / (double)c[0] : 0.0;
    if (n_corr)
        *n_corr = (int64_t)c[0];
    return GS_OK;
}

gs_status_t gs_pose_step(gs_ctx_t *ctx, int n, double *pose, double *state, const double *grad,
                         const double *pivot, int k, int iters, const gs_options_t *opt, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, opt));
    if (n < 0 || iters <= 0 || k < 0 || (n > 0 && (!pose || !state || !grad || !pivot)))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_pose_step: bad arguments");
    DeviceGuard dg(ctx->device);
    gsl::pose_step_raw(n, pose, state, grad, pivot, k, iters, opt->lr_rot, opt->lr_trans, opt->beta1, opt->beta2,
                       opt->adam_eps, opt->lr_final, (cudaStream_t)stream);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t gs_fuse(gs_ctx_t *ctx, int k, const double *est, const int32_t *reverse, const double *eps,
                    double *T_out, double *conf, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (k <= 0 || !est || !reverse || !eps || !T_out || !conf)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_fuse: bad arguments");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *pf = nullptr, *pc = nullptr;
    GS_TRY(upload(ctx, S_PFIRST, std::vector<int32_t>{0}, &pf, s));
    GS_TRY(upload(ctx, S_PCOUNT, std::vector<int32_t>{k}, &pc, s));
    gsl::FuseArgs a{};
    a.pose64 = est;
    a.eps = eps;
    a.reverse = reverse;
    a.prob_first = pf;
    a.prob_count = pc;
    a.n_problems = 1;
    a.T_out = T_out;
    a.conf = conf;
    gsl::fuse(a, s);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t gs_transform(gs_ctx_t *ctx, const gs_gaussians_t *g, const double *T_host, float *out_means,
                         float *out_quats, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_gaussians(ctx, g, "submap"));
    if (!T_host || (g->n > 0 && (!out_means || !out_quats || !aligned16(out_means) || !aligned16(out_quats))))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_transform: bad arguments");
    DeviceGuard dg(ctx->device);
    gsl::transform((const float4 *)g->means, (const float4 *)g->quats, g->n, T_host, (float4 *)out_means,
                   (float4 *)out_quats, (cudaStream_t)stream);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t sort_u32_impl(gs_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int bits, bool withhold,
                          cudaStream_t s)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (n < 0 || n > 0xfff00000ll || bits < 0 || bits > 32 || (n > 0 && (!keys || !vals)))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_sort_u32: bad arguments");
    if (n == 0 || bits == 0)
        return GS_OK;
    DeviceGuard dg(ctx->device);
    const uint32_t cap = (uint32_t)n;
    uint32_t *k2 = nullptr, *v2 = nullptr, *nd = nullptr;
    uint8_t *os = nullptr;
    int *flags = nullptr;
    GS_TRY(wsT(ctx, S_SK, cap, &k2));
    GS_TRY(wsT(ctx, S_SV, cap, &v2));
    GS_TRY(wsT(ctx, S_SN, 2, &nd));
    GS_TRY(wsT(ctx, S_OS, gsl::onesweep_scratch_bytes(cap, bits), &os));
    GS_TRY(wsT(ctx, S_FLAGS, 4, &flags));
    GS_CUDA(cudaMemcpyAsync(nd, &cap, sizeof cap, cudaMemcpyHostToDevice, s));
    GS_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), s));
    uint32_t *kk[2] = {keys, k2}, *vv[2] = {vals, v2};
    const int cur = gsl::onesweep_u32(kk, vv, nd, cap, bits, os, flags, s, withhold);
    if (cur != 0) {
        GS_CUDA(cudaMemcpyAsync(keys, k2, sizeof(uint32_t) * cap, cudaMemcpyDeviceToDevice, s));
        GS_CUDA(cudaMemcpyAsync(vals, v2, sizeof(uint32_t) * cap, cudaMemcpyDeviceToDevice, s));
    }
    int fl = 0;
    GS_CUDA(cudaMemcpyAsync(&fl, flags, sizeof fl, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (fl & gsk::kFlagTimeout)
        return fail(ctx, GS_ERR_TIMEOUT, "a sort pass gave up waiting for an earlier tile");
    return GS_OK;
}

gs_status_t gs_sort_u32(gs_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int bits, gs_stream_t stream)
{
    return sort_u32_impl(ctx, keys, vals, n, bits, false, (cudaStream_t)stream);
}

gs_status_t gs_selftest_bounded_wait(gs_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, gs_stream_t stream)
{
    return sort_u32_impl(ctx, keys, vals, n, 8, true, (cudaStream_t)stream);
}

gs_status_t gs_transform_batch(gs_ctx_t *ctx, const gs_gaussians_t *maps, int n_maps, const double *T_host,
                               float *const *out_means, float *const *out_quats, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    if (n_maps < 0 || (n_maps > 0 && (!maps || !T_host || !out_means || !out_quats)))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_transform_batch: bad arguments");
    std::vector<gsl::MapDesc> md;
    unsigned blocks = 0;
    for (int k = 0; k < n_maps; ++k) {
        GS_TRY(check_gaussians(ctx, &maps[k], "submap"));
        if (maps[k].n > 0 && (!out_means[k] || !out_quats[k] || !aligned16(out_means[k]) || !aligned16(out_quats[k])))
            return fail(ctx, GS_ERR_INVALID_ARG, "gs_transform_batch: bad output arrays");
        for (int j = 0; j < 12; ++j)
            if (!std::isfinite(T_host[12 * k + j]))
                return fail(ctx, GS_ERR_INVALID_ARG, "gs_transform_batch: non-finite transform");
        if (maps[k].n == 0)
            continue;
        gsl::MapDesc m{};
        m.means = (const float4 *)maps[k].means;
        m.quats = (const float4 *)maps[k].quats;
        m.out_means = (float4 *)out_means[k];
        m.out_quats = (float4 *)out_quats[k];
        m.n = maps[k].n;
        m.blk_base = blocks;
        std::memcpy(m.T, T_host + 12 * k, sizeof m.T);
        md.push_back(m);
        blocks += (unsigned)((m.n + 255) / 256);
    }
    if (md.empty())
        return GS_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gsl::MapDesc *dmd = nullptr;
    GS_TRY(upload(ctx, S_MAPS, md, &dmd, s));
    gsl::transform_batch(dmd, (int)md.size(), blocks, s);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
}

gs_status_t gs_probe_fp32(gs_ctx_t *ctx, double *tflops, int *sm_count, gs_stream_t stream)
{
    if (!ctx || !tflops)
        return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (sm_count)
        *sm_count = sms;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float *sink = nullptr;
    GS_TRY(wsT(ctx, S_PROBE, (size_t)blocks * threads, &sink));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    float best = 0.0f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 12 && err == cudaSuccess; ++rep) {
        err = cudaEventRecord(e0, s);
        // scalar and packed launches alternate; each form's first launch warms up
        if (rep % 2 == 0)
            k_fma_probe<false><<<blocks, threads, 0, s>>>(sink, iters, 0.9999999f, 1e-7f);
        else
            k_fma_probe<true><<<blocks, threads, 0, s>>>(sink, iters, 0.9999999f, 1e-7f);
        ++gsl::g_launches;
        if (err == cudaSuccess)
            err = cudaEventRecord(e1, s);
        if (err == cudaSuccess)
            err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess)
            err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 1 && ms > 0.0f) {
            const float tf = (float)((double)blocks * threads * iters * kProbeChains * 2.0 / (ms * 1e-3) / 1e12);
            best = std::max(best, tf);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess)
        return fail(ctx, GS_ERR_CUDA, std::string("fp32 probe: ") + cudaGetErrorString(err));
    *tflops = best;
    return GS_OK;
}

gs_status_t gs_register(gs_ctx_t *ctx, const gs_gaussians_t *src, const gs_gaussians_t *tgt,
                        const gs_view_t *src_views, int n_src_views, const gs_view_t *tgt_views, int n_tgt_views,
                        const gs_options_t *opt, int iters, double *T_out, double *confidence, double *eps_out,
                        double *est_out, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, opt));
    GS_TRY(check_gaussians(ctx, src, "src"));
    GS_TRY(check_gaussians(ctx, tgt, "tgt"));
    if (n_src_views < 0 || n_tgt_views < 0 || n_src_views + n_tgt_views == 0 || iters < 0 || !T_out ||
        !confidence || (n_src_views > 0 && !src_views) || (n_tgt_views > 0 && !tgt_views))
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_register: bad arguments");
    for (int k = 0; k < n_src_views; ++k) {
        GS_TRY(check_camera(ctx, src_views[k].cam));
        if (!src_views[k].rgb || !src_views[k].depth)
            return fail(ctx, GS_ERR_INVALID_ARG, "gs_register: null keyframe image");
    }
    for (int k = 0; k < n_tgt_views; ++k) {
        GS_TRY(check_camera(ctx, tgt_views[k].cam));
        if (!tgt_views[k].rgb || !tgt_views[k].depth)
            return fail(ctx, GS_ERR_INVALID_ARG, "gs_register: null keyframe image");
    }
    DeviceGuard dg(ctx->device);
    Plan P;
    int sets = 0;
    add_problem(P, src, tgt, src_views, n_src_views, tgt_views, n_tgt_views, 0, sets, opt);
    return run_registration(ctx, P, 1, opt, iters, (cudaStream_t)stream, T_out, confidence, eps_out, est_out);
}

gs_status_t gs_register_async(gs_ctx_t *ctx, const gs_gaussians_t *src, const gs_gaussians_t *tgt,
                              const gs_view_t *src_views, int n_src_views, const gs_view_t *tgt_views,
                              int n_tgt_views, const gs_options_t *opt, int iters, double *T_dev, double *conf_dev,
                              double *eps_dev, double *est_dev, int32_t *status_dev, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, opt));
    if (!src || !tgt || !T_dev || !conf_dev || !status_dev || iters < 0 || n_src_views < 0 || n_tgt_views < 0 ||
        n_src_views + n_tgt_views == 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_register_async: bad arguments");
    gs_problem_t q{};
    q.src = *src;
    q.tgt = *tgt;
    q.src_views = src_views;
    q.n_src_views = n_src_views;
    q.tgt_views = tgt_views;
    q.n_tgt_views = n_tgt_views;
    GS_TRY(check_problem(ctx, q));
    DeviceGuard dg(ctx->device);
    Plan P;
    int sets = 0;
    add_problem(P, src, tgt, src_views, n_src_views, tgt_views, n_tgt_views, 0, sets, opt);
    AsyncOut ao;
    ao.T = T_dev;
    ao.conf = conf_dev;
    ao.eps = eps_dev;
    ao.est = est_dev;
    ao.status = status_dev;
    return run_registration(ctx, P, 1, opt, iters, (cudaStream_t)stream, nullptr, nullptr, nullptr, nullptr, &ao);
}

gs_status_t gs_register_gradient(gs_ctx_t *ctx, const gs_gaussians_t *src, const gs_gaussians_t *tgt,
                                 const gs_view_t *src_views, int n_src_views, const gs_view_t *tgt_views,
                                 int n_tgt_views, const gs_options_t *opt, double *loss_out, double *grad_out,
                                 gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, opt));
    if (!src || !tgt || !grad_out || n_src_views < 0 || n_tgt_views < 0 || n_src_views + n_tgt_views == 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_register_gradient: bad arguments");
    gs_problem_t q{};
    q.src = *src;
    q.tgt = *tgt;
    q.src_views = src_views;
    q.n_src_views = n_src_views;
    q.tgt_views = tgt_views;
    q.n_tgt_views = n_tgt_views;
    GS_TRY(check_problem(ctx, q));
    DeviceGuard dg(ctx->device);
    Plan P;
    int sets = 0;
    add_problem(P, src, tgt, src_views, n_src_views, tgt_views, n_tgt_views, 0, sets, opt);
    double T[12], conf = 0.0;
    return run_registration(ctx, P, 1, opt, 1, (cudaStream_t)stream, T, &conf, loss_out, nullptr, nullptr,
                            grad_out);
}

gs_status_t gs_register_batch_async(gs_ctx_t *ctx, const gs_problem_t *problems, int n, const gs_options_t *opt,
                                    int iters, double *T_dev, double *conf_dev, double *eps_dev, int32_t *status_dev,
                                    gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, opt));
    if (n <= 0 || !problems || iters < 0 || !T_dev || !conf_dev || !status_dev)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_register_batch_async: bad arguments");
    for (int i = 0; i < n; ++i) {
        GS_TRY(check_problem(ctx, problems[i]));
        if (problems[i].opt)
            GS_TRY(check_options(ctx, problems[i].opt));
    }
    DeviceGuard dg(ctx->device);
    Plan P;
    int sets = 0;
    for (int i = 0; i < n; ++i) {
        const gs_problem_t &q = problems[i];
        add_problem(P, &q.src, &q.tgt, q.src_views, q.n_src_views, q.tgt_views, q.n_tgt_views, i, sets,
                    q.opt ? q.opt : opt);
    }
    AsyncOut ao;
    ao.T = T_dev;
    ao.conf = conf_dev;
    ao.eps = eps_dev;
    ao.status = status_dev;
    return run_registration(ctx, P, n, opt, iters, (cudaStream_t)stream, nullptr, nullptr, nullptr, nullptr, &ao);
}

gs_status_t gs_register_batch(gs_ctx_t *ctx, const gs_problem_t *problems, int n, const gs_options_t *opt, int iters,
                              double *T_out, double *conf_out, double *eps_out, gs_stream_t stream)
{
    if (!ctx)
        return GS_ERR_INVALID_ARG;
    GS_TRY(check_options(ctx, opt));
    if (n <= 0 || !problems || iters < 0 || !T_out || !conf_out)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_register_batch: bad arguments");
    for (int i = 0; i < n; ++i) {
        GS_TRY(check_problem(ctx, problems[i]));
        if (problems[i].opt)
            GS_TRY(check_options(ctx, problems[i].opt));
    }
    DeviceGuard dg(ctx->device);
    Plan P;
    int sets = 0;
    for (int i = 0; i < n; ++i) {
        const gs_problem_t &q = problems[i];
        add_problem(P, &q.src, &q.tgt, q.src_views, q.n_src_views, q.tgt_views, q.n_tgt_views, i, sets,
                    q.opt ? q.opt : opt);
    }
    return run_registration(ctx, P, n, opt, iters, (cudaStream_t)stream, T_out, conf_out, eps_out, nullptr);
}

}  // extern "C"

namespace {

// The registration engine behind gs_register and gs_register_batch: every
// keyframe problem of the plan (any mix of submaps, keyframe counts and
// image sizes) advances together, one CUDA graph per iteration.
// The status word of an asynchronous registration: the device flags and the
// residuals' finiteness as a gs_status_t.
__global__ void k_async_status(const int *flags, const double *eps, int nv, int32_t *status)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    const int f = *flags;
    int32_t st = GS_OK;
    if (f & gsk::kFlagNonFinite)
        st = GS_ERR_NONFINITE;
    else if (f & gsk::kFlagTimeout)
        st = GS_ERR_TIMEOUT;
    else if (f & gsk::kFlagCapacity)
        st = GS_ERR_CAPACITY;
    else
        for (int v = 0; v < nv; ++v)
            if (!isfinite(eps[v]))
                st = GS_ERR_DIVERGED;
    *status = st;
}

gs_status_t run_registration(gs_ctx *ctx, Plan &P, int n_problems, const gs_options_t *opt, int iters,
                             cudaStream_t s, double *T_out, double *conf_out, double *eps_out, double *est_out,
                             const AsyncOut *ao, double *grad_out)
{
    GS_TRY(finalize(ctx, P));
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    const int nv = (int)P.vps.size();
    const int n_sets = (int)P.set_vp.size();
    Pipe p;
    GS_TRY(alloc_pipe(ctx, P, true, p));
    float *pose32 = nullptr, *tloss = nullptr, *tf = nullptr;
    double *pose64 = nullptr, *adam = nullptr, *pivot = nullptr, *ccam = nullptr, *cent = nullptr, *lossd = nullptr,
           *Tdev = nullptr, *confd = nullptr, *est = nullptr;
    float2 *ttw = nullptr;
    int32_t *last = nullptr, *rev = nullptr, *pf = nullptr, *pc = nullptr;
    uint8_t *code = nullptr;
    const size_t npix = (size_t)std::max<int64_t>(P.n_pix, 1), ntl = (size_t)std::max<uint64_t>(P.n_tiles, 1);
    GS_TRY(wsT(ctx, S_POSE32, 12 * (size_t)nv, &pose32));
    GS_TRY(wsT(ctx, S_POSE64, 12 * (size_t)nv, &pose64));
    GS_TRY(wsT(ctx, S_ADAM, 13 * (size_t)nv, &adam));
    GS_TRY(wsT(ctx, S_PIVOT, 3 * (size_t)nv, &pivot));
    GS_TRY(wsT(ctx, S_CCAM, 3 * (size_t)nv, &ccam));
    GS_TRY(wsT(ctx, S_CENT, 3 * (size_t)n_sets, &cent));
    GS_TRY(wsT(ctx, S_LOSS, (size_t)nv, &lossd));
    GS_TRY(wsT(ctx, S_TF, npix, &tf));
    GS_TRY(wsT(ctx, S_LAST, npix, &last));
    GS_TRY(wsT(ctx, S_CODE, npix, &code));
    GS_TRY(wsT(ctx, S_TLOSS, ntl, &tloss));
    GS_TRY(wsT(ctx, S_TTWIST, 6 * ntl, &ttw));
    GS_TRY(wsT(ctx, S_TOUT, 12 * (size_t)n_problems, &Tdev));
    GS_TRY(wsT(ctx, S_CONF, (size_t)n_problems, &confd));
    GS_TRY(wsT(ctx, S_EST, 12 * (size_t)nv, &est));
    std::vector<int32_t> revh(nv), pfh(n_problems, 0), pch(n_problems, 0);
    for (int v = 0; v < nv; ++v) {
        revh[v] = P.vps[v].reverse;
        const int q = P.vps[v].problem;
        if (pch[q]++ == 0)
            pfh[q] = v;
    }
    GS_TRY(upload(ctx, S_REV, revh, &rev, s));
    GS_TRY(upload(ctx, S_PFIRST, pfh, &pf, s));
    GS_TRY(upload(ctx, S_PCOUNT, pch, &pc, s));

    gsl::PoseArgs pa{};
    pa.vps = D.vps;
    pa.n_vps = nv;
    pa.tile_twist = ttw;
    pa.tile_loss = tloss;
    pa.pose64 = pose64;
    pa.pose32 = pose32;
    pa.adam = adam;
    pa.pivot = pivot;
    pa.c_cam = ccam;
    pa.centroid = cent;
    pa.loss = lossd;
    pa.lr_rot = opt->lr_rot;
    pa.lr_trans = opt->lr_trans;
    pa.beta1 = opt->beta1;
    pa.beta2 = opt->beta2;
    pa.eps = opt->adam_eps;
    pa.lr_final = opt->lr_final;
    pa.iters = std::max(iters, 1);
    pa.update = 1;
    double *gradd = nullptr;
    if (grad_out) {
        // gradient mode (gs_register_gradient): one iteration that reduces
        // each keyframe's twist and updates nothing
        GS_TRY(wsT(ctx, S_GRAD, 6 * (size_t)std::max(nv, 1), &gradd));
        pa.grad = gradd;
        pa.update = 0;
    }

    unsigned long long *pairs = nullptr;
    GS_TRY(wsT(ctx, S_PAIRS, 2 * ntl, &pairs));  // per tile: walked, contributing
    const bool prof = opt->profile != 0 && iters > 0 && !ao;
    if (prof) {
        for (cudaEvent_t &e : ctx->tev)
            if (!e)
                GS_CUDA(cudaEventCreate(&e));
        while ((int)ctx->pool.size() < iters * (kPhases + 1)) {
            cudaEvent_t e;
            GS_CUDA(cudaEventCreate(&e));
            ctx->pool.push_back(e);
        }
    }

    gsl::RasterArgs expo_r{};
    GS_TRY(alloc_exposure(ctx, P, pa, expo_r));
    double headroom = opt->list_headroom;
    const auto key = std::make_tuple((uint64_t)P.n_tiles, P.vps.size(), (uint64_t)P.n_records);
    for (int attempt = 0; attempt < 3; ++attempt) {
        const long long l0 = gsl::g_launches;
        long long captured = 0, graph_kernels = 0, trial_kernels = 0;
        ctx->stats = gs_stats_t{};
        gsl::centroids(D.vps, D.set_vp, n_sets, cent, s);
        gsl::pose_init(pa, s);
        // size the duplicate lists at the initial poses (with headroom: the
        // count drifts as the poses move).  The asynchronous form takes the
        // largest count an earlier call saw for this plan shape, and counts
        // (synchronising once) only for a shape it has not seen.
        int cur = 0;
        uint32_t nd = 0;
        const auto seen = ctx->dups_seen.find(key);
        if (ao && seen != ctx->dups_seen.end()) {
            nd = seen->second;
        } else {
            GS_TRY(project_and_bin(ctx, P, D, p, pose32, opt, s, &cur, &nd));
            uint32_t &m = ctx->dups_seen[key];
            m = std::max(m, nd);
        }
        const uint64_t want = (uint64_t)(headroom * nd) + (headroom >= 1.0 ? 65536 : 0);
        if (p.cap < want)
            GS_TRY(alloc_sort(ctx, want, p));
        gsl::BinArgs b = bin_args(P, D, p);
        // the sizing rule's capacity, whatever earlier calls left allocated
        b.capacity = (uint32_t)std::max<uint64_t>(std::min<uint64_t>(want, p.cap), 1);
        gsl::RasterArgs r = raster_args(P, D, p, 0, opt);
        r.t_final = tf;
        r.last = last;
        r.code = code;
        r.tile_loss = tloss;
        r.tile_twist = ttw;
        r.c_cam = ccam;
        r.tile_pairs = pairs;
        r.expo32 = expo_r.expo32;
        r.tile_expo = expo_r.tile_expo;
        r.exposure = any_exposure(P);
        r.count_contrib = opt->profile >= 2;
        gsl::TrackArgs ta;
        GS_TRY(alloc_track(ctx, P, D, r, ta, tloss, s));
        uint32_t *order = nullptr, *order_cnt = nullptr, *queue = nullptr;
        GS_TRY(wsT(ctx, S_ORDER, ntl, &order));
        GS_TRY(wsT(ctx, S_ORDC, 128, &order_cnt));
        GS_TRY(wsT(ctx, S_QUEUE, 4, &queue));
        bool ordered = false, persistent = false, marking = prof;
        cudaError_t mark_err = cudaSuccess;
        auto mark = [&](int k, cudaStream_t st) {
            // an event record node of the captured graph (re-targeted per replay)
            if (marking && mark_err == cudaSuccess)
                mark_err = cudaEventRecordWithFlags(ctx->tev[k], st, cudaEventRecordExternal);
        };
        auto iteration = [&](cudaStream_t st) {
            mark(0, st);
            gsl::project(project_args(P, D, p, pose32, opt, false), st);
            mark(1, st);
            const int c = run_bin(b, st);
            if (ordered)
                gsl::tile_order(p.ranges, (uint32_t)P.n_tiles, order, order_cnt, st);
            mark(2, st);
            r.vals = p.vals[c];
            r.tile_order = ordered ? order : nullptr;
            r.queue = persistent ? queue : nullptr;
            if (opt->fuse_compositing && ta.n_track == 0) {
                gsl::forward_backward(r, st);
                mark(3, st);
            } else {
                gsl::forward(r, true, st);
                gsl::track_loss(ta, st);
                mark(3, st);
                gsl::backward(r, true, false, st);
            }
            mark(4, st);
            gsl::pose_update(pa, st);
            mark(5, st);
        };
        // one iteration captured into an executable graph
        auto capture = [&](cudaGraphExec_t *exec, cudaGraph_t *graph_out) -> gs_status_t {
            GS_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
            iteration(ctx->cap);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &graph);
            if (ce != cudaSuccess || !graph)
                return fail(ctx, GS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(graph);
                return fail(ctx, GS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
            }
            if (graph_out)
                *graph_out = graph;
            else
                cudaGraphDestroy(graph);
            return GS_OK;
        };
        // Autotuner: the CTA schedule of the compositing kernels for this
        // plan shape -- tile order (natural, or longest lists first) x launch
        // (one CTA per tile, or persistent CTAs pulling tiles from one work
        // queue over every keyframe problem) -- timed on trial iterations
        // 1 2 3 4 4 3 2 1 from the initial poses, then the poses start over.
        // Every schedule gives the same results.
        int sched = opt->tile_schedule;
        if (sched == 0) {
            const auto it = ctx->schedule.find(key);
            if (it != ctx->schedule.end()) {
                sched = it->second;
            } else if (iters >= 8 && P.n_tiles >= 2048 && !ao) {
                marking = false;
                cudaGraphExec_t g[4] = {};
                const long long t0 = gsl::g_launches;
                gs_status_t st = GS_OK;
                for (int k = 0; k < 4 && st == GS_OK; ++k) {
                    ordered = (k & 1) != 0;
                    persistent = (k & 2) != 0;
                    st = capture(&g[k], nullptr);
                }
                trial_kernels = gsl::g_launches - t0;  // each graph runs twice: count them once more
                cudaEvent_t e[9] = {};
                for (cudaEvent_t &x : e)
                    if (st == GS_OK && cudaEventCreate(&x) != cudaSuccess)
                        st = fail(ctx, GS_ERR_CUDA, "autotuner events");
                const int seq[8] = {0, 1, 2, 3, 3, 2, 1, 0};
                if (st == GS_OK && cudaEventRecord(e[0], s) != cudaSuccess)
                    st = fail(ctx, GS_ERR_CUDA, "autotuner events");
                for (int k = 0; k < 8 && st == GS_OK; ++k)
                    if (cudaGraphLaunch(g[seq[k]], s) != cudaSuccess || cudaEventRecord(e[k + 1], s) != cudaSuccess)
                        st = fail(ctx, GS_ERR_CUDA, "autotuner trial launch");
                float ms[4] = {0, 0, 0, 0};
                if (st == GS_OK && cudaEventSynchronize(e[8]) == cudaSuccess)
                    for (int k = 0; k < 8; ++k) {
                        float x = 0.0f;
                        cudaEventElapsedTime(&x, e[k], e[k + 1]);
                        ms[seq[k]] += x;
                    }
                for (cudaEvent_t x : e)
                    if (x)
                        cudaEventDestroy(x);
                for (cudaGraphExec_t x : g)
                    if (x)
                        cudaGraphExecDestroy(x);
                GS_TRY(st);
                int best = 0;
                for (int k = 1; k < 4; ++k)
                    if (ms[k] < ms[best])
                        best = k;
                sched = best + 1;
                ctx->schedule[key] = sched;
                ++ctx->tuned;
                gsl::pose_init(pa, s);  // back to the initial poses
                marking = prof;
            } else {
                sched = 1;
            }
        }
        ordered = sched == 2 || sched == 4;
        persistent = sched >= 3;
        const int sched_run = sched;
        GS_CUDA(cudaMemsetAsync(p.flags, 0, sizeof(int), s));
        GS_CUDA(cudaMemsetAsync(pairs, 0, sizeof(unsigned long long) * 2 * ntl, s));
        if (iters > 0) {
            const long long c0 = gsl::g_launches;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            GS_TRY(capture(&exec, &graph));
            captured = gsl::g_launches - c0;
            if (mark_err != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                return fail(ctx, GS_ERR_CUDA, std::string("profile events: ") + cudaGetErrorString(mark_err));
            }
            // kernel nodes and the phase-boundary event nodes of the graph
            size_t nn = 0;
            cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(graph, nodes.data(), &nn);
            cudaGraphNode_t evnode[kPhases + 1] = {};
            for (cudaGraphNode_t nd_ : nodes) {
                cudaGraphNodeType t;
                cudaGraphNodeGetType(nd_, &t);
                if (t == cudaGraphNodeTypeKernel)
                    ++graph_kernels;
                if (t == cudaGraphNodeTypeEventRecord) {
                    cudaEvent_t e;
                    cudaGraphEventRecordNodeGetEvent(nd_, &e);
                    for (int k = 0; k <= kPhases; ++k)
                        if (e == ctx->tev[k])
                            evnode[k] = nd_;
                }
            }
            cudaError_t le = cudaSuccess;
            for (int it = 0; it < iters && le == cudaSuccess; ++it) {
                if (prof)
                    for (int k = 0; k <= kPhases && le == cudaSuccess; ++k)
                        if (evnode[k])
                            le = cudaGraphExecEventRecordNodeSetEvent(exec, evnode[k],
                                                                     ctx->pool[(size_t)it * (kPhases + 1) + k]);
                if (le == cudaSuccess)
                    le = cudaGraphLaunch(exec, s);
            }
            cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            if (le != cudaSuccess)
                return fail(ctx, GS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(le));
        }
        // residual eps at the final poses, then Eq. 7
        r.tile_pairs = nullptr;
        r.tile_order = nullptr;
        r.queue = nullptr;
        gsl::project(project_args(P, D, p, pose32, opt, false), s);
        r.vals = p.vals[run_bin(b, s)];
        gsl::forward(r, true, s);
        gsl::track_loss(ta, s);
        gsl::PoseArgs fa = pa;
        fa.tile_twist = nullptr;
        fa.update = 0;
        gsl::pose_update(fa, s);
        gsl::FuseArgs f{};
        f.pose64 = pose64;
        f.eps = lossd;
        f.reverse = rev;
        f.prob_first = pf;
        f.prob_count = pc;
        f.n_problems = n_problems;
        f.T_out = Tdev;
        f.conf = confd;
        f.est_out = est;
        gsl::fuse(f, s);
        GS_CUDA(cudaGetLastError());
        if (ao) {
            // stream-ordered results in the caller's device buffers and a
            // device status word; nothing is read back, nothing is redone
            k_async_status<<<1, 32, 0, s>>>(p.flags, lossd, nv, ao->status);
            ++gsl::g_launches;
            GS_CUDA(cudaMemcpyAsync(ao->T, Tdev, 12 * sizeof(double) * n_problems, cudaMemcpyDeviceToDevice, s));
            GS_CUDA(cudaMemcpyAsync(ao->conf, confd, sizeof(double) * n_problems, cudaMemcpyDeviceToDevice, s));
            if (ao->eps)
                GS_CUDA(cudaMemcpyAsync(ao->eps, lossd, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
            if (ao->est)
                GS_CUDA(cudaMemcpyAsync(ao->est, est, 12 * sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
            GS_CUDA(cudaGetLastError());
            gs_stats_t &st = ctx->stats;
            st.kernel_launches = (gsl::g_launches - l0) - captured + graph_kernels * iters;
            st.n_dups = nd;
            st.n_pixels = P.n_pix;
            st.iterations = iters;
            st.schedule = sched_run;
            return GS_OK;
        }
        int flags = 0;
        GS_TRY(read_flags(ctx, p, s, &flags));
        if (flags & gsk::kFlagNonFinite)
            return fail(ctx, GS_ERR_NONFINITE, "non-finite Gaussian parameter");
        if (flags & gsk::kFlagTimeout)
            return fail(ctx, GS_ERR_TIMEOUT, "a sort pass gave up waiting for an earlier tile");
        if (flags & gsk::kFlagCapacity) {
            headroom = std::max(2.0 * headroom, 1.5);  // the lists outgrew the headroom: redo with more
            continue;
        }
        std::vector<double> epsh(nv);
        std::vector<unsigned long long> pairs_h(2 * ntl);
        GS_CUDA(cudaMemcpyAsync(T_out, Tdev, 12 * sizeof(double) * n_problems, cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(conf_out, confd, sizeof(double) * n_problems, cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(epsh.data(), lossd, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(pairs_h.data(), pairs, 2 * ntl * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                s));
        if (est_out)
            GS_CUDA(cudaMemcpyAsync(est_out, est, 12 * nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (grad_out)
            GS_CUDA(cudaMemcpyAsync(grad_out, gradd, 6 * nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaStreamSynchronize(s));
        gs_stats_t &st = ctx->stats;
        st.kernel_launches = (gsl::g_launches - l0) - captured + graph_kernels * iters + trial_kernels;
        st.n_dups = nd;
        st.n_pixels = P.n_pix;
        st.iterations = iters;
        st.schedule = sched_run;
        for (size_t k = 0; k < ntl; ++k) {
            st.pairs += (int64_t)pairs_h[k];
            st.contributing += (int64_t)pairs_h[ntl + k];
        }
        if (prof)
            for (int it = 0; it < iters; ++it)
                for (int k = 0; k < kPhases; ++k) {
                    float ms = 0.0f;
                    if (cudaEventElapsedTime(&ms, ctx->pool[(size_t)it * (kPhases + 1) + k],
                                             ctx->pool[(size_t)it * (kPhases + 1) + k + 1]) == cudaSuccess)
                        st.phase_ms[k] += ms;
                }
        if (eps_out)
            std::memcpy(eps_out, epsh.data(), nv * sizeof(double));
        for (double e : epsh)
            if (!std::isfinite(e))
                return fail(ctx, GS_ERR_DIVERGED, "registration residual is not finite");
        return GS_OK;
    }
    return fail(ctx, GS_ERR_CAPACITY, "tile duplicate lists kept outgrowing their capacity");
}

}  // namespace

// ===========================================================================
// gs_render_noalloc: gs_render on a fixed device array instead of a context
// arena, for callers that may not allocate device memory
// ===========================================================================
namespace {

// the fixed scratch; every GPU that loads the library holds it until exit
__device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

// The scratch's device address belongs to the module as loaded in one CUDA
// context: the primary context of a device, a context the caller created
// with the driver API, or the primary context re-created after
// cudaDeviceReset each have their own.  The address is therefore looked up
// once per context (keyed by the driver's context id, which is never
// reused within a process) with that context current, and cached.
std::mutex g_noalloc_mutex;
std::map<unsigned long long, void *> g_noalloc_addr;
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// id of the calling thread's current context, or false if it cannot be had
bool current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = (CtxGetCurrentFn)f1;
            get_id = (CtxGetIdFn)f2;
        }
        cudaGetLastError();
        looked_up = true;
    }
    void *c = nullptr;
    return get_current && get_id && get_current(&c) == 0 && c && get_id(c, id) == 0;
}

// Device address of the scratch in the current context.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress (once per context; on every call if the context id
// cannot be read).  The first call in a context does this set-up.
gs_status_t noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    const bool keyed = current_context_id(&id);
    if (keyed) {
        const auto it = g_noalloc_addr.find(id);
        if (it != g_noalloc_addr.end()) {
            *out = it->second;
            return GS_OK;
        }
    }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    if (keyed)
        g_noalloc_addr[id] = p;
    *out = p;
    return GS_OK;
}

// bump allocator over the fixed scratch (256-byte aligned pieces)
struct FixedCarve {
    char *base;
    size_t off, cap;
    template <typename T>
    T *take(size_t count)
    {
        const size_t bytes = ((count ? count : 1) * sizeof(T) + 255) & ~(size_t)255;
        if (off + bytes > cap)
            return nullptr;
        T *p = (T *)(base + off);
        off += bytes;
        return p;
    }
};

}  // namespace

extern "C" gs_status_t gs_render_noalloc(const gs_gaussians_t *g, const float *poses, const gs_camera_t *cams,
                                         int n_cams, const gs_options_t *opt, float *rgb, float *depth, float *alpha,
                                         float *t_final, int32_t *last, gs_stream_t stream)
{
    gs_ctx *ctx = nullptr;  // no context: failures are reported by status only
    GS_TRY(check_options(ctx, opt));
    GS_TRY(check_gaussians(ctx, g, "submap"));
    if (!poses || n_cams < 0 || (n_cams > 0 && !cams))
        return GS_ERR_INVALID_ARG;
    for (int c = 0; c < n_cams; ++c)
        GS_TRY(check_camera(ctx, cams[c]));
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    GS_TRY(noalloc_scratch(&base));
    Plan P = plan_for(g, cams, n_cams);
    GS_TRY(finalize(ctx, P));
    FixedCarve cv{(char *)base, 0, GS_NOALLOC_SCRATCH_BYTES};
    const size_t R = P.n_records ? P.n_records : 1;
    VpDesc *vps = cv.take<VpDesc>(P.vps.size());
    GroupDesc *groups = cv.take<GroupDesc>(P.groups.size());
    uint32_t *tile_vp = cv.take<uint32_t>(P.tile_vp.size());
    Pipe p;
    p.rec = cv.take<float4>(3 * R);
    p.counts = cv.take<int32_t>(R);
    p.partials = cv.take<uint32_t>(gsl::scan_partials(R));
    p.ndups = cv.take<uint32_t>(4);
    p.flags = cv.take<int>(4);
    p.ranges = cv.take<uint2>(P.n_tiles ? P.n_tiles : 1);
    if (!vps || !groups || !tile_vp || !p.rec || !p.counts || !p.partials || !p.ndups || !p.flags || !p.ranges)
        return GS_ERR_CAPACITY;
    if (!P.vps.empty() && cudaMemcpyAsync(vps, P.vps.data(), P.vps.size() * sizeof(VpDesc), cudaMemcpyHostToDevice,
                                          s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (!P.groups.empty() && cudaMemcpyAsync(groups, P.groups.data(), P.groups.size() * sizeof(GroupDesc),
                                             cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (!P.tile_vp.empty() && cudaMemcpyAsync(tile_vp, P.tile_vp.data(), P.tile_vp.size() * sizeof(uint32_t),
                                              cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GS_ERR_CUDA;
    DevPlan D;
    D.vps = vps;
    D.groups = groups;
    D.tile_vp = tile_vp;
    // the scratch keeps the previous call's contents: clear the status word
    if (cudaMemsetAsync(p.flags, 0, sizeof(int), s) != cudaSuccess)
        return GS_ERR_CUDA;
    gsl::project(project_args(P, D, p, poses, opt), s);
    gsl::BinArgs b = bin_args(P, D, p);
    gsl::bin_count(b, s);
    uint32_t nd = 0;
    if (cudaMemcpyAsync(&nd, p.ndups, sizeof nd, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (nd == 0xffffffffu)
        return GS_ERR_CAPACITY;
    const uint32_t cap = std::max<uint32_t>(nd, 1);
    p.keys[0] = cv.take<uint64_t>(cap);
    p.keys[1] = cv.take<uint64_t>(cap);
    p.vals[0] = cv.take<uint32_t>(cap);
    p.vals[1] = cv.take<uint32_t>(cap);
    const size_t hn = gsl::sort_hist_entries(cap);
    p.hist = cv.take<uint32_t>(hn);
    p.histp = cv.take<uint32_t>(gsl::scan_partials(hn));
    if (!p.keys[0] || !p.keys[1] || !p.vals[0] || !p.vals[1] || !p.hist || !p.histp)
        return GS_ERR_CAPACITY;
    p.cap = cap;
    b = bin_args(P, D, p);
    const int cur = gsl::bin(b, s);  // clears the tile ranges itself
    gsl::RasterArgs r = raster_args(P, D, p, cur, opt);
    r.out_rgb = rgb;
    r.out_depth = depth;
    r.out_alpha = alpha;
    r.t_final = t_final;
    r.last = last;
    gsl::forward(r, false, s);
    if (cudaGetLastError() != cudaSuccess)
        return GS_ERR_CUDA;
    int flags = 0;
    if (cudaMemcpyAsync(&flags, p.flags, sizeof flags, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GS_ERR_CUDA;
    return (flags & gsk::kFlagNonFinite) ? GS_ERR_NONFINITE : GS_OK;
}

// ===========================================================================
// Serving: continuous batching of registration requests (gs_server_*)
// ===========================================================================
namespace {

// per keyframe problem: pose64 [12], Adam state [13], pivot [3], camera-frame
// pivot [3], exposure state [7]
constexpr int kVpState = 38;

struct ServerReq {
    gs_gaussians_t src{}, tgt{};
    gs_options_t opt{};  // learning rates and loss of this request
    std::vector<gs_view_t> sv, tv;
    int iters = 0;
    int state = 0;       // 0 waiting, 1 in flight, 2 done
    int ran = 0;         // graph iterations run: iters pose updates + 1 at the frozen pose
    bool fresh = true;   // optimiser state not created yet
    int vp_first = 0;    // first keyframe problem in the current plan
    std::vector<double> st;  // [vps][kVpState]
    double T[12] = {}, conf = 0;
    std::vector<double> eps;
    double t_submit = 0, t_done = 0;
    size_t est_bytes = 0;  // scratch footprint from its measured tile duplicates
    int64_t dups = 0;      // tile duplicates at its starting poses, counted at submission
    bool held = false;     // once kept waiting by the memory budget
    int n_vps() const { return (int)(sv.size() + tv.size()); }
};

}  // namespace

struct gs_server {
    gs_ctx *ctx = nullptr;
    gs_ctx *mctx = nullptr;  // footprint measurement (own scratch and stream: never the in-flight plan's)
    int64_t measured = 0, held_back = 0;
    gs_options_t opt{};
    int max_kf = 0, max_round = 0;
    size_t budget = 0;
    std::vector<ServerReq> reqs;  // indexed by id
    std::vector<int64_t> waiting;  // FIFO (front = index `wait_head`)
    size_t wait_head = 0;
    std::vector<int64_t> active;
    bool dirty = true;
    double headroom = 1.5;
    int64_t rounds = 0, replans = 0, n_done = 0;
    std::chrono::steady_clock::time_point t0;
    // the current plan and its device state
    Plan P;
    DevPlan D;
    Pipe p;
    int n_vps = 0, n_problems = 0;
    float *pose32 = nullptr, *tloss = nullptr, *tf = nullptr;
    double *pose64 = nullptr, *adam = nullptr, *pivot = nullptr, *ccam = nullptr, *cent = nullptr,
           *lossd = nullptr, *Tdev = nullptr, *confd = nullptr;
    float2 *ttw = nullptr;
    int32_t *last = nullptr, *rev = nullptr, *pf = nullptr, *pc = nullptr;
    uint8_t *code = nullptr;
    gsl::PoseArgs pa{};
    cudaGraphExec_t exec = nullptr;
};

namespace {

double srv_now(const gs_server *srv)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - srv->t0).count();
}

// Scratch of a request in a plan, from its measured tile duplicates nd:
// per record 100 B (record 48, auxiliary 32, count 4, list entry 16); per
// list entry of capacity (headroom x nd; a plan's 64 Ki spare entries come
// out of the arena's slack) 12.5 B (depth bits, two value buffers,
// histogram share); per pixel 9 B (final transmittance,
// last contributor, loss sign code), 12 B more for tracking masks; per tile
// 92 B (range, keyframe, loss, twist, counters, cursors, order); per
// keyframe problem its FP64 optimiser state.
size_t footprint_bytes(const ServerReq &r, int64_t nd, double headroom)
{
    double rec = 0, px = 0, tiles = 0;
    auto add = [&](const gs_gaussians_t &g, const gs_view_t &v) {
        rec += (double)g.n;
        px += (double)v.cam.width * v.cam.height;
        tiles += (double)((v.cam.width + GS_TILE - 1) / GS_TILE) * ((v.cam.height + GS_TILE - 1) / GS_TILE);
    };
    for (const gs_view_t &v : r.sv)
        add(r.tgt, v);
    for (const gs_view_t &v : r.tv)
        add(r.src, v);
    const double per_px = 9.0 + (r.opt.tracking_loss ? 12.0 : 0.0);
    const double b = rec * 100.0 + headroom * (double)nd * 12.5 + px * per_px + tiles * 92.0 +
                     (double)r.n_vps() * kVpState * 8.0;
    return (size_t)b + 4096;
}

// Counts the request's tile duplicates at its starting poses (the identity)
// on the measuring context: projection and list counting only, on that
// context's own stream (synchronised), so nothing of the plan in flight is
// touched.
gs_status_t srv_measure(gs_server *srv, ServerReq &r)
{
    if (!srv->mctx)
        GS_TRY(gs_ctx_create(srv->ctx->device, 0, &srv->mctx));
    gs_ctx *ctx = srv->mctx;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = ctx->cap;
    Plan P;
    int sets = 0;
    add_problem(P, &r.src, &r.tgt, r.sv.data(), (int)r.sv.size(), r.tv.data(), (int)r.tv.size(), 0, sets, &r.opt);
    GS_TRY(finalize(ctx, P));
    DevPlan D;
    GS_TRY(upload_plan(ctx, P, D, s));
    Pipe p;
    GS_TRY(alloc_pipe(ctx, P, false, p));
    const int nv = (int)P.vps.size();
    std::vector<float> ident((size_t)12 * nv, 0.0f);
    for (int v = 0; v < nv; ++v)
        ident[12 * v] = ident[12 * v + 5] = ident[12 * v + 10] = 1.0f;
    float *pose32 = nullptr;
    GS_TRY(upload(ctx, S_POSE32, ident, &pose32, s));
    GS_CUDA(cudaMemsetAsync(p.flags, 0, sizeof(int), s));
    gsl::project(project_args(P, D, p, pose32, &r.opt), s);
    gsl::BinArgs b = bin_args(P, D, p);
    gsl::bin_count(b, s);
    uint32_t nd = 0;
    GS_CUDA(cudaMemcpyAsync(&nd, p.ndups, sizeof nd, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (nd == 0xffffffffu)
        return fail(srv->ctx, GS_ERR_CAPACITY, "more than 2^32 tile duplicates");
    r.dups = nd;
    ++srv->measured;
    return GS_OK;
}

// admits waiting requests (FIFO) within the keyframe and memory limits
void srv_admit(gs_server *srv)
{
    int kf = 0;
    size_t bytes = 0;
    for (int64_t id : srv->active) {
        kf += srv->reqs[id].n_vps();
        bytes += srv->reqs[id].est_bytes;
    }
    while (srv->wait_head < srv->waiting.size()) {
        ServerReq &r = srv->reqs[srv->waiting[srv->wait_head]];
        const bool empty = srv->active.empty();
        if (!empty && (kf + r.n_vps() > srv->max_kf || bytes + r.est_bytes > srv->budget)) {
            if (!r.held && kf + r.n_vps() <= srv->max_kf) {
                r.held = true;  // kept waiting by the memory budget
                ++srv->held_back;
            }
            break;
        }
        kf += r.n_vps();
        bytes += r.est_bytes;
        r.state = 1;
        srv->active.push_back(srv->waiting[srv->wait_head++]);
        srv->dirty = true;
    }
    if (srv->wait_head > 4096 && srv->wait_head * 2 > srv->waiting.size()) {
        srv->waiting.erase(srv->waiting.begin(), srv->waiting.begin() + (ptrdiff_t)srv->wait_head);
        srv->wait_head = 0;
    }
}

// builds the plan of the in-flight requests, restores their state and
// captures one iteration into a graph
gs_status_t srv_replan(gs_server *srv, cudaStream_t s)
{
    gs_ctx *ctx = srv->ctx;
    if (srv->exec) {
        cudaGraphExecDestroy(srv->exec);
        srv->exec = nullptr;
    }
    Plan &P = srv->P;
    P = Plan{};
    int sets = 0;
    for (size_t i = 0; i < srv->active.size(); ++i) {
        ServerReq &r = srv->reqs[srv->active[i]];
        r.vp_first = (int)P.vps.size();
        add_problem(P, &r.src, &r.tgt, r.sv.data(), (int)r.sv.size(), r.tv.data(), (int)r.tv.size(), (int)i, sets,
                    &r.opt);
        for (int v = r.vp_first; v < (int)P.vps.size(); ++v)
            P.vps[v].iters = r.iters;
    }
    GS_TRY(finalize(ctx, P));
    DevPlan &D = srv->D;
    GS_TRY(upload_plan(ctx, P, D, s));
    const int nv = (int)P.vps.size(), n_sets = (int)P.set_vp.size(), np = (int)srv->active.size();
    srv->n_vps = nv;
    srv->n_problems = np;
    Pipe &p = srv->p;
    p = Pipe{};
    GS_TRY(alloc_pipe(ctx, P, true, p));
    const size_t npix = (size_t)std::max<int64_t>(P.n_pix, 1), ntl = (size_t)std::max<uint64_t>(P.n_tiles, 1);
    GS_TRY(wsT(ctx, S_POSE32, 12 * (size_t)nv, &srv->pose32));
    GS_TRY(wsT(ctx, S_POSE64, 12 * (size_t)nv, &srv->pose64));
    GS_TRY(wsT(ctx, S_ADAM, 13 * (size_t)nv, &srv->adam));
    GS_TRY(wsT(ctx, S_PIVOT, 3 * (size_t)nv, &srv->pivot));
    GS_TRY(wsT(ctx, S_CCAM, 3 * (size_t)nv, &srv->ccam));
    GS_TRY(wsT(ctx, S_CENT, 3 * (size_t)std::max(n_sets, 1), &srv->cent));
    GS_TRY(wsT(ctx, S_LOSS, (size_t)nv, &srv->lossd));
    GS_TRY(wsT(ctx, S_TF, npix, &srv->tf));
    GS_TRY(wsT(ctx, S_LAST, npix, &srv->last));
    GS_TRY(wsT(ctx, S_CODE, npix, &srv->code));
    GS_TRY(wsT(ctx, S_TLOSS, ntl, &srv->tloss));
    GS_TRY(wsT(ctx, S_TTWIST, 6 * ntl, &srv->ttw));
    GS_TRY(wsT(ctx, S_TOUT, 12 * (size_t)np, &srv->Tdev));
    GS_TRY(wsT(ctx, S_CONF, (size_t)np, &srv->confd));
    std::vector<int32_t> revh(nv), pfh(np, 0), pch(np, 0);
    for (int v = 0; v < nv; ++v) {
        revh[v] = P.vps[v].reverse;
        const int q = P.vps[v].problem;
        if (pch[q]++ == 0)
            pfh[q] = v;
    }
    GS_TRY(upload(ctx, S_REV, revh, &srv->rev, s));
    GS_TRY(upload(ctx, S_PFIRST, pfh, &srv->pf, s));
    GS_TRY(upload(ctx, S_PCOUNT, pch, &srv->pc, s));

    gsl::PoseArgs &pa = srv->pa;
    pa = gsl::PoseArgs{};
    pa.vps = D.vps;
    pa.n_vps = nv;
    pa.tile_twist = srv->ttw;
    pa.tile_loss = srv->tloss;
    pa.pose64 = srv->pose64;
    pa.pose32 = srv->pose32;
    pa.adam = srv->adam;
    pa.pivot = srv->pivot;
    pa.c_cam = srv->ccam;
    pa.centroid = srv->cent;
    pa.loss = srv->lossd;
    pa.lr_rot = srv->opt.lr_rot;
    pa.lr_trans = srv->opt.lr_trans;
    pa.beta1 = srv->opt.beta1;
    pa.beta2 = srv->opt.beta2;
    pa.eps = srv->opt.adam_eps;
    pa.lr_final = srv->opt.lr_final;
    pa.iters = 0;  // every keyframe carries its request's count
    pa.update = 1;
    gsl::RasterArgs expo_r{};
    GS_TRY(alloc_exposure(ctx, P, pa, expo_r));

    // fresh requests start at the identity; the others resume their state
    gsl::centroids(D.vps, D.set_vp, n_sets, srv->cent, s);
    gsl::pose_init(pa, s);
    for (int64_t id : srv->active) {
        const ServerReq &r = srv->reqs[id];
        if (r.fresh)
            continue;
        for (int k = 0; k < r.n_vps(); ++k) {
            const double *st = r.st.data() + (size_t)k * kVpState;
            const size_t v = (size_t)r.vp_first + k;
            GS_CUDA(cudaMemcpyAsync(srv->pose64 + 12 * v, st, 12 * sizeof(double), cudaMemcpyHostToDevice, s));
            GS_CUDA(cudaMemcpyAsync(srv->adam + 13 * v, st + 12, 13 * sizeof(double), cudaMemcpyHostToDevice, s));
            GS_CUDA(cudaMemcpyAsync(srv->pivot + 3 * v, st + 25, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
            GS_CUDA(cudaMemcpyAsync(srv->ccam + 3 * v, st + 28, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
            GS_CUDA(cudaMemcpyAsync(pa.expo + 7 * v, st + 31, 7 * sizeof(double), cudaMemcpyHostToDevice, s));
        }
    }
    k_to_float<<<(12 * nv + 255) / 256, 256, 0, s>>>(srv->pose64, srv->pose32, 12 * nv);
    ++gsl::g_launches;
    gsl::exposure_floats(pa.expo, pa.expo32, nv, s);
    // size the duplicate lists at the current poses
    int cur = 0;
    uint32_t nd = 0;
    GS_TRY(project_and_bin(ctx, P, D, p, srv->pose32, &srv->opt, s, &cur, &nd));
    const uint64_t want = (uint64_t)(srv->headroom * nd) + 65536;
    if (p.cap < want)
        GS_TRY(alloc_sort(ctx, want, p));
    const gsl::BinArgs b = bin_args(P, D, p);
    gsl::RasterArgs r = raster_args(P, D, p, 0, &srv->opt);
    r.t_final = srv->tf;
    r.last = srv->last;
    r.code = srv->code;
    r.tile_loss = srv->tloss;
    r.tile_twist = srv->ttw;
    r.c_cam = srv->ccam;
    r.tile_pairs = nullptr;
    r.expo32 = expo_r.expo32;
    r.tile_expo = expo_r.tile_expo;
    r.exposure = any_exposure(P);
    gsl::TrackArgs ta;
    GS_TRY(alloc_track(ctx, P, D, r, ta, srv->tloss, s));
    GS_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    gsl::project(project_args(P, D, p, srv->pose32, &srv->opt, false), ctx->cap);
    r.vals = p.vals[run_bin(b, ctx->cap)];
    if (srv->opt.fuse_compositing && ta.n_track == 0) {
        gsl::forward_backward(r, ctx->cap);
    } else {
        gsl::forward(r, true, ctx->cap);
        gsl::track_loss(ta, ctx->cap);
        gsl::backward(r, true, false, ctx->cap);
    }
    gsl::pose_update(pa, ctx->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &graph);
    if (ce != cudaSuccess || !graph)
        return fail(ctx, GS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&srv->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        srv->exec = nullptr;
        return fail(ctx, GS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    srv->dirty = false;
    ++srv->replans;
    return GS_OK;
}

gs_status_t srv_round(gs_server *srv, cudaStream_t s, int64_t *done_ids, int max_done, int *n_done)
{
    gs_ctx *ctx = srv->ctx;
    *n_done = 0;
    srv_admit(srv);
    if (srv->active.empty())
        return GS_OK;
    for (int attempt = 0;; ++attempt) {
        if (srv->dirty)
            GS_TRY(srv_replan(srv, s));
        int S = std::max(srv->max_round, 1);
        for (int64_t id : srv->active) {
            const ServerReq &r = srv->reqs[id];
            S = std::min(S, r.iters + 1 - r.ran);
        }
        S = std::max(S, 1);
        GS_CUDA(cudaMemsetAsync(srv->p.flags, 0, sizeof(int), s));
        for (int it = 0; it < S; ++it)
            GS_CUDA(cudaGraphLaunch(srv->exec, s));
        const int nv = srv->n_vps;
        std::vector<double> pose(12 * (size_t)nv), adam(13 * (size_t)nv), piv(3 * (size_t)nv), cc(3 * (size_t)nv),
            loss(nv), expo(7 * (size_t)nv);
        int flags = 0;
        GS_CUDA(cudaMemcpyAsync(&flags, srv->p.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(pose.data(), srv->pose64, pose.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(adam.data(), srv->adam, adam.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(piv.data(), srv->pivot, piv.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(cc.data(), srv->ccam, cc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(loss.data(), srv->lossd, loss.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(expo.data(), srv->pa.expo, expo.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaStreamSynchronize(s));
        if (flags & gsk::kFlagNonFinite)
            return fail(ctx, GS_ERR_NONFINITE, "non-finite Gaussian parameter in an in-flight request");
        if (flags & gsk::kFlagTimeout)
            return fail(ctx, GS_ERR_TIMEOUT, "a sort pass gave up waiting for an earlier tile");
        if (flags & gsk::kFlagCapacity) {
            // the lists outgrew their headroom: redo the round from the saved states
            if (attempt >= 3)
                return fail(ctx, GS_ERR_CAPACITY, "tile duplicate lists kept outgrowing their capacity");
            srv->headroom *= 2.0;
            srv->dirty = true;
            continue;
        }
        ++srv->rounds;
        std::vector<int64_t> retiring;
        for (int64_t id : srv->active) {
            ServerReq &r = srv->reqs[id];
            r.st.resize((size_t)r.n_vps() * kVpState);
            for (int k = 0; k < r.n_vps(); ++k) {
                const size_t v = (size_t)r.vp_first + k;
                double *st = r.st.data() + (size_t)k * kVpState;
                std::memcpy(st, &pose[12 * v], 12 * sizeof(double));
                std::memcpy(st + 12, &adam[13 * v], 13 * sizeof(double));
                std::memcpy(st + 25, &piv[3 * v], 3 * sizeof(double));
                std::memcpy(st + 28, &cc[3 * v], 3 * sizeof(double));
                std::memcpy(st + 31, &expo[7 * v], 7 * sizeof(double));
            }
            r.fresh = false;
            r.ran += S;
            if (r.ran >= r.iters + 1)
                retiring.push_back(id);
        }
        if (retiring.empty())
            return GS_OK;
        // Eq. 7 over the in-flight problems (losses measured at the frozen poses)
        gsl::FuseArgs f{};
        f.pose64 = srv->pose64;
        f.eps = srv->lossd;
        f.reverse = srv->rev;
        f.prob_first = srv->pf;
        f.prob_count = srv->pc;
        f.n_problems = srv->n_problems;
        f.T_out = srv->Tdev;
        f.conf = srv->confd;
        f.est_out = nullptr;
        gsl::fuse(f, s);
        std::vector<double> T(12 * (size_t)srv->n_problems), conf(srv->n_problems);
        GS_CUDA(cudaMemcpyAsync(T.data(), srv->Tdev, T.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaMemcpyAsync(conf.data(), srv->confd, conf.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaStreamSynchronize(s));
        const double now = srv_now(srv);
        std::vector<int64_t> keep;
        for (size_t i = 0; i < srv->active.size(); ++i) {
            const int64_t id = srv->active[i];
            ServerReq &r = srv->reqs[id];
            if (r.ran < r.iters + 1) {
                keep.push_back(id);
                continue;
            }
            std::memcpy(r.T, &T[12 * i], 12 * sizeof(double));
            r.conf = conf[i];
            r.eps.assign(loss.begin() + r.vp_first, loss.begin() + r.vp_first + r.n_vps());
            r.state = 2;
            r.t_done = now;
            r.st.clear();
            r.st.shrink_to_fit();
            ++srv->n_done;
            if (done_ids && *n_done < max_done)
                done_ids[*n_done] = id;
            ++*n_done;
        }
        srv->active.swap(keep);
        srv->dirty = true;
        return GS_OK;
    }
}

}  // namespace

extern "C" {

gs_status_t gs_server_create(int device, size_t budget, int max_keyframes, int max_round_iters,
                             const gs_options_t *opt, gs_server_t **out)
{
    if (!out || !opt || max_keyframes < 1 || max_round_iters < 1)
        return GS_ERR_INVALID_ARG;
    *out = nullptr;
    // admission keeps the estimated scratch within `budget`; the arena gets
    // slack above it for the estimate's error
    const size_t adm = budget ? budget : ((size_t)16 << 30);
    gs_ctx_t *ctx = nullptr;
    GS_TRY(gs_ctx_create(device, adm + std::max(adm / 4, (size_t)256 << 20), &ctx));
    const gs_status_t st = check_options(ctx, opt);
    if (st != GS_OK) {
        gs_ctx_destroy(ctx);
        return st;
    }
    gs_server *srv = new gs_server();
    srv->ctx = ctx;
    srv->opt = *opt;
    srv->max_kf = max_keyframes;
    srv->max_round = max_round_iters;
    srv->budget = adm;
    srv->t0 = std::chrono::steady_clock::now();
    *out = srv;
    return GS_OK;
}

gs_status_t gs_server_destroy(gs_server_t *srv)
{
    if (!srv)
        return GS_ERR_INVALID_ARG;
    {
        DeviceGuard g(srv->ctx->device);
        if (srv->exec)
            cudaGraphExecDestroy(srv->exec);
    }
    gs_ctx_destroy(srv->ctx);
    if (srv->mctx)
        gs_ctx_destroy(srv->mctx);
    delete srv;
    return GS_OK;
}

const char *gs_server_last_error(const gs_server_t *srv) { return srv ? srv->ctx->err.c_str() : "null server"; }

gs_status_t gs_server_submit(gs_server_t *srv, const gs_problem_t *q, int iters, int64_t *id_out)
{
    if (!srv || !q || !id_out)
        return GS_ERR_INVALID_ARG;
    gs_ctx *ctx = srv->ctx;
    if (iters < 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "iters must be >= 0");
    GS_TRY(check_problem(ctx, *q));
    if (q->opt)
        GS_TRY(check_options(ctx, q->opt));
    if (q->n_src_views + q->n_tgt_views > srv->max_kf)
        return fail(ctx, GS_ERR_INVALID_ARG, "request has more keyframes than the server's max_keyframes");
    ServerReq r;
    r.opt = q->opt ? *q->opt : srv->opt;
    r.src = q->src;
    r.tgt = q->tgt;
    r.sv.assign(q->src_views, q->src_views + q->n_src_views);
    r.tv.assign(q->tgt_views, q->tgt_views + q->n_tgt_views);
    r.iters = iters;
    const gs_status_t ms = srv_measure(srv, r);
    if (ms != GS_OK)
        return fail(ctx, ms, "counting the request's tile lists: " + (srv->mctx ? srv->mctx->err : std::string()));
    r.est_bytes = footprint_bytes(r, r.dups, srv->headroom);
    if (r.est_bytes > srv->budget)
        return fail(ctx, GS_ERR_OOM, "the request's scratch (" + std::to_string(r.est_bytes) +
                                         " bytes for its measured tile lists) exceeds the server's budget");
    r.t_submit = srv_now(srv);
    *id_out = (int64_t)srv->reqs.size();
    srv->waiting.push_back(*id_out);
    srv->reqs.push_back(std::move(r));
    return GS_OK;
}

gs_status_t gs_server_step(gs_server_t *srv, gs_stream_t stream, int64_t *done_ids, int max_done, int *n_done)
{
    if (!srv || !n_done || max_done < 0)
        return GS_ERR_INVALID_ARG;
    DeviceGuard g(srv->ctx->device);
    const gs_status_t st = srv_round(srv, (cudaStream_t)stream, done_ids, max_done, n_done);
    if (st != GS_OK)
        srv->dirty = true;
    return st;
}

gs_status_t gs_server_poll(gs_server_t *srv, int64_t id, int *state, double *T_out, double *confidence,
                           double *eps_out, double *t_submit, double *t_done)
{
    if (!srv || id < 0 || id >= (int64_t)srv->reqs.size())
        return GS_ERR_INVALID_ARG;
    const ServerReq &r = srv->reqs[id];
    if (state)
        *state = r.state;
    if (t_submit)
        *t_submit = r.t_submit;
    if (r.state != 2)
        return GS_OK;
    if (T_out)
        std::memcpy(T_out, r.T, sizeof r.T);
    if (confidence)
        *confidence = r.conf;
    if (eps_out)
        std::memcpy(eps_out, r.eps.data(), r.eps.size() * sizeof(double));
    if (t_done)
        *t_done = r.t_done;
    return GS_OK;
}

gs_status_t gs_server_admission(const gs_server_t *srv, int64_t out[3])
{
    if (!srv || !out)
        return GS_ERR_INVALID_ARG;
    size_t bytes = 0;
    for (int64_t id : srv->active)
        bytes += srv->reqs[id].est_bytes;
    out[0] = srv->measured;
    out[1] = srv->held_back;
    out[2] = (int64_t)bytes;
    return GS_OK;
}

gs_status_t gs_server_footprint(const gs_server_t *srv, int64_t id, int64_t *dups, int64_t *bytes)
{
    if (!srv || id < 0 || id >= (int64_t)srv->reqs.size())
        return GS_ERR_INVALID_ARG;
    if (dups)
        *dups = srv->reqs[id].dups;
    if (bytes)
        *bytes = (int64_t)srv->reqs[id].est_bytes;
    return GS_OK;
}

gs_status_t gs_server_counts(const gs_server_t *srv, int64_t out[5])
{
    if (!srv || !out)
        return GS_ERR_INVALID_ARG;
    out[0] = (int64_t)(srv->waiting.size() - srv->wait_head);
    out[1] = (int64_t)srv->active.size();
    out[2] = srv->n_done;
    out[3] = srv->rounds;
    out[4] = srv->replans;
    return GS_OK;
}

}  // extern "C"
