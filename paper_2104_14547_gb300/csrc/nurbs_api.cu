// C-ABI of libnurbs: planning (tiling a ragged batch, workspace layout),
// binding a workspace, and the execution entry points declared in nurbs.h.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nurbs.h"
#include "nurbs_curve.cuh"
#include "nurbs_kernel.cuh"

using namespace nurbs;

namespace {

thread_local int32_t g_last_cuda_error = 0;

// An NVTX range named after the entry point, around its host work and launches
// (profilers can filter on it, e.g. ncu --nvtx); with no tool attached a push and
// a pop cost a pointer test each.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int align4(int x) { return (x + 3) & ~3; }

// Shared adjoint of a single-tile item: the n1 x m1 block plus (p+1) overflow
// rows per row group.
inline size_t smem_adjoint_bytes(const ItemDev& it, int nwr)
{
    return 16 * ((size_t)it.n1 * it.m1 + (size_t)nwr * (it.p + 1) * it.m1);
}

nurbs_status cuda_fail(cudaError_t e)
{
    g_last_cuda_error = (int32_t)e;
    return NURBS_ERR_CUDA;
}

}  // namespace

struct PlanGroup {
    int p, q;         // internal degrees (p == 0 for curves)
    int ck;           // 1: curve-kernel group (degree q, one warp per curve)
    int t0, t1;       // tile range
    int grid[6];      // CTAs per launch of each kernel variant (0 = unknown)
};

struct nurbs_plan {
    int32_t kind;
    int32_t warps;            // warps per CTA
    int32_t ctas_per_sm;      // 0 = occupancy limit
    int32_t max_ctas;         // 0 = no cap
    std::vector<ItemDev> items;
    std::vector<TileDev> tiles;
    int64_t points;
    // shared memory carve-up
    int R, C, acc_cap;
    int off_misc, off_su, off_u, off_nu, off_sv, off_v, off_nv, off_stage, off_beta, off_duc, off_dvc,
        off_jb, off_win, off_run, off_knots, off_w, off_acc, off_sa, off_dnu;
    int smem_bytes;           // gradient kernels
    int smem_eval;            // forward kernels (no shared adjoint)
    int smem_der;             // forward with tangents (derivative tables where the adjoint would be)
    int c_mc, c_wbytes, c_smem;   // curve kernels: control capacity, bytes per warp, per CTA
    int c_wbytes_f, c_smem_f;     // the same for the forward-only curve kernels
    int win_cap;                  // largest control net staged in shared memory (0: none)
    float knot_sigma;             // smoothed-indicator knot derivative bandwidth (0: off)
    int grad_homog;               // control-point gradients with respect to Pw
    // workspace layout (bytes)
    size_t items_off, tiles_off, counts_off, part_off, ws_bytes;
    // binding
    void* ws;
    size_t ws_len;
    std::vector<unsigned char> staging;   // host image of the tables (kept alive for async copies)
    std::vector<PlanGroup> groups;        // one kernel launch per (p, q) group
};

namespace {

nurbs_status check_desc(int32_t kind, const nurbs_desc& d)
{
    if (d.nu < 0 || d.n1 <= 0) return NURBS_ERR_ARG;
    if (d.p < 1 || d.p > NURBS_MAX_DEGREE || d.n1 < d.p + 1) return NURBS_ERR_DEGREE;
    if (d.n1 > NURBS_MAX_CTRL) return NURBS_ERR_SIZE;
    if (d.knot_u < 0 || d.ctrl < 0 || d.param_u < 0 || d.pts < 0) return NURBS_ERR_ARG;
    if (!(d.grad_scale >= 0.f) || !std::isfinite(d.grad_scale)) return NURBS_ERR_ARG;
    if (kind == NURBS_KIND_SURFACE) {
        if (d.nv < 0 || d.m1 <= 0) return NURBS_ERR_ARG;
        if (d.q < 1 || d.q > NURBS_MAX_DEGREE || d.m1 < d.q + 1) return NURBS_ERR_DEGREE;
        if (d.m1 > NURBS_MAX_CTRL) return NURBS_ERR_SIZE;
        if (d.knot_v < 0 || d.param_v < 0) return NURBS_ERR_ARG;
    }
    return NURBS_OK;
}

// Internal item: a curve is a surface with a degree-0, single-row u direction.
ItemDev make_item(int32_t kind, const nurbs_desc& d)
{
    ItemDev it;
    std::memset(&it, 0, sizeof it);
    if (kind == NURBS_KIND_CURVE) {
        it.p = 0; it.q = d.p; it.n1 = 1; it.m1 = d.n1; it.nu = d.nu > 0 ? 1 : 0; it.nv = d.nu;
        it.knot_u = 0; it.knot_v = d.knot_u; it.ctrl = d.ctrl;
        it.param_u = 0; it.param_v = d.param_u; it.pts = d.pts; it.curve = 1;
    } else {
        it.p = d.p; it.q = d.q; it.n1 = d.n1; it.m1 = d.m1; it.nu = d.nu; it.nv = d.nv;
        it.knot_u = d.knot_u; it.knot_v = d.knot_v; it.ctrl = d.ctrl;
        it.param_u = d.param_u; it.param_v = d.param_v; it.pts = d.pts; it.curve = 0;
    }
    it.adam_step = d.adam_step > 0 ? d.adam_step : 0;
    it.gscale = d.grad_scale;
    return it;
}

}  // namespace

extern "C" {

nurbs_status nurbs_plan_create(int32_t kind, const nurbs_desc* h_desc, int32_t count,
                               const nurbs_tile_cfg* cfg, nurbs_plan** out)
{
    if (out == nullptr) return NURBS_ERR_ARG;
    *out = nullptr;
    if (kind != NURBS_KIND_SURFACE && kind != NURBS_KIND_CURVE) return NURBS_ERR_ARG;
    if (count < 0 || (count > 0 && h_desc == nullptr)) return NURBS_ERR_ARG;
    for (int32_t k = 0; k < count; ++k) {
        nurbs_status st = check_desc(kind, h_desc[k]);
        if (st != NURBS_OK) return st;
    }
    nurbs_plan* pl = new (std::nothrow) nurbs_plan();
    if (pl == nullptr) return NURBS_ERR_ARG;
    pl->kind = kind;
    pl->warps = 8;
    pl->ctas_per_sm = 0;
    pl->max_ctas = 0;
    int rows_cfg = 0;
    if (cfg != nullptr) {
        if (cfg->warps < 0 || cfg->warps > 8 || cfg->rows < 0 || cfg->ctas_per_sm < 0 || cfg->max_ctas < 0) {
            delete pl;
            return NURBS_ERR_ARG;
        }
        if (cfg->warps > 0) pl->warps = cfg->warps;
        rows_cfg = cfg->rows;
        pl->ctas_per_sm = cfg->ctas_per_sm;
        pl->max_ctas = cfg->max_ctas;
    }
    const int NW = pl->warps;
    const int maxcols = 32 * NW;
    pl->points = 0;
    pl->items.reserve(count);
    int maxR = 1, maxC = 32, max_m1 = 1;
    long long part_floats = 0;
    for (int32_t k = 0; k < count; ++k) {
        ItemDev it = make_item(kind, h_desc[k]);
        pl->points += (int64_t)it.nu * it.nv;
        max_m1 = std::max(max_m1, it.m1);
        pl->items.push_back(it);
    }
    // curves with at most kCurveCtrlCap control points run on the curve kernels:
    // one tile (one warp) per curve, one group per degree
    pl->c_mc = 4;
    pl->c_wbytes = 0;
    pl->c_wbytes_f = 0;
    for (ItemDev& it : pl->items) {
        it.ck = (kind == NURBS_KIND_CURVE && it.m1 <= kCurveCtrlCap) ? 1 : 0;
        if (it.ck) pl->c_mc = std::max(pl->c_mc, it.m1);
    }
    // Within a group, items enter the queue longest first (most samples; ties in
    // item order), so the persistent CTAs end on short items rather than waiting
    // on one long item at the tail.  Results do not depend on the order.
    std::vector<int32_t> order(count);
    for (int32_t k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (int64_t)pl->items[a].nu * pl->items[a].nv > (int64_t)pl->items[b].nu * pl->items[b].nv;
    });
    for (int q = 1; q <= NURBS_MAX_DEGREE; ++q) {
        PlanGroup grp;
        grp.p = 0; grp.q = q; grp.ck = 1;
        grp.t0 = (int)pl->tiles.size();
        for (int v = 0; v < 6; ++v) grp.grid[v] = 0;
        for (int32_t k : order) {
            ItemDev& it = pl->items[k];
            if (!it.ck || it.q != q) continue;
            it.first_tile = (int)pl->tiles.size();
            it.ntiles = 1;
            TileDev tl;
            std::memset(&tl, 0, sizeof tl);
            tl.item = k;
            tl.nrows = it.nu;
            tl.ncols = it.nv;
            pl->tiles.push_back(tl);
        }
        grp.t1 = (int)pl->tiles.size();
        if (grp.t1 > grp.t0) {
            pl->groups.push_back(grp);
            pl->c_wbytes = std::max(pl->c_wbytes, curve_warp_bytes(pl->c_mc, q, true));
            pl->c_wbytes_f = std::max(pl->c_wbytes_f, curve_warp_bytes(pl->c_mc, q, false));
        }
    }
    pl->c_smem = kCurveWarps * pl->c_wbytes;
    pl->c_smem_f = kCurveWarps * pl->c_wbytes_f;
    // tiles, grouped by degree pair so that each group runs one specialised kernel
    for (int g = 0; g < kMaxGroups; ++g) {
        const int gp = g / 5, gq = g % 5 + 1;
        PlanGroup grp;
        grp.p = gp; grp.q = gq; grp.ck = 0;
        grp.t0 = (int)pl->tiles.size();
        for (int v = 0; v < 6; ++v) grp.grid[v] = 0;
        for (int32_t k : order) {
            ItemDev& it = pl->items[k];
            if (it.p != gp || it.q != gq || it.ck) continue;
            it.first_tile = (int)pl->tiles.size();
            // column tiles of at most 32*NW samples; row tiles of R rows split into row groups
            const int nct = std::max(1, (it.nv + maxcols - 1) / maxcols);
            const int cw = it.nv > 0 ? ((it.nv + nct - 1) / nct + 31) / 32 * 32 : 32;
            const int nwc = std::max(1, std::min(NW, cw / 32));
            int nwr = it.curve ? 1 : std::max(1, NW / nwc);
            int R = it.curve ? 1 : (rows_cfg > 0 ? rows_cfg : 16 * nwr);
            nwr = std::min(nwr, R);
            const int nrt = std::max(1, (it.nu + R - 1) / R);
            // row tiles of equal height (an item's tiles run side by side, so its longest
            // tile sets when it is done)
            const int Rb = std::max(1, (it.nu + nrt - 1) / nrt);
            it.rcap = it.n1;
            it.ku_cap = it.curve ? 0 : it.n1 + it.p + 1;
            it.kv_cap = it.m1 + it.q + 1;
            it.wbase = align4(12 + it.ku_cap + it.kv_cap);
            it.abase = 8;
            it.unit_slot = it.abase + 4 * it.rcap * it.m1;
            int ntl = 0;
            for (int rt = 0; rt < nrt; ++rt) {
                for (int ct = 0; ct < nct; ++ct) {
                    TileDev tl;
                    std::memset(&tl, 0, sizeof tl);
                    tl.item = k;
                    tl.row0 = rt * Rb;
                    tl.nrows = std::max(0, std::min(Rb, it.nu - tl.row0));
                    tl.col0 = ct * cw;
                    tl.ncols = std::max(0, std::min(cw, it.nv - tl.col0));
                    tl.tidx = ntl++;
                    tl.nwc = nwc;
                    tl.nwr = nwr;
                    tl.rpg = std::max(1, (tl.nrows + nwr - 1) / nwr);
                    tl.part = part_floats;
                    part_floats += it.wbase + (long long)nwr * it.unit_slot;
                    part_floats = (part_floats + 63) / 64 * 64;   // 256-byte aligned slots
                    pl->tiles.push_back(tl);
                    maxR = std::max(maxR, tl.nrows);
                    maxC = std::max(maxC, nwc * 32);
                }
            }
            it.ntiles = ntl;   // single-tile items keep their adjoint in shared memory when it fits (carve)
        }
        grp.t1 = (int)pl->tiles.size();
        if (grp.t1 > grp.t0) pl->groups.push_back(grp);
    }
    // shared memory carve-up for the largest tile
    int max_nwc = 1, max_nwr = 1, max_unit_cols = 32;
    for (const TileDev& tl : pl->tiles) {
        max_nwc = std::max(max_nwc, tl.nwc);
        max_nwr = std::max(max_nwr, tl.nwr);
        max_unit_cols = std::max(max_unit_cols, tl.nwr * tl.nwc * 32);
    }
    pl->R = maxR;
    pl->C = maxC;
    // per-degree table strides (the kernels' SU, SV, KU, KV)
    int su = 4, sv = 4, ku = 1, kv = 2;
    for (const ItemDev& it : pl->items) {
        su = std::max(su, align4(it.p + 1));
        sv = std::max(sv, align4(it.q + 1));
        ku = std::max(ku, 2 * it.p);
        kv = std::max(kv, 2 * it.q);
    }
    int max_knots = 4;
    for (const ItemDev& it : pl->items)
        max_knots = std::max(max_knots, align4(it.n1 + it.p + 1) + it.m1 + it.q + 1);
    int max_units = 1;
    for (const ItemDev& it : pl->items) {
        int u = 0;
        for (int t = it.first_tile; t < it.first_tile + it.ntiles; ++t) u += pl->tiles[t].nwr;
        max_units = std::max(max_units, u);
    }
    // Shared memory carve-up for the largest tile, given the rows of dL/dS (or target)
    // in flight per warp, the largest staged control net and the largest shared adjoint
    // (single-tile items whose adjoint exceeds it use the workspace instead).
    auto carve = [&](int win_cap, size_t sa_cap) {
        for (ItemDev& it : pl->items)
            it.smemA = (!it.ck && it.ntiles == 1 &&
                        smem_adjoint_bytes(it, pl->tiles[it.first_tile].nwr) <= sa_cap) ? 1 : 0;
        pl->win_cap = win_cap;
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 16); return (int)o; };
        pl->off_misc = take(256);
        pl->off_su = take(4 * maxR);
        pl->off_u = take(4 * maxR);
        pl->off_nu = take(4 * maxR * su);
        pl->off_sv = take(4 * maxC);
        pl->off_v = take(4 * maxC);
        pl->off_nv = take(4 * maxC * sv);
        pl->off_stage = take(16 * kBatch * max_unit_cols);
        pl->off_beta = take(4 * max_nwc * maxR * su);
        pl->off_duc = take(4 * maxR * ku);
        // column cotangents: one row of kv per (row group, column) of a tile; a tile has at
        // most as many (row group, column) pairs as its warps have lanes
        pl->off_dvc = take(4 * (size_t)max_unit_cols * kv);
        pl->off_jb = take(8 * kJbCap);
        pl->off_win = take(16 * (size_t)win_cap);
        pl->off_run = take(4 * maxR);
        pl->off_knots = take(4 * max_knots);
        pl->off_w = take(4 * (kJbCap + maxC * sv));
        size_t sa_bytes = 0;
        for (const ItemDev& it : pl->items)
            if (it.smemA) sa_bytes = std::max(sa_bytes, smem_adjoint_bytes(it, pl->tiles[it.first_tile].nwr));
        pl->smem_eval = (int)off;     // the forward kernels stop here
        // the row basis derivatives of the forward with tangents take the place of the
        // shared adjoint, which only the gradient kernels use
        pl->off_dnu = (int)off;
        pl->smem_der = (int)align_up(off + 4 * (size_t)maxR * su, 16);
        pl->off_sa = take(sa_bytes);
        pl->off_acc = pl->off_su;     // the final reduction reuses the tile tables
        const size_t min_acc = std::max<size_t>(16 * 1024, 32 * (size_t)max_units);
        if (off < (size_t)pl->off_acc + min_acc) off = pl->off_acc + min_acc;
        pl->acc_cap = (int)(off - pl->off_acc);
        pl->smem_bytes = (int)off;
    };
    carve(kWinCap, kSmemACap);
    // A plan asked for k >= 2 persistent CTAs per SM gets a carve-up that lets k gradient
    // CTAs share an SM (228 KB of shared memory per SM, 1 KB of it reserved per CTA):
    // first a smaller shared adjoint, then no staged control net (the kernels then read
    // control points from global memory).
    if (pl->ctas_per_sm >= 2) {
        const size_t budget = (size_t)kSmemPerSM / pl->ctas_per_sm - 1024;
        auto fit_sa = [&](int win_cap) {
            carve(win_cap, 0);
            const size_t rest = (size_t)pl->smem_bytes;
            carve(win_cap, rest < budget ? std::min<size_t>(budget - rest, kSmemACap) : 0);
        };
        if ((size_t)pl->smem_bytes > budget) fit_sa(kWinCap);
        if ((size_t)pl->smem_bytes > budget) fit_sa(0);
    }
    // workspace layout
    size_t w = kHeaderBytes;
    pl->items_off = w; w = align_up(w + sizeof(ItemDev) * pl->items.size(), 256);
    pl->tiles_off = w; w = align_up(w + sizeof(TileDev) * pl->tiles.size(), 256);
    pl->counts_off = w; w = align_up(w + 4 * pl->items.size(), 256);
    pl->part_off = w; w = align_up(w + 4 * (size_t)part_floats, 256);
    pl->ws_bytes = w;
    pl->ws = nullptr;
    pl->ws_len = 0;
    *out = pl;
    return NURBS_OK;
}

size_t nurbs_plan_workspace_size(const nurbs_plan* plan) { return plan ? plan->ws_bytes : 0; }

nurbs_status nurbs_plan_set_knot_sigma(nurbs_plan* plan, float sigma)
{
    if (plan == nullptr || !(sigma >= 0.f) || !std::isfinite(sigma)) return NURBS_ERR_ARG;
    plan->knot_sigma = sigma;
    return NURBS_OK;
}

nurbs_status nurbs_plan_set_grad_homogeneous(nurbs_plan* plan, int32_t on)
{
    if (plan == nullptr || (on != 0 && on != 1)) return NURBS_ERR_ARG;
    plan->grad_homog = on;
    return NURBS_OK;
}
int64_t nurbs_plan_points(const nurbs_plan* plan) { return plan ? plan->points : 0; }
int32_t nurbs_plan_tiles(const nurbs_plan* plan) { return plan ? (int32_t)plan->tiles.size() : 0; }

void nurbs_plan_destroy(nurbs_plan* plan) { delete plan; }

nurbs_status nurbs_plan_bind(nurbs_plan* pl, void* d_ws, size_t bytes, nurbs_stream_t stream)
{
    if (pl == nullptr) return NURBS_ERR_ARG;
    if (d_ws == nullptr || bytes < pl->ws_bytes || ((uintptr_t)d_ws & 255u) != 0) return NURBS_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pl->staging.assign(pl->part_off, 0);
    std::memcpy(pl->staging.data() + pl->items_off, pl->items.data(), sizeof(ItemDev) * pl->items.size());
    std::memcpy(pl->staging.data() + pl->tiles_off, pl->tiles.data(), sizeof(TileDev) * pl->tiles.size());
    cudaError_t e = cudaMemcpyAsync(d_ws, pl->staging.data(), pl->part_off, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    pl->ws = d_ws;
    pl->ws_len = bytes;
    return NURBS_OK;
}

nurbs_status nurbs_plan_get_error(nurbs_plan* pl, nurbs_stream_t stream, uint32_t* flags)
{
    if (pl == nullptr) return NURBS_ERR_ARG;
    if (pl->ws == nullptr) return NURBS_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, pl->ws, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->ws, 0, 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (flags) *flags = word;
    for (int b = 1; b < 32; ++b)
        if (word & (1u << b)) return (nurbs_status)b;
    return NURBS_OK;
}

}  // extern "C"

namespace {

KernelVariant variant_for(int v, int p, int q)
{
#define NURBS_TILE_V(pp)                                   \
    switch (v) {                                           \
        case 0: return tile_variant_p##pp##_v0(q);         \
        case 1: return tile_variant_p##pp##_v1(q);         \
        case 2: return tile_variant_p##pp##_v2(q);         \
        case 3: return tile_variant_p##pp##_v3(q);         \
        case 4: return tile_variant_p##pp##_v4(q);         \
        default: return tile_variant_p##pp##_v5(q);        \
    }
    switch (p) {
        case 0: NURBS_TILE_V(0)
        case 1: NURBS_TILE_V(1)
        case 2: NURBS_TILE_V(2)
        case 3: NURBS_TILE_V(3)
        case 4: NURBS_TILE_V(4)
        default: NURBS_TILE_V(5)
    }
#undef NURBS_TILE_V
}

// Dynamic shared memory a kernel launches with before its limit must be raised: the
// 48 KB default covers static and dynamic shared memory together, and the kernels'
// static shared memory is a few bytes, so the attribute is raised above 47 KB.
constexpr int kSmemNoOptin = 47 * 1024;

// Kernel, block, shared memory and queue slot of one group for variant v.
struct GroupLaunch {
    KernelVariant kv;
    int block, smem, qslot, units;   // units: tiles per CTA slot (curve kernels: warps)
};

GroupLaunch group_launch(const nurbs_plan* pl, const PlanGroup& grp, int v)
{
    if (grp.ck)
        return GroupLaunch{curve_variant(v, grp.q), 32 * kCurveWarps, (v == 0 || v == 5) ? pl->c_smem_f : pl->c_smem,
                           kMaxGroups + grp.q - 1, kCurveWarps};
    return GroupLaunch{variant_for(v, grp.p, grp.q), 32 * pl->warps,
                       v == 0 ? pl->smem_eval : v == 5 ? pl->smem_der : pl->smem_bytes,
                       grp.p * 5 + grp.q - 1, 1};
}

// Grid of a group for variant v (once per plan): as many persistent CTAs as fit,
// no more than its tiles need, capped by max_ctas when `cap`.
nurbs_status size_group(nurbs_plan* pl, PlanGroup& grp, int v, const GroupLaunch& gl, bool cap)
{
    if (grp.grid[v] != 0) return NURBS_OK;
    // the attribute is per kernel function: raise it to the device limit so that
    // no plan lowers it under another plan's launch size
    cudaError_t e = cudaSuccess;
    if (gl.smem > kSmemNoOptin) {
        int limit = 0;
        e = gl.kv.set_smem(&limit);
        if (e == cudaSuccess && gl.smem > limit) return NURBS_ERR_SIZE;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    int occ = 0, dev = 0, sms = 0;
    e = gl.kv.occupancy(&occ, gl.block, gl.smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (occ < 1) return NURBS_ERR_SIZE;
    if (pl->ctas_per_sm > 0) occ = std::min(occ, pl->ctas_per_sm);
    const int need = (grp.t1 - grp.t0 + gl.units - 1) / gl.units;
    grp.grid[v] = std::max(1, std::min(need, occ * sms));
    if (cap && pl->max_ctas > 0) grp.grid[v] = std::min(grp.grid[v], pl->max_ctas);
    return NURBS_OK;
}

// Workspace tables and shared-memory carve-up of a plan in the kernel parameters.
void fill_tables(KParams& kp, const nurbs_plan* pl, unsigned char* ws)
{
    kp.items = reinterpret_cast<const ItemDev*>(ws + pl->items_off);
    kp.tiles = reinterpret_cast<const TileDev*>(ws + pl->tiles_off);
    kp.hdr = reinterpret_cast<WsHeader*>(ws);
    kp.counts = reinterpret_cast<unsigned int*>(ws + pl->counts_off);
    kp.part = reinterpret_cast<float*>(ws + pl->part_off);
    kp.R = pl->R; kp.C = pl->C;
    kp.off_misc = pl->off_misc; kp.off_su = pl->off_su; kp.off_u = pl->off_u; kp.off_nu = pl->off_nu;
    kp.off_sv = pl->off_sv; kp.off_v = pl->off_v; kp.off_nv = pl->off_nv; kp.off_stage = pl->off_stage;
    kp.off_beta = pl->off_beta; kp.off_duc = pl->off_duc; kp.off_dvc = pl->off_dvc;
    kp.off_jb = pl->off_jb; kp.off_win = pl->off_win; kp.off_run = pl->off_run;
    kp.off_knots = pl->off_knots; kp.off_w = pl->off_w; kp.off_sa = pl->off_sa; kp.off_acc = pl->off_acc;
    kp.off_dnu = pl->off_dnu;
    kp.acc_cap = pl->acc_cap;
    kp.c_mc = pl->c_mc;
    kp.c_wbytes = pl->c_wbytes;
    kp.knot_sigma = pl->knot_sigma;
    kp.win_cap = pl->win_cap;
    kp.grad_homog = pl->grad_homog;
}

// Launch variant v (0 forward, 1/2 backward from dL/dS without/with knots, 3/4 the
// same from an MSE target): one persistent kernel per group, in group order on `s`.
nurbs_status launch_groups(nurbs_plan* pl, int v, KParams& kp, unsigned char* ws, cudaStream_t s, bool cap)
{
    fill_tables(kp, pl, ws);
    kp.c_wbytes = (v == 0 || v == 5) ? pl->c_wbytes_f : pl->c_wbytes;   // curve kernels' bytes per warp
    for (PlanGroup& grp : pl->groups) {
        const GroupLaunch gl = group_launch(pl, grp, v);
        nurbs_status st = size_group(pl, grp, v, gl, cap);
        if (st != NURBS_OK) return st;
        kp.t0 = grp.t0;
        kp.t1 = grp.t1;
        kp.queue = kp.hdr->queue + 2 * gl.qslot;
        cudaError_t e = gl.kv.launch(kp, grp.grid[v], gl.block, gl.smem, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return NURBS_OK;
}

nurbs_status launch(const nurbs_plan* cpl, int v, KParams& kp, cudaStream_t s)
{
    nurbs_plan* pl = const_cast<nurbs_plan*>(cpl);
    if (pl->ws == nullptr) return NURBS_ERR_WORKSPACE;
    if (pl->tiles.empty()) return NURBS_OK;
    return launch_groups(pl, v, kp, static_cast<unsigned char*>(pl->ws), s, true);
}

void zero_params(KParams& kp)
{
    std::memset(&kp, 0, sizeof kp);
}

}  // namespace

extern "C" {

int32_t nurbs_plan_ctas(const nurbs_plan* plan)
{
    if (plan == nullptr) return 0;
    int n = 0;
    for (const PlanGroup& g : plan->groups) n += *std::max_element(g.grid, g.grid + 6);
    return n;
}

nurbs_status nurbs_plan_occupancy(const nurbs_plan* plan, int32_t op, int32_t* ctas_per_sm, int32_t* smem_bytes)
{
    if (plan == nullptr || ctas_per_sm == nullptr || op < 0 || op > 5) return NURBS_ERR_ARG;
    int occ_min = 0, smem_max = 0;
    for (const PlanGroup& grp : plan->groups) {
        const GroupLaunch gl = group_launch(plan, grp, op);
        cudaError_t e = cudaSuccess;
        if (gl.smem > kSmemNoOptin) {
            int limit = 0;
            e = gl.kv.set_smem(&limit);
            if (e == cudaSuccess && gl.smem > limit) return NURBS_ERR_SIZE;
        }
        int occ = 0;
        if (e == cudaSuccess) e = gl.kv.occupancy(&occ, gl.block, gl.smem);
        if (e != cudaSuccess) return cuda_fail(e);
        occ_min = occ_min == 0 ? occ : std::min(occ_min, occ);
        smem_max = std::max(smem_max, gl.smem);
    }
    *ctas_per_sm = occ_min;
    if (smem_bytes != nullptr) *smem_bytes = smem_max;
    return NURBS_OK;
}

static nurbs_status eval_common(const nurbs_plan* pl, int32_t kind, const float* knots, const float* ctrl,
                                const float* params, float* pts, nurbs_stream_t stream)
{
    if (pl == nullptr) return NURBS_ERR_ARG;
    if (pl->kind != kind) return NURBS_ERR_KIND;
    if (pl->tiles.empty()) return NURBS_OK;
    if (knots == nullptr || ctrl == nullptr || params == nullptr || pts == nullptr) return NURBS_ERR_ARG;
    if (((uintptr_t)ctrl & 15u) != 0) return NURBS_ERR_ARG;
    KParams kp;
    zero_params(kp);
    kp.knots = knots;
    kp.ctrl = reinterpret_cast<const float4*>(ctrl);
    kp.params = params;
    kp.pts = pts;
    return launch(pl, 0, kp, reinterpret_cast<cudaStream_t>(stream));
}

nurbs_status nurbs_eval_surface(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                const float* params, float* pts, nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_eval_surface");
    return eval_common(plan, NURBS_KIND_SURFACE, knots, ctrl, params, pts, stream);
}

nurbs_status nurbs_eval_curve(const nurbs_plan* plan, const float* knots, const float* ctrl,
                              const float* params, float* pts, nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_eval_curve");
    return eval_common(plan, NURBS_KIND_CURVE, knots, ctrl, params, pts, stream);
}

static nurbs_status derivs_common(const nurbs_plan* pl, int32_t kind, const float* knots, const float* ctrl,
                                  const float* params, float* pts, float* du, float* dv, float* normals,
                                  nurbs_stream_t stream)
{
    if (pl == nullptr) return NURBS_ERR_ARG;
    if (pl->kind != kind) return NURBS_ERR_KIND;
    if (pl->tiles.empty()) return NURBS_OK;
    if (knots == nullptr || ctrl == nullptr || params == nullptr) return NURBS_ERR_ARG;
    if (pts == nullptr && du == nullptr && dv == nullptr && normals == nullptr) return NURBS_ERR_ARG;
    if (((uintptr_t)ctrl & 15u) != 0) return NURBS_ERR_ARG;
    KParams kp;
    zero_params(kp);
    kp.knots = knots;
    kp.ctrl = reinterpret_cast<const float4*>(ctrl);
    kp.params = params;
    kp.pts = pts;
    kp.d_du = du;
    kp.d_dv = dv;
    kp.d_nrm = normals;
    return launch(pl, 5, kp, reinterpret_cast<cudaStream_t>(stream));
}

nurbs_status nurbs_eval_surface_derivs(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                       const float* params, float* pts, float* du, float* dv, float* normals,
                                       nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_eval_surface_derivs");
    return derivs_common(plan, NURBS_KIND_SURFACE, knots, ctrl, params, pts, du, dv, normals, stream);
}

nurbs_status nurbs_eval_curve_derivs(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                     const float* params, float* pts, float* tangents, nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_eval_curve_derivs");
    // a curve runs as the v direction of its item: its tangent is the v-derivative
    return derivs_common(plan, NURBS_KIND_CURVE, knots, ctrl, params, pts, nullptr, tangents, nullptr, stream);
}

static nurbs_status grad_common(const nurbs_plan* pl, const float* knots, const float* ctrl, float* ctrl_w,
                                const float* params, const float* gin, int gsrc, float* pts,
                                float* grad_ctrl, float* grad_knots, float* loss_items, float grad_scale,
                                float* adam_m, float* adam_v, const nurbs_adam* hp, int32_t step,
                                nurbs_stream_t stream)
{
    if (pl == nullptr) return NURBS_ERR_ARG;
    if (pl->tiles.empty()) return NURBS_OK;
    if (knots == nullptr || ctrl == nullptr || params == nullptr || gin == nullptr) return NURBS_ERR_ARG;
    if (((uintptr_t)ctrl & 15u) != 0 || ((uintptr_t)grad_ctrl & 15u) != 0) return NURBS_ERR_ARG;
    KParams kp;
    zero_params(kp);
    kp.knots = knots;
    kp.ctrl = reinterpret_cast<const float4*>(ctrl);
    kp.ctrl_w = reinterpret_cast<float4*>(ctrl_w);
    kp.params = params;
    kp.pts = pts;
    kp.gin = gin;
    kp.gsrc = gsrc;
    kp.grad_ctrl = reinterpret_cast<float4*>(grad_ctrl);
    kp.grad_knots = grad_knots;
    kp.loss_items = loss_items;
    kp.grad_scale = grad_scale;
    if (hp != nullptr) {
        if (adam_m == nullptr || adam_v == nullptr || ctrl_w == nullptr || step < 1) return NURBS_ERR_ARG;
        if (((uintptr_t)adam_m & 15u) != 0 || ((uintptr_t)adam_v & 15u) != 0) return NURBS_ERR_ARG;
        const double bc1 = 1.0 - std::pow((double)hp->beta1, (double)step);
        const double bc2 = 1.0 - std::pow((double)hp->beta2, (double)step);
        kp.fit = 1;
        kp.lr = hp->lr;
        kp.step = step;
        kp.adam_m = reinterpret_cast<float4*>(adam_m);
        kp.adam_v = reinterpret_cast<float4*>(adam_v);
        kp.lr_t = (float)(hp->lr / bc1);
        kp.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
        kp.b1 = hp->beta1;
        kp.b2 = hp->beta2;
        kp.eps = hp->eps;
    }
    const int v = (gsrc == 1 ? 3 : 1) + (grad_knots != nullptr ? 1 : 0);
    return launch(pl, v, kp, reinterpret_cast<cudaStream_t>(stream));
}

nurbs_status nurbs_backward(const nurbs_plan* plan, const float* knots, const float* ctrl,
                            const float* params, const float* grad_pts, float* grad_ctrl,
                            float* grad_knots, nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_backward");
    return grad_common(plan, knots, ctrl, nullptr, params, grad_pts, 0, nullptr, grad_ctrl, grad_knots,
                       nullptr, 0.f, nullptr, nullptr, nullptr, 0, stream);
}

nurbs_status nurbs_mse_fwd_bwd(const nurbs_plan* plan, const float* knots, const float* ctrl,
                               const float* params, const float* target, float* pts,
                               float* grad_ctrl, float* grad_knots, float* loss_items,
                               float grad_scale, nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_mse_fwd_bwd");
    return grad_common(plan, knots, ctrl, nullptr, params, target, 1, pts, grad_ctrl, grad_knots,
                       loss_items, grad_scale, nullptr, nullptr, nullptr, 0, stream);
}

nurbs_status nurbs_fit_step(const nurbs_plan* plan, const float* knots, float* ctrl,
                            const float* params, const float* target, float* pts,
                            float* adam_m, float* adam_v, const nurbs_adam* hp, int32_t step,
                            float grad_scale, float* loss_items, float* grad_knots,
                            nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_fit_step");
    if (hp == nullptr) return NURBS_ERR_ARG;
    return grad_common(plan, knots, ctrl, ctrl, params, target, 1, pts, nullptr, grad_knots,
                       loss_items, grad_scale, adam_m, adam_v, hp, step, stream);
}

const char* nurbs_status_string(nurbs_status s)
{
    switch (s) {
        case NURBS_OK: return "ok";
        case NURBS_ERR_ARG: return "invalid argument";
        case NURBS_ERR_KNOTS: return "knot vector not non-decreasing or last span empty";
        case NURBS_ERR_DEGREE: return "degree out of range or too few control points";
        case NURBS_ERR_DOMAIN: return "sample outside the parametric domain";
        case NURBS_ERR_ORDER: return "samples not non-decreasing";
        case NURBS_ERR_WORKSPACE: return "workspace missing, too small, misaligned or not bound";
        case NURBS_ERR_CUDA: return "CUDA runtime error";
        case NURBS_ERR_SIZE: return "item exceeds a kernel limit";
        case NURBS_ERR_KIND: return "plan built for the other kind";
    }
    return "unknown status";
}

int32_t nurbs_last_cuda_error(void) { return g_last_cuda_error; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free fused MSE forward + backward (nurbs_mse_fwd_bwd_noalloc).
//
// For callers that cannot allocate device memory themselves, the workspace of
// this one entry point is a fixed array in the library's device image.  Every
// call shares it, so each call re-uploads the plan's item and tile tables into it
// and clears the queue/arrival counters before launching; the partial-sum slots
// need no clearing (every slot is written before it is read).  The error word at
// the head of the array is not cleared by a call: it collects the device checks
// of every call until nurbs_noalloc_get_error reads and clears it.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NURBS_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per device.
nurbs_status noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kNoallocMaxDevices) return NURBS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return NURBS_OK;
}

}  // namespace

extern "C" nurbs_status nurbs_mse_fwd_bwd_noalloc(const nurbs_plan* cpl, const float* knots, const float* ctrl,
                                                  const float* params, const float* target, float* pts,
                                                  float* grad_ctrl, float* grad_knots, float* loss_items,
                                                  float grad_scale, nurbs_stream_t stream)
{
    NvtxScope nvtx_("nurbs_mse_fwd_bwd_noalloc");
    if (cpl == nullptr) return NURBS_ERR_ARG;
    if (cpl->ws_bytes > (size_t)NURBS_NOALLOC_SCRATCH_BYTES) return NURBS_ERR_WORKSPACE;
    if (cpl->tiles.empty()) return NURBS_OK;
    if (knots == nullptr || ctrl == nullptr || params == nullptr || target == nullptr) return NURBS_ERR_ARG;
    if (((uintptr_t)ctrl & 15u) != 0 || ((uintptr_t)grad_ctrl & 15u) != 0) return NURBS_ERR_ARG;
    void* scratch = nullptr;
    nurbs_status st = noalloc_scratch(&scratch);
    if (st != NURBS_OK) return st;
    nurbs_plan* pl = const_cast<nurbs_plan*>(cpl);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(scratch);
    // tables from the plan's host copies; queue and arrival counters cleared (the
    // error word, the header's first 4 bytes, keeps what earlier calls raised)
    static_assert(offsetof(WsHeader, error) == 0 && sizeof(((WsHeader*)nullptr)->error) == 4, "error word");
    cudaError_t e = cudaMemsetAsync(ws + 4, 0, pl->items_off - 4, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + pl->items_off, pl->items.data(), sizeof(ItemDev) * pl->items.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + pl->tiles_off, pl->tiles.data(), sizeof(TileDev) * pl->tiles.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + pl->counts_off, 0, pl->part_off - pl->counts_off, s);
    if (e != cudaSuccess) return cuda_fail(e);

    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.knots = knots;
    kp.ctrl = reinterpret_cast<const float4*>(ctrl);
    kp.params = params;
    kp.pts = pts;
    kp.gin = target;
    kp.gsrc = 1;
    kp.grad_ctrl = reinterpret_cast<float4*>(grad_ctrl);
    kp.grad_knots = grad_knots;
    kp.loss_items = loss_items;
    kp.grad_scale = grad_scale;
    const int v = grad_knots != nullptr ? 4 : 3;
    // the same launch shape as nurbs_mse_fwd_bwd (CTA cap included)
    return launch_groups(pl, v, kp, ws, s, true);
}

extern "C" nurbs_status nurbs_noalloc_get_error(nurbs_stream_t stream, uint32_t* flags)
{
    void* scratch = nullptr;
    nurbs_status st = noalloc_scratch(&scratch);
    if (st != NURBS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, scratch, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (flags) *flags = word;
    for (int b = 1; b < 32; ++b)
        if (word & (1u << b)) return (nurbs_status)b;
    return NURBS_OK;
}
