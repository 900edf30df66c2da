// Device-side tables of a bound plan (shared by the host planner and the
// kernels).  Everything lives in the caller's workspace:
//
//   [0, 512)           WsHeader: error word, one persistent-queue pair per kernel group
//   items_off          ItemDev[count]
//   tiles_off          TileDev[ntiles]
//   counts_off         uint32 per item: tiles finished in the current launch
//   part_off           partial-sum slots (floats), one per tile (see below)
//
// Tile slot (float offsets from TileDev::part):
//   [0..7]    int: ku_lo, nku, kv_lo, nkv, valid, -, -, -
//   [8]       float: loss (sum of squared differences over the tile)
//   [12..)    dU partial (ku_cap floats), then dV partial (kv_cap floats)
//   wbase     unit slots, one per row group of the tile (ItemDev::unit_slot floats each):
//               [0..7] int: ilo, rows, jlo, CW, valid
//               abase  float4 A[rows][m1]: homogeneous adjoint partial for control
//                      rows ilo .. ilo+rows-1 and columns jlo .. jlo+CW-1
#pragma once
#include <stdint.h>

namespace nurbs {

constexpr int kHeaderBytes = 512;

constexpr int kMaxGroups = 30;   // distinct (p, q) pairs of the tile kernels: p in 0..5, q in 1..5
constexpr int kCurveGroups = 5;  // curve-kernel groups: degree 1..5

struct WsHeader {
    unsigned int error;                  // bit k set <=> nurbs_status k raised on the device
    unsigned int pad0;
    unsigned int queue[2 * (kMaxGroups + kCurveGroups)];   // per group: next tile, CTAs finished
};
static_assert(sizeof(WsHeader) <= kHeaderBytes, "workspace header");

struct ItemDev {
    int p, q, n1, m1, nu, nv;
    int first_tile, ntiles;
    int rcap;        // control rows a unit slot can hold (n1)
    int ku_cap, kv_cap;
    int wbase;       // float offset of the first unit slot inside a tile slot
    int unit_slot;   // floats per unit slot
    int abase;       // float offset of A inside a unit slot (16-byte aligned)
    int curve;       // 1: a curve item mapped onto the v direction (p == 0, n1 == 1)
    int adam_step;   // fit step: this item's Adam step (0 = the launch's)
    int smemA;       // single-tile item whose homogeneous adjoint stays in shared memory
    int ck;          // curve run by the curve kernels (one warp per curve, one tile)
    float gscale;    // MSE / fit step: this item's dL/dS scale (0 = the launch's)
    int pad_;
    long long knot_u, knot_v, ctrl, param_u, param_v, pts;
};

struct TileDev {
    int item, row0, nrows, col0, ncols, tidx;
    int nwc, nwr, rpg;   // column warps, row groups, rows per row group
    int pad;
    long long part;      // float offset of this tile's slot in the partial area
};

}  // namespace nurbs
