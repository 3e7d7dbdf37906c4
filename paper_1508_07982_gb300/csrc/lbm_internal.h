// Internal declarations of the GB300 refined-grid LBM library (host planner + device kernels).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm_gb300.h"

namespace lbm {

constexpr int Q = 19;
// D3Q19 velocities in the public direction order of lbm_gb300.h (Sec. 2, Fig. 1).
constexpr int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
constexpr int OPP[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
inline double weight(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// Cell kinds stored per cell (uint8).
enum : uint8_t {
    CK_FLUID = 0,  // owned fluid cell: collides and streams
    CK_GHOST = 1,  // fluid cell of ghost layers 1-2 (covered by the coarser level): streams only
    CK_FAR = 2,    // fluid cell of ghost layer 4 or beyond: never read
    CK_SOLID = 3,  // no-slip obstacle
    CK_G3 = 4,     // fluid cell of ghost layer 3: its value is the coarse parent's, never stored
};
// Neighbour-table codes for block positions that hold no brick of this level.
enum : int32_t { NB_WALL = -1, NB_FINER = -2, NB_COARSE = -3 };
// Brick attribute bits.
// BK_PURE: no obstacle cell.  BK_PLAIN (owned bricks): every pull of every cell is a plain load of a
// stored value (pure, no finer neighbour, all 26 neighbours present and pure).
enum : uint8_t { BK_PURE = 1, BK_TOUCH_FINER = 2, BK_GHOST = 4, BK_PLAIN = 8 };

struct HostLevel {
    int N[3] = {0, 0, 0};    // cells per axis on this level
    int nb[3] = {0, 0, 0};   // blocks per axis on this level
    int nown = 0, nghost = 0;
    std::vector<int32_t> pos;      // [nbricks][3] block coordinates (owned bricks first)
    std::vector<int32_t> nbr;      // [nbricks][27] neighbour brick, or an NB_* code
    std::vector<int32_t> parent;   // [nbricks] ghost: (L-1 brick) * 8 + octant; owned: -1
    std::vector<int32_t> child;    // [nown][8] ghost brick of L+1 under each octant, or -1
    std::vector<uint8_t> kind;     // [nbricks] BK_* bits
    std::vector<uint8_t> cell;     // [nbricks * B^3] CK_* per cell
    std::vector<uint32_t> link;    // [nown * B^3] per owned cell: bit q = link q is not a plain
                                   // same-level load; bit 29 = every such link is a bounce-back
                                   // (bits 25-27: wall face of its wall term, 7 = none); bit 28 =
                                   // every such link is a coalescence link; bit 31 = not fluid
    std::vector<uint32_t> colsolid;  // [nown * B^2] per column of an owned brick: bit z = the column
                                     // walk skips the cell (not fluid, or a coupled cell)
    std::vector<uint8_t> colspec;    // [nown * B^2] 1 if any cell of the column has a nonzero link mask
    // Ghost stream work of sub-step s+1: 4 words per entry {cell, need, coarse, special}: the
    // directions of the cell whose value a later pull reads, those whose source value is the
    // coarse parent's, and those that are not plain loads (bounce-back, wall).
    std::vector<uint32_t> gwork[2];
    // Explosion work: 4 words per entry {cell, directions, coarse parent cell, 0}: the ghost-layer-1
    // values that owned cells pull in sub-step 1, copied from the parent (Eq. ctof).
    std::vector<uint32_t> ework;
    // Coupled cells: owned fluid cells with a coalescence link (Eq. ftoc), the only owned cells
    // that read the finer level.  One cell index per entry, in cell order.
    std::vector<uint32_t> cwork;
    int64_t nghost12 = 0;          // fluid cells of ghost layers 1-2
    int64_t nfluid = 0;            // owned fluid cells
    int nbricks() const { return nown + nghost; }
};

struct Plan {
    lbm_forest_desc d{};
    int nlev = 0;
    int B = 0, LB = 0;
    bool per[3] = {false, false, false};
    std::vector<std::vector<uint8_t>> st;   // per level block state: 0 absent, 1 leaf, 2 split
    std::vector<HostLevel> lv;
};

bool build_plan(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag, void* user, Plan& p,
                std::string& err);
double scale_rate(double w0, int L);
double lambda_odd(double le, double magic);
// Sets the thread-local text that lbm_last_error returns.
void set_last_error(const char* msg);

}  // namespace lbm

struct lbm_plan {
    lbm::Plan p;
};
