// Structures shared between the host runtime (capi.cu) and the kernels, and the launchers that
// each per-precision translation unit provides.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_internal.h"

namespace lbm {

// Per-level parameters, device-resident so that captured graphs never need rebuilding.
struct LevelParams {
    double le, lo;        // lambda_e, lambda_o (omega, omega for SRT)
    double fa[3];         // 3 rho0 a_L: the body force term is F_a = w_a (e_a . fa), Sec. 2.1
    double acc[3];        // a_L
    float lef, lof;       // the same in FP32, for the FP32-arithmetic kernels
    float faf[3];
};

struct DevLevel {
    void* f[2];           // two PDF grids, [19][ncells]
    const uint8_t* cell;  // [ncells] CK_*
    const int32_t* nbr;   // [nbricks][27]
    const int32_t* parent;
    const int32_t* child;
    const int32_t* pos;   // [nbricks][3]
    const uint8_t* kind;  // [nbricks]
    const uint32_t* link;    // [nown * B^3] per owned cell: bit q set = link q needs the general
                             // pull; bits 25-29 fast-path codes; bit 31 = not a fluid cell
    const uint32_t* colsolid;  // [nown * B^2] per owned column: bit z = skipped by the column walk
                               // (not a fluid cell, or a coupled cell)
    const uint8_t* colspec;    // [nown * B^2] per owned column: 1 if any cell has a nonzero link mask
    const uint4* gwork[2];     // ghost stream work of sub-step 1 and 2: {cell, need, coarse, special}
    int ngwork[2];
    const uint4* ework;        // explosion work: {cell, directions, coarse parent cell, 0}
    int nework;
    const uint32_t* cwork;     // coupled cells (owned fluid cells with a coalescence link)
    int ncwork;
    int nown, nbricks;
    int64_t ncells;
    int N[3];
    double u0[3];         // storage shift velocity: shifted layouts hold f - f^eq(rho0, u0); 0 for FP64
};

struct StepArgs {
    DevLevel lv, co, fi;  // this level, the next coarser, the next finer
    int cur, cur_c, cur_f;
    int substep;          // 1: ghost layers hold the exploded (coarse) values; 2: layers 1-2 hold
                          // their sub-step-1 stream
    int LB;
    int lzc;              // log2 of the cells each thread walks along z
    int minb;             // CTAs per SM the kernel variant is compiled for (2, 3 or 4)
    int per;              // bit a set: axis a periodic
    int fslip;            // bit f set: face f (x-, x+, y-, y+, z-, z+) is free-slip
    const LevelParams* params;
    const double* wall;   // [8][19] bounce-back terms 6 w_a rho0 (e_a . (u_w - u0)): faces 0-5,
                          // row 7 obstacles (u_w = 0), row 6 unused
    double rho0, inv_rho0;
    double* totals;       // per-warp post-streaming moments of the owned cells, or NULL
    int obstacle_term;    // 1: obstacle bounce-backs add wall row 7 (a nonzero storage shift)
    float two_u0[3];      // 2 u0 and 2 e_a . u0 of the storage shift (FP32 arithmetic; 0 unshifted)
    float e_two_u0[19];
    int wctas;            // FP32/FP16 storage: the launch's persistent walk CTAs (its whole grid)
    int* wq;              // FP32/FP16 storage: the walk's chunk counter and finished-CTA counter,
                          // zero at the launch's start (its last CTA resets them)
};

// Bits of the per-cell link mask.
constexpr uint32_t LINK_NOT_FLUID = 1u << 31;
constexpr uint32_t LINK_BOUNCE_ONLY = 1u << 29;   // face of the wall term in bits 25-27
constexpr uint32_t LINK_COAL_ONLY = 1u << 28;
constexpr uint32_t LINK_ALL = 0x7FFFEu;   // directions 1..18

// Launchers (one set per storage precision: 0 FP64, 1 FP32S, 2 FP16S).
struct Launchers {
    void (*step)(const StepArgs& a, int collision, int grid, cudaStream_t s);
    void (*init)(const DevLevel& lv, int cur, int LB, const LevelParams* P, double rho0, const double* rho,
                 const double* u, int uniform, const double u_const[4], int collision, cudaStream_t s);
    void (*macro)(const DevLevel& lv, int cur, int LB, const LevelParams* P, double rho0, double* rho, double* u,
                  int64_t ustride, cudaStream_t s);
    void (*get_pdfs)(const DevLevel& lv, int cur, int LB, double rho0, double* out, cudaStream_t s);
    void (*set_pdfs)(const DevLevel& lv, int cur, int LB, double rho0, const double* in, cudaStream_t s);
    void (*reduce)(const DevLevel& lv, int cur, int LB, const LevelParams* P, double rho0, double w, double* partial,
                   int grid, cudaStream_t s);
    void (*totals)(const double* wpart, int64_t n, double w, const double shift[4], double* partial, int grid,
                   cudaStream_t s);
    void (*explode)(const DevLevel& lv, const DevLevel& co, int cur, int cur_c, cudaStream_t s);
    // One phase of a batch of forests: args[n] per forest, prefix[n+1] its first virtual CTA;
    // `grid` persistent CTAs walk the `total` virtual CTAs.
    void (*step_batch)(const StepArgs* args, const int* prefix, int n, int total, int grid, int collision, int LB,
                       int minb, cudaStream_t s);
    void (*explode_batch)(const StepArgs* args, const int* prefix, int n, int total, int grid, cudaStream_t s);
    // Sets the dynamic shared-memory limit of every step-kernel variant; call before launching
    // or capturing any of them (idempotent).
    cudaError_t (*prepare)();
    // CTAs per SM of the step kernel for block size 2^LB and the configured CTAs per SM (the shared
    // memory may allow fewer), and whether its column walk is persistent (FP32/FP16 storage).
    int (*ctas_per_sm)(int LB, int minb);
    bool persistent;
    // The coupled cells and ghost work of a persistent walk's F_L(s) (side_kernel), `grid` CTAs;
    // and of a batch of forests, as step_batch.
    void (*side)(const StepArgs& a, int collision, int grid, cudaStream_t s);
    void (*side_batch)(const StepArgs* args, const int* prefix, int n, int total, int grid, int collision, int LB,
                       cudaStream_t s);
};
const Launchers& launchers_f64();
const Launchers& launchers_f32();
const Launchers& launchers_f16();

}  // namespace lbm
