// Device kernels of the refined-grid D3Q19 LBM, templated on storage type T, compute type C
// and collision model.  Included by one translation unit per storage precision.
//
// Storage per level: two PDF grids (Sec. 4.1 two-grid approach), each [19][ncells] with the
// cells of brick k at [k * B^3, (k+1) * B^3), x fastest.  The grids hold the POST-COLLISION
// state of owned cells (f-tilde, stored by the fused kernel) and the ghost-layer values that a
// later pull reads: the exploded layer-1 values that owned cells pull in sub-step 1 (Eq. ctof:
// every ghost cell takes its coarse parent's post-collision PDFs) and the streamed values of
// layers 1-2.  The ghost stream reads the other exploded values it needs from the coarse parent
// in the coarser level's grid.  FP32/FP16 storage holds f - f^eq(rho0, u0) ("shifted"; u0 = 0
// gives f - w rho0); FP64 holds f.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.h"

namespace lbm {

// D3Q19 velocity components in the public direction order, as constexpr functions so that the
// fully unrolled direction loops fold them into immediates.
__host__ __device__ constexpr int dex(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1 : ((q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0);
}
__host__ __device__ constexpr int dey(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1 : ((q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0);
}
__host__ __device__ constexpr int dez(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1 : ((q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0);
}
__host__ __device__ constexpr int dopp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr double dw(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// ------------------------------------------------------------------ storage conversions
template <typename T> struct Store;
template <> struct Store<double> {
    static constexpr bool shifted = false;
    __device__ __forceinline__ static double ld(const double* p) { return __ldg(p); }
    __device__ __forceinline__ static void st(double* p, double v) { *p = v; }
    __device__ __forceinline__ static void st_d(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
    static constexpr bool shifted = true;
    __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
    __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
    __device__ __forceinline__ static void st_d(float* p, double v) { *p = float(v); }
};
template <> struct Store<__half> {
    static constexpr bool shifted = true;
    __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
    __device__ __forceinline__ static void st_d(__half* p, double v) { *p = __double2half(v); }
};

template <typename C> __device__ __forceinline__ C qnan();
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000ULL); }
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }

// Knuth's TwoSum: s = fl(a + b) and e with a + b = s + e exactly (round-to-nearest FP32).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// f^eq_q(rho0, u0): what the shifted layouts subtract from f_q (w_q rho0 when u0 = 0).
__device__ __forceinline__ double shift_value(int q, double rho0, const double (&u0)[3]) {
    const double eu = dex(q) * u0[0] + dey(q) * u0[1] + dez(q) * u0[2];
    const double usq = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
    return dw(q) * rho0 * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
}

// ------------------------------------------------------------------ shared-memory staging
// 4-byte asynchronous copies global -> shared (LDGSTS); a false predicate zero-fills without
// reading global memory.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool pred) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(pred ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Cells whose pulls are in flight per thread in the FP32 column walk (pipeline depth).
#ifndef LBM_CP_STAGES
#define LBM_CP_STAGES 2
#endif

// ------------------------------------------------------------------ collision (Sec. 2, 2.1)
// v holds f (or its shifted form) on entry and f-tilde on exit.  R is rho (or rho - rho0).
// SRT: f~ = f - omega (f - f^eq) + F;  TRT: f~ = f - le (f+ - f^eq+) - lo (f- - f^eq-) + F, with
// f^eq of Eq. (fequ) and F_a = 3 w_a rho0 e_a . a (Sec. 2.1); the velocity inside f^eq is
// sum_a e_a f_a / rho0, unmodified by the force.
// The body force enters as fa = 3 rho0 a (three values): F_q = w_q (e_q . fa), F_opp(q) = -F_q.
// rec(R, jx, jy, jz) receives the post-streaming moments the collision starts from.
// With FP32 arithmetic (the shifted layouts) v holds f - f^eq(rho0, u0): then R = rho - rho0,
// j = rho0 (u - u0), and the equilibrium is taken relative to the same shift; two_u0 = 2 u0 and
// e_two_u0[a] = 2 e_a . u0 (constants of the launch).  u0 = 0 gives the f - w rho0 layout.  FP64
// arithmetic (unshifted storage) ignores them.
template <typename C, int COLL, typename Rec>
__device__ __forceinline__ void collide(C (&v)[19], C le, C lo, const C (&fa)[3], C rho0, C inv_rho0,
                                        const float (&two_u0)[3], const float (&e_two_u0)[19], Rec&& rec) {
    constexpr bool kShift = sizeof(C) == 4;
    C R = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
    for (int q = 0; q < 19; q++) {
        R += v[q];
        if (dex(q)) jx += dex(q) > 0 ? v[q] : -v[q];
        if (dey(q)) jy += dey(q) > 0 ? v[q] : -v[q];
        if (dez(q)) jz += dez(q) > 0 ? v[q] : -v[q];
    }
    rec(R, jx, jy, jz);
    // d = j / rho0 (u - u0 when shifted): the shifted equilibrium's quadratic terms are
    // (e.u)^2 - (e.u0)^2 = (e.d)(e.d + 2 e.u0) and u^2 - u0^2 = d.(d + 2 u0)
    const C ux = jx * inv_rho0, uy = jy * inv_rho0, uz = jz * inv_rho0;
    C usq = ux * ux + uy * uy + uz * uz;
    if constexpr (kShift) usq += ux * C(two_u0[0]) + uy * C(two_u0[1]) + uz * C(two_u0[2]);
    const C base = C(1.5) * rho0 * usq;
    {
        const C feq0 = C(dw(0)) * (R - base);
        v[0] = v[0] - le * (v[0] - feq0);
    }
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const int p = q + 1;
        C eu = C(0);
        if (dex(q)) eu += dex(q) > 0 ? ux : -ux;
        if (dey(q)) eu += dey(q) > 0 ? uy : -uy;
        if (dez(q)) eu += dez(q) > 0 ? uz : -uz;
        C ea = C(0);
        if (dex(q)) ea += dex(q) > 0 ? fa[0] : -fa[0];
        if (dey(q)) ea += dey(q) > 0 ? fa[1] : -fa[1];
        if (dez(q)) ea += dez(q) > 0 ? fa[2] : -fa[2];
        const C w = C(dw(q));
        const C Fq = w * ea;
        C es = eu;
        if constexpr (kShift) es += C(e_two_u0[q]);
        const C eqp = w * (R + rho0 * (C(4.5) * eu * es) - base);
        const C eqm = w * rho0 * C(3.0) * eu;
        if (COLL == LBM_TRT) {
            const C fp = C(0.5) * (v[q] + v[p]);
            const C fm = C(0.5) * (v[q] - v[p]);
            const C dp = le * (fp - eqp);
            const C dm = lo * (fm - eqm);
            const C a = v[q] - dp - dm + Fq;
            const C b = v[p] - dp + dm - Fq;
            v[q] = a;
            v[p] = b;
        } else {
            const C a = v[q] - le * (v[q] - (eqp + eqm)) + Fq;
            const C b = v[p] - le * (v[p] - (eqp - eqm)) - Fq;
            v[q] = a;
            v[p] = b;
        }
    }
}

template <typename T, typename C>
struct Access {
    const StepArgs& a;
    int LB, M;
    __device__ __forceinline__ C load(const void* base, int64_t n, int q, int64_t idx) const {
        return C(Store<T>::ld(static_cast<const T*>(base) + int64_t(q) * n + idx));
    }
    // Exploded value of direction q in cell (lx, ly, lz) of ghost brick gb (Eq. ctof): the
    // post-collision PDF of the coarse parent cell, which the coarser level's current grid holds
    // unchanged while this level runs its two sub-steps.
    __device__ __forceinline__ C coarse(int gb, int lx, int ly, int lz, int q) const {
        const int P = __ldg(a.lv.parent + gb);
        const int cb = P >> 3, oct = P & 7, H = 1 << (LB - 1);
        const int cx = (oct & 1) * H + (lx >> 1), cy = ((oct >> 1) & 1) * H + (ly >> 1), cz = (oct >> 2) * H + (lz >> 1);
        const int64_t idx = (int64_t(cb) << (3 * LB)) + (cz << (2 * LB)) + (cy << LB) + cx;
        return load(a.co.f[a.cur_c], a.co.ncells, q, idx);
    }
    // Mean of the 8 finer children of owned cell (x, y, z) of brick b after both fine sub-steps
    // (coalescence, Eq. ftoc), summed pairwise in z-y-x bit order.  With FP64 storage the sum is
    // FP64.  With FP32/FP16 storage it is an FP32 double-word sum (Knuth's TwoSum at every
    // addition, the rounding errors carried in a second word): the children are FP32/FP16
    // values, so this carries the exact sum as the FP64 accumulation would, up to the final
    // rounding, while using the FP32 pipe (GB300 runs FP64 at a small fraction of FP32 rate,
    // and coalescing cells are often isolated lanes of a warp).
    __device__ __forceinline__ C children_mean(int b, int x, int y, int z, int q) const {
        const int oct = ((2 * x) >> LB) | (((2 * y) >> LB) << 1) | (((2 * z) >> LB) << 2);
        const int cb = __ldg(a.lv.child + b * 8 + oct);
        if (cb < 0) return qnan<C>();
        const int cx = (2 * x) & M, cy = (2 * y) & M, cz = (2 * z) & M;
        const int64_t base = (int64_t(cb) << (3 * LB)) + (cz << (2 * LB)) + (cy << LB) + cx;
        const int sy = 1 << LB, sz = 1 << (2 * LB);
        const T* f = static_cast<const T*>(a.fi.f[a.cur_f]) + int64_t(q) * a.fi.ncells + base;
        const C c0 = C(Store<T>::ld(f)), c1 = C(Store<T>::ld(f + 1));
        const C c2 = C(Store<T>::ld(f + sy)), c3 = C(Store<T>::ld(f + sy + 1));
        const C c4 = C(Store<T>::ld(f + sz)), c5 = C(Store<T>::ld(f + sz + 1));
        const C c6 = C(Store<T>::ld(f + sz + sy)), c7 = C(Store<T>::ld(f + sz + sy + 1));
        if constexpr (sizeof(C) == 8) {
            const C s = ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7));
            return s * C(0.125);
        } else {
            float e01, e23, e45, e67, e03, e47, e07;
            const float s01 = two_sum(c0, c1, e01), s23 = two_sum(c2, c3, e23);
            const float s45 = two_sum(c4, c5, e45), s67 = two_sum(c6, c7, e67);
            const float s03 = two_sum(s01, s23, e03), s47 = two_sum(s45, s67, e47);
            const float s07 = two_sum(s03, s47, e07);
            const float err = ((e01 + e23) + (e45 + e67)) + (e03 + e47) + e07;
            return (s07 + err) * 0.125f;
        }
    }
};

// Compute-precision view of the per-level parameters.
template <typename C> struct Par;
template <> struct Par<double> {
    __device__ __forceinline__ static double le(const LevelParams* P) { return P->le; }
    __device__ __forceinline__ static double lo(const LevelParams* P) { return P->lo; }
    __device__ __forceinline__ static double fa(const LevelParams* P, int k) { return P->fa[k]; }
};
template <> struct Par<float> {
    __device__ __forceinline__ static float le(const LevelParams* P) { return P->lef; }
    __device__ __forceinline__ static float lo(const LevelParams* P) { return P->lof; }
    __device__ __forceinline__ static float fa(const LevelParams* P, int k) { return P->faf[k]; }
};

// General pull of direction q into cell (x, y, z) of brick `brick` (owned or ghost), for the
// links the link mask routes here:
//   - coalescence (owned cells only): mean of the 8 finer children of x (Eq. ftoc);
//   - obstacle or domain wall: bounce-back of the cell's own opposite value (Sec. 2.2), plus
//     6 w rho0 e.(u_w - u0) (u_w = 0 except on velocity walls, u0 the storage shift), or the
//     specular reflection of free-slip faces; a source beyond several faces takes the first
//     non-free-slip face of
//     z+, z-, y+, y-, x+, x-.  A ghost cell's own value in sub-step 1 is the exploded one;
//   - otherwise the value of the source cell: stored (owned, or ghost layers 1-2 after their
//     sub-step-1 stream), or exploded (ghost layers in sub-step 1, layer 3 always).
template <typename T, typename C, int LB>
__device__ C pull_general(const StepArgs& a, const Access<T, C>& acc, int brick, int x, int y, int z, int q,
                          bool owned) {
    constexpr int B = 1 << LB, M = B - 1, B3s = 3 * LB;
    const int ex = dex(q), ey = dey(q), ez = dez(q);
    const int sx = x - ex, sy = y - ey, sz = z - ez;
    const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
    const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
    const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
    const int* nbr = a.lv.nbr + brick * 27;
    const int nb = (ox | oy | oz) ? __ldg(nbr + 13 + ox + 3 * oy + 9 * oz) : brick;
    const void* src = a.lv.f[a.cur];
    const int64_t n = a.lv.ncells;
    const int64_t cidx = (int64_t(brick) << B3s) + (z << (2 * LB)) + (y << LB) + x;
    if (owned && (__ldg(a.lv.kind + brick) & BK_TOUCH_FINER)) {
        bool coal = nb == NB_FINER;
        if (!coal && ex && ox) coal = __ldg(nbr + 13 + ox) == NB_FINER;
        if (!coal && ey && oy) coal = __ldg(nbr + 13 + 3 * oy) == NB_FINER;
        if (!coal && ez && oz) coal = __ldg(nbr + 13 + 9 * oz) == NB_FINER;
        if (coal) return acc.children_mean(brick, x, y, z, q);
    }
    const int qo = dopp(q);
    const bool own_exploded = !owned && a.substep == 1;
    if (nb >= 0) {
        const int64_t sidx = (int64_t(nb) << B3s) + ((sz & M) << (2 * LB)) + ((sy & M) << LB) + (sx & M);
        const uint8_t ck = __ldg(a.lv.cell + sidx);
        if (ck == CK_SOLID) {
            C t = own_exploded ? acc.coarse(brick, x, y, z, qo) : acc.load(src, n, qo, cidx);
            if (a.obstacle_term) t += C(__ldg(a.wall + 7 * 19 + q));
            return t;
        }
        if (ck == CK_FAR) return qnan<C>();   // never a source: layer 4+ holds no value
        if (nb >= a.lv.nown && (a.substep == 1 || ck == CK_G3)) return acc.coarse(nb, sx & M, sy & M, sz & M, q);
        return acc.load(src, n, q, sidx);
    }
    if (nb == NB_WALL) {
        const int* P = a.lv.pos + 3 * brick;
        const int g[3] = {P[0] * B + sx, P[1] * B + sy, P[2] * B + sz};
        // the first non-free-slip face the source lies beyond, in the order z+, z-, y+, y-, x+, x-
        int face = -1, mirror = 0;
        if (!a.fslip) {
            if (!(a.per & 4) && g[2] >= a.lv.N[2]) face = 5;
            else if (!(a.per & 4) && g[2] < 0) face = 4;
            else if (!(a.per & 2) && g[1] >= a.lv.N[1]) face = 3;
            else if (!(a.per & 2) && g[1] < 0) face = 2;
            else if (!(a.per & 1) && g[0] >= a.lv.N[0]) face = 1;
            else face = 0;
        } else {
#pragma unroll
            for (int f = 5; f >= 0; f--) {
                const int ax = f >> 1;
                if ((a.per >> ax) & 1) continue;
                if (!((f & 1) ? g[ax] >= a.lv.N[ax] : g[ax] < 0)) continue;
                if ((a.fslip >> f) & 1) {
                    mirror |= 1 << ax;
                } else {
                    face = f;
                    break;
                }
            }
        }
        if (face < 0 && owned) {
            // every face is free-slip: specular reflection.  The value comes from the tangential
            // neighbour (the source moved back inside along the mirrored axes), in direction q
            // with those components reversed; an obstacle there bounces it back instead.  The
            // neighbour is an owned cell of this level (no level interface meets a free-slip face).
            const int mx = (mirror & 1) ? x : sx, my = (mirror & 2) ? y : sy, mz = (mirror & 4) ? z : sz;
            const int mox = mx < 0 ? -1 : (mx > M ? 1 : 0);
            const int moy = my < 0 ? -1 : (my > M ? 1 : 0);
            const int moz = mz < 0 ? -1 : (mz > M ? 1 : 0);
            const int mb = (mox | moy | moz) ? __ldg(nbr + 13 + mox + 3 * moy + 9 * moz) : brick;
            const int rx = (mirror & 1) ? -ex : ex, ry = (mirror & 2) ? -ey : ey, rz = (mirror & 4) ? -ez : ez;
            int qm = q;
#pragma unroll
            for (int k = 1; k < 19; k++)
                if (dex(k) == rx && dey(k) == ry && dez(k) == rz) qm = k;
            if (mb >= 0) {
                const int64_t midx = (int64_t(mb) << B3s) + ((mz & M) << (2 * LB)) + ((my & M) << LB) + (mx & M);
                if (__ldg(a.lv.cell + midx) != CK_SOLID) {
                    // the shifted layouts store f - f^eq(rho0, u0): f^eq_qm - f^eq_q of the shift is
                    // w rho0 (1.5 (E' - E) + 1.125 (E'^2 - E^2)) with E = 2 e_q.u0, E' = 2 e_qm.u0
                    const float E = a.e_two_u0[q], Em = a.e_two_u0[qm];
                    return acc.load(src, n, qm, midx) +
                           C(float(dw(q)) * float(a.rho0) * (1.5f * (Em - E) + 1.125f * (Em * Em - E * E)));
                }
            }
            face = 7;   // obstacle at the mirrored cell: bounce-back, obstacle term
        }
        if (face < 0) face = 7;   // not reached: ghost cells never meet a free-slip face
        const C o = own_exploded ? acc.coarse(brick, x, y, z, qo) : acc.load(src, n, qo, cidx);
        return o + C(__ldg(a.wall + face * 19 + q));
    }
    return qnan<C>();
}

// One sub-step of one level (Alg. 2 StreamCollide generalised to every level): pull stream with
// boundary treatment and coalescence, then collide owned cells; ghost layers 1-2 are streamed
// only, and only the values a later pull reads.  The grid: first the coupled cells' CTAs (owned
// cells with a coalescence link, one thread per cell), then the column walk over the other owned
// cells, then the ghost work list of this sub-step.  In the walk each thread walks 2^lzc cells of
// one (x, y) column of a brick; the source offsets of a cell inside the brick are computed once
// per column, obstacle and coupled cells are skipped by a per-column bitmap, and a per-cell link
// mask (read where the brick needs it) routes the few links that are not plain loads to
// pull_general.
// FP32 storage stages each cell's 19 pulls in shared memory with cp.async, two cells deep; the
// other storage types load into registers.  The same array receives general-pull values.
template <typename T, typename C>
struct StepSmem {
    static constexpr bool kAsync = sizeof(T) == 4;
    static constexpr int kStages = LBM_CP_STAGES;
    C slow[kAsync ? kStages : 1][19][256];
    C tot[4][256];   // per-thread moments of the recording launch
};

// The work of CTA `bid` of one launch of F_L(s) (see step_kernel); every thread of the CTA calls it.
template <typename T, typename C, int COLL, int LB>
__device__ __forceinline__ void step_block(const StepArgs& a, int64_t bid, StepSmem<T, C>& smem) {
    constexpr int B = 1 << LB, M = B - 1, B2s = 2 * LB, B3s = 3 * LB;
    constexpr bool kAsync = StepSmem<T, C>::kAsync;
    auto& slow = smem.slow;
    const int zc = 1 << a.lzc;
    const int upb = (1 << B2s) << (LB - a.lzc);            // units (column chunks) per brick
    const int64_t owned_units = int64_t(a.lv.nown) * upb;
    const int64_t owned_ctas = (owned_units + 255) >> 8;
    const int64_t coupled_ctas = (int64_t(a.lv.ncwork) + 255) >> 8;
    const T* src = static_cast<const T*>(a.lv.f[a.cur]);
    T* dst = static_cast<T*>(a.lv.f[a.cur ^ 1]);
    const int64_t n = a.lv.ncells;
    const Access<T, C> acc{a, LB, M};
    const int tid = threadIdx.x;

    if (bid < coupled_ctas) {
        // coupled cells (those with a coalescence link, which the column walk skips), first in the
        // grid so that their longer dependent chains overlap the walk: one thread per cell, plain
        // pulls as in the walk, the marked links through the general path, then the collision; the
        // recording launch appends their moments, one entry per warp after the walk's entries
        const int j = int(bid * 256 + tid);
        const bool want_tot = a.totals != nullptr;
        C mom[4] = {C(0), C(0), C(0), C(0)};
        if (j < a.lv.ncwork) {
            const int c = int(__ldg(a.lv.cwork + j));
            const int brick = c >> B3s, local = c & ((1 << B3s) - 1);
            const int x = local & M, y = (local >> LB) & M, z = local >> B2s;
            const uint32_t mq = __ldg(a.lv.link + c) & LINK_ALL;
            const int* nbr = a.lv.nbr + brick * 27;
            C v[19];
            v[0] = acc.load(src, n, 0, c);
#pragma unroll
            for (int q = 1; q < 19; q++) {
                v[q] = C(0);
                if (!((mq >> q) & 1u)) {   // plain: the source holds the value (stored, in the grid)
                    const int sx = x - dex(q), sy = y - dey(q), sz = z - dez(q);
                    const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
                    const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
                    const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
                    const int nb = (ox | oy | oz) ? __ldg(nbr + 13 + ox + 3 * oy + 9 * oz) : brick;
                    const int sidx = (max(nb, 0) << B3s) + ((sz & M) << B2s) + ((sy & M) << LB) + (sx & M);
                    v[q] = acc.load(src, n, q, sidx);
                }
            }
            C(&buf)[19][256] = slow[0];
            for (int q = 1; q < 19; q++)
                if ((mq >> q) & 1u) buf[q][tid] = pull_general<T, C, LB>(a, acc, brick, x, y, z, q, true);
#pragma unroll
            for (int q = 1; q < 19; q++)
                if ((mq >> q) & 1u) v[q] = buf[q][tid];
            const LevelParams* P = a.params;
            const C fa[3] = {Par<C>::fa(P, 0), Par<C>::fa(P, 1), Par<C>::fa(P, 2)};
            collide<C, COLL>(v, Par<C>::le(P), Par<C>::lo(P), fa, C(a.rho0), C(a.inv_rho0), a.two_u0, a.e_two_u0,
                             [&](C R, C jx, C jy, C jz) {
                                 mom[0] = R;
                                 mom[1] = jx;
                                 mom[2] = jy;
                                 mom[3] = jz;
                             });
            T* p = dst + c;
#pragma unroll
            for (int q = 0; q < 19; q++) Store<T>::st(p + int64_t(q) * n, v[q]);
        }
        if (want_tot) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                C t = mom[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
                if ((tid & 31) == 0) a.totals[((owned_units >> 5) + bid * 8 + (tid >> 5)) * 4 + k] = double(t);
            }
        }
        return;
    }
    bid -= coupled_ctas;
    if (bid < owned_ctas) {
        const int64_t u = bid * 256 + tid;
        // totals of the state this launch writes (the level's last sub-step of a coarse step): the
        // post-streaming moments of its owned fluid cells, one {R, jx, jy, jz} per warp, summed in
        // shared memory per thread (registers held across the cell loop would spill)
        const bool want_tot = a.totals != nullptr;
        C(&tot)[4][256] = smem.tot;
        if (want_tot)
            for (int k = 0; k < 4; k++) tot[k][tid] = C(0);
        if (u >= owned_units) return;   // whole warps: owned_units is a multiple of 64
        const int brick = int(u / upb);
        const int r = int(u - int64_t(brick) * upb);
        const int col = r & ((1 << B2s) - 1);
        const int x = col & M, y = col >> LB;
        const int z0 = (r >> B2s) << a.lzc;
        const uint8_t bk = __ldg(a.lv.kind + brick);
        const int* nbr = a.lv.nbr + brick * 27;
        const bool need_mask = !(bk & BK_PLAIN) && __ldg(a.lv.colspec + (brick << B2s) + col);
        // source offsets of a cell inside the brick along z (in-plane neighbour bricks resolved)
        int off[19];
#pragma unroll
        for (int q = 1; q < 19; q++) {
            const int sx = x - dex(q), sy = y - dey(q);
            const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
            const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
            const int nb = (ox | oy) ? __ldg(nbr + 13 + ox + 3 * oy) : brick;
            off[q] = (max(nb, 0) << B3s) + ((sy & M) << LB) + (sx & M) - dez(q) * (1 << B2s);
        }
        // source index of pull q into the cell at height z; on the brick's z faces the links
        // that leave the brick read the z-neighbour brick (z is uniform in a warp)
        auto src_index = [&](int q, int z) -> int {
            int sidx = off[q] + (z << B2s);
            if ((dez(q) == 1 && z == 0) || (dez(q) == -1 && z == M)) {
                const int sx = x - dex(q), sy = y - dey(q), oz = dez(q) == 1 ? -1 : 1;
                const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
                const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
                const int nb = __ldg(nbr + 13 + ox + 3 * oy + 9 * oz);
                sidx = (max(nb, 0) << B3s) + ((oz < 0 ? M : 0) << B2s) + ((sy & M) << LB) + (sx & M);
            }
            return sidx;
        };
        // cells the walk skips: obstacle cells, and coupled cells (their own CTAs)
        const uint32_t solid = need_mask ? __ldg(a.lv.colsolid + (brick << B2s) + col) : 0u;
        const LevelParams* P = a.params;
        const C le = Par<C>::le(P), lo = Par<C>::lo(P);
        const C fa[3] = {Par<C>::fa(P, 0), Par<C>::fa(P, 1), Par<C>::fa(P, 2)};
        const C rho0 = C(a.rho0), inv_rho0 = C(a.inv_rho0);
        // Links the link mask marks are replaced after the plain pulls (every plain address lies
        // inside the level's grid, so nothing waits for the mask).
        auto finish = [&](int z, int cidx, uint32_t m, C (&v)[19], C (&buf)[19][256]) {
            const uint32_t mq = m & LINK_ALL;
            if (m & LINK_BOUNCE_ONLY) {
                // every marked link bounces back: the cell's own opposite value, plus the term of
                // one wall face (face 7: obstacle links only)
                const T* p = src + cidx;
                const int face = int((m >> 25) & 7u);
#pragma unroll
                for (int q = 1; q < 19; q++)
                    if ((mq >> q) & 1u) {
                        C t = C(Store<T>::ld(p + int64_t(dopp(q)) * n));
                        if (face != 7 || a.obstacle_term) t += C(__ldg(a.wall + face * 19 + q));
                        v[q] = t;
                    }
            } else if (m & LINK_COAL_ONLY) {
#pragma unroll
                for (int q = 1; q < 19; q++)
                    if ((mq >> q) & 1u) v[q] = acc.children_mean(brick, x, y, z, q);
            } else if (mq) {
                for (int q = 1; q < 19; q++)
                    if ((mq >> q) & 1u) buf[q][tid] = pull_general<T, C, LB>(a, acc, brick, x, y, z, q, true);
#pragma unroll
                for (int q = 1; q < 19; q++)
                    if ((mq >> q) & 1u) v[q] = buf[q][tid];
            }
            collide<C, COLL>(v, le, lo, fa, rho0, inv_rho0, a.two_u0, a.e_two_u0, [&](C R, C jx, C jy, C jz) {
                if (want_tot) {
                    tot[0][tid] += R;
                    tot[1][tid] += jx;
                    tot[2][tid] += jy;
                    tot[3][tid] += jz;
                }
            });
            T* p = dst + cidx;
#pragma unroll
            for (int q = 0; q < 19; q++) {
                Store<T>::st(p, v[q]);
                p += n;
            }
        };
        if constexpr (kAsync) {
            // pipeline: the pulls of the next kStages - 1 cells are in flight while cell k collides
            constexpr int kStages = StepSmem<T, C>::kStages;
            auto issue = [&](int k) -> uint32_t {
                const int z = z0 + k;
                const int cidx = (brick << B3s) + (z << B2s) + (y << LB) + x;
                const bool live = !((solid >> z) & 1u);
                C(&stage)[19][256] = slow[k % kStages];
                if (live) {   // an obstacle cell's stage is never read: no copies
                    const T* p = src;
                    cp_async4(&stage[0][tid], p + cidx, true);
#pragma unroll
                    for (int q = 1; q < 19; q++) {
                        p += n;
                        cp_async4(&stage[q][tid], p + src_index(q, z), true);
                    }
                }
                cp_async_commit();
                return (need_mask && live) ? __ldg(a.lv.link + cidx) : 0u;
            };
            uint32_t mq[kStages - 1];
#pragma unroll
            for (int j = 0; j < kStages - 1; j++) {
                mq[j] = 0u;
                if (j < zc) mq[j] = issue(j);
                else cp_async_commit();
            }
            for (int k = 0; k < zc; k++) {
                const uint32_t m = mq[0];
#pragma unroll
                for (int j = 0; j + 1 < kStages - 1; j++) mq[j] = mq[j + 1];
                if (k + kStages - 1 < zc) mq[kStages - 2] = issue(k + kStages - 1);
                else cp_async_commit();
                cp_async_wait<kStages - 1>();
                const int z = z0 + k;
                if ((solid >> z) & 1u) continue;
                const int cidx = (brick << B3s) + (z << B2s) + (y << LB) + x;
                C(&stage)[19][256] = slow[k % kStages];
                C v[19];
#pragma unroll
                for (int q = 0; q < 19; q++) v[q] = stage[q][tid];
                finish(z, cidx, m, v, stage);
            }
        } else {
            for (int k = 0; k < zc; k++) {
                const int z = z0 + k;
                const int cidx = (brick << B3s) + (z << B2s) + (y << LB) + x;
                if ((solid >> z) & 1u) continue;
                const uint32_t m = need_mask ? __ldg(a.lv.link + cidx) : 0u;
                C v[19];
                const T* p = src;
                v[0] = C(Store<T>::ld(p + cidx));
#pragma unroll
                for (int q = 1; q < 19; q++) {
                    p += n;
                    v[q] = C(Store<T>::ld(p + src_index(q, z)));
                }
                finish(z, cidx, m, v, slow[0]);
            }
        }
        if (want_tot) {
            // the warp's sum in the compute type (FP64 arithmetic runs at a small fraction of the
            // FP32 rate on this GPU, and a launch with one cell per thread would feel it)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                C t = tot[k][tid];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
                if ((tid & 31) == 0) a.totals[(bid * 8 + (tid >> 5)) * 4 + k] = double(t);
            }
        }
        return;
    }
    const int gs = a.substep - 1;
    // ghost layers 1-2: stream only, the directions the work entry needs; a source holding an
    // exploded value is read from the coarse parent, and bounce-back/wall links take the general pull
    const int i = int((bid - owned_ctas) * 256 + tid);
    if (i >= a.lv.ngwork[gs]) return;
    const uint4 e = __ldg(a.lv.gwork[gs] + i);
    const int c = int(e.x);
    const uint32_t need = e.y, cm = e.z, sm = e.w;
    const int brick = c >> B3s, local = c & ((1 << B3s) - 1);
    const int x = local & M, y = (local >> LB) & M, z = local >> B2s;
    const int* nbr = a.lv.nbr + brick * 27;
    C v[19];
#pragma unroll
    for (int q = 1; q < 19; q++) {
        v[q] = C(0);
        if (((need & ~sm) >> q) & 1u) {
            const int sx = x - dex(q), sy = y - dey(q), sz = z - dez(q);
            const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
            const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
            const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
            const int nb = (ox | oy | oz) ? __ldg(nbr + 13 + ox + 3 * oy + 9 * oz) : brick;
            if ((cm >> q) & 1u) {
                v[q] = acc.coarse(nb, sx & M, sy & M, sz & M, q);
            } else {
                const int sidx = (max(nb, 0) << B3s) + ((sz & M) << B2s) + ((sy & M) << LB) + (sx & M);
                v[q] = acc.load(src, n, q, sidx);
            }
        }
    }
    if (sm) {
        for (int q = 1; q < 19; q++)
            if ((sm >> q) & 1u) slow[0][q][tid] = pull_general<T, C, LB>(a, acc, brick, x, y, z, q, false);
#pragma unroll
        for (int q = 1; q < 19; q++)
            if ((sm >> q) & 1u) v[q] = slow[0][q][tid];
    }
    T* p = dst + c;
#pragma unroll
    for (int q = 1; q < 19; q++)
        if ((need >> q) & 1u) Store<T>::st(p + int64_t(q) * n, v[q]);
}

template <typename T, typename C, int COLL, int LB, int MINB>
__global__ void __launch_bounds__(256, MINB) step_kernel(const StepArgs a) {
    __shared__ StepSmem<T, C> sm;
    step_block<T, C, COLL, LB>(a, blockIdx.x, sm);
}

// Copies the launch arguments of the forest that owns virtual CTA v of a batched phase into shared
// memory; returns v's index within that forest's launch.  prefix[k] is the first virtual CTA of
// forest k (prefix[0] = 0, prefix[n] = the phase's total).  Every thread of the CTA calls it.
__device__ __forceinline__ int64_t batch_args(const StepArgs* args, const int* prefix, int n, int v, StepArgs& sa) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= v) lo = mid;
        else hi = mid;
    }
    __syncthreads();   // the previous iteration's readers of sa are done
    constexpr int words = int(sizeof(StepArgs) / 4);
    const int* s = reinterpret_cast<const int*>(args + lo);
    int* d = reinterpret_cast<int*>(&sa);
    for (int w = threadIdx.x; w < words; w += blockDim.x) d[w] = __ldg(s + w);
    __syncthreads();
    return int64_t(v - __ldg(prefix + lo));
}

// One phase F_L(s) of a batch of forests in one persistent launch: virtual CTA v of the phase
// (v < total) is CTA v - prefix[k] of forest k's own launch, with forest k's arguments.
template <typename T, typename C, int COLL, int LB, int MINB>
__global__ void __launch_bounds__(256, MINB) step_batch_kernel(const StepArgs* args, const int* prefix, int n, int total) {
    __shared__ StepSmem<T, C> sm;
    __shared__ StepArgs sa;
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int64_t bid = batch_args(args, prefix, n, v, sa);
        step_block<T, C, COLL, LB>(sa, bid, sm);
    }
}

// Explosion (Eq. ctof) at the start of every visit of a finer level: the ghost-layer-1 values
// that owned cells pull in sub-step 1 take their coarse parent's post-collision PDFs, in the finer
// level's current grid.  One thread per work entry, one predicated copy per direction it lists.
template <typename T>
__device__ __forceinline__ void explode_entry(const DevLevel& lv, const DevLevel& co, int cur, int cur_c, int i) {
    if (i >= lv.nework) return;
    const uint4 e = __ldg(lv.ework + i);
    const T* src = static_cast<const T*>(co.f[cur_c]) + e.z;
    T* dst = static_cast<T*>(lv.f[cur]) + e.x;
    T v[19];
#pragma unroll
    for (int q = 1; q < 19; q++)
        if ((e.y >> q) & 1u) v[q] = __ldg(src + int64_t(q) * co.ncells);
#pragma unroll
    for (int q = 1; q < 19; q++)
        if ((e.y >> q) & 1u) dst[int64_t(q) * lv.ncells] = v[q];
}

template <typename T>
__global__ void __launch_bounds__(256) explode_kernel(const DevLevel lv, const DevLevel co, int cur, int cur_c) {
    explode_entry<T>(lv, co, cur, cur_c, blockIdx.x * blockDim.x + threadIdx.x);
}

// E_L of a batch of forests in one persistent launch (virtual CTAs as in step_batch_kernel).
template <typename T>
__global__ void __launch_bounds__(256) explode_batch_kernel(const StepArgs* args, const int* prefix, int n, int total) {
    __shared__ StepArgs sa;
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int64_t bid = batch_args(args, prefix, n, v, sa);
        explode_entry<T>(sa.lv, sa.co, sa.cur, sa.cur_c, int(bid) * 256 + threadIdx.x);
    }
}

// Equilibrium start (Eq. fequ) followed by one collision, so the stored state is post-collision.
// Every non-owned or obstacle cell is set to NaN.
template <typename T, typename C, int COLL>
__global__ void init_kernel(const DevLevel lv, int cur, int LB, const LevelParams* P, double rho0, const double* rho,
                            const double* u, int uniform, double ur, double ux0, double uy0, double uz0) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= lv.ncells) return;
    T* f = static_cast<T*>(lv.f[cur]);
    T* g = static_cast<T*>(lv.f[cur ^ 1]);
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    const bool valid = i < nown_cells && lv.cell[i] == CK_FLUID;
    if (!valid) {
#pragma unroll
        for (int q = 0; q < 19; q++) {
            Store<T>::st(f + q * lv.ncells + i, qnan<C>());
            Store<T>::st(g + q * lv.ncells + i, qnan<C>());
        }
        return;
    }
    double r, vx, vy, vz;
    if (uniform) {
        r = ur; vx = ux0; vy = uy0; vz = uz0;
    } else {
        r = rho ? rho[i] : rho0;
        vx = u ? u[i] : 0.0;
        vy = u ? u[nown_cells + i] : 0.0;
        vz = u ? u[2 * nown_cells + i] : 0.0;
    }
    const double usq = vx * vx + vy * vy + vz * vz;
    C v[19];
#pragma unroll
    for (int q = 0; q < 19; q++) {
        const double eu = dex(q) * vx + dey(q) * vy + dez(q) * vz;
        const double feq = dw(q) * (r + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
        v[q] = C(Store<T>::shifted ? feq - shift_value(q, rho0, lv.u0) : feq);
    }
    const C fa[3] = {C(P->fa[0]), C(P->fa[1]), C(P->fa[2])};
    float two_u0[3], e_two_u0[19];
    for (int k = 0; k < 3; k++) two_u0[k] = float(2.0 * lv.u0[k]);
#pragma unroll
    for (int q = 0; q < 19; q++) e_two_u0[q] = float(2.0 * (dex(q) * lv.u0[0] + dey(q) * lv.u0[1] + dez(q) * lv.u0[2]));
    collide<C, COLL>(v, C(P->le), C(P->lo), fa, C(rho0), C(1.0 / rho0), two_u0, e_two_u0, [](C, C, C, C) {});
#pragma unroll
    for (int q = 0; q < 19; q++) {
        Store<T>::st(f + q * lv.ncells + i, v[q]);
        Store<T>::st(g + q * lv.ncells + i, qnan<C>());
    }
}

// rho and u (+ a/2) of owned cells from the stored post-collision state: collision keeps rho and
// adds rho0 a to the momentum, so u_out = j~/rho0 - a/2 (Sec. 2.1).  u holds the three components
// `us` values apart (the level's cell count, or the total over all levels for the all-level layout).
template <typename T>
__global__ void macro_kernel(const DevLevel lv, int cur, int LB, const LevelParams* P, double rho0, double* rho,
                             double* u, int64_t us) {
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nown_cells) return;
    if (lv.cell[i] != CK_FLUID) {
        if (rho) rho[i] = __longlong_as_double(0x7ff8000000000000ULL);
        if (u) u[i] = u[us + i] = u[2 * us + i] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    const T* f = static_cast<const T*>(lv.f[cur]);
    double R = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < 19; q++) {
        const double v = double(Store<T>::ld(f + q * lv.ncells + i));
        R += v;
        jx += dex(q) * v;
        jy += dey(q) * v;
        jz += dez(q) * v;
    }
    if (rho) rho[i] = Store<T>::shifted ? rho0 + R : R;
    if (u) {   // the shifted layouts hold j - rho0 u0
        u[i] = jx / rho0 + lv.u0[0] - 0.5 * P->acc[0];
        u[us + i] = jy / rho0 + lv.u0[1] - 0.5 * P->acc[1];
        u[2 * us + i] = jz / rho0 + lv.u0[2] - 0.5 * P->acc[2];
    }
}

template <typename T>
__global__ void get_pdfs_kernel(const DevLevel lv, int cur, int LB, double rho0, double* out) {
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nown_cells) return;
    const T* f = static_cast<const T*>(lv.f[cur]);
#pragma unroll
    for (int q = 0; q < 19; q++) {
        const double v = double(Store<T>::ld(f + q * lv.ncells + i));
        out[q * nown_cells + i] = Store<T>::shifted ? v + shift_value(q, rho0, lv.u0) : v;
    }
}

template <typename T>
__global__ void set_pdfs_kernel(const DevLevel lv, int cur, int LB, double rho0, const double* in) {
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= lv.ncells) return;
    T* f = static_cast<T*>(lv.f[cur]);
#pragma unroll
    for (int q = 0; q < 19; q++) {
        double v = __longlong_as_double(0x7ff8000000000000ULL);
        if (i < nown_cells && lv.cell[i] == CK_FLUID)
            v = Store<T>::shifted ? in[q * nown_cells + i] - shift_value(q, rho0, lv.u0) : in[q * nown_cells + i];
        Store<T>::st_d(f + q * lv.ncells + i, v);
    }
}

// Per-CTA FP64 partial totals of one level: {w rho, w (j~ - rho0 a)} over owned fluid cells, with
// w = 8^-L.  partial[blockIdx][4]; summed in a fixed order by reduce_final_kernel.


// Volume-weighted totals of one level from the per-warp moments the step kernel left: n warp
// entries {R, jx, jy, jz}, plus {s0, s1, s2, s3} = (fluid cells) x {rho0, rho0 u0} for the shifted
// layouts (they sum f - f^eq(rho0, u0)).  The moments are post-streaming: no force correction.
template <typename T>
__global__ void __launch_bounds__(256) totals_level_kernel(const double* __restrict__ wpart, int64_t n, double w,
                                                           double s0, double s1, double s2, double s3,
                                                           double* partial) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        for (int k = 0; k < 4; k++) s[k] += wpart[4 * i + k];
    __shared__ double red[4][256];
    for (int k = 0; k < 4; k++) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (int(threadIdx.x) < h)
            for (int k = 0; k < 4; k++) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 4) {
        const double sh = threadIdx.x == 0 ? s0 : threadIdx.x == 1 ? s1 : threadIdx.x == 2 ? s2 : s3;
        partial[blockIdx.x * 4 + threadIdx.x] = w * (red[threadIdx.x][0] + (blockIdx.x == 0 ? sh : 0.0));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) reduce_level_kernel(const DevLevel lv, int cur, int LB, const LevelParams* P,
                                                          double rho0, double w, double* partial) {
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const T* f = static_cast<const T*>(lv.f[cur]);
    // With shifted storage a cell's 19 values are small deviations (f - f^eq(rho0, u0)), so the cell's sums
    // are formed in FP32 (an error near 1e-10 per cell) and only the totals run in FP64: GB300's
    // FP64 pipe would otherwise make this the slowest kernel of a step.  FP64 storage sums in FP64.
    using A = typename std::conditional<Store<T>::shifted, float, double>::type;
    const A ax = A(rho0 * P->acc[0]), ay = A(rho0 * P->acc[1]), az = A(rho0 * P->acc[2]);
    int64_t cells = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nown_cells; i += int64_t(gridDim.x) * blockDim.x) {
        if (lv.cell[i] != CK_FLUID) continue;
        A R = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int q = 0; q < 19; q++) {
            const A v = A(Store<T>::ld(f + q * lv.ncells + i));
            R += v;
            if (dex(q)) jx += dex(q) > 0 ? v : -v;
            if (dey(q)) jy += dey(q) > 0 ? v : -v;
            if (dez(q)) jz += dez(q) > 0 ? v : -v;
        }
        s[0] += double(R);
        s[1] += double(jx - ax);
        s[2] += double(jy - ay);
        s[3] += double(jz - az);
        cells++;
    }
    // volume weight, and rho0 (mass) and rho0 u0 (momentum) per fluid cell for the shifted layouts
    const double nc = Store<T>::shifted ? rho0 * double(cells) : 0.0;
    s[0] = w * (s[0] + nc);
    s[1] = w * (s[1] + nc * lv.u0[0]);
    s[2] = w * (s[2] + nc * lv.u0[1]);
    s[3] = w * (s[3] + nc * lv.u0[2]);
    __shared__ double red[4][8];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int wdx = 0; wdx < 8; wdx++) v += red[threadIdx.x][wdx];
        partial[blockIdx.x * 4 + threadIdx.x] = v;
    }
}

}  // namespace lbm
