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
    __device__ __forceinline__ static double cv(double v) { return v; }
    __device__ __forceinline__ static void st(double* p, double v) { *p = v; }
    __device__ __forceinline__ static void st_d(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
    static constexpr bool shifted = true;
    __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
    __device__ __forceinline__ static float cv(float v) { return v; }
    __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
    __device__ __forceinline__ static void st_d(float* p, double v) { *p = float(v); }
};
template <> struct Store<__half> {
    static constexpr bool shifted = true;
    __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static float cv(__half v) { return __half2float(v); }
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
// 16-byte asynchronous copies global -> shared (LDGSTS, cached in L2 only), in commit groups.
__device__ __forceinline__ uint32_t sh_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sh_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------ collision (Sec. 2, 2.1)
// v holds f (or its shifted form) on entry and f-tilde on exit.
//   SRT: f~ = f - omega (f - f^eq) + F;  TRT: f~ = f - le (f+ - f^eq+) - lo (f- - f^eq-) + F,
// with f^eq of Eq. (fequ) and F_a = 3 w_a rho0 e_a . a (Sec. 2.1); the velocity inside f^eq is
// sum_a e_a f_a / rho0, unmodified by the force.  SRT is TRT with lo = le.  The body force enters
// as fa = 3 rho0 a (three values): F_q = w_q (e_q . fa), F_opp(q) = -F_q.
// The update is taken per opposite pair (q, qbar), with s = f_q + f_qbar and t = f_q - f_qbar:
//   f~_q = f_q - dp - dm',  f~_qbar = f_qbar - dp + dm',
//   dp  = le (s/2 - f^eq+_q),  f^eq+_q = w (R - base) + 4.5 w rho0 (e.d)(e.(d + 2 u0)),
//   dm' = lo t/2 - w e.(3 rho0 lo d + fa),          base = 1.5 rho0 d.(d + 2 u0),
// where R = sum_a v_a and d = sum_a e_a v_a / rho0.  For FP64 storage v = f, u0 = 0: R = rho,
// d = u.  The shifted layouts (FP32 arithmetic) hold f - f^eq(rho0, u0): then R = rho - rho0,
// d = u - u0, and the equilibrium is taken relative to the same shift (two_u0 = 2 u0, a launch
// constant; 0 for FP64).  rec(R, jx, jy, jz) receives the post-streaming moments the collision
// starts from.  collide2 computes the same update on two cells at once.
template <typename C, int COLL, typename Rec>
__device__ __forceinline__ void collide(C (&v)[19], C le, C lo, const C (&fa)[3], C rho0, C inv_rho0,
                                        const float (&two_u0)[3], Rec&& rec) {
    constexpr bool kShift = sizeof(C) == 4;
    if (COLL != LBM_TRT) lo = le;
    C s[19], t[19];   // indexed by the odd member of each opposite pair
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        s[q] = v[q] + v[q + 1];
        t[q] = v[q] - v[q + 1];
    }
    const C R = (((v[0] + s[1]) + (s[3] + s[5])) + ((s[7] + s[9]) + (s[11] + s[13]))) + (s[15] + s[17]);
    const C jx = (t[1] + t[7]) + ((t[9] + t[11]) + t[13]);
    const C jy = ((t[3] + t[7]) - t[9]) + (t[15] + t[17]);
    const C jz = (((t[5] + t[11]) - t[13]) + t[15]) - t[17];
    rec(R, jx, jy, jz);
    const C ux = jx * inv_rho0, uy = jy * inv_rho0, uz = jz * inv_rho0;
    const C wx = kShift ? ux + C(two_u0[0]) : ux, wy = kShift ? uy + C(two_u0[1]) : uy, wz = kShift ? uz + C(two_u0[2]) : uz;
    const C usq = uz * wz + (uy * wy + ux * wx);
    const C Rb = R - C(1.5) * rho0 * usq;
    const C w1 = C(dw(1)), w2 = C(dw(7));
    const C B1 = -le * w1 * Rb, B2 = -le * w2 * Rb;                        // -le w (R - base)
    const C K1 = -le * C(4.5) * rho0 * w1, K2 = -le * C(4.5) * rho0 * w2;   // -le 4.5 w rho0
    const C g3 = C(3.0) * rho0 * lo;
    const C gx = ux * g3 + fa[0], gy = uy * g3 + fa[1], gz = uz * g3 + fa[2];
    const C leh = C(0.5) * le, loh = C(0.5) * lo;
    v[0] = v[0] - le * (v[0] - C(dw(0)) * Rb);
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const bool diag = q >= 7;
        C eu = C(0), ew = C(0), eg = C(0);
        if (dex(q)) { eu += ux; ew += wx; eg += gx; }   // the first member of a pair has e_x >= 0
        if (dey(q)) {
            eu += dey(q) > 0 ? uy : -uy;
            ew += dey(q) > 0 ? wy : -wy;
            eg += dey(q) > 0 ? gy : -gy;
        }
        if (dez(q)) {
            eu += dez(q) > 0 ? uz : -uz;
            ew += dez(q) > 0 ? wz : -wz;
            eg += dez(q) > 0 ? gz : -gz;
        }
        const C dp = s[q] * leh + ((eu * ew) * (diag ? K2 : K1) + (diag ? B2 : B1));
        const C dm = t[q] * loh - (diag ? w2 : w1) * eg;
        const C a = (v[q] - dp) - dm;
        const C b = (v[q + 1] - dp) + dm;
        v[q] = a;
        v[q + 1] = b;
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
        if (face < 0) {
            // every face is free-slip: specular reflection.  The value comes from the tangential
            // neighbour (the source moved back inside along the mirrored axes), in direction q
            // with those components reversed; an obstacle there bounces it back instead.  Where a
            // level interface meets the face the neighbour may be a ghost cell (Sec. 4.1 extends
            // the boundary treatment to the ghost layers): it then holds the exploded value in
            // sub-step 1 and in layer 3, and its sub-step-1 stream otherwise, as any source does.
            const int mx = (mirror & 1) ? x : sx, my = (mirror & 2) ? y : sy, mz = (mirror & 4) ? z : sz;
            const int mox = mx < 0 ? -1 : (mx > M ? 1 : 0);
            const int moy = my < 0 ? -1 : (my > M ? 1 : 0);
            const int moz = mz < 0 ? -1 : (mz > M ? 1 : 0);
            const int mb = (mox | moy | moz) ? __ldg(nbr + 13 + mox + 3 * moy + 9 * moz) : brick;
            if (mb < 0) return qnan<C>();   // never a source: the planner checks every needed mirror
            const int rx = (mirror & 1) ? -ex : ex, ry = (mirror & 2) ? -ey : ey, rz = (mirror & 4) ? -ez : ez;
            int qm = q;
#pragma unroll
            for (int k = 1; k < 19; k++)
                if (dex(k) == rx && dey(k) == ry && dez(k) == rz) qm = k;
            const int64_t midx = (int64_t(mb) << B3s) + ((mz & M) << (2 * LB)) + ((my & M) << LB) + (mx & M);
            const uint8_t mck = __ldg(a.lv.cell + midx);
            if (mck != CK_SOLID) {
                if (mck == CK_FAR) return qnan<C>();
                const C v = (mb >= a.lv.nown && (a.substep == 1 || mck == CK_G3))
                                ? acc.coarse(mb, mx & M, my & M, mz & M, qm)
                                : acc.load(src, n, qm, midx);
                // the shifted layouts store f - f^eq(rho0, u0): f^eq_qm - f^eq_q of the shift is
                // w rho0 (1.5 (E' - E) + 1.125 (E'^2 - E^2)) with E = 2 e_q.u0, E' = 2 e_qm.u0
                const float E = a.e_two_u0[q], Em = a.e_two_u0[qm];
                return v + C(float(dw(q)) * float(a.rho0) * (1.5f * (Em - E) + 1.125f * (Em * Em - E * E)));
            }
            face = 7;   // obstacle at the mirrored cell: bounce-back, obstacle term
        }
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
// one (x, y) column of a brick, so each warp walks 32 / B rows of B cells along z; obstacle and
// coupled cells are skipped by a per-column bitmap, and a per-cell link mask (read where the brick
// needs it) routes the few links that are not plain loads to pull_general.
//
// Staging.  At each step of the walk the pulls of a row of B cells read, per direction q, one
// source row of B values shifted by -e_q: the row (y - e_qy, z - e_qz) of the brick or of its y/z
// neighbour, plus, for e_qx != 0, one value of the x-neighbour brick.  Each warp copies its rows'
// 19 source rows, and a 16-byte chunk holding each x-neighbour value, into its own part of shared
// memory with 16-byte asynchronous copies (cp.async, aligned, a few per lane), S steps ahead; its
// lanes then read their 19 pulls at x - e_qx of the staged rows.  The warps run independent
// pipelines (no CTA-wide barrier in the walk).  Rows whose cells are all skipped are not copied.
template <typename T, typename C, int LB, int MINB>
struct StepSmem {
    static constexpr int B = 1 << LB;
    static constexpr int H = 16 / int(sizeof(T));   // elements of one 16-byte chunk
    static constexpr int RS = B + 2 * H;            // staged row: [x-neighbour chunk][B values][chunk]
    static constexpr int CX = sizeof(T) < 8 ? 2 : 1;   // cells per thread along x (FP32 pairs)
    static constexpr int WR = 32 * CX / B;          // rows of one warp
    static constexpr int WSTAGE = WR * 19 * RS;     // elements of one warp's stage: [WR][19][RS]
    static constexpr int WSTAGE_BYTES = WSTAGE * int(sizeof(T));
    static constexpr int STAGE_BYTES = 8 * WSTAGE_BYTES;
    // the FP64 walk's thread writes general pulls into its own staged slots (each slot feeds exactly
    // one thread's pull); the coupled and ghost CTAs of its launch use the stages as their scratch
    static constexpr bool kSep = false;
    static constexpr int SCRATCH_BYTES = 19 * 256 * int(sizeof(C));
    static constexpr int TOT_BYTES = 4 * 256 * int(sizeof(C));
    // the FP16-storage walk also stages the link masks of each warp's rows: [WR][B] uint32 per warp
    static constexpr int LSTAGE = (CX == 2 && sizeof(T) == 2) ? WR * B : 0;
    static constexpr int LSTAGE_BYTES = 8 * LSTAGE * 4;
    static constexpr int kBudget = (227 * 1024) / MINB - 1024 - TOT_BYTES - 128;
    static constexpr int kFit = kBudget / (STAGE_BYTES + LSTAGE_BYTES);
    static constexpr int S = kFit > 6 ? 6 : (kFit < 2 ? 2 : kFit);   // pipeline depth in walk steps
    static constexpr int OFF_LINK = S * STAGE_BYTES;
    static constexpr int STAGES = OFF_LINK + S * LSTAGE_BYTES;
    static constexpr int AREA = STAGES > SCRATCH_BYTES ? STAGES : SCRATCH_BYTES;
    static constexpr int OFF_SCRATCH = 0;
    static constexpr int OFF_TOT = AREA;
    static constexpr int OFF_WALL = AREA + 4 * 256 * int(sizeof(C));   // [8][19] FP32 bounce-back terms
    static constexpr int BYTES = OFF_WALL + 8 * 19 * 4;
    // CTAs per SM the shared memory allows (228 KB per SM, 1 KB reserved per CTA, 128 bytes of
    // alignment slack): the launch bound asks for no more
    static constexpr int kFitCtas = (228 * 1024) / (BYTES + 128 + 1024);
    static constexpr int kMinCtas = MINB < kFitCtas ? MINB : (kFitCtas < 1 ? 1 : kFitCtas);
    static_assert(WSTAGE_BYTES % 16 == 0 && (RS * int(sizeof(T))) % 16 == 0 && OFF_LINK % 16 == 0,
                  "16-byte copies need 16-byte alignment");
};

// Directions with e_qx != 0, whose staged rows need the x-neighbour chunk.
__host__ __device__ constexpr int xdir(int k) {
    return k < 2 ? 1 + k : 5 + k;   // 1, 2, 7, 8, 9, 10, 11, 12, 13, 14
}

// The owned column walk of CTA `bid` (counted within the walk) of one launch of F_L(s).
template <typename T, typename C, int COLL, int LB, int MINB>
__device__ __forceinline__ void walk_block(const StepArgs& a, int64_t bid, unsigned char* smem) {
    using SP = StepSmem<T, C, LB, MINB>;
    constexpr int B = 1 << LB, M = B - 1, B2s = 2 * LB, B3s = 3 * LB;
    constexpr int S = SP::S, WR = SP::WR, RS = SP::RS, H = SP::H;
    constexpr int CR = B * int(sizeof(T)) / 16;   // 16-byte chunks of a row
    constexpr int JR = 19 * CR + 10;              // chunks of one row's staging: 19 rows + 10 x-chunks
    constexpr int JW = WR * JR;                   // copies per warp and step
    constexpr int JL = (JW + 31) / 32;            // copies per lane
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* wst = reinterpret_cast<T*>(smem) + warp * SP::WSTAGE;   // + s * 8 * WSTAGE
    C(&buf)[19][256] = *reinterpret_cast<C(*)[19][256]>(smem + SP::OFF_SCRATCH);
    C(&tot)[4][256] = *reinterpret_cast<C(*)[4][256]>(smem + SP::OFF_TOT);
    const int zc = 1 << a.lzc;
    const int upb = (1 << B2s) << (LB - a.lzc);            // units (column chunks) per brick
    const int64_t owned_units = int64_t(a.lv.nown) * upb;
    const T* src = static_cast<const T*>(a.lv.f[a.cur]);
    T* dst = static_cast<T*>(a.lv.f[a.cur ^ 1]);
    const int64_t n = a.lv.ncells;
    const Access<T, C> acc{a, LB, M};
    const bool want_tot = a.totals != nullptr;

    // this thread's cell column
    const int64_t u = bid * 256 + tid;
    const bool active = u < owned_units;
    int brick = 0, x = 0, y = 0, z0 = 0;
    uint32_t solid = 0xFFFFFFFFu;   // an inactive thread skips every cell
    bool need_mask = false;
    if (active) {
        brick = int(u / upb);
        const int r = int(u - int64_t(brick) * upb);
        const int col = r & ((1 << B2s) - 1);
        x = col & M;
        y = col >> LB;
        z0 = (r >> B2s) << a.lzc;
        const uint8_t bk = __ldg(a.lv.kind + brick);
        need_mask = !(bk & BK_PLAIN) && __ldg(a.lv.colspec + (brick << B2s) + col);
        // cells the walk skips: obstacle cells, and coupled cells (their own CTAs)
        solid = need_mask ? __ldg(a.lv.colsolid + (brick << B2s) + col) : 0u;
    }
    if (want_tot)
        for (int k = 0; k < 4; k++) tot[k][tid] = C(0);

    // This lane's copies (fixed for the walk): copy j = lane + 32 m of the warp is chunk kq of the
    // warp's row i: kq < 19 CR is chunk kq % CR of direction kq / CR, else the x-neighbour chunk of
    // direction xdir(kq - 19 CR).  Each row's brick and y come from its first lane; z = z0 + step is
    // the same for the whole warp.
    int jq[JL], jrow[JL], jc[JL];
    int jb[JL], jy[JL];
#pragma unroll
    for (int m = 0; m < JL; m++) {
        const int j = lane + 32 * m;
        const int i = j / JR, kq = j % JR;
        jrow[m] = j < JW ? i : -1;
        jq[m] = kq < 19 * CR ? kq / CR : xdir(kq - 19 * CR);
        jc[m] = kq < 19 * CR ? kq % CR : -1;
        const int src_lane = i * B;   // the row's first lane
        jb[m] = __shfl_sync(0xffffffffu, brick, src_lane & 31);
        jy[m] = __shfl_sync(0xffffffffu, y, src_lane & 31);
    }

    // the warp's rows with a cell to update at walk step k, one bit per row
    auto live_rows = [&](int k) -> uint32_t {
        const bool live = !((solid >> ((z0 + k) & 31)) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, live);
        uint32_t bits = 0;
#pragma unroll
        for (int i = 0; i < WR; i++)
            if ((bal >> (i * B)) & ((B == 32) ? 0xffffffffu : ((1u << (B & 31)) - 1u))) bits |= 1u << i;
        return bits;
    };
    // issues this lane's copies of walk step k into the warp's stage k % S (after the warp's last
    // reads of that stage) and commits them as one group
    auto issue = [&](int k) {
        const uint32_t lm = live_rows(k);
        T* st = wst + (k % S) * 8 * SP::WSTAGE;
        const int z = z0 + k;
#pragma unroll
        for (int m = 0; m < JL; m++) {
            const int i = jrow[m];
            if (i < 0 || !((lm >> i) & 1u)) continue;
            const int q = jq[m];
            const bool halo = jc[m] < 0;
            const int ex = dex(q), sy = jy[m] - dey(q), sz = z - dez(q);
            const int ox = halo ? (ex > 0 ? -1 : 1) : 0;
            const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
            const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
            int nb = (ox | oy | oz) ? __ldg(a.lv.nbr + jb[m] * 27 + 13 + ox + 3 * oy + 9 * oz) : jb[m];
            // a source outside this level's storage (wall, finer or absent block): copy any valid
            // row instead; the link mask routes every such pull to the general path
            if (nb < 0) nb = jb[m];
            const int sx = halo ? (ex > 0 ? B - H : 0) : jc[m] * H;
            const T* from = src + int64_t(q) * n + (int64_t(nb) << B3s) + ((sz & M) << B2s) + ((sy & M) << LB) + sx;
            T* to = st + (i * 19 + q) * RS + (halo ? (ex > 0 ? 0 : H + B) : H + sx);
            cp_async16(to, from);
        }
        cp_async_commit();
    };

    for (int k = 0; k < S - 1; k++) {
        if (k < zc) issue(k);
        else cp_async_commit();
    }

    const LevelParams* P = a.params;
    const C le = Par<C>::le(P), lo = Par<C>::lo(P);
    const C fa[3] = {Par<C>::fa(P, 0), Par<C>::fa(P, 1), Par<C>::fa(P, 2)};
    const C rho0 = C(a.rho0), inv_rho0 = C(a.inv_rho0);
    const int row = lane / B;   // this thread's row in the warp
    for (int k = 0; k < zc; k++) {
        const int kk = k + S - 1;
        if (kk < zc) {
            __syncwarp();   // the warp's lanes are done with stage kk % S (read in step k - 1)
            issue(kk);
        } else {
            cp_async_commit();
        }
        cp_async_wait<S - 1>();   // this lane's copies of step k have landed
        __syncwarp();             // and every lane's
        const int s = k % S;
        const int z = z0 + k;
        if (!((solid >> (z & 31)) & 1u)) {
            const int cidx = (brick << B3s) + (z << B2s) + (y << LB) + x;
            const uint32_t m = need_mask ? __ldg(a.lv.link + cidx) : 0u;
            T* st = wst + s * 8 * SP::WSTAGE + row * 19 * RS + H + x;   // + q * RS - e_qx
            C v[19];
#pragma unroll
            for (int q = 0; q < 19; q++) v[q] = C(Store<T>::cv(st[q * RS - dex(q)]));
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
                // general pulls through shared memory (a runtime direction index into v would put
                // v in local memory): the thread's own staged slots, or the FP32 scratch for FP16
                for (int q = 1; q < 19; q++)
                    if ((mq >> q) & 1u) {
                        const C g = pull_general<T, C, LB>(a, acc, brick, x, y, z, q, true);
                        if constexpr (SP::kSep) buf[q][tid] = g;
                        else st[q * RS - dex(q)] = T(g);
                    }
#pragma unroll
                for (int q = 1; q < 19; q++)
                    if ((mq >> q) & 1u) {
                        if constexpr (SP::kSep) v[q] = buf[q][tid];
                        else v[q] = C(st[q * RS - dex(q)]);
                    }
            }
            collide<C, COLL>(v, le, lo, fa, rho0, inv_rho0, a.two_u0, [&](C R, C jx, C jy, C jz) {
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
        }
    }
    cp_async_wait<0>();
    if (want_tot && active) {
        // the warp's sum in the compute type (FP64 arithmetic runs at a small fraction of the
        // FP32 rate on this GPU, and a launch with one cell per thread would feel it)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            C t = tot[q][tid];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) a.totals[(bid * 8 + warp) * 4 + q] = double(t);
        }
    }
}

// ------------------------------------------------------------------ packed FP32 pairs
// Two FP32 values in one 64-bit register pair, for the FP32x2 arithmetic of sm_100-class GPUs
// (add/sub/mul/fma .rn.f32x2: each half rounds exactly as the scalar .rn instruction would).
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_make(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 f2_dup(float a) { return f2_make(a, a); }
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float(unsigned(v & 0xffffffffull)); }
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float(unsigned(v >> 32)); }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a * b + c
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// e_q . (ax, ay, az) for the first member q of an opposite pair (q odd: its first nonzero
// component is +1); with q a constant of an unrolled loop this folds into at most one addition
__device__ __forceinline__ f2 f2_edot(int q, f2 ax, f2 ay, f2 az) {
    const int X = dex(q), Y = dey(q), Z = dez(q);
    if (X != 0 && Y != 0) return Y > 0 ? f2_add(ax, ay) : f2_sub(ax, ay);
    if (X != 0 && Z != 0) return Z > 0 ? f2_add(ax, az) : f2_sub(ax, az);
    if (Y != 0 && Z != 0) return Z > 0 ? f2_add(ay, az) : f2_sub(ay, az);
    if (X != 0) return ax;
    if (Y != 0) return ay;
    return az;
}

// Per-launch constants of the packed collision (both halves equal).
struct Collide2Consts {
    f2 inv_rho0, tu0x, tu0y, tu0z;   // 1/rho0; 2 u0 of the storage shift
    f2 c15r;                         // 1.5 rho0
    f2 nlew1, nlew2, w0;             // -le w for |e|^2 = 1, 2; the rest weight w0
    f2 nk1, nk2;                     // -le 4.5 rho0 w, |e|^2 = 1, 2
    f2 leh, loh, nle;                // le / 2, lo / 2, -le
    f2 c3rlo;                        // 3 rho0 lo
    f2 fax, fay, faz;                // 3 rho0 a (the body-force term: F_a = w_a e_a . fa)
    f2 nw1, nw2;                     // -w for |e|^2 = 1, 2
};

__device__ __forceinline__ Collide2Consts collide2_consts(float le, float lo, const float (&fa)[3], float rho0,
                                                          float inv_rho0, const float (&two_u0)[3]) {
    const float w1 = float(dw(1)), w2 = float(dw(7)), w0 = float(dw(0));
    Collide2Consts k;
    k.inv_rho0 = f2_dup(inv_rho0);
    k.tu0x = f2_dup(two_u0[0]);
    k.tu0y = f2_dup(two_u0[1]);
    k.tu0z = f2_dup(two_u0[2]);
    k.c15r = f2_dup(1.5f * rho0);
    k.nlew1 = f2_dup(-le * w1);
    k.nlew2 = f2_dup(-le * w2);
    k.w0 = f2_dup(w0);
    k.nk1 = f2_dup(-le * 4.5f * rho0 * w1);
    k.nk2 = f2_dup(-le * 4.5f * rho0 * w2);
    k.leh = f2_dup(0.5f * le);
    k.loh = f2_dup(0.5f * lo);
    k.nle = f2_dup(-le);
    k.c3rlo = f2_dup(3.0f * rho0 * lo);
    k.fax = f2_dup(fa[0]);
    k.fay = f2_dup(fa[1]);
    k.faz = f2_dup(fa[2]);
    k.nw1 = f2_dup(-w1);
    k.nw2 = f2_dup(-w2);
    return k;
}

// The collision (Sec. 2, 2.1) of two cells at once in FP32x2, for the shifted layouts (v holds
// f - f^eq(rho0, u0); R = rho - rho0, d = j / rho0 = u - u0), in TRT form (SRT: lo = le).  With
// s = f_q + f_qbar and t = f_q - f_qbar of an opposite pair, the update is
//   f~_q = f_q - dp - dm',  f~_qbar = f_qbar - dp + dm',
//   dp  = le (s/2 - f^eq+_q)      with f^eq+_q = w (R - base) + 4.5 w rho0 (e.d)(e.(d + 2 u0)),
//   dm' = lo t/2 - w e.(3 rho0 lo d + fa),
// base = 1.5 rho0 d.(d + 2 u0): the same relaxation of the even and odd parts and the same force
// term F_q = w e_q . fa as the scalar collide, with the equilibrium taken relative to the shift.
// rec(R, jx, jy, jz) receives the moments the collision starts from.
template <typename Rec>
__device__ __forceinline__ void collide2(f2 (&v)[19], const Collide2Consts& k, Rec&& rec) {
    f2 s[19], t[19];   // indexed by the odd member of each opposite pair
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        s[q] = f2_add(v[q], v[q + 1]);
        t[q] = f2_sub(v[q], v[q + 1]);
    }
    const f2 R = f2_add(f2_add(f2_add(f2_add(v[0], s[1]), f2_add(s[3], s[5])), f2_add(f2_add(s[7], s[9]), f2_add(s[11], s[13]))),
                        f2_add(s[15], s[17]));
    const f2 jx = f2_add(f2_add(t[1], t[7]), f2_add(f2_add(t[9], t[11]), t[13]));
    const f2 jy = f2_add(f2_sub(f2_add(t[3], t[7]), t[9]), f2_add(t[15], t[17]));
    const f2 jz = f2_sub(f2_add(f2_sub(f2_add(t[5], t[11]), t[13]), t[15]), t[17]);
    rec(R, jx, jy, jz);
    const f2 ux = f2_mul(jx, k.inv_rho0), uy = f2_mul(jy, k.inv_rho0), uz = f2_mul(jz, k.inv_rho0);
    const f2 wx = f2_add(ux, k.tu0x), wy = f2_add(uy, k.tu0y), wz = f2_add(uz, k.tu0z);
    const f2 usq = f2_fma(uz, wz, f2_fma(uy, wy, f2_mul(ux, wx)));
    const f2 Rb = f2_sub(R, f2_mul(k.c15r, usq));
    const f2 B1 = f2_mul(k.nlew1, Rb), B2 = f2_mul(k.nlew2, Rb);   // -le w (R - base)
    const f2 gx = f2_fma(ux, k.c3rlo, k.fax), gy = f2_fma(uy, k.c3rlo, k.fay), gz = f2_fma(uz, k.c3rlo, k.faz);
    // rest direction: f~_0 = f_0 - le (f_0 - w0 (R - base))
    v[0] = f2_fma(k.nle, f2_sub(v[0], f2_mul(k.w0, Rb)), v[0]);
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const bool diag = q >= 7;
        const f2 eu = f2_edot(q, ux, uy, uz);
        const f2 ew = f2_edot(q, wx, wy, wz);
        const f2 eg = f2_edot(q, gx, gy, gz);
        // dp = le s/2 - le f^eq+ = le/2 s + (-le w (R - base)) + (-le 4.5 w rho0)(e.d)(e.w)
        const f2 dp = f2_fma(s[q], k.leh, f2_fma(f2_mul(eu, ew), diag ? k.nk2 : k.nk1, diag ? B2 : B1));
        const f2 dm = f2_fma(t[q], k.loh, f2_mul(eg, diag ? k.nw2 : k.nw1));
        const f2 a = f2_sub(f2_sub(v[q], dp), dm);
        const f2 b = f2_add(f2_sub(v[q + 1], dp), dm);
        v[q] = a;
        v[q + 1] = b;
    }
}

// Two staged pulls of direction q (cells x and x + 1 of the row) as an FP32 pair.
template <typename T, int RS>
__device__ __forceinline__ f2 staged_pair(const T* st, int q) {
    const T* p = st + q * RS - dex(q);
    if constexpr (std::is_same<T, float>::value) {
        if (dex(q) == 0) {
            const float2 w = *reinterpret_cast<const float2*>(p);
            return f2_make(w.x, w.y);
        }
        return f2_make(p[0], p[1]);
    } else {
        if (dex(q) == 0) {
            const float2 w = __half22float2(*reinterpret_cast<const __half2*>(p));
            return f2_make(w.x, w.y);
        }
        return f2_make(__half2float(p[0]), __half2float(p[1]));
    }
}

// The stored value at p as FP32 if pred, else `other`: a predicated load (no branch), so that the
// loads of several bounce-back links issue back to back.
__device__ __forceinline__ float pred_ld(const float* p, bool pred, float other) {
    float r = other;
    asm("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q ld.global.nc.f32 %0, [%1];\n}\n" : "+f"(r) : "l"(p), "r"(int(pred)));
    return r;
}
__device__ __forceinline__ float pred_ld(const __half* p, bool pred, float other) {
    unsigned short h = 0;
    asm("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q ld.global.nc.b16 %0, [%1];\n}\n" : "+h"(h) : "l"(p), "r"(int(pred)));
    return pred ? __half2float(__ushort_as_half(h)) : other;
}

// Stores an FP32 pair as the two cells' values in storage type T.
template <typename T>
__device__ __forceinline__ void store_pair(T* p, f2 v) {
    if constexpr (std::is_same<T, float>::value) {
        *reinterpret_cast<float2*>(p) = make_float2(f2_lo(v), f2_hi(v));
    } else {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(f2_lo(v), f2_hi(v));
    }
}

// The owned column walk for the shifted layouts (FP32 or FP16 storage, FP32 arithmetic), CTA
// `cta` of the launch's `ncta` walk CTAs (persistent).  Each thread takes two x-adjacent cells (x,
// x + 1) of a row; a warp's 32 threads cover WR = 64 / B rows, a row group.  The work is divided
// into chunks (brick, block of ZC = 2^a.lzc planes, row group), row groups fastest, that the warps take one
// at a time from a counter of the launch (a.wq[0]), so that the warps working at any moment stage
// nearby rows of nearby planes and finish together.  Each warp runs one pipeline over its chunks:
// the staging of walk_block (16-byte copies per lane into the warp's own stages, S tasks ahead; a
// task is one plane of a chunk), with each lane's source pointers advanced by one plane per task
// and recomputed per chunk and where a task's source plane leaves the brick.  A pair whose two
// cells are fluid with no marked link collides in FP32x2; any other live cell takes the scalar
// path of walk_cell.  Each warp records one totals entry; the launch's last CTA resets the counter.
template <typename T, int COLL, int LB, int MINB>
__device__ __forceinline__ void walk_packed(const StepArgs& a, int cta, int ncta, unsigned char* smem) {
    using C = float;
    using SP = StepSmem<T, C, LB, MINB>;
    static_assert(SP::CX == 2, "two cells per thread");
    constexpr int B = 1 << LB, M = B - 1, B2s = 2 * LB, B3s = 3 * LB;
    constexpr int S = SP::S, WR = SP::WR, RS = SP::RS, H = SP::H;
    constexpr int CR = B * int(sizeof(T)) / 16;   // 16-byte chunks of a row
    constexpr int RPM = 32 / CR;                  // row sets one lane step covers
    constexpr int NRS = WR * 19;                  // row sets (row i, direction q) of a warp
    constexpr int MJ = (NRS + RPM - 1) / RPM;     // row copies per lane
    constexpr int NH = WR * 10;                   // x-neighbour chunks of a warp
    constexpr int HJ = (NH + 31) / 32;            // x-neighbour copies per lane
    constexpr int NG = B / WR;                    // row groups of a plane
    static_assert(WR <= 8 && MJ <= 10, "job packing");
    // planes of a chunk: 2^a.lzc (the launch's choice), at least S so that the pipeline spans at
    // most two chunks, at most B
    const int zl = a.lzc < (S > 4 ? 3 : S > 2 ? 2 : 1) ? (S > 4 ? 3 : S > 2 ? 2 : 1) : (a.lzc > LB ? LB : a.lzc);
    const int ZC = 1 << zl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* wst = reinterpret_cast<T*>(smem) + warp * SP::WSTAGE;   // + s * 8 * WSTAGE
    constexpr bool kLinkStaged = SP::LSTAGE > 0;                 // FP16 storage
    static_assert(!kLinkStaged || WR * B / 4 == 16, "a warp's link-mask rows are 16 chunks of 16 bytes");
    C(&tot)[4][256] = *reinterpret_cast<C(*)[4][256]>(smem + SP::OFF_TOT);
    const T* src = static_cast<const T*>(a.lv.f[a.cur]);
    T* dst = static_cast<T*>(a.lv.f[a.cur ^ 1]);
    const int64_t n = a.lv.ncells;
    const Access<T, C> acc{a, LB, M};
    const bool want_tot = a.totals != nullptr;
    if (want_tot)
        for (int k = 0; k < 4; k++) tot[k][tid] = C(0);
    // bounce-back terms 6 w rho0 e.(u_w - u0) per wall face and direction in FP32; row 7 (obstacle
    // links) only under a storage shift
    float* wt = reinterpret_cast<float*>(smem + SP::OFF_WALL);
    if (tid < 8 * 19) wt[tid] = (tid < 7 * 19 || a.obstacle_term) ? float(__ldg(a.wall + tid)) : 0.f;
    __syncthreads();
    const int64_t gw = int64_t(cta) * 8 + warp;
    const int nchunk = (a.lv.nown << (LB - zl)) * NG;
    // the next chunk of the launch, or -1
    auto fetch = [&]() -> int {
        int id = 0;
        if (lane == 0) id = atomicAdd(a.wq, 1);
        id = __shfl_sync(0xffffffffu, id, 0);
        return id < nchunk ? id : -1;
    };
    // task k (0 <= k < ZC) of chunk id: brick, row group, plane
    auto task = [&](int id, int k, int& brick, int& rg, int& z) {
        rg = id % NG;
        const int r = id / NG;
        brick = r >> (LB - zl);
        z = ((r & ((1 << (LB - zl)) - 1)) << zl) + k;
    };
    const int xl = 2 * (lane % (B / 2)), row = lane / (B / 2);   // this lane's cells x, x + 1 and row
    const int c = lane % CR, rs0 = lane / CR;                     // this lane's copy chunk and first row set
    // Column data of a task group (brick, row group): which cells of this lane's two columns the
    // walk skips (obstacle and coupled cells) and whether their link masks are needed.  Two
    // independent loads (columns x and x + 1 are adjacent); the issuing side takes them at a chunk's
    // first task and, with FP16 storage, the consuming side reuses them.
    struct Cols {
        uint32_t sol0, sol1;
        bool nm0, nm1;
    };
    auto columns = [&](int brick, int rg) -> Cols {
        const int col = (brick << B2s) + ((rg * WR + row) << LB) + xl;
        const uint2 sol = __ldg(reinterpret_cast<const uint2*>(a.lv.colsolid + col));
        const unsigned short sp = __ldg(reinterpret_cast<const unsigned short*>(a.lv.colspec + col));
        return Cols{sol.x, sol.y, (sp & 0xFFu) != 0u, (sp >> 8) != 0u};
    };
    // the same, skipping plain bricks (one load fewer there, a dependent chain elsewhere): fewer
    // registers, which the FP32-storage walk (at its register limit) needs
    auto columns_plain = [&](int brick, int rg) -> Cols {
        Cols k{0u, 0u, false, false};
        if (!(__ldg(a.lv.kind + brick) & BK_PLAIN)) {
            const int col = (brick << B2s) + ((rg * WR + row) << LB) + xl;
            k.nm0 = __ldg(a.lv.colspec + col) != 0;
            k.nm1 = __ldg(a.lv.colspec + col + 1) != 0;
            if (k.nm0) k.sol0 = __ldg(a.lv.colsolid + col);
            if (k.nm1) k.sol1 = __ldg(a.lv.colsolid + col + 1);
        }
        return k;
    };
    // source of a copy: direction q, row i of row group rg, chunk offset sx (elements) within the
    // source row, x-neighbour ox, at plane z of the brick (every neighbour resolved)
    auto source = [&](int brick, int rg, int q, int i, int sx, int ox, int z) -> const T* {
        const int sy = rg * WR + i - dey(q), sz = z - dez(q);
        const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
        const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
        int nb = (ox | oy | oz) ? __ldg(a.lv.nbr + brick * 27 + 13 + ox + 3 * oy + 9 * oz) : brick;
        // a source outside this level's storage (wall, finer or absent block): copy any valid row
        // instead; the link mask routes every such pull to the general path
        if (nb < 0) nb = brick;
        return src + int64_t(q) * n + (int64_t(nb) << B3s) + ((sz & M) << B2s) + ((sy & M) << LB) + sx;
    };
    // the same with the source plane z - e_qz taken unwrapped (one plane before or after the brick
    // at its z faces, where the copies are recomputed with `source`): advancing it by one plane
    // per task follows the brick's planes
    auto base = [&](int brick, int rg, int q, int i, int sx, int ox, int z) -> const T* {
        const int sy = rg * WR + i - dey(q);
        const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
        int nb = (ox | oy) ? __ldg(a.lv.nbr + brick * 27 + 13 + ox + 3 * oy) : brick;
        if (nb < 0) nb = brick;
        return src + int64_t(q) * n + (int64_t(nb) << B3s) + int64_t(z - dez(q)) * (1 << B2s) + ((sy & M) << LB) + sx;
    };
    // This lane's copies.  Row copy m: chunk c of row set rs = rs0 + RPM m, that is direction rs % 19
    // of the warp's row rs / 19, into [rs][H + c H] of the warp's stage.  x-neighbour copy mh: chunk
    // h = lane + 32 mh of the warp, direction xdir(h % 10) of row h / 10.
    const T* mp[MJ];
    const T* hp[HJ];
    int hdst[HJ];
    uint32_t mrow = 0;   // 3 bits per row copy: its row
#pragma unroll
    for (int m = 0; m < MJ; m++) {
        const int rs = rs0 + RPM * m;
        mrow |= uint32_t(rs < NRS ? rs / 19 : 0) << (3 * m);
        mp[m] = nullptr;
    }
#pragma unroll
    for (int mh = 0; mh < HJ; mh++) {
        const int h = lane + 32 * mh;
        const int i = h / 10, q = xdir(h - 10 * i);
        hdst[mh] = (i * 19 + q) * RS + (dex(q) < 0 ? H + B : 0);
        hp[mh] = nullptr;
    }
    // the issuing side: its chunk and next task (pointers mp / hp, column data icol)
    int ich = fetch(), ik = 0;
    Cols icol{0u, 0u, false, false};
    bool imask = false;   // FP16 storage: some lane of the chunk needs its link masks
    // issues the next task of the issuing side into stage k % S (after the warp's last reads of that
    // stage) and commits its copies as one group (an empty group once the launch has no work left)
    auto issue = [&](int k) {
        if (ich < 0) {
            cp_async_commit();
            return;
        }
        int brick, rg, z;
        task(ich, ik, brick, rg, z);
        if (ik == 0) {
            if constexpr (sizeof(T) == 2) {
                icol = columns(brick, rg);
                imask = __any_sync(0xffffffffu, icol.nm0 || icol.nm1);
            } else {
                icol = columns(brick, rg);
            }
#pragma unroll
            for (int m = 0; m < MJ; m++) {
                const int rs = rs0 + RPM * m;
                const int i = rs / 19;
                mp[m] = rs < NRS ? base(brick, rg, rs - 19 * i, i, c * H, 0, z) : nullptr;
            }
#pragma unroll
            for (int mh = 0; mh < HJ; mh++) {
                const int h = lane + 32 * mh;
                const int i = h / 10, q = xdir(h - 10 * i);
                const bool right = dex(q) < 0;   // the pull reads x + 1: the +x neighbour's first chunk
                hp[mh] = h < NH ? base(brick, rg, q, i, right ? 0 : B - H, right ? 1 : -1, z) : nullptr;
            }
        }
        // rows with a cell to update
        const bool live = !((icol.sol0 >> z) & (icol.sol1 >> z) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, live);
        uint32_t lm = 0;
#pragma unroll
        for (int i = 0; i < WR; i++)
            if ((bal >> (i * (B / 2))) & ((1u << (B / 2)) - 1u)) lm |= 1u << i;
        const bool all = lm == (1u << WR) - 1u;
        T* st = wst + (k % S) * 8 * SP::WSTAGE;
        const bool face = z == 0 || z == M;   // a source plane z - e_qz may lie in a z neighbour
#pragma unroll
        for (int m = 0; m < MJ; m++) {
            if (!mp[m]) continue;
            const int i = int((mrow >> (3 * m)) & 7u);
            const int rs = rs0 + RPM * m;
            if (all || ((lm >> i) & 1u))
                cp_async16(st + rs * RS + H + c * H, face ? source(brick, rg, rs - 19 * i, i, c * H, 0, z) : mp[m]);
            mp[m] += 1 << B2s;
        }
#pragma unroll
        for (int mh = 0; mh < HJ; mh++) {
            if (!hp[mh]) continue;
            const int h = lane + 32 * mh;
            const int i = h / 10;
            if (all || ((lm >> i) & 1u)) {
                const T* from = hp[mh];
                if (face) {
                    const int q = xdir(h - 10 * i);
                    const bool right = dex(q) < 0;
                    from = source(brick, rg, q, i, right ? 0 : B - H, right ? 1 : -1, z);
                }
                cp_async16(st + hdst[mh], from);
            }
            hp[mh] += 1 << B2s;
        }
        if constexpr (kLinkStaged) {
            // the link masks of the task's rows, where any lane of the chunk needs them: 16 lanes copy
            // one 16-byte chunk each
            if (imask && lane < 16) {
                constexpr int CPR = B / 4;   // 16-byte chunks per row of masks
                const int i = lane / CPR, cc = lane - CPR * i;
                uint32_t* ls = reinterpret_cast<uint32_t*>(smem + SP::OFF_LINK) + ((k % S) * 8 + warp) * SP::LSTAGE;
                if (all || ((lm >> i) & 1u))
                    cp_async16(ls + i * B + cc * 4,
                               a.lv.link + (int64_t(brick) << B3s) + (z << B2s) + ((rg * WR + i) << LB) + cc * 4);
            }
        }
        cp_async_commit();
        if (++ik == ZC) {
            ich = fetch();
            ik = 0;
        }
    };

    for (int k = 0; k < S - 1; k++) issue(k);

    const LevelParams* P = a.params;
    const Collide2Consts K = collide2_consts(P->lef, COLL == LBM_TRT ? P->lof : P->lef, P->faf, float(a.rho0),
                                             float(a.inv_rho0), a.two_u0);
    auto rec1 = [&](C R, C jx, C jy, C jz) {
        if (want_tot) {
            tot[0][tid] += R;
            tot[1][tid] += jx;
            tot[2][tid] += jy;
            tot[3][tid] += jz;
        }
    };
    // the consuming side: its chunk and task; it trails the issuing side by S - 1 <= ZC tasks, so
    // when it leaves a chunk the issuing side has moved to the next one (or found none)
    int cch = -2, ck = 0;
    Cols ccol{0u, 0u, false, false};
    for (int k = 0;; k++) {
        if (cch == -2) cch = ich;   // the first chunk: the one the issuing side started with
        if (cch < 0) break;
        __syncwarp();   // the warp's lanes are done with stage (k + S - 1) % S (read in task k - 1)
        issue(k + S - 1);
        cp_async_wait<S - 1>();   // this lane's copies of task k have landed
        __syncwarp();             // and every lane's
        int brick, rg, z;
        task(cch, ck, brick, rg, z);
        if (ck == 0) {
            // FP16 storage: the issuing side's copy (it is still within this chunk, S - 1 < ZC);
            // FP32 storage loads it again, which keeps it within its registers
            if constexpr (sizeof(T) == 2) ccol = icol;
            else ccol = columns(brick, rg);
        }
        const bool l0 = !((ccol.sol0 >> z) & 1u), l1 = !((ccol.sol1 >> z) & 1u);
        if (l0 || l1) {
            const int y = rg * WR + row;
            const int cidx = (brick << B3s) + (z << B2s) + (y << LB) + xl;
            uint32_t m0, m1;
            if constexpr (kLinkStaged) {
                // staged with the rows (copied whenever a lane of the chunk has a masked column)
                const uint32_t* lrow = reinterpret_cast<const uint32_t*>(smem + SP::OFF_LINK) +
                                       ((k % S) * 8 + warp) * SP::LSTAGE + row * B + xl;
                m0 = (ccol.nm0 && l0) ? lrow[0] : 0u;
                m1 = (ccol.nm1 && l1) ? lrow[1] : 0u;
            } else {
                m0 = (ccol.nm0 && l0) ? __ldg(a.lv.link + cidx) : 0u;
                m1 = (ccol.nm1 && l1) ? __ldg(a.lv.link + cidx + 1) : 0u;
            }
            T* st = wst + (k % S) * 8 * SP::WSTAGE + row * 19 * RS + H + xl;   // + q * RS - e_qx
            f2 v[19];
#pragma unroll
            for (int q = 0; q < 19; q++) v[q] = staged_pair<T, RS>(st, q);
            const uint32_t mm = (m0 | m1) & LINK_ALL;
            if (mm) {
                // bounce-back links (the only marked links the paired walk sees; the planner routes
                // every other kind to the coupled cells): the cell's own opposite value plus the term
                // of one wall face (face 7: obstacle links), loaded with predicates so that the loads
                // of all links issue together
                const T* p0 = src + cidx;
                const float* w0 = wt + 19 * int((m0 >> 25) & 7u);
                const float* w1 = wt + 19 * int((m1 >> 25) & 7u);
#pragma unroll
                for (int q = 1; q < 19; q++) {
                    const bool b0 = (m0 >> q) & 1u, b1 = (m1 >> q) & 1u;
                    float lo = pred_ld(p0 + int64_t(dopp(q)) * n, b0, f2_lo(v[q]));
                    float hi = pred_ld(p0 + 1 + int64_t(dopp(q)) * n, b1, f2_hi(v[q]));
                    if (b0) lo += w0[q];
                    if (b1) hi += w1[q];
                    v[q] = f2_make(lo, hi);
                }
            }
            collide2(v, K, [&](f2 R, f2 jx, f2 jy, f2 jz) {
                if (l0) rec1(f2_lo(R), f2_lo(jx), f2_lo(jy), f2_lo(jz));
                if (l1) rec1(f2_hi(R), f2_hi(jx), f2_hi(jy), f2_hi(jz));
            });
            T* p = dst + cidx;
            if (l0 && l1) {
#pragma unroll
                for (int q = 0; q < 19; q++) {
                    store_pair<T>(p, v[q]);
                    p += n;
                }
            } else {
                if (l1) p += 1;
#pragma unroll
                for (int q = 0; q < 19; q++) {
                    Store<T>::st(p, l0 ? f2_lo(v[q]) : f2_hi(v[q]));
                    p += n;
                }
            }
        }
        if (++ck == ZC) {
            cch = ich;   // the issuing side's chunk (the one after this), or -1
            ck = 0;
        }
    }
    cp_async_wait<0>();
    if (want_tot) {
        // the warp's sum in FP32 (see walk_block)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            C t = tot[q][tid];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) a.totals[gw * 4 + q] = double(t);
        }
    }
    // the launch's last CTA to finish resets the chunk counter for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(a.wq + 1, 1) == ncta - 1) {
            atomicExch(a.wq, 0);
            atomicExch(a.wq + 1, 0);
            __threadfence();
        }
    }
}

// Coupled cells (owned fluid cells with a coalescence link, which the column walk skips), virtual
// CTA `v` of them: one thread per cell, plain pulls as in the walk, the marked links through the
// general path, then the collision.  The recording launch writes their moments, one entry per
// warp, after the walk's `walk_entries` entries.
template <typename T, typename C, int COLL, int LB>
__device__ __forceinline__ void coupled_block(const StepArgs& a, int64_t v, int64_t walk_entries, C (&slow)[19][256]) {
    constexpr int B = 1 << LB, M = B - 1, B2s = 2 * LB, B3s = 3 * LB;
    const T* src = static_cast<const T*>(a.lv.f[a.cur]);
    T* dst = static_cast<T*>(a.lv.f[a.cur ^ 1]);
    const int64_t n = a.lv.ncells;
    const Access<T, C> acc{a, LB, M};
    const int tid = threadIdx.x;
    const int j = int(v * 256 + tid);
    const bool want_tot = a.totals != nullptr;
    C mom[4] = {C(0), C(0), C(0), C(0)};
    if (j < a.lv.ncwork) {
        const int c = int(__ldg(a.lv.cwork + j));
        const int brick = c >> B3s, local = c & ((1 << B3s) - 1);
        const int x = local & M, y = (local >> LB) & M, z = local >> B2s;
        const uint32_t mq = __ldg(a.lv.link + c) & LINK_ALL;
        const int* nbr = a.lv.nbr + brick * 27;
        C vv[19];
        vv[0] = acc.load(src, n, 0, c);
#pragma unroll
        for (int q = 1; q < 19; q++) {
            vv[q] = C(0);
            if (!((mq >> q) & 1u)) {   // plain: the source holds the value (stored, in the grid)
                const int sx = x - dex(q), sy = y - dey(q), sz = z - dez(q);
                const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
                const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
                const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
                const int nb = (ox | oy | oz) ? __ldg(nbr + 13 + ox + 3 * oy + 9 * oz) : brick;
                const int sidx = (max(nb, 0) << B3s) + ((sz & M) << B2s) + ((sy & M) << LB) + (sx & M);
                vv[q] = acc.load(src, n, q, sidx);
            }
        }
        for (int q = 1; q < 19; q++)
            if ((mq >> q) & 1u) slow[q][tid] = pull_general<T, C, LB>(a, acc, brick, x, y, z, q, true);
#pragma unroll
        for (int q = 1; q < 19; q++)
            if ((mq >> q) & 1u) vv[q] = slow[q][tid];
        const LevelParams* P = a.params;
        const C fa[3] = {Par<C>::fa(P, 0), Par<C>::fa(P, 1), Par<C>::fa(P, 2)};
        collide<C, COLL>(vv, Par<C>::le(P), Par<C>::lo(P), fa, C(a.rho0), C(a.inv_rho0), a.two_u0,
                         [&](C R, C jx, C jy, C jz) {
                             mom[0] = R;
                             mom[1] = jx;
                             mom[2] = jy;
                             mom[3] = jz;
                         });
        T* p = dst + c;
#pragma unroll
        for (int q = 0; q < 19; q++) Store<T>::st(p + int64_t(q) * n, vv[q]);
    }
    if (want_tot) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            C t = mom[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if ((tid & 31) == 0) a.totals[(walk_entries + v * 8 + (tid >> 5)) * 4 + k] = double(t);
        }
    }
}

// Ghost layers 1-2, virtual CTA `v` of this sub-step's ghost work list: stream only, the directions
// the work entry needs; a source holding an exploded value is read from the coarse parent, and
// bounce-back/wall links take the general pull.
template <typename T, typename C, int LB>
__device__ __forceinline__ void ghost_block(const StepArgs& a, int64_t v, C (&slow)[19][256]) {
    constexpr int B = 1 << LB, M = B - 1, B2s = 2 * LB, B3s = 3 * LB;
    const int gs = a.substep - 1;
    const int tid = threadIdx.x;
    const int i = int(v * 256 + tid);
    if (i >= a.lv.ngwork[gs]) return;
    const T* src = static_cast<const T*>(a.lv.f[a.cur]);
    T* dst = static_cast<T*>(a.lv.f[a.cur ^ 1]);
    const int64_t n = a.lv.ncells;
    const Access<T, C> acc{a, LB, M};
    const uint4 e = __ldg(a.lv.gwork[gs] + i);
    const int c = int(e.x);
    const uint32_t need = e.y, cm = e.z, sm = e.w;
    const int brick = c >> B3s, local = c & ((1 << B3s) - 1);
    const int x = local & M, y = (local >> LB) & M, z = local >> B2s;
    const int* nbr = a.lv.nbr + brick * 27;
    C vv[19];
#pragma unroll
    for (int q = 1; q < 19; q++) {
        vv[q] = C(0);
        if (((need & ~sm) >> q) & 1u) {
            const int sx = x - dex(q), sy = y - dey(q), sz = z - dez(q);
            const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
            const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
            const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
            const int nb = (ox | oy | oz) ? __ldg(nbr + 13 + ox + 3 * oy + 9 * oz) : brick;
            if ((cm >> q) & 1u) {
                vv[q] = acc.coarse(nb, sx & M, sy & M, sz & M, q);
            } else {
                const int sidx = (max(nb, 0) << B3s) + ((sz & M) << B2s) + ((sy & M) << LB) + (sx & M);
                vv[q] = acc.load(src, n, q, sidx);
            }
        }
    }
    if (sm) {
        for (int q = 1; q < 19; q++)
            if ((sm >> q) & 1u) slow[q][tid] = pull_general<T, C, LB>(a, acc, brick, x, y, z, q, false);
#pragma unroll
        for (int q = 1; q < 19; q++)
            if ((sm >> q) & 1u) vv[q] = slow[q][tid];
    }
    T* p = dst + c;
#pragma unroll
    for (int q = 1; q < 19; q++)
        if ((need >> q) & 1u) Store<T>::st(p + int64_t(q) * n, vv[q]);
}

// The work of CTA `bid` of one launch of F_L(s) (see step_kernel); every thread of the CTA calls it.
//  - FP64 storage: the grid is [coupled cells' CTAs][column walk CTAs][ghost work CTAs]; the coupled
//    CTAs come first so that their longer dependent chains overlap the walk.
//  - FP32 / FP16 storage: the grid is the a.wctas persistent CTAs of the column walk; the coupled
//    cells and the ghost work run in side_kernel, launched before it.
template <typename T, typename C, int COLL, int LB, int MINB>
__device__ __forceinline__ void step_block(const StepArgs& a, int64_t bid, unsigned char* smem) {
    using SP = StepSmem<T, C, LB, MINB>;
    constexpr int B2s = 2 * LB;
    C(&slow)[19][256] = *reinterpret_cast<C(*)[19][256]>(smem + SP::OFF_SCRATCH);
    const int64_t coupled_ctas = (int64_t(a.lv.ncwork) + 255) >> 8;
    if constexpr (SP::CX == 2) {
        walk_packed<T, COLL, LB, MINB>(a, int(bid), a.wctas, smem);
    } else {
        const int upb = (1 << B2s) << (LB - a.lzc);   // units (column chunks) per brick
        const int64_t owned_units = int64_t(a.lv.nown) * upb;
        const int64_t owned_ctas = (owned_units + 255) >> 8;
        if (bid < coupled_ctas) {
            coupled_block<T, C, COLL, LB>(a, bid, owned_units >> 5, slow);
            return;
        }
        bid -= coupled_ctas;
        if (bid < owned_ctas) {
            walk_block<T, C, COLL, LB, MINB>(a, bid, smem);
            return;
        }
        ghost_block<T, C, LB>(a, bid - owned_ctas, slow);
    }
}

// The dynamic shared memory rounded up to 128 bytes (launches request StepSmem::BYTES + 128).
__device__ __forceinline__ unsigned char* align_smem(unsigned char* p) {
    const uint32_t off = (128u - (sh_addr(p) & 127u)) & 127u;
    return p + off;
}

template <typename T, typename C, int COLL, int LB, int MINB>
__global__ void __launch_bounds__(256, (StepSmem<T, C, LB, MINB>::kMinCtas)) step_kernel(const StepArgs a) {
    extern __shared__ __align__(128) unsigned char step_smem[];
    step_block<T, C, COLL, LB, MINB>(a, blockIdx.x, align_smem(step_smem));
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
__global__ void __launch_bounds__(256, (StepSmem<T, C, LB, MINB>::kMinCtas)) step_batch_kernel(const StepArgs* args, const int* prefix, int n,
                                                                                         int total) {
    extern __shared__ __align__(128) unsigned char step_smem[];
    __shared__ StepArgs sa;
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int64_t bid = batch_args(args, prefix, n, v, sa);
        step_block<T, C, COLL, LB, MINB>(sa, bid, align_smem(step_smem));
    }
}

// The coupled cells and the ghost work of one F_L(s) whose column walk is persistent (FP32 / FP16
// storage): virtual CTA v < coupled CTAs is coupled_block(v), the rest ghost_block.  The coupled
// cells' totals entries follow the walk's a.wctas * 8.
template <typename T, typename C, int COLL, int LB>
__device__ __forceinline__ void side_block(const StepArgs& a, int64_t v, C (&slow)[19][256]) {
    const int64_t coupled_ctas = (int64_t(a.lv.ncwork) + 255) >> 8;
    if (v < coupled_ctas) coupled_block<T, C, COLL, LB>(a, v, int64_t(a.wctas) * 8, slow);
    else ghost_block<T, C, LB>(a, v - coupled_ctas, slow);
}

template <typename T, typename C, int COLL, int LB>
__global__ void __launch_bounds__(256, 3) side_kernel(const StepArgs a) {
    __shared__ C slow[19][256];
    side_block<T, C, COLL, LB>(a, blockIdx.x, slow);
}

// side_kernel of a batch of forests in one persistent launch (virtual CTAs as in step_batch_kernel).
template <typename T, typename C, int COLL, int LB>
__global__ void __launch_bounds__(256) side_batch_kernel(const StepArgs* args, const int* prefix, int n, int total) {
    __shared__ C slow[19][256];
    __shared__ StepArgs sa;
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        const int64_t bid = batch_args(args, prefix, n, v, sa);
        side_block<T, C, COLL, LB>(sa, bid, slow);
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
    float two_u0[3];
    for (int k = 0; k < 3; k++) two_u0[k] = float(2.0 * lv.u0[k]);
    collide<C, COLL>(v, C(P->le), C(P->lo), fa, C(rho0), C(1.0 / rho0), two_u0, [](C, C, C, C) {});
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
