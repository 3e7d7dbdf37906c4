// Device kernels of the refined-grid D3Q19 LBM, templated on storage type T, compute type C
// and collision model.  Included by one translation unit per storage precision.
//
// Storage per level: two PDF grids (Sec. 4.1 two-grid approach), each [19][ncells] with the
// cells of brick k at [k * B^3, (k+1) * B^3), x fastest.  The grids hold the POST-COLLISION
// state of owned cells (f-tilde, stored by the fused kernel) and the streamed values of ghost
// layers 1-2.  FP32/FP16 storage holds f - w rho0 ("shifted"); FP64 holds f.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

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

// ------------------------------------------------------------------ collision (Sec. 2, 2.1)
// v holds f (or f - w rho0 when shifted) on entry and f-tilde on exit.  R is rho (or rho - rho0).
// SRT: f~ = f - omega (f - f^eq) + F;  TRT: f~ = f - le (f+ - f^eq+) - lo (f- - f^eq-) + F, with
// f^eq of Eq. (fequ) and F_a = 3 w_a rho0 e_a . a (Sec. 2.1); the velocity inside f^eq is
// sum_a e_a f_a / rho0, unmodified by the force.
template <typename C, int COLL>
__device__ __forceinline__ void collide(C (&v)[19], C le, C lo, const C (&F)[19], C rho0, C inv_rho0) {
    C R = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
    for (int q = 0; q < 19; q++) {
        R += v[q];
        if (dex(q)) jx += dex(q) > 0 ? v[q] : -v[q];
        if (dey(q)) jy += dey(q) > 0 ? v[q] : -v[q];
        if (dez(q)) jz += dez(q) > 0 ? v[q] : -v[q];
    }
    const C ux = jx * inv_rho0, uy = jy * inv_rho0, uz = jz * inv_rho0;
    const C usq = ux * ux + uy * uy + uz * uz;
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
        const C w = C(dw(q));
        const C eqp = w * (R + rho0 * (C(4.5) * eu * eu) - base);
        const C eqm = w * rho0 * C(3.0) * eu;
        if (COLL == LBM_TRT) {
            const C fp = C(0.5) * (v[q] + v[p]);
            const C fm = C(0.5) * (v[q] - v[p]);
            const C dp = le * (fp - eqp);
            const C dm = lo * (fm - eqm);
            const C a = v[q] - dp - dm + F[q];
            const C b = v[p] - dp + dm + F[p];
            v[q] = a;
            v[p] = b;
        } else {
            const C a = v[q] - le * (v[q] - (eqp + eqm)) + F[q];
            const C b = v[p] - le * (v[p] - (eqp - eqm)) + F[p];
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
    // Value of the coarse parent of cell (x, y, z) of ghost brick g (explosion, Eq. ctof).
    __device__ __forceinline__ C coarse(int g, int x, int y, int z, int q) const {
        const int pk = __ldg(a.lv.parent + g);
        if (pk < 0) return qnan<C>();
        const int pb = pk >> 3, oct = pk & 7;
        const int B = 1 << LB;
        const int px = ((oct & 1) * B + x) >> 1, py = (((oct >> 1) & 1) * B + y) >> 1, pz = ((oct >> 2) * B + z) >> 1;
        const int64_t idx = (int64_t(pb) << (3 * LB)) + (pz << (2 * LB)) + (py << LB) + px;
        return load(a.co.f[a.cur_c], a.co.ncells, q, idx);
    }
    // Mean of the 8 finer children of owned cell (x, y, z) of brick b after both fine sub-steps
    // (coalescence, Eq. ftoc), summed pairwise in FP64 in z-y-x bit order.
    __device__ __forceinline__ C children_mean(int b, int x, int y, int z, int q) const {
        const int oct = ((2 * x) >> LB) | (((2 * y) >> LB) << 1) | (((2 * z) >> LB) << 2);
        const int cb = __ldg(a.lv.child + b * 8 + oct);
        if (cb < 0) return qnan<C>();
        const int cx = (2 * x) & M, cy = (2 * y) & M, cz = (2 * z) & M;
        const int64_t base = (int64_t(cb) << (3 * LB)) + (cz << (2 * LB)) + (cy << LB) + cx;
        const int sy = 1 << LB, sz = 1 << (2 * LB);
        const void* f = a.fi.f[a.cur_f];
        const int64_t n = a.fi.ncells;
        double c0 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base));
        double c1 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + 1));
        double c2 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + sy));
        double c3 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + sy + 1));
        double c4 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + sz));
        double c5 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + sz + 1));
        double c6 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + sz + sy));
        double c7 = double(Store<T>::ld(static_cast<const T*>(f) + int64_t(q) * n + base + sz + sy + 1));
        const double s = ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7));
        return C(s * 0.125);
    }
};

// One sub-step of one level: stream (pull) + boundary + explosion reads + coalescence, then
// collide owned cells (Alg. 2 StreamCollide generalised to every level).  CTAs [0, nown * B^3/256)
// cover owned bricks; the rest cover the ghost-layer-1/2 work list.
template <typename T, typename C, int COLL>
__global__ void __launch_bounds__(256) step_kernel(const StepArgs a) {
    const int LB = a.LB, B = 1 << LB, M = B - 1, B3s = 3 * LB;
    const int cpb = (1 << B3s) >> 8;
    const int owned_ctas = a.lv.nown * cpb;
    int brick, local;
    bool ghost;
    if (int(blockIdx.x) < owned_ctas) {
        brick = blockIdx.x / cpb;
        local = (blockIdx.x - brick * cpb) * 256 + threadIdx.x;
        ghost = false;
    } else {
        const int i = (blockIdx.x - owned_ctas) * 256 + threadIdx.x;
        if (i >= a.lv.ngcells) return;
        const int c = __ldg(a.lv.gcells + i);
        brick = c >> B3s;
        local = c & ((1 << B3s) - 1);
        ghost = true;
    }
    const int64_t cidx = (int64_t(brick) << B3s) + local;
    const uint8_t bk = __ldg(a.lv.kind + brick);
    if (!ghost && !(bk & BK_PURE) && __ldg(a.lv.cell + cidx) != CK_FLUID) return;
    const int lx = local & M, ly = (local >> LB) & M, lz = local >> (2 * LB);
    const void* src = a.lv.f[a.cur];
    const int64_t n = a.lv.ncells;
    const Access<T, C> acc{a, LB, M};
    // in the first sub-step the ghost layers hold the exploded coarse values (Eq. ctof)
    const bool exploded_self = ghost && a.substep == 1;
    const bool touch_finer = !ghost && (bk & BK_TOUCH_FINER);
    const int* nbr = a.lv.nbr + brick * 27;

    C v[19];
    v[0] = exploded_self ? acc.coarse(brick, lx, ly, lz, 0) : acc.load(src, n, 0, cidx);
#pragma unroll
    for (int q = 1; q < 19; q++) {
        const int ex = dex(q), ey = dey(q), ez = dez(q);
        const int sx = lx - ex, sy = ly - ey, sz = lz - ez;
        const int ox = sx < 0 ? -1 : (sx > M ? 1 : 0);
        const int oy = sy < 0 ? -1 : (sy > M ? 1 : 0);
        const int oz = sz < 0 ? -1 : (sz > M ? 1 : 0);
        const int nb = (ox | oy | oz) ? __ldg(nbr + 13 + ox + 3 * oy + 9 * oz) : brick;
        // coalescence: the PDF enters x from the finer level when the upwind cell along e_q, or
        // along one axis component of e_q, lies in the finer level (fine-to-coarse, Sec. 4.4)
        bool coal = false;
        if (touch_finer) {
            coal = nb == NB_FINER;
            if (!coal && ex && ox) coal = __ldg(nbr + 13 + ox) == NB_FINER;
            if (!coal && ey && oy) coal = __ldg(nbr + 13 + 3 * oy) == NB_FINER;
            if (!coal && ez && oz) coal = __ldg(nbr + 13 + 9 * oz) == NB_FINER;
        }
        C val;
        if (coal) {
            val = acc.children_mean(brick, lx, ly, lz, q);
        } else if (nb >= 0) {
            const int tx = sx & M, ty = sy & M, tz = sz & M;
            const int64_t sidx = (int64_t(nb) << B3s) + (tz << (2 * LB)) + (ty << LB) + tx;
            if (__ldg(a.lv.kind + nb) & BK_PURE) {
                val = acc.load(src, n, q, sidx);
            } else {
                const uint8_t ck = __ldg(a.lv.cell + sidx);
                if (ck == CK_SOLID) {
                    // no-slip bounce-back, pre-stream boundary treatment (Sec. 2.2)
                    val = exploded_self ? acc.coarse(brick, lx, ly, lz, dopp(q)) : acc.load(src, n, dopp(q), cidx);
                } else if (ck == CK_FLUID || (ck == CK_GHOST && a.substep == 2)) {
                    val = acc.load(src, n, q, sidx);
                } else {
                    val = acc.coarse(nb, tx, ty, tz, q);
                }
            }
        } else if (nb == NB_WALL) {
            // domain wall: bounce-back, plus 6 w rho0 e.u_w on velocity walls; a cell beyond
            // several faces takes the first of z+, z-, y+, y-, x+, x-
            const int* P = a.lv.pos + 3 * brick;
            const int gx = P[0] * B + sx, gy = P[1] * B + sy, gz = P[2] * B + sz;
            int face;
            if (!(a.per & 4) && gz >= a.lv.N[2]) face = 5;
            else if (!(a.per & 4) && gz < 0) face = 4;
            else if (!(a.per & 2) && gy >= a.lv.N[1]) face = 3;
            else if (!(a.per & 2) && gy < 0) face = 2;
            else if (!(a.per & 1) && gx >= a.lv.N[0]) face = 1;
            else face = 0;
            const C own = exploded_self ? acc.coarse(brick, lx, ly, lz, dopp(q)) : acc.load(src, n, dopp(q), cidx);
            val = own + C(a.wall[face * 19 + q]);
        } else {
            val = qnan<C>();
        }
        v[q] = val;
    }
    void* dstv = a.lv.f[a.cur ^ 1];
    T* dst = static_cast<T*>(dstv);
    if (!ghost) {
        const LevelParams* P = a.params;
        C F[19];
#pragma unroll
        for (int q = 0; q < 19; q++) F[q] = C(P->force[q]);
        collide<C, COLL>(v, C(P->le), C(P->lo), F, C(a.rho0), C(1.0 / a.rho0));
    }
#pragma unroll
    for (int q = 0; q < 19; q++) Store<T>::st(dst + int64_t(q) * n + cidx, v[q]);
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
        const double R = Store<T>::shifted ? r - rho0 : r;
        v[q] = C(dw(q) * (R + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq)));
    }
    C F[19];
#pragma unroll
    for (int q = 0; q < 19; q++) F[q] = C(P->force[q]);
    collide<C, COLL>(v, C(P->le), C(P->lo), F, C(rho0), C(1.0 / rho0));
#pragma unroll
    for (int q = 0; q < 19; q++) {
        Store<T>::st(f + q * lv.ncells + i, v[q]);
        Store<T>::st(g + q * lv.ncells + i, qnan<C>());
    }
}

// rho and u (+ a/2) of owned cells from the stored post-collision state: collision keeps rho and
// adds rho0 a to the momentum, so u_out = j~/rho0 - a/2 (Sec. 2.1).
template <typename T>
__global__ void macro_kernel(const DevLevel lv, int cur, int LB, const LevelParams* P, double rho0, double* rho,
                             double* u) {
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nown_cells) return;
    if (lv.cell[i] != CK_FLUID) {
        if (rho) rho[i] = __longlong_as_double(0x7ff8000000000000ULL);
        if (u) u[i] = u[nown_cells + i] = u[2 * nown_cells + i] = __longlong_as_double(0x7ff8000000000000ULL);
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
    if (u) {
        u[i] = jx / rho0 - 0.5 * P->acc[0];
        u[nown_cells + i] = jy / rho0 - 0.5 * P->acc[1];
        u[2 * nown_cells + i] = jz / rho0 - 0.5 * P->acc[2];
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
        out[q * nown_cells + i] = Store<T>::shifted ? v + dw(q) * rho0 : v;
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
        if (i < nown_cells && lv.cell[i] == CK_FLUID) v = Store<T>::shifted ? in[q * nown_cells + i] - dw(q) * rho0 : in[q * nown_cells + i];
        Store<T>::st_d(f + q * lv.ncells + i, v);
    }
}

// Per-CTA FP64 partial totals of one level: {w rho, w (j~ - rho0 a)} over owned fluid cells, with
// w = 8^-L.  partial[blockIdx][4]; summed in a fixed order by reduce_final_kernel.
template <typename T>
__global__ void __launch_bounds__(256) reduce_level_kernel(const DevLevel lv, int cur, int LB, const LevelParams* P,
                                                          double rho0, double w, double* partial) {
    const int64_t nown_cells = int64_t(lv.nown) << (3 * LB);
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const T* f = static_cast<const T*>(lv.f[cur]);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nown_cells; i += int64_t(gridDim.x) * blockDim.x) {
        if (lv.cell[i] != CK_FLUID) continue;
        double R = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int q = 0; q < 19; q++) {
            const double v = double(Store<T>::ld(f + q * lv.ncells + i));
            R += v;
            jx += dex(q) * v;
            jy += dey(q) * v;
            jz += dez(q) * v;
        }
        s[0] += w * (Store<T>::shifted ? rho0 + R : R);
        s[1] += w * (jx - rho0 * P->acc[0]);
        s[2] += w * (jy - rho0 * P->acc[1]);
        s[3] += w * (jz - rho0 * P->acc[2]);
    }
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
