// Learned warm start: a 3-D convolutional net that maps the coarse-only solution, upsampled onto a
// refined block (plus a halo), to the refined solution there.  The net's output initialises the
// refined levels with f = f^eq(rho, u) (Eq. fequ); the LBM then runs unmodified.
//
// Net: L layers of 3x3x3 convolutions (zero padding, stride 1), width 16, ReLU between layers,
// none after the last.  Tensors are channels-last volumes of 16 BF16 channels (32 bytes per
// voxel), `nvol` volumes of D x H x W voxels stored one after another, x fastest.  Products
// run on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulate).  Weights are kept
// in FP32 (master copy, Adam moments) and rounded to BF16 for the products.
//
//   forward   Z_l = b_l + sum_o W_l[o] X_l[v + o]          X_{l+1} = relu(Z_l)
//   backward  dW_l[o] += sum_v dZ_l[v] (x) X_l[v + o]      db_l = sum_v dZ_l[v]
//             dX_l[v] = sum_o W_l[o]^T dZ_l[v - o]         dZ_{l-1} = dX_l * [X_l > 0]
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "devmem.h"
#include "lbm_internal.h"

namespace {

constexpr int CH = 16;       // channels of every tensor (unused channels are zero)
constexpr int TAPS = 27;     // 3x3x3 offsets, o = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)

struct Dims {
    int D, H, W;   // voxels per volume along z, y, x
    int nvol;      // volumes
    long long V;   // voxels per volume
    long long N;   // all voxels
};

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Linear index of voxel v shifted by tap o, or -1 outside its volume (zero padding).
__device__ __forceinline__ long long shifted(const Dims& d, long long v, int o) {
    if (v >= d.N) return -1;
    const long long vol = v / d.V;
    long long r = v - vol * d.V;
    const int x = int(r % d.W);
    r /= d.W;
    const int y = int(r % d.H), z = int(r / d.H);
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int sx = x + dx, sy = y + dy, sz = z + dz;
    if (sx < 0 || sx >= d.W || sy < 0 || sy >= d.H || sz < 0 || sz >= d.D) return -1;
    return vol * d.V + ((long long)(sz) * d.H + sy) * d.W + sx;
}

// Z[v][n] = bias[n] + sum_o sum_k Wt[o][n][k] X[v + o][k] over 16 voxels per warp; then
// optionally relu (act = 1) or multiplication by [mask > 0] (act = 2, the ReLU derivative of the
// layer whose output `mask` is).  Wt is BF16 [27][16 out][16 in].
__global__ void __launch_bounds__(256) conv_kernel(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wt,
                                                   const float* __restrict__ bias, __nv_bfloat16* __restrict__ Z, Dims d,
                                                   int act, const __nv_bfloat16* __restrict__ mask) {
    __shared__ uint32_t sw[TAPS * CH * CH / 2];
    for (int i = threadIdx.x; i < TAPS * CH * CH / 2; i += blockDim.x) sw[i] = reinterpret_cast<const uint32_t*>(Wt)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long v0 = ((long long)(blockIdx.x) * 8 + (threadIdx.x >> 5)) * 16;
    if (v0 >= d.N) return;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const uint32_t* X32 = reinterpret_cast<const uint32_t*>(X);
    for (int o = 0; o < TAPS; o++) {
        const long long r0 = shifted(d, v0 + g, o), r1 = shifted(d, v0 + g + 8, o);
        uint32_t a[4];
        a[0] = r0 >= 0 ? __ldg(X32 + r0 * (CH / 2) + t) : 0u;
        a[1] = r1 >= 0 ? __ldg(X32 + r1 * (CH / 2) + t) : 0u;
        a[2] = r0 >= 0 ? __ldg(X32 + r0 * (CH / 2) + t + 4) : 0u;
        a[3] = r1 >= 0 ? __ldg(X32 + r1 * (CH / 2) + t + 4) : 0u;
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const int n = nt * 8 + g;
            const uint32_t b0 = sw[(o * CH + n) * (CH / 2) + t], b1 = sw[(o * CH + n) * (CH / 2) + t + 4];
            mma16816(acc[nt], a, b0, b1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const long long v = v0 + g + 8 * h;
            if (v >= d.N) continue;
            const int n = nt * 8 + 2 * t;
            float z0 = acc[nt][2 * h] + (bias ? bias[n] : 0.f), z1 = acc[nt][2 * h + 1] + (bias ? bias[n + 1] : 0.f);
            if (act == 1) {
                z0 = fmaxf(z0, 0.f);
                z1 = fmaxf(z1, 0.f);
            } else if (act == 2) {
                const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(mask)[v * (CH / 2) + n / 2];
                if (!(__bfloat162float(m.x) > 0.f)) z0 = 0.f;
                if (!(__bfloat162float(m.y) > 0.f)) z1 = 0.f;
            }
            reinterpret_cast<__nv_bfloat162*>(Z)[v * (CH / 2) + n / 2] = __floats2bfloat162_rn(z0, z1);
        }
}

// ---------------------------------------------------------------- tcgen05 convolution
// The same product as conv_kernel on the 5th-generation tensor cores.  One CTA (4 warps) walks
// (volume, z-plane) units.  For a unit it stages the input planes z-1, z, z+1 in shared memory as
// zero-padded (H + 2) x P slots (P = W + 2), in two halves of 8 channels: half c of slot s at
// byte 16 (c NSL + s) of its plane.  In this K-major, unswizzled layout the A operand of tap
// (dx, dy, dz) for 128 consecutive output slots s0.. is the same window shifted by dy P + dx slots
// in plane dz + 1, so each tap is one M128 N16 K16 BF16 MMA (tcgen05.mma kind::f16, FP32
// accumulator in TMEM) whose descriptor differs only in its start address; 27 of them accumulate
// a tile.  One thread issues them and commits to an mbarrier; the 4 warps then read their 32 TMEM
// lanes (tcgen05.ld 32x32b.x16: one output slot's 16 channels per thread), keep interior slots,
// and apply bias and activation as conv_kernel does.
constexpr int TC_W_BYTES = TAPS * 2 * CH * 8 * 2;   // weights [tap][half][n][8] BF16
constexpr int TC_A_OFF = 14336;                     // after the weights, barrier and TMEM slot
constexpr int TC_BAR_OFF = TC_W_BYTES;
constexpr int TC_TM_OFF = TC_W_BYTES + 8;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start address, leading byte offset (K direction), stride byte offset (M/N direction), all in
    // 16-byte units; bit 46: descriptor version of tcgen05; no swizzle, base offset 0
    return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

__global__ void __launch_bounds__(128) conv_tc_kernel(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Wt,
                                                      const float* __restrict__ bias, __nv_bfloat16* __restrict__ Z, Dims d,
                                                      int act, const __nv_bfloat16* __restrict__ mask, int P, int NSL,
                                                      int ntile, int tmcols, int* __restrict__ err, int wait_test) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(sm));
    const uint32_t bar = base + TC_BAR_OFF, wbase = base, abase = base + TC_A_OFF;
    // weights: Wt[o][n][k] -> [o][k / 8][n][k % 8]
    for (int i = tid; i < TAPS * CH * CH; i += blockDim.x) {
        const int o = i / (CH * CH), n = (i / CH) % CH, k = i % CH;
        reinterpret_cast<__nv_bfloat16*>(sm)[((o * 2 + k / 8) * CH + n) * 8 + k % 8] = Wt[i];
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(base + TC_TM_OFF), "r"(tmcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + TC_TM_OFF);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
    const int H = d.H, W = d.W, D = d.D;
    // the padding slots (plane borders and the tail beyond the plane) are zero for every unit:
    // fill them once; each unit then copies only the interior rows
    for (int i = tid; i < 6 * NSL; i += blockDim.x) *reinterpret_cast<uint4*>(sm + TC_A_OFF + i * 16) = make_uint4(0u, 0u, 0u, 0u);
    // this thread's place in the interior row copies: chunk xc of rows r0, r0 + rpp, ...
    const int cpr = 2 * W, rpp = blockDim.x / cpr;
    const int r0 = tid / cpr, xc = tid - (tid / cpr) * cpr;
    const bool copier = r0 < rpp;
    uint32_t phase = 0;
    for (long long unit = blockIdx.x; unit < (long long)d.nvol * D; unit += gridDim.x) {
        const long long vol = unit / D;
        const int z = int(unit - vol * D);
        // stage the interiors of the three input planes with asynchronous 16-byte copies; a plane
        // outside the volume is zero (a zero source size writes zeros without reading)
        if (copier)
            for (int p = 0; p < 3; p++) {
                const int zz = z + p - 1;
                const bool pv = zz >= 0 && zz < D;
                const long long row0 = (vol * D + (pv ? zz : 0)) * H;
                for (int y = r0; y < H; y += rpp) {
                    const int x = xc >> 1, c = xc & 1;
                    const int slot = (y + 1) * P + x + 1;
                    const void* src = reinterpret_cast<const uint4*>(X + ((row0 + y) * W + x) * CH) + c;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(abase + uint32_t(((p * 2 + c) * NSL + slot) * 16)),
                                 "l"(src), "r"(pv ? 16 : 0)
                                 : "memory");
                }
            }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && !wait_test) {
            // descriptors differ only in their start address (bits 0-13, 16-byte units): the tap
            // (dx, dy, dz) of tile t starts (dz + 1) 2 NSL + dy P + dx slots after the tile's slot
            const uint64_t a0 = smem_desc(abase, uint32_t(NSL * 16), 128u);
            const uint64_t b0 = smem_desc(wbase, uint32_t(CH * 16), 128u);
            for (int t = 0; t < ntile; t++) {
                const uint64_t at = a0 + uint64_t(P + 1 + 128 * t);
                int o = 0;
#pragma unroll
                for (int dz = 0; dz < 3; dz++)
#pragma unroll
                    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                        for (int dx = -1; dx <= 1; dx++, o++) {
                            const uint64_t ad = at + uint64_t(dz * 2 * NSL + dy * P + dx);
                            const uint64_t bd = b0 + uint64_t(o * 2 * CH * 8 * 2 / 16);
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + uint32_t(t * 16)),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(o));
                        }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
        }
        // bounded wait for this unit's products (the wait test issues none and gives up after a
        // short wait: nothing asynchronous is outstanding when the CTA then releases its TMEM)
        uint32_t done = 0;
        const int limit = wait_test ? (1 << 10) : (1 << 24);
        for (int it = 0; it < limit && !done; it++)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done) : "r"(bar), "r"(phase) : "memory");
        phase ^= 1u;
        if (__syncthreads_or(!done)) {
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int t = 0; t < ntile; t++) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tmem + (uint32_t(warp * 32) << 16) + uint32_t(t * 16)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int s = P + 1 + 128 * t + warp * 32 + lane;
            const int y = s / P, x = s - (s / P) * P;
            if (y < 1 || y > H || x < 1 || x > W) continue;
            const long long v = ((vol * D + z) * H + (y - 1)) * W + (x - 1);
            __nv_bfloat162 o2[8];
#pragma unroll
            for (int c = 0; c < 8; c++) {
                float z0 = __uint_as_float(r[2 * c]) + (bias ? bias[2 * c] : 0.f);
                float z1 = __uint_as_float(r[2 * c + 1]) + (bias ? bias[2 * c + 1] : 0.f);
                if (act == 1) {
                    z0 = fmaxf(z0, 0.f);
                    z1 = fmaxf(z1, 0.f);
                } else if (act == 2) {
                    const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(mask)[v * (CH / 2) + c];
                    if (!(__bfloat162float(m.x) > 0.f)) z0 = 0.f;
                    if (!(__bfloat162float(m.y) > 0.f)) z1 = 0.f;
                }
                o2[c] = __floats2bfloat162_rn(z0, z1);
            }
            uint4* dst = reinterpret_cast<uint4*>(Z + v * CH);
            dst[0] = *reinterpret_cast<uint4*>(&o2[0]);
            dst[1] = *reinterpret_cast<uint4*>(&o2[4]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmcols) : "memory");
}

// dW[o][m][n] += sum_v dZ[v][m] X[v + o][n] and db[m] += sum_v dZ[v][m].  Block (chunk, o): 8 warps,
// each over its share of the chunk's voxels in steps of 16; partial sums are added with atomics.
__global__ void __launch_bounds__(256) wgrad_kernel(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ dZ,
                                                    float* __restrict__ dW, float* __restrict__ db, Dims d, long long chunk) {
    const int o = blockIdx.y;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
    const long long begin = (long long)(blockIdx.x) * chunk, end = begin + chunk < d.N ? begin + chunk : d.N;
    const unsigned short* Xs = reinterpret_cast<const unsigned short*>(X);
    const unsigned short* Ds = reinterpret_cast<const unsigned short*>(dZ);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    float bsum = 0.f;
    for (long long v0 = begin + warp * 16; v0 < end; v0 += 8 * 16) {
        // A[m][k] = dZ[v0 + k][m]; B[k][n] = X[v0 + k + o][n]
        auto dz = [&](int k, int m) -> uint32_t {
            const long long v = v0 + k;
            return v < end ? uint32_t(__ldg(Ds + v * CH + m)) : 0u;
        };
        auto xs = [&](int k, int n) -> uint32_t {
            const long long v = v0 + k;
            if (v >= end) return 0u;
            const long long r = shifted(d, v, o);
            return r >= 0 ? uint32_t(__ldg(Xs + r * CH + n)) : 0u;
        };
        uint32_t a[4];
        a[0] = dz(2 * t, g) | (dz(2 * t + 1, g) << 16);
        a[1] = dz(2 * t, g + 8) | (dz(2 * t + 1, g + 8) << 16);
        a[2] = dz(2 * t + 8, g) | (dz(2 * t + 9, g) << 16);
        a[3] = dz(2 * t + 8, g + 8) | (dz(2 * t + 9, g + 8) << 16);
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const int n = nt * 8 + g;
            const uint32_t b0 = xs(2 * t, n) | (xs(2 * t + 1, n) << 16);
            const uint32_t b1 = xs(2 * t + 8, n) | (xs(2 * t + 9, n) << 16);
            mma16816(acc[nt], a, b0, b1);
        }
        if (o == 13 && lane < 16)
            for (int k = 0; k < 16; k++) {
                const long long v = v0 + k;
                if (v < end) bsum += __bfloat162float(__ushort_as_bfloat16(__ldg(Ds + v * CH + lane)));
            }
    }
    __shared__ float red[8][CH * CH];
    __shared__ float bred[8][CH];
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int m = g + 8 * h, n = nt * 8 + 2 * t;
            red[warp][m * CH + n] = acc[nt][2 * h];
            red[warp][m * CH + n + 1] = acc[nt][2 * h + 1];
        }
    if (lane < 16) bred[warp][lane] = bsum;
    __syncthreads();
    for (int i = threadIdx.x; i < CH * CH; i += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < 8; w++) s += red[w][i];
        atomicAdd(dW + o * CH * CH + i, s);
    }
    if (o == 13 && threadIdx.x < CH) {
        float s = 0.f;
        for (int w = 0; w < 8; w++) s += bred[w][threadIdx.x];
        atomicAdd(db + threadIdx.x, s);
    }
}

// Master FP32 weights [27][16 out][16 in] -> BF16 copies for the forward product and, flipped and
// transposed, for the backward data product: Wb[o'][k][m] = W[26 - o'][m][k].
__global__ void weights_kernel(const float* __restrict__ W, __nv_bfloat16* __restrict__ Wf, __nv_bfloat16* __restrict__ Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TAPS * CH * CH) return;
    const int o = i / (CH * CH), m = (i / CH) % CH, k = i % CH;
    const __nv_bfloat16 w = __float2bfloat16_rn(W[i]);
    Wf[i] = w;
    Wb[((TAPS - 1 - o) * CH + k) * CH + m] = w;
}

// Adam (Kingma & Ba 2015) with bias correction, on n parameters.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                            int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gr = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gr, vi = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Prediction = skip + Z (first `nout` channels) over the voxels `weight` marks; squared error
// against the target, summed in FP64; dZ = 2 weight (pred - target) / count as BF16 (other
// channels 0).  pred (FP32 [N][nout]) may be NULL.
__global__ void __launch_bounds__(256) loss_kernel(const __nv_bfloat16* __restrict__ Z, const float* __restrict__ skip,
                                                   const float* __restrict__ target, const float* __restrict__ weight,
                                                   long long N, int nout, float inv_count, __nv_bfloat16* __restrict__ dZ,
                                                   float* __restrict__ pred, double* __restrict__ loss) {
    const long long v = (long long)(blockIdx.x) * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (v < N) {
        const float w = weight ? weight[v] : 1.f;
        for (int c = 0; c < CH; c++) {
            float g = 0.f;
            if (c < nout) {
                const float p = __bfloat162float(Z[v * CH + c]) + (skip ? skip[v * nout + c] : 0.f);
                if (pred) pred[v * nout + c] = p;
                if (target) {
                    const float e = p - target[v * nout + c];
                    s += double(w) * double(e) * double(e);
                    g = 2.f * w * e * inv_count;
                }
            }
            if (dZ) dZ[v * CH + c] = __float2bfloat16_rn(g);
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (int(threadIdx.x) < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0]);
}

// ---------------------------------------------------------------- host side

lbm_status nfail(lbm_status s, const char* msg) {
    lbm::set_last_error(msg);
    return s;
}

#define NCU(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            char b_[256];                                                              \
            snprintf(b_, sizeof b_, "%s failed: %s", #call, cudaGetErrorString(e_));   \
            return nfail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, b_); \
        }                                                                              \
    } while (0)

// SplitMix64 (Steele, Lea & Flood 2014), for the weight initialisation.
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

struct lbm_net {
    int layers = 0, cin = 0, cout = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;   // per layer: W [27][16][16], b [16]
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    __nv_bfloat16* wf = nullptr;   // per layer: forward BF16 weights
    __nv_bfloat16* wb = nullptr;   // per layer: backward-data BF16 weights
    int64_t step = 0;
    // activations of the last forward pass: X_0 .. X_{L-1}, Z_{L-1}; and two gradient buffers
    std::vector<__nv_bfloat16*> act;
    __nv_bfloat16* g0 = nullptr;
    __nv_bfloat16* g1 = nullptr;
    long long cap = 0;       // voxels the activation buffers hold
    double* d_loss = nullptr;
    double* h_loss = nullptr;
    int* d_err = nullptr;    // set by the tcgen05 kernel if a wait ran out
    int backend = 1;         // 1: tcgen05 products where the volume fits, 0: mma.sync only
    int wait_test = 0;       // 1: the tcgen05 kernel issues no products, so its bounded wait runs out
    int sms = 0;
    Dims d{};
    lbm::DevMem mem;         // device memory: the caller's allocator hook or cudaMalloc
};

namespace {

constexpr int PER_LAYER = TAPS * CH * CH + CH;

void free_acts(lbm_net* n) {
    for (auto* p : n->act) n->mem.put(p);
    n->act.clear();
    n->mem.put(n->g0);
    n->mem.put(n->g1);
    n->g0 = n->g1 = nullptr;
    n->cap = 0;
}

lbm_status ensure_acts(lbm_net* n, long long N) {
    if (n->cap >= N) return LBM_OK;
    free_acts(n);
    const size_t bytes = size_t(N) * CH * sizeof(__nv_bfloat16);
    for (int l = 0; l <= n->layers; l++) {
        __nv_bfloat16* p = nullptr;
        if (!n->mem.get(&p, bytes)) return nfail(LBM_ENOMEM, "cannot allocate the activations");
        n->act.push_back(p);
    }
    if (!n->mem.get(&n->g0, bytes) || !n->mem.get(&n->g1, bytes))
        return nfail(LBM_ENOMEM, "cannot allocate the activation gradients");
    n->cap = N;
    return LBM_OK;
}

// Shared-memory and TMEM geometry of conv_tc_kernel for a volume; false if it does not fit.
struct TcGeom {
    int P, NSL, ntile, tmcols, per_sm;
    size_t smem;
};

bool tc_geometry(const Dims& d, TcGeom& g) {
    g.P = d.W + 2;
    g.NSL = (((d.H + 2) * g.P + 160) + 7) & ~7;
    g.ntile = (d.H * g.P + 127) / 128;
    g.tmcols = 32;
    while (g.tmcols < g.ntile * 16) g.tmcols *= 2;
    g.smem = size_t(TC_A_OFF) + size_t(6) * g.NSL * 16;
    if (g.tmcols > 512 || g.smem > 227 * 1024) return false;
    g.per_sm = int(std::min<size_t>(std::min<size_t>(228 * 1024 / (g.smem + 1024), 512 / g.tmcols), 16));
    return g.per_sm >= 1;
}

// Z = conv(X) (+ bias, activation) with the tensor-core kernel the net is set to use.
lbm_status conv(lbm_net* n, const __nv_bfloat16* X, const __nv_bfloat16* Wt, const float* bias, __nv_bfloat16* Z,
                const Dims& d, int act, const __nv_bfloat16* mask) {
    TcGeom g;
    if (n->backend == 1 && tc_geometry(d, g)) {
        static size_t attr_smem = 0;
        if (g.smem > attr_smem) {
            NCU(cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(g.smem)));
            attr_smem = g.smem;
        }
        const long long units = (long long)d.nvol * d.D;
        const int grid = int(std::min<long long>(units, (long long)n->sms * g.per_sm));
        conv_tc_kernel<<<grid, 128, g.smem, n->stream>>>(X, Wt, bias, Z, d, act, mask, g.P, g.NSL, g.ntile, g.tmcols,
                                                        n->d_err, n->wait_test);
    } else {
        conv_kernel<<<int((d.N + 127) / 128), 256, 0, n->stream>>>(X, Wt, bias, Z, d, act, mask);
    }
    NCU(cudaGetLastError());
    return LBM_OK;
}

// LBM_ETIMEOUT if a tcgen05 wait ran out since the last check (synchronises the stream).
lbm_status check_err(lbm_net* n) {
    int e = 0;
    NCU(cudaMemcpyAsync(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NCU(cudaStreamSynchronize(n->stream));
    if (e) {
        NCU(cudaMemset(n->d_err, 0, sizeof(int)));
        return nfail(LBM_ETIMEOUT, "a tensor-core wait ran out; the outputs of this call are incomplete");
    }
    return LBM_OK;
}

lbm_status refresh_weights(lbm_net* n) {
    for (int l = 0; l < n->layers; l++)
        weights_kernel<<<(TAPS * CH * CH + 255) / 256, 256, 0, n->stream>>>(
            n->params + size_t(l) * PER_LAYER, n->wf + size_t(l) * TAPS * CH * CH, n->wb + size_t(l) * TAPS * CH * CH);
    NCU(cudaGetLastError());
    return LBM_OK;
}

lbm_status check_dims(int D, int H, int W, int nvol, Dims& d) {
    if (D < 1 || H < 1 || W < 1 || nvol < 1) return nfail(LBM_EINVAL, "volume dimensions must be positive");
    d.D = D;
    d.H = H;
    d.W = W;
    d.nvol = nvol;
    d.V = (long long)D * H * W;
    d.N = d.V * nvol;
    if (d.N > (1LL << 40)) return nfail(LBM_EINVAL, "too many voxels");
    return LBM_OK;
}

// Forward pass over x (BF16 [N][16]); keeps every layer's input for the backward pass.
lbm_status forward(lbm_net* n, const __nv_bfloat16* x, const Dims& d) {
    lbm_status s = ensure_acts(n, d.N);
    if (s) return s;
    NCU(cudaMemcpyAsync(n->act[0], x, size_t(d.N) * CH * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, n->stream));
    for (int l = 0; l < n->layers; l++) {
        const float* b = n->params + size_t(l) * PER_LAYER + TAPS * CH * CH;
        lbm_status st = conv(n, n->act[l], n->wf + size_t(l) * TAPS * CH * CH, b, n->act[l + 1], d,
                             l + 1 < n->layers ? 1 : 0, nullptr);
        if (st) return st;
    }
    n->d = d;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_net_create(int32_t layers, int32_t in_channels, int32_t out_channels, uint64_t seed, void* stream,
                          const lbm_allocator* alloc, lbm_net** out) {
    if (!out) return nfail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (layers < 1 || layers > 16 || in_channels < 1 || in_channels > CH || out_channels < 1 || out_channels > CH)
        return nfail(LBM_EINVAL, "layers must be 1..16 and channel counts 1..16");
    lbm_net* n = new (std::nothrow) lbm_net;
    if (!n) return nfail(LBM_ENOMEM, "host allocation failed");
    n->layers = layers;
    n->cin = in_channels;
    n->cout = out_channels;
    n->stream = static_cast<cudaStream_t>(stream);
    if (!n->mem.bind(alloc, n->stream)) {
        delete n;
        return nfail(LBM_EINVAL, "an allocator hook with alloc needs release");
    }
    const size_t np = size_t(layers) * PER_LAYER;
    // He-uniform initialisation over the fan-in of each layer (27 taps x its input channels);
    // channels beyond a layer's inputs or outputs keep zero weights
    std::vector<float> h(np, 0.f);
    uint64_t st = seed;
    for (int l = 0; l < layers; l++) {
        const int ci = l == 0 ? in_channels : CH, co = l + 1 == layers ? out_channels : CH;
        const float bound = std::sqrt(6.f / float(TAPS * ci));
        for (int o = 0; o < TAPS; o++)
            for (int m = 0; m < co; m++)
                for (int k = 0; k < ci; k++) {
                    const double u = double(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
                    h[size_t(l) * PER_LAYER + (o * CH + m) * CH + k] = float((2.0 * u - 1.0) * bound);
                }
    }
    auto bail = [&](lbm_status s) {
        std::string keep = lbm_last_error();
        lbm_net_destroy(n);
        lbm::set_last_error(keep.c_str());
        return s;
    };
    if (!n->mem.get(&n->params, np * 4) || !n->mem.get(&n->grads, np * 4) || !n->mem.get(&n->m, np * 4) ||
        !n->mem.get(&n->v, np * 4) || !n->mem.get(&n->wf, size_t(layers) * TAPS * CH * CH * 2) ||
        !n->mem.get(&n->wb, size_t(layers) * TAPS * CH * CH * 2) || !n->mem.get(&n->d_loss, sizeof(double)) ||
        cudaMallocHost(&n->h_loss, sizeof(double)) != cudaSuccess || !n->mem.get(&n->d_err, sizeof(int)))
        return bail(nfail(LBM_ENOMEM, "cannot allocate the net"));
    if (cudaMemcpy(n->params, h.data(), np * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m, 0, np * 4) != cudaSuccess || cudaMemset(n->v, 0, np * 4) != cudaSuccess ||
        cudaMemset(n->d_err, 0, sizeof(int)) != cudaSuccess)
        return bail(nfail(LBM_ECUDA, "cannot initialise the net"));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(nfail(LBM_ECUDA, "no CUDA device"));
    lbm_status s = refresh_weights(n);
    if (s) return bail(s);
    *out = n;
    return LBM_OK;
}

lbm_status lbm_net_destroy(lbm_net* n) {
    if (!n) return LBM_OK;
    if (n->stream) cudaStreamSynchronize(n->stream);
    free_acts(n);
    for (const void* p : {static_cast<const void*>(n->params), static_cast<const void*>(n->grads),
                          static_cast<const void*>(n->m), static_cast<const void*>(n->v),
                          static_cast<const void*>(n->wf), static_cast<const void*>(n->wb),
                          static_cast<const void*>(n->d_loss), static_cast<const void*>(n->d_err)})
        n->mem.put(p);
    if (n->h_loss) cudaFreeHost(n->h_loss);
    delete n;
    return LBM_OK;
}

lbm_status lbm_net_num_params(const lbm_net* n, int64_t* count) {
    if (!n || !count) return nfail(LBM_EINVAL, "NULL argument");
    *count = int64_t(n->layers) * PER_LAYER;
    return LBM_OK;
}

lbm_status lbm_net_get_params(const lbm_net* n, float* host) {
    if (!n || !host) return nfail(LBM_EINVAL, "NULL argument");
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(host, n->params, size_t(n->layers) * PER_LAYER * 4, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_net_set_params(lbm_net* n, const float* host) {
    if (!n || !host) return nfail(LBM_EINVAL, "NULL argument");
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(n->params, host, size_t(n->layers) * PER_LAYER * 4, cudaMemcpyHostToDevice));
    return refresh_weights(n);
}

lbm_status lbm_net_forward(lbm_net* n, const void* x, int32_t D, int32_t H, int32_t W, int32_t nvol, void* z) {
    if (!n || !x || !z) return nfail(LBM_EINVAL, "NULL argument");
    Dims d;
    lbm_status s = check_dims(D, H, W, nvol, d);
    if (s || (s = forward(n, static_cast<const __nv_bfloat16*>(x), d))) return s;
    NCU(cudaMemcpyAsync(z, n->act[n->layers], size_t(d.N) * CH * 2, cudaMemcpyDeviceToDevice, n->stream));
    return check_err(n);
}

lbm_status lbm_net_predict(lbm_net* n, const void* x, const float* skip, int32_t D, int32_t H, int32_t W, int32_t nvol,
                           float* pred) {
    if (!n || !x || !pred) return nfail(LBM_EINVAL, "NULL argument");
    Dims d;
    lbm_status s = check_dims(D, H, W, nvol, d);
    if (s || (s = forward(n, static_cast<const __nv_bfloat16*>(x), d))) return s;
    loss_kernel<<<int((d.N + 255) / 256), 256, 0, n->stream>>>(n->act[n->layers], skip, nullptr, nullptr, d.N, n->cout,
                                                               0.f, nullptr, pred, nullptr);
    NCU(cudaGetLastError());
    return check_err(n);
}

lbm_status lbm_net_train_step(lbm_net* n, const void* x, const float* skip, const float* target, const float* weight,
                              int32_t D, int32_t H, int32_t W, int32_t nvol, float lr, double* loss) {
    if (!n || !x || !target) return nfail(LBM_EINVAL, "NULL argument");
    Dims d;
    lbm_status s = check_dims(D, H, W, nvol, d);
    if (s || (s = forward(n, static_cast<const __nv_bfloat16*>(x), d))) return s;
    lbm_status r = lbm_net_gradient(n, skip, target, weight, loss);
    if (r) return r;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = float(1.0 - std::pow(double(b1), double(n->step))), c2 = float(1.0 - std::pow(double(b2), double(n->step)));
    const int np = n->layers * PER_LAYER;
    adam_kernel<<<(np + 255) / 256, 256, 0, n->stream>>>(n->params, n->grads, n->m, n->v, np, lr, b1, b2, 1e-8f, c1, c2);
    NCU(cudaGetLastError());
    return refresh_weights(n);
}

lbm_status lbm_net_gradient(lbm_net* n, const float* skip, const float* target, const float* weight, double* loss) {
    if (!n || !target) return nfail(LBM_EINVAL, "NULL argument");
    if (n->act.empty() || n->d.N == 0) return nfail(LBM_EINVAL, "run a forward pass first");
    const Dims& d = n->d;
    // count of weighted target values (the MSE denominator)
    double count = 0.0;
    if (weight) {
        std::vector<float> hw(size_t(d.N));
        NCU(cudaMemcpyAsync(hw.data(), weight, size_t(d.N) * 4, cudaMemcpyDeviceToHost, n->stream));
        NCU(cudaStreamSynchronize(n->stream));
        for (float w : hw) count += w;
    } else {
        count = double(d.N);
    }
    count *= n->cout;
    if (!(count > 0.0)) return nfail(LBM_EINVAL, "the loss weights are all zero");
    NCU(cudaMemsetAsync(n->d_loss, 0, sizeof(double), n->stream));
    NCU(cudaMemsetAsync(n->grads, 0, size_t(n->layers) * PER_LAYER * 4, n->stream));
    loss_kernel<<<int((d.N + 255) / 256), 256, 0, n->stream>>>(n->act[n->layers], skip, target, weight, d.N, n->cout,
                                                               float(1.0 / count), n->g0, nullptr, n->d_loss);
    const long long chunk = 4096;
    const dim3 wg(unsigned((d.N + chunk - 1) / chunk), TAPS);
    __nv_bfloat16* dz = n->g0;
    __nv_bfloat16* dx = n->g1;
    for (int l = n->layers - 1; l >= 0; l--) {
        float* gw = n->grads + size_t(l) * PER_LAYER;
        wgrad_kernel<<<wg, 256, 0, n->stream>>>(n->act[l], dz, gw, gw + TAPS * CH * CH, d, chunk);
        if (l > 0) {
            lbm_status st = conv(n, dz, n->wb + size_t(l) * TAPS * CH * CH, nullptr, dx, d, 2, n->act[l]);
            if (st) return st;
            std::swap(dz, dx);
        }
    }
    NCU(cudaGetLastError());
    NCU(cudaMemcpyAsync(n->h_loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    NCU(cudaStreamSynchronize(n->stream));
    if (loss) *loss = *n->h_loss / count;
    return check_err(n);
}

lbm_status lbm_net_set_wait_test(lbm_net* n, int32_t on) {
    if (!n) return nfail(LBM_EINVAL, "net is NULL");
    n->wait_test = on ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_net_set_backend(lbm_net* n, int32_t backend) {
    if (!n || (backend != 0 && backend != 1)) return nfail(LBM_EINVAL, "backend must be 0 (mma.sync) or 1 (tcgen05)");
    n->backend = backend;
    return LBM_OK;
}

lbm_status lbm_net_get_grads(const lbm_net* n, float* host) {
    if (!n || !host) return nfail(LBM_EINVAL, "NULL argument");
    NCU(cudaStreamSynchronize(n->stream));
    NCU(cudaMemcpy(host, n->grads, size_t(n->layers) * PER_LAYER * 4, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- warm-start data movement
namespace {

// Coarse-only solution on a full level-0 grid of nb[3] blocks of B^3 cells, block-major in the
// forest's order (block (bx, by, bz) is block (bz nb1 + by) nb0 + bx).  Value of component `comp`
// of a field [ncomp][n0] at cell (i, j, k), with periodic axes wrapped and walled axes clamped.
struct Coarse {
    const double* rho;
    const double* u;
    long long n0;
    int nb[3], B, per;
    __device__ __forceinline__ int fold(int i, int a) const {
        const int N = nb[a] * B;
        if ((per >> a) & 1) return ((i % N) + N) % N;
        return i < 0 ? 0 : (i >= N ? N - 1 : i);
    }
    __device__ __forceinline__ long long index(int i, int j, int k) const {
        i = fold(i, 0);
        j = fold(j, 1);
        k = fold(k, 2);
        const long long blk = ((long long)(k / B) * nb[1] + j / B) * nb[0] + i / B;
        return blk * B * B * B + ((long long)(k % B) * B + j % B) * B + i % B;
    }
};

// Features of voxel (vx, vy, vz) of the volume around block `blk` of level L: the coarse solution
// sampled trilinearly at the voxel's cell centre (Sec. 2: cell-centred values), the obstacle /
// outside-domain flag and the level.
__global__ void features_kernel(Coarse c, int level, int B, int halo, const int* __restrict__ blocks, int nblocks,
                                const double* __restrict__ spheres, int nspheres, double rho_scale, double u_scale,
                                __nv_bfloat16* __restrict__ x, float* __restrict__ skip) {
    const int D = B + 2 * halo;
    const long long V = (long long)D * D * D;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= V * nblocks) return;
    const int b = int(id / V);
    long long r = id - b * V;
    const int vx = int(r % D);
    r /= D;
    const int vy = int(r % D), vz = int(r / D);
    const int g[3] = {blocks[3 * b] * B + vx - halo, blocks[3 * b + 1] * B + vy - halo, blocks[3 * b + 2] * B + vz - halo};
    const double s = 1.0 / double(1 << level);
    double p[3];
    bool outside = false;
    for (int a = 0; a < 3; a++) {
        p[a] = (g[a] + 0.5) * s;   // level-0 units
        if (!((c.per >> a) & 1) && (p[a] < 0.0 || p[a] >= double(c.nb[a] * c.B))) outside = true;
    }
    bool solid = outside;
    for (int i = 0; i < nspheres && !solid; i++) {
        const double* q = spheres + 4 * i;
        const double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
        solid = dx * dx + dy * dy + dz * dz < q[3] * q[3];
    }
    int i0[3];
    double w[3];
    for (int a = 0; a < 3; a++) {
        const double t = p[a] - 0.5;
        const double f = floor(t);
        i0[a] = int(f);
        w[a] = t - f;
    }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int corner = 0; corner < 8; corner++) {
        const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
        const double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
        const long long k = c.index(i0[0] + dx, i0[1] + dy, i0[2] + dz);
        const double rho = c.rho[k];
        if (!isfinite(rho)) continue;   // obstacle cells of the coarse solution hold no value
        v[0] += wt * (rho - 1.0);
        for (int a = 0; a < 3; a++) v[1 + a] += wt * c.u[a * c.n0 + k];
    }
    __nv_bfloat16* xo = x + id * CH;
    const float f0 = float(v[0] * rho_scale), f1 = float(v[1] * u_scale), f2 = float(v[2] * u_scale),
                f3 = float(v[3] * u_scale);
    const float vals[CH] = {f0, f1, f2, f3, solid ? 1.f : 0.f, float(level) * 0.5f};
    for (int ch = 0; ch < CH; ch++) xo[ch] = __float2bfloat16_rn(vals[ch]);
    if (skip) {
        skip[id * 4 + 0] = f0;
        skip[id * 4 + 1] = f1;
        skip[id * 4 + 2] = f2;
        skip[id * 4 + 3] = f3;
    }
}

// Refined solution (block-major rho[n], u[3][n] of one level) -> training targets on the interior
// of each volume; weight 1 there on fluid cells, 0 on the halo and on obstacle cells.
__global__ void targets_kernel(const double* __restrict__ rho, const double* __restrict__ u, long long n, int B, int halo,
                               int nblocks, double rho_scale, double u_scale, float* __restrict__ target,
                               float* __restrict__ weight) {
    const int D = B + 2 * halo;
    const long long V = (long long)D * D * D;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= V * nblocks) return;
    const int b = int(id / V);
    long long r = id - b * V;
    const int vx = int(r % D) - halo;
    r /= D;
    const int vy = int(r % D) - halo, vz = int(r / D) - halo;
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    float w = 0.f;
    if (vx >= 0 && vx < B && vy >= 0 && vy < B && vz >= 0 && vz < B) {
        const long long k = (long long)b * B * B * B + ((long long)vz * B + vy) * B + vx;
        if (isfinite(rho[k])) {
            t[0] = float((rho[k] - 1.0) * rho_scale);
            for (int a = 0; a < 3; a++) t[1 + a] = float(u[a * n + k] * u_scale);
            w = 1.f;
        }
    }
    for (int a = 0; a < 4; a++) target[id * 4 + a] = t[a];
    weight[id] = w;
}

// Prediction on the interior of each volume -> block-major rho[n], u[3][n] of one level.
__global__ void fields_kernel(const float* __restrict__ pred, int B, int halo, int nblocks, double rho_scale,
                              double u_scale, double* __restrict__ rho, double* __restrict__ u) {
    const long long n = (long long)nblocks * B * B * B;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = int(k / ((long long)B * B * B));
    long long r = k - (long long)b * B * B * B;
    const int x = int(r % B);
    r /= B;
    const int y = int(r % B), z = int(r / B);
    const int D = B + 2 * halo;
    const long long id = (long long)b * D * D * D + ((long long)(z + halo) * D + (y + halo)) * D + (x + halo);
    rho[k] = 1.0 + double(pred[id * 4]) / rho_scale;
    for (int a = 0; a < 3; a++) u[a * n + k] = double(pred[id * 4 + 1 + a]) / u_scale;
}

}  // namespace

extern "C" {

lbm_status lbm_warmstart_features(const double* coarse_rho, const double* coarse_u, const int32_t coarse_blocks[3],
                                  int32_t B, int32_t periodic_mask, int32_t level, int32_t halo, const int32_t* blocks,
                                  int32_t nblocks, const double* spheres, int32_t nspheres, double rho_scale,
                                  double u_scale, void* x, float* skip, void* stream) {
    if (!coarse_rho || !coarse_u || !coarse_blocks || !blocks || !x || (nspheres > 0 && !spheres))
        return nfail(LBM_EINVAL, "NULL argument");
    if (B < 1 || halo < 0 || level < 0 || level > 20 || nblocks < 0 || nspheres < 0)
        return nfail(LBM_EINVAL, "invalid sizes");
    if (nblocks == 0) return LBM_OK;
    Coarse c{coarse_rho, coarse_u, 0, {coarse_blocks[0], coarse_blocks[1], coarse_blocks[2]}, B, periodic_mask};
    c.n0 = (long long)c.nb[0] * c.nb[1] * c.nb[2] * B * B * B;
    const long long D = B + 2 * halo, total = D * D * D * nblocks;
    features_kernel<<<unsigned((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        c, level, B, halo, blocks, nblocks, spheres, nspheres, rho_scale, u_scale, static_cast<__nv_bfloat16*>(x), skip);
    NCU(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_warmstart_targets(const double* rho, const double* u, int32_t B, int32_t halo, int32_t nblocks,
                                 double rho_scale, double u_scale, float* target, float* weight, void* stream) {
    if (!rho || !u || !target || !weight) return nfail(LBM_EINVAL, "NULL argument");
    if (B < 1 || halo < 0 || nblocks < 0) return nfail(LBM_EINVAL, "invalid sizes");
    if (nblocks == 0) return LBM_OK;
    const long long D = B + 2 * halo, total = D * D * D * nblocks, n = (long long)nblocks * B * B * B;
    targets_kernel<<<unsigned((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        rho, u, n, B, halo, nblocks, rho_scale, u_scale, target, weight);
    NCU(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_warmstart_fields(const float* pred, int32_t B, int32_t halo, int32_t nblocks, double rho_scale,
                                double u_scale, double* rho, double* u, void* stream) {
    if (!pred || !rho || !u) return nfail(LBM_EINVAL, "NULL argument");
    if (B < 1 || halo < 0 || nblocks < 0) return nfail(LBM_EINVAL, "invalid sizes");
    if (nblocks == 0) return LBM_OK;
    const long long n = (long long)nblocks * B * B * B;
    fields_kernel<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(pred, B, halo, nblocks,
                                                                                          rho_scale, u_scale, rho, u);
    NCU(cudaGetLastError());
    return LBM_OK;
}

}  // extern "C"
