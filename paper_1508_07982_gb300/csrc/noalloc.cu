// Mass and momentum totals of a caller-owned PDF array, with no allocation of any kind.
//
// Some callers cannot allocate device memory at the time they need the totals: runtimes that
// hand out all device memory from their own pre-sized pool and forbid the CUDA allocator after
// start-up, and embedded or safety-certified hosts that allow no dynamic allocation once
// initialised.  The regular lbm_reduce_mass_momentum keeps its
// per-CTA partial sums in memory that lbm_create_forest allocated; this entry point instead
// keeps them in one file-scope device array of fixed size, reserved when the library is
// loaded, so the call itself allocates nothing.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxCtas = LBM_NOALLOC_MAX_CELLS / LBM_NOALLOC_CELLS_PER_CTA;

// Partial sums {rho, jx, jy, jz, skipped cells} of each CTA.  Every GPU that loads the library
// holds this array (kMaxCtas * 5 doubles) until the process exits.  All calls share it.
static __device__ __align__(256) double g_partial[kMaxCtas * 5];


__host__ __device__ constexpr int ex(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1 : ((q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1 : ((q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0);
}
__host__ __device__ constexpr int ez(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1 : ((q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0);
}

template <typename T> __device__ __forceinline__ double as_double(T v) { return double(v); }
template <> __device__ __forceinline__ double as_double<__half>(__half v) { return double(__half2float(v)); }

// One CTA per LBM_NOALLOC_CELLS_PER_CTA cells.  Cells whose 19 values do not sum to a finite number
// (obstacle cells hold NaN by design; a diverged fluid cell would too) are left out of the sums and
// counted in the fifth slot.  The shifted layouts hold f - f^eq(rho0, u0), whose moments are rho - rho0
// and j - rho0 u0: each finite cell adds rho0 and rho0 u0 back.
template <typename T, bool SHIFTED>
__global__ void __launch_bounds__(kThreads) partial_kernel(const T* f, long long n, double rho0, double u0x,
                                                           double u0y, double u0z, double* partial) {
    const long long begin = (long long)blockIdx.x * LBM_NOALLOC_CELLS_PER_CTA;
    const long long end = begin + LBM_NOALLOC_CELLS_PER_CTA < n ? begin + LBM_NOALLOC_CELLS_PER_CTA : n;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long i = begin + threadIdx.x; i < end; i += kThreads) {
        double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int q = 0; q < 19; q++) {
            const double v = as_double(f[q * n + i]);
            r += v;
            jx += ex(q) * v;
            jy += ey(q) * v;
            jz += ez(q) * v;
        }
        if (!isfinite(r)) {
            s[4] += 1.0;
            continue;
        }
        s[0] += SHIFTED ? rho0 + r : r;
        s[1] += SHIFTED ? jx + rho0 * u0x : jx;
        s[2] += SHIFTED ? jy + rho0 * u0y : jy;
        s[3] += SHIFTED ? jz + rho0 * u0z : jz;
    }
    __shared__ double red[5][kThreads / 32];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; w++) v += red[threadIdx.x][w];
        partial[blockIdx.x * 5 + threadIdx.x] = v;
    }
}

// Sums the partials of the CTAs that the call launched, in a fixed order.
__global__ void __launch_bounds__(kThreads) final_kernel(const double* partial, int nctas, double* out) {
    __shared__ double red[5][kThreads];
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nctas; i += kThreads)
        for (int k = 0; k < 5; k++) s[k] += partial[5 * i + k];
    for (int k = 0; k < 5; k++) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w)
            for (int k = 0; k < 5; k++) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = red[threadIdx.x][0];
}

// Device address of g_partial, looked up once per device (the host-side symbol is only a
// stand-in; a kernel handed it would fault or read the wrong memory).
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {};
std::mutex g_addr_lock;

lbm_status fail(lbm_status s, const char* msg) {
    lbm::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" lbm_status lbm_mass_momentum_noalloc(const void* pdfs, int32_t precision, int64_t n_cells, double rho0,
                                                const double* u_shift, double* out, void* stream) {
    if (!pdfs || !out) return fail(LBM_EINVAL, "pdfs and out must be device pointers");
    if (precision < LBM_FP64 || precision > LBM_FP16S) return fail(LBM_EINVAL, "unknown precision");
    if (n_cells < 0) return fail(LBM_EINVAL, "negative cell count");
    if (n_cells > LBM_NOALLOC_MAX_CELLS) {
        char buf[160];
        snprintf(buf, sizeof buf, "n_cells %lld exceeds the maximum of %d cells this entry point's fixed scratch array covers",
                 (long long)n_cells, LBM_NOALLOC_MAX_CELLS);
        return fail(LBM_EINVAL, buf);
    }
    const double u0[3] = {u_shift ? u_shift[0] : 0.0, u_shift ? u_shift[1] : 0.0, u_shift ? u_shift[2] : 0.0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(LBM_ECUDA, "no usable CUDA device");
    double* partial;
    {
        std::lock_guard<std::mutex> lock(g_addr_lock);
        if (!g_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_partial);
            if (e != cudaSuccess || !p) return fail(LBM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
            g_addr[dev] = static_cast<double*>(p);
        }
        partial = g_addr[dev];
    }
    // an error left pending by earlier work is reported as such, not as this call's launch failure
    const cudaError_t prior = cudaPeekAtLastError();
    if (prior != cudaSuccess) {
        std::string m = std::string("a CUDA error from earlier work is pending: ") + cudaGetErrorString(prior);
        return fail(LBM_ECUDA, m.c_str());
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nctas = int((n_cells + LBM_NOALLOC_CELLS_PER_CTA - 1) / LBM_NOALLOC_CELLS_PER_CTA);
    if (nctas > 0) {
        if (precision == LBM_FP64)
            partial_kernel<double, false><<<nctas, kThreads, 0, s>>>(static_cast<const double*>(pdfs), n_cells, rho0,
                                                                      u0[0], u0[1], u0[2], partial);
        else if (precision == LBM_FP32S)
            partial_kernel<float, true><<<nctas, kThreads, 0, s>>>(static_cast<const float*>(pdfs), n_cells, rho0,
                                                                    u0[0], u0[1], u0[2], partial);
        else
            partial_kernel<__half, true><<<nctas, kThreads, 0, s>>>(static_cast<const __half*>(pdfs), n_cells, rho0,
                                                                     u0[0], u0[1], u0[2], partial);
    }
    final_kernel<<<1, kThreads, 0, s>>>(partial, nctas, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::string m = std::string("kernel launch failed: ") + cudaGetErrorString(e);
        return fail(LBM_ECUDA, m.c_str());
    }
    return LBM_OK;
}
