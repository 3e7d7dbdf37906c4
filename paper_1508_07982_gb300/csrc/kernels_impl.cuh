// Launcher definitions for one storage type; included once per precision translation unit.
#pragma once
#include "step_kernel.cuh"

namespace lbm {

template <typename T, typename C>
struct LaunchImpl {
    template <int COLL, int LB, int MINB>
    static constexpr int smem_bytes() { return StepSmem<T, C, LB, MINB>::BYTES + 128; }
    template <int COLL, int MINB>
    static void step_m(const StepArgs& a, int grid, cudaStream_t s) {
        if (a.LB == 3) step_kernel<T, C, COLL, 3, MINB><<<grid, 256, smem_bytes<COLL, 3, MINB>(), s>>>(a);
        else if (a.LB == 4) step_kernel<T, C, COLL, 4, MINB><<<grid, 256, smem_bytes<COLL, 4, MINB>(), s>>>(a);
        else step_kernel<T, C, COLL, 5, MINB><<<grid, 256, smem_bytes<COLL, 5, MINB>(), s>>>(a);
    }
    template <int COLL, int LB, int MINB>
    static cudaError_t attr() {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<T, C, COLL, LB, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<COLL, LB, MINB>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_batch_kernel<T, C, COLL, LB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_bytes<COLL, LB, MINB>());
        return e;
    }
    template <int COLL, int LB>
    static cudaError_t attr_m() {
        cudaError_t e = attr<COLL, LB, 1>();
        if (e == cudaSuccess) e = attr<COLL, LB, 2>();
        if (e == cudaSuccess) e = attr<COLL, LB, 3>();
        if (e == cudaSuccess) e = attr<COLL, LB, 4>();
        return e;
    }
    template <int COLL>
    static cudaError_t attr_l() {
        cudaError_t e = attr_m<COLL, 3>();
        if (e == cudaSuccess) e = attr_m<COLL, 4>();
        if (e == cudaSuccess) e = attr_m<COLL, 5>();
        return e;
    }
    static cudaError_t prepare() {
        static const cudaError_t e = [] {
            cudaError_t r = attr_l<LBM_TRT>();
            if (r == cudaSuccess) r = attr_l<LBM_SRT>();
            return r;
        }();
        return e;
    }
    template <int COLL>
    static void step_b(const StepArgs& a, int grid, cudaStream_t s) {
        if (a.minb == 1) step_m<COLL, 1>(a, grid, s);
        else if (a.minb == 2) step_m<COLL, 2>(a, grid, s);
        else if (a.minb == 4) step_m<COLL, 4>(a, grid, s);
        else step_m<COLL, 3>(a, grid, s);
    }
    static void step(const StepArgs& a, int collision, int grid, cudaStream_t s) {
        if (grid <= 0) return;
        if (collision == LBM_TRT) step_b<LBM_TRT>(a, grid, s);
        else step_b<LBM_SRT>(a, grid, s);
    }
    static void init(const DevLevel& lv, int cur, int LB, const LevelParams* P, double rho0, const double* rho,
                     const double* u, int uniform, const double uc[4], int collision, cudaStream_t s) {
        if (lv.ncells == 0) return;
        const int grid = int((lv.ncells + 255) / 256);
        if (collision == LBM_TRT)
            init_kernel<T, C, LBM_TRT><<<grid, 256, 0, s>>>(lv, cur, LB, P, rho0, rho, u, uniform, uc[0], uc[1], uc[2], uc[3]);
        else
            init_kernel<T, C, LBM_SRT><<<grid, 256, 0, s>>>(lv, cur, LB, P, rho0, rho, u, uniform, uc[0], uc[1], uc[2], uc[3]);
    }
    static void macro(const DevLevel& lv, int cur, int LB, const LevelParams* P, double rho0, double* rho, double* u,
                      int64_t ustride, cudaStream_t s) {
        const int64_t n = int64_t(lv.nown) << (3 * LB);
        if (n == 0) return;
        macro_kernel<T><<<int((n + 255) / 256), 256, 0, s>>>(lv, cur, LB, P, rho0, rho, u, ustride);
    }
    static void get_pdfs(const DevLevel& lv, int cur, int LB, double rho0, double* out, cudaStream_t s) {
        const int64_t n = int64_t(lv.nown) << (3 * LB);
        if (n == 0) return;
        get_pdfs_kernel<T><<<int((n + 255) / 256), 256, 0, s>>>(lv, cur, LB, rho0, out);
    }
    static void set_pdfs(const DevLevel& lv, int cur, int LB, double rho0, const double* in, cudaStream_t s) {
        if (lv.ncells == 0) return;
        set_pdfs_kernel<T><<<int((lv.ncells + 255) / 256), 256, 0, s>>>(lv, cur, LB, rho0, in);
    }
    static void reduce(const DevLevel& lv, int cur, int LB, const LevelParams* P, double rho0, double w,
                       double* partial, int grid, cudaStream_t s) {
        if (grid <= 0) return;
        reduce_level_kernel<T><<<grid, 256, 0, s>>>(lv, cur, LB, P, rho0, w, partial);
    }
    static void totals(const double* wpart, int64_t n, double w, const double shift[4], double* partial, int grid,
                       cudaStream_t s) {
        if (grid <= 0) return;
        totals_level_kernel<T><<<grid, 256, 0, s>>>(wpart, n, w, shift[0], shift[1], shift[2], shift[3], partial);
    }
    static void explode(const DevLevel& lv, const DevLevel& co, int cur, int cur_c, cudaStream_t s) {
        if (lv.nework <= 0) return;
        explode_kernel<T><<<(lv.nework + 255) / 256, 256, 0, s>>>(lv, co, cur, cur_c);
    }
    template <int COLL, int MINB>
    static void step_batch_m(const StepArgs* args, const int* prefix, int n, int total, int grid, int LB, cudaStream_t s) {
        if (LB == 3)
            step_batch_kernel<T, C, COLL, 3, MINB><<<grid, 256, smem_bytes<COLL, 3, MINB>(), s>>>(args, prefix, n, total);
        else if (LB == 4)
            step_batch_kernel<T, C, COLL, 4, MINB><<<grid, 256, smem_bytes<COLL, 4, MINB>(), s>>>(args, prefix, n, total);
        else
            step_batch_kernel<T, C, COLL, 5, MINB><<<grid, 256, smem_bytes<COLL, 5, MINB>(), s>>>(args, prefix, n, total);
    }
    template <int COLL>
    static void step_batch_b(const StepArgs* args, const int* prefix, int n, int total, int grid, int LB, int minb,
                             cudaStream_t s) {
        if (minb == 1) step_batch_m<COLL, 1>(args, prefix, n, total, grid, LB, s);
        else if (minb == 2) step_batch_m<COLL, 2>(args, prefix, n, total, grid, LB, s);
        else if (minb == 4) step_batch_m<COLL, 4>(args, prefix, n, total, grid, LB, s);
        else step_batch_m<COLL, 3>(args, prefix, n, total, grid, LB, s);
    }
    static void step_batch(const StepArgs* args, const int* prefix, int n, int total, int grid, int collision, int LB,
                           int minb, cudaStream_t s) {
        if (total <= 0 || grid <= 0) return;
        if (collision == LBM_TRT) step_batch_b<LBM_TRT>(args, prefix, n, total, grid, LB, minb, s);
        else step_batch_b<LBM_SRT>(args, prefix, n, total, grid, LB, minb, s);
    }
    static void explode_batch(const StepArgs* args, const int* prefix, int n, int total, int grid, cudaStream_t s) {
        if (total <= 0 || grid <= 0) return;
        explode_batch_kernel<T><<<grid, 256, 0, s>>>(args, prefix, n, total);
    }
    template <int COLL>
    static void side_c(const StepArgs& a, int grid, cudaStream_t s) {
        if (a.LB == 3) side_kernel<T, C, COLL, 3><<<grid, 256, 0, s>>>(a);
        else if (a.LB == 4) side_kernel<T, C, COLL, 4><<<grid, 256, 0, s>>>(a);
        else side_kernel<T, C, COLL, 5><<<grid, 256, 0, s>>>(a);
    }
    static void side(const StepArgs& a, int collision, int grid, cudaStream_t s) {
        if (grid <= 0) return;
        if (collision == LBM_TRT) side_c<LBM_TRT>(a, grid, s);
        else side_c<LBM_SRT>(a, grid, s);
    }
    template <int COLL>
    static void side_batch_c(const StepArgs* args, const int* prefix, int n, int total, int grid, int LB, cudaStream_t s) {
        if (LB == 3) side_batch_kernel<T, C, COLL, 3><<<grid, 256, 0, s>>>(args, prefix, n, total);
        else if (LB == 4) side_batch_kernel<T, C, COLL, 4><<<grid, 256, 0, s>>>(args, prefix, n, total);
        else side_batch_kernel<T, C, COLL, 5><<<grid, 256, 0, s>>>(args, prefix, n, total);
    }
    static void side_batch(const StepArgs* args, const int* prefix, int n, int total, int grid, int collision, int LB,
                           cudaStream_t s) {
        if (total <= 0 || grid <= 0) return;
        if (collision == LBM_TRT) side_batch_c<LBM_TRT>(args, prefix, n, total, grid, LB, s);
        else side_batch_c<LBM_SRT>(args, prefix, n, total, grid, LB, s);
    }
    static int ctas_per_sm(int LB, int minb) {
        const int m = minb == 1 ? 1 : (minb == 2 ? 2 : (minb == 4 ? 4 : 3));
        auto fit = [](int lb, int mb) -> int {
            if (lb == 3) return mb == 1 ? StepSmem<T, C, 3, 1>::kMinCtas : mb == 2 ? StepSmem<T, C, 3, 2>::kMinCtas
                                 : mb == 4 ? StepSmem<T, C, 3, 4>::kMinCtas : StepSmem<T, C, 3, 3>::kMinCtas;
            if (lb == 4) return mb == 1 ? StepSmem<T, C, 4, 1>::kMinCtas : mb == 2 ? StepSmem<T, C, 4, 2>::kMinCtas
                                 : mb == 4 ? StepSmem<T, C, 4, 4>::kMinCtas : StepSmem<T, C, 4, 3>::kMinCtas;
            return mb == 1 ? StepSmem<T, C, 5, 1>::kMinCtas : mb == 2 ? StepSmem<T, C, 5, 2>::kMinCtas
                 : mb == 4 ? StepSmem<T, C, 5, 4>::kMinCtas : StepSmem<T, C, 5, 3>::kMinCtas;
        };
        return fit(LB, m);
    }
    static const Launchers& get() {
        static const Launchers L{&step,       &init,          &macro,   &get_pdfs,     &set_pdfs,
                                 &reduce,     &totals,        &explode, &step_batch,   &explode_batch,
                                 &prepare,    &ctas_per_sm,   StepSmem<T, C, 5, 3>::CX == 2,
                                 &side,       &side_batch};
        return L;
    }
};

}  // namespace lbm
