// C-ABI runtime: forest upload, level schedule, CUDA-graph replay, timing, reductions.
//
// The level schedule restates Alg. 1 with every collision fused into the preceding
// stream (the kernels store post-collision states, Alg. 2's StreamCollide applied on all
// levels).  Per coarse step, with F_L(s) the fused kernel of level L in its sub-step s and
// E_L the explosion into level L's ghost layers:
//     S(0) = [S(1)] F_0(1)      S(L) = E_L [S(L+1)] F_L(1) [S(L+1)] F_L(2)   (L >= 1)
// E_L copies the coarse post-collision state into the ghost-layer-1 values that owned cells of
// level L pull in sub-step 1 (Eq. ctof); the ghost stream reads the other exploded values it
// needs from the coarse parents, which level L-1 leaves unchanged until S(L) returns.  F_L(1)
// carries stream, coalescence (reads of the finer ghost layers) and the second collision of
// Alg. 1; F_L(2) carries the second stream and the first collision of the next visit.  Levels >= 1 flip their two-grid parity an even number of times
// per coarse step, level 0 once; the runtime therefore captures one graph per level-0 parity and
// replays them alternately.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "devmem.h"
#include "kernels.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CU(call)                                                                                              \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", #call,   \
                        cudaGetErrorString(e_));                                                              \
    } while (0)

struct Launch {
    int level, substep, grid;
    int type;   // 0: stream-collide F_L(substep), 1: explosion E_L, 2: coupled cells and ghost work of
                // F_L(substep) when its column walk is persistent (launched right before it)
    int lzc;    // log2 cells per thread along z of this level's stream-collide launch
    int tot = 0;   // 1: the level's last sub-step of a coarse step, which records the totals
    int wctas = 0;   // persistent column walk (FP32/FP16 storage): its CTAs, the whole grid
    int wslot = 0;   // its pair of work counters in the forest's counter array
};

struct DevBuf {
    void* f[2] = {nullptr, nullptr};
    uint8_t* cell = nullptr;
    int32_t *nbr = nullptr, *parent = nullptr, *child = nullptr, *pos = nullptr;
    uint8_t* kind = nullptr;
    uint32_t* link = nullptr;
    uint32_t* colsolid = nullptr;
    uint8_t* colspec = nullptr;
    uint32_t* gwork[2] = {nullptr, nullptr};
    uint32_t* ework = nullptr;
    uint32_t* cwork = nullptr;
    double* wpart = nullptr;   // per-warp moments of the level's last sub-step
};

__global__ void reduce_final_kernel(const double* partial, int n, double* out) {
    __shared__ double red[4][256];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int k = 0; k < 4; k++) s[k] += partial[4 * i + k];
    for (int k = 0; k < 4; k++) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w)
            for (int k = 0; k < 4; k++) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

// Volume-weighted sums {sum w |u - u_prev|^2, sum w |u|^2, fluid cells with a non-finite velocity}
// over the fluid cells of one level's velocity u[3][n] (cell classes `cell`; obstacle cells hold
// NaN by design); u_prev takes u.  One partial per CTA.
__global__ void residual_kernel(const double* __restrict__ u, double* __restrict__ uprev, const uint8_t* __restrict__ cell,
                                int64_t n, double w, double* __restrict__ partial) {
    double s0 = 0.0, s1 = 0.0, bad = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        if (cell[i] != CK_FLUID) continue;
        double d2 = 0.0, u2 = 0.0;
        bool ok = true;
        for (int a = 0; a < 3; a++) {
            const double v = u[a * n + i], p = uprev[a * n + i];
            ok = ok && isfinite(v);
            d2 += (v - p) * (v - p);
            u2 += v * v;
            uprev[a * n + i] = v;
        }
        if (ok) {
            s0 += w * d2;
            s1 += w * u2;
        } else {
            bad += 1.0;
        }
    }
    __shared__ double red[3][256];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = bad;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (int(threadIdx.x) < k)
            for (int c = 0; c < 3; c++) red[c][threadIdx.x] += red[c][threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[4 * blockIdx.x] = red[0][0];
        partial[4 * blockIdx.x + 1] = red[1][0];
        partial[4 * blockIdx.x + 2] = red[2][0];
        partial[4 * blockIdx.x + 3] = 0.0;
    }
}

const Launchers& launchers_for(int precision) {
    if (precision == LBM_FP64) return launchers_f64();
    if (precision == LBM_FP32S) return launchers_f32();
    return launchers_f16();
}

size_t elem_size(int precision) { return precision == LBM_FP64 ? 8 : (precision == LBM_FP32S ? 4 : 2); }

}  // namespace

void lbm::set_last_error(const char* msg) { g_err = msg; }

struct lbm_forest {
    Plan plan;
    double u0[3] = {0.0, 0.0, 0.0};   // storage shift velocity (shifted layouts only)
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;      // side branch: coupled cells and ghost work beside the walk
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    const Launchers* L = nullptr;
    size_t esize = 0;
    std::vector<DevBuf> buf;
    std::vector<DevLevel> dl;
    std::vector<LevelParams> hp;
    LevelParams* d_params = nullptr;
    double* d_wall = nullptr;
    double* d_partial = nullptr;
    std::vector<int> red_grid;
    int red_total = 0;
    double* d_out = nullptr;
    int* d_wq = nullptr;          // work counters of the persistent walk launches, 2 per launch
    size_t nwq = 0;
    double* h_out = nullptr;
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    int cur[LBM_MAX_LEVELS] = {};
    unsigned init_mask = 0;
    bool params_set = false;
    std::vector<Launch> sched;
    cudaGraph_t graph[2] = {};
    cudaGraphExec_t exec[2] = {};
    bool timing = false;
    int tmax = 0, tused = 0;
    std::vector<cudaEvent_t> tev;
    int64_t updates = 0;
    int lzc = 3;        // upper bound of log2 cells per thread along z (small levels use fewer)
    int minb = 3;       // CTAs per SM of the step-kernel variant
    std::vector<int64_t> tot_warps;   // per level: warp entries its recording launch writes
    bool totals_valid = false;        // the recorded moments describe the current state
    std::vector<double*> uprev;   // per level, the velocity of the previous residual call
    double* d_rpart = nullptr;    // residual partial sums
    DevMem mem;                   // device memory: the caller's allocator hook or cudaMalloc
};

namespace {

void free_graphs(lbm_forest* f) {
    for (int p = 0; p < 2; p++) {
        if (f->exec[p]) cudaGraphExecDestroy(f->exec[p]);
        if (f->graph[p]) cudaGraphDestroy(f->graph[p]);
        f->exec[p] = nullptr;
        f->graph[p] = nullptr;
    }
}

void free_timing(lbm_forest* f) {
    for (cudaEvent_t e : f->tev) cudaEventDestroy(e);
    f->tev.clear();
    f->timing = false;
    f->tmax = f->tused = 0;
}

// CTAs of a persistent column walk over `nown` owned bricks of B^3 cells: the `resident` CTAs the
// GPU holds at once, or fewer when the level has less than one chunk per warp (a chunk: the two
// cells of each of a warp's 32 threads in 8 planes, B^3 / 512 chunks per brick, 8 warps per CTA).
int walk_ctas(int nown, int B, int resident) {
    const int64_t chunks = int64_t(nown) * B * B * B / 512;
    return int(std::max<int64_t>(1, std::min<int64_t>((chunks + 7) / 8, resident)));
}

// log2 of the planes of a persistent walk's chunk: 8 planes where every warp of the `wctas` CTAs
// still gets about six chunks, fewer (down to 1; the kernel raises it to its pipeline depth)
// where the level is small, so that the warps finish together.
int chunk_planes_log2(int nown, int LB, int wctas) {
    const int64_t tasks = int64_t(nown) << (3 * LB - 6);   // warp tasks: 64 cells in one plane
    int zl = 3;
    while (zl > 0 && (tasks >> zl) < int64_t(6) * 8 * wctas) zl--;
    return std::min(zl, LB);
}

StepArgs make_args(const lbm_forest* f, const Launch& l, const int* cur) {
    StepArgs a{};
    const int L = l.level, n = f->plan.nlev;
    a.lv = f->dl[L];
    if (L > 0) a.co = f->dl[L - 1];
    if (L + 1 < n) a.fi = f->dl[L + 1];
    a.cur = cur[L];
    a.cur_c = L > 0 ? cur[L - 1] : 0;
    a.cur_f = L + 1 < n ? cur[L + 1] : 0;
    a.substep = l.substep;
    a.LB = f->plan.LB;
    a.lzc = l.lzc;
    a.minb = f->minb;
    a.per = (f->plan.per[0] ? 1 : 0) | (f->plan.per[1] ? 2 : 0) | (f->plan.per[2] ? 4 : 0);
    a.params = f->d_params + L;
    a.wall = f->d_wall;
    a.rho0 = f->plan.d.rho0;
    a.inv_rho0 = 1.0 / f->plan.d.rho0;
    a.totals = l.tot ? f->buf[L].wpart : nullptr;
    a.fslip = 0;
    for (int k = 0; k < 6; k++)
        if (f->plan.d.bc[k] == LBM_BC_FREESLIP) a.fslip |= 1 << k;
    a.obstacle_term = (f->u0[0] != 0.0 || f->u0[1] != 0.0 || f->u0[2] != 0.0) ? 1 : 0;
    for (int k = 0; k < 3; k++) a.two_u0[k] = float(2.0 * f->u0[k]);
    for (int q = 0; q < Q; q++) a.e_two_u0[q] = float(2.0 * (EX[q] * f->u0[0] + EY[q] * f->u0[1] + EZ[q] * f->u0[2]));
    a.wctas = l.wctas;
    a.wq = f->d_wq ? f->d_wq + 2 * l.wslot : nullptr;
    return a;
}

lbm_status build_schedule(lbm_forest* f) {
    f->sched.clear();
    const int n = f->plan.nlev, B = f->plan.B;
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    auto push = [&](int L, int s) {
        const HostLevel& V = f->plan.lv[L];
        const int64_t nwork = int64_t(V.gwork[s - 1].size() / 4);
        if (f->L->persistent) {
            const int resident = sms * f->L->ctas_per_sm(f->plan.LB, f->minb);
            const int w = walk_ctas(V.nown, B, resident);
            const int zl = chunk_planes_log2(V.nown, f->plan.LB, w);
            const int side = int((V.cwork.size() + 255) / 256) + int((nwork + 255) / 256);
            if (side > 0) f->sched.push_back({L, s, side, 2, zl, 0, w, int(f->sched.size()) + 1});
            f->sched.push_back({L, s, w, 0, zl, 0, w, int(f->sched.size())});
            return;
        }
        // cells per thread: the largest power of two up to the configured bound that still gives
        // about four waves of CTAs on this level
        int lzc = f->lzc;
        while (lzc > 0 && int64_t(V.nown) * B * B * (B >> lzc) / 256 < int64_t(4) * sms * f->minb) lzc--;
        const int64_t units = int64_t(V.nown) * B * B * (B >> lzc);
        int grid = int((units + 255) / 256) + int((nwork + 255) / 256) + int((V.cwork.size() + 255) / 256);
        f->sched.push_back({L, s, grid, 0, lzc});
    };
    auto explode = [&](int L) {
        const HostLevel& V = f->plan.lv[L];
        f->sched.push_back({L, 0, int((V.ework.size() / 4 + 255) / 256), 1, 0});
    };
    std::function<void(int)> rec = [&](int L) {
        if (L == 0) {
            if (n > 1) rec(1);
            push(0, 1);
            return;
        }
        explode(L);
        if (L + 1 < n) rec(L + 1);
        push(L, 1);
        if (L + 1 < n) rec(L + 1);
        push(L, 2);
    };
    rec(0);
    // work counters of the persistent walks (zero between launches)
    if (f->L->persistent && f->nwq < 2 * f->sched.size()) {
        f->mem.put(f->d_wq);
        f->d_wq = nullptr;
        f->nwq = 0;
        if (!f->mem.get(&f->d_wq, 2 * f->sched.size() * sizeof(int)))
            return fail(LBM_ENOMEM, "cannot allocate the walk's work counters");
        CU(cudaMemset(f->d_wq, 0, 2 * f->sched.size() * sizeof(int)));
        f->nwq = 2 * f->sched.size();
    }
    // the last sub-step of each level in the coarse step records the totals of what it writes; the
    // warp layout of what an earlier schedule recorded no longer matches
    f->totals_valid = false;
    f->tot_warps.assign(n, 0);
    for (int L = 0; L < n; L++)
        for (size_t k = f->sched.size(); k-- > 0;)
            if (f->sched[k].level == L && f->sched[k].type == 0) {
                Launch& l = f->sched[k];
                l.tot = 1;
                if (k > 0 && f->sched[k - 1].type == 2 && f->sched[k - 1].level == L) f->sched[k - 1].tot = 1;
                // the column walk's warps, then the coupled cells' warps
                const int64_t units = int64_t(f->plan.lv[L].nown) * B * B * (B >> l.lzc);
                f->tot_warps[L] = (l.wctas ? int64_t(l.wctas) * 8 : units / 32) +
                                  int64_t(f->plan.lv[L].cwork.size() + 255) / 256 * 8;
                break;
            }
    return LBM_OK;
}

// Enqueues every kernel of one coarse step on stream s; cur holds the two-grid parity of each
// level and is advanced.  With events, evs[k] is recorded before launch k and evs[k+1] after.
void enqueue_step(lbm_forest* f, cudaStream_t s, int* cur, cudaEvent_t* evs) {
    bool joined = true;
    for (size_t k = 0; k < f->sched.size(); k++) {
        const Launch& l = f->sched[k];
        if (evs) cudaEventRecord(evs[k], s);
        if (l.type == 1) {
            f->L->explode(f->dl[l.level], f->dl[l.level - 1], cur[l.level], cur[l.level - 1], s);
            continue;
        }
        if (l.type == 2 && evs) {   // timed alone, in series
            f->L->side(make_args(f, l, cur), f->plan.d.collision, l.grid, s);
            continue;
        }
        if (l.type == 2) {
            // the coupled cells and ghost work of the walk that follows (same parity), on a branch
            // beside it: they read the same grid and write cells the walk does not
            cudaEventRecord(f->ev_fork, s);
            cudaStreamWaitEvent(f->side, f->ev_fork, 0);
            f->L->side(make_args(f, l, cur), f->plan.d.collision, l.grid, f->side);
            cudaEventRecord(f->ev_join, f->side);
            joined = false;
            continue;
        }
        StepArgs a = make_args(f, l, cur);
        f->L->step(a, f->plan.d.collision, l.grid, s);
        if (!joined) {
            cudaStreamWaitEvent(s, f->ev_join, 0);
            joined = true;
        }
        cur[l.level] ^= 1;
    }
    if (evs) cudaEventRecord(evs[f->sched.size()], s);
}

lbm_status capture(lbm_forest* f, int parity) {
    int cur[LBM_MAX_LEVELS];
    std::memcpy(cur, f->cur, sizeof cur);
    cur[0] = parity;
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal));
    enqueue_step(f, f->cap, cur, nullptr);
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(f->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(LBM_ECUDA, "kernel launch during capture failed: %s", cudaGetErrorString(le));
    }
    if (ce != cudaSuccess) return fail(LBM_ECUDA, "stream capture failed: %s", cudaGetErrorString(ce));
    f->graph[parity] = g;
    CU(cudaGraphInstantiate(&f->exec[parity], g, 0));
    return LBM_OK;
}

lbm_status ensure_stage(lbm_forest* f, size_t bytes) {
    if (f->stage_bytes >= bytes) return LBM_OK;
    f->mem.put(f->d_stage);
    f->d_stage = nullptr;
    f->stage_bytes = 0;
    if (!f->mem.get(&f->d_stage, bytes)) return fail(LBM_ENOMEM, "cannot allocate %zu bytes of staging", bytes);
    f->stage_bytes = bytes;
    return LBM_OK;
}

template <typename T>
lbm_status upload(DevMem& mem, T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return LBM_OK;
    if (!mem.get(dst, v.size() * sizeof(T))) return fail(LBM_ENOMEM, "cannot allocate %zu bytes of tables", v.size() * sizeof(T));
    CU(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return LBM_OK;
}

lbm_status check_level(const lbm_forest* f, int level) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    if (level < 0 || level >= f->plan.nlev) return fail(LBM_EINVAL, "level %d out of range [0, %d)", level, f->plan.nlev);
    return LBM_OK;
}

int64_t owned_cells(const lbm_forest* f, int L) {
    return int64_t(f->plan.lv[L].nown) * f->plan.B * f->plan.B * f->plan.B;
}


// FP64 arithmetic probe: kProbeChains independent FMA chains per thread (enough to cover the FP64
// pipe's latency), `iters` FMAs each; the sum is written so that nothing is eliminated.
constexpr int kProbeChains = 8;
__device__ double g_probe_sink;   // written only if the chains reach an impossible value

__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(int iters) {
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) x[c] = 1.0 + 1e-9 * (threadIdx.x + c);
    const double a = 0.999999999, b = 1e-10;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kProbeChains; c++) x[c] = fma(x[c], a, b);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; c++) t += x[c];
    if (t == 12345.0) g_probe_sink = t;   // never true; keeps the chains live
}

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm_lattice(int32_t* e, double* w, int32_t* opp) {
    if (!e || !w || !opp) return fail(LBM_EINVAL, "NULL output");
    for (int q = 0; q < Q; q++) {
        e[3 * q] = EX[q];
        e[3 * q + 1] = EY[q];
        e[3 * q + 2] = EZ[q];
        w[q] = weight(q);
        opp[q] = OPP[q];
    }
    return LBM_OK;
}

lbm_status lbm_plan_create(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag, void* user,
                           lbm_plan** out) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_plan* p = new (std::nothrow) lbm_plan;
    if (!p) return fail(LBM_ENOMEM, "host allocation failed");
    std::string err;
    if (!build_plan(d, refine, flag, user, p->p, err)) {
        delete p;
        return fail(LBM_EINVAL, "%s", err.c_str());
    }
    *out = p;
    return LBM_OK;
}

lbm_status lbm_plan_num_levels(const lbm_plan* p, int32_t* n) {
    if (!p || !n) return fail(LBM_EINVAL, "NULL argument");
    *n = p->p.nlev;
    return LBM_OK;
}

lbm_status lbm_plan_leaves(const lbm_plan* p, int32_t level, int32_t* n, int32_t* blocks) {
    if (!p || !n) return fail(LBM_EINVAL, "NULL argument");
    if (level < 0 || level >= p->p.nlev) return fail(LBM_EINVAL, "level out of range");
    const HostLevel& V = p->p.lv[level];
    *n = V.nown;
    if (blocks) std::memcpy(blocks, V.pos.data(), size_t(V.nown) * 3 * sizeof(int32_t));
    return LBM_OK;
}

lbm_status lbm_plan_counts(const lbm_plan* p, int32_t level, int64_t counts[4]) {
    if (!p || !counts) return fail(LBM_EINVAL, "NULL argument");
    if (level < 0 || level >= p->p.nlev) return fail(LBM_EINVAL, "level out of range");
    const HostLevel& V = p->p.lv[level];
    counts[0] = V.nown;
    counts[1] = V.nfluid;
    counts[2] = V.nghost12;
    counts[3] = V.nghost;
    return LBM_OK;
}

lbm_status lbm_plan_ghost_work(const lbm_plan* p, int32_t level, int64_t work[4]) {
    if (!p || !work) return fail(LBM_EINVAL, "NULL argument");
    if (level < 0 || level >= p->p.nlev) return fail(LBM_EINVAL, "level out of range");
    const HostLevel& V = p->p.lv[level];
    for (int s = 0; s < 2; s++) {
        const std::vector<uint32_t>& g = V.gwork[s];
        int64_t values = 0;
        for (size_t i = 0; i < g.size(); i += 4) values += __builtin_popcount(g[i + 1]);
        work[2 * s] = int64_t(g.size() / 4);
        work[2 * s + 1] = values;
    }
    return LBM_OK;
}

lbm_status lbm_plan_destroy(lbm_plan* p) {
    delete p;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_forest* f) {
    if (!f) return LBM_OK;
    if (f->stream || f->cap) cudaStreamSynchronize(f->stream);
    free_graphs(f);
    free_timing(f);
    DevMem& m = f->mem;
    for (DevBuf& b : f->buf) {
        for (const void* p : {b.f[0], b.f[1]}) m.put(p);
        m.put(b.cell);
        m.put(b.nbr);
        m.put(b.parent);
        m.put(b.child);
        m.put(b.pos);
        m.put(b.kind);
        m.put(b.link);
        m.put(b.colsolid);
        m.put(b.colspec);
        m.put(b.gwork[0]);
        m.put(b.gwork[1]);
        m.put(b.ework);
        m.put(b.cwork);
        m.put(b.wpart);
    }
    for (double* p : f->uprev) m.put(p);
    m.put(f->d_rpart);
    m.put(f->d_params);
    m.put(f->d_wall);
    m.put(f->d_partial);
    m.put(f->d_out);
    m.put(f->d_wq);
    m.put(f->d_stage);
    if (f->h_out) cudaFreeHost(f->h_out);
    if (f->cap) cudaStreamDestroy(f->cap);
    if (f->side) cudaStreamDestroy(f->side);
    if (f->ev_fork) cudaEventDestroy(f->ev_fork);
    if (f->ev_join) cudaEventDestroy(f->ev_join);
    delete f;
    return LBM_OK;
}

lbm_status lbm_create_forest(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag, void* user,
                             void* stream, const lbm_allocator* alloc, lbm_forest** out) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_forest* f = new (std::nothrow) lbm_forest;
    if (!f) return fail(LBM_ENOMEM, "host allocation failed");
    std::string err;
    if (!build_plan(d, refine, flag, user, f->plan, err)) {
        delete f;
        return fail(LBM_EINVAL, "%s", err.c_str());
    }
    f->stream = static_cast<cudaStream_t>(stream);
    if (!f->mem.bind(alloc, f->stream)) {
        delete f;
        return fail(LBM_EINVAL, "an allocator hook with alloc needs release");
    }
    f->L = &launchers_for(f->plan.d.precision);
    f->esize = elem_size(f->plan.d.precision);
    const Plan& P = f->plan;
    const int B3 = P.B * P.B * P.B;
    for (int a = 0; a < 3; a++) f->u0[a] = P.d.precision == LBM_FP64 ? 0.0 : P.d.u_shift[a];
    auto bail = [&](lbm_status s) {
        std::string keep = g_err;
        lbm_destroy(f);
        g_err = keep;
        return s;
    };
    if (cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(LBM_ECUDA, "cannot create the capture stream (is a CUDA device present?)"));
    if (cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&f->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(LBM_ECUDA, "cannot create the side stream"));
    f->buf.resize(P.nlev);
    f->dl.resize(P.nlev);
    for (int L = 0; L < P.nlev; L++) {
        const HostLevel& V = P.lv[L];
        DevBuf& b = f->buf[L];
        const int64_t ncells = int64_t(V.nbricks()) * B3;
        for (int k = 0; k < 2; k++)
            if (!f->mem.get(&b.f[k], size_t(ncells) * Q * f->esize))
                return bail(fail(LBM_ENOMEM, "cannot allocate %lld bytes of PDFs on level %d",
                                 (long long)(ncells * Q * f->esize), L));
        lbm_status s;
        DevMem& m = f->mem;
        if ((s = upload(m, &b.cell, V.cell)) || (s = upload(m, &b.nbr, V.nbr)) || (s = upload(m, &b.parent, V.parent)) ||
            (s = upload(m, &b.child, V.child)) || (s = upload(m, &b.pos, V.pos)) || (s = upload(m, &b.kind, V.kind)) ||
            (s = upload(m, &b.link, V.link)) || (s = upload(m, &b.colsolid, V.colsolid)) ||
            (s = upload(m, &b.colspec, V.colspec)) || (s = upload(m, &b.gwork[0], V.gwork[0])) ||
            (s = upload(m, &b.gwork[1], V.gwork[1])) || (s = upload(m, &b.ework, V.ework)) ||
            (s = upload(m, &b.cwork, V.cwork)))
            return bail(s);
        // per-warp totals of the recording launch, sized for one cell per thread or a persistent walk
        // of up to 4,096 CTAs (the most warps), then the coupled cells' warps
        const int64_t wmax = std::max<int64_t>((int64_t(V.nown) * B3 + 255) / 256, 4 * 1024) * 8 +
                             int64_t(V.cwork.size() + 255) / 256 * 8;
        if (!f->mem.get(&b.wpart, size_t(wmax + 1) * 4 * sizeof(double)))
            return bail(fail(LBM_ENOMEM, "cannot allocate the totals of level %d", L));
        DevLevel& g = f->dl[L];
        g.f[0] = b.f[0];
        g.f[1] = b.f[1];
        g.cell = b.cell;
        g.nbr = b.nbr;
        g.parent = b.parent;
        g.child = b.child;
        g.pos = b.pos;
        g.kind = b.kind;
        g.link = b.link;
        g.colsolid = b.colsolid;
        g.colspec = b.colspec;
        g.ework = reinterpret_cast<const uint4*>(b.ework);
        g.nework = int(V.ework.size() / 4);
        g.cwork = b.cwork;
        g.ncwork = int(V.cwork.size());
        for (int k = 0; k < 2; k++) {
            g.gwork[k] = reinterpret_cast<const uint4*>(b.gwork[k]);
            g.ngwork[k] = int(V.gwork[k].size() / 4);
        }
        g.nown = V.nown;
        g.nbricks = V.nbricks();
        g.ncells = ncells;
        for (int a = 0; a < 3; a++) g.N[a] = V.N[a];
        for (int a = 0; a < 3; a++) g.u0[a] = f->u0[a];
        f->updates += V.nfluid << L;
    }
    // bounce-back terms 6 w_a rho0 (e_a . u_w) (velocity bounce-back; zero on no-slip faces and
    // obstacles, row 7); with a storage shift by f^eq(rho0, u0) a bounce-back also moves the
    // shift's odd part to the opposite direction, which adds -6 w_a rho0 (e_a . u0) to every row
    std::vector<double> wall(8 * Q, 0.0);
    for (int face = 0; face < 8; face++) {
        if (face == 6 || (face < 6 && P.d.bc[face] == LBM_BC_PERIODIC)) continue;
        double uw[3] = {0.0, 0.0, 0.0};
        if (face < 6 && P.d.bc[face] == LBM_BC_VELOCITY)
            for (int a = 0; a < 3; a++) uw[a] = P.d.bc_velocity[face][a];
        for (int a = 0; a < 3; a++) uw[a] -= f->u0[a];
        for (int q = 0; q < Q; q++)
            wall[face * Q + q] = 6.0 * weight(q) * P.d.rho0 * (EX[q] * uw[0] + EY[q] * uw[1] + EZ[q] * uw[2]);
    }
    lbm_status s;
    if ((s = upload(f->mem, &f->d_wall, wall))) return bail(s);
    f->hp.assign(P.nlev, LevelParams{});
    if (!f->mem.get(&f->d_params, sizeof(LevelParams) * P.nlev))
        return bail(fail(LBM_ENOMEM, "cannot allocate level parameters"));
    // reduction scratch: a fixed number of CTAs per level, so totals are summed in a fixed order
    f->red_grid.assign(P.nlev, 0);
    for (int L = 0; L < P.nlev; L++) {
        int64_t n = owned_cells(f, L);
        f->red_grid[L] = int(std::min<int64_t>((n + 255) / 256, 1216));
        f->red_total += f->red_grid[L];
    }
    if (!f->mem.get(&f->d_partial, sizeof(double) * 4 * std::max(f->red_total, 1)) ||
        !f->mem.get(&f->d_out, sizeof(double) * 4) || cudaMallocHost(&f->h_out, sizeof(double) * 4) != cudaSuccess)
        return bail(fail(LBM_ENOMEM, "cannot allocate reduction buffers"));
    if (f->L->prepare() != cudaSuccess) return bail(fail(LBM_ECUDA, "cannot set the step kernels' shared-memory limit"));
    // host staging of (rho, u) for the largest level, sized once: growing it later would free and
    // allocate device memory (cudaFree synchronises) in the middle of a caller's loop
    {
        int64_t nmax = 0;
        for (int L = 0; L < P.nlev; L++) nmax = std::max(nmax, owned_cells(f, L));
        lbm_status st = ensure_stage(f, size_t(nmax) * 4 * sizeof(double));
        if (st) return bail(st);
    }
    // cells per thread along z: 4 for 32^3 blocks, 2 for 16^3, 1 for 8^3 (the FP64 walk); the
    // paired walk of the shifted layouts runs two CTAs per SM with three planes staged ahead
    f->lzc = P.LB - 3;
    f->minb = P.d.precision == LBM_FP64 ? 3 : 2;
    if ((s = build_schedule(f))) return bail(s);
    *out = f;
    return LBM_OK;
}

lbm_status lbm_num_levels(const lbm_forest* f, int32_t* n) {
    if (!f || !n) return fail(LBM_EINVAL, "NULL argument");
    *n = f->plan.nlev;
    return LBM_OK;
}

lbm_status lbm_get_block_table(const lbm_forest* f, int32_t level, int32_t* n, int32_t* blocks) {
    lbm_status s = check_level(f, level);
    if (s) return s;
    if (!n) return fail(LBM_EINVAL, "n is NULL");
    const HostLevel& V = f->plan.lv[level];
    *n = V.nown;
    if (blocks) std::memcpy(blocks, V.pos.data(), size_t(V.nown) * 3 * sizeof(int32_t));
    return LBM_OK;
}

lbm_status lbm_cell_updates_per_coarse_step(const lbm_forest* f, int64_t* n) {
    if (!f || !n) return fail(LBM_EINVAL, "NULL argument");
    *n = f->updates;
    return LBM_OK;
}

lbm_status lbm_launches_per_coarse_step(const lbm_forest* f, int32_t* n) {
    if (!f || !n) return fail(LBM_EINVAL, "NULL argument");
    int c = 0;
    for (const Launch& l : f->sched) c += l.grid > 0;
    *n = c;
    return LBM_OK;
}

lbm_status lbm_set_level_params_explicit(lbm_forest* f, const double* le, const double* lo, const double* acc) {
    if (!f || !le || !lo) return fail(LBM_EINVAL, "NULL argument");
    const Plan& P = f->plan;
    for (int L = 0; L < P.nlev; L++) {
        if (!(le[L] > 0.0 && le[L] < 2.0) || !(lo[L] > 0.0 && lo[L] < 2.0))
            return fail(LBM_EINVAL, "relaxation rates of level %d outside ]0,2[", L);
        LevelParams& h = f->hp[L];
        h.le = le[L];
        h.lo = P.d.collision == LBM_TRT ? lo[L] : le[L];
        for (int k = 0; k < 3; k++) h.acc[k] = acc ? acc[3 * L + k] : 0.0;
        for (int k = 0; k < 3; k++) h.fa[k] = 3.0 * P.d.rho0 * h.acc[k];
        h.lef = float(h.le);
        h.lof = float(h.lo);
        for (int k = 0; k < 3; k++) h.faf[k] = float(h.fa[k]);
    }
    CU(cudaMemcpyAsync(f->d_params, f->hp.data(), sizeof(LevelParams) * P.nlev, cudaMemcpyHostToDevice, f->stream));
    CU(cudaStreamSynchronize(f->stream));
    f->params_set = true;
    return LBM_OK;
}

lbm_status lbm_set_level_params(lbm_forest* f, double le0, double magic, const double accel0[3]) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    const int n = f->plan.nlev;
    std::vector<double> le(n), lo(n), acc(3 * n);
    for (int L = 0; L < n; L++) {
        le[L] = scale_rate(le0, L);
        lo[L] = f->plan.d.collision == LBM_TRT ? lambda_odd(le[L], magic) : le[L];
        for (int k = 0; k < 3; k++) acc[3 * L + k] = accel0 ? std::ldexp(accel0[k], -L) : 0.0;
    }
    return lbm_set_level_params_explicit(f, le.data(), lo.data(), acc.data());
}

lbm_status lbm_init_equilibrium(lbm_forest* f, int32_t level, const double* rho, const double* u, int32_t on_device) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    if (!f->params_set) return fail(LBM_EINVAL, "set the level parameters before initialising");
    const Plan& P = f->plan;
    if (level == -1) {
        double uc[4] = {P.d.rho0, u ? u[0] : 0.0, u ? u[1] : 0.0, u ? u[2] : 0.0};
        for (int L = 0; L < P.nlev; L++) {
            f->cur[L] = 0;
            f->L->init(f->dl[L], 0, P.LB, f->d_params + L, P.d.rho0, nullptr, nullptr, 1, uc, P.d.collision, f->stream);
        }
        CU(cudaGetLastError());
        f->init_mask = (1u << P.nlev) - 1;
        f->totals_valid = false;
        return LBM_OK;
    }
    lbm_status s = check_level(f, level);
    if (s) return s;
    const int64_t n = owned_cells(f, level);
    const double *dr = rho, *du = u;
    if (!on_device && n && (rho || u)) {
        if ((s = ensure_stage(f, size_t(n) * 4 * sizeof(double)))) return s;
        double* st = static_cast<double*>(f->d_stage);
        if (rho) CU(cudaMemcpyAsync(st, rho, n * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        if (u) CU(cudaMemcpyAsync(st + n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        dr = rho ? st : nullptr;
        du = u ? st + n : nullptr;
    }
    double uc[4] = {0, 0, 0, 0};
    f->cur[level] = 0;
    f->L->init(f->dl[level], 0, P.LB, f->d_params + level, P.d.rho0, dr, du, 0, uc, P.d.collision, f->stream);
    CU(cudaGetLastError());
    if (!on_device) CU(cudaStreamSynchronize(f->stream));
    f->init_mask |= 1u << level;
    f->totals_valid = false;
    return LBM_OK;
}

lbm_status lbm_step_coarse(lbm_forest* f, int32_t n_steps) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    if (n_steps < 0) return fail(LBM_EINVAL, "negative step count");
    if (!f->params_set || f->init_mask != (1u << f->plan.nlev) - 1)
        return fail(LBM_EINVAL, "set the level parameters and initialise every level before stepping");
    for (int i = 0; i < n_steps; i++) {
        if (f->timing && f->tused < f->tmax) {
            // measured steps: the same launches, enqueued directly with an event between each
            // pair (host work per step is far below the step's GPU time)
            int cur[LBM_MAX_LEVELS];
            std::memcpy(cur, f->cur, sizeof cur);
            enqueue_step(f, f->stream, cur, &f->tev[size_t(f->tused) * (f->sched.size() + 1)]);
            CU(cudaGetLastError());
            f->tused++;
            f->cur[0] ^= 1;
            continue;
        }
        const int p = f->cur[0];
        if (!f->exec[p]) {
            lbm_status s = capture(f, p);
            if (s) return s;
        }
        CU(cudaGraphLaunch(f->exec[p], f->stream));
        f->cur[0] ^= 1;
    }
    if (n_steps > 0) f->totals_valid = true;
    return LBM_OK;
}

lbm_status lbm_get_macroscopic(lbm_forest* f, int32_t level, double* rho, double* u, int32_t on_device) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    lbm_status s = LBM_OK;
    const Plan& P = f->plan;
    // level -1: every level, level after level, in one array (u components N_all apart)
    const int L0 = level < 0 ? 0 : level, L1 = level < 0 ? P.nlev - 1 : level;
    if (level != -1 && (s = check_level(f, level))) return s;
    int64_t n = 0;
    for (int L = L0; L <= L1; L++) n += owned_cells(f, L);
    if (n == 0) return LBM_OK;
    double *dr = rho, *du = u;
    if (!on_device) {
        if ((s = ensure_stage(f, size_t(n) * 4 * sizeof(double)))) return s;
        double* st = static_cast<double*>(f->d_stage);
        dr = rho ? st : nullptr;
        du = u ? st + n : nullptr;
    }
    int64_t off = 0;
    for (int L = L0; L <= L1; L++) {
        f->L->macro(f->dl[L], f->cur[L], P.LB, f->d_params + L, P.d.rho0, dr ? dr + off : nullptr,
                    du ? du + off : nullptr, n, f->stream);
        off += owned_cells(f, L);
    }
    CU(cudaGetLastError());
    if (!on_device) {
        if (rho) CU(cudaMemcpyAsync(rho, dr, n * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        if (u) CU(cudaMemcpyAsync(u, du, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        CU(cudaStreamSynchronize(f->stream));
    }
    return LBM_OK;
}

lbm_status lbm_get_pdfs(lbm_forest* f, int32_t level, double* pdfs, int32_t on_device) {
    lbm_status s = check_level(f, level);
    if (s) return s;
    if (!pdfs) return fail(LBM_EINVAL, "pdfs is NULL");
    const int64_t n = owned_cells(f, level);
    if (n == 0) return LBM_OK;
    double* d = pdfs;
    if (!on_device) {
        if ((s = ensure_stage(f, size_t(n) * Q * sizeof(double)))) return s;
        d = static_cast<double*>(f->d_stage);
    }
    f->L->get_pdfs(f->dl[level], f->cur[level], f->plan.LB, f->plan.d.rho0, d, f->stream);
    CU(cudaGetLastError());
    if (!on_device) {
        CU(cudaMemcpyAsync(pdfs, d, n * Q * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        CU(cudaStreamSynchronize(f->stream));
    }
    return LBM_OK;
}

lbm_status lbm_set_pdfs(lbm_forest* f, int32_t level, const double* pdfs, int32_t on_device) {
    lbm_status s = check_level(f, level);
    if (s) return s;
    if (!pdfs) return fail(LBM_EINVAL, "pdfs is NULL");
    const int64_t n = owned_cells(f, level);
    const double* d = pdfs;
    if (!on_device && n) {
        if ((s = ensure_stage(f, size_t(n) * Q * sizeof(double)))) return s;
        CU(cudaMemcpyAsync(f->d_stage, pdfs, n * Q * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        d = static_cast<const double*>(f->d_stage);
    }
    f->cur[level] = 0;
    f->L->set_pdfs(f->dl[level], 0, f->plan.LB, f->plan.d.rho0, d, f->stream);
    CU(cudaGetLastError());
    if (!on_device) CU(cudaStreamSynchronize(f->stream));
    f->init_mask |= 1u << level;
    f->totals_valid = false;
    return LBM_OK;
}

lbm_status lbm_reduce_mass_momentum(lbm_forest* f, double out[4]) {
    if (!f || !out) return fail(LBM_EINVAL, "NULL argument");
    const Plan& P = f->plan;
    int off = 0;
    const bool shifted = P.d.precision != LBM_FP64;
    for (int L = 0; L < P.nlev; L++) {
        const double w = std::ldexp(1.0, -3 * L);
        // the shifted layouts' per-cell offsets: sum_a f^eq_a(rho0, u0) = rho0 and sum_a e_a
        // f^eq_a(rho0, u0) = rho0 u0
        const double nf = shifted ? P.d.rho0 * double(P.lv[L].nfluid) : 0.0;
        const double shift[4] = {nf, nf * f->u0[0], nf * f->u0[1], nf * f->u0[2]};
        if (f->totals_valid)   // the step recorded the moments of this state: sum them
            f->L->totals(f->buf[L].wpart, f->tot_warps[L], w, shift, f->d_partial + 4 * off, f->red_grid[L],
                         f->stream);
        else
            f->L->reduce(f->dl[L], f->cur[L], P.LB, f->d_params + L, P.d.rho0, w, f->d_partial + 4 * off,
                         f->red_grid[L], f->stream);
        off += f->red_grid[L];
    }
    reduce_final_kernel<<<1, 256, 0, f->stream>>>(f->d_partial, f->red_total, f->d_out);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(f->h_out, f->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    CU(cudaStreamSynchronize(f->stream));
    for (int k = 0; k < 4; k++) out[k] = f->h_out[k];
    for (int k = 0; k < 4; k++)
        if (!std::isfinite(out[k])) return fail(LBM_ENONFINITE, "non-finite total (component %d)", k);
    return LBM_OK;
}

lbm_status lbm_probe_fp64_fma(int32_t reps, double* gfma, void* stream) {
    if (!gfma || reps < 1) return fail(LBM_EINVAL, "invalid argument");
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = sms * 8, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fp64_fma_probe_kernel<<<grid, 256, 0, s>>>(iters);   // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; r++) fp64_fma_probe_kernel<<<grid, 256, 0, s>>>(iters);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return fail(LBM_ECUDA, "FP64 probe failed: %s", cudaGetErrorString(err));
    const double fmas = double(reps) * grid * 256.0 * iters * kProbeChains;
    *gfma = fmas / (double(ms) * 1e-3) / 1e9;
    return LBM_OK;
}

lbm_status lbm_velocity_residual(lbm_forest* f, double* r) {
    if (!f || !r) return fail(LBM_EINVAL, "NULL argument");
    if (!f->params_set || f->init_mask != (1u << f->plan.nlev) - 1)
        return fail(LBM_EINVAL, "set the level parameters and initialise every level first");
    const Plan& P = f->plan;
    constexpr int G = 128;
    if (!f->d_rpart && !f->mem.get(&f->d_rpart, size_t(P.nlev) * G * 4 * sizeof(double)))
        return fail(LBM_ENOMEM, "cannot allocate the residual sums");
    const bool first = f->uprev.empty();
    if (first) f->uprev.assign(P.nlev, nullptr);
    for (int L = 0; L < P.nlev; L++) {
        const int64_t n = owned_cells(f, L);
        double* part = f->d_rpart + size_t(L) * G * 4;
        if (n == 0) {
            CU(cudaMemsetAsync(part, 0, G * 4 * sizeof(double), f->stream));
            continue;
        }
        lbm_status s = ensure_stage(f, size_t(n) * 4 * sizeof(double));
        if (s) return s;
        double* st = static_cast<double*>(f->d_stage);
        if (!f->uprev[L]) {
            // zeroed: the first call's differences are discarded, but must be finite
            if (!f->mem.get(&f->uprev[L], size_t(n) * 3 * sizeof(double)))
                return fail(LBM_ENOMEM, "cannot allocate the residual's velocity history");
            CU(cudaMemsetAsync(f->uprev[L], 0, size_t(n) * 3 * sizeof(double), f->stream));
        }
        f->L->macro(f->dl[L], f->cur[L], P.LB, f->d_params + L, P.d.rho0, st, st + n, n, f->stream);
        residual_kernel<<<G, 256, 0, f->stream>>>(st + n, f->uprev[L], f->dl[L].cell, n, std::ldexp(1.0, -3 * L), part);
    }
    reduce_final_kernel<<<1, 256, 0, f->stream>>>(f->d_rpart, P.nlev * G, f->d_out);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(f->h_out, f->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    CU(cudaStreamSynchronize(f->stream));
    if (f->h_out[2] > 0.0 || !std::isfinite(f->h_out[0]) || !std::isfinite(f->h_out[1]))
        return fail(LBM_ENONFINITE, "non-finite velocity in %.0f fluid cells", f->h_out[2]);
    if (first) *r = HUGE_VAL;
    else *r = f->h_out[1] > 0.0 ? std::sqrt(f->h_out[0] / f->h_out[1]) : 0.0;
    return LBM_OK;
}

lbm_status lbm_set_kernel_config(lbm_forest* f, int32_t cells_per_thread_log2, int32_t ctas_per_sm) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    if (cells_per_thread_log2 < 0 || cells_per_thread_log2 > f->plan.LB)
        return fail(LBM_EINVAL, "cells per thread must be 2^k with 2^k <= B");
    if (ctas_per_sm < 1 || ctas_per_sm > 4) return fail(LBM_EINVAL, "ctas_per_sm must be 1, 2, 3 or 4");
    CU(cudaStreamSynchronize(f->stream));
    free_graphs(f);
    f->lzc = cells_per_thread_log2;
    f->minb = ctas_per_sm;
    return build_schedule(f);
}

lbm_status lbm_get_kernel_config(const lbm_forest* f, int32_t* cells_per_thread_log2, int32_t* ctas_per_sm) {
    if (!f || !cells_per_thread_log2 || !ctas_per_sm) return fail(LBM_EINVAL, "NULL argument");
    *cells_per_thread_log2 = f->lzc;
    *ctas_per_sm = f->minb;
    return LBM_OK;
}

lbm_status lbm_timing_begin(lbm_forest* f, int32_t max_steps) {
    if (!f || max_steps < 0) return fail(LBM_EINVAL, "invalid argument");
    free_timing(f);
    const size_t ne = f->sched.size() + 1;
    f->tev.resize(size_t(max_steps) * ne);
    for (auto& e : f->tev) CU(cudaEventCreate(&e));
    f->tmax = max_steps;
    f->tused = 0;
    f->timing = true;
    return LBM_OK;
}

lbm_status lbm_timing_end(lbm_forest* f, double* ms_per_level, int64_t* launches_per_level, double* ms_explode,
                          int64_t* launches_explode, double* ms_side, int64_t* launches_side) {
    if (!f) return fail(LBM_EINVAL, "forest is NULL");
    CU(cudaStreamSynchronize(f->stream));
    const int n = f->plan.nlev;
    std::vector<double> ms(3 * n, 0.0);
    std::vector<int64_t> cnt(3 * n, 0);
    const size_t ne = f->sched.size() + 1;
    for (int r = 0; r < f->tused; r++)
        for (size_t k = 0; k + 1 < ne; k++) {
            const Launch& l = f->sched[k];
            if (l.grid <= 0) continue;
            float t = 0.f;
            CU(cudaEventElapsedTime(&t, f->tev[r * ne + k], f->tev[r * ne + k + 1]));
            ms[3 * l.level + l.type] += t;
            cnt[3 * l.level + l.type] += 1;
        }
    for (int L = 0; L < n; L++) {
        if (ms_per_level) ms_per_level[L] = ms[3 * L];
        if (launches_per_level) launches_per_level[L] = cnt[3 * L];
        if (ms_explode) ms_explode[L] = ms[3 * L + 1];
        if (launches_explode) launches_explode[L] = cnt[3 * L + 1];
        if (ms_side) ms_side[L] = ms[3 * L + 2];
        if (launches_side) launches_side[L] = cnt[3 * L + 2];
    }
    free_timing(f);
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ kernel-config autotuning
namespace {

// Device copy of every level's two PDF grids and the parities, so that tuning runs leave the
// state as they found it.
struct Snapshot {
    std::vector<void*> bufs;
    std::vector<DevMem*> owner;   // the forest whose memory each buffer came from
    std::vector<std::vector<int>> cur;
};

lbm_status take_snapshot(const std::vector<lbm_forest*>& fs, cudaStream_t s, Snapshot& sn) {
    for (lbm_forest* f : fs) {
        sn.cur.emplace_back(f->cur, f->cur + LBM_MAX_LEVELS);
        for (int L = 0; L < f->plan.nlev; L++) {
            const size_t bytes = size_t(f->dl[L].ncells) * Q * f->esize;
            for (int k = 0; k < 2; k++) {
                void* p = nullptr;
                if (!f->mem.get(&p, bytes)) return fail(LBM_ENOMEM, "cannot allocate the autotuning snapshot");
                sn.bufs.push_back(p);
                sn.owner.push_back(&f->mem);
                if (bytes) CU(cudaMemcpyAsync(p, f->dl[L].f[k], bytes, cudaMemcpyDeviceToDevice, s));
            }
        }
    }
    return LBM_OK;
}

lbm_status restore_snapshot(const std::vector<lbm_forest*>& fs, cudaStream_t s, Snapshot& sn) {
    size_t k = 0;
    for (size_t i = 0; i < fs.size(); i++) {
        lbm_forest* f = fs[i];
        std::copy(sn.cur[i].begin(), sn.cur[i].end(), f->cur);
        for (int L = 0; L < f->plan.nlev; L++) {
            const size_t bytes = size_t(f->dl[L].ncells) * Q * f->esize;
            for (int g = 0; g < 2; g++, k++)
                if (bytes) CU(cudaMemcpyAsync(f->dl[L].f[g], sn.bufs[k], bytes, cudaMemcpyDeviceToDevice, s));
        }
    }
    CU(cudaStreamSynchronize(s));
    return LBM_OK;
}

void free_snapshot(Snapshot& sn) {
    for (size_t k = 0; k < sn.bufs.size(); k++) sn.owner[k]->put(sn.bufs[k]);
    sn.bufs.clear();
    sn.owner.clear();
}

// Times n_steps of `step` for every (cells per thread, CTAs per SM) the kernels support and
// keeps the fastest; `config` applies one.  Results do not depend on the configuration.
template <typename Config, typename Step>
lbm_status tune(const std::vector<lbm_forest*>& fs, cudaStream_t s, int LB, int n_steps, Config config, Step step,
                int32_t* best_lzc, int32_t* best_minb, double* best_ms) {
    Snapshot sn;
    lbm_status st = take_snapshot(fs, s, sn);
    if (st) {
        free_snapshot(sn);
        return st;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 1e300;
    int bl = LB - 3 > 0 ? LB - 3 : 0, bm = 3;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = fail(LBM_ECUDA, "cudaEventCreate failed");
    for (int lzc = 0; lzc <= LB && !st; lzc++)
        for (int minb = 1; minb <= 4 && !st; minb++) {
            if ((st = config(lzc, minb)) || (st = step(1))) break;   // the first step captures the graphs
            if (cudaEventRecord(e0, s) != cudaSuccess) st = fail(LBM_ECUDA, "cudaEventRecord failed");
            if (!st) st = step(n_steps);
            if (!st && cudaEventRecord(e1, s) != cudaSuccess) st = fail(LBM_ECUDA, "cudaEventRecord failed");
            float ms = 0.f;
            if (!st && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = fail(LBM_ECUDA, "timing a configuration failed");
            if (!st && ms / n_steps < best) {
                best = ms / n_steps;
                bl = lzc;
                bm = minb;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lbm_status rs = restore_snapshot(fs, s, sn);
    for (lbm_forest* f : fs) f->totals_valid = false;
    free_snapshot(sn);
    if (st) return st;
    if (rs) return rs;
    if ((st = config(bl, bm))) return st;
    if (best_lzc) *best_lzc = bl;
    if (best_minb) *best_minb = bm;
    if (best_ms) *best_ms = best;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_autotune(lbm_forest* f, int32_t n_steps, int32_t* cells_per_thread_log2, int32_t* ctas_per_sm,
                                   double* ms_per_step) {
    if (!f || n_steps < 1) return fail(LBM_EINVAL, "invalid argument");
    if (!f->params_set || f->init_mask != (1u << f->plan.nlev) - 1)
        return fail(LBM_EINVAL, "set the level parameters and initialise every level before tuning");
    if (f->timing) return fail(LBM_EINVAL, "timing is active");
    return tune(
        {f}, f->stream, f->plan.LB, n_steps, [&](int l, int m) { return lbm_set_kernel_config(f, l, m); },
        [&](int n) { return lbm_step_coarse(f, n); }, cells_per_thread_log2, ctas_per_sm, ms_per_step);
}

extern "C" lbm_status lbm_autotune_block_size(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag,
                                              void* user, double lambda_e0, double magic_lambda, const double accel0[3],
                                              void* stream, const lbm_allocator* alloc, int32_t n_steps,
                                              int32_t* block_cells, double ms_per_step[3]) {
    if (!d || !block_cells || n_steps < 1) return fail(LBM_EINVAL, "invalid argument");
    if (refine) return fail(LBM_EINVAL, "a refine callback takes block coordinates, which depend on the block size");
    double ms[3] = {-1.0, -1.0, -1.0};
    int best = -1;
    std::string last;
    for (int k = 0; k < 3; k++) {
        const int B = 8 << k;
        lbm_forest_desc e = *d;
        bool fits = true;
        for (int a = 0; a < 3; a++) {
            const int64_t N = int64_t(d->root_blocks[a]) * d->block_cells;
            fits = fits && N % B == 0;
            e.root_blocks[a] = int32_t(N / B);
        }
        if (!fits) continue;
        e.block_cells = B;
        lbm_forest* f = nullptr;
        lbm_status st = lbm_create_forest(&e, nullptr, flag, user, stream, alloc, &f);
        if (!st) st = lbm_set_level_params(f, lambda_e0, magic_lambda, accel0);
        if (!st) st = lbm_init_equilibrium(f, -1, nullptr, nullptr, 0);
        double t = 0.0;
        if (!st) st = lbm_autotune(f, n_steps, nullptr, nullptr, &t);
        if (st) last = g_err;
        lbm_destroy(f);
        if (st == LBM_ECUDA || st == LBM_ETIMEOUT) return fail(st, "block size %d: %s", B, last.c_str());
        if (st) continue;
        ms[k] = t;
        if (best < 0 || t < ms[best]) best = k;
    }
    if (ms_per_step)
        for (int k = 0; k < 3; k++) ms_per_step[k] = ms[k];
    if (best < 0) return fail(LBM_EINVAL, "no block size could be built%s%s", last.empty() ? "" : ": ", last.c_str());
    *block_cells = 8 << best;
    return LBM_OK;
}

// ------------------------------------------------------------------ batches of forests
namespace {

struct BatchPhase {
    int level, substep, type;   // type 0: stream-collide F_L(substep), 1: explosion E_L, 2: side work
    int n = 0, total = 0, grid = 0;
    StepArgs* args[2] = {nullptr, nullptr};   // per level-0 parity
    int* prefix = nullptr;
};

}  // namespace

struct lbm_batch {
    std::vector<lbm_forest*> fs;
    int* d_wq = nullptr;   // work counters of the persistent walk phases, 2 per (phase, member)
    cudaStream_t stream = nullptr, cap = nullptr;
    const Launchers* L = nullptr;
    int nlev = 0, LB = 0, collision = 0, sms = 152;
    int lzc = 2, minb = 3;
    std::vector<BatchPhase> phases;
    cudaGraphExec_t exec[2] = {};
    int64_t updates = 0;
    DevMem mem;            // device memory: the caller's allocator hook or cudaMalloc
};

namespace {

void free_phases(lbm_batch* b) {
    for (int p = 0; p < 2; p++) {
        if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
        b->exec[p] = nullptr;
    }
    for (BatchPhase& ph : b->phases) {
        b->mem.put(ph.args[0]);
        b->mem.put(ph.args[1]);
        b->mem.put(ph.prefix);
    }
    b->phases.clear();
    b->mem.put(b->d_wq);
    b->d_wq = nullptr;
}

// The phase list of one coarse step: Alg. 1 over the deepest member; a member without level L has
// no work in the phases of level L.  Each phase holds, per member with work, the launch arguments
// and grid of the member's own launch, for both level-0 parities.
lbm_status build_phases(lbm_batch* b) {
    free_phases(b);
    const int B = 1 << b->LB;
    // cells per thread per level: the largest up to the configured bound that gives about four
    // waves of CTAs over the whole batch
    std::vector<int> lzc(b->nlev);
    const int resident = b->sms * b->L->ctas_per_sm(b->LB, b->minb);
    for (int L = 0; L < b->nlev; L++) {
        int64_t bricks = 0;
        for (lbm_forest* f : b->fs)
            if (L < f->plan.nlev) bricks += f->plan.lv[L].nown;
        int z = b->lzc;
        while (z > 0 && bricks * B * B * (B >> z) / 256 < int64_t(4) * b->sms * b->minb) z--;
        lzc[L] = z;
    }
    std::vector<std::pair<int, int>> order0;   // (level, substep), substep 0 = explosion
    std::function<void(int)> rec = [&](int L) {
        if (L == 0) {
            if (b->nlev > 1) rec(1);
            order0.push_back({0, 1});
            return;
        }
        order0.push_back({L, 0});
        if (L + 1 < b->nlev) rec(L + 1);
        order0.push_back({L, 1});
        if (L + 1 < b->nlev) rec(L + 1);
        order0.push_back({L, 2});
    };
    rec(0);
    // phases (level, substep, type): a persistent walk's coupled cells and ghost work go first
    struct Ph {
        int first, second, type;
    };
    std::vector<Ph> order;
    for (const auto& o : order0) {
        if (o.second != 0 && b->L->persistent) order.push_back({o.first, o.second, 2});
        order.push_back({o.first, o.second, o.second == 0 ? 1 : 0});
    }
    std::vector<std::vector<StepArgs>> hargs[2];
    std::vector<std::vector<int>> hprefix;
    for (int p = 0; p < 2; p++) {
        std::vector<std::vector<int>> cur(b->fs.size());
        for (size_t i = 0; i < b->fs.size(); i++) {
            cur[i].assign(b->fs[i]->cur, b->fs[i]->cur + LBM_MAX_LEVELS);
            cur[i][0] = p;
        }
        for (const auto& o : order) {
            const int L = o.first, s = o.second;
            std::vector<StepArgs> args;
            std::vector<int> prefix{0};
            for (size_t i = 0; i < b->fs.size(); i++) {
                lbm_forest* f = b->fs[i];
                if (L >= f->plan.nlev) continue;
                const HostLevel& V = f->plan.lv[L];
                int grid, wctas = 0, zlb = lzc[L];
                if (s == 0) {
                    grid = int((V.ework.size() / 4 + 255) / 256);
                } else if (b->L->persistent) {
                    wctas = walk_ctas(V.nown, B, resident);
                    zlb = chunk_planes_log2(V.nown, b->LB, wctas);
                    grid = o.type == 2 ? int((V.cwork.size() + 255) / 256) + int((V.gwork[s - 1].size() / 4 + 255) / 256)
                                       : wctas;
                } else {
                    const int64_t units = int64_t(V.nown) * B * B * (B >> lzc[L]);
                    grid = int((units + 255) / 256) + int((V.gwork[s - 1].size() / 4 + 255) / 256) +
                           int((V.cwork.size() + 255) / 256);
                }
                if (grid > 0) {
                    Launch l{L, s == 0 ? 0 : s, grid, o.type, zlb, 0, wctas};
                    args.push_back(make_args(f, l, cur[i].data()));
                    prefix.push_back(prefix.back() + grid);
                }
                if (o.type == 0) cur[i][L] ^= 1;
            }
            hargs[p].push_back(args);
            if (p == 0) hprefix.push_back(prefix);
        }
    }
    // work counters: 2 per (walk phase, member), the same for both parities (phases run in order)
    size_t nwq = 0;
    for (size_t k = 0; k < order.size(); k++)
        if (order[k].type == 0) nwq += hargs[0][k].size();
    if (b->L->persistent && nwq > 0) {
        if (!b->mem.get(&b->d_wq, 2 * nwq * sizeof(int)))
            return fail(LBM_ENOMEM, "cannot allocate the batch's work counters");
        CU(cudaMemset(b->d_wq, 0, 2 * nwq * sizeof(int)));
        size_t slot = 0;
        for (size_t k = 0; k < order.size(); k++) {
            if (order[k].type != 0) continue;
            for (size_t i = 0; i < hargs[0][k].size(); i++, slot++) {
                hargs[0][k][i].wq = b->d_wq + 2 * slot;
                hargs[1][k][i].wq = b->d_wq + 2 * slot;
            }
        }
    }
    for (size_t k = 0; k < order.size(); k++) {
        BatchPhase ph;
        ph.level = order[k].first;
        ph.substep = order[k].second;
        ph.type = order[k].type;
        ph.n = int(hargs[0][k].size());
        ph.total = hprefix[k].back();
        const int slots = b->sms * (ph.type == 0 ? b->L->ctas_per_sm(b->LB, b->minb) : 8);
        ph.grid = std::min(ph.total, slots);
        b->phases.push_back(ph);
        BatchPhase& q = b->phases.back();
        if (ph.n == 0) continue;
        lbm_status st;
        if ((st = upload(b->mem, &q.args[0], hargs[0][k])) || (st = upload(b->mem, &q.args[1], hargs[1][k])) ||
            (st = upload(b->mem, &q.prefix, hprefix[k])))
            return st;
    }
    return LBM_OK;
}

lbm_status capture_batch(lbm_batch* b, int parity) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    for (const BatchPhase& ph : b->phases) {
        if (ph.n == 0) continue;
        if (ph.type == 1) b->L->explode_batch(ph.args[parity], ph.prefix, ph.n, ph.total, ph.grid, b->cap);
        else if (ph.type == 2) b->L->side_batch(ph.args[parity], ph.prefix, ph.n, ph.total, ph.grid, b->collision, b->LB, b->cap);
        else b->L->step_batch(ph.args[parity], ph.prefix, ph.n, ph.total, ph.grid, b->collision, b->LB, b->minb, b->cap);
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(LBM_ECUDA, "batch capture failed: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaError_t ie = cudaGraphInstantiate(&b->exec[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(LBM_ECUDA, "batch graph instantiation failed: %s", cudaGetErrorString(ie));
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    if (b->stream || b->cap) cudaStreamSynchronize(b->stream);
    free_phases(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return LBM_OK;
}

lbm_status lbm_batch_create(lbm_forest* const* forests, int32_t n, const lbm_allocator* alloc, lbm_batch** out) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!forests || n < 1) return fail(LBM_EINVAL, "a batch needs at least one forest");
    lbm_batch* b = new (std::nothrow) lbm_batch;
    if (!b) return fail(LBM_ENOMEM, "host allocation failed");
    const lbm_forest* f0 = forests[0];
    for (int i = 0; i < n; i++) {
        const lbm_forest* f = forests[i];
        if (!f) {
            delete b;
            return fail(LBM_EINVAL, "forest %d is NULL", i);
        }
        if (f->plan.d.precision != f0->plan.d.precision || f->plan.d.collision != f0->plan.d.collision ||
            f->plan.B != f0->plan.B || f->stream != f0->stream) {
            delete b;
            return fail(LBM_EINVAL, "forest %d differs from forest 0 in precision, collision, block size or stream", i);
        }
        for (int j = 0; j < i; j++)
            if (forests[j] == f) {
                delete b;
                return fail(LBM_EINVAL, "forest %d appears twice", i);
            }
        b->fs.push_back(const_cast<lbm_forest*>(f));
        b->nlev = std::max(b->nlev, f->plan.nlev);
        b->updates += f->updates;
    }
    b->stream = f0->stream;
    if (!b->mem.bind(alloc, b->stream)) {
        delete b;
        return fail(LBM_EINVAL, "an allocator hook with alloc needs release");
    }
    b->L = f0->L;
    b->LB = f0->plan.LB;
    b->collision = f0->plan.d.collision;
    b->lzc = std::max(0, b->LB - 3);
    b->minb = f0->plan.d.precision == LBM_FP64 ? 3 : 2;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return fail(LBM_ECUDA, "cannot create the capture stream");
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_set_kernel_config(lbm_batch* b, int32_t cells_per_thread_log2, int32_t ctas_per_sm) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (cells_per_thread_log2 < 0 || cells_per_thread_log2 > b->LB)
        return fail(LBM_EINVAL, "cells per thread must be 2^k with 2^k <= B");
    if (ctas_per_sm < 1 || ctas_per_sm > 4) return fail(LBM_EINVAL, "ctas_per_sm must be 1, 2, 3 or 4");
    CU(cudaStreamSynchronize(b->stream));
    free_phases(b);
    b->lzc = cells_per_thread_log2;
    b->minb = ctas_per_sm;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int32_t n_steps) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (n_steps < 0) return fail(LBM_EINVAL, "negative step count");
    const lbm_forest* f0 = b->fs[0];
    for (size_t i = 0; i < b->fs.size(); i++) {
        const lbm_forest* f = b->fs[i];
        if (!f->params_set || f->init_mask != (1u << f->plan.nlev) - 1)
            return fail(LBM_EINVAL, "forest %d: set the level parameters and initialise every level", int(i));
        if (f->timing) return fail(LBM_EINVAL, "forest %d: timing is active", int(i));
        for (int L = 0; L < std::min(f->plan.nlev, f0->plan.nlev); L++)
            if (f->cur[L] != f0->cur[L])
                return fail(LBM_EINVAL, "forest %d is not at the two-grid parity of forest 0 (step members together)", int(i));
        for (int L = f0->plan.nlev; L < f->plan.nlev; L++)
            if (f->cur[L] != 0) return fail(LBM_EINVAL, "forest %d has an unexpected parity on level %d", int(i), L);
    }
    if (b->phases.empty()) {
        lbm_status s = build_phases(b);
        if (s) return s;
    }
    for (int k = 0; k < n_steps; k++) {
        const int p = b->fs[0]->cur[0];
        if (!b->exec[p]) {
            lbm_status s = capture_batch(b, p);
            if (s) return s;
        }
        CU(cudaGraphLaunch(b->exec[p], b->stream));
        for (lbm_forest* f : b->fs) {
            f->cur[0] ^= 1;
            f->totals_valid = false;   // batched launches record no totals
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_cell_updates_per_coarse_step(const lbm_batch* b, int64_t* n) {
    if (!b || !n) return fail(LBM_EINVAL, "NULL argument");
    *n = b->updates;
    return LBM_OK;
}

lbm_status lbm_batch_launches_per_coarse_step(const lbm_batch* b, int32_t* n) {
    if (!b || !n) return fail(LBM_EINVAL, "NULL argument");
    if (b->phases.empty()) {
        lbm_status s = build_phases(const_cast<lbm_batch*>(b));
        if (s) return s;
    }
    int c = 0;
    for (const BatchPhase& ph : b->phases) c += ph.n > 0;
    *n = c;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t n_steps, int32_t* cells_per_thread_log2, int32_t* ctas_per_sm,
                              double* ms_per_step) {
    if (!b || n_steps < 1) return fail(LBM_EINVAL, "invalid argument");
    return tune(
        b->fs, b->stream, b->LB, n_steps, [&](int l, int m) { return lbm_batch_set_kernel_config(b, l, m); },
        [&](int n) { return lbm_batch_step(b, n); }, cells_per_thread_log2, ctas_per_sm, ms_per_step);
}

}  // extern "C"
