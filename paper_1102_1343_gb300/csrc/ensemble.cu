// Batched ensemble of independent fire runs (members of different mesh
// sizes, fuels, winds) advanced together by ONE persistent cooperative
// launch per call: the kernel loops over the steps, and within a step over
// a work list of (member, strip) items handed out round-robin to the
// resident CTAs; a grid-wide barrier separates the steps.  Each member is an
// ordinary fire context (same state layout, same marching-strip device code
// as fire_step), so a member advanced here matches the same member advanced
// alone.  The launch (with the reset of the barrier word) is captured in a
// CUDA graph and replayed while its arguments do not change.
//
// Two forms of the persistent kernel: FP32 ensembles run the warp-strip code
// of k_fire_warp, one (member, strip) item per warp, each warp loading its
// member's class table and wind-row weights into its own slice of shared
// memory; FP64 ensembles (or refinements above 30) run the marching-strip
// code of k_fire_march, one item per CTA.
//
// The barrier's wait is bounded: a CTA that waits longer than the spin limit
// sets the ensemble's TIMEOUT bit and an abort flag, and every CTA leaves the
// kernel at its next barrier, so a lost CTA ends the launch with an error
// instead of hanging the device.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "fire_internal.h"
#include "march_kernel.cuh"
#include "warp_kernel.cuh"

using namespace wf;

namespace {

struct EnsItem {
    int member, x0, y0;
};

struct GridBar {
    unsigned int count;
    unsigned int gen;
    int abort;
    unsigned int next[2];  // work-item counters of alternate steps
    int status;            // ensemble-wide status bits (TIMEOUT)
};

// values that change from call to call, read by the kernel from device memory
// so that a captured launch can be replayed
struct EnsRun {
    double t0;
    int parity0;
    int nsteps;
    long long spin_limit;
    int skip_block;  // test hook: this CTA never arrives at a barrier (-1: none)
};

struct EnsembleArgs {
    const StepArgs *margs;  // [2 * n_members]: parity 0 and 1 of each member
    const EnsItem *items;
    int n_items;
    int n_members;
    double dt;
    GridBar *bar;
    const EnsRun *run;
};

// grid-wide barrier with a bounded wait; returns false when the launch must end
__device__ bool grid_barrier(GridBar *b, long long spin_limit, bool skip) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile GridBar *vb = b;
        bool ok = vb->abort == 0;
        if (ok && !skip) {
            const unsigned int g = vb->gen;
            __threadfence();
            const unsigned int arrived = atomicAdd(&b->count, 1u);
            if (arrived == gridDim.x - 1) {
                b->count = 0;
                __threadfence();
                atomicAdd(&b->gen, 1u);
            } else {
                long long it = 0;
                while (vb->gen == g) {
                    if (vb->abort) {
                        ok = false;
                        break;
                    }
                    if (++it > spin_limit) {
                        atomicOr(&b->status, ST_TIMEOUT);
                        atomicExch(&b->abort, 1);
                        ok = false;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T, bool NC>
__global__ void __launch_bounds__(kMarchThreads, MarchOccupancy<T>::blocks)
    k_fire_ensemble(const EnsembleArgs e) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const EnsRun run = *e.run;
    double t = run.t0;
    __shared__ int s_item;
    for (int s = 0; s < run.nsteps; ++s) {
        const int par = (run.parity0 + s) & 1;
        // the counter of the next step was last used two steps ago
        if (blockIdx.x == 0 && threadIdx.x == 0) e.bar->next[(s + 1) & 1] = 0;
        for (;;) {
            // items are taken dynamically, largest first (the list is sorted)
            if (threadIdx.x == 0) s_item = (int)atomicAdd(&e.bar->next[s & 1], 1u);
            __syncthreads();
            const int i = s_item;
            __syncthreads();
            if (i >= e.n_items) break;
            const EnsItem it = e.items[i];
            const StepArgs &a = e.margs[2 * it.member + par];
            MarchSmem<T> sm;
            sm.carve(dyn_smem, a.ky * a.sry, a.ncls);
            MarchStrip<T, NC> strip(a, sm);
            strip.run(it.x0, it.y0, t);
            if (strip.st) atomicOr(a.status, strip.st);
            __syncthreads();  // shared memory is reused by the next item
        }
        t = t + e.dt;
        if (s + 1 < run.nsteps) {
            const bool skip = (int)blockIdx.x == run.skip_block;
            if (!grid_barrier(e.bar, run.spin_limit, skip)) return;
        }
    }
    // the members' device time after the last step
    if (blockIdx.x == 0) {
        const int pf = (run.parity0 + run.nsteps) & 1;
        for (int m = threadIdx.x; m < e.n_members; m += blockDim.x)
            *const_cast<double *>(e.margs[2 * m + pf].t_in) = t;
    }
}

// dynamic shared memory of the warp form: per warp a class table, the same
// coefficients doubled for pair loads, the Hq column, heat column sums and
// the wind-row weights of up to max_rows + 4 rows
template <typename T>
__host__ __device__ size_t ens_warp_slice(int max_rows) {
    size_t b = (size_t)FIRE_MAX_CLASSES * 21 * sizeof(T) + 128 * sizeof(T);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)(max_rows + 4) * sizeof(WRow<T>);
    return (b + 15) & ~(size_t)15;
}

template <typename T, bool NC>
__global__ void __launch_bounds__(kWarpCtaThreads, WOcc<T>::blocks)
    k_fire_ensemble_warp(const EnsembleArgs e, int max_rows) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *slice = dyn_smem + (size_t)warp * ens_warp_slice<T>(max_rows);
    T *lut = reinterpret_cast<T *>(slice);
    T *lut2 = lut + FIRE_MAX_CLASSES * 8;
    T *lutq = lut2 + FIRE_MAX_CLASSES * 12;
    T *hw = lutq + FIRE_MAX_CLASSES;
    WRow<T> *rows = reinterpret_cast<WRow<T> *>(
        slice + (((size_t)FIRE_MAX_CLASSES * 21 + 128) * sizeof(T) + 15 & ~(size_t)15));
    const EnsRun run = *e.run;
    double t = run.t0;
    for (int s = 0; s < run.nsteps; ++s) {
        const int par = (run.parity0 + s) & 1;
        // the counter of the next step was last used two steps ago
        if (blockIdx.x == 0 && threadIdx.x == 0) e.bar->next[(s + 1) & 1] = 0;
        for (;;) {
            // items are taken dynamically, largest first (the list is sorted)
            int i = 0;
            if (lane == 0) i = (int)atomicAdd(&e.bar->next[s & 1], 1u);
            i = __shfl_sync(0xffffffffu, i, 0);
            if (i >= e.n_items) break;
            const EnsItem it = e.items[i];
            const StepArgs &a = e.margs[2 * it.member + par];
            // the member's class table and the wind-row weights of the strip
            for (int k = lane; k < a.ncls; k += 32) {
                const double *co = a.coef + (size_t)k * K_N;
                T *l = lut + k * 8;
                l[0] = T(co[K_S0]);
                l[1] = T(co[K_R0]);
                l[2] = T(co[K_B]);
                l[3] = T(co[K_C]);
                l[4] = T(co[K_D]);
                l[5] = T(co[K_E]);
                l[6] = T(co[K_TF]);
                l[7] = T(co[K_HS]);
                lutq[k] = T(co[K_HQ]);
                T *l2 = lut2 + k * 12;
                for (int j = 0; j < 6; ++j) l2[2 * j] = l2[2 * j + 1] = l[j];
            }
            const int La = min(a.ky * a.sry, a.ny - it.y0);
            for (int q = lane; q < La + 4; q += 32) {
                const int r = it.y0 - 2 + q;
                WRow<T> w;
                w.ju0 = w.jv0 = 0;
                w.wyu = w.wyv = T(0);
                if (r >= 0 && r < a.ny) {
                    int j1;
                    const T yr = (T(r) + T(0.5)) / T(a.sry);
                    lin_idx<T>(yr - T(0.5), a.nya, w.ju0, j1, w.wyu);
                    lin_idx<T>(yr, a.nya + 1, w.jv0, j1, w.wyv);
                }
                rows[q] = w;
            }
            __syncwarp();
            WarpStrip<T, NC> strip(a, lut, lut2, lutq, hw, rows);
            strip.run(it.x0, it.y0, t);
            const int stw = __reduce_or_sync(0xffffffffu, strip.st);
            if (lane == 0 && stw) atomicOr(a.status, stw);
            __syncwarp();  // the slice is reused by the next item
        }
        t = t + e.dt;
        if (s + 1 < run.nsteps) {
            const bool skip = (int)blockIdx.x == run.skip_block;
            if (!grid_barrier(e.bar, run.spin_limit, skip)) return;
        }
    }
    if (blockIdx.x == 0) {
        const int pf = (run.parity0 + run.nsteps) & 1;
        for (int m = threadIdx.x; m < e.n_members; m += blockDim.x)
            *const_cast<double *>(e.margs[2 * m + pf].t_in) = t;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// members are ordinary contexts: the accessors below are defined in context.cu
namespace wf {
int ctx_step_args(fire_ctx *c, int parity, const void *u, const void *v, double dt, double *hs,
                  double *hl, StepArgs &a);
int ctx_info(const fire_ctx *c, int *prec, int *variant, int *nx, int *ny, int *srx, int *sry,
             int *kx, int *ky, int *ncls, int *cur, double *t);
int ctx_advance(fire_ctx *c, int nsteps, double dt);
bool ctx_ignition_active(fire_ctx *c, double t);
cudaStream_t ctx_stream(const fire_ctx *c);
int ctx_workspace(fire_ctx *c, size_t bytes, void **out);
int ctx_default_march(fire_ctx *c);
int ctx_default_warp_strips(fire_ctx *c);
int ctx_ensure_node_coefficients(fire_ctx *c);
bool ctx_has_node_coefficients(const fire_ctx *c);
}  // namespace wf

struct fire_ensemble {
    std::vector<fire_ctx *> members;
    int n = 0;
    int device = 0;  // the device current at fire_ensemble_create (its members')
    int prec = FIRE_FP32;
    cudaStream_t stream = nullptr;
    StepArgs *margs_dev = nullptr;
    StepArgs *margs_host = nullptr;  // pinned
    EnsItem *items_dev = nullptr;
    int n_items = 0;
    GridBar *bar = nullptr;
    EnsRun *run_dev = nullptr;
    EnsRun *run_host = nullptr;  // pinned
    cudaEvent_t staged = nullptr;  // the pinned staging buffers may be rewritten
    int grid = 0;
    size_t smem = 0;
    long long spin_limit = 20000000;  // x ~100 ns: about 2 s
    int skip_block = -1;
    cudaGraphExec_t graph = nullptr;
    bool capture_failed = false;
    int variant = FIRE_KERNEL_MARCH;  // member kernel: FIRE_KERNEL_MARCH or FIRE_KERNEL_WARP
    bool nc = false;  // members carry per-node coefficients (a per-node fuel moisture)
    int max_rows = 0;                 // warp form: tallest strip
    int g_nsteps = -1;
    double g_dt = 0;
    int g_grid = 0;
    size_t g_smem = 0;
    const void *g_first_u = nullptr;
};

namespace {

int ens_cuda_at(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return FIRE_OK;
    record_cuda_error(e, where);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FIRE_ERR_OOM;
    }
    return FIRE_ERR_CUDA;
}

#define ens_cuda(call) ens_cuda_at((call), #call)
#define ENS_CHECK(call)                   \
    do {                                  \
        int _r = ens_cuda(call);          \
        if (_r != FIRE_OK) return _r;     \
    } while (0)

void ens_release(fire_ensemble *e) {
    if (!e) return;
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->staged) cudaEventDestroy(e->staged);
    for (fire_ctx *c : e->members) fire_destroy(c);
    if (e->margs_dev) cudaFree(e->margs_dev);
    if (e->items_dev) cudaFree(e->items_dev);
    if (e->bar) cudaFree(e->bar);
    if (e->run_dev) cudaFree(e->run_dev);
    if (e->margs_host) cudaFreeHost(e->margs_host);
    if (e->run_host) cudaFreeHost(e->run_host);
    delete e;
}

// work list and launch shape for the members' current kernel configuration
int ens_plan(fire_ensemble *e) {
    // a captured launch holds the old work list (pointer and length): drop
    // it, after the stream has finished with it, before the list is replaced
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    std::vector<EnsItem> items;
    size_t smem = 0;
    int max_rows = 0;
    for (int m = 0; m < e->n; ++m) {
        int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
        double t;
        ctx_info(e->members[m], &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t);
        if (variant != e->variant) return FIRE_ERR_STATE;
        const int W = kx * srx, L = ky * sry;
        for (int y0 = 0; y0 < ny; y0 += L)
            for (int x0 = 0; x0 < nx; x0 += W) items.push_back(EnsItem{m, x0, y0});
        if (e->variant == FIRE_KERNEL_MARCH) {
            const size_t sm = e->prec == FIRE_FP64 ? march_smem_bytes<double>(ky, sry, ncls)
                                                   : march_smem_bytes<float>(ky, sry, ncls);
            smem = std::max(smem, sm);
        }
        max_rows = std::max(max_rows, L);
    }
    if (e->variant == FIRE_KERNEL_WARP)
        smem = kWarpStrips * (e->prec == FIRE_FP64 ? ens_warp_slice<double>(max_rows)
                                                   : ens_warp_slice<float>(max_rows));
    // largest items first (the kernel hands them out dynamically), then by
    // row and member
    std::vector<long long> cost(items.size());
    for (size_t q = 0; q < items.size(); ++q) {
        int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
        double t;
        ctx_info(e->members[items[q].member], &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky,
                 &ncls, &cur, &t);
        cost[q] = (long long)std::min(kx * srx, nx - items[q].x0) * std::min(ky * sry, ny - items[q].y0);
    }
    std::vector<size_t> order(items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        if (cost[a] != cost[b]) return cost[a] > cost[b];
        if (items[a].y0 != items[b].y0) return items[a].y0 < items[b].y0;
        return items[a].member < items[b].member;
    });
    {
        std::vector<EnsItem> sorted(items.size());
        for (size_t q = 0; q < order.size(); ++q) sorted[q] = items[order[q]];
        items.swap(sorted);
    }
    if (e->items_dev) cudaFree(e->items_dev);
    e->items_dev = nullptr;
    ENS_CHECK(cudaMalloc(&e->items_dev, sizeof(EnsItem) * items.size()));
    ENS_CHECK(cudaMemcpy(e->items_dev, items.data(), sizeof(EnsItem) * items.size(),
                         cudaMemcpyHostToDevice));
    e->n_items = (int)items.size();
    const void *fn;
    int threads;
    const bool f64 = e->prec == FIRE_FP64;
    if (e->variant == FIRE_KERNEL_WARP) {
        fn = e->nc ? (f64 ? (const void *)k_fire_ensemble_warp<double, true>
                          : (const void *)k_fire_ensemble_warp<float, true>)
                   : (f64 ? (const void *)k_fire_ensemble_warp<double, false>
                          : (const void *)k_fire_ensemble_warp<float, false>);
        threads = kWarpCtaThreads;
    } else {
        fn = e->nc ? (f64 ? (const void *)k_fire_ensemble<double, true>
                          : (const void *)k_fire_ensemble<float, true>)
                   : (f64 ? (const void *)k_fire_ensemble<double, false>
                          : (const void *)k_fire_ensemble<float, false>);
        threads = kMarchThreads;
    }
    {
        // the limit is a property of the kernel function on a device, shared by
        // all ensembles there
        static std::mutex mu;
        static size_t current[kMaxDevices][8] = {};
        std::lock_guard<std::mutex> lock(mu);
        const int dev = attr_device();
        const int form = (f64 ? 1 : 0) + (e->variant == FIRE_KERNEL_WARP ? 2 : 0) + (e->nc ? 4 : 0);
        if (dev < 0 || smem > current[dev][form]) {
            ENS_CHECK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            if (dev >= 0) current[dev][form] = smem;
        }
    }
    int per_sm = 0, dev = 0, sms = 0;
    ENS_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    ENS_CHECK(cudaGetDevice(&dev));
    ENS_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return FIRE_ERR_ARG;
    const int units = e->variant == FIRE_KERNEL_WARP ? (e->n_items + kWarpStrips - 1) / kWarpStrips
                                                     : e->n_items;
    e->grid = std::min(units, per_sm * sms);
    e->smem = smem;
    e->max_rows = max_rows;
    return FIRE_OK;
}

cudaError_t ens_launch(fire_ensemble *e, double dt, cudaStream_t s) {
    EnsembleArgs ea;
    ea.margs = e->margs_dev;
    ea.items = e->items_dev;
    ea.n_items = e->n_items;
    ea.n_members = e->n;
    ea.dt = dt;
    ea.bar = e->bar;
    ea.run = e->run_dev;
    cudaError_t err = cudaMemsetAsync(e->bar, 0, offsetof(GridBar, status), s);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(e->grid);
    cfg.blockDim = dim3(e->variant == FIRE_KERNEL_WARP ? kWarpCtaThreads : kMarchThreads);
    cfg.dynamicSmemBytes = e->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool f64 = e->prec == FIRE_FP64;
    if (e->variant == FIRE_KERNEL_WARP) {
        if (e->nc)
            return f64 ? cudaLaunchKernelEx(&cfg, k_fire_ensemble_warp<double, true>, ea, e->max_rows)
                       : cudaLaunchKernelEx(&cfg, k_fire_ensemble_warp<float, true>, ea, e->max_rows);
        return f64 ? cudaLaunchKernelEx(&cfg, k_fire_ensemble_warp<double, false>, ea, e->max_rows)
                   : cudaLaunchKernelEx(&cfg, k_fire_ensemble_warp<float, false>, ea, e->max_rows);
    }
    if (e->nc)
        return f64 ? cudaLaunchKernelEx(&cfg, k_fire_ensemble<double, true>, ea)
                   : cudaLaunchKernelEx(&cfg, k_fire_ensemble<float, true>, ea);
    return f64 ? cudaLaunchKernelEx(&cfg, k_fire_ensemble<double, false>, ea)
               : cudaLaunchKernelEx(&cfg, k_fire_ensemble<float, false>, ea);
}

}  // namespace

extern "C" {

int fire_ensemble_create(fire_ensemble **out, int n_members, const fire_member_desc *members,
                         void *cuda_stream) {
    if (!out) return FIRE_ERR_ARG;
    *out = nullptr;
    if (n_members < 1 || n_members > FIRE_MAX_MEMBERS || !members) return FIRE_ERR_ARG;
    const int prec = members[0].grid.precision;
    for (int m = 0; m < n_members; ++m)
        if (members[m].grid.precision != prec) return FIRE_ERR_ARG;
    fire_ensemble *e = new (std::nothrow) fire_ensemble();
    if (!e) return FIRE_ERR_OOM;
    e->n = n_members;
    e->prec = prec;
    if (cudaGetDevice(&e->device) != cudaSuccess) {
        delete e;
        return FIRE_ERR_CUDA;
    }
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    int r = FIRE_OK;
    for (int m = 0; m < n_members && r == FIRE_OK; ++m) {
        const fire_member_desc &d = members[m];
        fire_ctx *c = nullptr;
        r = fire_init(&c, &d.grid, d.classes, d.n_classes, d.fuel_class_dev, d.moisture_dev,
                      d.spread_mult_dev, d.dzdx_dev, d.dzdy_dev, d.ignitions, d.n_ign, cuda_stream);
        if (r == FIRE_OK) e->members.push_back(c);
    }
    // one member with a per-node moisture: every member takes the per-node
    // coefficient form of the kernel (the others' planes from their classes)
    if (r == FIRE_OK) {
        for (fire_ctx *c : e->members) e->nc = e->nc || ctx_has_node_coefficients(c);
        if (e->nc)
            for (fire_ctx *c : e->members)
                if (r == FIRE_OK) r = ctx_ensure_node_coefficients(c);
    }
    // the warp form when every member can take warp strips (FP32, refinement
    // <= 30), else the marching form for all; members start from the
    // large-mesh strips of that form (the persistent launch balances the
    // items itself, whatever a member's size)
    if (r == FIRE_OK) {
        bool warp = prec == FIRE_FP32;
        for (fire_ctx *c : e->members) {
            int prc, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
            double t;
            ctx_info(c, &prc, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t);
            warp = warp && srx <= kWarpMaxColumns / 2 && (long long)nx * ny <= kWarpMaxNodes;
        }
        e->variant = warp ? FIRE_KERNEL_WARP : FIRE_KERNEL_MARCH;
        for (fire_ctx *c : e->members)
            if (r == FIRE_OK && (warp ? ctx_default_warp_strips(c) : ctx_default_march(c)) != FIRE_OK)
                r = FIRE_ERR_ARG;
    }
#define ENS_TRY(call)                 \
    do {                              \
        if (r == FIRE_OK) r = ens_cuda(call); \
    } while (0)
    ENS_TRY(cudaMalloc(&e->margs_dev, sizeof(StepArgs) * 2 * n_members));
    ENS_TRY(cudaMallocHost(&e->margs_host, sizeof(StepArgs) * 2 * n_members));
    ENS_TRY(cudaMalloc(&e->bar, sizeof(GridBar)));
    ENS_TRY(cudaMalloc(&e->run_dev, sizeof(EnsRun)));
    ENS_TRY(cudaMallocHost(&e->run_host, sizeof(EnsRun)));
    ENS_TRY(cudaEventCreateWithFlags(&e->staged, cudaEventDisableTiming));
    ENS_TRY(cudaMemsetAsync(e->bar, 0, sizeof(GridBar), e->stream));
#undef ENS_TRY
    if (r == FIRE_OK) r = ens_plan(e);
    if (r == FIRE_OK) r = ens_cuda(cudaStreamSynchronize(e->stream));
    if (r != FIRE_OK) {
        ens_release(e);
        return r;
    }
    *out = e;
    return FIRE_OK;
}

int fire_ensemble_step(fire_ensemble *e, int nsteps, double dt, const void *const *wind_u_dev,
                       const void *const *wind_v_dev, double *const *heat_sens_dev,
                       double *const *heat_lat_dev) {
    if (!e || nsteps < 0 || !isfinite(dt) || !(dt > 0) || !wind_u_dev || !wind_v_dev)
        return FIRE_ERR_ARG;
    for (int m = 0; m < e->n; ++m)
        if (!wind_u_dev[m] || !wind_v_dev[m]) return FIRE_ERR_ARG;
    DeviceGuard dg(e->device);
    int done = 0;
    while (done < nsteps) {
        // an active ignition window needs its own step (fire_step applies it)
        bool ign = false;
        for (int m = 0; m < e->n; ++m) {
            int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
            double t;
            ctx_info(e->members[m], &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t);
            if (ctx_ignition_active(e->members[m], t)) ign = true;
        }
        if (ign) {
            for (int m = 0; m < e->n; ++m) {
                int r = fire_step(e->members[m], wind_u_dev[m], wind_v_dev[m], dt,
                                  heat_sens_dev ? heat_sens_dev[m] : nullptr,
                                  heat_lat_dev ? heat_lat_dev[m] : nullptr);
                if (r) return r;
            }
            ++done;
            continue;
        }
        // the rest (up to the next ignition window) in one persistent launch
        int chunk = 0;
        {
            int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
            double t0;
            ctx_info(e->members[0], &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t0);
            double t = t0;
            while (done + chunk < nsteps) {
                bool any = false;
                for (int m = 0; m < e->n && !any; ++m) any = ctx_ignition_active(e->members[m], t);
                if (any) break;
                t = t + dt;
                ++chunk;
            }
            ENS_CHECK(cudaEventSynchronize(e->staged));
            for (int m = 0; m < e->n; ++m) {
                for (int p = 0; p < 2; ++p) {
                    int r = ctx_step_args(e->members[m], p, wind_u_dev[m], wind_v_dev[m], dt,
                                          heat_sens_dev ? heat_sens_dev[m] : nullptr,
                                          heat_lat_dev ? heat_lat_dev[m] : nullptr,
                                          e->margs_host[2 * m + p]);
                    if (r) return r;
                }
            }
            e->run_host->t0 = t0;
            e->run_host->parity0 = cur;
            e->run_host->nsteps = chunk;
            e->run_host->spin_limit = e->spin_limit;
            e->run_host->skip_block = e->skip_block;
        }
        ENS_CHECK(cudaMemcpyAsync(e->margs_dev, e->margs_host, sizeof(StepArgs) * 2 * e->n,
                                  cudaMemcpyHostToDevice, e->stream));
        ENS_CHECK(cudaMemcpyAsync(e->run_dev, e->run_host, sizeof(EnsRun), cudaMemcpyHostToDevice,
                                  e->stream));
        ENS_CHECK(cudaEventRecord(e->staged, e->stream));
        // replay the captured launch when its shape is unchanged
        if (!e->capture_failed && (!e->graph || e->g_nsteps != chunk || e->g_dt != dt ||
                                   e->g_grid != e->grid || e->g_smem != e->smem)) {
            if (e->graph) {
                ENS_CHECK(cudaStreamSynchronize(e->stream));  // the old graph may be in flight
                cudaGraphExecDestroy(e->graph);
                e->graph = nullptr;
            }
            cudaStream_t cs;
            ENS_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t gr = nullptr;
            cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                err = ens_launch(e, dt, cs);
                cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
                if (err == cudaSuccess) err = e2;
            }
            if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cs);
            if (err != cudaSuccess) {
                // capture of the cooperative launch refused: launch directly
                record_cuda_error(err, "capture of the ensemble launch");
                cudaGetLastError();
                e->graph = nullptr;
                e->capture_failed = true;
            } else {
                e->g_nsteps = chunk;
                e->g_dt = dt;
                e->g_grid = e->grid;
                e->g_smem = e->smem;
            }
        }
        if (e->graph) ENS_CHECK(cudaGraphLaunch(e->graph, e->stream));
        else ENS_CHECK(ens_launch(e, dt, e->stream));
        for (int m = 0; m < e->n; ++m) ctx_advance(e->members[m], chunk, dt);
        done += chunk;
    }
    return FIRE_OK;
}

int fire_ensemble_member(fire_ensemble *e, int member, fire_ctx **ctx) {
    if (!e || !ctx || member < 0 || member >= e->n) return FIRE_ERR_ARG;
    *ctx = e->members[member];
    return FIRE_OK;
}

int fire_ensemble_status(fire_ensemble *e, int *member_status) {
    if (!e) return FIRE_ERR_ARG;
    DeviceGuard dg(e->device);
    ENS_CHECK(cudaStreamSynchronize(e->stream));
    GridBar b;
    ENS_CHECK(cudaMemcpy(&b, e->bar, sizeof b, cudaMemcpyDeviceToHost));
    int worst = FIRE_OK;
    for (int m = 0; m < e->n; ++m) {
        const int s = fire_status(e->members[m]);
        if (member_status) member_status[m] = s;
        if (s != FIRE_OK && worst != FIRE_ERR_BOUNDS &&
            (worst == FIRE_OK || s == FIRE_ERR_NONFINITE || s == FIRE_ERR_BOUNDS))
            worst = s;
    }
    if (b.status & ST_TIMEOUT) return FIRE_ERR_TIMEOUT;
    return worst;
}

int fire_ensemble_clear_status(fire_ensemble *e) {
    if (!e) return FIRE_ERR_ARG;
    for (fire_ctx *c : e->members) {
        int r = fire_clear_status(c);
        if (r) return r;
    }
    ENS_CHECK(cudaMemsetAsync(e->bar, 0, sizeof(GridBar), e->stream));
    return FIRE_OK;
}

int fire_ensemble_set_kernel(fire_ensemble *e, int strip_columns, int strip_rows) {
    if (!e || strip_columns < 2 || strip_rows < 1) return FIRE_ERR_ARG;
    DeviceGuard dg(e->device);
    for (fire_ctx *c : e->members) {
        int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
        double t;
        ctx_info(c, &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t);
        const int maxw = e->variant == FIRE_KERNEL_WARP ? kWarpMaxColumns : kMarchMaxColumns;
        int kxn = std::max(1, std::min(strip_columns, maxw) / srx);
        int kyn = std::max(1, strip_rows / sry);
        if ((kxn * srx) & 1) kxn = kxn > 1 ? kxn - 1 : 2;
        if (e->variant == FIRE_KERNEL_WARP && kyn * sry > kWarpMaxRows) kyn = kWarpMaxRows / sry;
        int r = fire_set_kernel(c, e->variant, kxn, kyn);
        if (r) return r;
    }
    return ens_plan(e);
}

// Times strip shapes (columns x rows of fire nodes) of the persistent
// launch: every candidate starts from the members' saved states, runs one
// untimed call (which also captures its graph) and one timed call of
// probe_steps steps; the fastest is kept and the states are put back.
int fire_ensemble_autotune(fire_ensemble *e, int probe_steps, double dt,
                           const void *const *wind_u_dev, const void *const *wind_v_dev,
                           int *strip_columns, int *strip_rows) {
    if (!e || probe_steps < 1 || !isfinite(dt) || !(dt > 0) || !wind_u_dev || !wind_v_dev)
        return FIRE_ERR_ARG;
    DeviceGuard dg(e->device);
    // the probe must not cross an ignition window (it would apply it)
    std::vector<double> t0(e->n);
    for (int m = 0; m < e->n; ++m) {
        int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
        ctx_info(e->members[m], &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur,
                 &t0[m]);
        double t = t0[m];
        for (int k = 0; k <= 2 * probe_steps; ++k) {
            if (ctx_ignition_active(e->members[m], t)) return FIRE_ERR_STATE;
            t = t + dt;
        }
    }
    // save the states in the members' workspaces
    const size_t E = e->prec == FIRE_FP64 ? 8 : 4;
    std::vector<unsigned char *> saved(e->n);
    std::vector<size_t> nn(e->n);
    for (int m = 0; m < e->n; ++m) {
        int nx = 0, ny = 0;
        fire_mesh_size(e->members[m], &nx, &ny);
        nn[m] = (size_t)nx * ny;
        void *w = nullptr;
        int r = ctx_workspace(e->members[m], nn[m] * (2 * E + sizeof(double)), &w);
        if (r) return r;
        saved[m] = static_cast<unsigned char *>(w);
        r = fire_get_state(e->members[m], saved[m], reinterpret_cast<double *>(saved[m] + 2 * nn[m] * E),
                           saved[m] + nn[m] * E, nullptr);
        if (r) return r;
    }
    auto restore = [&]() {
        for (int m = 0; m < e->n; ++m) {
            int r = fire_set_state(e->members[m], saved[m],
                                   reinterpret_cast<double *>(saved[m] + 2 * nn[m] * E),
                                   saved[m] + nn[m] * E, t0[m]);
            if (r) return r;
        }
        return (int)FIRE_OK;
    };
    const int cols_m[] = {40, 80, 120, 160, 200, 240}, rows_m[] = {20, 40, 80, 160, 320};
    const int cols_w[] = {20, 30, 40, 50, 60, 60}, rows_w[] = {40, 80, 160, 256, 320};
    const bool wv = e->variant == FIRE_KERNEL_WARP;
    const int *cols = wv ? cols_w : cols_m, *rows = wv ? rows_w : rows_m;
    cudaEvent_t a, b;
    ENS_CHECK(cudaEventCreate(&a));
    ENS_CHECK(cudaEventCreate(&b));
    float best = 0.f;
    int bc = 0, br = 0;
    int r = FIRE_OK;
    for (int ci = 0; ci < 6; ++ci) {
        const int C = cols[ci];
        if (ci > 0 && C == cols[ci - 1]) continue;
        for (int ri = 0; ri < 5; ++ri) {
            const int R = rows[ri];
            if (fire_ensemble_set_kernel(e, C, R) != FIRE_OK) continue;
            if ((r = restore())) break;
            if ((r = fire_ensemble_step(e, probe_steps, dt, wind_u_dev, wind_v_dev, nullptr,
                                        nullptr)))
                break;
            if ((r = restore())) break;
            if ((r = ens_cuda(cudaEventRecord(a, e->stream)))) break;
            if ((r = fire_ensemble_step(e, probe_steps, dt, wind_u_dev, wind_v_dev, nullptr,
                                        nullptr)))
                break;
            if ((r = ens_cuda(cudaEventRecord(b, e->stream)))) break;
            if ((r = ens_cuda(cudaEventSynchronize(b)))) break;
            float ms = 0.f;
            if ((r = ens_cuda(cudaEventElapsedTime(&ms, a, b)))) break;
            if (bc == 0 || ms < best) {
                best = ms;
                bc = C;
                br = R;
            }
        }
        if (r) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r) return r;
    if (bc == 0) return FIRE_ERR_ARG;
    r = fire_ensemble_set_kernel(e, bc, br);
    if (r) return r;
    r = restore();
    if (r) return r;
    if (strip_columns) *strip_columns = bc;
    if (strip_rows) *strip_rows = br;
    return FIRE_OK;
}

int fire_ensemble_get_kernel(const fire_ensemble *e, int *grid_ctas, int *work_items) {
    if (!e) return FIRE_ERR_ARG;
    if (grid_ctas) *grid_ctas = e->grid;
    if (work_items) *work_items = e->n_items;
    return FIRE_OK;
}

int fire_ensemble_set_barrier_test(fire_ensemble *e, int skip_block, long long spin_limit) {
    if (!e || spin_limit < 1) return FIRE_ERR_ARG;
    e->skip_block = skip_block;
    e->spin_limit = spin_limit;
    return FIRE_OK;
}

void fire_ensemble_destroy(fire_ensemble *e) {
    if (!e) return;
    DeviceGuard dg(e->device);
    cudaStreamSynchronize(e->stream);
    ens_release(e);
}

}  // extern "C"
