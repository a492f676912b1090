// Host side of the C ABI (include/wrffire.h): the model layer of the fire
// module -- state buffers, step sequencing (Sect. 5, the six-item list),
// ignition bookkeeping (Sect. 3.4), CUDA-graph replay of plain steps, the
// sticky status word, checkpoint/resume, kernel timing and the adaptive
// choice between the two FP32 warp-strip kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "fire_device.cuh"
#include "fire_internal.h"

using namespace wf;

struct fire_ctx {
    fire_grid_desc g{};
    int nx = 0, ny = 0;
    size_t n = 0;
    double dx = 0, dy = 0, psi_far = 0;
    int prec = FIRE_FP32;
    size_t esz = 4;
    cudaStream_t stream = nullptr;
    int device = 0;

    void *psi[2] = {nullptr, nullptr};
    void *frac[2] = {nullptr, nullptr};
    double *tign = nullptr;
    uint8_t *fuel = nullptr;
    void *dzdx = nullptr, *dzdy = nullptr, *mult = nullptr;
    // per-node fuel moisture (path precision, null: the class moisture) and
    // the per-node coefficients R0, c, d, H_s, H_q it gives (null when no
    // per-node moisture is set, unless an ensemble asked for them)
    void *moist = nullptr;
    void *nco[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    fire_fuel_class *classes_dev = nullptr;
    double *coef = nullptr;
    int ncls = 0;
    int *status = nullptr;  // device word
    double *tdev = nullptr;  // [2] device model time, ping-pong with psi
    int cur = 0;
    double t = 0.0;  // host copy of the model time

    std::vector<fire_ignition> ign;
    std::vector<unsigned char> applied;

    int variant = FIRE_KERNEL_MARCH;
    int kx = 0, ky = 0;
    int scheme = 0;  // fuel fraction: 0 subcell scheme, 1 exact for linear data (tiles)
    size_t smem = 0;
    size_t smem_max = 0;
    int n_sm = 1;  // SMs of the device (sizes the default launch shape)

    // host-buffer staging
    void *stage_u = nullptr, *stage_v = nullptr;
    double *stage_hs = nullptr, *stage_hl = nullptr;

    // graph of two plain steps (cur 0 -> 1 -> 0)
    cudaGraphExec_t graph = nullptr;
    const void *g_u = nullptr, *g_v = nullptr;
    double g_dt = 0;
    double *g_hs = nullptr, *g_hl = nullptr;
    int g_kx = 0, g_ky = 0, g_variant = -1;

    // workspace of fire_adjoint (grown on demand, freed with the context)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // captured segments of fire_adjoint (full and ragged length) and their keys
    cudaGraphExec_t adj_graph[2] = {nullptr, nullptr};
    unsigned long long adj_key[2] = {0, 0};

    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pairs
    long launches = 0;
    double ms_done = 0;

    // adaptive choice between the FP32 warp kernels (bitwise equal results):
    // the default strips on a nearly unburnt mesh, the dense variant with
    // shorter strips once enough of it burns; on while the context runs
    // fire_init's default warp strips
    bool adaptive = false;
    bool ad_dense = false;                       // the dense variant is chosen
    int ad_kx = 0, ad_ky = 0, ad_dense_ky = 0;   // the two shapes
    unsigned long long *ad_count_dev = nullptr;  // nodes with psi <= 0
    unsigned long long *ad_count_host = nullptr; // page-locked copy of it
    cudaEvent_t ad_ready = nullptr;              // that copy has landed
    bool ad_pending = false;                     // a count is in flight
    long ad_steps = 0;                           // steps since the last count
    long long ad_counts = 0;                     // count launches so far
    double ad_fraction = -1.0;                   // last burnt fraction seen
};

namespace wf {
namespace {
thread_local char g_last_error[256] = "no error";
}
const char *g_last_error_ptr() { return g_last_error; }
void record_cuda_error(cudaError_t e, const char *where) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s)", where, cudaGetErrorName(e),
             cudaGetErrorString(e));
}
}  // namespace wf

namespace wf {
// nodes with psi <= 0 (burnt or burning), one atomic add per warp
template <typename T>
__global__ void k_count_burnt(const T *__restrict__ psi, size_t n, unsigned long long *count) {
    unsigned k = 0;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < n;
         g += (size_t)gridDim.x * blockDim.x)
        k += psi[g] <= T(0) ? 1u : 0u;
    k = __reduce_add_sync(0xffffffffu, k);
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(count, (unsigned long long)k);
}

}  // namespace wf

namespace {

int cuda_err_at(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return FIRE_OK;
    record_cuda_error(e, where);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FIRE_ERR_OOM;
    }
    return FIRE_ERR_CUDA;
}

#define cuda_err(call) cuda_err_at((call), #call)
#define WF_CHECK(call)                         \
    do {                                       \
        int _r = cuda_err(call);               \
        if (_r != FIRE_OK) return _r;          \
    } while (0)

void release(fire_ctx *c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->ad_ready) cudaEventDestroy(c->ad_ready);
    if (c->ad_count_host) cudaFreeHost(c->ad_count_host);
    if (c->ad_count_dev) cudaFree(c->ad_count_dev);
    for (cudaGraphExec_t g : c->adj_graph)
        if (g) cudaGraphExecDestroy(g);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    void *bufs[] = {c->psi[0], c->psi[1], c->frac[0], c->frac[1], c->tign, c->fuel, c->dzdx,
                    c->dzdy, c->mult, c->classes_dev, c->coef, c->status, c->tdev,
                    c->stage_u, c->stage_v, c->stage_hs, c->stage_hl, c->ws, c->moist};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (void *b : c->nco)
        if (b) cudaFree(b);
    delete c;
}

// (re)computes the per-node coefficient planes from the class table and the
// per-node moisture (allocating them on first use)
int build_node_coefficients(fire_ctx *c) {
    const size_t N = c->n, E = c->esz;
    for (int q = 0; q < 5; ++q)
        if (!c->nco[q]) WF_CHECK(cudaMalloc(&c->nco[q], N * E));
    if (c->prec == FIRE_FP64) {
        double *pl[5];
        for (int q = 0; q < 5; ++q) pl[q] = static_cast<double *>(c->nco[q]);
        WF_CHECK(launch_node_coefficients<double>(c->classes_dev, c->ncls, c->fuel, c->moist, N,
                                                  pl, nullptr, c->stream));
    } else {
        float *pl[5];
        for (int q = 0; q < 5; ++q) pl[q] = static_cast<float *>(c->nco[q]);
        WF_CHECK(launch_node_coefficients<float>(c->classes_dev, c->ncls, c->fuel, c->moist, N,
                                                 pl, nullptr, c->stream));
    }
    return FIRE_OK;
}

// drops the captured step graph (its kernel arguments hold buffer pointers
// that are about to change); waits for the stream first
int drop_step_graph(fire_ctx *c) {
    WF_CHECK(cudaStreamSynchronize(c->stream));
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return FIRE_OK;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

int step_kernel_args(fire_ctx *c, const void *u, const void *v, double dt, double *hs,
                     double *hl, StepArgs &a) {
    memset(&a, 0, sizeof a);
    a.psi_in = c->psi[c->cur];
    a.psi_out = c->psi[1 - c->cur];
    a.F_in = c->frac[c->cur];
    a.F_out = c->frac[1 - c->cur];
    a.tign = c->tign;
    a.fuel = c->fuel;
    a.dzdx = c->dzdx;
    a.dzdy = c->dzdy;
    a.mult = c->mult;
    for (int q = 0; q < 5; ++q) a.nco[q] = c->nco[q];
    a.scheme = c->scheme;
    a.u = u;
    a.v = v;
    a.coef = c->coef;
    a.ncls = c->ncls;
    a.heat_s = hs;
    a.heat_l = hl;
    a.status = c->status;
    a.t_in = c->tdev + c->cur;
    a.t_out = c->tdev + (1 - c->cur);
    a.nx = c->nx;
    a.ny = c->ny;
    a.nxa = c->g.nx_atm;
    a.nya = c->g.ny_atm;
    a.srx = c->g.sr_x;
    a.sry = c->g.sr_y;
    a.kx = c->kx;
    a.ky = c->ky;
    a.band = c->g.boundary_band;
    a.dx = c->dx;
    a.dy = c->dy;
    a.eps = c->g.eps_visc;
    a.dt = dt;
    return FIRE_OK;
}

cudaError_t launch_variant(const fire_ctx *c, const StepArgs &a, cudaStream_t s) {
    if (c->variant == FIRE_KERNEL_MARCH)
        return c->prec == FIRE_FP64 ? launch_march<double>(a, s) : launch_march<float>(a, s);
    if (c->variant == FIRE_KERNEL_WARP)
        return c->prec == FIRE_FP64 ? launch_warp<double>(a, s) : launch_warp<float>(a, s);
    if (c->variant == FIRE_KERNEL_WARP4)
        return c->prec == FIRE_FP32 ? launch_warp4(a, s) : cudaErrorInvalidValue;
    if (c->variant == FIRE_KERNEL_WARP_DENSE)
        return c->prec == FIRE_FP32 ? launch_warp<float>(a, s, true) : cudaErrorInvalidValue;
    return c->prec == FIRE_FP64 ? launch_step<double>(a, s) : launch_step<float>(a, s);
}

// Ignitions active at a step starting at time t (Sect. 3.4), in list order.
// mark: record instantaneous ignitions as applied.
void active_segments(fire_ctx *c, double t, bool mark, std::vector<IgnSeg> &out) {
    out.clear();
    for (size_t q = 0; q < c->ign.size(); ++q) {
        const fire_ignition &g = c->ign[q];
        IgnSeg s{};
        s.ax = g.ax;
        s.ay = g.ay;
        s.bx = g.bx;
        s.by = g.by;
        s.tg = g.t_start;
        s.sg = g.speed;
        s.drip = 0;
        s.tnow = t;
        s.tlay = t;
        if (!(g.speed > 0.0)) {
            if (c->applied[q] || !(g.t_start <= t)) continue;
            s.rho = g.radius;
            if (mark) c->applied[q] = 1;
        } else if (g.vx != 0.0 || g.vy != 0.0) {
            // drip torch: the line laid by min{t, t_end}, the capped radius
            if (!(g.t_start <= t && t <= g.t_end + g.radius / g.speed)) continue;
            const double tt = t < g.t_end ? t : g.t_end;
            s.drip = 1;
            s.tlay = tt;
            s.bx = g.ax + g.vx * (tt - g.t_start);
            s.by = g.ay + g.vy * (tt - g.t_start);
            const double R = g.speed * (t - g.t_start);
            s.rho = R > g.radius ? g.radius : R;
        } else {
            if (!(g.t_start <= t && t <= g.t_start + g.radius / g.speed)) continue;
            s.rho = g.speed * (t - g.t_start);
        }
        out.push_back(s);
    }
}

int apply_ignitions(fire_ctx *c, const std::vector<IgnSeg> &segs) {
    size_t k = 0;
    while (k < segs.size()) {
        IgniteArgs a;
        memset(&a, 0, sizeof a);
        a.psi = c->psi[c->cur];
        a.tign = c->tign;
        a.nx = c->nx;
        a.ny = c->ny;
        a.dx = c->dx;
        a.dy = c->dy;
        int m = 0;
        while (k < segs.size() && m < kMaxSegPerLaunch) a.seg[m++] = segs[k++];
        a.nseg = m;
        cudaError_t e = c->prec == FIRE_FP64 ? launch_ignite<double>(a, c->stream)
                                             : launch_ignite<float>(a, c->stream);
        WF_CHECK(e);
    }
    return FIRE_OK;
}

int record_event(fire_ctx *c) {
    cudaEvent_t e;
    WF_CHECK(cudaEventCreate(&e));
    c->ev.push_back(e);
    WF_CHECK(cudaEventRecord(e, c->stream));
    return FIRE_OK;
}

int configure_kernel(fire_ctx *c, int variant, int kx, int ky) {
    if (kx < 1 || ky < 1) return FIRE_ERR_ARG;
    size_t sm;
    cudaError_t e;
    if (variant == FIRE_KERNEL_MARCH) {
        const long long W = (long long)kx * c->g.sr_x;
        if (W > kMarchMaxColumns || (W & 1)) return FIRE_ERR_ARG;
        sm = c->prec == FIRE_FP64 ? march_smem_bytes<double>(ky, c->g.sr_y, c->ncls)
                                  : march_smem_bytes<float>(ky, c->g.sr_y, c->ncls);
        if (sm > c->smem_max) return FIRE_ERR_ARG;
        e = c->prec == FIRE_FP64 ? prepare_march_kernel<double>(sm) : prepare_march_kernel<float>(sm);
    } else if (variant == FIRE_KERNEL_WARP || variant == FIRE_KERNEL_WARP_DENSE) {
        const long long W = (long long)kx * c->g.sr_x, L = (long long)ky * c->g.sr_y;
        if (W > kWarpMaxColumns || (W & 1) || L > kWarpMaxRows || (long long)c->n > kWarpMaxNodes)
            return FIRE_ERR_ARG;
        if (variant == FIRE_KERNEL_WARP_DENSE && c->prec != FIRE_FP32) return FIRE_ERR_ARG;
        sm = 0;
        e = cudaSuccess;
    } else if (variant == FIRE_KERNEL_WARP4) {
        const long long W = (long long)kx * c->g.sr_x, L = (long long)ky * c->g.sr_y;
        if (c->prec != FIRE_FP32 || W > kWarp4MaxColumns || L > kWarpMaxRows ||
            (long long)c->n > kWarpMaxNodes)
            return FIRE_ERR_ARG;
        sm = 0;
        e = cudaSuccess;
    } else if (variant == FIRE_KERNEL_TILE) {
        sm = c->prec == FIRE_FP64 ? step_smem_bytes<double>(kx, ky, c->g.sr_x, c->g.sr_y, c->ncls)
                                  : step_smem_bytes<float>(kx, ky, c->g.sr_x, c->g.sr_y, c->ncls);
        if (sm > c->smem_max) return FIRE_ERR_ARG;
        e = c->prec == FIRE_FP64 ? prepare_step_kernel<double>(sm) : prepare_step_kernel<float>(sm);
    } else {
        return FIRE_ERR_ARG;
    }
    WF_CHECK(e);
    c->variant = variant;
    c->kx = kx;
    c->ky = ky;
    c->smem = sm;
    return FIRE_OK;
}

// marching strips of up to 248 columns (an even number) x ~60 rows
int default_march(fire_ctx *c) {
    c->adaptive = false;  // an ensemble member keeps the ensemble's form
    if (c->g.sr_x > kMarchMaxColumns / 2) return FIRE_ERR_ARG;
    int kx = kMarchMaxColumns / c->g.sr_x, ky = 60 / c->g.sr_y;
    if (kx > c->g.nx_atm) kx = c->g.nx_atm;
    if ((kx * c->g.sr_x) & 1) kx = kx > 1 ? kx - 1 : 2;
    if (ky < 1) ky = 1;
    if (ky > c->g.ny_atm) ky = c->g.ny_atm;
    return configure_kernel(c, FIRE_KERNEL_MARCH, kx, ky);
}

// the warp strips of the large-mesh default (~60 x 160 nodes), FP32 only
int default_warp_strips(fire_ctx *c) {
    c->adaptive = false;  // an ensemble member keeps the ensemble's form
    if (c->prec != FIRE_FP32 || c->g.sr_x > kWarpMaxColumns / 2 || (long long)c->n > kWarpMaxNodes)
        return FIRE_ERR_ARG;
    int kx = kWarpMaxColumns / c->g.sr_x, ky = 160 / c->g.sr_y;
    if (kx > c->g.nx_atm) kx = c->g.nx_atm;
    // strips of an even width; one atmospheric column at an odd refinement
    // takes a strip of two (the kernel clips a strip at the mesh edge)
    if ((kx * c->g.sr_x) & 1) kx = kx > 1 ? kx - 1 : 2;
    if (ky < 1) ky = 1;
    if (ky > c->g.ny_atm) ky = c->g.ny_atm;
    return configure_kernel(c, FIRE_KERNEL_WARP, kx, ky);
}

int default_kernel(fire_ctx *c) {
    const DefaultShape d = default_shape(c->prec == FIRE_FP64, c->g.nx_atm, c->g.ny_atm,
                                         c->g.sr_x, c->g.sr_y, c->n_sm);
    if (configure_kernel(c, d.variant, d.kx, d.ky) == FIRE_OK) return FIRE_OK;
    // a strip shape whose shared memory does not fit: 2-D tiles, halved until
    // they fit
    int kx = d.variant == FIRE_KERNEL_TILE ? d.kx : (c->prec == FIRE_FP64 ? 40 : 80) / c->g.sr_x;
    int ky = d.variant == FIRE_KERNEL_TILE ? d.ky : 40 / c->g.sr_y;
    if (kx < 1) kx = 1;
    if (ky < 1) ky = 1;
    if (kx > c->g.nx_atm) kx = c->g.nx_atm;
    if (ky > c->g.ny_atm) ky = c->g.ny_atm;
    while (configure_kernel(c, FIRE_KERNEL_TILE, kx, ky) != FIRE_OK) {
        if (kx == 1 && ky == 1) return FIRE_ERR_ARG;
        if (kx >= ky && kx > 1) kx = (kx + 1) / 2;
        else ky = (ky + 1) / 2;
    }
    return FIRE_OK;
}

// burnt fraction at which the dense variant takes over, and below which the
// default strips come back; measured on the 8200x8200 mesh: the default
// strips are 6-10 % faster on a nearly unburnt mesh, the dense 6x6 strips
// 1 % faster at 0.6 % burnt and 11-15 % faster from 2 % burnt on
constexpr double kAdaptOn = 0.005, kAdaptOff = 0.0025;
constexpr long kAdaptEvery = 64;  // steps between counts

// enqueues a count of the current state's burnt nodes into ad_count_dev
int adaptive_count(fire_ctx *c) {
    if (!c->ad_count_dev) WF_CHECK(cudaMalloc(&c->ad_count_dev, sizeof(unsigned long long)));
    WF_CHECK(cudaMemsetAsync(c->ad_count_dev, 0, sizeof(unsigned long long), c->stream));
    const int blocks = c->n_sm * 8;
    if (c->prec == FIRE_FP64)
        k_count_burnt<double><<<blocks, 256, 0, c->stream>>>(
            static_cast<const double *>(c->psi[c->cur]), c->n, c->ad_count_dev);
    else
        k_count_burnt<float><<<blocks, 256, 0, c->stream>>>(
            static_cast<const float *>(c->psi[c->cur]), c->n, c->ad_count_dev);
    WF_CHECK(cudaGetLastError());
    c->ad_counts += 1;
    return FIRE_OK;
}

// the kernel for a counted number of burnt nodes (with hysteresis)
int adaptive_decide(fire_ctx *c, unsigned long long count) {
    c->ad_fraction = (double)count / (double)c->n;
    const bool dense = c->ad_dense ? c->ad_fraction >= kAdaptOff : c->ad_fraction >= kAdaptOn;
    if (dense == c->ad_dense) return FIRE_OK;
    const int r = configure_kernel(c, dense ? FIRE_KERNEL_WARP_DENSE : FIRE_KERNEL_WARP, c->ad_kx,
                                   dense ? c->ad_dense_ky : c->ad_ky);
    if (r == FIRE_OK) c->ad_dense = dense;
    return r;
}

// a count and its copy to page-locked host memory, read by adaptive_update
// once it has landed
int adaptive_enqueue(fire_ctx *c) {
    if (!c->ad_count_host) {
        WF_CHECK(cudaMallocHost(&c->ad_count_host, sizeof(unsigned long long)));
        WF_CHECK(cudaEventCreateWithFlags(&c->ad_ready, cudaEventDisableTiming));
    }
    int r = adaptive_count(c);
    if (r) return r;
    WF_CHECK(cudaMemcpyAsync(c->ad_count_host, c->ad_count_dev, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    WF_CHECK(cudaEventRecord(c->ad_ready, c->stream));
    c->ad_pending = true;
    c->ad_steps = 0;
    return FIRE_OK;
}

// the count of the current state, waited for (fire_init, which waits anyway)
int adaptive_count_now(fire_ctx *c) {
    int r = adaptive_count(c);
    if (r) return r;
    unsigned long long count = 0;
    WF_CHECK(cudaMemcpyAsync(&count, c->ad_count_dev, sizeof count, cudaMemcpyDeviceToHost,
                             c->stream));
    WF_CHECK(cudaStreamSynchronize(c->stream));
    c->ad_steps = 0;
    return adaptive_decide(c, count);
}

// before a step: take the last count if it has landed (no wait), switch the
// kernel when the burnt fraction crossed a threshold, and enqueue the next
// count every kAdaptEvery steps
int adaptive_update(fire_ctx *c) {
    if (!c->adaptive) return FIRE_OK;
    if (c->ad_pending) {
        const cudaError_t e = cudaEventQuery(c->ad_ready);
        if (e == cudaSuccess) {
            c->ad_pending = false;
            const int r = adaptive_decide(c, *c->ad_count_host);
            if (r) return r;
        } else if (e != cudaErrorNotReady) {
            WF_CHECK(e);
        }
    }
    if (!c->ad_pending && c->ad_steps >= kAdaptEvery) return adaptive_enqueue(c);
    return FIRE_OK;
}

// on while the context runs the default FP32 warp strips
void adaptive_setup(fire_ctx *c) {
    c->adaptive = c->prec == FIRE_FP32 && c->variant == FIRE_KERNEL_WARP;
    c->ad_dense = false;
    c->ad_kx = c->kx;
    c->ad_ky = c->ky;
    const int short_rows = 60 / c->g.sr_y;
    c->ad_dense_ky = c->ky < short_rows ? c->ky : (short_rows < 1 ? 1 : short_rows);
    c->ad_steps = kAdaptEvery;  // count before the first step
}

int one_step(fire_ctx *c, const void *u, const void *v, double dt, double *hs, double *hl) {
    int ra = adaptive_update(c);
    if (ra) return ra;
    c->ad_steps += 1;
    std::vector<IgnSeg> segs;
    active_segments(c, c->t, true, segs);
    if (!segs.empty()) {
        int r = apply_ignitions(c, segs);
        if (r) return r;
    }
    StepArgs a;
    step_kernel_args(c, u, v, dt, hs, hl, a);
    if (c->timing) {
        int r = record_event(c);
        if (r) return r;
    }
    WF_CHECK(launch_variant(c, a, c->stream));
    if (c->timing) {
        int r = record_event(c);
        if (r) return r;
        c->launches += 1;
    }
    c->cur = 1 - c->cur;
    c->t = c->t + dt;
    return FIRE_OK;
}

}  // namespace

// accessors used by the ensemble (ensemble.cu)
namespace wf {

#ifdef FIRE_BOUNDS_CHECK
// fire_bounds_selftest: the index check on -1, 0, 9, 10 of a 10-element
// buffer (the checked indices are not used for any access)
__global__ void k_bounds_selftest(int *flags) {
    const long long idx[4] = {-1, 0, 9, 10};
    for (int q = 0; q < 4; ++q) {
        int st = 0;
        (void)bounds_checked(idx[q], 10, st);
        flags[q] = (st & ST_BOUNDS) ? 1 : 0;
    }
}
#endif

static long cdiv_l(long a, long b) { return (a + b - 1) / b; }

DefaultShape default_shape(bool fp64, int nx_atm, int ny_atm, int srx, int sry, int n_sm) {
    const long nx = (long)nx_atm * srx, ny = (long)ny_atm * sry;
    if (n_sm < 1) n_sm = 1;
    // tallest strips (ky atmospheric rows, at most ky_max) with at least
    // waves2/2 waves of CTAs; 0 when even one-cell strips give under a
    // quarter wave
    auto height = [&](long ctas_x, int ky_max, long slots, int waves2) {
        int ky = ky_max < 1 ? 1 : (ky_max > ny_atm ? ny_atm : ky_max);
        while (ky > 1 && 2 * ctas_x * cdiv_l(ny, (long)ky * sry) < waves2 * slots) --ky;
        return 4 * ctas_x * cdiv_l(ny, (long)sry) < slots ? 0 : ky;
    };
    if (!fp64 && srx <= kWarpMaxColumns / 2 && (long long)nx * ny <= kWarpMaxNodes) {
        int kx = kWarpMaxColumns / srx;
        if (kx > nx_atm) kx = nx_atm;
        if ((kx * srx) & 1) kx = kx > 1 ? kx - 1 : 0;
        if (kx >= 1) {
            const long ctas_x = cdiv_l(cdiv_l(nx, (long)kx * srx), kWarpStrips);
            const int ky = height(ctas_x, 160 / sry, (long)n_sm * kWarpCtasPerSmF32, 7);
            if (ky >= 1) return {FIRE_KERNEL_WARP, kx, ky};
            return {FIRE_KERNEL_TILE, 1, 1};
        }
    }
    if (srx <= kMarchMaxColumns / 2) {
        int kx = kMarchMaxColumns / srx;
        if (kx > nx_atm) kx = nx_atm;
        if ((kx * srx) & 1) kx = kx > 1 ? kx - 1 : 2;
        const long ctas_x = cdiv_l(nx, (long)kx * srx);
        const long slots = (long)n_sm * (fp64 ? kMarchCtasPerSmF64 : kMarchCtasPerSmF32);
        const int ky = height(ctas_x, 60 / sry, slots, 5);
        if (ky >= 1) return {FIRE_KERNEL_MARCH, kx, ky};
        return {FIRE_KERNEL_TILE, 1, 1};
    }
    int kx = (fp64 ? 40 : 80) / srx, ky = 40 / sry;
    if (kx < 1) kx = 1;
    if (ky < 1) ky = 1;
    if (kx > nx_atm) kx = nx_atm;
    if (ky > ny_atm) ky = ny_atm;
    return {FIRE_KERNEL_TILE, kx, ky};
}

int ctx_step_args(fire_ctx *c, int parity, const void *u, const void *v, double dt, double *hs,
                  double *hl, StepArgs &a) {
    const int save = c->cur;
    c->cur = parity;
    step_kernel_args(c, u, v, dt, hs, hl, a);
    c->cur = save;
    return FIRE_OK;
}

int ctx_info(const fire_ctx *c, int *prec, int *variant, int *nx, int *ny, int *srx, int *sry,
             int *kx, int *ky, int *ncls, int *cur, double *t) {
    *prec = c->prec;
    *variant = c->variant;
    *nx = c->nx;
    *ny = c->ny;
    *srx = c->g.sr_x;
    *sry = c->g.sr_y;
    *kx = c->kx;
    *ky = c->ky;
    *ncls = c->ncls;
    *cur = c->cur;
    *t = c->t;
    return FIRE_OK;
}

int ctx_advance(fire_ctx *c, int nsteps, double dt) {
    for (int k = 0; k < nsteps; ++k) {
        c->cur = 1 - c->cur;
        c->t = c->t + dt;
    }
    return FIRE_OK;
}

bool ctx_ignition_active(fire_ctx *c, double t) {
    std::vector<IgnSeg> segs;
    active_segments(c, t, false, segs);
    return !segs.empty();
}

cudaStream_t ctx_stream(const fire_ctx *c) { return c->stream; }
int ctx_device(const fire_ctx *c) { return c->device; }

int ctx_default_march(fire_ctx *c) { return default_march(c); }
int ctx_default_warp_strips(fire_ctx *c) { return default_warp_strips(c); }

const fire_fuel_class *ctx_classes_dev(const fire_ctx *c) { return c->classes_dev; }
const void *ctx_moisture(const fire_ctx *c) { return c->moist; }
bool ctx_has_node_coefficients(const fire_ctx *c) { return c->nco[0] != nullptr; }
int ctx_scheme(const fire_ctx *c) { return c->scheme; }
int ctx_ensure_node_coefficients(fire_ctx *c) {
    if (c->nco[0]) return FIRE_OK;
    int r = drop_step_graph(c);
    if (r) return r;
    r = build_node_coefficients(c);
    if (r) return r;
    return cuda_err(cudaStreamSynchronize(c->stream));
}

cudaGraphExec_t *ctx_adjoint_graphs(fire_ctx *c, unsigned long long **keys) {
    *keys = c->adj_key;
    return c->adj_graph;
}

int ctx_workspace(fire_ctx *c, size_t bytes, void **out) {
    if (bytes > c->ws_bytes) {
        if (c->ws) {
            WF_CHECK(cudaStreamSynchronize(c->stream));  // the old one may be in use
            // captured adjoint segments point into the old workspace
            for (int k = 0; k < 2; ++k) {
                if (c->adj_graph[k]) cudaGraphExecDestroy(c->adj_graph[k]);
                c->adj_graph[k] = nullptr;
            }
            cudaFree(c->ws);
            c->ws = nullptr;
            c->ws_bytes = 0;
        }
        WF_CHECK(cudaMalloc(&c->ws, bytes));
        c->ws_bytes = bytes;
    }
    *out = c->ws;
    return FIRE_OK;
}
}  // namespace wf

extern "C" {

const char *fire_last_cuda_error(void) { return wf::g_last_error_ptr(); }

int fire_bounds_checked(void) {
#ifdef FIRE_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

int fire_bounds_selftest(int *flags_host) {
    if (!flags_host) return FIRE_ERR_ARG;
#ifdef FIRE_BOUNDS_CHECK
    int *d = nullptr;
    WF_CHECK(cudaMalloc(&d, 4 * sizeof(int)));
    wf::k_bounds_selftest<<<1, 1>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(flags_host, d, 4 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    WF_CHECK(e);
    return FIRE_OK;
#else
    return FIRE_ERR_STATE;
#endif
}

const char *fire_strerror(int code) {
    switch (code) {
        case FIRE_OK: return "ok";
        case FIRE_ERR_ARG: return "invalid argument";
        case FIRE_ERR_CUDA: return "CUDA runtime error";
        case FIRE_ERR_OOM: return "out of memory";
        case FIRE_ERR_BOUNDARY: return "fire reached the domain boundary";
        case FIRE_ERR_NONFINITE: return "non-finite wind or level-set value";
        case FIRE_ERR_TIMEOUT: return "a bounded device wait timed out";
        case FIRE_ERR_STATE: return "call not valid in this state";
        case FIRE_ERR_BOUNDS: return "index outside its buffer (bounds-checked build)";
        default: return "unknown error";
    }
}

int fire_init(fire_ctx **out, const fire_grid_desc *grid, const fire_fuel_class *classes,
              int n_classes, const uint8_t *fuel_class_dev, const void *moisture_dev,
              const void *spread_mult_dev, const void *dzdx_dev, const void *dzdy_dev,
              const fire_ignition *ignitions, int n_ign, void *cuda_stream) {
    if (!out) return FIRE_ERR_ARG;
    *out = nullptr;
    if (!grid || !classes || !fuel_class_dev || !dzdx_dev || !dzdy_dev) return FIRE_ERR_ARG;
    if (n_classes < 1 || n_classes > FIRE_MAX_CLASSES) return FIRE_ERR_ARG;
    if (n_ign < 0 || n_ign > FIRE_MAX_IGNITIONS || (n_ign > 0 && !ignitions)) return FIRE_ERR_ARG;
    const fire_grid_desc &g = *grid;
    if (g.nx_atm < 1 || g.ny_atm < 1 || g.sr_x < 1 || g.sr_y < 1) return FIRE_ERR_ARG;
    if (!finite_pos(g.dx_atm) || !finite_pos(g.dy_atm)) return FIRE_ERR_ARG;
    if (g.precision != FIRE_FP32 && g.precision != FIRE_FP64) return FIRE_ERR_ARG;
    if (g.boundary_band < 1 || !(g.eps_visc >= 0.0) || !isfinite(g.eps_visc)) return FIRE_ERR_ARG;
    if (!isfinite(g.psi_far)) return FIRE_ERR_ARG;
    const long long NX = (long long)g.nx_atm * g.sr_x, NY = (long long)g.ny_atm * g.sr_y;
    if (NX < 2 || NY < 2 || NX > (1 << 30) || NY > (1 << 30)) return FIRE_ERR_ARG;
    if (NX * NY > (1LL << 34)) return FIRE_ERR_OOM;
    for (int q = 0; q < n_ign; ++q) {
        const fire_ignition &s = ignitions[q];
        if (!isfinite(s.ax) || !isfinite(s.ay) || !isfinite(s.bx) || !isfinite(s.by) ||
            !isfinite(s.t_start) || !isfinite(s.radius) || !isfinite(s.speed) || s.radius < 0)
            return FIRE_ERR_ARG;
        if (!isfinite(s.vx) || !isfinite(s.vy) || !isfinite(s.t_end)) return FIRE_ERR_ARG;
        if ((s.vx != 0.0 || s.vy != 0.0) && !(s.speed > 0.0 && s.t_end >= s.t_start))
            return FIRE_ERR_ARG;
    }
    for (int k = 0; k < n_classes; ++k)
        if (!valid_fuel_class(classes[k])) return FIRE_ERR_ARG;

    fire_ctx *c = new (std::nothrow) fire_ctx();
    if (!c) return FIRE_ERR_OOM;
    c->g = g;
    c->nx = (int)NX;
    c->ny = (int)NY;
    c->n = (size_t)NX * (size_t)NY;
    c->dx = g.dx_atm / g.sr_x;
    c->dy = g.dy_atm / g.sr_y;
    c->psi_far = g.psi_far > 0 ? g.psi_far : hypot(NX * c->dx, NY * c->dy);
    c->prec = g.precision;
    c->esz = c->prec == FIRE_FP64 ? 8 : 4;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->ncls = n_classes;
    c->ign.assign(ignitions, ignitions + n_ign);
    c->applied.assign(n_ign, 0);
    int r = FIRE_OK;
#define WF_TRY(call)              \
    do {                          \
        r = cuda_err(call);       \
        if (r) {                  \
            release(c);           \
            return r;             \
        }                         \
    } while (0)
    WF_TRY(cudaGetDevice(&c->device));
    int smo = 0;
    WF_TRY(cudaDeviceGetAttribute(&smo, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    c->smem_max = (size_t)smo;
    WF_TRY(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device));
    const size_t N = c->n, E = c->esz;
    WF_TRY(cudaMalloc(&c->psi[0], N * E));
    WF_TRY(cudaMalloc(&c->psi[1], N * E));
    WF_TRY(cudaMalloc(&c->frac[0], N * E));
    WF_TRY(cudaMalloc(&c->frac[1], N * E));
    WF_TRY(cudaMalloc(&c->tign, N * sizeof(double)));
    WF_TRY(cudaMalloc(&c->fuel, N));
    WF_TRY(cudaMalloc(&c->dzdx, N * E));
    WF_TRY(cudaMalloc(&c->dzdy, N * E));
    if (spread_mult_dev) WF_TRY(cudaMalloc(&c->mult, N * E));
    if (moisture_dev) WF_TRY(cudaMalloc(&c->moist, N * E));
    WF_TRY(cudaMalloc(&c->classes_dev, sizeof(fire_fuel_class) * n_classes));
    WF_TRY(cudaMalloc(&c->coef, sizeof(double) * K_N * n_classes));
    WF_TRY(cudaMalloc(&c->status, sizeof(int)));
    WF_TRY(cudaMalloc(&c->tdev, 2 * sizeof(double)));
    cudaStream_t s = c->stream;
    WF_TRY(cudaMemcpyAsync(c->fuel, fuel_class_dev, N, cudaMemcpyDeviceToDevice, s));
    WF_TRY(cudaMemcpyAsync(c->dzdx, dzdx_dev, N * E, cudaMemcpyDeviceToDevice, s));
    WF_TRY(cudaMemcpyAsync(c->dzdy, dzdy_dev, N * E, cudaMemcpyDeviceToDevice, s));
    if (spread_mult_dev)
        WF_TRY(cudaMemcpyAsync(c->mult, spread_mult_dev, N * E, cudaMemcpyDeviceToDevice, s));
    if (moisture_dev)
        WF_TRY(cudaMemcpyAsync(c->moist, moisture_dev, N * E, cudaMemcpyDeviceToDevice, s));
    WF_TRY(cudaMemcpyAsync(c->classes_dev, classes, sizeof(fire_fuel_class) * n_classes,
                           cudaMemcpyHostToDevice, s));
    WF_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s));
    WF_TRY(cudaMemsetAsync(c->tdev, 0, 2 * sizeof(double), s));
    WF_TRY(launch_coefficients(c->classes_dev, n_classes, c->coef, s));
    if (moisture_dev) {
        r = build_node_coefficients(c);
        if (r) {
            release(c);
            return r;
        }
    }
    WF_TRY(c->prec == FIRE_FP64 ? launch_fill<double>(c->psi[0], c->tign, c->frac[0], N,
                                                      c->psi_far, s)
                                : launch_fill<float>(c->psi[0], c->tign, c->frac[0], N,
                                                     c->psi_far, s));
    // the model starts at t = 0: instantaneous ignitions with t_start <= 0
    {
        std::vector<IgnSeg> segs;
        for (size_t q = 0; q < c->ign.size(); ++q) {
            const fire_ignition &gq = c->ign[q];
            if (!(gq.speed > 0.0) && gq.t_start <= 0.0) {
                IgnSeg sg{};
                sg.ax = gq.ax;
                sg.ay = gq.ay;
                sg.bx = gq.bx;
                sg.by = gq.by;
                sg.tg = gq.t_start;
                sg.sg = gq.speed;
                sg.rho = gq.radius;
                segs.push_back(sg);
                c->applied[q] = 1;
            }
        }
        r = apply_ignitions(c, segs);
        if (r) {
            release(c);
            return r;
        }
    }
    r = default_kernel(c);
    if (r) {
        release(c);
        return r;
    }
    adaptive_setup(c);
    if (c->adaptive) {
        r = adaptive_count_now(c);  // the initial choice, from the state after the ignitions
        if (r) {
            release(c);
            return r;
        }
    }
    // the copies above read caller buffers: finish before returning
    WF_TRY(cudaStreamSynchronize(s));
#undef WF_TRY
    *out = c;
    return FIRE_OK;
}

int fire_step(fire_ctx *c, const void *u, const void *v, double dt, double *hs, double *hl) {
    if (!c || !u || !v || !finite_pos(dt)) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    return one_step(c, u, v, dt, hs, hl);
}

// device address of a page-locked host buffer the device can write, else
// null (pageable memory; the failed query's error is cleared)
static double *mapped_host(double *h) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return static_cast<double *>(at.devicePointer);
}

int fire_step_host(fire_ctx *c, const void *u, const void *v, double dt, double *hs,
                   double *hl) {
    if (!c || !u || !v || !finite_pos(dt)) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    const size_t nu = (size_t)c->g.ny_atm * (c->g.nx_atm + 1) * c->esz;
    const size_t nv = (size_t)(c->g.ny_atm + 1) * c->g.nx_atm * c->esz;
    const size_t nh = (size_t)c->g.ny_atm * c->g.nx_atm * sizeof(double);
    if (!c->stage_u) {
        WF_CHECK(cudaMalloc(&c->stage_u, nu));
        WF_CHECK(cudaMalloc(&c->stage_v, nv));
        WF_CHECK(cudaMalloc(&c->stage_hs, nh));
        WF_CHECK(cudaMalloc(&c->stage_hl, nh));
    }
    WF_CHECK(cudaMemcpyAsync(c->stage_u, u, nu, cudaMemcpyHostToDevice, c->stream));
    WF_CHECK(cudaMemcpyAsync(c->stage_v, v, nv, cudaMemcpyHostToDevice, c->stream));
    // heat written by the kernel straight into page-locked, device-mapped
    // host buffers (visible to the host once the stream is synchronised)
    double *hs_k = hs ? mapped_host(hs) : nullptr, *hl_k = hl ? mapped_host(hl) : nullptr;
    int r = one_step(c, c->stage_u, c->stage_v, dt, hs ? (hs_k ? hs_k : c->stage_hs) : nullptr,
                     hl ? (hl_k ? hl_k : c->stage_hl) : nullptr);
    if (r) return r;
    if (hs && !hs_k)
        WF_CHECK(cudaMemcpyAsync(hs, c->stage_hs, nh, cudaMemcpyDeviceToHost, c->stream));
    if (hl && !hl_k)
        WF_CHECK(cudaMemcpyAsync(hl, c->stage_hl, nh, cudaMemcpyDeviceToHost, c->stream));
    WF_CHECK(cudaStreamSynchronize(c->stream));
    return FIRE_OK;
}

int fire_run(fire_ctx *c, int nsteps, double dt, const void *u, const void *v, double *hs,
             double *hl) {
    if (!c || !u || !v || nsteps < 0 || !finite_pos(dt)) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    int k = 0;
    std::vector<IgnSeg> segs;
    while (k < nsteps) {
        // two plain steps starting from cur == 0 replay the captured graph
        bool plain = c->cur == 0 && nsteps - k >= 2 && !c->timing;
        if (plain) {
            active_segments(c, c->t, false, segs);
            plain = segs.empty();
        }
        if (plain) {
            active_segments(c, c->t + dt, false, segs);
            plain = segs.empty();
        }
        if (!plain) {
            int r = one_step(c, u, v, dt, hs, hl);
            if (r) return r;
            ++k;
            continue;
        }
        int ra = adaptive_update(c);
        if (ra) return ra;
        c->ad_steps += 2;
        if (!c->graph || c->g_u != u || c->g_v != v || c->g_dt != dt || c->g_hs != hs ||
            c->g_hl != hl || c->g_kx != c->kx || c->g_ky != c->ky || c->g_variant != c->variant) {
            if (c->graph) {
                WF_CHECK(cudaStreamSynchronize(c->stream));  // the old graph may be in flight
                cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
            }
            cudaStream_t cs;
            WF_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                StepArgs a;
                for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
                    step_kernel_args(c, u, v, dt, hs, hl, a);
                    a.psi_in = c->psi[h];
                    a.psi_out = c->psi[1 - h];
                    a.F_in = c->frac[h];
                    a.F_out = c->frac[1 - h];
                    a.t_in = c->tdev + h;
                    a.t_out = c->tdev + (1 - h);
                    e = launch_variant(c, a, cs);
                }
                cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cs);
            WF_CHECK(e);
            c->g_u = u;
            c->g_v = v;
            c->g_dt = dt;
            c->g_hs = hs;
            c->g_hl = hl;
            c->g_kx = c->kx;
            c->g_ky = c->ky;
            c->g_variant = c->variant;
        }
        WF_CHECK(cudaGraphLaunch(c->graph, c->stream));
        c->t = c->t + dt;
        c->t = c->t + dt;
        k += 2;
    }
    return FIRE_OK;
}

int fire_get_state(fire_ctx *c, void *psi, double *tign, void *frac, double *t_host) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    const size_t N = c->n, E = c->esz;
    if (psi) WF_CHECK(cudaMemcpyAsync(psi, c->psi[c->cur], N * E, cudaMemcpyDeviceToDevice, c->stream));
    if (tign)
        WF_CHECK(cudaMemcpyAsync(tign, c->tign, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (frac) WF_CHECK(cudaMemcpyAsync(frac, c->frac[c->cur], N * E, cudaMemcpyDeviceToDevice, c->stream));
    if (t_host) *t_host = c->t;
    return FIRE_OK;
}

int fire_set_state(fire_ctx *c, const void *psi, const double *tign, const void *frac, double t) {
    if (!c || !psi || !tign || !frac || !isfinite(t)) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    const size_t N = c->n, E = c->esz;
    WF_CHECK(cudaMemcpyAsync(c->psi[c->cur], psi, N * E, cudaMemcpyDeviceToDevice, c->stream));
    WF_CHECK(cudaMemcpyAsync(c->tign, tign, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    WF_CHECK(cudaMemcpyAsync(c->frac[c->cur], frac, N * E, cudaMemcpyDeviceToDevice, c->stream));
    c->t = t;
    // the device time follows through a host-pinned-free path: synchronous copy
    WF_CHECK(cudaMemcpyAsync(c->tdev + c->cur, &c->t, sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
    WF_CHECK(cudaStreamSynchronize(c->stream));
    c->ad_steps = kAdaptEvery;  // a new state: count it before the next step
    return FIRE_OK;
}

int fire_set_spread_mult(fire_ctx *c, const void *mult_dev) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    const size_t N = c->n, E = c->esz;
    const bool had = c->mult != nullptr;
    if (had != (mult_dev != nullptr)) {
        // the multiplier pointer changes: the captured step graph is stale
        WF_CHECK(cudaStreamSynchronize(c->stream));
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        if (had) {
            cudaFree(c->mult);
            c->mult = nullptr;
        } else {
            WF_CHECK(cudaMalloc(&c->mult, N * E));
        }
    }
    if (mult_dev)
        WF_CHECK(cudaMemcpyAsync(c->mult, mult_dev, N * E, cudaMemcpyDeviceToDevice, c->stream));
    WF_CHECK(cudaStreamSynchronize(c->stream));
    return FIRE_OK;
}

int fire_set_fuel_classes(fire_ctx *c, const fire_fuel_class *classes, int n_classes) {
    if (!c || !classes || n_classes != c->ncls) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    for (int k = 0; k < n_classes; ++k)
        if (!valid_fuel_class(classes[k])) return FIRE_ERR_ARG;
    WF_CHECK(cudaMemcpyAsync(c->classes_dev, classes, sizeof(fire_fuel_class) * n_classes,
                             cudaMemcpyHostToDevice, c->stream));
    WF_CHECK(launch_coefficients(c->classes_dev, n_classes, c->coef, c->stream));
    if (c->nco[0]) {
        const int r = build_node_coefficients(c);
        if (r) return r;
    }
    WF_CHECK(cudaStreamSynchronize(c->stream));
    return FIRE_OK;
}

int fire_set_moisture(fire_ctx *c, const void *moisture_dev) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    const size_t N = c->n, E = c->esz;
    if (!moisture_dev) {
        if (!c->moist) return FIRE_OK;
        int r = drop_step_graph(c);
        if (r) return r;
        cudaFree(c->moist);
        c->moist = nullptr;
        for (void *&b : c->nco) {
            cudaFree(b);
            b = nullptr;
        }
        return FIRE_OK;
    }
    if (!c->nco[0] || !c->moist) {
        int r = drop_step_graph(c);  // new buffers: the captured arguments are stale
        if (r) return r;
        if (!c->moist) WF_CHECK(cudaMalloc(&c->moist, N * E));
    }
    WF_CHECK(cudaMemcpyAsync(c->moist, moisture_dev, N * E, cudaMemcpyDeviceToDevice, c->stream));
    const int r = build_node_coefficients(c);
    if (r) return r;
    WF_CHECK(cudaStreamSynchronize(c->stream));
    return FIRE_OK;
}

int fire_status(fire_ctx *c) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    WF_CHECK(cudaStreamSynchronize(c->stream));
    int st = 0;
    WF_CHECK(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_BOUNDS) return FIRE_ERR_BOUNDS;
    if (st & ST_NONFINITE) return FIRE_ERR_NONFINITE;
    if (st & ST_BOUNDARY) return FIRE_ERR_BOUNDARY;
    if (st & ST_TIMEOUT) return FIRE_ERR_TIMEOUT;
    return FIRE_OK;
}

int fire_clear_status(fire_ctx *c) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    WF_CHECK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    return FIRE_OK;
}

int fire_mesh_size(const fire_ctx *c, int *nx, int *ny) {
    if (!c) return FIRE_ERR_ARG;
    if (nx) *nx = c->nx;
    if (ny) *ny = c->ny;
    return FIRE_OK;
}

double fire_time(const fire_ctx *c) { return c ? c->t : NAN; }

int fire_set_kernel(fire_ctx *c, int variant, int kx, int ky) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    if (c->scheme == 1 && variant != FIRE_KERNEL_TILE) return FIRE_ERR_ARG;
    const int r = configure_kernel(c, variant, kx, ky);
    if (r == FIRE_OK) c->adaptive = false;  // the caller's choice stays
    return r;
}

int fire_set_adaptive(fire_ctx *c, int on) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    if (!on) {
        c->adaptive = false;
        return FIRE_OK;
    }
    if (c->prec != FIRE_FP32 || c->scheme != 0 ||
        (c->variant != FIRE_KERNEL_WARP && c->variant != FIRE_KERNEL_WARP_DENSE))
        return FIRE_ERR_ARG;
    // the current strips become the default shape; the dense variant takes
    // the rows of the shorter strips
    const bool dense = c->variant == FIRE_KERNEL_WARP_DENSE;
    if (dense) {
        const int r = configure_kernel(c, FIRE_KERNEL_WARP, c->kx, c->ky);
        if (r) return r;
    }
    adaptive_setup(c);
    return FIRE_OK;
}

int fire_adaptive_info(const fire_ctx *c, int *on, long long *counts, double *burnt_fraction) {
    if (!c) return FIRE_ERR_ARG;
    if (on) *on = c->adaptive ? 1 : 0;
    if (counts) *counts = c->ad_counts;
    if (burnt_fraction) *burnt_fraction = c->ad_fraction;
    return FIRE_OK;
}

int fire_set_fraction_scheme(fire_ctx *c, int scheme) {
    if (!c || (scheme != 0 && scheme != 1)) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    if (scheme == c->scheme) return FIRE_OK;
    if (scheme == 1) c->adaptive = false;  // tiles only
    int r = drop_step_graph(c);  // the captured steps carry the scheme
    if (r) return r;
    if (scheme == 1 && c->variant != FIRE_KERNEL_TILE) {
        // the 2-D tile kernel at the large-refinement tile size, halved
        // until its shared memory fits
        const bool fp64 = c->prec == FIRE_FP64;
        int kx = (fp64 ? 40 : 80) / c->g.sr_x, ky = 40 / c->g.sr_y;
        kx = kx < 1 ? 1 : (kx > c->g.nx_atm ? c->g.nx_atm : kx);
        ky = ky < 1 ? 1 : (ky > c->g.ny_atm ? c->g.ny_atm : ky);
        for (;;) {
            if (configure_kernel(c, FIRE_KERNEL_TILE, kx, ky) == FIRE_OK) break;
            if (kx == 1 && ky == 1) return FIRE_ERR_ARG;
            if (kx >= ky && kx > 1) kx = (kx + 1) / 2;
            else ky = (ky + 1) / 2;
        }
    }
    c->scheme = scheme;
    return FIRE_OK;
}

// Candidate step-kernel shapes timed on a scratch copy of the state: the
// marching strip over widths of about 16..248 columns and heights of about
// 8..512 rows, and the 2-D tile over a few shapes; the fastest average of
// probe_steps launches (after one warm-up launch) is kept.
int fire_default_kernel(int precision, int nx_atm, int ny_atm, int sr_x, int sr_y, int n_sm,
                        int *variant, int *kx, int *ky) {
    if ((precision != FIRE_FP32 && precision != FIRE_FP64) || nx_atm < 1 || ny_atm < 1 ||
        sr_x < 1 || sr_y < 1 || n_sm < 1 || !variant || !kx || !ky)
        return FIRE_ERR_ARG;
    const DefaultShape d =
        default_shape(precision == FIRE_FP64, nx_atm, ny_atm, sr_x, sr_y, n_sm);
    *variant = d.variant;
    *kx = d.kx;
    *ky = d.ky;
    return FIRE_OK;
}

int fire_autotune(fire_ctx *c, const void *u, const void *v, double dt, int probe_steps,
                  int *variant_out, int *kx_out, int *ky_out) {
    if (!c || !u || !v || !finite_pos(dt) || probe_steps < 1) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    const size_t N = c->n, E = c->esz;
    const size_t na = (size_t)c->g.nx_atm * c->g.ny_atm;
    // scratch: psi x2, F x2, tign, heat x2, times, status
    const size_t o_psi = 0, o_F = o_psi + 2 * N * E, o_t = o_F + 2 * N * E;
    const size_t o_h = o_t + N * sizeof(double), o_tm = o_h + 2 * na * sizeof(double);
    const size_t bytes = o_tm + 4 * sizeof(double) + sizeof(int);
    void *wsv = nullptr;
    int r = wf::ctx_workspace(c, (bytes + 255) & ~(size_t)255, &wsv);
    if (r) return r;
    unsigned char *ws = static_cast<unsigned char *>(wsv);
    void *sp[2] = {ws + o_psi, ws + o_psi + N * E};
    void *sf[2] = {ws + o_F, ws + o_F + N * E};
    double *stign = reinterpret_cast<double *>(ws + o_t);
    double *shs = reinterpret_cast<double *>(ws + o_h), *shl = shs + na;
    double *stm = reinterpret_cast<double *>(ws + o_tm);
    int *sst = reinterpret_cast<int *>(ws + o_tm + 4 * sizeof(double));

    struct Cand {
        int variant, kx, ky;
    };
    std::vector<Cand> cands;
    const int srx = c->g.sr_x, sry = c->g.sr_y, nxa = c->g.nx_atm, nya = c->g.ny_atm;
    auto add = [&](int variant, int kx, int ky) {
        if (c->scheme == 1 && variant != FIRE_KERNEL_TILE) return;  // tiles only
        kx = kx < 1 ? 1 : (kx > nxa ? nxa : kx);
        ky = ky < 1 ? 1 : (ky > nya ? nya : ky);
        if (variant != FIRE_KERNEL_TILE && ((kx * srx) & 1)) {
            if (kx > 1) --kx;
            else if (2 <= nxa) kx = 2;
            else return;
        }
        for (const Cand &q : cands)
            if (q.variant == variant && q.kx == kx && q.ky == ky) return;
        cands.push_back(Cand{variant, kx, ky});
    };
    if (srx <= kMarchMaxColumns / 2) {
        const int widths[] = {16, 24, 32, 48, 64, 96, 128, 176, 248};
        const int heights[] = {8, 16, 32, 64, 128, 256, 512};
        for (int W : widths) {
            if (W / srx * srx > kMarchMaxColumns) continue;
            for (int L : heights) add(FIRE_KERNEL_MARCH, W / srx, L / sry);
        }
    }
    if (srx <= kWarpMaxColumns / 2) {
        const int widths[] = {20, 30, 40, 50, 60};
        const int heights[] = {16, 32, 64, 128, 256, 512};
        for (int W : widths) {
            if (W / srx * srx > kWarpMaxColumns || W / srx < 1) continue;
            for (int L : heights) {
                add(FIRE_KERNEL_WARP, W / srx, L / sry);
                if (c->prec == FIRE_FP32) add(FIRE_KERNEL_WARP_DENSE, W / srx, L / sry);
            }
        }
    }
    if (c->prec == FIRE_FP32 && srx <= kWarp4MaxColumns / 2) {
        const int widths[] = {60, 80, 100, 120};
        const int heights[] = {16, 32, 64, 128, 256};
        for (int W : widths) {
            if (W / srx * srx > kWarp4MaxColumns || W / srx < 1) continue;
            for (int L : heights) add(FIRE_KERNEL_WARP4, W / srx, L / sry);
        }
    }
    {
        const int widths[] = {32, 64, 128};
        const int heights[] = {8, 16, 32, 64};
        for (int W : widths)
            for (int L : heights) add(FIRE_KERNEL_TILE, W / srx, L / sry);
    }
    const int save_variant = c->variant, save_kx = c->kx, save_ky = c->ky;
    cudaEvent_t e0, e1;
    WF_CHECK(cudaEventCreate(&e0));
    WF_CHECK(cudaEventCreate(&e1));
    float best = 0.f;
    Cand win{save_variant, save_kx, save_ky};
    bool found = false;
    for (const Cand &q : cands) {
        if (configure_kernel(c, q.variant, q.kx, q.ky) != FIRE_OK) continue;
        // the same starting state for every candidate
        WF_CHECK(cudaMemcpyAsync(sp[0], c->psi[c->cur], N * E, cudaMemcpyDeviceToDevice, c->stream));
        WF_CHECK(cudaMemcpyAsync(sf[0], c->frac[c->cur], N * E, cudaMemcpyDeviceToDevice, c->stream));
        WF_CHECK(cudaMemcpyAsync(stign, c->tign, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
        WF_CHECK(cudaMemcpyAsync(stm, c->tdev + c->cur, sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
        StepArgs a;
        step_kernel_args(c, u, v, dt, shs, shl, a);
        a.tign = stign;
        a.status = sst;
        for (int k = 0; k <= probe_steps; ++k) {
            if (k == 1) WF_CHECK(cudaEventRecord(e0, c->stream));
            a.psi_in = sp[k & 1];
            a.psi_out = sp[(k + 1) & 1];
            a.F_in = sf[k & 1];
            a.F_out = sf[(k + 1) & 1];
            a.t_in = stm + (k & 1);
            a.t_out = stm + ((k + 1) & 1);
            WF_CHECK(launch_variant(c, a, c->stream));
        }
        WF_CHECK(cudaEventRecord(e1, c->stream));
        WF_CHECK(cudaEventSynchronize(e1));
        float ms = 0.f;
        WF_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (!found || ms < best) {
            best = ms;
            win = q;
            found = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    r = configure_kernel(c, win.variant, win.kx, win.ky);
    if (r) return r;
    c->adaptive = false;  // the measured choice stays
    if (variant_out) *variant_out = win.variant;
    if (kx_out) *kx_out = win.kx;
    if (ky_out) *ky_out = win.ky;
    return FIRE_OK;
}

int fire_get_kernel(const fire_ctx *c, int *variant, int *kx, int *ky) {
    if (!c) return FIRE_ERR_ARG;
    if (variant) *variant = c->variant;
    if (kx) *kx = c->kx;
    if (ky) *ky = c->ky;
    return FIRE_OK;
}

int fire_enable_timing(fire_ctx *c, int on) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    c->timing = on != 0;
    return FIRE_OK;
}

int fire_kernel_time_ms(fire_ctx *c, double *ms, long *launches) {
    if (!c) return FIRE_ERR_ARG;
    DeviceGuard dg(c->device);
    double total = c->ms_done;
    for (size_t k = 0; k + 1 < c->ev.size(); k += 2) {
        WF_CHECK(cudaEventSynchronize(c->ev[k + 1]));
        float m = 0;
        WF_CHECK(cudaEventElapsedTime(&m, c->ev[k], c->ev[k + 1]));
        total += m;
    }
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    if (ms) *ms = total;
    if (launches) *launches = c->launches;
    c->ms_done = 0;
    c->launches = 0;
    return FIRE_OK;
}

void fire_destroy(fire_ctx *c) {
    if (!c) return;
    DeviceGuard dg(c->device);
    cudaStreamSynchronize(c->stream);
    release(c);
}

}  // extern "C"
