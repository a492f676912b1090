// fire_step_noalloc: one fire step on caller-owned state that allocates no
// memory.
//
// Some callers cannot call cudaMalloc: host applications whose GPU memory is
// handed out by their own pool or by a host framework that forbids driver
// allocations after start-up, and coupled models that must not touch the
// allocator from their time loop (an allocation there can synchronise the
// device or fail once the pool owns the memory).  This entry point serves
// them: the caller passes every input and output buffer, and the few
// intermediate values the step needs (the fuel-class table, its spread-rate
// coefficients, the step's start and end time and, when the caller passes
// none, the status word) live in one file-scope __device__ array of fixed
// size instead of a cudaMalloc'ed buffer.  It launches the same kernels as
// fire_step.  With no status_dev the faults go to that array's status word,
// which no call reads back: a caller who wants to see faults passes one.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "fire_internal.h"

using namespace wf;

namespace {

constexpr int kNoAllocMaxClasses = FIRE_MAX_CLASSES;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    fire_fuel_class classes[kNoAllocMaxClasses];
    double coef[kNoAllocMaxClasses * K_N];
    double t[2];
    int status;
};

// The scratch of every call on a device: about 11 KB, held by each device
// that loads the library until the process exits.  Host code must not take
// its address directly (that is a host-side stand-in); it asks the runtime.
static __device__ __align__(256) unsigned char g_fire_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (first call
// per device: cudaGetSymbolAddress with that device current)
int scratch_address(NoAllocScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIRE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FIRE_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_fire_noalloc_scratch) != cudaSuccess || !p)
            return FIRE_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<NoAllocScratch *>(g_scratch_addr[dev]);
    return FIRE_OK;
}

struct SetupArgs {
    fire_fuel_class classes[kNoAllocMaxClasses];
    int n;
    double t;
    int clear_status;
};

// copies the class table (passed by value) and the start time into the
// scratch, and clears the scratch status word when it is the one in use
__global__ void k_noalloc_setup(const SetupArgs p, NoAllocScratch *s) {
    const int k = threadIdx.x;
    if (k < p.n) s->classes[k] = p.classes[k];
    if (k == 0) {
        s->t[0] = p.t;
        if (p.clear_status) s->status = 0;
    }
}

bool finite_positive(double x) { return isfinite(x) && x > 0.0; }

}  // namespace

extern "C" int fire_step_noalloc(const fire_grid_desc *grid, const fire_fuel_class *classes,
                                 int n_classes, const void *psi_in_dev, void *psi_out_dev,
                                 const void *frac_in_dev, void *frac_out_dev, double *tign_dev,
                                 const uint8_t *fuel_class_dev, const void *spread_mult_dev,
                                 const void *dzdx_dev, const void *dzdy_dev,
                                 const void *wind_u_dev, const void *wind_v_dev, double t,
                                 double dt, double *heat_sens_dev, double *heat_lat_dev,
                                 int *status_dev, void *cuda_stream) {
    if (!grid || !classes || !psi_in_dev || !psi_out_dev || !frac_in_dev || !frac_out_dev ||
        !tign_dev || !fuel_class_dev || !dzdx_dev || !dzdy_dev || !wind_u_dev || !wind_v_dev)
        return FIRE_ERR_ARG;
    if (n_classes < 1 || n_classes > kNoAllocMaxClasses) return FIRE_ERR_ARG;
    if (psi_in_dev == psi_out_dev || frac_in_dev == frac_out_dev) return FIRE_ERR_ARG;
    if (!isfinite(t) || !finite_positive(dt)) return FIRE_ERR_ARG;
    const fire_grid_desc &g = *grid;
    if (g.nx_atm < 1 || g.ny_atm < 1 || g.sr_x < 1 || g.sr_y < 1) return FIRE_ERR_ARG;
    if (!finite_positive(g.dx_atm) || !finite_positive(g.dy_atm)) return FIRE_ERR_ARG;
    if (g.precision != FIRE_FP32 && g.precision != FIRE_FP64) return FIRE_ERR_ARG;
    if (g.boundary_band < 1 || !(g.eps_visc >= 0.0) || !isfinite(g.eps_visc)) return FIRE_ERR_ARG;
    const long long NX = (long long)g.nx_atm * g.sr_x, NY = (long long)g.ny_atm * g.sr_y;
    if (NX < 2 || NY < 2 || NX > (1 << 30) || NY > (1 << 30)) return FIRE_ERR_ARG;
    for (int k = 0; k < n_classes; ++k)
        if (!valid_fuel_class(classes[k])) return FIRE_ERR_ARG;

    NoAllocScratch *s = nullptr;
    int r = scratch_address(&s);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bool fp64 = g.precision == FIRE_FP64;

    SetupArgs sa;
    memset(&sa, 0, sizeof sa);
    memcpy(sa.classes, classes, sizeof(fire_fuel_class) * n_classes);
    sa.n = n_classes;
    sa.t = t;
    sa.clear_status = status_dev ? 0 : 1;
    k_noalloc_setup<<<1, kNoAllocMaxClasses, 0, st>>>(sa, s);
    if (cudaGetLastError() != cudaSuccess) return FIRE_ERR_CUDA;
    if (launch_coefficients(s->classes, n_classes, s->coef, st) != cudaSuccess)
        return FIRE_ERR_CUDA;

    StepArgs a;
    memset(&a, 0, sizeof a);
    a.psi_in = psi_in_dev;
    a.psi_out = psi_out_dev;
    a.F_in = frac_in_dev;
    a.F_out = frac_out_dev;
    a.tign = tign_dev;
    a.fuel = fuel_class_dev;
    a.dzdx = dzdx_dev;
    a.dzdy = dzdy_dev;
    a.mult = spread_mult_dev;
    a.u = wind_u_dev;
    a.v = wind_v_dev;
    a.coef = s->coef;
    a.ncls = n_classes;
    a.heat_s = heat_sens_dev;
    a.heat_l = heat_lat_dev;
    a.status = status_dev ? status_dev : &s->status;
    a.t_in = &s->t[0];
    a.t_out = &s->t[1];
    a.nx = (int)NX;
    a.ny = (int)NY;
    a.nxa = g.nx_atm;
    a.nya = g.ny_atm;
    a.srx = g.sr_x;
    a.sry = g.sr_y;
    a.band = g.boundary_band;
    a.dx = g.dx_atm / g.sr_x;
    a.dy = g.dy_atm / g.sr_y;
    a.eps = g.eps_visc;
    a.dt = dt;

    // the step kernel fire_init would choose by default (default_shape)
    int smo = 0, dev = 0, n_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smo, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FIRE_ERR_CUDA;
    const DefaultShape d = default_shape(fp64, g.nx_atm, g.ny_atm, g.sr_x, g.sr_y, n_sm);
    cudaError_t e = cudaErrorInvalidValue;
    if (d.variant == FIRE_KERNEL_WARP && (long long)d.ky * g.sr_y <= kWarpMaxRows) {
        a.kx = d.kx;
        a.ky = d.ky;
        e = launch_warp<float>(a, st);
        return e == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
    }
    if (d.variant == FIRE_KERNEL_MARCH) {
        const size_t sm = fp64 ? march_smem_bytes<double>(d.ky, g.sr_y, n_classes)
                               : march_smem_bytes<float>(d.ky, g.sr_y, n_classes);
        if ((long long)d.kx * g.sr_x <= kMarchMaxColumns && sm <= (size_t)smo) {
            a.kx = d.kx;
            a.ky = d.ky;
            e = fp64 ? prepare_march_kernel<double>(sm) : prepare_march_kernel<float>(sm);
            if (e == cudaSuccess) e = fp64 ? launch_march<double>(a, st) : launch_march<float>(a, st);
            return e == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
        }
    }
    // tiles: the chosen one, else the large-refinement size, halved until
    // the shared memory fits
    int kx = d.variant == FIRE_KERNEL_TILE ? d.kx : (fp64 ? 40 : 80) / g.sr_x;
    int ky = d.variant == FIRE_KERNEL_TILE ? d.ky : 40 / g.sr_y;
    if (kx < 1) kx = 1;
    if (ky < 1) ky = 1;
    if (kx > g.nx_atm) kx = g.nx_atm;
    if (ky > g.ny_atm) ky = g.ny_atm;
    for (;;) {
        const size_t sm = fp64 ? step_smem_bytes<double>(kx, ky, g.sr_x, g.sr_y, n_classes)
                               : step_smem_bytes<float>(kx, ky, g.sr_x, g.sr_y, n_classes);
        if (sm <= (size_t)smo) {
            a.kx = kx;
            a.ky = ky;
            e = fp64 ? prepare_step_kernel<double>(sm) : prepare_step_kernel<float>(sm);
            if (e == cudaSuccess) e = fp64 ? launch_step<double>(a, st) : launch_step<float>(a, st);
            return e == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
        }
        if (kx == 1 && ky == 1) return FIRE_ERR_ARG;
        if (kx >= ky && kx > 1) kx = (kx + 1) / 2;
        else ky = (ky + 1) / 2;
    }
}
