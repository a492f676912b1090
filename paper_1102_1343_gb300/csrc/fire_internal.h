// Host-side declarations shared by the translation units of the library.
// (CUDA path only; nothing here is shared with the CPU oracle.)
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/wrffire.h"

namespace wf {

// sticky device status bits (ST_BOUNDS only in libraries built with
// FIRE_BOUNDS_CHECK)
enum { ST_BOUNDARY = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4, ST_BOUNDS = 8 };

// per-class coefficient slots: eq. (spread-WRF-Fire) + T_f + heat factors
enum { K_S0 = 0, K_R0, K_B, K_C, K_D, K_E, K_TF, K_HS, K_HQ, K_N };

// Function attributes (the dynamic shared-memory limit of a kernel) are
// per device: the caches that avoid setting them again are indexed by it.
constexpr int kMaxDevices = 64;

// The device of a context for the length of an entry point: switched to on
// entry when another one is current, switched back on exit (a context's
// stream and buffers belong to the device current at its fire_init).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess)
            prev = cur;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// the device a context was created on (context.cu)
int ctx_device(const fire_ctx *c);

// the current device as an index of the attribute caches (-1: none of them)
inline int attr_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}

constexpr int kThreadsX = 32;
constexpr int kThreadsY = 8;
constexpr int kThreads = kThreadsX * kThreadsY;
constexpr int kMaxSegPerLaunch = 64;

// Arguments of the fused step kernel.  Element type of the void pointers is
// the path precision T.
struct StepArgs {
    const void *psi_in;
    void *psi_out;
    const void *F_in;
    void *F_out;
    double *tign;
    const uint8_t *fuel;
    const void *dzdx, *dzdy, *mult;
    const void *u, *v;
    const double *coef;  // [ncls][K_N]
    int ncls;
    double *heat_s, *heat_l;  // nullable
    int *status;
    const double *t_in;  // model time at the step start (device scalar)
    double *t_out;       // receives t_in + dt (written by one thread)
    int nx, ny, nxa, nya, srx, sry;
    int kx, ky;  // tile = kx*srx by ky*sry nodes
    int band;
    double dx, dy, eps, dt;
    // per-node coefficients of a per-node fuel moisture, or all null: R0, c,
    // d, H_s, H_q, each [ny][nx] in the path precision (S0, b, e and T_f
    // stay per class)
    const void *nco[5];
    // fuel fraction: 0 the subcell scheme of Sect. 3.3, 1 the scheme exact
    // for linear psi and t_i (2-D tile kernel only)
    int scheme;
};

struct IgnSeg {
    double ax, ay, bx, by;
    double rho;      // current radius term: r_g (instantaneous) or S_g (t - t_g)
    double tg, sg;   // start time and growth speed (sg <= 0: instantaneous)
    // drip torch: the step start t and min{t, t_end}; the nearest point at
    // parameter u of [a, b] was laid at tg + u (tlay - tg)
    int drip;
    double tnow, tlay;
};

struct IgniteArgs {
    void *psi;
    double *tign;
    int nx, ny;
    double dx, dy;
    int nseg;
    IgnSeg seg[kMaxSegPerLaunch];
};

template <typename T>
size_t step_smem_bytes(int kx, int ky, int srx, int sry, int ncls);

template <typename T>
cudaError_t launch_step(const StepArgs &a, cudaStream_t s);

template <typename T>
cudaError_t launch_ignite(const IgniteArgs &a, cudaStream_t s);

template <typename T>
cudaError_t launch_fill(void *psi, double *tign, void *frac, size_t n, double psi_far,
                        cudaStream_t s);

template <typename T>
cudaError_t prepare_step_kernel(size_t smem_bytes);

template <typename T>
size_t march_smem_bytes(int ky, int sry, int ncls);

template <typename T>
cudaError_t launch_march(const StepArgs &a, cudaStream_t s);

template <typename T>
cudaError_t prepare_march_kernel(size_t smem_bytes);

constexpr int kMarchMaxColumns = 248;  // output columns of one marching strip (even)

template <typename T>
cudaError_t launch_warp(const StepArgs &a, cudaStream_t s, bool dense = false);

// four columns per lane (FP32 only): strips of <= 120 output columns
constexpr int kWarp4MaxColumns = 120;
cudaError_t launch_warp4(const StepArgs &a, cudaStream_t s);

constexpr int kWarpStrips = 4;       // warps (strips) per CTA of the warp kernel
constexpr int kWarpMaxColumns = 60;  // output columns of one warp strip (even)
constexpr int kWarpMaxRows = 512;    // output rows of one warp strip
// the warp kernel indexes the mesh with 32-bit offsets: nx * ny below 2^31
constexpr long long kWarpMaxNodes = 2147483647LL;

// resident CTAs per SM of the strip kernels (the minimum blocks of their
// __launch_bounds__, checked where the kernels are defined)
constexpr int kWarpCtasPerSmF32 = 3;
constexpr int kMarchCtasPerSmF32 = 5;
constexpr int kMarchCtasPerSmF64 = 2;

// Default launch shape of a single run's step (fire_init and
// fire_step_noalloc).  Strips (warp strips of <= 60 columns in FP32 when the
// refinement allows, else marching strips of <= 248 columns) of the largest
// height up to ~160 rows (warp) / ~60 rows (march) that still gives 3.5
// (warp) / 2.5 (march) waves of resident CTAs on n_sm SMs, else strips one
// atmospheric cell high; where even those fill under a quarter of one wave,
// 2-D tiles of one atmospheric cell; for refinements too large for either
// strip kernel, tiles of ~80x40 (FP32) / 40x40 (FP64) nodes.  The caller
// checks the shape's shared memory and halves tiles that do not fit.
struct DefaultShape {
    int variant, kx, ky;
};
DefaultShape default_shape(bool fp64, int nx_atm, int ny_atm, int srx, int sry, int n_sm);

cudaError_t launch_coefficients(const fire_fuel_class *classes_dev, int n, double *coef_dev,
                                cudaStream_t s);
// d(coefficients)/d(M_f) per class at the class moisture (forward-mode dual
// numbers through the same chain)
cudaError_t launch_coefficients_dMf(const fire_fuel_class *classes_dev, int n, double *dcoef_dev,
                                    cudaStream_t s);

// per-node coefficients at a per-node moisture (null: class moisture):
// planes is a host array of 5 device pointers (R0, c, d, H_s, H_q, each [n]
// in the path precision); aos (nullable) receives [n][K_N] doubles
template <typename T>
cudaError_t launch_node_coefficients(const fire_fuel_class *classes_dev, int ncls,
                                     const uint8_t *fuel, const void *moist, size_t n,
                                     T *const *planes, double *aos, cudaStream_t s);
// d(coefficients)/d(M_f) per node at the node's moisture: [n][K_N] doubles
template <typename T>
cudaError_t launch_node_coefficients_dMf(const fire_fuel_class *classes_dev, int ncls,
                                         const uint8_t *fuel, const void *moist, size_t n,
                                         double *daos, cudaStream_t s);

// a fuel class fire_init accepts: a positive weight (burn time), and for a
// Rothermel class with fuel (Table 2) a positive surface-area-to-volume
// ratio, depth, particle density, moisture of extinction and effective
// mineral content (the chain divides by or takes powers of each)
inline bool valid_fuel_class(const fire_fuel_class &f) {
    if (!(f.weight > 0)) return false;
    if (f.fgi > 0 && !f.chaparral &&
        !(f.savr > 0 && f.fueldepthm > 0 && f.fueldens > 0 && f.fuelmce > 0 && f.se > 0))
        return false;
    return true;
}

// remembers the last CUDA error an entry point saw on this host thread
// (read back through fire_last_cuda_error)
void record_cuda_error(cudaError_t e, const char *where);
const char *g_last_error_ptr();

}  // namespace wf
