// The two coupling steps around the fire step (Sect. "Coupling of the fire
// and the atmospheric models"): the wind at the height z_f by vertical
// log-linear interpolation (before the step), and the insertion of the
// averaged heat fluxes into the atmospheric tendencies with an
// exp(-z/z_ext) profile (after it).  Both are element-wise over columns:
// one thread per column (wind) or per column and level (heat), the levels
// of a column strided by the number of columns so that a warp reads
// consecutive columns; memory bound and tiny next to the fire step (atmos
// mesh, not fire mesh).
#include <cuda_runtime.h>
#include <math.h>

#include "fire_internal.h"

namespace wf {
namespace {

__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

// per column p: the piecewise linear interpolant in ln z of (ln z0, 0) and
// the levels above z0, at ln zf; 0 where zf <= z0; the top value above the
// highest level
template <typename T>
__global__ void k_wind_at_height(int nz, long long npts, const T *__restrict__ u3d,
                                 const T *__restrict__ z3d, const T *__restrict__ z0, T zf,
                                 T *__restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
        const T r = z0[p];
        if (!(zf > r)) {
            out[p] = T(0);
            continue;
        }
        const T x = log_t(zf);
        T xl = log_t(r), ul = T(0), val = T(0);
        bool done = false;
        for (int k = 0; k < nz; ++k) {
            const T zk = z3d[(long long)k * npts + p];
            if (!(zk > r)) continue;
            const T xk = log_t(zk), uk = u3d[(long long)k * npts + p];
            if (x <= xk) {
                val = ul + (uk - ul) * (x - xl) / (xk - xl);
                done = true;
                break;
            }
            xl = xk;
            ul = uk;
        }
        out[p] = done ? val : ul;
    }
}

// per column p and layer k: the layer average S of the convergence of the
// flux phi exp(-z/z_ext) between the faces zw_k, zw_{k+1}; the sources
// mu phi_h S / (cp rho) and mu phi_q S / (L rho) are added to the tendencies
__global__ void k_heat_insertion(int nz, long long n, const double *__restrict__ hs,
                                 const double *__restrict__ hl, const double *__restrict__ zw,
                                 const double *__restrict__ rho, const double *__restrict__ mu,
                                 double zext, double cp, double L, double *__restrict__ rth,
                                 double *__restrict__ rqv) {
    const long long total = (long long)nz * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long p = q % n;
        const double za = zw[q], zb = zw[q + n];
        const double S = (exp(-za / zext) - exp(-zb / zext)) / (zb - za);
        const double r = rho[q];
        if (rth) rth[q] += mu[p] * hs[p] / (cp * r) * S;
        if (rqv) rqv[q] += mu[p] * hl[p] / (L * r) * S;
    }
}

int grid_of(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 16) b = 152LL * 16;  // grid-stride beyond ~16 waves of 256-thread CTAs
    return (int)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace wf

using namespace wf;

extern "C" int fire_wind_at_height(int precision, int nz, long long npts, const void *u3d_dev,
                                   const void *z3d_dev, const void *z0_dev, double z_f,
                                   void *out_dev, void *cuda_stream) {
    if (nz < 1 || npts < 1 || !u3d_dev || !z3d_dev || !z0_dev || !out_dev || !isfinite(z_f))
        return FIRE_ERR_ARG;
    if (precision != FIRE_FP32 && precision != FIRE_FP64) return FIRE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (precision == FIRE_FP64)
        k_wind_at_height<double><<<grid_of(npts, 256), 256, 0, s>>>(
            nz, npts, static_cast<const double *>(u3d_dev), static_cast<const double *>(z3d_dev),
            static_cast<const double *>(z0_dev), z_f, static_cast<double *>(out_dev));
    else
        k_wind_at_height<float><<<grid_of(npts, 256), 256, 0, s>>>(
            nz, npts, static_cast<const float *>(u3d_dev), static_cast<const float *>(z3d_dev),
            static_cast<const float *>(z0_dev), (float)z_f, static_cast<float *>(out_dev));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        record_cuda_error(e, "k_wind_at_height");
        return FIRE_ERR_CUDA;
    }
    return FIRE_OK;
}

extern "C" int fire_heat_insertion(int nz, long long ncols, const double *heat_sens_dev,
                                   const double *heat_lat_dev, const double *zw_dev,
                                   const double *rho_dev, const double *mu_dev, double z_ext,
                                   double cp, double latent, double *rth_dev, double *rqv_dev,
                                   void *cuda_stream) {
    if (nz < 1 || ncols < 1 || !zw_dev || !rho_dev || !mu_dev) return FIRE_ERR_ARG;
    if ((rth_dev && !heat_sens_dev) || (rqv_dev && !heat_lat_dev) || (!rth_dev && !rqv_dev))
        return FIRE_ERR_ARG;
    if (!(z_ext > 0.0) || !(cp > 0.0) || !(latent > 0.0) || !isfinite(z_ext)) return FIRE_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_heat_insertion<<<grid_of((long long)nz * ncols, 256), 256, 0, s>>>(
        nz, ncols, heat_sens_dev, heat_lat_dev, zw_dev, rho_dev, mu_dev, z_ext, cp, latent,
        rth_dev, rqv_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        record_cuda_error(e, "k_heat_insertion");
        return FIRE_ERR_CUDA;
    }
    return FIRE_OK;
}
