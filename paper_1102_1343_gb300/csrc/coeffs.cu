// Init-time kernel: fuel-class properties (Table 1) -> the per-class
// coefficients of eq. (spread-WRF-Fire), the burn time T_f and the heat
// factors of eqs. (sensible-heat-flux), (latent-heat-flux).  One thread per
// class, FP64.
//
// The Rothermel chain of Table 2 runs in English units (the caption of
// Table 2 converts inputs from metric); the spread rate is
//   S = R0 (1 + phi_W + phi_S),  phi_W = C U_a^B (beta/beta_op)^(-E),
//   phi_S = 5.275 beta^(-0.3) tan^2(phi),  U_a = a U,
// with the CAWFE limits 0 <= U <= 30 m/s and tan(phi) >= 0, which gives the
// coefficient form S = max{S0, R0 + c min{e, max{0,U}}^b + d max{0,tan}^2}
// with b = B, c = R0 C (a * 196.85)^B (beta/beta_op)^(-E), d = 5.275 R0
// beta^(-0.3), e = 30 m/s, S0 = 0 (SI, U in m/s).  Chaparral (eq. chapparal):
// S0 = 0.03333, R0 = 0, b = 1, c = 1.2974, d = 0, e = 6/1.2974.
// Readings of the table's garbled entries: Gamma_max uses Rothermel's
// constant 0.0594; Q_ig = 250 + 1116 M_f; B = 0.02526 sigma^0.54 and
// beta_op = 3.348 sigma^(-0.8189).  eta_M is clamped to [0, 1]; a class
// without fuel load does not spread.
#include <cuda_runtime.h>
#include <math.h>

#include "fire_internal.h"

namespace wf {

namespace {

constexpr double kFt = 0.3048;          // m per ft
constexpr double kLb = 0.45359237;      // kg per lb
constexpr double kBtu = 1055.05585262;  // J per BTU
constexpr double kLatent = 2.5e6;       // L (J/kg)
constexpr double kWindMax = 30.0;       // m/s

// Scalars of the chain: double, or a forward-mode dual number (value and
// derivative with respect to the fuel moisture M_f) for the adjoint.
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return mk(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return mk(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return mk(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    return mk(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return mk(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return mk(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return mk(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return mk(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return mk(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return mk(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
    return mk(a / b.v, -a * b.d / (b.v * b.v));
}
__device__ __forceinline__ Dual pow_c(Dual a, double p) {
    return mk(pow(a.v, p), p * pow(a.v, p - 1.0) * a.d);
}
__device__ __forceinline__ double pow_c(double a, double p) { return pow(a, p); }
__device__ __forceinline__ Dual exp_s(Dual a) {
    const double e = exp(a.v);
    return mk(e, e * a.d);
}
__device__ __forceinline__ double exp_s(double a) { return exp(a); }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double val(double a) { return a; }
template <typename S>
__device__ __forceinline__ S constant(double x);
template <>
__device__ __forceinline__ double constant<double>(double x) { return x; }
template <>
__device__ __forceinline__ Dual constant<Dual>(double x) { return mk(x, 0.0); }

// The chain for one class at moisture Mf; co receives the K_N slots.
template <typename S>
__device__ void coefficient_chain(const fire_fuel_class &f, S Mf, S *co) {
    co[K_TF] = constant<S>(f.weight_is_tf ? f.weight : f.weight / (-1000.0 * log(0.6) / 600.0));
    co[K_HS] = f.fgi * f.cmbcnst / (1.0 + Mf);
    co[K_HQ] = (Mf + 0.56) / (1.0 + Mf) * kLatent * f.fgi;
    if (f.chaparral) {
        co[K_S0] = constant<S>(0.03333);
        co[K_R0] = constant<S>(0.0);
        co[K_B] = constant<S>(1.0);
        co[K_C] = constant<S>(1.2974);
        co[K_D] = constant<S>(0.0);
        co[K_E] = constant<S>(6.0 / 1.2974);
        return;
    }
    co[K_S0] = constant<S>(0.0);
    co[K_E] = constant<S>(kWindMax);
    if (!(f.fgi > 0.0)) {
        co[K_R0] = constant<S>(0.0);
        co[K_B] = constant<S>(1.0);
        co[K_C] = constant<S>(0.0);
        co[K_D] = constant<S>(0.0);
        return;
    }
    // English units
    const double sig = f.savr * kFt;                       // 1/ft
    const double load = f.fgi * kFt * kFt / kLb;           // lb/ft^2
    const double dep = f.fueldepthm / kFt;                 // ft
    const double rhoP = f.fueldens * kFt * kFt * kFt / kLb;  // lb/ft^3
    const double heat = f.cmbcnst * kLb / kBtu;            // BTU/lb
    // packing
    const S w0 = load / (1.0 + Mf);
    const S rhob = w0 / dep;
    const S beta = rhob / rhoP;
    const double bop = 3.348 * pow(sig, -0.8189);
    const S rel = beta / bop;
    // reaction intensity
    const double sig15 = pow(sig, 1.5);
    const double gmax = sig15 / (495.0 + 0.0594 * sig15);
    const double A = 1.0 / (4.77 * pow(sig, 0.1) - 7.27);
    const S gam = gmax * pow_c(rel, A) * exp_s(A * (1.0 - rel));
    const S wn = w0 / (1.0 + f.st);
    const S x = Mf / f.fuelmce;
    S etaM = 1.0 - 2.59 * x + 5.11 * x * x - 3.52 * x * x * x;
    if (val(x) >= 1.0 || val(etaM) < 0.0) etaM = constant<S>(0.0);
    if (val(etaM) > 1.0) etaM = constant<S>(1.0);
    const double etaS = 0.174 * pow(f.se, -0.19);
    const S IR = gam * wn * heat * etaM * etaS;
    // propagating flux, heat sink
    const S xi = exp_s((0.792 + 0.681 * sqrt(sig)) * (beta + 0.1)) / (192.0 + 0.2595 * sig);
    const double epsh = exp(-138.0 / sig);
    const S Qig = 250.0 + 1116.0 * Mf;
    const S R0 = IR * xi / (rhob * epsh * Qig) * (kFt / 60.0);  // ft/min -> m/s
    // wind and slope factors
    const double B = 0.02526 * pow(sig, 0.54);
    const double C = 7.47 * exp(-0.133 * pow(sig, 0.55));
    const double E = 0.715 * exp(-3.59e-4 * sig);
    co[K_R0] = R0;
    co[K_B] = constant<S>(B);
    co[K_C] = R0 * C * pow(f.windrf * (60.0 / kFt), B) * pow_c(rel, -E);
    co[K_D] = R0 * 5.275 * pow_c(beta, -0.3);
}

__global__ void k_coefficients(const fire_fuel_class *cls, int n, double *coef) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const fire_fuel_class f = cls[k];
    coefficient_chain<double>(f, f.fuelmc_g, coef + (size_t)k * K_N);
}

// d(coefficients)/d(M_f) at the class moisture (clamped branches of eta_M
// and the chaparral rule have derivative 0)
__global__ void k_coefficients_dMf(const fire_fuel_class *cls, int n, double *dcoef) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const fire_fuel_class f = cls[k];
    Dual co[K_N];
    coefficient_chain<Dual>(f, mk(f.fuelmc_g, 1.0), co);
    for (int q = 0; q < K_N; ++q) dcoef[(size_t)k * K_N + q] = co[q].d;
}

// Per-node coefficients for a per-node fuel moisture M_f (Table 1 M_f per
// grid point; eq. spread-WRF-Fire keeps its coefficients per node): the
// chain of the node's class at the node's moisture (the class moisture where
// moist is null).  R0, c, d and the two heat factors depend on M_f; S0, b, e
// and T_f do not and stay in the class table.  planes: [5][n] in the path
// precision (R0, c, d, H_s, H_q; skipped when null); aos (nullable): [n][K_N]
// doubles, every slot, for the adjoint.
template <typename T>
struct Planes5 {
    T *p[5];
};

template <typename T>
__global__ void k_node_coefficients(const fire_fuel_class *cls, int ncls, const uint8_t *fuel,
                                    const T *moist, size_t n, const Planes5<T> pl, double *aos) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        int c = fuel[k];
        c = c < ncls ? c : ncls - 1;
        const fire_fuel_class f = cls[c];
        double co[K_N];
        coefficient_chain<double>(f, moist ? (double)moist[k] : f.fuelmc_g, co);
        if (pl.p[0]) {
            pl.p[0][k] = T(co[K_R0]);
            pl.p[1][k] = T(co[K_C]);
            pl.p[2][k] = T(co[K_D]);
            pl.p[3][k] = T(co[K_HS]);
            pl.p[4][k] = T(co[K_HQ]);
        }
        if (aos)
            for (int q = 0; q < K_N; ++q) aos[k * K_N + q] = co[q];
    }
}

// d(coefficients)/d(M_f) per node at the node's moisture: [n][K_N]
template <typename T>
__global__ void k_node_coefficients_dMf(const fire_fuel_class *cls, int ncls, const uint8_t *fuel,
                                        const T *moist, size_t n, double *daos) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        int c = fuel[k];
        c = c < ncls ? c : ncls - 1;
        const fire_fuel_class f = cls[c];
        Dual co[K_N];
        coefficient_chain<Dual>(f, mk(moist ? (double)moist[k] : f.fuelmc_g, 1.0), co);
        for (int q = 0; q < K_N; ++q) daos[k * K_N + q] = co[q].d;
    }
}

int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 65535 * 8 ? b : 65535 * 8);
}

}  // namespace

template <typename T>
cudaError_t launch_node_coefficients(const fire_fuel_class *classes_dev, int ncls,
                                     const uint8_t *fuel, const void *moist, size_t n,
                                     T *const *planes, double *aos, cudaStream_t s) {
    Planes5<T> pl;
    for (int q = 0; q < 5; ++q) pl.p[q] = planes[q];
    k_node_coefficients<T><<<grid_for(n), 256, 0, s>>>(classes_dev, ncls, fuel,
                                                       static_cast<const T *>(moist), n, pl, aos);
    return cudaGetLastError();
}
template cudaError_t launch_node_coefficients<float>(const fire_fuel_class *, int,
                                                     const uint8_t *, const void *, size_t,
                                                     float *const *, double *, cudaStream_t);
template cudaError_t launch_node_coefficients<double>(const fire_fuel_class *, int,
                                                      const uint8_t *, const void *, size_t,
                                                      double *const *, double *, cudaStream_t);

template <typename T>
cudaError_t launch_node_coefficients_dMf(const fire_fuel_class *classes_dev, int ncls,
                                         const uint8_t *fuel, const void *moist, size_t n,
                                         double *daos, cudaStream_t s) {
    k_node_coefficients_dMf<T><<<grid_for(n), 256, 0, s>>>(classes_dev, ncls, fuel,
                                                           static_cast<const T *>(moist), n, daos);
    return cudaGetLastError();
}
template cudaError_t launch_node_coefficients_dMf<float>(const fire_fuel_class *, int,
                                                         const uint8_t *, const void *, size_t,
                                                         double *, cudaStream_t);
template cudaError_t launch_node_coefficients_dMf<double>(const fire_fuel_class *, int,
                                                          const uint8_t *, const void *, size_t,
                                                          double *, cudaStream_t);

cudaError_t launch_coefficients(const fire_fuel_class *classes_dev, int n, double *coef_dev,
                                cudaStream_t s) {
    k_coefficients<<<(n + 63) / 64, 64, 0, s>>>(classes_dev, n, coef_dev);
    return cudaGetLastError();
}

cudaError_t launch_coefficients_dMf(const fire_fuel_class *classes_dev, int n, double *dcoef_dev,
                                    cudaStream_t s) {
    k_coefficients_dMf<<<(n + 63) / 64, 64, 0, s>>>(classes_dev, n, dcoef_dev);
    return cudaGetLastError();
}

}  // namespace wf
