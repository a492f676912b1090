// Device functions shared by the fire-step kernels: precision-dependent
// math, the extrapolated ghost value, the spread rate of eq.
// (spread-WRF-Fire), the bilinear wind interpolation and the right-hand side
// of eq. (F-disc).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fire_internal.h"

namespace wf {

// Index checks of the checked build (compiled with -DFIRE_BOUNDS_CHECK): an
// index outside [0, n) sets ST_BOUNDS in the status variable st and becomes
// 0, so the access stays inside its buffer and the kernel runs on (no trap,
// the status reports it).  In the normal build WF_CHK(i, n, st) is i.  An
// access of two adjacent elements checks its first index against n - 1.
#ifdef FIRE_BOUNDS_CHECK
__device__ __forceinline__ long long bounds_checked(long long i, long long n, int &st) {
    if (i < 0 || i >= n) {
        st |= ST_BOUNDS;
        return 0;
    }
    return i;
}
#define WF_CHK(i, n, st) (::wf::bounds_checked((long long)(i), (long long)(n), (st)))
// offset off from a row start base (a pointer already advanced by base):
// base + off is checked, the offset returned
#define WF_CHK_AT(base, off, n, st) \
    (::wf::bounds_checked((long long)(base) + (long long)(off), (long long)(n), (st)) - \
     (long long)(base))
#else
#define WF_CHK(i, n, st) (i)
#define WF_CHK_AT(base, off, n, st) (off)
#endif

// ---------------------------------------------------------------------------
// precision-dependent math.  FP32: hardware approximations (the FP32 path is
// held to tolerances on ignition time, burnt area and total heat, not to
// ulps); FP64: the IEEE operations the plain formulas name.
// ---------------------------------------------------------------------------
template <typename T>
struct Mth;

// FP32: the hardware approximations of log2, 2^x, sqrt and 1/sqrt (PTX
// .approx, a few ulp) with subnormal inputs and results flushed to zero, one
// instruction each and no rescaling of subnormals around them
__device__ __forceinline__ float lg2_ftz(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_ftz(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_ftz(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <>
struct Mth<float> {
    static constexpr float kGradZero = 1e-6f;
    // smallest squared norm that unit() normalises (below it the vector is
    // scaled by 1/sqrt of this value and stays shorter than one)
    static constexpr float kNormMin = 1.17549435e-38f;
    // x^b for x >= 0 and b > 0 (the wind exponent of Table 2, 1 for
    // chaparral): 2^(b log2 x), and 2^-inf = 0 at x = 0
    static __device__ __forceinline__ float pw(float x, float b) { return ex2_ftz(b * lg2_ftz(x)); }
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
    // 1 - a/b as one fused multiply-add with the hardware reciprocal (the
    // same rounding wherever it is formed, scalar or packed; b a normal
    // float, as __fdividef wants it)
    static __device__ __forceinline__ float one_minus_div(float a, float b) {
        return fmaf(-a, rcp_ftz(b), 1.0f);
    }
    // x >= 0 (a sum of squares)
    static __device__ __forceinline__ float sqr(float x) { return sqrt_ftz(x); }
    // 1/sqrt(x) for x > 0
    static __device__ __forceinline__ float rsq(float x) { return rsqrt_ftz(x); }
    // unit vector of (cx, cy); zero vector when the norm vanishes
    static __device__ __forceinline__ void unit(float cx, float cy, float &nx, float &ny) {
        const float n2 = fmaf(cx, cx, cy * cy);
        const float r = rsqrt_ftz(fmaxf(n2, kNormMin));
        nx = cx * r;
        ny = cy * r;
    }
};

template <>
struct Mth<double> {
    static constexpr double kGradZero = 1e-9;
    static constexpr double kNormMin = 0.0;
    // x^b for x >= 0 and b > 0 as 2^(b log2 x): fewer FP64 instructions than
    // pow (this part's FP64 pipe bounds the FP64 step), within a few units
    // of 1e-16 relative for the wind speeds and exponents of the model;
    // x^b = 0 at x = 0 (the capped wind component on the upwind side of the
    // front) skips the call, and warps whose nodes all face away from the
    // wind skip it entirely
    static __device__ __forceinline__ double pw(double x, double b) {
        return x > 0.0 ? exp2(b * log2(x)) : 0.0;
    }
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
    static __device__ __forceinline__ double one_minus_div(double a, double b) {
        return 1.0 - a / b;
    }
    static __device__ __forceinline__ double sqr(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
    // unit vector of (cx, cy) (the reciprocal square root of the squared
    // norm, two products); zero vector when the norm vanishes
    static __device__ __forceinline__ void unit(double cx, double cy, double &nx, double &ny) {
        const double n2 = cx * cx + cy * cy;
        if (n2 > 0.0) {
            const double r = rsqrt(n2);
            nx = cx * r;
            ny = cy * r;
        } else {
            nx = 0.0;
            ny = 0.0;
        }
    }
};

// float and double versions of |x|, min and the finiteness test, so that no
// float operand is ever widened to double on the (1/64-rate) FP64 pipe
__device__ __forceinline__ float abs_val(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_val(double x) { return fabs(x); }
__device__ __forceinline__ float min_val(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_val(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ bool finite_val(float x) {
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}
__device__ __forceinline__ bool finite_val(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// extrapolated ghost value beyond the last node p0 (p1 the one before it),
// Sect. 3.1: max{p0 + (p0 - p1), p0, p1}
template <typename T>
__device__ __forceinline__ T ghost_value(T p0, T p1) {
    T g = p0 + (p0 - p1);
    g = p0 > g ? p0 : g;
    g = p1 > g ? p1 : g;
    return g;
}

// eq. (spread-WRF-Fire): S = max{S0, R0 + c min{e, max{0,U}}^b + d max{0,tan}^2}
template <typename T>
__device__ __forceinline__ T spread_rate(const T *co, T U, T tanphi) {
    T Up = U > T(0) ? U : T(0);
    T Ue = Up < co[K_E] ? Up : co[K_E];
    T tp = tanphi > T(0) ? tanphi : T(0);
    T s = co[K_R0] + co[K_C] * Mth<T>::pw(Ue, co[K_B]) + co[K_D] * tp * tp;
    return s > co[K_S0] ? s : co[K_S0];
}

// bilinear weights on points 0..n-1 at coordinate f, clamped to the end points
template <typename T>
__device__ __forceinline__ void lin_idx(T f, int n, int &k0, int &k1, T &w) {
    if (n == 1) {
        k0 = k1 = 0;
        w = T(0);
        return;
    }
    f = f < T(0) ? T(0) : f;
    f = f > T(n - 1) ? T(n - 1) : f;
    int k = (int)floor(f);
    k = k > n - 2 ? n - 2 : k;
    k = k < 0 ? 0 : k;
    k0 = k;
    k1 = k + 1;
    w = f - T(k);
}

// horizontal bilinear interpolation of the staggered wind to fire node
// (gx, gy) (Sect. 5, wind paragraph): u at (I, J+1/2), v at (I+1/2, J)
template <typename T>
__device__ __forceinline__ void wind_at(const T *__restrict__ u, const T *__restrict__ v,
                                        int nxa, int nya, int srx, int sry, int gx, int gy,
                                        T &un, T &vn, int &st) {
    T xa = (T(gx) + T(0.5)) / T(srx);
    T ya = (T(gy) + T(0.5)) / T(sry);
    int i0, i1, j0, j1;
    T wx, wy;
    lin_idx<T>(xa, nxa + 1, i0, i1, wx);
    lin_idx<T>(ya - T(0.5), nya, j0, j1, wy);
    const long long nu = (long long)nya * (nxa + 1);
    const size_t b0 = (size_t)j0 * (nxa + 1), b1 = (size_t)j1 * (nxa + 1);
    un = (T(1) - wy) * ((T(1) - wx) * __ldg(u + WF_CHK(b0 + i0, nu, st)) +
                        wx * __ldg(u + WF_CHK(b0 + i1, nu, st))) +
         wy * ((T(1) - wx) * __ldg(u + WF_CHK(b1 + i0, nu, st)) +
               wx * __ldg(u + WF_CHK(b1 + i1, nu, st)));
    lin_idx<T>(xa - T(0.5), nxa, i0, i1, wx);
    lin_idx<T>(ya, nya + 1, j0, j1, wy);
    const long long nv = (long long)(nya + 1) * nxa;
    const size_t c0 = (size_t)j0 * nxa, c1 = (size_t)j1 * nxa;
    vn = (T(1) - wy) * ((T(1) - wx) * __ldg(v + WF_CHK(c0 + i0, nv, st)) +
                        wx * __ldg(v + WF_CHK(c0 + i1, nv, st))) +
         wy * ((T(1) - wx) * __ldg(v + WF_CHK(c1 + i0, nv, st)) +
               wx * __ldg(v + WF_CHK(c1 + i1, nv, st)));
}

// Right-hand side of eq. (F-disc) at a node from its value p and its four
// neighbours (left, right, down, up): Godunov upwinded norm (eq. Godunov; its
// square is max(max(D-,0)^2, min(D+,0)^2)), normal from central differences,
// spread rate from the normal wind and slope, scaled Laplacian, viscosity
// eps*S*Lap.
template <typename T>
__device__ __forceinline__ T rhs_vals(T p, T pl, T pr, T pd, T pu, T idx, T idy, T i2dx, T i2dy,
                                      T eps, const T *co, T m, T un, T vn, T zx, T zy) {
    T dxm = (p - pl) * idx, dxp = (pr - p) * idx;
    T dym = (p - pd) * idy, dyp = (pu - p) * idy;
    T ax = dxm > T(0) ? dxm : T(0), bx = dxp < T(0) ? dxp : T(0);
    T ay = dym > T(0) ? dym : T(0), by = dyp < T(0) ? dyp : T(0);
    T gx2 = ax * ax > bx * bx ? ax * ax : bx * bx;
    T gy2 = ay * ay > by * by ? ay * ay : by * by;
    // a central difference at the rounding level of its two values counts
    // as zero: rounding noise at a symmetric point must not pick the normal
    T ddx = pr - pl, ddy = pu - pd;
    ddx = abs_val(ddx) <= Mth<T>::kGradZero * (abs_val(pr) + abs_val(pl)) ? T(0) : ddx;
    ddy = abs_val(ddy) <= Mth<T>::kGradZero * (abs_val(pu) + abs_val(pd)) ? T(0) : ddy;
    T nxv, nyv;
    Mth<T>::unit(ddx * i2dx, ddy * i2dy, nxv, nyv);
    T U = un * nxv + vn * nyv;
    T tp = zx * nxv + zy * nyv;
    T S = m * spread_rate<T>(co, U, tp);
    T lap = (dxp - dxm) + (dyp - dym);
    T grad = Mth<T>::sqr(gx2 + gy2);
    return -S * grad + eps * S * lap;
}

// the same at index c of a staged field B of row pitch W
template <typename T>
__device__ __forceinline__ T rhs_at(const T *B, int c, int W, T idx, T idy, T i2dx, T i2dy,
                                    T eps, const T *co, T m, T un, T vn, T zx, T zy) {
    return rhs_vals<T>(B[c], B[c - 1], B[c + 1], B[c - W], B[c + W], idx, idy, i2dx, i2dy, eps,
                       co, m, un, vn, zx, zy);
}


// an unset ignition time (+inf), tested on the bits (no FP64 instruction)
__device__ __forceinline__ bool tign_unset(double ti) {
    return ((unsigned long long)__double_as_longlong(ti) & 0x7fffffffffffffffull) ==
           0x7ff0000000000000ull;
}

// burned fraction of one subcell from its 4 vertex values (eqs. approx-area,
// approx-fraction with the exponent -(1/4) sum (t - t_i)/T_f)
template <typename T>
__device__ __forceinline__ T subcell_burned(T p0, T p1, T p2, T p3, T d0, T d1, T d2, T d3,
                                            T mquarter_over_tf) {
    T sp = ((p0 + p1) + p2) + p3;
    T sa = ((abs_val(p0) + abs_val(p1)) + abs_val(p2)) + abs_val(p3);
    T beta = sa > T(0) ? T(0.5) * Mth<T>::one_minus_div(sp, sa) : T(0);
    T s = ((d0 + d1) + d2) + d3;
    return beta * (T(1) - Mth<T>::ex(s * mquarter_over_tf));
}

// Fuel fraction of a cell from the 3x3 node neighbourhood of psi^{n+1}
// (pba = node (i + a - 1, j + b - 1)) and Dl = t - t_i (0 where psi >= 0)
// (Sect. 3.3, Fig. subcells): 9 vertices (centre, 4 edge midpoints = 2-node
// means, 4 corners = 4-node means), Dl zeroed where the interpolated psi >= 0,
// 4 subcells.
template <typename T>
__device__ __forceinline__ T cell_fraction_vals(T p00, T p01, T p02, T p10, T p11, T p12, T p20,
                                                T p21, T p22, T d00, T d01, T d02, T d10, T d11,
                                                T d12, T d20, T d21, T d22, T Tf) {
    T mn = min_val(min_val(min_val(p00, p01), min_val(p02, p10)),
                   min_val(min_val(p11, p12), min_val(min_val(p20, p21), p22)));
    if (mn >= T(0)) return T(1);  // no vertex burning: every beta is 0 exactly
    const T h = T(0.5), q = T(0.25);
    // edge midpoints W, E, S, N and corners SW, SE, NW, NE
    T pW = h * (p10 + p11), pE = h * (p11 + p12), pS = h * (p01 + p11), pN = h * (p11 + p21);
    T dW = h * (d10 + d11), dE = h * (d11 + d12), dS = h * (d01 + d11), dN = h * (d11 + d21);
    T pSW = q * (((p00 + p01) + p10) + p11), pSE = q * (((p01 + p02) + p11) + p12);
    T pNW = q * (((p10 + p11) + p20) + p21), pNE = q * (((p11 + p12) + p21) + p22);
    T dSW = q * (((d00 + d01) + d10) + d11), dSE = q * (((d01 + d02) + d11) + d12);
    T dNW = q * (((d10 + d11) + d20) + d21), dNE = q * (((d11 + d12) + d21) + d22);
    // compatibility at the vertices: t_i := t where psi >= 0
    T dC = p11 >= T(0) ? T(0) : d11;
    dW = pW >= T(0) ? T(0) : dW;
    dE = pE >= T(0) ? T(0) : dE;
    dS = pS >= T(0) ? T(0) : dS;
    dN = pN >= T(0) ? T(0) : dN;
    dSW = pSW >= T(0) ? T(0) : dSW;
    dSE = pSE >= T(0) ? T(0) : dSE;
    dNW = pNW >= T(0) ? T(0) : dNW;
    dNE = pNE >= T(0) ? T(0) : dNE;
    const T k = T(-0.25) / Tf;
    T bSW = subcell_burned<T>(p11, pW, pS, pSW, dC, dW, dS, dSW, k);
    T bSE = subcell_burned<T>(p11, pE, pS, pSE, dC, dE, dS, dSE, k);
    T bNW = subcell_burned<T>(p11, pW, pN, pNW, dC, dW, dN, dNW, k);
    T bNE = subcell_burned<T>(p11, pE, pN, pNE, dC, dE, dN, dNE, k);
    // one fused multiply-add, as in the packed two-cell version
    return fma(-q, ((bSW + bSE) + bNW) + bNE, T(1));
}

// ---------------------------------------------------------------------------
// The fuel-fraction scheme exact for linear psi and t - t_i (the
// alternative of the Discussion, which names the property, not a formula):
// the cell's 8 triangles (each subcell split along its centre-corner
// diagonal) carry the linear interpolants of the 9 vertex values, each is
// clipped to psi <= 0 (t - t_i = 0 on the cut, eq. ti-comp) and
// 1 - exp(-(t - t_i)/T_f) is integrated exactly over the clipped part.
// Nodes not yet ignited extend t - t_i as -lambda psi, lambda fitted on the
// neighbourhood's burning nodes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float expm1_t(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_t(double x) { return expm1(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

// (e^a - e^b)/(a - b), e^a at a == b
template <typename T>
__device__ __forceinline__ T dd1_exp(T a, T b) {
    const T d = a - b;
    if (d == T(0)) return exp_t(a);
    return exp_t(b) * (expm1_t(d) / d);
}

// second divided difference of exp: the integral of exp over a triangle with
// vertex values a, b, c is 2 area dd2_exp(a, b, c); a series in the spreads
// below a spread of 1, differences of dd1 above
template <typename T>
__device__ __forceinline__ T dd2_exp(T a, T b, T c) {
    T x0 = a, x1 = b, x2 = c, tmp;
    if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
    if (x1 > x2) { tmp = x1; x1 = x2; x2 = tmp; }
    if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
    const T R = x2 - x0;
    if (R < T(1)) {
        // sum over k of h_k(u, v)/(k+2)!, h_k the complete homogeneous
        // polynomial of degree k (h_k = u h_{k-1} + v^k)
        constexpr int K = sizeof(T) == 8 ? 24 : 12;
        const T u = x1 - x0, v = x2 - x0;
        T sum = T(0), h = T(1), vk = T(1), inv = T(0.5);
        for (int k = 0; k <= K; ++k) {
            if (k > 0) {
                vk *= v;
                h = u * h + vk;
            }
            sum += h * inv;
            inv /= T(k + 3);
        }
        return exp_t(x0) * sum;
    }
    return (dd1_exp<T>(x0, x1) - dd1_exp<T>(x1, x2)) / (x0 - x2);
}

// integral of 1 - exp(-D/Tf) over the part psi <= 0 of a triangle
template <typename T>
__device__ __forceinline__ T tri_burn(const T *x, const T *y, const T *ps, const T *ds, T Tf) {
    T px[4], py[4], pd[4];
    int m = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = k == 2 ? 0 : k + 1;
        if (ps[k] <= T(0)) {
            px[m] = x[k];
            py[m] = y[k];
            pd[m] = ds[k];
            ++m;
        }
        if ((ps[k] < T(0) && ps[q] > T(0)) || (ps[k] > T(0) && ps[q] < T(0))) {
            const T s = ps[k] / (ps[k] - ps[q]);
            px[m] = x[k] + s * (x[q] - x[k]);
            py[m] = y[k] + s * (y[q] - y[k]);
            pd[m] = T(0);
            ++m;
        }
    }
    T total = T(0);
    for (int k = 1; k + 1 < m; ++k) {
        const T ar = T(0.5) * abs_val((px[k] - px[0]) * (py[k + 1] - py[0]) -
                                      (px[k + 1] - px[0]) * (py[k] - py[0]));
        if (ar == T(0)) continue;
        total += ar - T(2) * ar * dd2_exp<T>(-pd[0] / Tf, -pd[k] / Tf, -pd[k + 1] / Tf);
    }
    return total;
}

// The cell's fuel fraction from the 3x3 node values of psi (p, row-major,
// [4] the cell's node) and of D = t - t_i (0 where psi >= 0)
template <typename T>
__device__ __forceinline__ T cell_fraction_linear_vals(const T *p, const T *D, T Tf) {
    T sD = T(0), sP = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k)
        if (p[k] < T(0)) {
            sD += D[k];
            sP += -p[k];
        }
    if (!(sP > T(0))) return T(1);
    const T lambda = sD / sP;
    T dn[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) dn[k] = p[k] < T(0) ? D[k] : -lambda * p[k];
    T vp[3][3], vd[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ia0 = a == 0 ? 0 : 1, ia1 = a == 2 ? 2 : 1;
            const int ib0 = b == 0 ? 0 : 1, ib1 = b == 2 ? 2 : 1;
            vp[b][a] = T(0.25) * ((p[ib0 * 3 + ia0] + p[ib0 * 3 + ia1]) +
                                  (p[ib1 * 3 + ia0] + p[ib1 * 3 + ia1]));
            vd[b][a] = T(0.25) * ((dn[ib0 * 3 + ia0] + dn[ib0 * 3 + ia1]) +
                                  (dn[ib1 * 3 + ia0] + dn[ib1 * 3 + ia1]));
        }
    T burned = T(0);
#pragma unroll
    for (int sb = 0; sb < 2; ++sb)
#pragma unroll
        for (int sa = 0; sa < 2; ++sa) {
            const int ax = 2 * sa, by = 2 * sb;
            const T kx = T(ax - 1), ky = T(by - 1);
            const T x1[3] = {T(0), T(0.5) * kx, T(0.5) * kx}, y1[3] = {T(0), T(0), T(0.5) * ky};
            const T p1[3] = {vp[1][1], vp[1][ax], vp[by][ax]};
            const T d1[3] = {vd[1][1], vd[1][ax], vd[by][ax]};
            const T x2[3] = {T(0), T(0.5) * kx, T(0)}, y2[3] = {T(0), T(0.5) * ky, T(0.5) * ky};
            const T p2[3] = {vp[1][1], vp[by][ax], vp[by][1]};
            const T d2[3] = {vd[1][1], vd[by][ax], vd[by][1]};
            burned += tri_burn<T>(x1, y1, p1, d1, Tf) + tri_burn<T>(x2, y2, p2, d2, Tf);
        }
    return T(1) - burned;
}

}  // namespace wf
