// Fused fire-step kernel (Sect. 5 items 2-6 of the paper) and the
// element-wise ignition / initialisation kernels, templated on the path
// precision T (float or double).  Included by step_f32.cu and step_f64.cu.
//
// One CTA owns a tile of kx x ky atmospheric cells = TX x TY fire nodes
// (TX = kx*srx, TY = ky*sry), so every atmospheric cell's heat average is
// reduced inside one CTA, deterministically.  The CTA stages the level-set
// function psi^n of its tile plus a 3-node halo in shared memory and runs
// the whole step there:
//   stage 1 (eq. Heun, first line)  on the tile + 2 halo -> psi*
//   stage 2 (eq. Heun, second line) on the tile + 1 halo -> psi^{n+1}
//   ignition-time crossing (eq. set-ignition-time) on the tile + 1 halo
//   fuel-fraction quadrature (Sect. 3.3) on the tile, which needs psi^{n+1}
//   and the compatible ignition time on the 3x3 neighbourhood
//   heat fluxes (eqs. sensible-/latent-heat-flux) and their average over the
//   tile's atmospheric cells (Sect. 5, item 6)
// The halo is recomputed redundantly by neighbouring CTAs, so one step costs
// one pass over the state in HBM.  Ghost nodes beyond the domain follow the
// extrapolation of Sect. 3.1 (x first, then y), recomputed for each stage.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fire_internal.h"

namespace wf {

// ---------------------------------------------------------------------------
// precision-dependent math.  FP32: hardware approximations (the FP32 path is
// judged on ignition time, burnt area and total heat, not ulps); FP64: the
// IEEE operations the plain formulas name.
// ---------------------------------------------------------------------------
template <typename T>
struct Mth;

template <>
struct Mth<float> {
    static __device__ __forceinline__ float pw(float x, float b) { return __powf(x, b); }
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float sqr(float x) { return sqrtf(x); }
    // unit vector of (cx, cy); zero vector when the norm vanishes
    static __device__ __forceinline__ void unit(float cx, float cy, float &nx, float &ny) {
        float n2 = cx * cx + cy * cy;
        float r = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
        nx = cx * r;
        ny = cy * r;
    }
};

template <>
struct Mth<double> {
    static __device__ __forceinline__ double pw(double x, double b) { return pow(x, b); }
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
    static __device__ __forceinline__ double sqr(double x) { return sqrt(x); }
    static __device__ __forceinline__ void unit(double cx, double cy, double &nx, double &ny) {
        double n = sqrt(cx * cx + cy * cy);
        if (n > 0.0) {
            nx = cx / n;
            ny = cy / n;
        } else {
            nx = 0.0;
            ny = 0.0;
        }
    }
};

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
                                        T &un, T &vn) {
    T xa = (T(gx) + T(0.5)) / T(srx);
    T ya = (T(gy) + T(0.5)) / T(sry);
    int i0, i1, j0, j1;
    T wx, wy;
    lin_idx<T>(xa, nxa + 1, i0, i1, wx);
    lin_idx<T>(ya - T(0.5), nya, j0, j1, wy);
    const T *r0 = u + (size_t)j0 * (nxa + 1);
    const T *r1 = u + (size_t)j1 * (nxa + 1);
    un = (T(1) - wy) * ((T(1) - wx) * __ldg(r0 + i0) + wx * __ldg(r0 + i1)) +
         wy * ((T(1) - wx) * __ldg(r1 + i0) + wx * __ldg(r1 + i1));
    lin_idx<T>(xa - T(0.5), nxa, i0, i1, wx);
    lin_idx<T>(ya, nya + 1, j0, j1, wy);
    r0 = v + (size_t)j0 * nxa;
    r1 = v + (size_t)j1 * nxa;
    vn = (T(1) - wy) * ((T(1) - wx) * __ldg(r0 + i0) + wx * __ldg(r0 + i1)) +
         wy * ((T(1) - wx) * __ldg(r1 + i0) + wx * __ldg(r1 + i1));
}

// Right-hand side of eq. (F-disc) at the node at index c of a staged field B
// of row pitch W: Godunov upwinded norm (eq. Godunov; its square is
// max(max(D-,0)^2, min(D+,0)^2)), normal from central differences, spread
// rate from the normal wind and slope, scaled Laplacian, viscosity eps*S*Lap.
template <typename T>
__device__ __forceinline__ T rhs_at(const T *B, int c, int W, T idx, T idy, T i2dx, T i2dy,
                                    T eps, const T *co, T m, T un, T vn, T zx, T zy) {
    T p = B[c], pl = B[c - 1], pr = B[c + 1], pd = B[c - W], pu = B[c + W];
    T dxm = (p - pl) * idx, dxp = (pr - p) * idx;
    T dym = (p - pd) * idy, dyp = (pu - p) * idy;
    T ax = dxm > T(0) ? dxm : T(0), bx = dxp < T(0) ? dxp : T(0);
    T ay = dym > T(0) ? dym : T(0), by = dyp < T(0) ? dyp : T(0);
    T gx2 = ax * ax > bx * bx ? ax * ax : bx * bx;
    T gy2 = ay * ay > by * by ? ay * ay : by * by;
    T nxv, nyv;
    Mth<T>::unit((pr - pl) * i2dx, (pu - pd) * i2dy, nxv, nyv);
    T U = un * nxv + vn * nyv;
    T tp = zx * nxv + zy * nyv;
    T S = m * spread_rate<T>(co, U, tp);
    T lap = (dxp - dxm) + (dyp - dym);
    T grad = Mth<T>::sqr(gx2 + gy2);
    return -S * grad + eps * S * lap;
}

// Fill the ghost ring of a staged field whose local (0,0) is the global node
// (ox, oy): x-ghost columns for the domain rows, then y-ghost rows over the
// extended columns (corners).  Block-uniform: all threads must call it.
template <typename T>
__device__ void fill_ghosts(T *B, int BW, int BH, int ox, int oy, int nx, int ny, int tid) {
    const int lxl = -1 - ox, lxr = nx - ox;
    const bool hasL = lxl >= 0 && lxl + 2 < BW, hasR = lxr - 2 >= 0 && lxr < BW;
    for (int ly = tid; ly < BH; ly += kThreads) {
        int gy = oy + ly;
        if (gy < 0 || gy >= ny) continue;
        T *row = B + ly * BW;
        if (hasL) row[lxl] = ghost_value<T>(row[lxl + 1], row[lxl + 2]);
        if (hasR) row[lxr] = ghost_value<T>(row[lxr - 1], row[lxr - 2]);
    }
    __syncthreads();
    const int lyb = -1 - oy, lyt = ny - oy;
    const bool hasB = lyb >= 0 && lyb + 2 < BH, hasT = lyt - 2 >= 0 && lyt < BH;
    for (int lx = tid; lx < BW; lx += kThreads) {
        int gx = ox + lx;
        if (gx < -1 || gx > nx) continue;
        if (hasB) B[lyb * BW + lx] = ghost_value<T>(B[(lyb + 1) * BW + lx], B[(lyb + 2) * BW + lx]);
        if (hasT) B[lyt * BW + lx] = ghost_value<T>(B[(lyt - 1) * BW + lx], B[(lyt - 2) * BW + lx]);
    }
    __syncthreads();
}

// Ghosts of psi^{n+1} (as fill_ghosts) and of Dl = t - t_i (compatible
// ignition time): a ghost copies its inner neighbour's value, then is 0
// where the ghost psi >= 0 (eq. ti-comp).
template <typename T>
__device__ void fill_ghosts_pd(T *P, T *Dl, int BW, int BH, int ox, int oy, int nx, int ny,
                               int tid) {
    const int lxl = -1 - ox, lxr = nx - ox;
    const bool hasL = lxl >= 0 && lxl + 2 < BW, hasR = lxr - 2 >= 0 && lxr < BW;
    for (int ly = tid; ly < BH; ly += kThreads) {
        int gy = oy + ly;
        if (gy < 0 || gy >= ny) continue;
        T *row = P + ly * BW;
        T *drow = Dl + ly * BW;
        if (hasL) {
            T g = ghost_value<T>(row[lxl + 1], row[lxl + 2]);
            row[lxl] = g;
            drow[lxl] = g >= T(0) ? T(0) : drow[lxl + 1];
        }
        if (hasR) {
            T g = ghost_value<T>(row[lxr - 1], row[lxr - 2]);
            row[lxr] = g;
            drow[lxr] = g >= T(0) ? T(0) : drow[lxr - 1];
        }
    }
    __syncthreads();
    const int lyb = -1 - oy, lyt = ny - oy;
    const bool hasB = lyb >= 0 && lyb + 2 < BH, hasT = lyt - 2 >= 0 && lyt < BH;
    for (int lx = tid; lx < BW; lx += kThreads) {
        int gx = ox + lx;
        if (gx < -1 || gx > nx) continue;
        if (hasB) {
            T g = ghost_value<T>(P[(lyb + 1) * BW + lx], P[(lyb + 2) * BW + lx]);
            P[lyb * BW + lx] = g;
            Dl[lyb * BW + lx] = g >= T(0) ? T(0) : Dl[(lyb + 1) * BW + lx];
        }
        if (hasT) {
            T g = ghost_value<T>(P[(lyt - 1) * BW + lx], P[(lyt - 2) * BW + lx]);
            P[lyt * BW + lx] = g;
            Dl[lyt * BW + lx] = g >= T(0) ? T(0) : Dl[(lyt - 1) * BW + lx];
        }
    }
    __syncthreads();
}

// burned fraction of one subcell from its 4 vertex values (eqs. approx-area,
// approx-fraction with the exponent -(1/4) sum (t - t_i)/T_f)
template <typename T>
__device__ __forceinline__ T subcell_burned(T p0, T p1, T p2, T p3, T d0, T d1, T d2, T d3,
                                            T mquarter_over_tf) {
    T sp = ((p0 + p1) + p2) + p3;
    T sa = ((fabs(p0) + fabs(p1)) + fabs(p2)) + fabs(p3);
    T beta = sa > T(0) ? T(0.5) * (T(1) - Mth<T>::dv(sp, sa)) : T(0);
    T s = ((d0 + d1) + d2) + d3;
    return beta * (T(1) - Mth<T>::ex(s * mquarter_over_tf));
}

// Fuel fraction of the cell at index c of the staged psi^{n+1} (P) and
// Dl = t - t_i (0 where psi >= 0), row pitch W (Sect. 3.3, Fig. subcells):
// 9 vertices (centre, 4 edge midpoints = 2-node means, 4 corners = 4-node
// means), Dl zeroed where the interpolated psi >= 0, 4 subcells.
template <typename T>
__device__ __forceinline__ T cell_fraction(const T *P, const T *Dl, int c, int W, T Tf) {
    // p[b][a] = node (i + a - 1, j + b - 1)
    T p00 = P[c - W - 1], p01 = P[c - W], p02 = P[c - W + 1];
    T p10 = P[c - 1], p11 = P[c], p12 = P[c + 1];
    T p20 = P[c + W - 1], p21 = P[c + W], p22 = P[c + W + 1];
    T mn = fmin(fmin(fmin(p00, p01), fmin(p02, p10)), fmin(fmin(p11, p12), fmin(fmin(p20, p21), p22)));
    if (mn >= T(0)) return T(1);  // no vertex burning: every beta is 0 exactly
    T d00 = Dl[c - W - 1], d01 = Dl[c - W], d02 = Dl[c - W + 1];
    T d10 = Dl[c - 1], d11 = Dl[c], d12 = Dl[c + 1];
    T d20 = Dl[c + W - 1], d21 = Dl[c + W], d22 = Dl[c + W + 1];
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
    return T(1) - q * (((bSW + bSE) + bNW) + bNE);
}

template <typename T>
__host__ __device__ inline int lut_slots(int ncls) {
    int n = ncls * K_N;
    return (n + 3) & ~3;
}

// ---------------------------------------------------------------------------
// the fused step kernel
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fire_step(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_status;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kThreadsX + tx;
    const int srx = a.srx, sry = a.sry, nx = a.nx, ny = a.ny;
    const int TX = a.kx * srx, TY = a.ky * sry;
    const int BW3 = TX + 6, BH3 = TY + 6;
    const int BW2 = TX + 4, BH2 = TY + 4;
    const int BW1 = TX + 2, BH1 = TY + 2;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int TXa = min(TX, nx - x0), TYa = min(TY, ny - y0);

    T *lut = reinterpret_cast<T *>(smem_raw);
    T *P0 = lut + lut_slots<T>(a.ncls);
    T *P1 = P0 + BW3 * BH3;
    T *F1 = P1 + BW2 * BH2;
    T *P2 = F1 + BW1 * BH1;
    T *Dl = P2 + BW1 * BH1;

    const T *__restrict__ psi_in = static_cast<const T *>(a.psi_in);
    T *__restrict__ psi_out = static_cast<T *>(a.psi_out);
    const T *__restrict__ F_in = static_cast<const T *>(a.F_in);
    T *__restrict__ F_out = static_cast<T *>(a.F_out);
    const T *__restrict__ dzdx = static_cast<const T *>(a.dzdx);
    const T *__restrict__ dzdy = static_cast<const T *>(a.dzdy);
    const T *__restrict__ mult = static_cast<const T *>(a.mult);
    const T *__restrict__ wu = static_cast<const T *>(a.u);
    const T *__restrict__ wv = static_cast<const T *>(a.v);
    const uint8_t *__restrict__ fuel = a.fuel;

    const T dt = T(a.dt);
    const T idx = T(1) / T(a.dx), idy = T(1) / T(a.dy);
    const T i2dx = T(1) / (T(2) * T(a.dx)), i2dy = T(1) / (T(2) * T(a.dy));
    const T eps = T(a.eps);
    const double tstart = *a.t_in;
    const double t1 = tstart + a.dt;
    const int ncm1 = a.ncls - 1;

    if (tid == 0) {
        s_status = 0;
        if (blockIdx.x == 0 && blockIdx.y == 0) *a.t_out = t1;
    }
    for (int k = tid; k < a.ncls * K_N; k += kThreads) lut[k] = T(a.coef[k]);

    // ---- A: psi^n on the tile + 3 halo (0 outside the domain)
    for (int ly = ty; ly < BH3; ly += kThreadsY) {
        const int gy = y0 - 3 + ly;
        const bool rowin = gy >= 0 && gy < ny;
        for (int lx = tx; lx < BW3; lx += kThreadsX) {
            const int gx = x0 - 3 + lx;
            T val = T(0);
            if (rowin && gx >= 0 && gx < nx) val = psi_in[(size_t)gy * nx + gx];
            P0[ly * BW3 + lx] = val;
        }
    }
    __syncthreads();
    const bool edge_tile = (x0 - 3 < 0) || (y0 - 3 < 0) || (x0 + TX + 3 > nx) || (y0 + TY + 3 > ny);
    if (edge_tile) fill_ghosts<T>(P0, BW3, BH3, x0 - 3, y0 - 3, nx, ny, tid);

    int st = 0;
    // ---- C: stage 1 on the tile + 2 halo: F1 = F(psi^n), psi* = psi^n + dt F1
    for (int ly = ty; ly < BH2; ly += kThreadsY) {
        const int gy = y0 - 2 + ly;
        for (int lx = tx; lx < BW2; lx += kThreadsX) {
            const int gx = x0 - 2 + lx;
            if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) {
                P1[ly * BW2 + lx] = T(0);
                continue;
            }
            const size_t g = (size_t)gy * nx + gx;
            int cls = fuel[g];
            cls = cls > ncm1 ? ncm1 : cls;
            T un, vn;
            wind_at<T>(wu, wv, a.nxa, a.nya, srx, sry, gx, gy, un, vn);
            if (!isfinite(un) || !isfinite(vn)) st |= ST_NONFINITE;
            const T m = mult ? mult[g] : T(1);
            const int c = (ly + 1) * BW3 + (lx + 1);
            const T F = rhs_at<T>(P0, c, BW3, idx, idy, i2dx, i2dy, eps, lut + cls * K_N, m, un,
                                  vn, dzdx[g], dzdy[g]);
            P1[ly * BW2 + lx] = P0[c] + dt * F;
            if (lx >= 1 && lx < BW2 - 1 && ly >= 1 && ly < BH2 - 1) F1[(ly - 1) * BW1 + (lx - 1)] = F;
        }
    }
    __syncthreads();
    if (edge_tile) fill_ghosts<T>(P1, BW2, BH2, x0 - 2, y0 - 2, nx, ny, tid);

    // ---- E: stage 2 on the tile + 1 halo, ignition-time crossing, Dl = t1 - t_i
    for (int ly = ty; ly < BH1; ly += kThreadsY) {
        const int gy = y0 - 1 + ly;
        for (int lx = tx; lx < BW1; lx += kThreadsX) {
            const int gx = x0 - 1 + lx;
            const int l1 = ly * BW1 + lx;
            if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) {
                P2[l1] = T(0);
                Dl[l1] = T(0);
                continue;
            }
            const size_t g = (size_t)gy * nx + gx;
            int cls = fuel[g];
            cls = cls > ncm1 ? ncm1 : cls;
            T un, vn;
            wind_at<T>(wu, wv, a.nxa, a.nya, srx, sry, gx, gy, un, vn);
            const T m = mult ? mult[g] : T(1);
            const T F2 = rhs_at<T>(P1, (ly + 1) * BW2 + (lx + 1), BW2, idx, idy, i2dx, i2dy, eps,
                                   lut + cls * K_N, m, un, vn, dzdx[g], dzdy[g]);
            const T p0 = P0[(ly + 2) * BW3 + (lx + 2)];
            const T pn = p0 + dt * (T(0.5) * F1[l1] + T(0.5) * F2);
            P2[l1] = pn;
            const bool own = lx >= 1 && lx <= TXa && ly >= 1 && ly <= TYa;
            T d = T(0);
            const bool cross = p0 > T(0) && pn <= T(0);
            if (cross || pn < T(0)) {
                double ti = a.tign[g];
                if (cross && isinf(ti)) {
                    const double q0 = (double)p0, q1 = (double)pn;
                    ti = tstart + q0 * a.dt / (q0 - q1);
                    if (own) a.tign[g] = ti;
                }
                if (pn < T(0)) d = T(t1 - ti);
            }
            Dl[l1] = d;
            if (own) {
                psi_out[g] = pn;
                if (!isfinite(pn)) st |= ST_NONFINITE;
                const bool band = gx < a.band || gy < a.band || gx >= nx - a.band || gy >= ny - a.band;
                if (band && pn < T(0)) st |= ST_BOUNDARY;
            }
        }
    }
    __syncthreads();
    if (edge_tile) fill_ghosts_pd<T>(P2, Dl, BW1, BH1, x0 - 1, y0 - 1, nx, ny, tid);

    // ---- G: fuel fraction on the tile, heat contributions dF * H per node
    T *Q = P0;  // P0/P1 are dead: 2 values per tile node
    for (int ly = ty; ly < TY; ly += kThreadsY) {
        const int gy = y0 + ly;
        for (int lx = tx; lx < TX; lx += kThreadsX) {
            T hs = T(0), hq = T(0);
            if (lx < TXa && ly < TYa) {
                const int gx = x0 + lx;
                const size_t g = (size_t)gy * nx + gx;
                int cls = fuel[g];
                cls = cls > ncm1 ? ncm1 : cls;
                const T *co = lut + cls * K_N;
                const T Fn = cell_fraction<T>(P2, Dl, (ly + 1) * BW1 + (lx + 1), BW1, co[K_TF]);
                const T Fo = F_in[g];
                F_out[g] = Fn;
                const T dF = Fo - Fn;
                hs = dF * co[K_HS];
                hq = dF * co[K_HQ];
            }
            Q[2 * (ly * TX + lx)] = hs;
            Q[2 * (ly * TX + lx) + 1] = hq;
        }
    }
    if (st) atomicOr(&s_status, st);
    __syncthreads();

    // ---- H: average over the atmospheric cells of the tile (Sect. 5, item 6)
    T *Sg = P2;  // P2/Dl are dead: 2 values per row segment of srx nodes
    const int nseg = TY * a.kx;
    for (int sgi = tid; sgi < nseg; sgi += kThreads) {
        const int row = sgi / a.kx, I = sgi - row * a.kx;
        const T *qr = Q + 2 * (row * TX + I * srx);
        T s0 = T(0), s1 = T(0);
        for (int k = 0; k < srx; ++k) {
            s0 += qr[2 * k];
            s1 += qr[2 * k + 1];
        }
        Sg[2 * sgi] = s0;
        Sg[2 * sgi + 1] = s1;
    }
    __syncthreads();
    const int kxa = TXa / srx, kya = TYa / sry;
    const double scale = 1.0 / (a.dt * (double)srx * (double)sry);
    for (int cell = tid; cell < a.kx * a.ky; cell += kThreads) {
        const int J = cell / a.kx, I = cell - J * a.kx;
        if (I >= kxa || J >= kya) continue;
        double h0 = 0.0, h1 = 0.0;
        for (int rr = 0; rr < sry; ++rr) {
            const T *s = Sg + 2 * ((J * sry + rr) * a.kx + I);
            if (s[0] != T(0)) h0 += (double)s[0];
            if (s[1] != T(0)) h1 += (double)s[1];
        }
        const size_t ga = (size_t)(y0 / sry + J) * a.nxa + (x0 / srx + I);
        if (a.heat_s) a.heat_s[ga] = h0 * scale;
        if (a.heat_l) a.heat_l[ga] = h1 * scale;
    }
    if (tid == 0 && s_status) atomicOr(a.status, s_status);
}

// ---------------------------------------------------------------------------
// ignition (Sect. 3.4): psi := min(psi, dist - rho) for each segment in
// order; newly ignited nodes (psi > 0 >= psi_g, no ignition time yet) get
// the arrival time.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_ignite(const IgniteArgs a) {
    const size_t n = (size_t)a.nx * a.ny;
    T *psi = static_cast<T *>(a.psi);
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < n;
         g += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(g / a.nx), i = (int)(g - (size_t)j * a.nx);
        T p = psi[g];
        double ti = a.tign[g];
        const double x = ((double)i + 0.5) * a.dx, y = ((double)j + 0.5) * a.dy;
        bool changed = false, tchanged = false;
        for (int q = 0; q < a.nseg; ++q) {
            const IgnSeg &s = a.seg[q];
            const double dxs = s.bx - s.ax, dys = s.by - s.ay;
            const double qx = x - s.ax, qy = y - s.ay;
            const double L2 = dxs * dxs + dys * dys;
            double u = 0.0;
            if (L2 > 0.0) {
                u = (qx * dxs + qy * dys) / L2;
                u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
            }
            const double rx = qx - u * dxs, ry = qy - u * dys;
            const double d = sqrt(rx * rx + ry * ry);
            const double pg = d - s.rho;
            if ((double)p > 0.0 && pg <= 0.0 && isinf(ti)) {
                ti = s.sg > 0.0 ? s.tg + d / s.sg : s.tg;
                tchanged = true;
            }
            if (pg < (double)p) {
                p = T(pg);
                changed = true;
            }
        }
        if (changed) psi[g] = p;
        if (tchanged) a.tign[g] = ti;
    }
}

template <typename T>
__global__ void k_fill(T *psi, double *tign, T *frac, size_t n, T psi_far) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        psi[k] = psi_far;
        tign[k] = __longlong_as_double(0x7ff0000000000000ULL);  // +inf
        frac[k] = T(1);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T>
size_t step_smem_bytes(int kx, int ky, int srx, int sry, int ncls) {
    const size_t TX = (size_t)kx * srx, TY = (size_t)ky * sry;
    size_t n = lut_slots<T>(ncls) + (TX + 6) * (TY + 6) + (TX + 4) * (TY + 4) + 3 * (TX + 2) * (TY + 2);
    return n * sizeof(T);
}

template <typename T>
cudaError_t prepare_step_kernel(size_t smem_bytes) {
    return cudaFuncSetAttribute(k_fire_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

template <typename T>
cudaError_t launch_step(const StepArgs &a, cudaStream_t s) {
    const int TX = a.kx * a.srx, TY = a.ky * a.sry;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    dim3 block(kThreadsX, kThreadsY);
    size_t smem = step_smem_bytes<T>(a.kx, a.ky, a.srx, a.sry, a.ncls);
    k_fire_step<T><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ignite(const IgniteArgs &a, cudaStream_t s) {
    const size_t n = (size_t)a.nx * a.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_ignite<T><<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill(void *psi, double *tign, void *frac, size_t n, double psi_far,
                        cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_fill<T><<<blocks, 256, 0, s>>>(static_cast<T *>(psi), tign, static_cast<T *>(frac), n,
                                     T(psi_far));
    return cudaGetLastError();
}

#define WF_INSTANTIATE(T)                                                                     \
    template size_t step_smem_bytes<T>(int, int, int, int, int);                              \
    template cudaError_t prepare_step_kernel<T>(size_t);                                      \
    template cudaError_t launch_step<T>(const StepArgs &, cudaStream_t);                      \
    template cudaError_t launch_ignite<T>(const IgniteArgs &, cudaStream_t);                  \
    template cudaError_t launch_fill<T>(void *, double *, void *, size_t, double, cudaStream_t);

}  // namespace wf
