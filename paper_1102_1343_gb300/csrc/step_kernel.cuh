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
#include <mutex>
#include <math.h>
#include <stdint.h>

#include "fire_device.cuh"
#include "fire_internal.h"

namespace wf {

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

// Fuel fraction of the cell at index c of the staged psi^{n+1} (P) and
// Dl = t - t_i (row pitch W).
template <typename T>
__device__ __forceinline__ T cell_fraction(const T *P, const T *Dl, int c, int W, T Tf) {
    return cell_fraction_vals<T>(P[c - W - 1], P[c - W], P[c - W + 1], P[c - 1], P[c], P[c + 1],
                                 P[c + W - 1], P[c + W], P[c + W + 1], Dl[c - W - 1], Dl[c - W],
                                 Dl[c - W + 1], Dl[c - 1], Dl[c], Dl[c + 1], Dl[c + W - 1],
                                 Dl[c + W], Dl[c + W + 1], Tf);
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
    // per-node R0, c, d, H_s, H_q of a per-node fuel moisture (all null
    // otherwise): they replace the class values
    const T *__restrict__ nR0 = static_cast<const T *>(a.nco[0]);
    const T *__restrict__ nc = static_cast<const T *>(a.nco[1]);
    const T *__restrict__ nd = static_cast<const T *>(a.nco[2]);
    const T *__restrict__ nhs = static_cast<const T *>(a.nco[3]);
    const T *__restrict__ nhq = static_cast<const T *>(a.nco[4]);
    auto node_coef = [&](int cls, size_t g, T *cn) {
#pragma unroll
        for (int q = 0; q < 6; ++q) cn[q] = lut[cls * K_N + q];
        if (nR0) {
            cn[K_R0] = nR0[g];
            cn[K_C] = nc[g];
            cn[K_D] = nd[g];
        }
    };

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

    int st = 0;
    // ---- A: psi^n on the tile + 3 halo (0 outside the domain)
    for (int ly = ty; ly < BH3; ly += kThreadsY) {
        const int gy = y0 - 3 + ly;
        const bool rowin = gy >= 0 && gy < ny;
        for (int lx = tx; lx < BW3; lx += kThreadsX) {
            const int gx = x0 - 3 + lx;
            T val = T(0);
            if (rowin && gx >= 0 && gx < nx) val = psi_in[WF_CHK((size_t)gy * nx + gx, (long long)nx * ny, st)];
            P0[ly * BW3 + lx] = val;
        }
    }
    __syncthreads();
    const bool edge_tile = (x0 - 3 < 0) || (y0 - 3 < 0) || (x0 + TX + 3 > nx) || (y0 + TY + 3 > ny);
    if (edge_tile) fill_ghosts<T>(P0, BW3, BH3, x0 - 3, y0 - 3, nx, ny, tid);

    // ---- C: stage 1 on the tile + 2 halo: F1 = F(psi^n), psi* = psi^n + dt F1
    for (int ly = ty; ly < BH2; ly += kThreadsY) {
        const int gy = y0 - 2 + ly;
        for (int lx = tx; lx < BW2; lx += kThreadsX) {
            const int gx = x0 - 2 + lx;
            if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) {
                P1[ly * BW2 + lx] = T(0);
                continue;
            }
            const size_t g = WF_CHK((size_t)gy * nx + gx, (long long)nx * ny, st);
            int cls = fuel[g];
            cls = cls > ncm1 ? ncm1 : cls;
            T un, vn;
            wind_at<T>(wu, wv, a.nxa, a.nya, srx, sry, gx, gy, un, vn, st);
            if (!finite_val(un) || !finite_val(vn)) st |= ST_NONFINITE;
            const T m = mult ? mult[g] : T(1);
            const int c = (ly + 1) * BW3 + (lx + 1);
            T cn[6];
            node_coef(cls, g, cn);
            const T F = rhs_at<T>(P0, c, BW3, idx, idy, i2dx, i2dy, eps, cn, m, un, vn, dzdx[g],
                                  dzdy[g]);
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
            const size_t g = WF_CHK((size_t)gy * nx + gx, (long long)nx * ny, st);
            int cls = fuel[g];
            cls = cls > ncm1 ? ncm1 : cls;
            T un, vn;
            wind_at<T>(wu, wv, a.nxa, a.nya, srx, sry, gx, gy, un, vn, st);
            const T m = mult ? mult[g] : T(1);
            T cn[6];
            node_coef(cls, g, cn);
            const T F2 = rhs_at<T>(P1, (ly + 1) * BW2 + (lx + 1), BW2, idx, idy, i2dx, i2dy, eps,
                                   cn, m, un, vn, dzdx[g], dzdy[g]);
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
                if (!finite_val(pn)) st |= ST_NONFINITE;
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
                const size_t g = WF_CHK((size_t)gy * nx + gx, (long long)nx * ny, st);
                int cls = fuel[g];
                cls = cls > ncm1 ? ncm1 : cls;
                const T *co = lut + cls * K_N;
                const int cc = (ly + 1) * BW1 + (lx + 1);
                T Fn;
                if (a.scheme == 1) {
                    T p9[9], d9[9];
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int h = 0; h < 3; ++h) {
                            p9[b * 3 + h] = P2[cc + (b - 1) * BW1 + (h - 1)];
                            d9[b * 3 + h] = Dl[cc + (b - 1) * BW1 + (h - 1)];
                        }
                    Fn = cell_fraction_linear_vals<T>(p9, d9, co[K_TF]);
                } else {
                    Fn = cell_fraction<T>(P2, Dl, cc, BW1, co[K_TF]);
                }
                const T Fo = F_in[g];
                F_out[g] = Fn;
                const T dF = Fo - Fn;
                hs = dF * (nhs ? nhs[g] : co[K_HS]);
                hq = dF * (nhq ? nhq[g] : co[K_HQ]);
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
        int sth = 0;
        const size_t ga = WF_CHK((size_t)(y0 / sry + J) * a.nxa + (x0 / srx + I),
                                 (long long)a.nxa * a.nya, sth);
        if (a.heat_s) a.heat_s[ga] = h0 * scale;
        if (a.heat_l) a.heat_l[ga] = h1 * scale;
        if (sth) atomicOr(a.status, sth);
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
            // FP32 prefilter (offsets taken in double, then rounded): skip the
            // segment only when the exact test below can change neither psi
            // (needs dist < psi + rho) nor the ignition time (dist <= rho);
            // delta bounds the FP32 error of the distance
            {
                const float qx = (float)(x - s.ax), qy = (float)(y - s.ay);
                const float sx = (float)(s.bx - s.ax), sy = (float)(s.by - s.ay);
                const float L2f = sx * sx + sy * sy;
                float u = L2f > 0.0f ? (qx * sx + qy * sy) / L2f : 0.0f;
                u = fminf(fmaxf(u, 0.0f), 1.0f);
                const float rx = qx - u * sx, ry = qy - u * sy;
                const float d2 = rx * rx + ry * ry;
                const float delta = 4e-7f * (fabsf(qx) + fabsf(qy) + fabsf(sx) + fabsf(sy)) + 1e-6f;
                const float lim = (float)((double)p + s.rho);
                const float dl = lim + delta + 1e-6f * fabsf(lim);
                const float rho = (float)s.rho;
                const float dr = rho + delta + 1e-6f * rho;
                const bool may_min = dl > 0.0f && d2 <= dl * dl;
                const bool may_ti = (double)p > 0.0 && isinf(ti) && d2 <= dr * dr;
                if (!may_min && !may_ti) continue;
            }
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
                if (s.drip) {
                    // the fire starts at the nearest point when the torch
                    // lays it and reaches the node at S_g, by t at the latest
                    const double ta = (s.tg + u * (s.tlay - s.tg)) + d / s.sg;
                    ti = ta < s.tnow ? ta : s.tnow;
                } else {
                    ti = s.sg > 0.0 ? s.tg + d / s.sg : s.tg;
                }
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

// raised monotonically: the limit is shared by every context in the process
template <typename T>
cudaError_t prepare_step_kernel(size_t smem_bytes) {
    static std::mutex mu;
    static size_t current[kMaxDevices] = {};  // per device (the attribute is)
    std::lock_guard<std::mutex> lock(mu);
    const int dev = attr_device();
    if (dev >= 0 && smem_bytes <= current[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fire_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e == cudaSuccess && dev >= 0) current[dev] = smem_bytes;
    return e;
}

template <typename T>
cudaError_t launch_step(const StepArgs &a, cudaStream_t s) {
    const int TX = a.kx * a.srx, TY = a.ky * a.sry;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    dim3 block(kThreadsX, kThreadsY);
    size_t smem = step_smem_bytes<T>(a.kx, a.ky, a.srx, a.sry, a.ncls);
    cudaError_t e = prepare_step_kernel<T>(smem);
    if (e != cudaSuccess) return e;
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
