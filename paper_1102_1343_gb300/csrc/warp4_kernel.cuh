// Warp-marching fire-step kernel with four columns per lane (FP32): the
// whole step of Sect. 5 (items 2-6) in one pass over the state, each warp
// marching alone down a strip of W <= 120 output columns.
//
// Lane l holds the four columns xa .. xa + 3, xa = x0 - 4 + 4 l, as two
// float2 pairs, so the warp computes the 128 columns x0 - 4 .. x0 + 123:
// the strip and four columns on each side.  One step reads psi^n three
// columns out (stage 1, stage 2, quadrature), so the warp's own lanes hold
// every value it needs: no extra halo loads; the outermost columns on each
// side take wrap-around neighbours from the shuffles and are never read.
// The per-row work that does not depend on the number of columns (row
// addressing, clamps, range tests, votes, branches, loop control) is shared
// by four columns instead of two; the arithmetic of the right-hand side is
// the packed f32x2 form of the two-column kernel, applied to both pairs.
// Per row (iteration k), as in the two-column kernel:
//   B  stage 1 (eq. Heun, first line) on row k+1
//   C  stage 2 (eq. Heun, second line), ignition-time crossing
//      (eq. set-ignition-time) and t - t_i on row k
//   D  fuel-fraction quadrature (Sect. 3.3) and heat flux
//      (eqs. sensible-/latent-heat-flux) on row k-1
// Shared memory: the class tables, the wind-row weights of the CTA's rows,
// the x-interpolation weights of each warp's 128 columns and a per-warp heat
// buffer.  Rows are read as float4 where the mesh width and the strip origin
// are multiples of 4 (16-byte aligned), else as float2 pairs or scalars.
#pragma once

#include "fire_device.cuh"
#include "fire_internal.h"
#include "pair_math.cuh"
#include "warp_kernel.cuh"

namespace wf {

constexpr int kWarp4CtaThreads = 32 * kWarpStrips;
constexpr int kWarp4Cols = 128;  // columns a warp computes

struct W4Col {  // x-interpolation of the wind for one column
    int iu0, iu1, iv0, iv1;
    float wxu, wxv;
};

struct W4Env {  // environment of a row: what stage 2 reuses from stage 1
    unsigned fb;    // raw fuel bytes (mode 4: the four bytes of the lane)
    int c[4];       // decoded classes
    float2 zx[2], zy[2], m[2], un[2], vn[2];
    float2 R0[2], cc[2], dd[2];  // per-node coefficients (NC only)
};

template <bool NC>
struct WarpStrip4 {
    using V = float2;
    const StepArgs &a;
    const float *lut;   // [ncls][8] S0 R0 b c d e Tf Hs
    const float *lut2;  // [ncls][12] S0 S0 R0 R0 b b c c d d e e
    const float *lutq;  // [ncls] Hq
    float *hw;          // [2][128] heat column sums of this warp
    const WRow<float> *rows;  // rows y0 - 2 .. y0 + La + 1 of the CTA's strips
    const W4Col *cols;        // the warp's 128 columns
    int bcnt;
    unsigned hist;  // bit b: some node of row k-b had psi^{n+1} <= 0 (warp vote)
    int lane, x0, y0, La, Wa, nx, ny, nxa, nya, srx, sry, ncm1, band;
    int xa;         // global column of the lane's first column
    int mode;       // 4: float4 rows, 2: float2 pairs, 1: scalars
    int xc[4];      // clamped load columns (mode 1) / xc[0]: clamped vector column
    bool in[4], out[4];
    bool pst;       // the four columns are output columns, stored as a float4
    bool slow;      // some lane of the warp stores single columns (warp-uniform)
    bool xedge;     // the warp touches the left or right domain boundary
    bool bedge;     // the strip touches the boundary band in x
    V idx2, idy2, i2dx2, i2dy2, eps2, ndt2, ndth2;
    double tstart, t1, hscale;
    int st;
    V poison;
    int ju_cur, jv_cur;
    V UA[2], dU[2], VA[2], dV[2];
    V acc_s[2], acc_q[2];

    __device__ __forceinline__ WarpStrip4(const StepArgs &args, const float *l, const float *l2,
                                          const float *lq, float *h, const WRow<float> *rw,
                                          const W4Col *cw)
        : a(args), lut(l), lut2(l2), lutq(lq), hw(h), rows(rw), cols(cw) {}

    // the lane's four values of row r of field f (columns outside the
    // domain from clamped ones: never used)
    __device__ __forceinline__ void ld(const float *__restrict__ f, int r, V &p0, V &p1) const {
        const int rowb = r * nx;
        if (mode == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(f + (rowb + xc[0]));
            p0 = make_float2(q.x, q.y);
            p1 = make_float2(q.z, q.w);
        } else if (mode == 2) {
            p0 = *reinterpret_cast<const float2 *>(f + (rowb + xc[0]));
            p1 = *reinterpret_cast<const float2 *>(f + (rowb + xc[1]));
        } else {
            p0 = make_float2(f[rowb + xc[0]], f[rowb + xc[1]]);
            p1 = make_float2(f[rowb + xc[2]], f[rowb + xc[3]]);
        }
    }

    __device__ __forceinline__ void load_env(int r, W4Env &e) const {
        const int rowb = r * nx;
        if (mode == 4) {
            e.fb = *reinterpret_cast<const unsigned *>(a.fuel + (rowb + xc[0]));
        } else if (mode == 2) {
            e.fb = (unsigned)*reinterpret_cast<const uint16_t *>(a.fuel + (rowb + xc[0])) |
                   ((unsigned)*reinterpret_cast<const uint16_t *>(a.fuel + (rowb + xc[1])) << 16);
        } else {
            e.fb = (unsigned)a.fuel[rowb + xc[0]] | ((unsigned)a.fuel[rowb + xc[1]] << 8) |
                   ((unsigned)a.fuel[rowb + xc[2]] << 16) | ((unsigned)a.fuel[rowb + xc[3]] << 24);
        }
        ld(static_cast<const float *>(a.dzdx), r, e.zx[0], e.zx[1]);
        ld(static_cast<const float *>(a.dzdy), r, e.zy[0], e.zy[1]);
        if (a.mult) {
            ld(static_cast<const float *>(a.mult), r, e.m[0], e.m[1]);
        } else {
            e.m[0] = e.m[1] = make_float2(1.0f, 1.0f);
        }
        if constexpr (NC) {
            ld(static_cast<const float *>(a.nco[0]), r, e.R0[0], e.R0[1]);
            ld(static_cast<const float *>(a.nco[1]), r, e.cc[0], e.cc[1]);
            ld(static_cast<const float *>(a.nco[2]), r, e.dd[0], e.dd[1]);
        }
    }

    __device__ __forceinline__ void decode(W4Env &e) const {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = (int)((e.fb >> (8 * q)) & 0xffu);
            e.c[q] = c > ncm1 ? ncm1 : c;
        }
    }

    __device__ __forceinline__ void coef(const W4Env &e, int pr, WCoef<float> &co) const {
        coef_pair_dup<float>(lut2, e.c[2 * pr], e.c[2 * pr + 1], co);
        if constexpr (NC) {
            co.R0 = e.R0[pr];
            co.c = e.cc[pr];
            co.d = e.dd[pr];
        }
    }

    // x-interpolated wind of atmos row J at the lane's columns
    __device__ __forceinline__ void wind_u_row(int J, V &w0, V &w1) const {
        const float *u = static_cast<const float *>(a.u) + (size_t)J * (nxa + 1);
        float r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const W4Col &c = cols[4 * lane + q];
            r[q] = (1.0f - c.wxu) * __ldg(u + c.iu0) + c.wxu * __ldg(u + c.iu1);
        }
        w0 = make_float2(r[0], r[1]);
        w1 = make_float2(r[2], r[3]);
    }
    __device__ __forceinline__ void wind_v_row(int J, V &w0, V &w1) const {
        const float *v = static_cast<const float *>(a.v) + (size_t)J * nxa;
        float r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const W4Col &c = cols[4 * lane + q];
            r[q] = (1.0f - c.wxv) * __ldg(v + c.iv0) + c.wxv * __ldg(v + c.iv1);
        }
        w0 = make_float2(r[0], r[1]);
        w1 = make_float2(r[2], r[3]);
    }

    // bilinear wind at fire row r (Sect. 5); a non-finite wind value sets
    // the poison when its atmospheric row is loaded
    __device__ __forceinline__ void wind(int r, W4Env &e) {
        const WRow<float> w = rows[r - (y0 - 2)];
        const int ju0 = w.ju0, jv0 = w.jv0, ju1 = nya == 1 ? ju0 : ju0 + 1, jv1 = jv0 + 1;
        if (ju0 != ju_cur) {
            V B0, B1;
            wind_u_row(ju0, UA[0], UA[1]);
            if (ju1 == ju0) {
                B0 = UA[0];
                B1 = UA[1];
            } else {
                wind_u_row(ju1, B0, B1);
            }
            const V z = splat<V>(0.0f);
            poison = fma2(B0, z, fma2(UA[0], z, poison));
            poison = fma2(B1, z, fma2(UA[1], z, poison));
            dU[0] = sub2(B0, UA[0]);
            dU[1] = sub2(B1, UA[1]);
            ju_cur = ju0;
        }
        if (jv0 != jv_cur) {
            V B0, B1;
            wind_v_row(jv0, VA[0], VA[1]);
            wind_v_row(jv1, B0, B1);
            const V z = splat<V>(0.0f);
            poison = fma2(B0, z, fma2(VA[0], z, poison));
            poison = fma2(B1, z, fma2(VA[1], z, poison));
            dV[0] = sub2(B0, VA[0]);
            dV[1] = sub2(B1, VA[1]);
            jv_cur = jv0;
        }
        const V wu = splat<V>(w.wyu), wv = splat<V>(w.wyv);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            e.un[p] = fma2(wu, dU[p], UA[p]);
            e.vn[p] = fma2(wv, dV[p], VA[p]);
        }
    }

    // the 5-point values of the lane's four columns at row r from the rows
    // below (d), at (c) and above (u), with the ghosts of Sect. 3.1 at the
    // domain boundary; L/R/D/U per pair
    __device__ __forceinline__ void stencil(const V *d, const V *c, const V *u, int r, V *L, V *R,
                                            V *D, V *U) const {
        const float lft = __shfl_up_sync(0xffffffffu, c[1].y, 1);
        const float rgt = __shfl_down_sync(0xffffffffu, c[0].x, 1);
        L[0] = make_float2(lft, c[0].x);
        R[0] = make_float2(c[0].y, c[1].x);
        L[1] = make_float2(c[0].y, c[1].x);
        R[1] = make_float2(c[1].y, rgt);
        D[0] = d[0];
        D[1] = d[1];
        U[0] = u[0];
        U[1] = u[1];
        if (xedge) {
            float v[4] = {c[0].x, c[0].y, c[1].x, c[1].y};
            float l[4] = {L[0].x, L[0].y, L[1].x, L[1].y};
            float rr[4] = {R[0].x, R[0].y, R[1].x, R[1].y};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (xa + q == 0) l[q] = ghost_value<float>(v[q], rr[q]);
                if (xa + q == nx - 1) rr[q] = ghost_value<float>(v[q], l[q]);
            }
            L[0] = make_float2(l[0], l[1]);
            L[1] = make_float2(l[2], l[3]);
            R[0] = make_float2(rr[0], rr[1]);
            R[1] = make_float2(rr[2], rr[3]);
        }
        if (r == 0) {
#pragma unroll
            for (int p = 0; p < 2; ++p)
                D[p] = make_float2(ghost_value<float>(c[p].x, u[p].x),
                                   ghost_value<float>(c[p].y, u[p].y));
        }
        if (r == ny - 1) {
#pragma unroll
            for (int p = 0; p < 2; ++p)
                U[p] = make_float2(ghost_value<float>(c[p].x, d[p].x),
                                   ghost_value<float>(c[p].y, d[p].y));
        }
    }

    __device__ __forceinline__ void run(int x0_, int y0_, double tstart_) {
        lane = threadIdx.x & 31;
        srx = a.srx;
        sry = a.sry;
        nx = a.nx;
        ny = a.ny;
        nxa = a.nxa;
        nya = a.nya;
        x0 = x0_;
        y0 = y0_;
        const int W = a.kx * srx;
        La = min(a.ky * sry, ny - y0);
        Wa = min(W, nx - x0);
        xa = x0 - 4 + 4 * lane;
        mode = ((nx & 3) == 0 && (x0 & 3) == 0 && nx >= 4) ? 4 : ((nx & 1) == 0 ? 2 : 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            in[q] = xa + q >= 0 && xa + q < nx;
            out[q] = xa + q >= x0 && xa + q < x0 + Wa;
        }
        if (mode == 4) {
            xc[0] = min(max(xa, 0), nx - 4);
        } else if (mode == 2) {
            xc[0] = min(max(xa, 0), nx - 2);
            xc[1] = min(max(xa + 2, 0), nx - 2);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) xc[q] = min(max(xa + q, 0), nx - 1);
        }
        pst = mode == 4 && out[0] && out[1] && out[2] && out[3];
        slow = __any_sync(0xffffffffu, !pst && (out[0] || out[1] || out[2] || out[3]));
        xedge = x0 - 4 <= 0 || x0 + 124 >= nx - 1;
        band = a.band;
        bedge = x0 < band || x0 + Wa > nx - band;
        ncm1 = a.ncls - 1;
        idx2 = splat<V>(1.0f / float(a.dx));
        idy2 = splat<V>(1.0f / float(a.dy));
        i2dx2 = splat<V>(1.0f / (2.0f * float(a.dx)));
        i2dy2 = splat<V>(1.0f / (2.0f * float(a.dy)));
        eps2 = splat<V>(float(a.eps));
        ndt2 = splat<V>(-float(a.dt));
        ndth2 = splat<V>(-(0.5f * float(a.dt)));
        tstart = tstart_;
        t1 = tstart + a.dt;
        hscale = 1.0 / (a.dt * (double)srx * (double)sry);
        st = 0;
        poison = splat<V>(0.0f);
        acc_s[0] = acc_s[1] = acc_q[0] = acc_q[1] = splat<V>(0.0f);
        bcnt = 0;
        hist = 0;
        ju_cur = jv_cur = -1;

        const int kb = y0 - 3, ke = y0 + La;
        const V Z = splat<V>(0.0f);
        // rows in registers (names by offset from the iteration's row k)
        V P0[2] = {Z, Z}, P1[2] = {Z, Z}, P2[2] = {Z, Z}, Pp[2] = {Z, Z};
        V Qm[2] = {Z, Z}, Q0[2] = {Z, Z}, Q1[2] = {Z, Z};
        V FA0[2] = {Z, Z}, FA1[2] = {Z, Z};
        V Nm2[2] = {Z, Z}, Nm1[2] = {Z, Z}, N0[2] = {Z, Z};
        V Dm2[2] = {Z, Z}, Dm1[2] = {Z, Z}, D0[2] = {Z, Z};
        V Fp[2] = {splat<V>(1.0f), splat<V>(1.0f)};
        W4Env eB, eC, eP;
        eB.fb = 0;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            eB.zx[p] = eB.zy[p] = eB.un[p] = eB.vn[p] = Z;
            eB.R0[p] = eB.cc[p] = eB.dd[p] = Z;
            eB.m[p] = splat<V>(1.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) eB.c[q] = 0;
        eC = eB;
        eP = eB;
        const float *psi_in = static_cast<const float *>(a.psi_in);
        const float *F_in = static_cast<const float *>(a.F_in);
        // unconditional loads from clamped rows (values outside the domain
        // are never used), so that a prefetched register is not merged with
        // its older value
        ld(psi_in, min(max(kb, 0), ny - 1), P0[0], P0[1]);
        ld(psi_in, min(max(kb + 1, 0), ny - 1), P1[0], P1[1]);
        ld(psi_in, min(max(kb + 2, 0), ny - 1), Pp[0], Pp[1]);
        load_env(min(max(kb + 1, 0), ny - 1), eP);

#pragma unroll 1
        for (int k = kb; k <= ke; ++k) {
            // ---- A: F^n of row k (used one iteration later), psi^n row k+3
            const V Fc0 = Fp[0], Fc1 = Fp[1];
            ld(F_in, min(max(k, 0), ny - 1), Fp[0], Fp[1]);
            P2[0] = Pp[0];
            P2[1] = Pp[1];
            ld(psi_in, min(max(k + 3, 0), ny - 1), Pp[0], Pp[1]);
            // ---- B: stage 1 on row k+1 (both stages in one basic block:
            // rows outside the domain are computed from clamped loads and
            // never read)
            const int rB = k + 1;
            eB = eP;
            decode(eB);
            load_env(min(max(rB + 1, 0), ny - 1), eP);
            wind(rB, eB);
            {
                V L[2], R[2], D[2], U[2];
                stencil(P0, P1, P2, rB, L, R, D, U);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    WCoef<float> co;
                    coef(eB, p, co);
                    FA1[p] = neg_rhs2<float>(P1[p], L[p], R[p], D[p], U[p], idx2, idy2, i2dx2,
                                             i2dy2, eps2, co, eB.m[p], eB.un[p], eB.vn[p],
                                             eB.zx[p], eB.zy[p]);
                    Q1[p] = fma2(ndt2, FA1[p], P1[p]);
                }
            }
            // ---- C: stage 2, crossing and t - t_i on row k
            const int rC = k;
            {
                V L[2], R[2], D[2], U[2];
                stencil(Qm, Q0, Q1, rC, L, R, D, U);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    WCoef<float> co;
                    coef(eC, p, co);
                    const V G2 = neg_rhs2<float>(Q0[p], L[p], R[p], D[p], U[p], idx2, idy2,
                                                 i2dx2, i2dy2, eps2, co, eC.m[p], eC.un[p],
                                                 eC.vn[p], eC.zx[p], eC.zy[p]);
                    N0[p] = fma2(ndth2, add2(FA0[p], G2), P0[p]);
                }
            }
            if (rC >= y0 - 1 && rC >= 0 && rC < ny) {
                poison = fma2(N0[0], Z, poison);
                poison = fma2(N0[1], Z, poison);
                const float nv[4] = {N0[0].x, N0[0].y, N0[1].x, N0[1].y};
                const float pv[4] = {P0[0].x, P0[0].y, P0[1].x, P0[1].y};
                const bool own_row = rC >= y0 && rC < y0 + La;
                if (own_row && (bedge || rC < band || rC >= ny - band)) {
                    const bool rb = rC < band || rC >= ny - band;
                    bool hit = false;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool e = rb || xa + q < band || xa + q >= nx - band;
                        hit = hit || (out[q] && e && nv[q] < 0.0f);
                    }
                    if (hit) st |= ST_BOUNDARY;
                }
                // ignition time and t - t_i where a node is burning (lanes 0
                // and 31 hold no column anybody reads at their outer end)
                bool nb[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) nb[q] = in[q] && nv[q] <= 0.0f;
                nb[0] = nb[0] && lane > 0;
                nb[3] = nb[3] && lane < 31;
                D0[0] = D0[1] = Z;
                const bool burn = __any_sync(0xffffffffu, nb[0] || nb[1] || nb[2] || nb[3]);
                hist |= burn ? 1u : 0u;
                if (burn) {
                    const int g = rC * nx + xa;
                    float dv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!nb[q]) continue;
                        double ti = a.tign[g + q];
                        if (pv[q] > 0.0f && isinf(ti)) {
                            const double q0 = (double)pv[q], q1 = (double)nv[q];
                            ti = tstart + q0 * a.dt / (q0 - q1);
                            if (own_row && out[q]) a.tign[g + q] = ti;
                        }
                        if (nv[q] < 0.0f) dv[q] = (float)(t1 - ti);
                    }
                    D0[0] = make_float2(dv[0], dv[1]);
                    D0[1] = make_float2(dv[2], dv[3]);
                }
                if (own_row) {
                    float *po = static_cast<float *>(a.psi_out);
                    const int g = rC * nx + xa;
                    if (pst)
                        *reinterpret_cast<float4 *>(po + g) =
                            make_float4(N0[0].x, N0[0].y, N0[1].x, N0[1].y);
                    if (slow && !pst) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (out[q]) po[g + q] = nv[q];
                    }
                }
            }
            // ---- D: fuel fraction and heat on row k-1
            const int rD = k - 1;
            if (rD >= y0 && rD < y0 + La) {
                V F1[2] = {splat<V>(1.0f), splat<V>(1.0f)};
                if ((hist & 7u) != 0u) gate(rD, Nm2, Nm1, N0, Dm2, Dm1, D0, F1);
                finish_row(rD, Fc0, Fc1, F1);
            }
            // ---- rotate
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                P0[p] = P1[p];
                P1[p] = P2[p];
                Qm[p] = Q0[p];
                Q0[p] = Q1[p];
                FA0[p] = FA1[p];
                Nm2[p] = Nm1[p];
                Nm1[p] = N0[p];
                Dm2[p] = Dm1[p];
                Dm1[p] = D0[p];
            }
            eC = eB;
            hist <<= 1;
        }
        if (!finite_val(poison.x) || !finite_val(poison.y)) st |= ST_NONFINITE;
    }

    // the quadrature of the row's output columns where psi^{n+1} <= 0 in
    // their 3x3 neighbourhood (in-domain values only; ghosts are never
    // below them)
    __device__ __forceinline__ void gate(int rD, const V *Na, const V *Nb, const V *Nc,
                                         const V *Da, const V *Db, const V *Dc, V *F1) {
        const float big = 1e30f;
        const float a4[4] = {Na[0].x, Na[0].y, Na[1].x, Na[1].y};
        const float b4[4] = {Nb[0].x, Nb[0].y, Nb[1].x, Nb[1].y};
        const float c4[4] = {Nc[0].x, Nc[0].y, Nc[1].x, Nc[1].y};
        float cm[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v = min_val(min_val(a4[q], b4[q]), c4[q]);
            if (rD == 0) v = min_val(b4[q], c4[q]);
            else if (rD == ny - 1) v = min_val(a4[q], b4[q]);
            cm[q] = in[q] ? v : big;
        }
        const float cl = __shfl_up_sync(0xffffffffu, cm[3], 1);
        const float cr = __shfl_down_sync(0xffffffffu, cm[0], 1);
        bool bq[4];
        bq[0] = out[0] && min_val(min_val(cl, cm[0]), cm[1]) < 0.0f;
        bq[1] = out[1] && min_val(min_val(cm[0], cm[1]), cm[2]) < 0.0f;
        bq[2] = out[2] && min_val(min_val(cm[1], cm[2]), cm[3]) < 0.0f;
        bq[3] = out[3] && min_val(min_val(cm[2], cm[3]), cr) < 0.0f;
        if (!__any_sync(0xffffffffu, bq[0] || bq[1] || bq[2] || bq[3])) return;
        // full quadrature: six values per row (the lane's four and one
        // neighbour on each side) of psi^{n+1} and t - t_i
        float q6[3][6], e6[3][6];
        const V *Nr[3] = {Na, Nb, Nc}, *Dr[3] = {Da, Db, Dc};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            q6[b][0] = __shfl_up_sync(0xffffffffu, Nr[b][1].y, 1);
            q6[b][1] = Nr[b][0].x;
            q6[b][2] = Nr[b][0].y;
            q6[b][3] = Nr[b][1].x;
            q6[b][4] = Nr[b][1].y;
            q6[b][5] = __shfl_down_sync(0xffffffffu, Nr[b][0].x, 1);
            e6[b][0] = __shfl_up_sync(0xffffffffu, Dr[b][1].y, 1);
            e6[b][1] = Dr[b][0].x;
            e6[b][2] = Dr[b][0].y;
            e6[b][3] = Dr[b][1].x;
            e6[b][4] = Dr[b][1].y;
            e6[b][5] = __shfl_down_sync(0xffffffffu, Dr[b][0].x, 1);
        }
        float fr[4] = {F1[0].x, F1[0].y, F1[1].x, F1[1].y};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!bq[j]) continue;
            float q[3][3], e[3][3];
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    q[b][h] = q6[b][j + h];
                    e[b][h] = e6[b][j + h];
                }
            const int x = xa + j;
            if (x == 0 || x == nx - 1 || rD == 0 || rD == ny - 1) {
                // ghost ring of psi^{n+1} (x first, then y) and of t - t_i
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int yy = rD + b - 1;
                    if (yy < 0 || yy >= ny) continue;
                    if (x == 0) {
                        q[b][0] = ghost_value<float>(q[b][1], q[b][2]);
                        e[b][0] = q[b][0] >= 0.0f ? 0.0f : e[b][1];
                    }
                    if (x == nx - 1) {
                        q[b][2] = ghost_value<float>(q[b][1], q[b][0]);
                        e[b][2] = q[b][2] >= 0.0f ? 0.0f : e[b][1];
                    }
                }
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    if (rD == 0) {
                        q[0][h] = ghost_value<float>(q[1][h], q[2][h]);
                        e[0][h] = q[0][h] >= 0.0f ? 0.0f : e[1][h];
                    }
                    if (rD == ny - 1) {
                        q[2][h] = ghost_value<float>(q[1][h], q[0][h]);
                        e[2][h] = q[2][h] >= 0.0f ? 0.0f : e[1][h];
                    }
                }
            }
            const int cls0 = a.fuel[rD * nx + x];
            const int cls = cls0 > ncm1 ? ncm1 : cls0;
            fr[j] = cell_fraction_vals<float>(q[0][0], q[0][1], q[0][2], q[1][0], q[1][1], q[1][2],
                                              q[2][0], q[2][1], q[2][2], e[0][0], e[0][1], e[0][2],
                                              e[1][0], e[1][1], e[1][2], e[2][0], e[2][1], e[2][2],
                                              lut[cls * 8 + 6]);
        }
        F1[0] = make_float2(fr[0], fr[1]);
        F1[1] = make_float2(fr[2], fr[3]);
    }

    // store F^{n+1} of the row, heat flux densities summed per column over
    // the band, and the per-cell average after the band's last row
    __device__ __forceinline__ void finish_row(int rD, V Fn0, V Fn1, const V *F1) {
        const int g = rD * nx + xa;
        float *fo = static_cast<float *>(a.F_out);
        if (pst) *reinterpret_cast<float4 *>(fo + g) = make_float4(F1[0].x, F1[0].y, F1[1].x, F1[1].y);
        if (slow && !pst) {
            const float fv[4] = {F1[0].x, F1[0].y, F1[1].x, F1[1].y};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (out[q]) fo[g + q] = fv[q];
        }
        const V dF0 = sub2(Fn0, F1[0]), dF1 = sub2(Fn1, F1[1]);
        if (__any_sync(0xffffffffu, dF0.x != 0.0f || dF0.y != 0.0f || dF1.x != 0.0f ||
                                        dF1.y != 0.0f)) {
            const float dv[4] = {out[0] ? dF0.x : 0.0f, out[1] ? dF0.y : 0.0f,
                                 out[2] ? dF1.x : 0.0f, out[3] ? dF1.y : 0.0f};
            // heat factors of the columns that burned (0 elsewhere: the
            // fused multiply-add then adds an exact 0)
            float hs[4] = {0.0f, 0.0f, 0.0f, 0.0f}, hq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (dv[q] == 0.0f) continue;
                if constexpr (NC) {
                    hs[q] = static_cast<const float *>(a.nco[3])[g + q];
                    hq[q] = static_cast<const float *>(a.nco[4])[g + q];
                } else {
                    int cls = a.fuel[g + q];
                    cls = cls > ncm1 ? ncm1 : cls;
                    hs[q] = lut[cls * 8 + 7];
                    hq[q] = lutq[cls];
                }
            }
            const V d0 = make_float2(dv[0], dv[1]), d1 = make_float2(dv[2], dv[3]);
            acc_s[0] = fma2(d0, make_float2(hs[0], hs[1]), acc_s[0]);
            acc_s[1] = fma2(d1, make_float2(hs[2], hs[3]), acc_s[1]);
            acc_q[0] = fma2(d0, make_float2(hq[0], hq[1]), acc_q[0]);
            acc_q[1] = fma2(d1, make_float2(hq[2], hq[3]), acc_q[1]);
        }
        // after the last row of an atmospheric band: average per cell
        if (++bcnt == sry) {
            bcnt = 0;
            *reinterpret_cast<float4 *>(hw + 4 * lane) =
                make_float4(acc_s[0].x, acc_s[0].y, acc_s[1].x, acc_s[1].y);
            *reinterpret_cast<float4 *>(hw + kWarp4Cols + 4 * lane) =
                make_float4(acc_q[0].x, acc_q[0].y, acc_q[1].x, acc_q[1].y);
            __syncwarp();
            const int cells = Wa / srx;
            if (lane < cells) {
                float h0 = 0.0f, h1 = 0.0f;
                for (int e = 0; e < srx; ++e) {
                    const int lc = 4 + lane * srx + e;
                    h0 += hw[lc];
                    h1 += hw[kWarp4Cols + lc];
                }
                const size_t ga = (size_t)(rD / sry) * nxa + (x0 / srx + lane);
                if (a.heat_s) a.heat_s[ga] = (double)h0 * hscale;
                if (a.heat_l) a.heat_l[ga] = (double)h1 * hscale;
            }
            __syncwarp();
            acc_s[0] = acc_s[1] = acc_q[0] = acc_q[1] = splat<V>(0.0f);
        }
    }
};

template <bool NC>
__global__ void __launch_bounds__(kWarp4CtaThreads, 2) k_fire_warp4(const StepArgs a) {
    __shared__ __align__(16) float lut[FIRE_MAX_CLASSES * 8];
    __shared__ __align__(16) float lut2[FIRE_MAX_CLASSES * 12];
    __shared__ float lutq[FIRE_MAX_CLASSES];
    __shared__ __align__(16) float hw[kWarpStrips][2 * kWarp4Cols];
    __shared__ __align__(16) WRow<float> rows[kWarpMaxRows + 4];
    __shared__ W4Col cols[kWarpStrips][kWarp4Cols];
    const int y0 = blockIdx.y * a.ky * a.sry;
    const int La = min(a.ky * a.sry, a.ny - y0);
    for (int i = threadIdx.x; i < La + 4; i += kWarp4CtaThreads) {
        const int r = y0 - 2 + i;
        WRow<float> w;
        w.ju0 = w.jv0 = 0;
        w.wyu = w.wyv = 0.0f;
        if (r >= 0 && r < a.ny) {
            int j1;
            const float yr = (float(r) + 0.5f) / float(a.sry);
            lin_idx<float>(yr - 0.5f, a.nya, w.ju0, j1, w.wyu);
            lin_idx<float>(yr, a.nya + 1, w.jv0, j1, w.wyv);
        }
        rows[i] = w;
    }
    for (int k = threadIdx.x; k < a.ncls; k += kWarp4CtaThreads) {
        const double *co = a.coef + (size_t)k * K_N;
        float *l = lut + k * 8;
        l[0] = float(co[K_S0]);
        l[1] = float(co[K_R0]);
        l[2] = float(co[K_B]);
        l[3] = float(co[K_C]);
        l[4] = float(co[K_D]);
        l[5] = float(co[K_E]);
        l[6] = float(co[K_TF]);
        l[7] = float(co[K_HS]);
        lutq[k] = float(co[K_HQ]);
        float *l2 = lut2 + k * 12;
        for (int j = 0; j < 6; ++j) l2[2 * j] = l2[2 * j + 1] = l[j];
    }
    const int w = threadIdx.x >> 5;
    const int W = a.kx * a.srx;
    const int x0 = (blockIdx.x * kWarpStrips + w) * W;
    {
        // x-weights of the wind for the warp's columns x0 - 4 .. x0 + 123
        const int lane = threadIdx.x & 31;
        for (int q = lane; q < kWarp4Cols; q += 32) {
            const int x = min(max(x0 - 4 + q, 0), a.nx - 1);
            const float xr = (float(x) + 0.5f) / float(a.srx);
            W4Col c;
            lin_idx<float>(xr, a.nxa + 1, c.iu0, c.iu1, c.wxu);
            lin_idx<float>(xr - 0.5f, a.nxa, c.iv0, c.iv1, c.wxv);
            cols[w][q] = c;
        }
    }
    __syncthreads();
    const double tstart = *a.t_in;
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) *a.t_out = tstart + a.dt;
    if (x0 >= a.nx) return;  // whole warp
    WarpStrip4<NC> s(a, lut, lut2, lutq, hw[w], rows, cols[w]);
    s.run(x0, y0, tstart);
    const int stw = __reduce_or_sync(0xffffffffu, s.st);
    if ((threadIdx.x & 31) == 0 && stw) atomicOr(a.status, stw);
}

cudaError_t launch_warp4(const StepArgs &a, cudaStream_t s) {
    const int W = a.kx * a.srx, L = a.ky * a.sry;
    if (W > kWarp4MaxColumns || W < 1 || L > kWarpMaxRows || L < 1 ||
        (long long)a.nx * a.ny > kWarpMaxNodes)
        return cudaErrorInvalidValue;
    const int strips = (a.nx + W - 1) / W;
    dim3 grid((strips + kWarpStrips - 1) / kWarpStrips, (a.ny + L - 1) / L);
    if (a.nco[0])
        k_fire_warp4<true><<<grid, kWarp4CtaThreads, 0, s>>>(a);
    else
        k_fire_warp4<false><<<grid, kWarp4CtaThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace wf
