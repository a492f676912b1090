// Warp-marching fire-step kernel: the whole step of Sect. 5 (items 2-6) in
// one pass over the state, each warp marching down its own strip with the
// rows it needs in registers.
//
// A warp owns W <= 60 output columns (W = kx*srx, even) and L = ky*sry
// output rows; lane l holds the two columns x0 - 2 + 2l and x0 - 1 + 2l, so
// the warp computes 64 columns: the strip, two halo columns on the left and
// up to two on the right (the outermost of them are garbage nobody reads).
// Horizontal neighbours come from the adjacent lane by shuffle, vertical
// ones from the rows the lane keeps in registers; no row of the state goes
// through shared memory (it holds the class tables, the wind-row weights
// and a heat buffer) and warps never wait for one another.  Mesh offsets
// are 32-bit (meshes below 2^31 nodes).  Per row (iteration k) the stages
// lag behind the loads:
//   B  stage 1 (eq. Heun, first line) on row k+1
//   C  stage 2 (eq. Heun, second line), ignition-time crossing
//      (eq. set-ignition-time) and t - t_i on row k
//   D  fuel-fraction quadrature (Sect. 3.3) and heat flux
//      (eqs. sensible-/latent-heat-flux) on row k-1
// The two columns of a lane are one float2 and the FP32 arithmetic of the
// right-hand side uses the packed f32x2 instructions.  The quadrature, the
// ignition-time arithmetic (double) and the domain-boundary ghosts
// (Sect. 3.1) run only in warps that need them (warp votes / uniform
// branches).  Heat is summed per column over each band of sry rows, then per
// atmospheric cell (Sect. 5, item 6) through a small per-warp buffer.
#pragma once

#include <mutex>

#include "fire_device.cuh"
#include "fire_internal.h"
#include "pair_math.cuh"

namespace wf {

constexpr int kWarpCtaThreads = 32 * kWarpStrips;

template <typename T>
struct WRow {  // y-interpolation of the wind for one fire row
    int ju0, jv0;
    T wyu, wyv;
};

template <typename T>
struct WOcc {
    static constexpr int blocks = 3;
};
template <>
struct WOcc<double> {
    static constexpr int blocks = 1;
};
static_assert(WOcc<float>::blocks == kWarpCtasPerSmF32, "default launch shapes assume this");

template <typename T>
struct WEnv {  // what stage 2 reuses from stage 1 of the same row
    using V = typename PairT<T>::t;
    int cls0, cls1;  // raw fuel bytes when loaded (see decode), classes after
    V zx, zy, m, un, vn;
    V R0, c, d;      // per-node coefficients (NC only)
};

// NC: per-node R0, c, d and heat factors (a per-node fuel moisture) read
// from the planes of StepArgs::nco instead of the class table.
// Dense (FP32, the FIRE_KERNEL_WARP_DENSE variant): t_i read one row ahead
// where psi^n <= 0 and the quadrature of the lane's two cells in one packed
// evaluation away from the domain boundary; the same results as the other
// instantiation bit for bit, faster where much of the mesh burns and slower
// where little does.
template <typename T, bool NC = false, bool Dense = false>
struct WarpStrip {
    using V = typename PairT<T>::t;
    const StepArgs &a;
    const T *lut;   // [ncls][8] S0 R0 b c d e Tf Hs
    const T *lut2;  // [ncls][12] S0 S0 R0 R0 b b c c d d e e
    const T *lutq;  // [ncls] Hq
    T *hw;          // [2][64] heat column sums of this warp
    const WRow<T> *rows;  // rows y0 - 2 .. y0 + La + 1 of the CTA's strips
    int bcnt;       // rows done in the current atmospheric band
    unsigned hist;  // bit b: some node of row k-b had psi^{n+1} <= 0 (warp vote)
    int lane, x0, y0, W, La, Wa, nx, ny, nxa, nya, srx, sry, ncm1, band;
    int xa;          // global column of the lane's first column
    bool vec;        // paired vector access (nx even)
    bool inA, inB;   // columns inside the domain
    bool outA, outB; // output columns of this warp
    bool pst;        // both columns are output columns and stored as a pair
    bool slow;       // some lane of the warp stores single columns (warp-uniform)
    int xcv, xcA, xcB;  // clamped columns of the paired / single loads
    bool xedge;      // the strip touches the left or right domain boundary
    bool bedge;      // the strip touches the boundary band in x
    V idx2, idy2, i2dx2, i2dy2, eps2, ndt2, ndth2;
    double tstart, t1, hscale;
    mutable int st;  // status bits (also set by the const loaders' index checks)
    V poison;
    // wind: x-interpolation per column, two atmos rows held per component
    int iu0[2], iu1[2], iv0[2], iv1[2];
    T wxu[2], wxv[2];
    int ju_cur, jv_cur;
    V UA, dU, VA, dV;  // wind of atmos rows j0 and the difference to row j0 + 1
    V acc_s, acc_q;

    __device__ __forceinline__ WarpStrip(const StepArgs &args, const T *l, const T *l2,
                                         const T *lq, T *h, const WRow<T> *rw)
        : a(args), lut(l), lut2(l2), lutq(lq), hw(h), rows(rw) {}

    // paired load of row r at the lane's columns.  Every lane loads, columns
    // outside the domain from the nearest inside one (their values are never
    // used), so a loaded register is not touched before its use one
    // iteration later and the prefetch hides the memory latency.
    __device__ __forceinline__ V ld(const T *__restrict__ f, int r) const {
        const int rowb = r * nx;
        if (vec) return *reinterpret_cast<const V *>(f + WF_CHK(rowb + xcv, nx * ny - 1, st));
        return mk2(f[WF_CHK(rowb + xcA, nx * ny, st)], f[WF_CHK(rowb + xcB, nx * ny, st)]);
    }

    // prefetch of a row's environment: raw fuel bytes (decoded by decode()
    // at use), terrain gradient and multiplier
    __device__ __forceinline__ void load_env(int r, WEnv<T> &e) const {
        const int rowb = r * nx;
        if (vec) {
            e.cls0 = *reinterpret_cast<const uint16_t *>(a.fuel + WF_CHK(rowb + xcv, nx * ny - 1, st));
        } else {
            e.cls0 = a.fuel[WF_CHK(rowb + xcA, nx * ny, st)];
            e.cls1 = a.fuel[WF_CHK(rowb + xcB, nx * ny, st)];
        }
        e.zx = ld(static_cast<const T *>(a.dzdx), r);
        e.zy = ld(static_cast<const T *>(a.dzdy), r);
        e.m = a.mult ? ld(static_cast<const T *>(a.mult), r) : splat<V>(T(1));
        if constexpr (NC) {
            e.R0 = ld(static_cast<const T *>(a.nco[0]), r);
            e.c = ld(static_cast<const T *>(a.nco[1]), r);
            e.d = ld(static_cast<const T *>(a.nco[2]), r);
        }
    }

    __device__ __forceinline__ void decode(WEnv<T> &e) const {
        int c0 = vec ? (e.cls0 & 0xff) : e.cls0, c1 = vec ? (e.cls0 >> 8) : e.cls1;
        e.cls0 = c0 > ncm1 ? ncm1 : c0;
        e.cls1 = c1 > ncm1 ? ncm1 : c1;
    }

    __device__ __forceinline__ void coef(const WEnv<T> &e, WCoef<T> &co) const {
        coef_pair_dup<T>(lut2, e.cls0, e.cls1, co);
        if constexpr (NC) {
            co.R0 = e.R0;
            co.c = e.c;
            co.d = e.d;
        }
    }

    // x-interpolated wind of atmos row J at this lane's columns
    __device__ __forceinline__ V wind_u_row(int J) const {
        const T *u = static_cast<const T *>(a.u) + (size_t)J * (nxa + 1);
        const int b = J * (nxa + 1), n = nya * (nxa + 1);  // (index checks only)
        return mk2((T(1) - wxu[0]) * __ldg(u + WF_CHK_AT(b, iu0[0], n, st)) +
                       wxu[0] * __ldg(u + WF_CHK_AT(b, iu1[0], n, st)),
                   (T(1) - wxu[1]) * __ldg(u + WF_CHK_AT(b, iu0[1], n, st)) +
                       wxu[1] * __ldg(u + WF_CHK_AT(b, iu1[1], n, st)));
    }
    __device__ __forceinline__ V wind_v_row(int J) const {
        const T *v = static_cast<const T *>(a.v) + (size_t)J * nxa;
        const int b = J * nxa, n = (nya + 1) * nxa;  // (index checks only)
        return mk2((T(1) - wxv[0]) * __ldg(v + WF_CHK_AT(b, iv0[0], n, st)) +
                       wxv[0] * __ldg(v + WF_CHK_AT(b, iv1[0], n, st)),
                   (T(1) - wxv[1]) * __ldg(v + WF_CHK_AT(b, iv0[1], n, st)) +
                       wxv[1] * __ldg(v + WF_CHK_AT(b, iv1[1], n, st)));
    }

    // bilinear wind at fire row r (Sect. 5), rows of the atmos wind cached;
    // a non-finite wind value sets the poison when its row is loaded
    __device__ __forceinline__ void wind(int r, V &un, V &vn) {
        const WRow<T> w = rows[r - (y0 - 2)];
        const int ju0 = w.ju0, jv0 = w.jv0, ju1 = nya == 1 ? ju0 : ju0 + 1, jv1 = jv0 + 1;
        if (ju0 != ju_cur) {
            UA = wind_u_row(ju0);
            const V UB = ju1 == ju0 ? UA : wind_u_row(ju1);
            poison = fma2(UB, splat<V>(T(0)), fma2(UA, splat<V>(T(0)), poison));
            dU = sub2(UB, UA);
            ju_cur = ju0;
        }
        if (jv0 != jv_cur) {
            VA = wind_v_row(jv0);
            const V VB = wind_v_row(jv1);
            poison = fma2(VB, splat<V>(T(0)), fma2(VA, splat<V>(T(0)), poison));
            dV = sub2(VB, VA);
            jv_cur = jv0;
        }
        un = mk2(fma(w.wyu, dU.x, UA.x), fma(w.wyu, dU.y, UA.y));
        vn = mk2(fma(w.wyv, dV.x, VA.x), fma(w.wyv, dV.y, VA.y));
    }

    // horizontal neighbours of a row of pairs: left of .x, right of .y
    __device__ __forceinline__ void sides(V v, T &l, T &r) const {
        l = __shfl_up_sync(0xffffffffu, v.y, 1);
        r = __shfl_down_sync(0xffffffffu, v.x, 1);
    }

    // 5-point values of the lane's two columns at row r from the rows below
    // (d), at (c) and above (u), with the ghosts of Sect. 3.1 at the domain
    // boundary; h replaces the left neighbour of lane 0 and the right one of
    // lane 31 (each lane's own halo column)
    __device__ __forceinline__ void stencil(V d, V c, V u, int r, bool use_halo, T h, V &L, V &R,
                                            V &D, V &Uu) const {
        T l, rr;
        sides(c, l, rr);
        if (use_halo) {
            if (lane == 0) l = h;
            if (lane == 31) rr = h;
        }
        L = mk2(l, c.x);
        R = mk2(c.y, rr);
        D = d;
        Uu = u;
        if (xedge) {
            if (xa == 0) L.x = ghost_value<T>(c.x, c.y);
            if (xa + 1 == nx - 1) R.y = ghost_value<T>(c.y, c.x);
            if (xa == nx - 1) R.x = ghost_value<T>(c.x, L.x);
        }
        if (r == 0) D = mk2(ghost_value<T>(c.x, u.x), ghost_value<T>(c.y, u.y));
        if (r == ny - 1) Uu = mk2(ghost_value<T>(c.x, d.x), ghost_value<T>(c.y, d.y));
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
        W = a.kx * srx;
        La = min(a.ky * sry, ny - y0);
        Wa = min(W, nx - x0);
        xa = x0 - 2 + 2 * lane;
        vec = (nx & 1) == 0;
        inA = xa >= 0 && xa < nx;
        inB = xa + 1 >= 0 && xa + 1 < nx;
        outA = xa >= x0 && xa < x0 + Wa;
        outB = xa + 1 >= x0 && xa + 1 < x0 + Wa;
        pst = vec && outA && outB;
        slow = __any_sync(0xffffffffu, !pst && (outA || outB));
        xcv = min(max(xa, 0), nx - 2);
        xcA = min(max(xa, 0), nx - 1);
        xcB = min(max(xa + 1, 0), nx - 1);
        xedge = x0 - 2 <= 0 || x0 + 62 >= nx - 1;
        band = a.band;
        bedge = x0 < band || x0 + Wa > nx - band;
        ncm1 = a.ncls - 1;
        idx2 = splat<V>(T(1) / T(a.dx));
        idy2 = splat<V>(T(1) / T(a.dy));
        i2dx2 = splat<V>(T(1) / (T(2) * T(a.dx)));
        i2dy2 = splat<V>(T(1) / (T(2) * T(a.dy)));
        eps2 = splat<V>(T(a.eps));
        ndt2 = splat<V>(-T(a.dt));
        ndth2 = splat<V>(-(T(0.5) * T(a.dt)));
        tstart = tstart_;
        t1 = tstart + a.dt;
        hscale = 1.0 / (a.dt * (double)srx * (double)sry);
        st = 0;
        poison = splat<V>(T(0));
        acc_s = acc_q = splat<V>(T(0));
        bcnt = 0;
        hist = 0;
        // x-weights of the wind
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = min(max(xa + j, 0), nx - 1);
            const T xr = (T(x) + T(0.5)) / T(srx);
            lin_idx<T>(xr, nxa + 1, iu0[j], iu1[j], wxu[j]);
            lin_idx<T>(xr - T(0.5), nxa, iv0[j], iv1[j], wxv[j]);
        }
        ju_cur = jv_cur = -1;

        const int kb = y0 - 3, ke = y0 + La;
        // rows in registers (names by offset from the iteration's row k)
        V P0 = splat<V>(T(0)), P1 = P0, P2 = P0, Ppre = P0;  // psi^n rows k, k+1, k+2, prefetch
        T h1 = T(0), h2 = T(0), hp = T(0);  // halo column of lanes 0 / 31, rows k+1, k+2, prefetch
        V Qm = P0, Q0 = P0, Q1 = P0;       // psi* rows k-1, k, k+1
        V FA0 = P0, FA1 = P0;              // -F(psi^n) rows k, k+1
        V Nm2 = P0, Nm1 = P0, N0 = P0;     // psi^{n+1} rows k-2, k-1, k
        V Dm2 = P0, Dm1 = P0, D0 = P0;     // t - t_i rows k-2, k-1, k
        V Fpre = splat<V>(T(1));           // F^n of row k-1 (at the top of iteration k)
        double tiA = 0.0, tiB = 0.0;       // t_i of row k where psi^n <= 0 (prefetched)
        WEnv<T> envB, envC, envPre;
        envB.cls0 = envB.cls1 = 0;
        envB.zx = envB.zy = envB.un = envB.vn = P0;
        envB.R0 = envB.c = envB.d = P0;
        envB.m = splat<V>(T(1));
        envC = envB;
        envPre = envB;
        const T *psi_in = static_cast<const T *>(a.psi_in);
        // unconditional loads (rows outside the domain from the nearest
        // inside row: their values are never used), so that the loaded
        // registers are not merged with older values when they arrive
        // lanes 0 and 31 also load the one column beyond the warp on their
        // side (x0 - 3, x0 + 62, clamped into the domain)
        const bool hlane = lane == 0 || lane == 31;
        const int hcol = lane == 0 ? max(xa - 1, 0) : min(xa + 2, nx - 1);
        auto load_psi = [&](int r, V &v, T &h) {
            r = min(max(r, 0), ny - 1);
            v = ld(psi_in, r);
            if (hlane) h = psi_in[WF_CHK(r * nx + hcol, nx * ny, st)];
        };
        load_psi(kb, P0, h1);  // h1 of row kb is not used
        load_psi(kb + 1, P1, h1);
        load_psi(kb + 2, Ppre, hp);
        load_env(min(max(kb + 1, 0), ny - 1), envPre);

#pragma unroll 1
        for (int k = kb; k <= ke; ++k) {
            // ---- A: psi^n of row k+2 arrives; prefetch row k+3
            // F^n of row k, used by the quadrature of the next iteration:
            // loaded here, a full iteration before the row k-1 value is used
            const V Fcur = Fpre;
            Fpre = ld(static_cast<const T *>(a.F_in), min(max(k, 0), ny - 1));
            P2 = Ppre;
            h2 = hp;
            load_psi(k + 3, Ppre, hp);
            // ---- B: stage 1 on row k+1.  Both stages run on every
            // iteration, also on rows outside the domain or before the
            // strip's first stage-2 row, from the clamped rows loaded there:
            // such values are never read (boundary rows take ghosts, the
            // quadrature starts at the strip's first row), and with no
            // branch around them the two stages share one basic block, so
            // their independent parts can be scheduled together
            const int rB = k + 1;
            envB = envPre;
            decode(envB);
            load_env(min(max(rB + 1, 0), ny - 1), envPre);
            {
                wind(rB, envB.un, envB.vn);
                V L, R, D, U;
                stencil(P0, P1, P2, rB, true, h1, L, R, D, U);
                WCoef<T> co;
                coef(envB, co);
                FA1 = neg_rhs2<T>(P1, L, R, D, U, idx2, idy2, i2dx2, i2dy2, eps2, co, envB.m,
                                  envB.un, envB.vn, envB.zx, envB.zy);
                Q1 = fma2(ndt2, FA1, P1);
            }
            // ---- C: stage 2, crossing and t - t_i on row k
            const int rC = k;
            {
                V L, R, D, U;
                stencil(Qm, Q0, Q1, rC, false, T(0), L, R, D, U);
                WCoef<T> co;
                coef(envC, co);
                const V G2 = neg_rhs2<T>(Q0, L, R, D, U, idx2, idy2, i2dx2, i2dy2, eps2, co,
                                         envC.m, envC.un, envC.vn, envC.zx, envC.zy);
                // P0 + dt (F0/2 + F2/2) = P0 - dt/2 (G0 + G2), the halving exact
                N0 = fma2(ndth2, add2(FA0, G2), P0);
            }
            if (rC >= y0 - 1 && rC >= 0 && rC < ny) {
                // every column of the warp is computed from in-domain values,
                // so a non-finite value anywhere in it comes from a
                // non-finite value of the step
                poison = fma2(N0, splat<V>(T(0)), poison);
                const bool own_row = rC >= y0 && rC < y0 + La;
                if (own_row) {
                    if (bedge || rC < band || rC >= ny - band) {
                        const bool ea = xa < band || xa >= nx - band || rC < band || rC >= ny - band;
                        const bool eb = xa + 1 < band || xa + 1 >= nx - band || rC < band ||
                                        rC >= ny - band;
                        if ((outA && ea && N0.x < T(0)) || (outB && eb && N0.y < T(0)))
                            st |= ST_BOUNDARY;
                    }
                }
                // ignition time and t - t_i, only where a node is burning
                const bool na = inA && lane > 0 && N0.x <= T(0);
                const bool nb = inB && lane < 31 && N0.y <= T(0);
                D0 = splat<V>(T(0));
                const bool burn = __any_sync(0xffffffffu, na || nb);
                hist |= burn ? 1u : 0u;
                if (burn) {
                    const int g = rC * nx + xa;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (!(j == 0 ? na : nb)) continue;
                        const T p0 = j == 0 ? P0.x : P0.y, pn = j == 0 ? N0.x : N0.y;
                        // Dense: prefetched where psi^n <= 0, read here at a crossing
                        double ti;
                        if constexpr (Dense)
                            ti = p0 <= T(0) ? (j == 0 ? tiA : tiB) : a.tign[WF_CHK(g + j, nx * ny, st)];
                        else
                            ti = a.tign[WF_CHK(g + j, nx * ny, st)];
                        if (p0 > T(0) && tign_unset(ti)) {
                            const double q0 = (double)p0, q1 = (double)pn;
                            ti = tstart + q0 * a.dt / (q0 - q1);
                            if (own_row && (j == 0 ? outA : outB)) a.tign[WF_CHK(g + j, nx * ny, st)] = ti;
                        }
                        if (pn < T(0)) {
                            if (j == 0) D0.x = T(t1 - ti);
                            else D0.y = T(t1 - ti);
                        }
                    }
                }
                if (own_row) {
                    T *po = static_cast<T *>(a.psi_out);
                    const int g = rC * nx + xa;
                    if (pst) *reinterpret_cast<V *>(po + WF_CHK(g, nx * ny - 1, st)) = N0;
                    if (slow) {
                        if (!pst && outA) po[WF_CHK(g, nx * ny, st)] = N0.x;
                        if (!pst && outB) po[WF_CHK(g + 1, nx * ny, st)] = N0.y;
                    }
                }
            }
            // Dense: t_i of row k+1 where psi^n <= 0, for stage C of the
            // next iteration (such nodes get no new t_i in this step, so no
            // other warp writes them); skipped by warps with no such node,
            // whose stage C then reads no prefetched value
            if (Dense && __any_sync(0xffffffffu, P1.x <= T(0) || P1.y <= T(0))) {
                const int rn = k + 1;
                const bool rin = rn >= y0 - 1 && rn >= 0 && rn < ny;
                const int g = rn * nx + xa;
                if (rin && inA && lane > 0 && P1.x <= T(0)) tiA = a.tign[WF_CHK(g, nx * ny, st)];
                if (rin && inB && lane < 31 && P1.y <= T(0)) tiB = a.tign[WF_CHK(g + 1, nx * ny, st)];
            }
            // ---- D: fuel fraction and heat on row k-1
            const int rD = k - 1;
            if (rD >= y0 && rD < y0 + La) {
                quadrature(rD, Nm2, Nm1, N0, Dm2, Dm1, D0, Fcur);
            }
            // ---- rotate
            P0 = P1;
            P1 = P2;
            h1 = h2;
            Qm = Q0;
            Q0 = Q1;
            FA0 = FA1;
            Nm2 = Nm1;
            Nm1 = N0;
            Dm2 = Dm1;
            Dm1 = D0;
            envC = envB;
            hist <<= 1;
        }
        if (!finite_val(poison.x) || !finite_val(poison.y)) st |= ST_NONFINITE;
    }

    __device__ __forceinline__ void quadrature(int rD, V Na, V Nb, V Nc, V Da, V Db, V Dc, V Fn) {
        V F1 = splat<V>(T(1));
        // no node of the three rows had psi^{n+1} <= 0 (the votes of stage
        // 2 cover every column the quadrature reads): every cell fraction is
        // 1, skip the test below
        if ((hist & 7u) != 0u) gate(rD, Na, Nb, Nc, Da, Db, Dc, F1);
        finish_row(rD, Fn, F1);
    }

    // minimum of psi^{n+1} over the 3x3 neighbourhood of each output column
    // (in-domain values only; ghosts are never below them), and the full
    // quadrature where it is negative
    __device__ __forceinline__ void gate(int rD, V Na, V Nb, V Nc, V Da, V Db, V Dc, V &F1) {
        const T big = T(1e30);
        T va = min_val(min_val(Na.x, Nb.x), Nc.x), vb = min_val(min_val(Na.y, Nb.y), Nc.y);
        if (rD == 0) {
            va = min_val(Nb.x, Nc.x);
            vb = min_val(Nb.y, Nc.y);
        } else if (rD == ny - 1) {
            va = min_val(Na.x, Nb.x);
            vb = min_val(Na.y, Nb.y);
        }
        va = inA ? va : big;
        vb = inB ? vb : big;
        T vl, vr;
        sides(mk2(va, vb), vl, vr);
        const T ma = min_val(min_val(vl, va), vb), mb = min_val(min_val(va, vb), vr);
        const bool ba = outA && ma < T(0), bb = outB && mb < T(0);
        if (__any_sync(0xffffffffu, ba || bb)) {
            // full quadrature: neighbours of three rows of psi and t - t_i
            T pl[3], pr[3], dl[3], dr[3];
            sides(Na, pl[0], pr[0]);
            sides(Nb, pl[1], pr[1]);
            sides(Nc, pl[2], pr[2]);
            sides(Da, dl[0], dr[0]);
            sides(Db, dl[1], dr[1]);
            sides(Dc, dl[2], dr[2]);
            const V Nr[3] = {Na, Nb, Nc}, Dr[3] = {Da, Db, Dc};
            if constexpr (Dense && sizeof(T) == 4) {
                // away from the domain boundary: both cells of the lane in
                // one packed evaluation; F = 1 stays where no node of a
                // cell's neighbourhood burns
                if (rD > 0 && rD < ny - 1 && xa > 0 && xa + 1 < nx - 1) {
                    if (ba || bb) {
                        float2 qp[3][3], ep[3][3];
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            qp[b][0] = mk2(pl[b], Nr[b].x);
                            qp[b][1] = Nr[b];
                            qp[b][2] = mk2(Nr[b].y, pr[b]);
                            ep[b][0] = mk2(dl[b], Dr[b].x);
                            ep[b][1] = Dr[b];
                            ep[b][2] = mk2(Dr[b].y, dr[b]);
                        }
                        const int g = rD * nx + xa;
                        const int ca = ba ? a.fuel[WF_CHK(g, nx * ny, st)] : 0;
                        const int cb = bb ? a.fuel[WF_CHK(g + 1, nx * ny, st)] : 0;
                        const float2 tf = mk2(lut[(ca > ncm1 ? ncm1 : ca) * 8 + 6],
                                              lut[(cb > ncm1 ? ncm1 : cb) * 8 + 6]);
                        const float2 f = cell_fraction_pair(qp, ep, tf);
                        F1.x = ba ? f.x : 1.0f;
                        F1.y = bb ? f.y : 1.0f;
                    }
                    return;
                }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (!(j == 0 ? ba : bb)) continue;
                T q[3][3], e[3][3];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (j == 0) {
                        q[b][0] = pl[b];
                        q[b][1] = Nr[b].x;
                        q[b][2] = Nr[b].y;
                        e[b][0] = dl[b];
                        e[b][1] = Dr[b].x;
                        e[b][2] = Dr[b].y;
                    } else {
                        q[b][0] = Nr[b].x;
                        q[b][1] = Nr[b].y;
                        q[b][2] = pr[b];
                        e[b][0] = Dr[b].x;
                        e[b][1] = Dr[b].y;
                        e[b][2] = dr[b];
                    }
                }
                const int x = xa + j;
                if (x == 0 || x == nx - 1 || rD == 0 || rD == ny - 1) {
                    // ghost ring of psi^{n+1} (x first, then y) and of t - t_i
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int yy = rD + b - 1;
                        if (yy < 0 || yy >= ny) continue;
                        if (x == 0) {
                            q[b][0] = ghost_value<T>(q[b][1], q[b][2]);
                            e[b][0] = q[b][0] >= T(0) ? T(0) : e[b][1];
                        }
                        if (x == nx - 1) {
                            q[b][2] = ghost_value<T>(q[b][1], q[b][0]);
                            e[b][2] = q[b][2] >= T(0) ? T(0) : e[b][1];
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 3; ++h) {
                        if (rD == 0) {
                            q[0][h] = ghost_value<T>(q[1][h], q[2][h]);
                            e[0][h] = q[0][h] >= T(0) ? T(0) : e[1][h];
                        }
                        if (rD == ny - 1) {
                            q[2][h] = ghost_value<T>(q[1][h], q[0][h]);
                            e[2][h] = q[2][h] >= T(0) ? T(0) : e[1][h];
                        }
                    }
                }
                const int cls0 = a.fuel[WF_CHK(rD * nx + x, nx * ny, st)];
                const int cls = cls0 > ncm1 ? ncm1 : cls0;
                const T f = cell_fraction_vals<T>(q[0][0], q[0][1], q[0][2], q[1][0], q[1][1],
                                                  q[1][2], q[2][0], q[2][1], q[2][2], e[0][0],
                                                  e[0][1], e[0][2], e[1][0], e[1][1], e[1][2],
                                                  e[2][0], e[2][1], e[2][2], lut[cls * 8 + 6]);
                if (j == 0) F1.x = f;
                else F1.y = f;
            }
        }
    }

    // store F^{n+1} of the row, heat flux densities summed per column over
    // the band, and the per-cell average after the band's last row
    __device__ __forceinline__ void finish_row(int rD, V Fn, V F1) {
        const int g = rD * nx + xa;
        T *fo = static_cast<T *>(a.F_out);
        if (pst) *reinterpret_cast<V *>(fo + WF_CHK(g, nx * ny - 1, st)) = F1;
        if (slow) {
            if (!pst && outA) fo[WF_CHK(g, nx * ny, st)] = F1.x;
            if (!pst && outB) fo[WF_CHK(g + 1, nx * ny, st)] = F1.y;
        }
        // heat flux densities of the row, summed per column over the band
        // (the vote on every column of the warp, the sums on output columns)
        const V dF = sub2(Fn, F1);
        if (__any_sync(0xffffffffu, dF.x != T(0) || dF.y != T(0))) {
            const T dFa = outA ? dF.x : T(0), dFb = outB ? dF.y : T(0);
            if constexpr (NC) {
                const T *hs = static_cast<const T *>(a.nco[3]);
                const T *hq = static_cast<const T *>(a.nco[4]);
                if (dFa != T(0)) {
                    acc_s.x += dFa * hs[WF_CHK(g, nx * ny, st)];
                    acc_q.x += dFa * hq[WF_CHK(g, nx * ny, st)];
                }
                if (dFb != T(0)) {
                    acc_s.y += dFb * hs[WF_CHK(g + 1, nx * ny, st)];
                    acc_q.y += dFb * hq[WF_CHK(g + 1, nx * ny, st)];
                }
            } else {
                if (dFa != T(0)) {
                    int cls = a.fuel[WF_CHK(g, nx * ny, st)];
                    cls = cls > ncm1 ? ncm1 : cls;
                    acc_s.x += dFa * lut[cls * 8 + 7];
                    acc_q.x += dFa * lutq[cls];
                }
                if (dFb != T(0)) {
                    int cls = a.fuel[WF_CHK(g + 1, nx * ny, st)];
                    cls = cls > ncm1 ? ncm1 : cls;
                    acc_s.y += dFb * lut[cls * 8 + 7];
                    acc_q.y += dFb * lutq[cls];
                }
            }
        }
        // after the last row of an atmospheric band: average per cell
        if (++bcnt == sry) {
            bcnt = 0;
            // a band with no heat anywhere in the warp (most of a sparse
            // fire) writes its zero averages without the reduction
            if (__any_sync(0xffffffffu, acc_s.x != T(0) || acc_s.y != T(0) ||
                                            acc_q.x != T(0) || acc_q.y != T(0))) {
                hw[2 * lane] = acc_s.x;
                hw[2 * lane + 1] = acc_s.y;
                hw[64 + 2 * lane] = acc_q.x;
                hw[64 + 2 * lane + 1] = acc_q.y;
                __syncwarp();
                if (lane * srx < Wa) {  // one lane per atmospheric cell
                    T h0 = T(0), h1 = T(0);
                    for (int e = 0; e < srx; ++e) {
                        const int lc = 2 + lane * srx + e;
                        h0 += hw[lc];
                        h1 += hw[64 + lc];
                    }
                    const size_t ga = WF_CHK((size_t)(rD / sry) * nxa + (x0 / srx + lane), nxa * nya, st);
                    if (a.heat_s) a.heat_s[ga] = (double)h0 * hscale;
                    if (a.heat_l) a.heat_l[ga] = (double)h1 * hscale;
                }
                __syncwarp();
                acc_s = acc_q = splat<V>(T(0));
            } else if (lane * srx < Wa) {
                const size_t ga = WF_CHK((size_t)(rD / sry) * nxa + (x0 / srx + lane), nxa * nya, st);
                if (a.heat_s) a.heat_s[ga] = 0.0;
                if (a.heat_l) a.heat_l[ga] = 0.0;
            }
        }
    }
};

template <typename T, bool NC, bool Dense>
__global__ void __launch_bounds__(kWarpCtaThreads, WOcc<T>::blocks) k_fire_warp(const StepArgs a) {
    __shared__ __align__(16) T lut[FIRE_MAX_CLASSES * 8];
    __shared__ __align__(16) T lut2[FIRE_MAX_CLASSES * 12];
    __shared__ T lutq[FIRE_MAX_CLASSES];
    __shared__ __align__(16) T hw[kWarpStrips][128];
    __shared__ __align__(16) WRow<T> rows[kWarpMaxRows + 4];
    const int y0 = blockIdx.y * a.ky * a.sry;
    const int La = min(a.ky * a.sry, a.ny - y0);
    for (int i = threadIdx.x; i < La + 4; i += kWarpCtaThreads) {
        const int r = y0 - 2 + i;
        WRow<T> w;
        w.ju0 = w.jv0 = 0;
        w.wyu = w.wyv = T(0);
        if (r >= 0 && r < a.ny) {
            int j1;
            const T yr = (T(r) + T(0.5)) / T(a.sry);
            lin_idx<T>(yr - T(0.5), a.nya, w.ju0, j1, w.wyu);
            lin_idx<T>(yr, a.nya + 1, w.jv0, j1, w.wyv);
        }
        rows[i] = w;
    }
    for (int k = threadIdx.x; k < a.ncls; k += kWarpCtaThreads) {
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
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const double tstart = *a.t_in;
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) *a.t_out = tstart + a.dt;
    const int W = a.kx * a.srx;
    const int x0 = (blockIdx.x * kWarpStrips + w) * W;
    if (x0 >= a.nx) return;  // whole warp
    WarpStrip<T, NC, Dense> s(a, lut, lut2, lutq, hw[w], rows);
    s.run(x0, y0, tstart);
    const int stw = __reduce_or_sync(0xffffffffu, s.st);
    if ((threadIdx.x & 31) == 0 && stw) atomicOr(a.status, stw);
}

// dense: the Dense instantiation (FP32 with the class table; elsewhere the
// other one, which gives the same results)
template <typename T>
cudaError_t launch_warp(const StepArgs &a, cudaStream_t s, bool dense) {
    const int W = a.kx * a.srx, L = a.ky * a.sry;
    if (W > 60 || (W & 1) || W < 2 || L > kWarpMaxRows || (long long)a.nx * a.ny > kWarpMaxNodes)
        return cudaErrorInvalidValue;
    const int strips = (a.nx + W - 1) / W;
    dim3 grid((strips + kWarpStrips - 1) / kWarpStrips, (a.ny + L - 1) / L);
    if (a.nco[0]) {
        k_fire_warp<T, true, false><<<grid, kWarpCtaThreads, 0, s>>>(a);
    } else if (dense && sizeof(T) == 4) {
        k_fire_warp<T, false, sizeof(T) == 4><<<grid, kWarpCtaThreads, 0, s>>>(a);
    } else {
        k_fire_warp<T, false, false><<<grid, kWarpCtaThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

#define WF_INSTANTIATE_WARP(T) \
    template cudaError_t launch_warp<T>(const StepArgs &, cudaStream_t, bool);

}  // namespace wf
