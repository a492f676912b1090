// Column-marching fire-step kernel: the whole step of Sect. 5 (items 2-6)
// in one pass over the state, two fire-mesh columns per thread.
//
// A CTA of 128 threads owns a strip of W = kx*srx output columns (W even,
// W <= 248) and L = ky*sry output rows; thread c holds the columns
// x0 - 4 + 2c and x0 - 3 + 2c, so the CTA covers the strip plus 4 halo
// columns on each side.  It marches down the strip one row per iteration,
// the stages lagging behind the loads:
//   iteration k:  A  stage psi^n of row k+3 (loaded one iteration earlier)
//                 B  stage 1 (eq. Heun, first line) on row k+2
//                 C  stage 2 (eq. Heun, second line), ignition-time crossing
//                    (eq. set-ignition-time) and t - t_i on row k+1
//                 D  fuel-fraction quadrature (Sect. 3.3) and heat flux
//                    (eqs. sensible-/latent-heat-flux) on row k-1
//                 one __syncthreads
// Every shared value read from another thread was written in an earlier
// iteration (values of the thread's own columns may come from the same
// iteration), so one barrier per row suffices; each stage keeps a ring of 4
// rows.  Stage 2 runs one row behind stage 1, so the fuel class, terrain
// gradient and wind of a row are loaded once and carried in registers.  Vertical neighbours cost no recomputation: the only redundant
// work is the 2+1 halo columns of the two stages.  Ghost values beyond the
// domain (Sect. 3.1, x first then y) are computed by the thread that needs
// them.  The wind is interpolated in x once per atmospheric row and column
// (a per-thread ring of 4 rows) and in y per node.  Heat is summed per
// column over each band of sry rows, then per atmospheric cell in double
// after the band's last row: the average of Sect. 5, item 6, inside the CTA.
#pragma once

#include <mutex>

#include "fire_device.cuh"
#include "fire_internal.h"
#include "pair_math.cuh"

namespace wf {

constexpr int kMarchThreads = 128;
constexpr int kMarchHalo = 4;  // columns on each side of the strip
constexpr int kMarchCols = 2;  // columns per thread

// resident CTAs per SM the register allocation aims for (FP64 needs more
// registers per thread)
template <typename T>
struct MarchOccupancy {
    static constexpr int blocks = 5;
};
template <>
struct MarchOccupancy<double> {
    static constexpr int blocks = 2;
};
static_assert(MarchOccupancy<float>::blocks == kMarchCtasPerSmF32 &&
                  MarchOccupancy<double>::blocks == kMarchCtasPerSmF64,
              "default launch shapes assume these");

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T>
struct MarchRow {  // y-interpolation of the wind for one fire row
    int ju0, jv0;
    T wyu, wyv;
};

template <typename T>
struct MarchCol {  // x-interpolation of the wind for one fire column
    int iu0, iu1, iv0, iv1;
    T wxu, wxv;
};

// dynamic shared memory layout of the marching kernel
template <typename T>
struct MarchSmem {
    using T2 = typename Vec2<T>::type;
    T2 *S0, *S1, *SF, *SQ, *SD;  // [4][NT] psi^n, psi*, -F(psi^n), psi^{n+1}, t - t_i
    T2 *UX, *VX;                 // [4][NT] x-interpolated wind of 4 atmos rows (per thread)
    T *lut;                      // [ncls][8] S0 R0 b c d e Tf Hs
    T *lutq;                     // [ncls] Hq
    T *HB;                       // [2][2][2 NT] heat column partials of 2 bands
    MarchCol<T> *col;            // [2 NT]
    MarchRow<T> *row;            // [L + 4]
    int *status;

    static __host__ __device__ size_t bytes(int L, int ncls) {
        const size_t NT = kMarchThreads;
        size_t b = 0;
        b += 7 * 4 * NT * sizeof(T2);
        b += (size_t)ncls * 8 * sizeof(T) + (size_t)ncls * sizeof(T);
        b = (b + 15) & ~(size_t)15;
        b += 2 * 2 * 2 * NT * sizeof(T);
        b += 2 * NT * sizeof(MarchCol<T>);
        b = (b + 15) & ~(size_t)15;
        b += (size_t)(L + 4) * sizeof(MarchRow<T>);
        b += 16;
        return b;
    }

    __device__ void carve(unsigned char *p, int L, int ncls) {
        const int NT = kMarchThreads;
        T2 *v = reinterpret_cast<T2 *>(p);
        S0 = v;
        S1 = v + 4 * NT;
        SF = v + 8 * NT;
        SQ = v + 12 * NT;
        SD = v + 16 * NT;
        UX = v + 20 * NT;
        VX = v + 24 * NT;
        unsigned char *q = reinterpret_cast<unsigned char *>(v + 28 * NT);
        lut = reinterpret_cast<T *>(q);
        lutq = lut + ncls * 8;
        q += (size_t)ncls * 9 * sizeof(T);
        q = reinterpret_cast<unsigned char *>(((uintptr_t)q + 15) & ~(uintptr_t)15);
        HB = reinterpret_cast<T *>(q);
        q += 2 * 2 * 2 * NT * sizeof(T);
        col = reinterpret_cast<MarchCol<T> *>(q);
        q += 2 * NT * sizeof(MarchCol<T>);
        q = reinterpret_cast<unsigned char *>(((uintptr_t)q + 15) & ~(uintptr_t)15);
        row = reinterpret_cast<MarchRow<T> *>(q);
        q += (size_t)(L + 4) * sizeof(MarchRow<T>);
        status = reinterpret_cast<int *>(q);
    }
};

template <typename T>
__device__ __forceinline__ T pick(const typename Vec2<T>::type &v, int j) {
    return j == 0 ? v.x : v.y;
}

// Per-thread state of one strip.  NC: per-node R0, c, d and heat factors (a
// per-node fuel moisture) from the planes of StepArgs::nco.
template <typename T, bool NC = false>
struct MarchStrip {
    using T2 = typename Vec2<T>::type;
    const StepArgs &a;
    MarchSmem<T> &sm;
    int c, x0, y0, Wa, La, nx, ny, nxa, nya, srx, sry, ncm1, band;
    int xa;  // global column of this thread's first column
    bool vec;  // paired vector access allowed (nx and x even)
    bool m_load[2], m_s1[2], m_s2[2], m_out[2];
    T dt, idx, idy, i2dx, i2dy, eps;
    T2 ndt2, idx2, idy2, i2dx2, i2dy2, eps2, ndth2;
    double tstart, t1;
    // running state
    T2 pf_psi;    // psi^n of the next row to stage
    T2 cur_psi;   // psi^n of the row staged this iteration
    int pf_fa, pf_fb;  // raw fuel-class bytes of the prefetched row (decoded at use)
    T2 pf_zx, pf_zy, pf_m;
    T2 pf_R0, pf_c, pf_d, e_R0, e_c, e_d;  // per-node coefficients (NC only)
    T2 pf_F;
    int e_cls[2];       // environment of the row stage 1 handled last iteration
    T2 e_zx, e_zy, e_m, e_un, e_vn;
    T acc_s[2], acc_q[2];
    double hscale;     // 1 / (dt srx sry)
    int ju_hi, jv_hi;  // highest atmos rows in this thread's wind ring
    int bcnt, bpar;    // rows done in the current band, band parity
    mutable int st;  // status bits (also set by the const loaders' index checks)

    __device__ __forceinline__ MarchStrip(const StepArgs &args, MarchSmem<T> &s) : a(args), sm(s) {}

    __device__ __forceinline__ bool in_rows(int r, int lo, int hi) const {
        return r >= lo && r < hi && r >= 0 && r < ny;
    }

    // paired load of a T field at (r, xa).  Every thread loads, columns
    // outside the domain from the nearest inside one (the values of those
    // columns are never used), so the loaded registers are not touched
    // before their use and a prefetch one row ahead hides the latency.
    __device__ __forceinline__ T2 ld2(const T *__restrict__ f, int r) const {
        const size_t rowb = (size_t)r * nx;
        if (vec) {
            const int xc = min(max(xa, 0), nx - 2);
            return *reinterpret_cast<const T2 *>(f + WF_CHK(rowb + xc, (long long)nx * ny - 1, st));
        }
        const int xA = min(max(xa, 0), nx - 1), xB = min(max(xa + 1, 0), nx - 1);
        return mk2(f[WF_CHK(rowb + xA, (long long)nx * ny, st)], f[WF_CHK(rowb + xB, (long long)nx * ny, st)]);
    }

    __device__ __forceinline__ void load_env(int r) {
        r = min(max(r, 0), ny - 1);
        const size_t rowb = (size_t)r * nx;
        if (vec) {
            const int xc = min(max(xa, 0), nx - 2);
            pf_fa = *reinterpret_cast<const uint16_t *>(a.fuel + WF_CHK(rowb + xc, (long long)nx * ny - 1, st));
        } else {
            pf_fa = a.fuel[WF_CHK(rowb + min(max(xa, 0), nx - 1), (long long)nx * ny, st)];
            pf_fb = a.fuel[WF_CHK(rowb + min(max(xa + 1, 0), nx - 1), (long long)nx * ny, st)];
        }
        pf_zx = ld2(static_cast<const T *>(a.dzdx), r);
        pf_zy = ld2(static_cast<const T *>(a.dzdy), r);
        if (a.mult) pf_m = ld2(static_cast<const T *>(a.mult), r);
        if constexpr (NC) {
            pf_R0 = ld2(static_cast<const T *>(a.nco[0]), r);
            pf_c = ld2(static_cast<const T *>(a.nco[1]), r);
            pf_d = ld2(static_cast<const T *>(a.nco[2]), r);
        }
    }

    // x-interpolated wind of atmos u-row J / v-row J for this thread's columns
    __device__ __forceinline__ void fill_wind_u(int J) {
        const T *u = static_cast<const T *>(a.u);
        const size_t b = (size_t)J * (nxa + 1);
        const long long n = (long long)nya * (nxa + 1);
        T2 v;
        const MarchCol<T> &c0 = sm.col[2 * c], &c1 = sm.col[2 * c + 1];
        v.x = (T(1) - c0.wxu) * __ldg(u + WF_CHK(b + c0.iu0, n, st)) +
              c0.wxu * __ldg(u + WF_CHK(b + c0.iu1, n, st));
        v.y = (T(1) - c1.wxu) * __ldg(u + WF_CHK(b + c1.iu0, n, st)) +
              c1.wxu * __ldg(u + WF_CHK(b + c1.iu1, n, st));
        sm.UX[(J & 3) * kMarchThreads + c] = v;
    }
    __device__ __forceinline__ void fill_wind_v(int J) {
        const T *w = static_cast<const T *>(a.v);
        const size_t b = (size_t)J * nxa;
        const long long n = (long long)(nya + 1) * nxa;
        T2 v;
        const MarchCol<T> &c0 = sm.col[2 * c], &c1 = sm.col[2 * c + 1];
        v.x = (T(1) - c0.wxv) * __ldg(w + WF_CHK(b + c0.iv0, n, st)) +
              c0.wxv * __ldg(w + WF_CHK(b + c0.iv1, n, st));
        v.y = (T(1) - c1.wxv) * __ldg(w + WF_CHK(b + c1.iv0, n, st)) +
              c1.wxv * __ldg(w + WF_CHK(b + c1.iv1, n, st));
        sm.VX[(J & 3) * kMarchThreads + c] = v;
    }

    // wind at fire row r for both columns (bilinear, as the staggered-grid
    // interpolation of Sect. 5); ensure=true extends this thread's ring
    __device__ __forceinline__ void wind(int r, bool ensure, T2 &un, T2 &vn) {
        const MarchRow<T> w = sm.row[r - (y0 - 2)];
        const int ju1 = nya == 1 ? w.ju0 : w.ju0 + 1;
        const int jv1 = w.jv0 + 1;
        if (ensure) {
            if (ju_hi < w.ju0 - 1) ju_hi = w.ju0 - 1;
            if (jv_hi < w.jv0 - 1) jv_hi = w.jv0 - 1;
            while (ju_hi < ju1) fill_wind_u(++ju_hi);
            while (jv_hi < jv1) fill_wind_v(++jv_hi);
        }
        const T2 ua = sm.UX[(w.ju0 & 3) * kMarchThreads + c];
        const T2 ub = sm.UX[(ju1 & 3) * kMarchThreads + c];
        const T2 va = sm.VX[(w.jv0 & 3) * kMarchThreads + c];
        const T2 vb = sm.VX[(jv1 & 3) * kMarchThreads + c];
        un.x = (T(1) - w.wyu) * ua.x + w.wyu * ub.x;
        un.y = (T(1) - w.wyu) * ua.y + w.wyu * ub.y;
        vn.x = (T(1) - w.wyv) * va.x + w.wyv * vb.x;
        vn.y = (T(1) - w.wyv) * va.y + w.wyv * vb.y;
    }

    // the 5-point values of both columns of the thread at row r from ring
    // slot sr of a staged field B (down: slot sd, up: value given), with
    // ghosts at the domain boundary (Sect. 3.1), and -F there (pair arithmetic)
    __device__ __forceinline__ T2 stage_rhs2(const T2 *B, int sr, int sd, T2 up, int r, int cls0,
                                             int cls1, T2 zx, T2 zy, T2 m, T2 un, T2 vn, T2 nR0,
                                             T2 nc, T2 nd) const {
        const int NT = kMarchThreads;
        const T2 own = B[sr * NT + c];
        T2 L = mk2(B[sr * NT + c - 1].y, own.x), R = mk2(own.y, B[sr * NT + c + 1].x);
        T2 D = B[sd * NT + c], U = up;
        if (xa <= 0 || xa + 1 >= nx - 1 || r == 0 || r == ny - 1) {
            const T2 L0 = L, D0 = D, U0 = U;
            if (xa == 0) L.x = ghost_value<T>(own.x, own.y);
            if (xa == nx - 1) R.x = ghost_value<T>(own.x, L0.x);
            if (xa + 1 == nx - 1) R.y = ghost_value<T>(own.y, own.x);
            if (r == 0) D = mk2(ghost_value<T>(own.x, U0.x), ghost_value<T>(own.y, U0.y));
            if (r == ny - 1) U = mk2(ghost_value<T>(own.x, D0.x), ghost_value<T>(own.y, D0.y));
        }
        WCoef<T> co;
        coef_pair<T>(sm.lut, cls0 > ncm1 ? ncm1 : cls0, cls1 > ncm1 ? ncm1 : cls1, co);
        if constexpr (NC) {
            co.R0 = nR0;
            co.c = nc;
            co.d = nd;
        }
        return neg_rhs2<T>(own, L, R, D, U, idx2, idy2, i2dx2, i2dy2, eps2, co, m, un, vn, zx, zy);
    }

    __device__ __forceinline__ void iter(int k) {
        const int NT = kMarchThreads;
        // ring slots: row k+3 -> s3, k+2 -> s2, k+1 -> s1, k -> s0, k-1 -> s3, k-2 -> s2
        const int s0 = k & 3, s1 = (k + 1) & 3, s2 = (k + 2) & 3, s3 = (k + 3) & 3;
        // F^n of row k, used by the quadrature of the next iteration: loaded
        // here, a full iteration before the row k-1 value is used
        const T2 Fcur = pf_F;
        pf_F = ld2(static_cast<const T *>(a.F_in), min(max(k, 0), ny - 1));
        // ---- A: stage psi^n of row k+3, prefetch row k+4
        {
            const int r = k + 3;
            cur_psi = pf_psi;
            if (r >= y0 - 3 && r < y0 + La + 3) sm.S0[s3 * NT + c] = cur_psi;
            // unconditional prefetches (rows outside the domain from the
            // nearest inside row, never used), so that a loaded register is
            // not merged with its older value when the load arrives
            pf_psi = ld2(static_cast<const T *>(a.psi_in), min(max(k + 4, 0), ny - 1));
        }
        // ---- B: stage 1 on row k+2 (its environment is carried to C)
        const int eb_cls0 = e_cls[0], eb_cls1 = e_cls[1];
        const T2 eb_zx = e_zx, eb_zy = e_zy, eb_m = e_m, eb_un = e_un, eb_vn = e_vn;
        T2 eb_R0, eb_c, eb_d;  // read by stage_rhs2 only with NC
        if constexpr (NC) {
            eb_R0 = e_R0;
            eb_c = e_c;
            eb_d = e_d;
        }
        {
            const int r = k + 2;
            e_cls[0] = vec ? (pf_fa & 0xff) : pf_fa;
            e_cls[1] = vec ? (pf_fa >> 8) : pf_fb;
            e_zx = pf_zx;
            e_zy = pf_zy;
            e_m = pf_m;
            if constexpr (NC) {
                e_R0 = pf_R0;
                e_c = pf_c;
                e_d = pf_d;
            }
            load_env(k + 3);
            if (in_rows(r, y0 - 2, y0 + La + 2) && (m_s1[0] || m_s1[1])) {
                wind(r, true, e_un, e_vn);
                if ((m_s1[0] && (!finite_val(e_un.x) || !finite_val(e_vn.x))) ||
                    (m_s1[1] && (!finite_val(e_un.y) || !finite_val(e_vn.y))))
                    st |= ST_NONFINITE;
                T2 F = stage_rhs2(sm.S0, s2, s1, cur_psi, r, e_cls[0], e_cls[1], e_zx, e_zy, e_m,
                                  e_un, e_vn, e_R0, e_c, e_d);
                F.x = m_s1[0] ? F.x : T(0);
                F.y = m_s1[1] ? F.y : T(0);
                const T2 own = sm.S0[s2 * NT + c];
                sm.S1[s2 * NT + c] = fma2(ndt2, F, own);
                sm.SF[s2 * NT + c] = F;
            }
        }
        // ---- C: stage 2, crossing, t - t_i on row k+1 (environment from B)
        {
            const int r = k + 1;
            if (in_rows(r, y0 - 1, y0 + La + 1) && (m_s2[0] || m_s2[1])) {
                const size_t g = (size_t)r * nx + xa;
                const T2 up = sm.S1[s2 * NT + c];
                const T2 p0v = sm.S0[s1 * NT + c];
                const T2 f1v = sm.SF[s1 * NT + c];
                const bool own_row = r >= y0 && r < y0 + La;
                T2 DL;
                const T2 F2 = stage_rhs2(sm.S1, s1, s0, up, r, eb_cls0, eb_cls1, eb_zx, eb_zy, eb_m,
                                         eb_un, eb_vn, eb_R0, eb_c, eb_d);
                T2 PN = fma2(ndth2, add2(f1v, F2), p0v);
                PN.x = m_s2[0] ? PN.x : T(0);
                PN.y = m_s2[1] ? PN.y : T(0);
                bool need[2] = {m_s2[0] && PN.x <= T(0), m_s2[1] && PN.y <= T(0)};
                if (own_row) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (!m_out[j]) continue;
                        const T pn = pick<T>(PN, j);
                        if (!finite_val(pn)) st |= ST_NONFINITE;
                        const int x = xa + j;
                        const bool edge = x < band || r < band || x >= nx - band || r >= ny - band;
                        if (edge && pn < T(0)) st |= ST_BOUNDARY;
                    }
                }
                DL.x = DL.y = T(0);
                // ignition time and t - t_i (double arithmetic) only in warps
                // that have a crossing or burning node: elsewhere the FP64
                // pipe is not touched at all
                if (__any_sync(__activemask(), need[0] || need[1])) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (!need[j]) continue;
                        const T p0 = pick<T>(p0v, j), pn = pick<T>(PN, j);
                        const bool cross = p0 > T(0);
                        double ti = a.tign[WF_CHK(g + j, (long long)nx * ny, st)];
                        if (cross && isinf(ti)) {
                            const double q0 = (double)p0, q1 = (double)pn;
                            ti = tstart + q0 * a.dt / (q0 - q1);
                            if (own_row && m_out[j]) a.tign[WF_CHK(g + j, (long long)nx * ny, st)] = ti;
                        }
                        if (pn < T(0)) {
                            if (j == 0) DL.x = T(t1 - ti);
                            else DL.y = T(t1 - ti);
                        }
                    }
                }
                sm.SQ[s1 * NT + c] = PN;
                sm.SD[s1 * NT + c] = DL;
                if (own_row) {
                    T *po = static_cast<T *>(a.psi_out);
                    if (vec && m_out[0] && m_out[1]) {
                        *reinterpret_cast<T2 *>(po + WF_CHK(g, (long long)nx * ny - 1, st)) = PN;
                    } else {
                        if (m_out[0]) po[WF_CHK(g, (long long)nx * ny, st)] = PN.x;
                        if (m_out[1]) po[WF_CHK(g + 1, (long long)nx * ny, st)] = PN.y;
                    }
                }
            }
        }
        // ---- D: fuel fraction and heat on row k-1
        const int rd = k - 1;
        const bool drow = rd >= y0 && rd < y0 + La;
        if (drow && (m_out[0] || m_out[1])) {
            // psi^{n+1} on rows rd-1 (slot s2), rd (s3), rd+1 (s0), columns -1..2
            T p[3][4];
            {
                const int sl[3] = {s2, s3, s0};
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T2 o = sm.SQ[sl[b] * NT + c];
                    p[b][0] = sm.SQ[sl[b] * NT + c - 1].y;
                    p[b][1] = o.x;
                    p[b][2] = o.y;
                    p[b][3] = sm.SQ[sl[b] * NT + c + 1].x;
                }
            }
            T vmin[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) vmin[h] = min_val(min_val(p[0][h], p[1][h]), p[2][h]);
            const T mid = min_val(vmin[1], vmin[2]);
            const T mn0 = min_val(vmin[0], mid), mn1 = min_val(mid, vmin[3]);
            const bool edge = xa <= 0 || xa + 1 >= nx - 1 || rd == 0 || rd == ny - 1;
            T Fn[2] = {T(1), T(1)};
            if (mn0 < T(0) || mn1 < T(0) || edge) {
                T d[3][4];
                const int sl[3] = {s2, s3, s0};
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T2 o = sm.SD[sl[b] * NT + c];
                    d[b][0] = sm.SD[sl[b] * NT + c - 1].y;
                    d[b][1] = o.x;
                    d[b][2] = o.y;
                    d[b][3] = sm.SD[sl[b] * NT + c + 1].x;
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (!m_out[j]) continue;
                    T q[3][3], e[3][3];
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int h = 0; h < 3; ++h) {
                            q[b][h] = p[b][j + h];
                            e[b][h] = d[b][j + h];
                        }
                    const int x = xa + j;
                    if (x == 0 || x == nx - 1 || rd == 0 || rd == ny - 1) {
                        // ghost ring of psi^{n+1} (x first, then y) and of t - t_i
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            const int yy = rd + b - 1;
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
                            if (rd == 0) {
                                q[0][h] = ghost_value<T>(q[1][h], q[2][h]);
                                e[0][h] = q[0][h] >= T(0) ? T(0) : e[1][h];
                            }
                            if (rd == ny - 1) {
                                q[2][h] = ghost_value<T>(q[1][h], q[0][h]);
                                e[2][h] = q[2][h] >= T(0) ? T(0) : e[1][h];
                            }
                        }
                    }
                    const int cls0 = a.fuel[WF_CHK((size_t)rd * nx + x, (long long)nx * ny, st)];
                    const int cls = cls0 > ncm1 ? ncm1 : cls0;
                    Fn[j] = cell_fraction_vals<T>(q[0][0], q[0][1], q[0][2], q[1][0], q[1][1],
                                                  q[1][2], q[2][0], q[2][1], q[2][2], e[0][0],
                                                  e[0][1], e[0][2], e[1][0], e[1][1], e[1][2],
                                                  e[2][0], e[2][1], e[2][2], sm.lut[cls * 8 + 6]);
                }
            }
            const size_t g = (size_t)rd * nx + xa;
            T *fo = static_cast<T *>(a.F_out);
            T2 FN;
            FN.x = Fn[0];
            FN.y = Fn[1];
            if (vec && m_out[0] && m_out[1]) {
                *reinterpret_cast<T2 *>(fo + WF_CHK(g, (long long)nx * ny - 1, st)) = FN;
            } else {
                if (m_out[0]) fo[WF_CHK(g, (long long)nx * ny, st)] = FN.x;
                if (m_out[1]) fo[WF_CHK(g + 1, (long long)nx * ny, st)] = FN.y;
            }
            // heat flux densities, only in warps where some fuel burned
            const T dF0 = m_out[0] ? Fcur.x - Fn[0] : T(0);
            const T dF1 = m_out[1] ? Fcur.y - Fn[1] : T(0);
            if (__any_sync(__activemask(), dF0 != T(0) || dF1 != T(0))) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const T dF = j == 0 ? dF0 : dF1;
                    if (dF != T(0)) {
                        if constexpr (NC) {
                            acc_s[j] += dF * static_cast<const T *>(a.nco[3])[WF_CHK(g + j, (long long)nx * ny, st)];
                            acc_q[j] += dF * static_cast<const T *>(a.nco[4])[WF_CHK(g + j, (long long)nx * ny, st)];
                        } else {
                            const int cls0 = a.fuel[WF_CHK(g + j, (long long)nx * ny, st)];
                            const int cls = cls0 > ncm1 ? ncm1 : cls0;
                            acc_s[j] += dF * sm.lut[cls * 8 + 7];
                            acc_q[j] += dF * sm.lutq[cls];
                        }
                    }
                }
            }
        }
        bool band_end = false;
        if (drow) {
            if (++bcnt == sry) {
                band_end = true;
                bcnt = 0;
                T *hb = sm.HB + bpar * 4 * NT;
                hb[2 * c] = acc_s[0];
                hb[2 * c + 1] = acc_s[1];
                hb[2 * NT + 2 * c] = acc_q[0];
                hb[2 * NT + 2 * c + 1] = acc_q[1];
                acc_s[0] = acc_s[1] = acc_q[0] = acc_q[1] = T(0);
            }
        }
        __syncthreads();
        // ---- average over the band's atmospheric cells (after its last row)
        if (band_end) {
            const int kxa = Wa / srx;
            if (c < kxa) {
                const T *hb = sm.HB + bpar * 4 * NT;
                // the cell's column sums in the path precision, one
                // conversion to double per atmospheric cell
                T h0 = T(0), h1 = T(0);
                for (int e = 0; e < srx; ++e) {
                    const int lc = kMarchHalo + c * srx + e;
                    h0 += hb[lc];
                    h1 += hb[2 * NT + lc];
                }
                const size_t ga = WF_CHK((size_t)(rd / sry) * nxa + (x0 / srx + c), (long long)nxa * nya, st);
                if (a.heat_s) a.heat_s[ga] = (double)h0 * hscale;
                if (a.heat_l) a.heat_l[ga] = (double)h1 * hscale;
            }
            bpar ^= 1;
        }
    }

    // one step of the strip with output origin (x0_, y0_); tstart_ is the
    // model time at the step start
    __device__ __forceinline__ void run(int x0_, int y0_, double tstart_) {
        const int NT = kMarchThreads;
        c = threadIdx.x;
        srx = a.srx;
        sry = a.sry;
        nx = a.nx;
        ny = a.ny;
        nxa = a.nxa;
        nya = a.nya;
        x0 = x0_;
        y0 = y0_;
        const int W = a.kx * srx, L = a.ky * sry;
        Wa = min(W, nx - x0);
        La = min(L, ny - y0);
        xa = x0 - kMarchHalo + kMarchCols * c;
        vec = (nx % 2) == 0;  // x0 and xa are even (W even)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int lc = kMarchCols * c + j, x = xa + j;
            const bool xin = x >= 0 && x < nx;
            m_load[j] = xin && lc >= 1 && lc < Wa + 7;
            m_s1[j] = xin && lc >= 2 && lc < Wa + 6;
            m_s2[j] = xin && lc >= 3 && lc < Wa + 5;
            m_out[j] = lc >= 4 && lc < Wa + 4;
        }
        dt = T(a.dt);
        idx = T(1) / T(a.dx);
        idy = T(1) / T(a.dy);
        i2dx = T(1) / (T(2) * T(a.dx));
        i2dy = T(1) / (T(2) * T(a.dy));
        eps = T(a.eps);
        ndt2 = mk2(-dt, -dt);
        idx2 = mk2(idx, idx);
        idy2 = mk2(idy, idy);
        i2dx2 = mk2(i2dx, i2dx);
        i2dy2 = mk2(i2dy, i2dy);
        eps2 = mk2(eps, eps);
        ndth2 = mk2(-(T(0.5) * dt), -(T(0.5) * dt));
        tstart = tstart_;
        t1 = tstart + a.dt;
        ncm1 = a.ncls - 1;
        band = a.band;
        st = 0;
        acc_s[0] = acc_s[1] = acc_q[0] = acc_q[1] = T(0);
        bcnt = 0;
        bpar = 0;
        ju_hi = -1;
        jv_hi = -1;

        // ---- set-up: coefficients, row and column wind weights
        for (int k = c; k < a.ncls; k += NT) {
            const double *co = a.coef + (size_t)k * K_N;
            T *l = sm.lut + k * 8;
            l[0] = T(co[K_S0]);
            l[1] = T(co[K_R0]);
            l[2] = T(co[K_B]);
            l[3] = T(co[K_C]);
            l[4] = T(co[K_D]);
            l[5] = T(co[K_E]);
            l[6] = T(co[K_TF]);
            l[7] = T(co[K_HS]);
            sm.lutq[k] = T(co[K_HQ]);
        }
        for (int i = c; i < La + 4; i += NT) {
            const int r = y0 - 2 + i;
            MarchRow<T> w;
            w.ju0 = w.jv0 = 0;
            w.wyu = w.wyv = T(0);
            if (r >= 0 && r < ny) {
                int j1;
                const T yr = (T(r) + T(0.5)) / T(sry);
                lin_idx<T>(yr - T(0.5), nya, w.ju0, j1, w.wyu);
                lin_idx<T>(yr, nya + 1, w.jv0, j1, w.wyv);
            }
            sm.row[i] = w;
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            MarchCol<T> cw;
            cw.iu0 = cw.iu1 = cw.iv0 = cw.iv1 = 0;
            cw.wxu = cw.wxv = T(0);
            const int x = xa + j;
            if (x >= 0 && x < nx) {
                const T xr = (T(x) + T(0.5)) / T(srx);
                lin_idx<T>(xr, nxa + 1, cw.iu0, cw.iu1, cw.wxu);
                lin_idx<T>(xr - T(0.5), nxa, cw.iv0, cw.iv1, cw.wxv);
            }
            sm.col[kMarchCols * c + j] = cw;
        }
        __syncthreads();

        const int k0 = y0 - 6, k1 = y0 + La;
        hscale = 1.0 / (a.dt * (double)srx * (double)sry);
        pf_psi.x = pf_psi.y = T(0);
        if (in_rows(k0 + 3, y0 - 3, y0 + La + 3))
            pf_psi = ld2(static_cast<const T *>(a.psi_in), k0 + 3);
        pf_fa = pf_fb = 0;
        pf_zx.x = pf_zx.y = pf_zy.x = pf_zy.y = T(0);
        pf_m.x = pf_m.y = T(1);
        if constexpr (NC) pf_R0 = pf_c = pf_d = pf_zx;
        load_env(k0 + 2);
        e_cls[0] = e_cls[1] = 0;
        e_zx = pf_zx;
        e_zy = pf_zy;
        e_m = pf_m;
        if constexpr (NC) {
            e_R0 = pf_R0;
            e_c = pf_c;
            e_d = pf_d;
        }
        e_un = pf_zx;
        e_vn = pf_zx;
        pf_F.x = pf_F.y = T(1);
#pragma unroll 1
        for (int k = k0; k <= k1; ++k) iter(k);
    }
};

template <typename T, bool NC>
__global__ void __launch_bounds__(kMarchThreads, MarchOccupancy<T>::blocks) k_fire_march(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    MarchSmem<T> sm;
    sm.carve(dyn_smem, a.ky * a.sry, a.ncls);
    if (threadIdx.x == 0) {
        *sm.status = 0;
        if (blockIdx.x == 0 && blockIdx.y == 0) *a.t_out = *a.t_in + a.dt;
    }
    MarchStrip<T, NC> s(a, sm);
    s.run(blockIdx.x * a.kx * a.srx, blockIdx.y * a.ky * a.sry, *a.t_in);
    if (s.st) atomicOr(sm.status, s.st);
    __syncthreads();
    if (threadIdx.x == 0 && *sm.status) atomicOr(a.status, *sm.status);
}

template <typename T>
size_t march_smem_bytes(int ky, int sry, int ncls) {
    return MarchSmem<T>::bytes(ky * sry, ncls);
}

// The dynamic shared-memory limit is an attribute of the kernel function,
// shared by every context in the process: raise it monotonically.
template <typename T>
cudaError_t prepare_march_kernel(size_t smem_bytes) {
    static std::mutex mu;
    static size_t current[kMaxDevices] = {};  // per device (the attribute is)
    std::lock_guard<std::mutex> lock(mu);
    const int dev = attr_device();
    if (dev >= 0 && smem_bytes <= current[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fire_march<T, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fire_march<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes);
    if (e == cudaSuccess && dev >= 0) current[dev] = smem_bytes;
    return e;
}

template <typename T>
cudaError_t launch_march(const StepArgs &a, cudaStream_t s) {
    const int W = a.kx * a.srx, L = a.ky * a.sry;
    dim3 grid((a.nx + W - 1) / W, (a.ny + L - 1) / L);
    const size_t smem = march_smem_bytes<T>(a.ky, a.sry, a.ncls);
    cudaError_t e = prepare_march_kernel<T>(smem);
    if (e != cudaSuccess) return e;
    if (a.nco[0])
        k_fire_march<T, true><<<grid, kMarchThreads, smem, s>>>(a);
    else
        k_fire_march<T, false><<<grid, kMarchThreads, smem, s>>>(a);
    return cudaGetLastError();
}

#define WF_INSTANTIATE_MARCH(T)                                               \
    template size_t march_smem_bytes<T>(int, int, int);                       \
    template cudaError_t launch_march<T>(const StepArgs &, cudaStream_t);     \
    template cudaError_t prepare_march_kernel<T>(size_t);

}  // namespace wf
