// Column-marching fire-step kernel: the whole step of Sect. 5 (items 2-6)
// in one pass over the state, one thread per fire-mesh column.
//
// A CTA of 128 threads owns a strip of W = kx*srx output columns (W <= 120)
// and L = ky*sry output rows; its threads cover the strip's columns plus 4
// halo columns on each side.  It marches down the strip one row per
// iteration, with the stages lagging behind the loads:
//   iteration k:  A  store psi^n of row k+4 (loaded one iteration earlier)
//                 B  stage 1 (eq. Heun, first line) on row k+3
//                 C  stage 2 (eq. Heun, second line), ignition-time crossing
//                    (eq. set-ignition-time) and t - t_i on row k+1
//                 D  fuel-fraction quadrature (Sect. 3.3) and heat flux
//                    (eqs. sensible-/latent-heat-flux) on row k-1
//                 one __syncthreads
// Every shared-memory value a phase reads from another thread was written in
// an earlier iteration, so one barrier per row suffices; each stage keeps a
// ring of 4 rows.  Vertical neighbours cost no recomputation, so the only
// redundant work is the 2+1 halo columns of the two stages.  Ghost values
// beyond the domain (Sect. 3.1, x first then y) are computed by the thread
// that needs them from values it reads anyway.  Heat is summed per column
// over each band of sry rows, then per atmospheric cell in double after the
// band's last row: the average of Sect. 5, item 6, reduced inside the CTA.
#pragma once

#include "fire_device.cuh"
#include "fire_internal.h"

namespace wf {

constexpr int kMarchThreads = 128;
constexpr int kMarchHalo = 4;   // columns on each side of the strip
constexpr int kRing = 4;        // rows kept per stage

template <typename T>
struct RowWeights {
    int ju0, ju1, jv0, jv1;  // atmos rows bracketing the node (u centres, v faces)
    T wyu, wyv;
};

template <typename T>
__host__ __device__ inline int march_max_width(int srx) {
    return (kMarchThreads - 2 * kMarchHalo) / srx;  // atmos cells per strip
}

template <typename T>
__global__ void __launch_bounds__(kMarchThreads) k_fire_march(const StepArgs a) {
    constexpr int NT = kMarchThreads;
    __shared__ T S0[kRing][NT];  // psi^n
    __shared__ T S1[kRing][NT];  // psi*
    __shared__ T SF[kRing][NT];  // F(psi^n)
    __shared__ T SQ[kRing][NT];  // psi^{n+1}
    __shared__ T SD[kRing][NT];  // t - t_i where psi^{n+1} < 0, else 0
    __shared__ T lut[FIRE_MAX_CLASSES * K_N];
    __shared__ T HB[2][2][NT];   // per-column heat partials of a band (2 bands in flight)
    __shared__ int s_status;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    RowWeights<T> *rw = reinterpret_cast<RowWeights<T> *>(dyn_smem);

    const int c = threadIdx.x;
    const int srx = a.srx, sry = a.sry, nx = a.nx, ny = a.ny, nxa = a.nxa, nya = a.nya;
    const int W = a.kx * srx, L = a.ky * sry;
    const int x0 = blockIdx.x * W, y0 = blockIdx.y * L;
    const int Wa = min(W, nx - x0), La = min(L, ny - y0);
    const int x = x0 - kMarchHalo + c;
    const bool xin = x >= 0 && x < nx;
    const bool c_load = xin && c >= 1 && c < Wa + 7;
    const bool c_s1 = xin && c >= 2 && c < Wa + 6;
    const bool c_s2 = xin && c >= 3 && c < Wa + 5;
    const bool c_out = c >= 4 && c < Wa + 4;

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
    double *__restrict__ tign = a.tign;

    const T dt = T(a.dt);
    const T idx = T(1) / T(a.dx), idy = T(1) / T(a.dy);
    const T i2dx = T(1) / (T(2) * T(a.dx)), i2dy = T(1) / (T(2) * T(a.dy));
    const T eps = T(a.eps);
    const double tstart = *a.t_in;
    const double t1 = tstart + a.dt;
    const int ncm1 = a.ncls - 1;
    const int band = a.band;

    // ---- set-up: coefficient table, row weights, this column's wind weights
    if (c == 0) {
        s_status = 0;
        if (blockIdx.x == 0 && blockIdx.y == 0) *a.t_out = t1;
    }
    for (int k = c; k < a.ncls * K_N; k += NT) lut[k] = T(a.coef[k]);
    for (int i = c; i < La + 4; i += NT) {
        const int r = y0 - 2 + i;
        RowWeights<T> w;
        w.ju0 = w.ju1 = w.jv0 = w.jv1 = 0;
        w.wyu = w.wyv = T(0);
        if (r >= 0 && r < ny) {
            const T ya = (T(r) + T(0.5)) / T(sry);
            lin_idx<T>(ya - T(0.5), nya, w.ju0, w.ju1, w.wyu);
            lin_idx<T>(ya, nya + 1, w.jv0, w.jv1, w.wyv);
        }
        rw[i] = w;
    }
    int iu0 = 0, iu1 = 0, iv0 = 0, iv1 = 0;
    T wxu = T(0), wxv = T(0);
    if (xin) {
        const T xa = (T(x) + T(0.5)) / T(srx);
        lin_idx<T>(xa, nxa + 1, iu0, iu1, wxu);
        lin_idx<T>(xa - T(0.5), nxa, iv0, iv1, wxv);
    }
    __syncthreads();

    // wind at (x, r), same formula as the bilinear interpolation of wind_at
    auto wind = [&](int r, T &un, T &vn) {
        const RowWeights<T> &w = rw[r - (y0 - 2)];
        const T *u0 = wu + (size_t)w.ju0 * (nxa + 1), *u1 = wu + (size_t)w.ju1 * (nxa + 1);
        un = (T(1) - w.wyu) * ((T(1) - wxu) * __ldg(u0 + iu0) + wxu * __ldg(u0 + iu1)) +
             w.wyu * ((T(1) - wxu) * __ldg(u1 + iu0) + wxu * __ldg(u1 + iu1));
        const T *v0 = wv + (size_t)w.jv0 * nxa, *v1 = wv + (size_t)w.jv1 * nxa;
        vn = (T(1) - w.wyv) * ((T(1) - wxv) * __ldg(v0 + iv0) + wxv * __ldg(v0 + iv1)) +
             w.wyv * ((T(1) - wxv) * __ldg(v1 + iv0) + wxv * __ldg(v1 + iv1));
    };

    const int k0 = y0 - 7, k1 = y0 + La;  // iterations: rows k0+4 .. k1-1
    const int a_lo = y0 - 3, a_hi = y0 + La + 3;  // psi^n rows staged
    auto load_psi = [&](int r) -> T {
        return (c_load && r >= 0 && r < ny && r >= a_lo && r < a_hi) ? psi_in[(size_t)r * nx + x]
                                                                      : T(0);
    };
    // prefetched values for the next iteration
    T pf_psi = load_psi(k0 + 4);
    int pf_cls = 0;
    T pf_zx = T(0), pf_zy = T(0), pf_m = T(1);
    auto load_env = [&](int r, int &cls, T &zx, T &zy, T &m) {
        if (c_s1 && r >= 0 && r < ny && r >= y0 - 2 && r < y0 + La + 2) {
            const size_t g = (size_t)r * nx + x;
            cls = fuel[g];
            zx = dzdx[g];
            zy = dzdy[g];
            m = mult ? mult[g] : T(1);
        }
    };
    load_env(k0 + 3, pf_cls, pf_zx, pf_zy, pf_m);
    T pf_F = T(0);
    T acc_s = T(0), acc_q = T(0);
    int st = 0;

    for (int k = k0; k <= k1; ++k) {
        // ---- A: stage psi^n of row k+4; prefetch row k+5
        {
            const int r = k + 4;
            if (r >= a_lo && r < a_hi) S0[r & 3][c] = pf_psi;
            pf_psi = load_psi(k + 5);
        }
        // ---- B: stage 1 on row k+3
        {
            const int r = k + 3;
            const int cls0 = pf_cls;
            const T zx = pf_zx, zy = pf_zy, m = pf_m;
            load_env(k + 4, pf_cls, pf_zx, pf_zy, pf_m);
            if (c_s1 && r >= y0 - 2 && r < y0 + La + 2 && r >= 0 && r < ny) {
                const T *R = S0[r & 3];
                const T p = R[c], pl0 = R[c - 1], pr0 = R[c + 1];
                const T pd0 = S0[(r - 1) & 3][c], pu0 = S0[(r + 1) & 3][c];
                const T pl = x > 0 ? pl0 : ghost_value<T>(p, pr0);
                const T pr = x < nx - 1 ? pr0 : ghost_value<T>(p, pl0);
                const T pd = r > 0 ? pd0 : ghost_value<T>(p, pu0);
                const T pu = r < ny - 1 ? pu0 : ghost_value<T>(p, pd0);
                T un, vn;
                wind(r, un, vn);
                if (!isfinite(un) || !isfinite(vn)) st |= ST_NONFINITE;
                const int cls = cls0 > ncm1 ? ncm1 : cls0;
                const T F = rhs_vals<T>(p, pl, pr, pd, pu, idx, idy, i2dx, i2dy, eps,
                                        lut + cls * K_N, m, un, vn, zx, zy);
                S1[r & 3][c] = p + dt * F;
                SF[r & 3][c] = F;
            }
        }
        // ---- C: stage 2, crossing and t - t_i on row k+1
        {
            const int r = k + 1;
            if (c_s2 && r >= y0 - 1 && r < y0 + La + 1 && r >= 0 && r < ny) {
                const size_t g = (size_t)r * nx + x;
                const T *R = S1[r & 3];
                const T q = R[c], ql0 = R[c - 1], qr0 = R[c + 1];
                const T qd0 = S1[(r - 1) & 3][c], qu0 = S1[(r + 1) & 3][c];
                const T ql = x > 0 ? ql0 : ghost_value<T>(q, qr0);
                const T qr = x < nx - 1 ? qr0 : ghost_value<T>(q, ql0);
                const T qd = r > 0 ? qd0 : ghost_value<T>(q, qu0);
                const T qu = r < ny - 1 ? qu0 : ghost_value<T>(q, qd0);
                int cls = fuel[g];
                cls = cls > ncm1 ? ncm1 : cls;
                const T m = mult ? mult[g] : T(1);
                T un, vn;
                wind(r, un, vn);
                const T F2 = rhs_vals<T>(q, ql, qr, qd, qu, idx, idy, i2dx, i2dy, eps,
                                         lut + cls * K_N, m, un, vn, dzdx[g], dzdy[g]);
                const T p0 = S0[r & 3][c];
                const T pn = p0 + dt * (T(0.5) * SF[r & 3][c] + T(0.5) * F2);
                const bool own = c_out && r >= y0 && r < y0 + La;
                T d = T(0);
                const bool cross = p0 > T(0) && pn <= T(0);
                if (cross || pn < T(0)) {
                    double ti = tign[g];
                    if (cross && isinf(ti)) {
                        const double q0 = (double)p0, q1 = (double)pn;
                        ti = tstart + q0 * a.dt / (q0 - q1);
                        if (own) tign[g] = ti;
                    }
                    if (pn < T(0)) d = T(t1 - ti);
                }
                SQ[r & 3][c] = pn;
                SD[r & 3][c] = d;
                if (own) {
                    psi_out[g] = pn;
                    if (!isfinite(pn)) st |= ST_NONFINITE;
                    const bool edge = x < band || r < band || x >= nx - band || r >= ny - band;
                    if (edge && pn < T(0)) st |= ST_BOUNDARY;
                }
            }
        }
        // ---- D: fuel fraction and heat on row k-1
        const int rd = k - 1;
        const bool drow = rd >= y0 && rd < y0 + La;
        if (drow && c_out) {
            T p[3][3], d[3][3];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int s = (rd + b - 1) & 3;
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    p[b][e] = SQ[s][c + e - 1];
                    d[b][e] = SD[s][c + e - 1];
                }
            }
            if (x == 0 || x == nx - 1 || rd == 0 || rd == ny - 1) {
                // ghost ring of psi^{n+1} (x first, then y) and of t - t_i
                // (inner neighbour's value, 0 where the ghost psi >= 0)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int yy = rd + b - 1;
                    if (yy < 0 || yy >= ny) continue;
                    if (x == 0) {
                        p[b][0] = ghost_value<T>(p[b][1], p[b][2]);
                        d[b][0] = p[b][0] >= T(0) ? T(0) : d[b][1];
                    }
                    if (x == nx - 1) {
                        p[b][2] = ghost_value<T>(p[b][1], p[b][0]);
                        d[b][2] = p[b][2] >= T(0) ? T(0) : d[b][1];
                    }
                }
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    if (rd == 0) {
                        p[0][e] = ghost_value<T>(p[1][e], p[2][e]);
                        d[0][e] = p[0][e] >= T(0) ? T(0) : d[1][e];
                    }
                    if (rd == ny - 1) {
                        p[2][e] = ghost_value<T>(p[1][e], p[0][e]);
                        d[2][e] = p[2][e] >= T(0) ? T(0) : d[1][e];
                    }
                }
            }
            const size_t g = (size_t)rd * nx + x;
            int cls = fuel[g];
            cls = cls > ncm1 ? ncm1 : cls;
            const T *co = lut + cls * K_N;
            const T Fn = cell_fraction_vals<T>(p[0][0], p[0][1], p[0][2], p[1][0], p[1][1], p[1][2],
                                               p[2][0], p[2][1], p[2][2], d[0][0], d[0][1], d[0][2],
                                               d[1][0], d[1][1], d[1][2], d[2][0], d[2][1], d[2][2],
                                               co[K_TF]);
            F_out[g] = Fn;
            const T dF = pf_F - Fn;
            acc_s += dF * co[K_HS];
            acc_q += dF * co[K_HQ];
        }
        // prefetch F^n of row k for the next iteration's quadrature
        pf_F = (c_out && k >= y0 && k < y0 + La) ? F_in[(size_t)k * nx + x] : T(0);
        const bool band_end = drow && ((rd - y0 + 1) % sry == 0);
        const int par = ((rd - y0) / sry) & 1;
        if (band_end) {
            HB[par][0][c] = acc_s;
            HB[par][1][c] = acc_q;
            acc_s = T(0);
            acc_q = T(0);
        }
        __syncthreads();
        // ---- average of the band's atmospheric cells (after its last row)
        if (band_end) {
            const int kxa = Wa / srx;
            if (c < kxa) {
                double h0 = 0.0, h1 = 0.0;
                for (int e = 0; e < srx; ++e) {
                    const T v0 = HB[par][0][kMarchHalo + c * srx + e];
                    const T v1 = HB[par][1][kMarchHalo + c * srx + e];
                    if (v0 != T(0)) h0 += (double)v0;
                    if (v1 != T(0)) h1 += (double)v1;
                }
                const double scale = 1.0 / (a.dt * (double)srx * (double)sry);
                const size_t ga = (size_t)(rd / sry) * nxa + (x0 / srx + c);
                if (a.heat_s) a.heat_s[ga] = h0 * scale;
                if (a.heat_l) a.heat_l[ga] = h1 * scale;
            }
        }
    }
    if (st) atomicOr(&s_status, st);
    __syncthreads();
    if (c == 0 && s_status) atomicOr(a.status, s_status);
}

template <typename T>
size_t march_smem_bytes(int ky, int sry) {
    return (size_t)(ky * sry + 4) * sizeof(RowWeights<T>);
}

template <typename T>
cudaError_t launch_march(const StepArgs &a, cudaStream_t s) {
    const int W = a.kx * a.srx, L = a.ky * a.sry;
    dim3 grid((a.nx + W - 1) / W, (a.ny + L - 1) / L);
    k_fire_march<T><<<grid, kMarchThreads, march_smem_bytes<T>(a.ky, a.sry), s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t prepare_march_kernel(size_t smem_bytes) {
    return cudaFuncSetAttribute(k_fire_march<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

#define WF_INSTANTIATE_MARCH(T)                                               \
    template size_t march_smem_bytes<T>(int, int);                            \
    template cudaError_t launch_march<T>(const StepArgs &, cudaStream_t);     \
    template cudaError_t prepare_march_kernel<T>(size_t);

}  // namespace wf
