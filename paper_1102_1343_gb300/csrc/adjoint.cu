// fire_adjoint: gradient of the arrival-time misfit
//   J = 1/2 sum over nodes ignited in both runs of (t_i - t_obs)^2
// (fire_adjoint_heat: of the heat misfit, see the HeatArgs section below,
// whose seeds enter the same reverse sweep)
// with respect to the per-node spread multiplier, the per-node fuel moisture
// and the staggered wind, by a reverse sweep through the Heun stages
// (eq. Heun), the upwinded right-hand side (eqs. F-disc, Godunov,
// spread-WRF-Fire) and the ignition-time interpolation
// (eq. set-ignition-time).  The paper motivates the level-set formulation by
// data assimilation (Sect. 7); the adjoint is what variational assimilation
// needs.
//
// Forward: the context advances nsteps steps with the step kernel it uses
// for fire_step, saving psi every K steps (checkpoints; with K = 1 every
// state is kept and nothing is recomputed).  Reverse: for each K-step
// segment, last first, the states psi^s of the segment are recomputed from
// its checkpoint with the same step kernel (bitwise the same values, hence
// the same branches), then each step is reversed:
//   mu      = lambda + dJ/dpsi^{s+1}   (nodes whose t_i was set in step s)
//   psi*    = psi^s + dt F(psi^s)
//   lam*    = J_F(psi*)^T (dt/2 mu)
//   w       = dt/2 mu + dt lam*
//   lambda  = mu + lam* + J_F(psi^s)^T w + dJ/dpsi^s (same nodes)
// with the parameter terms v^T dF/dp of both products summed per node.
// Branches (Godunov selection, max/min of the spread rate, the
// extrapolated ghosts, zeroed central differences) are those the forward
// values take.  A reverse step is one launch of tiles that form the whole
// chain above for their nodes in shared memory (k_adj_step); each product
// J^T v is formed without atomics, every node's five stencil contributions
// v_j dF_j/dpsi_k written first and then gathered per node k in a fixed
// order, so results do not depend on scheduling.
//
// Precision: the state, the partial derivatives, the adjoint fields and the
// stencil contributions are in the path precision T (FP32 or FP64); the
// arrival-time seeds are double, and the parameter gradients, summed over
// the whole run, are double in FP64 and compensated float pairs in FP32
// (double at the end), so the FP32 reverse step uses the FP64 pipe (a small
// fraction of the FP32 rate on this part) only at the nodes that cross.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "fire_device.cuh"
#include "fire_internal.h"

namespace wf {

int ctx_step_args(fire_ctx *c, int parity, const void *u, const void *v, double dt, double *hs,
                  double *hl, StepArgs &a);
int ctx_info(const fire_ctx *c, int *prec, int *variant, int *nx, int *ny, int *srx, int *sry,
             int *kx, int *ky, int *ncls, int *cur, double *t);
int ctx_advance(fire_ctx *c, int nsteps, double dt);
bool ctx_ignition_active(fire_ctx *c, double t);
cudaStream_t ctx_stream(const fire_ctx *c);
const fire_fuel_class *ctx_classes_dev(const fire_ctx *c);
const void *ctx_moisture(const fire_ctx *c);
int ctx_scheme(const fire_ctx *c);
int ctx_workspace(fire_ctx *c, size_t bytes, void **out);
cudaGraphExec_t *ctx_adjoint_graphs(fire_ctx *c, unsigned long long **keys);

namespace {

constexpr int kAdjThreads = 256;

// A sum over the run's steps of per-step contributions in T: FP64 adds in
// place; FP32 keeps a compensated pair (Kahan summation: the sum is s - c),
// so that the sum of 10^2..10^4 steps stays at FP32 rounding without an FP64
// instruction in the reverse step (the FP64 pipe of this part issues at a
// small fraction of the FP32 rate).
template <typename T>
struct GAcc;
template <>
struct GAcc<double> {
    using t = double;
    static __device__ __forceinline__ void add(double &g, double x) { g += x; }
};
template <>
struct GAcc<float> {
    using t = float2;  // (s, c)
    static __device__ __forceinline__ void add(float2 &g, float x) {
        const float y = x - g.y;
        const float t = g.x + y;
        g.y = (t - g.x) - y;
        g.x = t;
    }
};

template <typename T>
struct AdjArgs {
    const T *pa, *pb;  // psi^s, psi^{s+1}
    // the unfused reverse step (FP64): the field of the current Jacobian
    // product, psi*, mu, lam*, and the stencil contributions [5][n] that a
    // kernel writes (Cout) and the next gathers (Cin)
    const T *X;
    T *pstar, *mu, *ls;
    const T *Cin;
    T *Cout;
    const uint8_t *fuel;
    const T *zx, *zy, *mult;  // mult nullable (1)
    const T *u, *v;
    const T *unv;  // [n][2] node wind of the run (interpolated once), or null
    const double *coef, *dcoef;  // [ncls][K_N], or [n][K_N] per node when nodeco
    int ncls;
    int nodeco;  // coefficients per node (a per-node fuel moisture)
    const double *tign0, *tign, *tobs;
    const double *dJdt;  // dJ/dt_i per node instead of t_i - t_obs (heat misfit), or null
    const double *tsp;  // [2] start and end time of the step (device)
    double dt;
    const T *lin;  // lambda^{s+1}
    T *lout;       // lambda^s
    // parameter gradients summed over the run, [4][n]: multiplier, moisture,
    // node wind u, v (GAcc<T>::t each; the wind pair only with wind_grads)
    typename GAcc<T>::t *acc;
    int wind_grads;
    int nx, ny, nxa, nya, srx, sry;
    T idx, idy, i2dx, i2dy, eps, dtT, hdtT;  // dtT = dt, hdtT = dt/2 in T
    size_t n;
};

// stencil slots: centre, left, right, down, up
enum { P_C = 0, P_L, P_R, P_D, P_U };

// d(ghost)/d(p0), d(ghost)/d(p1) for the branch ghost_value takes
template <typename T>
__device__ __forceinline__ void ghost_partials(T p0, T p1, T &d0, T &d1) {
    const T g = p0 + (p0 - p1);
    d0 = T(2);
    d1 = T(-1);
    T h = g;
    if (p0 > h) {
        h = p0;
        d0 = T(1);
        d1 = T(0);
    }
    if (p1 > h) {
        d0 = T(0);
        d1 = T(1);
    }
}

template <typename T>
struct NodeEnv {
    T co[6];   // S0, R0, b, c, d, e
    T dco[4];  // d/dM_f of S0, R0, c, d
    T m, un, vn, zx, zy;
};

// the coefficients of node k (from the class table lut, [ncls][10] in T:
// the six coefficients, then d/dM_f of S0, R0, c, d; from the double tables
// when lut is null or the coefficients are per node), its multiplier, slope
// and node wind
template <typename T>
__device__ __forceinline__ void node_env(const AdjArgs<T> &a, const T *lut, size_t k, bool want_d,
                                         NodeEnv<T> &e) {
    if (a.nodeco || !lut) {
        size_t row = k;
        if (!a.nodeco) {
            const int cls = a.fuel[k];
            row = (size_t)(cls > a.ncls - 1 ? a.ncls - 1 : cls);
        }
        const double *co = a.coef + row * K_N;
#pragma unroll
        for (int q = 0; q < 6; ++q) e.co[q] = T(co[q]);
        if (want_d) {
            const double *dc = a.dcoef + row * K_N;
            e.dco[0] = T(dc[K_S0]);
            e.dco[1] = T(dc[K_R0]);
            e.dco[2] = T(dc[K_C]);
            e.dco[3] = T(dc[K_D]);
        }
    } else {
        int cls = a.fuel[k];
        cls = cls > a.ncls - 1 ? a.ncls - 1 : cls;
        const T *l = lut + cls * 10;
#pragma unroll
        for (int q = 0; q < 6; ++q) e.co[q] = l[q];
        if (want_d) {
#pragma unroll
            for (int q = 0; q < 4; ++q) e.dco[q] = l[6 + q];
        }
    }
    e.m = a.mult ? a.mult[k] : T(1);
    e.zx = a.zx[k];
    e.zy = a.zy[k];
    e.un = a.unv[2 * k];
    e.vn = a.unv[2 * k + 1];
}

// Partial derivatives of the right-hand side of eq. (F-disc) at one node,
// F = -S |grad psi| + eps S Lap psi with S = m max{S0, R0 + c Ue^b + d tp^2},
// with respect to the five stencil values and to m, S0, R0, c, d and the
// node wind, along the branches the values take (the forward arithmetic of
// rhs_vals, differentiated).
template <typename T>
struct Partials {
    T dpsi[5];
    T dm, dS0, dR0, dc, dd, dun, dvn;
};

template <typename T>
__device__ __forceinline__ void node_partials(T p, T pl, T pr, T pd, T pu, T idx, T idy, T i2dx,
                                              T i2dy, T eps, const NodeEnv<T> &e,
                                              Partials<T> &o) {
    const T dxm = (p - pl) * idx, dxp = (pr - p) * idx;
    const T dym = (p - pd) * idy, dyp = (pu - p) * idy;
    const T ax = dxm > T(0) ? dxm : T(0), bx = dxp < T(0) ? dxp : T(0);
    const T ay = dym > T(0) ? dym : T(0), by = dyp < T(0) ? dyp : T(0);
    const bool xm = ax * ax > bx * bx;  // D- taken along x (else D+)
    const bool ym = ay * ay > by * by;
    const T gx = xm ? ax : bx, gy = ym ? ay : by;
    const T grad = Mth<T>::sqr(gx * gx + gy * gy);
    // central differences, zeroed at the rounding level as in the forward
    T ddx = pr - pl, ddy = pu - pd;
    const bool kx = !(abs_val(ddx) <= Mth<T>::kGradZero * (abs_val(pr) + abs_val(pl)));
    const bool ky = !(abs_val(ddy) <= Mth<T>::kGradZero * (abs_val(pu) + abs_val(pd)));
    ddx = kx ? ddx : T(0);
    ddy = ky ? ddy : T(0);
    const T cx = ddx * i2dx, cy = ddy * i2dy;
    T nxv, nyv;
    Mth<T>::unit(cx, cy, nxv, nyv);
    const T cn2 = cx * cx + cy * cy;
    const T U = e.un * nxv + e.vn * nyv;
    const T tp = e.zx * nxv + e.zy * nyv;
    // spread rate and its branches
    const T Up = U > T(0) ? U : T(0);
    const T Ue = Up < e.co[K_E] ? Up : e.co[K_E];
    const T tpp = tp > T(0) ? tp : T(0);
    const T pwv = Mth<T>::pw(Ue, e.co[K_B]);
    const T inner = e.co[K_R0] + e.co[K_C] * pwv + e.co[K_D] * tpp * tpp;
    const bool active = inner > e.co[K_S0];
    const T St = active ? inner : e.co[K_S0];
    const T S = e.m * St;
    const T lap = (dxp - dxm) + (dyp - dym);
    const T Fs = -grad + eps * lap;  // dF/dS
    const T dSt_dU =
        (active && U > T(0) && U < e.co[K_E]) ? Mth<T>::dv(e.co[K_C] * e.co[K_B] * pwv, Ue) : T(0);
    const T dSt_dT = (active && tp > T(0)) ? T(2) * e.co[K_D] * tp : T(0);
    // the unit normal n = c/|c|: dn/dc = (I - n n^T)/|c|
    T dS_dcx = T(0), dS_dcy = T(0);
    if (cn2 > Mth<T>::kNormMin) {
        const T rc = Mth<T>::rsq(cn2);
        const T dU_dcx = (e.un - U * nxv) * rc, dU_dcy = (e.vn - U * nyv) * rc;
        const T dT_dcx = (e.zx - tp * nxv) * rc, dT_dcy = (e.zy - tp * nyv) * rc;
        dS_dcx = e.m * (dSt_dU * dU_dcx + dSt_dT * dT_dcx);
        dS_dcy = e.m * (dSt_dU * dU_dcy + dSt_dT * dT_dcy);
    }
    const T dcx = kx ? i2dx : T(0), dcy = ky ? i2dy : T(0);
    // d|grad|/d(one-sided differences) through the taken branch
    T wx = T(0), wy = T(0);
    if (grad > T(0)) {
        const T rg = Mth<T>::dv(T(1), grad);
        wx = gx * rg;
        wy = gy * rg;
    }
    T dG[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (xm) {
        dG[P_C] += wx * idx;
        dG[P_L] -= wx * idx;
    } else {
        dG[P_R] += wx * idx;
        dG[P_C] -= wx * idx;
    }
    if (ym) {
        dG[P_C] += wy * idy;
        dG[P_D] -= wy * idy;
    } else {
        dG[P_U] += wy * idy;
        dG[P_C] -= wy * idy;
    }
    const T dL[5] = {-T(2) * idx - T(2) * idy, idx, idx, idy, idy};
    const T dS[5] = {T(0), -dS_dcx * dcx, dS_dcx * dcx, -dS_dcy * dcy, dS_dcy * dcy};
#pragma unroll
    for (int q = 0; q < 5; ++q) o.dpsi[q] = Fs * dS[q] - S * dG[q] + eps * S * dL[q];
    const T fm = Fs * e.m;
    o.dm = Fs * St;
    o.dS0 = active ? T(0) : fm;
    o.dR0 = active ? fm : T(0);
    o.dc = active ? fm * pwv : T(0);
    o.dd = active ? fm * tpp * tpp : T(0);
    o.dun = fm * dSt_dU * nxv;
    o.dvn = fm * dSt_dU * nyv;
}

// whether node k's ignition time was set in step s (the forward test of
// eq. set-ignition-time: first crossing from > 0 to <= 0, the recorded time
// inside the step) and the node is observed
// (the tests that every node takes are on the bits and in T; only crossing
// nodes compare times in double)
__device__ __forceinline__ bool inf_bits(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) == 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
template <typename T>
__device__ __forceinline__ bool crossed(const AdjArgs<T> &a, size_t k, double &q0, double &q1,
                                        double &r) {
    const double t0 = a.tign0[k], ti = a.tign[k], to = a.dJdt ? a.dJdt[k] : a.tobs[k];
    if (!inf_bits(t0) || !finite_bits(ti) || !finite_bits(to)) return false;
    const T p0 = a.pa[k], p1 = a.pb[k];
    if (!(p0 > T(0) && p1 <= T(0))) return false;
    if (!(ti >= a.tsp[0] && ti <= a.tsp[1])) return false;
    q0 = (double)p0;
    q1 = (double)p1;
    r = a.dJdt ? to : ti - to;
    return true;
}

// the node wind of the run (the wind is held constant over it), once
template <typename T>
__global__ void k_adj_node_wind(const AdjArgs<T> a, T *unv) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < a.n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % a.nx), j = (int)(k / a.nx);
        T un, vn;
        int st = 0;  // indices are in range by construction; the step kernels report them
        wind_at<T>(a.u, a.v, a.nxa, a.nya, a.srx, a.sry, i, j, un, vn, st);
        unv[2 * k] = un;
        unv[2 * k + 1] = vn;
    }
}

// ---------------------------------------------------------------------------
// The reverse step of FP64 in four grid-wide kernels: no node's work is
// repeated (FP64 arithmetic bounds the step on this part).
// ---------------------------------------------------------------------------

// the five stencil values of node (i, j) of field X with the extrapolated
// ghosts of Sect. 3.1 at the domain boundary (nx, ny >= 2)
template <typename T>
__device__ __forceinline__ void stencil(const T *X, int nx, int ny, int i, int j, T &p, T &pl,
                                        T &pr, T &pd, T &pu) {
    const size_t k = (size_t)j * nx + i;
    p = X[k];
    pl = i > 0 ? X[k - 1] : ghost_value<T>(p, X[k + 1]);
    pr = i < nx - 1 ? X[k + 1] : ghost_value<T>(p, X[k - 1]);
    pd = j > 0 ? X[k - nx] : ghost_value<T>(p, X[k + nx]);
    pu = j < ny - 1 ? X[k + nx] : ghost_value<T>(p, X[k - nx]);
}

// seeds mu = lambda + dJ/dpsi^{s+1} and forms psi* = psi^s + dt F(psi^s)
template <typename T>
__global__ void k_adj_stage1(const AdjArgs<T> a) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < a.n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % a.nx), j = (int)(k / a.nx);
        T mu = a.lin[k];
        double q0, q1, r;
        if (crossed(a, k, q0, q1, r)) {
            const double den = q0 - q1;
            mu = T((double)mu + r * a.dt * q0 / (den * den));
        }
        a.mu[k] = mu;
        NodeEnv<T> e;
        node_env<T>(a, nullptr, k, false, e);
        T p, pl, pr, pd, pu;
        stencil(a.pa, a.nx, a.ny, i, j, p, pl, pr, pd, pu);
        const T F = rhs_vals<T>(p, pl, pr, pd, pu, a.idx, a.idy, a.i2dx, a.i2dy, a.eps, e.co,
                                e.m, e.un, e.vn, e.zx, e.zy);
        a.pstar[k] = p + a.dtT * F;
    }
}

// v^T dF/dp at node k added to the parameter sums, and the node's five
// stencil contributions v dF/dpsi written to Cout
template <typename T>
__device__ __forceinline__ void vjp_node(const AdjArgs<T> &a, size_t k, int i, int j, T v) {
    NodeEnv<T> e;
    node_env<T>(a, nullptr, k, true, e);
    T p, pl, pr, pd, pu;
    stencil(a.X, a.nx, a.ny, i, j, p, pl, pr, pd, pu);
    Partials<T> o;
    node_partials<T>(p, pl, pr, pd, pu, a.idx, a.idy, a.i2dx, a.i2dy, a.eps, e, o);
#pragma unroll
    for (int q = 0; q < 5; ++q) a.Cout[q * a.n + k] = v * o.dpsi[q];
    const T g[4] = {v * o.dm,
                    v * (o.dS0 * e.dco[0] + o.dR0 * e.dco[1] + o.dc * e.dco[2] + o.dd * e.dco[3]),
                    v * o.dun, v * o.dvn};
    const int nq = a.wind_grads ? 4 : 2;
    for (int q = 0; q < nq; ++q) GAcc<T>::add(a.acc[q * a.n + k], g[q]);
}

// (J_X^T v)_k: the contributions of the stencils that contain node k, with
// the extrapolated ghosts of the boundary rows and columns mapped back to
// the two nodes each was extrapolated from
template <typename T>
__device__ __forceinline__ T gather(const AdjArgs<T> &a, const T *C, const T *X, int i, int j) {
    const int nx = a.nx, ny = a.ny;
    const size_t n = a.n, k = (size_t)j * nx + i;
    T r = C[P_C * n + k];
    if (i > 0) r += C[P_R * n + k - 1];
    if (i < nx - 1) r += C[P_L * n + k + 1];
    if (j > 0) r += C[P_U * n + k - nx];
    if (j < ny - 1) r += C[P_D * n + k + nx];
    T d0, d1;
    const size_t row = (size_t)j * nx, col = (size_t)i;
    if (i <= 1) {  // left ghost of row j = ghost(X[j][0], X[j][1])
        ghost_partials<T>(X[row], X[row + 1], d0, d1);
        r += C[P_L * n + row] * (i == 0 ? d0 : d1);
    }
    if (i >= nx - 2) {  // right ghost = ghost(X[j][nx-1], X[j][nx-2])
        ghost_partials<T>(X[row + nx - 1], X[row + nx - 2], d0, d1);
        r += C[P_R * n + row + nx - 1] * (i == nx - 1 ? d0 : d1);
    }
    if (j <= 1) {  // bottom ghost of column i = ghost(X[0][i], X[1][i])
        ghost_partials<T>(X[col], X[col + nx], d0, d1);
        r += C[P_D * n + col] * (j == 0 ? d0 : d1);
    }
    if (j >= ny - 2) {  // top ghost = ghost(X[ny-1][i], X[ny-2][i])
        const size_t top = (size_t)(ny - 1) * nx + col;
        ghost_partials<T>(X[top], X[top - nx], d0, d1);
        r += C[P_U * n + top] * (j == ny - 1 ? d0 : d1);
    }
    return r;
}

// first product, at psi*: v = dt/2 mu
template <typename T>
__global__ void k_adj_vjp_star(const AdjArgs<T> a) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < a.n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % a.nx), j = (int)(k / a.nx);
        vjp_node(a, k, i, j, a.hdtT * a.mu[k]);
    }
}

// lam* = gather of the first product; second product at psi^s with
// w = dt/2 mu + dt lam*
template <typename T>
__global__ void k_adj_vjp_n(AdjArgs<T> a) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < a.n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % a.nx), j = (int)(k / a.nx);
        const T ls = gather(a, a.Cin, a.pstar, i, j);
        a.ls[k] = ls;
        vjp_node(a, k, i, j, a.hdtT * a.mu[k] + a.dtT * ls);
    }
}

// lambda = mu + lam* + J_F(psi^s)^T w + dJ/dpsi^s
template <typename T>
__global__ void k_adj_finish(const AdjArgs<T> a) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < a.n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % a.nx), j = (int)(k / a.nx);
        T lam = a.mu[k] + a.ls[k] + gather(a, a.Cin, a.pa, i, j);
        double q0, q1, r;
        if (crossed(a, k, q0, q1, r)) {
            const double den = q0 - q1;
            lam = T((double)lam + r * (-a.dt * q1 / (den * den)));
        }
        a.lout[k] = lam;
    }
}

// ---------------------------------------------------------------------------
// The reverse step of FP32 in one launch (memory latency and launch gaps,
// not arithmetic, bound the unfused FP32 step).  A CTA owns a tile of
// kRevTX x kRevTY nodes and forms in shared memory what its nodes'
// lambda^s needs, each field in a frame of the tile with the halo radius
// that field needs:
//   psi^s            radius 4  (read)
//   node inputs      radius 3  class, multiplier, slope, node wind (read)
//   mu               radius 2  lambda^{s+1} + the seed of crossing nodes
//   psi*             radius 3  psi^s + dt F(psi^s)
//   C* = v dF/dpsi   radius 2  at psi*, v = dt/2 mu, five stencil slots
//   lam*             radius 1  gather of C*
//   C  = w dF/dpsi   radius 1  at psi^s, w = dt/2 mu + dt lam*
//   lambda^s         the tile  mu + lam* + gather of C + the seed
// (a gather at a node reads contributions and psi within one node, the
// boundary ghosts included).  All reads from global memory happen in the
// first stage, in unrolled loops that load into registers before they
// store, so that the loads are in flight together.  Halo values are
// recomputed by every CTA that needs them with the same arithmetic, so a
// node's value does not depend on the tile that forms it; each node's
// parameter terms are added once, by its owner, the product at psi* first.
// lambda^{s+1} and lambda^s are separate fields (CTAs read their
// neighbours' lambda^{s+1}).
// ---------------------------------------------------------------------------
constexpr int kRevTX = 32, kRevTY = 16, kRevThreads = 256;
constexpr int kRevO = kRevTX * kRevTY;  // the tile
constexpr int rev_w(int h) { return kRevTX + 2 * h; }
constexpr int rev_rsize(int h) { return (kRevTX + 2 * h) * (kRevTY + 2 * h); }
constexpr int rev_iters(int h) { return (rev_rsize(h) + kRevThreads - 1) / kRevThreads; }

// shared memory: the seeds of the tile (double); fields of T: psi^s (radius
// 4), psi* and the multiplier, slope x, y, node wind u, v (radius 3), mu and
// the five contribution slots (radius 2), lam* (radius 1), the terms at psi*
// [4][tile], the class table [ncls][10]; the classes (bytes, radius 3)
template <typename T>
size_t rev_smem_bytes(int ncls) {
    const size_t nT = (size_t)rev_rsize(4) + 6 * rev_rsize(3) + 6 * rev_rsize(2) + rev_rsize(1) +
                      4 * kRevO + (size_t)ncls * 10;
    return sizeof(double) * kRevO + sizeof(T) * nT + rev_rsize(3);
}

// the five stencil values of frame position l (frame row width W, global
// node (x, y)) with the extrapolated ghosts of Sect. 3.1 at the domain
// boundary (nx, ny >= 2)
template <typename T>
__device__ __forceinline__ void rev_stencil(const T *X, int l, int W, int x, int y, int nx, int ny,
                                            T &p, T &pl, T &pr, T &pd, T &pu) {
    p = X[l];
    pl = x > 0 ? X[l - 1] : ghost_value<T>(p, X[l + 1]);
    pr = x < nx - 1 ? X[l + 1] : ghost_value<T>(p, X[l - 1]);
    pd = y > 0 ? X[l - W] : ghost_value<T>(p, X[l + W]);
    pu = y < ny - 1 ? X[l + W] : ghost_value<T>(p, X[l - W]);
}

// gather() above on the frames: contributions C at lc (slots F apart, row
// width Wc), psi X at lx (row width Wx)
template <typename T>
__device__ __forceinline__ T rev_gather(const T *C, int lc, int Wc, int F, const T *X, int lx,
                                        int Wx, int x, int y, int nx, int ny) {
    T r = C[P_C * F + lc];
    if (x > 0) r += C[P_R * F + lc - 1];
    if (x < nx - 1) r += C[P_L * F + lc + 1];
    if (y > 0) r += C[P_U * F + lc - Wc];
    if (y < ny - 1) r += C[P_D * F + lc + Wc];
    T d0, d1;
    if (x <= 1) {  // left ghost of row y = ghost(X[y][0], X[y][1])
        ghost_partials<T>(X[lx - x], X[lx - x + 1], d0, d1);
        r += C[P_L * F + lc - x] * (x == 0 ? d0 : d1);
    }
    if (x >= nx - 2) {  // right ghost = ghost(X[y][nx-1], X[y][nx-2])
        const int o = nx - 1 - x;
        ghost_partials<T>(X[lx + o], X[lx + o - 1], d0, d1);
        r += C[P_R * F + lc + o] * (x == nx - 1 ? d0 : d1);
    }
    if (y <= 1) {  // bottom ghost of column x = ghost(X[0][x], X[1][x])
        ghost_partials<T>(X[lx - y * Wx], X[lx - y * Wx + Wx], d0, d1);
        r += C[P_D * F + lc - y * Wc] * (y == 0 ? d0 : d1);
    }
    if (y >= ny - 2) {  // top ghost = ghost(X[ny-1][x], X[ny-2][x])
        const int o = ny - 1 - y;
        ghost_partials<T>(X[lx + o * Wx], X[lx + o * Wx - Wx], d0, d1);
        r += C[P_U * F + lc + o * Wc] * (y == ny - 1 ? d0 : d1);
    }
    return r;
}

template <typename T>
struct RevSm {
    T *pa, *ps, *mu, *ls, *C, *m, *zx, *zy, *un, *vn, *G, *lut;
    double *seed;
    unsigned char *cls;
};

// node inputs at radius-3 frame position l3 (the coefficients of a per-node
// moisture from global memory)
template <typename T>
__device__ __forceinline__ void rev_env(const AdjArgs<T> &a, const RevSm<T> &sm, int l3, size_t k,
                                        bool want_d, NodeEnv<T> &e) {
    if (a.nodeco) {
        const double *co = a.coef + k * K_N;
#pragma unroll
        for (int q = 0; q < 6; ++q) e.co[q] = T(co[q]);
        if (want_d) {
            const double *dc = a.dcoef + k * K_N;
            e.dco[0] = T(dc[K_S0]);
            e.dco[1] = T(dc[K_R0]);
            e.dco[2] = T(dc[K_C]);
            e.dco[3] = T(dc[K_D]);
        }
    } else {
        const T *c = sm.lut + sm.cls[l3] * 10;
#pragma unroll
        for (int q = 0; q < 6; ++q) e.co[q] = c[q];
        if (want_d) {
#pragma unroll
            for (int q = 0; q < 4; ++q) e.dco[q] = c[6 + q];
        }
    }
    e.m = sm.m[l3];
    e.zx = sm.zx[l3];
    e.zy = sm.zy[l3];
    e.un = sm.un[l3];
    e.vn = sm.vn[l3];
}

// the product v J_F^T at node (x, y) against X (its stencil at lx, row
// width Wx): the five stencil contributions into the radius-2 slots at l2
// and its parameter terms (multiplier, moisture, node wind) into g[4]
template <typename T>
__device__ __forceinline__ void rev_vjp(const AdjArgs<T> &a, const RevSm<T> &sm, const T *X,
                                        int lx, int Wx, int l3, int l2, int x, int y, size_t k,
                                        T v, T g[4]) {
    NodeEnv<T> e;
    rev_env(a, sm, l3, k, true, e);
    T p, pl, pr, pd, pu;
    rev_stencil(X, lx, Wx, x, y, a.nx, a.ny, p, pl, pr, pd, pu);
    Partials<T> o;
    node_partials<T>(p, pl, pr, pd, pu, a.idx, a.idy, a.i2dx, a.i2dy, a.eps, e, o);
#pragma unroll
    for (int q = 0; q < 5; ++q) sm.C[q * rev_rsize(2) + l2] = v * o.dpsi[q];
    g[0] = v * o.dm;
    g[1] = v * (o.dS0 * e.dco[0] + o.dR0 * e.dco[1] + o.dc * e.dco[2] + o.dd * e.dco[3]);
    g[2] = v * o.dun;
    g[3] = v * o.dvn;
}

template <typename T>
__global__ void __launch_bounds__(kRevThreads) k_adj_step(const AdjArgs<T> a) {
    extern __shared__ __align__(16) unsigned char rev_sm[];
    constexpr int F4 = rev_rsize(4), F3 = rev_rsize(3), F2 = rev_rsize(2), F1 = rev_rsize(1);
    constexpr int W4 = rev_w(4), W3 = rev_w(3), W2 = rev_w(2);
    RevSm<T> sm;
    sm.seed = reinterpret_cast<double *>(rev_sm);
    T *f = reinterpret_cast<T *>(sm.seed + kRevO);
    sm.pa = f;
    f += F4;
    sm.ps = f;
    sm.m = f + F3;
    sm.zx = f + 2 * F3;
    sm.zy = f + 3 * F3;
    sm.un = f + 4 * F3;
    sm.vn = f + 5 * F3;
    f += 6 * F3;
    sm.mu = f;
    sm.C = f + F2;
    f += 6 * F2;
    sm.ls = f;
    f += F1;
    sm.G = f;
    f += 4 * kRevO;
    sm.lut = f;
    sm.cls = reinterpret_cast<unsigned char *>(f + a.ncls * 10);
    const int nx = a.nx, ny = a.ny;
    const int x0 = blockIdx.x * kRevTX, y0 = blockIdx.y * kRevTY;
    const int tid = threadIdx.x;
    // frame position of node (x, y) in the frame of radius h
    auto at = [&](int h, int x, int y) { return (y - y0 + h) * rev_w(h) + (x - x0 + h); };
    // a region of radius h around the tile, clipped to the domain: position
    // e -> global (x, y)
    auto region = [&](int h, int e, int &x, int &y) -> bool {
        const int w = rev_w(h);
        x = x0 - h + e % w;
        y = y0 - h + e / w;
        return e < rev_rsize(h) && x >= 0 && x < nx && y >= 0 && y < ny;
    };
    // ---- every read from global memory (each loop loads into registers
    // first and stores to shared memory after)
    if (!a.nodeco) {
        for (int q = tid; q < a.ncls * 10; q += kRevThreads) {
            const int c = q / 10, m = q % 10;
            const int src = m < 6 ? m : (m == 6 ? K_S0 : m == 7 ? K_R0 : m == 8 ? K_C : K_D);
            sm.lut[q] = T((m < 6 ? a.coef : a.dcoef)[(size_t)c * K_N + src]);
        }
    }
    {
        constexpr int I4 = rev_iters(4);
        T v[I4];
        int ls[I4];
#pragma unroll
        for (int it = 0; it < I4; ++it) {
            int x, y;
            ls[it] = -1;
            if (region(4, tid + it * kRevThreads, x, y)) {
                v[it] = a.pa[(size_t)y * nx + x];
                ls[it] = at(4, x, y);
            }
        }
#pragma unroll
        for (int it = 0; it < I4; ++it)
            if (ls[it] >= 0) sm.pa[ls[it]] = v[it];
    }
    {
        constexpr int I3 = rev_iters(3);
        T vm[I3], vx[I3], vy[I3], vu[I3], vv[I3];
        int vc[I3], ls[I3];
#pragma unroll
        for (int it = 0; it < I3; ++it) {
            int x, y;
            ls[it] = -1;
            if (region(3, tid + it * kRevThreads, x, y)) {
                const size_t k = (size_t)y * nx + x;
                vc[it] = a.fuel[k];
                vm[it] = a.mult ? a.mult[k] : T(1);
                vx[it] = a.zx[k];
                vy[it] = a.zy[k];
                vu[it] = a.unv[2 * k];
                vv[it] = a.unv[2 * k + 1];
                ls[it] = at(3, x, y);
            }
        }
#pragma unroll
        for (int it = 0; it < I3; ++it) {
            const int l = ls[it];
            if (l < 0) continue;
            sm.cls[l] = (unsigned char)(vc[it] > a.ncls - 1 ? a.ncls - 1 : vc[it]);
            sm.m[l] = vm[it];
            sm.zx[l] = vx[it];
            sm.zy[l] = vy[it];
            sm.un[l] = vu[it];
            sm.vn[l] = vv[it];
        }
    }
    // mu (radius 2) and the seeds of the tile; the crossing test of a node
    // (crossed(), its reads issued together) needs psi^s, psi^{s+1}, both
    // ignition times and the observation
    auto cross_seed = [&](double t0, double ti, double to, T p0, T p1, double tlo, double thi,
                          double &q0, double &q1, double &rr) -> bool {
        if (!inf_bits(t0) || !finite_bits(ti) || !finite_bits(to)) return false;
        if (!(p0 > T(0) && p1 <= T(0))) return false;
        if (!(ti >= tlo && ti <= thi)) return false;
        q0 = (double)p0;
        q1 = (double)p1;
        rr = a.dJdt ? to : ti - to;
        return true;
    };
    const double *tobs = a.dJdt ? a.dJdt : a.tobs;
    {
        constexpr int I2 = rev_iters(2);
        T vl[I2], p0[I2], p1[I2];
        double t0[I2], ti[I2], to[I2];
        int ls[I2];
#pragma unroll
        for (int it = 0; it < I2; ++it) {
            int x, y;
            ls[it] = -1;
            if (region(2, tid + it * kRevThreads, x, y)) {
                const size_t k = (size_t)y * nx + x;
                vl[it] = a.lin[k];
                t0[it] = a.tign0[k];
                ti[it] = a.tign[k];
                to[it] = tobs[k];
                p0[it] = a.pa[k];
                p1[it] = a.pb[k];
                ls[it] = at(2, x, y);
            }
        }
        const double tlo = a.tsp[0], thi = a.tsp[1];
#pragma unroll
        for (int it = 0; it < I2; ++it) {
            if (ls[it] < 0) continue;
            T mu = vl[it];
            double q0, q1, r;
            if (cross_seed(t0[it], ti[it], to[it], p0[it], p1[it], tlo, thi, q0, q1, r)) {
                const double den = q0 - q1;
                mu = T((double)mu + r * a.dt * q0 / (den * den));
            }
            sm.mu[ls[it]] = mu;
        }
    }
    {
        constexpr int I0 = (kRevO + kRevThreads - 1) / kRevThreads;
        T p0[I0], p1[I0];
        double t0[I0], ti[I0], to[I0];
        bool in[I0];
#pragma unroll
        for (int it = 0; it < I0; ++it) {
            const int e = tid + it * kRevThreads;
            const int x = x0 + e % kRevTX, y = y0 + e / kRevTX;
            in[it] = x < nx && y < ny;
            if (in[it]) {
                const size_t k = (size_t)y * nx + x;
                t0[it] = a.tign0[k];
                ti[it] = a.tign[k];
                to[it] = tobs[k];
                p0[it] = a.pa[k];
                p1[it] = a.pb[k];
            }
        }
        const double tlo = a.tsp[0], thi = a.tsp[1];
#pragma unroll
        for (int it = 0; it < I0; ++it) {
            double sd = 0.0, q0, q1, r;
            if (in[it] && cross_seed(t0[it], ti[it], to[it], p0[it], p1[it], tlo, thi, q0, q1, r)) {
                const double den = q0 - q1;
                sd = r * (-a.dt * q1 / (den * den));
            }
            sm.seed[tid + it * kRevThreads] = sd;
        }
    }
    __syncthreads();
    // ---- psi* = psi^s + dt F(psi^s) (radius 3)
    for (int e = tid; e < F3; e += kRevThreads) {
        int x, y;
        if (!region(3, e, x, y)) continue;
        const int l3 = at(3, x, y);
        NodeEnv<T> en;
        rev_env(a, sm, l3, (size_t)y * nx + x, false, en);
        T p, pl, pr, pd, pu;
        rev_stencil(sm.pa, at(4, x, y), W4, x, y, nx, ny, p, pl, pr, pd, pu);
        const T F = rhs_vals<T>(p, pl, pr, pd, pu, a.idx, a.idy, a.i2dx, a.i2dy, a.eps, en.co,
                                en.m, en.un, en.vn, en.zx, en.zy);
        sm.ps[l3] = p + a.dtT * F;
    }
    __syncthreads();
    // ---- the product at psi* with v = dt/2 mu (radius 2)
    for (int e = tid; e < F2; e += kRevThreads) {
        int x, y;
        if (!region(2, e, x, y)) continue;
        const int l3 = at(3, x, y), l2 = at(2, x, y);
        T g[4];
        rev_vjp(a, sm, sm.ps, l3, W3, l3, l2, x, y, (size_t)y * nx + x, a.hdtT * sm.mu[l2], g);
        const int ox = x - x0, oy = y - y0;
        if (ox >= 0 && ox < kRevTX && oy >= 0 && oy < kRevTY) {
            const int o = oy * kRevTX + ox;
#pragma unroll
            for (int q = 0; q < 4; ++q) sm.G[q * kRevO + o] = g[q];
        }
    }
    __syncthreads();
    // ---- lam* (radius 1)
    for (int e = tid; e < F1; e += kRevThreads) {
        int x, y;
        if (region(1, e, x, y))
            sm.ls[at(1, x, y)] =
                rev_gather(sm.C, at(2, x, y), W2, F2, sm.ps, at(3, x, y), W3, x, y, nx, ny);
    }
    __syncthreads();
    // ---- the product at psi^s with w = dt/2 mu + dt lam* (radius 1); the
    // owner adds both products' parameter terms
    for (int e = tid; e < F1; e += kRevThreads) {
        int x, y;
        if (!region(1, e, x, y)) continue;
        const size_t k = (size_t)y * nx + x;
        const int l2 = at(2, x, y);
        T g[4];
        rev_vjp(a, sm, sm.pa, at(4, x, y), W4, at(3, x, y), l2, x, y, k,
                a.hdtT * sm.mu[l2] + a.dtT * sm.ls[at(1, x, y)], g);
        const int ox = x - x0, oy = y - y0;
        if (ox >= 0 && ox < kRevTX && oy >= 0 && oy < kRevTY) {
            const int o = oy * kRevTX + ox;
            const int nq = a.wind_grads ? 4 : 2;
            typename GAcc<T>::t acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nq) acc[q] = a.acc[q * a.n + k];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q >= nq) continue;
                GAcc<T>::add(acc[q], sm.G[q * kRevO + o]);
                GAcc<T>::add(acc[q], g[q]);
                a.acc[q * a.n + k] = acc[q];
            }
        }
    }
    __syncthreads();
    // ---- lambda^s on the tile
    for (int e = tid; e < kRevO; e += kRevThreads) {
        const int x = x0 + e % kRevTX, y = y0 + e / kRevTX;
        if (x >= nx || y >= ny) continue;
        const int l2 = at(2, x, y);
        T lam = sm.mu[l2] + sm.ls[at(1, x, y)] +
                rev_gather(sm.C, l2, W2, F2, sm.pa, at(4, x, y), W4, x, y, nx, ny);
        const double sd = sm.seed[e];
        if (sd != 0.0) lam = T((double)lam + sd);
        a.lout[(size_t)y * nx + x] = lam;
    }
}

// the FP32 sums of the run: a seed (the heat misfit's direct moisture term)
// into a compensated pair, and the pairs back to double at the end
__global__ void k_acc_seed(double *g, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const double x = g[k];
        const float s = (float)x;
        reinterpret_cast<float2 *>(g)[k] = make_float2(s, (float)((double)s - x));
    }
}
__global__ void k_acc_final(double *g, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const float2 p = reinterpret_cast<const float2 *>(g)[k];
        g[k] = (double)p.x - (double)p.y;
    }
}

// Adjoint of the bilinear wind interpolation (Sect. 5): every staggered
// face sums the node gradients times the weights the forward gave it.
// One warp per face: each lane takes every 32nd column of the candidate
// nodes (those within two cells), its rows in order, then the lanes' sums
// are added in a fixed tree, so the result does not depend on scheduling.
template <typename T>
__global__ void k_adj_wind(const AdjArgs<T> a, const double *gun, const double *gvn, double *gu,
                           double *gv) {
    const int nu = a.nya * (a.nxa + 1), nv = (a.nya + 1) * a.nxa;
    const int lane = threadIdx.x & 31;
    const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int f = w0; f < nu + nv; f += nw) {
        const bool isu = f < nu;
        const int q = isu ? f : f - nu;
        const int W = isu ? a.nxa + 1 : a.nxa;
        const int I = q % W, J = q / W;
        const int i_lo = max(0, (I - 2) * a.srx), i_hi = min(a.nx, (I + 2) * a.srx);
        const int j_lo = max(0, (J - 2) * a.sry), j_hi = min(a.ny, (J + 2) * a.sry);
        const double *g = isu ? gun : gvn;
        double s = 0.0;
        for (int i = i_lo + lane; i < i_hi; i += 32) {
            const T xr = (T(i) + T(0.5)) / T(a.srx);
            int i0, i1;
            T wx;
            if (isu) lin_idx<T>(xr, a.nxa + 1, i0, i1, wx);
            else lin_idx<T>(xr - T(0.5), a.nxa, i0, i1, wx);
            double cx = 0.0;
            if (i0 == I) cx += (double)(T(1) - wx);
            if (i1 == I) cx += (double)wx;
            if (cx == 0.0) continue;
            for (int j = j_lo; j < j_hi; ++j) {
                const T yr = (T(j) + T(0.5)) / T(a.sry);
                int j0, j1;
                T wy;
                if (isu) lin_idx<T>(yr - T(0.5), a.nya, j0, j1, wy);
                else lin_idx<T>(yr, a.nya + 1, j0, j1, wy);
                double cy = 0.0;
                if (j0 == J) cy += (double)(T(1) - wy);
                if (j1 == J) cy += (double)wy;
                if (cy != 0.0) s += g[(size_t)j * a.nx + i] * (cy * cx);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (isu) gu[q] = s;
            else gv[q] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Heat misfit.  Q_I = sensible heat released per unit area of atmospheric
// cell I over the run = sum over its fire cells of (F_start - F_end) H_s /
// (srx sry) (the time integral of eqs. sensible-heat-flux / average, which
// telescopes), J = 1/2 sum over observed cells of (Q_I - q_obs,I)^2.  Its
// seeds for the reverse sweep: dJ/dF_end through the quadrature of Sect. 3.3
// into dJ/dpsi_end and dJ/dt_i, and the moisture dependence of H_s.
// ---------------------------------------------------------------------------
template <typename T>
struct HeatArgs {
    const T *psi, *F0, *F1;  // psi and F at the end, F at the start of the run
    const double *tign;      // t_i at the end
    const uint8_t *fuel;
    const double *coef, *dcoef;  // [ncls][K_N], or [n][K_N] per node when nodeco
    int nodeco;
    int ncls, nx, ny, nxa, nya, srx, sry;
    double t1;               // model time at the end
    const double *qobs;      // [nya][nxa], NaN where unobserved
    double *Q, *res;         // [nya][nxa]
    double *gF, *gM;         // [n]: dJ/dF_end, moisture gradient (direct term)
    double *lamd, *dJdt;     // [n]: dJ/dpsi_end, dJ/dt_i
};

// Q and the residual per atmospheric cell (the fire cells summed row by row)
template <typename T>
__global__ void k_heat_residual(const HeatArgs<T> h) {
    const int na = h.nxa * h.nya;
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < na; I += gridDim.x * blockDim.x) {
        const int ia = I % h.nxa, ja = I / h.nxa;
        double q = 0.0;
        for (int j = ja * h.sry; j < (ja + 1) * h.sry; ++j)
            for (int i = ia * h.srx; i < (ia + 1) * h.srx; ++i) {
                const size_t k = (size_t)j * h.nx + i;
                const size_t c = h.nodeco ? k : (size_t)min((int)h.fuel[k], h.ncls - 1);
                q += ((double)h.F0[k] - (double)h.F1[k]) * h.coef[c * K_N + K_HS];
            }
        q /= (double)(h.srx * h.sry);
        h.Q[I] = q;
        h.res[I] = finite_bits(h.qobs[I]) ? q - h.qobs[I] : 0.0;
    }
}

// per fire cell: dJ/dF_end = -res H_s / (srx sry), and the direct moisture
// term res (F_start - F_end) dH_s/dM_f / (srx sry)
template <typename T>
__global__ void k_heat_seed(const HeatArgs<T> h) {
    const size_t n = (size_t)h.nx * h.ny;
    const double r2 = (double)(h.srx * h.sry);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % h.nx), j = (int)(k / h.nx);
        const double r = h.res[(j / h.sry) * h.nxa + i / h.srx];
        const size_t c = h.nodeco ? k : (size_t)min((int)h.fuel[k], h.ncls - 1);
        h.gF[k] = -r * h.coef[c * K_N + K_HS] / r2;
        h.gM[k] = r * ((double)h.F0[k] - (double)h.F1[k]) * h.dcoef[c * K_N + K_HS] / r2;
    }
}

// psi at position (x, y) of the ghost-extended mesh (x in -1..nx, y in
// -1..ny): the extrapolated ghosts of Sect. 3.1, x first, then y
template <typename T>
__device__ double ext_psi(const T *psi, int nx, int ny, int x, int y) {
    auto row = [&](int xx, int yy) -> double {  // yy inside the mesh
        if (xx >= 0 && xx < nx) return (double)psi[(size_t)yy * nx + xx];
        const size_t b = (size_t)yy * nx;
        return xx < 0 ? ghost_value<double>((double)psi[b], (double)psi[b + 1])
                      : ghost_value<double>((double)psi[b + nx - 1], (double)psi[b + nx - 2]);
    };
    if (y >= 0 && y < ny) return row(x, y);
    return y < 0 ? ghost_value<double>(row(x, 0), row(x, 1))
                 : ghost_value<double>(row(x, ny - 1), row(x, ny - 2));
}

// d F_cell / d(window psi) and d F_cell / d(window t^) of the quadrature of
// Sect. 3.3 (eqs. fuel_left_subcells, approx-fraction, ti-comp) for the cell
// whose 3x3 node window is w[9] (psi) and th[9] (t^, already t1 where the
// node's psi >= 0): four subcells of the cell centre, two edge midpoints
// and a corner (bilinear means of the nodes), burned = beta (1 - e),
// beta = (1 - sum psi / sum |psi|) / 2, e = exp(-sum (t1 - t^) / (4 T_f)),
// F = 1 - mean of the four burned fractions.  Branches as the forward took
// them: a vertex with psi >= 0 takes t1 (no t^ dependence), |x|' = sign(x).
__device__ void quad_partials(const double *w, const double *th, double t1, double Tf,
                              double *dw, double *dth) {
    // vertices: node lists (up to 4 nodes, mean) of the centre, the four edge
    // midpoints and the four corners, indexed by window position 3b + a
    double vp[9], vt[9];
    int vn[9][4], vc[9];
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            const int v = 3 * b + a, xs[2] = {a == 0 ? 0 : 1, a == 2 ? 2 : 1},
                      ys[2] = {b == 0 ? 0 : 1, b == 2 ? 2 : 1};
            int m = 0;
            for (int yy = 0; yy < (ys[0] == ys[1] ? 1 : 2); ++yy)
                for (int xx = 0; xx < (xs[0] == xs[1] ? 1 : 2); ++xx) vn[v][m++] = 3 * ys[yy] + xs[xx];
            vc[v] = m;
            double sp = 0.0, st = 0.0;
            if (m == 1) {
                sp = w[vn[v][0]];
                st = th[vn[v][0]];
            } else if (m == 2) {
                sp = 0.5 * (w[vn[v][0]] + w[vn[v][1]]);
                st = 0.5 * (th[vn[v][0]] + th[vn[v][1]]);
            } else {
                sp = 0.25 * (w[vn[v][0]] + w[vn[v][1]] + w[vn[v][2]] + w[vn[v][3]]);
                st = 0.25 * (th[vn[v][0]] + th[vn[v][1]] + th[vn[v][2]] + th[vn[v][3]]);
            }
            vp[v] = sp;
            vt[v] = sp >= 0.0 ? t1 : st;
        }
    double gv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int sub = 0; sub < 4; ++sub) {
        const int cx = (sub & 1) ? 2 : 0, cy = (sub & 2) ? 2 : 0;
        const int vs[4] = {4, 3 + cx, 3 * cy + 1, 3 * cy + cx};  // centre, x-edge, y-edge, corner
        double s = 0.0, a = 0.0, tau = 0.0;
        for (int q = 0; q < 4; ++q) {
            s += vp[vs[q]];
            a += fabs(vp[vs[q]]);
            tau += t1 - vt[vs[q]];
        }
        const double e = exp(-0.25 * tau / Tf);
        const double beta = a > 0.0 ? 0.5 * (1.0 - s / a) : 0.0;
        for (int q = 0; q < 4; ++q) {
            const double x = vp[vs[q]];
            const double sg = x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
            // dF/dbeta = -(1 - e)/4; dbeta/dx = (s sg / a - 1) / (2 a)
            if (a > 0.0) gv[vs[q]] += -0.25 * (1.0 - e) * 0.5 * (s * sg / a - 1.0) / a;
            // dF/dt^_vertex = -(1/4) d burned / dt^ = beta e / (16 T_f)
            gt[vs[q]] += 0.0625 * beta * e / Tf;
        }
    }
    for (int q = 0; q < 9; ++q) {
        dw[q] = 0.0;
        dth[q] = 0.0;
    }
    for (int v = 0; v < 9; ++v) {
        const double f = 1.0 / vc[v];
        for (int m = 0; m < vc[v]; ++m) {
            dw[vn[v][m]] += f * gv[v];
            if (vp[v] < 0.0) dth[vn[v][m]] += f * gt[v];
        }
    }
}

// the window of cell (i, j) at the end of the run and its partials times
// dJ/dF of the cell; false when the cell contributes nothing
template <typename T>
__device__ bool heat_cell(const HeatArgs<T> &h, int i, int j, double *dw, double *dth,
                          double *w) {
    const size_t k = (size_t)j * h.nx + i;
    const double g = h.gF[k];
    if (g == 0.0) return false;
    double th[9];
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            const int x = i + a - 1, y = j + b - 1;
            const double p = ext_psi(h.psi, h.nx, h.ny, x, y);
            // t^ of the position: t1 where its psi >= 0, else the copied t^ of
            // the nearest node (t_i where that node's psi < 0, else t1)
            const int xc = min(max(x, 0), h.nx - 1), yc = min(max(y, 0), h.ny - 1);
            const size_t kc = (size_t)yc * h.nx + xc;
            w[3 * b + a] = p;
            th[3 * b + a] = (p >= 0.0 || !((double)h.psi[kc] < 0.0)) ? h.t1 : h.tign[kc];
        }
    const size_t c = h.nodeco ? k : (size_t)min((int)h.fuel[k], h.ncls - 1);
    quad_partials(w, th, h.t1, h.coef[c * K_N + K_TF], dw, dth);
    for (int q = 0; q < 9; ++q) {
        dw[q] *= g;
        dth[q] *= g;
    }
    return true;
}

// per node: the contributions of the (up to 9) cells whose window holds the
// node itself (the ghost positions of the boundary cells are added by
// k_heat_ghosts)
template <typename T>
__global__ void k_heat_gather(const HeatArgs<T> h) {
    const size_t n = (size_t)h.nx * h.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % h.nx), j = (int)(k / h.nx);
        const bool tnode = (double)h.psi[k] < 0.0;
        double lp = 0.0, lt = 0.0, dw[9], dth[9], w[9];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int ci = i - dx, cj = j - dy;  // cell whose window has this node at (dx, dy)
                if (ci < 0 || ci >= h.nx || cj < 0 || cj >= h.ny) continue;
                if (!heat_cell(h, ci, cj, dw, dth, w)) continue;
                const int q = 3 * (dy + 1) + (dx + 1);
                lp += dw[q];
                if (tnode) lt += dth[q];
            }
        h.lamd[k] = lp;
        h.dJdt[k] = lt;
    }
}

// the ghost positions of the boundary cells' windows, one thread in a fixed
// order: psi ghosts back to the nodes they extrapolate (x ghosts, and y
// ghosts of the extended columns, corners included), t^ ghosts to the node
// they copy
template <typename T>
__global__ void k_heat_ghosts(const HeatArgs<T> h) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int nx = h.nx, ny = h.ny;
    auto add_row = [&](int x, int y, double d) {  // d/d(psi at (x, y)), y inside
        if (x >= 0 && x < nx) {
            h.lamd[(size_t)y * nx + x] += d;
            return;
        }
        const size_t b = (size_t)y * nx;
        const int e0 = x < 0 ? 0 : nx - 1, e1 = x < 0 ? 1 : nx - 2;
        double d0, d1;
        ghost_partials<double>((double)h.psi[b + e0], (double)h.psi[b + e1], d0, d1);
        h.lamd[b + e0] += d * d0;
        h.lamd[b + e1] += d * d1;
    };
    auto add_psi = [&](int x, int y, double d) {
        if (y >= 0 && y < ny) {
            add_row(x, y, d);
            return;
        }
        const int f0 = y < 0 ? 0 : ny - 1, f1 = y < 0 ? 1 : ny - 2;
        double d0, d1;
        ghost_partials<double>(ext_psi(h.psi, nx, ny, x, f0), ext_psi(h.psi, nx, ny, x, f1), d0,
                               d1);
        add_row(x, f0, d * d0);
        add_row(x, f1, d * d1);
    };
    double dw[9], dth[9], w[9];
    const long nb = 2L * nx + 2L * (ny - 2);
    for (long q = 0; q < nb; ++q) {
        int i, j;  // boundary cells: bottom row, top row, then the side columns
        if (q < nx) { i = (int)q; j = 0; }
        else if (q < 2L * nx) { i = (int)(q - nx); j = ny - 1; }
        else { const long r = q - 2L * nx; i = (r & 1) ? nx - 1 : 0; j = 1 + (int)(r >> 1); }
        if (!heat_cell(h, i, j, dw, dth, w)) continue;
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                const int x = i + a - 1, y = j + b - 1;
                if (x >= 0 && x < nx && y >= 0 && y < ny) continue;  // k_heat_gather's
                add_psi(x, y, dw[3 * b + a]);
                const int xc = min(max(x, 0), nx - 1), yc = min(max(y, 0), ny - 1);
                const size_t kc = (size_t)yc * nx + xc;
                if (w[3 * b + a] < 0.0 && (double)h.psi[kc] < 0.0) h.dJdt[kc] += dth[3 * b + a];
            }
    }
}

// lambda (path precision) at the end of the run from dJ/dpsi_end
template <typename T>
__global__ void k_heat_lambda(const double *lamd, T *lam, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        lam[k] = T(lamd[k]);
}

// J = 1/2 sum (t_i - t_obs)^2 over nodes ignited in both: fixed-shape tree
// sums (block partials, then one block), so the result is reproducible
__global__ void k_misfit_partial(const double *tign, const double *tobs, size_t n, double *part) {
    __shared__ double sh[kAdjThreads];
    double s = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const double ti = tign[k], to = tobs[k];
        if (isfinite(ti) && isfinite(to)) s += 0.5 * (ti - to) * (ti - to);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kAdjThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_misfit_final(const double *part, int nb, double *J) {
    __shared__ double sh[kAdjThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += kAdjThreads) s += part[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kAdjThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = sh[0];
}

constexpr int kMisfitBlocks = 304;

int cuda_fail(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return FIRE_OK;
    record_cuda_error(e, where);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return FIRE_ERR_OOM;
    }
    return FIRE_ERR_CUDA;
}
#define ADJ_CHECK(call)                                   \
    do {                                                  \
        int _r = cuda_fail((call), #call);                \
        if (_r != FIRE_OK) return _r;                     \
    } while (0)

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int c_nxa(fire_ctx *c) {
    StepArgs a;
    ctx_step_args(c, 0, nullptr, nullptr, 1.0, nullptr, nullptr, a);
    return a.nxa;
}
int c_nya(fire_ctx *c) {
    StepArgs a;
    ctx_step_args(c, 0, nullptr, nullptr, 1.0, nullptr, nullptr, a);
    return a.nya;
}

// tobs: the arrival-time misfit; qobs (with tobs null): the heat misfit
template <typename T>
int run_adjoint(fire_ctx *c, int nsteps, double dt, const void *u, const void *v,
                const double *tobs, const double *qobs, int K, double *J_host, double *g_mult,
                double *g_moist, double *g_u, double *g_v) {
    int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
    double t0;
    ctx_info(c, &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t0);
    const cudaStream_t st = ctx_stream(c);
    const size_t n = (size_t)nx * ny, E = sizeof(T);
    const bool grads = g_mult || g_moist || g_u || g_v;
    const int nseg = (nsteps + K - 1) / K;

    // host times of the step starts, as the context advances its clock
    std::vector<double> times(nsteps + 1);
    times[0] = t0;
    for (int s = 0; s < nsteps; ++s) times[s + 1] = times[s] + dt;
    for (int s = 0; s <= nsteps; ++s)
        if (ctx_ignition_active(c, times[s])) return FIRE_ERR_STATE;
    // the reverse sweep differentiates the subcell fuel-fraction scheme
    if (ctx_scheme(c) != 0) return FIRE_ERR_STATE;

    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    // checkpoints; with K = 1 every state psi^0..psi^nsteps
    const size_t o_ck = take((size_t)(K == 1 ? nsteps + 1 : nseg) * n * E);
    // the recomputed states of a segment (none when every state is kept)
    const size_t o_ring = take(K > 1 ? (size_t)(K + 1) * n * E : 0);
    const size_t o_F = take(2 * n * E);
    const size_t o_t0 = take(n * sizeof(double));
    const size_t o_ts = take(n * sizeof(double));
    const size_t o_times = take((nsteps + 2) * sizeof(double));
    const size_t o_tseg = take((K + 2) * sizeof(double));
    const size_t o_small = take(16 + kMisfitBlocks * sizeof(double) + 16);
    const size_t na = (size_t)c_nxa(c) * c_nya(c);
    // per-node coefficients of a per-node fuel moisture ([n][K_N] doubles)
    const void *moist = ctx_moisture(c);
    const bool nodeco = moist != nullptr;
    const size_t o_nco = take(nodeco ? n * K_N * sizeof(double) : 0);
    const size_t o_F0 = take(qobs ? n * E : 0);                   // F at the start (heat)
    const size_t o_Qr = take(qobs ? 2 * na * sizeof(double) : 0);  // Q, residual (heat)
    const size_t o_lam = take(2 * n * E);  // lambda^{s+1}, lambda^s
    // the unfused FP64 step: psi*, mu, lam* and two sets of stencil
    // contributions
    const bool fused = sizeof(T) == 4;
    const size_t o_mid = take(fused ? 0 : 13 * n * E);
    const size_t o_g = take(4 * n * sizeof(double));
    const size_t o_unv = take(2 * n * E);
    const size_t nu = (size_t)c_nya(c) * (c_nxa(c) + 1), nv = (size_t)(c_nya(c) + 1) * c_nxa(c);
    const size_t o_dco = take(sizeof(double) * K_N * (nodeco ? n : (size_t)ncls));
    const size_t o_wind = take(sizeof(double) * (nu + nv));
    const size_t o_hs = take(qobs ? 3 * n * sizeof(double) : 0);  // dJ/dF, dJ/dpsi, dJ/dt_i
    void *wsv = nullptr;
    int r = ctx_workspace(c, grads ? off : o_lam, &wsv);
    if (r) return r;
    unsigned char *ws = static_cast<unsigned char *>(wsv);
    T *ck = reinterpret_cast<T *>(ws + o_ck);
    T *ring = reinterpret_cast<T *>(ws + o_ring);
    T *Fs = reinterpret_cast<T *>(ws + o_F);
    double *tign0 = reinterpret_cast<double *>(ws + o_t0);
    double *tsc = reinterpret_cast<double *>(ws + o_ts);
    double *tdev = reinterpret_cast<double *>(ws + o_times);
    double *tseg = reinterpret_cast<double *>(ws + o_tseg);
    double *Jdev = reinterpret_cast<double *>(ws + o_small);
    int *stdev = reinterpret_cast<int *>(ws + o_small + 8);
    double *part = reinterpret_cast<double *>(ws + o_small + 16);

    // launches replayed from graphs the context keeps (two slots, each
    // with the key of what its launches read; captured on first use, issued
    // directly if the capture is refused)
    unsigned long long *keys = nullptr;
    cudaGraphExec_t *graphs = ctx_adjoint_graphs(c, &keys);
    auto mix = [](unsigned long long h, unsigned long long x) {
        return (h ^ x) * 0x100000001b3ULL + (h >> 29);
    };
    auto replay = [&](int slot, unsigned long long key, auto &&issue) -> int {
        if (!graphs[slot] || keys[slot] != key) {
            if (graphs[slot]) {
                ADJ_CHECK(cudaStreamSynchronize(st));  // the old graph may be in flight
                cudaGraphExecDestroy(graphs[slot]);
                graphs[slot] = nullptr;
            }
            cudaStream_t cs;
            ADJ_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                e = issue(cs);
                cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&graphs[slot], gr, 0);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) {
                record_cuda_error(e, "capture of adjoint launches");
                cudaGetLastError();
                graphs[slot] = nullptr;
                keys[slot] = 0;
                ADJ_CHECK(issue(st));
                return FIRE_OK;
            }
            keys[slot] = key;
        }
        ADJ_CHECK(cudaGraphLaunch(graphs[slot], st));
        return FIRE_OK;
    };

    StepArgs sa;
    ctx_step_args(c, cur, u, v, dt, nullptr, nullptr, sa);
    ADJ_CHECK(cudaMemcpyAsync(tign0, sa.tign, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // the coefficients the adjoint kernels read: per class, or per node
    const double *coef_rows = sa.coef;
    if (nodeco) {
        double *aos = reinterpret_cast<double *>(ws + o_nco);
        T *none[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        ADJ_CHECK(launch_node_coefficients<T>(ctx_classes_dev(c), ncls, sa.fuel, moist, n, none,
                                              aos, st));
        coef_rows = aos;
    }
    T *F0 = reinterpret_cast<T *>(ws + o_F0);
    if (qobs) ADJ_CHECK(cudaMemcpyAsync(F0, sa.F_in, n * E, cudaMemcpyDeviceToDevice, st));
    ADJ_CHECK(cudaMemcpyAsync(tdev, times.data(), (nsteps + 1) * sizeof(double),
                              cudaMemcpyHostToDevice, st));

    // the step kernel the context uses, on a state it does not own
    auto launch_step_kernel = [&](const StepArgs &ra, cudaStream_t cs) -> cudaError_t {
        return variant == FIRE_KERNEL_MARCH   ? launch_march<T>(ra, cs)
               : variant == FIRE_KERNEL_WARP  ? launch_warp<T>(ra, cs)
               : variant == FIRE_KERNEL_WARP_DENSE ? launch_warp<T>(ra, cs, true)
               : variant == FIRE_KERNEL_WARP4 ? (sizeof(T) == 4 ? launch_warp4(ra, cs)
                                                                : cudaErrorInvalidValue)
                                              : launch_step<T>(ra, cs);
    };
    // forward with checkpoints
    if (K == 1) {
        // every state is a checkpoint: each step reads and writes its slots
        // directly (the context's fraction, t_i, time and status buffers as
        // fire_run uses them), then the last state goes back to the context
        int pc, pv, a1, a2, a3, a4, a5, a6, a7, pcur;
        double tt;
        ctx_info(c, &pc, &pv, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &pcur, &tt);
        unsigned long long fk = 0x84222325cbf29ce4ULL;
        unsigned long long dtb;
        memcpy(&dtb, &dt, sizeof dtb);
        const void *fp[] = {ws, u, v, sa.mult, sa.coef, sa.fuel, sa.dzdy, sa.dzdx, sa.tign,
                            sa.nco[0], moist};
        for (const void *q : fp) fk = mix(fk, (unsigned long long)(uintptr_t)q);
        fk = mix(mix(mix(mix(mix(fk, dtb), (unsigned long long)nsteps), (unsigned long long)pcur),
                     (unsigned long long)variant),
                 (unsigned long long)(sa.kx * 65536 + sa.ky));
        r = replay(1, fk, [&](cudaStream_t cs) -> cudaError_t {
            StepArgs now;
            ctx_step_args(c, pcur, u, v, dt, nullptr, nullptr, now);
            cudaError_t e = cudaMemcpyAsync(ck, now.psi_in, n * E, cudaMemcpyDeviceToDevice, cs);
            for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
                StepArgs ra;
                ctx_step_args(c, (pcur + s) & 1, u, v, dt, nullptr, nullptr, ra);
                ra.psi_in = ck + (size_t)s * n;
                ra.psi_out = ck + (size_t)(s + 1) * n;
                e = launch_step_kernel(ra, cs);
            }
            StepArgs fin;
            ctx_step_args(c, (pcur + nsteps) & 1, u, v, dt, nullptr, nullptr, fin);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(const_cast<void *>(fin.psi_in), ck + (size_t)nsteps * n,
                                    n * E, cudaMemcpyDeviceToDevice, cs);
            return e;
        });
        if (r) return r;
        ctx_advance(c, nsteps, dt);
    }
    for (int q = 0; q < (K == 1 ? 0 : nseg); ++q) {
        StepArgs now;
        int pc, pv, a1, a2, a3, a4, a5, a6, a7, pcur;
        double tt;
        ctx_info(c, &pc, &pv, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &pcur, &tt);
        ctx_step_args(c, pcur, u, v, dt, nullptr, nullptr, now);
        ADJ_CHECK(cudaMemcpyAsync(ck + (size_t)q * n, now.psi_in, n * E, cudaMemcpyDeviceToDevice,
                                  st));
        const int len = (q + 1) * K <= nsteps ? K : nsteps - q * K;
        r = fire_run(c, len, dt, u, v, nullptr, nullptr);
        if (r) return r;
    }
    const double *tign_final = sa.tign;
    ADJ_CHECK(cudaGetLastError());
    HeatArgs<T> h;
    memset(&h, 0, sizeof h);
    if (qobs) {
        // the state at the end of the run
        StepArgs fin;
        int pc, pv, a1, a2, a3, a4, a5, a6, a7, pcur;
        double tt;
        ctx_info(c, &pc, &pv, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &pcur, &tt);
        ctx_step_args(c, pcur, u, v, dt, nullptr, nullptr, fin);
        h.psi = static_cast<const T *>(fin.psi_in);
        h.F0 = F0;
        h.F1 = static_cast<const T *>(fin.F_in);
        h.tign = tign_final;
        h.fuel = sa.fuel;
        h.coef = coef_rows;
        h.nodeco = nodeco ? 1 : 0;
        h.ncls = ncls;
        h.nx = nx;
        h.ny = ny;
        h.nxa = sa.nxa;
        h.nya = sa.nya;
        h.srx = srx;
        h.sry = sry;
        h.t1 = times[nsteps];
        h.qobs = qobs;
        h.Q = reinterpret_cast<double *>(ws + o_Qr);
        h.res = h.Q + na;
        k_heat_residual<T><<<(int)((na + kAdjThreads - 1) / kAdjThreads), kAdjThreads, 0, st>>>(h);
        k_misfit_partial<<<kMisfitBlocks, kAdjThreads, 0, st>>>(h.Q, qobs, na, part);
    } else {
        k_misfit_partial<<<kMisfitBlocks, kAdjThreads, 0, st>>>(tign_final, tobs, n, part);
    }
    k_misfit_final<<<1, kAdjThreads, 0, st>>>(part, kMisfitBlocks, Jdev);
    ADJ_CHECK(cudaGetLastError());
    ADJ_CHECK(cudaMemcpyAsync(J_host, Jdev, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!grads) {
        ADJ_CHECK(cudaStreamSynchronize(st));
        return FIRE_OK;
    }

    // lambda ping-pongs between lam and lam + n, starting in lam; the
    // parameter sums are four fields of n doubles (FP64), or of n
    // compensated float pairs in the same bytes (FP32), turned into doubles
    // in place after the sweep
    T *lam = reinterpret_cast<T *>(ws + o_lam);
    double *gm = reinterpret_cast<double *>(ws + o_g);
    double *gM = gm + n, *gun = gm + 2 * n, *gvn = gm + 3 * n;
    static_assert(sizeof(typename GAcc<T>::t) == sizeof(double), "sums in place of doubles");
    ADJ_CHECK(cudaMemsetAsync(lam, 0, n * E, st));
    ADJ_CHECK(cudaMemsetAsync(gm, 0, 4 * n * sizeof(double), st));
    ADJ_CHECK(cudaMemsetAsync(Fs, 0, 2 * n * E, st));

    // d(coefficients)/d(M_f) per class at the class moisture, or per node at
    // the node's moisture
    double *dcoef = reinterpret_cast<double *>(ws + o_dco);
    if (nodeco)
        ADJ_CHECK(launch_node_coefficients_dMf<T>(ctx_classes_dev(c), ncls, sa.fuel, moist, n,
                                                  dcoef, st));
    else
        ADJ_CHECK(launch_coefficients_dMf(ctx_classes_dev(c), ncls, dcoef, st));

    AdjArgs<T> a;
    memset(&a, 0, sizeof a);
    a.fuel = sa.fuel;
    a.zx = static_cast<const T *>(sa.dzdx);
    a.zy = static_cast<const T *>(sa.dzdy);
    a.mult = static_cast<const T *>(sa.mult);
    a.u = static_cast<const T *>(u);
    a.v = static_cast<const T *>(v);
    a.coef = coef_rows;
    a.dcoef = dcoef;
    a.nodeco = nodeco ? 1 : 0;
    a.ncls = ncls;
    a.tign0 = tign0;
    a.tign = tign_final;
    a.tobs = tobs;
    a.dJdt = nullptr;
    a.dt = dt;
    a.acc = reinterpret_cast<typename GAcc<T>::t *>(gm);
    a.wind_grads = (g_u || g_v) ? 1 : 0;
    a.nx = nx;
    a.ny = ny;
    a.nxa = sa.nxa;
    a.nya = sa.nya;
    a.srx = srx;
    a.sry = sry;
    // the step kernels' constants, rounded the same way
    a.idx = T(1) / T(sa.dx);
    a.idy = T(1) / T(sa.dy);
    a.i2dx = T(1) / (T(2) * T(sa.dx));
    a.i2dy = T(1) / (T(2) * T(sa.dy));
    a.eps = T(sa.eps);
    a.dtT = T(dt);
    a.hdtT = T(0.5 * dt);
    a.n = n;

    int dev = 0, sms = 0;
    ADJ_CHECK(cudaGetDevice(&dev));
    ADJ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    {
        T *unv = reinterpret_cast<T *>(ws + o_unv);
        const size_t wn = (n + kAdjThreads - 1) / kAdjThreads;
        k_adj_node_wind<T><<<(int)(wn < (size_t)sms * 8 ? wn : (size_t)sms * 8), kAdjThreads, 0,
                             st>>>(a, unv);
        ADJ_CHECK(cudaGetLastError());
        a.unv = unv;
    }
    const size_t want = (n + kAdjThreads - 1) / kAdjThreads;
    const int grid = (int)(want < (size_t)sms * 8 ? want : (size_t)sms * 8);
    if (qobs) {
        // seeds of the heat misfit: dJ/dF and the H_s moisture term, the
        // quadrature's transpose into dJ/dpsi_end (lambda) and dJ/dt_i
        double *hs = reinterpret_cast<double *>(ws + o_hs);
        h.dcoef = dcoef;
        h.gF = hs;
        h.gM = gM;
        h.lamd = hs + n;
        h.dJdt = hs + 2 * n;
        k_heat_seed<T><<<grid, kAdjThreads, 0, st>>>(h);
        k_heat_gather<T><<<grid, kAdjThreads, 0, st>>>(h);
        k_heat_ghosts<T><<<1, 1, 0, st>>>(h);
        k_heat_lambda<T><<<grid, kAdjThreads, 0, st>>>(h.lamd, lam, n);
        if (sizeof(T) == 4) k_acc_seed<<<grid, kAdjThreads, 0, st>>>(gM, n);
        ADJ_CHECK(cudaGetLastError());
        a.dJdt = h.dJdt;
    }

    // the reverse steps: tiles of the fused kernel, lambda^{s+1} in
    // lam + (r & 1) n for the r-th reverse step of a run of them
    if constexpr (sizeof(T) == 4) {
        // the kernel's attributes, once per device
        static std::mutex rev_mu;
        static bool rev_attr[kMaxDevices] = {};
        std::lock_guard<std::mutex> rev_lock(rev_mu);
        const int devid = attr_device();
        if (devid < 0 || !rev_attr[devid]) {
            ADJ_CHECK(cudaFuncSetAttribute(k_adj_step<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)rev_smem_bytes<T>(FIRE_MAX_CLASSES)));
            // all of the unified L1 as shared memory: four tiles per SM
            ADJ_CHECK(cudaFuncSetAttribute(k_adj_step<T>,
                                           cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            if (devid >= 0) rev_attr[devid] = true;
        }
    }
    const dim3 rgrid((nx + kRevTX - 1) / kRevTX, (ny + kRevTY - 1) / kRevTY);
    T *mid = reinterpret_cast<T *>(ws + o_mid);
    auto reverse = [&](AdjArgs<T> &b, const T *pa, const T *pb, const double *tsp, int r,
                       cudaStream_t cs) {
        b.pa = pa;
        b.pb = pb;
        b.tsp = tsp;
        b.lin = lam + (size_t)(r & 1) * n;
        b.lout = lam + (size_t)((r + 1) & 1) * n;
        if constexpr (sizeof(T) == 4) {
            k_adj_step<T><<<rgrid, kRevThreads, rev_smem_bytes<T>(ncls), cs>>>(b);
        } else {
            T *C1 = mid + 3 * n, *C2 = mid + 8 * n;
            b.pstar = mid;
            b.mu = mid + n;
            b.ls = mid + 2 * n;
            b.X = nullptr;
            b.Cin = nullptr;
            b.Cout = nullptr;
            k_adj_stage1<T><<<grid, kAdjThreads, 0, cs>>>(b);
            b.X = b.pstar;
            b.Cout = C1;
            k_adj_vjp_star<T><<<grid, kAdjThreads, 0, cs>>>(b);
            b.X = b.pa;
            b.Cin = C1;
            b.Cout = C2;
            k_adj_vjp_n<T><<<grid, kAdjThreads, 0, cs>>>(b);
            b.Cin = C2;
            k_adj_finish<T><<<grid, kAdjThreads, 0, cs>>>(b);
        }
    };

    // One segment: ring slot 0 holds its checkpoint and tseg its step times,
    // so every segment of a given length issues the same launches: the
    // recomputed states psi^{1..len} with the forward's step kernel, then the
    // reverse steps.  They are captured once per length in a CUDA graph (kept
    // by the context while the key below is unchanged) and replayed.
    auto issue_segment = [&](int len, cudaStream_t cs) -> cudaError_t {
        for (int j = 0; j < len; ++j) {
            StepArgs ra = sa;
            ra.psi_in = ring + (size_t)j * n;
            ra.psi_out = ring + (size_t)(j + 1) * n;
            ra.F_in = Fs + (size_t)(j & 1) * n;
            ra.F_out = Fs + (size_t)((j + 1) & 1) * n;
            ra.tign = tsc;
            ra.heat_s = nullptr;
            ra.heat_l = nullptr;
            ra.status = stdev;
            ra.t_in = tseg + j;
            ra.t_out = tseg + K + 1;
            ra.dt = dt;
            cudaError_t e = launch_step_kernel(ra, cs);
            if (e != cudaSuccess) return e;
        }
        AdjArgs<T> b = a;
        int rr = 0;
        for (int j = len - 1; j >= 0; --j, ++rr)
            reverse(b, ring + (size_t)j * n, ring + (size_t)(j + 1) * n, tseg + j, rr, cs);
        // every segment starts with lambda in lam
        if (len & 1) {
            cudaError_t e = cudaMemcpyAsync(lam, lam + n, n * E, cudaMemcpyDeviceToDevice, cs);
            if (e != cudaSuccess) return e;
        }
        return cudaGetLastError();
    };
    unsigned long long key0 = 0xcbf29ce484222325ULL;
    const void *ptrs[] = {ws, u, v, tobs, qobs, sa.mult, sa.coef, sa.fuel, sa.dzdy, sa.dzdx, sa.tign,
                          sa.nco[0], moist};
    for (const void *q : ptrs) key0 = mix(key0, (unsigned long long)(uintptr_t)q);
    unsigned long long dtb;
    memcpy(&dtb, &dt, sizeof dtb);
    key0 = mix(mix(mix(mix(mix(key0, dtb), (unsigned long long)K), (unsigned long long)n),
                   (unsigned long long)variant),
               (unsigned long long)(sa.kx * 65536 + sa.ky));
    key0 = mix(mix(key0, (unsigned long long)grid), (unsigned long long)a.wind_grads);
    if (K == 1) {
        // every state is a checkpoint: the reverse steps read them, nothing
        // is recomputed; the sweep is one graph
        r = replay(0, mix(mix(key0, (unsigned long long)nsteps), 0x5eedULL),
                   [&](cudaStream_t cs) -> cudaError_t {
                       AdjArgs<T> b = a;
                       for (int s = nsteps - 1, rr = 0; s >= 0; --s, ++rr)
                           reverse(b, ck + (size_t)s * n, ck + (size_t)(s + 1) * n, tdev + s, rr,
                                   cs);
                       return cudaGetLastError();
                   });
        if (r) return r;
    }
    for (int q = K == 1 ? -1 : nseg - 1; q >= 0; --q) {
        const int s0 = q * K, s1 = (q + 1) * K <= nsteps ? (q + 1) * K : nsteps;
        const int len = s1 - s0;
        ADJ_CHECK(cudaMemcpyAsync(ring, ck + (size_t)q * n, n * E, cudaMemcpyDeviceToDevice, st));
        ADJ_CHECK(cudaMemcpyAsync(tseg, tdev + s0, (len + 1) * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
        ADJ_CHECK(cudaMemcpyAsync(tsc, tign0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        r = replay(len == K ? 0 : 1, mix(key0, (unsigned long long)len),
                   [&](cudaStream_t cs) { return issue_segment(len, cs); });
        if (r) return r;
    }
    if (sizeof(T) == 4) {
        k_acc_final<<<grid, kAdjThreads, 0, st>>>(gm, (a.wind_grads ? 4 : 2) * n);
        ADJ_CHECK(cudaGetLastError());
    }
    if (g_u || g_v) {
        double *tmp = reinterpret_cast<double *>(ws + o_wind);
        double *gu = g_u ? g_u : tmp, *gv = g_v ? g_v : tmp + nu;
        // one warp per face
        const size_t wt = (nu + nv) * 32;
        const int wg = (int)((wt + kAdjThreads - 1) / kAdjThreads);
        k_adj_wind<T><<<wg, kAdjThreads, 0, st>>>(a, gun, gvn, gu, gv);
        ADJ_CHECK(cudaGetLastError());
    }
    if (g_mult)
        ADJ_CHECK(cudaMemcpyAsync(g_mult, gm, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (g_moist)
        ADJ_CHECK(cudaMemcpyAsync(g_moist, gM, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    ADJ_CHECK(cudaStreamSynchronize(st));
    return FIRE_OK;
}

}  // namespace
}  // namespace wf

extern "C" int fire_adjoint(fire_ctx *c, int nsteps, double dt, const void *wind_u_dev,
                            const void *wind_v_dev, const double *t_obs_dev, int ckpt_every,
                            double *J_host, double *g_mult_dev, double *g_moist_dev,
                            double *g_u_dev, double *g_v_dev) {
    if (!c || !wind_u_dev || !wind_v_dev || !t_obs_dev || !J_host || nsteps < 1 ||
        ckpt_every < 1 || !isfinite(dt) || !(dt > 0.0))
        return FIRE_ERR_ARG;
    wf::DeviceGuard dg(wf::ctx_device(c));
    int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
    double t;
    wf::ctx_info(c, &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t);
    const int K = ckpt_every < nsteps ? ckpt_every : nsteps;
    return prec == FIRE_FP64
               ? wf::run_adjoint<double>(c, nsteps, dt, wind_u_dev, wind_v_dev, t_obs_dev, nullptr,
                                         K, J_host, g_mult_dev, g_moist_dev, g_u_dev, g_v_dev)
               : wf::run_adjoint<float>(c, nsteps, dt, wind_u_dev, wind_v_dev, t_obs_dev, nullptr,
                                        K, J_host, g_mult_dev, g_moist_dev, g_u_dev, g_v_dev);
}

extern "C" int fire_adjoint_heat(fire_ctx *c, int nsteps, double dt, const void *wind_u_dev,
                                 const void *wind_v_dev, const double *q_obs_dev, int ckpt_every,
                                 double *J_host, double *g_mult_dev, double *g_moist_dev,
                                 double *g_u_dev, double *g_v_dev) {
    if (!c || !wind_u_dev || !wind_v_dev || !q_obs_dev || !J_host || nsteps < 1 ||
        ckpt_every < 1 || !isfinite(dt) || !(dt > 0.0))
        return FIRE_ERR_ARG;
    wf::DeviceGuard dg(wf::ctx_device(c));
    int prec, variant, nx, ny, srx, sry, kx, ky, ncls, cur;
    double t;
    wf::ctx_info(c, &prec, &variant, &nx, &ny, &srx, &sry, &kx, &ky, &ncls, &cur, &t);
    if (nx < 2 || ny < 2) return FIRE_ERR_ARG;
    const int K = ckpt_every < nsteps ? ckpt_every : nsteps;
    return prec == FIRE_FP64
               ? wf::run_adjoint<double>(c, nsteps, dt, wind_u_dev, wind_v_dev, nullptr, q_obs_dev,
                                         K, J_host, g_mult_dev, g_moist_dev, g_u_dev, g_v_dev)
               : wf::run_adjoint<float>(c, nsteps, dt, wind_u_dev, wind_v_dev, nullptr, q_obs_dev,
                                        K, J_host, g_mult_dev, g_moist_dev, g_u_dev, g_v_dev);
}
