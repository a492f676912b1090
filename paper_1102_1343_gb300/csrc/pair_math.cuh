// Arithmetic on pairs of values: the two fire-mesh columns a thread holds.
// FP32 uses the packed f32x2 instructions of sm_100 and later (one
// instruction for both columns); FP64 works element by element.  neg_rhs2 is
// the negated right-hand side of eq. (F-disc) for such a pair.
#pragma once

#include "fire_device.cuh"

namespace wf {

// ---------------------------------------------------------------------------
// pairs of values (the two columns of a lane)
// ---------------------------------------------------------------------------
template <typename T>
struct PairT;
template <>
struct PairT<float> {
    using t = float2;
};
template <>
struct PairT<double> {
    using t = double2;
};

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename V, typename T>
__device__ __forceinline__ V splat(T v) {
    return mk2(v, v);
}

__device__ __forceinline__ float max_val(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_val(double a, double b) { return fmax(a, b); }
// max of three (one three-input instruction in FP32)
__device__ __forceinline__ float max3_val(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double max3_val(double a, double b, double c) { return fmax(fmax(a, b), c); }

// unit vectors of two (cx, cy): Mth::unit on pairs
__device__ __forceinline__ void unit2(float2 cx, float2 cy, float2 &nx, float2 &ny) {
    const float2 n2 = fma2(cx, cx, mul2(cy, cy));
    const float2 r = make_float2(rsqrt_ftz(fmaxf(n2.x, Mth<float>::kNormMin)),
                                 rsqrt_ftz(fmaxf(n2.y, Mth<float>::kNormMin)));
    nx = mul2(cx, r);
    ny = mul2(cy, r);
}
__device__ __forceinline__ void unit2(double2 cx, double2 cy, double2 &nx, double2 &ny) {
    Mth<double>::unit(cx.x, cy.x, nx.x, ny.x);
    Mth<double>::unit(cx.y, cy.y, nx.y, ny.y);
}

// coefficients of eq. (spread-WRF-Fire) for the two columns
template <typename T>
struct WCoef {
    using V = typename PairT<T>::t;
    V S0, R0, b, c, d, e;
};

// Negated right-hand side G = -F of eq. (F-disc) for two columns (the
// arithmetic of rhs_vals on pairs): node values p, neighbours left / right /
// down / up, the grid constants 1/dx, 1/dy, 1/(2dx), 1/(2dy), eps as pairs,
// the coefficients, multiplier, node wind and terrain gradient of each
// column.  With the one-sided differences D-x = (p - pl)/dx and
// D+x = (pr - p)/dx formed as D-x and -D+x = (p - pr)/dx (likewise in y),
// Godunov's |D| = max(D-, -D+, 0) and the Laplacian -(D-x + (-D+x)) - (...)
// need no negated operand, and G = S (|grad psi| - eps Lap) =
// S (|grad psi| + eps (D-x - D+x + D-y - D+y)).
template <typename T>
__device__ __forceinline__ typename PairT<T>::t neg_rhs2(
    typename PairT<T>::t p, typename PairT<T>::t pl, typename PairT<T>::t pr,
    typename PairT<T>::t pd, typename PairT<T>::t pu, typename PairT<T>::t idx2,
    typename PairT<T>::t idy2, typename PairT<T>::t i2dx2, typename PairT<T>::t i2dy2,
    typename PairT<T>::t eps2, const WCoef<T> &co, typename PairT<T>::t m,
    typename PairT<T>::t un, typename PairT<T>::t vn, typename PairT<T>::t zx,
    typename PairT<T>::t zy) {
    using V = typename PairT<T>::t;
    const V dxm = mul2(sub2(p, pl), idx2), ndxp = mul2(sub2(p, pr), idx2);
    const V dym = mul2(sub2(p, pd), idy2), ndyp = mul2(sub2(p, pu), idy2);
    // Godunov (eq. Godunov): |D| = max(D-, -D+, 0) per direction
    V gx, gy;
    gx.x = max3_val(dxm.x, ndxp.x, T(0));
    gx.y = max3_val(dxm.y, ndxp.y, T(0));
    gy.x = max3_val(dym.x, ndyp.x, T(0));
    gy.y = max3_val(dym.y, ndyp.y, T(0));
    const V g2 = fma2(gx, gx, mul2(gy, gy));
    // central differences, zeroed at the rounding level of their values
    V ddx = sub2(pr, pl), ddy = sub2(pu, pd);
    const T z = Mth<T>::kGradZero;
    ddx.x = abs_val(ddx.x) <= z * (abs_val(pr.x) + abs_val(pl.x)) ? T(0) : ddx.x;
    ddx.y = abs_val(ddx.y) <= z * (abs_val(pr.y) + abs_val(pl.y)) ? T(0) : ddx.y;
    ddy.x = abs_val(ddy.x) <= z * (abs_val(pu.x) + abs_val(pd.x)) ? T(0) : ddy.x;
    ddy.y = abs_val(ddy.y) <= z * (abs_val(pu.y) + abs_val(pd.y)) ? T(0) : ddy.y;
    const V cx = mul2(ddx, i2dx2), cy = mul2(ddy, i2dy2);
    V nxv, nyv;
    unit2(cx, cy, nxv, nyv);
    const V U = fma2(un, nxv, mul2(vn, nyv));
    const V tp = fma2(zx, nxv, mul2(zy, nyv));
    // spread rate, eq. (spread-WRF-Fire)
    V Ue, tq, pw;
    Ue.x = min_val(max_val(U.x, T(0)), co.e.x);
    Ue.y = min_val(max_val(U.y, T(0)), co.e.y);
    tq.x = max_val(tp.x, T(0));
    tq.y = max_val(tp.y, T(0));
    pw.x = Mth<T>::pw(Ue.x, co.b.x);
    pw.y = Mth<T>::pw(Ue.y, co.b.y);
    V s = fma2(mul2(co.d, tq), tq, fma2(co.c, pw, co.R0));
    s.x = max_val(s.x, co.S0.x);
    s.y = max_val(s.y, co.S0.y);
    const V S = mul2(m, s);
    const V nlap = add2(add2(dxm, ndxp), add2(dym, ndyp));  // -Lap
    V grad;
    grad.x = Mth<T>::sqr(g2.x);
    grad.y = Mth<T>::sqr(g2.y);
    // S |grad| - eps S Lap
    return mul2(S, fma2(eps2, nlap, grad));
}

// the six coefficients of two classes from a per-class table of 8 values
// (S0 R0 b c d e Tf Hs): 16-byte shared loads in FP32
template <typename T>
__device__ __forceinline__ void coef_pair(const T *lut, int cls0, int cls1, WCoef<T> &co) {
    const T *l0 = lut + cls0 * 8, *l1 = lut + cls1 * 8;
    if constexpr (sizeof(T) == 4) {
        const float4 a0 = *reinterpret_cast<const float4 *>(l0);
        const float4 b0 = *reinterpret_cast<const float4 *>(l0 + 4);
        const float4 a1 = *reinterpret_cast<const float4 *>(l1);
        const float4 b1 = *reinterpret_cast<const float4 *>(l1 + 4);
        co.S0 = mk2(a0.x, a1.x);
        co.R0 = mk2(a0.y, a1.y);
        co.b = mk2(a0.z, a1.z);
        co.c = mk2(a0.w, a1.w);
        co.d = mk2(b0.x, b1.x);
        co.e = mk2(b0.y, b1.y);
    } else {
        co.S0 = mk2(l0[0], l1[0]);
        co.R0 = mk2(l0[1], l1[1]);
        co.b = mk2(l0[2], l1[2]);
        co.c = mk2(l0[3], l1[3]);
        co.d = mk2(l0[4], l1[4]);
        co.e = mk2(l0[5], l1[5]);
    }
}

// the same from a table of the six coefficients with each value twice
// (S0 S0 R0 R0 b b c c d d e e, 16-byte aligned rows): in FP32 the three
// 16-byte loads of class cls0 give both columns' pairs, and only where a
// column of the warp has a class cls1 != cls0 (a fuel boundary) are the
// second components reloaded.  Called by all 32 lanes of a warp.
template <typename T>
__device__ __forceinline__ void coef_pair_dup(const T *lut2, int cls0, int cls1, WCoef<T> &co) {
    const T *l0 = lut2 + cls0 * 12;
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(l0);
        const float4 b = *reinterpret_cast<const float4 *>(l0 + 4);
        const float4 c = *reinterpret_cast<const float4 *>(l0 + 8);
        co.S0 = mk2(a.x, a.y);
        co.R0 = mk2(a.z, a.w);
        co.b = mk2(b.x, b.y);
        co.c = mk2(b.z, b.w);
        co.d = mk2(c.x, c.y);
        co.e = mk2(c.z, c.w);
    } else {
        co.S0 = splat<typename PairT<T>::t>(l0[0]);
        co.R0 = splat<typename PairT<T>::t>(l0[2]);
        co.b = splat<typename PairT<T>::t>(l0[4]);
        co.c = splat<typename PairT<T>::t>(l0[6]);
        co.d = splat<typename PairT<T>::t>(l0[8]);
        co.e = splat<typename PairT<T>::t>(l0[10]);
    }
    if (__any_sync(0xffffffffu, cls1 != cls0)) {
        if (cls1 != cls0) {
            const T *l1 = lut2 + cls1 * 12;
            co.S0.y = l1[0];
            co.R0.y = l1[2];
            co.b.y = l1[4];
            co.c.y = l1[6];
            co.d.y = l1[8];
            co.e.y = l1[10];
        }
    }
}

// Fuel fraction (Sect. 3.3, the subcell scheme of cell_fraction_vals) of two
// cells at once, the two columns of a lane: q[b][h], e[b][h] the 3x3
// neighbourhoods of psi^{n+1} and t - t_i (0 where psi >= 0) of both cells
// as pairs, Tf the two burn times.  The sums, means and products are packed
// f32x2; the compatibility tests, |psi|, divisions and exponentials stay per
// element.  Each cell must have a node with psi < 0 in its neighbourhood
// (the caller keeps F = 1 for the others).
__device__ __forceinline__ float2 cell_fraction_pair(const float2 (&q)[3][3],
                                                     const float2 (&e)[3][3], float2 Tf) {
    const float2 h = make_float2(0.5f, 0.5f), qq = make_float2(0.25f, 0.25f);
    // vertices: centre, edge midpoints W E S N, corners SW SE NW NE
    const float2 pC = q[1][1];
    const float2 pW = mul2(h, add2(q[1][0], q[1][1])), pE = mul2(h, add2(q[1][1], q[1][2]));
    const float2 pS = mul2(h, add2(q[0][1], q[1][1])), pN = mul2(h, add2(q[1][1], q[2][1]));
    float2 dW = mul2(h, add2(e[1][0], e[1][1])), dE = mul2(h, add2(e[1][1], e[1][2]));
    float2 dS = mul2(h, add2(e[0][1], e[1][1])), dN = mul2(h, add2(e[1][1], e[2][1]));
    const float2 pSW = mul2(qq, add2(add2(add2(q[0][0], q[0][1]), q[1][0]), q[1][1]));
    const float2 pSE = mul2(qq, add2(add2(add2(q[0][1], q[0][2]), q[1][1]), q[1][2]));
    const float2 pNW = mul2(qq, add2(add2(add2(q[1][0], q[1][1]), q[2][0]), q[2][1]));
    const float2 pNE = mul2(qq, add2(add2(add2(q[1][1], q[1][2]), q[2][1]), q[2][2]));
    float2 dSW = mul2(qq, add2(add2(add2(e[0][0], e[0][1]), e[1][0]), e[1][1]));
    float2 dSE = mul2(qq, add2(add2(add2(e[0][1], e[0][2]), e[1][1]), e[1][2]));
    float2 dNW = mul2(qq, add2(add2(add2(e[1][0], e[1][1]), e[2][0]), e[2][1]));
    float2 dNE = mul2(qq, add2(add2(add2(e[1][1], e[1][2]), e[2][1]), e[2][2]));
    // compatibility at the vertices: t_i := t where psi >= 0
    auto compat = [](float2 p, float2 d) {
        return make_float2(p.x >= 0.0f ? 0.0f : d.x, p.y >= 0.0f ? 0.0f : d.y);
    };
    const float2 dC = compat(pC, e[1][1]);
    dW = compat(pW, dW);
    dE = compat(pE, dE);
    dS = compat(pS, dS);
    dN = compat(pN, dN);
    dSW = compat(pSW, dSW);
    dSE = compat(pSE, dSE);
    dNW = compat(pNW, dNW);
    dNE = compat(pNE, dNE);
    const float2 k = make_float2(-0.25f / Tf.x, -0.25f / Tf.y);
    // burned fraction of one subcell, eqs. (approx-area), (approx-fraction)
    auto sub = [&](float2 p0, float2 p1, float2 p2, float2 p3, float2 d0, float2 d1, float2 d2,
                   float2 d3) {
        const float2 sp = add2(add2(add2(p0, p1), p2), p3);
        const float sax = ((fabsf(p0.x) + fabsf(p1.x)) + fabsf(p2.x)) + fabsf(p3.x);
        const float say = ((fabsf(p0.y) + fabsf(p1.y)) + fabsf(p2.y)) + fabsf(p3.y);
        // beta = (1 - sum / sum of |.|) / 2 as Mth<float>::one_minus_div
        // forms it, 0 where every vertex value is 0
        const float2 ns = make_float2(sax > 0.0f ? -sp.x : -1.0f, say > 0.0f ? -sp.y : -1.0f);
        const float2 rc = make_float2(sax > 0.0f ? rcp_ftz(sax) : 1.0f,
                                      say > 0.0f ? rcp_ftz(say) : 1.0f);
        const float2 beta = mul2(h, fma2(ns, rc, make_float2(1.0f, 1.0f)));
        const float2 s = mul2(add2(add2(add2(d0, d1), d2), d3), k);
        const float2 ex = make_float2(__expf(s.x), __expf(s.y));
        return mul2(beta, sub2(make_float2(1.0f, 1.0f), ex));
    };
    const float2 bSW = sub(pC, pW, pS, pSW, dC, dW, dS, dSW);
    const float2 bSE = sub(pC, pE, pS, pSE, dC, dE, dS, dSE);
    const float2 bNW = sub(pC, pW, pN, pNW, dC, dW, dN, dNW);
    const float2 bNE = sub(pC, pE, pN, pNE, dC, dE, dN, dNE);
    return fma2(make_float2(-0.25f, -0.25f), add2(add2(add2(bSW, bSE), bNW), bNE),
                make_float2(1.0f, 1.0f));
}

}  // namespace wf
