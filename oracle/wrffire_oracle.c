/*
 * Plain FP64 CPU oracle of the WRF-Fire fire-model step
 * (Mandel, Beezley & Kochanski, "Coupled atmosphere-wildland fire modeling
 * with WRF-Fire version 3.3").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path
 * is checked against.  Only the tests, the smoke check of the entry module
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and it is deliberately
 * slow: one loop per step of the method, in the paper's order, no blocking,
 * no fusion.  Build with -O2 -ffp-contract=off so that every product and
 * sum is rounded separately.
 *
 * Each function cites the section / equation / table it follows.  Where the
 * paper is silent, garbled or ambiguous the reading taken is stated in the
 * comment ("Reading:").
 *
 * Parity status: every function below is pinned by a CPU test against a
 * closed form, an exactness claim of the paper, an invariant or a brute
 * force computation, except where its comment says "parity unpinned".
 *
 * Threads: built with OpenMP, the per-node loops of one step run over rows
 * in parallel (orc_set_threads; one thread unless asked).  Each such loop
 * computes every output value alone with the same operations in the same
 * order, and the two status flags are OR-reduced, so the results do not
 * depend on the number of threads.
 *
 * Layout conventions: fire mesh nodes (cell centres) are indexed (i, j),
 * i = 0..nx-1 along x, j = 0..ny-1 along y, stored row-major a[j*nx + i];
 * node (i, j) sits at ((i+1/2) dx, (j+1/2) dy).  The atmospheric mesh has
 * nxa x nya cells; nx = srx*nxa, ny = sry*nya.  The wind is given on the
 * staggered C-grid of Sect. "Domain, grids, and nodes": u[J*(nxa+1) + I]
 * at x-faces (I*DX, (J+1/2)*DY), v[J*nxa + I] at y-faces ((I+1/2)*DX, J*DY).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-node loops; returns the count in effect (1 without
 * OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n < 1) n = 1;
    omp_set_num_threads(n);
    return n;
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Fuel properties (Table 1), one class = 13 doubles in this order.    */
/* ------------------------------------------------------------------ */
enum {
    FC_WINDRF = 0,   /* a: wind reduction from 6.1 m to midflame height */
    FC_WEIGHT,       /* w: fuel weight (s); or T_f directly, see next */
    FC_WEIGHT_IS_TF, /* nonzero: FC_WEIGHT holds the burn time T_f (s) */
    FC_FGI,          /* w_l: total fuel load (kg m^-2) */
    FC_DEPTH,        /* delta_m: fuel depth (m) */
    FC_SAVR,         /* sigma: surface-area-to-volume ratio (1/m) */
    FC_MX,           /* M_x: moisture content of extinction */
    FC_DENS,         /* rho_P: ovendry particle density (kg m^-3) */
    FC_ST,           /* S_T: total mineral content */
    FC_SE,           /* S_E: effective mineral content */
    FC_H,            /* h: heat content of dry fuel (J/kg) */
    FC_MF,           /* M_f: fuel particle moisture content */
    FC_CHAPARRAL,    /* nonzero: chaparral rule, eq. (chapparal) */
    FC_N
};

/* Coefficient vector of eq. (spread-WRF-Fire) plus the burn time and the
 * two heat factors of eqs. (sensible-heat-flux), (latent-heat-flux). */
enum { CO_S0 = 0, CO_R0, CO_B, CO_C, CO_D, CO_E, CO_TF, CO_HS, CO_HQ, CO_N };

/* Unit conversions to the BTU-lb-ft-min system of Table 2. */
#define M_PER_FT   0.3048
#define KG_PER_LB  0.45359237
#define J_PER_BTU  1055.05585262
#define LATENT_L   2.5e6          /* L, J/kg, Sect. "Fuel burned and heat released" */
#define WIND_MAX   30.0           /* CAWFE wind limit, caption of Table 2 */
#define ORC_GRAD_ZERO 1e-9        /* relative rounding level of a central difference */


/* Rothermel quantities that do not depend on wind or slope (Table 2).
 * Returns R0 in ft/min and the wind/slope factors' ingredients.
 * Reading (garbles in Table 2):
 *   - Gamma_max = sigma^1.5/(495 + 0.0594 sigma^1.5): Rothermel's Eq. (36)
 *     constant is 0.0594; the table prints 0.594.
 *   - Q_ig = 250 + 1116 M_f: Rothermel's Eq. (12); the table's "250 beta"
 *     is a typesetting slip.
 *   - phi_W = C U_a^B (beta/beta_op)^(-E) with B = 0.02526 sigma^0.54 and
 *     beta_op = 3.348 sigma^(-0.8189) (Rothermel Eqs. 47-49, 37); the table
 *     leaves B and beta_op undefined.
 *   - eta_M is clamped to [0, 1] (zero when M_f >= M_x): silent in the paper.
 *   - a class with no fuel (w_l <= 0) does not spread: silent in the paper. */
typedef struct {
    double R0_ftmin, B, C, E, beta, beta_op;
    int nofuel;
    /* every intermediate of the chain, English units (for the pins) */
    double sigma, wl, depth, rho_p, h, w0, rho_b, A, Gmax, Gamma, wn, etaM, etaS, IR, xi,
           epsh, Qig;
} orc_rothermel_parts;

static orc_rothermel_parts rothermel_parts(const double *fc, double Mf)
{
    orc_rothermel_parts p;
    memset(&p, 0, sizeof p);
    if (!(fc[FC_FGI] > 0.0)) { p.nofuel = 1; return p; }
    /* metric -> English (caption of Table 2) */
    double sigma  = fc[FC_SAVR] * M_PER_FT;                       /* 1/ft */
    double wl     = fc[FC_FGI] * (M_PER_FT * M_PER_FT) / KG_PER_LB; /* lb/ft^2 */
    double depth  = fc[FC_DEPTH] / M_PER_FT;                      /* ft */
    double rho_p  = fc[FC_DENS] * (M_PER_FT * M_PER_FT * M_PER_FT) / KG_PER_LB; /* lb/ft^3 */
    double h      = fc[FC_H] * KG_PER_LB / J_PER_BTU;             /* BTU/lb */
    double Mx     = fc[FC_MX];
    double ST     = fc[FC_ST];
    double SE     = fc[FC_SE];

    double w0     = wl / (1.0 + Mf);                 /* net of moisture (CAWFE) */
    double rho_b  = w0 / depth;                      /* Eq. (40) */
    double beta   = rho_b / rho_p;                   /* Eq. (31) */
    double beta_op = 3.348 * pow(sigma, -0.8189);    /* Eq. (37) */
    double A      = 1.0 / (4.77 * pow(sigma, 0.1) - 7.27);          /* Eq. (39) */
    double s15    = pow(sigma, 1.5);
    double Gmax   = s15 / (495.0 + 0.0594 * s15);    /* Eq. (36), reading */
    double ratio  = beta / beta_op;
    double Gamma  = Gmax * pow(ratio, A) * exp(A * (1.0 - ratio));  /* Eq. (36) */
    double wn     = w0 / (1.0 + ST);                 /* Eq. (24) as printed */
    double rm     = Mf / Mx;
    double etaM   = 1.0 - 2.59 * rm + 5.11 * rm * rm - 3.52 * rm * rm * rm; /* Eq. (29) */
    if (rm >= 1.0 || etaM < 0.0) etaM = 0.0;
    if (etaM > 1.0) etaM = 1.0;
    double etaS   = 0.174 * pow(SE, -0.19);          /* Eq. (30) */
    double IR     = Gamma * wn * h * etaM * etaS;    /* Eq. (52) */
    double xi     = exp((0.792 + 0.681 * sqrt(sigma)) * (beta + 0.1))
                    / (192.0 + 0.2595 * sigma);      /* Eq. (42) */
    double epsh   = exp(-138.0 / sigma);             /* Eq. (14) */
    double Qig    = 250.0 + 1116.0 * Mf;             /* Eq. (12), reading */
    p.R0_ftmin    = IR * xi / (rho_b * epsh * Qig);  /* Eq. (52) */
    p.C           = 7.47 * exp(-0.133 * pow(sigma, 0.55));  /* Eq. (48) */
    p.B           = 0.02526 * pow(sigma, 0.54);      /* Rothermel Eq. (49) */
    p.E           = 0.715 * exp(-3.59e-4 * sigma);   /* Eq. (50) */
    p.beta        = beta;
    p.beta_op     = beta_op;
    p.sigma = sigma; p.wl = wl; p.depth = depth; p.rho_p = rho_p; p.h = h; p.w0 = w0;
    p.rho_b = rho_b; p.A = A; p.Gmax = Gmax; p.Gamma = Gamma; p.wn = wn; p.etaM = etaM;
    p.etaS = etaS; p.IR = IR; p.xi = xi; p.epsh = epsh; p.Qig = Qig;
    return p;
}

/* The intermediates of the Table 2 chain for one class at moisture Mf (< 0:
 * the class moisture), English units (BTU-lb-ft-min), in this order:
 * sigma (1/ft), w_l (lb/ft^2), delta (ft), rho_P (lb/ft^3), h (BTU/lb), w_0,
 * rho_b (lb/ft^3), beta, beta_op, A, Gamma_max, Gamma (1/min), w_n, eta_M,
 * eta_S, I_R (BTU/ft^2/min), xi, epsilon, Q_ig (BTU/lb), R0 (ft/min), B, C,
 * E, nofuel -- 24 values.  Bookkeeping only: the values rothermel_parts
 * computes, returned so that tests can pin each step. */
void orc_rothermel_intermediates(const double *fc, double Mf, double *out)
{
    if (Mf < 0.0) Mf = fc[FC_MF];
    orc_rothermel_parts p = rothermel_parts(fc, Mf);
    double v[24] = {p.sigma, p.wl, p.depth, p.rho_p, p.h, p.w0, p.rho_b, p.beta, p.beta_op,
                    p.A, p.Gmax, p.Gamma, p.wn, p.etaM, p.etaS, p.IR, p.xi, p.epsh, p.Qig,
                    p.R0_ftmin, p.B, p.C, p.E, (double)p.nofuel};
    for (int k = 0; k < 24; ++k) out[k] = v[k];
}

/* Direct evaluation of eq. (spread): S = R0 (1 + phi_W + phi_S), in m/s,
 * with the CAWFE limits of the caption of Table 2 (0 <= U <= 30 m/s,
 * tan(phi) >= 0) and the chaparral rule eq. (chapparal).  Mf < 0 means
 * "use the class moisture". */
double orc_rothermel_rate(const double *fc, double Mf, double U, double tanphi)
{
    if (Mf < 0.0) Mf = fc[FC_MF];
    if (fc[FC_CHAPARRAL] != 0.0) {
        double s = 1.2974 * U;
        if (s < 0.03333) s = 0.03333;
        if (s > 6.0) s = 6.0;
        return s;
    }
    orc_rothermel_parts p = rothermel_parts(fc, Mf);
    if (p.nofuel) return 0.0;
    double Ul = U;
    if (Ul < 0.0) Ul = 0.0;
    if (Ul > WIND_MAX) Ul = WIND_MAX;
    double tp = tanphi > 0.0 ? tanphi : 0.0;
    double Ua = fc[FC_WINDRF] * Ul * (60.0 / M_PER_FT);  /* U_a = a U, ft/min */
    double phiW = p.C * pow(Ua, p.B) * pow(p.beta / p.beta_op, -p.E);  /* Eq. (47) */
    double phiS = 5.275 * pow(p.beta, -0.3) * tp * tp;   /* Eq. (51) */
    return p.R0_ftmin * (1.0 + phiW + phiS) * (M_PER_FT / 60.0);
}

/* Coefficients of eq. (spread-WRF-Fire), SI units (U in m/s, S in m/s),
 * the burn time T_f (Sect. "Fuel burned and heat released") and the heat
 * factors H_s = w_l h/(1+M_f) and H_q = (M_f+0.56)/(1+M_f) L w_l of
 * eqs. (sensible-heat-flux), (latent-heat-flux).
 * Reading of the coefficient mapping (the paper gives the form only):
 *   R0 := R0 [m/s], b := B, c := R0 C (196.85 a)^B (beta/beta_op)^(-E),
 *   d := R0 5.275 beta^(-0.3), e := 30 m/s, S0 := 0;
 *   chaparral: S0 = 0.03333, R0 = 0, b = 1, c = 1.2974, d = 0, e = 6/1.2974.
 * Mf < 0 means "use the class moisture". */
void orc_fuel_coefficients(const double *fc, double Mf, double *co)
{
    if (Mf < 0.0) Mf = fc[FC_MF];
    for (int k = 0; k < CO_N; ++k) co[k] = 0.0;
    /* burn time: 0.6^((t-ti)/600 * 1000/w) = exp(-(t-ti)/T_f) */
    if (fc[FC_WEIGHT_IS_TF] != 0.0) co[CO_TF] = fc[FC_WEIGHT];
    else co[CO_TF] = -600.0 * fc[FC_WEIGHT] / (1000.0 * log(0.6));
    co[CO_HS] = fc[FC_FGI] * fc[FC_H] / (1.0 + Mf);
    co[CO_HQ] = (Mf + 0.56) / (1.0 + Mf) * LATENT_L * fc[FC_FGI];
    if (fc[FC_CHAPARRAL] != 0.0) {
        co[CO_S0] = 0.03333;
        co[CO_R0] = 0.0;
        co[CO_B]  = 1.0;
        co[CO_C]  = 1.2974;
        co[CO_D]  = 0.0;
        co[CO_E]  = 6.0 / 1.2974;
        return;
    }
    orc_rothermel_parts p = rothermel_parts(fc, Mf);
    co[CO_E] = WIND_MAX;
    co[CO_B] = 1.0;
    if (p.nofuel) return;
    double R0 = p.R0_ftmin * (M_PER_FT / 60.0);
    co[CO_R0] = R0;
    co[CO_B]  = p.B;
    co[CO_C]  = R0 * p.C * pow(fc[FC_WINDRF] * (60.0 / M_PER_FT), p.B)
                   * pow(p.beta / p.beta_op, -p.E);
    co[CO_D]  = R0 * 5.275 * pow(p.beta, -0.3);
}

/* Eq. (spread-WRF-Fire): S = max{S0, R0 + c min{e, max{0,U}}^b + d max{0,tan phi}^2}. */
double orc_spread_rate(const double *co, double U, double tanphi)
{
    double Up = U > 0.0 ? U : 0.0;
    double Ue = Up < co[CO_E] ? Up : co[CO_E];
    double tp = tanphi > 0.0 ? tanphi : 0.0;
    double s = co[CO_R0] + co[CO_C] * pow(Ue, co[CO_B]) + co[CO_D] * tp * tp;
    return s > co[CO_S0] ? s : co[CO_S0];
}

/* Per-node coefficients: class table [ncls][13], class map, optional per-node
 * moisture (NULL: the class moisture).  Output [n][9]. */
void orc_node_coefficients(const double *classes, int ncls, const unsigned char *fuel,
                           const double *moisture, long n, double *co)
{
    for (long k = 0; k < n; ++k) {
        int c = fuel[k];
        if (c >= ncls) c = ncls - 1;
        orc_fuel_coefficients(classes + (long)c * FC_N,
                              moisture ? moisture[k] : -1.0, co + k * CO_N);
    }
}

/* ------------------------------------------------------------------ */
/* Level-set core (Sect. "Fire propagation by the level-set method").  */
/* ------------------------------------------------------------------ */

/* Godunov upwind selection, eq. (Godunov), cases tested in the printed
 * order.  Reading: on a tie |D-| = |D+| in the last case, D- is taken
 * (both printed branches give the same magnitude). */
double orc_godunov(double dm, double dp)
{
    if (dm <= 0.0 && dp <= 0.0) return dp;
    if (dm >= 0.0 && dp >= 0.0) return dm;
    if (dm <= 0.0 && dp >= 0.0) return 0.0;
    if (fabs(dm) >= fabs(dp)) return dm;
    return dp;
}

/* One extrapolated ghost value (Sect. level set, boundary): the node beyond
 * the boundary gets max{p0 + (p0 - p1), p0, p1}, p0 the last node, p1 the
 * one before it. */
static double ghost(double p0, double p1)
{
    double g = p0 + (p0 - p1);
    if (p0 > g) g = p0;
    if (p1 > g) g = p1;
    return g;
}

/* Extend a field by one layer of ghost nodes.  ext is (nx+2) x (ny+2),
 * ext[(j+1)*(nx+2) + (i+1)] = a[j*nx + i].  Reading of "similarly in the
 * other cases": the x direction first (ghost columns for every real row),
 * then the y direction over the extended rows (this fills the corners).
 * Requires nx >= 2 and ny >= 2. */
void orc_extend(int nx, int ny, const double *a, double *ext)
{
    int W = nx + 2;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            ext[(j + 1) * W + (i + 1)] = a[j * nx + i];
    for (int j = 0; j < ny; ++j) {
        double *row = ext + (j + 1) * W;
        row[0]      = ghost(row[1], row[2]);
        row[nx + 1] = ghost(row[nx], row[nx - 1]);
    }
    for (int i = 0; i < W; ++i) {
        ext[i]                = ghost(ext[W + i], ext[2 * W + i]);
        ext[(ny + 1) * W + i] = ghost(ext[ny * W + i], ext[(ny - 1) * W + i]);
    }
}

/* Horizontal bilinear interpolation of the staggered wind to the fire-mesh
 * nodes (Sect. "Coupling", last paragraph of the wind interpolation).
 * Reading: beyond the outermost u-rows (y) and v-columns (x) the value of
 * the edge row/column is used (constant extension). */
static void interp_weights(double f, int n, int *k0, int *k1, double *w)
{
    /* f is a coordinate in index units on points 0..n-1 */
    if (f < 0.0) f = 0.0;
    if (f > (double)(n - 1)) f = (double)(n - 1);
    int k = (int)floor(f);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    if (n == 1) { *k0 = 0; *k1 = 0; *w = 0.0; return; }
    *k0 = k;
    *k1 = k + 1;
    *w = f - (double)k;
}

void orc_wind_at_nodes(int nxa, int nya, int srx, int sry,
                       const double *u, const double *v, double *un, double *vn)
{
    int nx = nxa * srx, ny = nya * sry;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double xa = ((double)i + 0.5) / (double)srx;  /* atmos index units */
            double ya = ((double)j + 0.5) / (double)sry;
            int i0, i1, j0, j1;
            double wx, wy;
            /* u: points at (I, J+1/2), I = 0..nxa, J = 0..nya-1 */
            interp_weights(xa, nxa + 1, &i0, &i1, &wx);
            interp_weights(ya - 0.5, nya, &j0, &j1, &wy);
            const double *ur0 = u + (long)j0 * (nxa + 1);
            const double *ur1 = u + (long)j1 * (nxa + 1);
            un[(long)j * nx + i] = (1.0 - wy) * ((1.0 - wx) * ur0[i0] + wx * ur0[i1])
                                 + wy * ((1.0 - wx) * ur1[i0] + wx * ur1[i1]);
            /* v: points at (I+1/2, J), I = 0..nxa-1, J = 0..nya */
            interp_weights(xa - 0.5, nxa, &i0, &i1, &wx);
            interp_weights(ya, nya + 1, &j0, &j1, &wy);
            const double *vr0 = v + (long)j0 * nxa;
            const double *vr1 = v + (long)j1 * nxa;
            vn[(long)j * nx + i] = (1.0 - wy) * ((1.0 - wx) * vr0[i0] + wx * vr0[i1])
                                 + wy * ((1.0 - wx) * vr1[i0] + wx * vr1[i1]);
        }
    }
}

/* Right-hand side of eq. (F-disc) at every node, from the ghost-extended
 * level-set function ext ((nx+2) x (ny+2)).
 *   - one-sided differences D+-x, D+-y and the Godunov selection eq. (Godunov);
 *   - the normal n from central differences (paragraph after eq. Godunov),
 *     n = 0 where the central gradient vanishes (reading: silent).  Reading:
 *     a central difference psi_{i+1} - psi_{i-1} at the rounding level of its
 *     two values (|diff| <= 1e-9 (|psi_{i+1}| + |psi_{i-1}|)) counts as zero,
 *     so that rounding noise at a symmetric point does not pick a direction
 *     for n (the spread rate, and through the viscosity the level set, jumps
 *     with that direction);
 *   - U = wind . n, tan(phi) = grad z . n, S from eq. (spread-WRF-Fire),
 *     times the optional per-node spread multiplier m;
 *   - the scaled Laplacian D+x - D-x + D+y - D-y;
 *   - Reading of the viscosity units: F = -S |grad psi| + eps S Lap~(psi).
 *     The scaled Laplacian is dimensionless, so the speed S makes the term a
 *     speed, consistent with calling eps "scale-free". */
void orc_rhs(int nx, int ny, double dx, double dy, double eps,
             const double *ext, const double *co, const double *mult,
             const double *un, const double *vn,
             const double *dzdx, const double *dzdy, double *F)
{
    int W = nx + 2;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            const double *e = ext + (j + 1) * W + (i + 1);
            double p = e[0], pl = e[-1], pr = e[1], pd = e[-W], pu = e[W];
            double dxm = (p - pl) / dx, dxp = (pr - p) / dx;
            double dym = (p - pd) / dy, dyp = (pu - p) / dy;
            double gx = orc_godunov(dxm, dxp);
            double gy = orc_godunov(dym, dyp);
            double ax = pr - pl, ay = pu - pd;
            if (fabs(ax) <= ORC_GRAD_ZERO * (fabs(pr) + fabs(pl))) ax = 0.0;
            if (fabs(ay) <= ORC_GRAD_ZERO * (fabs(pu) + fabs(pd))) ay = 0.0;
            double cx = ax / (2.0 * dx);
            double cy = ay / (2.0 * dy);
            double cn = sqrt(cx * cx + cy * cy);
            double nxv = 0.0, nyv = 0.0;
            if (cn > 0.0) { nxv = cx / cn; nyv = cy / cn; }
            double U = un[k] * nxv + vn[k] * nyv;
            double tanphi = dzdx[k] * nxv + dzdy[k] * nyv;
            double S = orc_spread_rate(co + k * CO_N, U, tanphi);
            if (mult) S = mult[k] * S;
            double lap = (dxp - dxm) + (dyp - dym);
            double grad = sqrt(gx * gx + gy * gy);
            F[k] = -S * grad + eps * S * lap;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Ignition (Sect. "Ignition").                                        */
/* ------------------------------------------------------------------ */

/* One ignition: 10 doubles {ax, ay, bx, by, t_g, r_g, S_g, vx, vy, t_h}.
 * S_g > 0, v = 0: the fire grows from the segment [a, b] at S_g until r_g is
 * reached, eqs. (ignition-lfn), (ignition-min); active at the start of
 * every step with t_g <= t <= t_g + r_g/S_g; newly ignited nodes get the
 * arrival time t_g + dist/S_g.
 * S_g > 0, v != 0: the drip torch of Sect. "Ignition": a torch leaves a at
 * t_g with velocity v until t_h, the ignition line at t is the segment
 * [a, a + v (min{t, t_h} - t_g)] (b is not used) and psi_g = dist - min{r_g,
 * S_g (t - t_g)}, applied at every step start with t_g <= t <= t_h +
 * r_g/S_g.  Reading of "the arrival time of the fire at the spread rate S_g
 * from the nearest point on the ignition segment": the fire at the nearest
 * point p starts when the torch lays p, at t_p = t_g + s (min{t, t_h} -
 * t_g) for p = a + s (b(t) - a), and reaches the node dist/S_g later; a node
 * psi_g covers at step start t is burning by t, so its time is min{t, t_p +
 * dist/S_g} (with v = 0, t_p = t_g: the fixed segment's t_g + dist/S_g).
 * S_g <= 0: reading for an instantaneous ignition of radius r_g (the earlier
 * mechanism the section describes): applied once, at the first step start
 * t >= t_g (or at initialisation when t_g <= 0), with ignition time t_g. */
enum { IG_AX = 0, IG_AY, IG_BX, IG_BY, IG_TG, IG_RG, IG_SG, IG_VX, IG_VY, IG_TH, IG_N };

static int is_drip(const double *g)
{
    return g[IG_SG] > 0.0 && (g[IG_VX] != 0.0 || g[IG_VY] != 0.0);
}

static double dist_to_segment(double x, double y, const double *g)
{
    double dxs = g[IG_BX] - g[IG_AX], dys = g[IG_BY] - g[IG_AY];
    double qx = x - g[IG_AX], qy = y - g[IG_AY];
    double L2 = dxs * dxs + dys * dys;
    double s = 0.0;
    if (L2 > 0.0) {
        s = (qx * dxs + qy * dys) / L2;
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
    }
    double rx = qx - s * dxs, ry = qy - s * dys;
    return sqrt(rx * rx + ry * ry);
}

/* Apply one segment at step start t: psi := min(psi, psi_g), eq.
 * (ignition-min); t_i of newly ignited nodes (psi > 0 >= psi_g, t_i not yet
 * set) := arrival time.  Reading: a node's ignition time is set once, at its
 * first ignition, and never overwritten. */
static void apply_segment(int nx, int ny, double dx, double dy, const double *g,
                          double t, double *psi, double *tign)
{
    if (is_drip(g)) {
        /* the drip torch's segment and radius at t (Sect. "Ignition") */
        double seg[IG_N];
        for (int k = 0; k < IG_N; ++k) seg[k] = g[k];
        double tt = t < g[IG_TH] ? t : g[IG_TH];
        seg[IG_BX] = g[IG_AX] + g[IG_VX] * (tt - g[IG_TG]);
        seg[IG_BY] = g[IG_AY] + g[IG_VY] * (tt - g[IG_TG]);
        double R = g[IG_SG] * (t - g[IG_TG]);
        if (R > g[IG_RG]) R = g[IG_RG];
        double dxs = seg[IG_BX] - seg[IG_AX], dys = seg[IG_BY] - seg[IG_AY];
        double L2 = dxs * dxs + dys * dys;
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                long k = (long)j * nx + i;
                double x = ((double)i + 0.5) * dx, y = ((double)j + 0.5) * dy;
                double d = dist_to_segment(x, y, seg);
                double pg = d - R;
                if (psi[k] > 0.0 && pg <= 0.0 && isinf(tign[k])) {
                    /* parameter of the nearest point, as in dist_to_segment */
                    double sp = 0.0;
                    if (L2 > 0.0) {
                        sp = ((x - seg[IG_AX]) * dxs + (y - seg[IG_AY]) * dys) / L2;
                        if (sp < 0.0) sp = 0.0;
                        if (sp > 1.0) sp = 1.0;
                    }
                    double tp = g[IG_TG] + sp * (tt - g[IG_TG]);
                    double ta = tp + d / g[IG_SG];
                    tign[k] = ta < t ? ta : t;
                }
                if (pg < psi[k]) psi[k] = pg;
            }
        }
        return;
    }
    int instant = !(g[IG_SG] > 0.0);
    double rho = instant ? g[IG_RG] : g[IG_SG] * (t - g[IG_TG]);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            double x = ((double)i + 0.5) * dx, y = ((double)j + 0.5) * dy;
            double d = dist_to_segment(x, y, g);
            double pg = d - rho;
            if (psi[k] > 0.0 && pg <= 0.0 && isinf(tign[k]))
                tign[k] = instant ? g[IG_TG] : g[IG_TG] + d / g[IG_SG];
            if (pg < psi[k]) psi[k] = pg;
        }
    }
}

/* Step 1 of the fire step (Sect. "Coupling", list item 1): apply every
 * active ignition in list order.  applied[] records instantaneous ignitions
 * already done. */
void orc_ignite(int nx, int ny, double dx, double dy, const double *ign, int n_ign,
                unsigned char *applied, double t, double *psi, double *tign)
{
    for (int q = 0; q < n_ign; ++q) {
        const double *g = ign + q * IG_N;
        if (!(g[IG_SG] > 0.0)) {
            if (!applied[q] && g[IG_TG] <= t) {
                apply_segment(nx, ny, dx, dy, g, t, psi, tign);
                applied[q] = 1;
            }
        } else if (is_drip(g)) {
            if (g[IG_TG] <= t && t <= g[IG_TH] + g[IG_RG] / g[IG_SG])
                apply_segment(nx, ny, dx, dy, g, t, psi, tign);
        } else if (g[IG_TG] <= t && t <= g[IG_TG] + g[IG_RG] / g[IG_SG]) {
            apply_segment(nx, ny, dx, dy, g, t, psi, tign);
        }
    }
}

/* Initial state (Sect. "Ignition", first paragraph): psi = psi_far > 0,
 * no ignition time, fuel fraction 1; then the instantaneous ignitions with
 * t_g <= 0 (reading: the model starts at t = 0). */
void orc_init_state(int nx, int ny, double dx, double dy, double psi_far,
                    const double *ign, int n_ign, unsigned char *applied,
                    double *psi, double *tign, double *frac)
{
    long n = (long)nx * ny;
    for (long k = 0; k < n; ++k) { psi[k] = psi_far; tign[k] = INFINITY; frac[k] = 1.0; }
    for (int q = 0; q < n_ign; ++q) applied[q] = 0;
    for (int q = 0; q < n_ign; ++q) {
        const double *g = ign + q * IG_N;
        if (!(g[IG_SG] > 0.0) && g[IG_TG] <= 0.0) {
            apply_segment(nx, ny, dx, dy, g, 0.0, psi, tign);
            applied[q] = 1;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Fuel fraction (Sect. "Computation of the fuel fraction").           */
/* ------------------------------------------------------------------ */

/* Burned fraction of one subcell from its 4 corner values, eqs.
 * (approx-area) and (approx-fraction).
 * Reading of the sign in eq. (approx-fraction): the exponent is
 * -(1/4) sum (t - t_i(x_k))/T_f, as in eqs. (fuel) and (fuel_left); the
 * printed t_i - t would make the burned fraction negative.
 * Reading: beta = 0 when all four corner values vanish (then every corner
 * has t_i = t, so the burned fraction is 0 for any beta). */
static double subcell_burned(const double ps[4], const double ts[4], double t, double Tf)
{
    double sp = 0.0, sa = 0.0;
    for (int k = 0; k < 4; ++k) { sp += ps[k]; sa += fabs(ps[k]); }
    double beta = sa > 0.0 ? 0.5 * (1.0 - sp / sa) : 0.0;
    double s = 0.0;
    for (int k = 0; k < 4; ++k) s += t - ts[k];
    return beta * (1.0 - exp(-0.25 * s / Tf));
}

/* Fuel fraction of one cell from the 3x3 node neighbourhood of its centre
 * node.  p and th are 3x3 arrays (row-major, [1][1] is the cell's node) of
 * the level-set function and of the compatible ignition time (t_i where
 * psi < 0, t elsewhere: eq. (ti-comp)).
 * The cell is split into 4 subcells (eq. fuel_left_subcells, Fig. subcells):
 * each has the cell centre, two edge midpoints and one cell corner as
 * vertices.  psi and t_i are interpolated bilinearly between the node
 * centres: an edge midpoint is the mean of 2 nodes, a cell corner the mean
 * of 4.  Where the interpolated psi >= 0 the interpolated t_i is replaced by
 * t (eq. ti-comp applied at the vertices).  Parity unpinned for this vertex
 * rule: for a partly burnt cell no closed form, limit or bound of the paper
 * tells it apart (a copy of the oracle without it passes every pin); the
 * rest of the function is pinned.
 * Reading: the cell fraction burned is the mean of the 4 subcell fractions
 * (the subcells have a quarter of the cell's area). */
double orc_cell_fuel_fraction(const double *p, const double *th, double t, double Tf)
{
    double ps[3][3], ts[3][3];  /* [b][a]: sample at (a-1)/2, (b-1)/2 cell widths */
    for (int b = 0; b < 3; ++b) {
        for (int a = 0; a < 3; ++a) {
            /* nodes that bracket this sample point */
            int ia0 = a == 0 ? 0 : 1, ia1 = a == 2 ? 2 : 1;
            int ib0 = b == 0 ? 0 : 1, ib1 = b == 2 ? 2 : 1;
            double pv, tv;
            if (ia0 == ia1 && ib0 == ib1) {
                pv = p[4];
                tv = th[4];
            } else if (ib0 == ib1) {
                pv = 0.5 * (p[ib0 * 3 + ia0] + p[ib0 * 3 + ia1]);
                tv = 0.5 * (th[ib0 * 3 + ia0] + th[ib0 * 3 + ia1]);
            } else if (ia0 == ia1) {
                pv = 0.5 * (p[ib0 * 3 + ia0] + p[ib1 * 3 + ia0]);
                tv = 0.5 * (th[ib0 * 3 + ia0] + th[ib1 * 3 + ia0]);
            } else {
                pv = 0.25 * (p[ib0 * 3 + ia0] + p[ib0 * 3 + ia1]
                           + p[ib1 * 3 + ia0] + p[ib1 * 3 + ia1]);
                tv = 0.25 * (th[ib0 * 3 + ia0] + th[ib0 * 3 + ia1]
                           + th[ib1 * 3 + ia0] + th[ib1 * 3 + ia1]);
            }
            if (pv >= 0.0) tv = t;
            ps[b][a] = pv;
            ts[b][a] = tv;
        }
    }
    double burned = 0.0;
    for (int sb = 0; sb < 2; ++sb) {
        for (int sa = 0; sa < 2; ++sa) {
            /* subcell with the cell centre (1,1) and the corner (2*sa, 2*sb) */
            int ax = 2 * sa, by = 2 * sb;
            double pc[4] = { ps[1][1], ps[1][ax], ps[by][1], ps[by][ax] };
            double tc[4] = { ts[1][1], ts[1][ax], ts[by][1], ts[by][ax] };
            burned += subcell_burned(pc, tc, t, Tf);
        }
    }
    return 1.0 - 0.25 * burned;
}

/* ---- The alternative scheme of the Discussion: exact when psi and the
 * time from ignition are linear in space (the paper names its property,
 * not its formula; this construction is the reading).
 * The cell is split into 8 triangles (each subcell of eq.
 * (fuel_left_subcells) along its diagonal from the cell centre to the cell
 * corner); on each, psi and D = t - t_i are the linear interpolants of the
 * vertex values (the same 9 vertex values as the subcell scheme: a node, a
 * 2-node mean, a 4-node mean, all exact for linear data).  The triangle is
 * clipped to psi <= 0 (on the cut D = 0: t_i = t on the fireline, eq.
 * ti-comp), and 1 - exp(-D/T_f) is integrated exactly over the clipped
 * polygon (fan triangles, the integral of exp of a linear function).
 * Nodes not yet ignited have no t_i: there D is extended as -lambda psi,
 * lambda = sum (t - t_i) / sum (-psi) over the neighbourhood's nodes with
 * psi < 0 (for linear psi and t_i the two are proportional, with that
 * constant of proportionality).  No node with psi < 0: nothing burns. */

/* (e^a - e^b)/(a - b) with its limit e^a at a == b (a, b <= 0 or small) */
static double dd1_exp(double a, double b)
{
    double d = a - b;
    if (d == 0.0) return exp(a);
    return exp(b) * (expm1(d) / d);
}

/* second divided difference of exp at a, b, c: integral of exp over a
 * triangle with vertex values a, b, c is 2 area dd2_exp(a, b, c) */
static double dd2_exp(double a, double b, double c)
{
    /* order x0 <= x1 <= x2 */
    double x0 = a, x1 = b, x2 = c, tmp;
    if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
    if (x1 > x2) { tmp = x1; x1 = x2; x2 = tmp; }
    if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
    double R = x2 - x0;
    if (R < 1.0) {
        /* sum over k of h_k(u, v)/(k+2)!, h_k the complete homogeneous
         * polynomial of degree k in u = x1 - x0, v = x2 - x0 (both in [0, 1)) */
        double u = x1 - x0, v = x2 - x0, sum = 0.0, fact = 2.0;
        for (int k = 0; k <= 24; ++k) {
            double h = 0.0, ui = 1.0;
            for (int i = 0; i <= k; ++i) {
                double vj = 1.0;
                for (int j = 0; j < k - i; ++j) vj *= v;
                h += ui * vj;
                ui *= u;
            }
            sum += h / fact;
            fact *= (double)(k + 3);
        }
        return exp(x0) * sum;
    }
    return (dd1_exp(x0, x1) - dd1_exp(x1, x2)) / (x0 - x2);
}

/* integral of 1 - exp(-D/Tf) over the part psi <= 0 of the triangle with
 * vertices (x[k], y[k]) and vertex values ps[k], ds[k] */
static double tri_burn(const double *x, const double *y, const double *ps, const double *ds,
                       double Tf)
{
    double px[4], py[4], pd[4];
    int m = 0;
    for (int k = 0; k < 3; ++k) {
        int q = (k + 1) % 3;
        if (ps[k] <= 0.0) { px[m] = x[k]; py[m] = y[k]; pd[m] = ds[k]; ++m; }
        if ((ps[k] < 0.0 && ps[q] > 0.0) || (ps[k] > 0.0 && ps[q] < 0.0)) {
            double s = ps[k] / (ps[k] - ps[q]);
            px[m] = x[k] + s * (x[q] - x[k]);
            py[m] = y[k] + s * (y[q] - y[k]);
            pd[m] = 0.0;   /* on the fireline t_i = t */
            ++m;
        }
    }
    double total = 0.0;
    for (int k = 1; k + 1 < m; ++k) {
        double ar = 0.5 * fabs((px[k] - px[0]) * (py[k + 1] - py[0])
                               - (px[k + 1] - px[0]) * (py[k] - py[0]));
        if (ar == 0.0) continue;
        double e = 2.0 * ar * dd2_exp(-pd[0] / Tf, -pd[k] / Tf, -pd[k + 1] / Tf);
        total += ar - e;
    }
    return total;
}

/* The cell's fuel fraction by this scheme from the same inputs as
 * orc_cell_fuel_fraction (3x3 psi and compatible ignition times). */
double orc_cell_fuel_fraction_linear(const double *p, const double *th, double t, double Tf)
{
    double sD = 0.0, sP = 0.0;
    for (int k = 0; k < 9; ++k)
        if (p[k] < 0.0) { sD += t - th[k]; sP += -p[k]; }
    if (!(sP > 0.0)) return 1.0;
    double lambda = sD / sP;
    double dn[9];
    for (int k = 0; k < 9; ++k) dn[k] = p[k] < 0.0 ? t - th[k] : -lambda * p[k];
    /* vertex values on the unit cell [-1/2, 1/2]^2 (the fraction is the
     * same on the real cell: an affine map keeps area ratios and linear
     * interpolants) */
    double vp[3][3], vd[3][3];
    for (int b = 0; b < 3; ++b) {
        for (int a = 0; a < 3; ++a) {
            int ia0 = a == 0 ? 0 : 1, ia1 = a == 2 ? 2 : 1;
            int ib0 = b == 0 ? 0 : 1, ib1 = b == 2 ? 2 : 1;
            vp[b][a] = 0.25 * ((p[ib0 * 3 + ia0] + p[ib0 * 3 + ia1])
                               + (p[ib1 * 3 + ia0] + p[ib1 * 3 + ia1]));
            vd[b][a] = 0.25 * ((dn[ib0 * 3 + ia0] + dn[ib0 * 3 + ia1])
                               + (dn[ib1 * 3 + ia0] + dn[ib1 * 3 + ia1]));
        }
    }
    double burned = 0.0;
    for (int sb = 0; sb < 2; ++sb) {
        for (int sa = 0; sa < 2; ++sa) {
            int ax = 2 * sa, by = 2 * sb;
            double cx = 0.0, cy = 0.0, kx = ax - 1.0, ky = by - 1.0;
            /* triangles (centre, x-edge midpoint, corner), (centre, corner, y-edge midpoint) */
            double x1[3] = {cx, 0.5 * kx, 0.5 * kx}, y1[3] = {cy, 0.0, 0.5 * ky};
            double p1[3] = {vp[1][1], vp[1][ax], vp[by][ax]};
            double d1[3] = {vd[1][1], vd[1][ax], vd[by][ax]};
            double x2[3] = {cx, 0.5 * kx, 0.0}, y2[3] = {cy, 0.5 * ky, 0.5 * ky};
            double p2[3] = {vp[1][1], vp[by][ax], vp[by][1]};
            double d2[3] = {vd[1][1], vd[by][ax], vd[by][1]};
            burned += tri_burn(x1, y1, p1, d1, Tf) + tri_burn(x2, y2, p2, d2, Tf);
        }
    }
    return 1.0 - burned;
}

/* ------------------------------------------------------------------ */
/* The fire step (Sect. "Coupling", the six-item list).                */
/* ------------------------------------------------------------------ */

typedef struct {
    int nxa, nya, srx, sry;
    double dx_atm, dy_atm;
    double eps;        /* artificial viscosity, 0.4 in the paper */
    int band;          /* width of the boundary ring checked for fire */
    int scheme;        /* fuel fraction: 0 the subcell scheme of Sect. 3.3,
                          1 the scheme exact for linear psi and t_i */
} orc_grid;

enum { ORC_BOUNDARY = 1, ORC_NONFINITE = 2 };

/* One fire step from time t to t + dt.  State (psi, tign, frac) is updated
 * in place; heat_s, heat_l ([nya][nxa]) receive the averaged sensible and
 * latent heat flux densities (W m^-2).  Returns status bits.
 *   1. ignitions active at t                 (Sect. Ignition)
 *   2. Heun stages of eq. (Heun) with eq. (F-disc); wind fixed in the step;
 *      ghosts re-extrapolated for each stage
 *   3. ignition time by eq. (set-ignition-time) where psi crossed from > 0
 *      to <= 0; fire in the boundary ring sets ORC_BOUNDARY
 *   4. fuel fraction at t + dt (Sect. fuel fraction)
 *   5. heat flux densities per fire cell, eqs. (sensible-/latent-heat-flux)
 *   6. average over the fire cells of each atmospheric cell
 * co: per-node coefficients [n][9]; mult: per-node multiplier or NULL. */
int orc_step(const orc_grid *g, const double *co, const double *mult,
             const double *dzdx, const double *dzdy,
             const double *u, const double *v,
             const double *ign, int n_ign, unsigned char *applied,
             double t, double dt,
             double *psi, double *tign, double *frac,
             double *heat_s, double *heat_l)
{
    int nx = g->nxa * g->srx, ny = g->nya * g->sry;
    long n = (long)nx * ny;
    long ne = (long)(nx + 2) * (ny + 2);
    double dx = g->dx_atm / g->srx, dy = g->dy_atm / g->sry;
    int status = 0;

    double *un = malloc(sizeof(double) * n), *vn = malloc(sizeof(double) * n);
    double *ext = malloc(sizeof(double) * ne);
    double *F1 = malloc(sizeof(double) * n), *F2 = malloc(sizeof(double) * n);
    double *ps = malloc(sizeof(double) * n), *pn = malloc(sizeof(double) * n);
    double *th = malloc(sizeof(double) * n), *fnew = malloc(sizeof(double) * n);
    double *ext_t = malloc(sizeof(double) * ne);

    /* 1. ignition */
    orc_ignite(nx, ny, dx, dy, ign, n_ign, applied, t, psi, tign);

    /* wind at the fire nodes; a non-finite wind is reported (the clamps of
     * eq. spread-WRF-Fire would otherwise read it as calm) */
    orc_wind_at_nodes(g->nxa, g->nya, g->srx, g->sry, u, v, un, vn);
#pragma omp parallel for schedule(static) reduction(|:status)
    for (long k = 0; k < n; ++k)
        if (!isfinite(un[k]) || !isfinite(vn[k])) status |= ORC_NONFINITE;

    /* 2. Heun: psi* = psi + dt F(psi); psi^{n+1} = psi + dt (F(psi)/2 + F(psi*)/2) */
    orc_extend(nx, ny, psi, ext);
    orc_rhs(nx, ny, dx, dy, g->eps, ext, co, mult, un, vn, dzdx, dzdy, F1);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) ps[k] = psi[k] + dt * F1[k];
    orc_extend(nx, ny, ps, ext);
    orc_rhs(nx, ny, dx, dy, g->eps, ext, co, mult, un, vn, dzdx, dzdy, F2);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) pn[k] = psi[k] + dt * (0.5 * F1[k] + 0.5 * F2[k]);

    /* 3. ignition time at the sign change, eq. (set-ignition-time) */
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        if (psi[k] > 0.0 && pn[k] <= 0.0 && isinf(tign[k]))
            tign[k] = t + psi[k] * dt / (psi[k] - pn[k]);
    }
#pragma omp parallel for schedule(static) reduction(|:status)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double pv = pn[(long)j * nx + i];
            if (!isfinite(pv)) status |= ORC_NONFINITE;
            int edge = i < g->band || j < g->band || i >= nx - g->band || j >= ny - g->band;
            if (edge && pv < 0.0) status |= ORC_BOUNDARY;
        }
    }
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) psi[k] = pn[k];

    /* 4. fuel fraction at t1 = t + dt */
    double t1 = t + dt;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) th[k] = psi[k] < 0.0 ? tign[k] : t1;   /* eq. (ti-comp) */
    orc_extend(nx, ny, psi, ext);
    /* Reading: ghost ignition times copy the adjacent node's (x first, then
     * y, as for psi), then eq. (ti-comp) is applied with the ghost psi. */
    {
        int W = nx + 2;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                ext_t[(j + 1) * W + (i + 1)] = th[(long)j * nx + i];
        for (int j = 1; j <= ny; ++j) {
            ext_t[j * W] = ext_t[j * W + 1];
            ext_t[j * W + nx + 1] = ext_t[j * W + nx];
        }
        for (int i = 0; i < W; ++i) {
            ext_t[i] = ext_t[W + i];
            ext_t[(ny + 1) * W + i] = ext_t[ny * W + i];
        }
#pragma omp parallel for schedule(static)
        for (long k = 0; k < ne; ++k)
            if (ext[k] >= 0.0) ext_t[k] = t1;
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            int W = nx + 2;
            double p9[9], t9[9];
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    p9[b * 3 + a] = ext[(j + b) * W + (i + a)];
                    t9[b * 3 + a] = ext_t[(j + b) * W + (i + a)];
                }
            long k = (long)j * nx + i;
            fnew[k] = g->scheme == 1
                          ? orc_cell_fuel_fraction_linear(p9, t9, t1, co[k * CO_N + CO_TF])
                          : orc_cell_fuel_fraction(p9, t9, t1, co[k * CO_N + CO_TF]);
        }
    }

    /* 5-6. heat flux densities and their average over each atmos cell */
#pragma omp parallel for schedule(static)
    for (int J = 0; J < g->nya; ++J) {
        for (int I = 0; I < g->nxa; ++I) {
            double sh = 0.0, sl = 0.0;
            for (int j = J * g->sry; j < (J + 1) * g->sry; ++j) {
                for (int i = I * g->srx; i < (I + 1) * g->srx; ++i) {
                    long k = (long)j * nx + i;
                    double rate = (frac[k] - fnew[k]) / dt;
                    sh += rate * co[k * CO_N + CO_HS];
                    sl += rate * co[k * CO_N + CO_HQ];
                }
            }
            heat_s[J * g->nxa + I] = sh / (double)(g->srx * g->sry);
            heat_l[J * g->nxa + I] = sl / (double)(g->srx * g->sry);
        }
    }
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) frac[k] = fnew[k];

    free(un); free(vn); free(ext); free(F1); free(F2); free(ps); free(pn);
    free(th); free(fnew); free(ext_t);
    return status;
}

/* ------------------------------------------------------------------ */
/* Reference adjoint of the arrival-time misfit.                       */
/* Not in the paper: data assimilation is its stated reason for the    */
/* level-set formulation (Sect. 7, "Data assimilation").  Plain reverse */
/* sweep through eqs. (Heun), (F-disc), (Godunov) and                  */
/* (set-ignition-time), every forward state stored, the branches of    */
/* the forward step (Godunov cases, max/min, extrapolation, zeroed     */
/* central differences) frozen.                                        */
/* J = 1/2 sum over nodes ignited in both runs of (t_i - t_obs)^2.     */
/* ------------------------------------------------------------------ */

/* forward-mode dual numbers for d(coefficients)/d(M_f) */
typedef struct { double v, d; } dnum;
static dnum dn(double v, double d) { dnum r; r.v = v; r.d = d; return r; }
static dnum dn_add(dnum a, dnum b) { return dn(a.v + b.v, a.d + b.d); }
static dnum dn_sub(dnum a, dnum b) { return dn(a.v - b.v, a.d - b.d); }
static dnum dn_mul(dnum a, dnum b) { return dn(a.v * b.v, a.d * b.v + a.v * b.d); }
static dnum dn_div(dnum a, dnum b) { return dn(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static dnum dn_scale(dnum a, double s) { return dn(a.v * s, a.d * s); }
static dnum dn_powc(dnum a, double p) { return dn(pow(a.v, p), p * pow(a.v, p - 1.0) * a.d); }
static dnum dn_exp(dnum a) { double e = exp(a.v); return dn(e, e * a.d); }

/* d(S0, R0, b, c, d, e, T_f, H_s, H_q)/d(M_f) of orc_fuel_coefficients, the
 * same Table 2 chain evaluated on dual numbers (clamped branches and the
 * chaparral rule have zero derivative). */
void orc_fuel_coefficients_dMf(const double *fc, double Mf, double *dco)
{
    if (Mf < 0.0) Mf = fc[FC_MF];
    for (int k = 0; k < CO_N; ++k) dco[k] = 0.0;
    dco[CO_HS] = -fc[FC_FGI] * fc[FC_H] / ((1.0 + Mf) * (1.0 + Mf));
    dco[CO_HQ] = 0.44 / ((1.0 + Mf) * (1.0 + Mf)) * LATENT_L * fc[FC_FGI];
    if (fc[FC_CHAPARRAL] != 0.0 || !(fc[FC_FGI] > 0.0)) return;
    double sigma  = fc[FC_SAVR] * M_PER_FT;
    double wl     = fc[FC_FGI] * (M_PER_FT * M_PER_FT) / KG_PER_LB;
    double depth  = fc[FC_DEPTH] / M_PER_FT;
    double rho_p  = fc[FC_DENS] * (M_PER_FT * M_PER_FT * M_PER_FT) / KG_PER_LB;
    double h      = fc[FC_H] * KG_PER_LB / J_PER_BTU;
    dnum mf = dn(Mf, 1.0);
    dnum w0 = dn_div(dn(wl, 0.0), dn_add(dn(1.0, 0.0), mf));
    dnum rho_b = dn_scale(w0, 1.0 / depth);
    dnum beta = dn_scale(rho_b, 1.0 / rho_p);
    double beta_op = 3.348 * pow(sigma, -0.8189);
    double A = 1.0 / (4.77 * pow(sigma, 0.1) - 7.27);
    double s15 = pow(sigma, 1.5);
    double Gmax = s15 / (495.0 + 0.0594 * s15);
    dnum ratio = dn_scale(beta, 1.0 / beta_op);
    dnum Gamma = dn_scale(dn_mul(dn_powc(ratio, A), dn_exp(dn_scale(dn_sub(dn(1.0, 0.0), ratio), A))), Gmax);
    dnum wn = dn_scale(w0, 1.0 / (1.0 + fc[FC_ST]));
    dnum rm = dn_scale(mf, 1.0 / fc[FC_MX]);
    dnum etaM = dn_add(dn_sub(dn(1.0, 0.0), dn_scale(rm, 2.59)),
                       dn_sub(dn_scale(dn_mul(rm, rm), 5.11), dn_scale(dn_mul(dn_mul(rm, rm), rm), 3.52)));
    if (rm.v >= 1.0 || etaM.v < 0.0) etaM = dn(0.0, 0.0);
    if (etaM.v > 1.0) etaM = dn(1.0, 0.0);
    double etaS = 0.174 * pow(fc[FC_SE], -0.19);
    dnum IR = dn_scale(dn_mul(dn_mul(Gamma, wn), etaM), h * etaS);
    dnum xi = dn_scale(dn_exp(dn_scale(dn_add(beta, dn(0.1, 0.0)), 0.792 + 0.681 * sqrt(sigma))),
                       1.0 / (192.0 + 0.2595 * sigma));
    double epsh = exp(-138.0 / sigma);
    dnum Qig = dn_add(dn(250.0, 0.0), dn_scale(mf, 1116.0));
    dnum R0f = dn_div(dn_mul(IR, xi), dn_scale(dn_mul(rho_b, Qig), epsh));
    dnum R0 = dn_scale(R0f, M_PER_FT / 60.0);
    double B = 0.02526 * pow(sigma, 0.54);
    double C = 7.47 * exp(-0.133 * pow(sigma, 0.55));
    double E = 0.715 * exp(-3.59e-4 * sigma);
    dnum c = dn_scale(dn_mul(R0, dn_powc(ratio, -E)), C * pow(fc[FC_WINDRF] * (60.0 / M_PER_FT), B));
    dnum d = dn_scale(dn_mul(R0, dn_powc(beta, -0.3)), 5.275);
    dco[CO_R0] = R0.d;
    dco[CO_C] = c.d;
    dco[CO_D] = d.d;
}

void orc_node_coefficients_dMf(const double *classes, int ncls, const unsigned char *fuel,
                               const double *moisture, long n, double *dco)
{
    for (long k = 0; k < n; ++k) {
        int c = fuel[k];
        if (c >= ncls) c = ncls - 1;
        orc_fuel_coefficients_dMf(classes + (long)c * FC_N, moisture ? moisture[k] : -1.0,
                                  dco + k * CO_N);
    }
}

/* value of eq. (Godunov) and which one-sided difference it took
 * (-1: D-, +1: D+, 0: neither) */
static double godunov_sel(double dm, double dp, int *sel)
{
    if (dm <= 0.0 && dp <= 0.0) { *sel = 1; return dp; }
    if (dm >= 0.0 && dp >= 0.0) { *sel = -1; return dm; }
    if (dm <= 0.0 && dp >= 0.0) { *sel = 0; return 0.0; }
    if (fabs(dm) >= fabs(dp)) { *sel = -1; return dm; }
    *sel = 1;
    return dp;
}

/* Partial derivatives of F at one node (the computation of orc_rhs with
 * its branches frozen) with respect to the 5 stencil values
 * (centre, left, right, down, up), the multiplier m, the coefficients
 * (S0, R0, c, d) and the node wind (un, vn). */
typedef struct {
    double dpsi[5];
    double dm, dS0, dR0, dc, dd, dun, dvn;
} orc_partials;

static void rhs_partials(double p, double pl, double pr, double pd, double pu, double dx,
                         double dy, double eps, const double *co, double m, double un,
                         double vn, double zx, double zy, orc_partials *o)
{
    memset(o, 0, sizeof *o);
    double dxm = (p - pl) / dx, dxp = (pr - p) / dx;
    double dym = (p - pd) / dy, dyp = (pu - p) / dy;
    int sx, sy;
    double gx = godunov_sel(dxm, dxp, &sx);
    double gy = godunov_sel(dym, dyp, &sy);
    double ax = pr - pl, ay = pu - pd;
    int zxk = 1, zyk = 1;
    if (fabs(ax) <= ORC_GRAD_ZERO * (fabs(pr) + fabs(pl))) { ax = 0.0; zxk = 0; }
    if (fabs(ay) <= ORC_GRAD_ZERO * (fabs(pu) + fabs(pd))) { ay = 0.0; zyk = 0; }
    double cx = ax / (2.0 * dx), cy = ay / (2.0 * dy);
    double cn = sqrt(cx * cx + cy * cy);
    double nxv = 0.0, nyv = 0.0;
    if (cn > 0.0) { nxv = cx / cn; nyv = cy / cn; }
    double U = un * nxv + vn * nyv;
    double T = zx * nxv + zy * nyv;
    /* spread rate, eq. (spread-WRF-Fire), with its branches */
    double Up = U > 0.0 ? U : 0.0;
    double Ue = Up < co[CO_E] ? Up : co[CO_E];
    double tp = T > 0.0 ? T : 0.0;
    double inner = co[CO_R0] + co[CO_C] * pow(Ue, co[CO_B]) + co[CO_D] * tp * tp;
    int active = inner > co[CO_S0];
    double St = active ? inner : co[CO_S0];
    double S = m * St;
    double lap = (dxp - dxm) + (dyp - dym);
    double grad = sqrt(gx * gx + gy * gy);
    double Fs = -grad + eps * lap;                      /* dF/dS */
    double dSt_dU = (active && U > 0.0 && U < co[CO_E])
                        ? co[CO_C] * co[CO_B] * pow(Ue, co[CO_B] - 1.0) : 0.0;
    double dSt_dT = (active && T > 0.0) ? 2.0 * co[CO_D] * T : 0.0;
    /* normal: dn/dc = (I - n n^T)/|c| */
    double dU_dcx = 0.0, dU_dcy = 0.0, dT_dcx = 0.0, dT_dcy = 0.0;
    if (cn > 0.0) {
        dU_dcx = (un - U * nxv) / cn;
        dU_dcy = (vn - U * nyv) / cn;
        dT_dcx = (zx - T * nxv) / cn;
        dT_dcy = (zy - T * nyv) / cn;
    }
    double dS_dcx = m * (dSt_dU * dU_dcx + dSt_dT * dT_dcx);
    double dS_dcy = m * (dSt_dU * dU_dcy + dSt_dT * dT_dcy);
    double dcx_dpr = zxk ? 1.0 / (2.0 * dx) : 0.0, dcy_dpu = zyk ? 1.0 / (2.0 * dy) : 0.0;
    /* dS/dpsi: C, L, R, D, U */
    double dS[5] = {0.0, -dS_dcx * dcx_dpr, dS_dcx * dcx_dpr, -dS_dcy * dcy_dpu, dS_dcy * dcy_dpu};
    /* d|grad|/dpsi through the selected one-sided differences */
    double dG[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (grad > 0.0) {
        double wx = gx / grad, wy = gy / grad;
        if (sx == -1) { dG[0] += wx / dx; dG[1] -= wx / dx; }
        if (sx == 1) { dG[2] += wx / dx; dG[0] -= wx / dx; }
        if (sy == -1) { dG[0] += wy / dy; dG[3] -= wy / dy; }
        if (sy == 1) { dG[4] += wy / dy; dG[0] -= wy / dy; }
    }
    double dL[5] = {-2.0 / dx - 2.0 / dy, 1.0 / dx, 1.0 / dx, 1.0 / dy, 1.0 / dy};
    for (int k = 0; k < 5; ++k)
        o->dpsi[k] = Fs * dS[k] - S * dG[k] + eps * S * dL[k];
    o->dm = Fs * St;
    o->dS0 = Fs * m * (active ? 0.0 : 1.0);
    o->dR0 = Fs * m * (active ? 1.0 : 0.0);
    o->dc = Fs * m * (active ? pow(Ue, co[CO_B]) : 0.0);
    o->dd = Fs * m * (active ? tp * tp : 0.0);
    o->dun = Fs * m * dSt_dU * nxv;
    o->dvn = Fs * m * dSt_dU * nyv;
}

/* d(ghost)/d(p0), d(ghost)/d(p1) for the extrapolation's taken branch */
static void ghost_partials(double p0, double p1, double *d0, double *d1)
{
    double g = p0 + (p0 - p1);
    *d0 = 2.0;
    *d1 = -1.0;
    if (p0 > g) { g = p0; *d0 = 1.0; *d1 = 0.0; }
    if (p1 > g) { *d0 = 0.0; *d1 = 1.0; }
}

/* r += J_F(psi)^T v for the field psi (with its extrapolated ghosts), and
 * the parameter terms v^T dF/dp accumulated per node. */
static void rhs_vjp(int nx, int ny, double dx, double dy, double eps, const double *psi,
                    const double *ext, const double *co, const double *dco, const double *mult,
                    const double *un, const double *vn, const double *dzdx, const double *dzdy,
                    const double *v, double *r, double *gm, double *gMf, double *gun, double *gvn)
{
    int W = nx + 2;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            if (v[k] == 0.0) continue;
            const double *e = ext + (j + 1) * W + (i + 1);
            orc_partials o;
            rhs_partials(e[0], e[-1], e[1], e[-W], e[W], dx, dy, eps, co + k * CO_N,
                         mult ? mult[k] : 1.0, un[k], vn[k], dzdx[k], dzdy[k], &o);
            double vk = v[k];
            /* stencil positions: C, L, R, D, U */
            int ii[5] = {i, i - 1, i + 1, i, i};
            int jj[5] = {j, j, j, j - 1, j + 1};
            for (int q = 0; q < 5; ++q) {
                double c = vk * o.dpsi[q];
                int a = ii[q], b = jj[q];
                if (a >= 0 && a < nx && b >= 0 && b < ny) {
                    r[(long)b * nx + a] += c;
                } else if (a < 0 || a >= nx) {  /* x-ghost of row b */
                    int i0 = a < 0 ? 0 : nx - 1, i1 = a < 0 ? 1 : nx - 2;
                    double d0, d1;
                    ghost_partials(psi[(long)b * nx + i0], psi[(long)b * nx + i1], &d0, &d1);
                    r[(long)b * nx + i0] += c * d0;
                    r[(long)b * nx + i1] += c * d1;
                } else {                        /* y-ghost of column a */
                    int j0 = b < 0 ? 0 : ny - 1, j1 = b < 0 ? 1 : ny - 2;
                    double d0, d1;
                    ghost_partials(psi[(long)j0 * nx + a], psi[(long)j1 * nx + a], &d0, &d1);
                    r[(long)j0 * nx + a] += c * d0;
                    r[(long)j1 * nx + a] += c * d1;
                }
            }
            gm[k] += vk * o.dm;
            const double *dc = dco + k * CO_N;
            gMf[k] += vk * (o.dS0 * dc[CO_S0] + o.dR0 * dc[CO_R0] + o.dc * dc[CO_C] + o.dd * dc[CO_D]);
            gun[k] += vk * o.dun;
            gvn[k] += vk * o.dvn;
        }
    }
}

/* Adjoint of the level-set part of one step (eq. Heun): given
 * mu = dJ/dpsi^{n+1} returns lam = dJ/dpsi^n and accumulates the parameter
 * terms:  lam* = dt/2 J_F(psi*)^T mu,  w = dt/2 mu + dt lam*,
 *         lam = mu + lam* + J_F(psi^n)^T w. */
static void adjoint_step(int nx, int ny, double dx, double dy, double eps, const double *psi,
                         const double *co, const double *dco, const double *mult,
                         const double *un, const double *vn, const double *dzdx,
                         const double *dzdy, double dt, const double *mu, double *lam,
                         double *gm, double *gMf, double *gun, double *gvn)
{
    long n = (long)nx * ny, ne = (long)(nx + 2) * (ny + 2);
    double *ext0 = malloc(sizeof(double) * ne), *ext1 = malloc(sizeof(double) * ne);
    double *F1 = malloc(sizeof(double) * n), *ps = malloc(sizeof(double) * n);
    double *v = malloc(sizeof(double) * n), *ls = calloc(n, sizeof(double));
    double *r1 = calloc(n, sizeof(double));
    orc_extend(nx, ny, psi, ext0);
    orc_rhs(nx, ny, dx, dy, eps, ext0, co, mult, un, vn, dzdx, dzdy, F1);
    for (long k = 0; k < n; ++k) ps[k] = psi[k] + dt * F1[k];
    orc_extend(nx, ny, ps, ext1);
    for (long k = 0; k < n; ++k) v[k] = 0.5 * dt * mu[k];
    rhs_vjp(nx, ny, dx, dy, eps, ps, ext1, co, dco, mult, un, vn, dzdx, dzdy, v, ls, gm, gMf,
            gun, gvn);
    for (long k = 0; k < n; ++k) v[k] = 0.5 * dt * mu[k] + dt * ls[k];
    rhs_vjp(nx, ny, dx, dy, eps, psi, ext0, co, dco, mult, un, vn, dzdx, dzdy, v, r1, gm, gMf,
            gun, gvn);
    for (long k = 0; k < n; ++k) lam[k] = mu[k] + ls[k] + r1[k];
    free(ext0); free(ext1); free(F1); free(ps); free(v); free(ls); free(r1);
}

/* Vector-Jacobian product of one level-set step of the state psi (the two
 * Heun stages of eq. Heun with eq. F-disc, ghosts as in orc_step, the wind
 * of u, v interpolated to the nodes): for a cotangent w on psi^{n+1},
 * lam = (d psi^{n+1} / d psi^n)^T w, and w^T d psi^{n+1} / dp added to gm
 * (per-node multiplier), gMf (per-node moisture, through dco = dco/dM_f
 * per node) and gun, gvn (node wind components).  The reverse step of
 * orc_adjoint without the arrival-time seeds; pinned by the dot-product
 * test against central differences of the forward step. */
void orc_step_vjp(const orc_grid *g, const double *co, const double *dco, const double *mult,
                  const double *dzdx, const double *dzdy, const double *u, const double *v,
                  double dt, const double *psi, const double *w, double *lam, double *gm,
                  double *gMf, double *gun, double *gvn)
{
    int nx = g->nxa * g->srx, ny = g->nya * g->sry;
    long n = (long)nx * ny;
    double dx = g->dx_atm / g->srx, dy = g->dy_atm / g->sry;
    double *un = malloc(sizeof(double) * n), *vn = malloc(sizeof(double) * n);
    orc_wind_at_nodes(g->nxa, g->nya, g->srx, g->sry, u, v, un, vn);
    adjoint_step(nx, ny, dx, dy, g->eps, psi, co, dco, mult, un, vn, dzdx, dzdy, dt, w, lam, gm,
                 gMf, gun, gvn);
    free(un); free(vn);
}

/* Whether node k's ignition time was set in the step [t_s, t_s + dt] that
 * took psi from a to b (eq. set-ignition-time): it was not ignited before
 * the run, the step crossed from > 0 to <= 0, and the recorded time lies in
 * the step (a later crossing after the level set rose again sets nothing). */
static int crossed_in_step(double tign0, double ti, double ts, double ts1, double a, double b)
{
    return isinf(tign0) && isfinite(ti) && a > 0.0 && b <= 0.0 && ti >= ts && ti <= ts1;
}

/* Forward run of nsteps steps from the given state (no ignitions during the
 * run), misfit J and its gradient with respect to the per-node multiplier
 * (at the given multiplier, 1 where mult is NULL), the per-node fuel
 * moisture (at the values that made co, with dco = dco/dM_f) and the
 * staggered wind u, v.  On return psi, tign, frac hold the final state.
 * Outputs g_* are overwritten.  Nodes without an observation carry a
 * non-finite tobs. */
/* Forward run of nsteps steps (no ignitions), keeping every state and the
 * step start times (used by both adjoints below). */
static void forward_run(const orc_grid *g, const double *co, const double *mult,
                        const double *dzdx, const double *dzdy, const double *u, const double *v,
                        double t0, double dt, int nsteps, double *psi, double *tign, double *frac,
                        double *states, double *times)
{
    long n = (long)g->nxa * g->srx * g->nya * g->sry;
    double *hs = malloc(sizeof(double) * g->nxa * g->nya), *hl = malloc(sizeof(double) * g->nxa * g->nya);
    unsigned char applied[1] = {1};
    memcpy(states, psi, sizeof(double) * n);
    double t = t0;
    times[0] = t;
    for (int s = 0; s < nsteps; ++s) {
        orc_step(g, co, mult, dzdx, dzdy, u, v, NULL, 0, applied, t, dt, psi, tign, frac, hs, hl);
        t = t + dt;
        times[s + 1] = t;
        memcpy(states + (long)(s + 1) * n, psi, sizeof(double) * n);
    }
    free(hs); free(hl);
}

/* The reverse sweep over the stored states: lam enters as dJ/dpsi at the
 * end of the run and leaves as dJ/dpsi at its start; dJdt[k] (finite where
 * J depends on node k's ignition time) seeds the nodes whose first crossing
 * was the step, through eq. (set-ignition-time); the parameter terms go to
 * g_mult, g_moist (added to) and the node wind gradients gun, gvn. */
static void adjoint_sweep(const orc_grid *g, const double *co, const double *dco,
                          const double *mult, const double *dzdx, const double *dzdy,
                          const double *un, const double *vn, double dt, int nsteps,
                          const double *states, const double *times, const double *tign0,
                          const double *tign, const double *dJdt, double *lam, double *g_mult,
                          double *g_moist, double *gun, double *gvn)
{
    int nx = g->nxa * g->srx, ny = g->nya * g->sry;
    long n = (long)nx * ny;
    double dx = g->dx_atm / g->srx, dy = g->dy_atm / g->sry;
    double *mu = malloc(sizeof(double) * n);
    for (int s = nsteps - 1; s >= 0; --s) {
        const double *pa = states + (long)s * n, *pb = states + (long)(s + 1) * n;
        /* eq. (set-ignition-time) at the nodes whose first crossing was this step */
        for (long k = 0; k < n; ++k) {
            mu[k] = lam[k];
            if (isfinite(dJdt[k]) &&
                crossed_in_step(tign0[k], tign[k], times[s], times[s + 1], pa[k], pb[k])) {
                double a = pa[k], b = pb[k], r = dJdt[k];
                mu[k] += r * dt * a / ((a - b) * (a - b));
            }
        }
        adjoint_step(nx, ny, dx, dy, g->eps, pa, co, dco, mult, un, vn, dzdx, dzdy, dt, mu, lam,
                     g_mult, g_moist, gun, gvn);
        for (long k = 0; k < n; ++k) {
            if (isfinite(dJdt[k]) &&
                crossed_in_step(tign0[k], tign[k], times[s], times[s + 1], pa[k], pb[k])) {
                double a = pa[k], b = pb[k], r = dJdt[k];
                lam[k] += r * (-dt * b / ((a - b) * (a - b)));
            }
        }
    }
    free(mu);
}

/* Adjoint of the bilinear wind interpolation of Sect. 5: every staggered
 * face sums the node gradients times the weights the forward gave it. */
static void wind_gather(const orc_grid *g, const double *gun, const double *gvn, double *g_u,
                        double *g_v)
{
    int nx = g->nxa * g->srx, ny = g->nya * g->sry;
    for (long q = 0; q < (long)g->nya * (g->nxa + 1); ++q) g_u[q] = 0.0;
    for (long q = 0; q < (long)(g->nya + 1) * g->nxa; ++q) g_v[q] = 0.0;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            double xa = ((double)i + 0.5) / (double)g->srx;
            double ya = ((double)j + 0.5) / (double)g->sry;
            int i0, i1, j0, j1;
            double wx, wy;
            interp_weights(xa, g->nxa + 1, &i0, &i1, &wx);
            interp_weights(ya - 0.5, g->nya, &j0, &j1, &wy);
            int W = g->nxa + 1;
            g_u[j0 * W + i0] += gun[k] * (1.0 - wy) * (1.0 - wx);
            g_u[j0 * W + i1] += gun[k] * (1.0 - wy) * wx;
            g_u[j1 * W + i0] += gun[k] * wy * (1.0 - wx);
            g_u[j1 * W + i1] += gun[k] * wy * wx;
            interp_weights(xa - 0.5, g->nxa, &i0, &i1, &wx);
            interp_weights(ya, g->nya + 1, &j0, &j1, &wy);
            W = g->nxa;
            g_v[j0 * W + i0] += gvn[k] * (1.0 - wy) * (1.0 - wx);
            g_v[j0 * W + i1] += gvn[k] * (1.0 - wy) * wx;
            g_v[j1 * W + i0] += gvn[k] * wy * (1.0 - wx);
            g_v[j1 * W + i1] += gvn[k] * wy * wx;
        }
    }
}

/* Partial derivatives of orc_cell_fuel_fraction with respect to its nine
 * psi and nine th window values, the branches frozen as the forward took
 * them (which vertices have psi >= 0 and so take t instead of the
 * interpolated th; the signs in sum |psi|; beta = 0 where sum |psi| = 0).
 * Reading: d|x|/dx = sign(x), 0 at x = 0. */
static void cell_fraction_partials(const double *p, const double *th, double t, double Tf,
                                   double *dp, double *dth)
{
    double ps[3][3], ts[3][3], w[3][3][9];
    int tfix[3][3];
    for (int b = 0; b < 3; ++b) {
        for (int a = 0; a < 3; ++a) {
            int ia0 = a == 0 ? 0 : 1, ia1 = a == 2 ? 2 : 1;
            int ib0 = b == 0 ? 0 : 1, ib1 = b == 2 ? 2 : 1;
            for (int q = 0; q < 9; ++q) w[b][a][q] = 0.0;
            /* the bilinear weights of the nodes bracketing the sample point */
            w[b][a][ib0 * 3 + ia0] += 0.25;
            w[b][a][ib0 * 3 + ia1] += 0.25;
            w[b][a][ib1 * 3 + ia0] += 0.25;
            w[b][a][ib1 * 3 + ia1] += 0.25;
            /* the sample values computed as orc_cell_fuel_fraction does */
            double pv, tv;
            if (ia0 == ia1 && ib0 == ib1) {
                pv = p[4];
                tv = th[4];
            } else if (ib0 == ib1) {
                pv = 0.5 * (p[ib0 * 3 + ia0] + p[ib0 * 3 + ia1]);
                tv = 0.5 * (th[ib0 * 3 + ia0] + th[ib0 * 3 + ia1]);
            } else if (ia0 == ia1) {
                pv = 0.5 * (p[ib0 * 3 + ia0] + p[ib1 * 3 + ia0]);
                tv = 0.5 * (th[ib0 * 3 + ia0] + th[ib1 * 3 + ia0]);
            } else {
                pv = 0.25 * (p[ib0 * 3 + ia0] + p[ib0 * 3 + ia1]
                           + p[ib1 * 3 + ia0] + p[ib1 * 3 + ia1]);
                tv = 0.25 * (th[ib0 * 3 + ia0] + th[ib0 * 3 + ia1]
                           + th[ib1 * 3 + ia0] + th[ib1 * 3 + ia1]);
            }
            tfix[b][a] = pv >= 0.0;
            ps[b][a] = pv;
            ts[b][a] = tfix[b][a] ? t : tv;
        }
    }
    double gps[3][3] = {{0.0}}, gts[3][3] = {{0.0}};
    for (int sb = 0; sb < 2; ++sb) {
        for (int sa = 0; sa < 2; ++sa) {
            int ax = 2 * sa, by = 2 * sb;
            int pb[4] = {1, 1, by, by}, pa[4] = {1, ax, 1, ax};
            double sp = 0.0, sabs = 0.0, sum = 0.0;
            for (int k = 0; k < 4; ++k) {
                double x = ps[pb[k]][pa[k]];
                sp += x;
                sabs += fabs(x);
                sum += t - ts[pb[k]][pa[k]];
            }
            double e = exp(-0.25 * sum / Tf);
            double beta = sabs > 0.0 ? 0.5 * (1.0 - sp / sabs) : 0.0;
            /* F = 1 - sum over subcells of burned / 4, burned = beta (1 - e) */
            for (int k = 0; k < 4; ++k) {
                double x = ps[pb[k]][pa[k]];
                double sg = x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
                double dbeta = sabs > 0.0 ? 0.5 * (-1.0 / sabs + sp * sg / (sabs * sabs)) : 0.0;
                gps[pb[k]][pa[k]] += -0.25 * (1.0 - e) * dbeta;
                gts[pb[k]][pa[k]] += -0.25 * (-beta * e * 0.25 / Tf);
            }
        }
    }
    for (int q = 0; q < 9; ++q) { dp[q] = 0.0; dth[q] = 0.0; }
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 9; ++q) {
                dp[q] += gps[b][a] * w[b][a][q];
                if (!tfix[b][a]) dth[q] += gts[b][a] * w[b][a][q];
            }
}

/* Adjoint of orc_extend: D holds d/d(ext) on the (nx+2) x (ny+2) extension
 * of a; adds the derivative with respect to the nodes of a to da (the y
 * ghosts first, as they were filled last, then the x ghosts). */
static void extend_adjoint(int nx, int ny, const double *a, double *D, double *da)
{
    int W = nx + 2;
    double *ext = malloc(sizeof(double) * W * (ny + 2));
    orc_extend(nx, ny, a, ext);
    for (int i = 0; i < W; ++i) {
        double d0, d1;
        ghost_partials(ext[W + i], ext[2 * W + i], &d0, &d1);
        D[W + i] += D[i] * d0;
        D[2 * W + i] += D[i] * d1;
        ghost_partials(ext[ny * W + i], ext[(ny - 1) * W + i], &d0, &d1);
        D[ny * W + i] += D[(ny + 1) * W + i] * d0;
        D[(ny - 1) * W + i] += D[(ny + 1) * W + i] * d1;
    }
    for (int j = 1; j <= ny; ++j) {
        double d0, d1;
        double *row = ext + j * W, *Dr = D + j * W;
        ghost_partials(row[1], row[2], &d0, &d1);
        Dr[1] += Dr[0] * d0;
        Dr[2] += Dr[0] * d1;
        ghost_partials(row[nx], row[nx - 1], &d0, &d1);
        Dr[nx] += Dr[nx + 1] * d0;
        Dr[nx - 1] += Dr[nx + 1] * d1;
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) da[(long)j * nx + i] += D[(j + 1) * W + (i + 1)];
    free(ext);
}

/* orc_extend's transpose for tests: da = (d ext / d a)^T D (da overwritten;
 * D is left unchanged). */
void orc_extend_vjp(int nx, int ny, const double *a, const double *D, double *da)
{
    long ne = (long)(nx + 2) * (ny + 2);
    double *Dc = malloc(sizeof(double) * ne);
    memcpy(Dc, D, sizeof(double) * ne);
    for (long k = 0; k < (long)nx * ny; ++k) da[k] = 0.0;
    extend_adjoint(nx, ny, a, Dc, da);
    free(Dc);
}

/* Heat misfit: the sensible heat released per unit area of each atmospheric
 * cell over the run, Q_I = sum over the fire cells k of I of
 * (F_k(start) - F_k(end)) H_s,k / (srx sry) -- the time integral of the
 * heat flux of eqs. (sensible-heat-flux, average), which telescopes -- and
 * J = 1/2 sum over the cells with a finite observation of (Q_I - q_obs,I)^2.
 * The run, gradients and outputs as in orc_adjoint.  Its seeds: dJ/dF at
 * the end through the quadrature of Sect. 3.3 (orc_cell_fuel_fraction with
 * the ghosts of orc_step) into dJ/dpsi at the end and dJ/dt_i (then eq.
 * set-ignition-time at each node's crossing step), and the moisture
 * dependence of H_s. */
double orc_adjoint_heat(const orc_grid *g, const double *co, const double *dco,
                        const double *mult, const double *dzdx, const double *dzdy,
                        const double *u, const double *v, double t0, double dt, int nsteps,
                        double *psi, double *tign, double *frac, const double *qobs,
                        double *g_mult, double *g_moist, double *g_u, double *g_v)
{
    int nx = g->nxa * g->srx, ny = g->nya * g->sry;
    long n = (long)nx * ny;
    int W = nx + 2;
    long ne = (long)W * (ny + 2);
    double r2 = (double)(g->srx * g->sry);
    double *states = malloc(sizeof(double) * n * (nsteps + 1));
    double *times = malloc(sizeof(double) * (nsteps + 1));
    double *tign0 = malloc(sizeof(double) * n), *frac0 = malloc(sizeof(double) * n);
    memcpy(tign0, tign, sizeof(double) * n);
    memcpy(frac0, frac, sizeof(double) * n);
    forward_run(g, co, mult, dzdx, dzdy, u, v, t0, dt, nsteps, psi, tign, frac, states, times);
    double t1 = times[nsteps];

    /* Q, J and dJ/dF per fire cell (0 under unobserved atmospheric cells) */
    double J = 0.0;
    double *gF = calloc(n, sizeof(double));
    for (long k = 0; k < n; ++k) g_moist[k] = 0.0;
    for (int Jc = 0; Jc < g->nya; ++Jc) {
        for (int Ic = 0; Ic < g->nxa; ++Ic) {
            double qo = qobs[Jc * g->nxa + Ic];
            if (!isfinite(qo)) continue;
            double q = 0.0;
            for (int j = Jc * g->sry; j < (Jc + 1) * g->sry; ++j)
                for (int i = Ic * g->srx; i < (Ic + 1) * g->srx; ++i) {
                    long k = (long)j * nx + i;
                    q += (frac0[k] - frac[k]) * co[k * CO_N + CO_HS];
                }
            q /= r2;
            J += 0.5 * (q - qo) * (q - qo);
            for (int j = Jc * g->sry; j < (Jc + 1) * g->sry; ++j)
                for (int i = Ic * g->srx; i < (Ic + 1) * g->srx; ++i) {
                    long k = (long)j * nx + i;
                    gF[k] = -(q - qo) * co[k * CO_N + CO_HS] / r2;
                    g_moist[k] = (q - qo) * (frac0[k] - frac[k]) * dco[k * CO_N + CO_HS] / r2;
                }
        }
    }

    /* the quadrature at the end of the run, as orc_step evaluated it */
    double *ext = malloc(sizeof(double) * ne), *ext_t = malloc(sizeof(double) * ne);
    orc_extend(nx, ny, psi, ext);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            ext_t[(j + 1) * W + (i + 1)] = psi[k] < 0.0 ? tign[k] : t1;
        }
    for (int j = 1; j <= ny; ++j) {
        ext_t[j * W] = ext_t[j * W + 1];
        ext_t[j * W + nx + 1] = ext_t[j * W + nx];
    }
    for (int i = 0; i < W; ++i) {
        ext_t[i] = ext_t[W + i];
        ext_t[(ny + 1) * W + i] = ext_t[ny * W + i];
    }
    for (long k = 0; k < ne; ++k)
        if (ext[k] >= 0.0) ext_t[k] = t1;
    double *Dp = calloc(ne, sizeof(double)), *Dt = calloc(ne, sizeof(double));
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            if (gF[k] == 0.0) continue;
            double p9[9], t9[9], dp9[9], dt9[9];
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    p9[b * 3 + a] = ext[(j + b) * W + (i + a)];
                    t9[b * 3 + a] = ext_t[(j + b) * W + (i + a)];
                }
            cell_fraction_partials(p9, t9, t1, co[k * CO_N + CO_TF], dp9, dt9);
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    Dp[(j + b) * W + (i + a)] += gF[k] * dp9[b * 3 + a];
                    Dt[(j + b) * W + (i + a)] += gF[k] * dt9[b * 3 + a];
                }
        }
    }
    /* dJ/dpsi at the end: through the ghosts of orc_extend */
    double *lam = calloc(n, sizeof(double));
    extend_adjoint(nx, ny, psi, Dp, lam);
    /* dJ/dt_i: the positions set to t1 carry nothing, the ghost copies
     * return to their sources (y then x), t_i only where psi < 0 */
    for (long k = 0; k < ne; ++k)
        if (ext[k] >= 0.0) Dt[k] = 0.0;
    for (int i = 0; i < W; ++i) {
        Dt[W + i] += Dt[i];
        Dt[ny * W + i] += Dt[(ny + 1) * W + i];
    }
    for (int j = 1; j <= ny; ++j) {
        Dt[j * W + 1] += Dt[j * W];
        Dt[j * W + nx] += Dt[j * W + nx + 1];
    }
    double *dJdt = malloc(sizeof(double) * n);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            long k = (long)j * nx + i;
            dJdt[k] = psi[k] < 0.0 ? Dt[(j + 1) * W + (i + 1)] : 0.0;
        }

    double *un = malloc(sizeof(double) * n), *vn = malloc(sizeof(double) * n);
    double *gun = calloc(n, sizeof(double)), *gvn = calloc(n, sizeof(double));
    orc_wind_at_nodes(g->nxa, g->nya, g->srx, g->sry, u, v, un, vn);
    for (long k = 0; k < n; ++k) g_mult[k] = 0.0;
    adjoint_sweep(g, co, dco, mult, dzdx, dzdy, un, vn, dt, nsteps, states, times, tign0, tign,
                  dJdt, lam, g_mult, g_moist, gun, gvn);
    wind_gather(g, gun, gvn, g_u, g_v);
    free(states); free(times); free(tign0); free(frac0); free(gF); free(ext); free(ext_t);
    free(Dp); free(Dt); free(lam); free(dJdt); free(un); free(vn); free(gun); free(gvn);
    return J;
}

double orc_adjoint(const orc_grid *g, const double *co, const double *dco, const double *mult,
                   const double *dzdx, const double *dzdy, const double *u, const double *v,
                   double t0, double dt, int nsteps, double *psi, double *tign, double *frac,
                   const double *tobs, double *g_mult, double *g_moist, double *g_u, double *g_v)
{
    int nx = g->nxa * g->srx, ny = g->nya * g->sry;
    long n = (long)nx * ny;
    double *states = malloc(sizeof(double) * n * (nsteps + 1));
    double *times = malloc(sizeof(double) * (nsteps + 1));
    double *tign0 = malloc(sizeof(double) * n);
    memcpy(tign0, tign, sizeof(double) * n);
    forward_run(g, co, mult, dzdx, dzdy, u, v, t0, dt, nsteps, psi, tign, frac, states, times);
    double J = 0.0;
    for (long k = 0; k < n; ++k)
        if (isfinite(tign[k]) && isfinite(tobs[k])) J += 0.5 * (tign[k] - tobs[k]) * (tign[k] - tobs[k]);
    /* dJ/dt_i at the observed nodes (NaN elsewhere) */
    double *dJdt = malloc(sizeof(double) * n);
    for (long k = 0; k < n; ++k) dJdt[k] = isfinite(tobs[k]) ? tign[k] - tobs[k] : NAN;

    double *un = malloc(sizeof(double) * n), *vn = malloc(sizeof(double) * n);
    double *gun = calloc(n, sizeof(double)), *gvn = calloc(n, sizeof(double));
    double *lam = calloc(n, sizeof(double));
    orc_wind_at_nodes(g->nxa, g->nya, g->srx, g->sry, u, v, un, vn);
    for (long k = 0; k < n; ++k) { g_mult[k] = 0.0; g_moist[k] = 0.0; }
    adjoint_sweep(g, co, dco, mult, dzdx, dzdy, un, vn, dt, nsteps, states, times, tign0, tign,
                  dJdt, lam, g_mult, g_moist, gun, gvn);
    wind_gather(g, gun, gvn, g_u, g_v);
    free(states); free(times); free(tign0); free(dJdt); free(un); free(vn);
    free(gun); free(gvn); free(lam);
    return J;
}

/* ------------------------------------------------------------------ */
/* Coupling with the atmosphere (Sect. "Coupling of the fire and the   */
/* atmospheric models"): the wind at z_f and the heat insertion.       */
/* ------------------------------------------------------------------ */

/* Wind at height z_f above the terrain by vertical log-linear
 * interpolation: at each of npts horizontal points, the piecewise linear
 * interpolant in ln z of the values u(z_0) = 0, u(z_1), u(z_2), ... at
 * ln z_0, ln z_1, ..., evaluated at ln z_f; 0 where z_f <= z_0.
 * u3d, z3d: [nz][npts] (level k of point p at k*npts + p), the wind and the
 * height above the terrain of the cell centres, increasing with k; z0:
 * [npts] roughness heights; out: [npts].
 * Readings: levels at or below z_0 are not used (the profile is 0 up to
 * z_0); above the highest level the top value is kept (the paper only
 * interpolates). */
void orc_wind_at_height(int nz, long npts, const double *u3d, const double *z3d,
                        const double *z0, double zf, double *out)
{
    for (long p = 0; p < npts; ++p) {
        double r = z0[p];
        if (!(zf > r)) { out[p] = 0.0; continue; }
        /* points of the interpolant: (ln z_0, 0), then levels above z_0 */
        double xl = log(r), ul = 0.0;   /* last point at or below ln z_f */
        double x = log(zf);
        double val = 0.0;
        int done = 0;
        for (int k = 0; k < nz; ++k) {
            double zk = z3d[(long)k * npts + p];
            if (!(zk > r)) continue;
            double xk = log(zk), uk = u3d[(long)k * npts + p];
            if (x <= xk) {
                val = ul + (uk - ul) * (x - xl) / (xk - xl);
                done = 1;
                break;
            }
            xl = xk;
            ul = uk;
        }
        out[p] = done ? val : ul;
    }
}

/* Heat insertion into the atmospheric tendencies of the potential
 * temperature and the vapour (the two equations after the fire step list):
 *   d(mu theta)/dt += mu phi_h / (sigma rho) * S(z),
 *   d(mu q_m)/dt   += mu phi_q / (L rho) * S(z),
 * with S the vertical profile of the inserted flux, exp(-z/z_ext).
 * Reading of the printed d/dz exp(-z/z_ext), whose sign would cool the air:
 * the source is the convergence of the upward flux phi exp(-z/z_ext), and
 * in a model layer between the face heights zw_k < zw_{k+1} it is the
 * layer average of that convergence,
 *   S_k = (exp(-zw_k/z_ext) - exp(-zw_{k+1}/z_ext)) / (zw_{k+1} - zw_k),
 * so that the column integral of sigma rho S_k dz_k times the heating is
 * phi_h (1 - exp(-zw_top/z_ext)).
 * hs, hl: [n] (n = nx*ny columns) sensible and latent flux densities
 * (W m^-2); zw: [nz+1][n] face heights above the terrain (zw_0 = 0);
 * rho: [nz][n] density (kg m^-3); mu: [n] (Pa); cp = sigma (J kg^-1 K^-1),
 * L (J kg^-1); rth, rqv: [nz][n], the sources are added to them. */
void orc_heat_insertion(int nz, long n, const double *hs, const double *hl,
                        const double *zw, const double *rho, const double *mu,
                        double zext, double cp, double L, double *rth, double *rqv)
{
    for (int k = 0; k < nz; ++k) {
        for (long p = 0; p < n; ++p) {
            double za = zw[(long)k * n + p], zb = zw[(long)(k + 1) * n + p];
            double S = (exp(-za / zext) - exp(-zb / zext)) / (zb - za);
            double r = rho[(long)k * n + p];
            rth[(long)k * n + p] += mu[p] * hs[p] / (cp * r) * S;
            rqv[(long)k * n + p] += mu[p] * hl[p] / (L * r) * S;
        }
    }
}
