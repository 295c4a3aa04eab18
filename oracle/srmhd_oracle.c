/*
 * srmhd_oracle.c -- plain FP64 CPU oracle of the CTU patch step for special
 * relativistic MHD with GLM cleaning (test infrastructure only; shares no
 * code with the CUDA path).
 *
 * What it follows (Mignone et al. 2012):
 *   - RMHD equations, total pressure and energy: Section 2.2, Eq. (rmhd);
 *     ideal-gas enthalpy w = rho + Gamma p/(Gamma-1), Eq. (gammaEos), or
 *     the Taub-Mathews enthalpy w = 5/2 p + sqrt(9/4 p^2 + rho^2),
 *     Eq. (TMEos).  Every function takes `gam`: Gamma of the ideal gas
 *     (> 1), or 0 for the Taub-Mathews equation of state;
 *   - GLM cleaning and its operator-split source: Section 3, Eq. (glm2x2);
 *   - unsplit update, n+1/2 Riemann problems, corner-coupled states with
 *     first-order transverse fluxes: Section 3.1, Eq. (update), (ctu_flux),
 *     (transv) with Pi = 0;
 *   - normal predictor in primitive variables (MUSCL-Hancock) with linear
 *     MC-limited primitive slopes and beta_+ = beta_- = 1: Section 3.3,
 *     Eq. (MUSCL-Hancock), (Linear), (MClim).
 * Not given by the paper, written here from the mathematics or a named
 * published method:
 *   - primitive recovery: Newton-Raphson on W = w gamma^2 (the variable of
 *     Mignone & McKinney 2007), safeguarded by bisection;
 *   - HLL fluxes (Harten, Lax & van Leer 1983) with the exact linear
 *     (B_n, psi) face solve of Dedner et al. (2002);
 *   - signal speeds: the relativistic sound-speed formula with the effective
 *     speed a^2 = c_s^2 + c_a^2 - c_s^2 c_a^2 (Leismann et al. 2005; Del Zanna
 *     et al. 2007), an upper bound of the fast magnetosonic speed that is
 *     exact for B = 0.
 * Variables: V = (rho, vx, vy, vz, p, Bx, By, Bz, psi),
 *            U = (D = rho gamma, mx, my, mz, E (= total energy - D), Bx, By, Bz, psi).
 * Layout as in ctu_oracle.c.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NVAR 9
#define NGHOST 4

static const int PERM_R[3][NVAR] = {
    {0, 1, 2, 3, 4, 5, 6, 7, 8},
    {0, 2, 1, 3, 4, 6, 5, 7, 8},
    {0, 3, 1, 2, 4, 7, 5, 6, 8},
};

/* Enthalpy density w(rho, p): Eq. (gammaEos) for gam > 0, Eq. (TMEos) for
 * gam == 0. */
static double enthalpy(double rho, double p, double gam)
{
    if (gam > 0.0)
        return rho + gam / (gam - 1.0) * p;
    return 2.5 * p + sqrt(2.25 * p * p + rho * rho);
}

/* Sound speed squared c_s^2 = (dp/de)_s / h for enthalpy density w:
 * Gamma p / w for the ideal gas; p (5 w - 8 p) / (3 w (w - p)) for the
 * Taub-Mathews equation of state (Mignone & McKinney 2007). */
static double sound2(double p, double w, double gam)
{
    if (gam > 0.0)
        return gam * p / w;
    return p * (5.0 * w - 8.0 * p) / (3.0 * w * (w - p));
}

/* U(V), Section 2.2: D = rho gamma, m = (W + B^2) v - (v.B) B,
 * E = W - p + (B^2 + E_el^2)/2 - D with W = w gamma^2, E_el = -v x B. */
void or_srmhd_prim2cons(const double *V, double gam, double *U)
{
    double rho = V[0], vx = V[1], vy = V[2], vz = V[3], p = V[4];
    double bx = V[5], by = V[6], bz = V[7];
    double v2 = vx * vx + vy * vy + vz * vz;
    double lor2 = 1.0 / (1.0 - v2);
    double lor = sqrt(lor2);
    double w = enthalpy(rho, p, gam);
    double W = w * lor2;
    double B2 = bx * bx + by * by + bz * bz;
    double vB = vx * bx + vy * by + vz * bz;
    double E2 = B2 * v2 - vB * vB;
    U[0] = rho * lor;
    U[1] = (W + B2) * vx - vB * bx;
    U[2] = (W + B2) * vy - vB * by;
    U[3] = (W + B2) * vz - vB * bz;
    U[4] = W - p + 0.5 * (B2 + E2) - U[0];
    U[5] = bx;
    U[6] = by;
    U[7] = bz;
    U[8] = V[8];
}

/* f(W) = W - p(W) + B^2 (1 + v^2(W))/2 - S^2/(2 W^2) - (E + D) and f'(W),
 * with v^2(W) = (m^2 W^2 + S^2 (2W + B^2)) / (W^2 (W + B^2)^2) and p from
 * w = W (1 - v^2) and rho = D sqrt(1 - v^2): the ideal gas
 * p = (Gamma-1)/Gamma (w - rho) (g1 = (Gamma-1)/Gamma > 0), or, for g1 = 0,
 * the inverse of Eq. (TMEos), p = (5 w - sqrt(9 w^2 + 16 rho^2))/8,
 * evaluated as 2 (w - rho)(w + rho)/(5 w + sqrt(9 w^2 + 16 rho^2)).
 * Returns 0 if v^2 >= 1 (W below the physical range), 1 otherwise. */
static int rec_eval(double W, double D, double m2, double S2, double B2, double tau, double g1,
                    double *f, double *df, double *v2o, double *po)
{
    double Wb = W + B2;
    double N = m2 * W * W + S2 * (2.0 * W + B2);
    double Dn = W * W * Wb * Wb;
    double v2 = N / Dn;
    double dN, dDn, dv2, s, p, dp;
    if (!(v2 < 1.0))
        return 0;
    dN = 2.0 * m2 * W + 2.0 * S2;
    dDn = 2.0 * W * Wb * (2.0 * W + B2);
    dv2 = (dN * Dn - N * dDn) / (Dn * Dn);
    s = sqrt(1.0 - v2);
    if (g1 > 0.0) {
        p = g1 * (W * (1.0 - v2) - D * s);
        dp = g1 * ((1.0 - v2) + dv2 * (0.5 * D / s - W));
    } else {
        double w = W * (1.0 - v2), rho = D * s;
        double q = sqrt(9.0 * w * w + 16.0 * rho * rho);
        double dpdw = (5.0 - 9.0 * w / q) / 8.0, dpdr = -2.0 * rho / q;
        p = 2.0 * (w - rho) * (w + rho) / (5.0 * w + q);
        /* dw/dW = (1 - v^2) - W dv^2/dW, drho/dW = -D dv^2/dW / (2 sqrt(1 - v^2)) */
        dp = dpdw * ((1.0 - v2) - W * dv2) - dpdr * 0.5 * D * dv2 / s;
    }
    *f = W - p + 0.5 * B2 * (1.0 + v2) - 0.5 * S2 / (W * W) - tau;
    *df = 1.0 - dp + 0.5 * B2 * dv2 + S2 / (W * W * W);
    *v2o = v2;
    *po = p;
    return 1;
}

/* V(U) by safeguarded Newton-Raphson on W.  Returns 0 on success, 1 for a
 * non-physical result (rho <= 0, p <= 0, v^2 >= 1) and 2 if the iteration
 * did not converge in 200 steps. */
int or_srmhd_cons2prim(const double *U, double gam, double *V)
{
    double D = U[0], mx = U[1], my = U[2], mz = U[3], tau = U[4] + U[0];
    double bx = U[5], by = U[6], bz = U[7];
    double m2 = mx * mx + my * my + mz * mz;
    double B2 = bx * bx + by * by + bz * bz;
    double S = mx * bx + my * by + mz * bz;
    double S2 = S * S;
    double g1 = gam > 0.0 ? (gam - 1.0) / gam : 0.0;
    double Wlo = 0.0, Whi, W, f = 0.0, df = 1.0, v2 = 0.0, p = 0.0;
    int it, k, conv = 0;

    if (!(D > 0.0) || !(tau > 0.0))
        return 1;
    /* upper bracket: f > 0 for all large W */
    Whi = tau + 1.0e-300;
    for (k = 0; k < 400; k++) {
        if (rec_eval(Whi, D, m2, S2, B2, tau, g1, &f, &df, &v2, &p) && f > 0.0)
            break;
        Wlo = Whi;
        Whi *= 2.0;
    }
    W = Whi;
    for (it = 0; it < 200; it++) {
        double Wn;
        if (!rec_eval(W, D, m2, S2, B2, tau, g1, &f, &df, &v2, &p)) {
            Wlo = W;
            W = 0.5 * (Wlo + Whi);
            continue;
        }
        if (f > 0.0)
            Whi = W;
        else
            Wlo = W;
        Wn = W - f / df;
        if (!(Wn > Wlo && Wn < Whi))
            Wn = 0.5 * (Wlo + Whi);
        if (fabs(Wn - W) <= 1.0e-15 * W) {
            W = Wn;
            conv = 1;
            break;
        }
        W = Wn;
    }
    if (!conv)
        return 2;
    if (!rec_eval(W, D, m2, S2, B2, tau, g1, &f, &df, &v2, &p))
        return 1;
    V[1] = (mx + S * bx / W) / (W + B2);
    V[2] = (my + S * by / W) / (W + B2);
    V[3] = (mz + S * bz / W) / (W + B2);
    V[0] = D * sqrt(1.0 - v2);
    V[4] = p;
    V[5] = bx;
    V[6] = by;
    V[7] = bz;
    V[8] = U[8];
    return (V[0] > 0.0 && p > 0.0) ? 0 : 1;
}

/* Lower and upper signal speeds along the local normal (Vloc[1] = v_n). */
void or_srmhd_fast_speeds(const double *V, double gam, double *lm, double *lp)
{
    double rho = V[0], vn = V[1], p = V[4];
    double v2 = V[1] * V[1] + V[2] * V[2] + V[3] * V[3];
    double B2 = V[5] * V[5] + V[6] * V[6] + V[7] * V[7];
    double vB = V[1] * V[5] + V[2] * V[6] + V[3] * V[7];
    double rh = enthalpy(rho, p, gam); /* rho h = w */
    double cs2 = sound2(p, rh, gam);
    double b2 = B2 * (1.0 - v2) + vB * vB; /* comoving b^2 = B^2/gamma^2 + (v.B)^2 */
    double ca2 = b2 / (rh + b2);
    double a2 = cs2 + ca2 - cs2 * ca2;
    double den = 1.0 - v2 * a2;
    double disc = a2 * (1.0 - v2) * (1.0 - v2 * a2 - vn * vn * (1.0 - a2));
    double sq;
    if (disc < 0.0)
        disc = 0.0;
    sq = sqrt(disc);
    *lm = (vn * (1.0 - a2) - sq) / den;
    *lp = (vn * (1.0 - a2) + sq) / den;
}

/* Physical RMHD flux along the local normal, Eq. (rmhd): F[5], F[8] (the
 * GLM pair) = (psi, c_h^2 B_n). */
static void rflux(const double *V, const double *U, double gam, double ch, double *F)
{
    double vx = V[1], vy = V[2], vz = V[3], p = V[4];
    double bx = V[5], by = V[6], bz = V[7];
    double v2 = vx * vx + vy * vy + vz * vz;
    double lor2 = 1.0 / (1.0 - v2);
    double w = enthalpy(V[0], p, gam);
    double W = w * lor2;
    double ex = -(vy * bz - vz * by), ey = -(vz * bx - vx * bz), ez = -(vx * by - vy * bx);
    double B2 = bx * bx + by * by + bz * bz;
    double E2 = ex * ex + ey * ey + ez * ez;
    double pt = p + 0.5 * (B2 + E2);
    F[0] = U[0] * vx;
    F[1] = W * vx * vx - bx * bx - ex * ex + pt;
    F[2] = W * vx * vy - bx * by - ex * ey;
    F[3] = W * vx * vz - bx * bz - ex * ez;
    F[4] = U[1] - U[0] * vx;
    F[5] = V[8];
    F[6] = vx * by - bx * vy;
    F[7] = vx * bz - bx * vz;
    F[8] = ch * ch * bx;
}

/* HLL flux with the exact (B_n, psi) face solve.  Returns 1 if an input
 * state is unphysical. */
int or_srmhd_riemann(const double *VL0, const double *VR0, double gam, double ch, double *F)
{
    double VL[NVAR], VR[NVAR], UL[NVAR], UR[NVAR], FL[NVAR], FR[NVAR];
    double Bm, pm, lmL, lpL, lmR, lpR, SL, SR;
    int q, bad;
    for (q = 0; q < NVAR; q++) {
        VL[q] = VL0[q];
        VR[q] = VR0[q];
    }
    bad = !(VL[0] > 0.0 && VL[4] > 0.0 && VR[0] > 0.0 && VR[4] > 0.0);
    Bm = 0.5 * (VL[5] + VR[5]) - 0.5 * (VR[8] - VL[8]) / ch;
    pm = 0.5 * (VL[8] + VR[8]) - 0.5 * ch * (VR[5] - VL[5]);
    VL[5] = Bm;
    VR[5] = Bm;
    or_srmhd_prim2cons(VL, gam, UL);
    or_srmhd_prim2cons(VR, gam, UR);
    rflux(VL, UL, gam, ch, FL);
    rflux(VR, UR, gam, ch, FR);
    or_srmhd_fast_speeds(VL, gam, &lmL, &lpL);
    or_srmhd_fast_speeds(VR, gam, &lmR, &lpR);
    SL = fmin(lmL, lmR);
    SR = fmax(lpL, lpR);
    if (SL >= 0.0) {
        for (q = 0; q < NVAR; q++)
            F[q] = FL[q];
    } else if (SR <= 0.0) {
        for (q = 0; q < NVAR; q++)
            F[q] = FR[q];
    } else {
        for (q = 0; q < NVAR; q++)
            F[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) / (SR - SL);
    }
    F[5] = pm;
    F[8] = ch * ch * Bm;
    return bad;
}

static double mm_r(double a, double b)
{
    if (a > 0.0 && b > 0.0)
        return fmin(a, b);
    if (a < 0.0 && b < 0.0)
        return fmax(a, b);
    return 0.0;
}

/* MUSCL-Hancock normal predictor of one cell, Section 3.3 (beta = 1):
 * vs[0..2] = V_(i-1), V_i, V_(i+1) (local order), U0 = U_i^n (local order).
 * Outputs V*_(i,+), V*_(i,-).  Returns nonzero on a failed recovery. */
int or_srmhd_mh_predict(const double *vs, const double *U0, double gam, double ch, double dtdx,
                        double *Vp, double *Vm)
{
    double dV[NVAR], Vpl[NVAR], Vmi[NVAR], Up[NVAR], Um[NVAR], Fp[NVAR], Fm[NVAR], Us[NVAR], Vs[NVAR];
    int q, st;
    for (q = 0; q < NVAR; q++) {
        double dl = vs[NVAR + q] - vs[q], dr = vs[2 * NVAR + q] - vs[NVAR + q];
        dV[q] = mm_r(0.5 * (dl + dr), 2.0 * mm_r(dl, dr)); /* MC, Eq. (MClim) */
        Vpl[q] = vs[NVAR + q] + 0.5 * dV[q];
        Vmi[q] = vs[NVAR + q] - 0.5 * dV[q];
    }
    or_srmhd_prim2cons(Vpl, gam, Up);
    or_srmhd_prim2cons(Vmi, gam, Um);
    rflux(Vpl, Up, gam, ch, Fp);
    rflux(Vmi, Um, gam, ch, Fm);
    for (q = 0; q < NVAR; q++)
        Us[q] = U0[q] - 0.5 * dtdx * (Fp[q] - Fm[q]);
    st = or_srmhd_cons2prim(Us, gam, Vs);
    for (q = 0; q < NVAR; q++) {
        Vp[q] = Vs[q] + 0.5 * dV[q];
        Vm[q] = Vs[q] - 0.5 * dV[q];
    }
    return st;
}

typedef struct {
    int n[3], g[3], N[3];
    long ncell;
} rgrid;

static void rgrid_init(rgrid *G, int nx, int ny, int nz, int ndim)
{
    int d;
    G->n[0] = nx;
    G->n[1] = ny;
    G->n[2] = nz;
    for (d = 0; d < 3; d++) {
        G->g[d] = d < ndim ? NGHOST : 0;
        G->N[d] = G->n[d] + 2 * G->g[d];
    }
    G->ncell = (long)G->N[0] * G->N[1] * G->N[2];
}

static long rcidx(const rgrid *G, const int *c)
{
    return ((long)(c[2] + G->g[2]) * G->N[1] + (c[1] + G->g[1])) * G->N[0] + (c[0] + G->g[0]);
}

static long rstride(const rgrid *G, int d)
{
    return d == 0 ? 1 : (d == 1 ? G->N[0] : (long)G->N[0] * G->N[1]);
}

/* max over interior cells of max_d max(|lambda_-|, |lambda_+|)/dx_d.
 * Returns -1 if a recovery failed. */
double or_srmhd_max_speed(const double *U, int nx, int ny, int nz, int ndim, double dx, double dy,
                          double dz, double gam)
{
    rgrid G;
    double h[3] = {dx, dy, dz}, m = 0.0;
    int c[3], d, q;
    rgrid_init(&G, nx, ny, nz, ndim);
    for (c[2] = 0; c[2] < G.n[2]; c[2]++)
        for (c[1] = 0; c[1] < G.n[1]; c[1]++)
            for (c[0] = 0; c[0] < G.n[0]; c[0]++) {
                long id = rcidx(&G, c);
                double Uc[NVAR], V[NVAR], Vl[NVAR], lm, lp;
                for (q = 0; q < NVAR; q++)
                    Uc[q] = U[q * G.ncell + id];
                if (or_srmhd_cons2prim(Uc, gam, V))
                    return -1.0;
                for (d = 0; d < ndim; d++) {
                    double s;
                    for (q = 0; q < NVAR; q++)
                        Vl[q] = V[PERM_R[d][q]];
                    or_srmhd_fast_speeds(Vl, gam, &lm, &lp);
                    s = fmax(fabs(lm), fabs(lp)) / h[d];
                    if (s > m)
                        m = s;
                }
            }
    return m;
}

/* One CTU step of a ghost-filled patch (same contract, windows and return
 * value as or_mhd_step). */
int or_srmhd_step(const double *U, double *Unew, int nx, int ny, int nz, int ndim, double dx,
                  double dy, double dz, double dt, double ch, double gam, double glm_alpha,
                  const long *win, const double *wgt, int nwin, double *reg)
{
    rgrid G;
    double h[3] = {dx, dy, dz};
    double *V, *F1[3] = {0, 0, 0}, *Up[3] = {0, 0, 0}, *Um[3] = {0, 0, 0}, *F[3] = {0, 0, 0};
    int c[3], d, q, bad = 0;
    long nc;

    rgrid_init(&G, nx, ny, nz, ndim);
    nc = G.ncell;
    V = (double *)malloc(sizeof(double) * NVAR * nc);

    /* 1. V = V(U) everywhere */
    for (long id = 0; id < nc; id++) {
        double Uc[NVAR], Vc[NVAR];
        for (q = 0; q < NVAR; q++)
            Uc[q] = U[q * nc + id];
        if (or_srmhd_cons2prim(Uc, gam, Vc)) {
            bad++;
            for (q = 0; q < NVAR; q++)
                Vc[q] = NAN;
        }
        for (q = 0; q < NVAR; q++)
            V[q * nc + id] = Vc[q];
    }

    /* 2. first-order transverse fluxes */
    for (d = 0; d < ndim; d++) {
        long st = rstride(&G, d);
        int lo[3], hi[3], e;
        F1[d] = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        for (e = 0; e < 3; e++) {
            if (e >= ndim) {
                lo[e] = 0;
                hi[e] = 0;
            } else if (e == d) {
                lo[e] = -1;
                hi[e] = G.n[e] - 1;
            } else {
                lo[e] = -1;
                hi[e] = G.n[e];
            }
        }
        for (c[2] = lo[2]; c[2] <= hi[2]; c[2]++)
            for (c[1] = lo[1]; c[1] <= hi[1]; c[1]++)
                for (c[0] = lo[0]; c[0] <= hi[0]; c[0]++) {
                    long id = rcidx(&G, c);
                    double VL[NVAR], VR[NVAR], Fl[NVAR];
                    for (q = 0; q < NVAR; q++) {
                        VL[q] = V[PERM_R[d][q] * nc + id];
                        VR[q] = V[PERM_R[d][q] * nc + id + st];
                    }
                    or_srmhd_riemann(VL, VR, gam, ch, Fl);
                    for (q = 0; q < NVAR; q++)
                        F1[d][PERM_R[d][q] * nc + id] = Fl[q];
                }
    }

    /* 3. MUSCL-Hancock normal predictors + transverse correction */
    for (d = 0; d < ndim; d++) {
        long st = rstride(&G, d);
        int lo[3], hi[3], e, tr[2], ntr = 0;
        for (e = 0; e < ndim; e++)
            if (e != d)
                tr[ntr++] = e;
        Up[d] = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        Um[d] = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        for (e = 0; e < 3; e++) {
            lo[e] = 0;
            hi[e] = e < ndim ? G.n[e] - 1 : 0;
        }
        lo[d] = -1;
        hi[d] = G.n[d];
        for (c[2] = lo[2]; c[2] <= hi[2]; c[2]++)
            for (c[1] = lo[1]; c[1] <= hi[1]; c[1]++)
                for (c[0] = lo[0]; c[0] <= hi[0]; c[0]++) {
                    long id = rcidx(&G, c);
                    double vs[3 * NVAR], U0[NVAR], Vp[NVAR], Vm[NVAR], Ul[NVAR], Ug[NVAR], T[NVAR];
                    int l, t;
                    for (l = 0; l < 3; l++)
                        for (q = 0; q < NVAR; q++)
                            vs[l * NVAR + q] = V[PERM_R[d][q] * nc + id + (l - 1) * st];
                    for (q = 0; q < NVAR; q++)
                        U0[q] = U[PERM_R[d][q] * nc + id];
                    if (or_srmhd_mh_predict(vs, U0, gam, ch, dt / h[d], Vp, Vm))
                        bad++;
                    for (q = 0; q < NVAR; q++)
                        T[q] = 0.0;
                    for (t = 0; t < ntr; t++) {
                        int e2 = tr[t];
                        long st2 = rstride(&G, e2);
                        for (q = 0; q < NVAR; q++)
                            T[q] += (F1[e2][q * nc + id - st2] - F1[e2][q * nc + id]) / h[e2];
                    }
                    or_srmhd_prim2cons(Vp, gam, Ul);
                    for (q = 0; q < NVAR; q++)
                        Ug[PERM_R[d][q]] = Ul[q];
                    for (q = 0; q < NVAR; q++)
                        Up[d][q * nc + id] = Ug[q] + 0.5 * dt * T[q];
                    or_srmhd_prim2cons(Vm, gam, Ul);
                    for (q = 0; q < NVAR; q++)
                        Ug[PERM_R[d][q]] = Ul[q];
                    for (q = 0; q < NVAR; q++)
                        Um[d][q * nc + id] = Ug[q] + 0.5 * dt * T[q];
                }
    }

    /* 4. n+1/2 Riemann problems */
    for (d = 0; d < ndim; d++) {
        long st = rstride(&G, d);
        int lo[3], hi[3], e;
        F[d] = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        for (e = 0; e < 3; e++) {
            lo[e] = 0;
            hi[e] = e < ndim ? G.n[e] - 1 : 0;
        }
        lo[d] = -1;
        for (c[2] = lo[2]; c[2] <= hi[2]; c[2]++)
            for (c[1] = lo[1]; c[1] <= hi[1]; c[1]++)
                for (c[0] = lo[0]; c[0] <= hi[0]; c[0]++) {
                    long id = rcidx(&G, c);
                    double UL[NVAR], UR[NVAR], VLg[NVAR], VRg[NVAR], VL[NVAR], VR[NVAR], Fl[NVAR];
                    for (q = 0; q < NVAR; q++) {
                        UL[q] = Up[d][q * nc + id];
                        UR[q] = Um[d][q * nc + id + st];
                    }
                    if (or_srmhd_cons2prim(UL, gam, VLg))
                        bad++;
                    if (or_srmhd_cons2prim(UR, gam, VRg))
                        bad++;
                    for (q = 0; q < NVAR; q++) {
                        VL[q] = VLg[PERM_R[d][q]];
                        VR[q] = VRg[PERM_R[d][q]];
                    }
                    or_srmhd_riemann(VL, VR, gam, ch, Fl);
                    for (q = 0; q < NVAR; q++)
                        F[d][PERM_R[d][q] * nc + id] = Fl[q];
                }
    }

    /* 5. update + psi source */
    memcpy(Unew, U, sizeof(double) * NVAR * nc);
    {
        double hmin = h[0], damp;
        for (d = 1; d < ndim; d++)
            hmin = fmin(hmin, h[d]);
        damp = exp(-glm_alpha * ch * dt / hmin);
        for (c[2] = 0; c[2] < G.n[2]; c[2]++)
            for (c[1] = 0; c[1] < G.n[1]; c[1]++)
                for (c[0] = 0; c[0] < G.n[0]; c[0]++) {
                    long id = rcidx(&G, c);
                    for (q = 0; q < NVAR; q++) {
                        double s = 0.0;
                        for (d = 0; d < ndim; d++)
                            s += (F[d][q * nc + id - rstride(&G, d)] - F[d][q * nc + id]) / h[d];
                        Unew[q * nc + id] = U[q * nc + id] + dt * s;
                    }
                    Unew[8 * nc + id] *= damp;
                }
    }

    /* 6. flux registers, Eq. (fluxcorr) */
    for (int w = 0; w < nwin; w++) {
        const long *W = win + 7 * w;
        int wd = (int)W[0], a = wd == 0 ? 1 : 0, b = wd == 2 ? 1 : 2;
        long na = W[3] - W[2], nb = W[5] - W[4];
        double area = h[a] * h[b];
        for (q = 0; q < NVAR; q++)
            for (long jb = 0; jb < nb; jb++)
                for (long ja = 0; ja < na; ja++) {
                    c[wd] = (int)W[1] - 1;
                    c[a] = (int)(W[2] + ja);
                    c[b] = (int)(W[4] + jb);
                    reg[W[6] + (q * nb + jb) * na + ja] +=
                        wgt[w] * dt * area * F[wd][q * nc + rcidx(&G, c)];
                }
    }

    free(V);
    for (d = 0; d < 3; d++) {
        free(F1[d]);
        free(Up[d]);
        free(Um[d]);
        free(F[d]);
    }
    return bad;
}
