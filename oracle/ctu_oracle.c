/*
 * ctu_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the
 * unsplit CTU patch step for ideal MHD with GLM divergence cleaning.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.  Build with
 *     gcc -O2 -ffp-contract=off -fPIC -shared
 * so that every expression is rounded exactly as written.
 *
 * What it follows (Mignone et al., "The PLUTO code for adaptive mesh
 * computations in astrophysical fluid dynamics"):
 *   - ideal MHD equations and ideal-gas energy: Section 2.1, Eq. (1)-(2)
 *   - GLM cleaning: Section 3, Eq. (glm2x2); psi source operator-split
 *   - unsplit update:             Section 3.1, Eq. (update), (incrementop_hyp)
 *   - n+1/2 face Riemann problems: Section 3.1, Eq. (ctu_flux)
 *   - corner-coupled states with first-order transverse fluxes:
 *                                  Section 3.1, Eq. (transv) with Pi = 0
 *   - CFL time step:               Section 3.1, Eq. (Ca)
 *   - characteristic projection:   Section 3.2, Eq. (char_var)
 *   - characteristic tracing, no reference state or the reference states
 *     w_(+/-), w_(i,0) and Colella-Woodward's with upwind selection:
 *                                  Section 3.2, Eq. (wnorm_predp), (wnorm_predm)
 *   - right-eigenvector recombination with the S_Bx and S_psi sources:
 *                                  Section 3.2 (V*_{i,+/-} expansion)
 *   - PPM, MC limiter, MinMod, parabolic limiter:
 *                                  Section 3.2, Eq. (ppm1), (MClim), (minmod),
 *                                  (ppm_parabolic_lim)
 *   - linear reconstruction:       Section 3.2, Eq. (Linear) with the MC,
 *                                  MinMod, harmonic (harmonic_lim) or Van
 *                                  Albada (vanalbada_lim) slope
 *   - improved third-order WENO:   Section 3.2, Eq. (WENO3), (WENO3a)
 *   - flux-register contribution:  Section 4.2, Eq. (fluxcorr)
 *   - optional density and pressure floors on the updated state: a reading
 *     (the paper fixes none), or_mhd_floor
 * The paper gives neither the primitive eigenvectors nor the Riemann solver
 * formulas; they are written here from the mathematics: the eigenvectors are
 * derived from the primitive Jacobian of Eq. (1) (Roe-Balsara normalisation),
 * the solver is HLLD (Miyoshi & Kusano 2005) with the exact linear (B_n, psi)
 * face solve of Dedner et al. (2002).
 *
 * Variable order.  Primitive V = (rho, vx, vy, vz, p, Bx, By, Bz, psi),
 * conservative U = (rho, mx, my, mz, E, Bx, By, Bz, psi).  Arrays are SoA:
 * U[var * ncell + cell], cell = (k * NY + j) * NX + i over the ghosted patch,
 * x fastest.  Active dimensions carry 4 ghost cells per side, inactive ones
 * (ndim < 3) carry none and have n = 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NVAR 9
#define NGHOST 4

/* Local 1-D frame for a sweep along d: local component q reads global
 * component PERM[d][q].  Local order: (rho, v_n, v_t1, v_t2, p, B_n, B_t1,
 * B_t2, psi) with (t1, t2) = (y, z), (x, z), (x, y) for d = x, y, z. */
static const int PERM[3][NVAR] = {
    {0, 1, 2, 3, 4, 5, 6, 7, 8},
    {0, 2, 1, 3, 4, 6, 5, 7, 8},
    {0, 3, 1, 2, 4, 7, 5, 6, 8},
};

/* ------------------------------------------------------------------ */
/* Equation of state and variable maps, Section 2.1                    */
/* ------------------------------------------------------------------ */

/* U(V): E = p/(Gamma-1) + rho v^2/2 + B^2/2 (ideal gas, Section 2.1). */
void or_mhd_prim2cons(const double *V, double gam, double *U)
{
    double rho = V[0];
    double v2 = V[1] * V[1] + V[2] * V[2] + V[3] * V[3];
    double B2 = V[5] * V[5] + V[6] * V[6] + V[7] * V[7];
    U[0] = rho;
    U[1] = rho * V[1];
    U[2] = rho * V[2];
    U[3] = rho * V[3];
    U[4] = V[4] / (gam - 1.0) + 0.5 * rho * v2 + 0.5 * B2;
    U[5] = V[5];
    U[6] = V[6];
    U[7] = V[7];
    U[8] = V[8];
}

/* V(U): p = (Gamma-1)(E - m^2/(2 rho) - B^2/2).  Returns 1 when rho <= 0 or
 * p <= 0 (or NaN), 0 otherwise. */
int or_mhd_cons2prim(const double *U, double gam, double *V)
{
    double rho = U[0];
    double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    double B2 = U[5] * U[5] + U[6] * U[6] + U[7] * U[7];
    V[0] = rho;
    V[1] = U[1] / rho;
    V[2] = U[2] / rho;
    V[3] = U[3] / rho;
    V[4] = (gam - 1.0) * (U[4] - 0.5 * m2 / rho - 0.5 * B2);
    V[5] = U[5];
    V[6] = U[6];
    V[7] = U[7];
    V[8] = U[8];
    return (rho > 0.0 && V[4] > 0.0) ? 0 : 1;
}

/* Fast magnetosonic speed along the local normal:
 * c_f^2 = ( a^2 + b^2 + sqrt((a^2 - b^2)^2 + 4 a^2 b_t^2) ) / 2,
 * the larger root of c^4 - (a^2 + b^2) c^2 + a^2 b_n^2 = 0 written with a
 * non-negative discriminant. */
double or_mhd_cfast(const double *Vloc, double gam)
{
    double rho = Vloc[0];
    double a2 = gam * Vloc[4] / rho;
    double bn2 = Vloc[5] * Vloc[5] / rho;
    double bt2 = (Vloc[6] * Vloc[6] + Vloc[7] * Vloc[7]) / rho;
    double b2 = bn2 + bt2;
    double disc = sqrt((a2 - b2) * (a2 - b2) + 4.0 * a2 * bt2);
    return sqrt(0.5 * (a2 + b2 + disc));
}

/* Physical MHD flux along the local normal, Eq. (1).  F[5] (B_n) and F[8]
 * (psi) are left at zero: the GLM face solve supplies them. */
static void mhd_flux(const double *V, const double *U, double *F)
{
    double rho = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
    double Bn = V[5], B1 = V[6], B2 = V[7];
    double Bsq = Bn * Bn + B1 * B1 + B2 * B2;
    double pt = p + 0.5 * Bsq;
    double vB = u * Bn + v * B1 + w * B2;
    F[0] = rho * u;
    F[1] = rho * u * u + pt - Bn * Bn;
    F[2] = rho * u * v - Bn * B1;
    F[3] = rho * u * w - Bn * B2;
    F[4] = (U[4] + pt) * u - Bn * vB;
    F[5] = 0.0;
    F[6] = u * B1 - Bn * v;
    F[7] = u * B2 - Bn * w;
    F[8] = 0.0;
}

/* ------------------------------------------------------------------ */
/* Eigen-structure of the primitive system along the local normal.     */
/* ------------------------------------------------------------------ */
/*
 * The 7-wave block acts on (rho, v_n, v_t1, v_t2, p, B_t1, B_t2) with B_n a
 * parameter; the 2-wave GLM block acts on (B_n, psi) with matrix
 * [[0, 1], [c_h^2, 0]].  Waves, in order of speed:
 *   0: v-c_f  1: v-c_a  2: v-c_s  3: v  4: v+c_s  5: v+c_a  6: v+c_f
 *   7: -c_h   8: +c_h
 * R[k][q] is component q of right eigenvector k, L[k][q] of left eigenvector
 * k, in the local order; L R = I.  The coupling of the 7-wave block to
 * d(B_n)/dn and d(psi)/dn is not part of this block: the step adds it as the
 * S_Bx, S_psi source of Section 3.2.
 */
void or_mhd_eigen(const double *V, double gam, double ch,
                  double *lam, double *L, double *R)
{
    int k, q;
    double rho = V[0], u = V[1], p = V[4];
    double Bn = V[5], B1 = V[6], B2 = V[7];
    double a2 = gam * p / rho;
    double a = sqrt(a2);
    double srho = sqrt(rho);
    double bn2 = Bn * Bn / rho;
    double bt2 = (B1 * B1 + B2 * B2) / rho;
    double b2 = bn2 + bt2;
    double disc = sqrt((a2 - b2) * (a2 - b2) + 4.0 * a2 * bt2); /* c_f^2 - c_s^2 */
    double cf2 = 0.5 * (a2 + b2 + disc);
    double cs2 = a2 * bn2 / cf2; /* c_f^2 c_s^2 = a^2 b_n^2 */
    double cf = sqrt(cf2), cs = sqrt(cs2), ca = sqrt(bn2);
    double af, as, b1, b2n, S, bt;
    double fa, sa; /* a^2 - c_s^2 and c_f^2 - a^2, each without cancellation */

    if (a2 >= b2) {
        fa = 0.5 * (a2 - b2 + disc);
        sa = (disc + (a2 - b2) > 0.0) ? 2.0 * a2 * bt2 / (disc + (a2 - b2)) : 0.0;
    } else {
        sa = 0.5 * (b2 - a2 + disc);
        fa = 2.0 * a2 * bt2 / (disc + (b2 - a2));
    }
    if (disc > 0.0) {
        af = sqrt(fa / disc);
        as = sqrt(sa / disc);
    } else { /* triple umbilic point: a = |b_n|, b_t = 0 */
        af = 1.0;
        as = 0.0;
    }
    bt = sqrt(B1 * B1 + B2 * B2);
    if (bt2 > 1.0e-24 * a2) {
        b1 = B1 / bt;
        b2n = B2 / bt;
    } else {
        b1 = 1.0 / sqrt(2.0);
        b2n = 1.0 / sqrt(2.0);
    }
    S = copysign(1.0, Bn);

    for (k = 0; k < NVAR * NVAR; k++) {
        L[k] = 0.0;
        R[k] = 0.0;
    }
#define RR(k, q) R[(k) * NVAR + (q)]
#define LL(k, q) L[(k) * NVAR + (q)]
    lam[0] = u - cf;
    lam[1] = u - ca;
    lam[2] = u - cs;
    lam[3] = u;
    lam[4] = u + cs;
    lam[5] = u + ca;
    lam[6] = u + cf;
    lam[7] = -ch;
    lam[8] = ch;

    /* fast waves, s = -1 (k = 0) and s = +1 (k = 6) */
    for (q = 0; q < 2; q++) {
        double s = q == 0 ? -1.0 : 1.0;
        k = q == 0 ? 0 : 6;
        RR(k, 0) = rho * af;
        RR(k, 1) = s * af * cf;
        RR(k, 2) = -s * as * cs * S * b1;
        RR(k, 3) = -s * as * cs * S * b2n;
        RR(k, 4) = rho * af * a2;
        RR(k, 6) = as * srho * a * b1;
        RR(k, 7) = as * srho * a * b2n;
        LL(k, 1) = s * af * cf / (2.0 * a2);
        LL(k, 2) = -s * as * cs * S * b1 / (2.0 * a2);
        LL(k, 3) = -s * as * cs * S * b2n / (2.0 * a2);
        LL(k, 4) = af / (2.0 * rho * a2);
        LL(k, 6) = as * b1 / (2.0 * srho * a);
        LL(k, 7) = as * b2n / (2.0 * srho * a);
    }
    /* Alfven waves, k = 1 (s = -1) and k = 5 (s = +1) */
    for (q = 0; q < 2; q++) {
        double s = q == 0 ? -1.0 : 1.0;
        k = q == 0 ? 1 : 5;
        RR(k, 2) = -b2n;
        RR(k, 3) = b1;
        RR(k, 6) = s * S * srho * b2n;
        RR(k, 7) = -s * S * srho * b1;
        LL(k, 2) = -0.5 * b2n;
        LL(k, 3) = 0.5 * b1;
        LL(k, 6) = s * S * b2n / (2.0 * srho);
        LL(k, 7) = -s * S * b1 / (2.0 * srho);
    }
    /* slow waves, k = 2 (s = -1) and k = 4 (s = +1) */
    for (q = 0; q < 2; q++) {
        double s = q == 0 ? -1.0 : 1.0;
        k = q == 0 ? 2 : 4;
        RR(k, 0) = rho * as;
        RR(k, 1) = s * as * cs;
        RR(k, 2) = s * af * cf * S * b1;
        RR(k, 3) = s * af * cf * S * b2n;
        RR(k, 4) = rho * as * a2;
        RR(k, 6) = -af * srho * a * b1;
        RR(k, 7) = -af * srho * a * b2n;
        LL(k, 1) = s * as * cs / (2.0 * a2);
        LL(k, 2) = s * af * cf * S * b1 / (2.0 * a2);
        LL(k, 3) = s * af * cf * S * b2n / (2.0 * a2);
        LL(k, 4) = as / (2.0 * rho * a2);
        LL(k, 6) = -af * b1 / (2.0 * srho * a);
        LL(k, 7) = -af * b2n / (2.0 * srho * a);
    }
    /* entropy wave */
    RR(3, 0) = 1.0;
    LL(3, 0) = 1.0;
    LL(3, 4) = -1.0 / a2;
    /* GLM waves on (B_n, psi) */
    RR(7, 5) = 1.0;
    RR(7, 8) = -ch;
    RR(8, 5) = 1.0;
    RR(8, 8) = ch;
    LL(7, 5) = 0.5;
    LL(7, 8) = -0.5 / ch;
    LL(8, 5) = 0.5;
    LL(8, 8) = 0.5 / ch;
#undef RR
#undef LL
}

/* ------------------------------------------------------------------ */
/* Riemann solver: GLM (B_n, psi) face solve + HLLD                    */
/* ------------------------------------------------------------------ */
/*
 * Numerical flux R(V_L, V_R) along the local normal.  The linear 2x2 GLM
 * system of Eq. (glm2x2) is solved exactly at the face (Dedner et al. 2002):
 *   B_m   = (B_nL + B_nR)/2 - (psi_R - psi_L)/(2 c_h)
 *   psi_m = (psi_L + psi_R)/2 - c_h (B_nR - B_nL)/2
 * with fluxes F(B_n) = psi_m, F(psi) = c_h^2 B_m; both states then carry
 * B_n = B_m (pressure kept) into the HLLD solver of Miyoshi & Kusano (2005).
 * Returns 1 if an input state has rho <= 0 or p <= 0.
 */
int or_mhd_riemann(const double *VL0, const double *VR0, double gam, double ch,
                   double *F)
{
    double VL[NVAR], VR[NVAR], UL[NVAR], UR[NVAR], FL[NVAR], FR[NVAR];
    double Bm, pm, Bn, cfL, cfR, cmax, SL, SR;
    double sdL, sdR, den, SM, pts;
    double rsL, rsR, vsL, vsR, wsL, wsR, B1sL, B1sR, B2sL, B2sR, EsL, EsR;
    double UsL[NVAR], UsR[NVAR];
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
    Bn = Bm;

    or_mhd_prim2cons(VL, gam, UL);
    or_mhd_prim2cons(VR, gam, UR);
    mhd_flux(VL, UL, FL);
    mhd_flux(VR, UR, FR);

    cfL = or_mhd_cfast(VL, gam);
    cfR = or_mhd_cfast(VR, gam);
    cmax = fmax(cfL, cfR);
    SL = fmin(VL[1], VR[1]) - cmax;
    SR = fmax(VL[1], VR[1]) + cmax;

    if (SL >= 0.0) {
        for (q = 0; q < NVAR; q++)
            F[q] = FL[q];
    } else if (SR <= 0.0) {
        for (q = 0; q < NVAR; q++)
            F[q] = FR[q];
    } else {
        double ptL = VL[4] + 0.5 * (Bn * Bn + VL[6] * VL[6] + VL[7] * VL[7]);
        double ptR = VR[4] + 0.5 * (Bn * Bn + VR[6] * VR[6] + VR[7] * VR[7]);
        double dL, dR, sqL, sqR, SLs, SRs;

        sdL = SL - VL[1];
        sdR = SR - VR[1];
        den = sdR * VR[0] - sdL * VL[0];
        SM = (sdR * VR[0] * VR[1] - sdL * VL[0] * VL[1] - ptR + ptL) / den;
        pts = (sdR * VR[0] * ptL - sdL * VL[0] * ptR +
               VL[0] * VR[0] * sdR * sdL * (VR[1] - VL[1])) / den;

        /* single-star states (MK05 Eq. 43-48) */
        rsL = VL[0] * sdL / (SL - SM);
        rsR = VR[0] * sdR / (SR - SM);
        dL = VL[0] * sdL * (SL - SM) - Bn * Bn;
        dR = VR[0] * sdR * (SR - SM) - Bn * Bn;
        if (fabs(dL) <= 1.0e-12 * (VL[0] * sdL * sdL + Bn * Bn)) {
            vsL = VL[2];
            wsL = VL[3];
            B1sL = VL[6];
            B2sL = VL[7];
        } else {
            double f = (VL[0] * sdL * sdL - Bn * Bn) / dL;
            vsL = VL[2] - Bn * VL[6] * (SM - VL[1]) / dL;
            wsL = VL[3] - Bn * VL[7] * (SM - VL[1]) / dL;
            B1sL = VL[6] * f;
            B2sL = VL[7] * f;
        }
        if (fabs(dR) <= 1.0e-12 * (VR[0] * sdR * sdR + Bn * Bn)) {
            vsR = VR[2];
            wsR = VR[3];
            B1sR = VR[6];
            B2sR = VR[7];
        } else {
            double f = (VR[0] * sdR * sdR - Bn * Bn) / dR;
            vsR = VR[2] - Bn * VR[6] * (SM - VR[1]) / dR;
            wsR = VR[3] - Bn * VR[7] * (SM - VR[1]) / dR;
            B1sR = VR[6] * f;
            B2sR = VR[7] * f;
        }
        {
            double vBL = VL[1] * Bn + VL[2] * VL[6] + VL[3] * VL[7];
            double vBR = VR[1] * Bn + VR[2] * VR[6] + VR[3] * VR[7];
            double vBsL = SM * Bn + vsL * B1sL + wsL * B2sL;
            double vBsR = SM * Bn + vsR * B1sR + wsR * B2sR;
            EsL = (sdL * UL[4] - ptL * VL[1] + pts * SM + Bn * (vBL - vBsL)) / (SL - SM);
            EsR = (sdR * UR[4] - ptR * VR[1] + pts * SM + Bn * (vBR - vBsR)) / (SR - SM);
        }
        UsL[0] = rsL; UsL[1] = rsL * SM; UsL[2] = rsL * vsL; UsL[3] = rsL * wsL;
        UsL[4] = EsL; UsL[5] = Bn; UsL[6] = B1sL; UsL[7] = B2sL; UsL[8] = 0.0;
        UsR[0] = rsR; UsR[1] = rsR * SM; UsR[2] = rsR * vsR; UsR[3] = rsR * wsR;
        UsR[4] = EsR; UsR[5] = Bn; UsR[6] = B1sR; UsR[7] = B2sR; UsR[8] = 0.0;

        sqL = sqrt(rsL);
        sqR = sqrt(rsR);
        SLs = SM - fabs(Bn) / sqL;
        SRs = SM + fabs(Bn) / sqR;

        if (SLs >= 0.0) {
            for (q = 0; q < NVAR; q++)
                F[q] = FL[q] + SL * (UsL[q] - UL[q]);
        } else if (SRs <= 0.0) {
            for (q = 0; q < NVAR; q++)
                F[q] = FR[q] + SR * (UsR[q] - UR[q]);
        } else {
            /* double-star states (MK05 Eq. 59-63) */
            double sB = copysign(1.0, Bn);
            double isq = 1.0 / (sqL + sqR);
            double vss = (sqL * vsL + sqR * vsR + (B1sR - B1sL) * sB) * isq;
            double wss = (sqL * wsL + sqR * wsR + (B2sR - B2sL) * sB) * isq;
            double B1ss = (sqL * B1sR + sqR * B1sL + sqL * sqR * (vsR - vsL) * sB) * isq;
            double B2ss = (sqL * B2sR + sqR * B2sL + sqL * sqR * (wsR - wsL) * sB) * isq;
            double vBss = SM * Bn + vss * B1ss + wss * B2ss;
            double Uss[NVAR];
            if (SM >= 0.0) {
                double vBsL = SM * Bn + vsL * B1sL + wsL * B2sL;
                Uss[0] = rsL; Uss[1] = rsL * SM; Uss[2] = rsL * vss; Uss[3] = rsL * wss;
                Uss[4] = EsL - sqL * (vBsL - vBss) * sB;
                Uss[5] = Bn; Uss[6] = B1ss; Uss[7] = B2ss; Uss[8] = 0.0;
                for (q = 0; q < NVAR; q++)
                    F[q] = FL[q] + SL * (UsL[q] - UL[q]) + SLs * (Uss[q] - UsL[q]);
            } else {
                double vBsR = SM * Bn + vsR * B1sR + wsR * B2sR;
                Uss[0] = rsR; Uss[1] = rsR * SM; Uss[2] = rsR * vss; Uss[3] = rsR * wss;
                Uss[4] = EsR + sqR * (vBsR - vBss) * sB;
                Uss[5] = Bn; Uss[6] = B1ss; Uss[7] = B2ss; Uss[8] = 0.0;
                for (q = 0; q < NVAR; q++)
                    F[q] = FR[q] + SR * (UsR[q] - UR[q]) + SRs * (Uss[q] - UsR[q]);
            }
        }
    }
    F[5] = pm;
    F[8] = ch * ch * Bm;
    return bad;
}

/* HLL flux (Harten, Lax & van Leer), the more diffusive solver of the
 * hybrid integration (appendix on shock detection): the same exact GLM face
 * solve and the same outer wave speeds S_L, S_R as or_mhd_riemann, then the
 * single HLL average state.  Returns 1 if an input state has rho <= 0 or
 * p <= 0. */
int or_mhd_riemann_hll(const double *VL0, const double *VR0, double gam, double ch, double *F)
{
    double VL[NVAR], VR[NVAR], UL[NVAR], UR[NVAR], FL[NVAR], FR[NVAR];
    double Bm, pm, cfL, cfR, cmax, SL, SR;
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
    or_mhd_prim2cons(VL, gam, UL);
    or_mhd_prim2cons(VR, gam, UR);
    mhd_flux(VL, UL, FL);
    mhd_flux(VR, UR, FR);
    cfL = or_mhd_cfast(VL, gam);
    cfR = or_mhd_cfast(VR, gam);
    cmax = fmax(cfL, cfR);
    SL = fmin(VL[1], VR[1]) - cmax;
    SR = fmax(VL[1], VR[1]) + cmax;
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

/* HLLC flux for MHD (Li 2005): the GLM face solve and outer speeds of
 * or_mhd_riemann; the HLL average state U_hll gives the contact speed
 * S_M = (rho u)_hll / rho_hll and the transverse field and velocity of both
 * star states, B*_t = B_t,hll, v*_t = (rho v_t)_hll / rho_hll; with the
 * total pressure p*_t = rho_L (S_L - u_L)(S_M - u_L) + p_t,L each star state
 * is rho* = rho (S - u)/(S - S_M), (rho u)* = rho* S_M,
 * (rho v_t)* = (rho v_t (S - u) - B_n (B*_t - B_t))/(S - S_M),
 * E* = (E (S - u) - p_t u + p*_t S_M + B_n (v.B - v*.B*))/(S - S_M), and the
 * flux is F + S (U* - U) on the side of the contact the face lies on.
 * Returns 1 if an input state has rho <= 0 or p <= 0. */
int or_mhd_riemann_hllc(const double *VL0, const double *VR0, double gam, double ch, double *F)
{
    double VL[NVAR], VR[NVAR], UL[NVAR], UR[NVAR], FL[NVAR], FR[NVAR], Uh[NVAR];
    double Bm, pm, cfL, cfR, cmax, SL, SR;
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
    or_mhd_prim2cons(VL, gam, UL);
    or_mhd_prim2cons(VR, gam, UR);
    mhd_flux(VL, UL, FL);
    mhd_flux(VR, UR, FR);
    cfL = or_mhd_cfast(VL, gam);
    cfR = or_mhd_cfast(VR, gam);
    cmax = fmax(cfL, cfR);
    SL = fmin(VL[1], VR[1]) - cmax;
    SR = fmax(VL[1], VR[1]) + cmax;
    if (SL >= 0.0) {
        for (q = 0; q < NVAR; q++)
            F[q] = FL[q];
    } else if (SR <= 0.0) {
        for (q = 0; q < NVAR; q++)
            F[q] = FR[q];
    } else {
        const double Bn = Bm;
        for (q = 0; q < NVAR; q++)
            Uh[q] = (SR * UR[q] - SL * UL[q] - FR[q] + FL[q]) / (SR - SL);
        const double SM = Uh[1] / Uh[0];
        const double vy = Uh[2] / Uh[0], vz = Uh[3] / Uh[0];
        const double By = Uh[6], Bz = Uh[7];
        const double ptL = VL[4] + 0.5 * (Bn * Bn + VL[6] * VL[6] + VL[7] * VL[7]);
        const double ptR = VR[4] + 0.5 * (Bn * Bn + VR[6] * VR[6] + VR[7] * VR[7]);
        const double pts = VL[0] * (SL - VL[1]) * (SM - VL[1]) + ptL;
        const double vBs = SM * Bn + vy * By + vz * Bz;
        const int right = SM < 0.0;
        const double *V = right ? VR : VL, *U = right ? UR : UL, *Fa = right ? FR : FL;
        const double S = right ? SR : SL, pt = right ? ptR : ptL;
        const double sd = S - V[1], den = S - SM;
        double Us[NVAR];
        const double vB = V[1] * Bn + V[2] * V[6] + V[3] * V[7];
        Us[0] = V[0] * sd / den;
        Us[1] = Us[0] * SM;
        Us[2] = (V[0] * V[2] * sd - Bn * (By - V[6])) / den;
        Us[3] = (V[0] * V[3] * sd - Bn * (Bz - V[7])) / den;
        Us[4] = (U[4] * sd - pt * V[1] + pts * SM + Bn * (vB - vBs)) / den;
        Us[5] = Bn;
        Us[6] = By;
        Us[7] = Bz;
        Us[8] = U[8];
        for (q = 0; q < NVAR; q++)
            F[q] = Fa[q] + S * (Us[q] - U[q]);
    }
    F[5] = pm;
    F[8] = ch * ch * Bm;
    return bad;
}

/* ------------------------------------------------------------------ */
/* Reconstruction, Section 3.2                                         */
/* ------------------------------------------------------------------ */

/* mm(a,b) = (sign a + sign b)/2 min(|a|,|b|), Eq. (minmod) */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0)
        return fmin(a, b);
    if (a < 0.0 && b < 0.0)
        return fmax(a, b);
    return 0.0;
}

/* MC-limited slope from the backward and forward undivided differences,
 * Eq. (MClim). */
static double mc_slope(double dm, double dp)
{
    return minmod(0.5 * (dp + dm), 2.0 * minmod(dm, dp));
}

/* Limited slope of the linear reconstruction from the backward and forward
 * undivided differences: recon 0 MC, Eq. (MClim); 2 MinMod, Eq. (minmod);
 * 3 harmonic mean, Eq. (harmonic_lim); 4 Van Albada, Eq. (vanalbada_lim). */
static double lin_slope(double dm, double dp, int recon)
{
    if (recon == 2)
        return minmod(dm, dp);
    if (recon == 3)
        return dp * dm > 0.0 ? 2.0 * dp * dm / (dp + dm) : 0.0;
    if (recon == 4)
        return dp * dm > 0.0 ? dp * dm * (dp + dm) / (dp * dp + dm * dm) : 0.0;
    return mc_slope(dm, dp);
}

/* Interface values w_(i,+) and w_(i,-) of one characteristic field from the
 * stencil w[0..4] = w_(i,-2) .. w_(i,+2).  recon = 1: PPM, Eq. (ppm1) with
 * the parabolic limiter of Eq. (ppm_parabolic_lim); recon = 5: improved
 * third-order WENO, Eq. (WENO3) with the weights of Eq. (WENO3a), dx the
 * cell width; otherwise linear, Eq. (Linear), with the slope of lin_slope. */
static void reconstruct(const double *w, int recon, double dx, double *wp, double *wm)
{
    double w0 = w[2];
    if (recon == 5) {
        double dp = w[3] - w[2], dm = w[2] - w[1];
        double d2 = (dp - dm) * (dp - dm);
        double ap = 1.0 + d2 / (dx * dx + dp * dp);
        double am = 1.0 + d2 / (dx * dx + dm * dm);
        *wp = w0 + (ap * dp + 0.5 * am * dm) / (2.0 * ap + am);
        *wm = w0 - (am * dm + 0.5 * ap * dp) / (2.0 * am + ap);
        return;
    }
    if (recon != 1) {
        double s0 = lin_slope(w[2] - w[1], w[3] - w[2], recon);
        *wp = w0 + 0.5 * s0;
        *wm = w0 - 0.5 * s0;
    } else {
        double s0 = mc_slope(w[2] - w[1], w[3] - w[2]);
        double sm = mc_slope(w[1] - w[0], w[2] - w[1]);
        double sp = mc_slope(w[3] - w[2], w[4] - w[3]);
        double p = 0.5 * (w0 + w[3]) - (sp - s0) / 6.0;
        double m = 0.5 * (w0 + w[1]) + (sm - s0) / 6.0;
        double dp = p - w0, dm = m - w0;
        double ndp, ndm;
        if (dp * dm > 0.0) {
            ndp = 0.0;
            ndm = 0.0;
        } else {
            ndp = (fabs(dp) >= 2.0 * fabs(dm)) ? -2.0 * dm : dp;
            ndm = (fabs(dm) >= 2.0 * fabs(dp)) ? -2.0 * dp : dm;
        }
        *wp = w0 + ndp;
        *wm = w0 + ndm;
    }
}

/* Characteristic tracing of one field to t^(n+1/2), Eq. (wnorm_predp) and
 * (wnorm_predm), w*_(+/-) = w_ref,(+/-) + beta_(+/-) (traced - w_ref,(+/-)):
 * mode = 0 (default): no reference state, every field is traced to both
 *   interfaces (beta_+ = beta_- = 1), the choice Section 3.2 recommends for
 *   smooth flows so that waves not reaching an edge still enter its value;
 * mode = 1: w_ref = w_(+/-) with the upwind selection beta_+ = [nu > 0],
 *   beta_- = [nu < 0];
 * mode = 2: w_ref = w_(i,0), the cell-centre value (Rider et al. 2007),
 *   upwind selection;
 * mode = 3: the reference state of Colella & Woodward (1984), the field
 *   traced with nu_max = max(0, max nu) to the + interface and with
 *   nu_min = min(0, min nu) to the - interface, upwind selection. */
static void trace(double wp, double w0, double wm, double nu, int mode, double numax, double numin,
                  double *tp, double *tm)
{
    double dw = wp - wm;
    double d2w = wp - 2.0 * w0 + wm;
    double rp = wp, rm = wm;
    if (mode == 2) {
        rp = w0;
        rm = w0;
    } else if (mode == 3) {
        rp = wp - 0.5 * numax * (dw + d2w * (3.0 - 2.0 * numax));
        rm = wm - 0.5 * numin * (dw - d2w * (3.0 + 2.0 * numin));
    }
    *tp = rp;
    *tm = rm;
    if (mode == 0 || nu > 0.0)
        *tp = wp - 0.5 * nu * (dw + d2w * (3.0 - 2.0 * nu));
    if (mode == 0 || nu < 0.0)
        *tm = wm - 0.5 * nu * (dw - d2w * (3.0 + 2.0 * nu));
}

/*
 * Normal predictor in characteristic variables for one cell (Section 3.2).
 * vs[l*NVAR + q], l = 0..4: primitive stencil V_(i-2) .. V_(i+2) in the local
 * order.  Outputs the time-centred interface primitives V*_(i,+), V*_(i,-)
 * (local order), including the S_Bx dBn/dx and S_psi dpsi/dx sources.
 */
void or_mhd_char_predict_dx(const double *vs, double gam, double ch, double dtdx, double dx,
                            int recon, int upwind, double *Vp, double *Vm)
{
    double lam[NVAR], L[NVAR * NVAR], R[NVAR * NVAR];
    double tp[NVAR], tm[NVAR], rp[NVAR], rm[NVAR];
    const double *V0 = vs + 2 * NVAR;
    double dBn, dpsi, src[NVAR];
    double vB;
    int k, l, q;

    or_mhd_eigen(V0, gam, ch, lam, L, R);
    /* the extreme Courant numbers of the seven MHD waves (u -/+ c_f) for the
     * reference state of trace mode 3 */
    const double numax = fmax(0.0, lam[6] * dtdx), numin = fmin(0.0, lam[0] * dtdx);
    for (k = 0; k < NVAR; k++) {
        double w[5];
        for (l = 0; l < 5; l++) {
            double s = 0.0;
            for (q = 0; q < NVAR; q++)
                s += L[k * NVAR + q] * vs[l * NVAR + q];
            w[l] = s;
        }
        reconstruct(w, recon, dx, &rp[k], &rm[k]);
        trace(rp[k], w[2], rm[k], lam[k] * dtdx, upwind, numax, numin, &tp[k], &tm[k]);
    }
    for (q = 0; q < NVAR; q++) {
        double sp = 0.0, sm = 0.0;
        for (k = 0; k < NVAR; k++) {
            sp += tp[k] * R[k * NVAR + q];
            sm += tm[k] * R[k * NVAR + q];
        }
        Vp[q] = sp;
        Vm[q] = sm;
    }
    /* undivided jumps of B_n and psi across the cell, from the (untraced)
     * reconstruction of the two GLM fields */
    dBn = (rp[7] - rm[7]) * R[7 * NVAR + 5] + (rp[8] - rm[8]) * R[8 * NVAR + 5];
    dpsi = (rp[7] - rm[7]) * R[7 * NVAR + 8] + (rp[8] - rm[8]) * R[8 * NVAR + 8];
    /* S_Bx and S_psi: minus the columns of the primitive Jacobian that couple
     * the 7-wave block to d(B_n)/dn and d(psi)/dn */
    vB = V0[1] * V0[5] + V0[2] * V0[6] + V0[3] * V0[7];
    for (q = 0; q < NVAR; q++)
        src[q] = 0.0;
    src[1] = V0[5] / V0[0] * dBn;
    src[2] = V0[6] / V0[0] * dBn;
    src[3] = V0[7] / V0[0] * dBn;
    src[4] = -(gam - 1.0) * vB * dBn + (gam - 1.0) * V0[5] * dpsi;
    src[6] = V0[2] * dBn;
    src[7] = V0[3] * dBn;
    for (q = 0; q < NVAR; q++) {
        Vp[q] += 0.5 * dtdx * src[q];
        Vm[q] += 0.5 * dtdx * src[q];
    }
}

/* or_mhd_char_predict_dx for the reconstructions that do not use the cell
 * width (all but WENO3). */
void or_mhd_char_predict(const double *vs, double gam, double ch, double dtdx,
                         int recon, int upwind, double *Vp, double *Vm)
{
    or_mhd_char_predict_dx(vs, gam, ch, dtdx, 0.0, recon, upwind, Vp, Vm);
}

/* ------------------------------------------------------------------ */
/* Patch geometry                                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    int n[3], g[3], N[3];
    long ncell;
    int ndim;
} grid_t;

static void grid_init(grid_t *G, int nx, int ny, int nz, int ndim)
{
    int d;
    G->n[0] = nx;
    G->n[1] = ny;
    G->n[2] = nz;
    G->ndim = ndim;
    for (d = 0; d < 3; d++) {
        G->g[d] = d < ndim ? NGHOST : 0;
        G->N[d] = G->n[d] + 2 * G->g[d];
    }
    G->ncell = (long)G->N[0] * G->N[1] * G->N[2];
}

static long cidx(const grid_t *G, const int *c)
{
    return ((long)(c[2] + G->g[2]) * G->N[1] + (c[1] + G->g[1])) * G->N[0] + (c[0] + G->g[0]);
}

static long dstride(const grid_t *G, int d)
{
    return d == 0 ? 1 : (d == 1 ? G->N[0] : (long)G->N[0] * G->N[1]);
}

/* ------------------------------------------------------------------ */
/* Shock detection of the hybrid integration (appendix)                */
/* ------------------------------------------------------------------ */

/* Flags of the hybrid integration from the primitive field V (all ghosted
 * cells).  A cell c is shocked (bit 1) when
 *   sum_d |q(c + e_d) - q(c - e_d)| / min(q(c + e_d), q(c - e_d)) > eps_q
 *   and  sum_d (v_d(c + e_d) - v_d(c - e_d)) / (2 dx_d) < 0,
 * q the thermal (qkind 0) or magnetic (qkind 1, B^2/2) pressure, over the
 * active dimensions; evaluated on the cells within three layers of the
 * interior ([-3, n + 3) on active dimensions).  A cell is reconstructed with
 * the MinMod limiter (bit 2) when a shocked cell lies within `reach` cells
 * of it along an active axis (its reconstruction stencil: 2 for PPM, 1 for
 * the three-point reconstructions); evaluated on [-1, n + 1).  Faces next to
 * a shocked cell take the HLL solver. */
static void shock_flags(const grid_t *G, const double *V, const double *h, double eps_q, int qkind, int reach,
                        unsigned char *flags)
{
    const long nc = G->ncell;
    int c[3], lo[3], hi[3], d;
    memset(flags, 0, (size_t)nc);
    for (d = 0; d < 3; d++) {
        lo[d] = d < G->ndim ? -3 : 0;
        hi[d] = d < G->ndim ? G->n[d] + 3 : 1;
    }
    for (c[2] = lo[2]; c[2] < hi[2]; c[2]++)
        for (c[1] = lo[1]; c[1] < hi[1]; c[1]++)
            for (c[0] = lo[0]; c[0] < hi[0]; c[0]++) {
                const long id = cidx(G, c);
                double S = 0.0, D = 0.0;
                for (d = 0; d < G->ndim; d++) {
                    const long st = dstride(G, d), ip = id + st, im = id - st;
                    double qp, qm;
                    if (qkind == 0) {
                        qp = V[4 * nc + ip];
                        qm = V[4 * nc + im];
                    } else {
                        qp = 0.5 * (V[5 * nc + ip] * V[5 * nc + ip] + V[6 * nc + ip] * V[6 * nc + ip] +
                                    V[7 * nc + ip] * V[7 * nc + ip]);
                        qm = 0.5 * (V[5 * nc + im] * V[5 * nc + im] + V[6 * nc + im] * V[6 * nc + im] +
                                    V[7 * nc + im] * V[7 * nc + im]);
                    }
                    S += fabs(qp - qm) / fmin(qp, qm);
                    D += (V[(1 + d) * nc + ip] - V[(1 + d) * nc + im]) / (2.0 * h[d]);
                }
                if (S > eps_q && D < 0.0)
                    flags[id] = 1;
            }
    for (d = 0; d < 3; d++) {
        lo[d] = d < G->ndim ? -1 : 0;
        hi[d] = d < G->ndim ? G->n[d] + 1 : 1;
    }
    for (c[2] = lo[2]; c[2] < hi[2]; c[2]++)
        for (c[1] = lo[1]; c[1] < hi[1]; c[1]++)
            for (c[0] = lo[0]; c[0] < hi[0]; c[0]++) {
                const long id = cidx(G, c);
                int m = 0;
                for (d = 0; d < G->ndim; d++)
                    for (int k = -reach; k <= reach; k++)
                        m |= flags[id + k * dstride(G, d)] & 1;
                if (m)
                    flags[id] |= 2;
            }
}

/* The flags of shock_flags for a ghost-filled patch U (test access). */
void or_mhd_shock_flags(const double *U, int nx, int ny, int nz, int ndim, double dx, double dy, double dz,
                        double gam, double eps_q, int qkind, int reach, unsigned char *flags)
{
    grid_t G;
    double h[3] = {dx, dy, dz};
    grid_init(&G, nx, ny, nz, ndim);
    const long nc = G.ncell;
    double *V = (double *)malloc(sizeof(double) * NVAR * nc);
    for (long id = 0; id < nc; id++) {
        double Uc[NVAR], Vc[NVAR];
        for (int q = 0; q < NVAR; q++)
            Uc[q] = U[q * nc + id];
        or_mhd_cons2prim(Uc, gam, Vc);
        for (int q = 0; q < NVAR; q++)
            V[q * nc + id] = Vc[q];
    }
    shock_flags(&G, V, h, eps_q, qkind, reach, flags);
    free(V);
}

/* ------------------------------------------------------------------ */
/* CFL, Eq. (Ca)                                                       */
/* ------------------------------------------------------------------ */

/* Eq. (Ca): max over interior cells of
 *     max_d (|v_d| + c_f,d)/dx_d + sum_d 2 D / dx_d^2,
 * with D the largest diffusion coefficient of the cell:
 * max((Gamma - 1) max(kappa, kpar) / rho, (4/3) nu, eta), the diffusivities of the
 * temperature under conduction, of the longitudinal velocity under viscosity
 * and of B under resistivity (0 when all three are 0).  The caller sets dt = C_a / max and c_h = max * min_d dx_d
 * (= C_a min_d dx_d / dt). */
double or_mhd_max_rate_par(const double *U, int nx, int ny, int nz, int ndim, double dx, double dy, double dz,
                           double gam, double kappa, double kpar, double nu, double eta)
{
    grid_t G;
    double h[3] = {dx, dy, dz}, m = 0.0;
    int c[3], d, q;
    grid_init(&G, nx, ny, nz, ndim);
    for (c[2] = 0; c[2] < G.n[2]; c[2]++)
        for (c[1] = 0; c[1] < G.n[1]; c[1]++)
            for (c[0] = 0; c[0] < G.n[0]; c[0]++) {
                long id = cidx(&G, c);
                double Uc[NVAR], V[NVAR], Vl[NVAR], s = 0.0;
                for (q = 0; q < NVAR; q++)
                    Uc[q] = U[q * G.ncell + id];
                or_mhd_cons2prim(Uc, gam, V);
                for (d = 0; d < ndim; d++) {
                    double sd;
                    for (q = 0; q < NVAR; q++)
                        Vl[q] = V[PERM[d][q]];
                    sd = (fabs(Vl[1]) + or_mhd_cfast(Vl, gam)) / h[d];
                    if (sd > s)
                        s = sd;
                }
                if (kappa > 0.0 || kpar > 0.0 || nu > 0.0 || eta > 0.0) {
                    double D = fmax(fmax((gam - 1.0) * fmax(kappa, kpar) / V[0], 4.0 / 3.0 * nu), eta);
                    for (d = 0; d < ndim; d++)
                        s += 2.0 * D / (h[d] * h[d]);
                }
                if (s > m)
                    m = s;
            }
    return m;
}

/* or_mhd_max_rate_par with conduction alone. */
double or_mhd_max_rate(const double *U, int nx, int ny, int nz, int ndim,
                       double dx, double dy, double dz, double gam, double kappa)
{
    return or_mhd_max_rate_par(U, nx, ny, nz, ndim, dx, dy, dz, gam, kappa, kappa, 0.0, 0.0);
}

/* max over interior cells of max_d (|v_d| + c_f,d)/dx_d (Eq. Ca without
 * parabolic terms). */
double or_mhd_max_speed(const double *U, int nx, int ny, int nz, int ndim,
                        double dx, double dy, double dz, double gam)
{
    return or_mhd_max_rate_par(U, nx, ny, nz, ndim, dx, dy, dz, gam, 0.0, 0.0, 0.0, 0.0);
}

/* ------------------------------------------------------------------ */
/* Parabolic terms: thermal conduction and viscosity                   */
/* ------------------------------------------------------------------ */

/* The parabolic fluxes of Section 2.1.1 on a Cartesian grid, from the
 * cell-centred fields W = (rho, v_x, v_y, v_z, T, B_x, B_y, B_z) (eight
 * arrays of ncell values, T = p / rho):
 *   - classical thermal conduction, the heat flux of Eq. (tc_flux) in the
 *     limit q -> infinity with constant kappa_perp = kappa and kappa_par = kpar:
 *     Pi_E += kappa dT/dx_d + (kpar - kappa) b_d (b . grad T), b the unit
 *     vector of the face's mean field (isotropic where it vanishes or
 *     kpar = kappa); with phi > 0 the saturated form of the paper's appendix
 *     on the heat flux (below);
 *   - isotropic viscosity, the stress of Eq. (visc_tens) with constant
 *     kinematic viscosity nu:
 *     tau_(d,i) = rho nu (dv_i/dx_d + dv_d/dx_i - (2/3) delta_(di) div v),
 *     Pi_(m_i) = tau_(d,i) and Pi_E += v . tau_d (the energy flux of the
 *     viscous stresses).
 * Face values follow Section 3.1 (Pi = g(U) df(U)/dx with g at the mean of
 * the two cells' states and second-order central differences): at the face
 * between c and c + e_d,
 *     df/dx_d = (f(c + e_d) - f(c)) / dx_d,
 *     df/dx_t = [f(c + e_t) - f(c - e_t) + f(c + e_d + e_t) - f(c + e_d - e_t)]
 *               / (4 dx_t)  for an active t != d (0 on an inactive axis),
 *     rho_f = (rho(c) + rho(c + e_d)) / 2,
 *     v_f = (rho v (c) + rho v (c + e_d)) / (rho(c) + rho(c + e_d)),
 * the last two being the density and velocity of the mean conserved state;
 *   - resistivity with constant eta (the induction term -curl(eta J),
 *     J = curl B, and the energy flux -eta J x B of Section 2.1.1).
 * Pi[1..3] receive the momentum fluxes, Pi[4] the energy flux and Pi[5..7]
 * the fluxes of B.  W holds (rho, v_x, v_y, v_z, T, B_x, B_y, B_z). */
static void parabolic_face(const grid_t *G, const double *W, const double *h, double kappa, double kpar, double phi,
                           double nu, double eta, long id, int d, double *Pi)
{
    const long nc = G->ncell, st = dstride(G, d), ip = id + st;
    int q;
    for (q = 0; q < NVAR; q++)
        Pi[q] = 0.0;
    if (phi > 0.0 && (kappa > 0.0 || kpar > 0.0)) {
        /* saturated conduction (the paper's appendix on the heat flux): the
         * classical flux F = kappa_perp grad T + (kappa_par - kappa_perp)
         * b (b . grad T) with the face gradient of T (normal two-point
         * difference, transverse mean of central differences), the upwind
         * saturated flux q = 5 phi p_u^(3/2) / sqrt(rho_f), p_u the pressure
         * of the cell on the side F_d points away from (the left one when
         * F_d < 0), and their harmonic mean q F_d / (|F| + q) */
        const double *T = W + 4 * nc;
        double gt[3], bf[3], b2 = 0.0, bg = 0.0, F[3], fm = 0.0, rf, pu, qs;
        int t;
        for (t = 0; t < 3; t++) {
            if (t == d) {
                gt[t] = (T[ip] - T[id]) / h[d];
            } else if (t < G->ndim) {
                const long s2 = dstride(G, t);
                gt[t] = (T[id + s2] - T[id - s2] + T[ip + s2] - T[ip - s2]) / (4.0 * h[t]);
            } else {
                gt[t] = 0.0;
            }
            bf[t] = 0.5 * (W[(5 + t) * nc + id] + W[(5 + t) * nc + ip]);
            b2 += bf[t] * bf[t];
            bg += bf[t] * gt[t];
        }
        for (t = 0; t < 3; t++) {
            F[t] = kappa * gt[t];
            if (kpar != kappa && b2 > 0.0)
                F[t] += (kpar - kappa) * bf[t] * bg / b2;
            fm += F[t] * F[t];
        }
        fm = sqrt(fm);
        rf = 0.5 * (W[id] + W[ip]);
        pu = F[d] < 0.0 ? W[id] * T[id] : W[ip] * T[ip];
        qs = 5.0 * phi * pu * sqrt(pu) / sqrt(rf);
        Pi[4] += qs * F[d] / (fm + qs);
    } else {
    if (kappa > 0.0 || kpar > 0.0)
        Pi[4] += kappa * (W[4 * nc + ip] - W[4 * nc + id]) / h[d];
    if (kpar != kappa) {
        /* anisotropic part of the classical heat flux of Eq. (tc_flux):
         * (kappa_par - kappa_perp) b (b . grad T), b = B_f / |B_f| the
         * direction of the face's mean field (none where B_f = 0) */
        const double *T = W + 4 * nc;
        double gt[3], bf[3], b2 = 0.0, bg = 0.0;
        int t;
        for (t = 0; t < 3; t++) {
            if (t == d) {
                gt[t] = (T[ip] - T[id]) / h[d];
            } else if (t < G->ndim) {
                const long s2 = dstride(G, t);
                gt[t] = (T[id + s2] - T[id - s2] + T[ip + s2] - T[ip - s2]) / (4.0 * h[t]);
            } else {
                gt[t] = 0.0;
            }
            bf[t] = 0.5 * (W[(5 + t) * nc + id] + W[(5 + t) * nc + ip]);
            b2 += bf[t] * bf[t];
        }
        if (b2 > 0.0) {
            for (t = 0; t < 3; t++)
                bg += bf[t] * gt[t];
            Pi[4] += (kpar - kappa) * bf[d] * bg / b2;
        }
    }
    }
    if (nu > 0.0) {
        double grad[3][3], div = 0.0, rf, vf[3];
        int i, t;
        for (t = 0; t < 3; t++)
            for (i = 0; i < 3; i++) {
                const double *v = W + (1 + i) * nc;
                if (t == d) {
                    grad[t][i] = (v[ip] - v[id]) / h[d];
                } else if (t < G->ndim) {
                    const long s2 = dstride(G, t);
                    grad[t][i] = (v[id + s2] - v[id - s2] + v[ip + s2] - v[ip - s2]) / (4.0 * h[t]);
                } else {
                    grad[t][i] = 0.0;
                }
            }
        for (i = 0; i < 3; i++)
            div += grad[i][i];
        rf = 0.5 * (W[id] + W[ip]);
        for (i = 0; i < 3; i++)
            vf[i] = (W[id] * W[(1 + i) * nc + id] + W[ip] * W[(1 + i) * nc + ip]) / (W[id] + W[ip]);
        for (i = 0; i < 3; i++) {
            double tau = rf * nu * (grad[d][i] + grad[i][d] - (i == d ? 2.0 / 3.0 * div : 0.0));
            Pi[1 + i] += tau;
            Pi[4] += vf[i] * tau;
        }
    }
    if (eta > 0.0) {
        /* resistivity: -curl(eta J) = div(eta (grad B^T - grad B)) for
         * constant eta, so the flux of B_i along d is eta (dB_i/dx_d -
         * dB_d/dx_i) (zero for B_d), and the energy flux -eta J x B along d
         * is sum_i B_i,f times it, B_f the mean of the two cells */
        double gb[3][3];
        int i, t;
        for (t = 0; t < 3; t++)
            for (i = 0; i < 3; i++) {
                const double *B = W + (5 + i) * nc;
                if (t == d) {
                    gb[t][i] = (B[ip] - B[id]) / h[d];
                } else if (t < G->ndim) {
                    const long s2 = dstride(G, t);
                    gb[t][i] = (B[id + s2] - B[id - s2] + B[ip + s2] - B[ip - s2]) / (4.0 * h[t]);
                } else {
                    gb[t][i] = 0.0;
                }
            }
        for (i = 0; i < 3; i++) {
            double f = eta * (gb[d][i] - gb[i][d]);
            double bf = 0.5 * (W[(5 + i) * nc + id] + W[(5 + i) * nc + ip]);
            Pi[5 + i] += f;
            Pi[4] += bf * f;
        }
    }
}

/* L_P = sum_d (Pi_(d,+) - Pi_(d,-)) / dx_d (Eq. incrementop_par, Cartesian)
 * for the momentum, the energy and B, LP[q * ncell + id] (q = 1..7), on the
 * cells lo <= c <= hi; the other entries are left as they are. */
static void parabolic_lp(const grid_t *G, const double *W, const double *h, double kappa, double kpar, double phi,
                         double nu, double eta, const int *lo, const int *hi, double *LP)
{
    int c[3], d, q;
    for (c[2] = lo[2]; c[2] <= hi[2]; c[2]++)
        for (c[1] = lo[1]; c[1] <= hi[1]; c[1]++)
            for (c[0] = lo[0]; c[0] <= hi[0]; c[0]++) {
                long id = cidx(G, c);
                double s[NVAR] = {0}, Pp[NVAR], Pm[NVAR];
                for (d = 0; d < G->ndim; d++) {
                    parabolic_face(G, W, h, kappa, kpar, phi, nu, eta, id, d, Pp);
                    parabolic_face(G, W, h, kappa, kpar, phi, nu, eta, id - dstride(G, d), d, Pm);
                    for (q = 1; q <= 7; q++)
                        s[q] += (Pp[q] - Pm[q]) / h[d];
                }
                for (q = 1; q <= 7; q++)
                    LP[q * G->ncell + id] = s[q];
            }
}

/* The fields W = (rho, v, T, B) of every ghosted cell of U; returns the
 * number of cells with rho <= 0 or p <= 0. */
static int parabolic_fields(const grid_t *G, const double *U, double gam, double *W)
{
    int bad = 0, q;
    const long nc = G->ncell;
    for (long id = 0; id < nc; id++) {
        double Uc[NVAR], Vc[NVAR];
        for (q = 0; q < NVAR; q++)
            Uc[q] = U[q * nc + id];
        bad += or_mhd_cons2prim(Uc, gam, Vc);
        W[id] = Vc[0];
        for (q = 1; q <= 3; q++)
            W[q * nc + id] = Vc[q];
        W[4 * nc + id] = Vc[4] / Vc[0];
        for (q = 5; q <= 7; q++)
            W[q * nc + id] = Vc[q];
    }
    return bad;
}

/* L_P of conduction, viscosity and resistivity on the interior cells of a
 * ghost-filled patch: LP[q * ncell + id] for the momentum (q = 1..3), the
 * energy (q = 4) and B (q = 5..7), ghosted layout (the other entries are
 * 0). */
void or_mhd_parabolic(const double *U, int nx, int ny, int nz, int ndim, double dx, double dy, double dz,
                      double gam, double kappa, double kpar, double phi, double nu, double eta, double *LP)
{
    grid_t G;
    double h[3] = {dx, dy, dz};
    int lo[3] = {0, 0, 0}, hi[3], d;
    double *W;
    grid_init(&G, nx, ny, nz, ndim);
    for (d = 0; d < 3; d++)
        hi[d] = G.n[d] - 1;
    W = (double *)malloc(sizeof(double) * 8 * G.ncell);
    parabolic_fields(&G, U, gam, W);
    memset(LP, 0, sizeof(double) * NVAR * G.ncell);
    parabolic_lp(&G, W, h, kappa, kpar, phi, nu, eta, lo, hi, LP);
    free(W);
}

/* The energy component of or_mhd_parabolic with conduction alone. */
void or_mhd_conduction(const double *U, int nx, int ny, int nz, int ndim, double dx, double dy, double dz,
                       double gam, double kappa, double *LP)
{
    grid_t G;
    double *A;
    grid_init(&G, nx, ny, nz, ndim);
    A = (double *)malloc(sizeof(double) * NVAR * G.ncell);
    or_mhd_parabolic(U, nx, ny, nz, ndim, dx, dy, dz, gam, kappa, kappa, 0.0, 0.0, 0.0, A);
    memcpy(LP, A + 4 * G.ncell, sizeof(double) * G.ncell);
    free(A);
}

/* ------------------------------------------------------------------ */
/* One CTU step on one ghost-filled patch                              */
/* ------------------------------------------------------------------ */
/*
 * Unew receives U with the interior advanced by dt; ghosts are copied.
 *
 * Flux registers, Eq. (fluxcorr): nwin face windows, window w described by
 * win[7*w .. 7*w+6] = (d, f, a0, a1, b0, b1, dst).  It covers the faces
 * normal to d on plane f (0 <= f <= n_d; plane f separates cells f-1 and f)
 * with the two other coordinates a in [a0, a1), b in [b0, b1) ((a, b) the
 * two other dimensions in increasing order).  For every such face
 *     reg[dst + (q * nb + (b - b0)) * na + (a - a0)] += wgt[w] * dt * A * F_q
 * with na = a1 - a0, nb = b1 - b0, A the face area (product of the two
 * transverse cell widths) and F the n+1/2 flux through the face in +d.
 * Returns the number of states met with rho <= 0 or p <= 0.
 */
int or_mhd_step_ex(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                   double dx, double dy, double dz, double dt, double ch,
                   double gam, double glm_alpha, int recon, int upwind,
                   const long *win, const double *wgt, int nwin, double *reg,
                   int solver, int shock, double eps_q, int qkind);

int or_mhd_step(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                double dx, double dy, double dz, double dt, double ch,
                double gam, double glm_alpha, int recon, int upwind,
                const long *win, const double *wgt, int nwin, double *reg)
{
    return or_mhd_step_ex(U, Unew, nx, ny, nz, ndim, dx, dy, dz, dt, ch, gam, glm_alpha, recon, upwind, win,
                          wgt, nwin, reg, 0, 0, 0.0, 0);
}

/* The Riemann solver of a face: HLL next to a cell the hybrid integration
 * flagged, else HLLD (solver 0) or HLLC (solver 2). */
static int face_riemann(const double *VL, const double *VR, double gam, double ch, int solver, int hll,
                        double *F)
{
    if (hll)
        return or_mhd_riemann_hll(VL, VR, gam, ch, F);
    if (solver == 2)
        return or_mhd_riemann_hllc(VL, VR, gam, ch, F);
    return or_mhd_riemann(VL, VR, gam, ch, F);
}

/* The step of or_mhd_step_ex, or_mhd_step_tc and or_mhd_step_par: with
 * kappa, nu or eta > 0, conduction, viscosity and resistivity (parabolic_lp)
 * enter as the parabolic term of Section 3.1 (Pi != 0): L_P^n from the cell-centred U^n
 * joins the transverse increments of every direction's predictor (Eq.
 * transv), and the update adds L_P^(n+1/2) from the cell-centred
 * U^(n+1/2) = U^n + dt/2 sum_d (L_(H,d)^n + L_(P,d)^n), L_H^n the first-order
 * (Godunov) divergences. */
static int step_core(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                     double dx, double dy, double dz, double dt, double ch,
                     double gam, double glm_alpha, int recon, int upwind,
                     const long *win, const double *wgt, int nwin, double *reg,
                     int solver, int shock, double eps_q, int qkind, double kappa, double kpar, double phi,
                     double nu, double eta, int corner)
{
    const int par = kappa > 0.0 || kpar > 0.0 || nu > 0.0 || eta > 0.0;
    unsigned char *flags = NULL;
    grid_t G;
    double h[3] = {dx, dy, dz};
    double *V, *F1[3] = {0, 0, 0}, *Up[3] = {0, 0, 0}, *Um[3] = {0, 0, 0}, *F[3] = {0, 0, 0};
    double *Wn = NULL, *LPn = NULL, *Wh = NULL, *LPh = NULL;
    int ring_lo[3], ring_hi[3];
    int c[3], d, q, bad = 0;
    long nc;

    grid_init(&G, nx, ny, nz, ndim);
    nc = G.ncell;
    V = (double *)malloc(sizeof(double) * NVAR * nc);

    /* 1. V = V(U) everywhere, ghosts included */
    for (long id = 0; id < nc; id++) {
        double Uc[NVAR], Vc[NVAR];
        for (q = 0; q < NVAR; q++)
            Uc[q] = U[q * nc + id];
        bad += or_mhd_cons2prim(Uc, gam, Vc);
        for (q = 0; q < NVAR; q++)
            V[q * nc + id] = Vc[q];
    }
    if (shock) {
        flags = (unsigned char *)malloc((size_t)nc);
        shock_flags(&G, V, h, eps_q, qkind, recon == 1 ? 2 : 1, flags);
    }
    /* the ring box: the interior and one layer around it on active axes */
    for (d = 0; d < 3; d++) {
        ring_lo[d] = d < ndim ? -1 : 0;
        ring_hi[d] = d < ndim ? G.n[d] : 0;
    }
    if (par) {
        /* L_P^n on the ring box, from W^n = (rho, v, p / rho, B)^n */
        Wn = (double *)malloc(sizeof(double) * 8 * nc);
        LPn = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        for (long id = 0; id < nc; id++) {
            for (q = 0; q < 8; q++)
                Wn[q * nc + id] = V[q * nc + id];
            Wn[4 * nc + id] = V[4 * nc + id] / V[id];
        }
        parabolic_lp(&G, Wn, h, kappa, kpar, phi, nu, eta, ring_lo, ring_hi, LPn);
    }

    /* 2. the transverse fluxes on the faces the transverse increments need;
     *    F1[d] at cell c is its upper face.  corner = 0: first-order Godunov
     *    fluxes F^n_d = R(U_c, U_(c+e_d)) between cell-centred states (Eq.
     *    transv).  corner = 1 (Pi = 0 only), the corner coupling of Mignone &
     *    Tzeferacos (2010) that Section 3.1 refers to: the Riemann problem
     *    between the normal predictor states of direction d, F*_d =
     *    R(U*_(c,+), U*_(c+e_d,-)), U* from the characteristic predictor of
     *    step 3 (time-centred along d, without transverse terms). */
    for (d = 0; d < ndim; d++) {
        long st = dstride(&G, d);
        int lo[3], hi[3], e;
        F1[d] = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        for (e = 0; e < 3; e++) {
            if (e >= ndim) {
                lo[e] = 0;
                hi[e] = 0;
            } else if (e == d) {
                /* with parabolic terms, also the outer faces of the ring box */
                lo[e] = par ? -2 : -1;
                hi[e] = par ? G.n[e] : G.n[e] - 1;
            } else {
                lo[e] = -1;
                hi[e] = G.n[e];
            }
        }
        for (c[2] = lo[2]; c[2] <= hi[2]; c[2]++)
            for (c[1] = lo[1]; c[1] <= hi[1]; c[1]++)
                for (c[0] = lo[0]; c[0] <= hi[0]; c[0]++) {
                    long id = cidx(&G, c);
                    double VL[NVAR], VR[NVAR], Fl[NVAR];
                    if (corner) {
                        double vs[5 * NVAR], Vx[NVAR];
                        int l;
                        for (l = 0; l < 5; l++)
                            for (q = 0; q < NVAR; q++)
                                vs[l * NVAR + q] = V[PERM[d][q] * nc + id + (l - 2) * st];
                        or_mhd_char_predict_dx(vs, gam, ch, dt / h[d], h[d],
                                               (flags && (flags[id] & 2)) ? 2 : recon, upwind, VL, Vx);
                        for (l = 0; l < 5; l++)
                            for (q = 0; q < NVAR; q++)
                                vs[l * NVAR + q] = V[PERM[d][q] * nc + id + (l - 1) * st];
                        or_mhd_char_predict_dx(vs, gam, ch, dt / h[d], h[d],
                                               (flags && (flags[id + st] & 2)) ? 2 : recon, upwind, Vx, VR);
                    } else {
                        for (q = 0; q < NVAR; q++) {
                            VL[q] = V[PERM[d][q] * nc + id];
                            VR[q] = V[PERM[d][q] * nc + id + st];
                        }
                    }
                    face_riemann(VL, VR, gam, ch, solver, flags && ((flags[id] | flags[id + st]) & 1), Fl);
                    for (q = 0; q < NVAR; q++)
                        F1[d][PERM[d][q] * nc + id] = Fl[q];
                }
    }

    /* 3. normal predictors + transverse correction, Eq. (transv) */
    for (d = 0; d < ndim; d++) {
        long st = dstride(&G, d);
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
                    long id = cidx(&G, c);
                    double vs[5 * NVAR], Vp[NVAR], Vm[NVAR], Ul[NVAR], Ug[NVAR], T[NVAR];
                    int l, t;
                    for (l = 0; l < 5; l++)
                        for (q = 0; q < NVAR; q++)
                            vs[l * NVAR + q] = V[PERM[d][q] * nc + id + (l - 2) * st];
                    or_mhd_char_predict_dx(vs, gam, ch, dt / h[d], h[d], (flags && (flags[id] & 2)) ? 2 : recon,
                                           upwind, Vp, Vm);
                    /* transverse increments L^n_d' = -(F_(d',+) - F_(d',-))/dx_d' */
                    for (q = 0; q < NVAR; q++)
                        T[q] = 0.0;
                    for (t = 0; t < ntr; t++) {
                        int e2 = tr[t];
                        long st2 = dstride(&G, e2);
                        for (q = 0; q < NVAR; q++)
                            T[q] += (F1[e2][q * nc + id - st2] - F1[e2][q * nc + id]) / h[e2];
                    }
                    /* the parabolic term of every direction, Eq. (transv) */
                    if (LPn)
                        for (q = 1; q <= 7; q++)
                            T[q] += LPn[q * nc + id];
                    or_mhd_prim2cons(Vp, gam, Ul);
                    for (q = 0; q < NVAR; q++)
                        Ug[PERM[d][q]] = Ul[q];
                    for (q = 0; q < NVAR; q++)
                        Up[d][q * nc + id] = Ug[q] + 0.5 * dt * T[q];
                    or_mhd_prim2cons(Vm, gam, Ul);
                    for (q = 0; q < NVAR; q++)
                        Ug[PERM[d][q]] = Ul[q];
                    for (q = 0; q < NVAR; q++)
                        Um[d][q * nc + id] = Ug[q] + 0.5 * dt * T[q];
                }
    }

    /* 4. n+1/2 Riemann problems, Eq. (ctu_flux); F[d] at c is its upper face */
    for (d = 0; d < ndim; d++) {
        long st = dstride(&G, d);
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
                    long id = cidx(&G, c);
                    double UL[NVAR], UR[NVAR], VLg[NVAR], VRg[NVAR], VL[NVAR], VR[NVAR], Fl[NVAR];
                    for (q = 0; q < NVAR; q++) {
                        UL[q] = Up[d][q * nc + id];
                        UR[q] = Um[d][q * nc + id + st];
                    }
                    bad += or_mhd_cons2prim(UL, gam, VLg);
                    bad += or_mhd_cons2prim(UR, gam, VRg);
                    for (q = 0; q < NVAR; q++) {
                        VL[q] = VLg[PERM[d][q]];
                        VR[q] = VRg[PERM[d][q]];
                    }
                    face_riemann(VL, VR, gam, ch, solver, flags && ((flags[id] | flags[id + st]) & 1), Fl);
                    for (q = 0; q < NVAR; q++)
                        F[d][PERM[d][q] * nc + id] = Fl[q];
                }
    }

    /* 4b. with parabolic terms: W^(n+1/2) of the cell-centred
     *     U^(n+1/2) = U^n + dt/2 (sum_d L_(H,d)^n + L_P^n) on the ring box,
     *     then L_P^(n+1/2) on the interior */
    if (par) {
        int ilo[3] = {0, 0, 0}, ihi[3];
        Wh = (double *)calloc((size_t)8 * nc, sizeof(double));
        LPh = (double *)calloc((size_t)NVAR * nc, sizeof(double));
        for (c[2] = ring_lo[2]; c[2] <= ring_hi[2]; c[2]++)
            for (c[1] = ring_lo[1]; c[1] <= ring_hi[1]; c[1]++)
                for (c[0] = ring_lo[0]; c[0] <= ring_hi[0]; c[0]++) {
                    long id = cidx(&G, c);
                    double Uh[NVAR], Vh[NVAR];
                    for (q = 0; q < NVAR; q++) {
                        double s = 0.0;
                        for (d = 0; d < ndim; d++)
                            s += (F1[d][q * nc + id - dstride(&G, d)] - F1[d][q * nc + id]) / h[d];
                        s += LPn[q * nc + id];
                        Uh[q] = U[q * nc + id] + 0.5 * dt * s;
                    }
                    bad += or_mhd_cons2prim(Uh, gam, Vh);
                    for (q = 0; q < 8; q++)
                        Wh[q * nc + id] = Vh[q];
                    Wh[4 * nc + id] = Vh[4] / Vh[0];
                }
        for (d = 0; d < 3; d++)
            ihi[d] = G.n[d] - 1;
        parabolic_lp(&G, Wh, h, kappa, kpar, phi, nu, eta, ilo, ihi, LPh);
    }

    /* 5. conservative update, Eq. (update): U + dt * (L_x + L_y + L_z) (+ L_P) */
    memcpy(Unew, U, sizeof(double) * NVAR * nc);
    {
        double hmin = h[0], damp;
        for (d = 1; d < ndim; d++)
            hmin = fmin(hmin, h[d]);
        /* psi source -(c_h^2/c_p^2) psi integrated exactly over dt (operator
         * split, Section 3.1), with c_h^2/c_p^2 = glm_alpha c_h / min dx */
        damp = exp(-glm_alpha * ch * dt / hmin);
        for (c[2] = 0; c[2] < G.n[2]; c[2]++)
            for (c[1] = 0; c[1] < G.n[1]; c[1]++)
                for (c[0] = 0; c[0] < G.n[0]; c[0]++) {
                    long id = cidx(&G, c);
                    for (q = 0; q < NVAR; q++) {
                        double s = 0.0;
                        for (d = 0; d < ndim; d++)
                            s += (F[d][q * nc + id - dstride(&G, d)] - F[d][q * nc + id]) / h[d];
                        if (LPh)
                            s += LPh[q * nc + id];
                        Unew[q * nc + id] = U[q * nc + id] + dt * s;
                    }
                    Unew[8 * nc + id] *= damp;
                }
    }

    /* 6. flux-register contributions, Eq. (fluxcorr) */
    for (int w = 0; w < nwin; w++) {
        const long *W = win + 7 * w;
        int wd = (int)W[0], a = wd == 0 ? 1 : 0, b = wd == 2 ? 1 : 2;
        long na = W[3] - W[2], nb = W[5] - W[4];
        double area = h[a] * h[b];
        for (q = 0; q < NVAR; q++)
            for (long jb = 0; jb < nb; jb++)
                for (long ja = 0; ja < na; ja++) {
                    long id;
                    double flux;
                    c[wd] = (int)W[1] - 1; /* F[d] at cell c is its upper face */
                    c[a] = (int)(W[2] + ja);
                    c[b] = (int)(W[4] + jb);
                    id = cidx(&G, c);
                    flux = F[wd][q * nc + id];
                    /* with parabolic terms the flux through the face is
                     * F - Pi^(n+1/2) (momentum, energy and B) */
                    if (Wh && q >= 1 && q <= 7) {
                        double Pi[NVAR];
                        parabolic_face(&G, Wh, h, kappa, kpar, phi, nu, eta, id, wd, Pi);
                        flux -= Pi[q];
                    }
                    reg[W[6] + (q * nb + jb) * na + ja] += wgt[w] * dt * area * flux;
                }
    }

    free(flags);
    free(V);
    free(Wn);
    free(LPn);
    free(Wh);
    free(LPh);
    for (d = 0; d < 3; d++) {
        free(F1[d]);
        free(Up[d]);
        free(Um[d]);
        free(F[d]);
    }
    return bad;
}

/* or_mhd_step with the Riemann solver `solver` (0 HLLD, 2 HLLC; the same
 * solver for the first-order and the n+1/2 fluxes) and, when shock != 0,
 * the hybrid integration of the appendix on shock detection: the flags of
 * shock_flags (eps_q, qkind) on V^n select the HLL solver at the faces of
 * shocked cells (first-order and n+1/2 fluxes) and the MinMod linear
 * reconstruction for the cells near them. */
int or_mhd_step_ex(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                   double dx, double dy, double dz, double dt, double ch,
                   double gam, double glm_alpha, int recon, int upwind,
                   const long *win, const double *wgt, int nwin, double *reg,
                   int solver, int shock, double eps_q, int qkind)
{
    return step_core(U, Unew, nx, ny, nz, ndim, dx, dy, dz, dt, ch, gam, glm_alpha, recon, upwind, win, wgt,
                     nwin, reg, solver, shock, eps_q, qkind, 0.0, 0.0, 0.0, 0.0, 0.0, 0);
}

/* or_mhd_step_ex with the corner coupling of Mignone & Tzeferacos (2010):
 * the transverse fluxes of Eq. (transv) from the normal predictor states
 * (step 2 of step_core with corner = 1) instead of the cell-centred states;
 * the case Pi = 0 of Section 3.1 ("constructed exactly as illustrated by
 * MT").  Six Riemann problems per zone as well, C_a <= 1/2 in 3-D. */
int or_mhd_step_mt(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                   double dx, double dy, double dz, double dt, double ch,
                   double gam, double glm_alpha, int recon, int upwind,
                   const long *win, const double *wgt, int nwin, double *reg,
                   int solver, int shock, double eps_q, int qkind)
{
    return step_core(U, Unew, nx, ny, nz, ndim, dx, dy, dz, dt, ch, gam, glm_alpha, recon, upwind, win, wgt,
                     nwin, reg, solver, shock, eps_q, qkind, 0.0, 0.0, 0.0, 0.0, 0.0, 1);
}

/* or_mhd_step_ex with thermal conduction of conductivities kappa >= 0 across
 * and kpar >= 0 along the field (saturated with phi > 0), viscosity of kinematic viscosity nu >= 0
 * and resistivity eta >= 0 (the
 * parabolic terms; see step_core and parabolic_face).  The flux registers
 * take the fluxes F - Pi^(n+1/2) of the momentum, the energy and B through
 * their faces. */
int or_mhd_step_par(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                    double dx, double dy, double dz, double dt, double ch,
                    double gam, double glm_alpha, int recon, int upwind,
                    const long *win, const double *wgt, int nwin, double *reg,
                    int solver, int shock, double eps_q, int qkind, double kappa, double kpar, double phi,
                    double nu, double eta)
{
    return step_core(U, Unew, nx, ny, nz, ndim, dx, dy, dz, dt, ch, gam, glm_alpha, recon, upwind, win, wgt,
                     nwin, reg, solver, shock, eps_q, qkind, kappa, kpar, phi, nu, eta, 0);
}

/* or_mhd_step_par with conduction alone. */
int or_mhd_step_tc(const double *U, double *Unew, int nx, int ny, int nz, int ndim,
                   double dx, double dy, double dz, double dt, double ch,
                   double gam, double glm_alpha, int recon, int upwind,
                   const long *win, const double *wgt, int nwin, double *reg,
                   int solver, int shock, double eps_q, int qkind, double kappa)
{
    return step_core(U, Unew, nx, ny, nz, ndim, dx, dy, dz, dt, ch, gam, glm_alpha, recon, upwind, win, wgt,
                     nwin, reg, solver, shock, eps_q, qkind, kappa, kappa, 0.0, 0.0, 0.0, 0);
}

/* ------------------------------------------------------------------ */
/* Optional floors on the updated state                                */
/* ------------------------------------------------------------------ */

/* The paper fixes no floor (its safeguard against non-physical states is
 * the shock-flagged hybrid integration of its appendix on shock detection);
 * this is the reading the library follows.  Applied to the
 * interior cells of U after the update and the psi damping:
 *   1. rho < rho_floor: rho becomes rho_floor; m, E, B and psi are kept;
 *   2. with that density, p = (Gamma-1)(E - m^2/(2 rho) - B^2/2); when
 *      p < p_floor, E becomes p_floor/(Gamma-1) + m^2/(2 rho) + B^2/2.
 * A floor of 0 is off.  A NaN state fails both tests and is left as it is.
 * Returns the number of cells that met either floor. */
long or_mhd_floor(double *U, int nx, int ny, int nz, int ndim, double gam, double p_floor, double rho_floor)
{
    grid_t G;
    int c[3];
    long count = 0;
    grid_init(&G, nx, ny, nz, ndim);
    const long nc = G.ncell;
    for (c[2] = 0; c[2] < G.n[2]; c[2]++)
        for (c[1] = 0; c[1] < G.n[1]; c[1]++)
            for (c[0] = 0; c[0] < G.n[0]; c[0]++) {
                const long id = cidx(&G, c);
                int hit = 0;
                double rho = U[id];
                if (rho_floor > 0.0 && rho < rho_floor) {
                    rho = rho_floor;
                    U[id] = rho;
                    hit = 1;
                }
                if (p_floor > 0.0) {
                    double m2 = U[nc + id] * U[nc + id] + U[2 * nc + id] * U[2 * nc + id] +
                                U[3 * nc + id] * U[3 * nc + id];
                    double B2 = U[5 * nc + id] * U[5 * nc + id] + U[6 * nc + id] * U[6 * nc + id] +
                                U[7 * nc + id] * U[7 * nc + id];
                    double p = (gam - 1.0) * (U[4 * nc + id] - 0.5 * m2 / rho - 0.5 * B2);
                    if (p < p_floor) {
                        U[4 * nc + id] = p_floor / (gam - 1.0) + 0.5 * m2 / rho + 0.5 * B2;
                        hit = 1;
                    }
                }
                count += hit;
            }
    return count;
}
