// mhd_device.cuh -- device arithmetic of the CTU-MHD step, templated on the
// working precision R (double for the FP64 path, float for the mixed path).
//
// Physics: ideal MHD, Section 2.1 Eq. (1)-(2) of Mignone et al. (2012), with
// GLM cleaning, Section 3 Eq. (glm2x2).  Local 1-D frame of a sweep along
// direction d: (rho, v_n, v_t1, v_t2, p, B_n, B_t1, B_t2, psi), with
// (t1, t2) = (y, z), (x, z), (x, y) for d = x, y, z.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace ctu {

constexpr int NV = 9;

// Local component q of a sweep along d reads global component perm(d, q).
__host__ __device__ __forceinline__ int perm(int d, int q)
{
    // d = 0: identity; d = 1: swap 1<->2 and 5<->6; d = 2: (3,1,2) and (7,5,6)
    if (d == 0) return q;
    if (d == 1) {
        if (q == 1) return 2;
        if (q == 2) return 1;
        if (q == 5) return 6;
        if (q == 6) return 5;
        return q;
    }
    if (q == 1) return 3;
    if (q == 2) return 1;
    if (q == 3) return 2;
    if (q == 5) return 7;
    if (q == 6) return 5;
    if (q == 7) return 6;
    return q;
}

template <class R> struct Tol;
template <> struct Tol<double> {
    static __device__ __forceinline__ double bt() { return 1.0e-24; }
    static __device__ __forceinline__ double hlld() { return 1.0e-12; }
};
// bt(): transverse field below which the Alfven basis is the degenerate
// one.  The same relative threshold in both precisions, so that a state
// with B_t != 0 in float64 (e.g. B_z = 0 exactly in 2-D, B_y small) keeps
// the basis along B_t and exact zeros of v_z, B_z stay exact; bt2 above
// 1e-24 a2 keeps B_t itself in the normal float range.
template <> struct Tol<float> {
    static __device__ __forceinline__ float bt() { return 1.0e-24f; }
    static __device__ __forceinline__ float hlld() { return 1.0e-6f; }
};

// ---------------------------------------------------------------- reconstruction

// MinMod, Eq. (minmod): (sign a + sign b)/2 * min(|a|, |b|)
template <class R> __device__ __forceinline__ R minmod(R a, R b)
{
    if (a > R(0) && b > R(0)) return fmin(a, b);
    if (a < R(0) && b < R(0)) return fmax(a, b);
    return R(0);
}

// Monotonised-central slope, Eq. (MClim): minmod((dm + dp)/2, 2 minmod(dm,
// dp)), i.e. for dm, dp of one sign that sign times min(|dm + dp|/2, 2|dm|,
// 2|dp|), else 0 (written without branches; a product dm dp below the
// normal range counts as zero).
template <class R> __device__ __forceinline__ R mc_slope(R dm, R dp)
{
    const R m = fmin(R(0.5) * fabs(dm + dp), R(2) * fmin(fabs(dm), fabs(dp)));
    return dm * dp > R(0) ? copysign(m, dm) : R(0);
}

// The linear reconstruction's other slopes (RECON_LIN, chosen at run time
// by lim = CTU_LINEAR_*): MinMod, Eq. (minmod); harmonic mean, Eq.
// (harmonic_lim); Van Albada, Eq. (vanalbada_lim).
template <class R> __device__ __forceinline__ R lin_slope(R dm, R dp, int lim)
{
    const R prod = dm * dp;
    R s;
    if (lim == 2)
        s = copysign(fmin(fabs(dm), fabs(dp)), dm);
    else if (lim == 3)
        s = R(2) * prod / (dm + dp);
    else
        s = prod * (dm + dp) / (dm * dm + dp * dp);
    return prod > R(0) ? s : R(0);
}

// Reconstruction kinds of the kernel templates: MC-linear, PPM, linear with a
// run-time slope, improved WENO3, and PPM and MC-linear again in kernels that
// also offer the reference states of the tracing (the kinds from RECON_LIN
// to RECON_MC_REF take the tracing mode at run time among all four; RECON_MC and
// RECON_PPM among the first two, as before).
// The hybrid kinds (RECON_PPM_HYB, RECON_MC_HYB) reconstruct with MinMod
// where the shock flags ask for it (lim == 2 at run time).
// RECON_PPM_HLLC and RECON_MC_HLLC take the HLLC solver on every face.
// RECON_PPM_PAR and RECON_MC_PAR add the parabolic terms, thermal
// conduction and viscosity (tracing modes ALL and UPWIND, as RECON_PPM and
// RECON_MC).
// RECON_PPM_MT and RECON_MC_MT take the transverse fluxes of the corner
// coupling from the normal predictor states (Mignone & Tzeferacos 2010).
enum {
    RECON_MC = 0, RECON_PPM = 1, RECON_LIN = 2, RECON_WENO3 = 3, RECON_PPM_REF = 4, RECON_MC_REF = 5,
    RECON_PPM_HYB = 6, RECON_MC_HYB = 7, RECON_PPM_HLLC = 8, RECON_MC_HLLC = 9, RECON_PPM_PAR = 10,
    RECON_MC_PAR = 11, RECON_PPM_MT = 12, RECON_MC_MT = 13
};

__host__ __device__ constexpr int recon_base(int r)
{
    return (r == RECON_PPM_REF || r == RECON_PPM_HYB || r == RECON_PPM_HLLC || r == RECON_PPM_PAR ||
            r == RECON_PPM_MT)
               ? RECON_PPM
               : ((r == RECON_MC_REF || r == RECON_MC_HYB || r == RECON_MC_HLLC || r == RECON_MC_PAR ||
                   r == RECON_MC_MT)
                      ? RECON_MC
                      : r);
}
__host__ __device__ constexpr bool recon_mt(int r) { return r == RECON_PPM_MT || r == RECON_MC_MT; }

__host__ __device__ constexpr bool recon_hybrid(int r) { return r == RECON_PPM_HYB || r == RECON_MC_HYB; }
__host__ __device__ constexpr bool recon_hllc(int r) { return r == RECON_PPM_HLLC || r == RECON_MC_HLLC; }
__host__ __device__ constexpr bool recon_par(int r) { return r == RECON_PPM_PAR || r == RECON_MC_PAR; }

// Interface values w_(i,+/-) of one characteristic field from w_(i-2..i+2):
// PPM, Eq. (ppm1) + parabolic limiter Eq. (ppm_parabolic_lim); linear,
// Eq. (Linear), with the MC slope or the slope `lim` selects; improved WENO3,
// Eq. (WENO3) with the weights of Eq. (WENO3a), where eps2 is the square of
// the cell width in this field's units (the Delta x^2 of Eq. WENO3a divided by
// the square of the factor that turns this field into the Roe-Balsara
// characteristic variable).
template <class R, int RK>
__device__ __forceinline__ void reconstruct(R w0m2, R w0m1, R w0, R w0p1, R w0p2, int lim, R eps2, R &wp, R &wm)
{
    constexpr int PPM = recon_base(RK);
    if (recon_hybrid(RK) && lim == 2) {  // MinMod near a shock
        const R dm = w0 - w0m1, dp = w0p1 - w0;
        const R s = dm * dp > R(0) ? copysign(fmin(fabs(dm), fabs(dp)), dm) : R(0);
        wp = w0 + R(0.5) * s;
        wm = w0 - R(0.5) * s;
        return;
    }
    if (PPM == RECON_WENO3) {
        const R dp = w0p1 - w0, dm = w0 - w0m1;
        const R d2 = (dp - dm) * (dp - dm);
        const R ap = R(1) + d2 / (eps2 + dp * dp);
        const R am = R(1) + d2 / (eps2 + dm * dm);
        wp = w0 + (ap * dp + R(0.5) * am * dm) / (R(2) * ap + am);
        wm = w0 - (am * dm + R(0.5) * ap * dp) / (R(2) * am + ap);
        return;
    }
    if (PPM == RECON_LIN) {
        const R s = lin_slope(w0 - w0m1, w0p1 - w0, lim);
        wp = w0 + R(0.5) * s;
        wm = w0 - R(0.5) * s;
        return;
    }
    R s0 = mc_slope(w0 - w0m1, w0p1 - w0);
    if (PPM == RECON_MC) {
        wp = w0 + R(0.5) * s0;
        wm = w0 - R(0.5) * s0;
        return;
    }
    R sm = mc_slope(w0m1 - w0m2, w0 - w0m1);
    R sp = mc_slope(w0p1 - w0, w0p2 - w0p1);
    R p = R(0.5) * (w0 + w0p1) - (sp - s0) * R(1.0 / 6.0);
    R m = R(0.5) * (w0 + w0m1) + (sm - s0) * R(1.0 / 6.0);
    R dp = p - w0, dm = m - w0;
    // a local extremum flattens the cell; otherwise the overshooting side is
    // pulled back so that the parabola stays monotone
    const bool extremum = dp * dm > R(0);
    const R ndp = (fabs(dp) >= R(2) * fabs(dm)) ? R(-2) * dm : dp;
    const R ndm = (fabs(dm) >= R(2) * fabs(dp)) ? R(-2) * dp : dm;
    wp = w0 + (extremum ? R(0) : ndp);
    wm = w0 + (extremum ? R(0) : ndm);
}

// Tracing of one characteristic field to t^(n+1/2), Eq. (wnorm_predp) and
// (wnorm_predm), w* = w_ref + beta (traced - w_ref).  mode 0
// (CTU_TRACE_ALL) traces every field to both interfaces (no reference
// state); the others apply beta_+ = [nu > 0], beta_- = [nu < 0] with
// w_ref = w_(+/-) (1, CTU_TRACE_UPWIND), the cell-centre value w_(i,0)
// (2, CTU_TRACE_CENTER) or Colella-Woodward's state, the field traced with
// numax to the + and numin to the - interface (3, CTU_TRACE_CW84).  Modes 2
// and 3 exist only where REF is set.
template <class R, bool REF>
__device__ __forceinline__ void trace(R wp, R w0, R wm, R nu, int mode, R numax, R numin, R &tp, R &tm)
{
    R dw = wp - wm;
    R d2w = wp - R(2) * w0 + wm;
    const R up = wp - R(0.5) * nu * (dw + d2w * (R(3) - R(2) * nu));
    const R um = wm - R(0.5) * nu * (dw - d2w * (R(3) + R(2) * nu));
    R rp = wp, rm = wm;
    if (REF) {
        if (mode == 2) {
            rp = w0;
            rm = w0;
        } else if (mode == 3) {
            rp = wp - R(0.5) * numax * (dw + d2w * (R(3) - R(2) * numax));
            rm = wm - R(0.5) * numin * (dw - d2w * (R(3) + R(2) * numin));
        }
    }
    tp = ((mode == 0) | (nu > R(0))) ? up : rp;
    tm = ((mode == 0) | (nu < R(0))) ? um : rm;
}

// ---------------------------------------------------------------- normal predictor

// Characteristic normal predictor of one cell, Section 3.2: project the
// primitive stencil vs[m] = V_(i+m-2) (local order) onto the left
// eigenvectors of V_i (Eq. char_var), reconstruct, trace, and recombine with
// the right eigenvectors, adding the S_Bx dB_n/dx + S_psi dpsi/dx source.
//
// Eigenvectors: primitive system of Eq. (1) along the normal, 7 MHD waves on
// (rho, v_n, v_t1, v_t2, p, B_t1, B_t2) (Roe-Balsara normalisation), plus the
// 2 GLM waves (+/- c_h) on (B_n, psi).  Each left eigenvector is used up to a
// positive factor, with the inverse factor on its right eigenvector;
// reconstruction and tracing are positively homogeneous, so the result is
// unchanged.
template <class R, int PPM>
__device__ __forceinline__ void char_predict(const R (&vs)[5][NV], R gam, R ch, R dtdx, int upwind, int lim,
                                             R dx2, R (&Vp)[NV], R (&Vm)[NV])
{
    constexpr bool REF = PPM >= RECON_LIN && PPM <= RECON_MC_REF;
    const R rho = vs[2][0], u = vs[2][1], v1c = vs[2][2], v2c = vs[2][3], pc = vs[2][4];
    const R Bn = vs[2][5], B1c = vs[2][6], B2c = vs[2][7];
    const R a2 = gam * pc / rho;
    const R a = sqrt(a2);
    const R srho = sqrt(rho);
    const R bn2 = Bn * Bn / rho;
    const R bt2 = (B1c * B1c + B2c * B2c) / rho;
    const R b2 = bn2 + bt2;
    const R disc = sqrt((a2 - b2) * (a2 - b2) + R(4) * a2 * bt2);
    const R cf2 = R(0.5) * (a2 + b2 + disc);
    const R cs2 = a2 * bn2 / cf2;
    const R cf = sqrt(cf2), cs = sqrt(cs2), ca = sqrt(bn2);
    R fa, sa;
    if (a2 >= b2) {
        fa = R(0.5) * (a2 - b2 + disc);
        sa = (disc + (a2 - b2) > R(0)) ? R(2) * a2 * bt2 / (disc + (a2 - b2)) : R(0);
    } else {
        sa = R(0.5) * (b2 - a2 + disc);
        fa = R(2) * a2 * bt2 / (disc + (b2 - a2));
    }
    R af, as;
    if (disc > R(0)) {
        af = sqrt(fa / disc);
        as = sqrt(sa / disc);
    } else {
        af = R(1);
        as = R(0);
    }
    R be1, be2;
    if (bt2 > Tol<R>::bt() * a2) {
        const R bt = sqrt(B1c * B1c + B2c * B2c);
        be1 = B1c / bt;
        be2 = B2c / bt;
    } else {
        be1 = R(0.70710678118654752440);
        be2 = R(0.70710678118654752440);
    }
    const R S = copysign(R(1), Bn);
    const R irho = R(1) / rho;
    const R isr = R(1) / srho;
    const R ich = R(1) / ch;

    // characteristic variables on the stencil (scaled left eigenvectors)
    R wf_p[5], wf_m[5], wa_p[5], wa_m[5], ws_p[5], ws_m[5], we[5], wg_m[5], wg_p[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const R um = vs[m][1], v1 = vs[m][2], v2 = vs[m][3], pm = vs[m][4];
        const R bnm = vs[m][5], b1 = vs[m][6], b2m = vs[m][7], psm = vs[m][8];
        const R PV = be1 * v1 + be2 * v2;
        const R PB = be1 * b1 + be2 * b2m;
        const R P = be1 * v2 - be2 * v1;
        const R Q = S * (be2 * b1 - be1 * b2m) * isr;
        const R Xf = af * cf * um - as * cs * S * PV;
        const R Yf = af * pm * irho + as * a * PB * isr;
        const R Xs = as * cs * um + af * cf * S * PV;
        const R Ys = as * pm * irho - af * a * PB * isr;
        wf_p[m] = Yf + Xf;
        wf_m[m] = Yf - Xf;
        ws_p[m] = Ys + Xs;
        ws_m[m] = Ys - Xs;
        wa_p[m] = P + Q;
        wa_m[m] = P - Q;
        we[m] = vs[m][0] - pm / a2;
        wg_p[m] = bnm + psm * ich;
        wg_m[m] = bnm - psm * ich;
    }
    R rp, rm, tpf_p, tmf_p, tpf_m, tmf_m, tpa_p, tma_p, tpa_m, tma_m;
    R tps_p, tms_p, tps_m, tms_m, tpe, tme, tpg_p, tmg_p, tpg_m, tmg_m;
    // WENO3's cell-width term in each field's units: the fields above are the
    // Roe-Balsara characteristic variables times 2 a^2 (fast, slow), 2
    // (Alfven, GLM) and 1 (entropy)
    const R e_fs = PPM == RECON_WENO3 ? dx2 * (R(4) * a2 * a2) : R(0);
    const R e_ag = PPM == RECON_WENO3 ? dx2 * R(4) : R(0);
    // the extreme Courant numbers of the seven MHD waves, for mode 3
    const R numax = REF ? fmax(R(0), (u + cf) * dtdx) : R(0);
    const R numin = REF ? fmin(R(0), (u - cf) * dtdx) : R(0);
    reconstruct<R, PPM>(wf_m[0], wf_m[1], wf_m[2], wf_m[3], wf_m[4], lim, e_fs, rp, rm);
    trace<R, REF>(rp, wf_m[2], rm, (u - cf) * dtdx, upwind, numax, numin, tpf_m, tmf_m);
    reconstruct<R, PPM>(wa_m[0], wa_m[1], wa_m[2], wa_m[3], wa_m[4], lim, e_ag, rp, rm);
    trace<R, REF>(rp, wa_m[2], rm, (u - ca) * dtdx, upwind, numax, numin, tpa_m, tma_m);
    reconstruct<R, PPM>(ws_m[0], ws_m[1], ws_m[2], ws_m[3], ws_m[4], lim, e_fs, rp, rm);
    trace<R, REF>(rp, ws_m[2], rm, (u - cs) * dtdx, upwind, numax, numin, tps_m, tms_m);
    reconstruct<R, PPM>(we[0], we[1], we[2], we[3], we[4], lim, dx2, rp, rm);
    trace<R, REF>(rp, we[2], rm, u * dtdx, upwind, numax, numin, tpe, tme);
    reconstruct<R, PPM>(ws_p[0], ws_p[1], ws_p[2], ws_p[3], ws_p[4], lim, e_fs, rp, rm);
    trace<R, REF>(rp, ws_p[2], rm, (u + cs) * dtdx, upwind, numax, numin, tps_p, tms_p);
    reconstruct<R, PPM>(wa_p[0], wa_p[1], wa_p[2], wa_p[3], wa_p[4], lim, e_ag, rp, rm);
    trace<R, REF>(rp, wa_p[2], rm, (u + ca) * dtdx, upwind, numax, numin, tpa_p, tma_p);
    reconstruct<R, PPM>(wf_p[0], wf_p[1], wf_p[2], wf_p[3], wf_p[4], lim, e_fs, rp, rm);
    trace<R, REF>(rp, wf_p[2], rm, (u + cf) * dtdx, upwind, numax, numin, tpf_p, tmf_p);
    R gpr, gmr, gpl, gml; // reconstructed (untraced) GLM fields at + and - interfaces
    reconstruct<R, PPM>(wg_m[0], wg_m[1], wg_m[2], wg_m[3], wg_m[4], lim, e_ag, gpl, gml);
    trace<R, REF>(gpl, wg_m[2], gml, -ch * dtdx, upwind, numax, numin, tpg_m, tmg_m);
    reconstruct<R, PPM>(wg_p[0], wg_p[1], wg_p[2], wg_p[3], wg_p[4], lim, e_ag, gpr, gmr);
    trace<R, REF>(gpr, wg_p[2], gmr, ch * dtdx, upwind, numax, numin, tpg_p, tmg_p);

    // recombination with the right eigenvectors (scaled accordingly)
    const R i2a2 = R(0.5) / a2;
    const R sq_a = srho * a;
    auto combine = [&](R fp, R fm, R ap, R am, R sp_, R sm_, R e, R gp, R gm, R (&V)[NV]) {
        const R fs = fp + fm, fd = fp - fm, ss = sp_ + sm_, sd = sp_ - sm_;
        const R as_ = ap + am, ad = ap - am;
        V[0] = (rho * af * fs + rho * as * ss) * i2a2 + e;
        V[1] = (af * cf * fd + as * cs * sd) * i2a2;
        const R tv = (-as * cs * fd + af * cf * sd) * S * i2a2;
        V[2] = tv * be1 - R(0.5) * be2 * as_;
        V[3] = tv * be2 + R(0.5) * be1 * as_;
        V[4] = R(0.5) * rho * (af * fs + as * ss);
        V[5] = R(0.5) * (gp + gm);
        const R tb = (as * fs - af * ss) * sq_a * i2a2;
        V[6] = tb * be1 + R(0.5) * S * srho * be2 * ad;
        V[7] = tb * be2 - R(0.5) * S * srho * be1 * ad;
        V[8] = R(0.5) * ch * (gp - gm);
    };
    combine(tpf_p, tpf_m, tpa_p, tpa_m, tps_p, tps_m, tpe, tpg_p, tpg_m, Vp);
    combine(tmf_p, tmf_m, tma_p, tma_m, tms_p, tms_m, tme, tmg_p, tmg_m, Vm);

    // S_Bx dB_n/dx + S_psi dpsi/dx: minus the primitive-Jacobian columns that
    // couple the 7-wave block to d(B_n)/dn and d(psi)/dn, with the undivided
    // jumps of the reconstructed GLM fields across the cell.
    const R dgp = gpr - gmr, dgm = gpl - gml;
    const R dBn = R(0.5) * (dgp + dgm);
    const R dps = R(0.5) * ch * (dgp - dgm);
    const R vB = u * Bn + v1c * B1c + v2c * B2c;
    const R h = R(0.5) * dtdx;
    const R s1 = h * Bn * irho * dBn;
    const R s2 = h * B1c * irho * dBn;
    const R s3 = h * B2c * irho * dBn;
    const R s4 = h * (gam - R(1)) * (Bn * dps - vB * dBn);
    const R s6 = h * v1c * dBn;
    const R s7 = h * v2c * dBn;
    Vp[1] += s1; Vm[1] += s1;
    Vp[2] += s2; Vm[2] += s2;
    Vp[3] += s3; Vm[3] += s3;
    Vp[4] += s4; Vm[4] += s4;
    Vp[6] += s6; Vm[6] += s6;
    Vp[7] += s7; Vm[7] += s7;
}

// ---------------------------------------------------------------- Riemann solver

template <class R> __device__ __forceinline__ R fast_speed(R rho, R p, R Bn, R B1, R B2, R gam)
{
    const R a2 = gam * p / rho;
    const R bn2 = Bn * Bn / rho;
    const R bt2 = (B1 * B1 + B2 * B2) / rho;
    const R b2 = bn2 + bt2;
    const R disc = sqrt((a2 - b2) * (a2 - b2) + R(4) * a2 * bt2);
    return sqrt(R(0.5) * (a2 + b2 + disc));
}

// Numerical flux along the local normal: exact linear (B_n, psi) face solve
// of the GLM system (Dedner et al. 2002), then HLLD (Miyoshi & Kusano 2005)
// with B_n set to the face value on both sides.  Returns true if an input
// state has rho <= 0 or p <= 0.
template <class R>
__device__ __forceinline__ bool riemann_hlld(const R (&L)[NV], const R (&Rt)[NV], R gam, R ch, R (&F)[NV])
{
    const bool bad = !(L[0] > R(0) && L[4] > R(0) && Rt[0] > R(0) && Rt[4] > R(0));
    const R Bm = R(0.5) * (L[5] + Rt[5]) - R(0.5) * (Rt[8] - L[8]) / ch;
    const R pm = R(0.5) * (L[8] + Rt[8]) - R(0.5) * ch * (Rt[5] - L[5]);
    const R Bn = Bm;
    const R igm = R(1) / (gam - R(1));

    const R rL = L[0], uL = L[1], vL = L[2], wL = L[3], pL = L[4], yL = L[6], zL = L[7];
    const R rR = Rt[0], uR = Rt[1], vR = Rt[2], wR = Rt[3], pR = Rt[4], yR = Rt[6], zR = Rt[7];
    const R BsqL = Bn * Bn + yL * yL + zL * zL;
    const R BsqR = Bn * Bn + yR * yR + zR * zR;
    const R ptL = pL + R(0.5) * BsqL, ptR = pR + R(0.5) * BsqR;
    const R EL = pL * igm + R(0.5) * rL * (uL * uL + vL * vL + wL * wL) + R(0.5) * BsqL;
    const R ER = pR * igm + R(0.5) * rR * (uR * uR + vR * vR + wR * wR) + R(0.5) * BsqR;
    const R vBL = uL * Bn + vL * yL + wL * zL;
    const R vBR = uR * Bn + vR * yR + wR * zR;

    // physical fluxes
    R FL[8], FR[8], UL[8], UR[8];
    FL[0] = rL * uL; FL[1] = rL * uL * uL + ptL - Bn * Bn; FL[2] = rL * uL * vL - Bn * yL;
    FL[3] = rL * uL * wL - Bn * zL; FL[4] = (EL + ptL) * uL - Bn * vBL; FL[5] = R(0);
    FL[6] = uL * yL - Bn * vL; FL[7] = uL * zL - Bn * wL;
    FR[0] = rR * uR; FR[1] = rR * uR * uR + ptR - Bn * Bn; FR[2] = rR * uR * vR - Bn * yR;
    FR[3] = rR * uR * wR - Bn * zR; FR[4] = (ER + ptR) * uR - Bn * vBR; FR[5] = R(0);
    FR[6] = uR * yR - Bn * vR; FR[7] = uR * zR - Bn * wR;
    UL[0] = rL; UL[1] = rL * uL; UL[2] = rL * vL; UL[3] = rL * wL; UL[4] = EL; UL[5] = Bn;
    UL[6] = yL; UL[7] = zL;
    UR[0] = rR; UR[1] = rR * uR; UR[2] = rR * vR; UR[3] = rR * wR; UR[4] = ER; UR[5] = Bn;
    UR[6] = yR; UR[7] = zR;

    const R cfL = fast_speed(rL, pL, Bn, yL, zL, gam);
    const R cfR = fast_speed(rR, pR, Bn, yR, zR, gam);
    const R cmax = fmax(cfL, cfR);
    const R SL = fmin(uL, uR) - cmax;
    const R SR = fmax(uL, uR) + cmax;

    R G[8];
    if (SL >= R(0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = FL[q];
    } else if (SR <= R(0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = FR[q];
    } else {
        const R sdL = SL - uL, sdR = SR - uR;
        const R den = sdR * rR - sdL * rL;
        const R SM = (sdR * rR * uR - sdL * rL * uL - ptR + ptL) / den;
        const R pts = (sdR * rR * ptL - sdL * rL * ptR + rL * rR * sdR * sdL * (uR - uL)) / den;
        const R rsL = rL * sdL / (SL - SM);
        const R rsR = rR * sdR / (SR - SM);
        const R dL = rL * sdL * (SL - SM) - Bn * Bn;
        const R dR = rR * sdR * (SR - SM) - Bn * Bn;
        R vsL, wsL, ysL, zsL, vsR, wsR, ysR, zsR;
        if (fabs(dL) <= Tol<R>::hlld() * (rL * sdL * sdL + Bn * Bn)) {
            vsL = vL; wsL = wL; ysL = yL; zsL = zL;
        } else {
            const R idL = R(1) / dL;
            const R f = (rL * sdL * sdL - Bn * Bn) * idL;
            const R g = Bn * (SM - uL) * idL;
            vsL = vL - yL * g; wsL = wL - zL * g; ysL = yL * f; zsL = zL * f;
        }
        if (fabs(dR) <= Tol<R>::hlld() * (rR * sdR * sdR + Bn * Bn)) {
            vsR = vR; wsR = wR; ysR = yR; zsR = zR;
        } else {
            const R idR = R(1) / dR;
            const R f = (rR * sdR * sdR - Bn * Bn) * idR;
            const R g = Bn * (SM - uR) * idR;
            vsR = vR - yR * g; wsR = wR - zR * g; ysR = yR * f; zsR = zR * f;
        }
        const R vBsL = SM * Bn + vsL * ysL + wsL * zsL;
        const R vBsR = SM * Bn + vsR * ysR + wsR * zsR;
        const R EsL = (sdL * EL - ptL * uL + pts * SM + Bn * (vBL - vBsL)) / (SL - SM);
        const R EsR = (sdR * ER - ptR * uR + pts * SM + Bn * (vBR - vBsR)) / (SR - SM);
        R UsL[8], UsR[8];
        UsL[0] = rsL; UsL[1] = rsL * SM; UsL[2] = rsL * vsL; UsL[3] = rsL * wsL; UsL[4] = EsL;
        UsL[5] = Bn; UsL[6] = ysL; UsL[7] = zsL;
        UsR[0] = rsR; UsR[1] = rsR * SM; UsR[2] = rsR * vsR; UsR[3] = rsR * wsR; UsR[4] = EsR;
        UsR[5] = Bn; UsR[6] = ysR; UsR[7] = zsR;
        const R sqL = sqrt(rsL), sqR = sqrt(rsR);
        const R SLs = SM - fabs(Bn) / sqL;
        const R SRs = SM + fabs(Bn) / sqR;
        if (SLs >= R(0)) {
#pragma unroll
            for (int q = 0; q < 8; ++q) G[q] = FL[q] + SL * (UsL[q] - UL[q]);
        } else if (SRs <= R(0)) {
#pragma unroll
            for (int q = 0; q < 8; ++q) G[q] = FR[q] + SR * (UsR[q] - UR[q]);
        } else {
            const R sB = copysign(R(1), Bn);
            const R isq = R(1) / (sqL + sqR);
            const R vss = (sqL * vsL + sqR * vsR + (ysR - ysL) * sB) * isq;
            const R wss = (sqL * wsL + sqR * wsR + (zsR - zsL) * sB) * isq;
            const R yss = (sqL * ysR + sqR * ysL + sqL * sqR * (vsR - vsL) * sB) * isq;
            const R zss = (sqL * zsR + sqR * zsL + sqL * sqR * (wsR - wsL) * sB) * isq;
            const R vBss = SM * Bn + vss * yss + wss * zss;
            R Uss[8];
            if (SM >= R(0)) {
                Uss[0] = rsL; Uss[1] = rsL * SM; Uss[2] = rsL * vss; Uss[3] = rsL * wss;
                Uss[4] = EsL - sqL * (vBsL - vBss) * sB;
                Uss[5] = Bn; Uss[6] = yss; Uss[7] = zss;
#pragma unroll
                for (int q = 0; q < 8; ++q) G[q] = FL[q] + SL * (UsL[q] - UL[q]) + SLs * (Uss[q] - UsL[q]);
            } else {
                Uss[0] = rsR; Uss[1] = rsR * SM; Uss[2] = rsR * vss; Uss[3] = rsR * wss;
                Uss[4] = EsR + sqR * (vBsR - vBss) * sB;
                Uss[5] = Bn; Uss[6] = yss; Uss[7] = zss;
#pragma unroll
                for (int q = 0; q < 8; ++q) G[q] = FR[q] + SR * (UsR[q] - UR[q]) + SRs * (Uss[q] - UsR[q]);
            }
        }
    }
    F[0] = G[0]; F[1] = G[1]; F[2] = G[2]; F[3] = G[3]; F[4] = G[4];
    F[5] = pm;
    F[6] = G[6]; F[7] = G[7];
    F[8] = ch * ch * Bm;
    return bad;
}

// HLL flux (Harten, Lax & van Leer), the solver of the hybrid integration at
// the faces of shocked cells: the same GLM face solve and outer wave speeds
// as riemann_hlld, then the single HLL average state.
template <class R>
__device__ __forceinline__ bool riemann_hll(const R (&L)[NV], const R (&Rt)[NV], R gam, R ch, R (&F)[NV])
{
    const bool bad = !(L[0] > R(0) && L[4] > R(0) && Rt[0] > R(0) && Rt[4] > R(0));
    const R Bm = R(0.5) * (L[5] + Rt[5]) - R(0.5) * (Rt[8] - L[8]) / ch;
    const R pm = R(0.5) * (L[8] + Rt[8]) - R(0.5) * ch * (Rt[5] - L[5]);
    const R Bn = Bm;
    const R igm = R(1) / (gam - R(1));
    const R rL = L[0], uL = L[1], vL = L[2], wL = L[3], pL = L[4], yL = L[6], zL = L[7];
    const R rR = Rt[0], uR = Rt[1], vR = Rt[2], wR = Rt[3], pR = Rt[4], yR = Rt[6], zR = Rt[7];
    const R BsqL = Bn * Bn + yL * yL + zL * zL;
    const R BsqR = Bn * Bn + yR * yR + zR * zR;
    const R ptL = pL + R(0.5) * BsqL, ptR = pR + R(0.5) * BsqR;
    const R EL = pL * igm + R(0.5) * rL * (uL * uL + vL * vL + wL * wL) + R(0.5) * BsqL;
    const R ER = pR * igm + R(0.5) * rR * (uR * uR + vR * vR + wR * wR) + R(0.5) * BsqR;
    const R vBL = uL * Bn + vL * yL + wL * zL;
    const R vBR = uR * Bn + vR * yR + wR * zR;
    R FL[8], FR[8], UL[8], UR[8];
    FL[0] = rL * uL; FL[1] = rL * uL * uL + ptL - Bn * Bn; FL[2] = rL * uL * vL - Bn * yL;
    FL[3] = rL * uL * wL - Bn * zL; FL[4] = (EL + ptL) * uL - Bn * vBL; FL[5] = R(0);
    FL[6] = uL * yL - Bn * vL; FL[7] = uL * zL - Bn * wL;
    FR[0] = rR * uR; FR[1] = rR * uR * uR + ptR - Bn * Bn; FR[2] = rR * uR * vR - Bn * yR;
    FR[3] = rR * uR * wR - Bn * zR; FR[4] = (ER + ptR) * uR - Bn * vBR; FR[5] = R(0);
    FR[6] = uR * yR - Bn * vR; FR[7] = uR * zR - Bn * wR;
    UL[0] = rL; UL[1] = rL * uL; UL[2] = rL * vL; UL[3] = rL * wL; UL[4] = EL; UL[5] = Bn;
    UL[6] = yL; UL[7] = zL;
    UR[0] = rR; UR[1] = rR * uR; UR[2] = rR * vR; UR[3] = rR * wR; UR[4] = ER; UR[5] = Bn;
    UR[6] = yR; UR[7] = zR;
    const R cfL = fast_speed(rL, pL, Bn, yL, zL, gam);
    const R cfR = fast_speed(rR, pR, Bn, yR, zR, gam);
    const R cmax = fmax(cfL, cfR);
    const R SL = fmin(uL, uR) - cmax;
    const R SR = fmax(uL, uR) + cmax;
    R G[8];
    if (SL >= R(0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = FL[q];
    } else if (SR <= R(0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = FR[q];
    } else {
        const R iw = R(1) / (SR - SL);
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) * iw;
    }
    F[0] = G[0]; F[1] = G[1]; F[2] = G[2]; F[3] = G[3]; F[4] = G[4];
    F[5] = pm;
    F[6] = G[6]; F[7] = G[7];
    F[8] = ch * ch * Bm;
    return bad;
}

// HLLC flux for MHD (Li 2005): the GLM face solve and outer speeds of
// riemann_hlld; the HLL average state gives the contact speed
// S_M = (rho u)_hll / rho_hll and the star states' transverse field and
// velocity, B*_t = B_t,hll and v*_t = (rho v_t)_hll / rho_hll; with
// p*_t = rho_L (S_L - u_L)(S_M - u_L) + p_t,L each star state is
// rho* = rho (S - u)/(S - S_M), (rho u)* = rho* S_M,
// (rho v_t)* = (rho v_t (S - u) - B_n (B*_t - B_t))/(S - S_M),
// E* = (E (S - u) - p_t u + p*_t S_M + B_n (v.B - v*.B*))/(S - S_M), and
// the flux is F + S (U* - U) on the face's side of the contact.
template <class R>
__device__ __forceinline__ bool riemann_hllc(const R (&L)[NV], const R (&Rt)[NV], R gam, R ch, R (&F)[NV])
{
    const bool bad = !(L[0] > R(0) && L[4] > R(0) && Rt[0] > R(0) && Rt[4] > R(0));
    const R Bm = R(0.5) * (L[5] + Rt[5]) - R(0.5) * (Rt[8] - L[8]) / ch;
    const R pm = R(0.5) * (L[8] + Rt[8]) - R(0.5) * ch * (Rt[5] - L[5]);
    const R Bn = Bm;
    const R igm = R(1) / (gam - R(1));
    const R rL = L[0], uL = L[1], vL = L[2], wL = L[3], pL = L[4], yL = L[6], zL = L[7];
    const R rR = Rt[0], uR = Rt[1], vR = Rt[2], wR = Rt[3], pR = Rt[4], yR = Rt[6], zR = Rt[7];
    const R BsqL = Bn * Bn + yL * yL + zL * zL;
    const R BsqR = Bn * Bn + yR * yR + zR * zR;
    const R ptL = pL + R(0.5) * BsqL, ptR = pR + R(0.5) * BsqR;
    const R EL = pL * igm + R(0.5) * rL * (uL * uL + vL * vL + wL * wL) + R(0.5) * BsqL;
    const R ER = pR * igm + R(0.5) * rR * (uR * uR + vR * vR + wR * wR) + R(0.5) * BsqR;
    const R vBL = uL * Bn + vL * yL + wL * zL;
    const R vBR = uR * Bn + vR * yR + wR * zR;
    R FL[8], FR[8], UL[8], UR[8];
    FL[0] = rL * uL; FL[1] = rL * uL * uL + ptL - Bn * Bn; FL[2] = rL * uL * vL - Bn * yL;
    FL[3] = rL * uL * wL - Bn * zL; FL[4] = (EL + ptL) * uL - Bn * vBL; FL[5] = R(0);
    FL[6] = uL * yL - Bn * vL; FL[7] = uL * zL - Bn * wL;
    FR[0] = rR * uR; FR[1] = rR * uR * uR + ptR - Bn * Bn; FR[2] = rR * uR * vR - Bn * yR;
    FR[3] = rR * uR * wR - Bn * zR; FR[4] = (ER + ptR) * uR - Bn * vBR; FR[5] = R(0);
    FR[6] = uR * yR - Bn * vR; FR[7] = uR * zR - Bn * wR;
    UL[0] = rL; UL[1] = rL * uL; UL[2] = rL * vL; UL[3] = rL * wL; UL[4] = EL; UL[5] = Bn;
    UL[6] = yL; UL[7] = zL;
    UR[0] = rR; UR[1] = rR * uR; UR[2] = rR * vR; UR[3] = rR * wR; UR[4] = ER; UR[5] = Bn;
    UR[6] = yR; UR[7] = zR;
    const R cfL = fast_speed(rL, pL, Bn, yL, zL, gam);
    const R cfR = fast_speed(rR, pR, Bn, yR, zR, gam);
    const R cmax = fmax(cfL, cfR);
    const R SL = fmin(uL, uR) - cmax;
    const R SR = fmax(uL, uR) + cmax;
    R G[8];
    if (SL >= R(0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = FL[q];
    } else if (SR <= R(0)) {
#pragma unroll
        for (int q = 0; q < 8; ++q) G[q] = FR[q];
    } else {
        const R iw = R(1) / (SR - SL);
        R Uh[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) Uh[q] = (SR * UR[q] - SL * UL[q] - FR[q] + FL[q]) * iw;
        const R irh = R(1) / Uh[0];
        const R SM = Uh[1] * irh, vs = Uh[2] * irh, ws = Uh[3] * irh;
        const R ys = Uh[6], zs = Uh[7];
        const R pts = rL * (SL - uL) * (SM - uL) + ptL;
        const R vBs = SM * Bn + vs * ys + ws * zs;
        const bool right = SM < R(0);
        const R rr = right ? rR : rL, uu = right ? uR : uL, vv = right ? vR : vL, ww = right ? wR : wL;
        const R yy = right ? yR : yL, zz = right ? zR : zL, EE = right ? ER : EL, pt = right ? ptR : ptL;
        const R vB = right ? vBR : vBL, S = right ? SR : SL;
        const R sd = S - uu, iden = R(1) / (S - SM);
        R Us[8];
        Us[0] = rr * sd * iden;
        Us[1] = Us[0] * SM;
        Us[2] = (rr * vv * sd - Bn * (ys - yy)) * iden;
        Us[3] = (rr * ww * sd - Bn * (zs - zz)) * iden;
        Us[4] = (EE * sd - pt * uu + pts * SM + Bn * (vB - vBs)) * iden;
        Us[5] = Bn;
        Us[6] = ys;
        Us[7] = zs;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const R Fa = right ? FR[q] : FL[q], Ua = right ? UR[q] : UL[q];
            G[q] = Fa + S * (Us[q] - Ua);
        }
    }
    F[0] = G[0]; F[1] = G[1]; F[2] = G[2]; F[3] = G[3]; F[4] = G[4];
    F[5] = pm;
    F[6] = G[6]; F[7] = G[7];
    F[8] = ch * ch * Bm;
    return bad;
}

} // namespace ctu
