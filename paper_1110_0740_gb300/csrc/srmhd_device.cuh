// srmhd_device.cuh -- device arithmetic of special-relativistic MHD (GLM):
// Section 2.2 of Mignone et al. (2012), Eq. (rmhd) with the ideal-gas
// enthalpy of Eq. (gammaEos) or the Taub-Mathews one of Eq. (TMEos) (every
// function's gam: Gamma, or 0 for Taub-Mathews); the primitive MUSCL-Hancock
// normal predictor
// of Section 3.3; HLL fluxes (Harten, Lax & van Leer) with the exact (B_n,
// psi) GLM face solve (Dedner et al. 2002); signal speeds from the effective
// sound speed a^2 = c_s^2 + c_a^2 - c_s^2 c_a^2 (Leismann et al. 2005, Del
// Zanna et al. 2007); primitive recovery by bracketed Newton-Raphson on
// W = w gamma^2 (the unknown of Mignone & McKinney 2007), in float64.
//
// Variables: V = (rho, v, p, B, psi), U = (D = rho gamma, m, E = total - D,
// B, psi), sweeps use the same local frame as the MHD path.
#pragma once

#include "df.cuh"
#include "mhd_device.cuh"

namespace ctu {

enum : unsigned int { ST_REC = 4u, ST_SUPER = 8u };

// 1/x and 1/sqrt(x) in float64 for positive normal x inside the float
// exponent range: a float32 seed refined by two Newton-Raphson steps
// (r <- r (2 - x r); y <- y (3 - x y^2)/2), each doubling the number of
// correct bits (2^-22 -> 2^-44 -> beyond double precision), so the result is
// within about one ulp; far cheaper on GB300's FP64 pipe than the IEEE
// float64 divide and square root.  The seed moves between float64 and
// float32 by integer operations (df.cuh), not on the FP64 pipe.
__device__ __forceinline__ double rcp64(double x)
{
    double r = f2d_int(1.0f / df_split(x).hi);
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

__device__ __forceinline__ double rsqrt64(double x)
{
    double y = f2d_int(rsqrtf(df_split(x).hi));
    y = y * fma(-0.5 * x, y * y, 1.5);
    y = y * fma(-0.5 * x, y * y, 1.5);
    return y;
}

// 1/x, 1/sqrt(x) and sqrt(x) (x >= 0) of the working precision: hardware
// float32 forms, or the float64 refinements above.
template <class T> __device__ __forceinline__ T rcp_t(T x);
template <> __device__ __forceinline__ float rcp_t<float>(float x) { return 1.0f / x; }
template <> __device__ __forceinline__ double rcp_t<double>(double x) { return rcp64(x); }
template <class T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt64(x); }
template <class T> __device__ __forceinline__ T sqrt_t(T x) { return x > T(0) ? x * rsqrt_t<T>(x) : T(0); }
template <> __device__ __forceinline__ float sqrt_t<float>(float x) { return sqrtf(x); }

// Enthalpy density w(rho, p): the ideal gas of Eq. (gammaEos) for gam > 0
// (Gamma = gam), the Taub-Mathews gas of Eq. (TMEos) for gam == 0.
template <class T> __device__ __forceinline__ T sr_w(T rho, T p, T gam)
{
    if (gam > T(0)) return rho + gam * rcp_t<T>(gam - T(1)) * p;
    return T(2.5) * p + sqrt_t<T>(T(2.25) * p * p + rho * rho);
}

// Sound speed squared for enthalpy density w: Gamma p / w (ideal gas), or
// p (5 w - 8 p) / (3 w (w - p)) (Taub-Mathews, Mignone & McKinney 2007).
template <class T> __device__ __forceinline__ T sr_cs2(T p, T w, T gam)
{
    if (gam > T(0)) return gam * p / w;
    return p * (T(5) * w - T(8) * p) / (T(3) * w * (w - p));
}

// U(V) in precision T (T = double for states that feed a recovery).
template <class T, class R>
__device__ __forceinline__ void sr_cons(const R (&V)[NV], T gam, T (&U)[NV])
{
    const T rho = V[0], vx = V[1], vy = V[2], vz = V[3], p = V[4];
    const T bx = V[5], by = V[6], bz = V[7];
    const T v2 = vx * vx + vy * vy + vz * vz;
    const T lor2 = rcp_t<T>(T(1) - v2);
    const T W = sr_w<T>(rho, p, gam) * lor2;
    const T B2 = bx * bx + by * by + bz * bz;
    const T vB = vx * bx + vy * by + vz * bz;
    const T E2 = B2 * v2 - vB * vB;
    U[0] = rho * rsqrt_t<T>(T(1) - v2);
    U[1] = (W + B2) * vx - vB * bx;
    U[2] = (W + B2) * vy - vB * by;
    U[3] = (W + B2) * vz - vB * bz;
    U[4] = W - p + T(0.5) * (B2 + E2) - U[0];
    U[5] = bx;
    U[6] = by;
    U[7] = bz;
    U[8] = V[8];
}

// f(W) and f'(W) of the energy equation at fixed D, |m|^2, S = m.B, B^2,
// tau = E + D: f = W - p + B^2 (1 + v^2)/2 - S^2/(2 W^2) - tau with
// v^2(W) = (m^2 W^2 + S^2 (2W + B^2)) / (W^2 (W + B^2)^2),
// p from w = W (1 - v^2) and rho = D sqrt(1 - v^2): the ideal gas
// p = (Gamma-1)/Gamma (w - rho) for g1 = (Gamma-1)/Gamma > 0, or for g1 == 0
// the Taub-Mathews inverse 2 (w - rho)(w + rho)/(5 w + sqrt(9 w^2 + 16 rho^2)).
// false if v^2 >= 1.  The same with dv^2/dW and dp/dW.
__device__ __forceinline__ bool sr_energy_d(double W, double D, double m2, double S2, double B2, double tau,
                                            double g1, double &f, double &df, double &v2, double &p, double &dv2,
                                            double &dp)
{
    const double Wb = W + B2;
    const double N = m2 * W * W + S2 * (2.0 * W + B2);
    const double Dn = W * W * Wb * Wb;
    const double iDn = rcp64(Dn);
    v2 = N * iDn;
    if (!(v2 < 1.0)) return false;
    const double dN = 2.0 * m2 * W + 2.0 * S2;
    const double dDn = 2.0 * W * Wb * (2.0 * W + B2);
    dv2 = (dN * Dn - N * dDn) * iDn * iDn;
    const double is = rsqrt64(1.0 - v2);  // gamma
    const double s = (1.0 - v2) * is;
    if (g1 > 0.0) {
        p = g1 * (W * (1.0 - v2) - D * s);
        dp = g1 * ((1.0 - v2) + dv2 * (0.5 * D * is - W));
    } else {
        const double w = W * (1.0 - v2), rho = D * s;
        const double q2 = 9.0 * w * w + 16.0 * rho * rho;
        const double iq = rsqrt64(q2), q = q2 * iq;
        const double dpdw = 0.625 - 1.125 * w * iq, dpdr = -2.0 * rho * iq;
        p = 2.0 * (w - rho) * (w + rho) * rcp64(5.0 * w + q);
        dp = dpdw * ((1.0 - v2) - W * dv2) - dpdr * 0.5 * D * dv2 * is;
    }
    const double iW = rcp64(W);
    f = W - p + 0.5 * B2 * (1.0 + v2) - 0.5 * S2 * iW * iW - tau;
    df = 1.0 - dp + 0.5 * B2 * dv2 + S2 * iW * iW * iW;
    return true;
}


__device__ __forceinline__ bool sr_energy(double W, double D, double m2, double S2, double B2, double tau,
                                          double g1, double &f, double &df, double &v2, double &p)
{
    double dv2, dp;
    return sr_energy_d(W, D, m2, S2, B2, tau, g1, f, df, v2, p, dv2, dp);
}

// f(W) and f'(W) in float32: the first stage of the mixed-path recovery.
__device__ __forceinline__ bool sr_energy_f(float W, float D, float m2, float S2, float B2, float tau, float g1,
                                            float &f, float &df)
{
    const float Wb = W + B2;
    const float N = m2 * W * W + S2 * (2.0f * W + B2);
    const float Dn = W * W * Wb * Wb;
    const float iDn = 1.0f / Dn;
    const float v2 = N * iDn;
    if (!(v2 < 1.0f)) return false;
    const float dN = 2.0f * m2 * W + 2.0f * S2;
    const float dDn = 2.0f * W * Wb * (2.0f * W + B2);
    const float dv2 = (dN * Dn - N * dDn) * iDn * iDn;
    const float is = rsqrtf(1.0f - v2);
    const float sq = (1.0f - v2) * is;
    float p, dp;
    if (g1 > 0.0f) {
        p = g1 * (W * (1.0f - v2) - D * sq);
        dp = g1 * ((1.0f - v2) + dv2 * (0.5f * D * is - W));
    } else {
        const float w = W * (1.0f - v2), rho = D * sq;
        const float q2 = 9.0f * w * w + 16.0f * rho * rho;
        const float iq = rsqrtf(q2), q = q2 * iq;
        const float dpdw = 0.625f - 1.125f * w * iq, dpdr = -2.0f * rho * iq;
        p = 2.0f * (w - rho) * (w + rho) / (5.0f * w + q);
        dp = dpdw * ((1.0f - v2) - W * dv2) - dpdr * 0.5f * D * dv2 * is;
    }
    const float iW = 1.0f / W;
    f = W - p + 0.5f * B2 * (1.0f + v2) - 0.5f * S2 * iW * iW - tau;
    df = 1.0f - dp + 0.5f * B2 * dv2 + S2 * iW * iW * iW;
    return true;
}

// V from the converged W (with v^2 and p at W): v = (m + (S/W) B)/(W + B^2),
// rho = D sqrt(1 - v^2), B and psi as in U.  Returns the status bits.
__device__ __forceinline__ unsigned int sr_prim_tail(const double (&U)[NV], double W, double v2, double p, double S,
                                                     double B2, double D, bool conv, bool phys, double (&V)[NV])
{
    V[5] = U[5];
    V[6] = U[6];
    V[7] = U[7];
    V[8] = U[8];
    const double iWB = rcp64(W + B2), SW = S * rcp64(W);
    V[1] = (U[1] + SW * U[5]) * iWB;
    V[2] = (U[2] + SW * U[6]) * iWB;
    V[3] = (U[3] + SW * U[7]) * iWB;
    V[0] = phys ? D * ((1.0 - v2) * rsqrt64(1.0 - v2)) : D;
    V[4] = p;
    unsigned int st = 0;
    if (!conv) st |= ST_REC;
    if (!phys) st |= ST_SUPER;
    if (!(V[0] > 0.0) || !(p > 0.0)) st |= 1u;
    return st;
}

// V(U) in float64.  With a guess W0 > 0 (the W of a nearby state) plain
// Newton steps are tried first (at most 12); if one leaves the physical
// range or does not converge, and always without a guess, the bracketed
// iteration runs: [Wlo, Whi] with f(Whi) > 0 found by doubling from tau,
// Newton steps outside the bracket replaced by bisection.  Bounded: at most
// 64 doublings and 100 iterations.  Returns status bits (0, ST_REC for no
// convergence, ST_NEG / ST_SUPER).
__device__ __forceinline__ unsigned int sr_prim64(const double (&U)[NV], double gam, double (&V)[NV],
                                                  double W0 = 0.0)
{
    const double D = U[0], tau = U[4] + U[0];
    const double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    const double B2 = U[5] * U[5] + U[6] * U[6] + U[7] * U[7];
    const double S = U[1] * U[5] + U[2] * U[6] + U[3] * U[7];
    const double S2 = S * S;
    const double g1 = gam > 0.0 ? (gam - 1.0) * rcp64(gam) : 0.0;
    V[5] = U[5]; V[6] = U[6]; V[7] = U[7]; V[8] = U[8];
    if (!(D > 0.0) || !(tau > 0.0)) {
        V[0] = D; V[1] = V[2] = V[3] = 0.0; V[4] = 0.0;
        return 1u; // ST_NEG
    }
    double f = 0.0, df = 1.0, v2 = 0.0, p = 0.0;
    // without a nearby state, seed with W = tau - B^2/2 (exact at rest up
    // to p; within a few per cent for magnetised beams)
    if (!(W0 > 0.0)) W0 = tau - 0.5 * B2;
    double W = W0;
    bool conv = false;
    if (W0 > 0.0) {
        for (int it = 0; it < 12; ++it) {
            if (!sr_energy(W, D, m2, S2, B2, tau, g1, f, df, v2, p)) break;
            const double Wn = W - f * rcp64(df);
            if (!(Wn > 0.0)) break;
            if (fabs(Wn - W) <= 1.0e-15 * W) {
                W = Wn;
                conv = true;
                break;
            }
            W = Wn;
        }
    }
    double Wlo = 0.0, Whi = tau;
    if (!conv) {
        for (int k = 0; k < 64; ++k) {
            if (sr_energy(Whi, D, m2, S2, B2, tau, g1, f, df, v2, p) && f > 0.0) break;
            Wlo = Whi;
            Whi *= 2.0;
        }
        W = Whi;
    }
    for (int it = 0; it < 100 && !conv; ++it) {
        if (!sr_energy(W, D, m2, S2, B2, tau, g1, f, df, v2, p)) {
            Wlo = W;
            W = 0.5 * (Wlo + Whi);
            continue;
        }
        if (f > 0.0) Whi = W; else Wlo = W;
        double Wn = W - f * rcp64(df);
        if (!(Wn > Wlo && Wn < Whi)) Wn = 0.5 * (Wlo + Whi);
        if (fabs(Wn - W) <= 1.0e-15 * W) {
            W = Wn;
            conv = true;
            break;
        }
        W = Wn;
    }
    const bool phys = sr_energy(W, D, m2, S2, B2, tau, g1, f, df, v2, p);
    return sr_prim_tail(U, W, v2, p, S, B2, D, conv, phys, V);
}

// V(U) for the mixed path.  Newton steps in float32 from the guess W0 (else
// tau - B^2/2) bring W near float accuracy on the FP32 pipe; then float64
// Newton steps on the float64 energy equation follow (at most three), each
// squaring the relative error: once a step moves W by at most 1e-5 W the
// error left is of order 1e-10 relative, below the float32 rounding of the
// mixed path's fluxes.  v^2 and p are carried from that evaluation to the
// final W by their first-order Taylor terms (remainder of the order of the
// step squared).  A non-physical iterate, or no acceptance within the three
// steps, hands over to the bracketed float64 iteration of sr_prim64.  Float64
// inputs are rounded to float by integer operations (df_split).
__device__ __forceinline__ unsigned int sr_prim_mixed(const double (&U)[NV], double gam, double (&V)[NV],
                                                      double W0 = 0.0)
{
    const double D = U[0], tau = U[4] + U[0];
    const double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    const double B2 = U[5] * U[5] + U[6] * U[6] + U[7] * U[7];
    const double S = U[1] * U[5] + U[2] * U[6] + U[3] * U[7];
    const double S2 = S * S;
    const double g1 = gam > 0.0 ? (gam - 1.0) * rcp64(gam) : 0.0;
    if (!(D > 0.0) || !(tau > 0.0)) return sr_prim64(U, gam, V, W0);
    auto tof = [](double x) {
        const df h = df_split(x);
        return h.hi + h.lo;
    };
    const float Df = tof(D), tauf = tof(tau), m2f = tof(m2), B2f = tof(B2), S2f = tof(S2), g1f = tof(g1);
    if (!(W0 > 0.0)) W0 = tau - 0.5 * B2;
    if (!(W0 > 0.0)) return sr_prim64(U, gam, V, 0.0);
    float Wf = tof(W0);
    for (int it = 0; it < 12; ++it) {
        float f, dfw;
        if (!sr_energy_f(Wf, Df, m2f, S2f, B2f, tauf, g1f, f, dfw)) return sr_prim64(U, gam, V, W0);
        const float Wn = Wf - f / dfw;
        if (!(Wn > 0.0f)) return sr_prim64(U, gam, V, W0);
        const bool done = fabsf(Wn - Wf) <= 2.0e-6f * Wf;
        Wf = Wn;
        if (done) break;
    }
    double W = f2d_int(Wf);
    for (int it = 0; it < 3; ++it) {
        double f, dfw, v2, p, dv2, dp;
        if (!sr_energy_d(W, D, m2, S2, B2, tau, g1, f, dfw, v2, p, dv2, dp)) break;
        const double dW = -f * rcp64(dfw);
        const double Wn = W + dW;
        if (!(Wn > 0.0)) break;
        if (fabs(dW) <= 1.0e-5 * W) {
            v2 += dv2 * dW;
            p += dp * dW;
            if (!(v2 < 1.0)) break;
            return sr_prim_tail(U, Wn, v2, p, S, B2, D, true, true, V);
        }
        W = Wn;
    }
    return sr_prim64(U, gam, V, W);
}

// The recovery of the working precision: float64 throughout for R = double,
// the mixed recovery for R = float.
template <class R> __device__ __forceinline__ unsigned int sr_prim(const double (&U)[NV], double gam, double (&V)[NV],
                                                                   double W0 = 0.0)
{
    if constexpr (sizeof(R) == 4)
        return sr_prim_mixed(U, gam, V, W0);
    else
        return sr_prim64(U, gam, V, W0);
}

// Lower / upper signal speeds along the local normal (V[1] = v_n).
template <class R>
__device__ __forceinline__ void sr_speeds(const R (&V)[NV], R gam, R &lm, R &lp)
{
    const R vn = V[1];
    const R v2 = V[1] * V[1] + V[2] * V[2] + V[3] * V[3];
    const R B2 = V[5] * V[5] + V[6] * V[6] + V[7] * V[7];
    const R vB = V[1] * V[5] + V[2] * V[6] + V[3] * V[7];
    const R rh = sr_w<R>(V[0], V[4], gam);
    const R cs2 = sr_cs2<R>(V[4], rh, gam);
    const R b2 = B2 * (R(1) - v2) + vB * vB;
    const R ca2 = b2 * rcp_t<R>(rh + b2);
    const R a2 = cs2 + ca2 - cs2 * ca2;
    const R den = R(1) - v2 * a2;
    R disc = a2 * (R(1) - v2) * (R(1) - v2 * a2 - vn * vn * (R(1) - a2));
    disc = fmax(disc, R(0));
    const R sq = sqrt_t<R>(disc);
    const R id = rcp_t<R>(den);
    lm = (vn * (R(1) - a2) - sq) * id;
    lp = (vn * (R(1) - a2) + sq) * id;
}

// Physical RMHD flux along the local normal; the GLM pair (F[5], F[8]) =
// (psi, c_h^2 B_n).  U must be U(V).
template <class R>
__device__ __forceinline__ void sr_flux(const R (&V)[NV], const R (&U)[NV], R gam, R ch, R (&F)[NV])
{
    const R vx = V[1], vy = V[2], vz = V[3], p = V[4];
    const R bx = V[5], by = V[6], bz = V[7];
    const R v2 = vx * vx + vy * vy + vz * vz;
    const R W = sr_w<R>(V[0], p, gam) * rcp_t<R>(R(1) - v2);
    const R ex = -(vy * bz - vz * by), ey = -(vz * bx - vx * bz), ez = -(vx * by - vy * bx);
    const R pt = p + R(0.5) * (bx * bx + by * by + bz * bz + ex * ex + ey * ey + ez * ez);
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

// HLL flux with the exact linear (B_n, psi) face solve.
template <class R>
__device__ __forceinline__ void riemann_hll_sr(const R (&L0)[NV], const R (&R0)[NV], R gam, R ch, R (&F)[NV])
{
    R L[NV], Rt[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) { L[q] = L0[q]; Rt[q] = R0[q]; }
    const R Bm = R(0.5) * (L[5] + Rt[5]) - R(0.5) * (Rt[8] - L[8]) * rcp_t<R>(ch);
    const R pm = R(0.5) * (L[8] + Rt[8]) - R(0.5) * ch * (Rt[5] - L[5]);
    L[5] = Bm;
    Rt[5] = Bm;
    R UL[NV], UR[NV], FL[NV], FR[NV];
    sr_cons<R, R>(L, gam, UL);
    sr_cons<R, R>(Rt, gam, UR);
    sr_flux(L, UL, gam, ch, FL);
    sr_flux(Rt, UR, gam, ch, FR);
    R lmL, lpL, lmR, lpR;
    sr_speeds(L, gam, lmL, lpL);
    sr_speeds(Rt, gam, lmR, lpR);
    const R SL = fmin(lmL, lmR), SR = fmax(lpL, lpR);
    if (SL >= R(0)) {
#pragma unroll
        for (int q = 0; q < NV; ++q) F[q] = FL[q];
    } else if (SR <= R(0)) {
#pragma unroll
        for (int q = 0; q < NV; ++q) F[q] = FR[q];
    } else {
        const R is = rcp_t<R>(SR - SL);
#pragma unroll
        for (int q = 0; q < NV; ++q) F[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) * is;
    }
    F[5] = pm;
    F[8] = ch * ch * Bm;
}

// MUSCL-Hancock normal predictor of one cell (Section 3.3, beta = 1):
// vs = V_(i-1), V_i, V_(i+1) (local order, precision R), U0 = U_i^n (local,
// float64).  U* = U0 - dt/(2 dx) [F(V_+) - F(V_-)] and its recovery in
// float64; V*_(+/-) = V(U*) +/- dV/2.
template <class R>
__device__ __forceinline__ unsigned int sr_mh_predict(const R (&vm1)[NV], const R (&v0)[NV], const R (&vp1)[NV],
                                                      const double (&U0)[NV], R gam, R ch, R dtdx, double gamd,
                                                      R (&Vp)[NV], R (&Vm)[NV])
{
    R dV[NV], Vpl[NV], Vmi[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        dV[q] = mc_slope(v0[q] - vm1[q], vp1[q] - v0[q]);
        Vpl[q] = v0[q] + R(0.5) * dV[q];
        Vmi[q] = v0[q] - R(0.5) * dV[q];
    }
    R Up[NV], Um[NV], Fp[NV], Fm[NV];
    sr_cons<R, R>(Vpl, gam, Up);
    sr_cons<R, R>(Vmi, gam, Um);
    sr_flux(Vpl, Up, gam, ch, Fp);
    sr_flux(Vmi, Um, gam, ch, Fm);
    double Us[NV], Vs[NV];
    const R h = R(0.5) * dtdx;
#pragma unroll
    for (int q = 0; q < NV; ++q) Us[q] = U0[q] - (double)(h * (Fp[q] - Fm[q]));
    // Newton starts from the cell-centre W = w gamma^2 (U* is an O(dt) update of U_i)
    const double v2c = (double)v0[1] * v0[1] + (double)v0[2] * v0[2] + (double)v0[3] * v0[3];
    const double Wc = sr_w<double>((double)v0[0], (double)v0[4], gamd) * rcp64(1.0 - v2c);
    const unsigned int st = sr_prim<R>(Us, gamd, Vs, Wc);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        Vp[q] = (R)Vs[q] + R(0.5) * dV[q];
        Vm[q] = (R)Vs[q] - R(0.5) * dV[q];
    }
    return st;
}

} // namespace ctu
