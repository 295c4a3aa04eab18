// par_ops.cuh -- the parabolic terms of the CTU step (Section 3.1 with
// Pi != 0): thermal conduction, Pi_E = kappa_perp grad T + (kappa_par -
// kappa_perp) b (b . grad T) (the classical flux of Eq. tc_flux, T = p / rho,
// b the direction of the face's mean field), saturated on request as in the
// paper's appendix on the heat flux, isotropic viscosity (Eq. visc_tens, constant kinematic
// viscosity nu), tau = rho nu (grad v + grad v^T - (2/3) I div v) with the
// momentum flux Pi_m = tau and the energy flux Pi_E += v . tau, and
// resistivity (constant eta), -curl(eta J) = div(eta (grad B^T - grad B)):
// the flux of B_i along d is eta (dB_i/dx_d - dB_d/dx_i) and Pi_E gains
// B_f . that flux (the energy flux -eta J x B).
//
// Face values (the central differences of Section 3.1, g(U) at the mean of
// the two cells' states): at the face between c and c + e_d the normal
// derivative is (f(c + e_d) - f(c)) / dx_d, a transverse one (active t != d)
// the mean of the two cells' central differences,
//   [f(c + e_t) - f(c - e_t) + f(c + e_d + e_t) - f(c + e_d - e_t)] / (4 dx_t),
// rho_f the mean density, v_f = (rho v (c) + rho v (c + e_d)) /
// (rho(c) + rho(c + e_d)) and B_f the mean field; L_P = sum_d (Pi_(d,+) -
// Pi_(d,-)) / dx_d acts on the momentum, the energy and B.
//
// Kernels between the first-order stage and the sweeps:
//   k_par_faces    the face pass: every face flux of the ring box (from the
//                  primitive fields of U^n) or of the interior (from the
//                  half-step fields) once, stored per face
//   k_par_half     on the ring box (the interior and one layer around it):
//                  L_P^n from the primitive fields of U^n (the predictors of
//                  every direction add dt/2 L_P^n, Eq. transv: those along
//                  y and z through L1_x, which it adds L_P^n to), and the
//                  fields (T, rho, v, B) of the cell-centred U^(n+1/2) = U^n +
//                  dt/2 (sum_d L_(H,d)^n + L_P^n), L_(H,d)^n the first-order
//                  stage's divergences, which that stage forms on the whole
//                  ring box for these kernels
//   k_par_register the flux registers' momentum, energy and B take -dt A Pi
//                  of the half-step face fluxes (Eq. fluxcorr)
//   k_par_lp       L_P^(n+1/2) of the interior cells from those face fluxes
// The x sweep adds L_P^(n+1/2) to its update (U^(n+1) = U^n + dt
// (L_H^(n+1/2) + L_P^(n+1/2)), Eq. update), with the diffusion term in the
// CFL rate of the result.
// The n+1/2 fields are float64 (FP64 path) or double-float (mixed path: no
// FP64-pipe instruction).
// Each combination of the terms is a kernel of its own (template TM: bit 1
// viscosity, bit 2 resistivity); conduction alone forms and stores only the
// temperature.
#pragma once

#include "ctu_kernels.cuh"

namespace ctu {

// Planes of the half-step fields: T, then with viscosity or resistivity rho,
// v_x, v_y, v_z, B_x, B_y, B_z.  Field index f: 0 rho, 1..3 v, 4 T, 5..7 B
// (the order of the primitive state).  FP64 path: a double plane each.
// Mixed path: T as double-float pairs (float2, the first 8 bytes per
// scratch cell), the others as float planes after it (par_fplane; the face
// pass takes them in float, as coefficients of a small increment).
__host__ __device__ __forceinline__ int par_plane(int f) { return f == 4 ? 0 : (f < 4 ? f + 1 : f); }
// float offset, in units of the scratch stride, of field f != 4's plane
__host__ __device__ __forceinline__ int par_fplane(int f) { return 1 + par_plane(f); }

// kappa_perp, kappa_par - kappa_perp and phi in the working precision (the
// entries NPAR and par_gk, par_nu, par_eta are in ctu_kernels.cuh, where the
// x sweep's update uses them).
template <class R> __device__ __forceinline__ R par_kappa(const StepArgs &a);
template <> __device__ __forceinline__ double par_kappa<double>(const StepArgs &a) { return a.kappa; }
template <> __device__ __forceinline__ float par_kappa<float>(const StepArgs &a) { return a.kappaf; }
template <class R> __device__ __forceinline__ R par_dkappa(const StepArgs &a);
template <> __device__ __forceinline__ double par_dkappa<double>(const StepArgs &a) { return a.kpar - a.kappa; }
template <> __device__ __forceinline__ float par_dkappa<float>(const StepArgs &a) { return a.dkappaf; }
template <class R> __device__ __forceinline__ R par_phi(const StepArgs &a);
template <> __device__ __forceinline__ double par_phi<double>(const StepArgs &a) { return a.phi; }
template <> __device__ __forceinline__ float par_phi<float>(const StepArgs &a) { return a.phif; }

// Gradient of the fields f0 .. f0 + 2 at the face between c and cp = c + e_d:
// g[t][i] = d f_(f0 + i) / dx_t.
template <class R, class Dif>
__device__ __forceinline__ void par_grad(const StepArgs &a, const DevPatch &P, long long c, long long cp, int d,
                                         int f0, Dif dif, R (&g)[3][3])
{
    const R ih = pidx<R>(P, d);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        if (t == d) {
#pragma unroll
            for (int i = 0; i < 3; ++i) g[t][i] = dif(f0 + i, cp, c) * ih;
        } else if (t < a.ndim) {
            const long long s2 = dstr(P, t);
            const R q4 = R(0.25) * pidx<R>(P, t);
#pragma unroll
            for (int i = 0; i < 3; ++i) g[t][i] = (dif(f0 + i, c + s2, c - s2) + dif(f0 + i, cp + s2, cp - s2)) * q4;
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) g[t][i] = R(0);
        }
    }
}

// Parabolic fluxes through the face between scratch cells c and c + e_d
// (entries as NPAR).  get(f, i): field f of cell i; dif(f, i, j): field f of
// cell i minus that of cell j.  TM: the terms beyond isotropic conduction
// compiled in, bit 1 viscosity, bit 2 resistivity, bit 4 the full face
// gradient of T (anisotropic or saturated conduction).
template <class R, int TM, class Get, class Dif>
__device__ __forceinline__ void par_face(const StepArgs &a, const DevPatch &P, long long c, int d, Get get,
                                         Dif dif, R (&Pi)[NPAR])
{
    const long long st = dstr(P, d), cp = c + st;
    const R ih = pidx<R>(P, d);
#pragma unroll
    for (int q = 0; q < NPAR; ++q) Pi[q] = R(0);
    if constexpr ((TM & 4) == 0) {
        if (a.par_cond) Pi[3] = par_kappa<R>(a) * dif(4, cp, c) * ih;
    } else {
        // the full face gradient of T: anisotropic and/or saturated flux.
        // F = kappa_perp grad T + (kappa_par - kappa_perp) b (b . grad T), b
        // the direction of the face's mean field (none where it vanishes);
        // saturated: q F_d / (|F| + q), q = 5 phi p_u^(3/2) / sqrt(rho_f), p_u
        // the upwind pressure (the left cell's when F_d < 0)
        R gt[3], bf[3];
        R b2 = R(0), bg = R(0);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t == d) {
                gt[t] = dif(4, cp, c) * ih;
            } else if (t < a.ndim) {
                const long long s2 = dstr(P, t);
                gt[t] = (dif(4, c + s2, c - s2) + dif(4, cp + s2, cp - s2)) * (R(0.25) * pidx<R>(P, t));
            } else {
                gt[t] = R(0);
            }
            bf[t] = a.par_aniso ? R(0.5) * (get(5 + t, c) + get(5 + t, cp)) : R(0);
            b2 += bf[t] * bf[t];
            bg += bf[t] * gt[t];
        }
        const R kp = par_kappa<R>(a);
        const R ak = b2 > R(0) ? par_dkappa<R>(a) * bg / b2 : R(0);
        R F[3], f2 = R(0);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            F[t] = kp * gt[t] + ak * bf[t];
            f2 += F[t] * F[t];
        }
        if (a.par_sat) {
            const R r0 = get(0, c), r1 = get(0, cp);
            const R pu = F[d] < R(0) ? r0 * get(4, c) : r1 * get(4, cp);
            const R qs = R(5) * par_phi<R>(a) * pu * sqrt(pu) / sqrt(R(0.5) * (r0 + r1));
            Pi[3] = qs * F[d] / (sqrt(f2) + qs);
        } else {
            Pi[3] = F[d];
        }
    }
    if constexpr ((TM & 2) != 0) {
        R g[3][3];  // g[t][i] = dB_i / dx_t at the face
        par_grad<R>(a, P, c, cp, d, 5, dif, g);
        const R eta = par_eta<R>(a);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R f = eta * (g[d][i] - g[i][d]);
            Pi[4 + i] = f;
            Pi[3] += R(0.5) * (get(5 + i, c) + get(5 + i, cp)) * f;
        }
    }
    if constexpr ((TM & 1) != 0) {
        R g[3][3];  // g[t][i] = dv_i / dx_t at the face
        par_grad<R>(a, P, c, cp, d, 1, dif, g);
        const R div = g[0][0] + g[1][1] + g[2][2];
        const R r0 = get(0, c), r1 = get(0, cp);
        const R rnu = R(0.5) * (r0 + r1) * par_nu<R>(a);
        const R irs = R(1) / (r0 + r1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R tau = rnu * (g[d][i] + g[i][d] - (i == d ? R(2.0 / 3.0) * div : R(0)));
            const R vf = (r0 * get(1 + i, c) + r1 * get(1 + i, cp)) * irs;
            Pi[i] += tau;
            Pi[3] += vf * tau;
        }
    }
}

// Cells of the ring box (the interior and one layer around it on the active
// axes), x fastest: coordinates in [-1, n_d] on active axes, 0 on the others.
__host__ __device__ __forceinline__ int par_ring_cells(const int *n, int ndim)
{
    return (n[0] + 2) * (ndim > 1 ? n[1] + 2 : 1) * (ndim > 2 ? n[2] + 2 : 1);
}

// Planes along z each thread of the face passes and of k_par_half takes in
// turn (sharing its set-up), and the threads of a face pass (its box) and of
// k_par_half (the ring box) with the z extent in groups of PAR_ZR planes.
#ifndef CTU_PAR_ZR
#define CTU_PAR_ZR 4
#endif
constexpr int PAR_ZR = CTU_PAR_ZR;
__host__ __device__ __forceinline__ int par_face_threads(const int *n, int ndim, int half)
{
    const int w = half ? 3 : 1;
    const int e2 = ndim > 2 ? n[2] + w : 1;
    return (n[0] + w) * (ndim > 1 ? n[1] + w : 1) * ((e2 + PAR_ZR - 1) / PAR_ZR);
}
__host__ __device__ __forceinline__ int par_ring_threads(const int *n, int ndim)
{
    const int e2 = ndim > 2 ? n[2] + 2 : 1;
    return (n[0] + 2) * (ndim > 1 ? n[1] + 2 : 1) * ((e2 + PAR_ZR - 1) / PAR_ZR);
}

// Face pass: every face flux once.  For every cell c of the box [b, n - b]
// on the active axes (b = -1 with HALF, the faces of the ring box, for
// L_P^n; b = 0, the faces of the interior, for L_P^(n+1/2)), the flux
// through its lower face along each active d whose transverse coordinates
// lie in [b, n - 1 - b] is stored in PiF[(d NPAR + q) S + c] for the entries
// q the terms change; a thread takes PAR_ZR cells along z in turn.  HALF:
// fields of U^n from the primitive state V (T = p / rho); otherwise the
// half-step fields Wh (par_plane, par_fplane).
template <class R, int TM, int HALF>
__global__ void __launch_bounds__(BLOCK) k_par_faces(StepArgs a, GroupTable gt, const R *Vs, const double *Wh,
                                                     R *PiF)
{
    const Where w = locate(gt);
    const DevPatch P = a.patches[w.patch];
    const int t = w.b * BLOCK + threadIdx.x;
    if (t >= par_face_threads(P.n, a.ndim, HALF)) return;
    constexpr int bb = HALF ? -1 : 0;
    const int e0 = P.n[0] + 1 - 2 * bb, e1 = a.ndim > 1 ? P.n[1] + 1 - 2 * bb : 1;
    const int e2 = a.ndim > 2 ? P.n[2] + 1 - 2 * bb : 1;
    int x[3];
    x[0] = t % e0 + bb;
    x[1] = (t / e0) % e1 + (a.ndim > 1 ? bb : 0);
    const int z0 = (t / (e0 * e1)) * PAR_ZR;  // this thread's planes z0 .. z0 + PAR_ZR - 1 of the box
    const long long S = a.sstride;
    long long c = 0;
    auto on = [](int q) -> bool { return q == 3 || (q < 3 ? (TM & 1) != 0 : (TM & 2) != 0); };
    auto pass = [&](auto get, auto dif) {
#pragma unroll 1
        for (int r = 0; r < PAR_ZR && z0 + r < e2; ++r) {
            x[2] = z0 + r + (a.ndim > 2 ? bb : 0);
            c = P.soff + lcell(P, x[0], x[1], x[2]);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= a.ndim) continue;
                bool ok = true;
#pragma unroll
                for (int e = 0; e < 3; ++e)
                    if (e != d && e < a.ndim) ok &= x[e] <= P.n[e] - 1 - bb;
                if (!ok) continue;
                R Pi[NPAR];
                par_face<R, TM>(a, P, c - dstr(P, d), d, get, dif, Pi);
#pragma unroll
                for (int q = 0; q < NPAR; ++q)
                    if (on(q)) PiF[(long long)(d * NPAR + q) * S + c] = Pi[q];
            }
        }
    };
    if constexpr (HALF) {
        auto get = [&](int f, long long i) -> R { return f == 4 ? Vs[4 * S + i] / Vs[i] : Vs[f * S + i]; };
        pass(get, [&](int f, long long i, long long j) -> R { return get(f, i) - get(f, j); });
    } else if constexpr (sizeof(R) == 8) {
        pass([&](int f, long long n) -> double { return Wh[par_plane(f) * S + n]; },
             [&](int f, long long n1, long long n2) -> double {
                 return Wh[par_plane(f) * S + n1] - Wh[par_plane(f) * S + n2];
             });
    } else {
        // temperature differences of the double-float fields, exact to float;
        // those of v and B, coefficients of a small increment, in float
        const float2 *W2 = reinterpret_cast<const float2 *>(Wh);
        const float *Wf = reinterpret_cast<const float *>(Wh);
        pass([&](int f, long long n) -> float { return f == 4 ? W2[n].x : Wf[par_fplane(f) * S + n]; },
             [&](int f, long long n1, long long n2) -> float {
                 if (f == 4) {
                     const float2 u = W2[n1], v = W2[n2];
                     return df_add(df{u.x, u.y}, df{-v.x, -v.y}).hi;
                 }
                 return Wf[par_fplane(f) * S + n1] - Wf[par_fplane(f) * S + n2];
             });
    }
}

// L_P at scratch cell c from the face pass: sum_d (Pi(c + e_d, d) -
// Pi(c, d)) / dx_d in the order x, y, z, for the entries the terms TM change.
template <class R, int TM>
__device__ __forceinline__ void par_lp_faces(const StepArgs &a, const DevPatch &P, long long c, const R *PiF,
                                             R (&lp)[NPAR])
{
    const long long S = a.sstride;
#pragma unroll
    for (int q = 0; q < NPAR; ++q) lp[q] = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) continue;
        const long long st = dstr(P, d);
        const R ih = pidx<R>(P, d);
#pragma unroll
        for (int q = 0; q < NPAR; ++q) {
            const bool on = q == 3 || (q < 3 ? (TM & 1) != 0 : (TM & 2) != 0);
            if (!on) continue;
            const R *F = PiF + (long long)(d * NPAR + q) * S + c;
            lp[q] += (F[st] - F[0]) * ih;
        }
    }
}

// The half step at one ring-box cell (ghosted-box index cl), whose
// first-order divergences the first-order stage formed in every direction
// (its EXT range).  L1: the first-order divergences (global order), L1_x
// gains L_P^n in 2-D and 3-D; LP: L_P^n per scratch cell, 7 planes of R
// (momentum, energy, B); Wh: the half-step fields (par_plane, par_fplane).
// TM: bit 1 viscosity, bit 2 resistivity, bit 4 anisotropic or saturated
// conduction (which need the B and rho fields).
template <class R, int TM>
__device__ __forceinline__ void par_half_cell(const StepArgs &a, const DevPatch &P, int cl, R *L1, R *LP, double *Wh,
                                              const R *PiF)
{
    const long long S = a.sstride;
    const long long c = P.soff + cl;
    // L_P^n from the face pass over the primitive fields of U^n (T = p / rho)
    R lp[NPAR];
    par_lp_faces<R, TM>(a, P, c, PiF, lp);
    // the components each term changes: momentum (viscosity), energy, B
    // (resistivity)
    auto on = [](int q) -> bool { return q == 3 || (q < 3 ? (TM & 1) != 0 : (TM & 2) != 0); };
#pragma unroll
    for (int q = 0; q < NPAR; ++q)
        if (on(q)) LP[q * S + c] = lp[q];
    // the cell-centred half-step state and its fields.  dt/2 L_P^n reaches
    // the predictors of the sweeps along y and z (Eq. transv) through their
    // transverse terms, which both take L1_x: L1_x gains L_P^n (the x sweep
    // adds it from LP)
    R s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) continue;
        R *Ld = L1 + (long long)d * NV * S + c;
        R l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            l[q] = Ld[q * S];
            s[q] += l[q];
        }
        if (d == 0 && a.ndim > 1) {
#pragma unroll
            for (int q = 0; q < NPAR; ++q)
                if (on(q)) Ld[(1 + q) * S] = l[1 + q] + lp[q];
        }
    }
#pragma unroll
    for (int q = 0; q < NPAR; ++q)
        if (on(q)) s[1 + q] += lp[q];
    const long long gi = P.base + cl;
    if constexpr (sizeof(R) == 8) {
        const double hdt = 0.5 * a.sp->dt;
        double U[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) U[q] = a.U[q * a.ustride + gi] + hdt * s[q];
        const double rho = U[0];
        const double m2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
        const double b2 = U[5] * U[5] + U[6] * U[6] + U[7] * U[7];
        const double p = (a.gam - 1.0) * (U[4] - 0.5 * m2 / rho - 0.5 * b2);
        const unsigned int f = state_flags(rho, p);
        if (f) atomicOr(a.status, f);
        Wh[c] = p / rho;
        {
            if constexpr ((TM & 5) != 0) Wh[S + c] = rho;
            if constexpr ((TM & 1) != 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) Wh[(2 + q) * S + c] = U[1 + q] / rho;
            }
            if constexpr ((TM & 6) != 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) Wh[(5 + q) * S + c] = U[5 + q];
            }
        }
    } else {
        // double-float (no FP64-pipe instruction): U^(n+1/2) = U^n + (dt/2) s
        // with the product exact, then p, T = p / rho and v = m / rho to
        // ~2^-44; T stored as a float pair (hi, lo), the others rounded to
        // float
        const float hdt = 0.5f * a.sp->dtf;
        df U[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) U[q] = df_add(df_split(a.U[q * a.ustride + gi]), two_prod(hdt, s[q]));
        const df m2 = df_add(df_add(df_sqr(U[1]), df_sqr(U[2])), df_sqr(U[3]));
        const df b2 = df_add(df_add(df_sqr(U[5]), df_sqr(U[6])), df_sqr(U[7]));
        const df ke = df_scale(df_div(m2, U[0]), 0.5f);
        const df eint = df_add(df_add(U[4], df_neg(ke)), df_neg(df_scale(b2, 0.5f)));
        const df p = df_mul(eint, df{a.gm1f, a.gm1lo});
        const df T = df_div(p, U[0]);
        unsigned int f = 0;
        if (!(U[0].hi > 0.0f) || !(p.hi > 0.0f)) f |= ST_NEG;
        if (!isfinite(U[0].hi) || !isfinite(p.hi)) f |= ST_NAN;
        if (f) atomicOr(a.status, f);
        float2 *W2 = reinterpret_cast<float2 *>(Wh);
        float *Wf = reinterpret_cast<float *>(Wh);
        W2[c] = make_float2(T.hi, T.lo);
        {
            if constexpr ((TM & 5) != 0) Wf[par_fplane(0) * S + c] = U[0].hi;
            if constexpr ((TM & 1) != 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) Wf[par_fplane(1 + q) * S + c] = df_div(U[1 + q], U[0]).hi;
            }
            if constexpr ((TM & 6) != 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) Wf[par_fplane(5 + q) * S + c] = U[5 + q].hi;
            }
        }
    }
}

// k_par_half: the ring box (par_ring_cells), a thread PAR_ZR cells along z.
template <class R, int TM>
__global__ void __launch_bounds__(BLOCK) k_par_half(StepArgs a, GroupTable gt, R *L1, R *LP, double *Wh,
                                                    const R *PiF)
{
    const Where w = locate(gt);
    const DevPatch P = a.patches[w.patch];
    const int t = w.b * BLOCK + threadIdx.x;
    if (t >= par_ring_threads(P.n, a.ndim)) return;
    const int e0 = P.n[0] + 2, e1 = a.ndim > 1 ? P.n[1] + 2 : 1, e2 = a.ndim > 2 ? P.n[2] + 2 : 1;
    const int x0 = t % e0 - 1, x1 = (t / e0) % e1 - (a.ndim > 1 ? 1 : 0);
    const int z0 = (t / (e0 * e1)) * PAR_ZR;  // this thread's planes z0 .. z0 + PAR_ZR - 1 of the box
#pragma unroll 1
    for (int r = 0; r < PAR_ZR && z0 + r < e2; ++r)
        par_half_cell<R, TM>(a, P, lcell(P, x0, x1, z0 + r - (a.ndim > 2 ? 1 : 0)), L1, LP, Wh, PiF);
}

// L_P^(n+1/2) on the interior cells (the k_maxspeed tiling) from the face
// pass of the half-step fields, for the x sweep's update: LPh, NPAR planes
// of R, the entries the terms TM change.
template <class R, int TM>
__global__ void __launch_bounds__(BLOCK) k_par_lp(StepArgs a, GroupTable gt, const R *PiF, R *LPh)
{
    const Where wh = locate(gt);
    const DevPatch P = a.patches[wh.patch];
    const Tile t(wh.xw);
    const int T0 = (P.n[0] + t.xw - 1) / t.xw, T1 = (P.n[1] + t.rows - 1) / t.rows;
    const int b = wh.b;
    const int i = (b % T0) * t.xw + t.tx(), j = ((b / T0) % T1) * t.rows + t.ty(), k = b / (T0 * T1);
    if (i >= P.n[0] || j >= P.n[1] || k >= P.n[2]) return;
    const long long c = P.soff + lcell(P, i, j, k);
    R lp[NPAR];
    par_lp_faces<R, TM>(a, P, c, PiF, lp);
#pragma unroll
    for (int q = 0; q < NPAR; ++q) {
        const bool on = q == 3 || (q < 3 ? (TM & 1) != 0 : (TM & 2) != 0);
        if (on) LPh[q * a.sstride + c] = lp[q];
    }
}

// Flux registers of the parabolic fluxes (Eq. fluxcorr with the flux F -
// Pi): the momentum, energy and B of every window's faces gain -dt A
// Pi^(n+1/2), Pi from the face pass of the half-step fields (PiF, the lower
// face of the cell on the window's plane).  Block (w, y) takes window w's
// faces y BLOCK + t, y BLOCK + t + gridDim.y BLOCK, ... within the patch
// (as the sweeps' register_face, which skips the window's faces beyond it).
template <class R, int TM>
__global__ void __launch_bounds__(BLOCK) k_par_register(StepArgs a, const R *PiF)
{
    const DevWindow W = a.win[blockIdx.x];
    const DevPatch P = a.patches[W.patch];
    const int D = W.dir;
    // the transverse dimensions ea < eb: (1, 2), (0, 2) or (0, 1)
    const int na = W.a1 - W.a0, nb = W.b1 - W.b0;
    const int fa = min(W.a1, D == 0 ? P.n[1] : P.n[0]) - W.a0;  // faces within the patch
    const int fb = min(W.b1, D == 2 ? P.n[1] : P.n[2]) - W.b0;
    if (fa <= 0 || fb <= 0) return;
    // the face area: the cell widths along the two transverse dimensions
    const double f = W.weight * a.sp->dt * (D == 0 ? P.dx[1] : P.dx[0]) * (D == 2 ? P.dx[1] : P.dx[2]);
    const long long S = a.sstride;
    for (int t = blockIdx.y * BLOCK + threadIdx.x; t < fa * fb; t += gridDim.y * BLOCK) {
        const int ja = t % fa, jb = t / fa;
        const int ca = W.a0 + ja, cb = W.b0 + jb;  // transverse coordinates, increasing dimension order
        const int x0 = D == 0 ? W.plane : ca, x1 = D == 1 ? W.plane : (D == 0 ? ca : cb), x2 = D == 2 ? W.plane : cb;
        const long long c = P.soff + lcell(P, x0, x1, x2);
        const long long o = W.dst + (long long)jb * na + ja;
#pragma unroll
        for (int q = 0; q < NPAR; ++q) {
            const bool on = q == 3 || (q < 3 ? (TM & 1) != 0 : (TM & 2) != 0);
            if (on) a.reg[o + (long long)(1 + q) * nb * na] += f * widen<R>(-PiF[(long long)(D * NPAR + q) * S + c]);
        }
    }
}

} // namespace ctu
