// tc_ops.cuh -- thermal conduction, the parabolic term of the CTU step
// (Section 3.1 with Pi != 0).  Classical isotropic heat flux (Eq. tc_flux
// with q -> infinity, kappa_par = kappa_perp = kappa): Pi_E = kappa grad T,
// T = p / rho, with the central-difference face values
//   Pi_(d,+) = kappa (T(c + e_d) - T(c)) / dx_d
// and L_P = sum_d (Pi_(d,+) - Pi_(d,-)) / dx_d on the energy.
//
// Two kernels around the hyperbolic step:
//   k_tc_half    after the first-order stage, on the ring box (the interior
//                and one layer around it): L_P^n from T^n (the predictors of
//                every direction add dt/2 L_P^n, Eq. transv), and T^(n+1/2) of
//                the cell-centred U^(n+1/2) = U^n + dt/2 (sum_d L_(H,d)^n +
//                L_P^n).  L_(H,d)^n is the first-order stage's divergence
//                where that stage formed it (c_d inside the patch) and is
//                solved here, with the same solver, on the ring's outer layer
//   k_tc_update  U^(n+1) += dt L_P^(n+1/2) on the interior (Eq. update), and
//                on request the CFL rate of the result (with the diffusion
//                term), in place of the fused reduction of the last sweep
// T^(n+1/2) and the update are float64 (FP64 path) or double-float with a
// float64 energy update (mixed path; no FP64-pipe instruction but the one
// update FMA).
#pragma once

#include "ctu_kernels.cuh"

namespace ctu {

// Adds (F(c - e_D/2) - F(c + e_D/2)) / dx_D at scratch cell c to s (global
// order), F from the cell-centred primitive states as in k_div1.
template <class R, int D>
__device__ __forceinline__ void tc_div1(const StepArgs &a, const DevPatch &P, const R *Vs, long long c, R gam,
                                        R ch, R (&s)[NV])
{
    const long long st = dstr(P, D);
    R Vm[NV], V0[NV], Vp[NV], Fm[NV], Fp[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        Vm[q] = Vs[gperm<D>(q) * a.sstride + c - st];
        V0[q] = Vs[gperm<D>(q) * a.sstride + c];
        Vp[q] = Vs[gperm<D>(q) * a.sstride + c + st];
    }
    riemann_any<PH_MHD, R>(Vm, V0, gam, ch, Fm);
    riemann_any<PH_MHD, R>(V0, Vp, gam, ch, Fp);
    const R iD = pidx<R>(P, D);
#pragma unroll
    for (int q = 0; q < NV; ++q) s[gperm<D>(q)] += (Fm[q] - Fp[q]) * iD;
}

// (Gamma - 1) kappa in the working precision.
template <class R> __device__ __forceinline__ R tc_gk(const StepArgs &a);
template <> __device__ __forceinline__ double tc_gk<double>(const StepArgs &a) { return (a.gam - 1.0) * a.kappa; }
template <> __device__ __forceinline__ float tc_gk<float>(const StepArgs &a) { return a.gm1f * a.kappaf; }

// L1: the first-order divergences (global order, ndim > 1); LP: L_P^n per
// scratch cell (R); Th: T^(n+1/2) per scratch cell, a double (FP64 path) or
// the double-float pair (hi, lo) (mixed path).
// Cells of the ring box outside the interior (its outer layer), enumerated
// compactly: the two x-faces (x = -1, n_x; y, z over the ring), the two
// y-faces (x inside; z over the ring), the two z-faces (x, y inside); in 1-D
// the whole ring box (the first-order stage does not run).
__host__ __device__ __forceinline__ int tc_shell_cells(const int *n, int ndim)
{
    if (ndim == 1) return n[0] + 2;
    const int e1 = n[1] + 2, e2 = ndim > 2 ? n[2] + 2 : 1;
    return 2 * e1 * e2 + 2 * n[0] * e2 + (ndim > 2 ? 2 * n[0] * n[1] : 0);
}

__device__ __forceinline__ void tc_shell_coords(const DevPatch &P, int ndim, int t, int (&x)[3])
{
    if (ndim == 1) {
        x[0] = t - 1;
        x[1] = x[2] = 0;
        return;
    }
    const int e1 = P.n[1] + 2, e2 = ndim > 2 ? P.n[2] + 2 : 1, lo2 = ndim > 2 ? 1 : 0;
    const int cx = 2 * e1 * e2, cy = 2 * P.n[0] * e2;
    if (t < cx) {
        const int side = t / (e1 * e2), r = t - side * e1 * e2;
        x[0] = side ? P.n[0] : -1;
        x[1] = r % e1 - 1;
        x[2] = r / e1 - lo2;
    } else if (t < cx + cy) {
        t -= cx;
        const int side = t / (P.n[0] * e2), r = t - side * P.n[0] * e2;
        x[0] = r % P.n[0];
        x[1] = side ? P.n[1] : -1;
        x[2] = r / P.n[0] - lo2;
    } else {
        t -= cx + cy;
        const int side = t / (P.n[0] * P.n[1]), r = t - side * P.n[0] * P.n[1];
        x[0] = r % P.n[0];
        x[1] = r / P.n[0];
        x[2] = side ? P.n[2] : -1;
    }
}

// SHELL = false: the interior cells (ndim > 1), whose first-order
// divergences the first-order stage formed in every direction, one thread
// per cell in the k_maxspeed tiling; SHELL = true: the ring's outer layer
// (tc_shell_cells), which solves the missing faces itself.  The split keeps
// the Riemann solver, and its registers, out of the kernel that covers
// almost all cells.
template <class R, bool SHELL>
__global__ void __launch_bounds__(BLOCK) k_tc_half(StepArgs a, GroupTable gt, const R *Vs, const R *L1, R *LP,
                                                   double *Th)
{
    const Where w = locate(gt);
    const DevPatch P = a.patches[w.patch];
    int x[3];
    if constexpr (SHELL) {
        const int t = w.b * BLOCK + threadIdx.x;
        if (t >= tc_shell_cells(P.n, a.ndim)) return;
        tc_shell_coords(P, a.ndim, t, x);
    } else {
        const Tile tl(w.xw);
        const int T0 = (P.n[0] + tl.xw - 1) / tl.xw, T1 = (P.n[1] + tl.rows - 1) / tl.rows;
        x[0] = (w.b % T0) * tl.xw + tl.tx();
        x[1] = ((w.b / T0) % T1) * tl.rows + tl.ty();
        x[2] = w.b / (T0 * T1);
        if (x[0] >= P.n[0] || x[1] >= P.n[1] || x[2] >= P.n[2]) return;
    }
    const int cl = lcell(P, x[0], x[1], x[2]);
    const long long S = a.sstride;
    const long long c = P.soff + cl;
    // L_P^n from T^n = p^n / rho^n
    const R kap = (R)a.kappa;
    const R T0 = Vs[4 * S + c] / Vs[c];
    R lp = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) continue;
        const long long st = dstr(P, d);
        const R ih = pidx<R>(P, d);
        const R Tp = Vs[4 * S + c + st] / Vs[c + st];
        const R Tm = Vs[4 * S + c - st] / Vs[c - st];
        lp += (kap * (Tp - T0) * ih - kap * (T0 - Tm) * ih) * ih;
    }
    LP[c] = lp;
    // the cell-centred half-step state and its temperature
    const R gam = pgam<R>(a), ch = pch<R>(a.sp);
    R s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) continue;
        if (!SHELL || (a.ndim > 1 && x[d] >= 0 && x[d] < P.n[d])) {  // formed by the first-order stage
            const R *Ld = L1 + (long long)d * NV * S + c;
#pragma unroll
            for (int q = 0; q < 8; ++q) s[q] += Ld[q * S];
        } else if constexpr (SHELL) {
            if (d == 0)
                tc_div1<R, 0>(a, P, Vs, c, gam, ch, s);
            else if (d == 1)
                tc_div1<R, 1>(a, P, Vs, c, gam, ch, s);
            else
                tc_div1<R, 2>(a, P, Vs, c, gam, ch, s);
        }
    }
    s[4] += lp;
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
        Th[c] = p / rho;
    } else {
        // double-float (no FP64-pipe instruction): U^(n+1/2) = U^n + (dt/2) s
        // with the product exact, then p and T = p / rho to ~2^-44; stored
        // as the float pair (hi, lo)
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
        reinterpret_cast<float2 *>(Th)[c] = make_float2(T.hi, T.lo);
    }
}

// Flux-register windows of the face of plane `plane` normal to D (transverse
// coordinates ca, cb in increasing dimension order): the energy flux through
// it gains -Pi^(n+1/2) (Eq. fluxcorr with the parabolic flux).
template <class R, int D>
__device__ __forceinline__ void tc_register(const StepArgs &a, const DevPatch &P, int patch, int plane, int ca,
                                            int cb, R pi, double dt)
{
    const int B = window_base(a, patch, D);
    if (B < 0) return;
    const int w0 = window_first(a, B, plane), w1 = window_first(a, B, plane + 1);
    if (w1 > w0) register_face_var<R, D>(a, P, w0, w1, ca, cb, 4, -pi, dt);
}

template <class R>
__device__ __forceinline__ void tc_register_d(const StepArgs &a, const DevPatch &P, int patch, int d, int plane,
                                              const int (&x)[3], R pi, double dt)
{
    if (d == 0)
        tc_register<R, 0>(a, P, patch, plane, x[1], x[2], pi, dt);
    else if (d == 1)
        tc_register<R, 1>(a, P, patch, plane, x[0], x[2], pi, dt);
    else
        tc_register<R, 2>(a, P, patch, plane, x[0], x[1], pi, dt);
}

// U_out's energy += dt L_P^(n+1/2) on the interior cells (the k_maxspeed
// tiling); the flux registers of the cell's lower faces (and of its upper
// faces on the patch's last plane) gain -dt Pi; with next != null also the
// CFL rate of the updated cell, Eq. (Ca) with the diffusion term, folded
// into *next.
template <int PHYS, class R>
__global__ void __launch_bounds__(BLOCK) k_tc_update(StepArgs a, GroupTable gt, const double *Th,
                                                     unsigned long long *next)
{
    const Where wh = locate(gt);
    const DevPatch P = a.patches[wh.patch];
    const Tile t(wh.xw);
    const int T0 = (P.n[0] + t.xw - 1) / t.xw, T1 = (P.n[1] + t.rows - 1) / t.rows;
    const int b = wh.b;
    const int i = (b % T0) * t.xw + t.tx(), j = ((b / T0) % T1) * t.rows + t.ty(), k = b / (T0 * T1);
    R m = R(0);
    if (i < P.n[0] && j < P.n[1] && k < P.n[2]) {
        const int cl = lcell(P, i, j, k);
        const long long c = P.soff + cl;
        double *Uo = a.Uout + P.base + cl;
        double E;
        const int x[3] = {i, j, k};
        if constexpr (sizeof(R) == 8) {
            const double Tc = Th[c];
            double lp = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= a.ndim) continue;
                const long long st = dstr(P, d);
                const double up = Th[c + st] - Tc, dn = Tc - Th[c - st];
                const double kd = a.kappa * (P.idx[d] * P.idx[d]);
                lp = fma(up - dn, kd, lp);
                if (a.reg) {
                    const double kh = a.kappa * P.idx[d];
                    tc_register_d<double>(a, P, wh.patch, d, x[d], x, kh * dn, a.sp->dt);
                    if (x[d] == P.n[d] - 1) tc_register_d<double>(a, P, wh.patch, d, x[d] + 1, x, kh * up, a.sp->dt);
                }
            }
            E = fma(a.sp->dt, lp, Uo[4 * a.ustride]);
        } else {
            // differences of the double-float temperatures, exact to float
            const float2 *Tf = reinterpret_cast<const float2 *>(Th);
            const float2 t0 = Tf[c];
            const df Tc{t0.x, t0.y};
            float lp = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= a.ndim) continue;
                const long long st = dstr(P, d);
                const float2 tp = Tf[c + st], tm = Tf[c - st];
                const float up = df_add(df{tp.x, tp.y}, df_neg(Tc)).hi;
                const float dn = df_add(Tc, df_neg(df{tm.x, tm.y})).hi;
                lp = fmaf(up - dn, a.kappaf * (P.idxf[d] * P.idxf[d]), lp);
                if (a.reg) {
                    const float kh = a.kappaf * P.idxf[d];
                    tc_register_d<float>(a, P, wh.patch, d, x[d], x, kh * dn, a.sp->dt);
                    if (x[d] == P.n[d] - 1) tc_register_d<float>(a, P, wh.patch, d, x[d] + 1, x, kh * up, a.sp->dt);
                }
            }
            E = fma(a.sp->dt, f2d_int(lp), Uo[4 * a.ustride]);
        }
        Uo[4 * a.ustride] = E;
        if (next) {
            double U[NV];
            R V[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) U[q] = q == 4 ? E : Uo[q * a.ustride];
            const unsigned int f = prim_any<PHYS, R>(U, a, V);
            if (f) atomicOr(a.status, f);
            m = cell_speed<PHYS, R>(V, a, P);
            const R D = tc_gk<R>(a) / V[0];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (d < a.ndim) m += R(2) * D * (pidx<R>(P, d) * pidx<R>(P, d));
        }
    }
    if (next) block_max_to<R>(m, next);
}

} // namespace ctu
