// ctu_kernels.cuh -- kernels of the CTU step, templated on the working
// precision R of the tracing / Riemann stages.  Instantiated once for
// R = double (FP64 path) and once for R = float (mixed path) by
// ctu_f64.cu and ctu_f32.cu.
//
// One step (Section 3.1 of Mignone et al. 2012, Eq. update / ctu_flux /
// transv with Pi = 0) is the kernel sequence
//   k_prim       V = V(U) on every cell (pressure recovery in float64)
//   k_flux1<d>   first-order Godunov fluxes F^n_d = R(U_c, U_c+e_d)
//   k_trace<d>   normal predictor + transverse correction -> V^(n+1/2)_(+/-)
//   k_riemann<d> F^(n+1/2)_d = R(V_(c,+), V_(c+e_d,-))
//   k_update     U^(n+1) = U^n + dt sum_d (F_(d,-) - F_(d,+))/dx_d, psi damping
//   k_registers  flux-register windows, Eq. (fluxcorr)
// Intermediate arrays live in a library-owned scratch buffer with the same
// ghosted-patch layout as the pool (one region per patch).
#pragma once

#include "mhd_device.cuh"

namespace ctu {

constexpr int NG = 4;

struct DevPatch {
    int n[3];      // interior cells
    int N[3];      // ghosted extent
    int g[3];      // ghosts per side
    double dx[3];
    long long base;  // pool offset of the first ghosted cell
    long long soff;  // scratch offset of the first ghosted cell
};

struct DevWindow {
    int patch, dir, plane, a0, a1, b0, b1, pad;
    double weight;
    long long dst;
};

struct StepArgs {
    const DevPatch *patches;
    int npatch;
    int ndim;
    double gam;
    double glm_alpha;
    int upwind;
    const double *U;       // pool in
    double *Uout;          // pool out
    long long ustride;     // pool variable stride
    long long sstride;     // scratch variable stride
    const double *dtch;    // device {dt, c_h}
    unsigned int *status;  // sticky status bits
};

enum : unsigned int { ST_NEG = 1u, ST_NAN = 2u };

__device__ __forceinline__ long long cell_of(const DevPatch &P, int i, int j, int k)
{
    return ((long long)(k + P.g[2]) * P.N[1] + (j + P.g[1])) * P.N[0] + (i + P.g[0]);
}

__device__ __forceinline__ long long dstride(const DevPatch &P, int d)
{
    return d == 0 ? 1LL : (d == 1 ? (long long)P.N[0] : (long long)P.N[0] * P.N[1]);
}

// Box [lo, lo + ext) of cell coordinates; thread t -> (i, j, k), x fastest.
struct Box {
    int lo[3], ext[3];
    __device__ __forceinline__ long long size() const { return (long long)ext[0] * ext[1] * ext[2]; }
    __device__ __forceinline__ void coords(long long t, int &i, int &j, int &k) const
    {
        i = lo[0] + (int)(t % ext[0]);
        long long r = t / ext[0];
        j = lo[1] + (int)(r % ext[1]);
        k = lo[2] + (int)(r / ext[1]);
    }
};

// ---------------------------------------------------------------- conversions

__device__ __forceinline__ bool prim_from_cons64(const double (&U)[NV], double gam, double (&V)[NV])
{
    const double rho = U[0];
    const double ir = 1.0 / rho;
    const double vx = U[1] * ir, vy = U[2] * ir, vz = U[3] * ir;
    const double ke = 0.5 * (U[1] * vx + U[2] * vy + U[3] * vz);
    const double me = 0.5 * (U[5] * U[5] + U[6] * U[6] + U[7] * U[7]);
    const double p = (gam - 1.0) * (U[4] - ke - me);
    V[0] = rho; V[1] = vx; V[2] = vy; V[3] = vz; V[4] = p;
    V[5] = U[5]; V[6] = U[6]; V[7] = U[7]; V[8] = U[8];
    return rho > 0.0 && p > 0.0;
}

// igm = 1/(Gamma - 1)
template <class R>
__device__ __forceinline__ void cons64_from_prim(const R (&V)[NV], double igm, double (&U)[NV])
{
    const double rho = V[0], vx = V[1], vy = V[2], vz = V[3], p = V[4];
    const double bx = V[5], by = V[6], bz = V[7];
    U[0] = rho; U[1] = rho * vx; U[2] = rho * vy; U[3] = rho * vz;
    U[4] = p * igm + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz);
    U[5] = bx; U[6] = by; U[7] = bz; U[8] = V[8];
}

__device__ __forceinline__ unsigned int state_flags(double rho, double p)
{
    unsigned int f = 0;
    if (!(rho > 0.0) || !(p > 0.0)) f |= ST_NEG;
    if (!isfinite(rho) || !isfinite(p)) f |= ST_NAN;
    return f;
}

// ---------------------------------------------------------------- kernels

// V = V(U) on every ghosted cell of every patch; stores V in precision R.
template <class R>
__global__ void k_prim(StepArgs a, R *Vs)
{
    const DevPatch P = a.patches[blockIdx.y];
    const long long ncell = (long long)P.N[0] * P.N[1] * P.N[2];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        double U[NV], V[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) U[q] = a.U[q * a.ustride + P.base + c];
        bool ok = prim_from_cons64(U, a.gam, V);
        if (!ok) atomicOr(a.status, state_flags(V[0], V[4]));
#pragma unroll
        for (int q = 0; q < NV; ++q) Vs[q * a.sstride + P.soff + c] = (R)V[q];
    }
}

// First-order Godunov fluxes through the upper d-face of cells with
// c_d in [-1, n_d - 1] and the other active coordinates in [-1, n].
template <class R>
__global__ void k_flux1(StepArgs a, int d, const R *Vs, R *F1)
{
    const DevPatch P = a.patches[blockIdx.y];
    Box b;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if (e >= a.ndim) { b.lo[e] = 0; b.ext[e] = 1; }
        else if (e == d) { b.lo[e] = -1; b.ext[e] = P.n[e] + 1; }
        else { b.lo[e] = -1; b.ext[e] = P.n[e] + 2; }
    }
    const R gam = (R)a.gam, ch = (R)a.dtch[1];
    const long long st = dstride(P, d);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b.size();
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        b.coords(t, i, j, k);
        const long long c = P.soff + cell_of(P, i, j, k);
        R L[NV], Rr[NV], F[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            L[q] = Vs[perm(d, q) * a.sstride + c];
            Rr[q] = Vs[perm(d, q) * a.sstride + c + st];
        }
        riemann_hlld(L, Rr, gam, ch, F);
#pragma unroll
        for (int q = 0; q < NV; ++q) F1[perm(d, q) * a.sstride + c] = F[q];
    }
}

// Normal predictor along d plus the transverse correction (Eq. transv):
// cells with c_d in [-1, n_d], other active coordinates in [0, n-1].
// Writes the primitive n+1/2 interface states to Vp, Vm.
//
// IFACE64 = 1: U* = U(V*) and U^(n+1/2) = U* + dt/2 T formed in float64,
//   pressure recovered from U^(n+1/2) in float64 (the FP64 path, and the
//   mixed path's literal variant).
// IFACE64 = 0 (mixed path): the same state in increment form.  With
//   d = dt/2 T, rho = rho* + d_rho, m = rho* v* + d_m, B = B* + d_B,
//     p = p* + (Gamma-1) [ d_E + (rho* v*^2 d_rho - 2 rho* v*.d_m - d_m^2)/(2 rho)
//                          - d_B.(B* + d_B/2) ],
//   which equals (Gamma-1)(E - m^2/2rho - B^2/2) exactly but never forms E, so
//   no catastrophic cancellation occurs and float32 keeps the accuracy the
//   float32 transverse fluxes allow.
template <class R, int PPM, int IFACE64>
__global__ void k_trace(StepArgs a, int d, const R *Vs, const R *F1x, const R *F1y, const R *F1z,
                        R *Vp, R *Vm)
{
    const DevPatch P = a.patches[blockIdx.y];
    Box b;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if (e >= a.ndim) { b.lo[e] = 0; b.ext[e] = 1; }
        else if (e == d) { b.lo[e] = -1; b.ext[e] = P.n[e] + 2; }
        else { b.lo[e] = 0; b.ext[e] = P.n[e]; }
    }
    const double dt = a.dtch[0];
    const R gam = (R)a.gam, ch = (R)a.dtch[1];
    const R dtdx = (R)(dt / P.dx[d]);
    const long long st = dstride(P, d);
    // transverse directions in fixed order
    int t1 = -1, t2 = -1;
    for (int e = 0; e < a.ndim; ++e)
        if (e != d) { if (t1 < 0) t1 = e; else t2 = e; }
    const R *F1t1 = t1 == 0 ? F1x : (t1 == 1 ? F1y : F1z);
    const R *F1t2 = t2 == 0 ? F1x : (t2 == 1 ? F1y : F1z);
    const long long s1 = t1 >= 0 ? dstride(P, t1) : 0, s2 = t2 >= 0 ? dstride(P, t2) : 0;
    const double ih1 = t1 >= 0 ? 1.0 / P.dx[t1] : 0.0, ih2 = t2 >= 0 ? 1.0 / P.dx[t2] : 0.0;
    const double igm = 1.0 / (a.gam - 1.0);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b.size();
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        b.coords(t, i, j, k);
        const long long c = P.soff + cell_of(P, i, j, k);
        R vs[5][NV];
#pragma unroll
        for (int m = 0; m < 5; ++m)
#pragma unroll
            for (int q = 0; q < NV; ++q) vs[m][q] = Vs[perm(d, q) * a.sstride + c + (m - 2) * st];
        R Vpl[NV], Vml[NV];
        char_predict<R, PPM>(vs, gam, ch, dtdx, a.upwind != 0, Vpl, Vml);
        R Vpg[NV], Vmg[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { Vpg[perm(d, q)] = Vpl[q]; Vmg[perm(d, q)] = Vml[q]; }
        unsigned int fl = 0;
        if (IFACE64) {
            // transverse increments L^n_d' = (F_(d',-) - F_(d',+)) / dx_d'
            double T[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) T[q] = 0.0;
            if (t1 >= 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q)
                    T[q] += ((double)F1t1[q * a.sstride + c - s1] - (double)F1t1[q * a.sstride + c]) * ih1;
            }
            if (t2 >= 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q)
                    T[q] += ((double)F1t2[q * a.sstride + c - s2] - (double)F1t2[q * a.sstride + c]) * ih2;
            }
            double Ui[NV], Vi[NV];
            cons64_from_prim(Vpg, igm, Ui);
#pragma unroll
            for (int q = 0; q < NV; ++q) Ui[q] += 0.5 * dt * T[q];
            if (!prim_from_cons64(Ui, a.gam, Vi)) fl |= state_flags(Vi[0], Vi[4]);
#pragma unroll
            for (int q = 0; q < NV; ++q) Vp[q * a.sstride + c] = (R)Vi[q];
            cons64_from_prim(Vmg, igm, Ui);
#pragma unroll
            for (int q = 0; q < NV; ++q) Ui[q] += 0.5 * dt * T[q];
            if (!prim_from_cons64(Ui, a.gam, Vi)) fl |= state_flags(Vi[0], Vi[4]);
#pragma unroll
            for (int q = 0; q < NV; ++q) Vm[q * a.sstride + c] = (R)Vi[q];
        } else {
            // half-step transverse increments d = dt/2 T, in R
            R D[NV];
            const R h1 = (R)(0.5 * dt * ih1), h2 = (R)(0.5 * dt * ih2);
#pragma unroll
            for (int q = 0; q < NV; ++q) D[q] = R(0);
            if (t1 >= 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q) D[q] += (F1t1[q * a.sstride + c - s1] - F1t1[q * a.sstride + c]) * h1;
            }
            if (t2 >= 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q) D[q] += (F1t2[q * a.sstride + c - s2] - F1t2[q * a.sstride + c]) * h2;
            }
            const R gm1 = gam - R(1);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const R(&W)[NV] = side == 0 ? Vpg : Vmg;
                R *out = side == 0 ? Vp : Vm;
                const R rs = W[0];
                const R rho = rs + D[0];
                const R irho = R(1) / rho;
                const R m1 = rs * W[1] + D[1], m2 = rs * W[2] + D[2], m3 = rs * W[3] + D[3];
                const R v2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
                const R vdm = W[1] * D[1] + W[2] * D[2] + W[3] * D[3];
                const R dm2 = D[1] * D[1] + D[2] * D[2] + D[3] * D[3];
                const R dke = (rs * v2 * D[0] - R(2) * rs * vdm - dm2) * (R(0.5) * irho);
                const R dme = -(D[5] * (W[5] + R(0.5) * D[5]) + D[6] * (W[6] + R(0.5) * D[6]) +
                                D[7] * (W[7] + R(0.5) * D[7]));
                const R p = W[4] + gm1 * (D[4] + dke + dme);
                out[0 * a.sstride + c] = rho;
                out[1 * a.sstride + c] = m1 * irho;
                out[2 * a.sstride + c] = m2 * irho;
                out[3 * a.sstride + c] = m3 * irho;
                out[4 * a.sstride + c] = p;
                out[5 * a.sstride + c] = W[5] + D[5];
                out[6 * a.sstride + c] = W[6] + D[6];
                out[7 * a.sstride + c] = W[7] + D[7];
                out[8 * a.sstride + c] = W[8] + D[8];
                if (!(rho > R(0)) || !(p > R(0))) fl |= ST_NEG;
                if (!isfinite(rho) || !isfinite(p)) fl |= ST_NAN;
            }
        }
        if (fl) atomicOr(a.status, fl);
    }
}

// n+1/2 fluxes through the upper d-face of cells c_d in [-1, n_d - 1].
template <class R>
__global__ void k_riemann(StepArgs a, int d, const R *Vp, const R *Vm, R *Fd)
{
    const DevPatch P = a.patches[blockIdx.y];
    Box b;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if (e >= a.ndim) { b.lo[e] = 0; b.ext[e] = 1; }
        else if (e == d) { b.lo[e] = -1; b.ext[e] = P.n[e] + 1; }
        else { b.lo[e] = 0; b.ext[e] = P.n[e]; }
    }
    const R gam = (R)a.gam, ch = (R)a.dtch[1];
    const long long st = dstride(P, d);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b.size();
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        b.coords(t, i, j, k);
        const long long c = P.soff + cell_of(P, i, j, k);
        R L[NV], Rr[NV], F[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            L[q] = Vp[perm(d, q) * a.sstride + c];
            Rr[q] = Vm[perm(d, q) * a.sstride + c + st];
        }
        riemann_hlld(L, Rr, gam, ch, F);
#pragma unroll
        for (int q = 0; q < NV; ++q) Fd[perm(d, q) * a.sstride + c] = F[q];
    }
}

// U^(n+1) = U^n + dt (L_x + L_y + L_z) on interior cells, then the psi
// source -(c_h^2/c_p^2) psi integrated exactly (operator split).
template <class R>
__global__ void k_update(StepArgs a, const R *Fx, const R *Fy, const R *Fz)
{
    const DevPatch P = a.patches[blockIdx.y];
    Box b;
#pragma unroll
    for (int e = 0; e < 3; ++e) { b.lo[e] = 0; b.ext[e] = P.n[e]; }
    __shared__ double s_damp, s_idx[3];
    const double dt = a.dtch[0];
    if (threadIdx.x == 0) {
        double hmin = P.dx[0];
        for (int e = 1; e < a.ndim; ++e) hmin = fmin(hmin, P.dx[e]);
        s_damp = exp(-a.glm_alpha * a.dtch[1] * dt / hmin);
        for (int e = 0; e < 3; ++e) s_idx[e] = 1.0 / P.dx[e];
    }
    __syncthreads();
    const double damp = s_damp;
    const R *F[3] = {Fx, Fy, Fz};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b.size();
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        b.coords(t, i, j, k);
        const long long cl = cell_of(P, i, j, k);
        const long long c = P.soff + cl;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            // flux divergence in R (float64 on the FP64 path), accumulation in float64
            R s = R(0);
            for (int d = 0; d < a.ndim; ++d) {
                const long long st = dstride(P, d);
                s += (F[d][q * a.sstride + c - st] - F[d][q * a.sstride + c]) * (R)s_idx[d];
            }
            double u = a.U[q * a.ustride + P.base + cl] + dt * (double)s;
            if (q == 8) u *= damp;
            a.Uout[q * a.ustride + P.base + cl] = u;
        }
    }
}

// Flux-register windows, Eq. (fluxcorr): one thread per (window face, var).
template <class R>
__global__ void k_registers(StepArgs a, const DevWindow *win, int nwin, const R *Fx, const R *Fy,
                            const R *Fz, double *reg)
{
    const int w = blockIdx.y;
    if (w >= nwin) return;
    const DevWindow W = win[w];
    if (W.patch >= a.npatch) return;
    const DevPatch P = a.patches[W.patch];
    const int d = W.dir;
    const int ea = d == 0 ? 1 : 0, eb = d == 2 ? 1 : 2;
    const long long na = W.a1 - W.a0, nb = W.b1 - W.b0;
    const double area = P.dx[ea] * P.dx[eb];
    const double f = W.weight * a.dtch[0] * area;
    const R *F = d == 0 ? Fx : (d == 1 ? Fy : Fz);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < NV * na * nb;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / (na * nb));
        const long long r = t % (na * nb);
        int c3[3];
        c3[d] = W.plane - 1;
        c3[ea] = W.a0 + (int)(r % na);
        c3[eb] = W.b0 + (int)(r / na);
        const long long c = P.soff + cell_of(P, c3[0], c3[1], c3[2]);
        reg[W.dst + t] += f * (double)F[q * a.sstride + c];
    }
}

// Max over interior cells of max_d (|v_d| + c_f,d)/dx_d, as the bits of a
// positive double (monotone in the value) -> atomicMax.
template <class R>
__global__ void k_maxspeed(StepArgs a, unsigned long long *out)
{
    const DevPatch P = a.patches[blockIdx.y];
    Box b;
#pragma unroll
    for (int e = 0; e < 3; ++e) { b.lo[e] = 0; b.ext[e] = P.n[e]; }
    double m = 0.0;
    const double idx[3] = {1.0 / P.dx[0], 1.0 / P.dx[1], 1.0 / P.dx[2]};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < b.size();
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        b.coords(t, i, j, k);
        const long long cl = cell_of(P, i, j, k);
        double U[NV], V[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) U[q] = a.U[q * a.ustride + P.base + cl];
        if (!prim_from_cons64(U, a.gam, V)) atomicOr(a.status, state_flags(V[0], V[4]));
        const R rho = (R)V[0], p = (R)V[4], g = (R)a.gam;
        for (int d = 0; d < a.ndim; ++d) {
            const int qn = 1 + d, bn = 5 + d;
            const int b1 = 5 + (d == 0 ? 1 : 0), b2 = 5 + (d == 2 ? 1 : 2);
            const R cf = fast_speed(rho, p, (R)V[bn], (R)V[b1], (R)V[b2], g);
            const R sp = (fabs((R)V[qn]) + cf) * (R)idx[d];
            m = fmax(m, (double)sp);
        }
    }
    // warp + block reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = m;
    __syncthreads();
    if (wid == 0) {
        m = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
    }
}

} // namespace ctu
