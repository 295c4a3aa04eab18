// ctu_kernels.cuh -- kernels of the CTU step, templated on the working
// precision R of the tracing / Riemann stages (double: FP64 path; float:
// mixed path) and on the sweep direction D.
//
// One step (Section 3.1 of Mignone et al. 2012, Eq. update / ctu_flux /
// transv with Pi = 0) is the kernel sequence
//   k_setup        {dt, c_h} -> per-step parameters (float copies)
//   k_prim         V = V(U) on every ghosted cell
//   k_div1<D>      first-order Godunov fluxes F^n_D = R(U_c, U_c+e_D) and
//                  their divergences L1_D (the transverse terms)
//   k_sweep_x      direction x: normal predictor + transverse correction,
//                  n+1/2 Riemann problems and L_x, one thread per traced cell
//                  of several rows in turn, interface states exchanged
//                  through shared memory
//   k_sweep_m<D>   directions y, z: the same, one thread per pencil segment
//                  marching along D with the 5-cell stencil in registers
// The last sweep of the step adds U^n + dt (L_x + L_y + L_z), applies the
// psi source and, on request, reduces the next step's CFL speed; every sweep
// accumulates the flux-register windows of its faces (Eq. fluxcorr).
//
// Scratch (library-owned, per-patch regions with the ghosted layout): V (9
// words per cell), the first-order divergences L1 (3 x 9), and the running
// sum A = L_x (+ L_y) (9), all in R.  Interface states and n+1/2 fluxes never leave the chip.
//
// Mixed path and the FP64 pipe: besides the float64 update accumulation
// (one DFMA per variable and cell) the mixed kernels issue no FP64
// instruction on the common path -- float64 inputs are split and widened
// with integer operations and the cell-centre pressure is recovered in
// double-float arithmetic (df.cuh); per-step parameters arrive as floats.
#pragma once

#include "df.cuh"
#include "mhd_device.cuh"
#include "srmhd_device.cuh"

namespace ctu {

// Physics of a kernel instance: ideal MHD (characteristic tracing, HLLD) or
// special-relativistic MHD (MUSCL-Hancock, HLL, float64 Newton recovery).
enum { PH_MHD = 0, PH_SR = 1 };

struct DevPatch {
    int n[3];        // interior cells
    int N[3];        // ghosted extent
    int g[3];        // ghosts per side (4 active, 0 inactive)
    float idxf[3];   // 1/dx in float
    double dx[3];
    double idx[3];   // 1/dx
    double hmin;     // min dx over active dimensions
    long long base;  // pool offset of the first ghosted cell
    long long soff;  // scratch offset of the first ghosted cell
};

struct DevWindow {
    int patch, dir, plane, a0, a1, b0, b1, pad;
    double weight;
    long long dst;
};

struct StepParams {
    double dt, ch;
    float dtf, chf;
};

struct StepArgs {
    const DevPatch *patches;
    int npatch;
    int ndim;
    double gam;
    double igm;            // 1/(Gamma-1)
    float gamf, gm1f;      // Gamma, Gamma-1 in float
    double glm_alpha;
    int upwind;            // tracing mode (CTU_TRACE_*); 2 and 3 only in the reference-state kernels
    int limiter;           // linear reconstruction's slope (CTU_LINEAR_*), RECON_LIN kernels
    // hybrid integration (shock flags): per scratch cell, bit 1 shocked (HLL
    // at its faces), bit 2 MinMod reconstruction; null when off
    unsigned char *flags;
    double shock_eps;
    int shock_q;           // 0 thermal, 1 magnetic pressure
    // parabolic terms (the RECON_*_PAR kernels): conductivities kappa and
    // kpar (along the field), kinematic viscosity nu and resistivity eta
    // (par_cond, par_visc, par_res, par_aniso: nonzero when on), L_P^n per
    // scratch cell (7 planes of the
    // working precision: momentum, energy, B) and the half-step fields
    // (planes of 8 bytes: T, then rho, v and B with viscosity or resistivity)
    double kappa, kpar, nu, eta;  // kappa: across the field (all directions when isotropic)
    double phi;                   // saturation parameter of the heat flux (par_sat)
    float phif;
    float kappaf, nuf, etaf;      // kappa, nu, eta in float
    float dkappaf, kmaxf;         // kpar - kappa, max(kappa, kpar) in float
    float gm1lo;                  // (Gamma-1) - gm1f in float: Gamma-1 as a double-float pair
    int par_cond, par_visc, par_res, par_aniso, par_sat;
    const void *lp;
    double *th;
    void *pif;             // face fluxes of the parabolic face pass (3 x NPAR planes of R)
    void *lph;             // L_P^(n+1/2) per scratch cell (NPAR planes of R)
    const double *U;       // pool in
    double *Uout;          // pool out
    long long ustride;     // pool variable stride
    long long sstride;     // scratch variable stride
    const double *dtch;    // device {dt, c_h}
    const StepParams *sp;  // device per-step parameters (written by k_setup)
    unsigned int *status;  // sticky status bits
    // flux registers: windows sorted by (patch, dir, plane); for patch*3+dir,
    // wbase[] is -1 or an offset B into wpos[] such that the windows on plane
    // pl are win[wpos[B + pl] .. wpos[B + pl + 1])
    const DevWindow *win;
    int nwin;              // windows in win (0 without registers)
    int wfaces;            // most faces of one window within its patch
    const int *wbase;
    const int *wpos;
    double *reg;
    unsigned long long *nextmax;  // nullable: max CFL speed of U^(n+1)
};

enum : unsigned int { ST_NEG = 1u, ST_NAN = 2u };

constexpr int BLOCK = 128;
#ifndef CTU_SEG
#define CTU_SEG 16
#endif
#ifndef CTU_MARCH_MINB
#define CTU_MARCH_MINB 3
#endif
#ifndef CTU_SWEEPX_MINB
#define CTU_SWEEPX_MINB 6
#endif
#ifndef CTU_SWEEPX_MINB_PAR
#define CTU_SWEEPX_MINB_PAR 5
#endif
#ifndef CTU_DIV1X_ROWS
#define CTU_DIV1X_ROWS 16
#endif
#ifndef CTU_SWEEPX_ROWS
#define CTU_SWEEPX_ROWS 16
#endif
#ifndef CTU_PRIM_CELLS
#define CTU_PRIM_CELLS 4
#endif
// cells each thread of k_prim takes in turn, BLOCK apart
constexpr int PRIM_CELLS = CTU_PRIM_CELLS;
// Rows each thread of the first-order x stage and of the x sweep takes in
// turn, so that the per-thread set-up (tile decode, patch and window look-up,
// the block reductions) is shared: up to `most` (per launch: the most that
// still leaves the launch enough blocks, launch_rows), and within that the x
// that minimises the patch's row slots ceil(nrows / (tile_rows x))
// tile_rows x weighted by (1 + 1/(8 x)), the set-up measured at about an
// eighth of a cell's work, so that small patches are not padded with idle
// rows (the larger x on a tie).  Chosen on the host per patch group; the
// kernels read it from the group table.
constexpr int DIV1X_ROWS = CTU_DIV1X_ROWS, SWEEPX_ROWS = CTU_SWEEPX_ROWS;
inline int rows_per_thread(int most, int nrows, int tile_rows)
{
    int best = 1;
    long long bc = -1;
    for (int x = 1; x <= most; ++x) {
        const long long rr = (long long)tile_rows * x;
        const long long slots = (nrows + rr - 1) / rr * rr;
        const long long cost = slots * (8 * x + 1) * (840 / x);  // slots (1 + 1/(8x)), times 8 * 840
        if (bc < 0 || cost <= bc) {
            bc = cost;
            best = x;
        }
    }
    return best;
}
constexpr int SEG = CTU_SEG;  // default cells per marching segment

// One launch covers every patch group of a batch (up to MAXG groups): block
// blockIdx.x belongs to the group g with start[g] <= blockIdx.x < start[g+1]
// and to its patch first[g] + (blockIdx.x - start[g]) / bpp[g].  Each group
// carries its own thread-tile width along x and marching segment length
// (chosen per patch shape, e.g. by the autotuner).  The table travels in the
// kernel parameters (constant bank); the block scheduler drains the blocks,
// largest patches first.
constexpr int MAXG = 16;
struct GroupTable {
    int n;
    int start[MAXG + 1];
    int first[MAXG];
    int bpp[MAXG];
    unsigned bm[MAXG];       // division by bpp: multiplier and shifts (divmagic)
    unsigned char bs1[MAXG], bs2[MAXG];
    int xw[MAXG];
    int seg[MAXG];
    unsigned char xr[MAXG];  // rows per thread of the x-tiled kernels that take several (rows_per_thread)
};

// Division of 0 <= x < 2^32 by an invariant divisor d >= 1 with one high
// multiply, two shifts and two adds (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Fig. 4.1):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, s1 = min(l, 1),
// s2 = max(l - 1, 0); x / d = (t + ((x - t) >> s1)) >> s2 with t = mulhi(m, x).
struct DivMagic {
    unsigned m;
    unsigned char s1, s2;
};
inline DivMagic divmagic(unsigned d)
{
    int l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    DivMagic r;
    r.m = (unsigned)((((1ull << l) - d) << 32) / d + 1);
    r.s1 = (unsigned char)(l < 1 ? l : 1);
    r.s2 = (unsigned char)(l > 1 ? l - 1 : 0);
    return r;
}

struct Where {
    int patch, b, xw, seg, xr;
};

__device__ __forceinline__ Where locate(const GroupTable &gt)
{
    const int bx = (int)blockIdx.x;
    int g = 0;
#pragma unroll 1
    while (g + 1 < gt.n && bx >= gt.start[g + 1]) ++g;
    const unsigned rel = (unsigned)(bx - gt.start[g]);
    const unsigned t = __umulhi(gt.bm[g], rel);
    const int q = (int)((t + ((rel - t) >> gt.bs1[g])) >> gt.bs2[g]);  // rel / bpp
    Where w;
    w.patch = gt.first[g] + q;
    w.b = (int)rel - q * gt.bpp[g];
    w.xw = gt.xw[g];
    w.seg = gt.seg[g];
    w.xr = gt.xr[g];
    return w;
}
// The marching sweeps are latency bound: they are compiled for at least
// CTU_MARCH_MINB resident blocks per SM (register cap 65536 / (BLOCK * MINB)),
// the float x sweep for CTU_SWEEPX_MINB (CTU_SWEEPX_MINB_PAR with the
// parabolic terms, whose staging needs the registers of one block fewer).

// Local component q of a sweep along D reads global component gperm<D>(q).
template <int D> __host__ __device__ constexpr int gperm(int q)
{
    return D == 0 ? q
                  : (D == 1 ? (q == 1 ? 2 : q == 2 ? 1 : q == 5 ? 6 : q == 6 ? 5 : q)
                            : (q == 1 ? 3 : q == 2 ? 1 : q == 3 ? 2 : q == 5 ? 7 : q == 6 ? 5 : q == 7 ? 6 : q));
}

__device__ __forceinline__ int lcell(const DevPatch &P, int i, int j, int k)
{
    return ((k + P.g[2]) * P.N[1] + (j + P.g[1])) * P.N[0] + (i + P.g[0]);
}

__device__ __forceinline__ int dstr(const DevPatch &P, int d)
{
    return d == 0 ? 1 : (d == 1 ? P.N[0] : P.N[0] * P.N[1]);
}

// x-width of a block's thread tile for a patch: 8, 16 or 32 lanes along x.
__host__ __device__ __forceinline__ int tile_xw(int nx)
{
    return nx >= 24 ? 32 : (nx >= 12 ? 16 : 8);
}

// Row width of the x sweep's tile: a patch row of up to 32 cells takes one
// row of n_x + 2 lanes (its traced cells, the rows packed BLOCK / (n_x + 2)
// to a block), so that small patches leave few lanes idle; wider rows take
// the group's width w (8, 16 or 32).  The exchange between the lanes of a row
// goes through shared memory, so a row need not be a power of two wide.
__host__ __device__ __forceinline__ int sweepx_xw(int nx, int w)
{
    return nx <= 32 ? nx + 2 : w;
}

// Row width of the marching first-order kernels (k_div1 and k_pred along y
// and z), whose lanes cover x in [-1, n_x]: the same packing, n_x + 2 lanes
// per row for rows of up to 32 cells (the lanes of a row do not exchange
// values, so any width serves).
__host__ __device__ __forceinline__ int ringx_xw(int nx, int w)
{
    return nx <= 32 ? nx + 2 : w;
}

// k_prim's trimmed box (see k_prim) serves patches whose ghosted rows are at
// most PRIM_TRIM_MAXN cells long.
constexpr int PRIM_TRIM_MAXN = 72;
__host__ __device__ __forceinline__ bool prim_trimmed(const int *N) { return N[0] <= PRIM_TRIM_MAXN; }

// Bring the cache line holding *p into L1 ahead of its use (no register is
// held while the load is in flight).
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Asynchronous global -> shared copies (cp.async, per thread): the data land
// in shared memory without occupying registers while in flight.
__device__ __forceinline__ void cp_async(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async(double *dst, const double *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most one committed group of this thread is still in flight
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// wait until every committed group of this thread has landed
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ unsigned int state_flags(double rho, double p)
{
    unsigned int f = 0;
    if (!(rho > 0.0) || !(p > 0.0)) f |= ST_NEG;
    if (!isfinite(rho) || !isfinite(p)) f |= ST_NAN;
    return f;
}

// ---------------------------------------------------------------- parameters in R

template <class R> __device__ __forceinline__ R pgam(const StepArgs &a);
template <> __device__ __forceinline__ double pgam<double>(const StepArgs &a) { return a.gam; }
template <> __device__ __forceinline__ float pgam<float>(const StepArgs &a) { return a.gamf; }
template <class R> __device__ __forceinline__ R pgm1(const StepArgs &a);
template <> __device__ __forceinline__ double pgm1<double>(const StepArgs &a) { return a.gam - 1.0; }
template <> __device__ __forceinline__ float pgm1<float>(const StepArgs &a) { return a.gm1f; }
template <class R> __device__ __forceinline__ R pdt(const StepParams *sp);
template <> __device__ __forceinline__ double pdt<double>(const StepParams *sp) { return sp->dt; }
template <> __device__ __forceinline__ float pdt<float>(const StepParams *sp) { return sp->dtf; }
template <class R> __device__ __forceinline__ R pch(const StepParams *sp);
template <> __device__ __forceinline__ double pch<double>(const StepParams *sp) { return sp->ch; }
template <> __device__ __forceinline__ float pch<float>(const StepParams *sp) { return sp->chf; }
template <class R> __device__ __forceinline__ R pidx(const DevPatch &P, int d);
template <> __device__ __forceinline__ double pidx<double>(const DevPatch &P, int d) { return P.idx[d]; }
template <> __device__ __forceinline__ float pidx<float>(const DevPatch &P, int d) { return P.idxf[d]; }

// ---------------------------------------------------------------- conversions

__device__ __forceinline__ bool prim_from_cons64(const double (&U)[NV], double gm1, double (&V)[NV])
{
    const double rho = U[0];
    const double ir = 1.0 / rho;
    const double vx = U[1] * ir, vy = U[2] * ir, vz = U[3] * ir;
    const double ke = 0.5 * (U[1] * vx + U[2] * vy + U[3] * vz);
    const double me = 0.5 * (U[5] * U[5] + U[6] * U[6] + U[7] * U[7]);
    const double p = gm1 * (U[4] - ke - me);
    V[0] = rho; V[1] = vx; V[2] = vy; V[3] = vz; V[4] = p;
    V[5] = U[5]; V[6] = U[6]; V[7] = U[7]; V[8] = U[8];
    return rho > 0.0 && p > 0.0;
}

// V(U) of a float64 state in precision R.  R = double: plain float64.
// R = float: every field rounded by integer splitting, p in double-float,
// v = m / rho in float32.  Returns status flags.
template <class R> __device__ __forceinline__ unsigned int prim_of(const double (&U)[NV], const StepArgs &a, R (&V)[NV]);

template <>
__device__ __forceinline__ unsigned int prim_of<double>(const double (&U)[NV], const StepArgs &a, double (&V)[NV])
{
    return prim_from_cons64(U, a.gam - 1.0, V) ? 0u : state_flags(V[0], V[4]);
}

template <>
__device__ __forceinline__ unsigned int prim_of<float>(const double (&U)[NV], const StepArgs &a, float (&V)[NV])
{
    // each component split once: its float value and, for the first 8, the
    // double-float pressure
    df u[8];
    float r[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const df sq = df_split(U[q]);
        if (q < 8) u[q] = sq;
        r[q] = sq.hi + sq.lo;
    }
    const float p = df_pressure_split(u, a.gm1f);
    const float ir = 1.0f / r[0];
    V[0] = r[0]; V[1] = r[1] * ir; V[2] = r[2] * ir; V[3] = r[3] * ir; V[4] = p;
    V[5] = r[5]; V[6] = r[6]; V[7] = r[7]; V[8] = r[8];
    return ((!(r[0] > 0.0f) | !(p > 0.0f)) ? ST_NEG : 0u) | ((!isfinite(r[0]) | !isfinite(p)) ? ST_NAN : 0u);
}

// R -> float64 for the update accumulation (integer widening for float).
template <class R> __device__ __forceinline__ double widen(R x);
template <> __device__ __forceinline__ double widen<double>(double x) { return x; }
template <> __device__ __forceinline__ double widen<float>(float x) { return f2d_int(x); }

// V(U) for either physics (SRMHD: float64 Newton recovery).  LIT64 (the
// CTU_MIXED_IFACE64 kernels): the ideal-MHD pressure of a float state is
// recovered in plain float64, p = (Gamma-1)(E - m^2/2rho - B^2/2), and V is
// then rounded to R.
template <int PHYS, class R, int LIT64 = 0>
__device__ __forceinline__ unsigned int prim_any(const double (&U)[NV], const StepArgs &a, R (&V)[NV])
{
    if (PHYS == PH_MHD && LIT64 && sizeof(R) == 4) {
        double Vd[NV];
        const bool ok = prim_from_cons64(U, a.gam - 1.0, Vd);
#pragma unroll
        for (int q = 0; q < NV; ++q) V[q] = (R)Vd[q];
        return ok ? 0u : state_flags(Vd[0], Vd[4]);
    }
    if (PHYS == PH_MHD) return prim_of<R>(U, a, V);
    double Vd[NV];
    const unsigned int st = sr_prim<R>(U, a.gam, Vd);
#pragma unroll
    for (int q = 0; q < NV; ++q) V[q] = (R)Vd[q];
    return st;
}

// CFL speed of one cell: max_d (largest |signal speed| along d) / dx_d.
template <int PHYS, class R>
__device__ __forceinline__ R cell_speed(const R (&V)[NV], const StepArgs &a, const DevPatch &P)
{
    const R g = pgam<R>(a);
    R m = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) continue;
        R s;
        if (PHYS == PH_MHD && sizeof(R) == 4) {
            // fast speed along d from the shared a^2 and B^2/rho
            const R irho = R(1) / V[0];
            const R a2 = g * V[4] * irho;
            const R b2 = (V[5] * V[5] + V[6] * V[6] + V[7] * V[7]) * irho;
            const R bn2 = V[5 + d] * V[5 + d] * irho;
            const R bt2 = b2 - bn2;
            const R disc = sqrt((a2 - b2) * (a2 - b2) + R(4) * a2 * bt2);
            s = fabs(V[1 + d]) + sqrt(R(0.5) * (a2 + b2 + disc));
        } else if (PHYS == PH_MHD) {
            const int b1 = 5 + (d == 0 ? 1 : 0), b2 = 5 + (d == 2 ? 1 : 2);
            s = fabs(V[1 + d]) + fast_speed(V[0], V[4], V[5 + d], V[b1], V[b2], g);
        } else {
            R Vl[NV], lm, lp;
#pragma unroll
            for (int q = 0; q < NV; ++q) Vl[q] = V[perm(d, q)];
            sr_speeds(Vl, g, lm, lp);
            s = fmax(fabs(lm), fabs(lp));
        }
        m = fmax(m, s * pidx<R>(P, d));
    }
    return m;
}

// ---------------------------------------------------------------- per-cell pieces

// Half-step transverse increments dt/2 sum_{d' != D} L^n_d' at cell c (global
// order) from the first-order flux divergences L1 (Eq. transv).
template <class R, int D>
__device__ __forceinline__ void transverse(const StepArgs &a, const R *L1, long long c, R hdt, R (&T)[NV])
{
#pragma unroll
    for (int q = 0; q < NV; ++q) T[q] = R(0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if (e == D || e >= a.ndim) continue;
        const R *Le = L1 + (long long)e * NV * a.sstride;
#pragma unroll
        for (int q = 0; q < NV; ++q) T[q] += Le[q * a.sstride + c] * hdt;
    }
}

// Interface primitive state at n+1/2 from V* (global order) and the
// half-step transverse increments T (Eq. transv).  IFACE64: U* = U(V*) and
// U* + T in float64, pressure recovered in float64.  Otherwise the exact
// increment form p = p* + (Gamma-1)[dE + (rho* v*^2 d_rho - 2 rho* v*.d_m -
// d_m^2)/(2 rho) - d_B.(B* + d_B/2)] in precision R.
template <class R, int IFACE64>
__device__ __forceinline__ unsigned int interface_state(const R (&W)[NV], const R (&T)[NV], const StepArgs &a,
                                                        R (&out)[NV])
{
    if (IFACE64) {
        const double rho = W[0], vx = W[1], vy = W[2], vz = W[3], p = W[4];
        const double bx = W[5], by = W[6], bz = W[7];
        double U[NV], V[NV];
        U[0] = rho + (double)T[0];
        U[1] = rho * vx + (double)T[1];
        U[2] = rho * vy + (double)T[2];
        U[3] = rho * vz + (double)T[3];
        U[4] = p * a.igm + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz) +
               (double)T[4];
        U[5] = bx + (double)T[5];
        U[6] = by + (double)T[6];
        U[7] = bz + (double)T[7];
        U[8] = (double)W[8] + (double)T[8];
        const bool ok = prim_from_cons64(U, a.gam - 1.0, V);
#pragma unroll
        for (int q = 0; q < NV; ++q) out[q] = (R)V[q];
        return ok ? 0u : state_flags(V[0], V[4]);
    } else {
        const R gm1 = pgm1<R>(a);
        const R rs = W[0];
        const R rho = rs + T[0];
        const R irho = R(1) / rho;
        const R v2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
        const R vdm = W[1] * T[1] + W[2] * T[2] + W[3] * T[3];
        const R dm2 = T[1] * T[1] + T[2] * T[2] + T[3] * T[3];
        const R dke = (rs * v2 * T[0] - R(2) * rs * vdm - dm2) * (R(0.5) * irho);
        const R dme = -(T[5] * (W[5] + R(0.5) * T[5]) + T[6] * (W[6] + R(0.5) * T[6]) + T[7] * (W[7] + R(0.5) * T[7]));
        const R p = W[4] + gm1 * (T[4] + dke + dme);
        out[0] = rho;
        out[1] = (rs * W[1] + T[1]) * irho;
        out[2] = (rs * W[2] + T[2]) * irho;
        out[3] = (rs * W[3] + T[3]) * irho;
        out[4] = p;
        out[5] = W[5] + T[5];
        out[6] = W[6] + T[6];
        out[7] = W[7] + T[7];
        out[8] = W[8] + T[8];
        return ((!(rho > R(0)) | !(p > R(0))) ? ST_NEG : 0u) | ((!isfinite(rho) | !isfinite(p)) ? ST_NAN : 0u);
    }
}

// SRMHD interface state at n+1/2: U(V*) + T formed in float64, recovered by
// the float64 Newton iteration (Eq. transv).
template <class R>
__device__ __forceinline__ unsigned int sr_interface(const R (&W)[NV], const R (&T)[NV], const StepArgs &a,
                                                     R (&out)[NV])
{
    double U[NV], V[NV];
    sr_cons<double, R>(W, a.gam, U);
    // Newton starts from the W of the predicted state V* (the transverse
    // correction T is an O(dt) change)
    const double v2 = (double)W[1] * W[1] + (double)W[2] * W[2] + (double)W[3] * W[3];
    const double W0 = sr_w<double>((double)W[0], (double)W[4], a.gam) * rcp64(1.0 - v2);
#pragma unroll
    for (int q = 0; q < NV; ++q) U[q] += (double)T[q];
    const unsigned int st = sr_prim<R>(U, a.gam, V, W0);
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = (R)V[q];
    return st;
}

// Trace one cell along D: stencil (local order) -> interface states (global).
// MHD: characteristic tracing (Section 3.2).  SRMHD: MUSCL-Hancock in
// primitive variables (Section 3.3) from V_(i-1..i+1) and U_i^n.
// T: the half-step transverse increments of the cell (see transverse()).
template <int PHYS, class R, int PPM, int IFACE64, int D>
__device__ __forceinline__ unsigned int trace_cell_t(const StepArgs &a, const DevPatch &P, const R (&vs)[5][NV],
                                                     const R (&T)[NV], long long c, R ch, R dtdx, R (&Vp)[NV],
                                                     R (&Vm)[NV])
{
    R pl[NV], ml[NV], pg[NV], mg[NV];
    unsigned int f = 0;
    // parabolic terms: dt/2 L_P^n joins the half-step increments of every
    // direction (Eq. transv with Pi != 0); the sweeps along y and z take it
    // through the transverse divergence L1_x, to which k_par_half added it
    R Tc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) Tc[q] = T[q];
    if (recon_par(PPM) && D == 0) {
        const R *lp = static_cast<const R *>(a.lp) + c;
        const R hd = R(0.5) * pdt<R>(a.sp);
        Tc[4] += hd * lp[3 * a.sstride];
        if (a.par_visc) {
#pragma unroll
            for (int q = 0; q < 3; ++q) Tc[1 + q] += hd * lp[q * a.sstride];
        }
        if (a.par_res) {
#pragma unroll
            for (int q = 4; q < 7; ++q) Tc[1 + q] += hd * lp[q * a.sstride];
        }
    }
    if (PHYS == PH_MHD) {
        const int lim = recon_hybrid(PPM) ? ((a.flags[c] & 2) ? 2 : 0) : a.limiter;
        char_predict<R, PPM>(vs, pgam<R>(a), ch, dtdx, a.upwind, lim,
                             PPM == RECON_WENO3 ? R(P.dx[D] * P.dx[D]) : R(0), pl, ml);
    } else {
        double U0[NV];
        const long long gi = P.base + (c - P.soff);
#pragma unroll
        for (int q = 0; q < NV; ++q) U0[q] = a.U[gperm<D>(q) * a.ustride + gi];
        f |= sr_mh_predict<R>(vs[1], vs[2], vs[3], U0, pgam<R>(a), ch, dtdx, a.gam, pl, ml);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        pg[gperm<D>(q)] = pl[q];
        mg[gperm<D>(q)] = ml[q];
    }
    if (PHYS == PH_MHD) {
        f |= interface_state<R, IFACE64>(pg, Tc, a, Vp);
        f |= interface_state<R, IFACE64>(mg, Tc, a, Vm);
    } else {
        f |= sr_interface<R>(pg, Tc, a, Vp);
        f |= sr_interface<R>(mg, Tc, a, Vm);
    }
    return f;
}

template <int PHYS, class R, int PPM, int IFACE64, int D>
__device__ __forceinline__ unsigned int trace_cell(const StepArgs &a, const DevPatch &P, const R (&vs)[5][NV],
                                                   const R *L1, long long c, R ch, R dtdx, R hdt, R (&Vp)[NV],
                                                   R (&Vm)[NV])
{
    R T[NV];
    transverse<R, D>(a, L1, c, hdt, T);
    return trace_cell_t<PHYS, R, PPM, IFACE64, D>(a, P, vs, T, c, ch, dtdx, Vp, Vm);
}

// Numerical flux along the local normal for either physics.
template <int PHYS, class R>
__device__ __forceinline__ void riemann_any(const R (&L)[NV], const R (&Rr)[NV], R gam, R ch, R (&F)[NV])
{
    if (PHYS == PH_MHD)
        riemann_hlld(L, Rr, gam, ch, F);
    else
        riemann_hll_sr(L, Rr, gam, ch, F);
}

// n+1/2 flux through a D-face from the left cell's + state and the right
// cell's - state (both global order); flux returned in global order.
template <int PHYS, class R, int D, bool HLLC = false>
__device__ __forceinline__ void face_flux(const R (&Lg)[NV], const R (&Rg)[NV], R gam, R ch, R (&Fg)[NV],
                                          bool hll = false)
{
    R L[NV], Rr[NV], F[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        L[q] = Lg[gperm<D>(q)];
        Rr[q] = Rg[gperm<D>(q)];
    }
    if (PHYS == PH_MHD && hll)
        riemann_hll(L, Rr, gam, ch, F);
    else if (PHYS == PH_MHD && HLLC)
        riemann_hllc(L, Rr, gam, ch, F);
    else
        riemann_any<PHYS, R>(L, Rr, gam, ch, F);
#pragma unroll
    for (int q = 0; q < NV; ++q) Fg[gperm<D>(q)] = F[q];
}

// First flux-register window of plane pl normal to D of a patch (windows of
// the plane: [window_first(pl), window_first(pl + 1))); 0 when the patch has
// none in direction D.  Kernels read these ahead of the face solves.
__device__ __forceinline__ int window_base(const StepArgs &a, int patch, int D)
{
    return a.reg ? a.wbase[patch * 3 + D] : -1;
}
__device__ __forceinline__ int window_first(const StepArgs &a, int B, int pl)
{
    return B >= 0 ? a.wpos[B + pl] : 0;
}

// Flux-register windows [w0, w1) of one face (normal to D, transverse
// coordinates ca, cb in increasing dimension order), Eq. (fluxcorr).
template <class R, int D>
__device__ __forceinline__ void register_face(const StepArgs &a, const DevPatch &P, int w0, int w1, int ca, int cb,
                                              const R (&Fg)[NV], double dt)
{
    for (int w = w0; w < w1; ++w) {
        const DevWindow W = a.win[w];
        if (ca < W.a0 || ca >= W.a1 || cb < W.b0 || cb >= W.b1) continue;
        constexpr int ea = D == 0 ? 1 : 0, eb = D == 2 ? 1 : 2;
        const double f = W.weight * dt * P.dx[ea] * P.dx[eb];
        const long long na = W.a1 - W.a0, nb = W.b1 - W.b0;
        const long long o = W.dst + (long long)(cb - W.b0) * na + (ca - W.a0);
#pragma unroll
        for (int q = 0; q < NV; ++q) a.reg[o + q * nb * na] += f * widen<R>(Fg[q]);
    }
}

// One variable q of register_face.
template <class R, int D>
__device__ __forceinline__ void register_face_var(const StepArgs &a, const DevPatch &P, int w0, int w1, int ca, int cb,
                                                  int q, R Fq, double dt)
{
    for (int w = w0; w < w1; ++w) {
        const DevWindow W = a.win[w];
        if (ca < W.a0 || ca >= W.a1 || cb < W.b0 || cb >= W.b1) continue;
        constexpr int ea = D == 0 ? 1 : 0, eb = D == 2 ? 1 : 2;
        const double f = W.weight * dt * P.dx[ea] * P.dx[eb];
        const long long na = W.a1 - W.a0, nb = W.b1 - W.b0;
        const long long o = W.dst + (long long)(cb - W.b0) * na + (ca - W.a0);
        a.reg[o + q * nb * na] += f * widen<R>(Fq);
    }
}

// ---- parabolic terms in the final update (the RECON_*_PAR kernels)

// Entries of L_P and of a face's Pi: 0..2 momentum, 3 energy, 4..6 B
// (conserved component 1 + q).
constexpr int NPAR = 7;

// (Gamma - 1) max(kappa_perp, kappa_par), nu and eta in the working precision.
template <class R> __device__ __forceinline__ R par_gk(const StepArgs &a);
template <> __device__ __forceinline__ double par_gk<double>(const StepArgs &a)
{
    return (a.gam - 1.0) * (a.kpar > a.kappa ? a.kpar : a.kappa);
}
template <> __device__ __forceinline__ float par_gk<float>(const StepArgs &a) { return a.gm1f * a.kmaxf; }
template <class R> __device__ __forceinline__ R par_nu(const StepArgs &a);
template <> __device__ __forceinline__ double par_nu<double>(const StepArgs &a) { return a.nu; }
template <> __device__ __forceinline__ float par_nu<float>(const StepArgs &a) { return a.nuf; }
template <class R> __device__ __forceinline__ R par_eta(const StepArgs &a);
template <> __device__ __forceinline__ double par_eta<double>(const StepArgs &a) { return a.eta; }
template <> __device__ __forceinline__ float par_eta<float>(const StepArgs &a) { return a.etaf; }

// Whether the parabolic terms change entry q of L_P: the energy always, the
// momentum with viscosity, B with resistivity.
__device__ __forceinline__ bool par_on(const StepArgs &a, int q)
{
    return q == 3 || (q < 3 ? a.par_visc != 0 : a.par_res != 0);
}

// The diffusion term of the CFL rate, Eq. (Ca): 2 D sum_d 1/dx_d^2 with
// D = max((Gamma - 1) kappa_max / rho, 4/3 nu, eta).
template <class R> __device__ __forceinline__ R diffusion_rate(const StepArgs &a, const DevPatch &P, R rho)
{
    const R D = max(max(par_gk<R>(a) / rho, R(4.0 / 3.0) * par_nu<R>(a)), par_eta<R>(a));
    R r = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < a.ndim) r += R(2) * D * (pidx<R>(P, d) * pidx<R>(P, d));
    return r;
}

// Final update of one interior cell: U^(n+1) = U^n + dt s, psi source, and
// the CFL speed of U^(n+1) if requested (returned in R; 0 otherwise), with
// the diffusion term when DIFF.  u0: U^n of the cell.
template <int PHYS, class R, int LIT64 = 0, bool DIFF = false>
__device__ __forceinline__ R finish_cell_u(const StepArgs &a, const DevPatch &P, int cl, const R (&s)[NV],
                                           const double (&u0)[NV], double dt, double damp, unsigned int &fl)
{
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = fma(dt, widen<R>(s[q]), u0[q]);
    u[8] *= damp;
#pragma unroll
    for (int q = 0; q < NV; ++q) a.Uout[q * a.ustride + P.base + cl] = u[q];
    if (!a.nextmax) return R(0);
    R V[NV];
    fl |= prim_any<PHYS, R, LIT64>(u, a, V);
    R m = cell_speed<PHYS, R>(V, a, P);
    if constexpr (DIFF) m += diffusion_rate<R>(a, P, V[0]);
    return m;
}

// Ideal MHD in float: as finish_cell_u, but the CFL speed of U^(n+1) comes
// from the primitive state V^n of the cell (global order) and the increment
// dt s through the exact increment form of the pressure (interface_state),
// so that U^(n+1) itself is never split or recovered in double-float.
template <class R, bool DIFF = false>
__device__ __forceinline__ R finish_cell_inc(const StepArgs &a, const DevPatch &P, int cl, const R (&s)[NV],
                                             const double (&u0)[NV], const R (&Vn)[NV], double dt, R dtr,
                                             double damp, unsigned int &fl)
{
    double u[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u[q] = fma(dt, widen<R>(s[q]), u0[q]);
    u[8] *= damp;
#pragma unroll
    for (int q = 0; q < NV; ++q) a.Uout[q * a.ustride + P.base + cl] = u[q];
    if (!a.nextmax) return R(0);
    R d[NV], V[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) d[q] = dtr * s[q];
    fl |= interface_state<R, 0>(Vn, d, a, V);
    R m = cell_speed<PH_MHD, R>(V, a, P);
    if constexpr (DIFF) m += diffusion_rate<R>(a, P, V[0]);
    return m;
}

template <int PHYS, class R, int LIT64 = 0, bool DIFF = false>
__device__ __forceinline__ R finish_cell(const StepArgs &a, const DevPatch &P, int cl, const R (&s)[NV],
                                         double dt, double damp, unsigned int &fl)
{
    double u0[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) u0[q] = a.U[q * a.ustride + P.base + cl];
    return finish_cell_u<PHYS, R, LIT64, DIFF>(a, P, cl, s, u0, dt, damp, fl);
}

// Block maximum of a non-negative value, folded into *out as the bits of a
// float64 (monotone in the value for non-negative doubles).
template <class R> __device__ __forceinline__ void block_max_to(R m, unsigned long long *out)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ R sm[BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = m;
    __syncthreads();
    if (wid == 0) {
        m = lane < BLOCK / 32 ? sm[lane] : R(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > R(0)) atomicMax(out, (unsigned long long)__double_as_longlong(widen<R>(m)));
    }
}

__device__ __forceinline__ double patch_damp(const StepArgs &a, const DevPatch &P)
{
    __shared__ double s_damp;
    if (threadIdx.x == 0) s_damp = exp(-a.glm_alpha * a.sp->ch * a.sp->dt / P.hmin);
    __syncthreads();
    return s_damp;
}

// Thread tile of a block: BLOCK threads as xw lanes along x times BLOCK/xw rows.
struct Tile {
    int xw, rows;
    __device__ __forceinline__ explicit Tile(int w)
    {
        xw = w;
        rows = BLOCK / xw;
    }
    __device__ __forceinline__ int tx() const { return threadIdx.x % xw; }
    __device__ __forceinline__ int ty() const { return threadIdx.x / xw; }
};

// Host mirror of the kernels' block counts per patch (same tiling), for an
// x tile width w (8, 16 or 32 lanes) and a marching segment of seg cells.
struct Tiles {
    static int xw(int nx) { return tile_xw(nx); }
    static long long prim(const int *N)
    {
        return ((long long)N[0] * N[1] * N[2] + BLOCK * PRIM_CELLS - 1) / (BLOCK * PRIM_CELLS);
    }
    // one thread per ghosted cell (the shock flags)
    static long long ghosted(const int *N) { return ((long long)N[0] * N[1] * N[2] + BLOCK - 1) / BLOCK; }
    // k_prim<..., TRIM>: on small patches (prim_trimmed) the ghosted box
    // without its outermost layer on active axes (N > 1 there)
    static long long prim_trim(const int *N)
    {
        if (!prim_trimmed(N)) return prim(N);
        return ((long long)(N[0] - 2) * (N[1] > 1 ? N[1] - 2 : 1) * (N[2] > 1 ? N[2] - 2 : 1) + BLOCK * PRIM_CELLS - 1) /
               (BLOCK * PRIM_CELLS);
    }
    // ext: along D also the ring's layers -1 and n_D (k_div1's EXT)
    // rows per thread of k_div1<0> and of k_sweep_x on patches of n cells,
    // at most `most`
    static int div1x_rows(const int *n, int ndim, int w, int most)
    {
        return rows_per_thread(most, ndim > 1 ? n[1] + 2 : 1, BLOCK / w);
    }
    static int sweepx_rows(const int *n, int w, int most)
    {
        return rows_per_thread(most, n[1], BLOCK / sweepx_xw(n[0], w));
    }
    static long long div1(const int *n, int ndim, int D, int w, int seg, bool ext = false, int most = DIV1X_ROWS)
    {
        const int r = BLOCK / w;
        const int x2 = ext ? 2 : 0;
        if (D == 0) {
            const int e1 = ndim > 1 ? n[1] + 2 : 1, e2 = ndim > 2 ? n[2] + 2 : 1;
            const int rr = r * div1x_rows(n, ndim, w, most);  // rows of a block
            return (long long)((n[0] + x2 + w - 2) / (w - 1)) * ((e1 + rr - 1) / rr) * e2;
        }
        const int O = D == 1 ? 2 : 1;
        const int eO = ndim > O ? n[O] + 2 : 1;
        const long long nseg = (n[D] + x2 + seg - 1) / seg;
        const int wr = ringx_xw(n[0], w), rr = BLOCK / wr;
        return (long long)((n[0] + 2 + wr - 1) / wr) * ((eO * nseg + rr - 1) / rr);
    }
    // the corner coupling's transverse fluxes along x (k_pred<0>): traced
    // cells [-1, n_x], rows and planes over the ring [-1, n]
    static long long pred_x(const int *n, int ndim, int w)
    {
        const int r = BLOCK / w;
        const int e1 = ndim > 1 ? n[1] + 2 : 1, e2 = ndim > 2 ? n[2] + 2 : 1;
        return (long long)((n[0] + w - 3) / (w - 2)) * ((e1 + r - 1) / r) * e2;
    }
    static long long sweep_x(const int *n, int w, int most = SWEEPX_ROWS)
    {
        const int xr = sweepx_rows(n, w, most);
        w = sweepx_xw(n[0], w);
        const int rr = (BLOCK / w) * xr;  // rows of a block
        return (long long)((n[0] + w - 3) / (w - 2)) * ((n[1] + rr - 1) / rr) * n[2];
    }
    static long long sweep_m(const int *n, int D, int w, int seg)
    {
        const int O = D == 1 ? 2 : 1;
        const int r = BLOCK / w;
        const long long nseg = (n[D] + seg - 1) / seg;
        return (long long)((n[0] + w - 1) / w) * ((n[O] * nseg + r - 1) / r);
    }
    static long long interior(const int *n, int w)
    {
        const int r = BLOCK / w;
        return (long long)((n[0] + w - 1) / w) * ((n[1] + r - 1) / r) * n[2];
    }
};

// ---------------------------------------------------------------- kernels

static __global__ void k_setup(const double *dtch, StepParams *sp)
{
    const double dt = dtch[0], ch = dtch[1];
    sp->dt = dt;
    sp->ch = ch;
    sp->dtf = (float)dt;
    sp->chf = (float)ch;
}

// V = V(U) on every ghosted cell (a flat range of the patch region);
// one block per BLOCK x PRIM_CELLS cells of a patch, a thread PRIM_CELLS
// cells BLOCK apart.  LIT64: float64 pressure recovery in
// the float kernels (CTU_MIXED_IFACE64).
// TRIM: on patches whose ghosted rows are at most PRIM_TRIM_MAXN cells long,
// only the cells within three ghost layers of the interior (the stencils of
// the first-order stage, the predictors and the parabolic face pass reach no
// further); the layer saved is a large part of a small patch, while on a
// large one the index arithmetic of the trimmed box would cost more than it
// saves.  The hybrid integration's shock flags, which read the fourth
// layer, take the whole ghosted box.

template <int PHYS, class R, int LIT64 = 0, bool TRIM = false>
__global__ void __launch_bounds__(BLOCK) k_prim(StepArgs a, GroupTable gt, R *Vs)
{
    const Where w = locate(gt);
    const DevPatch P = a.patches[w.patch];
    const bool trim = TRIM && prim_trimmed(P.N);
    // box of the ghosted patch without its outermost layer on active axes
    const int m0 = P.N[0] - 2, m1 = P.g[1] ? P.N[1] - 2 : 1, m2 = P.g[2] ? P.N[2] - 2 : 1;
    const int ncell = trim ? m0 * m1 * m2 : P.N[0] * P.N[1] * P.N[2];
    unsigned int f = 0;
#pragma unroll 1
    for (int r = 0; r < PRIM_CELLS; ++r) {
        int c = (w.b * PRIM_CELLS + r) * BLOCK + threadIdx.x;
        if (c >= ncell) break;
        if (trim) {
            const int x = c % m0 + 1, y = (c / m0) % m1 + (P.g[1] ? 1 : 0), z = c / (m0 * m1) + (P.g[2] ? 1 : 0);
            c = (z * P.N[1] + y) * P.N[0] + x;
        }
        double U[NV];
        R V[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) U[q] = a.U[q * a.ustride + P.base + c];
        f |= prim_any<PHYS, R, LIT64>(U, a, V);
#pragma unroll
        for (int q = 0; q < NV; ++q) Vs[q * a.sstride + P.soff + c] = V[q];
    }
    if (f) atomicOr(a.status, f);
}

// ---- hybrid integration: shock flags (appendix on shock detection) ----
// A cell within three layers of the interior is shocked when
//   S = sum_d |q(c + e_d) - q(c - e_d)| / min(q(c + e_d), q(c - e_d)) > eps_q
//   and D = sum_d (v_d(c + e_d) - v_d(c - e_d)) / (2 dx_d) < 0
// (q the thermal or magnetic pressure).  Both sums are formed from the
// working-precision primitives; a cell whose S or D lies within the
// relative margin of its threshold that bounds the difference between these
// primitives and float64 ones (1e-4 in float32, 1e-9 in float64) is decided
// again from the float64 state, in explicitly rounded operations in the
// order of the definition, so each flag is the float64 definition's.
__device__ __forceinline__ void prim_exact(const StepArgs &a, long long g, double gm1, int d, int qk, double &q,
                                           double &v)
{
    const double *U = a.U;
    const long long us = a.ustride;
    const double rho = U[g];
    if (qk == 0) {
        const double m0 = U[us + g], m1 = U[2 * us + g], m2 = U[3 * us + g];
        const double b0 = U[5 * us + g], b1 = U[6 * us + g], b2 = U[7 * us + g];
        const double mm = __dadd_rn(__dadd_rn(__dmul_rn(m0, m0), __dmul_rn(m1, m1)), __dmul_rn(m2, m2));
        const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)), __dmul_rn(b2, b2));
        q = __dmul_rn(gm1, __dsub_rn(__dsub_rn(U[4 * us + g], __ddiv_rn(__dmul_rn(0.5, mm), rho)), __dmul_rn(0.5, bb)));
    } else {
        const double b0 = U[5 * us + g], b1 = U[6 * us + g], b2 = U[7 * us + g];
        q = __dmul_rn(0.5, __dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)), __dmul_rn(b2, b2)));
    }
    v = __ddiv_rn(U[(1 + d) * us + g], rho);
}

template <class R>
__global__ void __launch_bounds__(BLOCK) k_shock(StepArgs a, GroupTable gt, const R *Vs)
{
    const Where w = locate(gt);
    const DevPatch P = a.patches[w.patch];
    const int c = w.b * BLOCK + threadIdx.x;
    if (c >= P.N[0] * P.N[1] * P.N[2]) return;
    const int gx = c % P.N[0], gy = (c / P.N[0]) % P.N[1], gz = c / (P.N[0] * P.N[1]);
    const int x[3] = {gx - P.g[0], gy - P.g[1], gz - P.g[2]};
    bool in = true;
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < a.ndim) in &= x[d] >= -3 && x[d] < P.n[d] + 3;
    unsigned char f = 0;
    if (in) {
        const long long sc = P.soff + c;
        const long long ss = a.sstride;
        const long long st[3] = {1, P.N[0], (long long)P.N[0] * P.N[1]};
        const R eps = (R)a.shock_eps;
        R S = R(0), D = R(0), Bd = R(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= a.ndim) break;
            const long long ip = sc + st[d], im = sc - st[d];
            R qp, qm;
            if (a.shock_q == 0) {
                qp = Vs[4 * ss + ip];
                qm = Vs[4 * ss + im];
            } else {
                qp = R(0.5) * (Vs[5 * ss + ip] * Vs[5 * ss + ip] + Vs[6 * ss + ip] * Vs[6 * ss + ip] +
                               Vs[7 * ss + ip] * Vs[7 * ss + ip]);
                qm = R(0.5) * (Vs[5 * ss + im] * Vs[5 * ss + im] + Vs[6 * ss + im] * Vs[6 * ss + im] +
                               Vs[7 * ss + im] * Vs[7 * ss + im]);
            }
            S += fabs(qp - qm) / fmin(qp, qm);
            const R h2 = R(0.5) * pidx<R>(P, d);
            const R vp = Vs[(1 + d) * ss + ip], vm = Vs[(1 + d) * ss + im];
            D += (vp - vm) * h2;
            Bd += (fabs(vp) + fabs(vm)) * h2;
        }
        const R tol = sizeof(R) == 4 ? R(1e-4) : R(1e-9);
        const R ms = tol * (S + eps + R(1)), md = tol * Bd;
        const bool s_yes = S - eps > ms, s_no = eps - S > ms;
        const bool d_yes = D < -md, d_no = D > md;
        if (s_yes && d_yes) {
            f = 1;
        } else if (!(s_no || d_no)) {
            const long long g = P.base + c;
            const double gm1 = a.gam - 1.0;
            double Se = 0.0, De = 0.0;
            for (int d = 0; d < a.ndim; ++d) {
                const long long sg = d == 0 ? 1 : (d == 1 ? (long long)P.N[0] : (long long)P.N[0] * P.N[1]);
                double qp, qm, vp, vm;
                prim_exact(a, g + sg, gm1, d, a.shock_q, qp, vp);
                prim_exact(a, g - sg, gm1, d, a.shock_q, qm, vm);
                Se = __dadd_rn(Se, __ddiv_rn(fabs(__dsub_rn(qp, qm)), fmin(qp, qm)));
                De = __dadd_rn(De, __ddiv_rn(__dsub_rn(vp, vm), __dmul_rn(2.0, P.dx[d])));
            }
            f = (Se > a.shock_eps && De < 0.0) ? 1 : 0;
        }
    }
    a.flags[P.soff + c] = f;
}

// MinMod flag (bit 2) on the cells [-1, n + 1): a shocked cell within
// `reach` cells along an active axis (2 for PPM, 1 for MC-linear).
static __global__ void __launch_bounds__(BLOCK) k_minmod(StepArgs a, GroupTable gt, int reach)
{
    const Where w = locate(gt);
    const DevPatch P = a.patches[w.patch];
    const int c = w.b * BLOCK + threadIdx.x;
    if (c >= P.N[0] * P.N[1] * P.N[2]) return;
    const int gx = c % P.N[0], gy = (c / P.N[0]) % P.N[1], gz = c / (P.N[0] * P.N[1]);
    const int x[3] = {gx - P.g[0], gy - P.g[1], gz - P.g[2]};
    bool in = true;
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (d < a.ndim) in &= x[d] >= -1 && x[d] < P.n[d] + 1;
    if (!in) return;
    const long long sc = P.soff + c;
    const long long st[3] = {1, P.N[0], (long long)P.N[0] * P.N[1]};
    unsigned m = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= a.ndim) break;
        for (int k = -reach; k <= reach; ++k) m |= a.flags[sc + k * st[d]];
    }
    if (m & 1) a.flags[sc] |= 2;
}

// First-order flux divergences L1_D = (F^n_(c - e_D/2) - F^n_(c + e_D/2)) / dx_D
// (Eq. transv; F^n from the cell-centred states) on the cells that the
// sweeps of the other directions trace: c_D in [0, n_D), the other active
// coordinates in [-1, n]; with EXT (the parabolic terms' half-step state)
// c_D in [-1, n_D] as well, the whole ring box.
//   D = x: one thread per face of several rows in turn (Tiles::div1x_rows);
//          a tile of xw lanes along x yields xw - 1 cells, the lower face of
//          a cell arriving from the previous lane.
//   D = y, z: one thread per segment of SEG cells marching along D with the
//          previous face flux and cell state in registers.
template <int PHYS, class R, int D, bool HYB = false, bool HLLC = false, bool EXT = false>
__global__ void __launch_bounds__(BLOCK) k_div1(StepArgs a, GroupTable gt, const R *Vs, R *L1)
{
    const Where wh = locate(gt);
    const DevPatch P = a.patches[wh.patch];
    const Tile t(D == 0 ? wh.xw : ringx_xw(P.n[0], wh.xw));
    const int SEGL = wh.seg;
    const R gam = pgam<R>(a), ch = pch<R>(a.sp);
    const R iD = pidx<R>(P, D);
    R *Ld = L1 + (long long)D * NV * a.sstride;
    const int b = wh.b;
    if constexpr (D == 0) {
        const int out = t.xw - 1;
        const int e1 = a.ndim > 1 ? P.n[1] + 2 : 1, e2 = a.ndim > 2 ? P.n[2] + 2 : 1;
        const int lo1 = a.ndim > 1 ? -1 : 0, lo2 = a.ndim > 2 ? -1 : 0;
        constexpr int X = EXT ? 1 : 0;
        const int xr = wh.xr;         // rows of a thread (Tiles::div1x_rows)
        const int RR = t.rows * xr;  // rows of a block
        const int T0 = (P.n[0] + 2 * X + out - 1) / out, T1 = (e1 + RR - 1) / RR;
        const int tx = t.tx();
        const int i = (b % T0) * out + tx - X;  // this lane's face lies between cells i - 1 and i
        const int jb = ((b / T0) % T1) * RR + t.ty();
        const int k = b / (T0 * T1);
        const long long row = (long long)P.N[0];  // scratch distance of adjacent rows
        long long c = P.soff + lcell(P, i, lo1 + jb, lo2 + (k < e2 ? k : 0));  // cell i of row jb
#pragma unroll 1
        for (int r = 0; r < xr; ++r, c += t.rows * row) {
            const int j = jb + r * t.rows;
            const bool face = j < e1 && k < e2 && i <= P.n[0] + X;
            R F[NV];
            if (face) {
                R L[NV], Rr[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    L[q] = Vs[q * a.sstride + c - 1];
                    Rr[q] = Vs[q * a.sstride + c];
                }
                if (HYB && PHYS == PH_MHD && ((a.flags[c - 1] | a.flags[c]) & 1))
                    riemann_hll(L, Rr, gam, ch, F);
                else if (HLLC && PHYS == PH_MHD)
                    riemann_hllc(L, Rr, gam, ch, F);
                else
                    riemann_any<PHYS, R>(L, Rr, gam, ch, F);
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) F[q] = R(0);
            }
            // every lane of the warp takes part in the exchange
            R Fm[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) Fm[q] = __shfl_up_sync(0xffffffffu, F[q], 1, t.xw);
            if (face && tx >= 1) {  // cell i - 1: lower face from lane tx - 1, upper face F
#pragma unroll
                for (int q = 0; q < NV; ++q) Ld[q * a.sstride + c - 1] = (Fm[q] - F[q]) * iD;
            }
        }
    } else {
        constexpr int O = D == 1 ? 2 : 1;  // the other transverse dimension
        constexpr int X = EXT ? 1 : 0;
        const int nD = P.n[D];
        const int eO = a.ndim > O ? P.n[O] + 2 : 1, loO = a.ndim > O ? -1 : 0;
        const int nseg = (nD + 2 * X + SEGL - 1) / SEGL;
        const int T0 = (P.n[0] + 2 + t.xw - 1) / t.xw;
        const int x = (b % T0) * t.xw + t.tx() - 1;
        const int comb = (b / T0) * t.rows + t.ty();
        const int o = comb / nseg, seg = comb % nseg;
        // (threads beyond the block's last full row take no work)
        if (t.ty() >= t.rows || x > P.n[0] || o >= eO) return;
        const int j0 = seg * SEGL - X, j1 = min(j0 + SEGL, nD + X);
        const int st = dstr(P, D);
        int cc[3];
        cc[0] = x;
        cc[O] = loO + o;
        cc[D] = j0 - 1;
        long long c = P.soff + lcell(P, cc[0], cc[1], cc[2]);  // cell j0 - 1
        R Vl[NV], Vr[NV], Fp[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            Vl[q] = Vs[gperm<D>(q) * a.sstride + c];
            Vr[q] = Vs[gperm<D>(q) * a.sstride + c + st];
            Fp[q] = R(0);
        }
        for (int j = j0; j <= j1; ++j) {
            c += st;  // cell j; the face below it separates j - 1 and j
            R Vn[NV];
            if (j < j1) {  // next cell, loaded ahead of the solve
#pragma unroll
                for (int q = 0; q < NV; ++q) Vn[q] = Vs[gperm<D>(q) * a.sstride + c + st];
            }
            R F[NV];
            if (HYB && PHYS == PH_MHD && ((a.flags[c - st] | a.flags[c]) & 1))
                riemann_hll(Vl, Vr, gam, ch, F);
            else if (HLLC && PHYS == PH_MHD)
                riemann_hllc(Vl, Vr, gam, ch, F);
            else
                riemann_any<PHYS, R>(Vl, Vr, gam, ch, F);
            if (j > j0) {  // cell j - 1
#pragma unroll
                for (int q = 0; q < NV; ++q) Ld[gperm<D>(q) * a.sstride + c - st] = (Fp[q] - F[q]) * iD;
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                Fp[q] = F[q];
                Vl[q] = Vr[q];
                Vr[q] = Vn[q];
            }
        }
    }
}

// The corner coupling of Mignone & Tzeferacos (2010) (the kinds
// RECON_PPM_MT, RECON_MC_MT; Section 3.1 with Pi = 0): in place of k_div1,
// the transverse fluxes come from Riemann problems between the normal
// predictor states, F*_D = R(V*_(c,+), V*_(c+e_D,-)) (characteristic
// predictor of Section 3.2, no transverse terms), and L1_D = (F*_(c - e_D/2)
// - F*_(c + e_D/2)) / dx_D on the cells the sweeps of the other directions
// trace: c_D in [0, n_D), the other active coordinates in [-1, n].
//   D = x: one thread per traced cell c_x in [-1, n_x]; a tile of xw lanes
//          yields xw - 2 cells, the right neighbour's - state and the left
//          neighbour's face flux arriving by warp shuffles (a row of the
//          tile lies within one warp).
//   D = y, z: one thread per segment marching along D, the 5-cell stencil,
//          the previous cell's + state and the previous face flux in
//          registers (the k_div1 tiling).
template <int PHYS, class R, int PPM, int D>
__global__ void __launch_bounds__(BLOCK) k_pred(StepArgs a, GroupTable gt, const R *Vs, R *L1)
{
    const Where wh = locate(gt);
    const DevPatch P = a.patches[wh.patch];
    const Tile t(D == 0 ? wh.xw : ringx_xw(P.n[0], wh.xw));
    const R gam = pgam<R>(a), ch = pch<R>(a.sp);
    const R dtr = pdt<R>(a.sp);
    const R iD = pidx<R>(P, D);
    const R dtdx = dtr * iD;
    R *Ld = L1 + (long long)D * NV * a.sstride;
    const int b = wh.b;
    if constexpr (D == 0) {
        const int out = t.xw - 2;
        const int e1 = a.ndim > 1 ? P.n[1] + 2 : 1, e2 = a.ndim > 2 ? P.n[2] + 2 : 1;
        const int lo1 = a.ndim > 1 ? -1 : 0, lo2 = a.ndim > 2 ? -1 : 0;
        const int T0 = (P.n[0] + out - 1) / out, T1 = (e1 + t.rows - 1) / t.rows;
        const int tx = t.tx();
        const int i = (b % T0) * out - 1 + tx;  // traced cell, >= -1
        const int j = ((b / T0) % T1) * t.rows + t.ty();
        const int k = b / (T0 * T1);
        const bool traced = j < e1 && k < e2 && i <= P.n[0];
        const long long c = traced ? P.soff + lcell(P, i, lo1 + j, lo2 + k) : 0;
        R pl[NV], ml[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { pl[q] = R(0); ml[q] = R(0); }
        if (traced) {
            R vs[5][NV];
#pragma unroll
            for (int m = 0; m < 5; ++m)
#pragma unroll
                for (int q = 0; q < NV; ++q) vs[m][q] = Vs[q * a.sstride + c + (m - 2)];
            char_predict<R, PPM>(vs, gam, ch, dtdx, a.upwind, a.limiter, R(0), pl, ml);
        }
        // face between cells i and i + 1 (every lane takes part in the shuffles)
        R Rr[NV], F[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            Rr[q] = __shfl_down_sync(0xffffffffu, ml[q], 1, t.xw);
            F[q] = R(0);
        }
        if (traced && tx < t.xw - 1 && i <= P.n[0] - 1) riemann_any<PHYS, R>(pl, Rr, gam, ch, F);
        R Fm[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) Fm[q] = __shfl_up_sync(0xffffffffu, F[q], 1, t.xw);
        if (traced && tx >= 1 && tx <= t.xw - 2 && i >= 0 && i < P.n[0]) {
#pragma unroll
            for (int q = 0; q < NV; ++q) Ld[q * a.sstride + c] = (Fm[q] - F[q]) * iD;
        }
    } else {
        constexpr int O = D == 1 ? 2 : 1;  // the other transverse dimension
        const int SEGL = wh.seg;
        const int nD = P.n[D];
        const int eO = a.ndim > O ? P.n[O] + 2 : 1, loO = a.ndim > O ? -1 : 0;
        const int nseg = (nD + SEGL - 1) / SEGL;
        const int T0 = (P.n[0] + 2 + t.xw - 1) / t.xw;
        const int x = (b % T0) * t.xw + t.tx() - 1;
        const int comb = (b / T0) * t.rows + t.ty();
        const int o = comb / nseg, seg = comb % nseg;
        if (t.ty() >= t.rows || x > P.n[0] || o >= eO) return;
        const int j0 = seg * SEGL, j1 = min(j0 + SEGL, nD);
        const int st = dstr(P, D);
        int cc[3];
        cc[0] = x;
        cc[O] = loO + o;
        cc[D] = j0 - 1;
        long long c = P.soff + lcell(P, cc[0], cc[1], cc[2]);  // traced cell j0 - 1
        R win[5][NV];
#pragma unroll
        for (int m = 0; m < 5; ++m)
#pragma unroll
            for (int q = 0; q < NV; ++q) win[m][q] = Vs[gperm<D>(q) * a.sstride + c + (m - 2) * st];
        R Pprev[NV], Fprev[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { Pprev[q] = R(0); Fprev[q] = R(0); }
        for (int j = j0 - 1; j <= j1; ++j, c += st) {
            if (j > j0 - 1) {
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int q = 0; q < NV; ++q) win[m][q] = win[m + 1][q];
#pragma unroll
                for (int q = 0; q < NV; ++q) win[4][q] = Vs[gperm<D>(q) * a.sstride + c + 2 * st];
            }
            R pl[NV], ml[NV];
            char_predict<R, PPM>(win, gam, ch, dtdx, a.upwind, a.limiter, R(0), pl, ml);
            if (j >= j0) {  // face between cells j - 1 and j
                R F[NV];
                riemann_any<PHYS, R>(Pprev, ml, gam, ch, F);
                if (j > j0) {  // cell j - 1
#pragma unroll
                    for (int q = 0; q < NV; ++q) Ld[gperm<D>(q) * a.sstride + c - st] = (Fprev[q] - F[q]) * iD;
                }
#pragma unroll
                for (int q = 0; q < NV; ++q) Fprev[q] = F[q];
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) Pprev[q] = pl[q];
        }
    }
}

// Sweep along x, one thread per traced cell of up to SWEEPX_ROWS rows.  A
// tile covers xw traced cells (xw - 2 updated cells) along x times BLOCK/xw
// rows along y, a block that many rows per thread in turn.  The last sweep
// of the step: U^(n+1) from U^n, dt (A + L_x) and the psi source, and the
// next step's CFL speed.  With the parabolic terms the update also adds
// dt L_P^(n+1/2) (k_par_lp), and the CFL rate gains the diffusion term.
template <int PHYS, class R, int PPM, int IFACE64, int LAST>
__global__ void __launch_bounds__(BLOCK, sizeof(R) == 4 ? (recon_par(PPM) ? CTU_SWEEPX_MINB_PAR : CTU_SWEEPX_MINB) : 1)
    k_sweep_x(StepArgs a, GroupTable gt, const R *Vs, const R *L1, R *A)
{
    const Where wh = locate(gt);
    const int patch = wh.patch;
    const DevPatch P = a.patches[patch];
    const Tile t(sweepx_xw(P.n[0], wh.xw));
    const int out_x = t.xw - 2;
    const int xr = wh.xr;         // rows of a thread (Tiles::sweepx_rows)
    const int RR = t.rows * xr;  // rows of a block
    const int T0 = (P.n[0] + out_x - 1) / out_x, T1 = (P.n[1] + RR - 1) / RR;
    const int b = wh.b;
    const int tx = t.tx(), ty = t.ty();
    const int i = (b % T0) * out_x - 1 + tx;  // traced cell, >= -1
    const int j0 = ((b / T0) % T1) * RR;      // the block's first row
    const int k = b / (T0 * T1);
    __shared__ R sP[BLOCK][NV], sM[BLOCK][NV], sF[BLOCK][NV];
    // faces of the block with flux-register windows: lane, first and end
    // window (the count alternates between two slots from row to row, so
    // that resetting one never races with reading the other)
    __shared__ int s_nreg[2], s_reg[BLOCK][3];
    const int me = threadIdx.x;
    const R gam = pgam<R>(a), ch = pch<R>(a.sp);
    const R dtr = pdt<R>(a.sp);
    const double dtd = a.sp->dt;
    const R dtdx = dtr * pidx<R>(P, 0);
    const R hdt = R(0.5) * dtr;
    unsigned int fl = 0;
    constexpr bool PAR = recon_par(PPM);
    constexpr bool PSTAGE = PAR && LAST && sizeof(R) == 4;
    __shared__ float sLp[PSTAGE ? NPAR : 1][BLOCK];
    const double damp = LAST ? patch_damp(a, P) : 1.0;  // includes a block barrier
    R m = R(0);
#pragma unroll 1
    for (int r = 0; r < xr; ++r) {
        const int j = j0 + r * t.rows + ty;
        // threads beyond the block's last full row (BLOCK not a multiple of
        // the row width) trace nothing
        const bool traced = ty < t.rows && j < P.n[1] && k < P.n[2] && i <= P.n[0];
        const long long c = traced ? P.soff + lcell(P, i, j, k) : 0;
        const bool out = traced && tx >= 1 && tx <= t.xw - 2 && i >= 0 && i < P.n[0];
        int *nreg = &s_nreg[r & 1];
        if (me == 0) *nreg = 0;
        // parabolic terms in float: the updated cell's L_P^(n+1/2) travels to
        // shared memory by cp.async while the cell is traced (its loads would
        // otherwise stall the update at the end)
        if constexpr (PSTAGE) {
            if (out) {
                const float *Lh = static_cast<const float *>(a.lph) + c;
#pragma unroll
                for (int q = 0; q < NPAR; ++q)
                    if (par_on(a, q)) cp_async(&sLp[q][me], Lh + q * a.sstride);
            }
            cp_async_commit();
        }
        // windows of this lane's face (plane i + 1), read ahead of the solves
        int w0 = 0, w1 = 0;
        if (traced && tx < t.xw - 1 && i <= P.n[0] - 1) {
            const int B = window_base(a, patch, 0);
            w0 = window_first(a, B, i + 1);
            w1 = window_first(a, B, i + 2);
        }
        if (traced) {
            R vs[5][NV];
#pragma unroll
            for (int mm = 0; mm < 5; ++mm)
#pragma unroll
                for (int q = 0; q < NV; ++q) vs[mm][q] = Vs[q * a.sstride + c + (mm - 2)];
            R Vp[NV], Vm[NV];
            fl |= trace_cell<PHYS, R, PPM, IFACE64, 0>(a, P, vs, L1, c, ch, dtdx, hdt, Vp, Vm);
#pragma unroll
            for (int q = 0; q < NV; ++q) { sP[me][q] = Vp[q]; sM[me][q] = Vm[q]; }
        }
        __syncthreads();
        if (traced && tx < t.xw - 1 && i <= P.n[0] - 1) {
            R L[NV], Rr[NV], F[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) { L[q] = sP[me][q]; Rr[q] = sM[me + 1][q]; }
            face_flux<PHYS, R, 0, recon_hllc(PPM)>(L, Rr, gam, ch, F,
                                                   recon_hybrid(PPM) && ((a.flags[c] | a.flags[c + 1]) & 1));
#pragma unroll
            for (int q = 0; q < NV; ++q) sF[me][q] = F[q];
            // faces on plane i+1; the tile's last face belongs to the next tile
            if (w1 > w0 && (tx < t.xw - 2 || i + 1 == P.n[0])) {
                const int slot = atomicAdd(nreg, 1);
                s_reg[slot][0] = me;
                s_reg[slot][1] = w0;
                s_reg[slot][2] = w1;
            }
        }
        __syncthreads();
        // the listed faces' register sums, one thread per (face, variable),
        // so that the float64 accumulation of a face is spread over lanes
        // instead of running on one lane of its warp
        {
            const int nr = *nreg;
            for (int it = me; it < nr * NV; it += BLOCK) {
                const int f = it / NV, q = it - f * NV;
                const int l = s_reg[f][0];
                const int jl = j0 + r * t.rows + l / t.xw;  // row of lane l; k is the block's
                register_face_var<R, 0>(a, P, s_reg[f][1], s_reg[f][2], jl, k, q, sF[l][q], dtd);
            }
        }
        if (LAST) {
            if (out) {
                const R ix = pidx<R>(P, 0);
                R s[NV];
                const int cl = lcell(P, i, j, k);
#pragma unroll
                for (int q = 0; q < NV; ++q) s[q] = (sF[me - 1][q] - sF[me][q]) * ix;
                if (a.ndim > 1) {  // A = the other directions' L, from the earlier sweeps
#pragma unroll
                    for (int q = 0; q < NV; ++q) s[q] = A[q * a.sstride + c] + s[q];
                }
                if constexpr (PSTAGE) {  // + L_P^(n+1/2) of the half-step fields
                    cp_async_wait_all();
#pragma unroll
                    for (int q = 0; q < NPAR; ++q)
                        if (par_on(a, q)) s[1 + q] += sLp[q][me];
                } else if constexpr (PAR) {
                    const R *Lh = static_cast<const R *>(a.lph) + c;
#pragma unroll
                    for (int q = 0; q < NPAR; ++q)
                        if (par_on(a, q)) s[1 + q] += Lh[q * a.sstride];
                }
                if constexpr (PHYS == PH_MHD && sizeof(R) == 4 && !IFACE64) {
                    double u0[NV];
                    R Vn[NV];
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        u0[q] = a.U[q * a.ustride + P.base + cl];
                        Vn[q] = Vs[q * a.sstride + c];
                    }
                    m = fmax(m, finish_cell_inc<R, PAR>(a, P, cl, s, u0, Vn, dtd, dtr, damp, fl));
                } else {
                    m = fmax(m, finish_cell<PHYS, R, IFACE64, PAR>(a, P, cl, s, dtd, damp, fl));
                }
            }
        } else if (out) {
            const R ix = pidx<R>(P, 0);
#pragma unroll
            for (int q = 0; q < NV; ++q) A[q * a.sstride + c] = (sF[me - 1][q] - sF[me][q]) * ix;
        }
    }
    if (LAST && a.nextmax) block_max_to<R>(m, a.nextmax);
    if (fl) atomicOr(a.status, fl);
}

// Shared-memory staging of the marching sweeps in float working precision.
// Per thread and stage: V of the cell entering the stencil (9 words), the
// transverse first-order divergences of the traced cell (2 dimensions x 9),
// and the running sum of the cell being updated (9); in the last sweep also
// that cell's float64 state U^n (9 doubles).  Two stages: the copies for the
// next cell are in flight while the current one is traced.  Slot k of thread
// t lies at [k * BLOCK + t], so a warp's accesses to one slot fall on
// consecutive banks.
constexpr int STG_V = 0, STG_F = 9, STG_A = 27, STG_N = 36;

// Role of a marching sweep in the step: the first writes A = L_D, a middle
// one adds L_D to A, the last one updates U (only when x is not swept, i.e.
// never in the standard order z, y, x).
enum { SW_MID = 0, SW_LAST = 1, SW_FIRST = 2 };

template <class R, int MODE> __host__ __device__ constexpr int sweep_m_smem()
{
    return sizeof(R) == 4 ? 2 * STG_N * BLOCK * 4 + (MODE == SW_LAST ? 2 * NV * BLOCK * 8 : 0) : 0;
}

// Sweep along D = 1 (y) or 2 (z): each thread marches one segment of SEG
// cells along D; the 5-cell stencil, the previous cell's + state and the
// previous face flux stay in registers.  A tile: xw lanes along x times
// BLOCK/xw (other-dimension, segment) pairs.  Float: the next cell's inputs
// are staged in shared memory by cp.async (sweep_m_smem bytes per block);
// double: they are prefetched into L1.
template <int PHYS, class R, int PPM, int IFACE64, int D, int MODE>
__global__ void __launch_bounds__(BLOCK, CTU_MARCH_MINB) k_sweep_m(StepArgs a, GroupTable gt, const R *Vs, const R *L1, R *A)
{
    constexpr int O = D == 1 ? 2 : 1;  // the other transverse dimension
    constexpr bool STAGED = sizeof(R) == 4;
    constexpr bool LAST = MODE == SW_LAST, FIRST = MODE == SW_FIRST;
    const Where wh = locate(gt);
    const int patch = wh.patch;
    const DevPatch P = a.patches[patch];
    const Tile t(wh.xw);
    const int SEGL = wh.seg;
    const int nD = P.n[D], nO = P.n[O];
    const int nseg = (nD + SEGL - 1) / SEGL;
    const int T0 = (P.n[0] + t.xw - 1) / t.xw;
    const int b = wh.b;
    const int x = (b % T0) * t.xw + t.tx();
    const int comb = (b / T0) * t.rows + t.ty();
    const int o = comb / nseg, seg = comb % nseg;
    const bool ok = x < P.n[0] && o < nO;
    const R gam = pgam<R>(a), ch = pch<R>(a.sp);
    const R dtr = pdt<R>(a.sp);
    const double dtd = a.sp->dt;
    const R dtdx = dtr * pidx<R>(P, D);
    const R hdt = R(0.5) * dtr;
    const R iD = pidx<R>(P, D);
    double damp = 1.0;
    if (LAST) damp = patch_damp(a, P);
    unsigned int fl = 0;
    R mx = R(0);
    if (ok) {
        const int j0 = seg * SEGL, j1 = min(j0 + SEGL, nD);
        const int st = dstr(P, D);
        int cc[3];
        cc[0] = x;
        cc[O] = o;
        cc[D] = j0 - 1;
        long long c = P.soff + lcell(P, cc[0], cc[1], cc[2]);  // traced cell j0 - 1
        R win[5][NV];
#pragma unroll
        for (int m = 0; m < 5; ++m)
#pragma unroll
            for (int q = 0; q < NV; ++q) win[m][q] = Vs[gperm<D>(q) * a.sstride + c + (m - 2) * st];
        R Pprev[NV], Fprev[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { Pprev[q] = R(0); Fprev[q] = R(0); }
        const int wb = window_base(a, patch, D);
        // face flux of plane j from Pprev (cell j - 1) and Vm (cell j); update
        // of cell j - 1 from the previous face flux, with its running sum A at
        // Ap[q * as] and (last sweep) its state U^n at Up[q * us]
        auto faces = [&](int j, long long cj, const R (&Vm)[NV], const R *Ap, long long as, const double *Up,
                         long long us) {
            R F[NV];
            face_flux<PHYS, R, D, recon_hllc(PPM)>(Pprev, Vm, gam, ch, F,
                                                   recon_hybrid(PPM) && ((a.flags[cj - st] | a.flags[cj]) & 1));
            // plane j; (a, b) = (x, o) are the two non-D dimensions in
            // increasing order; a segment's last face belongs to the next
            if (wb >= 0 && (j < j1 || j1 == nD)) {
                const int w0 = window_first(a, wb, j), w1 = window_first(a, wb, j + 1);
                register_face<R, D>(a, P, w0, w1, x, o, F, dtd);
            }
            if (j >= j0 + 1) {
                const long long cp = cj - st;  // cell j - 1
                R s[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) s[q] = (Fprev[q] - F[q]) * iD;
                if (LAST) {
                    double u[NV];
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        s[q] = Ap[q * as] + s[q];
                        u[q] = Up[q * us];
                    }
                    if constexpr (PHYS == PH_MHD && sizeof(R) == 4 && !IFACE64) {
                        R Vn[NV];  // V^n of cell j - 1, global order
#pragma unroll
                        for (int q = 0; q < NV; ++q) Vn[gperm<D>(q)] = win[1][q];
                        mx = fmax(mx, finish_cell_inc<R>(a, P, (int)(cp - P.soff), s, u, Vn, dtd, dtr, damp, fl));
                    } else {
                        mx = fmax(mx, finish_cell_u<PHYS, R, IFACE64>(a, P, (int)(cp - P.soff), s, u, dtd, damp, fl));
                    }
                } else if constexpr (FIRST) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) A[q * a.sstride + cp] = s[q];
                } else {
#pragma unroll
                    for (int q = 0; q < NV; ++q) A[q * a.sstride + cp] = Ap[q * as] + s[q];
                }
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) Fprev[q] = F[q];
        };
        if constexpr (STAGED) {
            extern __shared__ __align__(16) unsigned char sm_raw[];
            float *sf = reinterpret_cast<float *>(sm_raw) + threadIdx.x;
            double *sd = reinterpret_cast<double *>(sm_raw + 2 * STG_N * BLOCK * 4) + threadIdx.x;
            // copies for traced cell jn (scratch index cn) into stage sg
            auto issue = [&](int jn, long long cn, int sg) {
                float *bf = sf + sg * STG_N * BLOCK;
                if (jn > j0 - 1) {
#pragma unroll
                    for (int q = 0; q < NV; ++q)
                        cp_async(bf + (STG_V + q) * BLOCK, Vs + gperm<D>(q) * a.sstride + cn + 2 * st);
                }
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    if (e == D || e >= a.ndim) continue;
                    const int es = e < D ? e : e - 1;
                    const R *Le = L1 + (long long)e * NV * a.sstride + cn;
#pragma unroll
                    for (int q = 0; q < NV; ++q) cp_async(bf + (STG_F + es * 9 + q) * BLOCK, Le + q * a.sstride);
                }
                if (jn >= j0 + 1) {
                    if (!FIRST) {
#pragma unroll
                        for (int q = 0; q < NV; ++q) cp_async(bf + (STG_A + q) * BLOCK, A + q * a.sstride + cn - st);
                    }
                    if (LAST) {
                        double *bd = sd + sg * NV * BLOCK;
                        const long long gi = P.base + (cn - st - P.soff);
#pragma unroll
                        for (int q = 0; q < NV; ++q) cp_async(bd + q * BLOCK, a.U + q * a.ustride + gi);
                    }
                }
                cp_async_commit();
            };
            issue(j0 - 1, c, (j0 - 1) & 1);
            for (int j = j0 - 1; j <= j1; ++j, c += st) {
                const int sg = j & 1;
                // the stage written here was last read in iteration j - 1
                if (j < j1)
                    issue(j + 1, c + st, (j + 1) & 1);
                else
                    cp_async_commit();
                cp_async_wait_prev();
                const float *bf = sf + sg * STG_N * BLOCK;
                if (j > j0 - 1) {
#pragma unroll
                    for (int m = 0; m < 4; ++m)
#pragma unroll
                        for (int q = 0; q < NV; ++q) win[m][q] = win[m + 1][q];
#pragma unroll
                    for (int q = 0; q < NV; ++q) win[4][q] = bf[(STG_V + q) * BLOCK];
                }
                // half-step transverse increments, as in transverse()
                R T[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) T[q] = R(0);
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    if (e == D || e >= a.ndim) continue;
                    const int es = e < D ? e : e - 1;
#pragma unroll
                    for (int q = 0; q < NV; ++q) T[q] += bf[(STG_F + es * 9 + q) * BLOCK] * hdt;
                }
                R Vp[NV], Vm[NV];
                fl |= trace_cell_t<PHYS, R, PPM, IFACE64, D>(a, P, win, T, c, ch, dtdx, Vp, Vm);
                if (j >= j0) faces(j, c, Vm, bf + STG_A * BLOCK, BLOCK, sd + sg * NV * BLOCK, BLOCK);
#pragma unroll
                for (int q = 0; q < NV; ++q) Pprev[q] = Vp[q];
            }
        } else {
            for (int j = j0 - 1; j <= j1; ++j, c += st) {
                // prefetch what the next iteration reads: V(j+3), the transverse
                // first-order fluxes of cell j+1, the running sum (and the state)
                // of cell j
                if (j < j1) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) prefetch_l1(Vs + gperm<D>(q) * a.sstride + c + 3 * st);
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        if (e == D || e >= a.ndim) continue;
                        const R *Le = L1 + (long long)e * NV * a.sstride + c + st;
#pragma unroll
                        for (int q = 0; q < NV; ++q) prefetch_l1(Le + q * a.sstride);
                    }
                    if (j >= j0) {
#pragma unroll
                        for (int q = 0; q < NV; ++q) prefetch_l1(A + q * a.sstride + c);
                        if (LAST) {
#pragma unroll
                            for (int q = 0; q < NV; ++q) prefetch_l1(a.U + q * a.ustride + P.base + (c - P.soff));
                        }
                    }
                }
                if (j > j0 - 1) {
#pragma unroll
                    for (int m = 0; m < 4; ++m)
#pragma unroll
                        for (int q = 0; q < NV; ++q) win[m][q] = win[m + 1][q];
#pragma unroll
                    for (int q = 0; q < NV; ++q) win[4][q] = Vs[gperm<D>(q) * a.sstride + c + 2 * st];
                }
                R Vp[NV], Vm[NV];
                fl |= trace_cell<PHYS, R, PPM, IFACE64, D>(a, P, win, L1, c, ch, dtdx, hdt, Vp, Vm);
                if (j >= j0) faces(j, c, Vm, A + (c - st), a.sstride, a.U + P.base + (c - st - P.soff), a.ustride);
#pragma unroll
                for (int q = 0; q < NV; ++q) Pprev[q] = Vp[q];
            }
        }
    }
    if (LAST && a.nextmax) block_max_to<R>(mx, a.nextmax);
    if (fl) atomicOr(a.status, fl);
}

// ctu_dt: max over interior cells of max_d (|v_d| + c_f,d)/dx_d.
template <int PHYS, class R, int LIT64 = 0>
__global__ void __launch_bounds__(BLOCK) k_maxspeed(StepArgs a, GroupTable gt, unsigned long long *out)
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
        double U[NV];
        R V[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) U[q] = a.U[q * a.ustride + P.base + cl];
        const unsigned int f = prim_any<PHYS, R, LIT64>(U, a, V);
        if (f) atomicOr(a.status, f);
        m = cell_speed<PHYS, R>(V, a, P);
        if (a.par_cond | a.par_visc | a.par_res) {  // parabolic terms: + sum_d 2 D / dx_d^2
            // D = max((Gamma-1) max(kappa, kpar) / rho, (4/3) nu, eta)
            const R D = max(max((sizeof(R) == 8 ? (R)((a.gam - 1.0) * (a.kpar > a.kappa ? a.kpar : a.kappa))
                                                : (R)(a.gm1f * a.kmaxf)) / V[0],
                                R(4.0 / 3.0) * (sizeof(R) == 8 ? (R)a.nu : (R)a.nuf)),
                            sizeof(R) == 8 ? (R)a.eta : (R)a.etaf);
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (d < a.ndim) m += R(2) * D * (pidx<R>(P, d) * pidx<R>(P, d));
        }
    }
    block_max_to<R>(m, out);
}

} // namespace ctu
