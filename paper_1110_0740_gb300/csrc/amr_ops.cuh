// amr_ops.cuh -- the level operators around the CTU step, Section 4 of
// Mignone et al. (2012), Cartesian geometry, float64:
//   k_prolong   coarse-to-fine prolongation, Eq. (prolong), of the coarse
//               solution interpolated in time, Eq. (intalpha);
//   k_restrict  restriction (average down), Eq. (avgdown);
//   k_reflux    flux correction at coarse-fine interfaces from the flux
//               registers, Eq. (fluxcorr) and Eq. (addreflux).
// All three are data-parallel and HBM-bound: one thread per output cell
// (prolongation, restriction) or coarse face (reflux), a grid-stride loop
// over a box of cells, blockIdx.y = box.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ctu.h"

namespace ctu {

constexpr int AMR_BLOCK = 256;
constexpr int AMR_NG = 4;

struct AmrGeom {
    int n[3];
    int ndim;
    __device__ __forceinline__ long long cell(int x, int y, int z) const
    {
        const int g1 = ndim > 1 ? AMR_NG : 0, g2 = ndim > 2 ? AMR_NG : 0;
        const long long N0 = n[0] + 2 * AMR_NG, N1 = n[1] + 2 * g1;
        return ((long long)(z + g2) * N1 + (y + g1)) * N0 + (x + AMR_NG);
    }
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Monotonised-central slope, Eq. (MClim): for dm, dp of one sign that sign
// times min(|dm + dp|/2, 2|dm|, 2|dp|), else 0.
__device__ __forceinline__ double mc64(double dm, double dp)
{
    const double m = fmin(0.5 * fabs(dm + dp), 2.0 * fmin(fabs(dm), fabs(dp)));
    const bool same = (dm > 0.0 && dp > 0.0) || (dm < 0.0 && dp < 0.0);
    return same ? copysign(m, dm) : 0.0;
}

// Eq. (prolong) with Eq. (intalpha): fine cell x of the box takes
// U* = (1 - alpha) U_old + alpha U_new of its coarse cell c = origin +
// floor(x / r), plus, along each active dimension d, w_d times the
// MC-limited central difference of U* there, w_d = ((x_d mod r) + 1/2)/r - 1/2
// (the volume-coordinate ratio of Eq. prolong for Cartesian cells).
__global__ void __launch_bounds__(AMR_BLOCK) k_prolong(const ctu_level_box *boxes, int ndim, const double *Uco,
                                                        const double *Ucn, long long cs, double alpha, double *Uf,
                                                        long long fs)
{
    const ctu_level_box B = boxes[blockIdx.y];
    const AmrGeom gc{{B.cn[0], B.cn[1], B.cn[2]}, ndim}, gf{{B.fn[0], B.fn[1], B.fn[2]}, ndim};
    const int e0 = B.hi[0] - B.lo[0], e1 = B.hi[1] - B.lo[1], e2 = B.hi[2] - B.lo[2];
    const long long cnt = (long long)e0 * e1 * e2;
    const double beta = 1.0 - alpha;
    for (long long t = (long long)blockIdx.x * AMR_BLOCK + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * AMR_BLOCK) {
        const int xf[3] = {B.lo[0] + (int)(t % e0), B.lo[1] + (int)((t / e0) % e1), B.lo[2] + (int)(t / ((long long)e0 * e1))};
        int c[3];
        double w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d < ndim) {
                const int fl = floordiv(xf[d], B.ratio);
                c[d] = B.origin[d] + fl;
                w[d] = ((xf[d] - B.ratio * fl) + 0.5) / B.ratio - 0.5;
            } else {
                c[d] = 0;
                w[d] = 0.0;
            }
        }
        const long long fi = B.fbase + gf.cell(xf[0], xf[1], xf[2]);
        const long long c0 = B.cbase + gc.cell(c[0], c[1], c[2]);
        long long cm[3], cp[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const long long st = d == 0 ? 1 : (d == 1 ? gc.cell(0, 1, 0) - gc.cell(0, 0, 0) : gc.cell(0, 0, 1) - gc.cell(0, 0, 0));
            cm[d] = c0 - st;
            cp[d] = c0 + st;
        }
#pragma unroll 1
        for (int q = 0; q < 9; ++q) {
            const double *Po = Uco + q * cs, *Pn = Ucn + q * cs;
            const double u0 = beta * Po[c0] + alpha * Pn[c0];
            double u = u0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d >= ndim) continue;
                const double um = beta * Po[cm[d]] + alpha * Pn[cm[d]];
                const double up = beta * Po[cp[d]] + alpha * Pn[cp[d]];
                u += w[d] * mc64(u0 - um, up - u0);
            }
            Uf[q * fs + fi] = u;
        }
    }
}

// Eq. (avgdown): coarse cell c of the box becomes the mean of its r^ndim
// fine cells (c - origin) r + k (Cartesian: equal volumes), summed with the
// innermost index along x.
__global__ void __launch_bounds__(AMR_BLOCK) k_restrict(const ctu_level_box *boxes, int ndim, double *Uc,
                                                         long long cs, const double *Uf, long long fs)
{
    const ctu_level_box B = boxes[blockIdx.y];
    const AmrGeom gc{{B.cn[0], B.cn[1], B.cn[2]}, ndim}, gf{{B.fn[0], B.fn[1], B.fn[2]}, ndim};
    const int e0 = B.hi[0] - B.lo[0], e1 = B.hi[1] - B.lo[1], e2 = B.hi[2] - B.lo[2];
    const long long cnt = (long long)e0 * e1 * e2;
    const int r = B.ratio, k1 = ndim > 1 ? r : 1, k2 = ndim > 2 ? r : 1;
    const double nk = (double)r * k1 * k2;
    for (long long t = (long long)blockIdx.x * AMR_BLOCK + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * AMR_BLOCK) {
        const int x = B.lo[0] + (int)(t % e0), y = B.lo[1] + (int)((t / e0) % e1),
                  z = B.lo[2] + (int)(t / ((long long)e0 * e1));
        const long long ci = B.cbase + gc.cell(x, y, z);
#pragma unroll 1
        for (int q = 0; q < 9; ++q) {
            double s = 0.0;
            for (int c2 = 0; c2 < k2; ++c2)
                for (int c1 = 0; c1 < k1; ++c1)
                    for (int c0 = 0; c0 < r; ++c0) {
                        const int fx = (x - B.origin[0]) * r + c0;
                        const int fy = ndim > 1 ? (y - B.origin[1]) * r + c1 : 0;
                        const int fz = ndim > 2 ? (z - B.origin[2]) * r + c2 : 0;
                        s += Uf[q * fs + B.fbase + gf.cell(fx, fy, fz)];
                    }
            Uc[q * cs + ci] = s / nk;
        }
    }
}

// Eq. (fluxcorr) + Eq. (addreflux): coarse face (a, b) of the set collects
// its coarse register sum (bound with weight -1) and the sums of its r^2 fine
// faces (weight +1); the coarse cell beside it gains side x that total over
// its volume.  A coarse cell next to several interfaces receives several
// corrections, so the addition is atomic.
__global__ void __launch_bounds__(AMR_BLOCK) k_reflux(const ctu_reflux_set *sets, int ndim, double *Uc, long long cs,
                                                       const double *reg)
{
    const ctu_reflux_set S = sets[blockIdx.y];
    const AmrGeom gc{{S.cn[0], S.cn[1], S.cn[2]}, ndim};
    const int ea = S.dir == 0 ? 1 : 0, eb = S.dir == 2 ? 1 : 2;
    const int ra = ea < ndim ? S.ratio : 1, rb = eb < ndim ? S.ratio : 1;
    double vol = 1.0;
    for (int d = 0; d < ndim; ++d) vol *= S.dx[d];
    const long long na = S.a1 - S.a0, nb = S.b1 - S.b0;
    const long long cnt = na * nb;
    for (long long t = (long long)blockIdx.x * AMR_BLOCK + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * AMR_BLOCK) {
        const int a = S.a0 + (int)(t % na), b = S.b0 + (int)(t / na);
        int c[3];
        c[S.dir] = S.side > 0 ? S.plane : S.plane - 1;
        c[ea] = a;
        c[eb] = b;
        const long long ci = S.cbase + gc.cell(c[0], c[1], c[2]);
#pragma unroll 1
        for (int q = 0; q < 9; ++q) {
            double tot = reg[S.creg + q * na * nb + (long long)(b - S.b0) * na + (a - S.a0)];
            for (int j = 0; j < rb; ++j)
                for (int i = 0; i < ra; ++i) {
                    const long long fa = S.fa0 + (long long)(a - S.a0) * ra + i;
                    const long long fb = S.fb0 + (long long)(b - S.b0) * rb + j;
                    tot += reg[S.freg + q * (long long)S.fna * S.fnb + fb * S.fna + fa];
                }
            atomicAdd(Uc + q * cs + ci, S.side * tot / vol);
        }
    }
}

} // namespace ctu
