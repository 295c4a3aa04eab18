// amr_ops.cuh -- the level operators around the CTU step, Section 4 of
// Mignone et al. (2012), Cartesian geometry, float64:
//   k_prolong   coarse-to-fine prolongation, Eq. (prolong), of the coarse
//               solution interpolated in time, Eq. (intalpha);
//   k_restrict  restriction (average down), Eq. (avgdown);
//   k_reflux    flux correction at coarse-fine interfaces from the flux
//               registers, Eq. (fluxcorr) and Eq. (addreflux).
// All three are data-parallel and HBM-bound: one thread per coarse cell
// (prolongation: its children inside the box; restriction: the cell) or
// coarse face (reflux); the blocks of a launch are spread over the boxes in
// proportion to their work (BlockMap).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ctu.h"
#include "ctu_kernels.cuh"

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
// times min(|dm + dp|/2, 2|dm|, 2|dp|), else 0.  Non-negative float64
// values order like their bit patterns, so the minima, absolute values and
// sign tests run as integer operations; only the sum and the two exact
// scalings by 1/2 and 2 use the FP64 pipe (GB300 issues 2 FP64 operations
// per SM and cycle).
__device__ __forceinline__ double mc64(double dm, double dp)
{
    const long long bm = __double_as_longlong(dm), bp = __double_as_longlong(dp);
    const long long am = bm & 0x7FFFFFFFFFFFFFFFll, ap = bp & 0x7FFFFFFFFFFFFFFFll;
    const bool same = ((bm ^ bp) >= 0) && am != 0 && ap != 0;
    const double h = 0.5 * __longlong_as_double(__double_as_longlong(dm + dp) & 0x7FFFFFFFFFFFFFFFll);
    const double t = 2.0 * __longlong_as_double(am < ap ? am : ap);
    const long long bh = __double_as_longlong(h), bt = __double_as_longlong(t);
    const long long m = bh < bt ? bh : bt;
    return same ? __longlong_as_double(m | (bm & (long long)0x8000000000000000ull)) : 0.0;
}

// Blocks of a launch are spread over its boxes in proportion to their work:
// block b serves box blk_box[b], as its (b - box_start[box])-th block.
struct BlockMap {
    const int *box_start;
    const int *blk_box;
    __device__ __forceinline__ void locate(int &box, long long &first) const
    {
        box = blk_box[blockIdx.x];
        first = (long long)(blockIdx.x - box_start[box]) * AMR_BLOCK + threadIdx.x;
    }
};

// Eq. (prolong) with Eq. (intalpha): fine cell x of the box takes
// U* = (1 - alpha) U_old + alpha U_new of its coarse cell c = origin +
// floor(x / r), plus, along each active dimension d, w_d times the
// MC-limited central difference of U* there, w_d = ((x_d mod r) + 1/2)/r - 1/2
// (the volume-coordinate ratio of Eq. prolong for Cartesian cells).  One
// thread per coarse cell under the box: U* and its slopes are formed once
// and written to the cell's children inside the box.
template <bool BLEND>
__global__ void __launch_bounds__(AMR_BLOCK) k_prolong(const ctu_level_box *boxes, BlockMap map, int ndim,
                                                        const double *Uco, const double *Ucn, long long cs,
                                                        double alpha, double *Uf, long long fs)
{
    int bi;
    long long t;
    map.locate(bi, t);
    const ctu_level_box B = boxes[bi];
    const AmrGeom gc{{B.cn[0], B.cn[1], B.cn[2]}, ndim}, gf{{B.fn[0], B.fn[1], B.fn[2]}, ndim};
    const int r = B.ratio;
    int clo[3], ce[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d < ndim) {
            clo[d] = floordiv(B.lo[d], r);
            ce[d] = floordiv(B.hi[d] - 1, r) + 1 - clo[d];
        } else {
            clo[d] = 0;
            ce[d] = 1;
        }
    }
    if (t >= (long long)ce[0] * ce[1] * ce[2]) return;
    const int cr[3] = {clo[0] + (int)(t % ce[0]), clo[1] + (int)((t / ce[0]) % ce[1]),
                       clo[2] + (int)(t / ((long long)ce[0] * ce[1]))};  // coarse cell, fine-patch frame
    const long long c0 = B.cbase + gc.cell(B.origin[0] + cr[0], ndim > 1 ? B.origin[1] + cr[1] : 0,
                                           ndim > 2 ? B.origin[2] + cr[2] : 0);
    const long long st[3] = {1, gc.cell(0, 1, 0) - gc.cell(0, 0, 0), gc.cell(0, 0, 1) - gc.cell(0, 0, 0)};
    const double beta = 1.0 - alpha;
    const double ir = 1.0 / r;
    // children of this coarse cell inside the box, their weights per
    // dimension and their fine cell offsets
    int k0[3], k1[3];
    double w[3][4];  // ratio <= 4
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int f0 = d < ndim ? cr[d] * r : 0;
        const int fe = d < ndim ? r : 1;
        k0[d] = max(f0, B.lo[d]);
        k1[d] = min(f0 + fe, B.hi[d]);
#pragma unroll
        for (int m = 0; m < 4; ++m) w[d][m] = d < ndim ? ((k0[d] - f0 + m) + 0.5) * ir - 0.5 : 0.0;
    }
    const long long f00 = B.fbase + gf.cell(k0[0], k0[1], k0[2]);
    const long long fsy = gf.cell(0, 1, 0) - gf.cell(0, 0, 0), fsz = gf.cell(0, 0, 1) - gf.cell(0, 0, 0);
    const int nx = k1[0] - k0[0], ny = k1[1] - k0[1], nz = k1[2] - k0[2];
#pragma unroll 1
    for (int q = 0; q < 9; ++q) {
        const double *Po = Uco + q * cs, *Pn = Ucn + q * cs;
        // U* at an offset from c0: blended, or (alpha 0 or 1) the one state
        auto ustar = [&](long long o) { return BLEND ? beta * Po[o] + alpha * Pn[o] : Po[o]; };
        const double u0 = ustar(c0);
        double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= ndim) continue;
            // a coarse cell touching the domain boundary: the one-sided
            // difference to its neighbour inside the domain (Section 4)
            const int cd = B.origin[d] + cr[d];
            const bool at_lo = ((B.phys >> (2 * d)) & 1) && cd == 0;
            const bool at_hi = ((B.phys >> (2 * d + 1)) & 1) && cd == B.cn[d] - 1;
            if (at_lo && at_hi) {
                s[d] = 0.0;
            } else if (at_lo) {
                s[d] = ustar(c0 + st[d]) - u0;
            } else if (at_hi) {
                s[d] = u0 - ustar(c0 - st[d]);
            } else {
                const double um = ustar(c0 - st[d]);
                const double up = ustar(c0 + st[d]);
                s[d] = mc64(u0 - um, up - u0);
            }
        }
        double *Pf = Uf + q * fs + f00;
        for (int z = 0; z < nz; ++z) {
            const double uz = u0 + w[2][z] * s[2];
            for (int y = 0; y < ny; ++y) {
                const double uy = uz + w[1][y] * s[1];
                double *row = Pf + z * fsz + y * fsy;
                for (int x = 0; x < nx; ++x) row[x] = uy + w[0][x] * s[0];
            }
        }
    }
}

// Eq. (avgdown): coarse cell c of the box becomes the mean of its r^ndim
// fine cells (c - origin) r + k (Cartesian: equal volumes), summed with the
// innermost index along x.
__global__ void __launch_bounds__(AMR_BLOCK) k_restrict(const ctu_level_box *boxes, BlockMap map, int ndim,
                                                         double *Uc, long long cs, const double *Uf, long long fs)
{
    int bi;
    long long t;
    map.locate(bi, t);
    const ctu_level_box B = boxes[bi];
    const AmrGeom gc{{B.cn[0], B.cn[1], B.cn[2]}, ndim}, gf{{B.fn[0], B.fn[1], B.fn[2]}, ndim};
    const int e0 = B.hi[0] - B.lo[0], e1 = B.hi[1] - B.lo[1], e2 = B.hi[2] - B.lo[2];
    const long long cnt = (long long)e0 * e1 * e2;
    const int r = B.ratio, k1 = ndim > 1 ? r : 1, k2 = ndim > 2 ? r : 1;
    const double nk = (double)r * k1 * k2;
    // dividing by a power of two is multiplying by its exact reciprocal
    const bool pow2 = (r & (r - 1)) == 0;
    const double ink = 1.0 / nk;
    if (t < cnt) {
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
            Uc[q * cs + ci] = pow2 ? s * ink : s / nk;
        }
    }
}

// Eq. (fluxcorr) + Eq. (addreflux): coarse face (a, b) of the set collects
// its coarse register sum (bound with weight -1) and the sums of its r^2 fine
// faces (weight +1); the coarse cell beside it gains side x that total over
// its volume.  A coarse cell next to several interfaces receives several
// corrections, so the addition is atomic.
__global__ void __launch_bounds__(AMR_BLOCK) k_reflux(const ctu_reflux_set *sets, BlockMap map, int ndim, double *Uc,
                                                       long long cs, const double *reg)
{
    int si;
    long long t;
    map.locate(si, t);
    const ctu_reflux_set S = sets[si];
    const AmrGeom gc{{S.cn[0], S.cn[1], S.cn[2]}, ndim};
    const int ea = S.dir == 0 ? 1 : 0, eb = S.dir == 2 ? 1 : 2;
    const int ra = ea < ndim ? S.ratio : 1, rb = eb < ndim ? S.ratio : 1;
    double vol = 1.0;
    for (int d = 0; d < ndim; ++d) vol *= S.dx[d];
    const long long na = S.a1 - S.a0, nb = S.b1 - S.b0;
    const long long cnt = na * nb;
    if (t < cnt) {
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

// Conservation diagnostics of a batch: out[q] += U_q x cell volume over the
// interior cells (q = 0..8), out[9] = max |div B| with central differences
// (as the bits of a non-negative float64, which order like the values).
// blockIdx.y = patch; per block a shared-memory reduction, then one atomic
// per quantity.
__global__ void __launch_bounds__(AMR_BLOCK) k_diagnostics(const DevPatch *patches, int ndim, const double *U,
                                                            long long us, double *out)
{
    const DevPatch P = patches[blockIdx.y];
    const AmrGeom g{{P.n[0], P.n[1], P.n[2]}, ndim};
    const long long cnt = (long long)P.n[0] * P.n[1] * P.n[2];
    double vol = 1.0;
    for (int d = 0; d < ndim; ++d) vol *= P.dx[d];
    double acc[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = 0.0;
    for (long long t = (long long)blockIdx.x * AMR_BLOCK + threadIdx.x; t < cnt;
         t += (long long)gridDim.x * AMR_BLOCK) {
        const int x = (int)(t % P.n[0]), y = (int)((t / P.n[0]) % P.n[1]),
                  z = (int)(t / ((long long)P.n[0] * P.n[1]));
        const long long c = P.base + g.cell(x, y, z);
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] += U[q * us + c] * vol;
        double div = 0.0;
        for (int d = 0; d < ndim; ++d) {
            const long long st = d == 0 ? 1 : (d == 1 ? (long long)P.N[0] : (long long)P.N[0] * P.N[1]);
            div += (U[(5 + d) * us + c + st] - U[(5 + d) * us + c - st]) / (2.0 * P.dx[d]);
        }
        acc[9] = fmax(acc[9], fabs(div));
    }
    __shared__ double red[10][AMR_BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = q < 9 ? v + w : fmax(v, w);
        }
        if (lane == 0) red[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        const int q = threadIdx.x;
        double v = red[q][0];
        for (int k = 1; k < AMR_BLOCK / 32; ++k) v = q < 9 ? v + red[q][k] : fmax(v, red[q][k]);
        if (q < 9)
            atomicAdd(out + q, v);
        else
            atomicMax((unsigned long long *)(out + 9), (unsigned long long)__double_as_longlong(v));
    }
}

// Same-level ghost exchange: one thread per destination cell of a box, all
// nine variables; MODE 0 copies pool to pool, 1 packs the source cells into
// a buffer ([q][z][y][x] per box, boxes one after another), 2 unpacks a
// buffer into the destination cells.  HBM-bound: 72 B read and 72 B written
// per cell.
struct CopyDesc {
    int dn[3], sn[3], lo[3], ext[3], shift[3], pad;
    long long dbase, sbase, boff;
};

template <int MODE>
__global__ void __launch_bounds__(AMR_BLOCK) k_copy(const CopyDesc *boxes, BlockMap map, int ndim, double *Ud,
                                                     long long ds, const double *Us, long long ss)
{
    int bi;
    long long t;
    map.locate(bi, t);
    const CopyDesc B = boxes[bi];
    const long long nc = (long long)B.ext[0] * B.ext[1] * B.ext[2];
    if (t >= nc) return;
    const unsigned t32 = (unsigned)t, row = t32 / (unsigned)B.ext[0];
    const unsigned zz = row / (unsigned)B.ext[1];
    const int x = B.lo[0] + (int)(t32 - row * (unsigned)B.ext[0]);
    const int y = B.lo[1] + (int)(row - zz * (unsigned)B.ext[1]), z = B.lo[2] + (int)zz;
    if (MODE == 0 || MODE == 1) {
        const AmrGeom gs{{B.sn[0], B.sn[1], B.sn[2]}, ndim};
        const long long si = B.sbase + gs.cell(x + B.shift[0], y + B.shift[1], z + B.shift[2]);
        if (MODE == 0) {
            const AmrGeom gd{{B.dn[0], B.dn[1], B.dn[2]}, ndim};
            const long long di = B.dbase + gd.cell(x, y, z);
#pragma unroll
            for (int q = 0; q < 9; ++q) Ud[q * ds + di] = Us[q * ss + si];
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) Ud[B.boff + q * nc + t] = Us[q * ss + si];
        }
    } else {
        const AmrGeom gd{{B.dn[0], B.dn[1], B.dn[2]}, ndim};
        const long long di = B.dbase + gd.cell(x, y, z);
#pragma unroll
        for (int q = 0; q < 9; ++q) Ud[q * ds + di] = Us[B.boff + q * nc + t];
    }
}

} // namespace ctu
