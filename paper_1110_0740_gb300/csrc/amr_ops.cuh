// amr_ops.cuh -- the level operators around the CTU step, Section 4 of
// Mignone et al. (2012), Cartesian geometry, float64:
//   k_prolong   coarse-to-fine prolongation, Eq. (prolong), of the coarse
//               solution interpolated in time, Eq. (intalpha);
//   k_restrict  restriction (average down), Eq. (avgdown);
//   k_reflux    flux correction at coarse-fine interfaces from the flux
//               registers, Eq. (fluxcorr) and Eq. (addreflux).
// All three are data-parallel: one thread per variable and coarse cell
// (prolongation: the cell's children inside the box), per coarse cell
// (restriction, all nine variables) or per variable and coarse face
// (reflux); the blocks of a launch are spread over the boxes in proportion
// to their work (BlockMap).
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
    // block blk of the table (a launch over part of it passes its first block)
    __device__ __forceinline__ void locate(int &box, long long &first, unsigned blk) const
    {
        box = blk_box[blk];
        first = (long long)(blk - box_start[box]) * AMR_BLOCK + threadIdx.x;
    }
    __device__ __forceinline__ void locate(int &box, long long &first) const { locate(box, first, blockIdx.x); }
};

// Eq. (prolong) with Eq. (intalpha): fine cell x of the box takes
// U* = (1 - alpha) U_old + alpha U_new of its coarse cell c = origin +
// floor(x / r), plus, along each active dimension d, w_d times the
// MC-limited central difference of U* there, w_d = ((x_d mod r) + 1/2)/r - 1/2
// (the volume-coordinate ratio of Eq. prolong for Cartesian cells).  One
// thread per (variable, coarse cell under the box): U* and its slopes are
// formed once and written to the cell's children inside the box.  The cells
// of one variable are adjacent threads (the boxes of a ghost shell are
// small: packing the nine variables of a box fills the warps), and the index
// arithmetic is 32-bit (the host keeps 9 x the cells of a box below 2^31).
template <bool BLEND>
__global__ void __launch_bounds__(AMR_BLOCK) k_prolong(const ctu_level_box *boxes, BlockMap map, int ndim,
                                                        const double *Uco, const double *Ucn, long long cs,
                                                        double alpha, double *Uf, long long fs)
{
    int bi;
    long long tl;
    map.locate(bi, tl);
    const ctu_level_box *B = boxes + bi;
    const int r = B->ratio;
    // w_s[j]: weight of a child j cells into its parent along an active
    // dimension, (j + 1/2)/r - 1/2; the threads of a block serve one box
    __shared__ double w_s[4];
    if (threadIdx.x < (unsigned)r) w_s[threadIdx.x] = ((int)threadIdx.x + 0.5) * (1.0 / r) - 0.5;
    __syncthreads();
    const unsigned t = (unsigned)tl;
    const bool a1 = ndim > 1, a2 = ndim > 2;
    const int lo0 = B->lo[0], lo1 = B->lo[1], lo2 = B->lo[2];
    const int hi0 = B->hi[0], hi1 = B->hi[1], hi2 = B->hi[2];
    // coarse cells under the box, fine-patch frame
    const int clo0 = floordiv(lo0, r), clo1 = a1 ? floordiv(lo1, r) : 0, clo2 = a2 ? floordiv(lo2, r) : 0;
    const unsigned ce0 = floordiv(hi0 - 1, r) + 1 - clo0, ce1 = a1 ? floordiv(hi1 - 1, r) + 1 - clo1 : 1,
                   ce2 = a2 ? floordiv(hi2 - 1, r) + 1 - clo2 : 1;
    const unsigned cc = ce0 * ce1 * ce2;
    if (t >= 9u * cc) return;
    const unsigned q = t / cc, u = t - q * cc;
    const unsigned row = u / ce0, zz = row / ce1;
    const int cr0 = clo0 + (int)(u - row * ce0), cr1 = clo1 + (int)(row - zz * ce1), cr2 = clo2 + (int)zz;
    const AmrGeom gc{{B->cn[0], B->cn[1], B->cn[2]}, ndim}, gf{{B->fn[0], B->fn[1], B->fn[2]}, ndim};
    const int o0 = B->origin[0] + cr0, o1 = a1 ? B->origin[1] + cr1 : 0, o2 = a2 ? B->origin[2] + cr2 : 0;
    const long long c0 = B->cbase + gc.cell(o0, o1, o2);
    const long long sy = gc.cell(0, 1, 0) - gc.cell(0, 0, 0), sz = gc.cell(0, 0, 1) - gc.cell(0, 0, 0);
    const double beta = 1.0 - alpha;
    const double *Po = Uco + q * cs, *Pn = Ucn + q * cs;
    // U* at an offset from c0: blended, or (alpha 0 or 1) the one state
    auto ustar = [&](long long o) { return BLEND ? beta * Po[o] + alpha * Pn[o] : Po[o]; };
    const double u0 = ustar(c0);
    // the MC slope along one active dimension; a coarse cell touching the
    // domain boundary takes the one-sided difference to its neighbour inside
    // the domain (Section 4)
    const int phys = B->phys;
    auto slope = [&](int d, int cd, int cn, long long st) {
        const bool at_lo = ((phys >> (2 * d)) & 1) && cd == 0;
        const bool at_hi = ((phys >> (2 * d + 1)) & 1) && cd == cn - 1;
        if (at_lo && at_hi) return 0.0;
        if (at_lo) return ustar(c0 + st) - u0;
        if (at_hi) return u0 - ustar(c0 - st);
        const double um = ustar(c0 - st);
        const double up = ustar(c0 + st);
        return mc64(u0 - um, up - u0);
    };
    const double s0 = slope(0, o0, B->cn[0], 1);
    const double s1 = a1 ? slope(1, o1, B->cn[1], sy) : 0.0;
    const double s2 = a2 ? slope(2, o2, B->cn[2], sz) : 0.0;
    // children of this coarse cell inside the box
    const int f0 = cr0 * r, f1 = a1 ? cr1 * r : 0, f2 = a2 ? cr2 * r : 0;
    const int k00 = max(f0, lo0), k01 = max(f1, lo1), k02 = max(f2, lo2);
    const int nx = min(f0 + r, hi0) - k00, ny = min(f1 + (a1 ? r : 1), hi1) - k01,
              nz = min(f2 + (a2 ? r : 1), hi2) - k02;
    const long long fsy = gf.cell(0, 1, 0) - gf.cell(0, 0, 0), fsz = gf.cell(0, 0, 1) - gf.cell(0, 0, 0);
    double *Pf = Uf + q * fs + B->fbase + gf.cell(k00, k01, k02);
    for (int z = 0; z < nz; ++z) {
        const double uz = u0 + (a2 ? w_s[k02 - f2 + z] : 0.0) * s2;
        for (int y = 0; y < ny; ++y) {
            const double uy = uz + (a1 ? w_s[k01 - f1 + y] : 0.0) * s1;
            double *row_ = Pf + z * fsz + y * fsy;
            for (int x = 0; x < nx; ++x) row_[x] = uy + w_s[k00 - f0 + x] * s0;
        }
    }
}

// Eq. (avgdown): coarse cell c of the box becomes the mean of its r^ndim
// fine cells (c - origin) r + k (Cartesian: equal volumes), summed with the
// innermost index along x.  One thread per coarse cell and all nine
// variables (the children's offsets formed once), 32-bit index arithmetic.
__global__ void __launch_bounds__(AMR_BLOCK) k_restrict(const ctu_level_box *boxes, BlockMap map, int ndim,
                                                         double *Uc, long long cs, const double *Uf, long long fs)
{
    int bi;
    long long tl;
    map.locate(bi, tl);
    const unsigned t = (unsigned)tl;
    const ctu_level_box *B = boxes + bi;
    const unsigned e0 = B->hi[0] - B->lo[0], e1 = B->hi[1] - B->lo[1], e2 = B->hi[2] - B->lo[2];
    if (t >= e0 * e1 * e2) return;
    const unsigned row = t / e0, zz = row / e1;
    const int x = B->lo[0] + (int)(t - row * e0), y = B->lo[1] + (int)(row - zz * e1), z = B->lo[2] + (int)zz;
    const int r = B->ratio, k1 = ndim > 1 ? r : 1, k2 = ndim > 2 ? r : 1;
    const double nk = (double)r * k1 * k2;
    // dividing by a power of two is multiplying by its exact reciprocal
    const bool pow2 = (r & (r - 1)) == 0;
    const double ink = 1.0 / nk;
    const AmrGeom gc{{B->cn[0], B->cn[1], B->cn[2]}, ndim}, gf{{B->fn[0], B->fn[1], B->fn[2]}, ndim};
    const long long ci = B->cbase + gc.cell(x, y, z);
    const int fx0 = (x - B->origin[0]) * r, fy0 = ndim > 1 ? (y - B->origin[1]) * r : 0,
              fz0 = ndim > 2 ? (z - B->origin[2]) * r : 0;
    const long long fsy = gf.cell(0, 1, 0) - gf.cell(0, 0, 0), fsz = gf.cell(0, 0, 1) - gf.cell(0, 0, 0);
    const double *P = Uf + B->fbase + gf.cell(fx0, fy0, fz0);
    const bool r2x3 = r == 2 && k2 == 2;  // 3-D, ratio 2: the eight children unrolled, same order
#pragma unroll 3
    for (int q = 0; q < 9; ++q) {
        const double *Pq = P + q * fs;
        double s = 0.0;
        if (r2x3) {
            s += Pq[0];
            s += Pq[1];
            s += Pq[fsy];
            s += Pq[fsy + 1];
            s += Pq[fsz];
            s += Pq[fsz + 1];
            s += Pq[fsz + fsy];
            s += Pq[fsz + fsy + 1];
        } else {
            for (int c2 = 0; c2 < k2; ++c2)
                for (int c1 = 0; c1 < k1; ++c1)
                    for (int c0 = 0; c0 < r; ++c0) s += Pq[c2 * fsz + c1 * fsy + c0];
        }
        Uc[q * cs + ci] = pow2 ? s * ink : s / nk;
    }
}

// Eq. (fluxcorr) + Eq. (addreflux): coarse face (a, b) of the set collects
// its coarse register sum (bound with weight -1) and the sums of its r^2 fine
// faces (weight +1); the coarse cell beside it gains side x that total over
// its volume.  One launch covers the sets of one class (direction, side),
// blocks blk0 onwards of the table: the sets of a class reach disjoint
// coarse cells when the fine patches are disjoint, and a cell next to several
// interfaces takes their corrections in the fixed order of the class
// launches, so the result does not depend on scheduling.  The addition stays
// atomic so that sets sharing a cell within a class still all land.  One
// thread per (variable, face), the faces of a variable adjacent.
__global__ void __launch_bounds__(AMR_BLOCK) k_reflux(const ctu_reflux_set *sets, BlockMap map, unsigned blk0,
                                                       int ndim, double *Uc, long long cs, const double *reg)
{
    int si;
    long long tl;
    map.locate(si, tl, blk0 + blockIdx.x);
    const unsigned t = (unsigned)tl;
    const ctu_reflux_set *S = sets + si;
    const unsigned na = S->a1 - S->a0, nb = S->b1 - S->b0, cnt = na * nb;
    if (t >= 9u * cnt) return;
    const unsigned q = t / cnt, f = t - q * cnt;
    const unsigned fb_ = f / na;
    const int a = S->a0 + (int)(f - fb_ * na), b = S->b0 + (int)fb_;
    const int dir = S->dir;
    const int ea = dir == 0 ? 1 : 0, eb = dir == 2 ? 1 : 2;
    const int ra = ea < ndim ? S->ratio : 1, rb = eb < ndim ? S->ratio : 1;
    const double vol = S->dx[0] * (ndim > 1 ? S->dx[1] : 1.0) * (ndim > 2 ? S->dx[2] : 1.0);
    const AmrGeom gc{{S->cn[0], S->cn[1], S->cn[2]}, ndim};
    const int cp = S->side > 0 ? S->plane : S->plane - 1;  // the coarse cell's index along dir
    const long long ci = S->cbase + gc.cell(dir == 0 ? cp : a, dir == 1 ? cp : (dir == 0 ? a : b),
                                            dir == 2 ? cp : b);
    double tot = reg[S->creg + (long long)(q * cnt + f)];
    const long long fna = S->fna;
    const double *Fr = reg + S->freg + q * (fna * S->fnb);
    for (int j = 0; j < rb; ++j)
        for (int i = 0; i < ra; ++i) {
            const long long fa = S->fa0 + (long long)(a - S->a0) * ra + i;
            const long long fb = S->fb0 + (long long)(b - S->b0) * rb + j;
            tot += Fr[fb * fna + fa];
        }
    atomicAdd(Uc + q * cs + ci, S->side * tot / vol);
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
