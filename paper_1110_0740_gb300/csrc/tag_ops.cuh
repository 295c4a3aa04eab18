// tag_ops.cuh -- refinement tagging, Eq. (RefCrit) of Mignone et al. (2012),
// Section 4 (refinement criteria): the second-derivative error norm
//   chi = sqrt(sum_d (D+ - D-)^2 / sum_d (|D+| + |D-| + eps sigma_ref,d)^2)
// of sigma(U) over the active dimensions, D+ = sigma(c + e_d) - sigma(c),
// D- = sigma(c) - sigma(c - e_d), sigma_ref,d = |sigma(c + e_d)| +
// 2|sigma(c)| + |sigma(c - e_d)|; a cell is tagged when chi > chi_r.
//
// Every decision equals that of the float64 evaluation of the definition in
// the order written.  The kernels decide in float32 first: with every sigma
// value carried to within k u |sigma| (u = 2^-24; float64 inputs are
// rounded to float32 by integer operations, u, so k = 1 for rho and E, 4
// for E/rho, 8 for B^2/rho), each difference, sum and reference value of
// direction d is off by at most (k + 2.02) u R_d (R_d the exact
// sigma_ref,d), and the denominator's eps R_d term bounds the relative error
// of every ratio; so Q = num - chi_r^2 den is known to within
// M (num + chi_r^2 den), M from tag_margin.  A cell whose float32 Q clears
// twice that margin takes the sign of Q.  Every other cell, and every cell
// whose values leave the range where the bound holds (1e-12 <= R_d <= 1e17,
// no denormal intermediate; flagged by a NaN sigma), is decided by the
// float64 path, written as explicitly rounded operations in the order of the
// definition, whose chi is the definition's to the last bit.
//
// Two launch shapes: k_tag_tile marches 32 x 8 plane tiles of a patch
// along z (ndim >= 2, n_x >= 16): each sigma is formed once, its x and y
// neighbours come from shared memory and its z neighbours from registers;
// k_tag_flat takes one cell per thread with every stencil point from global
// memory (1-D patches, narrow patches, and the chi output, which evaluates
// every cell in float64).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "amr_ops.cuh"

namespace ctu {

struct TagPatch {
    int n[3];
    int slot;  // the patch's index in the caller's list (its count entry)
    long long base;
};

#ifndef CTU_TAG_TY
#define CTU_TAG_TY 8
#endif
#ifndef CTU_TAG_SZ
#define CTU_TAG_SZ 16
#endif
constexpr int TAG_TX = 32, TAG_TY = CTU_TAG_TY, TAG_SZ = CTU_TAG_SZ, TAG_TILE = TAG_TX * TAG_TY;

// float32 value of a float64 x rounded to nearest (ties away from zero) in
// integer operations: the significand is cut to 23 bits and the first
// dropped bit added back (a carry out of the significand moves into the
// exponent, as the encoding intends).  |result - x| <= 2^-24 |x| for
// 2^-126 <= |x| < 2^128 - 2^103; +-0 below 2^-126 (an absolute error under
// 2^-126); +-Inf or NaN beyond (the callers' range checks then fail).
__device__ __forceinline__ float f32_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned a = hi & 0x7FFFFFFFu, sg = hi & 0x80000000u;
    const unsigned mag = (((a - (896u << 20)) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
    const unsigned r = a >= (1151u << 20) ? 0x7FC00000u : (a < (897u << 20) ? sg : (sg | mag));
    return __uint_as_float(r);
}

template <int KIND>
__device__ __forceinline__ double tag_sigma64(const double *U, long long us, long long c)
{
    if (KIND == 0) return U[c];
    if (KIND == 1) return U[4 * us + c];
    if (KIND == 2) {
        const double b0 = U[5 * us + c], b1 = U[6 * us + c], b2 = U[7 * us + c];
        return __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(b0, b0), __dmul_rn(b1, b1)), __dmul_rn(b2, b2)), U[c]);
    }
    return __ddiv_rn(U[4 * us + c], U[c]);
}

// sigma in float32 from truncated inputs; NaN where an intermediate would
// lose its relative accuracy (denormal or overflow).
template <int KIND>
__device__ __forceinline__ float tag_sigma32(const double *U, long long us, long long c)
{
    if (KIND == 0) return f32_rn(U[c]);
    if (KIND == 1) return f32_rn(U[4 * us + c]);
    const float r = f32_rn(U[c]);
    const bool rok = r >= 1e-30f && r <= 1e30f;
    if (KIND == 2) {
        const float b0 = f32_rn(U[5 * us + c]), b1 = f32_rn(U[6 * us + c]), b2 = f32_rn(U[7 * us + c]);
        const float bb = __fadd_rn(__fadd_rn(__fmul_rn(b0, b0), __fmul_rn(b1, b1)), __fmul_rn(b2, b2));
        const bool ok = rok && (bb == 0.0f || (bb >= 1e-30f && bb <= 1e30f));
        return ok ? __fdiv_rn(bb, r) : __uint_as_float(0x7FC00000u);
    }
    const float e = f32_rn(U[4 * us + c]);
    const bool ok = rok && (e == 0.0f || (fabsf(e) >= 1e-30f && fabsf(e) <= 1e30f));
    return ok ? __fdiv_rn(e, r) : __uint_as_float(0x7FC00000u);
}

// One direction's float32 terms; R out of range (or NaN) clears ok.
__device__ __forceinline__ void tag_dir32(float sp, float s0, float sm, float eps32, float &num, float &den, bool &ok)
{
    const float a = sp - s0, b = s0 - sm, d2 = a - b;
    const float R = fabsf(sp) + 2.0f * fabsf(s0) + fabsf(sm);
    ok &= R >= 1e-12f && R <= 1e17f;
    const float T = fabsf(a) + fabsf(b) + eps32 * R;
    num += d2 * d2;
    den += T * T;
}

// The float64 evaluation of the definition at cell c (strides st[d]).
template <int KIND>
__device__ double tag_chi64(const double *U, long long us, long long c, const long long st[3], int ndim, double eps)
{
    const double s0 = tag_sigma64<KIND>(U, us, c);
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= ndim) break;
        const double sp = tag_sigma64<KIND>(U, us, c + st[d]);
        const double sm = tag_sigma64<KIND>(U, us, c - st[d]);
        const double dp = __dsub_rn(sp, s0), dm = __dsub_rn(s0, sm);
        const double a = __dsub_rn(dp, dm);
        num = __dadd_rn(num, __dmul_rn(a, a));
        const double ref = __dadd_rn(__dadd_rn(fabs(sp), __dmul_rn(2.0, fabs(s0))), fabs(sm));
        const double b = __dadd_rn(__dadd_rn(fabs(dp), fabs(dm)), __dmul_rn(eps, ref));
        den = __dadd_rn(den, __dmul_rn(b, b));
    }
    return __dsqrt_rn(__ddiv_rn(num, den));
}

struct TagArgs {
    const TagPatch *tp;
    BlockMap map;
    int ndim;
    const double *U;
    long long us;
    double eps, chi_r;
    float eps32, c2, filt;
    unsigned char *tags;
    unsigned long long *counts;
    double *chi;
};

__device__ __forceinline__ void tag_count(bool tag, unsigned &acc)
{
    const unsigned m = __ballot_sync(0xffffffffu, tag);
    acc += __popc(m);
}

__device__ __forceinline__ void tag_flush(const TagArgs &a, int slot, unsigned acc)
{
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(a.counts + slot, (unsigned long long)acc);
}

// One cell per thread, every stencil point from global memory.  Cells the
// float32 pass leaves undecided are queued in shared memory and evaluated in
// float64 by consecutive threads, so the slow float64 path runs on whole
// warps rather than on one lane of many warps.
template <int KIND, bool CHI>
__global__ void __launch_bounds__(AMR_BLOCK) k_tag_flat(TagArgs a)
{
    __shared__ long long fq[AMR_BLOCK];
    __shared__ unsigned fqn;
    if (threadIdx.x == 0) fqn = 0;
    __syncthreads();
    int bi;
    long long t;
    a.map.locate(bi, t);
    const TagPatch P = a.tp[bi];
    const long long cnt = (long long)P.n[0] * P.n[1] * P.n[2];
    const int g1 = a.ndim > 1 ? AMR_NG : 0;
    const long long N0 = P.n[0] + 2 * AMR_NG, N1 = P.n[1] + 2 * g1;
    const long long st[3] = {1, N0, N0 * N1};
    bool tag = false;
    if (t < cnt) {
        const unsigned t32 = (unsigned)t, row = t32 / (unsigned)P.n[0];
        const int x = (int)(t32 - row * (unsigned)P.n[0]);
        const unsigned zz = row / (unsigned)P.n[1];
        const int y = (int)(row - zz * (unsigned)P.n[1]), z = (int)zz;
        const int g2 = a.ndim > 2 ? AMR_NG : 0;
        const long long c = P.base + ((long long)(z + g2) * N1 + (y + g1)) * N0 + (x + AMR_NG);
        if (CHI) {
            const double x_ = tag_chi64<KIND>(a.U, a.us, c, st, a.ndim, a.eps);
            a.chi[c] = x_;
            tag = x_ > a.chi_r;
            a.tags[c] = tag ? 1 : 0;
        } else {
            bool ok = true;
            const float s0 = tag_sigma32<KIND>(a.U, a.us, c);
            float num = 0.0f, den = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (d < a.ndim)
                    tag_dir32(tag_sigma32<KIND>(a.U, a.us, c + st[d]), s0, tag_sigma32<KIND>(a.U, a.us, c - st[d]),
                              a.eps32, num, den, ok);
            const float Q = num - a.c2 * den;
            if (ok && fabsf(Q) > a.filt * (num + a.c2 * den)) {
                tag = Q > 0.0f;
                a.tags[c] = tag ? 1 : 0;
            } else {
                fq[atomicAdd(&fqn, 1u)] = c;
            }
        }
    }
    unsigned acc = 0;
    tag_count(tag, acc);
    if (!CHI) {
        __syncthreads();
        bool tq = false;
        if (threadIdx.x < fqn) {
            const long long c = fq[threadIdx.x];
            tq = tag_chi64<KIND>(a.U, a.us, c, st, a.ndim, a.eps) > a.chi_r;
            a.tags[c] = tq ? 1 : 0;
        }
        tag_count(tq, acc);
    }
    tag_flush(a, P.slot, acc);
}

// A 32 x 8 tile of one plane per block, marching TAG_SZ planes along z.
// Two shared-memory buffers hold sigma of consecutive planes with a
// one-cell halo in x and y; each thread carries sigma of its column at
// z - 1, z, z + 1 and z + 2, and the halo threads the next plane's halo
// value, so the loads of plane z + 1 (and of the column two planes ahead)
// are in flight while plane z is evaluated.  Undecided cells are queued
// (at most one per thread and plane) and evaluated in float64 at the end by
// consecutive threads.
template <int KIND>
__global__ void __launch_bounds__(TAG_TILE) k_tag_tile(TagArgs a)
{
    __shared__ float s[2][TAG_TY + 2][TAG_TX + 2];
    __shared__ unsigned q[TAG_SZ * TAG_TILE];
    __shared__ unsigned qn;
    const int box = a.map.blk_box[blockIdx.x];
    const int rel = blockIdx.x - a.map.box_start[box];
    const TagPatch P = a.tp[box];
    const int ntx = (P.n[0] + TAG_TX - 1) / TAG_TX, nty = (P.n[1] + TAG_TY - 1) / TAG_TY;
    const int tx = rel % ntx, ty = (rel / ntx) % nty, sz = rel / (ntx * nty);
    const int lx = threadIdx.x % TAG_TX, ly = threadIdx.x / TAG_TX;
    const int x = tx * TAG_TX + lx, y = ty * TAG_TY + ly;
    const int z0 = sz * TAG_SZ, z1 = min(z0 + TAG_SZ, P.n[2]);
    const bool z3 = a.ndim > 2;
    const int g2 = z3 ? AMR_NG : 0;
    const long long N0 = P.n[0] + 2 * AMR_NG, N1 = P.n[1] + 2 * AMR_NG, PS = N0 * N1;
    const long long st[3] = {1, N0, PS};
    // own column (x, y) may lie outside the interior (ragged tile); it is
    // read only where it is the interior or the ghost layer beside it
    const bool inside = x < P.n[0] && y < P.n[1];
    const bool own_ok = x <= P.n[0] && y <= P.n[1];
    const long long col = P.base + (long long)(y + AMR_NG) * N0 + (x + AMR_NG) + (long long)g2 * PS;
    // this thread's halo entry, if any: 2 (TX + 2) + 2 TY entries per plane
    constexpr int NH = 2 * (TAG_TX + 2) + 2 * TAG_TY;
    int hx = 0, hy = 0;
    bool hok = false;
    long long hoff = 0;
    if (threadIdx.x < NH) {
        const int h = threadIdx.x;
        if (h < 2 * (TAG_TX + 2)) {
            hx = h % (TAG_TX + 2);
            hy = h < TAG_TX + 2 ? 0 : TAG_TY + 1;
        } else {
            const int k = h - 2 * (TAG_TX + 2);
            hx = k < TAG_TY ? 0 : TAG_TX + 1;
            hy = 1 + (k % TAG_TY);
        }
        const int gx = tx * TAG_TX + hx - 1, gy = ty * TAG_TY + hy - 1;
        hok = gx <= P.n[0] && gy <= P.n[1];
        hoff = P.base + (long long)(gy + AMR_NG) * N0 + (gx + AMR_NG) + (long long)g2 * PS;
    }
    if (threadIdx.x == 0) qn = 0;
    float prev = 0.0f, cur = 0.0f, nxt = 0.0f, nn = 0.0f, hv = 0.0f;
    if (own_ok) {
        cur = tag_sigma32<KIND>(a.U, a.us, col + (long long)z0 * PS);
        if (z3) {
            prev = tag_sigma32<KIND>(a.U, a.us, col + (long long)(z0 - 1) * PS);
            nxt = tag_sigma32<KIND>(a.U, a.us, col + (long long)(z0 + 1) * PS);
            if (z0 + 1 < z1) nn = tag_sigma32<KIND>(a.U, a.us, col + (long long)(z0 + 2) * PS);
        }
    }
    if (hok) hv = tag_sigma32<KIND>(a.U, a.us, hoff + (long long)z0 * PS);
    s[0][ly + 1][lx + 1] = cur;
    if (threadIdx.x < NH) s[0][hy][hx] = hv;
    if (hok && z0 + 1 < z1) hv = tag_sigma32<KIND>(a.U, a.us, hoff + (long long)(z0 + 1) * PS);
    __syncthreads();
    unsigned acc = 0;
    for (int z = z0; z < z1; ++z) {
        const int b = (z - z0) & 1;
        bool tag = false;
        if (inside) {
            bool ok = true;
            float num = 0.0f, den = 0.0f;
            tag_dir32(s[b][ly + 1][lx + 2], cur, s[b][ly + 1][lx], a.eps32, num, den, ok);
            tag_dir32(s[b][ly + 2][lx + 1], cur, s[b][ly][lx + 1], a.eps32, num, den, ok);
            if (z3) tag_dir32(nxt, cur, prev, a.eps32, num, den, ok);
            const float Q = num - a.c2 * den;
            const long long c = col + (long long)z * PS;
            if (ok && fabsf(Q) > a.filt * (num + a.c2 * den)) {
                tag = Q > 0.0f;
                a.tags[c] = tag ? 1 : 0;
            } else {
                q[atomicAdd(&qn, 1u)] = (unsigned)(c - P.base);
            }
        }
        tag_count(tag, acc);
        if (z + 1 < z1) {
            s[b ^ 1][ly + 1][lx + 1] = nxt;
            if (threadIdx.x < NH) s[b ^ 1][hy][hx] = hv;
            if (hok && z + 2 < z1) hv = tag_sigma32<KIND>(a.U, a.us, hoff + (long long)(z + 2) * PS);
            prev = cur;
            cur = nxt;
            nxt = nn;
            if (own_ok && z + 2 < z1) nn = tag_sigma32<KIND>(a.U, a.us, col + (long long)(z + 3) * PS);
        }
        __syncthreads();
    }
    const unsigned nq = qn;
    for (unsigned i0 = 0; i0 < nq; i0 += TAG_TILE) {
        const unsigned i = i0 + threadIdx.x;
        bool tq = false;
        if (i < nq) {
            const long long c = P.base + q[i];
            tq = tag_chi64<KIND>(a.U, a.us, c, st, a.ndim, a.eps) > a.chi_r;
            a.tags[c] = tq ? 1 : 0;
        }
        tag_count(tq, acc);
    }
    tag_flush(a, P.slot, acc);
}

// The float32 decision margin 2M for sigma kind `kind` (infinite where the
// bound is too loose to be worth a float32 pass: eps or chi_r below 1e-3, or
// M above 0.05).
inline double tag_margin(int kind, double eps, double chi_r)
{
    const double u = 5.9604644775390625e-08;  // 2^-24
    if (!(eps >= 1e-3) || !(chi_r >= 1e-3)) return INFINITY;
    const double k = kind == 2 ? 8.0 : (kind == 3 ? 4.0 : 1.0), ck = k + 2.02;
    const double eT = (ck + eps * (k + 3.02)) * u / eps + 1.01 * u;
    const double eden = 2.0 * eT + eT * eT + 3.0 * u;
    const double M = ck * u / (eps * chi_r) + ck * ck * u * u / (eps * eps * chi_r * chi_r) + eden + 5.02 * u;
    return M > 0.05 ? INFINITY : 2.0 * M;
}

} // namespace ctu
