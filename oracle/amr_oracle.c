/* amr_oracle.c -- plain FP64 CPU oracle of the level operators around the
 * CTU step (test infrastructure): coarse-to-fine prolongation with time
 * interpolation, Eq. (prolong) and Eq. (intalpha); restriction, Eq.
 * (avgdown); reflux, Eq. (fluxcorr) and Eq. (addreflux) of Mignone et al.
 * (2012), Section 4; the same-level ghost exchange (copy, pack, unpack);
 * the refinement criterion, Eq. (RefCrit) of Section 4
 * (second-derivative error norm); and the conservation diagnostics of a
 * patch (conserved totals, max |div B|).  Cartesian geometry: the volume coordinate of a
 * direction is the coordinate itself and a cell's volume the product of its
 * widths.
 *
 * Arrays: one patch is float64 [9][N2][N1][N0] with N = n + 2 g, g = 4 on
 * active dimensions (d < ndim) and 0 otherwise; "interior" coordinates run
 * over [0, n) and may reach -g .. n + g - 1 in the ghosts.
 */
#include <math.h>
#include <stddef.h>

#define NV 9
#define NG 4

static long cell(const int n[3], int ndim, int x, int y, int z)
{
    const int g0 = NG, g1 = ndim > 1 ? NG : 0, g2 = ndim > 2 ? NG : 0;
    const long N0 = n[0] + 2 * g0, N1 = n[1] + 2 * g1;
    return ((long)(z + g2) * N1 + (y + g1)) * N0 + (x + g0);
}

static long cells(const int n[3], int ndim)
{
    long c = 1;
    for (int d = 0; d < 3; ++d) c *= n[d] + (d < ndim ? 2 * NG : 0);
    return c;
}

/* MinMod and the monotonised-central slope, Eq. (minmod) and Eq. (MClim). */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

static double mc(double dm, double dp) { return minmod(0.5 * (dm + dp), 2.0 * minmod(dm, dp)); }

/* floor(a / b) for b > 0 */
static int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

/* Eq. (prolong) with Eq. (intalpha): every fine cell x in the box [lo, hi)
 * of the fine patch takes U* of its coarse cell c = origin + floor(x / r)
 * plus, along each active dimension, (xi_fine - xi_coarse) / (xi_+ - xi_-)
 * times the MC-limited central difference of U* there, with
 * U* = (1 - alpha) Uold + alpha Unew.  For a Cartesian cell of width h the
 * weight is ((x mod r) + 1/2) / r - 1/2.
 * Cells touching the domain boundary take one-sided differences (Section
 * 4): bit 2d of phys says that the coarse patch's cell 0 along d lies on the
 * domain's lower boundary, bit 2d + 1 that its cell nc[d] - 1 lies on the
 * upper one; such a cell's difference along d is the one to its neighbour
 * inside the domain (the MC limiter of one difference is that difference),
 * and 0 if it touches both boundaries.  No value beyond the boundary is
 * read. */
void or_prolong(const double *Uco, const double *Ucn, const int nc[3], double alpha, double *Uf, const int nf[3],
                const int lo[3], const int hi[3], const int origin[3], int r, int ndim, int phys)
{
    const long Sc = cells(nc, ndim), Sf = cells(nf, ndim);
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                const int xf[3] = {x, y, z};
                int c[3];
                double w[3];
                for (int d = 0; d < 3; ++d) {
                    if (d < ndim) {
                        c[d] = origin[d] + fdiv(xf[d], r);
                        const int m = xf[d] - r * fdiv(xf[d], r);
                        w[d] = (m + 0.5) / r - 0.5;
                    } else {
                        c[d] = 0;
                        w[d] = 0.0;
                    }
                }
                const long fi = cell(nf, ndim, x, y, z);
                for (int q = 0; q < NV; ++q) {
                    const long c0 = cell(nc, ndim, c[0], c[1], c[2]);
                    const double u0 = (1.0 - alpha) * Uco[q * Sc + c0] + alpha * Ucn[q * Sc + c0];
                    double u = u0;
                    for (int d = 0; d < ndim; ++d) {
                        const int at_lo = (phys >> (2 * d)) & 1 && c[d] == 0;
                        const int at_hi = (phys >> (2 * d + 1)) & 1 && c[d] == nc[d] - 1;
                        int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
                        double slope;
                        cm[d] -= 1;
                        cp[d] += 1;
                        if (at_lo && at_hi) {
                            slope = 0.0;
                        } else if (at_lo) {
                            const long ip = cell(nc, ndim, cp[0], cp[1], cp[2]);
                            slope = (1.0 - alpha) * Uco[q * Sc + ip] + alpha * Ucn[q * Sc + ip] - u0;
                        } else if (at_hi) {
                            const long im = cell(nc, ndim, cm[0], cm[1], cm[2]);
                            slope = u0 - ((1.0 - alpha) * Uco[q * Sc + im] + alpha * Ucn[q * Sc + im]);
                        } else {
                            const long im = cell(nc, ndim, cm[0], cm[1], cm[2]);
                            const long ip = cell(nc, ndim, cp[0], cp[1], cp[2]);
                            const double um = (1.0 - alpha) * Uco[q * Sc + im] + alpha * Ucn[q * Sc + im];
                            const double up = (1.0 - alpha) * Uco[q * Sc + ip] + alpha * Ucn[q * Sc + ip];
                            slope = mc(u0 - um, up - u0);
                        }
                        u += w[d] * slope;
                    }
                    Uf[q * Sf + fi] = u;
                }
            }
}

/* Eq. (avgdown): every coarse cell c in the box [lo, hi) becomes the volume
 * average of its r^ndim fine cells f = (c - origin) r + k, 0 <= k < r. */
void or_restrict(double *Uc, const int nc[3], const double *Uf, const int nf[3], const int lo[3], const int hi[3],
                 const int origin[3], int r, int ndim)
{
    const long Sc = cells(nc, ndim), Sf = cells(nf, ndim);
    const int k1 = ndim > 1 ? r : 1, k2 = ndim > 2 ? r : 1;
    double nk = r;
    if (ndim > 1) nk *= r;
    if (ndim > 2) nk *= r;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                const long ci = cell(nc, ndim, x, y, z);
                for (int q = 0; q < NV; ++q) {
                    double s = 0.0;
                    for (int c2 = 0; c2 < k2; ++c2)
                        for (int c1 = 0; c1 < k1; ++c1)
                            for (int c0 = 0; c0 < r; ++c0) {
                                const int fx = (x - origin[0]) * r + c0;
                                const int fy = ndim > 1 ? (y - origin[1]) * r + c1 : 0;
                                const int fz = ndim > 2 ? (z - origin[2]) * r + c2 : 0;
                                s += Uf[q * Sf + cell(nf, ndim, fx, fy, fz)];
                            }
                    Uc[q * Sc + ci] = s / nk;
                }
            }
}

/* Eq. (fluxcorr) and Eq. (addreflux) for the coarse faces [a0, a1) x [b0, b1)
 * of plane `plane` normal to `dir` (a, b: the two other dimensions in
 * increasing order).  reg holds, per window [q][b][a], the sums a CTU step
 * accumulates: the coarse window with weight -1 (-dt A F_coarse), the fine
 * window with weight +1 (sum over substeps of dt_q A F_fine); the fine faces
 * of coarse face (a, b) are a' = fa0 + (a - a0) r + i, b' = fb0 + (b - b0) r
 * + j in a fine window of fna x fnb faces.  The coarse cell on the coarse
 * side of the interface (cell `plane` for side = +1, whose lower face it is;
 * cell `plane - 1` for side = -1) gains side x (coarse + fine sums) / volume. */
void or_reflux(double *Uc, const int nc[3], const double dxc[3], const double *reg, int dir, int plane, int side,
               int a0, int a1, int b0, int b1, long creg, long freg, int fa0, int fb0, int fna, int fnb, int r,
               int ndim)
{
    const long Sc = cells(nc, ndim);
    const int ea = dir == 0 ? 1 : 0, eb = dir == 2 ? 1 : 2;
    const int rb = eb < ndim ? r : 1, ra = ea < ndim ? r : 1;
    double vol = 1.0;
    for (int d = 0; d < ndim; ++d) vol *= dxc[d];
    const long na = a1 - a0, nb = b1 - b0;
    for (int b = b0; b < b1; ++b)
        for (int a = a0; a < a1; ++a) {
            int c[3];
            c[dir] = side > 0 ? plane : plane - 1;
            c[ea] = a;
            c[eb] = b;
            const long ci = cell(nc, ndim, c[0], c[1], c[2]);
            for (int q = 0; q < NV; ++q) {
                double t = reg[creg + q * na * nb + (long)(b - b0) * na + (a - a0)];
                for (int j = 0; j < rb; ++j)
                    for (int i = 0; i < ra; ++i) {
                        const long fa = fa0 + (long)(a - a0) * ra + i, fb = fb0 + (long)(b - b0) * rb + j;
                        t += reg[freg + q * (long)fna * fnb + fb * fna + fa];
                    }
                Uc[q * Sc + ci] += side * t / vol;
            }
        }
}

/* Diagnostics of one patch: out[q] = sum over interior cells of U_q times the
 * cell volume (the conserved totals, q = 0..8), out[9] = max over interior
 * cells of |div B| with central differences, sum_d (B_d(c + e_d) -
 * B_d(c - e_d)) / (2 dx_d) over the active dimensions. */
void or_diagnostics(const double *U, const int n[3], int ndim, const double dx[3], double out[10])
{
    const long S = cells(n, ndim);
    double vol = 1.0;
    for (int d = 0; d < ndim; ++d) vol *= dx[d];
    for (int q = 0; q < 10; ++q) out[q] = 0.0;
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x) {
                const long c = cell(n, ndim, x, y, z);
                for (int q = 0; q < NV; ++q) out[q] += U[q * S + c] * vol;
                double div = 0.0;
                for (int d = 0; d < ndim; ++d) {
                    int p[3] = {x, y, z}, m[3] = {x, y, z};
                    p[d] += 1;
                    m[d] -= 1;
                    div += (U[(5 + d) * S + cell(n, ndim, p[0], p[1], p[2])] -
                            U[(5 + d) * S + cell(n, ndim, m[0], m[1], m[2])]) / (2.0 * dx[d]);
                }
                if (fabs(div) > out[9]) out[9] = fabs(div);
            }
}

/* The quantity sigma(U) of the refinement criterion: 0 density (rho, or D in
 * relativistic MHD), 1 total energy density E, 2 B^2 / rho, 3 E / rho. */
static double tag_sigma(const double *U, long S, long c, int kind)
{
    switch (kind) {
    case 0: return U[c];
    case 1: return U[4 * S + c];
    case 2: return (U[5 * S + c] * U[5 * S + c] + U[6 * S + c] * U[6 * S + c] + U[7 * S + c] * U[7 * S + c]) / U[c];
    default: return U[4 * S + c] / U[c];
    }
}

/* Eq. (RefCrit), Section 4 (refinement criteria): for every interior cell,
 *   chi = sqrt( sum_d (D+ - D-)^2 / sum_d (|D+| + |D-| + eps sigma_ref,d)^2 )
 * over the active dimensions, with the undivided differences
 * D+ = sigma(c + e_d) - sigma(c), D- = sigma(c) - sigma(c - e_d) and
 * sigma_ref,d = |sigma(c + e_d)| + 2 |sigma(c)| + |sigma(c - e_d)|; the cell is
 * tagged when chi > chi_r.  Reads one ghost layer.  chi and tag are arrays of
 * the patch's ghosted layout (only interior entries written; chi may be
 * NULL).  A cell whose denominator is 0 (sigma = 0 at all its stencil points)
 * gets chi = NaN and no tag.  Returns the number of tagged cells. */
long or_tag(const double *U, const int n[3], int ndim, int kind, double eps, double chi_r, double *chi,
            unsigned char *tag)
{
    const long S = cells(n, ndim);
    long count = 0;
    for (int z = 0; z < n[2]; ++z)
        for (int y = 0; y < n[1]; ++y)
            for (int x = 0; x < n[0]; ++x) {
                const long c = cell(n, ndim, x, y, z);
                const double s0 = tag_sigma(U, S, c, kind);
                double num = 0.0, den = 0.0;
                for (int d = 0; d < ndim; ++d) {
                    int p[3] = {x, y, z}, m[3] = {x, y, z};
                    p[d] += 1;
                    m[d] -= 1;
                    const double sp = tag_sigma(U, S, cell(n, ndim, p[0], p[1], p[2]), kind);
                    const double sm = tag_sigma(U, S, cell(n, ndim, m[0], m[1], m[2]), kind);
                    const double dp = sp - s0, dm = s0 - sm;
                    const double a = dp - dm;
                    num += a * a;
                    const double ref = fabs(sp) + 2.0 * fabs(s0) + fabs(sm);
                    const double b = fabs(dp) + fabs(dm) + eps * ref;
                    den += b * b;
                }
                const double x_ = sqrt(num / den);
                if (chi) chi[c] = x_;
                tag[c] = x_ > chi_r ? 1 : 0;
                count += tag[c];
            }
    return count;
}

/* Same-level ghost exchange, the copy step of Section 4's level advance (a
 * patch's ghost cells that lie over a sibling's interior take the sibling's
 * values).  Box b copies the cells x in [lo, hi) of the destination patch
 * (interior coordinates, ghosts included) from cell x + shift of the source
 * patch, all nine variables.  Boxes are given as 16 ints each:
 *   dn[3], sn[3], lo[3], hi[3], shift[3], pad
 * with the pool offsets of the destination and source patches in dbase[b],
 * sbase[b].  Udst and Usrc may be the same pool. */
void or_copy_boxes(double *Ud, long dstride, const double *Us, long sstride, const int *box, const long *dbase,
                   const long *sbase, int nbox, int ndim)
{
    for (int b = 0; b < nbox; ++b) {
        const int *B = box + 16 * b;
        const int *dn = B, *sn = B + 3, *lo = B + 6, *hi = B + 9, *sh = B + 12;
        for (int z = lo[2]; z < hi[2]; ++z)
            for (int y = lo[1]; y < hi[1]; ++y)
                for (int x = lo[0]; x < hi[0]; ++x) {
                    const long di = dbase[b] + cell(dn, ndim, x, y, z);
                    const long si = sbase[b] + cell(sn, ndim, x + sh[0], y + sh[1], z + sh[2]);
                    for (int q = 0; q < NV; ++q) Ud[q * dstride + di] = Us[q * sstride + si];
                }
    }
}

/* Packing for an exchange between processes: the source cells of every box,
 * box after box, each as [q][z][y][x] over the box's extent; unpacking
 * writes such a buffer into the destination cells. */
void or_pack_boxes(double *buf, const double *Us, long sstride, const int *box, const long *sbase, int nbox,
                   int ndim)
{
    long o = 0;
    for (int b = 0; b < nbox; ++b) {
        const int *B = box + 16 * b;
        const int *sn = B + 3, *lo = B + 6, *hi = B + 9, *sh = B + 12;
        const long ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2], nc = ex * ey * ez;
        for (int q = 0; q < NV; ++q)
            for (int z = lo[2]; z < hi[2]; ++z)
                for (int y = lo[1]; y < hi[1]; ++y)
                    for (int x = lo[0]; x < hi[0]; ++x)
                        buf[o + q * nc + ((long)(z - lo[2]) * ey + (y - lo[1])) * ex + (x - lo[0])] =
                            Us[q * sstride + sbase[b] + cell(sn, ndim, x + sh[0], y + sh[1], z + sh[2])];
        o += NV * nc;
    }
}

void or_unpack_boxes(double *Ud, long dstride, const double *buf, const int *box, const long *dbase, int nbox,
                     int ndim)
{
    long o = 0;
    for (int b = 0; b < nbox; ++b) {
        const int *B = box + 16 * b;
        const int *dn = B, *lo = B + 6, *hi = B + 9;
        const long ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2], nc = ex * ey * ez;
        for (int q = 0; q < NV; ++q)
            for (int z = lo[2]; z < hi[2]; ++z)
                for (int y = lo[1]; y < hi[1]; ++y)
                    for (int x = lo[0]; x < hi[0]; ++x)
                        Ud[q * dstride + dbase[b] + cell(dn, ndim, x, y, z)] =
                            buf[o + q * nc + ((long)(z - lo[2]) * ey + (y - lo[1])) * ex + (x - lo[0])];
        o += NV * nc;
    }
}
