"""Pins of the oracle's level operators (Section 4 of Mignone et al. 2012):
prolongation with time interpolation, Eq. (prolong) + (intalpha);
restriction, Eq. (avgdown); reflux, Eq. (fluxcorr) + (addreflux).  Each is
checked against what the mathematics fixes: exact reproduction of linear
data, conservation of the coarse average, no new extrema, the inverse
relation of restriction and prolongation, brute force on tiny inputs, and
conservation of a two-level hierarchy."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W


def _patch(n, ndim, rng):
    return rng.standard_normal(O.shape(n, ndim))


def _fill_linear(n, ndim, a, b):
    """U_q(c) = a_q + sum_d b_qd c_d at every (ghosted) coarse cell c."""
    g = O.ghosts(ndim)
    U = np.zeros(O.shape(n, ndim))
    z, y, x = np.meshgrid(*[np.arange(-g[d], n[d] + g[d]) for d in (2, 1, 0)], indexing="ij")
    for q in range(9):
        U[q] = a[q] + b[q, 0] * x + b[q, 1] * y + b[q, 2] * z
    return U


@pytest.mark.parametrize("ndim,r", [(1, 2), (2, 2), (3, 2), (3, 3), (2, 4)])
def test_prolongation_reproduces_linear_data(ndim, r):
    """Equal differences pass the MC limiter unchanged, so a coarse field
    linear in the cell index is prolonged to the same linear function at
    the fine cell centres, ghosts included."""
    rng = np.random.default_rng(ndim * 10 + r)
    nc = [8 if d < ndim else 1 for d in range(3)]
    nf = [6 if d < ndim else 1 for d in range(3)]
    a = rng.standard_normal(9)
    b = rng.standard_normal((9, 3)) * np.array([1.0 if d < ndim else 0.0 for d in range(3)])
    Uc = _fill_linear(nc, ndim, a, b)
    origin = [2 if d < ndim else 0 for d in range(3)]
    Uf = np.zeros(O.shape(nf, ndim))
    g = O.ghosts(ndim)
    lo = [-g[d] for d in range(3)]
    hi = [nf[d] + g[d] for d in range(3)]
    O.prolong(Uc, Uc, nc, 0.3, Uf, nf, lo, hi, origin, r, ndim)
    z, y, x = np.meshgrid(*[np.arange(-g[d], nf[d] + g[d]) for d in (2, 1, 0)], indexing="ij")
    xs = [x, y, z]
    for q in range(9):
        ref = a[q] + sum(b[q, d] * (origin[d] + (xs[d] + 0.5) / r - 0.5) for d in range(ndim))
        assert np.allclose(Uf[q], ref, rtol=0, atol=1e-12 * (1 + np.abs(ref).max()))


@pytest.mark.parametrize("ndim", [2, 3])
def test_prolongation_conserves_the_coarse_average(ndim):
    """The r^ndim children of a coarse cell average to its time-interpolated
    value: the interpolant preserves the conservative properties (Section
    4), since the offsets of the children sum to zero along each direction."""
    rng = np.random.default_rng(7 + ndim)
    r = 2
    nc = [6 if d < ndim else 1 for d in range(3)]
    Uo, Un = _patch(nc, ndim, rng), _patch(nc, ndim, rng)
    alpha = 0.37
    nf = [2 * nc[d] if d < ndim else 1 for d in range(3)]
    Uf = np.zeros(O.shape(nf, ndim))
    O.prolong(Uo, Un, nc, alpha, Uf, nf, [0, 0, 0], nf, [0, 0, 0], r, ndim)
    Us = O.interior((1 - alpha) * Uo + alpha * Un, nc, ndim)
    If = O.interior(Uf, nf, ndim)
    for kz, ky, kx in itertools.product(*[range(nc[d]) for d in (2, 1, 0)]):
        sl = (slice(None), slice(kz * r, kz * r + r) if ndim > 2 else slice(0, 1),
              slice(ky * r, ky * r + r), slice(kx * r, kx * r + r))
        assert np.allclose(If[sl].reshape(9, -1).mean(axis=1), Us[:, kz, ky, kx], rtol=0, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_prolongation_adds_no_extrema_along_a_direction(d):
    """Data varying along one direction only: the MC-limited slope keeps
    every child within the range of its coarse cell and the two neighbours
    along that direction (Eq. MClim: no new local extrema)."""
    ndim, r = 3, 2
    rng = np.random.default_rng(11 + d)
    nc = [6, 6, 6]
    line = rng.standard_normal((9, nc[d] + 8))
    U = np.zeros(O.shape(nc, ndim))
    shape = [1, 1, 1]
    shape[2 - d] = nc[d] + 8
    for q in range(9):
        U[q] = line[q].reshape(shape)
    nf = [12, 12, 12]
    Uf = np.zeros(O.shape(nf, ndim))
    O.prolong(U, U, nc, 0.0, Uf, nf, [0, 0, 0], nf, [0, 0, 0], r, ndim)
    If = O.interior(Uf, nf, ndim)
    for c in range(nc[d]):
        nb = line[:, c + 4 - 1:c + 4 + 2]
        idx = [slice(None)] * 4
        idx[3 - d] = slice(c * r, c * r + r)
        kids = If[tuple(idx)].reshape(9, -1)
        assert np.all(kids <= nb.max(axis=1)[:, None] + 1e-14)
        assert np.all(kids >= nb.min(axis=1)[:, None] - 1e-14)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_prolongation_one_sided_at_the_domain_boundary(ndim):
    """Cells touching the domain boundary take one-sided differences (Section
    4).  A coarse patch whose first and last cells along every active axis
    touch the boundary (phys bits set), its ghosts beyond it NaN (no value
    there may be read): children of a boundary cell take U* + w (u_inside -
    u_0) (lower boundary) or U* + w (u_0 - u_inside) (upper), in closed form
    on data quadratic in the cell index (whose central and one-sided
    differences differ); interior cells keep the MC central slope; linear data
    are still reproduced exactly, and the children still average to their
    coarse cell."""
    r = 2
    nc = [5 if d < ndim else 1 for d in range(3)]
    nf = [2 * nc[d] if d < ndim else 1 for d in range(3)]
    phys = sum(3 << (2 * d) for d in range(ndim))
    g = O.ghosts(ndim)
    z, y, x = np.meshgrid(*[np.arange(-g[d], nc[d] + g[d]) for d in (2, 1, 0)], indexing="ij")
    xs = [x, y, z]
    U = np.zeros(O.shape(nc, ndim))
    for q in range(9):
        U[q] = 1.0 + 0.1 * q + sum((0.3 + 0.1 * d) * xs[d] ** 2 for d in range(ndim))
    inside = np.ones(U.shape[1:], dtype=bool)
    for d in range(ndim):
        inside &= (xs[d] >= 0) & (xs[d] < nc[d])
    U[:, ~inside] = np.nan
    Uf = np.zeros(O.shape(nf, ndim))
    O.prolong(U, U, nc, 0.25, Uf, nf, [0, 0, 0], nf, [0, 0, 0], r, ndim, phys=phys)
    If = O.interior(Uf, nf, ndim)
    assert np.all(np.isfinite(If))
    for kz, ky, kx in itertools.product(*[range(nf[d]) for d in (2, 1, 0)]):
        f = [kx, ky, kz]
        c = [f[d] // r for d in range(3)]
        for q in range(9):
            u0 = 1.0 + 0.1 * q + sum((0.3 + 0.1 * d) * c[d] ** 2 for d in range(ndim))
            val = u0
            for d in range(ndim):
                a = 0.3 + 0.1 * d
                w = ((f[d] % r) + 0.5) / r - 0.5
                if c[d] == 0:
                    s = a * 1.0                                   # u(1) - u(0)
                elif c[d] == nc[d] - 1:
                    s = a * (c[d] ** 2 - (c[d] - 1) ** 2)         # u(n-1) - u(n-2)
                else:
                    dm, dp = a * (2 * c[d] - 1), a * (2 * c[d] + 1)
                    s = min(0.5 * (dm + dp), 2 * dm, 2 * dp)     # MC of two positive differences
                val += w * s
            assert If[q, kz, ky, kx] == pytest.approx(val, rel=0, abs=1e-13)
    # without the boundary bits the boundary cells take the limited central
    # difference with the (NaN) ghost, which the MC limiter turns into no slope
    Ug = np.zeros_like(Uf)
    O.prolong(U, U, nc, 0.25, Ug, nf, [0, 0, 0], nf, [0, 0, 0], r, ndim, phys=0)
    assert not np.array_equal(O.interior(Ug, nf, ndim), If)


def test_prolongation_one_sided_keeps_linear_data_and_averages():
    rng = np.random.default_rng(21)
    ndim, r = 3, 2
    nc, nf = [4, 4, 4], [8, 8, 8]
    a, b = rng.standard_normal(9), rng.standard_normal((9, 3))
    Uc = _fill_linear(nc, ndim, a, b)
    Uf = np.zeros(O.shape(nf, ndim))
    O.prolong(Uc, Uc, nc, 0.0, Uf, nf, [0, 0, 0], nf, [0, 0, 0], r, ndim, phys=0b010110)
    z, y, x = np.meshgrid(*[np.arange(8) for _ in range(3)], indexing="ij")
    If = O.interior(Uf, nf, ndim)
    for q in range(9):
        ref = a[q] + sum(b[q, d] * ((xs + 0.5) / r - 0.5) for d, xs in enumerate((x, y, z)))
        assert np.allclose(If[q], ref, rtol=0, atol=1e-12)
    Uo = rng.standard_normal(O.shape(nc, ndim))
    O.prolong(Uo, Uo, nc, 0.0, Uf, nf, [0, 0, 0], nf, [0, 0, 0], r, ndim, phys=0b111111)
    If = O.interior(Uf, nf, ndim)
    Ic = O.interior(Uo, nc, ndim)
    avg = If.reshape(9, 4, 2, 4, 2, 4, 2).mean(axis=(2, 4, 6))
    assert np.allclose(avg, Ic, rtol=0, atol=1e-14)


def test_prolongation_one_cell_domain_has_no_slope():
    """A domain one coarse cell wide along x (both bits): the children equal
    their coarse cell's value along x."""
    nc, nf, ndim = [1, 3, 1], [2, 6, 1], 2
    rng = np.random.default_rng(5)
    U = rng.standard_normal(O.shape(nc, ndim))
    U[:, :, :, :4] = np.nan
    U[:, :, :, 5:] = np.nan
    Uf = np.zeros(O.shape(nf, ndim))
    O.prolong(U, U, nc, 0.0, Uf, nf, [0, 0, 0], nf, [0, 0, 0], 2, ndim, phys=0b11)
    If = O.interior(Uf, nf, ndim)
    assert np.all(np.isfinite(If))
    assert np.array_equal(If[:, :, :, 0], If[:, :, :, 1])


def test_prolongation_time_interpolation_is_linear_in_alpha():
    rng = np.random.default_rng(3)
    nc, nf, ndim = [6, 6, 6], [4, 4, 4], 3
    Uo, Un = _patch(nc, ndim, rng), _patch(nc, ndim, rng)
    out = []
    for alpha in (0.0, 1.0):
        Uf = np.zeros(O.shape(nf, ndim))
        O.prolong(Uo, Un, nc, alpha, Uf, nf, [-4] * 3, [8] * 3, [1, 1, 1], 2, ndim)
        out.append(Uf)
        Ug = np.zeros_like(Uf)
        same = Uo if alpha == 0.0 else Un
        O.prolong(same, same, nc, 0.5, Ug, nf, [-4] * 3, [8] * 3, [1, 1, 1], 2, ndim)
        assert np.array_equal(Uf, Ug)


def test_prolongation_brute_force_tiny():
    """One fine cell in 1-D written out by hand from the definition."""
    nc, nf, ndim = [4, 1, 1], [2, 1, 1], 1
    Uc = np.zeros(O.shape(nc, 1))
    vals = np.array([0.0, 1.0, 4.0, 5.0, 5.5, 9.0, 9.0, 9.0, 9.0, 9.0, 9.0, 9.0])
    Uc[:] = vals[None, None, None, :]
    Uf = np.zeros(O.shape(nf, 1))
    # fine cells 0, 1 lie in coarse cell 1 (origin 1); neighbours 0 and 2
    O.prolong(Uc, Uc, nc, 0.0, Uf, nf, [0, 0, 0], [2, 1, 1], [1, 0, 0], 2, 1)
    u0, um, up = vals[5], vals[4], vals[6]   # coarse cells 1, 0, 2 (ghost offset 4)
    dm, dp = u0 - um, up - u0               # 3.5, 0 -> minmod 0 -> slope 0
    assert dm > 0 and dp == 0
    assert np.allclose(Uf[0, 0, 0, 4:6], [u0, u0])
    O.prolong(Uc, Uc, nc, 0.0, Uf, nf, [0, 0, 0], [2, 1, 1], [0, 0, 0], 2, 1)
    u0, um, up = vals[4], vals[3], vals[5]   # 5.5, 5.0, 9.0: dm 0.5, dp 3.5
    s = min(0.5 * (0.5 + 3.5), 2 * 0.5)      # MC: min(2.0, 1.0) = 1.0
    assert np.allclose(Uf[0, 0, 0, 4:6], [u0 - 0.25 * s, u0 + 0.25 * s])


@pytest.mark.parametrize("ndim,r", [(2, 2), (3, 2), (3, 4)])
def test_restriction_inverts_prolongation_and_matches_brute_force(ndim, r):
    rng = np.random.default_rng(5 * r + ndim)
    nc = [8 if d < ndim else 1 for d in range(3)]
    Uc = _patch(nc, ndim, rng)
    nf = [4 * r if d < ndim else 1 for d in range(3)]
    origin = [2 if d < ndim else 0 for d in range(3)]
    Uf = np.zeros(O.shape(nf, ndim))
    g = O.ghosts(ndim)
    O.prolong(Uc, Uc, nc, 0.0, Uf, nf, [-g[d] for d in range(3)], [nf[d] + g[d] for d in range(3)],
              origin, r, ndim)
    Ur = Uc.copy()
    Ur[:] = 0.0
    lo = origin
    hi = [origin[d] + (4 if d < ndim else 1) for d in range(3)]
    O.restrict(Ur, nc, Uf, nf, lo, hi, origin, r, ndim)
    Ic, Ir = O.interior(Uc, nc, ndim), O.interior(Ur, nc, ndim)
    sl = tuple([slice(None)] + [slice(lo[d], hi[d]) for d in (2, 1, 0)])
    assert np.allclose(Ir[sl], Ic[sl], rtol=0, atol=1e-13)
    # brute force average of one coarse cell
    If = O.interior(Uf, nf, ndim)
    c = [origin[d] + 1 if d < ndim else 0 for d in range(3)]
    kids = []
    for k in itertools.product(*[range(r if d < ndim else 1) for d in range(3)]):
        f = [(c[d] - origin[d]) * r + k[d] if d < ndim else 0 for d in range(3)]
        kids.append(If[:, f[2], f[1], f[0]])
    assert np.allclose(np.mean(kids, axis=0), Ir[:, c[2], c[1], c[0]], rtol=0, atol=1e-14)


def test_reflux_restores_conservation_of_two_levels():
    """A fine patch (ratio 2, two substeps, registers on its boundary) in a
    periodic coarse patch (registers with weight -1 on the coarse faces of
    the interface): restriction plus the oracle's reflux conserves mass,
    momentum, energy and magnetic flux to round-off; without reflux it does
    not."""
    Nc = 32
    nc = [Nc, Nc, 1]
    hc = 1.0 / Nc
    hf = hc / 2
    U = W.mhd_turb_2d(Nc, seed=6)
    lo, hi = 8, 24
    nfc = hi - lo
    nf = [2 * nfc, 2 * nfc, 1]
    total0 = O.interior(U, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    cw, off = [], 0
    sets = []
    for d in (0, 1):
        for side, f in ((-1, lo), (+1, hi)):
            cw.append((d, f, lo, hi, 0, 1, off, -1.0))
            sets.append([d, f, side, lo, hi, 0, 1, off])
            off += 9 * nfc
    fw, fsize = O.boundary_windows(nf, 2, weight=1.0, base=off)
    reg = np.zeros(off + fsize)
    O.fill_periodic(U, nc, 2)
    dt, ch = O.dt_ch(O.mhd_max_speed(U, nc, 2, [hc, hc]), [hc, hc], 2, 0.4)
    Unew, bad = O.mhd_step(U, nc, 2, [hc, hc, 1], dt, ch, recon=1, windows=cw, reg=reg)
    assert bad == 0
    # the fine patch from the old coarse data, ghosts prolonged at each substep
    origin = [lo, lo, 0]
    Uf = np.zeros(O.shape(nf, 2))
    O.prolong(U, Unew, nc, 0.0, Uf, nf, [-4, -4, 0], [nf[0] + 4, nf[1] + 4, 1], origin, 2, 2)
    for q in range(2):
        Ufn, bad = O.mhd_step(Uf, nf, 2, [hf, hf, 1], dt / 2, ch, recon=1, windows=fw, reg=reg)
        assert bad == 0
        Uf = Ufn.copy()
        # ghosts of the next substep from the coarse level at alpha = (q + 1)/2
        for (l0, h0) in (((-4, -4), (0, nf[1] + 4)), ((nf[0], -4), (nf[0] + 4, nf[1] + 4)),
                         ((0, -4), (nf[0], 0)), ((0, nf[1]), (nf[0], nf[1] + 4))):
            O.prolong(U, Unew, nc, (q + 1) / 2, Uf, nf, [l0[0], l0[1], 0], [h0[0], h0[1], 1], origin, 2, 2)
    O.restrict(Unew, nc, Uf, nf, [lo, lo, 0], [hi, hi, 1], origin, 2, 2)
    no_reflux = O.interior(Unew, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    # fine windows: boundary_windows orders (dir, plane 0 / n) with rows of n_a faces
    fwin = {(w[0], w[1]): w for w in fw}
    for d, f, side, a0, a1, b0, b1, creg in sets:
        w = fwin[(d, 0 if side < 0 else nf[d])]
        fna, fnb = w[3] - w[2], w[5] - w[4]
        O.reflux(Unew, nc, [hc, hc], reg, d, f, side, a0, a1, b0, b1, creg, w[6], 0, 0, fna, fnb, 2, 2)
    total = O.interior(Unew, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    scale = np.abs(O.interior(Unew, nc, 2)).sum(axis=(1, 2, 3)) * hc * hc
    assert np.all(np.abs(total - total0)[:8] <= 1e-13 * scale[:8]), (total - total0)
    assert np.abs(no_reflux - total0)[[0, 4]].max() > 1e-8


def test_diagnostics_closed_forms():
    """Totals of a uniform state are value x volume; the central-difference
    divergence of a linear field is its trace, of the central-difference
    curl of any potential exactly zero (the differences commute)."""
    rng = np.random.default_rng(21)
    n, ndim = [10, 8, 6], 3
    dx = [0.1, 0.2, 0.05]
    U = np.zeros(O.shape(n, ndim))
    vals = rng.standard_normal(9)
    U[:] = vals[:, None, None, None]
    g = O.ghosts(ndim)
    z, y, x = np.meshgrid(*[(np.arange(-g[d], n[d] + g[d]) + 0.5) * dx[d] for d in (2, 1, 0)], indexing="ij")
    a, b, c = 0.7, -1.3, 2.1
    U[5], U[6], U[7] = 3.0 + a * x, -1.0 + b * y, 0.5 + c * z
    out = O.diagnostics(U, n, ndim, dx)
    vol = np.prod(dx) * np.prod(n)
    for q in (0, 1, 2, 3, 4, 8):
        assert out[q] == pytest.approx(vals[q] * vol, rel=1e-13)
    assert out[5] == pytest.approx(np.mean(3.0 + a * x[4:-4, 4:-4, 4:-4]) * vol, rel=1e-12)
    assert out[9] == pytest.approx(abs(a + b + c), rel=1e-12)
    # 2-D: B = central-difference curl of a random A_z
    n2 = [16, 12, 1]
    d2 = [1.0 / 16, 1.0 / 12]
    A = rng.standard_normal((12 + 8 + 2, 16 + 8 + 2))
    U2 = np.zeros(O.shape(n2, 2))
    U2[0] = 1.0
    U2[5, 0] = (A[2:, 1:-1] - A[:-2, 1:-1]) / (2 * d2[1])
    U2[6, 0] = -(A[1:-1, 2:] - A[1:-1, :-2]) / (2 * d2[0])
    out2 = O.diagnostics(U2, n2, 2, d2)
    scale = np.abs(U2[5:7]).max() / min(d2)
    assert out2[9] <= 1e-13 * scale
    assert out2[0] == pytest.approx(1.0, rel=1e-14)
