"""Pins of the oracle's refinement criterion, Eq. (RefCrit) (Section 4):
closed forms for a parabola and a step, exact zeros on linear data, the
bound chi <= 1, invariance under sigma -> -sigma and sigma -> 2 sigma
(bitwise: both are exact in binary floating point), symmetry under an axis
permutation, the derived sigma of each kind against the density kind on a
patch whose density is that sigma, and tags = [chi > chi_r]."""
import numpy as np

import oracle as O

EPS = 0.01


def _patch(n, ndim, rho=None, seed=0):
    rng = np.random.default_rng(seed)
    shp = O.shape(n, ndim)
    U = rng.uniform(0.5, 2.0, shp)
    if rho is not None:
        U[0] = rho
    return U


def _xgrid(n, ndim, axis):
    """Ghosted integer coordinates along `axis` (x = 0 at the first interior
    cell), broadcast to the patch's spatial shape."""
    shp = O.shape(n, ndim)[1:]
    g = O.ghosts(ndim)
    ax = 2 - axis
    c = np.arange(shp[ax]) - g[axis]
    view = [1, 1, 1]
    view[ax] = shp[ax]
    return np.broadcast_to(c.reshape(view), shp).astype(np.float64)


def test_linear_data_have_chi_zero():
    n = [9, 7, 5]
    x, y, z = (_xgrid(n, 3, a) for a in range(3))
    U = _patch(n, 3, rho=100.0 + 3.0 * x - 2.0 * y + 5.0 * z)
    t, chi, cnt = O.tag(U, n, 3, 0, EPS, 1e-6)
    assert cnt == 0
    assert np.all(O.interior(chi[None], n, 3) == 0.0)


def test_parabola_closed_form():
    """sigma = x^2 along x (exact integers): D+ - D- = 2, |D+| + |D-| =
    |2x + 1| + |2x - 1|, sigma_ref = 4x^2 + 2."""
    n = [12, 1, 1]
    x = _xgrid(n, 1, 0)
    U = _patch(n, 1, rho=(x - 5.0) ** 2)
    t, chi, cnt = O.tag(U, n, 1, 0, EPS, 0.3)
    xi = np.arange(12) - 5.0
    want = 2.0 / (np.abs(2 * xi + 1) + np.abs(2 * xi - 1) + EPS * (4 * xi ** 2 + 2))
    got = O.interior(chi[None], n, 1)[0].ravel()
    assert np.allclose(got, want, rtol=1e-15, atol=0)
    assert cnt == int(np.sum(want > 0.3))
    assert np.array_equal(O.interior(t[None], n, 1)[0].ravel(), (want > 0.3).astype(np.uint8))


def test_step_closed_form_in_each_direction():
    """sigma = 1 below a plane, 2 above it: the two cells beside the jump
    have D+ - D- = +-1 and |D+| + |D-| = 1 across it, with sigma_ref = 1 + 2 +
    2 = 5 on the low side and 1 + 4 + 2 = 7 on the high side; along the two
    other directions the differences vanish and sigma_ref = 4 sigma.  So
    chi = 1 / sqrt((1 + 5 eps)^2 + 2 (4 eps)^2) and
    1 / sqrt((1 + 7 eps)^2 + 2 (8 eps)^2); every other cell has chi = 0."""
    n = [8, 8, 8]
    for axis in range(3):
        x = _xgrid(n, 3, axis)
        U = _patch(n, 3, rho=np.where(x < 4, 1.0, 2.0))
        t, chi, cnt = O.tag(U, n, 3, 0, EPS, 0.5)
        C = O.interior(chi[None], n, 3)[0]
        xi = O.interior(x[None], n, 3)[0]
        lo = 1.0 / np.sqrt((1.0 + 5 * EPS) ** 2 + 2 * (4 * EPS) ** 2)
        hi = 1.0 / np.sqrt((1.0 + 7 * EPS) ** 2 + 2 * (8 * EPS) ** 2)
        assert np.allclose(C[xi == 3], lo, rtol=1e-15, atol=0)
        assert np.allclose(C[xi == 4], hi, rtol=1e-15, atol=0)
        assert np.all(C[(xi != 3) & (xi != 4)] == 0.0)
        assert cnt == 2 * 64


def test_bound_sign_and_scale_invariance():
    n = [10, 9, 8]
    U = _patch(n, 3, seed=1)
    U[0] = np.random.default_rng(2).normal(0.0, 1.0, U[0].shape)  # mixed signs
    t, chi, cnt = O.tag(U, n, 3, 0, EPS, 0.2)
    C = O.interior(chi[None], n, 3)[0]
    assert np.all((C >= 0.0) & (C <= 1.0))
    for f in (-1.0, 2.0, 0.25):
        V = U.copy()
        V[0] *= f
        t2, chi2, cnt2 = O.tag(V, n, 3, 0, EPS, 0.2)
        assert np.array_equal(chi2, chi) and cnt2 == cnt and np.array_equal(t2, t)
    assert np.array_equal(O.interior(t[None], n, 3)[0], (C > 0.2).astype(np.uint8))
    assert 0 < cnt < C.size


def test_axis_permutation():
    """Transposing x and z of the data transposes chi (to rounding: the sum
    over directions is taken in another order)."""
    n = [8, 8, 8]
    U = _patch(n, 3, seed=3)
    _, chi, _ = O.tag(U, n, 3, 0, EPS, 0.2)
    V = np.ascontiguousarray(np.transpose(U, (0, 3, 2, 1)))
    _, chiT, _ = O.tag(V, n, 3, 0, EPS, 0.2)
    a = O.interior(chi[None], n, 3)[0]
    b = np.transpose(O.interior(chiT[None], n, 3)[0], (2, 1, 0))
    assert np.allclose(a, b, rtol=1e-14, atol=0)


def test_each_sigma_kind_against_the_density_kind():
    n = [7, 6, 5]
    U = _patch(n, 3, seed=4)
    U[5:8] = np.random.default_rng(5).normal(0.0, 1.0, U[5:8].shape)
    sig = {1: U[4], 2: (U[5] * U[5] + U[6] * U[6] + U[7] * U[7]) / U[0], 3: U[4] / U[0]}
    for kind, s in sig.items():
        _, chi_k, cnt_k = O.tag(U, n, 3, kind, EPS, 0.05)
        V = U.copy()
        V[0] = s
        _, chi_d, cnt_d = O.tag(V, n, 3, 0, EPS, 0.05)
        assert np.array_equal(chi_k, chi_d) and cnt_k == cnt_d, kind


def test_zero_sigma_gives_nan_and_no_tag():
    n = [6, 6, 1]
    U = _patch(n, 2, rho=0.0)
    t, chi, cnt = O.tag(U, n, 2, 0, EPS, 0.0)
    assert cnt == 0 and np.all(np.isnan(O.interior(chi[None], n, 2)))
