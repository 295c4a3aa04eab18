"""Pins of the oracle's viscosity, the parabolic term of the CTU step for the
stress of Eq. (visc_tens) with constant kinematic viscosity nu (Section 3.1
with Pi != 0; face values by central differences with the transverse
derivatives averaged over the two cells of the face, the coefficient rho nu
and the velocity of the energy flux v . tau at the mean state of the face).

- The discrete operator in closed form on polynomial fields, where the face
  differences are exact: a quadratic shear profile (momentum rho nu f'', the
  energy flux v . tau to its exact discrete value), a quadratic compressive
  profile (the 4/3 of the normal stress), a bilinear 2-D field (the
  transverse-derivative and -(2/3) div v terms: L_P(m_x) = rho nu b / 3), and
  a quadratic density under a linear shear (the mean density of the face).
- The rate of Eq. Ca with the diffusion coefficient (4/3) nu.
- Conservation of momentum and energy on periodic boxes.
- A stationary shear wave in the viscosity-dominated regime against the
  exact decay of the spatially discrete operator, exp(-nu k_h^2 t),
  k_h^2 = (4/dx^2) sin^2(k dx/2): the time integration of the parabolic term
  is second order (forward Euler misses by far more).
- Second-order space-time convergence to the exact linear solutions: an
  advected shear wave (1-D), an oblique shear wave (2-D, the cross terms),
  and a viscously damped sound wave (matrix exponential of the linearised
  system with (4/3) nu k^2 on the velocity).
- Two levels with reflux conserve momentum and energy to round-off with the
  parabolic fluxes in the registers.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle as O
from paper_1110_0740_gb300 import workloads as W

G = 5.0 / 3.0


def _centres(n, ndim, d):
    g = O.ghosts(ndim)
    shp = O.shape(n, ndim)
    x = (np.arange(shp[3 - d]) - g[d] + 0.5) / n[d]
    view = [1, 1, 1]
    view[2 - d] = shp[3 - d]
    return x.reshape(view)


def _U(n, ndim, rho, v, p=1.0, B=(0.3, 0.2, 0.1)):
    z = np.zeros(O.shape(n, ndim)[1:])
    rho = rho + z
    return W.ideal_cons([rho, v[0] + z, v[1] + z, v[2] + z, p + z, z + B[0], z + B[1], z + B[2], z], G)


def test_quadratic_shear_and_its_energy_flux():
    n = [16, 1, 1]
    h = 1.0 / 16
    x = _centres(n, 1, 0)
    a, rho, nu = 0.8, 1.3, 0.05
    U = _U(n, 1, rho, (0.0, a * x ** 2, 0.0))
    LP = O.interior(O.mhd_parabolic(U, n, 1, [h], 0.0, nu, G), n, 1)
    xi = O.interior(x[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0]
    assert np.allclose(LP[2], rho * nu * 2 * a, rtol=0, atol=1e-11)
    assert np.allclose(LP[1], 0.0, atol=1e-12) and np.allclose(LP[3], 0.0, atol=1e-12)
    # v_f = a (x_f^2 + h^2/4) and tau = 2 a rho nu x_f at the face x_f, so
    # the difference of v_f tau over a cell is 2 a^2 rho nu (3 x^2 + h^2/2)
    assert np.allclose(LP[4], 2 * a * a * rho * nu * (3 * xi ** 2 + h * h / 2), rtol=1e-12, atol=1e-12)


def test_quadratic_compression_four_thirds():
    n = [16, 1, 1]
    x = _centres(n, 1, 0)
    a, rho, nu = -0.6, 0.7, 0.03
    U = _U(n, 1, rho, (a * x ** 2, 0.0, 0.0))
    LP = O.interior(O.mhd_parabolic(U, n, 1, [1.0 / 16], 0.0, nu, G), n, 1)
    assert np.allclose(LP[1], 4.0 / 3.0 * rho * nu * 2 * a, rtol=0, atol=1e-11)
    assert np.allclose(LP[2], 0.0, atol=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
def test_bilinear_field_cross_terms(ndim):
    """v = (0, b x y, 0): L_P(m_x) = d_x tau_xx + d_y tau_yx
    = -(2/3) rho nu b + rho nu b = rho nu b / 3, L_P(m_y) = 0."""
    n = [10, 12, 6 if ndim > 2 else 1]
    x, y = _centres(n, ndim, 0), _centres(n, ndim, 1)
    b, rho, nu = 0.9, 1.1, 0.04
    U = _U(n, ndim, rho, (0.0, b * x * y, 0.0))
    dx = [1.0 / n[d] for d in range(ndim)]
    LP = O.interior(O.mhd_parabolic(U, n, ndim, dx, 0.0, nu, G), n, ndim)
    assert np.allclose(LP[1], rho * nu * b / 3.0, rtol=0, atol=1e-11)
    assert np.allclose(LP[2], 0.0, atol=1e-11) and np.allclose(LP[3], 0.0, atol=1e-12)


def test_face_density_is_the_mean():
    """rho = r0 + r x^2, v_y = b x: tau_xy = nu b rho_f with rho_f the mean of
    the two cells, r0 + r (x_f^2 + h^2/4), so L_P(m_y) = 2 nu b r x."""
    n = [16, 1, 1]
    x = _centres(n, 1, 0)
    r0, r, b, nu = 1.0, 0.5, 0.7, 0.02
    U = _U(n, 1, r0 + r * x ** 2, (0.0, b * x, 0.0))
    LP = O.interior(O.mhd_parabolic(U, n, 1, [1.0 / 16], 0.0, nu, G), n, 1)
    xi = O.interior(x[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0]
    assert np.allclose(LP[2], 2 * nu * b * r * xi, rtol=1e-12, atol=1e-13)


def test_max_rate_closed_form():
    n = [8, 8, 8]
    rho, p, nu = 2.0, 3.0, 0.05
    U = _U(n, 3, rho, (0.0, 0.0, 0.0), p=p, B=(0.0, 0.0, 0.0))
    dx = [0.1, 0.2, 0.05]
    want = np.sqrt(G * p / rho) / min(dx) + sum(2 * (4.0 / 3.0) * nu / h ** 2 for h in dx)
    assert O.mhd_max_rate(U, n, 3, dx, G, 0.0, nu) == pytest.approx(want, rel=1e-14)
    # with conduction the larger coefficient counts
    k = 0.5
    want = np.sqrt(G * p / rho) / min(dx) + sum(2 * max((G - 1) * k / rho, 4 / 3 * nu) / h ** 2 for h in dx)
    assert O.mhd_max_rate(U, n, 3, dx, G, k, nu) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("ndim", [2, 3])
def test_conservation_periodic(ndim):
    N = 16
    n = [N, N, N if ndim > 2 else 1]
    U = W.mhd_blast_3d(N, seed=3) if ndim == 3 else W.mhd_turb_2d(N, seed=3)
    dx = [1.0 / N] * ndim
    a = O.interior(U, n, ndim).copy()
    R, t, _ = O.mhd_run(U, n, ndim, dx, 6, 0.3, recon=1, kappa=0.01, nu=0.01)
    b = O.interior(R, n, ndim)
    for q in range(8):
        assert abs(b[q].sum() - a[q].sum()) <= 1e-13 * (np.abs(a[q]).sum() + 1.0), q
    R0, _, _ = O.mhd_run(U, n, ndim, dx, 6, 0.3, recon=1, kappa=0.01)
    assert np.abs(O.interior(R0, n, ndim)[1:5] - b[1:5]).max() > 1e-6


def _shear(N, v0, eps, ndim=1):
    n = [N, N if ndim > 1 else 1, 1]
    if ndim == 1:
        x = _centres(n, 1, 0)
        ph = 2 * np.pi * x
        U = _U(n, 1, 1.0, (v0 + 0 * x, eps * np.sin(ph), 0.0), B=(0.0, 0.0, 0.0))
        return U, n, ph
    x, y = _centres(n, 2, 0), _centres(n, 2, 1)
    ph = 2 * np.pi * (x + y)
    nh, t1 = np.array([1.0, 1.0]) / np.sqrt(2), np.array([-1.0, 1.0]) / np.sqrt(2)
    w = eps * np.sin(ph)
    U = _U(n, 2, 1.0, (v0 * nh[0] + w * t1[0], v0 * nh[1] + w * t1[1], 0.0), B=(0.0, 0.0, 0.0))
    return U, n, ph


def test_stationary_shear_wave_semi_discrete_decay():
    """Viscosity-dominated (dt set by the diffusion term): the hyperbolic
    part leaves a stationary shear wave unchanged at linear order, so v_y
    follows the exact decay of the discrete operator to the time-integration
    error."""
    N, nu, eps, t_end = 32, 0.05, 1e-6, 0.5
    U, n, ph = _shear(N, 0.0, eps)
    R, t, _ = O.mhd_run(U, n, 1, [1.0 / N], None, 0.4, recon=1, t_end=t_end, nu=nu)
    h = 1.0 / N
    kh2 = 4.0 / h ** 2 * np.sin(np.pi * h) ** 2
    Ui = O.interior(R, n, 1)
    vy = Ui[2, 0, 0] / Ui[0, 0, 0]
    ex = eps * np.sin(O.interior(ph[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0, 0, 0]) * np.exp(-nu * kh2 * t)
    assert np.exp(-nu * kh2 * t) < 0.7
    assert np.abs(vy - ex).max() < 3e-4 * eps


def _shear_error(N, ndim, nu, t_end):
    eps, v0 = 1e-6, 0.3
    U, n, ph = _shear(N, v0, eps, ndim)
    dx = [1.0 / N] * ndim
    R, t, _ = O.mhd_run(U, n, ndim, dx, None, 0.4, recon=1, t_end=t_end, nu=nu)
    k = 2 * np.pi * np.sqrt(ndim)
    Ui = O.interior(R, n, ndim)
    if ndim == 1:
        w = Ui[2] / Ui[0]
    else:
        w = (-Ui[1] + Ui[2]) / Ui[0] / np.sqrt(2)
    phi = O.interior(ph[None] + np.zeros((1,) + U.shape[1:]), n, ndim)[0]
    ex = eps * np.sin(phi - k * v0 * t) * np.exp(-nu * k * k * t)
    return np.abs(w - ex).mean() / eps


def test_advected_shear_wave_second_order_1d():
    nu = 0.004
    e = [_shear_error(N, 1, nu, 1.0) for N in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.9, (e, orders)


def test_oblique_shear_wave_second_order_2d():
    nu = 0.002
    e = [_shear_error(N, 2, nu, 0.5) for N in (16, 32, 64)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.8, (e, orders)
    # the viscosity is visible at this time
    assert np.exp(-nu * 8 * np.pi ** 2 * 0.5) < 0.95


def _sound_error(N, nu, t_end):
    """Sound wave rho = 1 + eps cos(k x) at rest (p = 1): the linearised
    system with viscosity, rho_t = -i k u, u_t = -i k p - (4/3) nu k^2 u,
    p_t = -i k Gamma u, integrated exactly."""
    n = [N, 1, 1]
    x = _centres(n, 1, 0)
    eps = 1e-6
    k = 2 * np.pi
    cs = np.sqrt(G)
    # a right-going sound wave: rho = 1 + eps c, u = cs eps c, p = 1 + G eps c
    c = np.cos(k * x)
    U = _U(n, 1, 1.0 + eps * c, (cs * eps * c, 0.0, 0.0), p=1.0 + G * eps * c, B=(0.0, 0.0, 0.0))
    R, t, _ = O.mhd_run(U, n, 1, [1.0 / N], None, 0.4, recon=1, t_end=t_end, nu=nu)
    M = np.array([[0, -1j * k, 0], [0, -4.0 / 3.0 * nu * k * k, -1j * k], [0, -1j * k * G, 0]])
    a = expm(M * t) @ np.array([1.0, cs, G])
    xi = O.interior(x[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0, 0, 0]
    ex = 1.0 + eps * np.real(a[0] * np.exp(1j * k * xi))
    return np.abs(O.interior(R, n, 1)[0, 0, 0] - ex).mean() / eps, abs(a[0])


def test_damped_sound_wave_second_order():
    nu = 0.005
    res = [_sound_error(N, nu, 1.0) for N in (32, 64, 128)]
    e = [r[0] for r in res]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.9, (e, orders)
    assert res[-1][1] < 0.95  # the viscous damping is visible


def test_reflux_with_viscosity_restores_conservation_of_two_levels():
    Nc = 32
    nc = [Nc, Nc, 1]
    hc = 1.0 / Nc
    hf = hc / 2
    kappa, nu = 0.001, 0.001
    U = W.mhd_turb_2d(Nc, seed=6)
    lo, hi = 8, 24
    nfc = hi - lo
    nf = [2 * nfc, 2 * nfc, 1]
    total0 = O.interior(U, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    cw, off, sets = [], 0, []
    for d in (0, 1):
        for side, f in ((-1, lo), (+1, hi)):
            cw.append((d, f, lo, hi, 0, 1, off, -1.0))
            sets.append([d, f, side, lo, hi, 0, 1, off])
            off += 9 * nfc
    fw, fsize = O.boundary_windows(nf, 2, weight=1.0, base=off)
    reg = np.zeros(off + fsize)
    O.fill_periodic(U, nc, 2)
    dt, ch = O.dt_ch(O.mhd_max_rate(U, nc, 2, [hc, hc], G, kappa, nu), [hc, hc], 2, 0.4)
    Unew, bad = O.mhd_step(U, nc, 2, [hc, hc, 1], dt, ch, recon=1, windows=cw, reg=reg, kappa=kappa, nu=nu)
    assert bad == 0
    origin = [lo, lo, 0]
    Uf = np.zeros(O.shape(nf, 2))
    O.prolong(U, Unew, nc, 0.0, Uf, nf, [-4, -4, 0], [nf[0] + 4, nf[1] + 4, 1], origin, 2, 2)
    for q in range(2):
        Ufn, bad = O.mhd_step(Uf, nf, 2, [hf, hf, 1], dt / 2, ch, recon=1, windows=fw, reg=reg, kappa=kappa,
                              nu=nu)
        assert bad == 0
        Uf = Ufn.copy()
        for (l0, h0) in (((-4, -4), (0, nf[1] + 4)), ((nf[0], -4), (nf[0] + 4, nf[1] + 4)),
                         ((0, -4), (nf[0], 0)), ((0, nf[1]), (nf[0], nf[1] + 4))):
            O.prolong(U, Unew, nc, (q + 1) / 2, Uf, nf, [l0[0], l0[1], 0], [h0[0], h0[1], 1], origin, 2, 2)
    O.restrict(Unew, nc, Uf, nf, [lo, lo, 0], [hi, hi, 1], origin, 2, 2)
    no_reflux = O.interior(Unew, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    fwin = {(w[0], w[1]): w for w in fw}
    for d, f, side, a0, a1, b0, b1, creg in sets:
        w = fwin[(d, 0 if side < 0 else nf[d])]
        O.reflux(Unew, nc, [hc, hc], reg, d, f, side, a0, a1, b0, b1, creg, w[6], 0, 0, w[3] - w[2],
                 w[5] - w[4], 2, 2)
    total = O.interior(Unew, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    scale = np.abs(O.interior(Unew, nc, 2)).sum(axis=(1, 2, 3)) * hc * hc
    assert np.all(np.abs(total - total0)[:8] <= 1e-13 * scale[:8]), (total - total0)
    assert np.abs(no_reflux - total0)[[1, 2, 4]].max() > 1e-8
