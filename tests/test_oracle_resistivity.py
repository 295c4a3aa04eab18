"""Pins of the oracle's resistivity, the parabolic term of the CTU step for
the induction term -curl(eta J), J = curl B, with constant eta and its energy
flux -eta J x B (Section 2.1.1; Section 3.1 with Pi != 0): the flux of B_i
along d is eta (dB_i/dx_d - dB_d/dx_i), face values by central differences
with the transverse derivatives averaged over the two cells of the face,
and the energy flux is B_f times it, B_f the mean of the two cells.

- The discrete operator in closed form on polynomial fields: a quadratic B_y
  (eta B_y'' and the exact discrete energy flux), a quadratic normal
  component (no flux of B_d along d), a bilinear field (the transverse term:
  L_P(B_x) = -eta b for B = (0, b x y, 0)).
- The rate of Eq. Ca with D = eta.
- Conservation of B and energy on periodic boxes.
- A stationary diffusion mode against the exact decay of the discrete
  operator (resistivity-dominated, second-order time integration).
- Second-order space-time convergence to exact linear solutions: an
  advected diffusion mode (1-D), an oblique divergence-free mode (2-D, the
  cross terms) and a resistively damped Alfven wave (matrix exponential).
- Two levels with reflux conserve B and energy with the parabolic fluxes in
  the registers.
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


def _U(n, ndim, B, v=(0.0, 0.0, 0.0), rho=1.0, p=1.0):
    z = np.zeros(O.shape(n, ndim)[1:])
    return W.ideal_cons([rho + z, v[0] + z, v[1] + z, v[2] + z, p + z, B[0] + z, B[1] + z, B[2] + z, z], G)


def test_quadratic_field_and_its_energy_flux():
    n = [16, 1, 1]
    h = 1.0 / 16
    x = _centres(n, 1, 0)
    a, eta = 0.8, 0.05
    U = _U(n, 1, (0.2, a * x ** 2, 0.0), v=(0.3, 0.1, 0.0))
    LP = O.interior(O.mhd_parabolic(U, n, 1, [h], 0.0, 0.0, G, eta=eta), n, 1)
    xi = O.interior(x[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0]
    assert np.allclose(LP[6], eta * 2 * a, rtol=0, atol=1e-11)
    assert np.allclose(LP[5], 0.0, atol=1e-12) and np.allclose(LP[7], 0.0, atol=1e-12)
    assert np.allclose(LP[1:4], 0.0, atol=1e-12)
    # B_f = a (x_f^2 + h^2/4), flux 2 a eta x_f: the energy difference is
    # 2 a^2 eta (3 x^2 + h^2/2)
    assert np.allclose(LP[4], 2 * a * a * eta * (3 * xi ** 2 + h * h / 2), rtol=1e-12, atol=1e-12)


def test_normal_component_has_no_flux():
    n = [16, 1, 1]
    x = _centres(n, 1, 0)
    U = _U(n, 1, (0.5 + 0.7 * x ** 2, 0.1, 0.0))
    LP = O.interior(O.mhd_parabolic(U, n, 1, [1.0 / 16], 0.0, 0.0, G, eta=0.04), n, 1)
    assert np.allclose(LP[5:8], 0.0, atol=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
def test_bilinear_field_transverse_term(ndim):
    """B = (0, b x y, 0): L_P(B_x) = d_y [eta (dB_x/dy - dB_y/dx)] = -eta b,
    L_P(B_y) = d_x [eta (dB_y/dx - dB_x/dy)] = 0."""
    n = [10, 12, 6 if ndim > 2 else 1]
    x, y = _centres(n, ndim, 0), _centres(n, ndim, 1)
    b, eta = 0.9, 0.04
    U = _U(n, ndim, (0.0, b * x * y, 0.0))
    dx = [1.0 / n[d] for d in range(ndim)]
    LP = O.interior(O.mhd_parabolic(U, n, ndim, dx, 0.0, 0.0, G, eta=eta), n, ndim)
    assert np.allclose(LP[5], -eta * b, rtol=0, atol=1e-11)
    assert np.allclose(LP[6], 0.0, atol=1e-11) and np.allclose(LP[7], 0.0, atol=1e-12)


def test_max_rate_closed_form():
    n = [8, 8, 8]
    rho, p, eta = 2.0, 3.0, 0.07
    U = _U(n, 3, (0.0, 0.0, 0.0), rho=rho, p=p)
    dx = [0.1, 0.2, 0.05]
    want = np.sqrt(G * p / rho) / min(dx) + sum(2 * eta / h ** 2 for h in dx)
    assert O.mhd_max_rate(U, n, 3, dx, G, eta=eta) == pytest.approx(want, rel=1e-14)
    nu = 0.06  # (4/3) nu = 0.08 > eta
    want = np.sqrt(G * p / rho) / min(dx) + sum(2 * 4 / 3 * nu / h ** 2 for h in dx)
    assert O.mhd_max_rate(U, n, 3, dx, G, 0.0, nu, eta) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("ndim", [2, 3])
def test_conservation_periodic(ndim):
    N = 16
    n = [N, N, N if ndim > 2 else 1]
    U = W.mhd_blast_3d(N, seed=3) if ndim == 3 else W.mhd_turb_2d(N, seed=3)
    dx = [1.0 / N] * ndim
    a = O.interior(U, n, ndim).copy()
    R, t, _ = O.mhd_run(U, n, ndim, dx, 6, 0.3, recon=1, eta=0.01)
    b = O.interior(R, n, ndim)
    for q in range(8):
        assert abs(b[q].sum() - a[q].sum()) <= 1e-13 * (np.abs(a[q]).sum() + 1.0), q
    R0, _, _ = O.mhd_run(U, n, ndim, dx, 6, 0.3, recon=1)
    assert np.abs(O.interior(R0, n, ndim)[5:8] - b[5:8]).max() > 1e-6


def test_stationary_mode_semi_discrete_decay():
    """B = (0, eps sin(k x), 0) at rest: the hyperbolic part leaves it
    unchanged at linear order, so B_y follows exp(-eta k_h^2 t) to the
    time-integration error."""
    N, eta, eps, t_end = 32, 0.05, 1e-6, 0.5
    n = [N, 1, 1]
    x = _centres(n, 1, 0)
    U = _U(n, 1, (0.0, eps * np.sin(2 * np.pi * x), 0.0))
    R, t, _ = O.mhd_run(U, n, 1, [1.0 / N], None, 0.4, recon=1, t_end=t_end, eta=eta)
    h = 1.0 / N
    kh2 = 4.0 / h ** 2 * np.sin(np.pi * h) ** 2
    xi = O.interior(x[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0, 0, 0]
    ex = eps * np.sin(2 * np.pi * xi) * np.exp(-eta * kh2 * t)
    assert np.exp(-eta * kh2 * t) < 0.7
    assert np.abs(O.interior(R, n, 1)[6, 0, 0] - ex).max() < 3e-4 * eps


def _mode_error(N, ndim, eta, t_end):
    eps, v0 = 1e-6, 0.3
    n = [N, N if ndim > 1 else 1, 1]
    if ndim == 1:
        ph = 2 * np.pi * _centres(n, 1, 0)
        U = _U(n, 1, (0.0, eps * np.sin(ph), 0.0), v=(v0, 0.0, 0.0))
    else:
        ph = 2 * np.pi * (_centres(n, 2, 0) + _centres(n, 2, 1))
        s = eps * np.sin(ph) / np.sqrt(2)  # B along (-1, 1)/sqrt(2): divergence-free
        U = _U(n, 2, (-s, s, 0.0), v=(v0 / np.sqrt(2), v0 / np.sqrt(2), 0.0))
    dx = [1.0 / N] * ndim
    R, t, _ = O.mhd_run(U, n, ndim, dx, None, 0.4, recon=1, t_end=t_end, eta=eta)
    k = 2 * np.pi * np.sqrt(ndim)
    Ui = O.interior(R, n, ndim)
    b = Ui[6] if ndim == 1 else (-Ui[5] + Ui[6]) / np.sqrt(2)
    phi = O.interior(ph[None] + np.zeros((1,) + U.shape[1:]), n, ndim)[0]
    ex = eps * np.sin(phi - k * v0 * t) * np.exp(-eta * k * k * t)
    return np.abs(b - ex).mean() / eps


def test_advected_mode_second_order_1d():
    e = [_mode_error(N, 1, 0.004, 1.0) for N in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.9, (e, orders)


def test_oblique_mode_second_order_2d():
    eta = 0.002
    e = [_mode_error(N, 2, eta, 0.5) for N in (16, 32, 64)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.8, (e, orders)
    assert np.exp(-eta * 8 * np.pi ** 2 * 0.5) < 0.95


def _alfven_error(N, eta, t_end):
    """B = (1, eps cos(k x), 0) at rest, rho = p = 1: the linearised system
    v_y' = i k B_x B_y / rho, B_y' = i k B_x v_y - eta k^2 B_y."""
    n = [N, 1, 1]
    x = _centres(n, 1, 0)
    eps, k = 1e-6, 2 * np.pi
    U = _U(n, 1, (1.0, eps * np.cos(k * x), 0.0))
    R, t, _ = O.mhd_run(U, n, 1, [1.0 / N], None, 0.4, recon=1, t_end=t_end, eta=eta)
    M = np.array([[0, 1j * k], [1j * k, -eta * k * k]])
    a = expm(M * t) @ np.array([0.0, 1.0])
    xi = O.interior(x[None] + np.zeros((1,) + U.shape[1:]), n, 1)[0, 0, 0]
    ex = eps * np.real(a[1] * np.exp(1j * k * xi))
    return np.abs(O.interior(R, n, 1)[6, 0, 0] - ex).mean() / eps, abs(a[1])


def test_damped_alfven_wave_second_order():
    res = [_alfven_error(N, 0.005, 1.0) for N in (32, 64, 128)]
    e = [r[0] for r in res]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.9, (e, orders)


def test_reflux_with_resistivity_restores_conservation_of_two_levels():
    Nc = 32
    nc = [Nc, Nc, 1]
    hc = 1.0 / Nc
    hf = hc / 2
    eta, nu = 0.002, 0.001
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
    dt, ch = O.dt_ch(O.mhd_max_rate(U, nc, 2, [hc, hc], G, 0.0, nu, eta), [hc, hc], 2, 0.4)
    Unew, bad = O.mhd_step(U, nc, 2, [hc, hc, 1], dt, ch, recon=1, windows=cw, reg=reg, nu=nu, eta=eta)
    assert bad == 0
    origin = [lo, lo, 0]
    Uf = np.zeros(O.shape(nf, 2))
    O.prolong(U, Unew, nc, 0.0, Uf, nf, [-4, -4, 0], [nf[0] + 4, nf[1] + 4, 1], origin, 2, 2)
    for q in range(2):
        Ufn, bad = O.mhd_step(Uf, nf, 2, [hf, hf, 1], dt / 2, ch, recon=1, windows=fw, reg=reg, nu=nu, eta=eta)
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
    assert np.abs(no_reflux - total0)[[4, 5, 6]].max() > 1e-8
