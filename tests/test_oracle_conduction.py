"""Pins of the oracle's thermal conduction, the parabolic term of the CTU
step (Section 3.1 with Pi != 0; classical isotropic flux Pi_E = kappa grad T,
T = p / rho; diffusion term of Eq. Ca).

- The discrete operator in closed form: L_P of a quadratic temperature is
  kappa times its exact Laplacian; of a sinusoid, kappa times the symbol
  -(4/dx^2) sin^2(k dx/2) of the three-point second difference.  The density
  varies across the sinusoid's direction with p = rho T, so a flux built
  from p or from the specific internal energy fails.
- The time step of Eq. (Ca): the hyperbolic term plus 2 (Gamma-1) kappa /
  (rho dx^2) per dimension, in closed form for a uniform gas at rest.
- Conservation on periodic boxes: the parabolic flux telescopes.
- Space-time convergence at second order to the exact solution of the
  linearised Euler equations with conduction (matrix exponential of the
  3x3 mode system written from the PDE) in 1-D and obliquely in 2-D.  The
  time step is set by the hyperbolic CFL term (dt ~ dx), so a parabolic term
  lagged to t^n in the update, or missing from the predictor, shows as first
  order in time.
- The same linear system in the conduction-dominated regime, with the
  three-point symbol in place of k^2: the time integration of the parabolic
  term is second order (a forward-Euler parabolic term misses by 10x).
- Two levels (a fine patch in a periodic coarse one, two substeps): with
  the parabolic flux in the flux registers, reflux restores conservation to
  round-off; without reflux it does not.
- A vanishing conductivity takes the conduction code path and reproduces
  the plain step bit for bit.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle as O
from paper_1110_0740_gb300 import workloads as W

G = 5.0 / 3.0


def _prim_to_U(n, ndim, rho, vx, p, B=(0.0, 0.0, 0.0), vy=None):
    z = np.zeros_like(rho)
    vy = z if vy is None else vy
    return W.ideal_cons([rho, vx + z, vy + z, z, p, z + B[0], z + B[1], z + B[2], z], G)


def _centres(n, ndim, d):
    g = O.ghosts(ndim)
    shp = O.shape(n, ndim)
    x = (np.arange(shp[3 - d]) - g[d] + 0.5) / n[d]
    view = [1, 1, 1]
    view[2 - d] = shp[3 - d]
    return x.reshape(view)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_quadratic_temperature_exact_laplacian(ndim):
    n = [12, 10 if ndim > 1 else 1, 8 if ndim > 2 else 1]
    coef = [0.7, -0.4, 0.25][:ndim]
    shp = O.shape(n, ndim)
    T = np.ones(shp[1:])
    for d in range(ndim):
        T = T + coef[d] * _centres(n, ndim, d) ** 2
    rho = 1.0 + 0.0 * T
    U = _prim_to_U(n, ndim, rho, 0.0, rho * T, B=(0.3, 0.2, 0.1))
    kappa = 0.37
    dx = [1.0 / n[d] for d in range(ndim)]
    LP = O.interior(O.mhd_conduction(U, n, ndim, dx, kappa, G), n, ndim)
    assert np.allclose(LP, kappa * 2.0 * sum(coef), rtol=0, atol=2e-10)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_sinusoid_symbol_with_varying_density(ndim):
    n = [16, 8, 8][:ndim] + [1] * (3 - ndim)
    d0 = ndim - 1  # the sinusoid runs along the last active axis
    shp = O.shape(n, ndim)
    k = 2 * np.pi * 3
    xs = _centres(n, ndim, d0)
    eps = 0.05
    T = 1.0 + eps * np.sin(k * xs) + np.zeros(shp[1:])
    rho = 1.0 + np.zeros(shp[1:])
    if ndim > 1:
        rho = rho + 0.4 * np.cos(2 * np.pi * _centres(n, ndim, 0))
    U = _prim_to_U(n, ndim, rho, 0.0, rho * T)
    kappa = 0.2
    dx = [1.0 / n[d] for d in range(ndim)]
    LP = O.interior(O.mhd_conduction(U, n, ndim, dx, kappa, G), n, ndim)
    h = dx[d0]
    want = -kappa * 4.0 / h ** 2 * np.sin(k * h / 2) ** 2 * eps * np.sin(k * xs)
    want = O.interior(want + np.zeros(shp[1:]), n, ndim)
    assert np.allclose(LP, want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_max_rate_closed_form():
    n = [8, 8, 8]
    rho, p, kappa = 2.0, 3.0, 0.05
    shp = O.shape(n, 3)
    U = _prim_to_U(n, 3, rho + np.zeros(shp[1:]), 0.0, p)
    dx = [0.1, 0.2, 0.05]
    cs = np.sqrt(G * p / rho)
    D = (G - 1) * kappa / rho
    want = cs / min(dx) + sum(2 * D / h ** 2 for h in dx)
    assert O.mhd_max_rate(U, n, 3, dx, G, kappa) == pytest.approx(want, rel=1e-14)
    assert O.mhd_max_rate(U, n, 3, dx, G, 0.0) == O.mhd_max_speed(U, n, 3, dx, G)


@pytest.mark.parametrize("ndim", [2, 3])
def test_conservation_periodic(ndim):
    N = 16
    n = [N, N, N if ndim > 2 else 1]
    if ndim == 3:
        U = W.mhd_blast_3d(N, seed=3)
    else:
        U = W.mhd_turb_2d(N, seed=3)
    dx = [1.0 / N] * ndim
    a = O.interior(U, n, ndim).copy()
    R, t, _ = O.mhd_run(U, n, ndim, dx, 6, 0.3, recon=1, kappa=0.02)
    b = O.interior(R, n, ndim)
    for q in range(8):
        assert abs(b[q].sum() - a[q].sum()) <= 1e-13 * (np.abs(a[q]).sum() + 1.0), q
    # conduction changed the solution
    R0, _, _ = O.mhd_run(U, n, ndim, dx, 6, 0.3, recon=1)
    assert np.abs(O.interior(R0, n, ndim)[4] - b[4]).max() > 1e-6


def _linear_mode(n, ndim, kappa, eps, v0):
    """Entropy perturbation of a uniform gas (rho0 = p0 = 1, B = 0) moving with
    speed v0 along the wave vector (1, 0) in 1-D or (1, 1) in 2-D."""
    shp = O.shape(n, ndim)
    kv = np.array([1.0, 1.0][:ndim]) * 2 * np.pi
    phase = np.zeros(shp[1:])
    for d in range(ndim):
        phase = phase + kv[d] * _centres(n, ndim, d)
    nh = kv / np.linalg.norm(kv)
    rho = 1.0 + eps * np.cos(phase)
    vx = v0 * nh[0] + 0 * phase
    vy = v0 * nh[1] + 0 * phase if ndim > 1 else None
    return _prim_to_U(n, ndim, rho, vx, 1.0 + 0 * phase, vy=vy), kv, phase


def _exact_rho(kv, phase, t, kappa, eps, v0):
    """rho of the linearised Euler equations with conduction: for a mode
    exp(i k.x) with k = |kv| along the flow,
      rho_t = -i k v0 rho - i k rho0 u,   u_t = -i k v0 u - i k p / rho0,
      p_t = -i k v0 p - i k Gamma p0 u - (Gamma-1) kappa k^2 T,
      T = p / rho0 - p0 rho / rho0^2."""
    k = np.linalg.norm(kv)
    r0 = p0 = 1.0
    M = np.array([
        [-1j * k * v0, -1j * k * r0, 0],
        [0, -1j * k * v0, -1j * k / r0],
        [(G - 1) * kappa * k * k * p0 / r0 ** 2, -1j * k * G * p0, -1j * k * v0 - (G - 1) * kappa * k * k / r0],
    ])
    a = expm(M * t) @ np.array([1.0, 0.0, 0.0])
    return 1.0 + eps * np.real(a[0] * np.exp(1j * phase))


def _l1_error(N, ndim, kappa, t_end, cfl):
    n = [N, N if ndim > 1 else 1, 1]
    eps, v0 = 1e-6, 0.3
    U, kv, phase = _linear_mode(n, ndim, kappa, eps, v0)
    dx = [1.0 / N] * ndim
    R, t, _ = O.mhd_run(U, n, ndim, dx, None, cfl, recon=1, t_end=t_end, kappa=kappa)
    ex = O.interior(_exact_rho(kv, phase, t, kappa, eps, v0)[None], n, ndim)[0]
    return np.abs(O.interior(R, n, ndim)[0] - ex).mean() / eps


def test_linear_mode_second_order_1d():
    # D = (Gamma-1) kappa = 0.004: k^2 D t = 0.16 at t = 1, and the CFL step
    # is set by the hyperbolic term at every resolution below (dt ~ dx)
    kappa = 0.006
    e = [_l1_error(N, 1, kappa, 1.0, 0.4) for N in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.9, (e, orders)
    assert e[-1] < 2e-3
    # conduction is visible: the kappa = 0 solution is far from the exact one
    n = [128, 1, 1]
    U, kv, phase = _linear_mode(n, 1, kappa, 1e-6, 0.3)
    R, t, _ = O.mhd_run(U, n, 1, [1.0 / 128], None, 0.4, recon=1, t_end=1.0)
    ex = O.interior(_exact_rho(kv, phase, t, kappa, 1e-6, 0.3)[None], n, 1)[0]
    assert np.abs(O.interior(R, n, 1)[0] - ex).mean() / 1e-6 > 20 * e[-1]


def test_linear_mode_second_order_2d_oblique():
    kappa = 0.004
    e = [_l1_error(N, 2, kappa, 0.5, 0.4) for N in (16, 32, 64)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.8, (e, orders)


def test_strong_conduction_time_integration():
    """Conduction-dominated regime (D k^2 = 20 c k): over t = 1/80 the
    temperature mode decays by e^-2 while sound travels a tenth of a radian,
    and the CFL step is set by the diffusion term (dt D k_h^2 = 0.008 per
    step).  Reference: the linearised system above with the conduction terms'
    k^2 replaced by the symbol (4/dx^2) sin^2(k dx/2) of the three-point
    second difference, i.e. the exact time evolution of the spatially
    discrete conduction operator.  The pressure mode then matches to 6e-5 of
    the perturbation at 32 cells; a parabolic term integrated at first order
    in time (forward Euler: L_P at n+1/2 from a half-step state without L_P^n,
    or L_P^n in the update) misses by 6e-4 or more."""
    N, kappa, t_end, eps = 32, 6.0, 0.0125, 1e-6
    n = [N, 1, 1]
    U, kv, phase = _linear_mode(n, 1, kappa, eps, 0.0)
    R, t, _ = O.mhd_run(U, n, 1, [1.0 / N], None, 0.4, recon=1, t_end=t_end, kappa=kappa)
    k, h = kv[0], 1.0 / N
    kd2 = 4.0 / h ** 2 * np.sin(k * h / 2) ** 2
    M = np.array([[0, -1j * k, 0], [0, 0, -1j * k], [(G - 1) * kappa * kd2, -1j * k * G, -(G - 1) * kappa * kd2]])
    a = expm(M * t) @ np.array([1.0, 0.0, 0.0])
    Ui = O.interior(R, n, 1)[:, 0, 0, :]
    p = (G - 1) * (Ui[4] - 0.5 * (Ui[1] ** 2 + Ui[2] ** 2 + Ui[3] ** 2) / Ui[0]
                   - 0.5 * (Ui[5] ** 2 + Ui[6] ** 2 + Ui[7] ** 2))
    x = (np.arange(N) + 0.5) / N
    pex = 1.0 + eps * np.real(a[2] * np.exp(1j * k * x))
    assert abs(a[2]) > 0.8  # the pressure mode the conduction drives
    assert np.abs(p - pex).mean() / eps < 1.5e-4


def test_vanishing_kappa_is_the_plain_step():
    """A conductivity far below round-off of the state takes the conduction
    code path (wider first-order stage, half-step state) and changes no bit."""
    N = 12
    n = [N, N, 1]
    U = W.mhd_turb_2d(N, seed=5)
    O.fill_periodic(U, n, 2)
    dx = [1.0 / N] * 2
    dt, ch = O.dt_ch(O.mhd_max_speed(U, n, 2, dx), dx, 2, 0.3)
    a, _ = O.mhd_step(U, n, 2, dx, dt, ch, recon=1)
    b, _ = O.mhd_step(U, n, 2, dx, dt, ch, recon=1, kappa=1e-300)
    assert np.array_equal(a, b)


def test_reflux_with_conduction_restores_conservation_of_two_levels():
    """The two-level case of the AMR pins with conduction: the registers take
    F_E - Pi_E^(n+1/2), and restriction plus reflux conserve the totals to
    round-off; the energy without reflux misses by far more."""
    Nc = 32
    nc = [Nc, Nc, 1]
    hc = 1.0 / Nc
    hf = hc / 2
    kappa = 0.002
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
    dt, ch = O.dt_ch(O.mhd_max_rate(U, nc, 2, [hc, hc], G, kappa), [hc, hc], 2, 0.4)
    Unew, bad = O.mhd_step(U, nc, 2, [hc, hc, 1], dt, ch, recon=1, windows=cw, reg=reg, kappa=kappa)
    assert bad == 0
    origin = [lo, lo, 0]
    Uf = np.zeros(O.shape(nf, 2))
    O.prolong(U, Unew, nc, 0.0, Uf, nf, [-4, -4, 0], [nf[0] + 4, nf[1] + 4, 1], origin, 2, 2)
    for q in range(2):
        Ufn, bad = O.mhd_step(Uf, nf, 2, [hf, hf, 1], dt / 2, ch, recon=1, windows=fw, reg=reg, kappa=kappa)
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
    assert np.abs(no_reflux - total0)[4] > 1e-8


# ------------------------------------------------------------ anisotropic flux
# F_class = kappa_par b (b . grad T) + kappa_perp (grad T - b (b . grad T)) of
# Eq. (tc_flux), b = B / |B| at the face (the mean of the two cells).

@pytest.mark.parametrize("ndim", [2, 3])
def test_anisotropic_field_along_x_closed_form(ndim):
    """B along x, T = 1 + a x^2 + c y^2 (+ e z^2): the flux along x is
    kappa_par dT/dx and across it kappa_perp dT/dy, so
    L_P = kappa_par 2a + kappa_perp (2c + 2e), exactly."""
    n = [12, 10, 8 if ndim > 2 else 1]
    a, c, e = 0.6, -0.3, 0.2
    shp = O.shape(n, ndim)
    T = 1.0 + a * _centres(n, ndim, 0) ** 2 + c * _centres(n, ndim, 1) ** 2 + np.zeros(shp[1:])
    if ndim > 2:
        T = T + e * _centres(n, ndim, 2) ** 2
    rho = 1.0 + 0.0 * T
    U = _prim_to_U(n, ndim, rho, 0.0, rho * T, B=(0.7, 0.0, 0.0))
    kperp, kpar = 0.05, 0.8
    dx = [1.0 / n[d] for d in range(ndim)]
    LP = O.interior(O.mhd_parabolic(U, n, ndim, dx, kperp, 0.0, G, kappa_par=kpar), n, ndim)
    want = kpar * 2 * a + kperp * 2 * (c + (e if ndim > 2 else 0.0))
    assert np.allclose(LP[4], want, rtol=0, atol=1e-10)


def test_anisotropic_oblique_field_cross_terms():
    """B along (1, 1)/sqrt(2), T = 1 + c x y: div F = (kappa_par - kappa_perp) c,
    exactly (the transverse temperature derivatives at the faces)."""
    n = [12, 10, 1]
    c = 0.9
    shp = O.shape(n, 2)
    T = 1.0 + c * _centres(n, 2, 0) * _centres(n, 2, 1) + np.zeros(shp[1:])
    rho = 1.0 + 0.0 * T
    U = _prim_to_U(n, 2, rho, 0.0, rho * T, B=(0.5, 0.5, 0.0))
    kperp, kpar = 0.1, 0.7
    LP = O.interior(O.mhd_parabolic(U, n, 2, [1 / 12, 1 / 10], kperp, 0.0, G, kappa_par=kpar), n, 2)
    assert np.allclose(LP[4], (kpar - kperp) * c, rtol=0, atol=1e-11)


def test_anisotropic_equal_coefficients_is_isotropic():
    N = 12
    n = [N, N, 1]
    U = W.mhd_turb_2d(N, seed=7)
    O.fill_periodic(U, n, 2)
    dx = [1.0 / N] * 2
    dt, ch = O.dt_ch(O.mhd_max_rate(U, n, 2, dx, G, 0.02), dx, 2, 0.3)
    a, _ = O.mhd_step(U, n, 2, dx, dt, ch, recon=1, kappa=0.02)
    b, _ = O.mhd_step(U, n, 2, dx, dt, ch, recon=1, kappa=0.02, kappa_par=0.02, nu=1e-300)
    assert np.array_equal(a, b)
    # the rate takes the larger coefficient
    assert O.mhd_max_rate(U, n, 2, dx, G, 0.01, kappa_par=0.05) == pytest.approx(
        O.mhd_max_rate(U, n, 2, dx, G, 0.05), rel=1e-15)


@pytest.mark.parametrize("along", [True, False])
def test_anisotropic_mode_second_order(along):
    """A temperature mode along x with a uniform field along x (decays with
    kappa_par) or along y (kappa_perp): the linear system of the isotropic
    pins with that coefficient, second-order convergence."""
    kperp, kpar = 0.001, 0.006
    k_eff = kpar if along else kperp

    def err(N):
        n = [N, 1, 1]
        eps, v0 = 1e-6, 0.3
        U, kv, phase = _linear_mode(n, 1, k_eff, eps, v0)
        Bx, By = (1e-3, 0.0) if along else (0.0, 1e-3)
        Ui = U.copy()
        Ui[4] += 0.5 * (Bx * Bx + By * By)
        Ui[5] += Bx
        Ui[6] += By
        R, t, _ = O.mhd_run(Ui, n, 1, [1.0 / N], None, 0.4, recon=1, t_end=1.0, kappa=kperp, kappa_par=kpar)
        ex = O.interior(_exact_rho(kv, phase, t, k_eff, eps, v0)[None], n, 1)[0]
        return np.abs(O.interior(R, n, 1)[0] - ex).mean() / eps

    e = [err(N) for N in (32, 64, 128)]
    orders = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert orders[-1] > 1.9, (e, orders)
    assert e[-1] < 2e-3


def test_anisotropic_oblique_field_quadratic_closed_form():
    """B along (1, 1)/sqrt(2), T = 1 + c x^2 y: div F = 2 c kappa_perp y +
    (kappa_par - kappa_perp) c (y + 2 x), exactly: the transverse derivative
    of T at an x-face is the mean of the two cells' central differences
    (c x^2 is quadratic across the face)."""
    n = [12, 10, 1]
    c = 0.9
    shp = O.shape(n, 2)
    x, y = _centres(n, 2, 0), _centres(n, 2, 1)
    T = 1.0 + c * x * x * y + np.zeros(shp[1:])
    rho = 1.0 + 0.0 * T
    U = _prim_to_U(n, 2, rho, 0.0, rho * T, B=(0.5, 0.5, 0.0))
    kperp, kpar = 0.1, 0.7
    LP = O.interior(O.mhd_parabolic(U, n, 2, [1 / 12, 1 / 10], kperp, 0.0, G, kappa_par=kpar), n, 2)
    X = O.interior((x + 0 * T)[None], n, 2)[0]
    Y = O.interior((y + 0 * T)[None], n, 2)[0]
    want = 2 * c * kperp * Y + (kpar - kperp) * c * (Y + 2 * X)
    assert np.allclose(LP[4], want, rtol=0, atol=1e-11)


# ------------------------------------------------------------- saturated flux
# The paper's appendix on the heat flux: F_c = q F_class / (|F_class| + q) at
# each face, q = 5 phi p_u^(3/2) / sqrt(rho_f) with p_u upwind of F_class.

def test_saturation_off_in_the_classical_limit():
    """q >> |F_class| (phi huge): the harmonic mean is the classical flux."""
    N = 12
    n = [N, N, 1]
    U = W.mhd_turb_2d(N, seed=8)
    O.fill_periodic(U, n, 2)
    dx = [1.0 / N] * 2
    a = O.mhd_parabolic(U, n, 2, dx, 0.01, 0.0, G, kappa_par=0.05)
    b = O.mhd_parabolic(U, n, 2, dx, 0.01, 0.0, G, kappa_par=0.05, phi=1e30)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14 * np.abs(a).max())


@pytest.mark.parametrize("sign", [-1.0, 1.0])
def test_saturated_limit_upwind_closed_form(sign):
    """q << |F_class| (phi tiny): each face carries q in the direction of
    F_class, from the pressure of the upwind cell, so for T = 2 + s a x and
    rho = 1 + 0.3 x (p = rho T): L_P = 5 phi s (p_u(i+1/2)^1.5 / sqrt(rho_(i+1/2))
    - p_u(i-1/2)^1.5 / sqrt(rho_(i-1/2))) / dx, p_u the left cell's pressure
    for s < 0 and the right cell's for s > 0 (to a relative q/|F| ~ 1e-9)."""
    N = 16
    n = [N, 1, 1]
    h = 1.0 / N
    x = _centres(n, 1, 0)
    rho = 1.0 + 0.3 * x
    T = 2.0 + sign * 0.5 * x
    U = _prim_to_U(n, 1, rho + 0 * x, 0.0, rho * T)
    kappa, phi = 1.0, 1e-10
    LP = O.interior(O.mhd_parabolic(U, n, 1, [h], kappa, 0.0, G, phi=phi), n, 1)[4, 0, 0]
    p = (rho * T)[0, 0]
    r = rho[0, 0]
    g = 4
    i = np.arange(g, g + N)
    up = (i if sign < 0 else i + 1)      # the upwind cell of face i + 1/2
    um = (i - 1 if sign < 0 else i)      # of face i - 1/2
    qp = 5 * phi * p[up] ** 1.5 / np.sqrt(0.5 * (r[i] + r[i + 1]))
    qm = 5 * phi * p[um] ** 1.5 / np.sqrt(0.5 * (r[i - 1] + r[i]))
    want = sign * (qp - qm) / h
    assert np.allclose(LP, want, rtol=1e-7, atol=0)


def test_saturated_conservation_periodic():
    N = 16
    n = [N, N, 1]
    U = W.mhd_turb_2d(N, seed=9)
    dx = [1.0 / N] * 2
    a = O.interior(U, n, 2).copy()
    R, t, _ = O.mhd_run(U, n, 2, dx, 6, 0.3, recon=1, kappa=0.05, phi=0.05)
    b = O.interior(R, n, 2)
    for q in range(8):
        assert abs(b[q].sum() - a[q].sum()) <= 1e-13 * (np.abs(a[q]).sum() + 1.0), q
    R0, _, _ = O.mhd_run(U, n, 2, dx, 6, 0.3, recon=1, kappa=0.05)
    assert np.abs(O.interior(R0, n, 2)[4] - b[4]).max() > 1e-6


def test_saturated_harmonic_mean_uses_the_flux_vector():
    """2-D, T = 2 + a x + b y with p = 1 (rho = 1 / T): F_class = kappa (a, b)
    at every face, exactly, and in the intermediate regime (q ~ |F|) each face
    carries q F_d / (kappa sqrt(a^2 + b^2) + q), q = 5 phi / sqrt(rho_f)."""
    n = [12, 10, 1]
    dx = [1 / 12, 1 / 10]
    a, b, kappa = 0.6, -0.8, 1.0
    x, y = _centres(n, 2, 0), _centres(n, 2, 1)
    T = 2.0 + a * x + b * y + 0 * x * y
    rho = 1.0 / T
    U = _prim_to_U(n, 2, rho, 0.0, rho * T)
    fm = kappa * np.hypot(a, b)
    phi = fm / 7.0
    LP = O.interior(O.mhd_parabolic(U, n, 2, dx, kappa, 0.0, G, phi=phi), n, 2)[4, 0]
    r = rho[0]
    g = 4
    j, i = np.meshgrid(np.arange(g, g + n[1]), np.arange(g, g + n[0]), indexing="ij")

    def face(Fd, rl, rr):
        q = 5 * phi / np.sqrt(0.5 * (rl + rr))
        return q * Fd / (fm + q)

    want = ((face(kappa * a, r[j, i], r[j, i + 1]) - face(kappa * a, r[j, i - 1], r[j, i])) / dx[0]
            + (face(kappa * b, r[j, i], r[j + 1, i]) - face(kappa * b, r[j - 1, i], r[j, i])) / dx[1])
    assert np.allclose(LP, want, rtol=1e-10, atol=1e-12)
