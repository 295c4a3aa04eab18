"""Pins of the SRMHD oracle (Section 2.2 equations, Section 3.3 predictor)."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W

G43 = 4.0 / 3.0


def _state(rng, lor_max=10.0, bmax=1.0):
    V = np.zeros(9)
    V[0] = 10 ** rng.uniform(-1, 1)
    lor = 10 ** rng.uniform(0, np.log10(lor_max))
    d = rng.normal(size=3)
    V[1:4] = d / np.linalg.norm(d) * np.sqrt(1 - 1 / lor ** 2)
    V[4] = V[0] * 10 ** rng.uniform(-2, 1)
    V[5:8] = rng.normal(size=3) * bmax
    V[8] = 0.05
    return V


def _flux(V, gamma, ch):
    """RMHD flux along x written from Eq. (rmhd)."""
    rho, vx, vy, vz, p, bx, by, bz, psi = V
    v = np.array([vx, vy, vz])
    B = np.array([bx, by, bz])
    lor2 = 1 / (1 - v @ v)
    w = rho + gamma / (gamma - 1) * p
    E = -np.cross(v, B)
    pt = p + 0.5 * (B @ B + E @ E)
    U = W.srmhd_cons([np.array(x) for x in V], gamma)
    m = U[1:4]
    F = np.zeros(9)
    F[0] = rho * np.sqrt(lor2) * vx
    F[1:4] = w * lor2 * vx * v - bx * B - E[0] * E
    F[1] += pt
    F[4] = m[0] - F[0]
    F[5] = psi
    F[6] = vx * by - bx * vy
    F[7] = vx * bz - bx * vz
    F[8] = ch * ch * bx
    return F


def test_recovery_roundtrip():
    rng = np.random.default_rng(0)
    for _ in range(500):
        V = _state(rng)
        U = O.srmhd_prim2cons(V, G43)
        V2, st = O.srmhd_cons2prim(U, G43)
        assert st == 0
        assert np.allclose(V2, V, rtol=1e-11, atol=1e-12)
    # the workload generator's conversion agrees with the oracle's
    V = _state(rng)
    assert np.allclose(W.srmhd_cons([np.array(x) for x in V], G43), O.srmhd_prim2cons(V, G43),
                       rtol=1e-14)


def test_signal_speeds():
    """B = 0: relativistic velocity addition (v +- c_s)/(1 +- v c_s).  B != 0:
    the bound encloses the largest and smallest roots of the exact
    magnetosonic quartic rho h (1 - c_s^2) a^4 - (1 - l^2)[(rho h c_s^2 + b^2)
    a^2 - c_s^2 B^2] = 0, a = gamma (l - v_x), B = b^x - l b^0 (Anile 1989),
    and stays subluminal."""
    for v in (0.0, 0.5, -0.9, 0.99):
        V = np.array([1.0, v, 0, 0, 0.7, 0, 0, 0, 0])
        cs = np.sqrt(G43 * 0.7 / (1 + 4 * 0.7))
        lm, lp = O.srmhd_fast_speeds(V, G43)
        assert lm == pytest.approx((v - cs) / (1 - v * cs), rel=1e-13, abs=1e-15)
        assert lp == pytest.approx((v + cs) / (1 + v * cs), rel=1e-13, abs=1e-15)
    rng = np.random.default_rng(1)
    for _ in range(200):
        V = _state(rng, bmax=2.0)
        rho, p = V[0], V[4]
        v = V[1:4]
        B = V[5:8]
        lor = 1 / np.sqrt(1 - v @ v)
        rh = rho + G43 / (G43 - 1) * p
        cs2 = G43 * p / rh
        b0 = lor * (v @ B)
        bvec = B / lor + b0 * v
        b2 = B @ B / lor ** 2 + (v @ B) ** 2

        def quart(l):
            a = lor * (l - v[0])
            Bq = bvec[0] - l * b0
            return rh * (1 - cs2) * a ** 4 - (1 - l * l) * ((rh * cs2 + b2) * a * a - cs2 * Bq * Bq)

        xs = np.linspace(-1, 1, 5)
        coef = np.polyfit(xs, [quart(x) for x in xs], 4)
        roots = np.roots(coef)
        roots = roots[np.abs(roots.imag) < 1e-9].real
        roots = roots[(roots > -1 - 1e-12) & (roots < 1 + 1e-12)]
        lm, lp = O.srmhd_fast_speeds(V, G43)
        assert -1 < lm <= roots.min() + 1e-9 and roots.max() - 1e-9 <= lp < 1


def test_riemann_consistency():
    rng = np.random.default_rng(2)
    for _ in range(100):
        V = _state(rng)
        F = O.srmhd_riemann(V, V, G43, 0.9)
        assert np.allclose(F, _flux(V, G43, 0.9), rtol=1e-11, atol=1e-11)


def _advect_run(N, axis_v=(0.6, 0.0, 0.0), ndim=1, T=None):
    """Density wave rho = 1 + 0.3 sin(2 pi x) carried by uniform v, p, B: an
    exact solution of Eq. (rmhd)."""
    n = [N, 1, 1] if ndim == 1 else [N, N, 1]
    x = (np.arange(N) + 0.5) / N
    if ndim == 1:
        ph = 2 * np.pi * x
        shp = (1, 1, N)
    else:
        X, Y = np.meshgrid(x, x, indexing="xy")
        ph = 2 * np.pi * (X + Y)
        shp = (1, N, N)
    rho = 1 + 0.3 * np.sin(ph)
    z = np.zeros_like(rho)
    vx, vy, vz = axis_v
    Vp = [rho, z + vx, z + vy, z + vz, z + 0.5, z + 0.3, z + 0.4, z + 0.2, z]
    U = np.zeros(O.shape(n, ndim))
    O.interior(U, n, ndim)[:] = W.srmhd_cons(Vp, G43).reshape((9,) + shp)
    period = 1.0 / abs(vx) if ndim == 1 else 1.0 / abs(vx + vy)
    U, t, _ = O.srmhd_run(U, n, ndim, [1.0 / N] * 3, 0, 0.4, t_end=period)
    R = O.interior(U, n, ndim)
    U0 = W.srmhd_cons(Vp, G43).reshape((9,) + shp)
    return np.abs(R - U0).sum(axis=(1, 2, 3)) / N ** ndim


def test_density_wave_second_order():
    e = [_advect_run(N)[0] for N in (32, 64, 128)]
    assert np.log2(e[1] / e[2]) > 1.8, e
    e2 = [_advect_run(N, axis_v=(0.3, 0.4, 0.1), ndim=2)[0] for N in (16, 32)]
    assert np.log2(e2[0] / e2[1]) > 1.6, e2


def test_uniform_state_and_conservation():
    n = [12, 12, 12]
    U = W.srmhd_jet_3d(12, seed=3, lorentz=3.0)
    Vc = np.array([1.2, 0.3, -0.5, 0.6, 0.4, 0.7, -0.2, 0.9, 0.0])
    u = O.srmhd_prim2cons(Vc, G43)
    Uu = np.broadcast_to(u[:, None, None, None], U.shape).copy()
    Uu[8] = 0.3
    dx = [1 / 12] * 3
    dt, ch = O.dt_ch(O.srmhd_max_speed(Uu, n, 3, dx), dx, 3, 0.3)
    Un, bad = O.srmhd_step(Uu, n, 3, dx, dt, ch, glm_alpha=0.2)
    assert bad == 0
    I = O.interior(Un, n, 3)
    assert np.allclose(I[:8], O.interior(Uu, n, 3)[:8], rtol=1e-14, atol=1e-15)
    assert np.allclose(I[8], 0.3 * np.exp(-0.2 * ch * dt / dx[0]), rtol=1e-14)
    # conservation on the periodic jet box
    S0 = O.interior(U, n, 3).sum(axis=(1, 2, 3))
    scale = np.abs(O.interior(U, n, 3)).sum(axis=(1, 2, 3))
    U2, t, _ = O.srmhd_run(U, n, 3, dx, 3, 0.3)
    S = O.interior(U2, n, 3).sum(axis=(1, 2, 3))
    assert np.all(np.abs(S - S0)[:8] <= 1e-12 * np.maximum(scale[:8], 1e-3 * scale.max()))


def test_mirror_symmetry():
    n = [16, 16, 1]
    x = (np.arange(16) + 0.5) / 16
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = 1 + 0.5 * np.exp(-40 * ((X - 0.5) ** 2 + (Y - 0.3) ** 2))
    z = np.zeros_like(rho)
    Vp = [rho, 0.5 * np.sin(2 * np.pi * X), 0.3 * np.cos(2 * np.pi * Y), z, 0.2 + z,
          0.3 * np.cos(2 * np.pi * Y), 0.2 + z, z, z]
    U = np.zeros(O.shape(n, 2))
    O.interior(U, n, 2)[:] = W.srmhd_cons(Vp, G43)[:, None]

    def run(U):
        return O.interior(O.srmhd_run(U, n, 2, [1 / 16] * 3, 4, 0.4)[0], n, 2)

    ref = run(U)
    M = U[..., ::-1].copy()
    M[1] *= -1
    M[5] *= -1
    out = run(M)[..., ::-1].copy()
    out[1] *= -1
    out[5] *= -1
    scale = np.abs(ref).max(axis=(1, 2, 3))[:, None, None, None]
    assert np.all(np.abs(out - ref) <= 1e-12 * scale)
