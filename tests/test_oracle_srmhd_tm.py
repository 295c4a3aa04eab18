"""Pins of the oracle's Taub-Mathews equation of state, Eq. (TMEos), in the
relativistic MHD path (gam = 0 selects it):

- the primitive recovery inverts U(V) to 1e-11 up to Lorentz factor 10 and
  across temperatures p/rho from 1e-4 to 1e4;
- the enthalpy reduces to the ideal gas with Gamma = 5/3 for p << rho and
  with Gamma = 4/3 for p >> rho;
- the signal speeds at B = 0 equal the extreme eigenvalues of the hydro
  flux Jacobian dF/dU, formed by finite differences of the oracle's flux and
  U(V) and diagonalised by numpy (checks the sound speed formula against the
  equation of state itself);
- a density wave carried by uniform v, p and B (exact for any equation of
  state) converges at second order."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W

TM = 0.0


def _state(rng, theta, lor_max=10.0):
    lor = rng.uniform(1.0, lor_max)
    d = rng.normal(size=3)
    v = d / np.linalg.norm(d) * np.sqrt(1.0 - 1.0 / lor ** 2)
    rho = rng.uniform(0.5, 2.0)
    return np.array([rho, *v, theta * rho, *rng.normal(0, 1.0, 3), 0.0])


def test_recovery_roundtrip_tm():
    rng = np.random.default_rng(0)
    for theta in (1e-4, 1e-2, 1.0, 1e2, 1e4):
        for _ in range(20):
            V = _state(rng, theta)
            U = O.srmhd_prim2cons(V, TM)
            V2, st = O.srmhd_cons2prim(U, TM)
            assert st == 0
            assert np.allclose(V2, V, rtol=1e-10, atol=1e-11 * (1 + abs(V[4]))), (theta, V, V2)


def test_tm_limits():
    V = np.array([1.0, 0.3, 0.1, -0.2, 1e-7, 0.2, 0.1, 0.3, 0.0])
    a, b = O.srmhd_prim2cons(V, TM), O.srmhd_prim2cons(V, 5.0 / 3.0)
    assert np.allclose(a, b, rtol=1e-12, atol=0)
    V[0], V[4] = 1e-4, 1e4
    a, b = O.srmhd_prim2cons(V, TM), O.srmhd_prim2cons(V, 4.0 / 3.0)
    assert np.allclose(a, b, rtol=1e-8, atol=0)


def _hydro_jacobian_eigs(V, gam, h=1e-7):
    """Eigenvalues of dF/dU of the (D, m, E) block at B = 0, by central
    differences in (rho, v, p)."""
    def FU(Vv):
        F = O.srmhd_riemann(Vv, Vv, gam, 1.0)
        U = O.srmhd_prim2cons(Vv, gam)
        return F[:5], U[:5]
    dF = np.zeros((5, 5))
    dU = np.zeros((5, 5))
    for k in range(5):
        e = np.zeros(9)
        e[k] = h * max(1.0, abs(V[k]))
        Fp, Up = FU(V + e)
        Fm, Um = FU(V - e)
        dF[:, k] = (Fp - Fm) / (2 * e[k])
        dU[:, k] = (Up - Um) / (2 * e[k])
    return np.sort(np.linalg.eigvals(dF @ np.linalg.inv(dU)).real)


@pytest.mark.parametrize("gam", [TM, 4.0 / 3.0])
def test_signal_speeds_are_jacobian_eigenvalues(gam):
    rng = np.random.default_rng(3)
    for theta in (1e-2, 1.0, 30.0):
        for _ in range(5):
            V = _state(rng, theta, lor_max=3.0)
            V[5:8] = 0.0
            lam = _hydro_jacobian_eigs(V, gam)
            lm, lp = O.srmhd_fast_speeds(V, gam)
            assert lm == pytest.approx(lam[0], abs=2e-6) and lp == pytest.approx(lam[-1], abs=2e-6), (theta, lam)


def _advect(N):
    n = [N, 1, 1]
    x = (np.arange(N) + 0.5) / N
    rho = 1 + 0.3 * np.sin(2 * np.pi * x)
    z = np.zeros_like(rho)
    Vp = [rho, z + 0.6, z, z, z + 0.5, z + 0.3, z + 0.4, z + 0.2, z]
    U = np.zeros(O.shape(n, 1))
    O.interior(U, n, 1)[:] = W.srmhd_cons(Vp, TM).reshape(9, 1, 1, N)
    U, t, _ = O.srmhd_run(U, n, 1, [1.0 / N] * 3, 0, 0.4, gamma=TM, t_end=1.0 / 0.6)
    return np.abs(O.interior(U, n, 1)[0].ravel() - W.srmhd_cons(Vp, TM)[0]).mean()


def test_density_wave_second_order_tm():
    e = [_advect(N) for N in (32, 64, 128)]
    assert np.log2(e[1] / e[2]) > 1.8, e
