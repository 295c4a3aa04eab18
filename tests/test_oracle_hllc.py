"""Pins of the oracle's HLLC solver for MHD (Li 2005), `riemann = CTU_HLLC`:
consistency R(V, V) = F(V); the hydrodynamic limit (B = 0), where HLLD
reduces to HLLC and the two solvers must agree flux for flux; an exact
stationary contact; supersonic upwinding; and, in the step, second-order
convergence of travelling linear waves and first-order convergence to the
exact Sod solution."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.mhd_setup import oblique_wave_2d

G = 5.0 / 3.0


def _rand(rng, b=1.0):
    return np.array([rng.uniform(0.5, 2), *rng.normal(0, 1, 3), rng.uniform(0.5, 2), *rng.normal(0, b, 3),
                     rng.normal(0, 0.1)])


def test_consistency():
    rng = np.random.default_rng(0)
    for _ in range(50):
        V = _rand(rng)
        assert np.allclose(O.mhd_riemann_hllc(V, V, G, 1.3), O.mhd_riemann(V, V, G, 1.3), rtol=1e-13, atol=1e-13)


def test_hydro_limit_equals_hlld():
    rng = np.random.default_rng(1)
    for _ in range(200):
        VL, VR = _rand(rng, 0.0), _rand(rng, 0.0)
        VL[8] = VR[8] = 0.0
        a = O.mhd_riemann_hllc(VL, VR, 1.4, 1.0)
        b = O.mhd_riemann(VL, VR, 1.4, 1.0)
        assert np.allclose(a, b, rtol=1e-13, atol=1e-13)


def test_stationary_contact_and_upwinding():
    VL = np.array([1.0, 0.0, 0.3, -0.2, 1.0, 0.0, 0.0, 0.0, 0.0])
    VR = np.array([0.125, 0.0, 0.3, -0.2, 1.0, 0.0, 0.0, 0.0, 0.0])
    F = O.mhd_riemann_hllc(VL, VR, 1.4, 1.0)
    assert F[0] == 0.0 and F[1] == pytest.approx(1.0, abs=1e-15)
    VL = np.array([1.0, 20.0, 0.1, 0.0, 1.0, 0.5, 0.3, 0.2, 0.0])
    VR = np.array([0.5, 19.0, -0.1, 0.1, 0.8, 0.5, 0.1, 0.2, 0.0])
    F = O.mhd_riemann_hllc(VL, VR, G, 1.0)
    assert np.allclose(F[[0, 1, 2, 3, 4, 6, 7]], O.mhd_riemann(VL, VL, G, 1.0)[[0, 1, 2, 3, 4, 6, 7]],
                       rtol=1e-14)


@pytest.mark.parametrize("wave", ["fast", "alfven", "entropy"])
def test_travelling_waves_second_order(wave):
    errs = []
    for N in (16, 32, 64):
        U, U0, T = oblique_wave_2d(N, wave)
        n = [N, N, 1]
        U, t, _ = O.mhd_run(U, n, 2, [1.0 / N, 1.0 / N, 1.0], 0, 0.4, recon=1, t_end=T, riemann=2)
        errs.append(np.abs(O.interior(U, n, 2) - U0).sum() / 1e-6 / (N * N))
    assert np.log2(errs[1] / errs[2]) > 1.8, errs


def test_sod():
    g = 1.4
    errs = []
    for N in (50, 100, 200):
        n = [N, 1, 1]
        x = (np.arange(N) + 0.5) / N
        rho = np.where(x < 0.5, 1.0, 0.125)[None, None, :]
        p = np.where(x < 0.5, 1.0, 0.1)[None, None, :]
        z = np.zeros_like(rho)
        U = np.zeros(O.shape(n, 1))
        O.interior(U, n, 1)[:] = W.ideal_cons([rho, z, z, z, p, z, z, z, z], g)
        U, t, _ = O.mhd_run(U, n, 1, [1.0 / N, 1.0, 1.0], 0, 0.8, gamma=g, recon=1, bc="outflow", t_end=0.2,
                            riemann=2)
        ex = O.euler_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, (x - 0.5) / t)[:, 0]
        errs.append(np.abs(O.interior(U, n, 1)[0].ravel() - ex).mean())
    assert 0.7 < np.log2(errs[0] / errs[-1]) / 2 < 1.4 and errs[-1] < 6e-3, errs
