"""Pins of the oracle's other reconstructions (Section 3.2): the MinMod,
harmonic (harmonic_lim) and Van Albada (vanalbada_lim) slopes of the linear
reconstruction, and improved WENO3 (WENO3, WENO3a).

A stencil in which only the density varies (v = 0, p and B uniform) excites
only the entropy field, whose right eigenvector is the unit density
vector, so with dt = 0 the predictor's density interface values are the
reconstruction itself: closed forms of every limiter and of WENO3, the
other variables unchanged, exact reproduction of linear data, symmetry under
reflection, zero slope at an extremum (TVD limiters).  Then convergence of a
travelling linear eigenmode and the exact Sod solution for every choice."""
import numpy as np
import pytest

import oracle as O
from tests.mhd_setup import oblique_wave_2d

G = 5.0 / 3.0
V0 = np.array([1.0, 0.0, 0.0, 0.0, 0.6, 1.0, 1.4, 0.5, 0.0])
MINMOD, HARMONIC, VANALBADA, WENO3 = 2, 3, 4, 5


def _rho_interfaces(rho, recon, dx=0.1):
    vs = np.tile(V0, (5, 1))
    vs[:, 0] = rho
    Vp, Vm = O.mhd_char_predict(vs, G, 1.0, 0.0, recon, dx=dx)
    for V in (Vp, Vm):
        assert np.allclose(np.delete(V, 0), np.delete(V0, 0), rtol=0, atol=1e-15)
    return Vp[0], Vm[0]


def _slope(dm, dp, recon):
    """The limiters written from their equations, evaluated in closed form."""
    if dm * dp <= 0:
        return 0.0
    return {MINMOD: np.sign(dm) * min(abs(dm), abs(dp)), HARMONIC: 2 * dm * dp / (dm + dp),
            VANALBADA: dm * dp * (dm + dp) / (dm * dm + dp * dp)}[recon]


@pytest.mark.parametrize("recon", [MINMOD, HARMONIC, VANALBADA])
def test_limiter_closed_forms(recon):
    for dm, dp in ((0.01, 0.03), (0.03, 0.01), (-0.02, -0.005), (0.01, -0.02), (0.0, 0.4), (0.02, 0.02)):
        rho = [1.0 - 2 * dm, 1.0 - dm, 1.0, 1.0 + dp, 1.0 + 2 * dp]
        p, m = _rho_interfaces(rho, recon)
        s = _slope(dm, dp, recon)
        assert p == pytest.approx(1.0 + s / 2, abs=1e-15) and m == pytest.approx(1.0 - s / 2, abs=1e-15)
    # 1 : 3 slopes -- MinMod 1, Van Albada 1.2, harmonic 1.5, MC 2 (x 0.01)
    got = [(_rho_interfaces([0.98, 0.99, 1.0, 1.03, 1.06], r)) for r in (MINMOD, VANALBADA, HARMONIC, 0)]
    assert np.allclose([p - m for p, m in got], [0.01, 0.012, 0.015, 0.02], rtol=1e-12)


def test_weno3_closed_form_and_limits():
    dx = 0.05
    for dm, dp in ((0.01, 0.03), (0.04, -0.02), (0.0, 0.0), (0.3, 0.3)):
        rho = [1.0 - 2 * dm, 1.0 - dm, 1.0, 1.0 + dp, 1.0 + 2 * dp]
        p, m = _rho_interfaces(rho, WENO3, dx)
        d2 = (dp - dm) ** 2
        ap, am = 1 + d2 / (dx * dx + dp * dp), 1 + d2 / (dx * dx + dm * dm)
        assert p == pytest.approx(1.0 + (ap * dp + 0.5 * am * dm) / (2 * ap + am), abs=1e-15)
        assert m == pytest.approx(1.0 - (am * dm + 0.5 * ap * dp) / (2 * am + ap), abs=1e-15)
    # smooth data (|dw| << dx): the third-order interface value
    # (2 w_(i+1) + 5 w_i - w_(i-1)) / 6 and its mirror
    w = 1.0 + 1e-6 * np.array([-2.0, -1.0, 0.0, 1.5, 3.2]) ** 2
    p, m = _rho_interfaces(w, WENO3, 1.0)
    assert p == pytest.approx((2 * w[3] + 5 * w[2] - w[1]) / 6, abs=1e-14)
    assert m == pytest.approx((2 * w[1] + 5 * w[2] - w[3]) / 6, abs=1e-14)


@pytest.mark.parametrize("recon", [0, MINMOD, HARMONIC, VANALBADA, WENO3])
def test_linear_data_reflection_and_extrema(recon):
    # linear data: w_(+/-) = w_0 +/- slope/2 exactly
    p, m = _rho_interfaces([0.94, 0.97, 1.0, 1.03, 1.06], recon)
    assert p == pytest.approx(1.015, abs=1e-15) and m == pytest.approx(0.985, abs=1e-15)
    # reflection of the stencil swaps the two interfaces
    r = [0.9, 0.95, 1.0, 1.1, 1.3]
    p1, m1 = _rho_interfaces(r, recon)
    p2, m2 = _rho_interfaces(r[::-1], recon)
    assert p1 == pytest.approx(m2, abs=1e-15) and m1 == pytest.approx(p2, abs=1e-15)
    if recon != WENO3:  # TVD slopes vanish at an extremum
        p, m = _rho_interfaces([1.0, 1.05, 1.1, 1.02, 0.9], recon)
        assert p == m == 1.1


@pytest.mark.parametrize("recon,floor_", [(MINMOD, 1.5), (HARMONIC, 1.75), (VANALBADA, 1.75), (WENO3, 1.95)])
def test_travelling_eigenmode_converges(recon, floor_):
    """A fast mode travelling obliquely returns to its initial state after
    one period; the L1 error converges at the scheme's order (TVD limiters
    clip the extrema of the sine, so their order sits below 2)."""
    errs = []
    for N in (16, 32, 64):
        U, U0, T = oblique_wave_2d(N, "fast")
        n = [N, N, 1]
        U, t, _ = O.mhd_run(U, n, 2, [1.0 / N, 1.0 / N, 1.0], 0, 0.4, recon=recon, t_end=T)
        errs.append(np.abs(O.interior(U, n, 2) - U0).sum() / 1e-6 / (N * N))
    order = np.log2(errs[1] / errs[2])
    assert order > floor_, (errs, order)


@pytest.mark.parametrize("recon", [MINMOD, HARMONIC, VANALBADA, WENO3])
def test_sod_against_the_exact_solution(recon):
    """Sod's problem (B = 0) in 1-D: L1(rho) against Toro's exact solution
    decreases at about first order (the shock and contact are captured) and
    is small at N = 200, for every reconstruction."""
    from paper_1110_0740_gb300 import workloads as W
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
        U, t, _ = O.mhd_run(U, n, 1, [1.0 / N, 1.0, 1.0], 0, 0.8, gamma=g, recon=recon, bc="outflow", t_end=0.2)
        ex = O.euler_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, (x - 0.5) / t)[:, 0]
        errs.append(np.abs(O.interior(U, n, 1)[0].ravel() - ex).mean())
    order = np.log2(errs[0] / errs[-1]) / 2
    assert 0.7 < order < 1.4, errs
    assert errs[-1] < 6e-3, errs
