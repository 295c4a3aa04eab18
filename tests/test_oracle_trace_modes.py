"""Pins of the oracle's reference states of the characteristic tracing,
Eq. (wnorm_predp) and (wnorm_predm), Section 3.2: no reference state (mode 0,
every field traced to both interfaces), w_ref = w_(+/-) (1), the cell-centre
value w_(i,0) (2) and Colella-Woodward's nu_max / nu_min state (3), the last
three with the upwind selection beta_(+/-) = [+/-nu > 0].

A stencil in which only the density varies linearly excites only the
entropy field (speed u, unit density eigenvector), so the density interface
values are that field's traced values in closed form.  And the accuracy
Section 3.2 states: with a reference state the slow wave (which HLLD does not
resolve) converges at first order only; without one, at second order."""
import numpy as np
import pytest

import oracle as O
from tests.mhd_setup import oblique_wave_2d

G = 5.0 / 3.0


def _cf(V):
    a2 = G * V[4] / V[0]
    bn2, bt2 = V[5] ** 2 / V[0], (V[6] ** 2 + V[7] ** 2) / V[0]
    return np.sqrt(0.5 * (a2 + bn2 + bt2 + np.sqrt((a2 - bn2 - bt2) ** 2 + 4 * a2 * bt2)))


@pytest.mark.parametrize("u", [0.3, -0.3])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_entropy_field_closed_forms(mode, u):
    V0 = np.array([1.0, u, 0.0, 0.0, 0.6, 1.0, 1.4, 0.5, 0.0])
    d, dtdx = 0.01, 0.5
    vs = np.tile(V0, (5, 1))
    vs[:, 0] = 1.0 + d * np.arange(-2, 3)
    Vp, Vm = O.mhd_char_predict(vs, G, 1.0, dtdx, 0, upwind=mode)  # MC-linear: slope d, d2w = 0
    nu = u * dtdx
    cf = _cf(V0)
    numax, numin = max(0.0, (u + cf) * dtdx), min(0.0, (u - cf) * dtdx)
    wp, wm, w0 = d / 2, -d / 2, 0.0  # the field's values relative to the centre
    up, um = wp - nu / 2 * d, wm - nu / 2 * d
    ref = {1: (wp, wm), 2: (w0, w0), 3: (wp - numax / 2 * d, wm - numin / 2 * d)}
    if mode == 0:
        want = (up, um)
    else:
        rp, rm = ref[mode]
        want = (up if nu > 0 else rp, um if nu < 0 else rm)
    assert Vp[0] - 1.0 == pytest.approx(want[0], abs=1e-15)
    assert Vm[0] - 1.0 == pytest.approx(want[1], abs=1e-15)
    for V in (Vp, Vm):  # the other variables are untouched
        assert np.allclose(V[1:], V0[1:], rtol=0, atol=1e-15)


@pytest.mark.parametrize("mode,lo,hi", [(0, 1.9, 2.3), (1, 1.2, 1.8), (2, 0.85, 1.3), (3, 0.85, 1.3)])
def test_slow_wave_order(mode, lo, hi):
    errs = []
    for N in (16, 32, 64):
        U, U0, T = oblique_wave_2d(N, "slow")
        n = [N, N, 1]
        U, t, _ = O.mhd_run(U, n, 2, [1.0 / N, 1.0 / N, 1.0], 0, 0.4, recon=1, t_end=T, upwind=mode)
        errs.append(np.abs(O.interior(U, n, 2) - U0).sum() / 1e-6 / (N * N))
    order = np.log2(errs[1] / errs[2])
    assert lo < order < hi, (errs, order)


@pytest.mark.parametrize("mode", [2, 3])
def test_fast_wave_stays_second_order(mode):
    errs = []
    for N in (16, 32, 64):
        U, U0, T = oblique_wave_2d(N, "fast")
        n = [N, N, 1]
        U, t, _ = O.mhd_run(U, n, 2, [1.0 / N, 1.0 / N, 1.0], 0, 0.4, recon=1, t_end=T, upwind=mode)
        errs.append(np.abs(O.interior(U, n, 2) - U0).sum() / 1e-6 / (N * N))
    assert np.log2(errs[1] / errs[2]) > 1.8, errs
