"""Pins of the oracle's corner coupling of Mignone & Tzeferacos (2010), the
case Pi = 0 of Section 3.1 ("constructed exactly as illustrated by MT"):
the transverse fluxes of Eq. (transv) come from Riemann problems between the
normal predictor states of the other directions, F*_d = R(U*_(c,+),
U*_(c+e_d,-)), instead of between cell-centred states.

What fixes it, independently of the oracle: in 1-D there is no transverse
term, so the step equals the plain one bit for bit; a uniform state stays
uniform bit for bit; periodic boxes conserve rho, m, E and B to round-off;
the x-mirror, z-mirror and x <-> y swap symmetries of Eq. (1) + Eq.
(glm2x2); second-order convergence of travelling oblique linear waves whose
eigenvectors come from numpy.linalg.eig of the primitive Jacobian; linear
advection of a density at Courant numbers (1, 1), where the corner-coupled
step is the exact diagonal shift by one cell; and, on data with cross
second derivatives, an error below the cell-centred variant's (the
transverse fluxes are time-centred).  A last test plants mistakes in a
scratch copy of the oracle and checks that each fails one of these pins.
"""
import ctypes
import shutil
import subprocess
from contextlib import contextmanager
from pathlib import Path

import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.mhd_setup import mirror_x, mirror_z, oblique_wave_2d, swap_xy


def _run(U, n, ndim, steps, cfl, recon=1, corner=1, dx=None):
    dxs = dx or [1.0 / n[0]] * 3
    U = U.copy()
    for _ in range(steps):
        O.fill_periodic(U, n, ndim)
        dt, ch = O.dt_ch(O.mhd_max_speed(U, n, ndim, dxs), dxs, ndim, cfl)
        U, bad = O.mhd_step(U, n, ndim, dxs, dt, ch, recon=recon, corner=corner)
        assert bad == 0
    O.fill_periodic(U, n, ndim)
    return U


def one_d_identity():
    n = [48, 1, 1]
    x = (np.arange(48) + 0.5) / 48
    z = np.zeros(48)
    U = np.zeros(O.shape(n, 1))
    O.interior(U, n, 1)[:] = W.ideal_cons([1 + 0.3 * np.sin(2 * np.pi * x), 0.3 + z, 0.1 + z, z,
                                            1 + 0.2 * np.cos(2 * np.pi * x), 0.7 + z, 0.5 + z, 0.2 + z, z],
                                           5 / 3).reshape(9, 1, 1, 48)
    worst = 0.0
    for recon in (0, 1):
        a = _run(U, n, 1, 4, 0.8, recon=recon, corner=1)
        b = _run(U, n, 1, 4, 0.8, recon=recon, corner=0)
        worst = max(worst, np.abs(a - b).max())
    return worst


def diagonal_shift_error():
    """rho = 1 + 0.3 sin(2 pi x) cos(2 pi y) advected by v = (+-1, +-1) dx/dt,
    B = 0, p uniform, MC-linear (a linear profile traced at Courant number 1
    gives the exact upwind value), one step at |C_x| = |C_y| = 1: the result
    is the initial field shifted by one cell along the diagonal, in each of
    the four quadrants of the velocity (the upwind states are the left ones
    for positive and the right ones for negative components)."""
    N = 16
    n = [N, N, 1]
    h = 1.0 / N
    x = (np.arange(N) + 0.5) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = 1 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y + 0.4)
    z = np.zeros_like(rho)
    worst = 0.0
    for sx, sy in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
        U = np.zeros(O.shape(n, 2))
        O.interior(U, n, 2)[:] = W.ideal_cons([rho, z + sx, z + sy, z, z + 1.0, z, z, z, z], 1.4)[:, None]
        O.fill_periodic(U, n, 2)
        dt = h  # speeds 1 along x and y: |C_x| = |C_y| = 1
        Un, bad = O.mhd_step(U, n, 2, [h, h], dt, 1.0, gamma=1.4, recon=0, corner=1)
        assert bad == 0
        got = O.interior(Un, n, 2)[0, 0]
        worst = max(worst, np.abs(got - np.roll(np.roll(rho, sy, axis=0), sx, axis=1)).max())
    return worst


def convergence_orders():
    """Fitted L1 orders (32 -> 64) of oblique fast, Alfven and entropy waves
    after one period (PPM, CFL 0.4)."""
    orders = {}
    for wave in ("fast", "alfven", "entropy"):
        errs = []
        for N in (32, 64):
            U, U0, T = oblique_wave_2d(N, wave)
            n = [N, N, 1]
            U, t, _ = O.mhd_run(U, n, 2, [1.0 / N, 1.0 / N, 1.0], 0, 0.4, recon=1, t_end=T, corner=1)
            errs.append(np.abs(O.interior(U, n, 2) - U0).sum() / 1e-6 / (N * N))
        orders[wave] = np.log2(errs[0] / errs[1])
    return orders


def cross_term_ratio():
    """Density 1 + 0.3 x y^2 (cell averages, x, y in (0.5, 2.5)) advected by a
    uniform velocity, PPM (exact for 1-D quadratics): the error of one step,
    corner-coupled over cell-centred transverse fluxes."""
    h = 1.0 / 8
    n = [8, 8, 1]
    a, b = 0.7, 0.4
    xs = (np.arange(-4, 12) + 0.5) * h + 1.0
    X, Y = np.meshgrid(xs, xs, indexing="xy")

    def avg(xc, yc):  # cell average of x y^2
        return xc * (yc * yc + h * h / 12)
    rho = 1 + 0.3 * avg(X, Y)
    z = np.zeros_like(rho)
    U = W.ideal_cons([rho, z + a, z + b, z, z + 1.0, z, z, z, z], 1.4)[:, None]
    dt = 0.4 * h / a
    ex = 1 + 0.3 * avg(X[4:12, 4:12] - a * dt, Y[4:12, 4:12] - b * dt)
    err = []
    for corner in (1, 0):
        Un, bad = O.mhd_step(np.ascontiguousarray(U), n, 2, [h, h], dt, 1.0, gamma=1.4, recon=1, corner=corner)
        err.append(np.abs(O.interior(Un, n, 2)[0, 0] - ex).max())
    return err[0] / err[1]


def test_one_dimension_equals_the_plain_step():
    assert one_d_identity() == 0.0


def test_uniform_state_is_preserved():
    for ndim, n in ((2, [8, 8, 1]), (3, [6, 6, 6])):
        U = np.zeros(O.shape(n, ndim))
        U[:] = W.ideal_cons([1.2, 0.3, -0.2, 0.1, 0.8, 0.5, 0.4, -0.3, 0.0], 5 / 3).reshape(9, 1, 1, 1)
        out = _run(U, n, ndim, 2, 0.3)
        assert np.array_equal(out, U)


def test_conservation_periodic():
    for ndim, U, n in ((2, W.mhd_turb_2d(24, seed=1), [24, 24, 1]),
                       (3, W.mhd_blast_3d(12, seed=2, kmax=2), [12, 12, 12])):
        S0 = O.interior(U, n, ndim).sum(axis=(1, 2, 3))
        scale = np.abs(O.interior(U, n, ndim)).sum(axis=(1, 2, 3))
        out = _run(U, n, ndim, 5, 0.3)
        S = O.interior(out, n, ndim).sum(axis=(1, 2, 3))
        assert np.all(np.abs(S - S0)[:8] <= 1e-13 * scale[:8]), (S - S0)


def test_mirror_and_swap_symmetry():
    n = [20, 20, 1]
    U = W.mhd_turb_2d(20, seed=4)
    ref = O.interior(_run(U, n, 2, 3, 0.4), n, 2)
    scale = np.abs(ref).max(axis=(1, 2, 3))[:, None, None, None]
    for f in (mirror_x, swap_xy):
        out = O.interior(f(_run(f(U), n, 2, 3, 0.4)), n, 2)
        assert np.all(np.abs(out - ref) <= 1e-12 * scale)
    n3 = [10, 10, 10]
    U3 = W.mhd_blast_3d(10, seed=5, kmax=2)
    ref3 = O.interior(_run(U3, n3, 3, 2, 0.3), n3, 3)
    s3 = np.abs(ref3).max(axis=(1, 2, 3))[:, None, None, None]
    for f in (mirror_x, mirror_z):
        out = O.interior(f(_run(f(U3), n3, 3, 2, 0.3)), n3, 3)
        assert np.all(np.abs(out - ref3) <= 1e-12 * s3)


def test_second_order_convergence():
    orders = convergence_orders()
    assert all(o > 1.85 for o in orders.values()), orders


def test_unit_courant_diagonal_shift_is_exact():
    assert diagonal_shift_error() < 1e-13


def test_time_centred_transverse_fluxes_beat_cell_centred_ones():
    assert cross_term_ratio() < 0.6


# ------------------------------------------------------------ planted mistakes

MUTANTS = {
    "right state from the left cell's predictor": (
        "(flags && (flags[id + st] & 2)) ? 2 : recon, upwind, Vx, VR);",
        "(flags && (flags[id + st] & 2)) ? 2 : recon, upwind, VR, Vx);"),
    "right cell's stencil not shifted": (
        "vs[l * NVAR + q] = V[PERM[d][q] * nc + id + (l - 1) * st];",
        "vs[l * NVAR + q] = V[PERM[d][q] * nc + id + (l - 2) * st];"),
    "predictor over half the time step": (
        "or_mhd_char_predict_dx(vs, gam, ch, dt / h[d], h[d],\n                                               (flags && (flags[id] & 2)) ? 2 : recon, upwind, VL, Vx);",
        "or_mhd_char_predict_dx(vs, gam, ch, 0.5 * dt / h[d], h[d],\n                                               (flags && (flags[id] & 2)) ? 2 : recon, upwind, VL, Vx);"),
}


@contextmanager
def _oracle_from(tmp, name):
    """The oracle module bound to a scratch copy of its library with one
    planted mistake."""
    old, new = MUTANTS[name]
    src = O.HERE
    d = tmp / "mutant"
    d.mkdir()
    for s in O.SOURCES:
        txt = (src / s).read_text()
        if s == "ctu_oracle.c":
            assert txt.count(old) == 1, f"pattern of {name!r} not found once"
            txt = txt.replace(old, new)
        (d / s).write_text(txt)
    so = d / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared", "-o",
                    str(so)] + [str(d / s) for s in O.SOURCES] + ["-lm"], check=True)
    saved = (O._lib, O.LIB_PATH)
    O._lib, O.LIB_PATH = None, so
    try:
        yield
    finally:
        O._lib, O.LIB_PATH = saved


def _first_failing_pin():
    """The first pin (cheapest first) the oracle as loaded fails, or None."""
    if one_d_identity() != 0.0:
        return "1-D"
    if diagonal_shift_error() >= 1e-13:
        return "diagonal"
    if cross_term_ratio() >= 0.6:
        return "cross"
    if not all(o > 1.85 for o in convergence_orders().values()):
        return "order"
    return None


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(tmp_path, name):
    with _oracle_from(tmp_path, name):
        assert _first_failing_pin() is not None, name
