"""Pins of the oracle's hybrid integration (the appendix on shock detection):
the HLL solver, the shock flags and the flagged step.

- HLL: consistency R(V, V) = F(V) (equal to the HLLD flux of the same
  state), pure upwinding when supersonic, and the diffusion that HLLD does
  not have: a stationary hydrodynamic contact leaks mass under HLL and not
  under HLLD.
- Flags in closed form: a pressure (or magnetic-pressure) jump of ratio 10
  with converging flow flags the two cells beside it along its axis (the sum
  of the relative central differences is 9 > 5 and div v < 0); diverging
  flow, or a ratio of 5, flags nothing; the MinMod flag spreads the reach of
  the reconstruction (2 cells for PPM, 1 for the linear reconstructions).
- A step with nothing flagged equals the plain step bit for bit.
- The purpose: a strongly magnetised blast that breaks the plain PPM/HLLD
  step within a few steps runs 30 steps under the hybrid, conserving mass
  and energy.
"""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W

G = 5.0 / 3.0


def test_hll_consistency_and_upwinding():
    rng = np.random.default_rng(1)
    for _ in range(20):
        V = np.array([rng.uniform(0.5, 2), *rng.normal(0, 1, 3), rng.uniform(0.5, 2), *rng.normal(0, 1, 3), 0.1])
        F1 = O.mhd_riemann_hll(V, V, G, 2.0)
        F2 = O.mhd_riemann(V, V, G, 2.0)
        assert np.allclose(F1, F2, rtol=1e-13, atol=1e-13)
    # supersonic to the right: the left flux
    VL = np.array([1.0, 20.0, 0.1, 0.0, 1.0, 0.5, 0.3, 0.2, 0.0])
    VR = np.array([0.5, 19.0, -0.1, 0.1, 0.8, 0.5, 0.1, 0.2, 0.0])
    F = O.mhd_riemann_hll(VL, VR, G, 1.0)
    FL = O.mhd_riemann(VL, VL, G, 1.0)
    assert np.allclose(F[[0, 1, 2, 3, 4, 6, 7]], FL[[0, 1, 2, 3, 4, 6, 7]], rtol=1e-14)


def test_hll_diffuses_a_stationary_contact():
    VL = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0])
    VR = np.array([0.125, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0])
    Fd = O.mhd_riemann(VL, VR, 1.4, 1.0)
    Fh = O.mhd_riemann_hll(VL, VR, 1.4, 1.0)
    assert Fd[0] == 0.0
    assert Fh[0] > 0.05  # mass flows from the dense side


def _jump(n, axis, ratio, v, qkind=0):
    """A jump of q across the plane between cells 7 and 8 along `axis`, with
    velocity +v below and -v above along it (converging for v > 0)."""
    shp = O.shape(n, 3)
    c = np.arange(shp[3 - axis]) - 4
    view = [1, 1, 1]
    view[2 - axis] = shp[3 - axis]
    lo = (c < 8).reshape(view)
    z = np.zeros(shp[1:])
    one = np.ones(shp[1:])
    p = one * 1.0
    B = [z + 0.1, z + 0.1, z + 0.1]
    if qkind == 0:
        p = np.where(lo, 1.0, ratio) + z
    else:
        B = [z, z, np.sqrt(2.0) * np.where(lo, 1.0, np.sqrt(ratio)) + z]
    vel = [z, z, z]
    vel[axis] = np.where(lo, v, -v) + z
    return W.ideal_cons([one, vel[0], vel[1], vel[2], p, B[0], B[1], B[2], z], G)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("qkind", [0, 1])
def test_flags_closed_form(axis, qkind):
    n = [16, 16, 16]
    U = _jump(n, axis, 10.0, 1.0, qkind)
    for reach in (2, 1):
        f = O.mhd_shock_flags(U, n, 3, [1.0 / 16] * 3, 5.0, qkind, reach)
        I = np.moveaxis(f[4:-4, 4:-4, 4:-4], 2 - axis, 0)
        shocked = np.nonzero(np.any(I & 1, axis=(1, 2)))[0].tolist()
        assert shocked == [7, 8]
        assert np.all(I[7] & 1) and np.all(I[8] & 1)
        mm = np.nonzero(np.all(I & 2, axis=(1, 2)))[0].tolist()
        assert mm == list(range(7 - reach, 9 + reach))
        assert not np.any(np.delete(I, mm, axis=0) & 2)
    # diverging flow, or a ratio of 5 (sum 4 < 5): nothing
    assert not np.any(O.mhd_shock_flags(_jump(n, axis, 10.0, -1.0, qkind), n, 3, [1.0 / 16] * 3, 5.0, qkind))
    assert not np.any(O.mhd_shock_flags(_jump(n, axis, 5.0, 1.0, qkind), n, 3, [1.0 / 16] * 3, 5.0, qkind))


def test_unflagged_step_is_the_plain_step():
    n = [16, 16, 16]
    U = W.mhd_blast_3d(16, seed=2)
    dx = [1.0 / 16] * 3
    O.fill_periodic(U, n, 3)
    dt, ch = O.dt_ch(O.mhd_max_speed(U, n, 3, dx), dx, 3, 0.3)
    assert not np.any(O.mhd_shock_flags(U, n, 3, dx, 1e9, 0))
    a, _ = O.mhd_step(U, n, 3, dx, dt, ch, recon=1)
    b, _ = O.mhd_step(U, n, 3, dx, dt, ch, recon=1, shock=(1e9, 0))
    assert np.array_equal(a, b)
    # the blast's sphere is flagged at a low threshold, and the step changes
    assert np.any(O.mhd_shock_flags(U, n, 3, dx, 0.5, 0) & 1)


def _magnetised_blast(N=64):
    n = [N, N, 1]
    shp = O.shape(n, 2)
    x = (np.arange(shp[3]) - 4 + 0.5) / N
    y = (np.arange(shp[2]) - 4 + 0.5) / N
    X, Y = np.meshgrid(x, y)
    p = np.where(np.hypot(X - 0.5, Y - 0.5) < 0.1, 1e4, 0.1)
    z = np.zeros_like(p)
    one = np.ones_like(p)
    U = np.zeros(shp)
    U[:, 0] = W.ideal_cons([one, z, z, z, p, 3 / np.sqrt(2) * one, 3 / np.sqrt(2) * one, z, z], G)
    return U, n


def test_hybrid_survives_where_the_plain_step_fails():
    U, n = _magnetised_blast()
    dx = [1.0 / 64] * 2
    with pytest.raises(FloatingPointError):
        O.mhd_run(U, n, 2, dx, 10, 0.4, recon=1)
    R, t, _ = O.mhd_run(U, n, 2, dx, 30, 0.4, recon=1, shock=(5.0, 0))
    a, b = O.interior(U, n, 2), O.interior(R, n, 2)
    for q in (0, 1, 2, 4, 5, 6):
        assert abs(b[q].sum() - a[q].sum()) <= 1e-12 * (np.abs(a[q]).sum() + 1.0)


@pytest.mark.parametrize("recon,reach", [(1, 2), (0, 1)])
def test_hybrid_step_changes_exactly_the_reach_of_the_flags(recon, reach):
    """1-D: a jump between cells 11 and 12 with converging flow, on a gently
    modulated background (so that MinMod and the scheme's reconstruction
    differ everywhere).  Cells 11 and 12 are shocked; the hybrid step
    differs from the plain one exactly on the cells whose update uses a face
    next to a shocked cell or a MinMod interface state: [11 - reach - 1,
    12 + reach + 1] (MinMod on the cells within `reach` of a shocked cell,
    2 for PPM and 1 for MC)."""
    n = [24, 1, 1]
    shp = O.shape(n, 1)
    c = np.arange(shp[3]) - 4
    mod = 1.0 + 0.01 * np.sin(0.7 * c)
    rho = mod.copy()
    p = np.where(c < 12, 1.0, 10.0) * mod
    v = np.where(c < 12, 0.5, -0.5) + 0.01 * np.cos(0.9 * c)
    z = np.zeros_like(rho)
    U = np.zeros(shp)
    U[:, 0, 0] = W.ideal_cons([rho, v, z, z, p, z + 0.3, z + 0.2, z + 0.1, z], G)
    dx = [1.0 / 24]
    f = O.mhd_shock_flags(U, n, 1, dx, 5.0, 0, reach)
    assert np.nonzero(f[0, 0, 4:-4] & 1)[0].tolist() == [11, 12]
    dt, ch = 0.002, 1.0
    a, _ = O.mhd_step(U, n, 1, dx, dt, ch, recon=recon)
    b, _ = O.mhd_step(U, n, 1, dx, dt, ch, recon=recon, shock=(5.0, 0))
    diff = np.any(np.abs(O.interior(a, n, 1) - O.interior(b, n, 1)) > 1e-14, axis=(0, 1, 2))
    assert np.nonzero(diff)[0].tolist() == list(range(11 - reach - 1, 12 + reach + 2))
