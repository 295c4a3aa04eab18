"""Pins of the oracle's optional floors on the updated state (the library's
reading; the paper fixes no floor): rho < rho_floor takes rho_floor with m,
E, B, psi kept, then a pressure below p_floor (evaluated with the floored
density) is raised to p_floor through E alone.  Checked against the oracle's
own pinned cons2prim, exact invariants and the closed-form energy gain."""
import numpy as np

import oracle as O

G53 = 5.0 / 3.0


def _state(n, ndim, seed):
    """Ghost-filled patch with rho in [0.05, 2], p in [0.02, 2] and random v,
    B, psi."""
    rng = np.random.default_rng(seed)
    shp = O.shape(n, ndim)
    V = np.empty(shp)
    V[0] = rng.uniform(0.05, 2.0, shp[1:])
    V[1:4] = rng.normal(0.0, 1.0, (3,) + shp[1:])
    V[4] = rng.uniform(0.02, 2.0, shp[1:])
    V[5:8] = rng.normal(0.0, 1.0, (3,) + shp[1:])
    V[8] = rng.normal(0.0, 0.1, shp[1:])
    U = np.empty_like(V)
    flat_v = V.reshape(9, -1)
    flat_u = U.reshape(9, -1)
    for c in range(flat_v.shape[1]):
        flat_u[:, c] = O.mhd_prim2cons(flat_v[:, c], G53)
    return U


def _p(Uc):
    return O.mhd_cons2prim(Uc, G53)[0][4]


def test_floors_off_leave_the_state_bitwise():
    n = [6, 5, 4]
    U = _state(n, 3, 0)
    U2 = U.copy()
    assert O.mhd_floor(U2, n, 3, 0.0, 0.0) == 0
    assert np.array_equal(U, U2)


def test_floor_rules_cell_by_cell():
    n = [7, 6, 5]
    U0 = _state(n, 3, 1)
    U = U0.copy()
    rf, pf = 0.6, 0.5
    cnt = O.mhd_floor(U, n, 3, pf, rf)
    I0, I1 = O.interior(U0, n, 3), O.interior(U, n, 3)
    # ghosts untouched
    mask = np.ones(U.shape[1:], bool)
    mask[4:-4, 4:-4, 4:-4] = False
    assert np.array_equal(U[:, mask], U0[:, mask])
    changed = 0
    gain = 0.0
    for idx in np.ndindex(I0.shape[1:]):
        a, b = I0[(slice(None),) + idx], I1[(slice(None),) + idx]
        # m, B, psi never change; rho is max(rho, rho_floor) exactly
        assert np.array_equal(a[[1, 2, 3, 5, 6, 7, 8]], b[[1, 2, 3, 5, 6, 7, 8]])
        assert b[0] == max(a[0], rf)
        mid = a.copy()
        mid[0] = b[0]
        p_mid = _p(mid)
        if p_mid < pf:
            # pressure raised to the floor through E alone
            assert abs(_p(b) - pf) <= 1e-12 * pf
            gain += b[4] - a[4]
            assert abs((b[4] - a[4]) - (pf - p_mid) / (G53 - 1.0)) <= 1e-12 * (1.0 + abs(a[4]))
        else:
            assert b[4] == a[4]
            assert _p(b) >= pf
        # a density floor alone never lowers the pressure (less kinetic energy)
        if a[0] < rf:
            assert p_mid >= _p(a)
        hit = a[0] < rf or p_mid < pf
        changed += hit
        assert hit == (not np.array_equal(a, b))
    assert cnt == changed and 0 < cnt < I0[0].size
    assert gain > 0.0


def test_floor_count_of_each_kind():
    """Only a density floor, only a pressure floor, both: the count of the
    combined run is that of cells below either, computed from the separate
    runs (the density floor never lowers p, so the pressure test of the
    combined run sees a pressure >= the unfloored one)."""
    n = [8, 8, 1]
    U0 = _state(n, 2, 2)
    Ur, Up, Ub = U0.copy(), U0.copy(), U0.copy()
    cr = O.mhd_floor(Ur, n, 2, 0.0, 0.5)
    cp = O.mhd_floor(Up, n, 2, 0.3, 0.0)
    cb = O.mhd_floor(Ub, n, 2, 0.3, 0.5)
    assert cr > 0 and cp > 0
    assert max(cr, cp) <= cb <= cr + cp
    I0, Ir = O.interior(U0, n, 2), O.interior(Ur, n, 2)
    assert cr == int(np.sum(I0[0] < 0.5))
    assert np.array_equal(Ir[4], I0[4])


def test_step_then_floor_keeps_mass_above_the_floor():
    """A step of a strongly rarefying state, then the floors: every interior
    cell ends at or above both floors and the floors add mass only where the
    density was below them."""
    n = [16, 16, 1]
    shp = O.shape(n, 2)
    V = np.zeros(shp)
    V[0] = 1.0
    V[4] = 0.05
    x = (np.arange(shp[3]) - 4 + 0.5) / n[0]
    V[1] = np.where(x < 0.5, -2.0, 2.0)[None, None, :]
    V[5] = 0.1
    U = np.empty_like(V)
    for c in np.ndindex(shp[1:]):
        U[(slice(None),) + c] = O.mhd_prim2cons(V[(slice(None),) + c], G53)
    U = O.fill_outflow(U, n, 2)
    dx = [1.0 / 16] * 2
    sm = O.mhd_max_speed(U, n, 2, dx)
    dt, ch = O.dt_ch(sm, dx, 2, 0.4)
    Un, bad = O.mhd_step(U, n, 2, dx, dt, ch, recon=0)
    assert bad == 0
    low_rho = O.interior(Un, n, 2)[0].min()
    rf, pf = 0.5 * (low_rho + 1.0), 0.04
    Uf = Un.copy()
    cnt = O.mhd_floor(Uf, n, 2, pf, rf)
    assert cnt > 0
    I = O.interior(Uf, n, 2)
    for idx in np.ndindex(I.shape[1:]):
        c = I[(slice(None),) + idx]
        assert c[0] >= rf and _p(c) >= pf * (1 - 1e-12)
    dm = O.interior(Uf, n, 2)[0] - O.interior(Un, n, 2)[0]
    assert np.all(dm >= 0.0) and np.all((dm > 0.0) == (O.interior(Un, n, 2)[0] < rf))
