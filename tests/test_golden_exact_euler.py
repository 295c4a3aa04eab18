"""The oracle's exact Euler Riemann solver (oracle/exact_euler.c, used to pin
the CTU step on shock tubes) against the star-region values the textbook
prints for its five test problems (tests/golden/toro_table_4_3.txt), and
against an independent solution of the same pressure equation by scipy's
bracketing root finder."""
from pathlib import Path

import numpy as np
import pytest

import oracle as O

G = 1.4
ROWS = np.loadtxt(Path(__file__).parent / "golden" / "toro_table_4_3.txt")


def _star_scipy(rL, uL, pL, rR, uR, pR):
    """p*, u*, rho*_L, rho*_R from the pressure function f_L(p) + f_R(p) + du
    (shock branch: Rankine-Hugoniot; rarefaction branch: isentrope)."""
    from scipy.optimize import brentq

    def fk(p, r, pk):
        a = np.sqrt(G * pk / r)
        if p > pk:
            A, B = 2.0 / ((G + 1) * r), (G - 1) / (G + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2 * a / (G - 1) * ((p / pk) ** ((G - 1) / (2 * G)) - 1)

    f = lambda p: fk(p, rL, pL) + fk(p, rR, pR) + (uR - uL)
    p = brentq(f, 1e-12, 1e5, xtol=1e-14, rtol=1e-15)
    u = 0.5 * (uL + uR) + 0.5 * (fk(p, rR, pR) - fk(p, rL, pL))

    def rho(r, pk):
        if p > pk:
            q = (G - 1) / (G + 1)
            return r * (p / pk + q) / (q * p / pk + 1)
        return r * (p / pk) ** (1 / G)
    return p, u, rho(rL, pL), rho(rR, pR)


@pytest.mark.parametrize("k", range(len(ROWS)))
def test_star_region_against_the_textbook(k):
    rL, uL, pL, rR, uR, pR, ps, us, rsl, rsr = ROWS[k]
    p, u, a, b = _star_scipy(rL, uL, pL, rR, uR, pR)
    for got, want in ((p, ps), (u, us), (a, rsl), (b, rsr)):
        assert got == pytest.approx(want, rel=5e-5, abs=5e-6)
    # the oracle's sampler just left and right of the contact (x/t = u*)
    left = O.euler_sample((rL, uL, pL), (rR, uR, pR), G, np.array([u - 1e-7]))[0]
    right = O.euler_sample((rL, uL, pL), (rR, uR, pR), G, np.array([u + 1e-7]))[0]
    assert left[0] == pytest.approx(a, rel=1e-6) and right[0] == pytest.approx(b, rel=1e-6)
    assert left[1] == pytest.approx(u, rel=1e-6, abs=1e-9) and left[2] == pytest.approx(p, rel=1e-6)
    assert right[2] == pytest.approx(p, rel=1e-6)
