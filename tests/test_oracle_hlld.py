"""Closed-form pins of the oracle's HLLD solver (Miyoshi & Kusano 2005) in
its magnetised branches, B_n != 0 (the Riemann solver of Section 3.1, Eq.
ctu_flux, for the MHD system of Eq. 1).

HLLD resolves two isolated discontinuities exactly, and each gives a flux in
closed form, the upwind physical flux of Eq. (1):
  * a contact (entropy) discontinuity with B_n != 0: only rho jumps, while
    u, v_t, p and B are continuous.  It moves with u.  Its flux is F(U_L)
    for u > 0 and F(U_R) for u < 0; at u = 0 the two agree.
  * a rotational (Alfven) discontinuity: rho, u, p and |B_t| are continuous;
    B_t rotates, and v_t jumps by [v_t] = -s sgn(B_n) [B_t] / sqrt(rho)
    for the wave moving at lambda = u + s |B_n| / sqrt(rho) (s = +-1).
    Its flux is F(U_L) for lambda > 0 and F(U_R) for lambda < 0.  When the
    face lies inside the Alfven fan (s = -1, lambda < 0 < u), it is reached
    through the double-star state and its energy term.
  * the degenerate branch: with |B_t| -> 0 and B_n^2 > gamma p, the fast
    and Alfven speeds merge and rho(S - u)(S - S_M) - B_n^2 -> 0.  A contact
    swept through that limit must still give its exact flux.
A last test plants plausible mistakes in a scratch copy of the oracle (a
double-star sign, the energy term, an Alfven speed, the degenerate
threshold) and checks that each one fails one of these pins.
"""
import ctypes
import re
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

import oracle as O

G = 5.0 / 3.0
IDX = [0, 1, 2, 3, 4, 6, 7]  # the HLLD components (B_n and psi come from the GLM face solve)


def _flux(V, g):
    """Physical flux of Eq. (1) along the normal (written from the PDE)."""
    rho, u, v, w, p, Bn, B1, B2, _ = V
    B2s = Bn * Bn + B1 * B1 + B2 * B2
    E = p / (g - 1.0) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * B2s
    pt = p + 0.5 * B2s
    vB = u * Bn + v * B1 + w * B2
    return np.array([rho * u, rho * u * u + pt - Bn * Bn, rho * u * v - Bn * B1, rho * u * w - Bn * B2,
                     (E + pt) * u - Bn * vB, 0.0, u * B1 - Bn * v, u * B2 - Bn * w, 0.0])


def _err(F, ref):
    scale = max(np.abs(ref[IDX]).max(), 1e-300)
    return np.abs(F[IDX] - ref[IDX]).max() / scale


def contact_cases():
    """(VL, VR, exact flux) of isolated contacts with B_n != 0."""
    rng = np.random.default_rng(21)
    out = []
    for _ in range(40):
        rho = rng.uniform(0.2, 3.0, 2)
        u = rng.choice([rng.uniform(-2, 2), 0.0])
        vt = rng.normal(0, 1, 2)
        p = rng.uniform(0.1, 2.0)
        B = np.array([rng.choice([-1, 1]) * rng.uniform(0.2, 2.0), *rng.normal(0, 1, 2)])
        VL = np.array([rho[0], u, *vt, p, *B, 0.0])
        VR = np.array([rho[1], u, *vt, p, *B, 0.0])
        out.append((VL, VR, _flux(VL if u > 0 else VR, G)))
    return out


def degenerate_contacts():
    """Contacts swept through the degenerate limit of the left star state:
    B_n^2 = 2.25 > gamma p = 1/6 and rho_L < rho_R, so S_L = u - c_f,L, and
    |B_t| = eps -> 0 drives rho_L (S_L - u)(S_L - S_M) - B_n^2 to zero."""
    out = []
    for u in (0.0, 0.2, -0.3):
        for sgn in (1.0, -1.0):
            for eps in (1e-1, 1e-3, 1e-5, 1e-6, 3e-7, 1e-7, 1e-8, 1e-10, 0.0):
                VL = np.array([0.5, u, 0.3, -0.2, 0.1, 1.5 * sgn, eps, 0.5 * eps, 0.0])
                VR = np.array([2.0, u, 0.3, -0.2, 0.1, 1.5 * sgn, eps, 0.5 * eps, 0.0])
                out.append((VL, VR, _flux(VL if u > 0 else VR, G)))
    return out


def rotational_cases():
    """(VL, VR, exact flux) of isolated rotational discontinuities, in frames
    that put the face left of, inside and right of the Alfven fan."""
    rng = np.random.default_rng(22)
    out = []
    for s in (1.0, -1.0):
        for bn_sign in (1.0, -1.0):
            for u_frac in (-2.0, -0.5, 0.0, 0.5, 2.0):
                rho = rng.uniform(0.5, 2.0)
                p = rng.uniform(0.3, 1.5)
                Bn = bn_sign * rng.uniform(0.5, 1.5)
                ca = abs(Bn) / np.sqrt(rho)
                u = u_frac * ca
                b = rng.uniform(0.3, 1.2)
                thL, thR = rng.uniform(0, 2 * np.pi, 2)
                BtL = b * np.array([np.cos(thL), np.sin(thL)])
                BtR = b * np.array([np.cos(thR), np.sin(thR)])
                vtL = rng.normal(0, 0.5, 2)
                vtR = vtL - s * np.sign(Bn) * (BtR - BtL) / np.sqrt(rho)
                VL = np.array([rho, u, *vtL, p, Bn, *BtL, 0.0])
                VR = np.array([rho, u, *vtR, p, Bn, *BtR, 0.0])
                lam = u + s * ca
                out.append((VL, VR, _flux(VL if lam > 0 else VR, G), s, lam))
    return out


def compound_cases():
    """(VL, VR, exact flux) of a rotational discontinuity next to a contact:
    U_L | Alfven wave at u - |B_n|/sqrt(rho_L) | U_m | contact at u | U_R, and
    the mirror image with the Alfven wave right of the contact at
    u + |B_n|/sqrt(rho_R).  HLLD's fan has exactly these waves, with Alfven
    speeds from the densities on their own sides of the contact, so the flux
    is exact: F(U_L), F(U_m) or F(U_R) by the face's place in the fan."""
    rng = np.random.default_rng(23)
    out = []
    for left in (True, False):
        for bn_sign in (1.0, -1.0):
            for where in (-1.5, -0.5, 0.5, 1.5):
                rhoL, rhoR = rng.uniform(0.3, 0.8), rng.uniform(1.5, 3.0)
                if not left:
                    rhoL, rhoR = rhoR, rhoL
                p = rng.uniform(0.3, 1.5)
                Bn = bn_sign * rng.uniform(0.5, 1.5)
                b = rng.uniform(0.3, 1.2)
                th0, th1 = rng.uniform(0, 2 * np.pi, 2)
                Bt0 = b * np.array([np.cos(th0), np.sin(th0)])
                Bt1 = b * np.array([np.cos(th1), np.sin(th1)])
                vt0 = rng.normal(0, 0.5, 2)
                if left:   # Alfven wave (s = -1) in rho_L, then the contact
                    ca = abs(Bn) / np.sqrt(rhoL)
                    vt1 = vt0 + np.sign(Bn) * (Bt1 - Bt0) / np.sqrt(rhoL)
                    # where: the face left of the Alfven wave, between it and the
                    # contact (twice), or right of the contact
                    u = {-1.5: -ca * 1.5, -0.5: 0.5 * ca, 0.5: 0.25 * ca, 1.5: ca * 0.0 - 0.3}[where]
                    VL = np.array([rhoL, u, *vt0, p, Bn, *Bt0, 0.0])
                    Vm = np.array([rhoL, u, *vt1, p, Bn, *Bt1, 0.0])
                    VR = np.array([rhoR, u, *vt1, p, Bn, *Bt1, 0.0])
                    lam = u - ca
                    ref = VL if lam > 0 else (Vm if u > 0 else VR)
                else:      # the contact, then an Alfven wave (s = +1) in rho_R
                    ca = abs(Bn) / np.sqrt(rhoR)
                    vt1 = vt0 - np.sign(Bn) * (Bt1 - Bt0) / np.sqrt(rhoR)
                    u = {-1.5: ca * 1.5, -0.5: -0.5 * ca, 0.5: -0.25 * ca, 1.5: 0.3}[where]
                    VL = np.array([rhoL, u, *vt0, p, Bn, *Bt0, 0.0])
                    Vm = np.array([rhoR, u, *vt0, p, Bn, *Bt0, 0.0])
                    VR = np.array([rhoR, u, *vt1, p, Bn, *Bt1, 0.0])
                    lam = u + ca
                    ref = VL if u > 0 else (Vm if lam > 0 else VR)
                out.append((VL, VR, _flux(ref, G)))
    return out


def _cons(V, g):
    rho, u, v, w, p, Bn, B1, B2, psi = V
    return np.array([rho, rho * u, rho * v, rho * w,
                     p / (g - 1.0) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * (Bn * Bn + B1 * B1 + B2 * B2),
                     Bn, B1, B2, psi])


def _cfast(V, g):
    """Fast speed along the normal, the larger root of the quartic in c^2."""
    rho, p, Bn, B1, B2 = V[0], V[4], V[5], V[6], V[7]
    a2, b2, bt2 = g * p / rho, (Bn * Bn + B1 * B1 + B2 * B2) / rho, (B1 * B1 + B2 * B2) / rho
    return np.sqrt(0.5 * (a2 + b2 + np.sqrt((a2 - b2) ** 2 + 4.0 * a2 * bt2)))


def single_star_residual(riemann):
    """Worst residual of the single-star flux identity over general Riemann
    problems.  HLLD's outer star state U*_L is joined to U_L across S_L by
    the Rankine-Hugoniot condition with a star flux of the physical form
        F* = (rho* S_M, rho* S_M^2 + p_t* - B_n^2, rho* S_M v_t* - B_n B_t*,
              (E* + p_t*) S_M - B_n (v*.B*), S_M B_t* - B_n v_t*).
    With the face just right of S_L (the states boosted along the normal so
    that S_L = min(u_L, u_R) - max(c_f) lies at -delta), the returned flux
    F is F*, and U* = U_L + (F - F_L) / S_L; the residual of the identity
    above, for the star state recovered this way, vanishes to round-off.
    Frames where the recovered state puts S*_L = S_M - |B_n| / sqrt(rho*)
    at or below the face are skipped.  Returns (residual, frames used)."""
    rng = np.random.default_rng(24)
    worst, used = 0.0, 0
    for _ in range(40):
        VL = np.array([rng.uniform(0.5, 2), *rng.normal(0, 0.5, 3), rng.uniform(0.3, 2), 0.0, *rng.normal(0, 1, 2), 0.0])
        VR = np.array([rng.uniform(0.5, 2), *rng.normal(0, 0.5, 3), rng.uniform(0.3, 2), 0.0, *rng.normal(0, 1, 2), 0.0])
        VL[5] = VR[5] = Bn = rng.choice([-1.0, 1.0]) * rng.uniform(0.3, 1.5)
        s0 = min(VL[1], VR[1]) - max(_cfast(VL, G), _cfast(VR, G))
        for delta in (0.03, 0.1, 0.3):
            L, R = VL.copy(), VR.copy()
            L[1] -= s0 + delta
            R[1] -= s0 + delta
            F = riemann(L, R, G, 2.5)
            FL = _flux(L, G)
            Us = _cons(L, G) + (F - FL) / (-delta)
            rs = Us[0]
            SM, vs, ws, B1s, B2s = Us[1] / rs, Us[2] / rs, Us[3] / rs, Us[6], Us[7]
            if not (rs > 0 and SM - abs(Bn) / np.sqrt(rs) > 0.0):
                continue
            used += 1
            pts = F[1] - rs * SM * SM + Bn * Bn
            r = [F[0] - rs * SM, F[2] - (rs * SM * vs - Bn * B1s), F[3] - (rs * SM * ws - Bn * B2s),
                 F[4] - ((Us[4] + pts) * SM - Bn * (SM * Bn + vs * B1s + ws * B2s)),
                 F[6] - (SM * B1s - Bn * vs), F[7] - (SM * B2s - Bn * ws)]
            worst = max(worst, np.abs(r).max() / np.abs(F[IDX]).max())
    return worst, used


def pin_failures(riemann):
    """Worst relative flux error of each family (contacts, degenerate
    contacts, rotational discontinuities, rotational discontinuity beside a
    contact) and the single-star identity's residual, for a solver
    riemann(VL, VR, g, ch)."""
    res = {}
    for name, cases in (("contact", contact_cases()), ("degenerate", degenerate_contacts()),
                        ("rotational", rotational_cases()), ("compound", compound_cases())):
        res[name] = max(_err(riemann(c[0], c[1], G, 2.5), c[2]) for c in cases)
    res["single_star"] = single_star_residual(riemann)[0]
    return res


TOL = {"contact": 1e-13, "degenerate": 1e-12, "rotational": 1e-13, "compound": 1e-13, "single_star": 1e-12}


def test_exact_contact_with_normal_field():
    for VL, VR, ref in contact_cases():
        F = O.mhd_riemann(VL, VR, G, 2.5)
        assert _err(F, ref) < TOL["contact"], (VL, VR, F, ref)
        # the GLM face solve of a continuous B_n, psi = 0
        assert F[5] == 0.0 and F[8] == pytest.approx(2.5 ** 2 * VL[5], rel=1e-15)


def test_exact_contact_through_the_degenerate_limit():
    for VL, VR, ref in degenerate_contacts():
        assert _err(O.mhd_riemann(VL, VR, G, 2.5), ref) < TOL["degenerate"], (VL, VR)


def test_exact_rotational_discontinuity():
    for VL, VR, ref, _, _ in rotational_cases():
        assert _err(O.mhd_riemann(VL, VR, G, 2.5), ref) < TOL["rotational"], (VL, VR)


def test_exact_rotational_discontinuity_beside_a_contact():
    for VL, VR, ref in compound_cases():
        assert _err(O.mhd_riemann(VL, VR, G, 2.5), ref) < TOL["compound"], (VL, VR)


def test_single_star_flux_has_the_physical_form():
    worst, used = single_star_residual(O.mhd_riemann)
    assert used >= 60 and worst < TOL["single_star"], (used, worst)


def test_rotational_discontinuity_inside_the_fan_uses_the_double_star_energy():
    """For a left-going rotational discontinuity with the face between it and
    the contact, the exact flux F(U_R) differs from F(U_L) in every
    transverse and energy component: the pin is not passed by the upwind
    state alone."""
    hit = 0
    for VL, VR, ref, s, lam in rotational_cases():
        if s < 0 and lam < 0.0 <= VL[1]:
            FL = _flux(VL, G)
            assert abs(FL[4] - ref[4]) > 1e-3 * abs(ref[4])
            hit += 1
    assert hit >= 2


# ------------------------------------------------------------ planted mistakes

SRC = Path(O.__file__).resolve().parent

MUTANTS = {
    "double-star B_t sign": ("B1ss = (sqL * B1sR + sqR * B1sL + sqL * sqR * (vsR - vsL) * sB) * isq",
                             "B1ss = (sqL * B1sR + sqR * B1sL - sqL * sqR * (vsR - vsL) * sB) * isq"),
    "double-star v_t sign": ("vss = (sqL * vsL + sqR * vsR + (B1sR - B1sL) * sB) * isq",
                             "vss = (sqL * vsL + sqR * vsR - (B1sR - B1sL) * sB) * isq"),
    "double-star energy sign (left)": ("Uss[4] = EsL - sqL * (vBsL - vBss) * sB;",
                                       "Uss[4] = EsL + sqL * (vBsL - vBss) * sB;"),
    "double-star energy sign (right)": ("Uss[4] = EsR + sqR * (vBsR - vBss) * sB;",
                                        "Uss[4] = EsR - sqR * (vBsR - vBss) * sB;"),
    "Alfven speed from the other side": ("SLs = SM - fabs(Bn) / sqL;", "SLs = SM - fabs(Bn) / sqR;"),
    "single-star B_t factor": ("double f = (VL[0] * sdL * sdL - Bn * Bn) / dL;",
                               "double f = (VL[0] * sdL * sdL + Bn * Bn) / dL;"),
    "no degenerate branch": ("if (fabs(dL) <= 1.0e-12 * (VL[0] * sdL * sdL + Bn * Bn)) {",
                             "if (fabs(dL) <= 0.0 * (VL[0] * sdL * sdL + Bn * Bn)) {"),
    "single-star energy B_n term": ("EsL = (sdL * UL[4] - ptL * VL[1] + pts * SM + Bn * (vBL - vBsL)) / (SL - SM);",
                                    "EsL = (sdL * UL[4] - ptL * VL[1] + pts * SM - Bn * (vBL - vBsL)) / (SL - SM);"),
}


def _mutant_riemann(tmp, name):
    old, new = MUTANTS[name]
    src = (SRC / "ctu_oracle.c").read_text()
    assert src.count(old) == 1, f"pattern of mutant {name!r} not found once in the oracle"
    d = tmp / re.sub(r"\W+", "_", name)
    d.mkdir()
    (d / "ctu_oracle.c").write_text(src.replace(old, new))
    so = d / "lib.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared",
                    "-o", str(so), str(d / "ctu_oracle.c"), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    P, D = ctypes.POINTER(ctypes.c_double), ctypes.c_double
    L.or_mhd_riemann.argtypes = [P, P, D, D, P]
    L.or_mhd_riemann.restype = ctypes.c_int

    def riemann(VL, VR, g, ch):
        VL = np.ascontiguousarray(VL, dtype=np.float64)
        VR = np.ascontiguousarray(VR, dtype=np.float64)
        F = np.zeros(9)
        L.or_mhd_riemann(VL.ctypes.data_as(P), VR.ctypes.data_as(P), g, ch, F.ctypes.data_as(P))
        return F
    return riemann


def test_pins_hold_for_the_oracle():
    res = pin_failures(O.mhd_riemann)
    assert all(res[k] < TOL[k] for k in TOL), res


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(tmp_path, name):
    res = pin_failures(_mutant_riemann(tmp_path, name))
    assert any(res[k] >= TOL[k] for k in TOL), (name, res)
