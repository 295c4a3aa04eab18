"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: the references are the exact
Euler Riemann solution, eigenvectors from numpy.linalg.eig of the primitive
Jacobian written from the PDE, conservation laws, the analytic GLM damping,
symmetries of the equations, and closed-form special cases.
"""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.mhd_setup import (G53, IDX7, mirror_x, mirror_z, oblique_wave_2d,
                             primitive_jacobian_7, swap_xy)


def _rand_state(rng, bmag=1.0):
    V = np.zeros(9)
    V[0] = rng.uniform(0.5, 2.0)
    V[1:4] = rng.normal(size=3)
    V[4] = rng.uniform(0.2, 2.0)
    V[5:8] = bmag * rng.normal(size=3)
    V[8] = rng.normal() * 0.1
    return V


# --------------------------------------------------------------- eigen-system

@pytest.mark.parametrize("seed", range(6))
def test_eigenvectors_diagonalise_the_pde_jacobian(seed):
    """L R = I, L A R = diag(lambda) with A written from Eq. (1), and the wave
    speeds agree with numpy's eigenvalues of A."""
    rng = np.random.default_rng(seed)
    V = _rand_state(rng, bmag=[0.0, 0.3, 1.0, 3.0, 1.0, 0.5][seed])
    if seed == 4:
        V[6:8] = 0.0  # B_t = 0: Alfven/slow or Alfven/fast degeneracy
    if seed == 5:
        V[5] = 0.0  # B_n = 0: slow waves collapse onto the entropy wave
    ch = 2.5
    lam, L, R = O.mhd_eigen(V, G53, ch)
    assert np.allclose(L @ R.T, np.eye(9), atol=1e-12)
    A = primitive_jacobian_7(V, G53)
    L7 = L[:7][:, IDX7]
    R7 = R[:7][:, IDX7]
    assert np.allclose(L7 @ A @ R7.T, np.diag(lam[:7]), atol=1e-11)
    ev = np.sort(np.linalg.eigvals(A).real)
    assert np.allclose(np.sort(lam[:7]), ev, atol=1e-7)
    G = np.array([[0.0, 1.0], [ch * ch, 0.0]])
    Lg = L[7:][:, [5, 8]]
    Rg = R[7:][:, [5, 8]]
    assert np.allclose(Lg @ G @ Rg.T, np.diag(lam[7:]), atol=1e-12)


def test_fast_speed_is_largest_jacobian_eigenvalue():
    rng = np.random.default_rng(7)
    for _ in range(20):
        V = _rand_state(rng)
        V[1] = 0.0
        cf = O.mhd_cfast(V, G53)
        assert cf == pytest.approx(np.linalg.eigvals(primitive_jacobian_7(V, G53)).real.max(),
                                   rel=1e-9)


def test_prim_cons_roundtrip():
    rng = np.random.default_rng(3)
    for _ in range(50):
        V = _rand_state(rng)
        U = O.mhd_prim2cons(V, G53)
        V2, bad = O.mhd_cons2prim(U, G53)
        assert bad == 0
        assert np.allclose(V2, V, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------- Riemann solver

def _phys_flux(V, gamma):
    rho, u, v, w, p, Bn, B1, B2, psi = V
    B2s = Bn * Bn + B1 * B1 + B2 * B2
    E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w) + 0.5 * B2s
    pt = p + 0.5 * B2s
    vB = u * Bn + v * B1 + w * B2
    return np.array([rho * u, rho * u * u + pt - Bn * Bn, rho * u * v - Bn * B1,
                     rho * u * w - Bn * B2, (E + pt) * u - Bn * vB, 0.0,
                     u * B1 - Bn * v, u * B2 - Bn * w, 0.0])


def test_riemann_consistency():
    """R(V, V) = F(V) of Eq. (1), plus the GLM fluxes (psi, c_h^2 B_n)."""
    rng = np.random.default_rng(11)
    ch = 3.0
    for _ in range(30):
        V = _rand_state(rng)
        F = O.mhd_riemann(V, V, G53, ch)
        ref = _phys_flux(V, G53)
        ref[5] = V[8]
        ref[8] = ch * ch * V[5]
        assert np.allclose(F, ref, rtol=1e-12, atol=1e-12)


def test_riemann_supersonic_upwinding():
    """If both states move faster than every signal to the right, the flux is
    the left physical flux (and vice versa)."""
    rng = np.random.default_rng(12)
    for sgn in (1.0, -1.0):
        VL = _rand_state(rng, 0.2)
        VR = _rand_state(rng, 0.2)
        VL[8] = VR[8] = 0.0
        VR[5] = VL[5]
        VL[1] = VR[1] = 30.0 * sgn
        F = O.mhd_riemann(VL, VR, G53, 1.0)
        ref = _phys_flux(VL if sgn > 0 else VR, G53)
        assert np.allclose(F[[0, 1, 2, 3, 4, 6, 7]], ref[[0, 1, 2, 3, 4, 6, 7]], rtol=1e-12)


def test_riemann_hydro_contact_is_exact():
    """B = 0, an isolated contact (equal p and u): the HLLD middle states
    resolve it exactly, so the flux is the upwind physical flux."""
    VL = np.array([1.0, 0.3, 0.1, -0.2, 1.0, 0, 0, 0, 0])
    VR = np.array([0.125, 0.3, -0.4, 0.5, 1.0, 0, 0, 0, 0])
    F = O.mhd_riemann(VL, VR, 1.4, 1.0)
    assert np.allclose(F[[0, 1, 2, 3, 4]], _phys_flux(VL, 1.4)[[0, 1, 2, 3, 4]], rtol=1e-13)


# --------------------------------------------------------------- reconstruction pieces

def test_tracing_of_uniform_advection_at_unit_courant():
    """A pure density (entropy) wave, linear MC reconstruction, entropy-wave
    Courant number nu = 1: the traced + state is the half-step average of the
    linear profile over [1/2 - nu, 1/2], i.e. exactly w_0; the - state (traced
    as well, by the same profile) is w_0 - slope; with the literal upwind
    selection it stays at w_0 - slope/2."""
    g = 1.4
    rho = np.array([1.0, 1.1, 1.3, 1.45, 1.5])
    slope = 0.175  # MC: mm((0.2 + 0.15)/2, 2 mm(0.2, 0.15))
    vs = np.zeros((5, 9))
    vs[:, 0] = rho
    vs[:, 1] = 2.0
    vs[:, 4] = 1.0
    Vp, Vm = O.mhd_char_predict(vs, g, 1.0, 0.5, recon=0)  # nu = 2.0 * 0.5 = 1
    assert Vp[0] == pytest.approx(rho[2], rel=1e-13)
    assert Vm[0] == pytest.approx(rho[2] - slope, rel=1e-13)
    Vp, Vm = O.mhd_char_predict(vs, g, 1.0, 0.5, recon=0, upwind=1)
    assert Vp[0] == pytest.approx(rho[2], rel=1e-13)
    assert Vm[0] == pytest.approx(rho[2] - 0.5 * slope, rel=1e-13)


def test_monotone_data_give_monotone_interfaces():
    rng = np.random.default_rng(5)
    for recon in (0, 1):
        for _ in range(40):
            rho = np.sort(rng.uniform(0.5, 2.0, size=5))
            vs = np.zeros((5, 9))
            vs[:, 0] = rho
            vs[:, 4] = 1.0
            Vp, Vm = O.mhd_char_predict(vs, 1.4, 1.0, 0.0, recon)
            assert rho[1] - 1e-14 <= Vm[0] <= rho[2] + 1e-14
            assert rho[2] - 1e-14 <= Vp[0] <= rho[3] + 1e-14


def test_local_extremum_is_flattened():
    vs = np.zeros((5, 9))
    vs[:, 0] = [1.0, 1.2, 1.5, 1.1, 1.0]
    vs[:, 4] = 1.0
    for recon in (0, 1):
        Vp, Vm = O.mhd_char_predict(vs, 1.4, 1.0, 0.0, recon)
        assert Vp[0] == pytest.approx(1.5, abs=1e-14)
        assert Vm[0] == pytest.approx(1.5, abs=1e-14)


# --------------------------------------------------------------- whole-step pins

def _sod_along(axis, N):
    g = 1.4
    n = [2, 2, 2]
    n[axis] = N
    dxs = [1.0 / N] * 3
    x = (np.arange(N) + 0.5) / N
    rho = np.where(x < 0.5, 1.0, 0.125)
    p = np.where(x < 0.5, 1.0, 0.1)
    shp = [1, 1, 1]
    shp[2 - axis] = N
    z = np.zeros(n[::-1])
    r3 = z + rho.reshape(shp)
    p3 = z + p.reshape(shp)
    U = np.zeros(O.shape(n, 3))
    O.interior(U, n, 3)[:] = W.ideal_cons([r3, z, z, z, p3, z, z, z, z], g)
    U, t, _ = O.mhd_run(U, n, 3, dxs, 0, 0.4, gamma=g, recon=1, bc="outflow", t_end=0.2)
    rn = np.moveaxis(O.interior(U, n, 3)[0], 2 - axis, 0)[:, 0, 0]
    ex = O.euler_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, (x - 0.5) / t)[:, 0]
    return rn, np.abs(rn - ex).mean()


def test_exact_euler_riemann_problem():
    """Sod's problem (B = 0): L1(rho) against the exact solution decreases at
    about first order and is small; the same problem embedded along x, y and
    z of a 3-D patch gives the same result to round-off."""
    errs = []
    for N in (50, 100, 200):
        rx, e = _sod_along(0, N)
        errs.append(e)
    order = np.log2(errs[0] / errs[-1]) / 2
    assert 0.75 < order < 1.3, errs
    assert errs[-1] < 4e-3, errs
    for axis in (1, 2):
        r, e = _sod_along(axis, 200)
        assert np.allclose(r, rx, rtol=0, atol=1e-13)


def test_exact_euler_double_rarefaction():
    """Two symmetric rarefactions (a milder form of Toro's 123 problem)."""
    g = 1.4
    N = 200
    n = [N, 1, 1]
    x = (np.arange(N) + 0.5) / N
    rho = np.ones(N)
    u = np.where(x < 0.5, -1.0, 1.0)
    p = 0.4 * np.ones(N)
    z = np.zeros(N)
    U = np.zeros(O.shape(n, 1))
    O.interior(U, n, 1)[:] = W.ideal_cons([rho, u, z, z, p, z, z, z, z], g).reshape(9, 1, 1, N)
    U, t, _ = O.mhd_run(U, n, 1, [1.0 / N, 1, 1], 0, 0.4, gamma=g, recon=1, bc="outflow",
                        t_end=0.15)
    rn = O.interior(U, n, 1)[0].ravel()
    ex = O.euler_sample((1.0, -1.0, 0.4), (1.0, 1.0, 0.4), g, (x - 0.5) / t)[:, 0]
    err = np.abs(rn - ex).mean()
    assert err < 0.01, err


@pytest.mark.parametrize("wave", ["fast", "slow", "alfven", "entropy"])
def test_linear_eigenmode_second_order(wave):
    """A travelling linear eigenmode returns to its initial state after one
    period; the L1 error over all variables converges at second order."""
    errs = []
    for N in (16, 32, 64):
        U, U0, T = oblique_wave_2d(N, wave)
        n = [N, N, 1]
        U, t, _ = O.mhd_run(U, n, 2, [1.0 / N, 1.0 / N, 1.0], 0, 0.4, recon=1, t_end=T)
        errs.append(np.abs(O.interior(U, n, 2) - U0).sum() / 1e-6 / (N * N))
    order = np.log2(errs[1] / errs[2])
    assert order > 1.85, errs


def test_conservation_periodic_2d_and_3d():
    """Periodic boxes: sums of rho, m, E, B are constant to round-off; the psi
    sum is multiplied by exactly the damping factor each step."""
    for ndim, U, n in ((2, W.mhd_turb_2d(32, seed=1), [32, 32, 1]),
                       (3, W.mhd_blast_3d(16, seed=2, kmax=3), [16, 16, 16])):
        dxs = [1.0 / n[0]] * 3
        S0 = O.interior(U, n, ndim).sum(axis=(1, 2, 3))
        scale = np.abs(O.interior(U, n, ndim)).sum(axis=(1, 2, 3))
        psi_sum = S0[8]
        for k in range(6):
            O.fill_periodic(U, n, ndim)
            m = O.mhd_max_speed(U, n, ndim, dxs)
            dt, ch = O.dt_ch(m, dxs, ndim, 0.3)
            U, bad = O.mhd_step(U, n, ndim, dxs, dt, ch, recon=1)
            assert bad == 0
            psi_sum = psi_sum * np.exp(-0.1 * ch * dt / dxs[0])
        S = O.interior(U, n, ndim).sum(axis=(1, 2, 3))
        assert np.all(np.abs(S - S0)[:8] <= 1e-13 * scale[:8]), (S - S0, scale)
        assert abs(S[8] - psi_sum) < 1e-13 * scale[5:8].sum()
        assert np.abs(O.interior(U, n, ndim)[8]).max() > 1e-6  # psi was excited


def test_glm_uniform_psi_decays_at_the_analytic_rate():
    """Uniform divergence-free data with uniform psi_0: the state is preserved
    bitwise and psi_n = psi_0 prod_k exp(-alpha c_h dt_k / dx)."""
    n = [8, 8, 8]
    rho, p = 1.3, 0.7
    Vc = [rho, 0.2, -0.1, 0.3, p, 0.5, -0.4, 0.8, 0.25]
    shp = O.shape(n, 3)[1:]
    U = W.ideal_cons([np.full(shp, v) for v in Vc], G53)
    U0 = U.copy()
    dxs = [1.0 / 8] * 3
    psi = 0.25
    for k in range(5):
        O.fill_periodic(U, n, 3)
        m = O.mhd_max_speed(U, n, 3, dxs)
        dt, ch = O.dt_ch(m, dxs, 3, 0.3)
        U, bad = O.mhd_step(U, n, 3, dxs, dt, ch, glm_alpha=0.3, recon=1)
        psi *= np.exp(-0.3 * ch * dt / dxs[0])
    I = O.interior(U, n, 3)
    assert np.array_equal(I[:8], O.interior(U0, n, 3)[:8])
    assert np.allclose(I[8], psi, rtol=1e-14, atol=0)


def test_glm_telegraph_mode():
    """Injected div B error B_x = eps sin(2 pi x) on a static B = 0 background:
    linear theory of Eq. (glm2x2) gives B_x(t) = eps e^{-kt/2} [cos wt +
    k/(2w) sin wt] sin 2 pi x with k = c_h^2/c_p^2 and w^2 = c_h^2 (2 pi)^2 -
    k^2/4; the measured amplitude converges to it."""
    kap = 2.0
    T = 0.5
    eps = 1e-6
    errs = []
    for N in (32, 64, 128):
        n = [N, 1, 1]
        x = (np.arange(N) + 0.5) / N
        z = np.zeros(N)
        Bx = eps * np.sin(2 * np.pi * x)
        U = np.zeros(O.shape(n, 1))
        O.interior(U, n, 1)[:] = W.ideal_cons([z + 1, z, z, z, z + 1, Bx, z, z, z],
                                              G53).reshape(9, 1, 1, N)
        dx = 1.0 / N
        t = 0.0
        while t < T * (1 - 1e-14):
            O.fill_periodic(U, n, 1)
            m = O.mhd_max_speed(U, n, 1, [dx, 1, 1])
            dt, ch = O.dt_ch(m, [dx, 1, 1], 1, 0.8)
            dt = min(dt, T - t)
            alpha = kap * dx / ch  # c_h^2/c_p^2 = alpha c_h / dx = kap
            U, bad = O.mhd_step(U, n, 1, [dx, 1, 1], dt, ch, glm_alpha=alpha, recon=1)
            t += dt
        amp = 2.0 * np.mean(O.interior(U, n, 1)[5].ravel() * np.sin(2 * np.pi * x))
        w = np.sqrt(ch * ch * (2 * np.pi) ** 2 - kap * kap / 4)
        exact = eps * np.exp(-kap * T / 2) * (np.cos(w * T) + kap / (2 * w) * np.sin(w * T))
        errs.append(abs(amp - exact) / eps)
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.02, errs


def test_mirror_and_swap_symmetry():
    """x -> -x (v_x, B_x odd) and, in 2D, x <-> y are symmetries of Eq. (1) +
    Eq. (glm2x2); the step commutes with them to round-off."""
    n = [24, 24, 1]
    dxs = [1.0 / 24] * 3
    U = W.mhd_turb_2d(24, seed=4)

    def run(U):
        U = U.copy()
        for _ in range(4):
            O.fill_periodic(U, n, 2)
            dt, ch = O.dt_ch(O.mhd_max_speed(U, n, 2, dxs), dxs, 2, 0.4)
            U, bad = O.mhd_step(U, n, 2, dxs, dt, ch, recon=1)
        return O.interior(U, n, 2)

    ref = run(U)
    scale = np.abs(ref).max(axis=(1, 2, 3))[:, None, None, None]
    for fwd, inv in ((mirror_x, mirror_x), (swap_xy, swap_xy)):
        out = inv(run(fwd(U)))
        assert np.all(np.abs(out - ref) <= 1e-12 * scale)

    n3 = [12, 12, 12]
    d3 = [1.0 / 12] * 3
    U3 = W.mhd_blast_3d(12, seed=5, kmax=2)

    def run3(U):
        U = U.copy()
        for _ in range(3):
            O.fill_periodic(U, n3, 3)
            dt, ch = O.dt_ch(O.mhd_max_speed(U, n3, 3, d3), d3, 3, 0.3)
            U, bad = O.mhd_step(U, n3, 3, d3, dt, ch, recon=1)
        return O.interior(U, n3, 3)

    ref = run3(U3)
    scale = np.abs(ref).max(axis=(1, 2, 3))[:, None, None, None]
    for f in (mirror_x, mirror_z):
        assert np.all(np.abs(f(run3(f(U3))) - ref) <= 1e-12 * scale)


def test_flux_registers_restore_conservation_two_levels():
    """A fine patch (ratio 2, two substeps) inside a periodic coarse patch:
    refluxing with the coarse and fine registers, Eq. (fluxcorr) and
    (addreflux), and averaging down, Eq. (avgdown), conserves the totals to
    round-off; without the reflux they are off by far more."""
    Nc = 32
    nc = [Nc, Nc, 1]
    hc = 1.0 / Nc
    hf = hc / 2
    U = W.mhd_turb_2d(Nc, seed=6)
    Ic = O.interior(U, nc, 2)
    lo, hi = 8, 24
    nfc = hi - lo
    nf = [2 * nfc, 2 * nfc, 1]
    total0 = Ic.sum(axis=(1, 2, 3)) * hc * hc
    # coarse windows at the coarse-fine interface; each coarse face plane has
    # nfc faces; registers laid out one window after another
    cw = []
    off = 0
    for d in (0, 1):
        for f in (lo, hi):
            cw.append((d, f, lo, hi, 0, 1, off, 1.0))
            off += 9 * nfc
    regc = np.zeros(off)
    fw, fsize = O.boundary_windows(nf, 2, weight=1.0)
    regf = np.zeros(fsize)
    # coarse step
    O.fill_periodic(U, nc, 2)
    dt, ch = O.dt_ch(O.mhd_max_speed(U, nc, 2, [hc, hc]), [hc, hc], 2, 0.4)
    Unew, bad = O.mhd_step(U, nc, 2, [hc, hc, 1], dt, ch, recon=1, windows=cw, reg=regc)
    # fine patch initialised by injection; its ghosts come from the old coarse
    # data at both substeps
    gi = np.arange(-4, nf[0] + 4)
    ci = lo + np.floor_divide(gi, 2) + 4  # ghosted coarse index
    frame = U[:, :, ci][:, :, :, ci].copy()
    Uf = frame.copy()
    for q in range(2):
        Ufn, bad = O.mhd_step(Uf, nf, 2, [hf, hf, 1], dt / 2, ch, recon=1, windows=fw,
                              reg=regf)
        assert bad == 0
        Uf = frame.copy()
        Uf[:, :, 4:-4, 4:-4] = Ufn[:, :, 4:-4, 4:-4]
    In = O.interior(Unew, nc, 2)
    If = O.interior(Ufn, nf, 2)
    # average down (Eq. avgdown)
    In[:, 0, lo:hi, lo:hi] = 0.25 * (If[:, 0, 0::2, 0::2] + If[:, 0, 1::2, 0::2]
                                     + If[:, 0, 0::2, 1::2] + If[:, 0, 1::2, 1::2])
    no_reflux = In.sum(axis=(1, 2, 3)) * hc * hc
    # reflux (Eq. addreflux) into the uncovered coarse neighbours
    V = hc * hc
    k = 0
    for d in (0, 1):
        for side, f in enumerate((lo, hi)):
            rc = regc[9 * nfc * k: 9 * nfc * (k + 1)].reshape(9, nfc)
            k += 1
            fi = 2 * d + side
            rf = regf[9 * 2 * nfc * fi: 9 * 2 * nfc * (fi + 1)].reshape(9, 2 * nfc)
            rfs = rf[:, 0::2] + rf[:, 1::2]
            corr = (rc - rfs) if side == 0 else (rfs - rc)
            cell = f - 1 if side == 0 else f
            if d == 0:
                In[:, 0, lo:hi, cell] += corr / V
            else:
                In[:, 0, cell, lo:hi] += corr / V
    total = In.sum(axis=(1, 2, 3)) * hc * hc
    scale = np.abs(In).sum(axis=(1, 2, 3)) * hc * hc
    assert np.all(np.abs(total - total0)[:8] <= 1e-13 * scale[:8]), (total - total0)
    assert np.abs(no_reflux - total0)[[0, 4]].max() > 1e-8


def _cons_flux_x(U, gamma, ch):
    """Conservative GLM-MHD flux along x (Eq. 1 + Eq. glm2x2) as a function of U."""
    rho, mx, my, mz, E, bx, by, bz, psi = U
    u, v, w = mx / rho, my / rho, mz / rho
    B2 = bx * bx + by * by + bz * bz
    p = (gamma - 1) * (E - 0.5 * rho * (u * u + v * v + w * w) - 0.5 * B2)
    pt = p + 0.5 * B2
    vB = u * bx + v * by + w * bz
    return np.array([mx, mx * u + pt - bx * bx, my * u - bx * by, mz * u - bx * bz,
                     (E + pt) * u - bx * vB, psi, u * by - bx * v, u * bz - bx * w,
                     ch * ch * bx])


def test_glm_mhd_monopole_wave_second_order():
    """A div B != 0 perturbation (B_x = B_x0 + eps sin kx, plus density and
    pressure perturbations) on a moving magnetised background, 1-D.  The exact
    solution of the linearised conservative GLM-MHD system is
    U_k(t) = expm(-i k A t) U_k(0) with A the flux Jacobian (taken by central
    differences of the flux of Eq. 1 + Eq. glm2x2).  The step must converge to
    it at second order: this needs the S_Bx and S_psi terms of the primitive
    predictor, which vanish for divergence-free data."""
    from scipy.linalg import expm
    g = G53
    V0 = np.array([1.0, 0.2, 0.3, -0.1, 1.0, 0.8, 0.5, 0.2, 0.0])
    U0 = W.ideal_cons([np.array(v) for v in V0], g).astype(float)
    dU = np.array([0.5, 0.0, 0.0, 0.0, 0.7, 1.0, 0.0, 0.0, 0.0])
    eps, k, T = 1e-6, 2 * np.pi, 0.3
    errs = []
    for N in (32, 64, 128):
        n = [N, 1, 1]
        x = (np.arange(N) + 0.5) / N
        Ui = U0[:, None] + eps * dU[:, None] * np.sin(k * x)[None, :]
        U = np.zeros(O.shape(n, 1))
        O.interior(U, n, 1)[:] = Ui.reshape(9, 1, 1, N)
        dx = 1.0 / N
        t = 0.0
        chs = []
        while t < T * (1 - 1e-14):
            O.fill_periodic(U, n, 1)
            dt, ch = O.dt_ch(O.mhd_max_speed(U, n, 1, [dx, 1, 1]), [dx, 1, 1], 1, 0.6)
            dt = min(dt, T - t)
            U, bad = O.mhd_step(U, n, 1, [dx, 1, 1], dt, ch, glm_alpha=0.0, recon=1)
            chs.append(ch)
            t += dt
        ch = float(np.mean(chs))
        h = 1e-6
        A = np.zeros((9, 9))
        for j in range(9):
            e = np.zeros(9)
            e[j] = h
            A[:, j] = (_cons_flux_x(U0 + e, g, ch) - _cons_flux_x(U0 - e, g, ch)) / (2 * h)
        c0 = -0.5j * eps * dU  # sin(kx) = Im e^{ikx}: coefficient of e^{ikx}
        cT = expm(-1j * k * A * T) @ c0
        dUn = O.interior(U, n, 1).reshape(9, N) - U0[:, None]
        cn = (dUn * np.exp(-1j * k * x)[None, :]).mean(axis=1)
        errs.append(np.abs(cn - cT).sum() / eps)
    order = np.log2(errs[1] / errs[2])
    assert order > 1.8, errs
