"""The parabolic terms of the CTU step, thermal conduction, viscosity and
resistivity, on the GPU against the oracle: 3-D blast with PPM, 2-D turbulence with
MC-linear and 1-D diffusion-dominated cases, float64 (relative L1 1e-11) and
mixed (the float tracing bar of the plain step); a ragged batch of patches
in one call; the CFL rate with its diffusion term (ctu_dt and the step's
next dt); flux registers with the parabolic momentum, energy and B
fluxes."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import gpu_run, l1rel, oracle_run

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def _dev():
    import torch
    return torch.device("cuda:0")


@pytest.mark.parametrize("trace_mode,kappa,nu,eta", [(0, 0.01, 0.0, 0.0), (1, 0.01, 0.0, 0.0), (0, 0.0, 0.01, 0.0),
                                                     (0, 0.0, 0.0, 0.01), (1, 0.004, 0.004, 0.004)])
def test_parabolic_3d_blast_ppm(trace_mode, kappa, nu, eta):
    n = [24, 24, 24]
    U0 = W.mhd_blast_3d(24, seed=31)
    dx = [1.0 / 24] * 3
    ref, od = oracle_run(U0, n, 3, dx, 4, 0.3, recon=1, trace_mode=trace_mode, kappa=kappa, nu=nu, eta=eta)
    plain, _ = oracle_run(U0, n, 3, dx, 4, 0.3, recon=1, trace_mode=trace_mode)
    R = O.interior(ref, n, 3)
    # the parabolic terms change the state well above the tolerances below
    q = 4 if kappa else (1 if nu else 6)
    assert np.abs(R[q] - O.interior(plain, n, 3)[q]).sum() > 1e-3 * np.abs(R[q]).sum()
    for prec, tol in ((0, TOL64), (1, 2e-5)):
        got, gd, st = gpu_run(U0, n, 3, dx, 4, 0.3, precision=prec, recon=1, trace_mode=trace_mode, kappa=kappa,
                              nu=nu, eta=eta)
        assert st == 0
        e = l1rel(O.interior(got, n, 3), R, od[-1][1])
        assert np.all(e <= tol), (prec, e)
        if prec == 0:
            assert np.allclose(np.array(gd), np.array(od), rtol=1e-13, atol=0)


@pytest.mark.parametrize("kappa,nu,eta", [(0.02, 0.0, 0.0), (0.0, 0.01, 0.0), (0.0, 0.0, 0.01), (0.01, 0.01, 0.01)])
def test_parabolic_2d_turbulence_mc(kappa, nu, eta):
    n = [48, 48, 1]
    U0 = W.mhd_turb_2d(48, seed=32)
    dx = [1.0 / 48] * 2
    ref, od = oracle_run(U0, n, 2, dx, 10, 0.4, recon=0, kappa=kappa, nu=nu, eta=eta)
    R = O.interior(ref, n, 2)
    for prec, tol in ((0, TOL64), (1, 1e-4)):
        got, _, st = gpu_run(U0, n, 2, dx, 10, 0.4, precision=prec, recon=0, kappa=kappa, nu=nu, eta=eta)
        assert st == 0
        G = O.interior(got, n, 2)
        assert not np.any(G[3]) and not np.any(G[7])
        e = l1rel(G, R, od[-1][1])
        assert np.all(e <= tol), (prec, e)


@pytest.mark.parametrize("kappa,nu,eta", [(0.5, 0.0, 0.0), (0.0, 0.3, 0.0), (0.0, 0.0, 0.3), (0.2, 0.2, 0.2)])
def test_parabolic_1d_diffusion_dominated(kappa, nu, eta):
    """1-D, a density wave with a transverse shear on a moving gas, in the
    regime where the diffusion term sets dt (oracle pins: the linear modes)."""
    N = 64
    n = [N, 1, 1]
    shp = O.shape(n, 1)
    x = (np.arange(shp[3]) - 4 + 0.5) / N
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * x)
    z = np.zeros_like(rho)
    U0 = np.zeros(shp)
    U0[:, 0, 0] = W.ideal_cons([rho, z + 0.3, 0.1 * np.sin(2 * np.pi * x), z, z + 1.0, z + 0.4,
                                0.2 + 0.05 * np.cos(2 * np.pi * x), z, z], 5.0 / 3.0)
    dx = [1.0 / N]
    ref, od = oracle_run(U0, n, 1, dx, 30, 0.4, recon=1, kappa=kappa, nu=nu, eta=eta)
    R = O.interior(ref, n, 1)
    for prec, tol in ((0, TOL64), (1, 2e-5)):
        got, gd, st = gpu_run(U0, n, 1, dx, 30, 0.4, precision=prec, recon=1, kappa=kappa, nu=nu, eta=eta)
        assert st == 0
        e = l1rel(O.interior(got, n, 1), R, od[-1][1], group_floor=True)
        assert np.all(e <= tol), (prec, e)
    # the diffusion term sets dt here
    m_h = O.mhd_max_speed(U0, n, 1, dx)
    m = O.mhd_max_rate(U0, n, 1, dx, 5.0 / 3.0, kappa, nu, eta)
    assert m > 3 * m_h


@pytest.mark.parametrize("kappa,nu,eta", [(0.004, 0.0, 0.0), (0.002, 0.003, 0.003)])
def test_parabolic_batch_of_uneven_patches(kappa, nu, eta):
    """Four patches of different shapes and cell widths in one call, each
    against the oracle run patch by patch with the batch's dt."""
    import torch
    from paper_1110_0740_gb300 import ctu
    shapes = [(16, 16, 16), (8, 8, 8), (11, 1, 7), (5, 9, 3)]
    dxs = [(1 / 16,) * 3, (1 / 8,) * 3, (0.05, 0.07, 0.06), (0.08, 0.05, 0.1)]
    src = W.mhd_blast_3d(32, seed=33, kmax=3)
    arrays, bases, base = [], [], 0
    for i, n in enumerate(shapes):
        A = np.zeros(O.shape(list(n), 3))
        A[:] = src[:, 2 * i:2 * i + n[2] + 8, i:i + n[1] + 8, 3 * i:3 * i + n[0] + 8]
        arrays.append(A)
        bases.append(base)
        base += A[0].size + 13
    stride = base
    pool = np.zeros((9, stride))
    for A, b in zip(arrays, bases):
        pool[:, b:b + A[0].size] = A.reshape(9, -1)
    dev = _dev()
    U = torch.from_numpy(pool).to(dev)
    Uo = torch.zeros_like(U)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64, cfl=0.3, kappa=kappa, nu=nu,
                                  eta=eta))
    patches = ctu.make_patches([(n, dx, b) for n, dx, b in zip(shapes, dxs, bases)])
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.dt(U, stride, patches, dtch)
    ctx.step(U, Uo, stride, patches, dtch)
    assert ctx.status_sync() == 0
    dt, ch = dtch.cpu().tolist()
    m = max(O.mhd_max_rate(A, list(n), 3, list(dx), 5.0 / 3.0, kappa, nu, eta)
            for A, n, dx in zip(arrays, shapes, dxs))
    dt_ref = 0.3 / m
    assert abs(dt - dt_ref) <= 1e-13 * dt_ref
    out = Uo.cpu().numpy()
    for A, n, dx, b in zip(arrays, shapes, dxs, bases):
        R, bad = O.mhd_step(A, list(n), 3, list(dx), dt, ch, recon=1, kappa=kappa, nu=nu, eta=eta)
        assert bad == 0
        G = out[:, b:b + A[0].size].reshape(A.shape)
        e = l1rel(O.interior(G, list(n), 3), O.interior(R, list(n), 3), ch)
        assert np.all(e <= TOL64), (n, e)


@pytest.mark.parametrize("prec,nu,eta", [(0, 0.0, 0.0), (1, 0.0, 0.0), (0, 0.03, 0.0), (1, 0.03, 0.0), (0, 0.0, 0.08),
                                         (1, 0.0, 0.08)])
def test_parabolic_next_dt_matches_ctu_dt(prec, nu, eta):
    import torch
    from paper_1110_0740_gb300 import ctu
    n = [20, 12, 16]
    U0 = np.zeros(O.shape(n, 3))
    O.interior(U0, n, 3)[:] = O.interior(W.mhd_blast_3d(20, seed=4, kmax=3), [20] * 3, 3)[:, :16, :12, :]
    O.fill_periodic(U0, n, 3)
    dev = _dev()
    U = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
    Ua, Ub = torch.zeros_like(U), torch.zeros_like(U)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3, kappa=0.05, nu=nu, eta=eta))
    p = ctu.make_patches([(n, [1 / 20, 1 / 12, 1 / 16], 0)])
    d0 = torch.zeros(2, dtype=torch.float64, device=dev)
    d1 = torch.zeros_like(d0)
    d2 = torch.zeros_like(d0)
    ctx.dt(U, U.shape[1], p, d0)
    ctx.step(U, Ua, U.shape[1], p, d0)
    ctx.step_next_dt(U, Ub, U.shape[1], p, d0, d1)
    ctx.dt(Ub, U.shape[1], p, d2)
    assert ctx.status_sync() == 0
    assert torch.equal(Ua, Ub)
    a, b = d1.cpu().numpy(), d2.cpu().numpy()
    assert np.allclose(a, b, rtol=1e-13 if prec == 0 else 1e-6, atol=0), (a, b)
    # and against the oracle's rate (float64)
    if prec == 0:
        m = O.mhd_max_rate(U0, n, 3, [1 / 20, 1 / 12, 1 / 16], 5.0 / 3.0, 0.05, nu, eta)
        assert abs(d0.cpu().numpy()[0] - 0.3 / m) <= 1e-14 * 0.3 / m


@pytest.mark.parametrize("prec,nu,eta", [(0, 0.0, 0.0), (1, 0.0, 0.0), (0, 0.02, 0.02), (1, 0.02, 0.02)])
def test_parabolic_flux_registers(prec, nu, eta):
    """Register windows on every boundary face and on an interior plane of a
    3-D patch, two steps accumulated: with the parabolic terms the momentum
    energy and B entries carry F - Pi^(n+1/2), as in the oracle (which
    conserves two levels with them, see the oracle pins)."""
    import torch
    from paper_1110_0740_gb300 import ctu
    n = [12, 10, 8]
    dx = [1 / 12, 1 / 10, 1 / 8]
    U0 = np.zeros(O.shape(n, 3))
    O.interior(U0, n, 3)[:] = O.interior(W.mhd_blast_3d(12, seed=34, kmax=3), [12] * 3, 3)[:, :8, :10, :]
    O.fill_periodic(U0, n, 3)
    windows, ws, off = [], [], 0
    for d in range(3):
        a_, b_ = [e for e in range(3) if e != d]
        for plane in (0, n[d] // 2, n[d]):
            windows.append((0, d, plane, 0, n[a_], 0, n[b_], 0.75, off))
            ws.append((d, plane, 0, n[a_], 0, n[b_], off, 0.75))
            off += 9 * n[a_] * n[b_]
    dev = _dev()
    kappa = 0.02
    U = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
    Uo = torch.zeros_like(U)
    reg = torch.zeros(off, dtype=torch.float64, device=dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3, kappa=kappa, nu=nu,
                                  eta=eta))
    p = ctu.make_patches([(n, dx, 0)])
    ctx.flux_registers(reg, windows)
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.dt(U, U.shape[1], p, dtch)
    ctx.step(U, Uo, U.shape[1], p, dtch)
    ctx.step(U, Uo, U.shape[1], p, dtch)
    assert ctx.status_sync() == 0
    dt, ch = dtch.cpu().tolist()
    ref = np.zeros(off)
    R, bad = O.mhd_step(U0, n, 3, dx, dt, ch, recon=1, windows=ws, reg=ref, kappa=kappa, nu=nu, eta=eta)
    O.mhd_step(U0, n, 3, dx, dt, ch, recon=1, windows=ws, reg=ref, kappa=kappa, nu=nu, eta=eta)
    assert bad == 0
    got = reg.cpu().numpy()
    # the energy entries differ from the hyperbolic-only registers
    ref0 = np.zeros(off)
    O.mhd_step(U0, n, 3, dx, dt, ch, recon=1, windows=ws, reg=ref0)
    O.mhd_step(U0, n, 3, dx, dt, ch, recon=1, windows=ws, reg=ref0)
    scale = np.abs(ref).max()
    assert np.abs(ref - ref0).max() > 1e-4 * scale
    tol = 1e-12 if prec == 0 else 2e-5
    assert np.abs(got - ref).max() <= tol * scale, np.abs(got - ref).max() / scale
    G = Uo.cpu().numpy().reshape(U0.shape)
    e = l1rel(O.interior(G, n, 3), O.interior(R, n, 3), ch)
    assert np.all(e <= (TOL64 if prec == 0 else 2e-5)), e


@pytest.mark.parametrize("case", ["blast3d", "turb2d"])
def test_anisotropic_conduction(case):
    """Conduction along the field (kappa_par) ten times that across it, alone
    and with viscosity and resistivity: FP64 at 1e-11 and mixed at the plain
    step's bars, against the oracle."""
    if case == "blast3d":
        n, U0, dx, steps, cfl, recon, tol = [24] * 3, W.mhd_blast_3d(24, seed=35), [1 / 24] * 3, 4, 0.3, 1, 2e-5
        nd = 3
    else:
        n, U0, dx, steps, cfl, recon, tol = [48, 48, 1], W.mhd_turb_2d(48, seed=36), [1 / 48] * 2, 10, 0.4, 0, 1e-4
        nd = 2
    for kw in (dict(kappa=0.002, kappa_par=0.02), dict(kappa=0.0, kappa_par=0.01, nu=0.003, eta=0.003)):
        ref, od = oracle_run(U0, n, nd, dx, steps, cfl, recon=recon, **kw)
        iso, _ = oracle_run(U0, n, nd, dx, steps, cfl, recon=recon, kappa=kw["kappa_par"],
                            nu=kw.get("nu", 0.0), eta=kw.get("eta", 0.0))
        R = O.interior(ref, n, nd)
        assert np.abs(R[4] - O.interior(iso, n, nd)[4]).sum() > 1e-5 * np.abs(R[4]).sum()
        for prec, t in ((0, TOL64), (1, tol)):
            got, _, st = gpu_run(U0, n, nd, dx, steps, cfl, precision=prec, recon=recon, **kw)
            assert st == 0
            e = l1rel(O.interior(got, n, nd), R, od[-1][1])
            assert np.all(e <= t), (kw, prec, e)


def test_saturated_conduction():
    """The saturated heat flux (harmonic mean with the upwind saturated flux),
    isotropic and anisotropic, on the 3-D blast whose hot sphere saturates:
    FP64 at 1e-11 and mixed at the plain step's bar, against the oracle."""
    n, dx = [24] * 3, [1 / 24] * 3
    U0 = W.mhd_blast_3d(24, seed=37)
    for kw in (dict(kappa=0.02, phi=0.01), dict(kappa=0.002, kappa_par=0.02, phi=0.01)):
        ref, od = oracle_run(U0, n, 3, dx, 4, 0.3, recon=1, **kw)
        cls, _ = oracle_run(U0, n, 3, dx, 4, 0.3, recon=1, **{k: v for k, v in kw.items() if k != "phi"})
        R = O.interior(ref, n, 3)
        assert np.abs(R[4] - O.interior(cls, n, 3)[4]).sum() > 1e-5 * np.abs(R[4]).sum()
        for prec, t in ((0, TOL64), (1, 2e-5)):
            got, _, st = gpu_run(U0, n, 3, dx, 4, 0.3, precision=prec, recon=1, **kw)
            assert st == 0
            e = l1rel(O.interior(got, n, 3), R, od[-1][1])
            assert np.all(e <= t), (kw, prec, e)
