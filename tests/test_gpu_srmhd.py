"""Parity of the SRMHD CUDA path (MUSCL-Hancock, HLL, GLM, float64 Newton
recovery) with the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import gpu_run, l1rel, maxrel

pytestmark = pytest.mark.gpu
G43 = 4.0 / 3.0
TOL64 = 1e-11


def _oracle(U0, n, ndim, dx, steps, cfl):
    U, t, dts = O.srmhd_run(U0, n, ndim, list(dx) + [1.0] * (3 - len(dx)), steps, cfl, gamma=G43)
    return U, dts


def test_srmhd_2d_wave_fp64():
    n = [32, 32, 1]
    x = (np.arange(32) + 0.5) / 32
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = 1 + 0.3 * np.sin(2 * np.pi * (X + Y))
    z = np.zeros_like(rho)
    Vp = [rho, 0.3 + 0.1 * np.cos(2 * np.pi * Y), z + 0.4, z + 0.1, 0.5 + 0.1 * np.sin(2 * np.pi * X),
          z + 0.3, 0.4 + 0.1 * np.cos(2 * np.pi * X), z + 0.2, z]
    U0 = np.zeros(O.shape(n, 2))
    O.interior(U0, n, 2)[:] = W.srmhd_cons(Vp, G43)[:, None]
    got, gd, st = gpu_run(U0, n, 2, [1 / 32, 1 / 32], 10, 0.4, gamma=G43, physics=1)
    assert st == 0
    ref, od = _oracle(U0, n, 2, [1 / 32, 1 / 32], 10, 0.4)
    for (a, b), (c, d) in zip(gd, od):
        assert abs(a - c) <= 1e-13 * c and abs(b - d) <= 1e-13 * d
    e = l1rel(O.interior(got, n, 2), O.interior(ref, n, 2), od[-1][1])
    assert np.all(e <= TOL64), e


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, 2e-4)])
def test_srmhd_jet_3d(prec, tol):
    """The gamma-10 magnetised beam on 24^3, 5 steps."""
    n = [24, 24, 24]
    U0 = W.srmhd_jet_3d(24, seed=7)
    dx = [1 / 24] * 3
    got, gd, st = gpu_run(U0, n, 3, dx, 5, 0.3, precision=prec, gamma=G43, physics=1)
    assert st == 0
    ref, od = _oracle(U0, n, 3, dx, 5, 0.3)
    e = l1rel(O.interior(got, n, 3), O.interior(ref, n, 3), od[-1][1])
    assert np.all(e <= tol), e
    em = maxrel(O.interior(got, n, 3), O.interior(ref, n, 3), od[-1][1])
    assert np.all(em <= (TOL64 if prec == 0 else 1e-3)), em


def test_srmhd_full_size_sampled_256():
    """256^3 jet, one GPU step (FP64 and mixed) against the oracle on sampled
    6^3 blocks recomputed from their own ghosted neighbourhood."""
    import torch
    from paper_1110_0740_gb300 import ctu
    n = 256
    U0 = W.srmhd_jet_3d(n, seed=0)
    dev = torch.device("cuda:0")
    U = torch.from_numpy(U0.reshape(9, -1)).to(dev)
    Uo = torch.zeros_like(U)
    stride = U.shape[1]
    patches = ctu.make_patches([([n] * 3, [1.0 / n] * 3, 0)])
    rng = np.random.default_rng(3)
    # blocks through the beam edge and the ambient medium
    corners = [rng.integers(0, n - 6, size=3) for _ in range(4)]
    for prec, tol in ((ctu.CTU_FP64, TOL64), (ctu.CTU_MIXED, 2e-4)):
        cfg = ctu.make_config(ndim=3, gamma=G43, recon=ctu.CTU_LINEAR_MC, precision=prec, cfl=0.3,
                              physics=ctu.CTU_SRMHD, predictor=ctu.CTU_MUSCL_HANCOCK,
                              riemann=ctu.CTU_HLL)
        ctx = ctu.Ctx(cfg)
        dtch = torch.zeros(2, dtype=torch.float64, device=dev)
        ctx.dt(U, stride, patches, dtch)
        ctx.step(U, Uo, stride, patches, dtch)
        assert ctx.status_sync() == 0
        dt, ch = dtch.cpu().tolist()
        G = Uo.view(9, n + 8, n + 8, n + 8)
        for c in corners:
            k, j, i = (int(v) for v in c[::-1])
            blk = U0[:, k:k + 14, j:j + 14, i:i + 14].copy()
            R, bad = O.srmhd_step(blk, [6, 6, 6], 3, [1.0 / n] * 3, dt, ch, gamma=G43)
            assert bad == 0
            got = G[:, k + 4:k + 10, j + 4:j + 10, i + 4:i + 10].cpu().numpy()
            e = l1rel(got, O.interior(R, [6, 6, 6], 3), ch, group_floor=True)
            assert np.all(e <= tol), (prec, c, e)
        ctx.close()


def test_srmhd_bad_state_flags():
    import torch
    from paper_1110_0740_gb300 import ctu
    n = [8, 8, 8]
    U0 = W.srmhd_jet_3d(8, seed=1, lorentz=2.0)
    U0[4, 6, 6, 6] = -5.0  # total energy below the rest mass: no physical state
    dev = torch.device("cuda:0")
    U = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
    Uo = torch.zeros_like(U)
    cfg = ctu.make_config(ndim=3, gamma=G43, recon=ctu.CTU_LINEAR_MC, physics=ctu.CTU_SRMHD,
                          predictor=ctu.CTU_MUSCL_HANCOCK, riemann=ctu.CTU_HLL)
    ctx = ctu.Ctx(cfg)
    p = ctu.make_patches([(n, [1 / 8] * 3, 0)])
    dtch = torch.tensor([1e-3, 1.0], dtype=torch.float64, device=dev)
    ctx.step(U, Uo, U.shape[1], p, dtch)
    assert ctu.STATUS[ctx.status_sync()] in ("CTU_ENEGATIVE", "CTU_ERECOVERY", "CTU_ESUPERLUMINAL",
                                             "CTU_ENAN")


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, 2e-4)])
def test_srmhd_taub_mathews_jet_3d(prec, tol):
    """The Taub-Mathews equation of state (Eq. TMEos): the gamma-10 beam on
    24^3, 5 steps, against the oracle with the same equation of state.  The
    beam runs at p0 = 0.05: at the workload's 0.01 the Taub-Mathews gas,
    stiffer when cold (Gamma -> 5/3), reaches negative pressure at the beam
    edge by the second step in the oracle and on the GPU alike."""
    n = [24, 24, 24]
    U0 = W.srmhd_jet_3d(24, seed=8, gamma=0.0, p0=0.05)
    dx = [1 / 24] * 3
    got, gd, st = gpu_run(U0, n, 3, dx, 5, 0.3, precision=prec, gamma=0.0, physics=1, eos=1)
    assert st == 0
    ref, _, od = O.srmhd_run(U0, n, 3, dx, 5, 0.3, gamma=0.0)
    for (a, b), (c, d) in zip(gd, od):
        assert abs(a - c) <= (1e-13 if prec == 0 else 1e-5) * c
    e = l1rel(O.interior(got, n, 3), O.interior(ref, n, 3), od[-1][1], group_floor=True)
    assert np.all(e <= tol), e


def test_srmhd_taub_mathews_hot_wave_fp64():
    """A hot (p/rho ~ 10) relativistic 2-D wave with the Taub-Mathews gas."""
    n = [32, 32, 1]
    x = (np.arange(32) + 0.5) / 32
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = 1 + 0.3 * np.sin(2 * np.pi * (X + Y))
    z = np.zeros_like(rho)
    Vp = [rho, 0.3 + 0.1 * np.cos(2 * np.pi * Y), z + 0.4, z + 0.1, 10.0 + np.sin(2 * np.pi * X),
          z + 0.3, 0.4 + 0.1 * np.cos(2 * np.pi * X), z + 0.2, z]
    U0 = np.zeros(O.shape(n, 2))
    O.interior(U0, n, 2)[:] = W.srmhd_cons(Vp, 0.0)[:, None]
    got, gd, st = gpu_run(U0, n, 2, [1 / 32, 1 / 32], 10, 0.4, gamma=0.0, physics=1, eos=1)
    assert st == 0
    ref, _, od = O.srmhd_run(U0, n, 2, [1 / 32, 1 / 32, 1.0], 10, 0.4, gamma=0.0)
    e = l1rel(O.interior(got, n, 2), O.interior(ref, n, 2), od[-1][1])
    assert np.all(e <= TOL64), e


def test_taub_mathews_is_relativistic_only():
    from paper_1110_0740_gb300 import ctu
    with pytest.raises(ctu.CtuError) as e:
        ctu.Ctx(ctu.make_config(eos=ctu.CTU_EOS_TM))
    assert e.value.code == 4
