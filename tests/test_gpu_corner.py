"""Parity of the corner coupling of Mignone & Tzeferacos (CTU_CORNER_MT:
transverse fluxes from Riemann problems between the normal predictor states,
Section 3.1 with Pi = 0) with the oracle: FP64 within 1e-11 relative L1 and
elementwise, the mixed path within the plain step's mixed accuracy; 3-D
blast (PPM, both trace modes, a ragged patch), 2-D turbulence (MC), a batch
of uneven patches; unsupported combinations refused on the host."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import gpu_run, l1rel, maxrel, oracle_run

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


def _check(got, ref, n, ndim, ch, tol):
    G, R = O.interior(got, n, ndim), O.interior(ref, n, ndim)
    for q in range(9):
        if not np.any(R[q]):
            assert not np.any(G[q])
    e1, em = l1rel(G, R, ch), maxrel(G, R, ch)
    assert np.all(e1 <= tol[0]), e1
    assert np.all(em <= tol[1]), em


@pytest.mark.parametrize("recon,trace_mode", [(1, 0), (1, 1), (0, 0)])
def test_blast_3d_ragged(recon, trace_mode):
    n = [23, 17, 11]
    U0 = np.zeros(O.shape(n, 3))
    Ub = W.mhd_blast_3d(24, seed=31, kmax=3)
    O.interior(U0, n, 3)[:] = O.interior(Ub, [24] * 3, 3)[:, :11, :17, :23]
    dx = [1.0 / 23, 1.0 / 17, 1.0 / 11]
    ref, od = oracle_run(U0, n, 3, dx, 5, 0.3, recon=recon, trace_mode=trace_mode, corner=1)
    for prec, tol in ((0, (TOL64, TOL64)), (1, (5e-6, 5e-5))):
        got, gd, st = gpu_run(U0, n, 3, dx, 5, 0.3, precision=prec, recon=recon, trace_mode=trace_mode, corner=1)
        assert st == 0
        if prec == 0:
            for (a, b), (c, d) in zip(gd, od):
                assert abs(a - c) <= 1e-13 * c and abs(b - d) <= 1e-13 * d
        _check(got, ref, n, 3, od[-1][1], tol)


def test_blast_64_10_steps():
    n = [64, 64, 64]
    U0 = W.mhd_blast_3d(64, seed=0)
    dx = [1.0 / 64] * 3
    ref, od = oracle_run(U0, n, 3, dx, 10, 0.3, recon=1, corner=1)
    for prec, tol in ((0, (TOL64, TOL64)), (1, (2e-6, 2e-5))):
        got, _, st = gpu_run(U0, n, 3, dx, 10, 0.3, precision=prec, recon=1, corner=1)
        assert st == 0
        _check(got, ref, n, 3, od[-1][1], tol)


def test_turbulence_2d():
    n = [64, 64, 1]
    U0 = W.mhd_turb_2d(64, seed=2)
    dx = [1.0 / 64] * 2
    ref, od = oracle_run(U0, n, 2, dx, 10, 0.4, recon=0, corner=1)
    for prec, tol in ((0, (TOL64, TOL64)), (1, (5e-6, 5e-5))):
        got, _, st = gpu_run(U0, n, 2, dx, 10, 0.4, precision=prec, recon=0, corner=1)
        assert st == 0
        _check(got, ref, n, 2, od[-1][1], tol)


def test_uneven_batch_and_differs_from_cell_centred():
    """Four patch shapes in one call against the oracle patch by patch; the
    corner-coupled result differs from the cell-centred one."""
    import torch
    from paper_1110_0740_gb300 import ctu
    shapes = [(16, 16, 16), (8, 8, 8), (11, 1, 7), (5, 9, 6)]
    src = W.mhd_blast_3d(40, seed=33, kmax=3)
    arrays, bases, base = [], [], 0
    for i, n in enumerate(shapes):
        A = np.ascontiguousarray(src[:, 2 * i:2 * i + n[2] + 8, i:i + n[1] + 8, 3 * i:3 * i + n[0] + 8])
        arrays.append(A)
        bases.append(base)
        base += A[0].size + 11
    pool = np.zeros((9, base))
    for A, b in zip(arrays, bases):
        pool[:, b:b + A[0].size] = A.reshape(9, -1)
    dev = torch.device("cuda:0")
    U = torch.from_numpy(pool).to(dev)
    dx = [1.0 / 40] * 3
    P = ctu.make_patches([(list(n), dx, b) for n, b in zip(shapes, bases)])
    dtch = torch.tensor([2e-4, 1.5], dtype=torch.float64, device=dev)
    outs = {}
    for corner in (1, 0):
        Uo = torch.zeros_like(U)
        ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64, corner=corner))
        ctx.step(U, Uo, U.shape[1], P, dtch)
        assert ctx.status_sync() == 0
        outs[corner] = Uo.cpu().numpy()
        ctx.close()
    for A, n, b in zip(arrays, shapes, bases):
        R, bad = O.mhd_step(A, list(n), 3, dx, 2e-4, 1.5, recon=1, corner=1)
        assert bad == 0
        G = outs[1][:, b:b + A[0].size].reshape(A.shape)
        _check(G, R, list(n), 3, 1.5, (TOL64, TOL64))
    assert not np.allclose(outs[1], outs[0], rtol=1e-9, atol=0)


def test_unsupported_combinations_refused():
    import ctypes
    from paper_1110_0740_gb300 import ctu
    L = ctu._lib()
    h = ctypes.c_void_p()
    for kw in (dict(kappa=1e-3), dict(recon=ctu.CTU_WENO3), dict(precision=ctu.CTU_MIXED_IFACE64),
               dict(riemann=ctu.CTU_HLLC), dict(trace_mode=ctu.CTU_TRACE_CENTER), dict(shock=(5.0, 0))):
        cfg = ctu.make_config(corner=ctu.CTU_CORNER_MT, **kw)
        assert L.ctu_init(ctypes.byref(cfg), ctypes.byref(h)) == ctu.STATUS.index("CTU_EUNSUPPORTED"), kw
    cfg = ctu.make_config(corner=2)
    assert L.ctu_init(ctypes.byref(cfg), ctypes.byref(h)) == ctu.STATUS.index("CTU_EINVAL")
