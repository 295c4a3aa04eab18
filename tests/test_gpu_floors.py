"""Optional density and pressure floors of the updated state on the GPU
against the oracle's or_mhd_floor: bit-exact on a zero-dt step (the update
then returns U^n unchanged and only the floors act) over a batch of ragged
patches, and after real steps in float64 (relative L1 1e-11, the same cells
floored) and in the mixed path (floors hold exactly; the floored counts
differ only by cells whose unfloored value lies within the mixed error of a
floor)."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import l1rel

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def _pressure(U):
    m2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
    b2 = U[5] ** 2 + U[6] ** 2 + U[7] ** 2
    return (G53 - 1.0) * (U[4] - 0.5 * m2 / U[0] - 0.5 * b2)


def _sub(U, n):
    """A ghosted block of interior shape n cut from a larger ghosted patch."""
    return np.ascontiguousarray(U[:, :n[2] + 8, :n[1] + 8, :n[0] + 8])


def test_zero_dt_floor_is_bit_exact_over_a_batch():
    import torch
    from paper_1110_0740_gb300 import ctu
    big = W.mhd_blast_3d(32, seed=3)
    shapes = [[21, 13, 11], [8, 8, 8], [32, 32, 32], [5, 17, 9]]
    blocks = [_sub(big, n) if n != [32, 32, 32] else big.copy() for n in shapes]
    I = np.concatenate([O.interior(b, n, 3).reshape(9, -1) for b, n in zip(blocks, shapes)], axis=1)
    rf = float(np.quantile(I[0], 0.15))
    pf = float(np.quantile(_pressure(I), 0.3))
    bases, off = [], 0
    for b in blocks:
        bases.append(off)
        off += b[0].size
    pool = np.zeros((9, off))
    for b, base in zip(blocks, bases):
        pool[:, base:base + b[0].size] = b.reshape(9, -1)
    dev = torch.device("cuda:0")
    for prec in (ctu.CTU_FP64, ctu.CTU_MIXED):
        U = torch.from_numpy(pool).to(dev)
        Uo = U.clone()
        patches = ctu.make_patches([(n, [1.0 / 32] * 3, base) for n, base in zip(shapes, bases)])
        ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3,
                                      p_floor=pf, rho_floor=rf))
        dtch = torch.tensor([0.0, 1.0], dtype=torch.float64, device=dev)
        ctx.step(U, Uo, U.shape[1], patches, dtch)
        assert ctx.status_sync() == 0
        got = Uo.cpu().numpy()
        total = 0
        for b, n, base in zip(blocks, shapes, bases):
            ref = b.copy()
            total += O.mhd_floor(ref, n, 3, pf, rf)
            G = got[:, base:base + b[0].size].reshape(b.shape)
            assert np.array_equal(O.interior(G, n, 3), O.interior(ref, n, 3)), (prec, n)
        assert total > 0
        assert ctx.floor_count() == total
        assert ctx.floor_count() == 0  # the count resets
        ctx.close()


def _run_gpu(U0, n, steps, prec, pf, rf):
    import torch
    from paper_1110_0740_gb300 import ctu
    dev = torch.device("cuda:0")
    U = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
    Ub = torch.zeros_like(U)
    patches = ctu.make_patches([(n, [1.0 / n[0]] * 3, 0)])
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3,
                                  p_floor=pf, rho_floor=rf))
    d0 = torch.zeros(2, dtype=torch.float64, device=dev)
    d1 = torch.zeros_like(d0)
    ctx.fill_periodic(U, U.shape[1], patches)
    ctx.dt(U, U.shape[1], patches, d0)
    dts, counts = [], []
    for _ in range(steps):
        dts.append(tuple(d0.cpu().tolist()))
        ctx.step_next_dt(U, Ub, U.shape[1], patches, d0, d1)
        counts.append(ctx.floor_count())
        ctx.fill_periodic(Ub, U.shape[1], patches)
        U, Ub = Ub, U
        d0, d1 = d1, d0
    assert ctx.status_sync() == 0
    out = U.cpu().numpy().reshape(U0.shape)
    nxt = tuple(d0.cpu().tolist())
    ctx.close()
    return out, dts, counts, nxt


def _run_oracle(U0, n, steps, pf, rf):
    U = U0.copy()
    dx = [1.0 / n[0]] * 3
    dts, counts, near = [], [], []
    for _ in range(steps):
        U = O.fill_periodic(U, n, 3)
        dt, ch = O.dt_ch(O.mhd_max_speed(U, n, 3, dx), dx, 3, 0.3)
        dts.append((dt, ch))
        U, bad = O.mhd_step(U, n, 3, dx, dt, ch, recon=1)
        assert bad == 0
        near.append(O.interior(U, n, 3).copy())  # before the floors act on U
        counts.append(O.mhd_floor(U, n, 3, pf, rf))
    U = O.fill_periodic(U, n, 3)
    nxt = O.dt_ch(O.mhd_max_speed(U, n, 3, dx), dx, 3, 0.3)
    return U, dts, counts, near, nxt


def _floors_for(U0, n):
    I = O.interior(U0, n, 3)
    return float(np.quantile(_pressure(I), 0.2)), float(np.quantile(I[0], 0.1))


def test_floors_after_real_steps_fp64():
    n = [32, 32, 32]
    U0 = W.mhd_blast_3d(32, seed=4)
    pf, rf = _floors_for(U0, n)
    ref, odts, ocnt, unfloored, onext = _run_oracle(U0, n, 3, pf, rf)
    for I in unfloored:  # no cell within 1e-9 of a floor: both sides decide alike
        assert np.min(np.abs(I[0] / rf - 1.0)) > 1e-9
        assert np.min(np.abs(_pressure(I) / pf - 1.0)) > 1e-9
    got, gdts, gcnt, gnext = _run_gpu(U0, n, 3, 0, pf, rf)
    assert gcnt == ocnt and min(ocnt) > 0
    for (a, b), (c, d) in zip(gdts + [gnext], odts + [onext]):
        assert abs(a - c) <= 1e-12 * c and abs(b - d) <= 1e-12 * d
    e = l1rel(O.interior(got, n, 3), O.interior(ref, n, 3), odts[-1][1])
    assert np.all(e <= 1e-11), e


def test_floors_after_real_steps_mixed():
    n = [32, 32, 32]
    U0 = W.mhd_blast_3d(32, seed=4)
    pf, rf = _floors_for(U0, n)
    ref, odts, ocnt, unfloored, _ = _run_oracle(U0, n, 3, pf, rf)
    got, _, gcnt, _ = _run_gpu(U0, n, 3, 1, pf, rf)
    G = O.interior(got, n, 3)
    assert np.all(G[0] >= rf)
    assert np.all(_pressure(G) >= pf * (1.0 - 1e-12))
    for I, a, b in zip(unfloored, gcnt, ocnt):
        near = np.sum(np.abs(I[0] / rf - 1.0) < 1e-4) + np.sum(np.abs(_pressure(I) / pf - 1.0) < 1e-4)
        assert abs(a - b) <= near, (a, b, near)
    e = l1rel(G, O.interior(ref, n, 3), odts[-1][1])
    assert np.all(e <= 2e-5), e
