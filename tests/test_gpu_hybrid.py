"""The hybrid integration (shock flags, HLL at flagged faces, MinMod near
shocks) on the GPU against the oracle: the 3-D blast (the sphere's jump is
flagged) in float64 (relative L1 1e-11 -- a single differing flag would
change the result by orders of magnitude more) and in the mixed path
(2e-5); the strongly magnetised 2-D blast that breaks the plain step, for
10 steps under the hybrid (float64 1e-11, mixed 1e-4), with the plain GPU
step reporting the non-positive state like the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import l1rel
from tests.test_oracle_hybrid import _magnetised_blast

pytestmark = pytest.mark.gpu


def _gpu_run(U0, n, ndim, steps, cfl, prec, recon, shock):
    import torch
    from paper_1110_0740_gb300 import ctu
    dev = torch.device("cuda:0")
    U = torch.from_numpy(np.ascontiguousarray(U0).reshape(9, -1)).to(dev)
    Ub = torch.zeros_like(U)
    ctx = ctu.Ctx(ctu.make_config(ndim=ndim, recon=recon, precision=prec, cfl=cfl, shock=shock))
    dx3 = [1.0 / n[0]] * ndim + [1.0] * (3 - ndim)
    patches = ctu.make_patches([(n, dx3, 0)])
    d = torch.zeros(2, dtype=torch.float64, device=dev)
    for _ in range(steps):
        ctx.fill_periodic(U, U.shape[1], patches)
        ctx.dt(U, U.shape[1], patches, d)
        ctx.step(U, Ub, U.shape[1], patches, d)
        U, Ub = Ub, U
    ctx.fill_periodic(U, U.shape[1], patches)
    st = ctx.status_sync()
    out = U.cpu().numpy().reshape(U0.shape)
    ctx.close()
    return out, st


@pytest.mark.parametrize("recon", [1, 0])
def test_hybrid_3d_blast(recon):
    n = [32, 32, 32]
    U0 = W.mhd_blast_3d(32, seed=5)
    O.fill_periodic(U0, n, 3)
    assert np.any(O.mhd_shock_flags(U0, n, 3, [1.0 / 32] * 3, 5.0, 0) & 1)
    ref, _, od = O.mhd_run(U0, n, 3, [1.0 / 32] * 3, 4, 0.3, recon=recon, shock=(5.0, 0))
    R = O.interior(ref, n, 3)
    for prec, tol in ((0, 1e-11), (1, 2e-5)):
        got, st = _gpu_run(U0, n, 3, 4, 0.3, prec, recon, (5.0, 0))
        assert st == 0
        e = l1rel(O.interior(got, n, 3), R, od[-1][1])
        assert np.all(e <= tol), (recon, prec, e)


def test_hybrid_magnetised_blast():
    U0, n = _magnetised_blast()
    dx = [1.0 / 64] * 2
    ref, _, od = O.mhd_run(U0, n, 2, dx, 10, 0.4, recon=1, shock=(5.0, 0))
    R = O.interior(ref, n, 2)
    for prec, tol in ((0, 1e-11), (1, 1e-4)):
        got, st = _gpu_run(U0, n, 2, 10, 0.4, prec, 1, (5.0, 0))
        assert st == 0
        e = l1rel(O.interior(got, n, 2), R, od[-1][1])
        assert np.all(e <= tol), (prec, e)
    # without the hybrid the GPU meets the non-positive state as the oracle does
    _, st = _gpu_run(U0, n, 2, 10, 0.4, 0, 1, None)
    assert st == 5  # CTU_ENEGATIVE


def test_hybrid_magnetic_pressure_kind():
    n = [24, 24, 24]
    U0 = W.mhd_blast_3d(24, seed=6)
    O.fill_periodic(U0, n, 3)
    ref, _, od = O.mhd_run(U0, n, 3, [1.0 / 24] * 3, 3, 0.3, recon=1, shock=(5.0, 1))
    got, st = _gpu_run(U0, n, 3, 3, 0.3, 0, 1, (5.0, 1))
    assert st == 0
    e = l1rel(O.interior(got, n, 3), O.interior(ref, n, 3), od[-1][1])
    assert np.all(e <= 1e-11), e


def test_hybrid_unsupported_combinations():
    from paper_1110_0740_gb300 import ctu
    for kw in (dict(recon=5), dict(trace_mode=2), dict(precision=2)):
        with pytest.raises(ctu.CtuError) as e:
            ctu.Ctx(ctu.make_config(shock=(5.0, 0), **kw))
        assert e.value.code == 4
    with pytest.raises(ctu.CtuError) as e:
        ctu.Ctx(ctu.make_config(shock=(-1.0, 0)))
    assert e.value.code == 1
