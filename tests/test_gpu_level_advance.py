"""The batched AMR level advance on the GPU (paper_1110_0740_gb300.amr_advance,
Section 4), through the library's kernels:

- a coarse step depends on its input alone: three coarse steps from one input
  agree bit for bit (mixed precision, the seeded 149-patch hierarchy), although
  each leaves its second pools in a different state for the next;
- the composite solution is conserved: on a properly nested 3-level hierarchy,
  first restricted so that every covered coarse cell is the mean of its
  children, one float64 coarse step keeps the level-0 totals of mass,
  momentum, energy and magnetic field to round-off (Eq. fluxcorr, Eq.
  addreflux, Eq. avgdown), also with the parabolic terms, whose fluxes the
  registers carry.  Its level-2 patch against its parent's boundary is
  refluxed into the level-1 patch across that boundary;
- the float64 coarse step matches the oracle's: the same plan and launch
  sequence carried out by the oracle's operators, with the same dt_0 and c_h,
  every interior cell of every level within 1e-11 of its variable's largest
  value."""
import numpy as np
import pytest

from paper_1110_0740_gb300 import workloads as W
from tests.test_amr_plan import _oracle_coarse_step, nested_levels

pytestmark = pytest.mark.gpu


def _advance(levels, base, precision, **par):
    import torch
    from paper_1110_0740_gb300 import shard
    from paper_1110_0740_gb300.amr_advance import LevelAdvance
    adv = LevelAdvance(levels, base, precision=precision, cfl=0.3, device=torch.device("cuda:0"), **par)
    dx0 = levels[0]["patches"][0][1][0]
    adv.set_dt(*shard.agree_dt((adv.local_dt(), 0.0), 0.3, dx0))
    return adv


def _totals(levels, pool):
    """Sum over level 0's interior cells of U_q times the cell volume, and of
    |U_q| times the volume (the scale)."""
    tot, mag = np.zeros(9), np.zeros(9)
    for n, dx, base in (p[:3] for p in levels[0]["patches"]):
        N = [v + 8 for v in n]
        U = pool[:, base:base + N[0] * N[1] * N[2]].reshape(9, N[2], N[1], N[0])[:, 4:-4, 4:-4, 4:-4]
        vol = dx[0] * dx[1] * dx[2]
        tot += U.sum(axis=(1, 2, 3)) * vol
        mag += np.abs(U).sum(axis=(1, 2, 3)) * vol
    return tot, mag


def test_coarse_steps_from_one_input_agree_bit_for_bit():
    import torch
    from paper_1110_0740_gb300 import ctu
    levels = W.amr_hierarchy(seed=3, base=64, target=80)["levels"]
    adv = _advance(levels, 64, ctu.CTU_MIXED)
    init = [a.clone() for a in adv.A]
    res = []
    for _ in range(3):
        for a, a0 in zip(adv.A, init):
            a.copy_(a0)
        adv.coarse_step(None)
        assert all(c.status_sync() == 0 for c in adv.ctxs)
        res.append([o.cpu() for o in adv.outputs()])
    adv.close()
    for r in res[1:]:
        for x, y in zip(res[0], r):
            assert torch.equal(x, y)


@pytest.mark.parametrize("par", [{}, dict(kappa=0.002, nu=0.001, eta=0.001)])
def test_the_composite_solution_is_conserved(par):
    import torch
    from paper_1110_0740_gb300 import ctu
    levels = nested_levels()
    adv = _advance(levels, 32, ctu.CTU_FP64, **par)
    assert adv.plan.unmatched_faces == 0
    for lev in (2, 1):  # every covered coarse cell the mean of its children
        adv.ctxs[lev - 1].restrict(adv.A[lev - 1], adv.A[lev - 1].shape[1], adv.A[lev], adv.A[lev].shape[1],
                                   adv.ops[lev][1])
    torch.cuda.synchronize()
    tot0, mag = _totals(levels, adv.A[0].cpu().numpy())
    adv.coarse_step(None)
    assert all(c.status_sync() == 0 for c in adv.ctxs)
    tot1, _ = _totals(levels, adv.outputs()[0].cpu().numpy())
    adv.close()
    # psi (q = 8) is damped, not conserved
    assert np.all(np.abs(tot1 - tot0)[:8] <= 1e-13 * mag[:8]), (tot1 - tot0) / mag


@pytest.mark.parametrize("par", [{}, dict(kappa=0.002, nu=0.001, eta=0.001)])
def test_the_coarse_step_matches_the_oracle(par):
    import torch
    from paper_1110_0740_gb300 import ctu
    from paper_1110_0740_gb300.amr_advance import LevelAdvance
    levels = nested_levels()
    ref = {}
    _oracle_coarse_step(levels, 32, _plan(levels), par, ref)
    adv = LevelAdvance(levels, 32, precision=ctu.CTU_FP64, cfl=0.3, device=torch.device("cuda:0"), **par)
    adv.set_dt(ref["dt0"], ref["ch"])
    for lev in (2, 1):
        adv.ctxs[lev - 1].restrict(adv.A[lev - 1], adv.A[lev - 1].shape[1], adv.A[lev], adv.A[lev].shape[1],
                                   adv.ops[lev][1])
    adv.coarse_step(None)
    assert all(c.status_sync() == 0 for c in adv.ctxs)
    got = [o.cpu().numpy() for o in adv.outputs()]
    adv.close()
    for lev, lv in enumerate(levels):
        for n, dx, base in (p[:3] for p in lv["patches"]):
            N = [v + 8 for v in n]
            sl = slice(base, base + N[0] * N[1] * N[2])
            G = got[lev][:, sl].reshape(9, N[2], N[1], N[0])[:, 4:-4, 4:-4, 4:-4]
            R = ref["outputs"][lev][:, sl].reshape(9, N[2], N[1], N[0])[:, 4:-4, 4:-4, 4:-4]
            scale = np.abs(R).reshape(9, -1).max(axis=1)[:, None, None, None] + 1e-300
            assert np.all(np.abs(G - R) <= 1e-11 * scale), (lev, base, float((np.abs(G - R) / scale).max()))


def _plan(levels):
    from paper_1110_0740_gb300.amr_advance import LevelPlan
    return LevelPlan(levels, 32)
