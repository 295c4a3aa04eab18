"""The other reconstructions of Section 3.2 on the GPU against the oracle:
MinMod, harmonic and Van Albada linear slopes and improved WENO3, in float64
(relative L1 1e-11 per variable) and in the mixed path (2e-5 on the blast,
1e-4 on the 2-D turbulence state), on a ragged 3-D patch and a 2-D state."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import gpu_run, l1rel, oracle_run

pytestmark = pytest.mark.gpu
RECONS = [2, 3, 4, 5]


@pytest.mark.parametrize("recon", RECONS)
def test_recon_3d_blast(recon):
    n = [32, 32, 32]
    U0 = W.mhd_blast_3d(32, seed=recon)
    dx = [1.0 / 32] * 3
    ref, od = oracle_run(U0, n, 3, dx, 4, 0.3, recon=recon)
    R = O.interior(ref, n, 3)
    for prec, tol in ((0, 1e-11), (1, 2e-5)):
        got, gd, st = gpu_run(U0, n, 3, dx, 4, 0.3, precision=prec, recon=recon)
        assert st == 0
        if prec == 0:
            for (a, b), (c, d) in zip(gd, od):
                assert abs(a - c) <= 1e-13 * c
        e = l1rel(O.interior(got, n, 3), R, od[-1][1])
        assert np.all(e <= tol), (recon, prec, e)


@pytest.mark.parametrize("recon", RECONS)
def test_recon_2d_turbulence(recon):
    n = [64, 64, 1]
    big = W.mhd_turb_2d(64, seed=recon)
    dx = [1.0 / 64] * 2
    ref, od = oracle_run(big, n, 2, dx, 10, 0.4, recon=recon)
    R = O.interior(ref, n, 2)
    for prec, tol in ((0, 1e-11), (1, 1e-4)):
        got, _, st = gpu_run(big, n, 2, dx, 10, 0.4, precision=prec, recon=recon)
        assert st == 0
        G = O.interior(got, n, 2)
        e = l1rel(G, R, od[-1][1])
        for q in (3, 7):  # v_z, B_z stay exactly zero in 2-D
            assert not np.any(G[q]) and not np.any(R[q])
        assert np.all(e <= tol), (recon, prec, e)


def test_unsupported_combinations():
    from paper_1110_0740_gb300 import ctu
    for recon in RECONS:
        with pytest.raises(ctu.CtuError) as e:
            ctu.Ctx(ctu.make_config(recon=recon, precision=ctu.CTU_MIXED_IFACE64))
        assert e.value.code == 4
    with pytest.raises(ctu.CtuError) as e:
        ctu.Ctx(ctu.make_config(recon=6))
    assert e.value.code == 1


@pytest.mark.parametrize("recon,mode", [(1, 2), (1, 3), (0, 2), (0, 3), (5, 3), (3, 2), (5, 1)])
def test_reference_states_3d(recon, mode):
    """The reference states of the tracing (cell centre, Colella-Woodward) with
    PPM and MC-linear, and combined with the other reconstructions."""
    n = [24, 20, 16]
    U0 = W.mhd_blast_3d(24, seed=10 + mode)[:, :24, :28, :32].copy()
    dx = [1.0 / 24] * 3
    ref, od = oracle_run(U0, n, 3, dx, 4, 0.3, recon=recon, trace_mode=mode)
    R = O.interior(ref, n, 3)
    for prec, tol in ((0, 1e-11), (1, 2e-5)):
        got, _, st = gpu_run(U0, n, 3, dx, 4, 0.3, precision=prec, recon=recon, trace_mode=mode)
        assert st == 0
        e = l1rel(O.interior(got, n, 3), R, od[-1][1])
        assert np.all(e <= tol), (recon, mode, prec, e)


def test_reference_state_unsupported_combinations():
    from paper_1110_0740_gb300 import ctu
    for mode in (2, 3):
        with pytest.raises(ctu.CtuError) as e:
            ctu.Ctx(ctu.make_config(trace_mode=mode, precision=ctu.CTU_MIXED_IFACE64))
        assert e.value.code == 4
    with pytest.raises(ctu.CtuError) as e:
        ctu.Ctx(ctu.make_config(trace_mode=4))
    assert e.value.code == 1
