"""The HLLC solver (Li 2005) on the GPU against the oracle: PPM on the 3-D
blast and MC-linear on the 2-D turbulence state, float64 (relative L1 1e-11)
and mixed (2e-5 / 1e-4), with the upwind trace mode once; unsupported
combinations refused."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import gpu_run, l1rel, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("trace_mode", [0, 1])
def test_hllc_3d_blast_ppm(trace_mode):
    n = [32, 32, 32]
    U0 = W.mhd_blast_3d(32, seed=11)
    dx = [1.0 / 32] * 3
    ref, od = oracle_run(U0, n, 3, dx, 4, 0.3, recon=1, trace_mode=trace_mode, riemann=2)
    R = O.interior(ref, n, 3)
    for prec, tol in ((0, 1e-11), (1, 2e-5)):
        got, gd, st = gpu_run(U0, n, 3, dx, 4, 0.3, precision=prec, recon=1, trace_mode=trace_mode, riemann=2)
        assert st == 0
        e = l1rel(O.interior(got, n, 3), R, od[-1][1])
        assert np.all(e <= tol), (prec, e)


def test_hllc_2d_turbulence_mc():
    n = [64, 64, 1]
    U0 = W.mhd_turb_2d(64, seed=12)
    dx = [1.0 / 64] * 2
    ref, od = oracle_run(U0, n, 2, dx, 10, 0.4, recon=0, riemann=2)
    R = O.interior(ref, n, 2)
    for prec, tol in ((0, 1e-11), (1, 1e-4)):
        got, _, st = gpu_run(U0, n, 2, dx, 10, 0.4, precision=prec, recon=0, riemann=2)
        assert st == 0
        G = O.interior(got, n, 2)
        assert not np.any(G[3]) and not np.any(G[7])
        e = l1rel(G, R, od[-1][1])
        assert np.all(e <= tol), (prec, e)


def test_hllc_unsupported():
    from paper_1110_0740_gb300 import ctu
    for kw in (dict(recon=5), dict(trace_mode=2), dict(precision=2), dict(shock=(5.0, 0))):
        with pytest.raises(ctu.CtuError) as e:
            ctu.Ctx(ctu.make_config(riemann=ctu.CTU_HLLC, **kw))
        assert e.value.code == 4
