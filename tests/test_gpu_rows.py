"""Several rows per thread in the x-tiled kernels (the x sweep and the
first-order x stage) on a patch whose rows do not fill the last block: the
count a launch takes depends on the whole batch (enough blocks for several
waves), so the same patch runs at different counts alone and beside a large
neighbour; the result must not depend on it (bitwise), and must match the
oracle (FP64, relative L1 and elementwise within 1e-11)."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import l1rel, maxrel

pytestmark = pytest.mark.gpu

A_N = (200, 131, 67)  # 131 rows: not a multiple of any tile's rows
B_N = (256, 256, 64)


def _state(n, seed):
    """A seeded blast state on a non-cubic ghosted patch: a 64^3 blast's
    ghosted state repeated periodically (ghost layers included)."""
    src = O.interior(W.mhd_blast_3d(64, seed=seed, kmax=3), [64] * 3, 3)
    sh = O.shape(list(n), 3)
    iz = (np.arange(sh[1]) - 4) % 64
    iy = (np.arange(sh[2]) - 4) % 64
    ix = (np.arange(sh[3]) - 4) % 64
    return np.ascontiguousarray(src[:, iz][:, :, iy][:, :, :, ix])


def _step(ctu, torch, pool, shapes, bases, precision):
    dev = torch.device("cuda:0")
    U = torch.from_numpy(pool).to(dev)
    Uo = torch.zeros_like(U)
    stride = U.shape[1]
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=precision, cfl=0.3))
    patches = ctu.make_patches([(n, [1.0 / n[0]] * 3, b) for n, b in zip(shapes, bases)])
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    # the first patch's dt and c_h for both runs, so that they advance alike
    one = ctu.make_patches([(shapes[0], [1.0 / shapes[0][0]] * 3, bases[0])])
    ctx.dt(U, stride, one, dtch)
    ctx.step(U, Uo, stride, patches, dtch)
    assert ctx.status_sync() == 0
    out, d = Uo.cpu().numpy(), dtch.cpu().tolist()
    ctx.close()
    return out, d


@pytest.mark.parametrize("precision", [0, 1])
def test_rows_per_thread_do_not_change_the_step(precision):
    import torch
    from paper_1110_0740_gb300 import ctu
    A = _state(A_N, 5)
    B = _state(B_N, 6)
    sa = A[0].size
    alone, dta = _step(ctu, torch, A.reshape(9, -1).copy(), [A_N], [0], precision)
    pool = np.concatenate([A.reshape(9, -1), B.reshape(9, -1)], axis=1)
    both, dtb = _step(ctu, torch, pool, [A_N, B_N], [0, sa], precision)
    assert dta == dtb
    assert np.array_equal(alone[:, :sa], both[:, :sa])
    if precision == 0:  # against the oracle, one step with the same dt and c_h
        ref, bad = O.mhd_step(A, list(A_N), 3, [1.0 / A_N[0]] * 3, dta[0], dta[1], recon=1)
        assert bad == 0
        G = O.interior(alone[:, :sa].reshape(A.shape), list(A_N), 3)
        Rf = O.interior(ref, list(A_N), 3)
        assert np.all(l1rel(G, Rf, dta[1]) <= 1e-11)
        assert np.all(maxrel(G, Rf, dta[1]) <= 1e-11)
