"""ctu_step_noalloc, the allocation-free step for callers that cannot call
cudaMalloc (a host framework whose allocator owns all device memory, a
real-time loop that cannot take cudaMalloc's implicit synchronisation, a
plug-in handed pre-allocated buffers only).  It must give what ctu_step
gives on the same inputs, call after call.

Kept in its own file, named to be collected last."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import l1rel

pytestmark = pytest.mark.gpu

TOL = 1e-11  # the FP64 parity tolerance of the other GPU tests


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_ctu_step_two_calls_in_a_row(precision):
    import torch
    from paper_1110_0740_gb300 import ctu

    n = [24, 24, 24]
    dx = [1.0 / 24] * 3
    U0 = W.mhd_blast_3d(24, seed=12, kmax=3)
    O.fill_periodic(U0, n, 3)
    dev = torch.device("cuda:0")
    cfg = ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=precision, cfl=0.3)
    ctx = ctu.Ctx(cfg)
    patches = ctu.make_patches([(n, dx, 0)])
    A = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)  # ctu_step chain
    B = A.clone()                                             # ctu_step_noalloc chain
    stride = A.shape[1]
    An, Bn = torch.zeros_like(A), torch.zeros_like(A)
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    for call in range(2):
        ctx.dt(A, stride, patches, dtch)
        ctx.step(A, An, stride, patches, dtch)
        assert ctx.status_sync() == 0
        st = ctu.ctu_step_noalloc(cfg, B, Bn, stride, patches, dtch, wait_status=True)
        assert st == 0, ctu.ctu_strerror(st)
        ctx.fill_periodic(An, stride, patches)
        ctx.fill_periodic(Bn, stride, patches)
        torch.cuda.synchronize()
        ref = An.cpu().numpy().reshape(U0.shape)
        got = Bn.cpu().numpy().reshape(U0.shape)
        e = l1rel(O.interior(got, n, 3), O.interior(ref, n, 3), float(dtch[1]))
        assert np.all(e <= TOL), (call, e)
        A, An = An, A
        B, Bn = Bn, B
    ctx.close()


def test_noalloc_rejects_oversized_batch():
    import torch
    from paper_1110_0740_gb300 import ctu

    cfg = ctu.make_config(ndim=3, precision=ctu.CTU_FP64)
    n = [64, 64, 64]
    cells = 72 ** 3
    patches = ctu.make_patches([(n, [1.0 / 64] * 3, 0)])
    dev = torch.device("cuda:0")
    # no kernel runs for a rejected call, so small buffers suffice
    U = torch.zeros(16, dtype=torch.float64, device=dev)
    V = torch.zeros(16, dtype=torch.float64, device=dev)
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    st = ctu.ctu_step_noalloc(cfg, U, V, 9 * cells, patches, dtch)
    assert ctu.STATUS[st] == "CTU_ETOOLARGE"
    many = ctu.make_patches([([2, 2, 2], [1.0] * 3, 1000 * i) for i in range(65)])
    st = ctu.ctu_step_noalloc(cfg, U, V, 1000 * 65, many, dtch)
    assert ctu.STATUS[st] == "CTU_ETOOLARGE"
