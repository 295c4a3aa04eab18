"""ctu_step_noalloc, the allocation-free step for callers that cannot call
cudaMalloc (a host framework whose allocator owns all device memory, a
real-time loop that cannot take cudaMalloc's implicit synchronisation, a
plug-in handed pre-allocated buffers only).  It runs the same kernels on the
same inputs as ctu_step, so it must give ctu_step's result bit for bit, call
after call: on one patch, and on an uneven batch of more than 16 patch
shapes (each shape its own launch group, so the launches are split into
several group tables), for PPM and MC-linear, in 2-D and 3-D, in every
precision, with and without waiting for the status.

Kept in its own file, named to be collected last."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(ndim, shapes, seed):
    """A pool of ghosted patches cut from one periodic state, with ragged gaps."""
    src = W.mhd_blast_3d(48, seed=seed, kmax=3) if ndim == 3 else W.mhd_turb_2d(64, seed=seed)[:, :, :, :]
    arrays, bases, base = [], [], 0
    for i, n in enumerate(shapes):
        shp = O.shape(list(n), ndim)
        if ndim == 3:
            A = src[:, i % 5:i % 5 + shp[1], (2 * i) % 7:(2 * i) % 7 + shp[2], (3 * i) % 9:(3 * i) % 9 + shp[3]]
        else:
            A = src[:, :, (2 * i) % 7:(2 * i) % 7 + shp[2], (3 * i) % 9:(3 * i) % 9 + shp[3]]
        arrays.append(np.ascontiguousarray(A))
        bases.append(base)
        base += A[0].size + 13
    pool = np.zeros((9, base))
    for A, b in zip(arrays, bases):
        pool[:, b:b + A[0].size] = A.reshape(9, -1)
    return pool, bases


SHAPES3 = [(8, 8, 8), (9, 7, 6), (5, 8, 7), (12, 6, 5), (4, 4, 4), (6, 9, 8), (7, 5, 9), (10, 4, 6),
           (3, 5, 7), (8, 6, 4), (11, 3, 5), (6, 6, 10), (5, 10, 3), (7, 7, 7), (9, 4, 8), (4, 9, 5),
           (13, 5, 4), (6, 3, 11)]
SHAPES2 = [(n0, n1, 1) for (n0, n1, _) in SHAPES3]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("recon,ndim,case", [(1, 3, "one"), (1, 3, "batch"), (0, 3, "batch"), (0, 2, "batch"),
                                             (1, 2, "batch")])
def test_noalloc_matches_ctu_step_two_calls_in_a_row(precision, recon, ndim, case):
    import torch
    from paper_1110_0740_gb300 import ctu

    dev = torch.device("cuda:0")
    if case == "one":
        n = [24, 24, 24]
        U0 = W.mhd_blast_3d(24, seed=12, kmax=3)
        O.fill_periodic(U0, n, 3)
        pool, shapes, bases = U0.reshape(9, -1).copy(), [tuple(n)], [0]
    else:
        shapes = SHAPES3 if ndim == 3 else SHAPES2
        pool, bases = _batch(ndim, shapes, seed=13 + precision)
    dx = [1.0 / 48, 1.0 / 40, 1.0 / 44][:ndim] + [1.0] * (3 - ndim)
    cfg = ctu.make_config(ndim=ndim, recon=recon, precision=precision, cfl=0.3)
    ctx = ctu.Ctx(cfg)
    patches = ctu.make_patches([(list(s), dx, b) for s, b in zip(shapes, bases)])
    A = torch.from_numpy(pool).to(dev)   # ctu_step chain
    B = A.clone()                        # ctu_step_noalloc chain
    stride = A.shape[1]
    An, Bn = torch.zeros_like(A), torch.zeros_like(A)
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    for call in range(2):
        ctx.dt(A, stride, patches, dtch)
        ctx.step(A, An, stride, patches, dtch)
        assert ctx.status_sync() == 0
        wait = call == 0
        st = ctu.ctu_step_noalloc(cfg, B, Bn, stride, patches, dtch, wait_status=wait)
        assert st == 0, ctu.ctu_strerror(st)
        torch.cuda.synchronize()
        assert torch.equal(An, Bn), (call, (An - Bn).abs().max().item())
        # the next call starts from the two results, ghosts refreshed alike
        ctx.fill_periodic(An, stride, patches)
        ctx.fill_periodic(Bn, stride, patches)
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
