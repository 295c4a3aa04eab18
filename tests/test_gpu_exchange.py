"""Same-level ghost exchange on the GPU (ctu_copy / ctu_pack / ctu_unpack)
against the oracle's copy, pack and unpack: bit-exact on periodic
decompositions in 2-D and 3-D and on the whole finest level of the AMR
hierarchy; invalid boxes are refused.  Then the exchange in use: a
periodic 64^3 blast cut into 8 unequal patches, advanced 3 steps with the
exchange refreshing the ghosts, equals the single periodic patch advanced
the same way, bit for bit (the step's arithmetic per cell does not depend
on the patch a cell belongs to)."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import exchange as X
from paper_1110_0740_gb300 import workloads as W
from tests.test_exchange import _block, _pool, _setup, _wrapped

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch.device("cuda:0")


@pytest.mark.parametrize("ndim", [2, 3])
def test_copy_and_pack_bit_exact_on_periodic_decomposition(ndim):
    import torch
    from paper_1110_0740_gb300 import ctu
    domain, parts, big = _setup(ndim, 20 + ndim)
    pool, specs = _pool(big, parts, ndim)
    boxes = X.plan(specs, domain, [True] * 3, ndim)
    cb = ctu.make_copy_boxes(boxes)
    ctx = ctu.Ctx(ctu.make_config(ndim=ndim))
    U = torch.from_numpy(pool).to(_dev())
    ctx.copy(U, U.shape[1], U, U.shape[1], cb)
    ref = pool.copy()
    O.copy_boxes(ref, ref, boxes, ndim)
    got = U.cpu().numpy()
    assert np.array_equal(got, ref)
    for lo, n, base in specs:
        assert np.array_equal(_block(got, n, base, ndim), _wrapped(big, lo, n, ndim))
    # pack from the filled pool, unpack into the unfilled one
    V = torch.from_numpy(pool).to(_dev())
    buf = torch.full((9 * sum(X.cells(b) for b in boxes),), -1.0, dtype=torch.float64, device=_dev())
    ctx.pack(buf, U, U.shape[1], cb)
    assert np.array_equal(buf.cpu().numpy(), O.pack_boxes(ref, boxes, ndim))
    ctx.unpack(V, V.shape[1], buf, cb)
    assert np.array_equal(V.cpu().numpy(), ref)
    assert ctx.status_sync() == 0
    ctx.close()


def test_copy_amr_finest_level():
    import torch
    from paper_1110_0740_gb300 import ctu
    H = W.amr_hierarchy(seed=0)
    L2 = H["levels"][2]
    specs = [((o[2], o[1], o[0]), (s, s, s), p[2]) for (o, s), p in zip(L2["origins"], L2["patches"])]
    boxes = X.plan(specs, [512] * 3, [False] * 3, 3)
    assert len(boxes) > 100
    pool = L2["pool"].copy()
    ref = pool.copy()
    O.copy_boxes(ref, ref, boxes, 3)
    ctx = ctu.Ctx(ctu.make_config(ndim=3))
    U = torch.from_numpy(pool).to(_dev())
    ctx.copy(U, U.shape[1], U, U.shape[1], ctu.make_copy_boxes(boxes))
    assert np.array_equal(U.cpu().numpy(), ref)
    ctx.close()


def test_bad_boxes_are_refused():
    import torch
    from paper_1110_0740_gb300 import ctu
    domain, parts, big = _setup(3, 1)
    pool, specs = _pool(big, parts, 3)
    good = X.plan(specs, domain, [True] * 3, 3)[0]
    U = torch.from_numpy(pool).to(_dev())
    ctx = ctu.Ctx(ctu.make_config(ndim=3))
    bads = []
    for key, d, v in (("hi", 0, good["dn"][0] + 5), ("lo", 1, -5), ("shift", 2, 100)):
        b = dict(good)
        b[key] = list(b[key])
        b[key][d] = v
        bads.append(b)
    b = dict(good)
    b["dbase"] = pool.shape[1]
    bads.append(b)
    for b in bads:
        with pytest.raises(ctu.CtuError) as e:
            ctx.copy(U, U.shape[1], U, U.shape[1], ctu.make_copy_boxes([b]))
        assert e.value.code == 1
    ctx.close()


def test_decomposed_steps_equal_the_single_patch():
    import torch
    from paper_1110_0740_gb300 import ctu
    n = 64
    U0 = W.mhd_blast_3d(n, seed=2)
    big = O.interior(U0, [n] * 3, 3)
    cuts = [[0, 24, 64], [0, 40, 64], [0, 16, 64]]
    parts = [([x0, y0, z0], [x1 - x0, y1 - y0, z1 - z0])
             for z0, z1 in zip(cuts[2][:-1], cuts[2][1:]) for y0, y1 in zip(cuts[1][:-1], cuts[1][1:])
             for x0, x1 in zip(cuts[0][:-1], cuts[0][1:])]
    pool, specs = _pool(big, parts, 3, fill=0.0)
    boxes = ctu.make_copy_boxes(X.plan(specs, [n] * 3, [True] * 3, 3))
    dx = [1.0 / n] * 3
    dev = _dev()
    for prec in (ctu.CTU_FP64, ctu.CTU_MIXED):
        ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3))
        # the decomposed domain
        A = torch.from_numpy(pool).to(dev)
        B = torch.zeros_like(A)
        P = ctu.make_patches([(nn, dx, base) for lo, nn, base in specs])
        d = torch.zeros(2, dtype=torch.float64, device=dev)
        # the single patch
        S = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
        T = torch.zeros_like(S)
        P1 = ctu.make_patches([([n] * 3, dx, 0)])
        d1 = torch.zeros_like(d)
        for _ in range(3):
            ctx.copy(A, A.shape[1], A, A.shape[1], boxes)
            ctx.dt(A, A.shape[1], P, d)
            ctx.step(A, B, A.shape[1], P, d)
            A, B = B, A
            ctx.fill_periodic(S, S.shape[1], P1)
            ctx.dt(S, S.shape[1], P1, d1)
            ctx.step(S, T, S.shape[1], P1, d1)
            S, T = T, S
            assert torch.equal(d, d1)
        assert ctx.status_sync() == 0
        got, one = A.cpu().numpy(), O.interior(S.cpu().numpy().reshape(U0.shape), [n] * 3, 3)
        for lo, nn, base in specs:
            blk = O.interior(_block(got, nn, base, 3), nn, 3)
            want = one[:, lo[2]:lo[2] + nn[2], lo[1]:lo[1] + nn[1], lo[0]:lo[0] + nn[0]]
            assert np.array_equal(blk, want), (prec, lo, nn)
        ctx.close()
