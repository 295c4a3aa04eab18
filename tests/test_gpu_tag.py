"""Refinement tagging, Eq. (RefCrit), on the GPU against the oracle's
or_tag: chi bit-exact (the float64 path is the definition in its order with
IEEE division and square root), tags and per-patch counts bit-exact also on
the float32-filtered path -- at the paper's threshold and at the median chi,
where half of the cells sit near the threshold -- for every sigma kind, over
batches of ragged patches in 1, 2 and 3 dimensions (both launch shapes: the
tiled march and one cell per thread), the full 256^3 blast and the whole
finest level of the AMR hierarchy."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS = 0.01


def _pool(blocks):
    bases, off = [], 0
    for b in blocks:
        bases.append(off)
        off += b[0].size
    pool = np.zeros((9, off))
    for b, base in zip(blocks, bases):
        pool[:, base:base + b[0].size] = b.reshape(9, -1)
    return pool, bases


def _gpu_tag(pool, specs, ndim, kind, eps, chi_r, want_chi):
    import torch
    from paper_1110_0740_gb300 import ctu
    dev = torch.device("cuda:0")
    U = torch.from_numpy(pool).to(dev)
    stride = U.shape[1]
    tags = torch.full((stride,), 7, dtype=torch.uint8, device=dev)
    cnt = torch.full((len(specs),), -1, dtype=torch.int64, device=dev)
    chi = torch.zeros(stride, dtype=torch.float64, device=dev) if want_chi else None
    ctx = ctu.Ctx(ctu.make_config(ndim=ndim))
    patches = ctu.make_patches(specs)
    ctx.tag(U, stride, patches, kind, eps, chi_r, tags, cnt, chi)
    assert ctx.status_sync() == 0
    out = (tags.cpu().numpy(), cnt.cpu().numpy(), chi.cpu().numpy() if want_chi else None)
    ctx.close()
    return out


def _check(blocks, shapes, ndim, kind, eps, chi_r, want_chi):
    pool, bases = _pool(blocks)
    specs = [(n, [0.1] * 3, base) for n, base in zip(shapes, bases)]
    tags, cnt, chi = _gpu_tag(pool, specs, ndim, kind, eps, chi_r, want_chi)
    total = 0
    for i, (b, n, base) in enumerate(zip(blocks, shapes, bases)):
        t_ref, chi_ref, c_ref = O.tag(b, n, ndim, kind, eps, chi_r)
        sl = slice(base, base + b[0].size)
        T = tags[sl].reshape(b.shape[1:])
        assert np.array_equal(O.interior(T[None], n, ndim), O.interior(t_ref[None], n, ndim)), (kind, n)
        assert cnt[i] == c_ref
        if want_chi:
            C = chi[sl].reshape(b.shape[1:])
            assert np.array_equal(O.interior(C[None], n, ndim), O.interior(chi_ref[None], n, ndim),
                                  equal_nan=True), (kind, n)
        total += c_ref
    # ghost entries of the tag array are not written
    mask = np.ones(tags.shape, bool)
    for b, n, base in zip(blocks, shapes, bases):
        m = np.ones(b.shape[1:], bool)
        m[tuple(slice(g, g + k) for g, k in zip(O.ghosts(ndim)[::-1], n[::-1]))] = False
        mask[base:base + b[0].size] = m.ravel()
    assert np.all(tags[mask] == 7)
    return total


def _blocks3(seed):
    big = W.mhd_blast_3d(48, seed=seed)
    # tiled (x width >= 16) and one-cell-per-thread patches, ragged tiles
    # in x and y, several z segments with a ragged last one
    shapes = [[21, 13, 11], [8, 8, 8], [48, 48, 48], [5, 17, 9], [1, 1, 1], [40, 9, 37], [16, 8, 16]]
    blocks = [np.ascontiguousarray(big[:, :n[2] + 8, :n[1] + 8, :n[0] + 8]) for n in shapes]
    return blocks, shapes


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_tag_parity_3d_batch(kind):
    blocks, shapes = _blocks3(seed=kind)
    # the paper's threshold, with chi written (float64 everywhere), then the
    # filtered path at the same threshold and at the median chi
    assert _check(blocks, shapes, 3, kind, EPS, 0.1, True) >= 0
    _check(blocks, shapes, 3, kind, EPS, 0.1, False)
    chis = np.concatenate([O.interior(O.tag(b, n, 3, kind, EPS, 0.1)[1][None], n, 3).ravel()
                           for b, n in zip(blocks, shapes)])
    med = float(np.median(chis))
    assert _check(blocks, shapes, 3, kind, EPS, med, False) > 0


@pytest.mark.parametrize("ndim", [1, 2])
def test_tag_parity_low_dimensions(ndim):
    if ndim == 2:
        big = W.mhd_turb_2d(64, seed=1)
        shapes = [[64, 64, 1], [13, 29, 1], [7, 5, 1]]
        blocks = [np.ascontiguousarray(big[:, :, :n[1] + 8, :n[0] + 8]) for n in shapes]
    else:
        rng = np.random.default_rng(2)
        shapes = [[100, 1, 1], [9, 1, 1]]
        blocks = []
        for n in shapes:
            b = np.ones((9, 1, 1, n[0] + 8))
            b[0, 0, 0] = 1.0 + 0.3 * np.sin(np.arange(n[0] + 8) * 0.4) + 0.05 * rng.normal(size=n[0] + 8)
            b[4, 0, 0] = 2.0 + rng.normal(size=n[0] + 8)
            blocks.append(b)
    for kind in (0, 1, 2, 3):
        _check(blocks, shapes, ndim, kind, EPS, 0.1, True)
        _check(blocks, shapes, ndim, kind, EPS, 0.1, False)
        _check(blocks, shapes, ndim, kind, 0.0, 0.1, False)  # eps = 0: every cell in float64


def test_tag_zero_sigma_is_nan_and_untagged():
    n = [6, 6, 6]
    b = np.zeros(O.shape(n, 3))
    b[0] = 0.0
    pool, bases = _pool([b])
    tags, cnt, chi = _gpu_tag(pool, [(n, [0.1] * 3, 0)], 3, 0, EPS, 0.0, True)
    assert cnt[0] == 0
    assert np.all(np.isnan(O.interior(chi.reshape(b.shape[1:])[None], n, 3)))


def test_tag_full_size_blast_256():
    """The 256^3 blast workload: every cell's tag at the paper's threshold
    (density and total energy) and at the median chi, against the oracle."""
    n = [256] * 3
    U0 = W.mhd_blast_3d(256, seed=0)
    for kind in (0, 1):
        t_ref, chi_ref, c_ref = O.tag(U0, n, 3, kind, EPS, 0.1)
        tags, cnt, _ = _gpu_tag(U0.reshape(9, -1), [(n, [1.0 / 256] * 3, 0)], 3, kind, EPS, 0.1, False)
        assert cnt[0] == c_ref
        assert np.array_equal(O.interior(tags.reshape(t_ref.shape)[None], n, 3),
                              O.interior(t_ref[None], n, 3))
        med = float(np.median(O.interior(chi_ref[None], n, 3)))
        t2, _, c2 = O.tag(U0, n, 3, kind, EPS, med)
        tags, cnt, _ = _gpu_tag(U0.reshape(9, -1), [(n, [1.0 / 256] * 3, 0)], 3, kind, EPS, med, False)
        assert cnt[0] == c2 and c2 > 0
        assert np.array_equal(O.interior(tags.reshape(t2.shape)[None], n, 3), O.interior(t2[None], n, 3))


def test_tag_amr_finest_level():
    """All ~460 patches (8^3..64^3) of the AMR hierarchy's finest level in one
    call, sigma = B^2/rho as in the paper's magnetised tests."""
    H = W.amr_hierarchy(seed=0)
    L2 = H["levels"][2]
    pool = L2["pool"]
    specs = [p[:3] for p in L2["patches"]]
    tags, cnt, _ = _gpu_tag(pool, specs, 3, 2, EPS, 0.1, False)
    for i, (n, dx, base, _) in enumerate(L2["patches"]):
        N = [v + 8 for v in n]
        blk = pool[:, base:base + N[0] * N[1] * N[2]].reshape(9, N[2], N[1], N[0])
        t_ref, _, c_ref = O.tag(blk, list(n), 3, 2, EPS, 0.1)
        T = tags[base:base + blk[0].size].reshape(blk.shape[1:])
        assert cnt[i] == c_ref
        assert np.array_equal(O.interior(T[None], list(n), 3), O.interior(t_ref[None], list(n), 3))
