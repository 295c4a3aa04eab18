"""Same-level ghost exchange (host plan + the oracle's copy, pack and
unpack), pinned against the definition: a periodic domain cut into patches
of unequal sizes must, after one exchange, hold in every patch's ghosted
block exactly the periodically wrapped values of the whole domain (checked
with numpy's wrap-around indexing, not with the copy code); without
periodicity the ghosts outside the domain stay untouched.  Pack + unpack
equals the direct copy, and two gloo ranks that own alternate patches reach
the single-process result."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1110_0740_gb300 import exchange as X  # noqa: E402

G = 4


def _decomp(domain, cuts, ndim):
    """Patches of a box decomposition: cuts[d] are the split points."""
    out = []
    for z0, z1 in zip(cuts[2][:-1], cuts[2][1:]):
        for y0, y1 in zip(cuts[1][:-1], cuts[1][1:]):
            for x0, x1 in zip(cuts[0][:-1], cuts[0][1:]):
                out.append(([x0, y0, z0], [x1 - x0, y1 - y0, z1 - z0]))
    return out


def _pool(big, parts, ndim, fill=np.nan):
    """Pool with every patch's interior from `big` ([9][Z][Y][X]) and
    ghosts set to `fill`."""
    specs, off = [], 0
    for lo, n in parts:
        specs.append((lo, n, off))
        off += int(np.prod(O.shape(n, ndim)[1:]))
    pool = np.full((9, off), fill)
    for lo, n, base in specs:
        blk = np.full(O.shape(n, ndim), fill)
        g = [G if d < ndim else 0 for d in range(3)]
        blk[:, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]] = \
            big[:, lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]]
        pool[:, base:base + blk[0].size] = blk.reshape(9, -1)
    return pool, specs


def _block(pool, n, base, ndim):
    shp = O.shape(n, ndim)
    return pool[:, base:base + int(np.prod(shp[1:]))].reshape(shp)


def _wrapped(big, lo, n, ndim):
    """The ghosted block of a patch read from the periodic domain."""
    g = [G if d < ndim else 0 for d in range(3)]
    idx = [np.arange(lo[d] - g[d], lo[d] + n[d] + g[d]) for d in range(3)]
    return big.take(idx[2], axis=1, mode="wrap").take(idx[1], axis=2, mode="wrap").take(idx[0], axis=3, mode="wrap")


def _setup(ndim, seed):
    rng = np.random.default_rng(seed)
    if ndim == 3:
        domain, cuts = [24, 20, 16], [[0, 10, 24], [0, 8, 20], [0, 9, 16]]
    else:
        domain, cuts = [30, 22, 1], [[0, 7, 19, 30], [0, 12, 22], [0, 1]]
    big = rng.normal(size=(9, domain[2], domain[1], domain[0]))
    return domain, _decomp(domain, cuts, ndim), big


@pytest.mark.parametrize("ndim", [2, 3])
def test_periodic_decomposition_reproduces_the_wrapped_domain(ndim):
    domain, parts, big = _setup(ndim, ndim)
    pool, specs = _pool(big, parts, ndim)
    boxes = X.plan(specs, domain, [True] * 3, ndim)
    O.copy_boxes(pool, pool, boxes, ndim)
    ghost_cells = 0
    for lo, n, base in specs:
        got = _block(pool, n, base, ndim)
        assert np.array_equal(got, _wrapped(big, lo, n, ndim)), (lo, n)
        ghost_cells += got[0].size - int(np.prod(n))
    # every ghost cell is written by exactly one box
    assert sum(X.cells(b) for b in boxes) == ghost_cells


def test_single_patch_exchange_is_the_periodic_fill():
    n = [12, 10, 8]
    rng = np.random.default_rng(5)
    big = rng.normal(size=(9, 8, 10, 12))
    pool, specs = _pool(big, [([0, 0, 0], n)], 3)
    O.copy_boxes(pool, pool, X.plan(specs, n, [True] * 3, 3), 3)
    ref = _block(pool, n, 0, 3).copy()
    ref[:] = np.nan
    ref[:, G:G + 8, G:G + 10, G:G + 12] = big
    O.fill_periodic(ref, n, 3)
    assert np.array_equal(_block(pool, n, 0, 3), ref)


def test_non_periodic_leaves_outer_ghosts_untouched():
    domain, parts, big = _setup(3, 7)
    pool, specs = _pool(big, parts, 3)
    O.copy_boxes(pool, pool, X.plan(specs, domain, [False] * 3, 3), 3)
    for lo, n, base in specs:
        got = _block(pool, n, base, 3)
        want = _wrapped(big, lo, n, 3)
        for z in range(got.shape[1]):
            for y in range(got.shape[2]):
                for x in range(got.shape[3]):
                    c = [lo[0] - G + x, lo[1] - G + y, lo[2] - G + z]
                    inside = all(0 <= c[d] < domain[d] for d in range(3))
                    if inside:
                        assert np.array_equal(got[:, z, y, x], want[:, z, y, x])
                    else:
                        assert np.all(np.isnan(got[:, z, y, x]))


def test_pack_unpack_equals_copy():
    domain, parts, big = _setup(3, 11)
    pool, specs = _pool(big, parts, 3)
    boxes = X.plan(specs, domain, [True, False, True], 3)
    a = pool.copy()
    O.copy_boxes(a, a, boxes, 3)
    b = pool.copy()
    buf = O.pack_boxes(b, boxes, 3)
    assert buf.size == 9 * sum(X.cells(x) for x in boxes)
    O.unpack_boxes(b, buf, boxes, 3)
    assert np.array_equal(a, b, equal_nan=True)


def test_split_partitions_the_boxes():
    domain, parts, big = _setup(3, 1)
    specs = [(lo, n, 0) for lo, n in parts]
    boxes = X.plan(specs, domain, [True] * 3, 3)
    owner = [i % 3 for i in range(len(specs))]
    seen = 0
    for r in range(3):
        local, send, recv = X.split(boxes, owner, r)
        seen += len(local) + sum(len(v) for v in send.values())
        for peer, bl in send.items():
            assert bl == X.split(boxes, owner, peer)[2][r]
    assert seen == len(boxes)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        domain, parts, big = _setup(3, 13)
        owner = [i % world for i in range(len(parts))]
        # this rank's pool holds only its own patches
        mine = [i for i in range(len(parts)) if owner[i] == rank]
        pool, specs_m = _pool(big, [parts[i] for i in mine], 3)
        specs = [None] * len(parts)
        for k, i in enumerate(mine):
            specs[i] = specs_m[k]
        # the other ranks' bases are theirs; every rank derives them alike
        for r in range(world):
            if r == rank:
                continue
            idx = [i for i in range(len(parts)) if owner[i] == r]
            _, sp = _pool(big, [parts[i] for i in idx], 3)
            for k, i in enumerate(idx):
                specs[i] = sp[k]
        boxes = X.plan(specs, domain, [True] * 3, 3)

        def copy(U, bl):
            O.copy_boxes(U, U, bl, 3)

        def pack(U, bl):
            return torch.from_numpy(O.pack_boxes(U, bl, 3))

        def unpack(U, buf, bl):
            O.unpack_boxes(U, buf.numpy(), bl, 3)

        X.exchange(boxes, owner, rank, pool, copy, pack, unpack,
                   X.torch_sendrecv(torch.zeros(1, dtype=torch.float64)))
        res = {i: _block(pool, parts[i][1], specs[i][2], 3).copy() for i in mine}
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_like_one_process():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    domain, parts, big = _setup(3, 13)
    got = {}
    for _, r in res:
        got.update(r)
    assert sorted(got) == list(range(len(parts)))
    for i, (lo, n) in enumerate(parts):
        assert np.array_equal(got[i], _wrapped(big, lo, n, 3)), i


def _mask(n, ndim, boxes):
    g = [G if d < ndim else 0 for d in range(3)]
    m = np.zeros([n[2] + 2 * g[2], n[1] + 2 * g[1], n[0] + 2 * g[0]], dtype=np.int32)
    for lo, hi in boxes:
        m[lo[2] + g[2]:hi[2] + g[2], lo[1] + g[1]:hi[1] + g[1], lo[0] + g[0]:hi[0] + g[0]] += 1
    return m


def test_exchange_and_uncovered_boxes_tile_the_ghost_shell():
    """On every patch of the AMR hierarchy's finest level (non-periodic) and
    of a periodic decomposition, the exchange boxes and the uncovered boxes
    together cover each ghost cell exactly once and no interior cell."""
    from paper_1110_0740_gb300 import workloads as W
    H = W.amr_hierarchy(seed=2, base=32, target=60)
    cases = []
    lv = H["levels"][2]
    cases.append(([((o[2], o[1], o[0]), (s, s, s), 0) for (o, s) in lv["origins"]], [128] * 3, [False] * 3, 3))
    domain, parts, _ = _setup(3, 0)
    cases.append(([(lo, n, 0) for lo, n in parts], domain, [True] * 3, 3))
    cases.append(([(lo, n, 0) for lo, n in parts], domain, [False, True, False], 3))
    domain2, parts2, _ = _setup(2, 0)
    cases.append(([(lo, n, 0) for lo, n in parts2], domain2, [False] * 3, 2))
    for specs, dom, per, ndim in cases:
        boxes = X.plan(specs, dom, per, ndim)
        unc = X.uncovered(boxes, len(specs), [s[1] for s in specs], ndim)
        for i, (lo, n, _) in enumerate(specs):
            m = _mask(n, ndim, [(b["lo"], b["hi"]) for b in boxes if b["dst"] == i] + unc[i])
            inner = np.zeros_like(m, dtype=bool)
            g = [G if d < ndim else 0 for d in range(3)]
            inner[g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]] = True
            assert np.all(m[inner] == 0) and np.all(m[~inner] == 1), (i, per)
        if all(per[:ndim]):
            assert all(not u for u in unc)


def _reg_rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items, regs = _reg_case(world)
        reg = torch.from_numpy(regs[rank].copy())
        X.ship_registers(items, rank, reg, X.torch_sendrecv(reg))
        out.put((rank, reg.numpy()))
    finally:
        dist.destroy_process_group()


def _reg_case(world, S=400):
    """Register arrays of every rank (seeded) and windows of random sizes,
    each accumulated on one rank and refluxed on another (or the same)."""
    rng = np.random.default_rng(4)
    regs = [rng.normal(size=S) for _ in range(world)]
    items, used = [], [set() for _ in range(world)]
    for _ in range(12):
        s, d = (int(v) for v in rng.integers(0, world, 2))
        n = int(rng.integers(1, 20))
        so = int(rng.integers(0, S - n))
        # destination ranges of one rank do not overlap each other
        while True:
            do = int(rng.integers(0, S - n))
            if not (set(range(do, do + n)) & used[d]):
                used[d] |= set(range(do, do + n))
                break
        items.append((s, so, d, do, n))
    return items, regs


def test_registers_reach_the_coarse_owner():
    """Two gloo ranks ship register windows: every window whose ranks differ
    arrives at its destination range, everything else is untouched."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_reg_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    items, regs = _reg_case(world)
    want = [r.copy() for r in regs]
    for s, so, d, do, n in items:
        if s != d:
            want[d][do:do + n] = regs[s][so:so + n]
    assert any(s != d for s, _, d, _, _ in items)
    for r in range(world):
        assert np.array_equal(got[r], want[r])
