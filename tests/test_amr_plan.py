"""Host plan of the batched AMR level advance (paper_1110_0740_gb300.amr_advance),
checked without a GPU on a seeded 3-level hierarchy (ratio 2, base 64^3, 149
patches of 8^3 to 64^3):

- the flux-register windows tile one register array and sit on both sides of
  every coarse-fine interface (fine faces weight +1, the parent faces under
  them weight -1), also when the patches are sharded over two ranks;
- the reflux sets pair every coarse window with its fine window and leave
  out exactly the faces whose coarse neighbour lies outside the parent;
- each fine patch's ghost shell is filled once: by the prolongation boxes
  where no sibling covers it, by the exchange boxes elsewhere;
- the launch sequence of one coarse step follows the subcycling of Section 4
  and never reads a ghost cell left over from an earlier state: every state a
  step or a prolongation reads has had its ghosts filled since it was last
  written.  The same check rejects a sequence that skips the new coarse
  state's ghost fill."""
import numpy as np
import pytest

from paper_1110_0740_gb300 import shard, workloads as W
from paper_1110_0740_gb300.amr_advance import LevelAdvance, LevelPlan

BASE = 64


@pytest.fixture(scope="module")
def levels():
    return W.amr_hierarchy(seed=3, base=BASE, target=80)["levels"]


@pytest.fixture(scope="module")
def plan(levels):
    return LevelPlan(levels, BASE)


def _size(w):
    _, _, _, a0, a1, b0, b1, _, _ = w
    return 9 * (a1 - a0) * (b1 - b0)


def _zyx(o):
    return [int(o[2]), int(o[1]), int(o[0])]


def test_windows_tile_the_register_array(plan, levels):
    spans = sorted((w[8], _size(w)) for ws in plan.windows for w in ws)
    pos = 0
    for off, n in spans:
        assert off == pos and n > 0
        pos += n
    assert pos == plan.nreg
    # interface (l - 1, l) owns one contiguous range, in level order
    assert plan.reg_range[0] is None
    assert plan.reg_range[1][0] == 0 and plan.reg_range[-1][1] == plan.nreg
    for lev in range(2, len(levels)):
        assert plan.reg_range[lev][0] == plan.reg_range[lev - 1][1]


def _faces(levels, lev):
    """Every face of every level-lev patch: (fine patch, dir, side, fine
    plane, parent, the face's first coarse cell (a, b) in global coordinates,
    size in coarse cells, the corrected coarse layer along dir, global)."""
    dom = BASE * 2 ** (lev - 1)
    for fi, (n, _, _, _) in enumerate(levels[lev]["patches"]):
        parent, o_zyx, sz = levels[lev]["footprints"][fi]
        o, po = _zyx(o_zyx), _zyx(levels[lev - 1]["origins"][parent][0])
        for d in range(3):
            a_, b_ = [e for e in range(3) if e != d]
            for side, fplane in ((-1, 0), (+1, n[d])):
                layer = (po[d] + (o[d] - 1 if side < 0 else o[d] + sz)) % dom
                yield fi, d, side, fplane, parent, po[a_] + o[a_], po[b_] + o[b_], sz, layer


def _holder(levels, lev, d, layer, a, b):
    """The level lev - 1 patch holding global coarse cell (layer along d;
    a, b along the other two), or None."""
    a_, b_ = [e for e in range(3) if e != d]
    for q, (qo_zyx, qs) in enumerate(levels[lev - 1]["origins"]):
        qo = _zyx(qo_zyx)
        if qo[d] <= layer < qo[d] + qs and qo[a_] <= a < qo[a_] + qs and qo[b_] <= b < qo[b_] + qs:
            return q
    return None


def test_windows_sit_on_both_sides_of_every_interface(plan, levels):
    for lev in range(1, len(levels)):
        fine = {(w[0], w[1], w[2]): w for w in plan.windows[lev] if w[7] == 1.0}
        coarse = {w[8]: w for w in plan.windows[lev - 1] if w[7] == -1.0}
        npieces = 0
        for fi, (n, _, _, _) in enumerate(levels[lev]["patches"]):
            assert n[0] == n[1] == n[2]
            for d in range(3):
                a_, b_ = [e for e in range(3) if e != d]
                for plane in (0, n[d]):
                    w = fine[(fi, d, plane)]
                    assert w[3:7] == (0, n[a_], 0, n[b_])
                    assert plan.fine_dst[lev][(fi, d, plane)] == w[8]
        for fi, d, side, fplane, parent, ga, gb, sz, layer in _faces(levels, lev):
            a_, b_ = [e for e in range(3) if e != d]
            parent_o = _zyx(levels[lev]["footprints"][fi][1])
            po = _zyx(levels[lev - 1]["origins"][parent][0])
            cplane = parent_o[d] + (0 if side < 0 else sz)
            pieces = plan.coarse_dst[lev][(fi, d, side)]
            npieces += len(pieces)
            seen = np.zeros((sz, sz), dtype=np.int32)
            for off, q, a0, a1, b0, b1 in pieces:
                # registered by the parent on its own face, weight -1
                assert coarse[off] == (parent, d, cplane, a0 - po[a_], a1 - po[a_], b0 - po[b_], b1 - po[b_], -1.0,
                                       off)
                assert ga <= a0 < a1 <= ga + sz and gb <= b0 < b1 <= gb + sz
                assert _holder(levels, lev, d, layer, a0, b0) == q == _holder(levels, lev, d, layer, a1 - 1, b1 - 1)
                seen[a0 - ga:a1 - ga, b0 - gb:b1 - gb] += 1
            # every coarse cell beside the face that a level lev - 1 patch
            # holds is in exactly one piece; the others in none
            for a in range(sz):
                for b in range(sz):
                    held = _holder(levels, lev, d, layer, ga + a, gb + b) is not None
                    assert seen[a, b] == int(held)
        assert len(fine) == 6 * len(levels[lev]["patches"])
        assert len(coarse) == npieces


def test_shards_keep_every_window_once(plan, levels):
    world = 2
    mine = []
    for lv in levels:
        cells = [n[0] * n[1] * n[2] for (n, _, _, _) in lv["patches"]]
        mine.append(shard.partition(cells, world))
    fine_all, coarse_all = [], []
    for rank in range(world):
        m = [mine[lev][rank] for lev in range(len(levels))]
        p = LevelPlan(levels, BASE, mine=m, level_ops=False)
        assert p.ops is None and not p.xch
        for lev in range(1, len(levels)):
            fine_all += [(lev, gi, d, pl) for (gi, d, pl) in p.fine_dst[lev]]
            for (fi, d, side) in p.coarse_dst[lev]:
                parent = levels[lev]["footprints"][fi][0]
                assert parent in m[lev - 1]  # kept by the rank that owns the parent
                coarse_all.append((lev, fi, d, side))
    with pytest.raises(ValueError):  # the level operators need every patch on one rank
        LevelPlan(levels, BASE, mine=[mine[lev][0] for lev in range(len(levels))], level_ops=True)
    full_fine = [(lev, gi, d, pl) for lev in range(1, len(levels)) for (gi, d, pl) in plan.fine_dst[lev]]
    full_coarse = [(lev, fi, d, s) for lev in range(1, len(levels)) for (fi, d, s) in plan.coarse_dst[lev]]
    assert sorted(fine_all) == sorted(full_fine)
    assert sorted(coarse_all) == sorted(full_coarse)


def test_reflux_sets_pair_the_windows(plan, levels):
    shared = 0
    for lev in range(1, len(levels)):
        sets = plan.ops[lev][2]
        got = {S.creg: S for S in sets}
        assert len(got) == len(sets)
        cells = {}
        npieces = 0
        for fi, d, side, fplane, parent, ga, gb, sz, layer in _faces(levels, lev):
            a_, b_ = [e for e in range(3) if e != d]
            n = levels[lev]["patches"][fi][0]
            for off, q, a0, a1, b0, b1 in plan.coarse_dst[lev][(fi, d, side)]:
                npieces += 1
                S = got[off]
                qn, qdx, qbase = levels[lev - 1]["patches"][q][:3]
                qo = _zyx(levels[lev - 1]["origins"][q][0])
                cell = layer - qo[d]  # the corrected layer in patch q
                assert (S.dir, S.side, S.cbase, S.ratio) == (d, side, qbase, 2)
                assert S.plane == (cell if side > 0 else cell + 1)
                assert (S.a0, S.a1, S.b0, S.b1) == (a0 - qo[a_], a1 - qo[a_], b0 - qo[b_], b1 - qo[b_])
                assert S.freg == plan.fine_dst[lev][(fi, d, fplane)]
                assert (S.fna, S.fnb, S.fa0, S.fb0) == (n[a_], n[b_], 2 * (a0 - ga), 2 * (b0 - gb))
                assert list(S.cn) == list(qn) and list(S.dx) == list(qdx)
                for a in range(S.a0, S.a1):
                    for b in range(S.b0, S.b1):
                        c = [0, 0, 0]
                        c[d], c[a_], c[b_] = cell, a, b
                        k = (q, tuple(c))
                        cells[k] = cells.get(k, 0) + 1
        assert len(sets) == npieces
        shared += sum(1 for v in cells.values() if v > 1)
    # coarse cells beside two interfaces (inner corners) exist, so the
    # reflux order matters on this hierarchy
    assert shared > 0


def nested_levels():
    """A properly nested 3-level hierarchy on a 32^3 base (8 level-0 patches
    of 16^3) holding a smooth periodic state: level-1 siblings A and B (16^3)
    side by side across a level-0 patch boundary and an 8^3 patch C
    elsewhere; level-2 patches D (8^3, in A, against A's +x face with B
    across it) and E (8^3, inside B)."""
    lv0 = [((k, j, i), 16) for k in (0, 16) for j in (0, 16) for i in (0, 16)]
    lv1 = [((8, 8, 16), 16), ((8, 8, 32), 16), ((40, 40, 40), 8)]
    lv2 = [((24, 24, 56), 8), ((24, 24, 80), 8)]
    return W.amr_levels([lv0, lv1, lv2], [[], [0, 1, 7], [0, 1]], 32, None, None, smooth=True)["levels"]


def test_a_face_on_the_parent_boundary_refluxes_the_patch_across():
    levels = nested_levels()
    p = LevelPlan(levels, 32)
    assert p.unmatched_faces == 0  # properly nested: every corrected cell has a patch
    # D's +x face lies on A's boundary: its window is registered by A, and
    # its correction lands on B's first x layer
    (off, q, a0, a1, b0, b1), = p.coarse_dst[2][(0, 0, +1)]
    assert q == 1 and (a1 - a0, b1 - b0) == (4, 4)
    S, = [S for S in p.ops[2][2] if S.creg == off]
    assert (S.dir, S.side, S.plane, S.cbase) == (0, +1, 0, levels[1]["patches"][1][2])
    # level-1 faces on level-0 patch boundaries: B's -x face corrects
    # level-0 patch 0 (which holds A's footprint: covered, then restricted)
    (off, q, *_), = p.coarse_dst[1][(1, 0, -1)]
    assert q == 0


def test_the_bench_hierarchy_counts_its_improperly_nested_faces(plan, levels):
    """The seeded hierarchy places level-2 patches against the edge of the
    level-1 region; the coarse faces there have no level-1 patch to reflux
    and are counted, not corrected."""
    expect = 0
    for lev in range(1, len(levels)):
        for fi, d, side, fplane, parent, ga, gb, sz, layer in _faces(levels, lev):
            for a in range(sz):
                for b in range(sz):
                    expect += _holder(levels, lev, d, layer, ga + a, gb + b) is None
    assert plan.unmatched_faces == expect > 0


def test_ghost_shells_are_filled_once(plan, levels):
    for lev in range(1, len(levels)):
        pb = plan.ops[lev][0]
        xb = plan.xch.get(lev, [])
        for fi, (n, _, base, _) in enumerate(levels[lev]["patches"]):
            hits = np.zeros([v + 8 for v in n[::-1]], dtype=np.int32)  # (z, y, x), ghosts included
            for B in pb:
                if B.fbase != base:
                    continue
                hits[B.lo[2] + 4:B.hi[2] + 4, B.lo[1] + 4:B.hi[1] + 4, B.lo[0] + 4:B.hi[0] + 4] += 1
            for B in xb:
                if B.dbase != base:
                    continue
                hits[B.lo[2] + 4:B.hi[2] + 4, B.lo[1] + 4:B.hi[1] + 4, B.lo[0] + 4:B.hi[0] + 4] += 1
            interior = np.zeros_like(hits, dtype=bool)
            interior[4:-4, 4:-4, 4:-4] = True
            assert np.all(hits[interior] == 0)
            assert np.all(hits[~interior] == 1)


class _Buf:
    def __init__(self, name, lev):
        self.name, self.lev, self.shape = name, lev, (9, 1)


class _Reg:
    def __getitem__(self, sl):
        return self

    def zero_(self):
        pass


class _Ghosts:
    """Ghost validity of every state over one coarse step: a state's ghosts
    are valid once, since its interior was last written, it has had its
    prolongation (levels >= 1) and its same-level exchange."""

    def __init__(self):
        self.done = {}  # buffer -> set of fills since its last write
        self.log = []
        self.launches = 0

    def written(self, U):
        self.done[U.name] = set()

    def valid(self, U):
        need = {"exchange"} | ({"prolong"} if U.lev > 0 else set())
        return need <= self.done.get(U.name, set())


class _Ctx:
    def __init__(self, lev, g):
        self.lev, self.g = lev, g

    def step(self, src, dst, stride, P, D, stream=None):
        assert self.g.valid(src), f"step reads stale ghosts of {src.name}"
        self.g.written(dst)
        self.g.log.append(("step", src.name, dst.name))

    def prolong(self, po, pn, cs, alpha, U, fs, boxes, stream=None):
        if alpha < 1:
            assert self.g.valid(po), f"prolongation reads stale ghosts of {po.name}"
        if alpha > 0:
            assert self.g.valid(pn), f"prolongation reads stale ghosts of {pn.name}"
        self.g.done.setdefault(U.name, set()).add("prolong")
        self.g.log.append(("prolong", po.name, pn.name, alpha, U.name))

    def copy(self, d, ds, s, ss, boxes, stream=None):
        self.g.done.setdefault(d.name, set()).add("exchange")
        self.g.log.append(("exchange", d.name))

    def reflux(self, U, cs, reg, sets, stream=None):
        self.g.written(U)
        self.g.log.append(("reflux", U.name))
        self.g.launches += len({(S.dir, S.side) for S in sets})  # one launch per class

    def launches(self):
        return 7 + self.lev  # a step's kernel launches, any per-level count

    def restrict(self, U, cs, F, fs, boxes, stream=None):
        self.g.written(U)
        self.g.log.append(("restrict", U.name, F.name))


def _mock(plan, advance_cls=LevelAdvance):
    g = _Ghosts()
    adv = advance_cls.__new__(advance_cls)
    adv.nlev = plan.nlev
    adv.A = [_Buf(f"A{lev}", lev) for lev in range(plan.nlev)]
    adv.B = [_Buf(f"B{lev}", lev) for lev in range(plan.nlev)]
    adv.ctxs = [_Ctx(lev, g) for lev in range(plan.nlev)]
    adv.P, adv.D = [1] * plan.nlev, [None] * plan.nlev
    adv.ops, adv.xch, adv.reg_range, adv.reg = plan.ops, plan.xch, plan.reg_range, _Reg()
    return adv, g


def test_coarse_step_reads_no_stale_ghosts(plan):
    adv, g = _mock(plan)
    adv.coarse_step(None)
    steps = [e for e in g.log if e[0] == "step"]
    # level 0 once, level 1 twice, level 2 four times, ping-ponging
    assert [s[1:] for s in steps] == [("A0", "B0"), ("A1", "B1"), ("A2", "B2"), ("B2", "A2"),
                                      ("B1", "A1"), ("A2", "B2"), ("B2", "A2")]
    assert [(e[1], e[2], e[3]) for e in g.log if e[0] == "prolong"] == [
        ("A0", "B0", 0.0), ("A0", "B0", 0.5), ("A1", "B1", 0.0), ("A1", "B1", 0.5),
        ("A0", "B0", 0.5), ("A0", "B0", 1.0), ("B1", "A1", 0.0), ("B1", "A1", 0.5)]
    # every synchronisation refluxes, then restricts the parent's new state
    assert [e for e in g.log if e[0] in ("reflux", "restrict")] == [
        ("reflux", "B1"), ("restrict", "B1", "A2"), ("reflux", "A1"), ("restrict", "A1", "A2"),
        ("reflux", "B0"), ("restrict", "B0", "A1")]
    assert [b.name for b in adv.outputs()] == ["B0", "A1", "A2"]
    # the launch count the bench reports: every step's launches, one per
    # prolongation, exchange and restriction, one per reflux class
    lev_of = {"A0": 0, "B0": 0, "A1": 1, "B1": 1, "A2": 2, "B2": 2}
    issued = g.launches + sum(7 + lev_of[e[2]] for e in g.log if e[0] == "step")
    issued += sum(1 for e in g.log if e[0] in ("prolong", "exchange", "restrict"))
    assert adv.launches() == issued


def test_the_check_rejects_a_coarse_state_without_its_ghost_fill(plan):
    class NoNewStateFill(LevelAdvance):
        def _substeps(self, lev, pold, pnew, stream):
            A, B = self.A, self.B
            for k in range(2):
                s, d = (A[lev], B[lev]) if k == 0 else (B[lev], A[lev])
                self._ghosts(lev, pold, pnew, k / 2, s, stream)
                self._step(lev, s, d, stream)
                if lev + 1 < self.nlev:  # no ghost fill of d before the finer level prolongs from it
                    self._substeps(lev + 1, s, d, stream)
                    self._sync(lev + 1, d, A[lev + 1], stream)

    adv, _ = _mock(plan, NoNewStateFill)
    with pytest.raises(AssertionError, match="stale ghosts of B1"):
        adv.coarse_step(None)


# ---------------------------------------------------------------- the coarse
# step in the oracle: LevelAdvance's plan and launch sequence, every launch
# carried out by the oracle's operators on float64 host pools


class _RegArray:
    """The flux registers as a host array, with the slice zeroing the
    coarse step uses."""

    def __init__(self, n):
        self.arr = np.zeros(max(n, 1))

    def __getitem__(self, sl):
        arr = self.arr

        class _Slice:
            def zero_(self):
                arr[sl] = 0.0
        return _Slice()


def _block(pool, base, n):
    N = [v + 8 for v in n]
    return pool[:, base:base + N[0] * N[1] * N[2]].reshape(9, N[2], N[1], N[0])


class _OracleCtx:
    """One level's context: ctu_step, ctu_prolong, ctu_copy, ctu_reflux and
    ctu_restrict on host pools, each by the oracle's function of the same
    equation, patch by patch and box by box."""

    def __init__(self, windows, reg, par):
        import oracle as O
        self.O, self.reg, self.par = O, reg, par
        self.win = {}
        for (p, d, plane, a0, a1, b0, b1, wgt, off) in windows:
            self.win.setdefault(p, []).append((d, plane, a0, a1, b0, b1, off, wgt))

    def step(self, src, dst, stride, P, D, stream=None):
        dt, ch = D
        for i, p in enumerate(P):
            n = list(p.n)
            U = np.ascontiguousarray(_block(src, p.base, n))
            R, bad = self.O.mhd_step(U, n, 3, list(p.dx), dt, ch, recon=1, windows=self.win.get(i, []),
                                     reg=self.reg.arr, **self.par)
            assert bad == 0
            _block(dst, p.base, n)[:, 4:-4, 4:-4, 4:-4] = R[:, 4:-4, 4:-4, 4:-4]

    def prolong(self, po, pn, cs, alpha, U, fs, boxes, stream=None):
        for b in boxes:
            cn, fn = list(b.cn), list(b.fn)
            F = np.ascontiguousarray(_block(U, b.fbase, fn))
            self.O.prolong(np.ascontiguousarray(_block(po, b.cbase, cn)), np.ascontiguousarray(_block(pn, b.cbase, cn)),
                           cn, alpha, F, fn, list(b.lo), list(b.hi), list(b.origin), b.ratio, 3, b.phys)
            _block(U, b.fbase, fn)[...] = F

    def copy(self, d, ds, s, ss, boxes, stream=None):
        self.O.copy_boxes(d, s, [dict(dn=list(b.dn), sn=list(b.sn), lo=list(b.lo), hi=list(b.hi),
                                      shift=list(b.shift), dbase=b.dbase, sbase=b.sbase) for b in boxes], 3)

    def reflux(self, U, cs, reg, sets, stream=None):
        for S in sorted(sets, key=lambda S: (S.dir, S.side)):
            cn = list(S.cn)
            C = np.ascontiguousarray(_block(U, S.cbase, cn))
            self.O.reflux(C, cn, list(S.dx), reg.arr, S.dir, S.plane, S.side, S.a0, S.a1, S.b0, S.b1, S.creg,
                          S.freg, S.fa0, S.fb0, S.fna, S.fnb, S.ratio, 3)
            _block(U, S.cbase, cn)[...] = C

    def restrict(self, U, cs, F, fs, boxes, stream=None):
        for b in boxes:
            cn, fn = list(b.cn), list(b.fn)
            C = np.ascontiguousarray(_block(U, b.cbase, cn))
            self.O.restrict(C, cn, np.ascontiguousarray(_block(F, b.fbase, fn)), fn, list(b.lo), list(b.hi),
                            list(b.origin), b.ratio, 3)
            _block(U, b.cbase, cn)[...] = C


def _oracle_coarse_step(levels, base, plan, par, result=None):
    """Restrict the hierarchy (every covered coarse cell the mean of its
    children), then take one coarse step; returns level 0's totals of
    U_q x cell volume before and after, and the totals of |U_q| x volume.
    `result`, a dict, receives dt_0, c_h and every level's output pool."""
    import oracle as O
    from paper_1110_0740_gb300 import ctu
    adv = LevelAdvance.__new__(LevelAdvance)
    adv.nlev = len(levels)
    adv.A = [lv["pool"].copy() for lv in levels]
    adv.B = [a.copy() for a in adv.A]
    adv.reg = _RegArray(plan.nreg)
    adv.ctxs = [_OracleCtx(plan.windows[lev], adv.reg, par) for lev in range(len(levels))]
    adv.P = [ctu.make_patches([p[:3] for p in lv["patches"]]) for lv in levels]
    adv.ops, adv.xch, adv.reg_range = plan.ops, plan.xch, plan.reg_range
    # dt_0 from Eq. Ca on every level, dt_l = dt_0 / 2^l, one c_h
    dt0 = np.inf
    for lev, lv in enumerate(levels):
        for n, dx, b in (p[:3] for p in lv["patches"]):
            U = np.ascontiguousarray(_block(lv["pool"], b, n))
            rate = O.mhd_max_rate(U, n, 3, dx, **par) if par else O.mhd_max_speed(U, n, 3, dx)
            dt0 = min(dt0, O.dt_ch(rate, dx, 3, 0.3)[0] * 2 ** lev)
    ch = 0.3 * levels[0]["patches"][0][1][0] / dt0
    adv.D = [(dt0 / 2 ** lev, ch) for lev in range(len(levels))]
    for lev in (2, 1):
        adv.ctxs[lev - 1].restrict(adv.A[lev - 1], 0, adv.A[lev], 0, plan.ops[lev][1])

    def totals(pool):
        tot, mag = np.zeros(9), np.zeros(9)
        for n, dx, b in (p[:3] for p in levels[0]["patches"]):
            U = _block(pool, b, n)[:, 4:-4, 4:-4, 4:-4]
            tot += U.sum(axis=(1, 2, 3)) * dx[0] * dx[1] * dx[2]
            mag += np.abs(U).sum(axis=(1, 2, 3)) * dx[0] * dx[1] * dx[2]
        return tot, mag
    tot0, mag = totals(adv.A[0])
    adv.coarse_step(None)
    tot1, _ = totals(adv.outputs()[0])
    if result is not None:
        result.update(dt0=dt0, ch=ch, outputs=adv.outputs())
    return tot0, tot1, mag


@pytest.mark.parametrize("par", [{}, dict(kappa=0.002, nu=0.001, eta=0.001)])
def test_the_oracle_conserves_through_the_plan(par):
    """Eq. fluxcorr, Eq. addreflux, Eq. avgdown: the plan's registers, reflux
    sets (the pieces across a parent boundary included) and launch sequence
    keep the composite totals of a properly nested hierarchy to round-off,
    the operators being the oracle's."""
    levels = nested_levels()
    tot0, tot1, mag = _oracle_coarse_step(levels, 32, LevelPlan(levels, 32), par)
    assert np.all(np.abs(tot1 - tot0)[:8] <= 1e-13 * mag[:8]), (tot1 - tot0) / mag


def test_without_the_pieces_across_a_parent_boundary_the_totals_drift():
    """The same step with the reflux sets of the faces on a parent's boundary
    left out (the former plan): the flux there stays uncorrected."""
    from paper_1110_0740_gb300 import ctu
    levels = nested_levels()
    plan = LevelPlan(levels, 32)
    for lev in (1, 2):
        pb, rb, fs = plan.ops[lev]
        inside = set()
        for fi, d, side, fplane, parent, ga, gb, sz, layer in _faces(levels, lev):
            po = _zyx(levels[lev - 1]["origins"][parent][0])
            cn = levels[lev - 1]["patches"][parent][0]
            if 0 <= layer - po[d] < cn[d]:
                inside.update(off for off, *_ in plan.coarse_dst[lev][(fi, d, side)])
        keep = [S for S in fs if S.creg in inside]
        assert 0 < len(keep) < len(fs)
        sets = (ctu.ctu_reflux_set * len(keep))(*keep)
        plan.ops[lev] = (pb, rb, sets)
    tot0, tot1, mag = _oracle_coarse_step(levels, 32, plan, {})
    assert np.any(np.abs(tot1 - tot0)[:8] > 1e-10 * mag[:8])


def test_a_nested_seeded_hierarchy_conserves():
    """amr_hierarchy(nested=True) keeps one level-l cell of level l around
    every level-(l+1) patch, so every coarse face beside a fine patch has a
    patch to reflux (none unmatched), and the oracle-driven coarse step of
    the seeded hierarchy (smooth state, 61 patches) conserves to round-off."""
    levels = W.amr_hierarchy(seed=5, base=32, target=40, nested=True, smooth=True)["levels"]
    assert all(len(lv["patches"]) for lv in levels)
    plan = LevelPlan(levels, 32)
    assert plan.unmatched_faces == 0
    tot0, tot1, mag = _oracle_coarse_step(levels, 32, plan, {})
    assert np.all(np.abs(tot1 - tot0)[:8] <= 1e-13 * mag[:8]), (tot1 - tot0) / mag
