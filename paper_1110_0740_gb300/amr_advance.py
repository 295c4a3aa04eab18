"""Batched AMR level advance (Section 4): the subcycled coarse step of a
hierarchy of patch levels at refinement ratio 2 on one GPU.

One coarse step advances level 0 once and level l 2^l times (dt_l = dt_0 /
2^l, one c_h for every level), each substep one batched ctu_step over all of
the level's patches.  Around the steps run the level operators of Section 4:

- before a substep of level l >= 1, the ghost cells of its patches that no
  sibling covers are prolonged from level l - 1 interpolated in time
  (Eq. prolong, Eq. intalpha, at alpha = k/2 for substep k), then the rest
  are copied from the siblings (same-level exchange);
- a new state that a finer level prolongs from gets its ghosts at its new
  time as soon as it is computed (level 0 by its exchange, level l >= 1 by
  prolongation at alpha = (k + 1)/2 and exchange): the prolongation's slopes
  reach into the parent patch's own ghost cells;
- after the two substeps of level l within one substep of its parent, the
  parent is refluxed from the flux registers (Eq. fluxcorr, Eq. addreflux),
  then restricted (Eq. avgdown; reflux first, so that a correction landing on
  a covered coarse cell is overwritten by the restriction), and the
  interface's registers are zeroed.

Flux-register windows lie on both sides of every coarse-fine interface: on
the six faces of every fine patch (weight +1) and on the parent's faces under
them (weight -1).  With patch shards (`mine`, one rank's patches per level)
a coarse window is kept by the rank that owns its parent patch; the level
operators then need the cross-rank exchange, so they run on one rank only.

Host logic only: every step, copy, prolongation, reflux and restriction runs
in the library's kernels through the binding in `ctu`, on torch device
tensors; nothing here computes on the host.
"""
from __future__ import annotations

from . import ctu

RATIO = 2


def _xyz(o_zyx):
    """(z, y, x) -> [x, y, z] as ints."""
    return [int(o_zyx[2]), int(o_zyx[1]), int(o_zyx[0])]


class LevelPlan:
    """The host-side plan of a hierarchy's coarse step, built without a GPU:
    the flux-register windows of every level context and their offsets in
    one register array, and the level operators' descriptor tables.

    levels, domain, mine: as for LevelAdvance.  After construction:
    windows[l] (the windows bound to level l's context, local patch indices),
    fine_dst[l][(patch, dir, plane)] (a fine window's offset),
    coarse_dst[l][(fine patch, dir, side)] (the pieces of a coarse window,
    see _windows), unmatched_faces, reg_range[l] (the registers of interface
    (l - 1, l)), nreg; with level_ops, xch[l] (exchange boxes) and ops[l] =
    (prolongation boxes, restriction boxes, reflux sets) for l >= 1."""

    def __init__(self, levels, domain, *, mine=None, level_ops=True):
        self.levels = levels
        self.nlev = len(levels)
        if mine is None:
            mine = [list(range(len(lv["patches"]))) for lv in levels]
        self.mine = mine
        if level_ops and any(sorted(m) != list(range(len(lv["patches"]))) for m, lv in zip(mine, levels)):
            raise ValueError("the level operators run on one rank: mine must hold every patch of every level")
        self._windows([{g: i for i, g in enumerate(m)} for m in mine], domain)
        self.ops = None
        self.xch = {}
        if level_ops:
            self._level_ops(domain)

    # ------------------------------------------------------------ plan

    def _windows(self, loc, domain):
        """Flux-register windows per level context (local patch indices) and
        their offsets in one register array.

        Fine windows cover the six faces of every fine patch (weight +1).  The
        coarse window under a fine face lies on the parent's face there
        (weight -1, registered by the parent, which computes that coarse
        flux).  The coarse cells the correction lands on are the parent's when
        the face lies inside it; a face on the parent's boundary has them in
        the coarse patches across that boundary (periodic box), so its coarse
        window is split into one piece per such patch.  coarse_dst[l][(fine
        patch, dir, side)] lists the pieces: (register offset, coarse patch
        holding the corrected cells, a0, a1, b0, b1 in level l - 1's global
        cell coordinates); slab cells that no level l - 1 patch holds (a fine
        patch not properly nested) get no piece and are counted in
        unmatched_faces."""
        L, mine = self.levels, self.mine
        self.windows = [[] for _ in L]
        self.fine_dst = [dict() for _ in L]    # (patch, dir, plane) -> offset of a fine window
        self.coarse_dst = [dict() for _ in L]  # (fine patch, dir, side) -> pieces of its coarse window
        self.reg_range = [None for _ in L]     # registers of the interface (lev - 1, lev)
        self.unmatched_faces = 0               # coarse faces across a boundary that no patch holds
        off = 0
        for lev in range(1, len(L)):
            r0 = off
            for gi in mine[lev]:
                n = L[lev]["patches"][gi][0]
                for d in range(3):
                    a_, b_ = [e for e in range(3) if e != d]
                    for plane in (0, n[d]):
                        self.windows[lev].append((loc[lev][gi], d, plane, 0, n[a_], 0, n[b_], 1.0, off))
                        self.fine_dst[lev][(gi, d, plane)] = off
                        off += 9 * n[a_] * n[b_]
            dom = domain * RATIO ** (lev - 1)  # level lev - 1's cells per side
            corg = [_xyz(o) for (o, _) in L[lev - 1]["origins"]]
            csz = [s_ for (_, s_) in L[lev - 1]["origins"]]
            for fi, (parent, o_zyx, sz) in enumerate(L[lev]["footprints"]):
                if parent not in loc[lev - 1]:
                    continue
                o, po = _xyz(o_zyx), corg[parent]
                cn = L[lev - 1]["patches"][parent][0]
                for d in range(3):
                    a_, b_ = [e for e in range(3) if e != d]
                    ga0, gb0 = po[a_] + o[a_], po[b_] + o[b_]  # the face's first coarse cell, global
                    for side, plane in ((-1, o[d]), (+1, o[d] + sz)):
                        cell = o[d] - 1 if side < 0 else o[d] + sz
                        if 0 <= cell < cn[d]:
                            found = [(parent, ga0, ga0 + sz, gb0, gb0 + sz)]
                        else:
                            gd = (po[d] + cell) % dom
                            found = []
                            for q, (qo, qs) in enumerate(zip(corg, csz)):
                                if not qo[d] <= gd < qo[d] + qs:
                                    continue
                                a0, a1 = max(ga0, qo[a_]), min(ga0 + sz, qo[a_] + qs)
                                b0, b1 = max(gb0, qo[b_]), min(gb0 + sz, qo[b_] + qs)
                                if a0 < a1 and b0 < b1:
                                    found.append((q, a0, a1, b0, b1))
                            self.unmatched_faces += sz * sz - sum((a1 - a0) * (b1 - b0)
                                                                  for (_, a0, a1, b0, b1) in found)
                        pieces = []
                        for q, a0, a1, b0, b1 in found:
                            self.windows[lev - 1].append((loc[lev - 1][parent], d, plane, a0 - po[a_], a1 - po[a_],
                                                          b0 - po[b_], b1 - po[b_], -1.0, off))
                            pieces.append((off, q, a0, a1, b0, b1))
                            off += 9 * (a1 - a0) * (b1 - b0)
                        self.coarse_dst[lev][(fi, d, side)] = pieces
            self.reg_range[lev] = (r0, off)
        self.nreg = off

    def _level_ops(self, domain):
        """Descriptor tables of the level operators: per level the same-level
        exchange boxes (ghosts over a sibling's interior or a periodic image
        of one); per level l >= 1 the prolongation boxes (the ghost cells no
        sibling covers: the coarse-fine boundary), the restriction boxes (every
        patch's footprint) and the reflux sets (one per piece of every coarse
        window: the coarse cells beside every fine patch face, in the parent
        or in the coarse patch across the parent's boundary)."""
        from . import exchange as X
        L = self.levels
        xunc = {}
        for lev, lv in enumerate(L):
            specs = [((o[2], o[1], o[0]), (sz_, sz_, sz_), p_[2]) for (o, sz_), p_ in zip(lv["origins"], lv["patches"])]
            xb = X.plan(specs, [domain * RATIO ** lev] * 3, [True] * 3, 3)
            xunc[lev] = X.uncovered(xb, len(specs), [sp[1] for sp in specs], 3)
            if xb:
                self.xch[lev] = ctu.make_copy_boxes(xb)
        ops = {}
        for lev in range(1, len(L)):
            pb, rb, fs = [], [], []
            dom = domain * RATIO ** (lev - 1)
            corg = [_xyz(o) for (o, _) in L[lev - 1]["origins"]]
            for fi, (n, dx, base, *_rest) in enumerate(L[lev]["patches"]):
                parent, o_zyx, sz = L[lev]["footprints"][fi]
                cn, cdx, cbase = L[lev - 1]["patches"][parent][:3]
                o = _xyz(o_zyx)
                for lo_, hi_ in xunc[lev][fi]:
                    pb.append(dict(fn=n, cn=cn, fbase=base, cbase=cbase, lo=lo_, hi=hi_, origin=o, ratio=RATIO))
                rb.append(dict(fn=n, cn=cn, fbase=base, cbase=cbase, lo=o, hi=[o[e] + sz for e in range(3)],
                               origin=o, ratio=RATIO))
                po = corg[parent]
                for d in range(3):
                    a_, b_ = [e for e in range(3) if e != d]
                    ga0, gb0 = po[a_] + o[a_], po[b_] + o[b_]
                    for side, fplane in ((-1, 0), (+1, n[d])):
                        # the corrected coarse cells' layer, global
                        gd = (po[d] + (o[d] - 1 if side < 0 else o[d] + sz)) % dom
                        for creg, q, a0, a1, b0, b1 in self.coarse_dst[lev][(fi, d, side)]:
                            qn, qdx, qbase = L[lev - 1]["patches"][q][:3]
                            qo = corg[q]
                            cq = gd - qo[d]  # that layer in patch q
                            fs.append(dict(cn=qn, dir=d, plane=cq if side > 0 else cq + 1, side=side, cbase=qbase,
                                           dx=qdx, a0=a0 - qo[a_], a1=a1 - qo[a_], b0=b0 - qo[b_],
                                           b1=b1 - qo[b_], creg=creg, freg=self.fine_dst[lev][(fi, d, fplane)],
                                           fa0=RATIO * (a0 - ga0), fb0=RATIO * (b0 - gb0), fna=n[a_], fnb=n[b_],
                                           ratio=RATIO))
            ops[lev] = (ctu.make_level_boxes(pb), ctu.make_level_boxes(rb), ctu.make_reflux_sets(fs))
        self.ops = ops


class LevelAdvance:
    """The state and the launch plan of a hierarchy's coarse step.

    levels: per level, a dict with
      "patches": [(n, dx, base, ...)], n the interior cells (x, y, z), dx the
                 cell widths, base the pool offset of the patch's first
                 ghosted cell (4 ghost layers per side);
      "pool":    (9, cells) float64 host array, the level's patches;
      "origins": [(o_zyx, size)], every patch's first interior cell in the
                 level's index space (z, y, x) and its (cubic) size;
      "footprints" (levels >= 1): [(parent, o_zyx, size)], the patch's parent
                 on the level below and its footprint there in parent cells.
    domain: level 0's cells per side of the periodic box (level l: domain
            times 2^l).
    precision: ctu.CTU_MIXED or ctu.CTU_FP64; the parabolic coefficients
            (kappa, kappa_par, tc_phi, nu, eta) as in ctu.make_config.

    After construction: A[l], B[l] (the level's two device pools; a coarse
    step reads A and leaves level l's result in outputs()[l]), P[l] (this
    rank's patch list, None when it has none), D[l] (dt_l and c_h on the
    device, set by set_dt), ctxs[l], reg (the flux registers), plan (the
    LevelPlan) and its windows, reg_range, xch and ops.
    """

    def __init__(self, levels, domain, *, precision, cfl=0.3, mine=None, level_ops=True, device=None,
                 kappa=0.0, kappa_par=0.0, tc_phi=0.0, nu=0.0, eta=0.0):
        import torch
        L = levels
        self.levels = L
        self.nlev = len(L)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        plan = LevelPlan(L, domain, mine=mine, level_ops=level_ops)
        self.plan = plan
        self.mine, self.windows, self.reg_range = plan.mine, plan.windows, plan.reg_range
        self.ops, self.xch = plan.ops, plan.xch
        mine = plan.mine
        self.reg = torch.zeros(max(plan.nreg, 1), dtype=torch.float64, device=dev)
        self.ctxs, self.A, self.B, self.P, self.D = [], [], [], [], []
        for lev, lv in enumerate(L):
            c = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=precision, cfl=cfl, kappa=kappa,
                                        nu=nu, eta=eta, kappa_par=kappa_par, tc_phi=tc_phi))
            pool = torch.from_numpy(lv["pool"]).to(dev)
            self.A.append(pool)
            self.B.append(pool.clone())
            self.P.append(ctu.make_patches([lv["patches"][gi][:3] for gi in mine[lev]]) if mine[lev] else None)
            if self.windows[lev]:
                c.flux_registers(self.reg, self.windows[lev])
            self.ctxs.append(c)
            self.D.append(torch.zeros(2, dtype=torch.float64, device=dev))

    # ------------------------------------------------------------ time step

    def local_dt(self):
        """dt_0 that this rank's patches allow: the smallest over the levels
        of 2^l times the level's ctu_dt (Eq. Ca)."""
        import torch
        h = []
        for lev, c in enumerate(self.ctxs):
            if self.P[lev] is None:
                continue
            hd = torch.zeros(2, dtype=torch.float64, device=self.device)
            c.dt(self.A[lev], self.A[lev].shape[1], self.P[lev], hd)
            h.append(hd.cpu().tolist()[0] * RATIO ** lev)
        return min(h) if h else float("inf")

    def set_dt(self, dt0, ch):
        """dt_l = dt_0 / 2^l and the common c_h, written in place (a captured
        coarse step reads them from the same device arrays)."""
        import torch
        for lev in range(self.nlev):
            self.D[lev].copy_(torch.tensor([dt0 / RATIO ** lev, ch], dtype=torch.float64))

    # ------------------------------------------------------------ coarse step

    def _step(self, lev, src, dst, stream):
        if self.P[lev] is not None:
            self.ctxs[lev].step(src, dst, src.shape[1], self.P[lev], self.D[lev], stream=stream)

    def _exchange(self, lev, U, stream):
        if lev in self.xch:
            self.ctxs[lev].copy(U, U.shape[1], U, U.shape[1], self.xch[lev], stream=stream)

    def _ghosts(self, lev, pold, pnew, alpha, U, stream):
        """Ghosts of level lev's state U: prolongation from the parent's
        states pold, pnew at alpha (Eq. intalpha), then the exchange."""
        if len(self.ops[lev][0]):
            self.ctxs[lev].prolong(pold, pnew, pold.shape[1], alpha, U, U.shape[1], self.ops[lev][0],
                                   stream=stream)
        self._exchange(lev, U, stream)

    def _sync(self, lev, parent_new, fine_latest, stream):
        """Reflux level lev - 1, restrict level lev into it, clear the
        interface's registers."""
        _, rb, fs = self.ops[lev]
        c = self.ctxs[lev - 1]
        if len(fs):
            c.reflux(parent_new, parent_new.shape[1], self.reg, fs, stream=stream)
        if len(rb):
            c.restrict(parent_new, parent_new.shape[1], fine_latest, fine_latest.shape[1], rb, stream=stream)
        r0, r1 = self.reg_range[lev]
        self.reg[r0:r1].zero_()

    def _substeps(self, lev, pold, pnew, stream):
        """The two substeps of level lev within one substep of its parent
        (old and new parent states pold, pnew); the level's result is back in
        A[lev]."""
        ops = self.ops is not None
        A, B = self.A, self.B
        for k in range(RATIO):
            s, d = (A[lev], B[lev]) if k % 2 == 0 else (B[lev], A[lev])
            if ops:
                self._ghosts(lev, pold, pnew, k / RATIO, s, stream)
            self._step(lev, s, d, stream)
            if lev + 1 < self.nlev:
                if ops:  # the new state, which the finer level prolongs from
                    self._ghosts(lev, pold, pnew, (k + 1) / RATIO, d, stream)
                self._substeps(lev + 1, s, d, stream)
                if ops:
                    self._sync(lev + 1, d, A[lev + 1], stream)

    def coarse_step(self, stream):
        """One coarse step, every launch on `stream` (capturable in a CUDA
        graph once the descriptor tables are on the device, that is after one
        call outside the capture): level 0 from A[0] into B[0], then every
        finer level subcycled and synchronised."""
        ops = self.ops is not None
        if ops:
            self._exchange(0, self.A[0], stream)
        self._step(0, self.A[0], self.B[0], stream)
        if ops:
            self._exchange(0, self.B[0], stream)
        if self.nlev > 1:
            self._substeps(1, self.A[0], self.B[0], stream)
            if ops:
                self._sync(1, self.B[0], self.A[1], stream)

    def outputs(self):
        """Where a coarse step leaves each level's result."""
        return [self.B[0]] + [self.A[lev] for lev in range(1, self.nlev)]

    def launches(self):
        """The library's kernel launches in one coarse step (the registers'
        zeroing is a torch fill, not counted)."""
        n = sum(RATIO ** lev * self.ctxs[lev].launches() for lev in range(self.nlev) if self.P[lev] is not None)
        if self.ops is None:
            return n
        n += 2 * (0 in self.xch)
        for lev in range(1, self.nlev):
            pb, rb, fs = self.ops[lev]
            fills = RATIO ** lev * (2 if lev + 1 < self.nlev else 1)  # before each substep, and new states
            n += fills * ((len(pb) > 0) + (lev in self.xch))
            syncs = RATIO ** (lev - 1)  # reflux: one launch per class of sets (direction, side)
            n += syncs * (len({(S.dir, S.side) for S in fs}) + (len(rb) > 0))
        return n

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []
