"""The level operators of the CUDA path (ctu_prolong, ctu_restrict,
ctu_reflux) against the oracle's, element by element, and a two-level
hierarchy advanced on the GPU that conserves its totals to round-off."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch.device("cuda:0")


def _pool(arrays):
    bases, base = [], 0
    for A in arrays:
        bases.append(base)
        base += A[0].size + 13
    P = np.zeros((9, base))
    for A, b in zip(arrays, bases):
        P[:, b:b + A[0].size] = A.reshape(9, -1)
    return P, bases


def _box(fn, cn, fbase, cbase, lo, hi, origin, r):
    return dict(fn=fn, cn=cn, fbase=fbase, cbase=cbase, lo=lo, hi=hi, origin=origin, ratio=r)


@pytest.mark.parametrize("ndim,r", [(3, 2), (2, 2), (3, 3)])
def test_prolong_and_restrict_match_the_oracle(ndim, r):
    import torch
    from paper_1110_0740_gb300 import ctu
    rng = np.random.default_rng(ndim + 10 * r)
    nc = [12 if d < ndim else 1 for d in range(3)]
    nf = [(8 if d < ndim else 1) for d in range(3)]
    nf2 = [(6 if d < ndim else 1) for d in range(3)]
    Uo = rng.standard_normal(O.shape(nc, ndim)) + 3.0
    Un = rng.standard_normal(O.shape(nc, ndim)) + 3.0
    F1 = np.zeros(O.shape(nf, ndim))
    F2 = np.zeros(O.shape(nf2, ndim))
    (CP, cb), (FP, fb) = _pool([Uo]), _pool([F1, F2])
    CPn, _ = _pool([Un])
    g = O.ghosts(ndim)
    o1 = [3 if d < ndim else 0 for d in range(3)]
    o2 = [5 if d < ndim else 0 for d in range(3)]
    alpha = 0.625
    # fine patch 1: whole ghosted box; fine patch 2: the lower ghost slab along x and an interior box
    boxes = [_box(nf, nc, fb[0], cb[0], [-g[d] for d in range(3)], [nf[d] + g[d] for d in range(3)], o1, r),
             _box(nf2, nc, fb[1], cb[0], [-4, -g[1], -g[2]], [0, nf2[1] + g[1], nf2[2] + g[2]], o2, r),
             _box(nf2, nc, fb[1], cb[0], [1, 0, 0], [nf2[0] - 1, nf2[1], nf2[2]], o2, r)]
    dev = _dev()
    tC, tCn, tF = (torch.from_numpy(a).to(dev) for a in (CP, CPn, FP))
    ctx = ctu.Ctx(ctu.make_config(ndim=ndim, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64))
    ctx.prolong(tC, tCn, CP.shape[1], alpha, tF, FP.shape[1], ctu.make_level_boxes(boxes))
    got = tF.cpu().numpy()
    ref1, ref2 = F1.copy(), F2.copy()
    O.prolong(Uo, Un, nc, alpha, ref1, nf, boxes[0]["lo"], boxes[0]["hi"], o1, r, ndim)
    O.prolong(Uo, Un, nc, alpha, ref2, nf2, boxes[1]["lo"], boxes[1]["hi"], o2, r, ndim)
    O.prolong(Uo, Un, nc, alpha, ref2, nf2, boxes[2]["lo"], boxes[2]["hi"], o2, r, ndim)
    for ref, b in ((ref1, fb[0]), (ref2, fb[1])):
        G = got[:, b:b + ref[0].size].reshape(ref.shape)
        assert np.allclose(G, ref, rtol=1e-14, atol=1e-14), np.abs(G - ref).max()
    # restriction of fine patch 1 onto the coarse cells it covers
    cover_hi = [o1[d] + (nf[d] // r if d < ndim else 1) for d in range(3)]
    rbox = [_box(nf, nc, fb[0], cb[0], o1, cover_hi, o1, r)]
    tC2 = tC.clone()
    ctx.restrict(tC2, CP.shape[1], tF, FP.shape[1], ctu.make_level_boxes(rbox))
    refc = Uo.copy()
    O.restrict(refc, nc, ref1, nf, o1, cover_hi, o1, r, ndim)
    G = tC2.cpu().numpy()[:, cb[0]:cb[0] + Uo[0].size].reshape(Uo.shape)
    assert np.allclose(G, refc, rtol=1e-14, atol=1e-14)
    assert ctx.status_sync() == 0


@pytest.mark.parametrize("ndim", [2, 3])
def test_prolong_one_sided_at_the_domain_boundary(ndim):
    """A coarse patch whose cells touch the domain boundary on both sides of
    every active axis (phys bits), NaN beyond the boundary: the one-sided
    slopes read no ghost and the fine cells equal the oracle's bit for bit
    (up to 1e-14); a box with mixed bits (lower x and upper y only) as well;
    bits above 5 are refused."""
    import torch
    from paper_1110_0740_gb300 import ctu
    rng = np.random.default_rng(40 + ndim)
    nc = [6 if d < ndim else 1 for d in range(3)]
    nf = [12 if d < ndim else 1 for d in range(3)]
    U = rng.standard_normal(O.shape(nc, ndim)) + 3.0
    g = O.ghosts(ndim)
    inside = np.zeros(U.shape[1:], dtype=bool)
    inside[tuple(slice(g[d], g[d] + nc[d]) for d in (2, 1, 0))] = True
    U[:, ~inside] = np.nan
    F = np.zeros(O.shape(nf, ndim))
    (CP, cb), (FP, fb) = _pool([U]), _pool([F])
    dev = _dev()
    tC, tF = torch.from_numpy(CP).to(dev), torch.from_numpy(FP).to(dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=ndim, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64))
    # every side flagged, NaN beyond the boundary; then only the lower x and
    # upper y sides flagged, with finite ghosts (the other sides keep the MC
    # central slope, which needs its ghost)
    Ufin = U.copy()
    Ufin[:, ~inside] = rng.standard_normal(int((~inside).sum()))[None, :] + 3.0
    CPf, _ = _pool([Ufin])
    for phys, Uc, cpool in ((sum(3 << (2 * d) for d in range(ndim)), U, tC),
                            (0b1001, Ufin, torch.from_numpy(CPf).to(dev))):
        box = _box(nf, nc, fb[0], cb[0], [0, 0, 0], nf, [0, 0, 0], 2)
        box["phys"] = phys
        tF.zero_()
        ctx.prolong(cpool, cpool, CP.shape[1], 0.0, tF, FP.shape[1], ctu.make_level_boxes([box]))
        got = tF.cpu().numpy()[:, fb[0]:fb[0] + F[0].size].reshape(F.shape)
        ref = F.copy()
        O.prolong(Uc, Uc, nc, 0.0, ref, nf, [0, 0, 0], nf, [0, 0, 0], 2, ndim, phys=phys)
        I, R = O.interior(got, nf, ndim), O.interior(ref, nf, ndim)
        assert np.all(np.isfinite(I)) and np.all(np.isfinite(R))
        assert np.allclose(I, R, rtol=1e-14, atol=1e-14), np.abs(I - R).max()
    bad = _box(nf, nc, fb[0], cb[0], [0, 0, 0], nf, [0, 0, 0], 2)
    bad["phys"] = 64
    with pytest.raises(ctu.CtuError):
        ctx.prolong(tC, tC, CP.shape[1], 0.0, tF, FP.shape[1], ctu.make_level_boxes([bad]))
    assert ctx.status_sync() == 0


def test_level_operators_reject_boxes_outside_the_patches():
    import torch
    from paper_1110_0740_gb300 import ctu
    nc, nf = [8, 8, 8], [8, 8, 8]
    dev = _dev()
    C = torch.zeros((9, 16 ** 3), dtype=torch.float64, device=dev)
    F = torch.zeros((9, 16 ** 3), dtype=torch.float64, device=dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64))
    bad = [_box(nf, nc, 0, 0, [-5, 0, 0], [8, 8, 8], [2, 2, 2], 2),     # fine box beyond the ghosts
           _box(nf, nc, 0, 0, [-4, -4, -4], [12, 12, 12], [6, 2, 2], 2),  # coarse neighbour out of range
           _box(nf, nc, 1, 0, [0, 0, 0], [8, 8, 8], [2, 2, 2], 2)]      # fine patch beyond the pool
    for b in bad:
        with pytest.raises(ctu.CtuError):
            ctx.prolong(C, C.clone(), C.shape[1], 0.0, F, F.shape[1], ctu.make_level_boxes([b]))
    with pytest.raises(ctu.CtuError):
        ctx.restrict(C, C.shape[1], F, F.shape[1],
                     ctu.make_level_boxes([_box(nf, nc, 0, 0, [0, 0, 0], [8, 8, 8], [0, 0, 0], 2)]))


@pytest.mark.parametrize("par", [{}, dict(kappa=0.002, kappa_par=0.006, nu=0.001, eta=0.001)])
def test_two_level_hierarchy_on_the_gpu_conserves_and_matches_the_oracle(par):
    """Coarse 32^2 periodic patch (flux registers, weight -1, on the four
    coarse faces of the interface) and a 32^2 fine patch (ratio 2, weight +1
    registers on its boundary) advanced in FP64 on the GPU: ctu_step on both
    levels (two fine substeps with ghosts from ctu_prolong at alpha = 0, 1/2),
    ctu_restrict, ctu_reflux.  The result matches the same sequence in the
    oracle and conserves mass, momentum, energy and magnetic flux, also with
    the parabolic terms (whose fluxes the registers carry)."""
    import torch
    from paper_1110_0740_gb300 import ctu
    Nc = 32
    nc = [Nc, Nc, 1]
    hc, hf = 1.0 / Nc, 0.5 / Nc
    U = W.mhd_turb_2d(Nc, seed=6)
    O.fill_periodic(U, nc, 2)
    lo, hi = 8, 24
    nfc = hi - lo
    nf = [2 * nfc, 2 * nfc, 1]
    total0 = O.interior(U, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    cw, sets, off = [], [], 0
    for d in (0, 1):
        for side, f in ((-1, lo), (+1, hi)):
            cw.append((0, d, f, lo, hi, 0, 1, -1.0, off))
            sets.append((d, f, side, off))
            off += 9 * nfc
    fw = []
    for d in (0, 1):
        a_ = 1 - d
        for plane in (0, nf[d]):
            fw.append((0, d, plane, 0, nf[a_], 0, 1, 1.0, off))
            off += 9 * nf[a_]
    rate = (O.mhd_max_rate(U, nc, 2, [hc, hc], 5.0 / 3.0, **par) if par else O.mhd_max_speed(U, nc, 2, [hc, hc]))
    dt, ch = O.dt_ch(rate, [hc, hc], 2, 0.4)
    origin = [lo, lo, 0]
    dev = _dev()
    # ---- GPU
    Uf0 = np.zeros(O.shape(nf, 2))
    tUc = torch.from_numpy(U.reshape(9, -1).copy()).to(dev)
    tUcn = torch.zeros_like(tUc)
    tUf = torch.from_numpy(Uf0.reshape(9, -1)).to(dev)
    tUfn = torch.zeros_like(tUf)
    reg = torch.zeros(off, dtype=torch.float64, device=dev)
    cfg = ctu.make_config(ndim=2, recon=ctu.CTU_LINEAR_MC, precision=ctu.CTU_FP64, cfl=0.4, **par)
    cc, cf = ctu.Ctx(cfg), ctu.Ctx(cfg)
    cc.flux_registers(reg, cw)
    cf.flux_registers(reg, fw)
    Pc = ctu.make_patches([(nc, [hc, hc, 1.0], 0)])
    Pf = ctu.make_patches([(nf, [hf, hf, 1.0], 0)])
    dtc = torch.tensor([dt, ch], dtype=torch.float64, device=dev)
    dtf = torch.tensor([dt / 2, ch], dtype=torch.float64, device=dev)
    cc.step(tUc, tUcn, tUc.shape[1], Pc, dtc)
    full = ctu.make_level_boxes([_box(nf, nc, 0, 0, [-4, -4, 0], [nf[0] + 4, nf[1] + 4, 1], origin, 2)])
    shells = ctu.make_level_boxes([_box(nf, nc, 0, 0, l, h, origin, 2) for l, h in (
        ([-4, -4, 0], [0, nf[1] + 4, 1]), ([nf[0], -4, 0], [nf[0] + 4, nf[1] + 4, 1]),
        ([0, -4, 0], [nf[0], 0, 1]), ([0, nf[1], 0], [nf[0], nf[1] + 4, 1]))])
    cf.prolong(tUc, tUcn, tUc.shape[1], 0.0, tUf, tUf.shape[1], full)
    for q in range(2):
        cf.step(tUf, tUfn, tUf.shape[1], Pf, dtf)
        tUf.copy_(tUfn)
        cf.prolong(tUc, tUcn, tUc.shape[1], (q + 1) / 2, tUf, tUf.shape[1], shells)
    cc.restrict(tUcn, tUcn.shape[1], tUf, tUf.shape[1],
                ctu.make_level_boxes([_box(nf, nc, 0, 0, [lo, lo, 0], [hi, hi, 1], origin, 2)]))
    rsets = []
    fwin = {(w[1], w[2]): w for w in fw}
    for d, f, side, creg in sets:
        w = fwin[(d, 0 if side < 0 else nf[d])]
        rsets.append(dict(cn=nc, dir=d, plane=f, side=side, cbase=0, dx=[hc, hc, 1.0], a0=lo, a1=hi, b0=0, b1=1,
                          creg=creg, freg=w[8], fa0=0, fb0=0, fna=w[4] - w[3], fnb=1, ratio=2))
    cc.reflux(tUcn, tUcn.shape[1], reg, ctu.make_reflux_sets(rsets))
    assert cc.status_sync() == 0 and cf.status_sync() == 0
    got = tUcn.cpu().numpy().reshape(U.shape)
    total = O.interior(got, nc, 2).sum(axis=(1, 2, 3)) * hc * hc
    scale = np.abs(O.interior(got, nc, 2)).sum(axis=(1, 2, 3)) * hc * hc
    assert np.all(np.abs(total - total0)[:8] <= 1e-13 * scale[:8]), total - total0
    # ---- oracle, same sequence
    regr = np.zeros(off)
    cw_o = [(d, f, a0, a1, b0, b1, dst, wgt) for (_, d, f, a0, a1, b0, b1, wgt, dst) in cw]
    fw_o = [(d, pl, a0, a1, b0, b1, dst, wgt) for (_, d, pl, a0, a1, b0, b1, wgt, dst) in fw]
    Ucn, bad = O.mhd_step(U, nc, 2, [hc, hc, 1], dt, ch, recon=0, windows=cw_o, reg=regr, **par)
    Uf = np.zeros(O.shape(nf, 2))
    O.prolong(U, Ucn, nc, 0.0, Uf, nf, [-4, -4, 0], [nf[0] + 4, nf[1] + 4, 1], origin, 2, 2)
    for q in range(2):
        Uf, bad = O.mhd_step(Uf, nf, 2, [hf, hf, 1], dt / 2, ch, recon=0, windows=fw_o, reg=regr, **par)
        for b in shells:
            O.prolong(U, Ucn, nc, (q + 1) / 2, Uf, nf, list(b.lo), list(b.hi), origin, 2, 2)
    O.restrict(Ucn, nc, Uf, nf, [lo, lo, 0], [hi, hi, 1], origin, 2, 2)
    for s_ in rsets:
        O.reflux(Ucn, nc, [hc, hc], regr, s_["dir"], s_["plane"], s_["side"], s_["a0"], s_["a1"], s_["b0"],
                 s_["b1"], s_["creg"], s_["freg"], 0, 0, s_["fna"], 1, 2, 2)
    err = np.abs(O.interior(got, nc, 2) - O.interior(Ucn, nc, 2)).sum(axis=(1, 2, 3))
    ref = np.abs(O.interior(Ucn, nc, 2)).sum(axis=(1, 2, 3))
    assert np.all(err[:8] <= 1e-11 * ref[:8]), err / np.maximum(ref, 1e-300)



def test_reflux_is_reproducible_where_interfaces_meet():
    """Two disjoint fine boxes in an L (ratio 2, 3D) on a 16^3 coarse patch:
    the 4 coarse cells at the inner corner border the +x face of one and the
    +y face of the other, so each takes two corrections.  ctu_reflux applies
    them class by class (direction, then side), so the result is the same bit
    for bit whatever the order of the sets, and matches the oracle applying
    the same corrections in that order (Eq. fluxcorr, Eq. addreflux)."""
    import torch
    from paper_1110_0740_gb300 import ctu
    nc = [16, 16, 16]
    h = 1.0 / 16
    rng = np.random.default_rng(17)
    U = rng.standard_normal(O.shape(nc, 3))
    # (dir, plane, side, (a0, a1), (b0, b1)); a, b = the two other axes in order
    faces = [(0, 4, -1, (4, 12), (4, 8)), (0, 8, +1, (8, 12), (4, 8)), (1, 4, -1, (4, 8), (4, 8)),
             (1, 12, +1, (4, 8), (4, 8)), (2, 4, -1, (4, 8), (4, 12)), (2, 8, +1, (4, 8), (4, 12)),
             (0, 12, +1, (4, 8), (4, 8)), (1, 4, -1, (8, 12), (4, 8)), (1, 8, +1, (8, 12), (4, 8)),
             (2, 4, -1, (8, 12), (4, 8)), (2, 8, +1, (8, 12), (4, 8))]
    sets, off = [], 0
    for d, plane, side, (a0, a1), (b0, b1) in faces:
        na, nb = a1 - a0, b1 - b0
        creg, freg = off, off + 9 * na * nb
        off = freg + 9 * (2 * na) * (2 * nb)
        sets.append(dict(cn=nc, dir=d, plane=plane, side=side, cbase=0, dx=[h] * 3, a0=a0, a1=a1, b0=b0, b1=b1,
                         creg=creg, freg=freg, fa0=0, fb0=0, fna=2 * na, fnb=2 * nb, ratio=2))
    reg = rng.standard_normal(off)
    dev = _dev()
    treg = torch.from_numpy(reg).to(dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64, cfl=0.3))
    perm = rng.permutation(len(sets))
    got = []
    for order in (list(range(len(sets))), list(reversed(range(len(sets)))), list(perm)):
        tU = torch.from_numpy(U.reshape(9, -1).copy()).to(dev)
        ctx.reflux(tU, tU.shape[1], treg, ctu.make_reflux_sets([sets[i] for i in order]))
        assert ctx.status_sync() == 0
        got.append(tU.cpu().numpy().reshape(U.shape))
    ctx.close()
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[2])
    R = U.copy()
    for S in sorted(sets, key=lambda S: (S["dir"], S["side"])):
        O.reflux(R, nc, [h] * 3, reg, S["dir"], S["plane"], S["side"], S["a0"], S["a1"], S["b0"], S["b1"],
                 S["creg"], S["freg"], 0, 0, S["fna"], S["fnb"], 2, 3)
    g = O.ghosts(3)
    corner = (slice(None), slice(g[2] + 4, g[2] + 8), g[1] + 8, g[0] + 8)
    assert np.all(R[corner] != U[corner])  # both corrections reached the corner cells
    assert np.all(np.abs(got[0] - R) <= 1e-13 * (1.0 + np.abs(R)))


def test_diagnostics_match_the_oracle():
    """ctu_diagnostics over a batch of uneven patches: the conserved totals
    are the sums of the oracle's per-patch totals and the largest |div B| is
    the largest of theirs."""
    import torch
    from paper_1110_0740_gb300 import ctu
    shapes = [(16, 12, 8), (8, 8, 8), (24, 5, 7)]
    dxs = [(0.05, 0.07, 0.06), (0.1, 0.1, 0.1), (1 / 24, 0.2, 0.1)]
    src = W.mhd_blast_3d(32, seed=3, kmax=3)
    arrays = [np.ascontiguousarray(src[:, :n[2] + 8, :n[1] + 8, :n[0] + 8]) for n in shapes]
    P, bases = _pool(arrays)
    dev = _dev()
    U = torch.from_numpy(P).to(dev)
    out = torch.zeros(10, dtype=torch.float64, device=dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_MIXED))
    ctx.diagnostics(U, P.shape[1], ctu.make_patches([(n, dx, b) for n, dx, b in zip(shapes, dxs, bases)]), out)
    got = out.cpu().numpy()
    ref = [O.diagnostics(A, list(n), 3, list(dx)) for A, n, dx in zip(arrays, shapes, dxs)]
    tot = np.sum([r[:9] for r in ref], axis=0)
    scale = np.sum([np.abs(r[:9]) for r in ref], axis=0) + 1e-300
    assert np.all(np.abs(got[:9] - tot) <= 1e-13 * scale), (got[:9], tot)
    assert got[9] == pytest.approx(max(r[9] for r in ref), rel=1e-14)
    assert ctx.status_sync() == 0
