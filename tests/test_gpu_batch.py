"""Batched patches, flux registers, full-size sampled parity and status
flags of the CUDA path, against the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import l1rel, maxrel

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


def _dev():
    import torch
    return torch.device("cuda:0")


def test_batch_of_uneven_patches_and_registers():
    """Five patches of different shapes (one with a single interior cell
    along y, one with a different dx) in one ctu_step call, flux-register
    windows on every boundary face plus an interior plane; each patch and
    each register matches the oracle run patch by patch."""
    import torch
    from paper_1110_0740_gb300 import ctu
    shapes = [(16, 16, 16), (8, 8, 8), (11, 1, 7), (24, 9, 5), (3, 3, 3)]
    dxs = [(1 / 16,) * 3, (1 / 8,) * 3, (0.05, 0.07, 0.06), (1 / 24, 1 / 24, 1 / 24), (0.1,) * 3]
    src = W.mhd_blast_3d(40, seed=21, kmax=3)
    arrays, bases, base = [], [], 0
    for i, n in enumerate(shapes):
        A = np.zeros(O.shape(list(n), 3))
        g = src[:, 2 * i:2 * i + n[2] + 8, i:i + n[1] + 8, 3 * i:3 * i + n[0] + 8]
        A[:] = g
        arrays.append(A)
        bases.append(base)
        base += A[0].size + 17  # ragged gaps between patches
    stride = base
    pool = np.zeros((9, stride))
    for A, b in zip(arrays, bases):
        pool[:, b:b + A[0].size] = A.reshape(9, -1)
    windows, off = [], 0
    per_patch = []
    for p, n in enumerate(shapes):
        ws = []
        for d in range(3):
            a_, b_ = [e for e in range(3) if e != d]
            for plane in sorted({0, n[d] // 2, n[d]}):
                windows.append((p, d, plane, 0, n[a_], 0, n[b_], 0.5 + p, off))
                ws.append((d, plane, 0, n[a_], 0, n[b_], off, 0.5 + p))
                off += 9 * n[a_] * n[b_]
        per_patch.append(ws)
    dev = _dev()
    U = torch.from_numpy(pool).to(dev)
    Uo = torch.zeros_like(U)
    reg = torch.zeros(off, dtype=torch.float64, device=dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_FP64, cfl=0.3))
    patches = ctu.make_patches([(n, dx, b) for n, dx, b in zip(shapes, dxs, bases)])
    ctx.flux_registers(reg, windows)
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.dt(U, stride, patches, dtch)
    ctx.step(U, Uo, stride, patches, dtch)
    ctx.step(U, Uo, stride, patches, dtch)  # registers accumulate over calls
    assert ctx.status_sync() == 0
    dt, ch = dtch.cpu().tolist()
    # dt over the whole batch
    m = max(O.mhd_max_speed(A, list(n), 3, list(dx)) for A, n, dx in zip(arrays, shapes, dxs))
    dt_ref, ch_ref = O.dt_ch(m, [min(min(d) for d in dxs)] * 3, 3, 0.3)
    assert abs(dt - dt_ref) <= 1e-14 * dt_ref and abs(ch - ch_ref) <= 1e-14 * ch_ref
    out = Uo.cpu().numpy()
    regs = reg.cpu().numpy()
    ref_reg = np.zeros(off)
    for A, n, dx, b, ws in zip(arrays, shapes, dxs, bases, per_patch):
        R, bad = O.mhd_step(A, list(n), 3, list(dx), dt, ch, recon=1, windows=ws, reg=ref_reg)
        O.mhd_step(A, list(n), 3, list(dx), dt, ch, recon=1, windows=ws, reg=ref_reg)
        G = out[:, b:b + A[0].size].reshape(A.shape)
        e = l1rel(O.interior(G, list(n), 3), O.interior(R, list(n), 3), ch)
        assert np.all(e <= TOL64), (n, e)
        em = maxrel(O.interior(G, list(n), 3), O.interior(R, list(n), 3), ch)
        assert np.all(em <= TOL64), (n, em)
    scale = np.abs(ref_reg).max()
    assert np.abs(regs - ref_reg).max() <= 1e-12 * scale


def test_full_size_sampled_parity_256():
    """The bench workload (256^3, PPM, mixed and FP64, the bench's launch
    configuration: autotuned tiles for the mixed path): one GPU step, then 6
    sampled 6^3 blocks recomputed by the oracle from their own ghosted
    neighbourhood of the same input."""
    import torch
    from paper_1110_0740_gb300 import ctu
    n = 256
    U0 = W.mhd_blast_3d(n, seed=0)
    dev = _dev()
    U = torch.from_numpy(U0.reshape(9, -1)).to(dev)
    Uo = torch.zeros_like(U)
    stride = U.shape[1]
    patches = ctu.make_patches([([n] * 3, [1.0 / n] * 3, 0)])
    rng = np.random.default_rng(5)
    corners = [rng.integers(0, n - 6, size=3) for _ in range(5)] + [np.array([0, 0, n - 6])]
    for prec, tol in ((ctu.CTU_FP64, TOL64), (ctu.CTU_MIXED, 2e-5)):
        ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3))
        dtch = torch.zeros(2, dtype=torch.float64, device=dev)
        ctx.dt(U, stride, patches, dtch)
        if prec == ctu.CTU_MIXED:  # the bench's tiles
            ctx.autotune(U, Uo, stride, patches, dtch)
        ctx.step(U, Uo, stride, patches, dtch)
        assert ctx.status_sync() == 0
        dt, ch = dtch.cpu().tolist()
        G = Uo.view(9, n + 8, n + 8, n + 8)
        for c in corners:
            k, j, i = int(c[2]), int(c[1]), int(c[0])
            blk = U0[:, k:k + 14, j:j + 14, i:i + 14].copy()
            R, bad = O.mhd_step(blk, [6, 6, 6], 3, [1.0 / n] * 3, dt, ch, recon=1)
            assert bad == 0
            got = G[:, k + 4:k + 10, j + 4:j + 10, i + 4:i + 10].cpu().numpy()
            e = l1rel(got, O.interior(R, [6, 6, 6], 3), ch)
            assert np.all(e <= tol), (prec, c, e)
            em = maxrel(got, O.interior(R, [6, 6, 6], 3), ch)
            assert np.all(em <= tol), (prec, c, em)
        ctx.close()


def test_negative_density_sets_status_flag():
    import torch
    from paper_1110_0740_gb300 import ctu
    n = [8, 8, 8]
    U0 = W.mhd_blast_3d(8, seed=1, kmax=2)
    U0[0, 6, 6, 6] = -1.0
    dev = _dev()
    U = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
    Uo = torch.zeros_like(U)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, precision=ctu.CTU_FP64))
    patches = ctu.make_patches([(n, [1 / 8] * 3, 0)])
    dtch = torch.tensor([1e-3, 1.0], dtype=torch.float64, device=dev)
    ctx.step(U, Uo, U.shape[1], patches, dtch)
    assert ctu.STATUS[ctx.status_sync()] in ("CTU_ENEGATIVE", "CTU_ENAN")
    assert ctx.status_sync() == 0  # sticky bits are cleared by the read


def test_invalid_arguments_rejected_on_host():
    import torch
    from paper_1110_0740_gb300 import ctu
    dev = _dev()
    U = torch.zeros(9 * 1000, dtype=torch.float64, device=dev)
    ctx = ctu.Ctx(ctu.make_config(ndim=3))
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    p = ctu.make_patches([([2, 2, 2], [1.0] * 3, 0)])
    with pytest.raises(ctu.CtuError):  # aliasing in/out
        ctx.step(U, U, 1000, p, dtch)
    with pytest.raises(ctu.CtuError):  # patch beyond the stride
        ctx.step(U, torch.zeros_like(U), 999, p, dtch)
    bad = ctu.make_patches([([2, 2, 2], [0.0, 1.0, 1.0], 0)])
    with pytest.raises(ctu.CtuError):
        ctx.step(U, torch.zeros_like(U), 1000, bad, dtch)
    with pytest.raises(ctu.CtuError):
        ctu.Ctx(ctu.make_config(ndim=4))
    with pytest.raises(ctu.CtuError):
        ctu.Ctx(ctu.make_config(cfl=1.5))


@pytest.mark.parametrize("prec", [0, 1])
def test_step_next_dt_matches_ctu_dt_of_result(prec):
    import torch
    from paper_1110_0740_gb300 import ctu
    n = [20, 12, 16]
    U0 = np.zeros(O.shape(n, 3))
    O.interior(U0, n, 3)[:] = O.interior(W.mhd_blast_3d(20, seed=4, kmax=3), [20] * 3, 3)[:, :16, :12, :]
    O.fill_periodic(U0, n, 3)
    dev = _dev()
    U = torch.from_numpy(U0.reshape(9, -1).copy()).to(dev)
    Ua, Ub = torch.zeros_like(U), torch.zeros_like(U)
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3))
    p = ctu.make_patches([(n, [1 / 20, 1 / 12, 1 / 16], 0)])
    d0 = torch.zeros(2, dtype=torch.float64, device=dev)
    d1 = torch.zeros_like(d0)
    d2 = torch.zeros_like(d0)
    ctx.dt(U, U.shape[1], p, d0)
    ctx.step(U, Ua, U.shape[1], p, d0)
    ctx.step_next_dt(U, Ub, U.shape[1], p, d0, d1)
    ctx.dt(Ub, U.shape[1], p, d2)
    assert ctx.status_sync() == 0
    assert torch.equal(Ua, Ub) or prec == 0 and torch.allclose(Ua, Ub, rtol=0, atol=0)
    a, b = d1.cpu().numpy(), d2.cpu().numpy()
    assert np.allclose(a, b, rtol=1e-13 if prec == 0 else 1e-6, atol=0), (a, b)


@pytest.mark.parametrize("par", [{}, dict(kappa=0.002, kappa_par=0.006, tc_phi=0.05, nu=0.001, eta=0.001)])
def test_cuda_graph_replay_matches_direct_step(par):
    """A level step captured in a CUDA graph and replayed gives bitwise the
    same result as the direct call (patch list bound before capture), also
    with the parabolic terms."""
    import torch
    from paper_1110_0740_gb300 import ctu
    H = W.amr_hierarchy(seed=2, base=32, target=40)
    lv = H["levels"][1]
    dev = _dev()
    U = torch.from_numpy(lv["pool"]).to(dev)
    A, B = torch.zeros_like(U), torch.zeros_like(U)
    P = ctu.make_patches([(n, dx, b) for (n, dx, b, _) in lv["patches"]])
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_MIXED, **par))
    d = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.dt(U, U.shape[1], P, d)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        ctx.step(U, A, U.shape[1], P, d, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.step(U, B, U.shape[1], P, d, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert ctx.status_sync() == 0
    assert torch.equal(A, B)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_changes_only_the_launch_shape(prec):
    """ctu_autotune picks a tile width and a segment length per patch shape of
    an uneven batch; a step with the tuned tiles gives bitwise the result of
    a context with the default tiles, the tuning steps leave the bound flux
    registers untouched, and every choice is a valid one."""
    import torch
    from paper_1110_0740_gb300 import ctu
    H = W.amr_hierarchy(seed=4, base=32, target=50)
    lv = H["levels"][2]
    dev = _dev()
    U = torch.from_numpy(lv["pool"]).to(dev)
    stride = U.shape[1]
    P = ctu.make_patches([(n, dx, b) for (n, dx, b, _) in lv["patches"]])
    precision = ctu.CTU_FP64 if prec == 0 else ctu.CTU_MIXED
    cfg = ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=precision, cfl=0.3)
    ref, tuned = ctu.Ctx(cfg), ctu.Ctx(cfg)
    d = torch.zeros(2, dtype=torch.float64, device=dev)
    ref.dt(U, stride, P, d)
    A, B, S = torch.zeros_like(U), torch.zeros_like(U), torch.zeros_like(U)
    n0 = lv["patches"][0][0]
    reg = torch.zeros(9 * n0[1] * n0[2], dtype=torch.float64, device=dev)
    tuned.flux_registers(reg, [(0, 0, 0, 0, n0[1], 0, n0[2], 1.0, 0)])
    tuned.autotune(U, S, stride, P, d)
    assert torch.count_nonzero(reg) == 0
    ref.step(U, A, stride, P, d)
    tuned.step(U, B, stride, P, d)
    assert ref.status_sync() == 0 and tuned.status_sync() == 0
    assert torch.equal(A, B)
    assert torch.count_nonzero(reg) > 0
    for n in {tuple(p[0]) for p in lv["patches"]}:
        xw, seg = tuned.tile_params(n)
        assert xw in (8, 16, 32) and seg in (4, 8, 16, 32, 64)
        assert ref.tile_params(n) == (32 if n[0] >= 24 else 16 if n[0] >= 12 else 8, 16)


def test_full_size_lowbeta_sampled_256():
    """The low-beta Mach-10 variant at 256^3 in the mixed path (autotuned
    tiles): sampled 6^3 blocks against the oracle."""
    import torch
    from paper_1110_0740_gb300 import ctu
    n = 256
    U0 = W.mhd_lowbeta_3d(n, seed=1)
    dev = _dev()
    U = torch.from_numpy(U0.reshape(9, -1)).to(dev)
    Uo = torch.zeros_like(U)
    stride = U.shape[1]
    patches = ctu.make_patches([([n] * 3, [1.0 / n] * 3, 0)])
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_MIXED, cfl=0.3))
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.dt(U, stride, patches, dtch)
    ctx.autotune(U, Uo, stride, patches, dtch)
    ctx.step(U, Uo, stride, patches, dtch)
    assert ctx.status_sync() == 0
    dt, ch = dtch.cpu().tolist()
    G = Uo.view(9, n + 8, n + 8, n + 8)
    rng = np.random.default_rng(9)
    for c in [rng.integers(0, n - 6, size=3) for _ in range(5)]:
        k, j, i = int(c[2]), int(c[1]), int(c[0])
        blk = U0[:, k:k + 14, j:j + 14, i:i + 14].copy()
        R, bad = O.mhd_step(blk, [6, 6, 6], 3, [1.0 / n] * 3, dt, ch, recon=1)
        assert bad == 0
        got = G[:, k + 4:k + 10, j + 4:j + 10, i + 4:i + 10].cpu().numpy()
        e = l1rel(got, O.interior(R, [6, 6, 6], 3), ch)
        assert np.all(e <= 2e-5), (c, e)


def test_full_amr_level_sampled():
    """The AMR workload at full size (3 levels over 128^3, ~560 patches of
    8^3..64^3): the finest level advanced in one batched, autotuned mixed
    step and its ghosts prolonged from level 1 (alpha 1/2); sampled patches
    of every size against the oracle's step and prolongation of that patch."""
    import torch
    from paper_1110_0740_gb300 import ctu
    H = W.amr_hierarchy(seed=0)
    L1, L2 = H["levels"][1], H["levels"][2]
    dev = _dev()
    A1 = torch.from_numpy(L1["pool"]).to(dev)
    B1 = A1 * 1.0
    A2 = torch.from_numpy(L2["pool"]).to(dev)
    B2 = torch.zeros_like(A2)
    P2 = ctu.make_patches([p[:3] for p in L2["patches"]])
    ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=ctu.CTU_MIXED, cfl=0.3))
    d = torch.zeros(2, dtype=torch.float64, device=dev)
    ctx.dt(A2, A2.shape[1], P2, d)
    ctx.autotune(A2, B2, A2.shape[1], P2, d)
    ctx.step(A2, B2, A2.shape[1], P2, d)
    assert ctx.status_sync() == 0
    dt, ch = d.cpu().tolist()
    # ghost shells of every level-2 patch from its parent, between A1 and B1 (a perturbed copy)
    B1[4] *= 1.01
    boxes = []
    for fi, (n, dx, base, _) in enumerate(L2["patches"]):
        parent, o_zyx, sz = L2["footprints"][fi]
        cn, _, cbase, _ = L1["patches"][parent]
        o = [o_zyx[2], o_zyx[1], o_zyx[0]]
        for dd in range(3):
            for lo_d, hi_d in ((-4, 0), (n[dd], n[dd] + 4)):
                lo_ = [lo_d if e == dd else (0 if e < dd else -4) for e in range(3)]
                hi_ = [hi_d if e == dd else (n[e] if e < dd else n[e] + 4) for e in range(3)]
                boxes.append(dict(fn=n, cn=cn, fbase=base, cbase=cbase, lo=lo_, hi=hi_, origin=o, ratio=2))
    F = torch.zeros_like(A2)
    ctx.prolong(A1, B1, A1.shape[1], 0.5, F, F.shape[1], ctu.make_level_boxes(boxes))
    got_step = B2.cpu().numpy()
    got_pro = F.cpu().numpy()
    pool1, pool1n = L1["pool"], B1.cpu().numpy()
    by_size = {}
    for fi, (n, dx, base, _) in enumerate(L2["patches"]):
        by_size.setdefault(n[0], []).append(fi)
    for size, idx in sorted(by_size.items()):
        for fi in idx[:2]:
            n, dx, base, _ = L2["patches"][fi]
            N = [v + 8 for v in n]
            cells = N[0] * N[1] * N[2]
            blk = L2["pool"][:, base:base + cells].reshape(9, N[2], N[1], N[0])
            R, bad = O.mhd_step(blk, list(n), 3, list(dx), dt, ch, recon=1)
            assert bad == 0
            G = got_step[:, base:base + cells].reshape(blk.shape)
            e = l1rel(O.interior(G, list(n), 3), O.interior(R, list(n), 3), ch)
            assert np.all(e <= 2e-5), (size, fi, e)
            parent, o_zyx, sz = L2["footprints"][fi]
            cn, _, cbase, _ = L1["patches"][parent]
            Nc = [v + 8 for v in cn]
            cc = Nc[0] * Nc[1] * Nc[2]
            Co = pool1[:, cbase:cbase + cc].reshape(9, Nc[2], Nc[1], Nc[0])
            Cn = pool1n[:, cbase:cbase + cc].reshape(9, Nc[2], Nc[1], Nc[0])
            ref = np.zeros(O.shape(list(n), 3))
            o = [o_zyx[2], o_zyx[1], o_zyx[0]]
            for b in boxes:
                if b["fbase"] == base:
                    O.prolong(Co, Cn, list(cn), 0.5, ref, list(n), b["lo"], b["hi"], o, 2, 3)
            Gp = got_pro[:, base:base + cells].reshape(blk.shape)
            assert np.allclose(Gp, ref, rtol=1e-14, atol=1e-14), (size, fi)
