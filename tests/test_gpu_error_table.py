"""Per-variable error of every GPU precision against the FP64 oracle, for
each workload configuration at its own step count:

  C1  2-D turbulence 128^2, MC-linear, 20 steps (whole patch)
  C2/C3  3-D blast (|k| <= 8 spectrum + 100x pressure sphere), PPM,
      10 steps: a whole 64^3 patch, and the 256^3 patch itself on sampled
      blocks (the bench's launch configuration)
  C3  low beta 0.01, Mach 10, PPM, 10 steps (whole 64^3 patch)
  C4  the finest AMR level (459 patches of 8^3..64^3), one batched step
  C5  relativistic jet, MUSCL-Hancock + HLL, 10 steps (whole 48^3 patch)

Each run is held to two bars per variable: the relative L1 error
sum|g - r| / sum|r| (the FP64 path's contract is 1e-11), and the elementwise
bound max|g - r| / max|r|, so that an error confined to a few cells (a tile
seam, a patch corner) cannot hide in the L1 sum.  psi is measured against
c_h |B|.  With CTU_ERROR_TABLE set, the measured errors are written there as
markdown."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1110_0740_gb300 import workloads as W
from tests.gpu_util import gpu_run, l1rel, maxrel, oracle_run

pytestmark = pytest.mark.gpu
NAMES = ["rho", "m_x", "m_y", "m_z", "E", "B_x", "B_y", "B_z", "psi"]
PREC = {0: "FP64", 1: "MIXED", 2: "MIXED_IFACE64"}
ROWS = []

# Bars per variable (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi): relative L1
# and elementwise max.  FP64: the contract, 1e-11, for both.  The mixed
# paths: about ten times the errors measured on a GB300 (rounded up to 1, 2
# or 5 in the leading digit), so that a tenfold loss of accuracy fails; the
# two mixed variants share a bar.  A zero bar: the variable must stay exactly
# zero.
FP64_BARS = (1e-11, 1e-11)
MIXED_BARS = {
    "c1": ([1e-6, 5e-6, 5e-6, 0, 1e-6, 1e-6, 1e-6, 0, 5e-7], [5e-6, 1e-5, 1e-5, 0, 5e-6, 5e-6, 5e-6, 0, 2e-6]),
    "c2": ([2e-7, 2e-6, 1e-6, 2e-6, 1e-6, 5e-7, 5e-7, 5e-7, 5e-7], [5e-6, 1e-5, 1e-5, 1e-5, 1e-5, 1e-5, 5e-6, 5e-6, 5e-6]),
    "c3": ([2e-5, 5e-5, 2e-5, 5e-5, 2e-5, 5e-6, 5e-6, 2e-6, 5e-7],
           [5e-4, 5e-4, 5e-4, 5e-4, 5e-4, 2e-5, 2e-5, 1e-5, 5e-6]),
    "c2_256": ([2e-7, 2e-6, 1e-6, 1e-6, 5e-7, 5e-7, 5e-7, 5e-7, 5e-7],
               [1e-6, 5e-6, 5e-6, 2e-6, 2e-6, 2e-6, 2e-6, 2e-6, 2e-6]),
    "c4": ([2e-7, 1e-6, 1e-6, 1e-6, 5e-7, 5e-7, 5e-7, 5e-5, 1e-7], [2e-6, 5e-6, 5e-6, 5e-6, 5e-6, 5e-6, 5e-6, 2e-4, 1e-6]),
    # the transverse components of the beam (m_x, m_y, B_x, B_y) are near zero
    # on their own; the second row measures them against their whole vector
    "c5": ([2e-5, 1e-3, 1e-3, 5e-5, 2e-5, 1e-3, 1e-3, 2e-7, 1e-7], [1e-4, 2e-4, 2e-4, 2e-4, 2e-4, 2e-4, 1e-4, 2e-6, 1e-6]),
    "c5_vec": ([2e-5, 1e-6, 1e-6, 5e-5, 2e-5, 5e-8, 5e-8, 2e-7, 1e-7],
               [1e-4, 2e-4, 2e-4, 2e-4, 2e-4, 2e-4, 1e-4, 2e-6, 1e-6]),
}


def _record(label, precision, got, ref, ch, bars, group_floor=False):
    e1 = l1rel(got, ref, ch, group_floor=group_floor)
    em = maxrel(got, ref, ch)
    b1, bm = (np.broadcast_to(np.asarray(b, dtype=float), (9,)) for b in bars)
    ROWS.append((label, precision, e1, em, (b1, bm)))
    for q in range(9):
        if not np.any(ref[q]):
            assert not np.any(got[q]), f"{label} {precision}: var {q} must stay exactly zero"
    assert np.all(e1 <= b1), (label, precision, "L1", e1, b1)
    assert np.all(em <= bm), (label, precision, "max", em, bm)


def _bars(key):
    return (FP64_BARS, MIXED_BARS[key], MIXED_BARS[key])


def _mhd(label, U0, n, ndim, steps, cfl, recon, bars):
    dx = [1.0 / n[0]] * ndim
    ref, od = oracle_run(U0, n, ndim, dx, steps, cfl, recon=recon)
    R = O.interior(ref, n, ndim)
    for prec in (0, 1, 2):
        got, gd, st = gpu_run(U0, n, ndim, dx, steps, cfl, precision=prec, recon=recon)
        assert st == 0
        if prec == 0:  # the FP64 path takes the oracle's time steps
            for (a, b), (c, d) in zip(gd, od):
                assert abs(a - c) <= 1e-13 * c and abs(b - d) <= 1e-13 * d
        _record(label, PREC[prec], O.interior(got, n, ndim), R, od[-1][1], bars[prec])


def test_c1_2d_turbulence_20_steps():
    n = [128, 128, 1]
    _mhd("C1 2-D turbulence 128^2, MC-linear, 20 steps", W.mhd_turb_2d(128, seed=0), n, 2, 20, 0.4, 0,
         _bars("c1"))


def test_c2_blast_64_10_steps():
    n = [64, 64, 64]
    _mhd("C2/C3 3-D blast 64^3, PPM, 10 steps", W.mhd_blast_3d(64, seed=0), n, 3, 10, 0.3, 1, _bars("c2"))


def test_c3_lowbeta_64_10_steps():
    n = [64, 64, 64]
    _mhd("C3 low beta 0.01, Mach 10, 64^3, PPM, 10 steps", W.mhd_lowbeta_3d(64, seed=1), n, 3, 10, 0.3, 1,
         _bars("c3"))


def _wrap_block(Ui, lo, m):
    """The m^3 block of the periodic interior array Ui (9, n, n, n) whose
    first cell is lo = (x, y, z), indices wrapped."""
    n = Ui.shape[-1]
    ix = [(np.arange(m) + lo[d]) % n for d in range(3)]
    return Ui[:, ix[2]][:, :, ix[1]][:, :, :, ix[0]].copy()


def _oracle_block(Ui, lo, b, k, dx, dt, ch):
    """k oracle steps of the interior block of size b at lo, from the initial
    state alone: the step-j input is the ghosted block of interior
    b + 8 (k - j), its outer four layers the ghosts; each step's interior is
    the next step's ghosted input.  The block's final values depend only on
    the initial state inside that region (4 cells of reach per step)."""
    A = _wrap_block(Ui, [c - 4 * k for c in lo], b + 8 * k)
    for j in range(k):
        m = A.shape[-1] - 8
        R, bad = O.mhd_step(np.ascontiguousarray(A), [m] * 3, 3, dx, dt, ch, recon=1)
        assert bad == 0
        A = O.interior(R, [m] * 3, 3)
    return A


def test_c2_c3_256_sampled_blocks_10_steps():
    """The bench workload itself (256^3 blast, PPM; the mixed paths with the
    bench's autotuned tiles), 10 GPU steps at a fixed dt (the oracle's CFL
    step of the initial state), periodic ghosts refilled on the GPU between
    steps; 8^3 blocks (one across the periodic seam) against the oracle's 10
    steps of their domain of dependence."""
    import torch
    from paper_1110_0740_gb300 import ctu
    n, k, b = 256, 10, 8
    U0 = W.mhd_blast_3d(n, seed=0)
    dx = [1.0 / n] * 3
    dt, ch = O.dt_ch(O.mhd_max_speed(U0, [n] * 3, 3, dx), dx, 3, 0.3)
    Ui = O.interior(U0, [n] * 3, 3)
    rng = np.random.default_rng(11)
    corners = [rng.integers(0, n, size=3) for _ in range(3)] + [np.array([n - 3, 2, n - 5])]
    refs = [_oracle_block(Ui, c, b, k, dx, dt, ch) for c in corners]
    R = np.concatenate([r.reshape(9, -1) for r in refs], axis=1)
    dev = torch.device("cuda:0")
    patches = ctu.make_patches([([n] * 3, dx, 0)])
    dtch = torch.tensor([dt, ch], dtype=torch.float64, device=dev)
    for prec in (0, 1, 2):
        U = torch.from_numpy(U0.reshape(9, -1)).to(dev)
        Ub = torch.zeros_like(U)
        stride = U.shape[1]
        ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3))
        if prec != 0:
            ctx.autotune(U, Ub, stride, patches, dtch)
        for _ in range(k):
            ctx.fill_periodic(U, stride, patches)
            ctx.step(U, Ub, stride, patches, dtch)
            U, Ub = Ub, U
        assert ctx.status_sync() == 0
        G = O.interior(U.cpu().numpy().reshape(U0.shape), [n] * 3, 3)
        ctx.close()
        del U, Ub
        got = np.concatenate([_wrap_block(G, c, b).reshape(9, -1) for c in corners], axis=1)
        _record("C2/C3 3-D blast 256^3 (bench tiles), PPM, 10 steps, four 8^3 blocks", PREC[prec], got, R, ch,
                _bars("c2_256")[prec])


def test_c4_amr_finest_level_one_step():
    """All 459 patches of the AMR hierarchy's finest level (8^3..64^3 with
    prefilled ghosts) in one batched step, dt from the oracle's CFL over the
    level; every patch against the oracle's step of that patch."""
    import torch
    from paper_1110_0740_gb300 import ctu
    H = W.amr_hierarchy(seed=0)
    L2 = H["levels"][2]
    pool = L2["pool"]
    blocks = []
    for (n, dx, base, _) in L2["patches"]:
        N = [v + 8 for v in n]
        blocks.append(pool[:, base:base + N[0] * N[1] * N[2]].reshape(9, N[2], N[1], N[0]))
    m = max(O.mhd_max_speed(np.ascontiguousarray(B), list(n), 3, list(dx))
            for B, (n, dx, _, _) in zip(blocks, L2["patches"]))
    dxl = list(L2["patches"][0][1])
    dt, ch = O.dt_ch(m, dxl, 3, 0.3)
    refs = []
    for B, (n, dx, _, _) in zip(blocks, L2["patches"]):
        R, bad = O.mhd_step(np.ascontiguousarray(B), list(n), 3, list(dx), dt, ch, recon=1)
        assert bad == 0
        refs.append(O.interior(R, list(n), 3).reshape(9, -1))
    Rall = np.concatenate(refs, axis=1)
    dev = torch.device("cuda:0")
    U = torch.from_numpy(pool).to(dev)
    P = ctu.make_patches([p[:3] for p in L2["patches"]])
    dtch = torch.tensor([dt, ch], dtype=torch.float64, device=dev)
    for prec in (0, 1):
        Uo = torch.zeros_like(U)
        ctx = ctu.Ctx(ctu.make_config(ndim=3, recon=ctu.CTU_PPM, precision=prec, cfl=0.3))
        if prec:
            ctx.autotune(U, Uo, U.shape[1], P, dtch)
        ctx.step(U, Uo, U.shape[1], P, dtch)
        assert ctx.status_sync() == 0
        out = Uo.cpu().numpy()
        ctx.close()
        got = []
        for (n, dx, base, _) in L2["patches"]:
            N = [v + 8 for v in n]
            G = out[:, base:base + N[0] * N[1] * N[2]].reshape(9, N[2], N[1], N[0])
            got.append(O.interior(G, list(n), 3).reshape(9, -1))
        _record(f"C4 AMR finest level, {len(blocks)} patches 8^3..64^3, PPM, 1 batched step", PREC[prec],
                np.concatenate(got, axis=1), Rall, ch, _bars("c4")[prec])


def test_c5_srmhd_jet_48_10_steps():
    """The gamma-10 magnetised beam (density ratio 0.01, sigma 0.1, 1 % noise)
    at beam pressure 0.05: with the workload's default 0.01 the unlimited
    scheme, the oracle included, meets an unphysical state within 2-5 steps
    at 32^3-48^3, so a 10-step comparison takes the hotter beam.  The momentum
    rows are given both per component and against the whole momentum vector
    (the transverse components of the beam are nearly zero)."""
    n = [48, 48, 48]
    U0 = W.srmhd_jet_3d(48, seed=7, p0=0.05)
    dx = [1.0 / 48] * 3
    ref, t, od = O.srmhd_run(U0, n, 3, dx, 10, 0.3, gamma=4.0 / 3.0)
    R = O.interior(ref, n, 3)
    for prec in (0, 1):
        got, gd, st = gpu_run(U0, n, 3, dx, 10, 0.3, precision=prec, gamma=4.0 / 3.0, physics=1)
        assert st == 0
        G = O.interior(got, n, 3)
        _record("C5 SRMHD jet gamma 10, 48^3, MUSCL-Hancock, 10 steps", PREC[prec], G, R, od[-1][1],
                FP64_BARS if prec == 0 else MIXED_BARS["c5"])
        _record("C5 SRMHD jet (momentum and field against their vectors)", PREC[prec], G, R, od[-1][1],
                FP64_BARS if prec == 0 else MIXED_BARS["c5_vec"], group_floor=True)


def test_zz_write_table():
    path = os.environ.get("CTU_ERROR_TABLE")
    if not path or not ROWS:
        pytest.skip("CTU_ERROR_TABLE not set")
    lines = ["| workload | precision | measure | " + " | ".join(NAMES) + " | largest error / its bar |",
             "|---|---|---|" + "---:|" * len(NAMES) + "---:|"]
    for label, prec, e1, em, (b1, bm) in ROWS:
        def frac(e, b):
            return max((v / w for v, w in zip(e, b) if w > 0), default=0.0)
        lines.append(f"| {label} | {prec} | L1 | " + " | ".join(f"{v:.1e}" for v in e1) +
                     f" | {frac(e1, b1):.2f} |")
        lines.append("| | | max | " + " | ".join(f"{v:.1e}" for v in em) + f" | {frac(em, bm):.2f} |")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
