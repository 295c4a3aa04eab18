"""Algorithmic flop counts per cell update of the CTU-MHD step, counted in the
CPU oracle (test infrastructure).

Builds oracle/flopcount.cpp (the oracle compiled with a counting number
type that skips operations on exact zeros, i.e. the structural zeros of the
eigenvector matrices), feeds it stencils sampled from the blast workload
(advanced two steps) and prints
the per-building-block averages and the per-cell totals of each stage of
the step, in the large-patch limit (the relativistic step alike, from
records of the jet workload, with MUSCL-Hancock predict, HLL and the Newton
recovery in place of the MHD building blocks):

  prim        1 x cons2prim
  flux1 (d)   1 x riemann
  sweep (d)   predict (per reconstruction) + 2 prim2cons + 2 cons2prim + riemann
              + 18 (half-step transverse increments of two directions,
                    9 x (sub, mul) each) + 18 (U* + dt/2 T) + 18 (flux
                    difference x 1/dx)
  update      9 x 2 (dt x sum + U) + 2 (sum of three directions) x 9 + 1 (psi)
  next dt     cons2prim + ndim x (cfast + 2)

and the parabolic terms' stages (Section 3.1), per interior cell with
m = 1 + 3 (viscosity) + 3 (resistivity) conserved components changed and
one face flux per direction (par_face_* summed over the terms on):

  par half    T of U^n (1) + 3 faces + m x 8 (L_P: three differences and
              scalings, two sums) + 16 (three first-order divergences) + m
              + 16 (U^n + dt/2 sum) + 17 (pressure, T) + 3 (v, viscosity)
  par update  3 faces + m x 10 (L_P, dt FMA) + next dt + 13 (diffusion
              number: D / rho, 3 x (1/dx^2, x D, x 2, +)); the GPU step
              splits it over the face pass, par_lp and the x sweep
  sweep (d)   + 2 m (dt/2 L_P in the predictor)

    python oracle/flopcount.py [--out profiles/flops_per_cell.txt]
"""
import argparse
import os
import subprocess
import sys
import tempfile
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parent))


def build():
    exe = Path(tempfile.gettempdir()) / "ctu_flopcount"
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-I", str(HERE),
                    str(HERE / "flopcount.cpp"), "-o", str(exe)], check=True)
    return exe


def stencils(n=48, samples=2000, seed=0):
    """Stencils along x from the blast workload after two oracle steps (so that
    psi and every field is generic, not an exact zero)."""
    import oracle as O
    from paper_1110_0740_gb300 import workloads as W
    U = W.mhd_blast_3d(n, seed=seed)
    U, _, _ = O.mhd_run(U, [n] * 3, 3, [1.0 / n] * 3, 2, 0.3, recon=1)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(samples):
        k, j, i = (int(v) for v in rng.integers(4, n + 4, size=3))
        vs = []
        for m in range(-2, 3):
            V, bad = O.mhd_cons2prim(U[:, k, j, i + m], 5.0 / 3.0)
            vs.append(V)
        out.append(np.array(vs))
    return out


def sr_records(n=64, samples=2000, seed=0):
    """Relativistic records along x from the jet workload's initial state (the
    state the relativistic bench steps): V of cells i - 1, i, i + 1 (local
    order) and U of cell i, at randomly drawn cells."""
    import oracle as O
    from paper_1110_0740_gb300 import workloads as W
    U = W.srmhd_jet_3d(n, seed=seed)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(samples):
        k, j, i = (int(v) for v in rng.integers(4, n + 4, size=3))
        vs = []
        for m in (-1, 0, 1):
            V, bad = O.srmhd_cons2prim(U[:, k, j, i + m], 4.0 / 3.0)
            vs.append(V)
        out.append(np.concatenate([np.ravel(vs), U[:, k, j, i]]))
    return out


def _run(exe, txt, arg=None):
    res = subprocess.run([str(exe)] + ([arg] if arg else []), input=txt.encode(), capture_output=True,
                         check=True)
    c = {}
    for line in res.stdout.decode().splitlines():
        k, v = line.split()
        c[k] = float(v)
    return c


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    exe = build()
    st = stencils()
    txt = f"{len(st)} {5.0 / 3.0!r} 3.0 0.1\n" + "\n".join(" ".join(repr(float(x)) for x in s.ravel())
                                                           for s in st)
    c = _run(exe, txt)
    sr = sr_records()
    srt = f"{len(sr)} {4.0 / 3.0!r} 3.0 0.1\n" + "\n".join(" ".join(repr(float(x)) for x in r) for r in sr)
    csr = _run(exe, srt, "srmhd")
    prim = c["cons2prim"]
    flux1 = c["riemann"]
    recons = ("ppm", "linear", "minmod", "harmonic", "vanalbada", "weno3")
    sweep = {r: c[f"predict_{r}"] + 2 * c["prim2cons"] + 2 * c["cons2prim"] + c["riemann"] + 54
             for r in recons}
    update = 9 * 2 + 9 * 2 + 1
    nextdt = c["cons2prim"] + 3 * (c["cfast"] + 2)
    lines = ["# oracle flops per call, exact-zero operands not counted (averages over %d stencils"
             " of the blast workload after two steps)" % len(st),
             "# produced by: python oracle/flopcount.py --out profiles/flops_per_cell.txt"]
    lines += [f"{k} {v:.1f}" for k, v in c.items()]
    lines += ["# per interior cell update, large-patch limit, 3-D",
              f"prim {prim:.1f}", f"flux1_per_direction {flux1:.1f}",
              f"sweep_per_direction_ppm {sweep['ppm']:.1f}",
              f"sweep_per_direction_linear {sweep['linear']:.1f}"]
    lines += [f"sweep_per_direction_{r} {sweep[r]:.1f}" for r in recons[2:]]
    lines += [f"update {update:.1f}", f"next_dt {nextdt:.1f}",
              "# hand counts of the parabolic stages outside the face fluxes (the tallies in the",
              "# docstring of oracle/flopcount.py), not measured with the counting type:",
              "par_half_per_cell 50.0", "par_half_per_component 9.0", "par_half_visc 3.0",
              "par_update_per_component 10.0", "par_update_diffusion_number 13.0",
              "sweep_par_per_component 2.0",
              f"step_total_ppm {prim + 3 * flux1 + 3 * sweep['ppm'] + update + nextdt:.1f}"]
    # relativistic MHD: the same step structure with the MUSCL-Hancock
    # predictor, HLL and the Newton recovery (counted on the jet's states)
    sr_sweep = csr["sr_predict"] + 2 * csr["sr_prim2cons"] + 2 * csr["sr_cons2prim"] + csr["sr_riemann"] + 54
    sr_next = csr["sr_cons2prim"] + 3 * (csr["sr_fast_speeds"] + 2)
    lines += ["# relativistic MHD, oracle flops per call (averages over %d cells of the 64^3 jet's"
              " initial state)" % len(sr)]
    lines += [f"{k} {v:.1f}" for k, v in csr.items()]
    lines += ["# relativistic MHD per interior cell update, large-patch limit, 3-D",
              f"sr_prim {csr['sr_cons2prim']:.1f}", f"sr_flux1_per_direction {csr['sr_riemann']:.1f}",
              f"sr_sweep_per_direction {sr_sweep:.1f}", f"sr_next_dt {sr_next:.1f}",
              f"sr_step_total {csr['sr_cons2prim'] + 3 * csr['sr_riemann'] + 3 * sr_sweep + update + sr_next:.1f}"]
    text = "\n".join(lines) + "\n"
    print(text)
    if args.out:
        Path(args.out).write_text(text)


if __name__ == "__main__":
    main()
