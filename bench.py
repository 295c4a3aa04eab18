"""Benchmark of the CTU-MHD step on GB300: cell-updates/s, roofline, oracle baseline.

One "step" is the whole hot path over one batch: ctu_step_next_dt (prim,
first-order transverse fluxes, characteristic tracing + HLLD + update fused
per direction, psi damping, flux registers bound on the patch's six boundary
faces, and the CFL reduction of Eq. Ca on the result, which gives the next
step's dt; ctu_dt runs once before the loop).  Workload: one periodic 256^3 ideal-MHD
patch (+4 ghost layers, 1.32 GB of float64 state) with a seeded Fourier
spectrum (|k| <= 8) in rho, v and B (vector potential) plus a radius-0.1
sphere at 100x pressure; PPM + characteristic tracing, HLLD, GLM, CFL 0.3.
The state (1.3 GB in, 1.2 GB out) is far larger than L2, so no flush is
needed between timed steps.

The headline `value` is the mixed-precision path (float32 tracing and
Riemann fluxes, float64 pressure recovery / interface states / update); the
FP64 path is measured in the same run and reported under `fp64_path`.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 256
WORKLOAD = ("3D ideal MHD 256^3 periodic patch, seeded |k|<=8 spectrum in rho/v/B + "
            "100x pressure sphere (r=0.1); PPM + characteristic tracing, HLLD, GLM, CFL 0.3")
METRIC = "MHD cell-updates/s per CTU step"
# reconstruction of the characteristic variables (Section 3.2): the workload's
# PPM, and the other choices the library offers (measured with --recon)
RECONS = {"ppm": 1, "mc": 0, "minmod": 2, "harmonic": 3, "vanalbada": 4, "weno3": 5}
# Per-SM unit counts x max SM clock (2070 MHz) x 152 SMs, 2 flops per FMA.
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES = 128
FP32_PEAK = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6   # 80.5 TFLOP/s
FP64_PEAK = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6            # 1.26 TFLOP/s (2 DFMA/SM/clk)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_bytes(n):
    """Bytes the step must move per launch: read the ghosted state once and
    write the interior once (9 float64 variables), plus the flux registers
    (6 faces x n^2 x 9 float64, read-modify-write)."""
    ghosted = (n + 8) ** 3
    interior = n ** 3
    regs = 6 * n * n * 9 * 8 * 2
    return 9 * 8 * (ghosted + interior) + regs


class Clocks:
    """nvidia-smi sampler over the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                smax = float(c[2])
                pw.append(float(c[3]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        busy = [s for s, w in zip(sm, pw) if w > 200.0] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(pw) if pw else None}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ oracle (CPU)

def oracle_sample(U0, n_full, sub, steps=1, min_seconds=0.0, max_steps=64):
    """Time the CPU oracle on a bounded sample of the workload: a sub x sub x
    sub block of the 256^3 state (with its true neighbours as ghosts), one CTU
    step per repetition, `steps` repetitions or more until min_seconds have
    passed (at most max_steps).  Returns (cell-updates/s, seconds, sample
    text)."""
    import numpy as np
    import oracle as O
    g = 4
    lo = (n_full - sub) // 2
    blk = U0[:, lo:lo + sub + 2 * g, lo:lo + sub + 2 * g, lo:lo + sub + 2 * g].copy()
    n = [sub] * 3
    dx = [1.0 / n_full] * 3
    m = O.mhd_max_speed(blk, n, 3, dx)
    dt, ch = O.dt_ch(m, dx, 3, 0.3)
    t0 = time.perf_counter()
    done = 0
    while done < steps or (time.perf_counter() - t0 < min_seconds and done < max_steps):
        out, bad = O.mhd_step(blk, n, 3, dx, dt, ch, recon=1)
        done += 1
    el = time.perf_counter() - t0
    steps = done
    cells = sub ** 3 * steps
    return cells / el, el, f"{sub}^3 interior block of the 256^3 state, {steps} CTU step(s), 1 thread"


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1110_0740_gb300 import workloads as W
    U0 = W.mhd_blast_3d(N_CELLS, seed=0)
    vals = []
    sub = 64
    for _ in range(max(1, args.warmup)):
        oracle_sample(U0, N_CELLS, sub)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, el, txt = oracle_sample(U0, N_CELLS, sub)
        vals.append(v)
    total = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": txt},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1,
                             "kind": "oracle", "sample": txt},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import numpy as np
    import torch

    from paper_1110_0740_gb300 import ctu, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    n = args.n
    U0 = W.mhd_blast_3d(n, seed=rank)
    Uh = torch.from_numpy(U0.reshape(9, -1))
    stride = Uh.shape[1]
    U = Uh.to(dev)
    Uo = torch.empty_like(U)
    dx = [1.0 / n] * 3
    patches = ctu.make_patches([([n] * 3, dx, 0)])
    # flux registers on the 6 boundary faces of the patch
    windows, off = [], 0
    for d in range(3):
        for plane in (0, n):
            windows.append((0, d, plane, 0, n, 0, n, 1.0, off))
            off += 9 * n * n
    reg = torch.zeros(off, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def make(prec):
        c = ctu.Ctx(ctu.make_config(ndim=3, recon=RECONS[args.recon], precision=prec, cfl=0.3,
                                    shock=(args.shock, 0) if args.shock else None,
                                    riemann=ctu.CTU_HLLC if args.riemann == "hllc" else ctu.CTU_HLLD,
                                    kappa=args.kappa, nu=args.nu, eta=args.eta, kappa_par=args.kappa_par,
                                    tc_phi=args.tc_phi, corner=1 if args.corner == "mt" else 0))
        c.flux_registers(reg, windows)
        c.dt(U, stride, patches, dtch)
        if prec != ctu.CTU_FP64:  # tile width and segment for the patch shape
            c.autotune(U, Uo, stride, patches, dtch)
            tiles["xw_seg"] = list(c.tile_params([n] * 3))
        return c

    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    dtn = torch.zeros(2, dtype=torch.float64, device=dev)
    tiles = {}

    def step(c):
        # the step with its fused next-step CFL epilogue (Eq. Ca on U^(n+1));
        # {dt, c_h} of this step come from the previous step (ctu_dt once)
        c.step_next_dt(U, Uo, stride, patches, dtch, dtn)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def timed(c, K, W_, prof=False):
        for _ in range(W_):
            step(c)
        if prof:
            c.profile(True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step(c)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        kern = c.profile_read() if prof else {}
        if prof:
            c.profile(False)
        if pg is not None:
            t = torch.tensor([ms], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return ms, kern

    primary = {"mixed": ctu.CTU_MIXED, "fp64": ctu.CTU_FP64, "iface64": ctu.CTU_MIXED_IFACE64}[args.precision]
    other = ctu.CTU_FP64 if primary != ctu.CTU_FP64 else ctu.CTU_MIXED
    cells = n ** 3
    results = {}
    clocks = Clocks(local)
    for prec in (primary, other):
        if prec == other and args.skip_other:
            continue
        c = make(prec)
        K = args.steps if prec == primary else max(2, min(args.steps, args.other_steps))
        Wn = args.warmup if prec == primary else 1
        if prec == primary:
            clocks.start()
        ms, kern = timed(c, K, Wn, prof=False)
        if prec == primary:
            clk = clocks.stop()
            st = c.status_sync()
            launches_per_step = c.launches()  # kernels per step_next_dt call
            # kernel durations over a second, profiled pass of the same region
            _, kern = timed(c, K, 0, prof=True)
        else:
            st = c.status_sync()
            _, kern = timed(c, K, 0, prof=True)
        results[prec] = {"ms_total": ms, "K": K, "kern": kern, "status": st}
        c.close()

    res = results[primary]
    ms_step = res["ms_total"] / res["K"]
    value = world * cells / (ms_step * 1e-3)

    # roofline of the dominant kernel (ALU-bound: FP32 pipe for the mixed
    # path, FP64 pipe for the FP64 path), algorithmic flops per cell from the
    # oracle count in profiles/flops_per_cell.txt
    peaks, src = measured_peaks()
    kern = res["kern"]
    top_name, (top_ms, top_cnt) = max(kern.items(), key=lambda kv: kv[1][0])
    top_avg = top_ms / max(1, top_cnt)
    fl = kernel_flops(n, args.recon, args.kappa, args.kappa_par, args.tc_phi, args.nu, args.eta,
                      corner=args.corner)
    mixed = primary != ctu.CTU_FP64
    peak_tf = (FP32_PEAK if mixed else FP64_PEAK) / 1e12
    f_top = fl.get(top_name, 0.0)
    achieved = f_top / (top_avg * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": achieved / peak_tf, "traffic": kernel_traffic(top_name, n), "kernel": top_name,
            "pipe": "fp32" if mixed else "fp64",
            "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz" if mixed else
                            "derived: 152 SMs x 2 FP64 lanes x 2 x 2070 MHz (GB300 nominal 1.25 TF)"),
            "flops_per_launch": f_top, "kernel_avg_ms": top_avg,
            "kernels_ms_per_step": {k: v[0] / res["K"] for k, v in kern.items()}}
    # the FMA-throughput microbenchmark of the same pipe, beside the derived peak
    try:
        fma = ctu.ctu_fma_peak(not mixed, (1 << 16) if mixed else (1 << 12)) / 1e12
        roof["fma_measured"] = {"tflops": fma, "frac": achieved / fma,
                                "what": "ctu_fma_peak: 8 independent FMA chains per thread, 16 x 256 threads per SM"}
    except ctu.CtuError:
        roof["fma_measured"] = None
    step_ms = sum(v[0] for v in kern.values()) / res["K"]
    roof["step"] = {"flops": sum(fl.values()), "achieved_tflops": sum(fl.values()) / (step_ms * 1e-3) / 1e12,
                    "frac": sum(fl.values()) / (step_ms * 1e-3) / 1e12 / peak_tf}
    nbytes = algorithmic_bytes(n)
    hbm_achieved = nbytes / (step_ms * 1e-3) / 1e9
    roof["hbm_step"] = {"algorithmic_bytes": nbytes, "achieved_gbs": hbm_achieved,
                        "peak_gbs": peaks["hbm_gbs"], "frac": hbm_achieved / peaks["hbm_gbs"],
                        "peak_source": f"{src} hbm_gbs"}
    plain = not (args.shock or args.kappa or args.nu or args.eta or args.kappa_par or args.corner == "mt")
    if mixed and args.recon == "ppm" and args.riemann == "hlld" and plain:
        ps = precision_split_roofline(n, value / world, peaks["hbm_gbs"])
        # the kernels run the float64-designated recoveries in double-float on
        # the FP32 pipe, so the FP64 term of this bound does not bind them:
        # the bound they face is the FP32 one, with every operation counted
        ps["binds_these_kernels"] = False
        ps["fp32_everything"] = {"flops_per_cell": ps["fp32_flops_per_cell"] + ps["fp64_flops_per_cell"],
                                 "bound_cells_per_s": FP32_PEAK / (ps["fp32_flops_per_cell"]
                                                                   + ps["fp64_flops_per_cell"]),
                                 "frac": (value / world) / (FP32_PEAK / (ps["fp32_flops_per_cell"]
                                                                         + ps["fp64_flops_per_cell"]))}
        roof["precision_split"] = ps
    roof["bases"] = ("frac: the dominant kernel's oracle-counted flops per launch / its CUDA-event time, "
                     "against the FP32 (mixed) or FP64 pipe peak; step.frac: the whole step the same way; "
                     "precision_split.frac: the split-precision whole-step bound, whose FP64 term these "
                     "kernels do not face (double-float on the FP32 pipe); "
                     "precision_split.fp32_everything.frac: the bound they face")

    # end-to-end through the public API with host buffers
    # every step copies its input state (the interior, 9 float64 fields of
    # n^3 cells, packed) from pinned host memory and reads its result (the
    # updated interior, packed) back; on the device the library unpacks the
    # input into the ghosted patch, fills its periodic ghosts, steps and packs
    # the result (ctu_unpack, ctu_fill_periodic, ctu_step_next_dt, ctu_pack).
    # With two device copies of each buffer, the copy of step k + 1's input
    # and the read-back of step k - 1's result run on their own streams (both
    # copy directions) while step k computes, as a caller streaming states
    # through the library would arrange it
    e2e = None
    if not args.skip_e2e:
        c = make(primary)
        e2e = e2e_stream(c, Uh, U, Uo, n, stride, patches, dtch, dtn, max(4, args.steps), dev, world, barrier,
                         lanes=args.copy_lanes)
        c.close()

    fp64_path = None
    if other in results:
        r2 = results[other]
        ms2 = r2["ms_total"] / r2["K"]
        fp64_path = {"precision": "fp64" if other == ctu.CTU_FP64 else "mixed",
                     "value": world * cells / (ms2 * 1e-3), "ms_per_step": ms2, "steps": r2["K"],
                     "kernels_ms_per_step": {k: v[0] / r2["K"] for k, v in r2["kern"].items()}}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        v, el, txt = oracle_sample(U0, n, min(64, n), min_seconds=10.0)
        cpu = {"value": v, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": txt,
               "seconds": el}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
                "steps": res["K"], "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if primary != ctu.CTU_FP64 else "f64", "data": "synthetic",
                "config": {"workload": (WORKLOAD if args.recon == "ppm" else
                                        WORKLOAD.replace("PPM", f"{args.recon} reconstruction"))
                           + (f"; hybrid integration (shock flags, eps_q {args.shock})" if args.shock else "")
                           + ("; HLLC in place of HLLD" if args.riemann == "hllc" else "")
                           + (f"; thermal conduction, kappa {args.kappa}" if args.kappa else "")
                           + (f" (along the field {args.kappa_par})" if args.kappa_par else "")
                           + (f", saturated (phi {args.tc_phi})" if args.tc_phi else "")
                           + (f"; viscosity, nu {args.nu}" if args.nu else "")
                           + (f"; resistivity, eta {args.eta}" if args.eta else "")
                           + ("; corner coupling from the normal predictor states (Mignone & Tzeferacos)"
                              if args.corner == "mt" else ""),
                           "recon": args.recon, "shock_eps": args.shock or None,
                           "cells_per_gpu": cells, "patches_per_gpu": 1,
                           "precision": args.precision, "l2_flush": "inputs (1.3 GB) > L2",
                           "parallelism": f"replicas x{world}", "tiles_xw_seg": tiles.get("xw_seg")},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_path": fp64_path,
                "gpu_launches": launches_per_step * res["K"], "clocks": clk,
                "status": ctu.STATUS[res["status"]] if 0 <= res["status"] < 10 else res["status"],
                "gpu": torch.cuda.get_device_name(dev)}
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


def e2e_stream(c, Uh, U, Uo, n, stride, patches, dtch, dtn, E, dev, world, barrier, lanes=1):
    """End to end through the public API with host buffers, one periodic n^3
    patch: every step copies its input state (the interior, 9 float64 fields
    of n^3 cells, packed) from pinned host memory and reads its result (the
    updated interior, packed) back; on the device the library unpacks the
    input into the ghosted patch, fills its periodic ghosts, steps and packs
    the result (ctu_unpack, ctu_fill_periodic, ctu_step_next_dt, ctu_pack).
    With two device copies of each buffer, the copy of step k + 1's input and
    the read-back of step k - 1's result run on their own streams (both copy
    directions) while step k computes, as a caller streaming states through
    the library would arrange it.  The E timed steps include the pipeline's
    fill and drain; the streamed result is checked against the device step."""
    import torch
    from paper_1110_0740_gb300 import ctu
    box = ctu.make_copy_boxes([dict(dn=[n] * 3, sn=[n] * 3, lo=[0] * 3, hi=[n] * 3, shift=[0] * 3,
                                    dbase=0, sbase=0)])
    Ih_pin = Uh.reshape(9, n + 8, n + 8, n + 8)[:, 4:-4, 4:-4, 4:-4].contiguous().pin_memory()
    Ubuf = [U, torch.empty_like(U)]
    Obuf = [Uo, torch.empty_like(Uo)]
    Ibuf = [torch.empty(Ih_pin.shape, dtype=torch.float64, device=dev) for _ in range(2)]
    Pbuf = [torch.empty(Ih_pin.shape, dtype=torch.float64, device=dev) for _ in range(2)]
    Oh = [torch.empty_like(Ih_pin).pin_memory() for _ in range(2)]
    s_cmp = torch.cuda.Stream()
    # each direction's copy is split by variable over `lanes` streams, so that
    # several copy engines share it
    s_in = [torch.cuda.Stream() for _ in range(lanes)]
    s_out = [torch.cuda.Stream() for _ in range(lanes)]
    parts = [list(range(9))[i::lanes] for i in range(lanes)]
    ev_in = [[torch.cuda.Event() for _ in range(lanes)] for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [[torch.cuda.Event() for _ in range(lanes)] for _ in range(2)]

    def pipeline(K):
        for k in range(K):
            b = k % 2
            for i, qs in enumerate(parts):
                if k >= 2:
                    s_in[i].wait_event(ev_cmp[b])  # step k - 2 has read input buffer b
                with torch.cuda.stream(s_in[i]):
                    for q in qs:
                        Ibuf[b][q].copy_(Ih_pin[q], non_blocking=True)
                    ev_in[b][i].record(s_in[i])
                s_cmp.wait_event(ev_in[b][i])
                if k >= 2:
                    s_cmp.wait_event(ev_out[b][i])  # result buffer b has been read back
            c.unpack(Ubuf[b], stride, Ibuf[b], box, stream=s_cmp)
            c.fill_periodic(Ubuf[b], stride, patches, stream=s_cmp)
            c.step_next_dt(Ubuf[b], Obuf[b], stride, patches, dtch, dtn, stream=s_cmp)
            c.pack(Pbuf[b], Obuf[b], stride, box, stream=s_cmp)
            ev_cmp[b].record(s_cmp)
            for i, qs in enumerate(parts):
                s_out[i].wait_event(ev_cmp[b])
                with torch.cuda.stream(s_out[i]):
                    for q in qs:
                        Oh[b][q].copy_(Pbuf[b][q], non_blocking=True)
                    ev_out[b][i].record(s_out[i])

    pipeline(2)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s_in[0])
    for i in range(1, lanes):
        s_in[i].wait_event(t0)
    pipeline(E)
    for i in range(1, lanes):
        s_out[0].wait_stream(s_out[i])
    t1.record(s_out[0])
    barrier()
    ems = t0.elapsed_time(t1) / E
    torch.cuda.synchronize()
    # the streamed result is the device step's (same input every step)
    assert torch.equal(Oh[(E - 1) % 2], Obuf[(E - 1) % 2].reshape(9, n + 8, n + 8, n + 8)[:, 4:-4, 4:-4, 4:-4]
                       .contiguous().cpu())
    return {"value": world * n ** 3 / (ems * 1e-3), "unit": "cell-updates/s",
            "h2d_bytes_per_step": int(Ih_pin.numel() * 8), "d2h_bytes_per_step": int(Oh[0].numel() * 8),
            "ms_per_step": ems, "steps": E,
            "overlap": f"two device buffers; packed-interior input copy, unpack + periodic ghost fill + "
                       f"step + pack, and read-back on their own streams, each copy split by variable over "
                       f"{lanes} stream(s) per direction"}


def roofline_alu(kern, flops, mixed, traffic=None):
    """Kernel roofline of the dominant kernel group: kern maps a kernel name
    to (total ms, launches) over the timed region, flops maps it to the
    algorithmic flops of one launch; ALU-bound on the FP32 pipe (mixed) or the
    FP64 pipe."""
    top_name, (top_ms, top_cnt) = max(kern.items(), key=lambda kv: kv[1][0])
    top_avg = top_ms / max(1, top_cnt)
    peak_tf = (FP32_PEAK if mixed else FP64_PEAK) / 1e12
    f_top = flops.get(top_name, 0.0)
    achieved = f_top / (top_avg * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": achieved / peak_tf, "traffic": traffic, "kernel": top_name,
            "pipe": "fp32" if mixed else "fp64",
            "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz" if mixed else
                            "derived: 152 SMs x 2 FP64 lanes x 2 x 2070 MHz (GB300 nominal 1.25 TF)"),
            "flops_per_launch": f_top, "kernel_avg_ms": top_avg}


def run_amr(args):
    """Batched AMR level advance: the seeded 3-level hierarchy (refinement
    ratio 2, base 128^3, ~560 patches of 8^3..64^3) around an expanding
    spherical shock; one coarse step = level 0 once, level 1 twice, level 2
    four times (dt_l = dt_0 / 2^l, common c_h), all seven batched ctu_step
    calls captured in one CUDA graph; flux-register windows on both sides of
    every coarse-fine interface; on one GPU, before every level step the
    ghosts are filled (prolongation from the parent level in time, then the
    same-level exchange from siblings), so is every new state that a finer
    level prolongs from, and at every synchronisation the parent is
    refluxed and restricted.  dt_0 is fixed before timing from ctu_dt on
    every level (dt_0 = min_l 2^l dt_l).  With N > 1 ranks every rank builds
    the same hierarchy and advances its shard of each level (patches split by
    cell count, Section 4); the ranks agree on dt_0 (one scalar reduction) and
    the step time is the slowest rank's (strong scaling)."""
    import torch
    from paper_1110_0740_gb300 import ctu, shard, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    H = W.amr_hierarchy(seed=0, nested=args.amr_nested)
    L = H["levels"]
    prec = ctu.CTU_MIXED if args.precision == "mixed" else ctu.CTU_FP64
    # this rank's patches per level (indices into the level's patch list)
    mine = []
    for lv in L:
        cells_l = [n[0] * n[1] * n[2] for (n, _, _, _) in lv["patches"]]
        mine.append(shard.partition(cells_l, world)[rank])
    # the hierarchy's coarse step: pools, flux-register windows, level-operator
    # tables and the subcycled launch sequence (paper_1110_0740_gb300.amr_advance);
    # the level operators run on one rank (the cross-rank exchange is host-tested)
    from paper_1110_0740_gb300.amr_advance import LevelAdvance
    dx0 = L[0]["patches"][0][1][0]
    adv = LevelAdvance(L, int(round(1.0 / dx0)), precision=prec, cfl=0.3, mine=mine,
                       level_ops=world == 1 and not args.no_level_ops, device=dev, kappa=args.kappa,
                       kappa_par=args.kappa_par, tc_phi=args.tc_phi, nu=args.nu, eta=args.eta)
    ctxs, A, B, P, D = adv.ctxs, adv.A, adv.B, adv.P, adv.D
    ops, xch, wins = adv.ops, adv.xch, adv.windows
    dt0, ch = shard.agree_dt((adv.local_dt(), 0.0), 0.3, dx0, group=None if pg is None else pg.group.WORLD)
    adv.set_dt(dt0, ch)
    stream = torch.cuda.Stream(device=dev)
    # tile width and marching segment per patch shape of each level
    tiles = {}
    for lev in range(len(L)):
        if P[lev] is not None:
            ctxs[lev].autotune(A[lev], B[lev], A[lev].shape[1], P[lev], D[lev], stream=stream)
            for n in sorted({tuple(L[lev]["patches"][gi][0]) for gi in mine[lev]}):
                tiles[f"l{lev}_{n[0]}^3"] = list(ctxs[lev].tile_params(n))
    torch.cuda.synchronize()

    def coarse_step():
        adv.coarse_step(stream)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        coarse_step()  # binds patch lists, sizes scratch (before capture)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        coarse_step()
    for _ in range(args.warmup):
        g.replay()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            g.replay()
        e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = shard.slowest(e0.elapsed_time(e1) / args.steps,
                       group=None if pg is None else pg.group.WORLD)
    st = [c.status_sync() for c in ctxs]
    cells = [sum(n[0] * n[1] * n[2] for (n, _, _, _) in lv["patches"]) for lv in L]
    upd = cells[0] + 2 * cells[1] + 4 * cells[2]
    my_upd = sum(2 ** lev * sum(L[lev]["patches"][gi][0][0] ** 3 for gi in mine[lev]) for lev in range(len(L)))
    from collections import Counter
    hist = {lev: dict(sorted(Counter(n[0] for (n, _, _, _) in lv["patches"]).items()))
            for lev, lv in enumerate(L)}
    # per-kernel times of one (non-graph) coarse step
    for c in ctxs:
        c.profile(True)
    with torch.cuda.stream(stream):
        coarse_step()
    kern = {}
    for lev, c in enumerate(ctxs):
        for k_, (t_, n_) in c.profile_read().items():
            kern[f"l{lev}_{k_}"] = (t_, n_)
        c.profile(False)
    # kernel roofline of the dominant step kernel (ALU-bound; flops per launch
    # from the oracle's counts per interior cell times the level's cells on
    # this rank); the level operators (prolongation, exchange, reflux,
    # restriction) are float64 and carry no flop count
    mixed = prec == ctu.CTU_MIXED
    flops = {}
    for lev in range(len(L)):
        cl = sum(L[lev]["patches"][gi][0][0] * L[lev]["patches"][gi][0][1] * L[lev]["patches"][gi][0][2]
                 for gi in mine[lev])
        for k_, v_ in kernel_flops(1, "ppm", args.kappa, args.kappa_par, args.tc_phi, args.nu, args.eta,
                                   cells=cl).items():
            flops[f"l{lev}_{k_}"] = v_
    roof = roofline_alu({k: v for k, v in kern.items() if k in flops}, flops, mixed)
    roof["share_of_coarse_step"] = kern[roof["kernel"]][0] / sum(v[0] for v in kern.values())
    # the oracle on a bounded sample of the finest level's patches (every size
    # in turn), one step each, on one host core
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        import numpy as np
        import oracle as O
        L2 = L[-1]
        by = {}
        for gi, (n, dx, base, _) in enumerate(L2["patches"]):
            by.setdefault(n[0], []).append(gi)
        from itertools import zip_longest
        order = [gi for grp in zip_longest(*[by[k] for k in sorted(by)]) for gi in grp if gi is not None]
        dtl, chl = float(D[-1][0]), float(D[-1][1])
        t0, done, used = time.perf_counter(), 0, 0
        for gi in order:
            n, dx, base, _ = L2["patches"][gi]
            N = [v + 8 for v in n]
            blk = np.ascontiguousarray(L2["pool"][:, base:base + N[0] * N[1] * N[2]].reshape(9, N[2], N[1], N[0]))
            O.mhd_step(blk, list(n), 3, list(dx), dtl, chl, recon=1)
            done += n[0] * n[1] * n[2]
            used += 1
            if time.perf_counter() - t0 > 10.0:
                break
        el = time.perf_counter() - t0
        cpu = {"value": done / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"{used} finest-level patches (sizes {sorted(by)} in turn), one CTU step each, 1 thread",
               "seconds": el}
    # end to end through the public API with host buffers: every coarse step
    # copies every level's ghosted pool from pinned host memory, replays the
    # captured coarse step and reads every level's result pool back.  The
    # captured step works on fixed pools (its outputs land in some of its
    # input pools), so each step's host copies go through two device staging
    # sets on their own streams: the input of step k + 1 arrives while step k
    # computes, and the result of step k - 1 leaves meanwhile; the compute
    # stream moves staging -> pools before the replay and pools -> staging
    # after it (device copies)
    e2e = None
    if world == 1 and not args.skip_e2e:
        Hin = [torch.from_numpy(lv["pool"]).pin_memory() for lv in L]
        outs = adv.outputs()  # where the coarse step leaves each level
        Hout = [[torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs] for _ in range(2)]
        Ist = [[torch.empty_like(A[lev]) for lev in range(len(L))] for _ in range(2)]
        Ost = [[torch.empty_like(o) for o in outs] for _ in range(2)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def pipeline(K):
            for k in range(K):
                b = k % 2
                if k >= 2:
                    s_in.wait_event(ev_used[b])  # step k - 2 has taken staging input b
                with torch.cuda.stream(s_in):
                    for lev in range(len(L)):
                        Ist[b][lev].copy_(Hin[lev], non_blocking=True)
                    ev_in[b].record(s_in)
                stream.wait_event(ev_in[b])
                with torch.cuda.stream(stream):
                    for lev in range(len(L)):
                        A[lev].copy_(Ist[b][lev], non_blocking=True)
                    ev_used[b].record(stream)
                    g.replay()
                    if k >= 2:
                        stream.wait_event(ev_out[b])  # staging result b has been read back
                    for lev in range(len(L)):
                        Ost[b][lev].copy_(outs[lev], non_blocking=True)
                    ev_cmp[b].record(stream)
                s_out.wait_event(ev_cmp[b])
                with torch.cuda.stream(s_out):
                    for lev in range(len(L)):
                        Hout[b][lev].copy_(Ost[b][lev], non_blocking=True)
                    ev_out[b].record(s_out)

        pipeline(2)
        barrier()
        E = max(4, args.steps)
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(s_in)
        pipeline(E)
        t1e.record(s_out)
        barrier()
        ems = t0e.elapsed_time(t1e) / E
        # the streamed result is the device step's, bit for bit: one more
        # replay from the same input, in place (the coarse step reads no state
        # left by an earlier one, and the reflux sums in a fixed order)
        with torch.cuda.stream(stream):
            for lev in range(len(L)):
                A[lev].copy_(Hin[lev], non_blocking=True)
            g.replay()
        torch.cuda.synchronize()
        for lev in range(len(L)):
            assert torch.equal(Hout[(E - 1) % 2][lev], outs[lev].cpu()), f"level {lev}"
        e2e = {"value": upd / (ems * 1e-3), "unit": "cell-updates/s",
               "h2d_bytes_per_step": int(sum(h.numel() * 8 for h in Hin)),
               "d2h_bytes_per_step": int(sum(h.numel() * 8 for h in Hout[0])),
               "ms_per_step": ems, "steps": E,
               "overlap": "two device staging sets; every level's pool in, and the previous step's pools "
                          "out, on their own streams while the captured coarse step runs; staging <-> pools "
                          "by device copies on the compute stream"}
    launches = adv.launches()
    if rank == 0:
        line = {"metric": METRIC, "value": upd / (ms * 1e-3), "unit": "cell-updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32+f64" if prec == ctu.CTU_MIXED else "f64", "data": "synthetic",
                "config": {"workload": "batched AMR level advance: 3-level hierarchy, ratio 2, base "
                                       "128^3, PPM+HLLD+GLM, subcycled 1/2/4 in one CUDA graph, "
                                       "coarse-fine flux registers"
                                       + ("; properly nested (one coarse cell around every fine patch)"
                                          if args.amr_nested else "")
                                       + (f"; parabolic terms kappa {args.kappa} (along the field "
                                          f"{args.kappa_par or args.kappa}, phi {args.tc_phi}), nu {args.nu}, "
                                          f"eta {args.eta}"
                                          if (args.kappa or args.kappa_par or args.nu or args.eta) else ""),
                           "patches_per_level": [len(lv["patches"]) for lv in L],
                           "patch_sizes_per_level": hist, "cells_per_level": cells,
                           "cell_updates_per_coarse_step": upd, "windows_rank0": sum(len(w) for w in wins),
                           "rank0_share_of_updates": my_upd / upd,
                           "parallelism": f"patch shards x{world}" if world > 1 else "single GPU",
                           "level_ops": "ghost fill before every level step: same-level exchange from "
                                        "siblings, prolongation (in time) of the remaining coarse-fine ghosts "
                                        "on levels 1, 2; reflux + restriction at every synchronisation"
                                        if ops else "none",
                           "exchange_boxes_per_level": {lev: len(b) for lev, b in xch.items()},
                           "tiles_xw_seg": tiles,
                           "l2_flush": "inputs larger than L2"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches * args.steps, "clocks": clk,
                "kernels_ms_per_coarse_step": {k: v[0] for k, v in kern.items()},
                "status": [ctu.STATUS[x] for x in st], "gpu": torch.cuda.get_device_name(dev)}
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


def run_srmhd(args):
    """Special-relativistic jet (config: 256^3, Gamma 4/3, beam gamma 10,
    density ratio 0.01, sigma 0.1, 1% noise; MUSCL-Hancock, HLL, GLM, float64
    Newton recovery): one ctu_step_next_dt per step on one patch."""
    import torch
    from paper_1110_0740_gb300 import ctu, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    U0 = W.srmhd_jet_3d(n, seed=rank)
    U = torch.from_numpy(U0.reshape(9, -1)).to(dev)
    Uo = torch.empty_like(U)
    stride = U.shape[1]
    patches = ctu.make_patches([([n] * 3, [1.0 / n] * 3, 0)])
    res = {}
    for prec in ((ctu.CTU_MIXED, ctu.CTU_FP64) if not args.skip_other else (ctu.CTU_MIXED,)):
        c = ctu.Ctx(ctu.make_config(ndim=3, gamma=4.0 / 3.0, recon=ctu.CTU_LINEAR_MC, precision=prec,
                                    cfl=0.3, physics=ctu.CTU_SRMHD, predictor=ctu.CTU_MUSCL_HANCOCK,
                                    riemann=ctu.CTU_HLL))
        d0 = torch.zeros(2, dtype=torch.float64, device=dev)
        d1 = torch.zeros_like(d0)
        c.dt(U, stride, patches, d0)
        K = args.steps if prec == ctu.CTU_MIXED else max(2, min(args.steps, 3))
        for _ in range(args.warmup if prec == ctu.CTU_MIXED else 1):
            c.step_next_dt(U, Uo, stride, patches, d0, d1)
        torch.cuda.synchronize()
        c.profile(True)
        if prec == ctu.CTU_MIXED:
            clocks = Clocks(local)
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            c.step_next_dt(U, Uo, stride, patches, d0, d1)
        e1.record()
        torch.cuda.synchronize()
        if prec == ctu.CTU_MIXED:
            clk = clocks.stop()
        ms = e0.elapsed_time(e1) / K
        res[prec] = (ms, {k: v[0] / K for k, v in c.profile_read().items()}, c.status_sync(),
                     c.launches())
        if prec == ctu.CTU_MIXED:
            K_mixed = K
        c.close()
    ms, kern, st, nl = res[ctu.CTU_MIXED]
    roof = roofline_alu({k: (v * K_mixed, K_mixed) for k, v in kern.items()},
                        kernel_flops(n, physics="srmhd"), True)
    # the oracle on a bounded sample: a 32^3 block of the jet (its true
    # neighbours as ghosts), repeated steps for about 10 s, one host core
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        import oracle as O
        sub, g_ = min(32, n), 4
        c0 = [int(v * n) for v in (0.5, 0.5, 0.5)]
        lo = [min(max(0, c - sub // 2), n - sub) for c in c0]
        blk = U0[:, lo[2]:lo[2] + sub + 2 * g_, lo[1]:lo[1] + sub + 2 * g_, lo[0]:lo[0] + sub + 2 * g_].copy()
        dx = [1.0 / n] * 3
        m = O.srmhd_max_speed(blk, [sub] * 3, 3, dx)
        dt, chs = O.dt_ch(m, dx, 3, 0.3)
        t0, done = time.perf_counter(), 0
        while time.perf_counter() - t0 < 10.0 and done < 64:
            O.srmhd_step(blk, [sub] * 3, 3, dx, dt, chs, gamma=4.0 / 3.0)
            done += 1
        el = time.perf_counter() - t0
        cpu = {"value": sub ** 3 * done / el, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"{sub}^3 block of the {n}^3 jet, {done} CTU step(s), 1 thread", "seconds": el}
    e2e = None
    if not args.skip_e2e:
        c = ctu.Ctx(ctu.make_config(ndim=3, gamma=4.0 / 3.0, recon=ctu.CTU_LINEAR_MC, precision=ctu.CTU_MIXED,
                                    cfl=0.3, physics=ctu.CTU_SRMHD, predictor=ctu.CTU_MUSCL_HANCOCK,
                                    riemann=ctu.CTU_HLL))
        d0 = torch.zeros(2, dtype=torch.float64, device=dev)
        d1 = torch.zeros_like(d0)
        c.dt(U, stride, patches, d0)

        def barrier():
            torch.cuda.synchronize()
        e2e = e2e_stream(c, torch.from_numpy(U0.reshape(9, -1)), U, Uo, n, stride, patches, d0, d1,
                         max(4, args.steps), dev, world, barrier, lanes=args.copy_lanes)
        c.close()
    line = {"metric": METRIC, "value": world * n ** 3 / (ms * 1e-3), "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "3D SRMHD 256^3 jet, Gamma 4/3, gamma 10 beam, density ratio 0.01,"
                                   " sigma 0.1; MUSCL-Hancock, HLL, GLM, float64 Newton recovery"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "kernels_ms_per_step": kern, "gpu_launches": nl * args.steps,
            "status": ctu.STATUS[st], "gpu": torch.cuda.get_device_name(dev)}
    if ctu.CTU_FP64 in res:
        ms2, kern2, st2, _ = res[ctu.CTU_FP64]
        line["fp64_path"] = {"value": world * n ** 3 / (ms2 * 1e-3), "ms_per_step": ms2,
                             "kernels_ms_per_step": kern2, "status": ctu.STATUS[st2]}
    if rank == 0:
        print(json.dumps(line))


def run_tag(args):
    """Refinement tagging, Eq. (RefCrit), on the 256^3 blast state: one
    ctu_tag launch per step over the patch (sigma = density, then B^2/rho;
    eps 0.01, chi_r 0.1, the paper's values), L2 flushed before every launch,
    each launch timed with CUDA events on its stream.  The kernel is HBM-bound:
    algorithmic bytes are sigma's inputs over the interior plus one ghost
    layer (8 B per input variable) and one tag byte per interior cell."""
    import numpy as np
    import torch
    from paper_1110_0740_gb300 import ctu, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    U0 = W.mhd_blast_3d(n, seed=rank)
    Uh = torch.from_numpy(U0.reshape(9, -1))
    U = Uh.to(dev)
    stride = U.shape[1]
    tags = torch.zeros(stride, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    patches = ctu.make_patches([([n] * 3, [1.0 / n] * 3, 0)])
    stream = torch.cuda.current_stream()
    ctx = ctu.Ctx(ctu.make_config(ndim=3))
    peaks, src = measured_peaks()
    cells = n ** 3
    kinds = {"density": (ctu.CTU_TAG_DENSITY, 1), "B2_over_rho": (ctu.CTU_TAG_B2_OVER_RHO, 4)}
    res = {}
    clocks = Clocks(local)
    clocks.start()
    for name, (kind, nvar) in kinds.items():
        for _ in range(args.warmup):
            ctx.tag(U, stride, patches, kind, 0.01, 0.1, tags, cnt)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.tag(U, stride, patches, kind, 0.01, 0.1, tags, cnt)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / args.steps
        nbytes = 8 * nvar * (n + 2) ** 3 + cells
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "value": world * cells / (ms * 1e-3), "tagged": int(cnt.item()),
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                                  "algorithmic_bytes": nbytes, "peak_source": f"{src} hbm_gbs"}}
    clk = clocks.stop()
    st = ctx.status_sync()
    # end to end through the public API: the density plane the criterion
    # reads (the pool's first variable, contiguous) from pinned host memory,
    # the tags back to pinned host memory, every step
    rho_pin = Uh[0].pin_memory()
    th = torch.empty(stride, dtype=torch.uint8).pin_memory()
    E = max(1, args.steps)
    for it in range(E + 1):
        if it == 1:
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
        U[0].copy_(rho_pin, non_blocking=True)
        ctx.tag(U, stride, patches, ctu.CTU_TAG_DENSITY, 0.01, 0.1, tags, cnt)
        th.copy_(tags, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ems = t0.elapsed_time(t1) / E
    ctx.close()
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        import oracle as O
        m = min(96, n)
        blk = np.ascontiguousarray(U0[:, :m + 8, :m + 8, :m + 8])
        t = time.perf_counter()
        reps = 0
        while True:
            O.tag(blk, [m] * 3, 3, 0, 0.01, 0.1)
            reps += 1
            el = time.perf_counter() - t
            if el > 10.0 or reps >= 64:
                break
        cpu = {"value": reps * m ** 3 / el, "unit": "cell evaluations/s", "cores": 1, "kind": "oracle",
               "sample": f"or_tag of a {m}^3 block of the same state (density), {reps} passes",
               "seconds": el}
    if rank == 0:
        main_ = res["density"]
        line = {"metric": "refinement-criterion cell evaluations/s (Eq. RefCrit)", "value": main_["value"],
                "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": main_["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"Eq. RefCrit tags of the {n}^3 blast state, sigma = density, eps 0.01, "
                                       "chi_r 0.1", "l2_flush": "256 MB write before every launch"},
                "roofline": main_["roofline"], "b2_over_rho": res["B2_over_rho"], "tagged_cells": main_["tagged"],
                "cpu_baseline": cpu,
                "e2e": {"value": world * cells / (ems * 1e-3), "unit": "cells/s",
                        "h2d_bytes_per_step": int(stride * 8), "d2h_bytes_per_step": int(stride),
                        "ms_per_step": ems},
                "gpu_launches": args.steps, "clocks": clk, "status": ctu.STATUS[st],
                "gpu": torch.cuda.get_device_name(dev)}
        print(json.dumps(line))


def _profile_numbers(name):
    vals = {}
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    k, v = line.split()[:2]
                    vals[k] = v
    except OSError:
        pass
    return vals


def kernel_flops(n, recon="ppm", kappa=0.0, kappa_par=0.0, tc_phi=0.0, nu=0.0, eta=0.0, cells=None,
                 physics="mhd", corner="cell"):
    """Algorithmic flops per launch of each kernel group of one 3-D step on an
    n^3 patch (or on `cells` interior cells, a batch): the oracle's operation
    counts per interior cell (profiles/flops_per_cell.txt, exact-zero
    operands not counted) times the cells.  With parabolic terms par_half
    forms L_P^n and the half-step fields, the face passes evaluate every face
    flux once (one face flux is the count of the exact combination of terms
    on), par_lp differences L_P^(n+1/2), and the x sweep adds it to the
    update and the diffusion term to the next dt."""
    c = {k: float(v) for k, v in _profile_numbers("flops_per_cell.txt").items()}
    cells = float(n) ** 3 if cells is None else float(cells)
    if physics == "srmhd":
        sw = c.get("sr_sweep_per_direction", 0.0)
        return {"prim": c.get("sr_prim", 0.0) * cells, "flux1": 3 * c.get("sr_flux1_per_direction", 0.0) * cells,
                "sweep_z": sw * cells, "sweep_y": sw * cells,
                "sweep_x": (sw + c.get("update", 0.0) + c.get("sr_next_dt", 0.0)) * cells}
    sweep = c.get("sweep_per_direction_" + ("linear" if recon == "mc" else recon), 0.0)
    kp = kappa_par if kappa_par > 0 else kappa
    if corner == "mt":
        # the transverse fluxes from the normal predictor states: a predictor
        # and a Riemann problem per cell and direction in place of flux1
        pred = c.get("predict_" + ("linear" if recon == "mc" else recon), 0.0) + c.get("riemann", 0.0) + 18
        return {"prim": c.get("prim", 0.0) * cells, "pred1": 3 * pred * cells,
                "sweep_z": sweep * cells, "sweep_y": sweep * cells,
                "sweep_x": (sweep + c.get("update", 0.0) + c.get("next_dt", 0.0)) * cells}
    if not (kappa or kappa_par or nu or eta):
        # sweeps run z, y, x; the x sweep finishes the update and the next dt
        return {"prim": c.get("prim", 0.0) * cells, "flux1": 3 * c.get("flux1_per_direction", 0.0) * cells,
                "sweep_z": sweep * cells, "sweep_y": sweep * cells,
                "sweep_x": (sweep + c.get("update", 0.0) + c.get("next_dt", 0.0)) * cells}
    # one face flux with every term on, counted together
    cond = "none"
    if kappa or kp:
        cond = ("sat_" if tc_phi else "") + ("aniso" if kp != kappa else ("" if tc_phi else "cond"))
        cond = cond.rstrip("_")
    face = c.get(f"par_mask_{cond}_{1 if nu else 0}_{1 if eta else 0}", 0.0)
    m = 1 + (3 if nu else 0) + (3 if eta else 0)
    swp = sweep + m * c.get("sweep_par_per_component", 0.0)
    # the face passes evaluate every face once (three per cell); the half-step
    # kernel and par_lp difference them, and the x sweep adds L_P^(n+1/2) to
    # its update
    half = (c.get("par_half_per_cell", 0.0) + m * c.get("par_half_per_component", 0.0)
            + (c.get("par_half_visc", 0.0) if nu else 0.0))
    upd = m * c.get("par_update_per_component", 0.0)
    nxt = c.get("next_dt", 0.0) + c.get("par_update_diffusion_number", 0.0)
    return {"prim": c.get("prim", 0.0) * cells, "flux1": 3 * c.get("flux1_per_direction", 0.0) * cells,
            "par_faces_n": 3 * face * cells, "par_half": half * cells, "par_faces_h": 3 * face * cells,
            "par_lp": upd * cells, "sweep_z": swp * cells, "sweep_y": swp * cells,
            "sweep_x": (swp + c.get("update", 0.0) + nxt) * cells}


def precision_split_roofline(n, cells_per_s, hbm_gbs):
    """Whole-step roofline of the mixed path with the method's work split by
    the precision it is designated: the float64 work is the pressure
    recoveries (cell centres, six interface states, the next-step speed),
    the six interface prim->cons conversions and the update; the rest is
    float32 (oracle counts, profiles/flops_per_cell.txt).  The bound is the
    slowest of FP32 flops / FP32 peak, FP64 flops / FP64 peak and the
    algorithmic bytes / measured HBM bandwidth, in cell updates per second.
    This implementation runs the float64-designated recoveries in
    double-float arithmetic on the FP32 pipe, so it is not held to the FP64
    term; the fraction is reported beside the kernel roofline."""
    c = {k: float(v) for k, v in _profile_numbers("flops_per_cell.txt").items()}
    total = c.get("step_total_ppm", 0.0)
    f64 = (8 * c.get("cons2prim", 0.0) + 6 * c.get("prim2cons", 0.0) + c.get("update", 0.0))
    f32 = total - f64
    bpc = algorithmic_bytes(n) / float(n) ** 3
    bounds = {"fp32": FP32_PEAK / f32 if f32 > 0 else float("inf"),
              "fp64": FP64_PEAK / f64 if f64 > 0 else float("inf"),
              "hbm": hbm_gbs * 1e9 / bpc}
    binding = min(bounds, key=bounds.get)
    return {"fp32_flops_per_cell": f32, "fp64_flops_per_cell": f64, "bytes_per_cell": bpc,
            "bounds_cells_per_s": bounds, "binding": binding, "achieved_cells_per_s": cells_per_s,
            "frac": cells_per_s / bounds[binding]}


STEP_SOURCES = ("df.cuh", "mhd_device.cuh", "srmhd_device.cuh", "ctu_kernels.cuh", "ctu_launch.h",
                "ctu_launch.cuh", "par_ops.cuh", "ctu_f32.cu", "_build.py")


def kernel_source_hash():
    """Hash of the sources the step's kernels are compiled from (with the
    build flags), so that recorded per-kernel traffic stays valid across
    changes elsewhere in the library."""
    import hashlib
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1110_0740_gb300")
    for f in STEP_SOURCES:
        path = os.path.join(pkg, f) if f == "_build.py" else os.path.join(pkg, "csrc", f)
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(name, n):
    """DRAM bytes (read + write) per launch of `name` on an n^3 patch, scaled
    by cells from the ncu capture recorded in profiles/dram_traffic.txt; None
    if there is no record or the kernel sources changed since it was taken."""
    t = _profile_numbers("dram_traffic.txt")
    if t.get("source_hash") != kernel_source_hash() or f"{name}_bytes_per_cell" not in t:
        return None
    return float(t[f"{name}_bytes_per_cell"]) * float(n) ** 3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "iface64"])
    ap.add_argument("--n", type=int, default=N_CELLS)
    ap.add_argument("--other-steps", type=int, default=3)
    ap.add_argument("--skip-other", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-level-ops", action="store_true",
                    help="amr: advance the levels without prolongation, restriction and reflux")
    ap.add_argument("--amr-nested", action="store_true",
                    help="amr: the seeded hierarchy with proper nesting (every coarse face beside a fine "
                         "patch refluxed)")
    ap.add_argument("--riemann", default="hlld", choices=["hlld", "hllc"],
                    help="blast: the Riemann solver (the workload uses HLLD)")
    ap.add_argument("--kappa", type=float, default=0.0,
                    help="blast, amr: thermal conduction with this conductivity (0 = off)")
    ap.add_argument("--nu", type=float, default=0.0,
                    help="blast, amr: viscosity with this kinematic viscosity (0 = off)")
    ap.add_argument("--kappa-par", type=float, default=0.0,
                    help="blast, amr: thermal conductivity along the field, --kappa then across it "
                         "(0 = isotropic)")
    ap.add_argument("--tc-phi", type=float, default=0.0,
                    help="blast, amr: saturation parameter phi of the heat flux (0 = classical)")
    ap.add_argument("--eta", type=float, default=0.0,
                    help="blast, amr: resistivity with this magnetic diffusivity (0 = off)")
    ap.add_argument("--shock", type=float, default=0.0,
                    help="blast: the hybrid integration with this shock threshold (thermal pressure; 0 = off)")
    ap.add_argument("--recon", default="ppm", choices=sorted(RECONS),
                    help="blast: reconstruction of the characteristic variables (the workload uses ppm)")
    ap.add_argument("--copy-lanes", type=int, default=1,
                    help="streams per copy direction in the end-to-end leg (each copy split by variable)")
    ap.add_argument("--corner", default="cell", choices=["cell", "mt"],
                    help="transverse fluxes from cell-centred states (Eq. transv) or the normal predictor states")
    ap.add_argument("--config", default="blast", choices=["blast", "amr", "srmhd", "tag"],
                    help="blast: the 256^3 headline workload; amr: batched AMR level advance; "
                         "srmhd: relativistic jet; tag: refinement tagging of the 256^3 state")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "amr":
        run_amr(args)
    elif args.config == "srmhd":
        run_srmhd(args)
    elif args.config == "tag":
        run_tag(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
