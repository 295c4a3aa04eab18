"""Host-side pieces of bench.py, without a GPU: the algorithmic bytes of a
step against their closed form (151 B per cell update for the 256^3 patch:
the ghosted state read once and the interior written once, 9 float64
variables, plus the flux registers), and the reference arm's JSON line
(the CPU oracle timed on a bounded sample) with the keys the line must
carry."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_closed_form():
    sys.path.insert(0, ROOT)
    import bench
    n = 256
    per_cell = bench.algorithmic_bytes(n) / n ** 3
    # 72 ((n + 8)^3 + n^3) / n^3 = 150.96, registers 6 * 9 * 8 * 2 / n = 3.4
    assert per_cell == pytest.approx(72 * (264 ** 3 + 256 ** 3) / 256 ** 3 + 6 * 9 * 8 * 2 / 256, rel=1e-15)
    assert abs(per_cell - 6 * 9 * 8 * 2 / 256 - 151) < 0.1


@pytest.mark.parametrize("terms", [dict(kappa=1e-3), dict(kappa=1e-3, kappa_par=1e-2),
                                   dict(kappa=1e-3, tc_phi=1e-2), dict(kappa=1e-3, kappa_par=1e-2, tc_phi=1e-2),
                                   dict(nu=1e-3), dict(eta=1e-3), dict(kappa=1e-3, nu=1e-3, eta=1e-3)])
def test_kernel_flops_parabolic(terms):
    """Every kernel group a step with parabolic terms launches has a flop
    count, and the step's total is the plain step's plus the parabolic work:
    L_P twice (three faces each), the half-step state, the predictor terms
    and the diffusion number of the next dt."""
    sys.path.insert(0, ROOT)
    import bench
    c = {k: float(v) for k, v in bench._profile_numbers("flops_per_cell.txt").items()}
    plain = bench.kernel_flops(1, "ppm")
    fl = bench.kernel_flops(1, "ppm", **terms)
    for k in ("prim", "flux1", "par_faces_n", "par_half", "par_faces_h", "par_lp", "sweep_z", "sweep_y", "sweep_x"):
        assert fl[k] > 0, k
    kappa, kp = terms.get("kappa", 0.0), terms.get("kappa_par", 0.0) or terms.get("kappa", 0.0)
    cond = "none"
    if kappa:
        cond = {(False, False): "cond", (True, False): "aniso", (False, True): "sat",
                (True, True): "sat_aniso"}[(kp != kappa, bool(terms.get("tc_phi")))]
    # the face flux of the exact combination of terms, counted together
    face = c[f"par_mask_{cond}_{int(bool(terms.get('nu')))}_{int(bool(terms.get('eta')))}"]
    # one term alone: its combination count is its own line
    if sum(bool(terms.get(k)) for k in ("nu", "eta")) + (cond != "none") == 1:
        single = (c["par_face_" + cond] if cond != "none" else 0.0) + \
            (c["par_face_visc"] if terms.get("nu") else 0.0) + (c["par_face_res"] if terms.get("eta") else 0.0)
        assert face == single
    m = 1 + 3 * bool(terms.get("nu")) + 3 * bool(terms.get("eta"))
    extra = (6 * face + m * (c["par_half_per_component"] + c["par_update_per_component"]
                             + 3 * c["sweep_par_per_component"])
             + c["par_half_per_cell"] + c["par_update_diffusion_number"] + (c["par_half_visc"] if terms.get("nu") else 0))
    assert sum(fl.values()) == pytest.approx(sum(plain.values()) + extra, rel=1e-12)
    # the counted face work of each term is not trivial
    assert face >= 3


def test_kernel_flops_srmhd_and_batches():
    """The relativistic step's groups take the relativistic counts, and a
    batch's flops scale with its interior cells."""
    sys.path.insert(0, ROOT)
    import bench
    c = {k: float(v) for k, v in bench._profile_numbers("flops_per_cell.txt").items()}
    sr = bench.kernel_flops(1, physics="srmhd")
    assert sum(sr.values()) == pytest.approx(c["sr_step_total"], rel=1e-3)
    assert bench.kernel_flops(4, cells=1000)["sweep_y"] == pytest.approx(1000 * bench.kernel_flops(1)["sweep_y"])


def test_reference_arm_json_line():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "MHD cell-updates/s per CTU step" and d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "sample" in d["config"] and d["steps"] == 1 and d["warmup"] == 1
