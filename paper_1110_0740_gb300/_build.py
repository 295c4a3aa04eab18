"""Build libctu.so for sm_103a with nvcc (translation units in parallel)."""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libctu.so"
SOURCES = ["ctu_api.cu", "ctu_f64.cu", "ctu_f32.cu", "ctu_f32i.cu", "ctu_sr32.cu", "ctu_noalloc.cu",
           "ctu_var32.cu", "ctu_var64.cu", "ctu_ref32.cu", "ctu_ref64.cu", "ctu_hyb32.cu",
           "ctu_hyb64.cu", "ctu_hllc32.cu", "ctu_hllc64.cu", "ctu_par32.cu", "ctu_par64.cu", "ctu_mt32.cu",
           "ctu_mt64.cu"]
# The FMA-throughput microbenchmark (include/ctu_peaks.h) is a measurement aid
# for the roofline, built as a library of its own beside libctu.so.
PEAK_SOURCES = ["peaks/fma_peak.cu"]
LIB_PEAKS = OUT_DIR / "libctu_peaks.so"
# The float32 stages of the mixed paths divide and take square roots with the
# approximate hardware forms (<= 2 ulp) and flush float32 denormals; float64
# arithmetic is unaffected by these flags.
FLOAT_FAST = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
SOURCE_FLAGS = {"ctu_f32.cu": FLOAT_FAST, "ctu_f32i.cu": FLOAT_FAST, "ctu_sr32.cu": FLOAT_FAST,
                "ctu_var32.cu": FLOAT_FAST, "ctu_ref32.cu": FLOAT_FAST, "ctu_hyb32.cu": FLOAT_FAST,
                "ctu_hllc32.cu": FLOAT_FAST, "ctu_par32.cu": FLOAT_FAST, "ctu_mt32.cu": FLOAT_FAST}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def flags(extra=()):
    env = os.environ.get("CTU_NVCC_EXTRA", "").split()
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", str(ROOT / "include"), "-I", str(CSRC)] + env + list(extra)


def _link(objs, out):
    tmp = OUT_DIR / f"{out.stem}.{os.getpid()}.so"
    subprocess.run([nvcc(), "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + ["-lcudart"],
                   check=True)
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, extra=()) -> Path:
    """Build libctu.so (and the measurement library libctu_peaks.so); returns
    the path of libctu.so."""
    OUT_DIR.mkdir(exist_ok=True)
    deps = [CSRC / s for s in SOURCES + PEAK_SOURCES] + list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) \
        + list((ROOT / "include").glob("*.h"))
    if LIB.exists() and LIB_PEAKS.exists() and not force and not extra:
        if min(LIB.stat().st_mtime, LIB_PEAKS.stat().st_mtime) >= max(p.stat().st_mtime for p in deps):
            return LIB
    objs = []
    procs = []
    for s in SOURCES + PEAK_SOURCES:
        o = OUT_DIR / (Path(s).stem + ".o")
        cmd = [nvcc(), "-c", str(CSRC / s), "-o", str(o)] + SOURCE_FLAGS.get(s, []) + flags(extra)
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            print(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    npk = len(PEAK_SOURCES)
    _link(objs[:-npk], LIB)
    _link(objs[-npk:], LIB_PEAKS)
    return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
