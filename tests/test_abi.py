"""The C ABI library loads and exports every function include/ctu.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        txt = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ctu_\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1110_0740_gb300 import _build
    lib = _build.build()
    L = ctypes.CDLL(str(lib))
    names = declared()
    assert {"ctu_init", "ctu_dt", "ctu_step", "ctu_flux_registers", "ctu_status_sync",
            "ctu_step_noalloc"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_1110_0740_gb300 import ctu
    assert ctu.ctu_strerror(0) == "ok"
    assert "invalid" in ctu.ctu_strerror(1)
