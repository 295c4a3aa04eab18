"""The C ABI library loads and exports every function include/ctu.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared(header="ctu.h"):
    txt = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / header).read_text(), flags=re.S)
    return {m.group(1) for m in
            re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ctu_\w+)\s*\(", txt, re.M)}


def test_every_header_is_checked():
    assert sorted(h.name for h in (ROOT / "include").glob("*.h")) == ["ctu.h", "ctu_peaks.h"]


def test_library_exports_every_declared_symbol():
    from paper_1110_0740_gb300 import _build
    lib = _build.build()
    L = ctypes.CDLL(str(lib))
    names = declared("ctu.h")
    assert {"ctu_init", "ctu_dt", "ctu_step", "ctu_flux_registers", "ctu_status_sync",
            "ctu_step_noalloc"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_measurement_library_is_separate():
    """The FMA microbenchmark lives in libctu_peaks.so, not in libctu.so."""
    from paper_1110_0740_gb300 import _build
    _build.build()
    P = ctypes.CDLL(str(_build.LIB_PEAKS))
    assert declared("ctu_peaks.h") == {"ctu_fma_peak"}
    assert hasattr(P, "ctu_fma_peak")
    assert not hasattr(ctypes.CDLL(str(_build.LIB)), "ctu_fma_peak")


def test_strerror_without_gpu():
    from paper_1110_0740_gb300 import ctu
    assert ctu.ctu_strerror(0) == "ok"
    assert "invalid" in ctu.ctu_strerror(1)


def test_floor_config_validation_without_gpu():
    """Host-side validation of the floors returns before any CUDA call:
    a negative or infinite floor is CTU_EINVAL, a floor with the
    relativistic physics or with the allocation-free step CTU_EUNSUPPORTED."""
    import ctypes
    from paper_1110_0740_gb300 import ctu
    L = ctu._lib()
    h = ctypes.c_void_p()
    for pf, rf in ((-1.0, 0.0), (0.0, -0.5), (float("inf"), 0.0), (0.0, float("nan"))):
        cfg = ctu.make_config(p_floor=pf, rho_floor=rf)
        assert L.ctu_init(ctypes.byref(cfg), ctypes.byref(h)) == ctu.STATUS.index("CTU_EINVAL")
    cfg = ctu.make_config(physics=ctu.CTU_SRMHD, predictor=ctu.CTU_MUSCL_HANCOCK, riemann=ctu.CTU_HLL,
                          recon=ctu.CTU_LINEAR_MC, gamma=4.0 / 3.0, p_floor=1e-6)
    assert L.ctu_init(ctypes.byref(cfg), ctypes.byref(h)) == ctu.STATUS.index("CTU_EUNSUPPORTED")
    cfg = ctu.make_config(rho_floor=1e-6)
    patches = ctu.make_patches([([8, 8, 8], [0.1] * 3, 0)])
    st = L.ctu_step_noalloc(ctypes.byref(cfg), 16, 32, 4096, patches, 1, 48, 0, 0)
    assert st == ctu.STATUS.index("CTU_EUNSUPPORTED")


def test_parabolic_config_validation_without_gpu():
    """Host-side validation of the parabolic terms returns before any CUDA
    call: a negative, infinite or NaN conductivity, viscosity or resistivity is
    CTU_EINVAL; either term outside ideal MHD with PPM or MC-linear, HLLD, trace modes ALL or UPWIND,
    no hybrid integration and FP64 or CTU_MIXED is CTU_EUNSUPPORTED, and so is
    the allocation-free step with either."""
    import ctypes
    from paper_1110_0740_gb300 import ctu
    L = ctu._lib()
    h = ctypes.c_void_p()
    for k in (-1e-3, float("inf"), float("nan")):
        for kw in (dict(kappa=k), dict(nu=k), dict(eta=k), dict(kappa_par=k), dict(tc_phi=k)):
            cfg = ctu.make_config(**kw)
            assert L.ctu_init(ctypes.byref(cfg), ctypes.byref(h)) == ctu.STATUS.index("CTU_EINVAL")
    bad = (dict(recon=ctu.CTU_WENO3), dict(recon=ctu.CTU_LINEAR_MINMOD), dict(trace_mode=ctu.CTU_TRACE_CENTER),
           dict(riemann=ctu.CTU_HLLC), dict(shock=(5.0, 0)), dict(precision=ctu.CTU_MIXED_IFACE64),
           dict(physics=ctu.CTU_SRMHD, predictor=ctu.CTU_MUSCL_HANCOCK, riemann=ctu.CTU_HLL,
                recon=ctu.CTU_LINEAR_MC, gamma=4.0 / 3.0))
    for kw in bad:
        for par in (dict(kappa=0.01), dict(nu=0.01), dict(eta=0.01), dict(kappa_par=0.01)):
            cfg = ctu.make_config(**par, **kw)
            assert L.ctu_init(ctypes.byref(cfg), ctypes.byref(h)) == ctu.STATUS.index("CTU_EUNSUPPORTED"), kw
    patches = ctu.make_patches([([8, 8, 8], [0.1] * 3, 0)])
    for par in (dict(kappa=0.01), dict(nu=0.01), dict(eta=0.01), dict(kappa_par=0.01)):
        cfg = ctu.make_config(**par)
        st = L.ctu_step_noalloc(ctypes.byref(cfg), 16, 32, 4096, patches, 1, 48, 0, 0)
        assert st == ctu.STATUS.index("CTU_EUNSUPPORTED")
