"""Thin ctypes binding of libctu.so (the C ABI in include/ctu.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device arrays are passed as torch CUDA tensors (or raw
integer device addresses); torch provides device memory and streams.  If the
library is missing this module raises at load time -- there is no fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

from . import _build

# ---------------------------------------------------------------- ABI structs

CTU_MHD, CTU_SRMHD = 0, 1
CTU_EOS_IDEAL, CTU_EOS_TM = 0, 1
CTU_LINEAR_MC, CTU_PPM = 0, 1
CTU_LINEAR_MINMOD, CTU_LINEAR_HARMONIC, CTU_LINEAR_VANALBADA, CTU_WENO3 = 2, 3, 4, 5
CTU_CHAR_TRACE, CTU_MUSCL_HANCOCK = 0, 1
CTU_HLLD, CTU_HLL, CTU_HLLC = 0, 1, 2
CTU_FP64, CTU_MIXED, CTU_MIXED_IFACE64 = 0, 1, 2
CTU_TRACE_ALL, CTU_TRACE_UPWIND, CTU_TRACE_CENTER, CTU_TRACE_CW84 = 0, 1, 2, 3
CTU_CORNER_CELL, CTU_CORNER_MT = 0, 1
CTU_TAG_DENSITY, CTU_TAG_ENERGY, CTU_TAG_B2_OVER_RHO, CTU_TAG_E_OVER_RHO = 0, 1, 2, 3

STATUS = ["CTU_OK", "CTU_EINVAL", "CTU_ENOMEM", "CTU_ECUDA", "CTU_EUNSUPPORTED", "CTU_ENEGATIVE",
          "CTU_ENAN", "CTU_ERECOVERY", "CTU_ESUPERLUMINAL", "CTU_ETIMEOUT", "CTU_ETOOLARGE"]


class ctu_config(ctypes.Structure):
    _fields_ = [("physics", ctypes.c_int), ("eos", ctypes.c_int), ("gamma", ctypes.c_double),
                ("ndim", ctypes.c_int), ("recon", ctypes.c_int), ("predictor", ctypes.c_int),
                ("riemann", ctypes.c_int), ("precision", ctypes.c_int), ("cfl", ctypes.c_double),
                ("glm_alpha", ctypes.c_double), ("nghost", ctypes.c_int),
                ("trace_mode", ctypes.c_int), ("p_floor", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("shock_detect", ctypes.c_int), ("shock_q", ctypes.c_int),
                ("shock_eps", ctypes.c_double), ("kappa", ctypes.c_double),
                ("nu", ctypes.c_double), ("eta", ctypes.c_double), ("kappa_par", ctypes.c_double),
                ("tc_phi", ctypes.c_double), ("corner", ctypes.c_int)]


class ctu_patch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("dx", ctypes.c_double * 3), ("base", ctypes.c_int64),
                ("level", ctypes.c_int32), ("flags", ctypes.c_int32)]


class ctu_flux_window(ctypes.Structure):
    _fields_ = [("patch", ctypes.c_int32), ("dir", ctypes.c_int32), ("plane", ctypes.c_int32),
                ("a0", ctypes.c_int32), ("a1", ctypes.c_int32), ("b0", ctypes.c_int32),
                ("b1", ctypes.c_int32), ("pad", ctypes.c_int32), ("weight", ctypes.c_double),
                ("dst", ctypes.c_int64)]


class ctu_copy_box(ctypes.Structure):
    _fields_ = [("dn", ctypes.c_int32 * 3), ("sn", ctypes.c_int32 * 3), ("lo", ctypes.c_int32 * 3),
                ("hi", ctypes.c_int32 * 3), ("shift", ctypes.c_int32 * 3), ("pad", ctypes.c_int32),
                ("dbase", ctypes.c_int64), ("sbase", ctypes.c_int64)]


def make_copy_boxes(boxes):
    """boxes: dicts with dn, sn, lo, hi, shift, dbase, sbase (exchange.plan)."""
    arr = (ctu_copy_box * len(boxes))()
    for i, b in enumerate(boxes):
        for k in ("dn", "sn", "lo", "hi", "shift"):
            getattr(arr[i], k)[:] = [int(v) for v in b[k]]
        arr[i].pad = 0
        arr[i].dbase = int(b["dbase"])
        arr[i].sbase = int(b["sbase"])
    return arr


class ctu_level_box(ctypes.Structure):
    _fields_ = [("fn", ctypes.c_int32 * 3), ("cn", ctypes.c_int32 * 3), ("fbase", ctypes.c_int64),
                ("cbase", ctypes.c_int64), ("lo", ctypes.c_int32 * 3), ("hi", ctypes.c_int32 * 3),
                ("origin", ctypes.c_int32 * 3), ("ratio", ctypes.c_int32), ("phys", ctypes.c_int32)]


class ctu_reflux_set(ctypes.Structure):
    _fields_ = [("cn", ctypes.c_int32 * 3), ("dir", ctypes.c_int32), ("plane", ctypes.c_int32),
                ("side", ctypes.c_int32), ("cbase", ctypes.c_int64), ("dx", ctypes.c_double * 3),
                ("a0", ctypes.c_int32), ("a1", ctypes.c_int32), ("b0", ctypes.c_int32),
                ("b1", ctypes.c_int32), ("creg", ctypes.c_int64), ("freg", ctypes.c_int64),
                ("fa0", ctypes.c_int32), ("fb0", ctypes.c_int32), ("fna", ctypes.c_int32),
                ("fnb", ctypes.c_int32), ("ratio", ctypes.c_int32), ("pad", ctypes.c_int32)]


def make_level_boxes(boxes):
    """boxes: iterables of dicts with keys fn, cn, fbase, cbase, lo, hi, origin, ratio
    and optionally phys (the physical-boundary bits of ctu_prolong, default 0)."""
    arr = (ctu_level_box * len(boxes))()
    for i, b in enumerate(boxes):
        for k in ("fn", "cn", "lo", "hi", "origin"):
            getattr(arr[i], k)[:] = [int(v) for v in b[k]]
        arr[i].fbase, arr[i].cbase, arr[i].ratio = int(b["fbase"]), int(b["cbase"]), int(b["ratio"])
        arr[i].phys = int(b.get("phys", 0))
    return arr


def make_reflux_sets(sets):
    """sets: dicts with keys cn, dir, plane, side, cbase, dx, a0, a1, b0, b1, creg, freg, fa0, fb0,
    fna, fnb, ratio."""
    arr = (ctu_reflux_set * len(sets))()
    for i, d in enumerate(sets):
        arr[i].cn[:] = [int(v) for v in d["cn"]]
        arr[i].dx[:] = [float(v) for v in (list(d["dx"]) + [1.0] * (3 - len(d["dx"])))]
        for k in ("dir", "plane", "side", "cbase", "a0", "a1", "b0", "b1", "creg", "freg", "fa0", "fb0",
                  "fna", "fnb", "ratio"):
            setattr(arr[i], k, int(d[k]))
        arr[i].pad = 0
    return arr


class CtuError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        name = STATUS[code] if 0 <= code < len(STATUS) else str(code)
        super().__init__(f"{where}: {name} ({_lib().ctu_strerror(code).decode()})")


_L = None


def lib_path() -> Path:
    return _build.LIB


def _lib():
    global _L
    if _L is None:
        p = _build.LIB
        if not p.exists():
            raise RuntimeError(f"libctu.so not built at {p}: run __graft_entry__.build()")
        L = ctypes.CDLL(str(p))
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.ctu_init.argtypes = [ctypes.POINTER(ctu_config), ctypes.POINTER(vp)]
        L.ctu_dt.argtypes = [vp, vp, i64, ctypes.POINTER(ctu_patch), i32, vp, vp, vp]
        L.ctu_step.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctu_patch), i32, vp, vp]
        L.ctu_step_next_dt.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctu_patch), i32, vp, vp, vp]
        L.ctu_step_next_dt.restype = i32
        L.ctu_flux_registers.argtypes = [vp, vp, ctypes.POINTER(ctu_flux_window), i32]
        L.ctu_fill_periodic.argtypes = [vp, vp, i64, ctypes.POINTER(ctu_patch), i32, vp]
        L.ctu_status_sync.argtypes = [vp, vp]
        L.ctu_floor_count.argtypes = [vp, ctypes.POINTER(i64), vp]
        L.ctu_copy.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctu_copy_box), i32, vp]
        L.ctu_pack.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctu_copy_box), i32, vp]
        L.ctu_unpack.argtypes = [vp, vp, i64, vp, ctypes.POINTER(ctu_copy_box), i32, vp]
        L.ctu_tag.argtypes = [vp, vp, i64, ctypes.POINTER(ctu_patch), i32, i32, dbl, dbl, vp, vp, vp, vp]
        L.ctu_destroy.argtypes = [vp]
        L.ctu_destroy.restype = None
        L.ctu_strerror.argtypes = [i32]
        L.ctu_strerror.restype = ctypes.c_char_p
        L.ctu_last_launch_count.argtypes = [vp]
        L.ctu_profile.argtypes = [vp, i32]
        L.ctu_profile.restype = i32
        L.ctu_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]
        L.ctu_profile_read.restype = i32
        L.ctu_step_noalloc.argtypes = [ctypes.POINTER(ctu_config), vp, vp, i64,
                                       ctypes.POINTER(ctu_patch), i32, vp, i32, vp]
        L.ctu_step_noalloc.restype = i32
        L.ctu_autotune.argtypes = [vp, vp, vp, i64, ctypes.POINTER(ctu_patch), i32, vp, vp]
        L.ctu_autotune.restype = i32
        L.ctu_tile_params.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
        L.ctu_tile_params.restype = i32
        L.ctu_prolong.argtypes = [vp, vp, vp, i64, dbl, vp, i64, ctypes.POINTER(ctu_level_box), i32, vp]
        L.ctu_prolong.restype = i32
        L.ctu_restrict.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(ctu_level_box), i32, vp]
        L.ctu_restrict.restype = i32
        L.ctu_reflux.argtypes = [vp, vp, i64, vp, ctypes.POINTER(ctu_reflux_set), i32, vp]
        L.ctu_reflux.restype = i32
        L.ctu_diagnostics.argtypes = [vp, vp, i64, ctypes.POINTER(ctu_patch), i32, vp, vp]
        L.ctu_diagnostics.restype = i32
        for f in ("ctu_init", "ctu_dt", "ctu_step", "ctu_flux_registers", "ctu_fill_periodic",
                  "ctu_status_sync", "ctu_last_launch_count"):
            getattr(L, f).restype = i32
        _L = L
    return _L


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _check(code, where):
    if code != 0:
        raise CtuError(code, where)


def make_config(ndim=3, gamma=5.0 / 3.0, recon=CTU_PPM, precision=CTU_FP64, cfl=0.3,
                glm_alpha=0.1, trace_mode=CTU_TRACE_ALL, physics=CTU_MHD, riemann=CTU_HLLD,
                predictor=CTU_CHAR_TRACE, eos=CTU_EOS_IDEAL, p_floor=0.0, rho_floor=0.0, shock=None,
                kappa=0.0, nu=0.0, eta=0.0, kappa_par=0.0, tc_phi=0.0, corner=CTU_CORNER_CELL):
    """shock: None (off) or (eps_q, q) for the hybrid integration, q = 0
    thermal or 1 magnetic pressure.  kappa: isotropic thermal conductivity,
    nu: kinematic viscosity, eta: resistivity (0 = off); kappa_par: the
    conductivity along the field, kappa then across it (0 = isotropic);
    tc_phi: saturation parameter of the heat flux (0 = classical); corner:
    CTU_CORNER_CELL or CTU_CORNER_MT (transverse fluxes from the normal
    predictor states)."""
    return ctu_config(physics=physics, eos=eos, gamma=gamma, ndim=ndim, recon=recon,
                      predictor=predictor, riemann=riemann, precision=precision, cfl=cfl,
                      glm_alpha=glm_alpha, nghost=4, trace_mode=trace_mode, p_floor=p_floor,
                      rho_floor=rho_floor, shock_detect=0 if shock is None else 1,
                      shock_q=0 if shock is None else int(shock[1]),
                      shock_eps=0.0 if shock is None else float(shock[0]), kappa=float(kappa), nu=float(nu), eta=float(eta),
                      kappa_par=float(kappa_par), tc_phi=float(tc_phi), corner=int(corner))


def make_patches(specs):
    """specs: iterable of (n(3), dx(3), base[, level])."""
    specs = list(specs)
    arr = (ctu_patch * len(specs))()
    for i, s in enumerate(specs):
        n, dx, base = s[0], s[1], s[2]
        arr[i].n[:] = [int(v) for v in n]
        arr[i].dx[:] = [float(v) for v in dx]
        arr[i].base = int(base)
        arr[i].level = int(s[3]) if len(s) > 3 else 0
        arr[i].flags = 0
    return arr


# ---------------------------------------------------------------- C-ABI mirrors

def ctu_init(cfg: ctu_config):
    h = ctypes.c_void_p()
    _check(_lib().ctu_init(ctypes.byref(cfg), ctypes.byref(h)), "ctu_init")
    return h


def ctu_step_noalloc(cfg, U_in, U_out, stride, patches, d_dt_ch, wait_status=True, stream=None):
    """Allocation-free step (see include/ctu.h); returns the status code
    instead of raising, so callers can see CTU_ETOOLARGE."""
    return _lib().ctu_step_noalloc(ctypes.byref(cfg), _ptr(U_in), _ptr(U_out), int(stride), patches,
                                   len(patches), _ptr(d_dt_ch), int(bool(wait_status)),
                                   _stream(stream))


def ctu_destroy(ctx):
    _lib().ctu_destroy(ctx)


def ctu_dt(ctx, U, stride, patches, d_dt_ch, h_dt_ch=None, stream=None):
    _check(_lib().ctu_dt(ctx, _ptr(U), int(stride), patches, len(patches), _ptr(d_dt_ch),
                         h_dt_ch, _stream(stream)), "ctu_dt")


def ctu_step(ctx, U_in, U_out, stride, patches, d_dt_ch, stream=None):
    _check(_lib().ctu_step(ctx, _ptr(U_in), _ptr(U_out), int(stride), patches, len(patches),
                           _ptr(d_dt_ch), _stream(stream)), "ctu_step")


def ctu_step_next_dt(ctx, U_in, U_out, stride, patches, d_dt_ch, d_dt_ch_next, stream=None):
    _check(_lib().ctu_step_next_dt(ctx, _ptr(U_in), _ptr(U_out), int(stride), patches,
                                   len(patches), _ptr(d_dt_ch), _ptr(d_dt_ch_next),
                                   _stream(stream)), "ctu_step_next_dt")


def ctu_autotune(ctx, U_in, U_out, stride, patches, d_dt_ch, stream=None):
    _check(_lib().ctu_autotune(ctx, _ptr(U_in), _ptr(U_out), int(stride), patches, len(patches),
                               _ptr(d_dt_ch), _stream(stream)), "ctu_autotune")


def ctu_tile_params(ctx, n):
    """(tile width along x, marching segment) used for interior shape n."""
    arr = (ctypes.c_int * 3)(*[int(v) for v in n])
    xw, seg = ctypes.c_int(), ctypes.c_int()
    _check(_lib().ctu_tile_params(ctx, arr, ctypes.byref(xw), ctypes.byref(seg)), "ctu_tile_params")
    return xw.value, seg.value


def ctu_prolong(ctx, Uc_old, Uc_new, cstride, alpha, Uf, fstride, boxes, stream=None):
    _check(_lib().ctu_prolong(ctx, _ptr(Uc_old), _ptr(Uc_new), int(cstride), float(alpha), _ptr(Uf),
                              int(fstride), boxes, len(boxes), _stream(stream)), "ctu_prolong")


def ctu_restrict(ctx, Uc, cstride, Uf, fstride, boxes, stream=None):
    _check(_lib().ctu_restrict(ctx, _ptr(Uc), int(cstride), _ptr(Uf), int(fstride), boxes, len(boxes),
                               _stream(stream)), "ctu_restrict")


def ctu_reflux(ctx, Uc, cstride, reg, sets, stream=None):
    _check(_lib().ctu_reflux(ctx, _ptr(Uc), int(cstride), _ptr(reg), sets, len(sets), _stream(stream)),
           "ctu_reflux")


def ctu_diagnostics(ctx, U, stride, patches, d_out, stream=None):
    _check(_lib().ctu_diagnostics(ctx, _ptr(U), int(stride), patches, len(patches), _ptr(d_out),
                                  _stream(stream)), "ctu_diagnostics")


def ctu_flux_registers(ctx, reg, windows):
    if reg is None or not windows:
        _check(_lib().ctu_flux_registers(ctx, None, None, 0), "ctu_flux_registers")
        return
    arr = (ctu_flux_window * len(windows))()
    for i, w in enumerate(windows):
        (arr[i].patch, arr[i].dir, arr[i].plane, arr[i].a0, arr[i].a1, arr[i].b0, arr[i].b1) = \
            [int(v) for v in w[:7]]
        arr[i].weight = float(w[7])
        arr[i].dst = int(w[8])
    _check(_lib().ctu_flux_registers(ctx, _ptr(reg), arr, len(windows)), "ctu_flux_registers")


def ctu_fill_periodic(ctx, U, stride, patches, stream=None):
    _check(_lib().ctu_fill_periodic(ctx, _ptr(U), int(stride), patches, len(patches),
                                    _stream(stream)), "ctu_fill_periodic")


def ctu_status_sync(ctx, stream=None):
    return _lib().ctu_status_sync(ctx, _stream(stream))


def ctu_tag(ctx, U, stride, patches, sigma, eps, chi_r, tags, d_count=None, chi=None, stream=None):
    _check(_lib().ctu_tag(ctx, _ptr(U), int(stride), patches, len(patches), int(sigma), float(eps),
                          float(chi_r), _ptr(tags), _ptr(d_count) if d_count is not None else None,
                          _ptr(chi) if chi is not None else None, _stream(stream)), "ctu_tag")


_LP = None


def _peaks_lib():
    """The measurement library libctu_peaks.so (include/ctu_peaks.h), built
    beside libctu.so."""
    global _LP
    if _LP is None:
        p = _build.LIB_PEAKS
        if not p.exists():
            raise RuntimeError(f"libctu_peaks.so not built at {p}: run __graft_entry__.build()")
        L = ctypes.CDLL(str(p))
        L.ctu_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        L.ctu_fma_peak.restype = ctypes.c_int
        _LP = L
    return _LP


def ctu_fma_peak(fp64, iters=1 << 16, stream=None):
    """Measured FMA throughput (flop/s) of the float32 or float64 pipe
    (measurement aid from libctu_peaks.so, not part of libctu.so)."""
    v = ctypes.c_double(0.0)
    _check(_peaks_lib().ctu_fma_peak(int(bool(fp64)), int(iters), ctypes.byref(v), _stream(stream)),
           "ctu_fma_peak")
    return v.value


def ctu_copy(ctx, U_dst, dstride, U_src, sstride, boxes, stream=None):
    _check(_lib().ctu_copy(ctx, _ptr(U_dst), int(dstride), _ptr(U_src), int(sstride), boxes, len(boxes),
                           _stream(stream)), "ctu_copy")


def ctu_pack(ctx, buf, U_src, sstride, boxes, stream=None):
    _check(_lib().ctu_pack(ctx, _ptr(buf), _ptr(U_src), int(sstride), boxes, len(boxes), _stream(stream)),
           "ctu_pack")


def ctu_unpack(ctx, U_dst, dstride, buf, boxes, stream=None):
    _check(_lib().ctu_unpack(ctx, _ptr(U_dst), int(dstride), _ptr(buf), boxes, len(boxes), _stream(stream)),
           "ctu_unpack")


def ctu_floor_count(ctx, stream=None):
    """Cells the floors changed since the last call (resets; synchronises)."""
    c = ctypes.c_int64(0)
    _check(_lib().ctu_floor_count(ctx, ctypes.byref(c), _stream(stream)), "ctu_floor_count")
    return int(c.value)


def ctu_last_launch_count(ctx):
    return _lib().ctu_last_launch_count(ctx)


def ctu_profile(ctx, enable):
    _check(_lib().ctu_profile(ctx, int(bool(enable))), "ctu_profile")


def ctu_profile_read(ctx):
    """{kernel name: (total ms, launches)} since profiling was enabled."""
    L = _lib()
    n = L.ctu_profile_read(ctx, -1, None, None, None)
    out = {}
    for i in range(n):
        nm, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_longlong()
        L.ctu_profile_read(ctx, i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(cnt))
        out[nm.value.decode()] = (ms.value, cnt.value)
    return out


def ctu_strerror(code):
    return _lib().ctu_strerror(code).decode()


class Ctx:
    """Owning wrapper of a ctu_ctx with the same calls as methods."""

    def __init__(self, cfg: ctu_config):
        self.cfg = cfg
        self.h = ctu_init(cfg)

    def close(self):
        if self.h:
            ctu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dt(self, U, stride, patches, d_dt_ch, h_dt_ch=None, stream=None):
        ctu_dt(self.h, U, stride, patches, d_dt_ch, h_dt_ch, stream)

    def step(self, U_in, U_out, stride, patches, d_dt_ch, stream=None):
        ctu_step(self.h, U_in, U_out, stride, patches, d_dt_ch, stream)

    def step_next_dt(self, U_in, U_out, stride, patches, d_dt_ch, d_dt_ch_next, stream=None):
        ctu_step_next_dt(self.h, U_in, U_out, stride, patches, d_dt_ch, d_dt_ch_next, stream)

    def flux_registers(self, reg, windows):
        ctu_flux_registers(self.h, reg, windows)

    def autotune(self, U_in, U_out, stride, patches, d_dt_ch, stream=None):
        ctu_autotune(self.h, U_in, U_out, stride, patches, d_dt_ch, stream)

    def tile_params(self, n):
        return ctu_tile_params(self.h, n)

    def prolong(self, Uc_old, Uc_new, cstride, alpha, Uf, fstride, boxes, stream=None):
        ctu_prolong(self.h, Uc_old, Uc_new, cstride, alpha, Uf, fstride, boxes, stream)

    def restrict(self, Uc, cstride, Uf, fstride, boxes, stream=None):
        ctu_restrict(self.h, Uc, cstride, Uf, fstride, boxes, stream)

    def reflux(self, Uc, cstride, reg, sets, stream=None):
        ctu_reflux(self.h, Uc, cstride, reg, sets, stream)

    def diagnostics(self, U, stride, patches, d_out, stream=None):
        ctu_diagnostics(self.h, U, stride, patches, d_out, stream)

    def fill_periodic(self, U, stride, patches, stream=None):
        ctu_fill_periodic(self.h, U, stride, patches, stream)

    def status_sync(self, stream=None):
        return ctu_status_sync(self.h, stream)

    def tag(self, U, stride, patches, sigma, eps, chi_r, tags, d_count=None, chi=None, stream=None):
        ctu_tag(self.h, U, stride, patches, sigma, eps, chi_r, tags, d_count, chi, stream)

    def copy(self, U_dst, dstride, U_src, sstride, boxes, stream=None):
        ctu_copy(self.h, U_dst, dstride, U_src, sstride, boxes, stream)

    def pack(self, buf, U_src, sstride, boxes, stream=None):
        ctu_pack(self.h, buf, U_src, sstride, boxes, stream)

    def unpack(self, U_dst, dstride, buf, boxes, stream=None):
        ctu_unpack(self.h, U_dst, dstride, buf, boxes, stream)

    def floor_count(self, stream=None):
        return ctu_floor_count(self.h, stream)

    def launches(self):
        return ctu_last_launch_count(self.h)

    def profile(self, enable=True):
        ctu_profile(self.h, enable)

    def profile_read(self):
        return ctu_profile_read(self.h)
