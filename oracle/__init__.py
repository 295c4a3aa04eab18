"""Plain FP64 CPU oracle of the CTU-MHD patch step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA path never does, and nothing
here imports the CUDA path: the two share no code.  The arithmetic lives in
``ctu_oracle.c`` (the scheme of Mignone et al., Sections 3-4),
``srmhd_oracle.c`` (its relativistic counterpart), ``amr_oracle.c`` (the
level operators of Section 4: prolongation, restriction, reflux) and
``exact_euler.c`` (the exact Euler Riemann solution used to pin it); this
module only compiles them with ``gcc -O2 -ffp-contract=off`` and marshals
numpy arrays through ctypes.

Array convention: a patch is a C-contiguous float64 array of shape
``(9, NZ, NY, NX)`` with ``N = n + 2*g`` per dimension, ``g = 4`` for active
dimensions and 0 for inactive ones (``n = 1`` there).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
LIB_PATH = HERE / "liboracle.so"
SOURCES = ["ctu_oracle.c", "exact_euler.c", "srmhd_oracle.c", "amr_oracle.c"]
NG = 4
NVAR = 9

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle into ``oracle/liboracle.so``."""
    srcs = [HERE / s for s in SOURCES if (HERE / s).exists()]
    if LIB_PATH.exists() and not force:
        newest = max(p.stat().st_mtime for p in srcs)
        if LIB_PATH.stat().st_mtime >= newest:
            return LIB_PATH
    tmp = LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
           "-fPIC", "-shared", "-o", str(tmp)] + [str(s) for s in srcs] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB_PATH))
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        L.or_mhd_step.restype = I
        L.or_mhd_step.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, D, I, I,
                                  ctypes.POINTER(ctypes.c_long), P, I, P]
        L.or_mhd_floor.restype = ctypes.c_long
        L.or_mhd_floor.argtypes = [P, I, I, I, I, D, D, D]
        L.or_mhd_step_ex.restype = I
        L.or_mhd_step_ex.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, D, I, I,
                                     ctypes.POINTER(ctypes.c_long), P, I, P, I, I, D, I]
        L.or_mhd_step_mt.restype = I
        L.or_mhd_step_mt.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, D, I, I,
                                     ctypes.POINTER(ctypes.c_long), P, I, P, I, I, D, I]
        L.or_mhd_step_tc.restype = I
        L.or_mhd_step_tc.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, D, I, I,
                                     ctypes.POINTER(ctypes.c_long), P, I, P, I, I, D, I, D]
        L.or_mhd_step_par.restype = I
        L.or_mhd_step_par.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, D, I, I,
                                      ctypes.POINTER(ctypes.c_long), P, I, P, I, I, D, I, D, D, D, D, D]
        L.or_mhd_max_rate.restype = D
        L.or_mhd_max_rate.argtypes = [P, I, I, I, I, D, D, D, D, D]
        L.or_mhd_max_rate_par.restype = D
        L.or_mhd_max_rate_par.argtypes = [P, I, I, I, I, D, D, D, D, D, D, D, D]
        L.or_mhd_parabolic.restype = None
        L.or_mhd_parabolic.argtypes = [P, I, I, I, I, D, D, D, D, D, D, D, D, D, P]
        L.or_mhd_conduction.restype = None
        L.or_mhd_conduction.argtypes = [P, I, I, I, I, D, D, D, D, D, P]
        L.or_mhd_riemann_hllc.restype = I
        L.or_mhd_riemann_hllc.argtypes = [P, P, D, D, P]
        L.or_mhd_riemann_hll.restype = I
        L.or_mhd_riemann_hll.argtypes = [P, P, D, D, P]
        L.or_mhd_shock_flags.restype = None
        L.or_mhd_shock_flags.argtypes = [P, I, I, I, I, D, D, D, D, D, I, I, ctypes.POINTER(ctypes.c_ubyte)]
        L.or_mhd_max_speed.restype = D
        L.or_mhd_max_speed.argtypes = [P, I, I, I, I, D, D, D, D]
        L.or_mhd_eigen.restype = None
        L.or_mhd_eigen.argtypes = [P, D, D, P, P, P]
        L.or_mhd_riemann.restype = I
        L.or_mhd_riemann.argtypes = [P, P, D, D, P]
        L.or_mhd_char_predict.restype = None
        L.or_mhd_char_predict.argtypes = [P, D, D, D, I, I, P, P]
        L.or_mhd_char_predict_dx.restype = None
        L.or_mhd_char_predict_dx.argtypes = [P, D, D, D, D, I, I, P, P]
        L.or_mhd_prim2cons.restype = None
        L.or_mhd_prim2cons.argtypes = [P, D, P]
        L.or_mhd_cons2prim.restype = I
        L.or_mhd_cons2prim.argtypes = [P, D, P]
        L.or_mhd_cfast.restype = D
        L.or_mhd_cfast.argtypes = [P, D]
        L.or_euler_sample.restype = I
        L.or_euler_sample.argtypes = [D, D, D, D, D, D, D, D, P]
        if hasattr(L, "or_srmhd_step"):
            L.or_srmhd_step.restype = I
            L.or_srmhd_step.argtypes = [P, P, I, I, I, I, D, D, D, D, D, D, D,
                                        ctypes.POINTER(ctypes.c_long), P, I, P]
            L.or_srmhd_max_speed.restype = D
            L.or_srmhd_max_speed.argtypes = [P, I, I, I, I, D, D, D, D]
            L.or_srmhd_prim2cons.restype = None
            L.or_srmhd_prim2cons.argtypes = [P, D, P]
            L.or_srmhd_cons2prim.restype = I
            L.or_srmhd_cons2prim.argtypes = [P, D, P]
            L.or_srmhd_fast_speeds.restype = None
            L.or_srmhd_fast_speeds.argtypes = [P, D, P, P]
            L.or_srmhd_riemann.restype = I
            L.or_srmhd_riemann.argtypes = [P, P, D, D, P]
            L.or_srmhd_mh_predict.restype = I
            L.or_srmhd_mh_predict.argtypes = [P, P, D, D, D, P, P]
        I3 = ctypes.POINTER(ctypes.c_int)
        L.or_prolong.restype = None
        L.or_prolong.argtypes = [P, P, I3, D, P, I3, I3, I3, I3, I, I, I]
        L.or_restrict.restype = None
        L.or_restrict.argtypes = [P, I3, P, I3, I3, I3, I3, I, I]
        L.or_diagnostics.restype = None
        LP = ctypes.POINTER(ctypes.c_long)
        for f in ("or_copy_boxes", "or_pack_boxes", "or_unpack_boxes"):
            getattr(L, f).restype = None
        L.or_copy_boxes.argtypes = [P, ctypes.c_long, P, ctypes.c_long, I3, LP, LP, I, I]
        L.or_pack_boxes.argtypes = [P, P, ctypes.c_long, I3, LP, I, I]
        L.or_unpack_boxes.argtypes = [P, ctypes.c_long, P, I3, LP, I, I]
        L.or_tag.restype = ctypes.c_long
        L.or_tag.argtypes = [P, I3, I, I, D, D, P, ctypes.POINTER(ctypes.c_ubyte)]
        L.or_diagnostics.argtypes = [P, I3, I, P, P]
        L.or_reflux.restype = None
        L.or_reflux.argtypes = [P, I3, P, P, I, I, I, I, I, I, I, ctypes.c_long, ctypes.c_long,
                                I, I, I, I, I, I]
        _lib = L
    return _lib


def _i3(v):
    return (ctypes.c_int * 3)(*[int(x) for x in v])


# ---------------------------------------------------------------- level operators

def prolong(Uc_old, Uc_new, nc, alpha, Uf, nf, lo, hi, origin, ratio, ndim, phys=0):
    """Eq. (prolong) + (intalpha): fill the fine cells [lo, hi) of Uf (in place)
    from the coarse patch at U* = (1 - alpha) Uc_old + alpha Uc_new; fine cell
    x lies in coarse cell origin + floor(x / ratio).  phys: bit 2d (2d + 1)
    when the coarse patch's first (last) cell along d touches the domain
    boundary, where the slope is one-sided."""
    Uco = np.ascontiguousarray(Uc_old, dtype=np.float64)
    Ucn = np.ascontiguousarray(Uc_new, dtype=np.float64)
    assert Uco.shape == shape(nc, ndim) and Ucn.shape == Uco.shape and Uf.shape == shape(nf, ndim)
    assert Uf.flags.c_contiguous and Uf.dtype == np.float64
    lib().or_prolong(_dp(Uco), _dp(Ucn), _i3(nc), float(alpha), _dp(Uf), _i3(nf), _i3(lo), _i3(hi),
                     _i3(origin), int(ratio), int(ndim), int(phys))
    return Uf


def restrict(Uc, nc, Uf, nf, lo, hi, origin, ratio, ndim):
    """Eq. (avgdown): coarse cells [lo, hi) of Uc (in place) become the mean of
    their ratio^ndim fine cells (c - origin) * ratio + k."""
    Ufc = np.ascontiguousarray(Uf, dtype=np.float64)
    assert Uc.shape == shape(nc, ndim) and Ufc.shape == shape(nf, ndim)
    assert Uc.flags.c_contiguous and Uc.dtype == np.float64
    lib().or_restrict(_dp(Uc), _i3(nc), _dp(Ufc), _i3(nf), _i3(lo), _i3(hi), _i3(origin), int(ratio),
                      int(ndim))
    return Uc


def _boxes(boxes):
    """boxes: dicts with dn, sn, lo, hi, shift (3 ints each), dbase, sbase."""
    nb = len(boxes)
    b = np.zeros((max(1, nb), 16), dtype=np.int32)
    db = np.zeros(max(1, nb), dtype=np.int64)
    sb = np.zeros(max(1, nb), dtype=np.int64)
    for i, x in enumerate(boxes):
        b[i, 0:3], b[i, 3:6], b[i, 6:9], b[i, 9:12], b[i, 12:15] = x["dn"], x["sn"], x["lo"], x["hi"], x["shift"]
        db[i], sb[i] = x["dbase"], x["sbase"]
    LP = ctypes.POINTER(ctypes.c_long)
    return (b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), db.ctypes.data_as(LP), sb.ctypes.data_as(LP),
            (b, db, sb))


def copy_boxes(Ud, Us, boxes, ndim):
    """Same-level ghost exchange copy (or_copy_boxes) between float64 pools
    [9][stride] (Ud may be Us)."""
    assert Ud.dtype == np.float64 and Ud.flags.c_contiguous and Us.flags.c_contiguous
    bp, dp, sp, keep = _boxes(boxes)
    lib().or_copy_boxes(_dp(Ud), Ud.shape[1], _dp(Us), Us.shape[1], bp, dp, sp, len(boxes), int(ndim))


def box_cells(b):
    return int(np.prod([h - l for l, h in zip(b["lo"], b["hi"])]))


def pack_boxes(Us, boxes, ndim):
    buf = np.zeros(NVAR * sum(box_cells(b) for b in boxes))
    bp, dp, sp, keep = _boxes(boxes)
    lib().or_pack_boxes(_dp(buf), _dp(Us), Us.shape[1], bp, sp, len(boxes), int(ndim))
    return buf


def unpack_boxes(Ud, buf, boxes, ndim):
    bp, dp, sp, keep = _boxes(boxes)
    lib().or_unpack_boxes(_dp(Ud), Ud.shape[1], _dp(np.ascontiguousarray(buf)), bp, dp, len(boxes), int(ndim))


def tag(U, n, ndim, kind, eps, chi_r):
    """Eq. (RefCrit) refinement tags of one ghost-filled patch: returns
    (tag uint8, chi float64, count), both arrays in the ghosted layout with
    only interior entries written (tag 0 and chi 0 elsewhere).  kind: 0
    density, 1 total energy, 2 B^2/rho, 3 E/rho."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == shape(n, ndim)
    chi = np.zeros(U.shape[1:])
    t = np.zeros(U.shape[1:], dtype=np.uint8)
    cnt = lib().or_tag(_dp(U), _i3(n), int(ndim), int(kind), float(eps), float(chi_r), _dp(chi),
                       t.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return t, chi, int(cnt)


def diagnostics(U, n, ndim, dx):
    """Conserved totals (sum of U_q times the cell volume over the interior,
    q = 0..8) and max |div B| (central differences): an array of 10."""
    Uc = np.ascontiguousarray(U, dtype=np.float64)
    assert Uc.shape == shape(n, ndim)
    out = np.zeros(10)
    d = list(dx) + [1.0] * (3 - len(dx))
    lib().or_diagnostics(_dp(Uc), _i3(n), int(ndim), (ctypes.c_double * 3)(*d), _dp(out))
    return out


def reflux(Uc, nc, dxc, reg, dir, plane, side, a0, a1, b0, b1, creg, freg, fa0, fb0, fna, fnb, ratio, ndim):
    """Eq. (fluxcorr) + (addreflux) on the coarse faces [a0, a1) x [b0, b1) of
    plane `plane` normal to `dir` (in place); see amr_oracle.c."""
    regc = np.ascontiguousarray(reg, dtype=np.float64)
    assert Uc.shape == shape(nc, ndim) and Uc.flags.c_contiguous
    dx = list(dxc) + [1.0] * (3 - len(dxc))
    lib().or_reflux(_dp(Uc), _i3(nc), (ctypes.c_double * 3)(*dx), _dp(regc), int(dir), int(plane), int(side),
                    int(a0), int(a1), int(b0), int(b1), int(creg), int(freg), int(fa0), int(fb0), int(fna),
                    int(fnb), int(ratio), int(ndim))
    return Uc


# ---------------------------------------------------------------- geometry

def ghosts(ndim: int):
    return [NG if d < ndim else 0 for d in range(3)]


def shape(n, ndim):
    """Ghosted array shape (9, NZ, NY, NX) of a patch with interior n=(nx,ny,nz)."""
    g = ghosts(ndim)
    return (NVAR, n[2] + 2 * g[2], n[1] + 2 * g[1], n[0] + 2 * g[0])


def interior(A, n, ndim):
    g = ghosts(ndim)
    return A[..., g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]


def fill_periodic(U, n, ndim):
    """Fill the ghost cells of U in place with periodic copies."""
    g = ghosts(ndim)
    for d in range(ndim):
        ax = 3 - d
        nd, gd = n[d], g[d]
        sl = [slice(None)] * 4
        src = [slice(None)] * 4
        sl[ax] = slice(0, gd)
        src[ax] = slice(nd, nd + gd)
        U[tuple(sl)] = U[tuple(src)]
        sl[ax] = slice(nd + gd, nd + 2 * gd)
        src[ax] = slice(gd, 2 * gd)
        U[tuple(sl)] = U[tuple(src)]
    return U


def fill_outflow(U, n, ndim):
    """Zero-gradient ghost cells (copy of the nearest interior layer)."""
    g = ghosts(ndim)
    for d in range(ndim):
        ax = 3 - d
        nd, gd = n[d], g[d]
        for k in range(gd):
            sl = [slice(None)] * 4
            src = [slice(None)] * 4
            sl[ax] = k
            src[ax] = gd
            U[tuple(sl)] = U[tuple(src)]
            sl[ax] = nd + gd + k
            src[ax] = nd + gd - 1
            U[tuple(sl)] = U[tuple(src)]
    return U


# ---------------------------------------------------------------- MHD step

def mhd_step(U, n, ndim, dx, dt, ch, gamma=5.0 / 3.0, glm_alpha=0.1, recon=1,
             windows=None, reg=None, upwind=0, shock=None, riemann=0, kappa=0.0, nu=0.0, eta=0.0,
             kappa_par=None, phi=0.0, corner=0):
    """One CTU step of a ghost-filled patch; returns (Unew, n_bad_states).

    corner = 1: the transverse fluxes from the normal predictor states (the
    corner coupling of Mignone & Tzeferacos, or_mhd_step_mt; no parabolic
    terms); 0: from the cell-centred states (Eq. transv).

    windows: optional list of (d, f, a0, a1, b0, b1, dst, weight) flux-register
    windows accumulated into the float64 array `reg` (see or_mhd_step).
    kappa > 0: with isotropic thermal conduction; nu > 0: with isotropic
    viscosity; eta > 0: with resistivity (or_mhd_step_par).  kappa_par: the
    conductivity along the field (None: kappa, isotropic); phi > 0: the
    saturated heat flux."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == shape(n, ndim), (U.shape, shape(n, ndim))
    Un = np.empty_like(U)
    dx = list(dx) + [1.0] * (3 - len(dx))
    nwin = 0 if windows is None else len(windows)
    win = np.zeros(max(1, 7 * nwin), dtype=np.int64)
    wgt = np.zeros(max(1, nwin))
    for i, w in enumerate(windows or []):
        win[7 * i:7 * i + 7] = w[:7]
        wgt[i] = w[7]
    regp = None
    if nwin:
        assert reg.dtype == np.float64 and reg.flags.c_contiguous
        regp = _dp(reg)
    sh = (0, 0.0, 0) if shock is None else (1, float(shock[0]), int(shock[1]))
    args = (_dp(U), _dp(Un), int(n[0]), int(n[1]), int(n[2]), int(ndim),
            float(dx[0]), float(dx[1]), float(dx[2]), float(dt), float(ch),
            float(gamma), float(glm_alpha), int(recon), int(upwind),
            win.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(wgt),
            nwin, regp, int(riemann), *sh)
    kpar = kappa if kappa_par is None else kappa_par
    if corner:
        assert not (kappa > 0.0 or nu > 0.0 or eta > 0.0 or kpar > 0.0), "corner coupling with Pi = 0 only"
        bad = lib().or_mhd_step_mt(*args)
    elif nu > 0.0 or eta > 0.0 or kpar != kappa or phi > 0.0:
        bad = lib().or_mhd_step_par(*args, float(kappa), float(kpar), float(phi), float(nu), float(eta))
    elif kappa > 0.0:
        bad = lib().or_mhd_step_tc(*args, float(kappa))
    else:
        bad = lib().or_mhd_step_ex(*args)
    return Un, bad


def mhd_shock_flags(U, n, ndim, dx, eps_q=5.0, qkind=0, reach=2, gamma=5.0 / 3.0):
    """Flags of the hybrid integration (or_mhd_shock_flags), uint8 in the
    ghosted layout: bit 1 shocked (HLL at its faces), bit 2 MinMod."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    dx = list(dx) + [1.0] * (3 - len(dx))
    f = np.zeros(U.shape[1:], dtype=np.uint8)
    lib().or_mhd_shock_flags(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim), float(dx[0]), float(dx[1]),
                             float(dx[2]), float(gamma), float(eps_q), int(qkind), int(reach),
                             f.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return f


def mhd_riemann_hllc(VL, VR, gamma, ch):
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    F = np.zeros(NVAR)
    lib().or_mhd_riemann_hllc(_dp(VL), _dp(VR), float(gamma), float(ch), _dp(F))
    return F


def mhd_riemann_hll(VL, VR, gamma, ch):
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    F = np.zeros(NVAR)
    lib().or_mhd_riemann_hll(_dp(VL), _dp(VR), float(gamma), float(ch), _dp(F))
    return F


def mhd_floor(U, n, ndim, p_floor, rho_floor, gamma=5.0 / 3.0):
    """The optional floors of the updated state (see or_mhd_floor), applied in
    place to the interior cells of U; returns the number of floored cells."""
    assert U.dtype == np.float64 and U.flags.c_contiguous and U.shape == shape(n, ndim)
    return int(lib().or_mhd_floor(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim), float(gamma),
                                  float(p_floor), float(rho_floor)))


def boundary_windows(n, ndim, weight=1.0, base=0):
    """Windows covering the 2*ndim boundary faces of a patch, stored one after
    another from offset `base` in the order x-, x+, y-, y+, z-, z+."""
    out = []
    off = base
    for d in range(ndim):
        a, b = [e for e in range(3) if e != d]
        for f in (0, n[d]):
            out.append((d, f, 0, n[a], 0, n[b], off, weight))
            off += NVAR * n[a] * n[b]
    return out, off - base


def mhd_max_speed(U, n, ndim, dx, gamma=5.0 / 3.0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    dx = list(dx) + [1.0] * (3 - len(dx))
    return lib().or_mhd_max_speed(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim),
                                  float(dx[0]), float(dx[1]), float(dx[2]), float(gamma))


def mhd_max_rate(U, n, ndim, dx, gamma=5.0 / 3.0, kappa=0.0, nu=0.0, eta=0.0, kappa_par=None):
    """Eq. (Ca)'s max over interior cells of max_d (|v_d| + c_f,d)/dx_d
    + sum_d 2 D / dx_d^2, D = max((Gamma - 1) max(kappa, kappa_par) / rho,
    (4/3) nu, eta)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    dx = list(dx) + [1.0] * (3 - len(dx))
    kpar = kappa if kappa_par is None else kappa_par
    if nu > 0.0 or eta > 0.0 or kpar != kappa:
        return lib().or_mhd_max_rate_par(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim), float(dx[0]),
                                         float(dx[1]), float(dx[2]), float(gamma), float(kappa), float(kpar),
                                         float(nu), float(eta))
    return lib().or_mhd_max_rate(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim),
                                 float(dx[0]), float(dx[1]), float(dx[2]), float(gamma), float(kappa))


def mhd_parabolic(U, n, ndim, dx, kappa, nu, gamma=5.0 / 3.0, eta=0.0, kappa_par=None, phi=0.0):
    """L_P of conduction, viscosity and resistivity (or_mhd_parabolic) on the
    interior cells: array of the shape of U, momentum in components 1..3,
    energy in 4 and B in 5..7 (the rest and the ghosts 0)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    dx = list(dx) + [1.0] * (3 - len(dx))
    LP = np.zeros(U.shape)
    lib().or_mhd_parabolic(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim), float(dx[0]), float(dx[1]),
                           float(dx[2]), float(gamma), float(kappa),
                           float(kappa if kappa_par is None else kappa_par), float(phi), float(nu), float(eta),
                           _dp(LP))
    return LP


def mhd_conduction(U, n, ndim, dx, kappa, gamma=5.0 / 3.0):
    """L_P of isotropic thermal conduction (or_mhd_conduction) on the interior
    cells, in the ghosted layout (ghost entries 0)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    dx = list(dx) + [1.0] * (3 - len(dx))
    LP = np.zeros(U.shape[1:])
    lib().or_mhd_conduction(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim), float(dx[0]), float(dx[1]),
                            float(dx[2]), float(gamma), float(kappa), _dp(LP))
    return LP


def dt_ch(max_speed, dx, ndim, cfl):
    """dt = C_a / max_d(lambda_d/dx_d) (Eq. Ca) and c_h = C_a min(dx) / dt."""
    dt = cfl / max_speed
    ch = cfl * min(dx[:ndim]) / dt
    return dt, ch


def mhd_eigen(V, gamma, ch):
    V = np.ascontiguousarray(V, dtype=np.float64)
    lam = np.zeros(NVAR)
    L = np.zeros((NVAR, NVAR))
    R = np.zeros((NVAR, NVAR))
    lib().or_mhd_eigen(_dp(V), float(gamma), float(ch), _dp(lam), _dp(L), _dp(R))
    return lam, L, R


def mhd_riemann(VL, VR, gamma, ch):
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    F = np.zeros(NVAR)
    lib().or_mhd_riemann(_dp(VL), _dp(VR), float(gamma), float(ch), _dp(F))
    return F


def mhd_char_predict(vs, gamma, ch, dtdx, recon, upwind=0, dx=0.0):
    """Normal predictor of one cell (or_mhd_char_predict_dx); recon 0 MC,
    1 PPM, 2 MinMod, 3 harmonic, 4 Van Albada, 5 WENO3 (uses dx)."""
    vs = np.ascontiguousarray(vs, dtype=np.float64).reshape(5, NVAR)
    Vp = np.zeros(NVAR)
    Vm = np.zeros(NVAR)
    lib().or_mhd_char_predict_dx(_dp(vs), float(gamma), float(ch), float(dtdx), float(dx), int(recon),
                                 int(upwind), _dp(Vp), _dp(Vm))
    return Vp, Vm


def mhd_prim2cons(V, gamma):
    V = np.ascontiguousarray(V, dtype=np.float64)
    U = np.zeros(NVAR)
    lib().or_mhd_prim2cons(_dp(V), float(gamma), _dp(U))
    return U


def mhd_cons2prim(U, gamma):
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.zeros(NVAR)
    bad = lib().or_mhd_cons2prim(_dp(U), float(gamma), _dp(V))
    return V, bad


def mhd_cfast(Vloc, gamma):
    Vloc = np.ascontiguousarray(Vloc, dtype=np.float64)
    return lib().or_mhd_cfast(_dp(Vloc), float(gamma))


def euler_sample(left, right, gamma, xi):
    """Exact Euler Riemann solution (rho, u, p) at xi = x/t; xi may be an array."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((xi.size, 3))
    o = np.zeros(3)
    for i, x in enumerate(xi):
        it = lib().or_euler_sample(float(left[0]), float(left[1]), float(left[2]),
                                   float(right[0]), float(right[1]), float(right[2]),
                                   float(gamma), float(x), _dp(o))
        if it < 0:
            raise ValueError("vacuum generated")
        out[i] = o
    return out


def mhd_run(U, n, ndim, dx, steps, cfl, gamma=5.0 / 3.0, glm_alpha=0.1, recon=1,
            bc="periodic", t_end=None, upwind=0, shock=None, riemann=0, kappa=0.0, nu=0.0, eta=0.0,
            kappa_par=None, phi=0.0, corner=0):
    """Advance a patch `steps` CTU steps (or up to t_end), filling ghosts each
    step; returns (U, t, dts)."""
    U = np.array(U, dtype=np.float64, copy=True)
    fill = fill_periodic if bc == "periodic" else fill_outflow
    t = 0.0
    dts = []
    k = 0
    while True:
        if t_end is None and k >= steps:
            break
        if t_end is not None and t >= t_end * (1 - 1e-14):
            break
        fill(U, n, ndim)
        par = kappa > 0.0 or nu > 0.0 or eta > 0.0 or (kappa_par or 0.0) > 0.0
        m = (mhd_max_rate(U, n, ndim, dx, gamma, kappa, nu, eta, kappa_par) if par
             else mhd_max_speed(U, n, ndim, dx, gamma))
        dt, ch = dt_ch(m, list(dx), ndim, cfl)
        if t_end is not None and t + dt > t_end:
            dt = t_end - t
        U, bad = mhd_step(U, n, ndim, dx, dt, ch, gamma, glm_alpha, recon, upwind=upwind, shock=shock,
                          riemann=riemann, kappa=kappa, nu=nu, eta=eta, kappa_par=kappa_par, phi=phi,
                          corner=corner)
        if bad:
            raise FloatingPointError(f"oracle met {bad} unphysical states at step {k}")
        t += dt
        dts.append((dt, ch))
        k += 1
    fill(U, n, ndim)
    return U, t, dts


# ---------------------------------------------------------------- SRMHD

def _windows(windows):
    nwin = 0 if windows is None else len(windows)
    win = np.zeros(max(1, 7 * nwin), dtype=np.int64)
    wgt = np.zeros(max(1, nwin))
    for i, w in enumerate(windows or []):
        win[7 * i:7 * i + 7] = w[:7]
        wgt[i] = w[7]
    return nwin, win, wgt


def srmhd_step(U, n, ndim, dx, dt, ch, gamma=4.0 / 3.0, glm_alpha=0.1, windows=None, reg=None):
    """One SRMHD CTU step (MUSCL-Hancock, HLL, GLM); returns (Unew, n_bad)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == shape(n, ndim)
    Un = np.empty_like(U)
    dx = list(dx) + [1.0] * (3 - len(dx))
    nwin, win, wgt = _windows(windows)
    regp = _dp(reg) if nwin else None
    bad = lib().or_srmhd_step(_dp(U), _dp(Un), int(n[0]), int(n[1]), int(n[2]), int(ndim),
                              float(dx[0]), float(dx[1]), float(dx[2]), float(dt), float(ch),
                              float(gamma), float(glm_alpha),
                              win.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(wgt),
                              nwin, regp)
    return Un, bad


def srmhd_max_speed(U, n, ndim, dx, gamma=4.0 / 3.0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    dx = list(dx) + [1.0] * (3 - len(dx))
    return lib().or_srmhd_max_speed(_dp(U), int(n[0]), int(n[1]), int(n[2]), int(ndim),
                                    float(dx[0]), float(dx[1]), float(dx[2]), float(gamma))


def srmhd_prim2cons(V, gamma):
    V = np.ascontiguousarray(V, dtype=np.float64)
    U = np.zeros(NVAR)
    lib().or_srmhd_prim2cons(_dp(V), float(gamma), _dp(U))
    return U


def srmhd_cons2prim(U, gamma):
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.zeros(NVAR)
    st = lib().or_srmhd_cons2prim(_dp(U), float(gamma), _dp(V))
    return V, st


def srmhd_fast_speeds(Vloc, gamma):
    Vloc = np.ascontiguousarray(Vloc, dtype=np.float64)
    lm, lp = ctypes.c_double(), ctypes.c_double()
    lib().or_srmhd_fast_speeds(_dp(Vloc), float(gamma), ctypes.byref(lm), ctypes.byref(lp))
    return lm.value, lp.value


def srmhd_riemann(VL, VR, gamma, ch):
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    F = np.zeros(NVAR)
    lib().or_srmhd_riemann(_dp(VL), _dp(VR), float(gamma), float(ch), _dp(F))
    return F


def srmhd_run(U, n, ndim, dx, steps, cfl, gamma=4.0 / 3.0, glm_alpha=0.1, bc="periodic",
              t_end=None):
    U = np.array(U, dtype=np.float64, copy=True)
    fill = fill_periodic if bc == "periodic" else fill_outflow
    t, k, dts = 0.0, 0, []
    while True:
        if t_end is None and k >= steps:
            break
        if t_end is not None and t >= t_end * (1 - 1e-14):
            break
        fill(U, n, ndim)
        m = srmhd_max_speed(U, n, ndim, dx, gamma)
        if m < 0:
            raise FloatingPointError("oracle recovery failed")
        dt, ch = dt_ch(m, list(dx), ndim, cfl)
        if t_end is not None and t + dt > t_end:
            dt = t_end - t
        U, bad = srmhd_step(U, n, ndim, dx, dt, ch, gamma, glm_alpha)
        if bad:
            raise FloatingPointError(f"oracle met {bad} unphysical states at step {k}")
        t += dt
        dts.append((dt, ch))
        k += 1
    fill(U, n, ndim)
    return U, t, dts
