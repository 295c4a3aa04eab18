"""Seeded synthetic inputs for the CTU-MHD step (shared by tests and bench).

This module only builds initial data: smooth random fields from Fourier
modes, a vector-potential magnetic field, a pressure sphere, and the
periodic ghost frame.  It holds none of the scheme's arithmetic; the only
physics it writes out is the definition of the initial conserved state from
the primitive one (ideal-gas total energy, Section 2.1 of the paper), which
defines the test problem.  Both the CUDA path and the CPU oracle receive the
same float64 arrays from here.

Layout: ``(9, NZ, NY, NX)`` float64, conservative variables
(rho, mx, my, mz, E, Bx, By, Bz, psi), 4 ghost cells per side in each active
dimension, x fastest.
"""
from __future__ import annotations

import numpy as np

NG = 4
NVAR = 9


def ghosted(n, ndim):
    g = [NG if d < ndim else 0 for d in range(3)]
    return (NVAR, n[2] + 2 * g[2], n[1] + 2 * g[1], n[0] + 2 * g[0])


def pad_periodic(F, ndim):
    """Wrap-pad the last `ndim` spatial axes of F (shape (..., nz, ny, nx))."""
    pad = [(0, 0)] * (F.ndim - 3)
    for ax in range(3):  # z, y, x
        d = 2 - ax
        pad.append((NG, NG) if d < ndim else (0, 0))
    return np.pad(F, pad, mode="wrap")


def ideal_cons(V, gamma):
    """Conserved state of an ideal-gas MHD initial condition from primitives."""
    rho, vx, vy, vz, p, bx, by, bz, psi = V
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) \
        + 0.5 * (bx * bx + by * by + bz * bz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, E, bx, by, bz, psi])


def _modes_2d(rng, kmax):
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(0, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax and (ky > 0 or kx > 0)]
    ph = rng.uniform(0.0, 2.0 * np.pi, size=len(ks))
    return ks, ph


def _field_2d(rng, n, kmax):
    """sum_k cos(2 pi k.x + phi_k) over 0 < |k| <= kmax, scaled to max |f| = 1;
    also returns the pieces needed for an exact spectral curl."""
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")  # shape (ny, nx)
    ks, ph = _modes_2d(rng, kmax)
    f = np.zeros((n, n))
    fx = np.zeros((n, n))
    fy = np.zeros((n, n))
    for (kx, ky), p in zip(ks, ph):
        arg = 2.0 * np.pi * (kx * X + ky * Y) + p
        f += np.cos(arg)
        fx += -2.0 * np.pi * kx * np.sin(arg)
        fy += -2.0 * np.pi * ky * np.sin(arg)
    s = np.abs(f).max()
    return f / s, fx / s, fy / s


def mhd_turb_2d(n=128, seed=0, gamma=5.0 / 3.0):
    """2-D periodic ideal-MHD turbulence-like state on [0,1]^2 (interior n x n).

    rho = 1 + 0.2 f1, p = 1 + 0.1 f2, (vx, vy) = 0.5 (f3, f4), B = curl(A_z z)
    with A_z = 0.1 f5, where each f is a seeded random-phase sum of the modes
    0 < |k| <= 4 normalised to max|f| = 1; psi = 0.  Returns U with ghosts."""
    rng = np.random.default_rng(seed)
    f1, _, _ = _field_2d(rng, n, 4)
    f2, _, _ = _field_2d(rng, n, 4)
    f3, _, _ = _field_2d(rng, n, 4)
    f4, _, _ = _field_2d(rng, n, 4)
    a, ax, ay = _field_2d(rng, n, 4)
    rho = 1.0 + 0.2 * f1
    p = 1.0 + 0.1 * f2
    vx, vy = 0.5 * f3, 0.5 * f4
    bx, by = 0.1 * ay, -0.1 * ax
    z = np.zeros_like(rho)
    V = np.stack([rho, vx, vy, z, p, bx, by, z, z])[:, None, :, :]
    return pad_periodic(ideal_cons(V, gamma), 2)


def _field_3d(rng, n, kmax, deriv=False):
    """Real random-phase field with all modes 0 < |k| <= kmax, via inverse FFT.
    Returns f (max |f| = 1) and, if deriv, the spectral gradient of the same
    (unnormalised) field with the same scale factor."""
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz = k1[:, None, None]
    ky = k1[None, :, None]
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    mask = (k2 > 0) & (k2 <= kmax * kmax)
    spec = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    idx = np.nonzero(mask)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=idx[0].size)
    spec[idx] = np.exp(1j * ph)
    f = np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))
    s = np.abs(f).max()
    if not deriv:
        return f / s
    grads = []
    for kk in (kx, ky, kz):
        grads.append(np.fft.irfftn(spec * (2j * np.pi * kk), s=(n, n, n), axes=(0, 1, 2)) / s)
    return f / s, grads


def mhd_blast_3d(n=256, seed=0, gamma=5.0 / 3.0, kmax=8, sphere=100.0):
    """3-D periodic ideal-MHD state on [0,1]^3 with a pressure sphere.

    rho = 1 + 0.2 f_rho, v = 0.5 (f_x, f_y, f_z), B = curl A with A a seeded
    random vector potential (modes 0 < |k| <= kmax) scaled to max |B| = 1,
    p = 1 outside and `sphere` (100) inside a sphere of radius 0.1 at a seeded
    centre (periodic distance), psi = 0; sphere = 1 gives the smooth spectrum
    alone.  Returns U with ghosts, shape (9, n+8, n+8, n+8)."""
    rng = np.random.default_rng(seed)
    frho = _field_3d(rng, n, kmax)
    vx = 0.5 * _field_3d(rng, n, kmax)
    vy = 0.5 * _field_3d(rng, n, kmax)
    vz = 0.5 * _field_3d(rng, n, kmax)
    _, gax = _field_3d(rng, n, kmax, deriv=True)
    _, gay = _field_3d(rng, n, kmax, deriv=True)
    _, gaz = _field_3d(rng, n, kmax, deriv=True)
    # B = curl A: (dAz/dy - dAy/dz, dAx/dz - dAz/dx, dAy/dx - dAx/dy)
    bx = gaz[1] - gay[2]
    by = gax[2] - gaz[0]
    bz = gay[0] - gax[1]
    del gax, gay, gaz
    bmax = np.sqrt(bx * bx + by * by + bz * bz).max()
    bx /= bmax
    by /= bmax
    bz /= bmax
    c = rng.uniform(0.0, 1.0, size=3)
    x = (np.arange(n) + 0.5) / n
    dxs = [np.minimum(np.abs(x - c[d]), 1.0 - np.abs(x - c[d])) for d in range(3)]
    r2 = dxs[2][:, None, None] ** 2 + dxs[1][None, :, None] ** 2 + dxs[0][None, None, :] ** 2
    p = np.where(r2 < 0.01, float(sphere), 1.0)
    rho = 1.0 + 0.2 * frho
    z = np.zeros_like(rho)
    U = ideal_cons([rho, vx, vy, vz, p, bx, by, bz, z], gamma)
    del rho, vx, vy, vz, p, bx, by, bz, z, frho
    return pad_periodic(U, 3)


def mhd_lowbeta_3d(n=256, seed=0, gamma=5.0 / 3.0, kmax=8, beta=0.01, mach=10.0, kmax_v=2):
    """Low-beta, high-Mach variant: rho = 1 + 0.2 f (modes |k| <= kmax), p = 1,
    uniform B0 = sqrt(2 p / beta) along a seeded unit direction, and a seeded
    large-scale velocity field (modes |k| <= kmax_v) scaled to an rms Mach
    number `mach` (v_rms = mach sqrt(gamma p / rho0)).  The velocity is kept
    large-scale: with |k| up to 8 a Mach-10 field drives the unlimited PPM
    scheme to negative pressures within a step."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.2 * _field_3d(rng, n, kmax)
    v = [_field_3d(rng, n, kmax_v) for _ in range(3)]
    vrms = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    scale = mach * np.sqrt(gamma * 1.0 / 1.0) / vrms
    v = [c * scale for c in v]
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    b0 = np.sqrt(2.0 / beta)
    p = np.ones_like(rho)
    z = np.zeros_like(rho)
    U = ideal_cons([rho, v[0], v[1], v[2], p, z + b0 * d[0], z + b0 * d[1], z + b0 * d[2], z],
                   gamma)
    return pad_periodic(U, 3)


def srmhd_cons(V, gamma):
    """Conserved state (D, m, E - D... see below) of a special relativistic
    MHD initial condition from primitives (rho, v, p, B, psi):
    D = rho gamma, m = (W + B^2) v - (v.B) B, E = W - p + (B^2 + E_el^2)/2 - D
    with W = w gamma^2, E_el = -v x B and the enthalpy density of the ideal
    gas, w = rho + Gamma p/(Gamma-1) (gamma = Gamma > 1), or of the
    Taub-Mathews gas, w = 5/2 p + sqrt(9/4 p^2 + rho^2) (gamma = 0)."""
    rho, vx, vy, vz, p, bx, by, bz, psi = V
    v2 = vx * vx + vy * vy + vz * vz
    lor2 = 1.0 / (1.0 - v2)
    w = rho + gamma / (gamma - 1.0) * p if gamma > 0 else 2.5 * p + np.sqrt(2.25 * p * p + rho * rho)
    W = w * lor2
    B2 = bx * bx + by * by + bz * bz
    vB = vx * bx + vy * by + vz * bz
    E2 = B2 * v2 - vB * vB
    D = rho * np.sqrt(lor2)
    return np.stack([D, (W + B2) * vx - vB * bx, (W + B2) * vy - vB * by, (W + B2) * vz - vB * bz,
                     W - p + 0.5 * (B2 + E2) - D, bx, by, bz, psi])


def srmhd_jet_3d(n=256, seed=0, gamma=4.0 / 3.0, lorentz=10.0, rho_ratio=0.01, sigma=0.1,
                 p0=0.01, radius=0.1, pert=0.01):
    """Relativistic magnetised beam: a cylinder along z of radius 0.1 around a
    seeded axis position, rho = 1 and Lorentz factor up to `lorentz` inside
    (smooth tanh edge over ~2 cells), ambient rho = rho_ratio at rest, uniform
    p = p0, uniform B_z set so that sigma = B^2/(rho h gamma^2) = `sigma` on
    the beam axis, and seeded 1 % perturbations of rho and of the transverse
    velocity.  gamma = 0 takes the Taub-Mathews equation of state.  Periodic
    unit cube; returns U with ghosts."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    c = rng.uniform(0.3, 0.7, size=2)
    dxc = np.minimum(np.abs(x - c[0]), 1.0 - np.abs(x - c[0]))
    dyc = np.minimum(np.abs(x - c[1]), 1.0 - np.abs(x - c[1]))
    r = np.sqrt(dyc[:, None] ** 2 + dxc[None, :] ** 2)  # (ny, nx)
    prof = 0.5 * (1.0 - np.tanh((r - radius) / (2.0 / n)))
    prof3 = np.broadcast_to(prof[None, :, :], (n, n, n))
    lor = 1.0 + (lorentz - 1.0) * prof3
    vz = np.sqrt(1.0 - 1.0 / lor ** 2)
    rho = rho_ratio + (1.0 - rho_ratio) * prof3
    rho = rho * (1.0 + pert * (2.0 * rng.random((n, n, n)) - 1.0))
    vx = pert * (2.0 * rng.random((n, n, n)) - 1.0) * prof3
    vy = pert * (2.0 * rng.random((n, n, n)) - 1.0) * prof3
    vz = vz * np.sqrt(np.maximum(1.0 - (vx ** 2 + vy ** 2) / np.maximum(vz ** 2, 1e-300), 0.0))
    p = np.full((n, n, n), p0)
    # specific enthalpy on the axis (rho = 1): ideal gas, or Taub-Mathews (gamma = 0)
    h_axis = 1.0 + gamma / (gamma - 1.0) * p0 if gamma > 0 else 2.5 * p0 + np.sqrt(2.25 * p0 * p0 + 1.0)
    bz0 = np.sqrt(sigma * 1.0 * h_axis * lorentz ** 2)
    z = np.zeros((n, n, n))
    U = srmhd_cons([rho, vx, vy, vz, p, z, z, z + bz0, z], gamma)
    return pad_periodic(U, 3)


# ------------------------------------------------------------------ AMR hierarchy

def _cover(tags, sizes=(64, 32, 16, 8), fill=0.15):
    """Cover the True cells of a boolean 3-D array with aligned cubes, largest
    first: an aligned cube of size s is taken when it holds uncovered tags
    that fill more than `fill` of it (any tag for the smallest size).
    Returns [(origin(z,y,x), s)]."""
    left = tags.copy()
    out = []
    nz, ny, nx = tags.shape
    for s in sizes:
        if nz % s or ny % s or nx % s:
            continue
        blk = left.reshape(nz // s, s, ny // s, s, nx // s, s)
        frac = blk.mean(axis=(1, 3, 5))
        take = frac > (fill if s > sizes[-1] else 0.0)
        for (k, j, i) in zip(*np.nonzero(take)):
            out.append(((k * s, j * s, i * s), s))
        mask = np.repeat(np.repeat(np.repeat(take, s, 0), s, 1), s, 2)
        left &= ~mask
    return out


def _shock_prim(xc, yc, zc, c, r0, gamma):
    """Analytic state of an expanding spherical shock at cell centres: a
    shell of width 0.02 at radius r0 around c with 4x density, 20x pressure
    and radial outflow 1.5 behind it, uniform B = (0.6, 0.8, 0) / 2, psi = 0."""
    dx_, dy_, dz_ = xc - c[0], yc - c[1], zc - c[2]
    r = np.sqrt(dx_ * dx_ + dy_ * dy_ + dz_ * dz_) + 1e-12
    inside = 0.5 * (1.0 - np.tanh((r - r0) / 0.01))
    shell = np.exp(-((r - r0) / 0.02) ** 2)
    rho = 1.0 + 3.0 * shell
    p = 1.0 + 19.0 * inside
    vr = 1.5 * shell
    z = np.zeros_like(r)
    return [rho, vr * dx_ / r, vr * dy_ / r, vr * dz_ / r, p, z + 0.3, z + 0.4, z, z]


def _nest(cubes, parents, region, smallest=8):
    """Proper nesting: keep the level-(l+1) cubes [(origin (z, y, x), size)]
    whose footprint on level l, grown by one level-l cell on every side,
    lies inside `region` (level l's cells covered by its patches, periodic);
    a cube that does not is replaced by its eight children, down to the
    smallest size, below which it is dropped.  Returns (cubes, parents)."""
    dom = region.shape[0]
    out, par = [], []
    todo = list(zip(cubes, parents))
    while todo:
        (o, s), pi = todo.pop()
        idx = [np.arange(v // 2 - 1, (v + s) // 2 + 1) % dom for v in o]
        if region[np.ix_(*idx)].all():
            out.append((o, s))
            par.append(pi)
        elif s > smallest:
            h = s // 2
            todo += [(((o[0] + a * h, o[1] + b * h, o[2] + c * h), h), pi)
                     for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    return out, par


def amr_hierarchy(seed=0, base=128, target=600, gamma=5.0 / 3.0, nested=False, smooth=False):
    """Seeded 3-level hierarchy (refinement ratio 2, base `base`^3 cells on the
    unit cube as 8 patches of (base/2)^3) around an expanding spherical shock.
    Level l+1 tags the cells of level l within a shell around the shock
    radius and covers them with aligned cubes from {64, 32, 16, 8} (in level
    l+1 cells), largest first, each inside one level-l patch.  A level-2
    patch may then touch the edge of level 1's region; with `nested`, every
    level-(l+1) patch keeps one level-l cell of level l around it (proper
    nesting, see _nest).  The shell width is tuned by bisection so that the
    hierarchy has about `target` patches.  Returns a dict with, per level,
    the patch list [(n(3), dx(3), base offset)], the float64 pool (9,
    stride) with ghosts filled from the analytic state (or the smooth state
    of _smooth_prim with `smooth`), and the footprints of every level-(l+1)
    patch in its parent (parent index, origin in parent cells, size in
    parent cells)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.4, 0.6, size=3)
    r0 = rng.uniform(0.18, 0.25)

    def build(width):
        levels = [[((k, j, i), base // 2) for k in (0, base // 2) for j in (0, base // 2)
                   for i in (0, base // 2)]]
        parents = [[]]
        for lev in (1, 2):
            h = 1.0 / (base * 2 ** lev)
            plist, par = [], []
            for pi, (o, s) in enumerate(levels[-1]):
                # children cells of parent patch pi, in level-lev index space
                n = 2 * s
                oz, oy, ox = (2 * v for v in o)
                x = (np.arange(n) + ox + 0.5) * h
                y = (np.arange(n) + oy + 0.5) * h
                z = (np.arange(n) + oz + 0.5) * h
                rr = np.sqrt((z[:, None, None] - c[2]) ** 2 + (y[None, :, None] - c[1]) ** 2
                             + (x[None, None, :] - c[0]) ** 2)
                tags = np.abs(rr - r0) < width / lev
                for (lo, sz) in _cover(tags):
                    plist.append(((lo[0] + oz, lo[1] + oy, lo[2] + ox), sz))
                    par.append(pi)
            if nested and lev > 1:
                region = np.zeros((base * 2 ** (lev - 1),) * 3, dtype=bool)
                for (o, s) in levels[-1]:
                    region[o[0]:o[0] + s, o[1]:o[1] + s, o[2]:o[2] + s] = True
                plist, par = _nest(plist, par, region)
            levels.append(plist)
            parents.append(par)
        return levels, parents

    best = None
    for width in np.geomspace(0.004, 0.12, 16):
        levels, parents = build(width)
        if not all(levels):
            continue  # a level left empty (nesting can drop a thin level whole)
        tot = sum(len(L) for L in levels)
        if best is None or abs(tot - target) < abs(best[0] - target):
            best = (tot, levels, parents)
    tot, levels, parents = best
    return amr_levels(levels, parents, base, c, r0, gamma, smooth=smooth)


def _smooth_prim(xc, yc, zc):
    """A smooth state periodic on the unit cube: density 0.6 to 1.4, pressure
    0.8 to 1.2, velocity of amplitude 0.4 and a solenoidal field of amplitude
    0.3 (B_x(z), B_y(x), B_z(y)), psi = 0."""
    t = 2.0 * np.pi
    rho = 1.0 + 0.25 * np.sin(t * xc) * np.cos(t * yc) + 0.15 * np.sin(t * zc)
    p = 1.0 + 0.2 * np.cos(t * (xc + yc))
    z = np.zeros_like(rho)
    return [rho, 0.4 * np.sin(t * yc), 0.4 * np.sin(t * zc), 0.4 * np.sin(t * xc), p,
            0.3 * np.cos(t * zc), 0.3 * np.cos(t * xc), 0.3 * np.cos(t * yc), z]


def amr_levels(levels, parents, base, center, radius, gamma=5.0 / 3.0, smooth=False):
    """The level dicts of a hierarchy given its patches: levels[l] lists the
    (origin (z, y, x), size) cubes of level l in its own cells (level l: base
    x 2^l cells per side of the unit cube), parents[l][i] the index of patch
    i's parent on level l - 1 (parents[0] empty).  Every patch is filled,
    ghosts included, at its cell centres with the expanding spherical shock
    of amr_hierarchy (centre `center`, radius `radius`), or with the smooth
    periodic state of _smooth_prim when `smooth`.  Returns {"levels":
    [{"patches", "pool", "origins", "footprints"}], "center", "radius"} as
    amr_hierarchy does."""
    c, r0 = center, radius
    out = {"levels": [], "center": c, "radius": r0}
    for lev, plist in enumerate(levels):
        h = 1.0 / (base * 2 ** lev)
        specs, off, chunks = [], 0, []
        for (o, s) in plist:
            g = np.arange(-4, s + 4) + 0.5
            xc = (o[2] + g) * h
            yc = (o[1] + g) * h
            zc = (o[0] + g) * h
            Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
            U = ideal_cons(_smooth_prim(X, Y, Z) if smooth else _shock_prim(X, Y, Z, c, r0, gamma), gamma)
            specs.append(([s, s, s], [h, h, h], off, lev))
            chunks.append(U.reshape(9, -1))
            off += U[0].size
        pool = np.concatenate(chunks, axis=1)
        foot = []
        if lev > 0:
            for (o, s), pi in zip(plist, parents[lev]):
                po, ps = levels[lev - 1][pi]
                foot.append((pi, tuple((o[d] // 2 - po[d]) for d in range(3)), s // 2))
        out["levels"].append({"patches": specs, "pool": pool, "origins": plist, "footprints": foot})
    return out
