"""Helpers that drive the CUDA path through the C ABI (ctypes binding)."""
import numpy as np

import oracle as O


def torch_cuda():
    import torch
    return torch


def l1rel(got, ref, ch=None, group_floor=False):
    """Per-variable relative L1: sum|got - ref| / sum|ref|; for psi the
    denominator is c_h sum |B| (psi carries the units of c_h B).
    group_floor: a vector component is measured against at least the size of
    its whole vector (momentum also against D, i.e. rho gamma c with c = 1),
    for regions where one component of the reference is nearly zero."""
    out = []
    for q in range(9):
        num = np.abs(got[q] - ref[q]).sum()
        if q == 8:
            den = (ch if ch else 1.0) * np.abs(ref[5:8]).sum()
        else:
            den = np.abs(ref[q]).sum()
            if group_floor and q in (1, 2, 3):
                den = max(den, np.abs(ref[1:4]).sum(), np.abs(ref[0]).sum())
            if group_floor and q in (5, 6, 7):
                den = max(den, np.abs(ref[5:8]).sum())
        out.append(num / den if den > 0 else (0.0 if num == 0 else np.inf))
    return np.array(out)


def maxrel(got, ref, ch=None):
    """Per-variable elementwise bound: max|got - ref| / max|ref| (for psi the
    denominator is c_h max|B|), so that an error confined to a few cells (a
    tile seam, a patch corner) cannot hide in the L1 sum."""
    out = []
    for q in range(9):
        num = np.abs(got[q] - ref[q]).max()
        den = (ch if ch else 1.0) * np.abs(ref[5:8]).max() if q == 8 else np.abs(ref[q]).max()
        out.append(num / den if den > 0 else (0.0 if num == 0 else np.inf))
    return np.array(out)


def gpu_run(U0, n, ndim, dx, steps, cfl, precision=0, recon=1, trace_mode=0, glm_alpha=0.1,
            gamma=5.0 / 3.0, physics=0, eos=0, riemann=0, kappa=0.0, nu=0.0, eta=0.0, kappa_par=0.0, phi=0.0,
            corner=0):
    """Advance one periodic patch `steps` steps on the GPU; returns
    (U ghosted numpy, list of (dt, ch), status)."""
    import torch
    from paper_1110_0740_gb300 import ctu
    dev = torch.device("cuda:0")
    U = torch.from_numpy(np.ascontiguousarray(U0).reshape(9, -1)).to(dev)
    Ub = torch.zeros_like(U)
    stride = U.shape[1]
    if physics == ctu.CTU_SRMHD:
        cfg = ctu.make_config(ndim=ndim, gamma=gamma, recon=ctu.CTU_LINEAR_MC, precision=precision,
                              cfl=cfl, glm_alpha=glm_alpha, physics=ctu.CTU_SRMHD,
                              predictor=ctu.CTU_MUSCL_HANCOCK, riemann=ctu.CTU_HLL, eos=eos)
    else:
        cfg = ctu.make_config(ndim=ndim, gamma=gamma, recon=recon, precision=precision, cfl=cfl,
                              glm_alpha=glm_alpha, trace_mode=trace_mode, riemann=riemann, kappa=kappa, nu=nu, eta=eta,
                              kappa_par=kappa_par, tc_phi=phi, corner=corner)
    ctx = ctu.Ctx(cfg)
    dx3 = list(dx) + [1.0] * (3 - len(dx))
    patches = ctu.make_patches([(n, dx3, 0)])
    dtch = torch.zeros(2, dtype=torch.float64, device=dev)
    dts = []
    for _ in range(steps):
        ctx.fill_periodic(U, stride, patches)
        ctx.dt(U, stride, patches, dtch)
        ctx.step(U, Ub, stride, patches, dtch)
        dts.append(tuple(dtch.cpu().tolist()))
        U, Ub = Ub, U
    ctx.fill_periodic(U, stride, patches)
    st = ctx.status_sync()
    out = U.cpu().numpy().reshape(U0.shape)
    ctx.close()
    return out, dts, st


def oracle_run(U0, n, ndim, dx, steps, cfl, recon=1, trace_mode=0, glm_alpha=0.1,
               gamma=5.0 / 3.0, riemann=0, kappa=0.0, nu=0.0, eta=0.0, kappa_par=0.0, phi=0.0, corner=0):
    U, t, dts = O.mhd_run(U0, n, ndim, list(dx) + [1.0] * (3 - len(dx)), steps, cfl, gamma=gamma,
                          glm_alpha=glm_alpha, recon=recon, upwind=trace_mode, riemann=riemann, kappa=kappa, nu=nu, eta=eta,
                          kappa_par=kappa_par or None, phi=phi, corner=corner)
    return U, dts
