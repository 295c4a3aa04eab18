// ctu_launch.cuh -- launcher templates, instantiated per precision, physics
// and interface mode by ctu_f64.cu, ctu_f32.cu, ctu_f32i.cu and ctu_sr32.cu.
#pragma once

#include <atomic>
#include <type_traits>

#include "ctu_launch.h"
#include "par_ops.cuh"

namespace ctu {

#define CTU_MARK(nm) \
    if (li.prof) li.prof->mark(nm, s)

// Launch a kernel once over every patch group of the batch (MAXG groups per
// launch), in the order of li.groups (largest patches first).  bpp(G): blocks
// per patch of group G; go(table, blocks) launches; xr(G): rows per thread
// of the x-tiled kernels that take several (1 for the others).  Returns the
// number of launches.
struct OneRow {
    int operator()(const Group &) const { return 1; }
};
template <class BPP, class GO, class XR = OneRow>
static int over_groups(const LaunchInfo &li, BPP bpp, GO go, XR xr = XR())
{
    int launches = 0;
    for (int c0 = 0; c0 < li.ngroups; c0 += MAXG) {
        GroupTable gt;
        gt.n = li.ngroups - c0 < MAXG ? li.ngroups - c0 : MAXG;
        long long tot = 0;
        for (int k = 0; k < gt.n; ++k) {
            const Group &G = li.groups[c0 + k];
            gt.start[k] = (int)tot;
            gt.first[k] = G.first;
            gt.bpp[k] = (int)bpp(G);
            const DivMagic dm = divmagic((unsigned)(gt.bpp[k] > 0 ? gt.bpp[k] : 1));
            gt.bm[k] = dm.m;
            gt.bs1[k] = dm.s1;
            gt.bs2[k] = dm.s2;
            gt.xw[k] = G.xw;
            gt.seg[k] = G.seg;
            gt.xr[k] = (unsigned char)xr(G);
            tot += (long long)G.count * gt.bpp[k];
        }
        gt.start[gt.n] = (int)tot;
        if (tot > 0) {
            go(gt, (unsigned)tot);
            ++launches;
        }
    }
    return launches;
}

// Rows per thread of an x-tiled kernel for a launch (Tiles::div1x_rows,
// sweepx_rows): the largest power of two up to `most` at which the launch
// still has at least CTU_ROW_WAVES (8) waves of blocks (the device's SMs x 5
// resident blocks), so that the longer
// blocks leave no long tail on a small batch.  blocks(G, x): blocks of one
// patch of group G at x rows per thread.
#ifndef CTU_ROW_WAVES
#define CTU_ROW_WAVES 8
#endif
template <class BLK> static int launch_rows(const LaunchInfo &li, int most, BLK blocks)
{
    for (int x = most; x > 1; x /= 2) {
        long long tot = 0;
        for (int g = 0; g < li.ngroups; ++g) tot += (long long)li.groups[g].count * blocks(li.groups[g], x);
        if (tot >= (long long)CTU_ROW_WAVES * (li.sms > 0 ? li.sms : 152) * 5) return x;
    }
    return 1;
}

// The parabolic kernels' term mask (bit 1 viscosity, bit 2 resistivity, bit
// 4 anisotropic or saturated conduction) and a call of f with it as a compile-time
// constant.
static inline int par_mask(const StepArgs &a)
{
    return (a.par_visc ? 1 : 0) | (a.par_res ? 2 : 0) | (a.par_aniso || a.par_sat ? 4 : 0);
}
template <class F> static void with_tm(int tm, F &&f)
{
    switch (tm) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    default: f(std::integral_constant<int, 7>{}); break;
    }
}

// Kernels that stage through more than the default 48 KB of dynamic shared
// memory are opted in once per device (the carveout set to its maximum, so
// that the register-limited number of blocks still fits).
template <int PHYS, class R, int PPM, int IF64, int D, int MODE>
static int launch_sweep_m(const StepArgs &a, const LaunchInfo &li, const R *Vs, const R *L1, R *A, cudaStream_t s)
{
    constexpr int smem = sweep_m_smem<R, MODE>();
    if (smem > 48 * 1024) {
        static std::atomic<unsigned long long> done{0};
        int dev = 0;
        cudaGetDevice(&dev);
        const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
        if (!(done.load() & bit) || !bit) {
            cudaFuncSetAttribute(k_sweep_m<PHYS, R, PPM, IF64, D, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
            cudaFuncSetAttribute(k_sweep_m<PHYS, R, PPM, IF64, D, MODE>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            done.fetch_or(bit);
        }
    }
    return over_groups(
        li, [&](const Group &G) { return Tiles::sweep_m(G.n, D, G.xw, G.seg); },
        [&](const GroupTable &gt, unsigned nb) {
            k_sweep_m<PHYS, R, PPM, IF64, D, MODE><<<nb, BLOCK, smem, s>>>(a, gt, Vs, L1, A);
        });
}

template <int PHYS, class R, int PPM, int IF64>
static int launch_step_t(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    const long long S = a.sstride;
    R *base = (R *)li.scratch;
    R *Vs = base;
    R *L1 = base + 9 * S;
    R *A = base + 36 * S;
    int n = 0;
    CTU_MARK("setup");
    k_setup<<<1, 1, 0, s>>>(a.dtch, li.sp);
    CTU_MARK(nullptr);
    ++n;
    CTU_MARK("prim");
    if constexpr (recon_hybrid(PPM))  // the shock flags read the outermost ghost layer
        n += over_groups(
            li, [&](const Group &G) { return Tiles::prim(G.N); },
            [&](const GroupTable &gt, unsigned nb) { k_prim<PHYS, R, IF64><<<nb, BLOCK, 0, s>>>(a, gt, Vs); });
    else
        n += over_groups(
            li, [&](const Group &G) { return Tiles::prim_trim(G.N); },
            [&](const GroupTable &gt, unsigned nb) {
                k_prim<PHYS, R, IF64, true><<<nb, BLOCK, 0, s>>>(a, gt, Vs);
            });
    CTU_MARK(nullptr);
    if constexpr (recon_hybrid(PPM)) {  // shock flags of the hybrid integration
        CTU_MARK("shock");
        n += over_groups(
            li, [&](const Group &G) { return Tiles::ghosted(G.N); },
            [&](const GroupTable &gt, unsigned nb) { k_shock<R><<<nb, BLOCK, 0, s>>>(a, gt, Vs); });
        n += over_groups(
            li, [&](const Group &G) { return Tiles::ghosted(G.N); },
            [&](const GroupTable &gt, unsigned nb) {
                k_minmod<<<nb, BLOCK, 0, s>>>(a, gt, PPM == RECON_PPM_HYB ? 2 : 1);
            });
        CTU_MARK(nullptr);
    }
    // first-order stage: the transverse terms of the sweeps; with the
    // parabolic terms over the whole ring box and in every direction (their
    // half-step state needs sum_d L_(H,d)^n there, also in 1-D)
    constexpr bool EXT = recon_par(PPM);
    constexpr bool HY = recon_hybrid(PPM), HC = recon_hllc(PPM);
    if constexpr (recon_mt(PPM)) {
        // the corner coupling of Mignone & Tzeferacos: the transverse fluxes
        // from the normal predictor states
        if (a.ndim > 1) {
            CTU_MARK("pred1");
            n += over_groups(
                li, [&](const Group &G) { return Tiles::pred_x(G.n, a.ndim, G.xw); },
                [&](const GroupTable &gt, unsigned nb) { k_pred<PHYS, R, PPM, 0><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1); });
            n += over_groups(
                li, [&](const Group &G) { return Tiles::div1(G.n, a.ndim, 1, G.xw, G.seg); },
                [&](const GroupTable &gt, unsigned nb) { k_pred<PHYS, R, PPM, 1><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1); });
            if (a.ndim > 2)
                n += over_groups(
                    li, [&](const Group &G) { return Tiles::div1(G.n, a.ndim, 2, G.xw, G.seg); },
                    [&](const GroupTable &gt, unsigned nb) {
                        k_pred<PHYS, R, PPM, 2><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1);
                    });
            CTU_MARK(nullptr);
        }
    } else if (a.ndim > 1 || EXT) {
        CTU_MARK("flux1");
        const int xr1 = launch_rows(li, DIV1X_ROWS, [&](const Group &G, int x) {
            return Tiles::div1(G.n, a.ndim, 0, G.xw, G.seg, EXT, x);
        });
        n += over_groups(
            li, [&](const Group &G) { return Tiles::div1(G.n, a.ndim, 0, G.xw, G.seg, EXT, xr1); },
            [&](const GroupTable &gt, unsigned nb) { k_div1<PHYS, R, 0, HY, HC, EXT><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1); },
            [&](const Group &G) { return Tiles::div1x_rows(G.n, a.ndim, G.xw, xr1); });
        if (a.ndim > 1)
            n += over_groups(
                li, [&](const Group &G) { return Tiles::div1(G.n, a.ndim, 1, G.xw, G.seg, EXT); },
                [&](const GroupTable &gt, unsigned nb) { k_div1<PHYS, R, 1, HY, HC, EXT><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1); });
        if (a.ndim > 2)
            n += over_groups(
                li, [&](const Group &G) { return Tiles::div1(G.n, a.ndim, 2, G.xw, G.seg, EXT); },
                [&](const GroupTable &gt, unsigned nb) { k_div1<PHYS, R, 2, HY, HC, EXT><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1); });
        CTU_MARK(nullptr);
    }
    if constexpr (recon_par(PPM)) {
        // parabolic terms: L_P^n, the half-step fields and their face fluxes
        // (the x sweep differences these into L_P^(n+1/2) for the update)
        CTU_MARK("par_faces_n");
        auto par = [&](auto tm) {
            constexpr int V = decltype(tm)::value;
            n += over_groups(
                li, [&](const Group &G) { return ((long long)par_face_threads(G.n, a.ndim, 1) + BLOCK - 1) / BLOCK; },
                [&](const GroupTable &gt, unsigned nb) {
                    k_par_faces<R, V, 1><<<nb, BLOCK, 0, s>>>(a, gt, Vs, a.th, (R *)a.pif);
                });
            CTU_MARK(nullptr);
            CTU_MARK("par_half");
            n += over_groups(
                li, [&](const Group &G) { return ((long long)par_ring_threads(G.n, a.ndim) + BLOCK - 1) / BLOCK; },
                [&](const GroupTable &gt, unsigned nb) {
                    k_par_half<R, V><<<nb, BLOCK, 0, s>>>(a, gt, L1, (R *)a.lp, a.th, (const R *)a.pif);
                });
            CTU_MARK(nullptr);
            CTU_MARK("par_faces_h");
            n += over_groups(
                li, [&](const Group &G) { return ((long long)par_face_threads(G.n, a.ndim, 0) + BLOCK - 1) / BLOCK; },
                [&](const GroupTable &gt, unsigned nb) {
                    k_par_faces<R, V, 0><<<nb, BLOCK, 0, s>>>(a, gt, Vs, a.th, (R *)a.pif);
                });
            if (a.reg && a.nwin > 0 && a.wfaces > 0) {
                const int ny = (a.wfaces + BLOCK - 1) / BLOCK;
                k_par_register<R, V><<<dim3(a.nwin, ny < 65535 ? ny : 65535), BLOCK, 0, s>>>(a, (const R *)a.pif);
                ++n;
            }
            CTU_MARK(nullptr);
            CTU_MARK("par_lp");
            n += over_groups(
                li, [&](const Group &G) { return Tiles::interior(G.n, G.xw); },
                [&](const GroupTable &gt, unsigned nb) {
                    k_par_lp<R, V><<<nb, BLOCK, 0, s>>>(a, gt, (const R *)a.pif, (R *)a.lph);
                });
        };
        // one kernel per combination of the terms beyond isotropic conduction
        with_tm(par_mask(a), par);
        CTU_MARK(nullptr);
    }
    // sweeps in the order z, y, x: the first writes A = L_D, the middle one
    // adds to it, and the x sweep (thread per cell) finishes the update
    if (a.ndim > 2) {
        CTU_MARK("sweep_z");
        n += launch_sweep_m<PHYS, R, PPM, IF64, 2, SW_FIRST>(a, li, Vs, L1, A, s);
        CTU_MARK(nullptr);
    }
    if (a.ndim > 1) {
        CTU_MARK("sweep_y");
        if (a.ndim == 2)
            n += launch_sweep_m<PHYS, R, PPM, IF64, 1, SW_FIRST>(a, li, Vs, L1, A, s);
        else
            n += launch_sweep_m<PHYS, R, PPM, IF64, 1, SW_MID>(a, li, Vs, L1, A, s);
        CTU_MARK(nullptr);
    }
    CTU_MARK("sweep_x");
    const int xrs = launch_rows(li, SWEEPX_ROWS, [&](const Group &G, int x) { return Tiles::sweep_x(G.n, G.xw, x); });
    n += over_groups(
        li, [&](const Group &G) { return Tiles::sweep_x(G.n, G.xw, xrs); },
        [&](const GroupTable &gt, unsigned nb) {
            k_sweep_x<PHYS, R, PPM, IF64, 1><<<nb, BLOCK, 0, s>>>(a, gt, Vs, L1, A);
        },
        [&](const Group &G) { return Tiles::sweepx_rows(G.n, G.xw, xrs); });
    CTU_MARK(nullptr);
    return n;
}

// MHD: PPM or MC-linear characteristic tracing.
template <class R, int IF64> int launch_step_impl(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    return li.recon == RECON_PPM ? launch_step_t<PH_MHD, R, RECON_PPM, IF64>(a, li, s)
                                 : launch_step_t<PH_MHD, R, RECON_MC, IF64>(a, li, s);
}

// MHD with the other reconstructions of Section 3.2 (G = 0: linear with the
// MinMod, harmonic or Van Albada slope, or improved WENO3), with the
// reference states of the tracing (G = 1: PPM or MC-linear), with the
// hybrid integration (G = 2: PPM or MC-linear), with the HLLC solver
// (G = 3: PPM or MC-linear), or with the parabolic terms, conduction,
// viscosity and resistivity (G = 4: PPM or MC-linear).
template <class R, int IF64, int G> int launch_step_var(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    if constexpr (G == 4)  // the parabolic terms
        return li.recon == RECON_PPM_PAR ? launch_step_t<PH_MHD, R, RECON_PPM_PAR, IF64>(a, li, s)
                                         : launch_step_t<PH_MHD, R, RECON_MC_PAR, IF64>(a, li, s);
    else if constexpr (G == 3)  // the HLLC solver
        return li.recon == RECON_PPM_HLLC ? launch_step_t<PH_MHD, R, RECON_PPM_HLLC, IF64>(a, li, s)
                                          : launch_step_t<PH_MHD, R, RECON_MC_HLLC, IF64>(a, li, s);
    else if constexpr (G == 2)  // the hybrid integration of the shock-detection appendix
        return li.recon == RECON_PPM_HYB ? launch_step_t<PH_MHD, R, RECON_PPM_HYB, IF64>(a, li, s)
                                         : launch_step_t<PH_MHD, R, RECON_MC_HYB, IF64>(a, li, s);
    else if constexpr (G == 0)
        return li.recon == RECON_WENO3 ? launch_step_t<PH_MHD, R, RECON_WENO3, IF64>(a, li, s)
                                       : launch_step_t<PH_MHD, R, RECON_LIN, IF64>(a, li, s);
    else
        return li.recon == RECON_PPM_REF ? launch_step_t<PH_MHD, R, RECON_PPM_REF, IF64>(a, li, s)
                                         : launch_step_t<PH_MHD, R, RECON_MC_REF, IF64>(a, li, s);
}

// MHD with the corner coupling of Mignone & Tzeferacos (G = 5: PPM or
// MC-linear).
template <class R, int IF64> int launch_step_mt(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    return li.recon == RECON_PPM_MT ? launch_step_t<PH_MHD, R, RECON_PPM_MT, IF64>(a, li, s)
                                    : launch_step_t<PH_MHD, R, RECON_MC_MT, IF64>(a, li, s);
}

// SRMHD: MUSCL-Hancock with MC-linear primitive slopes.
template <class R> int launch_step_sr(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    return launch_step_t<PH_SR, R, 0, 1>(a, li, s);
}

template <int PHYS, class R, int LIT64 = 0>
int launch_maxspeed_impl(const StepArgs &a, const LaunchInfo &li, unsigned long long *out, cudaStream_t s)
{
    CTU_MARK("maxspeed");
    const int n = over_groups(
        li, [&](const Group &G) { return Tiles::interior(G.n, G.xw); },
        [&](const GroupTable &gt, unsigned nb) { k_maxspeed<PHYS, R, LIT64><<<nb, BLOCK, 0, s>>>(a, gt, out); });
    CTU_MARK(nullptr);
    return n;
}

#undef CTU_MARK

} // namespace ctu
