// ctu_launch.cuh -- launcher templates, instantiated per precision, physics
// and interface mode by ctu_f64.cu, ctu_f32.cu, ctu_f32i.cu and ctu_sr32.cu.
#pragma once

#include <atomic>

#include "ctu_launch.h"

namespace ctu {

#define CTU_MARK(nm) \
    if (li.prof) li.prof->mark(nm, s)

// Launch one marching sweep over a patch group.  Kernels that stage through
// more than the default 48 KB of dynamic shared memory are opted in once per
// device (the carveout set to its maximum, so that the register-limited
// number of blocks still fits).
template <int PHYS, class R, int PPM, int IF64, int D, int MODE>
static void launch_sweep_m(const StepArgs &a, const Group &G, const R *Vs, const R *L1, R *A, cudaStream_t s)
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
    const dim3 grid((unsigned)Tiles::sweep_m(G.n, D), (unsigned)G.count);
    k_sweep_m<PHYS, R, PPM, IF64, D, MODE><<<grid, BLOCK, smem, s>>>(a, G.first, Vs, L1, A);
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
    for (int g = 0; g < li.ngroups; ++g) {
        const Group &G = li.groups[g];
        k_prim<PHYS, R><<<dim3((unsigned)Tiles::prim(G.n, G.N), (unsigned)G.count), BLOCK, 0, s>>>(a, G.first, Vs);
        ++n;
    }
    CTU_MARK(nullptr);
    if (a.ndim > 1) {  // first-order stage: the transverse terms of the sweeps
        CTU_MARK("flux1");
        for (int g = 0; g < li.ngroups; ++g) {
            const Group &G = li.groups[g];
            const unsigned c = (unsigned)G.count;
            k_div1<PHYS, R, 0><<<dim3((unsigned)Tiles::div1(G.n, a.ndim, 0), c), BLOCK, 0, s>>>(a, G.first, Vs, L1);
            k_div1<PHYS, R, 1><<<dim3((unsigned)Tiles::div1(G.n, a.ndim, 1), c), BLOCK, 0, s>>>(a, G.first, Vs, L1);
            n += 2;
            if (a.ndim > 2) {
                k_div1<PHYS, R, 2><<<dim3((unsigned)Tiles::div1(G.n, a.ndim, 2), c), BLOCK, 0, s>>>(a, G.first, Vs,
                                                                                                 L1);
                ++n;
            }
        }
        CTU_MARK(nullptr);
    }
    // sweeps in the order z, y, x: the first writes A = L_D, the middle one
    // adds to it, and the x sweep (thread per cell) finishes the update
    if (a.ndim > 2) {
        CTU_MARK("sweep_z");
        for (int g = 0; g < li.ngroups; ++g) {
            launch_sweep_m<PHYS, R, PPM, IF64, 2, SW_FIRST>(a, li.groups[g], Vs, L1, A, s);
            ++n;
        }
        CTU_MARK(nullptr);
    }
    if (a.ndim > 1) {
        CTU_MARK("sweep_y");
        for (int g = 0; g < li.ngroups; ++g) {
            if (a.ndim == 2)
                launch_sweep_m<PHYS, R, PPM, IF64, 1, SW_FIRST>(a, li.groups[g], Vs, L1, A, s);
            else
                launch_sweep_m<PHYS, R, PPM, IF64, 1, SW_MID>(a, li.groups[g], Vs, L1, A, s);
            ++n;
        }
        CTU_MARK(nullptr);
    }
    CTU_MARK("sweep_x");
    for (int g = 0; g < li.ngroups; ++g) {
        const Group &G = li.groups[g];
        const dim3 grid((unsigned)Tiles::sweep_x(G.n), (unsigned)G.count);
        k_sweep_x<PHYS, R, PPM, IF64, 1><<<grid, BLOCK, 0, s>>>(a, G.first, Vs, L1, A);
        ++n;
    }
    CTU_MARK(nullptr);
    return n;
}

// MHD: PPM or MC-linear characteristic tracing.
template <class R, int IF64> int launch_step_impl(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    return li.recon ? launch_step_t<PH_MHD, R, 1, IF64>(a, li, s) : launch_step_t<PH_MHD, R, 0, IF64>(a, li, s);
}

// SRMHD: MUSCL-Hancock with MC-linear primitive slopes.
template <class R> int launch_step_sr(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    return launch_step_t<PH_SR, R, 0, 1>(a, li, s);
}

template <int PHYS, class R>
int launch_maxspeed_impl(const StepArgs &a, const LaunchInfo &li, unsigned long long *out, cudaStream_t s)
{
    CTU_MARK("maxspeed");
    for (int g = 0; g < li.ngroups; ++g) {
        const Group &G = li.groups[g];
        k_maxspeed<PHYS, R><<<dim3((unsigned)Tiles::interior(G.n), (unsigned)G.count), BLOCK, 0, s>>>(a, G.first,
                                                                                                      out);
    }
    CTU_MARK(nullptr);
    return li.ngroups;
}

#undef CTU_MARK

} // namespace ctu
