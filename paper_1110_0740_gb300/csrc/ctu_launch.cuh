// ctu_launch.cuh -- launcher templates, instantiated per precision.
#pragma once

#include "ctu_launch.h"

namespace ctu {

static inline dim3 grid_for(long long cells, int npatch, int block)
{
    long long bx = (cells + block - 1) / block;
    if (bx > (1LL << 20)) bx = 1LL << 20;
    if (bx < 1) bx = 1;
    return dim3((unsigned)bx, (unsigned)npatch, 1);
}

template <class R> int launch_step(const StepArgs &a, const LaunchInfo &li, cudaStream_t s)
{
    const long long S = a.sstride;
    R *base = (R *)li.scratch;
    R *Vs = base;
    R *F1[3] = {base + 9 * S, base + 18 * S, base + 27 * S};
    R *Vp = base + 36 * S;
    R *Vm = base + 45 * S;
    R *F[3] = {base + 54 * S, base + 63 * S, base + 72 * S};
    const int B = 128;
    const dim3 g = grid_for(li.max_cells, a.npatch, B);
    ProfHook *P = li.prof;
#define MARK(nm) \
    if (P) P->mark(nm, s)
    int n = 0;
    MARK("prim");
    k_prim<R><<<g, B, 0, s>>>(a, Vs);
    MARK(nullptr);
    ++n;
    for (int d = 0; d < a.ndim; ++d) {
        MARK("flux1");
        k_flux1<R><<<g, B, 0, s>>>(a, d, Vs, F1[d]);
        MARK(nullptr);
        ++n;
    }
    for (int d = 0; d < a.ndim; ++d) {
        MARK("trace");
        constexpr bool is64 = sizeof(R) == 8;
        if (li.recon && (is64 || li.iface64))
            k_trace<R, 1, 1><<<g, B, 0, s>>>(a, d, Vs, F1[0], F1[1], F1[2], Vp, Vm);
        else if (li.recon)
            k_trace<R, 1, is64 ? 1 : 0><<<g, B, 0, s>>>(a, d, Vs, F1[0], F1[1], F1[2], Vp, Vm);
        else if (is64 || li.iface64)
            k_trace<R, 0, 1><<<g, B, 0, s>>>(a, d, Vs, F1[0], F1[1], F1[2], Vp, Vm);
        else
            k_trace<R, 0, is64 ? 1 : 0><<<g, B, 0, s>>>(a, d, Vs, F1[0], F1[1], F1[2], Vp, Vm);
        MARK(nullptr);
        MARK("riemann");
        k_riemann<R><<<g, B, 0, s>>>(a, d, Vp, Vm, F[d]);
        MARK(nullptr);
        n += 2;
    }
    MARK("update");
    k_update<R><<<g, B, 0, s>>>(a, F[0], F[1], F[2]);
    MARK(nullptr);
    ++n;
    if (li.nwin > 0 && li.reg) {
        MARK("registers");
        k_registers<R><<<dim3(8, (unsigned)li.nwin, 1), 256, 0, s>>>(a, li.win, li.nwin, F[0], F[1], F[2],
                                                                     li.reg);
        MARK(nullptr);
        ++n;
    }
#undef MARK
    return n;
}

template <class R>
int launch_maxspeed(const StepArgs &a, long long max_cells, unsigned long long *out, cudaStream_t s,
                    ProfHook *prof)
{
    const int B = 256;
    if (prof) prof->mark("maxspeed", s);
    k_maxspeed<R><<<grid_for(max_cells, a.npatch, B), B, 0, s>>>(a, out);
    if (prof) prof->mark(nullptr, s);
    return 1;
}

} // namespace ctu
