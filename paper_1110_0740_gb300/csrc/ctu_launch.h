// ctu_launch.h -- host-side launchers of the CTU kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "ctu_kernels.cuh"

namespace ctu {

// Scratch elements of type R needed per unit of scratch stride.
constexpr int SCRATCH_ARRAYS = 9 /*V*/ + 27 /*F1*/ + 18 /*Vp,Vm*/ + 27 /*F*/;

// Optional per-kernel timing hook: mark(name) is called right before a
// launch and mark(nullptr) right after it, on the same stream.
struct ProfHook {
    virtual void mark(const char *name, cudaStream_t s) = 0;
    virtual ~ProfHook() {}
};

struct LaunchInfo {
    long long max_cells;   // largest ghosted patch
    int recon;             // 0 linear, 1 PPM
    const DevWindow *win;  // device windows (may be null)
    int nwin;
    double *reg;
    void *scratch;         // SCRATCH_ARRAYS * sstride elements of R
    ProfHook *prof;        // may be null
    int iface64;           // mixed path: 1 = float64 interface-state recovery
};

template <class R> int launch_step(const StepArgs &a, const LaunchInfo &li, cudaStream_t s);
template <class R> int launch_maxspeed(const StepArgs &a, long long max_cells, unsigned long long *out,
                                       cudaStream_t s, ProfHook *prof);

} // namespace ctu
