// ctu_launch.h -- host-side launchers of the CTU kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "ctu_kernels.cuh"

namespace ctu {

// Scratch words (of the working precision) per unit of scratch stride:
// V (9), first-order fluxes F^n (3 x 9), running sum A = L_x (+ L_y) (9).
constexpr int SCRATCH_ARRAYS = 9 + 27 + 9;

// Optional per-kernel timing hook: mark(name) is called right before a
// launch and mark(nullptr) right after it, on the same stream.
struct ProfHook {
    virtual void mark(const char *name, cudaStream_t s) = 0;
    virtual ~ProfHook() {}
};

// Patches of identical shape, contiguous in the device patch table, with the
// thread-tile width along x (8, 16 or 32) and the marching segment length
// their kernels use.  A launch covers up to MAXG groups (GroupTable).
struct Group {
    int first, count;
    int n[3], N[3];
    int xw, seg;
};

struct LaunchInfo {
    const Group *groups;   // host array, largest patches first
    int ngroups;
    int recon;             // RECON_* kernel kind (reconstruction, reference-state tracing)
    int iface64;           // mixed path: 1 = float64 interface-state recovery
    int physics;           // PH_MHD or PH_SR
    void *scratch;         // SCRATCH_ARRAYS * sstride elements of R
    StepParams *sp;        // device per-step parameters
    ProfHook *prof;        // may be null
    int sms;               // streaming multiprocessors of the device (launch_rows)
};

// Enqueue one CTU step; returns the number of kernel launches.
template <class R> int launch_step(const StepArgs &a, const LaunchInfo &li, cudaStream_t s);
// Enqueue the CFL reduction of ctu_dt into *out.
template <class R> int launch_maxspeed(const StepArgs &a, const LaunchInfo &li, unsigned long long *out,
                                       cudaStream_t s);

// Per-(precision, physics, interface-mode) instantiations, one translation
// unit each.
template <class R, int IF64> int launch_step_impl(const StepArgs &a, const LaunchInfo &li, cudaStream_t s);
template <class R> int launch_step_sr(const StepArgs &a, const LaunchInfo &li, cudaStream_t s);
template <class R, int IF64, int G> int launch_step_var(const StepArgs &a, const LaunchInfo &li, cudaStream_t s);
template <class R, int IF64> int launch_step_mt(const StepArgs &a, const LaunchInfo &li, cudaStream_t s);

} // namespace ctu
