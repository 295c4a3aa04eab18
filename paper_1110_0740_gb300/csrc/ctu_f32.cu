// Mixed-precision instantiation: tracing, projections and Riemann fluxes in
// float32; pressure recovery, interface conservative states and the update
// accumulation stay in float64 inside the kernels.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step<float>(const StepArgs &, const LaunchInfo &, cudaStream_t);
template int launch_maxspeed<float>(const StepArgs &, long long, unsigned long long *, cudaStream_t,
                                       ProfHook *);
} // namespace ctu
