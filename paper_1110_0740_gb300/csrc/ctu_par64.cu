// FP64 MHD path, PPM or MC-linear, with the parabolic terms
// (thermal conduction, viscosity).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<double, 1, 4>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
