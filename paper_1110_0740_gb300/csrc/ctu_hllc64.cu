// FP64 MHD path, PPM or MC-linear, with the HLLC Riemann solver
// (Li 2005) on every face.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<double, 1, 3>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
