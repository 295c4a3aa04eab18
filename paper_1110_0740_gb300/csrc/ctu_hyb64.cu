// FP64 MHD path, PPM or MC-linear, with the hybrid integration of the
// shock-detection appendix (HLL and MinMod where shocks are flagged).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<double, 1, 2>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
