// Mixed MHD path (CTU_MIXED), PPM or MC-linear, with the parabolic terms
// (thermal conduction, viscosity).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<float, 0, 4>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
