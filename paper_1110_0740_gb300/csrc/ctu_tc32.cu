// Mixed MHD path (CTU_MIXED), PPM or MC-linear, with thermal conduction (the
// parabolic term; float64 half-step temperature and update).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<float, 0, 4>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
