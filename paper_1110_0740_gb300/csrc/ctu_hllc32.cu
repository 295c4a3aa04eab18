// Mixed MHD path (CTU_MIXED), PPM or MC-linear, with the HLLC Riemann solver
// (Li 2005) on every face.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<float, 0, 3>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
