// FP64 MHD path, PPM or MC-linear, with the reference states of the tracing
// of Section 3.2 (cell centre, Colella-Woodward).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<double, 1, 1>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
