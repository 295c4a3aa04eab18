// Mixed MHD path (CTU_MIXED), PPM or MC-linear, with the reference states of
// the tracing of Section 3.2 (cell centre, Colella-Woodward).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<float, 0, 1>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
