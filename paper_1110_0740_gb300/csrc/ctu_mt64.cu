// FP64 MHD path, PPM or MC-linear, with the corner coupling of Mignone &
// Tzeferacos (transverse fluxes from the normal predictor states).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_mt<double, 1>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
