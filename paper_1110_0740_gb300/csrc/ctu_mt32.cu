// Mixed MHD path (CTU_MIXED), PPM or MC-linear, with the corner coupling of
// Mignone & Tzeferacos (transverse fluxes from the normal predictor states).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_mt<float, 0>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
