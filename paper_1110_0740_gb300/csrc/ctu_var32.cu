// Mixed MHD path (CTU_MIXED) with the other reconstructions of Section 3.2:
// linear with the MinMod, harmonic or Van Albada slope, improved WENO3.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_var<float, 0, 0>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
