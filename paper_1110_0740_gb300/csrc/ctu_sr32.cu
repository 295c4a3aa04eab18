// Mixed SRMHD path: float32 MUSCL-Hancock slopes, fluxes and HLL;
// float64 Newton-Raphson primitive recovery and update accumulation.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_sr<float>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
