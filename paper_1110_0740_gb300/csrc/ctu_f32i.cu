// Mixed path, CTU_MIXED_IFACE64 variant: interface states formed and their
// pressure recovered in float64.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_impl<float, 1>(const StepArgs &, const LaunchInfo &, cudaStream_t);
} // namespace ctu
