// FP64 paths: every stage in float64 (ideal MHD and SRMHD).
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_impl<double, 1>(const StepArgs &, const LaunchInfo &, cudaStream_t);
template int launch_step_sr<double>(const StepArgs &, const LaunchInfo &, cudaStream_t);
template <> int launch_maxspeed<double>(const StepArgs &a, const LaunchInfo &li, unsigned long long *out,
                                        cudaStream_t s)
{
    return li.physics == PH_SR ? launch_maxspeed_impl<PH_SR, double>(a, li, out, s)
                               : launch_maxspeed_impl<PH_MHD, double>(a, li, out, s);
}
} // namespace ctu
