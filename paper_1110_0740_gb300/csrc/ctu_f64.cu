// FP64 path: every stage in float64.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_impl<double, 1>(const StepArgs &, const LaunchInfo &, cudaStream_t);
template <> int launch_maxspeed<double>(const StepArgs &a, const LaunchInfo &li, unsigned long long *out,
                                        cudaStream_t s)
{
    return launch_maxspeed_impl<double>(a, li, out, s);
}
} // namespace ctu
