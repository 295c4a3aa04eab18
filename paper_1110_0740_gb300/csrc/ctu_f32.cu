// Mixed MHD path (CTU_MIXED): float32 tracing, projections, Riemann fluxes
// and interface states; float64 state, double-float pressure recovery at
// cell centres, float64 update accumulation.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step_impl<float, 0>(const StepArgs &, const LaunchInfo &, cudaStream_t);
template <> int launch_maxspeed<float>(const StepArgs &a, const LaunchInfo &li, unsigned long long *out,
                                       cudaStream_t s)
{
    if (li.physics == PH_SR) return launch_maxspeed_impl<PH_SR, float>(a, li, out, s);
    return li.iface64 ? launch_maxspeed_impl<PH_MHD, float, 1>(a, li, out, s)
                      : launch_maxspeed_impl<PH_MHD, float>(a, li, out, s);
}
} // namespace ctu
