// FP64 instantiation of the CTU kernels.
#include "ctu_launch.cuh"

namespace ctu {
template int launch_step<double>(const StepArgs &, const LaunchInfo &, cudaStream_t);
template int launch_maxspeed<double>(const StepArgs &, long long, unsigned long long *, cudaStream_t,
                                       ProfHook *);
} // namespace ctu
