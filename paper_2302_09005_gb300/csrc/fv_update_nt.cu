// fv_update_nt.cu -- the FP64 instantiations of the patch update / time-step
// kernel (fv_step.cuh) for one-warp, two-warp and eight-warp CTAs (small and
// large patch-size classes).
#include "fv_step.cuh"

namespace fv {

template cudaError_t launch_step_nt<double, 32>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<double, 32>(int, int, int, int, int*);
template cudaError_t launch_step_nt<double, 64>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<double, 64>(int, int, int, int, int*);
template cudaError_t launch_step_nt<double, 256>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<double, 256>(int, int, int, int, int*);

}  // namespace fv
