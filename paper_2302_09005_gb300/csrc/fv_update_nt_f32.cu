// fv_update_nt_f32.cu -- the FP32 instantiations of the patch update /
// time-step kernel (fv_step.cuh) for one-warp, two-warp and eight-warp CTAs.
#include "fv_step.cuh"

namespace fv {

template cudaError_t launch_step_nt<float, 32>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<float, 32>(int, int, int, int, int*);
template cudaError_t launch_step_nt<float, 64>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<float, 64>(int, int, int, int, int*);
template cudaError_t launch_step_nt<float, 256>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<float, 256>(int, int, int, int, int*);

}  // namespace fv
