// fv_update_f32.cu -- the FP32, 128-thread instantiations of the patch update
// / time-step kernel (fv_step.cuh), compiled in their own translation unit.
#include "fv_step.cuh"

namespace fv {

template cudaError_t launch_step_nt<float, 128>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<float, 128>(int, int, int, int, int*);

}  // namespace fv
