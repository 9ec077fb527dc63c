// fv_update.cu -- the FP64 instantiations of the patch update / time-step
// kernel (fv_step.cuh) and the precision dispatch of its launches.
#include "fv_step.cuh"

namespace fv {

template cudaError_t launch_step_prec<double>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_prec<double>(int, int, int, int, int*);
// the FP32 instantiations live in fv_update_f32.cu
extern template cudaError_t launch_step_prec<float>(const fv_batch*, const UpdateLaunch&, int);
extern template cudaError_t occupancy_prec<float>(int, int, int, int, int*);

size_t update_smem_bytes(int d, fv_precision prec, int pmax, int nstage) {
  const int es = prec == FV_FP64 ? 8 : 4;
  return d == 1   ? step_smem_bytes<1>(es, pmax, nstage)
         : d == 2 ? step_smem_bytes<2>(es, pmax, nstage)
                  : step_smem_bytes<3>(es, pmax, nstage);
}

cudaError_t launch_update(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return h->prec == FV_FP64 ? launch_step_prec<double>(h, l, grid)
                            : launch_step_prec<float>(h, l, grid);
}

cudaError_t step_occupancy(const fv_batch* h, int mode, int pmax, int nstage, int* bps) {
  return h->prec == FV_FP64 ? occupancy_prec<double>(h->d, mode, pmax, nstage, bps)
                            : occupancy_prec<float>(h->d, mode, pmax, nstage, bps);
}

}  // namespace fv
