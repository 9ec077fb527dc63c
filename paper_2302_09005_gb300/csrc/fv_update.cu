// fv_update.cu -- the FP64, 128-thread instantiations of the patch update /
// time-step kernel (fv_step.cuh) and the dispatch of its launches over
// precision and CTA size.
#include "fv_step.cuh"

namespace fv {

template cudaError_t launch_step_nt<double, 128>(const fv_batch*, const UpdateLaunch&, int);
template cudaError_t occupancy_nt<double, 128>(int, int, int, int, int*);
// the other instantiations live in fv_update_f32.cu, fv_update_nt.cu and
// fv_update_nt_f32.cu
#define FV_EXTERN(T, NT)                                                                    \
  extern template cudaError_t launch_step_nt<T, NT>(const fv_batch*, const UpdateLaunch&, \
                                                    int);                                   \
  extern template cudaError_t occupancy_nt<T, NT>(int, int, int, int, int*);
FV_EXTERN(float, 128)
FV_EXTERN(double, 32)
FV_EXTERN(double, 64)
FV_EXTERN(double, 256)
FV_EXTERN(float, 32)
FV_EXTERN(float, 64)
FV_EXTERN(float, 256)
#undef FV_EXTERN

size_t update_smem_bytes(int d, fv_precision prec, int pmax, int nstage) {
  const int es = prec == FV_FP64 ? 8 : 4;
  return d == 1   ? step_smem_bytes<1>(es, pmax, nstage)
         : d == 2 ? step_smem_bytes<2>(es, pmax, nstage)
                  : step_smem_bytes<3>(es, pmax, nstage);
}

template <typename T>
static cudaError_t launch_prec(const fv_batch* h, const UpdateLaunch& l, int grid) {
  switch (l.nt) {
    case 32: return launch_step_nt<T, 32>(h, l, grid);
    case 64: return launch_step_nt<T, 64>(h, l, grid);
    case 256: return launch_step_nt<T, 256>(h, l, grid);
    default: return launch_step_nt<T, 128>(h, l, grid);
  }
}

template <typename T>
static cudaError_t occupancy_prec(int d, int mode, int pmax, int nstage, int nt, int* bps) {
  switch (nt) {
    case 32: return occupancy_nt<T, 32>(d, mode, pmax, nstage, bps);
    case 64: return occupancy_nt<T, 64>(d, mode, pmax, nstage, bps);
    case 256: return occupancy_nt<T, 256>(d, mode, pmax, nstage, bps);
    default: return occupancy_nt<T, 128>(d, mode, pmax, nstage, bps);
  }
}

cudaError_t launch_update(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return h->prec == FV_FP64 ? launch_prec<double>(h, l, grid) : launch_prec<float>(h, l, grid);
}

cudaError_t step_occupancy(const fv_batch* h, int mode, int pmax, int nstage, int nt, int* bps) {
  return h->prec == FV_FP64 ? occupancy_prec<double>(h->d, mode, pmax, nstage, nt, bps)
                            : occupancy_prec<float>(h->d, mode, pmax, nstage, nt, bps);
}

}  // namespace fv
