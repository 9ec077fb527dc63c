// fv_noalloc.cu -- fv_conserved_totals_noalloc: the conservation sums without
// a handle and without any device allocation.
//
// Some callers cannot allocate device memory at all: an engine that hands
// the whole GPU to its own memory pool and forbids other allocations, or a
// latency-critical loop where cudaMalloc/cudaFree would synchronise the
// device.  Such callers cannot create an fv_batch (its workspace is
// allocated), yet may still want the fixed-order FP64 totals.  This entry
// point runs the same kernels as fv_conserved_totals, with the per-chunk
// partial sums kept in a fixed-size array in the library's own static device
// memory instead of a handle workspace.
#include <mutex>

#include "fv_device.cuh"
#include "fv_internal.h"

namespace {

// Partial sums of the two-stage reduction: one slot of 8 doubles per chunk
// of FV_SUM_CHUNK patches.  256 KiB, held on every device that loads the
// library until the process exits.
constexpr int kNoallocChunks = 4096;
static __device__ __align__(256) double g_noalloc_partials[kNoallocChunks * 8];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device.  Looked up once
// per device (with that device current) and cached; host code cannot use the
// array's name as a device address.
cudaError_t noalloc_partials(double** partials) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_partials_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *partials = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" fv_status fv_conserved_totals_noalloc(int d, int s, fv_precision precision,
                                                 const void* q_with_halo,
                                                 const int64_t* patch_offsets,
                                                 const int32_t* patch_sizes, int64_t n_patches,
                                                 double* totals, unsigned int* status_word,
                                                 void* cuda_stream) {
  if (d < 1 || d > 3 || s != d + 2) return FV_ERR_INVALID_ARG;
  if (precision != FV_FP64 && precision != FV_FP32) return FV_ERR_INVALID_ARG;
  // the status word is required: the library keeps no word of its own that
  // a caller could read, so without one bad patches would go unreported
  if (n_patches < 0 || !totals || !status_word) return FV_ERR_INVALID_ARG;
  if (n_patches > (int64_t)kNoallocChunks * FV_SUM_CHUNK) return FV_ERR_UNSUPPORTED;
  if (n_patches > 0) {
    if (!q_with_halo || !patch_offsets || !patch_sizes) return FV_ERR_INVALID_ARG;
    if (((uintptr_t)q_with_halo & 15u) || ((uintptr_t)patch_offsets & 7u) ||
        ((uintptr_t)patch_sizes & 3u))
      return FV_ERR_ALIGNMENT;
  }
  if ((uintptr_t)status_word & 3u) return FV_ERR_ALIGNMENT;
  double* partials = nullptr;
  if (noalloc_partials(&partials) != cudaSuccess) return FV_ERR_CUDA;

  // A handle-shaped description on the stack: no workspace, no allocation.
  fv_batch desc;
  desc.d = d;
  desc.s = s;
  desc.halo = 1;
  desc.prec = precision;
  desc.max_patch_size = 64;
  desc.stream = static_cast<cudaStream_t>(cuda_stream);

  const int nchunks = (int)((n_patches + FV_SUM_CHUNK - 1) / FV_SUM_CHUNK);
  cudaError_t e = cudaSuccess;
  if (nchunks > 0) {
    fv::SumLaunch l;
    l.q = q_with_halo;
    l.off = patch_offsets;
    l.sizes = patch_sizes;
    l.n = n_patches;
    l.halo = 1;
    l.partials = partials;  // every slot the finish reads is written first
    l.status = status_word;
    e = fv::launch_sums(&desc, l, nchunks);
  }
  if (e == cudaSuccess) e = fv::launch_sums_finish(&desc, partials, nchunks, totals);
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}
