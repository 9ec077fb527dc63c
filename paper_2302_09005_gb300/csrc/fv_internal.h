// fv_internal.h -- the handle and the kernel launchers behind the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "fv.h"

// Threads per CTA of the patch kernels.
#define FV_NT 128
// Maximum number of CTAs of a grid-stride reduction kernel (partials slots).
#define FV_MAX_RED_BLOCKS 4096
// Clock cycles a CTA waits for a copy before it reports FV_ERR_TIMEOUT
// (about one second at 2 GHz).
#define FV_WAIT_LIMIT 2000000000ll

struct fv_batch {
  int d = 0, s = 0, halo = 1;
  double gamma = 1.4;
  fv_precision prec = FV_FP64;
  int max_patch_size = 0;
  int nstage = 2;  // shared-memory stages of the update kernel
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  // device workspace (one allocation)
  void* ws = nullptr;
  unsigned int* d_status = nullptr;          // status bits
  double* d_dt = nullptr;                    // time step slot
  unsigned long long* d_lam = nullptr;       // two slots: bits of the global max wave speed
  int lam_cur = 0;                           // slot holding lambda of the current state
  unsigned long long* d_partials = nullptr;  // FV_MAX_RED_BLOCKS slots
  double* d_sum_partials = nullptr;          // FV_MAX_RED_BLOCKS * 8 slots
  unsigned long long* d_queue = nullptr;     // FV_SCHED_QUEUE: positions handed out
  int blocks_per_sm[3] = {0, 0, 0};          // occupancy by kernel mode (kModeUpdate..)
  // primitive carry of fv_run_steps: two buffers of prim_cap elements
  void* d_prim[2] = {nullptr, nullptr};
  int64_t prim_cap = 0;
  void* graph_cache = nullptr;               // captured multi-step graphs
  // schedule (fv_sched.cu): processing order sorted by size, size classes
  int sched = 0;                             // fv_schedule
  int32_t* d_order = nullptr;                // device int32[plan_cap]
  int64_t plan_cap = 0, plan_n = -1;
  const int32_t* plan_sizes = nullptr;       // the sizes array the plan was built from
  int ncls = 0;
  int cls_p[64] = {0};
  int64_t cls_begin[64] = {0}, cls_end[64] = {0};
  int occ_cache[3][64][4] = {{{0}}};         // CTAs per SM by (kernel mode, p, CTA size)
  int cls_nt[64] = {0};                      // CTA size of the size-class launches (0: 128)
  int cls_only = -1;                         // autotuner: launch only this class (-1: all)
  int cls_real[64] = {0};                    // class c holds one valid size (not the rejects)
  int occ_one[8][3] = {};                    // CTAs per SM of the FP32 one-size kernels, by p and mode
  int64_t pairs_launches = 0;                // launches that used an FP32 one-size kernel
  void* host_stage = nullptr;                // fv_patch_update_host: streams, staging buffers
  int smem_optin = 0;                        // opt-in shared memory per CTA
  long long wait_limit = FV_WAIT_LIMIT;      // step kernel: cycles of a copy wait
  char last_error[512] = {0};
};

namespace fv {

struct UpdateLaunch {
  const void* in = nullptr;
  void* out = nullptr;
  const int64_t* off = nullptr;
  const int32_t* sizes = nullptr;
  const int32_t* nbr = nullptr;    // time-step mode
  const int32_t* order = nullptr;  // processing order, or null for 0..n-1
  int64_t i_begin = 0, i_end = -1;  // positions to run (-1: n)
  int64_t n = 0;
  int64_t n_elems = 0;
  int pmax = 0;
  double gamma = 1.4;
  double dx = 0, dt = 0, cfl = 0;
  const double* dt_dev = nullptr;
  const unsigned long long* lam_in = nullptr;  // time-step mode
  unsigned long long* lam_next = nullptr;      // time-step mode
  double* dt_slot = nullptr;                   // time-step mode
  double* lam_patch = nullptr;
  const float* corr = nullptr;  // learned flux corrections (fv_learned.cu)
  int64_t corr_stride = 0;
  unsigned int* status = nullptr;
  bool fused = false;  // time-step mode: gather halos, dt from lam_in, reduce lam_next
  int nstage = 0;      // shared-memory stages (0: the handle's)
  int nt = 128;        // threads per CTA
  const double* dx_patch = nullptr;  // update mode: per-patch cell sizes, or null
  double* dt_patch = nullptr;        // with dx_patch: per-patch dt (in, or out with local_cfl)
  bool local_cfl = false;
  const void* prim_in = nullptr;  // time step: carried primitives of `in`, or null
  void* prim_out = nullptr;       // time step: primitives of `out`, or null
  int64_t prim_stride = 0;        // elements per patch of the primitive buffers
  int uniform_p = 0;              // every patch of the launch has this size (0: unknown)
  unsigned long long* queue = nullptr;  // zeroed counter: CTAs pop positions (null: stride)
};

// Kernel modes: update (halos filled by the caller), time step (halo gather,
// CFL from the device, next-step maximum), time step with primitive carry.
constexpr int kModeUpdate = 0;
constexpr int kModeStep = 1;
constexpr int kModePrim = 2;
inline int step_mode(const UpdateLaunch& l) {
  return !l.fused ? kModeUpdate : (l.prim_in != nullptr ? kModePrim : kModeStep);
}

// Elements per patch of a primitive buffer: (d + 3) p^d for p = pmax, rounded
// up to 16 bytes.
inline int64_t prim_stride_elems(int d, fv_precision prec, int pmax) {
  int64_t c = d + 3;
  for (int k = 0; k < d; ++k) c *= pmax;
  const int64_t vec = prec == FV_FP64 ? 2 : 4;
  return (c + vec - 1) / vec * vec;
}

// Serialises the check-and-raise of the kernels' dynamic shared-memory limits
// (cudaFuncSetAttribute), which handles on several host threads may request
// at once: without it one thread could lower a limit another just raised.
std::mutex& smem_attr_mutex();

// Shared memory bytes of the update kernel for patches up to pmax.
size_t update_smem_bytes(int d, fv_precision prec, int pmax, int nstage);
cudaError_t launch_update(const fv_batch* h, const UpdateLaunch& a, int grid);
cudaError_t step_occupancy(const fv_batch* h, int mode, int pmax, int nstage, int nt,
                           int* blocks_per_sm);
// Threads per CTA of the step kernel for one launch: 32, 64, 128 or 256.
inline bool valid_nt(int nt) { return nt == 32 || nt == 64 || nt == 128 || nt == 256; }
inline int nt_index(int nt) { return nt == 32 ? 0 : nt == 64 ? 1 : nt == 128 ? 2 : 3; }
// CTA size of launches nobody tuned, by the interior cells p^d of the
// patches: a warp for up to 64 cells (the small 2D patches and 3^3), eight
// warps for 3D patches above 200 cells, else four (measured on GB300: 2D
// 5x5 patches run 1.75x faster on one warp than on four; the size-class
// autotuner chose the same for 3^3, 5^3 and 7^3).  d = 1 runs 128 threads.
inline int default_nt(int d, int p) {
  if (d == 1) return 128;
  int n = 1;
  for (int k = 0; k < d; ++k) n *= p;
  if (n <= 64) return 32;
  if (d == 3 && n > 200) return 256;
  return 128;
}
// Per-precision, per-CTA-size launch and occupancy (fv_update.cu: double and
// 128 threads; fv_update_f32.cu: float and 128; fv_update_nt.cu and
// fv_update_nt_f32.cu: 32, 64 and 256 threads).
template <typename T, int NT>
cudaError_t launch_step_nt(const fv_batch* h, const UpdateLaunch& l, int grid);
template <typename T, int NT>
cudaError_t occupancy_nt(int d, int mode, int pmax, int nstage, int* bps);
// The same for launches of one 2D patch size, p = 3 .. 6 (fv_rows2d.cu: a lane
// per row of cells, four patches per warp, rows2d_patches_per_cta() patches
// per CTA and iteration).
bool rows2d_class(const fv_batch* h, int p);
bool rows2d_eligible(const fv_batch* h, const UpdateLaunch& l);
int rows2d_patches_per_cta();
cudaError_t launch_rows2d(const fv_batch* h, const UpdateLaunch& l, int grid);
cudaError_t rows2d_occupancy(int p, int mode, int* blocks_per_sm);
// The FP32 kernel for launches of 3D patches of size p = 3, 5 or 7 (fv_march3d.cu: a
// lane per row of cells, four patches per warp, each patch advanced plane by
// plane along z; march3d_patches_per_cta() patches per CTA and iteration):
// whether a size class / a launch can use it, its launch and its occupancy.
bool march3d_class(const fv_batch* h, int p);
bool march3d_eligible(const fv_batch* h, const UpdateLaunch& l);
int march3d_patches_per_cta();
cudaError_t launch_march3d(const fv_batch* h, const UpdateLaunch& l, int grid);
cudaError_t march3d_occupancy(int p, int mode, int* blocks_per_sm);
// Launches the update / time-step kernel(s) under the handle's schedule.
cudaError_t launch_scheduled(fv_batch* h, UpdateLaunch l);
// Frees the schedule plan of a handle.
void plan_free(fv_batch* h);
// Frees the host-offload staging of a handle (fv_host.cu).
void host_stage_free(fv_batch* h);

struct EigLaunch {
  const void* q;
  const int64_t* off;
  const int32_t* sizes;
  int64_t n;
  int halo;
  double gamma;
  double* per_patch;
  unsigned long long* partials;
  unsigned int* status;
};
cudaError_t launch_eig(const fv_batch* h, const EigLaunch& a, int grid);
// *p = 0 on the stream, by a one-thread kernel.
cudaError_t launch_zero_word(unsigned long long* p, cudaStream_t stream);
cudaError_t launch_eig_finish(const fv_batch* h, const unsigned long long* partials, int nparts,
                              double* global_out, unsigned long long* lam_slot, double* dt_slot,
                              double* dt_out, double cfl, double dx);

struct HaloLaunch {
  void* q;
  const int64_t* off;
  const int32_t* sizes;
  const int32_t* nbr;
  int64_t n;
  int halo;
  unsigned int* status;
};
cudaError_t launch_halo(const fv_batch* h, const HaloLaunch& a, int grid);

struct SumLaunch {
  const void* q;
  const int64_t* off;
  const int32_t* sizes;
  int64_t n;
  int halo;
  double* partials;  // [nchunks][s]
  unsigned int* status;
  double* per_patch = nullptr;  // [n][s] or null: each valid patch's sums
};
// Patches per chunk of the fixed-order conservation sum.
#define FV_SUM_CHUNK 1024
cudaError_t launch_sums(const fv_batch* h, const SumLaunch& a, int nchunks);
cudaError_t launch_sums_finish(const fv_batch* h, const double* partials, int nchunks,
                               double* totals);

cudaError_t launch_selftest_math(const double* x, double* out, int64_t n, int which);

}  // namespace fv
