// fv_api.cu -- the C ABI declared in include/fv.h: handle life cycle,
// host-side argument validation, launch geometry and status reporting.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <new>
#include <tuple>
#include <utility>

#include "fv_device.cuh"
#include "fv_internal.h"

namespace fv {

std::mutex& smem_attr_mutex() {
  static std::mutex m;
  return m;
}

}  // namespace fv

namespace {

// Instantiated CUDA graphs of fv_run_steps, keyed by every argument that is
// baked into the captured launches.
using GraphKey = std::tuple<const void*, const void*, const void*, const void*, const void*,
                            int64_t, double, double, int, int>;
struct GraphCache {
  std::map<GraphKey, cudaGraphExec_t> exec;
};

void graph_cache_clear(fv_batch* h) {
  auto* gc = static_cast<GraphCache*>(h->graph_cache);
  if (!gc) return;
  for (auto& kv : gc->exec) cudaGraphExecDestroy(kv.second);
  delete gc;
  h->graph_cache = nullptr;
}

fv_status set_err(fv_batch* h, fv_status st, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->last_error, sizeof(h->last_error), fmt, ap);
    va_end(ap);
  }
  return st;
}

fv_status cuda_err(fv_batch* h, cudaError_t e, const char* where) {
  return set_err(h, FV_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Grid of a grid-stride patch kernel: enough CTAs to fill every SM, never
// more than there are patches or partial slots.
int patch_grid(const fv_batch* h, int64_t n, int blocks_per_sm) {
  int64_t g = (int64_t)h->num_sms * (blocks_per_sm > 0 ? blocks_per_sm : 1);
  if (g > n) g = n;
  if (g > FV_MAX_RED_BLOCKS) g = FV_MAX_RED_BLOCKS;
  return (int)(g < 1 ? 1 : g);
}

fv_status check_meta(fv_batch* h, const void* buf, const int64_t* off, const int32_t* sizes,
                     int64_t n) {
  if (n < 0) return set_err(h, FV_ERR_INVALID_ARG, "n_patches < 0");
  if (n == 0) return FV_OK;
  if (!buf || !off || !sizes) return set_err(h, FV_ERR_INVALID_ARG, "null device pointer");
  if (!aligned16(buf)) return set_err(h, FV_ERR_ALIGNMENT, "buffer not 16-byte aligned");
  if (((uintptr_t)off & 7u) || ((uintptr_t)sizes & 3u))
    return set_err(h, FV_ERR_ALIGNMENT, "metadata arrays misaligned");
  return FV_OK;
}

}  // namespace

extern "C" {

void fv_options_default(fv_options* o) {
  if (!o) return;
  o->gamma = 1.4;
  o->halo = 1;
  o->precision = FV_FP64;
  o->max_patch_size = 0;
}

const char* fv_status_string(fv_status s) {
  switch (s) {
    case FV_OK: return "FV_OK";
    case FV_ERR_INVALID_ARG: return "FV_ERR_INVALID_ARG";
    case FV_ERR_ALIGNMENT: return "FV_ERR_ALIGNMENT";
    case FV_ERR_UNSUPPORTED: return "FV_ERR_UNSUPPORTED";
    case FV_ERR_CUDA: return "FV_ERR_CUDA";
    case FV_ERR_NONPHYSICAL: return "FV_ERR_NONPHYSICAL";
    case FV_ERR_TIMEOUT: return "FV_ERR_TIMEOUT";
    case FV_ERR_BAD_PATCH: return "FV_ERR_BAD_PATCH";
  }
  return "unknown fv_status";
}

fv_status fv_batch_create(fv_batch** out, int d, int s, const fv_options* o, void* stream) {
  if (!out) return FV_ERR_INVALID_ARG;
  *out = nullptr;
  fv_options opt;
  fv_options_default(&opt);
  if (o) opt = *o;
  if (d < 1 || d > 3 || s != d + 2) return FV_ERR_INVALID_ARG;
  if (!(opt.gamma > 1.0) || opt.halo < 1 || opt.halo > 4) return FV_ERR_INVALID_ARG;
  if (opt.precision != FV_FP64 && opt.precision != FV_FP32) return FV_ERR_INVALID_ARG;
  if (opt.max_patch_size < 0) return FV_ERR_INVALID_ARG;
  if (opt.max_patch_size == 0) opt.max_patch_size = d == 3 ? 8 : 17;
  if (opt.halo != 1) return FV_ERR_UNSUPPORTED;  // the Rusanov update reads one layer
  fv_batch* h = new (std::nothrow) fv_batch();
  if (!h) return FV_ERR_CUDA;
  h->d = d;
  h->s = s;
  h->halo = opt.halo;
  h->gamma = opt.gamma;
  h->prec = opt.precision;
  h->max_patch_size = opt.max_patch_size;
  h->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  int smem_optin = 0;
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  h->smem_optin = smem_optin;
#ifdef FV_FORCE_SINGLE_STAGE
  h->nstage = 1;
#else
  h->nstage = 2;
#endif
  if (e == cudaSuccess &&
      fv::update_smem_bytes(d, h->prec, h->max_patch_size, 2) > (size_t)smem_optin)
    h->nstage = 1;
  if (e == cudaSuccess &&
      fv::update_smem_bytes(d, h->prec, h->max_patch_size, 1) > (size_t)smem_optin) {
    delete h;
    return FV_ERR_UNSUPPORTED;  // max_patch_size too large for shared memory
  }
  // workspace: status | dt | lam | queue | partials (u64) | sum partials (double, 8
  // per slot)
  const size_t bytes = 256 + 8ull * FV_MAX_RED_BLOCKS + 64ull * FV_MAX_RED_BLOCKS;
  if (e == cudaSuccess) e = cudaMalloc(&h->ws, bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws, 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    if (h->ws) cudaFree(h->ws);
    delete h;
    return FV_ERR_CUDA;
  }
  char* w = static_cast<char*>(h->ws);
  h->d_status = reinterpret_cast<unsigned int*>(w);
  h->d_dt = reinterpret_cast<double*>(w + 64);
  h->d_lam = reinterpret_cast<unsigned long long*>(w + 128);
  h->d_queue = reinterpret_cast<unsigned long long*>(w + 192);
  h->d_partials = reinterpret_cast<unsigned long long*>(w + 256);
  h->d_sum_partials = reinterpret_cast<double*>(w + 256 + 8ull * FV_MAX_RED_BLOCKS);
  // CTAs per SM of the untuned launches (their CTA size follows the patch size)
  for (int mode = fv::kModeUpdate; mode <= fv::kModePrim && e == cudaSuccess; ++mode)
    e = fv::step_occupancy(h, mode, h->max_patch_size, h->nstage,
                           fv::default_nt(d, h->max_patch_size), &h->blocks_per_sm[mode]);
  if (e != cudaSuccess) {
    cudaFree(h->ws);
    delete h;
    return FV_ERR_CUDA;
  }
  *out = h;
  return FV_OK;
}

fv_status fv_batch_destroy(fv_batch* h) {
  if (!h) return FV_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  graph_cache_clear(h);
  fv::plan_free(h);
  fv::host_stage_free(h);
  for (void* pbuf : h->d_prim)
    if (pbuf) cudaFree(pbuf);
  cudaError_t e2 = cudaFree(h->ws);
  delete h;
  return (e == cudaSuccess && e2 == cudaSuccess) ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_batch_set_stream(fv_batch* h, void* stream) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return FV_OK;
}

fv_status fv_patch_update_batch_ex(fv_batch* h, const void* in, void* out, const int64_t* off,
                                   const int32_t* sizes, int64_t n, int d, int s, double dx,
                                   double dt, const fv_update_extras* ex) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (d != h->d || s != h->s) return set_err(h, FV_ERR_INVALID_ARG, "d/s differ from handle");
  if (!(dx > 0.0)) return set_err(h, FV_ERR_INVALID_ARG, "dx must be > 0");
  if (dt != dt) return set_err(h, FV_ERR_INVALID_ARG, "dt is NaN");
  fv_status st = check_meta(h, in, off, sizes, n);
  if (st != FV_OK) return st;
  if (n == 0) return FV_OK;
  if (!out) return set_err(h, FV_ERR_INVALID_ARG, "null output");
  if (!aligned16(out)) return set_err(h, FV_ERR_ALIGNMENT, "output not 16-byte aligned");
  if (in == out) return set_err(h, FV_ERR_INVALID_ARG, "in and out alias");
  int64_t n_elems = ex ? ex->n_elems : 0;
  if (n_elems < 0) return set_err(h, FV_ERR_INVALID_ARG, "n_elems < 0");
  if (n_elems > 0) {
    const size_t es = h->prec == FV_FP64 ? 8 : 4;
    const char* a = static_cast<const char*>(in);
    const char* b = static_cast<const char*>(out);
    if (a < b + n_elems * es && b < a + n_elems * es)
      return set_err(h, FV_ERR_INVALID_ARG, "in and out overlap");
  }
  fv::UpdateLaunch l;
  l.in = in;
  l.out = out;
  l.off = off;
  l.sizes = sizes;
  l.n = n;
  l.n_elems = n_elems;
  l.pmax = h->max_patch_size;
  l.gamma = h->gamma;
  l.dx = dx;
  l.dt = dt;
  l.dt_dev = h->d_dt;
  l.lam_patch = ex ? ex->lambda_patch : nullptr;
  l.corr = ex ? ex->corr : nullptr;
  l.corr_stride = 2ll * 4 * (h->max_patch_size + 1) * h->max_patch_size;
  if (l.corr && h->d != 2) return set_err(h, FV_ERR_UNSUPPORTED, "corrections are 2D");
  l.status = h->d_status;
  l.fused = false;
  cudaError_t e = fv::launch_scheduled(h, l);
  if (e != cudaSuccess) return cuda_err(h, e, "update kernel");
  return FV_OK;
}

fv_status fv_patch_update_batch(fv_batch* h, const void* in, void* out, const int64_t* off,
                                const int32_t* sizes, int64_t n, int d, int s, double dx,
                                double dt) {
  return fv_patch_update_batch_ex(h, in, out, off, sizes, n, d, s, dx, dt, nullptr);
}

fv_status fv_patch_update_local(fv_batch* h, const void* in, void* out, const int64_t* off,
                               const int32_t* sizes, int64_t n, const double* dx_patch,
                               double* dt_patch, double cfl, double* lambda_patch) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (cfl != cfl) return set_err(h, FV_ERR_INVALID_ARG, "cfl is NaN");
  fv_status st = check_meta(h, in, off, sizes, n);
  if (st != FV_OK) return st;
  if (n == 0) return FV_OK;
  if (!out || !dx_patch || !dt_patch)
    return set_err(h, FV_ERR_INVALID_ARG, "null output, dx_patch or dt_patch");
  if (!aligned16(out)) return set_err(h, FV_ERR_ALIGNMENT, "output not 16-byte aligned");
  if (((uintptr_t)dx_patch & 7u) || ((uintptr_t)dt_patch & 7u))
    return set_err(h, FV_ERR_ALIGNMENT, "dx_patch / dt_patch not 8-byte aligned");
  if (in == out) return set_err(h, FV_ERR_INVALID_ARG, "in and out alias");
  fv::UpdateLaunch l;
  l.in = in;
  l.out = out;
  l.off = off;
  l.sizes = sizes;
  l.n = n;
  l.pmax = h->max_patch_size;
  l.gamma = h->gamma;
  l.dx = 1.0;  // replaced per patch
  l.dt = 1.0;
  l.cfl = cfl;
  l.dt_dev = h->d_dt;
  l.lam_patch = lambda_patch;
  l.dx_patch = dx_patch;
  l.dt_patch = dt_patch;
  l.local_cfl = cfl > 0.0;
  l.status = h->d_status;
  l.fused = false;
  cudaError_t e = fv::launch_scheduled(h, l);
  if (e != cudaSuccess) return cuda_err(h, e, "update kernel");
  return FV_OK;
}

fv_status fv_halo_fill(fv_batch* h, void* q, const int64_t* off, const int32_t* sizes,
                       const int32_t* nbr, int64_t n) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  fv_status st = check_meta(h, q, off, sizes, n);
  if (st != FV_OK) return st;
  if (n == 0) return FV_OK;
  if (!nbr) return set_err(h, FV_ERR_INVALID_ARG, "null neighbour table");
  fv::HaloLaunch l;
  l.q = q;
  l.off = off;
  l.sizes = sizes;
  l.nbr = nbr;
  l.n = n;
  l.halo = h->halo;
  l.status = h->d_status;
  // 12 CTAs of four warps per SM (a warp per patch; under 40 registers)
  cudaError_t e = fv::launch_halo(h, l, patch_grid(h, n, 12));
  if (e != cudaSuccess) return cuda_err(h, e, "halo kernel");
  return FV_OK;
}

fv_status fv_max_eigenvalue_reduce(fv_batch* h, const void* q, const int64_t* off,
                                   const int32_t* sizes, int64_t n, double* per_patch,
                                   double* global_max, double cfl, double dx, double* dt_out) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (!(cfl > 0.0) || !(dx > 0.0)) return set_err(h, FV_ERR_INVALID_ARG, "cfl, dx must be > 0");
  fv_status st = check_meta(h, q, off, sizes, n);
  if (st != FV_OK) return st;
  int grid = 0;
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    grid = patch_grid(h, n, 8);
    fv::EigLaunch l;
    l.q = q;
    l.off = off;
    l.sizes = sizes;
    l.n = n;
    l.halo = h->halo;
    l.gamma = h->gamma;
    l.per_patch = per_patch;
    l.partials = h->d_partials;
    l.status = h->d_status;
    e = fv::launch_eig(h, l, grid);
    if (e != cudaSuccess) return cuda_err(h, e, "eigenvalue kernel");
  }
  e = fv::launch_eig_finish(h, h->d_partials, grid, global_max, &h->d_lam[h->lam_cur], h->d_dt,
                            dt_out, cfl, dx);
  if (e != cudaSuccess) return cuda_err(h, e, "eigenvalue finish kernel");
  return FV_OK;
}

static fv_status sums_impl(fv_batch* h, const void* q, const int64_t* off, const int32_t* sizes,
                           int64_t n, double* totals, double* per_patch) {
  fv_status st = check_meta(h, q, off, sizes, n);
  if (st != FV_OK) return st;
  const int64_t nchunks = (n + FV_SUM_CHUNK - 1) / FV_SUM_CHUNK;
  if (nchunks > FV_MAX_RED_BLOCKS)
    return set_err(h, FV_ERR_UNSUPPORTED, "more than %d patches", FV_MAX_RED_BLOCKS * FV_SUM_CHUNK);
  cudaError_t e = cudaSuccess;
  if (nchunks > 0) {
    fv::SumLaunch l;
    l.q = q;
    l.off = off;
    l.sizes = sizes;
    l.n = n;
    l.halo = h->halo;
    l.partials = h->d_sum_partials;
    l.status = h->d_status;
    l.per_patch = per_patch;
    e = fv::launch_sums(h, l, (int)nchunks);
    if (e != cudaSuccess) return cuda_err(h, e, "sums kernel");
  }
  if (totals) {
    e = fv::launch_sums_finish(h, h->d_sum_partials, (int)nchunks, totals);
    if (e != cudaSuccess) return cuda_err(h, e, "sums finish kernel");
  }
  return FV_OK;
}

fv_status fv_conserved_totals(fv_batch* h, const void* q, const int64_t* off,
                              const int32_t* sizes, int64_t n, double* totals) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (!totals) return set_err(h, FV_ERR_INVALID_ARG, "null totals");
  return sums_impl(h, q, off, sizes, n, totals, nullptr);
}

fv_status fv_patch_sums(fv_batch* h, const void* q, const int64_t* off, const int32_t* sizes,
                        int64_t n, double* per_patch, double* totals) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (!per_patch) return set_err(h, FV_ERR_INVALID_ARG, "null per_patch");
  if (reinterpret_cast<uintptr_t>(per_patch) % 8 != 0)
    return set_err(h, FV_ERR_ALIGNMENT, "per_patch not 8-byte aligned");
  return sums_impl(h, q, off, sizes, n, totals, per_patch);
}

static fv_status time_step_impl(fv_batch* h, const void* in, void* out, const int64_t* off,
                                const int32_t* sizes, const int32_t* nbr, int64_t n, double dx,
                                double cfl, double* lambda_patch, const float* corr,
                                const void* prim_in, void* prim_out);

fv_status fv_time_step(fv_batch* h, const void* in, void* out, const int64_t* off,
                       const int32_t* sizes, const int32_t* nbr, int64_t n, double dx,
                       double cfl, double* lambda_patch) {
  return time_step_impl(h, in, out, off, sizes, nbr, n, dx, cfl, lambda_patch, nullptr, nullptr,
                        nullptr);
}

fv_status fv_prim_stride(const fv_batch* h, int64_t* elems_per_patch) {
  if (!h || !elems_per_patch) return FV_ERR_INVALID_ARG;
  *elems_per_patch = fv::prim_stride_elems(h->d, h->prec, h->max_patch_size);
  return FV_OK;
}

fv_status fv_time_step_prim(fv_batch* h, const void* in, void* out, const void* prim_in,
                            void* prim_out, const int64_t* off, const int32_t* sizes,
                            const int32_t* nbr, int64_t n, double dx, double cfl,
                            double* lambda_patch) {
  return time_step_impl(h, in, out, off, sizes, nbr, n, dx, cfl, lambda_patch, nullptr, prim_in,
                        prim_out);
}

fv_status fv_time_step_corrected(fv_batch* h, const void* in, void* out, const int64_t* off,
                                 const int32_t* sizes, const int32_t* nbr, int64_t n, double dx,
                                 double cfl, const float* corr) {
  if (!h) return FV_ERR_INVALID_ARG;
  if (!corr) return set_err(h, FV_ERR_INVALID_ARG, "null corrections");
  if (h->d != 2) return set_err(h, FV_ERR_UNSUPPORTED, "corrections are 2D");
  return time_step_impl(h, in, out, off, sizes, nbr, n, dx, cfl, nullptr, corr, nullptr, nullptr);
}

static fv_status time_step_impl(fv_batch* h, const void* in, void* out, const int64_t* off,
                                const int32_t* sizes, const int32_t* nbr, int64_t n, double dx,
                                double cfl, double* lambda_patch, const float* corr,
                                const void* prim_in, void* prim_out) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (!(dx > 0.0) || !(cfl > 0.0)) return set_err(h, FV_ERR_INVALID_ARG, "dx, cfl must be > 0");
  fv_status st = check_meta(h, in, off, sizes, n);
  if (st != FV_OK) return st;
  if (n == 0) return FV_OK;
  if (!out || !nbr) return set_err(h, FV_ERR_INVALID_ARG, "null output or neighbour table");
  if (!aligned16(out)) return set_err(h, FV_ERR_ALIGNMENT, "output not 16-byte aligned");
  if (in == out) return set_err(h, FV_ERR_INVALID_ARG, "in and out alias");
  if ((prim_in && !aligned16(prim_in)) || (prim_out && !aligned16(prim_out)))
    return set_err(h, FV_ERR_ALIGNMENT, "primitive buffer not 16-byte aligned");
  if (prim_in && prim_in == prim_out)
    return set_err(h, FV_ERR_INVALID_ARG, "prim_in and prim_out alias");
  const int nxt = h->lam_cur ^ 1;
  cudaError_t e = fv::launch_zero_word(&h->d_lam[nxt], h->stream);
  if (e != cudaSuccess) return cuda_err(h, e, "time step: reset wave speed");
  fv::UpdateLaunch l;
  l.in = in;
  l.out = out;
  l.off = off;
  l.sizes = sizes;
  l.nbr = nbr;
  l.n = n;
  l.pmax = h->max_patch_size;
  l.gamma = h->gamma;
  l.dx = dx;
  l.cfl = cfl;
  l.lam_in = &h->d_lam[h->lam_cur];
  l.lam_next = &h->d_lam[nxt];
  l.dt_slot = h->d_dt;
  l.lam_patch = lambda_patch;
  l.status = h->d_status;
  l.fused = true;
  l.corr = corr;
  l.corr_stride = 2ll * 4 * (h->max_patch_size + 1) * h->max_patch_size;
  l.prim_in = prim_in;
  l.prim_out = prim_out;
  l.prim_stride = fv::prim_stride_elems(h->d, h->prec, h->max_patch_size);
  e = fv::launch_scheduled(h, l);
  if (e != cudaSuccess) return cuda_err(h, e, "time step kernel");
  h->lam_cur = nxt;
  return FV_OK;
}

fv_status fv_run_steps(fv_batch* h, void* q0, void* q1, const int64_t* off, const int32_t* sizes,
                       const int32_t* nbr, int64_t n, double dx, double cfl, int n_steps,
                       int use_graph) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (n_steps < 0) return set_err(h, FV_ERR_INVALID_ARG, "n_steps < 0");
  if (q0 == q1) return set_err(h, FV_ERR_INVALID_ARG, "q0 and q1 alias");
  // the primitive carry (FP64: it saves FP64-pipe work; FP32 kernels are
  // issue- and memory-bound and run faster without its extra bytes): two
  // buffers, grown (never shrunk) before any capture; graphs that refer to
  // the old buffers are dropped when they move
  const bool carry = h->prec == FV_FP64 && n_steps > 1;
  if (carry && n > 0) {
    const size_t es = h->prec == FV_FP64 ? 8 : 4;
    const int64_t need = n * fv::prim_stride_elems(h->d, h->prec, h->max_patch_size);
    if (need > h->prim_cap) {
      cudaError_t e = cudaStreamSynchronize(h->stream);
      graph_cache_clear(h);
      for (void*& pbuf : h->d_prim) {
        if (pbuf) cudaFree(pbuf);
        pbuf = nullptr;
      }
      h->prim_cap = 0;
      for (void*& pbuf : h->d_prim)
        if (e == cudaSuccess) e = cudaMalloc(&pbuf, es * (size_t)need);
      if (e != cudaSuccess) return cuda_err(h, e, "primitive buffers");
      h->prim_cap = need;
    }
  }
  auto enqueue = [&]() -> fv_status {
    fv_status s = fv_halo_fill(h, q0, off, sizes, nbr, n);
    if (s == FV_OK) s = fv_max_eigenvalue_reduce(h, q0, off, sizes, n, nullptr, nullptr, cfl, dx,
                                                 nullptr);
    void* a = q0;
    void* b = q1;
    for (int k = 0; k < n_steps && s == FV_OK; ++k) {
      // step k reads the primitives step k-1 left and hands on its own
      const void* pin = (!carry || k == 0) ? nullptr : h->d_prim[(k - 1) & 1];
      void* pout = (carry && k + 1 < n_steps) ? h->d_prim[k & 1] : nullptr;
      s = time_step_impl(h, a, b, off, sizes, nbr, n, dx, cfl, nullptr, nullptr, pin, pout);
      std::swap(a, b);
    }
    return s;
  };
  if (!use_graph) return enqueue();
  if (h->stream == nullptr)
    return set_err(h, FV_ERR_UNSUPPORTED, "graph capture needs a non-default stream");
  const int lam_start = h->lam_cur;
  const GraphKey key{q0, q1, off, sizes, nbr, n, dx, cfl, n_steps, lam_start};
  if (!h->graph_cache) h->graph_cache = new (std::nothrow) GraphCache();
  auto* gc = static_cast<GraphCache*>(h->graph_cache);
  if (!gc) return set_err(h, FV_ERR_CUDA, "out of host memory");
  auto it = gc->exec.find(key);
  if (it == gc->exec.end()) {
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(h, e, "begin capture");
    fv_status s = enqueue();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (s != FV_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      h->lam_cur = lam_start;
      return s != FV_OK ? s : cuda_err(h, e, "end capture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->lam_cur = lam_start;
      return cuda_err(h, e, "graph instantiate");
    }
    it = gc->exec.emplace(key, exec).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second, h->stream);
  if (e != cudaSuccess) return cuda_err(h, e, "graph launch");
  h->lam_cur = lam_start ^ (n_steps & 1);
  return FV_OK;
}

fv_status fv_read_dt(fv_batch* h, double* dt_host) {
  if (!h || !dt_host) return FV_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(dt_host, h->d_dt, sizeof(double), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? FV_OK : cuda_err(h, e, "read dt");
}

fv_status fv_get_dt_ptr(fv_batch* h, double** dt_device) {
  if (!h || !dt_device) return FV_ERR_INVALID_ARG;
  *dt_device = h->d_dt;
  return FV_OK;
}

fv_status fv_get_status(fv_batch* h) {
  if (!h) return FV_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_err(h, e, "stream synchronize");
  unsigned int bits = 0;
  e = cudaMemcpyAsync(&bits, h->d_status, sizeof(bits), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(bits), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_err(h, e, "status read");
  if (bits & fv::ST_BAD_PATCH) return set_err(h, FV_ERR_BAD_PATCH, "a patch had bad metadata");
  if (bits & fv::ST_NONPHYSICAL)
    return set_err(h, FV_ERR_NONPHYSICAL, "rho <= 0, p <= 0 or NaN met");
  if (bits & fv::ST_TIMEOUT) return set_err(h, FV_ERR_TIMEOUT, "a device wait gave up");
  return FV_OK;
}

const char* fv_last_error(const fv_batch* h) { return h ? h->last_error : "null handle"; }

fv_status fv_selftest_math(const double* x, double* out, int64_t n, int which) {
  if (n < 0 || (n > 0 && (!x || !out)) || (which != 0 && which != 1)) return FV_ERR_INVALID_ARG;
  if (n == 0) return FV_OK;
  cudaError_t e = fv::launch_selftest_math(x, out, n, which);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

}  // extern "C"
