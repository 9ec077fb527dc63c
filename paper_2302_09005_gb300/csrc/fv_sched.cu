// fv_sched.cu -- scheduling of the patch kernels over a batch of uneven
// patch sizes (the batched kernel of Sec. 3 with N patches of any size per
// launch):
//   FV_SCHED_STRIDE   one persistent launch, CTA b takes patches b, b+G, ...
//                     in index order; shared memory sized for the largest p;
//   FV_SCHED_LPT      one persistent launch over the patches sorted by size,
//                     largest first (longest-processing-time-first list
//                     scheduling: the big patches start early, the small ones
//                     fill the tail);
//   FV_SCHED_CLASSES  one launch per patch size, each with the shared memory,
//                     pipeline depth and occupancy of its own size;
//   FV_SCHED_QUEUE    one persistent launch whose CTAs pop the patches of the
//                     size-sorted order (largest first) from a work queue, a
//                     device counter zeroed by a one-thread kernel before
//                     the launch (a kernel node in a captured graph): dynamic list
//                     scheduling, a CTA that finishes early takes the next one.
// fv_batch_plan sorts the patches by size (a stable counting sort);
// fv_batch_autotune times the three on the caller's batch and keeps the
// fastest.
#include <stdio.h>

#include <vector>

#include "fv_device.cuh"
#include "fv_internal.h"

namespace fv {

void plan_free(fv_batch* h) {
  if (h->d_order) cudaFree(h->d_order);
  h->d_order = nullptr;
  h->plan_cap = 0;
  h->plan_n = -1;
  h->plan_sizes = nullptr;
  h->ncls = 0;
}

static int stages_for(const fv_batch* h, int p) {
  return update_smem_bytes(h->d, h->prec, p, 2) <= (size_t)h->smem_optin ? 2 : 1;
}

static int grid_for(const fv_batch* h, int64_t count, int bps) {
  int64_t g = (int64_t)h->num_sms * (bps > 0 ? bps : 1);
  if (g > count) g = count;
  if (g > FV_MAX_RED_BLOCKS) g = FV_MAX_RED_BLOCKS;
  return (int)(g < 1 ? 1 : g);
}

// A launch of patches of one size: the FP32 kernel built for that size (3D
// p = 3 .. 7: the plane sweep; 2D p = 3 .. 6: a lane per row) where it
// applies.
static cudaError_t launch_one_size(fv_batch* h, const UpdateLaunch& l, int64_t count,
                                   bool* done) {
  *done = false;
  const bool two = rows2d_eligible(h, l);
  if (!two && !march3d_eligible(h, l)) return cudaSuccess;
  const int f = step_mode(l);
  int& bps = h->occ_one[l.uniform_p & 7][f];  // p = 3 .. 7 (2D: 3 .. 6)
  if (bps == 0) {
    cudaError_t e = two ? rows2d_occupancy(l.uniform_p, f, &bps) : march3d_occupancy(l.uniform_p, f, &bps);
    if (e != cudaSuccess) return e;
  }
  *done = true;
  ++h->pairs_launches;
  // a CTA takes several patches at a time
  const int per = two ? rows2d_patches_per_cta() : march3d_patches_per_cta();
  const int grid = grid_for(h, (count + per - 1) / per, bps);
  return two ? launch_rows2d(h, l, grid) : launch_march3d(h, l, grid);
}

cudaError_t launch_scheduled(fv_batch* h, UpdateLaunch l) {
  const bool plan_ok = h->d_order != nullptr && h->plan_n == l.n && h->plan_sizes == l.sizes;
  const int f = step_mode(l);
  if (h->sched == FV_SCHED_CLASSES && plan_ok) {
    for (int c = 0; c < h->ncls; ++c) {
      const int64_t cnt = h->cls_end[c] - h->cls_begin[c];
      if (cnt <= 0 || (h->cls_only >= 0 && c != h->cls_only)) continue;
      UpdateLaunch lc = l;
      lc.order = h->d_order;
      lc.i_begin = h->cls_begin[c];
      lc.i_end = h->cls_end[c];
      lc.pmax = h->cls_p[c];
      if (h->cls_real[c]) {
        lc.uniform_p = lc.pmax;
        bool done = false;
        cudaError_t e = launch_one_size(h, lc, cnt, &done);
        if (e != cudaSuccess) return e;
        if (done) continue;
      }
      lc.nstage = stages_for(h, lc.pmax);
      const int pi = lc.pmax < 64 ? lc.pmax : 63;
      lc.nt = h->cls_nt[pi] > 0 ? h->cls_nt[pi] : default_nt(h->d, lc.pmax);
      int& bps = h->occ_cache[f][pi][nt_index(lc.nt)];
      if (bps == 0) {
        cudaError_t e = step_occupancy(h, f, lc.pmax, lc.nstage, lc.nt, &bps);
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = launch_update(h, lc, grid_for(h, cnt, bps));
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (plan_ok && h->ncls == 1 && h->cls_real[0]) {  // a planned batch of one size
    UpdateLaunch lu = l;
    lu.uniform_p = h->cls_p[0];
    lu.pmax = h->cls_p[0];
    bool done = false;
    cudaError_t e = launch_one_size(h, lu, l.n, &done);
    if (e != cudaSuccess || done) return e;
  }
  l.nt = default_nt(h->d, h->max_patch_size);
  int& bps = h->blocks_per_sm[f];
  if (bps == 0) {
    cudaError_t e = step_occupancy(h, f, h->max_patch_size, h->nstage, l.nt, &bps);
    if (e != cudaSuccess) return e;
  }
  if ((h->sched == FV_SCHED_LPT || h->sched == FV_SCHED_QUEUE) && plan_ok) {
    l.order = h->d_order;
    l.i_begin = 0;
    l.i_end = l.n;
    if (h->sched == FV_SCHED_QUEUE) {
      l.queue = h->d_queue;
      cudaError_t e = launch_zero_word(h->d_queue, h->stream);
      if (e != cudaSuccess) return e;
    }
  }
  return launch_update(h, l, grid_for(h, l.n, bps));
}

}  // namespace fv

namespace {
fv_status sched_err(fv_batch* h, fv_status st, const char* msg) {
  snprintf(h->last_error, sizeof(h->last_error), "%s", msg);
  return st;
}
}  // namespace

extern "C" {

fv_status fv_batch_plan(fv_batch* h, const int32_t* sizes, int64_t n) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (n < 0 || (n > 0 && !sizes)) return sched_err(h, FV_ERR_INVALID_ARG, "bad sizes / n");
  if (n > 0x7FFFFFFFll) return sched_err(h, FV_ERR_UNSUPPORTED, "more than 2^31-1 patches");
  const int pmax = h->max_patch_size;
  if (pmax + 2 > 80) return sched_err(h, FV_ERR_UNSUPPORTED, "max_patch_size too large to plan");
  cudaError_t e = cudaSuccess;
  if (n > h->plan_cap) {
    if (h->d_order) cudaFree(h->d_order);
    h->d_order = nullptr;
    h->plan_cap = 0;
    e = cudaMalloc(&h->d_order, sizeof(int32_t) * (size_t)n);
    if (e != cudaSuccess) return sched_err(h, FV_ERR_CUDA, "plan: out of device memory");
    h->plan_cap = n;
  }
  // the sizes to the host, a stable counting sort there (patches of a class
  // keep their index order, so a class launch walks its patches in memory
  // order, with the neighbours' halo cells close in L2), the order back
  std::vector<int32_t> hs((size_t)n), order((size_t)n);
  if (n > 0)
    e = cudaMemcpyAsync(hs.data(), sizes, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return sched_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
  // bucket of a patch size: 1..pmax, or pmax+1 for sizes the kernels reject
  auto bucket = [&](int32_t p) { return (p >= 1 && p <= pmax) ? p : pmax + 1; };
  int64_t count[80] = {0}, start[80] = {0};
  for (int64_t i = 0; i < n; ++i) ++count[bucket(hs[(size_t)i])];
  // positions: largest size first, rejected sizes last
  int64_t pos = 0;
  h->ncls = 0;
  for (int p = pmax; p >= 1; --p) {
    start[p] = pos;
    if (count[p] > 0) {
      h->cls_p[h->ncls] = p;
      h->cls_real[h->ncls] = 1;
      h->cls_begin[h->ncls] = pos;
      h->cls_end[h->ncls] = pos + count[p];
      ++h->ncls;
    }
    pos += count[p];
  }
  start[pmax + 1] = pos;
  if (count[pmax + 1] > 0) {  // rejected sizes: the kernels flag and skip them
    h->cls_p[h->ncls] = pmax;
    h->cls_real[h->ncls] = 0;
    h->cls_begin[h->ncls] = pos;
    h->cls_end[h->ncls] = pos + count[pmax + 1];
    ++h->ncls;
  }
  for (int64_t i = 0; i < n; ++i) order[(size_t)start[bucket(hs[(size_t)i])]++] = (int32_t)i;
  if (n > 0)
    e = cudaMemcpyAsync(h->d_order, order.data(), sizeof(int32_t) * (size_t)n,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // `order` lives on this stack
  if (e != cudaSuccess) return sched_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
  h->plan_n = n;
  h->plan_sizes = sizes;
  return FV_OK;
}

fv_status fv_batch_set_schedule(fv_batch* h, fv_schedule s) {
  if (!h) return FV_ERR_INVALID_ARG;
  if (s != FV_SCHED_STRIDE && s != FV_SCHED_LPT && s != FV_SCHED_CLASSES && s != FV_SCHED_QUEUE)
    return FV_ERR_INVALID_ARG;
  h->sched = (int)s;
  return FV_OK;
}

fv_status fv_batch_set_wait_limit(fv_batch* h, long long cycles) {
  if (!h) return FV_ERR_INVALID_ARG;
  if (cycles > FV_WAIT_LIMIT)
    return sched_err(h, FV_ERR_INVALID_ARG, "wait limit above the default (2e9 cycles)");
  h->wait_limit = cycles > 0 ? cycles : FV_WAIT_LIMIT;
  return FV_OK;
}

fv_status fv_batch_set_class_threads(fv_batch* h, int p, int threads) {
  if (!h) return FV_ERR_INVALID_ARG;
  if (p < 1 || p > h->max_patch_size || p >= 64)
    return sched_err(h, FV_ERR_INVALID_ARG, "patch size outside 1..max_patch_size");
  if (threads == 0) threads = fv::default_nt(h->d, p);
  if (!fv::valid_nt(threads)) return sched_err(h, FV_ERR_INVALID_ARG, "threads: 32, 64, 128, 256");
  if (h->d == 1 && threads != 128) return sched_err(h, FV_ERR_UNSUPPORTED, "d = 1: 128 threads");
  h->cls_nt[p] = threads;
  return FV_OK;
}

fv_status fv_batch_class_threads(const fv_batch* h, int p, int* threads) {
  if (!h || !threads || p < 1 || p >= 64) return FV_ERR_INVALID_ARG;
  *threads = h->cls_nt[p] > 0 ? h->cls_nt[p] : fv::default_nt(h->d, p);
  return FV_OK;
}

fv_status fv_batch_pairs_launches(const fv_batch* h, int64_t* launches) {
  if (!h || !launches) return FV_ERR_INVALID_ARG;
  *launches = h->pairs_launches;
  return FV_OK;
}

fv_status fv_batch_autotune(fv_batch* h, const void* in, void* scratch_out, const int64_t* off,
                            const int32_t* sizes, const int32_t* nbr, int64_t n, double dx,
                            double cfl, fv_schedule* chosen, double* ms_per_schedule) {
  if (!h) return FV_ERR_INVALID_ARG;
  if (n <= 0) return sched_err(h, FV_ERR_INVALID_ARG, "empty batch");
  if (!(dx > 0.0) || !(cfl > 0.0)) return sched_err(h, FV_ERR_INVALID_ARG, "dx, cfl > 0");
  if (h->plan_n != n || h->plan_sizes != sizes) {
    fv_status st = fv_batch_plan(h, sizes, n);
    if (st != FV_OK) return st;
  }
  // keep the caller's wave speed and time step: the trial steps overwrite them
  unsigned long long* backup = h->d_lam + 2;  // workspace slots 2, 3
  const int lam0 = h->lam_cur;
  cudaError_t e = cudaMemcpyAsync(backup, &h->d_lam[lam0], 8, cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(backup + 1, h->d_dt, 8, cudaMemcpyDeviceToDevice, h->stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return sched_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
  const int saved = h->sched;
  fv_status st = FV_OK;
  // average ms of three timed calls after one warm-up, under the current
  // schedule (and class restriction)
  auto time_calls = [&](double* avg) {
    float ms_total = 0.f;
    for (int rep = 0; rep < 4 && st == FV_OK; ++rep) {
      h->lam_cur = lam0;
      e = cudaMemcpyAsync(&h->d_lam[lam0], backup, 8, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      if (e != cudaSuccess) {
        st = sched_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
        break;
      }
      st = nbr ? fv_time_step(h, in, scratch_out, off, sizes, nbr, n, dx, cfl, nullptr)
               : fv_patch_update_batch(h, in, scratch_out, off, sizes, n, h->d, h->s, dx,
                                       cfl * dx);
      e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess && st == FV_OK) st = sched_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
      if (rep > 0) ms_total += ms;
    }
    *avg = ms_total / 3.0;
  };
  // 1. the CTA size of each size class (one-class launches)
  h->sched = FV_SCHED_CLASSES;
  for (int c = 0; c < h->ncls && st == FV_OK; ++c) {
    if (h->cls_real[c] && (fv::march3d_class(h, h->cls_p[c]) || fv::rows2d_class(h, h->cls_p[c])))
      continue;  // kernels with a fixed CTA size
    const int pi = h->cls_p[c] < 64 ? h->cls_p[c] : 63;
    const int keep = h->cls_nt[pi];
    double best_c = 1e300;
    int best_nt = keep;
    h->cls_only = c;
    for (int nt : {32, 64, 128, 256}) {
      if (h->d == 1 && nt != 128) continue;
      h->cls_nt[pi] = nt;
      double avg = 0;
      time_calls(&avg);
      if (st == FV_OK && avg < best_c) {
        best_c = avg;
        best_nt = nt;
      }
    }
    h->cls_nt[pi] = best_nt;
    h->cls_only = -1;
  }
  h->cls_only = -1;
  // 2. the schedule
  double best = 1e300;
  int best_s = saved;
  for (int s = 0; s < 3 && st == FV_OK; ++s) {
    h->sched = s;
    double avg = 0;
    time_calls(&avg);
    if (ms_per_schedule) ms_per_schedule[s] = avg;
    if (st == FV_OK && avg < best) {
      best = avg;
      best_s = s;
    }
  }
  h->sched = st == FV_OK ? best_s : saved;
  h->lam_cur = lam0;
  cudaMemcpyAsync(&h->d_lam[lam0], backup, 8, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->d_dt, backup + 1, 8, cudaMemcpyDeviceToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (chosen) *chosen = (fv_schedule)h->sched;
  return st;
}

}  // extern "C"
