// fv_host.cu -- the batched update with the patches in host memory: the
// paper's offload pattern (the engine keeps the patches and their halos on
// the host and ships a batch to the GPU for every update, Sec. 3) as a
// pipeline.  The batch is cut into chunks of consecutive patches; chunk c is
// copied host -> device on one copy stream, updated on the handle's stream
// and copied device -> host on a second copy stream, so the copies of
// neighbouring chunks overlap each other and the update of the chunk between
// them.  Three device staging slots (chunk buffer, metadata) are
// reused in turn, so the upload of a chunk need not wait for the download of
// the chunk before it (full-duplex link); events order the reuse.  Updated in
// place on the host (host_in == host_out), a chunk of equally spaced patches
// of one size travels as spans, 2D copies over the chunk's patches (the
// patch stride as pitch) of what the update reads and of what it writes; the
// halo cells are on the host already.  In, one span per patch from its first
// to its last face-halo cell (327 of the 343 cells of a 5^3 box).  Back, 1D
// and 2D patches one span from the first to the last interior cell; 3D
// patches one span per interior z-plane, cells (1, 1, z) .. (p, p, z) (x
// fastest): 165 cells of a 5^3 box instead of 229.  (Copy rates measured on
// this path fall with the row width of a 2D copy: 1,320-byte rows moved at
// 153 GB/s host to device against 210 GB/s for 9 KB rows, so the upload stays
// one span; the narrower rows of the download shorten the time the two
// directions share the link.)
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "fv_internal.h"

constexpr int kHostSlots = 3;

struct fv_host_stage {
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_h2d[kHostSlots] = {};   // slot's input (and metadata) on the device
  cudaEvent_t ev_comp[kHostSlots] = {};  // slot's update done
  cudaEvent_t ev_free[kHostSlots] = {};  // slot's output back on the host
  bool used[kHostSlots] = {};
  void* d_in[kHostSlots] = {};  // chunk input, updated in place
  size_t bytes = 0;  // capacity of each buffer
  int64_t* d_off[kHostSlots] = {};
  int32_t* d_sz[kHostSlots] = {};
  int64_t* h_off[kHostSlots] = {};  // pinned: rebased offsets of the chunk
  int32_t* h_sz[kHostSlots] = {};
  int64_t meta_cap = 0;
  size_t max_pitch = 0;  // largest pitch of a 2D copy (cudaDevAttrMaxPitch)
};

namespace fv {

void host_stage_free(fv_batch* h) {
  auto* st = static_cast<fv_host_stage*>(h->host_stage);
  if (!st) return;
  if (st->h2d) cudaStreamSynchronize(st->h2d);
  if (st->d2h) cudaStreamSynchronize(st->d2h);
  for (int k = 0; k < kHostSlots; ++k) {
    cudaFree(st->d_in[k]);
    cudaFree(st->d_off[k]);
    cudaFree(st->d_sz[k]);
    cudaFreeHost(st->h_off[k]);
    cudaFreeHost(st->h_sz[k]);
    if (st->ev_h2d[k]) cudaEventDestroy(st->ev_h2d[k]);
    if (st->ev_comp[k]) cudaEventDestroy(st->ev_comp[k]);
    if (st->ev_free[k]) cudaEventDestroy(st->ev_free[k]);
  }
  if (st->h2d) cudaStreamDestroy(st->h2d);
  if (st->d2h) cudaStreamDestroy(st->d2h);
  delete st;
  h->host_stage = nullptr;
}

}  // namespace fv

namespace {

fv_status herr(fv_batch* h, fv_status st, const char* msg) {
  snprintf(h->last_error, sizeof(h->last_error), "%s", msg);
  return st;
}

// Grows the staging of a handle to chunks of `bytes` bytes and `npatch`
// patches (never shrinks).
cudaError_t stage_reserve(fv_batch* h, size_t bytes, int64_t npatch) {
  auto* st = static_cast<fv_host_stage*>(h->host_stage);
  cudaError_t e = cudaSuccess;
  if (!st) {
    st = new (std::nothrow) fv_host_stage();
    if (!st) return cudaErrorMemoryAllocation;
    h->host_stage = st;
    int mp = 0;
    e = cudaDeviceGetAttribute(&mp, cudaDevAttrMaxPitch, h->device);
    st->max_pitch = mp > 0 ? (size_t)mp : 0;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st->d2h, cudaStreamNonBlocking);
    for (int k = 0; k < kHostSlots && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&st->ev_h2d[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_comp[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev_free[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
  }
  if (bytes > st->bytes) {
    for (int k = 0; k < kHostSlots; ++k) {
      if (st->used[k]) cudaEventSynchronize(st->ev_free[k]);
      cudaFree(st->d_in[k]);
      st->d_in[k] = nullptr;
    }
    st->bytes = 0;
    for (int k = 0; k < kHostSlots && e == cudaSuccess; ++k) {
      e = cudaMalloc(&st->d_in[k], bytes);
    }
    if (e != cudaSuccess) return e;
    st->bytes = bytes;
  }
  if (npatch > st->meta_cap) {
    for (int k = 0; k < kHostSlots; ++k) {
      if (st->used[k]) cudaEventSynchronize(st->ev_free[k]);
      cudaFree(st->d_off[k]);
      cudaFree(st->d_sz[k]);
      cudaFreeHost(st->h_off[k]);
      cudaFreeHost(st->h_sz[k]);
      st->d_off[k] = nullptr;
      st->d_sz[k] = nullptr;
      st->h_off[k] = nullptr;
      st->h_sz[k] = nullptr;
    }
    st->meta_cap = 0;
    for (int k = 0; k < kHostSlots && e == cudaSuccess; ++k) {
      e = cudaMalloc(&st->d_off[k], sizeof(int64_t) * (size_t)npatch);
      if (e == cudaSuccess) e = cudaMalloc(&st->d_sz[k], sizeof(int32_t) * (size_t)npatch);
      if (e == cudaSuccess) e = cudaMallocHost(&st->h_off[k], sizeof(int64_t) * (size_t)npatch);
      if (e == cudaSuccess) e = cudaMallocHost(&st->h_sz[k], sizeof(int32_t) * (size_t)npatch);
    }
    if (e != cudaSuccess) return e;
    st->meta_cap = npatch;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

fv_status fv_patch_update_host(fv_batch* h, const void* host_in, void* host_out,
                               const int64_t* off, const int32_t* sizes, int64_t n, double dx,
                               double dt, int64_t chunk_patches) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (n < 0) return herr(h, FV_ERR_INVALID_ARG, "n_patches < 0");
  if (n == 0) return FV_OK;
  if (!host_in || !host_out || !off || !sizes)
    return herr(h, FV_ERR_INVALID_ARG, "null pointer");
  if (!(dx > 0.0) || dt != dt) return herr(h, FV_ERR_INVALID_ARG, "dx must be > 0, dt not NaN");
  const size_t es = h->prec == FV_FP64 ? 8 : 4;
  const int vec = (int)(16 / es);
  const int d = h->d, s = h->s;
  // patch extents; offsets must ascend (consecutive patches form a chunk)
  auto len = [&](int64_t i) -> int64_t {
    int64_t e = 1;
    for (int m = 0; m < d; ++m) e *= sizes[i] + 2;
    return e * s;
  };
  for (int64_t i = 0; i < n; ++i) {
    if (sizes[i] < 1 || sizes[i] > h->max_patch_size)
      return herr(h, FV_ERR_BAD_PATCH, "patch size outside 1..max_patch_size");
    if (off[i] < 0 || off[i] % vec) return herr(h, FV_ERR_ALIGNMENT, "patch offset");
    if (i > 0 && off[i] < off[i - 1] + len(i - 1))
      return herr(h, FV_ERR_INVALID_ARG, "patch offsets must ascend without overlap");
  }
  const bool inplace = host_in == host_out;
  int64_t chunk = chunk_patches;
  if (chunk <= 0) {  // about 256 MB per chunk
    const int64_t per = len(0) * (int64_t)es;
    chunk = (256ll << 20) / (per > 0 ? per : 1);
    if (chunk < 1) chunk = 1;
  }
  if (chunk > n) chunk = n;
  const int64_t nchunks = (n + chunk - 1) / chunk;
  // the largest chunk in bytes (16-byte rounded)
  size_t maxb = 0;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int64_t p0 = c * chunk, p1 = p0 + chunk < n ? p0 + chunk : n;
    const size_t b = (size_t)(off[p1 - 1] + len(p1 - 1) - off[p0]) * es;
    maxb = b > maxb ? b : maxb;
  }
  maxb = (maxb + 15) & ~(size_t)15;
  cudaError_t e = stage_reserve(h, maxb, chunk);
  if (e != cudaSuccess) return herr(h, FV_ERR_CUDA, cudaGetErrorString(e));
  auto* st = static_cast<fv_host_stage*>(h->host_stage);
  // the spans of a patch, [lo, hi) in elements of its box: in (what the
  // update reads), back (what it writes)
  struct Span {
    int64_t lo, hi;
  };
  std::vector<Span> in_sp, back_sp;
  in_sp.reserve(1);
  back_sp.reserve((size_t)h->max_patch_size);
  // the chunks start once the work already on the handle's stream is done
  e = cudaEventRecord(st->ev_comp[0], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st->h2d, st->ev_comp[0], 0);
  for (int64_t c = 0; c < nchunks && e == cudaSuccess; ++c) {
    const int k = (int)(c % kHostSlots);
    const int64_t p0 = c * chunk, p1 = p0 + chunk < n ? p0 + chunk : n;
    const int64_t nc = p1 - p0;
    const int64_t base = off[p0];
    const size_t bytes = (size_t)(off[p1 - 1] + len(p1 - 1) - base) * es;
    // the slot's pinned metadata is free once its previous upload is done
    if (st->used[k]) e = cudaEventSynchronize(st->ev_h2d[k]);
    if (e != cudaSuccess) break;
    for (int64_t i = 0; i < nc; ++i) {
      st->h_off[k][i] = off[p0 + i] - base;
      st->h_sz[k][i] = sizes[p0 + i];
    }
    // in place, a chunk of equally spaced patches of one size moves spans
    bool span = inplace;
    const int64_t pitch = nc > 1 ? off[p0 + 1] - off[p0] : len(p0);
    for (int64_t i = p0 + 1; i < p1 && span; ++i)
      span = sizes[i] == sizes[p0] && off[i] - off[i - 1] == pitch;
    // a 2D copy takes pitches up to the device's limit; patches spaced wider
    // apart go as one 1D copy of the chunk
    if (span && (size_t)pitch * es > st->max_pitch) span = false;
    in_sp.clear();
    back_sp.clear();
    if (span) {
      const int64_t p = sizes[p0], ne = p + 2;
      // first face-halo cell (1, .., 1, 0) to past the last (p, .., p, p + 1)
      int64_t sum = 0, top = 1;  // sum_m ne^m (the cell (1, .., 1)); ne^(d-1)
      for (int m = 0; m < d; ++m) {
        sum += top;
        if (m + 1 < d) top *= ne;
      }
      in_sp.push_back({s * (sum - top), s * (p * (sum - top) + (p + 1) * top + 1)});
      if (d == 3) {  // each interior z-plane from (1, 1, z) to past (p, p, z)
        for (int64_t z = 1; z <= p; ++z)
          back_sp.push_back({s * (ne * ne * z + ne + 1), s * (ne * ne * z + ne * p + p + 1)});
      } else {  // first interior cell to past the last
        back_sp.push_back({s * sum, s * (p * sum + 1)});
      }
    }
    // host -> device, once the slot's previous output has left
    if (st->used[k]) e = cudaStreamWaitEvent(st->h2d, st->ev_free[k], 0);
    if (span) {
      for (size_t j = 0; j < in_sp.size() && e == cudaSuccess; ++j)
        e = cudaMemcpy2DAsync(static_cast<char*>(st->d_in[k]) + in_sp[j].lo * es,
                              (size_t)pitch * es,
                              static_cast<const char*>(host_in) + (base + in_sp[j].lo) * es,
                              (size_t)pitch * es, (size_t)(in_sp[j].hi - in_sp[j].lo) * es,
                              (size_t)nc, cudaMemcpyHostToDevice, st->h2d);
    } else if (e == cudaSuccess) {
      e = cudaMemcpyAsync(st->d_in[k], static_cast<const char*>(host_in) + base * es, bytes,
                          cudaMemcpyHostToDevice, st->h2d);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(st->d_off[k], st->h_off[k], sizeof(int64_t) * nc,
                          cudaMemcpyHostToDevice, st->h2d);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(st->d_sz[k], st->h_sz[k], sizeof(int32_t) * nc, cudaMemcpyHostToDevice,
                          st->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_h2d[k], st->h2d);
    // update in place: in update mode a CTA reads only its own patch box (the
    // bulk copy into shared memory, before any write) and writes only that
    // patch's interior cells, so the chunk buffer can be its own output; the
    // halo cells travel back unchanged.  After a span upload the cells outside
    // the spans (edges and corners, halo cells of the z-halo planes) hold
    // stale values: the update uses only interior and face-halo cells, and
    // every cell copied back was copied in.
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, st->ev_h2d[k], 0);
    if (e == cudaSuccess) {
      fv::UpdateLaunch l;
      l.in = st->d_in[k];
      l.out = st->d_in[k];
      l.off = st->d_off[k];
      l.sizes = st->d_sz[k];
      l.n = nc;
      l.n_elems = (int64_t)(bytes / es);
      l.pmax = h->max_patch_size;
      l.gamma = h->gamma;
      l.dx = dx;
      l.dt = dt;
      l.dt_dev = h->d_dt;
      l.status = h->d_status;
      l.fused = false;
      e = fv::launch_scheduled(h, l);
    }
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_comp[k], h->stream);
    // device -> host: the whole chunk, or the interior spans
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st->d2h, st->ev_comp[k], 0);
    if (span) {
      for (size_t j = 0; j < back_sp.size() && e == cudaSuccess; ++j)
        e = cudaMemcpy2DAsync(static_cast<char*>(host_out) + (base + back_sp[j].lo) * es,
                              (size_t)pitch * es,
                              static_cast<const char*>(st->d_in[k]) + back_sp[j].lo * es,
                              (size_t)pitch * es, (size_t)(back_sp[j].hi - back_sp[j].lo) * es,
                              (size_t)nc, cudaMemcpyDeviceToHost, st->d2h);
    } else if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(host_out) + base * es, st->d_in[k], bytes,
                          cudaMemcpyDeviceToHost, st->d2h);
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_free[k], st->d2h);
    st->used[k] = true;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->d2h);
  if (e != cudaSuccess) return herr(h, FV_ERR_CUDA, cudaGetErrorString(e));
  return FV_OK;
}

}  // extern "C"
