// fv_halo.cu -- face halo fill of every patch from its neighbours (the
// engine's halo consistency step, Sec. 2 of arXiv 2302.09005).
//
// One warp per patch (four per CTA, grid stride over the warps); lane t
// copies halo cells t, t + 32, ... of the patch, ordered (face, layer,
// transverse cell) with x fastest, so a warp walks rows of contiguous cells on
// the y and z faces.  Cells whose size is a multiple of 16 bytes (2D) move as
// 16-byte words.
#include "fv_device.cuh"
#include "fv_internal.h"

namespace fv {

template <typename T>
struct HaloParams {
  T* q;
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ sizes;
  const int32_t* __restrict__ nbr;
  int64_t n;
  int halo;
  int pmax;
  unsigned int* status;
};

// The S unknowns of one cell (16-byte aligned when S sizeof(T) is a multiple
// of 16, as patch offsets are multiples of 16 bytes).
template <typename T, int S>
__device__ __forceinline__ void copy_cell(const T* src, T (&v)[S]) {
  if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int u = 0; u < (int)(S * sizeof(T) / 16); ++u) {
      const uint4 w = reinterpret_cast<const uint4*>(src)[u];
      memcpy(&v[u * (16 / sizeof(T))], &w, 16);
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = src[u];
  }
}
template <typename T, int S>
__device__ __forceinline__ void store_cell(T* dst, const T (&v)[S]) {
  if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int u = 0; u < (int)(S * sizeof(T) / 16); ++u) {
      uint4 w;
      memcpy(&w, &v[u * (16 / sizeof(T))], 16);
      reinterpret_cast<uint4*>(dst)[u] = w;
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) dst[u] = v[u];
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(FV_NT) halo_kernel(HaloParams<T> a) {
  constexpr int S = D + 2;
  constexpr int VEC = 16 / sizeof(T);
  constexpr int NW = FV_NT / 32;
  const int h = a.halo;
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * NW + (threadIdx.x >> 5); i < a.n;
       i += (int64_t)gridDim.x * NW) {
    const int p = a.sizes[i];
    const int64_t off = a.off[i];
    if (!(p >= 1 && p <= a.pmax && p >= h && off >= 0 && (off % VEC) == 0)) {
      if (lane == 0) atomicOr(a.status, ST_BAD_PATCH);
      continue;
    }
    const int ne = p + 2 * h;
    const int ptr = D == 1 ? 1 : D == 2 ? p : p * p;
    const int per_face = h * ptr;
    const int total = 2 * D * per_face;
    T* Q = a.q + off;
    for (int t = lane; t < total; t += 32) {
      const int f = t / per_face;
      const int rem = t - f * per_face;
      const int l = rem / ptr;  // layer, 0 next to the interior
      int r = rem - l * ptr;
      const int k = f >> 1, side = f & 1;
      int c[3] = {0, 0, 0};
#pragma unroll
      for (int m = 0; m < D; ++m)
        if (m != k) {
          c[m] = h + r % p;
          r /= p;
        }
      const int32_t nb = a.nbr[i * 2 * D + f];
      const T* src_patch = Q;
      int src_k;
      const int dst_k = side == 0 ? h - 1 - l : h + p + l;
      if (nb >= 0) {
        bool ok = nb < a.n;
        int64_t noff = 0;
        if (ok) {
          noff = a.off[nb];
          ok = a.sizes[nb] == p && noff >= 0 && (noff % VEC) == 0;
        }
        if (!ok) {
          atomicOr(a.status, ST_BAD_PATCH);
          continue;
        }
        src_patch = a.q + noff;
        src_k = side == 0 ? dst_k + p : dst_k - p;
      } else if (nb == -1) {
        src_k = side == 0 ? h : h + p - 1;
      } else if (nb == -2) {
        src_k = side == 0 ? h + l : h + p - 1 - l;
      } else {
        atomicOr(a.status, ST_BAD_PATCH);
        continue;
      }
      int cd[3] = {c[0], c[1], c[2]}, cs[3] = {c[0], c[1], c[2]};
      cd[k] = dst_k;
      cs[k] = src_k;
      int64_t id = cd[D - 1], is = cs[D - 1];
#pragma unroll
      for (int m = D - 2; m >= 0; --m) {
        id = id * ne + cd[m];
        is = is * ne + cs[m];
      }
      T* dst = Q + id * S;
      const T* src = src_patch + is * S;
      T v[S];
      copy_cell<T, S>(src, v);
      if (nb == -2) v[1 + k] = -v[1 + k];
      store_cell<T, S>(dst, v);
    }
  }
}

template <typename T, int D>
static cudaError_t launch_halo_t(const fv_batch* h, const HaloLaunch& l, int grid) {
  HaloParams<T> a;
  a.q = static_cast<T*>(l.q);
  a.off = l.off;
  a.sizes = l.sizes;
  a.nbr = l.nbr;
  a.n = l.n;
  a.halo = l.halo;
  a.pmax = h->max_patch_size;
  a.status = l.status;
  halo_kernel<T, D><<<grid, FV_NT, 0, h->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_halo(const fv_batch* h, const HaloLaunch& l, int grid) {
  if (h->prec == FV_FP64) {
    if (h->d == 1) return launch_halo_t<double, 1>(h, l, grid);
    if (h->d == 2) return launch_halo_t<double, 2>(h, l, grid);
    return launch_halo_t<double, 3>(h, l, grid);
  }
  if (h->d == 1) return launch_halo_t<float, 1>(h, l, grid);
  if (h->d == 2) return launch_halo_t<float, 2>(h, l, grid);
  return launch_halo_t<float, 3>(h, l, grid);
}

}  // namespace fv
