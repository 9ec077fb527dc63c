// fv_halo.cu -- face halo fill of every patch from its neighbours (the
// engine's halo consistency step, Sec. 2 of arXiv 2302.09005).
//
// One warp per patch (four per CTA, grid stride over the warps); lane t
// copies halo cells t, t + 32, ... of the patch, ordered (face, layer,
// transverse cell) with x fastest, so a warp walks rows of contiguous cells on
// the y and z faces.  Cells whose size is a multiple of 16 bytes (2D) move as
// 16-byte words.  3D patches take halo_kernel_pipe (face sources resolved
// once per patch, the next patch's metadata loaded ahead, two cells per lane
// in flight).
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

// The S unknowns of one cell (16-byte aligned when S sizeof(T) is a multiple
// of 16, as patch offsets are multiples of 16 bytes), through the read-only
// path: the cells a halo fill reads are interior cells, which it never writes.
template <typename T, int S>
__device__ __forceinline__ void load_cell_ro(const T* src, T (&v)[S]) {
  if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int u = 0; u < (int)(S * sizeof(T) / 16); ++u) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(src) + u);
      memcpy(&v[u * (16 / sizeof(T))], &w, 16);
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = __ldg(src + u);
  }
}
// v[u] = -v[u] for u == neg (selects, so v stays in registers).
template <typename T, int S>
__device__ __forceinline__ void negate_comp(T (&v)[S], int neg) {
#pragma unroll
  for (int u = 0; u < S; ++u)
    if (u == neg) v[u] = -v[u];
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
#pragma unroll
      for (int m = 0; m < D; ++m)  // selects: a runtime index would put cd, cs in local memory
        if (m == k) {
          cd[m] = dst_k;
          cs[m] = src_k;
        }
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
      if (nb == -2) negate_comp<T, S>(v, 1 + k);
      store_cell<T, S>(dst, v);
    }
  }
}

// Where halo cell t of a patch comes from: returns the element offset of its
// source cell (-1 for a face whose source is invalid) and sets the cell's own
// element offset in the patch and the component a wall negates (-1: none).
template <int D>
__device__ __forceinline__ int64_t halo_src(int t, int p, int h, int per_face, int ptr, int ne,
                                            const int64_t (&soff)[2 * D],
                                            const int (&smode)[2 * D], int64_t& dst,
                                            int& neg) {
  constexpr int S = D + 2;
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
  // the face's source (selects over the 2D faces, not a runtime index)
  int64_t so = soff[0];
  int mode = smode[0];
#pragma unroll
  for (int g = 1; g < 2 * D; ++g)
    if (f == g) {
      so = soff[g];
      mode = smode[g];
    }
  const int dst_k = side == 0 ? h - 1 - l : h + p + l;
  int src_k;
  if (mode == 0) src_k = side == 0 ? dst_k + p : dst_k - p;  // the neighbour's interior
  else if (mode == 1) src_k = side == 0 ? h : h + p - 1;     // outflow: nearest interior
  else src_k = side == 0 ? h + l : h + p - 1 - l;            // wall: mirror image
  neg = mode == 2 ? 1 + k : -1;
  int cd[3] = {c[0], c[1], c[2]}, cs[3] = {c[0], c[1], c[2]};
#pragma unroll
  for (int m = 0; m < D; ++m)  // selects: a runtime index would put cd, cs in local memory
    if (m == k) {
      cd[m] = dst_k;
      cs[m] = src_k;
    }
  int64_t id = cd[D - 1], is = cs[D - 1];
#pragma unroll
  for (int m = D - 2; m >= 0; --m) {
    id = id * ne + cd[m];
    is = is * ne + cs[m];
  }
  dst = id * S;
  return mode == 3 ? -1 : so + is * S;
}

// 3D patches, where a warp makes several passes over a patch's halo cells:
// lanes 0 .. 5 resolve the sources of the patch's faces once (neighbour,
// outflow, wall) and share them by shuffles, the next patch's size, offset
// and neighbours are loaded while the current one is copied, and each lane
// keeps two cells in flight (both loads, through the read-only path, before
// both stores).  FP64 5^3 patches: 1.76 ms against 2.09 for 262,144 patches;
// on 5x5 patches (one pass) it measured slower, so 1D and 2D use halo_kernel.
template <typename T, int D>
__global__ void __launch_bounds__(FV_NT) halo_kernel_pipe(HaloParams<T> a) {
  constexpr int S = D + 2;
  constexpr int NF = 2 * D;
  constexpr int VEC = 16 / sizeof(T);
  constexpr int NW = FV_NT / 32;
  const int h = a.halo;
  const int lane = threadIdx.x & 31;
  const int64_t wstep = (int64_t)gridDim.x * NW;
  int64_t i = (int64_t)blockIdx.x * NW + (threadIdx.x >> 5);
  // a patch's size, offset and (lanes < 2D) neighbour across face `lane`,
  // loaded one patch ahead of its copy
  int pn = 0;
  int64_t offn = 0;
  int32_t nbn = 0;
  if (i < a.n) {
    pn = a.sizes[i];
    offn = a.off[i];
    if (lane < NF) nbn = a.nbr[i * NF + lane];
  }
  for (; i < a.n; i += wstep) {
    const int p = pn;
    const int64_t off = offn;
    const int32_t nb = nbn;
    if (i + wstep < a.n) {
      pn = a.sizes[i + wstep];
      offn = a.off[i + wstep];
      if (lane < NF) nbn = a.nbr[(i + wstep) * NF + lane];
    }
    if (!(p >= 1 && p <= a.pmax && p >= h && off >= 0 && (off % VEC) == 0)) {
      if (lane == 0) atomicOr(a.status, ST_BAD_PATCH);
      continue;
    }
    // lane f < 2D: face f's source, the element offset of the patch whose
    // cells fill it and how (0 neighbour, 1 outflow, 2 wall, 3 invalid)
    int64_t so = off;
    int mode = 3;
    if (lane < NF) {
      if (nb >= 0) {
        if (nb < a.n) {
          const int64_t noff = a.off[nb];
          if (a.sizes[nb] == p && noff >= 0 && (noff % VEC) == 0) {
            so = noff;
            mode = 0;
          }
        }
      } else if (nb == -1) {
        mode = 1;
      } else if (nb == -2) {
        mode = 2;
      }
      if (mode == 3) atomicOr(a.status, ST_BAD_PATCH);
    }
    int64_t soff[NF];
    int smode[NF];
#pragma unroll
    for (int g = 0; g < NF; ++g) {
      soff[g] = __shfl_sync(0xFFFFFFFFu, so, g);
      smode[g] = __shfl_sync(0xFFFFFFFFu, mode, g);
    }
    const int ne = p + 2 * h;
    const int ptr = D == 1 ? 1 : D == 2 ? p : p * p;
    const int per_face = h * ptr;
    const int total = NF * per_face;
    T* Q = a.q + off;
    // two cells per lane in flight: both loads (read-only: the kernel writes
    // halo cells only and reads interior cells only) before both stores
    for (int t = lane; t < total; t += 64) {
      int64_t d0 = 0, d1 = 0;
      int n0 = -1, n1 = -1;
      const int64_t s0 = halo_src<D>(t, p, h, per_face, ptr, ne, soff, smode, d0, n0);
      const int64_t s1 =
          t + 32 < total ? halo_src<D>(t + 32, p, h, per_face, ptr, ne, soff, smode, d1, n1) : -1;
      T v0[S], v1[S];
      if (s0 >= 0) load_cell_ro<T, S>(a.q + s0, v0);
      if (s1 >= 0) load_cell_ro<T, S>(a.q + s1, v1);
      if (s0 >= 0) {
        negate_comp<T, S>(v0, n0);
        store_cell<T, S>(Q + d0, v0);
      }
      if (s1 >= 0) {
        negate_comp<T, S>(v1, n1);
        store_cell<T, S>(Q + d1, v1);
      }
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
  if constexpr (D == 3)
    halo_kernel_pipe<T, D><<<grid, FV_NT, 0, h->stream>>>(a);
  else
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
