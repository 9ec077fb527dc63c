// fv_amr.cu -- face halos of patches on a 3:1 refined mesh (the paper's
// spacetree splits a cube into three parts along every axis, Sec. 2; each
// cube carries a patch and a halo layer the engine keeps consistent).
//
// A plan, built once on the host from every patch's level and tree-cell
// coordinates, lists for each face-halo cell the interior cells it is made
// of: one cell of a neighbour of the same level (a copy), the one cell of a
// coarser neighbour that contains it (constant prolongation), or the 3^d
// cells of finer neighbours it covers (restriction by averaging); cells
// beyond a non-periodic domain edge copy the own adjacent cell (outflow) or
// its mirror image (wall).  The device kernel then evaluates the plan: one
// thread per halo cell, sources summed in the plan's order (deterministic).
//
// Geometry: a level-l tree cell has edge 3^-l; its patch has p^d cells of
// edge 3^-l / p.  A cell's global index along an axis at level l is
// c p + a (c its tree cell, a its index in the patch); the level-(l-1) cell
// containing it has global index floor((c p + a) / 3), and the level-(l+1)
// cells inside it have global indices 3 (c p + a) + {0, 1, 2}.
#include <stdio.h>
#include <string.h>

#include <new>
#include <unordered_map>
#include <vector>

#include "fv_device.cuh"
#include "fv_internal.h"

struct fv_amr_plan {
  int d = 0, s = 0, p = 0;
  fv_precision prec = FV_FP64;
  int64_t ncell = 0;            // halo cells
  int64_t* d_dst = nullptr;     // element offset of each halo cell
  int64_t* d_start = nullptr;   // ncell + 1: sources of cell i at [start[i], start[i+1])
  int64_t* d_src = nullptr;     // element offsets of the source cells
  int32_t* d_neg = nullptr;     // unknown to negate (wall), or -1
};

namespace fv {

template <typename T>
__global__ void amr_halo_kernel(T* __restrict__ q, const int64_t* __restrict__ dst,
                                const int64_t* __restrict__ start,
                                const int64_t* __restrict__ src, const int32_t* __restrict__ neg,
                                int64_t ncell, int s) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = start[c], e = start[c + 1];
    const int ng = neg[c];
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
    for (int64_t j = b; j < e; ++j) {
      const T* v = q + src[j];
      for (int u = 0; u < s; ++u) acc[u] += v[u];
    }
    const int64_t cnt = e - b;
    T* o = q + dst[c];
    for (int u = 0; u < s; ++u) {
      T val = cnt == 1 ? acc[u] : acc[u] / (T)cnt;
      o[u] = (u == ng) ? -val : val;
    }
  }
}

}  // namespace fv

namespace {

fv_status amr_err(fv_batch* h, fv_status st, const char* msg) {
  if (h) snprintf(h->last_error, sizeof(h->last_error), "%s", msg);
  return st;
}

// Key of a tree cell: level and coordinates (each < 2^19).
uint64_t tree_key(int level, const int64_t* c, int d) {
  uint64_t k = (uint64_t)level;
  for (int m = 0; m < d; ++m) k = (k << 19) | (uint64_t)c[m];
  return k;
}

void plan_free(fv_amr_plan* pl) {
  if (!pl) return;
  cudaFree(pl->d_dst);
  cudaFree(pl->d_start);
  cudaFree(pl->d_src);
  cudaFree(pl->d_neg);
  delete pl;
}

}  // namespace

extern "C" {

fv_status fv_amr_plan_create(fv_batch* h, fv_amr_plan** out, int64_t n, const int32_t* level,
                             const int32_t* coord, const int64_t* off, int p, int boundary) {
  if (!h || !out) return FV_ERR_INVALID_ARG;
  *out = nullptr;
  h->last_error[0] = 0;
  const int d = h->d, s = h->s;
  if (n <= 0 || !level || !coord || !off) return amr_err(h, FV_ERR_INVALID_ARG, "empty mesh");
  if (p < 1 || p > h->max_patch_size) return amr_err(h, FV_ERR_INVALID_ARG, "patch size");
  if (boundary != 0 && boundary != -1 && boundary != -2)
    return amr_err(h, FV_ERR_INVALID_ARG, "boundary: 0 periodic, -1 outflow, -2 wall");
  const int vec = h->prec == FV_FP64 ? 2 : 4;
  std::unordered_map<uint64_t, int64_t> where;
  where.reserve((size_t)n * 2);
  int lmin = 1 << 30, lmax = -1;
  for (int64_t i = 0; i < n; ++i) {
    const int l = level[i];
    if (l < 0 || l > 11) return amr_err(h, FV_ERR_INVALID_ARG, "level outside 0..11");
    int64_t c[3] = {0, 0, 0};
    int64_t ncl = 1;
    for (int m = 0; m < l; ++m) ncl *= 3;
    for (int m = 0; m < d; ++m) {
      c[m] = coord[i * d + m];
      if (c[m] < 0 || c[m] >= ncl) return amr_err(h, FV_ERR_INVALID_ARG, "coordinate outside level");
    }
    if (off[i] < 0 || off[i] % vec) return amr_err(h, FV_ERR_ALIGNMENT, "patch offset");
    if (!where.emplace(tree_key(l, c, d), i).second)
      return amr_err(h, FV_ERR_INVALID_ARG, "two patches on one tree cell");
    lmin = l < lmin ? l : lmin;
    lmax = l > lmax ? l : lmax;
  }
  if (lmax > lmin && p < 3)
    return amr_err(h, FV_ERR_UNSUPPORTED, "refined meshes need p >= 3");
  const int ne = p + 2;
  auto elem = [&](int64_t j, const int64_t* a) -> int64_t {  // interior index a (0..p-1)
    int64_t idx = 0;
    for (int m = d - 1; m >= 0; --m) idx = idx * ne + (a[m] + 1);
    return off[j] + idx * s;
  };
  auto find = [&](int l, const int64_t* c) -> int64_t {
    auto it = where.find(tree_key(l, c, d));
    return it == where.end() ? -1 : it->second;
  };
  int64_t ptr = 1;
  for (int m = 1; m < d; ++m) ptr *= p;
  std::vector<int64_t> dst, start, src;
  std::vector<int32_t> neg;
  dst.reserve((size_t)(n * 2 * d * ptr));
  start.reserve((size_t)(n * 2 * d * ptr) + 1);
  start.push_back(0);
  for (int64_t i = 0; i < n; ++i) {
    const int l = level[i];
    int64_t ncl = 1;
    for (int m = 0; m < l; ++m) ncl *= 3;
    const int64_t dom = ncl * p;  // cells per axis at this level
    int64_t c[3] = {0, 0, 0};
    for (int m = 0; m < d; ++m) c[m] = coord[i * d + m];
    for (int k = 0; k < d; ++k) {
      for (int side = 0; side < 2; ++side) {
        int64_t cn[3] = {c[0], c[1], c[2]};
        cn[k] += side ? 1 : -1;
        const bool edge = cn[k] < 0 || cn[k] >= ncl;
        if (edge && boundary == 0) cn[k] = (cn[k] + ncl) % ncl;
        // which leaf covers the neighbouring tree cell
        int kind = 0;  // 0 edge, 1 same level, 2 coarser, 3 finer
        int64_t same = -1, coarse = -1;
        if (!edge || boundary == 0) {
          same = find(l, cn);
          if (same >= 0) {
            kind = 1;
          } else {
            int64_t cp[3] = {cn[0] / 3, cn[1] / 3, cn[2] / 3};
            coarse = l > 0 ? find(l - 1, cp) : -1;
            kind = coarse >= 0 ? 2 : 3;
          }
        }
        for (int64_t t = 0; t < ptr; ++t) {
          int64_t a[3] = {0, 0, 0};  // halo cell: local index, -1 or p along k
          int64_t r = t;
          for (int m = 0; m < d; ++m) {
            if (m == k) continue;
            a[m] = r % p;
            r /= p;
          }
          a[k] = side ? p : -1;
          dst.push_back(elem(i, a));
          int32_t ng = -1;
          if (kind == 0) {  // domain edge: own adjacent cell (wall: mirrored)
            int64_t b[3] = {a[0], a[1], a[2]};
            b[k] = side ? p - 1 : 0;
            src.push_back(elem(i, b));
            if (boundary == -2) ng = 1 + k;
          } else {
            int64_t g[3];  // global index of the halo cell at level l (wrapped)
            for (int m = 0; m < d; ++m) g[m] = ((c[m] * p + a[m]) % dom + dom) % dom;
            if (kind == 1) {
              int64_t b[3] = {a[0], a[1], a[2]};
              b[k] = side ? 0 : p - 1;
              src.push_back(elem(same, b));
            } else if (kind == 2) {  // the coarse cell containing it
              int64_t b[3] = {0, 0, 0};
              for (int m = 0; m < d; ++m) b[m] = g[m] / 3 - (cn[m] / 3) * p;
              for (int m = 0; m < d; ++m)
                if (b[m] < 0 || b[m] >= p)
                  return amr_err(h, FV_ERR_INVALID_ARG, "internal: coarse cell outside patch");
              src.push_back(elem(coarse, b));
            } else {  // the 3^d fine cells it covers
              int nsub = 1;
              for (int m = 0; m < d; ++m) nsub *= 3;
              for (int u = 0; u < nsub; ++u) {
                int64_t f[3] = {0, 0, 0}, fc[3] = {0, 0, 0}, b[3] = {0, 0, 0};
                int uu = u;
                for (int m = 0; m < d; ++m) {
                  f[m] = 3 * g[m] + uu % 3;
                  uu /= 3;
                  fc[m] = f[m] / p;
                  b[m] = f[m] - fc[m] * p;
                }
                const int64_t j = find(l + 1, fc);
                if (j < 0)
                  return amr_err(h, FV_ERR_INVALID_ARG,
                                 "neighbour region neither same, coarser nor finer by one level");
                src.push_back(elem(j, b));
              }
            }
          }
          neg.push_back(ng);
          start.push_back((int64_t)src.size());
        }
      }
    }
  }
  fv_amr_plan* pl = new (std::nothrow) fv_amr_plan();
  if (!pl) return amr_err(h, FV_ERR_CUDA, "out of host memory");
  pl->d = d;
  pl->s = s;
  pl->p = p;
  pl->prec = h->prec;
  pl->ncell = (int64_t)dst.size();
  cudaError_t e = cudaMalloc(&pl->d_dst, sizeof(int64_t) * dst.size());
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_start, sizeof(int64_t) * start.size());
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_src, sizeof(int64_t) * src.size());
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_neg, sizeof(int32_t) * neg.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_dst, dst.data(), sizeof(int64_t) * dst.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_start, start.data(), sizeof(int64_t) * start.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_src, src.data(), sizeof(int64_t) * src.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_neg, neg.data(), sizeof(int32_t) * neg.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    plan_free(pl);
    return amr_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = pl;
  return FV_OK;
}

fv_status fv_amr_halo_fill(fv_batch* h, const fv_amr_plan* pl, void* q) {
  if (!h || !pl || !q) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (pl->d != h->d || pl->prec != h->prec)
    return amr_err(h, FV_ERR_INVALID_ARG, "plan built for another handle kind");
  if (((uintptr_t)q & 15u) != 0) return amr_err(h, FV_ERR_ALIGNMENT, "buffer not 16-byte aligned");
  if (pl->ncell == 0) return FV_OK;
  const int64_t want = (pl->ncell + 255) / 256;
  const int grid = (int)(want < (int64_t)h->num_sms * 8 ? want : (int64_t)h->num_sms * 8);
  if (h->prec == FV_FP64)
    fv::amr_halo_kernel<double><<<grid, 256, 0, h->stream>>>(
        static_cast<double*>(q), pl->d_dst, pl->d_start, pl->d_src, pl->d_neg, pl->ncell, pl->s);
  else
    fv::amr_halo_kernel<float><<<grid, 256, 0, h->stream>>>(
        static_cast<float*>(q), pl->d_dst, pl->d_start, pl->d_src, pl->d_neg, pl->ncell, pl->s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : amr_err(h, FV_ERR_CUDA, cudaGetErrorString(e));
}

fv_status fv_amr_plan_destroy(fv_amr_plan* pl) {
  if (!pl) return FV_ERR_INVALID_ARG;
  plan_free(pl);
  return FV_OK;
}

}  // extern "C"
