// fv_update.cu -- the batched Rusanov patch update (Eq. 3-5, Algorithm 1 with
// the outer loop over patches).
//
// One CTA advances one patch at a time and walks the batch with a grid
// stride.  Per patch:
//   stage   the halo-inclusive patch is read from HBM with 16-byte loads and
//           transposed into shared memory, one array per unknown (SoA), so
//           consecutive threads read consecutive cells without bank conflicts;
//   cells   every interior and face-halo cell converts to primitives once and
//           writes, for each direction whose faces it touches, its flux f^k
//           and wave speed |u_k| + c (Eq. 2, 5) into a per-direction box;
//   faces   every face flux G = f_L + f_R - a (Q_R - Q_L) = 2 F (Eq. 4) is
//           computed exactly once and kept in shared memory;
//   update  every interior cell sums G_+ - G_- over the directions (x, then
//           y, then z) and writes Q - (dt / 2dx) sum to HBM (Eq. 3).
// The per-patch maximum of a over the faces (Algorithm 1 step 10) is reduced
// with warp shuffles on the integer bit patterns (exact, order free).
#include "fv_device.cuh"
#include "fv_internal.h"

namespace fv {

template <typename T>
struct UpdateParams {
  const T* __restrict__ in;
  T* __restrict__ out;
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ sizes;
  int64_t n;
  int64_t n_elems;
  int pmax;
  T gamma, gm1;
  double dx, dt;
  const double* dt_dev;
  double* lam_patch;
  unsigned int* status;
};

template <int D>
__host__ __device__ inline int ipow_d(int b) {
  return D == 1 ? b : D == 2 ? b * b : b * b * b;
}

// Elements of shared memory (in units of T) for one patch of size p.
template <int D>
__host__ __device__ inline int update_smem_elems(int p) {
  constexpr int S = D + 2;
  int ncell = ipow_d<D>(p + 2);
  int ptr = ipow_d<D>(p) / p;
  int nbox = (p + 2) * ptr, nface = (p + 1) * ptr;
  return S * ncell + D * (S + 1) * nbox + D * S * nface;
}

constexpr int kRedBytes = 8 * (FV_NT / 32);

template <typename T, int D, int P>
__device__ __forceinline__ void update_patch(const UpdateParams<T>& a, int p_rt, int64_t i,
                                             int64_t off, T hr, T* smem,
                                             unsigned long long* red) {
  constexpr int S = D + 2;
  constexpr int NT = FV_NT;
  const Geom<D, P> g(p_rt);
  const int p = g.p;
  const int ncell = g.ncell(), nbox = g.nbox(), nface = g.nface(), nint = g.nint();
  const int ptr = g.ptrans();
  T* Qs = smem;                    // [S][ncell]
  T* Fb = Qs + S * ncell;          // [D][S+1][nbox]: f^k then |u_k|+c
  T* Gb = Fb + D * (S + 1) * nbox;  // [D][S][nface]
  const int tid = threadIdx.x;

  // ---- stage: HBM -> shared memory, AoS -> SoA --------------------------
  {
    const T* src = a.in + off;
    const int nel = ncell * S;
    constexpr int VEC = 16 / sizeof(T);
    const int nvec = nel / VEC;
    for (int v = tid; v < nvec; v += NT) {
      T x[VEC];
      if constexpr (sizeof(T) == 8) {
        double2 w = __ldg(reinterpret_cast<const double2*>(src) + v);
        x[0] = w.x;
        x[1] = w.y;
      } else {
        float4 w = __ldg(reinterpret_cast<const float4*>(src) + v);
        x[0] = w.x;
        x[1] = w.y;
        x[2] = w.z;
        x[3] = w.w;
      }
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        int e = v * VEC + u;
        int c = e / S;
        Qs[(e - c * S) * ncell + c] = x[u];
      }
    }
    for (int e = nvec * VEC + tid; e < nel; e += NT) {
      int c = e / S;
      Qs[(e - c * S) * ncell + c] = __ldg(src + e);
    }
  }
  __syncthreads();

  // ---- cells: primitives once, flux and wave speed per needed direction --
  bool bad = false;
  {
    const int n1 = nint + 2 * D * ptr;
    for (int t = tid; t < n1; t += NT) {
      int c[3] = {0, 0, 0};
      int kdir;
      if (t < nint) {
        int r = t;
#pragma unroll
        for (int m = 0; m < D; ++m) {
          c[m] = 1 + r % p;
          r /= p;
        }
        kdir = -1;
      } else {
        int j = t - nint;
        int f = j / ptr;
        int r = j - f * ptr;
        kdir = f >> 1;
        g.untrans(r, kdir, c);
        c[kdir] = (f & 1) ? p + 1 : 0;
      }
      const int cid = g.cell(c);
      T q[S];
#pragma unroll
      for (int v = 0; v < S; ++v) q[v] = Qs[v * ncell + cid];
      Prim<T, D> w = primitives<T, D>(q, a.gm1, a.gamma, bad);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (kdir < 0 || kdir == k) {
          T f[S], lam;
          flux_dir<T, D>(q, w, k, f, lam);
          const int b = c[k] + (p + 2) * g.trans(c, k);
          T* F = Fb + k * (S + 1) * nbox;
#pragma unroll
          for (int v = 0; v < S; ++v) F[v * nbox + b] = f[v];
          F[S * nbox + b] = lam;
        }
      }
    }
  }
  __syncthreads();

  // ---- faces: G = f_L + f_R - a (Q_R - Q_L), once per face ---------------
  unsigned long long lmax = 0ull;
  {
    for (int t = tid; t < D * nface; t += NT) {
      const int k = t / nface;
      const int j = t - k * nface;
      const int tr = j / (p + 1);
      const int b = j - tr * (p + 1);
      int c[3] = {0, 0, 0};
      g.untrans(tr, k, c);
      c[k] = b;
      const int cl = g.cell(c);
      const int stride = k == 0 ? 1 : k == 1 ? (p + 2) : (p + 2) * (p + 2);
      const int cr = cl + stride;
      const T* F = Fb + k * (S + 1) * nbox;
      const int bl = b + (p + 2) * tr;
      const T am = max_by_bits(F[S * nbox + bl], F[S * nbox + bl + 1]);
      const unsigned long long ab = order_bits(am);
      lmax = ab > lmax ? ab : lmax;
      T* G = Gb + k * S * nface;
#pragma unroll
      for (int v = 0; v < S; ++v) {
        const T dq = Qs[v * ncell + cr] - Qs[v * ncell + cl];
        const T fs = F[v * nbox + bl] + F[v * nbox + bl + 1];
        G[v * nface + j] = fma(-am, dq, fs);
      }
    }
  }
  __syncthreads();

  // ---- update: Q - (dt/2dx) sum_k (G_+ - G_-), interior cells -------------
  {
    T* dst_base = a.out + off;
    for (int t = tid; t < nint; t += NT) {
      int c[3] = {0, 0, 0};
      int r = t;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        c[m] = 1 + r % p;
        r /= p;
      }
      const int cid = g.cell(c);
      T acc[S];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int jm = (c[k] - 1) + (p + 1) * g.trans(c, k);
        const T* G = Gb + k * S * nface;
#pragma unroll
        for (int v = 0; v < S; ++v) {
          const T dG = G[v * nface + jm + 1] - G[v * nface + jm];
          acc[v] = k == 0 ? dG : acc[v] + dG;
        }
      }
      T* dst = dst_base + (int64_t)cid * S;
#pragma unroll
      for (int v = 0; v < S; ++v) dst[v] = fma(-hr, acc[v], Qs[v * ncell + cid]);
    }
  }

  if (bad) atomicOr(a.status, ST_NONPHYSICAL);
  if (a.lam_patch != nullptr) {
    lmax = warp_max_u64(lmax);
    if ((tid & 31) == 0) red[tid >> 5] = lmax;
    __syncthreads();
    if (tid == 0) {
      unsigned long long m = red[0];
#pragma unroll
      for (int w = 1; w < NT / 32; ++w) m = red[w] > m ? red[w] : m;
      a.lam_patch[i] = order_value<T>(m);
    }
  }
  __syncthreads();  // shared memory is reused by the next patch
}

template <typename T, int D>
__device__ __forceinline__ void update_dispatch(const UpdateParams<T>& a, int p, int64_t i,
                                                int64_t off, T hr, T* smem,
                                                unsigned long long* red) {
  if constexpr (D == 3) {
    switch (p) {
      case 3: update_patch<T, 3, 3>(a, p, i, off, hr, smem, red); return;
      case 5: update_patch<T, 3, 5>(a, p, i, off, hr, smem, red); return;
      case 7: update_patch<T, 3, 7>(a, p, i, off, hr, smem, red); return;
      default: update_patch<T, 3, 0>(a, p, i, off, hr, smem, red); return;
    }
  } else if constexpr (D == 2) {
    switch (p) {
      case 3: update_patch<T, 2, 3>(a, p, i, off, hr, smem, red); return;
      case 5: update_patch<T, 2, 5>(a, p, i, off, hr, smem, red); return;
      case 8: update_patch<T, 2, 8>(a, p, i, off, hr, smem, red); return;
      case 17: update_patch<T, 2, 17>(a, p, i, off, hr, smem, red); return;
      default: update_patch<T, 2, 0>(a, p, i, off, hr, smem, red); return;
    }
  } else {
    update_patch<T, 1, 0>(a, p, i, off, hr, smem, red);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(FV_NT) update_kernel(UpdateParams<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem_raw);
  T* smem = reinterpret_cast<T*>(smem_raw + kRedBytes);
  constexpr int S = D + 2;
  constexpr int VEC = 16 / sizeof(T);
  const double dtv = a.dt > 0.0 ? a.dt : *a.dt_dev;
  const T hr = (T)(0.5 * (dtv / a.dx));
  for (int64_t i = blockIdx.x; i < a.n; i += gridDim.x) {
    const int p = a.sizes[i];
    const int64_t off = a.off[i];
    bool ok = p >= 1 && p <= a.pmax && off >= 0 && (off % VEC) == 0;
    if (ok && a.n_elems > 0) ok = off + (int64_t)ipow_d<D>(p + 2) * S <= a.n_elems;
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_BAD_PATCH);
      continue;
    }
    update_dispatch<T, D>(a, p, i, off, hr, smem, red);
  }
}

size_t update_smem_bytes(int d, fv_precision prec, int pmax) {
  size_t es = prec == FV_FP64 ? 8 : 4;
  int elems = d == 1 ? update_smem_elems<1>(pmax)
              : d == 2 ? update_smem_elems<2>(pmax)
                       : update_smem_elems<3>(pmax);
  return kRedBytes + es * (size_t)elems;
}

template <typename T, int D>
static cudaError_t launch_update_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
  UpdateParams<T> a;
  a.in = static_cast<const T*>(l.in);
  a.out = static_cast<T*>(l.out);
  a.off = l.off;
  a.sizes = l.sizes;
  a.n = l.n;
  a.n_elems = l.n_elems;
  a.pmax = l.pmax;
  a.gamma = (T)l.gamma;
  a.gm1 = (T)(l.gamma - 1.0);
  a.dx = l.dx;
  a.dt = l.dt;
  a.dt_dev = l.dt_dev;
  a.lam_patch = l.lam_patch;
  a.status = l.status;
  size_t smem = update_smem_bytes(D, h->prec, l.pmax);
  cudaError_t e = cudaFuncSetAttribute(update_kernel<T, D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  update_kernel<T, D><<<grid, FV_NT, smem, h->stream>>>(a);
  return cudaGetLastError();
}

template <typename T, int D>
static cudaError_t occupancy_t(const fv_batch* h, int* bps) {
  size_t smem = update_smem_bytes(D, h->prec, h->max_patch_size);
  cudaError_t e = cudaFuncSetAttribute(update_kernel<T, D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, update_kernel<T, D>, FV_NT, smem);
}

cudaError_t launch_update(const fv_batch* h, const UpdateLaunch& l, int grid) {
  if (h->prec == FV_FP64) {
    if (h->d == 1) return launch_update_t<double, 1>(h, l, grid);
    if (h->d == 2) return launch_update_t<double, 2>(h, l, grid);
    return launch_update_t<double, 3>(h, l, grid);
  }
  if (h->d == 1) return launch_update_t<float, 1>(h, l, grid);
  if (h->d == 2) return launch_update_t<float, 2>(h, l, grid);
  return launch_update_t<float, 3>(h, l, grid);
}

cudaError_t update_occupancy(const fv_batch* h, int* bps) {
  if (h->prec == FV_FP64) {
    if (h->d == 1) return occupancy_t<double, 1>(h, bps);
    if (h->d == 2) return occupancy_t<double, 2>(h, bps);
    return occupancy_t<double, 3>(h, bps);
  }
  if (h->d == 1) return occupancy_t<float, 1>(h, bps);
  if (h->d == 2) return occupancy_t<float, 2>(h, bps);
  return occupancy_t<float, 3>(h, bps);
}

}  // namespace fv
