// fv_reduce.cu -- maximum eigenvalue per patch and over the batch with the
// CFL time step (Eq. 5, Algorithm 1 step 10), and the fixed-order FP64
// conservation sums.
#include "fv_device.cuh"
#include "fv_internal.h"

namespace fv {

// ---------------------------------------------------------------------------
// Maximum eigenvalue.  The per-patch value is the largest a over the faces
// that bound interior cells; a face's a is the larger |u_k| + c of its two
// cells, so the patch value is the maximum of |u_k| + c over the interior
// cells (every k) and the face-halo cells (their normal k only).  One warp per
// patch (four per CTA, grid stride over the warps), the patch maximum by warp
// shuffles; cells are read straight from HBM, as 16-byte words where a cell's
// size is a multiple of 16 bytes (2D).
// ---------------------------------------------------------------------------
template <typename T>
struct EigParams {
  const T* __restrict__ q;
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ sizes;
  int64_t n;
  int halo;
  int pmax;
  T gamma, gm1;
  double* per_patch;
  unsigned long long* partials;
  unsigned int* status;
};

template <int D>
__device__ __forceinline__ int64_t ipow64(int b) {
  return D == 1 ? b : D == 2 ? (int64_t)b * b : (int64_t)b * b * b;
}

template <typename T, int D>
__global__ void __launch_bounds__(FV_NT) eig_kernel(EigParams<T> a) {
  constexpr int S = D + 2;
  constexpr int VEC = 16 / sizeof(T);
  constexpr int NW = FV_NT / 32;
  __shared__ unsigned long long red[NW];
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned long long warp_max = 0ull;  // over this warp's patches
  for (int64_t i = (int64_t)blockIdx.x * NW + (tid >> 5); i < a.n;
       i += (int64_t)gridDim.x * NW) {
    const int p = a.sizes[i];
    const int64_t off = a.off[i];
    const int h = a.halo;
    if (!(p >= 1 && p <= a.pmax && off >= 0 && (off % VEC) == 0)) {
      if (lane == 0) atomicOr(a.status, ST_BAD_PATCH);
      continue;
    }
    const int ne = p + 2 * h;
    const int ptr = D == 1 ? 1 : D == 2 ? p : p * p;
    const int nint = ptr * p;
    const T* Q = a.q + off;
    unsigned long long m = 0ull;
    bool bad = false;
    for (int t = lane; t < nint + 2 * D * ptr; t += 32) {
      int c[3] = {0, 0, 0};
      int kdir = -1;
      if (t < nint) {
        int r = t;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          c[k] = h + r % p;
          r /= p;
        }
      } else {
        int j = t - nint;
        int f = j / ptr;
        int r = j - f * ptr;
        kdir = f >> 1;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k != kdir) {
            c[k] = h + r % p;
            r /= p;
          }
        c[kdir] = (f & 1) ? h + p : h - 1;
      }
      int64_t cid = c[D - 1];
#pragma unroll
      for (int k = D - 2; k >= 0; --k) cid = cid * ne + c[k];
      T q[S];
      if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
        for (int u = 0; u < (int)(S * sizeof(T) / 16); ++u) {
          const uint4 w = __ldg(reinterpret_cast<const uint4*>(Q + cid * S) + u);
          memcpy(&q[u * (16 / sizeof(T))], &w, 16);
        }
      } else {
#pragma unroll
        for (int v = 0; v < S; ++v) q[v] = __ldg(Q + cid * S + v);
      }
      Prim<T, D> w = primitives<T, D>(q, a.gm1, a.gamma, bad);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (kdir < 0 || kdir == k) {
          const T lam = add_rn(abs_t(w.u[k]), w.c);
          const unsigned long long b = order_bits(lam);
          m = b > m ? b : m;
        }
      }
    }
    if (bad) atomicOr(a.status, ST_NONPHYSICAL);
    m = warp_max_u64(m);  // in every lane
    if (lane == 0 && a.per_patch) a.per_patch[i] = order_value<T>(m);
    warp_max = m > warp_max ? m : warp_max;
  }
  if (lane == 0) red[tid >> 5] = warp_max;
  __syncthreads();
  if (tid == 0) {
    unsigned long long mm = red[0];
#pragma unroll
    for (int w2 = 1; w2 < NW; ++w2) mm = red[w2] > mm ? red[w2] : mm;
    a.partials[blockIdx.x] = mm;
  }
}

// Reduces the per-CTA maxima (bit patterns of type T), writes the global
// maximum and dt = cfl dx / (d lambda_max).
template <typename T, int D>
__global__ void eig_finish_kernel(const unsigned long long* __restrict__ partials, int nparts,
                                  double* global_out, unsigned long long* lam_slot,
                                  double* dt_slot, double* dt_out, double cfl, double dx) {
  __shared__ unsigned long long red[32];
  unsigned long long m = 0ull;
  for (int j = threadIdx.x; j < nparts; j += blockDim.x) m = partials[j] > m ? partials[j] : m;
  m = warp_max_u64(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    m = red[0] > m ? red[0] : m;
    const double lam = order_value<T>(m);
    if (global_out) *global_out = lam;
    *lam_slot = m;  // bits, read by the next time step
    const double dt = (cfl * dx) / ((double)D * lam);
    *dt_slot = dt;
    if (dt_out) *dt_out = dt;
  }
}

template <typename T, int D>
static cudaError_t launch_eig_t(const fv_batch* h, const EigLaunch& l, int grid) {
  EigParams<T> a;
  a.q = static_cast<const T*>(l.q);
  a.off = l.off;
  a.sizes = l.sizes;
  a.n = l.n;
  a.halo = l.halo;
  a.pmax = h->max_patch_size;
  a.gamma = (T)l.gamma;
  a.gm1 = (T)(l.gamma - 1.0);
  a.per_patch = l.per_patch;
  a.partials = l.partials;
  a.status = l.status;
  eig_kernel<T, D><<<grid, FV_NT, 0, h->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_eig(const fv_batch* h, const EigLaunch& l, int grid) {
  if (h->prec == FV_FP64) {
    if (h->d == 1) return launch_eig_t<double, 1>(h, l, grid);
    if (h->d == 2) return launch_eig_t<double, 2>(h, l, grid);
    return launch_eig_t<double, 3>(h, l, grid);
  }
  if (h->d == 1) return launch_eig_t<float, 1>(h, l, grid);
  if (h->d == 2) return launch_eig_t<float, 2>(h, l, grid);
  return launch_eig_t<float, 3>(h, l, grid);
}

cudaError_t launch_eig_finish(const fv_batch* h, const unsigned long long* partials, int nparts,
                              double* global_out, unsigned long long* lam_slot, double* dt_slot,
                              double* dt_out, double cfl, double dx) {
#define FV_EIG_FIN(T, D)                                                                    \
  eig_finish_kernel<T, D><<<1, 256, 0, h->stream>>>(partials, nparts, global_out, lam_slot, \
                                                    dt_slot, dt_out, cfl, dx)
  if (h->prec == FV_FP64) {
    if (h->d == 1) FV_EIG_FIN(double, 1);
    else if (h->d == 2) FV_EIG_FIN(double, 2);
    else FV_EIG_FIN(double, 3);
  } else {
    if (h->d == 1) FV_EIG_FIN(float, 1);
    else if (h->d == 2) FV_EIG_FIN(float, 2);
    else FV_EIG_FIN(float, 3);
  }
#undef FV_EIG_FIN
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conservation sums in FP64, fixed order: chunk c holds patches
// [c*FV_SUM_CHUNK, (c+1)*FV_SUM_CHUNK); its CTA adds the patches in index
// order, each patch summed by a fixed thread-to-cell map and a fixed tree.
// A final single CTA adds the chunks with a fixed tree.  The result does not
// depend on the grid size or on timing.
// ---------------------------------------------------------------------------
template <typename T>
struct SumParams {
  const T* __restrict__ q;
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ sizes;
  int64_t n;
  int halo;
  int pmax;
  double* partials;
  unsigned int* status;
  double* per_patch;
};

template <int S>
__device__ __forceinline__ void block_sum_fixed(double (&v)[S], double* sh /*[FV_NT][S]*/) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < S; ++k) sh[tid * S + k] = v[k];
  __syncthreads();
  for (int w = FV_NT / 2; w > 0; w >>= 1) {
    if (tid < w) {
#pragma unroll
      for (int k = 0; k < S; ++k) sh[tid * S + k] = sh[tid * S + k] + sh[(tid + w) * S + k];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < S; ++k) v[k] = sh[k];
  __syncthreads();
}

template <typename T, int D>
__global__ void __launch_bounds__(FV_NT) sums_kernel(SumParams<T> a) {
  constexpr int S = D + 2;
  constexpr int VEC = 16 / sizeof(T);
  __shared__ double sh[FV_NT * S];
  double chunk[S];
#pragma unroll
  for (int k = 0; k < S; ++k) chunk[k] = 0.0;
  const int64_t i0 = (int64_t)blockIdx.x * FV_SUM_CHUNK;
  const int64_t i1 = i0 + FV_SUM_CHUNK < a.n ? i0 + FV_SUM_CHUNK : a.n;
  for (int64_t i = i0; i < i1; ++i) {
    const int p = a.sizes[i];
    const int64_t off = a.off[i];
    if (!(p >= 1 && p <= a.pmax && off >= 0 && (off % VEC) == 0)) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_BAD_PATCH);
      continue;
    }
    const int h = a.halo, ne = p + 2 * h;
    const int nint = D == 1 ? p : D == 2 ? p * p : p * p * p;
    double acc[S];
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = 0.0;
    for (int t = threadIdx.x; t < nint; t += FV_NT) {
      int c[3] = {0, 0, 0};
      int r = t;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        c[k] = h + r % p;
        r /= p;
      }
      int64_t cid = c[D - 1];
#pragma unroll
      for (int k = D - 2; k >= 0; --k) cid = cid * ne + c[k];
      const T* qc = a.q + off + cid * S;
#pragma unroll
      for (int k = 0; k < S; ++k) acc[k] = acc[k] + (double)__ldg(qc + k);
    }
    block_sum_fixed<S>(acc, sh);
    if (a.per_patch != nullptr && threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < S; ++k) a.per_patch[i * S + k] = acc[k];
    }
#pragma unroll
    for (int k = 0; k < S; ++k) chunk[k] = chunk[k] + acc[k];
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < S; ++k) a.partials[(int64_t)blockIdx.x * S + k] = chunk[k];
  }
}

template <int S>
__global__ void __launch_bounds__(FV_NT) sums_finish_kernel(const double* __restrict__ partials,
                                                            int nchunks, double* totals) {
  __shared__ double sh[FV_NT * S];
  double acc[S];
#pragma unroll
  for (int k = 0; k < S; ++k) acc[k] = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += FV_NT) {
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = acc[k] + partials[(int64_t)c * S + k];
  }
  block_sum_fixed<S>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < S; ++k) totals[k] = acc[k];
  }
}

template <typename T, int D>
static cudaError_t launch_sums_t(const fv_batch* h, const SumLaunch& l, int nchunks) {
  SumParams<T> a;
  a.q = static_cast<const T*>(l.q);
  a.off = l.off;
  a.sizes = l.sizes;
  a.n = l.n;
  a.halo = l.halo;
  a.pmax = h->max_patch_size;
  a.partials = l.partials;
  a.status = l.status;
  a.per_patch = l.per_patch;
  sums_kernel<T, D><<<nchunks, FV_NT, 0, h->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sums(const fv_batch* h, const SumLaunch& l, int nchunks) {
  if (h->prec == FV_FP64) {
    if (h->d == 1) return launch_sums_t<double, 1>(h, l, nchunks);
    if (h->d == 2) return launch_sums_t<double, 2>(h, l, nchunks);
    return launch_sums_t<double, 3>(h, l, nchunks);
  }
  if (h->d == 1) return launch_sums_t<float, 1>(h, l, nchunks);
  if (h->d == 2) return launch_sums_t<float, 2>(h, l, nchunks);
  return launch_sums_t<float, 3>(h, l, nchunks);
}

cudaError_t launch_sums_finish(const fv_batch* h, const double* partials, int nchunks,
                               double* totals) {
  if (h->d == 1) sums_finish_kernel<3><<<1, FV_NT, 0, h->stream>>>(partials, nchunks, totals);
  else if (h->d == 2) sums_finish_kernel<4><<<1, FV_NT, 0, h->stream>>>(partials, nchunks, totals);
  else sums_finish_kernel<5><<<1, FV_NT, 0, h->stream>>>(partials, nchunks, totals);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One 64-bit word set to zero on the stream (the wave-speed slot a time step
// accumulates into, the work-queue counter), by a one-thread kernel.
// ---------------------------------------------------------------------------
__global__ void zero_word_kernel(unsigned long long* p) { *p = 0ull; }

cudaError_t launch_zero_word(unsigned long long* p, cudaStream_t stream) {
  zero_word_kernel<<<1, 1, 0, stream>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-test of the FP64 reciprocal and square root used by the kernels.
// ---------------------------------------------------------------------------
__global__ void selftest_math_kernel(const double* __restrict__ x, double* __restrict__ out,
                                     int64_t n, int which) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = which == 0 ? recip(x[i]) : sqrt_t(x[i]);
}

cudaError_t launch_selftest_math(const double* x, double* out, int64_t n, int which) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  selftest_math_kernel<<<(int)blocks, 256>>>(x, out, n, which);
  return cudaGetLastError();
}

}  // namespace fv
