// fv_learned.cu -- the learned conservative face-flux correction on 2D patch
// meshes (an addition on top of the Rusanov flux of Eq. 4, not in the paper):
//
//   correction  every face of every patch gets C = sd_y * net((S - mu)/sd),
//               S the 4-cell stencil Q_{i-2..i+1} normal to the face in the
//               face's normal frame (rho, j_n, j_t, E), net the 16 -> 64 -> 64
//               -> 4 GELU network, evaluated by one warp per 16 faces on the
//               tensor cores (BF16 mma.sync, FP32 accumulation; hidden
//               activations stay in registers between layers).  The update
//               adds C to the face flux once per face, so both cells see the
//               same flux and the totals are conserved.  A face shared by two
//               patches gets the same C in both (same stencil, same arithmetic).
//   targets     the data the network is trained on: the fine solution at r
//               times the resolution, restricted by block averages, evolves
//               exactly by the time-and-face averages of the fine fluxes
//               through the coarse faces; the ideal correction is that
//               average minus the coarse Rusanov flux.
//
// Face indexing per patch (as in the update kernel): direction k, face
// j = tr + p b, b in [0, p] the halo-1 coordinate of the left cell along k,
// tr in [0, p) the transverse interior coordinate minus one.  Per-face arrays
// are laid out [patch][k][v][j].
#include <stdio.h>

#include "fv_device.cuh"
#include "fv_internal.h"
#include "fv_mma.cuh"

namespace fv {

constexpr int kLNT = 128;  // threads per CTA of the learned kernels
constexpr int kLPmax = 16;  // largest patch of the learned kernels

__host__ __device__ inline int64_t corr_stride_for(int pmax) {
  return 2ll * 4 * (pmax + 1) * pmax;
}

// ---------------------------------------------------------------------------
// Stage of one 2D patch with two cell layers around it along each face
// normal, as floats, in coordinates X, Y in [0, p+4) (interior 2..p+1).
// Outside cells come from the neighbours' interiors by the rules of
// fv_halo_fill (>= 0 neighbour, -1 outflow, -2 wall with the normal momentum
// negated), for two layers.
// ---------------------------------------------------------------------------
template <typename T>
struct MeshView {
  const T* q;
  const int64_t* off;
  const int32_t* sizes;
  const int32_t* nbr;
  int64_t n;
  unsigned int* status;
};

// Source of cell (x, y) in halo-1 coordinates of patch pid, x or y possibly
// outside [1, p] by up to two cells along one axis; returns a pointer to its
// 4 unknowns and whether the normal momentum is negated (component 1+k).
template <typename T>
__device__ __forceinline__ const T* cell_source(const MeshView<T>& m, int64_t pid, int p, int x,
                                                int y, int& neg_comp) {
  neg_comp = -1;
  int k = -1, side = 0, depth = 0;  // which face the cell lies beyond
  if (x < 1) { k = 0; side = 0; depth = 1 - x; }
  else if (x > p) { k = 0; side = 1; depth = x - p; }
  else if (y < 1) { k = 1; side = 0; depth = 1 - y; }
  else if (y > p) { k = 1; side = 1; depth = y - p; }
  int64_t src = pid;
  if (k >= 0) {
    const int32_t nb = m.nbr[pid * 4 + 2 * k + side];
    int along;  // interior coordinate (1..p) along k in the source patch
    if (nb >= 0 && nb < m.n && m.sizes[nb] == p) {
      src = nb;
      along = side ? depth : p + 1 - depth;
    } else {
      if (!(nb == -1 || nb == -2)) atomicOr(m.status, ST_BAD_PATCH);
      if (nb == -2) {  // wall: mirror image
        along = side ? p + 1 - depth : depth;
        neg_comp = 1 + k;
      } else {  // outflow: nearest interior cell
        along = side ? p : 1;
      }
    }
    if (k == 0) x = along; else y = along;
  }
  return m.q + m.off[src] + ((int64_t)y * (p + 2) + x) * 4;
}

template <typename T>
__device__ void fill_stage(const MeshView<T>& m, int64_t pid, int p, float* stage) {
  const int ns = p + 4;
  // interior p^2, then 4 sides x 2 layers x p
  const int total = p * p + 8 * p;
  for (int t = threadIdx.x; t < total; t += kLNT) {
    int x, y;
    if (t < p * p) {
      x = 1 + t % p;
      y = 1 + t / p;
    } else {
      const int u = t - p * p;
      const int side4 = u / (2 * p);  // 0: -x, 1: +x, 2: -y, 3: +y
      const int r = u - side4 * 2 * p;
      const int layer = r / p;  // 0: next to the face, 1: beyond
      const int tr = 1 + r % p;
      const int c = (side4 & 1) ? p + 1 + layer : -layer;
      if (side4 < 2) { x = c; y = tr; } else { x = tr; y = c; }
    }
    int neg;
    const T* s = cell_source(m, pid, p, x, y, neg);
    float* d = stage + ((y + 1) * ns + (x + 1)) * 4;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float val = (float)s[v];
      d[v] = (v == neg) ? -val : val;
    }
  }
}

// Normal-frame component vn (rho, j_n, j_t, E) of a cell for direction k.
__device__ __forceinline__ int phys_comp(int k, int vn) {
  return (k == 1 && (vn == 1 || vn == 2)) ? 3 - vn : vn;
}

// ---------------------------------------------------------------------------
// Correction kernel
// ---------------------------------------------------------------------------
struct NetSmem {
  uint16_t w1[64 * 16];
  uint16_t w2[64 * 64];
  uint16_t w3[8 * 64];  // rows 4..7 zero
  float b1[64], b2[64], b3[8];
  float mu[16], sd[16], sdy[4];
};

__device__ void load_net(const float* params, const float* norm, NetSmem& s) {
  for (int i = threadIdx.x; i < 64 * 16; i += kLNT) s.w1[i] = f32_to_bf16(params[kOffW1 + i]);
  for (int i = threadIdx.x; i < 64 * 64; i += kLNT) s.w2[i] = f32_to_bf16(params[kOffW2 + i]);
  for (int i = threadIdx.x; i < 8 * 64; i += kLNT)
    s.w3[i] = i < 4 * 64 ? f32_to_bf16(params[kOffW3 + i]) : (uint16_t)0;
  for (int i = threadIdx.x; i < 64; i += kLNT) {
    s.b1[i] = params[kOffB1 + i];
    s.b2[i] = params[kOffB2 + i];
  }
  if (threadIdx.x < 8) s.b3[threadIdx.x] = threadIdx.x < 4 ? params[kOffB3 + threadIdx.x] : 0.f;
  if (threadIdx.x < 16) {
    s.mu[threadIdx.x] = norm[threadIdx.x];
    s.sd[threadIdx.x] = norm[16 + threadIdx.x];
  }
  if (threadIdx.x < 4) s.sdy[threadIdx.x] = norm[32 + threadIdx.x];
}

// Normalised feature phi of face f (k, b, tr) from the stage.
__device__ __forceinline__ float feature(const NetSmem& s, const float* stage, int p, int k,
                                         int b, int tr, int phi) {
  const int c = phi >> 2, vn = phi & 3;
  const int along = b + c;  // stage coordinate along k of stencil cell c
  const int X = k == 0 ? along : tr + 2;
  const int Y = k == 0 ? tr + 2 : along;
  const float v = stage[(Y * (p + 4) + X) * 4 + phys_comp(k, vn)];
  return (v - s.mu[phi]) / s.sd[phi];
}

// One warp: corrections of faces [f0base, f0base + 16).
__device__ __forceinline__ void net_tile(const NetSmem& s, const float* stage, int p, int nf1,
                                         int fbase, float (&out)[2][2], int (&kk_out)[2],
                                         int (&j_out)[2]) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int nfaces = 2 * nf1;
  int fk[2], fb[2], ftr[2];
  bool ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int f = fbase + g + 8 * r;
    ok[r] = f < nfaces;
    const int fc = ok[r] ? f : 0;
    fk[r] = fc / nf1;
    const int j = fc - fk[r] * nf1;
    fb[r] = j / p;
    ftr[r] = j - fb[r] * p;
    kk_out[r] = ok[r] ? fk[r] : -1;
    j_out[r] = j;
  }
  auto F = [&](int r, int phi) -> float {
    return ok[r] ? feature(s, stage, p, fk[r], fb[r], ftr[r], phi) : 0.f;
  };
  uint32_t a[4];
  a[0] = pack_bf16(F(0, 2 * t), F(0, 2 * t + 1));
  a[1] = pack_bf16(F(1, 2 * t), F(1, 2 * t + 1));
  a[2] = pack_bf16(F(0, 2 * t + 8), F(0, 2 * t + 9));
  a[3] = pack_bf16(F(1, 2 * t + 8), F(1, 2 * t + 9));
  // layer 1: 16 -> 64
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    const uint16_t* w = s.w1 + (nt * 8 + g) * 16;
    const uint32_t b[2] = {*reinterpret_cast<const uint32_t*>(w + 2 * t),
                           *reinterpret_cast<const uint32_t*>(w + 2 * t + 8)};
    mma_16816(acc[nt], a, b);
  }
  uint32_t h[4][4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int nt = 2 * kk + half;
      const int n = nt * 8 + 2 * t;
      const float z0 = gelu_f(acc[nt][0] + s.b1[n]), z1 = gelu_f(acc[nt][1] + s.b1[n + 1]);
      const float z2 = gelu_f(acc[nt][2] + s.b1[n]), z3 = gelu_f(acc[nt][3] + s.b1[n + 1]);
      h[kk][2 * half] = pack_bf16(z0, z1);
      h[kk][2 * half + 1] = pack_bf16(z2, z3);
    }
  }
  // layer 2: 64 -> 64
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint16_t* w = s.w2 + (nt * 8 + g) * 64 + kk * 16;
      const uint32_t b[2] = {*reinterpret_cast<const uint32_t*>(w + 2 * t),
                             *reinterpret_cast<const uint32_t*>(w + 2 * t + 8)};
      const uint32_t ak[4] = {h[kk][0], h[kk][1], h[kk][2], h[kk][3]};
      mma_16816(acc[nt], ak, b);
    }
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int nt = 2 * kk + half;
      const int n = nt * 8 + 2 * t;
      const float z0 = gelu_f(acc[nt][0] + s.b2[n]), z1 = gelu_f(acc[nt][1] + s.b2[n + 1]);
      const float z2 = gelu_f(acc[nt][2] + s.b2[n]), z3 = gelu_f(acc[nt][3] + s.b2[n + 1]);
      h[kk][2 * half] = pack_bf16(z0, z1);
      h[kk][2 * half + 1] = pack_bf16(z2, z3);
    }
  }
  // layer 3: 64 -> 4 (padded to 8)
  float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint16_t* w = s.w3 + g * 64 + kk * 16;
    const uint32_t b[2] = {*reinterpret_cast<const uint32_t*>(w + 2 * t),
                           *reinterpret_cast<const uint32_t*>(w + 2 * t + 8)};
    const uint32_t ak[4] = {h[kk][0], h[kk][1], h[kk][2], h[kk][3]};
    mma_16816(y, ak, b);
  }
  // lanes t = 0, 1 hold output columns 2t, 2t+1 of rows g (y[0..1]), g+8 (y[2..3])
  const int c0 = 2 * t;
  out[0][0] = c0 < 4 ? (y[0] + s.b3[c0]) * s.sdy[c0] : 0.f;
  out[0][1] = c0 < 4 ? (y[1] + s.b3[c0 + 1]) * s.sdy[c0 + 1] : 0.f;
  out[1][0] = c0 < 4 ? (y[2] + s.b3[c0]) * s.sdy[c0] : 0.f;
  out[1][1] = c0 < 4 ? (y[3] + s.b3[c0 + 1]) * s.sdy[c0 + 1] : 0.f;
}

template <typename T>
__global__ void __launch_bounds__(kLNT) corr_kernel(MeshView<T> m, int pmax, const float* params,
                                                    const float* norm, float* corr,
                                                    int64_t stride) {
  __shared__ NetSmem s;
  __shared__ float stage[(kLPmax + 4) * (kLPmax + 4) * 4];
  load_net(params, norm, s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 3;
  for (int64_t pid = blockIdx.x; pid < m.n; pid += gridDim.x) {
    const int p = m.sizes[pid];
    if (p < 1 || p > pmax) {
      if (threadIdx.x == 0) atomicOr(m.status, ST_BAD_PATCH);
      continue;
    }
    __syncthreads();  // stage reuse, and the network loaded
    fill_stage(m, pid, p, stage);
    __syncthreads();
    const int nf1 = (p + 1) * p;
    const int ntiles = (2 * nf1 + 15) / 16;
    for (int tile = warp; tile < ntiles; tile += kLNT / 32) {
      float out[2][2];
      int kf[2], jf[2];
      net_tile(s, stage, p, nf1, tile * 16, out, kf, jf);
      if (t < 2) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (kf[r] < 0) continue;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int vn = 2 * t + c;
            corr[pid * stride + (kf[r] * 4 + phys_comp(kf[r], vn)) * nf1 + jf[r]] = out[r][c];
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Training data
// ---------------------------------------------------------------------------
// Rusanov flux (Eq. 4) of direction k between two 2D states (physical frame).
template <typename T>
__device__ __forceinline__ void rusanov2(const T* qL, const T* qR, int k, T gamma, T gm1,
                                         T (&F)[4]) {
  bool bad = false;
  const Prim<T, 2> wl = primitives<T, 2>(qL, gm1, gamma, bad);
  const Prim<T, 2> wr = primitives<T, 2>(qR, gm1, gamma, bad);
  T fl[4], fr[4], ll, lr;
  flux_dir<T, 2>(qL, wl, k, fl, ll);
  flux_dir<T, 2>(qR, wr, k, fr, lr);
  const T a = max_by_bits(ll, lr);
#pragma unroll
  for (int v = 0; v < 4; ++v) F[v] = T(0.5) * fma(a, qL[v] - qR[v], fl[v] + fr[v]);
}

struct MeshGeom {
  int p;        // patch size
  int px, py;   // patches per axis (patch index = a + px b)
};

// Coarse interior cell = mean of its r x r fine cells.
template <typename Tf, typename Tc>
__global__ void restrict_kernel(const Tf* __restrict__ qf, const int64_t* __restrict__ off_f,
                                MeshGeom gf, Tc* qc, const int64_t* __restrict__ off_c,
                                MeshGeom gc, int r) {
  const int64_t ncell = (int64_t)gc.px * gc.py * gc.p * gc.p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pc = e / (gc.p * gc.p);
    const int loc = (int)(e - pc * gc.p * gc.p);
    const int cx = loc % gc.p, cy = loc / gc.p;
    const int64_t I = (pc % gc.px) * gc.p + cx, J = (pc / gc.px) * gc.p + cy;
    double acc[4] = {0, 0, 0, 0};
    for (int b = 0; b < r; ++b)
      for (int a = 0; a < r; ++a) {
        const int64_t fx = I * r + a, fy = J * r + b;
        const int64_t pf = (fx / gf.p) + gf.px * (fy / gf.p);
        const int lx = (int)(fx % gf.p) + 1, ly = (int)(fy % gf.p) + 1;
        const Tf* c = qf + off_f[pf] + ((int64_t)ly * (gf.p + 2) + lx) * 4;
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += (double)c[v];
      }
    Tc* d = qc + off_c[pc] + ((int64_t)(cy + 1) * (gc.p + 2) + (cx + 1)) * 4;
    const double inv = 1.0 / ((double)r * r);
#pragma unroll
    for (int v = 0; v < 4; ++v) d[v] = (Tc)(acc[v] * inv);
  }
}

// acc[coarse face] += weight * mean of the r fine Rusanov fluxes on it.
template <typename Tf>
__global__ void accum_kernel(const Tf* __restrict__ qf, const int64_t* __restrict__ off_f,
                             MeshGeom gf, MeshGeom gc, int r, Tf gamma, double weight,
                             double* acc, int64_t stride) {
  const int nf1 = (gc.p + 1) * gc.p;
  const int64_t nfaces = (int64_t)gc.px * gc.py * 2 * nf1;
  const int64_t NfX = (int64_t)gf.px * gf.p, NfY = (int64_t)gf.py * gf.p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nfaces;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pc = e / (2 * nf1);
    const int rem = (int)(e - pc * 2 * nf1);
    const int k = rem / nf1, j = rem - k * nf1;
    const int b = j / gc.p, tr = j - b * gc.p;
    const int64_t A = (pc % gc.px) * gc.p, Bq = (pc / gc.px) * gc.p;  // patch origin
    // coarse face: along k at coarse coordinate (origin + b), transverse origin + tr
    double sum[4] = {0, 0, 0, 0};
    for (int a = 0; a < r; ++a) {
      int64_t fx, fy;  // fine cell right of / above the fine face
      if (k == 0) {
        fx = ((A + b) * r) % NfX;
        fy = (Bq + tr) * r + a;
      } else {
        fx = (A + tr) * r + a;
        fy = ((Bq + b) * r) % NfY;
      }
      const int64_t pf = (fx / gf.p) + gf.px * (fy / gf.p);
      const int lx = (int)(fx % gf.p) + 1, ly = (int)(fy % gf.p) + 1;
      const Tf* base = qf + off_f[pf];
      const Tf* qR = base + ((int64_t)ly * (gf.p + 2) + lx) * 4;
      const Tf* qL = k == 0 ? qR - 4 : qR - (int64_t)(gf.p + 2) * 4;  // halo when at the edge
      Tf F[4];
      rusanov2<Tf>(qL, qR, k, gamma, gamma - Tf(1), F);
#pragma unroll
      for (int v = 0; v < 4; ++v) sum[v] += (double)F[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v)
      acc[pc * stride + (k * 4 + v) * nf1 + j] += weight * sum[v] / (double)r;
  }
}

// Per coarse face: raw stencil (16, normal frame) and target C* = acc - F_c
// (4, normal frame), sample index = patch * 2 nf1 + k nf1 + j.
template <typename T>
__global__ void __launch_bounds__(kLNT) targets_kernel(MeshView<T> m, int pmax, T gamma,
                                                       const double* __restrict__ acc,
                                                       int64_t stride, float* x_raw,
                                                       float* t_raw) {
  __shared__ float stage[(kLPmax + 4) * (kLPmax + 4) * 4];
  for (int64_t pid = blockIdx.x; pid < m.n; pid += gridDim.x) {
    const int p = m.sizes[pid];
    if (p < 1 || p > pmax) continue;
    __syncthreads();
    fill_stage(m, pid, p, stage);
    __syncthreads();
    const int nf1 = (p + 1) * p;
    for (int f = threadIdx.x; f < 2 * nf1; f += kLNT) {
      const int k = f / nf1, j = f - k * nf1;
      const int b = j / p, tr = j - b * p;
      const int64_t sidx = pid * 2 * nf1 + f;
      for (int phi = 0; phi < 16; ++phi) {
        const int c = phi >> 2, vn = phi & 3, along = b + c;
        const int X = k == 0 ? along : tr + 2, Y = k == 0 ? tr + 2 : along;
        x_raw[sidx * 16 + phi] = stage[(Y * (p + 4) + X) * 4 + phys_comp(k, vn)];
      }
      // exact (un-rounded) left and right states of the face from the mesh
      int negL, negR;
      const int xl = k == 0 ? b : tr + 1, yl = k == 0 ? tr + 1 : b;
      const int xr = k == 0 ? b + 1 : tr + 1, yr = k == 0 ? tr + 1 : b + 1;
      const T* sl = cell_source(m, pid, p, xl, yl, negL);
      const T* sr = cell_source(m, pid, p, xr, yr, negR);
      T qL[4], qR[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qL[v] = v == negL ? -sl[v] : sl[v];
        qR[v] = v == negR ? -sr[v] : sr[v];
      }
      T F[4];
      rusanov2<T>(qL, qR, k, gamma, gamma - T(1), F);
#pragma unroll
      for (int vn = 0; vn < 4; ++vn) {
        const int v = phys_comp(k, vn);
        t_raw[sidx * 4 + vn] = (float)(acc[pid * stride + (k * 4 + v) * nf1 + j] - (double)F[v]);
      }
    }
  }
}

// Column sums and sums of squares (FP64), fixed chunks of rows per block.
__global__ void moments_kernel(const float* __restrict__ x, int64_t rows, int cols,
                               int64_t chunk, double* part) {
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = r0 + chunk < rows ? r0 + chunk : rows;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    double s = 0.0, s2 = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const double v = x[r * cols + c];
      s += v;
      s2 += v * v;
    }
    part[(blockIdx.x * 2) * cols + c] = s;
    part[(blockIdx.x * 2 + 1) * cols + c] = s2;
  }
}
__global__ void moments_finish_kernel(const double* __restrict__ part, int nb, int cols,
                                      double* sum, double* sumsq) {
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < nb; ++b) {
      s += part[(b * 2) * cols + c];
      s2 += part[(b * 2 + 1) * cols + c];
    }
    sum[c] = s;
    sumsq[c] = s2;
  }
}
__global__ void normalize_kernel(float* x, int64_t rows, int cols, const float* mu,
                                 const float* sd) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % cols);
    x[e] = (x[e] - (mu ? mu[c] : 0.f)) / sd[c];
  }
}

}  // namespace fv

namespace {
int grid_for_items(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}
fv_status lerr(fv_batch* h, fv_status st, const char* msg) {
  if (h) snprintf(h->last_error, sizeof(h->last_error), "%s", msg);
  return st;
}
}  // namespace

extern "C" {

int64_t fv_corr_stride(const fv_batch* h) {
  return h ? fv::corr_stride_for(h->max_patch_size) : 0;
}

fv_status fv_flux_correction(fv_batch* h, const void* q, const int64_t* off, const int32_t* sizes,
                             const int32_t* nbr, int64_t n, const float* params,
                             const float* norm, float* corr) {
  if (!h) return FV_ERR_INVALID_ARG;
  h->last_error[0] = 0;
  if (h->d != 2) return lerr(h, FV_ERR_UNSUPPORTED, "the learned correction is 2D");
  if (h->max_patch_size > fv::kLPmax) return lerr(h, FV_ERR_UNSUPPORTED, "patches > 16");
  if (n < 0) return lerr(h, FV_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return FV_OK;
  if (!q || !off || !sizes || !nbr || !params || !norm || !corr)
    return lerr(h, FV_ERR_INVALID_ARG, "null pointer");
  const int grid = (int)(n < (int64_t)h->num_sms * 8 ? n : (int64_t)h->num_sms * 8);
  const int64_t stride = fv::corr_stride_for(h->max_patch_size);
  if (h->prec == FV_FP64) {
    fv::MeshView<double> m{static_cast<const double*>(q), off, sizes, nbr, n, h->d_status};
    fv::corr_kernel<double><<<grid, fv::kLNT, 0, h->stream>>>(m, h->max_patch_size, params, norm,
                                                              corr, stride);
  } else {
    fv::MeshView<float> m{static_cast<const float*>(q), off, sizes, nbr, n, h->d_status};
    fv::corr_kernel<float><<<grid, fv::kLNT, 0, h->stream>>>(m, h->max_patch_size, params, norm,
                                                             corr, stride);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : lerr(h, FV_ERR_CUDA, cudaGetErrorString(e));
}

fv_status fv_restrict_mesh(fv_batch* hf, const void* qf, const int64_t* off_f, int pfx, int pfy,
                           fv_batch* hc, void* qc, const int64_t* off_c, int pcx, int pcy,
                           int ratio) {
  if (!hf || !hc || !qf || !qc || !off_f || !off_c || ratio < 1 || hf->d != 2 || hc->d != 2)
    return FV_ERR_INVALID_ARG;
  const fv::MeshGeom gf{hf->max_patch_size, pfx, pfy}, gc{hc->max_patch_size, pcx, pcy};
  if ((int64_t)pfx * gf.p != (int64_t)pcx * gc.p * ratio ||
      (int64_t)pfy * gf.p != (int64_t)pcy * gc.p * ratio || hf->prec != FV_FP64)
    return lerr(hc, FV_ERR_INVALID_ARG, "fine and coarse meshes do not match (or fine not FP64)");
  const int64_t ncell = (int64_t)pcx * pcy * gc.p * gc.p;
  if (hc->prec == FV_FP64)
    fv::restrict_kernel<double, double><<<grid_for_items(ncell), 256, 0, hc->stream>>>(
        static_cast<const double*>(qf), off_f, gf, static_cast<double*>(qc), off_c, gc, ratio);
  else
    fv::restrict_kernel<double, float><<<grid_for_items(ncell), 256, 0, hc->stream>>>(
        static_cast<const double*>(qf), off_f, gf, static_cast<float*>(qc), off_c, gc, ratio);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : lerr(hc, FV_ERR_CUDA, cudaGetErrorString(e));
}

fv_status fv_accumulate_face_flux(fv_batch* hf, const void* qf, const int64_t* off_f, int pfx,
                                  int pfy, fv_batch* hc, int pcx, int pcy, int ratio,
                                  double weight, double* acc) {
  if (!hf || !hc || !qf || !off_f || !acc || ratio < 1 || hf->d != 2 || hc->d != 2 ||
      hf->prec != FV_FP64)
    return FV_ERR_INVALID_ARG;
  const fv::MeshGeom gf{hf->max_patch_size, pfx, pfy}, gc{hc->max_patch_size, pcx, pcy};
  if ((int64_t)pfx * gf.p != (int64_t)pcx * gc.p * ratio ||
      (int64_t)pfy * gf.p != (int64_t)pcy * gc.p * ratio)
    return lerr(hc, FV_ERR_INVALID_ARG, "fine and coarse meshes do not match");
  const int64_t nfaces = (int64_t)pcx * pcy * 2 * (gc.p + 1) * gc.p;
  fv::accum_kernel<double><<<grid_for_items(nfaces), 256, 0, hf->stream>>>(
      static_cast<const double*>(qf), off_f, gf, gc, ratio, hf->gamma, weight, acc,
      fv::corr_stride_for(hc->max_patch_size));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : lerr(hc, FV_ERR_CUDA, cudaGetErrorString(e));
}

fv_status fv_correction_samples(fv_batch* hc, const void* qc, const int64_t* off,
                                const int32_t* sizes, const int32_t* nbr, int64_t n,
                                const double* acc, float* x_raw, float* t_raw) {
  if (!hc || !qc || !off || !sizes || !nbr || !acc || !x_raw || !t_raw || n < 1 || hc->d != 2 ||
      hc->prec != FV_FP64 || hc->max_patch_size > fv::kLPmax)
    return FV_ERR_INVALID_ARG;
  fv::MeshView<double> m{static_cast<const double*>(qc), off, sizes, nbr, n, hc->d_status};
  const int grid = (int)(n < (int64_t)hc->num_sms * 8 ? n : (int64_t)hc->num_sms * 8);
  fv::targets_kernel<double><<<grid, fv::kLNT, 0, hc->stream>>>(
      m, hc->max_patch_size, hc->gamma, acc, fv::corr_stride_for(hc->max_patch_size), x_raw,
      t_raw);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : lerr(hc, FV_ERR_CUDA, cudaGetErrorString(e));
}

fv_status fv_column_moments(const float* x, int64_t rows, int cols, double* sum, double* sumsq,
                            double* scratch, void* stream) {
  if (!x || !sum || !sumsq || !scratch || rows < 1 || cols < 1 || cols > 64)
    return FV_ERR_INVALID_ARG;
  const int64_t chunk = 65536;
  const int nb = (int)((rows + chunk - 1) / chunk);
  if (nb > 4096) return FV_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  fv::moments_kernel<<<nb, 64, 0, st>>>(x, rows, cols, chunk, scratch);
  fv::moments_finish_kernel<<<1, 64, 0, st>>>(scratch, nb, cols, sum, sumsq);
  return cudaGetLastError() == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_normalize_columns(float* x, int64_t rows, int cols, const float* mu, const float* sd,
                               void* stream) {
  if (!x || !sd || rows < 0 || cols < 1) return FV_ERR_INVALID_ARG;
  if (rows == 0) return FV_OK;
  fv::normalize_kernel<<<grid_for_items(rows * cols), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      x, rows, cols, mu, sd);
  return cudaGetLastError() == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

}  // extern "C"
