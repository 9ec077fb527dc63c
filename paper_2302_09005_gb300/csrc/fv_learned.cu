// fv_learned.cu -- the learned conservative face-flux correction on 2D patch
// meshes (an addition on top of the Rusanov flux of Eq. 4, not in the paper):
//
//   correction  every face of every patch gets C = sd_y * net((S - mu)/sd),
//               S the 4-cell stencil Q_{i-2..i+1} normal to the face in the
//               face's normal frame (rho, j_n, j_t, E), net the 16 -> 64 -> 64
//               -> 4 GELU network, evaluated 128 faces at a time on the
//               5th-generation tensor cores (tcgen05.mma, BF16 operands in
//               shared memory, FP32 accumulators in tensor memory; one thread
//               per face for the stencil, GELU and output).  The update
//               adds C to the face flux once per face, so both cells see the
//               same flux and the totals are conserved.  Every face is
//               evaluated once, and a face shared by two patches has its C
//               written into both patches' slots.
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
#include "fv_ptx.cuh"
#include "fv_tc.cuh"
#include "fv_x2.cuh"

namespace fv {

constexpr int kLNT = 128;  // threads per CTA of the learned kernels
// Clock cycles a CTA waits for its MMAs before it reports FV_ERR_TIMEOUT
// (about one second at 2 GHz).
constexpr long long kTcWaitLimit = 2000000000ll;
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
// Correction kernel: the network on the 5th-generation tensor cores
// ---------------------------------------------------------------------------
// Every face of the mesh is evaluated once.  A patch evaluates its low faces
// (b in [0, p) along each direction); the result of its face b = 0 is also
// the high face b = p of its low neighbour, and is written there too when
// the two patches name each other as neighbours along that direction (as on
// any regular mesh).  A patch evaluates its own high faces only where no
// neighbour does (walls, outflow, or a neighbour table that is not
// symmetric).  The faces are enumerated as slots in two ranges:
//   A: patch * 2 pmax^2 + lf, lf = k p^2 + p b + tr (b < p);
//   B: (after A) patch * 2 pmax + k p + tr, the high faces b = p, idle
//      unless the patch itself must evaluate them.
// A CTA of 256 threads takes tiles of 128 slots (idle slots are idle rows),
// in two warp groups:
//   producers (warps 4-7)  thread 128 + t gathers the stencil of row t of the
//                          next tile, normalises it into row t of that tile's
//                          A1 buffer (BF16, K-major, two buffers) and records
//                          where the row's result goes; whether the tile has
//                          any active row is reduced over the producers, and
//                          the consumers skip tiles that have none;
//   consumers (warps 0-3)  thread 0 issues the MMAs (tcgen05, FP32
//                          accumulators in tensor memory, D row t = TMEM lane
//                          t, which warp t / 32 may read); thread t reads its
//                          row back, applies GELU and writes row t of the next
//                          layer's A operand:
//   D1 = A1[128x16] W1^T (N = 64), D2 = A2[128x80] W2'^T (N = 64),
//   D3 = A2[128x80] W3'^T (N = 16, rows 4..15 of W3' zero).
// The biases of layers 2 and 3 ride in the products: columns 64, 65 of A2
// are ones, and the matching columns of the weight tiles hold the bias split
// into two BF16 parts (b = hi + lo to about 2^-17 of b); layer 1 adds its
// bias in FP32.  The GELU layers
// write 2 gelu(z) = z (1 + tanh(u)) (one FMA after the tanh) and W2', W3'
// hold W2 / 2, W3 / 2: the same products, exactly, as gelu(z) with W.
// The stencil loads of one tile (through the neighbour table) overlap the
// MMA / GELU chain of the previous one.  Named barriers hand the A1 buffers
// over: FULL[b] (producers arrive, consumers wait) and EMPTY[b] (consumers
// arrive once the MMA that read the buffer has completed, producers wait).
// D1, D2 and D3 share 64 TMEM columns; A2 serves layers 2 and 3 (each MMA has
// completed before its operands are overwritten).
constexpr int kTcRows = 128;  // faces per tile: the MMA's M
constexpr int kTcCols = 64;   // TMEM columns of a CTA
constexpr int kCorrNT = 256;  // consumers + producers
constexpr int kK1 = 16;       // layer-1 K: the 16 inputs
constexpr int kK2 = 80;       // layers 2, 3 K: 64 hidden, two ones columns, zeros

// Where a staged tile's patch and its two halo layers come from (the rules
// of cell_source, resolved once per patch): its size and offset; per side f
// (-x, +x, -y, +y) the source patch's offset, how the side is filled
// (0: neighbour, 1: outflow copy, 2: wall mirror) and the neighbour index;
// per direction whether the low neighbour names the patch back (it then
// takes the face b = 0 into its high-face slot).
struct alignas(8) CRec {
  long long off;
  long long soff[4];
  int p;
  int mode[4];
  int nb[4];
  int extok[2];
  unsigned rp1, rp2;  // ceil(2^16 / p), ceil(2^16 / 2p): x / p = (x rp1) >> 16
};

struct TcSmem {
  alignas(128) unsigned char a1[2][kTcRows * kK1 * 2];
  alignas(128) unsigned char a2[kTcRows * kK2 * 2];
  alignas(128) unsigned char w1[64 * kK1 * 2];
  alignas(128) unsigned char w2[64 * kK2 * 2];
  alignas(128) unsigned char w3[16 * kK2 * 2];
  alignas(16) float b1[64];
  float2 murs[16];  // per input: mean, 1 / standard deviation
  float sdy[4];
  int fpid[2][kTcRows];  // patch of each row's face, or -1 (idle row)
  int fext[2][kTcRows];  // low neighbour that shares the face (b = 0), or -1
  int fkj[2][kTcRows];   // j | nf1 << 10 | k << 20
  int fany[2];           // whether the tile has an active row
  CRec prec[2];          // the staged tiles' patch records (this tile, the next)
  alignas(8) uint64_t bar;
  uint32_t tmem;
};

// Named barriers (0 is __syncthreads): FULL[b], EMPTY[b], the consumers',
// the producers' reduction.
constexpr int kBarFull = 1, kBarEmpty = 3, kBarCons = 5, kBarProd = 7;
__device__ __forceinline__ void nbar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Barrier over n threads that also returns whether any of them passed true.
__device__ __forceinline__ bool nbar_or(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
      "barrier.cta.red.or.pred p, %1, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(id), "r"((uint32_t)v), "r"(n)
      : "memory");
  return r != 0;
}

// A stencil value as float.  FP64 states are narrowed by repacking the bits
// with integer operations (sign, rebased exponent, leading 23 fraction bits;
// truncation, values outside the float range flushed to 0 / infinity):
// the FP64 pipe, which the conversion instruction would use, is the scarce
// unit of this GPU, and the value is rounded to BF16 next anyway (2^-8 vs the
// 2^-23 of the truncation).
__device__ __forceinline__ float narrow(float v) { return v; }
__device__ __forceinline__ float narrow(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  const unsigned sign = hi & 0x80000000u;
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned bits = sign | ((unsigned)e << 23) | mant;
  bits = e <= 0 ? sign : bits;
  bits = e >= 255 ? (sign | 0x7F800000u) : bits;
  return __uint_as_float(bits);
}

__device__ __forceinline__ void store_bf16x8(unsigned char* dst, const float* v) {
  uint4 u;
  u.x = pack_bf16(v[0], v[1]);
  u.y = pack_bf16(v[2], v[3]);
  u.z = pack_bf16(v[4], v[5]);
  u.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(dst) = u;
}

// 2 gelu(z) on two values with the packed FP32 instructions, in the tanh form
// of gelu_f (fv_mma.cuh): u = z (c1 + c3 z^2), 2 gelu(z) = z + z tanh(u).
// Each half is rounded as the scalar operation would be; the tanh is one
// special-function instruction per value.
__device__ __forceinline__ f2 gelu2x2(f2 z) {
  const f2 c3 = f2_pack(0.0356774081f, 0.0356774081f), c1 = f2_pack(0.7978845608f, 0.7978845608f);
  const f2 u = mul2(z, fma2(c3, mul2(z, z), c1));
  float ul, uh;
  f2_unpack(u, ul, uh);
  return fma2(z, f2_pack(tanh_hw(ul), tanh_hw(uh)), z);
}

// Row `row` of a 64-wide hidden layer: TMEM accumulators (+ bias, where the
// product does not carry it) -> 2 gelu -> BF16 into columns 0..63 of the
// K-major A2 tile.
template <bool BIAS>
__device__ __forceinline__ void hidden_row(uint32_t trow, unsigned char* a, int row,
                                           const float* bias) {
#pragma unroll
  for (int c = 0; c < 64; c += 16) {
    float v[16];
    tc_ld16(trow + c, v);
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      f2 z = f2_pack(v[i], v[i + 1]);
      if (BIAS) z = add2(z, *reinterpret_cast<const f2*>(bias + c + i));
      const f2 g = gelu2x2(z);
      f2_unpack(g, v[i], v[i + 1]);
    }
    store_bf16x8(a + tc_kmajor_offset(row, c, kK2), v);
    store_bf16x8(a + tc_kmajor_offset(row, c + 8, kK2), v + 8);
  }
}

// Consumers: operands visible to the tensor cores, TMEM reads done; then
// thread 0 issues.
__device__ __forceinline__ void tc_handoff_cons() {
  fence_proxy_async_smem();
  tc_fence_before_sync();
  nbar_sync(kBarCons, kTcRows);
  tc_fence_after_sync();
}

// BF16 parts of a bias: b ~ hi + lo.
__device__ __forceinline__ void bias_parts(float b, uint16_t& hi, uint16_t& lo) {
  hi = f32_to_bf16(b);
  lo = f32_to_bf16(b - bf16_to_f32(hi));
}

// Slot decoding of one range: (pid, lf) = divmod(slot, per) advanced by the
// CTA stride each tile instead of divided anew.
struct SlotWalk {
  int64_t pid;
  int lf;
  int64_t qstep;
  int rstep;
  int per;
  __device__ __forceinline__ void init(int64_t slot, int per_, int64_t sstep) {
    per = per_;
    pid = slot / per;
    lf = (int)(slot - pid * per);
    qstep = sstep / per;
    rstep = (int)(sstep - qstep * per);
  }
  __device__ __forceinline__ void advance() {
    pid += qstep;
    lf += rstep;
    if (lf >= per) {
      lf -= per;
      ++pid;
    }
  }
};

// Stage of patch pid for the correction kernel's producers (thread `t` of
// `nt`): its interior and the two cell layers beyond each face, narrowed to
// float, one float4 per cell at (X, Y) = (x + 1, y + 1), X, Y in [0, p + 4).
template <typename T>
__device__ __forceinline__ void stage_patch(const MeshView<T>& m, int64_t pid, int p,
                                            float4* stage, int t, int nt) {
  const int ns = p + 4;
  const int total = p * p + 8 * p;  // interior, then 4 sides x 2 layers x p
  for (; t < total; t += nt) {
    int x, y;
    if (t < p * p) {
      y = t / p;
      x = 1 + t - y * p;
      ++y;
    } else {
      const int u = t - p * p;
      const int side4 = u / (2 * p);  // 0: -x, 1: +x, 2: -y, 3: +y
      const int r = u - side4 * 2 * p;
      const int layer = r / p;  // 0: next to the face, 1: beyond
      const int tr = 1 + r - layer * p;
      const int c = (side4 & 1) ? p + 1 + layer : -layer;
      if (side4 < 2) { x = c; y = tr; } else { x = tr; y = c; }
    }
    int neg;
    const T* src = cell_source(m, pid, p, x, y, neg);
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (u == neg) ? -narrow(src[u]) : narrow(src[u]);
    stage[(y + 1) * ns + (x + 1)] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// A staged tile's patch record in two dependent load steps, one per
// iteration of the producer loop, by the producer rows f = 0 .. 3 (side f):
// step 1, the patch's size and offset and its neighbour across side f; step
// 2, the neighbour's size and offset and its own neighbour back across the
// shared face.  Indices are clamped to valid entries, so every load is in
// bounds; corr_rec_finish applies cell_source's rules to the values.
struct CL1 {
  long long off;
  int64_t pid;
  int p, nb;
};
struct CL2 {
  long long onb;
  int snb, back;
};
template <typename T>
__device__ __forceinline__ CL1 corr_l1(const MeshView<T>& m, int64_t pid, int f) {
  CL1 r{0, pid, 0, -1};
  if (pid >= 0) {
    r.p = m.sizes[pid];
    r.off = m.off[pid];
    r.nb = m.nbr[pid * 4 + f];
  }
  return r;
}
template <typename T>
__device__ __forceinline__ CL2 corr_l2(const MeshView<T>& m, const CL1& a, int f) {
  CL2 r{0, 0, -1};
  if (a.pid >= 0) {
    const int64_t nc = (a.nb >= 0 && a.nb < m.n) ? (int64_t)a.nb : a.pid;
    r.snb = m.sizes[nc];
    r.onb = m.off[nc];
    r.back = m.nbr[nc * 4 + (f | 1)];
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void corr_rec_finish(const MeshView<T>& m, const CL1& a, const CL2& b,
                                                int f, int pmax, CRec* rec) {
  if (a.pid < 0) return;
  if (f == 0) {
    rec->p = a.p;
    rec->off = a.off;
    const unsigned pp = a.p >= 1 ? (unsigned)a.p : 1u;
    rec->rp1 = (65536u + pp - 1u) / pp;
    rec->rp2 = (65536u + 2u * pp - 1u) / (2u * pp);
  }
  const bool valid = a.nb >= 0 && a.nb < m.n && b.snb == a.p;
  if (!valid && a.nb != -1 && a.nb != -2 && a.p >= 1 && a.p <= pmax)
    atomicOr(m.status, ST_BAD_PATCH);
  rec->soff[f] = valid ? b.onb : a.off;
  rec->mode[f] = valid ? 0 : (a.nb == -2 ? 2 : 1);
  rec->nb[f] = a.nb;
  if ((f & 1) == 0) rec->extok[f >> 1] = (valid && b.back == (int)a.pid) ? 1 : 0;
}

// stage_patch from a patch record: the same cells, the same values.  The
// quotients by p and 2p are products with the record's rounded-up
// reciprocals, exact for the dividends here (below 8 p + p^2 <= 384): with
// r = ceil(2^16 / q) = (2^16 + e) / q, e < q <= 32, (x r) >> 16 = floor(x / q)
// whenever x e < 2^16.
template <typename T>
__device__ __forceinline__ void stage_patch_rec(const MeshView<T>& m, const CRec& rec,
                                                float4* stage, int t, int nt) {
  const int p = rec.p, ns = p + 4;
  const int total = p * p + 8 * p;  // interior, then 4 sides x 2 layers x p
  const unsigned rp1 = rec.rp1, rp2 = rec.rp2;
  for (; t < total; t += nt) {
    int x, y, neg = -1;
    long long so = rec.off;
    if (t < p * p) {
      y = (int)(((unsigned)t * rp1) >> 16);  // t / p
      x = 1 + t - y * p;
      ++y;
    } else {
      const int u = t - p * p;
      const int side4 = (int)(((unsigned)u * rp2) >> 16);  // u / 2p; 0: -x, 1: +x, 2: -y, 3: +y
      const int r = u - side4 * 2 * p;
      const int layer = (int)(((unsigned)r * rp1) >> 16);  // r / p; 0: next to the face, 1: beyond
      const int tr = 1 + r - layer * p;
      const int side = side4 & 1, depth = layer + 1;
      const int mode = rec.mode[side4];
      int along;
      if (mode == 0) {  // the neighbour's interior
        so = rec.soff[side4];
        along = side ? depth : p + 1 - depth;
      } else if (mode == 2) {  // wall: mirror image
        along = side ? p + 1 - depth : depth;
        neg = 1 + (side4 >> 1);
      } else {  // outflow: nearest interior cell
        along = side ? p : 1;
      }
      if (side4 < 2) { x = along; y = tr; } else { x = tr; y = along; }
      // the staged position: the cell beyond the face
      const int c = side ? p + 1 + layer : -layer;
      const T* src = m.q + so + ((int64_t)y * (p + 2) + x) * 4;
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = (q == neg) ? -narrow(src[q]) : narrow(src[q]);
      if (side4 < 2) stage[(tr + 1) * ns + (c + 1)] = make_float4(v[0], v[1], v[2], v[3]);
      else stage[(c + 1) * ns + (tr + 1)] = make_float4(v[0], v[1], v[2], v[3]);
      continue;
    }
    const T* src = m.q + so + ((int64_t)y * (p + 2) + x) * 4;
    stage[(y + 1) * ns + (x + 1)] =
        make_float4(narrow(src[0]), narrow(src[1]), narrow(src[2]), narrow(src[3]));
  }
}

// Whether patch q is a valid neighbour of size p that names `back` as its
// neighbour on side `side` of direction k.
template <typename T>
__device__ __forceinline__ bool links_back(const MeshView<T>& m, int64_t q, int p, int k,
                                           int side, int64_t back) {
  return q >= 0 && q < m.n && m.sizes[q] == p && m.nbr[q * 4 + 2 * k + side] == back;
}

template <typename T>
__global__ void __launch_bounds__(kCorrNT, 4)
    corr_kernel(MeshView<T> m, int pmax, const float* params, const float* norm, float* corr,
                int64_t stride) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw);
  float4* stage = reinterpret_cast<float4*>(smem_raw + sizeof(TcSmem));  // (pmax + 4)^2 cells
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights (BF16, K-major tiles) with the biases in the columns that meet
  // the ones of the A operands; W2, W3 halved for the 2 gelu of the layers
  // before them
  for (int i = tid; i < 64 * kK1; i += kCorrNT)
    *reinterpret_cast<uint16_t*>(s.w1 + tc_kmajor_offset(i >> 4, i & 15, kK1)) =
        f32_to_bf16(params[kOffW1 + i]);
  if (tid < 64) s.b1[tid] = params[kOffB1 + tid];
  for (int i = tid; i < 64 * kK2; i += kCorrNT) {
    const int r = i / kK2, c = i - r * kK2;
    uint16_t v = 0, hi, lo;
    if (c < 64) v = f32_to_bf16(0.5f * bf16_to_f32(f32_to_bf16(params[kOffW2 + r * 64 + c])));
    if (c == 64 || c == 65) {
      bias_parts(params[kOffB2 + r], hi, lo);
      v = c == 64 ? hi : lo;
    }
    *reinterpret_cast<uint16_t*>(s.w2 + tc_kmajor_offset(r, c, kK2)) = v;
  }
  for (int i = tid; i < 16 * kK2; i += kCorrNT) {
    const int r = i / kK2, c = i - r * kK2;
    uint16_t v = 0, hi, lo;
    if (r < 4 && c < 64)
      v = f32_to_bf16(0.5f * bf16_to_f32(f32_to_bf16(params[kOffW3 + r * 64 + c])));
    if (r < 4 && (c == 64 || c == 65)) {
      bias_parts(params[kOffB3 + r], hi, lo);
      v = c == 64 ? hi : lo;
    }
    *reinterpret_cast<uint16_t*>(s.w3 + tc_kmajor_offset(r, c, kK2)) = v;
  }
  // the constant columns of A2: ones at 64, 65, zeros after them
  for (int r = tid; r < kTcRows; r += kCorrNT) {
    *reinterpret_cast<uint4*>(s.a2 + tc_kmajor_offset(r, 64, kK2)) =
        make_uint4(0x3F803F80u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(s.a2 + tc_kmajor_offset(r, 72, kK2)) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid < 4) s.sdy[tid] = norm[32 + tid];
  if (tid < 16) s.murs[tid] = make_float2(norm[tid], 1.0f / norm[16 + tid]);
  if (tid == 0) {
    mbar_init(&s.bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(&s.tmem, kTcCols);
  fence_proxy_async_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tm = s.tmem;
  const int perA = 2 * pmax * pmax, perB = 2 * pmax;
  const int64_t nA = m.n * perA, nB = m.n * perB;
  const int64_t tilesA = (nA + kTcRows - 1) / kTcRows;
  const int64_t ntiles = tilesA + (nB + kTcRows - 1) / kTcRows;
  // every tile of range A lies within the slots of one patch
  const bool staged = perA % kTcRows == 0;
  constexpr uint32_t kId64 = tc_idesc_bf16(kTcRows, 64), kId16 = tc_idesc_bf16(kTcRows, 16);
  bool failed = false;

  if (warp >= 4) {
    // ---- producers: stencils of the tiles, one tile ahead of the consumers
    const int row = tid - kTcRows;
    const int64_t sstep = (int64_t)gridDim.x * kTcRows;
    SlotWalk wa, wb;
    wa.init((int64_t)blockIdx.x * kTcRows + row, perA, sstep);
    wb.init(0, perB, sstep);
    bool in_b = false;
    int pcur = 0, rp = 0;  // the patch size rp is for: ceil(2^16 / p), x / p = (x rp) >> 16
    int it = 0;
    // the staged tiles' patch records: this tile's ready, the next one's in
    // two load steps over this iteration and the one before (rows 0 .. 3)
    const int64_t gstep = gridDim.x;
    auto tile_pid = [&](int64_t tl) -> int64_t {  // the patch of a staged tile, else -1
      return (staged && tl < tilesA) ? tl * kTcRows / perA : -1;
    };
    CL1 l1n{0, -1, 0, -1};  // step 1 of the next tile's patch
    if (row < 4) {
      const CL1 a0 = corr_l1(m, tile_pid(blockIdx.x), row);
      corr_rec_finish(m, a0, corr_l2(m, a0, row), row, pmax, &s.prec[0]);
      l1n = corr_l1(m, tile_pid(blockIdx.x + gstep), row);
    }
    nbar_sync(kBarProd, kTcRows);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int b = it & 1;
      if (it >= 2) nbar_sync(kBarEmpty + b, kCorrNT);
      CL2 l2n{0, 0, -1};
      CL1 l1nn{0, -1, 0, -1};
      if (row < 4) {
        l2n = corr_l2(m, l1n, row);                          // step 2, the next tile
        l1nn = corr_l1(m, tile_pid(tile + 2 * gstep), row);  // step 1, the one after
      }
      const CRec& rec = s.prec[it & 1];
      if (tile >= tilesA && !in_b) {
        in_b = true;
        wb.init((tile - tilesA) * kTcRows + row, perB, sstep);
      }
      const int64_t slot = in_b ? (tile - tilesA) * kTcRows + row : tile * kTcRows + row;
      const int64_t pid = in_b ? wb.pid : wa.pid;
      const int lf = in_b ? wb.lf : wa.lf;
      bool act = slot < (in_b ? nB : nA);
      int p = 1, nf1 = 2, k = 0, j = 0, bb = 0, tr = 0;
      int ext = -1;
      if (act) {
        p = (staged && !in_b) ? rec.p : m.sizes[pid];
        if (p < 1 || p > pmax) {
          if (lf == 0) atomicOr(m.status, ST_BAD_PATCH);
          act = false;
        } else if (!in_b) {  // a low face, b < p
          act = lf < 2 * p * p;
          if (act) {
            k = lf >= p * p ? 1 : 0;
            const int jj = lf - k * p * p;
            if (p != pcur) {
              pcur = p;
              rp = (65536 + p - 1) / p;  // exact for jj < 2^16 / 16 and p <= 16
            }
            bb = (jj * rp) >> 16;
            tr = jj - bb * p;
          }
        } else {  // a high face, b = p: only where no neighbour evaluates it
          act = lf < 2 * p;
          if (act) {
            k = lf >= p ? 1 : 0;
            tr = lf - k * p;
            bb = p;
            act = !links_back(m, (int64_t)m.nbr[pid * 4 + 2 * k + 1], p, k, 0, pid);
          }
        }
        if (act) {
          nf1 = (p + 1) * p;
          j = tr + p * bb;
          if (bb == 0) {  // also the high face of the low neighbour
            if (staged && !in_b) {
              if (rec.extok[k]) ext = rec.nb[2 * k];
            } else {
              const int64_t nl = m.nbr[pid * 4 + 2 * k];
              if (links_back(m, nl, p, k, 1, pid)) ext = (int)nl;
            }
          }
        }
      }
      // normalised stencil Q_{b-1..b+2} in the face's normal frame -> A1 row
      float x[16];
      if (staged && !in_b) {
        // the tile's rows are the low faces of one patch: its cells and
        // halo layers are staged once, every stencil read from there
        if (p >= 1 && p <= pmax && slot < nA) stage_patch_rec(m, rec, stage, row, kTcRows);
        nbar_sync(kBarProd, kTcRows);
        const int ns = p + 4;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
          if (act) q4 = stage[k == 0 ? (tr + 2) * ns + (bb + c) : (bb + c) * ns + (tr + 2)];
          const float vn4[4] = {q4.x, k ? q4.z : q4.y, k ? q4.y : q4.z, q4.w};
#pragma unroll
          for (int vn = 0; vn < 4; ++vn) {
            const float2 mr = s.murs[4 * c + vn];
            x[4 * c + vn] = act ? (vn4[vn] - mr.x) * mr.y : 0.f;
          }
        }
      } else {
      // faces whose four cells lie inside the patch read them straight from
      // its block, the others through the neighbour table
      const bool inner = act && bb >= 2 && bb + 2 <= p;
      const T* cin = nullptr;
      int sal = 0;  // elements between neighbouring cells along the normal
      if (inner) {
        const int ne = p + 2;
        cin = m.q + m.off[pid] +
              (k == 0 ? ((tr + 1) * ne + (bb - 1)) * 4 : ((bb - 1) * ne + (tr + 1)) * 4);
        sal = k == 0 ? 4 : ne * 4;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (inner) {
          const T* src = cin + c * sal;
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = narrow(src[u]);
        } else if (act) {
          const int along = bb - 1 + c;
          int neg;
          const T* src = cell_source(m, pid, p, k == 0 ? along : tr + 1,
                                     k == 0 ? tr + 1 : along, neg);
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = (u == neg) ? -narrow(src[u]) : narrow(src[u]);
        }
        // normal frame: the momenta swap places for y faces (selects, not
        // a runtime index, which would put v in local memory)
        const float vn4[4] = {v[0], k ? v[2] : v[1], k ? v[1] : v[2], v[3]};
#pragma unroll
        for (int vn = 0; vn < 4; ++vn) {
          const float2 mr = s.murs[4 * c + vn];
          x[4 * c + vn] = act ? (vn4[vn] - mr.x) * mr.y : 0.f;
        }
      }
      }
      store_bf16x8(s.a1[b] + tc_kmajor_offset(row, 0, kK1), x);
      store_bf16x8(s.a1[b] + tc_kmajor_offset(row, 8, kK1), x + 8);
      s.fpid[b][row] = act ? (int)pid : -1;
      s.fext[b][row] = ext;
      s.fkj[b][row] = j | (nf1 << 10) | (k << 20) | (p << 21);
      fence_proxy_async_smem();
      if (row < 4) {  // the next tile's record, read after the barrier below
        corr_rec_finish(m, l1n, l2n, row, pmax, &s.prec[(it + 1) & 1]);
        l1n = l1nn;
      }
      const bool any = nbar_or(kBarProd, kTcRows, act);
      if (row == 0) s.fany[b] = any ? 1 : 0;
      nbar_arrive(kBarFull + b, kCorrNT);
      if (in_b) wb.advance(); else wa.advance();
    }
  } else {
    // ---- consumers: the network on the tensor cores, one row per thread
    const uint32_t trow = tm + ((uint32_t)(warp * 32) << 16);  // this warp's TMEM lanes
    uint32_t parity = 0;
    int it = 0;
    auto mma_wait = [&]() {
      failed |= !mbar_wait_sleep(&s.bar, parity, kTcWaitLimit);
      parity ^= 1u;
      tc_fence_after_sync();
    };
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int b = it & 1;
      tc_fence_before_sync();
      nbar_sync(kBarFull + b, kCorrNT);  // A1[b] written (and the last tile's D3 read)
      tc_fence_after_sync();
      const bool refill = tile + 2 * gridDim.x < ntiles;
      // this row's destination, read before buffer b is handed back
      const int pid = s.fpid[b][tid], ext = s.fext[b][tid], fkj = s.fkj[b][tid];
      if (s.fany[b] == 0) {  // no face of this tile is evaluated here
        if (refill) nbar_arrive(kBarEmpty + b, kCorrNT);
        continue;
      }
      const bool run = !failed;  // a wait that gave up stops the tensor work
      // ---- layer 1: 16 -> 64 (+ bias)
      if (tid == 0 && run) {
        tc_mma_bf16(tm, tc_smem_desc(s.a1[b], 128, kK1 * 16), tc_smem_desc(s.w1, 128, kK1 * 16),
                    kId64, 0);
        tc_commit(&s.bar);
      }
      if (run) mma_wait();
      // A1[b] has been read: the producers may refill it (if they will)
      if (refill) nbar_arrive(kBarEmpty + b, kCorrNT);
      if (run) hidden_row<true>(trow, s.a2, tid, s.b1);
      tc_handoff_cons();
      // ---- layer 2: 64 (+ bias) -> 64
      if (tid == 0 && run && !failed) {
#pragma unroll
        for (int kk = 0; kk < kK2 / 16; ++kk)
          tc_mma_bf16(tm, tc_smem_desc(s.a2 + kk * 256, 128, kK2 * 16),
                      tc_smem_desc(s.w2 + kk * 256, 128, kK2 * 16), kId64, kk > 0);
        tc_commit(&s.bar);
      }
      if (run) mma_wait();
      if (run) hidden_row<false>(trow, s.a2, tid, nullptr);
      tc_handoff_cons();
      // ---- layer 3: 64 (+ bias) -> 4 (N = 16)
      if (tid == 0 && run && !failed) {
#pragma unroll
        for (int kk = 0; kk < kK2 / 16; ++kk)
          tc_mma_bf16(tm, tc_smem_desc(s.a2 + kk * 256, 128, kK2 * 16),
                      tc_smem_desc(s.w3 + kk * 256, 128, kK2 * 16), kId16, kk > 0);
        tc_commit(&s.bar);
      }
      if (run) mma_wait();
      float y[4] = {0.f, 0.f, 0.f, 0.f};
      if (run) tc_ld4(trow, y);
      if (run && pid >= 0) {
        const int j = fkj & 1023, nf1 = (fkj >> 10) & 1023, k = (fkj >> 20) & 1, p = fkj >> 21;
#pragma unroll
        for (int vn = 0; vn < 4; ++vn) {
          const float c = y[vn] * s.sdy[vn];
          const int64_t col = (int64_t)(k * 4 + phys_comp(k, vn)) * nf1;
          corr[(int64_t)pid * stride + col + j] = c;
          if (ext >= 0) corr[(int64_t)ext * stride + col + j + p * p] = c;
        }
      }
    }
  }
  // a wait that gave up: report; the TMEM is released either way
  if (failed) atomicOr(m.status, ST_TIMEOUT);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tc_dealloc(tm, kTcCols);
}

// Dynamic shared memory of corr_kernel for patches up to pmax: the fixed part
// and the patch stage.
inline size_t corr_smem_bytes(int pmax) {
  return sizeof(TcSmem) + (size_t)(pmax + 4) * (pmax + 4) * 16;
}

// Dynamic shared memory of corr_kernel<T> raised once per device.
template <typename T>
cudaError_t corr_smem_attr() {
  static int set[64] = {0};
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(corr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)corr_smem_bytes(kLPmax));
  // four CTAs per SM need the largest shared-memory carveout
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(corr_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && dev >= 0 && dev < 64) set[dev] = 1;
  return e;
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
  if (n > 0x7FFFFFFFll) return lerr(h, FV_ERR_UNSUPPORTED, "more than 2^31 - 1 patches");
  const int64_t stride = fv::corr_stride_for(h->max_patch_size);
  // tiles of 128 face slots (the low faces, then the high faces); up to four
  // CTAs of 256 threads per SM (registers and shared memory; 4 x 64 TMEM
  // columns of 512)
  const int64_t pm = h->max_patch_size;
  const int64_t ntiles = (n * 2 * pm * pm + fv::kTcRows - 1) / fv::kTcRows +
                         (n * 2 * pm + fv::kTcRows - 1) / fv::kTcRows;
  const int64_t gmax = (int64_t)h->num_sms * 4;
  const int grid = (int)(ntiles < gmax ? ntiles : gmax);
  const size_t smem = fv::corr_smem_bytes(h->max_patch_size);
  cudaError_t e;
  if (h->prec == FV_FP64) {
    e = fv::corr_smem_attr<double>();
    fv::MeshView<double> m{static_cast<const double*>(q), off, sizes, nbr, n, h->d_status};
    if (e == cudaSuccess)
      fv::corr_kernel<double><<<grid, fv::kCorrNT, smem, h->stream>>>(m, h->max_patch_size,
                                                                      params, norm, corr, stride);
  } else {
    e = fv::corr_smem_attr<float>();
    fv::MeshView<float> m{static_cast<const float*>(q), off, sizes, nbr, n, h->d_status};
    if (e == cudaSuccess)
      fv::corr_kernel<float><<<grid, fv::kCorrNT, smem, h->stream>>>(m, h->max_patch_size,
                                                                     params, norm, corr, stride);
  }
  if (e != cudaSuccess) return lerr(h, FV_ERR_CUDA, cudaGetErrorString(e));
  e = cudaGetLastError();
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
