// fv_rows2d.cu -- the FP32 time step / update of a launch whose patches all
// have one 2D size (p = 5: a size class of the schedule, or a uniform batch
// after fv_batch_plan), one lane per row of cells.  Same method, same
// operations in the same order as the general kernel (fv_step.cuh; Eq. 2-5,
// Algorithm 1 steps 5-10), so the results are bitwise the same.
//
// A warp advances four patches at a time, eight lanes each: lane r of a group
// holds row y = r of its patch box (r = 0 and r = p + 1 the face-halo rows,
// lane 7 idle).  Everything stays in registers; no shared memory, no block
// barrier:
//
//  * loads: an interior row reads its p cells with 16-byte loads, and its two
//    x-halo cells from their sources (the own halo layer in update mode; in a
//    time step the neighbour's interior layer next to the face, a wall's
//    mirror or the outflow copy); a face-halo row reads the p cells of its
//    source row.  The patch box is read once, in whole rows; where the rows
//    come from (patch, neighbours) is resolved one iteration ahead;
//  * primitives of every cell of the row (Eq. 2);
//  * x faces: an interior row walks its p + 1 faces left to right and keeps
//    each cell's x flux difference;
//  * y faces: lane r takes the face between rows r and r + 1 of every column,
//    the upper cells' state and primitives by warp shuffle from lane r + 1;
//  * update: an interior row receives the fluxes of the faces below it from
//    lane r - 1 (shuffle), adds the y differences to its x differences (x then
//    y), takes one FMA with -dt / (2 dx), stores its p cells with 16-byte
//    stores and, in a time step, converts them for the next CFL maximum.
#include "fv_step.cuh"

// Resident CTAs of 128 threads per SM the register allocation is sized for.
#ifndef FV_ROWS2D_MINBLOCKS
#define FV_ROWS2D_MINBLOCKS 4
#endif

namespace fv {
namespace {

constexpr int kRowsNT = 128;     // threads per CTA: four independent warps
constexpr int kRowsGroup = 8;    // lanes per patch
constexpr int kRowsPerWarp = 4;  // patches per warp and iteration

__device__ __forceinline__ unsigned umax_u(unsigned a, unsigned b) { return a > b ? a : b; }
// |u| + c of a cell as its IEEE bits (>= 0 or NaN, so unsigned maxima order
// them like the values)
__device__ __forceinline__ unsigned wave_bits_f(float u, float c) {
  return __float_as_uint(add_rn(fabsf(u), c));
}
constexpr unsigned kMag = 0x7FFFFFFFu;
// positivity of rho and p accumulated as max(bits - 1): 0 < x < inf <=>
// bits(x) - 1 < 0x7F7FFFFF
constexpr unsigned kBad = 0x7F7FFFFFu;

// State and primitives of one cell: rho, j_x, j_y, E; u_x, u_y, p, c, E + p.
struct RCell {
  float q[4];
  float u[2], p, c, e;
};

// Primitives (Eq. 2) with the operations, in order, of primitives<float, 2>()
// of the general kernel; `need` keeps non-cells out of the positivity check.
__device__ __forceinline__ void rprims(RCell& x, float gm1, float gamma, bool need,
                                       unsigned& chk) {
  const float inv = recip(x.q[0]);
  x.u[0] = mul_rn(x.q[1], inv);
  x.u[1] = mul_rn(x.q[2], inv);
  float jj = mul_rn(x.q[1], x.u[0]);
  jj = fmaf(x.q[2], x.u[1], jj);
  x.p = mul_rn(gm1, fmaf(-0.5f, jj, x.q[3]));
  x.e = add_rn(x.q[3], x.p);
  x.c = sqrt_t(mul_rn(mul_rn(gamma, x.p), inv));
  const unsigned m = need ? ~0u : 0u;
  chk = umax_u(chk, (__float_as_uint(x.q[0]) - 1u) & m);
  chk = umax_u(chk, (__float_as_uint(x.p) - 1u) & m);
}

// G = 2F of one face along k (Eq. 4, 5) in the general kernel's operation
// order: g[v] for the unknowns v (rho, j_x, j_y, E); returns the bits of a.
template <int K>
__device__ __forceinline__ unsigned rflux(const RCell& L, const RCell& R, float (&g)[4]) {
  constexpr int N = 1 + K, T = 2 - K;  // normal and transverse momentum
  const unsigned ab = umax_u(wave_bits_f(L.u[K], L.c), wave_bits_f(R.u[K], R.c));
  const float am = __uint_as_float(ab);
  const float sL = add_rn(L.u[K], am), sR = sub_rn(R.u[K], am), ps = add_rn(L.p, R.p);
  g[0] = fmaf(L.q[0], sL, mul_rn(R.q[0], sR));
  g[T] = fmaf(L.q[T], sL, mul_rn(R.q[T], sR));
  g[N] = fmaf(L.q[N], sL, fmaf(R.q[N], sR, ps));
  g[3] = fmaf(am, sub_rn(L.q[3], R.q[3]), fmaf(L.e, L.u[K], mul_rn(R.e, R.u[K])));
  return ab;
}

__device__ __forceinline__ void ld_cell(RCell& x, const float* src, int negc) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(src));
  x.q[0] = v.x;
  x.q[1] = negc == 1 ? neg_t(v.y) : v.y;
  x.q[2] = negc == 2 ? neg_t(v.z) : v.z;
  x.q[3] = v.w;
}

// Where one lane's row comes from: the patch, and the sources of its halo
// cells (an interior row: faces -x, +x; a face-halo row: its face).
struct RowMeta {
  int64_t pid, off;
  long long s0, s1;  // source patch offsets
  int ck0, ck1;      // source layers along the face normal
  int neg0, neg1;    // wall: the normal momentum mirrored
  bool act;          // the patch is valid
};

__device__ __forceinline__ float shfl_dn(float v) { return __shfl_down_sync(0xFFFFFFFFu, v, 1); }
__device__ __forceinline__ float shfl_up(float v) { return __shfl_up_sync(0xFFFFFFFFu, v, 1); }

template <int P, bool STEP>
__global__ void __launch_bounds__(kRowsNT, FV_ROWS2D_MINBLOCKS) rows2d_kernel(StepParams<float> a) {
  constexpr int S = 4, NE = P + 2;
  static_assert(NE <= kRowsGroup, "a patch's rows fit one lane group");
  const int lane = threadIdx.x & 31;
  const int grp = lane >> 3, r = lane & 7;
  const bool row_on = r < NE;            // rows y = 0 .. P + 1
  const bool inner = r >= 1 && r <= P;   // interior rows
  const bool yface = r <= P;             // the face between rows r and r + 1
  const int64_t warp = (blockIdx.x * (int64_t)kRowsNT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kRowsNT) >> 5;

  double dtv;
  if constexpr (STEP) {
    const double lam = order_value<float>(*a.lam_in);
    dtv = (a.cfl * a.dx) / (2.0 * lam);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.dt_slot = dtv;
  } else {
    dtv = a.dt > 0.0 ? a.dt : *a.dt_dev;
  }
  const float mhr = neg_t((float)(0.5 * (dtv / a.dx)));  // -dt / (2 dx)
  const float gm1 = a.gm1, gam = a.gamma;
  unsigned chk = 0u, lam_next = 0u;

  // the patch of this lane's group at `base` and the sources of this row
  // (metadata one iteration ahead, so its chain of dependent loads overlaps
  // the arithmetic of the current patches)
  auto row_meta = [&](int64_t base) {
    RowMeta mt{0, 0, 0, 0, 0, 0, 0, 0, false};
    const int64_t pos = base + grp;
    if (pos < a.i_end) {
      mt.pid = a.order != nullptr ? (int64_t)a.order[pos] : pos;
      const int pj = a.sizes[mt.pid];
      mt.off = a.off[mt.pid];
      mt.act = pj == P && mt.off >= 0 && (mt.off % 4) == 0 &&
               (a.n_elems <= 0 || mt.off + (int64_t)NE * NE * S <= a.n_elems);
      if (!mt.act && r == 0) atomicOr(a.status, ST_BAD_PATCH);  // other size or bad layout
      if (mt.act && row_on) {
        const FaceSrc fa = face_source<float, 2, STEP>(a, mt.pid, P, mt.off,
                                                       inner ? 0 : (r == 0 ? 2 : 3));
        mt.s0 = fa.off;
        mt.ck0 = fa.ck;
        mt.neg0 = fa.neg;
        if (inner) {
          const FaceSrc fb = face_source<float, 2, STEP>(a, mt.pid, P, mt.off, 1);
          mt.s1 = fb.off;
          mt.ck1 = fb.ck;
          mt.neg1 = fb.neg;
        }
      }
    }
    return mt;
  };

  const int64_t stride = nwarps * kRowsPerWarp;
  RowMeta nxt = row_meta(a.i_begin + warp * kRowsPerWarp);
  for (int64_t base = a.i_begin + warp * kRowsPerWarp; base < a.i_end; base += stride) {
    const RowMeta mt = nxt;
    nxt = row_meta(base + stride);
    const bool act = mt.act;
    const int64_t pid = mt.pid, off = mt.off;
    const bool on = act && row_on;

    // ---- this row's cells x = 0 .. P + 1 and their primitives -------------
    RCell c[NE];
#pragma unroll
    for (int x = 0; x < NE; ++x) {
      c[x].q[0] = 1.f;  // a benign state where no cell is loaded
      c[x].q[1] = 0.f;
      c[x].q[2] = 0.f;
      c[x].q[3] = 1.f;
    }
    if (on) {
      if (inner) {
        const float* row = a.in + off + (int64_t)(r * NE) * S;
#pragma unroll
        for (int x = 1; x <= P; ++x) ld_cell(c[x], row + x * S, 0);
        ld_cell(c[0], a.in + mt.s0 + (int64_t)(r * NE + mt.ck0) * S, mt.neg0 ? 1 : 0);
        ld_cell(c[P + 1], a.in + mt.s1 + (int64_t)(r * NE + mt.ck1) * S, mt.neg1 ? 1 : 0);
      } else {
        const float* row = a.in + mt.s0 + (int64_t)(mt.ck0 * NE) * S;
#pragma unroll
        for (int x = 1; x <= P; ++x) ld_cell(c[x], row + x * S, mt.neg0 ? 2 : 0);
      }
    }
#pragma unroll
    for (int x = 0; x < NE; ++x)
      rprims(c[x], gm1, gam, on && (inner || (x >= 1 && x <= P)), chk);

    unsigned lmax = 0u;
    // ---- x faces of an interior row: flux differences of its cells -------
    float dg[P][S];
    {
      float gprev[S];
      const unsigned ab = rflux<0>(c[0], c[1], gprev);
      lmax = umax_u(lmax, ab & (inner ? kMag : 0u));
#pragma unroll
      for (int x = 1; x <= P; ++x) {
        float g[S];
        const unsigned abx = rflux<0>(c[x], c[x + 1], g);
        lmax = umax_u(lmax, abx & (inner ? kMag : 0u));
#pragma unroll
        for (int v = 0; v < S; ++v) {
          dg[x - 1][v] = sub_rn(g[v], gprev[v]);
          gprev[v] = g[v];
        }
      }
    }

    // ---- y faces: rows r | r + 1 of every interior column ----------------
    float gy[P][S];
#pragma unroll
    for (int x = 1; x <= P; ++x) {
      RCell up;
#pragma unroll
      for (int v = 0; v < S; ++v) up.q[v] = shfl_dn(c[x].q[v]);
      up.u[1] = shfl_dn(c[x].u[1]);
      up.p = shfl_dn(c[x].p);
      up.c = shfl_dn(c[x].c);
      up.e = shfl_dn(c[x].e);
      float g[S];
      const unsigned ab = rflux<1>(c[x], up, g);
      lmax = umax_u(lmax, ab & ((act && yface) ? kMag : 0u));
#pragma unroll
      for (int v = 0; v < S; ++v) gy[x - 1][v] = g[v];
    }
    if (a.lam_patch != nullptr) {  // the patch's maximum over its eight lanes
      lmax = umax_u(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, 4));
      lmax = umax_u(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, 2));
      lmax = umax_u(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, 1));
      if (act && r == 0) a.lam_patch[pid] = order_value<float>((unsigned long long)lmax);
    }

    // ---- update: Q - (dt / 2dx) sum_k (G+ - G-), x then y ----------------
#pragma unroll
    for (int x = 1; x <= P; ++x) {
      float qn[S];
#pragma unroll
      for (int v = 0; v < S; ++v) {
        const float below = shfl_up(gy[x - 1][v]);
        const float acc = add_rn(dg[x - 1][v], sub_rn(gy[x - 1][v], below));
        qn[v] = fmaf(mhr, acc, c[x].q[v]);
      }
      if (on && inner) {
        *reinterpret_cast<float4*>(a.out + off + (int64_t)(r * NE + x) * S) =
            make_float4(qn[0], qn[1], qn[2], qn[3]);
        if constexpr (STEP) {
          // primitives and wave speeds of the new state (next CFL maximum)
          RCell w;
#pragma unroll
          for (int v = 0; v < S; ++v) w.q[v] = qn[v];
          rprims(w, gm1, gam, true, chk);
#pragma unroll
          for (int k = 0; k < 2; ++k) lam_next = umax_u(lam_next, wave_bits_f(w.u[k], w.c) & kMag);
          if (a.prim_out != nullptr) {
            constexpr int NI = P * P;
            float* po = a.prim_out + pid * a.prim_stride + (x - 1) + P * (r - 1);
            po[0] = w.u[0];
            po[NI] = w.u[1];
            po[2 * NI] = w.p;
            po[3 * NI] = w.c;
            po[4 * NI] = w.e;
          }
        }
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, chk >= kBad) && lane == 0) atomicOr(a.status, ST_NONPHYSICAL);
  if constexpr (STEP) {
    const unsigned long long m = warp_max_u64((unsigned long long)lam_next);
    if (lane == 0 && m != 0ull) atomicMax(a.lam_next, m);
  }
}

template <int P, bool STEP>
cudaError_t launch_rows2d_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
  StepParams<float> a{};
  a.in = static_cast<const float*>(l.in);
  a.out = static_cast<float*>(l.out);
  a.off = l.off;
  a.sizes = l.sizes;
  a.nbr = l.nbr;
  a.order = l.order;
  a.i_begin = l.i_begin;
  a.i_end = l.i_end >= 0 ? l.i_end : l.n;
  a.n = l.n;
  a.n_elems = l.n_elems;
  a.pmax = P;
  a.nstage = 1;
  a.gamma = (float)l.gamma;
  a.gm1 = (float)(l.gamma - 1.0);
  a.dx = l.dx;
  a.dt = l.dt;
  a.cfl = l.cfl;
  a.dt_dev = l.dt_dev;
  a.lam_in = l.lam_in;
  a.lam_next = l.lam_next;
  a.dt_slot = l.dt_slot;
  a.lam_patch = l.lam_patch;
  a.status = l.status;
  a.one = 1.0f;
  a.mone = -1.0f;
  a.mzero = -0.0f;
  a.prim_out = static_cast<float*>(l.prim_out);
  a.prim_stride = l.prim_stride;
  rows2d_kernel<P, STEP><<<grid, kRowsNT, 0, h->stream>>>(a);
  return cudaGetLastError();
}

template <int P, bool STEP>
cudaError_t occupancy_rows2d_t(int* bps) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, rows2d_kernel<P, STEP>, kRowsNT, 0);
}

}  // namespace

bool rows2d_class(const fv_batch* h, int p) {
  return h->prec == FV_FP32 && h->d == 2 && h->s == 4 && p == 5;
}

bool rows2d_eligible(const fv_batch* h, const UpdateLaunch& l) {
  const int mode = step_mode(l);
  return rows2d_class(h, l.uniform_p) && mode != kModePrim && l.corr == nullptr &&
         l.dx_patch == nullptr && !l.local_cfl && (mode == kModeStep || l.prim_out == nullptr);
}

int rows2d_patches_per_cta() { return (kRowsNT / 32) * kRowsPerWarp; }

cudaError_t launch_rows2d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return step_mode(l) == kModeStep ? launch_rows2d_t<5, true>(h, l, grid)
                                   : launch_rows2d_t<5, false>(h, l, grid);
}

cudaError_t rows2d_occupancy(int mode, int* bps) {
  return mode == kModeStep ? occupancy_rows2d_t<5, true>(bps) : occupancy_rows2d_t<5, false>(bps);
}

}  // namespace fv
