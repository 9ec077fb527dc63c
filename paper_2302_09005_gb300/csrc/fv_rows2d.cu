// fv_rows2d.cu -- the FP32 time step / update of a launch whose patches all
// have one 2D size (p = 5: a size class of the schedule, or a uniform batch
// after fv_batch_plan), one lane per row of cells.  Same method, same
// operations in the same order as the general kernel (fv_step.cuh; Eq. 2-5,
// Algorithm 1 steps 5-10), so the results are bitwise the same.
//
// A warp advances four patches at a time, eight lanes each: lane r of a group
// holds row y = r of its patch box (r = 0 and r = p + 1 the face-halo rows,
// lane 7 idle).  The arithmetic stays in registers, with no block barrier:
//
//  * staging: each group copies its next patch into shared memory while it
//    computes the current one (cp.async, one 16-byte cell per copy, the eight
//    lanes taking consecutive cells so the copies coalesce): the rows 1 .. p
//    of the own box with their x-halo cells as one contiguous span, the two
//    y-halo rows from the y-face sources and, in a time step, the 2p x-halo
//    cells from the x-face sources (the neighbour's interior layer next to the
//    face, a wall's mirror, the outflow copy; the own halo layer in update
//    mode).  Where a patch's data come from is resolved two patches ahead
//    (its metadata loaded over the iterations before, one dependent step
//    each) and kept in a per-group record;
//  * primitives of every cell of the lane's row (Eq. 2);
//  * x faces: an interior row walks its p + 1 faces left to right and keeps
//    each cell's x flux difference;
//  * y faces: lane r takes the face between rows r and r + 1 of every column,
//    the upper cells' state and primitives by warp shuffle from lane r + 1;
//  * update: an interior row receives the fluxes of the faces below it from
//    lane r - 1 (shuffle), adds the y differences to its x differences (x then
//    y), takes one FMA with -dt / (2 dx) and, in a time step, converts the new
//    state for the next CFL maximum; the new state goes to the output through
//    shared memory, the group's lanes storing consecutive 16-byte cells.
#include "fv_meta.cuh"

// Resident one-warp CTAs per SM the register allocation is sized for.
#ifndef FV_ROWS2D_MINBLOCKS
#define FV_ROWS2D_MINBLOCKS 16
#endif

namespace fv {
namespace {

constexpr int kRowsNT = 32;      // threads per CTA: one warp (independent CTAs schedule best)
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
constexpr unsigned kSignR = 0x80000000u;  // the sign bit: a wall's mirrored momentum

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


// Shared-memory staging (floats) of patch size P, per group and stage: the
// rows 1 .. P of the own box with their x-halo cells (A, one contiguous
// span), the 2P x-halo cells from the x-face sources (X, time steps) and the
// two y-halo rows from the y-face sources (Y).  Cells are 16 bytes and patch
// offsets multiples of 4, so every cell is one aligned 16-byte chunk.
template <int P>
struct RGeom {
  static constexpr int S = 4, NE = P + 2;
  static constexpr int OA = 0, OX = OA + P * NE * S, OY = OX + 2 * P * S;
  static constexpr int SLOT = OY + 2 * P * S;
  static constexpr int REC = 16;                    // floats per patch record
  static constexpr int OUT = 2 * SLOT + 3 * REC;    // the new interior state, P * P cells
  static constexpr int GROUP = OUT + P * P * S;     // two stages, three records, output
  static constexpr int BYTES = (kRowsNT / 32) * kRowsPerWarp * GROUP * 4;
  static_assert(SLOT % 4 == 0 && GROUP % 4 == 0, "16-byte alignment of the stages");
};

// Where a group's patch comes from (one record per patch, a ring of three:
// the patch being computed, the one whose copies are in flight, the one
// resolved last): the four face sources (patch offset, source layer, wall
// flag) and the patch itself.
struct RRec {
  long long fo[4];
  int fck[4];  // source layer | wall << 8
  long long off;
  int pid, act;
};
static_assert(sizeof(RRec) <= 16 * 4, "record size");

__device__ __forceinline__ void write_rec2d(RRec* rec, const PatchSrc& n, int r) {
  if (r < 4) {
    rec->fo[r] = n.fo;
    rec->fck[r] = n.fck;
  } else if (r == 4) {
    rec->off = n.off;
    rec->pid = n.pid;
    rec->act = n.act;
  }
}

__device__ __forceinline__ void cp_cell(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}

// Issues the copies of the group's patch into `slot`, 16-byte cells, lane r
// of the group taking cells r, r + 8, ... of each part, so the eight lanes
// read consecutive cells.
template <int P, bool STEP>
__device__ __forceinline__ void issue_patch2d(const StepParams<float>& a, const RRec* m,
                                              float* slot, int r) {
  using G = RGeom<P>;
  constexpr int S = 4, NE = P + 2;
  if (!m->act) return;
  const float* sa = a.in + m->off + NE * S;  // cell (0, 1)
#pragma unroll
  for (int k = r; k < P * NE; k += kRowsGroup) cp_cell(slot + G::OA + S * k, sa + S * k);
#pragma unroll
  for (int c = r; c < 2 * P; c += kRowsGroup) {
    const int s = c >= P ? 1 : 0, x = c - s * P;
    const long long so = m->fo[2 + s] + (long long)(1 + x + NE * (m->fck[2 + s] & 0xFF)) * S;
    cp_cell(slot + G::OY + S * c, a.in + so);
  }
  if constexpr (STEP) {
#pragma unroll
    for (int c = r; c < 2 * P; c += kRowsGroup) {
      const int s = c >= P ? 1 : 0, row = c - s * P + 1;
      const long long so = m->fo[s] + (long long)((m->fck[s] & 0xFF) + NE * row) * S;
      cp_cell(slot + G::OX + S * c, a.in + so);
    }
  }
}

__device__ __forceinline__ void st_cell(RCell& x, const float* src, unsigned nm1, unsigned nm2) {
  const float4 v = *reinterpret_cast<const float4*>(src);
  x.q[0] = v.x;
  x.q[1] = __uint_as_float(__float_as_uint(v.y) ^ nm1);
  x.q[2] = __uint_as_float(__float_as_uint(v.z) ^ nm2);
  x.q[3] = v.w;
}

__device__ __forceinline__ float shfl_dn(float v) { return __shfl_down_sync(0xFFFFFFFFu, v, 1); }
__device__ __forceinline__ float shfl_up(float v) { return __shfl_up_sync(0xFFFFFFFFu, v, 1); }

// Resident CTAs per SM the registers are sized for (no spills): p <= 5 at
// 128 registers, 6 at 168.
template <int P>
constexpr int rows_blocks() {
  return P <= 5 ? FV_ROWS2D_MINBLOCKS : 12;
}

template <int P, bool STEP>
__global__ void __launch_bounds__(kRowsNT, rows_blocks<P>()) rows2d_kernel(StepParams<float> a) {
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

  using G = RGeom<P>;
  extern __shared__ __align__(16) float rsm[];
  float* const gbase = rsm + ((threadIdx.x >> 5) * kRowsPerWarp + grp) * G::GROUP;
  RRec* const recs = reinterpret_cast<RRec*>(gbase + 2 * G::SLOT);  // ring of three
  const int64_t stride = nwarps * kRowsPerWarp;
  const int64_t base0 = a.i_begin + warp * kRowsPerWarp;
  if (base0 >= a.i_end) return;  // the whole warp: no patch
  // the first two patches resolved, the first one's copies issued
  write_rec2d(recs, resolve_now<2, P, STEP>(a, base0 + grp, r & 3, r < 4, r == 0), r);
  write_rec2d(recs + 1, resolve_now<2, P, STEP>(a, base0 + stride + grp, r & 3, r < 4, r == 0), r);
  __syncwarp();
  // the metadata pipeline: patch 2 past its second step, patch 3 past its first
  MetaPatch q2 = meta_patch<2, STEP>(a, meta_pid(a, base0 + 2 * stride + grp), r & 3);
  int q3 = meta_pid(a, base0 + 3 * stride + grp);
  issue_patch2d<P, STEP>(a, recs, gbase, r);
  cp_async_commit();
  int rc = 0, rn = 1, rl = 2;  // records: computed, in flight, resolved last
  int st = 0;                  // stage of the patch being computed

  for (int64_t base = base0; base < a.i_end; base += stride) {
    // this iteration's metadata loads (patches two, three and four ahead),
    // consumed at its end or in the next iteration
    const MetaNbr t2 = meta_nbr<STEP>(a, q2);
    const MetaPatch n3 = meta_patch<2, STEP>(a, q3, r & 3);
    const int n4 = meta_pid(a, base + 4 * stride + grp);
    cp_async_wait_all();
    __syncwarp();
    // the next patch's copies land while this one is computed
    issue_patch2d<P, STEP>(a, recs + rn, gbase + (st ^ 1) * G::SLOT, r);
    cp_async_commit();
    const RRec* m = recs + rc;
    const float* slot = gbase + st * G::SLOT;
    const bool act = m->act != 0;
    const int64_t pid = m->pid, off = m->off;
    const bool on = act && row_on;

    // ---- this row's cells x = 0 .. P + 1 from the stage -------------------
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
        const float* row = slot + G::OA + (r - 1) * NE * S;
#pragma unroll
        for (int x = 1; x <= P; ++x) st_cell(c[x], row + x * S, 0u, 0u);
        if constexpr (STEP) {
          st_cell(c[0], slot + G::OX + (r - 1) * S, (m->fck[0] >> 8) ? kSignR : 0u, 0u);
          st_cell(c[P + 1], slot + G::OX + (P + r - 1) * S, (m->fck[1] >> 8) ? kSignR : 0u, 0u);
        } else {  // update mode: the own halo cells, in the span
          st_cell(c[0], row, 0u, 0u);
          st_cell(c[P + 1], row + (P + 1) * S, 0u, 0u);
        }
      } else {
        const int sy = r == 0 ? 0 : 1;
        const float* row = slot + G::OY + sy * P * S;
        const unsigned nm2 = (m->fck[2 + sy] >> 8) ? kSignR : 0u;
#pragma unroll
        for (int x = 1; x <= P; ++x) st_cell(c[x], row + (x - 1) * S, 0u, nm2);
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
        *reinterpret_cast<float4*>(gbase + G::OUT + ((r - 1) * P + x - 1) * S) =
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
    // the new state to the output: the group's lanes store consecutive
    // cells (from the output stage), so the stores coalesce
    __syncwarp();
    if (act) {
#pragma unroll
      for (int c = r; c < P * P; c += kRowsGroup) {
        const int yy = c / P, xx = c - yy * P;
        *reinterpret_cast<float4*>(a.out + off + (int64_t)((yy + 1) * NE + xx + 1) * S) =
            *reinterpret_cast<const float4*>(gbase + G::OUT + c * S);
      }
    }
    // the record of the patch two ahead, read after the next iteration's
    // warp barrier
    write_rec2d(recs + rl,
                finish_patch<2, P, STEP>(a, base + 2 * stride + grp, q2, t2, r & 3, r < 4, r == 0),
                r);
    q2 = n3;
    q3 = n4;
    const int t = rc;
    rc = rn;
    rn = rl;
    rl = t;
    st ^= 1;
  }
  cp_async_wait_all();
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
  rows2d_kernel<P, STEP><<<grid, kRowsNT, RGeom<P>::BYTES, h->stream>>>(a);
  return cudaGetLastError();
}

template <int P, bool STEP>
cudaError_t occupancy_rows2d_t(int* bps) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, rows2d_kernel<P, STEP>, kRowsNT,
                                                       RGeom<P>::BYTES);
}

}  // namespace

bool rows2d_class(const fv_batch* h, int p) {
  return h->prec == FV_FP32 && h->d == 2 && h->s == 4 && p >= 3 && p <= 6;
}

bool rows2d_eligible(const fv_batch* h, const UpdateLaunch& l) {
  const int mode = step_mode(l);
  return rows2d_class(h, l.uniform_p) && mode != kModePrim && l.corr == nullptr &&
         l.dx_patch == nullptr && !l.local_cfl && (mode == kModeStep || l.prim_out == nullptr);
}

int rows2d_patches_per_cta() { return (kRowsNT / 32) * kRowsPerWarp; }

template <int P>
static cudaError_t launch_rows2d_p(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return step_mode(l) == kModeStep ? launch_rows2d_t<P, true>(h, l, grid)
                                   : launch_rows2d_t<P, false>(h, l, grid);
}

cudaError_t launch_rows2d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  switch (l.uniform_p) {
    case 3:
      return launch_rows2d_p<3>(h, l, grid);
    case 4:
      return launch_rows2d_p<4>(h, l, grid);
    case 6:
      return launch_rows2d_p<6>(h, l, grid);
    default:
      return launch_rows2d_p<5>(h, l, grid);
  }
}

template <int P>
static cudaError_t occupancy_rows2d_p(int mode, int* bps) {
  return mode == kModeStep ? occupancy_rows2d_t<P, true>(bps) : occupancy_rows2d_t<P, false>(bps);
}

cudaError_t rows2d_occupancy(int p, int mode, int* bps) {
  switch (p) {
    case 3:
      return occupancy_rows2d_p<3>(mode, bps);
    case 4:
      return occupancy_rows2d_p<4>(mode, bps);
    case 6:
      return occupancy_rows2d_p<6>(mode, bps);
    default:
      return occupancy_rows2d_p<5>(mode, bps);
  }
}

}  // namespace fv
