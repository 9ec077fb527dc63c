// fv_lines3d.cu -- the FP32 time step / update of a launch whose patches all
// have the 3D size p = 3 (the 3^3 class of an uneven batch, or a uniform
// batch after fv_batch_plan), one lane per line of cells along x.  Same
// method, same operations in the same order as the general kernel
// (fv_step.cuh; Eq. 2-5, Algorithm 1 steps 5-10), so the results are bitwise
// the same.
//
// A warp advances one patch at a time.  Lane l = y + 5 z (y, z in 0 .. 4)
// holds the line (y, z) of the patch box: the 9 interior lines (cells x = 0 ..
// 4, the x halos included) and the 12 face-halo lines of y and z (cells x =
// 1 .. 3); the four corner lines and lanes 25 .. 31 hold no cells.  All state
// stays in registers:
//
//  * loads: an interior line reads its 3 cells and its two x-halo cells from
//    their sources (the own halo layer in update mode; in a time step the
//    neighbour's interior layer next to the face, a wall's mirror or the
//    outflow copy); a face-halo line reads the 3 cells of its source line.
//    Where the patches and neighbours are is resolved one patch ahead;
//  * primitives of every cell of the line (Eq. 2);
//  * x faces along an interior line;
//  * y and z faces: every line takes the face below it in each direction, the
//    lower line's cells by warp shuffle from lane l - 1 / l - 5; an interior
//    line takes the face above it from lane l + 1 / l + 5 (a face-halo line's
//    lower face is the patch boundary);
//  * update: the sum x then y then z, one FMA with -dt / (2 dx), the new state
//    stored and, in a time step, converted for the next CFL maximum.
#include "fv_step.cuh"
#include "fv_cell3.cuh"

// Resident CTAs of 128 threads per SM the register allocation is sized for.
#ifndef FV_LINES3D_MINBLOCKS
#define FV_LINES3D_MINBLOCKS 5
#endif

namespace fv {
namespace {

constexpr int kL3NT = 128;  // threads per CTA: four warps, a patch each
constexpr int kL3P = 3;     // the patch size
constexpr int kL3W = kL3P + 2;  // lines per axis of the lane grid

__device__ __forceinline__ void lload(LCell& x, const float* src, int negc) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float t = __ldg(src + v);
    x.q[v] = v == negc ? neg_t(t) : t;
  }
}

// The cells of the line below (delta lanes down), state and the primitives a
// face along K reads.
template <int K>
__device__ __forceinline__ LCell shfl_cell_up(const LCell& x, int delta) {
  LCell r;
#pragma unroll
  for (int v = 0; v < 5; ++v) r.q[v] = __shfl_up_sync(0xFFFFFFFFu, x.q[v], delta);
  r.u[K] = __shfl_up_sync(0xFFFFFFFFu, x.u[K], delta);
  r.p = __shfl_up_sync(0xFFFFFFFFu, x.p, delta);
  r.c = __shfl_up_sync(0xFFFFFFFFu, x.c, delta);
  r.e = __shfl_up_sync(0xFFFFFFFFu, x.e, delta);
  return r;
}

// A patch and where this lane's line comes from.
struct LMeta {
  int64_t pid, off;
  long long s0, s1;  // sources: the line (or the -x halo), the +x halo
  int ck0, ck1, neg0, neg1;
  bool act;
};

template <bool STEP>
__global__ void __launch_bounds__(kL3NT, FV_LINES3D_MINBLOCKS) lines3d_kernel(StepParams<float> a) {
  constexpr int P = kL3P, W = kL3W, S = 5, NE = P + 2;
  const int lane = threadIdx.x & 31;
  const int ly = lane % W, lz = lane / W;  // this lane's line
  const bool yin = ly >= 1 && ly <= P, zin = lz >= 1 && lz <= P;
  const bool grid = lane < W * W;
  const bool inner = grid && yin && zin;                    // interior line
  const bool yhalo = grid && zin && (ly == 0 || ly == W - 1);  // face-halo line of y
  const bool zhalo = grid && yin && (lz == 0 || lz == W - 1);  // face-halo line of z
  const bool has = inner || yhalo || zhalo;
  const int64_t warp = (blockIdx.x * (int64_t)kL3NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kL3NT) >> 5;

  double dtv;
  if constexpr (STEP) {
    const double lam = order_value<float>(*a.lam_in);
    dtv = (a.cfl * a.dx) / (3.0 * lam);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.dt_slot = dtv;
  } else {
    dtv = a.dt > 0.0 ? a.dt : *a.dt_dev;
  }
  const float mhr = neg_t((float)(0.5 * (dtv / a.dx)));  // -dt / (2 dx)
  const float gm1 = a.gm1, gam = a.gamma;
  unsigned chk = 0u, lam_next = 0u;

  auto meta = [&](int64_t pos) {
    LMeta mt{0, 0, 0, 0, 0, 0, 0, 0, false};
    if (pos < a.i_end) {
      mt.pid = a.order != nullptr ? (int64_t)a.order[pos] : pos;
      const int pj = a.sizes[mt.pid];
      mt.off = a.off[mt.pid];
      mt.act = pj == P && mt.off >= 0 && (mt.off % 4) == 0 &&
               (a.n_elems <= 0 || mt.off + (int64_t)NE * NE * NE * S <= a.n_elems);
      if (!mt.act && lane == 0) atomicOr(a.status, ST_BAD_PATCH);  // other size or bad layout
      if (mt.act && has) {
        const int f0 = inner ? 0 : (yhalo ? (ly == 0 ? 2 : 3) : (lz == 0 ? 4 : 5));
        const FaceSrc fa = face_source<float, 3, STEP>(a, mt.pid, P, mt.off, f0);
        mt.s0 = fa.off;
        mt.ck0 = fa.ck;
        mt.neg0 = fa.neg;
        if (inner) {
          const FaceSrc fb = face_source<float, 3, STEP>(a, mt.pid, P, mt.off, 1);
          mt.s1 = fb.off;
          mt.ck1 = fb.ck;
          mt.neg1 = fb.neg;
        }
      }
    }
    return mt;
  };

  LMeta nxt = meta(a.i_begin + warp);
  for (int64_t pos = a.i_begin + warp; pos < a.i_end; pos += nwarps) {
    const LMeta mt = nxt;
    nxt = meta(pos + nwarps);
    if (!mt.act) continue;  // the whole warp: one patch
    const int64_t off = mt.off, pid = mt.pid;

    // ---- this lane's line: cells x = 0 .. P + 1 --------------------------
    LCell c[NE];
#pragma unroll
    for (int x = 0; x < NE; ++x) {
      c[x].q[0] = 1.f;  // a benign state where no cell is loaded
      c[x].q[1] = 0.f;
      c[x].q[2] = 0.f;
      c[x].q[3] = 0.f;
      c[x].q[4] = 1.f;
    }
    if (inner) {
      const int64_t lrow = (int64_t)(lz * NE + ly) * NE;
      const float* row = a.in + off + lrow * S;
#pragma unroll
      for (int x = 1; x <= P; ++x) lload(c[x], row + x * S, -1);
      lload(c[0], a.in + mt.s0 + (lrow + mt.ck0) * S, mt.neg0 ? 1 : -1);
      lload(c[P + 1], a.in + mt.s1 + (lrow + mt.ck1) * S, mt.neg1 ? 1 : -1);
    } else if (yhalo) {  // cells (x, y = ck, z) of the source
      const float* row = a.in + mt.s0 + ((int64_t)(lz * NE + mt.ck0) * NE) * S;
#pragma unroll
      for (int x = 1; x <= P; ++x) lload(c[x], row + x * S, mt.neg0 ? 2 : -1);
    } else if (zhalo) {  // cells (x, y, z = ck) of the source
      const float* row = a.in + mt.s0 + ((int64_t)(mt.ck0 * NE + ly) * NE) * S;
#pragma unroll
      for (int x = 1; x <= P; ++x) lload(c[x], row + x * S, mt.neg0 ? 3 : -1);
    }
#pragma unroll
    for (int x = 0; x < NE; ++x)
      lprims(c[x], gm1, gam, inner || (has && x >= 1 && x <= P), chk);

    unsigned lmax = 0u;
    // ---- x faces: flux differences along an interior line ----------------
    float acc[P][S];
    {
      float gprev[S];
      unsigned ab = lflux<0>(c[0], c[1], gprev);
      lmax = umax_l(lmax, ab & (inner ? kMagL : 0u));
#pragma unroll
      for (int x = 1; x <= P; ++x) {
        float g[S];
        ab = lflux<0>(c[x], c[x + 1], g);
        lmax = umax_l(lmax, ab & (inner ? kMagL : 0u));
#pragma unroll
        for (int v = 0; v < S; ++v) {
          acc[x - 1][v] = sub_rn(g[v], gprev[v]);
          gprev[v] = g[v];
        }
      }
    }

    // ---- y faces (lines l -/+ 1), then z faces (l -/+ W) -----------------
    // the face below a line exists for y >= 1 (resp. z >= 1) inside the
    // other axis' interior: interior lines and the upper face-halo lines
    const bool ylow = grid && zin && ly >= 1, zlow = grid && yin && lz >= 1;
#pragma unroll
    for (int x = 1; x <= P; ++x) {
      float gl[S], gu[S];
      const LCell by = shfl_cell_up<1>(c[x], 1);
      unsigned ab = lflux<1>(by, c[x], gl);
      lmax = umax_l(lmax, ab & (ylow ? kMagL : 0u));
#pragma unroll
      for (int v = 0; v < S; ++v) {
        gu[v] = __shfl_down_sync(0xFFFFFFFFu, gl[v], 1);
        acc[x - 1][v] = add_rn(acc[x - 1][v], sub_rn(gu[v], gl[v]));
      }
    }
#pragma unroll
    for (int x = 1; x <= P; ++x) {
      float gl[S], gu[S];
      const LCell bz = shfl_cell_up<2>(c[x], W);
      unsigned ab = lflux<2>(bz, c[x], gl);
      lmax = umax_l(lmax, ab & (zlow ? kMagL : 0u));
#pragma unroll
      for (int v = 0; v < S; ++v) {
        gu[v] = __shfl_down_sync(0xFFFFFFFFu, gl[v], W);
        acc[x - 1][v] = add_rn(acc[x - 1][v], sub_rn(gu[v], gl[v]));
      }
    }
    if (a.lam_patch != nullptr) {
      const unsigned long long m = warp_max_u64((unsigned long long)lmax);
      if (lane == 0) a.lam_patch[pid] = order_value<float>(m);
    }

    // ---- update: Q - (dt / 2dx) sum_k (G+ - G-) --------------------------
    if (inner) {
      float* dst = a.out + off + ((int64_t)(lz * NE + ly) * NE) * S;
#pragma unroll
      for (int x = 1; x <= P; ++x) {
        LCell w;
#pragma unroll
        for (int v = 0; v < S; ++v) {
          w.q[v] = fmaf(mhr, acc[x - 1][v], c[x].q[v]);
          dst[x * S + v] = w.q[v];
        }
        if constexpr (STEP) {
          // primitives and wave speeds of the new state (next CFL maximum)
          lprims(w, gm1, gam, true, chk);
#pragma unroll
          for (int k = 0; k < 3; ++k) lam_next = umax_l(lam_next, wbits_l(w.u[k], w.c) & kMagL);
          if (a.prim_out != nullptr) {
            constexpr int NI = P * P * P;
            float* po = a.prim_out + pid * a.prim_stride + (x - 1) + P * ((ly - 1) + P * (lz - 1));
            po[0] = w.u[0];
            po[NI] = w.u[1];
            po[2 * NI] = w.u[2];
            po[3 * NI] = w.p;
            po[4 * NI] = w.c;
            po[5 * NI] = w.e;
          }
        }
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, chk >= kBadL) && lane == 0) atomicOr(a.status, ST_NONPHYSICAL);
  if constexpr (STEP) {
    const unsigned long long m = warp_max_u64((unsigned long long)lam_next);
    if (lane == 0 && m != 0ull) atomicMax(a.lam_next, m);
  }
}

template <bool STEP>
cudaError_t launch_lines3d_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
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
  a.pmax = kL3P;
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
  lines3d_kernel<STEP><<<grid, kL3NT, 0, h->stream>>>(a);
  return cudaGetLastError();
}

template <bool STEP>
cudaError_t occupancy_lines3d_t(int* bps) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, lines3d_kernel<STEP>, kL3NT, 0);
}

}  // namespace

bool lines3d_class(const fv_batch* h, int p) {
  return h->prec == FV_FP32 && h->d == 3 && h->s == 5 && p == kL3P;
}

bool lines3d_eligible(const fv_batch* h, const UpdateLaunch& l) {
  const int mode = step_mode(l);
  return lines3d_class(h, l.uniform_p) && mode != kModePrim && l.corr == nullptr &&
         l.dx_patch == nullptr && !l.local_cfl && (mode == kModeStep || l.prim_out == nullptr);
}

int lines3d_patches_per_cta() { return kL3NT / 32; }

cudaError_t launch_lines3d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return step_mode(l) == kModeStep ? launch_lines3d_t<true>(h, l, grid)
                                   : launch_lines3d_t<false>(h, l, grid);
}

cudaError_t lines3d_occupancy(int mode, int* bps) {
  return mode == kModeStep ? occupancy_lines3d_t<true>(bps) : occupancy_lines3d_t<false>(bps);
}

}  // namespace fv
