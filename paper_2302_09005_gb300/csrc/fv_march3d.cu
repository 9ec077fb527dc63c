// fv_march3d.cu -- the FP32 time step / update of a launch whose patches all
// have one 3D size P = 3 .. 7 (a size class of the schedule, or a uniform
// batch after fv_batch_plan): a lane per row of cells along x, the patch swept
// plane by plane along z.  Same method, same operations in the
// same order as the general kernel (fv_step.cuh; Eq. 2-5, Algorithm 1 steps
// 5-10), so the results are bitwise the same.
//
// A warp advances four patches at a time, eight lanes each; lane r of a group
// holds row y = r of the current plane z (r = 0 and r = P + 1 the face-halo
// rows; lanes past P + 1 idle; for P = 7 lane 7 holds row 7 and also converts
// the staged row 8).  Per plane:
//
//  * staging: the plane's data arrive in shared memory by cp.async copies of
//    16-byte chunks issued one plane ahead (the next patch's first plane
//    during the current patch's last): the rows 1 .. P of the plane as one
//    contiguous span (from the own box, or, for the two z-halo planes, from
//    the z-face sources: the neighbour's interior layer next to the face in a
//    time step, a wall's mirror, the outflow copy, the own halo layer in
//    update mode), the two y-halo rows from the y-face sources and, in a time
//    step, the 2P x-halo cells from the x-face sources.  Each span is copied
//    from its 16-byte-aligned start, so the eight lanes of a group read
//    consecutive chunks and the copies coalesce;
//  * z faces: the face between plane z - 1 and plane z of every cell of the
//    row; plane z - 1 (its state, the sum of its x and y flux differences and
//    the z flux of the face below it) stays in registers from the previous
//    plane, so no lane exchange is needed (its primitives are converted again
//    from its state: the same operations, fewer registers).  Plane z - 1 is then
//    complete: Q - (dt / 2dx)(dGx + dGy + dGz), stored through shared memory
//    as contiguous row segments and, in a time step, converted for the next
//    CFL maximum;
//  * x faces along the lane's row, y faces with the upper row's cells from
//    lane r + 1 (warp shuffle), the flux of the face below from lane r - 1:
//    dGx + dGy of plane z, carried to the next plane with its state.
//
// Where the next patch's data come from is loaded in the dependent steps of
// fv_meta.cuh, one per plane over the current patch's first planes.
#include "fv_cell3.cuh"
#include "fv_meta.cuh"

// Resident one-warp CTAs per SM the register allocation of P = 5 is sized
// for (12 x 32 threads x 168 registers: no spills).
#ifndef FV_MARCH3D_MINBLOCKS
#define FV_MARCH3D_MINBLOCKS 12
#endif

namespace fv {
namespace {

// threads per CTA: one warp.  Independent one-warp CTAs ran 5 % faster than
// four-warp CTAs at the same register count and occupancy (262,144 patches
// of 5^3: 0.605 against 0.634 ms per step).
constexpr int kMNT = 32;
constexpr int kMG = 8;     // lanes per patch
constexpr int kMPW = 4;    // patches per warp
constexpr int kMGroups = (kMNT / 32) * kMPW;  // patches per CTA and iteration

// Shared-memory layout (floats) of patch size P.  Per group and stage: the
// span of rows 1 .. P (A), the two y-halo rows (Y) and the 2P x-halo cells
// (X), each copied from its 16-byte-aligned start, so each holds up to 3
// floats before the data.  Groups lie GSTR floats apart, GSTR = 8 (mod 32),
// so the four groups of a warp read distinct banks.
template <int P>
struct MGeom {
  static constexpr int S = 5, NE = P + 2;
  // rows 0 .. NE - 1 on the group's lanes; for NE = kMG + 1 the last
  // interior lane also reads the upper y-halo row
  static_assert(NE <= kMG + 1, "the rows of a patch box fit a lane group");
  static constexpr int SPAN = P * NE * S;         // rows 1 .. P of a plane
  static constexpr int ROW = P * S;               // cells 1 .. P of a row
  static constexpr int NA = (SPAN + 6) / 4;       // chunks of the span, at most
  static constexpr int NY = (ROW + 6) / 4;        // chunks of a y-halo row, at most
  static constexpr int OA = 0, OY = 4 * NA, OX = OY + 2 * 4 * NY;
  static constexpr int SLOT = OX + 2 * P * 8;     // an x-halo cell: two chunks
  static constexpr int GSTR = SLOT + ((8 - SLOT % 32) + 32) % 32;
  static constexpr int STAGES = 2;
  static constexpr int OUT = P * P * S;           // new state of a plane's interior
  static constexpr int OSTR = OUT + ((8 - OUT % 32) + 32) % 32;
  static constexpr int META = 24;                 // floats per patch record
  static constexpr int F_STAGE = 0;
  static constexpr int F_OUT = F_STAGE + (kMNT / 32) * STAGES * kMPW * GSTR;
  static constexpr int F_META = F_OUT + kMGroups * OSTR;
  static constexpr int FLOATS = F_META + kMGroups * 2 * META;
  static constexpr int BYTES = FLOATS * 4;
  static_assert(GSTR % 4 == 0 && OSTR % 4 == 0 && F_OUT % 4 == 0 && F_META % 4 == 0,
                "16-byte alignment of the copy targets");
};

// Where a patch's data come from, in shared memory (one record per group and
// patch, double-buffered): the six face sources (patch offset, source layer
// and wall flag) and the patch itself.
struct MMeta {
  long long fo[6];  // source patch offsets
  int fck[6];       // source layer | wall << 8
  long long off;    // the patch's offset
  int pid;          // the patch's index
  int act;          // the patch is valid
};
static_assert(sizeof(MMeta) <= 24 * 4, "record size");

__device__ __forceinline__ void cp_chunk(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}

// Copies `len` floats starting at element `so` of `in` as the 16-byte chunks
// that cover them (the first chunk starts at so rounded down to a multiple of
// 4); lane r of the group takes chunks r, r + 8, ...  Every chunk holds at
// least one float of the span, so it lies inside the span's allocation.
__device__ __forceinline__ void copy_span(float* dst, const float* in, long long so, int len,
                                          int r) {
  const long long al = so & ~3ll;
  const int n = (int)((so - al) + len + 3) >> 2;
  for (int k = r; k < n; k += kMG) cp_chunk(dst + 4 * k, in + al + 4 * k);
}

__device__ __forceinline__ void write_record(MMeta* rec, const PatchSrc& n, int r) {
  if (r < 6) {
    rec->fo[r] = n.fo;
    rec->fck[r] = n.fck;
  } else if (r == 6) {
    rec->off = n.off;
    rec->pid = n.pid;
    rec->act = n.act;
  }
}

// Issues the copies of plane z of the group's patch into `slot` (Algorithm 1
// step 5, the face halo gathered with the plane that needs it).
template <int P, bool STEP>
__device__ __forceinline__ void issue_plane(const StepParams<float>& a, const MMeta* m, int z,
                                            float* slot, int r) {
  using G = MGeom<P>;
  constexpr int S = 5, NE = P + 2;
  if (!m->act) return;
  if (z >= 1 && z <= P) {
    copy_span(slot + G::OA, a.in, m->off + (long long)(NE * (1 + NE * z)) * S, G::SPAN, r);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int ck = m->fck[2 + s] & 0xFF;
      copy_span(slot + G::OY + s * 4 * G::NY, a.in,
                m->fo[2 + s] + (long long)(1 + NE * (ck + NE * z)) * S, G::ROW, r);
    }
    if constexpr (STEP) {
#pragma unroll
      for (int c = r; c < 2 * P; c += kMG) {
        const int side = c >= P ? 1 : 0;
        const int row = c - side * P + 1;
        const int ck = m->fck[side] & 0xFF;
        const long long so = m->fo[side] + (long long)(ck + NE * (row + NE * z)) * S;
        const long long al = so & ~3ll;
        cp_chunk(slot + G::OX + 8 * c, a.in + al);
        cp_chunk(slot + G::OX + 8 * c + 4, a.in + al + 4);
      }
    }
  } else {
    const int f = z == 0 ? 4 : 5;
    const int ck = m->fck[f] & 0xFF;
    copy_span(slot + G::OA, a.in, m->fo[f] + (long long)(NE * (1 + NE * ck)) * S, G::SPAN, r);
  }
}

// A cell's five unknowns from shared memory; nm<k> = the sign bit where a
// wall mirrors momentum component k (else 0).
__device__ __forceinline__ void sread(float (&q)[5], const float* p, unsigned nm1, unsigned nm2,
                                      unsigned nm3) {
  q[0] = p[0];
  q[1] = __uint_as_float(__float_as_uint(p[1]) ^ nm1);
  q[2] = __uint_as_float(__float_as_uint(p[2]) ^ nm2);
  q[3] = __uint_as_float(__float_as_uint(p[3]) ^ nm3);
  q[4] = p[4];
}
constexpr unsigned kSign = 0x80000000u;

// Resident CTAs per SM the registers are sized for (no spills): P = 3 at 128
// registers, 4 and 5 at 168, 6 and 7 (six and seven cells a row in
// flight) at 255.
template <int P>
constexpr int march_blocks() {
  return P <= 3 ? 16 : P <= 5 ? FV_MARCH3D_MINBLOCKS : 8;
}

template <int P, bool STEP, bool LAM>
__global__ void __launch_bounds__(kMNT, march_blocks<P>()) march3d_kernel(StepParams<float> a) {
  using G = MGeom<P>;
  constexpr int S = 5, NE = P + 2;
  constexpr bool TOP = NE == kMG + 1;  // lane P also converts the upper y-halo row
  extern __shared__ __align__(16) float msm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane >> 3, r = lane & 7;
  const bool inner = r >= 1 && r <= P;      // interior row
  const bool hrow = r == 0 || (!TOP && r == NE - 1);  // face-halo row of this lane
  const int ri = inner ? r - 1 : 0;         // span row this lane reads (a valid one)
  float* const stg = msm + G::F_STAGE + wid * (G::STAGES * kMPW * G::GSTR) + grp * G::GSTR;
  float* const outb = msm + G::F_OUT + (wid * kMPW + grp) * G::OSTR;
  MMeta* const rec = reinterpret_cast<MMeta*>(msm + G::F_META + (wid * kMPW + grp) * 2 * G::META);
  const int64_t warp = ((int64_t)blockIdx.x * kMNT + threadIdx.x) >> 5;
  const int64_t stride = (((int64_t)gridDim.x * kMNT) >> 5) * kMPW;

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

  int64_t base = a.i_begin + warp * kMPW;
  if (base >= a.i_end) return;  // the whole warp: no patch
  {
    const PatchSrc n0 = resolve_now<3, P, STEP>(a, base + grp, r < 6 ? r : 0, r < 6, r == 0);
    write_record(rec, n0, r);
    __syncwarp();
    issue_plane<P, STEP>(a, rec, 0, stg, r);
    cp_async_commit();
  }
  int cur = 0;  // record of the current patch
  int sc = 0;   // planes advanced (the stage of a plane: its count mod 2)

  // plane z - 1: state, dGx + dGy, z flux of the face below
  float pq[P][S], pacc[P][S], pglo[P][S];

  for (; base < a.i_end; base += stride) {
    // the next patch's metadata: for P <= 5 one dependent load step per
    // plane; for P = 7 all at once here, held in registers for the patch
    // (measured per FP32 step: 7^3 0.283 ms at once against 0.295 ms staged,
    // 3^3 0.097 ms staged against 0.101 ms at once)
    constexpr bool kStaged = P <= 5;
    const int64_t npos = base + stride + grp;
    int npid = 0;
    MetaPatch nm{0, 0, 0, -1};
    MetaNbr nt{0, 0};
    PatchSrc nx{0, 0, 0, 0, 0};
    if constexpr (!kStaged) nx = resolve_now<3, P, STEP>(a, npos, r < 6 ? r : 0, r < 6, r == 0);
    const MMeta* m = rec + cur;
    const bool act = m->act != 0;
    const long long off = m->off;
    const int64_t pid = m->pid;
    unsigned lmax = 0u;

    for (int z = 0; z < NE; ++z) {
      // ---- the copies of plane z are complete; issue those of the next plane
      cp_async_wait_all();
      __syncwarp();
      float* const slot = stg + (sc & 1) * (kMPW * G::GSTR);
      float* const nslot = stg + ((sc + 1) & 1) * (kMPW * G::GSTR);
      ++sc;
      if (z + 1 < NE) {
        issue_plane<P, STEP>(a, m, z + 1, nslot, r);
      } else {
        if constexpr (kStaged)
          nx = finish_patch<3, P, STEP>(a, npos, nm, nt, r < 6 ? r : 0, r < 6, r == 0);
        write_record(rec + (cur ^ 1), nx, r);
        __syncwarp();
        issue_plane<P, STEP>(a, rec + (cur ^ 1), 0, nslot, r);
      }
      cp_async_commit();
      if constexpr (kStaged) {
        if (z == 0) {
          npid = meta_pid(a, npos);
        } else if (z == 1) {
          nm = meta_patch<3, STEP>(a, npid, r < 6 ? r : 0);
        } else if (z == 2) {
          nt = meta_nbr<STEP>(a, nm);
        }
      }

      // ---- this lane's row of plane z: where it is staged, which component
      // a wall mirrors
      const float* rowp;
      unsigned nm2 = 0u, nm3 = 0u;
      if (z == 0 || z == NE - 1) {  // z-halo plane: interior rows from the z-face source
        const int f = z == 0 ? 4 : 5;
        const int fck = m->fck[f];
        const long long so = m->fo[f] + (long long)(NE * (1 + NE * (fck & 0xFF))) * S;
        rowp = slot + G::OA + (int)(so & 3) + ri * NE * S + S;
        nm3 = (fck >> 8) ? kSign : 0u;
      } else if (hrow) {  // y-halo row from the y-face source
        const int s = r == 0 ? 0 : 1;
        const int fck = m->fck[2 + s];
        const long long so = m->fo[2 + s] + (long long)(1 + NE * ((fck & 0xFF) + NE * z)) * S;
        rowp = slot + G::OY + s * 4 * G::NY + (int)(so & 3);
        nm2 = (fck >> 8) ? kSign : 0u;
      } else {  // interior row of the own plane (lane 7: row 1, unused)
        const long long so = off + (long long)(NE * (1 + NE * z)) * S;
        rowp = slot + G::OA + (int)(so & 3) + ri * NE * S + S;
      }

      if (z == 0) {  // plane 0: state and primitives only
#pragma unroll
        for (int i = 0; i < P; ++i) {
          LCell c;
          sread(c.q, rowp + i * S, 0u, nm2, nm3);
          lprims(c, gm1, gam, act && inner, chk);
#pragma unroll
          for (int v = 0; v < S; ++v) pq[i][v] = c.q[v];
        }
        continue;
      }

      // ---- z faces between plane z - 1 and plane z; plane z - 1 completes
      LCell cc[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        sread(cc[i].q, rowp + i * S, 0u, nm2, nm3);
        lprims(cc[i], gm1, gam, act && (inner || (hrow && z < NE - 1)), chk);
        LCell L;  // plane z - 1's cell, its primitives again (the same operations)
#pragma unroll
        for (int v = 0; v < S; ++v) L.q[v] = pq[i][v];
        lprims(L, gm1, gam, false, chk);
        float g[S];
        const unsigned ab = lflux<2>(L, cc[i], g);
        lmax = umax_l(lmax, ab & ((LAM && act && inner) ? kMagL : 0u));
        if (z >= 2) {
          float qn[S];
#pragma unroll
          for (int v = 0; v < S; ++v) {
            const float acc = add_rn(pacc[i][v], sub_rn(g[v], pglo[i][v]));
            qn[v] = fmaf(mhr, acc, pq[i][v]);
            if (inner) outb[ri * P * S + i * S + v] = qn[v];
          }
          if constexpr (STEP) {
            // primitives and wave speeds of the new state (next CFL maximum)
            LCell w;
#pragma unroll
            for (int v = 0; v < S; ++v) w.q[v] = qn[v];
            lprims(w, gm1, gam, act && inner, chk);
            if (act && inner) {
#pragma unroll
              for (int k = 0; k < 3; ++k) lam_next = umax_l(lam_next, wbits_l(w.u[k], w.c) & kMagL);
            }
          }
        }
#pragma unroll
        for (int v = 0; v < S; ++v) pglo[i][v] = g[v];
      }
      if constexpr (STEP) {
        if (z >= 2 && act && inner && a.prim_out != nullptr) {
          // the primitives of the new state to the carry block: converted
          // again from the output stage (the same operations, so the same
          // values), which keeps them out of the registers of the loop above
#pragma unroll
          for (int i = 0; i < P; ++i) {
            LCell w;
#pragma unroll
            for (int v = 0; v < S; ++v) w.q[v] = outb[ri * P * S + i * S + v];
            lprims(w, gm1, gam, false, chk);
            constexpr int NI = P * P * P;
            float* po = a.prim_out + pid * a.prim_stride + i + P * (ri + P * (z - 2));
            po[0] = w.u[0];
            po[NI] = w.u[1];
            po[2 * NI] = w.u[2];
            po[3 * NI] = w.p;
            po[4 * NI] = w.c;
            po[5 * NI] = w.e;
          }
        }
      }
      if (z >= 2) {  // plane z - 1 to the output, in contiguous row segments
        __syncwarp();
        if (act) {
          float* dst = a.out + off + (long long)(1 + NE * (1 + NE * (z - 1))) * S;
#pragma unroll
          for (int row = 0; row < P; ++row) {
#pragma unroll
            for (int j = r; j < P * S; j += kMG) dst[row * NE * S + j] = outb[row * P * S + j];
          }
        }
      }
      if (z == NE - 1) continue;  // the last z-halo plane has no x or y faces

      // ---- x faces along an interior row
      LCell h0, h1;
      if constexpr (STEP) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int fck = m->fck[s];
          const long long so =
              m->fo[s] + (long long)((fck & 0xFF) + NE * ((ri + 1) + NE * z)) * S;
          sread(s == 0 ? h0.q : h1.q, slot + G::OX + 8 * (s * P + ri) + (int)(so & 3),
                (fck >> 8) ? kSign : 0u, 0u, 0u);
        }
      } else {  // update mode: the own halo cells, in the span
        sread(h0.q, rowp - S, 0u, 0u, 0u);
        sread(h1.q, rowp + P * S, 0u, 0u, 0u);
      }
      lprims(h0, gm1, gam, act && inner, chk);
      lprims(h1, gm1, gam, act && inner, chk);
      // the upper y-halo row where it has no lane of its own
      const float* toprow = nullptr;
      unsigned topm = 0u;
      if constexpr (TOP) {
        const int fck = m->fck[3];
        const long long so = m->fo[3] + (long long)(1 + NE * ((fck & 0xFF) + NE * z)) * S;
        toprow = slot + G::OY + 4 * G::NY + (int)(so & 3);
        topm = (fck >> 8) ? kSign : 0u;
      }
      // ---- cell by cell: its upper x face (dGx), then its y faces: rows
      // r | r + 1 (the upper cells from lane r + 1), the face below from lane
      // r - 1; dGx + dGy carried with the state
      float gp[S];
      {
        const unsigned ab = lflux<0>(h0, cc[0], gp);
        lmax = umax_l(lmax, ab & ((LAM && act && inner) ? kMagL : 0u));
      }
#pragma unroll
      for (int i = 0; i < P; ++i) {
        float dg[S];
        {
          float g[S];
          const unsigned ab = lflux<0>(cc[i], i + 1 < P ? cc[i + 1] : h1, g);
          lmax = umax_l(lmax, ab & ((LAM && act && inner) ? kMagL : 0u));
#pragma unroll
          for (int v = 0; v < S; ++v) {
            dg[v] = sub_rn(g[v], gp[v]);
            gp[v] = g[v];
          }
        }
        LCell up;
#pragma unroll
        for (int v = 0; v < S; ++v) up.q[v] = __shfl_down_sync(0xFFFFFFFFu, cc[i].q[v], 1);
        up.u[0] = 0.f;
        up.u[1] = __shfl_down_sync(0xFFFFFFFFu, cc[i].u[1], 1);
        up.u[2] = 0.f;
        up.p = __shfl_down_sync(0xFFFFFFFFu, cc[i].p, 1);
        up.c = __shfl_down_sync(0xFFFFFFFFu, cc[i].c, 1);
        up.e = __shfl_down_sync(0xFFFFFFFFu, cc[i].e, 1);
        if constexpr (TOP) {
          if (r == P) {  // row P + 1: staged by the group, converted here
            sread(up.q, toprow + i * S, 0u, topm, 0u);
            lprims(up, gm1, gam, act, chk);
          }
        }
        float g[S];
        const unsigned ab = lflux<1>(cc[i], up, g);
        lmax = umax_l(lmax, ab & ((LAM && act && r <= P) ? kMagL : 0u));
#pragma unroll
        for (int v = 0; v < S; ++v) {
          const float below = __shfl_up_sync(0xFFFFFFFFu, g[v], 1);
          pacc[i][v] = add_rn(dg[v], sub_rn(g[v], below));
          pq[i][v] = cc[i].q[v];
        }
      }
    }
    if constexpr (LAM) {  // the patch's maximum over its eight lanes
      lmax = umax_l(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, 4));
      lmax = umax_l(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, 2));
      lmax = umax_l(lmax, __shfl_xor_sync(0xFFFFFFFFu, lmax, 1));
      if (act && r == 0) a.lam_patch[pid] = order_value<float>((unsigned long long)lmax);
    }
    cur ^= 1;
  }
  cp_async_wait_all();
  if (__any_sync(0xFFFFFFFFu, chk >= kBadL) && lane == 0) atomicOr(a.status, ST_NONPHYSICAL);
  if constexpr (STEP) {
    const unsigned long long m = warp_max_u64((unsigned long long)lam_next);
    if (lane == 0 && m != 0ull) atomicMax(a.lam_next, m);
  }
}

template <int P, bool STEP, bool LAM>
cudaError_t march3d_smem_attr() {
  static int set_bytes[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && set_bytes[dev] >= MGeom<P>::BYTES) return cudaSuccess;
  e = cudaFuncSetAttribute(march3d_kernel<P, STEP, LAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           MGeom<P>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(march3d_kernel<P, STEP, LAM>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && dev >= 0 && dev < 64) set_bytes[dev] = MGeom<P>::BYTES;
  return e;
}

template <int P, bool STEP, bool LAM>
cudaError_t launch_march3d_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
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
  cudaError_t e = march3d_smem_attr<P, STEP, LAM>();
  if (e != cudaSuccess) return e;
  march3d_kernel<P, STEP, LAM><<<grid, kMNT, MGeom<P>::BYTES, h->stream>>>(a);
  return cudaGetLastError();
}

template <int P, bool STEP>
cudaError_t occupancy_march3d_t(int* bps) {  // the kernel with per-patch maxima
  cudaError_t e = march3d_smem_attr<P, STEP, true>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, march3d_kernel<P, STEP, true>, kMNT,
                                                       MGeom<P>::BYTES);
}

}  // namespace

bool march3d_class(const fv_batch* h, int p) {
  return h->prec == FV_FP32 && h->d == 3 && h->s == 5 && p >= 3 && p <= 7;
}

bool march3d_eligible(const fv_batch* h, const UpdateLaunch& l) {
  const int mode = step_mode(l);
  return march3d_class(h, l.uniform_p) && mode != kModePrim && l.corr == nullptr &&
         l.dx_patch == nullptr && !l.local_cfl && (mode == kModeStep || l.prim_out == nullptr);
}

int march3d_patches_per_cta() { return kMGroups; }

template <int P>
static cudaError_t launch_march3d_p(const fv_batch* h, const UpdateLaunch& l, int grid) {
  const bool step = step_mode(l) == kModeStep, lam = l.lam_patch != nullptr;
  if (step)
    return lam ? launch_march3d_t<P, true, true>(h, l, grid)
               : launch_march3d_t<P, true, false>(h, l, grid);
  return lam ? launch_march3d_t<P, false, true>(h, l, grid)
             : launch_march3d_t<P, false, false>(h, l, grid);
}

cudaError_t launch_march3d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  switch (l.uniform_p) {
    case 3:
      return launch_march3d_p<3>(h, l, grid);
    case 4:
      return launch_march3d_p<4>(h, l, grid);
    case 6:
      return launch_march3d_p<6>(h, l, grid);
    case 7:
      return launch_march3d_p<7>(h, l, grid);
    default:
      return launch_march3d_p<5>(h, l, grid);
  }
}

template <int P>
static cudaError_t occupancy_march3d_p(int mode, int* bps) {
  return mode == kModeStep ? occupancy_march3d_t<P, true>(bps) : occupancy_march3d_t<P, false>(bps);
}

cudaError_t march3d_occupancy(int p, int mode, int* bps) {
  switch (p) {
    case 3:
      return occupancy_march3d_p<3>(mode, bps);
    case 4:
      return occupancy_march3d_p<4>(mode, bps);
    case 6:
      return occupancy_march3d_p<6>(mode, bps);
    case 7:
      return occupancy_march3d_p<7>(mode, bps);
    default:
      return occupancy_march3d_p<5>(mode, bps);
  }
}

}  // namespace fv
