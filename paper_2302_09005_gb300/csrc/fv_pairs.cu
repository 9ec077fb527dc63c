// fv_pairs.cu -- the FP32 time step / update of a launch whose patches all
// have one 3D size (a size class of the schedule, or a uniform batch after
// fv_batch_plan), laid out for instruction issue, which bounds the FP32 step
// of the general kernel (fv_step.cuh).  Same method, same operations in the
// same order (Eq. 2-5, Algorithm 1 steps 5-10): the results are bitwise
// those of the general kernel.  What changes is the work per thread:
//
//  * staging: the patch box arrives by one bulk copy (TMA engine, mbarrier
//    completion) as cells of 5 unknowns; the halo cells from the neighbours
//    are gathered with cp.async.  The cells then convert once, to shared
//    structure-of-arrays form: the state (rho, j, E) and the primitives
//    (u_y, u_z, p, c) of the interior and face-halo cells the y and z
//    faces and the update read, laid out so that two x-neighbours come with
//    one 64-bit load and the lanes of a warp hit distinct banks;
//  * packed arithmetic: two x-neighbouring cells (or faces) are computed
//    together with the f32x2 instructions (fv_x2.cuh): one instruction for
//    both elements, each rounded as the scalar operation;
//  * fixed indexing: every patch of the launch has the same size, so each
//    thread's cells, faces and shared-memory offsets are computed once per
//    launch, before the patch loop;
//  * roles: all warps convert the cells (x pairs); the items of the interior
//    rows also compute the x faces between their cells and the next item's
//    (neighbours exchange cells with warp shuffles) and keep the flux
//    difference G+ - G- of each cell in registers; warps 0 and 1 then walk
//    the y and z lines in x-pairs, each line in two halves on two lanes,
//    while warps 2 and 3 gather the halo cells of the next patch; the
//    interior-row threads then update their pairs (three differences per
//    unknown, fixed order x, y, z) and convert the new state for the next
//    CFL maximum;
//  * two box buffers: a patch's bulk copy starts two patches ahead, its
//    halo gather one patch ahead.
#include "fv_step.cuh"
#include "fv_x2.cuh"

// Resident CTAs per SM the register allocation is sized for (what the
// shared memory allows).
#ifndef FV_PAIRS_MINBLOCKS
#define FV_PAIRS_MINBLOCKS 5
#endif

namespace fv {
namespace {

// Geometry and shared-memory layout for interior size P (odd).
template <int P>
struct PairGeom {
  static_assert(P % 2 == 1 && P >= 3, "odd patch sizes");
  static constexpr int S = 5;                       // unknowns (3D Euler)
  static constexpr int NE = P + 2;                  // box cells per axis
  // SoA layout: cells x = 1 .. P+1 of a row (x = 0 and -1 never leave
  // registers) at columns x - 1; rows of RP floats, planes of PZ floats.
  // PZ is the smallest pitch >= RP * NE with PZ = -RP (mod 32): the P rows
  // of a y line pair, or of a z line pair, then fall on distinct banks.
  static constexpr int RP = P + 1;
  static constexpr int PZ = RP * NE + ((32 - RP) - (RP * NE) % 32 + 64) % 32;
  static constexpr int NSL = PZ * NE;               // floats per SoA quantity
  static constexpr int HP = (P + 1) / 2;            // x pairs of interior cells per row
  static constexpr int DP = 2 * HP;                 // flux-difference slots per row
  static constexpr int NROW = P * P;                // interior x rows
  // y and z flux differences of the interior cells, [v][z][y][slot] per
  // direction.  The z planes of the y block lie B1 floats apart, B1 = DP
  // (mod 32) with B1 >= P DP: the lanes storing the P lines of a y half-line
  // step then hit distinct banks (the z block's lines are DP apart already).
  static constexpr int B1 = P * DP + (DP - (P * DP) % 32 + 32) % 32;
  static constexpr int DGV1 = P * B1, DG2 = S * DGV1, DGV2 = NROW * DP;
  static constexpr int NDG = DG2 + S * DGV2;
  static constexpr int BOX = NE * NE * NE * S;      // cells of the staged box
  static constexpr int BOXP = (BOX + 3) / 4 * 4;
  // conversion items: x pairs of the interior rows (with their x halos),
  // which also compute the x faces, then those of the face-halo rows
  static constexpr int NRI = NROW * (HP + 1);       // interior-row items
  static constexpr int NA = NRI + 4 * P * HP;
  static constexpr int NHL = P * HP;                // y (or z) line pairs
  static constexpr int HA = (P + 1) / 2;            // faces of the first half of a line
  static constexpr int NC = NROW * HP;              // update items
  static constexpr int NT = 128;
  static constexpr int RA = (NA + NT - 1) / NT;     // conversion rounds
  // SoA quantities: state, u_y, u_z, p, c (E + p is recomputed from E and p
  // where it is read: the same add as in the conversion, the same bits)
  static constexpr int AQ = 0, AUY = 5, APR = 7, ACS = 8, NARR = 9;
  static constexpr int SMEM = kHdrBytes + 4 * (2 * BOXP + NARR * NSL + NDG);
  static_assert(NRI <= NT && NHL <= 16 && NC <= 96 && RA == 2, "roles sized for P = 5");
};

__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ void st2(float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; }
__device__ __forceinline__ unsigned umax(unsigned a, unsigned b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned fbits(float x) { return __float_as_uint(x); }
// |u| + c of a cell, as its IEEE bits (>= 0 or NaN: the sign bit is clear
// unless NaN, so unsigned maxima order them like the values)
__device__ __forceinline__ unsigned wave_bits(float u, float c) {
  return fbits(add_rn(fabsf(u), c));
}
constexpr unsigned kMagMask = 0x7FFFFFFFu;

// Primitives of two cells (Eq. 2), the operations of primitives() in
// fv_device.cuh on both halves.  The positivity of rho and p (checked there
// per cell) is accumulated instead: chk = max over the checked values of
// (bits - 1), unsigned, where 0 < x < inf <=> bits(x) - 1 < 0x7F7FFFFF; the
// masks keep cells that are no cells (m = 0) out of it.
struct Prim2 {
  f2 u[3], p, c, e;
};
__device__ __forceinline__ Prim2 prims2(const f2 (&q)[5], f2 gm1, f2 gamma, f2 mhalf,
                                        unsigned mlo, unsigned mhi, unsigned& chk) {
  Prim2 w;
  float r0, r1;
  f2_unpack(q[0], r0, r1);
  const f2 inv = f2_pack(recip(r0), recip(r1));
#pragma unroll
  for (int m = 0; m < 3; ++m) w.u[m] = mul2(q[1 + m], inv);
  f2 jj = mul2(q[1], w.u[0]);
  jj = fma2(q[2], w.u[1], jj);
  jj = fma2(q[3], w.u[2], jj);
  w.p = mul2(gm1, fma2(mhalf, jj, q[4]));
  w.e = add2(q[4], w.p);
  const f2 c2 = mul2(mul2(gamma, w.p), inv);
  float c0, c1;
  f2_unpack(c2, c0, c1);
  w.c = f2_pack(sqrt_t(c0), sqrt_t(c1));
  float p0, p1;
  f2_unpack(w.p, p0, p1);
  chk = umax(chk, (fbits(r0) - 1u) & mlo);
  chk = umax(chk, (fbits(p0) - 1u) & mlo);
  chk = umax(chk, (fbits(r1) - 1u) & mhi);
  chk = umax(chk, (fbits(p1) - 1u) & mhi);
  return w;
}
constexpr unsigned kBadChk = 0x7F7FFFFFu;

// A conversion item: two x-neighbouring cells of the box.
struct ItemA {
  int aos;    // float offset of the first cell in the staged box
  int slot;   // SoA slot of the first cell (even), or -1: not stored
  int valid;  // bit 0 / bit 1: the first / second cell is needed; 0: no item
};
template <int P>
__device__ __forceinline__ ItemA item_a(int t) {
  using G = PairGeom<P>;
  ItemA it{0, 0, 0};
  if (t >= G::NA) return it;
  int y, z, j;
  bool vlo = true, vhi = true;
  if (t < G::NROW * (G::HP + 1)) {  // interior row: cells x = -1 .. P + 1 in pairs
    const int r = t / (G::HP + 1);
    j = t - r * (G::HP + 1);
    y = 1 + r % P;
    z = 1 + r / P;
    vlo = j > 0;  // x = -1 is no cell
  } else {  // face-halo row: cells x = 1 .. P (+ the edge cell x = P + 1)
    const int u = t - G::NROW * (G::HP + 1);
    const int h = u / G::HP;
    j = 1 + (u - h * G::HP);
    if (h < 2 * P) {
      y = h < P ? 0 : P + 1;
      z = 1 + h % P;
    } else {
      const int g = h - 2 * P;
      z = g < P ? 0 : P + 1;
      y = 1 + g % P;
    }
    vhi = 2 * j <= P;
  }
  const int x0 = 2 * j - 1;
  it.aos = (x0 + G::NE * (y + G::NE * z)) * G::S;
  it.slot = j > 0 ? 2 * j - 2 + G::RP * y + G::PZ * z : -1;  // x = -1, 0: registers only
  it.valid = (vlo ? 1 : 0) | (vhi ? 2 : 0);
  return it;
}

// Two cells (or x-neighbouring lines) of a direction k as pairs: state with
// the momenta as (first transverse, normal, second transverse), and the
// primitives u_k, p, c, E + p.
struct Cell2 {
  f2 q0, qt1, qn, qt2, q4, u, p, c, e;
};
// The face fluxes G = 2F of two faces at once (Eq. 4, 5), in the operation
// order of the general kernel (fv_step.cuh).  g: rho, first transverse,
// normal, second transverse momentum, E.  bl / bh: bits of a per half.
__device__ __forceinline__ void flux2(const Cell2& L, const Cell2& R, f2 (&g)[5], unsigned& bl,
                                      unsigned& bh) {
  float uLl, uLh, cLl, cLh, uRl, uRh, cRl, cRh;
  f2_unpack(L.u, uLl, uLh);
  f2_unpack(L.c, cLl, cLh);
  f2_unpack(R.u, uRl, uRh);
  f2_unpack(R.c, cRl, cRh);
  bl = umax(wave_bits(uLl, cLl), wave_bits(uRl, cRl));
  bh = umax(wave_bits(uLh, cLh), wave_bits(uRh, cRh));
  const f2 am = f2_pack(__uint_as_float(bl), __uint_as_float(bh));
  const f2 sL = add2(L.u, am), sR = sub2(R.u, am), ps = add2(L.p, R.p);
  g[0] = fma2(L.q0, sL, mul2(R.q0, sR));
  g[1] = fma2(L.qt1, sL, mul2(R.qt1, sR));
  g[2] = fma2(L.qn, sL, fma2(R.qn, sR, ps));
  g[3] = fma2(L.qt2, sL, mul2(R.qt2, sR));
  g[4] = fma2(am, sub2(L.q4, R.q4), fma2(L.e, L.u, mul2(R.e, R.u)));
}

// A patch of the processing sequence: position, index, element offset.
struct Pat {
  long long pos, pid, off;
};
constexpr int kInfoOff = 448;  // shared slot of the patch two ahead
static_assert(kFaceSrcOff + 2 * 6 * (int)sizeof(FaceSrc) <= kInfoOff &&
                  kInfoOff + (int)sizeof(Pat) <= kHdrBytes,
              "header layout");

// The copy pipeline: two box buffers, each filled by a bulk copy (completion
// on its own mbarrier) and then by the halo gather.  The copy of a patch
// starts two patches ahead, as soon as its buffer has been converted; its
// halo cells are gathered one patch ahead, by warps 2 and 3 while warps 0
// and 1 compute the y and z face fluxes.
template <int P, bool STEP>
__global__ void __launch_bounds__(128, FV_PAIRS_MINBLOCKS) pairs_kernel(StepParams<float> a) {
  using G = PairGeom<P>;
  constexpr int S = G::S, NE = G::NE, RP = G::RP, PZ = G::PZ, NSL = G::NSL, HP = G::HP,
                DP = G::DP;
  constexpr unsigned FULL = 0xFFFFFFFFu;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // one per box buffer
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem_raw + kRedOff);
  FaceSrc* fs = reinterpret_cast<FaceSrc*>(smem_raw + kFaceSrcOff);  // [buffer][face]
  Pat* info = reinterpret_cast<Pat*>(smem_raw + kInfoOff);
  float* const box0 = reinterpret_cast<float*>(smem_raw + kHdrBytes);
  float* const soa = box0 + 2 * G::BOXP;
  float* const dg = soa + G::NARR * NSL;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  double dtv;
  if constexpr (STEP) {
    const double lam = order_value<float>(*a.lam_in);
    dtv = (a.cfl * a.dx) / (3.0 * lam);
    if (blockIdx.x == 0 && tid == 0) *a.dt_slot = dtv;
  } else {
    dtv = a.dt > 0.0 ? a.dt : *a.dt_dev;
  }
  const float mhr = neg_t((float)(0.5 * (dtv / a.dx)));  // -dt / (2 dx)
  const f2 mhr2 = f2_pack(mhr, mhr);
  const f2 gm1 = f2_pack(a.gm1, a.gm1), gam = f2_pack(a.gamma, a.gamma);
  const f2 mhalf = f2_pack(-0.5f, -0.5f);
  const bool want_lam = a.lam_patch != nullptr;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // the first valid position at or after `pos` (this CTA's stride); patches
  // that are invalid or of another size are reported and skipped
  auto next_valid = [&](long long pos) -> Pat {
    Pat r{pos, 0, 0};
    while (r.pos < a.i_end) {
      r.pid = a.order != nullptr ? (long long)a.order[r.pos] : r.pos;
      int pj = 0;
      int64_t offj = 0;
      const bool ok = patch_ok<float, 3>(a, r.pid, pj, offj);
      r.off = offj;
      if (ok && pj == P) break;
      atomicOr(a.status, ST_BAD_PATCH);
      r.pos += gridDim.x;
    }
    return r;
  };
  // the bulk copy of a patch into buffer b: in a time step only the span from
  // the first to the last interior cell (16-byte bounds; the face-halo cells
  // come from the gather), else the whole box but its ragged tail (which lies
  // in the last corner cell, never read)
  auto issue_box = [&](const Pat& pt, int b) {
    constexpr uint32_t lo = STEP ? ((1 + NE + NE * NE) * S * 4) & ~15u : 0u;
    constexpr uint32_t hi =
        STEP ? ((P + NE * P + NE * NE * P + 1) * S * 4 + 15) & ~15u : (G::BOX * 4) & ~15u;
    static_assert(hi <= G::BOX * 4 + 12 && hi <= G::BOXP * 4, "copy inside the box");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bar[b], hi - lo);
    bulk_copy_g2s(box0 + b * G::BOXP + lo / 4, a.in + pt.off + lo / 4, hi - lo, &bar[b]);
  };
  // warps 2, 3: the halo cells of faces 3 (w - 2) .. 3 (w - 2) + 2 of a patch
  // staged in buffer b, from sources resolved here (lanes 0-2)
  auto gather = [&](const Pat& pt, int b) {
    const int f0 = 3 * (warp - 2);
    FaceSrc* fsb = fs + 6 * b;
    if (lane < 3) fsb[f0 + lane] = face_source<float, 3, true>(a, pt.pid, P, pt.off, f0 + lane);
    __syncwarp();
    float* const bx = box0 + b * G::BOXP;
    const int ta = 1 + lane % P, tb = 1 + lane / P;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int f = f0 + i, k = f >> 1;
      const FaceSrc m = fsb[f];
      // the two transverse coordinates and the stride along k
      const int sk = k == 0 ? 1 : (k == 1 ? NE : NE * NE);
      const int tr = k == 0 ? NE * ta + NE * NE * tb : (k == 1 ? ta + NE * NE * tb : ta + NE * tb);
      if (lane < P * P) {
        float* dst = bx + (tr + ((f & 1) ? P + 1 : 0) * sk) * S;
        const float* src = a.in + m.off + (int64_t)(tr + m.ck * sk) * S;
        if (!m.neg) {
#pragma unroll
          for (int v = 0; v < S; ++v) cp_async_elem(dst + v, src + v);
        } else {  // wall: the normal momentum mirrored
#pragma unroll
          for (int v = 0; v < S; ++v) {
            if (v == 1 + k)
              dst[v] = neg_t(__ldg(src + v));
            else
              cp_async_elem(dst + v, src + v);
          }
        }
      }
    }
    cp_async_commit();
  };

  uint32_t parity = 0u, pending = 0u;  // bit b: buffer b
  bool timeout = false;
  unsigned chk = 0u, lam_next = 0u;
  auto wait_box = [&](int b) {
    if (mbar_wait_bounded(&bar[b], (parity >> b) & 1u, kWaitLimit)) {
      parity ^= 1u << b;
      pending &= ~(1u << b);
      return true;
    }
    timeout = true;
    return false;
  };

  Pat cur = next_valid(a.i_begin + blockIdx.x);
  Pat nx1 = cur.pos < a.i_end ? next_valid(cur.pos + gridDim.x) : cur;
  int s = 0;  // buffer of the current patch
  if (cur.pos < a.i_end) {
    if (tid == 0) issue_box(cur, 0);
    pending |= 1u;
    if (nx1.pos < a.i_end) {
      if (tid == 0) issue_box(nx1, 1);
      pending |= 2u;
    }
    if (wait_box(0) && STEP && warp >= 2) gather(cur, 0);
    cp_async_wait_all();
  }
  timeout = __syncthreads_or(timeout);
  if (timeout) cur.pos = a.i_end;

  // this thread's conversion items; the interior-row ones (round 0, t < NRI)
  // also compute the faces of the row between their cells and the next item's
  const ItemA ia0 = item_a<P>(tid), ia1 = item_a<P>(tid + G::NT);
  const bool xrow = tid < G::NRI;
  const int xr = tid / (HP + 1), xj = tid - (tid / (HP + 1)) * (HP + 1);
  const unsigned mflo = (xrow && xj >= 1) ? kMagMask : 0u;      // face x0 | x0+1 exists
  const unsigned mfhi = (xrow && xj <= HP - 1) ? kMagMask : 0u;  // face x0+1 | x0+2 exists

  while (cur.pos < a.i_end) {
    float* const box = box0 + s * G::BOXP;
    unsigned lmax = 0u;
    f2 dgx[5];  // x flux differences of this thread's update pair

    // ---- cells: state and primitives to SoA, two x-neighbours per item;
    //      the x faces of the interior rows ------------------------------------
    {
      f2 q[5];
#pragma unroll
      for (int v = 0; v < S; ++v) q[v] = f2_pack(box[ia0.aos + v], box[ia0.aos + S + v]);
      const Prim2 w = prims2(q, gm1, gam, mhalf, (ia0.valid & 1) ? ~0u : 0u,
                             (ia0.valid & 2) ? ~0u : 0u, chk);
      if (ia0.slot >= 0) {
        float* d = soa + ia0.slot;
#pragma unroll
        for (int v = 0; v < S; ++v) st2(d + (G::AQ + v) * NSL, q[v]);
        st2(d + G::AUY * NSL, w.u[1]);
        st2(d + (G::AUY + 1) * NSL, w.u[2]);
        st2(d + G::APR * NSL, w.p);
        st2(d + G::ACS * NSL, w.c);
      }
      // faces (x0 | x0+1) and (x0+1 | x0+2): left cells = this pair, right
      // cells = (second cell, the next item's first cell)
      auto nxt = [&](f2 v) {
        float lo, hi;
        f2_unpack(v, lo, hi);
        return f2_pack(hi, __shfl_down_sync(FULL, lo, 1));
      };
      const Cell2 L{q[0], q[2], q[1], q[3], q[4], w.u[0], w.p, w.c, w.e};
      const Cell2 R{nxt(q[0]), nxt(q[2]), nxt(q[1]), nxt(q[3]), nxt(q[4]),
                    nxt(w.u[0]), nxt(w.p), nxt(w.c), nxt(w.e)};
      f2 g[5];
      unsigned bl, bh;
      flux2(L, R, g, bl, bh);
      lmax = umax(lmax, bl & mflo);
      lmax = umax(lmax, bh & mfhi);
      // flux differences of cells x0 (G(x0+1/2) - G(x0-1/2), the latter the
      // previous item's second face) and x0+1, kept for the update of this
      // pair, which this thread does (with the pair's state)
      constexpr int PV[5] = {0, 2, 1, 3, 4};  // unknown of g[i]
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        float gl, gh;
        f2_unpack(g[i], gl, gh);
        const float gprev = __shfl_up_sync(FULL, gh, 1);
        dgx[PV[i]] = f2_pack(sub_rn(gl, gprev), sub_rn(gh, gl));
      }
    }
    if (ia1.valid) {
      f2 q[5];
#pragma unroll
      for (int v = 0; v < S; ++v) q[v] = f2_pack(box[ia1.aos + v], box[ia1.aos + S + v]);
      const Prim2 w = prims2(q, gm1, gam, mhalf, (ia1.valid & 1) ? ~0u : 0u,
                             (ia1.valid & 2) ? ~0u : 0u, chk);
      float* d = soa + ia1.slot;
#pragma unroll
      for (int v = 0; v < S; ++v) st2(d + (G::AQ + v) * NSL, q[v]);
      st2(d + G::AUY * NSL, w.u[1]);
      st2(d + (G::AUY + 1) * NSL, w.u[2]);
      st2(d + G::APR * NSL, w.p);
      st2(d + G::ACS * NSL, w.c);
    }
    __syncthreads();  // buffer s is converted: the copy two patches ahead may start

    // ---- y (warp 0) and z (warp 1) faces: half lines of x-neighbouring line
    //      pairs; warps 2, 3: the next patch's halo cells ----------------------
    if (warp < 2) {
      const int k = 1 + warp;
      const int h = lane >> 4, rem = lane & 15;
      const bool act = rem < G::NHL;
      const int t = rem / HP, j = rem - (rem / HP) * HP;
      const int s0 = 2 * j + (k == 1 ? PZ * (1 + t) : RP * (1 + t));
      const int st = k == 1 ? RP : PZ;                // SoA step along the line
      const unsigned hmask = 2 + 2 * j <= P ? kMagMask : 0u;  // second line real
      const int vn = 1 + k, vt2 = k == 1 ? 3 : 2;     // normal / 2nd transverse momentum
      auto load = [&](int b) {
        const float* sp = soa + s0 + b * st;
        const f2 e4 = ld2(sp + (G::AQ + 4) * NSL), pr = ld2(sp + G::APR * NSL);
        return Cell2{ld2(sp + G::AQ * NSL), ld2(sp + (G::AQ + 1) * NSL),
                     ld2(sp + (G::AQ + vn) * NSL), ld2(sp + (G::AQ + vt2) * NSL),
                     e4, ld2(sp + (G::AUY + k - 1) * NSL),
                     pr, ld2(sp + G::ACS * NSL), add2(e4, pr)};
      };
      // cell b of the line: k = 1: y = b, z = 1 + t; k = 2: y = 1 + t, z = b
      const int dgb = k == 1 ? t * G::B1 + 2 * j : G::DG2 + t * DP + 2 * j;
      const int dgs = k == 1 ? DP : P * DP;        // dG step along the line
      const int dgv = k == 1 ? G::DGV1 : G::DGV2;  // dG step per unknown
      auto store_dg = [&](int b, const f2 (&gpl)[5], const f2 (&gmi)[5]) {
        float* d = dg + dgb + (b - 1) * dgs;
        st2(d, sub2(gpl[0], gmi[0]));
        st2(d + 1 * dgv, sub2(gpl[1], gmi[1]));
        st2(d + vn * dgv, sub2(gpl[2], gmi[2]));
        st2(d + vt2 * dgv, sub2(gpl[3], gmi[3]));
        st2(d + 4 * dgv, sub2(gpl[4], gmi[4]));
      };
      f2 gfirst[5], glast[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) glast[v] = gfirst[v] = 0ull;
      if (act) {
        // half 0: faces 0 .. HA-1 (cells 0 .. HA); half 1: faces HA .. P
        const int b0 = h ? G::HA : 0;
        Cell2 Lc = load(b0);
#pragma unroll
        for (int f = 0; f < G::HA; ++f) {
          const Cell2 Rc = load(b0 + f + 1);
          f2 g[5];
          unsigned bl, bh;
          flux2(Lc, Rc, g, bl, bh);
          lmax = umax(lmax, bl & kMagMask);
          lmax = umax(lmax, bh & hmask);
          if (f > 0)
            store_dg(b0 + f, g, glast);
          else {
#pragma unroll
            for (int v = 0; v < 5; ++v) gfirst[v] = g[v];
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) glast[v] = g[v];
          Lc = Rc;
        }
      }
      // cell HA: G(face HA) (half 1's first) - G(face HA-1) (half 0's last)
      f2 gother[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float lo, hi;
        f2_unpack(glast[v], lo, hi);
        gother[v] = f2_pack(__shfl_xor_sync(FULL, lo, 16), __shfl_xor_sync(FULL, hi, 16));
      }
      if (act && h == 1) store_dg(G::HA, gfirst, gother);
    } else {
      if (nx1.pos < a.i_end) {
        if (wait_box(s ^ 1) && STEP) gather(nx1, s ^ 1);
      }
      if (tid == 96) {
        // the patch two ahead: find it, start its copy into buffer s
        const Pat nx2 = nx1.pos < a.i_end ? next_valid(nx1.pos + gridDim.x) : nx1;
        *info = nx2;
        if (nx2.pos < a.i_end) issue_box(nx2, s);
      }
    }
    if (want_lam) {
      const unsigned long long m = warp_max_u64((unsigned long long)lmax);
      if (lane == 0) red[warp] = m;
    }
    __syncthreads();  // flux differences complete

    const Pat nx2 = *info;
    if (nx2.pos < a.i_end) pending |= 1u << s;
    if (want_lam && tid == 0) {
      unsigned long long mm = red[0];
#pragma unroll
      for (int w = 1; w < 4; ++w) mm = red[w] > mm ? red[w] : mm;
      a.lam_patch[cur.pid] = order_value<float>(mm);
    }

    // ---- update: Q - (dt / 2dx) sum_k (G+ - G-), x pairs of cells, by the
    //      threads whose conversion item was the pair (interior rows, j >= 1)
    if (xrow && xj >= 1) {
      const int r = xr, j = xj - 1;
      const int y = 1 + r % P, z = 1 + r / P;
      const bool hi = 2 + 2 * j <= P;  // the second cell is a cell of the patch
      const unsigned mhi = hi ? ~0u : 0u;
      f2 acc[5];
#pragma unroll
      for (int v = 0; v < S; ++v) acc[v] = dgx[v];
#pragma unroll
      for (int v = 0; v < S; ++v)
        acc[v] = add2(acc[v], ld2(dg + v * G::DGV1 + (y - 1) * DP + (z - 1) * G::B1 + 2 * j));
#pragma unroll
      for (int v = 0; v < S; ++v)
        acc[v] = add2(acc[v], ld2(dg + G::DG2 + v * G::DGV2 + (y - 1) * DP + (z - 1) * P * DP + 2 * j));
      const int slot = 2 * j + RP * y + PZ * z;
      f2 qn[5];
#pragma unroll
      for (int v = 0; v < S; ++v) qn[v] = fma2(mhr2, acc[v], ld2(soa + (G::AQ + v) * NSL + slot));
      float* dst = a.out + cur.off + (int64_t)((1 + 2 * j) + NE * (y + NE * z)) * S;
#pragma unroll
      for (int v = 0; v < S; ++v) {
        float lo, hv;
        f2_unpack(qn[v], lo, hv);
        dst[v] = lo;
        if (hi) dst[S + v] = hv;
      }
      if constexpr (STEP) {
        // primitives and wave speeds of the new state (next CFL maximum)
        const Prim2 w = prims2(qn, gm1, gam, mhalf, ~0u, mhi, chk);
        float cl, ch;
        f2_unpack(w.c, cl, ch);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float ul, uh;
          f2_unpack(w.u[k], ul, uh);
          lam_next = umax(lam_next, wave_bits(ul, cl) & kMagMask);
          lam_next = umax(lam_next, wave_bits(uh, ch) & kMagMask & mhi);
        }
        if (a.prim_out != nullptr) {
          float* po = a.prim_out + cur.pid * a.prim_stride + 2 * j + P * (y - 1) +
                      P * P * (z - 1);
          constexpr int NI = P * P * P;
          const f2 vals[6] = {w.u[0], w.u[1], w.u[2], w.p, w.c, w.e};
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            float lo, hv;
            f2_unpack(vals[m], lo, hv);
            po[m * NI] = lo;
            if (hi) po[m * NI + 1] = hv;
          }
        }
      }
    }
    if (nx1.pos < a.i_end) {
      if (warp < 2) wait_box(s ^ 1);  // the others observed it before gathering
      cp_async_wait_all();
    }
    timeout = __syncthreads_or(timeout);
    if (timeout) break;
    cur = nx1;
    nx1 = nx2;
    s ^= 1;
  }
  if (timeout) {
    if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
    if (pending & 1u) mbar_wait_bounded(&bar[0], parity & 1u, kWaitLimit);
    if (pending & 2u) mbar_wait_bounded(&bar[1], (parity >> 1) & 1u, kWaitLimit);
    cp_async_wait_all();
    return;
  }
  if (chk >= kBadChk) atomicOr(a.status, ST_NONPHYSICAL);
  if constexpr (STEP) {
    const unsigned long long m = warp_max_u64((unsigned long long)lam_next);
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (tid == 0) {
      unsigned long long mm = red[0];
#pragma unroll
      for (int w = 1; w < 4; ++w) mm = red[w] > mm ? red[w] : mm;
      atomicMax(a.lam_next, mm);
    }
  }
}

template <int P, bool STEP>
cudaError_t pairs_smem_attr() {
  static int set_bytes[64] = {0};
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && set_bytes[dev] >= PairGeom<P>::SMEM) return cudaSuccess;
  e = cudaFuncSetAttribute(pairs_kernel<P, STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           PairGeom<P>::SMEM);
  if (e == cudaSuccess && dev >= 0 && dev < 64) set_bytes[dev] = PairGeom<P>::SMEM;
  return e;
}

template <int P, bool STEP>
cudaError_t launch_pairs_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
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
  cudaError_t e = pairs_smem_attr<P, STEP>();
  if (e != cudaSuccess) return e;
  pairs_kernel<P, STEP><<<grid, PairGeom<P>::NT, PairGeom<P>::SMEM, h->stream>>>(a);
  return cudaGetLastError();
}

template <int P, bool STEP>
cudaError_t occupancy_pairs_t(int* bps) {
  cudaError_t e = pairs_smem_attr<P, STEP>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, pairs_kernel<P, STEP>,
                                                       PairGeom<P>::NT, PairGeom<P>::SMEM);
}

}  // namespace

bool pairs_class(const fv_batch* h, int p) {
  return h->prec == FV_FP32 && h->d == 3 && h->s == 5 && p == 5;
}

bool pairs_eligible(const fv_batch* h, const UpdateLaunch& l) {
  const int mode = step_mode(l);
  return pairs_class(h, l.uniform_p) && mode != kModePrim && l.corr == nullptr &&
         l.dx_patch == nullptr && !l.local_cfl && (mode == kModeStep || l.prim_out == nullptr);
}

cudaError_t launch_pairs(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return step_mode(l) == kModeStep ? launch_pairs_t<5, true>(h, l, grid)
                                   : launch_pairs_t<5, false>(h, l, grid);
}

cudaError_t pairs_occupancy(int mode, int* bps) {
  return mode == kModeStep ? occupancy_pairs_t<5, true>(bps) : occupancy_pairs_t<5, false>(bps);
}

}  // namespace fv
