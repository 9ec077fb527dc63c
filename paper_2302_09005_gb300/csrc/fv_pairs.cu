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
//    (u, p, c, E + p) of every interior and face-halo cell, each quantity a
//    box of x rows padded to a multiple of four floats with cell x at
//    column x + 1, so that a thread reads a whole x row of a quantity with
//    128-bit loads, and two x-neighbours with one 64-bit load;
//  * packed arithmetic: two x-neighbouring cells (or faces) are computed
//    together with the f32x2 instructions (fv_x2.cuh): one instruction for
//    both elements, each rounded as the scalar operation;
//  * fixed indexing: every patch of the launch has the same size, so each
//    thread's cells, faces and shared-memory offsets are computed once per
//    launch, before the patch loop;
//  * roles: all warps convert the cells (x pairs); warp 0 then walks the x
//    lines of cells (a row in registers, every face once, scalar), warp 1
//    the y and z lines in x pairs (packed), each keeping the flux difference
//    G+ - G- of every cell of its line, while warps 2 and 3 gather the halo
//    cells of the next patch; warps 0-2 then update the cells in x pairs
//    (three differences per unknown, fixed order x, y, z) and convert the
//    new state for the next CFL maximum;
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
  static constexpr int PX = (P + 3 + 3) / 4 * 4;    // SoA row pitch (cell x at column x + 1)
  static constexpr int NSL = PX * NE * NE;          // floats per SoA quantity
  static constexpr int HP = (P + 1) / 2;            // x pairs of interior cells per row
  static constexpr int DP = 2 * HP;                 // flux-difference slots per row
  static constexpr int NROW = P * P;                // interior x rows
  static constexpr int NDG = 3 * S * NROW * DP;     // flux differences [k][v][row][slot]
  static constexpr int BOX = NE * NE * NE * S;      // cells of the staged box
  static constexpr int BOXP = (BOX + 3) / 4 * 4;
  // conversion items: x pairs of the interior rows (with their x halos) and
  // of the face-halo rows
  static constexpr int NA = NROW * (HP + 1) + 4 * P * HP;
  static constexpr int NYZ = 2 * P * HP;            // y and z line pairs
  static constexpr int NC = NROW * HP;              // update items
  static constexpr int NT = 128;
  static constexpr int RA = (NA + NT - 1) / NT;     // conversion rounds
  // SoA quantities: state, velocities, p, c, E + p
  static constexpr int AQ = 0, AU = 5, APR = 8, ACS = 9, AEP = 10, NARR = 11;
  static constexpr int SMEM = kHdrBytes + 4 * (2 * BOXP + NARR * NSL + NDG);
  static_assert(NROW <= 32 && NYZ <= 32 && NC <= 96, "roles sized for P <= 5");
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
  int slot;   // SoA column of the first cell (even)
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
  it.slot = 2 * j + G::PX * (y + G::NE * z);
  it.valid = (vlo ? 1 : 0) | (vhi ? 2 : 0);
  return it;
}

// The copy pipeline: two box buffers, each filled by a bulk copy (completion
// on its own mbarrier) and then by the halo gather.  The copy of a patch
// starts two patches ahead, as soon as its buffer has been converted; its
// halo cells are gathered one patch ahead, by warps 2 and 3 while warps 0
// and 1 compute the face fluxes.
template <int P, bool STEP>
__global__ void __launch_bounds__(128, FV_PAIRS_MINBLOCKS) pairs_kernel(StepParams<float> a) {
  using G = PairGeom<P>;
  constexpr int S = G::S, NE = G::NE, PX = G::PX, NSL = G::NSL, HP = G::HP, DP = G::DP,
                NROW = G::NROW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // one per box buffer
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem_raw + kRedOff);
  FaceSrc* fs = reinterpret_cast<FaceSrc*>(smem_raw + kFaceSrcOff);  // [buffer][face]
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

  auto pid_of = [&](int64_t pos) -> int64_t {
    return a.order != nullptr ? (int64_t)a.order[pos] : pos;
  };
  struct Pat {
    int64_t pos, pid, off;
  };
  // the first valid position at or after `pos` (this CTA's stride)
  auto next_valid = [&](int64_t pos) -> Pat {
    Pat r{pos, 0, 0};
    int pj = 0;
    while (r.pos < a.i_end) {
      r.pid = pid_of(r.pos);
      if (patch_ok<float, 3>(a, r.pid, pj, r.off)) {
        if (pj == P) break;
        if (tid == 0) atomicOr(a.status, ST_BAD_PATCH);
      }
      r.pos += gridDim.x;
    }
    return r;
  };
  auto issue_box = [&](const Pat& pt, int b) {
    issue_stage<float, 3, false>(a, pt.pid, P, pt.off,
                                 Stage<float>{box0 + b * G::BOXP, nullptr, nullptr}, &bar[b]);
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
  Pat nx1 = next_valid(cur.pos + gridDim.x);
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

  // per-thread indexing, fixed for the launch
  ItemA ia[G::RA];
#pragma unroll
  for (int r = 0; r < G::RA; ++r) ia[r] = item_a<P>(tid + r * G::NT);

  while (cur.pos < a.i_end) {
    const Pat nx2 = nx1.pos < a.i_end ? next_valid(nx1.pos + gridDim.x) : nx1;
    float* const box = box0 + s * G::BOXP;

    // ---- cells: state and primitives to SoA, two x-neighbours per item ----
#pragma unroll
    for (int r = 0; r < G::RA; ++r) {
      const ItemA it = ia[r];
      if (it.valid) {
        f2 q[5];
#pragma unroll
        for (int v = 0; v < S; ++v) q[v] = f2_pack(box[it.aos + v], box[it.aos + S + v]);
        const Prim2 w = prims2(q, gm1, gam, mhalf, (it.valid & 1) ? ~0u : 0u,
                               (it.valid & 2) ? ~0u : 0u, chk);
        float* d = soa + it.slot;
#pragma unroll
        for (int v = 0; v < S; ++v) st2(d + (G::AQ + v) * NSL, q[v]);
#pragma unroll
        for (int m = 0; m < 3; ++m) st2(d + (G::AU + m) * NSL, w.u[m]);
        st2(d + G::APR * NSL, w.p);
        st2(d + G::ACS * NSL, w.c);
        st2(d + G::AEP * NSL, w.e);
      }
    }
    __syncthreads();  // buffer s is converted: the copy two patches ahead may start

    if (nx2.pos < a.i_end) {
      if (tid == 0) issue_box(nx2, s);
      pending |= 1u << s;
    }

    // ---- faces: flux differences G+ - G- of every cell, per direction -------
    unsigned lmax = 0u;
    if (warp == 0) {
      if (lane < NROW) {
        // x line: the row's cells x = 0 .. P+1 in registers (columns 1 .. P+2)
        const int rb = PX * ((1 + lane % P) + NE * (1 + lane / P));
        float c[9][PX];
#pragma unroll
        for (int qi = 0; qi < 9; ++qi) {
          const int arr = qi < 5 ? G::AQ + qi : (qi == 5 ? G::AU : G::APR + (qi - 6));
#pragma unroll
          for (int c4 = 0; c4 < PX / 4; ++c4) {
            const float4 v4 = *reinterpret_cast<const float4*>(soa + arr * NSL + rb + 4 * c4);
            c[qi][4 * c4] = v4.x;
            c[qi][4 * c4 + 1] = v4.y;
            c[qi][4 * c4 + 2] = v4.z;
            c[qi][4 * c4 + 3] = v4.w;
          }
        }
        float gp[5], dgp[5];  // previous face's G; flux difference of an even slot
        float* const drow = dg + lane * DP;
#pragma unroll
        for (int f = 0; f <= P; ++f) {
          const int L = f + 1, R = f + 2;  // columns of the face's two cells
          const float uL = c[5][L], pL = c[6][L], cL = c[7][L], eL = c[8][L];
          const float uR = c[5][R], pR = c[6][R], cR = c[7][R], eR = c[8][R];
          const unsigned amb = umax(wave_bits(uL, cL), wave_bits(uR, cR));
          lmax = umax(lmax, amb & kMagMask);
          const float am = __uint_as_float(amb);
          const float sL = add_rn(uL, am), sR = sub_rn(uR, am), ps = add_rn(pL, pR);
          float g[5];
          g[0] = fmaf(c[0][L], sL, mul_rn(c[0][R], sR));
          g[1] = fmaf(c[1][L], sL, fmaf(c[1][R], sR, ps));
          g[2] = fmaf(c[2][L], sL, mul_rn(c[2][R], sR));
          g[3] = fmaf(c[3][L], sL, mul_rn(c[3][R], sR));
          g[4] = fmaf(am, sub_rn(c[4][L], c[4][R]), fmaf(eL, uL, mul_rn(eR, uR)));
          if (f > 0) {
            // cell x = f (slot f - 1): slots are stored in pairs; the last
            // cell's pair holds a zero for the column beyond the row
            const int sl = f - 1;
#pragma unroll
            for (int v = 0; v < S; ++v) {
              const float dv = sub_rn(g[v], gp[v]);
              if (sl % 2 == 0) {
                if (sl == P - 1)
                  st2(drow + v * NROW * DP + sl, f2_pack(dv, 0.0f));
                else
                  dgp[v] = dv;
              } else {
                st2(drow + v * NROW * DP + sl - 1, f2_pack(dgp[v], dv));
              }
            }
          }
#pragma unroll
          for (int v = 0; v < S; ++v) gp[v] = g[v];
        }
      }
    } else if (warp == 1) {
      if (lane < G::NYZ) {
        // y or z line pair: cells b = 0 .. P+1 of two x-neighbouring lines
        const int k = lane < P * HP ? 1 : 2;
        const int rem = lane - (k - 1) * P * HP;
        const int t = rem / HP, j = rem - t * HP;
        const int s0 = 2 + 2 * j + (k == 1 ? PX * NE * (1 + t) : PX * (1 + t));
        const int st = k == 1 ? PX : PX * NE;           // SoA step along the line
        const int r0 = k == 1 ? P * t : t;              // interior row of cell b = 1
        const int rs = k == 1 ? 1 : P;                  // row step along the line
        const unsigned hmask = 2 + 2 * j <= P ? kMagMask : 0u;  // second line real
        const int vn = 1 + k, vt2 = k == 1 ? 3 : 2;     // normal / 2nd transverse momentum
        struct C2 {
          f2 q0, qt1, qn, qt2, q4, u, p, c, e;
        };
        auto load = [&](int b) {
          const float* sp = soa + s0 + b * st;
          C2 x;
          x.q0 = ld2(sp + G::AQ * NSL);
          x.qt1 = ld2(sp + (G::AQ + 1) * NSL);
          x.qn = ld2(sp + (G::AQ + vn) * NSL);
          x.qt2 = ld2(sp + (G::AQ + vt2) * NSL);
          x.q4 = ld2(sp + (G::AQ + 4) * NSL);
          x.u = ld2(sp + (G::AU + k) * NSL);
          x.p = ld2(sp + G::APR * NSL);
          x.c = ld2(sp + G::ACS * NSL);
          x.e = ld2(sp + G::AEP * NSL);
          return x;
        };
        float* const dbase = dg + (k * S * NROW + r0) * DP + 2 * j;
        C2 Lc = load(0);
        f2 gp[5];
#pragma unroll
        for (int f = 0; f <= P; ++f) {
          const C2 Rc = load(f + 1);
          float uLl, uLh, cLl, cLh, uRl, uRh, cRl, cRh;
          f2_unpack(Lc.u, uLl, uLh);
          f2_unpack(Lc.c, cLl, cLh);
          f2_unpack(Rc.u, uRl, uRh);
          f2_unpack(Rc.c, cRl, cRh);
          const unsigned bl = umax(wave_bits(uLl, cLl), wave_bits(uRl, cRl));
          const unsigned bh = umax(wave_bits(uLh, cLh), wave_bits(uRh, cRh));
          lmax = umax(lmax, bl & kMagMask);
          lmax = umax(lmax, bh & hmask);
          const f2 am = f2_pack(__uint_as_float(bl), __uint_as_float(bh));
          const f2 sL = add2(Lc.u, am), sR = sub2(Rc.u, am), ps = add2(Lc.p, Rc.p);
          f2 g[5];  // unknowns 0, 1 (x momentum), normal, second transverse, 4
          g[0] = fma2(Lc.q0, sL, mul2(Rc.q0, sR));
          g[1] = fma2(Lc.qt1, sL, mul2(Rc.qt1, sR));
          g[2] = fma2(Lc.qn, sL, fma2(Rc.qn, sR, ps));
          g[3] = fma2(Lc.qt2, sL, mul2(Rc.qt2, sR));
          g[4] = fma2(am, sub2(Lc.q4, Rc.q4), fma2(Lc.e, Lc.u, mul2(Rc.e, Rc.u)));
          if (f > 0) {
            // cell b = f of both lines: G(face f) - G(face f - 1)
            float* d = dbase + (f - 1) * rs * DP;
            st2(d, sub2(g[0], gp[0]));
            st2(d + 1 * NROW * DP, sub2(g[1], gp[1]));
            st2(d + vn * NROW * DP, sub2(g[2], gp[2]));
            st2(d + vt2 * NROW * DP, sub2(g[3], gp[3]));
            st2(d + 4 * NROW * DP, sub2(g[4], gp[4]));
          }
#pragma unroll
          for (int v = 0; v < S; ++v) gp[v] = g[v];
          Lc = Rc;
        }
      }
    } else if (nx1.pos < a.i_end) {
      // the next patch: its box (copied a patch ago), its halo cells
      if (wait_box(s ^ 1) && STEP) gather(nx1, s ^ 1);
    }
    if (want_lam && warp < 2) {
      const unsigned long long m = warp_max_u64((unsigned long long)lmax);
      if (lane == 0) red[warp] = m;
    }
    __syncthreads();  // flux differences complete

    if (want_lam && tid == 0)
      a.lam_patch[cur.pid] = order_value<float>(red[0] > red[1] ? red[0] : red[1]);

    // ---- update: Q - (dt / 2dx) sum_k (G+ - G-), x pairs of cells ----------
    if (tid < G::NC) {
      const int r = tid / HP, j = tid - (tid / HP) * HP;
      const int y = 1 + r % P, z = 1 + r / P;
      const bool hi = 2 + 2 * j <= P;  // the second cell is a cell of the patch
      const unsigned mhi = hi ? ~0u : 0u;
      f2 acc[5];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int v = 0; v < S; ++v) {
          const f2 d2 = ld2(dg + ((k * S + v) * NROW + r) * DP + 2 * j);
          acc[v] = k == 0 ? d2 : add2(acc[v], d2);
        }
      }
      const int slot = 2 + 2 * j + PX * (y + NE * z);
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
