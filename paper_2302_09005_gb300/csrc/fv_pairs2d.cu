// fv_pairs2d.cu -- the FP32 time step / update of a launch whose patches all
// have one 2D size (p = 5: a size class of the schedule, or a uniform batch
// after fv_batch_plan), one warp per patch.  Same method, same operations in
// the same order as the general kernel (fv_step.cuh; Eq. 2-5, Algorithm 1
// steps 5-10), so the results are bitwise the same.  A 5 x 5 patch is 25
// cells, 60 faces: small enough for one warp, so the CTA is one warp and its
// barriers cost next to nothing, with up to 32 patches in flight per SM.
// Per patch:
//
//  * the box arrives by one bulk copy (TMA engine, mbarrier completion) two
//    patches ahead; in a time step the face-halo cells of the next patch are
//    gathered with cp.async by the lanes while the y faces of the current
//    one are computed;
//  * conversion: 26 lanes take an x pair of cells each (the interior rows
//    with their x halos, and the face-halo rows), compute the primitives of
//    both cells with the packed f32x2 instructions (fv_x2.cuh), keep the
//    state in registers and store what the y faces read (state, u_y, p, c)
//    in structure-of-arrays form; the interior-row lanes also compute the x
//    faces between their cells and the next lane's (warp shuffles) and keep
//    the x flux differences of their pair in registers;
//  * y faces: 18 lanes, one face of an x pair of columns each, store G;
//  * update: the 15 interior-row lanes owning a pair of interior cells add
//    the y differences to their x differences (x then y), take one FMA with
//    -dt / (2 dx) on the state they hold, and convert the new state for the
//    next CFL maximum.
#include "fv_step.cuh"
#include "fv_x2.cuh"

// Resident CTAs (warps) per SM the register allocation is sized for.
#ifndef FV_PAIRS2D_MINBLOCKS
#define FV_PAIRS2D_MINBLOCKS 24
#endif

namespace fv {
namespace {

// Geometry and shared-memory layout for interior size P (odd).
template <int P>
struct Geom2 {
  static_assert(P % 2 == 1 && P >= 3, "odd patch sizes");
  static constexpr int S = 4;                   // unknowns (2D Euler)
  static constexpr int NE = P + 2;              // box cells per axis
  // SoA: cells x = 1 .. P+1 of a row at columns x - 1, rows y = 0 .. P+1
  static constexpr int RP = P + 1;
  static constexpr int NSL = RP * NE;           // floats per SoA quantity
  static constexpr int HP = (P + 1) / 2;        // x pairs of interior cells per row
  static constexpr int NRI = P * (HP + 1);      // interior-row items (x = -1 .. P+1)
  static constexpr int NA = NRI + 2 * HP;       // + the face-halo rows y = 0, P+1
  static constexpr int NF = (P + 1) * HP;       // y faces of the x pairs of columns
  static constexpr int BOX = NE * NE * S;
  static constexpr int BOXP = (BOX + 3) / 4 * 4;
  // SoA quantities: state, u_y, p, c (E + p recomputed where it is read)
  static constexpr int AQ = 0, AUY = 4, APR = 5, ACS = 6, NARR = 7;
  static constexpr int GW = 2 * HP;             // y-face G: [v][face][2 HP]
  static constexpr int NG = S * (P + 1) * GW;
  static constexpr int SMEM = kHdrBytes + 4 * (2 * BOXP + NARR * NSL + NG);
  static constexpr int NT = 32;
  static_assert(NA <= NT && NF <= NT, "one warp per patch");
};

__device__ __forceinline__ f2 ld2(const float* p) { return *reinterpret_cast<const f2*>(p); }
__device__ __forceinline__ void st2(float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; }
__device__ __forceinline__ unsigned umax(unsigned a, unsigned b) { return a > b ? a : b; }
__device__ __forceinline__ unsigned fbits(float x) { return __float_as_uint(x); }
// |u| + c of a cell as its IEEE bits (>= 0 or NaN, so unsigned maxima order
// them like the values)
__device__ __forceinline__ unsigned wave_bits(float u, float c) {
  return fbits(add_rn(fabsf(u), c));
}
constexpr unsigned kMagMask = 0x7FFFFFFFu;
// positivity of rho and p accumulated as max(bits - 1): 0 < x < inf <=>
// bits(x) - 1 < 0x7F7FFFFF
constexpr unsigned kBadChk = 0x7F7FFFFFu;

// Primitives of two cells (Eq. 2), the operations of primitives<float, 2>()
// in fv_device.cuh on both halves; the masks keep non-cells out of chk.
struct Prim2 {
  f2 u[2], p, c, e;
};
__device__ __forceinline__ Prim2 prims2(const f2 (&q)[4], f2 gm1, f2 gamma, f2 mhalf,
                                        unsigned mlo, unsigned mhi, unsigned& chk) {
  Prim2 w;
  float r0, r1;
  f2_unpack(q[0], r0, r1);
  const f2 inv = f2_pack(recip(r0), recip(r1));
  w.u[0] = mul2(q[1], inv);
  w.u[1] = mul2(q[2], inv);
  f2 jj = mul2(q[1], w.u[0]);
  jj = fma2(q[2], w.u[1], jj);
  w.p = mul2(gm1, fma2(mhalf, jj, q[3]));
  w.e = add2(q[3], w.p);
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

// Two cells of a direction k as pairs: rho, transverse and normal momentum,
// E, and u_k, p, c, E + p.
struct Cell2 {
  f2 q0, qt, qn, q3, u, p, c, e;
};
// G = 2F of two faces (Eq. 4, 5) in the general kernel's operation order;
// g: rho, transverse momentum, normal momentum, E; bl / bh: bits of a.
__device__ __forceinline__ void flux2(const Cell2& L, const Cell2& R, f2 (&g)[4], unsigned& bl,
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
  g[1] = fma2(L.qt, sL, mul2(R.qt, sR));
  g[2] = fma2(L.qn, sL, fma2(R.qn, sR, ps));
  g[3] = fma2(am, sub2(L.q3, R.q3), fma2(L.e, L.u, mul2(R.e, R.u)));
}

// A conversion item: two x-neighbouring cells of the box.
struct ItemA {
  int aos;    // float offset of the first cell in the staged box
  int slot;   // SoA slot of the first cell, or -1: not stored
  int valid;  // bit 0 / bit 1: the first / second cell is a needed cell
};
template <int P>
__device__ __forceinline__ ItemA item_a(int t) {
  using G = Geom2<P>;
  ItemA it{0, 0, 0};
  if (t >= G::NA) return it;
  int y, j;
  bool vlo = true, vhi = true;
  if (t < G::NRI) {  // interior row y: cells x = -1 .. P + 1 in pairs
    const int r = t / (G::HP + 1);
    j = t - r * (G::HP + 1);
    y = 1 + r;
    vlo = j > 0;  // x = -1 is no cell
  } else {  // face-halo row y = 0 or P + 1: cells x = 1 .. P (+ a corner)
    const int u = t - G::NRI;
    const int h = u / G::HP;
    j = 1 + (u - h * G::HP);
    y = h ? P + 1 : 0;
    vhi = 2 * j <= P;
  }
  const int x0 = 2 * j - 1;
  it.aos = (x0 + G::NE * y) * G::S;
  it.slot = j > 0 ? 2 * j - 2 + G::RP * y : -1;
  it.valid = (vlo ? 1 : 0) | (vhi ? 2 : 0);
  return it;
}

struct Pat {
  long long pos, pid, off;
};

template <int P, bool STEP>
__global__ void __launch_bounds__(32, FV_PAIRS2D_MINBLOCKS) pairs2d_kernel(StepParams<float> a) {
  using G = Geom2<P>;
  constexpr int S = G::S, NE = G::NE, RP = G::RP, NSL = G::NSL, HP = G::HP, GW = G::GW;
  constexpr unsigned FULL = 0xFFFFFFFFu;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // one per box buffer
  FaceSrc* fs = reinterpret_cast<FaceSrc*>(smem_raw + kFaceSrcOff);  // [buffer][face]
  float* const box0 = reinterpret_cast<float*>(smem_raw + kHdrBytes);
  float* const soa = box0 + 2 * G::BOXP;
  float* const gy = soa + G::NARR * NSL;
  const int lane = threadIdx.x;

  double dtv;
  if constexpr (STEP) {
    const double lam = order_value<float>(*a.lam_in);
    dtv = (a.cfl * a.dx) / (2.0 * lam);
    if (blockIdx.x == 0 && lane == 0) *a.dt_slot = dtv;
  } else {
    dtv = a.dt > 0.0 ? a.dt : *a.dt_dev;
  }
  const float mhr = neg_t((float)(0.5 * (dtv / a.dx)));  // -dt / (2 dx)
  const f2 mhr2 = f2_pack(mhr, mhr);
  const f2 gm1 = f2_pack(a.gm1, a.gm1), gam = f2_pack(a.gamma, a.gamma);
  const f2 mhalf = f2_pack(-0.5f, -0.5f);
  const bool want_lam = a.lam_patch != nullptr;

  if (lane == 0) {
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
      const bool ok = patch_ok<float, 2>(a, r.pid, pj, offj);
      r.off = offj;
      if (ok && pj == P) break;
      atomicOr(a.status, ST_BAD_PATCH);
      r.pos += gridDim.x;
    }
    return r;
  };
  // the bulk copy of a patch into buffer b: in a time step the span from the
  // first to the last interior cell (16-byte bounds; the face-halo cells come
  // from the gather), else the whole box
  auto issue_box = [&](const Pat& pt, int b) {
    constexpr uint32_t lo = STEP ? ((1 + NE) * S * 4) & ~15u : 0u;
    constexpr uint32_t hi = STEP ? ((P + NE * P + 1) * S * 4 + 15) & ~15u : (G::BOX * 4) & ~15u;
    static_assert(hi <= G::BOX * 4 && hi <= G::BOXP * 4 && lo < hi, "copy inside the box");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bar[b], hi - lo);
    bulk_copy_g2s(box0 + b * G::BOXP + lo / 4, a.in + pt.off + lo / 4, hi - lo, &bar[b]);
  };
  // the face-halo cells of a patch staged in buffer b: lanes 0-3 resolve the
  // four faces' sources, lanes 0 .. 4P-1 copy one cell each
  auto gather = [&](const Pat& pt, int b) {
    FaceSrc* fsb = fs + 6 * b;
    if (lane < 4) fsb[lane] = face_source<float, 2, true>(a, pt.pid, P, pt.off, lane);
    __syncwarp();
    if (lane < 4 * P) {
      float* const bx = box0 + b * G::BOXP;
      const int f = lane / P, k = f >> 1, ta = 1 + (lane - f * P);
      const FaceSrc m = fsb[f];
      const int sk = k == 0 ? 1 : NE;
      const int tr = k == 0 ? NE * ta : ta;
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
    if (lane == 0) issue_box(cur, 0);
    pending |= 1u;
    if (nx1.pos < a.i_end) {
      if (lane == 0) issue_box(nx1, 1);
      pending |= 2u;
    }
    if (wait_box(0) && STEP) gather(cur, 0);
    cp_async_wait_all();
  }
  timeout = __syncthreads_or(timeout);
  if (timeout) cur.pos = a.i_end;

  // this lane's conversion item; the interior-row ones also compute the x
  // faces between their cells and the next lane's
  const ItemA ia = item_a<P>(lane);
  const bool xrow = lane < G::NRI;
  const int xr = lane / (HP + 1), xj = lane - (lane / (HP + 1)) * (HP + 1);
  const unsigned mflo = (xrow && xj >= 1) ? kMagMask : 0u;      // face x0 | x0+1 exists
  const unsigned mfhi = (xrow && xj <= HP - 1) ? kMagMask : 0u;  // face x0+1 | x0+2 exists
  // this lane's y face: between rows yf and yf + 1 of the column pair yj
  const bool yact = lane < G::NF;
  const int yf = lane / HP, yj = lane - (lane / HP) * HP;
  const unsigned yhi = 2 + 2 * yj <= P ? kMagMask : 0u;  // the second column is interior

  while (cur.pos < a.i_end) {
    float* const box = box0 + s * G::BOXP;
    unsigned lmax = 0u;
    f2 q[4];    // this lane's pair of cells (the update pair of interior-row lanes)
    f2 dgx[4];  // its x flux differences
    {
#pragma unroll
      for (int v = 0; v < S; ++v) q[v] = f2_pack(box[ia.aos + v], box[ia.aos + S + v]);
      const Prim2 w = prims2(q, gm1, gam, mhalf, (ia.valid & 1) ? ~0u : 0u,
                             (ia.valid & 2) ? ~0u : 0u, chk);
      if (ia.slot >= 0) {
        float* d = soa + ia.slot;
#pragma unroll
        for (int v = 0; v < S; ++v) st2(d + (G::AQ + v) * NSL, q[v]);
        st2(d + G::AUY * NSL, w.u[1]);
        st2(d + G::APR * NSL, w.p);
        st2(d + G::ACS * NSL, w.c);
      }
      // faces (x0 | x0+1) and (x0+1 | x0+2): left cells = this pair, right
      // cells = (second cell, the next lane's first cell)
      auto nxt = [&](f2 v) {
        float lo, hi;
        f2_unpack(v, lo, hi);
        return f2_pack(hi, __shfl_down_sync(FULL, lo, 1));
      };
      const Cell2 L{q[0], q[2], q[1], q[3], w.u[0], w.p, w.c, w.e};
      const Cell2 R{nxt(q[0]), nxt(q[2]), nxt(q[1]), nxt(q[3]),
                    nxt(w.u[0]), nxt(w.p), nxt(w.c), nxt(w.e)};
      f2 g[4];
      unsigned bl, bh;
      flux2(L, R, g, bl, bh);
      lmax = umax(lmax, bl & mflo);
      lmax = umax(lmax, bh & mfhi);
      // flux differences of cells x0 and x0+1 (the left face of x0 is the
      // previous lane's second face)
      constexpr int PV[4] = {0, 2, 1, 3};  // unknown of g[i]
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float gl, gh;
        f2_unpack(g[i], gl, gh);
        const float gprev = __shfl_up_sync(FULL, gh, 1);
        dgx[PV[i]] = f2_pack(sub_rn(gl, gprev), sub_rn(gh, gl));
      }
    }
    __syncthreads();  // buffer s is converted: the copy two patches ahead may start

    const Pat nx2 = nx1.pos < a.i_end ? next_valid(nx1.pos + gridDim.x) : nx1;
    if (nx2.pos < a.i_end) {
      if (lane == 0) issue_box(nx2, s);
      pending |= 1u << s;
    }
    if (nx1.pos < a.i_end) {
      if (wait_box(s ^ 1) && STEP) gather(nx1, s ^ 1);
    }

    // ---- y faces: one face of an x pair of columns per lane ----------------
    if (yact) {
      auto load = [&](int y) {
        const float* sp = soa + 2 * yj + RP * y;
        const f2 e3 = ld2(sp + (G::AQ + 3) * NSL), pr = ld2(sp + G::APR * NSL);
        return Cell2{ld2(sp + G::AQ * NSL), ld2(sp + (G::AQ + 1) * NSL),
                     ld2(sp + (G::AQ + 2) * NSL), e3, ld2(sp + G::AUY * NSL),
                     pr, ld2(sp + G::ACS * NSL), add2(e3, pr)};
      };
      const Cell2 L = load(yf), R = load(yf + 1);
      f2 g[4];
      unsigned bl, bh;
      flux2(L, R, g, bl, bh);
      lmax = umax(lmax, bl & kMagMask);
      lmax = umax(lmax, bh & yhi);
      // g: rho, transverse (j_x), normal (j_y), E -- the unknowns in order
#pragma unroll
      for (int v = 0; v < S; ++v) st2(gy + (v * (P + 1) + yf) * GW + 2 * yj, g[v]);
    }
    if (want_lam) {
      const unsigned long long m = warp_max_u64((unsigned long long)lmax);
      if (lane == 0) a.lam_patch[cur.pid] = order_value<float>(m);
    }
    __syncthreads();  // y-face fluxes complete

    // ---- update: Q - (dt / 2dx) sum_k (G+ - G-), by the interior-row lanes
    //      whose pair is a pair of interior cells --------------------------
    if (xrow && xj >= 1) {
      const int j = xj - 1, y = 1 + xr;
      const bool hi = 2 + 2 * j <= P;  // the second cell is a cell of the patch
      const unsigned mhi = hi ? ~0u : 0u;
      f2 acc[4];
#pragma unroll
      for (int v = 0; v < S; ++v) {
        const float* gv = gy + (v * (P + 1) + y) * GW + 2 * j;
        acc[v] = add2(dgx[v], sub2(ld2(gv), ld2(gv - GW)));
      }
      f2 qn[4];
#pragma unroll
      for (int v = 0; v < S; ++v) qn[v] = fma2(mhr2, acc[v], q[v]);
      float* dst = a.out + cur.off + (int64_t)((1 + 2 * j) + NE * y) * S;
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
        for (int k = 0; k < 2; ++k) {
          float ul, uh;
          f2_unpack(w.u[k], ul, uh);
          lam_next = umax(lam_next, wave_bits(ul, cl) & kMagMask);
          lam_next = umax(lam_next, wave_bits(uh, ch) & kMagMask & mhi);
        }
        if (a.prim_out != nullptr) {
          constexpr int NI = P * P;
          float* po = a.prim_out + cur.pid * a.prim_stride + 2 * j + P * (y - 1);
          const f2 vals[5] = {w.u[0], w.u[1], w.p, w.c, w.e};
#pragma unroll
          for (int m = 0; m < 5; ++m) {
            float lo, hv;
            f2_unpack(vals[m], lo, hv);
            po[m * NI] = lo;
            if (hi) po[m * NI + 1] = hv;
          }
        }
      }
    }
    if (nx1.pos < a.i_end) cp_async_wait_all();
    timeout = __syncthreads_or(timeout);
    if (timeout) break;
    cur = nx1;
    nx1 = nx2;
    s ^= 1;
  }
  if (timeout) {
    if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    if (pending & 1u) mbar_wait_bounded(&bar[0], parity & 1u, kWaitLimit);
    if (pending & 2u) mbar_wait_bounded(&bar[1], (parity >> 1) & 1u, kWaitLimit);
    cp_async_wait_all();
    return;
  }
  if (chk >= kBadChk) atomicOr(a.status, ST_NONPHYSICAL);
  if constexpr (STEP) {
    const unsigned long long m = warp_max_u64((unsigned long long)lam_next);
    if (lane == 0) atomicMax(a.lam_next, m);
  }
}

template <int P, bool STEP>
cudaError_t pairs2d_smem_attr() {
  static int set_bytes[64] = {0};
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && set_bytes[dev] >= Geom2<P>::SMEM) return cudaSuccess;
  e = cudaFuncSetAttribute(pairs2d_kernel<P, STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           Geom2<P>::SMEM);
  if (e == cudaSuccess && dev >= 0 && dev < 64) set_bytes[dev] = Geom2<P>::SMEM;
  return e;
}

template <int P, bool STEP>
cudaError_t launch_pairs2d_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
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
  cudaError_t e = pairs2d_smem_attr<P, STEP>();
  if (e != cudaSuccess) return e;
  pairs2d_kernel<P, STEP><<<grid, Geom2<P>::NT, Geom2<P>::SMEM, h->stream>>>(a);
  return cudaGetLastError();
}

template <int P, bool STEP>
cudaError_t occupancy_pairs2d_t(int* bps) {
  cudaError_t e = pairs2d_smem_attr<P, STEP>();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, pairs2d_kernel<P, STEP>,
                                                       Geom2<P>::NT, Geom2<P>::SMEM);
}

}  // namespace

bool pairs2d_class(const fv_batch* h, int p) {
  return h->prec == FV_FP32 && h->d == 2 && h->s == 4 && p == 5;
}

bool pairs2d_eligible(const fv_batch* h, const UpdateLaunch& l) {
  const int mode = step_mode(l);
  return pairs2d_class(h, l.uniform_p) && mode != kModePrim && l.corr == nullptr &&
         l.dx_patch == nullptr && !l.local_cfl && (mode == kModeStep || l.prim_out == nullptr);
}

cudaError_t launch_pairs2d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  return step_mode(l) == kModeStep ? launch_pairs2d_t<5, true>(h, l, grid)
                                   : launch_pairs2d_t<5, false>(h, l, grid);
}

cudaError_t pairs2d_occupancy(int mode, int* bps) {
  return mode == kModeStep ? occupancy_pairs2d_t<5, true>(bps)
                           : occupancy_pairs2d_t<5, false>(bps);
}

}  // namespace fv
