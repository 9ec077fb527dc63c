// fv_step.cuh -- the batched Rusanov patch update (Eq. 3-5, Algorithm 1 with
// the outer loop over patches), one kernel template with three modes:
//
//   update     (fv_patch_update_batch) the halo cells are read from the input
//              patch, as filled by fv_halo_fill;
//   time step  (fv_time_step) the face-halo cells are gathered straight from
//              the neighbours' interiors (periodic / outflow / wall as in
//              fv_halo_fill), dt comes from the CFL condition on the maximum
//              wave speed the previous step left on the device, and the
//              kernel reduces the maximum wave speed of the new state for the
//              next step.  One launch replaces halo fill + reduce + update
//              and gives bitwise the same result;
//   primitive  (fv_time_step_prim) a time step that also receives the
//   carry      primitive state (u, p, c, E + p) of its input from the
//              previous step and hands that of its output to the next.  The
//              time step computes the primitives of the new state anyway (for
//              the next CFL maximum), so carrying them removes the conversion
//              of every interior and face-halo cell from the next step:
//              a quarter of the FP64 work of a 3D step.  Bitwise equal to the
//              time step without the carry.
//
// Each CTA is persistent and walks its patches i = blockIdx.x + k*gridDim.x,
// or pops them one at a time from a work queue (a zeroed device counter).
// While it computes patch i, the TMA engine copies patch i+1 (and, carrying
// primitives, their interior block) into the other of two shared-memory
// stages (cp.async.bulk, completion on an mbarrier), and the halo cells of
// patch i+1 that live elsewhere are gathered with cp.async.
// Per patch:
//   cells   (not when primitives are carried) every interior and face-halo
//           cell converts to primitives once (Eq. 2); interior cells keep
//           all of (u, p, c, E + p), halo cells the normal velocity, p, c,
//           E + p.  The two groups start on warp boundaries;
//   faces   every face flux G = f_L + f_R - a (Q_R - Q_L) = 2F (Eq. 4, 5) is
//           computed exactly once, from the states and primitives of its two
//           cells, and shared by both;
//   update  every interior cell sums G_+ - G_- over x, then y, then z and
//           writes Q - (dt / 2dx) sum (Eq. 3); a time step then converts the
//           new state to primitives for the next CFL maximum (and the carry).
// Every floating-point operation is written out (fma or an explicitly
// rounded add / multiply), so the compiler cannot contract differently in
// different modes: the modes agree bitwise.  Maxima (per-patch a of
// Algorithm 1 step 10, next-step wave speed) are taken on integer bit
// patterns: exact and independent of the order of work.
#pragma once

#include "fv_device.cuh"
#include "fv_internal.h"
#include "fv_ptx.cuh"

namespace fv {

template <typename T>
struct StepParams {
  const T* __restrict__ in;
  T* __restrict__ out;
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ sizes;
  const int32_t* __restrict__ nbr;  // time-step modes
  const int32_t* __restrict__ order;  // processing order (patch indices), or null
  int64_t i_begin, i_end;             // positions of the sequence this launch runs
  int64_t n;                          // patches in the batch
  int64_t n_elems;
  int pmax;
  int nstage;  // shared-memory stages: 2 (copy overlaps compute) or 1
  T gamma, gm1;
  double dx, dt, cfl;
  const double* dt_dev;               // update mode with dt <= 0
  const unsigned long long* lam_in;   // time-step modes: bits of lambda(Q^n)
  unsigned long long* lam_next;       // time-step modes: bits of lambda(Q^n+1)
  double* dt_slot;                    // time-step modes: dt used, written once
  double* lam_patch;
  unsigned int* status;
  const float* corr;    // per-face flux corrections [patch][k][v][face], or null
  int64_t corr_stride;  // floats per patch of corr
  T one, mone, mzero;  // 1, -1, -0 as arguments (see Arith)
  const double* dx_patch;  // update mode: per-patch cell size (or null: dx)
  double* dt_patch;        // with dx_patch: per-patch dt (input, or output under local CFL)
  int local_cfl;           // with dx_patch: dt_i = cfl dx_i / (d lambda_i) per patch
  const T* __restrict__ prim_in;  // carried primitives of `in` (primitive-carry mode)
  T* __restrict__ prim_out;       // primitives of `out` (time-step modes), or null
  int64_t prim_stride;            // elements per patch of prim_in / prim_out
  long long wait_limit = FV_WAIT_LIMIT;  // cycles of a wait for a patch's copy
  unsigned long long* queue = nullptr;    // zeroed counter of positions handed out, or null
};

template <int D>
__host__ __device__ inline int ipow_d(int b) {
  return D == 1 ? b : D == 2 ? b * b : b * b * b;
}
// state box of a patch with its halo: (p+2)^D cells of D+2 unknowns
template <int D>
__host__ __device__ inline int stage_elems(int p) {
  return ipow_d<D>(p + 2) * (D + 2);
}
// interior primitives: D+3 components (u_1..u_D, p, c, E+p) of p^D cells
template <int D>
__host__ __device__ inline int iprim_elems(int p) {
  return (D + 3) * ipow_d<D>(p);
}
// face-halo primitives: 2D faces x 4 components (u_normal, p, c, E+p) x p^(D-1)
template <int D>
__host__ __device__ inline int hprim_elems(int p) {
  return 2 * D * 4 * (ipow_d<D>(p) / p);
}
// face fluxes G: D directions x (D+2) unknowns x (p+1) p^(D-1) faces
template <int D>
__host__ __device__ inline int gface_elems(int p) {
  return D * (D + 2) * (p + 1) * (ipow_d<D>(p) / p);
}
__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Unroll factors of the cell and face loops.
#ifndef FV_UNROLL_CELLS
#define FV_UNROLL_CELLS 1
#endif
#ifndef FV_UNROLL_FACES
#define FV_UNROLL_FACES 1
#endif
#define FV_STR_(x) #x
#define FV_PRAGMA_UNROLL(n) _Pragma(FV_STR_(unroll n))

// Where the face-halo cells of one face come from: a patch (its index and
// element offset), the layer along the face normal in that patch (halo-
// inclusive coordinate), and whether the normal momentum is negated (wall).
struct FaceSrc {
  long long off;
  int ck;
  int neg;
  int pidx;
  int pad;
};

// Threads per CTA the kernel is built for: one CTA advances one patch at a
// time; small patches use a warp or two, the largest eight warps.
constexpr int kMaxNT = 256;
// Shared-memory header: two mbarriers (16 B), per-warp reduction slots, and
// the face sources of the two stages (2 x 6 x 24 B).
constexpr int kRedOff = 16;
constexpr int kFaceSrcOff = 128;
constexpr int kHdrBytes = 512;
static_assert(kRedOff + 8 * (kMaxNT / 32) <= kFaceSrcOff, "header too small");
static_assert(kFaceSrcOff + 2 * 6 * (int)sizeof(FaceSrc) <= kHdrBytes, "header too small");

// Shared-memory carve-up for patches up to pmax (element counts of T).  A
// stage holds the state box, the interior primitives and the face-halo
// primitives of one patch; two stages let the copy of the next patch overlap
// the current one (one stage when two do not fit: the copy of the next
// patch then starts after the current patch is done).  The face fluxes G
// follow the stages.
template <int D>
struct Carve {
  int nstage, box, ip, hp, stage, g;
  __host__ __device__ Carve(int pmax, int vec, int nstage_)
      : nstage(nstage_),
        box(round_up(stage_elems<D>(pmax), vec)),
        ip(round_up(iprim_elems<D>(pmax), vec)),
        hp(round_up(hprim_elems<D>(pmax), vec)),
        stage(box + ip + hp),
        g(round_up(gface_elems<D>(pmax), vec)) {}
  __host__ __device__ int total() const { return nstage * stage + g; }
};

template <typename T>
struct Stage {
  T* box;  // state, AoS cells (x fastest), halo-inclusive
  T* ip;   // interior primitives [component][interior cell]
  T* hp;   // face-halo primitives [face][component][transverse index]
};

// Clock cycles a CTA waits for a copy before it reports FV_ERR_TIMEOUT
// (about one second at 2 GHz).  The step kernel's waits for the copies of the
// patches it is about to process take the launch's limit (StepParams::
// wait_limit, normally this value); once a wait has given up, the waits for
// the copies still in flight take this full limit, so no CTA leaves with a
// bulk copy pending.
constexpr long long kWaitLimit = FV_WAIT_LIMIT;

// Wait for a patch's copy with the launch's limit: the default limit with
// try_wait; a shortened one (a test of the timeout path) by polling.
__device__ __forceinline__ bool wait_patch_copy(uint64_t* bar, uint32_t parity,
                                                long long limit) {
  return limit >= kWaitLimit ? mbar_wait_bounded(bar, parity, limit)
                             : mbar_wait_polled(bar, parity, limit);
}

// ---------------------------------------------------------------------------
// Copies into a stage
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ bool patch_ok(const StepParams<T>& a, int64_t j, int& pj,
                                         int64_t& offj) {
  constexpr int VEC = 16 / sizeof(T);
  pj = a.sizes[j];
  offj = a.off[j];
  bool ok = pj >= 1 && pj <= a.pmax && offj >= 0 && (offj % VEC) == 0;
  if (ok && a.n_elems > 0) ok = offj + (int64_t)stage_elems<D>(pj) <= a.n_elems;
  if (!ok && threadIdx.x == 0) atomicOr(a.status, ST_BAD_PATCH);
  return ok;
}

// Thread 0: bulk copy of the 16-byte-aligned body of patch j into a stage,
// and, carrying primitives, of its interior primitive block.  The state's
// ragged tail (< 16 bytes) lies in the last cell of the patch, a corner
// (d >= 2, never read) or the +x halo cell (d = 1, gathered separately).
template <typename T, int D, bool PRIMIN>
__device__ __forceinline__ void issue_stage(const StepParams<T>& a, int64_t pid, int pj,
                                            int64_t offj, const Stage<T>& st, uint64_t* bar) {
  const uint32_t bytes = (uint32_t)(stage_elems<D>(pj) * sizeof(T)) & ~15u;
  uint32_t pbytes = 0;
  if constexpr (PRIMIN) pbytes = (uint32_t)round_up(iprim_elems<D>(pj) * (int)sizeof(T), 16);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, bytes + pbytes);
  bulk_copy_g2s(st.box, a.in + offj, bytes, bar);
  if constexpr (PRIMIN) bulk_copy_g2s(st.ip, a.prim_in + pid * a.prim_stride, pbytes, bar);
}

// The source of the halo cells of face f of patch j (the neighbour table and
// the neighbour's metadata are read and checked here once, not per halo
// element).  Time-step modes follow the rules of fv_halo_fill; update mode
// with d = 1 re-reads the patch's own halo cells.
template <typename T, int D, bool GATHER>
__device__ __forceinline__ FaceSrc face_source(const StepParams<T>& a, int64_t j, int pj,
                                               int64_t offj, int f) {
  constexpr int VEC = 16 / sizeof(T);
  const int side = f & 1;
  FaceSrc r;
  r.off = offj;
  r.neg = 0;
  r.pidx = (int)j;
  r.pad = 0;
  if constexpr (!GATHER) {
    r.ck = side ? pj + 1 : 0;  // the own halo layer
  } else {
    r.ck = side ? pj : 1;  // outflow: the own interior layer next to the face
    const int32_t nb = a.nbr[j * 2 * D + f];
    if (nb >= 0) {
      bool ok = nb < a.n;
      int64_t onb = 0;
      if (ok) {
        onb = a.off[nb];
        ok = a.sizes[nb] == pj && onb >= 0 && (onb % VEC) == 0 &&
             (a.n_elems <= 0 || onb + (int64_t)stage_elems<D>(pj) <= a.n_elems);
      }
      if (ok) {
        r.off = onb;
        r.pidx = nb;
        r.ck = side ? 1 : pj;  // the neighbour's interior layer next to the face
      } else {
        atomicOr(a.status, ST_BAD_PATCH);
      }
    } else if (nb == -2) {
      r.neg = 1;  // wall: mirror of the own interior layer
    } else if (nb != -1) {
      atomicOr(a.status, ST_BAD_PATCH);
    }
  }
  return r;
}

// Threads 0 .. 2d-1: the sources of the 2d faces of patch j.
template <typename T, int D, bool GATHER>
__device__ __forceinline__ void face_sources(const StepParams<T>& a, int64_t j, int pj,
                                             int64_t offj, FaceSrc* fs) {
  if constexpr (!GATHER && D != 1) return;
  const int f = threadIdx.x;
  if (f >= 2 * D) return;
  fs[f] = face_source<T, D, GATHER>(a, j, pj, offj, f);
}

// Whether the halo gather of a compile-time patch size runs in warp slots
// (one face per warp and iteration): when its warp iterations are not more
// than 1.25 times those of the flat loop (each slot iteration is much cheaper:
// constant indexing, one source).
template <int D, int P, int NT>
__host__ __device__ constexpr bool kGatherSlots() {
  if (P <= 0 || D == 1) return false;
  const int ptr = D == 2 ? P : P * P;
  const int slot_iters = 2 * D * ((ptr + 31) / 32);
  const int total = 2 * D * ptr;
  const int flat_iters = (total / NT) * (NT / 32) + ((total % NT) + 31) / 32;
  return 4 * slot_iters <= 5 * flat_iters;
}

// All threads: fetch the face-halo cells of a patch that do not come with its
// bulk copy, from the sources resolved by face_sources, as cp.async element
// copies (a wall's negated normal momentum with a plain load and store); when
// primitives are carried, also the face-halo primitives (u_normal, p, c,
// E + p) from the sources' carried blocks (a wall negates u_normal).
template <typename T, int D, int P, bool GATHER, bool PRIMIN, int NT>
__device__ __forceinline__ void gather_halo(const StepParams<T>& a, int pj, const Stage<T>& s,
                                            const FaceSrc* fs) {
  if constexpr (!GATHER && D != 1) return;
  constexpr int S = D + 2;
  const Geom<D, P> g(pj);
  const int p = g.p;
  const int ptr = g.ptrans();
  // halo cell r of face f (direction k = f / 2) from its source m
  auto cell = [&](const int k, const int f, const int r, const FaceSrc& m) {
    const int cd = g.cell_kt(k, (f & 1) ? p + 1 : 0, r);
    const int cs = g.cell_kt(k, m.ck, r);
    T* dst = s.box + cd * S;
    const T* src = a.in + m.off + (int64_t)cs * S;
    T* pd = s.hp + f * 4 * ptr + r;
    const T* ps = nullptr;
    if constexpr (PRIMIN)
      ps = a.prim_in + (int64_t)m.pidx * a.prim_stride + g.icell_kt(k, m.ck - 1, r);
    if (!m.neg) {
#pragma unroll
      for (int v = 0; v < S; ++v) cp_async_elem(dst + v, src + v);
      if constexpr (PRIMIN) cp_async_elem(pd, ps + k * g.nint());
    } else {  // wall: the normal momentum and velocity mirrored
#pragma unroll
      for (int v = 0; v < S; ++v) {
        if (v == 1 + k)
          dst[v] = neg_t(__ldg(src + v));
        else
          cp_async_elem(dst + v, src + v);
      }
      if constexpr (PRIMIN) pd[0] = neg_t(__ldg(ps + k * g.nint()));
    }
    if constexpr (PRIMIN) {
#pragma unroll
      for (int v = 1; v < 4; ++v) cp_async_elem(pd + v * ptr, ps + (D + v - 1) * g.nint());
    }
  };
  if constexpr (kGatherSlots<D, P, NT>()) {
    // warp slots: a warp fetches cells of one face (one source, one
    // direction: compile-time indexing, uniform branches)
    const int spf = (ptr + 31) >> 5;  // slots per face
    const int lane = threadIdx.x & 31;
    for (int ws = threadIdx.x >> 5; ws < 2 * D * spf; ws += NT / 32) {
      const int f = ws / spf;
      const int r = (ws - f * spf) * 32 + lane;
      const FaceSrc m = fs[f];
      if (r < ptr) {
        if (f < 2) {
          cell(0, f, r, m);
        } else if constexpr (D >= 2) {
          if (f < 4) {
            cell(1, f, r, m);
          } else if constexpr (D == 3) {
            cell(2, f, r, m);
          }
        }
      }
    }
  } else {
    for (int hc = threadIdx.x; hc < 2 * D * ptr; hc += NT) {
      const int f = hc / ptr;
      cell(f >> 1, f, hc - f * ptr, fs[f]);
    }
  }
  cp_async_commit();
}

// Patch sizes with a compile-time specialisation, per CTA size: the common
// sizes for 128 threads, small ones for one or two warps, large ones for 256.
template <int D, int NT>
__host__ __device__ constexpr bool specialised(int p) {
  if (D == 1) return false;
  if (NT <= 64) return D == 3 ? p == 3 : (p == 3 || p == 5 || p == 8);
  if (NT >= 256) return D == 3 ? p == 7 : p == 17;
  return D == 3 ? (p == 3 || p == 5 || p == 7) : (p == 3 || p == 5 || p == 8 || p == 17);
}

template <typename T, int D, bool GATHER, bool PRIMIN, int NT>
__device__ __forceinline__ void gather_dispatch(const StepParams<T>& a, int pj,
                                                const Stage<T>& s, const FaceSrc* fs) {
  if constexpr (!GATHER && D != 1) return;
#define FV_GH(PP)                                                               \
  if constexpr (specialised<D, NT>(PP)) {                                       \
    if (pj == PP) return gather_halo<T, D, PP, GATHER, PRIMIN, NT>(a, pj, s, fs); \
  }
  FV_GH(3)
  FV_GH(5)
  FV_GH(7)
  FV_GH(8)
  gather_halo<T, D, 0, GATHER, PRIMIN, NT>(a, pj, s, fs);
#undef FV_GH
}

// State of the copy pipeline of one CTA.
struct Pipe {
  uint64_t* bar;
  uint32_t parity;   // bit s: parity of the next completion of bar[s]
  uint32_t pending;  // bit s: a bulk copy into stage s is in flight
  bool timeout;
};

template <typename T>
struct NextPatch {
  int64_t j;    // position in the processing sequence; >= i_end: none
  int64_t pid;  // patch index
  int p;
  int64_t off;
  Stage<T> st;
  FaceSrc* fs;
  int slot;
};

// Inside a patch, after a barrier: wait for the bulk copy of the next patch
// and start its halo gather, so both overlap the rest of this patch.
template <typename T, int D, bool GATHER, bool PRIMIN, int NT>
__device__ __forceinline__ void mid_hook(const StepParams<T>& a, Pipe& pp,
                                         const NextPatch<T>& nx) {
  if (nx.j >= a.i_end) return;
  const bool ok = wait_patch_copy(&pp.bar[nx.slot], (pp.parity >> nx.slot) & 1u, a.wait_limit);
  if (ok) {
    pp.parity ^= 1u << nx.slot;
    pp.pending &= ~(1u << nx.slot);
  }
  if (!ok) {
    pp.timeout = true;
    return;
  }
  gather_dispatch<T, D, GATHER, PRIMIN, NT>(a, nx.p, nx.st, nx.fs);
}

// ---------------------------------------------------------------------------
// One patch: cells, faces, update.
// ---------------------------------------------------------------------------
// Whether the face loop walks lines of cells (pencils): each cell loaded once
// for its two faces along the line, far fewer instructions per face but one
// thread per line, so fewer busy lanes.  For FP32, which the instruction
// count limits; FP64 is limited by its arithmetic pipe, which idle lanes
// would waste.
template <typename T, int D, int P, int NT>
__host__ __device__ constexpr bool kPencilFaces() {
  return sizeof(T) == 4 && P > 0 && D >= 2;
}

// Whether the face loop of a compile-time patch size runs in warp slots (one
// direction per warp and iteration) rather than over all faces flat: when it
// keeps at least as many lanes busy (to 2 %).
template <int D, int P, int NT>
__host__ __device__ constexpr bool kWarpSlots() {
  if constexpr (P <= 0 || D == 1) {
    return false;
  } else {
    const int nface = (P + 1) * (D == 2 ? P : P * P);
    const int slot_lanes = D * ((nface + 31) / 32) * 32;
    const int total = D * nface;
    const int flat_full = total / NT, flat_rest = total - flat_full * NT;
    const int flat_lanes = flat_full * NT + (flat_rest + 31) / 32 * 32;
    return 100 * total / slot_lanes + 2 >= 100 * total / flat_lanes;
  }
}

template <typename T, int D, int P, bool GATHER, bool FUSED, bool PRIMIN, int NT>
__device__ __forceinline__ void patch_compute(const StepParams<T>& a, int p_rt, int64_t i,
                                              int64_t off, const Stage<T>& cur, T* G, T mhr,
                                              unsigned long long* red,
                                              unsigned long long& lam_next, Pipe& pp,
                                              const NextPatch<T>& nx) {
  constexpr int S = D + 2;
  const Geom<D, P> g(p_rt);
  const int p = g.p;
  const int nface = g.nface(), nint = g.nint(), ptr = g.ptrans();
  const int tid = threadIdx.x;
  const T* __restrict__ st = cur.box;
  T* ip = cur.ip;
  T* hp = cur.hp;
  const Arith<T> ar{a.one, a.mone, a.mzero};
  bool bad = false;

  // ---- cells: primitives of the interior and face-halo cells ---------------
  if constexpr (!PRIMIN) {
    const int nint_pad = (nint + 31) & ~31;
    const int nA = nint_pad + 2 * D * ptr;
    FV_PRAGMA_UNROLL(FV_UNROLL_CELLS)
    for (int t = tid; t < nA; t += NT) {
      if (t < nint) {
        int c[3] = {0, 0, 0};
        int r = t;
#pragma unroll
        for (int m = 0; m < D; ++m) {
          c[m] = 1 + r % p;
          r /= p;
        }
        const int cid = g.cell(c);
        T q[S];
#pragma unroll
        for (int v = 0; v < S; ++v) q[v] = st[cid * S + v];
        const Prim<T, D> w = primitives<T, D>(q, a.gm1, a.gamma, bad, ar);
#pragma unroll
        for (int m = 0; m < D; ++m) ip[m * nint + t] = w.u[m];
        ip[D * nint + t] = w.p;
        ip[(D + 1) * nint + t] = w.c;
        ip[(D + 2) * nint + t] = w.ep;
      } else if (t >= nint_pad) {
        const int hc = t - nint_pad;
        const int f = hc / ptr;
        const int r = hc - f * ptr;
        const int k = f >> 1;
        const int cid = g.cell_kt(k, (f & 1) ? p + 1 : 0, r);
        T q[S];
#pragma unroll
        for (int v = 0; v < S; ++v) q[v] = st[cid * S + v];
        const Prim<T, D> w = primitives<T, D>(q, a.gm1, a.gamma, bad, ar);
        T uk = w.u[0];
#pragma unroll
        for (int m = 1; m < D; ++m) uk = (k == m) ? w.u[m] : uk;
        T* h = hp + f * 4 * ptr + r;
        h[0] = uk;
        h[ptr] = w.p;
        h[2 * ptr] = w.c;
        h[3 * ptr] = w.ep;
      }
    }
    __syncthreads();
    mid_hook<T, D, GATHER, PRIMIN, NT>(a, pp, nx);
  }

  // ---- faces: G = f_L + f_R - a (Q_R - Q_L), once per face -------------------
  // Cell b (halo-inclusive, 0..p+1) along k at transverse index tr: its state
  // and the primitives of direction k (face-halo block at the patch
  // boundary, interior block inside).
  struct CellK {
    T q[S];
    T u, pr, c, e;
  };
  // (lo / hi: whether b may be the lower / upper halo cell, constants at the
  // call sites)
  auto load_cell = [&](const int k, const int b, const int tr, CellK& x, const bool lo,
                       const bool hi) {
    const int cid = g.cell_kt(k, b, tr);
#pragma unroll
    for (int v = 0; v < S; ++v) x.q[v] = st[cid * S + v];
    const bool h0 = lo && b == 0, h1 = hi && b == p + 1;
    const int ic = g.icell_kt(k, h0 ? 0 : (h1 ? p - 1 : b - 1), tr);
    const T* pu = h0 ? hp + 8 * k * ptr + tr
                     : (h1 ? hp + (8 * k + 4) * ptr + tr : ip + k * nint + ic);
    const T* pp_ = h0 ? hp + (8 * k + 1) * ptr + tr
                      : (h1 ? hp + (8 * k + 5) * ptr + tr : ip + D * nint + ic);
    const int sp = (h0 || h1) ? ptr : nint;
    x.u = pu[0];
    x.pr = pp_[0];
    x.c = pp_[sp];
    x.e = pp_[2 * sp];
  };
  // The flux of face j (k) between cells L and R, stored into G.
  auto flux = [&](const int k, const int j, const CellK& L, const CellK& R,
                  unsigned long long& lmax) {
    const T uL = L.u, pL = L.pr, cL = L.c, eL = L.e;
    const T uR = R.u, pR = R.pr, cR = R.c, eR = R.e;
    const T* qL = L.q;
    const T* qR = R.q;
    // a = max(|u_k| + c) over the two cells (Eq. 5)
    const T am = max_by_bits(ar.add(abs_t(uL), cL), ar.add(abs_t(uR), cR));
    const unsigned long long ab = order_bits(am);
    lmax = ab > lmax ? ab : lmax;
    // G = f_L + f_R - a (Q_R - Q_L) = (f_L + a Q_L) + (f_R - a Q_R).  The
    // fluxes of rho and of the momenta are the conserved value times u_k
    // (Eq. 2: j_k = rho u_k; j_m u_k, plus p on the normal momentum), so
    // f + a Q folds to Q (u_k + a) (+ p): with s_L = u_L + a, s_R = u_R - a,
    //   G_rho = rho_L s_L + rho_R s_R,
    //   G_m   = j_mL s_L + j_mR s_R + (p_L + p_R) [m = k],
    //   G_E   = (E + p)_L u_L + (E + p)_R u_R + a (E_L - E_R).
    const T sL = ar.add(uL, am), sR = ar.sub(uR, am);
    const T ps = ar.add(pL, pR);
    T gs[S];
    gs[0] = fma(qL[0], sL, ar.mul(qR[0], sR));
#pragma unroll
    for (int m = 0; m < D; ++m)
      gs[1 + m] = fma(qL[1 + m], sL, fma(qR[1 + m], sR, (m == k) ? ps : T(-0.0)));
    gs[D + 1] = fma(am, ar.sub(qL[D + 1], qR[D + 1]), fma(eL, uL, ar.mul(eR, uR)));
    T* Gk = G + k * S * nface;
#pragma unroll
    for (int v = 0; v < S; ++v) {
      T gv = gs[v];
      // learned correction C of this face (G = 2F, so G + 2C = 2(F + C)); 2C
      // is exact in FP32, and its widening to FP64 runs on the integer pipe
      if (a.corr != nullptr)
        gv = ar.add(gv, to_t(2.f * a.corr[i * a.corr_stride + (k * S + v) * nface + j],
                             (T*)nullptr));
      Gk[v * nface + j] = gv;
    }
  };
  // Face (k, j) of the patch, j = tr + ptr b: between cells b and b+1 along k.
  auto face = [&](const int k, const int j, unsigned long long& lmax) {
    const int b = j / ptr;
    const int tr = j - b * ptr;
    CellK L, R;
    load_cell(k, b, tr, L, true, false);
    load_cell(k, b + 1, tr, R, false, true);
    flux(k, j, L, R, lmax);
  };
  // All faces of one line of cells along k (transverse index tr), walking b:
  // every cell is loaded once and serves its two faces.
  auto pencil = [&](const int k, const int tr, unsigned long long& lmax) {
    CellK A, B;
    load_cell(k, 0, tr, A, true, false);
    for (int b = 0; b <= p; b += 2) {
      load_cell(k, b + 1, tr, B, false, true);
      flux(k, tr + ptr * b, A, B, lmax);
      if (b + 1 > p) break;
      load_cell(k, b + 2, tr, A, false, true);
      flux(k, tr + ptr * (b + 1), B, A, lmax);
    }
  };
  unsigned long long lmax = 0ull;
  if constexpr (kPencilFaces<T, D, P, NT>()) {
    // pencils in warp slots: a warp takes 32 lines of one direction
    const int spk = (ptr + 31) >> 5;
    const int lane = tid & 31;
    for (int ws = tid >> 5; ws < D * spk; ws += NT / 32) {
      const int k = ws / spk;
      const int tr = (ws - k * spk) * 32 + lane;
      if (tr < ptr) {
        if (k == 0) {
          pencil(0, tr, lmax);
        } else if constexpr (D >= 2) {
          if (k == 1) {
            pencil(1, tr, lmax);
          } else if constexpr (D == 3) {
            pencil(2, tr, lmax);
          }
        }
      }
    }
  } else if constexpr (kWarpSlots<D, P, NT>()) {
    // warp slots: a warp takes 32 faces of one direction, so k is the same in
    // every lane and compiles to constants (strides, cell indexing, the
    // momentum with the pressure term)
    const int spk = (nface + 31) >> 5;  // slots per direction
    const int lane = tid & 31;
    for (int ws = tid >> 5; ws < D * spk; ws += NT / 32) {
      const int k = ws / spk;
      const int j = (ws - k * spk) * 32 + lane;
      if (j < nface) {
        if (k == 0) {
          face(0, j, lmax);
        } else if constexpr (D >= 2) {
          if (k == 1) {
            face(1, j, lmax);
          } else if constexpr (D == 3) {
            face(2, j, lmax);
          }
        }
      }
    }
  } else {
    FV_PRAGMA_UNROLL(FV_UNROLL_FACES)
    for (int t = tid; t < D * nface; t += NT) {
      const int k = t / nface;
      face(k, t - k * nface, lmax);
    }
  }
  // per-patch maximum of a over the faces (Algorithm 1 step 10)
  const bool want_lam = a.lam_patch != nullptr || a.local_cfl;
  if (want_lam) {
    lmax = warp_max_u64(lmax);
    if ((tid & 31) == 0) red[tid >> 5] = lmax;
  }
  __syncthreads();
  if constexpr (PRIMIN) mid_hook<T, D, GATHER, PRIMIN, NT>(a, pp, nx);
  unsigned long long lam_bits = 0ull;
  if (want_lam) {
    lam_bits = red[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) lam_bits = red[w] > lam_bits ? red[w] : lam_bits;
    if (tid == 0 && a.lam_patch != nullptr) a.lam_patch[i] = order_value<T>(lam_bits);
  }
  // per-patch cell size and time step (update mode): dt_i given, or from the
  // patch's own CFL condition on its maximum wave speed
  if (a.dx_patch != nullptr) {
    const double dxi = a.dx_patch[i];
    double dti;
    if (a.local_cfl) {
      dti = (a.cfl * dxi) / ((double)D * order_value<T>(lam_bits));
      if (tid == 0) a.dt_patch[i] = dti;
    } else {
      dti = a.dt_patch[i];
    }
    mhr = neg_t((T)(0.5 * (dti / dxi)));
  }

  // ---- update: Q - (dt/2dx) sum_k (G_+ - G_-) -----------------------------------
  T* dst_base = a.out + off;
  for (int t = tid; t < nint; t += NT) {
    int c[3] = {0, 0, 0};
    int r = t;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      c[m] = 1 + r % p;
      r /= p;
    }
    const int cid = g.cell(c);
    T acc[S];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int jm = g.trans(c, k) + ptr * (c[k] - 1);
      const T* Gk = G + k * S * nface;
#pragma unroll
      for (int v = 0; v < S; ++v) {
        const T dG = ar.sub(Gk[v * nface + jm + ptr], Gk[v * nface + jm]);
        acc[v] = k == 0 ? dG : ar.add(acc[v], dG);
      }
    }
    T qn[S];
#pragma unroll
    for (int v = 0; v < S; ++v) qn[v] = fma(mhr, acc[v], st[cid * S + v]);
    T* dst = dst_base + (int64_t)cid * S;
#pragma unroll
    for (int v = 0; v < S; ++v) dst[v] = qn[v];
    if constexpr (FUSED) {
      // primitives and wave speed of the new state, for the next step's CFL
      // condition (and its primitive carry)
      const Prim<T, D> w = primitives<T, D>(qn, a.gm1, a.gamma, bad, ar);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const unsigned long long lb = order_bits(ar.add(abs_t(w.u[k]), w.c));
        lam_next = lb > lam_next ? lb : lam_next;
      }
      if (a.prim_out != nullptr) {
        T* po = a.prim_out + i * a.prim_stride + t;
#pragma unroll
        for (int m = 0; m < D; ++m) po[m * nint] = w.u[m];
        po[D * nint] = w.p;
        po[(D + 1) * nint] = w.c;
        po[(D + 2) * nint] = w.ep;
      }
    }
  }

  if (bad) atomicOr(a.status, ST_NONPHYSICAL);
}

template <typename T, int D, bool GATHER, bool FUSED, bool PRIMIN, int NT>
__device__ __forceinline__ void patch_dispatch(const StepParams<T>& a, int p, int64_t i,
                                               int64_t off, const Stage<T>& st, T* G, T hr,
                                               unsigned long long* red,
                                               unsigned long long& lam_next, Pipe& pp,
                                               const NextPatch<T>& nx) {
#define FV_PC(PP)                                                                           \
  if constexpr (specialised<D, NT>(PP)) {                                                   \
    if (p == PP)                                                                            \
      return patch_compute<T, D, PP, GATHER, FUSED, PRIMIN, NT>(a, p, i, off, st, G, hr, red, \
                                                                lam_next, pp, nx);          \
  }
  FV_PC(3)
  FV_PC(5)
  FV_PC(7)
  FV_PC(8)
  FV_PC(17)
  patch_compute<T, D, 0, GATHER, FUSED, PRIMIN, NT>(a, p, i, off, st, G, hr, red, lam_next, pp,
                                                    nx);
#undef FV_PC
}

// Resident CTAs per SM the register allocation is sized for, given as the
// resident threads per SM (3 CTAs of 128 threads for FP64, 6 for FP32).
#ifndef FV_MINBLOCKS_FP64
#define FV_MINBLOCKS_FP64 3
#endif
#ifndef FV_MINBLOCKS_FP32
#define FV_MINBLOCKS_FP32 6
#endif
template <typename T, int NT>
constexpr int min_blocks() {
  const int threads = 128 * (sizeof(T) == 8 ? FV_MINBLOCKS_FP64 : FV_MINBLOCKS_FP32);
  return threads / NT > 0 ? threads / NT : 1;
}

template <typename T, int D, bool GATHER, bool FUSED, bool PRIMIN, int NT>
__global__ void __launch_bounds__(NT, (min_blocks<T, NT>()))
    step_kernel(StepParams<T> a) {
  static_assert(!PRIMIN || (GATHER && FUSED), "the primitive carry is a time-step mode");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem_raw + kRedOff);
  FaceSrc* fsrc = reinterpret_cast<FaceSrc*>(smem_raw + kFaceSrcOff);  // [stage][face]
  constexpr int VEC = 16 / sizeof(T);
  const Carve<D> cv(a.pmax, VEC, a.nstage);
  const bool single = a.nstage == 1;
  T* const sbase = reinterpret_cast<T*>(smem_raw + kHdrBytes);
  // stage s (0 or 1; the same one when single), built by arithmetic so the
  // pointers stay in registers
  auto stage_at = [&](int s) -> Stage<T> {
    T* b = sbase + (single ? 0 : s) * cv.stage;
    return Stage<T>{b, b + cv.box, b + cv.box + cv.ip};
  };
  T* G = sbase + cv.nstage * cv.stage;
  const int tid = threadIdx.x;

  double dtv;
  if constexpr (FUSED) {
    const double lam = order_value<T>(*a.lam_in);
    dtv = (a.cfl * a.dx) / ((double)D * lam);
    if (blockIdx.x == 0 && tid == 0) *a.dt_slot = dtv;
  } else {
    dtv = a.dt > 0.0 ? a.dt : *a.dt_dev;
  }
  const T hr = neg_t((T)(0.5 * (dtv / a.dx)));  // -dt / (2 dx), passed as mhr

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  Pipe pp{bar, 0u, 0u, false};
  unsigned long long lam_next = 0ull;

  // Processing sequence: positions [i_begin, i_end), patch order[pos] (or
  // pos itself).  CTA b takes positions i_begin + b, + gridDim.x, ...; or,
  // with a queue, the next position not yet handed out (one atomic per
  // patch, by thread 0, broadcast through shared memory), so CTAs that
  // finish early take more patches.
  auto pid_of = [&](int64_t pos) -> int64_t {
    return a.order != nullptr ? (int64_t)a.order[pos] : pos;
  };
  __shared__ long long qpos;
  auto next_pos = [&](int64_t pos) -> int64_t {
    if (a.queue == nullptr) return pos + gridDim.x;
    if (tid == 0) qpos = a.i_begin + (long long)atomicAdd(a.queue, 1ull);
    __syncthreads();
    const int64_t v = qpos;
    __syncthreads();  // read by every thread before the next pop
    return v;
  };
  // first valid patch of this CTA, staged before the loop
  int64_t cur = a.queue != nullptr ? next_pos(0) : a.i_begin + blockIdx.x;
  int64_t pidc = 0;
  int pc = 0;
  int64_t oc = 0;
  while (cur < a.i_end && !patch_ok<T, D>(a, pidc = pid_of(cur), pc, oc)) cur = next_pos(cur);
  int s = 0;
  if (cur < a.i_end) {
    face_sources<T, D, GATHER>(a, pidc, pc, oc, fsrc);
    if (tid == 0) issue_stage<T, D, PRIMIN>(a, pidc, pc, oc, stage_at(0), &bar[0]);
    pp.pending = 1u;
    __syncthreads();  // face sources visible
    const bool ok = wait_patch_copy(&bar[0], 0u, a.wait_limit);
    if (ok) {
      pp.parity ^= 1u;
      pp.pending = 0u;
      gather_dispatch<T, D, GATHER, PRIMIN, NT>(a, pc, stage_at(0), fsrc);
    } else {
      pp.timeout = true;
    }
    cp_async_wait_all();
  }
  if (__syncthreads_or(pp.timeout)) cur = a.i_end;

  while (cur < a.i_end) {
    NextPatch<T> nx;
    nx.j = next_pos(cur);
    nx.pid = 0;
    while (nx.j < a.i_end && !patch_ok<T, D>(a, nx.pid = pid_of(nx.j), nx.p, nx.off))
      nx.j = next_pos(nx.j);
    nx.slot = single ? 0 : s ^ 1;
    nx.st = stage_at(nx.slot);
    nx.fs = fsrc + 6 * nx.slot;
    // visible to all threads after the barrier inside the patch
    if (nx.j < a.i_end) face_sources<T, D, GATHER>(a, nx.pid, nx.p, nx.off, nx.fs);
    NextPatch<T> nx_mid = nx;  // what the mid-patch hook waits for and gathers
    if (single) {
      nx_mid.j = a.i_end;  // the one stage is busy until this patch is done
    } else if (nx.j < a.i_end) {
      if (tid == 0) issue_stage<T, D, PRIMIN>(a, nx.pid, nx.p, nx.off, nx.st, &bar[nx.slot]);
      pp.pending |= 1u << nx.slot;
    }
    patch_dispatch<T, D, GATHER, FUSED, PRIMIN, NT>(a, pc, pidc, oc, stage_at(s), G, hr, red,
                                                    lam_next, pp, nx_mid);
    cp_async_wait_all();
    if (__syncthreads_or(pp.timeout)) break;
    if (single && nx.j < a.i_end) {
      if (tid == 0) issue_stage<T, D, PRIMIN>(a, nx.pid, nx.p, nx.off, nx.st, &bar[0]);
      pp.pending |= 1u;
      mid_hook<T, D, GATHER, PRIMIN, NT>(a, pp, nx);
      cp_async_wait_all();
      if (__syncthreads_or(pp.timeout)) break;
    }
    cur = nx.j;
    pidc = nx.pid;
    pc = nx.p;
    oc = nx.off;
    if (!single) s ^= 1;
  }
  if (pp.timeout) {
    // a copy did not complete in time: report, give the copies in flight a
    // second bounded wait, and leave
    if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
    if (pp.pending & 1u) mbar_wait_bounded(&bar[0], pp.parity & 1u, kWaitLimit);
    if (pp.pending & 2u) mbar_wait_bounded(&bar[1], (pp.parity >> 1) & 1u, kWaitLimit);
    cp_async_wait_all();
    return;
  }
  if constexpr (FUSED) {
    lam_next = warp_max_u64(lam_next);
    if ((tid & 31) == 0) red[tid >> 5] = lam_next;
    __syncthreads();
    if (tid == 0) {
      unsigned long long m = red[0];
#pragma unroll
      for (int w = 1; w < NT / 32; ++w) m = red[w] > m ? red[w] : m;
      atomicMax(a.lam_next, m);
    }
  }
}

// Bytes of dynamic shared memory of the kernel for patches up to pmax.
template <int D>
inline size_t step_smem_bytes(int es, int pmax, int nstage) {
  return kHdrBytes + (size_t)es * Carve<D>(pmax, 16 / es, nstage).total();
}

// Raises the kernel's dynamic shared-memory limit on the current device once
// (not per launch, so launches can be captured into CUDA graphs).
template <typename T, int D, bool GATHER, bool FUSED, bool PRIMIN, int NT>
static cudaError_t ensure_smem(size_t smem) {
  static int set_bytes[64] = {0};
  std::lock_guard<std::mutex> lock(smem_attr_mutex());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && set_bytes[dev] >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(step_kernel<T, D, GATHER, FUSED, PRIMIN, NT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) set_bytes[dev] = (int)smem;
  return e;
}

template <typename T, int D, bool GATHER, bool FUSED, bool PRIMIN, int NT>
static cudaError_t launch_step_t(const fv_batch* h, const UpdateLaunch& l, int grid) {
  StepParams<T> a;
  a.in = static_cast<const T*>(l.in);
  a.out = static_cast<T*>(l.out);
  a.off = l.off;
  a.sizes = l.sizes;
  a.nbr = l.nbr;
  a.order = l.order;
  a.i_begin = l.i_begin;
  a.i_end = l.i_end >= 0 ? l.i_end : l.n;
  a.n = l.n;
  a.n_elems = l.n_elems;
  a.pmax = l.pmax;
  a.nstage = l.nstage > 0 ? l.nstage : h->nstage;
  a.gamma = (T)l.gamma;
  a.gm1 = (T)(l.gamma - 1.0);
  a.dx = l.dx;
  a.dt = l.dt;
  a.cfl = l.cfl;
  a.dt_dev = l.dt_dev;
  a.lam_in = l.lam_in;
  a.lam_next = l.lam_next;
  a.dt_slot = l.dt_slot;
  a.lam_patch = l.lam_patch;
  a.corr = l.corr;
  a.corr_stride = l.corr_stride;
  a.status = l.status;
  a.one = T(1);
  a.mone = T(-1);
  a.mzero = T(-0.0);
  a.dx_patch = l.dx_patch;
  a.dt_patch = l.dt_patch;
  a.local_cfl = l.local_cfl ? 1 : 0;
  a.prim_in = static_cast<const T*>(l.prim_in);
  a.prim_out = static_cast<T*>(l.prim_out);
  a.prim_stride = l.prim_stride;
  a.wait_limit = h->wait_limit;
  a.queue = l.queue;
  const size_t smem = step_smem_bytes<D>((int)sizeof(T), l.pmax, a.nstage);
  cudaError_t e = ensure_smem<T, D, GATHER, FUSED, PRIMIN, NT>(smem);
  if (e != cudaSuccess) return e;
  step_kernel<T, D, GATHER, FUSED, PRIMIN, NT><<<grid, NT, smem, h->stream>>>(a);
  return cudaGetLastError();
}

template <typename T, int D, bool GATHER, bool FUSED, bool PRIMIN, int NT>
static cudaError_t occupancy_t(int pmax, int nstage, int* bps) {
  const size_t smem = step_smem_bytes<D>((int)sizeof(T), pmax, nstage);
  cudaError_t e = ensure_smem<T, D, GATHER, FUSED, PRIMIN, NT>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      bps, step_kernel<T, D, GATHER, FUSED, PRIMIN, NT>, NT, smem);
}

// Launch / occupancy of one precision and CTA size, dispatched over d and
// the mode (explicitly instantiated in the fv_update*.cu translation units).
// d = 1 is built for 128 threads only.
template <typename T, int NT, bool G_, bool F_, bool P_>
static cudaError_t launch_by_d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  if (h->d == 2) return launch_step_t<T, 2, G_, F_, P_, NT>(h, l, grid);
  if (h->d == 3) return launch_step_t<T, 3, G_, F_, P_, NT>(h, l, grid);
  if constexpr (NT == 128) return launch_step_t<T, 1, G_, F_, P_, NT>(h, l, grid);
  return cudaErrorInvalidConfiguration;
}

template <typename T, int NT, bool G_, bool F_, bool P_>
static cudaError_t occupancy_by_d(int d, int pmax, int nstage, int* bps) {
  if (d == 2) return occupancy_t<T, 2, G_, F_, P_, NT>(pmax, nstage, bps);
  if (d == 3) return occupancy_t<T, 3, G_, F_, P_, NT>(pmax, nstage, bps);
  if constexpr (NT == 128) return occupancy_t<T, 1, G_, F_, P_, NT>(pmax, nstage, bps);
  return cudaErrorInvalidConfiguration;
}

template <typename T, int NT>
cudaError_t launch_step_nt(const fv_batch* h, const UpdateLaunch& l, int grid) {
  const int mode = step_mode(l);
  if (mode == kModePrim) return launch_by_d<T, NT, true, true, true>(h, l, grid);
  if (mode == kModeStep) return launch_by_d<T, NT, true, true, false>(h, l, grid);
  return launch_by_d<T, NT, false, false, false>(h, l, grid);
}

template <typename T, int NT>
cudaError_t occupancy_nt(int d, int mode, int pmax, int nstage, int* bps) {
  if (mode == kModePrim) return occupancy_by_d<T, NT, true, true, true>(d, pmax, nstage, bps);
  if (mode == kModeStep) return occupancy_by_d<T, NT, true, true, false>(d, pmax, nstage, bps);
  return occupancy_by_d<T, NT, false, false, false>(d, pmax, nstage, bps);
}

}  // namespace fv
