// fv_update.cu -- the batched Rusanov patch update (Eq. 3-5, Algorithm 1 with
// the outer loop over patches), in two modes sharing one kernel:
//
//   update     (fv_patch_update_batch) the halo cells are read from the input
//              patch, as filled by fv_halo_fill;
//   time step  (fv_time_step) the face-halo cells are gathered straight from
//              the neighbours' interiors (periodic / outflow / wall as in
//              fv_halo_fill), dt comes from the CFL condition on the maximum
//              wave speed the previous step left on the device, and the
//              kernel reduces the maximum wave speed of the new state for the
//              next step.  One launch replaces halo fill + reduce + update
//              and gives bitwise the same result.
//
// Each CTA is persistent and walks its patches i = blockIdx.x + k*gridDim.x.
// While it computes patch i, the TMA engine copies patch i+1 into the other
// of two shared-memory stages (cp.async.bulk, completion on an mbarrier), and
// the halo cells of patch i+1 that live elsewhere are gathered with cp.async.
// Per patch:
//   cells   every interior cell converts to primitives once and writes, per
//           direction, its flux f^k and wave speed |u_k| + c (Eq. 2, 5) into
//           a per-direction box; then every face-halo cell does the same for
//           its normal direction only.  The two groups start on warp
//           boundaries, and halo lanes select their direction without
//           branching, so warps never diverge.
//   faces   every face flux G = f_L + f_R - a (Q_R - Q_L) = 2F (Eq. 4) is
//           computed exactly once and shared by its two cells;
//   update  every interior cell sums G_+ - G_- over x, then y, then z and
//           writes Q - (dt / 2dx) sum (Eq. 3).
// Maxima (per-patch a of Algorithm 1 step 10, next-step wave speed) are taken
// on integer bit patterns: exact and independent of the order of work.
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
  const int32_t* __restrict__ nbr;  // time-step mode
  const int32_t* __restrict__ order;  // processing order (patch indices), or null
  int64_t i_begin, i_end;             // positions of the sequence this launch runs
  int64_t n;                          // patches in the batch
  int64_t n_elems;
  int pmax;
  int nstage;  // shared-memory stages: 2 (copy overlaps compute) or 1
  T gamma, gm1;
  double dx, dt, cfl;
  const double* dt_dev;               // update mode with dt <= 0
  const unsigned long long* lam_in;   // time-step mode: bits of lambda(Q^n)
  unsigned long long* lam_next;       // time-step mode: bits of lambda(Q^n+1)
  double* dt_slot;                    // time-step mode: dt used, written once
  double* lam_patch;
  unsigned int* status;
  const float* corr;    // per-face flux corrections [patch][k][v][face], or null
  int64_t corr_stride;  // floats per patch of corr
};

template <int D>
__host__ __device__ inline int ipow_d(int b) {
  return D == 1 ? b : D == 2 ? b * b : b * b * b;
}
template <int D>
__host__ __device__ inline int stage_elems(int p) {
  return ipow_d<D>(p + 2) * (D + 2);
}
template <int D>
__host__ __device__ inline int fbox_elems(int p) {
  return D * (D + 3) * (p + 2) * (ipow_d<D>(p) / p);
}
template <int D>
__host__ __device__ inline int gface_elems(int p) {
  return D * (D + 2) * (p + 1) * (ipow_d<D>(p) / p);
}
__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Unroll factors of the cell and face loops (two independent work items per
// thread let the FP64 chains of one interleave with the other's latency).
#ifndef FV_UNROLL_CELLS
#define FV_UNROLL_CELLS 1
#endif
#ifndef FV_UNROLL_FACES
#define FV_UNROLL_FACES 1
#endif
#define FV_STR_(x) #x
#define FV_PRAGMA_UNROLL(n) _Pragma(FV_STR_(unroll n))

// Shared-memory header: two mbarriers (16 B), per-warp reduction slots, and
// the face sources of the two stages (2 x 6 x 16 B).
constexpr int kRedOff = 16;
constexpr int kFaceSrcOff = 64;
constexpr int kHdrBytes = 256;
static_assert(kRedOff + 8 * (FV_NT / 32) <= kFaceSrcOff, "header too small");
static_assert(kFaceSrcOff + 2 * 6 * 16 <= kHdrBytes, "header too small");

// Shared-memory carve-up for patches up to pmax (element counts of T).  Two
// stages let the copy of the next patch overlap the current one; when two do
// not fit in shared memory (large patches) one stage is used and the copy of
// the next patch starts after the current patch is done.
template <int D>
struct Carve {
  int nstage, stage, fbox, gface;
  __host__ __device__ Carve(int pmax, int vec, int nstage_)
      : nstage(nstage_),
        stage(round_up(stage_elems<D>(pmax), vec)),
        fbox(round_up(fbox_elems<D>(pmax), vec)),
        gface(round_up(gface_elems<D>(pmax), vec)) {}
  __host__ __device__ int total() const { return nstage * stage + fbox + gface; }
};

// Clock cycles a CTA waits for a copy before it reports FV_ERR_TIMEOUT
// (about one second at 2 GHz).
constexpr long long kWaitLimit = 2000000000ll;

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

// Thread 0: bulk copy of the 16-byte-aligned body of patch j into a stage.
// The ragged tail (< 16 bytes) lies in the last cell of the patch, a corner
// (d >= 2, never read) or the +x halo cell (d = 1, gathered separately).
template <typename T, int D>
__device__ __forceinline__ void issue_stage(const StepParams<T>& a, int pj, int64_t offj, T* st,
                                            uint64_t* bar) {
  const uint32_t bytes = (uint32_t)(stage_elems<D>(pj) * sizeof(T)) & ~15u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, bytes);
  bulk_copy_g2s(st, a.in + offj, bytes, bar);
}

// Where the face-halo cells of one face come from: a patch (element offset),
// the layer along the face normal in that patch, and whether the normal
// momentum is negated (wall).
struct FaceSrc {
  long long off;
  int ck;
  int neg;
};

// Threads 0 .. 2d-1: resolve the sources of the 2d faces of patch j once (the
// neighbour table and the neighbour's metadata are read and checked here, not
// per halo element).  Time-step mode follows the rules of fv_halo_fill;
// update mode with d = 1 re-reads the patch's own halo cells.
template <typename T, int D, bool GATHER>
__device__ __forceinline__ void face_sources(const StepParams<T>& a, int64_t j, int pj,
                                             int64_t offj, FaceSrc* fs) {
  if constexpr (!GATHER && D != 1) return;
  constexpr int VEC = 16 / sizeof(T);
  const int f = threadIdx.x;
  if (f >= 2 * D) return;
  const int side = f & 1;
  FaceSrc r;
  r.off = offj;
  r.neg = 0;
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
  fs[f] = r;
}

// All threads: fetch the face-halo cells of a patch that do not come with its
// bulk copy, from the sources resolved by face_sources, as cp.async element
// copies (a wall's negated normal momentum with a plain load and store).
template <typename T, int D, int P, bool GATHER>
__device__ __forceinline__ void gather_halo(const StepParams<T>& a, int pj, T* st,
                                            const FaceSrc* fs) {
  if constexpr (!GATHER && D != 1) return;
  constexpr int S = D + 2;
  const Geom<D, P> g(pj);
  const int p = g.p;
  const int ptr = g.ptrans();
  for (int hc = threadIdx.x; hc < 2 * D * ptr; hc += FV_NT) {
    const int f = hc / ptr;
    const int r = hc - f * ptr;
    const int k = f >> 1;
    const FaceSrc m = fs[f];
    const int cd = g.cell_kt(k, (f & 1) ? p + 1 : 0, r);
    const int cs = g.cell_kt(k, m.ck, r);
    T* dst = st + cd * S;
    const T* src = a.in + m.off + (int64_t)cs * S;
#pragma unroll
    for (int v = 0; v < S; ++v) {
      if (m.neg && v == 1 + k)
        dst[v] = neg_t(__ldg(src + v));
      else
        cp_async_elem(dst + v, src + v);
    }
  }
  cp_async_commit();
}

template <typename T, int D, bool GATHER>
__device__ __forceinline__ void gather_dispatch(const StepParams<T>& a, int pj, T* st,
                                                const FaceSrc* fs) {
  if constexpr (!GATHER && D != 1) return;
  if constexpr (D == 3) {
    switch (pj) {
      case 3: gather_halo<T, D, 3, GATHER>(a, pj, st, fs); return;
      case 5: gather_halo<T, D, 5, GATHER>(a, pj, st, fs); return;
      case 7: gather_halo<T, D, 7, GATHER>(a, pj, st, fs); return;
      default: gather_halo<T, D, 0, GATHER>(a, pj, st, fs); return;
    }
  } else if constexpr (D == 2) {
    switch (pj) {
      case 3: gather_halo<T, D, 3, GATHER>(a, pj, st, fs); return;
      case 5: gather_halo<T, D, 5, GATHER>(a, pj, st, fs); return;
      case 8: gather_halo<T, D, 8, GATHER>(a, pj, st, fs); return;
      default: gather_halo<T, D, 0, GATHER>(a, pj, st, fs); return;
    }
  } else {
    gather_halo<T, D, 0, GATHER>(a, pj, st, fs);
  }
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
  T* st;
  FaceSrc* fs;
  int slot;
};

// Between the cell and face phases: wait for the bulk copy of the next patch
// and start its halo gather, so both overlap the rest of this patch.
template <typename T, int D, bool GATHER>
__device__ __forceinline__ void mid_hook(const StepParams<T>& a, Pipe& pp,
                                         const NextPatch<T>& nx) {
  if (nx.j >= a.i_end) return;
  const bool ok = mbar_wait_bounded(&pp.bar[nx.slot], (pp.parity >> nx.slot) & 1u, kWaitLimit);
  if (ok) {
    pp.parity ^= 1u << nx.slot;
    pp.pending &= ~(1u << nx.slot);
  }
  if (!ok) {
    pp.timeout = true;
    return;
  }
  gather_dispatch<T, D, GATHER>(a, nx.p, nx.st, nx.fs);
}

// ---------------------------------------------------------------------------
// One patch: cells, faces, update.
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void flux_dir_sel(const T* q, const Prim<T, D>& w, int k, T* f,
                                             T& lam) {
  // direction chosen per lane with selects; fma(x, y, -0) == x * y bitwise
  T uk = w.u[0], jk = q[1];
#pragma unroll
  for (int m = 1; m < D; ++m) {
    uk = (k == m) ? w.u[m] : uk;
    jk = (k == m) ? q[1 + m] : jk;
  }
  f[0] = jk;
#pragma unroll
  for (int m = 0; m < D; ++m) f[1 + m] = fma(q[1 + m], uk, (m == k) ? w.p : T(-0.0));
  f[D + 1] = w.ep * uk;
  lam = abs_t(uk) + w.c;
}

template <typename T, int D, int P, bool GATHER, bool FUSED>
__device__ __forceinline__ void patch_compute(const StepParams<T>& a, int p_rt, int64_t i,
                                              int64_t off, const T* __restrict__ st, T* F, T* G,
                                              T mhr, unsigned long long* red,
                                              unsigned long long& lam_next, Pipe& pp,
                                              const NextPatch<T>& nx) {
  constexpr int S = D + 2;
  constexpr int NT = FV_NT;
  const Geom<D, P> g(p_rt);
  const int p = g.p;
  const int nbox = g.nbox(), nface = g.nface(), nint = g.nint(), ptr = g.ptrans();
  const int tid = threadIdx.x;
  bool bad = false;

  // ---- cells ----------------------------------------------------------------
  {
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
        const Prim<T, D> w = primitives<T, D>(q, a.gm1, a.gamma, bad);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          T f[S], lam;
          flux_dir<T, D>(q, w, k, f, lam);
          const int b = g.trans(c, k) + ptr * c[k];
          T* Fk = F + k * (S + 1) * nbox;
#pragma unroll
          for (int v = 0; v < S; ++v) Fk[v * nbox + b] = f[v];
          Fk[S * nbox + b] = lam;
        }
      } else if (t >= nint_pad) {
        const int hc = t - nint_pad;
        const int f = hc / ptr;
        const int r = hc - f * ptr;
        const int k = f >> 1;
        const int ck = (f & 1) ? p + 1 : 0;
        const int cid = g.cell_kt(k, ck, r);
        T q[S];
#pragma unroll
        for (int v = 0; v < S; ++v) q[v] = st[cid * S + v];
        const Prim<T, D> w = primitives<T, D>(q, a.gm1, a.gamma, bad);
        T fl[S], lam;
        flux_dir_sel<T, D>(q, w, k, fl, lam);
        const int b = r + ptr * ck;
        T* Fk = F + k * (S + 1) * nbox;
#pragma unroll
        for (int v = 0; v < S; ++v) Fk[v * nbox + b] = fl[v];
        Fk[S * nbox + b] = lam;
      }
    }
  }
  __syncthreads();
  mid_hook<T, D, GATHER>(a, pp, nx);

  // ---- faces: G = f_L + f_R - a (Q_R - Q_L), once per face -------------------
  unsigned long long lmax = 0ull;
  FV_PRAGMA_UNROLL(FV_UNROLL_FACES)
  for (int t = tid; t < D * nface; t += NT) {
    const int k = t / nface;
    const int j = t - k * nface;
    const int b = j / ptr;
    const int tr = j - b * ptr;
    const int cl = g.cell_kt(k, b, tr);
    const int cr = cl + g.stride(k);
    const T* Fk = F + k * (S + 1) * nbox;
    const int bl = tr + ptr * b;  // box index of the left cell; right: bl + ptr
    const T am = max_by_bits(Fk[S * nbox + bl], Fk[S * nbox + bl + ptr]);
    const unsigned long long ab = order_bits(am);
    lmax = ab > lmax ? ab : lmax;
    T* Gk = G + k * S * nface;
#pragma unroll
    for (int v = 0; v < S; ++v) {
      // f_L + f_R - a (Q_R - Q_L), with the sign folded into the difference
      const T dqn = st[cl * S + v] - st[cr * S + v];
      const T fs = Fk[v * nbox + bl] + Fk[v * nbox + bl + ptr];
      T gv = fma(am, dqn, fs);
      // learned correction C of this face (G = 2F, so G + 2C = 2(F + C))
      if (a.corr != nullptr) gv += T(2) * (T)a.corr[i * a.corr_stride + (k * S + v) * nface + j];
      Gk[v * nface + j] = gv;
    }
  }
  __syncthreads();

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
        const T dG = Gk[v * nface + jm + ptr] - Gk[v * nface + jm];
        acc[v] = k == 0 ? dG : acc[v] + dG;
      }
    }
    T qn[S];
#pragma unroll
    for (int v = 0; v < S; ++v) qn[v] = fma(mhr, acc[v], st[cid * S + v]);
    T* dst = dst_base + (int64_t)cid * S;
#pragma unroll
    for (int v = 0; v < S; ++v) dst[v] = qn[v];
    if constexpr (FUSED) {
      // wave speed of the new state for the next step's CFL condition
      const Prim<T, D> w = primitives<T, D>(qn, a.gm1, a.gamma, bad);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const unsigned long long lb = order_bits(abs_t(w.u[k]) + w.c);
        lam_next = lb > lam_next ? lb : lam_next;
      }
    }
  }

  if (bad) atomicOr(a.status, ST_NONPHYSICAL);
  if (a.lam_patch != nullptr) {
    lmax = warp_max_u64(lmax);
    if ((tid & 31) == 0) red[tid >> 5] = lmax;
    __syncthreads();
    if (tid == 0) {
      unsigned long long m = red[0];
#pragma unroll
      for (int w = 1; w < NT / 32; ++w) m = red[w] > m ? red[w] : m;
      a.lam_patch[i] = order_value<T>(m);
    }
  }
}

template <typename T, int D, bool GATHER, bool FUSED>
__device__ __forceinline__ void patch_dispatch(const StepParams<T>& a, int p, int64_t i,
                                               int64_t off, const T* st, T* F, T* G, T hr,
                                               unsigned long long* red,
                                               unsigned long long& lam_next, Pipe& pp,
                                               const NextPatch<T>& nx) {
#define FV_PC(PP) \
  patch_compute<T, D, PP, GATHER, FUSED>(a, p, i, off, st, F, G, hr, red, lam_next, pp, nx)
  if constexpr (D == 3) {
    switch (p) {
      case 3: FV_PC(3); return;
      case 5: FV_PC(5); return;
      case 7: FV_PC(7); return;
      default: FV_PC(0); return;
    }
  } else if constexpr (D == 2) {
    switch (p) {
      case 3: FV_PC(3); return;
      case 5: FV_PC(5); return;
      case 8: FV_PC(8); return;
      case 17: FV_PC(17); return;
      default: FV_PC(0); return;
    }
  } else {
    FV_PC(0);
  }
#undef FV_PC
}

// Resident CTAs per SM the register allocation is sized for.
#ifndef FV_MINBLOCKS_FP64
#define FV_MINBLOCKS_FP64 3
#endif
#ifndef FV_MINBLOCKS_FP32
#define FV_MINBLOCKS_FP32 6
#endif

template <typename T, int D, bool GATHER, bool FUSED>
__global__ void __launch_bounds__(FV_NT, sizeof(T) == 8 ? FV_MINBLOCKS_FP64 : FV_MINBLOCKS_FP32)
    step_kernel(StepParams<T> a) {
  constexpr int VEC = 16 / sizeof(T);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem_raw + kRedOff);
  FaceSrc* fsrc = reinterpret_cast<FaceSrc*>(smem_raw + kFaceSrcOff);  // [stage][face]
  const Carve<D> cv(a.pmax, VEC, a.nstage);
  const bool single = a.nstage == 1;
  T* stage[2];
  stage[0] = reinterpret_cast<T*>(smem_raw + kHdrBytes);
  stage[1] = single ? stage[0] : stage[0] + cv.stage;
  T* F = stage[0] + cv.nstage * cv.stage;
  T* G = F + cv.fbox;
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
  // pos itself), CTA b takes positions i_begin + b, + gridDim.x, ...
  auto pid_of = [&](int64_t pos) -> int64_t {
    return a.order != nullptr ? (int64_t)a.order[pos] : pos;
  };
  // first valid patch of this CTA, staged before the loop
  int64_t cur = a.i_begin + blockIdx.x;
  int64_t pidc = 0;
  int pc = 0;
  int64_t oc = 0;
  while (cur < a.i_end && !patch_ok<T, D>(a, pidc = pid_of(cur), pc, oc)) cur += gridDim.x;
  int s = 0;
  if (cur < a.i_end) {
    face_sources<T, D, GATHER>(a, pidc, pc, oc, fsrc);
    if (tid == 0) issue_stage<T, D>(a, pc, oc, stage[0], &bar[0]);
    pp.pending = 1u;
    __syncthreads();  // face sources visible
    const bool ok = mbar_wait_bounded(&bar[0], 0u, kWaitLimit);
    if (ok) {
      pp.parity ^= 1u;
      pp.pending = 0u;
      gather_dispatch<T, D, GATHER>(a, pc, stage[0], fsrc);
    } else {
      pp.timeout = true;
    }
    cp_async_wait_all();
  }
  if (__syncthreads_or(pp.timeout)) cur = a.i_end;

  while (cur < a.i_end) {
    NextPatch<T> nx;
    nx.j = cur + gridDim.x;
    nx.pid = 0;
    while (nx.j < a.i_end && !patch_ok<T, D>(a, nx.pid = pid_of(nx.j), nx.p, nx.off))
      nx.j += gridDim.x;
    nx.slot = single ? 0 : s ^ 1;
    nx.st = stage[nx.slot];
    nx.fs = fsrc + 6 * nx.slot;
    // visible to all threads after the barrier that ends the cell phase
    if (nx.j < a.i_end) face_sources<T, D, GATHER>(a, nx.pid, nx.p, nx.off, nx.fs);
    NextPatch<T> nx_mid = nx;  // what the mid-patch hook waits for and gathers
    if (single) {
      nx_mid.j = a.i_end;  // the one stage is busy until this patch is done
    } else if (nx.j < a.i_end) {
      if (tid == 0) issue_stage<T, D>(a, nx.p, nx.off, nx.st, &bar[nx.slot]);
      pp.pending |= 1u << nx.slot;
    }
    patch_dispatch<T, D, GATHER, FUSED>(a, pc, pidc, oc, stage[s], F, G, hr, red, lam_next, pp,
                                        nx_mid);
    cp_async_wait_all();
    if (__syncthreads_or(pp.timeout)) break;
    if (single && nx.j < a.i_end) {
      if (tid == 0) issue_stage<T, D>(a, nx.p, nx.off, nx.st, &bar[0]);
      pp.pending |= 1u;
      mid_hook<T, D, GATHER>(a, pp, nx);
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
      for (int w = 1; w < FV_NT / 32; ++w) m = red[w] > m ? red[w] : m;
      atomicMax(a.lam_next, m);
    }
  }
}

size_t update_smem_bytes(int d, fv_precision prec, int pmax, int nstage) {
  const int es = prec == FV_FP64 ? 8 : 4;
  const int vec = 16 / es;
  const int elems = d == 1   ? Carve<1>(pmax, vec, nstage).total()
                    : d == 2 ? Carve<2>(pmax, vec, nstage).total()
                             : Carve<3>(pmax, vec, nstage).total();
  return kHdrBytes + (size_t)es * elems;
}

// Raises the kernel's dynamic shared-memory limit on the current device once
// (not per launch, so launches can be captured into CUDA graphs).
template <typename T, int D, bool GATHER, bool FUSED>
static cudaError_t ensure_smem(size_t smem) {
  static int set_bytes[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && set_bytes[dev] >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(step_kernel<T, D, GATHER, FUSED>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < 64) set_bytes[dev] = (int)smem;
  return e;
}

template <typename T, int D, bool GATHER, bool FUSED>
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
  const size_t smem = update_smem_bytes(D, h->prec, l.pmax, a.nstage);
  cudaError_t e = ensure_smem<T, D, GATHER, FUSED>(smem);
  if (e != cudaSuccess) return e;
  step_kernel<T, D, GATHER, FUSED><<<grid, FV_NT, smem, h->stream>>>(a);
  return cudaGetLastError();
}

template <typename T, bool GATHER, bool FUSED>
static cudaError_t launch_by_d(const fv_batch* h, const UpdateLaunch& l, int grid) {
  if (h->d == 1) return launch_step_t<T, 1, GATHER, FUSED>(h, l, grid);
  if (h->d == 2) return launch_step_t<T, 2, GATHER, FUSED>(h, l, grid);
  return launch_step_t<T, 3, GATHER, FUSED>(h, l, grid);
}

cudaError_t launch_update(const fv_batch* h, const UpdateLaunch& l, int grid) {
  if (l.fused) {
    return h->prec == FV_FP64 ? launch_by_d<double, true, true>(h, l, grid)
                              : launch_by_d<float, true, true>(h, l, grid);
  }
  return h->prec == FV_FP64 ? launch_by_d<double, false, false>(h, l, grid)
                            : launch_by_d<float, false, false>(h, l, grid);
}

template <typename T, int D, bool GATHER, bool FUSED>
static cudaError_t occupancy_t(const fv_batch* h, int pmax, int nstage, int* bps) {
  const size_t smem = update_smem_bytes(D, h->prec, pmax, nstage);
  cudaError_t e = ensure_smem<T, D, GATHER, FUSED>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, step_kernel<T, D, GATHER, FUSED>,
                                                       FV_NT, smem);
}

template <typename T, bool GATHER, bool FUSED>
static cudaError_t occ_by_d(const fv_batch* h, int pmax, int nstage, int* bps) {
  if (h->d == 1) return occupancy_t<T, 1, GATHER, FUSED>(h, pmax, nstage, bps);
  if (h->d == 2) return occupancy_t<T, 2, GATHER, FUSED>(h, pmax, nstage, bps);
  return occupancy_t<T, 3, GATHER, FUSED>(h, pmax, nstage, bps);
}

cudaError_t step_occupancy(const fv_batch* h, bool fused, int pmax, int nstage, int* bps) {
  if (fused)
    return h->prec == FV_FP64 ? occ_by_d<double, true, true>(h, pmax, nstage, bps)
                              : occ_by_d<float, true, true>(h, pmax, nstage, bps);
  return h->prec == FV_FP64 ? occ_by_d<double, false, false>(h, pmax, nstage, bps)
                            : occ_by_d<float, false, false>(h, pmax, nstage, bps);
}

cudaError_t update_occupancy(const fv_batch* h, bool fused, int* bps) {
  return step_occupancy(h, fused, h->max_patch_size, h->nstage, bps);
}

}  // namespace fv
