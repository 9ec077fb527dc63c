// fv_meta.cuh -- where a patch's data come from, for the FP32 kernels built
// for one patch size (fv_rows2d.cu, fv_march3d.cu), loaded in three
// dependent steps that those kernels spread over their loop iterations, so
// that no iteration waits on its own loads:
//
//   1. the patch index (the schedule's order, or the position itself);
//   2. the patch's size and offset, and its neighbour across face f;
//   3. the neighbour's size and offset.
//
// Every index is clamped to a valid entry (a position past the launch: the
// launch's first; a neighbour that is not a patch: the patch itself), so each
// load stays in bounds whatever the table holds.  finish_patch() then applies
// the rules of the general kernel's face_source (Algorithm 1 step 5: the
// face-halo cells come from the neighbour's interior layer next to the face,
// a wall's mirror of the own layer, or the outflow copy of it; in update mode
// from the own halo layer) and flags what the general kernel flags.
#pragma once

#include "fv_step.cuh"

namespace fv {

struct MetaPatch {  // after step 2
  long long off;
  int pid, pj, nb;
};
struct MetaNbr {  // after step 3
  long long onb;
  int snb;
};
// A patch and the source of one of its faces: the source patch's offset, the
// source layer along the face normal | wall flag << 8.
struct PatchSrc {
  long long fo, off;
  int fck, pid, act;
};

__device__ __forceinline__ int meta_pid(const StepParams<float>& a, int64_t pos) {
  const int64_t pc = pos < a.i_end ? pos : a.i_begin;
  return a.order != nullptr ? a.order[pc] : (int)pc;
}

// Step 2 for face f (2D faces per patch in the neighbour table).
template <int D, bool STEP>
__device__ __forceinline__ MetaPatch meta_patch(const StepParams<float>& a, int pid, int f) {
  MetaPatch m;
  m.pid = pid;
  m.pj = a.sizes[pid];
  m.off = a.off[pid];
  m.nb = -1;
  if constexpr (STEP) m.nb = a.nbr[(int64_t)pid * (2 * D) + f];
  return m;
}

template <bool STEP>
__device__ __forceinline__ MetaNbr meta_nbr(const StepParams<float>& a, const MetaPatch& m) {
  MetaNbr t{0, 0};
  if constexpr (STEP) {
    const int nc = (m.nb >= 0 && m.nb < a.n) ? m.nb : m.pid;
    t.onb = a.off[nc];
    t.snb = a.sizes[nc];
  }
  return t;
}

// The patch at `pos` and the source of its face f (want_face: this lane
// records one) from the loaded metadata.  `flag` lanes report a patch of
// another size or layout (one lane per patch).
template <int D, int P, bool STEP>
__device__ __forceinline__ PatchSrc finish_patch(const StepParams<float>& a, int64_t pos,
                                                 const MetaPatch& m, const MetaNbr& t, int f,
                                                 bool want_face, bool flag) {
  const int BOX = stage_elems<D>(P);
  PatchSrc n{0, 0, 0, 0, 0};
  if (pos >= a.i_end) return n;
  const bool act = m.pj == P && m.off >= 0 && (m.off % 4) == 0 &&
                   (a.n_elems <= 0 || m.off + (int64_t)BOX <= a.n_elems);
  if (!act && flag) atomicOr(a.status, ST_BAD_PATCH);  // other size or bad layout
  n.pid = m.pid;
  n.off = m.off;
  n.act = act ? 1 : 0;
  if (act && want_face) {
    const int side = f & 1;
    long long so = m.off;
    int ck, neg = 0;
    if constexpr (!STEP) {
      ck = side ? P + 1 : 0;  // the own halo layer
    } else {
      ck = side ? P : 1;  // outflow: the own interior layer next to the face
      if (m.nb >= 0) {
        const bool ok = m.nb < a.n && t.snb == P && t.onb >= 0 && (t.onb % 4) == 0 &&
                        (a.n_elems <= 0 || t.onb + (int64_t)BOX <= a.n_elems);
        if (ok) {
          so = t.onb;
          ck = side ? 1 : P;  // the neighbour's interior layer next to the face
        } else {
          atomicOr(a.status, ST_BAD_PATCH);
        }
      } else if (m.nb == -2) {
        neg = 1;  // wall: mirror of the own interior layer
      } else if (m.nb != -1) {
        atomicOr(a.status, ST_BAD_PATCH);
      }
    }
    n.fo = so;
    n.fck = ck | (neg << 8);
  }
  return n;
}

// All three steps at once (the first patches of a warp).
template <int D, int P, bool STEP>
__device__ __forceinline__ PatchSrc resolve_now(const StepParams<float>& a, int64_t pos, int f,
                                                bool want_face, bool flag) {
  const MetaPatch m = meta_patch<D, STEP>(a, meta_pid(a, pos), f);
  return finish_patch<D, P, STEP>(a, pos, m, meta_nbr<STEP>(a, m), f, want_face, flag);
}

}  // namespace fv
