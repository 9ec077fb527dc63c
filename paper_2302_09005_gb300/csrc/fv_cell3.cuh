// fv_cell3.cuh -- one FP32 3D Euler cell in registers for the kernel built
// for one 3D patch size (fv_march3d.cu): its state and
// primitives (Eq. 2) and the Rusanov flux G = 2F of a face (Eq. 4, 5), with
// the operations, in order, of primitives<float, 3>() and of the face flux of
// the general kernel (fv_step.cuh), so results are bitwise the same.
#pragma once

#include "fv_device.cuh"

namespace fv {

__device__ __forceinline__ unsigned umax_l(unsigned a, unsigned b) { return a > b ? a : b; }
// |u| + c of a cell as its IEEE bits (>= 0 or NaN, so unsigned maxima order
// them like the values)
__device__ __forceinline__ unsigned wbits_l(float u, float c) {
  return __float_as_uint(add_rn(fabsf(u), c));
}
constexpr unsigned kMagL = 0x7FFFFFFFu;
// positivity of rho and p accumulated as max(bits - 1): 0 < x < inf <=>
// bits(x) - 1 < 0x7F7FFFFF
constexpr unsigned kBadL = 0x7F7FFFFFu;

// State and primitives of one cell: rho, j_x, j_y, j_z, E; u, p, c, E + p.
struct LCell {
  float q[5];
  float u[3], p, c, e;
};

// Primitives (Eq. 2); `need` keeps non-cells out of the positivity check.
__device__ __forceinline__ void lprims(LCell& x, float gm1, float gamma, bool need,
                                       unsigned& chk) {
  const float inv = recip(x.q[0]);
  x.u[0] = mul_rn(x.q[1], inv);
  x.u[1] = mul_rn(x.q[2], inv);
  x.u[2] = mul_rn(x.q[3], inv);
  float jj = mul_rn(x.q[1], x.u[0]);
  jj = fmaf(x.q[2], x.u[1], jj);
  jj = fmaf(x.q[3], x.u[2], jj);
  x.p = mul_rn(gm1, fmaf(-0.5f, jj, x.q[4]));
  x.e = add_rn(x.q[4], x.p);
  x.c = sqrt_t(mul_rn(mul_rn(gamma, x.p), inv));
  const unsigned m = need ? ~0u : 0u;
  chk = umax_l(chk, (__float_as_uint(x.q[0]) - 1u) & m);
  chk = umax_l(chk, (__float_as_uint(x.p) - 1u) & m);
}

// G = 2F of one face along k between the cells L (below) and R (above),
// g[v] for the unknowns v; returns the bits of the face's wave speed a.
template <int K>
__device__ __forceinline__ unsigned lflux(const LCell& L, const LCell& R, float (&g)[5]) {
  const unsigned ab = umax_l(wbits_l(L.u[K], L.c), wbits_l(R.u[K], R.c));
  const float am = __uint_as_float(ab);
  const float sL = add_rn(L.u[K], am), sR = sub_rn(R.u[K], am), ps = add_rn(L.p, R.p);
  g[0] = fmaf(L.q[0], sL, mul_rn(R.q[0], sR));
#pragma unroll
  for (int m = 0; m < 3; ++m)
    g[1 + m] = m == K ? fmaf(L.q[1 + m], sL, fmaf(R.q[1 + m], sR, ps))
                      : fmaf(L.q[1 + m], sL, mul_rn(R.q[1 + m], sR));
  g[4] = fmaf(am, sub_rn(L.q[4], R.q[4]), fmaf(L.e, L.u[K], mul_rn(R.e, R.u[K])));
  return ab;
}

}  // namespace fv
