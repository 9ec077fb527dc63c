// fv_x2.cuh -- packed FP32 pairs for sm_100-class GPUs: two floats in one
// 64-bit register, added, subtracted, multiplied or fused-multiply-added by
// one instruction (add / sub / mul / fma .rn.f32x2).  Each half rounds
// exactly like the scalar .rn operation, so a packed expression gives
// bitwise the results of the same expression written per element; it costs
// half the instruction issue.
#pragma once

#include <stdint.h>

namespace fv {

typedef unsigned long long f2;  // low half: first element, high half: second

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float f2_lo(f2 v) {
  float lo, hi;
  f2_unpack(v, lo, hi);
  return lo;
}
__device__ __forceinline__ float f2_hi(f2 v) {
  float lo, hi;
  f2_unpack(v, lo, hi);
  return hi;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

}  // namespace fv
