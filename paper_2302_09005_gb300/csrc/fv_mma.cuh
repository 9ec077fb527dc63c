// fv_mma.cuh -- BF16 conversions, the activation of the learned face-flux
// correction network and the layout of its parameter vector (shared by the
// tcgen05 training and correction kernels).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace fv {

// Two floats -> two bf16 (round to nearest even) packed low, high.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_bf16_raw(uint16_t lo, uint16_t hi) {
  return (uint32_t)lo | ((uint32_t)hi << 16);
}
__device__ __forceinline__ float bf16_to_f32(uint16_t x) {
  return __uint_as_float((uint32_t)x << 16);
}
__device__ __forceinline__ uint16_t f32_to_bf16(float x) {
  const __nv_bfloat16 v = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&v);
}

// gelu(z) = z Phi(z), Phi the standard normal distribution function,
// evaluated on the GPU in its tanh form
//   gelu(z) ~ z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
// with the hardware tanh (one special-function instruction instead of the
// polynomial of erf).  The tanh form stays within 5e-4 of z Phi(z) (2e-4
// relative, the worst near z = 2.7) and the hardware tanh within 2^-11
// relative; both below the BF16 rounding the activations get next (2^-9
// relative).  Training uses the same form and its
// exact derivative, so the network is trained for what it evaluates.
__device__ __forceinline__ float tanh_hw(float u) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return t;
}
__device__ __forceinline__ float gelu_f(float z) {
  const float u = z * fmaf(0.0356774081f, z * z, 0.7978845608f);
  const float h = 0.5f * z;
  return fmaf(h, tanh_hw(u), h);
}
// d/dz of the tanh form: (1 + t)/2 + z/2 (1 - t^2) sqrt(2/pi) (1 + 3 0.044715 z^2).
__device__ __forceinline__ float gelu_prime_f(float z) {
  const float z2 = z * z;
  const float t = tanh_hw(z * fmaf(0.0356774081f, z2, 0.7978845608f));
  const float du = fmaf(0.1070322244f, z2, 0.7978845608f);
  return fmaf(0.5f * z * du, fmaf(-t, t, 1.0f), fmaf(0.5f, t, 0.5f));
}

// Layout of the flat parameter vector of the 16 -> 64 -> 64 -> 4 network:
// W1 (64x16, output-major), b1 (64), W2 (64x64), b2 (64), W3 (4x64), b3 (4).
constexpr int kMlpIn = 16, kMlpHid = 64, kMlpOut = 4;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHid * kMlpIn;    // 1024
constexpr int kOffW2 = kOffB1 + kMlpHid;             // 1088
constexpr int kOffB2 = kOffW2 + kMlpHid * kMlpHid;   // 5184
constexpr int kOffW3 = kOffB2 + kMlpHid;             // 5248
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpHid;   // 5504
constexpr int kMlpParams = kOffB3 + kMlpOut;         // 5508
// Normalisation block: mu_x (16), sd_x (16), sd_y (4).
constexpr int kNormLen = 36;

}  // namespace fv
