// fv_device.cuh -- device-side building blocks of the Rusanov patch kernels:
// Euler physics (Eq. 2, Eq. 5), bit-level helpers for exact maxima and
// positivity checks, and the compile-time patch geometry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fv {

// Status bits of the handle's device status word.
enum : unsigned int {
  ST_BAD_PATCH = 1u,
  ST_NONPHYSICAL = 2u,
  ST_TIMEOUT = 4u,
};

// ---------------------------------------------------------------------------
// Bit-level helpers.  A wave speed |u|+c is >= 0 or NaN.  With the sign bit
// cleared, the IEEE bit pattern orders non-negative values like the values
// themselves and puts every NaN above +inf, so maxima taken on the integer
// patterns are exact, order independent, and propagate NaN.  They run on the
// integer pipe, which keeps the FP64 pipe free.
// ---------------------------------------------------------------------------
// The mask is applied in inline PTX: written as C++, the compiler recognises
// "clear the sign bit" as |x| and spends an FP64 add on it.
__device__ __forceinline__ unsigned long long order_bits(double x) {
  unsigned long long r;
  asm("and.b64 %0, %1, 0x7FFFFFFFFFFFFFFF;" : "=l"(r) : "l"(__double_as_longlong(x)));
  return r;
}
__device__ __forceinline__ unsigned long long order_bits(float x) {
  unsigned int r;
  asm("and.b32 %0, %1, 0x7FFFFFFF;" : "=r"(r) : "r"(__float_as_uint(x)));
  return (unsigned long long)r;
}
// Value of a maximum taken on order_bits of type T, as a double.
template <typename T>
__device__ __forceinline__ double order_value(unsigned long long b);
template <>
__device__ __forceinline__ double order_value<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}
template <>
__device__ __forceinline__ double order_value<float>(unsigned long long b) {
  return (double)__uint_as_float((unsigned int)b);
}
template <typename T>
__device__ __forceinline__ T max_by_bits(T a, T b);
template <>
__device__ __forceinline__ double max_by_bits<double>(double a, double b) {
  return order_bits(a) >= order_bits(b) ? a : b;
}
template <>
__device__ __forceinline__ float max_by_bits<float>(float a, float b) {
  return order_bits(a) >= order_bits(b) ? a : b;
}

// 0 < x < +inf (not NaN), tested on the bit pattern with integer ops.
__device__ __forceinline__ bool positive_finite(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b - 1ull) < 0x7FEFFFFFFFFFFFFFull;
}
__device__ __forceinline__ bool positive_finite(float x) {
  unsigned int b = __float_as_uint(x);
  return (b - 1u) < 0x7F7FFFFFu;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// ---------------------------------------------------------------------------
// |x| and -x on the sign bit with integer operations: exact, and they keep
// the scarce FP64 pipe out of sign manipulations the compiler does not fold
// into a neighbouring instruction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double abs_t(double x) {
  return __hiloint2double(__double2hiint(x) & 0x7FFFFFFF, __double2loint(x));
}
__device__ __forceinline__ float abs_t(float x) { return fabsf(x); }
__device__ __forceinline__ double neg_t(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ float neg_t(float x) { return -x; }

// Explicitly rounded add, subtract and multiply: never contracted into an
// FMA, so an expression rounds the same way wherever it is inlined.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// ---------------------------------------------------------------------------
// The adds, subtracts and multiplies of the FP64 kernels as FMAs.  On GB300
// the FP64 pipe retires DFMA about 1.19 times faster than DADD or DMUL
// (measured: 0.60 vs 0.50 T instructions/s), and
//   a + b = fma(a, 1, b),   a - b = fma(b, -1, a),   a * b = fma(a, b, -0)
// hold bitwise (the product is exact, or the addend -0 leaves it as it is,
// and there is one rounding), signed zeros included.  The constants 1, -1
// and -0 come in as kernel arguments: a literal would let the compiler fold
// the FMA back into the slower instruction.  FP32 keeps plain operations
// (FADD and FMUL run at the FFMA rate).
// ---------------------------------------------------------------------------
template <typename T>
struct Arith {
  T one, mone, mzero;
  __device__ __forceinline__ T add(T a, T b) const { return add_rn(a, b); }
  __device__ __forceinline__ T sub(T a, T b) const { return sub_rn(a, b); }
  __device__ __forceinline__ T mul(T a, T b) const { return mul_rn(a, b); }
};
template <>
struct Arith<double> {
  double one, mone, mzero;
  __device__ __forceinline__ double add(double a, double b) const { return fma(a, one, b); }
  __device__ __forceinline__ double sub(double a, double b) const { return fma(b, mone, a); }
  __device__ __forceinline__ double mul(double a, double b) const { return fma(a, b, mzero); }
};
// A float as a double, exactly, with integer operations (sign; exponent
// rebased from 127 to 1023; the 23 fraction bits on top of the 52): the
// conversion instruction would run on the FP64 pipe, the scarce unit of this
// GPU.  Zero and subnormal floats give a signed zero (subnormals, below
// 1.2e-38, are flushed); infinities and NaNs keep their class.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu, sign = u & 0x80000000u, m = u & 0x7FFFFFu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = u << 29;
  hi = e == 0u ? sign : hi;
  lo = e == 0u ? 0u : lo;
  hi = e == 255u ? (sign | 0x7FF00000u | (m >> 3)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double to_t(float f, double*) { return widen_f32(f); }
__device__ __forceinline__ float to_t(float f, float*) { return f; }

// The same operations with literal constants (the compiler may use plain
// adds and multiplies; the results are the same bits).
template <typename T>
__device__ __forceinline__ Arith<T> plain_arith() {
  return Arith<T>{T(1), T(-1), T(-0.0)};
}

// ---------------------------------------------------------------------------
// Reciprocal and square root, once per cell of the interior and face halo.
//
// FP64 is the scarce unit on GB300 (two FP64 lanes per SM), so the FP64
// forms refine a cheap seed with FMAs instead of running the full IEEE
// division and square root sequences:
//   1/a     Newton-Raphson in its cubic form: with y0 ~ 1/a and
//           e = 1 - a y0, 1/a = y0 / (1 - e) = y0 (1 + e + e^2 + ...), so
//           y = y0 + y0 (e + e^2) leaves a relative error of order e^3;
//   sqrt(x) with r0 ~ x^(-1/2), s0 = x r0 and e = 1 - s0 r0 = 1 - x r0^2,
//           sqrt(x) = s0 (1 - e)^(-1/2) = s0 (1 + e/2 + 3e^2/8 + ...),
//           truncated after the e^2 term (binomial series).
// The seeds come from the FP32 special-function unit, not from the f64
// approximation instructions (which spend FP64 operations of their own): the
// double's sign, exponent and leading 20 fraction bits are repacked as a
// float with integer operations, the float reciprocal / reciprocal square
// root is taken, and the result is repacked as a double.  The seed is good
// to about 2^-20, so the cubic step leaves ~2^-60 for 1/a and the two-term
// series ~2^-62 for sqrt: within an ulp or two of the correctly rounded
// result (measured by fv_selftest_math against the IEEE operations), far
// inside the 1e-12 tolerance of the update.  Arguments outside the float
// exponent range (and zero, negative, non-finite values) take the IEEE
// operation.  The FP32 forms are the special-function unit's approximations
// themselves (one instruction each, within about an ulp and two ulps): the
// FP32 path is bound by instruction issue, where the IEEE sequences cost
// about ten instructions per cell each, and its error target (1e-5 after a
// step) is far above an ulp of FP32.
// ---------------------------------------------------------------------------

// Double -> float carrying the double's leading 20 fraction bits (truncated);
// false if the exponent does not fit a normal float with margin.
__device__ __forceinline__ bool f64_seed_as_f32(double x, float& f) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const int ef = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if ((hi >> 31) != 0u || ef < 4 || ef > 250) return false;
  f = __uint_as_float(((unsigned)ef << 23) | ((hi & 0xFFFFFu) << 3));
  return true;
}
// Exact float -> double by repacking the fields (positive normal floats).
__device__ __forceinline__ double f32_as_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = ((b >> 23) & 0xFFu) - 127u + 1023u;
  return __hiloint2double((int)((e << 20) | ((b & 0x7FFFFFu) >> 3)), (int)((b & 7u) << 29));
}

__device__ __forceinline__ double recip(double a, const Arith<double>& ar = plain_arith<double>()) {
  float f;
  if (!f64_seed_as_f32(a, f)) return 1.0 / a;
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f));
  const double y = f32_as_f64(rf);
  const double e = fma(neg_t(a), y, 1.0);
  const double t = fma(e, e, e);
  return fma(y, t, y);
}
__device__ __forceinline__ float recip(float a, const Arith<float>& = plain_arith<float>()) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

__device__ __forceinline__ double sqrt_t(double x, const Arith<double>& ar = plain_arith<double>()) {
  float f;
  if (!f64_seed_as_f32(x, f)) return sqrt(x);
  float rf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f));
  const double r = f32_as_f64(rf);
  const double s0 = ar.mul(x, r);
  const double e = fma(neg_t(s0), r, 1.0);
  const double t = ar.mul(e, fma(e, 0.375, 0.5));
  return fma(s0, t, s0);
}
__device__ __forceinline__ float sqrt_t(float x, const Arith<float>& = plain_arith<float>()) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------------------
// Euler physics of one cell, Eq. 2: q = (rho, j_1..j_D, E),
// u = j / rho, p = (gamma - 1)(E - j.u / 2), c = sqrt(gamma p / rho).
// ---------------------------------------------------------------------------
template <typename T, int D>
struct Prim {
  T u[D];
  T p;
  T c;
  T ep;  // E + p, shared by the energy flux of every direction
};

template <typename T, int D>
__device__ __forceinline__ Prim<T, D> primitives(const T* q, T gm1, T gamma, bool& bad,
                                                 const Arith<T>& ar = plain_arith<T>()) {
  Prim<T, D> w;
  T inv = recip(q[0], ar);
  T jj = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    w.u[k] = ar.mul(q[1 + k], inv);
    jj = k == 0 ? ar.mul(q[1], w.u[0]) : fma(q[1 + k], w.u[k], jj);
  }
  w.p = ar.mul(gm1, fma(T(-0.5), jj, q[D + 1]));
  w.ep = ar.add(q[D + 1], w.p);
  T c2 = ar.mul(ar.mul(gamma, w.p), inv);
  w.c = sqrt_t(c2, ar);
  bad |= !(positive_finite(q[0]) && positive_finite(w.p));
  return w;
}

// Flux f^k (S = D + 2 values) and wave speed |u_k| + c of one cell (Eq. 2, 5).
template <typename T, int D>
__device__ __forceinline__ void flux_dir(const T* q, const Prim<T, D>& w, int k, T* f, T& lam) {
  T uk = w.u[k];
  f[0] = q[1 + k];
#pragma unroll
  for (int m = 0; m < D; ++m) f[1 + m] = (m == k) ? fma(q[1 + m], uk, w.p) : mul_rn(q[1 + m], uk);
  f[D + 1] = mul_rn(w.ep, uk);
  lam = add_rn(abs_t(uk), w.c);
}

// ---------------------------------------------------------------------------
// Patch geometry with a one-cell halo.  P > 0: compile-time patch size;
// P == 0: runtime size (generic path).
// ---------------------------------------------------------------------------
template <int D, int P>
struct Geom {
  int p;
  __device__ __forceinline__ explicit Geom(int p_rt) : p(P > 0 ? P : p_rt) {}
  __device__ __forceinline__ int ne() const { return p + 2; }
  __device__ __forceinline__ int ncell() const {  // halo-inclusive cells
    return D == 1 ? p + 2 : D == 2 ? (p + 2) * (p + 2) : (p + 2) * (p + 2) * (p + 2);
  }
  __device__ __forceinline__ int ptrans() const {  // p^(D-1)
    return D == 1 ? 1 : D == 2 ? p : p * p;
  }
  __device__ __forceinline__ int nint() const { return ptrans() * p; }     // p^D
  __device__ __forceinline__ int nbox() const { return (p + 2) * ptrans(); }  // cells per dir box
  __device__ __forceinline__ int nface() const { return (p + 1) * ptrans(); }  // faces per dir
  // linear cell index of halo-inclusive coordinates
  __device__ __forceinline__ int cell(const int* c) const {
    int idx = c[D - 1];
#pragma unroll
    for (int m = D - 2; m >= 0; --m) idx = idx * (p + 2) + c[m];
    return idx;
  }
  // transverse index of coordinates c (each interior, 1..p) for direction k:
  // the coordinates other than k, lowest axis fastest, shifted to 0..p-1.
  __device__ __forceinline__ int trans(const int* c, int k) const {
    int t = 0;
#pragma unroll
    for (int m = D - 1; m >= 0; --m)
      if (m != k) t = t * p + (c[m] - 1);
    return t;
  }
  // inverse of trans: fill the coordinates other than k from t
  __device__ __forceinline__ void untrans(int t, int k, int* c) const {
#pragma unroll
    for (int m = 0; m < D; ++m)
      if (m != k) {
        c[m] = 1 + t % p;
        t /= p;
      }
  }
  // Cell index of the cell with coordinate ck along a runtime direction k and
  // transverse index t, built with selects (no dynamically indexed arrays,
  // which would live in local memory).
  __device__ __forceinline__ int cell_kt(int k, int ck, int t) const {
    const int ne = p + 2;
    if constexpr (D == 1) {
      return ck;
    } else if constexpr (D == 2) {
      const int a = 1 + t;
      const int c0 = k == 0 ? ck : a;
      const int c1 = k == 0 ? a : ck;
      return c0 + ne * c1;
    } else {
      const int a = 1 + t % p, b = 1 + t / p;
      const int c0 = k == 0 ? ck : a;
      const int c1 = k == 0 ? a : (k == 1 ? ck : b);
      const int c2 = k == 2 ? ck : b;
      return c0 + ne * (c1 + ne * c2);
    }
  }
  // Interior cell index (0-based coordinates, x fastest, stride p) of the
  // cell with interior coordinate c along direction k and transverse index t.
  __device__ __forceinline__ int icell_kt(int k, int c, int t) const {
    if constexpr (D == 1) {
      return c;
    } else if constexpr (D == 2) {
      return k == 0 ? c + p * t : t + p * c;
    } else {
      const int a = t % p, b = t / p;
      const int c0 = k == 0 ? c : a;
      const int c1 = k == 0 ? a : (k == 1 ? c : b);
      const int c2 = k == 2 ? c : b;
      return c0 + p * (c1 + p * c2);
    }
  }
  // Stride of the cell index along direction k.
  __device__ __forceinline__ int stride(int k) const {
    return k == 0 ? 1 : k == 1 ? (p + 2) : (p + 2) * (p + 2);
  }
};

}  // namespace fv
