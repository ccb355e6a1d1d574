// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, i.e. about 48 significant bits computed on the FP32 units (GB300 issues FP32
// at 64 times its FP64 rate). The element arithmetic of nc_element.cuh instantiates with it.
//
// Building blocks (published error-free transformations):
// * TwoSum (Knuth, TAOCP vol. 2): s + e = a + b exactly, no precondition;
// * FastTwoSum (Dekker 1971): s + e = a + b exactly when |a| >= |b| (or a = 0);
// * TwoProd with a fused multiply-add: p + e = a * b exactly.
// Operations:
// * sum: TwoSum of the high parts, low parts added into the error, renormalised by FastTwoSum
//   (Dekker's double-length addition); its error is at most about 2 u^2 (|a| + |b|), u = 2^-24,
//   the same form as an FP64 sum with 4e-15 in place of 1.1e-16;
// * product: TwoProd of the high parts plus the two cross products by FMA, renormalised
//   (the double-word product of Joldes, Muller and Popescu, ACM TOMS 2017); relative error
//   about 5 u^2; the lo * lo term (u^2 smaller) is dropped;
// * reciprocal square root: the FP32 estimate y0 refined by one Newton step
//   y = y0 + y0 (1 - x y0^2) / 2 evaluated in double-float (relative error about 1.5 e0^2, e0 the
//   estimate's error).
// Host code only constructs constants (from double); all arithmetic is device code. Compile without
// fast-math and without reassociation (the default), so the error-free transformations hold.
#pragma once

#include <cuda_runtime.h>

namespace nc {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ df64(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df64(s, e);
}

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  const float e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  return df64(s, e);
}

__device__ __forceinline__ df64 operator+(const df64 a, const df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df64 operator-(const df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(const df64 a, const df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(const df64 a, const df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64& operator+=(df64& a, const df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64& operator-=(df64& a, const df64 b) { a = a - b; return a; }
__device__ __forceinline__ df64& operator*=(df64& a, const df64 b) { a = a * b; return a; }

__device__ __forceinline__ df64 df_rsqrt(const df64 x) {
  const df64 y0(rsqrtf(x.hi), 0.0f);
  const df64 r = x * (y0 * y0);                 // 1 + O(e0)
  const df64 d = df64(1.0f, 0.0f) - r;          // formed accurately: r is close to 1
  return y0 + (y0 * d) * df64(0.5f, 0.0f);
}

// Reciprocal: one Newton step y0 + y0 (1 - x y0) from the FP32 reciprocal of the leading part.
__device__ __forceinline__ df64 df_rcp(const df64 x) {
  const df64 y0(__frcp_rn(x.hi), 0.0f);
  const df64 d = df64(1.0f, 0.0f) - x * y0;     // formed accurately: x y0 is close to 1
  return y0 + y0 * d;
}

// Split of FP64 values into double-float (used by the kernels that convert their inputs once).
__device__ __forceinline__ df64 df_from_double(double d) {
  const float h = __double2float_rn(d);
  return df64(h, __double2float_rn(d - (double)h));
}

}  // namespace nc
