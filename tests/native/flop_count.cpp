// Operation count of the element arithmetic (nc_element.cuh) per element: the templates are
// instantiated on the host with a number type that counts additions and multiplications (a fused
// multiply-add counts as one of each). Device-only intrinsics are replaced by host stand-ins that
// are never counted. Prints one "name adds muls" line per element routine and form (the FP64 kernels'
// Gauss-point form, then the ScaleSums form with names ending in "_sums").
#include <cmath>
#include <cstdio>

#include <cuda_runtime.h>
inline void atomicAdd(float2*, float2) {}
inline void atomicAdd(double*, double) {}
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fmaf_rn(float a, float b, float c) { return a * b + c; }
inline float __frcp_rn(float a) { return 1.0f / a; }
inline float __double2float_rn(double d) { return (float)d; }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
#include "nc_element.cuh"

// Counting number type; SUMS selects the element code's ScaleSums form (false: the FP64 kernels'
// form, true: the FP32 and double-float kernels').
struct Tally { static long adds, muls; };
long Tally::adds = 0, Tally::muls = 0;
template <bool SUMS>
struct CntT {
  double v;
  CntT() = default;
  CntT(double x) : v(x) {}
  CntT(int x) : v(x) {}
  explicit operator double() const { return v; }
};
template <bool S> inline CntT<S> operator+(CntT<S> a, CntT<S> b) { Tally::adds++; return CntT<S>(a.v + b.v); }
template <bool S> inline CntT<S> operator-(CntT<S> a, CntT<S> b) { Tally::adds++; return CntT<S>(a.v - b.v); }
template <bool S> inline CntT<S> operator-(CntT<S> a) { return CntT<S>(-a.v); }
template <bool S> inline CntT<S> operator*(CntT<S> a, CntT<S> b) { Tally::muls++; return CntT<S>(a.v * b.v); }
template <bool S> inline CntT<S>& operator+=(CntT<S>& a, CntT<S> b) { a = a + b; return a; }
template <bool S> inline CntT<S>& operator-=(CntT<S>& a, CntT<S> b) { a = a - b; return a; }
template <bool S> inline CntT<S>& operator*=(CntT<S>& a, CntT<S> b) { a = a * b; return a; }
typedef CntT<false> Cnt;
typedef CntT<true> CntS;
namespace nc {
template <> inline Cnt nc_rsqrt<Cnt>(Cnt x) { return Cnt(1.0 / std::sqrt(x.v)); }
template <> inline CntS nc_rsqrt<CntS>(CntS x) { return CntS(1.0 / std::sqrt(x.v)); }
template <> inline Cnt nc_rcp<Cnt>(Cnt x) { return Cnt(1.0 / x.v); }
template <> inline CntS nc_rcp<CntS>(CntS x) { return CntS(1.0 / x.v); }
template <> struct ScaleSums<Cnt> { static constexpr bool value = false; };
template <> struct ScaleSums<CntS> { static constexpr bool value = true; };
}  // namespace nc

using namespace nc;

static void show(const char* name, bool sums) {
  std::printf("%s%s %ld %ld\n", name, sums ? "_sums" : "", Tally::adds, Tally::muls);
  Tally::adds = Tally::muls = 0;
}

// Every element routine in one counting form; names get "_sums" for the ScaleSums form.
template <typename T>
static void count_all() {
  const bool sums = ScaleSums<T>::value;
  ElemConst<T> C;
  C.cm = 0.21; C.ih = 16; C.w = 1e-4; C.wih = 1e-3; C.wih2 = 1e-2; C.beta = 1e4; C.betah = 1e3;
  C.rc = 1; C.rcih2 = 256; C.imu = 1; C.c4he2 = 1; C.itau3sq = 1;
  T p[8], t[8], dp[8], dt[8], oP[8], oT[8];
  for (int a = 0; a < 8; ++a) { p[a] = 0.1 * a; t[a] = 0.2 + 0.01 * a; dp[a] = 0.3 - 0.02 * a; dt[a] = 0.05 * a; }
  Tally::adds = Tally::muls = 0;
  elem_residual<T>(C, p, t, T(1e-3), T(2.0), T(1.0), oP, oT);
  show("residual", sums);
  ElemState<T> st;
  elem_state<T>(C, p, t, T(1e-3), T(1.0), st);
  show("state", sums);
  elem_jv_dir<T>(C, st, T(2.0), dp, dt, oP, oT);
  show("jv", sums);
  elem_jtv<T, false>(C, st, T(2.0), dp, dt, oP, oT, nullptr, nullptr);
  show("jtv", sums);
  T a, b;
  elem_jtv<T, true>(C, st, T(2.0), dp, dt, oP, oT, &a, &b);
  show("sens", sums);
  for (int col = 0; col < 16; ++col) elem_jac_column<T>(C, st, T(2.0), col, oP, oT);
  show("jac16", sums);
  elem_picard<T>(C, T(1e-3), T(2.0), T(0.1), T(0.2), T(0.3), T(0.01), dp, dt, oP, oT);
  show("picard", sums);
  elem_picard_t<T>(C, T(1e-3), T(2.0), T(0.1), T(0.2), T(0.3), T(0.01), dp, dt, oP, oT);
  show("picard_t", sums);
  elem_picard_modal<T, false>(C, T(1e-3), T(2.0), T(0.1), T(0.2), T(0.3), T(0.01), dp, dt, oP, oT);
  show("picard_modal", sums);
  elem_picard_modal<T, true>(C, T(1e-3), T(2.0), T(0.1), T(0.2), T(0.3), T(0.01), dp, dt, oP, oT);
  show("picard_modal_t", sums);
}

int main() {
  count_all<Cnt>();
  count_all<CntS>();
  return 0;
}
