// Operation count of the element arithmetic (nc_element.cuh) per element: the templates are
// instantiated on the host with a number type that counts additions and multiplications (a fused
// multiply-add counts as one of each). Device-only intrinsics are replaced by host stand-ins that
// are never counted. Prints one "name adds muls" line per element routine.
#include <cmath>
#include <cstdio>

#include <cuda_runtime.h>
inline void atomicAdd(float2*, float2) {}
inline void atomicAdd(double*, double) {}
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fmaf_rn(float a, float b, float c) { return a * b + c; }
inline float __double2float_rn(double d) { return (float)d; }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
#include "nc_element.cuh"

struct Cnt {
  double v;
  static long adds, muls;
  Cnt() = default;
  Cnt(double x) : v(x) {}
  Cnt(int x) : v(x) {}
  explicit operator double() const { return v; }
};
long Cnt::adds = 0, Cnt::muls = 0;
inline Cnt operator+(Cnt a, Cnt b) { Cnt::adds++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { Cnt::adds++; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { Cnt::muls++; return Cnt(a.v * b.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
namespace nc {
template <> inline Cnt nc_rsqrt<Cnt>(Cnt x) { return Cnt(1.0 / std::sqrt(x.v)); }
}  // namespace nc

using namespace nc;

static void show(const char* name) {
  std::printf("%s %ld %ld\n", name, Cnt::adds, Cnt::muls);
  Cnt::adds = Cnt::muls = 0;
}

int main() {
  ElemConst<Cnt> C;
  C.cm = 0.21; C.ih = 16; C.w = 1e-4; C.wih = 1e-3; C.wih2 = 1e-2; C.beta = 1e4; C.betah = 1e3;
  C.rc = 1; C.rcih2 = 256; C.imu = 1; C.c4he2 = 1; C.itau3sq = 1;
  Cnt p[8], t[8], dp[8], dt[8], oP[8], oT[8];
  for (int a = 0; a < 8; ++a) { p[a] = 0.1 * a; t[a] = 0.2 + 0.01 * a; dp[a] = 0.3 - 0.02 * a; dt[a] = 0.05 * a; }
  Cnt::adds = Cnt::muls = 0;
  elem_residual<Cnt>(C, p, t, Cnt(1e-3), Cnt(2.0), Cnt(1.0), oP, oT);
  show("residual");
  ElemState<Cnt> st;
  elem_state<Cnt>(C, p, t, Cnt(1e-3), Cnt(1.0), st);
  show("state");
  elem_jv_dir<Cnt>(C, st, Cnt(2.0), dp, dt, oP, oT);
  show("jv");
  elem_jtv<Cnt, false>(C, st, Cnt(2.0), dp, dt, oP, oT, nullptr, nullptr);
  show("jtv");
  Cnt a, b;
  elem_jtv<Cnt, true>(C, st, Cnt(2.0), dp, dt, oP, oT, &a, &b);
  show("sens");
  for (int col = 0; col < 16; ++col) elem_jac_column<Cnt>(C, st, Cnt(2.0), col, oP, oT);
  show("jac16");
  elem_picard<Cnt>(C, Cnt(1e-3), Cnt(2.0), Cnt(0.1), Cnt(0.2), Cnt(0.3), Cnt(0.01), dp, dt, oP, oT);
  show("picard");
  elem_picard_t<Cnt>(C, Cnt(1e-3), Cnt(2.0), Cnt(0.1), Cnt(0.2), Cnt(0.3), Cnt(0.01), dp, dt, oP, oT);
  show("picard_t");
  return 0;
}
