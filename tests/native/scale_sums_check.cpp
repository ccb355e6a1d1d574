// Host check of the two forms of the element routines in nc_element.cuh: the Gauss-point form (row
// factors w c / h^2 and w k / h^2 applied to the Gauss-point values; the FP64 kernels') and the
// ScaleSums form (factors applied to the 8 test sums; the FP32 and double-float kernels'). Both are
// instantiated in FP64 arithmetic, the second through a double wrapper type that selects it, on
// random elements: residual, element state, J v, J^T w with design derivatives and element-Jacobian
// columns. Prints the largest relative difference per routine and "ALL OK" when all are within
// 1e-13 of the largest output; exits 1 otherwise.
#include <cmath>
#include <cstdio>
#include <random>

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

// double arithmetic that selects the ScaleSums form
struct DS {
  double v;
  DS() = default;
  DS(double x) : v(x) {}
  DS(int x) : v(x) {}
  explicit operator double() const { return v; }
};
inline DS operator+(DS a, DS b) { return DS(a.v + b.v); }
inline DS operator-(DS a, DS b) { return DS(a.v - b.v); }
inline DS operator-(DS a) { return DS(-a.v); }
inline DS operator*(DS a, DS b) { return DS(a.v * b.v); }
inline DS& operator+=(DS& a, DS b) { a.v += b.v; return a; }
inline DS& operator-=(DS& a, DS b) { a.v -= b.v; return a; }
inline DS& operator*=(DS& a, DS b) { a.v *= b.v; return a; }
namespace nc {
template <> inline DS nc_rsqrt<DS>(DS x) { return DS(1.0 / std::sqrt(x.v)); }
template <> inline DS nc_rcp<DS>(DS x) { return DS(1.0 / x.v); }
template <> struct ScaleSums<DS> { static constexpr bool value = true; };
}  // namespace nc

using namespace nc;

template <typename T>
static ElemConst<T> consts(double h, double beta, double rc) {
  ElemConst<T> C;
  const double g = 1.0 / std::sqrt(3.0);
  C.cm = 0.5 * (1.0 - g);
  C.ih = 1.0 / h;
  C.w = 0.125 * h * h * h;
  C.wih = 0.125 * h * h;
  C.wih2 = 0.125 * h;
  C.beta = beta;
  C.betah = beta * h;
  C.rc = rc;
  C.rcih2 = rc / (h * h);
  C.imu = 1.0;
  C.c4he2 = 4.0 / (3.0 * h * h);
  C.itau3sq = 1.0;
  return C;
}

static double worst[5] = {0, 0, 0, 0, 0};
static int bad = 0;

static void compare(int which, const double* a, const DS* b, int n) {
  double scale = 0.0, diff = 0.0;
  for (int q = 0; q < n; ++q) {
    scale = std::fmax(scale, std::fabs(a[q]));
    diff = std::fmax(diff, std::fabs(a[q] - b[q].v));
  }
  const double rel = scale > 0 ? diff / scale : diff;
  worst[which] = std::fmax(worst[which], rel);
  if (!(rel <= 1e-13)) ++bad;
}

int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(-1.0, 1.0), P(0.1, 2.0);
  for (int trial = 0; trial < 100; ++trial) {
    const double h = P(rng) * 0.05, beta = P(rng) * 1e3, rc = P(rng);
    const ElemConst<double> Cd = consts<double>(h, beta, rc);
    const ElemConst<DS> Cs = consts<DS>(h, beta, rc);
    const double kap = P(rng) * 1e-2, kc = P(rng) * 10.0, Q = P(rng);
    double p[8], t[8], dp[8], dt[8];
    DS ps[8], ts[8], dps[8], dts[8];
    for (int a = 0; a < 8; ++a) {
      p[a] = 50.0 * U(rng); t[a] = U(rng); dp[a] = U(rng); dt[a] = U(rng);
      ps[a] = p[a]; ts[a] = t[a]; dps[a] = dp[a]; dts[a] = dt[a];
    }
    double oP[16], oT[8];
    DS sP[16], sT[8];
    elem_residual<double>(Cd, p, t, kap, kc, Q, oP, oT);
    elem_residual<DS>(Cs, ps, ts, DS(kap), DS(kc), DS(Q), sP, sT);
    for (int a = 0; a < 8; ++a) { oP[8 + a] = oT[a]; sP[8 + a] = sT[a]; }
    compare(0, oP, sP, 16);
    ElemState<double> st;
    ElemState<DS> ss;
    elem_state<double>(Cd, p, t, kap, Q, st);
    elem_state<DS>(Cs, ps, ts, DS(kap), DS(Q), ss);
    elem_jv_dir<double>(Cd, st, kc, dp, dt, oP, oT);
    elem_jv_dir<DS>(Cs, ss, DS(kc), dps, dts, sP, sT);
    for (int a = 0; a < 8; ++a) { oP[8 + a] = oT[a]; sP[8 + a] = sT[a]; }
    compare(1, oP, sP, 16);
    double dk1, dk2;
    DS ek1, ek2;
    elem_jtv<double, true>(Cd, st, kc, dp, dt, oP, oT, &dk1, &dk2);
    elem_jtv<DS, true>(Cs, ss, DS(kc), dps, dts, sP, sT, &ek1, &ek2);
    for (int a = 0; a < 8; ++a) { oP[8 + a] = oT[a]; sP[8 + a] = sT[a]; }
    compare(2, oP, sP, 16);
    const double dd[2] = {dk1, dk2};
    const DS de[2] = {ek1, ek2};
    compare(3, dd, de, 2);
    for (int col = 0; col < 16; ++col) {
      elem_jac_column<double>(Cd, st, kc, col, oP, oT);
      elem_jac_column<DS>(Cs, ss, DS(kc), col, sP, sT);
      for (int a = 0; a < 8; ++a) { oP[8 + a] = oT[a]; sP[8 + a] = sT[a]; }
      compare(4, oP, sP, 16);
    }
  }
  const char* names[5] = {"residual", "J v", "J^T w", "design derivatives", "Jacobian columns"};
  for (int r = 0; r < 5; ++r) std::printf("%s: largest relative difference %.3e\n", names[r], worst[r]);
  std::printf(bad ? "FAILED %d\n" : "ALL OK\n", bad);
  return bad ? 1 : 0;
}
