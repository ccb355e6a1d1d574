// Check on the host of the frozen-coefficient element operator in the modal basis
// (elem_picard_modal) against its Gauss-point form (elem_picard / elem_picard_t), both instantiated
// in FP64 from nc_element.cuh: random element data (size, material, velocity, tau, buoyancy) and
// random nodal values, the operator and its transpose. Prints the largest relative difference of
// each and "ALL OK" when every case is within 1e-13 of the largest output; exits 1 otherwise.
// Device-only intrinsics get host stand-ins (unused by these routines).
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

using namespace nc;

int main() {
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0), P(0.1, 2.0);
  int bad = 0;
  double worst[2] = {0.0, 0.0};
  for (int trial = 0; trial < 200; ++trial) {
    const double h = P(rng) * 0.05;
    ElemConst<double> C;
    const double g = 1.0 / std::sqrt(3.0);
    C.cm = 0.5 * (1.0 - g);
    C.ih = 1.0 / h;
    C.w = 0.125 * h * h * h;
    C.wih = 0.125 * h * h;
    C.wih2 = 0.125 * h;
    C.beta = P(rng) * 1e3;
    C.betah = C.beta * h;
    C.rc = P(rng);
    C.rcih2 = C.rc / (h * h);
    C.imu = 1.0;
    C.c4he2 = 1.0;
    C.itau3sq = 1.0;
    const double c = P(rng) * 1e-2, kc = P(rng) * 10.0;
    const double ux = U(rng), uy = U(rng), uz = U(rng), tau = P(rng) * 0.1;
    double dp[8], dt[8];
    for (int a = 0; a < 8; ++a) { dp[a] = U(rng); dt[a] = U(rng); }
    for (int tr = 0; tr < 2; ++tr) {
      double gP[8], gT[8], mP[8], mT[8];
      if (tr) {
        elem_picard_t<double>(C, c, kc, ux, uy, uz, tau, dp, dt, gP, gT);
        elem_picard_modal<double, true>(C, c, kc, ux, uy, uz, tau, dp, dt, mP, mT);
      } else {
        elem_picard<double>(C, c, kc, ux, uy, uz, tau, dp, dt, gP, gT);
        elem_picard_modal<double, false>(C, c, kc, ux, uy, uz, tau, dp, dt, mP, mT);
      }
      double scale = 0.0, diff = 0.0;
      for (int a = 0; a < 8; ++a) {
        scale = std::fmax(scale, std::fmax(std::fabs(gP[a]), std::fabs(gT[a])));
        diff = std::fmax(diff, std::fmax(std::fabs(gP[a] - mP[a]), std::fabs(gT[a] - mT[a])));
      }
      const double rel = diff / scale;
      worst[tr] = std::fmax(worst[tr], rel);
      if (!(rel <= 1e-13)) {
        ++bad;
        if (bad < 5) std::printf("trial %d %s: relative difference %.3e\n", trial, tr ? "transpose" : "forward", rel);
      }
    }
  }
  std::printf("forward: largest relative difference %.3e\ntranspose: largest relative difference %.3e\n", worst[0],
              worst[1]);
  std::printf(bad ? "FAILED %d\n" : "ALL OK\n", bad);
  return bad ? 1 : 0;
}
