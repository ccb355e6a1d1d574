// Element-level arithmetic of the stabilised Darcy-Boussinesq weak form (App. A of the paper),
// written once, templated on the arithmetic type (double, float or double-float df64).
//
// Weak form (Eq. weakstable), per element with permeability kappa, conductivity k, source Q:
//   R^P_a = sum_q w ( -grad N_a . u_q )                                 (continuity rows)
//   R^T_a = sum_q w ( N*_a,q (rho0 c_p u_q . grad T_q - Q) + k grad N_a . grad T_q )
// with the Darcy velocity u = -kappa/mu (grad P + rho0 alpha g T), g = (0, 0, -g) (Eq. finaldarcy),
// the SUPG test function N* = N + tau u0 . grad N (App. A), u0 the centroid velocity (the mean of
// the Gauss-point velocities for a trilinear field), and
//   tau = (4 |u0|^2 / h_e^2 + 1 / tau3^2)^(-1/2),  h_e = sqrt(3) h,
// the Tezduyar combination of tau1 = h_e / (2 |u0|) and tau3 (App. A; tau3 = rho0 c_p h_e^2 /(4 k_f),
// which is the printed h_e^2/4 for unit properties).
// Quadrature: 2x2x2 Gauss-Legendre. Values and gradients at the 8 Gauss points are obtained by
// sum factorisation (three 1D stages of 2x2 interpolation / differencing), and the test-function
// side (sum over points of N_a A_q + grad N_a . B_q) by the transposed stages.
//
// Units: gradients are carried in element units, i.e. multiplied by h (a 1D stage yields the nodal
// difference f1 - f0 = h df/dx); every factor 1/h is folded into per-element constants, and the
// test-function stage takes its gradient weights pre-multiplied by 1/h. A 1D stage evaluates the
// Gauss-point values cp f0 + cm f1 and cm f0 + cp f1 (cp = 1 - cm) as f0 + cm d and f1 - cm d with
// d = f1 - f0: one subtraction and two fused multiply-adds per node pair.
//
// Index conventions: local node a = ax + 2 ay + 4 az; Gauss point q = qx + 2 qy + 4 qz with
// reference coordinate (2 q_d - 1)/sqrt(3) along each axis.
#pragma once

#include "nc_common.cuh"
#include "nc_df64.cuh"

namespace nc {

template <typename R>
struct ElemConst {
  R cm;         // 1D interpolation weight (1 - 1/sqrt3)/2 of the far node at a Gauss point
  R ih;         // 1 / h
  R w;          // Gauss weight x det J = (h/2)^3
  R wih;        // w / h
  R wih2;       // w / h^2
  R beta;       // rho0 alpha g
  R betah;      // rho0 alpha g h
  R rc;         // rho0 c_p
  R rcih2;      // rho0 c_p / h^2
  R imu;        // 1 / mu
  R c4he2;      // 4 / h_e^2
  R itau3sq;    // 1 / tau3^2
};

// One 1D stage on a node pair: the values at the two Gauss points and the difference f1 - f0.
template <typename R>
__device__ __forceinline__ void q1_pair(const R f0, const R f1, const R cm, R& v0, R& v1, R& d) {
  d = f1 - f0;
  v0 = f0 + cm * d;
  v1 = f1 - cm * d;
}

// Values and element-unit gradients (h grad f) of the trilinear interpolant of nodal values f at the
// 8 Gauss points.
template <typename R>
__device__ __forceinline__ void q1_forward(const R f[8], const R cm, R v[8], R gx[8], R gy[8], R gz[8]) {
  R A[8], Dx[4];
#pragma unroll
  for (int yz = 0; yz < 4; ++yz)            // yz = ay + 2 az; A index qx + 2 ay + 4 az
    q1_pair(f[2 * yz], f[2 * yz + 1], cm, A[2 * yz], A[2 * yz + 1], Dx[yz]);
  R B[8], Dy[4], Cx[4], dd;
#pragma unroll
  for (int qx = 0; qx < 2; ++qx)
#pragma unroll
    for (int az = 0; az < 2; ++az)          // B index qx + 2 qy + 4 az, Dy index qx + 2 az
      q1_pair(A[qx + 4 * az], A[qx + 2 + 4 * az], cm, B[qx + 4 * az], B[qx + 2 + 4 * az], Dy[qx + 2 * az]);
#pragma unroll
  for (int az = 0; az < 2; ++az)            // Cx index qy + 2 az
    q1_pair(Dx[2 * az], Dx[1 + 2 * az], cm, Cx[2 * az], Cx[1 + 2 * az], dd);
  R Gz[4], Gy[4], Gx[4];
#pragma unroll
  for (int xy = 0; xy < 4; ++xy)            // xy = qx + 2 qy; Gz index qx + 2 qy
    q1_pair(B[xy], B[xy + 4], cm, v[xy], v[xy + 4], Gz[xy]);
#pragma unroll
  for (int qx = 0; qx < 2; ++qx)            // Gy index qx + 2 qz
    q1_pair(Dy[qx], Dy[qx + 2], cm, Gy[qx], Gy[qx + 2], dd);
#pragma unroll
  for (int qy = 0; qy < 2; ++qy)            // Gx index qy + 2 qz
    q1_pair(Cx[qy], Cx[qy + 2], cm, Gx[qy], Gx[qy + 2], dd);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
    gx[q] = Gx[qy + 2 * qz];
    gy[q] = Gy[qx + 2 * qz];
    gz[q] = Gz[qx + 2 * qy];
  }
}

// Transposed 1D stage: (a0, a1) at the Gauss points -> the two nodes, minus / plus d (the summed
// gradient weight of the pair): o0 = cp a0 + cm a1 - d = a0 + cm s - d, o1 = a1 - cm s + d, s = a1 - a0.
template <typename R>
__device__ __forceinline__ void q1_pair_t(const R a0, const R a1, const R d, const R cm, R& o0, R& o1) {
  const R s = a1 - a0;
  o0 = (a0 - d) + cm * s;
  o1 = (a1 + d) - cm * s;
}

// out_a = sum_q ( N_a(q) A_q + h dN_a/dx(q) Bx_q + h dN_a/dy(q) By_q + h dN_a/dz(q) Bz_q ), i.e. the
// test-function sums sum_q ( N_a A_q + grad N_a . B_q ) for gradient weights given as B / h.
// HAS_A = false treats A as zero.
template <typename R, bool HAS_A>
__device__ __forceinline__ void q1_test(const R* A, const R Bx[8], const R By[8], const R Bz[8],
                                        const R cm, R out[8]) {
  R bx[4], by[4], bz[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int lo = i & 1, hi = i >> 1;
    bx[i] = Bx[2 * lo + 4 * hi] + Bx[1 + 2 * lo + 4 * hi];   // bx index qy + 2 qz
    by[i] = By[lo + 4 * hi] + By[lo + 2 + 4 * hi];           // by index qx + 2 qz
    bz[i] = Bz[lo + 2 * hi] + Bz[lo + 2 * hi + 4];           // bz index qx + 2 qy
  }
  R Az[8];                                                    // index qx + 2 qy + 4 az
#pragma unroll
  for (int xy = 0; xy < 4; ++xy) {
    if (HAS_A) q1_pair_t(A[xy], A[xy + 4], bz[xy], cm, Az[xy], Az[xy + 4]);
    else { Az[xy] = -bz[xy]; Az[xy + 4] = bz[xy]; }
  }
  R byz[4], bxz[4], dd;                                       // index qx + 2 az, qy + 2 az
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    q1_pair(by[l], by[l + 2], cm, byz[l], byz[l + 2], dd);
    q1_pair(bx[l], bx[l + 2], cm, bxz[l], bxz[l + 2], dd);
  }
  R Ay[8];                                                    // index qx + 2 ay + 4 az
#pragma unroll
  for (int qx = 0; qx < 2; ++qx)
#pragma unroll
    for (int az = 0; az < 2; ++az)
      q1_pair_t(Az[qx + 4 * az], Az[qx + 2 + 4 * az], byz[qx + 2 * az], cm, Ay[qx + 4 * az], Ay[qx + 2 + 4 * az]);
  R bxy[4];                                                   // index ay + 2 az
#pragma unroll
  for (int az = 0; az < 2; ++az) q1_pair(bxz[2 * az], bxz[1 + 2 * az], cm, bxy[2 * az], bxy[1 + 2 * az], dd);
#pragma unroll
  for (int yz = 0; yz < 4; ++yz) q1_pair_t(Ay[2 * yz], Ay[2 * yz + 1], bxy[yz], cm, out[2 * yz], out[2 * yz + 1]);
}

template <typename R> __device__ __forceinline__ R nc_rsqrt(R x);
template <> __device__ __forceinline__ double nc_rsqrt<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float nc_rsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ df64 nc_rsqrt<df64>(df64 x) { return df_rsqrt(x); }
// Reciprocal of a positive element factor (|x| within FP32's normal range). FP64: Newton's iteration
// for 1/x, y <- y + y (1 - x y), twice from the FP32 reciprocal (each step squares the relative
// error: 2^-24 -> 2^-48 -> below FP64 rounding), four FMAs and no branch.
template <typename R> __device__ __forceinline__ R nc_rcp(R x);
template <> __device__ __forceinline__ double nc_rcp<double>(double x) {
  double y = (double)__frcp_rn((float)x);
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}
template <> __device__ __forceinline__ float nc_rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ df64 nc_rcp<df64>(df64 x) { return df_rcp(x); }

// Whether the element routines apply the rows' constant factors (w c / h^2 of the continuity rows,
// w k / h^2 of the energy rows) to the 8 test sums instead of the 24 Gauss-point values (the test
// sums are linear): fewer multiplications for one reciprocal of w k / h^2 per element. Measured on
// GB300 (128^3 whole path): faster FP32 operators and double-float adjoint residual; the FP64 kernels,
// bound by the FP64 pipe, were not faster (the accepting adjoint product 3 % slower), so FP64 keeps
// the factors at the Gauss points.
template <typename R> struct ScaleSums { static constexpr bool value = true; };
template <> struct ScaleSums<double> { static constexpr bool value = false; };

// Gauss-point state of an element: V_q = h (grad P_q - beta T_q e_z) (so u_q = -(c/h) V_q, c = kappa/mu),
// H_q = h grad T_q, S_q = rho0 c_p u_q . grad T_q - Q, centroid velocity u0 and tau (u0, S, tau in
// physical units).
template <typename R>
struct ElemState {
  R vx[8], vy[8], vz[8];
  R hx[8], hy[8], hz[8];
  R S[8];
  R u0x, u0y, u0z, tau, c;
};

template <typename R>
__device__ __forceinline__ void elem_state(const ElemConst<R>& C, const R p[8], const R t[8],
                                           const R kappa, const R Q, ElemState<R>& st) {
  R T[8];
  q1_forward(p, C.cm, T, st.vx, st.vy, st.vz);   // T reused as scratch for P values
  q1_forward(t, C.cm, T, st.hx, st.hy, st.hz);
  st.c = kappa * C.imu;
  R sx = 0, sy = 0, sz = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    st.vz[q] -= C.betah * T[q];
    sx += st.vx[q]; sy += st.vy[q]; sz += st.vz[q];
  }
  const R m = -st.c * C.ih * R(0.125);
  st.u0x = m * sx; st.u0y = m * sy; st.u0z = m * sz;
  st.tau = nc_rsqrt<R>(C.c4he2 * (st.u0x * st.u0x + st.u0y * st.u0y + st.u0z * st.u0z) + C.itau3sq);
  const R mrc = -st.c * C.rcih2;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    st.S[q] = mrc * (st.vx[q] * st.hx[q] + st.vy[q] * st.hy[q] + st.vz[q] * st.hz[q]) - Q;
}

// Element residual (R^P, R^T) of Eq. weakstable / Eq. finalsyseq.
template <typename R>
__device__ __forceinline__ void elem_residual(const ElemConst<R>& C, const R p[8], const R t[8],
                                              const R kappa, const R kc, const R Q,
                                              R RP[8], R RT[8]) {
  ElemState<R> st;
  elem_state(C, p, t, kappa, Q, st);
  const R wc = C.wih2 * st.c;    // B^P / h = -w u / h = (w c / h^2) V
  R A[8], bx[8], by[8], bz[8];
  const R wk = C.wih2 * kc;
  if constexpr (ScaleSums<R>::value) {
    q1_test<R, false>(nullptr, st.vx, st.vy, st.vz, C.cm, RP);
#pragma unroll
    for (int a = 0; a < 8; ++a) RP[a] *= wc;
    // energy rows: A_q = w S_q, B_q / h = (w tau / h) S_q u0 + (w k / h^2) H_q = wk (s_q u0 + H_q)
    const R iwk = nc_rcp<R>(wk);
    const R wt = C.wih * st.tau * iwk, wa = C.w * iwk;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      A[q] = wa * st.S[q];
      const R s = wt * st.S[q];
      bx[q] = s * st.u0x + st.hx[q];
      by[q] = s * st.u0y + st.hy[q];
      bz[q] = s * st.u0z + st.hz[q];
    }
    q1_test<R, true>(A, bx, by, bz, C.cm, RT);
#pragma unroll
    for (int a = 0; a < 8; ++a) RT[a] *= wk;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) { bx[q] = wc * st.vx[q]; by[q] = wc * st.vy[q]; bz[q] = wc * st.vz[q]; }
    q1_test<R, false>(nullptr, bx, by, bz, C.cm, RP);
    const R wt = C.wih * st.tau;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      A[q] = C.w * st.S[q];
      const R s = wt * st.S[q];
      bx[q] = s * st.u0x + wk * st.hx[q];
      by[q] = s * st.u0y + wk * st.hy[q];
      bz[q] = s * st.u0z + wk * st.hz[q];
    }
    q1_test<R, true>(A, bx, by, bz, C.cm, RT);
  }
}

// Exact Newton Jacobian product at the element state st for a direction given at the Gauss points
// (element units): dV_q = h (grad dP_q - beta dT_q e_z) and dH_q = h grad dT_q (includes d tau and
// d N*).
template <typename R>
__device__ __forceinline__ void elem_jv_gauss(const ElemConst<R>& C, const ElemState<R>& st, const R kc,
                                              const R dvx[8], const R dvy[8], const R dvz[8],
                                              const R dhx[8], const R dhy[8], const R dhz[8],
                                              R oP[8], R oT[8]) {
  R sx = 0, sy = 0, sz = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) { sx += dvx[q]; sy += dvy[q]; sz += dvz[q]; }
  const R m = -st.c * C.ih * R(0.125);
  const R du0x = m * sx, du0y = m * sy, du0z = m * sz;
  const R tau = st.tau;
  const R dtau = -tau * tau * tau * C.c4he2 * (st.u0x * du0x + st.u0y * du0y + st.u0z * du0z);
  const R mrc = -st.c * C.rcih2;
  const R wc = C.wih2 * st.c;
  const R wk = C.wih2 * kc;
  constexpr bool kSums = ScaleSums<R>::value;
  // with kSums the energy rows' factor w k / h^2 is applied to the 8 test sums: the Gauss-point
  // coefficients are divided by it and the dT gradient enters unscaled
  const R iwk = kSums ? nc_rcp<R>(wk) : R(1);
  const R wt = kSums ? C.wih * tau * iwk : C.wih * tau;
  const R wdt = kSums ? C.wih * dtau * iwk : C.wih * dtau;
  const R wa = kSums ? C.w * iwk : C.w;
  R A[8], bx[8], by[8], bz[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    // dS = rho0 c_p (du . grad T + u . grad dT), u = -(c/h) V
    const R dS = mrc * (dvx[q] * st.hx[q] + dvy[q] * st.hy[q] + dvz[q] * st.hz[q]
                      + st.vx[q] * dhx[q] + st.vy[q] * dhy[q] + st.vz[q] * dhz[q]);
    A[q] = wa * dS;
    const R a = wt * dS + wdt * st.S[q];      // coefficient of u0 (divided by h)
    const R b = wt * st.S[q];                 // coefficient of du0 (divided by h)
    if constexpr (kSums) {
      bx[q] = a * st.u0x + b * du0x + dhx[q];
      by[q] = a * st.u0y + b * du0y + dhy[q];
      bz[q] = a * st.u0z + b * du0z + dhz[q];
    } else {
      bx[q] = a * st.u0x + b * du0x + wk * dhx[q];
      by[q] = a * st.u0y + b * du0y + wk * dhy[q];
      bz[q] = a * st.u0z + b * du0z + wk * dhz[q];
    }
  }
  q1_test<R, true>(A, bx, by, bz, C.cm, oT);
  if constexpr (kSums) {
#pragma unroll
    for (int a = 0; a < 8; ++a) oT[a] *= wk;
    q1_test<R, false>(nullptr, dvx, dvy, dvz, C.cm, oP);
#pragma unroll
    for (int a = 0; a < 8; ++a) oP[a] *= wc;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) { bx[q] = wc * dvx[q]; by[q] = wc * dvy[q]; bz[q] = wc * dvz[q]; }
    q1_test<R, false>(nullptr, bx, by, bz, C.cm, oP);
  }
}

// Exact Newton Jacobian product J_e (dp, dt) at the element state st.
template <typename R>
__device__ __forceinline__ void elem_jv_dir(const ElemConst<R>& C, const ElemState<R>& st,
                                            const R kc, const R dp[8], const R dt[8],
                                            R oP[8], R oT[8]) {
  R dvx[8], dvy[8], dvz[8], dT[8];
  q1_forward(dp, C.cm, dT, dvx, dvy, dvz);
  R dhx[8], dhy[8], dhz[8];
  q1_forward(dt, C.cm, dT, dhx, dhy, dhz);
#pragma unroll
  for (int q = 0; q < 8; ++q) dvz[q] -= C.betah * dT[q];
  elem_jv_gauss(C, st, kc, dvx, dvy, dvz, dhx, dhy, dhz, oP, oT);
}

// Column b of the element Jacobian (b < 8: P at local node b, else T at node b - 8): the
// Gauss-point values of the unit direction are products of the 1D shape-function tables (the
// 1D shape function is cp = 1 - cm at the near Gauss point and cm at the far one; its element-unit
// derivative is -1 or +1).
template <typename R>
__device__ __forceinline__ void elem_jac_column(const ElemConst<R>& C, const ElemState<R>& st, const R kc,
                                                int b, R oP[8], R oT[8]) {
  const int a = b & 7;
  const bool isT = b >= 8;
  const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
  const R cp = R(1) - C.cm;
  const R gxd = ax ? R(1) : R(-1), gyd = ay ? R(1) : R(-1), gzd = az ? R(1) : R(-1);
  R dvx[8], dvy[8], dvz[8], dhx[8], dhy[8], dhz[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
    const R nx = (qx == ax) ? cp : C.cm, ny = (qy == ay) ? cp : C.cm, nz = (qz == az) ? cp : C.cm;
    const R gx = gxd * ny * nz, gy = nx * gyd * nz, gz = nx * ny * gzd;
    if (isT) {
      dvx[q] = R(0); dvy[q] = R(0); dvz[q] = -C.betah * nx * ny * nz;
      dhx[q] = gx; dhy[q] = gy; dhz[q] = gz;
    } else {
      dvx[q] = gx; dvy[q] = gy; dvz[q] = gz;
      dhx[q] = R(0); dhy[q] = R(0); dhz[q] = R(0);
    }
  }
  elem_jv_gauss(C, st, kc, dvx, dvy, dvz, dhx, dhy, dhz, oP, oT);
}

// Adjoint side: given multipliers (lp, lt) of the element rows, the gradient of
// L = lp . R^P + lt . R^T with respect to the element state (J_e^T l), and optionally the
// derivatives dL/dkappa and dL/dk used by the design sensitivities. Gradients of lp, lt at the
// Gauss points are in element units (h grad); G below is h dL/du_q.
template <typename R, bool SENS>
__device__ __forceinline__ void elem_jtv(const ElemConst<R>& C, const ElemState<R>& st,
                                         const R kc, const R lp[8], const R lt[8],
                                         R oP[8], R oT[8], R* dL_dkappa, R* dL_dk) {
  R Mx[8], My[8], Mz[8], m[8];
  q1_forward(lp, C.cm, m, Mx, My, Mz);
  R Nx[8], Ny[8], Nz[8];
  q1_forward(lt, C.cm, m, Nx, Ny, Nz);
  const R c = st.c;
  // with ScaleSums the energy rows' factor w k / h^2 and the continuity rows' -c / h^2 are applied to
  // the 8 test sums (linear) instead of the Gauss-point values
  constexpr bool kSums = ScaleSums<R>::value;
  const R wk2 = C.wih2 * kc;
  const R iwk2 = kSums ? nc_rcp<R>(wk2) : R(1);
  const R tih = st.tau * C.ih;
  const R cih2 = c * C.ih * C.ih;
  const R acih = kSums ? -cih2 * iwk2 : -cih2;
  R gx[8], gy[8], gz[8];         // h dL/du_q (without the centroid part)
  R g0x = 0, g0y = 0, g0z = 0, sdot = 0, kdot = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const R u0M = st.u0x * Nx[q] + st.u0y * Ny[q] + st.u0z * Nz[q];   // h u0 . grad lt
    const R W = m[q] + tih * u0M;                                      // sum_a lt_a N*_a(q)
    const R wWrc = C.w * W * C.rc;
    gx[q] = -C.w * Mx[q] + wWrc * st.hx[q];
    gy[q] = -C.w * My[q] + wWrc * st.hy[q];
    gz[q] = -C.w * Mz[q] + wWrc * st.hz[q];
    const R wS = C.w * st.S[q];
    g0x += wS * Nx[q]; g0y += wS * Ny[q]; g0z += wS * Nz[q];
    sdot += wS * u0M;
    if (SENS) kdot += Nx[q] * st.hx[q] + Ny[q] * st.hy[q] + Nz[q] * st.hz[q];
    // dL/dgrad T_q / h = (w W rho0 c_p u_q + w k grad lt_q) / h, u_q = -(c/h) V_q; stored in N
    // (with ScaleSums divided by w k / h^2)
    const R a = wWrc * acih;
    if constexpr (kSums) {
      Nx[q] = a * st.vx[q] + Nx[q];
      Ny[q] = a * st.vy[q] + Ny[q];
      Nz[q] = a * st.vz[q] + Nz[q];
    } else {
      Nx[q] = a * st.vx[q] + wk2 * Nx[q];
      Ny[q] = a * st.vy[q] + wk2 * Ny[q];
      Nz[q] = a * st.vz[q] + wk2 * Nz[q];
    }
  }
  const R t3 = -st.tau * st.tau * st.tau * C.c4he2 * sdot;
  g0x = R(0.125) * (st.tau * g0x + t3 * st.u0x);
  g0y = R(0.125) * (st.tau * g0y + t3 * st.u0y);
  g0z = R(0.125) * (st.tau * g0z + t3 * st.u0z);
  R kap = 0;
  const R cbih = kSums ? c * C.beta * C.ih * iwk2 : c * C.beta * C.ih;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    gx[q] += g0x; gy[q] += g0y; gz[q] += g0z;
    if (SENS) kap += gx[q] * st.vx[q] + gy[q] * st.vy[q] + gz[q] * st.vz[q];
    m[q] = cbih * gz[q];   // dL/dT_q (with ScaleSums divided by w k / h^2)
  }
  if (SENS) { *dL_dkappa = -C.imu * C.ih * C.ih * kap; *dL_dk = C.wih2 * kdot; }
  q1_test<R, true>(m, Nx, Ny, Nz, C.cm, oT);
  if constexpr (kSums) {
#pragma unroll
    for (int a = 0; a < 8; ++a) oT[a] *= wk2;
    q1_test<R, false>(nullptr, gx, gy, gz, C.cm, oP);
    const R mcih2 = -cih2;
#pragma unroll
    for (int a = 0; a < 8; ++a) oP[a] *= mcih2;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) { gx[q] *= -cih2; gy[q] *= -cih2; gz[q] *= -cih2; }
    q1_test<R, false>(nullptr, gx, gy, gz, C.cm, oP);
  }
}

// Frozen-coefficient (Picard) element operator, a cheaper stand-in for J_e on the multigrid's finest
// level (the outer Krylov solver is flexible, so its preconditioner may use another operator): the
// continuity rows exactly as J_e (they are linear in the state); the energy rows
//   sum_q w [ N*_a(q) rho0 c_p u0 . grad dT_q + k grad N_a . grad dT_q ],  N* = N + tau u0 . grad N,
// with the centroid velocity u0 and tau of the linearisation state frozen: no derivatives of u, u0 or
// tau and no coupling of dP into the energy rows. c = kappa / mu, kc = k.
template <typename R>
__device__ __forceinline__ void elem_picard(const ElemConst<R>& C, const R c, const R kc, const R u0x, const R u0y,
                                            const R u0z, const R tau, const R dp[8], const R dt[8],
                                            R oP[8], R oT[8]) {
  R vx[8], vy[8], vz[8], dT[8];
  q1_forward(dp, C.cm, dT, vx, vy, vz);    // dT: scratch for the (unused) P values
  R hx[8], hy[8], hz[8];
  q1_forward(dt, C.cm, dT, hx, hy, hz);
  // the factors w c / h^2 (continuity rows) and w k / h^2 (energy rows) are applied to the 8 test
  // sums (linear) instead of the Gauss-point values
  R bz[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) bz[q] = vz[q] - C.betah * dT[q];
  q1_test<R, false>(nullptr, vx, vy, bz, C.cm, oP);
  const R wc = C.wih2 * c;
#pragma unroll
  for (int a = 0; a < 8; ++a) oP[a] *= wc;
  const R wk = C.wih2 * kc;
  const R iwk = nc_rcp<R>(wk);
  const R a = C.wih * C.rc * iwk;  // A_q = w rho0 c_p u0 . grad dT_q = (w rho0 c_p / h) u0 . H_q, / wk
  const R th = tau * C.ih;         // B_q / h = (tau / h) A_q u0 + (w k / h^2) H_q, / wk
  R A[8], bx[8], by[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    A[q] = a * (u0x * hx[q] + u0y * hy[q] + u0z * hz[q]);
    const R sq = th * A[q];
    bx[q] = sq * u0x + hx[q];
    by[q] = sq * u0y + hy[q];
    bz[q] = sq * u0z + hz[q];
  }
  q1_test<R, true>(A, bx, by, bz, C.cm, oT);
#pragma unroll
  for (int a2 = 0; a2 < 8; ++a2) oT[a2] *= wk;
}

// Transpose of elem_picard: the gradient of L = lp . A^P(d) + lt . A^T(d) with respect to d = (dP, dT).
template <typename R>
__device__ __forceinline__ void elem_picard_t(const ElemConst<R>& C, const R c, const R kc, const R u0x, const R u0y,
                                              const R u0z, const R tau, const R lp[8], const R lt[8],
                                              R oP[8], R oT[8]) {
  R Mx[8], My[8], Mz[8], lv[8];
  q1_forward(lp, C.cm, lv, Mx, My, Mz);    // lv: scratch for the (unused) lp values
  R Nx[8], Ny[8], Nz[8];
  q1_forward(lt, C.cm, lv, Nx, Ny, Nz);
  // the factors w c / h^2 and w k / h^2 are applied to the 8 test sums instead of the Gauss-point values
  q1_test<R, false>(nullptr, Mx, My, Mz, C.cm, oP);
  const R wc = C.wih2 * c;
#pragma unroll
  for (int a = 0; a < 8; ++a) oP[a] *= wc;
  const R wk = C.wih2 * kc;
  const R iwk = nc_rcp<R>(wk);
  const R ab = -C.wih * c * C.beta * iwk;   // continuity rows into dT: A_q = -(w c beta / h) h dlp/dz, / wk
  const R a = C.wih * C.rc * iwk;           // energy rows: B_q / h = (w rho0 c_p / h) lt*_q u0 + (w k / h^2) h grad lt, / wk
  const R th = tau * C.ih;                  // lt*_q = lt_q + tau u0 . grad lt_q
  R bx[8], by[8], bz[8], A[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    A[q] = ab * Mz[q];
    const R sq = a * (lv[q] + th * (u0x * Nx[q] + u0y * Ny[q] + u0z * Nz[q]));
    bx[q] = sq * u0x + Nx[q];
    by[q] = sq * u0y + Ny[q];
    bz[q] = sq * u0z + Nz[q];
  }
  q1_test<R, true>(A, bx, by, bz, C.cm, oT);
#pragma unroll
  for (int a2 = 0; a2 < 8; ++a2) oT[a2] *= wk;
}

// ---- the frozen-coefficient operator in the modal basis of the element ---------------------------
// Every term of the frozen-coefficient operator is, per element, a constant coefficient times an
// integral of products of Q1 shape functions and their derivatives, and the 2x2x2 Gauss rule
// integrates these exactly. In the basis {1, 2s - 1} of each axis (s in [0, 1] the element
// coordinate) the 1D integrals are diagonal or have one entry: mass diag(1, 1/3), stiffness
// diag(0, 4), phi_m phi_n' nonzero only at (0, 1) (= 2) and phi_m' phi_n only at (1, 0) (= 2). So the
// element Laplacian and the streamline-diffusion diagonal act mode by mode, and the convection,
// buoyancy and cross streamline terms couple a mode with one other. The operator is then applied as:
// nodal values -> modal coefficients (three butterfly stages), the sparse modal operator, modal test
// sums -> nodal rows (the transposed butterflies); the same values as the Gauss-point form up to
// rounding, with about a third of its arithmetic.

// Per axis (f0, f1) -> (f0 + f1, f1 - f0): 8 x the coefficients of f in the basis {1, 2s - 1}^3.
// Mode index m = mx + 2 my + 4 mz, bit d set for the factor 2 s_d - 1.
template <typename R>
__device__ __forceinline__ void q1_to_modal(const R f[8], R F[8]) {
  R a[8], b[8];
#pragma unroll
  for (int yz = 0; yz < 4; ++yz) { a[2 * yz] = f[2 * yz] + f[2 * yz + 1]; a[2 * yz + 1] = f[2 * yz + 1] - f[2 * yz]; }
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      b[x + 4 * z] = a[x + 4 * z] + a[x + 2 + 4 * z];
      b[x + 2 + 4 * z] = a[x + 2 + 4 * z] - a[x + 4 * z];
    }
#pragma unroll
  for (int xy = 0; xy < 4; ++xy) { F[xy] = b[xy] + b[xy + 4]; F[xy + 4] = b[xy + 4] - b[xy]; }
}

// Transpose of q1_to_modal: modal test sums Y -> nodal rows, per axis (Y0, Y1) -> (Y0 - Y1, Y0 + Y1).
template <typename R>
__device__ __forceinline__ void q1_from_modal(const R Y[8], R y[8]) {
  R a[8], b[8];
#pragma unroll
  for (int xy = 0; xy < 4; ++xy) { b[xy] = Y[xy] - Y[xy + 4]; b[xy + 4] = Y[xy] + Y[xy + 4]; }
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      a[x + 4 * z] = b[x + 4 * z] - b[x + 2 + 4 * z];
      a[x + 2 + 4 * z] = b[x + 4 * z] + b[x + 2 + 4 * z];
    }
#pragma unroll
  for (int yz = 0; yz < 4; ++yz) { y[2 * yz] = a[2 * yz] - a[2 * yz + 1]; y[2 * yz + 1] = a[2 * yz] + a[2 * yz + 1]; }
}

// 1D modal mass of mode bit b: 1 or 1/3; the 3D mass of the axes other than d (and e) of mode m.
__host__ __device__ constexpr double q1m_mu(int b) { return b ? 1.0 / 3.0 : 1.0; }
__host__ __device__ constexpr double q1m_mass_but(int m, int d) {
  return (d == 0 ? 1.0 : q1m_mu(m & 1)) * (d == 1 ? 1.0 : q1m_mu((m >> 1) & 1)) * (d == 2 ? 1.0 : q1m_mu((m >> 2) & 1));
}
// Stiffness along axis d of mode m (diagonal): 4 x the mass of the other axes if bit d is set.
__host__ __device__ constexpr double q1m_stiff(int m, int d) { return ((m >> d) & 1) ? 4.0 * q1m_mass_but(m, d) : 0.0; }
__host__ __device__ constexpr double q1m_lambda(int m) { return q1m_stiff(m, 0) + q1m_stiff(m, 1) + q1m_stiff(m, 2); }
// k x, without the multiplication when the compile-time weight k is 1.
template <typename R> __device__ __forceinline__ R q1m_scale(double k, R x) { return k == 1.0 ? x : R(k) * x; }
// Mass of the third axis f (f != d, e) of mode m.
__host__ __device__ constexpr double q1m_mass_third(int m, int d, int e) {
  return q1m_mu((m >> (3 - d - e)) & 1);
}

// The frozen-coefficient element operator (TR: its transpose) in the modal basis: the same inputs,
// outputs and values (up to rounding) as elem_picard / elem_picard_t. The element integrals over
// s in [0, 1]^3 are, with the 1/64 of the two unnormalised transforms folded into the coefficients
// (h = 8 w/h^2, h^2 = 8 w/h):
//   continuity rows  c h (grad phi_m . grad phi_n) P_n  -  c beta h^2 (d phi_m / dz) phi_n T_n
//   energy rows      k h (grad phi_m . grad phi_n) T_n  +  rho0 c_p h^2 phi_m (u0 . grad phi_n) T_n
//                    + tau rho0 c_p h (u0 . grad phi_m)(u0 . grad phi_n) T_n
template <typename R, bool TR>
__device__ __forceinline__ void elem_picard_modal(const ElemConst<R>& C, const R c, const R kc, const R u0x,
                                                  const R u0y, const R u0z, const R tau, const R dp[8],
                                                  const R dt[8], R oP[8], R oT[8]) {
  R FP[8], FT[8];
  q1_to_modal(dp, FP);
  q1_to_modal(dt, FT);
  const R q = R(0.125);
  const R cP = q * C.wih2 * c;                    // c h / 64
  const R cB = R(-0.25) * C.wih * C.beta * c;     // -c beta h^2 / 64 x 2 (the 1D integral of phi_1' phi_0)
  const R cT = q * C.wih2 * kc;                   // k h / 64
  const R cC = R(0.25) * C.wih * C.rc;            // rho0 c_p h^2 / 64 x 2 (the 1D integral of phi_0 phi_1')
  const R cS = q * C.wih2 * C.rc * tau;           // tau rho0 c_p h / 64
  const R u[3] = {u0x, u0y, u0z};
  R uc[3], uu[3];
  const R cS4 = R(4) * cS;
#pragma unroll
  for (int d = 0; d < 3; ++d) { uc[d] = cC * u[d]; uu[d] = cS4 * u[d] * u[d]; }
  R ux[3][3];                                     // 4 tau rho0 c_p h / 64 u_d u_e (d != e)
  ux[0][1] = ux[1][0] = cS4 * u[0] * u[1];
  ux[0][2] = ux[2][0] = cS4 * u[0] * u[2];
  ux[1][2] = ux[2][1] = cS4 * u[1] * u[2];
  // the Laplacian's eigenvalues 4 (one bit), 8/3 (two), 4/3 (three) times c h / 64 and k h / 64
  const R lP[3] = {R(4) * cP, R(8.0 / 3.0) * cP, R(4.0 / 3.0) * cP};
  const R lT[3] = {R(4) * cT, R(8.0 / 3.0) * cT, R(4.0 / 3.0) * cT};
  R YP[8], YT[8];
  YP[0] = R(0);                                   // the constant mode: no gradient
  YT[0] = R(0);
#pragma unroll
  for (int m = 1; m < 8; ++m) {
    // mode-diagonal parts: Laplacians, streamline diffusion along each axis with bit set
    const int nb = (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1);
    YP[m] = lP[nb - 1] * FP[m];
    R dT = lT[nb - 1];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if ((m >> d) & 1) dT += q1m_scale(q1m_mass_but(m, d), uu[d]);
    YT[m] = dT * FT[m];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    // buoyancy: continuity test mode with bit z, temperature mode without it
    const R b = q1m_scale(q1m_mass_but(m, 2), cB);
    if (TR) YT[m] += b * FP[m + 4];
    else YP[m + 4] += b * FT[m];
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int bd = 1 << d;
      // convection: test mode without bit d, trial mode with it (transposed: the other way round)
      if (!TR && !(m & bd)) YT[m] += uc[d] * q1m_scale(q1m_mass_but(m, d), FT[m | bd]);
      if (TR && (m & bd)) YT[m] += uc[d] * q1m_scale(q1m_mass_but(m, d), FT[m & ~bd]);
      // cross streamline diffusion (symmetric): test bit d set and e clear, trial the reverse
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int be = 1 << e;
        if (e != d && (m & bd) && !(m & be)) YT[m] += q1m_scale(q1m_mass_third(m, d, e), ux[d][e]) * FT[m ^ bd ^ be];
      }
    }
  }
  q1_from_modal(YP, oP);
  q1_from_modal(YT, oT);
}

}  // namespace nc
