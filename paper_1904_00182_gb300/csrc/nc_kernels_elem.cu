// Element-sweep kernels: residual R(s), Jacobian products J v and J^T w, design sensitivities and
// centroid velocities. One thread per element (3D launch: 32 x 4 element columns per block, one
// z-layer per blockIdx.z, 32-bit index arithmetic) gathers its 8 nodes, evaluates the element
// arithmetic of nc_element.cuh and scatters the 16 row contributions with atomic adds
// (with kBcTop the Dirichlet rows on the top plane are skipped; otherwise the caller zeroes or sets the
// fixed rows, see fixed_bits).
#include "nc_launch.h"

namespace nc {

namespace {

template <typename R, typename V>
__device__ __forceinline__ void gather_state(const Grid& g, const V* __restrict__ s, int n0,
                                             R p[8], R t[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const V v = s[n0 + corner_off(g, a)];
    p[a] = (R)v.x;
    t[a] = (R)v.y;
  }
}

// Gather a direction vector; with `top` (kBcTop, element below the top plane) its Dirichlet entries are
// treated as zero (other boundary conditions keep every vector zero on the fixed set).
template <typename R, typename V>
__device__ __forceinline__ void gather_dir(const Grid& g, const V* __restrict__ v, int n0, bool top,
                                           R p[8], R t[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (top && (a >> 2)) { p[a] = R(0); t[a] = R(0); continue; }
    const V x = v[n0 + corner_off(g, a)];
    p[a] = (R)x.x;
    t[a] = (R)x.y;
  }
}

template <typename O, typename R>
__device__ __forceinline__ void scatter_add(const Grid& g, O* __restrict__ out, int n0, bool top,
                                            const R oP[8], const R oT[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (top && (a >> 2)) continue;
    const int n = n0 + corner_off(g, a);
    atomic_add_pair(out + 2 * n, (O)oP[a], (O)oT[a]);
  }
}

#define NC_ELEM_PROLOGUE()                                      \
  NC_IJK_3D();                                                  \
  if (i >= g.nx || j >= g.ny) return;                           \
  const int n0 = i + g.NX * j + g.NXY * k;                      \
  const int e = i + g.nx * (j + g.ny * k);                      \
  const bool top = g.bc == kBcTop && (k + 1 == g.nz);

template <typename R>
__device__ __forceinline__ R elem_source(const Phys& ph, int i, int j, int k) {
  return elem_heated(ph, i, j, k) ? (R)ph.Q : R(0);
}

__global__ void k_residual(Grid g, Phys ph, ElemConst<double> C, const double2* __restrict__ s,
                           const double2* __restrict__ mat, double* __restrict__ out) {
  NC_ELEM_PROLOGUE();
  double p[8], t[8];
  gather_state<double>(g, s, n0, p, t);
  const double2 m = mat[e];
  double RP[8], RT[8];
  elem_residual<double>(C, p, t, m.x, m.y, elem_source<double>(ph, i, j, k), RP, RT);
  scatter_add(g, out, n0, top, RP, RT);
}

// Dirichlet rows of the residual: R_d = s_d (boundary value 0), per fixed component.
__global__ void k_residual_bc(Grid g, const double2* __restrict__ s, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!boundary_node(g, t, i, j, k)) return;
  const int b = fixed_bits(g, i, j, k);
  const long long n = i + (long long)g.NX * (j + (long long)g.NY * k);
  if (b & 1) out[2 * n] = s[n].x;
  if (b & 2) out[2 * n + 1] = s[n].y;
}

// J v or J^T w. With DL (transpose only), the pass also stores the element derivatives
// (dL/dkappa_e, dL/dk_e) of L = w . R_e, the design derivatives the sensitivities need at this w.
template <typename R, typename SV, typename O, bool TRANSPOSE, bool DL = false>
__global__ void __launch_bounds__(128, 3) k_jprod(Grid g, Phys ph, ElemConst<R> C, const SV* __restrict__ s,
                        const typename Vec2<R>::type* __restrict__ mat, const double2* __restrict__ v,
                        O* __restrict__ out, double2* __restrict__ dl) {
  NC_ELEM_PROLOGUE();
  R p[8], t[8], dp[8], dt[8];
  gather_state<R>(g, s, n0, p, t);
  gather_dir<R>(g, v, n0, top, dp, dt);
  const typename Vec2<R>::type m = mat[e];
  ElemState<R> st;
  elem_state(C, p, t, m.x, elem_source<R>(ph, i, j, k), st);
  R oP[8], oT[8];
  if (TRANSPOSE && DL) {
    R dkap, dk;
    elem_jtv<R, true>(C, st, m.y, dp, dt, oP, oT, &dkap, &dk);
    dl[e] = make_double2((double)dkap, (double)dk);
  } else if (TRANSPOSE) {
    elem_jtv<R, false>(C, st, m.y, dp, dt, oP, oT, nullptr, nullptr);
  } else {
    elem_jv_dir<R>(C, st, m.y, dp, dt, oP, oT);
  }
  scatter_add(g, out, n0, top, oP, oT);
}

// df/dgamma~_e = -(dL/dkappa kappa' + dL/dk k') from stored element derivatives; 0 on passive elements.
__global__ void k_sens_from_dl(Grid g, Phys ph, const double2* __restrict__ dl, const double2* __restrict__ dmat,
                               double* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.ne; e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    elem_ijk(g, e, i, j, k);
    const double2 a = dl[e], d = dmat[e];
    out[e] = elem_design(ph, i, j, k) ? -(a.x * d.x + a.y * d.y) : 0.0;
  }
}

__global__ void k_sens(Grid g, Phys ph, ElemConst<double> C, const double2* __restrict__ s,
                       const double2* __restrict__ lam, const double2* __restrict__ mat,
                       const double2* __restrict__ dmat, double* __restrict__ out) {
  NC_ELEM_PROLOGUE();
  if (!elem_design(ph, i, j, k)) { out[e] = 0.0; return; }
  double p[8], t[8], lp[8], lt[8];
  gather_state<double>(g, s, n0, p, t);
  gather_dir<double>(g, lam, n0, top, lp, lt);
  const double2 m = mat[e];
  ElemState<double> st;
  elem_state(C, p, t, m.x, 0.0, st);
  double oP[8], oT[8], dkap, dk;
  elem_jtv<double, true>(C, st, m.y, lp, lt, oP, oT, &dkap, &dk);
  const double2 d = dmat[e];
  out[e] = -(dkap * d.x + dk * d.y);
}

__global__ void k_u_centroid(Grid g, Phys ph, ElemConst<double> C, const double2* __restrict__ s,
                             const double2* __restrict__ mat, double* __restrict__ u) {
  NC_ELEM_PROLOGUE();
  (void)top;
  double p[8], t[8];
  gather_state<double>(g, s, n0, p, t);
  ElemState<double> st;
  elem_state(C, p, t, mat[e].x, 0.0, st);
  u[3 * e] = st.u0x;
  u[3 * e + 1] = st.u0y;
  u[3 * e + 2] = st.u0z;
}

// Thermal compliance of Eq. objdiscr on one heated element, f_e = f_tQ,e . t_e with the SUPG-weighted
// source load f_tQ,e,a = sum_q w Q N*_a(q), N* = N + tau u0 . grad N. With sum_q N_a(q) = 1 on the
// 2x2x2 rule: f_e = Q w (sum_a t_a + tau u0 . G), G = sum_q grad T_q. Its state derivative (the
// adjoint load) follows from du0 = -(c/8) sum_q (grad dP_q - beta dT_q e_z) and
// dtau = -tau^3 (4/h_e^2) u0 . du0:
//   df_e = Q w [ sum_q dT_q + tau u0 . sum_q grad dT_q + A . du0 ],  A = tau G - tau^3 (4/h_e^2)(u0 . G) u0,
// i.e. test-function sums with constant coefficients: T rows N-part Q w (1 + (c/8) beta A_z) and
// gradient part Q w tau u0; P rows gradient part -Q w (c/8) A. Gradients are in element units here
// (Gh = h G, Ah = h A) and the test-function stage takes its gradient weights divided by h.
__global__ void k_obj_supg(Grid g, Phys ph, ElemConst<double> C, const double2* __restrict__ s,
                           const double2* __restrict__ mat, double* __restrict__ fe, double* __restrict__ d) {
  NC_ELEM_PROLOGUE();
  double p[8], t[8];
  gather_state<double>(g, s, n0, p, t);
  const double2 m = mat[e];
  const double Q = elem_source<double>(ph, i, j, k);
  ElemState<double> st;
  elem_state(C, p, t, m.x, Q, st);
  double Gx = 0, Gy = 0, Gz = 0, tsum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) { Gx += st.hx[q]; Gy += st.hy[q]; Gz += st.hz[q]; tsum += t[q]; }
  const double Qw = Q * C.w;
  const double u0G = st.u0x * Gx + st.u0y * Gy + st.u0z * Gz;   // h u0 . G
  fe[e] = Qw * (tsum + st.tau * C.ih * u0G);
  const double t3 = st.tau * st.tau * st.tau * C.c4he2 * u0G;
  const double Ax = st.tau * Gx - t3 * st.u0x, Ay = st.tau * Gy - t3 * st.u0y, Az = st.tau * Gz - t3 * st.u0z;
  const double cb = 0.125 * st.c;
  double An[8], Bx[8], By[8], Bz[8], oP[8], oT[8];
  const double Qwt = Qw * st.tau * C.ih;
  const double Qwc = -Qw * cb * C.ih * C.ih;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    An[q] = Qw * (1.0 + cb * C.beta * C.ih * Az);
    Bx[q] = Qwt * st.u0x; By[q] = Qwt * st.u0y; Bz[q] = Qwt * st.u0z;
  }
  q1_test<double, true>(An, Bx, By, Bz, C.cm, oT);
#pragma unroll
  for (int q = 0; q < 8; ++q) { Bx[q] = Qwc * Ax; By[q] = Qwc * Ay; Bz[q] = Qwc * Az; }
  q1_test<double, false>(nullptr, Bx, By, Bz, C.cm, oP);
  scatter_add(g, d, n0, top, oP, oT);
}

// ---- double-float variants (mixed-precision path) ----
// Minimum resident blocks of 128 threads per SM (register budget) of the double-float kernels.
#ifndef NC_LB_RESIDUAL_DF
#define NC_LB_RESIDUAL_DF 4
#endif
#ifndef NC_LB_JTV_DF
#define NC_LB_JTV_DF 4
#endif
#ifndef NC_LB_SENS_DF
#define NC_LB_SENS_DF 2
#endif
// Inputs arrive split once per call: state and direction as float4 (P.hi, P.lo, T.hi, T.lo) per
// node, materials as float4 (kappa.hi, kappa.lo, k.hi, k.lo) per element. Outputs are converted to
// FP64 (hi + lo) and accumulated with FP64 atomics, as in the FP64 kernels.

__global__ void k_split2(const double2* __restrict__ x, float4* __restrict__ y, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    const df64 a = df_from_double(v.x), b = df_from_double(v.y);
    y[t] = make_float4(a.hi, a.lo, b.hi, b.lo);
  }
}

__device__ __forceinline__ void gather_df(const Grid& g, const float4* __restrict__ s, int n0, bool zero_top,
                                          df64 p[8], df64 t[8]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (zero_top && (a >> 2)) { p[a] = df64(0.0f, 0.0f); t[a] = df64(0.0f, 0.0f); continue; }
    const float4 v = s[n0 + corner_off(g, a)];
    p[a] = df64(v.x, v.y);
    t[a] = df64(v.z, v.w);
  }
}

__global__ void __launch_bounds__(128, NC_LB_RESIDUAL_DF) k_residual_df(Grid g, Phys ph, ElemConst<df64> C, df64 Qh, const float4* __restrict__ s,
                              const float4* __restrict__ mat, double* __restrict__ out) {
  NC_ELEM_PROLOGUE();
  df64 p[8], t[8];
  gather_df(g, s, n0, false, p, t);
  const float4 m = mat[e];
  const df64 Q = elem_heated(ph, i, j, k) ? Qh : df64(0.0f, 0.0f);
  df64 RP[8], RT[8];
  elem_residual<df64>(C, p, t, df64(m.x, m.y), df64(m.z, m.w), Q, RP, RT);
  scatter_add(g, out, n0, top, RP, RT);
}

template <bool DL>
__global__ void __launch_bounds__(128, NC_LB_JTV_DF) k_jtv_df(Grid g, Phys ph, ElemConst<df64> C, df64 Qh, const float4* __restrict__ s,
                         const float4* __restrict__ mat, const float4* __restrict__ w, double* __restrict__ out,
                         double2* __restrict__ dl) {
  NC_ELEM_PROLOGUE();
  df64 p[8], t[8], lp[8], lt[8];
  gather_df(g, s, n0, false, p, t);
  gather_df(g, w, n0, top, lp, lt);
  const float4 m = mat[e];
  ElemState<df64> st;
  elem_state(C, p, t, df64(m.x, m.y), elem_heated(ph, i, j, k) ? Qh : df64(0.0f, 0.0f), st);
  df64 oP[8], oT[8];
  if (DL) {
    df64 dkap, dk;
    elem_jtv<df64, true>(C, st, df64(m.z, m.w), lp, lt, oP, oT, &dkap, &dk);
    dl[e] = make_double2((double)dkap, (double)dk);
  } else {
    elem_jtv<df64, false>(C, st, df64(m.z, m.w), lp, lt, oP, oT, nullptr, nullptr);
  }
  scatter_add(g, out, n0, top, oP, oT);
}

__global__ void __launch_bounds__(128, NC_LB_SENS_DF) k_sens_df(Grid g, Phys ph, ElemConst<df64> C, const float4* __restrict__ s,
                          const float4* __restrict__ lam, const float4* __restrict__ mat,
                          const double2* __restrict__ dmat, double* __restrict__ out) {
  NC_ELEM_PROLOGUE();
  if (!elem_design(ph, i, j, k)) { out[e] = 0.0; return; }
  df64 p[8], t[8], lp[8], lt[8];
  gather_df(g, s, n0, false, p, t);
  gather_df(g, lam, n0, top, lp, lt);
  const float4 m = mat[e];
  ElemState<df64> st;
  elem_state(C, p, t, df64(m.x, m.y), df64(0.0f, 0.0f), st);
  df64 oP[8], oT[8], dkap, dk;
  elem_jtv<df64, true>(C, st, df64(m.z, m.w), lp, lt, oP, oT, &dkap, &dk);
  const double2 d = dmat[e];
  out[e] = -((double)dkap * d.x + (double)dk * d.y);
}

}  // namespace

cudaError_t launch_obj_supg(const Grid& g, const Phys& ph, const double2* s, const double2* mat, double* fe,
                            double* d, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(d, 0, sizeof(double) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  Launch3 L = launch_elems(g);
  // boxes: the source lies in the bottom heated layers only; cylinders: every layer is visited
  if (ph.shape != 1) L.grid.z = (unsigned)ph.heated_layers;
  k_obj_supg<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<double>(ph), s, mat, fe, d);
  if (c) { c->launches += 1; c->bytes += 16.0 * g.nn + 24.0 * g.nx * g.ny * L.grid.z; }
  return cudaGetLastError();
}

cudaError_t launch_split2(const double2* x, float4* y, long long n, cudaStream_t st, Counters* c) {
  k_split2<<<grid_blocks(n, 256, 152 * 16), 256, 0, st>>>(x, y, n);
  if (c) { c->launches += 1; c->bytes += 32.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_residual_df(const Grid& g, const Phys& ph, const double2* s, const float4* mat_df,
                               float4* s_df, double* out, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(out, 0, sizeof(double) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  err = launch_split2(s, s_df, g.nn, st, c);
  if (err != cudaSuccess) return err;
  const Launch3 L = launch_elems(g);
  k_residual_df<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<df64>(ph), df64(ph.Q), s_df, mat_df, out);
  k_residual_bc<<<grid_blocks(boundary_count(g), 256), 256, 0, st>>>(g, s, out);
  if (c) { c->launches += 2; c->bytes += 16.0 * g.nn * 2 + 16.0 * g.ne; c->flops += kFlopsResidualDF * g.ne; }
  return cudaGetLastError();
}

cudaError_t launch_jtv_df(const Grid& g, const Phys& ph, const double2* s, const float4* mat_df, float4* s_df,
                          const double2* w, float4* w_df, double* out, double2* dl, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(out, 0, sizeof(double) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  if ((err = launch_split2(s, s_df, g.nn, st, c)) != cudaSuccess) return err;
  if ((err = launch_split2(w, w_df, g.nn, st, c)) != cudaSuccess) return err;
  const Launch3 L = launch_elems(g);
  if (dl) k_jtv_df<true><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<df64>(ph), df64(ph.Q), s_df, mat_df, w_df, out, dl);
  else k_jtv_df<false><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<df64>(ph), df64(ph.Q), s_df, mat_df, w_df, out, dl);
  if (c) {
    c->launches += 1;
    c->bytes += (32.0 + 16.0) * g.nn + 16.0 * g.ne;
    c->flops += (kFlopsStateDF + (dl ? kFlopsSensDF : kFlopsJtvDF)) * g.ne;
  }
  return cudaGetLastError();
}

cudaError_t launch_sens_df(const Grid& g, const Phys& ph, const double2* s, const double2* lam, const float4* mat_df,
                           const double2* dmat, float4* s_df, float4* l_df, double* out, cudaStream_t st, Counters* c) {
  cudaError_t err;
  if ((err = launch_split2(s, s_df, g.nn, st, c)) != cudaSuccess) return err;
  if ((err = launch_split2(lam, l_df, g.nn, st, c)) != cudaSuccess) return err;
  const Launch3 L = launch_elems(g);
  k_sens_df<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<df64>(ph), s_df, l_df, mat_df, dmat, out);
  if (c) { c->launches += 1; c->bytes += 32.0 * g.nn + 40.0 * g.ne; c->flops += (kFlopsStateDF + kFlopsSensDF) * g.ne; }
  return cudaGetLastError();
}

cudaError_t launch_residual(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                            double* out, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(out, 0, sizeof(double) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  const Launch3 L = launch_elems(g);
  k_residual<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<double>(ph), s, mat, out);
  k_residual_bc<<<grid_blocks(boundary_count(g), 256), 256, 0, st>>>(g, s, out);
  if (c) { c->launches += 2; c->bytes += 16.0 * g.nn * 2 + 16.0 * g.ne; c->flops += kFlopsResidual * g.ne; }
  return cudaGetLastError();
}

template <typename R, typename SV, bool TR>
static cudaError_t jprod(const Grid& g, const Phys& ph, const SV* s, const typename Vec2<R>::type* mat,
                         const double2* v, double* out, double2* dl, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(out, 0, sizeof(double) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  const Launch3 L = launch_elems(g);
  if constexpr (TR) {
    if (dl) k_jprod<R, SV, double, true, true><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, v, out, dl);
    else k_jprod<R, SV, double, true, false><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, v, out, dl);
  } else {
    k_jprod<R, SV, double, false, false><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, v, out, dl);
  }
  if (c) {
    c->launches += 1;
    c->bytes += (2.0 * sizeof(SV) + 32.0) * g.nn + 2.0 * sizeof(R) * g.ne + (dl ? 16.0 * g.ne : 0.0);
    static_assert(!ScaleSums<R>::value, "the FP64 flop counts assume the Gauss-point form");
    c->flops += (kFlopsState + (TR ? (dl ? kFlopsSens : kFlopsJtv) : kFlopsJv)) * g.ne;
  }
  return cudaGetLastError();
}

cudaError_t launch_jv_f64(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                          const double2* v, double* out, cudaStream_t st, Counters* c) {
  return jprod<double, double2, false>(g, ph, s, mat, v, out, nullptr, st, c);
}
cudaError_t launch_jtv_f64(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                           const double2* w, double* out, double2* dl, cudaStream_t st, Counters* c) {
  return jprod<double, double2, true>(g, ph, s, mat, w, out, dl, st, c);
}

cudaError_t launch_sens_from_dl(const Grid& g, const Phys& ph, const double2* dl, const double2* dmat, double* out,
                                cudaStream_t st, Counters* c) {
  k_sens_from_dl<<<grid_blocks(g.ne, 256, 152 * 16), 256, 0, st>>>(g, ph, dl, dmat, out);
  if (c) { c->launches += 1; c->bytes += 40.0 * g.ne; }
  return cudaGetLastError();
}

cudaError_t launch_sens_elem(const Grid& g, const Phys& ph, const double2* s, const double2* lam,
                             const double2* mat, const double2* dmat, double* out, cudaStream_t st,
                             Counters* c) {
  const Launch3 L = launch_elems(g);
  k_sens<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<double>(ph), s, lam, mat, dmat, out);
  if (c) { c->launches += 1; c->bytes += 32.0 * g.nn + 40.0 * g.ne; c->flops += (kFlopsState + kFlopsSens) * g.ne; }
  return cudaGetLastError();
}

cudaError_t launch_u_centroid(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                              double* u, cudaStream_t st, Counters* c) {
  const Launch3 L = launch_elems(g);
  k_u_centroid<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<double>(ph), s, mat, u);
  if (c) { c->launches += 1; c->bytes += 16.0 * g.nn + 40.0 * g.ne; }
  return cudaGetLastError();
}

}  // namespace nc
