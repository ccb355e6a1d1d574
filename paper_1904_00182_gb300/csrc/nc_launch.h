// Host-side launchers of the natconv kernels (all asynchronous on the given stream).
#pragma once

#include <cuda_runtime.h>
#include "nc_common.cuh"
#include "nc_element.cuh"

namespace nc {

// Physical constants of one problem, in FP64; converted to ElemConst<R> per launch.
// Regions of elements: heated (passive solid with the source) [0, heat_nx) x [0, heat_ny) x
// [0, heated_layers); design [0, design_nx) x [0, design_ny) x [heated_layers, design_z1) minus the
// heated box; every other element is passive fluid. With the full extents (the default) the heated
// region is the bottom layers and every element above them is a design element.
// With shape = 1 (cylinders about the z axis through the corner x = y = 0) an element is heated when
// its centroid lies within the heat radius and its layer in [z0, z0 + heated_layers), and a design
// element when its centroid lies within the design radius (and not the heat radius) over the same
// layers. The radius tests are exact integer ones: (2i+1)^2 + (2j+1)^2 < 4 r^2, held as
// q < ceil(4 r^2).
struct Phys {
  double h, beta, rc, mu, he, tau3, Q;  // Q: source in the heated region (already ramped)
  int heated_layers;
  int heat_nx, heat_ny;
  int design_nx, design_ny, design_z1;
  int shape, z0, q_heat, q_design;
};

__host__ __device__ __forceinline__ int centroid_q(int i, int j) { return (2 * i + 1) * (2 * i + 1) + (2 * j + 1) * (2 * j + 1); }

__host__ __device__ __forceinline__ bool elem_heated(const Phys& ph, int i, int j, int k) {
  if (ph.shape == 1) return k >= ph.z0 && k < ph.z0 + ph.heated_layers && centroid_q(i, j) < ph.q_heat;
  return i < ph.heat_nx && j < ph.heat_ny && k < ph.heated_layers;
}
__host__ __device__ __forceinline__ bool elem_design(const Phys& ph, int i, int j, int k) {
  if (ph.shape == 1)
    return k >= ph.z0 && k < ph.z0 + ph.heated_layers && centroid_q(i, j) < ph.q_design &&
           centroid_q(i, j) >= ph.q_heat;
  return !elem_heated(ph, i, j, k) && i < ph.design_nx && j < ph.design_ny && k >= ph.heated_layers &&
         k < ph.design_z1;
}

template <typename R>
inline ElemConst<R> make_econst(const Phys& p) {
  ElemConst<R> C;
  const double g = 1.0 / 1.7320508075688772935;   // 1/sqrt(3)
  C.cm = (R)(0.5 * (1.0 - g));
  C.ih = (R)(1.0 / p.h);
  C.w = (R)(0.125 * p.h * p.h * p.h);
  C.wih = (R)(0.125 * p.h * p.h);
  C.wih2 = (R)(0.125 * p.h);
  C.beta = (R)p.beta;
  C.betah = (R)(p.beta * p.h);
  C.rc = (R)p.rc;
  C.rcih2 = (R)(p.rc / (p.h * p.h));
  C.imu = (R)(1.0 / p.mu);
  C.c4he2 = (R)(4.0 / (p.he * p.he));
  C.itau3sq = (R)(1.0 / (p.tau3 * p.tau3));
  return C;
}

// Counters of one call (kernel launches and algorithmic bytes).
struct Counters {
  long long launches = 0;
  double bytes = 0.0;
  double flops = 0.0;
};

// Floating-point operations per element of the element kernels (adds + multiplies, an FMA counts
// two), counted from nc_element.cuh by instantiating it with a counting number type: residual;
// element state; J v direction part; J^T w part; J^T w with design derivatives; one element-Jacobian
// column (the mean of the 8 P and 8 T columns). FP64 form (row factors at the Gauss points), then
// the ScaleSums form of the FP32 kernels (row factors on the test sums).
const double kFlopsResidual = 629.0, kFlopsState = 290.0, kFlopsJv = 743.0, kFlopsJtv = 778.0,
             kFlopsSens = 878.0, kFlopsJacColumn = 608.0;
const double kFlopsJvS = 714.0, kFlopsJtvS = 748.0, kFlopsJacColumnS = 579.0;
template <typename R> constexpr double flops_jv() { return ScaleSums<R>::value ? kFlopsJvS : kFlopsJv; }
template <typename R> constexpr double flops_jtv() { return ScaleSums<R>::value ? kFlopsJtvS : kFlopsJtv; }
template <typename R> constexpr double flops_jac_column() {
  return ScaleSums<R>::value ? kFlopsJacColumnS : kFlopsJacColumn;
}
// Frozen-coefficient (Picard) element operator and its transpose: the Gauss-point form, and the modal
// form the kernels use.
const double kFlopsPicard = 545.0, kFlopsPicardT = 548.0;
const double kFlopsPicardModal = 239.0, kFlopsPicardModalT = 239.0;
// The same element code (ScaleSums form) in double-float arithmetic, in FP32 flops: a double-float
// sum is 11 FP32 additions, a product 1 multiplication + 3 FMAs + 3 additions (10 flops). Adds /
// multiplies per element: residual 351 / 248, element state 167 / 123, J^T w part 399 / 349, with
// design derivatives 447 / 401.
const double kDfAdd = 11.0, kDfMul = 10.0;
const double kFlopsResidualDF = 351 * kDfAdd + 248 * kDfMul, kFlopsStateDF = 167 * kDfAdd + 123 * kDfMul,
             kFlopsJtvDF = 399 * kDfAdd + 349 * kDfMul, kFlopsSensDF = 447 * kDfAdd + 401 * kDfMul;

// ---------------- element operators (nc_kernels_elem.cu) ----------------
// out (2N doubles) = R(s); Dirichlet rows = s. s: double2 per node; mat: (kappa, k) per element.
cudaError_t launch_residual(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                            double* out, cudaStream_t st, Counters* c);
// out = J(s) v (projected: Dirichlet inputs ignored, Dirichlet outputs 0); FP64 arithmetic.
cudaError_t launch_jv_f64(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                          const double2* v, double* out, cudaStream_t st, Counters* c);
// out = J(s)^T w (projected), FP64. dl (nullable, E): element derivatives (dL/dkappa, dL/dk) of
// L = w . R_e, stored by the same pass.
cudaError_t launch_jtv_f64(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                           const double2* w, double* out, double2* dl, cudaStream_t st, Counters* c);
// df/dgamma~ = -(dL/dkappa kappa' + dL/dk k') from stored dl; 0 on passive (heated, fluid) elements.
cudaError_t launch_sens_from_dl(const Grid& g, const Phys& ph, const double2* dl, const double2* dmat, double* out,
                                cudaStream_t st, Counters* c);
// d f / d gamma~_e = -(dL/dkappa kappa' + dL/dk k'), 0 on passive elements; dmat: (kappa', k').
cudaError_t launch_sens_elem(const Grid& g, const Phys& ph, const double2* s, const double2* lam,
                             const double2* mat, const double2* dmat, double* out, cudaStream_t st,
                             Counters* c);
// Double-float (df64, about 48-bit) variants of the residual, J^T w and the sensitivities for the
// mixed-precision path: FP64 inputs are split into float4 (hi, lo) scratch arrays (s_df, w_df,
// l_df: one per node) and the materials come pre-split (mat_df: one per element); outputs are FP64.
cudaError_t launch_split2(const double2* x, float4* y, long long n, cudaStream_t st, Counters* c);
cudaError_t launch_residual_df(const Grid& g, const Phys& ph, const double2* s, const float4* mat_df,
                               float4* s_df, double* out, cudaStream_t st, Counters* c);
cudaError_t launch_jtv_df(const Grid& g, const Phys& ph, const double2* s, const float4* mat_df, float4* s_df,
                          const double2* w, float4* w_df, double* out, double2* dl, cudaStream_t st, Counters* c);
cudaError_t launch_sens_df(const Grid& g, const Phys& ph, const double2* s, const double2* lam, const float4* mat_df,
                           const double2* dmat, float4* s_df, float4* l_df, double* out, cudaStream_t st, Counters* c);
// Thermal compliance of Eq. objdiscr on the heated elements: fe[e] = f_tQ,e . t_e for e in the heated
// layers (boxes; every element for cylinders; other entries untouched) and d = its state derivative
// (2N, zeroed first).
cudaError_t launch_obj_supg(const Grid& g, const Phys& ph, const double2* s, const double2* mat, double* fe,
                            double* d, cudaStream_t st, Counters* c);
// Centroid Darcy velocity (3 per element).
cudaError_t launch_u_centroid(const Grid& g, const Phys& ph, const double2* s, const double2* mat,
                              double* u, cudaStream_t st, Counters* c);

// ---------------- vector / reduction / design kernels (nc_kernels_vec.cu) ----------------
// Deterministic reductions: partial sums per block, then a fixed-order final sum. At most
// kReduceBlocksMax blocks (8 per SM, enough loads in flight to stream vectors at full bandwidth).
const int kReduceBlocksMax = 1216;
int reduce_blocks(long long n);
// res[i] = <V_i, w> for i < nvec, V_i = V + i*ld; n entries each. part: nvec*reduce_blocks(n).
// FP32 vectors: FP32 products and per-thread sums, FP64 block and grid sums.
cudaError_t launch_multidot(const double* V, long long ld, int nvec, const double* w, long long n,
                            double* part, double* res, cudaStream_t st, Counters* c);
cudaError_t launch_multidot(const float* V, long long ld, int nvec, const float* w, long long n,
                            double* part, double* res, cudaStream_t st, Counters* c);
// res[0] = sum of a[0..n) (deterministic two-stage reduction).
cudaError_t launch_sum(const double* a, long long n, double* part, double* res, cudaStream_t st, Counters* c);
// res[0] = sum over free entries of a^2, for a state vector (kBcTop: the rows below the top plane;
// kBcCavity: every row, the fixed ones being zero in every vector this is called on).
cudaError_t launch_norm2_free(const Grid& g, const double* a, double* part, double* res,
                              cudaStream_t st, Counters* c);
// Gram-Schmidt step of FGMRES (nvec <= 32) from the first-pass dots d1 (device: V_i . w, then w . w):
// w <- (w - V d1) / sqrt(ww - |d1|^2) when ww - |d1|^2 >= thr ww (the projection kept at least the
// fraction thr of ||w||^2; thr = 1/2 is the Daniel-Gragg-Kaufman-Stewart test); otherwise classical
// Gram-Schmidt is applied twice and d2 receives the second-pass dots and ||w'||^2. The branch is
// taken on the device; the host repeats the same test on the read-back values.
cudaError_t launch_cgs(double* w, const double* V, long long ld, int nvec, const double* d1, double* d2, long long n,
                      double thr, double* part, cudaStream_t st, Counters* cnt);
cudaError_t launch_cgs(float* w, const float* V, long long ld, int nvec, const double* d1, double* d2, long long n,
                      double thr, double* part, cudaStream_t st, Counters* cnt);
// y += sum_i coef[i] * V_i (nvec <= 64), n entries.
cudaError_t launch_axpy_multi(double* y, const double* V, long long ld, int nvec, const double* coef,
                              long long n, cudaStream_t st, Counters* c);
cudaError_t launch_axpy_multi(double* y, const float* V, long long ld, int nvec, const double* coef,
                              long long n, cudaStream_t st, Counters* c);
cudaError_t launch_axpy_multi(float* y, const float* V, long long ld, int nvec, const double* coef,
                              long long n, cudaStream_t st, Counters* c);
// y = a*x + b*y
cudaError_t launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st,
                         Counters* c);
// y = y * a (in place)
cudaError_t launch_scale(double* y, double a, long long n, cudaStream_t st, Counters* c);
cudaError_t launch_scale(float* y, double a, long long n, cudaStream_t st, Counters* c);
// y = x * a
cudaError_t launch_scale_copy(double* y, const double* x, double a, long long n, cudaStream_t st,
                              Counters* c);
cudaError_t launch_scale_copy(float* y, const double* x, double a, long long n, cudaStream_t st,
                              Counters* c);
cudaError_t launch_cast_d2f(float* y, const double* x, long long n, cudaStream_t st, Counters* c);
cudaError_t launch_cast_f2d(double* y, const float* x, long long n, cudaStream_t st, Counters* c);
// Zero the Dirichlet entries of a state vector (the fixed set of g.bc).
cudaError_t launch_zero_dirichlet(const Grid& g, double* a, cudaStream_t st, Counters* c);
cudaError_t launch_zero_dirichlet(const Grid& g, float* a, cudaStream_t st, Counters* c);
// Design check: flag = 1 if any value is NaN or outside [0,1].
cudaError_t launch_check_design(const double* rho, long long ne, int* flag, cudaStream_t st);
// Filter pieces (Helmholtz (r^2 K + M) x = T^T gamma, Q1 nodal, element mean out).
struct FilterConst { double A[64]; double C27[27]; double t0; double diag; };
struct FilterConstF { float A[64]; float C27[27]; };
struct FilterConstDF { df64 A[64]; df64 C27[27]; };
// Double-float refinement steps of the filter solve (op): 0 bd = b64 in double-float; 1 x += dx;
// 2 r = bd - (r^2 K + M) x in double-float, rf = its FP32 leading part, r64 = r in FP64; 3 y64 = x.
cudaError_t launch_filter_df(int op, const Grid& g, const FilterConstDF* F, const double* b64, df64* bd, df64* x,
                             const float* dx, float* rf, double* r64, double* y64, cudaStream_t st, Counters* c);
// y = (r^2 K + M) x (FP64 residual with F; FP32 inside the Chebyshev step with Ff); Chebyshev iteration
// in FP32 on D^-1 (r^2 K + M):
//   init: x = 0, d = c0 dinv r;   step: x += d, r -= A d, dn = c1 d + c2 dinv r
cudaError_t launch_cheb_init(long long n, const float* dinv, const float* r, float* x, float* d, float c0,
                             cudaStream_t st, Counters* c);
cudaError_t launch_cheb_step(const Grid& g, const FilterConstF& F, const float* dinv, const float* d, float* dn,
                             float* x, float* r, float c1, float c2, cudaStream_t st, Counters* c);
// y += (double) x
cudaError_t launch_add_f2d(double* y, const float* x, long long n, cudaStream_t st, Counters* c);
// t /= the filter operator's eigenvalue of each node's mode in the per-axis cosine basis (lam: 1D
// stiffness, mu: 1D mass eigenvalues of x, y, z; r2: the filter's r^2).
cudaError_t launch_filter_scale(const Grid& g, float* t, const float* const lam[3], const float* const mu[3],
                                float r2, cudaStream_t st, Counters* c);
// b = T^T g with g = gamma on design elements, 1 on heated and 0 on fluid elements (passive=true) or
// g = gamma everywhere (passive=false).
cudaError_t launch_filter_rhs(const Grid& g, const Phys& ph, bool passive, const double* gamma, double scale_elem,
                              double* b, cudaStream_t st, Counters* c);
cudaError_t launch_helmholtz(const Grid& g, const FilterConst& F, const double* x, double* y,
                             cudaStream_t st, Counters* c);
cudaError_t launch_helmholtz_diag(const Grid& g, const FilterConst& F, double* dinv, cudaStream_t st);
// out_e = scale * sum_a x_{n(e,a)}; if heated_value >= 0, heated elements get heated_value and fluid
// elements 0
cudaError_t launch_elem_from_nodes(const Grid& g, const Phys& ph, const double* x, double scale,
                                   double heated_value, double* out, cudaStream_t st, Counters* c);
// RAMP (Eqs. condRAMP, permRAMP): mat = (kappa, k), dmat = (kappa', k'), mat32 FP32 copy.
struct RampConst { double kappa_f, kappa_s, k_f, k_s, q_c, q_p; };
cudaError_t launch_ramp(const double* gt, long long ne, const RampConst& r, double2* mat, double2* dmat,
                        float2* mat32, cudaStream_t st, Counters* c);
// Objective weights df/ds (mean T over the heated region) and objective value.
cudaError_t launch_dfds(const Grid& g, const Phys& ph, double w_node, double* out, cudaStream_t st,
                        Counters* c);

// ---------------- multigrid (nc_kernels_mg.cu) ----------------
// Largest coarsest-level system (rows of the dense matrix) the coarse solve stages in shared memory.
constexpr int kMaxCoarseDofs = 2048;
template <typename R> struct MGLevelDev {
  Grid g;
  typename Vec2<R>::type* x;
  typename Vec2<R>::type* xn;
  typename Vec2<R>::type* b;
  typename Vec2<R>::type* y;
  R* ebe;       // 256 per element (levels >= 1)
  R* S;         // assembled 27-point 2x2-block stencil, 108 per node, 27 planes of 2x2 blocks (levels 1 .. L-2)
  R* dinv;      // 4 per node (2x2 block-diagonal inverse, row major), 0 on Dirichlet nodes
  R* lf;        // z-line smoother factors, 24 per node (levels 1 .. L-2 with the z-line smoother), else null
};

// Fused multigrid tail: the part of a V-cycle on levels l0 .. L-1 (the small coarse grids) run by
// one thread-block cluster, its steps separated by cluster barriers instead of kernel launches.
// lev[0] is level l0, lev[nlev-1] the coarsest (solved with Ainv32 / Ac as launch_coarse_solve).
// The kernel swaps x and xn of each non-coarsest level (nu1 - 1 + nu2) times, like the launch
// sequence; the caller applies the same swaps to its pointers.
const int kTailMaxLevels = 8;
template <typename R> struct TailLevel {
  Grid g;
  const R* S;
  const R* dinv;
  typename Vec2<R>::type* x;
  typename Vec2<R>::type* xn;
  typename Vec2<R>::type* b;
};
template <typename R> struct TailArgs {
  TailLevel<R> lev[kTailMaxLevels];
  int nlev;
  const double* Ac;
  const float* Ainv32;
  double* cw;   // 3 nf
  int nf;
  R omega;
  int nu1, nu2;
  int ctas;     // CTAs of the cluster (1..16); 0: the largest cluster the device schedules (16, else 8)
};
template <typename R>
cudaError_t launch_mg_tail(const TailArgs<R>& a, bool transpose, cudaStream_t st, Counters* c);

// Level-0 set-up: element matrices of J(s) (picard: of the frozen-coefficient operator at s) in R
// arithmetic -> block diagonal of level 0 and Galerkin element matrices of level 1 (P^T A P with
// trilinear P).
template <typename R>
cudaError_t launch_galerkin_fine(const Grid& gf, const Grid& gc, const Phys& ph,
                                 const typename Vec2<R>::type* s, const typename Vec2<R>::type* mat,
                                 R* diag_f, R* ebe_c, cudaStream_t st, Counters* c, bool picard = false);
// Level l -> l+1 Galerkin from stored element matrices; accumulates the block diagonal of level l.
template <typename R>
cudaError_t launch_galerkin_coarse(const Grid& gf, const Grid& gc, const R* ebe_f, R* diag_f, R* ebe_c,
                                   cudaStream_t st, Counters* c);
// Invert the 2x2 blocks in place (Dirichlet nodes -> 0). flag = 1 on a singular block.
template <typename R>
cudaError_t launch_invert_diag(const Grid& g, R* diag, int* flag, cudaStream_t st, Counters* c);
// y = A x on the finest level: matrix-free J(s) (or J^T).
// Frozen coefficients (u0x, u0y, u0z, tau) per element of the Picard operator at the FP32 state s.
cudaError_t launch_frozen(const Grid& g, const Phys& ph, const float2* s, const float2* mat, float4* fz,
                          cudaStream_t st, Counters* c);
// y = A x (transpose: A^T x) with the frozen-coefficient (Picard) finest-level operator, FP32.
// kc: elements per thread along z (column walking; 0: automatic), or -1: one thread per element.
cudaError_t launch_level0_picard(const Grid& g, const Phys& ph, const float4* fz, const float2* mat, const float2* x,
                                 float2* y, bool transpose, cudaStream_t st, Counters* c, int kc);
template <typename R>
cudaError_t launch_level0_apply(const Grid& g, const Phys& ph, const typename Vec2<R>::type* s,
                                const typename Vec2<R>::type* mat, const typename Vec2<R>::type* x,
                                typename Vec2<R>::type* y, bool transpose, cudaStream_t st, Counters* c, int kc = -1);
// x_new = x + omega D^-1 (b - y)   (y = A x; first == true: x = 0, y unused)
template <typename R>
cudaError_t launch_jacobi_update(const Grid& g, const R* dinv, const typename Vec2<R>::type* b,
                                 const typename Vec2<R>::type* y, const typename Vec2<R>::type* x,
                                 typename Vec2<R>::type* xn, R omega, bool transpose, bool first,
                                 cudaStream_t st, Counters* c);
// The finest-level update of a preconditioner call with FP64 input / output: first = true reads b
// from b64 (storing its R copy in b); z64 (nullable) also receives the new x in FP64.
template <typename R>
cudaError_t launch_jacobi_io(const Grid& g, const R* dinv, typename Vec2<R>::type* b, const double* b64,
                             const typename Vec2<R>::type* y, const typename Vec2<R>::type* x,
                             typename Vec2<R>::type* xn, double* z64, R omega, bool transpose, bool first,
                             cudaStream_t st, Counters* c);
// b_c = P^T r_f (full weighting, Dirichlet coarse rows 0). With xc, also the coarse level's first
// block-Jacobi sweep from zero, x_c = omega D_c^-1 b_c (transpose: D_c^-T; dinv_c: the inverted
// 2x2 blocks).
template <typename R>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* rf,
                            typename Vec2<R>::type* bc, cudaStream_t st, Counters* c, const R* dinv_c = nullptr,
                            typename Vec2<R>::type* xc = nullptr, R omega = R(0), bool transpose = false);
// Restriction of the residual b - y formed on the fly (level 0: no residual vector is stored); the
// optional first coarse sweep as for launch_restrict.
template <typename R>
cudaError_t launch_restrict_residual(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* b,
                                     const typename Vec2<R>::type* y, typename Vec2<R>::type* bc, cudaStream_t st,
                                     Counters* c, const R* dinv_c = nullptr, typename Vec2<R>::type* xc = nullptr,
                                     R omega = R(0), bool transpose = false);
// x_f += P x_c
template <typename R>
cudaError_t launch_prolong_add(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* xc,
                               typename Vec2<R>::type* xf, cudaStream_t st, Counters* c);
// Coarsest level: dense FP64 matrix of the free DOFs from element matrices; its FP32 inverse
// (one-block Gauss-Jordan, work: nf x 2nf floats); and the solve x = A^-1 b (or A^-T b) from the
// FP32 inverse with one FP64 refinement step (nf <= 1024; work: 3 nf doubles).
template <typename R>
cudaError_t launch_dense_assemble(const Grid& g, const R* ebe, double* A, int nf, cudaStream_t st,
                                  Counters* c);
cudaError_t launch_coarse_factor(const double* A, float* work, float* Ainv32, int nf, int* flag, cudaStream_t st,
                                 Counters* c);
template <typename R>
cudaError_t launch_coarse_solve(const double* A, const float* Ainv32, double* work, int nf,
                                const typename Vec2<R>::type* b, typename Vec2<R>::type* x, long long nn,
                                bool transpose, cudaStream_t st, Counters* c);
// Assembled stencil of a coarse level from its element matrices (Dirichlet rows/columns zero), and
// its application: mode 0 y = A x, mode 1 r = b - A x, mode 2 x_new = x + omega D^-1 (b - A x).
template <typename R>
cudaError_t launch_stencil_build(const Grid& g, const R* ebe, R* S, cudaStream_t st, Counters* c);
template <typename R>
cudaError_t launch_stencil_apply(const Grid& g, const R* S, const typename Vec2<R>::type* x,
                                 const typename Vec2<R>::type* b, const R* dinv, R omega,
                                 typename Vec2<R>::type* out, bool transpose, int mode, cudaStream_t st,
                                 Counters* c);
// z-line block-Jacobi smoother of a level with an assembled stencil. launch_line_factor eliminates
// down every node column of S and of its transpose (LF: 24 nn values, the forward direction's 12 nn
// first; flag = 1 on a singular pivot block); launch_line_smooth updates x <- x + omega T^-1 r with T
// the column-tridiagonal part of the operator (transpose: of A^T), overwriting r, or with first:
// x <- omega T^-1 r from x = 0 (r is kept).
template <typename R>
cudaError_t launch_line_factor(const Grid& g, const R* S, R* LF, int* flag, cudaStream_t st, Counters* c);
template <typename R>
cudaError_t launch_line_smooth(const Grid& g, const R* LF, const typename Vec2<R>::type* r,
                               typename Vec2<R>::type* x, R omega, bool transpose, bool first, cudaStream_t st,
                               Counters* c);
// Cast a multigrid-type state vector to FP64.
template <typename R>
cudaError_t launch_from_mg(const typename Vec2<R>::type* x, double* z, long long nn, cudaStream_t st,
                           Counters* c);

}  // namespace nc
