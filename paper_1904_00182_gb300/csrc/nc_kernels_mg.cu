// Geometric multigrid kernels, templated on the multigrid arithmetic type R (float: mixed
// precision preconditioner; double: the all-FP64 path).
//
// Hierarchy: level l has (nx/2^l, ny/2^l, nz/2^l) elements. Transfer operators are trilinear
// interpolation P and its transpose (full weighting) R = P^T. Coarse operators are Galerkin
// products P^T A P assembled element by element: a coarse element's matrix is the sum over its 8
// children of P_c^T A_c P_c, where P_c interpolates the child's 8 nodes from the parent's 8
// corners (exact for nested trilinear spaces). Level 0 applies the Newton Jacobian J(s) matrix
// free; levels >= 1 store 16x16 element matrices (rows/cols: P_0..7, T_0..7) for the set-up of the
// next level and, for their application, the assembled 27-point 2x2-block stencil (gathered per
// node, no atomics). The smoother is damped 2x2 node-block Jacobi; the coarsest level is solved with
// an FP32 Gauss-Jordan inverse (partial pivoting) and one step of FP64 iterative refinement (the
// coarse residual is computed in FP64 against the FP64 Galerkin matrix).
#include <cooperative_groups.h>

#include <mutex>
#include <type_traits>

#include "nc_launch.h"

namespace nc {

namespace {

const int kMaxDevices = 64;   // per-device caches of function attributes

// Loads of the node bodies of the transfer and stencil operators: plain (separate launches; read-only data may take the
// non-coherent path) or L2-coherent (the fused tail kernel, whose vectors change between its steps).
struct LdPlain {
  template <typename T> __device__ __forceinline__ T operator()(const T* p) const { return *p; }
};
struct LdCG {
  template <typename T> __device__ __forceinline__ T operator()(const T* p) const { return __ldcg(p); }
};

// out[A] = sum_l P_c[l][A] in[l]: transpose of the trilinear interpolation from the parent's 8
// corners A to the 8 nodes l of child c, applied as three 1D stages. Along an axis where the child
// bit is 0 the child's nodes sit at parent positions (0, 1/2): P1 = [[1, 0], [1/2, 1/2]];
// where it is 1 they sit at (1/2, 1): P1 = [[1/2, 1/2], [0, 1]] (rows: child node, columns: corner).
template <typename R>
__device__ __forceinline__ void interp_T(int child, const R in[8], R out[8]) {
  R t[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) t[q] = in[q];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = 1 << d;
    const bool hi = (child >> d) & 1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q & st) continue;
      const R v0 = t[q], v1 = t[q + st];
      if (!hi) { t[q] = v0 + R(0.5) * v1; t[q + st] = R(0.5) * v1; }
      else { t[q] = R(0.5) * v0; t[q + st] = R(0.5) * v0 + v1; }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) out[q] = t[q];
}

template <typename R>
__device__ __forceinline__ void add_diag_block(R* __restrict__ diag, long long n, int idx, R v) {
  atomicAdd(diag + 4 * n + idx, v);
}

// Galerkin product of one coarse element from its children's matrices Jc[c] (16 rows of stride
// NC_LD, shared memory): Tc = Jc P_c (per row, both field blocks), Uc = P_c^T Tc (per column),
// out = sum_c Uc. 128 threads. The row stride 17 keeps row and column accesses conflict-free.
#define NC_LD 17
template <typename R>
__device__ __forceinline__ void galerkin_phase2(R (*Jc)[16 * NC_LD], R (*Tc)[16 * NC_LD], R* __restrict__ out) {
  const int t = threadIdx.x;
  for (int it = t; it < 128; it += blockDim.x) {   // (child, row) pairs
    const int c = it >> 4, row = it & 15;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      R in[8], o[8];
#pragma unroll
      for (int l = 0; l < 8; ++l) in[l] = Jc[c][row * NC_LD + f * 8 + l];
      interp_T<R>(c, in, o);
#pragma unroll
      for (int A = 0; A < 8; ++A) Tc[c][row * NC_LD + f * 8 + A] = o[A];
    }
  }
  __syncthreads();
  for (int it = t; it < 128; it += blockDim.x) {   // (child, column) pairs
    const int c = it >> 4, col = it & 15;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      R in[8], o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) in[k] = Tc[c][(f * 8 + k) * NC_LD + col];
      interp_T<R>(c, in, o);
#pragma unroll
      for (int A = 0; A < 8; ++A) Jc[c][(f * 8 + A) * NC_LD + col] = o[A];
    }
  }
  __syncthreads();
  for (int idx = t; idx < 256; idx += blockDim.x) {
    const int r = idx >> 4, q = idx & 15;
    R acc = R(0);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) acc += Jc[cc][r * NC_LD + q];
    out[idx] = acc;
  }
}

// Columns of the element Jacobian per thread (block of 128 / CPT threads): the thread computes its
// child's Gauss-point state once for its CPT columns.
#ifndef NC_GALERKIN_CPT
#define NC_GALERKIN_CPT 4
#endif

// PIC: the element matrices of the frozen-coefficient operator (its u0 and tau from the same element
// state), columns by elem_picard_modal on unit directions; otherwise those of the exact J(s).
template <typename R, bool PIC>
__global__ void __launch_bounds__(128 / NC_GALERKIN_CPT) k_galerkin_fine(Grid gf, Grid gc, Phys ph, ElemConst<R> C,
                                                       const typename Vec2<R>::type* __restrict__ s,
                                                       const typename Vec2<R>::type* __restrict__ mat,
                                                       R* __restrict__ diag_f, R* __restrict__ ebe_c) {
  __shared__ R Jc[8][16 * NC_LD];
  __shared__ R Tc[8][16 * NC_LD];
  const long long E = blockIdx.x;
  int I, J, K;
  elem_ijk(gc, E, I, J, K);
  constexpr int kCols = 16 / NC_GALERKIN_CPT;   // threads per child
  const int t = threadIdx.x;
  const int c = t / kCols, col0 = t % kCols;
  const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
  R p[8], tt[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const typename Vec2<R>::type v = s[corner_node(gf, i, j, k, a)];
    p[a] = v.x;
    tt[a] = v.y;
  }
  const long long e = i + (long long)gf.nx * (j + (long long)gf.ny * k);
  const typename Vec2<R>::type m = mat[e];
  ElemState<R> st;
  elem_state(C, p, tt, m.x, elem_heated(ph, i, j, k) ? (R)ph.Q : R(0), st);
  for (int cc = 0; cc < NC_GALERKIN_CPT; ++cc) {
    const int col = col0 + cc * kCols;
    R oP[8], oT[8];
    if constexpr (PIC) {
      R dp[8], dt[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) { dp[q] = R(q == col ? 1 : 0); dt[q] = R(q + 8 == col ? 1 : 0); }
      elem_picard_modal<R, false>(C, st.c, m.y, st.u0x, st.u0y, st.u0z, st.tau, dp, dt, oP, oT);
    } else {
      elem_jac_column<R>(C, st, m.y, col, oP, oT);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      Jc[c][r * NC_LD + col] = oP[r];
      Jc[c][(8 + r) * NC_LD + col] = oT[r];
    }
    // block diagonal of level 0 (row-major [PP PT; TP TT]) on free nodes
    const int a = col & 7;
    if (gf.bc != kBcTop || k + (a >> 2) < gf.nz) {
      const long long n = corner_node(gf, i, j, k, a);
      if (col < 8) { add_diag_block(diag_f, n, 0, oP[a]); add_diag_block(diag_f, n, 2, oT[a]); }
      else { add_diag_block(diag_f, n, 1, oP[a]); add_diag_block(diag_f, n, 3, oT[a]); }
    }
  }
  __syncthreads();
  galerkin_phase2<R>(Jc, Tc, ebe_c + E * 256);
}

template <typename R>
__global__ void __launch_bounds__(128) k_galerkin_coarse(Grid gf, Grid gc, const R* __restrict__ ebe_f,
                                                         R* __restrict__ diag_f, R* __restrict__ ebe_c) {
  __shared__ R Jc[8][16 * NC_LD];
  __shared__ R Tc[8][16 * NC_LD];
  const long long E = blockIdx.x;
  int I, J, K;
  elem_ijk(gc, E, I, J, K);
  const int t = threadIdx.x;
  for (int idx = t; idx < 8 * 256; idx += 128) {
    const int c = idx >> 8, r = idx & 255;
    const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    const long long e = i + (long long)gf.nx * (j + (long long)gf.ny * k);
    Jc[c][(r >> 4) * NC_LD + (r & 15)] = ebe_f[e * 256 + r];
  }
  __syncthreads();
  if (t < 64) {
    const int c = t >> 3, a = t & 7;
    const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    if (gf.bc != kBcTop || k + (a >> 2) < gf.nz) {
      const long long n = corner_node(gf, i, j, k, a);
      add_diag_block(diag_f, n, 0, Jc[c][a * NC_LD + a]);
      add_diag_block(diag_f, n, 1, Jc[c][a * NC_LD + 8 + a]);
      add_diag_block(diag_f, n, 2, Jc[c][(8 + a) * NC_LD + a]);
      add_diag_block(diag_f, n, 3, Jc[c][(8 + a) * NC_LD + 8 + a]);
    }
  }
  __syncthreads();
  galerkin_phase2<R>(Jc, Tc, ebe_c + E * 256);
}

template <typename R>
__global__ void k_invert_diag(Grid g, R* __restrict__ diag, int* flag) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  R* d = diag + 4 * n;
  int i, j, k;
  node_ijk(g, n, i, j, k);
  const int fb = fixed_bits(g, i, j, k);
  if (fb == 3) { d[0] = d[1] = d[2] = d[3] = R(0); return; }
  if (fb) {   // one fixed component: invert the free one alone, zero rows and columns of the fixed one
    const R v = fb == 2 ? d[0] : d[3];
    if (!(v != R(0)) || !isfinite((double)v)) { atomicExch(flag, 1); d[0] = d[1] = d[2] = d[3] = R(0); return; }
    d[1] = d[2] = R(0);
    d[0] = fb == 2 ? R(1) / v : R(0);
    d[3] = fb == 2 ? R(0) : R(1) / v;
    return;
  }
  const R a = d[0], b = d[1], c = d[2], e = d[3];
  const R det = a * e - b * c;
  if (!(det != R(0)) || !isfinite((double)det)) { atomicExch(flag, 1); d[0] = d[1] = d[2] = d[3] = R(0); return; }
  const R id = R(1) / det;
  d[0] = e * id; d[1] = -b * id; d[2] = -c * id; d[3] = a * id;
}

template <typename R, bool TR>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 6 : 1) k_level0_apply(Grid g, Phys ph, ElemConst<R> C, const typename Vec2<R>::type* __restrict__ s,
                               const typename Vec2<R>::type* __restrict__ mat,
                               const typename Vec2<R>::type* __restrict__ x, R* __restrict__ y) {
  NC_IJK_3D();
  if (i >= g.nx || j >= g.ny) return;
  const int n0 = i + g.NX * j + g.NXY * k;
  const bool top = g.bc == kBcTop && (k + 1 == g.nz);
  R p[8], t[8], dp[8], dt[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int n = n0 + corner_off(g, a);
    const typename Vec2<R>::type v = s[n];
    p[a] = v.x; t[a] = v.y;
    if (top && (a >> 2)) { dp[a] = R(0); dt[a] = R(0); }
    else { const typename Vec2<R>::type w = x[n]; dp[a] = w.x; dt[a] = w.y; }
  }
  const typename Vec2<R>::type m = mat[i + g.nx * (j + g.ny * k)];
  ElemState<R> st;
  elem_state(C, p, t, m.x, elem_heated(ph, i, j, k) ? (R)ph.Q : R(0), st);
  R oP[8], oT[8];
  if (TR) elem_jtv<R, false>(C, st, m.y, dp, dt, oP, oT, nullptr, nullptr);
  else elem_jv_dir<R>(C, st, m.y, dp, dt, oP, oT);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (top && (a >> 2)) continue;
    const int n = n0 + corner_off(g, a);
    atomic_add_pair(y + 2 * n, oP[a], oT[a]);
  }
}

// Frozen coefficients of the Picard operator: centroid velocity u0 and tau of each element at the
// state s (the same element state as the exact operator), as (u0x, u0y, u0z, tau).
__global__ void k_frozen(Grid g, Phys ph, ElemConst<float> C, const float2* __restrict__ s,
                         const float2* __restrict__ mat, float4* __restrict__ fz) {
  NC_IJK_3D();
  if (i >= g.nx || j >= g.ny) return;
  const int n0 = i + g.NX * j + g.NXY * k;
  float p[8], t[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const float2 v = s[n0 + corner_off(g, a)];
    p[a] = v.x; t[a] = v.y;
  }
  const int e = i + g.nx * (j + g.ny * k);
  ElemState<float> st;
  elem_state(C, p, t, mat[e].x, 0.f, st);
  fz[e] = make_float4(st.u0x, st.u0y, st.u0z, st.tau);
}

// Frozen-coefficient (Picard) finest-level operator y = A x (TR: A^T x), FP32, one thread per element,
// the element operator applied in its modal basis (elem_picard_modal).
template <bool TR>
__global__ void __launch_bounds__(128, 12) k_level0_picard(Grid g, ElemConst<float> C, const float4* __restrict__ fz,
                                const float2* __restrict__ mat, const float2* __restrict__ x, float* __restrict__ y) {
  NC_IJK_3D();
  if (i >= g.nx || j >= g.ny) return;
  const int n0 = i + g.NX * j + g.NXY * k;
  const bool top = g.bc == kBcTop && (k + 1 == g.nz);
  float dp[8], dt[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (top && (a >> 2)) { dp[a] = 0.f; dt[a] = 0.f; }
    else { const float2 w = x[n0 + corner_off(g, a)]; dp[a] = w.x; dt[a] = w.y; }
  }
  const int e = i + g.nx * (j + g.ny * k);
  const float2 m = mat[e];
  const float4 f = fz[e];
  const float c = m.x * C.imu;
  float oP[8], oT[8];
  elem_picard_modal<float, TR>(C, c, m.y, f.x, f.y, f.z, f.w, dp, dt, oP, oT);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (top && (a >> 2)) continue;
    atomic_add_pair(y + 2 * (n0 + corner_off(g, a)), oP[a], oT[a]);
  }
}

// ---- finest-level operators, column-walking form (FP32) -----------------------------------------
// One thread per (i, j) column of elements walks KC elements up in z. The node plane an element
// shares with the one below is kept in registers: its 4 corner values (x, and the state s of the
// exact operator) are loaded once, and the contributions of both elements to its rows are summed in
// registers before they leave the thread. A plane leaves as the (i, j) and (i, j + 1) nodes of each
// lane, the x-neighbour's (i + 1) contributions added by a warp shuffle, so about 2 float2 atomic
// adds per element remain instead of 8. Warps are one row (fixed j) of 32 columns.
// MODE 0: the exact Jacobian J(s) (TR: J^T) at the state s; MODE 1: the frozen-coefficient operator.

// Adds the plane totals aP, aT (corners ax + 2 ay of this lane's column) into y at plane kp.
__device__ __forceinline__ void emit_plane(const Grid& g, float* __restrict__ y, int lane, int i, int j, int kp,
                                           const float aP[4], const float aT[4]) {
  const int base = i + g.NX * j + g.NXY * kp;
#pragma unroll
  for (int ay = 0; ay < 2; ++ay) {
    const float lP = __shfl_up_sync(0xffffffffu, aP[1 + 2 * ay], 1);
    const float lT = __shfl_up_sync(0xffffffffu, aT[1 + 2 * ay], 1);
    float vP = aP[2 * ay], vT = aT[2 * ay];
    if (lane > 0) { vP += lP; vT += lT; }
    const int n = base + ay * g.NX;
    if (i <= g.nx) atomic_add_pair(y + 2 * n, vP, vT);
    if (lane == 31 && i < g.nx) atomic_add_pair(y + 2 * (n + 1), aP[1 + 2 * ay], aT[1 + 2 * ay]);
  }
}

template <int MODE, bool TR, int KC>
__global__ void __launch_bounds__(128) k_level0_z(Grid g, Phys ph, ElemConst<float> C, const float2* __restrict__ s,
                                                  const float4* __restrict__ fz, const float2* __restrict__ mat,
                                                  const float2* __restrict__ x, float* __restrict__ y) {
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 32 + lane;
  const int j = blockIdx.y * 4 + threadIdx.y;
  if (j >= g.ny) return;                     // whole warps
  const bool act = i < g.nx;
  const int k0 = blockIdx.z * KC;
  const int k1 = min(k0 + KC, g.nz);
  const bool bctop = g.bc == kBcTop;
  const int col = i + g.NX * j;
  float dpb[4], dtb[4], pb[4], tb[4];         // bottom-plane corners (ax + 2 ay) of x and s
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    dpb[c] = dtb[c] = pb[c] = tb[c] = 0.f;
    if (act) {
      const int n = col + (c & 1) + (c >> 1) * g.NX + k0 * g.NXY;
      const float2 w = x[n];
      dpb[c] = w.x; dtb[c] = w.y;
      if (MODE == 0) { const float2 v = s[n]; pb[c] = v.x; tb[c] = v.y; }
    }
  }
  float aP[4] = {0.f, 0.f, 0.f, 0.f}, aT[4] = {0.f, 0.f, 0.f, 0.f};   // the element below's share of the bottom plane
  for (int k = k0; k < k1; ++k) {
    float dp[8], dt[8], oP[8], oT[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) { dp[c] = dpb[c]; dt[c] = dtb[c]; }
    const bool topx = bctop && k + 1 == g.nz;   // Dirichlet plane above: direction entries are 0 there
    float p[8], t[8];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      dp[4 + c] = dt[4 + c] = 0.f;
      p[4 + c] = t[4 + c] = 0.f;
      p[c] = pb[c]; t[c] = tb[c];
      if (act) {
        const int n = col + (c & 1) + (c >> 1) * g.NX + (k + 1) * g.NXY;
        if (!topx) { const float2 w = x[n]; dp[4 + c] = w.x; dt[4 + c] = w.y; }
        if (MODE == 0) { const float2 v = s[n]; p[4 + c] = v.x; t[4 + c] = v.y; }
      }
    }
    if (act) {
      const int e = i + g.nx * (j + g.ny * k);
      const float2 m = mat[e];
      if (MODE == 0) {
        ElemState<float> st;
        elem_state(C, p, t, m.x, elem_heated(ph, i, j, k) ? (float)ph.Q : 0.f, st);
        if (TR) elem_jtv<float, false>(C, st, m.y, dp, dt, oP, oT, nullptr, nullptr);
        else elem_jv_dir<float>(C, st, m.y, dp, dt, oP, oT);
      } else {
        const float4 f = fz[e];
        const float c = m.x * C.imu;
        elem_picard_modal<float, TR>(C, c, m.y, f.x, f.y, f.z, f.w, dp, dt, oP, oT);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a) { oP[a] = 0.f; oT[a] = 0.f; }
    }
    float tP[4], tT[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { tP[c] = aP[c] + oP[c]; tT[c] = aT[c] + oT[c]; }
    emit_plane(g, y, lane, i, j, k, tP, tT);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      aP[c] = oP[4 + c]; aT[c] = oT[4 + c];
      dpb[c] = dp[4 + c]; dtb[c] = dt[4 + c];
      pb[c] = p[4 + c]; tb[c] = t[4 + c];
    }
  }
  if (!(bctop && k1 == g.nz)) emit_plane(g, y, lane, i, j, k1, aP, aT);
}

template <int MODE, bool TR>
static void launch_level0_z(const Grid& g, const Phys& ph, const float2* s, const float4* fz, const float2* mat,
                            const float2* x, float* y, int kc, cudaStream_t st) {
  const dim3 block(32, 4, 1);
  const unsigned gx = (unsigned)((g.nx + 31) / 32), gy = (unsigned)((g.ny + 3) / 4);
  const ElemConst<float> C = make_econst<float>(ph);
#define NC_L0Z(KC) k_level0_z<MODE, TR, KC><<<dim3(gx, gy, (unsigned)((g.nz + KC - 1) / KC)), block, 0, st>>>(g, ph, C, s, fz, mat, x, y)
  switch (kc) {
    case 1: NC_L0Z(1); break;
    case 2: NC_L0Z(2); break;
    case 8: NC_L0Z(8); break;
    case 16: NC_L0Z(16); break;
    default: NC_L0Z(4); break;
  }
#undef NC_L0Z
}

// Elements per thread along z of the column-walking kernels (nc_params.elem_chunk >= 0): 0 picks 4.
static int level0_kc(int requested) { return requested > 0 ? requested : 4; }

template <typename R, bool TR, bool FIRST>
__global__ void k_jacobi(long long nn, const R* __restrict__ dinv, const typename Vec2<R>::type* __restrict__ b,
                         const typename Vec2<R>::type* __restrict__ y, const typename Vec2<R>::type* __restrict__ x,
                         typename Vec2<R>::type* __restrict__ xn, R omega) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const typename Vec2<R>::type bb = b[n];
  R r0 = bb.x, r1 = bb.y;
  R x0 = R(0), x1 = R(0);
  if (!FIRST) {
    const typename Vec2<R>::type yy = y[n];
    const typename Vec2<R>::type xx = x[n];
    r0 -= yy.x; r1 -= yy.y;
    x0 = xx.x; x1 = xx.y;
  }
  const R* d = dinv + 4 * n;
  R z0, z1;
  if (TR) { z0 = d[0] * r0 + d[2] * r1; z1 = d[1] * r0 + d[3] * r1; }
  else { z0 = d[0] * r0 + d[1] * r1; z1 = d[2] * r0 + d[3] * r1; }
  xn[n] = mk2<R>(x0 + omega * z0, x1 + omega * z1);
}

// The same update at the finest level of a preconditioner call, reading and writing the caller's FP64
// vectors directly: FIRST takes b from b64 (and keeps its R copy in b for the later sweeps); z64
// (nullable) receives the new x in FP64 as well.
template <typename R, bool TR, bool FIRST>
__global__ void k_jacobi_io(long long nn, const R* __restrict__ dinv, typename Vec2<R>::type* __restrict__ b,
                            const double2* __restrict__ b64, const typename Vec2<R>::type* __restrict__ y,
                            const typename Vec2<R>::type* __restrict__ x, typename Vec2<R>::type* __restrict__ xn,
                            double2* __restrict__ z64, R omega) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  R r0, r1;
  if (FIRST) {
    const double2 v = b64[n];
    r0 = (R)v.x; r1 = (R)v.y;
    b[n] = mk2<R>(r0, r1);
  } else {
    const typename Vec2<R>::type bb = b[n];
    r0 = bb.x; r1 = bb.y;
  }
  R x0 = R(0), x1 = R(0);
  if (!FIRST) {
    const typename Vec2<R>::type yy = y[n];
    const typename Vec2<R>::type xx = x[n];
    r0 -= yy.x; r1 -= yy.y;
    x0 = xx.x; x1 = xx.y;
  }
  const R* d = dinv + 4 * n;
  R z0, z1;
  if (TR) { z0 = d[0] * r0 + d[2] * r1; z1 = d[1] * r0 + d[3] * r1; }
  else { z0 = d[0] * r0 + d[1] * r1; z1 = d[2] * r0 + d[3] * r1; }
  const R o0 = x0 + omega * z0, o1 = x1 + omega * z1;
  xn[n] = mk2<R>(o0, o1);
  if (z64) z64[n] = make_double2((double)o0, (double)o1);
}

// The value v at node (i, j, k) with its fixed components set to zero.
template <typename R>
__device__ __forceinline__ typename Vec2<R>::type mask_fixed(const Grid& g, int i, int j, int k,
                                                             typename Vec2<R>::type v) {
  const int b = fixed_bits(g, i, j, k);
  if (b & 1) v.x = R(0);
  if (b & 2) v.y = R(0);
  return v;
}

// Full weighting (R = P^T) at coarse node (I, J, K): the fine residual rf at the 27 fine nodes
// around it, weights 1, 1/2, 1/4, 1/8 by distance; `top` (the kBcTop Dirichlet plane) gets 0, and the
// callers zero the fixed components of other boundary conditions (mask_fixed).
template <typename R, typename FETCH>
__device__ __forceinline__ typename Vec2<R>::type restrict_node_f(const Grid& gf, int I, int J, int K, bool top,
                                                                  FETCH fetch) {
  R a0 = R(0), a1 = R(0);
  if (!top) {
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      const int k = 2 * K + dk;
      if (k < 0 || k > gf.nz) continue;
      const R wk = dk ? R(0.5) : R(1);
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        const int j = 2 * J + dj;
        if (j < 0 || j > gf.ny) continue;
        const R wj = wk * (dj ? R(0.5) : R(1));
        const int row = gf.NX * j + gf.NXY * k;
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const int i = 2 * I + di;
          if (i < 0 || i > gf.nx) continue;
          const R w = wj * (di ? R(0.5) : R(1));
          const typename Vec2<R>::type v = fetch(row + i);
          a0 += w * v.x;
          a1 += w * v.y;
        }
      }
    }
  }
  return mk2<R>(a0, a1);
}

template <typename R, typename LD>
__device__ __forceinline__ typename Vec2<R>::type restrict_node(const Grid& gf, const typename Vec2<R>::type* rf,
                                                                int I, int J, int K, bool top, LD ld) {
  return restrict_node_f<R>(gf, I, J, K, top, [&](int m) { return ld(rf + m); });
}

// Optional first pre-smoothing sweep of the coarse level, fused into the restriction that produces
// its right-hand side: the block-Jacobi sweep from x = 0, x_c = omega D_c^-1 b_c (SW = 1), or with
// D_c^-T for the transposed hierarchy (SW = 2); SW = 0 stores b_c only.
template <typename R> struct FirstSweep {
  const R* dinv;
  typename Vec2<R>::type* x;
  R omega;
};

template <typename R, int SW>
__device__ __forceinline__ void store_restricted(int n, typename Vec2<R>::type v, typename Vec2<R>::type* bc,
                                                 const FirstSweep<R>& fs) {
  bc[n] = v;
  if (SW) {
    const R* d = fs.dinv + 4 * n;
    R z0, z1;
    if (SW == 2) { z0 = d[0] * v.x + d[2] * v.y; z1 = d[1] * v.x + d[3] * v.y; }
    else { z0 = d[0] * v.x + d[1] * v.y; z1 = d[2] * v.x + d[3] * v.y; }
    fs.x[n] = mk2<R>(fs.omega * z0, fs.omega * z1);
  }
}

// Full weighting of the fine residual r = b - y formed on the fly (no stored residual vector).
template <typename R, int SW>
__global__ void k_restrict_res(Grid gf, Grid gc, const typename Vec2<R>::type* __restrict__ b,
                               const typename Vec2<R>::type* __restrict__ y, typename Vec2<R>::type* __restrict__ bc,
                               FirstSweep<R> fs) {
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (pidx >= gc.NXY) return;
  const int K = blockIdx.y;
  const int J = pidx / gc.NX;
  const int I = pidx - J * gc.NX;
  store_restricted<R, SW>(pidx + gc.NXY * K, mask_fixed<R>(gc, I, J, K, restrict_node_f<R>(gf, I, J, K, gc.bc == kBcTop && K >= gc.nz, [&](int m) {
    const typename Vec2<R>::type bb = b[m], yy = y[m];
    return mk2<R>(bb.x - yy.x, bb.y - yy.y);
  })), bc, fs);
}

template <typename R, int SW>
__global__ void k_restrict(Grid gf, Grid gc, const typename Vec2<R>::type* __restrict__ rf,
                           typename Vec2<R>::type* __restrict__ bc, FirstSweep<R> fs) {
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (pidx >= gc.NXY) return;
  const int K = blockIdx.y;
  const int J = pidx / gc.NX;
  const int I = pidx - J * gc.NX;
  store_restricted<R, SW>(pidx + gc.NXY * K,
      mask_fixed<R>(gc, I, J, K, restrict_node<R>(gf, rf, I, J, K, gc.bc == kBcTop && K >= gc.nz, LdPlain())), bc, fs);
}

// Trilinear interpolation of the coarse correction at fine node (i, j, k), added to xf.
template <typename R, typename LD>
__device__ __forceinline__ void prolong_node(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* xc,
                                             typename Vec2<R>::type* xf, int n, int i, int j, int k, LD ld) {
  const int ci = i >> 1, cj = j >> 1, ck = k >> 1;
  const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
  const R wi = (i & 1) ? R(0.5) : R(1), wj = (j & 1) ? R(0.5) : R(1), wk = (k & 1) ? R(0.5) : R(1);
  const R w = wi * wj * wk;
  R a0 = R(0), a1 = R(0);
  for (int c = 0; c < nk; ++c)
    for (int b = 0; b < nj; ++b) {
      const int row = gc.NX * (cj + b) + gc.NXY * (ck + c) + ci;
      for (int a = 0; a < ni; ++a) {
        const typename Vec2<R>::type v = ld(xc + row + a);
        a0 += v.x;
        a1 += v.y;
      }
    }
  typename Vec2<R>::type o = ld(xf + n);
  o.x += w * a0;
  o.y += w * a1;
  xf[n] = o;
}

template <typename R>
__global__ void k_prolong_add(Grid gf, Grid gc, const typename Vec2<R>::type* __restrict__ xc,
                              typename Vec2<R>::type* __restrict__ xf) {
  NC_NODE_FLAT(gf);
  if (fixed_bits(gf, i, j, k) == 3) return;   // a partly fixed node receives zero in its fixed component
  prolong_node<R>(gf, gc, xc, xf, pidx + gf.NXY * k, i, j, k, LdPlain());
}

template <typename R>
__global__ void k_dense_assemble(Grid g, const R* __restrict__ ebe, double* __restrict__ A, int nf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ne * 256) return;
  const long long e = t >> 8;
  const int r = (int)(t & 255) >> 4, q = (int)(t & 15);
  int i, j, k;
  elem_ijk(g, e, i, j, k);
  const int ar = r & 7, aq = q & 7;
  if ((fixed_bits(g, i + (ar & 1), j + ((ar >> 1) & 1), k + (ar >> 2)) >> (r >> 3)) & 1) return;
  if ((fixed_bits(g, i + (aq & 1), j + ((aq >> 1) & 1), k + (aq >> 2)) >> (q >> 3)) & 1) return;
  const long long row = 2 * corner_node(g, i, j, k, ar) + (r >> 3);
  const long long col = 2 * corner_node(g, i, j, k, aq) + (q >> 3);
  atomicAdd(A + row * nf + col, (double)ebe[t]);
}

// Identity rows for the fixed components of a level whose dense system keeps every node (kBcCavity).
__global__ void k_dense_fixed_rows(Grid g, double* __restrict__ A, int nf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!boundary_node(g, t, i, j, k)) return;
  const int b = fixed_bits(g, i, j, k);
  const long long n = i + (long long)g.NX * (j + (long long)g.NY * k);
  for (int f = 0; f < 2; ++f)
    if ((b >> f) & 1) {
      const long long r = 2 * n + f;
      if (r < nf) A[r * nf + r] = 1.0;
    }
}

template <typename R>
__global__ void k_from_mg(const typename Vec2<R>::type* __restrict__ x, double2* __restrict__ z, long long nn) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const typename Vec2<R>::type a = x[n];
  z[n] = make_double2((double)a.x, (double)a.y);
}


// ---- assembled 27-point block stencils of the coarse levels ----------------------------------
// Slot of offset (oi,oj,ok) in {-1,0,1}^3 and block entry (f,g): ((o * 4) + 2 f + g), o = (oi+1) +
// 3 (oj+1) + 9 (ok+1). Storage: one 2x2 block per (offset, node), blocks of an offset contiguous over
// the nodes: S[(o * nn + node) * 4 + 2 f + g] (27 planes of 4-vectors; a warp's loads of one offset
// are contiguous 16-byte vectors).

template <typename R>
__global__ void k_stencil_build(Grid g, const R* __restrict__ ebe, R* __restrict__ S) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nn * 27) return;
  const int o = (int)(t % 27);
  const long long n = t / 27;
  int i, j, k;
  node_ijk(g, n, i, j, k);
  const int oi = o % 3 - 1, oj = (o / 3) % 3 - 1, ok = o / 9 - 1;
  const int mi = i + oi, mj = j + oj, mk = k + ok;
  R acc[4] = {R(0), R(0), R(0), R(0)};
  const bool valid = mi >= 0 && mi <= g.nx && mj >= 0 && mj <= g.ny && mk >= 0 && mk <= g.nz;
  if (valid) {
    // elements containing both node (i,j,k) and node (mi,mj,mk)
    const int ei0 = oi ? min(i, mi) : i - 1, ei1 = oi ? min(i, mi) : i;
    const int ej0 = oj ? min(j, mj) : j - 1, ej1 = oj ? min(j, mj) : j;
    const int ek0 = ok ? min(k, mk) : k - 1, ek1 = ok ? min(k, mk) : k;
    for (int ek = ek0; ek <= ek1; ++ek) {
      if (ek < 0 || ek >= g.nz) continue;
      for (int ej = ej0; ej <= ej1; ++ej) {
        if (ej < 0 || ej >= g.ny) continue;
        for (int ei = ei0; ei <= ei1; ++ei) {
          if (ei < 0 || ei >= g.nx) continue;
          const long long e = ei + (long long)g.nx * (ej + (long long)g.ny * ek);
          const int a = (i - ei) + 2 * (j - ej) + 4 * (k - ek);
          const int b = (mi - ei) + 2 * (mj - ej) + 4 * (mk - ek);
          const R* A = ebe + e * 256;
          acc[0] += A[a * 16 + b];
          acc[1] += A[a * 16 + 8 + b];
          acc[2] += A[(8 + a) * 16 + b];
          acc[3] += A[(8 + a) * 16 + 8 + b];
        }
      }
    }
    // Dirichlet rows and columns stay zero, per component (entry (f, c): row field f, column field c)
    const int rb = fixed_bits(g, i, j, k), cb = fixed_bits(g, mi, mj, mk);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (((rb >> (q >> 1)) & 1) || ((cb >> (q & 1)) & 1)) acc[q] = R(0);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) S[((long long)o * g.nn + n) * 4 + q] = acc[q];
}

// One 2x2 stencil block (entries (0,0), (0,1), (1,0), (1,1)); read-only data.
template <typename R> struct Blk4 { R a00, a01, a10, a11; };
__device__ __forceinline__ Blk4<float> ld_blk(const float* __restrict__ S, int idx) {
  const float4 v = reinterpret_cast<const float4*>(S)[idx];
  return Blk4<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Blk4<double> ld_blk(const double* __restrict__ S, int idx) {
  const double2 u = reinterpret_cast<const double2*>(S)[2 * idx];
  const double2 v = reinterpret_cast<const double2*>(S)[2 * idx + 1];
  return Blk4<double>{u.x, u.y, v.x, v.y};
}

// y = A x (MODE 0), r = b - A x (MODE 1) or x_new = x + omega D^-1 (b - A x) (MODE 2), with A the
// assembled stencil or (TR) its transpose, at node n = (i, j, k) (below the top plane for kBcTop): gathers the
// 27 neighbours. A neighbour outside the grid is read at the node itself (always in range) and its
// value replaced by zero, so the loop has no branches and all 54 loads can be in flight together.
// S and dinv are read-only; x and b go through the load policy.
template <typename R, bool TR, int MODE, typename LD>
__device__ __forceinline__ void stencil_node(const Grid& g, const R* __restrict__ S,
                                             const typename Vec2<R>::type* x, const typename Vec2<R>::type* b,
                                             const R* __restrict__ dinv, R omega, typename Vec2<R>::type* out,
                                             int n, int i, int j, int k, LD ld) {
  const int nn = (int)g.nn;
  typename Vec2<R>::type xv[27];
  Blk4<R> c[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int oi = o % 3 - 1, oj = (o / 3) % 3 - 1, ok = o / 9 - 1;
    const bool inside = !((oi < 0 && i == 0) || (oi > 0 && i == g.nx) || (oj < 0 && j == 0) ||
                          (oj > 0 && j == g.ny) || (ok < 0 && k == 0) || (ok > 0 && k == g.nz));
    const int m = inside ? n + oi + g.NX * oj + g.NXY * ok : n;
    xv[o] = ld(x + m);
    c[o] = TR ? ld_blk(S, (26 - o) * nn + m) : ld_blk(S, o * nn + n);   // TR: offset -o seen from m
    if (!inside) { xv[o].x = R(0); xv[o].y = R(0); }
  }
  R y0 = R(0), y1 = R(0);
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    if (!TR) {
      y0 += c[o].a00 * xv[o].x + c[o].a01 * xv[o].y;
      y1 += c[o].a10 * xv[o].x + c[o].a11 * xv[o].y;
    } else {
      y0 += c[o].a00 * xv[o].x + c[o].a10 * xv[o].y;
      y1 += c[o].a01 * xv[o].x + c[o].a11 * xv[o].y;
    }
  }
  if (MODE == 0) { out[n] = mk2<R>(y0, y1); return; }
  const typename Vec2<R>::type bb = ld(b + n);
  const R r0 = bb.x - y0, r1 = bb.y - y1;
  if (MODE == 1) { out[n] = mk2<R>(r0, r1); return; }
  const R* d = dinv + 4 * n;
  R z0, z1;
  if (TR) { z0 = d[0] * r0 + d[2] * r1; z1 = d[1] * r0 + d[3] * r1; }
  else { z0 = d[0] * r0 + d[1] * r1; z1 = d[2] * r0 + d[3] * r1; }
  const typename Vec2<R>::type xs = ld(x + n);
  out[n] = mk2<R>(xs.x + omega * z0, xs.y + omega * z1);
}

// One thread per node (flat z-plane launch); with kBcTop the top (Dirichlet) plane gets 0, otherwise the
// zero stencil rows and block inverses of fixed components keep them at zero.
template <typename R, bool TR, int MODE>
__global__ void __launch_bounds__(128) k_stencil_apply(Grid g, const R* __restrict__ S,
                                                       const typename Vec2<R>::type* __restrict__ x,
                                                       const typename Vec2<R>::type* __restrict__ b,
                                                       const R* __restrict__ dinv, R omega,
                                                       typename Vec2<R>::type* __restrict__ out) {
  NC_NODE_FLAT(g);
  const int n = pidx + g.NXY * k;
  if (g.bc == kBcTop && k == g.nz) { out[n] = mk2<R>(R(0), R(0)); return; }
  stencil_node<R, TR, MODE>(g, S, x, b, dinv, omega, out, n, i, j, k, LdPlain());
}

// ---- z-line block-Jacobi smoother (levels with an assembled stencil) -----------------------------
// The couplings of a node column (i, j, k = 0 .. nz) with itself form a block-tridiagonal matrix
// T = tridiag(L_k, D_k, U_k) of 2x2 blocks: D_k is the stencil's centre block, L_k its (0,0,-1) block
// and U_k its (0,0,+1) block (transposed operator: D_k^T, L_k = U_{k-1}^T, U_k = L_{k+1}^T). The
// smoother uses T where block Jacobi uses D, every column from the same x:
// x <- x + omega T^-1 (b - A x). The set-up eliminates down each column, without pivoting between
// nodes: E_0 = D_0, E_k = D_k - L_k G_{k-1}, G_k = E_k^-1 U_k. LF holds, per direction, E_k^-1, G_k
// and M_k = E_k^-1 L_k as three planes of 2x2 blocks (12 nn values). The solve is the pair of
// first-order recurrences y_k = E_k^-1 r_k - M_k y_{k-1} (down the column) and d_k = y_k - G_k d_{k+1}
// (back up). Fixed components have zero rows and columns in every block, and E_k is inverted on its
// free components only, so they stay zero.

template <typename R> __device__ __forceinline__ Blk4<R> blk_mul(const Blk4<R>& a, const Blk4<R>& b) {
  return Blk4<R>{a.a00 * b.a00 + a.a01 * b.a10, a.a00 * b.a01 + a.a01 * b.a11,
                 a.a10 * b.a00 + a.a11 * b.a10, a.a10 * b.a01 + a.a11 * b.a11};
}
template <typename R> __device__ __forceinline__ Blk4<R> blk_t(const Blk4<R>& a) {
  return Blk4<R>{a.a00, a.a10, a.a01, a.a11};
}
__device__ __forceinline__ void st_blk(float* P, long long idx, const Blk4<float>& b) {
  reinterpret_cast<float4*>(P)[idx] = make_float4(b.a00, b.a01, b.a10, b.a11);
}
__device__ __forceinline__ void st_blk(double* P, long long idx, const Blk4<double>& b) {
  reinterpret_cast<double2*>(P)[2 * idx] = make_double2(b.a00, b.a01);
  reinterpret_cast<double2*>(P)[2 * idx + 1] = make_double2(b.a10, b.a11);
}

// Inverse of the free components of a 2x2 block (fb: fixed bits, bit 0 P, bit 1 T); the rows and
// columns of fixed components are zero. False on a singular or non-finite block.
template <typename R> __device__ __forceinline__ bool blk_inv_free(const Blk4<R>& a, int fb, Blk4<R>& o) {
  o = Blk4<R>{R(0), R(0), R(0), R(0)};
  if (fb == 3) return true;
  if (fb) {
    const R v = fb == 2 ? a.a00 : a.a11;
    if (!(v != R(0)) || !isfinite((double)v)) return false;
    if (fb == 2) o.a00 = R(1) / v; else o.a11 = R(1) / v;
    return true;
  }
  const R det = a.a00 * a.a11 - a.a01 * a.a10;
  if (!(det != R(0)) || !isfinite((double)det)) return false;
  const R id = R(1) / det;
  o = Blk4<R>{a.a11 * id, -a.a01 * id, -a.a10 * id, a.a00 * id};
  return true;
}

// One thread per node column c = i + NX j.
template <typename R, bool TR>
__global__ void __launch_bounds__(32) k_line_factor(Grid g, const R* __restrict__ S, R* __restrict__ LF,
                                                    int* __restrict__ flag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.NXY) return;
  const int nn = (int)g.nn, i = c % g.NX, j = c / g.NX;
  const Blk4<R> zero{R(0), R(0), R(0), R(0)};
  Blk4<R> G = zero;
  bool bad = false;
  for (int k = 0; k <= g.nz; ++k) {
    const int n = c + g.NXY * k;
    Blk4<R> D = ld_blk(S, 13 * nn + n);
    if (TR) D = blk_t(D);
    Blk4<R> L = zero;
    if (k > 0) {
      L = TR ? blk_t(ld_blk(S, 22 * nn + n - g.NXY)) : ld_blk(S, 4 * nn + n);
      const Blk4<R> LG = blk_mul(L, G);
      D = Blk4<R>{D.a00 - LG.a00, D.a01 - LG.a01, D.a10 - LG.a10, D.a11 - LG.a11};
    }
    Blk4<R> Ei;
    if (!blk_inv_free(D, fixed_bits(g, i, j, k), Ei)) bad = true;
    Blk4<R> U = zero;
    if (k < g.nz) U = TR ? blk_t(ld_blk(S, 4 * nn + n + g.NXY)) : ld_blk(S, 22 * nn + n);
    G = blk_mul(Ei, U);
    st_blk(LF, n, Ei);
    st_blk(LF, (long long)nn + n, G);
    st_blk(LF, 2LL * nn + n, blk_mul(Ei, L));
  }
  if (bad) atomicExch(flag, 1);
}

// Inclusive scan over the warp's lanes of affine maps v -> a + B v (2x2 B), composed in lane order:
// lane q ends with the composition of the maps of lanes q, q-1, ..., 0 (lane 0's applied first).
template <typename R>
__device__ __forceinline__ void warp_scan_affine(R& b00, R& b01, R& b10, R& b11, R& a0, R& a1, int lane) {
  constexpr unsigned kFull = 0xffffffffu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R p00 = __shfl_up_sync(kFull, b00, off), p01 = __shfl_up_sync(kFull, b01, off);
    const R p10 = __shfl_up_sync(kFull, b10, off), p11 = __shfl_up_sync(kFull, b11, off);
    const R q0 = __shfl_up_sync(kFull, a0, off), q1 = __shfl_up_sync(kFull, a1, off);
    if (lane >= off) {
      const R n0 = a0 + b00 * q0 + b01 * q1, n1 = a1 + b10 * q0 + b11 * q1;
      const R m00 = b00 * p00 + b01 * p10, m01 = b00 * p01 + b01 * p11;
      const R m10 = b10 * p00 + b11 * p10, m11 = b10 * p01 + b11 * p11;
      a0 = n0; a1 = n1; b00 = m00; b01 = m01; b10 = m10; b11 = m11;
    }
  }
}

// x <- x + omega T^-1 r (FIRST: x <- omega T^-1 r from x = 0). One warp per column, 32 nodes of it
// at a time, one per lane: each recurrence step is an affine map of the previous value, so a chunk is
// one warp scan of those maps, applied to the value carried in from the chunk before; the next
// chunk's loads are issued before the current chunk's scan. The forward values y_k go to ybuf (x when
// FIRST, otherwise r itself, which the caller no longer needs).
template <typename R, bool FIRST>
__global__ void __launch_bounds__(128) k_line_smooth(Grid g, const R* __restrict__ LF, const typename Vec2<R>::type* r,
                                                     typename Vec2<R>::type* ybuf, typename Vec2<R>::type* x,
                                                     R omega) {
  typedef typename Vec2<R>::type V2;
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= g.NXY) return;   // uniform over the warp
  const int nn = (int)g.nn, K = g.nz + 1, P = g.NXY;
  // down the column: lane q of the chunk at k0 takes node k0 + q (past the top: the top node, unused)
  R c0 = R(0), c1 = R(0);
  int n = c + P * min(lane, K - 1);
  Blk4<R> E = ld_blk(LF, n), M = ld_blk(LF, 2 * nn + n);
  V2 rv = r[n];
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int nx = c + P * min(k0 + 32 + lane, K - 1);
    Blk4<R> En = E, Mn = M;
    V2 rn = rv;
    if (k0 + 32 < K) { En = ld_blk(LF, nx); Mn = ld_blk(LF, 2 * nn + nx); rn = r[nx]; }
    R a0 = E.a00 * rv.x + E.a01 * rv.y, a1 = E.a10 * rv.x + E.a11 * rv.y;
    R b00 = -M.a00, b01 = -M.a01, b10 = -M.a10, b11 = -M.a11;
    warp_scan_affine(b00, b01, b10, b11, a0, a1, lane);
    const R y0 = a0 + b00 * c0 + b01 * c1, y1 = a1 + b10 * c0 + b11 * c1;
    if (k0 + lane < K) ybuf[n] = mk2<R>(y0, y1);
    c0 = __shfl_sync(kFull, y0, 31);
    c1 = __shfl_sync(kFull, y1, 31);
    n = nx; E = En; M = Mn; rv = rn;
  }
  // back up the column: lane q of the chunk at k1 takes node k1 - q (below the bottom: node 0, unused)
  c0 = R(0); c1 = R(0);
  n = c + P * max(K - 1 - lane, 0);
  Blk4<R> G = ld_blk(LF, nn + n);
  V2 yv = ybuf[n], xv = yv;
  if (!FIRST) xv = x[n];
  for (int k1 = K - 1; k1 >= 0; k1 -= 32) {
    const int nx = c + P * max(k1 - 32 - lane, 0);
    Blk4<R> Gn = G;
    V2 yn = yv, xn = yv;
    if (k1 - 32 >= 0) { Gn = ld_blk(LF, nn + nx); yn = ybuf[nx]; if (!FIRST) xn = x[nx]; }
    R a0 = yv.x, a1 = yv.y;
    R b00 = -G.a00, b01 = -G.a01, b10 = -G.a10, b11 = -G.a11;
    warp_scan_affine(b00, b01, b10, b11, a0, a1, lane);
    const R d0 = a0 + b00 * c0 + b01 * c1, d1 = a1 + b10 * c0 + b11 * c1;
    if (k1 - lane >= 0) x[n] = FIRST ? mk2<R>(omega * d0, omega * d1) : mk2<R>(xv.x + omega * d0, xv.y + omega * d1);
    c0 = __shfl_sync(kFull, d0, 31);
    c1 = __shfl_sync(kFull, d1, 31);
    n = nx; G = Gn; yv = yn;
    if (!FIRST) xv = xn;
  }
}

// ---- coarsest level: FP32 Gauss-Jordan inverse with partial pivoting ----------------------------
// Ainv32 receives the inverse of the FP64 matrix A rounded to FP32; flag = 1 on a zero pivot.

// Gauss-Jordan inversion with partial pivoting for coarse matrices too large for one block's shared
// memory (FP32), spread over the whole GPU with one launch pair per column and no block waiting on
// another. W = [A | I] (nf x 2nf, global memory). Step k: the pivot kernel (one block) picks the row p
// not yet used as a pivot with the largest |W[p][k]| (partial pivoting without row exchanges; ties to
// the lower row), records the multipliers m_r = W[r][k] of the other rows and scales row p by
// 1 / W[p][k]; the update kernel subtracts m_r times row p from every other row r. Columns left of k
// are zero outside the earlier pivot rows, so the update starts at column k. After nf steps the left
// half is the permutation with a 1 at (piv[k], k), the right half is that permutation times A^-1, and
// row k of A^-1 is row piv[k] of the right half.
__global__ void k_gjm_init(const double* __restrict__ A, float* __restrict__ W, int nf, int* __restrict__ used) {
  const long long w2 = 2LL * nf;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nf * w2;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / w2), c = (int)(idx % w2);
    W[idx] = c < nf ? (float)A[(long long)r * nf + c] : (c - nf == r ? 1.f : 0.f);
    if (idx < nf) used[idx] = 0;
  }
}

__global__ void __launch_bounds__(1024) k_gjm_pivot(float* __restrict__ W, int nf, int k, int* __restrict__ piv,
                                                    int* __restrict__ used, float* __restrict__ m, int* flag) {
  __shared__ float s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  const int t = threadIdx.x, nt = blockDim.x;
  const long long w2 = 2LL * nf;
  float best = -1.f;
  int bi = nf;
  for (int r = t; r < nf; r += nt) {
    if (used[r]) continue;
    const float v = fabsf(W[r * w2 + k]);
    if (v > best || (v == best && r < bi)) { best = v; bi = r; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if ((t & 31) == 0) { s_val[t >> 5] = best; s_idx[t >> 5] = bi; }
  __syncthreads();
  if (t == 0) {
    float bb = -1.f;
    int bidx = nf;
    for (int w = 0; w < (nt >> 5); ++w)
      if (s_val[w] > bb || (s_val[w] == bb && s_idx[w] < bidx)) { bb = s_val[w]; bidx = s_idx[w]; }
    const bool ok = bb > 0.f && isfinite(bb) && bidx < nf;
    s_piv = ok ? bidx : -1;
    piv[k] = s_piv;
    if (ok) used[bidx] = 1;
    else atomicExch(flag, 1);
  }
  __syncthreads();
  const int p = s_piv;
  if (p < 0) return;
  for (int r = t; r < nf; r += nt) m[r] = r == p ? 0.f : W[r * w2 + k];
  const float inv = 1.f / W[p * w2 + k];
  __syncthreads();   // every thread has read W[p][k] before row p is scaled
  for (long long c = k + t; c < w2; c += nt) W[p * w2 + c] *= inv;
}

__global__ void k_gjm_update(float* __restrict__ W, int nf, int k, const int* __restrict__ piv,
                             const float* __restrict__ m) {
  const int p = piv[k];
  const int r = blockIdx.y;
  if (p < 0 || r == p) return;
  const float mr = m[r];
  if (mr == 0.f) return;
  const long long w2 = 2LL * nf;
  for (long long c = k + (long long)blockIdx.x * blockDim.x + threadIdx.x; c < w2;
       c += (long long)gridDim.x * blockDim.x)
    W[r * w2 + c] -= mr * W[p * w2 + c];
}

__global__ void k_gjm_permute(const float* __restrict__ W, int nf, const int* __restrict__ piv,
                              float* __restrict__ Ainv32) {
  const long long w2 = 2LL * nf;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)nf * nf;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / nf), c = (int)(idx % nf);
    const int p = piv[k];
    Ainv32[idx] = p >= 0 ? W[p * w2 + nf + c] : 0.f;
  }
}

// In-place Gauss-Jordan inversion with partial pivoting held in registers (FP32, nf <= 224): one block
// of 16 x 32 threads; thread (ty, tx) holds M[r][c] for the rows r = ty + 16 a (a < RA) and columns
// c = tx + 32 b (b < CB). Pivoting is implicit (no row exchange): step k takes as pivot the row p, not
// yet used, with the largest |M[p][k]| (ties to the lower row), forms the pivot row
// prow = M[p] / d with prow[k] = 1 / d (d = M[p][k]), sets M[i][k] = 0 and subtracts
// M_old[i][k] prow from every other row i, and stores prow as row p. Each warp reads its rows'
// column-k values from lane k mod 32 by a shuffle; the pivot candidates (one per warp) and the pivot
// row pass through double-buffered shared memory, so a step needs two barriers. With p_k the pivot of
// step k and q its inverse permutation, the result M satisfies A^-1[q[r]][p_c] = M[r][c].
// One elimination step of k_gj32_reg for column k = 32 KB + kl (KB a compile-time column block, so
// every register access below has a constant index). Returns false if no usable pivot is left.
template <int RA, int CB, int KB>
__device__ __forceinline__ bool gj_step(float (&M)[RA][CB], unsigned& used, int kl, int nf, int tx, int ty,
                                        float (*s_best)[16], float (*s_d)[16], int (*s_row)[16],
                                        float (*s_prow)[CB * 32], int* s_piv, int* s_inv) {
  const int k = 32 * KB + kl, buf = k & 1;
  // pivot candidate of this warp's rows: column k from lane kl
  float best = -1.f, bd = 0.f;
  int br = nf;
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const float m = __shfl_sync(0xffffffffu, M[a][KB], kl);
    const float am = fabsf(m);
    if (!((used >> a) & 1u) && am > best) { best = am; bd = m; br = ty + 16 * a; }
  }
  if (tx == 0) { s_best[buf][ty] = best; s_d[buf][ty] = bd; s_row[buf][ty] = br; }
  __syncthreads();
  float pb = -1.f, d = 0.f;
  int p = nf;
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    const float v = s_best[buf][w];
    const int r = s_row[buf][w];
    if (v > pb || (v == pb && r < p)) { pb = v; p = r; d = s_d[buf][w]; }
  }
  if (!(pb > 0.f) || !isfinite(pb) || p >= nf) return false;   // the same decision in every thread
  const float inv = 1.f / d;
  if (ty == (p & 15)) {   // the warp holding row p publishes it, scaled
    const int ap = p >> 4;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      float v = 0.f;
#pragma unroll
      for (int a = 0; a < RA; ++a) v = (a == ap) ? M[a][b] : v;
      const int c = tx + 32 * b;
      s_prow[buf][c] = (c == k) ? inv : v * inv;
    }
    if (tx == 0) { s_piv[k] = p; s_inv[p] = k; }
  }
  __syncthreads();
  const float* pr = s_prow[buf] + tx;   // pivot row entries of this thread's columns: pr[32 b]
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const float m = __shfl_sync(0xffffffffu, M[a][KB], kl);
    if (ty + 16 * a == p) {
#pragma unroll
      for (int b = 0; b < CB; ++b) M[a][b] = pr[32 * b];
      used |= 1u << a;
    } else {
      if (tx == kl) M[a][KB] = 0.f;
#pragma unroll
      for (int b = 0; b < CB; ++b) M[a][b] -= m * pr[32 * b];
    }
  }
  return true;
}

template <int RA, int CB, int KB>
__device__ __forceinline__ bool gj_block(float (&M)[RA][CB], unsigned& used, int nf, int tx, int ty,
                                         float (*s_best)[16], float (*s_d)[16], int (*s_row)[16],
                                         float (*s_prow)[CB * 32], int* s_piv, int* s_inv) {
  if constexpr (KB < CB) {
    const int kend = min(32, nf - 32 * KB);
    for (int kl = 0; kl < kend; ++kl)
      if (!gj_step<RA, CB, KB>(M, used, kl, nf, tx, ty, s_best, s_d, s_row, s_prow, s_piv, s_inv)) return false;
    return gj_block<RA, CB, KB + 1>(M, used, nf, tx, ty, s_best, s_d, s_row, s_prow, s_piv, s_inv);
  }
  return true;
}

// In-place Gauss-Jordan inversion with partial pivoting held in registers (FP32, nf <= 224): one block
// of 16 x 32 threads; thread (ty, tx) holds M[r][c] for the rows r = ty + 16 a (a < RA) and columns
// c = tx + 32 b (b < CB). Pivoting is implicit (no row exchange): step k takes as pivot the row p, not
// yet used, with the largest |M[p][k]| (ties to the lower row), forms the pivot row
// prow = M[p] / d with prow[k] = 1 / d (d = M[p][k]), sets M[i][k] = 0 and subtracts
// M_old[i][k] prow from every other row i, and stores prow as row p. Each warp reads its rows'
// column-k values from lane k mod 32 by a shuffle (the steps run in blocks of 32 columns, so the
// register holding column k is known at compile time); the pivot candidates (one per warp) and the
// pivot row pass through double-buffered shared memory, so a step needs two barriers. With p_k the
// pivot of step k and q its inverse permutation, the result M satisfies A^-1[q[r]][p_c] = M[r][c].
template <int RA, int CB>
__global__ void __launch_bounds__(512) k_gj32_reg(const double* __restrict__ A, float* __restrict__ Ainv32, int nf,
                                                  int* flag) {
  __shared__ float s_best[2][16], s_d[2][16];
  __shared__ int s_row[2][16];
  __shared__ float s_prow[2][CB * 32];
  __shared__ int s_piv[RA * 16], s_inv[RA * 16];
  const int tx = threadIdx.x, ty = threadIdx.y;
  float M[RA][CB];
  unsigned used = 0;
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int r = ty + 16 * a;
    if (r >= nf) used |= 1u << a;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int c = tx + 32 * b;
      M[a][b] = (r < nf && c < nf) ? (float)A[(long long)r * nf + c] : 0.f;
    }
  }
  if (!gj_block<RA, CB, 0>(M, used, nf, tx, ty, s_best, s_d, s_row, s_prow, s_piv, s_inv)) {
    if (tx == 0 && ty == 0) atomicExch(flag, 1);
    return;
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int r = ty + 16 * a;
    if (r >= nf) continue;
    const int row = s_inv[r];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int c = tx + 32 * b;
      if (c < nf) Ainv32[(long long)row * nf + s_piv[c]] = M[a][b];
    }
  }
}

// x = A^-1 b on the free DOFs of the coarsest level (or A^-T b), in three launches:
//   x0 = Ainv32 b (FP32), r = b - A x0 (FP64, A the FP64 Galerkin matrix), x = x0 + Ainv32 r (FP32).
// One warp per row; row-major matrices are read along rows (coalesced) for A x and along columns for
// A^T x. xr holds x0 (FP64) and r (FP64) between the launches.
template <typename T, typename AccT, bool TR>
__device__ __forceinline__ AccT row_dot(const T* __restrict__ M, int nf, int r, const double* __restrict__ v) {
  const int lane = threadIdx.x & 31;
  AccT acc = AccT(0);
  for (int c = lane; c < nf; c += 32)
    acc += (AccT)(TR ? M[(long long)c * nf + r] : M[(long long)r * nf + c]) * (AccT)v[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename R, bool TR>
__global__ void __launch_bounds__(256) k_coarse_x0(const float* __restrict__ Ainv32, int nf, const R* __restrict__ b,
                                                   double* __restrict__ bd, double* __restrict__ x0) {
  __shared__ double sb[kMaxCoarseDofs];
  for (int c = threadIdx.x; c < nf; c += blockDim.x) sb[c] = (double)b[c];
  __syncthreads();
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nf) return;
  const float acc = row_dot<float, float, TR>(Ainv32, nf, r, sb);
  if ((threadIdx.x & 31) == 0) { x0[r] = (double)acc; bd[r] = sb[r]; }
}

template <bool TR>
__global__ void __launch_bounds__(256) k_coarse_resid(const double* __restrict__ A, int nf, const double* __restrict__ bd,
                                                      const double* __restrict__ x0, double* __restrict__ rd) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nf) return;
  const double acc = row_dot<double, double, TR>(A, nf, r, x0);
  if ((threadIdx.x & 31) == 0) rd[r] = bd[r] - acc;
}

template <typename R, bool TR>
__global__ void __launch_bounds__(256) k_coarse_fix(const float* __restrict__ Ainv32, int nf, const double* __restrict__ x0,
                                                    const double* __restrict__ rd, R* __restrict__ x, int n2) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r < nf) {
    const float acc = row_dot<float, float, TR>(Ainv32, nf, r, rd);
    if ((threadIdx.x & 31) == 0) x[r] = (R)(x0[r] + (double)acc);
  }
  for (int q = nf + blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += gridDim.x * blockDim.x) x[q] = R(0);
}

// ---- fused multigrid tail (one thread-block cluster) ---------------------------------------------
// The steps of vcycle() on levels l0 .. L-1 in launch order; every step is a grid-stride loop over
// the cluster's threads followed by a cluster barrier (release/acquire at cluster scope). Vectors
// written inside the kernel are read through L2 (LdCG).
template <typename R, bool TR>
__global__ void __launch_bounds__(1024, 1) k_mg_tail(const TailArgs<R> A) {
  typedef typename Vec2<R>::type V;
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int T = blockDim.x * gridDim.x;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const LdCG ld;
  const int L = A.nlev;
  V* x[kTailMaxLevels];
  V* xn[kTailMaxLevels];
#pragma unroll
  for (int l = 0; l < kTailMaxLevels; ++l) {
    x[l] = l < L ? A.lev[l].x : nullptr;
    xn[l] = l < L ? A.lev[l].xn : nullptr;
  }
  // cluster barrier: arrive has release and wait acquire semantics at cluster scope, which orders
  // the global-memory writes of one step before the reads of the next in every CTA of the cluster
  auto barrier = [&]() { cl.sync(); };
  auto smooth = [&](int l) {   // xn = x + omega D^-1 (b - A x), then swap
    const TailLevel<R>& d = A.lev[l];
    for (int n = t; n < (int)d.g.nn; n += T) {
      const int i = n % d.g.NX, j = (n / d.g.NX) % d.g.NY, k = n / d.g.NXY;
      if (d.g.bc == kBcTop && k == d.g.nz) xn[l][n] = mk2<R>(R(0), R(0));
      else stencil_node<R, TR, 2>(d.g, d.S, x[l], d.b, d.dinv, A.omega, xn[l], n, i, j, k, ld);
    }
    barrier();
    V* tmp = x[l]; x[l] = xn[l]; xn[l] = tmp;
  };
  // descent: pre-smoothing, residual, restriction
  for (int l = 0; l < L - 1; ++l) {
    const TailLevel<R>& d = A.lev[l];
    for (int n = t; n < (int)d.g.nn; n += T) {   // first sweep from x = 0: x = omega D^-1 b
      const V bb = ld(d.b + n);
      const R* dd = d.dinv + 4 * n;
      const R z0 = TR ? dd[0] * bb.x + dd[2] * bb.y : dd[0] * bb.x + dd[1] * bb.y;
      const R z1 = TR ? dd[1] * bb.x + dd[3] * bb.y : dd[2] * bb.x + dd[3] * bb.y;
      x[l][n] = mk2<R>(A.omega * z0, A.omega * z1);
    }
    barrier();
    for (int it = 1; it < A.nu1; ++it) smooth(l);
    for (int n = t; n < (int)d.g.nn; n += T) {   // residual into xn
      const int i = n % d.g.NX, j = (n / d.g.NX) % d.g.NY, k = n / d.g.NXY;
      if (d.g.bc == kBcTop && k == d.g.nz) xn[l][n] = mk2<R>(R(0), R(0));
      else stencil_node<R, TR, 1>(d.g, d.S, x[l], d.b, d.dinv, A.omega, xn[l], n, i, j, k, ld);
    }
    barrier();
    const Grid& gc = A.lev[l + 1].g;
    for (int n = t; n < (int)gc.nn; n += T) {
      const int I = n % gc.NX, J = (n / gc.NX) % gc.NY, K = n / gc.NXY;
      A.lev[l + 1].b[n] = mask_fixed<R>(gc, I, J, K, restrict_node<R>(d.g, xn[l], I, J, K, gc.bc == kBcTop && K >= gc.nz, ld));
    }
    barrier();
  }
  // coarsest level: x0 = Ainv32 b (FP32), r = b - A x0 (FP64), x = x0 + Ainv32 r (FP32)
  {
    const int nf = A.nf;
    double* bd = A.cw;
    double* x0 = A.cw + nf;
    double* rd = A.cw + 2 * nf;
    const R* bc = (const R*)A.lev[L - 1].b;
    R* xc = (R*)x[L - 1];
    const int lane = t & 31, gw = t >> 5, W = T >> 5;
    for (int c = t; c < nf; c += T) bd[c] = (double)ld(bc + c);
    barrier();
    for (int r = gw; r < nf; r += W) {
      float acc = 0.f;
      for (int c = lane; c < nf; c += 32)
        acc += (TR ? A.Ainv32[(long long)c * nf + r] : A.Ainv32[(long long)r * nf + c]) * (float)ld(bd + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) x0[r] = (double)acc;
    }
    barrier();
    for (int r = gw; r < nf; r += W) {
      double acc = 0.0;
      for (int c = lane; c < nf; c += 32)
        acc += (TR ? A.Ac[(long long)c * nf + r] : A.Ac[(long long)r * nf + c]) * ld(x0 + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) rd[r] = ld(bd + r) - acc;
    }
    barrier();
    for (int r = gw; r < nf; r += W) {
      float acc = 0.f;
      for (int c = lane; c < nf; c += 32)
        acc += (TR ? A.Ainv32[(long long)c * nf + r] : A.Ainv32[(long long)r * nf + c]) * (float)ld(rd + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) xc[r] = (R)(ld(x0 + r) + (double)acc);
    }
    const int n2 = (int)(2 * A.lev[L - 1].g.nn);
    for (int q = nf + t; q < n2; q += T) xc[q] = R(0);
    barrier();
  }
  // ascent: prolongation and post-smoothing
  for (int l = L - 2; l >= 0; --l) {
    const TailLevel<R>& d = A.lev[l];
    for (int n = t; n < (int)d.g.nn; n += T) {
      const int i = n % d.g.NX, j = (n / d.g.NX) % d.g.NY, k = n / d.g.NXY;
      if (fixed_bits(d.g, i, j, k) != 3) prolong_node<R>(d.g, A.lev[l + 1].g, x[l + 1], x[l], n, i, j, k, ld);
    }
    barrier();
    for (int it = 0; it < A.nu2; ++it) smooth(l);
  }
}

}  // namespace

template <typename R>
cudaError_t launch_galerkin_fine(const Grid& gf, const Grid& gc, const Phys& ph, const typename Vec2<R>::type* s,
                                 const typename Vec2<R>::type* mat, R* diag_f, R* ebe_c, cudaStream_t st,
                                 Counters* c, bool picard) {
  if (picard)
    k_galerkin_fine<R, true><<<(unsigned)gc.ne, 128 / NC_GALERKIN_CPT, 0, st>>>(gf, gc, ph, make_econst<R>(ph), s, mat,
                                                                              diag_f, ebe_c);
  else
    k_galerkin_fine<R, false><<<(unsigned)gc.ne, 128 / NC_GALERKIN_CPT, 0, st>>>(gf, gc, ph, make_econst<R>(ph), s, mat,
                                                                               diag_f, ebe_c);
  if (c) {
    c->launches += 1;
    c->bytes += sizeof(R) * (2.0 * gf.nn + 2.0 * gf.ne + 4.0 * gf.nn + 256.0 * gc.ne);
    // one element state, 16 columns
    c->flops += (kFlopsState + 16.0 * (picard ? kFlopsPicardModal : flops_jac_column<R>())) * gf.ne;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_galerkin_coarse(const Grid& gf, const Grid& gc, const R* ebe_f, R* diag_f, R* ebe_c,
                                   cudaStream_t st, Counters* c) {
  k_galerkin_coarse<R><<<(unsigned)gc.ne, 128, 0, st>>>(gf, gc, ebe_f, diag_f, ebe_c);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (256.0 * gf.ne + 4.0 * gf.nn + 256.0 * gc.ne); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_invert_diag(const Grid& g, R* diag, int* flag, cudaStream_t st, Counters* c) {
  k_invert_diag<R><<<grid_blocks(g.nn, 256), 256, 0, st>>>(g, diag, flag);
  if (c) c->launches += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_level0_apply(const Grid& g, const Phys& ph, const typename Vec2<R>::type* s,
                                const typename Vec2<R>::type* mat, const typename Vec2<R>::type* x,
                                typename Vec2<R>::type* y, bool transpose, cudaStream_t st, Counters* c, int kc) {
  cudaError_t err = cudaMemsetAsync(y, 0, sizeof(R) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  bool done = false;
  if constexpr (std::is_same<R, float>::value) {
    if (kc >= 0) {
      if (transpose) launch_level0_z<0, true>(g, ph, s, nullptr, mat, x, (float*)y, level0_kc(kc), st);
      else launch_level0_z<0, false>(g, ph, s, nullptr, mat, x, (float*)y, level0_kc(kc), st);
      done = true;
    }
  }
  if (!done) {
    const Launch3 L = launch_elems(g);
    if (transpose)
      k_level0_apply<R, true><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, x, (R*)y);
    else
      k_level0_apply<R, false><<<L.grid, L.block, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, x, (R*)y);
  }
  if (c) {
    c->launches += 1;
    c->bytes += sizeof(R) * (6.0 * g.nn + 2.0 * g.ne);   // s, x, y per node; (kappa, k) per element
    c->flops += (kFlopsState + (transpose ? flops_jtv<R>() : flops_jv<R>())) * g.ne;
  }
  return cudaGetLastError();
}

cudaError_t launch_frozen(const Grid& g, const Phys& ph, const float2* s, const float2* mat, float4* fz,
                          cudaStream_t st, Counters* c) {
  const Launch3 L = launch_elems(g);
  k_frozen<<<L.grid, L.block, 0, st>>>(g, ph, make_econst<float>(ph), s, mat, fz);
  if (c) {
    c->launches += 1;
    c->bytes += 8.0 * g.nn + 24.0 * g.ne;
    c->flops += kFlopsState * g.ne;
  }
  return cudaGetLastError();
}

cudaError_t launch_level0_picard(const Grid& g, const Phys& ph, const float4* fz, const float2* mat, const float2* x,
                                 float2* y, bool transpose, cudaStream_t st, Counters* c, int kc) {
  cudaError_t err = cudaMemsetAsync(y, 0, sizeof(float) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  if (kc >= 0) {
    if (transpose) launch_level0_z<1, true>(g, ph, nullptr, fz, mat, x, (float*)y, level0_kc(kc), st);
    else launch_level0_z<1, false>(g, ph, nullptr, fz, mat, x, (float*)y, level0_kc(kc), st);
  } else {
    const Launch3 L = launch_elems(g);
    if (transpose) k_level0_picard<true><<<L.grid, L.block, 0, st>>>(g, make_econst<float>(ph), fz, mat, x, (float*)y);
    else k_level0_picard<false><<<L.grid, L.block, 0, st>>>(g, make_econst<float>(ph), fz, mat, x, (float*)y);
  }
  if (c) {
    c->launches += 1;
    c->bytes += 4.0 * (4.0 * g.nn + 6.0 * g.ne);   // x, y per node; (kappa, k), (u0, tau) per element
    c->flops += (transpose ? kFlopsPicardModalT : kFlopsPicardModal) * g.ne;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_jacobi_update(const Grid& g, const R* dinv, const typename Vec2<R>::type* b,
                                 const typename Vec2<R>::type* y, const typename Vec2<R>::type* x,
                                 typename Vec2<R>::type* xn, R omega, bool transpose, bool first, cudaStream_t st,
                                 Counters* c) {
  const unsigned nb = grid_blocks(g.nn, 256);
  if (first) {
    if (transpose) k_jacobi<R, true, true><<<nb, 256, 0, st>>>(g.nn, dinv, b, y, x, xn, omega);
    else k_jacobi<R, false, true><<<nb, 256, 0, st>>>(g.nn, dinv, b, y, x, xn, omega);
  } else {
    if (transpose) k_jacobi<R, true, false><<<nb, 256, 0, st>>>(g.nn, dinv, b, y, x, xn, omega);
    else k_jacobi<R, false, false><<<nb, 256, 0, st>>>(g.nn, dinv, b, y, x, xn, omega);
  }
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (first ? 8.0 : 12.0) * g.nn; }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_jacobi_io(const Grid& g, const R* dinv, typename Vec2<R>::type* b, const double* b64,
                             const typename Vec2<R>::type* y, const typename Vec2<R>::type* x,
                             typename Vec2<R>::type* xn, double* z64, R omega, bool transpose, bool first,
                             cudaStream_t st, Counters* c) {
  const unsigned nb = grid_blocks(g.nn, 256);
  const double2* bi = (const double2*)b64;
  double2* zo = (double2*)z64;
  if (first) {
    if (transpose) k_jacobi_io<R, true, true><<<nb, 256, 0, st>>>(g.nn, dinv, b, bi, y, x, xn, zo, omega);
    else k_jacobi_io<R, false, true><<<nb, 256, 0, st>>>(g.nn, dinv, b, bi, y, x, xn, zo, omega);
  } else {
    if (transpose) k_jacobi_io<R, true, false><<<nb, 256, 0, st>>>(g.nn, dinv, b, bi, y, x, xn, zo, omega);
    else k_jacobi_io<R, false, false><<<nb, 256, 0, st>>>(g.nn, dinv, b, bi, y, x, xn, zo, omega);
  }
  if (c) {
    c->launches += 1;
    c->bytes += (first ? 16.0 + 2.0 * sizeof(R) : 6.0 * sizeof(R)) * g.nn + 4.0 * sizeof(R) * g.nn +
                2.0 * sizeof(R) * g.nn + (z64 ? 16.0 * g.nn : 0.0);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* rf,
                            typename Vec2<R>::type* bc, cudaStream_t st, Counters* c, const R* dinv_c,
                            typename Vec2<R>::type* xc, R omega, bool transpose) {
  const Launch3 L = launch_nodes_flat(gc);
  const FirstSweep<R> fs{dinv_c, xc, omega};
  if (!xc) k_restrict<R, 0><<<L.grid, L.block, 0, st>>>(gf, gc, rf, bc, fs);
  else if (transpose) k_restrict<R, 2><<<L.grid, L.block, 0, st>>>(gf, gc, rf, bc, fs);
  else k_restrict<R, 1><<<L.grid, L.block, 0, st>>>(gf, gc, rf, bc, fs);
  // + D_c^-1 and x_c for the fused first sweep
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (2.0 * (gf.nn + gc.nn) + (xc ? 6.0 * gc.nn : 0.0)); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_restrict_residual(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* b,
                                     const typename Vec2<R>::type* y, typename Vec2<R>::type* bc, cudaStream_t st,
                                     Counters* c, const R* dinv_c, typename Vec2<R>::type* xc, R omega,
                                     bool transpose) {
  const Launch3 L = launch_nodes_flat(gc);
  const FirstSweep<R> fs{dinv_c, xc, omega};
  if (!xc) k_restrict_res<R, 0><<<L.grid, L.block, 0, st>>>(gf, gc, b, y, bc, fs);
  else if (transpose) k_restrict_res<R, 2><<<L.grid, L.block, 0, st>>>(gf, gc, b, y, bc, fs);
  else k_restrict_res<R, 1><<<L.grid, L.block, 0, st>>>(gf, gc, b, y, bc, fs);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (2.0 * (2.0 * gf.nn + gc.nn) + (xc ? 6.0 * gc.nn : 0.0)); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prolong_add(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* xc,
                               typename Vec2<R>::type* xf, cudaStream_t st, Counters* c) {
  const Launch3 L = launch_nodes_flat(gf);
  k_prolong_add<R><<<L.grid, L.block, 0, st>>>(gf, gc, xc, xf);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * 2.0 * (2.0 * gf.nn + gc.nn); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dense_assemble(const Grid& g, const R* ebe, double* A, int nf, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(A, 0, sizeof(double) * nf * nf, st);
  if (err != cudaSuccess) return err;
  k_dense_assemble<R><<<grid_blocks(g.ne * 256, 256), 256, 0, st>>>(g, ebe, A, nf);
  if (c) c->launches += 1;
  if (g.bc != kBcTop) {
    k_dense_fixed_rows<<<grid_blocks(boundary_count(g), 256), 256, 0, st>>>(g, A, nf);
    if (c) c->launches += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_coarse_factor(const double* A, float* work, float* Ainv32, int nf, int* flag, cudaStream_t st,
                                 Counters* c) {
  if (nf <= 224) {
    const dim3 blk(32, 16);
#define NC_GJR(RA) case RA: k_gj32_reg<RA, (RA + 1) / 2><<<1, blk, 0, st>>>(A, Ainv32, nf, flag); break
    switch ((nf + 15) / 16) {   // row tiles of 16
      NC_GJR(1); NC_GJR(2); NC_GJR(3); NC_GJR(4); NC_GJR(5); NC_GJR(6); NC_GJR(7);
      NC_GJR(8); NC_GJR(9); NC_GJR(10); NC_GJR(11); NC_GJR(12); NC_GJR(13); default: NC_GJR(14);
    }
#undef NC_GJR
    if (c) c->launches += 1;
  } else {
    // work: W (nf x 2nf floats), then piv, used (nf ints each) and the multipliers (nf floats)
    float* W = work;
    int* piv = reinterpret_cast<int*>(W + 2LL * nf * nf);
    int* used = piv + nf;
    float* m = reinterpret_cast<float*>(used + nf);
    k_gjm_init<<<grid_blocks(2LL * nf * nf, 256, 152 * 16), 256, 0, st>>>(A, W, nf, used);
    const dim3 ug((unsigned)((2 * nf + 255) / 256), (unsigned)nf);
    for (int k = 0; k < nf; ++k) {
      k_gjm_pivot<<<1, 1024, 0, st>>>(W, nf, k, piv, used, m, flag);
      k_gjm_update<<<ug, 256, 0, st>>>(W, nf, k, piv, m);
    }
    k_gjm_permute<<<grid_blocks((long long)nf * nf, 256, 152 * 16), 256, 0, st>>>(W, nf, piv, Ainv32);
    if (c) c->launches += 2 + 2LL * nf;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_stencil_build(const Grid& g, const R* ebe, R* S, cudaStream_t st, Counters* c) {
  k_stencil_build<R><<<grid_blocks(g.nn * 27, 256), 256, 0, st>>>(g, ebe, S);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (256.0 * g.ne + 108.0 * g.nn); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_stencil_apply(const Grid& g, const R* S, const typename Vec2<R>::type* x,
                                 const typename Vec2<R>::type* b, const R* dinv, R omega,
                                 typename Vec2<R>::type* out, bool transpose, int mode, cudaStream_t st,
                                 Counters* c) {
  const Launch3 L = launch_nodes_flat(g);
#define NC_ST(TRV, MV) k_stencil_apply<R, TRV, MV><<<L.grid, L.block, 0, st>>>(g, S, x, b, dinv, omega, out)
  if (transpose) {
    if (mode == 0) NC_ST(true, 0); else if (mode == 1) NC_ST(true, 1); else NC_ST(true, 2);
  } else {
    if (mode == 0) NC_ST(false, 0); else if (mode == 1) NC_ST(false, 1); else NC_ST(false, 2);
  }
#undef NC_ST
  if (c) {
    c->launches += 1;
    // 108 stencil coefficients, x and the output per node; + b (modes 1, 2); + D^-1 (mode 2)
    c->bytes += sizeof(R) * (108.0 + 2.0 + 2.0 + (mode ? 2.0 : 0.0) + (mode == 2 ? 4.0 : 0.0)) * g.nn;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_coarse_solve(const double* A, const float* Ainv32, double* work, int nf,
                                const typename Vec2<R>::type* b, typename Vec2<R>::type* x, long long nn,
                                bool transpose, cudaStream_t st, Counters* c) {
  // work: 3 nf doubles (b, x0, r)
  double* bd = work;
  double* x0 = work + nf;
  double* rd = work + 2 * nf;
  const unsigned nb = (unsigned)((nf + 7) / 8);
  const int n2 = (int)(2 * nn);
  if (transpose) {
    k_coarse_x0<R, true><<<nb, 256, 0, st>>>(Ainv32, nf, (const R*)b, bd, x0);
    k_coarse_resid<true><<<nb, 256, 0, st>>>(A, nf, bd, x0, rd);
    k_coarse_fix<R, true><<<nb, 256, 0, st>>>(Ainv32, nf, x0, rd, (R*)x, n2);
  } else {
    k_coarse_x0<R, false><<<nb, 256, 0, st>>>(Ainv32, nf, (const R*)b, bd, x0);
    k_coarse_resid<false><<<nb, 256, 0, st>>>(A, nf, bd, x0, rd);
    k_coarse_fix<R, false><<<nb, 256, 0, st>>>(Ainv32, nf, x0, rd, (R*)x, n2);
  }
  if (c) c->launches += 3;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_from_mg(const typename Vec2<R>::type* x, double* z, long long nn, cudaStream_t st, Counters* c) {
  k_from_mg<R><<<grid_blocks(nn, 256), 256, 0, st>>>(x, (double2*)z, nn);
  if (c) { c->launches += 1; c->bytes += (16.0 + 2.0 * sizeof(R)) * nn; }
  return cudaGetLastError();
}

// Cluster size of the tail kernel: 16 (non-portable) where the device schedules it, else 8.
template <typename R, bool TR>
static int tail_cluster_size() {
  // decided once per device (function attributes and occupancy are per device)
  static std::mutex mu;
  static int cs_dev[kMaxDevices] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 8;
  std::lock_guard<std::mutex> lock(mu);
  int& cs = cs_dev[dev];
  if (cs) return cs;
  cs = 8;
  if (cudaFuncSetAttribute(k_mg_tail<R, TR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(1024);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_mg_tail<R, TR>, &cfg) == cudaSuccess && nclusters > 0) cs = 16;
  }
  cudaGetLastError();
  return cs;
}

template <typename R>
cudaError_t launch_mg_tail(const TailArgs<R>& a, bool transpose, cudaStream_t st, Counters* c) {
  if (a.nlev < 2 || a.nlev > kTailMaxLevels || a.nf > kMaxCoarseDofs) return cudaErrorInvalidValue;
  const int cmax = transpose ? tail_cluster_size<R, true>() : tail_cluster_size<R, false>();
  const int cs = a.ctas > 0 ? std::min(a.ctas, cmax) : cmax;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(1024);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = transpose ? cudaLaunchKernelEx(&cfg, k_mg_tail<R, true>, a) : cudaLaunchKernelEx(&cfg, k_mg_tail<R, false>, a);
  if (c) {
    c->launches += 1;
    for (int l = 0; l + 1 < a.nlev; ++l)   // stencil sweeps: 108 coefficients + x, b, out per node
      c->bytes += sizeof(R) * 114.0 * a.lev[l].g.nn * (a.nu1 + a.nu2 + 1);
  }
  return e;
}

template <typename R>
cudaError_t launch_line_factor(const Grid& g, const R* S, R* LF, int* flag, cudaStream_t st, Counters* c) {
  const unsigned nb = grid_blocks(g.NXY, 32);
  k_line_factor<R, false><<<nb, 32, 0, st>>>(g, S, LF, flag);
  k_line_factor<R, true><<<nb, 32, 0, st>>>(g, S, LF + 12 * g.nn, flag);
  if (c) { c->launches += 2; c->bytes += 2.0 * sizeof(R) * 24.0 * g.nn; }   // 3 blocks read, 3 written
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_line_smooth(const Grid& g, const R* LF, const typename Vec2<R>::type* r,
                               typename Vec2<R>::type* x, R omega, bool transpose, bool first, cudaStream_t st,
                               Counters* c) {
  const unsigned nb = grid_blocks(g.NXY, 4);   // 4 columns (warps) per block
  const R* lf = LF + (transpose ? 12 * g.nn : 0);
  typedef typename Vec2<R>::type V2;
  if (first) k_line_smooth<R, true><<<nb, 128, 0, st>>>(g, lf, r, x, x, omega);
  else k_line_smooth<R, false><<<nb, 128, 0, st>>>(g, lf, r, const_cast<V2*>(r), x, omega);
  if (c) {
    c->launches += 1;
    // E^-1, M, r, y written; G, y, x (not first), x written
    c->bytes += sizeof(R) * (8.0 + 2.0 + 2.0 + 4.0 + 2.0 + (first ? 0.0 : 2.0) + 2.0) * g.nn;
  }
  return cudaGetLastError();
}

#define NC_INSTANTIATE_MG(R)                                                                                    \
  template cudaError_t launch_galerkin_fine<R>(const Grid&, const Grid&, const Phys&, const Vec2<R>::type*,   \
                                               const Vec2<R>::type*, R*, R*, cudaStream_t, Counters*, bool);   \
  template cudaError_t launch_galerkin_coarse<R>(const Grid&, const Grid&, const R*, R*, R*, cudaStream_t,    \
                                                 Counters*);                                                   \
  template cudaError_t launch_invert_diag<R>(const Grid&, R*, int*, cudaStream_t, Counters*);                 \
  template cudaError_t launch_level0_apply<R>(const Grid&, const Phys&, const Vec2<R>::type*,                 \
                                              const Vec2<R>::type*, const Vec2<R>::type*, Vec2<R>::type*,     \
                                              bool, cudaStream_t, Counters*, int);                             \
  template cudaError_t launch_jacobi_update<R>(const Grid&, const R*, const Vec2<R>::type*,                   \
                                               const Vec2<R>::type*, const Vec2<R>::type*, Vec2<R>::type*, R, \
                                               bool, bool, cudaStream_t, Counters*);                           \
  template cudaError_t launch_jacobi_io<R>(const Grid&, const R*, Vec2<R>::type*, const double*,              \
                                           const Vec2<R>::type*, const Vec2<R>::type*, Vec2<R>::type*, double*, \
                                           R, bool, bool, cudaStream_t, Counters*);                             \
  template cudaError_t launch_restrict<R>(const Grid&, const Grid&, const Vec2<R>::type*, Vec2<R>::type*,     \
                                          cudaStream_t, Counters*, const R*, Vec2<R>::type*, R, bool);        \
  template cudaError_t launch_restrict_residual<R>(const Grid&, const Grid&, const Vec2<R>::type*,            \
                                                   const Vec2<R>::type*, Vec2<R>::type*, cudaStream_t, Counters*, \
                                                   const R*, Vec2<R>::type*, R, bool);                          \
  template cudaError_t launch_prolong_add<R>(const Grid&, const Grid&, const Vec2<R>::type*, Vec2<R>::type*,  \
                                             cudaStream_t, Counters*);                                         \
  template cudaError_t launch_dense_assemble<R>(const Grid&, const R*, double*, int, cudaStream_t, Counters*);\
  template cudaError_t launch_coarse_solve<R>(const double*, const float*, double*, int, const Vec2<R>::type*, \
                                              Vec2<R>::type*, long long, bool, cudaStream_t, Counters*);        \
  template cudaError_t launch_from_mg<R>(const Vec2<R>::type*, double*, long long, cudaStream_t, Counters*); \
  template cudaError_t launch_stencil_build<R>(const Grid&, const R*, R*, cudaStream_t, Counters*);           \
  template cudaError_t launch_stencil_apply<R>(const Grid&, const R*, const Vec2<R>::type*,                  \
                                               const Vec2<R>::type*, const R*, R, Vec2<R>::type*, bool, int, \
                                               cudaStream_t, Counters*);                                       \
  template cudaError_t launch_mg_tail<R>(const TailArgs<R>&, bool, cudaStream_t, Counters*);             \
  template cudaError_t launch_line_factor<R>(const Grid&, const R*, R*, int*, cudaStream_t, Counters*);     \
  template cudaError_t launch_line_smooth<R>(const Grid&, const R*, const Vec2<R>::type*, Vec2<R>::type*, R, \
                                             bool, bool, cudaStream_t, Counters*);

NC_INSTANTIATE_MG(float)
NC_INSTANTIATE_MG(double)

}  // namespace nc
