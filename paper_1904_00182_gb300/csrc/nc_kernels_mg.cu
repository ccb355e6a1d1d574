// Geometric multigrid kernels, templated on the multigrid arithmetic type R (float: mixed
// precision preconditioner; double: the all-FP64 path).
//
// Hierarchy: level l has (nx/2^l, ny/2^l, nz/2^l) elements. Transfer operators are trilinear
// interpolation P and its transpose (full weighting) R = P^T. Coarse operators are Galerkin
// products P^T A P assembled element by element: a coarse element's matrix is the sum over its 8
// children of P_c^T A_c P_c, where P_c interpolates the child's 8 nodes from the parent's 8
// corners (exact for nested trilinear spaces). Level 0 applies the Newton Jacobian J(s) matrix
// free; levels >= 1 store 16x16 element matrices (rows/cols: P_0..7, T_0..7). The smoother is
// damped 2x2 node-block Jacobi; the coarsest level is solved with an explicit FP64 inverse.
#include "nc_launch.h"

namespace nc {

namespace {

template <typename R>
__device__ __forceinline__ R interp_w(int child, int l, int A) {
  // weight of parent corner A at the child's local node l (tensor product of 1D hat values)
  R w = R(1);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int cd = (child >> d) & 1, ld = (l >> d) & 1, Ad = (A >> d) & 1;
    const R t = R(0.5) * R(cd + ld);
    w *= Ad ? t : R(1) - t;
  }
  return w;
}

template <typename R>
__device__ __forceinline__ void add_diag_block(R* __restrict__ diag, long long n, int idx, R v) {
  atomicAdd(diag + 4 * n + idx, v);
}

// Phase 2 shared by both Galerkin kernels: Jc[c][16][16] in shared memory -> coarse element matrix.
template <typename R>
__device__ __forceinline__ void galerkin_phase2(R (*Jc)[256], R (*Tc)[256], R* __restrict__ out) {
  const int t = threadIdx.x;
  {
    const int c = t >> 4, row = t & 15;
#pragma unroll 4
    for (int J = 0; J < 16; ++J) {
      const int fj = J >> 3, A = J & 7;
      R acc = R(0);
#pragma unroll
      for (int l = 0; l < 8; ++l) acc += Jc[c][row * 16 + fj * 8 + l] * interp_w<R>(c, l, A);
      Tc[c][row * 16 + J] = acc;
    }
  }
  __syncthreads();
  {
    const int I = t >> 3;
    const int fi = I >> 3, Ai = I & 7;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int J = (t & 7) * 2 + jj;
      R acc = R(0);
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += interp_w<R>(c, k, Ai) * Tc[c][(fi * 8 + k) * 16 + J];
      out[I * 16 + J] = acc;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(128) k_galerkin_fine(Grid gf, Grid gc, Phys ph, ElemConst<R> C,
                                                       const typename Vec2<R>::type* __restrict__ s,
                                                       const typename Vec2<R>::type* __restrict__ mat,
                                                       R* __restrict__ diag_f, R* __restrict__ ebe_c) {
  __shared__ R Jc[8][256];
  __shared__ R Tc[8][256];
  const long long E = blockIdx.x;
  int I, J, K;
  elem_ijk(gc, E, I, J, K);
  const int t = threadIdx.x;
  const int c = t >> 4, col = t & 15;
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
  elem_state(C, p, tt, m.x, k < ph.heated_layers ? (R)ph.Q : R(0), st);
  R dp[8], dt[8], oP[8], oT[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) { dp[a] = (col == a) ? R(1) : R(0); dt[a] = (col == 8 + a) ? R(1) : R(0); }
  elem_jv_dir<R>(C, st, m.y, dp, dt, oP, oT);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    Jc[c][r * 16 + col] = oP[r];
    Jc[c][(8 + r) * 16 + col] = oT[r];
  }
  // block diagonal of level 0 (row-major [PP PT; TP TT]) on free nodes
  const int a = col & 7;
  if (k + (a >> 2) < gf.nz) {
    const long long n = corner_node(gf, i, j, k, a);
    if (col < 8) { add_diag_block(diag_f, n, 0, oP[a]); add_diag_block(diag_f, n, 2, oT[a]); }
    else { add_diag_block(diag_f, n, 1, oP[a]); add_diag_block(diag_f, n, 3, oT[a]); }
  }
  __syncthreads();
  galerkin_phase2<R>(Jc, Tc, ebe_c + E * 256);
}

template <typename R>
__global__ void __launch_bounds__(128) k_galerkin_coarse(Grid gf, Grid gc, const R* __restrict__ ebe_f,
                                                         R* __restrict__ diag_f, R* __restrict__ ebe_c) {
  __shared__ R Jc[8][256];
  __shared__ R Tc[8][256];
  const long long E = blockIdx.x;
  int I, J, K;
  elem_ijk(gc, E, I, J, K);
  const int t = threadIdx.x;
  for (int idx = t; idx < 8 * 256; idx += 128) {
    const int c = idx >> 8, r = idx & 255;
    const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    const long long e = i + (long long)gf.nx * (j + (long long)gf.ny * k);
    Jc[c][r] = ebe_f[e * 256 + r];
  }
  __syncthreads();
  if (t < 64) {
    const int c = t >> 3, a = t & 7;
    const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
    if (k + (a >> 2) < gf.nz) {
      const long long n = corner_node(gf, i, j, k, a);
      add_diag_block(diag_f, n, 0, Jc[c][a * 16 + a]);
      add_diag_block(diag_f, n, 1, Jc[c][a * 16 + 8 + a]);
      add_diag_block(diag_f, n, 2, Jc[c][(8 + a) * 16 + a]);
      add_diag_block(diag_f, n, 3, Jc[c][(8 + a) * 16 + 8 + a]);
    }
  }
  galerkin_phase2<R>(Jc, Tc, ebe_c + E * 256);
}

template <typename R>
__global__ void k_diag_from_ebe(Grid g, const R* __restrict__ ebe, R* __restrict__ diag) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  int i, j, k;
  elem_ijk(g, e, i, j, k);
  const R* A = ebe + e * 256;
  for (int a = 0; a < 8; ++a) {
    if (k + (a >> 2) == g.nz) continue;
    const long long n = corner_node(g, i, j, k, a);
    add_diag_block(diag, n, 0, A[a * 16 + a]);
    add_diag_block(diag, n, 1, A[a * 16 + 8 + a]);
    add_diag_block(diag, n, 2, A[(8 + a) * 16 + a]);
    add_diag_block(diag, n, 3, A[(8 + a) * 16 + 8 + a]);
  }
}

template <typename R>
__global__ void k_invert_diag(Grid g, R* __restrict__ diag, int* flag) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  R* d = diag + 4 * n;
  if (n >= (long long)g.NX * g.NY * g.nz) { d[0] = d[1] = d[2] = d[3] = R(0); return; }
  const R a = d[0], b = d[1], c = d[2], e = d[3];
  const R det = a * e - b * c;
  if (!(det != R(0)) || !isfinite((double)det)) { atomicExch(flag, 1); d[0] = d[1] = d[2] = d[3] = R(0); return; }
  const R id = R(1) / det;
  d[0] = e * id; d[1] = -b * id; d[2] = -c * id; d[3] = a * id;
}

template <typename R, bool TR>
__global__ void k_level0_apply(Grid g, Phys ph, ElemConst<R> C, const typename Vec2<R>::type* __restrict__ s,
                               const typename Vec2<R>::type* __restrict__ mat,
                               const typename Vec2<R>::type* __restrict__ x, R* __restrict__ y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  int i, j, k;
  elem_ijk(g, e, i, j, k);
  R p[8], t[8], dp[8], dt[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = corner_node(g, i, j, k, a);
    const typename Vec2<R>::type v = s[n];
    p[a] = v.x; t[a] = v.y;
    if (k + (a >> 2) == g.nz) { dp[a] = R(0); dt[a] = R(0); }
    else { const typename Vec2<R>::type w = x[n]; dp[a] = w.x; dt[a] = w.y; }
  }
  const typename Vec2<R>::type m = mat[e];
  ElemState<R> st;
  elem_state(C, p, t, m.x, k < ph.heated_layers ? (R)ph.Q : R(0), st);
  R oP[8], oT[8];
  if (TR) elem_jtv<R, false>(C, st, m.y, dp, dt, oP, oT, nullptr, nullptr);
  else elem_jv_dir<R>(C, st, m.y, dp, dt, oP, oT);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (k + (a >> 2) == g.nz) continue;
    const long long n = corner_node(g, i, j, k, a);
    atomicAdd(y + 2 * n, oP[a]);
    atomicAdd(y + 2 * n + 1, oT[a]);
  }
}

template <typename R, bool TR>
__global__ void k_ebe_apply(Grid g, const R* __restrict__ ebe, const typename Vec2<R>::type* __restrict__ x,
                            R* __restrict__ y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  int i, j, k;
  elem_ijk(g, e, i, j, k);
  R xe[16];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (k + (a >> 2) == g.nz) { xe[a] = R(0); xe[8 + a] = R(0); continue; }
    const typename Vec2<R>::type w = x[corner_node(g, i, j, k, a)];
    xe[a] = w.x; xe[8 + a] = w.y;
  }
  const R* A = ebe + e * 256;
  R ye[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) ye[r] = R(0);
  if (TR) {
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const R xr = xe[r];
#pragma unroll
      for (int q = 0; q < 16; ++q) ye[q] += A[r * 16 + q] * xr;
    }
  } else {
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      R acc = R(0);
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += A[r * 16 + q] * xe[q];
      ye[r] = acc;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (k + (a >> 2) == g.nz) continue;
    const long long n = corner_node(g, i, j, k, a);
    atomicAdd(y + 2 * n, ye[a]);
    atomicAdd(y + 2 * n + 1, ye[8 + a]);
  }
}

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

template <typename R>
__global__ void k_sub(long long nn, const typename Vec2<R>::type* __restrict__ b,
                      const typename Vec2<R>::type* __restrict__ y, typename Vec2<R>::type* __restrict__ r) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const typename Vec2<R>::type bb = b[n], yy = y[n];
  r[n] = mk2<R>(bb.x - yy.x, bb.y - yy.y);
}

template <typename R>
__global__ void k_restrict(Grid gf, Grid gc, const typename Vec2<R>::type* __restrict__ rf,
                           typename Vec2<R>::type* __restrict__ bc) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= gc.nn) return;
  int I, J, K;
  node_ijk(gc, n, I, J, K);
  R a0 = R(0), a1 = R(0);
  if (K < gc.nz) {
    for (int dk = -1; dk <= 1; ++dk) {
      const int k = 2 * K + dk;
      if (k < 0 || k > gf.nz) continue;
      const R wk = dk ? R(0.5) : R(1);
      for (int dj = -1; dj <= 1; ++dj) {
        const int j = 2 * J + dj;
        if (j < 0 || j > gf.ny) continue;
        const R wj = dj ? R(0.5) : R(1);
        for (int di = -1; di <= 1; ++di) {
          const int i = 2 * I + di;
          if (i < 0 || i > gf.nx) continue;
          const R w = wk * wj * (di ? R(0.5) : R(1));
          const typename Vec2<R>::type v = rf[i + (long long)gf.NX * (j + (long long)gf.NY * k)];
          a0 += w * v.x;
          a1 += w * v.y;
        }
      }
    }
  }
  bc[n] = mk2<R>(a0, a1);
}

template <typename R>
__global__ void k_prolong_add(Grid gf, Grid gc, const typename Vec2<R>::type* __restrict__ xc,
                              typename Vec2<R>::type* __restrict__ xf) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= gf.nn) return;
  int i, j, k;
  node_ijk(gf, n, i, j, k);
  if (k == gf.nz) return;
  int ci[2], cj[2], ck[2];
  R wi[2], wj[2], wk[2];
  int ni, nj, nk;
  if (i & 1) { ci[0] = i >> 1; ci[1] = (i >> 1) + 1; wi[0] = wi[1] = R(0.5); ni = 2; } else { ci[0] = i >> 1; wi[0] = R(1); ni = 1; }
  if (j & 1) { cj[0] = j >> 1; cj[1] = (j >> 1) + 1; wj[0] = wj[1] = R(0.5); nj = 2; } else { cj[0] = j >> 1; wj[0] = R(1); nj = 1; }
  if (k & 1) { ck[0] = k >> 1; ck[1] = (k >> 1) + 1; wk[0] = wk[1] = R(0.5); nk = 2; } else { ck[0] = k >> 1; wk[0] = R(1); nk = 1; }
  R a0 = R(0), a1 = R(0);
  for (int c = 0; c < nk; ++c)
    for (int b = 0; b < nj; ++b)
      for (int a = 0; a < ni; ++a) {
        const R w = wi[a] * wj[b] * wk[c];
        const typename Vec2<R>::type v = xc[ci[a] + (long long)gc.NX * (cj[b] + (long long)gc.NY * ck[c])];
        a0 += w * v.x;
        a1 += w * v.y;
      }
  typename Vec2<R>::type o = xf[n];
  o.x += a0;
  o.y += a1;
  xf[n] = o;
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
  if (k + (ar >> 2) == g.nz || k + (aq >> 2) == g.nz) return;
  const long long row = 2 * corner_node(g, i, j, k, ar) + (r >> 3);
  const long long col = 2 * corner_node(g, i, j, k, aq) + (q >> 3);
  atomicAdd(A + row * nf + col, (double)ebe[t]);
}

// Gauss-Jordan inverse with partial pivoting of A (nf x nf, row major), one block of 1024 threads.
// work: nf x 2 nf scratch. On success A holds the inverse; flag = 1 on a zero pivot.
__global__ void __launch_bounds__(1024) k_dense_invert(double* __restrict__ A, double* __restrict__ W, int nf,
                                                       int* flag) {
  extern __shared__ double fac[];          // nf factors
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  const int t = threadIdx.x, nt = blockDim.x;
  const int w2 = 2 * nf;
  for (long long idx = t; idx < (long long)nf * w2; idx += nt) {
    const int r = (int)(idx / w2), c = (int)(idx % w2);
    W[idx] = c < nf ? A[(long long)r * nf + c] : (c - nf == r ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nf; ++k) {
    double best = -1.0;
    int bi = k;
    for (int r = k + t; r < nf; r += nt) {
      const double v = fabs(W[(long long)r * w2 + k]);
      if (v > best) { best = v; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((t & 31) == 0) { s_val[t >> 5] = best; s_idx[t >> 5] = bi; }
    __syncthreads();
    if (t == 0) {
      double b = -1.0;
      int bidx = k;
      for (int w = 0; w < (nt >> 5); ++w)
        if (s_val[w] > b || (s_val[w] == b && s_idx[w] < bidx)) { b = s_val[w]; bidx = s_idx[w]; }
      s_piv = (b > 0.0) ? bidx : -1;
    }
    __syncthreads();
    const int p = s_piv;
    if (p < 0) { if (t == 0) *flag = 1; return; }
    if (p != k)
      for (int c = t; c < w2; c += nt) {
        const double a = W[(long long)k * w2 + c];
        W[(long long)k * w2 + c] = W[(long long)p * w2 + c];
        W[(long long)p * w2 + c] = a;
      }
    __syncthreads();
    const double inv = 1.0 / W[(long long)k * w2 + k];
    __syncthreads();
    for (int c = t; c < w2; c += nt) W[(long long)k * w2 + c] *= inv;
    for (int r = t; r < nf; r += nt) fac[r] = W[(long long)r * w2 + k];
    __syncthreads();
    for (long long idx = t; idx < (long long)nf * w2; idx += nt) {
      const int r = (int)(idx / w2), c = (int)(idx % w2);
      if (r == k || c < k) continue;
      W[idx] -= fac[r] * W[(long long)k * w2 + c];
    }
    __syncthreads();
  }
  for (long long idx = t; idx < (long long)nf * nf; idx += nt) {
    const int r = (int)(idx / nf), c = (int)(idx % nf);
    A[idx] = W[(long long)r * w2 + nf + c];
  }
}

template <typename R, bool TR>
__global__ void k_dense_solve(const double* __restrict__ Ainv, int nf, const R* __restrict__ b, R* __restrict__ x,
                              long long n2) {
  for (int r = threadIdx.x + blockIdx.x * blockDim.x; r < n2; r += blockDim.x * gridDim.x) {
    if (r >= nf) { x[r] = R(0); continue; }
    double acc = 0.0;
    if (TR) { for (int c = 0; c < nf; ++c) acc += Ainv[(long long)c * nf + r] * (double)b[c]; }
    else { for (int c = 0; c < nf; ++c) acc += Ainv[(long long)r * nf + c] * (double)b[c]; }
    x[r] = (R)acc;
  }
}

template <typename R>
__global__ void k_to_mg(const double2* __restrict__ v, typename Vec2<R>::type* __restrict__ b, long long nn) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const double2 a = v[n];
  b[n] = mk2<R>((R)a.x, (R)a.y);
}

template <typename R>
__global__ void k_from_mg(const typename Vec2<R>::type* __restrict__ x, double2* __restrict__ z, long long nn) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const typename Vec2<R>::type a = x[n];
  z[n] = make_double2((double)a.x, (double)a.y);
}

}  // namespace

template <typename R>
cudaError_t launch_galerkin_fine(const Grid& gf, const Grid& gc, const Phys& ph, const typename Vec2<R>::type* s,
                                 const typename Vec2<R>::type* mat, R* diag_f, R* ebe_c, cudaStream_t st,
                                 Counters* c) {
  k_galerkin_fine<R><<<(unsigned)gc.ne, 128, 0, st>>>(gf, gc, ph, make_econst<R>(ph), s, mat, diag_f, ebe_c);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (2.0 * gf.nn + 2.0 * gf.ne + 4.0 * gf.nn + 256.0 * gc.ne); }
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
cudaError_t launch_diag_from_ebe(const Grid& g, const R* ebe, R* diag, cudaStream_t st, Counters* c) {
  k_diag_from_ebe<R><<<grid_blocks(g.ne, 128), 128, 0, st>>>(g, ebe, diag);
  if (c) c->launches += 1;
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
                                typename Vec2<R>::type* y, bool transpose, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(y, 0, sizeof(R) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  if (transpose)
    k_level0_apply<R, true><<<grid_blocks(g.ne, 128), 128, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, x, (R*)y);
  else
    k_level0_apply<R, false><<<grid_blocks(g.ne, 128), 128, 0, st>>>(g, ph, make_econst<R>(ph), s, mat, x, (R*)y);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (6.0 * g.nn + 2.0 * g.ne); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ebe_apply(const Grid& g, const R* ebe, const typename Vec2<R>::type* x,
                             typename Vec2<R>::type* y, bool transpose, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(y, 0, sizeof(R) * 2 * g.nn, st);
  if (err != cudaSuccess) return err;
  if (transpose) k_ebe_apply<R, true><<<grid_blocks(g.ne, 128), 128, 0, st>>>(g, ebe, x, (R*)y);
  else k_ebe_apply<R, false><<<grid_blocks(g.ne, 128), 128, 0, st>>>(g, ebe, x, (R*)y);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * (4.0 * g.nn + 256.0 * g.ne); }
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
cudaError_t launch_sub(const Grid& g, const typename Vec2<R>::type* b, const typename Vec2<R>::type* y,
                       typename Vec2<R>::type* r, cudaStream_t st, Counters* c) {
  k_sub<R><<<grid_blocks(g.nn, 256), 256, 0, st>>>(g.nn, b, y, r);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * 6.0 * g.nn; }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* rf,
                            typename Vec2<R>::type* bc, cudaStream_t st, Counters* c) {
  k_restrict<R><<<grid_blocks(gc.nn, 256), 256, 0, st>>>(gf, gc, rf, bc);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * 2.0 * (gf.nn + gc.nn); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prolong_add(const Grid& gf, const Grid& gc, const typename Vec2<R>::type* xc,
                               typename Vec2<R>::type* xf, cudaStream_t st, Counters* c) {
  k_prolong_add<R><<<grid_blocks(gf.nn, 256), 256, 0, st>>>(gf, gc, xc, xf);
  if (c) { c->launches += 1; c->bytes += sizeof(R) * 2.0 * (2.0 * gf.nn + gc.nn); }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dense_assemble(const Grid& g, const R* ebe, double* A, int nf, cudaStream_t st, Counters* c) {
  cudaError_t err = cudaMemsetAsync(A, 0, sizeof(double) * nf * nf, st);
  if (err != cudaSuccess) return err;
  k_dense_assemble<R><<<grid_blocks(g.ne * 256, 256), 256, 0, st>>>(g, ebe, A, nf);
  if (c) c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_dense_invert(double* A, double* work, int nf, int* flag, cudaStream_t st, Counters* c) {
  k_dense_invert<<<1, 1024, sizeof(double) * nf, st>>>(A, work, nf, flag);
  if (c) c->launches += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dense_solve(const double* Ainv, int nf, const typename Vec2<R>::type* b,
                               typename Vec2<R>::type* x, long long nn, bool transpose, cudaStream_t st,
                               Counters* c) {
  const long long n2 = 2 * nn;
  const unsigned nb = grid_blocks(n2, 128, 64);
  if (transpose) k_dense_solve<R, true><<<nb, 128, 0, st>>>(Ainv, nf, (const R*)b, (R*)x, n2);
  else k_dense_solve<R, false><<<nb, 128, 0, st>>>(Ainv, nf, (const R*)b, (R*)x, n2);
  if (c) c->launches += 1;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_to_mg(const double* v, typename Vec2<R>::type* b, long long nn, cudaStream_t st, Counters* c) {
  k_to_mg<R><<<grid_blocks(nn, 256), 256, 0, st>>>((const double2*)v, b, nn);
  if (c) { c->launches += 1; c->bytes += (16.0 + 2.0 * sizeof(R)) * nn; }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_from_mg(const typename Vec2<R>::type* x, double* z, long long nn, cudaStream_t st, Counters* c) {
  k_from_mg<R><<<grid_blocks(nn, 256), 256, 0, st>>>(x, (double2*)z, nn);
  if (c) { c->launches += 1; c->bytes += (16.0 + 2.0 * sizeof(R)) * nn; }
  return cudaGetLastError();
}

#define NC_INSTANTIATE_MG(R)                                                                                    \
  template cudaError_t launch_galerkin_fine<R>(const Grid&, const Grid&, const Phys&, const Vec2<R>::type*,   \
                                               const Vec2<R>::type*, R*, R*, cudaStream_t, Counters*);         \
  template cudaError_t launch_galerkin_coarse<R>(const Grid&, const Grid&, const R*, R*, R*, cudaStream_t,    \
                                                 Counters*);                                                   \
  template cudaError_t launch_diag_from_ebe<R>(const Grid&, const R*, R*, cudaStream_t, Counters*);           \
  template cudaError_t launch_invert_diag<R>(const Grid&, R*, int*, cudaStream_t, Counters*);                 \
  template cudaError_t launch_level0_apply<R>(const Grid&, const Phys&, const Vec2<R>::type*,                 \
                                              const Vec2<R>::type*, const Vec2<R>::type*, Vec2<R>::type*,     \
                                              bool, cudaStream_t, Counters*);                                  \
  template cudaError_t launch_ebe_apply<R>(const Grid&, const R*, const Vec2<R>::type*, Vec2<R>::type*, bool, \
                                           cudaStream_t, Counters*);                                           \
  template cudaError_t launch_jacobi_update<R>(const Grid&, const R*, const Vec2<R>::type*,                   \
                                               const Vec2<R>::type*, const Vec2<R>::type*, Vec2<R>::type*, R, \
                                               bool, bool, cudaStream_t, Counters*);                           \
  template cudaError_t launch_sub<R>(const Grid&, const Vec2<R>::type*, const Vec2<R>::type*, Vec2<R>::type*, \
                                     cudaStream_t, Counters*);                                                 \
  template cudaError_t launch_restrict<R>(const Grid&, const Grid&, const Vec2<R>::type*, Vec2<R>::type*,     \
                                          cudaStream_t, Counters*);                                            \
  template cudaError_t launch_prolong_add<R>(const Grid&, const Grid&, const Vec2<R>::type*, Vec2<R>::type*,  \
                                             cudaStream_t, Counters*);                                         \
  template cudaError_t launch_dense_assemble<R>(const Grid&, const R*, double*, int, cudaStream_t, Counters*);\
  template cudaError_t launch_dense_solve<R>(const double*, int, const Vec2<R>::type*, Vec2<R>::type*,        \
                                             long long, bool, cudaStream_t, Counters*);                        \
  template cudaError_t launch_to_mg<R>(const double*, Vec2<R>::type*, long long, cudaStream_t, Counters*);    \
  template cudaError_t launch_from_mg<R>(const Vec2<R>::type*, double*, long long, cudaStream_t, Counters*);

NC_INSTANTIATE_MG(float)
NC_INSTANTIATE_MG(double)

}  // namespace nc
