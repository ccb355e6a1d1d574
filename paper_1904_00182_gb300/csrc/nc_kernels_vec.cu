// Vector, reduction and design-pipeline kernels.
//
// Reductions are deterministic: each block sums a fixed contiguous segment, the partial sums are
// added in a fixed order by one block, so results do not depend on scheduling.
#include "nc_launch.h"

namespace nc {

namespace {

const int kRedThreads = 256;
const int kRedBlocksMax = kReduceBlocksMax;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  __syncthreads();
  return r;
}

// Per-thread accumulation type of the Krylov kernels: FP32 vectors accumulate a thread's few
// entries in FP32 (products of FP32 numbers, about n / 300k terms per thread) and the block and
// grid sums are FP64; FP64 vectors accumulate in FP64 throughout.
template <typename T> struct KAcc { typedef double type; };
template <> struct KAcc<float> { typedef float type; };

// part[i * gridDim.x + b] = sum over segment b of V_i . w. Register tile of NV >= nvec vectors:
// every element of w and of each V_i is read once.
template <int NV, typename T>
__global__ void __launch_bounds__(256) k_multidot_part(const T* __restrict__ V, long long ld, int nvec,
                                                       const T* __restrict__ w, long long n,
                                                       double* __restrict__ part) {
  const int nv = NV <= 12 ? NV : nvec;   // exact tile for small counts: no guarded slots
  typedef typename KAcc<T>::type A;
  __shared__ double sh[32];
  A acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0;
  const long long seg = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = seg * blockIdx.x;
  const long long hi = min(n, lo + seg);
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    const A x = w[t];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) acc[i] += (A)V[(long long)i * ld + t] * x;
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i >= nv) break;
    const double r = block_sum((double)acc[i], sh);
    if (threadIdx.x == 0) part[(long long)i * gridDim.x + blockIdx.x] = r;
  }
}

// One block per vector sums its nb partials: fixed strided assignment, then a fixed shuffle tree.
__global__ void k_sum_parts(const double* __restrict__ part, int nb, int nvec, double* __restrict__ res) {
  __shared__ double sh[32];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(long long)i * nb + b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) res[i] = s;
}

// Gram-Schmidt step after the first-pass dots d1 = (V_i . w for i < nvec, w . w at index nvec).
// With s = sum_i d1_i^2, the Pythagorean norm ww - s of the projected vector is accurate unless the
// projection removed most of w. If ww - s >= ww / 2 (the Daniel-Gragg-Kaufman-Stewart test) the
// pass writes the normalised vector (w - V d1) / sqrt(ww - s) and computes nothing else; otherwise
// it writes w - V d1 and the partial sums of the second-pass dots (V_i . w', w' . w') for a
// re-orthogonalisation. The test reads the same device values in every kernel and on the host.
__device__ __forceinline__ bool cgs_fast(const double* __restrict__ d1, int nvec, double thr, double* s_out,
                                         double* ww_out) {
  double s = 0.0;
  for (int i = 0; i < nvec; ++i) s += d1[i] * d1[i];
  const double ww = d1[nvec];
  *s_out = s;
  *ww_out = ww;
  return ww - s >= thr * ww;
}

template <int NV, typename T>
__global__ void __launch_bounds__(256) k_cgs_update(T* __restrict__ w, const T* __restrict__ V, long long ld,
                                                    int nvec, const double* __restrict__ d1, double thr,
                                                    long long n, double* __restrict__ part) {
  const int nv = NV <= 12 ? NV : nvec;   // exact tile for small counts: no guarded slots
  typedef typename KAcc<T>::type A;
  __shared__ double sh[32];
  double sum2, ww;
  const bool fast = cgs_fast(d1, nv, thr, &sum2, &ww);
  A cc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) cc[i] = i < nv ? (A)d1[i] : (A)0;
  const long long seg = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = seg * blockIdx.x;
  const long long hi = min(n, lo + seg);
  if (fast) {
    const A inv = (A)(1.0 / sqrt(ww - sum2));
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
      A x = w[t];
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nv) x -= cc[i] * (A)V[(long long)i * ld + t];
      w[t] = (T)(x * inv);
    }
    return;
  }
  A acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0;
  A accw = 0;
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    A v[NV];
    A x = w[t];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = i < nv ? (A)V[(long long)i * ld + t] : (A)0;
      x -= cc[i] * v[i];
    }
    w[t] = (T)x;
    x = (A)(T)x;   // the dots see the stored value
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += v[i] * x;
    accw += x * x;
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i >= nv) break;
    const double r = block_sum((double)acc[i], sh);
    if (threadIdx.x == 0) part[(long long)i * gridDim.x + blockIdx.x] = r;
  }
  const double r = block_sum((double)accw, sh);
  if (threadIdx.x == 0) part[(long long)nv * gridDim.x + blockIdx.x] = r;
}

// Sum of the second-pass partials (re-orthogonalisation only).
__global__ void k_cgs_sum(const double* __restrict__ part, int nb, int nvec, const double* __restrict__ d1,
                          double thr, double* __restrict__ d2) {
  double s, ww;
  if (cgs_fast(d1, nvec, thr, &s, &ww)) return;
  __shared__ double sh[32];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(long long)i * nb + b];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) d2[i] = acc;
}

// Re-orthogonalisation: w <- (w - sum_i d2_i V_i) / sqrt(d2[nvec] - sum d2_i^2) (only if the test failed).
template <int NV, typename T>
__global__ void __launch_bounds__(256) k_cgs_reorth(T* __restrict__ w, const T* __restrict__ V, long long ld,
                                                    int nvec, const double* __restrict__ d1, double thr,
                                                    const double* __restrict__ d2, long long n) {
  const int nv = NV <= 12 ? NV : nvec;   // exact tile for small counts: no guarded slots
  typedef typename KAcc<T>::type A;
  double s1, ww1;
  if (cgs_fast(d1, nv, thr, &s1, &ww1)) return;
  A cc[NV];
  double corr = 0.0;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double c = i < nv ? d2[i] : 0.0;
    cc[i] = (A)c;
    corr += c * c;
  }
  const double h2 = d2[nv] - corr;
  const A inv = (A)(h2 > 0.0 ? 1.0 / sqrt(h2) : 0.0);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    A x = w[t];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) x -= cc[i] * (A)V[(long long)i * ld + t];
    w[t] = (T)(x * inv);
  }
}

// Sum of squares over the leading nfree2 entries of a state vector: the free rows for kBcTop, every row
// for kBcCavity (whose fixed entries are zero in every vector this is applied to).
__global__ void k_norm2_free_part(const double* __restrict__ a, long long nfree2, double* __restrict__ part) {
  __shared__ double sh[32];
  const long long seg = (nfree2 + gridDim.x - 1) / gridDim.x;
  const long long lo = seg * blockIdx.x;
  const long long hi = min(nfree2, lo + seg);
  double acc = 0.0;
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) acc += a[t] * a[t];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Plain sum of a vector (segment per block).
__global__ void k_sum_part(const double* __restrict__ a, long long n, double* __restrict__ part) {
  __shared__ double sh[32];
  const long long seg = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = seg * blockIdx.x;
  const long long hi = min(n, lo + seg);
  double acc = 0.0;
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) acc += a[t];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

struct Coef64 { double c[64]; };

// y += sum_i c_i V_i; FP32 basis vectors are combined in FP32 and the sum is added to y in y's type.
template <typename TY, typename T>
__global__ void k_axpy_multi(TY* __restrict__ y, const T* __restrict__ V, long long ld, int nvec,
                             Coef64 coef, long long n) {
  typedef typename KAcc<T>::type A;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    A acc = 0;
    for (int i = 0; i < nvec; ++i) acc += (A)coef.c[i] * (A)V[(long long)i * ld + t];
    y[t] = y[t] + (TY)acc;
  }
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = a * x[t] + b * y[t];
}

template <typename T>
__global__ void k_scale(T* __restrict__ y, double a, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (T)((typename KAcc<T>::type)a * y[t]);
}

template <typename T>
__global__ void k_scale_copy(T* __restrict__ y, const double* __restrict__ x, double a, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (T)(a * x[t]);
}

__global__ void k_cast_d2f(float* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}

__global__ void k_cast_f2d(double* __restrict__ y, const float* __restrict__ x, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (double)x[t];
}

template <typename T>
__global__ void k_zero_dirichlet(Grid g, T* __restrict__ a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!boundary_node(g, t, i, j, k)) return;
  const int b = fixed_bits(g, i, j, k);
  const long long n = i + (long long)g.NX * (j + (long long)g.NY * k);
  if (b & 1) a[2 * n] = (T)0;
  if (b & 2) a[2 * n + 1] = (T)0;
}

__global__ void k_check_design(const double* __restrict__ rho, long long n, int* flag) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = rho[t];
    if (!(v >= 0.0 && v <= 1.0)) atomicExch(flag, 1);   // NaN fails both comparisons
  }
}

// Node n gathers from the (up to 8) elements around it. Element (ei,ej,ek) contains node n as
// local corner a = (i-ei) + 2 (j-ej) + 4 (k-ek).
__global__ void k_filter_rhs(Grid g, Phys ph, bool passive, const double* __restrict__ gamma, double t0,
                             double* __restrict__ b) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  int i, j, k;
  node_ijk(g, n, i, j, k);
  double acc = 0.0;
  for (int dk = -1; dk <= 0; ++dk) {
    const int ek = k + dk;
    if (ek < 0 || ek >= g.nz) continue;
    for (int dj = -1; dj <= 0; ++dj) {
      const int ej = j + dj;
      if (ej < 0 || ej >= g.ny) continue;
      for (int di = -1; di <= 0; ++di) {
        const int ei = i + di;
        if (ei < 0 || ei >= g.nx) continue;
        const double v = !passive || elem_design(ph, ei, ej, ek)
                             ? gamma[ei + (long long)g.nx * (ej + (long long)g.ny * ek)]
                             : (elem_heated(ph, ei, ej, ek) ? 1.0 : 0.0);
        acc += v;
      }
    }
  }
  b[n] = t0 * acc;
}

// (r^2 K + M) x at node (i,j,k). Interior nodes use the constant 27-point stencil C27 (the sum of
// the element matrices of the 8 surrounding elements); nodes on the boundary gather element by
// element from the 8x8 element matrix A.
template <typename R, typename FC>
__device__ __forceinline__ R helm_node(const Grid& g, const FC& F, const R* __restrict__ x, int i, int j, int k,
                                       int n) {
  R acc = R(0);
  if (i > 0 && i < g.nx && j > 0 && j < g.ny && k > 0 && k < g.nz) {
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int oi = o % 3 - 1, oj = (o / 3) % 3 - 1, ok = o / 9 - 1;
      acc += (R)F.C27[o] * x[n + oi + g.NX * oj + g.NXY * ok];
    }
    return acc;
  }
  for (int dk = -1; dk <= 0; ++dk) {
    const int ek = k + dk;
    if (ek < 0 || ek >= g.nz) continue;
    for (int dj = -1; dj <= 0; ++dj) {
      const int ej = j + dj;
      if (ej < 0 || ej >= g.ny) continue;
      for (int di = -1; di <= 0; ++di) {
        const int ei = i + di;
        if (ei < 0 || ei >= g.nx) continue;
        const int a = -di + 2 * (-dj) + 4 * (-dk);
        const int e0 = ei + g.NX * ej + g.NXY * ek;
#pragma unroll
        for (int b = 0; b < 8; ++b) acc += (R)F.A[a * 8 + b] * x[e0 + corner_off(g, b)];
      }
    }
  }
  return acc;
}

template <typename R, typename FC>
__global__ void k_helmholtz(Grid g, FC F, const R* __restrict__ x, R* __restrict__ y) {
  NC_NODE_FLAT(g);
  const int n = pidx + g.NXY * k;
  y[n] = helm_node<R>(g, F, x, i, j, k, n);
}

__global__ void k_cheb_init(long long nn, const float* __restrict__ dinv, const float* __restrict__ r,
                            float* __restrict__ x, float* __restrict__ d, float c0) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  x[n] = 0.f;
  d[n] = c0 * dinv[n] * r[n];
}

__global__ void k_cheb_step(Grid g, FilterConstF F, const float* __restrict__ dinv, const float* __restrict__ d,
                            float* __restrict__ dn, float* __restrict__ x, float* __restrict__ r, float c1, float c2) {
  NC_NODE_FLAT(g);
  const int n = pidx + g.NXY * k;
  const float q = helm_node<float>(g, F, d, i, j, k, n);
  const float dv = d[n];
  x[n] += dv;
  const float rv = r[n] - q;
  r[n] = rv;
  dn[n] = c1 * dv + c2 * dinv[n] * rv;
}

// ---- double-float refinement of the filter solve ----
// b (FP64) -> double-float; the FP32 correction added to the double-float solution; the residual
// r = b - (r^2 K + M) x in double-float arithmetic (element constants in double-float), stored as
// its FP32 leading part (the next inner solve's right-hand side) and as FP64 (for its norm); the
// solution back to FP64.
__global__ void k_d2df(const double* __restrict__ b, df64* __restrict__ bd, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    bd[t] = df_from_double(b[t]);
}

__global__ void k_add_df(df64* __restrict__ x, const float* __restrict__ dx, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    x[t] = x[t] + df64(dx[t], 0.0f);
}

__global__ void k_helm_res_df(Grid g, FilterConstDF F, const df64* __restrict__ b, const df64* __restrict__ x,
                              float* __restrict__ rf, double* __restrict__ r64) {
  NC_NODE_FLAT(g);
  const int n = pidx + g.NXY * k;
  const df64 r = b[n] - helm_node<df64>(g, F, x, i, j, k, n);
  rf[n] = r.hi;
  r64[n] = (double)r.hi + (double)r.lo;
}

__global__ void k_df2d(const df64* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = (double)x[t].hi + (double)x[t].lo;
}

__global__ void k_add_f2d(double* __restrict__ y, const float* __restrict__ x, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] += (double)x[t];
}

__global__ void k_helmholtz_diag(Grid g, double d, double* __restrict__ dinv) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  int i, j, k;
  node_ijk(g, n, i, j, k);
  const int cx = (i > 0) + (i < g.nx), cy = (j > 0) + (j < g.ny), cz = (k > 0) + (k < g.nz);
  dinv[n] = 1.0 / (d * cx * cy * cz);
}

__global__ void k_elem_from_nodes(Grid g, Phys ph, const double* __restrict__ x, double scale,
                                  double heated_value, double* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  int i, j, k;
  elem_ijk(g, e, i, j, k);
  if (heated_value >= 0.0 && !elem_design(ph, i, j, k)) {
    out[e] = elem_heated(ph, i, j, k) ? heated_value : 0.0;
    return;
  }
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) acc += x[corner_node(g, i, j, k, a)];
  out[e] = scale * acc;
}

__global__ void k_ramp(const double* __restrict__ gt, long long n, RampConst r, double2* __restrict__ mat,
                       double2* __restrict__ dmat, float2* __restrict__ mat32) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    // one division per denominator (FP64 divisions dominate this kernel)
    const double x = gt[e];
    const double idc = 1.0 / (1.0 + r.q_c * (1.0 - x));
    const double k = r.k_f + x * idc * (r.k_s - r.k_f);
    const double dk = (r.k_s - r.k_f) * (1.0 + r.q_c) * (idc * idc);
    const double idp = 1.0 / (1.0 + r.q_p * x);
    const double kap = r.kappa_s + (1.0 - x) * idp * (r.kappa_f - r.kappa_s);
    const double dkap = -(r.kappa_f - r.kappa_s) * (1.0 + r.q_p) * (idp * idp);
    mat[e] = make_double2(kap, k);
    dmat[e] = make_double2(dkap, dk);
    mat32[e] = make_float2((float)kap, (float)k);
  }
}

// df/ds for f = (1/|Omega_h|) sum_{e in Omega_h} int_e N t_e: T entry = w_node x (number of heated
// elements around the node; the heated region is a box at the origin corner), P entry 0, Dirichlet
// rows 0.
__global__ void k_dfds(Grid g, Phys ph, double w_node, double* __restrict__ out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  int i, j, k;
  node_ijk(g, n, i, j, k);
  int cnt = 0;
  if (!(fixed_bits(g, i, j, k) & 2)) {
    if (ph.shape == 1) {   // count the heated elements among the (up to 8) around the node
      for (int ek = k - 1; ek <= k; ++ek)
        for (int ej = j - 1; ej <= j; ++ej)
          for (int ei = i - 1; ei <= i; ++ei)
            if (ei >= 0 && ei < g.nx && ej >= 0 && ej < g.ny && ek >= 0 && ek < g.nz && elem_heated(ph, ei, ej, ek))
              ++cnt;
    } else {
      const int hx = min(ph.heat_nx, g.nx), hy = min(ph.heat_ny, g.ny), hz = min(ph.heated_layers, g.nz);
      const int cx = (i > 0 && i - 1 < hx) + (i < hx), cy = (j > 0 && j - 1 < hy) + (j < hy);
      const int cz = (k > 0 && k - 1 < hz) + (k < hz);
      cnt = cx * cy * cz;
    }
  }
  out[2 * n] = 0.0;
  out[2 * n + 1] = w_node * cnt;
}

unsigned stream_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

int reduce_blocks(long long n) {
  long long b = (n + 4095) / 4096;
  if (b > kRedBlocksMax) b = kRedBlocksMax;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t launch_multidot_t(const T* V, long long ld, int nvec, const T* w, long long n,
                              double* part, double* res, cudaStream_t st, Counters* c) {
  const int nb = reduce_blocks(n);
#define NC_MD(NV) k_multidot_part<NV, T><<<nb, kRedThreads, 0, st>>>(V, ld, nvec, w, n, part)
  switch (nvec) {   // exact tiles up to 12 vectors, rounded-up tiles beyond
    case 1: NC_MD(1); break;
    case 2: NC_MD(2); break;
    case 3: NC_MD(3); break;
    case 4: NC_MD(4); break;
    case 5: NC_MD(5); break;
    case 6: NC_MD(6); break;
    case 7: NC_MD(7); break;
    case 8: NC_MD(8); break;
    case 9: NC_MD(9); break;
    case 10: NC_MD(10); break;
    case 11: NC_MD(11); break;
    case 12: NC_MD(12); break;
    default:
      if (nvec <= 16) NC_MD(16);
      else if (nvec <= 32) NC_MD(32);
      else NC_MD(66);
  }
#undef NC_MD
  k_sum_parts<<<nvec, 256, 0, st>>>(part, nb, nvec, res);
  if (c) { c->launches += 2; c->bytes += (double)sizeof(T) * n * (nvec + 1); c->flops += 2.0 * n * nvec; }
  return cudaGetLastError();
}

cudaError_t launch_multidot(const double* V, long long ld, int nvec, const double* w, long long n,
                            double* part, double* res, cudaStream_t st, Counters* c) {
  return launch_multidot_t<double>(V, ld, nvec, w, n, part, res, st, c);
}

cudaError_t launch_multidot(const float* V, long long ld, int nvec, const float* w, long long n,
                            double* part, double* res, cudaStream_t st, Counters* c) {
  return launch_multidot_t<float>(V, ld, nvec, w, n, part, res, st, c);
}

cudaError_t launch_sum(const double* a, long long n, double* part, double* res, cudaStream_t st, Counters* c) {
  const int nb = reduce_blocks(n);
  k_sum_part<<<nb, kRedThreads, 0, st>>>(a, n, part);
  k_sum_parts<<<1, 256, 0, st>>>(part, nb, 1, res);
  if (c) { c->launches += 2; c->bytes += 8.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_norm2_free(const Grid& g, const double* a, double* part, double* res, cudaStream_t st,
                              Counters* c) {
  const long long nfree2 = g.bc == kBcTop ? 2LL * g.NX * g.NY * g.nz : 2LL * g.nn;
  const int nb = reduce_blocks(nfree2);
  k_norm2_free_part<<<nb, kRedThreads, 0, st>>>(a, nfree2, part);
  k_sum_parts<<<1, 256, 0, st>>>(part, nb, 1, res);
  if (c) { c->launches += 2; c->bytes += 8.0 * nfree2; }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cgs_t(T* w, const T* V, long long ld, int nvec, const double* d1, double* d2, long long n,
                         double thr, double* part, cudaStream_t st, Counters* cnt) {
  const int nb = reduce_blocks(n);
  const unsigned ns = stream_blocks(n);
#define NC_CGS(NV)                                                                     \
  do {                                                                                 \
    k_cgs_update<NV, T><<<nb, kRedThreads, 0, st>>>(w, V, ld, nvec, d1, thr, n, part); \
    k_cgs_sum<<<nvec + 1, 256, 0, st>>>(part, nb, nvec, d1, thr, d2);                  \
    k_cgs_reorth<NV, T><<<ns, 256, 0, st>>>(w, V, ld, nvec, d1, thr, d2, n);           \
  } while (0)
  if (nvec <= 12) {   // exact tiles up to 12 vectors
    switch (nvec) {
      case 1: NC_CGS(1); break;
      case 2: NC_CGS(2); break;
      case 3: NC_CGS(3); break;
      case 4: NC_CGS(4); break;
      case 5: NC_CGS(5); break;
      case 6: NC_CGS(6); break;
      case 7: NC_CGS(7); break;
      case 8: NC_CGS(8); break;
      case 9: NC_CGS(9); break;
      case 10: NC_CGS(10); break;
      case 11: NC_CGS(11); break;
      default: NC_CGS(12); break;
    }
  } else if (nvec <= 16) NC_CGS(16);
  else if (nvec <= 32) NC_CGS(32);
  else return cudaErrorInvalidValue;
#undef NC_CGS
  if (cnt) { cnt->launches += 3; cnt->bytes += (double)sizeof(T) * n * (nvec + 2); cnt->flops += 2.0 * n * nvec; }
  return cudaGetLastError();
}

cudaError_t launch_cgs(double* w, const double* V, long long ld, int nvec, const double* d1, double* d2, long long n,
                      double thr, double* part, cudaStream_t st, Counters* cnt) {
  return launch_cgs_t<double>(w, V, ld, nvec, d1, d2, n, thr, part, st, cnt);
}

cudaError_t launch_cgs(float* w, const float* V, long long ld, int nvec, const double* d1, double* d2, long long n,
                      double thr, double* part, cudaStream_t st, Counters* cnt) {
  return launch_cgs_t<float>(w, V, ld, nvec, d1, d2, n, thr, part, st, cnt);
}

template <typename TY, typename T>
cudaError_t launch_axpy_multi_t(TY* y, const T* V, long long ld, int nvec, const double* coef,
                                long long n, cudaStream_t st, Counters* c) {
  if (nvec > 64) return cudaErrorInvalidValue;
  Coef64 cf;
  for (int i = 0; i < nvec; ++i) cf.c[i] = coef[i];
  k_axpy_multi<TY, T><<<stream_blocks(n), 256, 0, st>>>(y, V, ld, nvec, cf, n);
  if (c) { c->launches += 1; c->bytes += (double)n * (sizeof(T) * nvec + 2 * sizeof(TY)); }
  return cudaGetLastError();
}

cudaError_t launch_axpy_multi(double* y, const double* V, long long ld, int nvec, const double* coef,
                              long long n, cudaStream_t st, Counters* c) {
  return launch_axpy_multi_t<double, double>(y, V, ld, nvec, coef, n, st, c);
}

cudaError_t launch_axpy_multi(double* y, const float* V, long long ld, int nvec, const double* coef,
                              long long n, cudaStream_t st, Counters* c) {
  return launch_axpy_multi_t<double, float>(y, V, ld, nvec, coef, n, st, c);
}

cudaError_t launch_axpy_multi(float* y, const float* V, long long ld, int nvec, const double* coef,
                              long long n, cudaStream_t st, Counters* c) {
  return launch_axpy_multi_t<float, float>(y, V, ld, nvec, coef, n, st, c);
}

cudaError_t launch_axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t st,
                         Counters* c) {
  k_axpby<<<stream_blocks(n), 256, 0, st>>>(y, x, a, b, n);
  if (c) { c->launches += 1; c->bytes += 24.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(double* y, const double* x, double a, long long n, cudaStream_t st,
                              Counters* c) {
  k_scale_copy<double><<<stream_blocks(n), 256, 0, st>>>(y, x, a, n);
  if (c) { c->launches += 1; c->bytes += 16.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_scale(double* y, double a, long long n, cudaStream_t st, Counters* c) {
  k_scale<double><<<stream_blocks(n), 256, 0, st>>>(y, a, n);
  if (c) { c->launches += 1; c->bytes += 16.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_scale(float* y, double a, long long n, cudaStream_t st, Counters* c) {
  k_scale<float><<<stream_blocks(n), 256, 0, st>>>(y, a, n);
  if (c) { c->launches += 1; c->bytes += 8.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(float* y, const double* x, double a, long long n, cudaStream_t st,
                              Counters* c) {
  k_scale_copy<float><<<stream_blocks(n), 256, 0, st>>>(y, x, a, n);
  if (c) { c->launches += 1; c->bytes += 12.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_cast_d2f(float* y, const double* x, long long n, cudaStream_t st, Counters* c) {
  k_cast_d2f<<<stream_blocks(n), 256, 0, st>>>(y, x, n);
  if (c) { c->launches += 1; c->bytes += 12.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_cast_f2d(double* y, const float* x, long long n, cudaStream_t st, Counters* c) {
  k_cast_f2d<<<stream_blocks(n), 256, 0, st>>>(y, x, n);
  if (c) { c->launches += 1; c->bytes += 12.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_zero_dirichlet(const Grid& g, double* a, cudaStream_t st, Counters* c) {
  k_zero_dirichlet<<<grid_blocks(boundary_count(g), 256), 256, 0, st>>>(g, a);
  if (c) c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_zero_dirichlet(const Grid& g, float* a, cudaStream_t st, Counters* c) {
  k_zero_dirichlet<<<grid_blocks(boundary_count(g), 256), 256, 0, st>>>(g, a);
  if (c) c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_check_design(const double* rho, long long ne, int* flag, cudaStream_t st) {
  k_check_design<<<stream_blocks(ne), 256, 0, st>>>(rho, ne, flag);
  return cudaGetLastError();
}

cudaError_t launch_filter_rhs(const Grid& g, const Phys& ph, bool passive, const double* gamma, double t0, double* b,
                              cudaStream_t st, Counters* c) {
  k_filter_rhs<<<grid_blocks(g.nn, 256), 256, 0, st>>>(g, ph, passive, gamma, t0, b);
  if (c) { c->launches += 1; c->bytes += 8.0 * (g.ne + g.nn); }
  return cudaGetLastError();
}

cudaError_t launch_helmholtz(const Grid& g, const FilterConst& F, const double* x, double* y, cudaStream_t st,
                             Counters* c) {
  const Launch3 L = launch_nodes_flat(g);
  k_helmholtz<double, FilterConst><<<L.grid, L.block, 0, st>>>(g, F, x, y);
  if (c) { c->launches += 1; c->bytes += 16.0 * g.nn; }
  return cudaGetLastError();
}

cudaError_t launch_cheb_init(long long n, const float* dinv, const float* r, float* x, float* d, float c0,
                             cudaStream_t st, Counters* c) {
  k_cheb_init<<<grid_blocks(n, 256), 256, 0, st>>>(n, dinv, r, x, d, c0);
  if (c) { c->launches += 1; c->bytes += 16.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(const Grid& g, const FilterConstF& F, const float* dinv, const float* d, float* dn,
                             float* x, float* r, float c1, float c2, cudaStream_t st, Counters* c) {
  const Launch3 L = launch_nodes_flat(g);
  k_cheb_step<<<L.grid, L.block, 0, st>>>(g, F, dinv, d, dn, x, r, c1, c2);
  if (c) { c->launches += 1; c->bytes += 32.0 * g.nn; }
  return cudaGetLastError();
}

// Division by the eigenvalues of the filter operator in the cosine basis of each axis:
// t /= r^2 (lx_i my_j mz_k + mx_i ly_j mz_k + mx_i my_j lz_k) + mx_i my_j mz_k, with (l, m) the 1D
// stiffness and mass eigenvalues of the axis.
__global__ void k_filter_scale(Grid g, float* __restrict__ t, const float* __restrict__ lx,
                               const float* __restrict__ mx, const float* __restrict__ ly,
                               const float* __restrict__ my, const float* __restrict__ lz,
                               const float* __restrict__ mz, float r2) {
  NC_NODE_FLAT(g);
  const float ax = lx[i], bx = mx[i], ay = ly[j], by = my[j], az = lz[k], bz = mz[k];
  const float byz = by * bz;
  const float d = r2 * (ax * byz + bx * (ay * bz + by * az)) + bx * byz;
  const long long n = pidx + (long long)g.NXY * k;
  t[n] = t[n] / d;
}

cudaError_t launch_filter_scale(const Grid& g, float* t, const float* const lam[3], const float* const mu[3],
                                float r2, cudaStream_t st, Counters* c) {
  const Launch3 L = launch_nodes_flat(g);
  k_filter_scale<<<L.grid, L.block, 0, st>>>(g, t, lam[0], mu[0], lam[1], mu[1], lam[2], mu[2], r2);
  if (c) { c->launches += 1; c->bytes += 8.0 * g.nn; }
  return cudaGetLastError();
}

cudaError_t launch_filter_df(int op, const Grid& g, const FilterConstDF* F, const double* b64, df64* bd, df64* x,
                             const float* dx, float* rf, double* r64, double* y64, cudaStream_t st, Counters* c) {
  const long long n = g.nn;
  switch (op) {
    case 0: k_d2df<<<stream_blocks(n), 256, 0, st>>>(b64, bd, n); if (c) c->bytes += 16.0 * n; break;
    case 1: k_add_df<<<stream_blocks(n), 256, 0, st>>>(x, dx, n); if (c) c->bytes += 20.0 * n; break;
    case 2: {
      const Launch3 L = launch_nodes_flat(g);
      k_helm_res_df<<<L.grid, L.block, 0, st>>>(g, *F, bd, x, rf, r64);
      if (c) c->bytes += 28.0 * n;
      break;
    }
    default: k_df2d<<<stream_blocks(n), 256, 0, st>>>(x, y64, n); if (c) c->bytes += 16.0 * n; break;
  }
  if (c) c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_add_f2d(double* y, const float* x, long long n, cudaStream_t st, Counters* c) {
  k_add_f2d<<<stream_blocks(n), 256, 0, st>>>(y, x, n);
  if (c) { c->launches += 1; c->bytes += 20.0 * n; }
  return cudaGetLastError();
}

cudaError_t launch_helmholtz_diag(const Grid& g, const FilterConst& F, double* dinv, cudaStream_t st) {
  k_helmholtz_diag<<<grid_blocks(g.nn, 256), 256, 0, st>>>(g, F.diag, dinv);
  return cudaGetLastError();
}

cudaError_t launch_elem_from_nodes(const Grid& g, const Phys& ph, const double* x, double scale,
                                   double heated_value, double* out, cudaStream_t st, Counters* c) {
  k_elem_from_nodes<<<grid_blocks(g.ne, 256), 256, 0, st>>>(g, ph, x, scale, heated_value, out);
  if (c) { c->launches += 1; c->bytes += 8.0 * (g.ne + g.nn); }
  return cudaGetLastError();
}

cudaError_t launch_ramp(const double* gt, long long ne, const RampConst& r, double2* mat, double2* dmat,
                        float2* mat32, cudaStream_t st, Counters* c) {
  k_ramp<<<stream_blocks(ne), 256, 0, st>>>(gt, ne, r, mat, dmat, mat32);
  if (c) { c->launches += 1; c->bytes += 48.0 * ne; }
  return cudaGetLastError();
}

cudaError_t launch_dfds(const Grid& g, const Phys& ph, double w_node, double* out, cudaStream_t st,
                        Counters* c) {
  k_dfds<<<grid_blocks(g.nn, 256), 256, 0, st>>>(g, ph, w_node, out);
  if (c) { c->launches += 1; c->bytes += 16.0 * g.nn; }
  return cudaGetLastError();
}

}  // namespace nc
