// C ABI of the natconv library: problem object, design pipeline, damped Newton state solve,
// FGMRES with a geometric-multigrid preconditioner, adjoint and sensitivities.
//
// Method (paper sections): design pipeline Sec. 5.1-5.2 (PDE filter, RAMP); Newton with a
// residual-minimising damping factor, stopping on a relative residual reduction and ramping the
// heat source when it fails (Sec. 5.4); linear solves by flexible GMRES (Sec. 5.4, Table 4);
// adjoint sensitivities (Sec. 5.1). The multigrid preconditioner and the precision split are this
// library's design: in NC_PREC_MIXED the V-cycle and the Krylov operator run in FP32 while the
// Newton residual, the Krylov orthogonalisation and the coarse solve are FP64, so the outer FP64
// Newton (state) and refinement (adjoint) iterations recover FP64 accuracy.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <cublas_v2.h>

#include "natconv.h"
#include "nc_launch.h"

using namespace nc;

namespace {

const int kMaxRestart = 64;
const size_t kBlasWorkspace = 32u << 20;   // cuBLAS workspace of the spectral filter transforms


double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Damping of Sec. 5.4 and the Newton forcing term, shared by state solve and tests.
double kappa_f_tuned(double alpha, double dT) {
  // Eq. nusselt5 with H = 1, L = 0.5, beta_m = nu = g = Pr = 1.
  const double H = 1.0, L = 0.5, Pr = 1.0;
  return std::pow(H, 1.74) / (std::pow(alpha * dT, 0.42) * L * L) * 0.0324 *
         std::pow(Pr * Pr / (0.2 + Pr), 0.58);
}

struct Levels {
  std::vector<Grid> g;
  int nf = 0;   // free DOFs of the coarsest level
};

Levels plan_levels(const Grid& g0, int max_levels) {
  Levels L;
  L.g.push_back(g0);
  while (true) {
    const Grid& c = L.g.back();
    if (max_levels > 0 && (int)L.g.size() >= max_levels) break;
    if (c.nx % 2 || c.ny % 2 || c.nz % 2) break;
    Grid gc = make_grid(c.nx / 2, c.ny / 2, c.nz / 2, c.h * 2.0);
    gc.bc = g0.bc;
    L.g.push_back(gc);
  }
  L.nf = coarse_rows(L.g.back());
  return L;
}

template <typename R>
struct MG {
  typedef typename Vec2<R>::type R2;
  std::vector<MGLevelDev<R>> lev;
  double* Ac = nullptr;     // coarsest-level Galerkin matrix (FP64, free DOFs)
  float* Ainv32 = nullptr; // its FP32 inverse
  float* W = nullptr;      // Gauss-Jordan scratch (nf x 2nf, then 3 nf of pivot bookkeeping)
  double* cw = nullptr;    // coarse-solve scratch (3 nf)
  int nf = 0;
  // during a preconditioner call with FP64 vectors: its input (read by the first finest-level
  // update) and output (written by the last one); null otherwise
  const double* in64 = nullptr;
  double* out64 = nullptr;
  bool factored = false;   // Ainv32 holds an inverse of some earlier coarsest matrix
  // the V-cycle below the finest level (levels 1 .. L-1) captured as a CUDA graph, per direction
  // (0: A, 1: A^T), and the counters its launches add
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  Counters graph_cnt[2];
};

}  // namespace

struct nc_problem {
  int device = 0;
  Grid g;
  nc_params par;
  Phys ph;
  double Q_full = 0.0, kappa_f = 0.0, kappa_s = 0.0, vol_h = 0.0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<void*> allocs;
  size_t bytes = 0;
  // state, design
  double2 *s = nullptr, *s_try = nullptr, *lam = nullptr, *s_start = nullptr;
  double *R = nullptr, *R_try = nullptr, *dx = nullptr, *w = nullptr, *rhs = nullptr;
  double *rho = nullptr, *gamma_t = nullptr, *gsens = nullptr, *u = nullptr;
  double2 *mat = nullptr, *dmat = nullptr;
  double2* dl = nullptr;   // element (dL/dkappa, dL/dk) at the adjoint solution (see dl_ready)
  bool dl_ready = false;   // dl holds the derivatives of the current lambda
  float2 *mat32 = nullptr, *s32 = nullptr, *v32 = nullptr, *y32 = nullptr;
  float4* fz = nullptr;   // frozen (u0, tau) per element of the Picard finest-level operator (NC_MGOP_PICARD)
  // double-float copies (mixed path with NC_ARITH_DF64): materials per element, split scratch per node
  float4 *mat_df = nullptr, *s_df = nullptr, *w_df = nullptr;
  // Krylov
  int m = 30;
  double *V = nullptr, *Z = nullptr;      // FP64 basis (NC_PREC_FP64)
  float *V32 = nullptr, *Z32 = nullptr;   // FP32 basis (mixed precision)
  double *part = nullptr, *dres = nullptr, *hres = nullptr;
  // filter PCG (node vectors)
  double *fx = nullptr, *fb = nullptr, *fr = nullptr, *fq = nullptr, *fdinv = nullptr;
  float *fxf = nullptr, *frf = nullptr, *fd0 = nullptr, *fd1 = nullptr, *fdinvf = nullptr;
  FilterConst F;
  FilterConstF Ff;
  FilterConstDF Fd;                   // the filter element constants in double-float
  df64 *fxd = nullptr, *fbd = nullptr; // double-float solution and right-hand side of the refinement
  double cheb_a = 0.0, cheb_b = 0.0;   // bounds of the spectrum of D^-1 (r^2 K + M)
  int cheb_iters = 0;                  // FP32 Chebyshev steps per refinement pass
  // spectral filter solve: per axis the cosine matrix C_ij = cos(pi i j / n) (FP32, symmetric) and
  // the eigenvalues of the 1D stiffness and mass matrices in that basis; the cuBLAS handle of the
  // axis transforms (dense FP32 GEMMs) and its workspace
  float* fC[3] = {nullptr, nullptr, nullptr};
  float* flam[3] = {nullptr, nullptr, nullptr};
  float* fmu[3] = {nullptr, nullptr, nullptr};
  cublasHandle_t blas = nullptr;
  void* blas_ws = nullptr;
  // multigrid
  Levels lv;
  MG<float> mg32;
  MG<double> mg64;
  int *dflag = nullptr, *hflag = nullptr;
  // bookkeeping
  int stage = 0;         // 0 created, 1 design set, 2 state solved, 3 adjoint solved
  bool start_zero = true; // the Newton start is the zero state (its residual is R0)
  bool first_setup = true; // next multigrid set-up is the first of this solve call
  bool mg_ready = false;   // a hierarchy from this state solve exists (reused by the adjoint)
  bool have_R0 = false;   // R0 = R(0) with the full source: minus the SUPG-weighted source load,
  double* R0 = nullptr;   // which does not depend on the design (u = 0, N* = N at s = 0)
  double ref_norm = 0.0; // ||R_free(0)|| with the full source
  double t_start = 0.0;
  Counters cnt;       // per call
  Counters total;     // since creation
  // per-launch event timing of kernel classes (nc_set_profiling)
  struct Pending { int cls; cudaEvent_t a, b; double bytes, flops; };
  int prof_mask = 0;
  std::vector<cudaEvent_t> evpool;
  std::vector<Pending> pending;
  double prof_ms[NC_PROF_NCLASSES] = {0};
  long long prof_n[NC_PROF_NCLASSES] = {0};
  double prof_bytes[NC_PROF_NCLASSES] = {0};
  double prof_flops[NC_PROF_NCLASSES] = {0};
};

namespace {

thread_local std::string g_create_error = "no error";   // per thread: problems are created from several threads

nc_status fail(nc_problem* pb, nc_status s, const std::string& msg) {
  if (pb) pb->err = msg; else g_create_error = msg;
  return s;
}

nc_status cuda_fail(nc_problem* pb, cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error in %s: %s", what, cudaGetErrorString(e));
  return fail(pb, e == cudaErrorMemoryAllocation ? NC_ERR_OOM : NC_ERR_CUDA, buf);
}

#define CK(x)                                                   \
  do {                                                          \
    cudaError_t _e = (x);                                       \
    if (_e != cudaSuccess) return cuda_fail(pb, _e, #x);        \
  } while (0)

#define CKS(x)                                                  \
  do {                                                          \
    nc_status _s = (x);                                         \
    if (_s != NC_OK) return _s;                                 \
  } while (0)

cudaEvent_t prof_event(nc_problem* pb) {
  if (!pb->evpool.empty()) {
    cudaEvent_t e = pb->evpool.back();
    pb->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Accumulate the timed launches whose events have completed (called after a stream sync).
void prof_flush(nc_problem* pb) {
  for (auto& p : pb->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      pb->prof_ms[p.cls] += ms;
      pb->prof_n[p.cls] += 1;
      pb->prof_bytes[p.cls] += p.bytes;
      pb->prof_flops[p.cls] += p.flops;
    } else {
      cudaGetLastError();
    }
    pb->evpool.push_back(p.a);
    pb->evpool.push_back(p.b);
  }
  pb->pending.clear();
}

// Brackets one launch of class cls with timing events when profiling is on.
struct ProfScope {
  nc_problem* pb;
  int cls;
  cudaEvent_t a = nullptr;
  double bytes0, flops0;
  ProfScope(nc_problem* p, int c) : pb(p), cls(c), bytes0(p->cnt.bytes), flops0(p->cnt.flops) {
    if (((pb->prof_mask >> cls) & 1) && (a = prof_event(pb))) cudaEventRecord(a, pb->st);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(pb);
    if (!b) { pb->evpool.push_back(a); return; }
    cudaEventRecord(b, pb->st);
    pb->pending.push_back({cls, a, b, pb->cnt.bytes - bytes0, pb->cnt.flops - flops0});
    if (pb->pending.size() > 4096) {
      cudaStreamSynchronize(pb->st);
      prof_flush(pb);
    }
  }
};

#define PCK(cls, x)                                             \
  do {                                                          \
    ProfScope _ps(pb, cls);                                     \
    cudaError_t _e = (x);                                       \
    if (_e != cudaSuccess) return cuda_fail(pb, _e, #x);        \
  } while (0)

template <typename T>
nc_status dalloc(nc_problem* pb, T** p, size_t count) {
  size_t b = sizeof(T) * std::max<size_t>(count, 1);
  b = (b + 255) & ~size_t(255);
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof(buf), "cudaMalloc of %zu bytes failed: %s", b, cudaGetErrorString(e));
    return fail(pb, NC_ERR_OOM, buf);
  }
  pb->allocs.push_back(q);
  pb->bytes += b;
  *p = (T*)q;
  return NC_OK;
}

nc_status sync(nc_problem* pb, const char* what) {
  cudaError_t e = cudaStreamSynchronize(pb->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(pb, e, what);
  if (!pb->pending.empty()) prof_flush(pb);
  return NC_OK;
}

nc_status check_timeout(nc_problem* pb) {
  if (now_s() - pb->t_start > pb->par.timeout_s) return fail(pb, NC_ERR_TIMEOUT, "call exceeded timeout_s");
  return NC_OK;
}

// ---------------------------------------------------------------- reductions -------
template <typename T>
nc_status dots(nc_problem* pb, const T* V, long long ld, int nvec, const T* w, long long n, double* out) {
  PCK(NC_PROF_KRYLOV_VEC, launch_multidot(V, ld, nvec, w, n, pb->part, pb->dres, pb->st, &pb->cnt));
  CK(cudaMemcpyAsync(pb->hres, pb->dres, sizeof(double) * nvec, cudaMemcpyDeviceToHost, pb->st));
  CKS(sync(pb, "dot products"));
  for (int i = 0; i < nvec; ++i) out[i] = pb->hres[i];
  return NC_OK;
}

nc_status norm2_free(nc_problem* pb, const double* a, double* out) {
  PCK(NC_PROF_KRYLOV_VEC, launch_norm2_free(pb->g, a, pb->part, pb->dres, pb->st, &pb->cnt));
  CK(cudaMemcpyAsync(pb->hres, pb->dres, sizeof(double), cudaMemcpyDeviceToHost, pb->st));
  CKS(sync(pb, "norm"));
  *out = pb->hres[0];
  return NC_OK;
}

// ---------------------------------------------------------------- design pipeline --
// (r^2 K + M) fx = fb, FP64 result. Each refinement pass solves the correction equation for the
// current FP64 residual with a fixed number of FP32 Chebyshev steps (Jacobi-preconditioned, bounds
// from the stencil's Fourier symbol, no reductions), then recomputes the residual in FP64.
// Direct FP32 solve of the filter system (r^2 K + M) x = b on the node grid (homogeneous Neumann
// boundaries, uniform h). The 1D Q1 stiffness and consistent mass matrices with Neumann ends are
// both diagonalised by the cosine matrix C_ij = cos(pi i j / n) (C^T K C and C^T M C are diagonal),
// so with C3 = Cx (x) Cy (x) Cz the 3D operator r^2 (K M M + M K M + M M K) + M M M satisfies
// C3^T A C3 = D diagonal and x = C3 D^-1 C3^T b (C symmetric: C3^T = C3). Each axis transform is one
// dense FP32 GEMM with the axis' cosine matrix (a batch of them for the middle axis); fd0 and fd1
// are the work vectors. The FP64 refinement of filter_solve corrects the FP32 rounding.
cudaError_t spectral_filter(nc_problem* pb, const float* in, float* out) {
  const Grid& g = pb->g;
  const int NX = g.NX, NY = g.NY, NZ = g.NZ, NXY = g.NXY;
  const float one = 1.0f, zero = 0.0f;
  float* t1 = pb->fd0;
  float* t2 = pb->fd1;
  auto ok = [](cublasStatus_t e) { return e == CUBLAS_STATUS_SUCCESS; };
  auto tx = [&](const float* a, float* b) {   // along x: b = Cx a, a as NX x (NY NZ)
    return ok(cublasSgemm(pb->blas, CUBLAS_OP_N, CUBLAS_OP_N, NX, NY * NZ, NX, &one, pb->fC[0], NX, a, NX, &zero, b, NX));
  };
  auto ty = [&](const float* a, float* b) {   // along y: per z plane b_k = a_k Cy, a_k as NX x NY
    return ok(cublasSgemmStridedBatched(pb->blas, CUBLAS_OP_N, CUBLAS_OP_N, NX, NY, NY, &one, a, NX, NXY, pb->fC[1],
                                        NY, 0, &zero, b, NX, NXY, NZ));
  };
  auto tz = [&](const float* a, float* b) {   // along z: b = a Cz, a as (NX NY) x NZ
    return ok(cublasSgemm(pb->blas, CUBLAS_OP_N, CUBLAS_OP_N, NXY, NZ, NZ, &one, a, NXY, pb->fC[2], NZ, &zero, b, NXY));
  };
  if (!tx(in, t1) || !ty(t1, t2) || !tz(t2, t1)) return cudaErrorUnknown;
  const double r = pb->par.filter_radius * g.h / (2.0 * std::sqrt(3.0));
  cudaError_t e = launch_filter_scale(g, t1, pb->flam, pb->fmu, (float)(r * r), pb->st, nullptr);
  if (e != cudaSuccess) return e;
  if (!tx(t1, t2) || !ty(t2, t1) || !tz(t1, out)) return cudaErrorUnknown;
  pb->cnt.launches += 7;
  pb->cnt.bytes += 4.0 * 13.0 * g.nn;   // six transforms read and write the vector, the scaling reads it
  pb->cnt.flops += 4.0 * g.nn * (NX + NY + NZ) + 8.0 * g.nn;
  return cudaGetLastError();
}

// Cosine matrices and 1D eigenvalues of the spectral filter solve (per axis, from the grid alone),
// and the cuBLAS handle on the problem's stream with a workspace from the problem's allocations.
nc_status spectral_setup(nc_problem* pb) {
  const Grid& g = pb->g;
  const int ns[3] = {g.nx, g.ny, g.nz};
  const double h = g.h;
  for (int d = 0; d < 3; ++d) {
    const int n = ns[d], N = n + 1;
    std::vector<float> C((size_t)N * N), lam(N), mu(N);
    std::vector<double> v(N);
    for (int j = 0; j < N; ++j) {
      for (int i = 0; i < N; ++i) {
        // cos(pi i j / n) with the argument reduced to [0, 2 pi) in integers
        v[i] = std::cos(M_PI * (double)(((long long)i * j) % (2LL * n)) / n);
        C[(size_t)j * N + i] = (float)v[i];
      }
      // v^T K v and v^T M v with the assembled 1D matrices: K = (1/h) tridiag(-1, 2, -1), M = (h/6)
      // tridiag(1, 4, 1), their end rows halved on the diagonal (Neumann ends)
      double kv = 0.0, mv = 0.0;
      for (int i = 0; i < N; ++i) {
        const bool end = (i == 0 || i == n);
        double Kv = (end ? 1.0 : 2.0) * v[i], Mv = (end ? 2.0 : 4.0) * v[i];
        if (i > 0) { Kv -= v[i - 1]; Mv += v[i - 1]; }
        if (i < n) { Kv -= v[i + 1]; Mv += v[i + 1]; }
        kv += v[i] * Kv / h;
        mv += v[i] * Mv * h / 6.0;
      }
      lam[j] = (float)kv;
      mu[j] = (float)mv;
    }
    CKS(dalloc(pb, &pb->fC[d], (size_t)N * N));
    CKS(dalloc(pb, &pb->flam[d], (size_t)N));
    CKS(dalloc(pb, &pb->fmu[d], (size_t)N));
    CK(cudaMemcpy(pb->fC[d], C.data(), sizeof(float) * C.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pb->flam[d], lam.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pb->fmu[d], mu.data(), sizeof(float) * N, cudaMemcpyHostToDevice));
  }
  if (cublasCreate(&pb->blas) != CUBLAS_STATUS_SUCCESS) { pb->blas = nullptr; return fail(pb, NC_ERR_CUDA, "cublasCreate failed"); }
  CKS(dalloc(pb, (char**)&pb->blas_ws, kBlasWorkspace));
  if (cublasSetStream(pb->blas, pb->st) != CUBLAS_STATUS_SUCCESS ||
      cublasSetMathMode(pb->blas, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS ||
      cublasSetWorkspace(pb->blas, pb->blas_ws, kBlasWorkspace) != CUBLAS_STATUS_SUCCESS)
    return fail(pb, NC_ERR_CUDA, "cuBLAS set-up failed");
  return NC_OK;
}

// The filter system solved to filter_rtol by iterative refinement around an FP32 inner solve
// (spectral or Chebyshev). On the mixed-precision path, with filter_rtol >= 1e-13, the refinement
// keeps its solution and forms its residual in double-float arithmetic (about 48 significant bits:
// the residual's rounding stays near 1e-14 of its terms) on the FP32 pipes; otherwise in FP64.
nc_status filter_solve(nc_problem* pb) {
  const Grid& g = pb->g;
  const long long n = g.nn;
  double bb;
  CKS(dots(pb, pb->fb, 0, 1, pb->fb, n, &bb));
  PCK(NC_PROF_FILTER, cudaMemsetAsync(pb->fx, 0, sizeof(double) * n, pb->st));
  if (bb == 0.0) return NC_OK;
  const bool df = pb->par.precision != NC_PREC_FP64 && pb->par.filter_rtol >= 1e-13;
  if (df) {
    PCK(NC_PROF_FILTER, launch_filter_df(0, g, nullptr, pb->fb, pb->fbd, nullptr, nullptr, nullptr, nullptr, nullptr,
                                         pb->st, &pb->cnt));
    PCK(NC_PROF_FILTER, cudaMemsetAsync(pb->fxd, 0, sizeof(df64) * n, pb->st));
  }
  PCK(NC_PROF_FILTER, launch_cast_d2f(pb->frf, pb->fb, n, pb->st, &pb->cnt));
  const double a = pb->cheb_a, b = pb->cheb_b;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  const double tol2 = pb->par.filter_rtol * pb->par.filter_rtol * bb;
  for (int pass = 0; pass < 12; ++pass) {
    // correction fxf from the FP32 residual frf
    if (pb->par.filter_method == NC_FILTER_SPECTRAL) {
      PCK(NC_PROF_FILTER, spectral_filter(pb, pb->frf, pb->fxf));
    } else {
      PCK(NC_PROF_FILTER, launch_cheb_init(n, pb->fdinvf, pb->frf, pb->fxf, pb->fd0, (float)(1.0 / theta), pb->st,
                                           &pb->cnt));
      double rho = 1.0 / sigma;
      float* d0 = pb->fd0;
      float* d1 = pb->fd1;
      for (int it = 0; it < pb->cheb_iters; ++it) {
        const double rho1 = 1.0 / (2.0 * sigma - rho);
        PCK(NC_PROF_FILTER, launch_cheb_step(g, pb->Ff, pb->fdinvf, d0, d1, pb->fxf, pb->frf, (float)(rho1 * rho),
                                             (float)(2.0 * rho1 / delta), pb->st, &pb->cnt));
        rho = rho1;
        std::swap(d0, d1);
      }
    }
    if (df) {
      PCK(NC_PROF_FILTER, launch_filter_df(1, g, nullptr, nullptr, nullptr, pb->fxd, pb->fxf, nullptr, nullptr, nullptr,
                                           pb->st, &pb->cnt));
      PCK(NC_PROF_FILTER, launch_filter_df(2, g, &pb->Fd, nullptr, pb->fbd, pb->fxd, nullptr, pb->frf, pb->fr, nullptr,
                                           pb->st, &pb->cnt));
    } else {
      PCK(NC_PROF_FILTER, launch_add_f2d(pb->fx, pb->fxf, n, pb->st, &pb->cnt));
      PCK(NC_PROF_FILTER, launch_helmholtz(g, pb->F, pb->fx, pb->fq, pb->st, &pb->cnt));
      CK(cudaMemcpyAsync(pb->fr, pb->fb, sizeof(double) * n, cudaMemcpyDeviceToDevice, pb->st));
      PCK(NC_PROF_FILTER, launch_axpby(pb->fr, pb->fq, -1.0, 1.0, n, pb->st, &pb->cnt));
      PCK(NC_PROF_FILTER, launch_cast_d2f(pb->frf, pb->fr, n, pb->st, &pb->cnt));
    }
    double rr;
    CKS(dots(pb, pb->fr, 0, 1, pb->fr, n, &rr));
    if (!std::isfinite(rr)) return fail(pb, NC_ERR_NAN, "non-finite residual in the filter solve");
    if (rr <= tol2) {
      if (df)
        PCK(NC_PROF_FILTER, launch_filter_df(3, g, nullptr, nullptr, nullptr, pb->fxd, nullptr, nullptr, nullptr, pb->fx,
                                             pb->st, &pb->cnt));
      return NC_OK;
    }
  }
  return fail(pb, NC_ERR_MAXIT, "filter refinement did not converge");
}

// ---------------------------------------------------------------- operators --------
// Outer residuals (Newton residual, adjoint refinement residual, sensitivities) in double-float?
bool outer_df(const nc_problem* pb) {
  return pb->par.precision != NC_PREC_FP64 && pb->par.outer_arith == NC_ARITH_DF64;
}

// J(s)^T w in the arithmetic of the outer residuals; dl (nullable): element design derivatives of
// w . R stored by the same pass.
nc_status outer_jtv(nc_problem* pb, int cls, const double2* s, const double2* w, double* out, double2* dl = nullptr) {
  if (outer_df(pb))
    PCK(cls, launch_jtv_df(pb->g, pb->ph, s, pb->mat_df, pb->s_df, w, pb->w_df, out, dl, pb->st, &pb->cnt));
  else
    PCK(cls, launch_jtv_f64(pb->g, pb->ph, s, pb->mat, w, out, dl, pb->st, &pb->cnt));
  return NC_OK;
}

// Adjoint refinement residual w = df/ds - J^T lambda on the free rows, rr = ||w||^2. steer: J^T lambda
// in double-float (a residual that only steers the next correction); otherwise in the arithmetic of
// the outer residuals, storing the element design derivatives in dl.
nc_status adjoint_residual(nc_problem* pb, bool steer, double* rr) {
  const long long n = 2 * pb->g.nn;
  if (steer)
    PCK(NC_PROF_ADJ_DF64, launch_jtv_df(pb->g, pb->ph, pb->s, pb->mat_df, pb->s_df, pb->lam, pb->w_df, pb->w, nullptr,
                                        pb->st, &pb->cnt));
  else
    CKS(outer_jtv(pb, NC_PROF_OUTER_OP64, pb->s, pb->lam, pb->w, pb->dl));
  PCK(NC_PROF_OTHER, launch_axpby(pb->w, pb->rhs, 1.0, -1.0, n, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(pb->g, pb->w, pb->st, &pb->cnt));
  CKS(norm2_free(pb, pb->w, rr));
  return NC_OK;
}

nc_status residual(nc_problem* pb, const double2* s, double* R, double* phi) {
  if (outer_df(pb))
    PCK(NC_PROF_RESIDUAL, launch_residual_df(pb->g, pb->ph, s, pb->mat_df, pb->s_df, R, pb->st, &pb->cnt));
  else
    PCK(NC_PROF_RESIDUAL, launch_residual(pb->g, pb->ph, s, pb->mat, R, pb->st, &pb->cnt));
  CKS(norm2_free(pb, R, phi));
  if (!std::isfinite(*phi)) return fail(pb, NC_ERR_NAN, "non-finite residual");
  return NC_OK;
}

// Outer Krylov operator: J(s) or J(s)^T, FP64 or FP32 arithmetic. The FP32 product casts x to
// FP32, applies the same matrix-free kernel as the multigrid's finest level (FP32 state copy s32)
// and casts the result back.
nc_status outer_op(nc_problem* pb, bool transpose, bool fp32, const double* x, double* y) {
  const Grid& g = pb->g;
  if (fp32) {
    PCK(NC_PROF_OUTER_OP32, launch_cast_d2f((float*)pb->v32, x, 2 * g.nn, pb->st, &pb->cnt));
    PCK(NC_PROF_OUTER_OP32, launch_level0_apply<float>(g, pb->ph, pb->s32, pb->mat32, pb->v32, pb->y32, transpose,
                                                       pb->st, &pb->cnt, pb->par.elem_chunk));
    PCK(NC_PROF_OUTER_OP32, launch_cast_f2d(y, (const float*)pb->y32, 2 * g.nn, pb->st, &pb->cnt));
  } else {
    if (transpose) PCK(NC_PROF_OUTER_OP64, launch_jtv_f64(g, pb->ph, pb->s, pb->mat, (const double2*)x, y, nullptr, pb->st, &pb->cnt));
    else PCK(NC_PROF_OUTER_OP64, launch_jv_f64(g, pb->ph, pb->s, pb->mat, (const double2*)x, y, pb->st, &pb->cnt));
  }
  // with kBcTop the element kernels leave the Dirichlet rows zero; otherwise they are zeroed here
  if (g.bc != kBcTop) PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, y, pb->st, &pb->cnt));
  return NC_OK;
}

// The FP32 state copy used by the FP32 Krylov operator and the finest multigrid level, and with
// NC_MGOP_PICARD the frozen coefficients of the finest-level operator at that state.
nc_status refresh_state32(nc_problem* pb, const double2* s, int cls) {
  PCK(cls, launch_cast_d2f((float*)pb->s32, (const double*)s, 2 * pb->g.nn, pb->st, &pb->cnt));
  if (pb->par.mg_op0 == NC_MGOP_PICARD)
    PCK(cls, launch_frozen(pb->g, pb->ph, pb->s32, pb->mat32, pb->fz, pb->st, &pb->cnt));
  return NC_OK;
}

// ---------------------------------------------------------------- multigrid --------
template <typename R> MG<R>& mg_of(nc_problem* pb);
template <> MG<float>& mg_of<float>(nc_problem* pb) { return pb->mg32; }
template <> MG<double>& mg_of<double>(nc_problem* pb) { return pb->mg64; }

template <typename R> const typename Vec2<R>::type* mg_state(nc_problem* pb);
template <> const float2* mg_state<float>(nc_problem* pb) { return pb->s32; }
template <> const double2* mg_state<double>(nc_problem* pb) { return pb->s; }
template <typename R> const typename Vec2<R>::type* mg_mat(nc_problem* pb);
template <> const float2* mg_mat<float>(nc_problem* pb) { return pb->mat32; }
template <> const double2* mg_mat<double>(nc_problem* pb) { return pb->mat; }

template <typename R>
nc_status mg_alloc(nc_problem* pb) {
  MG<R>& mg = mg_of<R>(pb);
  const int L = (int)pb->lv.g.size();
  mg.lev.resize(L);
  for (int l = 0; l < L; ++l) {
    MGLevelDev<R>& d = mg.lev[l];
    d.g = pb->lv.g[l];
    CKS(dalloc(pb, &d.x, d.g.nn));
    CKS(dalloc(pb, &d.xn, d.g.nn));
    CKS(dalloc(pb, &d.b, d.g.nn));
    CKS(dalloc(pb, &d.y, d.g.nn));
    d.S = nullptr;
    d.ebe = nullptr;
    d.dinv = nullptr;
    d.lf = nullptr;
    if (l < L - 1) CKS(dalloc(pb, &d.dinv, 4 * d.g.nn));
    if (pb->par.mg_smoother == NC_SMOOTH_ZLINE && l > 0 && l < L - 1) CKS(dalloc(pb, &d.lf, 24 * d.g.nn));
    if (l > 0) CKS(dalloc(pb, &d.ebe, 256 * d.g.ne));
    if (l > 0 && l < L - 1) CKS(dalloc(pb, &d.S, 108 * d.g.nn));
  }
  mg.nf = pb->lv.nf;
  CKS(dalloc(pb, &mg.Ac, (size_t)mg.nf * mg.nf));
  CKS(dalloc(pb, &mg.Ainv32, (size_t)mg.nf * mg.nf));
  CKS(dalloc(pb, &mg.W, (size_t)mg.nf * 2 * mg.nf + 3 * (size_t)mg.nf));   // + pivot bookkeeping
  CKS(dalloc(pb, &mg.cw, (size_t)3 * mg.nf));
  return NC_OK;
}

template <typename R>
nc_status mg_setup(nc_problem* pb, bool refactor) {
  MG<R>& mg = mg_of<R>(pb);
  const int L = (int)mg.lev.size();
  if (sizeof(R) == 4) CKS(refresh_state32(pb, pb->s, NC_PROF_MG_COARSE_SETUP));
  for (int l = 0; l < L - 1; ++l) CK(cudaMemsetAsync(mg.lev[l].dinv, 0, sizeof(R) * 4 * mg.lev[l].g.nn, pb->st));
  CK(cudaMemsetAsync(pb->dflag, 0, sizeof(int), pb->st));
  if (L == 1) return fail(pb, NC_ERR_ARG, "grid dimensions must be even for the multigrid hierarchy");
  // the hierarchy of the frozen-coefficient operator (mixed precision, mg_galerkin = NC_MGOP_PICARD) or of J(s)
  const bool gal_picard = sizeof(R) == 4 && pb->par.mg_galerkin == NC_MGOP_PICARD;
  PCK(NC_PROF_MG_SETUP, launch_galerkin_fine<R>(mg.lev[0].g, mg.lev[1].g, pb->ph, mg_state<R>(pb), mg_mat<R>(pb), mg.lev[0].dinv,
                             mg.lev[1].ebe, pb->st, &pb->cnt, gal_picard));
  for (int l = 1; l < L - 1; ++l)
    PCK(NC_PROF_MG_COARSE_SETUP, launch_galerkin_coarse<R>(mg.lev[l].g, mg.lev[l + 1].g, mg.lev[l].ebe, mg.lev[l].dinv, mg.lev[l + 1].ebe,
                                 pb->st, &pb->cnt));
  for (int l = 1; l < L - 1; ++l)
    PCK(NC_PROF_MG_COARSE_SETUP, launch_stencil_build<R>(mg.lev[l].g, mg.lev[l].ebe, mg.lev[l].S, pb->st, &pb->cnt));
  PCK(NC_PROF_MG_COARSE_SETUP, launch_dense_assemble<R>(mg.lev[L - 1].g, mg.lev[L - 1].ebe, mg.Ac, mg.nf, pb->st, &pb->cnt));
  // The FP32 inverse of the coarsest matrix is refreshed at the first set-up of each solve call
  // (every set-up with coarse_refactor = 1, once per problem with 2); later set-ups keep it and the coarse solve's
  // FP64 refinement step against the current matrix corrects for the change.
  const bool factor = pb->par.coarse_refactor == 1 || !mg.factored ||
                      (pb->par.coarse_refactor == 0 && refactor);
  mg.factored = true;
  if (factor)
    PCK(NC_PROF_COARSE_FACTOR, launch_coarse_factor(mg.Ac, mg.W, mg.Ainv32, mg.nf, pb->dflag, pb->st, &pb->cnt));
  for (int l = 0; l < L - 1; ++l) PCK(NC_PROF_MG_COARSE_SETUP, launch_invert_diag<R>(mg.lev[l].g, mg.lev[l].dinv, pb->dflag, pb->st, &pb->cnt));
  for (int l = 1; l < L - 1; ++l)
    if (mg.lev[l].lf)
      PCK(NC_PROF_MG_COARSE_SETUP, launch_line_factor<R>(mg.lev[l].g, mg.lev[l].S, mg.lev[l].lf, pb->dflag, pb->st, &pb->cnt));
  CK(cudaMemcpyAsync(pb->hflag, pb->dflag, sizeof(int), cudaMemcpyDeviceToHost, pb->st));
  CKS(sync(pb, "multigrid set-up"));
  if (*pb->hflag) return fail(pb, NC_ERR_NAN, "singular block in the multigrid set-up");
  return NC_OK;
}

template <typename R>
nc_status level_apply(nc_problem* pb, int l, bool tr, const typename Vec2<R>::type* x, typename Vec2<R>::type* y) {
  MG<R>& mg = mg_of<R>(pb);
  if (l != 0) return fail(pb, NC_ERR_ARG, "level_apply is for the finest level");
  if constexpr (std::is_same<R, float>::value) {
    if (pb->par.mg_op0 == NC_MGOP_PICARD) {
      PCK(NC_PROF_MG_OP0_PICARD, launch_level0_picard(mg.lev[0].g, pb->ph, pb->fz, pb->mat32, x, y, tr, pb->st, &pb->cnt, pb->par.elem_chunk));
      return NC_OK;
    }
  }
  PCK(NC_PROF_MG_OP0, launch_level0_apply<R>(mg.lev[0].g, pb->ph, mg_state<R>(pb), mg_mat<R>(pb), x, y, tr, pb->st, &pb->cnt, pb->par.elem_chunk));
  return NC_OK;
}

// First level of the fused multigrid tail (levels with at most mg_tail_nodes nodes, below the
// finest, with at least one level above the coarsest), or 0 if there is none.
int tail_level(const nc_problem* pb) {
  const int L = (int)pb->lv.g.size();
  if (pb->par.mg_tail_nodes <= 0) return 0;
  for (int l = 1; l < L - 1; ++l)
    if (pb->lv.g[l].nn <= pb->par.mg_tail_nodes) return (L - l <= kTailMaxLevels) ? l : 0;
  return 0;
}

template <typename R>
nc_status vcycle(nc_problem* pb, int l, bool tr);

// Whether level l takes its first pre-smoothing sweep (block Jacobi from zero) from the restriction
// that produces its right-hand side: levels between the finest and the coarsest, smoothed by block
// Jacobi, above the fused tail.
template <typename R>
bool first_sweep_in_restrict(nc_problem* pb, int l) {
  const MG<R>& mg = mg_of<R>(pb);
  const int tl = tail_level(pb);
  return l > 0 && l < (int)mg.lev.size() - 1 && !mg.lev[l].lf && (tl == 0 || l < tl);
}

// Post-smoothing sweeps on level l >= 1: mg_nu_coarse from level mg_nu_coarse_level on, else nu_post.
int coarse_post_sweeps(const nc_problem* pb, int l) {
  const int from = std::max(1, pb->par.mg_nu_coarse_level);
  return (pb->par.mg_nu_coarse > 0 && l >= from) ? pb->par.mg_nu_coarse : std::max(0, pb->par.nu_post);
}

// Kernel classes launched by the V-cycle below the finest level.
const int kCoarseCycleClasses = (1 << NC_PROF_SMOOTH) | (1 << NC_PROF_MG_STENCIL) | (1 << NC_PROF_MG_STENCIL_L1) |
                                (1 << NC_PROF_COARSE_SOLVE) | (1 << NC_PROF_MG_TAIL);

void drop_graphs(nc_problem* pb) {
  for (int t = 0; t < 2; ++t) {
    if (pb->mg32.graph[t]) cudaGraphExecDestroy(pb->mg32.graph[t]);
    if (pb->mg64.graph[t]) cudaGraphExecDestroy(pb->mg64.graph[t]);
    pb->mg32.graph[t] = pb->mg64.graph[t] = nullptr;
  }
}

// The V-cycle on levels 1 .. L-1 (called from the finest level). Its launch sequence and arguments
// are the same at every call once the hierarchy exists (set-ups change values, not buffers), and its
// dozens of small launches are latency bound, so it is captured once per direction as a CUDA graph
// and replayed. Replaying is equivalent when the x / xn exchanges of a cycle leave every level's
// pointers as they were (an even number of sweeps after the first); it is skipped while one of its
// kernel classes is being timed (nc_set_profiling), since timing events cannot be replayed.
template <typename R>
nc_status coarse_cycle(nc_problem* pb, bool tr) {
  MG<R>& mg = mg_of<R>(pb);
  bool odd = false;
  for (int l = 1; l < (int)mg.lev.size() - 1; ++l)   // the z-line smoother updates x in place
    if (!mg.lev[l].lf) odd |= ((std::max(1, pb->par.nu_pre) - 1 + coarse_post_sweeps(pb, l)) & 1) != 0;
  if (odd || (pb->prof_mask & kCoarseCycleClasses)) return vcycle<R>(pb, 1, tr);
  const int t = tr ? 1 : 0;
  if (!mg.graph[t]) {
    const Counters before = pb->cnt;
    CK(cudaStreamBeginCapture(pb->st, cudaStreamCaptureModeThreadLocal));
    const nc_status s = vcycle<R>(pb, 1, tr);
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(pb->st, &gr);
    if (s != NC_OK) { if (gr) cudaGraphDestroy(gr); return s; }
    if (e != cudaSuccess) return cuda_fail(pb, e, "capture of the coarse V-cycle");
    const cudaError_t ei = cudaGraphInstantiate(&mg.graph[t], gr, 0);
    cudaGraphDestroy(gr);
    if (ei != cudaSuccess) { mg.graph[t] = nullptr; return cuda_fail(pb, ei, "graph instantiation"); }
    mg.graph_cnt[t].launches = pb->cnt.launches - before.launches;
    mg.graph_cnt[t].bytes = pb->cnt.bytes - before.bytes;
    mg.graph_cnt[t].flops = pb->cnt.flops - before.flops;
  } else {
    pb->cnt.launches += mg.graph_cnt[t].launches;
    pb->cnt.bytes += mg.graph_cnt[t].bytes;
    pb->cnt.flops += mg.graph_cnt[t].flops;
  }
  CK(cudaGraphLaunch(mg.graph[t], pb->st));
  return NC_OK;
}

// V-cycle on level l: solves approximately A_l x_l = b_l; the result is left in lev[l].x.
// Level 0 applies the matrix-free Jacobian and updates separately; coarser levels fuse the
// stencil product with the Jacobi update or the residual.
template <typename R>
nc_status vcycle(nc_problem* pb, int l, bool tr) {
  MG<R>& mg = mg_of<R>(pb);
  MGLevelDev<R>& d = mg.lev[l];
  const int L = (int)mg.lev.size();
  if (l == L - 1) {
    PCK(NC_PROF_COARSE_SOLVE, launch_coarse_solve<R>(mg.Ac, mg.Ainv32, mg.cw, mg.nf, d.b, d.x, d.g.nn, tr, pb->st, &pb->cnt));
    return NC_OK;
  }
  const R om = (R)pb->par.omega;
  const int nu1 = std::max(1, pb->par.nu_pre), nu2 = l > 0 ? coarse_post_sweeps(pb, l) : std::max(0, pb->par.nu_post);
  if (l > 0 && l == tail_level(pb)) {
    // levels l .. L-1 in one cluster kernel; the host pointers follow its x / xn swaps
    TailArgs<R> a;
    for (int q = l; q < L; ++q) {
      TailLevel<R>& tl = a.lev[q - l];
      const MGLevelDev<R>& dq = mg.lev[q];
      tl.g = dq.g; tl.S = dq.S; tl.dinv = dq.dinv; tl.x = dq.x; tl.xn = dq.xn; tl.b = dq.b;
    }
    a.nlev = L - l; a.Ac = mg.Ac; a.Ainv32 = mg.Ainv32; a.cw = mg.cw; a.nf = mg.nf;
    a.omega = om; a.nu1 = nu1; a.nu2 = nu2; a.ctas = pb->par.mg_tail_ctas;
    PCK(NC_PROF_MG_TAIL, launch_mg_tail<R>(a, tr, pb->st, &pb->cnt));
    for (int q = l; q < L - 1; ++q)
      for (int sw = 0; sw < (nu1 - 1) + nu2; ++sw) std::swap(mg.lev[q].x, mg.lev[q].xn);
    return NC_OK;
  }
  auto sweep = [&](bool last) -> nc_status {
    if (d.lf) {
      // z-line smoother: residual into xn, then x += omega T^-1 r in place (no exchange of x and xn)
      PCK(l == 1 ? NC_PROF_MG_STENCIL_L1 : NC_PROF_MG_STENCIL,
          launch_stencil_apply<R>(d.g, d.S, d.x, d.b, d.dinv, om, d.xn, tr, 1, pb->st, &pb->cnt));
      PCK(NC_PROF_SMOOTH, launch_line_smooth<R>(d.g, d.lf, d.xn, d.x, om, tr, false, pb->st, &pb->cnt));
      return NC_OK;
    }
    if (l == 0) {
      CKS(level_apply<R>(pb, l, tr, d.x, d.y));
      if (last && mg.out64)
        PCK(NC_PROF_SMOOTH, launch_jacobi_io<R>(d.g, d.dinv, d.b, nullptr, d.y, d.x, d.xn, mg.out64, om, tr, false,
                                                pb->st, &pb->cnt));
      else
        PCK(NC_PROF_SMOOTH, launch_jacobi_update<R>(d.g, d.dinv, d.b, d.y, d.x, d.xn, om, tr, false, pb->st, &pb->cnt));
    } else {
      PCK(l == 1 ? NC_PROF_MG_STENCIL_L1 : NC_PROF_MG_STENCIL,
          launch_stencil_apply<R>(d.g, d.S, d.x, d.b, d.dinv, om, d.xn, tr, 2, pb->st, &pb->cnt));
    }
    std::swap(d.x, d.xn);
    return NC_OK;
  };
  if (l == 0 && mg.in64)
    PCK(NC_PROF_SMOOTH, launch_jacobi_io<R>(d.g, d.dinv, d.b, mg.in64, d.y, d.x, d.x, nullptr, om, tr, true, pb->st,
                                            &pb->cnt));
  else if (d.lf)
    PCK(NC_PROF_SMOOTH, launch_line_smooth<R>(d.g, d.lf, d.b, d.x, om, tr, true, pb->st, &pb->cnt));
  else if (!first_sweep_in_restrict<R>(pb, l))   // otherwise the restriction into b already swept
    PCK(NC_PROF_SMOOTH, launch_jacobi_update<R>(d.g, d.dinv, d.b, d.y, d.x, d.x, om, tr, true, pb->st, &pb->cnt));
  for (int it = 1; it < nu1; ++it) CKS(sweep(false));
  MGLevelDev<R>& c = mg.lev[l + 1];
  // the coarse level's first sweep fused into its restriction where it is block Jacobi
  const bool fuse = first_sweep_in_restrict<R>(pb, l + 1);
  if (l == 0) {
    // residual b - A x restricted directly, without storing it
    CKS(level_apply<R>(pb, l, tr, d.x, d.y));
    PCK(NC_PROF_SMOOTH, launch_restrict_residual<R>(d.g, c.g, d.b, d.y, c.b, pb->st, &pb->cnt, c.dinv,
                                                    fuse ? c.x : nullptr, om, tr));
  } else {
    PCK(l == 1 ? NC_PROF_MG_STENCIL_L1 : NC_PROF_MG_STENCIL,
        launch_stencil_apply<R>(d.g, d.S, d.x, d.b, d.dinv, om, d.xn, tr, 1, pb->st, &pb->cnt));
    PCK(NC_PROF_SMOOTH, launch_restrict<R>(d.g, c.g, d.xn, c.b, pb->st, &pb->cnt, c.dinv, fuse ? c.x : nullptr,
                                           om, tr));
  }
  CKS(l == 0 ? coarse_cycle<R>(pb, tr) : vcycle<R>(pb, l + 1, tr));
  PCK(NC_PROF_SMOOTH, launch_prolong_add<R>(d.g, c.g, c.x, d.x, pb->st, &pb->cnt));
  for (int it = 0; it < nu2; ++it) CKS(sweep(it == nu2 - 1));
  return NC_OK;
}

// z = M^-1 v (one V-cycle), v and z FP64 state vectors.
nc_status precondition(nc_problem* pb, bool tr, const double* v, double* z) {
  // the finest level's first and last updates read v and write z directly (no separate casts);
  // without post-smoothing z is copied out after the cycle
  const bool post = pb->par.nu_post > 0;
  if (pb->par.precision == NC_PREC_FP64) {
    MG<double>& mg = pb->mg64;
    mg.in64 = v;
    mg.out64 = post ? z : nullptr;
    nc_status s = vcycle<double>(pb, 0, tr);
    mg.in64 = nullptr;
    mg.out64 = nullptr;
    CKS(s);
    if (!post) PCK(NC_PROF_OTHER, launch_from_mg<double>(mg.lev[0].x, z, pb->g.nn, pb->st, &pb->cnt));
  } else {
    MG<float>& mg = pb->mg32;
    mg.in64 = v;
    mg.out64 = post ? z : nullptr;
    nc_status s = vcycle<float>(pb, 0, tr);
    mg.in64 = nullptr;
    mg.out64 = nullptr;
    CKS(s);
    if (!post) PCK(NC_PROF_OTHER, launch_from_mg<float>(mg.lev[0].x, z, pb->g.nn, pb->st, &pb->cnt));
  }
  return NC_OK;
}

nc_status mg_setup_any(nc_problem* pb, bool refactor) {
  if (pb->par.precision == NC_PREC_FP64) return mg_setup<double>(pb, refactor);
  return mg_setup<float>(pb, refactor);
}

// ---------------------------------------------------------------- FGMRES ------------
// Krylov vectors are FP64 (FP64 path; mixed path with NC_BASIS_FP64) or FP32 (mixed path with
// NC_BASIS_FP32, where the operator J or J^T on the FP32 state copy and the preconditioner are FP32
// as well). The Hessenberg matrix, the Givens rotations and the update of the FP64 solution are FP64
// in every case.

// z = M^-1 v for FP32 vectors: the V-cycle reads v in place and leaves its result in z.
nc_status kry_precondition(nc_problem* pb, bool tr, const float* v, float* z) {
  MGLevelDev<float>& d = pb->mg32.lev[0];
  float2* const b0 = d.b;
  float2* const x0 = d.x;
  float2* const xn0 = d.xn;
  d.b = (float2*)v;   // level 0 only reads b
  d.x = (float2*)z;
  nc_status s = vcycle<float>(pb, 0, tr);
  if (s == NC_OK && d.x != (float2*)z)
    CK(cudaMemcpyAsync(z, d.x, sizeof(float2) * pb->g.nn, cudaMemcpyDeviceToDevice, pb->st));
  d.b = b0;
  d.x = x0;
  d.xn = xn0;
  return s;
}

nc_status kry_precondition(nc_problem* pb, bool tr, const double* v, double* z) {
  return precondition(pb, tr, v, z);
}

nc_status kry_op(nc_problem* pb, bool tr, bool fp32, const float* z, float* w) {
  (void)fp32;
  PCK(NC_PROF_OUTER_OP32, launch_level0_apply<float>(pb->g, pb->ph, pb->s32, pb->mat32, (const float2*)z, (float2*)w,
                                                     tr, pb->st, &pb->cnt, pb->par.elem_chunk));
  if (pb->g.bc != kBcTop) PCK(NC_PROF_OTHER, launch_zero_dirichlet(pb->g, w, pb->st, &pb->cnt));
  return NC_OK;
}

nc_status kry_op(nc_problem* pb, bool tr, bool fp32, const double* z, double* w) {
  if (fp32) {
    // z was just produced by the FP32 preconditioner: its FP32 copy (z rounded to FP32, exactly the
    // finest level's x) is still in the hierarchy, so the operator reads it without a cast
    const Grid& g = pb->g;
    PCK(NC_PROF_OUTER_OP32, launch_level0_apply<float>(g, pb->ph, pb->s32, pb->mat32, pb->mg32.lev[0].x, pb->y32, tr,
                                                       pb->st, &pb->cnt, pb->par.elem_chunk));
    PCK(NC_PROF_OUTER_OP32, launch_cast_f2d(w, (const float*)pb->y32, 2 * g.nn, pb->st, &pb->cnt));
    if (g.bc != kBcTop) PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, w, pb->st, &pb->cnt));
    return NC_OK;
  }
  return outer_op(pb, tr, false, z, w);
}

// Default re-orthogonalisation threshold of FP64 bases: a second pass only when the first cancelled
// more than 99 % of the norm (two digits of the 16); an FP32 basis uses the DGKS value 1/2.
const double kReorthFP64 = 1e-2;

// Right-preconditioned flexible GMRES(m) with classical Gram-Schmidt applied twice. Solves
// op(x) = b on the free DOFs from x = 0; stops when the (Arnoldi) residual is <= rtol ||b||.
// b is not modified (it may be any FP64 work vector other than x and R_try).
template <typename T>
nc_status fgmres_t(nc_problem* pb, bool tr, bool fp32, T* V, T* Z, const double* b, double* x, double rtol,
                   int maxit, int* its_out, double* relres_out) {
  const long long n = 2 * pb->g.nn;
  const int m = pb->m;
  // second Gram-Schmidt pass when the first kept less than this fraction of ||w||^2
  const double thr = pb->par.krylov_reorth > 0 ? pb->par.krylov_reorth : (sizeof(T) == 4 ? 0.5 : kReorthFP64);
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, pb->st));
  double bb;
  CKS(norm2_free(pb, b, &bb));
  const double bnorm = std::sqrt(bb);
  *its_out = 0;
  *relres_out = 0.0;
  if (bnorm == 0.0) return NC_OK;
  // r = b
  double beta = bnorm;
  PCK(NC_PROF_KRYLOV_VEC, launch_scale_copy(V, b, 1.0 / beta, n, pb->st, &pb->cnt));
  PCK(NC_PROF_KRYLOV_VEC, launch_zero_dirichlet(pb->g, V, pb->st, &pb->cnt));
  int total = 0;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m), h(m + 2), h2(m + 2), resh(m);
  while (true) {
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m && total < maxit; ++j, ++total) {
      CKS(check_timeout(pb));
      T* vj = V + (long long)j * n;
      T* zj = Z + (long long)j * n;
      T* wv = V + (long long)(j + 1) * n;
      CKS(kry_precondition(pb, tr, vj, zj));
      CKS(kry_op(pb, tr, fp32, zj, wv));
      double hn;
      if (j + 1 <= 32) {
        // CGS2 with coefficients kept on the device; one host synchronisation per iteration
        double* d1 = pb->dres;
        double* d2 = pb->dres + 66;
        // d1: V_i . w (i <= j) and w . w (w is V_{j+1}); d2: second-pass dots when re-orthogonalising
        PCK(NC_PROF_KRYLOV_VEC, launch_multidot(V, n, j + 2, wv, n, pb->part, d1, pb->st, &pb->cnt));
        PCK(NC_PROF_KRYLOV_VEC, launch_cgs(wv, V, n, j + 1, d1, d2, n, thr, pb->part, pb->st, &pb->cnt));
        CK(cudaMemcpyAsync(pb->hres, pb->dres, sizeof(double) * 132, cudaMemcpyDeviceToHost, pb->st));
        CKS(sync(pb, "Gram-Schmidt"));
        // the device's test (DGKS on the Pythagorean norm) repeated on the same values
        double s1 = 0.0;
        for (int i = 0; i <= j; ++i) s1 += pb->hres[i] * pb->hres[i];
        const double ww = pb->hres[j + 1];
        const bool fast = ww - s1 >= thr * ww;
        double hn2;
        if (fast) {
          for (int i = 0; i <= j; ++i) h[i] = pb->hres[i];
          hn2 = ww - s1;
        } else {
          double corr = 0.0;
          for (int i = 0; i <= j; ++i) {
            const double c2 = pb->hres[66 + i];
            h[i] = pb->hres[i] + c2;
            corr += c2 * c2;
          }
          hn2 = pb->hres[66 + j + 1] - corr;
        }
        if (!std::isfinite(hn2)) return fail(pb, NC_ERR_NAN, "non-finite Krylov vector");
        hn = hn2 > 0.0 ? std::sqrt(hn2) : 0.0;
      } else {
        CKS(dots(pb, V, n, j + 1, wv, n, h.data()));
        for (int i = 0; i <= j; ++i) h2[i] = -h[i];
        PCK(NC_PROF_KRYLOV_VEC, launch_axpy_multi(wv, V, n, j + 1, h2.data(), n, pb->st, &pb->cnt));
        CKS(dots(pb, V, n, j + 2, wv, n, h2.data()));   // second pass dots and ||w||^2
        double ww = h2[j + 1];
        double corr = 0.0;
        for (int i = 0; i <= j; ++i) { h[i] += h2[i]; corr += h2[i] * h2[i]; h2[i] = -h2[i]; }
        PCK(NC_PROF_KRYLOV_VEC, launch_axpy_multi(wv, V, n, j + 1, h2.data(), n, pb->st, &pb->cnt));
        double hn2 = ww - corr;
        if (!std::isfinite(hn2)) return fail(pb, NC_ERR_NAN, "non-finite Krylov vector");
        hn = hn2 > 0.0 ? std::sqrt(hn2) : 0.0;
        if (hn > 0.0) PCK(NC_PROF_KRYLOV_VEC, launch_scale(wv, 1.0 / hn, n, pb->st, &pb->cnt));
      }
      for (int i = 0; i <= j; ++i) H[i * m + j] = h[i];
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], b2 = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * b2;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b2;
      }
      const double a = H[j * m + j], b2 = H[(j + 1) * m + j];
      const double r = std::hypot(a, b2);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? b2 / r : 0.0;
      H[j * m + j] = r;
      H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      const double res = std::fabs(gv[j + 1]);
      *relres_out = res / bnorm;
      if (res <= rtol * bnorm || hn == 0.0) { ++j; ++total; done = true; break; }
      // FP64 operator: an Arnoldi estimate within a factor 100 of the tolerance that has not halved
      // over three iterations is checked against the true residual by restarting early (near a
      // tight tolerance the estimate can stall while the true residual keeps falling)
      resh[j] = res;
      if (!fp32 && j >= 3 && res < 1e2 * rtol * bnorm && res > 0.5 * resh[j - 3]) { ++j; ++total; break; }
    }
    // x += Z y, y = H^-1 g (upper triangular j x j)
    for (int i = j - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int k = i + 1; k < j; ++k) acc -= H[i * m + k] * y[k];
      y[i] = acc / H[i * m + i];
    }
    if (j > 0) PCK(NC_PROF_KRYLOV_VEC, launch_axpy_multi(x, Z, n, j, y.data(), n, pb->st, &pb->cnt));
    *its_out = total;
    if (done) return NC_OK;
    if (total >= maxit) return NC_OK;   // caller judges the reached residual
    // restart with the residual r = b - op(x) (op in the path's Krylov precision), in R_try
    double* r = pb->R_try;
    CKS(outer_op(pb, tr, fp32, x, r));
    PCK(NC_PROF_KRYLOV_VEC, launch_axpby(r, b, 1.0, -1.0, n, pb->st, &pb->cnt));
    PCK(NC_PROF_KRYLOV_VEC, launch_zero_dirichlet(pb->g, r, pb->st, &pb->cnt));
    double rr;
    CKS(norm2_free(pb, r, &rr));
    beta = std::sqrt(rr);
    *relres_out = beta / bnorm;
    if (beta <= rtol * bnorm) return NC_OK;
    PCK(NC_PROF_KRYLOV_VEC, launch_scale_copy(V, r, 1.0 / beta, n, pb->st, &pb->cnt));
  }
}

// FGMRES on the FP64 path (fp32 false) or the mixed-precision path (fp32 true: FP32 operator and
// preconditioner; basis as nc_params.krylov_basis).
nc_status fgmres(nc_problem* pb, bool tr, bool fp32, const double* b, double* x, double rtol, int maxit,
                 int* its_out, double* relres_out) {
  if (fp32 != (pb->par.precision != NC_PREC_FP64)) return fail(pb, NC_ERR_ARG, "Krylov precision mismatch");
  if (pb->V32) return fgmres_t<float>(pb, tr, fp32, pb->V32, pb->Z32, b, x, rtol, maxit, its_out, relres_out);
  return fgmres_t<double>(pb, tr, fp32, pb->V, pb->Z, b, x, rtol, maxit, its_out, relres_out);
}

// ---------------------------------------------------------------- Newton ------------
struct NewtonResult {
  bool converged = false;
  bool failed = false;   // no damping factor decreased the residual
};

// phi(lam) = ||R_free(s + lam dx)||^2 into R_try / s_try.
nc_status trial(nc_problem* pb, double lam, double* phi, nc_stats* stats) {
  const long long n = 2 * pb->g.nn;
  CK(cudaMemcpyAsync(pb->s_try, pb->s, sizeof(double) * n, cudaMemcpyDeviceToDevice, pb->st));
  PCK(NC_PROF_OTHER, launch_axpby((double*)pb->s_try, pb->dx, lam, 1.0, n, pb->st, &pb->cnt));
  CKS(residual(pb, pb->s_try, pb->R_try, phi));
  if (stats) stats->residual_evals++;
  return NC_OK;
}

nc_status accept_trial(nc_problem* pb) {
  std::swap(pb->s, pb->s_try);
  std::swap(pb->R, pb->R_try);
  return NC_OK;
}

// Damping factor (Sec. 5.4: the minimiser of ||R(s + lam dx)||): full step if it reduces
// phi = ||R||^2 by the fraction 1e-4, else the best of phi(1), phi(1/2) and the minimiser of the
// parabola through phi(0), phi(1/2), phi(1) clamped to [0.05, 1], else halving from 1/4.
nc_status damping(nc_problem* pb, double phi0, double* lam_out, double* phi_out, bool* ok, nc_stats* stats) {
  *ok = false;
  double phi1;
  CKS(trial(pb, 1.0, &phi1, stats));
  if (phi1 <= (1.0 - 1e-4) * phi0) { *lam_out = 1.0; *phi_out = phi1; *ok = true; return accept_trial(pb); }
  double phih;
  CKS(trial(pb, 0.5, &phih, stats));
  double best_lam = 0.5, best_phi = phih;
  if (phi1 < best_phi) { best_lam = 1.0; best_phi = phi1; }
  const double c1 = 4.0 * phih - 3.0 * phi0 - phi1;
  const double c2 = 2.0 * phi1 + 2.0 * phi0 - 4.0 * phih;
  if (c2 > 0.0) {
    const double lam = std::min(1.0, std::max(0.05, -c1 / (2.0 * c2)));
    if (lam != 0.5 && lam != 1.0) {
      double p;
      CKS(trial(pb, lam, &p, stats));
      if (p < best_phi || (p == best_phi && lam > best_lam)) { best_lam = lam; best_phi = p; }
    }
  }
  if (best_phi < phi0) {
    double p;
    CKS(trial(pb, best_lam, &p, stats));
    *lam_out = best_lam; *phi_out = p; *ok = true;
    return accept_trial(pb);
  }
  double lam = 0.25;
  for (int i = 0; i < 8; ++i) {
    double p;
    CKS(trial(pb, lam, &p, stats));
    if (p < phi0) { *lam_out = lam; *phi_out = p; *ok = true; return accept_trial(pb); }
    lam *= 0.5;
  }
  return NC_OK;
}

nc_status newton(nc_problem* pb, double rtol, double ref, nc_stats* stats, bool* failed, bool from_zero) {
  *failed = false;
  double phi;
  if (from_zero && pb->ph.Q == pb->Q_full) {
    CK(cudaMemcpyAsync(pb->R, pb->R0, sizeof(double) * 2 * pb->g.nn, cudaMemcpyDeviceToDevice, pb->st));
    phi = pb->ref_norm * pb->ref_norm;
  } else {
    CKS(residual(pb, pb->s, pb->R, &phi));
    if (stats) stats->residual_evals++;
  }
  const long long n = 2 * pb->g.nn;
  const bool fp32 = pb->par.precision != NC_PREC_FP64;
  double rel_prev = -1.0, eta_prev = pb->par.krylov_rtol;
  for (int it = 0;; ++it) {
    const double rel = ref > 0 ? std::sqrt(phi) / ref : 0.0;
    if (stats) stats->rel_residual = rel;
    if (rel <= rtol) return NC_OK;
    if (it >= pb->par.newton_maxit) return fail(pb, NC_ERR_MAXIT, "Newton iteration limit reached");
    CKS(check_timeout(pb));
    // forcing term: Eisenstat-Walker (choice 2, gamma 0.9) safeguarded, and no tighter than
    // needed to reach rtol in this step
    double eta = pb->par.krylov_rtol;
    if (rel_prev > 0.0) {
      const double r = rel / rel_prev;
      eta = 0.9 * r * r;
      if (0.9 * eta_prev * eta_prev > 0.1) eta = std::max(eta, 0.9 * eta_prev * eta_prev);
      eta = std::min(eta, pb->par.krylov_rtol);
    }
    eta = std::max(eta, 0.5 * rtol / rel);
    const double eta_min = pb->par.krylov_eta_min > 0 ? pb->par.krylov_eta_min : 1e-12;
    eta = std::max(std::min(eta, pb->par.krylov_rtol), eta_min);
    double t0 = now_s();
    // lagged preconditioner: once the residual is below mg_reuse_below, the hierarchy of the previous
    // Newton step is kept (the state changes little; FGMRES absorbs the difference)
    if (!pb->mg_ready || rel > pb->par.mg_reuse_below) {
      CKS(mg_setup_any(pb, pb->first_setup));
      pb->first_setup = false;
      pb->mg_ready = true;
      if (stats) stats->mg_setups++;
    } else if (pb->par.precision != NC_PREC_FP64) {
      // the Krylov operator and the finest multigrid level use the current state
      CKS(refresh_state32(pb, pb->s, NC_PROF_MG_COARSE_SETUP));
    }
    double t1 = now_s();
    PCK(NC_PROF_OTHER, launch_scale_copy(pb->rhs, pb->R, -1.0, n, pb->st, &pb->cnt));
    PCK(NC_PROF_OTHER, launch_zero_dirichlet(pb->g, pb->rhs, pb->st, &pb->cnt));
    int its = 0;
    double lres = 0.0;
    CKS(fgmres(pb, false, fp32, pb->rhs, pb->dx, eta, pb->par.krylov_maxit, &its, &lres));
    double t2 = now_s();
    if (stats) {
      stats->t_setup_ms += 1e3 * (t1 - t0);
      stats->t_krylov_ms += 1e3 * (t2 - t1);
      stats->krylov_its += its;
      if (stats->newton_its < 64) stats->krylov_hist[stats->newton_its] = its;
    }
    double lam, phi_new;
    bool ok;
    CKS(damping(pb, phi, &lam, &phi_new, &ok, stats));
    if (!ok) { *failed = true; return NC_OK; }
    phi = phi_new;
    rel_prev = rel;
    eta_prev = eta;
    if (stats) {
      const double rn = ref > 0 ? std::sqrt(phi) / ref : 0.0;
      if (stats->newton_its < 64) stats->res_hist[stats->newton_its] = rn;
      stats->newton_its++;
    }
  }
}

void set_q_scale(nc_problem* pb, double scale) { pb->ph.Q = pb->Q_full * scale; }

nc_status reference_norm(nc_problem* pb) {
  // ||R_free(0)|| with the full source: R(0) is minus the SUPG-weighted source load, which does
  // not depend on the design, so it is evaluated once per problem and kept in R0.
  if (pb->have_R0) return NC_OK;
  CK(cudaMemsetAsync(pb->s_try, 0, sizeof(double) * 2 * pb->g.nn, pb->st));
  set_q_scale(pb, 1.0);
  double phi;
  CKS(residual(pb, pb->s_try, pb->R0, &phi));
  pb->ref_norm = std::sqrt(phi);
  pb->have_R0 = true;
  return NC_OK;
}

nc_status copy_in(nc_problem* pb, void* dst, const void* src, size_t bytes) {
  if (!src) return fail(pb, NC_ERR_ARG, "NULL input pointer");
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, pb->st));
  return NC_OK;
}

nc_status copy_out(nc_problem* pb, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, pb->st));
  return NC_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

nc_status validate(const nc_grid* g, const nc_params* p, std::string* why) {
  if (!g || !p) { *why = "NULL grid or params"; return NC_ERR_ARG; }
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->h > 0.0) || !std::isfinite(g->h)) {
    *why = "grid needs nx, ny, nz >= 1 and h > 0"; return NC_ERR_ARG;
  }
  if ((long long)g->nx * g->ny * g->nz > (1LL << 31)) { *why = "grid too large"; return NC_ERR_ARG; }
  if (p->heated_layers < 0 || p->heated_layers >= g->nz) { *why = "heated_layers must be in [0, nz)"; return NC_ERR_ARG; }
  if (!(p->mu > 0) || !(p->rho0 > 0) || !(p->cp > 0) || !(p->k_f > 0) || !(p->k_s > 0) || !(p->kappa_ratio > 0)) {
    *why = "material parameters must be positive"; return NC_ERR_ARG;
  }
  if (p->alpha < 0 || p->g < 0 || p->q_c < 0 || p->q_p < 0) { *why = "alpha, g, q_c, q_p must be >= 0"; return NC_ERR_ARG; }
  if (p->restart < 1 || p->restart > kMaxRestart) { *why = "restart must be in [1, 64]"; return NC_ERR_ARG; }
  if (p->precision != NC_PREC_MIXED && p->precision != NC_PREC_FP64) { *why = "unknown precision"; return NC_ERR_ARG; }
  if (p->outer_arith != NC_ARITH_DF64 && p->outer_arith != NC_ARITH_FP64) { *why = "unknown outer_arith"; return NC_ERR_ARG; }
  if (p->krylov_basis != NC_BASIS_FP32 && p->krylov_basis != NC_BASIS_FP64) { *why = "unknown krylov_basis"; return NC_ERR_ARG; }
  if (!(p->krylov_reorth <= 1.0)) { *why = "krylov_reorth must be <= 1"; return NC_ERR_ARG; }
  if (p->mg_tail_nodes < 0) { *why = "mg_tail_nodes must be >= 0"; return NC_ERR_ARG; }
  if (!(p->mg_reuse_below >= 0.0)) { *why = "mg_reuse_below must be >= 0"; return NC_ERR_ARG; }
  if (p->adjoint_df64_steps != 0 && p->adjoint_df64_steps != 1) { *why = "adjoint_df64_steps must be 0 or 1"; return NC_ERR_ARG; }
  if (p->mg_op0 != NC_MGOP_EXACT && p->mg_op0 != NC_MGOP_PICARD) { *why = "unknown mg_op0"; return NC_ERR_ARG; }
  if (p->mg_tail_ctas < 0 || p->mg_tail_ctas > 16) { *why = "mg_tail_ctas must be in [0, 16]"; return NC_ERR_ARG; }
  if (p->mg_nu_coarse < 0 || p->mg_nu_coarse > 16) { *why = "mg_nu_coarse must be in [0, 16]"; return NC_ERR_ARG; }
  if (p->mg_nu_coarse_level < 0) { *why = "mg_nu_coarse_level must be >= 0"; return NC_ERR_ARG; }
  if (p->mg_smoother != NC_SMOOTH_BLOCK_JACOBI && p->mg_smoother != NC_SMOOTH_ZLINE) { *why = "unknown mg_smoother"; return NC_ERR_ARG; }
  if (p->filter_method != NC_FILTER_SPECTRAL && p->filter_method != NC_FILTER_CHEBYSHEV) { *why = "unknown filter_method"; return NC_ERR_ARG; }
  if (p->mg_galerkin != NC_MGOP_EXACT && p->mg_galerkin != NC_MGOP_PICARD) { *why = "unknown mg_galerkin"; return NC_ERR_ARG; }
  if (p->mg_smoother == NC_SMOOTH_ZLINE && p->mg_tail_nodes > 0) {
    *why = "the fused multigrid tail smooths with block Jacobi (NC_SMOOTH_ZLINE needs mg_tail_nodes = 0)"; return NC_ERR_ARG;
  }
  if (p->elem_chunk != -1 && p->elem_chunk != 0 && p->elem_chunk != 1 && p->elem_chunk != 2 && p->elem_chunk != 4 &&
      p->elem_chunk != 8 && p->elem_chunk != 16) { *why = "elem_chunk must be -1, 0, 1, 2, 4, 8 or 16"; return NC_ERR_ARG; }
  if (p->coarse_refactor < 0 || p->coarse_refactor > 2) { *why = "coarse_refactor must be 0, 1 or 2"; return NC_ERR_ARG; }
  if (!(p->newton_rtol > 0) || p->newton_maxit < 0 || p->krylov_maxit < 1) { *why = "bad tolerances"; return NC_ERR_ARG; }
  if (!(p->filter_radius >= 0) || !(p->filter_rtol > 0)) { *why = "bad filter parameters"; return NC_ERR_ARG; }
  if (p->bc != NC_BC_TOP && p->bc != NC_BC_CAVITY) { *why = "unknown bc"; return NC_ERR_ARG; }
  if (p->region_shape != NC_REGION_BOX && p->region_shape != NC_REGION_CYLINDER) {
    *why = "unknown region_shape"; return NC_ERR_ARG;
  }
  if (p->region_shape == NC_REGION_CYLINDER &&
      (!(p->heat_radius > 0) || !(p->design_radius >= p->heat_radius) || p->heat_z0 < 0 ||
       p->heat_z0 + p->heated_layers > g->nz || p->heated_layers < 1 ||
       4.0 * p->design_radius * p->design_radius > 2e9)) {
    *why = "cylinder regions need 0 < heat_radius <= design_radius and layers inside the grid"; return NC_ERR_ARG;
  }
  if (p->heat_nx < 0 || p->heat_nx > g->nx || p->heat_ny < 0 || p->heat_ny > g->ny || p->design_nx < 0 ||
      p->design_nx > g->nx || p->design_ny < 0 || p->design_ny > g->ny || p->design_nz < 0 ||
      p->heated_layers + p->design_nz > g->nz) {
    *why = "heated and design boxes must lie inside the grid"; return NC_ERR_ARG;
  }
  Grid g0 = make_grid(g->nx, g->ny, g->nz, g->h);
  g0.bc = p->bc;
  Levels lv = plan_levels(g0, p->mg_levels);
  if (lv.g.size() < 2) { *why = "the multigrid hierarchy needs even grid dimensions"; return NC_ERR_ARG; }
  if (lv.nf > kMaxCoarseDofs) { *why = "coarsest multigrid level too large (use more levels)"; return NC_ERR_ARG; }
  return NC_OK;
}

size_t footprint(const nc_grid* gr, const nc_params* p) {
  Grid g = make_grid(gr->nx, gr->ny, gr->nz, gr->h);
  g.bc = p->bc;
  Levels lv = plan_levels(g, p->mg_levels);
  auto al = [](size_t b) { return (std::max<size_t>(b, 1) + 255) & ~size_t(255); };
  size_t b = 0;
  const size_t nn = g.nn, ne = g.ne, m = p->restart;
  b += 4 * al(16 * nn);                 // s, s_try, lam, s_start
  b += 6 * al(16 * nn);                 // R, R_try, dx, w, rhs, R0
  b += 3 * al(8 * ne) + al(24 * ne);    // rho, gamma_t, gsens, u
  b += 3 * al(16 * ne) + al(8 * ne) + 3 * al(8 * nn);   // mat, dmat, dl, mat32, s32, v32, y32
  b += al(16 * ne);                                      // fz
  const size_t ks = (p->precision == NC_PREC_FP64 || p->krylov_basis == NC_BASIS_FP64) ? 8 : 4;   // basis entry
  b += al(2 * ks * nn * (m + 1)) + al(2 * ks * nn * m);     // V, Z
  if (p->precision != NC_PREC_FP64) b += al(16 * ne) + 2 * al(16 * nn);   // mat_df, s_df, w_df
  b += al(8 * 66 * kReduceBlocksMax) + al(8 * 132);
  b += 5 * al(8 * nn) + 5 * al(4 * nn) + 2 * al(8 * nn); // filter vectors (+ double-float solution, rhs)
  for (const int n1 : {gr->nx, gr->ny, gr->nz})   // spectral filter: cosine matrix and 1D eigenvalues per axis
    b += al(4 * (size_t)(n1 + 1) * (n1 + 1)) + 2 * al(4 * (size_t)(n1 + 1));
  b += al(kBlasWorkspace);
  b += size_t(64) << 20;   // the cuBLAS handle's own device allocations (measured: about 64 MiB)
  const size_t rs = p->precision == NC_PREC_FP64 ? 8 : 4;
  for (size_t l = 0; l < lv.g.size(); ++l) {
    b += 4 * al(2 * rs * lv.g[l].nn);
    if (l + 1 < lv.g.size()) b += al(4 * rs * lv.g[l].nn);
    if (l > 0) b += al(256 * rs * lv.g[l].ne);
    if (l > 0 && l + 1 < lv.g.size()) b += al(108 * rs * lv.g[l].nn);
    if (p->mg_smoother == NC_SMOOTH_ZLINE && l > 0 && l + 1 < lv.g.size()) b += al(24 * rs * lv.g[l].nn);
  }
  // coarsest level: Ac (FP64), Ainv32, the Gauss-Jordan work array W and the coarse-solve scratch cw (3 nf FP64)
  b += al(8 * (size_t)lv.nf * lv.nf) + al(4 * (size_t)lv.nf * lv.nf) + al(8 * (size_t)lv.nf * lv.nf + 12 * (size_t)lv.nf);
  b += al(24 * (size_t)lv.nf);
  b += al(4);
  return b;
}

// Derived constants of a problem from its parameters (physics, filter, Chebyshev bounds).
void apply_params(nc_problem* pb, const nc_params* p) {
  pb->par = *p;
  const Grid& g = pb->g;
  pb->kappa_f = p->kappa_f > 0 ? p->kappa_f : kappa_f_tuned(p->alpha, p->tune_dT);
  pb->kappa_s = p->kappa_ratio * pb->kappa_f;
  pb->ph.heat_nx = p->heat_nx > 0 ? p->heat_nx : g.nx;
  pb->ph.heat_ny = p->heat_ny > 0 ? p->heat_ny : g.ny;
  pb->ph.design_nx = p->design_nx > 0 ? p->design_nx : g.nx;
  pb->ph.design_ny = p->design_ny > 0 ? p->design_ny : g.ny;
  pb->ph.design_z1 = p->design_nz > 0 ? p->heated_layers + p->design_nz : g.nz;
  pb->ph.shape = p->region_shape;
  pb->ph.z0 = p->heat_z0;
  pb->ph.q_heat = (int)std::ceil(4.0 * p->heat_radius * p->heat_radius);
  pb->ph.q_design = (int)std::ceil(4.0 * p->design_radius * p->design_radius);
  pb->ph.heated_layers = p->heated_layers;
  if (p->region_shape == NC_REGION_CYLINDER) {
    long long cross = 0;   // heated elements of one layer
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) cross += elem_heated(pb->ph, i, j, p->heat_z0) ? 1 : 0;
    pb->vol_h = (double)cross * p->heated_layers * g.h * g.h * g.h;
  } else {
    pb->vol_h = (double)pb->ph.heat_nx * pb->ph.heat_ny * p->heated_layers * g.h * g.h * g.h;
  }
  pb->Q_full = p->Q > 0 ? p->Q : (pb->vol_h > 0 ? 1.0 / pb->vol_h : 0.0);
  pb->ph.h = g.h;
  pb->ph.beta = p->rho0 * p->alpha * p->g;
  pb->ph.rc = p->rho0 * p->cp;
  pb->ph.mu = p->mu;
  pb->ph.he = std::sqrt(3.0) * g.h;
  pb->ph.tau3 = p->rho0 * p->cp * pb->ph.he * pb->ph.he / (4.0 * p->k_f);
  pb->ph.Q = pb->Q_full;
  // filter element matrix r^2 K0 + M0 (Q1 cube: K0 = h/12 [4,0,-1,-1], M0 = h^3/216 [8,4,2,1] by
  // the number of differing reference coordinates), r = R / (2 sqrt 3)
  {
    const double r = p->filter_radius * g.h / (2.0 * std::sqrt(3.0));
    const double kc[4] = {4.0, 0.0, -1.0, -1.0}, mc[4] = {8.0, 4.0, 2.0, 1.0};
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) {
        const int d = __builtin_popcount(a ^ b);
        pb->F.A[a * 8 + b] = r * r * g.h / 12.0 * kc[d] + g.h * g.h * g.h / 216.0 * mc[d];
      }
    // interior 27-point stencil: offset o couples node n to n + o through the elements holding both
    for (int o = 0; o < 27; ++o) {
      const int od[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      double c = 0.0;
      for (int e = 0; e < 8; ++e) {            // element at offset -(e bits) from the node
        int a = 0, b = 0;
        bool in = true;
        for (int d = 0; d < 3; ++d) {
          const int ad = (e >> d) & 1;         // node's local coordinate in this element
          const int bd = ad + od[d];           // neighbour's local coordinate
          if (bd < 0 || bd > 1) in = false;
          a |= ad << d;
          b |= (bd & 1) << d;
        }
        if (in) c += pb->F.A[a * 8 + b];
      }
      pb->F.C27[o] = c;
    }
    pb->F.t0 = g.h * g.h * g.h / 8.0;
    for (int q = 0; q < 64; ++q) pb->Ff.A[q] = (float)pb->F.A[q];
    for (int q = 0; q < 27; ++q) pb->Ff.C27[q] = (float)pb->F.C27[q];
    for (int q = 0; q < 64; ++q) pb->Fd.A[q] = df64(pb->F.A[q]);
    for (int q = 0; q < 27; ++q) pb->Fd.C27[q] = df64(pb->F.C27[q]);
    // spectrum of D^-1 A from the interior symbol sum_o C27[o] cos(theta . o) / C27[centre]
    // (Neumann boundaries do not widen it), widened by 5 % on each side
    double lmin = 1e300, lmax = -1e300;
    const int T = 32;
    for (int tz = 0; tz <= T; ++tz)
      for (int ty = 0; ty <= T; ++ty)
        for (int tx = 0; tx <= T; ++tx) {
          const double th[3] = {M_PI * tx / T, M_PI * ty / T, M_PI * tz / T};
          double sym = 0.0;
          for (int o = 0; o < 27; ++o)
            sym += pb->F.C27[o] * std::cos(th[0] * (o % 3 - 1) + th[1] * ((o / 3) % 3 - 1) + th[2] * (o / 9 - 1));
          sym /= pb->F.C27[13];
          lmin = std::min(lmin, sym);
          lmax = std::max(lmax, sym);
        }
    pb->cheb_a = 0.95 * lmin;
    pb->cheb_b = 1.05 * lmax;
    const double kap = pb->cheb_b / pb->cheb_a;
    const double rq = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    pb->cheb_iters = std::max(4, (int)std::ceil(std::log(5e-7) / std::log(rq)));
    pb->F.diag = pb->F.A[0];
  }
}

}  // namespace

// ====================================================================================
extern "C" {

nc_status nc_default_params(nc_params* p) {
  if (!p) return NC_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->alpha = 1e3;
  p->kappa_f = 0.0;
  p->tune_dT = 1.0;
  p->kappa_ratio = 1e-6;
  p->k_f = 1.0;
  p->k_s = 100.0;
  p->q_c = 8.81;
  p->q_p = 8.0;
  p->Q = 0.0;
  p->heated_layers = 2;
  p->rho0 = p->mu = p->cp = p->g = 1.0;
  p->filter_radius = 2.5;
  p->newton_rtol = 1e-8;
  p->newton_maxit = 50;
  p->krylov_rtol = 1e-2;
  p->krylov_maxit = 300;
  p->restart = 30;
  p->precision = NC_PREC_MIXED;
  p->mg_levels = 0;
  p->nu_pre = 1;
  p->nu_post = 2;
  p->omega = 0.9;
  p->filter_rtol = 1e-12;
  p->timeout_s = 600.0;
  p->adjoint_rtol = 0.0;
  p->coarse_refactor = 0;
  p->krylov_eta_min = 0.0;
  p->adjoint_eta_first = 0.0;
  p->outer_arith = NC_ARITH_FP64;
  p->krylov_basis = NC_BASIS_FP64;
  p->krylov_reorth = 0.0;
  p->mg_tail_nodes = 0;
  p->mg_op0 = NC_MGOP_PICARD;
  p->mg_smoother = NC_SMOOTH_BLOCK_JACOBI;
  p->filter_method = NC_FILTER_SPECTRAL;
  p->mg_galerkin = NC_MGOP_PICARD;
  p->elem_chunk = -1;
  p->mg_reuse_below = 1e-2;
  p->adjoint_df64_steps = 1;
  return NC_OK;
}

nc_status nc_footprint_bytes(const nc_grid* g, const nc_params* p, size_t* bytes) {
  std::string why;
  if (!bytes) return NC_ERR_ARG;
  nc_status s = validate(g, p, &why);
  if (s != NC_OK) return fail(nullptr, s, why);
  *bytes = footprint(g, p);
  return NC_OK;
}

nc_status nc_create_problem(const nc_grid* gr, const nc_params* p, void* stream, nc_problem** out) {
  if (!out) return fail(nullptr, NC_ERR_ARG, "NULL output pointer");
  *out = nullptr;
  std::string why;
  nc_status vs = validate(gr, p, &why);
  if (vs != NC_OK) return fail(nullptr, vs, why);
  nc_problem* pb = new nc_problem();
  cudaGetDevice(&pb->device);
  pb->g = make_grid(gr->nx, gr->ny, gr->nz, gr->h);
  pb->g.bc = p->bc;
  pb->par = *p;
  pb->m = p->restart;
  const Grid& g = pb->g;
  apply_params(pb, p);
  if (stream) pb->st = (cudaStream_t)stream;
  else {
    cudaError_t e = cudaStreamCreateWithFlags(&pb->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { g_create_error = cudaGetErrorString(e); delete pb; return NC_ERR_CUDA; }
    pb->own_stream = true;
  }
  pb->lv = plan_levels(g, p->mg_levels);
  nc_status s = NC_OK;
  const long long nn = g.nn, ne = g.ne;
  auto A = [&](nc_status x) { if (s == NC_OK) s = x; };
  A(dalloc(pb, &pb->s, nn)); A(dalloc(pb, &pb->s_try, nn)); A(dalloc(pb, &pb->lam, nn)); A(dalloc(pb, &pb->s_start, nn));
  A(dalloc(pb, &pb->R, 2 * nn)); A(dalloc(pb, &pb->R_try, 2 * nn)); A(dalloc(pb, &pb->dx, 2 * nn));
  A(dalloc(pb, &pb->w, 2 * nn)); A(dalloc(pb, &pb->rhs, 2 * nn)); A(dalloc(pb, &pb->R0, 2 * nn));
  A(dalloc(pb, &pb->rho, ne)); A(dalloc(pb, &pb->gamma_t, ne)); A(dalloc(pb, &pb->gsens, ne)); A(dalloc(pb, &pb->u, 3 * ne));
  A(dalloc(pb, &pb->mat, ne)); A(dalloc(pb, &pb->dmat, ne)); A(dalloc(pb, &pb->dl, ne)); A(dalloc(pb, &pb->mat32, ne)); A(dalloc(pb, &pb->s32, nn));
  A(dalloc(pb, &pb->v32, nn)); A(dalloc(pb, &pb->y32, nn)); A(dalloc(pb, &pb->fz, ne));
  if (p->precision == NC_PREC_FP64 || p->krylov_basis == NC_BASIS_FP64) {
    A(dalloc(pb, &pb->V, (size_t)2 * nn * (pb->m + 1))); A(dalloc(pb, &pb->Z, (size_t)2 * nn * pb->m));
  } else {
    A(dalloc(pb, &pb->V32, (size_t)2 * nn * (pb->m + 1))); A(dalloc(pb, &pb->Z32, (size_t)2 * nn * pb->m));
  }
  if (p->precision != NC_PREC_FP64) {
    A(dalloc(pb, &pb->mat_df, ne)); A(dalloc(pb, &pb->s_df, nn)); A(dalloc(pb, &pb->w_df, nn));
  }
  A(dalloc(pb, &pb->part, 66 * kReduceBlocksMax)); A(dalloc(pb, &pb->dres, 132));
  A(dalloc(pb, &pb->fx, nn)); A(dalloc(pb, &pb->fb, nn)); A(dalloc(pb, &pb->fr, nn));
  A(dalloc(pb, &pb->fq, nn)); A(dalloc(pb, &pb->fdinv, nn));
  A(dalloc(pb, &pb->fxf, nn)); A(dalloc(pb, &pb->frf, nn)); A(dalloc(pb, &pb->fd0, nn)); A(dalloc(pb, &pb->fd1, nn));
  A(dalloc(pb, &pb->fdinvf, nn));
  A(dalloc(pb, &pb->fxd, nn)); A(dalloc(pb, &pb->fbd, nn));
  A(dalloc(pb, &pb->dflag, 1));
  if (s == NC_OK) s = spectral_setup(pb);
  if (s == NC_OK) s = p->precision == NC_PREC_FP64 ? mg_alloc<double>(pb) : mg_alloc<float>(pb);
  if (s == NC_OK) {
    cudaError_t e = cudaMallocHost(&pb->hres, sizeof(double) * 132);
    if (e == cudaSuccess) e = cudaMallocHost(&pb->hflag, sizeof(int));
    if (e != cudaSuccess) { cudaGetLastError(); s = fail(pb, NC_ERR_OOM, "pinned host allocation failed"); }
  }
  if (s == NC_OK) {
    cudaError_t e = launch_helmholtz_diag(g, pb->F, pb->fdinv, pb->st);
    if (e == cudaSuccess) e = launch_cast_d2f(pb->fdinvf, pb->fdinv, nn, pb->st, nullptr);
    if (e == cudaSuccess) e = cudaMemsetAsync(pb->s, 0, sizeof(double2) * nn, pb->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pb->st);
    if (e != cudaSuccess) s = cuda_fail(pb, e, "create");
  }
  if (s != NC_OK) {
    g_create_error = pb->err;
    nc_destroy_problem(pb);
    return s;
  }
  *out = pb;
  return NC_OK;
}

nc_status nc_destroy_problem(nc_problem* pb) {
  if (!pb) return NC_OK;
  DeviceGuard dg(pb->device);
  if (pb->st) cudaStreamSynchronize(pb->st);
  prof_flush(pb);
  drop_graphs(pb);
  for (cudaEvent_t e : pb->evpool) cudaEventDestroy(e);
  if (pb->blas) cublasDestroy(pb->blas);
  for (void* q : pb->allocs) cudaFree(q);
  if (pb->hres) cudaFreeHost(pb->hres);
  if (pb->hflag) cudaFreeHost(pb->hflag);
  if (pb->own_stream && pb->st) cudaStreamDestroy(pb->st);
  delete pb;
  return NC_OK;
}

nc_status nc_set_params(nc_problem* pb, const nc_params* p) {
  if (!pb || !p) return NC_ERR_ARG;
  nc_grid gr{pb->g.nx, pb->g.ny, pb->g.nz, pb->g.h};
  std::string why;
  nc_status vs = validate(&gr, p, &why);
  if (vs != NC_OK) return fail(pb, vs, why);
  if (p->precision != pb->par.precision || p->mg_levels != pb->par.mg_levels || p->restart != pb->par.restart ||
      p->krylov_basis != pb->par.krylov_basis || p->bc != pb->par.bc || p->mg_smoother != pb->par.mg_smoother)
    return fail(pb, NC_ERR_ARG, "precision, mg_levels, restart, krylov_basis, bc and mg_smoother are fixed at creation");
  DeviceGuard dg(pb->device);
  CKS(sync(pb, "set_params"));
  drop_graphs(pb);   // omega, sweeps and the tail choice are arguments of the captured launches
  apply_params(pb, p);
  CK(launch_helmholtz_diag(pb->g, pb->F, pb->fdinv, pb->st));   // the filter radius may have changed
  CK(launch_cast_d2f(pb->fdinvf, pb->fdinv, pb->g.nn, pb->st, nullptr));
  CKS(sync(pb, "set_params"));
  pb->have_R0 = false;   // R(0) depends on the source and the heated layers
  pb->mg32.factored = pb->mg64.factored = false;   // a new operator: invert the coarsest matrix anew
  pb->stage = 0;
  return NC_OK;
}

nc_status nc_set_design(nc_problem* pb, const double* rho) {
  if (!pb) return NC_ERR_ARG;
  DeviceGuard dg(pb->device);
  pb->t_start = now_s();
  const Grid& g = pb->g;
  CKS(copy_in(pb, pb->rho, rho, sizeof(double) * g.ne));
  CK(cudaMemsetAsync(pb->dflag, 0, sizeof(int), pb->st));
  PCK(NC_PROF_OTHER, launch_check_design(pb->rho, g.ne, pb->dflag, pb->st));
  CK(cudaMemcpyAsync(pb->hflag, pb->dflag, sizeof(int), cudaMemcpyDeviceToHost, pb->st));
  CKS(sync(pb, "design check"));
  if (*pb->hflag) return fail(pb, NC_ERR_ARG, "design values must be finite and in [0, 1]");
  // filter: b = T^T gamma with gamma = 1 on the heated region
  PCK(NC_PROF_FILTER, launch_filter_rhs(g, pb->ph, true, pb->rho, pb->F.t0, pb->fb, pb->st, &pb->cnt));
  CKS(filter_solve(pb));
  PCK(NC_PROF_FILTER, launch_elem_from_nodes(g, pb->ph, pb->fx, 0.125, 1.0, pb->gamma_t, pb->st, &pb->cnt));
  RampConst rc{pb->kappa_f, pb->kappa_s, pb->par.k_f, pb->par.k_s, pb->par.q_c, pb->par.q_p};
  PCK(NC_PROF_OTHER, launch_ramp(pb->gamma_t, g.ne, rc, pb->mat, pb->dmat, pb->mat32, pb->st, &pb->cnt));
  if (pb->mat_df) PCK(NC_PROF_OTHER, launch_split2(pb->mat, pb->mat_df, g.ne, pb->st, &pb->cnt));
  CK(cudaMemsetAsync(pb->s, 0, sizeof(double2) * g.nn, pb->st));
  CK(cudaMemsetAsync(pb->s_start, 0, sizeof(double2) * g.nn, pb->st));
  CKS(reference_norm(pb));
  pb->start_zero = true;
  pb->stage = 1;
  return NC_OK;
}

nc_status nc_set_state(nc_problem* pb, const double* P, const double* T) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "set_state needs a design");
  if (!P || !T) return fail(pb, NC_ERR_ARG, "NULL P or T");
  DeviceGuard dg(pb->device);
  const long long nn = pb->g.nn;
  CK(cudaMemcpy2DAsync((double*)pb->s_start, 16, P, 8, 8, nn, cudaMemcpyDefault, pb->st));
  CK(cudaMemcpy2DAsync((double*)pb->s_start + 1, 16, T, 8, 8, nn, cudaMemcpyDefault, pb->st));
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(pb->g, (double*)pb->s_start, pb->st, &pb->cnt));
  CK(cudaMemcpyAsync(pb->s, pb->s_start, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, pb->st));
  CKS(sync(pb, "set_state"));
  pb->start_zero = false;
  pb->stage = 1;
  return NC_OK;
}

nc_status nc_solve_state(nc_problem* pb, nc_stats* stats) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "solve_state needs a design");
  DeviceGuard dg(pb->device);
  pb->t_start = now_s();
  pb->total.launches += pb->cnt.launches;
  pb->total.bytes += pb->cnt.bytes;
  pb->cnt = Counters();
  if (stats) memset(stats, 0, sizeof(*stats));
  const long long nn = pb->g.nn;
  CK(cudaMemcpyAsync(pb->s, pb->s_start, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, pb->st));
  set_q_scale(pb, 1.0);
  pb->first_setup = true;
  pb->mg_ready = false;
  bool failed = false;
  nc_status s = newton(pb, pb->par.newton_rtol, pb->ref_norm, stats, &failed, pb->start_zero);
  if (s == NC_OK && failed) {
    // source ramping (Sec. 5.4): 1/4, 1/2, then the full source, each from the previous state
    if (stats) stats->ramped = 1;
    CK(cudaMemcpyAsync(pb->s, pb->s_start, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, pb->st));
    const double scales[3] = {0.25, 0.5, 1.0};
    for (int i = 0; i < 3 && s == NC_OK; ++i) {
      set_q_scale(pb, scales[i]);
      double ref = pb->ref_norm * scales[i];
      s = newton(pb, i < 2 ? std::max(1e-6, pb->par.newton_rtol) : pb->par.newton_rtol, ref, stats, &failed,
                 false);
      if (s == NC_OK && failed) s = fail(pb, NC_ERR_DIVERGED, "no damping factor reduces the residual");
    }
    set_q_scale(pb, 1.0);
  }
  if (stats) {
    stats->t_total_ms = 1e3 * (now_s() - pb->t_start);
    stats->alg_bytes = pb->cnt.bytes;
    stats->kernel_launches = pb->cnt.launches;
  }
  if (s == NC_OK) pb->stage = 2;
  return s;
}

nc_status nc_objective(nc_problem* pb, int objective, double* f) {
  if (!pb || !f) return NC_ERR_ARG;
  if (objective != NC_OBJ_MEAN_T_HEATED && objective != NC_OBJ_SUPG_COMPLIANCE)
    return fail(pb, NC_ERR_ARG, "unknown objective");
  if (pb->stage < 2) return fail(pb, NC_ERR_STATE, "objective needs a solved state");
  DeviceGuard dg(pb->device);
  const Grid& g = pb->g;
  if (objective == NC_OBJ_SUPG_COMPLIANCE) {
    set_q_scale(pb, 1.0);
    const long long nh = pb->ph.shape == 1 ? g.ne : (long long)g.nx * g.ny * pb->par.heated_layers;
    PCK(NC_PROF_OTHER, launch_obj_supg(g, pb->ph, pb->s, pb->mat, pb->gsens, pb->rhs, pb->st, &pb->cnt));
    PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, pb->rhs, pb->st, &pb->cnt));
    PCK(NC_PROF_OTHER, launch_sum(pb->gsens, nh, pb->part, pb->dres, pb->st, &pb->cnt));
    CK(cudaMemcpyAsync(pb->hres, pb->dres, sizeof(double), cudaMemcpyDeviceToHost, pb->st));
    CKS(sync(pb, "objective"));
    *f = pb->hres[0];
    return NC_OK;
  }
  PCK(NC_PROF_OTHER, launch_dfds(g, pb->ph, g.h * g.h * g.h / 8.0 / pb->vol_h, pb->rhs, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, pb->rhs, pb->st, &pb->cnt));
  CKS(dots(pb, pb->rhs, 0, 1, (const double*)pb->s, 2 * g.nn, f));
  return NC_OK;
}

nc_status nc_solve_adjoint(nc_problem* pb, int objective, double* f_out, nc_stats* stats) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 2) return fail(pb, NC_ERR_STATE, "solve_adjoint needs a solved state");
  DeviceGuard dg(pb->device);
  pb->t_start = now_s();
  pb->total.launches += pb->cnt.launches;
  pb->total.bytes += pb->cnt.bytes;
  pb->cnt = Counters();
  if (stats) memset(stats, 0, sizeof(*stats));
  double f;
  CKS(nc_objective(pb, objective, &f));   // leaves df/ds in rhs
  if (f_out) *f_out = f;
  const Grid& g = pb->g;
  const long long n = 2 * g.nn;
  set_q_scale(pb, 1.0);
  // The multigrid hierarchy of the last Newton step (built at the iterate before the converged
  // state) preconditions the transposed system; only the FP32 state copy of the Krylov operator is
  // refreshed. A hierarchy is built here if none exists for this state (e.g. a warm start that was
  // already converged).
  double t0 = now_s();
  if (pb->mg_ready) {
    if (pb->par.precision != NC_PREC_FP64)
      CKS(refresh_state32(pb, pb->s, NC_PROF_MG_COARSE_SETUP));
  } else {
    CKS(mg_setup_any(pb, true));
  }
  if (stats) stats->t_setup_ms += 1e3 * (now_s() - t0);
  double bb;
  CKS(norm2_free(pb, pb->rhs, &bb));
  const double bnorm = std::sqrt(bb);
  CK(cudaMemsetAsync(pb->lam, 0, sizeof(double) * n, pb->st));
  pb->dl_ready = false;
  if (bnorm == 0.0) { pb->stage = 3; return NC_OK; }
  const bool fp32 = pb->par.precision != NC_PREC_FP64;
  const double kAdjointRtol = pb->par.adjoint_rtol > 0 ? pb->par.adjoint_rtol : pb->par.newton_rtol;
  // refinement: r = b - J^T lam in FP64, correction from FGMRES on the (FP32 or FP64) operator.
  // With adjoint_df64_steps, a residual that cannot be expected to meet the tolerance (the previous
  // one times the reduction the last FGMRES reached is above 10x the tolerance) only steers the next
  // correction and is computed in double-float; acceptance is decided on an FP64 residual only.
  const bool steer_df = fp32 && pb->par.adjoint_df64_steps && !outer_df(pb);
  double rel_prev = 1.0, red_prev = 1.0;
  for (int pass = 0;; ++pass) {
    double rr;
    if (pass == 0) {
      CK(cudaMemcpyAsync(pb->w, pb->rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, pb->st));
      rr = bb;
    } else {
      // an FP64 pass stores the element design derivatives at this lambda; if it is the last
      // (converged) one, the sensitivities need no element sweep of their own
      const bool steer = steer_df && rel_prev * red_prev > 10.0 * kAdjointRtol;
      CKS(adjoint_residual(pb, steer, &rr));
      if (steer && std::sqrt(rr) / bnorm <= kAdjointRtol) CKS(adjoint_residual(pb, false, &rr));
    }
    const double rel = std::sqrt(rr) / bnorm;
    if (stats) {
      stats->rel_residual = rel;
      if (pass < 64) stats->res_hist[pass] = rel;
    }
    if (!std::isfinite(rel)) return fail(pb, NC_ERR_NAN, "non-finite adjoint residual");
    if (rel <= kAdjointRtol) {
      pb->dl_ready = pass > 0;   // the last J^T pass was at this (final) lambda
      break;
    }
    if (pass >= 30) return fail(pb, NC_ERR_MAXIT, "adjoint refinement did not converge");
    CKS(check_timeout(pb));
    int its;
    double lres;
    // FP32 inner solves: the first pass asks for 1e-5 and reaches a true reduction of about 1e-3
    // (the FP32 operator's accuracy on the smooth part of the error); later passes ask for what is
    // left to reach the tolerance (at least 1e-6), so that two passes usually suffice.
    // FP64: one pass to the tolerance.
    double eta;
    if (fp32) {
      const double first = pb->par.adjoint_eta_first > 0 ? pb->par.adjoint_eta_first : 1e-5;
      eta = pass == 0 ? first : std::max(1e-6, 0.3 * kAdjointRtol / rel);
    } else {
      eta = std::max(0.5 * kAdjointRtol / rel, 1e-12);
      if (pass == 0 && pb->par.adjoint_eta_first > 0) eta = pb->par.adjoint_eta_first;
    }
    double t1 = now_s();
    CKS(fgmres(pb, true, fp32, pb->w, pb->dx, std::min(eta, 1e-1), pb->par.krylov_maxit, &its, &lres));
    if (stats) {
      stats->t_krylov_ms += 1e3 * (now_s() - t1);
      stats->krylov_its += its;
      if (pass < 64) stats->krylov_hist[pass] = its;
      stats->newton_its++;
    }
    PCK(NC_PROF_OTHER, launch_axpby((double*)pb->lam, pb->dx, 1.0, 1.0, n, pb->st, &pb->cnt));
    rel_prev = rel;
    red_prev = lres;
  }
  CKS(sync(pb, "adjoint"));
  if (stats) {
    stats->t_total_ms = 1e3 * (now_s() - pb->t_start);
    stats->alg_bytes = pb->cnt.bytes;
    stats->kernel_launches = pb->cnt.launches;
  }
  pb->stage = 3;
  return NC_OK;
}

nc_status nc_sensitivities(nc_problem* pb, double* dfdrho) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 3) return fail(pb, NC_ERR_STATE, "sensitivities need a solved adjoint");
  if (!dfdrho) return fail(pb, NC_ERR_ARG, "NULL output");
  DeviceGuard dg(pb->device);
  pb->t_start = now_s();
  const Grid& g = pb->g;
  set_q_scale(pb, 1.0);
  if (pb->dl_ready)
    PCK(NC_PROF_SENS, launch_sens_from_dl(g, pb->ph, pb->dl, pb->dmat, pb->gsens, pb->st, &pb->cnt));
  else if (outer_df(pb))
    PCK(NC_PROF_SENS, launch_sens_df(g, pb->ph, pb->s, pb->lam, pb->mat_df, pb->dmat, pb->s_df, pb->w_df, pb->gsens,
                                     pb->st, &pb->cnt));
  else
    PCK(NC_PROF_SENS, launch_sens_elem(g, pb->ph, pb->s, pb->lam, pb->mat, pb->dmat, pb->gsens, pb->st, &pb->cnt));
  // filter transpose: gamma~_e = (1/8) sum_a x_a, x = A^-1 T^T gamma  =>  df/dgamma = T A^-1 (1/8 sum)
  PCK(NC_PROF_FILTER, launch_filter_rhs(g, pb->ph, false, pb->gsens, 0.125, pb->fb, pb->st, &pb->cnt));
  CKS(filter_solve(pb));
  PCK(NC_PROF_FILTER, launch_elem_from_nodes(g, pb->ph, pb->fx, pb->F.t0, 0.0, pb->gsens, pb->st, &pb->cnt));
  CKS(copy_out(pb, dfdrho, pb->gsens, sizeof(double) * g.ne));
  CKS(sync(pb, "sensitivities"));
  return NC_OK;
}

nc_status nc_get_fields(const nc_problem* cpb, double* P, double* T, double* u) {
  nc_problem* pb = const_cast<nc_problem*>(cpb);
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "no state yet");
  DeviceGuard dg(pb->device);
  const long long nn = pb->g.nn;
  if (P) CK(cudaMemcpy2DAsync(P, 8, (const double*)pb->s, 16, 8, nn, cudaMemcpyDefault, pb->st));
  if (T) CK(cudaMemcpy2DAsync(T, 8, (const double*)pb->s + 1, 16, 8, nn, cudaMemcpyDefault, pb->st));
  if (u) {
    PCK(NC_PROF_OTHER, launch_u_centroid(pb->g, pb->ph, pb->s, pb->mat, pb->u, pb->st, &pb->cnt));
    CKS(copy_out(pb, u, pb->u, sizeof(double) * 3 * pb->g.ne));
  }
  CKS(sync(pb, "get_fields"));
  return NC_OK;
}

nc_status nc_get_permeabilities(const nc_problem* pb, double* kappa_f, double* kappa_s) {
  if (!pb) return NC_ERR_ARG;
  if (kappa_f) *kappa_f = pb->kappa_f;
  if (kappa_s) *kappa_s = pb->kappa_s;
  return NC_OK;
}

nc_status nc_get_adjoint(const nc_problem* cpb, double* lam) {
  nc_problem* pb = const_cast<nc_problem*>(cpb);
  if (!pb || !lam) return NC_ERR_ARG;
  if (pb->stage < 3) return fail(pb, NC_ERR_STATE, "no adjoint solution yet");
  DeviceGuard dg(pb->device);
  CKS(copy_out(pb, lam, pb->lam, sizeof(double) * 2 * pb->g.nn));
  CKS(sync(pb, "get_adjoint"));
  return NC_OK;
}

nc_status nc_get_design_fields(const nc_problem* cpb, double* gamma_tilde, double* kappa, double* k) {
  nc_problem* pb = const_cast<nc_problem*>(cpb);
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "no design yet");
  DeviceGuard dg(pb->device);
  const long long ne = pb->g.ne;
  if (gamma_tilde) CKS(copy_out(pb, gamma_tilde, pb->gamma_t, sizeof(double) * ne));
  if (kappa) CK(cudaMemcpy2DAsync(kappa, 8, (const double*)pb->mat, 16, 8, ne, cudaMemcpyDefault, pb->st));
  if (k) CK(cudaMemcpy2DAsync(k, 8, (const double*)pb->mat + 1, 16, 8, ne, cudaMemcpyDefault, pb->st));
  CKS(sync(pb, "get_design_fields"));
  return NC_OK;
}

nc_status nc_eval_residual(nc_problem* pb, const double* s, double* R, double* norm2_free_out) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "residual needs a design");
  if (!R) return fail(pb, NC_ERR_ARG, "NULL output");
  DeviceGuard dg(pb->device);
  const long long n = 2 * pb->g.nn;
  set_q_scale(pb, 1.0);
  CKS(copy_in(pb, pb->s_try, s, sizeof(double) * n));
  double phi;
  CKS(residual(pb, pb->s_try, pb->R_try, &phi));
  if (norm2_free_out) *norm2_free_out = phi;
  CKS(copy_out(pb, R, pb->R_try, sizeof(double) * n));
  CKS(sync(pb, "eval_residual"));
  return NC_OK;
}

static nc_status apply_generic(nc_problem* pb, const double* s, const double* v, double* out, bool tr, bool fp32) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "operator needs a design");
  if (!out) return fail(pb, NC_ERR_ARG, "NULL output");
  DeviceGuard dg(pb->device);
  const long long n = 2 * pb->g.nn;
  set_q_scale(pb, 1.0);
  CKS(copy_in(pb, pb->s_try, s, sizeof(double) * n));
  CKS(copy_in(pb, pb->w, v, sizeof(double) * n));
  const Grid& g = pb->g;
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, pb->w, pb->st, &pb->cnt));   // the operator acts on free entries
  if (fp32) {
    CKS(refresh_state32(pb, pb->s_try, NC_PROF_OTHER));
    CKS(outer_op(pb, tr, true, pb->w, pb->R_try));
  } else {
    if (tr) CKS(outer_jtv(pb, NC_PROF_OTHER, pb->s_try, (const double2*)pb->w, pb->R_try));
    else PCK(NC_PROF_OTHER, launch_jv_f64(g, pb->ph, pb->s_try, pb->mat, (const double2*)pb->w, pb->R_try, pb->st, &pb->cnt));
  }
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, pb->R_try, pb->st, &pb->cnt));   // Dirichlet rows of the projected operator
  CKS(copy_out(pb, out, pb->R_try, sizeof(double) * n));
  CKS(sync(pb, "operator"));
  return NC_OK;
}

nc_status nc_apply_picard(nc_problem* pb, const double* s, const double* v, double* out, int transpose) {
  if (!pb) return NC_ERR_ARG;
  if (pb->stage < 1) return fail(pb, NC_ERR_STATE, "operator needs a design");
  if (!out) return fail(pb, NC_ERR_ARG, "NULL output");
  DeviceGuard dg(pb->device);
  const long long n = 2 * pb->g.nn;
  const Grid& g = pb->g;
  CKS(copy_in(pb, pb->s_try, s, sizeof(double) * n));
  CKS(copy_in(pb, pb->w, v, sizeof(double) * n));
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, pb->w, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_cast_d2f((float*)pb->s32, (const double*)pb->s_try, n, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_frozen(g, pb->ph, pb->s32, pb->mat32, pb->fz, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_cast_d2f((float*)pb->v32, pb->w, n, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_level0_picard(g, pb->ph, pb->fz, pb->mat32, pb->v32, pb->y32, transpose != 0, pb->st, &pb->cnt, pb->par.elem_chunk));
  PCK(NC_PROF_OTHER, launch_cast_f2d(pb->R_try, (const float*)pb->y32, n, pb->st, &pb->cnt));
  PCK(NC_PROF_OTHER, launch_zero_dirichlet(g, pb->R_try, pb->st, &pb->cnt));
  CKS(copy_out(pb, out, pb->R_try, sizeof(double) * n));
  CKS(sync(pb, "operator"));
  return NC_OK;
}

nc_status nc_apply_jacobian(nc_problem* pb, const double* s, const double* v, double* out, int precision) {
  return apply_generic(pb, s, v, out, false, precision != NC_PREC_FP64);
}

nc_status nc_apply_jacobian_transpose(nc_problem* pb, const double* s, const double* w, double* out) {
  return apply_generic(pb, s, w, out, true, false);
}

nc_status nc_set_profiling(nc_problem* pb, int class_mask) {
  if (!pb) return NC_ERR_ARG;
  DeviceGuard dg(pb->device);
  CKS(sync(pb, "set_profiling"));
  pb->prof_mask = class_mask;
  for (int c = 0; c < NC_PROF_NCLASSES; ++c) {
    pb->prof_ms[c] = 0; pb->prof_n[c] = 0; pb->prof_bytes[c] = 0; pb->prof_flops[c] = 0;
  }
  return NC_OK;
}

nc_status nc_get_profile(const nc_problem* cpb, int cls, double* ms, long long* launches, double* bytes,
                         double* flops) {
  nc_problem* pb = const_cast<nc_problem*>(cpb);
  if (!pb || cls < 0 || cls >= NC_PROF_NCLASSES) return NC_ERR_ARG;
  DeviceGuard dg(pb->device);
  CKS(sync(pb, "get_profile"));
  if (ms) *ms = pb->prof_ms[cls];
  if (launches) *launches = pb->prof_n[cls];
  if (bytes) *bytes = pb->prof_bytes[cls];
  if (flops) *flops = pb->prof_flops[cls];
  return NC_OK;
}

nc_status nc_counters(const nc_problem* cpb, long long* launches, double* bytes) {
  nc_problem* pb = const_cast<nc_problem*>(cpb);
  if (!pb) return NC_ERR_ARG;
  if (launches) *launches = pb->total.launches + pb->cnt.launches;
  if (bytes) *bytes = pb->total.bytes + pb->cnt.bytes;
  return NC_OK;
}

const char* nc_last_error(const nc_problem* pb) {
  if (!pb) return g_create_error.c_str();
  return pb->err.empty() ? "no error" : pb->err.c_str();
}

}  // extern "C"
