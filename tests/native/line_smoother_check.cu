// Check of the z-line block-Jacobi smoother kernels of the library (nc::launch_line_factor and
// nc::launch_line_smooth, called through the library's exported launchers) against a dense FP64
// solve of every node column's block-tridiagonal system, written out here.
//
// A random 27-point stencil of 2x2 blocks (diagonal blocks made dominant, rows and columns of fixed
// components zero as the library's stencil assembly leaves them) is set on small grids with both
// boundary-condition sets. For the operator A and for its transpose the program checks
//   first:  x = omega T^-1 r           (T: the column-tridiagonal part of A or A^T)
//   update: x = x0 + omega T^-1 r
// where the dense reference forms T of each column from the stencil (transposed operator: block
// (n, m) of A^T is block (m, n) of A, transposed), keeps the free components, and solves it by
// Gaussian elimination with partial pivoting. Prints one line per check and "ALL OK" at the end;
// exits 1 on a mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "nc_launch.h"

using namespace nc;

static Grid grid(int nx, int ny, int nz, int bc) {
  Grid g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.NX = nx + 1; g.NY = ny + 1; g.NZ = nz + 1;
  g.NXY = g.NX * g.NY;
  g.nn = (long long)g.NXY * g.NZ;
  g.ne = (long long)nx * ny * nz;
  g.h = 1.0 / nz;
  g.bc = bc;
  return g;
}

// entry (f, c) of block o at node n of A (row field f, column field c)
template <typename R>
static double blk(const std::vector<R>& S, const Grid& g, int o, long long n, int f, int c) {
  return (double)S[((long long)o * g.nn + n) * 4 + 2 * f + c];
}

// dense solve (partial pivoting) of M z = v, M m x m row-major; returns false if singular
static bool dense_solve(std::vector<double> M, std::vector<double>& v, int m) {
  for (int p = 0; p < m; ++p) {
    int q = p;
    for (int r = p + 1; r < m; ++r)
      if (std::fabs(M[(size_t)r * m + p]) > std::fabs(M[(size_t)q * m + p])) q = r;
    if (M[(size_t)q * m + p] == 0.0) return false;
    if (q != p) {
      for (int c = 0; c < m; ++c) std::swap(M[(size_t)p * m + c], M[(size_t)q * m + c]);
      std::swap(v[p], v[q]);
    }
    for (int r = p + 1; r < m; ++r) {
      const double f = M[(size_t)r * m + p] / M[(size_t)p * m + p];
      if (f == 0.0) continue;
      for (int c = p; c < m; ++c) M[(size_t)r * m + c] -= f * M[(size_t)p * m + c];
      v[r] -= f * v[p];
    }
  }
  for (int p = m - 1; p >= 0; --p) {
    double s = v[p];
    for (int c = p + 1; c < m; ++c) s -= M[(size_t)p * m + c] * v[c];
    v[p] = s / M[(size_t)p * m + p];
  }
  return true;
}

template <typename R>
static int run_case(int nx, int ny, int nz, int bc, unsigned seed, double tol) {
  typedef typename Vec2<R>::type V2;
  const Grid g = grid(nx, ny, nz, bc);
  const long long nn = g.nn;
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<R> S(27 * nn * 4);
  for (long long n = 0; n < nn; ++n) {
    const int i = (int)(n % g.NX), j = (int)((n / g.NX) % g.NY), k = (int)(n / g.NXY);
    const int rb = fixed_bits(g, i, j, k);
    for (int o = 0; o < 27; ++o) {
      const int oi = o % 3 - 1, oj = (o / 3) % 3 - 1, ok = o / 9 - 1;
      const int mi = i + oi, mj = j + oj, mk = k + ok;
      const bool valid = mi >= 0 && mi <= g.nx && mj >= 0 && mj <= g.ny && mk >= 0 && mk <= g.nz;
      const int cb = valid ? fixed_bits(g, mi, mj, mk) : 3;
      for (int q = 0; q < 4; ++q) {
        const int f = q >> 1, c = q & 1;
        double v = valid ? U(rng) : 0.0;
        if (o == 13 && f == c) v += (v >= 0 ? 6.0 : -6.0);      // dominant diagonal
        if (((rb >> f) & 1) || ((cb >> c) & 1)) v = 0.0;
        S[((long long)o * nn + n) * 4 + q] = (R)v;
      }
    }
  }
  std::vector<V2> r(nn), x0(nn);
  for (long long n = 0; n < nn; ++n) {
    const int i = (int)(n % g.NX), j = (int)((n / g.NX) % g.NY), k = (int)(n / g.NXY);
    const int fb = fixed_bits(g, i, j, k);
    r[n].x = (R)U(rng); r[n].y = (R)U(rng);
    x0[n].x = (fb & 1) ? R(0) : (R)U(rng);
    x0[n].y = (fb & 2) ? R(0) : (R)U(rng);
  }
  const R omega = (R)0.8;
  R *dS, *dLF;
  V2 *dr, *dx;
  int* dflag;
  cudaMalloc(&dS, sizeof(R) * S.size());
  cudaMalloc(&dLF, sizeof(R) * 24 * nn);
  cudaMalloc(&dr, sizeof(V2) * nn);
  cudaMalloc(&dx, sizeof(V2) * nn);
  cudaMalloc(&dflag, sizeof(int));
  cudaMemcpy(dS, S.data(), sizeof(R) * S.size(), cudaMemcpyHostToDevice);
  cudaMemset(dflag, 0, sizeof(int));
  if (launch_line_factor<R>(g, dS, dLF, dflag, 0, nullptr) != cudaSuccess) { printf("factor launch failed\n"); return 1; }
  int flag = 0;
  cudaMemcpy(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost);
  if (flag) { printf("factor flagged a singular block\n"); return 1; }
  int bad = 0;
  for (int tr = 0; tr < 2; ++tr) {
    for (int first = 1; first >= 0; --first) {
      cudaMemcpy(dr, r.data(), sizeof(V2) * nn, cudaMemcpyHostToDevice);
      cudaMemcpy(dx, x0.data(), sizeof(V2) * nn, cudaMemcpyHostToDevice);
      if (launch_line_smooth<R>(g, dLF, dr, dx, omega, tr != 0, first != 0, 0, nullptr) != cudaSuccess) {
        printf("smooth launch failed\n");
        return 1;
      }
      std::vector<V2> x(nn);
      if (cudaMemcpy(x.data(), dx, sizeof(V2) * nn, cudaMemcpyDeviceToHost) != cudaSuccess) { printf("copy failed\n"); return 1; }
      double err = 0.0, ref = 0.0;
      for (int c = 0; c < g.NXY; ++c) {
        const int i = c % g.NX, j = c / g.NX, K = g.nz + 1;
        // free components of the column and their positions
        std::vector<int> idx;   // 2 k + f
        for (int k = 0; k < K; ++k)
          for (int f = 0; f < 2; ++f)
            if (!((fixed_bits(g, i, j, k) >> f) & 1)) idx.push_back(2 * k + f);
        const int m = (int)idx.size();
        std::vector<double> M((size_t)m * m, 0.0), v(m);
        for (int a = 0; a < m; ++a) {
          const int ka = idx[a] / 2, fa = idx[a] % 2;
          const long long na = c + (long long)g.NXY * ka;
          v[a] = fa ? (double)r[na].y : (double)r[na].x;
          for (int b = 0; b < m; ++b) {
            const int kb = idx[b] / 2, fb = idx[b] % 2;
            if (std::abs(kb - ka) > 1) continue;
            const long long nb = c + (long long)g.NXY * kb;
            // A: row node na, offset kb - ka; A^T: block (na, nb) of A^T = block (nb, na) of A transposed
            M[(size_t)a * m + b] = tr ? blk(S, g, 13 + 9 * (ka - kb), nb, fb, fa) : blk(S, g, 13 + 9 * (kb - ka), na, fa, fb);
          }
        }
        if (!dense_solve(M, v, m)) { printf("reference singular\n"); return 1; }
        std::vector<double> d(2 * K, 0.0);
        for (int a = 0; a < m; ++a) d[idx[a]] = v[a];
        for (int k = 0; k < K; ++k) {
          const long long n = c + (long long)g.NXY * k;
          const double e0 = (first ? 0.0 : (double)x0[n].x) + (double)omega * d[2 * k];
          const double e1 = (first ? 0.0 : (double)x0[n].y) + (double)omega * d[2 * k + 1];
          err = std::fmax(err, std::fmax(std::fabs((double)x[n].x - e0), std::fabs((double)x[n].y - e1)));
          ref = std::fmax(ref, std::fmax(std::fabs(e0), std::fabs(e1)));
        }
      }
      const bool ok = err <= tol * ref;
      printf("%s %dx%dx%d bc=%d %s %s: max |x - x_ref| / max |x_ref| = %.3e %s\n", sizeof(R) == 4 ? "float" : "double",
             nx, ny, nz, bc, tr ? "transpose" : "forward", first ? "first" : "update", err / ref, ok ? "ok" : "FAIL");
      bad += ok ? 0 : 1;
    }
  }
  cudaFree(dS); cudaFree(dLF); cudaFree(dr); cudaFree(dx); cudaFree(dflag);
  return bad;
}

int main() {
  int bad = 0;
  // column lengths (nz + 1 nodes) below, at and above the 32-node chunks of the solve
  bad += run_case<float>(6, 5, 9, kBcTop, 1, 2e-5);
  bad += run_case<float>(4, 6, 16, kBcCavity, 2, 2e-5);
  bad += run_case<float>(3, 3, 1, kBcCavity, 3, 2e-5);
  bad += run_case<float>(3, 2, 31, kBcTop, 6, 2e-5);
  bad += run_case<float>(2, 3, 32, kBcCavity, 7, 2e-5);
  bad += run_case<float>(3, 3, 70, kBcCavity, 8, 2e-5);
  bad += run_case<double>(6, 5, 9, kBcCavity, 4, 1e-12);
  bad += run_case<double>(5, 4, 12, kBcTop, 5, 1e-12);
  bad += run_case<double>(2, 2, 63, kBcTop, 9, 1e-12);
  bad += run_case<double>(3, 2, 100, kBcCavity, 10, 1e-12);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("device error\n"); return 1; }
  printf(bad ? "FAILED %d\n" : "ALL OK\n", bad);
  return bad ? 1 : 0;
}
