// Common types and index helpers of the natconv CUDA library.
//
// Grid: nx x ny x nz cubic Q1 elements of edge h; node (i,j,k) -> i + NX*(j + NY*k) with
// NX = nx+1, NY = ny+1 (x fastest); element (i,j,k) -> i + nx*(j + ny*k). A state vector is
// node-interleaved (P, T): double2 (FP64) or float2 (FP32) per node. Dirichlet values are 0; the
// fixed set depends on the boundary conditions (Grid::bc): kBcTop fixes P and T on the top node plane
// k = nz; kBcCavity (the quarter of a closed cavity, symmetry planes x = 0 and y = 0) fixes T on the
// outer walls i = nx, j = ny and the top k = nz, and P at the top outer corner (nx, ny, nz). Both sets
// are unions of grid planes and a grid corner, so on every multigrid level they are the same planes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nc {

constexpr int kBcTop = 0, kBcCavity = 1;

struct Grid {
  int nx, ny, nz;   // elements
  int NX, NY, NZ;   // nodes per direction
  int NXY;          // nodes per z-plane
  long long nn;     // nodes (< 2^31: node indices fit in int)
  long long ne;     // elements
  double h;
  int bc;           // kBcTop or kBcCavity
};

// Fixed components of node (i, j, k): bit 0 P, bit 1 T.
__host__ __device__ __forceinline__ int fixed_bits(const Grid& g, int i, int j, int k) {
  if (g.bc == kBcTop) return k == g.nz ? 3 : 0;
  const int t = (i == g.nx || j == g.ny || k == g.nz) ? 2 : 0;
  return t | ((i == g.nx && j == g.ny && k == g.nz) ? 1 : 0);
}

// Nodes carrying fixed components, enumerated plane by plane (kBcTop: the top plane; kBcCavity: the
// top plane, then the planes i = nx and j = ny; edge nodes appear in more than one plane).
__host__ __device__ __forceinline__ long long boundary_count(const Grid& g) {
  return g.bc == kBcTop ? (long long)g.NXY : (long long)g.NXY + (long long)g.NY * g.NZ + (long long)g.NX * g.NZ;
}
__device__ __forceinline__ bool boundary_node(const Grid& g, long long t, int& i, int& j, int& k) {
  if (t < g.NXY) { k = g.nz; j = (int)(t / g.NX); i = (int)(t - (long long)j * g.NX); return true; }
  if (g.bc == kBcTop) return false;
  t -= g.NXY;
  if (t < (long long)g.NY * g.NZ) { i = g.nx; k = (int)(t / g.NY); j = (int)(t - (long long)k * g.NY); return true; }
  t -= (long long)g.NY * g.NZ;
  if (t < (long long)g.NX * g.NZ) { j = g.ny; k = (int)(t / g.NX); i = (int)(t - (long long)k * g.NX); return true; }
  return false;
}

// Free (P, T) rows of the level's dense coarse system: kBcTop keeps the nodes below the top plane
// (their rows lead the node order); kBcCavity keeps every node (fixed rows become identity rows).
inline int coarse_rows(const Grid& g) {
  return g.bc == kBcTop ? 2 * g.NX * g.NY * g.nz : (int)(2 * g.nn);
}

inline Grid make_grid(int nx, int ny, int nz, double h) {
  Grid g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.NX = nx + 1; g.NY = ny + 1; g.NZ = nz + 1;
  g.NXY = g.NX * g.NY;
  g.nn = (long long)g.NX * g.NY * g.NZ;
  g.ne = (long long)nx * ny * nz;
  g.h = h;
  g.bc = kBcTop;
  return g;
}

template <typename R> struct Vec2;
template <> struct Vec2<double> { typedef double2 type; };
template <> struct Vec2<float> { typedef float2 type; };

template <typename R>
__device__ __forceinline__ typename Vec2<R>::type mk2(R a, R b) {
  typename Vec2<R>::type v; v.x = a; v.y = b; return v;
}

// Atomic add of a (P, T) pair to p[0], p[1] (p 8-byte aligned for float: one vector reduction).
__device__ __forceinline__ void atomic_add_pair(float* p, float a, float b) {
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(a, b));
}
__device__ __forceinline__ void atomic_add_pair(double* p, double a, double b) {
  atomicAdd(p, a);
  atomicAdd(p + 1, b);
}

// Node index of local corner a = ax + 2 ay + 4 az of element (i,j,k).
__device__ __forceinline__ long long corner_node(const Grid& g, int i, int j, int k, int a) {
  return (long long)(i + (a & 1)) + (long long)g.NX * ((j + ((a >> 1) & 1)) + (long long)g.NY * (k + (a >> 2)));
}

__device__ __forceinline__ void elem_ijk(const Grid& g, long long e, int& i, int& j, int& k) {
  i = (int)(e % g.nx);
  long long r = e / g.nx;
  j = (int)(r % g.ny);
  k = (int)(r / g.ny);
}

__device__ __forceinline__ void node_ijk(const Grid& g, long long n, int& i, int& j, int& k) {
  i = (int)(n % g.NX);
  long long r = n / g.NX;
  j = (int)(r % g.NY);
  k = (int)(r / g.NY);
}

// Node offset of local corner a = ax + 2 ay + 4 az from corner 0 of an element.
__device__ __forceinline__ int corner_off(const Grid& g, int a) {
  return (a & 1) + ((a >> 1) & 1) * g.NX + (a >> 2) * g.NXY;
}

// 3D launch geometry: blocks of 32 x 4 threads over (i, j), one z-slice per blockIdx.z.
struct Launch3 { dim3 grid, block; };
inline Launch3 launch_elems(const Grid& g) {
  Launch3 L;
  L.block = dim3(32, 4, 1);
  L.grid = dim3((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 3) / 4), (unsigned)g.nz);
  return L;
}
inline Launch3 launch_nodes(const Grid& g) {
  Launch3 L;
  L.block = dim3(32, 4, 1);
  L.grid = dim3((unsigned)((g.NX + 31) / 32), (unsigned)((g.NY + 3) / 4), (unsigned)g.NZ);
  return L;
}
// Flat launch over the nodes of one z-plane per blockIdx.y (no idle lanes when NX is not a multiple
// of the block width): blockIdx.x * blockDim.x + threadIdx.x indexes the NX * NY nodes of plane
// k = blockIdx.y.
inline Launch3 launch_nodes_flat(const Grid& g, int threads = 128) {
  Launch3 L;
  L.block = dim3(threads, 1, 1);
  L.grid = dim3((unsigned)((g.NXY + threads - 1) / threads), (unsigned)g.NZ, 1);
  return L;
}
#define NC_NODE_FLAT(g)                                                      \
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;                    \
  if (pidx >= (g).NXY) return;                                               \
  const int k = blockIdx.y;                                                  \
  const int j = pidx / (g).NX;                                               \
  const int i = pidx - j * (g).NX;

#define NC_IJK_3D()                                   \
  const int i = blockIdx.x * 32 + threadIdx.x;        \
  const int j = blockIdx.y * 4 + threadIdx.y;         \
  const int k = blockIdx.z;

inline unsigned grid_blocks(long long work, int threads, long long cap = 1LL << 30) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

}  // namespace nc
