// Allocation-free variant of the free-DOF squared-norm reduction (the norm of the Newton stopping
// test). Its per-block partial sums live in a fixed file-scope device array instead of buffers
// owned by an nc_problem, so a caller can evaluate it without any device allocation: for callers
// that hand out all device memory from their own pre-reserved pool, run under a hard memory
// budget, or must not call cudaMalloc / cudaFree on this path because those calls can synchronise
// the device.
//
// The array is shared by every call on a device and keeps the last call's contents. Every block
// overwrites its own slot before the final sum reads it, so nothing has to start at zero; calls that
// overlap on the GPU (different streams or host threads without ordering) race on the array.
#include <mutex>

#include "natconv.h"
#include "nc_common.cuh"

namespace {

// One partial sum per NC_NOALLOC_CHUNK free entries; NC_NOALLOC_MAX_PARTS partials at most
// (64 KiB of device memory held by every device that loads the library, until exit).
#define NC_NOALLOC_CHUNK 4096
#define NC_NOALLOC_MAX_PARTS 8192

static __device__ __align__(256) double g_noalloc_parts[NC_NOALLOC_MAX_PARTS];

// Partial sums of squares over NC_NOALLOC_CHUNK entries per block. With kBcTop the free rows are the
// leading 2 NX NY nz entries (nodes below the top plane) and nfree2 is their count; otherwise every
// row of the 2 nn entries is visited and the fixed components of the grid's set are skipped.
__global__ void k_noalloc_norm2_parts(nc::Grid g, const double* __restrict__ a, long long nfree2,
                                      double* __restrict__ parts) {
  __shared__ double sh[32];
  const long long lo = (long long)blockIdx.x * NC_NOALLOC_CHUNK;
  const long long hi = min(nfree2, lo + NC_NOALLOC_CHUNK);
  double acc = 0.0;
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (g.bc != nc::kBcTop) {
      int i, j, k;
      nc::node_ijk(g, t >> 1, i, j, k);
      if ((nc::fixed_bits(g, i, j, k) >> (t & 1)) & 1) continue;
    }
    acc += a[t] * a[t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    parts[blockIdx.x] = s;
  }
}

__global__ void k_noalloc_sum(const double* __restrict__ parts, int nparts, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += parts[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    *out = r;
  }
}

// Device address of g_noalloc_parts, looked up once per device (with that device current) at the
// first call on it and kept for the life of the process. A cudaDeviceReset ends the context that
// address belongs to: a process that resets a device must not call this entry point on it again.
const int kMaxDevices = 64;
double* g_parts_addr[kMaxDevices] = {nullptr};
std::mutex g_parts_mutex;

cudaError_t parts_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_parts_mutex);
  if (!g_parts_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_parts);
    if (e != cudaSuccess) return e;
    g_parts_addr[dev] = (double*)p;
  }
  *out = g_parts_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" nc_status nc_norm2_free_noalloc(const nc_grid* g, int bc, const double* s_dev, double* out_dev,
                                           void* stream) {
  if (!g || !s_dev || !out_dev) return NC_ERR_ARG;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return NC_ERR_ARG;
  if (bc != NC_BC_TOP && bc != NC_BC_CAVITY) return NC_ERR_ARG;
  nc::Grid gr = nc::make_grid(g->nx, g->ny, g->nz, g->h);
  gr.bc = bc == NC_BC_TOP ? nc::kBcTop : nc::kBcCavity;
  if (gr.nn >= (1LL << 31)) return NC_ERR_ARG;
  const long long nfree2 = bc == NC_BC_TOP ? 2LL * gr.NXY * gr.nz : 2LL * gr.nn;
  const long long nparts = (nfree2 + NC_NOALLOC_CHUNK - 1) / NC_NOALLOC_CHUNK;
  if (nparts > NC_NOALLOC_MAX_PARTS) return NC_ERR_ARG;   // beyond the fixed scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { cudaGetLastError(); return NC_ERR_CUDA; }
  double* parts = nullptr;
  if (parts_address(dev, &parts) != cudaSuccess) { cudaGetLastError(); return NC_ERR_CUDA; }
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_norm2_parts<<<(unsigned)nparts, 256, 0, st>>>(gr, s_dev, nfree2, parts);
  k_noalloc_sum<<<1, 256, 0, st>>>(parts, (int)nparts, out_dev);
  return cudaGetLastError() == cudaSuccess ? NC_OK : NC_ERR_CUDA;
}
