// Residual norm without any device allocation.
//
// Some callers cannot let a library allocate GPU memory: an application that gives every component
// a fixed slice of device memory through its own pool, and enforces that budget, would have its
// accounting bypassed (or the call fail under a hard cap); a latency-critical loop cannot afford the
// device-wide synchronisation that cudaMalloc and cudaFree may imply, which stalls work queued on
// other streams.  This entry point therefore keeps its scratch (the partial sums of the reduction)
// in a fixed array that is part of the loaded module, and allocates nothing at call time.
#include <mutex>

#include "internal.cuh"

#define NOALLOC_TILE 1024          // cells per partial sum
#define NOALLOC_MAX_TILES 65536    // partial sums held by the module (512 KiB)

// scratch shared by every call: one partial sum per tile of NOALLOC_TILE cells; each call overwrites
// the entries it uses, so nothing has to start at zero
static __device__ __align__(256) double g_norm_tiles[NOALLOC_MAX_TILES];

// device addresses of g_norm_tiles, looked up once per device (host code may not use the symbol
// itself as an address)
static std::mutex g_tiles_mutex;
static double* g_tiles_ptr[64] = {nullptr};

__global__ void k_norm_tile_sums(int64_t n, const double* __restrict__ res_rho, const double* __restrict__ vol,
                                 double* __restrict__ tiles) {
  __shared__ double s[256];
  const int64_t base = (int64_t)blockIdx.x * NOALLOC_TILE;
  double acc = 0.0;
  for (int k = threadIdx.x; k < NOALLOC_TILE; k += blockDim.x) {
    const int64_t i = base + k;
    if (i < n) {
      const double x = res_rho[i] / vol[i];
      acc += x * x;
    }
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) tiles[blockIdx.x] = s[0];
}

__global__ void k_norm_tile_total(int64_t ntiles, int64_t n, const double* __restrict__ tiles, double* __restrict__ out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) acc += tiles[t];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(s[0] / (double)n);
}

extern "C" cgks_status cgks_density_norm_noalloc(const double* res_rho, const double* vol, int64_t n,
                                                 void* cuda_stream, double* norm) {
  if (!res_rho || !vol || !norm || n <= 0) return cgks_fail(nullptr, CGKS_EINVAL, "cgks_density_norm_noalloc: NULL array or n <= 0");
  const int64_t ntiles = (n + NOALLOC_TILE - 1) / NOALLOC_TILE;
  if (ntiles > NOALLOC_MAX_TILES)
    return cgks_fail(nullptr, CGKS_EINVAL,
                     "cgks_density_norm_noalloc: n = " + std::to_string(n) + " exceeds the maximum of " +
                         std::to_string((int64_t)NOALLOC_MAX_TILES * NOALLOC_TILE) + " cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cgks_fail(nullptr, CGKS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return cgks_fail(nullptr, CGKS_EUNSUPPORTED, "cgks_density_norm_noalloc: device index >= 64");
  double* tiles = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_tiles_mutex);
    if (!g_tiles_ptr[dev]) {
      // first call on this device: look up the device address of the module's scratch array
      e = cudaGetSymbolAddress((void**)&g_tiles_ptr[dev], g_norm_tiles);
      if (e != cudaSuccess) {
        g_tiles_ptr[dev] = nullptr;
        return cgks_fail(nullptr, CGKS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    tiles = g_tiles_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_norm_tile_sums<<<(unsigned)ntiles, 256, 0, st>>>(n, res_rho, vol, tiles);
  k_norm_tile_total<<<1, 256, 0, st>>>(ntiles, n, tiles, norm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cgks_fail(nullptr, CGKS_ECUDA, std::string("cgks_density_norm_noalloc: ") + cudaGetErrorString(e));
  return CGKS_OK;
}
