// Allocation-free variant of the two-pass Gram-Schmidt entry point.
//
// mor_orthonormalize needs a handle, and the handle allocates its own device
// workspace.  Some callers cannot let a library allocate: a framework whose
// caching allocator owns all device memory and has been given a fixed budget,
// an embedded or real-time loop that must keep its memory map constant, or
// code that must not pay cudaMalloc / cudaFree's implicit device
// synchronisation.  This file serves them with a handle-free entry point
// whose scratch (the per-block partial sums of the Gram kernel, the
// Gram-Schmidt coefficients and the block counters) lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded and
// held by every GPU that loads it until the process exits.
#include "mor_spai.h"
#include "mor_internal.h"
#include <algorithm>
#include <mutex>

namespace {

constexpr int NA_MAXK = 64;              // widest block accepted
// Gram-kernel grid cap: 4 blocks per SM of the device, at most NA_GRID (the
// capacity of the partials region; the skinny Gram kernel uses at most
// NA_GRID / 2 blocks per group of 8 columns, 8 groups, 8 partials each)
constexpr int NA_GRID = 608;
constexpr size_t NA_H = 0;                               // Gram-Schmidt coefficients (64)
constexpr size_t NA_NORMS = 64;                          // per-column norms (2 x 64)
constexpr size_t NA_PART = NA_NORMS + 2 * NA_MAXK;       // block partials (NA_GRID x 64)
constexpr size_t NA_CNT = NA_PART + (size_t)NA_GRID * NA_MAXK;   // block counters (8 words used)
constexpr size_t NA_DOUBLES = NA_CNT + 32;               // 39,136 doubles = 313,088 bytes in total
static_assert(NA_DOUBLES * sizeof(double) == 313088, "scratch size stated in the header");

__device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

std::mutex g_mu;
double* g_addr[64] = {nullptr};          // device address of the scratch, per device

}  // namespace

extern "C" int mor_orthonormalize_noalloc(double* X, int64_t n, int k, void* stream) {
  if (!X || n < 1 || n > 0x7fffffffLL || k < 1 || k > NA_MAXK) return MOR_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MOR_ECUDA;
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MOR_ECUDA;
      g_addr[dev] = (double*)p;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return MOR_ECUDA;
  const int grid_cap = std::min(NA_GRID, 4 * sms);
  double* hbuf = base + NA_H;
  double* norms = base + NA_NORMS;
  double* part = base + NA_PART;
  unsigned* counter = (unsigned*)(base + NA_CNT);
  // the array keeps whatever the previous call left: the counters (one per
  // group of eight columns of the Gram kernel) must start at zero
  if (cudaMemsetAsync(counter, 0, 8 * sizeof(unsigned), s) != cudaSuccess) return MOR_ECUDA;
  for (int j = 0; j < k; ++j) {
    double* v = X + (size_t)j * n;
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      if (dense_launch_gram((int)n, j, 1, X, n, v, n, hbuf, part, counter, grid_cap, s)) return MOR_ECUDA;
      if (dense_launch_gs_update((int)n, j, X, n, hbuf, v, s)) return MOR_ECUDA;
    }
    if (dense_launch_gram((int)n, 1, 1, v, n, v, n, norms + j, part, counter, grid_cap, s)) return MOR_ECUDA;
    if (dense_launch_scale((int)n, v, norms + j, s)) return MOR_ECUDA;
  }
  return MOR_OK;
}
