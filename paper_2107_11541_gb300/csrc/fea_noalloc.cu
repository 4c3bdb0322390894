// fea_noalloc.cu -- CSR row pointers from per-row counts without allocating device memory.
//
// This is the row-pointer scan of fea_pattern_build offered on its own for callers that
// cannot allocate: for example a program whose device memory all belongs to another
// allocator (a framework's memory pool or a fixed arena) and which must not let a library
// call cudaMalloc behind its back.  The caller passes the counts and the output; the
// per-tile partial sums the scan needs live in a fixed array in this file instead of in a
// temporary allocation.
#include <cuda_runtime.h>

#include <mutex>

#include "fea_internal.cuh"

namespace fea {
namespace noalloc {

constexpr int THREADS = 256;
constexpr int ITEMS = 8;
constexpr int TILE = THREADS * ITEMS;          // counts summed per block
constexpr int64_t MAX_TILES = 16384;           // scratch entries: rows up to MAX_TILES * TILE
constexpr int64_t MAX_ROWS = MAX_TILES * TILE; // 33,554,432

// Per-tile sums shared by every call of fea_csr_rowptr_noalloc in this process (128 KiB on
// each device that loads the library).  Host code must not pass the symbol itself to a
// kernel: it is a host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) int64_t g_tile_sums[MAX_TILES];

constexpr int MAX_DEVICES = 64;
static std::mutex g_mu;
static int64_t* g_scratch[MAX_DEVICES] = {nullptr};

// Device address of g_tile_sums on the current device, looked up once per device and kept for
// the life of the process (a cudaDeviceReset would invalidate it; the header says so).
static fea_status scratch_address(int64_t** out) {
  int dev = 0;
  FEA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(FEA_ERR_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tile_sums);
    if (e != cudaSuccess)
      return fail(FEA_ERR_CUDA, "cudaGetSymbolAddress of the scan scratch failed: %s", cudaGetErrorString(e));
    g_scratch[dev] = static_cast<int64_t*>(p);
  }
  *out = g_scratch[dev];
  return FEA_OK;
}

// Exclusive scan of ITEMS values per thread across one block; returns the block total.
__device__ int64_t block_scan(int64_t v[ITEMS], int64_t* sh) {
  int64_t t = 0;
  for (int i = 0; i < ITEMS; ++i) {
    int64_t x = v[i];
    v[i] = t;
    t += x;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = t;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < THREADS / 32 ? sh[lane] : 0, si = s;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < THREADS / 32) sh[lane] = si - s;
    if (lane == THREADS / 32 - 1) sh[THREADS / 32] = si;
  }
  __syncthreads();
  const int64_t off = sh[w] + inc - t;
  for (int i = 0; i < ITEMS; ++i) v[i] += off;
  const int64_t total = sh[THREADS / 32];
  __syncthreads();
  return total;
}

__global__ void k_tile_totals(const int32_t* __restrict__ counts, int64_t n, int64_t* tiles) {
  __shared__ int64_t sh[THREADS / 32 + 1];
  int64_t v[ITEMS];
  const int64_t b = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  for (int i = 0; i < ITEMS; ++i) v[i] = b + i < n ? (int64_t)counts[b + i] : 0;
  const int64_t total = block_scan(v, sh);
  if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

// One block: exclusive scan of the tile totals in place.
__global__ void k_tile_offsets(int64_t* tiles, int64_t n_tiles) {
  __shared__ int64_t sh[THREADS / 32 + 1];
  int64_t carry = 0;
  for (int64_t base = 0; base < n_tiles; base += TILE) {
    int64_t v[ITEMS];
    for (int i = 0; i < ITEMS; ++i) {
      const int64_t j = base + (int64_t)threadIdx.x * ITEMS + i;
      v[i] = j < n_tiles ? tiles[j] : 0;
    }
    const int64_t total = block_scan(v, sh);
    for (int i = 0; i < ITEMS; ++i) {
      const int64_t j = base + (int64_t)threadIdx.x * ITEMS + i;
      if (j < n_tiles) tiles[j] = v[i] + carry;
    }
    carry += total;
    __syncthreads();
  }
}

__global__ void k_rowptr(const int32_t* __restrict__ counts, int64_t n, const int64_t* tiles, int64_t* rowptr) {
  __shared__ int64_t sh[THREADS / 32 + 1];
  int64_t v[ITEMS];
  const int64_t b = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  for (int i = 0; i < ITEMS; ++i) v[i] = b + i < n ? (int64_t)counts[b + i] : 0;
  const int64_t total = block_scan(v, sh);
  const int64_t off = tiles[blockIdx.x];
  for (int i = 0; i < ITEMS; ++i)
    if (b + i < n) rowptr[b + i] = v[i] + off;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) rowptr[n] = off + total;
}

__global__ void k_zero_first(int64_t* rowptr) { rowptr[0] = 0; }

}  // namespace noalloc
}  // namespace fea

using namespace fea;

extern "C" fea_status fea_csr_rowptr_noalloc(const int32_t* counts, int64_t n, int64_t* rowptr, void* stream) {
  if (n < 0 || !rowptr || (n > 0 && !counts)) return fail(FEA_ERR_ARG, "fea_csr_rowptr_noalloc: bad argument");
  if (n > noalloc::MAX_ROWS)
    return fail(FEA_ERR_TOO_LARGE, "fea_csr_rowptr_noalloc: %lld rows exceed the fixed scratch (at most %lld rows)",
                (long long)n, (long long)noalloc::MAX_ROWS);
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    noalloc::k_zero_first<<<1, 1, 0, s>>>(rowptr);
    FEA_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return FEA_OK;
  }
  int64_t* tiles = nullptr;
  FEA_TRY(noalloc::scratch_address(&tiles));
  const unsigned n_tiles = (unsigned)((n + noalloc::TILE - 1) / noalloc::TILE);
  noalloc::k_tile_totals<<<n_tiles, noalloc::THREADS, 0, s>>>(counts, n, tiles);
  noalloc::k_tile_offsets<<<1, noalloc::THREADS, 0, s>>>(tiles, n_tiles);
  noalloc::k_rowptr<<<n_tiles, noalloc::THREADS, 0, s>>>(counts, n, tiles, rowptr);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(3);
  return FEA_OK;
}
