// fea_api.cu -- C ABI entry points, mesh upload and validation, CSR pattern
// build on the device (Sec. 4.2: CSR storage of the assembled matrix).
#include <cuda_runtime.h>

#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fea_internal.cuh"
#include "fea_plan.cuh"

namespace fea {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

fea_status fail(fea_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

fea_status status_to_error(uint32_t bits) {
  if (bits & ST_RANGE) return fail(FEA_ERR_RANGE, "connectivity holds a node id outside [0, n_node)");
  if (bits & ST_DUP) return fail(FEA_ERR_DUP_NODE, "an element lists the same node twice");
  if (bits & ST_INVERTED) return fail(FEA_ERR_INVERTED, "an element has det J <= 0 at a Gauss point or corner");
  if (bits & ST_ROW_TOO_LONG) return fail(FEA_ERR_TOO_LARGE, "a node touches too many elements (row candidate list over limit)");
  if (bits & ST_TIMEOUT) return fail(FEA_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (bits & ST_SCHEDULE) return fail(FEA_ERR_STATE, "row-owned schedule does not match the mesh");
  return FEA_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ small device helpers

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_ITEMS = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of SCAN_TILE int64 items held 8 per thread.
__device__ int64_t block_exclusive_scan(int64_t v[SCAN_ITEMS], int64_t* sh) {
  int64_t tsum = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t x = v[i];
    v[i] = tsum;
    tsum += x;
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = tsum;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < SCAN_THREADS / 32 ? sh[lane] : 0;
    int64_t si = s;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < SCAN_THREADS / 32) sh[lane] = si - s;
    if (lane == SCAN_THREADS / 32 - 1) sh[SCAN_THREADS / 32] = si;
  }
  __syncthreads();
  int64_t off = sh[w] + incl - tsum;
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] += off;
  int64_t total = sh[SCAN_THREADS / 32];
  __syncthreads();
  return total;
}

template <typename TIn>
__global__ void k_tile_sums(const TIn* in, int64_t n, int64_t* tile_sums) {
  __shared__ int64_t sh[SCAN_THREADS / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t v[SCAN_ITEMS];
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
    v[i] = idx < n ? (int64_t)in[idx] : 0;
  }
  int64_t total = block_exclusive_scan(v, sh);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Exclusive scan of the tile sums in one block (loops over chunks).
__global__ void k_scan_tile_sums(int64_t* sums, int64_t n) {
  __shared__ int64_t sh[SCAN_THREADS / 32 + 1];
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += SCAN_TILE) {
    int64_t v[SCAN_ITEMS];
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
      v[i] = idx < n ? sums[idx] : 0;
    }
    int64_t total = block_exclusive_scan(v, sh);
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
      if (idx < n) sums[idx] = v[i] + carry;
    }
    carry += total;
    __syncthreads();
  }
}

// out[i] = sum_{j<i} in[j] for i in [0, n], out has n+1 entries.
template <typename TIn>
__global__ void k_scan_apply(const TIn* in, int64_t n, const int64_t* tile_offsets, int64_t* out) {
  __shared__ int64_t sh[SCAN_THREADS / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t v[SCAN_ITEMS];
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
    v[i] = idx < n ? (int64_t)in[idx] : 0;
  }
  int64_t total = block_exclusive_scan(v, sh);
  int64_t off = tile_offsets[blockIdx.x];
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
    if (idx < n) out[idx] = v[i] + off;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

// Exclusive scan with total: out[0..n] (n+1 entries). Uses a temporary of ceil(n/TILE) int64.
template <typename TIn>
static fea_status exclusive_scan(const TIn* in, int64_t n, int64_t* out, cudaStream_t s) {
  int64_t tiles = std::max<int64_t>(1, (n + SCAN_TILE - 1) / SCAN_TILE);
  int64_t* sums = nullptr;
  FEA_CUDA_TRY(cudaMallocAsync(&sums, sizeof(int64_t) * tiles, s));
  k_tile_sums<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums);
  k_scan_tile_sums<<<1, SCAN_THREADS, 0, s>>>(sums, tiles);
  k_scan_apply<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums, out);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(sums, s);
  if (e != cudaSuccess) return fail(FEA_ERR_CUDA, "scan launch: %s", cudaGetErrorString(e));
  return FEA_OK;
}

// ------------------------------------------------------------------ mesh validation

template <int TYPE>
__global__ void k_validate(const double* __restrict__ coords, const int32_t* __restrict__ conn, int64_t n_node,
                           int64_t n_elem, uint32_t* status) {
  constexpr int NEN = Elem<TYPE>::NEN, NG = Elem<TYPE>::NG;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  const int32_t* ce = conn + e * NEN;
  int32_t ids[NEN];
  bool ok = true;
  for (int a = 0; a < NEN; ++a) {
    ids[a] = ce[a];
    if (ids[a] < 0 || ids[a] >= n_node) ok = false;
  }
  if (!ok) { atomicOr(status, ST_RANGE); return; }
  for (int a = 0; a < NEN; ++a)
    for (int b = a + 1; b < NEN; ++b)
      if (ids[a] == ids[b]) ok = false;
  if (!ok) { atomicOr(status, ST_DUP); return; }
  double x0[3];
  for (int i = 0; i < 3; ++i) x0[i] = coords[(int64_t)ids[0] * 3 + i];
  for (int p = 0; p < NG + n_corners<TYPE>(); ++p) {
    double xi[3], w;
    if (p < NG) gauss_point<TYPE>(p, xi, w);
    else corner_point<TYPE>(p - NG, xi);
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < NEN; ++a) {
      double N, dN[3];
      shape<TYPE>(a, xi, N, dN);
      for (int i = 0; i < 3; ++i) {
        double xa = coords[(int64_t)ids[a] * 3 + i] - x0[i];
        for (int j = 0; j < 3; ++j) J[i][j] += xa * dN[j];
      }
    }
    if (!(det3(J) > 0.0)) { atomicOr(status, ST_INVERTED); return; }
  }
}

// hi/lo float split of every coordinate, SoA.
__global__ void k_split_coords(const double* __restrict__ coords, int64_t n_node, float* xhi, float* xlo) {
  int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_node) return;
  for (int i = 0; i < 3; ++i) {
    double x = coords[n * 3 + i];
    float hi = (float)x;
    xhi[(int64_t)i * n_node + n] = hi;
    xlo[(int64_t)i * n_node + n] = (float)(x - (double)hi);
  }
}

// ------------------------------------------------------------------ pattern kernels

// Connectivity slots below 0 are the padding of a mesh of several element types.
__global__ void k_inc_count(const int32_t* __restrict__ conn, int64_t total, int32_t* cnt) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total && conn[t] >= 0) atomicAdd(&cnt[conn[t]], 1);
}

__global__ void k_inc_fill(const int32_t* __restrict__ conn, int64_t total, int nen, const int64_t* inc_ptr,
                           int32_t* cursor, int32_t* inc_elem) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int32_t n = conn[t];
  if (n < 0) return;
  int32_t k = atomicAdd(&cursor[n], 1);
  inc_elem[inc_ptr[n] + k] = (int32_t)(t / nen);
}

static constexpr int ROW_WARPS = 4;
static constexpr int ROW_CAP = 4096;  // candidate columns per row (incident elements x nen)

// Per-warp bitonic sort of n (power of two) ints in shared memory.
__device__ void warp_bitonic_sort(int32_t* s, int n) {
  int lane = threadIdx.x & 31;
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n; i += 32) {
        int ixj = i ^ j;
        if (ixj > i) {
          int32_t a = s[i], b = s[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) { s[i] = b; s[ixj] = a; }
        }
      }
      __syncwarp();
    }
  }
}

// One warp per row: gather the nodes of every incident element, sort, unique.
// mode 0 writes the unique count to rowcnt; mode 1 writes the columns (and sorts
// the incidence list of the row so later schedules are deterministic).
__global__ void __launch_bounds__(ROW_WARPS * 32)
k_rows(const int32_t* __restrict__ conn, int nen, const int64_t* __restrict__ inc_ptr, int32_t* inc_elem,
       int64_t n_node, int mode, int32_t* rowcnt, const int64_t* __restrict__ rowptr, int32_t* colind,
       uint32_t* status) {
  extern __shared__ int32_t sm_rows[];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* s = sm_rows + w * ROW_CAP;
  int64_t warps_total = (int64_t)gridDim.x * ROW_WARPS;
  for (int64_t r = (int64_t)blockIdx.x * ROW_WARPS + w; r < n_node; r += warps_total) {
    int64_t i0 = inc_ptr[r], i1 = inc_ptr[r + 1];
    int64_t cnt = (i1 - i0) * nen;
    if (cnt > ROW_CAP) {
      if (lane == 0) atomicOr(status, ST_ROW_TOO_LONG);
      continue;
    }
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    if (n2 < 2) n2 = 2;
    if (mode == 1) {
      // sort this row's incidence list (ascending element ids)
      int m = (int)(i1 - i0), m2 = 2;
      while (m2 < m) m2 <<= 1;
      for (int i = lane; i < m2; i += 32) s[i] = i < m ? inc_elem[i0 + i] : INT_MAX;
      __syncwarp();
      warp_bitonic_sort(s, m2);
      for (int i = lane; i < m; i += 32) inc_elem[i0 + i] = s[i];
      __syncwarp();
    }
    for (int i = lane; i < n2; i += 32) {
      int32_t v = INT_MAX;
      if (i < cnt) {
        int64_t t = i0 + i / nen;
        v = conn[(int64_t)inc_elem[t] * nen + (i % nen)];
        if (v < 0) v = INT_MAX;  // padding slot: sorts last, never a column
      }
      s[i] = v;
    }
    __syncwarp();
    warp_bitonic_sort(s, n2);
    // unique
    int64_t written = 0;
    for (int base = 0; base < cnt; base += 32) {
      int i = base + lane;
      bool first = i < cnt && s[i] != INT_MAX && (i == 0 || s[i] != s[i - 1]);
      unsigned m = __ballot_sync(0xffffffffu, first);
      if (mode == 1 && first) {
        int off = __popc(m & ((1u << lane) - 1u));
        colind[rowptr[r] + written + off] = s[i];
      }
      written += __popc(m);
    }
    if (mode == 0 && lane == 0) rowcnt[r] = (int32_t)written;
    __syncwarp();
  }
}

// Local index of node r in each of its incident elements (after the lists are sorted).
__global__ void k_inc_local(const int32_t* __restrict__ conn, int nen, const int64_t* __restrict__ inc_ptr,
                            const int32_t* __restrict__ inc_elem, int64_t n_node, uint8_t* __restrict__ inc_local) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_node; r += (int64_t)gridDim.x * blockDim.x)
    for (int64_t t = inc_ptr[r]; t < inc_ptr[r + 1]; ++t) {
      const int32_t* ce = conn + (int64_t)inc_elem[t] * nen;
      int a = 0;
      while (a < nen - 1 && ce[a] != r) ++a;
      inc_local[t] = (uint8_t)a;
    }
}

// Longest row: max of the row counts, into *out (zeroed by the caller).
__global__ void k_maxlen(const int32_t* __restrict__ rowcnt, int64_t n, int32_t* out) {
  int32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, rowcnt[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_posmap(const int32_t* __restrict__ conn, int64_t n_elem, int nen, const int64_t* __restrict__ rowptr,
                         const int32_t* __restrict__ colind, int32_t* pos) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = n_elem * nen * nen;
  if (t >= total) return;
  int64_t e = t / (nen * nen);
  int ab = (int)(t % (nen * nen));
  int a = ab / nen, b = ab % nen;
  int32_t r = conn[e * nen + a], c = conn[e * nen + b];
  int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (colind[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  pos[t] = (int32_t)lo;
}

static unsigned grid_for(int64_t n, int threads) { return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads); }

}  // namespace fea

using namespace fea;

// ------------------------------------------------------------------ C ABI helpers

static fea_status check_assemble_args(fea_mesh* m, const fea_pattern* p, const void* vel, const void* kd,
                                      const void* sr, const void* phi, double dt, int32_t n_eq,
                                      const fea_assemble_opts* o, const void* values, const void* rhs) {
  if (!m || !p) return fail(FEA_ERR_ARG, "mesh/pattern is null");
  if (p->mesh != m) return fail(FEA_ERR_STATE, "pattern was built for another mesh");
  if (n_eq <= 0) return fail(FEA_ERR_ARG, "n_eq must be > 0 (got %d)", n_eq);
  if (!(dt > 0.0)) return fail(FEA_ERR_ARG, "dt must be > 0");
  if (!vel || !kd || !sr || !phi || !values || !rhs) return fail(FEA_ERR_ARG, "a field or output pointer is null");
  if (o->precision != FEA_F64_PLAIN && o->precision != FEA_F32_FUSED) return fail(FEA_ERR_ARG, "unknown precision");
  if (o->terms & ~FEA_TERM_ALL) return fail(FEA_ERR_ARG, "unknown term bits");
  if (o->scatter < FEA_SCATTER_AUTO || o->scatter > FEA_SCATTER_GATHER) return fail(FEA_ERR_ARG, "unknown scatter");
  if (o->scatter == FEA_SCATTER_GATHER && o->precision != FEA_F32_FUSED)
    return fail(FEA_ERR_ARG, "the gather scatter is an FP32 path");
  if (o->cancel_check != 0 && o->cancel_check != 1) return fail(FEA_ERR_ARG, "cancel_check must be 0 or 1");
  if (o->cancel_check && o->accumulate) return fail(FEA_ERR_ARG, "cancel_check cannot be combined with accumulate");
  if (o->host_parts < 0) return fail(FEA_ERR_ARG, "host_parts must be >= 0");
  if (o->contraction < FEA_CONTRACT_AUTO || o->contraction > FEA_CONTRACT_TC_TF32X3)
    return fail(FEA_ERR_ARG, "unknown contraction");
  if (o->mapping < FEA_MAP_AUTO || o->mapping > FEA_MAP_TWO_THREADS_PER_ITEM) return fail(FEA_ERR_ARG, "unknown mapping");
  if (o->elems_per_cta < 0 || o->elems_per_cta > 256) return fail(FEA_ERR_ARG, "elems_per_cta must be in [0, 256]");
  if (m->mixed && (o->scatter == FEA_SCATTER_ROWOWNED || o->scatter == FEA_SCATTER_GATHER || o->cancel_check))
    return fail(FEA_ERR_ARG, "a mesh of several element types scatters with atomics (no row-owned, gather or "
                             "cancellation check)");
  return FEA_OK;
}

// The arguments restricted to one element block (the whole mesh for a single-type mesh).
template <typename T>
static void set_block(AsmArgs<T>& a, const fea_mesh::Block& b, const fea_pattern* p) {
  a.conn = b.conn;
  a.pos = p->pos + b.pos0;
  a.n_elem = b.n_elem;
}

template <typename T>
static AsmArgs<T> make_args(fea_mesh* m, const fea_pattern* p, const void* vel, const void* kd, const void* sr,
                            const void* phi, double dt, int32_t n_eq, const fea_assemble_opts* o, void* values,
                            void* rhs) {
  AsmArgs<T> a;
  a.conn = m->conn;
  a.coords = m->coords;
  a.xhi = m->xhi;
  a.xlo = m->xlo;
  a.pos = p->pos;
  a.rowptr = p->rowptr;
  a.colind = p->colind;
  a.vel = (const T*)vel;
  a.kd = (const T*)kd;
  a.sr = (const T*)sr;
  a.phi = (const T*)phi;
  a.values = (T*)values;
  a.rhs = (T*)rhs;
  a.em = nullptr;
  a.inc_ptr = p->inc_ptr;
  a.inc_elem = p->inc_elem;
  a.inc_local = p->inc_local;
  a.phi_eval = nullptr;
  a.resid = nullptr;
  a.n_node = m->n_node;
  a.n_elem = m->n_elem;
  a.nnz = p->nnz;
  a.n_eq = n_eq;
  a.eq0 = 0;
  a.eq_count = n_eq;
  a.terms = o->terms;
  a.dt = dt;
  a.kappa_threshold = o->kappa_threshold;
  a.status = m->status;
  a.elem_order = (!m->mixed && m->type == FEA_TET4) ? p->elem_order : nullptr;
  a.t4_rows = (!m->mixed && m->type == FEA_TET4) ? p->t4_rows : nullptr;
  a.contraction = o->contraction == FEA_CONTRACT_AUTO ? FEA_CONTRACT_CUDA : o->contraction;
  a.mapping = o->mapping == FEA_MAP_AUTO ? FEA_MAP_TYPE_KERNEL : o->mapping;
  a.batch = o->elems_per_cta;
  return a;
}



// ------------------------------------------------------------------ strategies and the autotuner

namespace {

// One complete choice of how an FP32 assembly runs (a fea_tuning without the bookkeeping).
struct Strategy {
  int scatter;      // fea_scatter, never AUTO here except before resolution
  int groups;       // equation groups of the row-owned scatter
  int mapping;      // fea_mapping (TYPE_KERNEL or WARP_PER_ELEMENT)
  int batch;        // elements_per_cta, 0 = the kernel's rule
  int contraction;  // fea_contraction (CUDA or a tensor-core variant)
};

Strategy from_tuning(const fea_tuning& t) { return Strategy{t.scatter, t.eq_groups, t.mapping, t.elems_per_cta, t.contraction}; }
fea_tuning to_tuning(const Strategy& s, int from_cache, float ms) {
  return fea_tuning{s.scatter, s.groups, s.mapping, s.batch, s.contraction, from_cache, ms};
}

// FP32 element-parallel launch over every element block: the batched Hex8 kernel for Hex8
// blocks (its node-major field scratch held by the plan of a single-type mesh, else by the
// pattern), the per-type kernels behind launch_generic_f32 for the others; with the
// warp-per-element mapping the generic kernel for every block.
fea_status elem_f32(fea_mesh* m, fea_pattern* p, const AsmArgs<float>& a0, cudaStream_t s) {
  for (const fea_mesh::Block& b : m->blocks) {
    if (b.n_elem == 0) continue;
    AsmArgs<float> a = a0;
    set_block(a, b, p);
    if (b.type == FEA_HEX8 && a.mapping != FEA_MAP_WARP_PER_ELEMENT) {
      if (p->plan) FEA_TRY(plan_elem(p->plan, a, s));
      else FEA_TRY(hex8_elem(p->hex8_fnode, p->hex8_fnode_bytes, a, s));
    } else if (b.type == FEA_TET4 && !m->mixed && a.eq_count == 1 && a.mapping != FEA_MAP_WARP_PER_ELEMENT &&
               p->t4_node) {  // one equation: node records read with three 16-byte loads per node
      a.t4_node = p->t4_node;
      FEA_TRY(tet4_node_records(a, p->t4_node, s));
      FEA_TRY(launch_generic_f32(a, b.type, s));
    } else {
      FEA_TRY(launch_generic_f32(a, b.type, s));
    }
  }
  return FEA_OK;
}

// The plain FP64 path over every element block: one launch per equation and block.
fea_status elem_f64(fea_mesh* m, const fea_pattern* p, const AsmArgs<double>& a0, int32_t n_eq, cudaStream_t s) {
  for (const fea_mesh::Block& b : m->blocks) {
    if (b.n_elem == 0) continue;
    AsmArgs<double> a = a0;
    set_block(a, b, p);
    for (int q = 0; q < n_eq; ++q) {  // geometry recomputed each time
      a.eq0 = q;
      a.eq_count = 1;
      FEA_TRY(launch_generic_f64(a, b.type, s));
    }
  }
  return FEA_OK;
}

bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Runs one assembly with a resolved strategy (FP64: always the plain per-equation path).
fea_status run_strategy(fea_mesh* m, fea_pattern* p, const void* vel, const void* kd, const void* sr, const void* phi,
                        double dt, int32_t n_eq, const fea_assemble_opts& o, void* values, void* rhs,
                        Strategy st) {
  cudaStream_t s = m->stream;
  size_t es = o.precision == FEA_F64_PLAIN ? sizeof(double) : sizeof(float);
  const bool f32 = o.precision == FEA_F32_FUSED;
  bool rowowned = false;
  if (f32 && (st.scatter == FEA_SCATTER_ROWOWNED || st.scatter == FEA_SCATTER_AUTO)) {
    FEA_TRY(plan_prepare(p->plan, plan_group_size(n_eq, st.groups), st.batch, &rowowned));
    if (st.scatter == FEA_SCATTER_ROWOWNED && !rowowned)
      return fail(FEA_ERR_ARG, "row-owned scatter is not available for this mesh type, precision or equation count");
  }
  const bool gather = f32 && st.scatter == FEA_SCATTER_GATHER;
  if (gather && m->n_elem > 0) {
    const size_t need = gather_scratch_bytes(m->n_elem, m->nen, n_eq);
    if (p->em_bytes < need) {
      if (stream_capturing(s)) return fail(FEA_ERR_STATE, "gather scratch must be allocated before stream capture");
      FEA_CUDA_TRY(cudaStreamSynchronize(s));  // the old scratch may still be in use on the stream
      cudaFree(p->em);
      p->em = nullptr;
      p->em_bytes = 0;
      if (cudaMalloc(&p->em, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(FEA_ERR_OOM, "gather scatter: %zu bytes of element-matrix scratch", need);
      }
      p->em_bytes = need;
    }
  }
  if (!o.accumulate && !rowowned && !(gather && m->n_elem > 0)) {
    FEA_CUDA_TRY(cudaMemsetAsync(values, 0, es * (size_t)n_eq * (size_t)p->nnz, s));
    FEA_CUDA_TRY(cudaMemsetAsync(rhs, 0, es * (size_t)n_eq * (size_t)m->n_node, s));
  }
  if (o.event_begin) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o.event_begin, s));
  if (m->n_elem > 0) {
    if (!f32) {
      AsmArgs<double> a = make_args<double>(m, p, vel, kd, sr, phi, dt, n_eq, &o, values, rhs);
      FEA_TRY(elem_f64(m, p, a, n_eq, s));
    } else {
      AsmArgs<float> a = make_args<float>(m, p, vel, kd, sr, phi, dt, n_eq, &o, values, rhs);
      a.mapping = st.mapping;
      a.batch = st.batch;
      a.contraction = st.contraction;
      if (rowowned) {
        FEA_TRY(plan_assemble(p->plan, a, o.accumulate, st.groups, s));
      } else if (gather) {
        a.em = (float*)p->em;
        FEA_TRY(elem_f32(m, p, a, s));
        FEA_TRY(launch_gather_f32(a, m->type, p->maxcol, o.accumulate != 0, s));
      } else {
        FEA_TRY(elem_f32(m, p, a, s));
      }
    }
  }
  if (o.event_end) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o.event_end, s));
  return FEA_OK;
}

// The strategy an explicit (non-AUTO) opts asks for.
Strategy explicit_strategy(const fea_assemble_opts& o) {
  return Strategy{o.scatter, std::max(1, o.eq_groups), o.mapping == FEA_MAP_AUTO ? (int)FEA_MAP_TYPE_KERNEL : o.mapping,
                  o.elems_per_cta, o.contraction == FEA_CONTRACT_AUTO ? (int)FEA_CONTRACT_CUDA : o.contraction};
}

const char* type_name(const fea_mesh* m) {
  if (m->mixed) return "mixed";
  switch (m->type) {
    case FEA_TET4: return "tet4";
    case FEA_HEX8: return "hex8";
    case FEA_HEX27: return "hex27";
    case FEA_PEN6: return "pen6";
    case FEA_PYR5: return "pyr5";
  }
  return "unknown";
}

// The candidates of FEA_SCATTER_AUTO, in the order they are timed.  Row-owned schedules with
// batch sizes other than the kernel's rule are listed for every group count here; the tuner
// times them for the best group count only.
std::vector<Strategy> candidates(fea_mesh* m, fea_pattern* p, int32_t n_eq, int terms) {
  std::vector<Strategy> c;
  const int T = FEA_MAP_TYPE_KERNEL, W = FEA_MAP_WARP_PER_ELEMENT, CU = FEA_CONTRACT_CUDA;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const bool gather_fits = !m->mixed && gather_scratch_bytes(m->n_elem, m->nen, n_eq) <= free_b / 2;
  // atomics into DRAM run at a few G/s, and the warp-per-element kernel is several times slower
  // than the type kernels: time them only where a trial stays short
  const double work = (double)m->n_elem * m->nen * m->nen * n_eq;
  const bool short_trial = work < 2e9;
  if (m->mixed) {
    c.push_back(Strategy{FEA_SCATTER_ATOMIC, 1, T, 0, CU});
    if (short_trial) c.push_back(Strategy{FEA_SCATTER_ATOMIC, 1, W, 0, CU});
    return c;
  }
  if (p->plan) {  // Hex8: row-owned schedules per group count, then batch sizes
    int last = -1;
    for (int g = 1; g <= 4 && g <= n_eq; ++g) {
      const int size = plan_group_size(n_eq, g);
      if (size == last) continue;
      last = size;
      for (int mp : {T, (int)FEA_MAP_TWO_THREADS_PER_ITEM}) {
        if (mp != T && terms != FEA_TERM_ALL) continue;  // the two-thread kernel forms the full operator
        c.push_back(Strategy{FEA_SCATTER_ROWOWNED, g, mp, 0, CU});
        for (int be : {16, 32}) c.push_back(Strategy{FEA_SCATTER_ROWOWNED, g, mp, be, CU});
      }
    }
  }
  std::vector<int> batches{0};
  if (m->type == FEA_HEX8) batches = {0, 32};
  if (m->type == FEA_TET4) batches = {0, 128};
  if (m->type == FEA_PEN6 || m->type == FEA_PYR5) batches = {0, 64};
  std::vector<int> contractions{CU};
  if (m->type == FEA_HEX27 && terms == FEA_TERM_ALL && n_eq <= 12) contractions.push_back(FEA_CONTRACT_TC_TF32X3);
  for (int sc : {(int)FEA_SCATTER_GATHER, (int)FEA_SCATTER_ATOMIC}) {
    if (sc == FEA_SCATTER_GATHER && !gather_fits) continue;
    if (sc == FEA_SCATTER_ATOMIC && !short_trial && !c.empty()) continue;
    for (int be : batches)
      for (int ct : contractions) c.push_back(Strategy{sc, 1, T, be, ct});
    if (short_trial) c.push_back(Strategy{sc, 1, W, 0, CU});
  }
  if (c.empty()) c.push_back(Strategy{FEA_SCATTER_ATOMIC, 1, T, 0, CU});
  return c;
}

// ---- the tuning cache file

std::string cache_path() {
  const char* e = getenv("FEA_TUNE_CACHE");
  if (e) return (strcmp(e, "off") == 0 || !*e) ? std::string() : std::string(e);
  const char* x = getenv("XDG_CACHE_HOME");
  if (x && *x) return std::string(x) + "/fea_gb300/tuning.json";
  const char* h = getenv("HOME");
  if (h && *h) return std::string(h) + "/.cache/fea_gb300/tuning.json";
  return std::string();
}

std::string cache_key(fea_mesh* m, int32_t n_eq, int terms) {
  cudaDeviceProp prop;
  std::string gpu = cudaGetDeviceProperties(&prop, m->device) == cudaSuccess ? prop.name : "gpu";
  for (char& ch : gpu)
    if (ch == '"' || ch == '\\') ch = '_';
  auto log2r = [](int64_t n) { return n <= 1 ? 0 : (int)std::lround(std::log2((double)n)); };
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%s|q%d|t%d|f32|E2^%d|N2^%d", gpu.c_str(), type_name(m), n_eq, terms,
           log2r(m->n_elem), log2r(m->n_node));
  return buf;
}

// The file is one JSON object of "key": {"scatter": s, "eq_groups": g, "mapping": m,
// "elems_per_cta": b, "contraction": c, "ms": t} entries, one per line (as written below).
std::map<std::string, fea_tuning> cache_read(const std::string& path) {
  std::map<std::string, fea_tuning> out;
  FILE* f = path.empty() ? nullptr : fopen(path.c_str(), "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    const char* q0 = strchr(line, '"');
    const char* q1 = q0 ? strchr(q0 + 1, '"') : nullptr;
    if (!q1) continue;
    fea_tuning t{};
    int sc, g, mp, be, ct;
    float ms;
    if (sscanf(q1 + 1, " : {\"scatter\": %d, \"eq_groups\": %d, \"mapping\": %d, \"elems_per_cta\": %d, "
                       "\"contraction\": %d, \"ms\": %f}", &sc, &g, &mp, &be, &ct, &ms) != 6)
      continue;
    t.scatter = sc;
    t.eq_groups = g;
    t.mapping = mp;
    t.elems_per_cta = be;
    t.contraction = ct;
    t.ms = ms;
    out[std::string(q0 + 1, q1)] = t;
  }
  fclose(f);
  return out;
}

void cache_write(const std::string& path, const std::string& key, const fea_tuning& t) {
  if (path.empty()) return;
  std::map<std::string, fea_tuning> all = cache_read(path);
  all[key] = t;
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) {  // create the directories (mkdir -p), ignoring failures
    for (size_t i = 1; i <= slash; ++i)
      if (path[i] == '/' || i == slash) {
        const std::string d = path.substr(0, i == slash ? slash : i);
        if (!d.empty()) mkdir(d.c_str(), 0755);
      }
  }
  const std::string tmp = path + "." + std::to_string((long long)getpid()) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : all) {
    const fea_tuning& v = kv.second;
    fprintf(f, " \"%s\": {\"scatter\": %d, \"eq_groups\": %d, \"mapping\": %d, \"elems_per_cta\": %d, "
               "\"contraction\": %d, \"ms\": %.4f}%s\n", kv.first.c_str(), v.scatter, v.eq_groups, v.mapping,
            v.elems_per_cta, v.contraction, v.ms, ++i < all.size() ? "," : "");
  }
  fprintf(f, "}\n");
  const bool ok = fclose(f) == 0;
  if (ok) rename(tmp.c_str(), path.c_str());
  else remove(tmp.c_str());
}

// Whether a cached strategy still applies to this pattern (the row-owned schedule builds).
bool strategy_valid(fea_mesh* m, fea_pattern* p, int32_t n_eq, int terms, const Strategy& st) {
  for (const Strategy& c : candidates(m, p, n_eq, terms))
    if (c.scatter == st.scatter && c.groups == st.groups && c.mapping == st.mapping && c.batch == st.batch &&
        c.contraction == st.contraction) {
      if (st.scatter != FEA_SCATTER_ROWOWNED) return true;
      bool ok = false;
      return plan_prepare(p->plan, plan_group_size(n_eq, st.groups), st.batch, &ok) == FEA_OK && ok;
    }
  return false;
}

// Resolves FEA_SCATTER_AUTO for an FP32 call.  The first call for a pattern, equation count
// and term mask takes the choice from the tuning cache file, or else times the candidates on
// the caller's own inputs (each result overwrites values and rhs, so the outputs end up
// assembled whichever ran last), keeps the fastest and records it in the file.
fea_status choose_strategy(fea_mesh* m, fea_pattern* p, const void* vel, const void* kd, const void* sr,
                           const void* phi, double dt, int32_t n_eq, const fea_assemble_opts& o, void* values,
                           void* rhs, Strategy* out) {
  const std::pair<int, int> tkey(n_eq, o.terms);
  auto it = p->tuned.find(tkey);
  if (it != p->tuned.end()) {
    *out = from_tuning(it->second);
    return FEA_OK;
  }
  bool ro1 = false;
  FEA_TRY(plan_prepare(p->plan, n_eq, 0, &ro1));
  const Strategy fallback{ro1 ? FEA_SCATTER_ROWOWNED : FEA_SCATTER_ATOMIC, 1, FEA_MAP_TYPE_KERNEL, 0, FEA_CONTRACT_CUDA};
  if (o.accumulate || m->n_elem == 0 || stream_capturing(m->stream)) {  // cannot run trials
    *out = fallback;
    return FEA_OK;
  }
  const std::string path = cache_path(), key = cache_key(m, n_eq, o.terms);
  {
    const std::map<std::string, fea_tuning> cached = cache_read(path);
    auto ci = cached.find(key);
    if (ci != cached.end() && strategy_valid(m, p, n_eq, o.terms, from_tuning(ci->second))) {
      fea_tuning t = ci->second;
      t.from_cache = 1;
      p->tuned[tkey] = t;
      *out = from_tuning(t);
      return FEA_OK;
    }
  }
  const std::vector<Strategy> all = candidates(m, p, n_eq, o.terms);
  fea_assemble_opts oq = o;
  oq.event_begin = oq.event_end = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FEA_CUDA_TRY(cudaEventCreate(&e0));
  FEA_CUDA_TRY(cudaEventCreate(&e1));
  Strategy best = fallback;
  float best_ms = 0.f;
  fea_status status = FEA_OK;
  auto time_one = [&](const Strategy& c) -> fea_status {
    if (c.scatter == FEA_SCATTER_ROWOWNED) {
      bool ok = false;
      FEA_TRY(plan_prepare(p->plan, plan_group_size(n_eq, c.groups), c.batch, &ok));
      if (!ok) return FEA_OK;  // no schedule for this group size or batch: not a candidate
    }
    float ms = 0.f;
    fea_status s1 = run_strategy(m, p, vel, kd, sr, phi, dt, n_eq, oq, values, rhs, c);  // warm-up
    if (s1 == FEA_OK) s1 = fea_sync(m);
    if (s1 == FEA_OK && cudaEventRecord(e0, m->stream) != cudaSuccess) s1 = FEA_ERR_CUDA;
    if (s1 == FEA_OK) s1 = run_strategy(m, p, vel, kd, sr, phi, dt, n_eq, oq, values, rhs, c);
    if (s1 == FEA_OK && cudaEventRecord(e1, m->stream) != cudaSuccess) s1 = FEA_ERR_CUDA;
    if (s1 == FEA_OK) s1 = fea_sync(m);
    if (s1 == FEA_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s1 = FEA_ERR_CUDA;
    if (s1 == FEA_ERR_OOM || s1 == FEA_ERR_TOO_LARGE) return FEA_OK;  // a candidate that does not fit is skipped
    if (s1 != FEA_OK) return s1;
    if (best_ms == 0.f || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
    return FEA_OK;
  };
  // stage 1: every candidate with the kernels' own batch rule (and every non-row-owned one)
  for (const Strategy& c : all) {
    if (c.scatter == FEA_SCATTER_ROWOWNED && c.batch != 0) continue;
    if ((status = time_one(c)) != FEA_OK) break;
  }
  // stage 2: the row-owned batch sizes, for the best group count and mapping only
  if (status == FEA_OK && best.scatter == FEA_SCATTER_ROWOWNED) {
    const int g = best.groups, mp = best.mapping;
    for (const Strategy& c : all)
      if (c.scatter == FEA_SCATTER_ROWOWNED && c.batch != 0 && c.groups == g && c.mapping == mp)
        if ((status = time_one(c)) != FEA_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != FEA_OK) return status;
  const fea_tuning t = to_tuning(best, 0, best_ms);
  p->tuned[tkey] = t;
  cache_write(path, key, t);
  // keep the resources of the winners (this call's and those tuned before) only
  std::vector<int> keep;
  bool any_gather = false;
  for (const auto& kv : p->tuned) {
    if (kv.second.scatter == FEA_SCATTER_ROWOWNED)
      keep.push_back(plan_key(plan_group_size(kv.first.first, kv.second.eq_groups), kv.second.elems_per_cta));
    any_gather |= kv.second.scatter == FEA_SCATTER_GATHER;
  }
  keep.push_back(plan_key(n_eq, 0));  // the fallback schedule (stream capture, accumulate)
  plan_trim(p->plan, keep);
  if (!any_gather) {
    cudaFree(p->em);
    p->em = nullptr;
    p->em_bytes = 0;
  }
  *out = best;
  return FEA_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

const char* fea_last_error(void) { return g_last_error.c_str(); }
int32_t fea_version(void) { return 10000; }
int64_t fea_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

fea_status fea_default_opts(fea_assemble_opts* o) {
  if (!o) return fail(FEA_ERR_ARG, "opts is null");
  memset(o, 0, sizeof *o);
  o->precision = FEA_F32_FUSED;
  o->terms = FEA_TERM_ALL;
  o->scatter = FEA_SCATTER_AUTO;
  o->accumulate = 0;
  o->kappa_threshold = 1e3;
  return FEA_OK;
}

fea_status fea_pack_plan(const int64_t* count_by_type, int32_t n_types, int32_t vector_size, int64_t* packs,
                         int64_t* pads) {
  if (!count_by_type || !packs || !pads || n_types < 0 || vector_size <= 0)
    return fail(FEA_ERR_ARG, "fea_pack_plan: bad argument");
  for (int t = 0; t < n_types; ++t) {
    if (count_by_type[t] < 0) return fail(FEA_ERR_ARG, "fea_pack_plan: negative count");
    packs[t] = (count_by_type[t] + vector_size - 1) / vector_size;
    pads[t] = packs[t] * vector_size - count_by_type[t];
  }
  return FEA_OK;
}

}  // extern "C"
static int nen_of(fea_elem_t t) {
  return t == FEA_TET4 ? 4 : t == FEA_HEX8 ? 8 : t == FEA_HEX27 ? 27 : t == FEA_PEN6 ? 6 : t == FEA_PYR5 ? 5 : 0;
}

static void launch_validate(fea_elem_t type, const double* coords, const int32_t* conn, int64_t n_node,
                            int64_t n_elem, uint32_t* status, cudaStream_t s) {
  if (n_elem <= 0) return;
  unsigned g = grid_for(n_elem, 128);
  switch (type) {
    case FEA_TET4: k_validate<FEA_TET4><<<g, 128, 0, s>>>(coords, conn, n_node, n_elem, status); break;
    case FEA_HEX8: k_validate<FEA_HEX8><<<g, 128, 0, s>>>(coords, conn, n_node, n_elem, status); break;
    case FEA_HEX27: k_validate<FEA_HEX27><<<g, 128, 0, s>>>(coords, conn, n_node, n_elem, status); break;
    case FEA_PEN6: k_validate<FEA_PEN6><<<g, 128, 0, s>>>(coords, conn, n_node, n_elem, status); break;
    case FEA_PYR5: k_validate<FEA_PYR5><<<g, 128, 0, s>>>(coords, conn, n_node, n_elem, status); break;
  }
}

// Block b's connectivity rows [n][nen_b] into the padded array [n][nen_max] (-1 fills).
__global__ void k_pad_conn(const int32_t* __restrict__ conn, int64_t n, int nen, int nen_max, int32_t* out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nen_max) return;
  int64_t e = t / nen_max;
  int a = (int)(t - e * nen_max);
  out[t] = a < nen ? conn[e * nen + a] : -1;
}

extern "C" {
fea_status fea_mesh_destroy(fea_mesh* m) {
  if (!m) return FEA_OK;
  cudaFree(m->coords);
  cudaFree(m->xhi);
  cudaFree(m->xlo);
  cudaFree(m->conn);
  cudaFree(m->conn_blocks);
  cudaFree(m->status);
  if (m->copy_ready) {
    for (int i = 0; i < fea_mesh::N_COPY; ++i) cudaStreamDestroy(m->copy_stream[i]);
    for (int i = 0; i <= fea_mesh::N_COPY; ++i) cudaEventDestroy(m->copy_event[i]);
    for (int i = 0; i < fea_mesh::N_IN; ++i) cudaStreamDestroy(m->in_stream[i]);
    for (cudaEvent_t e : m->part_events) cudaEventDestroy(e);
  }
  delete m;
  return FEA_OK;
}

fea_status fea_mesh_set_stream(fea_mesh* m, void* stream) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is null");
  m->stream = (cudaStream_t)stream;
  return FEA_OK;
}

fea_status fea_sync(fea_mesh* m) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is null");
  FEA_CUDA_TRY(cudaStreamSynchronize(m->stream));
  uint32_t bits = 0;
  FEA_CUDA_TRY(cudaMemcpy(&bits, m->status, sizeof bits, cudaMemcpyDeviceToHost));
  return status_to_error(bits);
}

fea_status fea_mesh_create(const double* coords, int64_t n_node, const int32_t* conn, int64_t n_elem, fea_elem_t type,
                           void* stream, fea_mesh** out) {
  if (!out) return fail(FEA_ERR_ARG, "out is null");
  *out = nullptr;
  int nen = nen_of(type);
  if (!nen) return fail(FEA_ERR_ARG, "unknown element type %d", (int)type);
  if (n_node <= 0 || n_elem < 0) return fail(FEA_ERR_ARG, "n_node must be > 0 and n_elem >= 0");
  if (!coords || (n_elem > 0 && !conn)) return fail(FEA_ERR_ARG, "coords/conn is null");
  if (n_node >= INT32_MAX) return fail(FEA_ERR_TOO_LARGE, "n_node %lld exceeds int32 ids", (long long)n_node);
  if (n_elem > (int64_t)INT32_MAX / (nen * nen))
    return fail(FEA_ERR_TOO_LARGE, "n_elem %lld too large for int32 position-map indexing", (long long)n_elem);
  fea_mesh* m = new (std::nothrow) fea_mesh();
  if (!m) return fail(FEA_ERR_OOM, "host allocation failed");
  m->type = type;
  m->nen = nen;
  m->n_node = n_node;
  m->n_elem = n_elem;
  m->stream = (cudaStream_t)stream;
  cudaGetDevice(&m->device);
  cudaStream_t s = m->stream;
  auto cleanup = [&](fea_status st) { fea_mesh_destroy(m); return st; };
  size_t cb = sizeof(double) * 3 * n_node, eb = sizeof(int32_t) * nen * std::max<int64_t>(n_elem, 1);
  if (cudaMalloc(&m->coords, cb) != cudaSuccess || cudaMalloc(&m->xhi, sizeof(float) * 3 * n_node) != cudaSuccess ||
      cudaMalloc(&m->xlo, sizeof(float) * 3 * n_node) != cudaSuccess || cudaMalloc(&m->conn, eb) != cudaSuccess ||
      cudaMalloc(&m->status, sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(FEA_ERR_OOM, "device allocation of the mesh failed"));
  }
  cudaMemcpyKind kc = is_device_ptr(coords) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(m->coords, coords, cb, kc, s) != cudaSuccess) return cleanup(fail(FEA_ERR_CUDA, "coords copy failed"));
  if (n_elem > 0) {
    cudaMemcpyKind ke = is_device_ptr(conn) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(m->conn, conn, sizeof(int32_t) * nen * n_elem, ke, s) != cudaSuccess)
      return cleanup(fail(FEA_ERR_CUDA, "conn copy failed"));
  }
  cudaMemsetAsync(m->status, 0, sizeof(uint32_t), s);
  k_split_coords<<<grid_for(n_node, 256), 256, 0, s>>>(m->coords, n_node, m->xhi, m->xlo);
  launch_validate(type, m->coords, m->conn, n_node, n_elem, m->status, s);
  m->blocks.push_back(fea_mesh::Block{type, nen, 0, n_elem, m->conn, 0});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(fail(FEA_ERR_CUDA, "validation launch: %s", cudaGetErrorString(e)));
  fea_status st = fea_sync(m);
  if (st != FEA_OK) return cleanup(st);
  *out = m;
  return FEA_OK;
}

fea_status fea_mesh_create_mixed(const double* coords, int64_t n_node, int32_t n_blocks, const fea_elem_t* types,
                                 const int32_t* const* conns, const int64_t* n_elems, void* stream, fea_mesh** out) {
  if (!out) return fail(FEA_ERR_ARG, "out is null");
  *out = nullptr;
  if (n_blocks <= 0 || !types || !conns || !n_elems) return fail(FEA_ERR_ARG, "n_blocks must be > 0, arrays non-null");
  if (n_blocks == 1) return fea_mesh_create(coords, n_node, conns[0], n_elems[0], types[0], stream, out);
  if (n_node <= 0 || !coords) return fail(FEA_ERR_ARG, "n_node must be > 0 and coords non-null");
  if (n_node >= INT32_MAX) return fail(FEA_ERR_TOO_LARGE, "n_node %lld exceeds int32 ids", (long long)n_node);
  int nen_max = 0;
  int64_t E = 0, conn_total = 0;
  for (int b = 0; b < n_blocks; ++b) {
    const int nen = nen_of(types[b]);
    if (!nen) return fail(FEA_ERR_ARG, "block %d: unknown element type %d", b, (int)types[b]);
    if (n_elems[b] < 0 || (n_elems[b] > 0 && !conns[b])) return fail(FEA_ERR_ARG, "block %d: bad size or null conn", b);
    if (n_elems[b] > (int64_t)INT32_MAX / (nen * nen))
      return fail(FEA_ERR_TOO_LARGE, "block %d: too many elements for int32 position-map indexing", b);
    nen_max = std::max(nen_max, nen);
    E += n_elems[b];
    conn_total += n_elems[b] * nen;
  }
  if (E > (int64_t)INT32_MAX / nen_max) return fail(FEA_ERR_TOO_LARGE, "too many elements for int32 element ids");
  fea_mesh* m = new (std::nothrow) fea_mesh();
  if (!m) return fail(FEA_ERR_OOM, "host allocation failed");
  m->type = types[0];
  m->nen = nen_max;
  m->n_node = n_node;
  m->n_elem = E;
  m->mixed = true;
  m->stream = (cudaStream_t)stream;
  cudaGetDevice(&m->device);
  cudaStream_t s = m->stream;
  auto cleanup = [&](fea_status st) { fea_mesh_destroy(m); return st; };
  size_t cb = sizeof(double) * 3 * n_node;
  if (cudaMalloc(&m->coords, cb) != cudaSuccess || cudaMalloc(&m->xhi, sizeof(float) * 3 * n_node) != cudaSuccess ||
      cudaMalloc(&m->xlo, sizeof(float) * 3 * n_node) != cudaSuccess ||
      cudaMalloc(&m->conn, sizeof(int32_t) * std::max<int64_t>(E * nen_max, 1)) != cudaSuccess ||
      cudaMalloc(&m->conn_blocks, sizeof(int32_t) * std::max<int64_t>(conn_total, 1)) != cudaSuccess ||
      cudaMalloc(&m->status, sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(FEA_ERR_OOM, "device allocation of the mesh failed"));
  }
  cudaMemcpyKind kc = is_device_ptr(coords) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(m->coords, coords, cb, kc, s) != cudaSuccess) return cleanup(fail(FEA_ERR_CUDA, "coords copy failed"));
  cudaMemsetAsync(m->status, 0, sizeof(uint32_t), s);
  k_split_coords<<<grid_for(n_node, 256), 256, 0, s>>>(m->coords, n_node, m->xhi, m->xlo);
  int64_t e0 = 0, c0 = 0, pos0 = 0;
  for (int b = 0; b < n_blocks; ++b) {
    const int nen = nen_of(types[b]);
    const int64_t n = n_elems[b];
    int32_t* cdst = m->conn_blocks + c0;
    if (n > 0) {
      cudaMemcpyKind ke = is_device_ptr(conns[b]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
      if (cudaMemcpyAsync(cdst, conns[b], sizeof(int32_t) * nen * n, ke, s) != cudaSuccess)
        return cleanup(fail(FEA_ERR_CUDA, "block %d: conn copy failed", b));
      k_pad_conn<<<grid_for(n * nen_max, 256), 256, 0, s>>>(cdst, n, nen, nen_max, m->conn + e0 * nen_max);
      launch_validate(types[b], m->coords, cdst, n_node, n, m->status, s);
    }
    m->blocks.push_back(fea_mesh::Block{types[b], nen, e0, n, cdst, pos0});
    e0 += n;
    c0 += n * nen;
    pos0 += n * nen * nen;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(fail(FEA_ERR_CUDA, "mesh setup launch: %s", cudaGetErrorString(e)));
  fea_status st = fea_sync(m);
  if (st != FEA_OK) return cleanup(st);
  *out = m;
  return FEA_OK;
}

fea_status fea_pattern_destroy(fea_pattern* p) {
  if (!p) return FEA_OK;
  cudaFree(p->rowptr);
  cudaFree(p->colind);
  cudaFree(p->pos);
  cudaFree(p->inc_ptr);
  cudaFree(p->inc_elem);
  cudaFree(p->inc_local);
  cudaFree(p->ws);
  cudaFree(p->em);
  cudaFree(p->diag);
  cudaFree(p->pcg_ws);
  cudaFree(p->lumped[0]);
  cudaFree(p->lumped[1]);
  cudaFree(p->rk_ws);
  cudaFree(p->elem_order);
  cudaFree(p->t4_rows);
  cudaFree(p->t4_node);
  cudaFree(p->hex8_fnode);
  for (auto& kv : p->cancel) {
    cudaFree(kv.second.rows);
    cudaFree(kv.second.count);
  }
  cudaFree(p->cancel_flags);
  plan_destroy(p->plan);
  delete p;
  return FEA_OK;
}

fea_status fea_pattern_get(const fea_pattern* p, const int64_t** rowptr, const int32_t** colind, const int32_t** pos,
                           int64_t* nnz) {
  if (!p) return fail(FEA_ERR_ARG, "pattern is null");
  if (rowptr) *rowptr = p->rowptr;
  if (colind) *colind = p->colind;
  if (pos) *pos = p->pos;
  if (nnz) *nnz = p->nnz;
  return FEA_OK;
}

static int64_t pos_total(const fea_mesh* m) {
  int64_t t = 0;
  for (const fea_mesh::Block& b : m->blocks) t += b.n_elem * b.nen * b.nen;
  return t;
}

fea_status fea_pattern_build(fea_mesh* m, fea_pattern** out) {
  if (!m || !out) return fail(FEA_ERR_ARG, "mesh/out is null");
  *out = nullptr;
  fea_pattern* p = new (std::nothrow) fea_pattern();
  if (!p) return fail(FEA_ERR_OOM, "host allocation failed");
  p->mesh = m;
  cudaStream_t s = m->stream;
  auto cleanup = [&](fea_status st) { fea_pattern_destroy(p); return st; };
  int64_t N = m->n_node, E = m->n_elem;
  int nen = m->nen;
  int64_t tot = E * nen;
  int32_t *cnt = nullptr, *rowcnt = nullptr;
  if (cudaMalloc(&p->inc_ptr, sizeof(int64_t) * (N + 1)) != cudaSuccess ||
      cudaMalloc(&p->inc_elem, sizeof(int32_t) * std::max<int64_t>(tot, 1)) != cudaSuccess ||
      cudaMalloc(&p->rowptr, sizeof(int64_t) * (N + 1)) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(int32_t) * N) != cudaSuccess || cudaMalloc(&rowcnt, sizeof(int32_t) * N) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(cnt);
    cudaFree(rowcnt);
    return cleanup(fail(FEA_ERR_OOM, "device allocation of the pattern failed"));
  }
  auto done = [&](fea_status st) { cudaFree(cnt); cudaFree(rowcnt); return st == FEA_OK ? st : cleanup(st); };
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s);
  cudaMemsetAsync(m->status, 0, sizeof(uint32_t), s);
  if (tot > 0) k_inc_count<<<grid_for(tot, 256), 256, 0, s>>>(m->conn, tot, cnt);
  fea_status st = exclusive_scan(cnt, N, p->inc_ptr, s);
  if (st != FEA_OK) return done(st);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s);
  if (tot > 0) k_inc_fill<<<grid_for(tot, 256), 256, 0, s>>>(m->conn, tot, nen, p->inc_ptr, cnt, p->inc_elem);
  size_t smem = sizeof(int32_t) * ROW_CAP * ROW_WARPS;
  cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  unsigned rg = (unsigned)std::min<int64_t>(grid_for(N, ROW_WARPS), 152 * 16);
  k_rows<<<rg, ROW_WARPS * 32, smem, s>>>(m->conn, nen, p->inc_ptr, p->inc_elem, N, 0, rowcnt, nullptr, nullptr,
                                          m->status);
  st = exclusive_scan(rowcnt, N, p->rowptr, s);
  if (st != FEA_OK) return done(st);
  int64_t nnz = 0;
  int32_t maxcol = 0;
  if (cudaMemcpyAsync(&nnz, p->rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return done(fail(FEA_ERR_CUDA, "nnz readback failed"));
  if (N > 0) {  // longest row, into cnt[0] (the incidence counters are no longer needed)
    cudaMemsetAsync(cnt, 0, sizeof(int32_t), s);
    k_maxlen<<<(unsigned)std::min<int64_t>(grid_for(N, 256), 152 * 8), 256, 0, s>>>(rowcnt, N, cnt);
    if (cudaMemcpyAsync(&maxcol, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return done(fail(FEA_ERR_CUDA, "row length readback failed"));
  }
  st = fea_sync(m);
  if (st != FEA_OK) return done(st);
  if (nnz >= (int64_t)INT32_MAX) return done(fail(FEA_ERR_TOO_LARGE, "nnz %lld >= 2^31", (long long)nnz));
  p->nnz = nnz;
  p->maxcol = maxcol;
  if (cudaMalloc(&p->colind, sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
      cudaMalloc(&p->pos, sizeof(int32_t) * std::max<int64_t>(pos_total(m), 1)) != cudaSuccess) {
    cudaGetLastError();
    return done(fail(FEA_ERR_OOM, "device allocation of colind/pos failed"));
  }
  k_rows<<<rg, ROW_WARPS * 32, smem, s>>>(m->conn, nen, p->inc_ptr, p->inc_elem, N, 1, nullptr, p->rowptr, p->colind,
                                          m->status);
  for (const fea_mesh::Block& b : m->blocks)  // each block's own [n][nen_b][nen_b] map
    if (b.n_elem > 0)
      k_posmap<<<grid_for(b.n_elem * b.nen * b.nen, 256), 256, 0, s>>>(b.conn, b.n_elem, b.nen, p->rowptr,
                                                                        p->colind, p->pos + b.pos0);
  if (cudaMalloc(&p->inc_local, std::max<int64_t>(tot, 1)) != cudaSuccess) {
    cudaGetLastError();
    return done(fail(FEA_ERR_OOM, "device allocation of the incidence index failed"));
  }
  if (N > 0)
    k_inc_local<<<(unsigned)std::min<int64_t>(grid_for(N, 256), 152 * 16), 256, 0, s>>>(m->conn, nen, p->inc_ptr,
                                                                                         p->inc_elem, N, p->inc_local);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return done(fail(FEA_ERR_CUDA, "pattern launch: %s", cudaGetErrorString(e)));
  st = fea_sync(m);
  if (st != FEA_OK) return done(st);
  if (!m->mixed && m->type == FEA_TET4) {  // the thread-per-item Tet4 kernel walks elements in this order
    st = element_order(m, &p->elem_order);
    if (st == FEA_OK) st = tet4_rows(m, p->elem_order, p->pos, &p->t4_rows);
    if (st == FEA_OK && cudaMalloc(&p->t4_node, 48 * (size_t)std::max<int64_t>(N, 1)) != cudaSuccess) {
      cudaGetLastError();
      p->t4_node = nullptr;  // optional: the kernel then reads the node arrays directly
    }
    if (st == FEA_OK) st = fea_sync(m);
    if (st != FEA_OK) return done(st);
  }
  st = plan_build(m, p, &p->plan);
  if (st != FEA_OK) return done(st);
  *out = p;
  return done(FEA_OK);
}

fea_status fea_assemble(fea_mesh* m, const fea_pattern* p, const void* vel, const void* kd, const void* sr,
                        const void* phi, double dt, int32_t n_eq, const fea_assemble_opts* opts, void* values,
                        void* rhs) {
  fea_assemble_opts o;
  if (opts) o = *opts;
  else fea_default_opts(&o);
  FEA_TRY(check_assemble_args(m, p, vel, kd, sr, phi, dt, n_eq, &o, values, rhs));
  fea_pattern* pw = const_cast<fea_pattern*>(p);  // schedules, scratch and the tuning cache belong to the pattern
  Strategy st = explicit_strategy(o);
  if (o.precision == FEA_F32_FUSED && o.scatter == FEA_SCATTER_AUTO)
    FEA_TRY(choose_strategy(m, pw, vel, kd, sr, phi, dt, n_eq, o, values, rhs, &st));
  const bool check = o.cancel_check && o.precision == FEA_F32_FUSED && m->n_elem > 0;
  if (!check) return run_strategy(m, pw, vel, kd, sr, phi, dt, n_eq, o, values, rhs, st);
  // the main assembly, then the FP64 recomputation of the flagged rows (inside the events)
  fea_assemble_opts om = o;
  om.event_end = nullptr;
  FEA_TRY(run_strategy(m, pw, vel, kd, sr, phi, dt, n_eq, om, values, rhs, st));
  AsmArgs<float> a = make_args<float>(m, p, vel, kd, sr, phi, dt, n_eq, &o, values, rhs);
  auto it = pw->cancel.find(n_eq);
  if (it == pw->cancel.end()) {  // the flag and row buffers: allocated once, before any capture
    if (stream_capturing(m->stream))
      return fail(FEA_ERR_STATE, "the first checked assembly for an equation count allocates the cancellation "
                                 "buffers and cannot run under stream capture");
    const size_t n = (size_t)std::max<int64_t>(m->n_node, 1);
    fea_pattern::CancelRows cr{nullptr, nullptr};
    if ((!pw->cancel_flags && cudaMalloc(&pw->cancel_flags, n) != cudaSuccess) ||
        cudaMalloc(&cr.rows, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&cr.count, sizeof *cr.count) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(cr.rows);
      return fail(FEA_ERR_OOM, "cancellation check: device allocation failed");
    }
    FEA_CUDA_TRY(cudaMemsetAsync(cr.count, 0, sizeof *cr.count, m->stream));
    it = pw->cancel.emplace(n_eq, cr).first;
  }
  FEA_TRY(cancel_check_rows(a, m->type, p->maxcol, pw->cancel_flags, it->second.rows, it->second.count, m->stream));
  if (o.event_end) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o.event_end, m->stream));
  return FEA_OK;
}

fea_status fea_residual(fea_mesh* m, const fea_pattern* p, const void* vel, const void* kd, const void* sr,
                        const void* phi_old, const void* phi, double dt, int32_t n_eq, const fea_assemble_opts* opts,
                        void* r) {
  fea_assemble_opts o;
  if (opts) o = *opts;
  else fea_default_opts(&o);
  FEA_TRY(check_assemble_args(m, p, vel, kd, sr, phi_old, dt, n_eq, &o, r, r));
  if (!phi) return fail(FEA_ERR_ARG, "fea_residual: phi is null");
  cudaStream_t s = m->stream;
  const size_t es = o.precision == FEA_F64_PLAIN ? sizeof(double) : sizeof(float);
  if (!o.accumulate) FEA_CUDA_TRY(cudaMemsetAsync(r, 0, es * (size_t)n_eq * (size_t)m->n_node, s));
  if (o.event_begin) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o.event_begin, s));
  if (m->n_elem > 0) {
    if (o.precision == FEA_F64_PLAIN) {
      AsmArgs<double> a = make_args<double>(m, p, vel, kd, sr, phi_old, dt, n_eq, &o, nullptr, nullptr);
      a.phi_eval = (const double*)phi;
      a.resid = (double*)r;
      FEA_TRY(elem_f64(m, p, a, n_eq, s));
    } else {
      AsmArgs<float> a = make_args<float>(m, p, vel, kd, sr, phi_old, dt, n_eq, &o, nullptr, nullptr);
      a.phi_eval = (const float*)phi;
      a.resid = (float*)r;
      FEA_TRY(elem_f32(m, const_cast<fea_pattern*>(p), a, s));  // the field scratch belongs to the pattern
    }
  }
  if (o.event_end) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o.event_end, s));
  return FEA_OK;
}

fea_status fea_cancel_rows(const fea_pattern* p, int32_t n_eq, int64_t* count) {
  if (!p || !count) return fail(FEA_ERR_ARG, "fea_cancel_rows: null argument");
  auto it = p->cancel.find(n_eq);
  if (it == p->cancel.end()) return fail(FEA_ERR_STATE, "no checked assembly for %d equations yet", n_eq);
  unsigned long long c = 0;
  FEA_CUDA_TRY(cudaStreamSynchronize(p->mesh->stream));
  FEA_CUDA_TRY(cudaMemcpy(&c, it->second.count, sizeof c, cudaMemcpyDeviceToHost));
  *count = (int64_t)c;
  return FEA_OK;
}

fea_status fea_tuned_strategy(const fea_pattern* p, int32_t n_eq, int32_t* scatter, int32_t* eq_groups) {
  if (!p || !scatter || !eq_groups) return fail(FEA_ERR_ARG, "fea_tuned_strategy: null argument");
  auto it = p->tuned.find(std::make_pair((int)n_eq, (int)FEA_TERM_ALL));
  if (it == p->tuned.end()) return fail(FEA_ERR_STATE, "no tuned strategy for %d equations yet", n_eq);
  *scatter = it->second.scatter;
  *eq_groups = it->second.eq_groups;
  return FEA_OK;
}

fea_status fea_tuned_config(const fea_pattern* p, int32_t n_eq, int32_t terms, fea_tuning* out) {
  if (!p || !out) return fail(FEA_ERR_ARG, "fea_tuned_config: null argument");
  auto it = p->tuned.find(std::make_pair((int)n_eq, (int)terms));
  if (it == p->tuned.end()) return fail(FEA_ERR_STATE, "no tuned configuration for %d equations, terms %d", n_eq, terms);
  *out = it->second;
  return FEA_OK;
}

fea_status fea_tune_candidates(const fea_pattern* p, int32_t n_eq, int32_t terms, fea_tuning* out, int32_t cap,
                               int32_t* count) {
  if (!p || !count || (cap > 0 && !out) || n_eq <= 0) return fail(FEA_ERR_ARG, "fea_tune_candidates: bad argument");
  fea_pattern* pw = const_cast<fea_pattern*>(p);
  const std::vector<Strategy> c = candidates(pw->mesh, pw, n_eq, terms);
  *count = (int32_t)c.size();
  for (int i = 0; i < (int)c.size() && i < cap; ++i) out[i] = to_tuning(c[i], 0, 0.f);
  return FEA_OK;
}

fea_status fea_assemble_host(fea_mesh* m, const fea_pattern* cp, const void* vel, const void* kd, const void* sr,
                             const void* phi, double dt, int32_t n_eq, const fea_assemble_opts* opts, void* values,
                             void* rhs) {
  fea_assemble_opts o;
  if (opts) o = *opts;
  else fea_default_opts(&o);
  FEA_TRY(check_assemble_args(m, cp, vel, kd, sr, phi, dt, n_eq, &o, values, rhs));
  fea_pattern* p = const_cast<fea_pattern*>(cp);
  cudaStream_t s = m->stream;
  size_t es = o.precision == FEA_F64_PLAIN ? sizeof(double) : sizeof(float);
  size_t N = (size_t)m->n_node, Q = (size_t)n_eq, nnz = (size_t)p->nnz;
  size_t b_vel = es * 3 * N, b_f = es * Q * N, b_val = es * Q * nnz;
  size_t need = b_vel + 3 * b_f + b_val + b_f + 8 * 256;
  if (p->ws_bytes < need) {
    cudaFree(p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    FEA_CUDA_TRY(cudaMalloc(&p->ws, need));
    p->ws_bytes = need;
  }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* base = (char*)p->ws;
  char* d_vel = base;
  char* d_kd = d_vel + al(b_vel);
  char* d_sr = d_kd + al(b_f);
  char* d_phi = d_sr + al(b_f);
  char* d_val = d_phi + al(b_f);
  char* d_rhs = d_val + al(b_val);
  // Copies run on N_COPY side streams at once (one copy engine per stream), ordered against
  // the assembly on the mesh stream by events: several concurrent copies move host data
  // faster than one.
  constexpr int NC = fea_mesh::N_COPY;
  if (!m->copy_ready) {
    for (int i = 0; i < NC; ++i) FEA_CUDA_TRY(cudaStreamCreateWithFlags(&m->copy_stream[i], cudaStreamNonBlocking));
    for (int i = 0; i <= NC; ++i) FEA_CUDA_TRY(cudaEventCreateWithFlags(&m->copy_event[i], cudaEventDisableTiming));
    for (int i = 0; i < fea_mesh::N_IN; ++i)
      FEA_CUDA_TRY(cudaStreamCreateWithFlags(&m->in_stream[i], cudaStreamNonBlocking));
    m->copy_ready = true;
  }
  cudaEvent_t start = m->copy_event[NC];  // recorded on s before each batch of copies
  struct Copy { void* dst; const void* src; size_t bytes; };
  // copies after the work on s so far; join = s waits for them (else join_copies does later)
  auto join_copies = [&]() -> fea_status {
    for (int i = 0; i < NC; ++i) {
      FEA_CUDA_TRY(cudaEventRecord(m->copy_event[i], m->copy_stream[i]));
      FEA_CUDA_TRY(cudaStreamWaitEvent(s, m->copy_event[i], 0));
    }
    return FEA_OK;
  };
  auto run_copies = [&](const Copy* c, int n, cudaMemcpyKind kind, bool join) -> fea_status {
    FEA_CUDA_TRY(cudaEventRecord(start, s));
    for (int i = 0; i < NC; ++i) FEA_CUDA_TRY(cudaStreamWaitEvent(m->copy_stream[i], start, 0));
    for (int i = 0; i < n; ++i)
      if (c[i].bytes) FEA_CUDA_TRY(cudaMemcpyAsync(c[i].dst, c[i].src, c[i].bytes, kind, m->copy_stream[i % NC]));
    return join ? join_copies() : FEA_OK;
  };
  // large arrays in NC pieces, cut at 256-byte boundaries
  auto split = [&](Copy* out, int& n, char* d, const char* h, size_t bytes, bool to_dev) {
    const size_t piece = ((bytes + NC - 1) / NC + 255) & ~(size_t)255;
    for (size_t off = 0; off < bytes; off += piece) {
      const size_t b = std::min(piece, bytes - off);
      out[n++] = to_dev ? Copy{d + off, h + off, b} : Copy{(void*)(h + off), d + off, b};
    }
  };
  // Large outputs: the equations are assembled in parts, each an independent assembly of its
  // slices, so that part k's values travel back while part k+1 computes.  About 16 GB of values
  // per part, 3 parts at least: fewer equations per part share each element's geometry less
  // (Hex8 256^3: 44, 55, 87 and 173 ms for 4, 8, 16 and 32 equations), more parts overlap more
  // of the copies; on 58 GB of values 4 parts took 389 ms, 2, 8 and 16 parts 424, 415 and
  // 667 ms, and on 5 GB 3 parts measured best of 3 and 6.
  const int parts = o.host_parts > 0 ? std::min(o.host_parts, n_eq)
                    : (b_val > ((size_t)256 << 20) && n_eq >= 3)
                        ? std::min<int>(n_eq, std::max<int>(3, (int)((b_val + (16ull << 30) - 1) / (16ull << 30))))
                        : 1;
  const int per = (n_eq + parts - 1) / parts;
  if (o.accumulate) {  // the outputs travel in as well: every input first, then the parts
    Copy in[4 + 2 * NC];
    int n_in = 0;
    in[n_in++] = Copy{d_vel, vel, b_vel};
    in[n_in++] = Copy{d_kd, kd, b_f};
    in[n_in++] = Copy{d_sr, sr, b_f};
    in[n_in++] = Copy{d_phi, phi, b_f};
    split(in, n_in, d_val, (const char*)values, b_val, true);
    in[n_in++] = Copy{d_rhs, rhs, b_f};
    FEA_TRY(run_copies(in, n_in, cudaMemcpyHostToDevice, true));
  } else {
    // each part's inputs on the host-to-device streams, so that part k's assembly waits only for
    // its own slices (the velocity goes first); the copies start after the work already on s
    constexpr int NI = fea_mesh::N_IN;
    while ((int)m->part_events.size() < NI * parts) {
      cudaEvent_t e;
      FEA_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      m->part_events.push_back(e);
    }
    FEA_CUDA_TRY(cudaEventRecord(start, s));
    for (int i = 0; i < NI; ++i) FEA_CUDA_TRY(cudaStreamWaitEvent(m->in_stream[i], start, 0));
    FEA_CUDA_TRY(cudaMemcpyAsync(d_vel, vel, b_vel, cudaMemcpyHostToDevice, m->in_stream[0]));
    for (int k = 0, q0 = 0; q0 < n_eq; ++k, q0 += per) {
      const int cnt = std::min(per, n_eq - q0);
      const size_t fo = es * (size_t)q0 * N, fb = es * (size_t)cnt * N;
      const char* src[3] = {(const char*)kd, (const char*)sr, (const char*)phi};
      char* dst[3] = {d_kd, d_sr, d_phi};
      for (int f = 0; f < 3; ++f) {  // each slice in NI pieces, cut at 256-byte boundaries
        const size_t piece = ((fb + NI - 1) / NI + 255) & ~(size_t)255;
        for (size_t off = 0, i = 0; off < fb; off += piece, ++i) {
          const size_t b = std::min(piece, fb - off);
          FEA_CUDA_TRY(cudaMemcpyAsync(dst[f] + fo + off, src[f] + fo + off, b, cudaMemcpyHostToDevice,
                                       m->in_stream[i % NI]));
        }
      }
      for (int i = 0; i < NI; ++i) FEA_CUDA_TRY(cudaEventRecord(m->part_events[NI * k + i], m->in_stream[i]));
    }
  }
  for (int k = 0, q0 = 0; q0 < n_eq; ++k, q0 += per) {
    const int cnt = std::min(per, n_eq - q0);
    const size_t fo = es * (size_t)q0 * N, vo = es * (size_t)q0 * nnz;
    if (!o.accumulate)
      for (int i = 0; i < fea_mesh::N_IN; ++i) FEA_CUDA_TRY(cudaStreamWaitEvent(s, m->part_events[fea_mesh::N_IN * k + i], 0));
    FEA_TRY(fea_assemble(m, p, d_vel, d_kd + fo, d_sr + fo, d_phi + fo, dt, cnt, &o, d_val + vo, d_rhs + fo));
    Copy outc[2 * NC + 1];
    int n_out = 0;
    split(outc, n_out, d_val + vo, (const char*)values + vo, es * (size_t)cnt * nnz, false);
    outc[n_out++] = Copy{(char*)rhs + fo, d_rhs + fo, es * (size_t)cnt * N};
    FEA_TRY(run_copies(outc, n_out, cudaMemcpyDeviceToHost, false));  // overlaps the next part
  }
  FEA_TRY(join_copies());
  return fea_sync(m);
}

}  // extern "C"
