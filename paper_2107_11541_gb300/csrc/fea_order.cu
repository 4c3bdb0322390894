// fea_order.cu -- a locality order of a mesh's elements (setup, built with the pattern).
//
// The element kernels that scatter with atomics walk the elements in the order of the
// Morton code of their centroids, so that the lanes of a warp hold elements of one small
// region: their atomic adds land on a few CSR rows and their node loads on a few lines.
// (Unstructured meshes number elements arbitrarily; the paper's packs group elements by
// type only, Sec. 4.3.)  Steps: the bounding box of the nodes (block partials, then one
// block), a 30-bit key per element from its centroid quantised to 1024 cells per axis, and a
// radix sort of (key, element id) pairs.
#include <cub/cub.cuh>

#include <algorithm>
#include <cfloat>

#include "fea_internal.cuh"

namespace fea {
namespace {

constexpr int OT = 256;
constexpr int BBOX_BLOCKS = 304;

__global__ void __launch_bounds__(OT) k_bbox_partial(const double* __restrict__ coords, int64_t n, double* part) {
  __shared__ double lo[3][OT], hi[3][OT];
  double l[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, h[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t i = (int64_t)blockIdx.x * OT + threadIdx.x; i < n; i += (int64_t)gridDim.x * OT)
    for (int d = 0; d < 3; ++d) {
      const double x = coords[i * 3 + d];
      l[d] = fmin(l[d], x);
      h[d] = fmax(h[d], x);
    }
  for (int d = 0; d < 3; ++d) {
    lo[d][threadIdx.x] = l[d];
    hi[d][threadIdx.x] = h[d];
  }
  __syncthreads();
  for (int s = OT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        lo[d][threadIdx.x] = fmin(lo[d][threadIdx.x], lo[d][threadIdx.x + s]);
        hi[d][threadIdx.x] = fmax(hi[d][threadIdx.x], hi[d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 3; ++d) {
      part[blockIdx.x * 6 + d] = lo[d][0];
      part[blockIdx.x * 6 + 3 + d] = hi[d][0];
    }
}

__global__ void k_bbox_final(double* part, int nparts) {
  if (threadIdx.x != 0) return;
  for (int b = 1; b < nparts; ++b)
    for (int d = 0; d < 3; ++d) {
      part[d] = fmin(part[d], part[b * 6 + d]);
      part[3 + d] = fmax(part[3 + d], part[b * 6 + 3 + d]);
    }
}

// Spreads the low 10 bits of v to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_morton(const double* __restrict__ coords, const int32_t* __restrict__ conn, int64_t n_elem, int nen,
                         const double* __restrict__ bbox, uint32_t* keys, int32_t* ids) {
  const int64_t e = (int64_t)blockIdx.x * OT + threadIdx.x;
  if (e >= n_elem) return;
  uint32_t q[3];
  for (int d = 0; d < 3; ++d) {
    double c = 0.0;
    for (int a = 0; a < nen; ++a) c += coords[(int64_t)conn[e * nen + a] * 3 + d];
    c /= nen;
    const double ext = bbox[3 + d] - bbox[d];
    const double t = ext > 0.0 ? (c - bbox[d]) / ext : 0.0;
    q[d] = (uint32_t)fmin(fmax(t * 1024.0, 0.0), 1023.0);
  }
  keys[e] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  ids[e] = (int32_t)e;
}

}  // namespace

fea_status element_order(const fea_mesh* m, int32_t** out) {
  *out = nullptr;
  const int64_t E = m->n_elem, N = m->n_node;
  if (m->mixed || E < 2) return FEA_OK;
  cudaStream_t s = m->stream;
  double* part = nullptr;
  uint32_t *k0 = nullptr, *k1 = nullptr;
  int32_t *i0 = nullptr, *i1 = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  auto done = [&](fea_status st) {
    cudaFree(part);
    cudaFree(k0);
    cudaFree(k1);
    cudaFree(i0);
    cudaFree(tmp);
    if (st != FEA_OK) cudaFree(i1);
    return st;
  };
  FEA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k0, k1, i0, i1, (int)E, 0, 30, s));
  if (cudaMalloc(&part, sizeof(double) * 6 * BBOX_BLOCKS) != cudaSuccess ||
      cudaMalloc(&k0, sizeof(uint32_t) * E) != cudaSuccess || cudaMalloc(&k1, sizeof(uint32_t) * E) != cudaSuccess ||
      cudaMalloc(&i0, sizeof(int32_t) * E) != cudaSuccess || cudaMalloc(&i1, sizeof(int32_t) * E) != cudaSuccess ||
      cudaMalloc(&tmp, std::max<size_t>(tmp_bytes, 1)) != cudaSuccess) {
    cudaGetLastError();
    return done(fail(FEA_ERR_OOM, "element order: device allocation failed"));
  }
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((N + OT - 1) / OT, BBOX_BLOCKS));
  k_bbox_partial<<<nb, OT, 0, s>>>(m->coords, N, part);
  k_bbox_final<<<1, 32, 0, s>>>(part, nb);
  k_morton<<<(unsigned)((E + OT - 1) / OT), OT, 0, s>>>(m->coords, m->conn, E, m->nen, part, k0, i0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return done(fail(FEA_ERR_CUDA, "element order launch: %s", cudaGetErrorString(e)));
  e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k0, k1, i0, i1, (int)E, 0, 30, s);
  if (e != cudaSuccess) return done(fail(FEA_ERR_CUDA, "element order sort: %s", cudaGetErrorString(e)));
  e = cudaStreamSynchronize(s);  // the temporaries are freed below
  if (e != cudaSuccess) return done(fail(FEA_ERR_CUDA, "element order: %s", cudaGetErrorString(e)));
  *out = i1;
  return done(FEA_OK);
}

namespace {
__global__ void k_tet4_rows(const int32_t* __restrict__ order, const int32_t* __restrict__ conn,
                            const int32_t* __restrict__ pos, int64_t n_elem, int32_t* __restrict__ out) {
  const int64_t total = n_elem * 20;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / 20, j = i - k * 20, e = order ? (int64_t)order[k] : k;  // no order: the given one
    out[i] = j < 4 ? conn[e * 4 + j] : pos[e * 16 + (j - 4)];
  }
}
}  // namespace

fea_status tet4_rows(const fea_mesh* m, const int32_t* order, const int32_t* pos, int32_t** out) {
  *out = nullptr;
  const int64_t E = m->n_elem;
  if (E == 0) return FEA_OK;
  int32_t* rows = nullptr;
  if (cudaMalloc(&rows, sizeof(int32_t) * 20 * (size_t)E) != cudaSuccess) {
    cudaGetLastError();
    return fail(FEA_ERR_OOM, "Tet4 element rows: %lld bytes", (long long)(80 * E));
  }
  const int64_t total = 20 * E;
  k_tet4_rows<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, m->stream>>>(order, m->conn, pos,
                                                                                                  E, rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(rows);
    return fail(FEA_ERR_CUDA, "Tet4 element rows: %s", cudaGetErrorString(e));
  }
  count_launches(1);
  *out = rows;
  return FEA_OK;
}

}  // namespace fea
