// fea_pcg.cu -- Jacobi-preconditioned conjugate gradients on the n_eq FP32 matrices that
// share one CSR pattern (Sec. 2, Alg. 1: the algebraic solver is a preconditioned CG; the
// preconditioner is not named, the diagonal one is used here).
//
// All equations iterate together, each with its own scalars (kept in FP64 on the device):
//   r = b - A x, z = D^-1 r, p = z, rz = r.z
//   repeat:  Ap = A p;  alpha = rz / p.Ap;  x += alpha p;  r -= alpha Ap;  z = D^-1 r;
//            beta = r.z_new / rz;  p = z + beta p
// An equation stops when ||r||_2 <= rtol ||b||_2 or after max_iter iterations; the decision
// is taken on the device (the host reads the flags every few iterations to end the loop).
// Vectors are [n_eq][n_node] float; the dot products are block reductions added in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fea_internal.cuh"

namespace fea {
namespace {

constexpr int T = 256;

struct Scal {
  double bb, rr, rz, rz_new, pAp, alpha, beta;
  int active, iters, breakdown, pad;
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;  // valid on thread 0
}

// Position of the diagonal entry of every row (column r in row r).
__global__ void k_diag_pos(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind, int64_t n,
                           int32_t* diag) {
  for (int64_t r = (int64_t)blockIdx.x * T + threadIdx.x; r < n; r += (int64_t)gridDim.x * T) {
    int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (colind[mid] < r) lo = mid + 1;
      else hi = mid;
    }
    diag[r] = (int32_t)lo;
  }
}

// D^-1 per equation; a non-positive diagonal marks the equation as broken down.
__global__ void k_inv_diag(const float* __restrict__ values, const int32_t* __restrict__ diag, int64_t n, int64_t nnz,
                           float* inv_diag, Scal* sc) {
  const int q = blockIdx.y;
  for (int64_t r = (int64_t)blockIdx.x * T + threadIdx.x; r < n; r += (int64_t)gridDim.x * T) {
    const float d = values[(int64_t)q * nnz + diag[r]];
    if (!(d > 0.f)) {
      sc[q].breakdown = 1;
      inv_diag[(int64_t)q * n + r] = 1.f;
    } else {
      inv_diag[(int64_t)q * n + r] = 1.f / d;
    }
  }
}

// r = b - Ax (Ax in ap), z = D^-1 r, p = z; rz, rr, bb.
__global__ void __launch_bounds__(T) k_init(const float* __restrict__ b, const float* __restrict__ ap,
                                            const float* __restrict__ inv_diag, float* r, float* z, float* p,
                                            int64_t n, Scal* sc) {
  __shared__ double sh[T / 32];
  const int q = blockIdx.y;
  const int64_t o = (int64_t)q * n;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T) {
    const float bi = b[o + i], ri = bi - ap[o + i], zi = inv_diag[o + i] * ri;
    r[o + i] = ri;
    z[o + i] = zi;
    p[o + i] = zi;
    rz += (double)ri * zi;
    rr += (double)ri * ri;
    bb += (double)bi * bi;
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&sc[q].rz, rz);
    atomicAdd(&sc[q].rr, rr);
    atomicAdd(&sc[q].bb, bb);
  }
}

// Which equations iterate: not yet within rtol, no breakdown, iterations left.
__global__ void k_start(Scal* sc, int n_eq, double rtol2, int max_iter) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_eq) return;
  Scal& s = sc[q];
  s.iters = 0;
  s.active = !s.breakdown && max_iter > 0 && s.rr > rtol2 * s.bb;
  if (s.active) s.rr = 0.0;  // the iterations sum the new residual; a stopped equation keeps its ||r||^2
}

// p.Ap of the active equations.
__global__ void __launch_bounds__(T) k_dot_pap(const float* __restrict__ p, const float* __restrict__ ap, int64_t n,
                                               Scal* sc) {
  __shared__ double sh[T / 32];
  const int q = blockIdx.y;
  if (!sc[q].active) return;  // uniform over the block
  const int64_t o = (int64_t)q * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T)
    s += (double)p[o + i] * ap[o + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) atomicAdd(&sc[q].pAp, s);
}

// alpha = rz / p.Ap (a non-positive p.Ap is a breakdown: the matrix is not positive definite).
__global__ void k_alpha(Scal* sc, int n_eq) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_eq) return;
  Scal& s = sc[q];
  s.alpha = 0.0;
  if (!s.active) return;
  if (!(s.pAp > 0.0)) {
    s.breakdown = 1;
    s.active = 0;
    return;
  }
  s.alpha = s.rz / s.pAp;
}

// x += alpha p, r -= alpha Ap, z = D^-1 r; r.z and r.r of the new residual.
__global__ void __launch_bounds__(T) k_update(float* x, float* r, float* z, const float* __restrict__ p,
                                              const float* __restrict__ ap, const float* __restrict__ inv_diag,
                                              int64_t n, Scal* sc) {
  __shared__ double sh[T / 32];
  const int q = blockIdx.y;
  if (!sc[q].active) return;
  const float alpha = (float)sc[q].alpha;
  const int64_t o = (int64_t)q * n;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T) {
    x[o + i] = fmaf(alpha, p[o + i], x[o + i]);
    const float ri = fmaf(-alpha, ap[o + i], r[o + i]), zi = inv_diag[o + i] * ri;
    r[o + i] = ri;
    z[o + i] = zi;
    rz += (double)ri * zi;
    rr += (double)ri * ri;
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&sc[q].rz_new, rz);
    atomicAdd(&sc[q].rr, rr);
  }
}

// beta, the iteration count and the stopping test; resets the sums of the next iteration.
__global__ void k_beta(Scal* sc, int n_eq, double rtol2, int max_iter) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_eq) return;
  Scal& s = sc[q];
  s.beta = 0.0;
  if (s.active) {
    s.iters += 1;
    s.beta = s.rz > 0.0 ? s.rz_new / s.rz : 0.0;
    s.rz = s.rz_new;
    if (s.rr <= rtol2 * s.bb || s.iters >= max_iter) s.active = 0;
  }
  s.rz_new = 0.0;
  s.pAp = 0.0;
  if (s.active) s.rr = 0.0;  // a stopped equation keeps its last ||r||^2
}

// p = z + beta p.
__global__ void __launch_bounds__(T) k_direction(float* p, const float* __restrict__ z, int64_t n, const Scal* sc) {
  const int q = blockIdx.y;
  if (!sc[q].active) return;
  const float beta = (float)sc[q].beta;
  const int64_t o = (int64_t)q * n;
  for (int64_t i = (int64_t)blockIdx.x * T + threadIdx.x; i < n; i += (int64_t)gridDim.x * T)
    p[o + i] = fmaf(beta, p[o + i], z[o + i]);
}

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" {

fea_status fea_pcg(const fea_pattern* cp, const float* values, const float* b, float* x, int32_t n_eq,
                   int32_t max_iter, double rtol, int32_t* iters, double* rel_resid, void* stream) {
  if (!cp || !values || !b || !x) return fail(FEA_ERR_ARG, "fea_pcg: null argument");
  if (n_eq <= 0) return fail(FEA_ERR_ARG, "fea_pcg: n_eq must be > 0 (got %d)", n_eq);
  if (n_eq > 65535) return fail(FEA_ERR_ARG, "fea_pcg: at most 65535 equations per call");
  if (max_iter < 0 || !(rtol >= 0.0)) return fail(FEA_ERR_ARG, "fea_pcg: max_iter >= 0 and rtol >= 0 required");
  fea_pattern* p = const_cast<fea_pattern*>(cp);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = p->mesh->n_node;
  const size_t vec = sizeof(float) * (size_t)n_eq * (size_t)n;
  const size_t need = 5 * ((vec + 255) & ~(size_t)255) + sizeof(Scal) * (size_t)n_eq + 256;
  if (!p->diag) {
    FEA_CUDA_TRY(cudaMalloc(&p->diag, sizeof(int32_t) * std::max<int64_t>(n, 1)));
    if (n > 0) {
      k_diag_pos<<<(unsigned)std::min<int64_t>((n + T - 1) / T, 152 * 8), T, 0, s>>>(p->rowptr, p->colind, n, p->diag);
      FEA_CUDA_TRY(cudaGetLastError());
      count_launches(1);
    }
  }
  if (p->pcg_bytes < need) {
    FEA_CUDA_TRY(cudaStreamSynchronize(s));  // the old workspace may still be in use on the stream
    cudaFree(p->pcg_ws);
    p->pcg_ws = nullptr;
    p->pcg_bytes = 0;
    FEA_CUDA_TRY(cudaMalloc(&p->pcg_ws, need));
    p->pcg_bytes = need;
  }
  const size_t va = (vec + 255) & ~(size_t)255;
  char* base = (char*)p->pcg_ws;
  float* r = (float*)base;
  float* z = (float*)(base + va);
  float* pv = (float*)(base + 2 * va);
  float* ap = (float*)(base + 3 * va);
  float* dinv = (float*)(base + 4 * va);
  Scal* sc = (Scal*)(base + 5 * va);
  FEA_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(Scal) * (size_t)n_eq, s));
  const double rtol2 = rtol * rtol;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + T - 1) / T, std::max(1, 1216 / n_eq)));
  const dim3 gv(gx, (unsigned)n_eq);
  const unsigned gs = (unsigned)((n_eq + 127) / 128);
  if (n > 0) {
    k_inv_diag<<<gv, T, 0, s>>>(values, p->diag, n, p->nnz, dinv, sc);
    FEA_TRY(launch_spmv_f32(p, values, x, ap, n_eq, false, s));
    k_init<<<gv, T, 0, s>>>(b, ap, dinv, r, z, pv, n, sc);
    count_launches(2);
  }
  k_start<<<gs, 128, 0, s>>>(sc, n_eq, rtol2, max_iter);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  std::vector<Scal> host((size_t)n_eq);
  constexpr int CHECK = 8;  // iterations between reads of the stopping flags
  for (int it = 0; it < max_iter && n > 0; ++it) {
    if (it % CHECK == 0) {
      FEA_CUDA_TRY(cudaMemcpyAsync(host.data(), sc, sizeof(Scal) * (size_t)n_eq, cudaMemcpyDeviceToHost, s));
      FEA_CUDA_TRY(cudaStreamSynchronize(s));
      bool any = false;
      for (const Scal& h : host) any |= h.active != 0;
      if (!any) break;
    }
    FEA_TRY(launch_spmv_f32(p, values, pv, ap, n_eq, false, s));
    k_dot_pap<<<gv, T, 0, s>>>(pv, ap, n, sc);
    k_alpha<<<gs, 128, 0, s>>>(sc, n_eq);
    k_update<<<gv, T, 0, s>>>(x, r, z, pv, ap, dinv, n, sc);
    k_beta<<<gs, 128, 0, s>>>(sc, n_eq, rtol2, max_iter);
    k_direction<<<gv, T, 0, s>>>(pv, z, n, sc);
    FEA_CUDA_TRY(cudaGetLastError());
    count_launches(5);
  }
  FEA_CUDA_TRY(cudaMemcpyAsync(host.data(), sc, sizeof(Scal) * (size_t)n_eq, cudaMemcpyDeviceToHost, s));
  FEA_CUDA_TRY(cudaStreamSynchronize(s));
  int broken = -1;
  for (int q = 0; q < n_eq; ++q) {
    if (iters) iters[q] = host[q].iters;
    if (rel_resid) rel_resid[q] = host[q].bb > 0.0 ? std::sqrt(host[q].rr / host[q].bb) : std::sqrt(host[q].rr);
    if (host[q].breakdown && broken < 0) broken = q;
  }
  if (broken >= 0)
    return fail(FEA_ERR_ARG, "fea_pcg: equation %d is not positive definite (diagonal or p.Ap <= 0)", broken);
  return FEA_OK;
}

}  // extern "C"
