// fea_explicit.cu -- one explicit time step of the transport equations with a lumped mass.
//
// Sec. 2 advances heat and species with a third-order Runge-Kutta scheme and no algebraic
// solver.  The semi-discrete system is M_L dphi/dt = -A phi: A the convection, diffusion and
// reaction operator (the terms of the assembled matrix without the mass and SUPG parts),
// applied element by element by the matrix-free residual kernels (fea_residual with those
// terms gives r = -A phi, the RHS being zero), and M_L[i] = sum_j M_ij = int N_i dV the
// row-sum lumped mass, computed once per pattern and precision as -r of the mass term
// applied to the vector of ones.  The stages combine as
//     out = alpha x + beta (y + dt r / M_L)
// in one elementwise kernel: forward Euler is (0, 1) on phi; the strong-stability-preserving
// RK3 scheme is phi1 = (0, 1)(phi, phi), phi2 = (3/4, 1/4)(phi, phi1), phi = (1/3, 2/3)(phi, phi2).
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {
namespace {

template <typename T>
__global__ void k_rk_combine(const T* x, const T* __restrict__ y, const T* __restrict__ r, const T* __restrict__ ml,
                             int64_t n_node, int64_t total, T alpha, T beta, T dt, T* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i % n_node;
    const T step = y[i] + dt * r[i] / ml[n];
    out[i] = alpha == T(0) ? beta * step : alpha * x[i] + beta * step;  // x may alias out
  }
}

template <typename T>
__global__ void k_fill(T* a, int64_t n, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = v;
}

template <typename T>
__global__ void k_negate(T* a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a[i] = -a[i];
}

unsigned grid_for(int64_t total) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)nsm * 8));
}

template <typename T>
fea_status step_t(fea_mesh* m, fea_pattern* p, const void* vel, const void* kd, const void* sr, T* phi, double dt,
                  int32_t n_eq, int32_t stages, const fea_assemble_opts& o0) {
  cudaStream_t s = m->stream;
  const int64_t N = m->n_node, total = N * (int64_t)n_eq;
  const int slot = sizeof(T) == sizeof(double) ? 1 : 0;
  // the lumped mass of this precision: -(M 1), M the mass term (dt = 1) applied to ones
  if (!p->lumped[slot]) {
    void* ml = nullptr;
    void* tmp = nullptr;
    if (cudaMalloc(&ml, sizeof(T) * (size_t)std::max<int64_t>(N, 1)) != cudaSuccess ||
        cudaMalloc(&tmp, 2 * sizeof(T) * (size_t)std::max<int64_t>(N, 1)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ml);
      return fail(FEA_ERR_OOM, "explicit step: lumped mass allocation failed");
    }
    T* zeros = (T*)tmp;
    T* ones = zeros + N;
    fea_status st = FEA_OK;
    if (N > 0) {
      k_fill<T><<<grid_for(N), 256, 0, s>>>(zeros, N, T(0));
      k_fill<T><<<grid_for(N), 256, 0, s>>>(ones, N, T(1));
      count_launches(2);
      fea_assemble_opts om = o0;
      om.terms = FEA_TERM_MASS;
      om.accumulate = 0;
      om.event_begin = om.event_end = nullptr;
      st = fea_residual(m, p, vel, kd, sr, zeros, ones, 1.0, 1, &om, ml);
      if (st == FEA_OK) {
        k_negate<T><<<grid_for(N), 256, 0, s>>>((T*)ml, N);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) st = fail(FEA_ERR_CUDA, "explicit step: lumped mass kernels failed");
      }
      if (st == FEA_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(FEA_ERR_CUDA, "explicit step: sync failed");
    }
    cudaFree(tmp);
    if (st != FEA_OK) {
      cudaFree(ml);
      return st;
    }
    p->lumped[slot] = ml;
  }
  // workspace: r, phi1, phi2 [n_eq][N]
  const size_t one = sizeof(T) * (size_t)total, need = 3 * ((one + 255) & ~(size_t)255);
  if (p->rk_bytes < need) {
    FEA_CUDA_TRY(cudaStreamSynchronize(s));  // the old workspace may still be in use on the stream
    cudaFree(p->rk_ws);
    p->rk_ws = nullptr;
    p->rk_bytes = 0;
    if (cudaMalloc(&p->rk_ws, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(FEA_ERR_OOM, "explicit step: %zu bytes of stage workspace", need);
    }
    p->rk_bytes = need;
  }
  char* base = (char*)p->rk_ws;
  T* r = (T*)base;
  T* p1 = (T*)(base + ((one + 255) & ~(size_t)255));
  T* p2 = (T*)(base + 2 * ((one + 255) & ~(size_t)255));
  const T* ml = (const T*)p->lumped[slot];
  fea_assemble_opts ox = o0;  // r = -A x: convection, diffusion and reaction only (the RHS is zero)
  ox.terms = o0.terms & (FEA_TERM_CONV | FEA_TERM_DIFF | FEA_TERM_REAC);
  ox.accumulate = 0;
  ox.event_begin = ox.event_end = nullptr;
  auto residual = [&](const T* x) { return fea_residual(m, p, vel, kd, sr, x, x, dt, n_eq, &ox, r); };
  auto combine = [&](const T* x, const T* y, double alpha, double beta, T* out) -> fea_status {
    if (total > 0) k_rk_combine<T><<<grid_for(total), 256, 0, s>>>(x, y, r, ml, N, total, T(alpha), T(beta), T(dt), out);
    FEA_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return FEA_OK;
  };
  if (o0.event_begin) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o0.event_begin, s));
  if (stages == 1) {
    FEA_TRY(residual(phi));
    FEA_TRY(combine(phi, phi, 0.0, 1.0, phi));
  } else {
    FEA_TRY(residual(phi));
    FEA_TRY(combine(phi, phi, 0.0, 1.0, p1));
    FEA_TRY(residual(p1));
    FEA_TRY(combine(phi, p1, 0.75, 0.25, p2));
    FEA_TRY(residual(p2));
    FEA_TRY(combine(phi, p2, 1.0 / 3.0, 2.0 / 3.0, phi));
  }
  if (o0.event_end) FEA_CUDA_TRY(cudaEventRecord((cudaEvent_t)o0.event_end, s));
  return FEA_OK;
}

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" fea_status fea_explicit_step(fea_mesh* m, const fea_pattern* p, const void* vel, const void* kd,
                                        const void* sr, void* phi, double dt, int32_t n_eq, int32_t stages,
                                        const fea_assemble_opts* opts) {
  fea_assemble_opts o;
  if (opts) o = *opts;
  else fea_default_opts(&o);
  if (!m || !p || !vel || !kd || !sr || !phi) return fail(FEA_ERR_ARG, "fea_explicit_step: null argument");
  if (p->mesh != m) return fail(FEA_ERR_STATE, "pattern was built for another mesh");
  if (n_eq <= 0) return fail(FEA_ERR_ARG, "fea_explicit_step: n_eq must be > 0 (got %d)", n_eq);
  if (!(dt > 0.0)) return fail(FEA_ERR_ARG, "fea_explicit_step: dt must be > 0");
  if (stages != 1 && stages != 3) return fail(FEA_ERR_ARG, "fea_explicit_step: stages must be 1 or 3 (got %d)", stages);
  if (o.precision != FEA_F64_PLAIN && o.precision != FEA_F32_FUSED) return fail(FEA_ERR_ARG, "unknown precision");
  if (!(o.terms & (FEA_TERM_CONV | FEA_TERM_DIFF | FEA_TERM_REAC)))
    return fail(FEA_ERR_ARG, "fea_explicit_step: the terms select none of convection, diffusion, reaction");
  fea_pattern* pw = const_cast<fea_pattern*>(p);  // the lumped mass and the stage workspace belong to the pattern
  if (o.precision == FEA_F64_PLAIN) return step_t<double>(m, pw, vel, kd, sr, (double*)phi, dt, n_eq, stages, o);
  return step_t<float>(m, pw, vel, kd, sr, (float*)phi, dt, n_eq, stages, o);
}
