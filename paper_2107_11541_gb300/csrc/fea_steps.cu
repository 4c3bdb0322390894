// fea_steps.cu -- the per-time-step field update and the multi-step CUDA graph.
//
// A time step of the transport solve reassembles the matrix and RHS from the latest
// nodal fields (the assembly is redone every step: it is the part of the step whose
// cost the paper measures, Tab. 1).  Here a step is: assemble, then move phi_old on by
// a smooth seeded perturbation, phi[q][n] += A_q sin(k_q . x_n + psi_q), whose
// parameters (A, k, psi per equation and step) are drawn by the caller and passed in.
// fea_graph_capture_steps records n_steps such steps into one CUDA graph, so a run of
// steps costs one graph launch instead of 3 n_steps kernel launches from the host.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {

// phi[q][n] += p[q].amp * sin(p[q].k . x_n + p[q].phase) over all equations and nodes;
// x_n = xhi + xlo (the float split of the FP64 coordinate), p = [n_eq][5] floats.
__global__ void k_update_fields(const float* __restrict__ xhi, const float* __restrict__ xlo, int64_t n_node,
                                float* __restrict__ phi, int n_eq, const float* __restrict__ params) {
  const int64_t total = n_node * n_eq;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / n_node);
    const int64_t n = i - (int64_t)q * n_node;
    const float* p = params + 5 * q;
    const float x = xhi[n] + xlo[n], y = xhi[n_node + n] + xlo[n_node + n],
                z = xhi[2 * n_node + n] + xlo[2 * n_node + n];
    const float arg = fmaf(p[1], x, fmaf(p[2], y, fmaf(p[3], z, p[4])));
    phi[i] = fmaf(p[0], sinf(arg), phi[i]);
  }
}

static fea_status launch_update(fea_mesh* m, float* phi, int n_eq, const float* params, cudaStream_t s) {
  const int64_t total = m->n_node * (int64_t)n_eq;
  if (total == 0) return FEA_OK;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)nsm * 8));
  k_update_fields<<<grid, 256, 0, s>>>(m->xhi, m->xlo, m->n_node, phi, n_eq, params);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

}  // namespace fea

using namespace fea;

struct fea_graph {
  fea_mesh* mesh = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches_per_run = 0;
};

extern "C" {

fea_status fea_update_fields(fea_mesh* m, void* phi, int32_t n_eq, const float* params) {
  if (!m || !phi || !params) return fail(FEA_ERR_ARG, "fea_update_fields: null argument");
  if (n_eq <= 0) return fail(FEA_ERR_ARG, "fea_update_fields: n_eq must be > 0 (got %d)", n_eq);
  return launch_update(m, (float*)phi, n_eq, params, m->stream);
}

fea_status fea_graph_capture_steps(fea_mesh* m, const fea_pattern* p, const void* vel, const void* kd, const void* sr,
                                   void* phi, double dt, int32_t n_eq, const fea_assemble_opts* opts, void* values,
                                   void* rhs, const float* params, int32_t n_steps, fea_graph** out) {
  if (!out) return fail(FEA_ERR_ARG, "fea_graph_capture_steps: out is null");
  *out = nullptr;
  if (!m || !params) return fail(FEA_ERR_ARG, "fea_graph_capture_steps: null argument");
  if (n_steps <= 0) return fail(FEA_ERR_ARG, "fea_graph_capture_steps: n_steps must be > 0 (got %d)", n_steps);
  fea_assemble_opts o;
  if (opts) o = *opts;
  else fea_default_opts(&o);
  if (o.precision != FEA_F32_FUSED) return fail(FEA_ERR_ARG, "fea_graph_capture_steps: the step graph is FP32");
  if (o.accumulate) return fail(FEA_ERR_ARG, "fea_graph_capture_steps: accumulate would add every step");
  o.event_begin = o.event_end = nullptr;
  // One eager assembly first: builds the schedules and scratch the assembly needs (host work and
  // allocations cannot be captured).  values/rhs are overwritten by every step of the graph.
  FEA_TRY(fea_assemble(m, p, vel, kd, sr, phi, dt, n_eq, &o, values, rhs));
  FEA_TRY(fea_sync(m));

  fea_graph* g = new (std::nothrow) fea_graph();
  if (!g) return fail(FEA_ERR_OOM, "host allocation failed");
  g->mesh = m;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    delete g;
    return fail(FEA_ERR_CUDA, "fea_graph_capture_steps: stream creation failed");
  }
  cudaStream_t saved = m->stream;
  m->stream = cs;  // every launch of the steps is recorded on the capture stream
  const int64_t launches0 = fea_kernel_launches();
  fea_status st = FEA_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = fail(FEA_ERR_CUDA, "fea_graph_capture_steps: begin capture failed");
  } else {
    for (int s = 0; s < n_steps && st == FEA_OK; ++s) {
      st = fea_assemble(m, p, vel, kd, sr, phi, dt, n_eq, &o, values, rhs);
      if (st == FEA_OK) st = launch_update(m, (float*)phi, n_eq, params + (size_t)5 * n_eq * s, cs);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (st == FEA_OK && e != cudaSuccess) st = fail(FEA_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    g->graph = graph;
    if (st == FEA_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess)
      st = fail(FEA_ERR_CUDA, "fea_graph_capture_steps: graph instantiation failed");
  }
  g->launches_per_run = fea_kernel_launches() - launches0;
  count_launches(-g->launches_per_run);  // recorded, not launched
  m->stream = saved;
  cudaStreamDestroy(cs);
  if (st != FEA_OK) {
    cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return st;
  }
  *out = g;
  return FEA_OK;
}

fea_status fea_graph_launch(fea_graph* g) {
  if (!g || !g->exec) return fail(FEA_ERR_ARG, "fea_graph_launch: graph is null");
  FEA_CUDA_TRY(cudaGraphLaunch(g->exec, g->mesh->stream));
  count_launches(g->launches_per_run);
  return FEA_OK;
}

fea_status fea_graph_destroy(fea_graph* g) {
  if (!g) return FEA_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return FEA_OK;
}

}  // extern "C"
