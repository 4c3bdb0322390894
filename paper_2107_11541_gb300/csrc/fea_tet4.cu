// fea_tet4.cu -- FP32 Tet4 assembly, one thread per (element, equation) item.
//
// The P1 tetrahedron has constant shape-function gradients, so an element's geometry is
// one 3x3 Jacobian J = [x1-x0 | x2-x0 | x3-x0], det J = 6 V_e, grad N_a = J^-T grad_xi N_a
// (grad N_0 = -(grad N_1 + grad N_2 + grad N_3)); the 4-point rule (barycentric
// (alpha, beta, beta, beta) permutations, weight 1/24) carries the interpolated u, k, s,
// phi_old and tau.  The operator is the one of Sec. 4.2, Listing 1 extended to the full
// Galerkin + SUPG form; each item keeps its 4x4 element matrix and 4 RHS entries in
// registers and adds them with atomics into the CSR values and RHS (whose single
// equation slice of a large Tet4 mesh stays resident in the 129 MB L2), or stores them
// to the gather scratch.  Gauss points of badly conditioned elements (condition estimate
// above the threshold, or det <= 0 in FP32) get J^-1 from the FP64 coordinates.  Elements
// are visited in the pattern's Morton order of their centroids, so that the lanes of a warp
// hold neighbouring elements and their atomics land on few rows; the pattern keeps each
// element's node ids and CSR positions in that order too, as 80-byte records, so that a warp's
// loads of them are contiguous.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {
namespace {

constexpr float T4_ALPHA = 0.58541019662496845446f;  // (5 + 3 sqrt 5) / 20
constexpr float T4_BETA = 0.13819660112501051518f;   // (5 - sqrt 5) / 20

__global__ void __launch_bounds__(256) k_tet4_f32(AsmArgs<float> p) {
  const int64_t items = p.n_elem * p.eq_count;
  const int64_t N = p.n_node;
  const float inv_dt = (float)(1.0 / p.dt);
  const bool t_mass = p.terms & FEA_TERM_MASS, t_conv = p.terms & FEA_TERM_CONV, t_diff = p.terms & FEA_TERM_DIFF,
             t_reac = p.terms & FEA_TERM_REAC, t_supg = p.terms & FEA_TERM_SUPG;
  // 16-byte loads of an element's connectivity and position rows, when the block's arrays start
  // 16-byte aligned (a Tet4 block after blocks of other types may not)
  const bool vec = ((reinterpret_cast<uintptr_t>(p.conn) | reinterpret_cast<uintptr_t>(p.pos)) & 15) == 0;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t eo = it / p.eq_count;
    const int qq = (int)(it - eo * p.eq_count), q = p.eq0 + qq;
    const int64_t e = p.elem_order ? (int64_t)__ldg(p.elem_order + eo) : eo;
    int32_t n[4];
    const int4* rec = p.t4_rows ? reinterpret_cast<const int4*>(p.t4_rows) + eo * 5 : nullptr;  // 80-byte record
    if (rec) {
      const int4 c4 = __ldg(rec);
      n[0] = c4.x;
      n[1] = c4.y;
      n[2] = c4.z;
      n[3] = c4.w;
    } else if (vec) {
      const int4 c4 = __ldg(reinterpret_cast<const int4*>(p.conn) + e);  // conn [E][4]: 16-byte rows
      n[0] = c4.x;
      n[1] = c4.y;
      n[2] = c4.z;
      n[3] = c4.w;
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) n[a] = __ldg(p.conn + e * 4 + a);
    }
    // node data: coordinates (float hi/lo), velocity and the equation's k, s, phi_old, from the
    // per-call node records (one equation: 48 bytes per node, three 16-byte loads) or the arrays
    float xh[4][3], xl[4][3], un[4][3], kn[4], sn[4], pn[4];
    const int64_t fo = (int64_t)q * N;
    if (p.t4_node) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4* r = p.t4_node + (int64_t)n[a] * 3;
        const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2);
        xh[a][0] = r0.x;
        xh[a][1] = r0.y;
        xh[a][2] = r0.z;
        xl[a][0] = r0.w;
        xl[a][1] = r1.x;
        xl[a][2] = r1.y;
        un[a][0] = r1.z;
        un[a][1] = r1.w;
        un[a][2] = r2.x;
        kn[a] = r2.y;
        sn[a] = r2.z;
        pn[a] = r2.w;
      }
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          xh[a][i] = __ldg(p.xhi + (int64_t)i * N + n[a]);
          xl[a][i] = __ldg(p.xlo + (int64_t)i * N + n[a]);
          un[a][i] = __ldg(p.vel + (int64_t)i * N + n[a]);
        }
        kn[a] = __ldg(p.kd + fo + n[a]);
        sn[a] = __ldg(p.sr + fo + n[a]);
        pn[a] = __ldg(p.phi + fo + n[a]);
      }
    }
    float J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) J[i][j] = (xh[j + 1][i] - xh[0][i]) + (xl[j + 1][i] - xl[0][i]);
    float det = det3(J), G[3][3];
    inv_transpose3(J, det, G);
    float nj = 0.f, ni = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        nj = fmaf(J[i][j], J[i][j], nj);
        ni = fmaf(G[i][j], G[i][j], ni);
      }
    if (!(det > 0.f) || !(nj * ni <= (float)(p.kappa_threshold * p.kappa_threshold))) {
      double Jd[3][3], Gd[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Jd[i][j] = p.coords[(int64_t)n[j + 1] * 3 + i] - p.coords[(int64_t)n[0] * 3 + i];
      const double dd = det3(Jd);
      if (!(dd > 0.0)) atomicOr(p.status, ST_INVERTED);
      inv_transpose3(Jd, dd, Gd);
      det = (float)dd;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[i][j] = (float)Gd[i][j];
    }
    // grad N_a: column a-1 of J^-T for a = 1..3 (grad_xi N_a = e_{a-1}), grad N_0 = -sum
    float gr[4][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gr[1][i] = G[i][0];
      gr[2][i] = G[i][1];
      gr[3][i] = G[i][2];
      gr[0][i] = -(G[i][0] + G[i][1] + G[i][2]);
    }
    const float dv = det * (1.0f / 24.0f);  // w_g det J, the same at every point
    const float h = cbrtf(4.0f * dv);       // V_e^(1/3), V_e = sum_g dv
    const float c_k = 4.0f / (h * h), c_u = 2.0f / h;
    float A[4][4], b[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      b[a] = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) A[a][c] = 0.f;
    }
    float kd_sum = 0.f;  // sum_g dv k_g: the diffusion matrix is (grad N_a . grad N_b) times it
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float Ng[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) Ng[a] = a == g ? T4_ALPHA : T4_BETA;
      float ug[3] = {0.f, 0.f, 0.f}, kg = 0.f, sg = 0.f, pg = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int i = 0; i < 3; ++i) ug[i] = fmaf(Ng[a], un[a][i], ug[i]);
        kg = fmaf(Ng[a], kn[a], kg);
        sg = fmaf(Ng[a], sn[a], sg);
        pg = fmaf(Ng[a], pn[a], pg);
      }
      float ua[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ua[a] = ug[0] * gr[a][0] + ug[1] * gr[a][1] + ug[2] * gr[a][2];
      const float unorm = sqrtf(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
      const float den = c_k * kg + c_u * unorm + sg;
      const float tau = den > 0.f ? 1.0f / den : 0.f;
      kd_sum = fmaf(dv, kg, kd_sum);
      // test function part (N_a, SUPG) and trial part ((mass, reaction) N_b, convection)
      const float sig = (t_mass ? inv_dt : 0.f) + (t_reac ? sg : 0.f);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float Pa = dv * Ng[a];
        const float Sa = t_supg ? dv * tau * ua[a] : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v = Pa * (sig * Ng[c] + (t_conv ? ua[c] : 0.f));
          v = fmaf(Sa, inv_dt * Ng[c] + ua[c] + sg * Ng[c], v);
          A[a][c] += v;
        }
        b[a] = fmaf((t_mass ? Pa : 0.f) + Sa, pg * inv_dt, b[a]);
      }
    }
    if (t_diff) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          A[a][c] = fmaf(kd_sum, gr[a][0] * gr[c][0] + gr[a][1] * gr[c][1] + gr[a][2] * gr[c][2], A[a][c]);
    }
    if (p.resid) {  // matrix-free: b_a - (A^e phi)_a
      const float* fq = p.phi_eval + fo;
      float ph[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) ph[c] = __ldg(fq + n[c]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        float y = b[a];
#pragma unroll
        for (int c = 0; c < 4; ++c) y = fmaf(-A[a][c], ph[c], y);
        atomicAdd(p.resid + fo + n[a], y);
      }
    } else if (p.em) {
      float* d = p.em + e * 20 * p.eq_count + qq;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int c = 0; c < 4; ++c) d[(a * 4 + c) * p.eq_count] = A[a][c];
        d[(16 + a) * p.eq_count] = b[a];
      }
    } else {
      float* vq = p.values + (int64_t)q * p.nnz;
      const int32_t* pe = p.pos + e * 16;  // pos [E][4][4]
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int4 k4 = rec   ? __ldg(rec + 1 + a)
                        : vec ? __ldg(reinterpret_cast<const int4*>(pe) + a)
                              : make_int4(__ldg(pe + 4 * a), __ldg(pe + 4 * a + 1), __ldg(pe + 4 * a + 2),
                                          __ldg(pe + 4 * a + 3));
        atomicAdd(vq + k4.x, A[a][0]);
        atomicAdd(vq + k4.y, A[a][1]);
        atomicAdd(vq + k4.z, A[a][2]);
        atomicAdd(vq + k4.w, A[a][3]);
        atomicAdd(p.rhs + fo + n[a], b[a]);
      }
    }
  }
}

// Per-call node records of one equation: xhi, xlo, u, k, s, phi_old as three float4 per node.
__global__ void k_t4_nodes(const float* __restrict__ xhi, const float* __restrict__ xlo, const float* __restrict__ vel,
                           const float* __restrict__ kd, const float* __restrict__ sr, const float* __restrict__ phi,
                           int64_t n_node, float4* __restrict__ out) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < n_node; n += (int64_t)gridDim.x * blockDim.x) {
    const int64_t N = n_node;
    out[3 * n] = make_float4(xhi[n], xhi[N + n], xhi[2 * N + n], xlo[n]);
    out[3 * n + 1] = make_float4(xlo[N + n], xlo[2 * N + n], vel[n], vel[N + n]);
    out[3 * n + 2] = make_float4(vel[2 * N + n], kd[n], sr[n], phi[n]);
  }
}

}  // namespace

fea_status tet4_node_records(const AsmArgs<float>& a, float4* out, cudaStream_t s) {
  if (a.n_node == 0) return FEA_OK;
  const int64_t fo = (int64_t)a.eq0 * a.n_node;
  k_t4_nodes<<<(unsigned)std::min<int64_t>((a.n_node + 255) / 256, 152 * 16), 256, 0, s>>>(
      a.xhi, a.xlo, a.vel, a.kd + fo, a.sr + fo, a.phi + fo, a.n_node, out);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

fea_status launch_tet4_f32(const AsmArgs<float>& a, cudaStream_t s) {
  const int64_t items = a.n_elem * a.eq_count;
  if (items == 0) return FEA_OK;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int threads = a.batch == 128 ? 128 : 256;  // one (element, equation) item per thread
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((items + threads - 1) / threads, (int64_t)nsm * 16 * (256 / threads)));
  k_tet4_f32<<<grid, threads, 0, s>>>(a);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

}  // namespace fea
