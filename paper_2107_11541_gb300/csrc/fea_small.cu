// fea_small.cu -- FP32 assembly of the small non-affine elements (Pen6 prisms, Pyr5
// pyramids), one thread per (element, equation) item.
//
// Each item gathers its element's nodes (coordinate differences from the FP32 hi/lo split,
// velocity, and its equation's k, s, phi_old), then walks the Gauss points twice:
//   1. J = sum_a (x_a - x_0) dN_a/dxi, det J and J^-T (FP64 from the FP64 coordinates where
//      the condition estimate exceeds the threshold or det <= 0 in FP32), dV = w det J; the
//      element volume V = sum_g dV gives h = V^(1/3);
//   2. J, det J and J^-T again (the same arithmetic, so the same dV), grad N_a = J^-T
//      grad_xi N_a, u_g, k_g, s_g, phi_g, tau_g, and the element
//      matrix and RHS of Sec. 4.2, Listing 1 extended to the full Galerkin + SUPG operator,
//      accumulated in registers.
// The reference shape functions, their gradients and the weights at the Gauss points sit in
// a shared-memory table filled once per block.  The result goes out as atomic adds into the
// CSR values and RHS, as stores to the gather scratch, or as the matrix-free residual.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {
namespace {

// J^-T at point g of the element whose FP32 coordinate differences are xd (FP64 from the
// FP64 coordinates when badly conditioned); returns det J.
template <int TYPE>
__device__ __forceinline__ float point_inverse(const AsmArgs<float>& p, const float (*dNg)[3], const float xd[][3],
                                               const int32_t* n, int g, float G[3][3]) {
  constexpr int NEN = Elem<TYPE>::NEN;
  float J[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
  for (int a = 0; a < NEN; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) J[i][j] = fmaf(xd[a][i], dNg[a][j], J[i][j]);
  float det = det3(J);
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
    double xid[3], w, Jd[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Gd[3][3];
    gauss_point<TYPE>(g, xid, w);
    for (int a = 0; a < NEN; ++a) {
      double Nd, dNd[3];
      shape<TYPE>(a, xid, Nd, dNd);
      for (int i = 0; i < 3; ++i) {
        const double xa = p.coords[(int64_t)n[a] * 3 + i] - p.coords[(int64_t)n[0] * 3 + i];
        for (int j = 0; j < 3; ++j) Jd[i][j] += xa * dNd[j];
      }
    }
    const double dd = det3(Jd);
    if (!(dd > 0.0)) atomicOr(p.status, ST_INVERTED);
    inv_transpose3(Jd, dd, Gd);
    det = (float)dd;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) G[i][j] = (float)Gd[i][j];
  }
  return det;
}

template <int TYPE>
__global__ void __launch_bounds__(128) k_small_f32(AsmArgs<float> p) {
  constexpr int NEN = Elem<TYPE>::NEN, NG = Elem<TYPE>::NG;
  __shared__ float Nt[NG][NEN], dNt[NG][NEN][3], wq[NG];
  for (int i = threadIdx.x; i < NG * NEN; i += blockDim.x) {
    const int g = i / NEN, a = i - g * NEN;
    double xi[3], w, Nd, dNd[3];
    gauss_point<TYPE>(g, xi, w);
    shape<TYPE>(a, xi, Nd, dNd);
    Nt[g][a] = (float)Nd;
    dNt[g][a][0] = (float)dNd[0];
    dNt[g][a][1] = (float)dNd[1];
    dNt[g][a][2] = (float)dNd[2];
    if (a == 0) wq[g] = (float)w;
  }
  __syncthreads();
  const int64_t items = p.n_elem * p.eq_count;
  const int64_t N = p.n_node;
  const float inv_dt = (float)(1.0 / p.dt);
  const bool t_mass = p.terms & FEA_TERM_MASS, t_conv = p.terms & FEA_TERM_CONV, t_diff = p.terms & FEA_TERM_DIFF,
             t_reac = p.terms & FEA_TERM_REAC, t_supg = p.terms & FEA_TERM_SUPG;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = it / p.eq_count;
    const int qq = (int)(it - e * p.eq_count), q = p.eq0 + qq;
    int32_t n[NEN];
#pragma unroll
    for (int a = 0; a < NEN; ++a) n[a] = __ldg(p.conn + e * NEN + a);
    float xd[NEN][3], ue[NEN][3], kn[NEN], sn[NEN], pn[NEN];
    const int64_t fo = (int64_t)q * N;
#pragma unroll
    for (int a = 0; a < NEN; ++a) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t o = (int64_t)i * N;
        xd[a][i] = (__ldg(p.xhi + o + n[a]) - __ldg(p.xhi + o + n[0])) + (__ldg(p.xlo + o + n[a]) - __ldg(p.xlo + o + n[0]));
        ue[a][i] = __ldg(p.vel + o + n[a]);
      }
      kn[a] = __ldg(p.kd + fo + n[a]);
      sn[a] = __ldg(p.sr + fo + n[a]);
      pn[a] = __ldg(p.phi + fo + n[a]);
    }
    // pass 1: the element volume (pass 2 forms the same dV again)
    float V = 0.f;
#pragma unroll 1
    for (int g = 0; g < NG; ++g) {
      float G[3][3];
      V += wq[g] * point_inverse<TYPE>(p, dNt[g], xd, n, g, G);
    }
    const float h = cbrtf(V);  // order 1
    const float c_k = 4.0f / (h * h), c_u = 2.0f / h;
    float A[NEN][NEN], b[NEN];
#pragma unroll
    for (int a = 0; a < NEN; ++a) {
      b[a] = 0.f;
#pragma unroll
      for (int c = 0; c < NEN; ++c) A[a][c] = 0.f;
    }
    // pass 2: the element matrix
#pragma unroll 1
    for (int g = 0; g < NG; ++g) {
      float G[3][3];
      const float w = wq[g] * point_inverse<TYPE>(p, dNt[g], xd, n, g, G);
      float gr[NEN][3], ug[3] = {0.f, 0.f, 0.f}, kg = 0.f, sg = 0.f, pg = 0.f;
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        const float na = Nt[g][a], d0 = dNt[g][a][0], d1 = dNt[g][a][1], d2 = dNt[g][a][2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          gr[a][i] = G[i][0] * d0 + G[i][1] * d1 + G[i][2] * d2;
          ug[i] = fmaf(na, ue[a][i], ug[i]);
        }
        kg = fmaf(na, kn[a], kg);
        sg = fmaf(na, sn[a], sg);
        pg = fmaf(na, pn[a], pg);
      }
      float ua[NEN];
#pragma unroll
      for (int a = 0; a < NEN; ++a) ua[a] = ug[0] * gr[a][0] + ug[1] * gr[a][1] + ug[2] * gr[a][2];
      const float unorm = sqrtf(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
      const float den = c_k * kg + c_u * unorm + sg;
      const float tau = den > 0.f ? 1.0f / den : 0.f;
      const float sig = (t_mass ? inv_dt : 0.f) + (t_reac ? sg : 0.f);
      const float kw = t_diff ? w * kg : 0.f;
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        const float Pa = w * Nt[g][a];
        const float Sa = t_supg ? w * tau * ua[a] : 0.f;
#pragma unroll
        for (int c = 0; c < NEN; ++c) {
          const float nc = Nt[g][c];
          float v = Pa * (sig * nc + (t_conv ? ua[c] : 0.f));
          v = fmaf(Sa, inv_dt * nc + ua[c] + sg * nc, v);
          v = fmaf(kw, gr[a][0] * gr[c][0] + gr[a][1] * gr[c][1] + gr[a][2] * gr[c][2], v);
          A[a][c] += v;
        }
        b[a] = fmaf((t_mass ? Pa : 0.f) + Sa, pg * inv_dt, b[a]);
      }
    }
    if (p.resid) {  // matrix-free: b_a - (A^e phi)_a
      const float* fq = p.phi_eval + fo;
      float ph[NEN];
#pragma unroll
      for (int c = 0; c < NEN; ++c) ph[c] = __ldg(fq + n[c]);
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        float y = b[a];
#pragma unroll
        for (int c = 0; c < NEN; ++c) y = fmaf(-A[a][c], ph[c], y);
        atomicAdd(p.resid + fo + n[a], y);
      }
    } else if (p.em) {  // gather scratch em[e][entry][q]
      constexpr int ENT = NEN * NEN + NEN;
      float* d = p.em + e * ENT * p.eq_count + qq;
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
#pragma unroll
        for (int c = 0; c < NEN; ++c) d[(a * NEN + c) * p.eq_count] = A[a][c];
        d[(NEN * NEN + a) * p.eq_count] = b[a];
      }
    } else {
      float* vq = p.values + (int64_t)q * p.nnz;
      const int32_t* pe = p.pos + e * NEN * NEN;
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
#pragma unroll
        for (int c = 0; c < NEN; ++c) atomicAdd(vq + __ldg(pe + a * NEN + c), A[a][c]);
        atomicAdd(p.rhs + fo + n[a], b[a]);
      }
    }
  }
}

template <int TYPE>
fea_status launch_t(const AsmArgs<float>& a, cudaStream_t s) {
  const int64_t items = a.n_elem * a.eq_count;
  if (items == 0) return FEA_OK;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int threads = a.batch == 64 ? 64 : 128;  // one (element, equation) item per thread
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_f32<TYPE>, threads, 0);
  const int64_t cap = (int64_t)nsm * std::max(per_sm, 1) * 8;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + threads - 1) / threads, cap));
  k_small_f32<TYPE><<<grid, threads, 0, s>>>(a);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

}  // namespace

fea_status launch_small_f32(const AsmArgs<float>& a, fea_elem_t type, cudaStream_t s) {
  switch (type) {
    case FEA_PEN6: return launch_t<FEA_PEN6>(a, s);
    case FEA_PYR5: return launch_t<FEA_PYR5>(a, s);
    default: break;
  }
  return fail(FEA_ERR_ARG, "launch_small_f32: element type %d has no thread-per-item kernel", (int)type);
}

}  // namespace fea
