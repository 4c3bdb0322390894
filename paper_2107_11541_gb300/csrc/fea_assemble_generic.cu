// fea_assemble_generic.cu -- element-parallel assembly for any element type.
//
// One warp per element.  Lanes g < NG compute the Gauss-point geometry
// (Jacobian, det, inverse, physical gradients, w det J, interpolated velocity)
// once per element; then, per equation, the per-point coefficients (k, s, phi,
// tau) and the NEN x NEN element matrix (Sec. 4.2, Listing 1, generalised to the
// full Galerkin + SUPG operator) are formed with entries spread over the lanes,
// and scatter-added with atomics into the zeroed CSR values and RHS -- or, for the
// gather scatter, stored to the element-matrix scratch [e][entry][equation]
// (entries a*NEN+b, then NEN*NEN+a for the RHS) for the row gather.
//
// Used as (a) the plain FP64 path: one launch per equation (eq_count = 1), the
// geometry recomputed every launch; and (b) the portable FP32 fused path: one
// launch for all equations, geometry computed once per element.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {

template <typename T> __device__ __forceinline__ void atomic_add(T* p, T v) { atomicAdd(p, v); }

template <typename T, int TYPE>
struct GenericSmem {
  static constexpr int NEN = Elem<TYPE>::NEN, NG = Elem<TYPE>::NG;
  // offsets in units of T within one warp's region
  static constexpr int GRAD = 0;                       // [NG][NEN][3]
  static constexpr int UA = GRAD + NG * NEN * 3;       // [NG][NEN]  u_g . grad N_a
  static constexpr int DV = UA + NG * NEN;             // [NG]
  static constexpr int UG = DV + NG;                   // [NG][3]
  static constexpr int UN = UG + 3 * NG;               // [NG] |u_g|
  static constexpr int KG = UN + NG;                   // [NG]
  static constexpr int SG = KG + NG;                   // [NG]
  static constexpr int PG = SG + NG;                   // [NG]
  static constexpr int TAU = PG + NG;                  // [NG]
  static constexpr int XE = TAU + NG;                  // [NEN][3]
  static constexpr int UE = XE + 3 * NEN;              // [NEN][3]
  static constexpr int KE = UE + 3 * NEN;              // [NEN]
  static constexpr int SE = KE + NEN;
  static constexpr int PE = SE + NEN;
  static constexpr int NODE = PE + NEN;                // NEN int32 stored in T-sized slots
  static constexpr int PER_WARP = NODE + NEN;
  static constexpr int TABLE = NG * NEN;               // N[g][a], shared by the block
};

template <typename T>
__device__ __forceinline__ T coord_diff(const AsmArgs<T>& p, int32_t n, int32_t n0, int i);
template <>
__device__ __forceinline__ double coord_diff<double>(const AsmArgs<double>& p, int32_t n, int32_t n0, int i) {
  return p.coords[(int64_t)n * 3 + i] - p.coords[(int64_t)n0 * 3 + i];
}
template <>
__device__ __forceinline__ float coord_diff<float>(const AsmArgs<float>& p, int32_t n, int32_t n0, int i) {
  int64_t o = (int64_t)i * p.n_node;
  return (p.xhi[o + n] - p.xhi[o + n0]) + (p.xlo[o + n] - p.xlo[o + n0]);
}

template <typename T> __device__ __forceinline__ T cube_root(T v);
template <> __device__ __forceinline__ double cube_root<double>(double v) { return cbrt(v); }
template <> __device__ __forceinline__ float cube_root<float>(float v) { return cbrtf(v); }
template <typename T> __device__ __forceinline__ T sqrt_t(T v);
template <> __device__ __forceinline__ double sqrt_t<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float sqrt_t<float>(float v) { return sqrtf(v); }

template <typename T, int TYPE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_generic(AsmArgs<T> p) {
  using L = GenericSmem<T, TYPE>;
  constexpr int NEN = L::NEN, NG = L::NG, ORDER = Elem<TYPE>::ORDER;
  constexpr int64_t EM_ENTRIES = NEN * NEN + NEN;
  extern __shared__ __align__(16) unsigned char sm_generic[];
  T* Nt = reinterpret_cast<T*>(sm_generic);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* S = Nt + L::TABLE + w * L::PER_WARP;
  int32_t* node = reinterpret_cast<int32_t*>(S + L::NODE);

  for (int idx = threadIdx.x; idx < NG * NEN; idx += blockDim.x) {
    int g = idx / NEN, a = idx % NEN;
    double xi[3], wq, dN[3], N;
    gauss_point<TYPE>(g, xi, wq);
    shape<TYPE>(a, xi, N, dN);
    Nt[idx] = (T)N;
  }
  __syncthreads();

  const T inv_dt = T(1.0 / p.dt);
  const bool t_mass = p.terms & FEA_TERM_MASS, t_conv = p.terms & FEA_TERM_CONV, t_diff = p.terms & FEA_TERM_DIFF,
             t_reac = p.terms & FEA_TERM_REAC, t_supg = p.terms & FEA_TERM_SUPG;
  const int64_t N = p.n_node;
  const int64_t warps_total = (int64_t)gridDim.x * WARPS;

  for (int64_t e = (int64_t)blockIdx.x * WARPS + w; e < p.n_elem; e += warps_total) {
    const int32_t* ce = p.conn + e * NEN;
    const int32_t n0 = ce[0];
    for (int a = lane; a < NEN; a += 32) {
      int32_t n = ce[a];
      node[a] = n;
      for (int i = 0; i < 3; ++i) {
        S[L::XE + a * 3 + i] = coord_diff<T>(p, n, n0, i);
        S[L::UE + a * 3 + i] = p.vel[(int64_t)i * N + n];
      }
    }
    __syncwarp();
    T dv_lane = T(0);
    for (int g = lane; g < NG; g += 32) {
      double xid[3], wq;
      gauss_point<TYPE>(g, xid, wq);
      T xi[3] = {(T)xid[0], (T)xid[1], (T)xid[2]};
      T J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int a = 0; a < NEN; ++a) {
        T Na, dN[3];
        shape<TYPE>(a, xi, Na, dN);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) J[i][j] += S[L::XE + a * 3 + i] * dN[j];
      }
      T det = det3(J);
      if (!(det > T(0))) atomicOr(p.status, ST_INVERTED);
      T G[3][3];
      inv_transpose3(J, det, G);
      T ug[3] = {0, 0, 0};
      for (int a = 0; a < NEN; ++a) {
        T Na = Nt[g * NEN + a];
        for (int i = 0; i < 3; ++i) ug[i] += Na * S[L::UE + a * 3 + i];
      }
      for (int a = 0; a < NEN; ++a) {
        T Na, dN[3];
        shape<TYPE>(a, xi, Na, dN);
        T gr[3];
        for (int i = 0; i < 3; ++i) {
          gr[i] = G[i][0] * dN[0] + G[i][1] * dN[1] + G[i][2] * dN[2];
          S[L::GRAD + (g * NEN + a) * 3 + i] = gr[i];
        }
        S[L::UA + g * NEN + a] = ug[0] * gr[0] + ug[1] * gr[1] + ug[2] * gr[2];
      }
      T dv = (T)wq * det;
      S[L::DV + g] = dv;
      for (int i = 0; i < 3; ++i) S[L::UG + g * 3 + i] = ug[i];
      S[L::UN + g] = sqrt_t(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
      dv_lane += dv;
    }
    for (int o = 16; o > 0; o >>= 1) dv_lane += __shfl_xor_sync(0xffffffffu, dv_lane, o);
    const T h = cube_root(dv_lane) / T(ORDER);
    const T c_k = T(4) / (h * h), c_u = T(2) / h;
    __syncwarp();

    for (int q = p.eq0; q < p.eq0 + p.eq_count; ++q) {
      const int64_t fo = (int64_t)q * N;
      for (int a = lane; a < NEN; a += 32) {
        int32_t n = node[a];
        S[L::KE + a] = p.kd[fo + n];
        S[L::SE + a] = p.sr[fo + n];
        S[L::PE + a] = p.phi[fo + n];
      }
      __syncwarp();
      for (int g = lane; g < NG; g += 32) {
        T kg = 0, sg = 0, pg = 0;
        for (int a = 0; a < NEN; ++a) {
          T Na = Nt[g * NEN + a];
          kg += Na * S[L::KE + a];
          sg += Na * S[L::SE + a];
          pg += Na * S[L::PE + a];
        }
        T den = c_k * kg + c_u * S[L::UN + g] + sg;
        S[L::KG + g] = kg;
        S[L::SG + g] = sg;
        S[L::PG + g] = pg;
        S[L::TAU + g] = den > T(0) ? T(1) / den : T(0);
      }
      __syncwarp();
      T* vq = p.values + (int64_t)q * p.nnz;
      const int32_t* pe = p.pos + e * NEN * NEN;
      for (int idx = lane; idx < NEN * NEN; idx += 32) {
        const int a = idx / NEN, b = idx % NEN;
        T acc = T(0);
        for (int g = 0; g < NG; ++g) {
          const T Na = Nt[g * NEN + a], Nb = Nt[g * NEN + b];
          const T uaa = S[L::UA + g * NEN + a], uab = S[L::UA + g * NEN + b];
          const T sg = S[L::SG + g];
          T t = T(0);
          if (t_mass) t += Na * Nb * inv_dt;
          if (t_conv) t += Na * uab;
          if (t_diff) {
            const T* ga = S + L::GRAD + (g * NEN + a) * 3;
            const T* gb = S + L::GRAD + (g * NEN + b) * 3;
            t += S[L::KG + g] * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
          }
          if (t_reac) t += sg * Na * Nb;
          if (t_supg) t += S[L::TAU + g] * uaa * (Nb * inv_dt + uab + sg * Nb);
          acc += S[L::DV + g] * t;
        }
        if (p.em) p.em[((e * EM_ENTRIES) + idx) * p.eq_count + (q - p.eq0)] = acc;
        else atomic_add(vq + pe[idx], acc);
      }
      for (int a = lane; a < NEN; a += 32) {
        T acc = T(0);
        for (int g = 0; g < NG; ++g) {
          T test = T(0);
          if (t_mass) test += Nt[g * NEN + a];
          if (t_supg) test += S[L::TAU + g] * S[L::UA + g * NEN + a];
          acc += S[L::DV + g] * test * S[L::PG + g] * inv_dt;
        }
        if (p.em) p.em[((e * EM_ENTRIES) + NEN * NEN + a) * p.eq_count + (q - p.eq0)] = acc;
        else atomic_add(p.rhs + fo + node[a], acc);
      }
      __syncwarp();
    }
  }
}

template <typename T, int TYPE>
static fea_status launch_t(const AsmArgs<T>& a, cudaStream_t s) {
  constexpr int WARPS = 4;
  using L = GenericSmem<T, TYPE>;
  size_t smem = sizeof(T) * (L::TABLE + WARPS * L::PER_WARP);
  auto kern = k_generic<T, TYPE, WARPS>;
  FEA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t blocks = (a.n_elem + WARPS - 1) / WARPS;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  int64_t cap = (int64_t)nsm * std::max(per_sm, 1) * 4;
  unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, cap));
  kern<<<grid, WARPS * 32, smem, s>>>(a);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

template <typename T>
static fea_status launch_any(const AsmArgs<T>& a, fea_elem_t type, cudaStream_t s) {
  switch (type) {
    case FEA_TET4: return launch_t<T, FEA_TET4>(a, s);
    case FEA_HEX8: return launch_t<T, FEA_HEX8>(a, s);
    case FEA_HEX27: return launch_t<T, FEA_HEX27>(a, s);
  }
  return fail(FEA_ERR_ARG, "unknown element type");
}

fea_status launch_generic_f64(const AsmArgs<double>& a, fea_elem_t type, cudaStream_t s) { return launch_any(a, type, s); }
fea_status launch_generic_f32(const AsmArgs<float>& a, fea_elem_t type, cudaStream_t s) { return launch_any(a, type, s); }

}  // namespace fea
