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

#include "fea_generic_elem.cuh"

namespace fea {

template <typename T> __device__ __forceinline__ void atomic_add(T* p, T v) { atomicAdd(p, v); }

template <typename T, int TYPE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_generic(AsmArgs<T> p) {
  using L = GenericSmem<T, TYPE>;
  constexpr int NEN = L::NEN;
  constexpr int64_t EM_ENTRIES = NEN * NEN + NEN;
  extern __shared__ __align__(16) unsigned char sm_generic[];
  T* Nt = reinterpret_cast<T*>(sm_generic);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* S = Nt + L::TABLE + w * L::PER_WARP;
  const int32_t* node = reinterpret_cast<const int32_t*>(S + L::NODE);
  fill_shape_table<T, TYPE>(Nt);
  __syncthreads();

  const T inv_dt = T(1.0 / p.dt);
  const int64_t warps_total = (int64_t)gridDim.x * WARPS;
  for (int64_t e = (int64_t)blockIdx.x * WARPS + w; e < p.n_elem; e += warps_total) {
    const T h = warp_geometry<T, T, TYPE>(p, e, S, Nt, lane);
    for (int q = p.eq0; q < p.eq0 + p.eq_count; ++q) {
      warp_coeffs<T, T, TYPE>(p, q, S, Nt, lane, h);
      if (p.resid) {  // matrix-free: lane a forms row a of A^e and adds b_a - (A^e phi)_a
        const T* fq = p.phi_eval + (int64_t)q * p.n_node;
        for (int a = lane; a < NEN; a += 32) {
          T y = element_rhs<T, TYPE>(S, Nt, a, inv_dt, p.terms);
          for (int b = 0; b < NEN; ++b) y -= element_entry<T, TYPE>(S, Nt, a, b, inv_dt, p.terms) * fq[node[b]];
          atomic_add(p.resid + (int64_t)q * p.n_node + node[a], y);
        }
        __syncwarp();
        continue;
      }
      T* vq = p.values + (int64_t)q * p.nnz;
      const int32_t* pe = p.pos + e * NEN * NEN;
      for (int idx = lane; idx < NEN * NEN; idx += 32) {
        const T acc = element_entry<T, TYPE>(S, Nt, idx / NEN, idx % NEN, inv_dt, p.terms);
        if (p.em) p.em[((e * EM_ENTRIES) + idx) * p.eq_count + (q - p.eq0)] = acc;
        else atomic_add(vq + pe[idx], acc);
      }
      for (int a = lane; a < NEN; a += 32) {
        const T acc = element_rhs<T, TYPE>(S, Nt, a, inv_dt, p.terms);
        if (p.em) p.em[((e * EM_ENTRIES) + NEN * NEN + a) * p.eq_count + (q - p.eq0)] = acc;
        else atomic_add(p.rhs + (int64_t)q * p.n_node + node[a], acc);
      }
      __syncwarp();  // the next equation (or element) overwrites the coefficients read above
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
    case FEA_PEN6: return launch_t<T, FEA_PEN6>(a, s);
    case FEA_PYR5: return launch_t<T, FEA_PYR5>(a, s);
  }
  return fail(FEA_ERR_ARG, "unknown element type");
}

fea_status launch_generic_f64(const AsmArgs<double>& a, fea_elem_t type, cudaStream_t s) { return launch_any(a, type, s); }
fea_status launch_generic_f32(const AsmArgs<float>& a, fea_elem_t type, cudaStream_t s) {
  if (a.mapping == FEA_MAP_WARP_PER_ELEMENT) return launch_any(a, type, s);  // one warp per element
  if (type == FEA_TET4) return launch_tet4_f32(a, s);  // constant gradients: one thread per item
  if (type == FEA_PEN6 || type == FEA_PYR5) return launch_small_f32(a, type, s);  // one thread per item
  if (type == FEA_HEX27 && hex27_kernel_applies(a)) return launch_hex27_f32(a, s);  // one CTA per element
  // (the Hex27 CTA kernel covers the residual mode too)
  return launch_any(a, type, s);
}

}  // namespace fea
