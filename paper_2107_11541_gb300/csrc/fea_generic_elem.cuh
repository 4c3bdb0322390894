// fea_generic_elem.cuh -- one warp computes one element of any type (Sec. 4.2, Listing 1,
// generalised to the full Galerkin + SUPG operator): Gauss-point geometry once per element,
// then per equation the per-point coefficients and any entry of the element matrix / RHS.
//
// Shared by the element-parallel kernel (fea_assemble_generic.cu) and the row
// recomputation kernels of the cancellation check (fea_cancel.cu).  TC is the arithmetic
// type, TI the type of the nodal input arrays (FP32 inputs may be recomputed in FP64).
#pragma once
#include "fea_internal.cuh"

namespace fea {

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

// x_n - x_n0, component i: from the FP64 coordinates in FP64, from the hi/lo float split in FP32.
template <typename TC, typename TI>
__device__ __forceinline__ TC coord_diff(const AsmArgs<TI>& p, int32_t n, int32_t n0, int i) {
  if constexpr (sizeof(TC) == 8) {
    return p.coords[(int64_t)n * 3 + i] - p.coords[(int64_t)n0 * 3 + i];
  } else {
    int64_t o = (int64_t)i * p.n_node;
    return (p.xhi[o + n] - p.xhi[o + n0]) + (p.xlo[o + n] - p.xlo[o + n0]);
  }
}

template <typename T> __device__ __forceinline__ T cube_root(T v);
template <> __device__ __forceinline__ double cube_root<double>(double v) { return cbrt(v); }
template <> __device__ __forceinline__ float cube_root<float>(float v) { return cbrtf(v); }
template <typename T> __device__ __forceinline__ T sqrt_t(T v);
template <> __device__ __forceinline__ double sqrt_t<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float sqrt_t<float>(float v) { return sqrtf(v); }

// Fills the block's table Nt[g][a] = N_a(xi_g) (all threads of the block call it).
template <typename T, int TYPE>
__device__ void fill_shape_table(T* Nt) {
  constexpr int NEN = Elem<TYPE>::NEN, NG = Elem<TYPE>::NG;
  for (int idx = threadIdx.x; idx < NG * NEN; idx += blockDim.x) {
    int g = idx / NEN, a = idx % NEN;
    double xi[3], wq, dN[3], N;
    gauss_point<TYPE>(g, xi, wq);
    shape<TYPE>(a, xi, N, dN);
    Nt[idx] = (T)N;
  }
}

// Geometry of element e into the warp's region S (node ids, coordinates, velocity, per
// Gauss point gradients, u.grad N_a, dV, u_g, |u_g|).  All 32 lanes call it; returns
// h = V_e^(1/3) / order on every lane.
template <typename TC, typename TI, int TYPE>
__device__ TC warp_geometry(const AsmArgs<TI>& p, int64_t e, TC* S, const TC* Nt, int lane) {
  using L = GenericSmem<TC, TYPE>;
  constexpr int NEN = L::NEN, NG = L::NG, ORDER = Elem<TYPE>::ORDER;
  int32_t* node = reinterpret_cast<int32_t*>(S + L::NODE);
  const int64_t N = p.n_node;
  const int32_t* ce = p.conn + e * NEN;
  const int32_t n0 = ce[0];
  for (int a = lane; a < NEN; a += 32) {
    int32_t n = ce[a];
    node[a] = n;
    for (int i = 0; i < 3; ++i) {
      S[L::XE + a * 3 + i] = coord_diff<TC>(p, n, n0, i);
      S[L::UE + a * 3 + i] = (TC)p.vel[(int64_t)i * N + n];
    }
  }
  __syncwarp();
  TC dv_lane = TC(0);
  for (int g = lane; g < NG; g += 32) {
    double xid[3], wq;
    gauss_point<TYPE>(g, xid, wq);
    TC xi[3] = {(TC)xid[0], (TC)xid[1], (TC)xid[2]};
    TC J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < NEN; ++a) {
      TC Na, dN[3];
      shape<TYPE>(a, xi, Na, dN);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] += S[L::XE + a * 3 + i] * dN[j];
    }
    TC det = det3(J);
    TC G[3][3];
    inv_transpose3(J, det, G);
    if constexpr (sizeof(TC) == 4) {
      // condition estimate |J|_F |J^-1|_F (an upper bound of the 2-norm condition number); above the
      // threshold (or det <= 0 in FP32) det and
      // J^-1 are redone in FP64 from the FP64 coordinates
      TC nj = 0, ni = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          nj += J[i][j] * J[i][j];
          ni += G[i][j] * G[i][j];
        }
      if (!(det > TC(0)) || !(nj * ni <= (TC)(p.kappa_threshold * p.kappa_threshold))) {
        double Jd[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Gd[3][3];
        for (int a = 0; a < NEN; ++a) {
          double Nd, dNd[3];
          shape<TYPE>(a, xid, Nd, dNd);
          for (int i = 0; i < 3; ++i) {
            const double xa = p.coords[(int64_t)node[a] * 3 + i] - p.coords[(int64_t)n0 * 3 + i];
            for (int j = 0; j < 3; ++j) Jd[i][j] += xa * dNd[j];
          }
        }
        const double dd = det3(Jd);
        if (!(dd > 0.0)) atomicOr(p.status, ST_INVERTED);
        inv_transpose3(Jd, dd, Gd);
        det = (TC)dd;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) G[i][j] = (TC)Gd[i][j];
      }
    } else {
      if (!(det > TC(0))) atomicOr(p.status, ST_INVERTED);
    }
    TC ug[3] = {0, 0, 0};
    for (int a = 0; a < NEN; ++a) {
      TC Na = Nt[g * NEN + a];
      for (int i = 0; i < 3; ++i) ug[i] += Na * S[L::UE + a * 3 + i];
    }
    for (int a = 0; a < NEN; ++a) {
      TC Na, dN[3];
      shape<TYPE>(a, xi, Na, dN);
      TC gr[3];
      for (int i = 0; i < 3; ++i) {
        gr[i] = G[i][0] * dN[0] + G[i][1] * dN[1] + G[i][2] * dN[2];
        S[L::GRAD + (g * NEN + a) * 3 + i] = gr[i];
      }
      S[L::UA + g * NEN + a] = ug[0] * gr[0] + ug[1] * gr[1] + ug[2] * gr[2];
    }
    TC dv = (TC)wq * det;
    S[L::DV + g] = dv;
    for (int i = 0; i < 3; ++i) S[L::UG + g * 3 + i] = ug[i];
    S[L::UN + g] = sqrt_t(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
    dv_lane += dv;
  }
  for (int o = 16; o > 0; o >>= 1) dv_lane += __shfl_xor_sync(0xffffffffu, dv_lane, o);
  __syncwarp();
  return cube_root(dv_lane) / TC(ORDER);
}

// Per-equation coefficients of equation q at the Gauss points (k_g, s_g, phi_g, tau_g)
// into S.  All lanes call it; h from warp_geometry.
template <typename TC, typename TI, int TYPE>
__device__ void warp_coeffs(const AsmArgs<TI>& p, int q, TC* S, const TC* Nt, int lane, TC h) {
  using L = GenericSmem<TC, TYPE>;
  constexpr int NEN = L::NEN, NG = L::NG;
  const int32_t* node = reinterpret_cast<const int32_t*>(S + L::NODE);
  const TC c_k = TC(4) / (h * h), c_u = TC(2) / h;
  const int64_t fo = (int64_t)q * p.n_node;
  for (int a = lane; a < NEN; a += 32) {
    int32_t n = node[a];
    S[L::KE + a] = (TC)p.kd[fo + n];
    S[L::SE + a] = (TC)p.sr[fo + n];
    S[L::PE + a] = (TC)p.phi[fo + n];
  }
  __syncwarp();
  for (int g = lane; g < NG; g += 32) {
    TC kg = 0, sg = 0, pg = 0;
    for (int a = 0; a < NEN; ++a) {
      TC Na = Nt[g * NEN + a];
      kg += Na * S[L::KE + a];
      sg += Na * S[L::SE + a];
      pg += Na * S[L::PE + a];
    }
    TC den = c_k * kg + c_u * S[L::UN + g] + sg;
    S[L::KG + g] = kg;
    S[L::SG + g] = sg;
    S[L::PG + g] = pg;
    S[L::TAU + g] = den > TC(0) ? TC(1) / den : TC(0);
  }
  __syncwarp();
}

// Entry (a, b) of the element matrix of the equation whose coefficients are in S.
template <typename TC, int TYPE>
__device__ __forceinline__ TC element_entry(const TC* S, const TC* Nt, int a, int b, TC inv_dt, int terms) {
  using L = GenericSmem<TC, TYPE>;
  constexpr int NEN = L::NEN, NG = L::NG;
  const bool t_mass = terms & FEA_TERM_MASS, t_conv = terms & FEA_TERM_CONV, t_diff = terms & FEA_TERM_DIFF,
             t_reac = terms & FEA_TERM_REAC, t_supg = terms & FEA_TERM_SUPG;
  TC acc = TC(0);
  for (int g = 0; g < NG; ++g) {
    const TC Na = Nt[g * NEN + a], Nb = Nt[g * NEN + b];
    const TC uaa = S[L::UA + g * NEN + a], uab = S[L::UA + g * NEN + b];
    const TC sg = S[L::SG + g];
    TC t = TC(0);
    if (t_mass) t += Na * Nb * inv_dt;
    if (t_conv) t += Na * uab;
    if (t_diff) {
      const TC* ga = S + L::GRAD + (g * NEN + a) * 3;
      const TC* gb = S + L::GRAD + (g * NEN + b) * 3;
      t += S[L::KG + g] * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
    }
    if (t_reac) t += sg * Na * Nb;
    if (t_supg) t += S[L::TAU + g] * uaa * (Nb * inv_dt + uab + sg * Nb);
    acc += S[L::DV + g] * t;
  }
  return acc;
}

// Entry a of the element RHS of the equation whose coefficients are in S.
template <typename TC, int TYPE>
__device__ __forceinline__ TC element_rhs(const TC* S, const TC* Nt, int a, TC inv_dt, int terms) {
  using L = GenericSmem<TC, TYPE>;
  constexpr int NEN = L::NEN, NG = L::NG;
  const bool t_mass = terms & FEA_TERM_MASS, t_supg = terms & FEA_TERM_SUPG;
  TC acc = TC(0);
  for (int g = 0; g < NG; ++g) {
    TC test = TC(0);
    if (t_mass) test += Nt[g * NEN + a];
    if (t_supg) test += S[L::TAU + g] * S[L::UA + g * NEN + a];
    acc += S[L::DV + g] * test * S[L::PG + g] * inv_dt;
  }
  return acc;
}

}  // namespace fea
