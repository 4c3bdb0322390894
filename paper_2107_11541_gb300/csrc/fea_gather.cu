// fea_gather.cu -- the row gather of the two-phase (gather) scatter.
//
// The element kernel has stored every element matrix and RHS, for all equations, in the
// scratch em[e][entry][q] (entry a*NEN+b of A^e, then NEN*NEN+a of b^e; equation fastest).
// Row r of the global system (Sec. 4.2: the CSR matrix the element contributions are
// summed into) is then the sum, over the elements e incident to node r, of row a(e, r) of
// A^e placed at the CSR positions pos[e][a][.], and of b^e_a for the RHS.
//
// One CTA owns R consecutive rows, i.e. the contiguous CSR range [rowptr[r0], rowptr[r1])
// of every equation, held in shared memory as acc[q][k - rowptr[r0]] and racc[q][r - r0].
// One warp sums one row over its incident elements in ascending element order (the order
// is fixed, so the result is bitwise reproducible): the lanes first load the element rows
// of several incident elements (NEN columns x n_eq equations plus the RHS, contiguous in
// the scratch; the local index of the row's node comes from the pattern), then add them in
// one element at a time.  Distinct rows own distinct positions, so no two warps touch the
// same word.  The CTA then writes
// each equation's range of values and RHS entries with consecutive threads on
// consecutive addresses, once.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {
namespace {

constexpr int GATHER_THREADS = 256;
constexpr size_t GATHER_SMEM_TARGET = 96 * 1024;  // two CTAs per SM when the rows allow it
constexpr size_t GATHER_SMEM_MAX = 227 * 1024;

struct GatherArgs {
  const float* em;
  const int32_t* pos;
  const int64_t* rowptr;
  const int64_t* inc_ptr;
  const int32_t* inc_elem;
  const uint8_t* inc_local;
  float* values;
  float* rhs;
  int64_t n_node, nnz;
  int n_eq, eq0, rows, accs, raccs, accumulate;
};

template <int NEN>
__global__ void __launch_bounds__(GATHER_THREADS) k_gather(GatherArgs g) {
  extern __shared__ __align__(16) float sm_gather[];
  constexpr int64_t ENTRIES = NEN * NEN + NEN;
  constexpr int K = 16;                         // element-row values in flight per lane
  float* acc = sm_gather;                       // [n_eq][accs]
  float* racc = sm_gather + g.n_eq * g.accs;    // [n_eq][raccs]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * g.rows;
  const int64_t r1 = min(g.n_node, r0 + g.rows);
  const int64_t k0 = g.rowptr[r0], k1 = g.rowptr[r1];
  const int nq = g.n_eq;
  const int per = (NEN + 1) * nq;               // values of one element row: NEN columns + RHS, all equations
  const int J = max(1, min(32, (32 * K) / per));  // elements whose values are loaded before any is added
  // this lane's values of a load round: flat index f = lane + 32 i = jj * per + b * nq + q
  // (b == NEN: the RHS entry), packed as jj | b << 8 | q << 16, or -1 past the round
  int code[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int f = lane + 32 * i, jj = f / per, rem = f - jj * per, b = rem / nq;
    code[i] = jj < J ? jj | (b << 8) | ((rem - b * nq) << 16) : -1;
  }
  for (int i = threadIdx.x; i < nq * (g.accs + g.raccs); i += GATHER_THREADS) sm_gather[i] = 0.f;
  __syncthreads();

  for (int64_t r = r0 + warp; r < r1; r += GATHER_THREADS / 32) {
    const int64_t t0 = g.inc_ptr[r];
    const int m = (int)(g.inc_ptr[r + 1] - t0);
    for (int j0 = 0; j0 < m; j0 += 32) {
      // lane l holds incident element j0 + l and the row's local index in it
      int64_t e_l = 0;
      int a_l = 0;
      if (j0 + lane < m) {
        e_l = g.inc_elem[t0 + j0 + lane];
        a_l = g.inc_local[t0 + j0 + lane];
      }
      const int mj = min(32, m - j0);
      for (int jb = 0; jb < mj; jb += J) {
        const int nj = min(J, mj - jb);
        // flat index f = jj * per + b * nq + q (b == NEN: the RHS entry): lane takes f = lane + 32 i
        float val[K];
        int dst[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
          dst[i] = -1;
          val[i] = 0.f;
          const int jj = code[i] & 0xff, b = (code[i] >> 8) & 0xff, q = code[i] >> 16;
          const int64_t e = __shfl_sync(0xffffffffu, e_l, min(jb + jj, 31));
          const int a = __shfl_sync(0xffffffffu, a_l, min(jb + jj, 31));
          if (code[i] >= 0 && jj < nj) {
            if (b < NEN) {
              val[i] = __ldcs(g.em + (e * ENTRIES + (int64_t)a * NEN + b) * nq + q);
              dst[i] = q * g.accs + (int)(g.pos[(e * NEN + a) * NEN + b] - k0);
            } else {
              val[i] = __ldcs(g.em + (e * ENTRIES + NEN * NEN + a) * nq + q);
              dst[i] = nq * g.accs + q * g.raccs + (int)(r - r0);
            }
          }
        }
        // add element by element: within one element the words are distinct
        for (int jj = 0; jj < nj; ++jj) {
#pragma unroll
          for (int i = 0; i < K; ++i)
            if (dst[i] >= 0 && (code[i] & 0xff) == jj) sm_gather[dst[i]] += val[i];
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();

  const int64_t len = k1 - k0, nr = r1 - r0;
  for (int q = 0; q < nq; ++q) {
    float* dv = g.values + (int64_t)(g.eq0 + q) * g.nnz + k0;
    const float* sv = acc + q * g.accs;
    float* dr = g.rhs + (int64_t)(g.eq0 + q) * g.n_node + r0;
    const float* sr = racc + q * g.raccs;
    if (g.accumulate) {
      for (int64_t i = threadIdx.x; i < len; i += GATHER_THREADS) dv[i] += sv[i];
      for (int64_t i = threadIdx.x; i < nr; i += GATHER_THREADS) dr[i] += sr[i];
    } else {
      for (int64_t i = threadIdx.x; i < len; i += GATHER_THREADS) __stcs(dv + i, sv[i]);
      for (int64_t i = threadIdx.x; i < nr; i += GATHER_THREADS) __stcs(dr + i, sr[i]);
    }
  }
}

template <int NEN>
fea_status launch_t(const GatherArgs& g0, int maxcol, cudaStream_t s) {
  GatherArgs g = g0;
  // rows per CTA: every row of the CTA must fit, R rows of at most maxcol entries each
  if ((int64_t)g.n_eq * (NEN + 1) > 32 * 16)
    return fail(FEA_ERR_TOO_LARGE, "gather: %d equations x %d columns exceed one load round", g.n_eq, NEN + 1);
  const size_t per_row = sizeof(float) * (size_t)g.n_eq * ((size_t)std::max(maxcol, 1) + 1);
  int rows = (int)std::max<size_t>(1, GATHER_SMEM_TARGET / per_row);
  rows = std::min(rows, 1024);
  auto smem_for = [&](int R) {
    const int accs = (R * std::max(maxcol, 1)) | 1;  // odd strides: equations of one column on distinct banks
    const int raccs = R | 1;
    return std::make_pair(sizeof(float) * (size_t)g.n_eq * (size_t)(accs + raccs), std::make_pair(accs, raccs));
  };
  auto sm = smem_for(rows);
  if (sm.first > GATHER_SMEM_MAX) return fail(FEA_ERR_TOO_LARGE, "gather: one row of %d entries x %d equations "
                                              "does not fit in shared memory", maxcol, g.n_eq);
  g.rows = rows;
  g.accs = sm.second.first;
  g.raccs = sm.second.second;
  auto kern = k_gather<NEN>;
  FEA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm.first));
  const int64_t blocks = (g.n_node + rows - 1) / rows;
  if (blocks > INT32_MAX) return fail(FEA_ERR_TOO_LARGE, "gather: too many row blocks");
  if (blocks > 0) kern<<<(unsigned)blocks, GATHER_THREADS, sm.first, s>>>(g);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

}  // namespace

size_t gather_scratch_bytes(int64_t n_elem, int nen, int n_eq) {
  return sizeof(float) * (size_t)n_elem * (size_t)(nen * nen + nen) * (size_t)n_eq;
}

fea_status launch_gather_f32(const AsmArgs<float>& a, fea_elem_t type, int maxcol, bool accumulate, cudaStream_t s) {
  GatherArgs g;
  g.em = a.em;
  g.pos = a.pos;
  g.rowptr = a.rowptr;
  g.inc_ptr = a.inc_ptr;
  g.inc_elem = a.inc_elem;
  g.inc_local = a.inc_local;
  g.values = a.values;
  g.rhs = a.rhs;
  g.n_node = a.n_node;
  g.nnz = a.nnz;
  g.n_eq = a.eq_count;
  g.eq0 = a.eq0;
  g.accumulate = accumulate ? 1 : 0;
  g.rows = g.accs = g.raccs = 0;
  switch (type) {
    case FEA_TET4: return launch_t<4>(g, maxcol, s);
    case FEA_HEX8: return launch_t<8>(g, maxcol, s);
    case FEA_HEX27: return launch_t<27>(g, maxcol, s);
    case FEA_PEN6: return launch_t<6>(g, maxcol, s);
    case FEA_PYR5: return launch_t<5>(g, maxcol, s);
  }
  return fail(FEA_ERR_ARG, "unknown element type");
}

}  // namespace fea
