// fea_cancel.cu -- the cancellation check: rows whose entries are small differences of large
// element contributions get their sums redone in FP64.
//
// A row i of equation q is flagged when, over its entries with |A_ij| > 1e-3 max_j |A_ij|,
// some entry has sum_e |A^e_ij| / |A_ij| > 1e3, or when sum_e |b^e_i| / |b_i| > 1e3.  Every
// checked assembly computes the flags afresh from its own inputs, in one FP32 pass over every
// row (a row is flagged if any equation flags it), so that rows that start to cancel when the
// fields change (a new time step, new properties) are caught.  The flagged rows are then
// recomputed after the main assembly: each incident element's row is formed and summed in
// FP64 from the same (FP32) inputs, and the rounded sums overwrite the row.  All of it is
// stream-ordered device work: the FP64 pass reads the number of flagged rows from device
// memory, so a checked assembly can be recorded in a CUDA graph.
//
// Both passes are row-centric: one warp per row walks the row's incident elements in
// ascending order, computes each element's geometry and the row of its element matrix
// (the per-warp element code of the element-parallel kernel) and adds it into the row's
// accumulators in shared memory.  An element is recomputed once per node it owns in the
// pass: the flag pass costs several times the element work of the assembly itself, which is
// why the check is an option; the FP64 pass touches only the few flagged rows.
#include <algorithm>

#include "fea_generic_elem.cuh"

namespace fea {
namespace {

constexpr float CANCEL_RATIO = 1e3f;
constexpr float CANCEL_ENTRY_CUTOFF = 1e-3f;

struct RowArgs {
  AsmArgs<float> a;
  const int32_t* rows;  // FIX: the flagged rows; FLAG: null (all rows)
  int64_t n_rows;       // FLAG: rows to walk
  const unsigned long long* n_rows_dev;  // FIX: the number of flagged rows, read on the device
  uint8_t* flags;       // FLAG: [n_node] output
  int acc_stride;       // maxcol + 1 (the RHS is column maxcol)
  int warps;
};

enum { MODE_FLAG = 0, MODE_FIX = 1 };

template <typename TC, int TYPE, int MODE>
__global__ void k_rows_recompute(RowArgs r) {
  using L = GenericSmem<TC, TYPE>;
  constexpr int NEN = L::NEN;
  const AsmArgs<float>& p = r.a;
  extern __shared__ __align__(16) unsigned char sm_rows_rc[];
  TC* Nt = reinterpret_cast<TC*>(sm_rows_rc);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_eq = p.eq_count;
  const int per_warp = L::PER_WARP + (MODE == MODE_FLAG ? 2 : 1) * r.acc_stride * n_eq;
  TC* S = Nt + L::TABLE + w * per_warp;
  TC* acc = S + L::PER_WARP;                    // [n_eq][acc_stride] signed sums
  TC* aab = acc + r.acc_stride * n_eq;          // FLAG: [n_eq][acc_stride] sums of magnitudes
  fill_shape_table<TC, TYPE>(Nt);
  __syncthreads();
  const TC inv_dt = TC(1.0 / p.dt);
  const int64_t n_rows = MODE == MODE_FIX ? (int64_t)*r.n_rows_dev : r.n_rows;

  for (int64_t i = (int64_t)blockIdx.x * r.warps + w; i < n_rows; i += (int64_t)gridDim.x * r.warps) {
    const int64_t row = MODE == MODE_FIX ? (int64_t)r.rows[i] : i;
    const int64_t k0 = p.rowptr[row];
    const int len = (int)(p.rowptr[row + 1] - k0);
    for (int j = lane; j < (MODE == MODE_FLAG ? 2 : 1) * r.acc_stride * n_eq; j += 32) acc[j] = TC(0);
    __syncwarp();
    for (int64_t t = p.inc_ptr[row]; t < p.inc_ptr[row + 1]; ++t) {
      const int64_t e = p.inc_elem[t];
      const int32_t cn = lane < NEN ? p.conn[e * NEN + lane] : -1;
      const int a = __ffs(__ballot_sync(0xffffffffu, (int64_t)cn == row)) - 1;
      const TC h = warp_geometry<TC, float, TYPE>(p, e, S, Nt, lane);
      const int32_t* pe = p.pos + (e * NEN + a) * NEN;
      for (int q = 0; q < n_eq; ++q) {
        warp_coeffs<TC, float, TYPE>(p, p.eq0 + q, S, Nt, lane, h);
        TC* aq = acc + q * r.acc_stride;
        for (int b = lane; b < NEN; b += 32) {  // distinct b: distinct columns, no two lanes on one word
          const TC v = element_entry<TC, TYPE>(S, Nt, a, b, inv_dt, p.terms);
          const int c = (int)(pe[b] - k0);
          aq[c] += v;
          if (MODE == MODE_FLAG) aab[q * r.acc_stride + c] += v < TC(0) ? -v : v;
        }
        if (lane == 0) {
          const TC v = element_rhs<TC, TYPE>(S, Nt, a, inv_dt, p.terms);
          aq[r.acc_stride - 1] += v;
          if (MODE == MODE_FLAG) aab[q * r.acc_stride + r.acc_stride - 1] += v < TC(0) ? -v : v;
        }
        __syncwarp();
      }
    }
    if (MODE == MODE_FIX) {
      for (int j = lane; j < n_eq * (len + 1); j += 32) {
        const int q = j / (len + 1), c = j - q * (len + 1);
        if (c < len) p.values[(int64_t)(p.eq0 + q) * p.nnz + k0 + c] = (float)acc[q * r.acc_stride + c];
        else p.rhs[(int64_t)(p.eq0 + q) * p.n_node + row] = (float)acc[q * r.acc_stride + r.acc_stride - 1];
      }
    } else {
      bool flag = false;
      for (int q = 0; q < n_eq; ++q) {
        const TC* aq = acc + q * r.acc_stride;
        const TC* bq = aab + q * r.acc_stride;
        TC m = TC(0);
        for (int c = lane; c < len; c += 32) m = fmax(m, fabs(aq[c]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        for (int c = lane; c < len; c += 32) {
          const TC v = fabs(aq[c]);
          if (v > TC(CANCEL_ENTRY_CUTOFF) * m && bq[c] > TC(CANCEL_RATIO) * v) flag = true;
        }
        if (lane == 0) {
          const TC v = fabs(aq[r.acc_stride - 1]), s = bq[r.acc_stride - 1];
          if (s > TC(CANCEL_RATIO) * v) flag = true;  // includes b_i = 0 with nonzero contributions
        }
      }
      flag = __any_sync(0xffffffffu, flag);
      if (lane == 0) r.flags[row] = flag ? 1 : 0;
    }
    __syncwarp();
  }
}

__global__ void k_compact_flags(const uint8_t* __restrict__ flags, int64_t n, int32_t* rows, unsigned long long* count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) rows[atomicAdd(count, 1ull)] = (int32_t)i;
}

template <typename TC, int TYPE, int MODE>
fea_status launch_rows(const RowArgs& r0, cudaStream_t s) {
  using L = GenericSmem<TC, TYPE>;
  RowArgs r = r0;
  const size_t per_warp = sizeof(TC) * ((size_t)L::PER_WARP + (MODE == MODE_FLAG ? 2 : 1) * (size_t)r.acc_stride * r.a.eq_count);
  const size_t table = sizeof(TC) * L::TABLE;
  int warps = 4;
  while (warps > 1 && table + warps * per_warp > 227 * 1024) --warps;
  const size_t smem = table + warps * per_warp;
  if (smem > 227 * 1024) return fail(FEA_ERR_TOO_LARGE, "cancellation check: a row of %d entries x %d equations does "
                                     "not fit in shared memory", r.acc_stride - 1, r.a.eq_count);
  r.warps = warps;
  auto kern = k_rows_recompute<TC, TYPE, MODE>;
  FEA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
  // FLAG walks every row; FIX at most every row (its count is known only on the device), in
  // one wave of CTAs that stride over the flagged rows
  const int64_t want = (r.n_rows + warps - 1) / warps;
  const int64_t cap = (int64_t)nsm * std::max(per_sm, 1) * (MODE == MODE_FLAG ? 8 : 1);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, cap));
  if (r.n_rows > 0) kern<<<grid, warps * 32, smem, s>>>(r);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

template <typename TC, int MODE>
fea_status launch_rows_any(const RowArgs& r, fea_elem_t type, cudaStream_t s) {
  switch (type) {
    case FEA_TET4: return launch_rows<TC, FEA_TET4, MODE>(r, s);
    case FEA_HEX8: return launch_rows<TC, FEA_HEX8, MODE>(r, s);
    case FEA_HEX27: return launch_rows<TC, FEA_HEX27, MODE>(r, s);
    case FEA_PEN6: return launch_rows<TC, FEA_PEN6, MODE>(r, s);
    case FEA_PYR5: return launch_rows<TC, FEA_PYR5, MODE>(r, s);
  }
  return fail(FEA_ERR_ARG, "unknown element type");
}

}  // namespace

fea_status cancel_check_rows(const AsmArgs<float>& a, fea_elem_t type, int maxcol, uint8_t* flags, int32_t* rows,
                             unsigned long long* count, cudaStream_t s) {
  const int64_t N = a.n_node;
  if (N == 0) return FEA_OK;
  RowArgs r;
  r.a = a;
  r.rows = nullptr;
  r.n_rows = N;
  r.n_rows_dev = nullptr;
  r.flags = flags;
  r.acc_stride = maxcol + 1;
  r.warps = 0;
  FEA_TRY((launch_rows_any<float, MODE_FLAG>(r, type, s)));
  FEA_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof *count, s));
  k_compact_flags<<<(unsigned)std::min<int64_t>((N + 255) / 256, 152 * 8), 256, 0, s>>>(flags, N, rows, count);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  r.rows = rows;
  r.n_rows_dev = count;
  r.flags = nullptr;
  return launch_rows_any<double, MODE_FIX>(r, type, s);
}

}  // namespace fea
