// fea_internal.cuh -- shared internals of the CUDA assembly library: handle
// structs, error plumbing and the reference elements (shape functions and
// Gauss rules) as the device code evaluates them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "fea.h"

namespace fea {

// ------------------------------------------------------------------ errors

void set_error(const char* fmt, ...);
fea_status fail(fea_status st, const char* fmt, ...);
// Adds n to the process-wide count of kernels this library launched.
void count_launches(int64_t n);

#define FEA_CUDA_TRY(call)                                                                       \
  do {                                                                                           \
    cudaError_t e__ = (call);                                                                    \
    if (e__ != cudaSuccess) {                                                                    \
      return ::fea::fail(e__ == cudaErrorMemoryAllocation ? FEA_ERR_OOM : FEA_ERR_CUDA,          \
                         "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__), __FILE__,      \
                         __LINE__);                                                              \
    }                                                                                            \
  } while (0)

#define FEA_TRY(call)                         \
  do {                                        \
    fea_status s__ = (call);                  \
    if (s__ != FEA_OK) return s__;            \
  } while (0)

// Device status word bits (written by kernels, never trapped on).
enum : uint32_t {
  ST_RANGE = 1u,
  ST_DUP = 2u,
  ST_INVERTED = 4u,
  ST_ROW_TOO_LONG = 8u,
  ST_TIMEOUT = 16u,
  ST_SCHEDULE = 32u,
};
fea_status status_to_error(uint32_t bits);

// ------------------------------------------------------------------ handles

}  // namespace fea

struct fea_mesh {
  fea_elem_t type;
  int nen;
  int64_t n_node;
  int64_t n_elem;
  cudaStream_t stream;
  int device;
  double* coords;     // [n_node][3] FP64
  float* xhi;         // [3][n_node] high part of each coordinate (float)
  float* xlo;         // [3][n_node] low part: coordinate - hi, rounded to float
  int32_t* conn;      // [n_elem][nen]; several types: padded with -1 to the largest nen (pattern build)
  uint32_t* status;   // device status word
  // element blocks, one per type (a single-type mesh has one block whose conn is conn)
  struct Block {
    fea_elem_t type;
    int nen;
    int64_t e0, n_elem;  // first element (numbered block by block) and count
    int32_t* conn;       // [n_elem][nen], device
    int64_t pos0;        // offset of the block's [n_elem][nen][nen] position map
  };
  std::vector<Block> blocks;
  bool mixed;            // more than one block
  int32_t* conn_blocks;  // several types: the blocks' own connectivity, concatenated
  // fea_assemble_host: side streams and events for concurrent host<->device copies (N_COPY
  // device-to-host streams, N_IN host-to-device streams, and per-part events grown on demand)
  static constexpr int N_COPY = 4;
  static constexpr int N_IN = 2;
  cudaStream_t copy_stream[N_COPY];
  cudaEvent_t copy_event[N_COPY + 1];
  cudaStream_t in_stream[N_IN];
  std::vector<cudaEvent_t> part_events;
  bool copy_ready;
};

struct fea_rowowned_plan;  // schedules of the row-owned kernels (per element type)

struct fea_pattern {
  fea_mesh* mesh;
  int64_t nnz;
  int64_t* rowptr;     // [n_node+1]
  int32_t* colind;     // [nnz]
  int32_t* pos;        // [n_elem][nen][nen]
  int64_t* inc_ptr;    // [n_node+1] node -> element incidence
  int32_t* inc_elem;   // [nen*n_elem]
  uint8_t* inc_local;  // [nen*n_elem] local index of the node in each incident element
  fea_rowowned_plan* plan;  // may be null (row-owned path unavailable for this mesh)
  int32_t maxcol;      // longest row
  // element-matrix scratch of the gather scatter, grown on demand
  void* em;
  size_t em_bytes;
  // autotuned configuration per (equation count, term mask)
  std::map<std::pair<int, int>, fea_tuning> tuned;
  // cancellation check: the per-row flags every checked call recomputes ([n_node], shared by
  // all equation counts), and per equation count the device list of the rows the most recent
  // checked call flagged, with its device-side length
  uint8_t* cancel_flags;
  struct CancelRows {
    int32_t* rows;                // [n_node]
    unsigned long long* count;    // device
  };
  std::map<int, CancelRows> cancel;
  // device workspace for fea_assemble_host
  void* ws;
  size_t ws_bytes;
  // locality order of the elements (Tet4 meshes; null otherwise), and per element in that
  // order its 4 node ids and 16 CSR positions as one 80-byte record
  int32_t* elem_order;
  int32_t* t4_rows;
  float4* t4_node;       // Tet4, one equation: node records rebuilt every call ([N][3])
  // fea_pcg: diagonal position of every row, and the solver's vectors and scalars
  int32_t* diag;
  void* pcg_ws;
  size_t pcg_bytes;
  // fea_explicit_step: lumped mass per precision ([0] FP32, [1] FP64, [N]) and the stage workspace
  void* lumped[2];
  void* rk_ws;
  size_t rk_bytes;
  // node-major fields for the batched Hex8 kernel on the Hex8 block of a mixed mesh
  float* hex8_fnode;
  size_t hex8_fnode_bytes;
};

namespace fea {

// ------------------------------------------------------------------ reference elements
//
// Tet4: N = (1-xi-eta-zeta, xi, eta, zeta); 4-point rule whose point g has
//   barycentric weight alpha on vertex g and beta on the others,
//   alpha = (5+3 sqrt5)/20, beta = (5-sqrt5)/20, weight 1/24 (degree 2 exact).
// Hex8:  trilinear, node a = i+2j+4k <-> (xi,eta,zeta) = (+-1,+-1,+-1);
//   2x2x2 Gauss-Legendre, points +-1/sqrt3, weight 1.
// Hex27: triquadratic, node a = i+3j+9k <-> {-1,0,1}^3;
//   3x3x3 Gauss-Legendre, points 0, +-sqrt(3/5), weights 8/9, 5/9.
// Gauss points are numbered like the nodes (x fastest).
// Pen6:  prism, linear triangle (1-xi-eta, xi, eta) times linear (1-+zeta)/2; node i + 3k is
//   triangle vertex i ((0,0), (1,0), (0,1)) on zeta = -1 (k = 0) or +1 (k = 1); triangle
//   points (1/6,1/6), (2/3,1/6), (1/6,2/3) (weight 1/6) times Gauss +-1/sqrt3, point t + 3k.
// Pyr5:  pyramid |xi|,|eta| <= 1-zeta, 0 <= zeta <= 1; base corners (-1,-1), (1,-1), (1,1),
//   (-1,1) with N_a = [(1-zeta) + xa xi + ya eta + xa ya xi eta/(1-zeta)]/4, apex N_4 = zeta;
//   points of a collapsed cube: xi = r (1-zeta), eta = s (1-zeta), r, s = +-1/sqrt3, zeta the
//   3 Gauss points mapped to [0,1], weight w_zeta/2 (1-zeta)^2; point i + 2j + 4k.

template <int TYPE> struct Elem;
template <> struct Elem<FEA_TET4> { static constexpr int NEN = 4, NG = 4, ORDER = 1; };
template <> struct Elem<FEA_HEX8> { static constexpr int NEN = 8, NG = 8, ORDER = 1; };
template <> struct Elem<FEA_HEX27> { static constexpr int NEN = 27, NG = 27, ORDER = 2; };
template <> struct Elem<FEA_PEN6> { static constexpr int NEN = 6, NG = 6, ORDER = 1; };
template <> struct Elem<FEA_PYR5> { static constexpr int NEN = 5, NG = 12, ORDER = 1; };

// 1-D Lagrange basis on [-1,1]: value and derivative of function i at t.
template <int ORDER, typename T>
__host__ __device__ inline void basis1d(int i, T t, T& v, T& d) {
  if (ORDER == 1) {
    v = i == 0 ? (T(1) - t) * T(0.5) : (T(1) + t) * T(0.5);
    d = i == 0 ? T(-0.5) : T(0.5);
  } else {
    if (i == 0) { v = T(0.5) * t * (t - T(1)); d = t - T(0.5); }
    else if (i == 1) { v = T(1) - t * t; d = T(-2) * t; }
    else { v = T(0.5) * t * (t + T(1)); d = t + T(0.5); }
  }
}

// Reference coordinates and weight of Gauss point g.
template <int TYPE>
__host__ __device__ inline void gauss_point(int g, double xi[3], double& w) {
  if (TYPE == FEA_TET4) {
    const double alpha = 0.58541019662496845446;  // (5 + 3 sqrt 5) / 20
    const double beta = 0.13819660112501051518;   // (5 - sqrt 5) / 20
    xi[0] = g == 1 ? alpha : beta;
    xi[1] = g == 2 ? alpha : beta;
    xi[2] = g == 3 ? alpha : beta;
    w = 1.0 / 24.0;
  } else if (TYPE == FEA_HEX8) {
    const double p = 0.57735026918962576451;  // 1 / sqrt 3
    xi[0] = (g & 1) ? p : -p;
    xi[1] = (g & 2) ? p : -p;
    xi[2] = (g & 4) ? p : -p;
    w = 1.0;
  } else if (TYPE == FEA_PEN6) {
    const int t = g % 3;
    xi[0] = t == 1 ? 2.0 / 3.0 : 1.0 / 6.0;
    xi[1] = t == 2 ? 2.0 / 3.0 : 1.0 / 6.0;
    xi[2] = g < 3 ? -0.57735026918962576451 : 0.57735026918962576451;
    w = 1.0 / 6.0;
  } else if (TYPE == FEA_PYR5) {
    const double p = 0.57735026918962576451, q = 0.77459666924148337704;  // 1/sqrt3, sqrt(3/5)
    const int k = g >> 2;
    const double t = k == 0 ? -q : (k == 1 ? 0.0 : q), wz = k == 1 ? 8.0 / 9.0 : 5.0 / 9.0;
    const double z = 0.5 * (1.0 + t), c = 1.0 - z;
    xi[0] = ((g & 1) ? p : -p) * c;
    xi[1] = ((g & 2) ? p : -p) * c;
    xi[2] = z;
    w = 0.5 * wz * c * c;
  } else {
    const double p = 0.77459666924148337704;  // sqrt(3/5)
    const double pt[3] = {-p, 0.0, p};
    const double wt[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    int i = g % 3, j = (g / 3) % 3, k = g / 9;
    xi[0] = pt[i];
    xi[1] = pt[j];
    xi[2] = pt[k];
    w = wt[i] * wt[j] * wt[k];
  }
}

// Shape function a and its reference gradient at xi.
template <int TYPE, typename T>
__host__ __device__ inline void shape(int a, const T xi[3], T& N, T dN[3]) {
  if (TYPE == FEA_TET4) {
    if (a == 0) { N = T(1) - xi[0] - xi[1] - xi[2]; dN[0] = dN[1] = dN[2] = T(-1); }
    else { N = xi[a - 1]; dN[0] = a == 1; dN[1] = a == 2; dN[2] = a == 3; }
  } else if (TYPE == FEA_PEN6) {
    const int i = a % 3;
    const T l = a < 3 ? T(0.5) * (T(1) - xi[2]) : T(0.5) * (T(1) + xi[2]), dl = a < 3 ? T(-0.5) : T(0.5);
    const T L = i == 0 ? T(1) - xi[0] - xi[1] : xi[i - 1];
    const T dLx = i == 0 ? T(-1) : (i == 1 ? T(1) : T(0)), dLy = i == 0 ? T(-1) : (i == 2 ? T(1) : T(0));
    N = L * l;
    dN[0] = dLx * l;
    dN[1] = dLy * l;
    dN[2] = L * dl;
  } else if (TYPE == FEA_PYR5) {
    if (a == 4) {
      N = xi[2];
      dN[0] = dN[1] = T(0);
      dN[2] = T(1);
    } else {
      const T sx = (a == 1 || a == 2) ? T(1) : T(-1), sy = a >= 2 ? T(1) : T(-1), c = T(1) - xi[2];
      const T sxy = sx * sy;
      N = T(0.25) * (c + sx * xi[0] + sy * xi[1] + sxy * xi[0] * xi[1] / c);
      dN[0] = T(0.25) * (sx + sxy * xi[1] / c);
      dN[1] = T(0.25) * (sy + sxy * xi[0] / c);
      dN[2] = T(0.25) * (T(-1) + sxy * xi[0] * xi[1] / (c * c));
    }
  } else {
    constexpr int ORDER = Elem<TYPE>::ORDER, Q = ORDER + 1;
    int i = a % Q, j = (a / Q) % Q, k = a / (Q * Q);
    T lx, dx, ly, dy, lz, dz;
    basis1d<ORDER>(i, xi[0], lx, dx);
    basis1d<ORDER>(j, xi[1], ly, dy);
    basis1d<ORDER>(k, xi[2], lz, dz);
    N = lx * ly * lz;
    dN[0] = dx * ly * lz;
    dN[1] = lx * dy * lz;
    dN[2] = lx * ly * dz;
  }
}

// Corner points used by the orientation check (Tet4 and Pen6 vertices, hex corners, the
// pyramid's base corners: its rational functions are singular at the apex).
template <int TYPE>
__host__ __device__ inline void corner_point(int c, double xi[3]) {
  if (TYPE == FEA_TET4) {
    xi[0] = c == 1; xi[1] = c == 2; xi[2] = c == 3;
  } else if (TYPE == FEA_PEN6) {
    xi[0] = c % 3 == 1; xi[1] = c % 3 == 2; xi[2] = c < 3 ? -1.0 : 1.0;
  } else if (TYPE == FEA_PYR5) {
    xi[0] = (c == 1 || c == 2) ? 1.0 : -1.0; xi[1] = c >= 2 ? 1.0 : -1.0; xi[2] = 0.0;
  } else {
    xi[0] = (c & 1) ? 1.0 : -1.0;
    xi[1] = (c & 2) ? 1.0 : -1.0;
    xi[2] = (c & 4) ? 1.0 : -1.0;
  }
}
template <int TYPE> constexpr int n_corners() {
  return TYPE == FEA_TET4 ? 4 : TYPE == FEA_PEN6 ? 6 : TYPE == FEA_PYR5 ? 4 : 8;
}

template <typename T>
__host__ __device__ inline T det3(const T J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// Inverse transpose scaled by 1/det: returns G with G[i][j] = (J^-1)[j][i].
template <typename T>
__host__ __device__ inline void inv_transpose3(const T J[3][3], T det, T G[3][3]) {
  T r = T(1) / det;
  G[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * r;
  G[1][0] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
  G[2][0] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
  G[0][1] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * r;
  G[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
  G[2][1] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
  G[0][2] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * r;
  G[1][2] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
  G[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
}

// Parameters shared by the assembly kernels.
template <typename T>
struct AsmArgs {
  const int32_t* conn;
  const int32_t* elem_order = nullptr;  // Tet4 atomic kernel: element visit order (null: 0, 1, ...)
  const int32_t* t4_rows = nullptr;     // Tet4: [E][20] node ids and positions of the elements in that order
  const float4* t4_node = nullptr;      // Tet4, one equation: per-call node records [N][3] (tet4_node_records)
  const double* coords;  // [N][3]
  const float* xhi;      // [3][N]
  const float* xlo;      // [3][N]
  const int32_t* pos;
  const int64_t* rowptr;
  const int32_t* colind;
  const T* vel;    // [3][N]
  const T* kd;     // [n_eq][N]
  const T* sr;     // [n_eq][N]
  const T* phi;    // [n_eq][N]
  T* values;       // [n_eq][nnz]
  T* rhs;          // [n_eq][N]
  T* em;           // gather scatter: [n_elem][nen*nen + nen][eq_count] element matrices and RHS
                   // (written instead of the atomic adds); null otherwise
  const int64_t* inc_ptr;   // [n_node+1] node -> incident elements
  const int32_t* inc_elem;  // ascending element ids per node
  const uint8_t* inc_local; // local index of the node in each incident element
  // matrix-free residual mode (resid != null): resid[q][n] += b^e_a - (A^e phi)_a, no CSR output
  const T* phi_eval;        // [n_eq][N] the field A is applied to
  T* resid;                 // [n_eq][N]
  int64_t n_node;
  int64_t n_elem;
  int64_t nnz;
  int n_eq;        // total equations (array strides)
  int eq0;         // first equation handled by this launch
  int eq_count;    // equations handled by this launch
  int terms;
  double dt;
  double kappa_threshold;
  uint32_t* status;
  int contraction = 0;  // Hex27 element matrices: fea_contraction (resolved: never AUTO here)
  int mapping = 1;      // fea_mapping (resolved: never AUTO here)
  int batch = 0;        // elements per batch (Hex8 kernels) or threads per CTA (Tet4, Pen6, Pyr5); 0 = rule
};

// Asynchronous global -> shared copies (4 bytes, or 16 bytes with both addresses 16-byte
// aligned); a thread's copies become visible to the CTA after cp_async_wait_all and a barrier.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Launchers (defined in the kernel translation units).
fea_status launch_generic_f64(const AsmArgs<double>& a, fea_elem_t type, cudaStream_t s);
fea_status launch_generic_f32(const AsmArgs<float>& a, fea_elem_t type, cudaStream_t s);
// FP32 Tet4: one thread per (element, equation) (atomics, or the gather scratch if a.em).
fea_status launch_tet4_f32(const AsmArgs<float>& a, cudaStream_t s);
// The node records of the Tet4 kernel for the launch's single equation eq0: [N][3] float4 =
// (xhi, xlo.x), (xlo.y, xlo.z, u.x, u.y), (u.z, k, s, phi_old).
fea_status tet4_node_records(const AsmArgs<float>& a, float4* out, cudaStream_t s);
// FP32 Pen6 / Pyr5: one thread per (element, equation) item, per-point geometry in registers.
fea_status launch_small_f32(const AsmArgs<float>& a, fea_elem_t type, cudaStream_t s);
// FP32 Hex27, one CTA per element, full operator and up to 12 equations (hex27_kernel_applies).
bool hex27_kernel_applies(const AsmArgs<float>& a);
fea_status launch_hex27_f32(const AsmArgs<float>& a, cudaStream_t s);
// Morton order of the element centroids (device array of n_elem ids, owned by the caller; null
// for meshes of several types or fewer than two elements).  Waits for the mesh's stream.
fea_status element_order(const fea_mesh* m, int32_t** out);
// Per element in the given order (null: element order 0, 1, ... as element_order returns for
// meshes of fewer than 2 elements), its 4 node ids and 16 CSR positions ([E][20] int32).
fea_status tet4_rows(const fea_mesh* m, const int32_t* order, const int32_t* pos, int32_t** out);
// y_q = A_q x_q for the n_eq FP32 matrices on pattern p (overwrite or add), on stream s.
fea_status launch_spmv_f32(const fea_pattern* p, const float* values, const float* x, float* y, int n_eq,
                           bool accumulate, cudaStream_t s);
// Row gather of the element matrices in a.em into a.values / a.rhs (overwrite or add).
fea_status launch_gather_f32(const AsmArgs<float>& a, fea_elem_t type, int maxcol, bool accumulate, cudaStream_t s);
// Bytes of element-matrix scratch the gather scatter needs.
size_t gather_scratch_bytes(int64_t n_elem, int nen, int n_eq);
// Cancellation check: one FP32 pass flags rows (device list, owned by the caller afterwards,
// and its length; waits for the GPU), and the FP64 recomputation of the listed rows.
// The cancellation check of one assembly, all on the stream (no host wait, capturable): the FP32
// flag pass over every row into flags[n_node], the flagged rows compacted into rows[] with their
// number in *count, then those rows recomputed in FP64.
fea_status cancel_check_rows(const AsmArgs<float>& a, fea_elem_t type, int maxcol, uint8_t* flags, int32_t* rows,
                             unsigned long long* count, cudaStream_t s);

}  // namespace fea
