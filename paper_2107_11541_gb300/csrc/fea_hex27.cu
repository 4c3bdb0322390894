// fea_hex27.cu -- FP32 Hex27 element matrices, one CTA per element (full operator, up to 12
// equations): the 27 x 27 matrices of all equations of an element share its geometry.
//
// Per Gauss point g (Sec. 4.2, Listing 1 extended to the full Galerkin + SUPG operator):
//   A_ab = sum_g P_a(g) Q_b(g) + sum_g dV k_g D_ab(g),  b_a = sum_g P_a(g) phi_g / dt,
//   P_a = dV (N_a + tau u.grad N_a),  Q_b = (1/dt + s) N_b + u.grad N_b,
//   D_ab = grad N_a . grad N_b   (symmetric, the same for every equation).
// The RHS rides along as column 27 of Q (Q_27(g) = phi_g / dt), so b_a = (P^T Q)_a,27.
// Steps, each spread over the CTA's threads with a barrier between:
//   0. the element's node data (coordinates as FP32 hi/lo, velocity, k, s, phi_old, and the
//      CSR positions for the atomic scatter) arrive in a staging buffer by cp.async, issued
//      after the previous element's contraction (connectivity earlier, with its first step);
//   1. x_a - x_0, u_g;  2. J per (g, i, j);  3. det J and J^-T per g (FP64 when badly
//      conditioned), dV;  4. grad N and u.grad N per (g, a), h = V^(1/3)/2;
//   5. k, s, phi, tau, 1/dt + s per (equation, g) and the diffusion weights dV k_g; D in
//      4 x 4 blocks (a-block <= b-block), one thread per (g, block pair);
//   6. P and Q per (equation, g, four columns);
//   7. the contractions in registers, all as one kind of task: a 16 x 4 outer product summed
//      over the 27 points, fed by 16-byte shared loads into packed FP32x2 FMAs.  A P^T Q task
//      covers 16 rows a x 4 columns b of one equation (2 x 7 tasks per equation); a
//      diffusion task covers 16 entries of D (one 4 x 4 block) x 4 equations;
//   8. the results to shared memory with 16-byte stores;
//   9. out: A = P^T Q + diffusion (the D entry of (a, b) from a table), to the gather
//      scratch em[e][entry][q], as atomic adds into the CSR values and RHS (one position
//      load per entry for all equations), or as the matrix-free residual.
//
// Tensor-core variant (TCP = 2: BF16 parts, TCP = 4: TF32 parts): steps 5b-8 become one matrix
// product per element on the fifth-generation tensor cores.  For equation q the element matrix
// is A_q = L_q R^T with the right factor shared by all equations and the left factor per
// equation (K = 135 = 27 + 27 + 81):
//   R[b][k] = [ N_b(g) | u.grad N_b(g) | grad N_b(g) (3 per g) ],
//   L_q[a][k] = [ (1/dt + s) P_a(g) | P_a(g) | dV k_g grad N_a(g) ],
// so that sum_k L_q[a][k] R[b][k] = sum_g P_a Q_b + dV k_g D_ab.  The rows (q, a) of all
// equations are stacked (m = 27 q + a) into 128-row tiles; each tile is one M = 128, N = 32
// product over K (zero padded to whole instructions) accumulated in tensor memory, columns
// 32 t .. 32 t + 31 for tile t.  Each FP32 operand is split in two parts x = x_hi + x_lo and
// three products hi hi + hi lo + lo hi are summed: with BF16 parts ("bf16x3") about 16 bits
// of each operand survive, with TF32 parts (x_hi = x with its 13 low mantissa bits cleared,
// x_lo = x - x_hi, "3xTF32") about 22.  The tiles are built and multiplied in K chunks through
// two buffers, so that one chunk is built while the tensor cores multiply the previous one.
// The RHS b_a = sum_g P_a(g) phi_g / dt is formed on the CUDA cores.
#include <algorithm>

#include <cuda_bf16.h>

#include "fea_internal.cuh"
#include "fea_tc.cuh"

namespace fea {
namespace {

constexpr int NN = 27, PAD = 28;          // nodes / Gauss points; padded row length
constexpr int NB = 7;                     // 4-wide blocks of a padded row
constexpr int NBP = NB * (NB + 1) / 2;    // 28 blocks (A <= B) of the symmetric D
constexpr int BPS = 20;                   // a block pair's 16 entries, padded: 8 consecutive pairs on distinct banks
constexpr int DSTRIDE = NBP * BPS;        // D per Gauss point
constexpr int DQS = 564;                  // one equation's diffusion sums: >= NBP * BPS, 20 mod 32
constexpr int ENT = NN * NN + NN;         // element matrix entries and RHS entries
constexpr int RQ = NN * PAD;              // one equation's results: rows a, columns b and the RHS (27)
constexpr int H27_THREADS = 256;
constexpr int H27_QMAX = 12;
static_assert(H27_QMAX * 2 * NB + NBP * (H27_QMAX / 4) <= H27_THREADS, "one task per thread");
static_assert(NBP * BPS <= DQS && DQS % 4 == 0 && H27_QMAX * DQS <= NN * DSTRIDE, "diffusion sums fit where D was");

// Tensor-core operand shapes for element size ES (2: BF16, 4: TF32).  A core-matrix row is 16
// bytes (VPC values); an instruction covers K = 2 core columns (32 bytes); K = 135 is padded to
// whole instructions; a chunk is CS instructions of one 128-row tile.
template <int ES>
struct TcShape {
  static constexpr int VPC = 16 / ES;
  static constexpr int KP = ES == 2 ? 144 : 136;
  static constexpr int KC = KP / VPC;                 // core columns: 18 or 34
  static constexpr int STEPS = KC / 2;                // instructions per tile: 9 or 17
  static constexpr int CS = ES == 2 ? 3 : 6;          // instructions per chunk
  static constexpr int NCH = (STEPS + CS - 1) / CS;   // chunks per tile: 3
  static constexpr int PLANE_B = 32 * KC * 16;        // bytes of one part of R (32 rows)
  static constexpr int PLANE_C = 128 * 2 * CS * 16;   // bytes of one part of a chunk (128 rows)
};
constexpr int TC_M = 128, TC_N = 32;                  // one MMA tile
constexpr int TC_TMEM_COLS = 128;                     // 3 tiles x 32 columns, rounded to a power of two
static_assert(TcShape<2>::NCH == 3 && TcShape<4>::NCH == 3, "three chunks per tile");

// Shared-memory layout in floats; QP = equations padded to a multiple of 4; SR staged rows
// of 27 node values (padded to 28): x hi (3), x lo (3), u (3), then k, s, phi_old per equation.
struct H27Layout {
  int QP, SR, nt, dnt, rowp, wq, sym, bpt, cn, stage, spos, xd, jg, dv, un, ug, gr, ua, kgt, pg, tau, sig, p, q, d,
      misc, total;
  int tiles, cf, opb, opa, mbar, tslot;  // tensor-core variant only
  __host__ __device__ H27Layout(int Q, int tcp = 0) {
    QP = (Q + 3) & ~3;
    SR = 9 + 3 * Q;
    int o = 0;
    nt = o;    o += NN * PAD;          // N_a(g)             [g][a]
    dnt = o;   o += NN * NN * 3;       // dN_a/dxi_j(g)      [g][a][j]
    o = (o + 1) & ~1;
    rowp = o;  o += 2 * SR;            // source array of staged row r (64-bit pointers)
    wq = o;    o += NN;                // Gauss weights
    sym = o;   o += (NN * NN + 1) / 2; // diffusion slot of (a, b) (16-bit)
    bpt = o;   o += NBP;               // (A, B) of block pair bp, packed A | B << 8 (int bits)
    cn = o;    o += 2 * PAD;           // connectivity, two buffers (int bits)
    o = (o + 3) & ~3;
    stage = o; o += 2 * SR * PAD;      // staged node data, two buffers [buf][row][a]
    spos = o;  o += 2 * NN * NN;       // staged CSR positions, two buffers (int bits)
    xd = o;    o += NN * 3;            // x_a - x_0          [a][i]
    jg = o;    o += NN * 9;            // J, then J^-T       [g][3][3]
    dv = o;    o += NN;                // w det J            [g]
    un = o;    o += NN;                // |u_g|
    ug = o;    o += NN * 3;            // u_g                [g][i]
    o = (o + 3) & ~3;                  // 16-byte rows for the float4 accesses below
    gr = o;    o += NN * 3 * PAD;      // grad N             [g][i][a]
    ua = o;    o += NN * PAD;          // u.grad N           [g][a]
    kgt = o;   o += NN * QP;           // dV k_g             [g][q]
    pg = o;    o += Q * NN;            // phi_g              [q][g]
    tau = o;   o += Q * NN;
    sig = o;   o += Q * NN;            // 1/dt + s_g
    o = (o + 3) & ~3;
    tiles = cf = opb = opa = mbar = tslot = 0;
    if (tcp == 0) {
      p = o;     o += Q * NN * PAD;      // P [q][g][a]; after the contractions P^T Q [q][a][b], b = 27: RHS
      q = o;     o += Q * NN * PAD;      // Q [q][g][b]
      d = o;     o += NN * DSTRIDE;      // D [g][pair][BPS]; after the contractions the diffusion sums [q][pair][BPS]
      misc = o;  o += 4;                 // h
      total = o;
      return;
    }
    tiles = (Q * NN + TC_M - 1) / TC_M;
    cf = o;    o += 4 * Q * NN;        // per (q, g): dV sigma, dV sigma tau, dV, dV tau (16-byte aligned)
    misc = o;  o += 4;
    mbar = o;  o += 4;                 // two 8-byte mbarriers (offset even: 8-byte aligned)
    tslot = o; o += 4;                 // tensor-memory base address
    o = (o + 31) & ~31;                // 128-byte aligned operands
    const int plane_b = tcp == 2 ? TcShape<2>::PLANE_B : TcShape<4>::PLANE_B;
    const int plane_c = tcp == 2 ? TcShape<2>::PLANE_C : TcShape<4>::PLANE_C;
    opb = o;   o += 2 * plane_b / 4;   // R, two parts
    opa = o;   o += 2 * 2 * plane_c / 4;  // two chunk buffers of two parts; the results [q][a][PAD] reuse them
    p = q = d = opa;
    total = o;
  }
};
static_assert(H27_QMAX * NN * PAD * 4 <= 2 * 2 * TcShape<2>::PLANE_C, "the results fit in the chunk buffers");

// Block pair (A <= B) of the 7 x 7 block grid, row-major upper triangle.
__host__ __device__ inline int block_pair(int A, int B) { return A * NB - A * (A - 1) / 2 + (B - A); }

// Slot of grad N_a . grad N_b among one equation's diffusion sums: entry r * 4 + c of block
// pair (A, B) is (4A + r, 4B + c), and pair bp starts at bp * BPS.
__host__ __device__ inline int d_slot(int a, int b) {
  if (a / 4 > b / 4) {
    const int t = a;
    a = b;
    b = t;
  }
  return block_pair(a / 4, b / 4) * BPS + (a & 3) * 4 + (b & 3);
}

// Entry k of the shared right factor for node b: [N_b(g) | u.grad N_b(g) | grad N_b(g)], zero
// in the padding (b >= 27 or k >= 135).
__device__ __forceinline__ float tc_rval(const float* sm, const H27Layout& L, int b, int k) {
  if (b >= NN) return 0.f;
  if (k < NN) return sm[L.nt + k * PAD + b];
  if (k < 2 * NN) return sm[L.ua + (k - NN) * PAD + b];
  if (k < 5 * NN) {
    const int j = k - 2 * NN, g = j / 3, i = j - 3 * g;
    return sm[L.gr + (g * 3 + i) * PAD + b];
  }
  return 0.f;
}

// Entry k of equation q's left factor for node a: [(1/dt + s) P_a(g) | P_a(g) | dV k_g grad N_a(g)],
// P_a = dV (N_a + tau u.grad N_a), from the coefficients cf[q][g] = (dV sigma, dV sigma tau, dV, dV tau).
__device__ __forceinline__ float tc_lval(const float* sm, const H27Layout& L, int q, int a, int k) {
  if (k < 2 * NN) {
    const int g = k < NN ? k : k - NN;
    const float4 c = reinterpret_cast<const float4*>(sm + L.cf)[q * NN + g];
    const float n = sm[L.nt + g * PAD + a], u = sm[L.ua + g * PAD + a];
    return k < NN ? fmaf(c.y, u, c.x * n) : fmaf(c.w, u, c.z * n);
  }
  if (k < 5 * NN) {
    const int j = k - 2 * NN, g = j / 3, i = j - 3 * g;
    return sm[L.kgt + g * L.QP + q] * sm[L.gr + (g * 3 + i) * PAD + a];
  }
  return 0.f;
}

// One 16-byte core-matrix row of VPC consecutive values in two parts x = hi + lo: BF16 (hi the
// rounded value, lo the rounded remainder) or TF32 (hi with the 13 low mantissa bits cleared,
// lo = x - hi, exact).
template <int ES>
__device__ __forceinline__ void split_row(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
  if constexpr (ES == 2) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      const __nv_bfloat162 r = __floats2bfloat162_rn(v[2 * j] - __low2float(b), v[2 * j + 1] - __high2float(b));
      h[j] = *reinterpret_cast<const uint32_t*>(&b);
      l[j] = *reinterpret_cast<const uint32_t*>(&r);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = __float_as_uint(v[j]) & 0xFFFFE000u;
      l[j] = __float_as_uint(v[j] - __uint_as_float(h[j]));
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

template <bool EM, int TCP>
__global__ void __launch_bounds__(H27_THREADS, 1) k_hex27(AsmArgs<float> p) {
  extern __shared__ __align__(128) float sm27[];
  const int Q = p.eq_count;
  const H27Layout L(Q, TCP);
  const int tid = threadIdx.x;
  const int64_t N = p.n_node;
  const float inv_dt = (float)(1.0 / p.dt);
  const bool stage_pos = !EM && p.resid == nullptr;  // the atomic scatter reads pos[e]
  const int n_pq = Q * 2 * NB;                   // (q, 16-row block, 4-column block)
  const int n_task = n_pq + NBP * (L.QP / 4);    // + (block pair, 4 equations)
  uint16_t* symt = reinterpret_cast<uint16_t*>(sm27 + L.sym);
  int* bpt = reinterpret_cast<int*>(sm27 + L.bpt);
  const float** rowp = reinterpret_cast<const float**>(sm27 + L.rowp);

  // constant tables
  for (int i = tid; i < NN * PAD; i += H27_THREADS) {
    const int g = i / PAD, a = i - g * PAD;
    float v = 0.f;
    if (a < NN) {
      double xi[3], w, Nd, dN[3];
      gauss_point<FEA_HEX27>(g, xi, w);
      shape<FEA_HEX27>(a, xi, Nd, dN);
      v = (float)Nd;
      sm27[L.dnt + (g * NN + a) * 3 + 0] = (float)dN[0];
      sm27[L.dnt + (g * NN + a) * 3 + 1] = (float)dN[1];
      sm27[L.dnt + (g * NN + a) * 3 + 2] = (float)dN[2];
      if (a == 0) sm27[L.wq + g] = (float)w;
    }
    sm27[L.nt + i] = v;
  }
  for (int i = tid; i < NN * NN; i += H27_THREADS) symt[i] = (uint16_t)d_slot(i / NN, i - (i / NN) * NN);
  if (tid < NB)
    for (int B = tid; B < NB; ++B) bpt[block_pair(tid, B)] = tid | (B << 8);
  for (int r = tid; r < L.SR; r += H27_THREADS) {
    const float* src;
    if (r < 3) src = p.xhi + (int64_t)r * N;
    else if (r < 6) src = p.xlo + (int64_t)(r - 3) * N;
    else if (r < 9) src = p.vel + (int64_t)(r - 6) * N;
    else {
      const int f = (r - 9) / Q, q = (r - 9) - f * Q;
      src = (f == 0 ? p.kd : f == 1 ? p.sr : p.phi) + (int64_t)(p.eq0 + q) * N;
    }
    rowp[r] = src;
  }
  for (int r = tid; r < 2 * L.SR; r += H27_THREADS) sm27[L.stage + r * PAD + NN] = 0.f;  // padded column
  // the first element's connectivity (plain loads) and node data (cp.async)
  if (blockIdx.x < p.n_elem && tid < NN)
    reinterpret_cast<int*>(sm27 + L.cn)[tid] = p.conn[(int64_t)blockIdx.x * NN + tid];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm27 + L.mbar);
  uint32_t tmem = 0, phase0 = 0, phase1 = 0;
  if constexpr (TCP > 0) {
    if (tid == 0) {
      tc::mbar_init(mbar, 1);
      tc::mbar_init(mbar + 1, 1);
    }
    if (tid < 32) tc::tmem_alloc(reinterpret_cast<uint32_t*>(sm27 + L.tslot), TC_TMEM_COLS);
    tc::fence_before_sync();
  }
  __syncthreads();
  if constexpr (TCP > 0) {
    tc::fence_after_sync();
    tmem = *reinterpret_cast<const uint32_t*>(sm27 + L.tslot);
  }
  // staged node data of element e into buffer buf (connectivity already in cn[buf])
  auto stage_issue = [&](int64_t e, int buf) {
    const int* cb = reinterpret_cast<const int*>(sm27 + L.cn + buf * PAD);
    float* dst = sm27 + L.stage + buf * L.SR * PAD;
    for (int i = tid; i < L.SR * NN; i += H27_THREADS) {
      const int r = i / NN, a = i - r * NN;
      cp_async4(dst + r * PAD + a, rowp[r] + cb[a]);
    }
    if (stage_pos) {
      const int32_t* pe = p.pos + e * (NN * NN);
      int32_t* dp = reinterpret_cast<int32_t*>(sm27 + L.spos + buf * NN * NN);
      for (int i = tid; i < NN * NN; i += H27_THREADS) cp_async4(dp + i, pe + i);
    }
    cp_async_commit();
  };
  if (blockIdx.x < p.n_elem) stage_issue(blockIdx.x, 0);

  int cur = 0;
  for (int64_t e = blockIdx.x; e < p.n_elem; e += gridDim.x, cur ^= 1) {
    const int64_t en = e + gridDim.x;
    const int* ce = reinterpret_cast<const int*>(sm27 + L.cn + cur * PAD);
    const float* st = sm27 + L.stage + cur * L.SR * PAD;  // [row][a]
    cp_async_wait_all();
    __syncthreads();  // element e's staged data is visible; the previous element's results are written
    if (en < p.n_elem && tid < NN) cp_async4(sm27 + L.cn + (cur ^ 1) * PAD + tid, p.conn + en * NN + tid);
    cp_async_commit();
    // 1. x_a - x_0 (hi/lo split), u_g = sum_a N_a(g) u_a
    if (tid < NN * 3) {
      const int a = tid / 3, c = tid - a * 3;
      sm27[L.xd + tid] = (st[c * PAD + a] - st[c * PAD]) + (st[(3 + c) * PAD + a] - st[(3 + c) * PAD]);
    } else if (tid >= 128 && tid < 128 + NN * 3) {
      const int i = tid - 128, g = i / 3, c = i - g * 3;
      const float* u = st + (6 + c) * PAD;
      float s = 0.f;
      for (int a = 0; a < NN; ++a) s = fmaf(sm27[L.nt + g * PAD + a], u[a], s);
      sm27[L.ug + i] = s;
    }
    __syncthreads();
    // 2. J_gij = sum_a (x_a - x_0)_i dN_a/dxi_j(g)
    for (int i = tid; i < NN * 9; i += H27_THREADS) {
      const int g = i / 9, ij = i - g * 9, ii = ij / 3, j = ij - ii * 3;
      float s = 0.f;
      for (int a = 0; a < NN; ++a) s = fmaf(sm27[L.xd + a * 3 + ii], sm27[L.dnt + (g * NN + a) * 3 + j], s);
      sm27[L.jg + i] = s;
    }
    __syncthreads();
    // 3. det, J^-T (FP64 above the condition threshold), dV, |u_g|
    if (tid < NN) {
      const int g = tid;
      float J[3][3], G[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = sm27[L.jg + g * 9 + i * 3 + j];
      float det = det3(J);
      inv_transpose3(J, det, G);
      float nj = 0.f, ni = 0.f;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          nj = fmaf(J[i][j], J[i][j], nj);
          ni = fmaf(G[i][j], G[i][j], ni);
        }
      if (!(det > 0.f) || !(nj * ni <= (float)(p.kappa_threshold * p.kappa_threshold))) {
        double xid[3], w;
        gauss_point<FEA_HEX27>(g, xid, w);
        double Jd[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Gd[3][3];
        for (int a = 0; a < NN; ++a) {
          double Nd, dNd[3];
          shape<FEA_HEX27>(a, xid, Nd, dNd);
          for (int i = 0; i < 3; ++i) {
            const double xa = p.coords[(int64_t)ce[a] * 3 + i] - p.coords[(int64_t)ce[0] * 3 + i];
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
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) sm27[L.jg + g * 9 + i * 3 + j] = G[i][j];
      sm27[L.dv + g] = sm27[L.wq + g] * det;
      const float* u = sm27 + L.ug + g * 3;
      sm27[L.un + g] = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
    __syncthreads();
    // 4. grad N_a(g) = J^-T grad_xi N_a and u_g . grad N_a(g) per (g, a); padded column a = 27 is zero
    for (int i = tid; i < NN * PAD; i += H27_THREADS) {
      const int g = i / PAD, a = i - g * PAD;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f;
      if (a < NN) {
        const float* G = sm27 + L.jg + g * 9;
        const float* dn = sm27 + L.dnt + (g * NN + a) * 3;
        const float d0 = dn[0], d1 = dn[1], d2 = dn[2];
        g0 = G[0] * d0 + G[1] * d1 + G[2] * d2;
        g1 = G[3] * d0 + G[4] * d1 + G[5] * d2;
        g2 = G[6] * d0 + G[7] * d1 + G[8] * d2;
      }
      float* gg = sm27 + L.gr + g * 3 * PAD + a;
      gg[0] = g0;
      gg[PAD] = g1;
      gg[2 * PAD] = g2;
      const float* u = sm27 + L.ug + g * 3;
      sm27[L.ua + i] = u[0] * g0 + u[1] * g1 + u[2] * g2;
    }
    if (tid == H27_THREADS - 1) {
      float v = 0.f;
      for (int g = 0; g < NN; ++g) v += sm27[L.dv + g];
      sm27[L.misc] = cbrtf(v) * 0.5f;  // h = V^(1/3) / 2
    }
    __syncthreads();
    // 5a. k, s, phi, tau, 1/dt + s per (q, g) (padded node columns are zero); the weight dV k_g
    {
      const float h = sm27[L.misc], c_k = 4.0f / (h * h), c_u = 2.0f / h;
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, g = i - q * NN;
        const float4* n4 = reinterpret_cast<const float4*>(sm27 + L.nt + g * PAD);
        const float4* k4 = reinterpret_cast<const float4*>(st + (9 + q) * PAD);
        const float4* s4 = reinterpret_cast<const float4*>(st + (9 + Q + q) * PAD);
        const float4* p4 = reinterpret_cast<const float4*>(st + (9 + 2 * Q + q) * PAD);
        float kg = 0.f, sg = 0.f, pg = 0.f;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          const float4 n = n4[c], k = k4[c], sv = s4[c], ph = p4[c];
          kg = fmaf(n.x, k.x, kg);
          kg = fmaf(n.y, k.y, kg);
          kg = fmaf(n.z, k.z, kg);
          kg = fmaf(n.w, k.w, kg);
          sg = fmaf(n.x, sv.x, sg);
          sg = fmaf(n.y, sv.y, sg);
          sg = fmaf(n.z, sv.z, sg);
          sg = fmaf(n.w, sv.w, sg);
          pg = fmaf(n.x, ph.x, pg);
          pg = fmaf(n.y, ph.y, pg);
          pg = fmaf(n.z, ph.z, pg);
          pg = fmaf(n.w, ph.w, pg);
        }
        const float den = c_k * kg + c_u * sm27[L.un + g] + sg;
        const float dvg = sm27[L.dv + g], tg = den > 0.f ? 1.0f / den : 0.f, sgm = inv_dt + sg;
        sm27[L.kgt + g * L.QP + q] = dvg * kg;
        sm27[L.pg + i] = pg;
        sm27[L.tau + i] = tg;
        sm27[L.sig + i] = sgm;
        if (TCP) reinterpret_cast<float4*>(sm27 + L.cf)[i] = make_float4(dvg * sgm, dvg * sgm * tg, dvg, dvg * tg);
      }
      for (int i = tid; i < NN * (L.QP - Q); i += H27_THREADS) {  // padded equations of k_g: zero
        const int g = i / (L.QP - Q), q = Q + (i - g * (L.QP - Q));
        sm27[L.kgt + g * L.QP + q] = 0.f;
      }
    }
    // 5b. D_ab(g) = grad N_a . grad N_b in 4 x 4 blocks (A <= B), one thread per (g, block pair)
    for (int i = tid; i < (TCP ? 0 : NN * NBP); i += H27_THREADS) {
      const int g = i / NBP, bp = i - g * NBP, AB = bpt[bp], A = AB & 0xff, B = AB >> 8;
      const float* gg = sm27 + L.gr + g * 3 * PAD;
      float4 xa[3], xb[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xa[c] = *reinterpret_cast<const float4*>(gg + c * PAD + 4 * A);
        xb[c] = *reinterpret_cast<const float4*>(gg + c * PAD + 4 * B);
      }
      float4* dst = reinterpret_cast<float4*>(sm27 + L.d + g * DSTRIDE + bp * BPS);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float a0 = (&xa[0].x)[r], a1 = (&xa[1].x)[r], a2 = (&xa[2].x)[r];
        float4 v;
        v.x = a0 * xb[0].x + a1 * xb[1].x + a2 * xb[2].x;
        v.y = a0 * xb[0].y + a1 * xb[1].y + a2 * xb[2].y;
        v.z = a0 * xb[0].z + a1 * xb[1].z + a2 * xb[2].z;
        v.w = a0 * xb[0].w + a1 * xb[1].w + a2 * xb[2].w;
        dst[r] = v;
      }
    }
    __syncthreads();
    if constexpr (TCP > 0) {
      using S = TcShape<TCP>;
      constexpr int VPC = S::VPC;
      // TC 1. the shared right factor R, one 16-byte core row (node b, VPC consecutive k) per item
      unsigned char* opb = reinterpret_cast<unsigned char*>(sm27 + L.opb);
      for (int it = tid; it < TC_N * S::KC; it += H27_THREADS) {
        const int b = it & (TC_N - 1), kc = it / TC_N;
        float v[VPC];
#pragma unroll
        for (int j = 0; j < VPC; ++j) v[j] = tc_rval(sm27, L, b, kc * VPC + j);
        uint4 hi, lo;
        split_row<TCP>(v, hi, lo);
        unsigned char* dst = opb + ((b >> 3) * S::KC + kc) * 128 + (b & 7) * 16;
        *reinterpret_cast<uint4*>(dst) = hi;
        *reinterpret_cast<uint4*>(dst + S::PLANE_B) = lo;
      }
      cp_async_wait_all();  // the next element's connectivity
      __syncthreads();
      if (en < p.n_elem) stage_issue(en, cur ^ 1);  // the next element's node data starts to arrive
      // TC 2. chunks (tile t, instructions s0 .. s0 + CS - 1): built into buffer c & 1 while the
      // tensor cores multiply the chunk before; one thread issues each chunk's products
      constexpr int PA[3] = {0, 0, 1}, PB[3] = {0, 1, 0};  // parts: hi hi, hi lo, lo hi
      bool ok = true;
      int pend0 = 0, pend1 = 0;
      auto wait_buf = [&](int b) {
        uint32_t& ph = b ? phase1 : phase0;
        ok = tc::mbar_wait(mbar + b, ph, 1 << 22) && ok;
        ph ^= 1u;
      };
      unsigned char* opa = reinterpret_cast<unsigned char*>(sm27 + L.opa);
      for (int c = 0; c < L.tiles * S::NCH; ++c) {
        const int t = c / S::NCH, j = c - t * S::NCH, bsel = c & 1;
        const int s0 = j * S::CS, ns = min(S::CS, S::STEPS - s0);
        if (bsel ? pend1 : pend0) {  // the products that read this buffer must have finished
          wait_buf(bsel);
          (bsel ? pend1 : pend0) = 0;
        }
        unsigned char* buf = opa + bsel * 2 * S::PLANE_C;
        for (int it = tid; it < TC_M * 2 * ns; it += H27_THREADS) {
          const int r = it & (TC_M - 1), lc = it / TC_M, m = t * TC_M + r, q = m / NN, a = m - q * NN;
          const int k0 = (2 * s0 + lc) * VPC;
          float v[VPC];
#pragma unroll
          for (int jj = 0; jj < VPC; ++jj) v[jj] = q < Q ? tc_lval(sm27, L, q, a, k0 + jj) : 0.f;
          uint4 hi, lo;
          split_row<TCP>(v, hi, lo);
          unsigned char* dst = buf + ((r >> 3) * 2 * S::CS + lc) * 128 + (r & 7) * 16;
          *reinterpret_cast<uint4*>(dst) = hi;
          *reinterpret_cast<uint4*>(dst + S::PLANE_C) = lo;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_addr(buf), b0 = tc::smem_addr(opb);
          for (int ls = 0; ls < ns; ++ls)
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
              const uint64_t da = tc::smem_desc(a0 + PA[pr] * S::PLANE_C + ls * 256, 128, 2 * S::CS * 128);
              const uint64_t db = tc::smem_desc(b0 + PB[pr] * S::PLANE_B + (s0 + ls) * 256, 128, S::KC * 128);
              const uint32_t acc = (j > 0 || ls > 0 || pr > 0) ? 1u : 0u;
              if constexpr (TCP == 2) tc::mma_bf16(tmem + TC_N * t, da, db, tc::idesc_bf16_f32(TC_M, TC_N), acc);
              else tc::mma_tf32(tmem + TC_N * t, da, db, tc::idesc_tf32_f32(TC_M, TC_N), acc);
            }
          tc::commit(mbar + bsel);
        }
        (bsel ? pend1 : pend0) = 1;
      }
      if (pend0) wait_buf(0);
      if (pend1) wait_buf(1);
      tc::fence_after_sync();
      if (__syncthreads_or(!ok)) {  // a product never completed: report it and stop
        if (tid == 0) atomicOr(p.status, ST_TIMEOUT);
        break;
      }
      // TC 3. the accumulators to shared memory as [q][a][PAD] (m = 27 q + a): warp w reads the
      // lanes 32 (w % 4) .. + 31 of every tile, columns 16 (w / 4) .. + 15
      float* R = sm27 + L.opa;
      {
        const int w = tid >> 5, lq = w & 3, ch = w >> 2;
        for (int t = 0; t < L.tiles; ++t) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(TC_N * t + 16 * ch), v);
          const int m = t * TC_M + 32 * lq + (tid & 31);
          if (m < Q * NN) {
            float* dst = R + m * PAD + 16 * ch;
            reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
            if (ch == 0) {
              reinterpret_cast<float4*>(dst)[2] = make_float4(v[8], v[9], v[10], v[11]);
              reinterpret_cast<float4*>(dst)[3] = make_float4(v[12], v[13], v[14], v[15]);
            } else {  // columns 24 .. 26; 27 .. 31 are padding (column 27 takes the RHS)
              dst[8] = v[8];
              dst[9] = v[9];
              dst[10] = v[10];
            }
          }
        }
      }
      tc::fence_before_sync();
      // TC 4. the RHS b_a = sum_g P_a(g) phi_g / dt per (q, a), into column 27
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, a = i - q * NN;
        float sum = 0.f;
        for (int g = 0; g < NN; ++g) {
          const int qg = q * NN + g;
          const float P = sm27[L.dv + g] * fmaf(sm27[L.tau + qg], sm27[L.ua + g * PAD + a], sm27[L.nt + g * PAD + a]);
          sum = fmaf(P, sm27[L.pg + qg] * inv_dt, sum);
        }
        R[i * PAD + NN] = sum;
      }
      __syncthreads();
    } else {
    // 6. P and Q per (q, g, four columns a); the padded column: P 0, Q phi_g / dt (the RHS)
    for (int i = tid; i < Q * NN * NB; i += H27_THREADS) {
      const int qg = i / NB, c4 = (i - qg * NB) * 4, g = qg - (qg / NN) * NN;
      const float4 na = *reinterpret_cast<const float4*>(sm27 + L.nt + g * PAD + c4);
      const float4 ua = *reinterpret_cast<const float4*>(sm27 + L.ua + g * PAD + c4);
      const float dvg = sm27[L.dv + g], t = sm27[L.tau + qg], sgm = sm27[L.sig + qg];
      float4 pv, qv;
      pv.x = dvg * fmaf(t, ua.x, na.x);
      pv.y = dvg * fmaf(t, ua.y, na.y);
      pv.z = dvg * fmaf(t, ua.z, na.z);
      pv.w = dvg * fmaf(t, ua.w, na.w);
      qv.x = fmaf(sgm, na.x, ua.x);
      qv.y = fmaf(sgm, na.y, ua.y);
      qv.z = fmaf(sgm, na.z, ua.z);
      qv.w = c4 == PAD - 4 ? sm27[L.pg + qg] * inv_dt : fmaf(sgm, na.w, ua.w);
      *reinterpret_cast<float4*>(sm27 + L.p + qg * PAD + c4) = pv;
      *reinterpret_cast<float4*>(sm27 + L.q + qg * PAD + c4) = qv;
    }
    cp_async_wait_all();  // the next element's connectivity
    __syncthreads();
    // 7. the contractions, acc[r][c] = sum_g x_r(g) y_c(g)
    const int task = tid;
    const float* X;  // 16 consecutive values per point, stride sx
    const float* Y;  // 4 consecutive values per point, stride sy
    int sx, sy;
    if (task < n_pq) {  // P^T Q: rows 16 rb .. 16 rb + 15 (rows past 26 are discarded), columns 4 cb ..
      const int tq = task / (2 * NB), rem = task - tq * 2 * NB, rb = rem / NB, cb = rem - rb * NB;
      X = sm27 + L.p + tq * NN * PAD + rb * 16;
      Y = sm27 + L.q + tq * NN * PAD + cb * 4;
      sx = sy = PAD;
    } else {  // diffusion: the 16 entries of block pair bp x equations 4 qb ..
      const int t = min(task, n_task - 1) - n_pq, qb = t / NBP, bp = t - qb * NBP;
      X = sm27 + L.d + bp * BPS;
      Y = sm27 + L.kgt + qb * 4;
      sx = DSTRIDE;
      sy = L.QP;
    }
    float2 acc2[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc2[i] = make_float2(0.f, 0.f);
    if (task < n_task) {
#pragma unroll 3
      for (int g = 0; g < NN; ++g) {
        const float4* xg = reinterpret_cast<const float4*>(X + g * sx);
        const float4 x0 = xg[0], x1 = xg[1], x2 = xg[2], x3 = xg[3];
        const float4 y = *reinterpret_cast<const float4*>(Y + g * sy);
        const float xr[16] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w,
                              x2.x, x2.y, x2.z, x2.w, x3.x, x3.y, x3.z, x3.w};
        const float2 y01 = make_float2(y.x, y.y), y23 = make_float2(y.z, y.w);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          acc2[2 * r] = __ffma2_rn(make_float2(xr[r], xr[r]), y01, acc2[2 * r]);
          acc2[2 * r + 1] = __ffma2_rn(make_float2(xr[r], xr[r]), y23, acc2[2 * r + 1]);
        }
      }
    }
    __syncthreads();  // P, Q and D are no longer read: P^T Q goes where P was, the diffusion sums where D was
    if (en < p.n_elem) stage_issue(en, cur ^ 1);  // the next element's node data starts to arrive
    float* R = sm27 + L.p;   // [q][a][PAD]: P^T Q, column 27 the RHS
    float* Dq = sm27 + L.d;  // [q][DQS]: sum_g dV k_g grad N_a . grad N_b at d_slot(a, b)
    if (task < n_pq) {
      const int tq = task / (2 * NB), rem = task - tq * 2 * NB, rb = rem / NB, cb = rem - rb * NB;
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (rb * 16 + r < NN)
          *reinterpret_cast<float4*>(R + tq * RQ + (rb * 16 + r) * PAD + cb * 4) =
              make_float4(acc2[2 * r].x, acc2[2 * r].y, acc2[2 * r + 1].x, acc2[2 * r + 1].y);
    } else if (task < n_task) {
      const int t = task - n_pq, qb = t / NBP, bp = t - qb * NBP;
      float* d0 = Dq + qb * 4 * DQS + bp * BPS;
#pragma unroll
      for (int r = 0; r < 16; r += 4) {
        *reinterpret_cast<float4*>(d0 + r) = make_float4(acc2[2 * r].x, acc2[2 * r + 2].x, acc2[2 * r + 4].x, acc2[2 * r + 6].x);
        *reinterpret_cast<float4*>(d0 + DQS + r) =
            make_float4(acc2[2 * r].y, acc2[2 * r + 2].y, acc2[2 * r + 4].y, acc2[2 * r + 6].y);
        *reinterpret_cast<float4*>(d0 + 2 * DQS + r) =
            make_float4(acc2[2 * r + 1].x, acc2[2 * r + 3].x, acc2[2 * r + 5].x, acc2[2 * r + 7].x);
        *reinterpret_cast<float4*>(d0 + 3 * DQS + r) =
            make_float4(acc2[2 * r + 1].y, acc2[2 * r + 3].y, acc2[2 * r + 5].y, acc2[2 * r + 7].y);
      }
    }
    __syncthreads();
    }  // CUDA-core contraction
    float* R = sm27 + L.p;   // [q][a][PAD]: the element matrices (CUDA cores: P^T Q only), column 27 the RHS
    const float* Dq = sm27 + L.d;  // CUDA cores: the diffusion sums [q][DQS]
    // 9. out
    if (p.resid) {  // matrix-free: b_a - sum_b A_ab phi_b, one thread per (q, a)
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, a = i - q * NN;
        const float* fq = p.phi_eval + (int64_t)(p.eq0 + q) * N;
        const float* Ra = R + q * RQ + a * PAD;
        const uint16_t* sa = symt + a * NN;
        float y = Ra[NN];
        const float* Dr = Dq + q * DQS;
        for (int b = 0; b < NN; ++b) y = fmaf(-(Ra[b] + (TCP == 0 ? Dr[sa[b]] : 0.f)), fq[ce[b]], y);
        atomicAdd(p.resid + (int64_t)(p.eq0 + q) * N + ce[a], y);
      }
    } else if (EM) {  // em[e][entry][q]: entry a * 27 + b of A, then 729 + a of the RHS
      float* dst = p.em + e * ENT * Q;
      const float invQ = 1.0f / (float)Q;  // i / Q for i < 2^20 as a float quotient (exact here)
      for (int i = tid; i < ENT * Q; i += H27_THREADS) {
        const int ent = (int)(((float)i + 0.5f) * invQ), q = i - ent * Q;
        float v;
        if (ent < NN * NN) {
          const int a = ent / NN, b = ent - a * NN;
          v = R[q * RQ + a * PAD + b];
          if (TCP == 0) v += Dq[q * DQS + symt[ent]];
        } else {
          v = R[q * RQ + (ent - NN * NN) * PAD + NN];
        }
        dst[i] = v;
      }
    } else {  // one thread per result slot (a, column), all equations
      const int32_t* pe = reinterpret_cast<const int32_t*>(sm27 + L.spos + cur * NN * NN);
      for (int j = tid; j < RQ; j += H27_THREADS) {
        const int a = j / PAD, b = j - a * PAD;
        const bool mat = b < NN;
        const int ent = a * NN + b;
        const int k = mat ? symt[ent] : 0;
        float* dst = mat ? p.values + (int64_t)p.eq0 * p.nnz + pe[ent] : p.rhs + (int64_t)p.eq0 * N + ce[a];
        const int64_t stride = mat ? p.nnz : N;
        for (int q = 0; q < Q; ++q) {
          float v = R[q * RQ + j];
          if (TCP == 0 && mat) v += Dq[q * DQS + k];
          atomicAdd(dst + q * stride, v);
        }
      }
    }
  }
  cp_async_wait_all();  // no copy is left in flight when the CTA exits
  if constexpr (TCP > 0) {  // every tensor-memory load has completed (each thread waited on its own)
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, TC_TMEM_COLS);
  }
}

fea_status launch(const AsmArgs<float>& a, cudaStream_t s) {
  // the tensor-core products serve the assembly (atomic or gather scatter), not the residual
  const int tcp = a.resid ? 0 : a.contraction == FEA_CONTRACT_TC_BF16X3 ? 2 : a.contraction == FEA_CONTRACT_TC_TF32X3 ? 4 : 0;
  const H27Layout L(a.eq_count, tcp);
  const size_t smem = sizeof(float) * (size_t)L.total;
  if (smem > 227 * 1024) return fail(FEA_ERR_TOO_LARGE, "hex27 kernel: shared memory");
  auto kern = tcp == 2 ? (a.em ? k_hex27<true, 2> : k_hex27<false, 2>)
            : tcp == 4 ? (a.em ? k_hex27<true, 4> : k_hex27<false, 4>)
                       : (a.em ? k_hex27<true, 0> : k_hex27<false, 0>);
  FEA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, H27_THREADS, smem);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.n_elem, (int64_t)nsm * std::max(per_sm, 1)));
  kern<<<grid, H27_THREADS, smem, s>>>(a);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

}  // namespace

bool hex27_kernel_applies(const AsmArgs<float>& a) { return a.terms == FEA_TERM_ALL && a.eq_count <= H27_QMAX; }

fea_status launch_hex27_f32(const AsmArgs<float>& a, cudaStream_t s) {
  if (a.n_elem == 0) return FEA_OK;
  return launch(a, s);
}

}  // namespace fea
