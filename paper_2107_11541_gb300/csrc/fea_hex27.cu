// fea_hex27.cu -- FP32 Hex27 element matrices, one CTA per element (full operator, up to 12
// equations): the 27 x 27 matrices of all equations of an element share its geometry.
//
// Per Gauss point g (Sec. 4.2, Listing 1 extended to the full Galerkin + SUPG operator):
//   A_ab = sum_g P_a(g) Q_b(g) + sum_g k_g D_ab(g),  b_a = sum_g P_a(g) phi_g / dt,
//   P_a = dV (N_a + tau u.grad N_a),  Q_b = (1/dt + s) N_b + u.grad N_b,
//   D_ab = dV grad N_a . grad N_b   (symmetric, the same for every equation).
// Steps, each spread over the CTA's threads with a barrier between:
//   1. node data: coordinate differences (FP32 hi/lo split), velocity, k, s, phi_old;
//   2. geometry: J per (g, i, j), det J and J^-T per g (FP64 when badly conditioned),
//      u_g, grad N per (g, i, a), u.grad N per (g, a), h = V^(1/3)/2;
//   3. k, s, phi, tau, 1/dt + s per (equation, g); P and Q per (equation, g, a); the RHS;
//      D per (g, a <= b);
//   4. the contractions in registers: P^T Q as 8 x 8 tiles over the 27 points, the
//      diffusion as 8 symmetric entries x all equations (the D loads are shared by the
//      equations), 16-byte shared loads feeding packed FP32x2 FMAs;
//   5. results through shared memory to the gather scratch em[e][entry][q] (consecutive
//      threads on consecutive addresses) or as atomic adds into the CSR values and RHS.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {
namespace {

constexpr int NN = 27, PAD = 28;       // nodes / Gauss points; padded row length
constexpr int SYM = NN * (NN + 1) / 2;  // 378 symmetric entries
constexpr int DSTRIDE = 384;            // D row per Gauss point (multiple of 8)
constexpr int H27_THREADS = 256;

// Shared-memory layout in floats; QP = equations padded to a multiple of 4.
struct H27Layout {
  int QP, nt, dnt, xd, ue, fk, fs, fp, jg, dv, un, ug, gr, ua, kgt, sg, pg, tau, sig, p, q, d, ab, rhs, misc, total;
  __host__ __device__ H27Layout(int Q) {
    QP = (Q + 3) & ~3;
    int o = 0;
    nt = o;   o += NN * PAD;          // N_a(g)          [g][a]
    dnt = o;  o += NN * NN * 3;       // dN_a/dxi_j(g)   [g][a][j]
    xd = o;   o += NN * 3;            // x_a - x_0       [a][i]
    ue = o;   o += NN * 3;            // u_a             [a][i]
    fk = o;   o += Q * NN;            // k               [q][a]
    fs = o;   o += Q * NN;
    fp = o;   o += Q * NN;
    jg = o;   o += NN * 9;            // J, then J^-T    [g][3][3]
    dv = o;   o += NN;                // w det J         [g]
    un = o;   o += NN;                // |u_g|
    ug = o;   o += NN * 3;            // u_g             [g][i]
    gr = o;   o += NN * 3 * PAD;      // grad N          [g][i][a]
    ua = o;   o += NN * PAD;          // u.grad N        [g][a]
    o = (o + 3) & ~3;                 // 16-byte rows for the float4 loads of k_g
    kgt = o;  o += NN * QP;           // k_g             [g][q]
    sg = o;   o += Q * NN;            // s_g             [q][g]
    pg = o;   o += Q * NN;            // phi_g
    tau = o;  o += Q * NN;
    sig = o;  o += Q * NN;            // 1/dt + s_g
    o = (o + 3) & ~3;
    p = o;    o += Q * NN * PAD;      // P               [q][g][a]; later the results [q][entry]
    q = o;    o += Q * NN * PAD;      // Q               [q][g][b]
    d = o;    o += NN * DSTRIDE;      // D               [g][sym]
    ab = o;   o += DSTRIDE;           // (a, b) of symmetric entry k, packed a | b << 8 (int bits)
    rhs = o;  o += Q * NN;            // b_a             [q][a]
    misc = o; o += 4;                 // h
    total = o;
  }
};

template <int QMAX, bool EM>
__global__ void __launch_bounds__(H27_THREADS, 1) k_hex27(AsmArgs<float> p) {
  extern __shared__ __align__(16) float sm27[];
  const int Q = p.eq_count;
  const H27Layout L(Q);
  const int tid = threadIdx.x;
  const int64_t N = p.n_node;
  const float inv_dt = (float)(1.0 / p.dt);
  constexpr int DB = 8;                          // symmetric entries per diffusion task
  constexpr int ACC = DB * QMAX / 2 > 32 ? DB * QMAX / 2 : 32;
  const int n_pq = Q * 16;                       // (q, a-block, b-block) tiles of 8 x 8
  const int n_d = (SYM + DB - 1) / DB;           // n_pq + n_d <= 12 * 16 + 48 = 240 threads

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
    }
    sm27[L.nt + i] = v;
  }
  int* abt = reinterpret_cast<int*>(sm27 + L.ab);
  if (tid < NN)  // row a of the upper triangle starts at a NN - a (a - 1) / 2
    for (int b = tid, k = tid * NN - tid * (tid - 1) / 2; b < NN; ++b, ++k) abt[k] = tid | (b << 8);
  const float invQ = 1.0f / (float)Q;  // i / Q for i < 2^20 as a float quotient (exact here)

  for (int64_t e = blockIdx.x; e < p.n_elem; e += gridDim.x) {
    const int32_t* ce = p.conn + e * NN;
    __syncthreads();  // the previous element's results are written
    // 1. node data
    for (int i = tid; i < NN * 6; i += H27_THREADS) {
      const int a = i / 6, c = i - a * 6;
      const int32_t n = ce[a];
      if (c < 3) {
        const int32_t n0 = ce[0];
        const int64_t o = (int64_t)c * N;
        sm27[L.xd + a * 3 + c] = (p.xhi[o + n] - p.xhi[o + n0]) + (p.xlo[o + n] - p.xlo[o + n0]);
      } else {
        sm27[L.ue + a * 3 + (c - 3)] = p.vel[(int64_t)(c - 3) * N + n];
      }
    }
    for (int i = tid; i < 3 * Q * NN; i += H27_THREADS) {
      const int fq = i / NN, a = i - fq * NN, f = (int)(((float)fq + 0.5f) * invQ), q = fq - f * Q;
      const int64_t idx = (int64_t)(p.eq0 + q) * N + ce[a];
      sm27[(f == 0 ? L.fk : f == 1 ? L.fs : L.fp) + q * NN + a] = f == 0 ? p.kd[idx] : f == 1 ? p.sr[idx] : p.phi[idx];
    }
    __syncthreads();
    // 2a. J_gij = sum_a (x_a - x_0)_i dN_a/dxi_j(g)
    for (int i = tid; i < NN * 9; i += H27_THREADS) {
      const int g = i / 9, ij = i - g * 9, ii = ij / 3, j = ij - ii * 3;
      float s = 0.f;
      for (int a = 0; a < NN; ++a) s = fmaf(sm27[L.xd + a * 3 + ii], sm27[L.dnt + (g * NN + a) * 3 + j], s);
      sm27[L.jg + i] = s;
    }
    // 2c. u_g
    for (int i = tid; i < NN * 3; i += H27_THREADS) {
      const int g = i / 3, c = i - g * 3;
      float s = 0.f;
      for (int a = 0; a < NN; ++a) s = fmaf(sm27[L.nt + g * PAD + a], sm27[L.ue + a * 3 + c], s);
      sm27[L.ug + i] = s;
    }
    __syncthreads();
    // 2b. det, J^-T (FP64 above the condition threshold), dV, |u_g|
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
      double xid[3], w;
      gauss_point<FEA_HEX27>(g, xid, w);
      if (!(det > 0.f) || !(nj * ni <= 9.0f * (float)(p.kappa_threshold * p.kappa_threshold))) {
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
      sm27[L.dv + g] = (float)w * det;
      const float* u = sm27 + L.ug + g * 3;
      sm27[L.un + g] = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
    __syncthreads();
    // 2d. grad N_a(g) = J^-T grad_xi N_a; padded column a = 27 is zero
    for (int i = tid; i < NN * 3 * PAD; i += H27_THREADS) {
      const int g = i / (3 * PAD), rem = i - g * 3 * PAD, c = rem / PAD, a = rem - c * PAD;
      float s = 0.f;
      if (a < NN) {
        const float* G = sm27 + L.jg + g * 9 + c * 3;
        const float* dn = sm27 + L.dnt + (g * NN + a) * 3;
        s = G[0] * dn[0] + G[1] * dn[1] + G[2] * dn[2];
      }
      sm27[L.gr + i] = s;
    }
    if (tid == 0) {
      float v = 0.f;
      for (int g = 0; g < NN; ++g) v += sm27[L.dv + g];
      sm27[L.misc] = cbrtf(v) * 0.5f;  // h = V^(1/3) / 2
    }
    __syncthreads();
    // 2e. u.grad N_a(g); 3a. k, s, phi, tau, 1/dt + s per (q, g)
    for (int i = tid; i < NN * PAD; i += H27_THREADS) {
      const int g = i / PAD, a = i - g * PAD;
      const float* u = sm27 + L.ug + g * 3;
      const float* gg = sm27 + L.gr + g * 3 * PAD + a;
      sm27[L.ua + i] = a < NN ? u[0] * gg[0] + u[1] * gg[PAD] + u[2] * gg[2 * PAD] : 0.f;
    }
    {
      const float h = sm27[L.misc], c_k = 4.0f / (h * h), c_u = 2.0f / h;
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, g = i - q * NN;
        float kg = 0.f, sg = 0.f, pg = 0.f;
        for (int a = 0; a < NN; ++a) {
          const float na = sm27[L.nt + g * PAD + a];
          kg = fmaf(na, sm27[L.fk + q * NN + a], kg);
          sg = fmaf(na, sm27[L.fs + q * NN + a], sg);
          pg = fmaf(na, sm27[L.fp + q * NN + a], pg);
        }
        const float den = c_k * kg + c_u * sm27[L.un + g] + sg;
        sm27[L.kgt + g * L.QP + q] = kg;
        sm27[L.sg + i] = sg;
        sm27[L.pg + i] = pg;
        sm27[L.tau + i] = den > 0.f ? 1.0f / den : 0.f;
        sm27[L.sig + i] = inv_dt + sg;
      }
      for (int i = tid; i < NN * (L.QP - Q); i += H27_THREADS) {  // padded equations of k_g: zero
        const int g = i / (L.QP - Q), q = Q + (i - g * (L.QP - Q));
        sm27[L.kgt + g * L.QP + q] = 0.f;
      }
    }
    // 3c. D_ab(g) = dV grad N_a . grad N_b, a <= b (padding entries zero)
    for (int i = tid; i < NN * DSTRIDE; i += H27_THREADS) {
      const int g = i / DSTRIDE, k = i - g * DSTRIDE;
      float v = 0.f;
      if (k < SYM) {
        const int ab2 = abt[k], a = ab2 & 0xff, b = ab2 >> 8;
        const float* gg = sm27 + L.gr + g * 3 * PAD;
        v = sm27[L.dv + g] * (gg[a] * gg[b] + gg[PAD + a] * gg[PAD + b] + gg[2 * PAD + a] * gg[2 * PAD + b]);
      }
      sm27[L.d + i] = v;
    }
    __syncthreads();
    // 3b. P and Q per (q, g, a); padded column zero
    for (int i = tid; i < Q * NN * PAD; i += H27_THREADS) {
      const int q = i / (NN * PAD), rem = i - q * NN * PAD, g = rem / PAD, a = rem - g * PAD;
      float pv = 0.f, qv = 0.f;
      if (a < NN) {
        const float na = sm27[L.nt + g * PAD + a], ua = sm27[L.ua + g * PAD + a];
        pv = sm27[L.dv + g] * fmaf(sm27[L.tau + q * NN + g], ua, na);
        qv = fmaf(sm27[L.sig + q * NN + g], na, ua);
      }
      sm27[L.p + i] = pv;
      sm27[L.q + i] = qv;
    }
    __syncthreads();
    // 4. contractions in registers; RHS b_a = sum_g P_a phi_g / dt
    float2 acc2[ACC];  // PQ task: 8 x 8 tile; diffusion task: DB entries x QMAX equations
#pragma unroll
    for (int i = 0; i < ACC; ++i) acc2[i] = make_float2(0.f, 0.f);
    const int task = tid;
    int tq = 0, ab = 0, bb = 0;
    if (task < n_pq) {
      tq = task / 16;
      ab = (task / 4) & 3;
      bb = task & 3;
      const float* P = sm27 + L.p + tq * NN * PAD + ab * 8;
      const float* Qm = sm27 + L.q + tq * NN * PAD + bb * 8;
#pragma unroll 3
      for (int g = 0; g < NN; ++g) {
        const float4 p0 = *reinterpret_cast<const float4*>(P + g * PAD);
        const float4 p1 = *reinterpret_cast<const float4*>(P + g * PAD + 4);
        const float4 q0 = *reinterpret_cast<const float4*>(Qm + g * PAD);
        const float4 q1 = *reinterpret_cast<const float4*>(Qm + g * PAD + 4);
        const float pa[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
        const float2 qb[4] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                              make_float2(q1.z, q1.w)};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc2[a * 4 + b] = __ffma2_rn(make_float2(pa[a], pa[a]), qb[b], acc2[a * 4 + b]);
      }
    } else if (task >= n_pq + n_d) {
      // threads without a contraction task: the RHS, b_a = sum_g P_a phi_g / dt
      for (int i = task - (n_pq + n_d); i < Q * NN; i += H27_THREADS - (n_pq + n_d)) {
        const int qq = i / NN, a = i - qq * NN;
        float s0 = 0.f;
        for (int g = 0; g < NN; ++g) s0 = fmaf(sm27[L.p + (qq * NN + g) * PAD + a], sm27[L.pg + qq * NN + g], s0);
        sm27[L.rhs + i] = s0 * inv_dt;
      }
    } else {
      const int k0 = (task - n_pq) * DB;
      const float* D = sm27 + L.d + k0;
      const float* K = sm27 + L.kgt;
#pragma unroll 3
      for (int g = 0; g < NN; ++g) {
        float dv8[DB];
#pragma unroll
        for (int j = 0; j < DB; j += 4) {
          const float4 x = *reinterpret_cast<const float4*>(D + g * DSTRIDE + j);
          dv8[j] = x.x;
          dv8[j + 1] = x.y;
          dv8[j + 2] = x.z;
          dv8[j + 3] = x.w;
        }
        float2 kq[QMAX / 2];
#pragma unroll
        for (int j = 0; j < QMAX; j += 4) {
          const float4 x = *reinterpret_cast<const float4*>(K + g * L.QP + j);
          kq[j / 2] = make_float2(x.x, x.y);
          kq[j / 2 + 1] = make_float2(x.z, x.w);
        }
#pragma unroll
        for (int j = 0; j < DB; ++j)
#pragma unroll
          for (int c = 0; c < QMAX / 2; ++c)
            acc2[j * (QMAX / 2) + c] = __ffma2_rn(make_float2(dv8[j], dv8[j]), kq[c], acc2[j * (QMAX / 2) + c]);
      }
    }
    __syncthreads();  // P and Q are no longer read: the results go where P was
    float* R = sm27 + L.p;  // [q][NN*NN + NN]
    const int ENT = NN * NN + NN;
    if (task < n_pq) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int ra = ab * 8 + a, cb = bb * 8 + 2 * b;
          if (ra < NN && cb < NN) R[tq * ENT + ra * NN + cb] = acc2[a * 4 + b].x;
          if (ra < NN && cb + 1 < NN) R[tq * ENT + ra * NN + cb + 1] = acc2[a * 4 + b].y;
        }
    }
    for (int i = tid; i < Q * NN; i += H27_THREADS) {  // the RHS after the matrix entries
      const int q = i / NN, a = i - q * NN;
      R[q * ENT + NN * NN + a] = sm27[L.rhs + i];
    }
    __syncthreads();
    if (task >= n_pq && task < n_pq + n_d) {
      const int k0 = (task - n_pq) * DB;
#pragma unroll
      for (int j = 0; j < DB; ++j) {
        const int k = k0 + j;
        if (k >= SYM) break;
        const int ab2 = abt[k], a = ab2 & 0xff, b = ab2 >> 8;
#pragma unroll
        for (int c = 0; c < QMAX / 2; ++c) {
          const float2 v = acc2[j * (QMAX / 2) + c];
          const int q0 = 2 * c;
          if (q0 < Q) {
            R[q0 * ENT + a * NN + b] += v.x;
            if (a != b) R[q0 * ENT + b * NN + a] += v.x;
          }
          if (q0 + 1 < Q) {
            R[(q0 + 1) * ENT + a * NN + b] += v.y;
            if (a != b) R[(q0 + 1) * ENT + b * NN + a] += v.y;
          }
        }
      }
    }
    __syncthreads();
    // 5. out
    if (p.resid) {  // matrix-free: b_a - sum_b A_ab phi_b, one thread per (q, a)
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, a = i - q * NN;
        const float* fq = p.phi_eval + (int64_t)(p.eq0 + q) * N;
        const float* Ra = R + q * ENT + a * NN;
        float y = R[q * ENT + NN * NN + a];
        for (int b = 0; b < NN; ++b) y = fmaf(-Ra[b], fq[ce[b]], y);
        atomicAdd(p.resid + (int64_t)(p.eq0 + q) * N + ce[a], y);
      }
    } else if (EM) {
      float* dst = p.em + e * ENT * Q;
      for (int i = tid; i < ENT * Q; i += H27_THREADS) {
        const int ent = (int)(((float)i + 0.5f) * invQ), q = i - ent * Q;
        dst[i] = R[q * ENT + ent];
      }
    } else {
      const int32_t* pe = p.pos + e * NN * NN;
      for (int i = tid; i < ENT * Q; i += H27_THREADS) {
        const int q = i / ENT, ent = i - q * ENT;
        if (ent < NN * NN) atomicAdd(p.values + (int64_t)(p.eq0 + q) * p.nnz + pe[ent], R[i]);
        else atomicAdd(p.rhs + (int64_t)(p.eq0 + q) * N + ce[ent - NN * NN], R[i]);
      }
    }
  }
}

template <int QMAX>
fea_status launch_q(const AsmArgs<float>& a, cudaStream_t s) {
  const H27Layout L(a.eq_count);
  const size_t smem = sizeof(float) * (size_t)L.total;
  if (smem > 227 * 1024) return fail(FEA_ERR_TOO_LARGE, "hex27 kernel: shared memory");
  auto kern = a.em ? k_hex27<QMAX, true> : k_hex27<QMAX, false>;
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

bool hex27_kernel_applies(const AsmArgs<float>& a) { return a.terms == FEA_TERM_ALL && a.eq_count <= 12; }

fea_status launch_hex27_f32(const AsmArgs<float>& a, cudaStream_t s) {
  if (a.n_elem == 0) return FEA_OK;
  if (a.eq_count <= 4) return launch_q<4>(a, s);
  if (a.eq_count <= 8) return launch_q<8>(a, s);
  return launch_q<12>(a, s);
}

}  // namespace fea
