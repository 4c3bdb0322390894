// fea_hex27.cu -- FP32 Hex27 element matrices, one CTA per element (full operator, up to 12
// equations): the 27 x 27 matrices of all equations of an element share its geometry.
//
// Per Gauss point g (Sec. 4.2, Listing 1 extended to the full Galerkin + SUPG operator):
//   A_ab = sum_g P_a(g) Q_b(g) + sum_g k_g D_ab(g),  b_a = sum_g P_a(g) phi_g / dt,
//   P_a = dV (N_a + tau u.grad N_a),  Q_b = (1/dt + s) N_b + u.grad N_b,
//   D_ab = dV grad N_a . grad N_b   (symmetric, the same for every equation).
// Steps, each spread over the CTA's threads with a barrier between:
//   0. the element's node data (coordinates as FP32 hi/lo, velocity, k, s, phi_old, and the
//      CSR positions for the atomic scatter) arrive in a staging buffer by cp.async, issued
//      during the previous element's contraction (connectivity one more phase ahead);
//   1. x_a - x_0, u_g;  2. J per (g, i, j);  3. det J and J^-T per g (FP64 when badly
//      conditioned), dV;  4. grad N and u.grad N per (g, a), h = V^(1/3)/2;
//   5. k, s, phi, tau, 1/dt + s per (equation, g), the diffusion weights dV k_g; D per
//      (a <= b, g) without dV, one thread per symmetric entry;
//   6. P and Q per (equation, g, four columns);
//   7. the contractions in registers: P^T Q as 8 x 8 tiles over the 27 points, the
//      diffusion as 8 symmetric entries x all equations (the D loads are shared by the
//      equations), 16-byte shared loads feeding packed FP32x2 FMAs; the RHS on the threads
//      left over;
//   8. P^T Q tiles and the symmetric diffusion sums to shared memory (separate arrays);
//   9. out: A = P^T Q + diffusion (entry (a, b) of the symmetric part looked up in a table),
//      to the gather scratch em[e][entry][q], as atomic adds into the CSR values and RHS
//      (one position load per entry for all equations), or as the matrix-free residual.
#include <algorithm>

#include "fea_internal.cuh"

namespace fea {
namespace {

constexpr int NN = 27, PAD = 28;       // nodes / Gauss points; padded row length
constexpr int SYM = NN * (NN + 1) / 2;  // 378 symmetric entries
constexpr int DSTRIDE = 384;            // D row per Gauss point (multiple of 8)
constexpr int ENT = NN * NN + NN;       // element matrix entries and RHS entries
constexpr int H27_THREADS = 256;

// Shared-memory layout in floats; QP = equations padded to a multiple of 4; SR staged rows
// of 27 node values: x hi (3), x lo (3), u (3), then k, s, phi_old of each equation.
struct H27Layout {
  int QP, SR, nt, dnt, rowp, wq, sym, cn, stage, spos, xd, jg, dv, un, ug, gr, ua, kgt, sg, pg, tau, sig, p, q, d,
      ab, rhs, misc, total;
  __host__ __device__ H27Layout(int Q) {
    QP = (Q + 3) & ~3;
    SR = 9 + 3 * Q;
    int o = 0;
    nt = o;    o += NN * PAD;          // N_a(g)             [g][a]
    dnt = o;   o += NN * NN * 3;       // dN_a/dxi_j(g)      [g][a][j]
    o = (o + 1) & ~1;
    rowp = o;  o += 2 * SR;            // source array of staged row r (64-bit pointers)
    wq = o;    o += NN;                // Gauss weights
    sym = o;   o += (NN * NN + 1) / 2; // symmetric index of entry (a, b) (16-bit)
    cn = o;    o += 2 * PAD;           // connectivity, two buffers (int bits)
    stage = o; o += 2 * SR * NN;       // staged node data, two buffers [buf][row][a]
    spos = o;  o += 2 * NN * NN;       // staged CSR positions, two buffers (int bits)
    xd = o;    o += NN * 3;            // x_a - x_0          [a][i]
    jg = o;    o += NN * 9;            // J, then J^-T       [g][3][3]
    dv = o;    o += NN;                // w det J            [g]
    un = o;    o += NN;                // |u_g|
    ug = o;    o += NN * 3;            // u_g                [g][i]
    o = (o + 3) & ~3;                  // 16-byte rows for the float4 loads below
    gr = o;    o += NN * 3 * PAD;      // grad N             [g][i][a]
    ua = o;    o += NN * PAD;          // u.grad N           [g][a]
    kgt = o;   o += NN * QP;           // dV k_g             [g][q]
    sg = o;    o += Q * NN;            // s_g                [q][g]
    pg = o;    o += Q * NN;            // phi_g
    tau = o;   o += Q * NN;
    sig = o;   o += Q * NN;            // 1/dt + s_g
    o = (o + 3) & ~3;
    p = o;     o += Q * NN * PAD;      // P [q][g][a]; after the contractions P^T Q and the RHS [q][entry]
    q = o;     o += Q * NN * PAD;      // Q                  [q][g][b]
    d = o;     o += NN * DSTRIDE;      // grad N_a . grad N_b [g][sym]; after the contractions [q][sym]
    ab = o;    o += DSTRIDE;           // (a, b) of symmetric entry k, packed a | b << 8 (int bits)
    rhs = o;   o += Q * NN;            // b_a                [q][a]
    misc = o;  o += 4;                 // h
    total = o;
  }
};

// Index of entry (a, b) in the row-major upper triangle (row a starts at a NN - a (a - 1) / 2).
__device__ __forceinline__ int sym_index(int a, int b) {
  const int lo = min(a, b), hi = max(a, b);
  return lo * NN - lo * (lo - 1) / 2 + (hi - lo);
}

template <int QMAX, bool EM>
__global__ void __launch_bounds__(H27_THREADS, 1) k_hex27(AsmArgs<float> p) {
  extern __shared__ __align__(16) float sm27[];
  const int Q = p.eq_count;
  const H27Layout L(Q);
  const int tid = threadIdx.x;
  const int64_t N = p.n_node;
  const float inv_dt = (float)(1.0 / p.dt);
  const bool stage_pos = !EM && p.resid == nullptr;  // the atomic scatter reads pos[e]
  constexpr int DB = 8;                          // symmetric entries per diffusion task
  constexpr int ACC = DB * QMAX / 2 > 32 ? DB * QMAX / 2 : 32;
  const int n_pq = Q * 16;                       // (q, a-block, b-block) tiles of 8 x 8
  const int n_d = (SYM + DB - 1) / DB;           // n_pq + n_d <= 12 * 16 + 48 = 240 threads
  int* abt = reinterpret_cast<int*>(sm27 + L.ab);
  uint16_t* symt = reinterpret_cast<uint16_t*>(sm27 + L.sym);
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
  if (tid < NN)
    for (int b = tid, k = tid * NN - tid * (tid - 1) / 2; b < NN; ++b, ++k) abt[k] = tid | (b << 8);
  for (int i = tid; i < NN * NN; i += H27_THREADS) symt[i] = (uint16_t)sym_index(i / NN, i - (i / NN) * NN);
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
  // the first element's connectivity (plain loads) and node data (cp.async)
  if (blockIdx.x < p.n_elem && tid < NN)
    reinterpret_cast<int*>(sm27 + L.cn)[tid] = p.conn[(int64_t)blockIdx.x * NN + tid];
  __syncthreads();
  // staged node data of element e into buffer buf (connectivity already in cn[buf])
  auto stage_issue = [&](int64_t e, int buf) {
    const int* cb = reinterpret_cast<const int*>(sm27 + L.cn + buf * PAD);
    float* dst = sm27 + L.stage + buf * L.SR * NN;
    for (int i = tid; i < L.SR * NN; i += H27_THREADS) {
      const int r = i / NN, a = i - r * NN;
      cp_async4(dst + i, rowp[r] + cb[a]);
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
    const float* st = sm27 + L.stage + cur * L.SR * NN;  // [row][a]
    cp_async_wait_all();
    __syncthreads();  // element e's staged data is visible; the previous element's results are written
    if (en < p.n_elem && tid < NN) cp_async4(sm27 + L.cn + (cur ^ 1) * PAD + tid, p.conn + en * NN + tid);
    cp_async_commit();
    // 1. x_a - x_0 (hi/lo split), u_g = sum_a N_a(g) u_a
    if (tid < NN * 3) {
      const int a = tid / 3, c = tid - a * 3;
      sm27[L.xd + tid] = (st[c * NN + a] - st[c * NN]) + (st[(3 + c) * NN + a] - st[(3 + c) * NN]);
    } else if (tid >= 128 && tid < 128 + NN * 3) {
      const int i = tid - 128, g = i / 3, c = i - g * 3;
      const float* u = st + (6 + c) * NN;
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
      if (!(det > 0.f) || !(nj * ni <= 9.0f * (float)(p.kappa_threshold * p.kappa_threshold))) {
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
    // 5a. k, s, phi, tau, 1/dt + s per (q, g); the diffusion weight dV k_g
    {
      const float h = sm27[L.misc], c_k = 4.0f / (h * h), c_u = 2.0f / h;
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, g = i - q * NN;
        const float* fk = st + (9 + q) * NN;
        const float* fs = st + (9 + Q + q) * NN;
        const float* fp = st + (9 + 2 * Q + q) * NN;
        float kg = 0.f, sg = 0.f, pg = 0.f;
        for (int a = 0; a < NN; ++a) {
          const float na = sm27[L.nt + g * PAD + a];
          kg = fmaf(na, fk[a], kg);
          sg = fmaf(na, fs[a], sg);
          pg = fmaf(na, fp[a], pg);
        }
        const float den = c_k * kg + c_u * sm27[L.un + g] + sg;
        sm27[L.kgt + g * L.QP + q] = sm27[L.dv + g] * kg;
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
    // 5b. D_ab(g) = grad N_a . grad N_b, a <= b, one thread per symmetric entry (padding zero):
    // entry tid, and entry tid + 128 on the upper half of the threads (the lower ones may have
    // two (q, g) items above)
    for (int rep = 0; rep < 2; ++rep) {
      const int k = rep == 0 ? tid : tid + (DSTRIDE - H27_THREADS);
      if (k >= DSTRIDE || (rep == 1 && tid < 2 * H27_THREADS - DSTRIDE)) break;
      float* Dk = sm27 + L.d + k;
      if (k < SYM) {
        const int ab2 = abt[k], a = ab2 & 0xff, b = ab2 >> 8;
#pragma unroll 9
        for (int g = 0; g < NN; ++g) {
          const float* gg = sm27 + L.gr + g * 3 * PAD;
          Dk[g * DSTRIDE] = gg[a] * gg[b] + gg[PAD + a] * gg[PAD + b] + gg[2 * PAD + a] * gg[2 * PAD + b];
        }
      } else {
        for (int g = 0; g < NN; ++g) Dk[g * DSTRIDE] = 0.f;
      }
    }
    __syncthreads();
    // 6. P and Q per (q, g, four columns a); the padded column is zero because N and u.grad N are
    for (int i = tid; i < Q * NN * (PAD / 4); i += H27_THREADS) {
      const int qg = i / (PAD / 4), c4 = (i - qg * (PAD / 4)) * 4, g = qg - (qg / NN) * NN;
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
      qv.w = fmaf(sgm, na.w, ua.w);
      *reinterpret_cast<float4*>(sm27 + L.p + qg * PAD + c4) = pv;
      *reinterpret_cast<float4*>(sm27 + L.q + qg * PAD + c4) = qv;
    }
    cp_async_wait_all();  // the next element's connectivity
    __syncthreads();
    // 7. the next element's node data starts to arrive; contractions in registers; RHS
    if (en < p.n_elem) stage_issue(en, cur ^ 1);
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
    __syncthreads();  // P, Q and D are no longer read: P^T Q goes where P was, the diffusion sums where D was
    float* R = sm27 + L.p;   // [q][ENT]: P^T Q, then the RHS
    float* Dq = sm27 + L.d;  // [q][DSTRIDE]: sum_g dV k_g grad N_a . grad N_b, entry sym(a, b)
    if (task < n_pq) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int ra = ab * 8 + a, cb = bb * 8 + 2 * b;
          if (ra < NN && cb < NN) R[tq * ENT + ra * NN + cb] = acc2[a * 4 + b].x;
          if (ra < NN && cb + 1 < NN) R[tq * ENT + ra * NN + cb + 1] = acc2[a * 4 + b].y;
        }
    } else if (task < n_pq + n_d) {
      const int k0 = (task - n_pq) * DB;
#pragma unroll
      for (int j = 0; j < DB; ++j)
#pragma unroll
        for (int c = 0; c < QMAX / 2; ++c) {
          const float2 v = acc2[j * (QMAX / 2) + c];
          if (2 * c < Q) Dq[2 * c * DSTRIDE + k0 + j] = v.x;
          if (2 * c + 1 < Q) Dq[(2 * c + 1) * DSTRIDE + k0 + j] = v.y;
        }
    }
    for (int i = tid; i < Q * NN; i += H27_THREADS) {  // the RHS after the matrix entries
      const int q = i / NN, a = i - q * NN;
      R[q * ENT + NN * NN + a] = sm27[L.rhs + i];
    }
    __syncthreads();
    // 9. out
    if (p.resid) {  // matrix-free: b_a - sum_b A_ab phi_b, one thread per (q, a)
      for (int i = tid; i < Q * NN; i += H27_THREADS) {
        const int q = i / NN, a = i - q * NN;
        const float* fq = p.phi_eval + (int64_t)(p.eq0 + q) * N;
        const float* Ra = R + q * ENT + a * NN;
        const float* Dr = Dq + q * DSTRIDE;
        const uint16_t* sa = symt + a * NN;
        float y = R[q * ENT + NN * NN + a];
        for (int b = 0; b < NN; ++b) y = fmaf(-(Ra[b] + Dr[sa[b]]), fq[ce[b]], y);
        atomicAdd(p.resid + (int64_t)(p.eq0 + q) * N + ce[a], y);
      }
    } else if (EM) {
      float* dst = p.em + e * ENT * Q;
      const float invQ = 1.0f / (float)Q;  // i / Q for i < 2^20 as a float quotient (exact here)
      for (int i = tid; i < ENT * Q; i += H27_THREADS) {
        const int ent = (int)(((float)i + 0.5f) * invQ), q = i - ent * Q;
        float v = R[q * ENT + ent];
        if (ent < NN * NN) v += Dq[q * DSTRIDE + symt[ent]];
        dst[i] = v;
      }
    } else {
      const int32_t* pe = reinterpret_cast<const int32_t*>(sm27 + L.spos + cur * NN * NN);
      for (int ent = tid; ent < ENT; ent += H27_THREADS) {
        const bool mat = ent < NN * NN;
        const int k = mat ? symt[ent] : 0;
        float* dst = mat ? p.values + (int64_t)p.eq0 * p.nnz + pe[ent] : p.rhs + (int64_t)p.eq0 * N + ce[ent - NN * NN];
        const int64_t stride = mat ? p.nnz : N;
        for (int q = 0; q < Q; ++q) {
          float v = R[q * ENT + ent];
          if (mat) v += Dq[q * DSTRIDE + k];
          atomicAdd(dst + q * stride, v);
        }
      }
    }
  }
  cp_async_wait_all();  // no copy is left in flight when the CTA exits
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
