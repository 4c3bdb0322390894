// fea_rowowned_kernel.cuh -- the row-owned Hex8 kernel (included by fea_rowowned.cu,
// inside namespace fea::ro, after the plan types).
//
// One CTA of THREADS threads walks its work units batch by batch.  Per batch t:
//   stage     node ids and scatter offsets (plan data) and raw coordinates/velocity
//             arrive in shared memory by cp.async, issued one and two batches ahead;
//   geometry  warps 0..ceil(8 nv/32)-1, one thread per (element, Gauss point):
//             Jacobian, det, J^-T, physical gradients, u.grad N_a,
//             dV grad N_a . grad N_b, |u|; FP64 Jacobian for badly conditioned points;
//   matrices  one thread per (element, equation) item, one or two items per thread:
//             nodal fields from the node-major copy, the element matrix and RHS as sums
//             over Gauss points (packed FP32x2 FMAs), added with plain load-add-store
//             into the shared-memory rows in four rounds (local rows a and a+4 in round
//             a & 3, a barrier after each): elements of a batch share an owned node
//             only if they reach it in different rounds;
//   flush     between its first and second item, each warp writes its share of the
//             rows completed by batch t-1 to HBM once, with plain stores, and clears
//             their slots (the stores overlap the other warps' arithmetic).  The plan
//             hands such a slot out again from batch t+1 on; the rows the unit's last
//             batch completes are written once it ends.

struct RoArgs {
  AsmArgs<float> a;
  const int32_t* unit_batch;
  const int32_t* batch_visit;
  const int32_t* batch_flush;
  const int32_t* visit_nodes;
  const uint16_t* visit_off;
  const int4* flush_meta;  // [n_flush] {row, slot entry base, first CSR position, row length}
  const float* fnode;  // [N][rec] node-major k, s, phi_old (equation fastest), then u
  int n_units, n_slots, row_stride, maxcol, neqs, accumulate, be, rec;
};

// 1-D linear basis at the 2-point Gauss abscissae: l_0(-p) = l_1(p) = AL, l_0(p) = l_1(-p) = BL.
constexpr float AL = 0.78867513459481288225f;  // (1 + 1/sqrt 3) / 2
constexpr float BL = 0.21132486540518711775f;  // (1 - 1/sqrt 3) / 2
constexpr int RAW = 9;                         // per node: xhi[3], xlo[3], u[3]

// N_a at Gauss point g of the trilinear hex: AL^(3-d) BL^d, d = axes where a and g differ.
__host__ __device__ constexpr float hex_n(int a, int g) {
  return (((a ^ g) & 1) ? BL : AL) * (((a ^ g) & 2) ? BL : AL) * (((a ^ g) & 4) ? BL : AL);
}

__host__ __device__ constexpr int sym_index(int a, int b) {  // a <= b
  return a * NEN - a * (a - 1) / 2 + (b - a);
}

// Values of a nodal field at the 8 Gauss points by sum factorisation (x, then y, then z).
__device__ __forceinline__ void interp8(const float v[NEN], float out[NG]) {
  float tx[2][4], ty[2][2][2];
#pragma unroll
  for (int jk = 0; jk < 4; ++jk) {
    tx[0][jk] = fmaf(AL, v[2 * jk], BL * v[2 * jk + 1]);
    tx[1][jk] = fmaf(BL, v[2 * jk], AL * v[2 * jk + 1]);
  }
#pragma unroll
  for (int gx = 0; gx < 2; ++gx)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      ty[gx][0][k] = fmaf(AL, tx[gx][2 * k], BL * tx[gx][2 * k + 1]);
      ty[gx][1][k] = fmaf(BL, tx[gx][2 * k], AL * tx[gx][2 * k + 1]);
    }
#pragma unroll
  for (int gx = 0; gx < 2; ++gx)
#pragma unroll
    for (int gy = 0; gy < 2; ++gy) {
      out[gx + 2 * gy] = fmaf(AL, ty[gx][gy][0], BL * ty[gx][gy][1]);
      out[gx + 2 * gy + 4] = fmaf(BL, ty[gx][gy][0], AL * ty[gx][gy][1]);
    }
}

// Per-batch staging buffer in shared memory.
struct Stage {
  int32_t* nid;    // [be][8]
  uint16_t* off;   // [be][OFFS]
  float* raw;      // [be][8][RAW]
};

// Issues the copies of the plan data (node ids, offsets) of batch t into buffer s (a CTA of NT threads).
template <int NT = THREADS>
__device__ __forceinline__ void stage_plan(const RoArgs& r, int t, const Stage& s) {
  const int v0 = r.batch_visit[t], nv = r.batch_visit[t + 1] - v0;
  const int32_t* vn = r.visit_nodes + (int64_t)v0 * NEN;
  for (int i = threadIdx.x; i < nv * NEN; i += NT) cp_async4(s.nid + i, vn + i);
  const uint32_t* vo = reinterpret_cast<const uint32_t*>(r.visit_off + (int64_t)v0 * OFFS);
  uint32_t* so = reinterpret_cast<uint32_t*>(s.off);
  for (int i = threadIdx.x; i < nv * OFFS / 2; i += NT) cp_async4(so + i, vo + i);
}

// Issues the gathers of the raw node data of batch t (node ids already in buffer s).
template <int NT = THREADS>
__device__ __forceinline__ void stage_nodes(const RoArgs& r, int t, const Stage& s) {
  const AsmArgs<float>& A_ = r.a;
  const int nv = r.batch_visit[t + 1] - r.batch_visit[t];
  const int64_t N = A_.n_node;
  for (int i = threadIdx.x; i < nv * NEN * RAW; i += NT) {
    const int node = i / RAW, c = i - node * RAW;
    const int64_t n = s.nid[node];
    const float* src = c < 3   ? A_.xhi + (int64_t)c * N + n
                       : c < 6 ? A_.xlo + (int64_t)(c - 3) * N + n
                               : r.fnode + n * r.rec + 3 * A_.eq_count + (c - 6);
    cp_async4(s.raw + i, src);
  }
}

// Writes the rows completed by batch tb to HBM and clears their slots; warp w of nw takes a
// contiguous share of the batch's records.  Row by row, lane c holds column c: it loads 8
// equations' values (consecutive words of the slot) before storing them, so one store
// instruction writes one equation's row segment (consecutive CSR positions); the row's RHS is one
// store with the lanes over the equations.  Every value is written once (plain stores;
// accumulating calls add).
__device__ __forceinline__ void flush_rows(const RoArgs& r, float* win, int tb, int w0, int nw) {
  const AsmArgs<float>& A_ = r.a;
  const int lane = threadIdx.x & 31, n_eq = A_.eq_count;
  const int fb = r.batch_flush[tb], nb = r.batch_flush[tb + 1] - fb;
  const int f0 = fb + (int)(((int64_t)nb * w0) / nw), nf = fb + (int)(((int64_t)nb * (w0 + 1)) / nw) - f0;
  float* const values = A_.values + (int64_t)A_.eq0 * A_.nnz;
  float* const rhs = A_.rhs + (int64_t)A_.eq0 * A_.n_node;
  const bool acc = r.accumulate != 0;
  constexpr int QG = 8;
  for (int f = 0; f < nf; f += 32) {
    const int nr = min(32, nf - f);
    int4 rec = make_int4(0, 0, 0, 0);
    if (lane < nr) rec = __ldg(r.flush_meta + f0 + f + lane);
    for (int i = 0; i < nr; ++i) {
      const int row = __shfl_sync(0xffffffffu, rec.x, i), rb = __shfl_sync(0xffffffffu, rec.y, i);
      const int64_t k0 = (uint32_t)__shfl_sync(0xffffffffu, rec.z, i);  // first CSR position (nnz < 2^31)
      const int len = __shfl_sync(0xffffffffu, rec.w, i);
      for (int c = lane; c < len; c += 32) {
        const float* src = win + (rb + c) * r.neqs;
        float* dst = values + k0 + c;
        for (int q0 = 0; q0 < n_eq; q0 += QG) {
          float v[QG];
#pragma unroll
          for (int k = 0; k < QG; ++k) v[k] = q0 + k < n_eq ? src[q0 + k] : 0.f;
#pragma unroll
          for (int k = 0; k < QG; ++k)
            if (q0 + k < n_eq) {
              float* d = dst + (int64_t)(q0 + k) * A_.nnz;
              *d = acc ? *d + v[k] : v[k];
            }
        }
      }
      const float* src = win + (rb + r.maxcol) * r.neqs;
      for (int q = lane; q < n_eq; q += 32) {
        float* d = rhs + (int64_t)q * A_.n_node + row;
        *d = acc ? *d + src[q] : src[q];
      }
    }
    __syncwarp();
    // clear the slots (contiguous, 16-byte aligned: row_stride is a multiple of 4)
    for (int i = 0; i < nr; ++i) {
      const int rb = __shfl_sync(0xffffffffu, rec.y, i);
      float4* z = reinterpret_cast<float4*>(win + rb * r.neqs);
      for (int k = lane; k < r.row_stride * r.neqs / 4; k += 32) z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
  }
}

// Geometry of element ge at Gauss point g of the batch in S into geo; all 32 lanes of the
// calling warp must call it (the element volume is a shuffle reduction over 8 lanes).
__device__ __forceinline__ void geometry(const RoArgs& r, const Stage& S, float* geo, int ge, int g, bool gact) {
  const AsmArgs<float>& A_ = r.a;
  float dv = 0.f, un = 0.f, ua[NEN], gr[NEN][3];
  if (gact) {
    const float pp = 0.57735026918962576451f;
    const float xi[3] = {(g & 1) ? pp : -pp, (g & 2) ? pp : -pp, (g & 4) ? pp : -pp};
    float J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dN[NEN][3], ug[3] = {0, 0, 0};
    const float* d = S.raw + ge * NEN * RAW;
#pragma unroll
    for (int a = 0; a < NEN; ++a) {
      float Na;
      shape<FEA_HEX8>(a, xi, Na, dN[a]);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float xa = (d[a * RAW + i] - d[i]) + (d[a * RAW + 3 + i] - d[3 + i]);
#pragma unroll
        for (int j = 0; j < 3; ++j) J[i][j] = fmaf(xa, dN[a][j], J[i][j]);
        ug[i] = fmaf(Na, d[a * RAW + 6 + i], ug[i]);
      }
    }
    float det = det3(J), Gt[3][3];
    inv_transpose3(J, det, Gt);
    // condition estimate |J|_F |J^-1|_F (an upper bound of the 2-norm condition number); above the
    // threshold the Jacobian is redone in FP64
    float nj = 0.f, ni = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        nj = fmaf(J[i][j], J[i][j], nj);
        ni = fmaf(Gt[i][j], Gt[i][j], ni);
      }
    if (!(det > 0.f) || nj * ni > (float)(A_.kappa_threshold * A_.kappa_threshold)) {
      const int32_t* ids = S.nid + ge * NEN;
      const double pd = 0.57735026918962576451;
      const double xid[3] = {(g & 1) ? pd : -pd, (g & 2) ? pd : -pd, (g & 4) ? pd : -pd};
      double Jd[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Gd[3][3];
      for (int a = 0; a < NEN; ++a) {
        double Nd, dNd[3];
        shape<FEA_HEX8>(a, xid, Nd, dNd);
        for (int i = 0; i < 3; ++i) {
          double xa = A_.coords[(int64_t)ids[a] * 3 + i] - A_.coords[(int64_t)ids[0] * 3 + i];
          for (int j = 0; j < 3; ++j) Jd[i][j] += xa * dNd[j];
        }
      }
      const double dd = det3(Jd);
      if (!(dd > 0.0)) atomicOr(A_.status, ST_INVERTED);
      inv_transpose3(Jd, dd, Gd);
      det = (float)dd;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Gt[i][j] = (float)Gd[i][j];
    }
#pragma unroll
    for (int a = 0; a < NEN; ++a) {
#pragma unroll
      for (int i = 0; i < 3; ++i) gr[a][i] = Gt[i][0] * dN[a][0] + Gt[i][1] * dN[a][1] + Gt[i][2] * dN[a][2];
      ua[a] = ug[0] * gr[a][0] + ug[1] * gr[a][1] + ug[2] * gr[a][2];
    }
    dv = det;  // Gauss weight 1
    un = sqrtf(ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
  }
  float vol = dv;
  vol += __shfl_xor_sync(0xffffffffu, vol, 1);
  vol += __shfl_xor_sync(0xffffffffu, vol, 2);
  vol += __shfl_xor_sync(0xffffffffu, vol, 4);
  if (gact) {
    const float h = cbrtf(vol);
    float4* G4 = reinterpret_cast<float4*>(geo + ge * GEO_ELEM + g * GEO);
    float gv[GEO];
    gv[0] = dv;
    gv[1] = 2.f * un / h;
#pragma unroll
    for (int a = 0; a < NEN; ++a) gv[2 + a] = ua[a];
#pragma unroll
    for (int a = 0; a < NEN; ++a)
#pragma unroll
      for (int b = a; b < NEN; ++b)
        gv[10 + sym_index(a, b)] = dv * (gr[a][0] * gr[b][0] + gr[a][1] * gr[b][1] + gr[a][2] * gr[b][2]);
    gv[46] = gv[47] = 0.f;
#pragma unroll
    for (int k2 = 0; k2 < GEO / 4; ++k2) G4[k2] = make_float4(gv[4 * k2], gv[4 * k2 + 1], gv[4 * k2 + 2], gv[4 * k2 + 3]);
    if (g == 0) geo[ge * GEO_ELEM + NG * GEO] = 4.f / (h * h);
  }
}

// Nodal k, s, phi_old of equation q at the nodes of batch element el, from the node-major copy
// (the threads of one element read consecutive equations: contiguous memory).
__device__ __forceinline__ void load_fields(const RoArgs& r, const Stage& S, int el, int q, float kn[NEN],
                                            float sn[NEN], float pn[NEN]) {
  const int n_eq = r.a.eq_count;
#pragma unroll
  for (int a = 0; a < NEN; ++a) {
    const float* F = r.fnode + (int64_t)S.nid[el * NEN + a] * r.rec + q;
    kn[a] = __ldg(F);
    sn[a] = __ldg(F + n_eq);
    pn[a] = __ldg(F + 2 * n_eq);
  }
}

// The Gauss-point sums of one (element, equation) item (all Hex8 kernels): the element
// matrix as the packed product Am and the symmetric diffusion Dm, and the RHS bv2, from the
// element's geometry Ge (GEO floats per point, then 4/h^2) and the interpolated k, s, phi.
template <bool FULL>
__device__ __forceinline__ void item_sums(const float* Ge, float ck, const float kg[NG], const float sg[NG],
                                          const float pg[NG], float inv_dt, bool t_mass, bool t_conv, bool t_diff,
                                          bool t_reac, bool t_supg, float2 (&Am)[NEN][NEN / 2], float2 (&Dm)[18],
                                          float2 (&bv2)[NEN / 2]) {
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const float4* G4 = reinterpret_cast<const float4*>(Ge + g * GEO);
    float gv[GEO];
#pragma unroll
    for (int k2 = 0; k2 < GEO / 4 - 1; ++k2) {
      const float4 x = G4[k2];
      gv[4 * k2] = x.x;
      gv[4 * k2 + 1] = x.y;
      gv[4 * k2 + 2] = x.z;
      gv[4 * k2 + 3] = x.w;
    }
    {
      const float4 x = G4[GEO / 4 - 1];
      gv[GEO - 4] = x.x;
      gv[GEO - 3] = x.y;
    }
    const float dv = gv[0];
    const float den = fmaf(ck, kg[g], gv[1] + sg[g]);
    const float tau = den > 0.f ? __fdividef(1.f, den) : 0.f;
    const float dvt = t_supg ? dv * tau : 0.f;
    const float sigs = inv_dt + sg[g];
    float P[NEN], Q[NEN];
    if (FULL) {
      // all terms: dV (N_a + tau u.gradN_a)((1/dt + s) N_b + u.gradN_b), one rank-1 product
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        P[a] = fmaf(dvt, gv[2 + a], dv * hex_n(a, g));
        Q[a] = fmaf(sigs, hex_n(a, g), gv[2 + a]);
      }
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        const float2 pa = make_float2(P[a], P[a]);
#pragma unroll
        for (int b = 0; b < NEN / 2; ++b) Am[a][b] = __ffma2_rn(pa, make_float2(Q[2 * b], Q[2 * b + 1]), Am[a][b]);
      }
    } else {
      // dV N_a (sig N_b + [conv] u.gradN_b) + [supg] dV tau u.gradN_a ((1/dt + s) N_b + u.gradN_b)
      const float sig = (t_mass ? inv_dt : 0.f) + (t_reac ? sg[g] : 0.f);
      float Ps[NEN], R[NEN];
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        P[a] = dv * hex_n(a, g);
        Ps[a] = dvt * gv[2 + a];
        Q[a] = sig * hex_n(a, g) + (t_conv ? gv[2 + a] : 0.f);
        R[a] = fmaf(sigs, hex_n(a, g), gv[2 + a]);
      }
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        const float2 pa = make_float2(P[a], P[a]), ps = make_float2(Ps[a], Ps[a]);
#pragma unroll
        for (int b = 0; b < NEN / 2; ++b) {
          Am[a][b] = __ffma2_rn(pa, make_float2(Q[2 * b], Q[2 * b + 1]), Am[a][b]);
          Am[a][b] = __ffma2_rn(ps, make_float2(R[2 * b], R[2 * b + 1]), Am[a][b]);
        }
      }
      if (!t_mass) {
#pragma unroll
        for (int a = 0; a < NEN; ++a) P[a] = 0.f;
      }
#pragma unroll
      for (int a = 0; a < NEN; ++a) P[a] += Ps[a];
    }
    if (t_diff) {
      const float2 k2v = make_float2(kg[g], kg[g]);
#pragma unroll
      for (int k2 = 0; k2 < 18; ++k2) Dm[k2] = __ffma2_rn(k2v, make_float2(gv[10 + 2 * k2], gv[11 + 2 * k2]), Dm[k2]);
    }
    const float2 pdt = make_float2(pg[g] * inv_dt, pg[g] * inv_dt);
#pragma unroll
    for (int a = 0; a < NEN / 2; ++a) bv2[a] = __ffma2_rn(make_float2(P[2 * a], P[2 * a + 1]), pdt, bv2[a]);
  }
}

template <bool FULL>
__global__ void __launch_bounds__(THREADS, 1) k_rowowned_hex8(RoArgs r) {
  extern __shared__ __align__(16) float sm_ro[];
  const AsmArgs<float>& A_ = r.a;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int be = r.be;
  const int win_floats = r.n_slots * r.row_stride * r.neqs;
  float* win = sm_ro;
  float* geo = win + ((win_floats + 3) & ~3);
  float* const stage0 = geo + be * GEO_ELEM;
  const int stage_floats = be * (NEN * RAW + NEN + OFFS / 2);
  auto stage = [&](int b) {  // staging buffer b in {0, 1}, addressed without a local array
    float* p = stage0 + b * stage_floats;
    Stage s;
    s.raw = p;
    s.nid = reinterpret_cast<int32_t*>(p + be * NEN * RAW);
    s.off = reinterpret_cast<uint16_t*>(p + be * NEN * RAW + be * NEN);
    return s;
  };
  const float inv_dt = (float)(1.0 / A_.dt);
  const bool t_mass = A_.terms & FEA_TERM_MASS, t_conv = A_.terms & FEA_TERM_CONV,
             t_diff = A_.terms & FEA_TERM_DIFF, t_reac = A_.terms & FEA_TERM_REAC,
             t_supg = A_.terms & FEA_TERM_SUPG;
  const int n_eq = A_.eq_count;

  for (int i = tid; i < win_floats; i += THREADS) win[i] = 0.f;

  // Units are sorted by size; CTA b takes units b, 2G-1-b, 2G+b, ... (snake order).
  const int G = gridDim.x;
  for (int k = 0;; ++k) {
    const int u = (k & 1) ? (k + 1) * G - 1 - (int)blockIdx.x : k * G + (int)blockIdx.x;
    if (u >= r.n_units) break;
    const int t0 = r.unit_batch[2 * u], t1 = r.unit_batch[2 * u + 1];
    // prologue: batch t0 into buffer 0, plan data of t0+1 into buffer 1
    stage_plan(r, t0, stage(0));
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    stage_nodes(r, t0, stage(0));
    cp_async_commit();
    if (t0 + 1 < t1) stage_plan(r, t0 + 1, stage(1));
    cp_async_commit();
    for (int t = t0; t < t1; ++t) {
      const Stage S = stage((t - t0) & 1);
      const Stage Sn = stage((t - t0 + 1) & 1);
      const int nv = r.batch_visit[t + 1] - r.batch_visit[t];
      const int items = nv * n_eq;
      cp_async_wait_all();  // raw node data of t, plan data of t+1
      // batch t's data has landed; batch t-1 is computed and the rows of t-2 are written
      __syncthreads();
      if (t + 1 < t1) stage_nodes(r, t + 1, Sn);
      cp_async_commit();
      // geometry of batch t
      const int gw = (nv * NG + 31) / 32;
      if (warp < gw) geometry(r, S, geo, tid >> 3, tid & 7, (tid >> 3) < nv);
      __syncthreads();
      float kn[NEN], sn[NEN], pn[NEN];
      if (tid < items) load_fields(r, S, tid / n_eq, tid % n_eq, kn, sn, pn);
      // element matrices: items tid, tid + THREADS, ... (element = item / n_eq, equation = item % n_eq)
      const int rounds = max(1, (items + THREADS - 1) / THREADS);
      const int flush_at = rounds >= 2 ? 1 : 0;  // the same for every thread
      for (int it = 0; it < rounds; ++it) {
        if (it == flush_at && t > t0) flush_rows(r, win, t - 1, warp, THREADS / 32);
        const int item = tid + it * THREADS;
        const bool has = item < items;  // threads without an item still meet every barrier
        const int el = has ? item / n_eq : 0, q = has ? item - el * n_eq : 0;
        const uint32_t* eo = reinterpret_cast<const uint32_t*>(S.off + el * OFFS);
        float2 Am[NEN][NEN / 2], Dm[18], bv2[NEN / 2];
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
          for (int b = 0; b < NEN / 2; ++b) Am[a][b] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k2 = 0; k2 < 18; ++k2) Dm[k2] = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < NEN / 2; ++a) bv2[a] = make_float2(0.f, 0.f);
        if (has) {
          const float* Ge = geo + el * GEO_ELEM;
          const float ck = Ge[NG * GEO];
          float kg[NG], sg[NG], pg[NG];
          interp8(kn, kg);
          interp8(sn, sg);
          interp8(pn, pg);
          if (item + THREADS < items)  // prefetch the next item's fields while this one computes
            load_fields(r, S, (item + THREADS) / n_eq, (item + THREADS) % n_eq, kn, sn, pn);
          item_sums<FULL>(Ge, ck, kg, sg, pg, inv_dt, t_mass, t_conv, t_diff, t_reac, t_supg, Am, Dm, bv2);
        }  // has
        // add into the shared-memory rows (offsets are in row-window entries of neqs floats):
        // local rows a and a + 4 in round a & 3.  The plan lets two elements of a batch share
        // an owned node only in different rounds, so no two threads touch the same word
        // between two barriers.  Per matrix row the 9 words (8 columns and the RHS) are
        // distinct, so all 9 are loaded before any is stored (the compiler cannot prove that
        // and would otherwise serialise every load behind the previous store).
        // an element's offsets: 16 bytes per matrix row (8 columns), then 16 bytes of RHS offsets
        const uint4* eo4 = reinterpret_cast<const uint4*>(eo);
        const uint4 rw4 = has ? eo4[NEN] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t rws[4] = {rw4.x, rw4.y, rw4.z, rw4.w};
#pragma unroll
        for (int rho = 0; rho < ROUNDS; ++rho) {
#pragma unroll
          for (int a = rho; a < NEN; a += ROUNDS) {
            if (!has) break;
            const uint32_t rw = rws[a / 2];
            const uint32_t ro = (a & 1) ? (rw >> 16) : (rw & 0xFFFFu);
            if (ro == NONE) continue;
            const uint4 c4 = eo4[a];
            const uint32_t cws[4] = {c4.x, c4.y, c4.z, c4.w};
            float* p[NEN + 1];
            float add[NEN + 1];
#pragma unroll
            for (int b = 0; b < NEN; b += 2) {
              const uint32_t w2 = cws[b / 2];
              const int i0 = a <= b ? sym_index(a, b) : sym_index(b, a);
              const int i1 = a <= b + 1 ? sym_index(a, b + 1) : sym_index(b + 1, a);
              p[b] = win + (int)(w2 & 0xFFFFu) * r.neqs + q;
              p[b + 1] = win + (int)(w2 >> 16) * r.neqs + q;
              add[b] = Am[a][b / 2].x + ((i0 & 1) ? Dm[i0 >> 1].y : Dm[i0 >> 1].x);
              add[b + 1] = Am[a][b / 2].y + ((i1 & 1) ? Dm[i1 >> 1].y : Dm[i1 >> 1].x);
            }
            p[NEN] = win + (int)ro * r.neqs + q;
            add[NEN] = (a & 1) ? bv2[a / 2].y : bv2[a / 2].x;
            float old[NEN + 1];
#pragma unroll
            for (int b = 0; b <= NEN; ++b) old[b] = *p[b];
#pragma unroll
            for (int b = 0; b <= NEN; ++b) *p[b] = old[b] + add[b];
          }
          __syncthreads();
        }
      }
      // the last round's barrier: every thread is done with the plan data in S
      if (t + 2 < t1) stage_plan(r, t + 2, S);
      cp_async_commit();
    }
    // the rows the last batch completed, by all warps
    __syncthreads();
    flush_rows(r, win, t1 - 1, warp, THREADS / 32);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ two threads per item

// The half-item sums of the full operator: rows a = 4H .. 4H + 3 of one (element, equation)
// item's matrix and RHS.  The same Gauss-point sums as item_sums<true>, restricted to four
// rows: Am[r][c] = sum_g P_(4H+r)(g) (Q_(2c), Q_(2c+1))(g), Dh[r][c] the diffusion entries of
// those rows (the symmetric storage read for both (a, b) and (b, a)), bv2 the RHS of the rows.
template <int H>
__device__ __forceinline__ void half_sums(const float* Ge, float ck, const float kg[NG], const float sg[NG],
                                          const float pg[NG], float inv_dt, float2 (&Am)[4][NEN / 2],
                                          float2 (&Dh)[4][NEN / 2], float2 (&bv2)[2]) {
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const float4* G4 = reinterpret_cast<const float4*>(Ge + g * GEO);
    float gv[12];
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
      const float4 x = G4[k2];
      gv[4 * k2] = x.x;
      gv[4 * k2 + 1] = x.y;
      gv[4 * k2 + 2] = x.z;
      gv[4 * k2 + 3] = x.w;
    }
    const float dv = gv[0];
    const float den = fmaf(ck, kg[g], gv[1] + sg[g]);
    const float tau = den > 0.f ? __fdividef(1.f, den) : 0.f;
    const float dvt = dv * tau;
    const float sigs = inv_dt + sg[g];
    float P[4], Q[NEN];
#pragma unroll
    for (int a = 0; a < 4; ++a) P[a] = fmaf(dvt, gv[2 + 4 * H + a], dv * hex_n(4 * H + a, g));
#pragma unroll
    for (int b = 0; b < NEN; ++b) Q[b] = fmaf(sigs, hex_n(b, g), gv[2 + b]);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 pa = make_float2(P[a], P[a]);
#pragma unroll
      for (int c = 0; c < NEN / 2; ++c) Am[a][c] = __ffma2_rn(pa, make_float2(Q[2 * c], Q[2 * c + 1]), Am[a][c]);
    }
    // diffusion: entry (a, b) of the symmetric D sits at gv[10 + sym_index(min, max)]; walk the
    // stored entries in float4 pieces and add each to the rows of this half it belongs to
    const float kk = kg[g];
#pragma unroll
    for (int c4 = 2; c4 < GEO / 4; ++c4) {
      const float4 x = G4[c4];
      const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = 4 * c4 + j - 10;  // symmetric index of this stored entry
        if (e < 0 || e >= 36) continue;
        int a = 0;
        while (a < NEN - 1 && sym_index(a + 1, a + 1) <= e) ++a;  // row of e in the upper triangle
        const int b = a + (e - sym_index(a, a));
        if (a >= 4 * H && a < 4 * H + 4) {
          float& dst = (b & 1) ? Dh[a - 4 * H][b / 2].y : Dh[a - 4 * H][b / 2].x;
          dst = fmaf(kk, xv[j], dst);
        }
        if (b != a && b >= 4 * H && b < 4 * H + 4) {
          float& dst = (a & 1) ? Dh[b - 4 * H][a / 2].y : Dh[b - 4 * H][a / 2].x;
          dst = fmaf(kk, xv[j], dst);
        }
      }
    }
    const float pdt = pg[g] * inv_dt;
    bv2[0] = __ffma2_rn(make_float2(P[0], P[1]), make_float2(pdt, pdt), bv2[0]);
    bv2[1] = __ffma2_rn(make_float2(P[2], P[3]), make_float2(pdt, pdt), bv2[1]);
  }
}

// The row-owned kernel with two threads per (element, equation) item, each forming four rows of
// the element matrix (half H = 0: rows 0-3, H = 1: rows 4-7), in CTAs of THREADS_HALF threads:
// half the accumulators per thread, so twice the warps per SM, at the price of the
// interpolation and the Gauss-point scalars computed by both threads.  Items run as
// [half][element][equation], each half padded to whole warps, so a warp's threads share H.
// Same plan, batches, scatter rounds (round rho writes row 4 H + rho) and flush as
// k_rowowned_hex8; full operator only.
constexpr int THREADS_HALF = 512;

__global__ void __launch_bounds__(THREADS_HALF, 1) k_rowowned_hex8_half(RoArgs r) {
  constexpr int NT = THREADS_HALF;
  extern __shared__ __align__(16) float sm_roh[];
  const AsmArgs<float>& A_ = r.a;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int be = r.be;
  const int win_floats = r.n_slots * r.row_stride * r.neqs;
  float* win = sm_roh;
  float* geo = win + ((win_floats + 3) & ~3);
  float* const stage0 = geo + be * GEO_ELEM;
  const int stage_floats = be * (NEN * RAW + NEN + OFFS / 2);
  auto stage = [&](int b) {
    float* p = stage0 + b * stage_floats;
    Stage s;
    s.raw = p;
    s.nid = reinterpret_cast<int32_t*>(p + be * NEN * RAW);
    s.off = reinterpret_cast<uint16_t*>(p + be * NEN * RAW + be * NEN);
    return s;
  };
  const float inv_dt = (float)(1.0 / A_.dt);
  const int n_eq = A_.eq_count;

  for (int i = tid; i < win_floats; i += NT) win[i] = 0.f;

  const int G = gridDim.x;
  for (int k = 0;; ++k) {
    const int u = (k & 1) ? (k + 1) * G - 1 - (int)blockIdx.x : k * G + (int)blockIdx.x;
    if (u >= r.n_units) break;
    const int t0 = r.unit_batch[2 * u], t1 = r.unit_batch[2 * u + 1];
    stage_plan<NT>(r, t0, stage(0));
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    stage_nodes<NT>(r, t0, stage(0));
    cp_async_commit();
    if (t0 + 1 < t1) stage_plan<NT>(r, t0 + 1, stage(1));
    cp_async_commit();
    for (int t = t0; t < t1; ++t) {
      const Stage S = stage((t - t0) & 1);
      const Stage Sn = stage((t - t0 + 1) & 1);
      const int nv = r.batch_visit[t + 1] - r.batch_visit[t];
      const int items1 = nv * n_eq, hstride = (items1 + 31) & ~31;  // items of one half, padded
      cp_async_wait_all();
      __syncthreads();
      if (t + 1 < t1) stage_nodes<NT>(r, t + 1, Sn);
      cp_async_commit();
      const int gw = (nv * NG + 31) / 32;
      if (warp < gw) geometry(r, S, geo, tid >> 3, tid & 7, (tid >> 3) < nv);
      __syncthreads();
      const int rounds = max(1, (2 * hstride + NT - 1) / NT);
      const int flush_at = rounds >= 2 ? 1 : 0;
      for (int it = 0; it < rounds; ++it) {
        if (it == flush_at && t > t0) flush_rows(r, win, t - 1, warp, NT / 32);
        const int item = tid + it * NT;
        const int H = item >= hstride ? 1 : 0;  // the same for the whole warp (hstride % 32 == 0)
        const int li = item - H * hstride;
        const bool has = H < 2 && item < 2 * hstride && li < items1;
        const int el = has ? li / n_eq : 0, q = has ? li - el * n_eq : 0;
        const uint32_t* eo = reinterpret_cast<const uint32_t*>(S.off + el * OFFS);
        float2 Am[4][NEN / 2], Dh[4][NEN / 2], bv2[2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < NEN / 2; ++c) Am[a][c] = Dh[a][c] = make_float2(0.f, 0.f);
        bv2[0] = bv2[1] = make_float2(0.f, 0.f);
        if (has) {
          float kn[NEN], sn[NEN], pn[NEN];
          load_fields(r, S, el, q, kn, sn, pn);
          const float* Ge = geo + el * GEO_ELEM;
          const float ck = Ge[NG * GEO];
          float kg[NG], sg[NG], pg[NG];
          interp8(kn, kg);
          interp8(sn, sg);
          interp8(pn, pg);
          if (H == 0) half_sums<0>(Ge, ck, kg, sg, pg, inv_dt, Am, Dh, bv2);
          else half_sums<1>(Ge, ck, kg, sg, pg, inv_dt, Am, Dh, bv2);
        }
        // round rho: this thread's row a = 4 H + rho (rows rho and rho + 4 of every element are
        // written in round rho, as in the one-thread kernel)
        const uint4* eo4 = reinterpret_cast<const uint4*>(eo);  // as in k_rowowned_hex8
#pragma unroll
        for (int rho = 0; rho < ROUNDS; ++rho) {
          if (has) {
            const int a = 4 * H + rho;
            const uint32_t rw = eo[(NEN * NEN + a) / 2];
            const uint32_t ro = (a & 1) ? (rw >> 16) : (rw & 0xFFFFu);
            if (ro != NONE) {
              const uint4 c4 = eo4[a];
              const uint32_t cws[4] = {c4.x, c4.y, c4.z, c4.w};
              float* p[NEN + 1];
              float add[NEN + 1];
#pragma unroll
              for (int b = 0; b < NEN; b += 2) {
                const uint32_t w2 = cws[b / 2];
                p[b] = win + (int)(w2 & 0xFFFFu) * r.neqs + q;
                p[b + 1] = win + (int)(w2 >> 16) * r.neqs + q;
                add[b] = Am[rho][b / 2].x + Dh[rho][b / 2].x;
                add[b + 1] = Am[rho][b / 2].y + Dh[rho][b / 2].y;
              }
              p[NEN] = win + (int)ro * r.neqs + q;
              add[NEN] = (rho & 1) ? bv2[rho / 2].y : bv2[rho / 2].x;
              float old[NEN + 1];
#pragma unroll
              for (int b = 0; b <= NEN; ++b) old[b] = *p[b];
#pragma unroll
              for (int b = 0; b <= NEN; ++b) *p[b] = old[b] + add[b];
            }
          }
          __syncthreads();
        }
      }
      if (t + 2 < t1) stage_plan<NT>(r, t + 2, S);
      cp_async_commit();
    }
    __syncthreads();
    flush_rows(r, win, t1 - 1, warp, NT / 32);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ element-parallel Hex8

// One CTA takes batches of `be` consecutive elements: node data into shared memory, the
// geometry of the batch (one thread per (element, Gauss point)), then one thread per
// (element, equation) item forms the same sums as the row-owned kernel and sends them out
// by MODE: atomic adds into the CSR values and RHS, stores to the gather scratch, or the
// matrix-free residual b^e - A^e phi^e added into r.  No schedule, no halo recompute.
enum { EMODE_ATOMIC = 0, EMODE_SCRATCH = 1, EMODE_RESIDUAL = 2 };

template <bool FULL, int MODE>
__global__ void __launch_bounds__(THREADS, (MODE == EMODE_RESIDUAL && FULL) ? 2 : 1) k_hex8_elem(RoArgs r) {
  extern __shared__ __align__(16) float sm_el[];
  const AsmArgs<float>& A_ = r.a;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int be = r.be, n_eq = A_.eq_count;
  float* geo = sm_el;
  Stage S;
  S.raw = geo + be * GEO_ELEM;
  S.nid = reinterpret_cast<int32_t*>(S.raw + be * NEN * RAW);
  S.off = nullptr;
  const float inv_dt = (float)(1.0 / A_.dt);
  const bool t_mass = A_.terms & FEA_TERM_MASS, t_conv = A_.terms & FEA_TERM_CONV,
             t_diff = A_.terms & FEA_TERM_DIFF, t_reac = A_.terms & FEA_TERM_REAC,
             t_supg = A_.terms & FEA_TERM_SUPG;
  const int64_t N = A_.n_node, E = A_.n_elem;
  const int64_t nb = (E + be - 1) / be;
  for (int64_t bt = blockIdx.x; bt < nb; bt += gridDim.x) {
    const int64_t e0 = bt * be;
    const int nv = (int)((E - e0) < (int64_t)be ? (E - e0) : (int64_t)be);
    __syncthreads();  // the previous batch is done with geo and the staged nodes
    for (int i = tid; i < nv * NEN; i += THREADS) S.nid[i] = A_.conn[e0 * NEN + i];
    __syncthreads();
    for (int i = tid; i < nv * NEN * RAW; i += THREADS) {
      const int node = i / RAW, c = i - node * RAW;
      const int64_t n = S.nid[node];
      S.raw[i] = c < 3 ? A_.xhi[(int64_t)c * N + n] : c < 6 ? A_.xlo[(int64_t)(c - 3) * N + n]
                                                            : r.fnode[n * r.rec + 3 * n_eq + (c - 6)];
    }
    __syncthreads();
    // one thread per (element, Gauss point), THREADS / NG elements per pass; a warp takes part in a
    // pass when it holds one of the batch's elements (the shuffles inside span the whole warp)
    for (int eb = 0; eb < nv; eb += THREADS / NG) {
      const int ge = eb + (tid >> 3);
      if (eb + warp * (32 / NG) < nv) geometry(r, S, geo, ge, tid & 7, ge < nv);
    }
    __syncthreads();
    const int items = nv * n_eq;
    for (int item = tid; item < items; item += THREADS) {
      const int el = item / n_eq, q = item - el * n_eq;
      float kn[NEN], sn[NEN], pn[NEN];
      load_fields(r, S, el, q, kn, sn, pn);
      if (MODE == EMODE_RESIDUAL && FULL) {
        // Matrix-free, without the element matrix: per Gauss point
        //   y_a += P_a (phi_old_g / dt - (1/dt + s_g) phi_g - u.grad phi_g) - k_g sum_b D_ab phi_b
        // with P_a = dV (N_a + tau u.grad N_a) (the full operator, whose trial part is
        // (1/dt + s) N_b + u.grad N_b).
        const float* Ge = geo + el * GEO_ELEM;
        const float ck = Ge[NG * GEO];
        const int32_t* ids = S.nid + el * NEN;
        const int qg = A_.eq0 + q;
        float ph[NEN], kg[NG], sg[NG], pg[NG], fg[NG];
#pragma unroll
        for (int b = 0; b < NEN; ++b) ph[b] = __ldg(A_.phi_eval + (int64_t)qg * N + ids[b]);
        interp8(kn, kg);
        interp8(sn, sg);
        interp8(pn, pg);
        interp8(ph, fg);
        float y[NEN];
#pragma unroll
        for (int a = 0; a < NEN; ++a) y[a] = 0.f;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const float* G = Ge + g * GEO;
          const float dv = G[0];
          const float den = fmaf(ck, kg[g], G[1] + sg[g]);
          const float tau = den > 0.f ? __fdividef(1.f, den) : 0.f;
          float ua[NEN], ugp = 0.f;
#pragma unroll
          for (int a = 0; a < NEN; a += 2) {  // u.grad N_a sits at offset 2 of the record: 8-byte aligned pairs
            const float2 x = *reinterpret_cast<const float2*>(G + 2 + a);
            ua[a] = x.x;
            ua[a + 1] = x.y;
          }
#pragma unroll
          for (int b = 0; b < NEN; ++b) ugp = fmaf(ua[b], ph[b], ugp);  // u.grad phi at g
          const float rg = fmaf(-(inv_dt + sg[g]), fg[g], fmaf(pg[g], inv_dt, -ugp));
          const float dvr = dv * rg, dvtr = dv * tau * rg;
#pragma unroll
          for (int a = 0; a < NEN; ++a) y[a] = fmaf(dvtr, ua[a], fmaf(dvr, hex_n(a, g), y[a]));
          // diffusion: y -= k_g D phi, D symmetric (entries a <= b)
          const float kgg = kg[g];
#pragma unroll
          for (int a = 0; a < NEN; ++a) {
#pragma unroll
            for (int b = a; b < NEN; ++b) {
              const float d = kgg * G[10 + sym_index(a, b)];
              y[a] = fmaf(-d, ph[b], y[a]);
              if (b != a) y[b] = fmaf(-d, ph[a], y[b]);
            }
          }
        }
#pragma unroll
        for (int a = 0; a < NEN; ++a) atomicAdd(A_.resid + (int64_t)qg * N + ids[a], y[a]);
        continue;
      }
      const float* Ge = geo + el * GEO_ELEM;
      float kg[NG], sg[NG], pg[NG];
      interp8(kn, kg);
      interp8(sn, sg);
      interp8(pn, pg);
      float2 Am[NEN][NEN / 2], Dm[18], bv2[NEN / 2];
#pragma unroll
      for (int a = 0; a < NEN; ++a)
#pragma unroll
        for (int b = 0; b < NEN / 2; ++b) Am[a][b] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k2 = 0; k2 < 18; ++k2) Dm[k2] = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < NEN / 2; ++a) bv2[a] = make_float2(0.f, 0.f);
      item_sums<FULL>(Ge, Ge[NG * GEO], kg, sg, pg, inv_dt, t_mass, t_conv, t_diff, t_reac, t_supg, Am, Dm, bv2);
      const int64_t e = e0 + el;
      const int32_t* ids = S.nid + el * NEN;
      const int qg = A_.eq0 + q;
      float phe[NEN];
      if (MODE == EMODE_RESIDUAL) {
#pragma unroll
        for (int b = 0; b < NEN; ++b) phe[b] = __ldg(A_.phi_eval + (int64_t)qg * N + ids[b]);
      }
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        float row[NEN];
#pragma unroll
        for (int b = 0; b < NEN; b += 2) {
          const int i0 = a <= b ? sym_index(a, b) : sym_index(b, a);
          const int i1 = a <= b + 1 ? sym_index(a, b + 1) : sym_index(b + 1, a);
          row[b] = Am[a][b / 2].x + ((i0 & 1) ? Dm[i0 >> 1].y : Dm[i0 >> 1].x);
          row[b + 1] = Am[a][b / 2].y + ((i1 & 1) ? Dm[i1 >> 1].y : Dm[i1 >> 1].x);
        }
        const float ba = (a & 1) ? bv2[a / 2].y : bv2[a / 2].x;
        if (MODE == EMODE_RESIDUAL) {
          float y = ba;
#pragma unroll
          for (int b = 0; b < NEN; ++b) y = fmaf(-row[b], phe[b], y);
          atomicAdd(A_.resid + (int64_t)qg * N + ids[a], y);
        } else if (MODE == EMODE_SCRATCH) {
          float* d = A_.em + ((e * (NEN * NEN + NEN)) + a * NEN) * n_eq + q;
#pragma unroll
          for (int b = 0; b < NEN; ++b) d[b * n_eq] = row[b];
          A_.em[((e * (NEN * NEN + NEN)) + NEN * NEN + a) * n_eq + q] = ba;
        } else {
          const int32_t* pe = A_.pos + (e * NEN + a) * NEN;
          float* vq = A_.values + (int64_t)qg * A_.nnz;
#pragma unroll
          for (int b = 0; b < NEN; ++b) atomicAdd(vq + __ldg(pe + b), row[b]);
          atomicAdd(A_.rhs + (int64_t)qg * N + ids[a], ba);
        }
      }
    }
  }
}
