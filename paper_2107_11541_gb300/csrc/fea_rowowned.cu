// fea_rowowned.cu -- row-owned fused FP32 assembly of Hex8 meshes.
//
// Every CSR row (node) is owned by exactly one work unit.  A unit is a pencil of
// nodes (a tile in x-y, a range in z) together with every element incident to
// its nodes, swept in z order in batches.  Element matrices of all equations
// are accumulated in shared memory rows and each row is written to HBM once,
// with plain stores, as soon as its last incident element has been processed:
// no output zeroing, no global atomics, and the result does not depend on
// scheduling (bitwise reproducible).  Elements on the boundary of a pencil are
// computed by each unit that owns one of their nodes (halo recompute).  Also here: the
// element-parallel Hex8 kernel (no schedule) behind the atomic, gather and residual paths.
//
// Per element and Gauss point the geometry (Jacobian, det, inverse-transpose,
// physical gradients, w det J, u.grad N_a, the symmetric products
// dV grad N_a . grad N_b and |u|) is computed once and shared by all equations
// through shared memory; per equation a lane forms the Galerkin + SUPG element
// matrix as a sum over Gauss points of the rank-1 products P_a Q_b
// (P_a = dV (N_a + tau u.grad N_a), Q_b = (1/dt + s) N_b + u.grad N_b) plus
// the diffusion sum k_g dV grad N_a . grad N_b (Sec. 4.2, Listing 1,
// generalised to the full operator).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "fea_plan.cuh"

namespace fea {
namespace ro {

constexpr int NEN = 8, NG = 8;
constexpr int BEMAX = 32;               // elements per batch at most: one thread per (element, Gauss point)
constexpr int THREADS = 256;            // 8 warps (384 at 168 registers spills and measured 17% slower)
constexpr int ROUNDS = 4;               // scatter rounds: local rows a and a + 4 in round a & 3
constexpr int round_of(int a) { return a & 3; }
constexpr int LOOKAHEAD = 64;           // sweep positions scanned when forming a batch
constexpr int GEO = 48;                 // floats per Gauss point: dv, cu, ua[8], Gd[36], pad[2]
constexpr int GEO_ELEM = NG * GEO + 4;  // + ck (4/h^2) and padding
constexpr int OFFS = NEN * NEN + NEN;   // entry offsets per element visit (matrix, then RHS)
constexpr uint16_t NONE = 0xFFFF;
constexpr int SMEM_LIMIT = 232448;      // opt-in shared memory per block on sm_103

struct Variant {
  int n_eq = 0, neqs = 0, n_units = 0, n_slots = 0, row_stride = 0, maxcol = 0, be = 0;
  int64_t n_visits = 0, n_batches = 0, n_flush = 0;
  size_t smem = 0;
  bool unused_nodes = false;
  int32_t* unit_batch = nullptr;   // [n_units][2] first and end batch, largest unit first
  int32_t* batch_visit = nullptr;  // [n_batches+1]
  int32_t* batch_flush = nullptr;  // [n_batches+1]
  int32_t* visit_nodes = nullptr;  // [n_visits][NEN] node ids of the visited element
  uint16_t* visit_off = nullptr;   // [n_visits][OFFS]
  int32_t* flush_meta = nullptr;   // [n_flush][4] row, slot entry base, first CSR position, row length
  float* fnode = nullptr;          // [N][3 n_eq + 3] node-major k, s, phi_old (equation fastest) and u
  bool ok = false;
};

// Batch size: one thread per (element, equation), at least one element.
// Two (element, equation) items per thread when that keeps the threads busy, else one.
static int batch_elems(int n_eq) {
  int be2 = std::max(1, std::min(BEMAX, 2 * THREADS / n_eq));
  if (be2 * n_eq >= (2 * THREADS * 85) / 100) return be2;
  return std::max(1, std::min(BEMAX, THREADS / n_eq));
}

// Batch size of the element-parallel kernel: the same rule with a larger cap, so that with few
// equations the (element, equation) items still fill the CTA (its geometry runs in passes of
// THREADS / NG elements).  The cap keeps the batch's shared memory within one CTA's share.
static int elem_batch(int n_eq, int cap) {
  int be2 = std::max(1, std::min(cap, 2 * THREADS / n_eq));
  if (be2 * n_eq >= (2 * THREADS * 85) / 100) return be2;
  return std::max(1, std::min(cap, THREADS / n_eq));
}

// Shared memory besides the row window, for batches of `be` elements.
// Geometry of a batch plus two staging buffers (raw node data, node ids, offsets).
static size_t smem_fixed(int be) {
  return sizeof(float) * (size_t)be * (GEO_ELEM + 2 * (NEN * 9 + NEN + OFFS / 2));
}

}  // namespace ro
}  // namespace fea

struct fea_rowowned_plan {
  fea_mesh* mesh = nullptr;
  fea_pattern* pattern = nullptr;
  std::mutex mu;
  std::map<int, fea::ro::Variant*> variants;
  // host copies, filled on the first prepare
  bool host_ready = false;
  std::vector<int32_t> conn;
  std::vector<double> coords;
  std::vector<int64_t> rowptr, inc_ptr;
  std::vector<int32_t> colind, inc_elem;
  float* elem_fnode = nullptr;  // node-major fields for the element-parallel kernel
  size_t elem_fnode_bytes = 0;
};

namespace fea {
namespace ro {

// ------------------------------------------------------------------ host schedule

struct Builder {
  const fea_rowowned_plan& P;
  int64_t N, E;
  int n_slots, maxcol, row_stride, be;
  std::vector<int32_t> owner;      // unit being simulated that owns the node, or -1
  std::vector<int32_t> slot_of;    // node -> slot during simulation
  std::vector<int32_t> last_use;   // node -> last element position in the unit
  std::vector<uint8_t> touched;    // node already holds a slot
  std::vector<uint8_t> round_mask; // scatter rounds in which the current batch writes the node
  // outputs
  std::vector<int32_t> unit_batch{0}, batch_visit{0}, batch_flush{0}, visit_nodes, flush_meta;
  int64_t flushes() const { return (int64_t)flush_meta.size() / 4; }
  int64_t visits() const { return (int64_t)visit_nodes.size() / NEN; }
  std::vector<uint16_t> visit_off;

  Builder(const fea_rowowned_plan& p, int slots, int mc, int batch)
      : P(p), N((int64_t)p.rowptr.size() - 1), E((int64_t)p.conn.size() / NEN), n_slots(slots), maxcol(mc),
        row_stride(((mc + 1) + 3) & ~3), be(batch), owner(N, -1), slot_of(N, -1), last_use(N, -1), touched(N, 0), round_mask(N, 0) {}

  double cz(int32_t e, int d) const {
    double s = 0;
    for (int a = 0; a < NEN; ++a) s += P.coords[(int64_t)P.conn[(int64_t)e * NEN + a] * 3 + d];
    return s / NEN;
  }

  int colpos(int32_t r, int32_t c) const {
    const int32_t* b = P.colind.data() + P.rowptr[r];
    const int32_t* e = P.colind.data() + P.rowptr[r + 1];
    return (int)(std::lower_bound(b, e, c) - b);
  }

  // Simulates the sweep of one unit; appends its schedule and returns true, or
  // returns false (nothing appended) when some batch cannot fit in the slots.
  bool unit(const std::vector<int32_t>& nodes, int32_t uid) {
    for (int32_t n : nodes) owner[n] = uid;
    std::vector<int32_t> els;
    for (int32_t n : nodes)
      for (int64_t t = P.inc_ptr[n]; t < P.inc_ptr[n + 1]; ++t) els.push_back(P.inc_elem[t]);
    std::sort(els.begin(), els.end());
    els.erase(std::unique(els.begin(), els.end()), els.end());
    std::vector<std::array<double, 3>> key(els.size());
    for (size_t i = 0; i < els.size(); ++i) key[i] = {cz(els[i], 2), cz(els[i], 1), cz(els[i], 0)};
    std::vector<int32_t> order(els.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      if (key[a] != key[b]) return key[a] < key[b];
      return els[a] < els[b];
    });
    std::vector<int32_t> seq(els.size());
    for (size_t i = 0; i < els.size(); ++i) seq[i] = els[order[i]];
    // remaining[n] (kept in last_use): incident elements of owned node n not yet processed
    for (int32_t e : seq)
      for (int a = 0; a < NEN; ++a) {
        int32_t n = P.conn[(int64_t)e * NEN + a];
        if (owner[n] == uid) last_use[n] = (last_use[n] < 0 ? 0 : last_use[n]) + 1;
      }

    size_t mark_b = batch_visit.size(), mark_v = (size_t)visits(), mark_f = flush_meta.size();
    std::vector<int32_t> free_slots(n_slots);
    for (int i = 0; i < n_slots; ++i) free_slots[i] = n_slots - 1 - i;
    std::vector<uint8_t> done(seq.size(), 0);
    int live = 0;
    size_t head = 0;
    bool ok = true;
    std::vector<int32_t> fresh, batch, in_batch, completed, flushing;
    while (head < seq.size()) {
      // Greedy batching in a look-ahead window of the sweep.  The kernel adds local rows
      // a and a+4 of every element in scatter round a & 3, with a barrier between rounds,
      // so two elements of a batch may share an owned node only if they reach it in
      // different rounds; then no two threads update the same word at the same time.
      fresh.clear();
      batch.clear();
      int scanned = 0;
      for (size_t i = head; i < seq.size() && (int)batch.size() < be && scanned < LOOKAHEAD; ++i) {
        if (done[i]) continue;
        ++scanned;
        const int32_t* ce = &P.conn[(int64_t)seq[i] * NEN];
        bool clash = false;
        int k = 0;
        for (int a = 0; a < NEN; ++a) {
          if (owner[ce[a]] != uid) continue;
          if (round_mask[ce[a]] & (1u << round_of(a))) clash = true;
          if (!touched[ce[a]] && !round_mask[ce[a]]) ++k;
        }
        if (clash) continue;
        if (live + (int)fresh.size() + k > n_slots) break;
        for (int a = 0; a < NEN; ++a) {
          if (owner[ce[a]] != uid) continue;
          if (!touched[ce[a]] && !round_mask[ce[a]]) fresh.push_back(ce[a]);
          round_mask[ce[a]] |= (uint8_t)(1u << round_of(a));
          in_batch.push_back(ce[a]);
        }
        done[i] = 1;
        batch.push_back(seq[i]);
      }
      for (int32_t n : in_batch) {
        touched[n] = 1;
        round_mask[n] = 0;
      }
      in_batch.clear();
      if (batch.empty() && flushing.empty()) { ok = false; break; }
      // An empty batch (every candidate waits for a slot still being written out) only
      // lets the rows of the previous batch be flushed; its slots are free afterwards.
      while (head < seq.size() && done[head]) ++head;
      for (int32_t n : fresh) {
        slot_of[n] = free_slots.back();
        free_slots.pop_back();
      }
      live += (int)fresh.size();
      for (int32_t e : batch) {
        const int32_t* ce = &P.conn[(int64_t)e * NEN];
        visit_nodes.insert(visit_nodes.end(), ce, ce + NEN);
        uint16_t off[OFFS];
        for (int a = 0; a < NEN; ++a) {
          bool own = owner[ce[a]] == uid;
          int base = own ? slot_of[ce[a]] * row_stride : 0;
          for (int b = 0; b < NEN; ++b) off[a * NEN + b] = own ? (uint16_t)(base + colpos(ce[a], ce[b])) : NONE;
          off[NEN * NEN + a] = own ? (uint16_t)(base + maxcol) : NONE;
        }
        visit_off.insert(visit_off.end(), off, off + OFFS);
      }
      for (int32_t e : batch)
        for (int a = 0; a < NEN; ++a) {
          int32_t n = P.conn[(int64_t)e * NEN + a];
          if (owner[n] != uid || --last_use[n] > 0) continue;
          const int64_t k0 = P.rowptr[n];
          flush_meta.insert(flush_meta.end(), {n, slot_of[n] * row_stride, (int32_t)k0, (int32_t)(P.rowptr[n + 1] - k0)});
          completed.push_back(slot_of[n]);
        }
      // A row completed by batch b is written out while batch b+1 computes, so its slot
      // is free again from batch b+2 on.
      free_slots.insert(free_slots.end(), flushing.begin(), flushing.end());
      live -= (int)flushing.size();
      flushing.swap(completed);
      completed.clear();
      {  // the batch's completed rows in row order: consecutive records are adjacent CSR rows
        const size_t f0 = (size_t)batch_flush.back() * 4, nf = flush_meta.size() / 4 - (size_t)batch_flush.back();
        std::vector<std::array<int32_t, 4>> recs(nf);
        for (size_t i = 0; i < nf; ++i)
          for (int c = 0; c < 4; ++c) recs[i][c] = flush_meta[f0 + 4 * i + c];
        std::sort(recs.begin(), recs.end());
        for (size_t i = 0; i < nf; ++i)
          for (int c = 0; c < 4; ++c) flush_meta[f0 + 4 * i + c] = recs[i][c];
      }
      batch_visit.push_back((int32_t)visits());
      batch_flush.push_back((int32_t)flushes());
    }
    for (int32_t n : nodes) {
      owner[n] = -1;
      touched[n] = 0;
      last_use[n] = -1;
    }
    if (!ok) {
      batch_visit.resize(mark_b);
      batch_flush.resize(mark_b);
      visit_nodes.resize(mark_v * NEN);
      visit_off.resize(mark_v * OFFS);
      flush_meta.resize(mark_f);
      return false;
    }
    unit_batch.push_back((int32_t)(batch_visit.size() - 1));
    return true;
  }
};

// Splits a node set in two by the median of the wider of x and y.
static void split_xy(const std::vector<double>& coords, std::vector<int32_t>& nodes, std::vector<int32_t>& other) {
  double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
  for (int32_t n : nodes)
    for (int d = 0; d < 2; ++d) {
      lo[d] = std::min(lo[d], coords[(int64_t)n * 3 + d]);
      hi[d] = std::max(hi[d], coords[(int64_t)n * 3 + d]);
    }
  int d = (hi[0] - lo[0] >= hi[1] - lo[1]) ? 0 : 1;
  std::sort(nodes.begin(), nodes.end(), [&](int32_t a, int32_t b) {
    double xa = coords[(int64_t)a * 3 + d], xb = coords[(int64_t)b * 3 + d];
    return xa != xb ? xa < xb : a < b;
  });
  size_t h = nodes.size() / 2;
  other.assign(nodes.begin() + h, nodes.end());
  nodes.resize(h);
}

template <typename T>
static fea_status upload(T** dst, const std::vector<T>& src) {
  size_t n = std::max<size_t>(src.size(), 1);
  FEA_CUDA_TRY(cudaMalloc(dst, n * sizeof(T)));
  if (!src.empty()) FEA_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FEA_OK;
}

static void free_variant(Variant* v) {
  if (!v) return;
  cudaFree(v->unit_batch);
  cudaFree(v->batch_visit);
  cudaFree(v->batch_flush);
  cudaFree(v->visit_nodes);
  cudaFree(v->visit_off);
  cudaFree(v->flush_meta);
  cudaFree(v->fnode);
  delete v;
}

static fea_status host_copies(fea_rowowned_plan* P) {
  if (P->host_ready) return FEA_OK;
  fea_mesh* m = P->mesh;
  fea_pattern* p = P->pattern;
  int64_t N = m->n_node, E = m->n_elem;
  P->conn.resize((size_t)E * NEN);
  P->coords.resize((size_t)N * 3);
  P->rowptr.resize(N + 1);
  P->colind.resize(p->nnz);
  P->inc_ptr.resize(N + 1);
  P->inc_elem.resize((size_t)E * NEN);
  FEA_CUDA_TRY(cudaStreamSynchronize(m->stream));
  FEA_CUDA_TRY(cudaMemcpy(P->conn.data(), m->conn, P->conn.size() * 4, cudaMemcpyDeviceToHost));
  FEA_CUDA_TRY(cudaMemcpy(P->coords.data(), m->coords, P->coords.size() * 8, cudaMemcpyDeviceToHost));
  FEA_CUDA_TRY(cudaMemcpy(P->rowptr.data(), p->rowptr, P->rowptr.size() * 8, cudaMemcpyDeviceToHost));
  FEA_CUDA_TRY(cudaMemcpy(P->colind.data(), p->colind, P->colind.size() * 4, cudaMemcpyDeviceToHost));
  FEA_CUDA_TRY(cudaMemcpy(P->inc_ptr.data(), p->inc_ptr, P->inc_ptr.size() * 8, cudaMemcpyDeviceToHost));
  FEA_CUDA_TRY(cudaMemcpy(P->inc_elem.data(), p->inc_elem, P->inc_elem.size() * 4, cudaMemcpyDeviceToHost));
  P->host_ready = true;
  return FEA_OK;
}

static fea_status build_variant(fea_rowowned_plan* P, int n_eq, int batch, Variant* v) {
  FEA_TRY(host_copies(P));
  int64_t N = P->mesh->n_node, E = P->mesh->n_elem;
  int maxcol = 0;
  bool unused = false;
  for (int64_t r = 0; r < N; ++r) {
    maxcol = std::max<int>(maxcol, (int)(P->rowptr[r + 1] - P->rowptr[r]));
    if (P->inc_ptr[r + 1] == P->inc_ptr[r]) unused = true;
  }
  v->n_eq = n_eq;
  v->neqs = n_eq | 1;  // odd stride: conflict-free column-wise reads of the row window
  v->maxcol = maxcol;
  v->row_stride = ((maxcol + 1) + 3) & ~3;  // slots start 16-byte aligned (bulk zeroing)
  v->unused_nodes = unused;
  v->be = batch > 0 ? std::min(batch, BEMAX) : batch_elems(n_eq);
  size_t fixed = smem_fixed(v->be);
  if (fixed + 4096 > (size_t)SMEM_LIMIT) return FEA_OK;
  // per slot: its row of row_stride entries of neqs floats
  const size_t per_slot = sizeof(float) * (size_t)v->row_stride * v->neqs;
  int n_slots = (int)std::min<size_t>((SMEM_LIMIT - fixed) / per_slot, (NONE - 1) / v->row_stride);
  if (n_slots < 2 * NEN) return FEA_OK;  // too many equations for this kernel
  v->n_slots = n_slots;
  v->smem = fixed + per_slot * (size_t)n_slots;
  v->smem = (v->smem + 15) & ~(size_t)15;
  if (v->smem > (size_t)SMEM_LIMIT) return FEA_OK;

  // pencil tiling in x-y, chunks in z, bin edges midway between grid lines
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t n = 0; n < N; ++n)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], P->coords[n * 3 + d]);
      hi[d] = std::max(hi[d], P->coords[n * 3 + d]);
    }
  double vol = std::max(1e-300, (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]));
  double spacing = std::cbrt(vol / std::max<int64_t>(1, E));  // hex cell width
  // node columns per tile: two planes live plus the slots still being written out; 0.35 of the
  // slots measured best on Hex8 128^3 (0.25-0.55 swept: fuller tiles cut the halo but leave
  // fewer, larger units to balance over the CTAs)
  int cols = std::max(1, (int)(0.35 * n_slots));
  // tiles about 3x wider in x (the fastest node-id direction) than in y: the rows a batch
  // completes form runs of consecutive CSR rows (measured a few percent faster than square)
  const double aspect = 3.0;
  int tx0 = std::max(1, (int)std::floor(std::sqrt((double)cols * aspect)));
  int ty0 = std::max(1, cols / tx0);
  // spread the node planes of each axis evenly over the tiles (fractional widths)
  auto even = [&](int d, int t) {
    double planes = std::floor((hi[d] - lo[d]) / spacing + 0.5) + 1.0;
    double chunks = std::max(1.0, std::ceil(planes / t));
    return planes / chunks;
  };
  const double tx = even(0, tx0), ty = even(1, ty0), tz = even(2, 32);
  auto bin = [&](double x, double l, double t) { return (int64_t)std::floor(((x - l) / spacing + 0.5) / t); };
  std::map<std::array<int64_t, 3>, std::vector<int32_t>> units;
  for (int64_t n = 0; n < N; ++n) {
    const double* x = &P->coords[n * 3];
    units[{bin(x[2], lo[2], tz), bin(x[1], lo[1], ty), bin(x[0], lo[0], tx)}].push_back((int32_t)n);
  }
  Builder B(*P, n_slots, maxcol, v->be);
  std::vector<std::vector<int32_t>> work;
  for (auto& kv : units) work.push_back(std::move(kv.second));
  int32_t uid = 0;
  while (!work.empty()) {
    std::vector<int32_t> nodes = std::move(work.back());
    work.pop_back();
    if (B.unit(nodes, uid)) {
      ++uid;
      continue;
    }
    if (nodes.size() <= 1) return FEA_OK;  // cannot fit even one node's elements
    std::vector<int32_t> other;
    split_xy(P->coords, nodes, other);
    work.push_back(std::move(nodes));
    work.push_back(std::move(other));
  }
  v->n_units = uid;
  v->n_visits = B.visits();
  v->n_batches = (int64_t)B.batch_visit.size() - 1;
  v->n_flush = B.flushes();
  if (v->n_visits >= INT32_MAX / OFFS) return FEA_OK;
  // units as (first batch, end batch) pairs, largest first (the kernel deals them out in snake order)
  std::vector<int32_t> order(uid);
  std::iota(order.begin(), order.end(), 0);
  auto cost = [&](int32_t u) { return B.batch_visit[B.unit_batch[u + 1]] - B.batch_visit[B.unit_batch[u]]; };
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost(a) > cost(b); });
  std::vector<int32_t> ranges(2 * (size_t)uid);
  for (int32_t k = 0; k < uid; ++k) {
    ranges[2 * k] = B.unit_batch[order[k]];
    ranges[2 * k + 1] = B.unit_batch[order[k] + 1];
  }
  FEA_TRY(upload(&v->unit_batch, ranges));
  FEA_TRY(upload(&v->batch_visit, B.batch_visit));
  FEA_TRY(upload(&v->batch_flush, B.batch_flush));
  FEA_TRY(upload(&v->visit_nodes, B.visit_nodes));
  FEA_TRY(upload(&v->visit_off, B.visit_off));
  FEA_TRY(upload(&v->flush_meta, B.flush_meta));
  FEA_CUDA_TRY(cudaMalloc(&v->fnode, sizeof(float) * (size_t)N * (3 * n_eq + 3)));
  v->ok = true;
  return FEA_OK;
}

#include "fea_rowowned_kernel.cuh"

}  // namespace ro

fea_status plan_build(fea_mesh* m, fea_pattern* p, fea_rowowned_plan** out) {
  *out = nullptr;
  if (m->mixed || m->type != FEA_HEX8 || m->n_elem == 0) return FEA_OK;
  fea_rowowned_plan* P = new (std::nothrow) fea_rowowned_plan();
  if (!P) return fail(FEA_ERR_OOM, "host allocation failed");
  P->mesh = m;
  P->pattern = p;
  *out = P;
  return FEA_OK;
}

void plan_destroy(fea_rowowned_plan* P) {
  if (!P) return;
  for (auto& kv : P->variants) ro::free_variant(kv.second);
  cudaFree(P->elem_fnode);
  delete P;
}

int plan_key(int n_eq, int batch) { return n_eq | (std::max(0, std::min(batch, ro::BEMAX)) << 16); }

fea_status plan_prepare(fea_rowowned_plan* P, int n_eq, int batch, bool* ok) {
  *ok = false;
  if (!P) return FEA_OK;
  std::lock_guard<std::mutex> lk(P->mu);
  const int key = plan_key(n_eq, batch);
  auto it = P->variants.find(key);
  if (it == P->variants.end()) {
    ro::Variant* v = new (std::nothrow) ro::Variant();
    if (!v) return fail(FEA_ERR_OOM, "host allocation failed");
    fea_status st = ro::build_variant(P, n_eq, batch, v);
    if (st != FEA_OK) {
      ro::free_variant(v);
      return st;
    }
    it = P->variants.emplace(key, v).first;
  }
  *ok = it->second->ok;
  return FEA_OK;
}

namespace ro {
// Node-major copy of the per-step inputs, so that the (element, equation) threads of one
// element read contiguous memory: out[n][f n_eq + q] for f = k, s, phi_old, then
// out[n][3 n_eq + c] = u_c.  One block transposes tn nodes (a multiple of 32) through shared
// memory: a warp reads 4 tn bytes of one input row, then the block writes the tn records
// contiguously.
__global__ void k_fields_nodemajor(const float* __restrict__ kd, const float* __restrict__ sr,
                                   const float* __restrict__ phi, const float* __restrict__ vel, int64_t N, int n_eq,
                                   int tn, float* __restrict__ out) {
  extern __shared__ float tile[];  // [rec][tn + 1]
  const int rec = 3 * n_eq + 3, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * tn;
  for (int j = threadIdx.x >> 5; j < rec; j += blockDim.x >> 5) {
    const float* src = j < n_eq       ? kd + (int64_t)j * N
                       : j < 2 * n_eq ? sr + (int64_t)(j - n_eq) * N
                       : j < 3 * n_eq ? phi + (int64_t)(j - 2 * n_eq) * N
                                      : vel + (int64_t)(j - 3 * n_eq) * N;
    for (int k = lane; k < tn; k += 32) {
      const int64_t n = n0 + k;
      tile[j * (tn + 1) + k] = n < N ? __ldcs(src + n) : 0.f;
    }
  }
  __syncthreads();
  const int cnt = (int)((N - n0) < tn ? (N - n0) : tn);
  float* const o = out + n0 * rec;
  for (int idx = threadIdx.x; idx < cnt * rec; idx += blockDim.x) {
    const int node = idx / rec, j = idx - node * rec;
    o[idx] = tile[j * (tn + 1) + node];
  }
}

// Launches k_fields_nodemajor for equations eq0 .. eq0 + eq_count - 1 of a into out: 128 nodes
// per block, fewer where the [rec][tn + 1] tile would not fit in shared memory.
fea_status fields_nodemajor(const AsmArgs<float>& a, float* out, cudaStream_t s) {
  const int rec = 3 * a.eq_count + 3;
  int tn = 128;
  while (tn > 32 && sizeof(float) * (size_t)rec * (tn + 1) > 200 * 1024) tn /= 2;
  const size_t tsm = sizeof(float) * (size_t)rec * (tn + 1);
  if (tsm > (size_t)SMEM_LIMIT) return fail(FEA_ERR_ARG, "too many equations for the node-major field copy");
  const int64_t fo = (int64_t)a.eq0 * a.n_node;
  FEA_CUDA_TRY(cudaFuncSetAttribute(k_fields_nodemajor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
  k_fields_nodemajor<<<(unsigned)((a.n_node + tn - 1) / tn), 256, tsm, s>>>(a.kd + fo, a.sr + fo, a.phi + fo, a.vel,
                                                                            a.n_node, a.eq_count, tn, out);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}
}  // namespace ro

int plan_group_size(int n_eq, int groups) { return (n_eq + groups - 1) / groups; }

void plan_trim(fea_rowowned_plan* P, const std::vector<int>& keep) {
  if (!P) return;
  std::lock_guard<std::mutex> lk(P->mu);
  for (auto it = P->variants.begin(); it != P->variants.end();) {
    if (std::find(keep.begin(), keep.end(), it->first) == keep.end()) {
      ro::free_variant(it->second);
      it = P->variants.erase(it);
    } else {
      ++it;
    }
  }
}

// One group of equations [a.eq0, a.eq0 + a.eq_count) with the schedule of variant v.
static fea_status assemble_group(ro::Variant* v, const AsmArgs<float>& a, int accumulate, cudaStream_t s) {
  const int rec = 3 * a.eq_count + 3;
  FEA_TRY(ro::fields_nodemajor(a, v->fnode, s));
  ro::RoArgs r;
  r.a = a;
  r.fnode = v->fnode;
  r.rec = rec;
  r.unit_batch = v->unit_batch;
  r.batch_visit = v->batch_visit;
  r.batch_flush = v->batch_flush;
  r.visit_nodes = v->visit_nodes;
  r.visit_off = v->visit_off;
  r.flush_meta = reinterpret_cast<const int4*>(v->flush_meta);
  r.n_units = v->n_units;
  r.n_slots = v->n_slots;
  r.row_stride = v->row_stride;
  r.maxcol = v->maxcol;
  r.neqs = v->neqs;
  r.accumulate = accumulate;
  r.be = v->be;
  const bool two = a.mapping == FEA_MAP_TWO_THREADS_PER_ITEM && a.terms == FEA_TERM_ALL;
  auto kern = two ? ro::k_rowowned_hex8_half
                  : a.terms == FEA_TERM_ALL ? ro::k_rowowned_hex8<true> : ro::k_rowowned_hex8<false>;
  FEA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  unsigned grid = (unsigned)std::max(1, std::min(v->n_units, nsm));
  kern<<<grid, two ? ro::THREADS_HALF : ro::THREADS, v->smem, s>>>(r);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

fea_status hex8_elem(float*& fnode, size_t& fnode_bytes, const AsmArgs<float>& a, cudaStream_t s) {
  // node-major fields of all the launch's equations, in the caller's scratch (grown here)
  const int rec = 3 * a.eq_count + 3;
  const size_t need = sizeof(float) * (size_t)a.n_node * rec;
  if (fnode_bytes < need) {
    FEA_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(fnode);
    fnode = nullptr;
    fnode_bytes = 0;
    if (cudaMalloc(&fnode, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(FEA_ERR_OOM, "element kernel: %zu bytes of node-major fields", need);
    }
    fnode_bytes = need;
  }
  FEA_TRY(ro::fields_nodemajor(a, fnode, s));
  ro::RoArgs r{};
  r.a = a;
  r.fnode = fnode;
  r.rec = rec;
  const bool full = a.terms == FEA_TERM_ALL;
  // 96 elements take 180 KB; the residual kernel of the full operator runs two CTAs per SM: 48
  r.be = a.batch > 0 ? std::min(a.batch, 96) : ro::elem_batch(a.eq_count, a.resid && full ? 48 : 96);
  const size_t smem = sizeof(float) * (size_t)r.be * (ro::GEO_ELEM + ro::NEN * ro::RAW + ro::NEN);
  auto pick = [&](auto full_k, auto part_k) { return full ? full_k : part_k; };
  void (*kern)(ro::RoArgs) =
      a.resid ? pick(ro::k_hex8_elem<true, ro::EMODE_RESIDUAL>, ro::k_hex8_elem<false, ro::EMODE_RESIDUAL>)
      : a.em  ? pick(ro::k_hex8_elem<true, ro::EMODE_SCRATCH>, ro::k_hex8_elem<false, ro::EMODE_SCRATCH>)
              : pick(ro::k_hex8_elem<true, ro::EMODE_ATOMIC>, ro::k_hex8_elem<false, ro::EMODE_ATOMIC>);
  FEA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nb = (a.n_elem + r.be - 1) / r.be;
  int per_sm = 1;  // the matrix-free residual needs few registers: several CTAs per SM
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ro::THREADS, smem);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)nsm * std::max(per_sm, 1)));
  if (a.n_elem > 0) kern<<<grid, ro::THREADS, smem, s>>>(r);
  FEA_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return FEA_OK;
}

fea_status plan_elem(fea_rowowned_plan* P, const AsmArgs<float>& a, cudaStream_t s) {
  return hex8_elem(P->elem_fnode, P->elem_fnode_bytes, a, s);
}

fea_status plan_assemble(fea_rowowned_plan* P, const AsmArgs<float>& a, int accumulate, int groups, cudaStream_t s) {
  const int gsize = plan_group_size(a.eq_count, groups);
  ro::Variant* v = P->variants.at(plan_key(gsize, a.batch));
  if (v->unused_nodes && !accumulate)
    FEA_CUDA_TRY(cudaMemsetAsync(a.rhs + (int64_t)a.eq0 * a.n_node, 0,
                                 sizeof(float) * (size_t)a.eq_count * (size_t)a.n_node, s));
  // equations in groups of gsize: the geometry is recomputed per group, the row window of a
  // group holds gsize equations per row, so more rows fit (larger tiles, fuller batches)
  for (int g0 = 0; g0 < a.eq_count; g0 += gsize) {
    AsmArgs<float> ag = a;
    ag.eq0 = a.eq0 + g0;
    ag.eq_count = std::min(gsize, a.eq_count - g0);
    FEA_TRY(assemble_group(v, ag, accumulate, s));
  }
  return FEA_OK;
}

}  // namespace fea
