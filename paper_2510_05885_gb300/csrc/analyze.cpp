// Host symbolic analysis: KKT pattern, nested-dissection ordering,
// elimination tree, relaxed supernodes and the multifrontal schedule.
//
// Done once per pattern and reused for every numeric factorisation, as the
// paper reuses the symbolic factorisation across Newton steps (Section 4.1).
// The ordering is free because the stabilized system is symmetric
// quasi-definite once H + Sigma + delta I is positive definite, and such a
// matrix has an LDL^T factorisation under every symmetric permutation
// (Section 3.2); the condensed system is then positive definite (Section 3.4).
#include "plan.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <exception>
#include <mutex>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <thread>

namespace ncl {
namespace {

// Run f(lo, hi) over [0, n) split into contiguous ranges on up to 16 host
// threads (each range is processed by exactly one thread, so results do not
// depend on the thread count when f writes only its own range).
template <typename F>
void parallel_ranges(int64_t n, int64_t min_chunk, F&& f) {
  const int64_t hw = std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)std::thread::hardware_concurrency()));
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw, n / std::max<int64_t>(1, min_chunk)));
  if (nt <= 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; t++) th.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

struct Contrib {
  uint64_t key;   // col * dim + row  (lower: row >= col)
  int32_t a, b;
  int8_t type;    // 0 H, 1 J, 2 primal diag, 3 dual diag, 4 J^T J product
};

struct PatternError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

// ---------------------------------------------------------------------------
// 1. KKT lower pattern and value recipes
// ---------------------------------------------------------------------------
void build_pattern(const AnalyzeInput& in, Plan& P) {
  P.form = in.form;
  P.inst.resize(in.count);
  int64_t row = 0, hoff = 0, joff = 0, soff = 0, coff = 0;
  for (int i = 0; i < in.count; i++) {
    Instance& I = P.inst[i];
    I.n = in.n[i];
    I.m = in.m[i];
    if (I.n < 0 || I.m < 0) throw PatternError("pattern: negative size");
    if (I.n > 0 && (!in.H_rowptr[i] || (in.H_rowptr[i][I.n] > 0 && !in.H_colind[i])))
      throw PatternError("pattern: NULL H pattern");
    if (I.m > 0 && (!in.J_rowptr[i] || (in.J_rowptr[i][I.m] > 0 && !in.J_colind[i])))
      throw PatternError("pattern: NULL J pattern");
    I.dim = I.n + (in.form == 0 ? I.m : 0);
    I.row_off = row;
    I.H_off = hoff;
    I.J_off = joff;
    I.S_off = soff;
    I.nnzH = I.n > 0 ? in.H_rowptr[i][I.n] : 0;
    I.nnzJ = I.m > 0 ? in.J_rowptr[i][I.m] : 0;
    if (I.n > 0 && in.H_rowptr[i][0] != 0) throw PatternError("pattern: H_rowptr[0] != 0");
    if (I.m > 0 && in.J_rowptr[i][0] != 0) throw PatternError("pattern: J_rowptr[0] != 0");
    row += I.dim;
    hoff += I.nnzH;
    joff += I.nnzJ;
    soff += I.n;
    coff += I.m;
  }
  P.dim = row;
  P.nnzH_total = hoff;
  P.nnzJ_total = joff;
  P.nS_total = soff;
  P.mcon_total = coff;
  if (P.dim >= (int64_t)INT32_MAX) throw PatternError("pattern: dimension too large");
  if (hoff >= INT32_MAX || joff >= INT32_MAX) throw PatternError("pattern: too many values");

  const uint64_t D = (uint64_t)P.dim;
  P.row_inst.assign(P.dim, 0);
  P.row_sign.assign(P.dim, 1);
  P.H_row.resize(hoff);
  P.H_col.resize(hoff);
  P.J_row.resize(joff);
  P.J_col.resize(joff);
  P.J_inst.resize(joff);
  P.var_row.resize(soff);
  P.con_row.assign(coff, -1);
  P.J_rowptr_all.assign(coff + 1, 0);

  // validation, in the order the pattern is read
  for (int i = 0; i < in.count; i++) {
    const Instance& I = P.inst[i];
    const int32_t* Hp = in.H_rowptr[i];
    const int32_t* Hc = in.H_colind[i];
    const int32_t* Jp = in.J_rowptr[i];
    const int32_t* Jc = in.J_colind[i];
    for (int32_t r = 0; r < I.n; r++) {
      if (Hp[r + 1] < Hp[r]) throw PatternError("pattern: H_rowptr decreasing");
      for (int32_t p = Hp[r]; p < Hp[r + 1]; p++) {
        int32_t c = Hc[p];
        if (c < 0 || c > r) throw PatternError("pattern: H entry outside the lower triangle");
        if (p > Hp[r] && c <= Hc[p - 1]) throw PatternError("pattern: H columns not sorted/unique");
      }
    }
    for (int32_t r = 0; r < I.m; r++) {
      if (Jp[r + 1] < Jp[r]) throw PatternError("pattern: J_rowptr decreasing");
      for (int32_t p = Jp[r]; p < Jp[r + 1]; p++) {
        int32_t c = Jc[p];
        if (c < 0 || c >= I.n) throw PatternError("pattern: J column out of range");
        if (p > Jp[r] && c <= Jc[p - 1]) throw PatternError("pattern: J columns not sorted/unique");
      }
    }
  }

  // contributions: one work unit per H row and per J row of every instance,
  // each writing its contributions at a prefix offset (units in parallel)
  std::vector<int64_t> unit_off(in.count + 1, 0);   // first unit of each instance
  for (int i = 0; i < in.count; i++) unit_off[i + 1] = unit_off[i] + P.inst[i].n + P.inst[i].m;
  const int64_t nunits = unit_off[in.count];
  std::vector<int64_t> coff_u((size_t)nunits + 1, 0);
  {
    int64_t u = 0, con = 0;
    for (int i = 0; i < in.count; i++) {
      const Instance& I = P.inst[i];
      const int32_t* Hp = in.H_rowptr[i];
      const int32_t* Jp = in.J_rowptr[i];
      for (int32_t r = 0; r < I.n; r++, u++) coff_u[u + 1] = (Hp[r + 1] - Hp[r]) + 1;
      for (int32_t r = 0; r < I.m; r++, u++, con++) {
        const int64_t k = Jp[r + 1] - Jp[r];
        coff_u[u + 1] = in.form == 0 ? k + 1 : k * (k + 1) / 2;
        P.J_rowptr_all[con + 1] = P.J_rowptr_all[con] + k;
      }
    }
    for (int64_t q = 0; q < nunits; q++) coff_u[q + 1] += coff_u[q];
  }
  std::vector<Contrib> C((size_t)coff_u[nunits]);
  std::vector<int64_t> con0(in.count + 1, 0);
  for (int i = 0; i < in.count; i++) con0[i + 1] = con0[i] + P.inst[i].m;
  parallel_ranges(nunits, 4096, [&](int64_t u0, int64_t u1) {
    int i = (int)(std::upper_bound(unit_off.begin(), unit_off.end(), u0) - unit_off.begin()) - 1;
    for (int64_t u = u0; u < u1; u++) {
      while (u >= unit_off[i + 1]) i++;
      const Instance& I = P.inst[i];
      const int32_t* Hp = in.H_rowptr[i];
      const int32_t* Hc = in.H_colind[i];
      const int32_t* Jp = in.J_rowptr[i];
      const int32_t* Jc = in.J_colind[i];
      int64_t q = coff_u[u];
      const int64_t lu = u - unit_off[i];
      if (lu < I.n) {
        const int32_t r = (int32_t)lu;
        P.var_row[I.S_off + r] = (int32_t)(I.row_off + r);
        for (int32_t p = Hp[r]; p < Hp[r + 1]; p++) {
          const uint64_t gr = I.row_off + r, gc = I.row_off + Hc[p];
          C[q++] = {gc * D + gr, (int32_t)(I.H_off + p), 0, 0};
          P.H_row[I.H_off + p] = (int32_t)gr;
          P.H_col[I.H_off + p] = (int32_t)gc;
        }
        const uint64_t g = I.row_off + r;
        C[q++] = {g * D + g, (int32_t)(I.S_off + r), 0, 2};
      } else {
        const int32_t r = (int32_t)(lu - I.n);
        const int64_t con = con0[i] + r;
        for (int32_t p = Jp[r]; p < Jp[r + 1]; p++) {
          P.J_col[I.J_off + p] = (int32_t)(I.row_off + Jc[p]);
          P.J_inst[I.J_off + p] = i;
          P.J_row[I.J_off + p] = (int32_t)con;
        }
        if (in.form == 0) {
          const uint64_t gr = I.row_off + I.n + r;
          P.con_row[con] = (int32_t)gr;
          for (int32_t p = Jp[r]; p < Jp[r + 1]; p++) {
            const uint64_t gc = I.row_off + Jc[p];
            C[q++] = {gc * D + gr, (int32_t)(I.J_off + p), 0, 1};
          }
          C[q++] = {gr * D + gr, i, 0, 3};
        } else {
          // rho * J^T J: every pair of entries of one constraint row
          for (int32_t a = Jp[r]; a < Jp[r + 1]; a++)
            for (int32_t b = Jp[r]; b <= a; b++) {
              const uint64_t gr = I.row_off + Jc[a], gc = I.row_off + Jc[b];
              C[q++] = {gc * D + gr, (int32_t)(I.J_off + a), (int32_t)(I.J_off + b), 4};
            }
        }
      }
    }
  });
  for (int i = 0; i < in.count; i++) {
    const Instance& I = P.inst[i];
    for (int64_t r = 0; r < I.dim; r++) {
      P.row_inst[I.row_off + r] = i;
      P.row_sign[I.row_off + r] = (in.form == 0 && r >= I.n) ? -1 : 1;
    }
  }

  // order by (key, type, a, b): a counting sort by column (the scatter in
  // parallel, in any order), then each column's few contributions by (row,
  // type, a, b), a total order, so the result does not depend on the scatter
  std::vector<int64_t> cp((size_t)P.dim + 1, 0);
  {
    auto less = [](const Contrib& x, const Contrib& y) {
      if (x.key != y.key) return x.key < y.key;
      if (x.type != y.type) return x.type < y.type;
      if (x.a != y.a) return x.a < y.a;
      return x.b < y.b;
    };
    std::vector<std::atomic<int64_t>> cnt((size_t)P.dim);
    for (auto& x : cnt) x.store(0, std::memory_order_relaxed);
    const int64_t nc = (int64_t)C.size();
    parallel_ranges(nc, 1 << 16, [&](int64_t lo, int64_t hi) {
      for (int64_t q = lo; q < hi; q++) cnt[C[q].key / D].fetch_add(1, std::memory_order_relaxed);
    });
    for (int64_t i = 0; i < P.dim; i++) cp[i + 1] = cp[i] + cnt[i].load(std::memory_order_relaxed);
    for (int64_t i = 0; i < P.dim; i++) cnt[i].store(cp[i], std::memory_order_relaxed);
    std::vector<Contrib> S(C.size());
    parallel_ranges(nc, 1 << 16, [&](int64_t lo, int64_t hi) {
      for (int64_t q = lo; q < hi; q++) S[cnt[C[q].key / D].fetch_add(1, std::memory_order_relaxed)] = C[q];
    });
    std::vector<Contrib>().swap(C);
    parallel_ranges(P.dim, 4096, [&](int64_t lo, int64_t hi) {
      for (int64_t c = lo; c < hi; c++)
        if (cp[c + 1] - cp[c] > 1) std::sort(S.begin() + cp[c], S.begin() + cp[c + 1], less);
    });
    C.swap(S);
  }

  // group into entries, column by column in parallel: count the entries and
  // products of each column, then fill at the prefix offsets
  std::vector<int64_t> eoff((size_t)P.dim + 1, 0), poff((size_t)P.dim + 1, 0);
  parallel_ranges(P.dim, 4096, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; c++) {
      int64_t ne = 0, np = 0;
      for (int64_t q = cp[c]; q < cp[c + 1]; q++) {
        if (q == cp[c] || C[q].key != C[q - 1].key) ne++;
        if (C[q].type == 4) np++;
      }
      eoff[c + 1] = ne;
      poff[c + 1] = np;
    }
  });
  for (int64_t c = 0; c < P.dim; c++) {
    eoff[c + 1] += eoff[c];
    poff[c + 1] += poff[c];
  }
  const size_t nent = (size_t)eoff[P.dim], npair = (size_t)poff[P.dim];
  P.A_colptr.assign(eoff.begin(), eoff.end());
  P.A_row.resize(nent);
  P.e_h.resize(nent);
  P.e_j.resize(nent);
  P.e_kind.resize(nent);
  P.e_var.resize(nent);
  P.pair_ptr.resize(nent + 1);
  P.pair_ptr[0] = 0;
  P.pair_p.resize(npair);
  P.pair_q.resize(npair);
  parallel_ranges(P.dim, 4096, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; c++) {
      int64_t e = eoff[c], np = poff[c];
      int64_t k = cp[c];
      while (k < cp[c + 1]) {
        const uint64_t key = C[k].key;
        int32_t h = -1, j = -1, var = -1;
        int8_t kind = DIAG_NONE;
        for (; k < cp[c + 1] && C[k].key == key; k++) {
          const Contrib& ct = C[k];
          switch (ct.type) {
            case 0: h = ct.a; break;
            case 1: j = ct.a; break;
            case 2: kind = DIAG_PRIMAL; var = ct.a; break;
            case 3: kind = DIAG_DUAL; var = ct.a; break;
            case 4:
              P.pair_p[np] = ct.a;
              P.pair_q[np++] = ct.b;
              break;
          }
        }
        P.A_row[e] = (int32_t)(key % D);
        P.e_h[e] = h;
        P.e_j[e] = j;
        P.e_kind[e] = kind;
        P.e_var[e] = var;
        P.pair_ptr[e + 1] = np;
        e++;
      }
    }
  });
  P.nnzA = (int64_t)P.A_row.size();
  if (P.nnzA >= INT32_MAX) throw PatternError("pattern: too many KKT entries");
  std::vector<Contrib>().swap(C);

  // full symmetric CSR (natural numbering)
  P.F_rowptr.assign(P.dim + 1, 0);
  for (int64_t c = 0; c < P.dim; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
      int64_t r = P.A_row[p];
      P.F_rowptr[r + 1]++;
      if (r != c) P.F_rowptr[c + 1]++;
    }
  for (int64_t r = 0; r < P.dim; r++) P.F_rowptr[r + 1] += P.F_rowptr[r];
  P.F_col.resize(P.F_rowptr[P.dim]);
  P.F_src.resize(P.F_rowptr[P.dim]);
  std::vector<int64_t> fill(P.F_rowptr.begin(), P.F_rowptr.end() - 1);
  // rows of column c arrive in increasing column order if we sweep columns
  // for the upper part first... simplest: fill then sort each row by column.
  for (int64_t c = 0; c < P.dim; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
      int64_t r = P.A_row[p];
      P.F_col[fill[r]] = (int32_t)c;
      P.F_src[fill[r]++] = (int32_t)p;
      if (r != c) {
        P.F_col[fill[c]] = (int32_t)r;
        P.F_src[fill[c]++] = (int32_t)p;
      }
    }
  // rows are already sorted: for row r the entries (r, c<=r) come from
  // columns c in increasing order, then (r, c>r) from column r in increasing
  // row order -- both appended in increasing c.  Verify cheaply in debug.
}

// ---------------------------------------------------------------------------
// 2. Nested dissection (automatic, level-structure separators)
//
// A subgraph is split by a breadth-first level structure rooted at a
// pseudo-peripheral vertex: one level is a vertex separator (edges only join
// adjacent levels).  Among the levels that leave at least 30% of the
// vertices on each side the smallest is taken, then trimmed of vertices
// with no neighbour beyond it.  Parts are ordered before the separator,
// recursively; leaves are ordered by minimum degree on their own graph.
// ---------------------------------------------------------------------------
struct Graph {
  std::vector<int64_t> xadj;
  std::vector<int32_t> adj;
  int64_t n = 0;
};

Graph make_graph(const Plan& P) {
  Graph G;
  G.n = P.dim;
  G.xadj.assign(P.dim + 1, 0);
  for (int64_t c = 0; c < P.dim; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
      int64_t r = P.A_row[p];
      if (r == c) continue;
      G.xadj[r + 1]++;
      G.xadj[c + 1]++;
    }
  for (int64_t i = 0; i < P.dim; i++) G.xadj[i + 1] += G.xadj[i];
  G.adj.resize(G.xadj[P.dim]);
  std::vector<int64_t> f(G.xadj.begin(), G.xadj.end() - 1);
  for (int64_t c = 0; c < P.dim; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
      int64_t r = P.A_row[p];
      if (r == c) continue;
      G.adj[f[r]++] = (int32_t)c;
      G.adj[f[c]++] = (int32_t)r;
    }
  return G;
}

// Vertex -> subgraph id of the task that owns it (0: none).  Tasks own
// disjoint vertex sets and only compare a neighbour's id with their own, so
// concurrent tasks never observe each other's ids as their own; the atomics
// make those reads well defined.
using PartArray = std::vector<std::atomic<int32_t>>;

inline int32_t part_of(const PartArray& part, int32_t v) { return part[v].load(std::memory_order_relaxed); }
inline void set_part(PartArray& part, int32_t v, int32_t id) { part[v].store(id, std::memory_order_relaxed); }

// minimum degree on a small dense graph (k <= 256): bitset elimination graph
void leaf_min_degree(const Graph& G, const PartArray& part, int32_t id,
                     const std::vector<int32_t>& verts, std::vector<int32_t>& local, int32_t* out) {
  const int k = (int)verts.size();
  const int W = (k + 63) / 64;
  std::vector<uint64_t> adj((size_t)k * W, 0);
  for (int a = 0; a < k; a++) local[verts[a]] = a;
  for (int a = 0; a < k; a++) {
    int32_t v = verts[a];
    for (int64_t p = G.xadj[v]; p < G.xadj[v + 1]; p++) {
      int32_t u = G.adj[p];
      if (part_of(part, u) != id) continue;
      int b = local[u];
      adj[(size_t)a * W + b / 64] |= 1ull << (b % 64);
    }
  }
  std::vector<char> done(k, 0);
  std::vector<int> deg(k);
  for (int a = 0; a < k; a++) {
    int d = 0;
    for (int w = 0; w < W; w++) d += __builtin_popcountll(adj[(size_t)a * W + w]);
    deg[a] = d;
  }
  for (int t = 0; t < k; t++) {
    int best = -1;
    for (int a = 0; a < k; a++)
      if (!done[a] && (best < 0 || deg[a] < deg[best])) best = a;
    done[best] = 1;
    out[t] = verts[best];
    uint64_t* rb = &adj[(size_t)best * W];
    // neighbours of best become a clique
    for (int w = 0; w < W; w++) {
      uint64_t bits = rb[w];
      while (bits) {
        int b = w * 64 + __builtin_ctzll(bits);
        bits &= bits - 1;
        uint64_t* ru = &adj[(size_t)b * W];
        for (int x = 0; x < W; x++) ru[x] |= rb[x];
        ru[b / 64] &= ~(1ull << (b % 64));
        ru[best / 64] &= ~(1ull << (best % 64));
        int d = 0;
        for (int x = 0; x < W; x++) d += __builtin_popcountll(ru[x]);
        deg[b] = d;
      }
    }
    for (int w = 0; w < W; w++) rb[w] = 0;
  }
  for (int a = 0; a < k; a++) local[verts[a]] = -1;
}

struct NdTask {
  std::vector<int32_t> v;
  int64_t lo;
};

// Shared state of one nested dissection; a task reads and writes only the
// entries of its own vertices (part, lvl, local) and its own range of order.
struct NdState {
  const Graph& G;
  int leaf;
  std::vector<int32_t> order, lvl, local;
  PartArray part;
  std::atomic<int32_t> next_id{1};
  NdState(const Graph& g, int lf) : G(g), leaf(lf), order(g.n, -1), lvl(g.n, -1), local(g.n, -1), part(g.n) {
    for (auto& x : part) x.store(0, std::memory_order_relaxed);
  }
};

// One task: order a leaf, or split off a component, or find a level-structure
// separator (ordered last in the task's range) and return the two parts.
void nd_task(NdState& S, NdTask& t, std::vector<int32_t>& queue, std::vector<NdTask>& out) {
  const Graph& G = S.G;
  const int64_t sz = (int64_t)t.v.size();
  if (sz == 0) return;
  if ((int64_t)queue.size() < sz) queue.resize(sz);
  const int32_t id = S.next_id.fetch_add(1, std::memory_order_relaxed);
  for (int32_t v : t.v) set_part(S.part, v, id);
  auto release = [&] {
    for (int32_t v : t.v) set_part(S.part, v, 0);
  };
  if (sz <= S.leaf) {
    leaf_min_degree(G, S.part, id, t.v, S.local, &S.order[t.lo]);
    release();
    return;
  }
  // BFS restricted to the task's subgraph from root; fills lvl[] and
  // queue[0..reached); nlev = number of levels
  auto bfs = [&](int32_t root, int& nlev) -> int64_t {
    int64_t head = 0, tail = 0;
    queue[tail++] = root;
    S.lvl[root] = 0;
    int maxl = 0;
    while (head < tail) {
      int32_t v = queue[head++];
      int lv = S.lvl[v];
      for (int64_t p = G.xadj[v]; p < G.xadj[v + 1]; p++) {
        int32_t u = G.adj[p];
        if (part_of(S.part, u) != id || S.lvl[u] >= 0) continue;
        S.lvl[u] = lv + 1;
        if (lv + 1 > maxl) maxl = lv + 1;
        queue[tail++] = u;
      }
    }
    nlev = maxl + 1;
    return tail;
  };
  auto clear_lvl = [&](int64_t cnt) {
    for (int64_t i = 0; i < cnt; i++) S.lvl[queue[i]] = -1;
  };
  // pseudo-peripheral root: two sweeps from the vertex of smallest degree
  int32_t root = t.v[0];
  int nlev = 0;
  int64_t reached = bfs(root, nlev);
  if (reached < sz) {
    // disconnected: split off this component
    std::vector<int32_t> comp(queue.begin(), queue.begin() + reached);
    clear_lvl(reached);
    for (int32_t v : comp) set_part(S.part, v, -1);
    std::vector<int32_t> rest;
    rest.reserve(sz - reached);
    for (int32_t v : t.v)
      if (part_of(S.part, v) == id) rest.push_back(v);
    release();
    out.push_back(NdTask{std::move(comp), t.lo});
    out.push_back(NdTask{std::move(rest), t.lo + reached});
    return;
  }
  for (int sweep = 0; sweep < 2; sweep++) {
    // farthest vertex of smallest degree in the last level
    int32_t best = queue[reached - 1];
    int lastl = S.lvl[best];
    int64_t bestdeg = G.xadj[best + 1] - G.xadj[best];
    for (int64_t i = reached - 1; i >= 0 && S.lvl[queue[i]] == lastl; i--) {
      int64_t d = G.xadj[queue[i] + 1] - G.xadj[queue[i]];
      if (d < bestdeg) {
        bestdeg = d;
        best = queue[i];
      }
    }
    clear_lvl(reached);
    int nl2 = 0;
    reached = bfs(best, nl2);
    if (nl2 <= nlev && sweep > 0) {
      nlev = nl2;
      break;
    }
    nlev = nl2;
  }
  if (nlev < 3) {
    // (nearly) complete subgraph: no useful separator
    clear_lvl(reached);
    if (sz <= 256) leaf_min_degree(G, S.part, id, t.v, S.local, &S.order[t.lo]);
    else
      for (int64_t i = 0; i < sz; i++) S.order[t.lo + i] = t.v[i];
    release();
    return;
  }
  std::vector<int64_t> cnt(nlev + 1, 0);
  for (int64_t i = 0; i < reached; i++) cnt[S.lvl[queue[i]] + 1]++;
  std::vector<int64_t> levsz(nlev);
  for (int l = 0; l < nlev; l++) levsz[l] = cnt[l + 1];
  for (int l = 0; l < nlev; l++) cnt[l + 1] += cnt[l];
  // choose the separator level
  int sep = -1;
  double bestcost = 1e300;
  for (int l = 1; l < nlev - 1; l++) {
    int64_t below = cnt[l], above = sz - cnt[l + 1];
    double lo = (double)std::min(below, above), hi = (double)std::max(below, above);
    if (lo < 0.3 * (double)sz && !(sep < 0 && l == nlev / 2)) continue;
    double cost = (double)levsz[l] * (1.0 + 0.5 * (hi - lo) / (double)sz);
    if (cost < bestcost) {
      bestcost = cost;
      sep = l;
    }
  }
  if (sep < 0) sep = nlev / 2;
  std::vector<int32_t> A, B, Sp;
  A.reserve(cnt[sep]);
  B.reserve(sz - cnt[sep + 1]);
  for (int64_t i = 0; i < reached; i++) {
    int32_t v = queue[i];
    int l = S.lvl[v];
    if (l < sep) A.push_back(v);
    else if (l > sep) B.push_back(v);
    else {
      bool above = false;
      for (int64_t p = G.xadj[v]; p < G.xadj[v + 1]; p++) {
        int32_t u = G.adj[p];
        if (part_of(S.part, u) == id && S.lvl[u] == sep + 1) {
          above = true;
          break;
        }
      }
      if (above) Sp.push_back(v);
      else A.push_back(v);
    }
  }
  clear_lvl(reached);
  release();
  int64_t hi = t.lo + sz;
  for (size_t i = 0; i < Sp.size(); i++) S.order[hi - (int64_t)Sp.size() + (int64_t)i] = Sp[i];
  int64_t na = (int64_t)A.size();
  out.push_back(NdTask{std::move(A), t.lo});
  out.push_back(NdTask{std::move(B), t.lo + na});
}

// Tasks are independent (disjoint vertices and ranges of order), so they run
// on a pool of host threads; the ordering does not depend on their timing.
std::vector<int32_t> nested_dissection(const Graph& G, int leaf) {
  NdState S(G, leaf);
  std::vector<NdTask> stack;
  {
    NdTask t;
    t.v.resize(G.n);
    std::iota(t.v.begin(), t.v.end(), 0);
    t.lo = 0;
    stack.push_back(std::move(t));
  }
  const int nth = (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)std::thread::hardware_concurrency()));
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;
  std::exception_ptr failure;
  auto worker = [&] {
    std::vector<int32_t> queue;
    std::vector<NdTask> out;
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv.wait(lk, [&] { return !stack.empty() || active == 0 || failure; });
      if (failure || (stack.empty() && active == 0)) break;
      NdTask t = std::move(stack.back());
      stack.pop_back();
      active++;
      lk.unlock();
      out.clear();
      try {
        nd_task(S, t, queue, out);
      } catch (...) {
        lk.lock();
        if (!failure) failure = std::current_exception();
        active--;
        cv.notify_all();
        break;
      }
      lk.lock();
      for (auto& o : out) stack.push_back(std::move(o));
      active--;
      cv.notify_all();
    }
  };
  if (nth <= 1 || G.n < 20000) {
    worker();
  } else {
    std::vector<std::thread> th;
    for (int i = 0; i < nth; i++) th.emplace_back(worker);
    for (auto& x : th) x.join();
  }
  if (failure) std::rethrow_exception(failure);
  return std::move(S.order);
}

// ---------------------------------------------------------------------------
// 3. Elimination tree, postorder, supernodes
// ---------------------------------------------------------------------------

// etree of the matrix whose strictly-upper pattern by column is (up_ptr, up_row)
std::vector<int32_t> etree(int64_t N, const std::vector<int64_t>& up_ptr,
                           const std::vector<int32_t>& up_row) {
  std::vector<int32_t> parent(N, -1), anc(N, -1);
  for (int64_t k = 0; k < N; k++) {
    for (int64_t p = up_ptr[k]; p < up_ptr[k + 1]; p++) {
      int32_t i = up_row[p];
      while (i != -1 && i < k) {
        int32_t nx = anc[i];
        anc[i] = (int32_t)k;
        if (nx == -1) {
          parent[i] = (int32_t)k;
          break;
        }
        i = nx;
      }
    }
  }
  return parent;
}

std::vector<int32_t> postorder(int64_t N, const std::vector<int32_t>& parent) {
  std::vector<int32_t> head(N, -1), next(N, -1), post;
  post.reserve(N);
  for (int64_t j = N - 1; j >= 0; j--) {
    if (parent[j] == -1) continue;
    next[j] = head[parent[j]];
    head[parent[j]] = (int32_t)j;
  }
  std::vector<int32_t> st;
  for (int64_t r = 0; r < N; r++) {
    if (parent[r] != -1) continue;
    st.push_back((int32_t)r);
    while (!st.empty()) {
      int32_t v = st.back();
      if (head[v] != -1) {
        int32_t c = head[v];
        head[v] = next[c];
        st.push_back(c);
      } else {
        st.pop_back();
        post.push_back(v);
      }
    }
  }
  return post;
}

// strictly-upper pattern by column of P A P^T given perm (new->old) / iperm
void permuted_upper(const Plan& P, const std::vector<int32_t>& iperm, std::vector<int64_t>& ptr,
                    std::vector<int32_t>& row) {
  const int64_t N = P.dim;
  ptr.assign(N + 1, 0);
  for (int64_t c = 0; c < N; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
      int64_t r = P.A_row[p];
      if (r == c) continue;
      int32_t a = iperm[r], b = iperm[c];
      ptr[std::max(a, b) + 1]++;
    }
  for (int64_t i = 0; i < N; i++) ptr[i + 1] += ptr[i];
  row.resize(ptr[N]);
  std::vector<int64_t> f(ptr.begin(), ptr.end() - 1);
  for (int64_t c = 0; c < N; c++)
    for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
      int64_t r = P.A_row[p];
      if (r == c) continue;
      int32_t a = iperm[r], b = iperm[c];
      row[f[std::max(a, b)]++] = std::min(a, b);
    }
}

struct SNode {
  std::vector<int32_t> cols;   // columns (perm1 numbering), in elimination order
  std::vector<int32_t> below;  // rows below the columns (perm1 numbering, sorted)
  int64_t nrow = 0, ncol = 0;
  int64_t zeros = 0;           // padded zeros in the trapezoid
  int32_t parent = -1;         // fundamental-tree parent
  int32_t rep = -1;            // representative after amalgamation (-1 = self)
  std::vector<int32_t> kids;
};

inline int64_t trap(int64_t ncol, int64_t nrow) { return ncol * nrow - ncol * (ncol - 1) / 2; }

int32_t find_rep(std::vector<SNode>& S, int32_t s) {
  while (S[s].rep >= 0) s = S[s].rep;
  return s;
}

bool relax_ok(int64_t ncol, double zfrac) {
  if (ncol <= 8) return true;
  if (ncol <= 32) return zfrac <= 0.5;
  if (ncol <= 64) return zfrac <= 0.2;
  if (ncol <= 128) return zfrac <= 0.08;
  return zfrac <= 0.03;
}

void symbolic(Plan& P, const std::vector<int32_t>& perm0) {
  const int64_t N = P.dim;
  std::vector<int32_t> iperm0(N);
  for (int64_t k = 0; k < N; k++) iperm0[perm0[k]] = (int32_t)k;
  std::vector<int64_t> up_ptr;
  std::vector<int32_t> up_row;
  permuted_upper(P, iperm0, up_ptr, up_row);
  std::vector<int32_t> parent0 = etree(N, up_ptr, up_row);
  std::vector<int32_t> post = postorder(N, parent0);
  // perm1 = perm0 o post
  std::vector<int32_t> perm1(N), iperm1(N), ipost(N);
  for (int64_t k = 0; k < N; k++) {
    perm1[k] = perm0[post[k]];
    ipost[post[k]] = (int32_t)k;
  }
  for (int64_t k = 0; k < N; k++) iperm1[perm1[k]] = (int32_t)k;
  std::vector<int32_t> parent(N);
  for (int64_t k = 0; k < N; k++) {
    int32_t p0 = parent0[post[k]];
    parent[k] = p0 < 0 ? -1 : ipost[p0];
  }
  // lower pattern by column in perm1 numbering (rows > col)
  std::vector<int64_t> lo_ptr(N + 1, 0);
  std::vector<int32_t> lo_row;
  {
    for (int64_t c = 0; c < N; c++)
      for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
        int64_t r = P.A_row[p];
        if (r == c) continue;
        int32_t a = iperm1[r], b = iperm1[c];
        lo_ptr[std::min(a, b) + 1]++;
      }
    for (int64_t i = 0; i < N; i++) lo_ptr[i + 1] += lo_ptr[i];
    lo_row.resize(lo_ptr[N]);
    std::vector<int64_t> f(lo_ptr.begin(), lo_ptr.end() - 1);
    for (int64_t c = 0; c < N; c++)
      for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
        int64_t r = P.A_row[p];
        if (r == c) continue;
        int32_t a = iperm1[r], b = iperm1[c];
        lo_row[f[std::min(a, b)]++] = std::max(a, b);
      }
  }
  std::vector<int32_t> nchild(N, 0);
  for (int64_t j = 0; j < N; j++)
    if (parent[j] >= 0) nchild[parent[j]]++;

  // column counts and fundamental supernodes.  Column j joins the supernode
  // t of its only child j-1 when its own lower entries all lie in the
  // structure of j-1 (then struct(j) = struct(j-1) minus j and the counts
  // differ by one); only the first column of each supernode gets an explicit
  // structure: its lower entries and the structures of its children's
  // supernodes, whose last columns are its etree children.
  std::vector<int32_t> chead(N, -1), cnext(N, -1);
  for (int64_t c = N - 1; c >= 0; c--)
    if (parent[c] >= 0) {
      cnext[c] = chead[parent[c]];
      chead[parent[c]] = (int32_t)c;
    }
  std::vector<int32_t> mark(N, -1);   // supernode whose first-column structure holds the row
  std::vector<int64_t> colcount(N);
  std::vector<SNode> S;
  std::vector<int32_t> sn_of(N);
  P.nnzL = 0;
  P.flops = 0;
  P.inst_flops.assign(P.inst.size(), 0.0);
  P.inst_nnzL.assign(P.inst.size(), 0);
  for (int64_t j = 0; j < N; j++) {
    bool join = false;
    if (nchild[j] == 1 && j > 0 && parent[j - 1] == j) {
      const int32_t t = sn_of[j - 1];
      join = true;
      for (int64_t p = lo_ptr[j]; p < lo_ptr[j + 1]; p++)
        if (mark[lo_row[p]] != t) {
          join = false;
          break;
        }
    }
    int64_t cj;
    if (join) {
      const int32_t t = sn_of[j - 1];
      cj = colcount[j - 1] - 1;
      S[t].cols.push_back((int32_t)j);
      S[t].ncol++;
      sn_of[j] = t;
    } else {
      const int32_t s = (int32_t)S.size();
      std::vector<int32_t> st;
      for (int32_t c = chead[j]; c >= 0; c = cnext[c]) {
        // struct(c): the rows of c's supernode below its columns
        const SNode& T = S[sn_of[c]];
        for (size_t q = (size_t)(T.ncol - 1); q < T.below.size(); q++) {
          const int32_t r = T.below[q];
          if (r > j && mark[r] != s) {
            mark[r] = s;
            st.push_back(r);
          }
        }
      }
      for (int64_t p = lo_ptr[j]; p < lo_ptr[j + 1]; p++) {
        const int32_t r = lo_row[p];
        if (mark[r] != s) {
          mark[r] = s;
          st.push_back(r);
        }
      }
      std::sort(st.begin(), st.end());
      cj = (int64_t)st.size();
      SNode sn;
      sn.cols.push_back((int32_t)j);
      sn.ncol = 1;
      sn.below = std::move(st);
      sn.nrow = 1 + cj;
      S.push_back(std::move(sn));
      sn_of[j] = s;
    }
    colcount[j] = cj;
    P.nnzL += cj;
    const double fj = (double)cj * (double)cj + 3.0 * (double)cj;
    P.flops += fj;
    const int32_t ij = P.row_inst[perm1[j]];
    P.inst_flops[ij] += fj;
    P.inst_nnzL[ij] += cj;
  }
  // within a fundamental supernode, below rows = below(first) minus its own cols
  for (auto& s : S) {
    if (s.ncol > 1) {
      std::vector<int32_t> b;
      b.reserve(s.below.size());
      int32_t last = s.cols.back();
      for (int32_t r : s.below)
        if (r > last) b.push_back(r);
      s.below.swap(b);
    }
    s.nrow = s.ncol + (int64_t)s.below.size();
  }
  const int32_t ns0 = (int32_t)S.size();
  for (int32_t s = 0; s < ns0; s++) {
    int32_t last = S[s].cols.back();
    S[s].parent = parent[last] < 0 ? -1 : sn_of[parent[last]];
    if (S[s].parent >= 0) S[S[s].parent].kids.push_back(s);
  }
  // relaxed amalgamation, bottom-up (supernodes are in postorder)
  for (int32_t p = 0; p < ns0; p++) {
    std::vector<int32_t> kids = S[p].kids;
    std::vector<int32_t> newkids;
    for (int32_t c : kids) {
      SNode& C = S[c];
      SNode& Pn = S[p];
      int64_t ncol = C.ncol + Pn.ncol;
      int64_t nrow = Pn.nrow + C.ncol;
      int64_t tot = trap(ncol, nrow);
      int64_t nz = (trap(C.ncol, C.nrow) - C.zeros) + (trap(Pn.ncol, Pn.nrow) - Pn.zeros);
      int64_t zeros = tot - nz;
      double zf = (double)zeros / (double)tot;
      bool same_inst = P.row_inst[perm1[C.cols[0]]] == P.row_inst[perm1[Pn.cols[0]]];
      if (same_inst && relax_ok(ncol, zf)) {
        std::vector<int32_t> cols = C.cols;
        cols.insert(cols.end(), Pn.cols.begin(), Pn.cols.end());
        Pn.cols.swap(cols);
        Pn.ncol = ncol;
        Pn.nrow = nrow;
        Pn.zeros = zeros;
        C.rep = p;
        for (int32_t g : C.kids) newkids.push_back(g);
        std::vector<int32_t>().swap(C.cols);
        std::vector<int32_t>().swap(C.below);
      } else {
        newkids.push_back(c);
      }
    }
    S[p].kids.swap(newkids);
  }
  // final supernodes: representatives; postorder over the amalgamated tree
  std::vector<int32_t> reps;
  for (int32_t s = 0; s < ns0; s++)
    if (S[s].rep < 0) reps.push_back(s);
  std::vector<int32_t> rid(ns0, -1);
  for (size_t i = 0; i < reps.size(); i++) rid[reps[i]] = (int32_t)i;
  const int32_t ns = (int32_t)reps.size();
  std::vector<int32_t> rpar(ns, -1);
  for (int32_t i = 0; i < ns; i++) {
    int32_t fp = S[reps[i]].parent;
    rpar[i] = fp < 0 ? -1 : rid[find_rep(S, fp)];
  }
  std::vector<int32_t> rpost = postorder(ns, rpar);
  // new column numbering
  std::vector<int32_t> newcol(N, -1);
  std::vector<int32_t> perm2(N);
  int32_t nextc = 0;
  std::vector<int32_t> spos(ns);
  for (int32_t k = 0; k < ns; k++) {
    int32_t s = reps[rpost[k]];
    spos[rpost[k]] = k;
    for (int32_t c : S[s].cols) {
      newcol[c] = nextc;
      perm2[nextc] = perm1[c];
      nextc++;
    }
  }
  P.perm = perm2;
  P.iperm.assign(N, 0);
  for (int64_t k = 0; k < N; k++) P.iperm[perm2[k]] = (int32_t)k;

  P.ns = ns;
  P.sn_col0.resize(ns);
  P.sn_ncol.resize(ns);
  P.sn_nrow.resize(ns);
  P.sn_parent.resize(ns);
  P.sn_rows_off.assign(ns + 1, 0);
  std::vector<std::vector<int32_t>> rows(ns);
  for (int32_t k = 0; k < ns; k++) {
    int32_t s = reps[rpost[k]];
    const SNode& X = S[s];
    P.sn_col0[k] = newcol[X.cols[0]];
    P.sn_ncol[k] = (int32_t)X.ncol;
    int32_t rp = rpar[rpost[k]];
    P.sn_parent[k] = rp < 0 ? -1 : spos[rp];
    std::vector<int32_t>& R = rows[k];
    R.reserve(X.nrow);
    for (int32_t c = 0; c < X.ncol; c++) R.push_back(P.sn_col0[k] + c);
    std::vector<int32_t> b;
    b.reserve(X.below.size());
    for (int32_t r : X.below) b.push_back(newcol[r]);
    std::sort(b.begin(), b.end());
    R.insert(R.end(), b.begin(), b.end());
    P.sn_nrow[k] = (int32_t)R.size();
  }
  for (int32_t k = 0; k < ns; k++) P.sn_rows_off[k + 1] = P.sn_rows_off[k] + P.sn_nrow[k];
  P.sn_rows.resize(P.sn_rows_off[ns]);
  for (int32_t k = 0; k < ns; k++)
    std::copy(rows[k].begin(), rows[k].end(), P.sn_rows.begin() + P.sn_rows_off[k]);
}

// ---------------------------------------------------------------------------
// 4. Schedule and maps
// ---------------------------------------------------------------------------
void schedule(Plan& P, int colpad) {
  const int32_t ns = P.ns;
  const int64_t N = P.dim;
  // contiguity check of supernode columns
  std::vector<int32_t> sn_of_col(N, -1);
  for (int32_t s = 0; s < ns; s++)
    for (int32_t c = 0; c < P.sn_ncol[s]; c++) sn_of_col[P.sn_col0[s] + c] = s;
  for (int64_t c = 0; c < N; c++)
    if (sn_of_col[c] < 0) throw std::runtime_error("internal: column without supernode");
  // children
  P.child_ptr.assign(ns + 1, 0);
  for (int32_t s = 0; s < ns; s++)
    if (P.sn_parent[s] >= 0) P.child_ptr[P.sn_parent[s] + 1]++;
  for (int32_t s = 0; s < ns; s++) P.child_ptr[s + 1] += P.child_ptr[s];
  P.child_list.resize(P.child_ptr[ns]);
  {
    std::vector<int32_t> f(P.child_ptr.begin(), P.child_ptr.end() - 1);
    for (int32_t s = 0; s < ns; s++)
      if (P.sn_parent[s] >= 0) P.child_list[f[P.sn_parent[s]]++] = s;
  }
  // levels (height above the leaves)
  P.sn_level.assign(ns, 0);
  int32_t maxl = 0;
  for (int32_t s = 0; s < ns; s++) {
    int32_t l = 0;
    for (int32_t k = P.child_ptr[s]; k < P.child_ptr[s + 1]; k++)
      l = std::max(l, P.sn_level[P.child_list[k]] + 1);
    P.sn_level[s] = l;
    maxl = std::max(maxl, l);
  }
  P.nlevels = ns ? maxl + 1 : 0;
  P.level_ptr.assign(P.nlevels + 1, 0);
  for (int32_t s = 0; s < ns; s++) P.level_ptr[P.sn_level[s] + 1]++;
  for (int32_t l = 0; l < P.nlevels; l++) P.level_ptr[l + 1] += P.level_ptr[l];
  P.level_list.resize(ns);
  {
    std::vector<int32_t> f(P.level_ptr.begin(), P.level_ptr.end() - 1);
    // within a level: larger fronts first (they start the long kernels early)
    std::vector<int32_t> idx(ns);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
      return (int64_t)P.sn_nrow[a] * P.sn_ncol[a] > (int64_t)P.sn_nrow[b] * P.sn_ncol[b];
    });
    for (int32_t s : idx) P.level_list[f[P.sn_level[s]]++] = s;
  }
  // storage
  P.sn_ncolp.resize(ns);
  P.sn_Loff.assign(ns + 1, 0);
  P.sn_Uoff.assign(ns + 1, 0);
  P.sn_Woff.assign(ns + 1, 0);
  P.max_front = 0;
  P.max_pivots = 0;
  for (int32_t s = 0; s < ns; s++) {
    int64_t ncp = (P.sn_ncol[s] + colpad - 1) / colpad * colpad;
    P.sn_ncolp[s] = (int32_t)ncp;
    int64_t nb = P.sn_nrow[s] - P.sn_ncol[s];
    int64_t lsz = (int64_t)P.sn_nrow[s] * ncp;
    lsz = (lsz + 31) / 32 * 32;
    int64_t usz = nb * nb;
    usz = (usz + 31) / 32 * 32;
    P.sn_Loff[s + 1] = P.sn_Loff[s] + lsz;
    P.sn_Uoff[s + 1] = P.sn_Uoff[s] + usz;
    P.sn_Woff[s + 1] = P.sn_Woff[s] + nb;
    P.max_front = std::max<int64_t>(P.max_front, P.sn_nrow[s]);
    P.max_pivots = std::max<int64_t>(P.max_pivots, P.sn_ncol[s]);
  }
  P.L_stored = P.sn_Loff[ns];
  P.U_stored = P.sn_Uoff[ns];
  // relmap
  P.relmap_off.assign(ns + 1, 0);
  for (int32_t s = 0; s < ns; s++) P.relmap_off[s + 1] = P.relmap_off[s] + (P.sn_nrow[s] - P.sn_ncol[s]);
  P.relmap.resize(P.relmap_off[ns]);
  for (int32_t s = 0; s < ns; s++) {
    int32_t p = P.sn_parent[s];
    int64_t nb = P.sn_nrow[s] - P.sn_ncol[s];
    if (nb == 0) continue;
    if (p < 0) throw std::runtime_error("internal: root supernode with rows below");
    const int32_t* cr = &P.sn_rows[P.sn_rows_off[s] + P.sn_ncol[s]];
    const int32_t* pr = &P.sn_rows[P.sn_rows_off[p]];
    int64_t pn = P.sn_nrow[p];
    int64_t q = 0;
    for (int64_t a = 0; a < nb; a++) {
      while (q < pn && pr[q] < cr[a]) q++;
      if (q >= pn || pr[q] != cr[a]) throw std::runtime_error("internal: child row not in parent");
      P.relmap[P.relmap_off[s] + a] = (int32_t)q;
    }
  }
  // assembly map by front row
  const int64_t totrows = P.sn_rows_off[ns];
  P.amap_ptr.assign(totrows + 1, 0);
  std::vector<int64_t> frow(P.nnzA);
  std::vector<int32_t> fcol(P.nnzA);
  // front row and column of every entry (columns in parallel), then the
  // counts in entry order
  std::atomic<bool> outside{false};
  parallel_ranges(N, 8192, [&](int64_t c0, int64_t c1) {
    for (int64_t c = c0; c < c1; c++)
      for (int64_t p = P.A_colptr[c]; p < P.A_colptr[c + 1]; p++) {
        int32_t a = P.iperm[P.A_row[p]], b = P.iperm[c];
        int32_t r = std::max(a, b), cc = std::min(a, b);
        int32_t s = sn_of_col[cc];
        int64_t lr;
        if (r < P.sn_col0[s] + P.sn_ncol[s]) lr = r - P.sn_col0[s];
        else {
          const int32_t* beg = &P.sn_rows[P.sn_rows_off[s] + P.sn_ncol[s]];
          const int32_t* end = &P.sn_rows[P.sn_rows_off[s + 1]];
          const int32_t* it = std::lower_bound(beg, end, r);
          if (it == end || *it != r) {
            outside.store(true, std::memory_order_relaxed);
            lr = 0;
          } else {
            lr = P.sn_ncol[s] + (it - beg);
          }
        }
        frow[p] = P.sn_rows_off[s] + lr;
        fcol[p] = cc - P.sn_col0[s];
      }
  });
  if (outside.load()) throw std::runtime_error("internal: entry outside supernode rows");
  for (int64_t p = 0; p < P.nnzA; p++) P.amap_ptr[frow[p] + 1]++;
  for (int64_t r = 0; r < totrows; r++) P.amap_ptr[r + 1] += P.amap_ptr[r];
  P.amap_col.resize(P.nnzA);
  P.amap_src.resize(P.nnzA);
  {
    std::vector<int64_t> f(P.amap_ptr.begin(), P.amap_ptr.end() - 1);
    for (int64_t p = 0; p < P.nnzA; p++) {
      int64_t q = f[frow[p]]++;
      P.amap_col[q] = fcol[p];
      P.amap_src[q] = (int32_t)p;
    }
  }
  P.col_inst.resize(N);
  P.col_sign.resize(N);
  for (int64_t k = 0; k < N; k++) {
    P.col_inst[k] = P.row_inst[P.perm[k]];
    P.col_sign[k] = P.row_sign[P.perm[k]];
  }
}

}  // namespace

std::string analyze(const AnalyzeInput& in, Plan& P) {
  auto t0 = std::chrono::steady_clock::now();
  try {
    build_pattern(in, P);
    std::vector<int32_t> perm0;
    {
      Graph G = make_graph(P);
      perm0 = nested_dissection(G, std::max(8, std::min(in.leaf_size, 256)));
    }
    symbolic(P, perm0);
    schedule(P, std::max(1, in.colpad));
  } catch (const PatternError& e) {
    return e.what();
  } catch (const std::bad_alloc&) {
    return "oom: host allocation failed in analyze";
  } catch (const std::exception& e) {
    return std::string("internal: ") + e.what();
  }
  P.analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return "";
}

}  // namespace ncl
