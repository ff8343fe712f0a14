// Init-time layout of the spanning tree (sparsify_init).  The tree is fixed
// for the life of a handle, so its shape is laid out once; every recovery
// then recomputes the tree's numbers from it (step A2: root distances, hop
// depths and the range-minimum structure of the LCA queries).
//
//   * Vertices are relabelled in DFS preorder of T (per graph of a batch,
//     inside the graph's own vertex range, the root first).  Every subtree is
//     then a contiguous label range, so
//       - LCA(u, v), u < v, is the parent of any vertex of minimum depth among
//         the labels (u, v] (a range-minimum query, step A3), and
//       - the children of an LCA order the same way as the endpoints below
//         them, which orients the records of step A5 without a search.
//     The canonical edge list keeps its order (canonical ids are unchanged);
//     its endpoints are stored as (smaller label, larger label), and the
//     inverse labelling maps results back to the caller's vertex ids.
//   * The Euler tour of T: 2(n - G) arcs in tour order, each the label of the
//     vertex entered (a step down) or the complement of the label left (a
//     step up).  A prefix sum over the tour of +edge word / -edge word gives
//     every vertex's root distance and depth at its down arc (step A2).
//
// Construction: tree adjacency with reverse arcs, rows sorted (so the tour is
// deterministic), the tour successor (after x->y the arc following y->x in
// y's row), cut at each root, list ranking by pointer jumping (one packed
// word per arc), the preorder
// rank of every down arc from a prefix count over the tour.
#include <algorithm>
#include <climits>
#include <type_traits>
#include <vector>

#include "pdg_internal.cuh"
#include "pdg_tour.cuh"

namespace pdg {

namespace {

__global__ void k_lay_tflag(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                            const int32_t* __restrict__ parent, int64_t m, uint8_t* __restrict__ tflag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    tflag[e] = (parent[ev[e]] == eu[e] || parent[eu[e]] == ev[e]) ? 1 : 0;
}

// the tour of each tree ends with the arc into its root that precedes the
// root's first arc
__global__ void k_lay_cut(const int32_t* __restrict__ parent, const int64_t* __restrict__ tptr,
                          const int32_t* __restrict__ tdeg, const int32_t* __restrict__ rev, int64_t n,
                          int32_t* __restrict__ succ, int32_t* __restrict__ rd) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (parent[v] >= 0 || tdeg[v] == 0) continue;
    const int32_t tail = rev[tptr[v] + tdeg[v] - 1];
    succ[tail] = -1;
    rd[tail] = 0;
  }
}

// Position of every arc in the concatenated tour (graph g's tour starts at
// 2 (vtx_ptr[g] - g)), in original labels: y for x->y when x is y's parent
// (down), ~x otherwise (up, leaving x); dflag marks the down arcs.
// List ranking by pointer jumping on one packed word per arc, (successor << 32) | arcs to the end: one
// gather per arc and round instead of two.
__global__ void k_lay_pack(const int32_t* __restrict__ succ, const int32_t* __restrict__ rd, int64_t A,
                           uint64_t* __restrict__ out) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (int64_t)gridDim.x * blockDim.x)
    out[a] = ((uint64_t)(uint32_t)succ[a] << 32) | (uint32_t)rd[a];
}

__global__ void k_lay_rank(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t A) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = in[a];
    const int32_t s = (int32_t)(w >> 32);
    if (s < 0) {
      out[a] = w;
    } else {
      const uint64_t x = in[s];
      out[a] = (x & 0xffffffff00000000ull) | (uint32_t)((uint32_t)w + (uint32_t)x);
    }
  }
}

// An arc whose list did not end after the ranking rounds lies on a tour that
// no root cut: a cycle of parent links away from the root.  Such an arc, or a
// position outside its graph's tour, marks the tree bad and is not written.
__global__ void k_lay_arcs(const int32_t* __restrict__ tadj, const int64_t* __restrict__ tptr,
                           const int32_t* __restrict__ parent, const uint64_t* __restrict__ ranked,
                           const int64_t* __restrict__ vtx_ptr, int32_t G, int64_t n, int32_t* __restrict__ tour,
                           int32_t* __restrict__ dflag, int32_t* __restrict__ bad) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = tptr[x], e = tptr[x + 1];
    if (b == e) continue;
    const int32_t g = (G == 1) ? 0 : part_of(vtx_ptr, G, x);
    const int64_t len = 2 * (vtx_ptr[g + 1] - vtx_ptr[g] - 1);
    const int64_t base = 2 * (vtx_ptr[g] - g);
    for (int64_t a = b; a < e; a++) {
      const int32_t y = tadj[a];
      const int32_t succ = (int32_t)(ranked[a] >> 32), rd = (int32_t)(uint32_t)ranked[a];
      if (succ != -1 || rd < 0 || rd >= len) {
        *bad = 1;
        continue;
      }
      const int64_t pos = base + len - 1 - rd;
      const bool down = parent[y] == (int32_t)x;
      tour[pos] = down ? y : ~(int32_t)x;
      dflag[pos] = down ? 1 : 0;
    }
  }
}

// preorder label of the vertex entered by each down arc: the graph's first
// label, + 1 for its root, + the down arcs before it in the graph's tour
// (dpre: exclusive prefix count over the whole tour, which holds
// vtx_ptr[g] - g down arcs of the graphs before g)
__global__ void k_lay_pre(const int32_t* __restrict__ tour, const int64_t* __restrict__ dpre, int64_t A,
                          const int64_t* __restrict__ vtx_ptr, int32_t G, int32_t* __restrict__ pre_of) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t y = tour[p];
    if (y < 0) continue;
    const int32_t g = (G == 1) ? 0 : part_of(vtx_ptr, G, y);
    pre_of[y] = (int32_t)(dpre[p] + g + 1);
  }
}

// the largest hop depth: after the down arc at tour position p the depth is
// (down arcs up to p) - (up arcs before p) = 2 dpre[p] + 1 - p (every graph's
// tour starts after as many down arcs as its offset counts)
__global__ void k_lay_depth(const int32_t* __restrict__ tour, const int64_t* __restrict__ dpre, int64_t A,
                            DevScalars* dsc) {
  long long mx = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A; p += (int64_t)gridDim.x * blockDim.x)
    if (tour[p] >= 0) mx = max(mx, (long long)(2 * dpre[p] + 1 - p));
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax((long long*)&dsc->max_depth, mx);
}

__global__ void k_lay_roots(const int32_t* __restrict__ parent, const int64_t* __restrict__ vtx_ptr, int32_t G,
                            int64_t n, int32_t* __restrict__ pre_of) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (parent[v] >= 0) continue;
    const int32_t g = (G == 1) ? 0 : part_of(vtx_ptr, G, v);
    pre_of[v] = (int32_t)vtx_ptr[g];
  }
}

// inverse labelling, the parent array in labels, and the roots' fixed values
// (root distance 0, depth 0)
__global__ void k_lay_vertices(const int32_t* __restrict__ pre_of, const int32_t* __restrict__ parent, int64_t n,
                               int32_t* __restrict__ vtx_of_pre, int32_t* __restrict__ parent_pre,
                               u128* __restrict__ P, uint64_t* __restrict__ val0, int32_t* __restrict__ bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = pre_of[v];
    const int32_t p = parent[v];
    if (x < 0 || x >= n || (p >= 0 && (pre_of[p] < 0 || pre_of[p] >= n))) {  // a vertex the tour missed
      *bad = 1;
      continue;
    }
    vtx_of_pre[x] = (int32_t)v;
    parent_pre[x] = p < 0 ? -1 : pre_of[p];
    if (p < 0) {
      P[x] = 0;
      val0[x] = 0;  // never inside a query range (every range starts after a vertex of the root's graph)
    }
  }
}

__global__ void k_lay_tour(int32_t* __restrict__ tour, const int32_t* __restrict__ pre_of, int64_t A, int64_t n,
                           int32_t* __restrict__ bad) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t y = tour[p];
    const int32_t v = y >= 0 ? y : ~y;
    if (v < 0 || v >= n) {  // a position the arcs did not fill
      *bad = 1;
      tour[p] = 0;
      continue;
    }
    tour[p] = y >= 0 ? pre_of[v] : ~pre_of[v];
  }
}

__global__ void k_lay_edges(int32_t* __restrict__ eu, int32_t* __restrict__ ev, const int32_t* __restrict__ pre_of,
                            int64_t m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = pre_of[eu[e]], b = pre_of[ev[e]];
    eu[e] = min(a, b);
    ev[e] = max(a, b);
  }
}

}  // namespace

int build_tree_layout(Handle& h) {
  const int64_t n = h.n, m = h.m;
  const int32_t G = h.G;
  const int64_t A = 2 * (n - G);  // arcs of all tours
  cudaStream_t s = h.stream;
  const int gn = grid_for(h, n), gm = grid_for(h, std::max<int64_t>(m, 1)), ga = grid_for(h, std::max<int64_t>(A, 1));
  std::vector<void*> temps;
  auto cleanup = [&]() {
    for (void* p : temps) cudaFreeAsync(p, s);
    temps.clear();
  };
  auto fail = [&](int code) {
    cudaGetLastError();
    cleanup();
    return code;
  };
  auto talloc = [&](auto** p, int64_t count) -> bool {
    void* q = nullptr;
    if (cudaMallocAsync(&q, sizeof(**p) * (size_t)std::max<int64_t>(count, 1), s) != cudaSuccess) return false;
    temps.push_back(q);
    *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    return true;
  };
  int st;
  // resident layout
  if ((st = device_alloc(h, (void**)&h.tour, sizeof(int32_t) * (size_t)std::max<int64_t>(A, 1))) ||
      (st = device_alloc(h, (void**)&h.vtx_of_pre, sizeof(int32_t) * (size_t)n)) ||
      (st = device_alloc(h, (void**)&h.P, sizeof(u128) * (size_t)n)))
    return st;
  // range-minimum levels: level j + 1 holds the minima of the 32-entry groups of level j, up to one group;
  // when level 2 is small enough, it and everything above it is one sparse table instead
  h.rmq_levels = 0;
  h.rmq_st = nullptr;
  h.rmq_st_rows = 0;
  for (int64_t sz = n;; sz = (sz + 31) / 32) {
    if (h.rmq_levels >= kRmqMaxLevels) return PDG_E_INVALID_ARG;
    if (h.rmq_levels == 2 && sz <= kRmqStMax) {
      int rows = 1;
      while ((1ll << rows) <= sz) rows++;  // rows t = 0 .. floor(log2 sz)
      if ((st = device_alloc(h, (void**)&h.rmq_st, sizeof(uint64_t) * (size_t)sz * rows))) return st;
      h.rmq_st_rows = rows;
      h.rmq_size[2] = sz;
      h.rmq_val[2] = h.rmq_st;  // row 0: the level-2 entries themselves
      h.rmq_levels = 3;
      break;
    }
    h.rmq_size[h.rmq_levels] = sz;
    if ((st = device_alloc(h, (void**)&h.rmq_val[h.rmq_levels], sizeof(uint64_t) * (size_t)sz)) ||
        (st = device_alloc(h, (void**)&h.rmq_mask[h.rmq_levels], sizeof(uint32_t) * (size_t)sz)))
      return st;
    if (sz > 32 &&  // below the top level, queries read partial groups from these
        ((st = device_alloc(h, (void**)&h.rmq_pmin[h.rmq_levels], sizeof(uint64_t) * (size_t)sz)) ||
         (st = device_alloc(h, (void**)&h.rmq_smin[h.rmq_levels], sizeof(uint64_t) * (size_t)sz))))
      return st;
    h.rmq_levels++;
    if (sz <= 32) break;
  }
  uint8_t* tflag = nullptr;
  int32_t *tdeg = nullptr, *cur = nullptr, *tadj = nullptr, *rev = nullptr, *arc_uv = nullptr, *dflag = nullptr;
  int32_t *succ = nullptr, *rd = nullptr, *pre_of = nullptr, *parent_pre = nullptr;
  uint64_t* ranked[2] = {nullptr, nullptr};
  int64_t *tptr = nullptr, *dpre = nullptr;
  int32_t* bad = nullptr;
  if (!talloc(&tflag, m) || !talloc(&tdeg, n) || !talloc(&cur, n) || !talloc(&tptr, n + 1) || !talloc(&tadj, A) ||
      !talloc(&rev, A) || !talloc(&arc_uv, m) || !talloc(&succ, A) || !talloc(&rd, A) || !talloc(&ranked[0], A) ||
      !talloc(&ranked[1], A) || !talloc(&dflag, A) || !talloc(&dpre, A + 1) || !talloc(&pre_of, n) ||
      !talloc(&parent_pre, n) || !talloc(&bad, 1))
    return fail(PDG_E_OOM);
#define LAY_CK(x)                                    \
  do {                                               \
    if ((x) != cudaSuccess) return fail(PDG_E_CUDA); \
  } while (0)
  LAY_CK(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  LAY_CK(cudaMemsetAsync(pre_of, 0xff, sizeof(int32_t) * n, s));  // -1: not reached
  if (A > 0) LAY_CK(cudaMemsetAsync(h.tour, 0xff, sizeof(int32_t) * A, s));
  LAY_CK(cudaMemsetAsync(tdeg, 0, sizeof(int32_t) * n, s));
  LAY_CK(cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, s));
  if (m > 0) {
    k_lay_tflag<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, h.parent, m, tflag);
    k_st_tdeg<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tdeg);
  }
  if ((st = scan_excl_i32(h, tdeg, tptr, n, nullptr, n))) return fail(st);
  if (A > 0) {
    k_st_fill<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tptr, cur, tadj, rev, arc_uv);
    k_tour_sort_rows<<<gn, kBlock, 0, s>>>(tptr, n, tadj);
    k_tour_fix_rev<<<gn, kBlock, 0, s>>>(tptr, tadj, n, rev);
    k_st_succ<<<ga, kBlock, 0, s>>>(tadj, rev, tptr, tdeg, n, succ, rd);
    k_lay_cut<<<gn, kBlock, 0, s>>>(h.parent, tptr, tdeg, rev, n, succ, rd);
    k_lay_pack<<<ga, kBlock, 0, s>>>(succ, rd, A, ranked[0]);
    int bits = 1;
    while ((1ll << bits) <= A) bits++;
    int c = 0;
    for (int it = 0; it < bits; it++) {
      k_lay_rank<<<ga, kBlock, 0, s>>>(ranked[c], ranked[c ^ 1], A);
      c ^= 1;
    }
    k_lay_arcs<<<gn, kBlock, 0, s>>>(tadj, tptr, h.parent, ranked[c], h.d_vtx_ptr, G, n, h.tour, dflag, bad);
    if ((st = ensure_scan_status(h, A)) || (st = scan_excl_i32(h, dflag, dpre, A, nullptr, A))) return fail(st);
    k_lay_pre<<<ga, kBlock, 0, s>>>(h.tour, dpre, A, h.d_vtx_ptr, G, pre_of);
    LAY_CK(cudaMemsetAsync(&h.dsc->max_depth, 0, sizeof(int64_t), s));
    k_lay_depth<<<ga, kBlock, 0, s>>>(h.tour, dpre, A, h.dsc);
  }
  k_lay_roots<<<gn, kBlock, 0, s>>>(h.parent, h.d_vtx_ptr, G, n, pre_of);
  k_lay_vertices<<<gn, kBlock, 0, s>>>(pre_of, h.parent, n, h.vtx_of_pre, parent_pre, h.P, h.rmq_val[0], bad);
  if (A > 0) k_lay_tour<<<ga, kBlock, 0, s>>>(h.tour, pre_of, A, n, bad);
  {
    int32_t hbad = 0;
    if (A == 0) LAY_CK(cudaMemsetAsync(&h.dsc->max_depth, 0, sizeof(int64_t), s));
    LAY_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LAY_CK(cudaMemcpyAsync(h.hsc, h.dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    LAY_CK(cudaStreamSynchronize(s));
    if (hbad) return fail(PDG_E_NOT_A_TREE);  // the parent links are not a tree the tour covers (a cycle)
    // the fixed-point range of the exact root distances: 2^(e_max - e_min + 53) per edge, max_depth edges
    h.max_depth = h.hsc->max_depth;
    int dep_bits = 0;
    while ((1ll << dep_bits) <= h.max_depth) dep_bits++;
    if (h.hsc->e_max != INT_MIN && h.hsc->e_max - h.hsc->e_min + 53 + dep_bits > 96) return fail(PDG_E_RANGE);
  }
  if (m > 0) k_lay_edges<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, pre_of, m);
  LAY_CK(cudaMemcpyAsync(h.parent, parent_pre, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  LAY_CK(cudaGetLastError());
#undef LAY_CK
  h.A = A;
  cleanup();
  return PDG_OK;
}

}  // namespace pdg
