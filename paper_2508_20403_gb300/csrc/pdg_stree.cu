// Spanning-tree generation, the step before recovery (Sec. 2.2: feGRASS
// builds its spanning tree from the effective weight of Eq. weff, then
// recovers off-tree edges against it).
//
// Two trees, both the maximum spanning forest for a strict total order on
// the edges (key descending, canonical edge id ascending), so each is unique:
//   PDG_TREE_MAX_WEIGHT  key = w(e);
//   PDG_TREE_FEGRASS     key = W_eff(e) = fl(fl(w * L) / (d(u) + d(v))) with
//                        L = fl(log(max(deg u, deg v))) and d = unweighted BFS
//                        distance from the maximum-degree vertex (Eq. weff);
//                        the graph must be connected.
// Each tree is rooted at the maximum-degree vertex of its component (ties:
// smaller id) and returned as a parent array.
//
// Forest: Boruvka rounds.  Every component finds its maximum incident edge
// leaving it (an atomicMax on the key bits, then an atomicMin on the edge id
// among the edges carrying that key), hooks to the component across it (two
// components that chose the same edge: the smaller id stays the root; with a
// strict order no longer cycle exists), and pointer jumping relabels the
// vertices.  Rooting: an Euler tour of the forest (arc x->y is followed by
// the arc after y->x in y's tree adjacency, cut at each root) ranked by
// pointer jumping; of the two arcs of a tree edge, the earlier one runs from
// the parent to the child.
#include <climits>
#include <cmath>
#include <type_traits>
#include <vector>

#include "pdg_internal.cuh"
#include "pdg_tour.cuh"

namespace pdg {

namespace {

constexpr int32_t kNoEdge = INT_MAX;

__device__ __forceinline__ unsigned long long degree_key(const int64_t* __restrict__ row_ptr, int64_t v) {
  // larger degree first, then smaller id
  return ((unsigned long long)(row_ptr[v + 1] - row_ptr[v]) << 32) | (0xffffffffull - (unsigned long long)v);
}

__global__ void k_st_maxdeg(const int64_t* __restrict__ row_ptr, int64_t n, unsigned long long* best) {
  unsigned long long b = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    b = max(b, degree_key(row_ptr, v));
  for (int o = 16; o; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
  if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

// one BFS level: every vertex at distance `level` labels its unvisited neighbours
__global__ void k_st_bfs(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                         int32_t* dist, int32_t level, int32_t* grew) {
  int any = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (dist[v] != level) continue;
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; p++) {
      const int32_t u = col[p];
      if (dist[u] < 0 && atomicCAS(&dist[u], -1, level + 1) == -1) any = 1;
    }
  }
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *grew = 1;
}

__global__ void k_st_unreached(const int32_t* __restrict__ dist, int64_t n, int32_t* flag) {
  int any = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (dist[v] < 0) any = 1;
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *flag = 1;
}

__global__ void k_st_keys_weight(const double* __restrict__ ew, int64_t m, uint64_t* __restrict__ key) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    key[e] = (uint64_t)__double_as_longlong(ew[e]);
}

// W_eff(e) = fl(fl(w * L[max deg]) / (d(u) + d(v))) (Eq. weff); non-negative,
// so its bits order like the value
__global__ void k_st_keys_weff(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                               const double* __restrict__ ew, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ dist, const double* __restrict__ ltab, int64_t m,
                               uint64_t* __restrict__ key) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = eu[e], v = ev[e];
    const int64_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
    const double s = (double)((int64_t)dist[u] + (int64_t)dist[v]);  // >= 1: u != v
    const double x = __ddiv_rn(__dmul_rn(ew[e], ltab[max(du, dv)]), s);
    key[e] = (uint64_t)__double_as_longlong(x);
  }
}

__global__ void k_st_iota(int32_t* __restrict__ a, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    a[v] = (int32_t)v;
}

__global__ void k_st_reset_best(unsigned long long* __restrict__ bk, int32_t* __restrict__ bid, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    bk[v] = 0;
    bid[v] = kNoEdge;
  }
}

__global__ void k_st_best_key(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                              const uint64_t* __restrict__ key, const int32_t* __restrict__ comp, int64_t m,
                              unsigned long long* bk) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t cu = comp[eu[e]], cv = comp[ev[e]];
    if (cu == cv) continue;
    const unsigned long long k = key[e];
    if (k > bk[cu]) atomicMax(&bk[cu], k);
    if (k > bk[cv]) atomicMax(&bk[cv], k);
  }
}

__global__ void k_st_best_id(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                             const uint64_t* __restrict__ key, const int32_t* __restrict__ comp, int64_t m,
                             const unsigned long long* __restrict__ bk, int32_t* bid) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t cu = comp[eu[e]], cv = comp[ev[e]];
    if (cu == cv) continue;
    const unsigned long long k = key[e];
    if (k == bk[cu]) atomicMin(&bid[cu], (int32_t)e);
    if (k == bk[cv]) atomicMin(&bid[cv], (int32_t)e);
  }
}

// every component root hooks across its chosen edge; the edge joins the tree
__global__ void k_st_hook(const int32_t* __restrict__ comp, const int32_t* __restrict__ bid,
                          const int32_t* __restrict__ eu, const int32_t* __restrict__ ev, int64_t n,
                          int32_t* __restrict__ nxt, uint8_t* __restrict__ tflag, int32_t* hooks) {
  int any = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    if (comp[c] != (int32_t)c) continue;
    const int32_t e = bid[c];
    if (e == kNoEdge) {
      nxt[c] = (int32_t)c;
      continue;
    }
    const int32_t cu = comp[eu[e]], cv = comp[ev[e]];
    const int32_t other = (cu == (int32_t)c) ? cv : cu;
    tflag[e] = 1;
    any = 1;
    // two components that chose the same edge: the smaller id stays a root
    nxt[c] = (bid[other] == e && (int32_t)c < other) ? (int32_t)c : other;
  }
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *hooks = 1;
}

// pointer jumping over the hooks (in place: a jump only shortens a path)
__global__ void k_st_jump(const int32_t* __restrict__ comp, int32_t* nxt, int64_t n, int32_t* changed) {
  int any = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    if (comp[c] != (int32_t)c) continue;
    const int32_t a = nxt[c];
    const int32_t b = nxt[a];
    if (a != b) {
      nxt[c] = b;
      any = 1;
    }
  }
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *changed = 1;
}

__global__ void k_st_relabel(int32_t* comp, const int32_t* __restrict__ nxt, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    comp[v] = nxt[comp[v]];
}

__global__ void k_st_comp_root(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ comp, int64_t n,
                               unsigned long long* rk) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicMax(&rk[comp[v]], degree_key(row_ptr, v));
}

__device__ __forceinline__ bool is_root(const int32_t* __restrict__ comp, const unsigned long long* __restrict__ rk,
                                        int64_t v) {
  return (0xffffffffull - (rk[comp[v]] & 0xffffffffull)) == (unsigned long long)v;
}

// the tour of a component ends with the arc into its root that precedes the
// root's first arc
__global__ void k_st_cut(const int32_t* __restrict__ comp, const unsigned long long* __restrict__ rk,
                         const int64_t* __restrict__ tptr, const int32_t* __restrict__ tdeg,
                         const int32_t* __restrict__ rev, int64_t n, int32_t* __restrict__ succ,
                         int32_t* __restrict__ rd) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (tdeg[v] == 0 || !is_root(comp, rk, v)) continue;
    const int32_t tail = rev[tptr[v] + tdeg[v] - 1];
    succ[tail] = -1;
    rd[tail] = 0;
  }
}

// of the two arcs of a tree edge the earlier (farther from the end) leads
// from the parent to the child
__global__ void k_st_parent(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                            const uint8_t* __restrict__ tflag, const int32_t* __restrict__ arc_uv,
                            const int32_t* __restrict__ rev, const int32_t* __restrict__ rd, int64_t m,
                            int32_t* __restrict__ parent) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    if (!tflag[e]) continue;
    const int32_t a = arc_uv[e];
    if (rd[a] > rd[rev[a]]) parent[ev[e]] = eu[e];
    else parent[eu[e]] = ev[e];
  }
}

}  // namespace

// a failed CUDA call releases the temporaries and reports PDG_E_CUDA
#define ST_CK(x)                                   \
  do {                                             \
    if ((x) != cudaSuccess) return fail(PDG_E_CUDA); \
  } while (0)

int spanning_tree(Handle& h, int tree_kind, int32_t* parent) {
  const int64_t n = h.n, m = h.m;
  const int gn = grid_for(h, n), gm = grid_for(h, std::max<int64_t>(m, 1));
  cudaStream_t s = h.stream;
  std::vector<void*> temps;
  auto cleanup = [&]() {
    for (void* p : temps) cudaFreeAsync(p, s);
    temps.clear();
  };
  auto talloc = [&](auto** p, int64_t count) -> bool {
    void* q = nullptr;
    if (cudaMallocAsync(&q, sizeof(**p) * (size_t)std::max<int64_t>(count, 1), s) != cudaSuccess) return false;
    temps.push_back(q);
    *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    return true;
  };
  uint64_t* key = nullptr;
  int32_t *comp = nullptr, *nxt = nullptr, *bid = nullptr, *dist = nullptr, *tdeg = nullptr, *cur = nullptr;
  int32_t *tadj = nullptr, *rev = nullptr, *arc_uv = nullptr, *succ[2] = {nullptr, nullptr};
  int32_t *rd[2] = {nullptr, nullptr}, *flags = nullptr;
  unsigned long long *bk = nullptr, *rk = nullptr;
  uint8_t* tflag = nullptr;
  int64_t* tptr = nullptr;
  double* ltab = nullptr;
  const int64_t A = 2 * std::max<int64_t>(n - 1, 0);  // arcs of a spanning forest, at most
  if (!talloc(&key, m) || !talloc(&comp, n) || !talloc(&nxt, n) || !talloc(&bid, n) || !talloc(&bk, n) ||
      !talloc(&rk, n) || !talloc(&tflag, m) || !talloc(&tdeg, n) || !talloc(&cur, n) || !talloc(&tptr, n + 1) ||
      !talloc(&tadj, A) || !talloc(&rev, A) || !talloc(&arc_uv, m) || !talloc(&succ[0], A) || !talloc(&succ[1], A) ||
      !talloc(&rd[0], A) || !talloc(&rd[1], A) || !talloc(&flags, 64) ||
      (tree_kind == PDG_TREE_FEGRASS && !talloc(&dist, n))) {
    cudaGetLastError();
    cleanup();
    return PDG_E_OOM;
  }
  int32_t* hflags = reinterpret_cast<int32_t*>(h.hsc);  // pinned staging of the flags (the scalars are not in use)
  auto read_flags = [&](int count) -> bool {
    return cudaMemcpyAsync(hflags, flags, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
  };
  int st = PDG_OK;
  auto fail = [&](int code) {
    cudaGetLastError();
    cleanup();
    return code;
  };
  // 1. edge keys
  if (tree_kind == PDG_TREE_FEGRASS) {
    unsigned long long* best = rk;  // scratch
    ST_CK(cudaMemsetAsync(best, 0, sizeof(unsigned long long), s));
    k_st_maxdeg<<<gn, kBlock, 0, s>>>(h.row_ptr, n, best);
    unsigned long long bh = 0;
    if (cudaMemcpyAsync(&bh, best, sizeof(bh), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(PDG_E_CUDA);
    const int32_t root = (int32_t)(0xffffffffull - (bh & 0xffffffffull));
    const int64_t maxdeg = (int64_t)(bh >> 32);
    // unweighted BFS distances from the root, 16 levels per host check
    ST_CK(cudaMemsetAsync(dist, 0xff, sizeof(int32_t) * n, s));
    ST_CK(cudaMemsetAsync(dist + root, 0, sizeof(int32_t), s));
    bool done = false;
    for (int64_t level = 0; level <= n && !done; level += 16) {
      ST_CK(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 16, s));
      for (int i = 0; i < 16; i++) k_st_bfs<<<gn, kBlock, 0, s>>>(h.row_ptr, h.col, n, dist, (int32_t)(level + i), flags + i);
      if (!read_flags(16)) return fail(PDG_E_CUDA);
      done = hflags[15] == 0;
    }
    ST_CK(cudaMemsetAsync(flags, 0, sizeof(int32_t), s));
    k_st_unreached<<<gn, kBlock, 0, s>>>(dist, n, flags);
    if (!read_flags(1)) return fail(PDG_E_CUDA);
    if (!done || hflags[0]) return fail(PDG_E_INVALID_ARG);  // not connected
    // log of the degrees, from the host math library (one table, both sides of every comparison)
    std::vector<double> lh((size_t)maxdeg + 1, 0.0);
    for (int64_t d = 1; d <= maxdeg; d++) lh[d] = std::log((double)d);
    if (!talloc(&ltab, maxdeg + 1)) return fail(PDG_E_OOM);
    ST_CK(cudaMemcpyAsync(ltab, lh.data(), sizeof(double) * lh.size(), cudaMemcpyHostToDevice, s));
    k_st_keys_weff<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, h.el_w, h.row_ptr, dist, ltab, m, key);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PDG_E_CUDA);  // the host table is released below
  } else {
    k_st_keys_weight<<<gm, kBlock, 0, s>>>(h.el_w, m, key);
  }
  // 2. Boruvka rounds
  k_st_iota<<<gn, kBlock, 0, s>>>(comp, n);
  ST_CK(cudaMemsetAsync(tflag, 0, (size_t)std::max<int64_t>(m, 1), s));
  bool merged_all = false;
  for (int round = 0; round < 64; round++) {
    k_st_reset_best<<<gn, kBlock, 0, s>>>(bk, bid, n);
    k_st_best_key<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, key, comp, m, bk);
    k_st_best_id<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, key, comp, m, bk, bid);
    ST_CK(cudaMemsetAsync(flags, 0, sizeof(int32_t), s));
    k_st_hook<<<gn, kBlock, 0, s>>>(comp, bid, h.el_u, h.el_v, n, nxt, tflag, flags);
    if (!read_flags(1)) return fail(PDG_E_CUDA);
    if (hflags[0] == 0) {
      merged_all = true;
      break;
    }
    bool flat = false;
    for (int it = 0; it < 64 && !flat; it += 4) {
      ST_CK(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, s));
      for (int i = 0; i < 4; i++) k_st_jump<<<gn, kBlock, 0, s>>>(comp, nxt, n, flags + i);
      if (!read_flags(4)) return fail(PDG_E_CUDA);
      flat = hflags[3] == 0;
    }
    if (!flat) return fail(PDG_E_CUDA);
    k_st_relabel<<<gn, kBlock, 0, s>>>(comp, nxt, n);
  }
  if (!merged_all) return fail(PDG_E_CUDA);
  // 3. roots, tree adjacency, Euler tour
  ST_CK(cudaMemsetAsync(rk, 0, sizeof(unsigned long long) * n, s));
  k_st_comp_root<<<gn, kBlock, 0, s>>>(h.row_ptr, comp, n, rk);
  ST_CK(cudaMemsetAsync(tdeg, 0, sizeof(int32_t) * n, s));
  ST_CK(cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, s));
  k_st_tdeg<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tdeg);
  if ((st = ensure_scan_status(h, n)) || (st = scan_excl_i32(h, tdeg, tptr, n, nullptr, n))) return fail(st);
  {  // a forest has at most n - 1 edges: the arc arrays are sized for that
    int64_t arcs = 0;
    if (cudaMemcpyAsync(&arcs, tptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(PDG_E_CUDA);
    if (arcs < 0 || arcs > A) return fail(PDG_E_CUDA);
  }
  k_st_fill<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tptr, cur, tadj, rev, arc_uv);
  const int ga = grid_for(h, std::max<int64_t>(A, 1));
  k_st_succ<<<ga, kBlock, 0, s>>>(tadj, rev, tptr, tdeg, n, succ[0], rd[0]);
  k_st_cut<<<gn, kBlock, 0, s>>>(comp, rk, tptr, tdeg, rev, n, succ[0], rd[0]);
  int bits = 1;
  while ((1ll << bits) <= A) bits++;
  int c = 0;
  for (int r = 0; r < bits; r++) {
    k_st_rank<<<ga, kBlock, 0, s>>>(succ[c], rd[c], succ[c ^ 1], rd[c ^ 1], tptr, n);
    c ^= 1;
  }
  ST_CK(cudaMemsetAsync(parent, 0xff, sizeof(int32_t) * n, s));
  k_st_parent<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, arc_uv, rev, rd[c], m, parent);
  if (cudaGetLastError() != cudaSuccess) return fail(PDG_E_CUDA);
  cleanup();
  return PDG_OK;
}

#undef ST_CK

}  // namespace pdg
