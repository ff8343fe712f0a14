// Input validation of sparsify_init / sparsify_batch_init (the problem
// statement of Sec. 2.1 and Algorithm 1's input: a weighted undirected graph
// and a spanning tree of it).  Runs once per handle, outside recovery.
//
// Checks: CSR shape (monotone row_ptr, columns in range, no self loops,
// strictly increasing neighbours), symmetric weights (bitwise), weights in
// [2^-900, 2^900], no edge between two graphs of a batch, parent[] with one
// root per graph whose links are edges of G and acyclic, and the fixed-point
// range of the exact root distances.  Acyclicity and the maximum hop depth
// (which sets that range) come from pointer jumping here for the callers that
// build no tree layout; sparsify_init takes both from the layout's Euler tour.
#include <climits>
#include <cmath>

#include "pdg_internal.cuh"

namespace pdg {

namespace {

__device__ __forceinline__ int32_t graph_of_vertex(const int64_t* __restrict__ vtx_ptr, int32_t G, int64_t v) {
  return G == 1 ? 0 : part_of(vtx_ptr, G, v);
}

__global__ void k_val_rowptr(const int64_t* __restrict__ row_ptr, int64_t n, DevScalars* dsc) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    if (row_ptr[u] > row_ptr[u + 1]) atomicOr(&dsc->err, ERR_NOT_CSR);
}

// Every thread takes kValRun consecutive entries: one search for the row of the
// first, then the row advances with the entries.
constexpr int kValRun = 8;

__global__ void __launch_bounds__(kBlock) k_val_entries(const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ w, int64_t n, int64_t nnz,
                                                        const int64_t* __restrict__ vtx_ptr, int32_t G,
                                                        DevScalars* dsc) {
  const double lo = ldexp(1.0, -900), hi = ldexp(1.0, 900);
  int err = 0;
  for (int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kValRun; p0 < nnz;
       p0 += (int64_t)gridDim.x * blockDim.x * kValRun) {
    int64_t u = row_of(row_ptr, n, p0);
    for (int64_t p = p0; p < p0 + kValRun && p < nnz; p++) {
    while (row_ptr[u + 1] <= p) u++;  // empty rows are passed over (row_ptr is monotone: checked before)
    const int32_t v = col[p];
    const double x = w[p];
    if (!(x >= lo && x <= hi)) err |= ERR_BAD_WEIGHT;
    if (v < 0 || v >= n || v == u) {
      err |= ERR_NOT_CSR;
      continue;
    }
    if (p + 1 < row_ptr[u + 1] && !(col[p + 1] > v)) err |= ERR_NOT_CSR;
    if (graph_of_vertex(vtx_ptr, G, u) != graph_of_vertex(vtx_ptr, G, v)) err |= ERR_CROSS_GRAPH;
    const int64_t b = row_ptr[v], e = row_ptr[v + 1];
    const int64_t q = lower_bound_i32(col, b, e, (int32_t)u);
    if (q >= e || col[q] != (int32_t)u || __double_as_longlong(w[q]) != __double_as_longlong(x))
      err |= ERR_NOT_SYMMETRIC;
    }
  }
  if (err) atomicOr(&dsc->err, err);
}

__global__ void k_val_parent(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const double* __restrict__ w, const int32_t* __restrict__ parent, int64_t n,
                             const int64_t* __restrict__ vtx_ptr, int32_t G, DevScalars* dsc,
                             int64_t* __restrict__ roots, int32_t* __restrict__ jmp, int64_t* __restrict__ dep) {
  int err = 0;
  int lmin = INT_MAX, lmax = INT_MIN;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = parent[v];
    jmp[v] = p;
    dep[v] = (p == -1) ? 0 : 1;
    if (p == -1) {
      atomicAdd((unsigned long long*)&roots[graph_of_vertex(vtx_ptr, G, v)], 1ull);
      continue;
    }
    if (p < 0 || p >= n || p == v || graph_of_vertex(vtx_ptr, G, p) != graph_of_vertex(vtx_ptr, G, v)) {
      err |= ERR_NOT_A_TREE;
      jmp[v] = -1;
      continue;
    }
    const int64_t b = row_ptr[v], e = row_ptr[v + 1];
    const int64_t q = lower_bound_i32(col, b, e, p);
    if (q >= e || col[q] != p) {
      err |= ERR_NOT_A_TREE;
      continue;
    }
    const double r = 1.0 / w[q];
    const int ex = (int)((__double_as_longlong(r) >> 52) & 0x7ff) - 1023;
    lmin = min(lmin, ex);
    lmax = max(lmax, ex);
  }
  if (err) atomicOr(&dsc->err, err);
  if (lmin != INT_MAX) {
    atomicMin(&dsc->e_min, lmin);
    atomicMax(&dsc->e_max, lmax);
  }
}

__global__ void k_val_jump(const int32_t* __restrict__ jin, int32_t* __restrict__ jout, const int64_t* __restrict__ din,
                           int64_t* __restrict__ dout, int64_t n, DevScalars* dsc) {
  unsigned long long active = 0;
  long long mx = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = jin[v];
    int64_t d = din[v];
    int32_t na = -1;
    if (a >= 0) {
      d += din[a];
      na = jin[a];
    }
    if (na >= 0) active++;
    jout[v] = na;
    dout[v] = d;
    mx = max(mx, (long long)d);
  }
  for (int o = 16; o; o >>= 1) {
    active += __shfl_down_sync(0xffffffffu, active, o);
    mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (active) atomicAdd((unsigned long long*)&dsc->active, active);
    atomicMax((long long*)&dsc->max_depth, mx);
  }
}

__global__ void k_val_reset(DevScalars* dsc) {
  dsc->err = 0;
  dsc->e_min = INT_MAX;
  dsc->e_max = INT_MIN;
  dsc->active = 0;
  dsc->max_depth = 0;
}

__global__ void k_val_active_reset(DevScalars* dsc) { dsc->active = 0; }

}  // namespace

// The CSR checks alone (spanning-tree generation has no parent array yet).
int validate_csr(Handle& h) {
  const int64_t n = h.n;
  const int grid = grid_for(h, std::max<int64_t>(n, h.nnz));
  auto fetch = [&]() -> bool {
    return cudaMemcpyAsync(h.hsc, h.dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h.stream) == cudaSuccess &&
           cudaStreamSynchronize(h.stream) == cudaSuccess;
  };
  k_val_reset<<<1, 1, 0, h.stream>>>(h.dsc);
  k_val_rowptr<<<grid, kBlock, 0, h.stream>>>(h.row_ptr, n, h.dsc);
  if (!fetch()) return check_cuda(cudaGetLastError());
  if (h.hsc->err) return PDG_E_NOT_CSR;  // the entry checks below search rows: only on a monotone row_ptr
  if (h.nnz > 0) k_val_entries<<<grid, kBlock, 0, h.stream>>>(h.row_ptr, h.col, h.w, n, h.nnz, h.d_vtx_ptr, h.G, h.dsc);
  if (!fetch()) return check_cuda(cudaGetLastError());
  const int err = h.hsc->err;
  if (err & ERR_NOT_CSR) return PDG_E_NOT_CSR;
  if (err & ERR_BAD_WEIGHT) return PDG_E_BAD_WEIGHT;
  if (err & ERR_CROSS_GRAPH) return PDG_E_INVALID_ARG;
  if (err & ERR_NOT_SYMMETRIC) return PDG_E_NOT_SYMMETRIC;
  return PDG_OK;
}

int validate_graph(Handle& h, bool acyclic) {
  const int64_t n = h.n;
  const int grid = grid_for(h, std::max<int64_t>(n, h.nnz));
  // read the device scalars back on the handle's stream (no legacy-stream sync)
  auto fetch = [&]() -> bool {
    return cudaMemcpyAsync(h.hsc, h.dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h.stream) == cudaSuccess &&
           cudaStreamSynchronize(h.stream) == cudaSuccess;
  };
  k_val_reset<<<1, 1, 0, h.stream>>>(h.dsc);
  k_val_rowptr<<<grid, kBlock, 0, h.stream>>>(h.row_ptr, n, h.dsc);
  if (!fetch()) return check_cuda(cudaGetLastError());
  if (h.hsc->err) return PDG_E_NOT_CSR;
  if (h.nnz > 0) k_val_entries<<<grid, kBlock, 0, h.stream>>>(h.row_ptr, h.col, h.w, n, h.nnz, h.d_vtx_ptr, h.G, h.dsc);
  // temporaries for the acyclicity check (stream-ordered)
  int32_t* jmp[2] = {nullptr, nullptr};
  int64_t* dep[2] = {nullptr, nullptr};
  int64_t* roots = nullptr;
  int st = PDG_OK;
  auto cleanup = [&]() {
    void* ps[] = {jmp[0], jmp[1], dep[0], dep[1], roots};
    for (void* p : ps)
      if (p) cudaFreeAsync(p, h.stream);
  };
  if (cudaMallocAsync((void**)&jmp[0], sizeof(int32_t) * n, h.stream) != cudaSuccess ||
      cudaMallocAsync((void**)&jmp[1], sizeof(int32_t) * n, h.stream) != cudaSuccess ||
      cudaMallocAsync((void**)&dep[0], sizeof(int64_t) * n, h.stream) != cudaSuccess ||
      cudaMallocAsync((void**)&dep[1], sizeof(int64_t) * n, h.stream) != cudaSuccess ||
      cudaMallocAsync((void**)&roots, sizeof(int64_t) * h.G, h.stream) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return PDG_E_OOM;
  }
  cudaMemsetAsync(roots, 0, sizeof(int64_t) * h.G, h.stream);
  k_val_parent<<<grid, kBlock, 0, h.stream>>>(h.row_ptr, h.col, h.w, h.parent, n, h.d_vtx_ptr, h.G, h.dsc, roots,
                                              jmp[0], dep[0]);
  std::vector<int64_t> roots_h(h.G);
  if (cudaMemcpyAsync(roots_h.data(), roots, sizeof(int64_t) * h.G, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
      !fetch()) {
    cleanup();
    return check_cuda(cudaGetLastError());
  }
  int err = h.hsc->err;
  for (int64_t r : roots_h)
    if (r != 1) err |= ERR_NOT_A_TREE;
  if (acyclic && !(err & (ERR_NOT_CSR | ERR_BAD_WEIGHT | ERR_NOT_A_TREE | ERR_CROSS_GRAPH))) {
    // acyclicity and depth by pointer jumping (sparsify_init leaves both to the tree layout, whose Euler tour
    // reaches every vertex only if the parent links are acyclic, and checks the fixed-point range there)
    int bits = 0;
    while ((1ll << bits) <= n) bits++;
    int cur = 0;
    bool done = false;
    for (int round = 0; round <= bits + 1; round++) {
      k_val_active_reset<<<1, 1, 0, h.stream>>>(h.dsc);
      k_val_jump<<<grid, kBlock, 0, h.stream>>>(jmp[cur], jmp[cur ^ 1], dep[cur], dep[cur ^ 1], n, h.dsc);
      cur ^= 1;
      if (!fetch()) {
        cleanup();
        return check_cuda(cudaGetLastError());
      }
      if (h.hsc->active == 0) {
        done = true;
        break;
      }
    }
    if (!done) err |= ERR_NOT_A_TREE;
    h.max_depth = h.hsc->max_depth;
    if (!done) h.max_depth = 0;
    // fixed-point range of the exact root distances
    int dep_bits = 0;
    while ((1ll << dep_bits) <= h.max_depth) dep_bits++;
    if (done && h.hsc->e_max != INT_MIN && h.hsc->e_max - h.hsc->e_min + 53 + dep_bits > 96) err |= ERR_RANGE;
  }
  cleanup();
  if (err & ERR_NOT_CSR) st = PDG_E_NOT_CSR;
  else if (err & ERR_BAD_WEIGHT) st = PDG_E_BAD_WEIGHT;
  else if (err & ERR_CROSS_GRAPH) st = PDG_E_INVALID_ARG;
  else if (err & ERR_NOT_SYMMETRIC) st = PDG_E_NOT_SYMMETRIC;
  else if (err & ERR_NOT_A_TREE) st = PDG_E_NOT_A_TREE;
  else if (err & ERR_RANGE) st = PDG_E_RANGE;
  return st;
}

}  // namespace pdg
