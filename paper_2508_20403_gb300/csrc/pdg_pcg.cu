// Sparsifier quality: preconditioned conjugate gradients on L_G x = b with
// the sparsifier's Laplacian L_P (spanning tree T plus the recovered edges A)
// as the preconditioner, to a relative residual tol (Sec. 5 measures
// sparsifiers by these iteration counts, tol 1e-3).
//
//   b' = b - mean(b); x = 0, r = b', z = M(r), p = z
//   repeat: a = (r.z) / (p.L_G p); x += a p; r -= a L_G p;
//           stop when ||r|| <= tol ||b'||;
//           z = M(r); beta = (r.z)_new / (r.z)_old; p = z + beta p
//
// M(r) solves L_P z = r grounded at the tree root (z(root) = 0, the root's
// equation dropped), then centres z.  Grounded, L_P = L_T + U W U^T with U
// the incidence columns of the k recovered edges, so (Woodbury)
//   L_P^-1 = L_T^-1 - L_T^-1 U C^-1 U^T L_T^-1,  C = W^-1 + U^T L_T^-1 U (k x k, SPD).
// A grounded tree solve L_T x = y is two prefix sums over the Euler tour:
// the flow on the edge above c is the sum of y over the subtree of c (the
// positions between c's entry and exit arcs), and x(v) sums flow / w over
// the root path of v (+ at each entry, - at each exit, read at v's entry).
// C is built column by column from k tree solves and inverted once
// (Gauss-Jordan; C is SPD, so no pivoting); every sum runs in a fixed order,
// so the result is deterministic.  Dense C: k <= kPcgMaxEdges.
#include <cmath>
#include <type_traits>
#include <vector>

#include "pdg_internal.cuh"
#include "pdg_tour.cuh"

namespace pdg {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_pc_tflag(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                           const int32_t* __restrict__ parent, int64_t m, uint8_t* __restrict__ tflag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    tflag[e] = (parent[ev[e]] == eu[e] || parent[eu[e]] == ev[e]) ? 1 : 0;
}

__global__ void k_pc_cut(const int32_t* __restrict__ rev, const int64_t* __restrict__ tptr,
                         const int32_t* __restrict__ tdeg, int32_t root, int32_t* __restrict__ succ,
                         int32_t* __restrict__ rd) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && tdeg[root] > 0) {
    const int32_t tail = rev[tptr[root] + tdeg[root] - 1];
    succ[tail] = -1;
    rd[tail] = 0;
  }
}

// entry / exit positions of every non-root vertex and the weight of the edge above it
__global__ void k_pc_times(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                           const double* __restrict__ ew, const uint8_t* __restrict__ tflag,
                           const int32_t* __restrict__ arc_uv, const int32_t* __restrict__ rev,
                           const int32_t* __restrict__ rd, const int64_t* __restrict__ tptr, int64_t n, int64_t m,
                           int32_t* __restrict__ tin, int32_t* __restrict__ tout, double* __restrict__ wup) {
  const int64_t last = tptr[n] - 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    if (!tflag[e]) continue;
    const int32_t a1 = arc_uv[e], a2 = rev[a1];
    const bool down1 = rd[a1] > rd[a2];  // u -> v comes first: u is the parent
    const int32_t child = down1 ? ev[e] : eu[e];
    tin[child] = (int32_t)(last - rd[down1 ? a1 : a2]);
    tout[child] = (int32_t)(last - rd[down1 ? a2 : a1]);
    wup[child] = ew[e];
  }
}

// --- exclusive scans of doubles (fixed order: tile scans, one scan of the tile sums, add) ---
__device__ __forceinline__ double warp_incl_scan_d(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// exclusive scan of this block's kScanTile elements; returns the tile total to thread 0's caller via *tot
__device__ double block_excl_scan_d(double (&v)[kScanItems], double* sh, double* tot) {
  double s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    const double t = v[i];
    v[i] = s;
    s += t;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double incl = warp_incl_scan_d(s);
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    const double x = (lane < kScanThreads / 32) ? sh[lane] : 0.0;
    const double xi = warp_incl_scan_d(x);
    sh[lane] = xi - x;
    if (lane == 31) sh[32] = xi;
  }
  __syncthreads();
  const double base = sh[w] + incl - s;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) v[i] += base;
  *tot = sh[32];
  return base;
}

__global__ void __launch_bounds__(kScanThreads) k_pc_scan_tiles(const double* __restrict__ in, int64_t N,
                                                                double* __restrict__ out, double* __restrict__ sums) {
  __shared__ double sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  double v[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; i++) v[i] = (base + i < N) ? in[base + i] : 0.0;
  double tot;
  block_excl_scan_d(v, sh, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; i++)
    if (base + i < N) out[base + i] = v[i];
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of the tile sums (at most kScanTile tiles)
__global__ void __launch_bounds__(kScanThreads) k_pc_scan_sums(double* __restrict__ sums, int64_t T) {
  __shared__ double sh[33];
  const int64_t base = (int64_t)threadIdx.x * kScanItems;
  double v[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; i++) v[i] = (base + i < T) ? sums[base + i] : 0.0;
  double tot;
  block_excl_scan_d(v, sh, &tot);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; i++)
    if (base + i < T) sums[base + i] = v[i];
}

__global__ void k_pc_scan_add(double* __restrict__ out, int64_t N, const double* __restrict__ sums) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] += sums[i / kScanTile];
}

// --- the grounded tree solve ---
__global__ void k_pc_place(const double* __restrict__ y, const int32_t* __restrict__ tin, int64_t n, int32_t root,
                           double* __restrict__ Y) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (v != root) Y[tin[v]] = y[v];
}

// flow over the edge above c = sum of y over c's subtree; potential drop = flow / w
__global__ void k_pc_drops(const double* __restrict__ E, const int32_t* __restrict__ tin,
                           const int32_t* __restrict__ tout, const double* __restrict__ wup, int64_t n, int32_t root,
                           double* __restrict__ Z) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    if (c == root) continue;
    const double t = (E[tout[c]] - E[tin[c]]) / wup[c];
    Z[tin[c]] = t;
    Z[tout[c]] = -t;
  }
}

__global__ void k_pc_potential(const double* __restrict__ E2, const double* __restrict__ Z,
                               const int32_t* __restrict__ tin, int64_t n, int32_t root, double* __restrict__ x) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = (v == root) ? 0.0 : E2[tin[v]] + Z[tin[v]];
}

// --- the k recovered edges ---
__global__ void k_pc_edges(const int32_t* __restrict__ ids, int64_t k, int64_t m, const int32_t* __restrict__ eu,
                           const int32_t* __restrict__ ev, const double* __restrict__ ew,
                           const uint8_t* __restrict__ tflag, int32_t* __restrict__ ea, int32_t* __restrict__ eb,
                           double* __restrict__ ewk, int32_t* __restrict__ bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t id = ids[i];
    if (id < 0 || id >= m || tflag[id]) {
      *bad = 1;
      ea[i] = eb[i] = 0;
      ewk[i] = 1.0;
      continue;
    }
    ea[i] = eu[id];
    eb[i] = ev[id];
    ewk[i] = ew[id];
  }
}

__global__ void k_pc_dups(const int32_t* __restrict__ ids, int64_t k, int64_t m, int32_t* __restrict__ seen,
                          int32_t* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t id = ids[i];
    if (id >= 0 && id < m && atomicAdd(&seen[id], 1) != 0) *bad = 1;
  }
}

// column j of C: C[i][j] = x(a_i) - x(b_i) (+ 1 / w_j on the diagonal), x = L_T^-1 (e_a_j - e_b_j)
__global__ void k_pc_unit(int32_t a, int32_t b, int32_t root, double* __restrict__ y) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (a != root) y[a] = 1.0;
    if (b != root) y[b] = -1.0;
  }
}

__global__ void k_pc_unit_clear(int32_t a, int32_t b, double* __restrict__ y) {
  if (blockIdx.x == 0 && threadIdx.x == 0) y[a] = y[b] = 0.0;
}

__global__ void k_pc_column(const double* __restrict__ x, const int32_t* __restrict__ ea,
                            const int32_t* __restrict__ eb, const double* __restrict__ ewk, int64_t k, int64_t j,
                            double* __restrict__ C) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    C[i * k + j] = x[ea[i]] - x[eb[i]] + (i == j ? 1.0 / ewk[j] : 0.0);
}

// Gauss-Jordan inversion in place, pivot p: copy the pivot row and column, then update
__global__ void k_pc_gj_copy(const double* __restrict__ C, int64_t k, int64_t p, double* __restrict__ row,
                             double* __restrict__ col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    row[i] = C[p * k + i];
    col[i] = C[i * k + p];
  }
}

__global__ void k_pc_gj_update(double* __restrict__ C, int64_t k, int64_t p, const double* __restrict__ row,
                               const double* __restrict__ col) {
  const double d = 1.0 / row[p];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < k * k; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / k, j = q % k;
    double v;
    if (i == p && j == p) v = d;
    else if (i == p) v = row[j] * d;
    else if (j == p) v = -col[i] * d;
    else v = C[q] - col[i] * row[j] * d;
    C[q] = v;
  }
}

// s_i = t(a_i) - t(b_i)
__global__ void k_pc_gather_s(const double* __restrict__ t, const int32_t* __restrict__ ea,
                              const int32_t* __restrict__ eb, int64_t k, double* __restrict__ s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    s[i] = t[ea[i]] - t[eb[i]];
}

// q = C^-1 s, one warp per row
__global__ void k_pc_gemv(const double* __restrict__ Ci, const double* __restrict__ s, int64_t k,
                          double* __restrict__ q) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < k; i += nw) {
    double acc = 0;
    for (int64_t j = lane; j < k; j += 32) acc += Ci[i * k + j] * s[j];
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) q[i] = acc;
  }
}

// y(v) = sum over the recovered edges at v of +-q_i, in edge order (incidence lists)
__global__ void k_pc_incident(const int64_t* __restrict__ iptr, const int32_t* __restrict__ iedge,
                              const int32_t* __restrict__ ea, const double* __restrict__ q, int64_t n,
                              double* __restrict__ y) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0;
    for (int64_t p = iptr[v]; p < iptr[v + 1]; p++) {
      const int32_t i = iedge[p];
      acc += (ea[i] == (int32_t)v) ? q[i] : -q[i];
    }
    y[v] = acc;
  }
}

__global__ void k_pc_inc_count(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, int64_t k,
                               int32_t* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    atomicAdd(&cnt[ea[i]], 1);
    atomicAdd(&cnt[eb[i]], 1);
  }
}

__global__ void k_pc_inc_fill(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb, int64_t k,
                              const int64_t* __restrict__ iptr, int32_t* __restrict__ cur, int32_t* __restrict__ iedge) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    iedge[iptr[ea[i]] + atomicAdd(&cur[ea[i]], 1)] = (int32_t)i;
    iedge[iptr[eb[i]] + atomicAdd(&cur[eb[i]], 1)] = (int32_t)i;
  }
}

// each incidence list in increasing edge order (a fixed summation order)
__global__ void k_pc_inc_sort(const int64_t* __restrict__ iptr, int64_t n, int32_t* __restrict__ iedge) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = iptr[v], e = iptr[v + 1];
    for (int64_t p = b + 1; p < e; p++) {
      const int32_t x = iedge[p];
      int64_t q = p - 1;
      while (q >= b && iedge[q] > x) {
        iedge[q + 1] = iedge[q];
        q--;
      }
      iedge[q + 1] = x;
    }
  }
}

// --- vectors ---
__global__ void k_pc_degw(const int64_t* __restrict__ row_ptr, const double* __restrict__ w, int64_t n,
                          double* __restrict__ dw) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; p++) s += w[p];
    dw[v] = s;
  }
}

// y = L_G x (row order of the CSR)
__global__ void k_pc_spmv(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                          const double* __restrict__ w, const double* __restrict__ dw, const double* __restrict__ x,
                          int64_t n, double* __restrict__ y) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double s = dw[v] * x[v];
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; p++) s -= w[p] * x[col[p]];
    y[v] = s;
  }
}

constexpr int kDotBlocks = 256;

// partial sums of a.b per block (grid-stride in a fixed assignment), then one block adds them in order
__global__ void __launch_bounds__(256) k_pc_dot_part(const double* __restrict__ a, const double* __restrict__ b,
                                                     int64_t n, double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (b ? a[i] * b[i] : a[i]);
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < 8; i++) t += sh[i];
    part[blockIdx.x] = t;
  }
}

__global__ void k_pc_dot_final(const double* __restrict__ part, double* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < kDotBlocks; i++) t += part[i];
    *out = t;
  }
}

// v -= sum / n (centring against the all-ones null space)
__global__ void k_pc_center(double* __restrict__ v, int64_t n, const double* __restrict__ sum) {
  const double mu = *sum / (double)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] -= mu;
}

__global__ void k_pc_axpy(double* __restrict__ y, const double* __restrict__ x, double a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

// p = z + beta p
__global__ void k_pc_xpby(double* __restrict__ p, const double* __restrict__ z, double beta, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

__global__ void k_pc_sub(double* __restrict__ z, const double* __restrict__ t, const double* __restrict__ u,
                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = t[i] - u[i];
}

}  // namespace

// a failed CUDA call releases the temporaries and reports PDG_E_CUDA
#define PC_CK(x)                                     \
  do {                                               \
    if ((x) != cudaSuccess) return fail(PDG_E_CUDA); \
  } while (0)

int pcg_quality(Handle& h, const int32_t* ids, int64_t k, const double* b, double tol, int32_t max_iter,
                int32_t* iters, double* relres, double* hist, double* z0) {
  const int64_t n = h.n, m = h.m;
  cudaStream_t s = h.stream;
  const int gn = grid_for(h, n), gm = grid_for(h, std::max<int64_t>(m, 1)), gk = grid_for(h, std::max<int64_t>(k, 1));
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
  // the root of the tree
  int32_t root = -1;
  {
    std::vector<int32_t> par(n);
    if (cudaMemcpyAsync(par.data(), h.parent, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(PDG_E_CUDA);
    for (int64_t v = 0; v < n && root < 0; v++)
      if (par[v] < 0) root = (int32_t)v;
  }
  if (root < 0) return fail(PDG_E_NOT_A_TREE);
  const int64_t A = 2 * (n - 1);
  const int64_t T = (A + 1 + kScanTile - 1) / kScanTile;  // scan tiles over A + 1 positions
  if (T > kScanTile) return fail(PDG_E_INVALID_ARG);      // one block scans the tile sums
  uint8_t* tflag = nullptr;
  int32_t *tdeg = nullptr, *cur = nullptr, *tadj = nullptr, *rev = nullptr, *arc_uv = nullptr;
  int32_t *succ[2] = {nullptr, nullptr}, *rd[2] = {nullptr, nullptr}, *tin = nullptr, *tout = nullptr;
  int32_t *ea = nullptr, *eb = nullptr, *seen = nullptr, *flags = nullptr, *icnt = nullptr, *iedge = nullptr;
  int64_t *tptr = nullptr, *iptr = nullptr;
  double *wup = nullptr, *Y = nullptr, *E = nullptr, *Z = nullptr, *E2 = nullptr, *sums = nullptr, *ewk = nullptr;
  double *C = nullptr, *grow = nullptr, *gcol = nullptr, *dw = nullptr, *bb = nullptr, *x = nullptr, *r = nullptr;
  double *z = nullptr, *p = nullptr, *Ap = nullptr, *t = nullptr, *u = nullptr, *yv = nullptr, *sv = nullptr;
  double *qv = nullptr, *part = nullptr, *dsc = nullptr;
  if (!talloc(&tflag, m) || !talloc(&tdeg, n) || !talloc(&cur, n) || !talloc(&tptr, n + 1) ||
      !talloc(&tadj, A) || !talloc(&rev, A) || !talloc(&arc_uv, m) || !talloc(&succ[0], A) || !talloc(&succ[1], A) ||
      !talloc(&rd[0], A) || !talloc(&rd[1], A) || !talloc(&tin, n) || !talloc(&tout, n) || !talloc(&wup, n) ||
      !talloc(&Y, A + 1) || !talloc(&E, A + 1) || !talloc(&Z, A + 1) || !talloc(&E2, A + 1) || !talloc(&sums, T) ||
      !talloc(&ea, k) || !talloc(&eb, k) || !talloc(&ewk, k) || !talloc(&seen, m) || !talloc(&flags, 4) ||
      !talloc(&icnt, n) || !talloc(&iptr, n + 1) || !talloc(&iedge, 2 * k) || !talloc(&C, k * k) ||
      !talloc(&grow, k) || !talloc(&gcol, k) || !talloc(&dw, n) || !talloc(&bb, n) || !talloc(&x, n) ||
      !talloc(&r, n) || !talloc(&z, n) || !talloc(&p, n) || !talloc(&Ap, n) || !talloc(&t, n) || !talloc(&u, n) ||
      !talloc(&yv, n) || !talloc(&sv, k) || !talloc(&qv, k) || !talloc(&part, kDotBlocks) || !talloc(&dsc, 4))
    return fail(PDG_E_OOM);
  int st = PDG_OK;
  // Euler tour of the tree
  k_pc_tflag<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, h.parent, m, tflag);
  PC_CK(cudaMemsetAsync(tdeg, 0, sizeof(int32_t) * n, s));
  PC_CK(cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, s));
  k_st_tdeg<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tdeg);
  if ((st = ensure_scan_status(h, n)) || (st = scan_excl_i32(h, tdeg, tptr, n, nullptr, n))) return fail(st);
  {
    int64_t arcs = -1;
    if (cudaMemcpyAsync(&arcs, tptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(PDG_E_CUDA);
    if (arcs != A) return fail(PDG_E_NOT_A_TREE);  // the parent links are the n - 1 tree edges
  }
  k_st_fill<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tptr, cur, tadj, rev, arc_uv);
  // rows in neighbour order: the tour, and so every sum along it, is the same on every run
  k_tour_sort_rows<<<gn, kBlock, 0, s>>>(tptr, n, tadj);
  k_tour_fix_rev<<<gn, kBlock, 0, s>>>(tptr, tadj, n, rev);
  k_tour_fix_arcs<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, tflag, m, tptr, tadj, arc_uv);
  const int ga = grid_for(h, std::max<int64_t>(A, 1));
  k_st_succ<<<ga, kBlock, 0, s>>>(tadj, rev, tptr, tdeg, n, succ[0], rd[0]);
  k_pc_cut<<<1, 32, 0, s>>>(rev, tptr, tdeg, root, succ[0], rd[0]);
  int bits = 1;
  while ((1ll << bits) <= A) bits++;
  int c = 0;
  for (int it = 0; it < bits; it++) {
    k_st_rank<<<ga, kBlock, 0, s>>>(succ[c], rd[c], succ[c ^ 1], rd[c ^ 1], tptr, n);
    c ^= 1;
  }
  k_pc_times<<<gm, kBlock, 0, s>>>(h.el_u, h.el_v, h.el_w, tflag, arc_uv, rev, rd[c], tptr, n, m, tin, tout, wup);
  // the grounded tree solve x = L_T^-1 y
  const int64_t NA = A + 1;
  const int tiles = (int)T;
  auto scan = [&](const double* in, double* out) {
    k_pc_scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, NA, out, sums);
    k_pc_scan_sums<<<1, kScanThreads, 0, s>>>(sums, T);
    k_pc_scan_add<<<grid_for(h, NA), kBlock, 0, s>>>(out, NA, sums);
  };
  auto tree_solve = [&](const double* yin, double* xout) -> bool {
    if (cudaMemsetAsync(Y, 0, sizeof(double) * NA, s) != cudaSuccess) return false;
    k_pc_place<<<gn, kBlock, 0, s>>>(yin, tin, n, root, Y);
    scan(Y, E);
    if (cudaMemsetAsync(Z, 0, sizeof(double) * NA, s) != cudaSuccess) return false;
    k_pc_drops<<<gn, kBlock, 0, s>>>(E, tin, tout, wup, n, root, Z);
    scan(Z, E2);
    k_pc_potential<<<gn, kBlock, 0, s>>>(E2, Z, tin, n, root, xout);
    return true;
  };
  // the recovered edges (distinct off-tree canonical ids)
  PC_CK(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 4, s));
  PC_CK(cudaMemsetAsync(seen, 0, sizeof(int32_t) * std::max<int64_t>(m, 1), s));
  if (k > 0) {
    k_pc_edges<<<gk, kBlock, 0, s>>>(ids, k, m, h.el_u, h.el_v, h.el_w, tflag, ea, eb, ewk, flags);
    k_pc_dups<<<gk, kBlock, 0, s>>>(ids, k, m, seen, flags + 1);
  }
  {
    int32_t hf[2] = {0, 0};
    if (cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(PDG_E_CUDA);
    if (hf[0] || hf[1]) return fail(PDG_E_INVALID_ARG);
  }
  // capacitance matrix C and its inverse
  if (k > 0) {
    PC_CK(cudaMemsetAsync(yv, 0, sizeof(double) * n, s));
    std::vector<int32_t> ha(k), hb(k);
    if (cudaMemcpyAsync(ha.data(), ea, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hb.data(), eb, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(PDG_E_CUDA);
    for (int64_t j = 0; j < k; j++) {
      k_pc_unit<<<1, 32, 0, s>>>(ha[j], hb[j], root, yv);
      if (!tree_solve(yv, t)) return fail(PDG_E_CUDA);
      k_pc_column<<<gk, kBlock, 0, s>>>(t, ea, eb, ewk, k, j, C);
      k_pc_unit_clear<<<1, 32, 0, s>>>(ha[j], hb[j], yv);
    }
    const int gkk = grid_for(h, k * k);
    for (int64_t q = 0; q < k; q++) {
      k_pc_gj_copy<<<gk, kBlock, 0, s>>>(C, k, q, grow, gcol);
      k_pc_gj_update<<<gkk, kBlock, 0, s>>>(C, k, q, grow, gcol);
    }
    // incidence lists of the recovered edges, in edge order
    PC_CK(cudaMemsetAsync(icnt, 0, sizeof(int32_t) * n, s));
    PC_CK(cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, s));
    k_pc_inc_count<<<gk, kBlock, 0, s>>>(ea, eb, k, icnt);
    if ((st = scan_excl_i32(h, icnt, iptr, n, nullptr, n))) return fail(st);
    k_pc_inc_fill<<<gk, kBlock, 0, s>>>(ea, eb, k, iptr, cur, iedge);
    k_pc_inc_sort<<<gn, kBlock, 0, s>>>(iptr, n, iedge);
  }
  // the preconditioner M(v) -> zout
  auto precond = [&](const double* vin, double* zout) -> bool {
    if (!tree_solve(vin, t)) return false;
    if (k > 0) {
      k_pc_gather_s<<<gk, kBlock, 0, s>>>(t, ea, eb, k, sv);
      k_pc_gemv<<<grid_for(h, 32 * k), kBlock, 0, s>>>(C, sv, k, qv);
      k_pc_incident<<<gn, kBlock, 0, s>>>(iptr, iedge, ea, qv, n, yv);
      if (!tree_solve(yv, u)) return false;
      k_pc_sub<<<gn, kBlock, 0, s>>>(zout, t, u, n);
    } else if (cudaMemcpyAsync(zout, t, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      return false;
    }
    k_pc_dot_part<<<kDotBlocks, 256, 0, s>>>(zout, nullptr, n, part);
    k_pc_dot_final<<<1, 32, 0, s>>>(part, dsc + 3);
    k_pc_center<<<gn, kBlock, 0, s>>>(zout, n, dsc + 3);
    return true;
  };
  auto dot = [&](const double* a, const double* bv, double* out_h) -> bool {
    k_pc_dot_part<<<kDotBlocks, 256, 0, s>>>(a, bv, n, part);
    k_pc_dot_final<<<1, 32, 0, s>>>(part, dsc);
    return cudaMemcpyAsync(out_h, dsc, sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
  };
  // PCG
  k_pc_degw<<<gn, kBlock, 0, s>>>(h.row_ptr, h.w, n, dw);
  PC_CK(cudaMemcpyAsync(bb, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  k_pc_dot_part<<<kDotBlocks, 256, 0, s>>>(bb, nullptr, n, part);
  k_pc_dot_final<<<1, 32, 0, s>>>(part, dsc + 3);
  k_pc_center<<<gn, kBlock, 0, s>>>(bb, n, dsc + 3);
  PC_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  PC_CK(cudaMemcpyAsync(r, bb, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  double nb2 = 0, rz = 0, pAp = 0, rr = 0;
  if (!dot(bb, bb, &nb2)) return fail(PDG_E_CUDA);
  const double nb = std::sqrt(nb2);
  if (!(nb > 0)) {
    *iters = 0;
    *relres = 0.0;
    cleanup();
    return PDG_OK;
  }
  if (!precond(r, z)) return fail(PDG_E_CUDA);
  if (z0) {  // the preconditioner applied to b' (host copy for the caller)
    PC_CK(cudaMemcpyAsync(z0, z, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    PC_CK(cudaStreamSynchronize(s));
  }
  PC_CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (!dot(r, z, &rz)) return fail(PDG_E_CUDA);
  double rel = 1.0;
  int32_t it = 0;
  for (it = 1; it <= max_iter; it++) {
    k_pc_spmv<<<gn, kBlock, 0, s>>>(h.row_ptr, h.col, h.w, dw, p, n, Ap);
    if (!dot(p, Ap, &pAp)) return fail(PDG_E_CUDA);
    const double a = rz / pAp;
    k_pc_axpy<<<gn, kBlock, 0, s>>>(x, p, a, n);
    k_pc_axpy<<<gn, kBlock, 0, s>>>(r, Ap, -a, n);
    if (!dot(r, r, &rr)) return fail(PDG_E_CUDA);
    rel = std::sqrt(rr) / nb;
    if (hist) hist[it - 1] = rel;
    if (rel <= tol) break;
    if (!precond(r, z)) return fail(PDG_E_CUDA);
    double rz_new = 0;
    if (!dot(r, z, &rz_new)) return fail(PDG_E_CUDA);
    k_pc_xpby<<<gn, kBlock, 0, s>>>(p, z, rz_new / rz, n);
    rz = rz_new;
  }
  *iters = std::min(it, max_iter);
  *relres = rel;
  if (cudaGetLastError() != cudaSuccess) return fail(PDG_E_CUDA);
  cleanup();
  return PDG_OK;
}

#undef PC_CK

}  // namespace pdg
