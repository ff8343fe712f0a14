// Step A2: tree preprocessing of Algorithm 1 (root distances "dists" and the
// skip table for LCA queries, Algorithm 1 step 1; Sec. 4.2 work/span analysis).
//
// Root distances are EXACT: every r(v) = fl(1/w(v, parent v)) is a multiple
// of 2^-S with S = 52 - min_v exponent(r(v)), so D(v) = sum of r on the root
// path is an integer in units of 2^-S.  Integer addition is associative, so
// pointer jumping produces the same bits as any sequential walk, and
// R_T(u, v) = D(u) + D(v) - 2 D(LCA) is exact before its single rounding.
//
// Each vertex carries one 128-bit word P(v) = D(v) * 2^32 + hops(v): one
// 16-byte gather moves both the distance and the hop depth, and one 128-bit
// add advances both during pointer jumping (depth < 2^30 never carries into
// D).  D must stay below 2^96; this is checked from the exponent range and
// the maximum depth before jumping (PDG_E_RANGE otherwise).
//
// Pointer jumping: after round j, jump(v) = anc_{2^(j+1)}(v) and P(v) sums
// the path from v up to (not including) jump(v), or to the root.  The jump
// pointers of the rounds are the binary-lifting table (level j = anc_{2^j}).
#include <climits>

#include "pdg_internal.cuh"

namespace pdg {

namespace {

// P(v) of the bare edge to the parent: fixed(r(v)) * 2^32 + 1 (0 at a root).
// fixed(r) = mant * 2^(e - 52 + S) with S = 52 - e_min.
__device__ __forceinline__ u128 edge_word(double r, int e_min, bool range_ok) {
  const uint64_t b = (uint64_t)__double_as_longlong(r);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = e - e_min;
  const u128 fixed = (range_ok && sh >= 0 && sh <= 74) ? ((u128)mant << sh) : (u128)0;
  return (fixed << 32) | (u128)1;
}

__device__ __forceinline__ bool range_fits(DevScalars* dsc, int dep_bits) {
  const int e_min = dsc->e_min, e_max = dsc->e_max;
  const bool ok = (e_max == INT_MIN) || (e_max - e_min + 53 + dep_bits <= 96);
  if (blockIdx.x == 0 && threadIdx.x == 0 && !ok) atomicOr(&dsc->err, ERR_RANGE);
  return ok;
}

// The edge words alone (a forest of single vertices has no jumping round).
__global__ void k_tree_init(const int32_t* __restrict__ parent, const double* __restrict__ rtree, int64_t n,
                            int dep_bits, DevScalars* dsc, u128* __restrict__ P0) {
  const bool range_ok = range_fits(dsc, dep_bits);
  const int e_min = dsc->e_min;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    P0[v] = parent[v] >= 0 ? edge_word(rtree[v], e_min, range_ok) : (u128)0;
}

// Round 0 of the pointer jumping with the edge words built on the fly:
// P(v) = word(v) + word(parent v), jump(v) = parent(parent v).
__global__ void __launch_bounds__(kBlock) k_tree_first(const int32_t* __restrict__ parent,
                                                       const double* __restrict__ rtree, int64_t n, int dep_bits,
                                                       DevScalars* dsc, u128* __restrict__ Pout,
                                                       int32_t* __restrict__ jout) {
  const bool range_ok = range_fits(dsc, dep_bits);
  const int e_min = dsc->e_min;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = parent[v];
    u128 p = 0;
    int32_t na = -1;
    if (a >= 0) {
      p = edge_word(rtree[v], e_min, range_ok);
      na = parent[a];
      if (na >= 0) p += edge_word(rtree[a], e_min, range_ok);
    }
    Pout[v] = p;
    if (jout) jout[v] = na;
  }
}

__global__ void __launch_bounds__(kBlock) k_tree_jump(const u128* __restrict__ Pin, u128* __restrict__ Pout,
                                                      const int32_t* __restrict__ jin,
                                                      int32_t* __restrict__ jout, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = jin[v];
    u128 p = Pin[v];
    int32_t na = -1;
    if (a >= 0) {
      p += Pin[a];
      na = jin[a];
    }
    Pout[v] = p;
    if (jout) jout[v] = na;
  }
}

}  // namespace

int step_tree(Handle& h) {
  const int64_t n = h.n;
  const int grid = grid_for(h, n);
  int dep_bits = 0;
  while ((1ll << dep_bits) <= h.max_depth) dep_bits++;
  int cur = 0;
  if (h.J == 0) {  // no vertex has a parent
    ++h.launches;
    k_tree_init<<<grid, kBlock, 0, h.stream>>>(h.parent, h.rtree, n, dep_bits, h.dsc, h.P[0]);
  } else {
    ++h.launches;
    k_tree_first<<<grid, kBlock, 0, h.stream>>>(h.parent, h.rtree, n, dep_bits, h.dsc, h.P[1],
                                                 h.J > 1 ? h.up : nullptr);
    cur = 1;
  }
  PDG_CUDA(cudaGetLastError());
  for (int j = 1; j < h.J; j++) {
    const int32_t* jin = h.up + (int64_t)(j - 1) * n;
    int32_t* jout = (j + 1 < h.J) ? h.up + (int64_t)j * n : nullptr;
    ++h.launches;
    k_tree_jump<<<grid, kBlock, 0, h.stream>>>(h.P[cur], h.P[cur ^ 1], jin, jout, n);
    cur ^= 1;
  }
  PDG_CUDA(cudaGetLastError());
  h.p_final = cur;
  return PDG_OK;
}

}  // namespace pdg
