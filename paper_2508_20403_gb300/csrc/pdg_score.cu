// Step A3: score every off-tree edge (Algorithm 1 step 1: LCA_query,
// distance_query, compute_resistance).
//
//   l   = LCA_T(u, v): with preorder labels u < v, l is the parent of any
//         vertex of minimum depth among the labels (u, v] -- every vertex
//         there lies in the subtree of l but is not l, and the child of l on
//         v's side lies there -- so one range-minimum query over
//         val0[x] = depth(x) * 2^32 + parent(x) returns depth(l) + 1 and l
//   R_T = D(u) + D(v) - 2 D(l)                       (Eq. RT), exact integer
//         then ONE round-to-nearest-even conversion to FP64
//   score = fl(w * R_T) (STRETCH) or R_T (RESISTANCE)
//
// The query reads at most two partial groups per level of the range-minimum
// structure; the addresses depend only on (u, v), so all mask loads are
// issued together, then all key loads: three dependent rounds of gathers per
// edge (P(u), P(v) with the masks; the keys; P(l)).  The conversion and the
// product run on the integer pipes (pdg_fp.cuh).
//
// The score is positive, so its IEEE bit pattern read as an unsigned integer
// orders like the score itself; key[i] stores those bits for the selection
// and sort steps.
#include "pdg_fp.cuh"
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kScoreTile = 256;  // off-tree edges per warp ticket

struct ScoreArgs {
  const int32_t* ou;
  const int32_t* ov;
  const double* ow;
  const u128* P;
  const uint64_t* val[kRmqMaxLevels];
  const uint32_t* mask[kRmqMaxLevels];
  int S;
  int score_mode;
  uint32_t n;
  int* err;
  uint64_t* key;
  int32_t* lca;
};

// minimum of val0 over the labels [lo, hi] (lo <= hi), by depth.  Level j
// holds the query range [a_j, b_j]; it is answered there if both ends share a
// group, else the tail of a_j's group and the head of b_j's group are read and
// the groups strictly between become the range of level j + 1.
__device__ __forceinline__ uint64_t range_min(const ScoreArgs& A, uint32_t lo, uint32_t hi) {
  uint32_t a[kRmqMaxLevels], b[kRmqMaxLevels];
  int nlev = kRmqMaxLevels;  // levels holding a query
  bool single = false;       // the last of them is one group
#pragma unroll
  for (int j = 0; j < kRmqMaxLevels; j++) {
    a[j] = lo;
    b[j] = hi;
    if (j < nlev) {
      if ((lo >> 5) == (hi >> 5)) {
        nlev = j + 1;
        single = true;
      } else {
        lo = (lo >> 5) + 1;
        hi = (hi >> 5) - 1;
        if (lo > hi) nlev = j + 1;
      }
    }
  }
  uint32_t m0[kRmqMaxLevels], m1[kRmqMaxLevels];
#pragma unroll
  for (int j = 0; j < kRmqMaxLevels; j++) {
    const bool one = single && j == nlev - 1;
    m0[j] = (j < nlev) ? __ldg(A.mask[j] + (one ? b[j] : (a[j] | 31u))) : 0u;
    m1[j] = (j < nlev && !one) ? __ldg(A.mask[j] + b[j]) : 0u;
  }
  uint64_t best = ~0ull;
#pragma unroll
  for (int j = 0; j < kRmqMaxLevels; j++) {
    if (j < nlev) {
      const bool one = single && j == nlev - 1;
      const uint32_t o = a[j] & 31u;
      const uint32_t g0 = (one ? b[j] : a[j]) & ~31u;
      best = min(best, __ldg(A.val[j] + (g0 | (o + __ffs(m0[j] >> o) - 1))));
      if (!one) best = min(best, __ldg(A.val[j] + ((b[j] & ~31u) | (__ffs(m1[j]) - 1))));
    }
  }
  return best;
}

__device__ __forceinline__ void score_edge(const ScoreArgs& A, int64_t i) {
  const int32_t u = A.ou[i], v = A.ov[i];  // preorder labels, u < v
  const u128 Pu = A.P[u], Pv = A.P[v];
  const uint64_t mn = range_min(A, (uint32_t)u + 1, (uint32_t)v);
  int32_t l = (int32_t)(uint32_t)mn;
  if ((uint32_t)l >= A.n) {  // cannot happen for a valid layout: report instead of reading out of range
    atomicOr(A.err, ERR_BOUNDS);
    l = u;
  }
  const u128 Pl = A.P[l];
  const u128 r_fixed = (Pu >> 32) + (Pv >> 32) - ((Pl >> 32) << 1);
  const uint64_t rb = fixed_to_bits(r_fixed, A.S);
  uint64_t sb = rb;
  if (A.score_mode != PDG_SCORE_RESISTANCE) {
    const double w = A.ow[i];
    bool ok;
    sb = mul_rn_bits((uint64_t)__double_as_longlong(w), rb, &ok);
    if (!ok) sb = (uint64_t)__double_as_longlong(__dmul_rn(w, __longlong_as_double((long long)rb)));
  }
  A.key[i] = sb;
  A.lca[i] = l;
}

// Long edge lists (a big packed batch) are scored in tiles of kScoreTile
// edges that warps take in id order from a ticket counter: the edges in
// flight then stay a narrow window, so the tree tables being gathered from
// (those of a few graphs) stay in L2 however many graphs the batch holds.
// Shorter lists use a plain grid-stride loop, whose window is narrower still.
constexpr int64_t kTicketMinEdges = 1ll << 24;

__global__ void __launch_bounds__(kBlock) k_score(ScoreArgs A, int64_t E, DevScalars* __restrict__ dsc) {
  A.S = 52 - dsc->e_min;
  if (E < kTicketMinEdges) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x)
      score_edge(A, i);
    return;
  }
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(&dsc->score_ticket, 1ull);
    tk = __shfl_sync(0xffffffffu, tk, 0);
    const int64_t i0 = (int64_t)tk * kScoreTile;
    if (i0 >= E) break;
    const int64_t i1 = min(E, i0 + kScoreTile);
    for (int64_t i = i0 + lane; i < i1; i += 32) score_edge(A, i);
  }
}

}  // namespace

int step_score(Handle& h, int score_mode) {
  if (h.E_off == 0) return PDG_OK;
  ++h.launches;
  ScoreArgs A{};
  A.ou = h.off_u;
  A.ov = h.off_v;
  A.ow = h.off_w;
  A.P = h.P;
  for (int j = 0; j < kRmqMaxLevels; j++) {
    A.val[j] = h.rmq_val[j < h.rmq_levels ? j : h.rmq_levels - 1];
    A.mask[j] = h.rmq_mask[j < h.rmq_levels ? j : h.rmq_levels - 1];
  }
  A.score_mode = score_mode;
  A.n = (uint32_t)h.n;
  A.err = &h.dsc->err;
  A.key = h.key;
  A.lca = h.lca;
  k_score<<<grid_for(h, h.E_off), kBlock, 0, h.stream>>>(A, h.E_off, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
