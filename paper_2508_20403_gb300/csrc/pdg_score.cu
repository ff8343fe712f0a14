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
// edge (P(u), P(v) with the masks; the keys; P(l)).  The conversion runs on
// the integer pipes (pdg_fp.cuh); the product is one FP64 multiply, which the
// FP64 pipe takes in fewer issue slots than an integer version of it.
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
  const uint64_t* pmin[kRmqMaxLevels];
  const uint64_t* smin[kRmqMaxLevels];
  const uint64_t* st;  // level 2 and up as a sparse table (null: as levels)
  int64_t st_n;        // its row length (the level-2 entries)
  int S;
  int score_mode;
  uint32_t n;
  int* err;
  uint64_t* key;
  int32_t* lca;
  uint32_t* hist;  // nullable: the first-level selection histogram (key >> 52) of a single graph
};

// minimum of val0 over the labels [lo, hi] (lo <= hi), by depth.  Level j
// holds the query range [a_j, b_j].  If both ends share a group the range is
// answered there by its mask and one key; otherwise the tail of a_j's group
// (smin) and the head of b_j's group (pmin) are single loads, and the groups
// strictly between become the range of level j + 1.  When level 2 and up are
// one sparse table, a range that reaches level 2 is answered there by two
// loads.  Every address depends only on (lo, hi), so all loads but the last
// key are issued together.
__device__ __forceinline__ uint64_t range_min(const ScoreArgs& A, uint32_t lo, uint32_t hi) {
  uint64_t best = ~0ull;
  bool done = false;
  uint32_t fa = 0, fb = 0;  // the single-group range of the last level, if any
  int fj = -1;
#pragma unroll
  for (int j = 0; j < kRmqMaxLevels; j++) {
    if (!done && j == 2 && A.st) {  // the rest of the range, on level 2, from two entries of the sparse table
      const int t = 31 - __clz(hi - lo + 1);
      const uint64_t* row = A.st + (int64_t)t * A.st_n;
      best = min(best, min(__ldg(row + lo), __ldg(row + hi + 1 - (1u << t))));
      done = true;
    }
    if (!done) {
      if ((lo >> 5) == (hi >> 5)) {
        fa = lo;
        fb = hi;
        fj = j;
        done = true;
      } else {
        best = min(best, min(__ldg(A.smin[j] + lo), __ldg(A.pmin[j] + hi)));
        lo = (lo >> 5) + 1;
        hi = (hi >> 5) - 1;
        done = lo > hi;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kRmqMaxLevels; j++) {
    if (j == fj) {
      const uint32_t m = __ldg(A.mask[j] + fb);
      const uint32_t o = fa & 31u;
      best = min(best, __ldg(A.val[j] + ((fb & ~31u) | (o + __ffs(m >> o) - 1))));
    }
  }
  return best;
}

__device__ __forceinline__ void score_edge(const ScoreArgs& A, int64_t i, uint32_t* s_hist) {
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
  const uint64_t rb = fixed_hl_to_bits((uint64_t)(r_fixed >> 64), (uint64_t)r_fixed, A.S);  // below 2^97
  uint64_t sb = rb;
  if (A.score_mode != PDG_SCORE_RESISTANCE)  // one IEEE multiply, rounded to nearest-even
    sb = (uint64_t)__double_as_longlong(__dmul_rn(A.ow[i], __longlong_as_double((long long)rb)));
  A.key[i] = sb;
  A.lca[i] = l;
  if (s_hist) atomicAdd(&s_hist[sb >> 52], 1u);
}

// Long edge lists (a big packed batch) are scored in tiles of kScoreTile
// edges that warps take in id order from a ticket counter: the edges in
// flight then stay a narrow window, so the tree tables being gathered from
// (those of a few graphs) stay in L2 however many graphs the batch holds.
// Shorter lists use a plain grid-stride loop, whose window is narrower still.
constexpr int64_t kTicketMinEdges = 1ll << 24;

// Eight blocks per SM (32 registers, a few bytes spilled): the gathers of a
// full SM's warps in flight hide more of their latency than the registers saved.
__global__ void __launch_bounds__(kBlock, 8) k_score(ScoreArgs A, int64_t E, DevScalars* __restrict__ dsc) {
  dep_sync();
  __shared__ uint32_t s_hist[kSelBins];
  uint32_t* sh = A.hist ? s_hist : nullptr;  // uniform over the grid
  if (sh) {
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
  }
  A.S = 52 - dsc->e_min;
  if (E < kTicketMinEdges) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x)
      score_edge(A, i, sh);
  } else {
    const int lane = threadIdx.x & 31;
    for (;;) {
      unsigned long long tk = 0;
      if (lane == 0) tk = atomicAdd(&dsc->score_ticket, 1ull);
      tk = __shfl_sync(0xffffffffu, tk, 0);
      const int64_t i0 = (int64_t)tk * kScoreTile;
      if (i0 >= E) break;
      const int64_t i1 = min(E, i0 + kScoreTile);
      for (int64_t i = i0 + lane; i < i1; i += 32) score_edge(A, i, sh);
    }
  }
  if (sh) {
    __syncthreads();
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
      if (sh[i]) atomicAdd(&A.hist[i], sh[i]);
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
    const int jj = j < h.rmq_levels ? j : h.rmq_levels - 1;
    A.val[j] = h.rmq_val[jj];
    A.mask[j] = h.rmq_mask[jj];
    A.pmin[j] = h.rmq_pmin[jj];
    A.smin[j] = h.rmq_smin[jj];
  }
  A.st = h.rmq_st;
  A.st_n = h.rmq_st ? h.rmq_size[2] : 0;
  A.score_mode = score_mode;
  A.n = (uint32_t)h.n;
  A.err = &h.dsc->err;
  A.key = h.key;
  A.lca = h.lca;
  A.hist = h.fuse_hist ? h.hist : nullptr;
  launch_k(h, k_score, grid_for(h, h.E_off), kBlock, 0, A, h.E_off, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
