// Step A3: score every off-tree edge (Algorithm 1 step 1: LCA_query,
// distance_query, compute_resistance).
//
//   l   = LCA_T(u, v) by binary lifting over the pointer-jumping table; the
//         children of l toward u and v fall out of the same search and give
//         the record orientation used by the acceptance step (side[i])
//   R_T = D(u) + D(v) - 2 D(l)                       (Eq. RT), exact integer
//         then ONE round-to-nearest-even conversion to FP64
//   score = fl(w * R_T) (STRETCH) or R_T (RESISTANCE)
//
// The score is positive, so its IEEE bit pattern read as an unsigned integer
// orders like the score itself; key[i] stores those bits for the selection
// and sort steps.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kScoreTile = 256;  // off-tree edges per warp ticket

__device__ __forceinline__ int32_t up_level(const int32_t* __restrict__ parent, const int32_t* __restrict__ up,
                                            uint32_t n, int j, int32_t x) {
  // level j >= 1 starts at up + (j - 1) n (a 32 x 32 -> 64-bit product)
  return j == 0 ? __ldg(parent + x) : __ldg(up + (uint64_t)(uint32_t)(j - 1) * n + x);
}

// x * 2^-S rounded to nearest, ties to even; x > 0 and the result is normal.
__device__ __forceinline__ double fixed_to_double(u128 x, int S) {
  const uint64_t hi = (uint64_t)(x >> 64), lo = (uint64_t)x;
  int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  uint64_t q;
  if (p <= 52) {
    q = lo << (52 - p);
  } else {
    const int sh = p - 52;
    q = (uint64_t)(x >> sh);
    const u128 rem = x & ((((u128)1) << sh) - 1);
    const u128 half = ((u128)1) << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) {
      q++;
      if (q == (1ull << 53)) {
        q >>= 1;
        p++;
      }
    }
  }
  const uint64_t bits = ((uint64_t)(p - S + 1023) << 52) | (q & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// The same when x < 2^64: the integer -> FP64 conversion rounds to nearest
// even, and the scaling by 2^-S (scale) is exact because the result is normal.
__device__ __forceinline__ double fixed_to_double_fast(u128 x, int S, double scale) {
  const uint64_t hi = (uint64_t)(x >> 64);
  if (hi == 0) return __dmul_rn(__ull2double_rn((unsigned long long)x), scale);
  return fixed_to_double(x, S);
}

struct ScoreArgs {
  const int32_t* ou;
  const int32_t* ov;
  const double* ow;
  const u128* P;
  const int32_t* parent;
  const int32_t* up;
  uint32_t n;
  int S;
  double scale;  // 2^-S
  int score_mode;
  uint64_t* key;
  int32_t* lca;
  uint8_t* side;
};

__device__ __forceinline__ void score_edge(const ScoreArgs& A, int64_t i) {
  const int32_t* __restrict__ parent = A.parent;
  const int32_t* __restrict__ up = A.up;
  const int32_t u = A.ou[i], v = A.ov[i];
  const u128 Pu = A.P[u], Pv = A.P[v];
  int32_t a = u, b = v;
  uint32_t da = (uint32_t)Pu, db = (uint32_t)Pv;
  const bool swapped = da < db;
  if (swapped) {
    int32_t t = a; a = b; b = t;
    uint32_t s = da; da = db; db = s;
  }
  const int32_t deep = a;
  const uint32_t diff0 = da - db;
  // lift the deeper endpoint by the depth difference, one level per set bit
  for (uint32_t diff = diff0; diff; diff &= diff - 1) a = up_level(parent, up, A.n, __ffs(diff) - 1, a);
  int32_t l = a;
  int32_t sd, so;  // children of the LCA toward the deeper / the other endpoint
  if (a != b) {
    for (int j = 31 - __clz((int)max(db, 1u)); j >= 0; j--) {
      const int32_t ua = up_level(parent, up, A.n, j, a);
      const int32_t ub = up_level(parent, up, A.n, j, b);
      if (ua != ub) {
        a = ua;
        b = ub;
      }
    }
    l = __ldg(parent + a);
    sd = a;
    so = b;
  } else {
    // the shallower endpoint is the LCA and is its own side; the deeper
    // side is its ancestor diff0 - 1 levels up
    so = l;
    sd = deep;
    for (uint32_t d = diff0 - 1; d; d &= d - 1) sd = up_level(parent, up, A.n, __ffs(d) - 1, sd);
  }
  A.side[i] = (swapped ? sd < so : so < sd) ? 1 : 0;
  const u128 Pl = A.P[l];
  const u128 r_fixed = (Pu >> 32) + (Pv >> 32) - ((Pl >> 32) << 1);
  const double R = fixed_to_double_fast(r_fixed, A.S, A.scale);
  const double sc = (A.score_mode == PDG_SCORE_RESISTANCE) ? R : __dmul_rn(A.ow[i], R);
  A.key[i] = (uint64_t)__double_as_longlong(sc);
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
  // 2^-S as a double: S lies in [-848, 952] for weights in [2^-900, 2^900]
  A.scale = __longlong_as_double((long long)((uint64_t)(1023 - A.S) << 52));
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
  ScoreArgs A{h.off_u, h.off_v, h.off_w, h.P[h.p_final], h.parent, h.up, (uint32_t)h.n, 0, 0.0, score_mode,
              h.key,   h.lca,   h.side};
  k_score<<<grid_for(h, h.E_off), kBlock, 0, h.stream>>>(A, h.E_off, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
