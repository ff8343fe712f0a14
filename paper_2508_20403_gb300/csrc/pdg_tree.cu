// Step A2: tree preprocessing of Algorithm 1 step 1 -- the root distances
// ("dists") and the structure that answers LCA queries (the skip table's
// role), recomputed by every recovery from the tree layout built at init.
//
// Root distances are EXACT: every r(v) = fl(1/w(v, parent v)) is a multiple
// of 2^-S with S = 52 - min_v exponent(r(v)), so D(v) = sum of r on the root
// path is an integer in units of 2^-S, and R_T(u, v) = D(u) + D(v) - 2 D(LCA)
// (Eq. RT) is exact before its single rounding.  Each vertex carries one
// 128-bit word P(v) = D(v) * 2^32 + depth(v); D < 2^96 is checked from the
// exponent range and the maximum depth (PDG_E_RANGE otherwise).
//
// k_tree_sum + k_tree_scan: one prefix sum over the Euler tour.  A down arc
// into v adds word(v) = fixed(r(v)) * 2^32 + 1, an up arc out of v subtracts
// it, so the running sum at v's down arc is P(v).  Integer addition is
// associative: the tiled scan gives the same bits as a sequential walk.  The
// same pass writes, per vertex (preorder label x), the range-minimum key
// val0[x] = depth(x) * 2^32 + parent(x).
//
// k_rmq_levels: the range-minimum structure over val0.  Level j + 1 holds the
// minima of the 32-entry groups of level j, up to a single group.  Inside a
// group, mask[k] has bit i set when entry i (i <= k) has a smaller depth than
// every later entry up to k (a suffix minimum); the minimum depth over [i, k]
// in one group is then found at the lowest set bit of mask[k] at or above i.
// A query (step A3) combines at most two partial groups per level.
#include <algorithm>
#include <climits>

#include "pdg_internal.cuh"

namespace pdg {

namespace {

// word(v) of the edge to the parent: fixed(r(v)) * 2^32 + 1, with
// fixed(r) = mant * 2^(e - 52 + S) and S = 52 - e_min
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

__device__ __forceinline__ u128 shfl_up_u128(u128 x, int d) {
  const uint64_t lo = __shfl_up_sync(0xffffffffu, (unsigned long long)(uint64_t)x, d);
  const uint64_t hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(uint64_t)(x >> 64), d);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 x, int d) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)x, d);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)(x >> 64), d);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 warp_incl_scan_u128(u128 x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const u128 y = shfl_up_u128(x, d);
    if (lane >= d) x += y;
  }
  return x;
}

// The tour is scanned in tiles of 256 threads x 8 arcs, reduce-then-scan:
// k_tree_sum adds each tile's arcs (the last block to finish turns the tile
// sums into exclusive prefixes), k_tree_scan rescans every tile from its
// prefix and writes the vertices.  No tile waits on another (a chained scan
// would have to pass the running prefix through every tile in order).
constexpr int kTsThreads = 256;
constexpr int kTsItems = 8;
constexpr int kTsTile = kTsThreads * kTsItems;

struct TreeScanArgs {
  const int32_t* tour;
  int64_t A;
  const double* rtree;
  const int32_t* parent;
  int dep_bits;
  DevScalars* dsc;
  u128* P;
  uint64_t* val0;
  u128* tsum;     // [tiles] tile sums, then their exclusive prefixes
  uint32_t* done;  // blocks of k_tree_sum finished (the last one resets it)
};

// the tile's arcs of this thread (INT_MIN past the end) and the r of their vertices
__device__ __forceinline__ void load_arcs(const TreeScanArgs& a, int64_t base, int32_t (&arc)[kTsItems],
                                          double (&r)[kTsItems]) {
  if (base + kTsItems <= a.A) {
    const int4* p4 = reinterpret_cast<const int4*>(a.tour + base);
    const int4 x = __ldg(p4), y = __ldg(p4 + 1);
    arc[0] = x.x; arc[1] = x.y; arc[2] = x.z; arc[3] = x.w;
    arc[4] = y.x; arc[5] = y.y; arc[6] = y.z; arc[7] = y.w;
  } else {
#pragma unroll
    for (int i = 0; i < kTsItems; i++) arc[i] = (base + i < a.A) ? __ldg(a.tour + base + i) : INT_MIN;
  }
#pragma unroll
  for (int i = 0; i < kTsItems; i++) {
    const int32_t x = arc[i] >= 0 ? arc[i] : ~arc[i];
    r[i] = (arc[i] != INT_MIN) ? __ldg(a.rtree + x) : 0.0;
  }
}

// +word(x) for the down arc into x, -word(x) for the up arc out of x
__device__ __forceinline__ u128 arc_word(int32_t arc, double r, int e_min, bool range_ok) {
  if (arc == INT_MIN) return 0;
  const u128 w = edge_word(r, e_min, range_ok);
  return arc >= 0 ? w : (u128)0 - w;
}

__device__ __forceinline__ u128 block_sum_u128(u128 x, u128* s_warp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d; d >>= 1) x += shfl_xor_u128(x, d);
  if (lane == 0) s_warp[wid] = x;
  __syncthreads();
  u128 t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_warp[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kTsThreads) k_tree_sum(TreeScanArgs a) {
  __shared__ u128 s_warp[kTsThreads / 32];
  __shared__ int s_last;
  const bool range_ok = range_fits(a.dsc, a.dep_bits);
  const int e_min = a.dsc->e_min;
  const int64_t t = blockIdx.x;
  int32_t arc[kTsItems];
  double r[kTsItems];
  load_arcs(a, t * kTsTile + (int64_t)threadIdx.x * kTsItems, arc, r);
  u128 s = 0;
#pragma unroll
  for (int i = 0; i < kTsItems; i++) s += arc_word(arc[i], r[i], e_min, range_ok);
  const u128 tot = block_sum_u128(s, s_warp);
  if (threadIdx.x == 0) {
    a.tsum[t] = tot;
    __threadfence();
    s_last = (atomicAdd(a.done, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  // the last block: exclusive prefixes of the tile sums, in chunks of one value per thread
  __threadfence();
  const int64_t tiles = gridDim.x;
  u128 run = 0;
  for (int64_t c0 = 0; c0 < tiles; c0 += kTsThreads) {
    const int64_t i = c0 + threadIdx.x;
    u128 v = 0;
    if (i < tiles) {
      const ulonglong2 q = __ldcg(reinterpret_cast<const ulonglong2*>(a.tsum + i));
      v = ((u128)q.y << 64) | q.x;
    }
    const u128 incl = warp_incl_scan_u128(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    u128 before = run;
    for (int w = 0; w < wid; w++) before += s_warp[w];
    u128 chunk = 0;
    for (int w = 0; w < kTsThreads / 32; w++) chunk += s_warp[w];
    if (i < tiles) a.tsum[i] = before + incl - v;
    run += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.done = 0;
}

__global__ void __launch_bounds__(kTsThreads) k_tree_scan(TreeScanArgs a) {
  __shared__ u128 s_warp[kTsThreads / 32];
  const bool range_ok = range_fits(a.dsc, a.dep_bits);
  const int e_min = a.dsc->e_min;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t t = blockIdx.x;
  int32_t arc[kTsItems];
  double r[kTsItems];
  load_arcs(a, t * kTsTile + (int64_t)threadIdx.x * kTsItems, arc, r);
  u128 s = 0;
#pragma unroll
  for (int i = 0; i < kTsItems; i++) s += arc_word(arc[i], r[i], e_min, range_ok);
  const u128 incl = warp_incl_scan_u128(s);
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  const ulonglong2 q = __ldcg(reinterpret_cast<const ulonglong2*>(a.tsum + t));  // the tile's prefix
  u128 p = ((u128)q.y << 64) | q.x;
  for (int w = 0; w < wid; w++) p += s_warp[w];
  p += incl - s;  // prefix of every arc before this thread's first
#pragma unroll
  for (int i = 0; i < kTsItems; i++) {
    if (arc[i] == INT_MIN) continue;
    p += arc_word(arc[i], r[i], e_min, range_ok);
    if (arc[i] >= 0) {  // the down arc into x: P(x) and the range-minimum key
      const int32_t x = arc[i];
      a.P[x] = p;
      a.val0[x] = ((uint64_t)(uint32_t)p << 32) | (uint32_t)__ldg(a.parent + x);
    }
  }
}

// The range-minimum structure in one launch.  Each block takes 8192 entries
// of level 0 (256 groups) and then the 256 group minima it produced (8 groups
// of level 1); the last block to finish builds the remaining, small levels.
// A group's masks come from one thread walking its 32 entries in order with
// a stack of suffix minima kept as a bit set: an entry pops the stacked
// entries whose depth is not below its own, then pushes itself, and the
// stack after entry k is mask[k].  Entries are staged in shared memory with
// a padded row per group, so loads, walks and stores are conflict-free.
constexpr int kRmqThreads = 256;
constexpr int kRmqChunk = kRmqThreads * 32;  // entries per block and pass

struct RmqArgs {
  uint64_t* val[kRmqMaxLevels];
  uint32_t* mask[kRmqMaxLevels];
  uint64_t* pmin[kRmqMaxLevels];
  uint64_t* smin[kRmqMaxLevels];
  int64_t size[kRmqMaxLevels];
  int levels;
  uint32_t* done;  // blocks finished (the last one resets it)
};

// entries [base, base + len) of one level (len <= kRmqChunk, base a multiple
// of 32): their masks, the minima from the group start up to each entry
// (pmin) and from each entry to the group end (smin), and the minimum of
// every group to val_next[entry / 32] when val_next is given.  Both minima
// come from the masks: the lowest set bit of mask[k] is the minimum of
// [0, k], and the first set bit of mask[31] at or above k the minimum of
// [k, 31] (padding past the level's end is deeper than any entry).
// (FROM_PREV: the level was written by an earlier kernel, so its reads may use
// the read-only cache; levels written by this kernel are read from L2)
__device__ __forceinline__ uint64_t rmq_load(const uint64_t* p, bool from_prev) {
  return from_prev ? __ldg(p) : __ldcg(p);
}

__device__ void rmq_chunk(const uint64_t* __restrict__ val, int64_t size, int64_t base, int len,
                          uint32_t* __restrict__ mask, uint64_t* __restrict__ pmin, uint64_t* __restrict__ smin,
                          uint64_t* __restrict__ val_next, uint32_t (*s_d)[33], bool from_prev) {
  const int t = threadIdx.x;
  const int ngroups = (len + 31) / 32;
  for (int i = t; i < ngroups * 32; i += kRmqThreads) {
    const int64_t idx = base + i;
    s_d[i >> 5][i & 31] = (i < len && idx < size) ? (uint32_t)(rmq_load(val + idx, from_prev) >> 32) : 0xffffffffu;
  }
  __syncthreads();
  const bool walk = t < ngroups && base + 32 * t < size;
  uint32_t m[32];
  if (walk) {
    uint32_t stack = 0;
#pragma unroll
    for (int k = 0; k < 32; k++) {
      const uint32_t d = s_d[t][k];
      while (stack) {  // pop the entries whose depth is not below d
        const int top = 31 - __clz(stack);
        if (s_d[t][top] < d) break;
        stack &= ~(1u << top);
      }
      stack |= 1u << k;
      m[k] = stack;
    }
    if (val_next) val_next[(base >> 5) + t] = rmq_load(val + base + 32 * t + (__ffs(stack) - 1), from_prev);
  }
  __syncthreads();  // every walk is done: the rows now take the masks
  if (walk) {
#pragma unroll
    for (int k = 0; k < 32; k++) s_d[t][k] = m[k];
  }
  __syncthreads();
  for (int i = t; i < len; i += kRmqThreads) {
    const int64_t idx = base + i;
    if (idx >= size) continue;
    const int g = i >> 5, k = i & 31;
    const uint32_t mk = s_d[g][k];
    mask[idx] = mk;
    if (pmin) {
      const int64_t g0 = base + 32 * g;
      pmin[idx] = rmq_load(val + g0 + (__ffs(mk) - 1), from_prev);
      smin[idx] = rmq_load(val + g0 + k + (__ffs(s_d[g][31] >> k) - 1), from_prev);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kRmqThreads) k_rmq_build(RmqArgs a) {
  __shared__ uint32_t s_d[kRmqThreads][33];
  __shared__ int s_last;
  const int64_t b0 = (int64_t)blockIdx.x * kRmqChunk;
  rmq_chunk(a.val[0], a.size[0], b0, kRmqChunk, a.mask[0], a.pmin[0], a.smin[0], a.levels > 1 ? a.val[1] : nullptr,
            s_d, true);
  if (a.levels > 1)
    rmq_chunk(a.val[1], a.size[1], b0 / 32, kRmqThreads, a.mask[1], a.pmin[1], a.smin[1],
              a.levels > 2 ? a.val[2] : nullptr, s_d, false);
  if (a.levels <= 2) return;  // uniform
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(a.done, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int j = 2; j < a.levels; j++)
    for (int64_t base = 0; base < a.size[j]; base += kRmqChunk)
      rmq_chunk(a.val[j], a.size[j], base, (int)min((int64_t)kRmqChunk, a.size[j] - base), a.mask[j], a.pmin[j],
                a.smin[j], j + 1 < a.levels ? a.val[j + 1] : nullptr, s_d, false);
  if (threadIdx.x == 0) *a.done = 0;
}

}  // namespace

int step_tree(Handle& h) {
  int dep_bits = 0;
  while ((1ll << dep_bits) <= h.max_depth) dep_bits++;
  if (h.A > 0) {
    const int64_t tiles = (h.A + kTsTile - 1) / kTsTile;
    TreeScanArgs a{h.tour, h.A, h.rtree, h.parent, dep_bits, h.dsc, h.P, h.rmq_val[0], h.ts_sum, h.ts_done};
    ++h.launches;
    k_tree_sum<<<(int)tiles, kTsThreads, 0, h.stream>>>(a);
    ++h.launches;
    k_tree_scan<<<(int)tiles, kTsThreads, 0, h.stream>>>(a);
    PDG_CUDA(cudaGetLastError());
  }
  // the range-minimum structure over val0
  RmqArgs r{};
  for (int j = 0; j < h.rmq_levels; j++) {
    r.val[j] = h.rmq_val[j];
    r.mask[j] = h.rmq_mask[j];
    r.pmin[j] = h.rmq_pmin[j];
    r.smin[j] = h.rmq_smin[j];
    r.size[j] = h.rmq_size[j];
  }
  r.levels = h.rmq_levels;
  r.done = h.ts_done + 1;
  ++h.launches;
  k_rmq_build<<<(int)((h.rmq_size[0] + kRmqChunk - 1) / kRmqChunk), kRmqThreads, 0, h.stream>>>(r);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

// the tree-scan work space for a tour of A arcs (tile sums, two block counters)
int tree_scan_workspace(Handle& h) {
  const int64_t tiles = std::max<int64_t>((h.A + kTsTile - 1) / kTsTile, 1);
  int st;
  if ((st = device_alloc(h, (void**)&h.ts_sum, sizeof(u128) * (size_t)tiles)) ||
      (st = device_alloc(h, (void**)&h.ts_done, sizeof(uint32_t) * 2)))
    return st;
  PDG_CUDA(cudaMemsetAsync(h.ts_done, 0, sizeof(uint32_t) * 2, h.stream));
  return PDG_OK;
}

}  // namespace pdg
