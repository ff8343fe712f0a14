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
// k_rmq_build: the range-minimum structure over val0.  Level j + 1 holds the
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
// k_tree_sum adds each tile's arcs, k_tree_scan adds up the sums of the
// tiles before its own (every block for itself: a few loads per thread,
// no serial pass over the tiles) and rescans its tile from that prefix,
// writing the vertices.  No tile waits on another (a chained scan would
// have to pass the running prefix through every tile in order).
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
  u128* tsum;  // [tiles] tile sums
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
  dep_sync();
  __shared__ u128 s_warp[kTsThreads / 32];
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
  if (threadIdx.x == 0) a.tsum[t] = tot;
}

__global__ void __launch_bounds__(kTsThreads, 4) k_tree_scan(TreeScanArgs a) {
  dep_sync();
  __shared__ u128 s_warp[kTsThreads / 32];
  __shared__ u128 s_pre[kTsThreads / 32];
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
  // the tile's prefix: the sums of all earlier tiles, added up by this block itself (loads four deep)
  u128 pre[4] = {0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < t; i += 4 * kTsThreads) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int64_t j = i + (int64_t)k * kTsThreads;
      if (j < t) {
        const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2*>(a.tsum + j));
        pre[k] += ((u128)q.y << 64) | q.x;
      }
    }
  }
  u128 p = block_sum_u128(pre[0] + pre[1] + pre[2] + pre[3], s_pre);
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
// A group's masks are the stacks of suffix minima, as a bit set, that a walk
// over its 32 entries would hold: entry k pops the stacked entries whose
// depth is not below its own, then pushes itself, and the stack after entry
// k is mask[k] (built without the walk, see rmq_chunk).
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
  uint64_t* st;    // level 2 and up as one sparse table (null: as levels)
  int st_rows;
};

// entries [base, base + len) of one level (len <= kRmqChunk, base a multiple
// of 32): their masks, the minima from the group start up to each entry
// (pmin) and from each entry to the group end (smin), and the minimum of
// every group to val_next[entry / 32] when val_next is given.
// The chunk is staged in shared memory by coalesced loads; then one thread
// takes one group into registers and builds it without a data-dependent
// step: the stack after entry k keeps the earlier stack entries shallower
// than entry k, so mask[k] = (mask[k-1] & {j < k : depth j < depth k}) | bit k,
// where the set is 31 comparisons of registers; pmin and smin are running
// minima of the 64-bit keys (a minimum-depth entry of the range; ties carry
// the same parent inside any query range).  Padding past the level's end is
// deeper than any entry.
// (FROM_PREV: the level was written by an earlier kernel, so its reads may use
// the read-only cache; levels written by this kernel are read from L2)
__device__ __forceinline__ uint64_t rmq_load(const uint64_t* p, bool from_prev) {
  return from_prev ? __ldg(p) : __ldcg(p);
}

struct RmqSmem {
  uint64_t v[kRmqChunk / 32][33];  // values, a padded row per group (then the minima being written out)
  uint32_t m[kRmqChunk / 32][33];  // masks
};

__device__ void rmq_chunk(const uint64_t* __restrict__ val, int64_t size, int64_t base, int len,
                          uint32_t* __restrict__ mask, uint64_t* __restrict__ pmin, uint64_t* __restrict__ smin,
                          uint64_t* __restrict__ val_next, RmqSmem& sm, bool from_prev) {
  constexpr int kPer = kRmqChunk / kRmqThreads;
  const int t = threadIdx.x;
  const int ngroups = (len + 31) / 32;
  {
    uint64_t x[kPer];  // a thread's loads are independent and in flight together
#pragma unroll
    for (int i = 0; i < kPer; i++) {
      const int li = i * kRmqThreads + t;
      const int64_t idx = base + li;
      x[i] = (li < ngroups * 32 && li < len && idx < size) ? rmq_load(val + idx, from_prev) : ~0ull;
    }
#pragma unroll
    for (int i = 0; i < kPer; i++) {
      const int li = i * kRmqThreads + t;
      if (li < ngroups * 32) sm.v[li >> 5][li & 31] = x[i];
    }
  }
  __syncthreads();
  uint64_t v[32];
  const bool own = t < ngroups;
  if (own) {
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = sm.v[t][k];
    uint32_t mk = 0;
#pragma unroll
    for (int k = 0; k < 32; k++) {
      const uint32_t dk = (uint32_t)(v[k] >> 32);
      uint32_t shallower = 0;
#pragma unroll
      for (int j = 0; j < k; j++) shallower |= ((uint32_t)(v[j] >> 32) < dk ? 1u : 0u) << j;
      mk = (mk & shallower) | (1u << k);
      sm.m[t][k] = mk;
    }
    uint64_t pm = ~0ull;
#pragma unroll
    for (int k = 0; k < 32; k++) {
      pm = min(pm, v[k]);
      sm.v[t][k] = pm;  // only this thread reads its row
    }
    if (val_next && base + 32 * t < size) val_next[(base >> 5) + t] = pm;
    uint64_t sf = ~0ull;
#pragma unroll
    for (int k = 31; k >= 0; k--) {
      sf = min(sf, v[k]);
      v[k] = sf;
    }
  }
  __syncthreads();
  for (int i = t; i < len; i += kRmqThreads) {
    const int64_t idx = base + i;
    if (idx >= size) break;  // idx grows with i
    mask[idx] = sm.m[i >> 5][i & 31];
    if (pmin) pmin[idx] = sm.v[i >> 5][i & 31];
  }
  if (pmin) {  // uniform
    __syncthreads();
    if (own) {
#pragma unroll
      for (int k = 0; k < 32; k++) sm.v[t][k] = v[k];
    }
    __syncthreads();
    for (int i = t; i < len; i += kRmqThreads) {
      const int64_t idx = base + i;
      if (idx >= size) break;
      smin[idx] = sm.v[i >> 5][i & 31];
    }
  }
  __syncthreads();
}

// Level 2 and up as a sparse table: row t holds the minimum of the 2^t entries from each position, so any range
// [lo, hi] of level 2 is the smaller of two entries of row floor(log2(hi - lo + 1)).  Row 0 is level 2 itself
// (written by the blocks as their level-1 group minima); each further row comes from the one before, kept in
// shared memory (two rows of at most kRmqStMax entries), and is stored as it is made.
__device__ void rmq_sparse_table(const RmqArgs& a, uint64_t* buf) {
  const int64_t n2 = a.size[2];
  uint64_t* cur = buf;
  uint64_t* nxt = buf + kRmqStMax;
  for (int64_t i = threadIdx.x; i < n2; i += kRmqThreads) cur[i] = __ldcg(a.st + i);
  __syncthreads();
  for (int r = 1; r < a.st_rows; r++) {
    const int64_t h = 1ll << (r - 1);
    uint64_t* row = a.st + (int64_t)r * n2;
    for (int64_t i = threadIdx.x; i + 2 * h <= n2; i += kRmqThreads) {
      const uint64_t x = min(cur[i], cur[i + h]);
      nxt[i] = x;
      row[i] = x;
    }
    __syncthreads();
    uint64_t* t = cur;
    cur = nxt;
    nxt = t;
  }
}

__global__ void __launch_bounds__(kRmqThreads, 2) k_rmq_build(RmqArgs a) {
  dep_sync();
  extern __shared__ __align__(16) unsigned char rmq_smem[];
  RmqSmem& sm = *reinterpret_cast<RmqSmem*>(rmq_smem);
  __shared__ int s_last;
  const int64_t b0 = (int64_t)blockIdx.x * kRmqChunk;
  // the chunks this block builds, in order (one call site keeps the register budget of one chunk):
  // its 8192 entries of level 0, their 256 minima on level 1, and for the last block every chunk of level 2 up
  int j = 0;
  int64_t base = b0;
  int len = kRmqChunk;
  bool tail = false;
  for (;;) {
    rmq_chunk(a.val[j], a.size[j], base, len, a.mask[j], a.pmin[j], a.smin[j],
              j + 1 < a.levels ? a.val[j + 1] : nullptr, sm, j == 0);
    if (!tail) {
      if (j == 0 && a.levels > 1) {
        j = 1;
        base = b0 / 32;
        len = kRmqThreads;
        continue;
      }
      if (a.levels <= 2) return;  // uniform
      if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(a.done, 1u) == gridDim.x - 1) ? 1 : 0;
      }
      __syncthreads();
      if (!s_last) return;
      __threadfence();
      if (a.st) {  // uniform: the sparse table over level 2, two rows at a time in shared memory
        rmq_sparse_table(a, reinterpret_cast<uint64_t*>(&sm));
        break;
      }
      tail = true;
      j = 2;
      base = 0;
    } else {
      base += kRmqChunk;
      if (base >= a.size[j]) {
        if (++j >= a.levels) break;
        base = 0;
      }
    }
    len = (int)min((int64_t)kRmqChunk, a.size[j] - base);
  }
  if (threadIdx.x == 0) *a.done = 0;
}

}  // namespace

// the range-minimum build's shared memory, granted once per process (first asked at init, outside any
// stream capture; thread-safe initialisation)
static cudaError_t rmq_smem_attr() {
  static const cudaError_t e =
      cudaFuncSetAttribute(k_rmq_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RmqSmem));
  return e;
}

int step_tree(Handle& h) {
  int dep_bits = 0;
  while ((1ll << dep_bits) <= h.max_depth) dep_bits++;
  if (h.A > 0) {
    const int64_t tiles = (h.A + kTsTile - 1) / kTsTile;
    TreeScanArgs a{h.tour, h.A, h.rtree, h.parent, dep_bits, h.dsc, h.P, h.rmq_val[0], h.ts_sum};
    ++h.launches;
    launch_k(h, k_tree_sum, (int)tiles, kTsThreads, 0, a);
    ++h.launches;
    launch_k(h, k_tree_scan, (int)tiles, kTsThreads, 0, a);
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
  r.st = h.rmq_st;
  r.st_rows = h.rmq_st_rows;
  r.done = h.ts_done;
  PDG_CUDA(rmq_smem_attr());
  ++h.launches;
  launch_k(h, k_rmq_build, (int)((h.rmq_size[0] + kRmqChunk - 1) / kRmqChunk), kRmqThreads, sizeof(RmqSmem), r);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

// the tree-scan work space for a tour of A arcs (tile sums) and the range-minimum build's block counter
int tree_scan_workspace(Handle& h) {
  PDG_CUDA(rmq_smem_attr());
  const int64_t tiles = std::max<int64_t>((h.A + kTsTile - 1) / kTsTile, 1);
  int st;
  if ((st = device_alloc(h, (void**)&h.ts_sum, sizeof(u128) * (size_t)tiles)) ||
      (st = device_alloc(h, (void**)&h.ts_done, sizeof(uint32_t))))
    return st;
  PDG_CUDA(cudaMemsetAsync(h.ts_done, 0, sizeof(uint32_t), h.stream));
  return PDG_OK;
}

}  // namespace pdg
