// Internal declarations of the GB300 off-tree edge-recovery library.
// Kernels live in one .cu file per step of Algorithm 1; this header carries
// the device helpers they share and the handle layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pdgrass.h"

namespace pdg {

typedef unsigned __int128 u128;

constexpr int kBlock = 256;         // threads per block for streaming kernels
constexpr int kItems = 8;           // items per thread in blocked tiles
constexpr int kTile = kBlock * kItems;
constexpr int kSelBins = 4096;      // 12-bit digits of the candidate selection
constexpr int kRadixPassesMax = 16; // 8 score digits + <= 4 graph digits + <= 4 LCA digits
// Block tier: one block per subtask of warp_tier_max+1 .. block_tier_max
// candidates, its markers in a shared-memory table of at most kBlockTierSlots
// pair slots (12 bytes each); a subtask of S candidates needs 2 (c+1)^2 S.
constexpr int kBlockTierSlots = 16384;
constexpr int kBlockTierMax = 896;      // <= kBlockTierSlots / (2 * 9)
constexpr int kBlockTierDefault = 0;  // off: on the mesh and R-MAT workloads the cooperative tier is faster
constexpr int kRadixHistOnesweep = 16 * 256 + 2 * kRadixPassesMax;  // per-pass sort: histograms, skip flags, buffers
constexpr int kRadixHistWords = kRadixHistOnesweep + 3 * 8 * 256;     // + the one-launch sort's key-set histograms
constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kRmqMaxLevels = 6;  // levels of the range-minimum structure (n < 2^30: 30 / 5)
constexpr int kRmqStMax = 6144;   // level-2 entries up to which levels 2+ are one sparse table (n <= 6.29M)

// error bits raised by validation kernels (mapped to a status on the host)
enum : int {
  ERR_NOT_CSR = 1,
  ERR_BAD_WEIGHT = 2,
  ERR_NOT_SYMMETRIC = 4,
  ERR_NOT_A_TREE = 8,
  ERR_CROSS_GRAPH = 16,
  ERR_RANGE = 32,
  ERR_TIMEOUT = 64,
  ERR_CAPACITY = 128,
  ERR_TABLE = 256,
  ERR_BOUNDS = 512,  // a saved index was out of range (checked and skipped; bounds_site says where)
};

// candidate state in the cooperative tier
enum : uint8_t { ST_UNDECIDED = 0, ST_ACCEPTED = 1, ST_REJECTED = 2, ST_ACCEPTED_NEW = 3 };

// per-graph outcome of the budget cut
enum : int32_t { G_OK = 0, G_UNDER = 1, G_RETRY = 2 };

// Scalars that kernels produce and the host reads back in one copy.
// Errors that invalidate the current attempt: the host discards it (and
// retries with larger tables where that helps).  Kernels that index with
// data produced earlier in the attempt return at once when one is set, so an
// attempt cut short never reads half-built structures.
constexpr int kAbortErr = ERR_TABLE | ERR_TIMEOUT | ERR_BOUNDS;

struct DevScalars {
  int32_t err;          // ERR_* bits
  int32_t e_min;        // min / max binary exponent of r = 1/w over tree edges
  int32_t e_max;
  int32_t rounds_used;  // cooperative-tier rounds
  int64_t n_cand;       // candidates selected (all graphs)
  int64_t n_seg;        // subtasks among the candidates
  int64_t n_warp_seg;   // subtasks handled by the warp tier
  int64_t n_block_seg;  // subtasks handled by the block tier
  int64_t n_block;      // candidates in the block tier
  unsigned long long block_ticket;  // block tier: next subtask to take
  int64_t n_big;        // candidates in the cooperative tier
  int64_t n_big_seg;    // subtasks in the cooperative tier
  int64_t max_seg;      // largest subtask
  int64_t big_regs;     // registrations the cooperative tier will make
  int64_t undecided;    // cooperative tier: still undecided after a round
  int64_t active;       // validation: vertices whose pointer jump is not done
  int64_t max_depth;
  int32_t radix_sel;    // radix sort: which ping-pong buffer holds the keys
  int32_t radix_skip;   // radix sort: the current digit is uniform
  int64_t radix_len;    // radix sort: histogram length (256 * tiles)
  int64_t n_warp_cand;  // candidates in the warp tier
  int64_t n_cand_wanted;  // candidates the selection produced (may exceed capacity)
  int64_t n_constrained;  // cooperative tier: candidates with a possible earlier marker
  int64_t n_big_chunk;    // cooperative tier: chunks of at most kBigChunk positions
  unsigned long long score_ticket;  // step A3: next tile of off-tree edges to score
  uint32_t epoch;       // attempts so far (tags the cooperative tier's undecided entries)
  int32_t bounds_site;  // first failed bounds check (see ERR_BOUNDS)
  int32_t bounds_where;  // its round (99: serial finisher)
  int64_t bounds_pos, bounds_val;  // its position and offending value
  int64_t finish_left;  // cooperative tier: candidates the rounds left to the serial finisher
};

// Programmatic dependent launch.  A kernel started by launch_k may be put on
// the SMs as the kernel before it on the stream drains (its blocks exiting),
// before that grid's completion has been signalled; every kernel of the
// recovery calls dep_sync() first, before it touches device memory:
// griddepcontrol.wait returns once the previous kernel has completed and its
// writes are visible (at once when the launch was an ordinary one).  No kernel
// releases its successor earlier than its own exit (launch_dependents): blocks
// placed early, while the previous grid still ran, made recoveries slower.
__device__ __forceinline__ void dep_sync() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// (set by earlier kernels of the stream, so a plain load sees it)
__device__ __forceinline__ bool attempt_aborted(const DevScalars* d) { return (d->err & kAbortErr) != 0; }

// Cooperative tier: pair table slot (16 bytes; all-ones = empty) and exact
// entry (16 bytes; 16 per flagged pair, indexed j * 4 + j').
struct PairSlot {
  unsigned long long key;  // (z1 << 32) | z2
  uint32_t minr;           // smallest rank that registered the pair
  uint32_t xidx;           // block of exact entries, or all-ones
};
struct ExactEnt {
  uint32_t acc;            // smallest accepted rank
  uint32_t pad;
  unsigned long long und;  // round tag (high 32) | smallest undecided rank
};

// Per-graph selection state (candidate prefix of the global order).
struct GraphSel {
  int64_t want;     // requested prefix size R0_g
  int64_t above1;   // edges strictly above the level-1 bucket
  int64_t above2;   // edges of the level-1 bucket strictly above the level-2 bucket
  int64_t count;    // selected candidates
  uint64_t thresh;  // selected = key >= thresh
  int32_t b1, b2;
  int32_t take_all;
  int32_t pad;
};

// What a captured recovery graph depends on besides the pinned parameters it
// reads at replay time (budgets, prefix sizes, output offsets).
struct GraphKey {
  int c = -1, score_mode = -1, any_select = -1, rounds = -1;
  int64_t Rcap = -1, table_cap = -1, xcap = -1;
  void* out_ids = nullptr;
  void* out_scores = nullptr;
  int64_t out_total = -1;
  bool operator==(const GraphKey& o) const {
    return c == o.c && score_mode == o.score_mode && any_select == o.any_select && rounds == o.rounds && Rcap == o.Rcap &&
           table_cap == o.table_cap && xcap == o.xcap && out_ids == o.out_ids && out_scores == o.out_scores &&
           out_total == o.out_total;
  }
};

struct Handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  pdg_options opt;
  int num_sms = 0;

  // sizes
  int64_t n = 0, nnz = 0, m = 0, E_off = 0, max_depth = 0;
  int32_t G = 1;
  std::vector<int64_t> vtx_ptr_h, edge_ptr_h, off_ptr_h;  // G+1 each

  // resident graph
  int64_t* row_ptr = nullptr;  // input CSR: resident during init only
  int32_t* col = nullptr;
  double* w = nullptr;
  // canonical edge list in id order, resident; after the tree layout its
  // endpoints are preorder labels, el_u < el_v
  int32_t* el_u = nullptr;
  int32_t* el_v = nullptr;
  double* el_w = nullptr;
  int32_t* parent = nullptr;  // in preorder labels once the tree layout is built
  // tree layout (sparsify_init): Euler tour (A arcs: label entered, or ~label
  // left), the caller's vertex id of every preorder label
  int32_t* tour = nullptr;
  int64_t A = 0;
  int32_t* vtx_of_pre = nullptr;
  int64_t* d_vtx_ptr = nullptr;
  int64_t* d_edge_ptr = nullptr;
  int64_t* d_off_ptr = nullptr;

  // step 1 outputs
  int32_t* off_u = nullptr;
  int32_t* off_v = nullptr;
  int32_t* off_id = nullptr;
  double* off_w = nullptr;
  double* rtree = nullptr;  // r(v) = fl(1/w(v, parent v))
  int64_t* blk_a = nullptr; // per-block counters (classification, scans)
  int64_t* cls_off = nullptr;  // write offsets of the classification's block chunks (counted at init)
  int64_t* blk_b = nullptr;
  int nblk = 0;

  // tree: P(x) = D(x) * 2^32 + depth(x); D = exact root distance in units of 2^-S
  u128* P = nullptr;
  // range-minimum structure over val0[x] = depth(x) * 2^32 + parent(x):
  // level j + 1 holds the minima of the 32-entry groups of level j
  int rmq_levels = 0;
  int64_t rmq_size[kRmqMaxLevels] = {0};
  uint64_t* rmq_val[kRmqMaxLevels] = {nullptr};
  uint32_t* rmq_mask[kRmqMaxLevels] = {nullptr};
  uint64_t* rmq_pmin[kRmqMaxLevels] = {nullptr};  // per entry: minimum from its group's start (null: top level)
  uint64_t* rmq_smin[kRmqMaxLevels] = {nullptr};  // per entry: minimum to its group's end
  uint64_t* rmq_st = nullptr;  // sparse table over level 2 (row t: minima of 2^t entries; row 0 is level 2)
  int rmq_st_rows = 0;
  u128* ts_sum = nullptr;        // tree scan: tile sums
  uint32_t* ts_done = nullptr;   // range-minimum build: blocks finished

  // scores
  uint64_t* key = nullptr;  // FP64 score bits (positive -> order preserving)
  int32_t* lca = nullptr;   // preorder label of the LCA

  // selection
  uint32_t* hist = nullptr;  // G * kSelBins
  bool fuse_hist = false;    // this attempt's first histogram level comes from step A3
  GraphSel* sel = nullptr;   // G
  std::vector<int64_t> want_h;  // requested prefix per graph
  // prefix that sufficed per graph in the last call, for the budget k_mem and
  // (c_mem, score mode mode_mem): a later call with the same parameters starts
  // there (any prefix holding the first k recovered edges gives the same set)
  std::vector<int64_t> want_mem, k_mem;
  int c_mem = -1, mode_mem = -1;
  // cooperative-tier rounds a later recovery with (c_mem, mode_mem) launches:
  // the rounds the last one ran, one more if it left candidates to the serial
  // finisher (which completes whatever a short round count leaves, so any
  // count is exact; -1: no recovery yet)
  int rounds_mem = -1;
  int64_t* d_cand_ptr = nullptr;  // G+1
  int64_t* d_graph_tmp = nullptr;  // G+1 scratch

  // candidate buffers (grow-only, capacity Rcap)
  int64_t Rcap = 0;
  int32_t* cand_idx = nullptr;     // off-tree index of each candidate (id order within graph)
  uint64_t* rk[2] = {nullptr, nullptr};  // radix keys ping-pong
  int32_t* rv[2] = {nullptr, nullptr};   // radix values ping-pong
  int32_t* rank_cand = nullptr;    // rank -> candidate index
  int32_t* lsort_rank = nullptr;   // position in (lca, rank) order -> rank
  int64_t* scan_tmp = nullptr;     // Rcap + 1
  uint32_t* radix_hist = nullptr;      // [8][256] histograms, [8][256] offsets, skip flags, buffer choices
  uint32_t* radix_status = nullptr;    // look-back words: kRadixPassesMax * tiles * 256
  uint32_t* radix_counters = nullptr;  // per pass: tile ticket (and one spare word)
  uint64_t* scan_status = nullptr;     // single-pass scan: flag | value per tile, zero between scans
  uint32_t* scan_ctr = nullptr;        // single-pass scan: tile ticket, blocks finished
  int64_t scan_tiles_cap = 0;
  uint32_t* radix_dtot = nullptr;      // 256
  // records in (lca, rank) order
  int32_t* rec_u = nullptr;
  int32_t* rec_v = nullptr;
  int32_t* rec_anc = nullptr;  // 2 * PDG_MAX_C arrays of Rcap
  int32_t* rec_du = nullptr;
  int32_t* rec_dv = nullptr;
  int32_t* rec_rank = nullptr;
  int32_t* rec_lca = nullptr;
  uint8_t* rec_b = nullptr;
  uint8_t* state = nullptr;      // cooperative tier state per position
  uint8_t* acc_flag = nullptr;   // accepted, by rank
  int32_t* seg_begin = nullptr;  // Rcap + 1
  int32_t* warp_seg = nullptr;   // subtasks of the warp tier
  int32_t* block_seg = nullptr;  // subtasks of the block tier
  int32_t* big_pos = nullptr;    // positions of the cooperative tier
  int32_t* big_seg = nullptr;    // subtasks of the cooperative tier
  int64_t* big_chunk = nullptr;  // (subtask index << 32) | first position offset, one per chunk
  int32_t* pos_x = nullptr;      // per position: index of its cooperative subtask
  int64_t* seg_regs = nullptr;   // per cooperative subtask: pair registrations
  int64_t* seg_pref = nullptr;   // their exclusive prefix (R + 1)
  // cooperative tier: pair table, exact entries, per-position probe masks and slots
  int64_t table_cap = 0;
  int64_t xcap = 0;
  PairSlot* ptab = nullptr;
  ExactEnt* xtab = nullptr;
  unsigned long long* xund1 = nullptr;  // odd rounds' undecided ranks, one per exact entry
  uint32_t epochs = 0;                  // attempts since the epoch last restarted (host count)
  uint32_t* pmask = nullptr;
  int32_t* reg_slot = nullptr;
  int32_t* pslot = nullptr;
  uint32_t* flagbits = nullptr;  // one bit per pair slot: the pair was flagged (has an exact block)
  int32_t* und_list = nullptr;    // positions left undecided by phase A

  // budget
  int32_t* gstat = nullptr;      // G
  int64_t* gcount = nullptr;     // G
  int64_t* d_k = nullptr;        // G
  int64_t* d_out_ptr = nullptr;  // G+1
  int32_t* out_ids = nullptr;    // library-owned output staging
  double* out_scores = nullptr;
  int64_t out_cap = 0;

  DevScalars* dsc = nullptr;   // device
  DevScalars* hsc = nullptr;   // pinned host mirror
  int64_t stats[12] = {0};
  int64_t launches = 0;  // kernels launched by the current recovery
  // CUDA-graph replay of a whole recovery (opt.use_graph)
  cudaStream_t gstream = nullptr;  // private stream: capture and replay
  cudaEvent_t ev_order = nullptr;  // orders gstream after the caller's stream
  cudaStream_t sstream = nullptr;  // side stream: the warp/block tiers beside the cooperative tier
  // launch_k launches programmatic dependents only inside a recovery (dep_armed)
  // and only after a kernel it launched itself (dep_ok; cleared by stream_op)
  bool dep_armed = false;
  bool dep_ok = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  GraphKey gkey;
  int64_t glaunches = 0;
  float timings[8] = {0};
  cudaEvent_t ev[16] = {};
  size_t device_bytes = 0;
  std::vector<void*> allocs;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ int64_t row_of(const int64_t* __restrict__ row_ptr, int64_t n, int64_t p) {
  // largest u with row_ptr[u] <= p
  int64_t lo = 0, hi = n;  // row_ptr[lo] <= p < row_ptr[hi] (row_ptr[n] = nnz > p)
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid) <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// index of the first entry >= x in a sorted int32 range, or end
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// graph owning position p of a contiguous partition ptr[0..G]
__device__ __forceinline__ int32_t part_of(const int64_t* __restrict__ ptr, int32_t G, int64_t p) {
  int32_t lo = 0, hi = G;
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (ptr[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 31;
  x *= 0x7fb5d329728ea185ull;
  x ^= x >> 27;
  x *= 0x81dadef4bc2dd44dull;
  x ^= x >> 33;
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive block scan (blockDim.x == kBlock); returns the exclusive prefix,
// *total receives the block sum.  smem must hold kBlock/32 + 1 values.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* smem, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = warp_incl_scan(x);
  if (lane == 31) smem[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = (lane < kBlock / 32) ? smem[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < kBlock / 32) smem[lane] = si - s;
    if (lane == kBlock / 32 - 1) smem[kBlock / 32] = si;
  }
  __syncthreads();
  T res = smem[wid] + inc - x;
  *total = smem[kBlock / 32];
  __syncthreads();
  return res;
}

// The same for blocks of NT threads (NT a multiple of 32, at most 1024);
// smem must hold NT/32 + 1 values.
template <int NT, typename T>
__device__ __forceinline__ T block_excl_scan_n(T x, T* smem, T* total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = warp_incl_scan(x);
  if (lane == 31) smem[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = (lane < NW) ? smem[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < NW) smem[lane] = si - s;
    if (lane == NW - 1) smem[NW] = si;
  }
  __syncthreads();
  T res = smem[wid] + inc - x;
  *total = smem[NW];
  __syncthreads();
  return res;
}

// Tiles of the single-pass (look-back) kernels: 1024 threads x kItems.
constexpr int kLbThreads = 1024;
constexpr int kLbTile = kLbThreads * kItems;

template <typename T>
__device__ __forceinline__ T block_sum(T x, T* smem) {
  T tot;
  block_excl_scan(x, smem, &tot);
  return tot;
}

// Decoupled look-back of a single-pass tile scan (executed by one full warp).
// status[t] holds kStA | tile sum once tile t is scanned and kStP | inclusive
// prefix once its prefix is known (0 before).  Publishes tile t's sum,
// collects the exclusive prefix of tile t -- lane l reads tile j0 - l, so 32
// earlier tiles per memory round trip -- and publishes the inclusive prefix.
// Every wait is bounded by spin_limit; *timed_out reports a wait that ran out.
constexpr uint64_t kStA = 1ull << 62;          // tile sum published
constexpr uint64_t kStP = 2ull << 62;          // inclusive prefix published
constexpr uint64_t kStVal = (1ull << 62) - 1;  // value bits

__device__ __forceinline__ int64_t warp_lookback(uint64_t* status, int64_t t, int64_t tot, int64_t spin_limit,
                                                 bool* timed_out) {
  const int lane = threadIdx.x & 31;
  volatile uint64_t* st = status;
  if (lane == 0) st[t] = (t == 0 ? kStP : kStA) | (uint64_t)tot;
  int64_t excl = 0;
  bool out = false;
  for (int64_t j0 = t - 1; j0 >= 0;) {
    // tiles before the first count as a zero prefix
    const int64_t j = j0 - lane;
    uint64_t w = (j >= 0) ? (uint64_t)st[j] : (uint64_t)kStP;
    int64_t spins = 0;
    while ((w >> 62) == 0 && spins < spin_limit) {
      w = st[j];
      spins++;
    }
    if (__any_sync(0xffffffffu, (w >> 62) == 0)) {  // an earlier tile never published
      out = true;
      break;
    }
    const unsigned pmask = __ballot_sync(0xffffffffu, (w & kStP) != 0);
    const int first = pmask ? __ffs(pmask) - 1 : 32;  // nearest inclusive prefix
    int64_t val = (lane <= first) ? (int64_t)(w & kStVal) : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    excl += val;
    if (first < 32) break;
    j0 -= 32;
  }
  if (lane == 0 && t > 0) st[t] = kStP | (uint64_t)(excl + tot);
  *timed_out = out;
  return excl;
}

// ---------------------------------------------------------------- host side

int check_cuda(cudaError_t e);
#define PDG_CUDA(call)                            \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return check_cuda(e_); \
  } while (0)

int grid_for(const Handle& h, int64_t work, int per_block = kBlock);

// Launches kernel k (which begins with dep_sync()) on the handle's stream:
// inside a recovery as a programmatic dependent of the kernel before it when
// that one was launched by launch_k as well, else as an ordinary launch.
// Errors as for <<<>>>: the launch status is also left for cudaGetLastError.
template <typename... P, typename... A>
inline cudaError_t launch_k(Handle& h, void (*k)(P...), dim3 grid, dim3 block, size_t smem, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = (h.dep_armed && h.dep_ok) ? 1 : 0;
  h.dep_ok = true;
  return cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

// After a copy, a fill, an event record or an event wait on the handle's
// stream: the next kernel waits for it in full.
inline void stream_op(Handle& h) { h.dep_ok = false; }

// Arms launch_k for the duration of one recovery.
struct DepScope {
  Handle& h;
  explicit DepScope(Handle& hh) : h(hh) {
    h.dep_armed = true;
    h.dep_ok = false;
  }
  ~DepScope() {
    h.dep_armed = false;
    h.dep_ok = false;
  }
};

// device-wide exclusive scan: out[i] = sum in[0..i), out[N] = total.
// N may live on the device (n_dev != nullptr) or be given on the host.
int ensure_scan_status(Handle& h, int64_t n_max);  // scans of up to n_max elements can run
int scan_excl_i64(Handle& h, const int64_t* in, int64_t* out, int64_t n_host, const int64_t* n_dev, int64_t n_max);
int scan_excl_i32(Handle& h, const int32_t* in, int64_t* out, int64_t n_host, const int64_t* n_dev, int64_t n_max);
int scan_excl_u32(Handle& h, const uint32_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max);
int scan_excl_u8(Handle& h, const uint8_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max);

// steps
int validate_graph(Handle& h, bool acyclic);    // input checks; acyclic: also acyclicity, max depth, range
int build_edge_list(Handle& h);                 // init: canonical edge list from the CSR
int build_tree_layout(Handle& h);               // init: preorder labels, Euler tour, relabelled edges and parents
int tree_scan_workspace(Handle& h);             // init: look-back space of the tree scan
int classify_layout(Handle& h);                 // init: off-tree edges per classification chunk
int step_classify(Handle& h);                   // A1
int step_tree(Handle& h);                       // A2
int step_score(Handle& h, int score_mode);      // A3
int step_select(Handle& h);                     // A4a: candidate prefix per graph
int sort_setup();                               // per-device kernel attributes of the sort
int accept_setup();                             // per-device kernel attributes of the block tier
int coop_rounds(const Handle& h, int c);        // cooperative-tier rounds the next recovery launches
int validate_csr(Handle& h);                    // CSR shape, symmetry and weights only
int spanning_tree(Handle& h, int tree_kind, int32_t* parent);  // parent array of the generated tree (device)
constexpr int64_t kPcgMaxEdges = 8192;  // recovered edges of the PCG quality measure (dense k x k capacitance)
// device ids and b; host results (hist: nullable, the relative residual after each iteration;
// z0: nullable, the preconditioner applied to the centred right-hand side, n values)
int pcg_quality(Handle& h, const int32_t* ids, int64_t k, const double* b, double tol, int32_t max_iter,
                int32_t* iters, double* relres, double* hist = nullptr, double* z0 = nullptr);
int step_sort(Handle& h);                       // A4b: (graph, score desc, id asc) then (lca, rank)
int step_accept(Handle& h, int c);              // A5 + A6
int step_budget(Handle& h, int32_t* out_ids, double* out_scores);  // A7
int ensure_candidates(Handle& h, int64_t R, int c);
int grow_tables(Handle& h, int64_t slots, int64_t xblocks);
int device_alloc(Handle& h, void** p, size_t bytes);

}  // namespace pdg
