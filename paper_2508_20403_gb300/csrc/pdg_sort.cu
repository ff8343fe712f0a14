// Step A4b: order the candidates and form the subtasks (Algorithm 1 steps 2-3).
//
//   1. Stable LSD radix sort by the descending score (8-bit digits of the
//      complemented FP64 bits).  Candidates arrive in canonical id order, so
//      equal scores stay in ascending id order: this is the global order of
//      Algorithm 1 step 2.  In a batch, further passes on the graph index
//      keep each graph's candidates contiguous.  Position = rank.
//   2. Stable LSD radix sort of the ranks by LCA: every subtask (all
//      candidates sharing an LCA, Lemma "share LCA") becomes a contiguous
//      segment whose members stay in rank order (Algorithm 1 step 3: the
//      index-linked lists per LCA, here a segment CSR).
//
// One-sweep LSD: one kernel histograms every digit position of a key set at
// once, one kernel scans those histograms (and fixes which ping-pong buffer
// each pass reads), and each pass is then a single scatter kernel.  Its blocks take tiles in order from an atomic counter,
// rank the tile's digits stably (ballot peer masks + per-warp counters), publish the
// tile's digit counts and obtain the counts of all earlier tiles by looking
// back through published values ("decoupled look-back"), a window of tiles
// per memory round trip.  Every wait on an
// earlier tile is bounded (spin_limit); a timeout sets an error bit and the
// recovery reports PDG_E_TIMEOUT instead of hanging.  A digit shared by all
// keys is detected from the histogram and its pass moves nothing.  Sizes are
// read on the device, so the sequence can be captured in a CUDA graph.
#include <algorithm>
#include <mutex>

#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kRdxBins = 256;
// Scatter tiles are 512 threads x 6 keys = 3072 keys and the look-back reads
// 8 tiles per round trip: at the candidate counts of a recovery (10^5 .. 10^7
// keys) a pass is a chain of dependent steps rather than a stream, and these
// sizes gave the shortest passes on the 3 x 10^5-key mesh 128^3 sort among
// 2048..8192-key tiles and 4..32-tile windows (fewer tiles shorten the
// look-back chain; more keys per thread lengthen the ranking).
// The keys per thread are a template parameter (4, 6 or 8: 2048, 3072 or
// 4096-key tiles) that the sort_tile_keys option, and so the autotuner, picks.
constexpr int kOsThreads = 512;
constexpr int kOsItemsDefault = 6;
constexpr int kRdxWarps = kOsThreads / 32;
constexpr int kMaxDigits = 8;
constexpr int kLookWin = 8;  // look-back words fetched per round trip
constexpr uint32_t kFlagA = 1u << 30;  // tile aggregate published
constexpr uint32_t kFlagP = 2u << 30;  // inclusive prefix published
constexpr uint32_t kCountMask = (1u << 30) - 1;


// Histograms of `ndig` digit positions (starting at bit `shift0`) of the keys
// in the current buffer: ghist[d][bin].
__global__ void __launch_bounds__(kBlock) k_os_hist(const uint64_t* k0, const uint64_t* k1, const DevScalars* dsc,
                                                    int shift0, int ndig, uint32_t* __restrict__ ghist) {
  dep_sync();
  __shared__ uint32_t sh[kMaxDigits][kRdxBins];
  const int64_t N = dsc->n_cand;
  const uint64_t* keys = dsc->radix_sel ? k1 : k0;
  for (int i = threadIdx.x; i < kMaxDigits * kRdxBins; i += kBlock) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i] >> shift0;
    for (int d = 0; d < ndig; d++) atomicAdd(&sh[d][(k >> (8 * d)) & 0xff], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ndig * kRdxBins; i += kBlock) {
    const uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// Exclusive scan of each digit's 256 bins (one warp per digit) and the
// uniform-digit test; also clears the histogram for the next key set.  The
// passes' ping-pong buffer choices follow from the skips, so they are fixed
// here (sel[d]: the buffer pass d reads) together with the final choice.
__global__ void k_os_scan(uint32_t* __restrict__ ghist, int ndig, DevScalars* dsc, uint32_t* __restrict__ goff,
                          int32_t* __restrict__ skip, int32_t* __restrict__ sel) {
  dep_sync();
  __shared__ int32_t s_skip[kMaxDigits];
  const int lane = threadIdx.x & 31, d = threadIdx.x >> 5;  // launched with 32 * ndig threads
  const uint32_t N = (uint32_t)dsc->n_cand;
  uint32_t v[8], s = 0;
  for (int i = 0; i < 8; i++) {
    v[i] = ghist[d * kRdxBins + lane * 8 + i];
    s += v[i];
  }
  const uint32_t incl = warp_incl_scan(s);
  uint32_t run = incl - s;
  bool uniform = false;
  for (int i = 0; i < 8; i++) {
    goff[d * kRdxBins + lane * 8 + i] = run;
    run += v[i];
    if (v[i] == N) uniform = true;
    ghist[d * kRdxBins + lane * 8 + i] = 0;
  }
  uniform = __any_sync(0xffffffffu, uniform) || N == 0;
  if (lane == 0) {
    skip[d] = uniform ? 1 : 0;
    s_skip[d] = uniform ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cur = dsc->radix_sel;
    for (int q = 0; q < ndig; q++) {
      sel[q] = cur;
      if (!s_skip[q]) cur ^= 1;
    }
    dsc->radix_sel = cur;
  }
}

// Dynamic shared memory of one scatter block: the tile's keys and values
// bucketed by digit, the per-warp digit counters and the per-digit offsets.
constexpr size_t os_smem_bytes(int items) {
  return (size_t)kOsThreads * items * (sizeof(uint64_t) + sizeof(int32_t)) +
         sizeof(uint32_t) * ((size_t)kRdxWarps * kRdxBins + 2 * kRdxBins + 32);
}

template <int kOsItems>
__global__ void __launch_bounds__(kOsThreads, 1) k_os_scatter(const uint64_t* k0, const uint64_t* k1, const int32_t* v0,
                                                       const int32_t* v1, uint64_t* ko0, uint64_t* ko1, int32_t* vo0,
                                                       int32_t* vo1, DevScalars* dsc, int shift,
                                                       const uint32_t* __restrict__ goff, const int32_t* skip,
                                                       const int32_t* selp, uint32_t* status, uint32_t* counters,
                                                       int64_t spin_limit) {
  dep_sync();
  constexpr int kOsTile = kOsThreads * kOsItems;
  constexpr int kRdxPerWarp = kOsTile / kRdxWarps;  // kOsItems rounds of 32
  extern __shared__ __align__(16) unsigned char os_smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(os_smem);                        // [kOsTile]
  int32_t* sval = reinterpret_cast<int32_t*>(skey + kOsTile);                   // [kOsTile]
  uint32_t(*wcnt)[kRdxBins] = reinterpret_cast<uint32_t(*)[kRdxBins]>(sval + kOsTile);  // [warps][256]
  uint32_t* s_loff = &wcnt[kRdxWarps][0];  // tile-local start of each digit's bucket
  uint32_t* s_base = s_loff + kRdxBins;    // output position of bucket slot 0, per digit
  uint32_t* s_wsum = s_base + kRdxBins;    // per-warp totals of the digit scan
  __shared__ int64_t s_tile;
  const int64_t N = dsc->n_cand;
  const int sel = *selp;
  if (!*skip) {
    const uint64_t* keys = sel ? k1 : k0;
    const int32_t* vals = sel ? v1 : v0;
    uint64_t* ko = sel ? ko0 : ko1;
    int32_t* vo = sel ? vo0 : vo1;
    const int64_t T = (N + kOsTile - 1) / kOsTile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(&counters[0], 1u);  // tiles in launch order
    __syncthreads();
    const int64_t t = s_tile;
    if (t < T) {  // uniform over the block
      const int64_t t0 = t * kOsTile;
      const int tile_n = (int)(N - t0 < kOsTile ? N - t0 : kOsTile);
      for (int d = lane; d < kRdxBins; d += 32) wcnt[w][d] = 0;
      __syncwarp();
      uint64_t kk[kOsItems];
      int32_t vv[kOsItems];
      uint32_t rnk[kOsItems];
      const int64_t base = t0 + (int64_t)w * kRdxPerWarp;
      // all loads first (independent, in flight together), then the ranking
#pragma unroll
      for (int i = 0; i < kOsItems; i++) {
        const int64_t idx = base + i * 32 + lane;
        kk[i] = idx < N ? __ldcg(keys + idx) : 0;  // written by other blocks: bypass L1
        vv[i] = idx < N ? __ldcg(vals + idx) : 0;
      }
#pragma unroll
      for (int i = 0; i < kOsItems; i++) {
        const bool valid = base + i * 32 + lane < N;
        const int dig = (int)((kk[i] >> shift) & 0xff);
        // lanes holding the same digit: one ballot per digit bit
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; b++) {
          const bool bit = (dig >> b) & 1;
          const unsigned bb = __ballot_sync(0xffffffffu, bit);
          peers &= bit ? bb : ~bb;
        }
        rnk[i] = valid ? wcnt[w][dig] + __popc(peers & lt) : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[w][dig] += __popc(peers);
        __syncwarp();
      }
      __syncthreads();
      // thread d < 256: the tile's count of digit d (published at once), the
      // per-warp offsets inside the digit, and the scan over digits
      const int d = threadIdx.x;
      uint32_t run = 0, incl = 0;
      volatile uint32_t* st = status;
      if (d < kRdxBins) {
        for (int ww = 0; ww < kRdxWarps; ww++) {
          const uint32_t c = wcnt[ww][d];
          wcnt[ww][d] = run;
          run += c;
        }
        st[t * kRdxBins + d] = (t == 0 ? kFlagP : kFlagA) | run;
        incl = warp_incl_scan(run);
        if (lane == 31) s_wsum[w] = incl;
      }
      __syncthreads();
      if (d < kRdxBins) {
        uint32_t before = 0;
        for (int ww = 0; ww < w; ww++) before += s_wsum[ww];
        s_loff[d] = before + incl - run;
      }
      __syncthreads();
      // bucket the tile by digit in shared memory (stable: warp order, then rank)
#pragma unroll
      for (int i = 0; i < kOsItems; i++) {
        if (base + i * 32 + lane < N) {
          const int dig = (int)((kk[i] >> shift) & 0xff);
          const uint32_t lp = s_loff[dig] + wcnt[w][dig] + rnk[i];
          skey[lp] = kk[i];
          sval[lp] = vv[i];
        }
      }
      // look back kLookWin tiles per round trip: the window's words are
      // loaded together, then consumed newest first until a prefix
      if (d < kRdxBins) {
        uint32_t excl = 0;
        if (t > 0) {
          bool done = false;
          for (int64_t j0 = t - 1; j0 >= 0 && !done; j0 -= kLookWin) {
            uint32_t win[kLookWin];
#pragma unroll
            for (int q = 0; q < kLookWin; q++) win[q] = (j0 - q >= 0) ? st[(j0 - q) * kRdxBins + d] : 0u;
#pragma unroll
            for (int q = 0; q < kLookWin; q++) {
              const int64_t j = j0 - q;
              if (!done && j >= 0) {
                uint32_t v = win[q];
                int64_t spins = 0;
                while ((v & ~kCountMask) == 0 && spins < spin_limit) {
                  v = st[j * kRdxBins + d];
                  spins++;
                }
                if ((v & ~kCountMask) == 0) {  // an earlier tile never published: give up, report
                  atomicOr(&dsc->err, ERR_TIMEOUT);
                  done = true;
                } else {
                  excl += v & kCountMask;
                  if (v & kFlagP) done = true;
                }
              }
            }
          }
          __threadfence();
          st[t * kRdxBins + d] = kFlagP | (excl + run);
        }
        s_base[d] = goff[d] + excl - s_loff[d];  // modulo 2^32; the sums below are < N
      }
      __syncthreads();
      // consecutive threads write consecutive slots of each digit's run
      for (int j = threadIdx.x; j < tile_n; j += kOsThreads) {
        const uint64_t k = skey[j];
        const uint32_t pos = s_base[(k >> shift) & 0xff] + (uint32_t)j;
        if (pos < (uint64_t)N) {
          ko[pos] = k;
          vo[pos] = sval[j];
        }
      }
    }
  }
}

}  // namespace

int sort_setup() {
  PDG_CUDA(cudaFuncSetAttribute(k_os_scatter<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem_bytes(4)));
  PDG_CUDA(cudaFuncSetAttribute(k_os_scatter<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem_bytes(6)));
  PDG_CUDA(cudaFuncSetAttribute(k_os_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)os_smem_bytes(8)));
  return PDG_OK;
}

namespace {

// keys := graph index of the candidate held as value (keeps graphs contiguous)
__global__ void k_key_graph(uint64_t* __restrict__ k0, uint64_t* __restrict__ k1, const int32_t* __restrict__ v0,
                            const int32_t* __restrict__ v1, const int64_t* __restrict__ cand_ptr, int32_t G,
                            DevScalars* dsc) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t N = dsc->n_cand;
  uint64_t* k = dsc->radix_sel ? k1 : k0;
  const int32_t* v = dsc->radix_sel ? v1 : v0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    k[i] = (uint64_t)part_of(cand_ptr, G, v[i]);
}

// rank_cand[r] = candidate at rank r; then keys := LCA, values := rank
__global__ void k_key_lca(uint64_t* __restrict__ k0, uint64_t* __restrict__ k1, int32_t* __restrict__ v0,
                          int32_t* __restrict__ v1, const int32_t* __restrict__ cand_idx,
                          const int32_t* __restrict__ lca, int32_t* __restrict__ rank_cand, DevScalars* dsc) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t N = dsc->n_cand;
  uint64_t* k = dsc->radix_sel ? k1 : k0;
  int32_t* v = dsc->radix_sel ? v1 : v0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = v[i];
    rank_cand[i] = c;
    k[i] = (uint64_t)lca[cand_idx[c]];
    v[i] = (int32_t)i;
  }
}

__global__ void k_copy_vals(const int32_t* __restrict__ v0, const int32_t* __restrict__ v1, int32_t* __restrict__ out,
                            DevScalars* dsc) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t N = dsc->n_cand;
  const int32_t* v = dsc->radix_sel ? v1 : v0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v[i];
}

}  // namespace

// keys per thread of the scatter tiles (option sort_tile_keys = 2048, 3072 or 4096)
static int sort_items(const Handle& h) {
  switch (h.opt.sort_tile_keys) {
    case 2048: return 4;
    case 4096: return 8;
    default: return kOsItemsDefault;
  }
}

static int64_t sort_tiles(const Handle& h) {
  const int64_t tile = (int64_t)kOsThreads * sort_items(h);
  return (h.Rcap + tile - 1) / tile;
}

// Sort the current key buffer by `ndig` 8-bit digits starting at bit shift0;
// `pass0` indexes this key set's passes in the status / skip / counter arrays.
static int onesweep(Handle& h, int shift0, int ndig, int pass0) {
  if (ndig <= 0) return PDG_OK;  // a single possible key value: already sorted
  const int grid_hist = h.num_sms * 2;
  const int64_t tiles_max = sort_tiles(h);
  const int items = sort_items(h);
  uint32_t* ghist = h.radix_hist;                // [8][256], kept zero between uses
  uint32_t* goff = h.radix_hist + 8 * kRdxBins;  // [8][256]
  int32_t* skip = reinterpret_cast<int32_t*>(h.radix_hist + 16 * kRdxBins) + pass0;
  int32_t* sel = reinterpret_cast<int32_t*>(h.radix_hist + 16 * kRdxBins) + kRadixPassesMax + pass0;
  ++h.launches;
  launch_k(h, k_os_hist, grid_hist, kBlock, 0, h.rk[0], h.rk[1], h.dsc, shift0, ndig, ghist);
  ++h.launches;
  launch_k(h, k_os_scan, 1, 32 * ndig, 0, ghist, ndig, h.dsc, goff, skip, sel);
  for (int d = 0; d < ndig; d++) {
    const int p = pass0 + d;
    uint32_t* status = h.radix_status + (int64_t)p * tiles_max * kRdxBins;
    uint32_t* counters = h.radix_counters + 2 * p;
    ++h.launches;
    const int grid = (int)std::max<int64_t>(tiles_max, 1);
#define PDG_OS_SCATTER(I)                                                                                    \
  launch_k(h, k_os_scatter<I>, grid, kOsThreads, os_smem_bytes(I), h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.rk[0], \
           h.rk[1], h.rv[0], h.rv[1], h.dsc, shift0 + 8 * d, goff + d * kRdxBins, skip + d, sel + d, status,   \
           counters, h.opt.spin_limit)
    if (items == 4) PDG_OS_SCATTER(4);
    else if (items == 8) PDG_OS_SCATTER(8);
    else PDG_OS_SCATTER(6);
#undef PDG_OS_SCATTER
  }
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

namespace {

// ---------------------------------------------------------------- one launch
//
// When every tile of the candidate keys fits in one co-resident block, the
// whole of step A4b runs as ONE cooperative kernel: all passes of all three
// key sets (score, graph index in a batch, LCA), the re-keying between them
// and the final copy, with grid-wide barriers between the phases of a pass
// instead of kernel boundaries and look-back chains.  A pass:
//   rank   each block ranks its tile by the digit (stable: warp ballots and
//          per-warp counters) and publishes the tile's 256 digit counts;
//   scan   block b turns column b of the (tile x digit) count matrix into
//          exclusive prefixes over the tiles;
//   place  each block writes its keys to digit base + tile prefix + rank.
// Digit bases and uniform (skipped) digits come from histograms of each key
// set taken at its start.  Barriers count arrivals on one word (zeroed before
// the launch); a wait that runs out sets ERR_TIMEOUT and the block goes on,
// so the recovery reports the error instead of hanging.
constexpr int kCoThreads = 512;
constexpr int kCoItems = 6;
constexpr int kCoTile = kCoThreads * kCoItems;
constexpr int kCoWarps = kCoThreads / 32;
constexpr int kCoKeySets = 3;

struct CoopSortArgs {
  uint64_t* k[2];
  int32_t* v[2];
  DevScalars* dsc;
  const int32_t* cand_idx;
  const int32_t* lca;
  int32_t* rank_cand;
  int32_t* lsort_rank;
  const int64_t* cand_ptr;
  int32_t G;
  int nd_graph, nd_lca;
  uint32_t* counts;  // [tiles][256]
  uint32_t* totals;  // [kCoKeySets][kMaxDigits][256], zero at launch
  uint32_t* bar;     // barrier arrivals, zero at launch
  int64_t spin_limit;
};

struct CoopSmem {
  uint64_t key[kCoTile];
  int32_t val[kCoTile];
  uint32_t wcnt[kCoWarps][kRdxBins];
  uint32_t loff[kRdxBins];
  uint32_t base[kRdxBins];
  uint32_t wsum[32];
  uint32_t bases[kMaxDigits][kRdxBins];  // exclusive digit bases of the current key set
  int32_t uniform[kMaxDigits];
};

// Thread 0 of each block announces the block's arrival with a release
// reduction (the block's writes, ordered before it by __syncthreads, become
// visible with it) and polls the count with acquire loads: no full fence and
// no returned atomic on the path.  The wait is bounded (spin_limit).
__device__ __forceinline__ void coop_barrier(const CoopSortArgs& a, uint32_t& target) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bar) : "memory");
    uint32_t v;
    int64_t spins = 0;
    do {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a.bar) : "memory");
    } while (v < target && ++spins < a.spin_limit);
    if (v < target) atomicOr(&a.dsc->err, ERR_TIMEOUT);
  }
  __syncthreads();
}

// one key set: histograms, then one rank / scan / place pass per non-uniform digit
__device__ __forceinline__ void coop_keyset(const CoopSortArgs& a, CoopSmem& sm, int ks, int ndig, int& cur,
                                            uint32_t& target,
                            int64_t N, int64_t tiles) {
  const int64_t t = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t t0 = t * kCoTile;
  uint32_t* tot = a.totals + (int64_t)ks * kMaxDigits * kRdxBins;
  // histograms of every digit of the key set (the order of the keys does not matter)
  for (int i = threadIdx.x; i < ndig * kRdxBins; i += kCoThreads) (&sm.wcnt[0][0])[i] = 0;
  __syncthreads();
  if (t < tiles) {
    const uint64_t* keys = a.k[cur];
    for (int64_t i = t0 + threadIdx.x; i < N && i < t0 + kCoTile; i += kCoThreads) {
      const uint64_t kk = __ldcg(keys + i);
      for (int d = 0; d < ndig; d++) atomicAdd(&(&sm.wcnt[0][0])[d * kRdxBins + ((kk >> (8 * d)) & 0xff)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ndig * kRdxBins; i += kCoThreads) {
      const uint32_t c = (&sm.wcnt[0][0])[i];
      if (c) atomicAdd(&tot[i], c);
    }
  }
  coop_barrier(a, target);
  // digit bases (exclusive scans of the histograms) and uniform digits, in every block
  for (int d = w; d < ndig; d += kCoWarps) {
    uint32_t v[8], sum = 0;
    bool uni = false;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      v[i] = __ldcg(&tot[d * kRdxBins + lane * 8 + i]);
      sum += v[i];
      if (v[i] == (uint32_t)N) uni = true;
    }
    const uint32_t incl = warp_incl_scan(sum);
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      sm.bases[d][lane * 8 + i] = run;
      run += v[i];
    }
    uni = __any_sync(0xffffffffu, uni) || N == 0;
    if (lane == 0) sm.uniform[d] = uni ? 1 : 0;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1;
  for (int d = 0; d < ndig; d++) {
    if (sm.uniform[d]) continue;  // uniform over the grid: every block read the same totals
    const int shift = 8 * d;
    const uint64_t* keys = a.k[cur];
    const int32_t* vals = a.v[cur];
    uint64_t kk[kCoItems];
    int32_t vv[kCoItems];
    uint32_t rnk[kCoItems];
    const int64_t base = t0 + (int64_t)w * (kCoTile / kCoWarps);
    int tile_n = 0;
    // rank: stable order inside the tile, digit counts of the tile
    if (t < tiles) {
      tile_n = (int)(N - t0 < kCoTile ? N - t0 : kCoTile);
      for (int dd = lane; dd < kRdxBins; dd += 32) sm.wcnt[w][dd] = 0;
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kCoItems; i++) {
        const int64_t idx = base + i * 32 + lane;
        kk[i] = idx < N ? __ldcg(keys + idx) : 0;  // written by other blocks: bypass L1
        vv[i] = idx < N ? __ldcg(vals + idx) : 0;
      }
#pragma unroll
      for (int i = 0; i < kCoItems; i++) {
        const bool valid = base + i * 32 + lane < N;
        const int dig = (int)((kk[i] >> shift) & 0xff);
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; b++) {
          const bool bit = (dig >> b) & 1;
          const unsigned bb = __ballot_sync(0xffffffffu, bit);
          peers &= bit ? bb : ~bb;
        }
        rnk[i] = valid ? sm.wcnt[w][dig] + __popc(peers & lt) : 0;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) sm.wcnt[w][dig] += __popc(peers);
        __syncwarp();
      }
      __syncthreads();
      const int dg = threadIdx.x;
      if (dg < kRdxBins) {
        uint32_t run = 0;
        for (int ww = 0; ww < kCoWarps; ww++) {
          const uint32_t c = sm.wcnt[ww][dg];
          sm.wcnt[ww][dg] = run;
          run += c;
        }
        a.counts[t * kRdxBins + dg] = run;
        const uint32_t incl = warp_incl_scan(run);
        if (lane == 31) sm.wsum[w] = incl;
        sm.base[dg] = run;  // the tile's count, kept for the local offsets below
      }
      __syncthreads();
      if (dg < kRdxBins) {
        uint32_t before = 0;
        for (int ww = 0; ww < w; ww++) before += sm.wsum[ww];
        const uint32_t incl = warp_incl_scan(sm.base[dg]);
        sm.loff[dg] = before + incl - sm.base[dg];
      }
      __syncthreads();
      // bucket the tile by digit in shared memory (stable: warp order, then rank)
#pragma unroll
      for (int i = 0; i < kCoItems; i++) {
        if (base + i * 32 + lane < N) {
          const int dig = (int)((kk[i] >> shift) & 0xff);
          const uint32_t lp = sm.loff[dig] + sm.wcnt[w][dig] + rnk[i];
          sm.key[lp] = kk[i];
          sm.val[lp] = vv[i];
        }
      }
    }
    coop_barrier(a, target);
    // the tile's prefix per digit: counts of the earlier tiles, summed by every block for itself.  The
    // 256 counts of a tile are one 1 KB row: 64 threads read a row (16 bytes each), the eight row
    // groups take every eighth earlier tile, then add up in shared memory.
    if (t < tiles) {
      const int q = threadIdx.x & 63, rg = threadIdx.x >> 6;
      // sixteen rows in flight per thread: the rows of up to 128 earlier tiles in one round of loads
      // (the block is alone on its SM, so the registers are there)
      constexpr int kRows = 16;
      uint4 acc = make_uint4(0, 0, 0, 0);
      for (int64_t r0 = rg; r0 < t; r0 += 8 * kRows) {
        uint4 x[kRows];
#pragma unroll
        for (int u = 0; u < kRows; u++) {
          const int64_t r = r0 + 8 * u;
          x[u] = r < t ? __ldcg(reinterpret_cast<const uint4*>(a.counts + r * kRdxBins) + q) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kRows; u++) {
          acc.x += x[u].x;
          acc.y += x[u].y;
          acc.z += x[u].z;
          acc.w += x[u].w;
        }
      }
      reinterpret_cast<uint4*>(&sm.wcnt[rg][0])[q] = acc;  // the per-warp counters are free after bucketing
      __syncthreads();
      const int dg = threadIdx.x;
      if (dg < kRdxBins) {
        uint32_t before = 0;
#pragma unroll
        for (int g = 0; g < kCoThreads / 64; g++) before += sm.wcnt[g][dg];
        sm.base[dg] = sm.bases[d][dg] + before - sm.loff[dg];
      }
      __syncthreads();
    }
    // place: consecutive threads write consecutive slots of each digit's run
    if (t < tiles) {
      uint64_t* ko = a.k[cur ^ 1];
      int32_t* vo = a.v[cur ^ 1];
      for (int j = threadIdx.x; j < tile_n; j += kCoThreads) {
        const uint64_t k = sm.key[j];
        const uint32_t pos = sm.base[(k >> shift) & 0xff] + (uint32_t)j;
        if (pos < (uint64_t)N) {
          ko[pos] = k;
          vo[pos] = sm.val[j];
        }
      }
    }
    cur ^= 1;
    coop_barrier(a, target);
  }
}

__global__ void __launch_bounds__(kCoThreads) k_sort_coop(CoopSortArgs a) {
  dep_sync();
  extern __shared__ __align__(16) unsigned char co_smem[];
  CoopSmem& sm = *reinterpret_cast<CoopSmem*>(co_smem);
  if (attempt_aborted(a.dsc)) return;  // the attempt is void (uniform over the grid: set before the launch)
  const int64_t N = a.dsc->n_cand;
  const int64_t tiles = (N + kCoTile - 1) / kCoTile;
  if (tiles > gridDim.x) {  // cannot happen: the host launches this path only when the capacity fits
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.dsc->err, ERR_CAPACITY);
    return;
  }
  const int64_t t0 = (int64_t)blockIdx.x * kCoTile;
  uint32_t target = 0;
  int cur = a.dsc->radix_sel;
  // 1. score descending (ties keep ascending id order)
  coop_keyset(a, sm, 0, 8, cur, target, N, tiles);
  // 2. in a batch, the graph index of each candidate (keeps graphs contiguous)
  if (a.G > 1) {
    if (blockIdx.x < tiles)
      for (int64_t i = t0 + threadIdx.x; i < N && i < t0 + kCoTile; i += kCoThreads)
        a.k[cur][i] = (uint64_t)part_of(a.cand_ptr, a.G, __ldcg(a.v[cur] + i));
    __syncthreads();
    coop_keyset(a, sm, 1, a.nd_graph, cur, target, N, tiles);
  }
  // 3. rank_cand[r] = candidate at rank r; keys := LCA, values := rank; group by LCA
  if (blockIdx.x < tiles)
    for (int64_t i = t0 + threadIdx.x; i < N && i < t0 + kCoTile; i += kCoThreads) {
      const int32_t c = __ldcg(a.v[cur] + i);
      a.rank_cand[i] = c;
      a.k[cur][i] = (uint64_t)a.lca[a.cand_idx[c]];
      a.v[cur][i] = (int32_t)i;
    }
  __syncthreads();
  coop_keyset(a, sm, 2, a.nd_lca, cur, target, N, tiles);
  if (blockIdx.x < tiles)
    for (int64_t i = t0 + threadIdx.x; i < N && i < t0 + kCoTile; i += kCoThreads)
      a.lsort_rank[i] = __ldcg(a.v[cur] + i);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.dsc->radix_sel = cur;
}

}  // namespace

// blocks of the one-launch sort that fit on the device at once (0: not available)
static int coop_sort_grid() {
  static int grid = -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (grid >= 0) return grid;
  grid = 0;
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return grid;
  }
  if (cudaFuncSetAttribute(k_sort_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CoopSmem)) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_coop, kCoThreads, sizeof(CoopSmem)) !=
          cudaSuccess) {
    cudaGetLastError();
    return grid;
  }
  grid = std::min(per_sm * sms, kCoThreads);  // the scan phase gives one thread to each tile
  return grid;
}

static int step_sort_coop(Handle& h, int grid_max) {
  // one block per tile of the candidate capacity: fewer arrivals per barrier than a full device
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid_max, (h.Rcap + kCoTile - 1) / kCoTile));
  // barrier word and the key-set histograms start at zero
  PDG_CUDA(cudaMemsetAsync(h.radix_counters, 0, sizeof(uint32_t) * 2 * kRadixPassesMax, h.stream));
  uint32_t* totals = h.radix_hist + kRadixHistOnesweep;  // beside the words the per-pass path keeps zero
  PDG_CUDA(cudaMemsetAsync(totals, 0, sizeof(uint32_t) * kCoKeySets * kMaxDigits * kRdxBins, h.stream));
  stream_op(h);
  CoopSortArgs a{};
  a.k[0] = h.rk[0];
  a.k[1] = h.rk[1];
  a.v[0] = h.rv[0];
  a.v[1] = h.rv[1];
  a.dsc = h.dsc;
  a.cand_idx = h.cand_idx;
  a.lca = h.lca;
  a.rank_cand = h.rank_cand;
  a.lsort_rank = h.lsort_rank;
  a.cand_ptr = h.d_cand_ptr;
  a.G = h.G;
  a.nd_graph = 0;
  while ((1ll << (8 * a.nd_graph)) < h.G) a.nd_graph++;
  a.nd_lca = 0;
  while ((1ll << (8 * a.nd_lca)) < h.n) a.nd_lca++;
  a.counts = h.radix_status;
  a.totals = totals;
  a.bar = h.radix_counters;
  a.spin_limit = h.opt.spin_limit;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kCoThreads);
  cfg.dynamicSmemBytes = sizeof(CoopSmem);
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++h.launches;
  PDG_CUDA(cudaLaunchKernelEx(&cfg, k_sort_coop, a));  // an ordinary (cooperative) launch
  h.dep_ok = true;  // it begins with dep_sync(): the next kernel may depend on it programmatically
  return PDG_OK;
}

int step_sort(Handle& h) {
  // one cooperative launch when every tile of the candidate capacity has its own resident block
  const int cgrid = h.opt.sort_one_launch ? coop_sort_grid() : 0;
  if (cgrid > 0 && (h.Rcap + kCoTile - 1) / kCoTile <= cgrid &&
      kRadixHistOnesweep + (int64_t)kCoKeySets * kMaxDigits * kRdxBins <= kRadixHistWords &&
      (int64_t)cgrid * kRdxBins <= (int64_t)kRadixPassesMax * 256 * ((h.Rcap + kTile - 1) / kTile))
    return step_sort_coop(h, cgrid);
  const int grid = h.num_sms * 4;
  const int64_t tiles_max = sort_tiles(h);
  // look-back status and tile counters start clean for every pass
  PDG_CUDA(cudaMemsetAsync(h.radix_status, 0, sizeof(uint32_t) * (size_t)kRadixPassesMax * tiles_max * kRdxBins,
                           h.stream));
  PDG_CUDA(cudaMemsetAsync(h.radix_counters, 0, sizeof(uint32_t) * 2 * kRadixPassesMax, h.stream));
  stream_op(h);
  int st;
  int pass = 0;
  // 1. score descending (ties keep ascending id order)
  if ((st = onesweep(h, 0, 8, pass))) return st;
  pass += 8;
  if (h.G > 1) {
    ++h.launches;
    launch_k(h, k_key_graph, grid, kBlock, 0, h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.d_cand_ptr, h.G, h.dsc);
    int nd = 0;
    while ((1ll << (8 * nd)) < h.G) nd++;
    if ((st = onesweep(h, 0, nd, pass))) return st;
    pass += nd;
  }
  // 2. group ranks by LCA
  ++h.launches;
  launch_k(h, k_key_lca, grid, kBlock, 0, h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.cand_idx, h.lca, h.rank_cand, h.dsc);
  int nd = 0;
  while ((1ll << (8 * nd)) < h.n) nd++;
  if ((st = onesweep(h, 0, nd, pass))) return st;
  ++h.launches;
  launch_k(h, k_copy_vals, grid, kBlock, 0, h.rv[0], h.rv[1], h.lsort_rank, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
