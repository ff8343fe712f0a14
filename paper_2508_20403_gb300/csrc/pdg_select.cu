// Step A4a: select, per graph, a prefix of the global order (score
// descending, id ascending) that is large enough to contain the first k
// recovered edges.
//
// Why a prefix suffices: by Lemma "share LCA" an edge can only be marked by
// an earlier edge of its own subtask, so whether an edge is recovered depends
// only on the edges ranked before it.  Running the greedy on the prefix
// {score >= t} therefore recovers exactly the edges the full pass recovers
// inside that prefix; if at least k of them survive, the first k are the
// answer, otherwise the prefix is enlarged (step A7 reports a retry).
//
// The threshold comes from a two-level radix select on the score bits
// (12 bits: sign + exponent, then the next 12 mantissa bits); every edge of
// the boundary bucket is kept, so the candidate set is always a prefix.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kSelChunkBlocks = 1024;
constexpr int kHistUnroll = 8;  // keys in flight per thread in the histogram passes

__device__ __forceinline__ int64_t sel_chunk(int64_t E, int nb) {
  int64_t c = (E + nb - 1) / nb;
  return (c + kTile - 1) / kTile * kTile;
}

__device__ __forceinline__ void sel_count(uint32_t* h, uint64_t k, int lvl, int32_t b1) {
  if (lvl == 0) atomicAdd(&h[k >> 52], 1u);
  else if ((int32_t)(k >> 52) == b1) atomicAdd(&h[(k >> 40) & 0xfff], 1u);
}

// level 1 (lvl == 0): bins of key >> 52; level 2: bins of (key >> 40) & 0xfff
// restricted to the level-1 bucket of the edge's graph.
__global__ void __launch_bounds__(kBlock) k_sel_hist(const uint64_t* __restrict__ key, int64_t E,
                                                     const int64_t* __restrict__ off_ptr, int32_t G,
                                                     const GraphSel* __restrict__ sel, int lvl,
                                                     uint32_t* __restrict__ hist) {
  dep_sync();
  __shared__ uint32_t sh[kSelBins];
  const int64_t chunk = sel_chunk(E, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(E, b0 + chunk);
  if (b0 >= b1) return;
  const int32_t g0 = (G == 1) ? 0 : part_of(off_ptr, G, b0);
  const int32_t g1 = (G == 1) ? 0 : part_of(off_ptr, G, b1 - 1);
  // one graph at a time: a shared-memory histogram for long ranges, direct
  // global atomics for short ones (many small graphs per chunk)
  for (int32_t g = g0; g <= g1; g++) {
    const int64_t r0 = (G == 1) ? b0 : max(b0, off_ptr[g]);
    const int64_t r1 = (G == 1) ? b1 : min(b1, off_ptr[g + 1]);
    const GraphSel s = sel[g];
    if (s.take_all || r0 >= r1) continue;
    uint32_t* hg = hist + (int64_t)g * kSelBins;
    if (r1 - r0 < 256) {  // too short to amortise clearing and flushing 4096 shared bins
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) sel_count(hg, key[i], lvl, s.b1);
      continue;
    }
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t i0 = r0; i0 < r1; i0 += (int64_t)kBlock * kHistUnroll) {
      uint64_t k[kHistUnroll];
#pragma unroll
      for (int u = 0; u < kHistUnroll; u++) {
        const int64_t i = i0 + u * kBlock + threadIdx.x;
        k[u] = i < r1 ? key[i] : 0;
      }
#pragma unroll
      for (int u = 0; u < kHistUnroll; u++)
        if (i0 + u * kBlock + threadIdx.x < r1) sel_count(sh, k[u], lvl, s.b1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
      if (sh[i]) atomicAdd(&hg[i], sh[i]);
    __syncthreads();
  }
}

// One block per graph: walk the bins from the top until `need` edges are
// covered; clears the histogram for the next level.  Thread t owns the 16
// bins just below the 16 t highest ones.
constexpr int kPickPer = kSelBins / kBlock;
static_assert(kPickPer == 16, "pick layout");

__global__ void __launch_bounds__(kBlock) k_sel_pick(uint32_t* __restrict__ hist, GraphSel* __restrict__ sel,
                                                     const int64_t* __restrict__ off_ptr, int32_t G, int lvl,
                                                     int64_t* __restrict__ count_out, int64_t* __restrict__ cand_ptr) {
  dep_sync();
  __shared__ int64_t sm[kBlock / 32 + 1];
  __shared__ int s_owner;
  const int32_t g = blockIdx.x;
  GraphSel s = sel[g];
  uint32_t* hg = hist + (int64_t)g * kSelBins;
  if (s.take_all) {
    if (lvl == 1 && threadIdx.x == 0) {
      s.count = off_ptr[g + 1] - off_ptr[g];
      s.thresh = 0;
      sel[g] = s;
      count_out[g] = s.count;
      if (G == 1) {  // a single graph's candidate offsets need no scan
        cand_ptr[0] = 0;
        cand_ptr[1] = s.count;
      }
    }
    return;
  }
  const int64_t need = (lvl == 0) ? s.want : s.want - s.above1;
  const int lo = kSelBins - kPickPer * (threadIdx.x + 1);  // lowest bin of this thread
  uint32_t c[kPickPer];
  const uint4* h4 = reinterpret_cast<const uint4*>(hg + lo);
#pragma unroll
  for (int q = 0; q < kPickPer / 4; q++) {
    const uint4 x = h4[q];
    c[4 * q] = x.x;
    c[4 * q + 1] = x.y;
    c[4 * q + 2] = x.z;
    c[4 * q + 3] = x.w;
  }
  int64_t mine = 0;
#pragma unroll
  for (int i = 0; i < kPickPer; i++) mine += c[i];
  int64_t tot;
  const int64_t excl = block_excl_scan(mine, sm, &tot);  // counts of the higher bins
  // owner: the first thread whose inclusive sum reaches need, else the last
  if (threadIdx.x == 0) s_owner = kBlock - 1;
  __syncthreads();
  if (excl < need && excl + mine >= need) s_owner = threadIdx.x;  // at most one thread
  if (threadIdx.x == 0 && need <= 0) s_owner = 0;
  __syncthreads();
  if (threadIdx.x == s_owner) {
    int64_t run = excl;  // edges in the bins above `bin`
    int bin = lo;        // lowest bin of the thread if need is never reached
    uint32_t bin_count = c[0];
    bool found = false;
#pragma unroll
    for (int i = kPickPer - 1; i >= 0; i--) {
      if (found) continue;
      if (run + c[i] >= need) {
        bin = lo + i;
        bin_count = c[i];
        found = true;
      } else {
        run += c[i];
      }
    }
    if (lvl == 0) {
      s.b1 = bin;
      s.above1 = run;
    } else {
      s.b2 = bin;
      s.above2 = run;
      s.count = s.above1 + run + bin_count;
      s.thresh = ((uint64_t)s.b1 << 52) | ((uint64_t)bin << 40);
      count_out[g] = s.count;
      if (G == 1) {
        cand_ptr[0] = 0;
        cand_ptr[1] = s.count;
      }
    }
    sel[g] = s;
  }
  uint4* w4 = reinterpret_cast<uint4*>(hg + lo);
#pragma unroll
  for (int q = 0; q < kPickPer / 4; q++) w4[q] = make_uint4(0u, 0u, 0u, 0u);
}

// Ordered compaction of the selected edges (key >= the graph's threshold), in
// canonical id order: a count pass per block chunk, then a write pass whose
// blocks add up the counts of the blocks before them and place each tile's
// selected edges by a block scan.  Both passes stream the keys with vector
// loads.
template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_sel_compact(const uint64_t* __restrict__ key, int64_t E,
                                                        const int64_t* __restrict__ off_ptr, int32_t G,
                                                        const GraphSel* __restrict__ sel,
                                                        int64_t* __restrict__ bcount, int64_t cap,
                                                        int32_t* __restrict__ cand_idx,
                                                        uint64_t* __restrict__ rkey, int32_t* __restrict__ rval,
                                                        const int64_t* __restrict__ cand_ptr, DevScalars* dsc) {
  dep_sync();
  __shared__ int64_t sm[kBlock / 32 + 1];
  const int64_t chunk = sel_chunk(E, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(E, b0 + chunk);
  int64_t run = 0;
  if (WRITE) {  // this block's offset: the counts of the blocks before it, added up here (no separate scan)
    int64_t c = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += kBlock) c += bcount[i];
    run = block_sum(c, sm);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {  // the last block's end is the total
      const int64_t total = run + bcount[blockIdx.x];
      dsc->n_cand_wanted = total;
      if (total > cap || total != cand_ptr[G]) {
        // nothing downstream may touch more than `cap` candidates: run it empty
        dsc->n_cand = 0;
        atomicOr(&dsc->err, ERR_CAPACITY);
      } else {
        dsc->n_cand = total;
      }
    }
  }
  int64_t tot = 0;
  for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kItems;
    uint32_t pick = 0;
    uint64_t k[kItems];
    if (base < b1) {
      // graph of the first item, then advanced item by item
      int32_t g = (G == 1) ? 0 : part_of(off_ptr, G, base);
      int64_t g_end = (G == 1) ? INT64_MAX : off_ptr[g + 1];
      uint64_t th = sel[g].thresh;
      if (base + kItems <= b1) {
        const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(key + base);
#pragma unroll
        for (int q = 0; q < kItems / 2; q++) {
          const ulonglong2 x = k2[q];
          k[2 * q] = x.x;
          k[2 * q + 1] = x.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < kItems; i++) k[i] = (base + i < b1) ? key[base + i] : 0;
      }
#pragma unroll
      for (int i = 0; i < kItems; i++) {
        const int64_t p = base + i;
        if (p < b1) {
          while (p >= g_end) {
            g++;
            g_end = off_ptr[g + 1];
            th = sel[g].thresh;
          }
          if (k[i] >= th) pick |= 1u << i;
        }
      }
    }
    const int64_t cnt = __popc(pick);
    if (!WRITE) {
      tot += cnt;
      continue;
    }
    int64_t tile_tot;
    int64_t pos = run + block_excl_scan(cnt, sm, &tile_tot);
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      if (pick & (1u << i)) {
        if (pos < cap) {
          cand_idx[pos] = (int32_t)(base + i);
          rkey[pos] = ~k[i];  // ascending ~score = descending score
          rval[pos] = (int32_t)pos;
        }
        pos++;
      }
    }
    run += tile_tot;
  }
  if (!WRITE) {
    tot = block_sum(tot, sm);
    if (threadIdx.x == 0) bcount[blockIdx.x] = tot;
  }
}

}  // namespace

int step_select(Handle& h) {
  const int64_t E = h.E_off;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kSelChunkBlocks, (E + kTile - 1) / kTile));
  bool any_select = false;
  for (int32_t g = 0; g < h.G; g++)
    if (h.want_h[g] < h.off_ptr_h[g + 1] - h.off_ptr_h[g]) any_select = true;
  for (int lvl = 0; lvl < 2; lvl++) {
    if (any_select && !(lvl == 0 && h.fuse_hist)) {
      ++h.launches;
      launch_k(h, k_sel_hist, nb, kBlock, 0, h.key, E, h.d_off_ptr, h.G, h.sel, lvl, h.hist);
    }
    ++h.launches;
    launch_k(h, k_sel_pick, h.G, kBlock, 0, h.hist, h.sel, h.d_off_ptr, h.G, lvl, h.d_graph_tmp, h.d_cand_ptr);
  }
  PDG_CUDA(cudaGetLastError());
  int st;
  if (h.G > 1 && (st = scan_excl_i64(h, h.d_graph_tmp, h.d_cand_ptr, h.G, nullptr, h.G))) return st;
  int64_t* bcount = h.blk_a;
  ++h.launches;
  launch_k(h, k_sel_compact<false>, nb, kBlock, 0, h.key, E, h.d_off_ptr, h.G, h.sel, bcount, 0, nullptr, nullptr,
           nullptr, h.d_cand_ptr, h.dsc);
  ++h.launches;
  launch_k(h, k_sel_compact<true>, nb, kBlock, 0, h.key, E, h.d_off_ptr, h.G, h.sel, bcount, h.Rcap, h.cand_idx,
           h.rk[0], h.rv[0], h.d_cand_ptr, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
