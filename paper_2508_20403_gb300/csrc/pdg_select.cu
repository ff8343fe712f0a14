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

__device__ __forceinline__ int64_t sel_chunk(int64_t E, int nb) {
  int64_t c = (E + nb - 1) / nb;
  return (c + kTile - 1) / kTile * kTile;
}

// level 1 (lvl == 0): bins of key >> 52; level 2: bins of (key >> 40) & 0xfff
// restricted to the level-1 bucket of the edge's graph.
__global__ void __launch_bounds__(kBlock) k_sel_hist(const uint64_t* __restrict__ key, int64_t E,
                                                     const int64_t* __restrict__ off_ptr, int32_t G,
                                                     const GraphSel* __restrict__ sel, int lvl,
                                                     uint32_t* __restrict__ hist) {
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
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const uint64_t k = key[i];
        if (lvl == 0) atomicAdd(&hg[k >> 52], 1u);
        else if ((int32_t)(k >> 52) == s.b1) atomicAdd(&hg[(k >> 40) & 0xfff], 1u);
      }
      continue;
    }
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const uint64_t k = key[i];
      if (lvl == 0) atomicAdd(&sh[k >> 52], 1u);
      else if ((int32_t)(k >> 52) == s.b1) atomicAdd(&sh[(k >> 40) & 0xfff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
      if (sh[i]) atomicAdd(&hg[i], sh[i]);
    __syncthreads();
  }
}

// One warp per graph: walk the bins from the top until `need` edges are
// covered; clears the histogram for the next level.
__global__ void k_sel_pick(uint32_t* __restrict__ hist, GraphSel* __restrict__ sel, const int64_t* __restrict__ off_ptr,
                           int32_t G, int lvl, int64_t* __restrict__ count_out) {
  const int lane = threadIdx.x & 31;
  const int32_t g = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (g >= G) return;
  GraphSel s = sel[g];
  uint32_t* hg = hist + (int64_t)g * kSelBins;
  if (s.take_all) {
    if (lvl == 1 && lane == 0) {
      s.count = off_ptr[g + 1] - off_ptr[g];
      s.thresh = 0;
      sel[g] = s;
      count_out[g] = s.count;
    }
    return;
  }
  const int64_t need = (lvl == 0) ? s.want : s.want - s.above1;
  // lane 0 owns the top 128 bins, lane 31 the lowest
  constexpr int per = kSelBins / 32;
  const int top = kSelBins - 1 - lane * per;
  int64_t mine = 0;
  for (int i = 0; i < per; i++) mine += hg[top - i];
  const int64_t incl = warp_incl_scan(mine);
  const int64_t excl = incl - mine;
  // first lane whose inclusive sum reaches need (or the last lane)
  const unsigned hit = __ballot_sync(0xffffffffu, incl >= need);
  const int owner = hit ? (__ffs(hit) - 1) : 31;
  int bin = 0;
  int64_t above = 0;
  if (lane == owner) {
    int64_t run = excl;
    bin = top - per + 1;  // lowest bin of the lane if need is never reached
    for (int i = 0; i < per; i++) {
      const uint32_t c = hg[top - i];
      if (run + c >= need) {
        bin = top - i;
        break;
      }
      run += c;
    }
    above = run;
  }
  bin = __shfl_sync(0xffffffffu, bin, owner);
  above = __shfl_sync(0xffffffffu, above, owner);
  const uint32_t bin_count = hg[bin];
  __syncwarp();
  for (int i = lane; i < kSelBins; i += 32) hg[i] = 0;
  if (lane == 0) {
    if (lvl == 0) {
      s.b1 = bin;
      s.above1 = above;
    } else {
      s.b2 = bin;
      s.above2 = above;
      s.count = s.above1 + above + bin_count;
      s.thresh = ((uint64_t)s.b1 << 52) | ((uint64_t)bin << 40);
      count_out[g] = s.count;
    }
    sel[g] = s;
  }
}

template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_sel_compact(const uint64_t* __restrict__ key, int64_t E,
                                                        const int64_t* __restrict__ off_ptr, int32_t G,
                                                        const GraphSel* __restrict__ sel,
                                                        int64_t* __restrict__ bcount, const int64_t* __restrict__ boff,
                                                        int64_t cap, int32_t* __restrict__ cand_idx,
                                                        uint64_t* __restrict__ rkey, int32_t* __restrict__ rval) {
  __shared__ int64_t sm[kBlock / 32 + 1];
  const int64_t chunk = sel_chunk(E, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(E, b0 + chunk);
  int64_t run = WRITE ? boff[blockIdx.x] : 0;
  int64_t tot = 0;
  for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kItems;
    uint32_t pick = 0;
    uint64_t k[kItems];
    // graph of the first item, then advanced item by item
    int32_t g = (G == 1 || base >= b1) ? 0 : part_of(off_ptr, G, base);
    int64_t g_end = (G == 1) ? INT64_MAX : off_ptr[g + 1];
    uint64_t th = sel[g].thresh;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t p = base + i;
      k[i] = 0;
      if (p < b1) {
        while (p >= g_end) {
          g++;
          g_end = off_ptr[g + 1];
          th = sel[g].thresh;
        }
        k[i] = key[p];
        if (k[i] >= th) pick |= 1u << i;
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

__global__ void k_sel_total(const int64_t* __restrict__ boff, int nb, const int64_t* __restrict__ cand_ptr,
                            int32_t G, int64_t cap, DevScalars* dsc) {
  const int64_t total = boff[nb];
  dsc->n_cand_wanted = total;
  if (total > cap || total != cand_ptr[G]) {
    // nothing downstream may touch more than `cap` candidates: run it empty
    dsc->n_cand = 0;
    atomicOr(&dsc->err, ERR_CAPACITY);
  } else {
    dsc->n_cand = total;
  }
}

}  // namespace

int step_select(Handle& h) {
  const int64_t E = h.E_off;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kSelChunkBlocks, (E + kTile - 1) / kTile));
  const int warps_per_block = 8;
  const int pick_grid = (h.G + warps_per_block - 1) / warps_per_block;
  bool any_select = false;
  for (int32_t g = 0; g < h.G; g++)
    if (h.want_h[g] < h.off_ptr_h[g + 1] - h.off_ptr_h[g]) any_select = true;
  for (int lvl = 0; lvl < 2; lvl++) {
    if (any_select) {
      ++h.launches;
      k_sel_hist<<<nb, kBlock, 0, h.stream>>>(h.key, E, h.d_off_ptr, h.G, h.sel, lvl, h.hist);
    }
    ++h.launches;
    k_sel_pick<<<pick_grid, warps_per_block * 32, 0, h.stream>>>(h.hist, h.sel, h.d_off_ptr, h.G, lvl, h.d_graph_tmp);
  }
  PDG_CUDA(cudaGetLastError());
  int st = scan_excl_i64(h, h.d_graph_tmp, h.d_cand_ptr, h.G, nullptr, h.G);
  if (st) return st;
  int64_t* bcount = h.blk_a;
  int64_t* boff = h.blk_a + 2560;
  ++h.launches;
  k_sel_compact<false><<<nb, kBlock, 0, h.stream>>>(h.key, E, h.d_off_ptr, h.G, h.sel, bcount, nullptr, 0, nullptr,
                                                    nullptr, nullptr);
  st = scan_excl_i64(h, bcount, boff, nb, nullptr, nb);
  if (st) return st;
  ++h.launches;
  k_sel_compact<true><<<nb, kBlock, 0, h.stream>>>(h.key, E, h.d_off_ptr, h.G, h.sel, nullptr, boff, h.Rcap,
                                                   h.cand_idx, h.rk[0], h.rv[0]);
  ++h.launches;
  k_sel_total<<<1, 1, 0, h.stream>>>(boff, nb, h.d_cand_ptr, h.G, h.Rcap, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
