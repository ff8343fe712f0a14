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
// Digits shared by every key are detected from the histogram and their
// scatter is skipped.  Problem sizes are read on the device so the whole
// sequence can be captured in a CUDA graph.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kRdxBins = 256;
constexpr int kRdxWarps = kBlock / 32;
constexpr int kRdxPerWarp = kTile / kRdxWarps;  // 256 items, 8 rounds of 32

__device__ __forceinline__ int64_t tiles_of(int64_t N) { return (N + kTile - 1) / kTile; }

__global__ void __launch_bounds__(kBlock) k_rdx_hist(const uint64_t* __restrict__ k0, const uint64_t* __restrict__ k1,
                                                     DevScalars* dsc, int shift, uint32_t* __restrict__ hist,
                                                     uint32_t* __restrict__ dtot) {
  __shared__ uint32_t cnt[kRdxBins];
  const int64_t N = dsc->n_cand;
  const uint64_t* keys = dsc->radix_sel ? k1 : k0;
  const int64_t T = tiles_of(N);
  if (blockIdx.x == 0 && threadIdx.x == 0) dsc->radix_len = (int64_t)kRdxBins * T;
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = t * kTile;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t idx = base + (int64_t)i * kBlock + threadIdx.x;
      if (idx < N) atomicAdd(&cnt[(keys[idx] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    const uint32_t c = cnt[threadIdx.x];
    hist[(int64_t)threadIdx.x * T + t] = c;
    if (c) atomicAdd(&dtot[threadIdx.x], c);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kBlock) k_rdx_scatter(const uint64_t* k0, const uint64_t* k1,
                                                        const int32_t* v0, const int32_t* v1,
                                                        uint64_t* ko0, uint64_t* ko1,
                                                        int32_t* vo0, int32_t* vo1,
                                                        DevScalars* dsc, int shift, const int64_t* __restrict__ off,
                                                        const uint32_t* __restrict__ dtot) {
  __shared__ uint32_t wcnt[kRdxWarps][kRdxBins];
  const int64_t N = dsc->n_cand;
  if (N == 0) return;
  const int sel = dsc->radix_sel;
  const uint64_t* keys = sel ? k1 : k0;
  const int32_t* vals = sel ? v1 : v0;
  uint64_t* ko = sel ? ko0 : ko1;
  int32_t* vo = sel ? vo0 : vo1;
  if (dtot[(keys[0] >> shift) & 0xff] == (uint32_t)N) return;  // uniform digit: nothing moves
  const int64_t T = tiles_of(N);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1;
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    for (int d = lane; d < kRdxBins; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    uint64_t kk[kItems];
    int32_t vv[kItems];
    int dig[kItems];
    uint32_t rnk[kItems];
    const int64_t base = t * kTile + (int64_t)w * kRdxPerWarp;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t idx = base + i * 32 + lane;
      const bool valid = idx < N;
      kk[i] = valid ? keys[idx] : 0;
      vv[i] = valid ? vals[idx] : 0;
      dig[i] = valid ? (int)((kk[i] >> shift) & 0xff) : kRdxBins;
      const unsigned peers = __match_any_sync(0xffffffffu, dig[i]);
      rnk[i] = valid ? wcnt[w][dig[i]] + __popc(peers & lt) : 0;
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) wcnt[w][dig[i]] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      uint32_t run = 0;
      for (int ww = 0; ww < kRdxWarps; ww++) {
        const uint32_t c = wcnt[ww][threadIdx.x];
        wcnt[ww][threadIdx.x] = run;
        run += c;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      if (dig[i] < kRdxBins) {
        const int64_t pos = off[(int64_t)dig[i] * T + t] + wcnt[w][dig[i]] + rnk[i];
        ko[pos] = kk[i];
        vo[pos] = vv[i];
      }
    }
    __syncthreads();
  }
}

__global__ void k_rdx_flip(DevScalars* dsc, int shift, const uint64_t* __restrict__ k0,
                           const uint64_t* __restrict__ k1, uint32_t* __restrict__ dtot) {
  // runs after the scatter: decide from the same histogram whether it moved data
  __shared__ int moved;
  const int64_t N = dsc->n_cand;
  if (threadIdx.x == 0) {
    const uint64_t* keys = dsc->radix_sel ? k1 : k0;
    moved = (N > 0) && (dtot[(keys[0] >> shift) & 0xff] != (uint32_t)N);
  }
  __syncthreads();
  dtot[threadIdx.x] = 0;
  if (threadIdx.x == 0 && moved) dsc->radix_sel ^= 1;
}

// keys := graph index of the candidate held as value (keeps graphs contiguous)
__global__ void k_key_graph(uint64_t* __restrict__ k0, uint64_t* __restrict__ k1, const int32_t* __restrict__ v0,
                            const int32_t* __restrict__ v1, const int64_t* __restrict__ cand_ptr, int32_t G,
                            DevScalars* dsc) {
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
  const int64_t N = dsc->n_cand;
  const int32_t* v = dsc->radix_sel ? v1 : v0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v[i];
}

}  // namespace

int scan_excl_u32(Handle& h, const uint32_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max);

static int radix_pass_full(Handle& h, int shift) {
  const int grid = h.num_sms * 4;
  const int64_t tiles_max = (h.Rcap + kTile - 1) / kTile;
  ++h.launches;
  k_rdx_hist<<<grid, kBlock, 0, h.stream>>>(h.rk[0], h.rk[1], h.dsc, shift, h.radix_hist, h.radix_dtot);
  PDG_CUDA(cudaGetLastError());
  int st = scan_excl_u32(h, h.radix_hist, h.radix_off, &h.dsc->radix_len, kRdxBins * tiles_max);
  if (st) return st;
  ++h.launches;
  k_rdx_scatter<<<grid, kBlock, 0, h.stream>>>(h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.rk[0], h.rk[1], h.rv[0], h.rv[1],
                                               h.dsc, shift, h.radix_off, h.radix_dtot);
  ++h.launches;
  k_rdx_flip<<<1, kRdxBins, 0, h.stream>>>(h.dsc, shift, h.rk[0], h.rk[1], h.radix_dtot);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

int step_sort(Handle& h) {
  const int grid = h.num_sms * 4;
  int st;
  // 1. score descending (ties keep ascending id order)
  for (int shift = 0; shift < 64; shift += 8)
    if ((st = radix_pass_full(h, shift))) return st;
  if (h.G > 1) {
    ++h.launches;
    k_key_graph<<<grid, kBlock, 0, h.stream>>>(h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.d_cand_ptr, h.G, h.dsc);
    PDG_CUDA(cudaGetLastError());
    for (int shift = 0; (1ll << shift) < h.G; shift += 8)
      if ((st = radix_pass_full(h, shift))) return st;
  }
  // 2. group ranks by LCA
  ++h.launches;
  k_key_lca<<<grid, kBlock, 0, h.stream>>>(h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.cand_idx, h.lca, h.rank_cand, h.dsc);
  PDG_CUDA(cudaGetLastError());
  for (int shift = 0; (1ll << shift) < h.n; shift += 8)
    if ((st = radix_pass_full(h, shift))) return st;
  ++h.launches;
  k_copy_vals<<<grid, kBlock, 0, h.stream>>>(h.rv[0], h.rv[1], h.lsort_rank, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
