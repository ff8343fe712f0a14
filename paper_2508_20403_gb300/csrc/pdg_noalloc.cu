// pdg_edge_endpoints_noalloc: the id -> (u, v) mapping of pdg_edge_endpoints
// for callers that cannot allocate device memory, e.g. code that runs while
// a caller-owned memory pool is the only allowed source of device memory,
// code inside a stream that must not trigger the implicit synchronisation of
// cudaMalloc/cudaFree, or latency-bound serving loops that must not block on
// the allocator.  It reads the caller's CSR directly (no handle) and keeps its
// only scratch -- the per-row prefix of upper-triangle entry counts and the
// scan's block sums -- in one file-scope device array of fixed size.
//
// Limits and sharing rules:
//   * n <= PDG_NOALLOC_MAX_N (2^21 vertices): the scratch array holds
//     PDG_NOALLOC_MAX_N + 1 + kNaBlocks int64 values plus an error word
//     (about 16 MB), reserved on every device that loads the library, until
//     the process exits.
//   * Every call shares that array.  Two calls that overlap on the same
//     device (different streams or host threads) race on it and may return
//     wrong endpoints; serialise them.
//   * The device address of the array is looked up once per device, on the
//     first call made with that device current (cudaGetSymbolAddress).  Make
//     that first call before any stream capture begins.
//   * The call waits for its stream on the host (it reads the error word
//     back), and clears a launch error left by earlier unrelated work before
//     it checks its own launches.
#include <mutex>

#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int64_t kNaMaxN = PDG_NOALLOC_MAX_N;
constexpr int kNaBlocks = 1024;  // blocks of the scan
constexpr int64_t kNaWords = kNaMaxN + 1 + kNaBlocks + 1;

// [0, n]            exclusive prefix of upper entries per row (row pointer of canonical ids)
// [kNaMaxN+1, ...)  block sums of the scan
// [kNaWords-1]      error word (non-zero: an id was out of range)
static __device__ __align__(256) int64_t g_na_scratch[kNaWords];

std::mutex g_na_mutex;
int64_t* g_na_addr[64] = {nullptr};  // device address of g_na_scratch per device ordinal

__device__ __forceinline__ int64_t na_chunk(int64_t N, int nb) {
  int64_t c = (N + nb - 1) / nb;
  return (c + kBlock - 1) / kBlock * kBlock;
}

// counts of entries with col > row, per row; block sums of those counts
__global__ void __launch_bounds__(kBlock) k_na_count(const int64_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col, int64_t n,
                                                     int64_t* __restrict__ scratch) {
  __shared__ int64_t sm[kBlock / 32 + 1];
  int64_t* cnt = scratch;
  int64_t* bsum = scratch + kNaMaxN + 1;
  const int64_t chunk = na_chunk(n, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  int64_t s = 0;
  for (int64_t u = b0 + threadIdx.x; u < b1; u += kBlock) {
    const int64_t b = row_ptr[u], e = row_ptr[u + 1];
    const int64_t c = e - lower_bound_i32(col, b, e, (int32_t)(u + 1));
    cnt[u] = c;
    s += c;
  }
  s = block_sum(s, sm);
  if (threadIdx.x == 0) bsum[blockIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) scratch[kNaWords - 1] = 0;  // clear the error word
}

__global__ void k_na_scan_blocks(int64_t* __restrict__ scratch, int nb) {
  if (threadIdx.x != 0) return;  // nb <= 1024 values: one thread is enough
  int64_t* bsum = scratch + kNaMaxN + 1;
  int64_t run = 0;
  for (int b = 0; b < nb; b++) {
    const int64_t x = bsum[b];
    bsum[b] = run;
    run += x;
  }
}

// in place: cnt[u] -> exclusive prefix; the last block also writes cnt[n]
__global__ void __launch_bounds__(kBlock) k_na_scan_rows(int64_t n, int64_t* __restrict__ scratch) {
  __shared__ int64_t sm[kBlock / 32 + 1];
  int64_t* cnt = scratch;
  const int64_t* bsum = scratch + kNaMaxN + 1;
  const int64_t chunk = na_chunk(n, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  int64_t run = bsum[blockIdx.x];
  for (int64_t t0 = b0; t0 < b1; t0 += kBlock) {
    const int64_t u = t0 + threadIdx.x;
    const int64_t x = (u < b1) ? cnt[u] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan(x, sm, &tot);
    if (u < b1) cnt[u] = run + ex;
    run += tot;
  }
  if (b1 == n && b0 < b1 && threadIdx.x == 0) cnt[n] = run;
}

__global__ void __launch_bounds__(kBlock) k_na_endpoints(const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col, int64_t n,
                                                         const int32_t* __restrict__ ids, int64_t count,
                                                         int32_t* __restrict__ ou, int32_t* __restrict__ ov,
                                                         int64_t* __restrict__ scratch) {
  const int64_t* up = scratch;  // up[u] = canonical id of row u's first upper entry
  const int64_t m = up[n];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = ids[i];
    if (id < 0 || id >= m) {
      scratch[kNaWords - 1] = 1;
      ou[i] = ov[i] = -1;
      continue;
    }
    int64_t lo = 0, hi = n;  // up[lo] <= id < up[hi]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (up[mid] <= id) lo = mid; else hi = mid;
    }
    const int64_t b = row_ptr[lo], e = row_ptr[lo + 1];
    const int64_t first = lower_bound_i32(col, b, e, (int32_t)(lo + 1));
    ou[i] = (int32_t)lo;
    ov[i] = col[first + (id - up[lo])];
  }
}

}  // namespace

}  // namespace pdg

extern "C" int pdg_edge_endpoints_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* ids,
                                          int64_t count, int32_t* u, int32_t* v, void* stream) {
  using namespace pdg;
  if (n < 1 || n > kNaMaxN || !row_ptr || !col || count < 0 || (count > 0 && (!ids || !u || !v)))
    return PDG_E_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PDG_E_CUDA;
  int64_t* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PDG_E_CUDA;
      }
      g_na_addr[dev] = static_cast<int64_t*>(p);
    }
    scratch = g_na_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();  // an earlier, unrelated launch error must not be reported as ours
  int num_sms = 0;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kNaBlocks, (n + kBlock - 1) / kBlock));
  k_na_count<<<nb, kBlock, 0, s>>>(row_ptr, col, n, scratch);
  k_na_scan_blocks<<<1, 32, 0, s>>>(scratch, nb);
  k_na_scan_rows<<<nb, kBlock, 0, s>>>(n, scratch);
  if (count > 0) {
    const int64_t blocks = std::min<int64_t>((count + kBlock - 1) / kBlock, (int64_t)std::max(num_sms, 1) * 16);
    k_na_endpoints<<<(int)blocks, kBlock, 0, s>>>(row_ptr, col, n, ids, count, u, v, scratch);
  }
  if (cudaGetLastError() != cudaSuccess) return PDG_E_CUDA;
  int64_t err = 0;
  if (cudaMemcpyAsync(&err, scratch + (kNaWords - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PDG_E_CUDA;
  return err ? PDG_E_INVALID_ARG : PDG_OK;
}
