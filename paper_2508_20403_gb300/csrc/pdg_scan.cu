// Device-wide exclusive prefix sums (reduce -> scan of block sums -> scan),
// used by every compaction of the pipeline.  The length may be a device
// value so that launches do not depend on data read back to the host.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kScanBlocksMax = 1024;

__device__ __forceinline__ int64_t load_n(int64_t n_host, const int64_t* n_dev) {
  return n_dev ? *n_dev : n_host;
}

__device__ __forceinline__ int64_t chunk_of(int64_t N, int nb) {
  int64_t c = (N + nb - 1) / nb;
  return (c + kTile - 1) / kTile * kTile;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_scan_reduce(const T* __restrict__ in, int64_t n_host,
                                                        const int64_t* n_dev, int64_t* __restrict__ bsum) {
  __shared__ int64_t sm[kBlock / 32 + 1];
  const int64_t N = load_n(n_host, n_dev);
  const int64_t chunk = chunk_of(N, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(N, b0 + chunk);
  int64_t s = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kBlock) s += (int64_t)in[i];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_top(int64_t* __restrict__ bsum, int nb, int64_t n_host,
                                                   const int64_t* n_dev, int64_t* __restrict__ out) {
  __shared__ int64_t sm[33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = (threadIdx.x < nb) ? bsum[threadIdx.x] : 0;
  int64_t inc = warp_incl_scan(x);
  if (lane == 31) sm[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t s = sm[lane];
    int64_t si = warp_incl_scan(s);
    sm[lane] = si - s;
    if (lane == 31) sm[32] = si;
  }
  __syncthreads();
  int64_t ex = sm[wid] + inc - x;
  if (threadIdx.x < nb) bsum[threadIdx.x] = ex;
  if (threadIdx.x == 0) out[load_n(n_host, n_dev)] = sm[32];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_scan_down(const T* __restrict__ in, int64_t* __restrict__ out,
                                                      int64_t n_host, const int64_t* n_dev,
                                                      const int64_t* __restrict__ bsum) {
  __shared__ int64_t sm[kBlock / 32 + 1];
  const int64_t N = load_n(n_host, n_dev);
  const int64_t chunk = chunk_of(N, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(N, b0 + chunk);
  int64_t run = bsum[blockIdx.x];
  for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
    int64_t base = t0 + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      v[i] = (base + i < b1) ? (int64_t)in[base + i] : 0;
      s += v[i];
    }
    int64_t tot;
    int64_t ex = block_excl_scan(s, sm, &tot) + run;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      if (base + i < b1) out[base + i] = ex;
      ex += v[i];
    }
    run += tot;
  }
}

template <typename T>
int scan_impl(Handle& h, const T* in, int64_t* out, int64_t n_host, const int64_t* n_dev, int64_t n_max) {
  if (n_max <= 0) n_max = 1;
  int nb = (int)std::min<int64_t>(kScanBlocksMax, (n_max + kTile - 1) / kTile);
  if (nb < 1) nb = 1;
  ++h.launches;
  k_scan_reduce<T><<<nb, kBlock, 0, h.stream>>>(in, n_host, n_dev, h.blk_b);
  ++h.launches;
  k_scan_top<<<1, 1024, 0, h.stream>>>(h.blk_b, nb, n_host, n_dev, out);
  ++h.launches;
  k_scan_down<T><<<nb, kBlock, 0, h.stream>>>(in, out, n_host, n_dev, h.blk_b);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace

int scan_excl_i64(Handle& h, const int64_t* in, int64_t* out, int64_t n_host, const int64_t* n_dev, int64_t n_max) {
  return scan_impl<int64_t>(h, in, out, n_host, n_dev, n_max);
}

int scan_excl_i32(Handle& h, const int32_t* in, int64_t* out, int64_t n_host, const int64_t* n_dev, int64_t n_max) {
  return scan_impl<int32_t>(h, in, out, n_host, n_dev, n_max);
}

int scan_excl_u32(Handle& h, const uint32_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max) {
  return scan_impl<uint32_t>(h, in, out, 0, n_dev, n_max);
}

int scan_excl_u8(Handle& h, const uint8_t* in, int64_t* out, const int64_t* n_dev, int64_t n_max) {
  return scan_impl<uint8_t>(h, in, out, 0, n_dev, n_max);
}

}  // namespace pdg
