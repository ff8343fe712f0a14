// Device-wide exclusive prefix sums, used by every compaction of the
// pipeline: out[i] = sum of in[0..i), out[N] = the total.  The length may be
// a device value so that launches do not depend on data read back to the
// host (the whole recovery is captured in a CUDA graph).
//
// One launch per scan.  Short inputs (capacity up to kScanSmall) are walked
// by a single block, tile after tile.  Longer ones use a single pass with
// decoupled look-back: blocks take tiles in order from a ticket counter, scan
// their tile, publish its sum, and add the sums of the earlier tiles read
// back through the published words -- one warp reads 32 of them per memory
// round trip.  Every wait is bounded (spin_limit): a timeout sets an error
// bit instead of hanging.  The last block to finish clears the status words
// and counters, so the next scan starts clean without a memset.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int64_t kScanSmall = 8 * kTile;

__device__ __forceinline__ int64_t load_n(int64_t n_host, const int64_t* n_dev) {
  return n_dev ? *n_dev : n_host;
}

// Loads the kItems values of this thread in tile t0 (zero past N); returns their sum.
template <typename T>
__device__ __forceinline__ int64_t load_items(const T* __restrict__ in, int64_t base, int64_t N,
                                              int64_t (&v)[kItems]) {
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    v[i] = (base + i < N) ? (int64_t)in[base + i] : 0;
    s += v[i];
  }
  return s;
}

__device__ __forceinline__ void store_items(int64_t* __restrict__ out, int64_t base, int64_t N, int64_t ex,
                                            const int64_t (&v)[kItems]) {
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    if (base + i < N) out[base + i] = ex;
    ex += v[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_scan_small(const T* __restrict__ in, int64_t* __restrict__ out,
                                                       int64_t n_host, const int64_t* n_dev) {
  dep_sync();
  __shared__ int64_t sm[kBlock / 32 + 1];
  const int64_t N = load_n(n_host, n_dev);
  int64_t run = 0;
  for (int64_t t0 = 0; t0 < N; t0 += kTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    const int64_t s = load_items(in, base, N, v);
    int64_t tot;
    const int64_t ex = block_excl_scan(s, sm, &tot) + run;
    store_items(out, base, N, ex, v);
    run += tot;
  }
  if (threadIdx.x == 0) out[N] = run;
}

template <typename T>
__global__ void __launch_bounds__(kLbThreads) k_scan_onepass(const T* __restrict__ in, int64_t* __restrict__ out,
                                                             int64_t n_host, const int64_t* n_dev, uint64_t* status,
                                                             uint32_t* ctr, int64_t spin_limit, DevScalars* dsc) {
  dep_sync();
  __shared__ int64_t sm[kLbThreads / 32 + 1];
  __shared__ int64_t s_tile, s_excl;
  __shared__ int s_last;
  const int64_t N = load_n(n_host, n_dev);
  const int64_t nt = (N + kLbTile - 1) / kLbTile;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(&ctr[0], 1u);  // tiles in launch order
  __syncthreads();
  const int64_t t = s_tile;
  if (t < nt) {
    const int64_t base = t * kLbTile + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    const int64_t s = load_items(in, base, N, v);
    int64_t tot;
    const int64_t ex = block_excl_scan_n<kLbThreads>(s, sm, &tot);
    if (threadIdx.x < 32) {
      bool timed_out;
      const int64_t excl = warp_lookback(status, t, tot, spin_limit, &timed_out);
      if (lane == 0) {
        if (timed_out) atomicOr(&dsc->err, ERR_TIMEOUT);
        s_excl = excl;
        if (t == nt - 1) out[N] = excl + tot;
      }
    }
    __syncthreads();
    store_items(out, base, N, s_excl + ex, v);
  }
  // the last block to finish clears the status words and the counters
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&ctr[1], 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) {
    for (int64_t i = threadIdx.x; i < nt; i += kLbThreads) status[i] = 0;
    if (threadIdx.x == 0) {
      ctr[0] = 0;
      ctr[1] = 0;
      if (nt == 0) out[N] = 0;
    }
  }
}

template <typename T>
int scan_impl(Handle& h, const T* in, int64_t* out, int64_t n_host, const int64_t* n_dev, int64_t n_max) {
  if (n_max <= 0) n_max = 1;
  ++h.launches;
  if (n_max <= kScanSmall) {
    launch_k(h, k_scan_small<T>, 1, kBlock, 0, in, out, n_host, n_dev);
  } else {
    const int64_t tiles = (n_max + kLbTile - 1) / kLbTile;
    if (tiles > h.scan_tiles_cap || tiles > 0x7fffffff) return PDG_E_INVALID_ARG;  // sized at init / growth
    launch_k(h, k_scan_onepass<T>, (int)tiles, kLbThreads, 0, in, out, n_host, n_dev, h.scan_status, h.scan_ctr,
             h.opt.spin_limit, h.dsc);
  }
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
