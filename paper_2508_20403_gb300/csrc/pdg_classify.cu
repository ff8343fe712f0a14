// Step A1: split the edges of G into tree and off-tree edges (Sec. 2.2: every
// edge of G is either a tree edge or an off-tree edge) and compact the
// off-tree edges, in canonical id order, into structure-of-arrays form.
//
// Canonical id of {u, v}, u < v: rank of the CSR entry (u, v) among all
// entries with row < col in row-major order.  Edge (u, v) is a tree edge iff
// parent[v] == u or parent[u] == v.  The write pass also records, for every
// non-root vertex u, r(u) = fl(1/w(u, parent u)) (the resistive weight
// W_re = 1/w of Eq. RT).
//
// Layout: each block owns a contiguous chunk of CSR entries; each thread
// reads kItems consecutive entries (vector loads) and follows the row index
// incrementally from one binary search, so skewed rows cost the same as
// short ones.  Two passes: the count pass streams only the column indices,
// the write pass also the weights.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

__device__ __forceinline__ int64_t cls_chunk(int64_t nnz, int nb) {
  int64_t c = (nnz + nb - 1) / nb;
  return (c + kTile - 1) / kTile * kTile;
}

// Loads kItems column indices starting at base (base is a multiple of kItems).
__device__ __forceinline__ void load_cols(const int32_t* __restrict__ col, int64_t base, int64_t end,
                                          int32_t (&c)[kItems]) {
  if (base + kItems <= end) {
    const int4* c4 = reinterpret_cast<const int4*>(col + base);
    int4 a = __ldg(c4), b = __ldg(c4 + 1);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < kItems; i++) c[i] = (base + i < end) ? __ldg(col + base + i) : 0;
  }
}

__device__ __forceinline__ void load_weights(const double* __restrict__ w, int64_t base, int64_t end,
                                             double (&x)[kItems]) {
  if (base + kItems <= end) {
    const double2* w2 = reinterpret_cast<const double2*>(w + base);
#pragma unroll
    for (int i = 0; i < kItems / 2; i++) {
      double2 t = __ldg(w2 + i);
      x[2 * i] = t.x;
      x[2 * i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kItems; i++) x[i] = (base + i < end) ? __ldg(w + base + i) : 0.0;
  }
}

template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_classify(const int64_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col,
                                                     const double* __restrict__ w,
                                                     const int32_t* __restrict__ parent, int64_t n,
                                                     int64_t nnz, int64_t* __restrict__ cnt_up,
                                                     int64_t* __restrict__ cnt_off,
                                                     const int64_t* __restrict__ off_up,
                                                     const int64_t* __restrict__ off_off,
                                                     double* __restrict__ rtree, int32_t* __restrict__ ou,
                                                     int32_t* __restrict__ ov, int32_t* __restrict__ oid,
                                                     double* __restrict__ ow) {
  __shared__ int64_t sm[kBlock / 32 + 1];
  const int64_t chunk = cls_chunk(nnz, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(nnz, b0 + chunk);
  int64_t run_up = WRITE ? off_up[blockIdx.x] : 0;
  int64_t run_off = WRITE ? off_off[blockIdx.x] : 0;
  int64_t tot_up = 0, tot_off = 0;
  for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kItems;
    int32_t c[kItems];
    double x[kItems];
    uint32_t is_up = 0, is_off = 0;
    int32_t rows[kItems];
    if (base < b1) {
      load_cols(col, base, b1, c);
      if (WRITE) load_weights(w, base, b1, x);
      int64_t u = row_of(row_ptr, n, base);
      int64_t next = __ldg(row_ptr + u + 1);
      int32_t pu = __ldg(parent + u);
#pragma unroll
      for (int i = 0; i < kItems; i++) {
        const int64_t p = base + i;
        if (p < b1) {
          while (p >= next) {
            u++;
            next = __ldg(row_ptr + u + 1);
            pu = __ldg(parent + u);
          }
          rows[i] = (int32_t)u;
          const int32_t v = c[i];
          if (WRITE && pu == v) rtree[u] = 1.0 / x[i];
          if (u < v) {
            is_up |= 1u << i;
            const bool tree = (__ldg(parent + v) == (int32_t)u) || (pu == v);
            if (!tree) is_off |= 1u << i;
          }
        }
      }
    }
    const int64_t n_up = __popc(is_up), n_off = __popc(is_off);
    if (!WRITE) {
      tot_up += n_up;
      tot_off += n_off;
      continue;
    }
    int64_t tile_tot;
    int64_t ex = block_excl_scan((n_up << 32) | n_off, sm, &tile_tot);
    int64_t id = run_up + (ex >> 32);
    int64_t pos = run_off + (ex & 0xffffffffll);
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      if (is_up & (1u << i)) {
        if (is_off & (1u << i)) {
          ou[pos] = rows[i];
          ov[pos] = c[i];
          oid[pos] = (int32_t)id;
          ow[pos] = x[i];
          pos++;
        }
        id++;
      }
    }
    run_up += tile_tot >> 32;
    run_off += tile_tot & 0xffffffffll;
  }
  if (!WRITE) {
    tot_up = block_sum(tot_up, sm);
    tot_off = block_sum(tot_off, sm);
    if (threadIdx.x == 0) {
      cnt_up[blockIdx.x] = tot_up;
      cnt_off[blockIdx.x] = tot_off;
    }
  }
}

}  // namespace

int step_classify(Handle& h) {
  if (h.nnz == 0) return PDG_OK;
  const int nb = h.nblk;
  int64_t* cnt_up = h.blk_a;
  int64_t* cnt_off = h.blk_a + 2560;
  int64_t* off_up = h.blk_a + 5120;
  int64_t* off_off = h.blk_a + 7680;
  ++h.launches;
  k_classify<false><<<nb, kBlock, 0, h.stream>>>(h.row_ptr, h.col, h.w, h.parent, h.n, h.nnz, cnt_up, cnt_off,
                                                 nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  PDG_CUDA(cudaGetLastError());
  int st = scan_excl_i64(h, cnt_up, off_up, nb, nullptr, nb);
  if (st) return st;
  st = scan_excl_i64(h, cnt_off, off_off, nb, nullptr, nb);
  if (st) return st;
  ++h.launches;
  k_classify<true><<<nb, kBlock, 0, h.stream>>>(h.row_ptr, h.col, h.w, h.parent, h.n, h.nnz, nullptr, nullptr,
                                                off_up, off_off, h.rtree, h.off_u, h.off_v, h.off_id, h.off_w);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
