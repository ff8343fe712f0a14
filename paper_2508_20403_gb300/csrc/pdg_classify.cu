// Step A1: split the edges of G into tree and off-tree edges (Sec. 2.2: every
// edge of G is either a tree edge or an off-tree edge) and compact the
// off-tree edges, in canonical id order, into structure-of-arrays form.
//
// Canonical id of {u, v}, u < v: rank of the CSR entry (u, v) among all
// entries with row < col in row-major order.  The handle keeps the graph as
// its canonical edge list (id order; built once from the CSR by
// build_edge_list at init, endpoints then relabelled in the tree's preorder
// as (a, b), a < b), so every recovery classifies by streaming that list: a
// parent's label is below its child's, so edge (a, b) is a tree edge iff
// parent[b] == a.  The write pass also records, for every non-root vertex x,
// r(x) = fl(1/w(x, parent x)) (the resistive weight W_re = 1/w of Eq. RT),
// computed on the integer pipes (pdg_fp.cuh), and the exponent range of these
// r that fixes the fixed-point scale of step A2.
//
// Layout: each block owns a contiguous chunk of edges (CSR entries for the
// edge-list build), taken in tiles of kTile; each thread reads kItems
// consecutive items with vector loads.  Two passes: a count pass, then a
// write pass that places each tile's output as one contiguous run.
#include <climits>

#include "pdg_fp.cuh"
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

// Row of CSR entry p (largest u with row_ptr[u] <= p), found by one warp with
// 32-way splits: about log32(n) dependent loads instead of log2(n).
__device__ __forceinline__ int64_t warp_row_of(const int64_t* __restrict__ row_ptr, int64_t n, int64_t p) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;  // row_ptr[lo] <= p < row_ptr[hi]
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t q = lo + lane * step;
    const bool ok = q < hi && __ldg(row_ptr + q) <= p;
    const int last = 31 - __clz(__ballot_sync(0xffffffffu, ok));  // lane 0 is always ok
    lo += last * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

constexpr int kSpanMax = kTile;  // rows staged per tile (enough when no row is empty)

// Edge-list build (init): every CSR entry with row < col, in row-major order.
// The row starts a tile spans are staged in shared memory, so a thread finds
// its row by a short search there and then follows it incrementally; skewed
// rows cost the same as short ones.
template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_edge_list(const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ w, int64_t n, int64_t nnz,
                                                      int64_t* __restrict__ cnt_up,
                                                      const int64_t* __restrict__ off_up,
                                                      int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                                                      double* __restrict__ ew) {
  dep_sync();
  __shared__ int64_t sm[kBlock / 32 + 1];
  // row starts of the tile, relative to its first entry and clipped to
  // [-1, kTile + 1]: s_rp[j] = row_ptr[r0 + j] - t0
  __shared__ int16_t s_rp[kSpanMax + 1];
  __shared__ int64_t s_r0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t chunk = cls_chunk(nnz, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(nnz, b0 + chunk);
  int64_t run_up = WRITE ? off_up[blockIdx.x] : 0;
  int64_t tot_up = 0;
  if (b0 < b1 && wid == 0) {
    const int64_t r = warp_row_of(row_ptr, n, b0);
    if (lane == 0) s_r0 = r;
  }
  for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
    const int tlen = (int)min((int64_t)kTile, b1 - t0);
    __syncthreads();  // s_r0 is set; the previous tile's shared reads are done
    const int64_t r0 = s_r0;
    // stage row starts kBlock at a time until they cover the tile
    if (threadIdx.x == 0) s_rp[0] = (int16_t)max(__ldg(row_ptr + r0) - t0, (int64_t)-1);
    int span = 0;
    for (;;) {
      const int j = span + 1 + threadIdx.x;
      const int64_t r = r0 + j;
      const int64_t rel = (r <= n) ? __ldg(row_ptr + r) - t0 : (int64_t)kTile + 1;
      s_rp[j] = (int16_t)min(max(rel, (int64_t)-1), (int64_t)kTile + 1);
      __syncthreads();
      span += kBlock;
      if (s_rp[span] >= tlen || span >= kSpanMax) break;  // uniform
    }
    const bool covered = s_rp[span] >= tlen;  // else (many empty rows): global row_ptr
    const int rel0 = threadIdx.x * kItems;
    int32_t c[kItems];
    double x[kItems];
    int32_t rows[kItems];
    uint32_t is_up = 0;
    if (rel0 < tlen) {
      const int64_t base = t0 + rel0;
      load_cols(col, base, t0 + tlen, c);
      if (WRITE) load_weights(w, base, t0 + tlen, x);
      int64_t u, next;
      if (covered) {
        int lo = 0, hi = span;  // s_rp[lo] <= rel0 < s_rp[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_rp[mid] <= rel0) lo = mid; else hi = mid;
        }
        u = r0 + lo;
        next = t0 + s_rp[lo + 1];
      } else {
        u = row_of(row_ptr, n, base);
        next = __ldg(row_ptr + u + 1);
      }
#pragma unroll
      for (int i = 0; i < kItems; i++) {
        const int64_t p = base + i;
        if (i < tlen - rel0) {
          while (p >= next) {
            u++;
            next = covered ? t0 + s_rp[u - r0 + 1] : __ldg(row_ptr + u + 1);
          }
          rows[i] = (int32_t)u;
          if (u < c[i]) is_up |= 1u << i;
        }
      }
      if (rel0 + kItems >= tlen) s_r0 = u;  // row of the tile's last entry: the next tile starts there
    }
    const int64_t n_up = __popc(is_up);
    if (!WRITE) {
      tot_up += n_up;
      continue;
    }
    int64_t tile_tot;
    int64_t pos = run_up + block_excl_scan(n_up, sm, &tile_tot);
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      if (is_up & (1u << i)) {
        eu[pos] = rows[i];
        ev[pos] = c[i];
        ew[pos] = x[i];
        pos++;
      }
    }
    run_up += tile_tot;
  }
  if (!WRITE) {
    tot_up = block_sum(tot_up, sm);
    if (threadIdx.x == 0) cnt_up[blockIdx.x] = tot_up;
  }
}

// Recovery-time classification of the canonical edge list.  Count pass:
// off-tree edges per block.  Write pass: r(x) for the tree edges (queued per
// warp so the reciprocals run densely, every lane on a tree edge) and the
// off-tree SoA, staged per tile and written as one coalesced run.
template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_classify(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                                     const double* __restrict__ ew,
                                                     const int32_t* __restrict__ parent, int64_t m,
                                                     int64_t* __restrict__ cnt_off,
                                                     const int64_t* __restrict__ off_off,
                                                     double* __restrict__ rtree, int32_t* __restrict__ ou,
                                                     int32_t* __restrict__ ov, int32_t* __restrict__ oid,
                                                     double* __restrict__ ow, DevScalars* __restrict__ dsc) {
  dep_sync();
  __shared__ int64_t sm[kBlock / 32 + 1];
  // write pass: per-warp queue of (child, weight) for the reciprocals, then
  // the tile's off-tree records (a tile holds at most kTile entries of each)
  __shared__ double st_w[WRITE ? kTile : 1];
  __shared__ int32_t st_u[WRITE ? kTile : 1], st_v[WRITE ? kTile : 1], st_id[WRITE ? kTile : 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t chunk = cls_chunk(m, gridDim.x);
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(m, b0 + chunk);
  int64_t run_off = WRITE ? off_off[blockIdx.x] : 0;
  int64_t tot_off = 0;
  int e_lo = INT_MAX, e_hi = INT_MIN;  // exponent range of the r(x) this thread writes
  for (int64_t t0 = b0; t0 < b1; t0 += kTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kItems;
    int32_t a[kItems], b[kItems], child[kItems];
    double x[kItems];
    uint32_t is_off = 0, is_tree = 0;
    if (base < b1) {
      load_cols(eu, base, b1, a);
      load_cols(ev, base, b1, b);
      if (WRITE) load_weights(ew, base, b1, x);
      int32_t pb[kItems];
#pragma unroll
      for (int i = 0; i < kItems; i++) pb[i] = (base + i < b1) ? __ldg(parent + b[i]) : -1;
#pragma unroll
      for (int i = 0; i < kItems; i++) {
        if (base + i >= b1) continue;
        if (pb[i] == a[i]) {
          is_tree |= 1u << i;
          child[i] = b[i];
        } else {
          is_off |= 1u << i;
        }
      }
    }
    const int64_t n_off = __popc(is_off);
    if (!WRITE) {
      tot_off += n_off;
      continue;
    }
    {
      const int ntree = __popc(is_tree);
      const int incl = warp_incl_scan(ntree);
      int slot = wid * (kTile / (kBlock / 32)) + incl - ntree;
#pragma unroll
      for (int i = 0; i < kItems; i++) {
        if (is_tree & (1u << i)) {
          st_u[slot] = child[i];
          st_w[slot] = x[i];
          slot++;
        }
      }
      __syncwarp();
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      for (int j = lane; j < tot; j += 32) {
        const int q = wid * (kTile / (kBlock / 32)) + j;
        const double wq = st_w[q];
        bool ok;
        const uint64_t rb = rcp_rn_bits((uint64_t)__double_as_longlong(wq), &ok);
        const double r = ok ? __longlong_as_double((long long)rb) : __drcp_rn(wq);
        rtree[st_u[q]] = r;
        const int e = (int)(((uint64_t)__double_as_longlong(r) >> 52) & 0x7ff) - 1023;
        e_lo = min(e_lo, e);
        e_hi = max(e_hi, e);
      }
    }
    int64_t tile_tot;
    int lpos = (int)block_excl_scan(n_off, sm, &tile_tot);  // also orders the queue reads
    // stage the tile's off-tree records in shared memory ...
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      if (is_off & (1u << i)) {
        st_u[lpos] = a[i];
        st_v[lpos] = b[i];
        st_id[lpos] = (int32_t)(base + i);
        st_w[lpos] = x[i];
        lpos++;
      }
    }
    __syncthreads();
    // ... and write them out as one contiguous, coalesced run
    const int cnt = (int)tile_tot;
    for (int j = threadIdx.x; j < cnt; j += kBlock) {
      ou[run_off + j] = st_u[j];
      ov[run_off + j] = st_v[j];
      oid[run_off + j] = st_id[j];
      ow[run_off + j] = st_w[j];
    }
    run_off += tile_tot;
    __syncthreads();
  }
  if (!WRITE) {
    tot_off = block_sum(tot_off, sm);
    if (threadIdx.x == 0) cnt_off[blockIdx.x] = tot_off;
  } else {
    // the exponent range of r over the tree (it fixes the fixed-point scale of
    // step A2): one atomic pair per block
    e_lo = __reduce_min_sync(0xffffffffu, e_lo);
    e_hi = __reduce_max_sync(0xffffffffu, e_hi);
    __shared__ int s_lo, s_hi;
    if (threadIdx.x == 0) {
      s_lo = INT_MAX;
      s_hi = INT_MIN;
    }
    __syncthreads();
    if (lane == 0) {
      atomicMin(&s_lo, e_lo);
      atomicMax(&s_hi, e_hi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_lo != INT_MAX) atomicMin(&dsc->e_min, s_lo);
      if (s_hi != INT_MIN) atomicMax(&dsc->e_max, s_hi);
    }
  }
}

}  // namespace

int build_edge_list(Handle& h) {
  if (h.nnz == 0) return PDG_OK;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(2048, (h.nnz + kTile - 1) / kTile));
  int64_t* cnt = h.blk_a;
  int64_t* off = h.blk_a + 2560;
  ++h.launches;
  launch_k(h, k_edge_list<false>, nb, kBlock, 0, h.row_ptr, h.col, h.w, h.n, h.nnz, cnt, nullptr, nullptr, nullptr,
           nullptr);
  PDG_CUDA(cudaGetLastError());
  int st = scan_excl_i64(h, cnt, off, nb, nullptr, nb);
  if (st) return st;
  ++h.launches;
  launch_k(h, k_edge_list<true>, nb, kBlock, 0, h.row_ptr, h.col, h.w, h.n, h.nnz, nullptr, off, h.el_u, h.el_v, h.el_w);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

// Init: the number of off-tree edges in each block's chunk of the edge list is
// a fact of the fixed tree, so the write offsets of the recovery's compaction
// are counted once here (a count pass and a scan) and kept.
int classify_layout(Handle& h) {
  if (h.m == 0) return PDG_OK;
  const int nb = h.nblk;
  int st;
  if ((st = device_alloc(h, (void**)&h.cls_off, sizeof(int64_t) * (size_t)(nb + 1)))) return st;
  int64_t* cnt_off = h.blk_a;
  ++h.launches;
  launch_k(h, k_classify<false>, nb, kBlock, 0, h.el_u, h.el_v, h.el_w, h.parent, h.m, cnt_off, nullptr, nullptr,
           nullptr, nullptr, nullptr, nullptr, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return scan_excl_i64(h, cnt_off, h.cls_off, nb, nullptr, nb);
}

// Recovery: one pass classifies every edge, writes r(x) of the tree edges
// and the off-tree records at the offsets counted at init.
int step_classify(Handle& h) {
  if (h.m == 0) return PDG_OK;
  ++h.launches;
  launch_k(h, k_classify<true>, h.nblk, kBlock, 0, h.el_u, h.el_v, h.el_w, h.parent, h.m, nullptr, h.cls_off,
           h.rtree, h.off_u, h.off_v, h.off_id, h.off_w, h.dsc);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
