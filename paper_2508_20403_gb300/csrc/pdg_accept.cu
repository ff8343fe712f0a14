// Steps A5 + A6: density-aware scheduling of the subtasks and the
// strict-similarity greedy inside each of them (Sec. 4.1; Algorithm 1 step 4).
//
// Semantics (per subtask, candidates in rank order): a candidate is recovered
// unless an earlier recovered candidate e = (u, v) of the subtask has it
// strictly similar, i.e. (u' in S_u and v' in S_v) or (u' in S_v and v' in
// S_u), with S_x = the beta*_e-hop neighbourhood of x in T (Def. "Similar
// edge (Strict)", Eq. beta-new).  Tree facts used instead of a BFS:
//   hops(x, y) <= b  <=>  exists i, j >= 0, i + j <= b, anc_i(x) == anc_j(y)
// where anc_i is the i-th ancestor.  Every candidate carries its endpoints'
// ancestors anc_0..c.
//
// Tiers (the paper's mixed strategy, re-cut for a GPU):
//   size 1            recovered outright (no earlier edge can mark it);
//   2..warp_tier_max  one warp per subtask: lane t holds candidate t, a
//                     32-bit conflict mask per lane is built from shuffled
//                     records, then the in-order resolution (an edge survives
//                     iff no earlier survivor's bit is set in its mask) runs
//                     as a 32-step shuffle loop -- the sequential semantics
//                     without any shared-memory round trip;
//   ..block_tier_max  one block per subtask, chunks of 32 in rank order: the
//                     recovered candidates of earlier chunks are markers in
//                     a shared-memory pair table, each chunk is resolved like
//                     a warp-tier subtask (the paper's per-subtask marking,
//                     with the marked set kept as ancestor pairs);
//   larger            the cooperative tier: all candidates of all large
//                     subtasks at once, in two phases over hash indexes.
//
// Cooperative tier.  Candidate e = (u, v) "registers" the ancestor pairs
// (anc_j(u), anc_j'(v)) for j, j' <= beta*_e.  If e marks e' = (x, y), then
// for one orientation and some i, i' <= c the pair (anc_i(x), anc_i'(y)) is
// one of e's registered pairs, and rank(e) < rank(e').
//   Phase A (one pass).  A pair table keeps, per pair, the smallest rank that
//   registered it.  Each candidate probes its <= 2(c+1)^2 pairs: if none was
//   registered by an earlier rank, no earlier edge can mark it and it is
//   recovered ("free").  Every pair that did show an earlier registrant is
//   flagged and given a block of exact entries, one per (j, j').
//   Phase B (rounds over the remaining "constrained" candidates).  Exact
//   entries keep the smallest rank of an ACCEPTED registrant and the smallest
//   rank of a still-UNDECIDED registrant (tagged with the round).  A probe of
//   pair (z1, z2) at (i, i') reads entry (j, j') only when the registrant
//   would reach it: hops(u, l) = j + hops(x, l) - i and hops(v, l) =
//   j' + hops(y, l) - i' fix beta*_e, and the entry is read iff i + j <= beta*_e
//   and i' + j' <= beta*_e -- so every hit is a true marker.  Per round an
//   undecided candidate is REJECTED if some hit has an accepted rank below its
//   own, ACCEPTED if no hit has an undecided rank below its own, else it
//   waits.  The earliest undecided candidate of every subtask always decides,
//   so the rounds reproduce the sequential result; after max_rounds a serial
//   finisher (one thread per subtask, in rank order) completes what is left.
// Keys determine their subtask (they sit at or below its LCA on the two
// sides), so one global table serves all subtasks at once.
#include "pdg_internal.cuh"

namespace pdg {

namespace {

constexpr int kA = PDG_MAX_C + 1;  // ancestors anc_0..anc_c per endpoint
constexpr uint32_t kNone = 0xffffffffu;

struct Rec {
  int32_t U[kA], V[kA];
  int32_t du, dv, b, rank;
};

struct RecArrays {
  const int32_t* u;
  const int32_t* v;
  const int32_t* anc;
  const int32_t* du;
  const int32_t* dv;
  const uint8_t* b;
  const int32_t* rank;
  int64_t cap;
};

__device__ __forceinline__ void load_rec(const RecArrays& ra, int64_t s, int c, Rec& r) {
  r.U[0] = ra.u[s];
  r.V[0] = ra.v[s];
#pragma unroll
  for (int j = 1; j < kA; j++) {
    r.U[j] = (j <= c) ? ra.anc[(int64_t)(j - 1) * ra.cap + s] : -1;
    r.V[j] = (j <= c) ? ra.anc[(int64_t)(c + j - 1) * ra.cap + s] : -1;
  }
  r.du = ra.du[s];
  r.dv = ra.dv[s];
  r.b = ra.b[s];
  r.rank = ra.rank[s];
}

// hops(x', x) <= b, given anc_0..b of both (X[j] is valid for j <= b)
__device__ __forceinline__ bool in_ball(const int32_t (&Xp)[kA], const int32_t (&X)[kA], int b) {
  bool hit = false;
#pragma unroll
  for (int j = 0; j < kA; j++)
#pragma unroll
    for (int i = 0; i < kA; i++)
      if (i + j <= b && Xp[i] == X[j]) hit = true;
  return hit;
}

// is e' (Up, Vp) strictly similar to e (U, V, b)?
__device__ __forceinline__ bool strictly_similar(const int32_t (&Up)[kA], const int32_t (&Vp)[kA],
                                                 const int32_t (&U)[kA], const int32_t (&V)[kA], int b) {
  return (in_ball(Up, U, b) && in_ball(Vp, V, b)) || (in_ball(Up, V, b) && in_ball(Vp, U, b));
}

// Records in (LCA, rank) order.  Each record is oriented by preorder label
// (first endpoint = the smaller label): the subtrees of the LCA's children
// are disjoint label ranges, so this orders the two children below the
// endpoints the same way for every edge of the subtask (an endpoint equal to
// the LCA is its own side and has the smaller label).  A marker with
// beta* >= 1 has both endpoints strictly inside the two child subtrees, so it
// can only mark an edge whose endpoints sit in the same two subtrees in the
// same order: one probe orientation suffices unless the prober has an
// endpoint on the LCA.  Ancestors anc_1..c come from the parent array.
__global__ void __launch_bounds__(kBlock) k_build_records(
    const int32_t* __restrict__ lsort_rank, const int32_t* __restrict__ rank_cand, const int32_t* __restrict__ cand_idx,
    const int32_t* __restrict__ ou, const int32_t* __restrict__ ov, const int32_t* __restrict__ lca,
    const u128* __restrict__ P, const int32_t* __restrict__ parent,
    int c, const DevScalars* __restrict__ dsc, int64_t cap, int32_t* __restrict__ rec_u, int32_t* __restrict__ rec_v,
    int32_t* __restrict__ rec_anc, int32_t* __restrict__ rec_du, int32_t* __restrict__ rec_dv,
    uint8_t* __restrict__ rec_b, int32_t* __restrict__ rec_rank, int32_t* __restrict__ rec_lca) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t N = dsc->n_cand;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = lsort_rank[s];
    const int32_t i = cand_idx[rank_cand[r]];
    const int32_t u = ou[i], v = ov[i];  // u < v
    const int32_t l = lca[i];
    const int32_t dl = (int32_t)(uint32_t)P[l];
    const int32_t du = (int32_t)(uint32_t)P[u] - dl, dv = (int32_t)(uint32_t)P[v] - dl;
    rec_u[s] = u;
    rec_v[s] = v;
    int32_t au = u, av = v;
    for (int j = 1; j <= c; j++) {
      au = au < 0 ? -1 : parent[au];
      av = av < 0 ? -1 : parent[av];
      rec_anc[(int64_t)(j - 1) * cap + s] = au;
      rec_anc[(int64_t)(c + j - 1) * cap + s] = av;
    }
    rec_du[s] = du;
    rec_dv[s] = dv;
    rec_b[s] = (uint8_t)min(min(du, dv), c);
    rec_rank[s] = r;
    rec_lca[s] = l;
  }
}

// Subtask boundaries: the positions whose LCA differs from the previous
// position's, in order (single pass: tiles in ticket order, block scan plus
// decoupled look-back); seg_begin[n_seg] = N closes the last segment.
__global__ void __launch_bounds__(kLbThreads) k_seg_starts(const int32_t* __restrict__ rec_lca, DevScalars* dsc,
                                                          int32_t* __restrict__ seg_begin, uint64_t* status,
                                                          uint32_t* ctr, int64_t spin_limit) {
  dep_sync();
  __shared__ int64_t sm[kLbThreads / 32 + 1];
  __shared__ int64_t s_tile, s_excl;
  __shared__ int s_last;
  const int64_t N = dsc->n_cand;
  const int64_t nt = (N + kLbTile - 1) / kLbTile;
  if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(&ctr[0], 1u);
  __syncthreads();
  const int64_t t = s_tile;
  if (t < nt) {
    const int64_t base = t * kLbTile + (int64_t)threadIdx.x * kItems;
    uint32_t head = 0;
    int32_t prev = (base > 0 && base < N) ? rec_lca[base - 1] : -1;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
      const int64_t p = base + i;
      if (p < N) {
        const int32_t l = rec_lca[p];
        if (p == 0 || l != prev) head |= 1u << i;
        prev = l;
      }
    }
    int64_t tile_tot;
    const int64_t local = block_excl_scan_n<kLbThreads>((int64_t)__popc(head), sm, &tile_tot);
    if (threadIdx.x < 32) {
      bool timed_out;
      const int64_t excl = warp_lookback(status, t, tile_tot, spin_limit, &timed_out);
      if (threadIdx.x == 0) {
        if (timed_out) atomicOr(&dsc->err, ERR_TIMEOUT);
        s_excl = excl;
        if (t == nt - 1) {
          dsc->n_seg = excl + tile_tot;
          seg_begin[excl + tile_tot] = (int32_t)N;
        }
      }
    }
    __syncthreads();
    int64_t pos = s_excl + local;
#pragma unroll
    for (int i = 0; i < kItems; i++)
      if (head & (1u << i)) seg_begin[pos++] = (int32_t)(base + i);
  }
  // the last block to finish clears the look-back words and the counters
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
      if (nt == 0) {
        dsc->n_seg = 0;
        seg_begin[0] = 0;
      }
    }
  }
}

// Appends the lanes with `pred` to list[*count ...] (one atomic per warp; the
// list keeps the lanes' order within a warp, not across warps).
__device__ __forceinline__ void warp_append(bool pred, int32_t value, int32_t* __restrict__ list, int64_t* count) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if (!b) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd((unsigned long long*)count, (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) list[base + __popc(b & ((1u << lane) - 1))] = value;
}

// Per subtask: singletons are recovered outright; the warp tier (2..warp_max
// candidates) and the cooperative tier (larger) are listed; the largest
// subtask is recorded.
constexpr int kBigChunk = 1024;  // positions per warp when listing the cooperative tier

__global__ void k_seg_tier(const int32_t* __restrict__ seg_begin, DevScalars* dsc, int warp_max, int block_max,
                           const int32_t* __restrict__ rec_rank, uint8_t* __restrict__ acc_flag,
                           int32_t* __restrict__ warp_seg, int32_t* __restrict__ block_seg,
                           int32_t* __restrict__ big_seg, int64_t* __restrict__ big_chunk,
                           int64_t* __restrict__ seg_regs) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t S = dsc->n_seg;
  const int lane = threadIdx.x & 31;
  int64_t mx = 0;
  unsigned long long nblk = 0;
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); q0 < S;
       q0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = q0 + lane;
    const int32_t b = (q < S) ? seg_begin[q] : 0;
    const int64_t sz = (q < S) ? seg_begin[q + 1] - b : 0;
    if (sz == 1) acc_flag[rec_rank[b]] = 1;
    warp_append(sz >= 2 && sz <= warp_max, (int32_t)q, warp_seg, &dsc->n_warp_seg);
    const bool blk = sz > warp_max && sz <= block_max;
    warp_append(blk, (int32_t)q, block_seg, &dsc->n_block_seg);
    nblk += blk ? sz : 0;
    // the cooperative subtask list (x = index in big_seg)
    const bool big = sz > max(warp_max, block_max);
    const unsigned bm = __ballot_sync(0xffffffffu, big);
    int64_t x = -1;
    if (bm) {
      unsigned long long xb = 0;
      if (lane == 0) xb = atomicAdd((unsigned long long*)&dsc->n_big_seg, (unsigned long long)__popc(bm));
      xb = __shfl_sync(0xffffffffu, xb, 0);
      if (big) {
        x = (int64_t)xb + __popc(bm & ((1u << lane) - 1));
        big_seg[x] = (int32_t)q;
        seg_regs[x] = 0;
      }
    }
    // cooperative subtasks are also cut into chunks, one warp each below
    const int nch = big ? (int)((sz + kBigChunk - 1) / kBigChunk) : 0;
    const int incl = warp_incl_scan(nch);
    const int wtot = __shfl_sync(0xffffffffu, incl, 31);
    if (wtot) {
      unsigned long long base = 0;
      if (lane == 31) base = atomicAdd((unsigned long long*)&dsc->n_big_chunk, (unsigned long long)wtot);
      base = __shfl_sync(0xffffffffu, base, 31);
      for (int k = 0; k < nch; k++)
        big_chunk[base + incl - nch + k] = (x << 32) | (int64_t)k * kBigChunk;
    }
    mx = max(mx, sz);
  }
  mx = __reduce_max_sync(0xffffffffu, (unsigned)min(mx, (int64_t)0x7fffffff));
  if (lane == 0 && mx) atomicMax((unsigned long long*)&dsc->max_seg, (unsigned long long)mx);
  for (int o = 16; o; o >>= 1) nblk += __shfl_down_sync(0xffffffffu, nblk, o);
  if (lane == 0 && nblk) atomicAdd((unsigned long long*)&dsc->n_block, nblk);
}

// One warp per chunk of a cooperative subtask: its positions join big_pos
// (contiguous, in order), start undecided and learn their subtask index x;
// pair registrations are counted per subtask (they size its table region).
__global__ void k_big_positions(const int64_t* __restrict__ big_chunk, const int32_t* __restrict__ big_seg,
                                const int32_t* __restrict__ seg_begin, DevScalars* dsc,
                                const uint8_t* __restrict__ rec_b, int32_t* __restrict__ big_pos,
                                uint8_t* __restrict__ state, int32_t* __restrict__ pos_x,
                                int64_t* __restrict__ seg_regs) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t nch = dsc->n_big_chunk;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long regs_all = 0;
  for (int64_t w = warp; w < nch; w += nwarps) {
    const int64_t c = big_chunk[w];
    const int32_t x = (int32_t)(c >> 32);
    const int32_t q = big_seg[x];
    const int32_t b = seg_begin[q] + (int32_t)(c & 0xffffffff);
    const int32_t e = min(seg_begin[q + 1], b + kBigChunk);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd((unsigned long long*)&dsc->n_big, (unsigned long long)(e - b));
    base = __shfl_sync(0xffffffffu, base, 0);
    unsigned long long regs = 0;
    for (int32_t s = b + lane; s < e; s += 32) {
      big_pos[base + (s - b)] = s;
      state[s] = ST_UNDECIDED;
      pos_x[s] = x;
      const unsigned bb = rec_b[s];
      if (bb > 0) regs += (unsigned long long)(bb + 1) * (bb + 1);
    }
    for (int o = 16; o; o >>= 1) regs += __shfl_down_sync(0xffffffffu, regs, o);
    if (lane == 0 && regs) atomicAdd((unsigned long long*)&seg_regs[x], regs);
    regs_all += regs;
  }
  if (lane == 0 && regs_all) atomicAdd((unsigned long long*)&dsc->big_regs, regs_all);
}

// ------------------------------------------------------------------ warp tier

__global__ void __launch_bounds__(kBlock) k_accept_warp(const int32_t* __restrict__ warp_seg,
                                                        const DevScalars* __restrict__ dsc,
                                                        const int32_t* __restrict__ seg_begin, int c, RecArrays ra,
                                                        uint8_t* __restrict__ acc_flag) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t nw = dsc->n_warp_seg;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = warp; x < nw; x += nwarps) {
    const int32_t q = warp_seg[x];
    const int32_t b0 = seg_begin[q];
    const int sz = seg_begin[q + 1] - b0;
    Rec me;
    if (lane < sz) load_rec(ra, b0 + lane, c, me);
    else {
#pragma unroll
      for (int j = 0; j < kA; j++) me.U[j] = me.V[j] = -1;
      me.b = 0;
      me.rank = 0;
    }
    unsigned mask = 0;  // bit s: my edge is strictly similar to lane s's edge (s < me)
    for (int s = 0; s < sz - 1; s++) {
      int32_t U[kA], V[kA];
#pragma unroll
      for (int j = 0; j < kA; j++) {
        U[j] = __shfl_sync(0xffffffffu, me.U[j], s);
        V[j] = __shfl_sync(0xffffffffu, me.V[j], s);
      }
      const int b = __shfl_sync(0xffffffffu, me.b, s);
      if (lane > s && lane < sz && strictly_similar(me.U, me.V, U, V, b)) mask |= 1u << s;
    }
    unsigned acc = 0;
    for (int s = 0; s < sz; s++) {
      const unsigned ms = __shfl_sync(0xffffffffu, mask, s);
      if ((ms & acc) == 0) acc |= 1u << s;
    }
    if (lane < sz) acc_flag[me.rank] = (acc >> lane) & 1u;
  }
}

__device__ __forceinline__ uint64_t pair_key(int32_t z1, int32_t z2) {
  return ((uint64_t)(uint32_t)z1 << 32) | (uint64_t)(uint32_t)z2;
}

// A saved index failed its range check: report (first site wins) and skip.
__device__ __noinline__ void bounds_fail(DevScalars* dsc, int site, int where = 0, int64_t pos = -1,
                                        int64_t val = -1) {
  if (atomicCAS(&dsc->bounds_site, 0, site) == 0) {
    dsc->bounds_where = where;
    dsc->bounds_pos = pos;
    dsc->bounds_val = val;
  }
  atomicOr(&dsc->err, ERR_BOUNDS);
}

// ------------------------------------------------------------------ block tier
//
// One warp-sized block per subtask of warp_tier_max+1 .. block_tier_max
// candidates, in chunks of 32 in rank order.  The RECOVERED candidates of the
// earlier chunks live in a shared-memory marker table: a recovered e = (u, v)
// with b = beta*_e enters every pair (anc_j(u), anc_j'(v)), j, j' <= b, with
// the bit of its slack (b - j, b - j').  A later e' hits the pair at (i, i')
// (its own ancestors anc_i, anc_i') exactly when i + j <= b and i' + j' <= b,
// i.e. when some stored slack dominates (i, i') -- the same reach test as the
// cooperative tier's exact entries, so a hit is a true marker and every
// marker hits.  Inside a chunk the warp tier's conflict masks and 32-step
// resolution decide the candidates that no earlier chunk marked; the
// recovered ones then enter the table.  Sequential semantics, no global
// atomics but the subtask ticket.

constexpr uint32_t kSlackBits = 4;  // slack index s * 4 + s' (c <= 3)

// slack bits (s, s') with s >= i and s' >= i'
__device__ __forceinline__ uint32_t dominating(int i, int ip) {
  uint32_t m = 0;
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
      if (s >= i && sp >= ip) m |= 1u << (s * kSlackBits + sp);
  return m;
}

template <int C>
__global__ void __launch_bounds__(32) k_accept_block(const int32_t* __restrict__ block_seg, DevScalars* dsc,
                                                     const int32_t* __restrict__ seg_begin, RecArrays ra,
                                                     int slots_log2, uint8_t* __restrict__ acc_flag) {
  dep_sync();
  extern __shared__ __align__(16) unsigned char bt_smem[];
  uint64_t* keys = reinterpret_cast<uint64_t*>(bt_smem);
  uint32_t* slack = reinterpret_cast<uint32_t*>(keys + (1 << slots_log2));
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int lane = threadIdx.x;
  const int64_t nb = dsc->n_block_seg;
  bool bad = false;
  for (;;) {
    unsigned long long x = 0;
    if (lane == 0) x = atomicAdd(&dsc->block_ticket, 1ull);
    x = __shfl_sync(0xffffffffu, x, 0);
    if ((int64_t)x >= nb) break;
    const int32_t q = block_seg[x];
    const int32_t b0 = seg_begin[q];
    const int sz = seg_begin[q + 1] - b0;
    // table of this subtask: load <= 1/2 even if every candidate is recovered
    int tl = 6;
    while ((1 << tl) < 2 * (C + 1) * (C + 1) * sz && tl < slots_log2) tl++;
    const uint32_t tmask = (1u << tl) - 1;
    for (int i = lane; i <= (int)tmask; i += 32) {
      keys[i] = kEmptyKey;
      slack[i] = 0;
    }
    __syncwarp();
    for (int p0 = 0; p0 < sz; p0 += 32) {
      const int n = min(32, sz - p0);
      const bool valid = lane < n;
      Rec me;
      if (valid) {
        load_rec(ra, b0 + p0 + lane, C, me);
      } else {
#pragma unroll
        for (int j = 0; j < kA; j++) me.U[j] = me.V[j] = -1;
        me.du = me.dv = me.b = 0;
        me.rank = 0;
      }
      // 1. markers recovered in earlier chunks
      bool marked = false;
      if (valid && p0 > 0) {
#pragma unroll
        for (int o = 0; o < 2; o++) {
          if (o == 1 && me.du > 0 && me.dv > 0) break;  // records are side-ordered
#pragma unroll
          for (int i = 0; i <= C; i++)
#pragma unroll
            for (int ip = 0; ip <= C; ip++) {
              const int32_t z1 = o ? me.V[i] : me.U[i], z2 = o ? me.U[ip] : me.V[ip];
              if (marked || z1 < 0 || z2 < 0) continue;
              const uint64_t key = pair_key(z1, z2);
              uint32_t h = (uint32_t)mix64(key) & tmask;
              for (uint32_t k = 0; k <= tmask; k++) {
                const uint64_t kk = keys[h];
                if (kk == key) {
                  if (slack[h] & dominating(i, ip)) marked = true;
                  break;
                }
                if (kk == kEmptyKey) break;
                h = (h + 1) & tmask;
              }
            }
        }
      }
      // 2. the chunk's own order among the candidates no earlier chunk marked
      const unsigned live = __ballot_sync(0xffffffffu, valid && !marked);
      unsigned mask = 0;  // bit s: my edge is strictly similar to lane s's edge (s < me)
      for (int s2 = 0; s2 < n - 1; s2++) {
        if (!((live >> s2) & 1u)) continue;  // uniform over the warp
        int32_t U[kA], V[kA];
#pragma unroll
        for (int j = 0; j < kA; j++) {
          U[j] = __shfl_sync(0xffffffffu, me.U[j], s2);
          V[j] = __shfl_sync(0xffffffffu, me.V[j], s2);
        }
        const int bs = __shfl_sync(0xffffffffu, me.b, s2);
        if (lane > s2 && ((live >> lane) & 1u) && strictly_similar(me.U, me.V, U, V, bs)) mask |= 1u << s2;
      }
      unsigned acc = 0;
      for (int s2 = 0; s2 < n; s2++) {
        const unsigned ms = __shfl_sync(0xffffffffu, mask, s2);
        if (((live >> s2) & 1u) && (ms & acc) == 0) acc |= 1u << s2;
      }
      const bool accepted = (acc >> lane) & 1u;
      if (valid) acc_flag[me.rank] = accepted ? 1 : 0;
      // 3. the recovered candidates become markers for the later chunks
      if (accepted && me.b > 0 && p0 + 32 < sz) {
#pragma unroll
        for (int j = 0; j <= C; j++)
#pragma unroll
          for (int jp = 0; jp <= C; jp++) {
            if (j > me.b || jp > me.b) continue;
            const uint64_t key = pair_key(me.U[j], me.V[jp]);
            const uint32_t bit = 1u << ((me.b - j) * kSlackBits + (me.b - jp));
            uint32_t h = (uint32_t)mix64(key) & tmask;
            uint32_t k = 0;
            for (; k <= tmask; k++) {
              const unsigned long long old =
                  atomicCAS(reinterpret_cast<unsigned long long*>(&keys[h]), (unsigned long long)kEmptyKey,
                            (unsigned long long)key);
              if (old == kEmptyKey || old == key) {
                atomicOr(&slack[h], bit);
                break;
              }
              h = (h + 1) & tmask;
            }
            if (k > tmask) bad = true;  // cannot happen at load <= 1/2
          }
      }
      __syncwarp();
    }
    __syncwarp();  // the next subtask clears the table
  }
  if (bad) bounds_fail(dsc, 8);
}

// ------------------------------------------------------------- cooperative tier




// Undecided entries carry a tag of (attempt, round) in their high word; later
// attempts and rounds have smaller tags, so an atomicMin registration always
// replaces an entry left by an earlier attempt, and a probe ignores entries
// whose tag is not its own round's.  The buffers are filled with all-ones
// when allocated and never need clearing.
__device__ __forceinline__ uint64_t und_tag(uint32_t epoch, int round) {
  return (uint64_t)(0xffffffffu - (epoch * 128u + (uint32_t)round)) << 32;
}

struct CoopArgs {
  RecArrays ra;
  const int32_t* big_pos;
  uint8_t* state;
  uint32_t* pmask;     // per position: probe bits (o, i, i') that showed an earlier registrant
  int32_t* reg_slot;   // per position: pair slot of each registered (j, j'), 16 per position
  int32_t* pslot;      // per position: pair slot of each flagged probe (o, i, i'), 32 per position
  PairSlot* ptab;
  ExactEnt* xtab;      // 16 entries (j * 4 + j') per flagged pair; their und field serves the even rounds
  unsigned long long* xund1;  // the undecided ranks of the odd rounds, one per entry of xtab
  const uint64_t* cap;  // effective pair-table capacity (device)
  int64_t* n_flag;     // flagged pairs (exact blocks handed out)
  int64_t xcap;        // exact blocks available
  int64_t* und_count;  // per round: candidates still waiting
  uint32_t* flagbits;  // one bit per pair slot: the pair has an exact block
  int32_t* und_list;   // positions left undecided by phase A (any order)
  int64_t* n_und;      // their number
  const int32_t* pos_x;     // per position: index of its cooperative subtask
  const int64_t* seg_pref;  // exclusive prefix of the subtasks' registrations
  DevScalars* dsc;
};

// The pair table is cut into one region per cooperative subtask (pairs never
// cross subtasks): region x holds 2 * registrations + 16 slots, so a thread
// works inside its own subtask's region, and the regions of the subtasks in
// flight stay few and small enough for L2.
struct Region {
  uint64_t base, size;
};

// (a subtask index outside [0, nbs) sets `bad`, which the caller reports)
__device__ __forceinline__ Region region_of(const CoopArgs& a, int32_t x, int64_t nbs, bool& bad) {
  if (x < 0 || x >= nbs) {
    bad = true;
    x = 0;
  }
  const int64_t p0 = a.seg_pref[x], p1 = a.seg_pref[x + 1];
  return Region{(uint64_t)(2 * p0 + 16 * (int64_t)x), (uint64_t)(2 * (p1 - p0) + 16)};
}

__device__ __forceinline__ uint32_t region_slot(const Region& r, uint64_t key) {
  return (uint32_t)(r.base + __umul64hi(mix64(key), r.size));
}

__device__ __forceinline__ bool slot_flagged(const uint32_t* __restrict__ bits, int32_t slot) {
  return (bits[slot >> 5] >> (slot & 31)) & 1u;
}

__global__ void k_coop_clear(PairSlot* __restrict__ tab, uint32_t* __restrict__ flagbits, DevScalars* dsc,
                             int64_t table_cap, uint64_t* __restrict__ cap_out, int64_t* __restrict__ n_flag,
                             int64_t* __restrict__ n_und, const int64_t* __restrict__ seg_pref) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  // slots of all subtask regions: twice the registrations (load <= 0.5) + 16 each
  const int64_t nbs = dsc->n_big_seg;
  int64_t want = 2 * seg_pref[nbs] + 16 * nbs;
  if (want < 1024) want = 1024;
  if (want > table_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&dsc->err, ERR_TABLE);
    want = table_cap;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cap_out = (uint64_t)want;
    *n_flag = 0;
    *n_und = 0;
  }
  if (dsc->n_big == 0) return;
  uint4* t4 = reinterpret_cast<uint4*>(tab);
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < want; i += (int64_t)gridDim.x * blockDim.x)
    t4[i] = ones;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= want / 32;
       i += (int64_t)gridDim.x * blockDim.x)
    flagbits[i] = 0;
}

// Phase A1: register every (anc_j(u), anc_j'(v)), j, j' <= beta*, with its rank.
// A candidate's keys advance through their probe sequences together: each
// round issues one CAS per still-unplaced key, so a thread waits for about
// as many rounds as its longest chain, not for the sum of its chains.
template <int C>
__global__ void __launch_bounds__(kBlock, 4) k_pair_register(CoopArgs a, DevScalars* dsc) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // e.g. the regions do not fit: the host retries with a larger table
  const int64_t nb = dsc->n_big, nbs = dsc->n_big_seg;
  bool bad = false;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = a.big_pos[q];
    Rec r;
    load_rec(a.ra, s, C, r);
    if (r.b == 0) continue;  // a 0-hop neighbourhood pair only matches the edge itself
    const Region rg = region_of(a, a.pos_x[s], nbs, bad);
    const uint32_t rend = (uint32_t)(rg.base + rg.size);
    constexpr int NP = (C + 1) * (C + 1);
    uint64_t key[NP];
    uint32_t slot[NP];  // capacities stay below 2^32 slots
    uint32_t want = 0;
#pragma unroll
    for (int t = 0; t < NP; t++) {
      const int j = t / (C + 1), jp = t % (C + 1);
      key[t] = pair_key(r.U[j], r.V[jp]);
      slot[t] = region_slot(rg, key[t]);
      if (j <= r.b && jp <= r.b) want |= 1u << t;
    }
    uint32_t pend = want;
    for (uint64_t step = 0; pend && step < rg.size; step++) {
      unsigned long long old[NP];
#pragma unroll
      for (int t = 0; t < NP; t++)
        old[t] = (pend >> t & 1u) ? atomicCAS(&a.ptab[slot[t]].key, (unsigned long long)kEmptyKey,
                                               (unsigned long long)key[t])
                                  : 0ull;
#pragma unroll
      for (int t = 0; t < NP; t++) {
        if (!(pend >> t & 1u)) continue;
        if (old[t] == kEmptyKey || old[t] == key[t]) pend &= ~(1u << t);
        else if (++slot[t] == rend) slot[t] = (uint32_t)rg.base;
      }
    }
    if (pend) {  // the table is full: report; the host retries with a larger one
      atomicOr(&dsc->err, ERR_TABLE);
      return;
    }
#pragma unroll
    for (int t = 0; t < NP; t++) {
      if (!(want >> t & 1u)) continue;
      const int j = t / (C + 1), jp = t % (C + 1);
      atomicMin(&a.ptab[slot[t]].minr, (uint32_t)r.rank);
      a.reg_slot[(int64_t)s * 16 + j * 4 + jp] = (int32_t)slot[t];
    }
  }
  if (bad) bounds_fail(dsc, 1);
}

// Phase A2: free candidates are recovered; probed pairs with an earlier
// registrant are flagged and get a block of exact entries.  Lookups advance
// together, one slot per round, like the inserts of phase A1.
template <int C>
__global__ void __launch_bounds__(kBlock, 4) k_pair_probe(CoopArgs a, DevScalars* dsc) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // e.g. the regions do not fit: the host retries with a larger table
  const int64_t nb = dsc->n_big, nbs = dsc->n_big_seg;
  bool bad = false;
  unsigned long long cons = 0;
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: every lane of a warp runs the same iterations
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); q0 < nb;
       q0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = q0 + lane;
    const bool valid = q < nb;
    const int32_t s = valid ? a.big_pos[q] : 0;
    Rec r;
    if (valid) load_rec(a.ra, s, C, r);
    uint32_t pm = 0;
    int nclaim = 0;
    constexpr int NQ = (C + 1) * (C + 1);
    const Region rg = valid ? region_of(a, a.pos_x[s], nbs, bad) : Region{0, 1};
    const uint32_t rend = (uint32_t)(rg.base + rg.size);
#pragma unroll
    for (int o = 0; o < 2 && valid; o++) {
      if (o == 1 && r.du > 0 && r.dv > 0) break;  // records are side-ordered: one orientation suffices
      const int dx = o ? r.dv : r.du, dy = o ? r.du : r.dv;
      uint64_t key[NQ];
      uint32_t slot[NQ];
      uint32_t pend = 0, found = 0;
#pragma unroll
      for (int t = 0; t < NQ; t++) {
        const int i = t / (C + 1), ip = t % (C + 1);
        const int32_t z1 = o ? r.V[i] : r.U[i];
        const int32_t z2 = o ? r.U[ip] : r.V[ip];
        key[t] = pair_key(z1, z2);
        slot[t] = region_slot(rg, key[t]);
        if (i <= dx && ip <= dy) pend |= 1u << t;
      }
      for (uint64_t step = 0; pend && step < rg.size; step++) {
        unsigned long long k[NQ];
#pragma unroll
        for (int t = 0; t < NQ; t++) k[t] = (pend >> t & 1u) ? a.ptab[slot[t]].key : 0ull;
#pragma unroll
        for (int t = 0; t < NQ; t++) {
          if (!(pend >> t & 1u)) continue;
          if (k[t] == key[t]) {
            found |= 1u << t;
            pend &= ~(1u << t);
          } else if (k[t] == kEmptyKey) {
            pend &= ~(1u << t);
          } else if (++slot[t] == rend) {
            slot[t] = (uint32_t)rg.base;
          }
        }
      }
      uint64_t info[NQ];  // minr | xidx << 32 of the found slots
#pragma unroll
      for (int t = 0; t < NQ; t++)
        info[t] = (found >> t & 1u) ? reinterpret_cast<const uint64_t*>(a.ptab + slot[t])[1] : 0ull;
#pragma unroll
      for (int t = 0; t < NQ; t++) {
        if (!(found >> t & 1u)) continue;
        const int i = t / (C + 1), ip = t % (C + 1);
        if ((uint32_t)info[t] >= (uint32_t)r.rank) continue;
        pm |= 1u << (o * 16 + i * 4 + ip);
        a.pslot[(int64_t)s * 32 + o * 16 + i * 4 + ip] = (int32_t)slot[t];
        if ((uint32_t)(info[t] >> 32) == kNone) nclaim++;
      }
    }
    if (valid) a.pmask[s] = pm;
    // flag the probed pairs: the first claimant hands a pair a block of exact
    // entries; block indices come from one atomic per warp
    int pre = warp_incl_scan(nclaim);
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    unsigned long long base = 0;
    if (lane == 0 && total) base = atomicAdd((unsigned long long*)a.n_flag, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0);
    unsigned long long xi = base + (unsigned long long)(pre - nclaim);
    for (int bit = 0; nclaim && bit < 32; bit++) {
      if (!(pm & (1u << bit))) continue;
      const int32_t slt = a.pslot[(int64_t)s * 32 + bit];
      if (*reinterpret_cast<volatile uint32_t*>(&a.ptab[slt].xidx) != kNone) continue;
      nclaim--;
      if ((int64_t)xi >= a.xcap) {
        atomicOr(&dsc->err, ERR_TABLE);
        break;
      }
      if (atomicCAS(&a.ptab[slt].xidx, kNone, (uint32_t)xi) == kNone) {
        ExactEnt* e = a.xtab + xi * 16;
        for (int w = 0; w < 16; w++) e[w].acc = kNone;  // undecided entries need no clearing (tags)
        atomicOr(&a.flagbits[slt >> 5], 1u << (slt & 31));
      }
      xi++;
    }
    if (valid) {
      a.state[s] = pm ? ST_UNDECIDED : ST_ACCEPTED_NEW;
      cons += pm ? 1 : 0;
    }
    // undecided positions join the list that the rounds of phase B walk
    const unsigned ub = __ballot_sync(0xffffffffu, valid && pm);
    if (ub) {
      int ubase = 0;
      if (lane == 0) ubase = (int)atomicAdd((unsigned long long*)a.n_und, (unsigned long long)__popc(ub));
      ubase = __shfl_sync(0xffffffffu, ubase, 0);
      if (valid && pm) a.und_list[ubase + __popc(ub & ((1u << lane) - 1))] = s;
    }
  }
  for (int o = 16; o; o >>= 1) cons += __shfl_down_sync(0xffffffffu, cons, o);
  if ((threadIdx.x & 31) == 0 && cons) atomicAdd((unsigned long long*)&dsc->n_constrained, cons);
  if (bad) bounds_fail(dsc, 1);
}

// exact registration of one candidate's flagged pairs (its pair slots, their
// exact blocks and the updates each issued as one batch)
//
// FIRST: reg_slot holds pair slots (round 1); an undecided candidate then
// overwrites them with the exact-block indices (all-ones: none), which later
// rounds and the finisher read directly.
template <int C, bool FIRST>
__device__ __forceinline__ void exact_register(const CoopArgs& a, int32_t s, int b, int32_t rank, bool accepted,
                                               uint64_t und_val, uint64_t cap, int buf) {
  if (b == 0) return;  // never registered (matches only itself)
  constexpr int NP = (C + 1) * (C + 1);
  int32_t sl[NP];
  uint32_t xi[NP];
#pragma unroll
  for (int t = 0; t < NP; t++) {
    const int j = t / (C + 1), jp = t % (C + 1);
    sl[t] = (j <= b && jp <= b) ? a.reg_slot[(int64_t)s * 16 + j * 4 + jp] : -1;
  }
  uint32_t bad = 0;  // failed range checks (1: pair slot, 2: exact block), reported once below
  if (FIRST) {
#pragma unroll
    for (int t = 0; t < NP; t++) {
      if (sl[t] >= 0 && (uint64_t)sl[t] >= cap) {
        bad |= 1u;
        sl[t] = -1;
      }
      xi[t] = (sl[t] >= 0 && slot_flagged(a.flagbits, sl[t])) ? a.ptab[sl[t]].xidx : kNone;
    }
    if (!accepted) {
#pragma unroll
      for (int t = 0; t < NP; t++) {
        const int j = t / (C + 1), jp = t % (C + 1);
        if (j <= b && jp <= b) a.reg_slot[(int64_t)s * 16 + j * 4 + jp] = (int32_t)xi[t];
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < NP; t++) xi[t] = (uint32_t)sl[t];
  }
#pragma unroll
  for (int t = 0; t < NP; t++) {
    if (xi[t] == kNone) continue;
    if ((int64_t)xi[t] >= a.xcap) {
      bad |= 2u;
      continue;
    }
    const int j = t / (C + 1), jp = t % (C + 1);
    const int64_t ei = (int64_t)xi[t] * 16 + j * 4 + jp;
    if (accepted) atomicMin(&a.xtab[ei].acc, (uint32_t)rank);
    else atomicMin(buf ? &a.xund1[ei] : &a.xtab[ei].und, (unsigned long long)und_val);
  }
  if (bad) bounds_fail(a.dsc, (bad & 1u) ? 2 : (FIRST ? 3 : 4), 0, s);
}

// exact probes: 2 = rejected, 1 = must wait, 0 = free of earlier markers.
// The pair slots of the flagged probes were saved by phase A2 (pslot); the
// first round replaces them by the exact-block indices.  The entries one
// flagged probe may read are loaded together.
template <int C, bool WITH_UND, bool FIRST>
__device__ __forceinline__ int exact_probe(const CoopArgs& a, int32_t s, const Rec& r, uint32_t pm, uint64_t tag,
                                           int where, uint64_t cap, int buf) {
  int res = 0;
  uint32_t xis[2][C + 1][C + 1];
  uint32_t bad = 0;  // failed range checks (1: pair slot, 2: exact block), reported once below
#pragma unroll
  for (int o = 0; o < 2; o++)
#pragma unroll
    for (int i = 0; i <= C; i++)
#pragma unroll
      for (int ip = 0; ip <= C; ip++) {
        const int bit = o * 16 + i * 4 + ip;
        int32_t v = (pm & (1u << bit)) ? a.pslot[(int64_t)s * 32 + bit] : -1;
        if (FIRST && v >= 0 && (uint64_t)v >= cap) {
          bad |= 1u;
          v = -1;
        }
        uint32_t xv = (FIRST && v >= 0) ? a.ptab[v].xidx : (uint32_t)v;
        if (xv != kNone && (int64_t)xv >= a.xcap) {
          bad |= 2u;
          xv = kNone;
        }
        xis[o][i][ip] = xv;
      }
  if (bad) bounds_fail(a.dsc, (bad & 1u) ? 5 : (FIRST ? 6 : 7), where, s);
  if (FIRST) {
#pragma unroll
    for (int o = 0; o < 2; o++)
#pragma unroll
      for (int i = 0; i <= C; i++)
#pragma unroll
        for (int ip = 0; ip <= C; ip++) {
          const int bit = o * 16 + i * 4 + ip;
          if (pm & (1u << bit)) a.pslot[(int64_t)s * 32 + bit] = (int32_t)xis[o][i][ip];
        }
  }
#pragma unroll
  for (int o = 0; o < 2; o++) {
    const int dx = o ? r.dv : r.du, dy = o ? r.du : r.dv;
#pragma unroll
    for (int i = 0; i <= C; i++)
#pragma unroll
      for (int ip = 0; ip <= C; ip++) {
        const uint32_t xi = xis[o][i][ip];
        if (xi == kNone) continue;
        const int h1 = dx - i, h2 = dy - ip;
        ulonglong2 ent[C + 1][C + 1];
#pragma unroll
        for (int j = 0; j + i <= C; j++)
#pragma unroll
          for (int jp = 0; jp + ip <= C; jp++) {
            const int bb = min(min(j + h1, jp + h2), C);
            const int64_t ei = (int64_t)xi * 16 + j * 4 + jp;
            ent[j][jp] = (i + j <= bb && ip + jp <= bb) ? __ldcg(reinterpret_cast<const ulonglong2*>(a.xtab + ei))
                                                        : make_ulonglong2(~0ull, ~0ull);
            if (WITH_UND && buf && i + j <= bb && ip + jp <= bb) ent[j][jp].y = __ldcg(a.xund1 + ei);
          }
#pragma unroll
        for (int j = 0; j + i <= C; j++)
#pragma unroll
          for (int jp = 0; jp + ip <= C; jp++) {
            const uint32_t acc = (uint32_t)ent[j][jp].x;
            const uint64_t und = ent[j][jp].y;
            if (acc < (uint32_t)r.rank) return 2;
            if (WITH_UND && (und & 0xffffffff00000000ull) == tag && (uint32_t)und < (uint32_t)r.rank) res = 1;
          }
      }
  }
  return res;
}

// Round 1 registrations: every cooperative candidate (the ones phase A
// accepted as accepted markers, the undecided ones as undecided, in the odd
// rounds' buffer); round 1 also replaces the saved pair slots by exact-block
// indices.
template <int C>
__global__ void __launch_bounds__(kBlock) k_exact_register(CoopArgs a, DevScalars* dsc) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  if (dsc->n_constrained == 0) return;
  const int64_t nb = dsc->n_big;
  const uint64_t cap = *a.cap;
  const uint64_t tag = und_tag(dsc->epoch, 1);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = a.big_pos[q];
    const uint8_t st = a.state[s];
    if (st != ST_UNDECIDED && st != ST_ACCEPTED_NEW) continue;
    const int b = a.ra.b[s];
    const int32_t rank = a.ra.rank[s];
    if (st == ST_UNDECIDED) {
      exact_register<C, true>(a, s, b, rank, false, tag | (uint64_t)(uint32_t)rank, cap, 1);
    } else {
      exact_register<C, true>(a, s, b, rank, true, 0, cap, 1);
      a.state[s] = ST_ACCEPTED;
    }
  }
}

// Round r (one launch): every undecided candidate probes the round-r entries
// (undecided ranks in buffer r & 1) and then registers for round r + 1 at
// once -- accepted ranks as final markers, still-undecided ranks in buffer
// (r + 1) & 1, which no probe of round r reads.  A probe of round r may
// already see markers accepted during round r; acceptance is final, so that
// only settles the prober earlier.
template <int C>
__global__ void __launch_bounds__(kBlock) k_exact_round(CoopArgs a, DevScalars* dsc, int round) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  if (dsc->n_constrained == 0) return;
  if (round > 1 && a.und_count[round - 1] == 0) return;
  const int64_t nb = *a.n_und;
  const uint64_t tag = und_tag(dsc->epoch, round), next_tag = und_tag(dsc->epoch, round + 1);
  const uint64_t cap = *a.cap;
  unsigned long long waiting = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = a.und_list[q];
    if (a.state[s] != ST_UNDECIDED) continue;
    Rec r;
    load_rec(a.ra, s, C, r);
    const int res = (round == 1) ? exact_probe<C, true, true>(a, s, r, a.pmask[s], tag, round, cap, round & 1)
                                 : exact_probe<C, true, false>(a, s, r, a.pmask[s], tag, round, cap, round & 1);
    if (res == 2) {
      a.state[s] = ST_REJECTED;
    } else if (res == 0) {
      exact_register<C, false>(a, s, r.b, r.rank, true, 0, cap, 0);
      a.state[s] = ST_ACCEPTED;
    } else {
      waiting++;
      exact_register<C, false>(a, s, r.b, r.rank, false, next_tag | (uint64_t)(uint32_t)r.rank, cap, (round + 1) & 1);
    }
  }
  for (int o = 16; o; o >>= 1) waiting += __shfl_down_sync(0xffffffffu, waiting, o);
  if ((threadIdx.x & 31) == 0 && waiting) atomicAdd((unsigned long long*)&a.und_count[round], waiting);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&dsc->rounds_used, round);
}

// The cooperative tier's end: every candidate's recovered flag (by rank).  In
// the common case the rounds decided every candidate, and the threads write
// the flags of all positions; otherwise one thread per cooperative subtask
// completes it serially in rank order and writes its flags as it goes.
template <int C>
__global__ void k_exact_finish(CoopArgs a, DevScalars* dsc, const int32_t* __restrict__ big_seg,
                               const int32_t* __restrict__ seg_begin, int last_round, uint8_t* __restrict__ acc_flag) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t left = dsc->n_constrained == 0 ? 0 : a.und_count[last_round];
  if (blockIdx.x == 0 && threadIdx.x == 0) dsc->finish_left = left;  // sizes the next recovery's rounds
  if (left == 0) {
    const int64_t nb = dsc->n_big;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x) {
      const int32_t s = a.big_pos[q];
      const uint8_t st = a.state[s];
      acc_flag[a.ra.rank[s]] = (st == ST_ACCEPTED || st == ST_ACCEPTED_NEW) ? 1 : 0;
    }
    return;
  }
  const int64_t ns = dsc->n_big_seg;
  const uint64_t cap = *a.cap;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ns; x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = big_seg[x];
    for (int32_t s = seg_begin[q]; s < seg_begin[q + 1]; s++) {
      const uint8_t st = a.state[s];
      if (st == ST_ACCEPTED || st == ST_REJECTED) {
        acc_flag[a.ra.rank[s]] = st == ST_REJECTED ? 0 : 1;
        continue;
      }
      Rec r;
      load_rec(a.ra, s, C, r);
      if (st == ST_UNDECIDED && exact_probe<C, false, false>(a, s, r, a.pmask[s], 0, 99, cap, 0) == 2) {
        a.state[s] = ST_REJECTED;
        acc_flag[r.rank] = 0;
        continue;
      }
      exact_register<C, false>(a, s, r.b, r.rank, true, 0, cap, 0);
      a.state[s] = ST_ACCEPTED;
      acc_flag[r.rank] = 1;
    }
  }
}

template <int C>
int run_coop(Handle& h, const CoopArgs& a, int grid, int rounds) {
  ++h.launches;
  launch_k(h, k_pair_register<C>, grid, kBlock, 0, a, h.dsc);
  ++h.launches;
  launch_k(h, k_pair_probe<C>, grid, kBlock, 0, a, h.dsc);
  // round 1 registers every cooperative candidate; the rest of the rounds only
  // walk the (shorter) list of candidates phase A left undecided
  const int grid_und = std::max(1, h.num_sms * 2);
  ++h.launches;
  launch_k(h, k_exact_register<C>, grid, kBlock, 0, a, h.dsc);
  for (int r = 1; r <= rounds; r++) {
    ++h.launches;
    launch_k(h, k_exact_round<C>, grid_und, kBlock, 0, a, h.dsc, r);
  }
  ++h.launches;
  launch_k(h, k_exact_finish<C>, grid, kBlock, 0, a, h.dsc, h.big_seg, h.seg_begin, rounds, h.acc_flag);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace

// The block tier's size bound for this c: the table of a subtask of S
// candidates holds 2 (c+1)^2 S slots, at most kBlockTierSlots.
static int block_tier_max(const Handle& h, int c) {
  const int fit = kBlockTierSlots / (2 * (c + 1) * (c + 1));
  return std::min(h.opt.block_tier_max, fit);
}

int coop_rounds(const Handle& h, int c) {
  int R = std::max(1, std::min(h.opt.max_rounds, 64));
  if (h.rounds_mem >= 0 && h.c_mem == c && h.mode_mem == h.opt.score_mode) R = std::min(R, std::max(1, h.rounds_mem));
  return R;
}

int accept_setup() {
  const int smem = kBlockTierSlots * (int)(sizeof(uint64_t) + sizeof(uint32_t));
  PDG_CUDA(cudaFuncSetAttribute(k_accept_block<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  PDG_CUDA(cudaFuncSetAttribute(k_accept_block<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  PDG_CUDA(cudaFuncSetAttribute(k_accept_block<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  PDG_CUDA(cudaFuncSetAttribute(k_accept_block<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return PDG_OK;
}

static int accept_coop(Handle& h, int c, int grid, const RecArrays& ra);

int step_accept(Handle& h, int c) {
  const int grid = h.num_sms * 8;
  const int64_t cap = h.Rcap;
  int st;
  ++h.launches;
  launch_k(h, k_build_records, grid, kBlock, 0, h.lsort_rank, h.rank_cand, h.cand_idx, h.off_u, h.off_v, h.lca,
           h.P, h.parent, c, h.dsc, cap, h.rec_u, h.rec_v, h.rec_anc,
           h.rec_du, h.rec_dv, h.rec_b, h.rec_rank, h.rec_lca);
  // subtask boundaries, tier lists, per-position tiers
  const int64_t lb_tiles = (cap + kLbTile - 1) / kLbTile;
  if (lb_tiles > h.scan_tiles_cap || lb_tiles > 0x7fffffff) return PDG_E_INVALID_ARG;  // sized with the buffers
  ++h.launches;
  launch_k(h, k_seg_starts, (int)std::max<int64_t>(lb_tiles, 1), kLbThreads, 0,
           h.rec_lca, h.dsc, h.seg_begin, h.scan_status, h.scan_ctr, h.opt.spin_limit);
  ++h.launches;
  const int block_max = block_tier_max(h, c);
  launch_k(h, k_seg_tier, grid, kBlock, 0, h.seg_begin, h.dsc, h.opt.warp_tier_max, block_max, h.rec_rank,
           h.acc_flag, h.warp_seg, h.block_seg, h.big_seg, h.big_chunk,
           h.seg_regs);
  ++h.launches;
  launch_k(h, k_big_positions, grid, kBlock, 0, h.big_chunk, h.big_seg, h.seg_begin, h.dsc, h.rec_b, h.big_pos,
           h.state, h.pos_x, h.seg_regs);
  PDG_CUDA(cudaGetLastError());
  // table regions of the cooperative subtasks
  if ((st = scan_excl_i64(h, h.seg_regs, h.seg_pref, 0, &h.dsc->n_big_seg, cap))) return st;
  const RecArrays ra{h.rec_u, h.rec_v, h.rec_anc, h.rec_du, h.rec_dv, h.rec_b, h.rec_rank, cap};
  // The warp and block tiers decide other candidates than the cooperative
  // tier: they run on the side stream beside it (a fork and a join, also in
  // the captured graph), joined back before this step returns.
  const bool fork = h.sstream != nullptr && h.ev_fork != nullptr && h.ev_join != nullptr;
  const cudaStream_t side = fork ? h.sstream : h.stream;
  if (fork) {
    PDG_CUDA(cudaEventRecord(h.ev_fork, h.stream));
    PDG_CUDA(cudaStreamWaitEvent(h.sstream, h.ev_fork, 0));
    stream_op(h);
  }
  // warp tier
  ++h.launches;
  k_accept_warp<<<grid, kBlock, 0, side>>>(h.warp_seg, h.dsc, h.seg_begin, c, ra, h.acc_flag);
  PDG_CUDA(cudaGetLastError());
  // block tier
  if (block_max > h.opt.warp_tier_max) {
    int tl = 6;
    while ((1 << tl) < 2 * (c + 1) * (c + 1) * block_max) tl++;
    const size_t smem = ((size_t)1 << tl) * (sizeof(uint64_t) + sizeof(uint32_t));
    // as many one-warp blocks as the shared memory of an SM holds (227 KB, 1 KB reserved per block)
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(32, (size_t)(227 * 1024) / (smem + 1024)));
    const int bgrid = h.num_sms * per_sm;
    ++h.launches;
    switch (c) {
      case 0: k_accept_block<0><<<bgrid, 32, smem, side>>>(h.block_seg, h.dsc, h.seg_begin, ra, tl, h.acc_flag); break;
      case 1: k_accept_block<1><<<bgrid, 32, smem, side>>>(h.block_seg, h.dsc, h.seg_begin, ra, tl, h.acc_flag); break;
      case 2: k_accept_block<2><<<bgrid, 32, smem, side>>>(h.block_seg, h.dsc, h.seg_begin, ra, tl, h.acc_flag); break;
      default: k_accept_block<3><<<bgrid, 32, smem, side>>>(h.block_seg, h.dsc, h.seg_begin, ra, tl, h.acc_flag); break;
    }
    PDG_CUDA(cudaGetLastError());
  }
  if (fork) PDG_CUDA(cudaEventRecord(h.ev_join, h.sstream));
  st = accept_coop(h, c, grid, ra);
  if (fork && cudaStreamWaitEvent(h.stream, h.ev_join, 0) != cudaSuccess && st == PDG_OK) st = PDG_E_CUDA;
  stream_op(h);  // the next kernel waits for the side stream's tiers in full
  return st;
}

// the cooperative tier and the flags of its candidates (handle's stream)
static int accept_coop(Handle& h, int c, int grid, const RecArrays& ra) {
  int st;
  // cooperative tier; blk_a[9800..9916) is reserved for it (other steps use [0, 9729))
  uint64_t* d_cap = reinterpret_cast<uint64_t*>(h.blk_a + 9800);
  int64_t* n_flag = h.blk_a + 9801;
  int64_t* und_count = h.blk_a + 9850;  // [0 .. max_rounds], max_rounds <= 64
  int64_t* n_und = h.blk_a + 9802;
  const int R = coop_rounds(h, c);
  PDG_CUDA(cudaMemsetAsync(und_count, 0, sizeof(int64_t) * (R + 1), h.stream));
  stream_op(h);
  ++h.launches;
  launch_k(h, k_coop_clear, grid, kBlock, 0, h.ptab, h.flagbits, h.dsc, h.table_cap, d_cap, n_flag, n_und,
           h.seg_pref);
  const CoopArgs a{ra,        h.big_pos, h.state,   h.pmask,    h.reg_slot, h.pslot, h.ptab, h.xtab, h.xund1,
                   d_cap,     n_flag,    h.xcap,    und_count,  h.flagbits, h.und_list, n_und, h.pos_x,
                   h.seg_pref, h.dsc};
  switch (c) {
    case 0: st = run_coop<0>(h, a, grid, R); break;
    case 1: st = run_coop<1>(h, a, grid, R); break;
    case 2: st = run_coop<2>(h, a, grid, R); break;
    default: st = run_coop<3>(h, a, grid, R); break;
  }
  if (st) return st;
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
