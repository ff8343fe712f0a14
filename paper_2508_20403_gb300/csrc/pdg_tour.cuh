// Euler tours of a forest given by tree-edge flags over the canonical edge
// list: tree adjacency (both arcs of every tree edge, each knowing its
// reverse), the tour successor, and list ranking by pointer jumping.  Shared
// by spanning-tree generation (rooting) and the PCG quality measure (tree
// solves as prefix sums over the tour).  After x->y the tour takes the arc
// following y->x in y's adjacency row (cyclically); cutting the tour of a
// component at its root gives a list whose ranks order the arcs.
#pragma once

#include "pdg_internal.cuh"

namespace pdg {

namespace {

__global__ void k_st_tdeg(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                          const uint8_t* __restrict__ tflag, int64_t m, int32_t* tdeg) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    if (!tflag[e]) continue;
    atomicAdd(&tdeg[eu[e]], 1);
    atomicAdd(&tdeg[ev[e]], 1);
  }
}

// tree adjacency: both arcs of every tree edge, each knowing its reverse
__global__ void k_st_fill(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                          const uint8_t* __restrict__ tflag, int64_t m, const int64_t* __restrict__ tptr, int32_t* cur,
                          int32_t* __restrict__ tadj, int32_t* __restrict__ rev, int32_t* __restrict__ arc_uv) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    if (!tflag[e]) continue;
    const int32_t u = eu[e], v = ev[e];
    const int32_t pu = (int32_t)(tptr[u] + atomicAdd(&cur[u], 1));
    const int32_t pv = (int32_t)(tptr[v] + atomicAdd(&cur[v], 1));
    tadj[pu] = v;
    tadj[pv] = u;
    rev[pu] = pv;
    rev[pv] = pu;
    arc_uv[e] = pu;
  }
}

// Euler tour successor: after x->y comes the arc following y->x in y's row
// (cyclically); rd = 1 (one arc to the successor)
__global__ void k_st_succ(const int32_t* __restrict__ tadj, const int32_t* __restrict__ rev,
                          const int64_t* __restrict__ tptr, const int32_t* __restrict__ tdeg, int64_t n,
                          int32_t* __restrict__ succ, int32_t* __restrict__ rd) {
  const int64_t A = tptr[n];
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t y = tadj[a];
    const int64_t base = tptr[y];
    succ[a] = (int32_t)(base + (rev[a] - base + 1) % tdeg[y]);
    rd[a] = 1;
  }
}

// list ranking by pointer jumping: rd = arcs from a to the end of its tour
__global__ void k_st_rank(const int32_t* __restrict__ sin, const int32_t* __restrict__ rin,
                          int32_t* __restrict__ sout, int32_t* __restrict__ rout, const int64_t* __restrict__ tptr,
                          int64_t n) {
  const int64_t A = tptr[n];
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = sin[a];
    if (s < 0) {
      sout[a] = -1;
      rout[a] = rin[a];
    } else {
      sout[a] = sin[s];
      rout[a] = rin[a] + rin[s];
    }
  }
}

}  // namespace

}  // namespace pdg

namespace pdg {

namespace {

// Canonical tree adjacency (rows in increasing neighbour order) so that the
// Euler tour, and every sum taken along it, does not depend on the order in
// which the atomic fill placed the arcs.
__global__ void k_tour_sort_rows(const int64_t* __restrict__ tptr, int64_t n, int32_t* __restrict__ tadj) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = tptr[v], e = tptr[v + 1];
    for (int64_t p = b + 1; p < e; p++) {
      const int32_t x = tadj[p];
      int64_t q = p - 1;
      while (q >= b && tadj[q] > x) {
        tadj[q + 1] = tadj[q];
        q--;
      }
      tadj[q + 1] = x;
    }
  }
}

__device__ __forceinline__ int32_t tour_find(const int64_t* __restrict__ tptr, const int32_t* __restrict__ tadj,
                                            int32_t row, int32_t x) {
  int64_t lo = tptr[row], hi = tptr[row + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (tadj[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return (int32_t)lo;
}

// reverse arcs and the u->v arc of every tree edge, after the rows were sorted
__global__ void k_tour_fix_rev(const int64_t* __restrict__ tptr, const int32_t* __restrict__ tadj, int64_t n,
                               int32_t* __restrict__ rev) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    for (int64_t p = tptr[x]; p < tptr[x + 1]; p++) rev[p] = tour_find(tptr, tadj, tadj[p], (int32_t)x);
}

__global__ void k_tour_fix_arcs(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                const uint8_t* __restrict__ tflag, int64_t m, const int64_t* __restrict__ tptr,
                                const int32_t* __restrict__ tadj, int32_t* __restrict__ arc_uv) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    if (tflag[e]) arc_uv[e] = tour_find(tptr, tadj, eu[e], ev[e]);
}

}  // namespace

}  // namespace pdg
