// Step A7: the recovery budget (Sec. 2.2: recover alpha*|V| edges, one pass).
//
// Recovered flags are indexed by rank, so a prefix count over ranks gives,
// per graph, the order in which the sequential greedy would have recovered
// them.  The first k_g are written out (local canonical ids, recovery order).
// A graph whose prefix held fewer than k_g survivors is marked for a retry
// with a longer prefix unless the prefix already was the whole edge list, in
// which case all survivors are returned (PDG_UNDER_BUDGET).
#include "pdg_internal.cuh"

namespace pdg {

namespace {

// One pass: each graph's status and count (written by one thread per graph)
// and the output of every recovered candidate within its graph's budget, both
// taken from the prefix count over ranks.
__global__ void __launch_bounds__(kBlock) k_budget_write(
    const uint8_t* __restrict__ acc_flag, const int64_t* __restrict__ scan, const int64_t* __restrict__ cand_ptr,
    int32_t G, const int64_t* __restrict__ kk, const GraphSel* __restrict__ sel, int32_t* __restrict__ gstat,
    int64_t* __restrict__ gcount, const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ rank_cand,
    const int32_t* __restrict__ cand_idx, const int32_t* __restrict__ off_id, const uint64_t* __restrict__ key,
    const int64_t* __restrict__ edge_ptr, const DevScalars* __restrict__ dsc, int32_t* __restrict__ out_ids,
    double* __restrict__ out_scores) {
  dep_sync();
  if (attempt_aborted(dsc)) return;  // the attempt is void
  const int64_t N = dsc->n_cand;
  if (N != cand_ptr[G]) return;  // selection overflowed: the host grows and repeats
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = tid; g < G; g += nth) {
    const int64_t cnt = scan[cand_ptr[g + 1]] - scan[cand_ptr[g]];
    const int64_t k = kk[g];
    gstat[g] = (cnt >= k) ? G_OK : (sel[g].take_all ? G_UNDER : G_RETRY);
    gcount[g] = min(cnt, k);
  }
  for (int64_t r = tid; r < N; r += nth) {
    if (!acc_flag[r]) continue;
    const int32_t g = (G == 1) ? 0 : part_of(cand_ptr, G, r);
    const int64_t c0 = scan[cand_ptr[g]], cnt = scan[cand_ptr[g + 1]] - c0, k = kk[g];
    if (cnt < k && !sel[g].take_all) continue;  // the graph is retried with a longer prefix
    const int64_t j = scan[r] - c0;
    if (j >= min(cnt, k)) continue;
    const int32_t i = cand_idx[rank_cand[r]];
    const int64_t pos = out_ptr[g] + j;
    out_ids[pos] = (int32_t)(off_id[i] - edge_ptr[g]);
    if (out_scores) out_scores[pos] = __longlong_as_double((long long)key[i]);
  }
}

}  // namespace

int step_budget(Handle& h, int32_t* out_ids, double* out_scores) {
  const int grid = h.num_sms * 4;
  int st = scan_excl_u8(h, h.acc_flag, h.scan_tmp, &h.dsc->n_cand, h.Rcap);
  if (st) return st;
  ++h.launches;
  launch_k(h, k_budget_write, grid, kBlock, 0, h.acc_flag, h.scan_tmp, h.d_cand_ptr, h.G, h.d_k, h.sel, h.gstat,
           h.gcount, h.d_out_ptr, h.rank_cand, h.cand_idx, h.off_id, h.key, h.d_edge_ptr, h.dsc, out_ids,
           out_scores);
  PDG_CUDA(cudaGetLastError());
  return PDG_OK;
}

}  // namespace pdg
