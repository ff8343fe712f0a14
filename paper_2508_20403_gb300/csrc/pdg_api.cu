// C ABI of the library (include/pdgrass.h): handle life cycle, input upload,
// the recovery driver (steps A1-A7 on the handle's stream, with the prefix
// retry of step A7) and small queries.
#include <cstdio>
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>

#include "pdg_internal.cuh"

namespace pdg {

int check_cuda(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return PDG_E_OOM;
  }
  return PDG_E_CUDA;
}

int grid_for(const Handle& h, int64_t work, int per_block) {
  int64_t blocks = (work + per_block - 1) / per_block;
  int64_t cap = (int64_t)h.num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// handle's stream): handles on different streams never synchronise each
// other through the allocator, which keeps concurrent batches overlapping.
// The device's default pool keeps freed memory cached for reuse.
static std::mutex g_pool_mutex;
static bool g_pool_ready[64] = {false};

static void prepare_pool(int device) {
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (device < 0 || device >= 64 || g_pool_ready[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  g_pool_ready[device] = true;
}

int device_alloc(Handle& h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  prepare_pool(h.device);
  cudaError_t e = cudaMallocAsync(p, bytes, h.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return PDG_E_OOM;
  }
  h.allocs.push_back(*p);
  h.device_bytes += bytes;
  return PDG_OK;
}

static void device_release(Handle& h, void* p) {
  if (!p) return;
  auto it = std::find(h.allocs.begin(), h.allocs.end(), p);
  if (it != h.allocs.end()) h.allocs.erase(it);
  cudaFreeAsync(p, h.stream);
}

// Pinned host staging is recycled across handles (cudaFreeHost would
// synchronise the whole device).
static std::mutex g_pinned_mutex;
static std::vector<std::pair<size_t, void*>> g_pinned_free;

static void* pinned_alloc(size_t bytes) {
  bytes = (bytes + 63) & ~(size_t)63;
  {
    std::lock_guard<std::mutex> lock(g_pinned_mutex);
    for (size_t i = 0; i < g_pinned_free.size(); i++)
      if (g_pinned_free[i].first == bytes) {
        void* p = g_pinned_free[i].second;
        g_pinned_free.erase(g_pinned_free.begin() + i);
        return p;
      }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void pinned_release(void* p, size_t bytes) {
  if (!p) return;
  bytes = (bytes + 63) & ~(size_t)63;
  std::lock_guard<std::mutex> lock(g_pinned_mutex);
  g_pinned_free.emplace_back(bytes, p);
}

template <typename T>
static int alloc_n(Handle& h, T** p, int64_t count) {
  return device_alloc(h, reinterpret_cast<void**>(p), sizeof(T) * (size_t)std::max<int64_t>(count, 1));
}

namespace {

__global__ void k_gather_rowptr(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ vtx_ptr, int32_t G,
                                int64_t* __restrict__ out) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x) out[g] = row_ptr[vtx_ptr[g]];
}

__global__ void k_reset_recover(DevScalars* dsc) {
  dep_sync();
  dsc->err = 0;
  dsc->e_min = INT_MAX;
  dsc->e_max = INT_MIN;
  dsc->score_ticket = 0;
}

__global__ void k_reset_attempt(DevScalars* dsc) {
  dep_sync();
  dsc->err &= ERR_RANGE | ERR_TIMEOUT | ERR_BOUNDS;  // errors of steps A1-A3 end the recovery
  dsc->epoch++;
  dsc->bounds_site = 0;
  dsc->rounds_used = 0;
  dsc->n_cand = 0;
  dsc->n_seg = 0;
  dsc->n_warp_seg = 0;
  dsc->n_block_seg = 0;
  dsc->block_ticket = 0;
  dsc->n_block = 0;
  dsc->n_big = 0;
  dsc->n_big_seg = 0;
  dsc->max_seg = 0;
  dsc->big_regs = 0;
  dsc->undecided = 0;
  dsc->radix_sel = 0;
  dsc->radix_skip = 0;
  dsc->radix_len = 0;
  dsc->n_warp_cand = 0;
  dsc->n_constrained = 0;
  dsc->n_big_chunk = 0;
  dsc->finish_left = 0;
}

// endpoints of canonical ids in the caller's vertex ids (u < v): the edge
// list holds preorder labels, vtx_of_pre maps them back
__global__ void k_endpoints(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev, int64_t m,
                            const int32_t* __restrict__ vtx_of_pre, const int32_t* __restrict__ ids, int64_t count,
                            int32_t* __restrict__ ou, int32_t* __restrict__ ov, DevScalars* dsc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = ids[i];
    if (id < 0 || id >= m) {
      atomicOr(&dsc->err, ERR_CAPACITY);
      ou[i] = ov[i] = -1;
      continue;
    }
    const int32_t a = vtx_of_pre[eu[id]], b = vtx_of_pre[ev[id]];
    ou[i] = min(a, b);
    ov[i] = max(a, b);
  }
}

}  // namespace

// status words of the single-pass scan for inputs of up to n_max elements
int ensure_scan_status(Handle& h, int64_t n_max) {
  const int64_t tiles = (std::max<int64_t>(n_max, 1) + kTile - 1) / kTile;
  if (h.scan_ctr == nullptr) {
    int st = alloc_n(h, &h.scan_ctr, 2);
    if (st) return st;
    PDG_CUDA(cudaMemsetAsync(h.scan_ctr, 0, 2 * sizeof(uint32_t), h.stream));
  }
  if (tiles <= h.scan_tiles_cap) return PDG_OK;
  device_release(h, h.scan_status);
  h.scan_status = nullptr;
  h.scan_tiles_cap = 0;
  int st = alloc_n(h, &h.scan_status, tiles);
  if (st) return st;
  PDG_CUDA(cudaMemsetAsync(h.scan_status, 0, sizeof(uint64_t) * tiles, h.stream));
  h.scan_tiles_cap = tiles;
  return PDG_OK;
}

int ensure_candidates(Handle& h, int64_t R, int c) {
  const int64_t Rmax = std::max<int64_t>(h.E_off, 1);
  R = std::min<int64_t>(std::max<int64_t>(R, 1), Rmax);
  int st;
  if (R > h.Rcap) {
    void* old[] = {h.cand_idx, h.rk[0], h.rk[1], h.rv[0], h.rv[1], h.rank_cand, h.lsort_rank, h.scan_tmp,
                   h.radix_status, h.rec_u, h.rec_v, h.rec_anc, h.rec_du, h.rec_dv, h.rec_rank,
                   h.rec_lca, h.rec_b, h.state, h.acc_flag, h.seg_begin, h.warp_seg, h.block_seg, h.big_pos, h.big_seg, h.big_chunk,
                   h.pos_x, h.seg_regs, h.seg_pref,
                   h.pmask, h.reg_slot, h.pslot, h.und_list};
    for (void* p : old) device_release(h, p);
    const int64_t tiles = (R + kTile - 1) / kTile;
    if ((st = alloc_n(h, &h.cand_idx, R)) || (st = alloc_n(h, &h.rk[0], R)) || (st = alloc_n(h, &h.rk[1], R)) ||
        (st = alloc_n(h, &h.rv[0], R)) || (st = alloc_n(h, &h.rv[1], R)) || (st = alloc_n(h, &h.rank_cand, R)) ||
        (st = alloc_n(h, &h.lsort_rank, R)) || (st = alloc_n(h, &h.scan_tmp, R + 1)) ||
        (st = alloc_n(h, &h.radix_status, (int64_t)kRadixPassesMax * 256 * tiles)) ||
        (st = alloc_n(h, &h.rec_u, R)) ||
        (st = alloc_n(h, &h.rec_v, R)) || (st = alloc_n(h, &h.rec_anc, 2 * PDG_MAX_C * R)) ||
        (st = alloc_n(h, &h.rec_du, R)) || (st = alloc_n(h, &h.rec_dv, R)) || (st = alloc_n(h, &h.rec_rank, R)) ||
        (st = alloc_n(h, &h.rec_lca, R)) || (st = alloc_n(h, &h.rec_b, R)) || (st = alloc_n(h, &h.state, R)) ||
        (st = alloc_n(h, &h.acc_flag, R)) || (st = alloc_n(h, &h.seg_begin, R + 1)) ||
        (st = alloc_n(h, &h.warp_seg, R)) || (st = alloc_n(h, &h.block_seg, R)) || (st = alloc_n(h, &h.big_pos, R)) || (st = alloc_n(h, &h.big_seg, R)) || (st = alloc_n(h, &h.big_chunk, R)) ||
        (st = alloc_n(h, &h.pos_x, R)) || (st = alloc_n(h, &h.seg_regs, R)) || (st = alloc_n(h, &h.seg_pref, R + 1)) ||
        (st = alloc_n(h, &h.pmask, R)) || (st = alloc_n(h, &h.reg_slot, 16 * R)) || (st = alloc_n(h, &h.und_list, R)) ||
        (st = alloc_n(h, &h.pslot, 32 * R))) {
      h.Rcap = 0;
      return st;
    }
    h.Rcap = R;
  }
  if ((st = ensure_scan_status(h, h.Rcap + 1))) return st;
  // pair table: twice the registrations plus 16 slots per cooperative subtask (at most R / 33 subtasks)
  return grow_tables(h, std::max<int64_t>(1024, 2 * (int64_t)(c + 1) * (c + 1) * h.Rcap + h.Rcap), 0);
}

// pair table of `slots` slots; exact entries for slots / 16 flagged pairs (or `xblocks`)
int grow_tables(Handle& h, int64_t slots, int64_t xblocks) {
  int st;
  slots = std::min<int64_t>(slots, (1ll << 32) - 1);  // slot indices are 32-bit on the device
  if (slots > h.table_cap) {
    device_release(h, h.ptab);
    device_release(h, h.flagbits);
    h.ptab = nullptr;
    h.flagbits = nullptr;
    if ((st = alloc_n(h, &h.ptab, slots)) || (st = alloc_n(h, &h.flagbits, slots / 32 + 1))) {
      h.table_cap = 0;
      return st;
    }
    h.table_cap = slots;
  }
  xblocks = std::max<int64_t>(xblocks, std::max<int64_t>(64, h.table_cap / 16));
  if (xblocks > h.xcap) {
    device_release(h, h.xtab);
    device_release(h, h.xund1);
    h.xtab = nullptr;
    h.xund1 = nullptr;
    if ((st = alloc_n(h, &h.xtab, 16 * xblocks)) || (st = alloc_n(h, &h.xund1, 16 * xblocks))) {
      h.xcap = 0;
      return st;
    }
    // all-ones undecided entries: any registration replaces them (their tags stay above every real one)
    PDG_CUDA(cudaMemsetAsync(h.xtab, 0xff, sizeof(ExactEnt) * 16 * (size_t)xblocks, h.stream));
    PDG_CUDA(cudaMemsetAsync(h.xund1, 0xff, sizeof(unsigned long long) * 16 * (size_t)xblocks, h.stream));
    h.xcap = xblocks;
  }
  return PDG_OK;
}

// Pinned host staging of the per-recovery parameters (kept alive for
// asynchronous copies).
struct HostStage {
  GraphSel* sel = nullptr;
  int64_t* k = nullptr;
  int64_t* out_ptr = nullptr;
  int32_t* gstat = nullptr;
  int64_t* gcount = nullptr;
  int32_t G = 0;
};

}  // namespace pdg

using namespace pdg;

struct pdg_sparsifier {
  Handle h;
  HostStage stage;
};

extern "C" {

void pdg_default_options(pdg_options* opt) {
  if (!opt) return;
  opt->score_mode = PDG_SCORE_STRETCH;
  opt->warp_tier_max = 32;
  opt->k_override = -1;
  opt->candidate_factor = 1.5;
  opt->max_rounds = 8;
  opt->use_graph = 0;
  opt->spin_limit = 1ll << 26;
  opt->profile = 0;
  opt->block_tier_max = kBlockTierDefault;
  opt->sort_tile_keys = 3072;
  opt->sort_one_launch = 1;
}

const char* pdg_status_string(int status) {
  switch (status) {
    case PDG_OK: return "ok";
    case PDG_UNDER_BUDGET: return "fewer than k edges survive one pass; all survivors returned";
    case PDG_E_INVALID_ARG: return "invalid argument";
    case PDG_E_NOT_SYMMETRIC: return "CSR is not symmetric (structure or weights)";
    case PDG_E_NOT_A_TREE: return "parent[] is not a spanning tree of the graph";
    case PDG_E_BAD_WEIGHT: return "edge weight not finite or outside [2^-900, 2^900]";
    case PDG_E_RANGE: return "exact root distances would overflow the 96-bit fixed point";
    case PDG_E_CAPACITY: return "output capacity too small";
    case PDG_E_OOM: return "device allocation failed";
    case PDG_E_CUDA: return "CUDA runtime error";
    case PDG_E_TIMEOUT: return "bounded device wait timed out";
    case PDG_E_NOT_CSR: return "malformed CSR (row_ptr, range, self loop, order or duplicates)";
    default: return "unknown status";
  }
}

void sparsifier_free(pdg_handle hp) {
  if (!hp) return;
  Handle& h = hp->h;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h.device);
  for (void* p : h.allocs) cudaFreeAsync(p, h.stream);
  h.allocs.clear();
  cudaStreamSynchronize(h.stream);  // pinned staging below may be reused at once
  for (cudaEvent_t e : h.ev)
    if (e) cudaEventDestroy(e);
  if (h.gexec) cudaGraphExecDestroy(h.gexec);
  if (h.ev_order) cudaEventDestroy(h.ev_order);
  if (h.ev_fork) cudaEventDestroy(h.ev_fork);
  if (h.ev_join) cudaEventDestroy(h.ev_join);
  if (h.sstream) {
    cudaStreamSynchronize(h.sstream);
    cudaStreamDestroy(h.sstream);
  }
  if (h.gstream) cudaStreamDestroy(h.gstream);
  pinned_release(h.hsc, sizeof(DevScalars));
  HostStage& s = hp->stage;
  const size_t G = (size_t)std::max(s.G, 1);
  pinned_release(s.sel, sizeof(GraphSel) * G);
  pinned_release(s.k, sizeof(int64_t) * G);
  pinned_release(s.out_ptr, sizeof(int64_t) * (G + 1));
  pinned_release(s.gstat, sizeof(int32_t) * G);
  pinned_release(s.gcount, sizeof(int64_t) * G);
  cudaGetLastError();
  cudaSetDevice(prev);
  delete hp;
}

int sparsify_batch_init(pdg_handle* out, int32_t num_graphs, const int64_t* vtx_ptr, const int64_t* row_ptr,
                        const int32_t* col, const double* w, const int32_t* parent, int mem_kind,
                        const pdg_options* opt, void* stream) {
  if (!out) return PDG_E_INVALID_ARG;
  *out = nullptr;
  if (num_graphs < 1 || !vtx_ptr || !row_ptr || !parent || (mem_kind != PDG_MEM_HOST && mem_kind != PDG_MEM_DEVICE))
    return PDG_E_INVALID_ARG;
  if (vtx_ptr[0] != 0) return PDG_E_INVALID_ARG;
  for (int32_t g = 0; g < num_graphs; g++)
    if (vtx_ptr[g + 1] <= vtx_ptr[g]) return PDG_E_INVALID_ARG;
  const int64_t n = vtx_ptr[num_graphs];
  if (n < 1 || n >= (1ll << 30)) return PDG_E_INVALID_ARG;
  pdg_sparsifier* hp = new (std::nothrow) pdg_sparsifier();
  if (!hp) return PDG_E_OOM;
  Handle& h = hp->h;
  if (opt) h.opt = *opt; else pdg_default_options(&h.opt);
  if (h.opt.warp_tier_max < 1 || h.opt.warp_tier_max > 32) h.opt.warp_tier_max = 32;
  if (h.opt.block_tier_max < 0) h.opt.block_tier_max = 0;
  if (h.opt.block_tier_max > kBlockTierMax) h.opt.block_tier_max = kBlockTierMax;
  if (h.opt.sort_tile_keys != 2048 && h.opt.sort_tile_keys != 4096) h.opt.sort_tile_keys = 3072;
  if (!(h.opt.candidate_factor >= 1.0)) h.opt.candidate_factor = 1.5;
  if (h.opt.max_rounds < 1) h.opt.max_rounds = 1;
  if (h.opt.max_rounds > 64) h.opt.max_rounds = 64;
  cudaGetDevice(&h.device);
  cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device);
  h.stream = (cudaStream_t)stream;
  if (h.opt.use_graph) {
    if (cudaStreamCreateWithFlags(&h.gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h.ev_order, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      h.opt.use_graph = 0;  // replay is an optimisation; run without it
    }
  }
  if (cudaStreamCreateWithFlags(&h.sstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (h.sstream) cudaStreamDestroy(h.sstream);
    h.sstream = nullptr;  // the tiers then run one after the other on the handle's stream
  }
  h.G = num_graphs;
  h.n = n;
  h.vtx_ptr_h.assign(vtx_ptr, vtx_ptr + num_graphs + 1);
  int st = PDG_OK;
  auto fail = [&](int code) {
    sparsifier_free(hp);
    return code;
  };
  if ((st = sort_setup()) || (st = accept_setup())) return fail(st);
  const cudaMemcpyKind kind = (mem_kind == PDG_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  // nnz
  int64_t ends[2];
  if (mem_kind == PDG_MEM_HOST) {
    ends[0] = row_ptr[0];
    ends[1] = row_ptr[n];
  } else {
    if (cudaMemcpyAsync(&ends[0], row_ptr, 8, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
        cudaMemcpyAsync(&ends[1], row_ptr + n, 8, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
        cudaStreamSynchronize(h.stream) != cudaSuccess)
      return fail(PDG_E_CUDA);
  }
  if (ends[0] != 0 || ends[1] < 0) return fail(PDG_E_NOT_CSR);
  h.nnz = ends[1];
  if (h.nnz > 0 && (!col || !w)) return fail(PDG_E_INVALID_ARG);
  if (h.nnz % 2) return fail(PDG_E_NOT_SYMMETRIC);
  h.m = h.nnz / 2;
  if (h.m >= (1ll << 31)) return fail(PDG_E_INVALID_ARG);
  if (!(h.hsc = static_cast<DevScalars*>(pinned_alloc(sizeof(DevScalars))))) return fail(PDG_E_OOM);
  if ((st = alloc_n(h, &h.dsc, 1))) return fail(st);
  if (cudaMemsetAsync(h.dsc, 0, sizeof(DevScalars), h.stream) != cudaSuccess) return fail(PDG_E_CUDA);
  if ((st = alloc_n(h, &h.row_ptr, n + 1)) || (st = alloc_n(h, &h.col, h.nnz)) || (st = alloc_n(h, &h.w, h.nnz)) ||
      (st = alloc_n(h, &h.parent, n)) || (st = alloc_n(h, &h.d_vtx_ptr, num_graphs + 1)) ||
      (st = alloc_n(h, &h.blk_a, 10240)) || (st = alloc_n(h, &h.blk_b, 2048)))
    return fail(st);
  if (cudaMemcpyAsync(h.row_ptr, row_ptr, sizeof(int64_t) * (n + 1), kind, h.stream) != cudaSuccess ||
      (h.nnz && cudaMemcpyAsync(h.col, col, sizeof(int32_t) * h.nnz, kind, h.stream) != cudaSuccess) ||
      (h.nnz && cudaMemcpyAsync(h.w, w, sizeof(double) * h.nnz, kind, h.stream) != cudaSuccess) ||
      cudaMemcpyAsync(h.parent, parent, sizeof(int32_t) * n, kind, h.stream) != cudaSuccess ||
      cudaMemcpyAsync(h.d_vtx_ptr, vtx_ptr, sizeof(int64_t) * (num_graphs + 1), cudaMemcpyHostToDevice, h.stream) !=
          cudaSuccess)
    return fail(PDG_E_CUDA);
  h.nblk = (int)std::max<int64_t>(1, std::min<int64_t>(2048, (h.m + kTile - 1) / kTile));
  if ((st = validate_graph(h, false))) return fail(st);  // acyclicity, depth and range: build_tree_layout
  // per-graph edge counts from the row offsets at the graph boundaries
  std::vector<int64_t> rp_at(num_graphs + 1);
  {
    int64_t* tmp = nullptr;
    if ((st = alloc_n(h, &tmp, num_graphs + 1))) return fail(st);
    ++h.launches;
    k_gather_rowptr<<<(num_graphs + 256) / 256, 256, 0, h.stream>>>(h.row_ptr, h.d_vtx_ptr, num_graphs, tmp);
    if (cudaMemcpyAsync(rp_at.data(), tmp, sizeof(int64_t) * (num_graphs + 1), cudaMemcpyDeviceToHost, h.stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h.stream) != cudaSuccess)
      return fail(PDG_E_CUDA);
    device_release(h, tmp);
  }
  // the graph stays resident as its canonical edge list; the CSR is dropped
  if ((st = alloc_n(h, &h.el_u, std::max<int64_t>(h.m, 1))) || (st = alloc_n(h, &h.el_v, std::max<int64_t>(h.m, 1))) ||
      (st = alloc_n(h, &h.el_w, std::max<int64_t>(h.m, 1))) || (st = build_edge_list(h)))
    return fail(st);
  device_release(h, h.row_ptr);
  device_release(h, h.col);
  device_release(h, h.w);
  h.row_ptr = nullptr;
  h.col = nullptr;
  h.w = nullptr;
  h.edge_ptr_h.assign(num_graphs + 1, 0);
  h.off_ptr_h.assign(num_graphs + 1, 0);
  for (int32_t g = 0; g < num_graphs; g++) {
    const int64_t entries = rp_at[g + 1] - rp_at[g];
    if (entries % 2) return fail(PDG_E_NOT_SYMMETRIC);
    const int64_t mg = entries / 2, ng = vtx_ptr[g + 1] - vtx_ptr[g];
    if (mg < ng - 1) return fail(PDG_E_NOT_A_TREE);
    h.edge_ptr_h[g + 1] = h.edge_ptr_h[g] + mg;
    h.off_ptr_h[g + 1] = h.off_ptr_h[g] + (mg - ng + 1);
  }
  h.E_off = h.off_ptr_h[num_graphs];
  // workspace
  const int64_t E = std::max<int64_t>(h.E_off, 1);
  if ((st = alloc_n(h, &h.d_edge_ptr, num_graphs + 1)) || (st = alloc_n(h, &h.d_off_ptr, num_graphs + 1)) ||
      (st = alloc_n(h, &h.off_u, E)) || (st = alloc_n(h, &h.off_v, E)) || (st = alloc_n(h, &h.off_id, E)) ||
      (st = alloc_n(h, &h.off_w, E)) || (st = alloc_n(h, &h.rtree, n)) ||
      (st = alloc_n(h, &h.key, E)) || (st = alloc_n(h, &h.lca, E)) ||
      (st = alloc_n(h, &h.hist, (int64_t)num_graphs * kSelBins)) || (st = alloc_n(h, &h.sel, num_graphs)) ||
      (st = alloc_n(h, &h.d_cand_ptr, num_graphs + 1)) || (st = alloc_n(h, &h.d_graph_tmp, num_graphs + 1)) ||
      (st = alloc_n(h, &h.gstat, num_graphs)) || (st = alloc_n(h, &h.gcount, num_graphs)) ||
      (st = alloc_n(h, &h.d_k, num_graphs)) || (st = alloc_n(h, &h.d_out_ptr, num_graphs + 1)) ||
      (st = alloc_n(h, &h.radix_dtot, 256)) || (st = alloc_n(h, &h.radix_hist, kRadixHistWords)) ||
      (st = alloc_n(h, &h.radix_counters, 2 * kRadixPassesMax)) ||
      (st = ensure_scan_status(h, std::max<int64_t>(std::max<int64_t>(n, num_graphs), E) + 1)))
    return fail(st);
  // the tree's layout: preorder labels, Euler tour, the relabelled edge list and parents
  if ((st = build_tree_layout(h)) || (st = tree_scan_workspace(h)) || (st = classify_layout(h))) return fail(st);
  HostStage& s = hp->stage;
  s.G = num_graphs;
  s.sel = static_cast<GraphSel*>(pinned_alloc(sizeof(GraphSel) * num_graphs));
  s.k = static_cast<int64_t*>(pinned_alloc(sizeof(int64_t) * num_graphs));
  s.out_ptr = static_cast<int64_t*>(pinned_alloc(sizeof(int64_t) * (num_graphs + 1)));
  s.gstat = static_cast<int32_t*>(pinned_alloc(sizeof(int32_t) * num_graphs));
  s.gcount = static_cast<int64_t*>(pinned_alloc(sizeof(int64_t) * num_graphs));
  if (!s.sel || !s.k || !s.out_ptr || !s.gstat || !s.gcount) return fail(PDG_E_OOM);
  if (cudaMemcpyAsync(h.d_edge_ptr, h.edge_ptr_h.data(), sizeof(int64_t) * (num_graphs + 1), cudaMemcpyHostToDevice,
                      h.stream) != cudaSuccess ||
      cudaMemcpyAsync(h.d_off_ptr, h.off_ptr_h.data(), sizeof(int64_t) * (num_graphs + 1), cudaMemcpyHostToDevice,
                      h.stream) != cudaSuccess ||
      cudaMemsetAsync(h.hist, 0, sizeof(uint32_t) * (size_t)num_graphs * kSelBins, h.stream) != cudaSuccess ||
      cudaMemsetAsync(h.radix_dtot, 0, sizeof(uint32_t) * 256, h.stream) != cudaSuccess ||
      cudaMemsetAsync(h.radix_hist, 0, sizeof(uint32_t) * kRadixHistWords, h.stream) != cudaSuccess ||
      cudaStreamSynchronize(h.stream) != cudaSuccess)
    return fail(PDG_E_CUDA);
  h.want_h.assign(num_graphs, 0);
  h.want_mem.assign(num_graphs, 0);
  h.k_mem.assign(num_graphs, -1);
  *out = hp;
  return PDG_OK;
}

int pdg_spanning_tree(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, int mem_kind,
                      int tree_kind, int32_t* parent_out, int out_mem_kind, void* stream) {
  if (n < 1 || n >= (1ll << 30) || !row_ptr || !parent_out ||
      (mem_kind != PDG_MEM_HOST && mem_kind != PDG_MEM_DEVICE) ||
      (out_mem_kind != PDG_MEM_HOST && out_mem_kind != PDG_MEM_DEVICE) ||
      (tree_kind != PDG_TREE_MAX_WEIGHT && tree_kind != PDG_TREE_FEGRASS))
    return PDG_E_INVALID_ARG;
  pdg_sparsifier* hp = new (std::nothrow) pdg_sparsifier();
  if (!hp) return PDG_E_OOM;
  Handle& h = hp->h;
  pdg_default_options(&h.opt);
  cudaGetDevice(&h.device);
  cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device);
  h.stream = (cudaStream_t)stream;
  h.G = 1;
  h.n = n;
  h.vtx_ptr_h = {0, n};
  auto fail = [&](int code) {
    sparsifier_free(hp);
    return code;
  };
  const cudaMemcpyKind kind = (mem_kind == PDG_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int64_t ends[2];
  if (mem_kind == PDG_MEM_HOST) {
    ends[0] = row_ptr[0];
    ends[1] = row_ptr[n];
  } else if (cudaMemcpyAsync(&ends[0], row_ptr, 8, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
             cudaMemcpyAsync(&ends[1], row_ptr + n, 8, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
             cudaStreamSynchronize(h.stream) != cudaSuccess) {
    return fail(PDG_E_CUDA);
  }
  if (ends[0] != 0 || ends[1] < 0) return fail(PDG_E_NOT_CSR);
  h.nnz = ends[1];
  if (h.nnz > 0 && (!col || !w)) return fail(PDG_E_INVALID_ARG);
  if (h.nnz % 2) return fail(PDG_E_NOT_SYMMETRIC);
  h.m = h.nnz / 2;
  if (h.m >= (1ll << 31)) return fail(PDG_E_INVALID_ARG);
  int st = PDG_OK;
  const int64_t vp[2] = {0, n};
  if (!(h.hsc = static_cast<DevScalars*>(pinned_alloc(sizeof(DevScalars))))) return fail(PDG_E_OOM);
  if ((st = alloc_n(h, &h.dsc, 1)) || (st = alloc_n(h, &h.row_ptr, n + 1)) || (st = alloc_n(h, &h.col, h.nnz)) ||
      (st = alloc_n(h, &h.w, h.nnz)) || (st = alloc_n(h, &h.parent, n)) || (st = alloc_n(h, &h.d_vtx_ptr, 2)) ||
      (st = alloc_n(h, &h.blk_a, 10240)) || (st = alloc_n(h, &h.blk_b, 2048)))
    return fail(st);
  if (cudaMemcpyAsync(h.row_ptr, row_ptr, sizeof(int64_t) * (n + 1), kind, h.stream) != cudaSuccess ||
      (h.nnz && cudaMemcpyAsync(h.col, col, sizeof(int32_t) * h.nnz, kind, h.stream) != cudaSuccess) ||
      (h.nnz && cudaMemcpyAsync(h.w, w, sizeof(double) * h.nnz, kind, h.stream) != cudaSuccess) ||
      cudaMemcpyAsync(h.d_vtx_ptr, vp, sizeof(vp), cudaMemcpyHostToDevice, h.stream) != cudaSuccess)
    return fail(PDG_E_CUDA);
  if ((st = validate_csr(h))) return fail(st);
  if ((st = alloc_n(h, &h.el_u, std::max<int64_t>(h.m, 1))) || (st = alloc_n(h, &h.el_v, std::max<int64_t>(h.m, 1))) ||
      (st = alloc_n(h, &h.el_w, std::max<int64_t>(h.m, 1))) || (st = build_edge_list(h)))
    return fail(st);
  int32_t* pdev = (out_mem_kind == PDG_MEM_DEVICE) ? parent_out : h.parent;
  if ((st = spanning_tree(h, tree_kind, pdev))) return fail(st);
  if (out_mem_kind == PDG_MEM_HOST &&
      cudaMemcpyAsync(parent_out, pdev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess)
    return fail(PDG_E_CUDA);
  if (cudaStreamSynchronize(h.stream) != cudaSuccess) return fail(PDG_E_CUDA);
  sparsifier_free(hp);
  return PDG_OK;
}

}  // extern "C"

// pdg_pcg_quality and pdg_pcg_trace: hist and z0 are nullable host outputs
static int pcg_entry(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                     const int32_t* edge_ids, int64_t n_edges, const double* b, double tol, int32_t max_iter,
                     int mem_kind, int32_t* out_iters, double* out_relres, double* hist, double* z0, void* stream) {
  if (n < 2 || n >= (1ll << 30) || !row_ptr || !parent || !b || !out_iters || !out_relres || n_edges < 0 ||
      n_edges > kPcgMaxEdges || (n_edges > 0 && !edge_ids) || !(tol > 0) || max_iter < 1 ||
      (mem_kind != PDG_MEM_HOST && mem_kind != PDG_MEM_DEVICE))
    return PDG_E_INVALID_ARG;
  pdg_sparsifier* hp = new (std::nothrow) pdg_sparsifier();
  if (!hp) return PDG_E_OOM;
  Handle& h = hp->h;
  pdg_default_options(&h.opt);
  cudaGetDevice(&h.device);
  cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device);
  h.stream = (cudaStream_t)stream;
  h.G = 1;
  h.n = n;
  h.vtx_ptr_h = {0, n};
  auto fail = [&](int code) {
    sparsifier_free(hp);
    return code;
  };
  const cudaMemcpyKind kind = (mem_kind == PDG_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int64_t ends[2];
  if (mem_kind == PDG_MEM_HOST) {
    ends[0] = row_ptr[0];
    ends[1] = row_ptr[n];
  } else if (cudaMemcpyAsync(&ends[0], row_ptr, 8, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
             cudaMemcpyAsync(&ends[1], row_ptr + n, 8, cudaMemcpyDeviceToHost, h.stream) != cudaSuccess ||
             cudaStreamSynchronize(h.stream) != cudaSuccess) {
    return fail(PDG_E_CUDA);
  }
  if (ends[0] != 0 || ends[1] < 0) return fail(PDG_E_NOT_CSR);
  h.nnz = ends[1];
  if (h.nnz > 0 && (!col || !w)) return fail(PDG_E_INVALID_ARG);
  if (h.nnz % 2) return fail(PDG_E_NOT_SYMMETRIC);
  h.m = h.nnz / 2;
  if (h.m >= (1ll << 31)) return fail(PDG_E_INVALID_ARG);
  int st = PDG_OK;
  const int64_t vp[2] = {0, n};
  int32_t* d_ids = nullptr;
  double* d_b = nullptr;
  if (!(h.hsc = static_cast<DevScalars*>(pinned_alloc(sizeof(DevScalars))))) return fail(PDG_E_OOM);
  if ((st = alloc_n(h, &h.dsc, 1)) || (st = alloc_n(h, &h.row_ptr, n + 1)) || (st = alloc_n(h, &h.col, h.nnz)) ||
      (st = alloc_n(h, &h.w, h.nnz)) || (st = alloc_n(h, &h.parent, n)) || (st = alloc_n(h, &h.d_vtx_ptr, 2)) ||
      (st = alloc_n(h, &h.blk_a, 10240)) || (st = alloc_n(h, &h.blk_b, 2048)) ||
      (st = alloc_n(h, &d_ids, std::max<int64_t>(n_edges, 1))) || (st = alloc_n(h, &d_b, n)))
    return fail(st);
  if (cudaMemcpyAsync(h.row_ptr, row_ptr, sizeof(int64_t) * (n + 1), kind, h.stream) != cudaSuccess ||
      (h.nnz && cudaMemcpyAsync(h.col, col, sizeof(int32_t) * h.nnz, kind, h.stream) != cudaSuccess) ||
      (h.nnz && cudaMemcpyAsync(h.w, w, sizeof(double) * h.nnz, kind, h.stream) != cudaSuccess) ||
      cudaMemcpyAsync(h.parent, parent, sizeof(int32_t) * n, kind, h.stream) != cudaSuccess ||
      (n_edges && cudaMemcpyAsync(d_ids, edge_ids, sizeof(int32_t) * n_edges, kind, h.stream) != cudaSuccess) ||
      cudaMemcpyAsync(d_b, b, sizeof(double) * n, kind, h.stream) != cudaSuccess ||
      cudaMemcpyAsync(h.d_vtx_ptr, vp, sizeof(vp), cudaMemcpyHostToDevice, h.stream) != cudaSuccess)
    return fail(PDG_E_CUDA);
  if ((st = validate_graph(h, true))) return fail(st);
  if ((st = alloc_n(h, &h.el_u, std::max<int64_t>(h.m, 1))) || (st = alloc_n(h, &h.el_v, std::max<int64_t>(h.m, 1))) ||
      (st = alloc_n(h, &h.el_w, std::max<int64_t>(h.m, 1))) || (st = build_edge_list(h)))
    return fail(st);
  int32_t it = 0;
  double rel = 0.0;
  if ((st = pcg_quality(h, d_ids, n_edges, d_b, tol, max_iter, &it, &rel, hist, z0))) return fail(st);
  *out_iters = it;
  *out_relres = rel;
  sparsifier_free(hp);
  return PDG_OK;
}

extern "C" {

int pdg_pcg_quality(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                    const int32_t* edge_ids, int64_t n_edges, const double* b, double tol, int32_t max_iter,
                    int mem_kind, int32_t* out_iters, double* out_relres, void* stream) {
  return pcg_entry(n, row_ptr, col, w, parent, edge_ids, n_edges, b, tol, max_iter, mem_kind, out_iters, out_relres,
                   nullptr, nullptr, stream);
}

int pdg_pcg_trace(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                  const int32_t* edge_ids, int64_t n_edges, const double* b, double tol, int32_t max_iter,
                  int mem_kind, int32_t* out_iters, double* out_relres, double* out_history, double* out_precond_b,
                  void* stream) {
  if (!out_history || !out_precond_b) return PDG_E_INVALID_ARG;
  return pcg_entry(n, row_ptr, col, w, parent, edge_ids, n_edges, b, tol, max_iter, mem_kind, out_iters, out_relres,
                   out_history, out_precond_b, stream);
}

int sparsify_init(pdg_handle* out, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w,
                  const int32_t* parent, int mem_kind, const pdg_options* opt, void* stream) {
  if (!out) return PDG_E_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || n >= (1ll << 30)) return PDG_E_INVALID_ARG;
  const int64_t vp[2] = {0, n};
  return sparsify_batch_init(out, 1, vp, row_ptr, col, w, parent, mem_kind, opt, stream);
}

}  // extern "C"

namespace pdg {

// The recovery driver shared by recover_offtree and recover_offtree_batch.
// Diagnostics for a failed index check: where position p sits in the
// segment and tier lists of the attempt that failed.
static void debug_position(Handle& h, int64_t p) {
  const int64_t N = h.hsc->n_cand, S = h.hsc->n_seg, NB = h.hsc->n_big, NBS = h.hsc->n_big_seg;
  std::vector<int32_t> seg(S + 1), bpos(NB), bseg(NBS);
  std::vector<uint8_t> st(N);
  cudaMemcpy(seg.data(), h.seg_begin, sizeof(int32_t) * (S + 1), cudaMemcpyDeviceToHost);
  cudaMemcpy(bpos.data(), h.big_pos, sizeof(int32_t) * NB, cudaMemcpyDeviceToHost);
  cudaMemcpy(bseg.data(), h.big_seg, sizeof(int32_t) * NBS, cudaMemcpyDeviceToHost);
  cudaMemcpy(st.data(), h.state, N, cudaMemcpyDeviceToHost);
  int64_t q = std::upper_bound(seg.begin(), seg.end(), (int32_t)p) - seg.begin() - 1;
  bool mono = true;
  for (int64_t i = 0; i < S; i++)
    if (seg[i + 1] <= seg[i]) mono = false;
  const bool in_bpos = std::find(bpos.begin(), bpos.end(), (int32_t)p) != bpos.end();
  const bool seg_big = std::find(bseg.begin(), bseg.end(), (int32_t)q) != bseg.end();
  std::vector<char> seen(N, 0);
  int64_t dup = 0;
  for (int32_t v : bpos)
    if (v >= 0 && v < N) dup += seen[v]++ ? 1 : 0;
  int64_t big_total = 0;
  for (int32_t x : bseg)
    if (x >= 0 && x < S) big_total += seg[x + 1] - seg[x];
  fprintf(stderr, "pdgrass debug: p %lld N %lld n_seg %lld mono %d seg %lld [%d, %d) in_big_pos %d seg_in_big_seg %d "
                  "state %d n_big %lld sum_big_seg_sizes %lld dups %lld seg_end %d\n",
          (long long)p, (long long)N, (long long)S, (int)mono, (long long)q, seg[q], seg[q + 1], (int)in_bpos,
          (int)seg_big, (int)st[p], (long long)NB, (long long)big_total, (long long)dup, seg[S]);
}

static int run_recovery(pdg_sparsifier* hp, const double* alpha, int32_t c, const int64_t* user_out_ptr,
                        int32_t* out_ids, double* out_scores, int out_mem_kind, int64_t* out_count,
                        int32_t* graph_status) {
  Handle& h = hp->h;
  HostStage& s = hp->stage;
  const int32_t G = h.G;
  if (c < 0 || c > PDG_MAX_C || (out_mem_kind != PDG_MEM_HOST && out_mem_kind != PDG_MEM_DEVICE))
    return PDG_E_INVALID_ARG;
  int prev_dev = 0;
  cudaGetDevice(&prev_dev);
  if (prev_dev != h.device) cudaSetDevice(h.device);
  struct Restore {
    int d, cur;
    ~Restore() {
      if (d != cur) cudaSetDevice(d);
    }
  } restore{prev_dev, h.device};
  // budgets and initial prefix sizes
  std::vector<int64_t> kg(G), eoff(G);
  int64_t total_k = 0;
  for (int32_t g = 0; g < G; g++) {
    const int64_t ng = h.vtx_ptr_h[g + 1] - h.vtx_ptr_h[g];
    eoff[g] = h.off_ptr_h[g + 1] - h.off_ptr_h[g];
    int64_t k;
    if (h.opt.k_override >= 0) {
      k = h.opt.k_override;
    } else {
      const double a = alpha[g];
      if (!(a >= 0.0) || !std::isfinite(a)) return PDG_E_INVALID_ARG;
      const double kd = std::floor(a * (double)ng);
      k = (kd >= 9.0e18) ? INT64_MAX / 4 : (int64_t)kd;
    }
    kg[g] = k;
    const int64_t take = std::min(k, eoff[g]);
    if (user_out_ptr[g + 1] - user_out_ptr[g] < take) return PDG_E_CAPACITY;
    total_k += take;
    int64_t want = (int64_t)std::ceil((double)k * h.opt.candidate_factor) + 32;
    if (want < k) want = k;
    if (h.k_mem[g] == k && h.c_mem == c && h.mode_mem == h.opt.score_mode) want = std::max(want, h.want_mem[g]);
    h.want_h[g] = std::min(want, eoff[g]);
    s.k[g] = k;
    s.out_ptr[g] = user_out_ptr[g];
  }
  s.out_ptr[G] = user_out_ptr[G];
  const int64_t out_total = user_out_ptr[G];
  // output staging (device) when the caller's buffers are host memory
  int32_t* dev_ids = out_ids;
  double* dev_scores = out_scores;
  int st;
  if (out_mem_kind == PDG_MEM_HOST) {
    if (out_total > h.out_cap) {
      device_release(h, h.out_ids);
      device_release(h, h.out_scores);
      h.out_ids = nullptr;
      h.out_scores = nullptr;
      h.out_cap = 0;
      if ((st = alloc_n(h, &h.out_ids, out_total)) || (st = alloc_n(h, &h.out_scores, out_total))) return st;
      h.out_cap = out_total;
    }
    dev_ids = h.out_ids;
    dev_scores = out_scores ? h.out_scores : nullptr;
  }
  h.launches = 0;
  DepScope dep_scope(h);  // kernels of the recovery may launch as programmatic dependents
  const bool prof = h.opt.profile != 0;
  if (prof && !h.ev[0])
    for (cudaEvent_t& e : h.ev) PDG_CUDA(cudaEventCreate(&e));
  bool capturing = false;
  auto mark = [&](int i) {
    if (prof && !capturing) {
      cudaEventRecord(h.ev[i], h.stream);
      stream_op(h);  // the steps timed apart do not overlap
    }
  };
  float acc_ms[8] = {0};
  // Enqueue one attempt on h.stream: steps A1-A3 (first attempt only; they
  // do not depend on the prefix), then A4-A7 and the read-back of the status.
  bool any_select_cur = false;
  auto enqueue = [&](bool first) -> int {
    int e;
    stream_op(h);  // the previous attempt ended with copies
    // a single graph's first selection histogram is taken by the scoring kernel itself
    h.fuse_hist = first && G == 1 && any_select_cur;
    if (first) {
      PDG_CUDA(cudaMemcpyAsync(h.d_k, s.k, sizeof(int64_t) * G, cudaMemcpyHostToDevice, h.stream));
      PDG_CUDA(cudaMemcpyAsync(h.d_out_ptr, s.out_ptr, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, h.stream));
      mark(0);
      ++h.launches;
      launch_k(h, k_reset_recover, 1, 1, 0, h.dsc);
      if ((e = step_classify(h))) return e;
      mark(1);
      if ((e = step_tree(h))) return e;
      mark(2);
      if ((e = step_score(h, h.opt.score_mode))) return e;
      mark(3);
    }
    ++h.launches;
    launch_k(h, k_reset_attempt, 1, 1, 0, h.dsc);
    PDG_CUDA(cudaMemcpyAsync(h.sel, s.sel, sizeof(GraphSel) * G, cudaMemcpyHostToDevice, h.stream));
    stream_op(h);
    mark(4);
    if ((e = step_select(h))) return e;
    mark(5);
    if ((e = step_sort(h))) return e;
    mark(6);
    if ((e = step_accept(h, c))) return e;
    mark(7);
    if ((e = step_budget(h, dev_ids, dev_scores))) return e;
    mark(8);
    PDG_CUDA(cudaMemcpyAsync(h.hsc, h.dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h.stream));
    PDG_CUDA(cudaMemcpyAsync(s.gstat, h.gstat, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, h.stream));
    PDG_CUDA(cudaMemcpyAsync(s.gcount, h.gcount, sizeof(int64_t) * G, cudaMemcpyDeviceToHost, h.stream));
    return PDG_OK;
  };
  int attempts = 0, retries = 0;
  bool first = true;
  for (;;) {
    if (++attempts > 40) return PDG_E_CUDA;
    // every attempt advances the device epoch that tags the cooperative tier's undecided entries; long before
    // the tags would wrap, the entries are refilled and the epoch restarts
    if (++h.epochs >= (1u << 24)) {
      if (h.xtab) {
        PDG_CUDA(cudaMemsetAsync(h.xtab, 0xff, sizeof(ExactEnt) * 16 * (size_t)h.xcap, h.stream));
        PDG_CUDA(cudaMemsetAsync(h.xund1, 0xff, sizeof(unsigned long long) * 16 * (size_t)h.xcap, h.stream));
      }
      PDG_CUDA(cudaMemsetAsync(&h.dsc->epoch, 0, sizeof(uint32_t), h.stream));
      h.epochs = 1;
    }
    int64_t need = 0;
    bool any_select = false;
    for (int32_t g = 0; g < G; g++) {
      GraphSel& gs = s.sel[g];
      std::memset(&gs, 0, sizeof(gs));
      gs.want = h.want_h[g];
      gs.take_all = (h.want_h[g] >= eoff[g]) ? 1 : 0;
      need += gs.take_all ? eoff[g] : h.want_h[g];
      if (!gs.take_all) any_select = true;
    }
    any_select_cur = any_select;
    if ((st = ensure_candidates(h, std::max<int64_t>(h.Rcap, need + need / 4 + 4096), c))) return st;
    // the launch sequence a CUDA graph bakes in
    const GraphKey key{c, h.opt.score_mode, any_select ? 1 : 0, coop_rounds(h, c), h.Rcap, h.table_cap, h.xcap,
                       (void*)dev_ids, (void*)dev_scores, out_total};
    bool replayed = false;
    if (first && h.opt.use_graph && h.gexec && key == h.gkey) {
      // replay on the private stream, ordered after the caller's stream
      PDG_CUDA(cudaEventRecord(h.ev_order, h.stream));
      PDG_CUDA(cudaStreamWaitEvent(h.gstream, h.ev_order, 0));
      PDG_CUDA(cudaGraphLaunch(h.gexec, h.gstream));
      PDG_CUDA(cudaStreamSynchronize(h.gstream));
      h.launches = h.glaunches;
      replayed = true;
    } else {
      if ((st = enqueue(first))) return st;
      PDG_CUDA(cudaStreamSynchronize(h.stream));
    }
    if (prof && !replayed) {
      float t;
      for (int i = 0; i < 4; i++) {
        cudaEventElapsedTime(&t, h.ev[4 + i], h.ev[5 + i]);
        acc_ms[3 + i] += t;
      }
      if (first)
        for (int i = 0; i < 3; i++) cudaEventElapsedTime(&acc_ms[i], h.ev[i], h.ev[i + 1]);
    }
    const int err = h.hsc->err;
    if (getenv("PDG_DEBUG_ATTEMPTS"))
      fprintf(stderr, "pdgrass: attempt %d err %d n_cand %lld n_big %lld n_big_seg %lld big_regs %lld table_cap %lld "
                      "xcap %lld Rcap %lld\n", attempts, err, (long long)h.hsc->n_cand, (long long)h.hsc->n_big,
              (long long)h.hsc->n_big_seg, (long long)h.hsc->big_regs, (long long)h.table_cap, (long long)h.xcap,
              (long long)h.Rcap);
    if (err & ERR_RANGE) return PDG_E_RANGE;
    if (err & ERR_TIMEOUT) return PDG_E_TIMEOUT;
    if (err & ERR_TABLE) {
      // pair table too small for the registrations, or too few exact blocks
      const int64_t slots = std::max<int64_t>(h.table_cap, 2 * h.hsc->big_regs + 16 * h.hsc->n_big_seg + 1024);
      if ((st = grow_tables(h, slots, 4 * h.xcap))) return st;
      continue;
    }
    if (err & ERR_BOUNDS) {  // an internal index check failed (the access was skipped)
      h.stats[11] = h.hsc->bounds_site;
      if (getenv("PDG_DEBUG_BOUNDS"))
        fprintf(stderr, "pdgrass: bounds check %d failed (round %d, pos*64+bit %lld, value %lld; n_big %lld, "
                        "constrained %lld, rounds %d, attempt %d)\n", h.hsc->bounds_site, h.hsc->bounds_where,
                (long long)h.hsc->bounds_pos, (long long)h.hsc->bounds_val, (long long)h.hsc->n_big,
                (long long)h.hsc->n_constrained, h.hsc->rounds_used, attempts);
      if (getenv("PDG_DEBUG_BOUNDS") && h.hsc->bounds_pos >= 0) debug_position(h, h.hsc->bounds_pos / 64);
      return PDG_E_CUDA;
    }
    if (err & ERR_CAPACITY) {
      const int64_t wanted = h.hsc->n_cand_wanted;
      if (wanted <= h.Rcap) return PDG_E_CUDA;  // inconsistent selection
      if ((st = ensure_candidates(h, wanted + wanted / 8 + 4096, c))) return st;
      continue;
    }
    if (err) return PDG_E_CUDA;
    bool again = false;
    for (int32_t g = 0; g < G; g++)
      if (s.gstat[g] == G_RETRY) {
        h.want_h[g] = std::min(eoff[g], std::max<int64_t>(h.want_h[g] * 4, 64));
        again = true;
      }
    if (!again) {
      for (int32_t g = 0; g < G; g++) {
        h.want_mem[g] = h.want_h[g];
        h.k_mem[g] = kg[g];
      }
      h.c_mem = c;
      h.mode_mem = h.opt.score_mode;
      h.rounds_mem = h.hsc->rounds_used + (h.hsc->finish_left > 0 ? 1 : 0);
      if (first && !replayed && h.opt.use_graph && attempts == 1) {
        // this call needed one attempt: capture it for replay by later calls
        const cudaStream_t user = h.stream;
        const int64_t launched = h.launches;
        h.stream = h.gstream;
        capturing = true;
        h.launches = 0;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(h.gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          const int cst = enqueue(true);
          const cudaError_t ce = cudaStreamEndCapture(h.gstream, &graph);
          if (cst == PDG_OK && ce == cudaSuccess && graph) {
            if (h.gexec) cudaGraphExecDestroy(h.gexec);
            h.gexec = nullptr;
            if (cudaGraphInstantiate(&h.gexec, graph, 0) == cudaSuccess) {
              h.gkey = key;
              h.gkey.rounds = coop_rounds(h, c);  // the capture already used the remembered round count
              h.glaunches = h.launches;
            } else {
              h.gexec = nullptr;
            }
          }
          if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();  // a failed capture only disables replay
        capturing = false;
        h.stream = user;
        h.launches = launched;
      }
      break;
    }
    first = false;
    retries++;
  }
  if (prof) {
    float total = 0;
    for (int i = 0; i < 7; i++) total += acc_ms[i];
    acc_ms[7] = total;
    for (int i = 0; i < 8; i++) h.timings[i] = acc_ms[i];
  }
  // statistics of the last attempt
  h.stats[0] = h.hsc->n_cand;
  h.stats[1] = h.hsc->n_seg;
  h.stats[2] = h.hsc->max_seg;
  h.stats[3] = h.hsc->n_cand - h.hsc->n_big;
  h.stats[4] = h.hsc->n_big;
  h.stats[5] = h.hsc->rounds_used;
  h.stats[6] = retries;
  h.stats[7] = attempts;
  h.stats[8] = h.launches;
  h.stats[9] = h.hsc->n_constrained;
  h.stats[10] = h.hsc->big_regs;
  int result = PDG_OK;
  for (int32_t g = 0; g < G; g++) {
    out_count[g] = s.gcount[g];
    const int gst = (s.gstat[g] == G_UNDER) ? PDG_UNDER_BUDGET : PDG_OK;
    if (graph_status) graph_status[g] = gst;
    if (gst == PDG_UNDER_BUDGET) result = PDG_UNDER_BUDGET;
  }
  if (out_mem_kind == PDG_MEM_HOST) {
    const int64_t copy = (G == 1) ? out_count[0] : out_total;
    if (copy > 0) {
      PDG_CUDA(cudaMemcpyAsync(out_ids, h.out_ids, sizeof(int32_t) * copy, cudaMemcpyDeviceToHost, h.stream));
      if (out_scores)
        PDG_CUDA(cudaMemcpyAsync(out_scores, h.out_scores, sizeof(double) * copy, cudaMemcpyDeviceToHost, h.stream));
    }
    PDG_CUDA(cudaStreamSynchronize(h.stream));
  }
  return result;
}

}  // namespace pdg

extern "C" {

int recover_offtree(pdg_handle hp, double alpha, int32_t c, int32_t* out_edge_ids, int64_t out_capacity,
                    int64_t* out_count, double* out_scores, int out_mem_kind) {
  if (!hp || !out_count || out_capacity < 0 || (out_capacity > 0 && !out_edge_ids)) return PDG_E_INVALID_ARG;
  if (hp->h.G != 1) return PDG_E_INVALID_ARG;
  *out_count = 0;
  const int64_t op[2] = {0, out_capacity};
  return run_recovery(hp, &alpha, c, op, out_edge_ids, out_scores, out_mem_kind, out_count, nullptr);
}

int recover_offtree_batch(pdg_handle hp, const double* alpha, int32_t c, const int64_t* out_ptr, int32_t* out_edge_ids,
                          int64_t* out_count, double* out_scores, int32_t* graph_status, int out_mem_kind) {
  if (!hp || !alpha || !out_ptr || !out_count) return PDG_E_INVALID_ARG;
  const int32_t G = hp->h.G;
  if (out_ptr[0] != 0) return PDG_E_INVALID_ARG;
  for (int32_t g = 0; g < G; g++)
    if (out_ptr[g + 1] < out_ptr[g]) return PDG_E_INVALID_ARG;
  if (out_ptr[G] > 0 && !out_edge_ids) return PDG_E_INVALID_ARG;
  for (int32_t g = 0; g < G; g++) out_count[g] = 0;
  return run_recovery(hp, alpha, c, out_ptr, out_edge_ids, out_scores, out_mem_kind, out_count, graph_status);
}

int pdg_handle_info(pdg_handle hp, int64_t* n, int64_t* m, int64_t* n_offtree, int32_t* num_graphs,
                    int64_t* max_depth, int64_t* device_bytes) {
  if (!hp) return PDG_E_INVALID_ARG;
  Handle& h = hp->h;
  if (n) *n = h.n;
  if (m) *m = h.m;
  if (n_offtree) *n_offtree = h.E_off;
  if (num_graphs) *num_graphs = h.G;
  if (max_depth) *max_depth = h.max_depth;
  if (device_bytes) *device_bytes = (int64_t)h.device_bytes;
  return PDG_OK;
}

int pdg_last_timings(pdg_handle hp, float* ms) {
  if (!hp || !ms) return PDG_E_INVALID_ARG;
  for (int i = 0; i < 8; i++) ms[i] = hp->h.timings[i];
  return PDG_OK;
}

int pdg_last_stats(pdg_handle hp, int64_t* stats) {
  if (!hp || !stats) return PDG_E_INVALID_ARG;
  for (int i = 0; i < 12; i++) stats[i] = hp->h.stats[i];
  return PDG_OK;
}

int pdg_edge_endpoints(pdg_handle hp, const int32_t* ids, int64_t count, int32_t* u, int32_t* v, int mem_kind) {
  if (!hp || count < 0 || (count > 0 && (!ids || !u || !v)) || (mem_kind != PDG_MEM_HOST && mem_kind != PDG_MEM_DEVICE))
    return PDG_E_INVALID_ARG;
  if (count == 0) return PDG_OK;
  Handle& h = hp->h;
  int st;
  const int32_t* d_ids = ids;
  int32_t* d_u = u;
  int32_t* d_v = v;
  int32_t* tmp = nullptr;
  if (mem_kind == PDG_MEM_HOST) {
    if ((st = alloc_n(h, &tmp, 3 * count))) return st;
    PDG_CUDA(cudaMemcpyAsync(tmp, ids, sizeof(int32_t) * count, cudaMemcpyHostToDevice, h.stream));
    d_ids = tmp;
    d_u = tmp + count;
    d_v = tmp + 2 * count;
  }
  ++h.launches;
  k_reset_attempt<<<1, 1, 0, h.stream>>>(h.dsc);
  ++h.launches;
  k_endpoints<<<grid_for(h, count), kBlock, 0, h.stream>>>(h.el_u, h.el_v, h.m, h.vtx_of_pre, d_ids, count, d_u,
                                                            d_v, h.dsc);
  if (mem_kind == PDG_MEM_HOST) {
    PDG_CUDA(cudaMemcpyAsync(u, d_u, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, h.stream));
    PDG_CUDA(cudaMemcpyAsync(v, d_v, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, h.stream));
  }
  PDG_CUDA(cudaMemcpyAsync(h.hsc, h.dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h.stream));
  PDG_CUDA(cudaStreamSynchronize(h.stream));
  if (tmp) device_release(h, tmp);
  return (h.hsc->err & ERR_CAPACITY) ? PDG_E_INVALID_ARG : PDG_OK;
}

}  // extern "C"
