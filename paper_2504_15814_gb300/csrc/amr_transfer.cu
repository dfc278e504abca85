// C ABI of the transfer library: plan lifecycle and kernel launches.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "builder.hpp"
#include "adjoint_kernels.cuh"
#include "csr_kernels.cuh"
#include "transfer_kernels.cuh"
#include "restrict_kernels.cuh"
#include "diagonal_kernels.cuh"
#include "fixed_kernels.cuh"
#include "fixed_adjoint.cuh"

namespace {

thread_local std::string g_cuda_error = "no CUDA error";

amr_status cuda_fail(cudaError_t e, const char* where) {
  g_cuda_error = std::string(where) + ": " + cudaGetErrorString(e);
  return AMR_ERR_CUDA;
}

#define AMR_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

constexpr int kThreads = 256;           // default CTA size
constexpr int kSmemBudget = 64 * 1024;  // default shared memory budget per interpolation tile

std::mutex g_tables_mutex;
std::vector<int> g_tables_ready;  // per device

amr_status upload_tables(int device) {
  std::lock_guard<std::mutex> lock(g_tables_mutex);
  if ((int)g_tables_ready.size() <= device) g_tables_ready.resize(device + 1, 0);
  if (g_tables_ready[device]) return AMR_OK;
  const amr::Tables& t = amr::tables();
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_wt_interp, t.wt_interp, sizeof t.wt_interp));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_wt_restrict, t.wt_restrict, sizeof t.wt_restrict));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_wt_interp_f, t.wt_interp_f, sizeof t.wt_interp_f));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_wt_restrict_f, t.wt_restrict_f, sizeof t.wt_restrict_f));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_ls, t.ls, sizeof t.ls));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_ls_f, t.ls_f, sizeof t.ls_f));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_rw, t.rw, sizeof t.rw));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_rw_hi, t.rw_hi, sizeof t.rw_hi));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_rw_lo, t.rw_lo, sizeof t.rw_lo));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_fxw, t.fxw, sizeof t.fxw));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_rwx, t.rwx, sizeof t.rwx));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_rw_den, t.rw_den, sizeof t.rw_den));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_lsx, t.lsx, sizeof t.lsx));
  AMR_CUDA(cudaMemcpyToSymbol(amr::c_ls_den, t.ls_den, sizeof t.ls_den));
  g_tables_ready[device] = 1;
  return AMR_OK;
}

template <typename T>
amr_status upload(const std::vector<T>& h, T** d) {
  *d = nullptr;
  if (h.empty()) return AMR_OK;
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return AMR_ERR_OUT_OF_MEMORY; }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(*d);
    *d = nullptr;
    return cuda_fail(e, "cudaMemcpy");
  }
  return AMR_OK;
}

bool ranges_overlap(const void* a, int64_t abytes, const void* b, int64_t bbytes) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + bbytes && pb < pa + abytes;
}

}  // namespace

// Mean device time of `reps` runs of f on stream s (after one warm-up run).
template <typename F>
static amr_status time_runs(cudaStream_t s, int reps, F f, float* ms) {
  cudaEvent_t a, b;
  AMR_CUDA(cudaEventCreate(&a));
  AMR_CUDA(cudaEventCreate(&b));
  amr_status st = f();
  if (st == AMR_OK) {
    cudaEventRecord(a, s);
    for (int r = 0; r < reps && st == AMR_OK; ++r) st = f();
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) st = cuda_fail(e, "autotune timing");
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    *ms = t / reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

struct amr_transfer_plan {
  int device = 0;
  int U = 0;
  int precision = 0;
  int64_t coarse_elems = 0, fine_elems = 0;
  amr_transfer_item* items_d = nullptr;
  amr::Tile* itiles_d = nullptr;
  amr::Tile* rtiles_d = nullptr;
  int n_itiles = 0, n_rtiles = 0;
  int n_iseg[4] = {0, 0, 0, 0};  // interpolation tile segments: FD, FD + CUT, least squares, least squares + CUT
  // least-squares derivative tables (items with scheme 1)
  float* ls_wf_d = nullptr;
  double* ls_wd_d = nullptr;
  int64_t* ls_off_d = nullptr;
  // forward sparse rows of the items routed to the CSR kernels
  int n_cpt = 0, n_crt = 0;
  amr::CsrTile *cpt_d = nullptr, *crt_d = nullptr;
  int32_t *pf_row_d = nullptr, *rf_row_d = nullptr;
  uint32_t *pf_col_d = nullptr, *rf_col_d = nullptr, *pf_out_d = nullptr, *rf_out_d = nullptr;
  uint32_t *pf_base_d = nullptr, *rf_base_d = nullptr;
  double *pf_val_d = nullptr, *rf_val_d = nullptr;
  float* pf_valf_d = nullptr;
  int32_t flags = 0;
  int64_t* incr_off_d = nullptr;            // float32 increment offsets per item
  amr::AdjointTile* incr_tiles_d = nullptr;  // apply_increments work
  int n_incr_tiles = 0;
  int interp_smem = 0;  // bytes of dynamic shared memory per interpolation CTA
  amr_transfer_plan_info info{};
  amr_transfer_tuning tuning{kThreads, kSmemBudget, kThreads, 2, 0};
  cudaGraphExec_t step_exec = nullptr;
  // adjoint tables, built on the first adjoint call
  std::vector<amr_transfer_item> items_h;
  bool adj_ready = false;
  int n_pt_tiles = 0, n_rt_tiles = 0;
  amr::AdjointTile *pt_tiles_d = nullptr, *rt_tiles_d = nullptr;
  int n_fx_pt_tiles = 0, n_rtt_tiles = 0, fx_adj_smem = 0;
  // whether the factorised kernels write every value of the gradient buffer
  // (then the adjoint calls need no zero fill first)
  bool pt_covers = false, rt_covers = false;
  amr::AdjointTile* fx_pt_tiles_d = nullptr;
  amr::Tile* rtt_tiles_d = nullptr;
  int32_t *group_ptr_d = nullptr, *group_items_d = nullptr, *item_class_d = nullptr;
  int32_t *cls_pt_rows_d = nullptr, *cls_rt_rows_d = nullptr, *pt_row_ptr_d = nullptr, *rt_row_ptr_d = nullptr;
  uint32_t *pt_col_d = nullptr, *rt_col_d = nullptr;
  double *pt_val_d = nullptr, *rt_val_d = nullptr;
  // diagonal-halo tables, built on the first such call
  bool diag_ready = false;
  int n_diag_tiles = 0;
  int64_t diag_elems = 0;
  amr::AdjointTile* diag_tiles_d = nullptr;
  int64_t* diag_off_d = nullptr;
};

static void drop_graph(amr_transfer_plan* p) {
  if (p->step_exec) cudaGraphExecDestroy(p->step_exec);
  p->step_exec = nullptr;
}

static void free_plan(amr_transfer_plan* p) {
  if (!p) return;
  drop_graph(p);
  void* csr[] = {p->cpt_d, p->crt_d, p->pf_row_d, p->rf_row_d, p->pf_col_d, p->rf_col_d, p->pf_out_d,
                 p->rf_out_d, p->pf_base_d, p->rf_base_d, p->pf_val_d, p->rf_val_d, p->pf_valf_d};
  for (void* q : csr) cudaFree(q);
  void* ls[] = {p->ls_wf_d, p->ls_wd_d, p->ls_off_d, p->diag_tiles_d, p->diag_off_d};
  for (void* q : ls) cudaFree(q);
  void* ptrs[] = {p->items_d, p->itiles_d, p->rtiles_d, p->incr_off_d, p->incr_tiles_d, p->pt_tiles_d, p->rt_tiles_d,
                  p->fx_pt_tiles_d, p->rtt_tiles_d, p->group_ptr_d,
                  p->group_items_d, p->item_class_d, p->cls_pt_rows_d, p->cls_rt_rows_d, p->pt_row_ptr_d,
                  p->rt_row_ptr_d, p->pt_col_d, p->rt_col_d, p->pt_val_d, p->rt_val_d};
  for (void* q : ptrs) cudaFree(q);
  delete p;
}

// Build and upload the transposed operators (synchronous; first adjoint call).
// Items with overlap 4 or 5 (two layers of interpolation centres) are served
// by interpolate and restrict only.
static bool has_deep_overlap(const amr_transfer_plan* p) {
  for (const amr_transfer_item& x : p->items_h)
    if (x.overlap > 3) return true;
  return false;
}

static amr_status ensure_adjoint(amr_transfer_plan* p) {
  if (p->adj_ready) return AMR_OK;
  if (has_deep_overlap(p)) return AMR_ERR_UNSUPPORTED;  // adjoints serve overlaps 1..3
  amr_transfer_desc d{};
  d.abi_version = AMR_TRANSFER_ABI_VERSION;
  d.num_unknowns = p->U;
  d.num_items = (int64_t)p->items_h.size();
  d.items = p->items_h.data();
  amr::AdjointBuild ab;
  try {
    ab = amr::build_adjoint(d);
  } catch (const std::bad_alloc&) {
    return AMR_ERR_OUT_OF_MEMORY;
  }
  amr_status st;
  auto drop = [&]() {
    void** ptrs[] = {(void**)&p->pt_tiles_d, (void**)&p->rt_tiles_d, (void**)&p->fx_pt_tiles_d,
                     (void**)&p->rtt_tiles_d, (void**)&p->group_ptr_d,
                     (void**)&p->group_items_d, (void**)&p->item_class_d, (void**)&p->cls_pt_rows_d,
                     (void**)&p->cls_rt_rows_d, (void**)&p->pt_row_ptr_d, (void**)&p->pt_col_d, (void**)&p->pt_val_d,
                     (void**)&p->rt_row_ptr_d, (void**)&p->rt_col_d, (void**)&p->rt_val_d};
    for (void** q : ptrs) {
      cudaFree(*q);
      *q = nullptr;
    }
  };
  if ((st = upload(ab.pt_tiles, &p->pt_tiles_d)) != AMR_OK || (st = upload(ab.rt_tiles, &p->rt_tiles_d)) != AMR_OK ||
      (st = upload(ab.group_ptr, &p->group_ptr_d)) != AMR_OK ||
      (st = upload(ab.group_items, &p->group_items_d)) != AMR_OK ||
      (st = upload(ab.item_class, &p->item_class_d)) != AMR_OK ||
      (st = upload(ab.cls_pt_rows, &p->cls_pt_rows_d)) != AMR_OK ||
      (st = upload(ab.cls_rt_rows, &p->cls_rt_rows_d)) != AMR_OK ||
      (st = upload(ab.pt.row_ptr, &p->pt_row_ptr_d)) != AMR_OK || (st = upload(ab.pt.col, &p->pt_col_d)) != AMR_OK ||
      (st = upload(ab.pt.val, &p->pt_val_d)) != AMR_OK || (st = upload(ab.rt.row_ptr, &p->rt_row_ptr_d)) != AMR_OK ||
      (st = upload(ab.rt.col, &p->rt_col_d)) != AMR_OK || (st = upload(ab.rt.val, &p->rt_val_d)) != AMR_OK ||
      (st = upload(ab.fx_pt_tiles, &p->fx_pt_tiles_d)) != AMR_OK ||
      (st = upload(ab.rt_taylor_tiles, &p->rtt_tiles_d)) != AMR_OK) {
    drop();
    return st;
  }
  if (ab.fx_smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute((const void*)amr::interp_adjoint_fixed_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, ab.fx_smem);
    if (e != cudaSuccess) {
      drop();
      return cuda_fail(e, "cudaFuncSetAttribute");
    }
  }
  p->n_fx_pt_tiles = (int)ab.fx_pt_tiles.size();
  p->n_rtt_tiles = (int)ab.rt_taylor_tiles.size();
  // coverage: the arrays the factorised kernels overwrite, sorted, must tile
  // [0, elems) without gaps, and no item may be left to the sparse-row kernels
  auto covers = [](std::vector<std::pair<int64_t, int64_t>>& iv, int64_t elems) {
    std::sort(iv.begin(), iv.end());
    int64_t at = 0;
    for (const auto& r : iv) {
      if (r.first > at) return false;
      at = std::max(at, r.second);
    }
    return at >= elems;
  };
  {
    std::vector<std::pair<int64_t, int64_t>> iv;
    for (const amr::AdjointTile& t : ab.fx_pt_tiles) {
      const amr_transfer_item& x = p->items_h[ab.group_items[ab.group_ptr[t.index]]];
      iv.push_back({x.coarse_offset, x.coarse_offset + 2LL * x.overlap * x.patch_size * x.patch_size * p->U});
    }
    p->pt_covers = ab.pt_tiles.empty() && covers(iv, p->coarse_elems);
    iv.clear();
    for (const amr::Tile& t : ab.rt_taylor_tiles) {
      const amr_transfer_item& x = p->items_h[t.item];
      const int64_t arr = 2LL * x.overlap * x.patch_size * x.patch_size * p->U;
      iv.push_back({x.fine_offset + t.slot * arr, x.fine_offset + (t.slot + 1) * arr});
    }
    p->rt_covers = ab.rt_tiles.empty() && covers(iv, p->fine_elems);
  }
  p->fx_adj_smem = ab.fx_smem;
  p->n_pt_tiles = (int)ab.pt_tiles.size();
  p->n_rt_tiles = (int)ab.rt_tiles.size();
  p->adj_ready = true;
  return AMR_OK;
}

// Tables of the diagonal-halo call: one tile per fine face array and chunk of
// <= 128 unknowns, and the element offset of each item's widened boxes.
static amr_status ensure_diagonal(amr_transfer_plan* p) {
  if (p->diag_ready) return AMR_OK;
  std::vector<amr::AdjointTile> tiles;
  std::vector<int64_t> off;
  int64_t total = 0;
  for (size_t i = 0; i < p->items_h.size(); ++i) {
    const amr_transfer_item& x = p->items_h[i];
    if (x.overlap > 3 || (x.order >= 2 && x.scheme != 0)) return AMR_ERR_UNSUPPORTED;
    const int nsub = x.subface < 0 ? 9 : 1;
    const int64_t W = x.patch_size + 2LL * x.overlap;
    off.push_back(total);
    total += nsub * x.overlap * W * W * p->U;
    for (int sl = 0; sl < nsub; ++sl)
      for (int64_t u0 = 0; u0 < p->U; u0 += 128)
        tiles.push_back({(int32_t)i, (int16_t)sl, 0, (int16_t)u0, (int16_t)std::min<int64_t>(128, p->U - u0)});
  }
  amr_status st;
  if ((st = upload(tiles, &p->diag_tiles_d)) != AMR_OK) return st;
  if ((st = upload(off, &p->diag_off_d)) != AMR_OK) {
    cudaFree(p->diag_tiles_d);
    p->diag_tiles_d = nullptr;
    return st;
  }
  p->n_diag_tiles = (int)tiles.size();
  p->diag_elems = total;
  p->diag_ready = true;
  return AMR_OK;
}

extern "C" {

const char* amr_status_string(amr_status s) {
  switch (s) {
    case AMR_OK: return "ok";
    case AMR_ERR_INVALID_ARGUMENT: return "invalid argument";
    case AMR_ERR_UNSUPPORTED: return "unsupported";
    case AMR_ERR_OUT_OF_MEMORY: return "out of memory";
    case AMR_ERR_CUDA: return "CUDA error";
    case AMR_ERR_TIMEOUT: return "timeout";
    case AMR_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* amr_last_cuda_error(void) { return g_cuda_error.c_str(); }

// Kernel launches of one interpolate call.
static int interp_launch_count(const amr_transfer_plan* p) {
  int n = p->n_cpt > 0 ? 1 : 0;
  for (int q = 0; q < 4; ++q) n += p->n_iseg[q] > 0 ? 1 : 0;
  return n;
}

// (Re)build the forward tiles of a plan for its tuning (synchronous).
static amr_status rebuild_tiles(amr_transfer_plan* p) {
  amr_transfer_desc d{};
  d.abi_version = AMR_TRANSFER_ABI_VERSION;
  d.num_unknowns = p->U;
  d.precision = p->precision;
  d.num_items = (int64_t)p->items_h.size();
  d.items = p->items_h.data();
  d.coarse_elems = p->coarse_elems;
  d.fine_elems = p->fine_elems;
  d.flags = p->flags;
  amr::BuildResult br;
  try {
    const bool per_warp = p->tuning.interp_lanes == 32 || p->precision == AMR_PREC_FIXED;
    br = amr::build_plan(d, p->tuning.interp_smem_budget, per_warp ? 32 : 32767);
  } catch (const std::bad_alloc&) {
    return AMR_ERR_OUT_OF_MEMORY;
  }
  if (br.status != AMR_OK) {
    g_cuda_error = br.message;
    return br.status;
  }
  if (br.interp_tiles.size() > (size_t)INT32_MAX || br.restrict_tiles.size() > (size_t)INT32_MAX)
    return AMR_ERR_UNSUPPORTED;
  if (br.max_interp_smem > 227 * 1024) return AMR_ERR_UNSUPPORTED;
  amr::Tile *it = nullptr, *rt = nullptr;
  int64_t* io = nullptr;
  amr::AdjointTile* itl = nullptr;
  amr_status st;
  if ((st = upload(br.interp_tiles, &it)) != AMR_OK || (st = upload(br.restrict_tiles, &rt)) != AMR_OK ||
      (st = upload(br.incr_off, &io)) != AMR_OK || (st = upload(br.incr_tiles, &itl)) != AMR_OK) {
    cudaFree(it);
    cudaFree(rt);
    cudaFree(io);
    cudaFree(itl);
    return st;
  }
  if (br.max_interp_smem > 48 * 1024) {
    const void* fns[] = {(const void*)amr::interp_kernel<false>, (const void*)amr::interp_kernel<true, 0>,
                         (const void*)amr::interp_kernel<true, 1>, (const void*)amr::interp_kernel<true, 2>,
                         (const void*)amr::interp_kernel<true, 3>, (const void*)amr::interp_kernel<true, 0, true>,
                         (const void*)amr::interp_kernel<false, 2, false, true>,
                         (const void*)amr::interp_kernel<true, 2, false, true>,
                         (const void*)amr::interp_kernel<true, 0, true, true>,
                         (const void*)amr::interp_kernel<false, 2, false, false, true>,
                         (const void*)amr::interp_kernel<false, 2, false, true, true>,
                         (const void*)amr::interp_kernel<true, 2, false, false, true>,
                         (const void*)amr::interp_kernel<true, 2, false, true, true>,
                         (const void*)amr::interp_fixed_kernel<false, 0>, (const void*)amr::interp_fixed_kernel<false, 1>,
                         (const void*)amr::interp_fixed_kernel<false, 2>, (const void*)amr::interp_fixed_kernel<false, 3>,
                         (const void*)amr::interp_fixed_kernel<true, 0>, (const void*)amr::interp_fixed_kernel<true, 1>,
                         (const void*)amr::interp_fixed_kernel<true, 2>, (const void*)amr::interp_fixed_kernel<true, 3>};
    cudaError_t e = cudaSuccess;
    for (size_t q = 0; q < sizeof fns / sizeof fns[0] && e == cudaSuccess; ++q)
      e = cudaFuncSetAttribute(fns[q], cudaFuncAttributeMaxDynamicSharedMemorySize, br.max_interp_smem);
    if (e != cudaSuccess) {
      cudaFree(it);
      cudaFree(rt);
      cudaFree(io);
      cudaFree(itl);
      return cuda_fail(e, "cudaFuncSetAttribute");
    }
  }
  cudaFree(p->itiles_d);
  cudaFree(p->rtiles_d);
  cudaFree(p->incr_off_d);
  cudaFree(p->incr_tiles_d);
  p->itiles_d = it;
  p->rtiles_d = rt;
  p->incr_off_d = io;
  p->incr_tiles_d = itl;
  p->n_incr_tiles = (int)br.incr_tiles.size();
  p->info.increment_elems = br.incr_elems;
  p->n_itiles = (int)br.interp_tiles.size();
  for (int q = 0; q < 4; ++q) p->n_iseg[q] = (int)br.interp_segments[q];
  p->n_rtiles = (int)br.restrict_tiles.size();
  p->interp_smem = br.max_interp_smem;
  p->info.num_items = d.num_items;
  p->info.interp_outputs = br.interp_outputs;
  p->info.restrict_outputs = br.restrict_outputs;
  p->info.interp_bytes = br.interp_bytes;
  p->info.restrict_bytes = br.restrict_bytes;
  p->info.interp_launches = interp_launch_count(p);
  p->info.restrict_launches = (p->n_rtiles > 0 ? 1 : 0) + (p->n_crt > 0 ? 1 : 0);
  return AMR_OK;
}

// Upload the forward sparse rows of the CSR-routed items (plan create).
static amr_status build_csr_tables(amr_transfer_plan* p, const amr_transfer_desc& d) {
  amr::CsrBuild cb;
  try {
    cb = amr::build_csr(d);
  } catch (const std::bad_alloc&) {
    return AMR_ERR_OUT_OF_MEMORY;
  }
  if (cb.ptiles.empty() && cb.rtiles.empty()) return AMR_OK;
  std::vector<float> valf(cb.pf.val.begin(), cb.pf.val.end());
  amr_status st;
  if ((st = upload(cb.ptiles, &p->cpt_d)) != AMR_OK || (st = upload(cb.rtiles, &p->crt_d)) != AMR_OK ||
      (st = upload(cb.pf.row_ptr, &p->pf_row_d)) != AMR_OK || (st = upload(cb.rf.row_ptr, &p->rf_row_d)) != AMR_OK ||
      (st = upload(cb.pf.col, &p->pf_col_d)) != AMR_OK || (st = upload(cb.rf.col, &p->rf_col_d)) != AMR_OK ||
      (st = upload(cb.pf.out_vol, &p->pf_out_d)) != AMR_OK || (st = upload(cb.rf.out_vol, &p->rf_out_d)) != AMR_OK ||
      (st = upload(cb.pf.base_vol, &p->pf_base_d)) != AMR_OK ||
      (st = upload(cb.rf.base_vol, &p->rf_base_d)) != AMR_OK || (st = upload(cb.pf.val, &p->pf_val_d)) != AMR_OK ||
      (st = upload(cb.rf.val, &p->rf_val_d)) != AMR_OK || (st = upload(valf, &p->pf_valf_d)) != AMR_OK)
    return st;
  p->n_cpt = (int)cb.ptiles.size();
  p->n_crt = (int)cb.rtiles.size();
  p->info.interp_launches = interp_launch_count(p);
  p->info.restrict_launches = (p->n_rtiles > 0 ? 1 : 0) + (p->n_crt > 0 ? 1 : 0);
  return AMR_OK;
}

// Upload the least-squares derivative tables of the scheme-1 items (plan create).
static amr_status upload_ls_tables(amr_transfer_plan* p, const amr_transfer_desc& d) {
  amr::LsTables lt;
  try {
    lt = amr::build_ls_tables(d);
  } catch (const std::bad_alloc&) {
    return AMR_ERR_OUT_OF_MEMORY;
  }
  if (lt.wd.empty()) return AMR_OK;
  amr_status st;
  if ((st = upload(lt.wd, &p->ls_wd_d)) != AMR_OK || (st = upload(lt.wf, &p->ls_wf_d)) != AMR_OK ||
      (st = upload(lt.item_off, &p->ls_off_d)) != AMR_OK)
    return st;
  return AMR_OK;
}

amr_status amr_transfer_plan_create(const amr_transfer_desc* desc, amr_transfer_plan** out) {
  if (!out) return AMR_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (!desc) return AMR_ERR_INVALID_ARGUMENT;
  amr::BuildResult br;
  try {
    br = amr::build_plan(*desc, kSmemBudget);  // validation (tiles are rebuilt below)
  } catch (const std::bad_alloc&) {
    return AMR_ERR_OUT_OF_MEMORY;
  }
  if (br.status != AMR_OK) {
    g_cuda_error = br.message;
    return br.status;
  }
  int device = 0;
  AMR_CUDA(cudaGetDevice(&device));
  amr_status st = upload_tables(device);
  if (st != AMR_OK) return st;
  amr_transfer_plan* p = new (std::nothrow) amr_transfer_plan;
  if (!p) return AMR_ERR_OUT_OF_MEMORY;
  p->device = device;
  p->U = desc->num_unknowns;
  p->precision = desc->precision;
  p->coarse_elems = desc->coarse_elems;
  p->fine_elems = desc->fine_elems;
  p->items_h.assign(desc->items, desc->items + desc->num_items);
  p->flags = desc->flags;
  if ((st = upload(p->items_h, &p->items_d)) != AMR_OK || (st = rebuild_tiles(p)) != AMR_OK ||
      (st = build_csr_tables(p, *desc)) != AMR_OK || (st = upload_ls_tables(p, *desc)) != AMR_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return AMR_OK;
}

static amr_status check_call(const amr_transfer_plan* p, const void* in, int64_t in_elems, const void* out,
                             int64_t out_elems) {
  if (!p) return AMR_ERR_INVALID_ARGUMENT;
  if ((in_elems > 0 && !in) || (out_elems > 0 && !out)) return AMR_ERR_INVALID_ARGUMENT;
  if (in && out && ranges_overlap(in, in_elems * 8, out, out_elems * 8)) return AMR_ERR_INVALID_ARGUMENT;
  int dev = -1;
  AMR_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) return AMR_ERR_INVALID_ARGUMENT;
  return AMR_OK;
}

amr_status amr_transfer_plan_interpolate(amr_transfer_plan* p, const double* coarse, double* fine, void* stream) {
  amr_status st = check_call(p, coarse, p ? p->coarse_elems : 0, fine, p ? p->fine_elems : 0);
  if (st != AMR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->n_cpt > 0) {
    const dim3 blk(32, 8);
    if (p->precision == AMR_PREC_SPLIT)
      amr::csr_apply_kernel<true, true><<<p->n_cpt, blk, 0, s>>>(p->items_d, p->cpt_d, p->pf_row_d, p->pf_col_d,
                                                                p->pf_val_d, p->pf_valf_d, p->pf_out_d, p->pf_base_d,
                                                                p->U, coarse, fine);
    else
      amr::csr_apply_kernel<false, true><<<p->n_cpt, blk, 0, s>>>(p->items_d, p->cpt_d, p->pf_row_d, p->pf_col_d,
                                                                 p->pf_val_d, p->pf_valf_d, p->pf_out_d, p->pf_base_d,
                                                                 p->U, coarse, fine);
    AMR_CUDA(cudaGetLastError());
  }
  const dim3 b(p->tuning.interp_threads);
  const int L = p->tuning.interp_lanes;
  const amr::Tile* seg = p->itiles_d;
  const bool split = p->precision == AMR_PREC_SPLIT;
  const bool fixed = p->precision == AMR_PREC_FIXED;
  for (int q = 0; q < 4; seg += p->n_iseg[q], ++q) {
    if (p->n_iseg[q] == 0) continue;
    const dim3 g(p->n_iseg[q]);
    const int z = p->interp_smem;
    const amr_transfer_item* it = p->items_d;
    const int U = p->U;
    if (q < 2 && fixed) {
      switch (p->tuning.interp_addback + 4 * q) {
        case 0: amr::interp_fixed_kernel<false, 0><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        case 1: amr::interp_fixed_kernel<false, 1><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        case 2: amr::interp_fixed_kernel<false, 2><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        case 3: amr::interp_fixed_kernel<false, 3><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        case 4: amr::interp_fixed_kernel<true, 0><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        case 5: amr::interp_fixed_kernel<true, 1><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        case 6: amr::interp_fixed_kernel<true, 2><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
        default: amr::interp_fixed_kernel<true, 3><<<g, b, z, s>>>(it, seg, U, coarse, fine); break;
      }
    } else if (q == 0 && split) {
      switch (p->tuning.interp_addback) {
        case 0: amr::interp_kernel<true, 0><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L); break;
        case 1: amr::interp_kernel<true, 1><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L); break;
        case 3: amr::interp_kernel<true, 3><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L); break;
        default: amr::interp_kernel<true, 2><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L); break;
      }
    } else if (q == 0) {
      amr::interp_kernel<false><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L);
    } else if (q == 1 && split) {
      amr::interp_kernel<true, 2, false, true><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L);
    } else if (q == 1) {
      amr::interp_kernel<false, 2, false, true><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L);
    } else if (q == 2 && split) {
      amr::interp_kernel<true, 2, false, false, true><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L,
                                                                       p->ls_wf_d, p->ls_wd_d, p->ls_off_d);
    } else if (q == 2) {
      amr::interp_kernel<false, 2, false, false, true><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L,
                                                                        p->ls_wf_d, p->ls_wd_d, p->ls_off_d);
    } else if (split) {
      amr::interp_kernel<true, 2, false, true, true><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L,
                                                                      p->ls_wf_d, p->ls_wd_d, p->ls_off_d);
    } else {
      amr::interp_kernel<false, 2, false, true, true><<<g, b, z, s>>>(it, seg, U, coarse, fine, nullptr, nullptr, L,
                                                                       p->ls_wf_d, p->ls_wd_d, p->ls_off_d);
    }
    AMR_CUDA(cudaGetLastError());
  }
  return AMR_OK;
}

amr_status amr_transfer_plan_interpolate_increments(amr_transfer_plan* p, const double* coarse, float* increments,
                                                    void* stream) {
  // check_call counts 8-byte elements: the float32 increments take (n + 1) / 2 of them
  amr_status st = check_call(p, coarse, p ? p->coarse_elems : 0, increments, p ? (p->info.increment_elems + 1) / 2 : 0);
  if (st != AMR_OK) return st;
  if (p->n_cpt > 0 || p->n_crt > 0) return AMR_ERR_UNSUPPORTED;  // increments come from the factorised kernel
  if (has_deep_overlap(p)) return AMR_ERR_UNSUPPORTED;            // increments serve overlaps 1..3
  if (p->n_iseg[2] > 0 || p->n_iseg[3] > 0) return AMR_ERR_UNSUPPORTED;  // finite-difference items only
  if (p->n_iseg[0] > 0) {
    amr::interp_kernel<true, 0, true><<<p->n_iseg[0], p->tuning.interp_threads, p->interp_smem, (cudaStream_t)stream>>>(
        p->items_d, p->itiles_d, p->U, coarse, nullptr, increments, p->incr_off_d, p->tuning.interp_lanes);
    AMR_CUDA(cudaGetLastError());
  }
  if (p->n_iseg[1] > 0) {
    amr::interp_kernel<true, 0, true, true><<<p->n_iseg[1], p->tuning.interp_threads, p->interp_smem,
                                              (cudaStream_t)stream>>>(p->items_d, p->itiles_d + p->n_iseg[0], p->U,
                                                                      coarse, nullptr, increments, p->incr_off_d,
                                                                      p->tuning.interp_lanes);
    AMR_CUDA(cudaGetLastError());
  }
  return AMR_OK;
}

amr_status amr_transfer_plan_apply_increments(amr_transfer_plan* p, const double* coarse, const float* increments,
                                              double* fine, void* stream) {
  amr_status st = check_call(p, coarse, p ? p->coarse_elems : 0, fine, p ? p->fine_elems : 0);
  if (st != AMR_OK) return st;
  if (p->info.increment_elems > 0 && !increments) return AMR_ERR_INVALID_ARGUMENT;
  const int64_t ibytes = p->info.increment_elems * 4;
  if (increments && (ranges_overlap(increments, ibytes, fine, p->fine_elems * 8) ||
                     ranges_overlap(increments, ibytes, coarse, p->coarse_elems * 8)))
    return AMR_ERR_INVALID_ARGUMENT;
  if (p->n_cpt > 0 || p->n_crt > 0) return AMR_ERR_UNSUPPORTED;
  if (has_deep_overlap(p)) return AMR_ERR_UNSUPPORTED;
  if (p->n_incr_tiles == 0) return AMR_OK;
  amr::apply_increments_kernel<<<p->n_incr_tiles, kThreads, 0, (cudaStream_t)stream>>>(
      p->items_d, p->incr_tiles_d, p->incr_off_d, p->U, coarse, increments, fine);
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

amr_status amr_transfer_plan_restrict(amr_transfer_plan* p, const double* fine, double* coarse, void* stream) {
  amr_status st = check_call(p, fine, p ? p->fine_elems : 0, coarse, p ? p->coarse_elems : 0);
  if (st != AMR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->n_crt > 0) {
    amr::csr_apply_kernel<false, false><<<p->n_crt, dim3(32, 8), 0, s>>>(
        p->items_d, p->crt_d, p->rf_row_d, p->rf_col_d, p->rf_val_d, nullptr, p->rf_out_d, p->rf_base_d, p->U, fine,
        coarse);
    AMR_CUDA(cudaGetLastError());
  }
  if (p->n_rtiles == 0) return AMR_OK;
  if (p->precision == AMR_PREC_SPLIT)
    amr::restrict_kernel<amr::kRestrictSplit><<<p->n_rtiles, p->tuning.restrict_threads, 0, s>>>(
        p->items_d, p->rtiles_d, p->U, fine, coarse);
  else if (p->precision == AMR_PREC_FIXED)
    amr::restrict_kernel<amr::kRestrictFixed><<<p->n_rtiles, p->tuning.restrict_threads, 0, s>>>(
        p->items_d, p->rtiles_d, p->U, fine, coarse);
  else
    amr::restrict_kernel<amr::kRestrictF64><<<p->n_rtiles, p->tuning.restrict_threads, 0, s>>>(
        p->items_d, p->rtiles_d, p->U, fine, coarse);
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

amr_status amr_transfer_plan_interpolate_adjoint(amr_transfer_plan* p, const double* g_fine, double* g_coarse,
                                                 void* stream) {
  amr_status st = check_call(p, g_fine, p ? p->fine_elems : 0, g_coarse, p ? p->coarse_elems : 0);
  if (st != AMR_OK) return st;
  if ((st = ensure_adjoint(p)) != AMR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->coarse_elems > 0 && !p->pt_covers) AMR_CUDA(cudaMemsetAsync(g_coarse, 0, (size_t)p->coarse_elems * 8, s));
  if (p->n_fx_pt_tiles > 0) {
    amr::adjoint_emax_kernel<<<p->n_fx_pt_tiles, amr::kAdjThreads, 0, s>>>(
        p->items_d, p->fx_pt_tiles_d, p->group_ptr_d, p->group_items_d, p->U, g_fine, g_coarse);
    AMR_CUDA(cudaGetLastError());
    amr::interp_adjoint_fixed_kernel<<<p->n_fx_pt_tiles, amr::kAdjThreads, p->fx_adj_smem, s>>>(
        p->items_d, p->fx_pt_tiles_d, p->group_ptr_d, p->group_items_d, p->U, g_fine, g_coarse);
    AMR_CUDA(cudaGetLastError());
  }
  if (p->n_pt_tiles > 0) {
    amr::interp_adjoint_kernel<<<p->n_pt_tiles, kThreads, 0, s>>>(
        p->items_d, p->pt_tiles_d, p->group_ptr_d, p->group_items_d, p->item_class_d, p->cls_pt_rows_d,
        p->pt_row_ptr_d, p->pt_col_d, p->pt_val_d, p->U, g_fine, g_coarse);
    AMR_CUDA(cudaGetLastError());
  }
  return AMR_OK;
}

amr_status amr_transfer_plan_interpolate_diagonal(amr_transfer_plan* p, const double* coarse, double* diag,
                                                  int64_t diag_elems, void* stream) {
  amr_status st = check_call(p, coarse, p ? p->coarse_elems : 0, diag, diag_elems);
  if (st != AMR_OK) return st;
  if ((st = ensure_diagonal(p)) != AMR_OK) return st;
  if (diag_elems < p->diag_elems) return AMR_ERR_INVALID_ARGUMENT;
  if (p->n_diag_tiles == 0) return AMR_OK;
  amr::interp_diagonal_kernel<<<p->n_diag_tiles, 256, 0, (cudaStream_t)stream>>>(
      p->items_d, p->diag_tiles_d, p->U, p->diag_off_d, coarse, diag);
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

amr_status amr_transfer_plan_restrict_adjoint(amr_transfer_plan* p, const double* g_coarse, double* g_fine,
                                              void* stream) {
  amr_status st = check_call(p, g_coarse, p ? p->coarse_elems : 0, g_fine, p ? p->fine_elems : 0);
  if (st != AMR_OK) return st;
  if ((st = ensure_adjoint(p)) != AMR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->fine_elems > 0 && !p->rt_covers) AMR_CUDA(cudaMemsetAsync(g_fine, 0, (size_t)p->fine_elems * 8, s));
  if (p->n_rtt_tiles > 0) {
    amr::restrict_adjoint_taylor_kernel<<<p->n_rtt_tiles, kThreads, 0, s>>>(p->items_d, p->rtt_tiles_d, p->U,
                                                                            g_coarse, g_fine);
    AMR_CUDA(cudaGetLastError());
  }
  if (p->n_rt_tiles > 0) {
    amr::restrict_adjoint_kernel<<<p->n_rt_tiles, kThreads, 0, s>>>(p->items_d, p->rt_tiles_d, p->cls_rt_rows_d,
                                                                    p->rt_row_ptr_d, p->rt_col_d, p->rt_val_d, p->U,
                                                                    g_coarse, g_fine);
    AMR_CUDA(cudaGetLastError());
  }
  return AMR_OK;
}

amr_status amr_transfer_plan_get_tuning(const amr_transfer_plan* p, amr_transfer_tuning* out) {
  if (!p || !out) return AMR_ERR_INVALID_ARGUMENT;
  *out = p->tuning;
  return AMR_OK;
}

static bool tuning_valid(const amr_transfer_tuning& t, int precision) {
  auto ok_threads = [](int n, int max) { return n >= 32 && n <= max && n % 32 == 0; };
  const int max_interp = precision == AMR_PREC_SPLIT   ? amr::kMaxSplitInterpThreads
                         : precision == AMR_PREC_FIXED ? amr::kMaxFixedThreads
                                                       : 256;
  return ok_threads(t.interp_threads, max_interp) && ok_threads(t.restrict_threads, 256) &&
         t.interp_smem_budget >= 4096 && t.interp_smem_budget <= 196 * 1024 && t.interp_addback >= 0 &&
         t.interp_addback <= 3 && (t.interp_lanes == 0 || t.interp_lanes == 32);
}

amr_status amr_transfer_plan_set_tuning(amr_transfer_plan* p, const amr_transfer_tuning* t) {
  if (!p || !t || !tuning_valid(*t, p->precision)) return AMR_ERR_INVALID_ARGUMENT;
  drop_graph(p);
  const amr_transfer_tuning old = p->tuning;
  p->tuning = *t;
  amr_status st = rebuild_tiles(p);
  if (st != AMR_OK) {
    p->tuning = old;
    rebuild_tiles(p);
  }
  return st;
}

amr_status amr_transfer_plan_autotune(amr_transfer_plan* p, const double* coarse, double* fine, double* coarse_out,
                                      void* stream, amr_transfer_tuning* chosen) {
  amr_status st = check_call(p, coarse, p ? p->coarse_elems : 0, fine, p ? p->fine_elems : 0);
  if (st != AMR_OK) return st;
  if ((st = check_call(p, fine, p->fine_elems, coarse_out, p->coarse_elems)) != AMR_OK) return st;
  drop_graph(p);
  cudaStream_t s = (cudaStream_t)stream;
  const int reps = 3;
  amr_transfer_tuning best = p->tuning;
  float best_i = 1e30f, best_r = 1e30f;
  // (lanes, CTA size, shared-memory budget): dense packing over a range of
  // budgets; one warp per centre with budgets that fit 32 unknowns of the
  // common tile regions
  struct Shape { int lanes, threads, budget; };
  std::vector<Shape> shapes;
  if (p->precision != AMR_PREC_FIXED)
    for (int th : {128, 256})
      for (int kb : {24, 32, 48, 64, 96}) shapes.push_back({0, th, kb * 1024});
  if (p->precision == AMR_PREC_FIXED)
    for (int th : {amr::kMaxFixedThreads / 2, amr::kMaxFixedThreads})
      for (int kb : {64, 112}) shapes.push_back({32, th, kb * 1024});
  if (p->precision == AMR_PREC_SPLIT)
    for (int th : {256, amr::kMaxSplitInterpThreads})
      for (int kb : {64, 112}) shapes.push_back({32, th, kb * 1024});
  for (const Shape& sh : shapes) {
    amr_transfer_tuning t = p->tuning;
    t.interp_lanes = sh.lanes;
    t.interp_threads = sh.threads;
    t.interp_smem_budget = sh.budget;
    p->tuning = t;
    if ((st = rebuild_tiles(p)) != AMR_OK) continue;  // e.g. a budget the device cannot hold
    float ms = 0.f;
    if ((st = time_runs(s, reps, [&] { return amr_transfer_plan_interpolate(p, coarse, fine, stream); }, &ms)) !=
        AMR_OK)
      return st;
    if (ms < best_i) {
      best_i = ms;
      best.interp_lanes = sh.lanes;
      best.interp_threads = sh.threads;
      best.interp_smem_budget = sh.budget;
    }
  }
  if (p->precision == AMR_PREC_SPLIT || p->precision == AMR_PREC_FIXED) {
    p->tuning = best;
    if ((st = rebuild_tiles(p)) != AMR_OK) return st;
    for (int mode = 0; mode <= 3; ++mode) {
      p->tuning.interp_addback = mode;
      float ms = 0.f;
      if ((st = time_runs(s, reps, [&] { return amr_transfer_plan_interpolate(p, coarse, fine, stream); }, &ms)) !=
          AMR_OK)
        return st;
      if (ms < best_i) {
        best_i = ms;
        best.interp_addback = mode;
      }
    }
    p->tuning = best;
  }
  for (int th : {128, 256}) {
    p->tuning.restrict_threads = th;
    float ms = 0.f;
    if ((st = time_runs(s, reps, [&] { return amr_transfer_plan_restrict(p, fine, coarse_out, stream); }, &ms)) !=
        AMR_OK)
      return st;
    if (ms < best_r) {
      best_r = ms;
      best.restrict_threads = th;
    }
  }
  p->tuning = best;
  if ((st = rebuild_tiles(p)) != AMR_OK) return st;
  if (chosen) *chosen = best;
  return AMR_OK;
}

amr_status amr_transfer_plan_capture_step(amr_transfer_plan* p, const double* coarse, double* fine,
                                          double* coarse_out) {
  amr_status st = check_call(p, coarse, p ? p->coarse_elems : 0, fine, p ? p->fine_elems : 0);
  if (st != AMR_OK) return st;
  if ((st = check_call(p, fine, p->fine_elems, coarse_out, p->coarse_elems)) != AMR_OK) return st;
  drop_graph(p);
  cudaStream_t cs;
  AMR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = amr_transfer_plan_interpolate(p, coarse, fine, cs);
    if (st == AMR_OK) st = amr_transfer_plan_restrict(p, fine, coarse_out, cs);
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (e == cudaSuccess && st == AMR_OK) e = cudaGraphInstantiate(&p->step_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (st != AMR_OK) return st;
  if (e != cudaSuccess) {
    p->step_exec = nullptr;
    return cuda_fail(e, "step graph capture");
  }
  return AMR_OK;
}

amr_status amr_transfer_plan_launch_step(amr_transfer_plan* p, void* stream) {
  if (!p || !p->step_exec) return AMR_ERR_INVALID_ARGUMENT;
  AMR_CUDA(cudaGraphLaunch(p->step_exec, (cudaStream_t)stream));
  return AMR_OK;
}

amr_status amr_transfer_plan_get_info(const amr_transfer_plan* p, amr_transfer_plan_info* info) {
  if (!p || !info) return AMR_ERR_INVALID_ARGUMENT;
  *info = p->info;
  return AMR_OK;
}

amr_status amr_transfer_plan_destroy(amr_transfer_plan* p) {
  if (!p) return AMR_OK;
  const int dev = p->device;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  free_plan(p);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return AMR_OK;
}

}  // extern "C"
