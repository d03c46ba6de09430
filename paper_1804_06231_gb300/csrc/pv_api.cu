// pv_api.cu -- host side of the C ABI declared in include/pv.h: argument
// checks, scratch allocation, and the launch sequence of each call.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pv_internal.cuh"

using pv::GridDev;

struct pv_grid {
  GridDev d{};
  std::vector<pv_box_desc> boxes;
  std::vector<void*> allocs;
  int64_t n = 0, ncell = 0;
  int device = 0, num_sms = 0;
  bool sorted = false;
  size_t bytes = 0;
  int64_t launches = 0;  // kernels launched by this grid so far
  int ctas[2] = {pv::kDensityCtasDefault, pv::kBackwardCtasDefault};  // sweep CTAs per SM
  int task_blk[2] = {pv::kTaskBlkDefault, pv::kTaskBlkDefault};        // particles per task
  // sweep timing (pv_grid_time_sweeps): a ring of event pairs per sweep kind
  static constexpr int kRing = 64;
  bool timing = false;
  std::vector<cudaEvent_t> ev;      // 2 kinds x kRing x {start, stop}
  int head[2] = {0, 0}, pending[2] = {0, 0};
  double ms[2] = {0.0, 0.0};
  int64_t timed[2] = {0, 0};
};

namespace {

thread_local char g_cuda_err[256] = "no error";

pv_status cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? PV_ERR_OUT_OF_MEMORY : PV_ERR_CUDA;
}

}  // namespace

pv_status pv::record_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

namespace {

#define PV_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <typename T>
pv_status dev_alloc(pv_grid* g, T** p, size_t count) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  g->allocs.push_back(ptr);
  g->bytes += bytes;
  *p = static_cast<T*>(ptr);
  return PV_OK;
}

#define PV_TRY(x)                   \
  do {                              \
    pv_status s_ = (x);             \
    if (s_ != PV_OK) return s_;     \
  } while (0)

// Folds the oldest pending event pair of `kind` into the totals.
pv_status retire_oldest(pv_grid* g, int kind) {
  const int slot = (g->head[kind] - g->pending[kind] + pv_grid::kRing) % pv_grid::kRing;
  cudaEvent_t a = g->ev[(kind * pv_grid::kRing + slot) * 2];
  cudaEvent_t b = g->ev[(kind * pv_grid::kRing + slot) * 2 + 1];
  PV_CUDA(cudaEventSynchronize(b));
  float t = 0.0f;
  PV_CUDA(cudaEventElapsedTime(&t, a, b));
  g->ms[kind] += t;
  g->timed[kind] += 1;
  g->pending[kind] -= 1;
  return PV_OK;
}

// The next event pair of `kind` (nullptrs when timing is off).
pv_status next_pair(pv_grid* g, int kind, cudaEvent_t* a, cudaEvent_t* b) {
  *a = *b = nullptr;
  if (!g->timing) return PV_OK;
  if (g->pending[kind] == pv_grid::kRing) PV_TRY(retire_oldest(g, kind));
  const int slot = g->head[kind];
  *a = g->ev[(kind * pv_grid::kRing + slot) * 2];
  *b = g->ev[(kind * pv_grid::kRing + slot) * 2 + 1];
  g->head[kind] = (slot + 1) % pv_grid::kRing;
  g->pending[kind] += 1;
  return PV_OK;
}

void free_all(pv_grid* g) {
  for (void* p : g->allocs) cudaFree(p);
  g->allocs.clear();
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  g->ev.clear();
}

pv_status build(pv_grid* g, const pv_grid_desc* desc) {
  const double gamma = desc->gamma > 0 ? desc->gamma : 1.825742;
  std::vector<pv::BoxDev> hb(desc->n_boxes);
  std::vector<int64_t> hfirst(desc->n_boxes);
  int64_t n = 0, ncell = 0;
  for (int b = 0; b < desc->n_boxes; b++) {
    const pv_box_desc& bd = desc->boxes[b];
    if (bd.n < 0 || !(bd.L > 0) || !std::isfinite(bd.L)) return PV_ERR_INVALID_ARGUMENT;
    if (bd.first != n) return PV_ERR_INVALID_ARGUMENT;  // contiguous, in order
    if (bd.nc < 3) return PV_ERR_CELL_TOO_SMALL;
    if (bd.nc > 1290) return PV_ERR_TOO_LARGE;  // nc^3 fits in int32
    pv::BoxDev& B = hb[b];
    B.L = bd.L;
    B.inv_L = 1.0 / bd.L;
    B.edge = bd.L / bd.nc;
    B.inv_edge = bd.nc / bd.L;
    B.edge_f = (float)B.edge;
    // projections of FP32 offsets carry < 2^-21 edge of rounding each; the
    // window pad covers two of them plus the FP32 cell shift
    B.pad = (float)(std::ldexp(B.edge, -18));
    B.guard = 0.0f;
    B.h_limit = pv::support_h_limit(gamma, B.edge);
    B.nc = bd.nc;
    B.cell_base = (int32_t)ncell;
    B.first = bd.first;
    B.n = bd.n;
    hfirst[b] = bd.first;
    n += bd.n;
    ncell += (int64_t)bd.nc * bd.nc * bd.nc;
    // thread indices over (cell, slot) pairs and task counts stay in int32
    if (n > 0x7fffffffLL / 32 * 32 - 64 || ncell * pv::kNSlot > 0x7fffffffLL)
      return PV_ERR_TOO_LARGE;
  }
  g->n = n;
  g->ncell = ncell;
  g->boxes.assign(desc->boxes, desc->boxes + desc->n_boxes);
  PV_CUDA(cudaGetDevice(&g->device));
  PV_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));

  GridDev& d = g->d;
  d.n_boxes = desc->n_boxes;
  d.n = (int32_t)n;
  d.ncell = (int32_t)ncell;
  d.gamma = (float)gamma;
  d.gamma_d = gamma;
  const size_t N = (size_t)n, C = (size_t)ncell;
  pv::BoxDev* boxes_d;
  int64_t* first_d;
  PV_TRY(dev_alloc(g, &boxes_d, hb.size()));
  PV_TRY(dev_alloc(g, &first_d, hfirst.size()));
  PV_CUDA(cudaMemcpy(boxes_d, hb.data(), hb.size() * sizeof(pv::BoxDev), cudaMemcpyHostToDevice));
  PV_CUDA(cudaMemcpy(first_d, hfirst.data(), hfirst.size() * sizeof(int64_t),
                     cudaMemcpyHostToDevice));
  d.boxes = boxes_d;
  d.box_first = first_d;
  PV_TRY(dev_alloc(g, &d.cell_count, C));
  PV_TRY(dev_alloc(g, &d.cell_start, C + 1));
  PV_TRY(dev_alloc(g, &d.cell_box, C));
  PV_TRY(dev_alloc(g, &d.cell_Hmax, C));
  PV_TRY(dev_alloc(g, &d.big_cells, C));
  PV_TRY(dev_alloc(g, &d.small_cells, C));
  PV_TRY(dev_alloc(g, &d.tile_sum, (size_t)pv::scan_tiles(ncell)));
  PV_TRY(dev_alloc(g, &d.pcell, N));
  PV_TRY(dev_alloc(g, &d.prank, N));
  PV_TRY(dev_alloc(g, &d.xm, N));
  PV_TRY(dev_alloc(g, &d.xm_ref, N));
  PV_TRY(dev_alloc(g, &d.hs, N));
  PV_TRY(dev_alloc(g, &d.orig, N));
  PV_TRY(dev_alloc(g, &d.pos64, 3 * N));
  PV_TRY(dev_alloc(g, &d.perm, pv::kNDir * N));
  PV_TRY(dev_alloc(g, &d.dist, pv::kNDir * N));
  PV_TRY(dev_alloc(g, &d.acc, 3 * N));
  PV_TRY(dev_alloc(g, &d.gacc, 5 * N));
  PV_TRY(dev_alloc(g, &d.bx, N));
  PV_TRY(dev_alloc(g, &d.ba, N));
  PV_TRY(dev_alloc(g, &d.bwd_cmax, C));
  PV_TRY(dev_alloc(g, &d.bwd_hmin, C));
  PV_TRY(dev_alloc(g, &d.plan, (size_t)pv::kNSlot * C));
  PV_TRY(dev_alloc(g, &d.ccells, C));
  PV_TRY(dev_alloc(g, &d.tcells, C));
  PV_TRY(dev_alloc(g, &d.ycells, C));
  const int64_t mt = pv::max_tasks_for(n, ncell);
  if (mt > 0x7fffffffLL) return PV_ERR_TOO_LARGE;
  d.max_tasks = (int32_t)mt;
  d.task_blk = pv::kTaskBlkDefault;
  d.slot_mask = pv::kAllSlots;
  d.moved = 0;
  PV_TRY(dev_alloc(g, &d.tasks, (size_t)d.max_tasks));
  // scalars in one allocation
  int32_t* sc;
  PV_TRY(dev_alloc(g, &sc, 16));
  d.flags = reinterpret_cast<uint32_t*>(sc + 0);
  PV_TRY(dev_alloc(g, &d.m_max, hb.size()));
  PV_TRY(dev_alloc(g, &d.box_disp, hb.size()));
  PV_CUDA(cudaMemset(d.box_disp, 0, hb.size() * sizeof(float)));
  d.max_count = sc + 2;
  d.n_big = sc + 3;
  d.n_small = sc + 12;
  d.n_large = sc + 13;
  d.n_huge = sc + 14;
  d.ntask = sc + 4;
  d.task_next = sc + 5;
  d.n_ccells = sc + 6;
  d.ccell_next = sc + 7;
  d.n_tcells = sc + 8;
  d.n_ycells = sc + 10;
  d.ycell_next = sc + 11;
  unsigned long long* cnt;
  PV_TRY(dev_alloc(g, &cnt, 16));
  d.counters = cnt;
  PV_CUDA(cudaMemset(sc, 0, 16 * sizeof(int32_t)));
  PV_CUDA(cudaMemset(cnt, 0, 16 * sizeof(unsigned long long)));
  if (N) {
    PV_CUDA(cudaMemset(d.acc, 0, 3 * N * sizeof(long long)));
    PV_CUDA(cudaMemset(d.gacc, 0, 5 * N * sizeof(long long)));
  }
  // cell -> box map
  std::vector<int32_t> cbox(C);
  for (int b = 0; b < desc->n_boxes; b++) {
    const int64_t c0 = hb[b].cell_base, c1 = c0 + (int64_t)hb[b].nc * hb[b].nc * hb[b].nc;
    for (int64_t c = c0; c < c1; c++) cbox[c] = b;
  }
  if (C) PV_CUDA(cudaMemcpy(d.cell_box, cbox.data(), C * sizeof(int32_t), cudaMemcpyHostToDevice));
  return PV_OK;
}

}  // namespace

extern "C" {

const char* pv_status_str(pv_status s) {
  switch (s) {
    case PV_OK: return "ok";
    case PV_ERR_INVALID_ARGUMENT: return "invalid argument";
    case PV_ERR_CELL_TOO_SMALL: return "cell grid too coarse (nc < 3)";
    case PV_ERR_OUT_OF_MEMORY: return "out of memory";
    case PV_ERR_CUDA: return "CUDA error";
    case PV_ERR_NOT_SORTED: return "pv_sort_cells has not been called on this grid";
    case PV_ERR_DEVICE: return "a kernel latched an input error (see device_flags)";
    case PV_ERR_TOO_LARGE: return "too many particles or cells";
  }
  return "unknown status";
}

const char* pv_last_cuda_error(void) { return g_cuda_err; }

pv_status pv_grid_create(const pv_grid_desc* desc, pv_grid** out) {
  if (!desc || !out || desc->n_boxes < 1 || !desc->boxes || desc->flags != 0)
    return PV_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  pv_grid* g = new (std::nothrow) pv_grid();
  if (!g) return PV_ERR_OUT_OF_MEMORY;
  pv_status s = build(g, desc);
  if (s != PV_OK) {
    free_all(g);
    delete g;
    return s;
  }
  *out = g;
  return PV_OK;
}

pv_status pv_grid_destroy(pv_grid* g) {
  if (!g) return PV_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_all(g);
  delete g;
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  return PV_OK;
}

pv_status pv_sort_cells(pv_grid* g, const double* pos, const float* h, const float* m,
                        float m_uniform, void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (g->n > 0 && (!pos || !h)) return PV_ERR_INVALID_ARGUMENT;
  if (!m && !(m_uniform >= 0.0f && std::isfinite(m_uniform))) return PV_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GridDev& d = g->d;
  PV_CUDA(pv::launch_clear(d, st));
  PV_CUDA(pv::launch_bin(d, pos, h, m, m_uniform, st));
  PV_CUDA(pv::launch_scan(d, st));
  PV_CUDA(pv::launch_scatter(d, st));
  PV_CUDA(pv::launch_sort(d, pos, h, m, m_uniform, st));
  d.moved = 0;
  g->launches += g->n > 0 ? 11 : 3;  // clear, bin, scan (x2), scatter, gather, cell sorts (x2), big-cell sorts (x3)
  g->sorted = true;
  return PV_OK;
}

pv_status pv_update_positions(pv_grid* g, const double* pos, const float* h, void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (g->n > 0 && (!pos || !h)) return PV_ERR_INVALID_ARGUMENT;
  if (!g->sorted) return PV_ERR_NOT_SORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GridDev& d = g->d;
  PV_CUDA(cudaMemsetAsync(d.cell_Hmax, 0, (size_t)g->ncell * sizeof(float), st));
  PV_CUDA(cudaMemsetAsync(d.box_disp, 0, g->boxes.size() * sizeof(float), st));
  PV_CUDA(pv::launch_update(d, pos, h, st));
  d.moved = 1;
  g->launches += g->n > 0 ? 2 : 0;  // update, update_check
  return PV_OK;
}

pv_status pv_density(pv_grid* g, float* rho, float* drho_dh, int32_t* n_ngb, void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (g->n > 0 && !rho) return PV_ERR_INVALID_ARGUMENT;
  if (!g->sorted) return PV_ERR_NOT_SORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GridDev& d = g->d;
  cudaEvent_t t0, t1;  // (the plan kernel clears the pass's counters)
  PV_TRY(next_pair(g, 0, &t0, &t1));
  d.task_blk = g->task_blk[0];
  PV_CUDA(pv::launch_density(d, rho, drho_dh, n_ngb, g->num_sms, g->ctas[0], st, t0, t1));
  g->launches += g->n > 0 ? 6 : 0;  // plan_slots, plan_cells, plan_tasks, cells, tasks, finalize_t
  return PV_OK;
}

pv_status pv_density_symmetric(pv_grid* g, float* rho, float* drho_dh, int32_t* n_ngb,
                               void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (g->n > 0 && !rho) return PV_ERR_INVALID_ARGUMENT;
  if (!g->sorted) return PV_ERR_NOT_SORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GridDev& d = g->d;
  PV_CUDA(cudaMemsetAsync(d.ntask, 0, 5 * sizeof(int32_t), st));  // ccell_next among them
  PV_CUDA(cudaMemsetAsync(d.counters, 0, 2 * sizeof(unsigned long long), st));
  if (g->n) PV_CUDA(cudaMemsetAsync(d.acc, 0, 3 * (size_t)g->n * sizeof(long long), st));
  PV_CUDA(pv::launch_density_symmetric(d, rho, drho_dh, n_ngb, g->num_sms, st));
  g->launches += g->n > 0 ? 3 : 0;  // plan_slots, sweep, finalize
  return PV_OK;
}

pv_status pv_density_backward(pv_grid* g, const float* g_rho, const float* g_drho_dh,
                              float* g_pos, float* g_h, void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (g->n > 0 && (!g_rho || !g_pos)) return PV_ERR_INVALID_ARGUMENT;
  if (!g->sorted) return PV_ERR_NOT_SORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GridDev& d = g->d;
  cudaEvent_t t0, t1;
  PV_TRY(next_pair(g, 1, &t0, &t1));
  d.task_blk = g->task_blk[1];
  PV_CUDA(pv::launch_backward(d, g_rho, g_drho_dh, g_pos, g_h, g->num_sms, g->ctas[1], st, t0,
                              t1));
  g->launches += g->n > 0 ? 7 : 0;  // plan x3, prep, cells, tasks, finalize_t
  return PV_OK;
}

pv_status pv_count_candidates(pv_grid* g, void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (!g->sorted) return PV_ERR_NOT_SORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PV_CUDA(cudaMemsetAsync(g->d.counters + 2, 0, 14 * sizeof(unsigned long long), st));
  PV_CUDA(pv::launch_count_candidates(g->d, st));
  g->launches += 3;
  return PV_OK;
}

pv_status pv_grid_sync(pv_grid* g, void* stream) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  PV_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  uint32_t flags = 0;
  PV_CUDA(cudaMemcpy(&flags, g->d.flags, sizeof(flags), cudaMemcpyDeviceToHost));
  return flags ? PV_ERR_DEVICE : PV_OK;
}

pv_status pv_grid_stats(pv_grid* g, pv_stats* out) {
  if (!g || !out) return PV_ERR_INVALID_ARGUMENT;
  PV_CUDA(cudaDeviceSynchronize());
  int32_t sc[4];
  unsigned long long cnt[16];
  PV_CUDA(cudaMemcpy(sc, g->d.flags, sizeof(sc), cudaMemcpyDeviceToHost));
  PV_CUDA(cudaMemcpy(cnt, g->d.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof(*out));
  out->n_particles = g->n;
  out->n_cells = g->ncell;
  out->max_cell_count = g->sorted ? sc[2] : 0;
  out->device_flags = (uint32_t)sc[0];
  out->interactions = (int64_t)cnt[0];
  out->guard_pairs = (int64_t)cnt[1];
  out->candidates = (int64_t)cnt[2];
  out->candidates_adjoint = (int64_t)cnt[3];
  out->pairs_adjoint = (int64_t)cnt[4];
  for (int c = 0; c < 4; c++) {
    out->orientation[c][0] = (int64_t)cnt[8 + 2 * c];
    out->orientation[c][1] = (int64_t)cnt[9 + 2 * c];
  }
  out->device_bytes = (int64_t)g->bytes;
  out->kernel_launches = g->launches;
  return out->device_flags ? PV_ERR_DEVICE : PV_OK;
}

pv_status pv_grid_set_tuning(pv_grid* g, const pv_tuning* t) {
  if (!g || !t) return PV_ERR_INVALID_ARGUMENT;
  for (int r : t->reserved)
    if (r != 0) return PV_ERR_INVALID_ARGUMENT;
  const int d = t->density_ctas_per_sm ? t->density_ctas_per_sm : pv::kDensityCtasDefault;
  const int b = t->backward_ctas_per_sm ? t->backward_ctas_per_sm : pv::kBackwardCtasDefault;
  const int td = t->density_task_block ? t->density_task_block : pv::kTaskBlkDefault;
  const int tb = t->backward_task_block ? t->backward_task_block : pv::kTaskBlkDefault;
  auto blk_ok = [](int v) { return v == 64 || v == 128 || v == 256; };
  if (d < 1 || d > 4 || b < 1 || b > 3 || !blk_ok(td) || !blk_ok(tb))
    return PV_ERR_INVALID_ARGUMENT;
  g->ctas[0] = d;
  g->ctas[1] = b;
  g->task_blk[0] = td;
  g->task_blk[1] = tb;
  return PV_OK;
}

pv_status pv_grid_get_tuning(const pv_grid* g, pv_tuning* out) {
  if (!g || !out) return PV_ERR_INVALID_ARGUMENT;
  std::memset(out, 0, sizeof(*out));
  out->density_ctas_per_sm = g->ctas[0];
  out->backward_ctas_per_sm = g->ctas[1];
  out->density_task_block = g->task_blk[0];
  out->backward_task_block = g->task_blk[1];
  return PV_OK;
}

pv_status pv_raw_interactions(const float* xi, int64_t n_i, const float* xj, int64_t n_j,
                              float H, int32_t reps, float* out, void* stream) {
  if (n_i < 0 || n_j < 0 || reps < 1 || !(H > 0.0f) || !std::isfinite(H))
    return PV_ERR_INVALID_ARGUMENT;
  if (n_i > 0x7fffffff || n_j > 0x7fffffff) return PV_ERR_TOO_LARGE;
  if (n_i > 0 && (!xi || !out || (n_j > 0 && !xj))) return PV_ERR_INVALID_ARGUMENT;
  if ((reinterpret_cast<uintptr_t>(xi) | reinterpret_cast<uintptr_t>(xj) |
       reinterpret_cast<uintptr_t>(out)) & 15u)
    return PV_ERR_INVALID_ARGUMENT;
  PV_CUDA(pv::launch_raw_density(reinterpret_cast<const float4*>(xi), (int)n_i,
                                 reinterpret_cast<const float4*>(xj), (int)n_j, H, reps,
                                 reinterpret_cast<float2*>(out),
                                 static_cast<cudaStream_t>(stream)));
  return PV_OK;
}

pv_status pv_fp32_probe(int32_t packed, int32_t iters, float* sink, int64_t threads,
                        double* flops, void* stream) {
  if (iters < 1 || threads < 0 || threads % 256 || !flops || (threads > 0 && !sink))
    return PV_ERR_INVALID_ARGUMENT;
  if (threads / 256 > 0x7fffffff) return PV_ERR_TOO_LARGE;
  PV_CUDA(pv::launch_fp32_probe(packed != 0, iters, sink, threads, flops,
                                static_cast<cudaStream_t>(stream)));
  return PV_OK;
}

pv_status pv_grid_set_slot_mask(pv_grid* g, uint32_t mask) {
  if (!g || (mask & ~pv::kAllSlots)) return PV_ERR_INVALID_ARGUMENT;
  g->d.slot_mask = mask;
  return PV_OK;
}

pv_status pv_grid_time_sweeps(pv_grid* g, int enable) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  if (enable && g->ev.empty()) {
    g->ev.assign(2 * pv_grid::kRing * 2, nullptr);
    for (auto& e : g->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        for (auto& f : g->ev)
          if (f) cudaEventDestroy(f);
        g->ev.clear();
        return cuda_fail(r, "cudaEventCreate");
      }
    }
  }
  for (int k = 0; k < 2; k++)
    while (g->pending[k]) PV_TRY(retire_oldest(g, k));
  g->timing = enable != 0 && !g->ev.empty();
  g->ms[0] = g->ms[1] = 0.0;
  g->timed[0] = g->timed[1] = 0;
  return PV_OK;
}

pv_status pv_grid_sweep_times(pv_grid* g, double* ms, int64_t* launches) {
  if (!g) return PV_ERR_INVALID_ARGUMENT;
  for (int k = 0; k < 2; k++)
    while (g->pending[k]) PV_TRY(retire_oldest(g, k));
  for (int k = 0; k < 2; k++) {
    if (ms) ms[k] = g->ms[k];
    if (launches) launches[k] = g->timed[k];
    g->ms[k] = 0.0;
    g->timed[k] = 0;
  }
  return PV_OK;
}

}  // extern "C"
