// pv_noalloc.cu -- pv_density_static: sort + density of one periodic box
// without allocating anything.
//
// Who needs this: callers that must not call cudaMalloc/cudaFree while they
// run -- an application whose memory pool owns all device memory and forbids
// allocations behind its back, a plugin loaded into such a host, or a
// latency-critical loop that cannot afford the implicit device
// synchronisation and allocator locks of cudaMalloc/cudaFree.  They pass
// their own inputs and outputs; every intermediate array lives in one
// file-scope __device__ array of fixed size that each GPU loading this
// library keeps until the process exits.
//
// The kernels are the same ones pv_sort_cells + pv_density launch; only the
// scratch pointers differ (carved from the static array instead of a
// pv_grid's cudaMalloc'd buffers).
#include <cuda_runtime.h>

#include <cmath>

#include "pv_internal.cuh"

namespace {

constexpr int64_t kMaxParticles = PV_STATIC_MAX_PARTICLES;
constexpr int64_t kMaxCells = PV_STATIC_MAX_CELLS;
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Bytes of scratch for n particles and c cells (forward pass only).
constexpr size_t scratch_bytes(int64_t n, int64_t c) {
  const size_t N = (size_t)n, C = (size_t)c;
  return align_up(sizeof(pv::BoxDev)) + align_up(sizeof(int64_t)) +
         4 * align_up(C * sizeof(int32_t)) + align_up((C + 1) * sizeof(int32_t)) +
         align_up((size_t)pv::scan_tiles(c) * sizeof(int32_t)) +
         align_up(C * sizeof(float)) +
         align_up(pv::kNSlot * C * sizeof(int4)) + 3 * align_up(C * sizeof(int32_t)) +  // plan
         2 * align_up(N * sizeof(int32_t)) +          // pcell, prank
         2 * align_up(N * sizeof(float4)) + align_up(N * sizeof(float)) +
         align_up(N * sizeof(int32_t)) + align_up(3 * N * sizeof(double)) +
         align_up(pv::kNDir * N * sizeof(uint16_t)) + align_up(pv::kNDir * N * sizeof(float)) +
         align_up(3 * N * sizeof(long long)) +
         align_up((size_t)((int64_t)pv::kNSlot * (n / pv::kTaskBlkMin + c) + 64) * sizeof(int4)) +
         align_up(16 * sizeof(int32_t)) + align_up(16 * sizeof(unsigned long long));
}

constexpr size_t kScratchBytes = scratch_bytes(kMaxParticles, kMaxCells);

}  // namespace

// The scratch itself.  Host code must not pass this name to a kernel: on the
// host it only stands for the symbol; the device address comes from
// cudaGetSymbolAddress (see static_scratch below).
static __device__ __align__(256) unsigned char g_pv_static_scratch[kScratchBytes];

namespace {

// Device address of the scratch on the current device.  Looked up on every
// call, not cached: after cudaDeviceReset the module is loaded again and the
// array may sit at another address.
cudaError_t static_scratch(void** out) { return cudaGetSymbolAddress(out, g_pv_static_scratch); }

template <typename T>
T* carve(unsigned char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += align_up(count * sizeof(T));
  return p;
}

// Writes the box description and the cell -> box map (all zero: one box)
// into the scratch from kernel parameters, so no host buffer has to outlive
// the call.
__global__ void k_static_setup(pv::BoxDev* box, pv::BoxDev val, int64_t* first, int32_t* cell_box,
                               int ncell) {
  pv::pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *box = val;
    *first = 0;
  }
  if (i < ncell) cell_box[i] = 0;
}

// the same error record as the other entry points (pv_last_cuda_error)
pv_status fail(cudaError_t e, const char* what) { return pv::record_cuda_error(e, what); }

}  // namespace

extern "C" pv_status pv_density_static(const double* pos, const float* h, const float* m,
                                       float m_uniform, int64_t n, double L, int32_t nc,
                                       double gamma, float* rho, float* drho_dh,
                                       int32_t* n_ngb, uint32_t* flags_out, void* stream) {
  if (n < 0 || !(L > 0.0) || L != L) return PV_ERR_INVALID_ARGUMENT;
  if (nc < 3) return PV_ERR_CELL_TOO_SMALL;
  const int64_t ncell = (int64_t)nc * nc * nc;
  if (n > kMaxParticles || ncell > kMaxCells) return PV_ERR_TOO_LARGE;
  if (n > 0 && (!pos || !h || !rho)) return PV_ERR_INVALID_ARGUMENT;
  if (!m && !(m_uniform >= 0.0f && m_uniform < 3.0e38f)) return PV_ERR_INVALID_ARGUMENT;
  if (!(gamma > 0.0)) gamma = 1.825742;  // also maps a NaN to the default
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  void* base = nullptr;
  cudaError_t e = static_scratch(&base);
  if (e != cudaSuccess) return fail(e, "cudaGetSymbolAddress");
  int dev = 0, num_sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail(e, "cudaDeviceGetAttribute");

  const size_t N = (size_t)n, C = (size_t)ncell;
  unsigned char* cur = static_cast<unsigned char*>(base);
  pv::GridDev d{};
  pv::BoxDev* box = carve<pv::BoxDev>(cur, 1);
  int64_t* first = carve<int64_t>(cur, 1);
  d.cell_count = carve<int32_t>(cur, C);
  d.cell_box = carve<int32_t>(cur, C);
  d.big_cells = carve<int32_t>(cur, C);
  d.small_cells = carve<int32_t>(cur, C);
  d.tile_sum = carve<int32_t>(cur, (size_t)pv::scan_tiles(ncell));
  d.cell_start = carve<int32_t>(cur, C + 1);
  d.cell_Hmax = carve<float>(cur, C);
  d.plan = carve<int4>(cur, pv::kNSlot * C);
  d.ccells = carve<int32_t>(cur, C);
  d.tcells = carve<int32_t>(cur, C);
  d.ycells = carve<int32_t>(cur, C);
  d.pcell = carve<int32_t>(cur, N);
  d.prank = carve<int32_t>(cur, N);
  d.xm = carve<float4>(cur, N);
  d.xm_ref = carve<float4>(cur, N);
  d.hs = carve<float>(cur, N);
  d.orig = carve<int32_t>(cur, N);
  d.pos64 = carve<double>(cur, 3 * N);
  d.perm = carve<uint16_t>(cur, pv::kNDir * N);
  d.dist = carve<float>(cur, pv::kNDir * N);
  d.acc = carve<long long>(cur, 3 * N);
  d.max_tasks = (int32_t)pv::max_tasks_for(n, ncell);
  d.task_blk = pv::kTaskBlkDefault;
  d.slot_mask = pv::kAllSlots;
  d.moved = 0;
  d.tasks = carve<int4>(cur, (size_t)d.max_tasks);
  int32_t* sc = carve<int32_t>(cur, 16);
  d.counters = carve<unsigned long long>(cur, 16);
  if ((size_t)(cur - static_cast<unsigned char*>(base)) > kScratchBytes) return PV_ERR_TOO_LARGE;
  d.flags = reinterpret_cast<uint32_t*>(sc + 0);
  d.m_max = reinterpret_cast<float*>(sc + 1);  // one box
  d.box_disp = reinterpret_cast<float*>(sc + 9);  // one box, zero (the scalars are cleared)
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
  d.gacc = nullptr;
  d.bwd_cmax = nullptr;
  d.bwd_hmin = nullptr;
  d.bx = nullptr;
  d.ba = nullptr;
  d.n_boxes = 1;
  d.n = (int32_t)n;
  d.ncell = (int32_t)ncell;
  d.gamma = (float)gamma;
  d.gamma_d = gamma;
  d.boxes = box;
  d.box_first = first;

  pv::BoxDev B{};
  B.L = L;
  B.inv_L = 1.0 / L;
  B.edge = L / nc;
  B.inv_edge = nc / L;
  B.edge_f = (float)B.edge;
  B.pad = (float)std::ldexp(B.edge, -18);
  B.guard = 0.0f;
  B.h_limit = pv::support_h_limit(gamma, B.edge);
  B.nc = nc;
  B.cell_base = 0;
  B.first = 0;
  B.n = n;

  // The array keeps whatever the previous call left: clear what must start
  // at zero (occupancies, cell maxima, flags and counters, accumulators).
  k_static_setup<<<(int)((C + 255) / 256), 256, 0, st>>>(box, B, first, d.cell_box, (int)C);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "k_static_setup");
  if ((e = cudaMemsetAsync(d.cell_count, 0, C * sizeof(int32_t), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc, 0, 16 * sizeof(int32_t), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d.cell_Hmax, 0, C * sizeof(float), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d.counters, 0, 16 * sizeof(unsigned long long), st)) != cudaSuccess ||
      (N && (e = cudaMemsetAsync(d.acc, 0, 3 * N * sizeof(long long), st)) != cudaSuccess))
    return fail(e, "cudaMemsetAsync");
  if ((e = pv::launch_bin(d, pos, h, m, m_uniform, st)) != cudaSuccess) return fail(e, "bin");
  if ((e = pv::launch_scan(d, st)) != cudaSuccess) return fail(e, "scan");
  if ((e = pv::launch_scatter(d, st)) != cudaSuccess) return fail(e, "scatter");
  if ((e = pv::launch_sort(d, pos, h, m, m_uniform, st)) != cudaSuccess) return fail(e, "sort");
  if ((e = pv::launch_density(d, rho, drho_dh, n_ngb, num_sms, pv::kDensityCtasDefault, st)) != cudaSuccess)
    return fail(e, "density");
  if (flags_out &&
      (e = cudaMemcpyAsync(flags_out, d.flags, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)) !=
          cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  return PV_OK;
}
