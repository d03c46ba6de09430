// pv_density.cu -- the density gather over the sorted cell pairs.
//
// For every cell a and each of its 27 neighbour slots (the cell itself and
// the 26 cells b = a + o), the particles of a that can reach b are visited
// in order of decreasing projection on the axis u = o/|o| (nearest to the
// common face first, Section 3.1), and each gathers from the particles of b
// in order of increasing projection, stopping once the projected distance
// reaches its own support (Section 2 and Section 3.3).  Particles of a that
// lie further than the cell's largest support from b are skipped ("first_a",
// Section 3.3).  The self slot uses a two-sided window on the axis (0,0,1).
//
// GPU mapping (gather only, no scatter, so no atomics between particles):
//   * a task is (cell a, slot o, block of up to 128 particles of a in the
//     slot's order); the plan kernel enumerates them and their window in b;
//   * one CTA (4 warps) pops tasks from a device queue; it stages the window
//     of b in sorted order into shared memory (the particle cache of Section
//     3.2: FP32 offsets, SoA order of the sweep) and each warp sweeps it for
//     its 32 particles, one particle per lane;
//   * the per-particle partial sums of a task are added to fixed-point
//     accumulators (integer atomics, so the result is independent of the
//     order in which tasks run), converted by the finalize kernel.
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {

namespace {

constexpr int kBlkI = 128;    // particles of a per task
constexpr int kTileJ = 1024;  // particles of b per shared-memory tile

struct Task {
  int a, o, p0, p1, j0, j1;
};

__device__ __forceinline__ Task decode(int4 t) {
  Task r;
  r.a = t.x;
  r.o = t.y;
  r.p0 = t.z & 0xffff;
  r.p1 = (int)((unsigned)t.z >> 16);
  r.j0 = t.w & 0xffff;
  r.j1 = (int)((unsigned)t.w >> 16);
  return r;
}

// Projection of the t-th particle of cell c (start cs, count cnt) in the
// ascending-along-u order of slot (k, s), plus the cell shift `off`.
__device__ __forceinline__ float proj_asc(const GridDev& g, int k, int s, int cs, int cnt, int t,
                                          float off) {
  return s * g.dist[(size_t)k * g.n + cs + order_pos(s, t, cnt)] + off;
}

// ---- plan -------------------------------------------------------------------
// One thread per (cell a, slot o).  Counts the particles of a that can reach
// b (first_a trimming with the cell's largest support) and, per block of
// kBlkI of them, the window of b they can touch.  `wide` widens every window
// to the larger of the two cells' largest supports (backward pass).
__global__ void k_plan(GridDev g, int wide) {
  if (*g.flags) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell * kNSlot) return;
  const int a = idx / kNSlot, o = idx % kNSlot;
  const int na = g.cell_count[a];
  if (na == 0) return;
  const int b = neighbour_cell(g, a, o);
  const int nb = g.cell_count[b];
  if (nb == 0) return;
  const BoxDev& B = g.boxes[g.cell_box[a]];
  const Slot sl = slot_info(o);
  const int ca = g.cell_start[a], cb = g.cell_start[b];
  float reach = g.cell_Hmax[a];
  if (wide) reach = fmaxf(reach, g.cell_Hmax[b]);
  reach += B.pad;
  const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
  int nblk, nI;
  if (o == kSelfSlot) {
    nI = na;
  } else {
    // descending order along u: position p <-> ascending index na-1-p
    const float db_min = proj_asc(g, sl.k, sl.s, cb, nb, 0, off);
    int lo = 0, hi = na;  // nI = #{p : d(p) + reach > db_min}, d decreasing in p
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      float d = proj_asc(g, sl.k, sl.s, ca, na, na - 1 - mid, 0.0f);
      if (d + reach > db_min) lo = mid + 1; else hi = mid;
    }
    nI = lo;
  }
  if (nI == 0) return;
  nblk = (nI + kBlkI - 1) / kBlkI;
  const int base = atomicAdd(g.ntask, nblk);
  if (base + nblk > g.max_tasks) {  // cannot happen with the allocated bound
    atomicOr(g.flags, PV_FLAG_CELL_OVERFLOW);
    return;
  }
  for (int bk = 0; bk < nblk; bk++) {
    const int p0 = bk * kBlkI, p1 = min(nI, p0 + kBlkI);
    int j0, j1;
    if (o == kSelfSlot) {
      const float* d = g.dist + cb;  // axis 0, ascending
      j0 = upper_bound_f(d, nb, d[p0] - reach);
      j1 = lower_bound_f(d, nb, d[p1 - 1] + reach);
    } else {
      const float dmax = proj_asc(g, sl.k, sl.s, ca, na, na - 1 - p0, 0.0f);
      const float lim = dmax + reach;
      int lo = 0, hi = nb;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (proj_asc(g, sl.k, sl.s, cb, nb, mid, off) < lim) lo = mid + 1; else hi = mid;
      }
      j0 = 0;
      j1 = lo;
    }
    g.tasks[base + bk] = make_int4(a, o, (int)((unsigned)p0 | ((unsigned)p1 << 16)),
                                   (int)((unsigned)j0 | ((unsigned)j1 << 16)));
  }
}

// ---- forward sweep -------------------------------------------------------------

struct LaneI {
  float x, y, z;           // position of i in b's frame: x'_i - o edge
  float Hsq_hi, Hsq_lo;    // guard band around H_i^2
  float Hinv2;             // 1 / H_i^2
  double Hd;               // FP64 support, for the guard re-decision
  int si;                  // cell-order index of i
  float rho, D;            // sum_j m_j wh, sum_j m_j th
  int n;                   // pairs with r < H_i (j = i included)
};

__global__ void __launch_bounds__(kBlkI) k_density_tasks(GridDev g) {
  __shared__ float4 s_x[kTileJ];
  __shared__ float s_d[kTileJ];
  __shared__ int s_j[kTileJ];
  __shared__ int s_task;
  if (*g.flags) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntask = *g.ntask;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(g.task_next, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= ntask) break;
    const Task tk = decode(g.tasks[t]);
    const int a = tk.a, o = tk.o;
    const int b = neighbour_cell(g, a, o);
    const int na = g.cell_count[a], nb = g.cell_count[b];
    const int ca = g.cell_start[a], cb = g.cell_start[b];
    const BoxDev B = g.boxes[g.cell_box[a]];
    const Slot sl = slot_info(o);
    const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    const size_t kbase = (size_t)sl.k * g.n;

    // lane setup
    LaneI L;
    const int p = tk.p0 + warp * 32 + lane;
    const bool valid = p < tk.p1;
    float d_lo = 3.0e38f, d_hi = -3.0e38f;
    L.rho = 0.0f; L.D = 0.0f; L.n = 0;
    L.x = L.y = L.z = 0.0f;
    L.Hsq_hi = -1.0f; L.Hsq_lo = -1.0f; L.Hinv2 = 0.0f; L.Hd = 0.0; L.si = 0;
    if (valid) {
      const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
      const int il = g.perm[kbase + ca + pos_i];
      L.si = ca + il;
      const float4 xi = g.xm[L.si];
      const float h = g.hs[L.si];
      const float H = g.gamma * h;
      L.x = xi.x - sl.ox * B.edge_f;
      L.y = xi.y - sl.oy * B.edge_f;
      L.z = xi.z - sl.oz * B.edge_f;
      const float Hsq = H * H, gb = guard_band(H, B.edge_f);
      L.Hsq_hi = Hsq + gb;
      L.Hsq_lo = Hsq - gb;
      L.Hinv2 = 1.0f / Hsq;
      L.Hd = g.gamma_d * (double)h;
      const float di = sl.s * g.dist[kbase + ca + pos_i];
      d_lo = di - H - B.pad;
      d_hi = di + H + B.pad;
    }
    // window of the warp (in b's ascending order)
    float w_lo = d_lo, w_hi = d_hi;
    for (int s = 16; s > 0; s >>= 1) {
      w_lo = fminf(w_lo, __shfl_xor_sync(0xffffffffu, w_lo, s));
      w_hi = fmaxf(w_hi, __shfl_xor_sync(0xffffffffu, w_hi, s));
    }
    int guards = 0;
    for (int j0 = tk.j0; j0 < tk.j1; j0 += kTileJ) {
      const int len = min(kTileJ, tk.j1 - j0);
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int pos_j = order_pos(sl.s, j0 + e, nb);
        const int jl = g.perm[kbase + cb + pos_j];
        s_x[e] = g.xm[cb + jl];
        s_d[e] = sl.s * g.dist[kbase + cb + pos_j] + off;
        s_j[e] = cb + jl;
      }
      __syncthreads();
      if (w_hi > w_lo) {
        const int lo = (o == kSelfSlot) ? upper_bound_f(s_d, len, w_lo) : 0;
        const int hi = lower_bound_f(s_d, len, w_hi);
        for (int e = lo; e < hi; e++) {
          const float4 xj = s_x[e];
          const float dx = L.x - xj.x, dy = L.y - xj.y, dz = L.z - xj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (r2 < L.Hsq_hi) {
            bool in = true;
            if (r2 >= L.Hsq_lo) {
              in = guard_inside(g.pos64, L.si, s_j[e], B.L, B.inv_L, L.Hd);
              guards++;
            }
            if (in) {
              const float q2 = r2 * L.Hinv2;
              const float q = q2 * rsqrtf(fmaxf(q2, 1e-30f));
              float wh, th;
              spline_half(q, q2, wh, th);
              L.rho = fmaf(xj.w, wh, L.rho);
              L.D = fmaf(xj.w, th, L.D);
              L.n++;
            }
          }
        }
      }
      __syncthreads();
    }
    if (valid && L.n > 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[L.si]),
                (unsigned long long)__float2ll_rn(L.rho * (float)kFixScale));
      atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[(size_t)g.n + L.si]),
                (unsigned long long)__float2ll_rn(L.D * (float)kFixScale));
      atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[2 * (size_t)g.n + L.si]),
                (unsigned long long)L.n);
    }
    if (guards) atomicAdd(&g.counters[1], (unsigned long long)guards);
  }
}

// ---- finalize: fixed point -> caller order ---------------------------------------
__global__ void k_finalize(GridDev g, float* __restrict__ rho, float* __restrict__ drho_dh,
                           int32_t* __restrict__ n_ngb) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  long long nn = 0;
  if (s < g.n && !*g.flags) {
    const int i = g.orig[s];
    const double h = (double)g.hs[s];
    const double H = g.gamma_d * h;
    const double c = (16.0 / 3.14159265358979323846) * (double)*g.m_max / (H * H * H);
    const double sr = (double)g.acc[s] * kFixInv;
    const double sd = (double)g.acc[(size_t)g.n + s] * kFixInv;
    nn = g.acc[2 * (size_t)g.n + s] - 1;  // the self pair j = i
    rho[i] = (float)(c * sr);
    if (drho_dh) drho_dh[i] = (float)(-c * sd / h);
    if (n_ngb) n_ngb[i] = (int32_t)nn;
  }
  if (s < g.n) {
    g.acc[s] = 0;
    g.acc[(size_t)g.n + s] = 0;
    g.acc[2 * (size_t)g.n + s] = 0;
  }
  for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
  if ((threadIdx.x & 31) == 0 && nn) atomicAdd(&g.counters[0], (unsigned long long)nn);
}

// ---- candidates of the method's windows (diagnostic) -------------------------------
// One thread per (cell a, slot o): for every particle of a, the number of
// particles of b inside its window on the sorted axis (exact per-particle
// window, no padding): |d_j - d_i| < H_i for the self slot, d_j < d_i + H_i
// for a neighbour slot.
__global__ void k_count_candidates(GridDev g) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt = 0;
  if (idx < g.ncell * kNSlot && !*g.flags) {
    const int a = idx / kNSlot, o = idx % kNSlot;
    const int na = g.cell_count[a];
    const int b = na ? neighbour_cell(g, a, o) : a;
    const int nb = g.cell_count[b];
    if (na && nb) {
      const BoxDev& B = g.boxes[g.cell_box[a]];
      const Slot sl = slot_info(o);
      const int ca = g.cell_start[a], cb = g.cell_start[b];
      const size_t kb = (size_t)sl.k * g.n;
      const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
      for (int p = 0; p < na; p++) {
        const int pos = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
        const float H = g.gamma * g.hs[ca + g.perm[kb + ca + pos]];
        const float di = sl.s * g.dist[kb + ca + pos];
        if (o == kSelfSlot) {
          const float* d = g.dist + cb;
          cnt += lower_bound_f(d, nb, di + H) - upper_bound_f(d, nb, di - H);
        } else {
          int lo = 0, hi = nb;
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (proj_asc(g, sl.k, sl.s, cb, nb, mid, off) < di + H) lo = mid + 1; else hi = mid;
          }
          cnt += lo;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&g.counters[2], cnt);
}

}  // namespace

cudaError_t launch_plan(const GridDev& g, int wide, cudaStream_t st) {
  const int nthr = g.ncell * kNSlot;
  if (nthr == 0) return cudaSuccess;
  k_plan<<<(nthr + 255) / 256, 256, 0, st>>>(g, wide);
  return cudaGetLastError();
}

int64_t max_tasks_for(int64_t n, int64_t ncell) {
  return (int64_t)kNSlot * (n / kBlkI + ncell) + 64;
}

cudaError_t launch_density(const GridDev& g, float* rho, float* drho_dh, int32_t* n_ngb,
                           int num_sms, cudaStream_t st) {
  cudaError_t e = launch_plan(g, 0, st);
  if (e != cudaSuccess) return e;
  if (g.n == 0) return cudaSuccess;
  k_density_tasks<<<num_sms * 8, kBlkI, 0, st>>>(g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_finalize<<<(g.n + 255) / 256, 256, 0, st>>>(g, rho, drho_dh, n_ngb);
  return cudaGetLastError();
}

cudaError_t launch_count_candidates(const GridDev& g, cudaStream_t st) {
  const int nthr = g.ncell * kNSlot;
  if (nthr == 0) return cudaSuccess;
  k_count_candidates<<<(nthr + 255) / 256, 256, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace pv
