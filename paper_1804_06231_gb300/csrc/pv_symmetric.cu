// pv_symmetric.cu -- the density with the paper's symmetric pair update.
//
// Section 3.3 (last paragraph): instead of each particle of a gathering from b
// and, separately, each particle of b gathering from a, one sweep of the cell
// pair evaluates every pair (i, j) once and updates both particles, the cache
// holding the particles of both cells that can reach the other one.  In the
// gather form of this density (each particle uses its own support, Section
// 3.1) a pair contributes to i when r < H_i and to j when r < H_j, so the
// sweep's window is the larger of the two reaches.
//
// GPU mapping: a work unit is a cell a with one of its 14 half-stencil slots,
// the cell itself or the neighbour b = a + v_k along one of the 13 axes; every
// unordered pair of cells then appears in exactly one unit.  A persistent CTA
// takes units from a counter.  It stages b's window (sorted, trimmed by the
// plan to what a's farthest-reaching particle can touch, in tiles) in shared
// memory with one fixed-point accumulator per staged particle; its warps take
// runs of 32 of a's reaching particles, pre-filter the window by r^2 <
// max(H_i^2, H_j^2) (plus guard) into per-lane hit masks, and evaluate each
// hit once for both sides: i's terms in the lane's registers, j's terms added
// to j's shared accumulator.  Within the self cell a lane pairs only with the
// particles after its own in the sorted order.  Both sides end in 64-bit
// fixed-point global sums, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {
namespace {

constexpr int kSymThreads = 256;
constexpr int kSymTile = 512;        // staged particles of b per tile
constexpr int kSymSlots = 14;        // self + the 13 positive axes
constexpr int kSymPad = 32;

__device__ __forceinline__ int sym_slot(int q) { return q == 0 ? kSelfSlot : kSelfSlot + q; }

struct SymShared {
  float4 x[kSymTile + kSymPad];   // {x', y', z', H^2 + guard} of b, in b's frame
  float4 a[kSymTile + kSymPad];   // {m/m_max, H, 1/H^2, |1-q| guard band}
  float d[kSymTile];              // projection along the slot's axis (ascending)
  int j[kSymTile];                // cell-order index
  unsigned long long accw[kSymTile], accd[kSymTile];
  int accn[kSymTile];
  int unit, item_next;
};

// rho and drho/dh terms of one side of a pair (half-scaled spline, see
// spline_half) and its count, the count re-decided in FP64 near the cut-off.
struct Side {
  float wh, th;
  int n;
};

__device__ __forceinline__ Side side_terms(float r2, float hinv2, float dq, const GridDev& g,
                                           const BoxDev& B, int si, int sj, float h_s) {
  Side o;
  const float q = sqrt_approx(r2 * hinv2);
  spline_half(fminf(q, 1.0f), o.wh, o.th);
  o.n = q < 1.0f ? 1 : 0;
  if (fabsf(1.0f - q) < dq)
    o.n = guard_inside(g.pos64, si, sj, B.L, B.inv_L, g.gamma_d * (double)h_s) ? 1 : 0;
  return o;
}

__global__ void __launch_bounds__(kSymThreads) k_density_sym(GridDev g) {
  pdl_enter();
  __shared__ SymShared sh;
  if (*g.flags) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nunits = g.ncell * kSymSlots;
  const double fix = kFixScale;
  for (;;) {
    __syncthreads();  // every thread has read the previous unit
    if (tid == 0) sh.unit = atomicAdd(g.ccell_next, 1);
    __syncthreads();
    const int unit = sh.unit;
    if (unit >= nunits) break;
    const int a = unit / kSymSlots, o = sym_slot(unit % kSymSlots);
    const bool self = o == kSelfSlot;
    const int na = g.cell_count[a];
    const int b = neighbour_cell(g, a, o);
    const int nb = g.cell_count[b];
    const int4 pl = g.plan[(size_t)a * kNSlot + o];
    const int I = self ? na : pl.x, J1 = self ? na : pl.z;
    if (I == 0 || J1 == 0) continue;  // uniform over the CTA; no shared state touched
    const int ca = g.cell_start[a], cb = g.cell_start[b];
    const BoxDev B = g.boxes[g.cell_box[a]];
    const Slot sl = slot_info(o);
    const float offv = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    const float padw = window_pad(g, B, g.cell_box[a]);
    const float Hmax_b = g.cell_Hmax[b];
    const size_t kb = (size_t)sl.k * g.n;
    const int nitems = (I + 31) >> 5;
    for (int j0 = 0; j0 < J1; j0 += kSymTile) {
      const int len = min(kSymTile, J1 - j0);
      for (int e = tid; e < len; e += kSymThreads) {
        const int pos = order_pos(sl.s, j0 + e, nb);
        const int sj = cb + g.perm[kb + cb + pos];
        const float4 xm = g.xm[sj];
        const float h = g.hs[sj];
        const float H = g.gamma * h, Hsq = H * H, gb = guard_band(H, B.edge_f);
        const float hinv2 = __fdividef(1.0f, Hsq);
        sh.x[e] = make_float4(xm.x, xm.y, xm.z, Hsq + gb);
        sh.a[e] = make_float4(xm.w, h, hinv2, gb * hinv2);
        sh.d[e] = sl.s * g.dist[kb + cb + pos] + offv;
        sh.j[e] = sj;
        sh.accw[e] = 0;
        sh.accd[e] = 0;
        sh.accn[e] = 0;
      }
      if (tid == 0) sh.item_next = 0;
      __syncthreads();
      for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&sh.item_next, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const int p = (it << 5) + lane;
        const bool valid = p < I;
        float xi = 0.0f, yi = 0.0f, zi = 0.0f, Ei = -1.0f, hinv_i = 0.0f, dq_i = 0.0f, mi = 0.0f,
              hi = 1.0f;
        int si = 0;
        float d_hi = -3.0e38f;
        int after = 0;  // self cell: only partners after this position (tile index)
        if (valid) {
          const int pos_i = self ? p : order_pos(sl.s, na - 1 - p, na);
          si = ca + g.perm[kb + ca + pos_i];
          const float4 xm = g.xm[si];
          hi = g.hs[si];
          const float H = g.gamma * hi, Hsq = H * H, gb = guard_band(H, B.edge_f);
          xi = xm.x - sl.ox * B.edge_f;
          yi = xm.y - sl.oy * B.edge_f;
          zi = xm.z - sl.oz * B.edge_f;
          Ei = Hsq + gb;
          hinv_i = __fdividef(1.0f, Hsq);
          dq_i = gb * hinv_i;
          mi = xm.w;
          const float di = sl.s * g.dist[kb + ca + pos_i];
          d_hi = di + fmaxf(H, Hmax_b) + padw;
          after = self ? p + 1 - j0 : 0;
        }
        // the window of the run: up to the farthest reach of its particles
        float w_hi = d_hi;
        for (int s = 16; s > 0; s >>= 1) w_hi = fmaxf(w_hi, __shfl_xor_sync(0xffffffffu, w_hi, s));
        const int hi_e = lower_bound_f(sh.d, len, w_hi);
        int lo_e = self ? max(0, (it << 5) + 1 - j0) : 0;
        float pw = 0.0f, pd = 0.0f;
        int pn = 0;
        for (int base = lo_e; base < hi_e; base += 32) {
          const int cnt = min(32, hi_e - base);
          unsigned m = 0;
          for (int c = 0; c < cnt; c++) {
            const float4 q = sh.x[base + c];
            const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const bool hit = valid && base + c >= after && r2 < fmaxf(Ei, q.w);
            m |= (hit ? 1u : 0u) << c;
          }
          while (m != 0u) {
            const int c = __ffs(m) - 1;
            m &= m - 1u;
            const int e = base + c;
            const float4 q = sh.x[e];
            const float4 qa = sh.a[e];
            const float dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 < Ei) {  // i gathers j
              const Side s = side_terms(r2, hinv_i, dq_i, g, B, si, sh.j[e], hi);
              pw = fmaf(qa.x, s.wh, pw);
              pd = fmaf(qa.x, s.th, pd);
              pn += s.n;
            }
            if (r2 < q.w) {  // j gathers i
              const Side s = side_terms(r2, qa.z, qa.w, g, B, sh.j[e], si, qa.y);
              atomicAdd(&sh.accw[e], (unsigned long long)__float2ll_rn(mi * s.wh * (float)fix));
              atomicAdd(&sh.accd[e], (unsigned long long)__float2ll_rn(mi * s.th * (float)fix));
              if (s.n) atomicAdd(&sh.accn[e], s.n);
            }
          }
        }
        if (valid && self && j0 == 0) {  // the pair j = i, once
          float wh0, th0;
          spline_half(0.0f, wh0, th0);
          pw = fmaf(mi, wh0, pw);
          pd = fmaf(mi, th0, pd);
          pn += 1;
        }
        if (valid && (pn != 0 || pw != 0.0f)) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[si]),
                    (unsigned long long)__float2ll_rn(pw * (float)fix));
          atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[(size_t)g.n + si]),
                    (unsigned long long)__float2ll_rn(pd * (float)fix));
          atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[2 * (size_t)g.n + si]),
                    (unsigned long long)pn);
        }
      }
      __syncthreads();
      for (int e = tid; e < len; e += kSymThreads) {
        if (sh.accn[e] == 0 && sh.accw[e] == 0) continue;
        const int sj = sh.j[e];
        atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[sj]), sh.accw[e]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[(size_t)g.n + sj]), sh.accd[e]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[2 * (size_t)g.n + sj]),
                  (unsigned long long)sh.accn[e]);
      }
      __syncthreads();
    }
  }
}

// Fixed point -> outputs in the caller's order for every particle; clears the
// sums for the next pass.
__global__ void k_sym_finalize(GridDev g, float* __restrict__ rho, float* __restrict__ drho_dh,
                               int32_t* __restrict__ n_ngb) {
  pdl_enter();
  if (*g.flags) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long inter = 0;
  if (s < g.n) {
    const size_t N = (size_t)g.n;
    const int i = g.orig[s];
    const int bx = box_of_particle(g, i);
    const float h = g.hs[s];
    const float H = g.gamma * h;
    const float c = (float)(16.0 / 3.14159265358979323846 * kFixInv) * g.m_max[bx] / (H * H * H);
    const long long an = g.acc[2 * N + s];
    rho[i] = c * __ll2float_rn(g.acc[s]);
    if (drho_dh) drho_dh[i] = -(c / h) * __ll2float_rn(g.acc[N + s]);
    if (n_ngb) n_ngb[i] = (int32_t)an - 1;
    inter = (unsigned long long)(an - 1);
    g.acc[s] = 0;
    g.acc[N + s] = 0;
    g.acc[2 * N + s] = 0;
  }
  for (int o = 16; o > 0; o >>= 1) inter += __shfl_xor_sync(0xffffffffu, inter, o);
  if ((threadIdx.x & 31) == 0 && inter) atomicAdd(&g.counters[0], inter);
}

}  // namespace

cudaError_t launch_density_symmetric(const GridDev& g, float* rho, float* drho_dh,
                                     int32_t* n_ngb, int num_sms, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  cudaError_t e = launch_plan_slots(g, 1, st);
  if (e != cudaSuccess) return e;
  PV_LAUNCH(k_density_sym, num_sms * 4, kSymThreads, 0, st, g);
  PV_LAUNCH(k_sym_finalize, (g.n + 255) / 256, 256, 0, st, g, rho, drho_dh, n_ngb);
  return cudaSuccess;
}

}  // namespace pv
