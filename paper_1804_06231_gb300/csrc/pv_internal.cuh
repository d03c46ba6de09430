// pv_internal.cuh -- device-side data layout and helpers shared by the CUDA
// translation units of the pseudo-Verlet density library (sm_103a).
//
// Layout in HBM (all particle arrays are in "cell order": the particles of a
// cell are contiguous, cells in global cell-id order, boxes one after the
// other):
//   xm    float4 [N]       {x', y', z', m/m_max(box)}: FP32 offset of the particle
//                          from its cell centre (Section 3.2: shift, then
//                          convert to single precision) and normalised mass
//   hs    float  [N]       smoothing length h (support H = gamma h)
//   orig  int32  [N]       index of the particle in the caller's arrays
//   pos64 double [N][3]    wrapped FP64 position (only read to re-decide
//                          pairs whose FP32 distance is within rounding of H)
//   perm  uint16 [13][N]   per cell and axis k: cell-local index of the t-th
//                          particle in ascending projection on u_k
//   dist  float  [13][N]   the projection itself (the "dist"/"index" arrays
//                          of Section 2)
//   cell_start int32 [C+1], cell_Hmax float [C]
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <stdint.h>

#include "pv.h"

namespace pv {

constexpr int kNDir = 13;   // distinct axes joining neighbouring cell centres
constexpr int kNSlot = 27;  // neighbour offsets (ox,oy,oz) in {-1,0,1}^3
constexpr int kSelfSlot = 13;
constexpr int kTinyCell = 32;  // cells of at most this many particles: one warp, all 27 slots
constexpr uint32_t kAllSlots = (1u << 27) - 1u;
constexpr double kFixScale = 68719476736.0;         // fixed-point scale 2^36
constexpr double kFixInv = 1.0 / 68719476736.0;
constexpr float kPiF = 3.14159265358979f;

struct BoxDev {
  double L, inv_L, edge, inv_edge;
  float edge_f;    // FP32 cell edge
  float pad;       // window pad covering FP32 rounding of projections
  float guard;     // guard half-width factor for r^2 (see guard_band())
  float h_limit;   // largest FP32 h whose support gamma h (FP64) is within the edge
  int32_t nc;
  int32_t cell_base;  // first global cell id of the box
  int64_t first, n;
};

// The largest FP32 h with gamma * (double)h <= edge: for FP32 h the test
// h > h_limit is then the same as the FP64 test gamma h > edge (the product
// is monotone in h), with no FP64 arithmetic per particle.
inline float support_h_limit(double gamma, double edge) {
  float h = (float)(edge / gamma);
  while (h > 0.0f && gamma * (double)h > edge) h = std::nextafter(h, 0.0f);
  while (gamma * (double)std::nextafter(h, INFINITY) <= edge) h = std::nextafter(h, INFINITY);
  return h;
}

// Everything a kernel needs, passed by value.
struct GridDev {
  int32_t n_boxes, n, ncell;
  float gamma;
  double gamma_d;
  const BoxDev* boxes;
  const int64_t* box_first;  // [n_boxes] (for particle -> box lookup)
  // per cell
  int32_t* cell_count;  // [C]
  int32_t* cell_start;  // [C+1]
  int32_t* cell_box;    // [C]
  float* cell_Hmax;     // [C]
  // cell lists of the sort paths (two lists per array, one from each end)
  int32_t* small_cells;  // [C] front: cells sorted by one CTA each; back: the largest
  int32_t* n_small;      // [1] entries at the front
  int32_t* n_huge;       // [1] entries at the back
  int32_t* big_cells;    // [C] cells sorted one axis per CTA: mid-sized ones from the
                         // front, large ones from the back
  int32_t* n_big;        // [1] entries at the front
  int32_t* n_large;      // [1] entries at the back
  int32_t* tile_sum;     // [scan_tiles(C)] occupancy totals of the scan's tiles
  // per particle, caller order
  int32_t* pcell;
  int32_t* prank;
  // per particle, cell order
  float4* xm;
  float4* xm_ref;  // [N] xm at the last sort (reference of pv_update_positions)
  float* hs;
  int32_t* orig;
  double* pos64;
  uint16_t* perm;  // [13][N]
  float* dist;     // [13][N]
  // density accumulators (cell order), fixed point
  long long* acc;    // [3][N]: rho, drho/dh (2^36 scale), n
  // adjoint accumulators of the task path (cell order), 64-bit fixed point
  // [5][N]: sum m th, sum m uh (units 2^-36), gx, gy, gz (units set per cell
  // by the bound of its neighbourhood's terms)
  long long* gacc;
  float* bwd_cmax;   // [C] largest (|G'| + |K|) H of the cell's particles (adjoint term bound)
  float* bwd_hmin;   // [C] smallest support H of the cell's particles (adjoint)
  float4* bx;        // [N] backward, cell order: {x', y', z', H^2 + guard}
  float4* ba;        // [N] backward, cell order: {m/m_max, g/H^5, k/(h H^5), H}
  // plan: per (cell, slot) {reachable count of a, window [J0, J1) of b, 0}
  int4* plan;        // [C][27]
  int32_t* ccells;   // [C] cells for the cell-centric kernel
  int32_t* n_ccells;
  int32_t* ccell_next;
  int32_t* tcells;   // [C] cells expanded into tasks
  int32_t* n_tcells;
  int32_t* ycells;   // [C] cells of at most kTinyCell particles (one warp each)
  int32_t* n_ycells;
  int32_t* ycell_next;  // next entry of ycells to take
  // tasks
  int4* tasks;
  int32_t* ntask;
  int32_t* task_next;
  int32_t max_tasks;
  int32_t task_blk;    // particles of a per task of the pass (64, 128 or 256)
  uint32_t slot_mask;  // neighbour slots the sweeps visit (bit o of slot o; all 27 normally)
  int32_t moved;       // positions updated since the sort: windows use the stored projections
  // scalars
  uint32_t* flags;
  float* m_max;     // [n_boxes] largest mass of each box (mass unit of the accumulators)
  float* box_disp;  // [n_boxes] largest displacement since the last sort (0 right after it)
  int32_t* max_count;
  unsigned long long* counters;  // [0] interactions, [1] guard pairs, [2] candidates,
                                 // [3] adjoint candidates, [4] adjoint pairs,
                                 // [8 + 2c], [9 + 2c]: candidates, interactions of
                                 // orientation class c (self, face, edge, corner)
};

// ---- direction slots ------------------------------------------------------
// Slot o = (ox+1)*9 + (oy+1)*3 + (oz+1) for the neighbour offset (ox,oy,oz).
// The slot number orders offsets lexicographically, so the 13 axes v_k (the
// lexicographically positive offsets, Section 2) are the slots 14..26 with
// k = o - 14, and slot o < 13 is -v_k with k = 12 - o.  The self slot is 13.
struct Slot {
  int ox, oy, oz;  // offset of the neighbour cell
  int k, s;        // axis index and sign: (ox,oy,oz) = s v_k
  int v2;          // |v|^2: 1 face, 2 edge, 3 corner (0 for the self slot)
};

__host__ __device__ __forceinline__ Slot slot_info(int o) {
  Slot r;
  r.ox = o / 9 - 1;
  r.oy = (o / 3) % 3 - 1;
  r.oz = o % 3 - 1;
  r.v2 = r.ox * r.ox + r.oy * r.oy + r.oz * r.oz;
  if (o > kSelfSlot) { r.k = o - 14; r.s = 1; }
  else if (o < kSelfSlot) { r.k = 12 - o; r.s = -1; }
  else { r.k = 0; r.s = 1; }  // the self sweep uses axis (0,0,1)
  return r;
}

// |v|^-1 for |v|^2 = 1, 2, 3 (FP32-rounded 1, 1/sqrt2, 1/sqrt3)
__host__ __device__ __forceinline__ float inv_norm(int v2) {
  return v2 == 1 ? 1.0f : (v2 == 2 ? 0.70710678f : 0.57735027f);
}
__host__ __device__ __forceinline__ float vnorm(int v2) {
  return v2 == 1 ? 1.0f : (v2 == 2 ? 1.41421356f : 1.73205081f);
}

// unit axis u_k
__host__ __device__ __forceinline__ void axis_u(int k, float& ux, float& uy, float& uz) {
  Slot sl = slot_info(14 + k);
  float in = inv_norm(sl.v2);
  ux = sl.ox * in; uy = sl.oy * in; uz = sl.oz * in;
}

// projection of an FP32 offset on u_k (the sort key and the stored dist)
__device__ __forceinline__ float project(float4 x, float ux, float uy, float uz) {
  return fmaf(x.x, ux, fmaf(x.y, uy, x.z * uz));
}

// neighbour cell of global cell a at slot o (periodic wrap inside the box)
// Box of the particle with caller index p: the last box whose first index is
// <= p (boxes are contiguous and ordered).
__device__ __forceinline__ int box_of_particle(const GridDev& g, int p) {
  int lo = 0, hi = g.n_boxes - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.box_first[mid] <= (int64_t)p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int neighbour_cell(const GridDev& g, int a, int o) {
  const BoxDev& B = g.boxes[g.cell_box[a]];
  int nc = B.nc, loc = a - B.cell_base;
  int cx = loc / (nc * nc), cy = (loc / nc) % nc, cz = loc % nc;
  const Slot si = slot_info(o);
  cx += si.ox; cy += si.oy; cz += si.oz;
  cx = cx < 0 ? cx + nc : (cx >= nc ? cx - nc : cx);
  cy = cy < 0 ? cy + nc : (cy >= nc ? cy - nc : cy);
  cz = cz < 0 ? cz + nc : (cz >= nc ? cz - nc : cz);
  return B.cell_base + (cx * nc + cy) * nc + cz;
}

// ---- float <-> orderable int for atomicMax on non-negative floats ---------
// Raises *p to v (both non-negative floats, ordered as their bit patterns).
// The current value is read first and the atomic issued only when it can
// raise it: the value only grows, so a stale read costs at most one needless
// atomic, and threads holding the same value (a uniform mass, say) do not
// queue on one address.
__device__ __forceinline__ void atomic_max_nonneg(float* p, float v) {
  if (v > __ldcg(p)) atomicMax(reinterpret_cast<int*>(p), __float_as_int(v));
}

// Pre-filter of 8 consecutive staged particles (float4 {x, y, z, |x|^2} at
// shared-memory byte address `saddr`) for one particle i: shifts the sign of
// |x_j|^2 - 2 x_i.x_j - ci (nx, ny, nz = -2 x_i) into `m`, first candidate
// first (one load, one subtract, three fused multiply-adds and one funnel
// shift per candidate).
__device__ __forceinline__ void prefilter8(unsigned& m, unsigned saddr, float nx, float ny,
                                           float nz, float ci) {
  asm volatile(
      "{\n\t.reg .f32 a<4>, b<4>, d, e;\n\t"
      "ld.shared.v4.f32 {a0,a1,a2,a3}, [%1];\n\t"
      "ld.shared.v4.f32 {b0,b1,b2,b3}, [%1+16];\n\t"
      "sub.f32 d, a3, %5;\n\tfma.rn.f32 d, %4, a2, d;\n\tfma.rn.f32 d, %3, a1, d;\n\t"
      "fma.rn.f32 d, %2, a0, d;\n\t"
      "sub.f32 e, b3, %5;\n\tfma.rn.f32 e, %4, b2, e;\n\tfma.rn.f32 e, %3, b1, e;\n\t"
      "fma.rn.f32 e, %2, b0, e;\n\t"
      "shf.l.wrap.b32 %0, d, %0, 1;\n\tshf.l.wrap.b32 %0, e, %0, 1;\n\t"
      "ld.shared.v4.f32 {a0,a1,a2,a3}, [%1+32];\n\t"
      "ld.shared.v4.f32 {b0,b1,b2,b3}, [%1+48];\n\t"
      "sub.f32 d, a3, %5;\n\tfma.rn.f32 d, %4, a2, d;\n\tfma.rn.f32 d, %3, a1, d;\n\t"
      "fma.rn.f32 d, %2, a0, d;\n\t"
      "sub.f32 e, b3, %5;\n\tfma.rn.f32 e, %4, b2, e;\n\tfma.rn.f32 e, %3, b1, e;\n\t"
      "fma.rn.f32 e, %2, b0, e;\n\t"
      "shf.l.wrap.b32 %0, d, %0, 1;\n\tshf.l.wrap.b32 %0, e, %0, 1;\n\t"
      "ld.shared.v4.f32 {a0,a1,a2,a3}, [%1+64];\n\t"
      "ld.shared.v4.f32 {b0,b1,b2,b3}, [%1+80];\n\t"
      "sub.f32 d, a3, %5;\n\tfma.rn.f32 d, %4, a2, d;\n\tfma.rn.f32 d, %3, a1, d;\n\t"
      "fma.rn.f32 d, %2, a0, d;\n\t"
      "sub.f32 e, b3, %5;\n\tfma.rn.f32 e, %4, b2, e;\n\tfma.rn.f32 e, %3, b1, e;\n\t"
      "fma.rn.f32 e, %2, b0, e;\n\t"
      "shf.l.wrap.b32 %0, d, %0, 1;\n\tshf.l.wrap.b32 %0, e, %0, 1;\n\t"
      "ld.shared.v4.f32 {a0,a1,a2,a3}, [%1+96];\n\t"
      "ld.shared.v4.f32 {b0,b1,b2,b3}, [%1+112];\n\t"
      "sub.f32 d, a3, %5;\n\tfma.rn.f32 d, %4, a2, d;\n\tfma.rn.f32 d, %3, a1, d;\n\t"
      "fma.rn.f32 d, %2, a0, d;\n\t"
      "sub.f32 e, b3, %5;\n\tfma.rn.f32 e, %4, b2, e;\n\tfma.rn.f32 e, %3, b1, e;\n\t"
      "fma.rn.f32 e, %2, b0, e;\n\t"
      "shf.l.wrap.b32 %0, d, %0, 1;\n\tshf.l.wrap.b32 %0, e, %0, 1;\n\t}"
      : "+r"(m)
      : "r"(saddr), "f"(nx), "f"(ny), "f"(nz), "f"(ci));
}

// sqrt with the hardware approximation (about 1 ulp; 0 -> 0)
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// last t in [0, n) with a[t] <= v, for a ascending, a[0] <= v and n <= 32; the
// whole warp calls it with the same v (one ballot instead of a search)
__device__ __forceinline__ int warp_seg_of(const int* a, int n, int v, int lane) {
  const bool le = lane < n && a[lane] <= v;
  return __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// Warp-cooperative search: the first e in [0, len) with pred(e), for a
// predicate that is false on a prefix and true after it (len if none).  The
// whole warp calls it with the same arguments; each round probes 32 evenly
// spaced points, so two rounds cover len <= 1024 and three len <= 32768.
template <typename Pred>
__device__ __forceinline__ int warp_first_true(int len, int lane, Pred pred) {
  int lo = 0, hi = len;  // the answer lies in [lo, hi]
  while (hi > lo) {
    const int step = (hi - lo + 31) >> 5;
    const int p = lo + lane * step;
    const bool f = p < hi && !pred(p);
    const int nf = __popc(__ballot_sync(0xffffffffu, f));  // probes before the answer
    if (step == 1) return lo + nf;
    if (nf == 0) return lo;
    lo += (nf - 1) * step + 1;
    hi = min(lo - 1 + step, hi);
  }
  return lo;
}

// first index t in [0, n) with a[t] >= x (a ascending), n if none
__device__ __forceinline__ int lower_bound_f(const float* a, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// first index t in [0, n) with a[t] > x, n if none
__device__ __forceinline__ int upper_bound_f(const float* a, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Projection of particle p of cell c on axis k, in the frame of cell a,
// along u = s u_k, in ascending order t = 0 .. cnt-1:
//   stored order for s = +1, reversed for s = -1; d = s dist + offset.
__host__ __device__ __forceinline__ int order_pos(int s, int t, int cnt) { return s > 0 ? t : cnt - 1 - t; }

// ---- cubic spline, half-scaled ---------------------------------------------
// With w(q) the shape function of the workload (8/pi factor included),
// wh(q) = w(q) / (16/pi) and th(q) = (3 w(q) + q w'(q)) / (16/pi).  Writing
// s = 1 - q and t = max(1/2 - q, 0), the two cubic pieces combine into
//   wh = s^3 - 4 t^3
//   th = s^2 (3 - 6q) - t^2 (6 - 24q)
// (for q < 1/2 this expands to 1/2 - 3q^2 + 3q^3 and 3/2 - 15q^2 + 18q^3), so
// rho_i = (16/pi) H_i^-3 sum_j m_j wh(q_ij) and
// drho/dh_i = -(16/pi) / (h_i H_i^3) sum_j m_j th(q_ij).
__device__ __forceinline__ void spline_half(float q, float& wh, float& th) {
  const float s = 1.0f - q;
  const float t = fmaxf(0.5f - q, 0.0f);
  const float s2 = s * s, t2 = t * t;
  wh = fmaf(-4.0f * t, t2, s2 * s);
  th = fmaf(s2, fmaf(-6.0f, q, 3.0f), -t2 * fmaf(-24.0f, q, 6.0f));
}

// Guard band of the FP32 distance test.  The FP32 r^2 of a pair differs from
// the exact one by less than
//   2 r |d(dx)| sqrt(3) + 3 ulp(r^2)  with |d(dx)| <= 2^-22 edge
// (offsets rounded to 2^-24 edge, the shifted i position to 2^-23 edge, the
// difference to 2^-24 H), i.e. < 1.2e-6 H edge + 3.6e-7 H^2 for r ~ H.
// Pairs whose FP32 r^2 lies within twice that of H^2 are re-decided in FP64.
__device__ __forceinline__ float guard_band(float H, float edge) {
  return 2.4e-6f * H * edge + 8.0e-7f * H * H;
}

// FP64 re-decision of r_ij < H_i for a pair in the guard band, from the
// wrapped FP64 positions with the minimum-image convention.
static __device__ __forceinline__ bool guard_inside(const double* __restrict__ pos64, int si,
                                                 int sj, double L, double inv_L, double Hd) {
  double r2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double d = pos64[3 * (size_t)si + c] - pos64[3 * (size_t)sj + c];
    d -= L * rint(d * inv_L);
    r2 = fma(d, d, r2);
  }
  return r2 < Hd * Hd;
}

// Asynchronous global -> shared copies (cp.async): the data goes to shared
// memory without passing through registers, so a thread can have many in
// flight.  16-byte copies are cached in L2 only (.cg); 4-byte ones in L1 too.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Waits for all of this thread's cp.async copies.
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Stages the windows of a cell, one flat range [0, total) with window q at
// [off[q], off[q+1]): thread t takes elements t, t + nthr, ... (so every warp
// stays full across window boundaries), follows its window index forward
// instead of searching for it, and keeps U elements in flight: index(f, q)
// for U elements (the sorted-order lookups), then fetch(sj) for the U (the
// particle data), then put(f, q, value).
template <int U, typename Index, typename Fetch, typename Put>
__device__ __forceinline__ void stage_flat(const int* off, int total, int tid, int nthr,
                                           Index index, Fetch fetch, Put put) {
  int q = 0;
  for (int f0 = tid; f0 < total; f0 += U * nthr) {
    int sj[U], sq[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int f = f0 + u * nthr;
      sj[u] = -1;
      sq[u] = 0;
      if (f < total) {
        while (off[q + 1] <= f) q++;
        sj[u] = index(f, q);
        sq[u] = q;
      }
    }
    decltype(fetch(0)) v[U];
#pragma unroll
    for (int u = 0; u < U; u++)
      if (sj[u] >= 0) v[u] = fetch(sj[u]);
#pragma unroll
    for (int u = 0; u < U; u++)
      if (sj[u] >= 0) put(f0 + u * nthr, sq[u], v[u]);
  }
}

// Projection of the t-th particle of cell c (start cs, count cnt) in the
// ascending-along-u order of slot (k, s), plus the cell shift `off`.
__device__ __forceinline__ float proj_asc(const GridDev& g, int k, int s, int cs, int cnt, int t,
                                          float off) {
  return s * g.dist[(size_t)k * g.n + cs + order_pos(s, t, cnt)] + off;
}

// Widening of every sorted window in box `bx`: projection rounding plus twice
// the largest displacement since the last sort.
__device__ __forceinline__ float window_pad(const GridDev& g, const BoxDev& B, int bx) {
  return B.pad + 2.0f * g.box_disp[bx];
}

// ---- warp-per-cell kernels (cells of at most kTinyCell particles) ----------
// Per-warp slot table of the warp-per-cell kernels: the staged range of slot q
// is [off[q], off[q + 1]); win[q] = {J0, cell start of b, count of b, o}.
struct TinySlots {
  int off[kNSlot + 1];
  int4 win[kNSlot];
};

// Fills the slot table of cell a from the plan (lane q < 27: slot q); returns
// the total window length (warp-uniform).
__device__ __forceinline__ int tiny_slots(const GridDev& g, int a, int lane, TinySlots& ts) {
  int len = 0;
  int4 w = make_int4(0, 0, 0, 0);
  if (lane < kNSlot) {
    const int4 p = g.plan[(size_t)a * kNSlot + lane];
    if (p.x > 0) {  // some particle of a reaches b
      const int b = neighbour_cell(g, a, lane);
      w = make_int4(p.y, g.cell_start[b], g.cell_count[b], lane);
      len = p.z - p.y;
    }
  }
  int incl = len;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, s);
    if (lane >= s) incl += v;
  }
  if (lane < kNSlot) {
    ts.off[lane] = incl - len;
    ts.win[lane] = w;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane == 0) ts.off[kNSlot] = total;
  __syncwarp();
  return total;
}

// Cell-order index of staged candidate f (slot q of the table) and the shift
// o edge of its cell relative to a.
__device__ __forceinline__ int tiny_candidate(const GridDev& g, const TinySlots& ts, int q, int f,
                                              float edge, float& sx, float& sy, float& sz) {
  const int4 w = ts.win[q];
  const Slot sl = slot_info(w.w);
  const int pos = order_pos(sl.s, w.x + f - ts.off[q], w.z);
  sx = sl.ox * edge;
  sy = sl.oy * edge;
  sz = sl.oz * edge;
  return w.y + (int)g.perm[(size_t)sl.k * g.n + w.y + pos];
}

// ---- host-side launchers (defined in the .cu files) ------------------------
// The sort of pv_sort_cells in launch order: clear, bin, scan, scatter, sort.
// launch_clear zeroes the occupancies, flags, max_count, n_big, m_max and
// box_disp; launch_sort gathers every cell into cell order (xm, xm_ref, hs,
// pos64, cell_Hmax) and writes perm and dist.
cudaError_t launch_clear(const GridDev& g, cudaStream_t st);
cudaError_t launch_bin(const GridDev& g, const double* pos, const float* h, const float* m,
                       float m_uniform, cudaStream_t st);
// tiles of the occupancy scan
constexpr int kScanTile = 1024;  // cells per CTA
constexpr int scan_tiles(int64_t ncell) { return (int)((ncell + kScanTile - 1) / kScanTile); }
cudaError_t launch_scan(const GridDev& g, cudaStream_t st);
cudaError_t launch_scatter(const GridDev& g, cudaStream_t st);
cudaError_t launch_sort(const GridDev& g, const double* pos, const float* h, const float* m,
                        float m_uniform, cudaStream_t st);
cudaError_t launch_update(const GridDev& g, const double* pos, const float* h, cudaStream_t st);
// Per-(cell, slot) plan, then per-cell routing: cells whose staged windows fit
// `smem_budget` bytes (elem_j bytes per staged particle, elem_a per particle
// of the cell, elem_i per entry of the slots' lists of reaching particles) go
// to the cell-centric kernel, the others are split into tasks.
cudaError_t launch_plan(const GridDev& g, int wide, int smem_budget, int elem_j, int elem_a,
                        int elem_i, cudaStream_t st);
// Only the per-(cell, slot) plan (no routing), as launch_plan's first kernel.
cudaError_t launch_plan_slots(const GridDev& g, int wide, cudaStream_t st);
int64_t max_tasks_for(int64_t n, int64_t ncell);
// The density by the symmetric pair update (pv_symmetric.cu); the grid's
// fixed-point sums `acc` and the counter ccell_next must be zero.
cudaError_t launch_density_symmetric(const GridDev& g, float* rho, float* drho_dh,
                                     int32_t* n_ngb, int num_sms, cudaStream_t st);
// ctas_per_sm: resident CTAs of the cell-centric sweep kernel per SM (1..4
// forward, 1..3 adjoint); it sets the kernel's shared memory and so which
// cells the plan routes to it.  t0/t1 (optional): events recorded on `st`
// just before and after that kernel.
cudaError_t launch_density(const GridDev& g, float* rho, float* drho_dh, int32_t* n_ngb,
                           int num_sms, int ctas_per_sm, cudaStream_t st,
                           cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr);
cudaError_t launch_backward(const GridDev& g, const float* g_rho, const float* g_drho_dh,
                            float* g_pos, float* g_h, int num_sms, int ctas_per_sm,
                            cudaStream_t st, cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr);
constexpr int kDensityCtasDefault = 3, kBackwardCtasDefault = 3;
// particles per task of the task path: the default and the smallest (which
// sizes the task array)
constexpr int kTaskBlkDefault = 128, kTaskBlkMin = 64;

// Warp-wide min / max of a float by one integer reduction (redux.sync): the
// map below is monotone from floats (no NaN) to signed integers and its own
// inverse.
__device__ __forceinline__ int float_order_key(float f) {
  const int i = __float_as_int(f);
  return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float warp_min_f(float v) {
  return __int_as_float(float_order_key(__int_as_float(
      __reduce_min_sync(0xffffffffu, float_order_key(v)))));
}
__device__ __forceinline__ float warp_max_f(float v) {
  return __int_as_float(float_order_key(__int_as_float(
      __reduce_max_sync(0xffffffffu, float_order_key(v)))));
}

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_enter(): it waits until the grids it depends on have completed and their
// writes are visible (a no-op for a kernel launched without the attribute),
// then allows the next kernel of the stream to be scheduled.  A kernel launched
// by PV_LAUNCH may therefore be resident while its predecessor still runs;
// its threads do nothing before the wait, so the stream order of the results
// is unchanged and only the launch latency overlaps.  The next grid is
// scheduled only once every CTA of this one has started, so waiting CTAs can
// never hold back a CTA they depend on.  (A kernel launched without the
// attribute waits for its predecessor as usual; pdl_enter is then a no-op.)
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_k(bool pdl, void (*kernel)(P...), unsigned grid, unsigned block,
                            size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}
// launch_k(true, ...) / launch_k(false, ...) in a function returning
// cudaError_t: returns its error.  PV_LAUNCH_PLAIN is for the kernels measured
// slower as dependents (the persistent big-cell sorts and the task kernels, on
// clustered boxes).
#define PV_LAUNCH(...)                                        \
  do {                                                        \
    const cudaError_t pv_le_ = pv::launch_k(true, __VA_ARGS__); \
    if (pv_le_ != cudaSuccess) return pv_le_;                 \
  } while (0)
#define PV_LAUNCH_PLAIN(...)                                   \
  do {                                                         \
    const cudaError_t pv_le_ = pv::launch_k(false, __VA_ARGS__); \
    if (pv_le_ != cudaSuccess) return pv_le_;                  \
  } while (0)

// Raises `func`'s dynamic shared-memory limit to `bytes`.  The limit is an
// attribute of the kernel in the current CUDA context, so it is set again on
// every launch: a context created after cudaDeviceReset gets it too.  While
// `st` is being captured into a CUDA graph the call only checks that an
// earlier launch in this context set the limit, and returns
// cudaErrorStreamCaptureUnsupported if none did (make one eager call first).
inline cudaError_t set_max_dynamic_smem(const void* func, int bytes, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusNone)
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
  return fa.maxDynamicSharedSizeBytes >= bytes ? cudaSuccess : cudaErrorStreamCaptureUnsupported;
}
// Records `e` and `what` as the calling thread's last CUDA error (the text
// pv_last_cuda_error returns) and maps `e` to a status code.
pv_status record_cuda_error(cudaError_t e, const char* what);
cudaError_t launch_count_candidates(const GridDev& g, cudaStream_t st);
cudaError_t launch_fp32_probe(int packed, int iters, float* sink, int64_t threads,
                              double* flops, cudaStream_t st);
cudaError_t launch_raw_density(const float4* xi, int ni, const float4* xj, int nj, float H,
                               int reps, float2* out, cudaStream_t st);

}  // namespace pv
