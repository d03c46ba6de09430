// pv_density.cu -- the density gather over the sorted cell pairs.
//
// For every cell a and each of its 27 neighbour slots (the cell itself and
// the 26 cells b = a + o), the particles of a that can reach b are visited
// in order of decreasing projection on the axis u = o/|o| (nearest to the
// common face first, Section 3.1), and each gathers from the particles of b
// in order of increasing projection, stopping once the projected distance
// reaches its own support (Section 2 and Section 3.3).  Particles of a that
// lie further than the cell's largest support from b are skipped ("first_a",
// Section 3.3), and only the part of b that the nearest particle of a can
// reach is loaded ("max_index_a[count_a-1]", Section 3.3).  The self slot
// uses a two-sided window on the axis (0,0,1).
//
// GPU mapping (gather only):
//   * plan: per (cell, slot) the reachable count of a and the window of b;
//     per cell, whether its 27 windows fit the shared-memory budget;
//   * k_density_cells (the common case): one CTA owns a cell.  It stages the
//     27 trimmed windows of its neighbours, in sorted order, into shared
//     memory (the particle cache of Section 3.2), then its warps pull work
//     items (slot, run of 32 sorted particles of a) from a shared counter.  A
//     warp sweeps the union of its 32 windows; each lane first tests 32
//     candidates and records the in-range ones in a bit mask, then evaluates
//     the kernel only for those (so the spline is not executed under a mask
//     for every candidate).  Partial sums go to per-particle fixed-point
//     accumulators in shared memory and the CTA writes the outputs;
//   * k_density_tasks: cells whose windows do not fit (very dense cells) are
//     split into tasks (cell, slot, block of 128 particles of a) that stage
//     the window of b in tiles and add to fixed-point accumulators in global
//     memory, converted by k_finalize_t.
// Fixed-point (2^36 units of the largest mass) integer accumulation makes the
// result independent of which warp or CTA processed which item.
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {

namespace {

constexpr int kTileJ = 512;      // particles of b per tile (task path)
constexpr int kCellThreads = 256;
// dynamic shared memory of k_density_cells for 1..4 resident CTAs per SM (the
// SM's 228 KB less 1 KB reserved and the static part per CTA); 3 by default
constexpr int kCellSmemFor[5] = {0, 200 * 1024, 110 * 1024, 72 * 1024, 54 * 1024};
constexpr int kPad = 32;         // slack after staged arrays for the 32-wide sweep

// slots ordered by expected cost: self, faces, edges, corners
__constant__ int8_t c_slot_order[kNSlot] = {13, 4,  10, 12, 14, 16, 22, 1,  3,  5,  7,  9, 11, 15,
                                            17, 19, 21, 23, 25, 0,  2,  6,  8,  18, 20, 24, 26};

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


// #{t : proj_asc(t) < lim} (ascending)
__device__ __forceinline__ int count_below(const GridDev& g, int k, int s, int cs, int cnt,
                                           float off, float lim) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (proj_asc(g, k, s, cs, cnt, mid, off) < lim) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ---- plan ------------------------------------------------------------------------
// One thread per (cell a, slot o): the number of particles of a that can reach
// b (first_a trimming with the cell's largest support) and the window [J0, J1)
// of b that the nearest of them can touch.  `wide` widens every reach to the
// larger of the two cells' largest supports (adjoint pass).  The two binary
// searches are independent and run in lockstep, so that their global loads
// are in flight together; a grid with latched input errors gets empty plans.
__global__ void k_plan_slots(GridDev g, int wide) {
  pdl_enter();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  // the adjoint's per-cell term bounds and smallest supports are reduced
  // afresh by k_bwd_prep
  if (wide && g.bwd_cmax && idx < g.ncell) {
    g.bwd_cmax[idx] = 0.0f;
    g.bwd_hmin[idx] = 3.0e38f;
  }
  if (idx >= g.ncell * kNSlot) return;
  const uint32_t flagged = *g.flags;
  const int a = idx / kNSlot, o = idx % kNSlot;
  const int na = g.cell_count[a];
  int4 pl = make_int4(0, 0, 0, 0);
  if (na > 0 && ((g.slot_mask >> o) & 1u)) {
    const int b = neighbour_cell(g, a, o);
    const int nb = g.cell_count[b];
    if (nb > 0) {
      const BoxDev& B = g.boxes[g.cell_box[a]];
      const Slot sl = slot_info(o);
      const int ca = g.cell_start[a], cb = g.cell_start[b];
      float reach = g.cell_Hmax[a];
      if (wide) reach = fmaxf(reach, g.cell_Hmax[b]);
      reach += window_pad(g, B, g.cell_box[a]);
      if (o == kSelfSlot) {
        pl = make_int4(na, 0, nb, 0);
      } else {
        const float off = vnorm(sl.v2) * B.edge_f;
        const float db_min = proj_asc(g, sl.k, sl.s, cb, nb, 0, off);
        const float lim = proj_asc(g, sl.k, sl.s, ca, na, na - 1, 0.0f) + reach;
        // lo1: particles of a, in descending order along u (position p is
        // ascending index na-1-p), whose reach passes b's nearest particle;
        // lo2: particles of b below the reach of a's farthest one
        int lo1 = 0, hi1 = na, lo2 = 0, hi2 = nb;
        while (lo1 < hi1 || lo2 < hi2) {
          const int m1 = (lo1 + hi1) >> 1, m2 = (lo2 + hi2) >> 1;
          const bool s1 = lo1 < hi1, s2 = lo2 < hi2;
          const float d1 = s1 ? proj_asc(g, sl.k, sl.s, ca, na, na - 1 - m1, 0.0f) : 0.0f;
          const float d2 = s2 ? proj_asc(g, sl.k, sl.s, cb, nb, m2, off) : 0.0f;
          if (s1) {
            if (d1 + reach > db_min) lo1 = m1 + 1; else hi1 = m1;
          }
          if (s2) {
            if (d2 < lim) lo2 = m2 + 1; else hi2 = m2;
          }
        }
        if (lo1 > 0) pl = make_int4(lo1, 0, lo2, 0);
      }
    }
  }
  g.plan[idx] = flagged ? make_int4(0, 0, 0, 0) : pl;
  if (idx == 0) {  // the routing lists and work counters of the pass start empty
    *g.n_ycells = 0;
    *g.ycell_next = 0;
    *g.ntask = 0;
    *g.task_next = 0;
    *g.n_ccells = 0;
    *g.ccell_next = 0;
    *g.n_tcells = 0;
    if (!wide) g.counters[0] = g.counters[1] = 0ull;  // interactions, FP64 re-decisions
  }
}

// One thread per cell: route a cell of at most kTinyCell particles to the
// warp-per-cell kernel, any other cell to the cell-centric kernel when its
// staged windows fit `smem_budget`, else to the task kernel, reserving one
// task of g.task_blk particles per block of each slot (the first task's index goes
// to plan.w; k_plan_tasks fills the tasks in).  The list appends and the task
// reservations are aggregated per warp (one atomic per warp and list instead
// of one per cell: a clustered box has tens of thousands of cells).
__global__ void k_plan_cells(GridDev g, int smem_budget, int elem_j, int elem_a, int elem_i) {
  pdl_enter();
  if (*g.flags) return;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int na = 0;
  int4* pl = nullptr;
  bool fits = false, tiny = false;
  int nblk_tot = 0;  // task blocks of this cell (task-path cells only)
  if (a < g.ncell) {
    na = g.cell_count[a];
    tiny = na > 0 && na <= kTinyCell;
    if (na > 0 && !tiny) {
      pl = g.plan + (size_t)a * kNSlot;
      int total = 0, sum_i = 0;  // windows padded to groups of four
      for (int o = 0; o < kNSlot; o++) {
        total += (pl[o].z - pl[o].y + 3) & ~3;
        sum_i += pl[o].x;
      }
      fits = elem_j * (total + kPad + 4) + elem_a * na + elem_i * sum_i + 16 <= smem_budget;
      if (!fits)
        for (int o = 0; o < kNSlot; o++) nblk_tot += (pl[o].x + g.task_blk - 1) / g.task_blk;
    }
  }
  const bool task = na > 0 && !tiny && !fits;
  const unsigned below = (1u << lane) - 1u;
  const unsigned mc = __ballot_sync(0xffffffffu, fits), mt = __ballot_sync(0xffffffffu, task);
  const unsigned my = __ballot_sync(0xffffffffu, tiny);
  int incl = nblk_tot;  // inclusive scan of the task blocks over the warp
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, s);
    if (lane >= s) incl += v;
  }
  int bc = 0, bt = 0, bk = 0, by = 0;
  if (lane == 31) {
    if (my) by = atomicAdd(g.n_ycells, __popc(my));
    if (mc) bc = atomicAdd(g.n_ccells, __popc(mc));
    if (mt) bt = atomicAdd(g.n_tcells, __popc(mt));
    if (incl) bk = atomicAdd(g.ntask, incl);
  }
  bc = __shfl_sync(0xffffffffu, bc, 31);
  bt = __shfl_sync(0xffffffffu, bt, 31);
  bk = __shfl_sync(0xffffffffu, bk, 31);
  by = __shfl_sync(0xffffffffu, by, 31);
  if (tiny) g.ycells[by + __popc(my & below)] = a;
  if (fits) g.ccells[bc + __popc(mc & below)] = a;
  if (!task) return;
  g.tcells[bt + __popc(mt & below)] = a;
  int base = bk + incl - nblk_tot;
  if (base + nblk_tot > g.max_tasks) {  // cannot happen with the allocated bound
    atomicOr(g.flags, PV_FLAG_CELL_OVERFLOW);
    return;
  }
  for (int o = 0; o < kNSlot; o++) {
    const int nI = pl[o].x;
    if (nI == 0) continue;
    pl[o].w = base;
    base += (nI + g.task_blk - 1) / g.task_blk;
  }
}

// One warp per (task cell, slot), lanes over its blocks of g.task_blk particles:
// each task gets its particles [p0, p1) of a in the slot's order and the
// window [j0, j1) of b that they can reach.
__global__ void k_plan_tasks(GridDev g, int wide) {
  pdl_enter();
  if (*g.flags) return;
  const int nt = *g.n_tcells;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int pair = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pair < nt * kNSlot;
       pair += nw) {
    const int a = g.tcells[pair / kNSlot], o = pair % kNSlot;
    const int4 pl = g.plan[(size_t)a * kNSlot + o];
    const int nI = pl.x;
    if (nI == 0) continue;
    const int na = g.cell_count[a], ca = g.cell_start[a];
    const int b = neighbour_cell(g, a, o);
    const int nb = g.cell_count[b], cb = g.cell_start[b];
    const BoxDev& B = g.boxes[g.cell_box[a]];
    const Slot sl = slot_info(o);
    float reach = g.cell_Hmax[a];
    if (wide) reach = fmaxf(reach, g.cell_Hmax[b]);
    reach += window_pad(g, B, g.cell_box[a]);
    const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    const int nblk = (nI + g.task_blk - 1) / g.task_blk;
    for (int bk = lane; bk < nblk; bk += 32) {
      const int p0 = bk * g.task_blk, p1 = min(nI, p0 + g.task_blk);
      int j0, j1;
      if (o == kSelfSlot) {
        // upper bound of d[p0] - reach and lower bound of d[p1 - 1] + reach,
        // in lockstep so that the two searches' loads are in flight together
        const float* d = g.dist + cb;  // axis 0, ascending
        const float x0 = d[p0] - reach, x1 = d[p1 - 1] + reach;
        int lo0 = 0, hi0 = nb, lo1 = 0, hi1 = nb;
        while (lo0 < hi0 || lo1 < hi1) {
          const int m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
          const bool s0 = lo0 < hi0, s1 = lo1 < hi1;
          const float v0 = s0 ? d[m0] : 0.0f;
          const float v1 = s1 ? d[m1] : 0.0f;
          if (s0) {
            if (v0 <= x0) lo0 = m0 + 1; else hi0 = m0;
          }
          if (s1) {
            if (v1 < x1) lo1 = m1 + 1; else hi1 = m1;
          }
        }
        j0 = lo0;
        j1 = lo1;
      } else {
        const float dmax = proj_asc(g, sl.k, sl.s, ca, na, na - 1 - p0, 0.0f);
        j0 = 0;
        j1 = count_below(g, sl.k, sl.s, cb, nb, off, dmax + reach);
      }
      g.tasks[pl.w + bk] = make_int4(a, o, (int)((unsigned)p0 | ((unsigned)p1 << 16)),
                                     (int)((unsigned)j0 | ((unsigned)j1 << 16)));
    }
  }
}

// ---- the sweep ------------------------------------------------------------------
//
// Staged candidates are kept in groups of four: group g (80 bytes) holds the
// negated x, y, z offsets, W = |x|^2 and the normalised mass M of candidates
// 4g .. 4g+3 as five 16-byte vectors (negated, so that the differences
// x_i - x_j are packed additions with no constant operand).  The pre-filter reads one vector per field for four
// candidates and tests them two at a time with packed FP32 (fma.rn.f32x2: two
// FP32 operations per issued instruction); the evaluation reads a hit's four
// fields at fixed offsets from one address.  The sweep addresses shared memory
// through 32-bit shared-window addresses.
constexpr int kGroup = 20;  // floats per group of four staged candidates

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float4 lds4(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ float lds1(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
// byte offset of candidate c from the start of its group-aligned run
__device__ __forceinline__ unsigned cand_off(int c) {
  return (unsigned)((c >> 2) * (kGroup * 4) + ((c & 3) << 2));
}
// field offsets within a group (bytes): -x, -y, -z, W, M
constexpr unsigned kOffY = 16, kOffZ = 32, kOffW = 48, kOffM = 64;

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

struct LaneI {
  float2 x2, y2, z2;        // i in b's frame (x'_i - o edge), each twice (packed pairs)
  float2 px2, py2, pz2;     // 2 x_i (pre-filter, against the negated staged x_j), twice
  float2 nc2;               // -(H_i^2 + guard - |x_i|^2 + margin), twice (pre-filter)
  float2 hinv2;             // 1 / H_i^2, twice
  float dq;                 // hits with |1 - q| < dq are re-decided in FP64
  int si;                   // cell-order index of i
  float2 accW, accE, accN;  // per half of the hit pairs: sum m wh, sum m (s^2 - 2 t^2), count
  int ncorr;                // FP64 corrections of the count
};

// An inactive lane's pre-filter bound never passes (d >= 3e38).
__device__ __forceinline__ void lane_init(LaneI& L) {
  L.x2 = L.y2 = L.z2 = dup2(0.0f);
  L.px2 = L.py2 = L.pz2 = dup2(0.0f);
  L.nc2 = dup2(3.0e38f);
  L.hinv2 = dup2(0.0f);
  L.dq = 0.0f;
  L.si = 0;
  L.accW = L.accE = L.accN = dup2(0.0f);
  L.ncorr = 0;
}

// xh = {x', y', z', h} of particle i (cell order index si), slot sl of box B.
__device__ __forceinline__ void lane_set(LaneI& L, const BoxDev& B, float gamma, const Slot& sl,
                                         int si, float4 xh) {
  const float H = gamma * xh.w;
  const float x = xh.x - sl.ox * B.edge_f;
  const float y = xh.y - sl.oy * B.edge_f;
  const float z = xh.z - sl.oz * B.edge_f;
  L.si = si;
  L.x2 = dup2(x);
  L.y2 = dup2(y);
  L.z2 = dup2(z);
  L.px2 = dup2(2.0f * x);
  L.py2 = dup2(2.0f * y);
  L.pz2 = dup2(2.0f * z);
  const float Hsq = H * H, gb = guard_band(H, B.edge_f);
  const float hinv = __fdividef(1.0f, Hsq);
  L.hinv2 = dup2(hinv);
  // |1 - q| < gb / H^2 holds for every pair whose FP32 r^2 lies within the
  // guard band gb of H^2 (the band is at least 3.2e-6 H^2, twice the square
  // root's share plus the rounding of q), so a count decided by q < 1 outside
  // it agrees with the FP64 decision
  L.dq = gb * hinv;
  // pre-filter r^2 < H^2 + gb as |x_j|^2 - 2 x_i.x_j < H^2 + gb - |x_i|^2.  Its FP32
  // rounding is below 3 ulp of (|x_i| + |x_j|)^2 <= 12 edge^2, i.e. < 5e-6 edge^2;
  // the margin 1e-5 edge^2 keeps every in-range pair (the exact test follows).
  const float xi2 = fmaf(x, x, fmaf(y, y, z * z));
  L.nc2 = dup2(-((Hsq + gb - xi2) + 1.0e-5f * B.edge_f * B.edge_f));
}

// rho, drho/dh and count sums of a lane (drho/dh from th = 6 wh - 3 (s^2 - 2 t^2))
__device__ __forceinline__ void lane_sums(const LaneI& L, float& rho, float& D, int& n) {
  rho = L.accW.x + L.accW.y;
  D = fmaf(6.0f, rho, -3.0f * (L.accE.x + L.accE.y));
  n = (int)(L.accN.x + L.accN.y) + L.ncorr;
}

// Pre-filter of the 4 staged candidates of the group at shared address a:
// shifts the sign of |x_j|^2 - 2 x_i.x_j - bound of each into m, first
// candidate first.
__device__ __forceinline__ void prefilter4(unsigned& m, unsigned a, const LaneI& L) {
  const float4 x = lds4(a);
  const float4 y = lds4(a + kOffY);
  const float4 z = lds4(a + kOffZ);
  const float4 w = lds4(a + kOffW);
  float2 d0 = __fadd2_rn(make_float2(w.x, w.y), L.nc2);
  float2 d1 = __fadd2_rn(make_float2(w.z, w.w), L.nc2);
  d0 = __ffma2_rn(L.pz2, make_float2(z.x, z.y), d0);
  d1 = __ffma2_rn(L.pz2, make_float2(z.z, z.w), d1);
  d0 = __ffma2_rn(L.py2, make_float2(y.x, y.y), d0);
  d1 = __ffma2_rn(L.py2, make_float2(y.z, y.w), d1);
  d0 = __ffma2_rn(L.px2, make_float2(x.x, x.y), d0);
  d1 = __ffma2_rn(L.px2, make_float2(x.z, x.w), d1);
  m = __funnelshift_l(__float_as_uint(d0.x), m, 1);
  m = __funnelshift_l(__float_as_uint(d0.y), m, 1);
  m = __funnelshift_l(__float_as_uint(d1.x), m, 1);
  m = __funnelshift_l(__float_as_uint(d1.y), m, 1);
}

// Takes the highest set bit of m (candidate c of the chunk at bit 31 - c) and
// returns c (32 when m is empty).
__device__ __forceinline__ int take_hit(unsigned& m) {
  const int c = __clz(m);
  m &= ~__funnelshift_rc(0x80000000u, 0u, c);  // nothing to clear for c = 32
  return c;
}

// Kernel terms of two hits (candidates cA, cB of the chunk at shared address
// P; 32 for a lane with no hit left, which then reads the chunk's first
// candidate, a staged finite value, and adds nothing), added to lane i's
// packed sums.
// With s = 1 - q and t = max(1/2 - q, 0): wh = s^3 - 4 t^3 and
// 3 wh + q wh' = 6 wh - 3 (s^2 - 2 t^2).  q < 1 decides the pair (and the
// count); mn keeps the smallest |1 - q| for the FP64 re-decision of the count
// near the cut-off.
__device__ __forceinline__ void eval2(LaneI& L, unsigned P, int cA, int cB, float& mn) {
  const unsigned aA = P + cand_off(cA & 31), aB = P + cand_off(cB & 31);
  const float2 dx = __fadd2_rn(L.x2, make_float2(lds1(aA), lds1(aB)));
  const float2 dy = __fadd2_rn(L.y2, make_float2(lds1(aA + kOffY), lds1(aB + kOffY)));
  const float2 dz = __fadd2_rn(L.z2, make_float2(lds1(aA + kOffZ), lds1(aB + kOffZ)));
  const float2 mj = make_float2(lds1(aA + kOffM), lds1(aB + kOffM));
  float2 r2 = __fmul2_rn(dz, dz);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dx, dx, r2);
  const float2 u = __fmul2_rn(r2, L.hinv2);
  const float qa = cA < 32 ? sqrt_approx(u.x) : 2.0f;
  const float qb = cB < 32 ? sqrt_approx(u.y) : 2.0f;
  const float2 nq = make_float2(-qa, -qb);
  const float2 in = make_float2(qa < 1.0f ? 1.0f : 0.0f, qb < 1.0f ? 1.0f : 0.0f);
  const float2 s = __fadd2_rn(dup2(1.0f), nq);
  mn = fminf(mn, fminf(fabsf(s.x), fabsf(s.y)));
  float2 t = __fadd2_rn(dup2(0.5f), nq);
  t.x = fmaxf(t.x, 0.0f);
  t.y = fmaxf(t.y, 0.0f);
  const float2 me = __fmul2_rn(in, mj);
  const float2 s2 = __fmul2_rn(s, s);
  const float2 s3 = __fmul2_rn(s2, s);
  const float2 t2 = __fmul2_rn(t, t);
  const float2 wh = __ffma2_rn(__fmul2_rn(t, dup2(-4.0f)), t2, s3);
  const float2 e = __ffma2_rn(t2, dup2(-2.0f), s2);
  L.accW = __ffma2_rn(me, wh, L.accW);
  L.accE = __ffma2_rn(me, e, L.accE);
  L.accN = __fadd2_rn(L.accN, in);
}

// Sweeps the staged candidates [lo, hi) (groups at shared address S) for the
// warp's 32 particles; jidx(e) returns the cell-order index of staged
// candidate e (read only for the rare FP64 re-decisions near the cut-off).
// Reads the staged groups from lo rounded down to a group up to the group
// after hi + 2 (the staged arrays carry slack).
//
// Chunk by chunk (32 candidates): the pre-filter gives each lane a 32-bit hit
// mask in a register (candidate c at bit 31 - c); then the warp runs as many
// rounds as the busiest lane has hits in the chunk, two hits per round, each
// lane evaluating its own.
template <typename JIndex>
__device__ __forceinline__ void sweep_fwd(LaneI& L, unsigned S, int lo, int hi, const GridDev& g,
                                          const BoxDev& B, JIndex jidx, int& guards) {
  for (int base = lo & ~3; base < hi; base += 32) {
    const int cnt = min(32, hi - base);
    const unsigned P = S + (unsigned)(base >> 2) * (kGroup * 4);
    unsigned m = 0;
    if (cnt == 32) {
#pragma unroll
      for (int c = 0; c < 8; c++) prefilter4(m, P + c * (kGroup * 4), L);
    } else {
      const int n4 = (cnt + 3) >> 2;
#pragma unroll 1
      for (int c = 0; c < n4; c++) prefilter4(m, P + c * (kGroup * 4), L);
      m = (m << (32 - 4 * n4)) & (0xffffffffu << (32 - cnt));
    }
    if (base < lo) m &= 0xffffffffu >> (lo - base);
    const unsigned m0 = m;
    const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(m));
    float mn = 2.0f;
#pragma unroll 1
    for (int r = 0; r < rounds; r += 2) {
      const int cA = take_hit(m);
      const int cB = take_hit(m);
      eval2(L, P, cA, cB, mn);
    }
    // FP64 re-decision of the count for hits near the cut-off (rare): the lane
    // walks its hits of the chunk again
    if (__any_sync(0xffffffffu, mn < L.dq)) {
      if (mn < L.dq) {
        const float xi = L.x2.x, yi = L.y2.x, zi = L.z2.x, hinv = L.hinv2.x;
        unsigned mm = m0;
        while (mm != 0u) {
          const int c = take_hit(mm);
          const unsigned a = P + cand_off(c);
          const float dx = xi + lds1(a), dy = yi + lds1(a + kOffY), dz = zi + lds1(a + kOffZ);
          const float q = sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * hinv);
          if (fabsf(1.0f + (-q)) < L.dq) {
            guards++;
            const bool in64 = guard_inside(g.pos64, L.si, jidx(base + c), B.L, B.inv_L,
                                           g.gamma_d * (double)g.hs[L.si]);
            L.ncorr += (int)in64 - (q < 1.0f ? 1 : 0);
          }
        }
      }
    }
  }
}

// Stores particle x (cell-order record {x', y', z', m/m_max}) shifted by
// (sx, sy, sz) as staged candidate f.
__device__ __forceinline__ void put_staged(float* S, int f, float4 x, float sx, float sy,
                                           float sz) {
  float* p = S + (f >> 2) * kGroup + (f & 3);
  const float px = x.x + sx, py = x.y + sy, pz = x.z + sz;
  p[0] = -px;
  p[4] = -py;
  p[8] = -pz;
  p[12] = fmaf(px, px, fmaf(py, py, pz * pz));
  p[16] = x.w;
}

// floats of a staged buffer for n candidates (whole groups, with the slack the
// sweep reads past the end)
__host__ __device__ constexpr int staged_floats(int n) { return ((n + kPad + 3) >> 2) * kGroup; }

__device__ __forceinline__ float warp_min(float v) { return warp_min_f(v); }
__device__ __forceinline__ float warp_max(float v) { return warp_max_f(v); }

// rho, drho/dh, n of one particle from its fixed-point sums (FP32 scaling)
__device__ __forceinline__ void write_out(const GridDev& g, int s, long long ar, long long ad,
                                          int an, float* rho, float* drho_dh, int32_t* n_ngb,
                                          float mscale) {
  const int i = g.orig[s];
  const float h = g.hs[s];
  const float H = g.gamma * h;
  const float c = mscale / (H * H * H);  // (16/pi) m_max 2^-36 / H^3
  rho[i] = c * __ll2float_rn(ar);
  if (drho_dh) drho_dh[i] = -(c / h) * __ll2float_rn(ad);
  if (n_ngb) n_ngb[i] = an - 1;  // the self pair j = i
}

// ---- warp-per-cell kernel (cells of at most kTinyCell particles) -------------------
// A clustered box or a small box has tens of thousands of cells with a few
// particles each; as a CTA-sized cell each of them would cost a CTA's staging
// and barriers plus up to 27 warp items of a few active lanes.  Instead, once
// the cell-centric kernel's CTA-sized cells are all taken, its warps take the
// tiny cells one per warp: lane l holds the particle ca + l of cell a.  The 27 trimmed
// windows of the plan are staged one after the other, each neighbour's
// particles shifted into a's frame (x_j + o edge: the pair shift of Section
// 3.2 applied to j instead of i), and swept in one pass: the pre-filter of a
// lane runs over all staged candidates and the evaluation costs the largest
// total hit count of a lane instead of a sum of per-slot maxima.  Windows
// longer than kTinyBuf in total (a tiny cell next to a dense one) are staged
// in passes.  Each lane keeps its particle's sums in registers across the
// slots and writes its outputs itself.
constexpr int kTinyBuf = 128;  // staged candidates per warp and pass

// Bytes of a warp's tiny-cell buffers (staged groups, cell-order indices, slot
// table), carved from the cell kernel's dynamic shared memory once its
// CTA-sized cells are done.
constexpr int kTinyWarpBytes = staged_floats(kTinyBuf) * 4 + (kTinyBuf + kPad) * 4 +
                               (int)((sizeof(TinySlots) + 15) / 16 * 16);

template <typename Out>
__device__ __forceinline__ void tiny_phase_fwd(const GridDev& g, unsigned char* buf, int lane,
                                               Out out, unsigned long long& inter, int& guards) {
  float* S = reinterpret_cast<float*>(buf);
  int* Sj = reinterpret_cast<int*>(S + staged_floats(kTinyBuf));
  TinySlots& ts = *reinterpret_cast<TinySlots*>(Sj + kTinyBuf + kPad);
  const Slot self = slot_info(kSelfSlot);
  const int nt = *g.n_ycells;
  if (nt == 0) return;  // no tiny cells: leave the counter alone
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(g.ycell_next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= nt) break;
    const int a = g.ycells[w];
    const int na = g.cell_count[a], ca = g.cell_start[a];
    const BoxDev& B = g.boxes[g.cell_box[a]];
    const float edge = B.edge_f;
    const int total = tiny_slots(g, a, lane, ts);
    LaneI L;
    lane_init(L);
    if (lane < na) {
      const float4 xm = g.xm[ca + lane];
      lane_set(L, B, g.gamma, self, ca + lane, make_float4(xm.x, xm.y, xm.z, g.hs[ca + lane]));
    }
    int q = 0;  // slot of this lane's next staged candidate (non-decreasing)
    for (int f0 = 0; f0 < total; f0 += kTinyBuf) {
      const int len = min(kTinyBuf, total - f0);
      for (int e = lane; e < len; e += 32) {
        const int f = f0 + e;
        while (ts.off[q + 1] <= f) q++;
        float sx, sy, sz;
        const int sj = tiny_candidate(g, ts, q, f, edge, sx, sy, sz);
        put_staged(S, e, g.xm[sj], sx, sy, sz);
        Sj[e] = sj;
      }
      __syncwarp();
      auto jidx = [&](int j) { return Sj[j]; };
      sweep_fwd(L, smem_addr(S), 0, len, g, B, jidx, guards);
      __syncwarp();  // the buffers are rewritten next
    }
    if (lane < na) {
      float rho, D;
      int n;
      lane_sums(L, rho, D, n);
      out(a, ca + lane, rho, D, n);
      inter += (unsigned long long)(n - 1);
    }
  }
}

// ---- cell-centric kernel ------------------------------------------------------------

constexpr int kCellWarps = kCellThreads / 32;
static_assert(kCellWarps * kTinyWarpBytes <= kCellSmemFor[4],
              "the tiny-cell buffers fit the smallest dynamic shared memory");
// Staged bytes per candidate of a window (groups of four, with slack), bytes
// per particle of the cell ({x', y', z', h} and three fixed-point sums) and per
// entry of the slots' particle lists (16-bit index).
constexpr int kCellElemJ = 20;
constexpr int kCellElemA = 36;
constexpr int kCellElemI = 2;

struct CellShared {
  int I[kNSlot], J0[kNSlot];
  int off[kNSlot + 1];      // staged segment of the q-th slot of c_slot_order
  int runs[kNSlot + 1];     // prefix of run counts, same order
  int ioff[kNSlot + 1];     // the slot's list of particles of a, same order
  int nb_[kNSlot], cb_[kNSlot];
  float offv[kNSlot];
  int cell, item_next;
};

// projection of a staged particle in the frame of slot (k, s): the same FP32
// expression the sort used for `dist`, so the values are bit-identical
__device__ __forceinline__ float staged_proj(unsigned a, float ux, float uy, float uz, int s,
                                             float off) {
  return s * fmaf(-lds1(a), ux, fmaf(-lds1(a + kOffY), uy, -lds1(a + kOffZ) * uz)) + off;
}

__global__ void __launch_bounds__(kCellThreads, 4) k_density_cells(GridDev g, float* __restrict__ rho,
                                                                float* __restrict__ drho_dh,
                                                                int32_t* __restrict__ n_ngb) {
  pdl_enter();
  extern __shared__ float4 dsm[];
  __shared__ CellShared cs;
  if (*g.flags) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncells = *g.n_ccells;
  const float munit = (float)(16.0 / 3.14159265358979323846 * kFixInv);
  float4* var = dsm;
  int guards = 0;
  unsigned long long inter = 0;
  for (;;) {
    if (tid == 0) cs.cell = atomicAdd(g.ccell_next, 1);
    __syncthreads();
    const int ci = cs.cell;
    if (ci >= ncells) break;
    const int a = g.ccells[ci];
    const int na = g.cell_count[a], ca = g.cell_start[a];
    const BoxDev B = g.boxes[g.cell_box[a]];
    const float mscale = munit * g.m_max[g.cell_box[a]];
    const float padw = window_pad(g, B, g.cell_box[a]);
    const int4* pl = g.plan + (size_t)a * kNSlot;
    if (tid < kNSlot) {
      const int o = c_slot_order[tid];
      const int4 p = pl[o];
      cs.I[tid] = p.x;
      cs.J0[tid] = p.y;
      cs.off[tid + 1] = p.z - p.y;
      cs.runs[tid + 1] = (p.x + 31) >> 5;
      cs.ioff[tid + 1] = p.x;
      const int b = neighbour_cell(g, a, o);
      cs.nb_[tid] = g.cell_count[b];
      cs.cb_[tid] = g.cell_start[b];
      const Slot sl = slot_info(o);
      cs.offv[tid] = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    }
    if (tid == 0) {
      cs.off[0] = 0;
      cs.runs[0] = 0;
      cs.ioff[0] = 0;
      cs.item_next = 0;
    }
    __syncthreads();
    if (tid == 0) {
      for (int q = 0; q < kNSlot; q++) {
        cs.off[q + 1] += cs.off[q];
        cs.runs[q + 1] += cs.runs[q];
        cs.ioff[q + 1] += cs.ioff[q];
      }
    }
    __syncthreads();
    const int total = cs.off[kNSlot];
    const int sumI = cs.ioff[kNSlot];
    // variable part (checked by the plan): kCellElemJ (total + kPad + 4) +
    // kCellElemA na + kCellElemI sumI bytes
    float* S = reinterpret_cast<float*>(var);                          // staged groups
    float4* Ax = reinterpret_cast<float4*>(S + staged_floats(total));  // [na] {x', y', z', h}
    long long* acc_r = reinterpret_cast<long long*>(Ax + na);          // [na]
    long long* acc_d = acc_r + na;                                     // [na]
    int* acc_n = reinterpret_cast<int*>(acc_d + na);                   // [na]
    uint16_t* SI = reinterpret_cast<uint16_t*>(acc_n + na);            // [sumI]
    // stage the 27 windows in sorted order (synchronous loads, three lookups
    // in flight per thread: more would spill at this kernel's 64 registers),
    // the slots' particle lists of a, and cell a
    stage_flat<3>(
        cs.off, total, tid, kCellThreads,
        [&](int f, int q) {
          const Slot sl = slot_info(c_slot_order[q]);
          const int cb = cs.cb_[q];
          const int pos = order_pos(sl.s, cs.J0[q] + f - cs.off[q], cs.nb_[q]);
          return cb + (int)g.perm[(size_t)sl.k * g.n + cb + pos];
        },
        [&](int sj) { return g.xm[sj]; },
        [&](int f, int, float4 x) { put_staged(S, f, x, 0.0f, 0.0f, 0.0f); });
    for (int t = tid, q = 0; t < sumI; t += kCellThreads) {
      while (cs.ioff[q + 1] <= t) q++;
      const int o = c_slot_order[q];
      const Slot sl = slot_info(o);
      const int p = t - cs.ioff[q];
      const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
      SI[t] = g.perm[(size_t)sl.k * g.n + ca + pos_i];
    }
    for (int t = tid; t < na; t += kCellThreads) {
      const float4 xm = g.xm[ca + t];
      Ax[t] = make_float4(xm.x, xm.y, xm.z, g.hs[ca + t]);
      acc_r[t] = 0;
      acc_d[t] = 0;
      acc_n[t] = 0;
    }
    __syncthreads();
    // work items: (slot, run of 32 particles of a), pulled by warps
    const int nitems = cs.runs[kNSlot];
    for (;;) {
      int it = 0;
      if (lane == 0) it = atomicAdd(&cs.item_next, 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      if (it >= nitems) break;
      const int q = warp_seg_of(cs.runs, kNSlot, it, lane);
      const int o = c_slot_order[q];
      const Slot sl = slot_info(o);
      float ux, uy, uz;
      axis_u(sl.k, ux, uy, uz);
      const int p = ((it - cs.runs[q]) << 5) + lane;
      LaneI L;
      lane_init(L);
      float d_lo = 3.0e38f, d_hi = -3.0e38f;
      int il = 0;
      if (p < cs.I[q]) {
        il = SI[cs.ioff[q] + p];
        const float4 xh = Ax[il];
        float di;
        if (g.moved) {  // windows from the sort's projections
          const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
          di = sl.s * g.dist[(size_t)sl.k * g.n + ca + pos_i];
        } else {
          di = sl.s * project(xh, ux, uy, uz);
        }
        lane_set(L, B, g.gamma, sl, ca + il, xh);
        const float H = g.gamma * xh.w;
        d_lo = di - H - padw;
        d_hi = di + H + padw;
      }
      const float w_lo = warp_min(d_lo), w_hi = warp_max(d_hi);
      const int s0 = cs.off[q], len = cs.off[q + 1] - s0;
      const float offv = cs.offv[q];
      const int J0q = cs.J0[q], nbq = cs.nb_[q], cbq = cs.cb_[q];
      // after pv_update_positions the staged positions are no longer in sorted
      // order: the window searches then read the sort's projections
      const unsigned Sa = smem_addr(S);
      auto proj = [&](int e) {  // projection of staged element e, as sorted
        return g.moved ? proj_asc(g, sl.k, sl.s, cbq, nbq, J0q + e, offv)
                       : staged_proj(Sa + cand_off(s0 + e), ux, uy, uz, sl.s, offv);
      };
      const int lo = s0 + ((o == kSelfSlot)
                               ? warp_first_true(len, lane, [&](int e) { return proj(e) > w_lo; })
                               : 0);
      const int hi = s0 + warp_first_true(len, lane, [&](int e) { return proj(e) >= w_hi; });
      const size_t kbq = (size_t)sl.k * g.n + cbq;
      auto jidx = [&](int j) {
        return cbq + (int)g.perm[kbq + order_pos(sl.s, J0q + j - s0, nbq)];
      };
      sweep_fwd(L, smem_addr(S), lo, hi, g, B, jidx, guards);
      float prho, pD;
      int pn;
      lane_sums(L, prho, pD, pn);
      if (p < cs.I[q] && pn > 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&acc_r[il]),
                  (unsigned long long)__float2ll_rn(prho * (float)kFixScale));
        atomicAdd(reinterpret_cast<unsigned long long*>(&acc_d[il]),
                  (unsigned long long)__float2ll_rn(pD * (float)kFixScale));
        atomicAdd(&acc_n[il], pn);
      }
    }
    __syncthreads();
    for (int t = tid; t < na; t += kCellThreads) {
      write_out(g, ca + t, acc_r[t], acc_d[t], acc_n[t], rho, drho_dh, n_ngb, mscale);
      inter += (unsigned long long)(acc_n[t] - 1);
    }
    __syncthreads();
  }
  // then the tiny cells, one per warp, in the dynamic shared memory that the
  // cells no longer use (at least kCellWarps * kTinyWarpBytes of it)
  tiny_phase_fwd(
      g, reinterpret_cast<unsigned char*>(var) + warp * kTinyWarpBytes, lane,
      [&](int a, int s, float prho, float pD, int pn) {
        const int i = g.orig[s];
        const float h = g.hs[s];
        const float H = g.gamma * h;
        const float c = (float)(16.0 / 3.14159265358979323846) * g.m_max[g.cell_box[a]] /
                        (H * H * H);
        rho[i] = c * prho;
        if (drho_dh) drho_dh[i] = -(c / h) * pD;
        if (n_ngb) n_ngb[i] = pn - 1;  // the self pair j = i
      },
      inter, guards);
  for (int s = 16; s > 0; s >>= 1) {
    inter += __shfl_xor_sync(0xffffffffu, inter, s);
    guards += __shfl_xor_sync(0xffffffffu, guards, s);
  }
  if (lane == 0) {
    if (inter) atomicAdd(&g.counters[0], inter);
    if (guards) atomicAdd(&g.counters[1], (unsigned long long)guards);
  }
}

// ---- task kernel (cells too dense for the cell-centric kernel) ---------------------

// BlkI particles (and threads) per task; 1024 threads per SM for every BlkI.
template <int BlkI>
__global__ void __launch_bounds__(BlkI, 1024 / BlkI) k_density_tasks(GridDev g) {
  pdl_enter();
  __shared__ __align__(16) float s_S[staged_floats(kTileJ)];
  __shared__ float s_d[kTileJ];
  __shared__ int s_j[kTileJ + kPad];
  __shared__ int s_task;
  if (*g.flags) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntask = *g.ntask;
  if (ntask == 0) return;  // no task cells: leave without touching the task counter
  int guards = 0;
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
    LaneI L;
    lane_init(L);
    const int p = tk.p0 + warp * 32 + lane;
    const bool valid = p < tk.p1;
    float d_lo = 3.0e38f, d_hi = -3.0e38f;
    if (valid) {
      const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
      const int si = ca + g.perm[kbase + ca + pos_i];
      const float h = g.hs[si];
      const float4 xm = g.xm[si];
      lane_set(L, B, g.gamma, sl, si, make_float4(xm.x, xm.y, xm.z, h));
      const float di = sl.s * g.dist[kbase + ca + pos_i];
      const float H = g.gamma * h;
      d_lo = di - H - window_pad(g, B, g.cell_box[a]);
      d_hi = di + H + window_pad(g, B, g.cell_box[a]);
    }
    const float w_lo = warp_min(d_lo), w_hi = warp_max(d_hi);
    for (int j0 = tk.j0; j0 < tk.j1; j0 += kTileJ) {
      const int len = min(kTileJ, tk.j1 - j0);
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int pos_j = order_pos(sl.s, j0 + e, nb);
        const int jl = g.perm[kbase + cb + pos_j];
        put_staged(s_S, e, g.xm[cb + jl], 0.0f, 0.0f, 0.0f);
        s_d[e] = sl.s * g.dist[kbase + cb + pos_j] + off;
        s_j[e] = cb + jl;
      }
      __syncthreads();
      if (w_hi > w_lo) {
        const int lo = (o == kSelfSlot) ? upper_bound_f(s_d, len, w_lo) : 0;
        const int hi = lower_bound_f(s_d, len, w_hi);
        auto jidx = [&](int j) { return s_j[j]; };
        sweep_fwd(L, smem_addr(s_S), lo, hi, g, B, jidx, guards);
      }
      __syncthreads();
    }
    float prho, pD;
    int pn;
    lane_sums(L, prho, pD, pn);
    if (valid && pn > 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[L.si]),
                (unsigned long long)__float2ll_rn(prho * (float)kFixScale));
      atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[(size_t)g.n + L.si]),
                (unsigned long long)__float2ll_rn(pD * (float)kFixScale));
      atomicAdd(reinterpret_cast<unsigned long long*>(&g.acc[2 * (size_t)g.n + L.si]),
                (unsigned long long)pn);
    }
  }
  for (int s = 16; s > 0; s >>= 1) guards += __shfl_xor_sync(0xffffffffu, guards, s);
  if (lane == 0 && guards) atomicAdd(&g.counters[1], (unsigned long long)guards);
}

// Fixed point -> caller order for the particles of the task-path cells.  The
// self-slot tasks of a cell cover its positions [0, na) in blocks of g.task_blk,
// so one warp per self-slot task finalises cell-local indices [p0, p1): big
// cells are spread over many warps.  (A pass whose slot mask leaves out the
// self slot has no such tasks: one block per task cell then.)
constexpr int kFinBatch = 4;  // particles per thread in flight in the task-path finalize
__global__ void k_finalize_t(GridDev g, float* __restrict__ rho, float* __restrict__ drho_dh,
                             int32_t* __restrict__ n_ngb) {
  pdl_enter();
  if (*g.flags) return;
  const int lane = threadIdx.x & 31;
  const float munit = (float)(16.0 / 3.14159265358979323846 * kFixInv);
  unsigned long long inter = 0;
  const size_t N = (size_t)g.n;
  // The slots ca + t0 + k stride (k < kFinBatch, below t1) of one thread: every
  // load first, so that the batch's random accesses are in flight together,
  // then the outputs, then the clears.
  auto fin = [&](int ca, int t0, int stride, int t1, float mscale) {
    long long ar[kFinBatch], ad[kFinBatch], an[kFinBatch];
#pragma unroll
    for (int k = 0; k < kFinBatch; k++) {
      const int t = t0 + k * stride;
      if (t < t1) {
        const size_t s = (size_t)ca + t;
        ar[k] = g.acc[s];
        ad[k] = g.acc[N + s];
        an[k] = g.acc[2 * N + s];
      }
    }
#pragma unroll
    for (int k = 0; k < kFinBatch; k++) {
      const int t = t0 + k * stride;
      if (t < t1) {
        write_out(g, ca + t, ar[k], ad[k], (int)an[k], rho, drho_dh, n_ngb, mscale);
        inter += (unsigned long long)(an[k] - 1);
      }
    }
#pragma unroll
    for (int k = 0; k < kFinBatch; k++) {
      const int t = t0 + k * stride;
      if (t < t1) {
        const size_t s = (size_t)ca + t;
        g.acc[s] = 0;
        g.acc[N + s] = 0;
        g.acc[2 * N + s] = 0;
      }
    }
  };
  if ((g.slot_mask >> kSelfSlot) & 1u) {
    const int ntask = *g.ntask;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntask;
         w += (gridDim.x * blockDim.x) >> 5) {
      const Task tk = decode(g.tasks[w]);
      if (tk.o != kSelfSlot) continue;
      const int ca = g.cell_start[tk.a];
      const float mscale = munit * g.m_max[g.cell_box[tk.a]];
      for (int t0 = tk.p0 + lane; t0 < tk.p1; t0 += 32 * kFinBatch) fin(ca, t0, 32, tk.p1, mscale);
    }
  } else {
    const int nt = *g.n_tcells;
    for (int c = blockIdx.x; c < nt; c += gridDim.x) {
      const int a = g.tcells[c];
      const int ca = g.cell_start[a], na = g.cell_count[a];
      const float mscale = munit * g.m_max[g.cell_box[a]];
      for (int t0 = threadIdx.x; t0 < na; t0 += blockDim.x * kFinBatch)
        fin(ca, t0, blockDim.x, na, mscale);
    }
  }
  for (int s = 16; s > 0; s >>= 1) inter += __shfl_xor_sync(0xffffffffu, inter, s);
  if ((threadIdx.x & 31) == 0 && inter) atomicAdd(&g.counters[0], inter);
}

// ---- candidates of the method's windows (diagnostic) -------------------------------
// One thread per (cell a, slot o): for every particle of a, the number of
// particles of b inside its window on the sorted axis (exact per-particle
// window, no padding): |d_j - d_i| < H_i for the self slot, d_j < d_i + H_i
// for a neighbour slot.
__global__ void k_count_candidates(GridDev g) {
  pdl_enter();
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
          cnt += count_below(g, sl.k, sl.s, cb, nb, off, di + H);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&g.counters[2], cnt);
}

// Counts of the adjoint sweep (diagnostic): one warp per (cell a, slot o),
// lanes over the particles of a.  For each particle i, the particles j of the
// sorted window whose projected distance is below max(H_i, H_j)
// ("candidates", counters[3]) and those with r_ij < max(H_i, H_j) (counters[4]),
// j = i included.
__global__ void k_count_adjoint(GridDev g) {
  pdl_enter();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  unsigned long long cand = 0, pairs = 0;
  if (wid < g.ncell * kNSlot && !*g.flags) {
    const int a = wid / kNSlot, o = wid % kNSlot;
    const int na = g.cell_count[a];
    const int b = na ? neighbour_cell(g, a, o) : a;
    const int nb = g.cell_count[b];
    if (na && nb) {
      const BoxDev& B = g.boxes[g.cell_box[a]];
      const Slot sl = slot_info(o);
      const int ca = g.cell_start[a], cb = g.cell_start[b];
      const size_t kb = (size_t)sl.k * g.n;
      const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
      const float Hmb = g.cell_Hmax[b];
      for (int p = lane; p < na; p += 32) {
        const int pos = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
        const int si = ca + g.perm[kb + ca + pos];
        const float Hi = g.gamma * g.hs[si];
        const float di = sl.s * g.dist[kb + ca + pos];
        const float4 xi = g.xm[si];
        const float x = xi.x - sl.ox * B.edge_f, y = xi.y - sl.oy * B.edge_f,
                    z = xi.z - sl.oz * B.edge_f;
        const float R0 = fmaxf(Hi, Hmb);
        int j = 0, j1 = nb;
        if (o == kSelfSlot) {
          j = upper_bound_f(g.dist + cb, nb, di - R0);
          j1 = lower_bound_f(g.dist + cb, nb, di + R0);
        }
        for (; j < j1; j++) {
          const float dj = proj_asc(g, sl.k, sl.s, cb, nb, j, off);
          if (dj - di >= R0) break;
          const int sj = cb + g.perm[kb + cb + order_pos(sl.s, j, nb)];
          const float R = fmaxf(Hi, g.gamma * g.hs[sj]);
          if (fabsf(dj - di) < R) {
            cand++;
            const float4 xj = g.xm[sj];
            const float dx = x - xj.x, dy = y - xj.y, dz = z - xj.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < R * R) pairs++;
          }
        }
      }
    }
  }
  for (int s = 16; s > 0; s >>= 1) {
    cand += __shfl_xor_sync(0xffffffffu, cand, s);
    pairs += __shfl_xor_sync(0xffffffffu, pairs, s);
  }
  if (lane == 0) {
    if (cand) atomicAdd(&g.counters[3], cand);
    if (pairs) atomicAdd(&g.counters[4], pairs);
  }
}

// Per orientation class (self, face, edge, corner) of the slot: the distance
// tests of the method's sorted windows (self: |d_j - d_i| < H_i, j = i
// included; pairs: d_j < d_i + H_i) into counters[8 + 2c], and the pairs
// j != i with r < H_i into counters[9 + 2c].  One warp per (cell, slot), lanes
// over the particles of the cell (diagnostic).
__global__ void k_count_classes(GridDev g) {
  pdl_enter();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  unsigned long long cand = 0, inter = 0;
  int cls = 0;
  if (wid < g.ncell * kNSlot && !*g.flags) {
    const int a = wid / kNSlot, o = wid % kNSlot;
    const int na = g.cell_count[a];
    const int b = na ? neighbour_cell(g, a, o) : a;
    const int nb = g.cell_count[b];
    const Slot sl = slot_info(o);
    cls = sl.v2;
    if (na && nb) {
      const BoxDev& B = g.boxes[g.cell_box[a]];
      const int ca = g.cell_start[a], cb = g.cell_start[b];
      const size_t kb = (size_t)sl.k * g.n;
      const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
      for (int p = lane; p < na; p += 32) {
        const int pos = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
        const int si = ca + g.perm[kb + ca + pos];
        const float Hi = g.gamma * g.hs[si];
        const float di = sl.s * g.dist[kb + ca + pos];
        const float4 xi = g.xm[si];
        const float x = xi.x - sl.ox * B.edge_f, y = xi.y - sl.oy * B.edge_f,
                    z = xi.z - sl.oz * B.edge_f;
        int j = 0, j1 = nb;
        if (o == kSelfSlot) {
          j = upper_bound_f(g.dist + cb, nb, di - Hi);
          j1 = lower_bound_f(g.dist + cb, nb, di + Hi);
        }
        for (; j < j1; j++) {
          const float dj = proj_asc(g, sl.k, sl.s, cb, nb, j, off);
          if (dj - di >= Hi) break;
          cand++;
          const int sj = cb + g.perm[kb + cb + order_pos(sl.s, j, nb)];
          if (sj == si) continue;
          const float4 xj = g.xm[sj];
          const float dx = x - xj.x, dy = y - xj.y, dz = z - xj.z;
          if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < Hi * Hi) inter++;
        }
      }
    }
  }
  // the lanes of a warp share (cell, slot), so one class per warp
  for (int s = 16; s > 0; s >>= 1) {
    cand += __shfl_xor_sync(0xffffffffu, cand, s);
    inter += __shfl_xor_sync(0xffffffffu, inter, s);
  }
  if (lane == 0) {
    if (cand) atomicAdd(&g.counters[8 + 2 * cls], cand);
    if (inter) atomicAdd(&g.counters[9 + 2 * cls], inter);
  }
}

}  // namespace

cudaError_t launch_plan_slots(const GridDev& g, int wide, cudaStream_t st) {
  const int nthr = g.ncell * kNSlot;
  if (nthr == 0) return cudaSuccess;
  PV_LAUNCH(k_plan_slots, (nthr + 255) / 256, 256, 0, st, g, wide);
  return cudaSuccess;
}

cudaError_t launch_plan(const GridDev& g, int wide, int smem_budget, int elem_j, int elem_a,
                        int elem_i, cudaStream_t st) {
  const int nthr = g.ncell * kNSlot;
  PV_LAUNCH(k_plan_slots, (nthr + 255) / 256, 256, 0, st, g, wide);
  PV_LAUNCH(k_plan_cells, (g.ncell + 127) / 128, 128, 0, st,
            g, smem_budget, elem_j, elem_a, elem_i);
  // one warp per (task cell, slot): enough warps that the big cells' many
  // (cell, slot) pairs do not queue behind each other
  PV_LAUNCH(k_plan_tasks, 2048, 256, 0, st, g, wide);
  return cudaSuccess;
}

int64_t max_tasks_for(int64_t n, int64_t ncell) {
  return (int64_t)kNSlot * (n / kTaskBlkMin + ncell) + 64;
}

cudaError_t launch_density(const GridDev& g, float* rho, float* drho_dh, int32_t* n_ngb,
                           int num_sms, int ctas_per_sm, cudaStream_t st, cudaEvent_t t0,
                           cudaEvent_t t1) {
  if (g.n == 0) return cudaSuccess;
  if (ctas_per_sm < 1 || ctas_per_sm > 4) return cudaErrorInvalidValue;
  cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(&k_density_cells),
                                       kCellSmemFor[1], st);
  if (e != cudaSuccess) return e;
  const int smem = kCellSmemFor[ctas_per_sm];
  if ((e = launch_plan(g, 0, smem, kCellElemJ, kCellElemA, kCellElemI, st)) != cudaSuccess)
    return e;
  if (t0 && (e = cudaEventRecord(t0, st)) != cudaSuccess) return e;
  PV_LAUNCH(k_density_cells, num_sms * ctas_per_sm, kCellThreads, smem, st, g, rho, drho_dh,
            n_ngb);
  if (t1 && (e = cudaEventRecord(t1, st)) != cudaSuccess) return e;
  // (a plain launch: as a dependent of the persistent cell kernel, the task
  // kernel made the 4M clustered step 0.6 ms slower)
  switch (g.task_blk) {
    case 64: PV_LAUNCH_PLAIN(k_density_tasks<64>, num_sms * 16, 64, 0, st, g); break;
    case 256: PV_LAUNCH_PLAIN(k_density_tasks<256>, num_sms * 4, 256, 0, st, g); break;
    default: PV_LAUNCH_PLAIN(k_density_tasks<128>, num_sms * 8, 128, 0, st, g); break;
  }
  PV_LAUNCH(k_finalize_t, num_sms * 8, 256, 0, st, g, rho, drho_dh, n_ngb);
  return cudaSuccess;
}

cudaError_t launch_count_candidates(const GridDev& g, cudaStream_t st) {
  const int nthr = g.ncell * kNSlot;
  if (nthr == 0) return cudaSuccess;
  PV_LAUNCH(k_count_candidates, (nthr + 255) / 256, 256, 0, st, g);
  PV_LAUNCH(k_count_adjoint, (nthr * 32 + 255) / 256, 256, 0, st, g);
  PV_LAUNCH(k_count_classes, (nthr * 32 + 255) / 256, 256, 0, st, g);
  return cudaSuccess;
}

}  // namespace pv
