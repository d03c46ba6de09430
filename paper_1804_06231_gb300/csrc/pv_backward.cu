// pv_backward.cu -- adjoint of the density gather.
//
// With g_i = dL/drho_i, k_i = dL/d(drho/dh)_i, W_r = dW/dr and W_hr =
// d2W/dh dr:
//   dL/dh_i = g_i drho/dh_i + k_i sum_j m_j d2W/dh2(r_ij, h_i)
//   dL/dx_i = sum_{j!=i} (x_i - x_j)/r_ij [ m_j (g_i W_r(r,H_i) + k_i W_hr(r,h_i)) [r<H_i]
//                                          + m_i (g_j W_r(r,H_j) + k_j W_hr(r,h_j)) [r<H_j] ]
// Both terms are gathered for particle i while sweeping the same sorted cell
// pairs as the forward pass (the second, "transposed" term is the scatter of
// the pair's symmetric position derivative, done as a gather), with the
// window widened to max(H_i, H_max of the other cell).
//
// Half-scaled shape functions (w, w', w'' of the workload's spline, divided
// by 16/pi; s = 1 - q):
//   th = (3w + q w')            q<1/2: 3/2 + q^2 (18q - 15)    else s^2 (3 - 6q)
//   uh = (12w + 8q w' + q^2 w'') q<1/2: 6 + q^2 (126q - 90)    else 6 s (7s^2 - 6s + 1)
//   vr = w'/q                   q<1/2: -6 + 9q                 else -3 s^2 / q
//   vh = (4w' + q w'')/q        q<1/2: -30 + 54q               else -12 s^2/q + 6 s
// so that dW/dh = -(16/pi) th/(h H^3), d2W/dh2 = (16/pi) uh/(h^2 H^3),
// W_r/r = (16/pi) vr/H^5 and W_hr/r = -(16/pi) vh/(h H^5).  With
// G = g/H^5 and K = k/(h H^5) per particle:
//   dL/dx_i = (16/pi) sum_j (x_i-x_j) [ m_j (G_i vr_i - K_i vh_i) + m_i (G_j vr_j - K_j vh_j) ]
//   dL/dh_i = (16/pi)/(h_i H_i^3) [ -g_i sum_j m_j th_i + (k_i/h_i) sum_j m_j uh_i ]
//
// Mapping: the cell-centric kernel of the forward pass (one CTA per cell, 27
// staged windows, warps pulling (slot, run) items, candidates pre-filtered 32
// at a time into per-lane hit masks held in registers), with both the own and
// the transposed cut-off in the pre-filter; per-particle sums in 32-bit fixed-point shared-memory
// accumulators (one integer addition per particle and work item, so the
// result does not depend on which warp took which item).  A staged particle
// takes 32 bytes ({x, y, z, H^2 + guard} and {m, G', K, H}), so three CTAs fit
// an SM.  Cells whose windows exceed the shared-memory budget run as tasks
// (cell, slot, block of 128 particles) with 64-bit fixed-point global
// accumulators.
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {

namespace {

constexpr int kTileJ = 512;
constexpr int kCellThreads = 256;
// dynamic shared memory of k_backward_cells for 1 to 3 resident CTAs per SM
// (its registers allow no more than three)
constexpr int kCellSmemFor[4] = {0, 200 * 1024, 110 * 1024, 72 * 1024};
constexpr int kPad = 32;
constexpr int kElemJ = 32;   // staged bytes per particle of a window: {x,y,z,E}, {m,G,K,H}
constexpr int kElemA = 32;   // bytes per particle of the cell: 3 x 64-bit + 2 x 32-bit fixed point

__constant__ int8_t c_border[kNSlot] = {13, 4,  10, 12, 14, 16, 22, 1,  3,  5,  7,  9, 11, 15,
                                        17, 19, 21, 23, 25, 0,  2,  6,  8,  18, 20, 24, 26};

struct TaskB {
  int a, o, p0, p1, j0, j1;
};

__device__ __forceinline__ TaskB decode_b(int4 t) {
  TaskB r;
  r.a = t.x;
  r.o = t.y;
  r.p0 = t.z & 0xffff;
  r.p1 = (int)((unsigned)t.z >> 16);
  r.j0 = t.w & 0xffff;
  r.j1 = (int)((unsigned)t.w >> 16);
  return r;
}

// Upstream gradients to cell order, with the per-particle constants of the
// sweep, in the form the sweeps stage them: bx = {x', y', z', E = H^2 +
// guard} and ba = {m / m_max, G' = G - 4K, K, H} with G = g/H^5 and
// K = k/(h H^5).
// A non-finite upstream gradient latches PV_FLAG_BAD_GRADIENT (the sweeps
// then leave the outputs untouched); every particle raises its cell's bound
// (|G'| + |K|) H of the fixed-point units and lowers its cell's smallest
// support H (which decides whether the task sweeps test their chunks).
__global__ void k_bwd_prep(GridDev g, const float* __restrict__ g_rho,
                           const float* __restrict__ g_D) {
  pdl_enter();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (*g.flags) return;  // the same for the whole warp
  int cell = -1;
  float bound = 0.0f, Hs = 3.0e38f;
  if (s < g.n) {
    const int i = g.orig[s];
    const BoxDev& B = g.boxes[box_of_particle(g, i)];
    const float h = g.hs[s];
    const float H = g.gamma * h;
    const float H2 = H * H;
    const float iH5 = 1.0f / (H2 * H2 * H);
    const float gi = g_rho[i];
    const float ki = g_D ? g_D[i] : 0.0f;
    if (!isfinite(gi) || !isfinite(ki)) atomicOr(g.flags, PV_FLAG_BAD_GRADIENT);
    const float gb = guard_band(H, B.edge_f);
    const float4 xm = g.xm[s];
    const float K = ki * iH5 / h;
    const float Gp = fmaf(-4.0f, K, gi * iH5);
    g.bx[s] = make_float4(-xm.x, -xm.y, -xm.z, H2 + gb);  // negated offsets
    g.ba[s] = make_float4(xm.w, Gp, K, H);
    cell = g.pcell[i];
    bound = (fabsf(Gp) + fabsf(K)) * H;
    Hs = H;
  }
  // particles are in cell order, so a warp spans a few cells: one atomic per
  // cell and warp (non-negative floats order as their bit patterns)
  const unsigned same = __match_any_sync(0xffffffffu, cell);
  const unsigned mx = __reduce_max_sync(same, __float_as_uint(bound));
  const unsigned mn = __reduce_min_sync(same, __float_as_uint(Hs));
  if (cell >= 0 && (threadIdx.x & 31) == __ffs(same) - 1) {
    atomic_max_nonneg(&g.bwd_cmax[cell], __uint_as_float(mx));
    atomicMin(reinterpret_cast<unsigned*>(&g.bwd_hmin[cell]), mn);
  }
}

// Fixed-point units of the adjoint sums.  Per pair, with normalised masses
// m <= 1: |th| <= 3/2 and |uh| <= 6; the own gradient term is at most
// 6 (|G'_i| + |K_i|) r with r < H_i and the transposed one 6 (|G'_j| + |K_j|) r
// with r < H_j (|vr|, |w6| <= 6), so |cc dx| <= 13 Bn, Bn being the largest
// (|G'| + |K|) H in the 27 cells around the particle's cell (the 13 instead of
// 12 covers the guard band of the cut-offs).  A cell-centric cell meets each of
// its particles with at most `staged` + 1 partners, a task-path cell at most
// 27 x 65535: the units below keep every sum under 2^30 (32-bit th, uh sums of
// a cell-centric cell), 2^62 (64-bit gradient sums) and 2^62 (64-bit th, uh
// sums of the task path, units 2^-36).  A bound per neighbourhood, not per box,
// keeps the resolution fine where the supports of a clustered box span
// orders of magnitude.
__device__ __forceinline__ float fix_scale_s32(int staged) { return 1073741824.0f / (6.0f * (staged + 1)); }
__device__ __forceinline__ float fix_scale_g64(float bn, float pairs) {
  return 4611686018427387904.0f / (13.0f * fmaxf(bn, 1.0e-30f) * pairs);  // 2^62 / (13 Bn pairs)
}
constexpr float kTaskPairs = 27.0f * 65535.0f + 1.0f;
constexpr double kFixS64 = 68719476736.0;  // 2^36

// Bn of cell a: the largest per-cell bound over a and its 26 neighbours, the
// warp's lanes taking one neighbour each (the whole warp calls it).  The
// bounds are non-negative, so their order is that of the bit patterns
// (fmaxf with 0 also drops a NaN, as a running fmaxf would).
__device__ __forceinline__ float nbhd_bound(const GridDev& g, int a, int lane) {
  const float v = lane < kNSlot ? fmaxf(g.bwd_cmax[neighbour_cell(g, a, lane)], 0.0f) : 0.0f;
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

// Half-scaled kernel factors of the adjoint, without branches.  With
// s = 1 - q, each factor is one polynomial on q < 1/2 and one on 1/2 <= q < 1
// (the two cubic pieces of the spline), chosen by one predicate:
//   th = 3w + q w'                 q<1/2: 3/2 + q^2 (18q - 15)   else s^2 (3 - 6q)
//   uh = 12w + 8q w' + q^2 w''     q<1/2: 6 + q^2 (126q - 90)    else 6 s (7s^2 - 6s + 1)
//   vr = w'/q                      q<1/2: 9q - 6                 else -3 s^2 / q
//   w6 = (4w' + q w'')/q - 4 vr    q<1/2: 18q - 6                else 6 s
// (vh = 4 vr + w6 is the factor of W_hr; s is clamped at 0, so every factor
// vanishes for q >= 1).  The gradient coefficient G vr - K vh is formed as
// (G - 4K) vr - K w6, with G' = G - 4K stored per particle.
__device__ __forceinline__ void spline_bwd(float q, float qinv, float& th, float& uh, float& vr,
                                           float& w6) {
  const bool lo = q < 0.5f;
  const float s = fmaxf(1.0f - q, 0.0f), s2 = s * s, q2 = q * q;
  th = lo ? fmaf(q2, fmaf(18.0f, q, -15.0f), 1.5f) : s2 * fmaf(-6.0f, q, 3.0f);
  uh = lo ? fmaf(q2, fmaf(126.0f, q, -90.0f), 6.0f) : 6.0f * s * fmaf(7.0f, s2, fmaf(-6.0f, s, 1.0f));
  vr = lo ? fmaf(9.0f, q, -6.0f) : (-3.0f * s2) * qinv;
  w6 = lo ? fmaf(18.0f, q, -6.0f) : 6.0f * s;
}

__device__ __forceinline__ void spline_bwd_v(float q, float qinv, float& vr, float& w6) {
  const bool lo = q < 0.5f;
  const float s = fmaxf(1.0f - q, 0.0f);
  vr = lo ? fmaf(9.0f, q, -6.0f) : (-3.0f * s * s) * qinv;
  w6 = lo ? fmaf(18.0f, q, -6.0f) : 6.0f * s;
}

__device__ __forceinline__ float warp_min_b(float v) { return warp_min_f(v); }
__device__ __forceinline__ float warp_max_b(float v) { return warp_max_f(v); }

// shared-memory loads through 32-bit shared-window addresses
__device__ __forceinline__ unsigned smem_addr_b(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float4 lds4_b(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}

struct LaneB {
  float2 xy;             // x, y of i in b's frame (a packed pair)
  float z;
  float Hsq_hi, Hsq_lo, Hinv, H, G, K, m;  // G holds G' = G - 4K
  int si;
  float Sth, Suh, gx, gy, gz;
  float2 Sth2, Suh2, g2x, g2y, g2z;  // sums of the packed rounds (halves added at the end)
};

// folds the packed rounds' sums into the scalar ones
__device__ __forceinline__ void laneb_fold(LaneB& L) {
  L.Sth += L.Sth2.x + L.Sth2.y;
  L.Suh += L.Suh2.x + L.Suh2.y;
  L.gx += L.g2x.x + L.g2x.y;
  L.gy += L.g2y.x + L.g2y.y;
  L.gz += L.g2z.x + L.g2z.y;
  L.Sth2 = L.Suh2 = L.g2x = L.g2y = L.g2z = make_float2(0.0f, 0.0f);
}

// An inactive lane sits far outside every window (its r^2 is ~1e36), so the
// pre-filter gives it no hits.
__device__ __forceinline__ void laneb_init(LaneB& L) {
  L.xy = make_float2(1.0e18f, 1.0e18f);
  L.z = 1.0e18f;
  L.Hsq_hi = L.Hsq_lo = -1.0f;
  L.Hinv = L.H = L.G = L.K = L.m = 0.0f;
  L.si = 0;
  L.Sth = L.Suh = L.gx = L.gy = L.gz = 0.0f;
  L.Sth2 = L.Suh2 = L.g2x = L.g2y = L.g2z = make_float2(0.0f, 0.0f);
}

// The staged records hold the negated offsets (bx = {-x', -y', -z', E}), so
// that x_i - x_j is an addition.
__device__ __forceinline__ void laneb_set(LaneB& L, const GridDev& g, const BoxDev& B,
                                          const Slot& sl, int si) {
  const float4 xe = g.bx[si];
  const float4 ak = g.ba[si];
  L.si = si;
  L.xy = make_float2(-xe.x - sl.ox * B.edge_f, -xe.y - sl.oy * B.edge_f);
  L.z = -xe.z - sl.oz * B.edge_f;
  L.m = ak.x; L.G = ak.y; L.K = ak.z; L.H = ak.w;
  L.Hsq_hi = xe.w;
  // H^2 - guard = 2 H^2 - (H^2 + guard), to within an ulp: the band only has
  // to cover the FP32 rounding of r^2, which it does twice over
  L.Hsq_lo = fmaf(2.0f * L.H, L.H, -xe.w);
  L.Hinv = 1.0f / L.H;
}

// Adds the own (scaled by mo = m_j or 0) and transposed (mt = m_i or 0) terms
// of the pair (i, j) to lane i's five sums (aj = {m_j, G'_j, K_j, H_j}).
__device__ __forceinline__ void bwd_pair(LaneB& L, float dx, float dy, float dz, float r2,
                                         float4 aj, float mo, float mt) {
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float r = r2 * rinv;
  float th, uh, vr, w6, vrj, w6j;
  spline_bwd(r * L.Hinv, L.H * rinv, th, uh, vr, w6);
  spline_bwd_v(__fdividef(r, aj.w), aj.w * rinv, vrj, w6j);
  L.Sth = fmaf(mo, th, L.Sth);
  L.Suh = fmaf(mo, uh, L.Suh);
  const float cc = fmaf(mo, fmaf(L.G, vr, -L.K * w6), mt * fmaf(aj.y, vrj, -aj.z * w6j));
  L.gx = fmaf(cc, dx, L.gx);
  L.gy = fmaf(cc, dy, L.gy);
  L.gz = fmaf(cc, dz, L.gz);
}

// Two pairs at once in packed FP32 (fma.rn.f32x2).  The factors come from
// the half-scaled shape function w = s^3 - 4 t^3 (s = max(1 - q, 0),
// t = max(1/2 - q, 0), the two cubic pieces without a branch) and its
// derivatives w' = 12 t^2 - 3 s^2, w'' = 6 s - 24 t:
//   th = 3 w + q w',  uh = 12 w + 8 q w' + q^2 w'',  vr = w' / q,  w6 = w''
// (the same values as spline_bwd: on q < 1/2, w' = 9 q^2 - 6 q).
__device__ __forceinline__ float2 max0(float2 v) {
  return make_float2(fmaxf(v.x, 0.0f), fmaxf(v.y, 0.0f));
}
__device__ __forceinline__ void wprime2(float2 q, float2& s, float2& s2, float2& w1, float2& w2) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  s = max0(__ffma2_rn(q, m1, make_float2(1.0f, 1.0f)));
  const float2 t = max0(__ffma2_rn(q, m1, make_float2(0.5f, 0.5f)));
  s2 = __fmul2_rn(s, s);
  const float2 t2 = __fmul2_rn(t, t);
  w1 = __ffma2_rn(t2, make_float2(12.0f, 12.0f), __fmul2_rn(s2, make_float2(-3.0f, -3.0f)));
  w2 = __ffma2_rn(t, make_float2(-24.0f, -24.0f), __fmul2_rn(s, make_float2(6.0f, 6.0f)));
  s = __fmul2_rn(s2, s);  // s^3
  s2 = __fmul2_rn(t2, t);  // t^3
}

// The own and transposed terms of two pairs A and B (records qA/aA, qB/aB;
// differences dxy, dz as bwd_r2 forms them) with masses mo (own: m_j or 0)
// and mt (transposed: m_i or 0), added to lane i's five sums.
__device__ __forceinline__ void bwd_pair2(LaneB& L, float2 r2, float2 dx, float2 dy, float2 dz,
                                          float4 aA, float4 aB, float2 mo, float2 mt) {
  const float2 rinv = make_float2(rsqrtf(fmaxf(r2.x, 1e-30f)), rsqrtf(fmaxf(r2.y, 1e-30f)));
  const float2 r = __fmul2_rn(r2, rinv);
  // own side, q = r / H_i
  const float2 q = __fmul2_rn(r, make_float2(L.Hinv, L.Hinv));
  float2 s3, t3, w1, w2;
  wprime2(q, s3, t3, w1, w2);
  const float2 w = __ffma2_rn(t3, make_float2(-4.0f, -4.0f), s3);
  const float2 qw1 = __fmul2_rn(q, w1);
  const float2 th = __ffma2_rn(w, make_float2(3.0f, 3.0f), qw1);
  const float2 uh = __ffma2_rn(__fmul2_rn(q, q), w2,
                               __ffma2_rn(w, make_float2(12.0f, 12.0f),
                                          __fmul2_rn(qw1, make_float2(8.0f, 8.0f))));
  const float2 qinv = __fmul2_rn(make_float2(L.H, L.H), rinv);
  const float2 vr = __fmul2_rn(w1, qinv);
  // transposed side, q_j = r / H_j
  const float2 Hj = make_float2(aA.w, aB.w);
  const float2 qj = make_float2(__fdividef(r.x, Hj.x), __fdividef(r.y, Hj.y));
  float2 sj3, tj3, wj1, wj2;
  wprime2(qj, sj3, tj3, wj1, wj2);
  const float2 vrj = __fmul2_rn(wj1, __fmul2_rn(Hj, rinv));
  L.Sth2 = __ffma2_rn(mo, th, L.Sth2);
  L.Suh2 = __ffma2_rn(mo, uh, L.Suh2);
  const float2 co = __ffma2_rn(make_float2(L.G, L.G), vr, __fmul2_rn(make_float2(-L.K, -L.K), w2));
  const float2 ct = __ffma2_rn(make_float2(aA.y, aB.y), vrj,
                               __fmul2_rn(make_float2(-aA.z, -aB.z), wj2));
  const float2 cc = __ffma2_rn(mo, co, __fmul2_rn(mt, ct));
  L.g2x = __ffma2_rn(cc, dx, L.g2x);
  L.g2y = __ffma2_rn(cc, dy, L.g2y);
  L.g2z = __ffma2_rn(cc, dz, L.g2z);
}

// r^2 of lane i and a staged record q = {-x_j, -y_j, -z_j, E_j}, and the
// differences: the same FP32 expression in the pre-filter and the
// evaluation, so a hit is exactly a pair in range of the own or the
// transposed test.
__device__ __forceinline__ float bwd_r2(const LaneB& L, float4 q, float2& dxy, float& dz) {
  dxy = __fadd2_rn(L.xy, make_float2(q.x, q.y));
  dz = L.z + q.z;
  const float2 sq = __fmul2_rn(dxy, dxy);
  return fmaf(dz, dz, sq.x) + sq.y;
}

// Adjoint sweep over the staged records [lo, hi) (Sx {-x, -y, -z, E_j = H_j^2 +
// guard_j} and Sa {m_j, G'_j, K_j, H_j} at shared addresses, 16 bytes each);
// jidx(e) gives the cell-order index of staged particle e (read only for FP64
// re-decisions near a cut-off).  Chunk by chunk (32 candidates): the
// pre-filter keeps the candidates with r < max(H_i, H_j) (plus guard; the
// windows themselves reach max(H_i, H_max of the other cell)) in a per-lane
// hit mask held in a register (candidate c at bit 31 - c), then the warp runs
// as many rounds as its busiest lane has hits and each lane applies the exact
// own (r < H_i) and transposed (r < H_j) tests to its own hits.
//
// With sk.on (the task kernel, for the dense cells), a chunk is skipped when
// no lane of the warp can have a pair in it.  The staged tile carries
// summaries per block of 32 from its start (sk.bs, the tile starting at staged
// index sk.s0): the smallest and
// largest projection d_j and the smallest d_j - H_j - pad and largest
// d_j + H_j + pad.  A pair in range of the own cut-off has d_j inside
// (d_i - H_i - pad, d_i + H_i + pad), one in range of the transposed cut-off
// has d_i inside (d_j - H_j - pad, d_j + H_j + pad); a chunk whose blocks
// meet neither the warp's own reach [sk.own_lo, sk.own_hi] nor the warp's
// projections [sk.i_lo, sk.i_hi] holds neither.  The windows reach
// max(H_i, H_max of the other cell), so in a dense cell whose neighbours hold
// a few particles of large support this skips most of them (on the 4M
// clustered box, about 93 % of the chunks of its densest cells' tasks).
struct ChunkSkip {
  unsigned bs;
  int s0;
  float own_lo, own_hi, i_lo, i_hi;
  bool on;
};
constexpr int kSkipMinLen = 96;  // windows this long test their chunks
// ... in tasks whose other cell's largest support exceeds the smallest support
// of the task's cell by this factor (else the reach max(H_i, H_max of b) is
// close to the lanes' own and few chunks would be skipped)
constexpr float kSkipRatio = 1.5f;

// The warp's skip descriptor (the whole warp calls it): lane i at projection
// di with support H (valid lanes only).
__device__ __forceinline__ ChunkSkip chunk_skip(unsigned bs, int s0, bool valid, float di,
                                                float H, float padw) {
  ChunkSkip sk;
  sk.bs = bs;
  sk.s0 = s0;
  sk.own_lo = warp_min_b(valid ? di - H - padw : 3.0e38f);
  sk.own_hi = warp_max_b(valid ? di + H + padw : -3.0e38f);
  sk.i_lo = warp_min_b(valid ? di : 3.0e38f);
  sk.i_hi = warp_max_b(valid ? di : -3.0e38f);
  sk.on = true;
  return sk;
}

template <typename JIndex>
__device__ __forceinline__ void sweep_bwd(LaneB& L, unsigned Sx, unsigned Sa, int lo, int hi,
                                          const GridDev& g, const BoxDev& B, JIndex jidx,
                                          const ChunkSkip& sk) {
  for (int base = lo; base < hi; base += 32) {
    const int cnt = min(32, hi - base);
    if (sk.on) {  // (the same values on every lane: a warp-uniform branch)
      const float4 a0 = lds4_b(sk.bs + 16u * (unsigned)((base - sk.s0) >> 5));
      const float4 a1 = lds4_b(sk.bs + 16u * (unsigned)((base + cnt - 1 - sk.s0) >> 5));
      if (!((fmaxf(a0.y, a1.y) > sk.own_lo && fminf(a0.x, a1.x) < sk.own_hi) ||
            (fmaxf(a0.w, a1.w) > sk.i_lo && fminf(a0.z, a1.z) < sk.i_hi)))
        continue;
    }
    const unsigned px = Sx + 16u * base;
    unsigned m = 0;
    if (cnt == 32) {
#pragma unroll
      for (int c = 0; c < 32; c++) {
        float2 dxy;
        float dz;
        const float4 q = lds4_b(px + 16u * c);
        const float d = bwd_r2(L, q, dxy, dz) - fmaxf(L.Hsq_hi, q.w);
        m = __funnelshift_l(__float_as_uint(d), m, 1);
      }
    } else {
#pragma unroll 1
      for (int c = 0; c < cnt; c++) {
        float2 dxy;
        float dz;
        const float4 q = lds4_b(px + 16u * c);
        const float d = bwd_r2(L, q, dxy, dz) - fmaxf(L.Hsq_hi, q.w);
        m = __funnelshift_l(__float_as_uint(d), m, 1);
      }
      m <<= 32 - cnt;
    }
    const unsigned m0 = m;
    const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(m));
    bool amb = false;
    // two hits per round, evaluated as packed pairs
#pragma unroll 1
    for (int round = 0; round < rounds; round += 2) {
      const int cA = __clz(m);  // 32: this lane has no hit left
      m &= ~__funnelshift_rc(0x80000000u, 0u, cA);
      const int cB = __clz(m);
      m &= ~__funnelshift_rc(0x80000000u, 0u, cB);
      const unsigned oA = 16u * (unsigned)(base + (cA & 31)), oB = 16u * (unsigned)(base + (cB & 31));
      const float4 qA = lds4_b(Sx + oA), qB = lds4_b(Sx + oB);
      const float4 aA = lds4_b(Sa + oA), aB = lds4_b(Sa + oB);
      float2 dA, dB;
      float zA, zB;
      const float rA = bwd_r2(L, qA, dA, zA), rB = bwd_r2(L, qB, dB, zB);
      // pairs within rounding of a cut-off count as in range here and are
      // re-decided in FP64 after the rounds (H_j^2 - guard_j = 2 H_j^2 - E_j)
      const bool oAin = (cA < 32) && (rA < L.Hsq_hi), tAin = (cA < 32) && (rA < qA.w);
      const bool oBin = (cB < 32) && (rB < L.Hsq_hi), tBin = (cB < 32) && (rB < qB.w);
      amb |= (oAin && rA >= L.Hsq_lo) || (tAin && rA >= fmaf(2.0f * aA.w, aA.w, -qA.w)) ||
             (oBin && rB >= L.Hsq_lo) || (tBin && rB >= fmaf(2.0f * aB.w, aB.w, -qB.w));
      bwd_pair2(L, make_float2(rA, rB), make_float2(dA.x, dB.x), make_float2(dA.y, dB.y),
                make_float2(zA, zB), aA, aB, make_float2(oAin ? aA.x : 0.0f, oBin ? aB.x : 0.0f),
                make_float2(tAin ? L.m : 0.0f, tBin ? L.m : 0.0f));
    }
    if (__any_sync(0xffffffffu, amb)) {
      if (amb) {
        unsigned mm = m0;
        while (mm != 0u) {
          const int c = __clz(mm);
          mm &= ~(0x80000000u >> c);
          const int e = base + c;
          const float4 q = lds4_b(Sx + 16u * e);
          const float4 aj = lds4_b(Sa + 16u * e);
          float2 dxy;
          float dz;
          const float r2 = bwd_r2(L, q, dxy, dz);
          const bool gown = r2 < L.Hsq_hi && r2 >= L.Hsq_lo;
          const bool gtr = r2 < q.w && r2 >= fmaf(2.0f * aj.w, aj.w, -q.w);
          if (gown || gtr) {
            const int sj = jidx(e);
            const bool out_o = gown && !guard_inside(g.pos64, L.si, sj, B.L, B.inv_L,
                                                   g.gamma_d * (double)g.hs[L.si]);
            const bool out_t = gtr && !guard_inside(g.pos64, L.si, sj, B.L, B.inv_L,
                                                   g.gamma_d * (double)g.hs[sj]);
            if (out_o || out_t)
              bwd_pair(L, dxy.x, dxy.y, dz, r2, aj, out_o ? -aj.x : 0.0f, out_t ? -L.m : 0.0f);
          }
        }
      }
    }
  }
}

// outputs of one particle from its five sums
__device__ __forceinline__ void write_bwd(const GridDev& g, int s, double Sth, double Suh,
                                          double gx, double gy, double gz,
                                          const float* __restrict__ g_rho,
                                          const float* __restrict__ g_D, float* __restrict__ g_pos,
                                          float* __restrict__ g_h, float mscale) {
  const int i = g.orig[s];
  const float h = g.hs[s];
  const float H = g.gamma * h;
  g_pos[3 * (size_t)i + 0] = mscale * (float)gx;
  g_pos[3 * (size_t)i + 1] = mscale * (float)gy;
  g_pos[3 * (size_t)i + 2] = mscale * (float)gz;
  if (g_h) {
    const float gi = g_rho[i];
    const float ki = g_D ? g_D[i] : 0.0f;
    g_h[i] = mscale / (h * H * H * H) * (float)(-(double)gi * Sth + (double)(ki / h) * Suh);
  }
}

// ---- tiny cells (at most kTinyCell particles) ---------------------------------------
// As in the forward sweep: once the cell-centric kernel's CTA-sized cells are
// all taken, its warps take the tiny cells one per warp (lane l: particle ca +
// l), stage the 27 windows of the widened plan with each neighbour's records
// shifted into a's frame, and run one adjoint sweep over them; each lane keeps
// its five sums in registers and writes its outputs.
constexpr int kTinyBufB = 128;  // staged candidates per warp and pass
constexpr int kTinyWarpBytesB =
    (kTinyBufB + kPad) * (16 + 16 + 4) + (int)((sizeof(TinySlots) + 15) / 16 * 16);

__device__ __forceinline__ void tiny_phase_bwd(const GridDev& g, unsigned char* buf, int lane,
                                               const float* __restrict__ g_rho,
                                               const float* __restrict__ g_D,
                                               float* __restrict__ g_pos,
                                               float* __restrict__ g_h) {
  float4* Sx = reinterpret_cast<float4*>(buf);
  float4* Sa = Sx + kTinyBufB + kPad;
  int* Sj = reinterpret_cast<int*>(Sa + kTinyBufB + kPad);
  TinySlots& ts = *reinterpret_cast<TinySlots*>(Sj + kTinyBufB + kPad);
  const Slot self = slot_info(kSelfSlot);
  const float munit = (float)(16.0 / 3.14159265358979323846);
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
    LaneB L;
    laneb_init(L);
    if (lane < na) laneb_set(L, g, B, self, ca + lane);
    int q = 0;  // slot of this lane's next staged candidate (non-decreasing)
    for (int f0 = 0; f0 < total; f0 += kTinyBufB) {
      const int len = min(kTinyBufB, total - f0);
      for (int e = lane; e < len; e += 32) {
        const int f = f0 + e;
        while (ts.off[q + 1] <= f) q++;
        float sx, sy, sz;
        const int sj = tiny_candidate(g, ts, q, f, edge, sx, sy, sz);
        const float4 xe = g.bx[sj];  // negated offsets
        Sx[e] = make_float4(xe.x - sx, xe.y - sy, xe.z - sz, xe.w);
        Sa[e] = g.ba[sj];
        Sj[e] = sj;
      }
      __syncwarp();
      auto jidx = [&](int j) { return Sj[j]; };
      sweep_bwd(L, smem_addr_b(Sx), smem_addr_b(Sa), 0, len, g, B, jidx, ChunkSkip{});
      __syncwarp();  // the buffers are rewritten next
    }
    laneb_fold(L);
    if (lane < na)
      write_bwd(g, ca + lane, (double)L.Sth, (double)L.Suh, (double)L.gx, (double)L.gy,
                (double)L.gz, g_rho, g_D, g_pos, g_h, munit * g.m_max[g.cell_box[a]]);
  }
}

struct CellSharedB {
  int I[kNSlot], J0[kNSlot];
  int off[kNSlot + 1];
  int runs[kNSlot + 1];
  int nb_[kNSlot], cb_[kNSlot];
  float offv[kNSlot], Hmaxb[kNSlot];
  float cmx[kNSlot];  // the neighbour cells' bounds of the adjoint terms
  float bn;           // their largest: the unit of the cell's gradient sums
  int cell, item_next;
};

constexpr int kCellWarps = kCellThreads / 32;
static_assert(kCellWarps * kTinyWarpBytesB <= kCellSmemFor[3],
              "the tiny-cell buffers fit the smallest dynamic shared memory");

// projection of a staged record (negated offsets) in the frame of slot (k, s):
// the same FP32 expression the sort used for `dist`
__device__ __forceinline__ float sproj(float4 x, float ux, float uy, float uz, int s, float off) {
  return s * fmaf(-x.x, ux, fmaf(-x.y, uy, -x.z * uz)) + off;
}

__global__ void __launch_bounds__(kCellThreads, 3) k_backward_cells(
    GridDev g, const float* __restrict__ g_rho, const float* __restrict__ g_D,
    float* __restrict__ g_pos, float* __restrict__ g_h) {
  pdl_enter();
  extern __shared__ float4 dsm[];
  __shared__ CellSharedB cs;
  if (*g.flags) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncells = *g.n_ccells;
  const float munit = (float)(16.0 / 3.14159265358979323846);
  float4* var = dsm;
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
      const int o = c_border[tid];
      const int4 p = pl[o];
      cs.I[tid] = p.x;
      cs.J0[tid] = p.y;
      cs.off[tid + 1] = p.z - p.y;
      cs.runs[tid + 1] = (p.x + 31) >> 5;
      const int b = neighbour_cell(g, a, o);
      cs.nb_[tid] = g.cell_count[b];
      cs.cb_[tid] = g.cell_start[b];
      cs.Hmaxb[tid] = g.cell_Hmax[b];
      cs.cmx[tid] = g.bwd_cmax[b];
      const Slot sl = slot_info(o);
      cs.offv[tid] = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    }
    if (tid == 0) {
      cs.off[0] = 0;
      cs.runs[0] = 0;
      cs.item_next = 0;
    }
    __syncthreads();
    if (tid == 0) {
      float bn = 0.0f;
      for (int q = 0; q < kNSlot; q++) {
        cs.off[q + 1] += cs.off[q];
        cs.runs[q + 1] += cs.runs[q];
        bn = fmaxf(bn, cs.cmx[q]);
      }
      cs.bn = bn;
    }
    __syncthreads();
    const int total = cs.off[kNSlot];
    // variable carve: kElemJ (total + kPad) + kElemA na bytes, checked by the plan
    float4* Sx = var;                                  // [total + kPad] {x, y, z, E}
    float4* Sa = Sx + total + kPad;                    // [total + kPad] {m, G', K, H}
    // fixed-point sums: gx, gy, gz (64-bit), th, uh (32-bit)
    long long* accg = reinterpret_cast<long long*>(Sa + total + kPad);  // [3][na]
    int* accs = reinterpret_cast<int*>(accg + 3 * na);                  // [2][na]
    const float ks = fix_scale_s32(total);
    const float kg = fix_scale_g64(cs.bn, (float)(total + 1));
    stage_flat<8>(  // eight index lookups in flight per thread (latency-bound)
        cs.off, total, tid, kCellThreads,
        [&](int f, int q) {
          const Slot sl = slot_info(c_border[q]);
          const int cb = cs.cb_[q];
          const int pos = order_pos(sl.s, cs.J0[q] + f - cs.off[q], cs.nb_[q]);
          return cb + (int)g.perm[(size_t)sl.k * g.n + cb + pos];
        },
        [](int sj) { return sj; },
        [&](int f, int, int sj) {  // cp.async: both records straight to shared memory
          cp_async16(&Sx[f], &g.bx[sj]);
          cp_async16(&Sa[f], &g.ba[sj]);
        });
    for (int t = tid; t < 3 * na; t += kCellThreads) accg[t] = 0;
    for (int t = tid; t < 2 * na; t += kCellThreads) accs[t] = 0;
    cp_async_wait_all();
    __syncthreads();
    const int nitems = cs.runs[kNSlot];
    for (;;) {
      int it = 0;
      if (lane == 0) it = atomicAdd(&cs.item_next, 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      if (it >= nitems) break;
      const int q = warp_seg_of(cs.runs, kNSlot, it, lane);
      const int o = c_border[q];
      const Slot sl = slot_info(o);
      float ux, uy, uz;
      axis_u(sl.k, ux, uy, uz);
      const int p = ((it - cs.runs[q]) << 5) + lane;
      const bool valid = p < cs.I[q];
      LaneB L;
      laneb_init(L);
      float d_lo = 3.0e38f, d_hi = -3.0e38f;
      int il = 0;
      const float Hmb = cs.Hmaxb[q];
      if (valid) {
        const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
        const size_t kb = (size_t)sl.k * g.n + ca + pos_i;
        il = g.perm[kb];
        laneb_set(L, g, B, sl, ca + il);
        const float di = sl.s * g.dist[kb];
        const float reach = fmaxf(L.H, Hmb) + padw;
        d_lo = di - reach;
        d_hi = di + reach;
      }
      const float w_lo = warp_min_b(d_lo), w_hi = warp_max_b(d_hi);
      const int s0 = cs.off[q], len = cs.off[q + 1] - s0;
      const float offv = cs.offv[q];
      const int J0q = cs.J0[q], nbq = cs.nb_[q], cbq = cs.cb_[q];
      // after pv_update_positions the staged positions are no longer in sorted
      // order: the window searches then read the sort's projections
      auto proj = [&](int e) {  // projection of staged element e, as sorted
        return g.moved ? proj_asc(g, sl.k, sl.s, cbq, nbq, J0q + e, offv)
                       : sproj(Sx[s0 + e], ux, uy, uz, sl.s, offv);
      };
      const int lo = s0 + ((o == kSelfSlot)
                               ? warp_first_true(len, lane, [&](int e) { return proj(e) > w_lo; })
                               : 0);
      const int hi = s0 + warp_first_true(len, lane, [&](int e) { return proj(e) >= w_hi; });
      const size_t kbq = (size_t)sl.k * g.n + cbq;
      auto jidx = [&](int j) {
        return cbq + (int)g.perm[kbq + order_pos(sl.s, J0q + j - s0, nbq)];
      };
      sweep_bwd(L, smem_addr_b(Sx), smem_addr_b(Sa), lo, hi, g, B, jidx, ChunkSkip{});
      // lanes whose windows held no pair in range have nothing to add
      laneb_fold(L);
      if (valid && (L.Sth != 0.0f || L.Suh != 0.0f || L.gx != 0.0f || L.gy != 0.0f ||
                    L.gz != 0.0f)) {
        atomicAdd(&accs[il], __float2int_rn(L.Sth * ks));
        atomicAdd(&accs[na + il], __float2int_rn(L.Suh * ks));
        atomicAdd(reinterpret_cast<unsigned long long*>(&accg[il]),
                  (unsigned long long)__float2ll_rn(L.gx * kg));
        atomicAdd(reinterpret_cast<unsigned long long*>(&accg[na + il]),
                  (unsigned long long)__float2ll_rn(L.gy * kg));
        atomicAdd(reinterpret_cast<unsigned long long*>(&accg[2 * na + il]),
                  (unsigned long long)__float2ll_rn(L.gz * kg));
      }
    }
    __syncthreads();
    const double is = 1.0 / (double)ks, ig = 1.0 / (double)kg;
    for (int t = tid; t < na; t += kCellThreads)
      write_bwd(g, ca + t, accs[t] * is, accs[na + t] * is, accg[t] * ig, accg[na + t] * ig,
                accg[2 * na + t] * ig, g_rho, g_D, g_pos, g_h, mscale);
    __syncthreads();
  }
  // then the tiny cells, one per warp, in the dynamic shared memory that the
  // cells no longer use (at least kCellWarps * kTinyWarpBytesB of it)
  tiny_phase_bwd(g, reinterpret_cast<unsigned char*>(var) + warp * kTinyWarpBytesB, lane,
                 g_rho, g_D, g_pos, g_h);
}

// ---- task kernel (cells too dense for the cell-centric kernel) ----------------------

// BlkI particles (and threads) per task, as g.task_blk (the plan's).
template <int BlkI>
__global__ void __launch_bounds__(BlkI, 896 / BlkI) k_backward_tasks(GridDev g) {
  pdl_enter();
  __shared__ float4 s_x[kTileJ + kPad];
  __shared__ float4 s_a[kTileJ + kPad];
  __shared__ float s_d[kTileJ];
  __shared__ int s_j[kTileJ + kPad];
  __shared__ float4 s_bs[kTileJ / 32];  // chunk summaries of the tile
  __shared__ int s_task;
  if (*g.flags) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntask = *g.ntask;
  if (ntask == 0) return;  // no task cells: leave without touching the task counter
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(g.task_next, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= ntask) break;
    const TaskB tk = decode_b(g.tasks[t]);
    const int a = tk.a, o = tk.o;
    const int b = neighbour_cell(g, a, o);
    const int na = g.cell_count[a], nb = g.cell_count[b];
    const int ca = g.cell_start[a], cb = g.cell_start[b];
    const BoxDev B = g.boxes[g.cell_box[a]];
    const Slot sl = slot_info(o);
    const float off = sl.v2 ? vnorm(sl.v2) * B.edge_f : 0.0f;
    const size_t kbase = (size_t)sl.k * g.n;
    const float Hmax_b = g.cell_Hmax[b];
    const int p = tk.p0 + warp * 32 + lane;
    const bool valid = p < tk.p1;
    LaneB L;
    laneb_init(L);
    const float padw = window_pad(g, B, g.cell_box[a]);
    float d_lo = 3.0e38f, d_hi = -3.0e38f, di = 0.0f;
    if (valid) {
      const int pos_i = (o == kSelfSlot) ? p : order_pos(sl.s, na - 1 - p, na);
      const int si = ca + g.perm[kbase + ca + pos_i];
      laneb_set(L, g, B, sl, si);
      di = sl.s * g.dist[kbase + ca + pos_i];
      const float reach = fmaxf(L.H, Hmax_b) + padw;
      d_lo = di - reach;
      d_hi = di + reach;
    }
    const float w_lo = warp_min_b(d_lo), w_hi = warp_max_b(d_hi);
    // whether some warp of the task may skip chunks (the same on every thread)
    const bool skip_task = Hmax_b > kSkipRatio * g.bwd_hmin[a];
    for (int j0 = tk.j0; j0 < tk.j1; j0 += kTileJ) {
      const int len = min(kTileJ, tk.j1 - j0);
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int pos_j = order_pos(sl.s, j0 + e, nb);
        const int sj = cb + g.perm[kbase + cb + pos_j];
        s_x[e] = g.bx[sj];
        s_a[e] = g.ba[sj];
        s_d[e] = sl.s * g.dist[kbase + cb + pos_j] + off;
        s_j[e] = sj;
      }
      __syncthreads();
      // the tile's chunk summaries (blocks of 32 from the tile start; the
      // projections are the sort's, as the lanes' d_i)
      for (int bi = warp; skip_task && bi < ((len + 31) >> 5); bi += BlkI / 32) {
        const int e = (bi << 5) + lane;
        float dmn = 3.0e38f, dmx = -3.0e38f, lmn = 3.0e38f, rmx = -3.0e38f;
        if (e < len) {
          const float d = s_d[e], r = s_a[e].w + padw;
          dmn = dmx = d;
          lmn = d - r;
          rmx = d + r;
        }
        dmn = warp_min_b(dmn);
        dmx = warp_max_b(dmx);
        lmn = warp_min_b(lmn);
        rmx = warp_max_b(rmx);
        if (lane == 0) s_bs[bi] = make_float4(dmn, dmx, lmn, rmx);
      }
      if (skip_task) __syncthreads();
      if (w_hi > w_lo) {
        const int lo = (o == kSelfSlot) ? upper_bound_f(s_d, len, w_lo) : 0;
        const int hi = lower_bound_f(s_d, len, w_hi);
        auto jidx = [&](int j) { return s_j[j]; };
        ChunkSkip sk{};
        if (skip_task && hi - lo >= kSkipMinLen)
          sk = chunk_skip(smem_addr_b(s_bs), 0, valid, di, L.H, padw);
        sweep_bwd(L, smem_addr_b(s_x), smem_addr_b(s_a), lo, hi, g, B, jidx, sk);
      }
      __syncthreads();
    }
    laneb_fold(L);
    const float bn = nbhd_bound(g, a, lane);
    if (valid && (L.Sth != 0.0f || L.Suh != 0.0f || L.gx != 0.0f || L.gy != 0.0f ||
                  L.gz != 0.0f)) {
      // 64-bit fixed point: the sum does not depend on the order of the tasks
      unsigned long long* acc = reinterpret_cast<unsigned long long*>(g.gacc);
      const size_t N = (size_t)g.n;
      const float ks = (float)kFixS64;
      const float kg = fix_scale_g64(bn, kTaskPairs);
      atomicAdd(&acc[L.si], (unsigned long long)__float2ll_rn(L.Sth * ks));
      atomicAdd(&acc[N + L.si], (unsigned long long)__float2ll_rn(L.Suh * ks));
      atomicAdd(&acc[2 * N + L.si], (unsigned long long)__float2ll_rn(L.gx * kg));
      atomicAdd(&acc[3 * N + L.si], (unsigned long long)__float2ll_rn(L.gy * kg));
      atomicAdd(&acc[4 * N + L.si], (unsigned long long)__float2ll_rn(L.gz * kg));
    }
  }
}

constexpr int kFinBatchB = 4;  // particles per thread in flight in the task-path finalize
__global__ void k_bwd_finalize_t(GridDev g, const float* __restrict__ g_rho,
                                 const float* __restrict__ g_D, float* __restrict__ g_pos,
                                 float* __restrict__ g_h) {
  pdl_enter();
  if (*g.flags) return;
  const float munit = (float)(16.0 / 3.14159265358979323846);
  long long* acc = g.gacc;
  const size_t N = (size_t)g.n;
  const int lane = threadIdx.x & 31;
  // units as in k_backward_tasks (the float rounding of the scale is the same)
  // The slots ca + t0 + k stride (k < kFinBatchB, below t1) of one thread:
  // every load first, so that the batch's random accesses are in flight
  // together, then the outputs, then the clears.
  auto fin = [&](int ca, int t0, int stride, int t1, float ig, float mscale) {
    const double is = 1.0 / (double)(float)kFixS64;
    long long v[kFinBatchB][5];
#pragma unroll
    for (int k = 0; k < kFinBatchB; k++) {
      const int t = t0 + k * stride;
      if (t < t1) {
        const size_t s = (size_t)ca + t;
#pragma unroll
        for (int q = 0; q < 5; q++) v[k][q] = acc[q * N + s];
      }
    }
#pragma unroll
    for (int k = 0; k < kFinBatchB; k++) {
      const int t = t0 + k * stride;
      if (t < t1)
        write_bwd(g, ca + t, v[k][0] * is, v[k][1] * is, v[k][2] * ig, v[k][3] * ig,
                  v[k][4] * ig, g_rho, g_D, g_pos, g_h, mscale);
    }
#pragma unroll
    for (int k = 0; k < kFinBatchB; k++) {
      const int t = t0 + k * stride;
      if (t < t1) {
        const size_t s = (size_t)ca + t;
#pragma unroll
        for (int q = 0; q < 5; q++) acc[q * N + s] = 0;
      }
    }
  };
  // as the forward finalize: one warp per self-slot task (blocks of g.task_blk
  // cell-local indices), or one block per task cell when the self slot is
  // masked out
  if ((g.slot_mask >> kSelfSlot) & 1u) {
    const int ntask = *g.ntask;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ntask;
         w += (gridDim.x * blockDim.x) >> 5) {
      const TaskB tk = decode_b(g.tasks[w]);
      if (tk.o != kSelfSlot) continue;
      const int ca = g.cell_start[tk.a];
      const float mscale = munit * g.m_max[g.cell_box[tk.a]];
      const float ig = 1.0f / fix_scale_g64(nbhd_bound(g, tk.a, lane), kTaskPairs);
      for (int t0 = tk.p0 + lane; t0 < tk.p1; t0 += 32 * kFinBatchB)
        fin(ca, t0, 32, tk.p1, ig, mscale);
    }
  } else {
    const int nt = *g.n_tcells;
    for (int c = blockIdx.x; c < nt; c += gridDim.x) {
      const int a = g.tcells[c];
      const int ca = g.cell_start[a], na = g.cell_count[a];
      const float mscale = munit * g.m_max[g.cell_box[a]];
      const float ig = 1.0f / fix_scale_g64(nbhd_bound(g, a, lane), kTaskPairs);
      for (int t0 = threadIdx.x; t0 < na; t0 += blockDim.x * kFinBatchB)
        fin(ca, t0, blockDim.x, na, ig, mscale);
    }
  }
}

}  // namespace

cudaError_t launch_backward(const GridDev& g, const float* g_rho, const float* g_drho_dh,
                            float* g_pos, float* g_h, int num_sms, int ctas_per_sm,
                            cudaStream_t st, cudaEvent_t t0, cudaEvent_t t1) {
  if (g.n == 0) return cudaSuccess;
  if (ctas_per_sm < 1 || ctas_per_sm > 3) return cudaErrorInvalidValue;
  cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(&k_backward_cells),
                                       kCellSmemFor[1], st);
  if (e != cudaSuccess) return e;
  const int smem = kCellSmemFor[ctas_per_sm];
  const int nb = (g.n + 255) / 256;
  // the plan (which also clears bwd_cmax) needs nothing of k_bwd_prep's
  if ((e = launch_plan(g, 1, smem, kElemJ, kElemA, 0, st)) != cudaSuccess) return e;
  PV_LAUNCH(k_bwd_prep, nb, 256, 0, st, g, g_rho, g_drho_dh);
  if (t0 && (e = cudaEventRecord(t0, st)) != cudaSuccess) return e;
  PV_LAUNCH(k_backward_cells, num_sms * ctas_per_sm, kCellThreads, smem, st,
            g, g_rho, g_drho_dh, g_pos, g_h);
  if (t1 && (e = cudaEventRecord(t1, st)) != cudaSuccess) return e;
  // (a plain launch: as a dependent of the persistent cell kernel, the task
  // kernel made the 4M clustered step 0.6 ms slower)
  switch (g.task_blk) {
    case 64: PV_LAUNCH_PLAIN(k_backward_tasks<64>, num_sms * 16, 64, 0, st, g); break;
    case 256: PV_LAUNCH_PLAIN(k_backward_tasks<256>, num_sms * 4, 256, 0, st, g); break;
    default: PV_LAUNCH_PLAIN(k_backward_tasks<128>, num_sms * 8, 128, 0, st, g); break;
  }
  PV_LAUNCH(k_bwd_finalize_t, num_sms * 8, 256, 0, st, g, g_rho, g_drho_dh, g_pos,
            g_h);
  return cudaSuccess;
}

}  // namespace pv
