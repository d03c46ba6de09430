// pv_grid.cu -- cell grid and the 13 sorted projections per cell.
//
// Section 2 of the paper: the domain is split into cells of edge C_l >= the
// largest interaction radius and the particles of a cell are stored
// together; for each of the 13 axes joining a cell centre to its neighbours'
// centres the particles are sorted by their projection on the axis ("dist"
// and "index" arrays).  Section 3.2: positions are shifted to a cell-local
// frame in double precision and only then converted to single precision.
//
// Kernels (all HBM-bound except the sort, which is shared-memory bound):
//   k_clear    zeroes the occupancies and the per-sort scalars
//   k_bin      particle -> cell id, occupancy histogram, box m_max, input
//              checks (latched flags)
//   k_scan     exclusive scan of the occupancies, list of big cells
//   k_scatter  caller index of every cell-order slot
//   k_cell_sort   one CTA per cell of more than 64 particles: gathers the
//              cell's particles into cell order (FP32 offsets + normalised
//              mass, h, wrapped FP64 position) with coalesced writes, the
//              cell's H_max, and, for a cell of <= 384 particles, the 13
//              sorts, one warp per axis: bucket (counting) sort in shared
//              memory, exact order inside a bucket by (projection, caller
//              index)
//   k_cell_sort_tiny  the same for cells of <= 64 particles, one warp per
//              cell (the 13 axes in turn)
//   k_sort_big    one CTA per (larger cell, axis), the same algorithm with up
//              to 8192 buckets in shared memory
//   k_update, k_update_check  new positions on a kept sort (pv_update_positions)
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {

namespace {

// cells of up to kSortTinyMax particles are gathered and sorted by one warp
// (all 13 axes in turn), cells of up to kSortSmallMax particles by one CTA
// (74 KB of shared memory, three CTAs per SM, one warp per axis); larger
// ones are gathered by that CTA and sorted with one CTA per (cell, axis)
constexpr int kSortTinyMax = 64;
constexpr int kSortTinyWarps = 8;
constexpr int kSortSmallMax = 384;
static_assert(kSortSmallMax % 32 == 0, "whole particles per lane in the cell sort");
constexpr int kSortThreads = kNDir * 32;

__device__ __forceinline__ bool valid_h_m(float hv, float mv) {
  return hv > 0.0f && isfinite(hv) && mv >= 0.0f && isfinite(mv);
}

// isfinite(x) and 0 <= x < L (L > 0) on the FP64 bit patterns, in integer
// arithmetic: sm_103 has few FP64 units.  Non-negative doubles order as their
// bit patterns; -0.0 passes, as in the FP64 comparison.
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}
__device__ __forceinline__ bool in_box_bits(double x, double L) {
  const long long b = __double_as_longlong(x);
  return (b >= 0 && b < __double_as_longlong(L)) || b == (long long)0x8000000000000000ULL;
}

__device__ __forceinline__ double wrap_coord(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y = 0.0;
  if (y < 0.0) y = 0.0;
  return y;
}

__global__ void k_clear(GridDev g) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < g.ncell) g.cell_count[i] = 0;
  if (i < g.n_boxes) {
    g.m_max[i] = 0.0f;
    g.box_disp[i] = 0.0f;
  }
  if (i == 0) {
    *g.flags = 0u;
    *g.max_count = 0;
    *g.n_big = 0;
  }
}

__global__ void k_bin(GridDev g, const double* __restrict__ pos, const float* __restrict__ h,
                      const float* __restrict__ m, float m_uniform) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  float mw = 0.0f;
  int bx = -1;
  if (p < g.n) {
    bx = box_of_particle(g, p);
    const BoxDev B = g.boxes[bx];
    uint32_t flags = 0;
    int c3[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double x = pos[3 * (size_t)p + c];
      if (!finite_bits(x)) { flags |= PV_FLAG_BAD_POSITION; x = 0.0; }
      if (!in_box_bits(x, B.L)) x = wrap_coord(x, B.L);  // FP64 division only when needed
      const int ci = (int)(x * B.inv_edge);
      c3[c] = ci < 0 ? 0 : (ci >= B.nc ? B.nc - 1 : ci);
    }
    const int cell = B.cell_base + (c3[0] * B.nc + c3[1]) * B.nc + c3[2];
    const float hv = h[p];
    const float mv = m ? m[p] : m_uniform;
    if (!valid_h_m(hv, mv)) flags |= PV_FLAG_BAD_SMOOTHING;
    else if (hv > B.h_limit) flags |= PV_FLAG_SUPPORT_EXCEEDS_CELL;  // gamma h > edge
    if (flags) atomicOr(g.flags, flags);
    g.pcell[p] = cell;
    g.prank[p] = atomicAdd(&g.cell_count[cell], 1);
    mw = (mv > 0.0f && isfinite(mv)) ? mv : 0.0f;
  }
  // m_max of a box is one address for all its particles: reduce over the
  // warp first when the warp lies in one box (the common case)
  const int b0 = __shfl_sync(0xffffffffu, bx, 0);
  if (__all_sync(0xffffffffu, bx == b0 || bx < 0)) {
    for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
    if ((threadIdx.x & 31) == 0 && mw > 0.0f && b0 >= 0) atomic_max_nonneg(&g.m_max[b0], mw);
  } else if (bx >= 0 && mw > 0.0f) {
    atomic_max_nonneg(&g.m_max[bx], mw);
  }
}

// Single-CTA exclusive scan of the cell occupancies (C is at most a few
// million; each thread scans a contiguous chunk).
__global__ void __launch_bounds__(1024) k_scan(GridDev g) {
  pdl_enter();
  __shared__ int s_part[1024];
  __shared__ int s_max[32];
  const int C = g.ncell, T = blockDim.x, t = threadIdx.x;
  const int per = (C + T - 1) / T;
  const int c0 = min(C, t * per), c1 = min(C, c0 + per);
  int sum = 0, mx = 0;
  for (int c = c0; c < c1; c++) {
    int v = g.cell_count[c];
    sum += v;
    mx = max(mx, v);
  }
  s_part[t] = sum;
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) s_max[t >> 5] = mx;
  __syncthreads();
  // Hillis-Steele inclusive scan of the chunk sums
  for (int o = 1; o < T; o <<= 1) {
    int v = t >= o ? s_part[t - o] : 0;
    __syncthreads();
    s_part[t] += v;
    __syncthreads();
  }
  int run = s_part[t] - sum;
  for (int c = c0; c < c1; c++) {
    int v = g.cell_count[c];
    g.cell_start[c] = run;
    run += v;
    if (v > kSortSmallMax) g.big_cells[atomicAdd(g.n_big, 1)] = c;
  }
  if (t == T - 1) g.cell_start[C] = s_part[T - 1];
  if (t == 0) {
    int m = 0;
    for (int w = 0; w < T / 32; w++) m = max(m, s_max[w]);
    *g.max_count = m;
    if (m > PV_MAX_CELL_COUNT) atomicOr(g.flags, PV_FLAG_CELL_OVERFLOW);
  }
}

__global__ void k_scatter(GridDev g) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < g.n) g.orig[g.cell_start[g.pcell[p]] + g.prank[p]] = p;
}

// New positions and smoothing lengths for the sorted grid (pv_update_positions):
// particle p keeps its cell and slot; its offset is taken from that cell's
// centre (nearest periodic image), and its displacement from the offset at the
// sort raises the box's largest displacement.
__global__ void k_update(GridDev g, const double* __restrict__ pos,
                         const float* __restrict__ h) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  float disp = 0.0f;
  int bx = -1;
  if (p < g.n) {
    const int cell = g.pcell[p];
    bx = g.cell_box[cell];
    const BoxDev B = g.boxes[bx];
    const int s = g.cell_start[cell] + g.prank[p];
    const int loc = cell - B.cell_base;
    const int c3[3] = {loc / (B.nc * B.nc), (loc / B.nc) % B.nc, loc % B.nc};
    uint32_t flags = 0;
    float off[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double x = pos[3 * (size_t)p + c];
      if (!finite_bits(x)) { flags |= PV_FLAG_BAD_POSITION; x = 0.0; }
      if (!in_box_bits(x, B.L)) x = wrap_coord(x, B.L);
      double d = fma(-(c3[c] + 0.5), B.edge, x);  // as at the sort for an unmoved particle
      d -= B.L * rint(d * B.inv_L);               // nearest image of the cell centre
      off[c] = (float)d;
      g.pos64[3 * (size_t)s + c] = x;
    }
    float hv = h[p];
    if (!(hv > 0.0f) || !isfinite(hv)) {
      flags |= PV_FLAG_BAD_SMOOTHING;
      hv = 0.0f;
    }
    const float4 r = g.xm_ref[s];
    const float dx = off[0] - r.x, dy = off[1] - r.y, dz = off[2] - r.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    // FP32 rounding of the norm and of the offsets: a relative and an
    // absolute margin keep disp above the exact displacement
    disp = d2 > 0.0f ? fmaf(sqrtf(d2), 1.0f + 1e-6f, ldexpf(B.edge_f, -20)) : 0.0f;
    g.xm[s] = make_float4(off[0], off[1], off[2], r.w);
    g.hs[s] = hv;
    atomic_max_nonneg(&g.cell_Hmax[cell], g.gamma * hv);
    if (flags) atomicOr(g.flags, flags);
  }
  const int b0 = __shfl_sync(0xffffffffu, bx, 0);
  if (__all_sync(0xffffffffu, bx == b0 || bx < 0)) {
    for (int o = 16; o > 0; o >>= 1) disp = fmaxf(disp, __shfl_xor_sync(0xffffffffu, disp, o));
    if ((threadIdx.x & 31) == 0 && disp > 0.0f && b0 >= 0) atomic_max_nonneg(&g.box_disp[b0], disp);
  } else if (bx >= 0 && disp > 0.0f) {
    atomic_max_nonneg(&g.box_disp[bx], disp);
  }
}

// Every cell must keep H_max + 2 delta within its edge (delta: the box's
// largest displacement since the sort), else the 27-cell stencil of the last
// sort no longer holds all pairs in range.
__global__ void k_update_check(GridDev g) {
  pdl_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell || g.cell_count[c] == 0) return;
  const int bx = g.cell_box[c];
  const BoxDev& B = g.boxes[bx];
  if (g.cell_Hmax[c] + window_pad(g, B, bx) > B.edge_f) atomicOr(g.flags, PV_FLAG_SKIN_EXCEEDED);
}

__device__ __forceinline__ bool key_less(float ka, int oa, float kb, int ob) {
  return ka < kb || (ka == kb && oa < ob);
}

// Exclusive prefix of v over the group (a warp, or the whole block when
// kBlock; `scratch` holds one int per warp of the block).
template <bool kBlock>
__device__ __forceinline__ int group_exclusive_scan(int v, int rank, int* scratch) {
  const int lane = rank & 31;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (!kBlock) return x - v;
  const int warp = rank >> 5, nw = (int)(blockDim.x >> 5);
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = lane < nw ? scratch[lane] : 0;
    const int t0 = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) scratch[lane] = t - t0;
  }
  __syncthreads();
  const int r = x - v + scratch[warp];
  __syncthreads();
  return r;
}

// Bucket b of a scan in which each of nthr threads owns per = nb / nthr
// consecutive buckets sits at b + b / per (sh = log2 per): one pad word per
// chunk puts the chunks' i-th buckets in distinct shared-memory banks.
__device__ __forceinline__ int bucket_slot(int b, int sh) { return b + (b >> sh); }

// Sorts the cnt <= 32 kPer particles of one cell along one axis with one
// warp.  Lane l holds in kr[j] the key of the particle t = l + 32 j (for
// t < cnt); the shared arrays are key[cnt] (the same keys, read by the other
// lanes), orig[cnt] (caller indices, the tie break), tmp[cnt], out[cnt]
// (cell-local indices) and bucket[nb + 32] (nb a power of two, 32 <= nb;
// bucket b at bucket_slot(b, log2(nb / 32))).
// Buckets are monotone in the key: a counting sort by bucket leaves only the
// order inside each bucket, which every particle then settles by counting the
// members of its bucket that precede it in (key, caller index) order.  The
// per-lane particles are unrolled, so that their shared-memory accesses and
// atomics are in flight together.
template <int kPer>
__device__ __forceinline__ void warp_sort_axis(int cnt, const float (&kr)[kPer],
                                               const float* key, const int* orig,
                                               uint16_t* tmp, uint16_t* out, int* bucket,
                                               int nb, int lane, float kmin, float kmax) {
  const float scale = kmax > kmin ? (float)nb / (kmax - kmin) : 0.0f;
  int bk[kPer];
#pragma unroll
  for (int j = 0; j < kPer; j++)
    bk[j] = lane + 32 * j < cnt ? min(nb - 1, max(0, (int)((kr[j] - kmin) * scale))) : -1;
  const int per = nb >> 5, sh = __ffs(per) - 1;
  for (int b = lane; b < nb + 32; b += 32) bucket[b] = 0;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < kPer; j++)
    if (bk[j] >= 0) atomicAdd(&bucket[bucket_slot(bk[j], sh)], 1);
  __syncwarp();
  // exclusive scan: each lane owns nb / 32 consecutive buckets
  const int p0 = bucket_slot(lane * per, sh);
  int sum = 0;
  for (int b = p0; b < p0 + per; b++) sum += bucket[b];
  int run = group_exclusive_scan<false>(sum, lane, nullptr);
  for (int b = p0; b < p0 + per; b++) {
    const int v = bucket[b];
    bucket[b] = run;
    run += v;
  }
  __syncwarp();
  int at[kPer];
#pragma unroll
  for (int j = 0; j < kPer; j++)
    at[j] = bk[j] >= 0 ? atomicAdd(&bucket[bucket_slot(bk[j], sh)], 1) : 0;
#pragma unroll
  for (int j = 0; j < kPer; j++)
    if (bk[j] >= 0) tmp[at[j]] = (uint16_t)(lane + 32 * j);
  __syncwarp();
  // bucket[b] is now the end of bucket b (= the start of bucket b+1); a
  // particle alone in its bucket is already in place
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    if (bk[j] < 0) continue;
    const int t = lane + 32 * j;
    const int s0 = bk[j] ? bucket[bucket_slot(bk[j] - 1, sh)] : 0;
    const int s1 = bucket[bucket_slot(bk[j], sh)];
    int r = 0;
    if (s1 - s0 > 1) {
      const int ot = orig[t];
      for (int u = s0; u < s1; u++) {
        const int v = tmp[u];
        r += key_less(key[v], orig[v], kr[j], ot) ? 1 : 0;
      }
    }
    out[s0 + r] = (uint16_t)t;
  }
  __syncwarp();
}

// Shared memory of k_cell_sort<kMax>: staged particles, keys, buckets (a
// power of two >= kMax), and the 16-bit index arrays of the 13 axes.
template <int kMax>
__host__ __device__ constexpr int sort_small_buckets() {
  return kMax <= 32 ? 32 : 2 * sort_small_buckets<(kMax + 1) / 2>();
}
template <int kMax>
constexpr size_t sort_small_smem() {
  return (size_t)kMax * (sizeof(float4) + sizeof(int)) +
         (size_t)kNDir * (kMax * (sizeof(float) + 2 * sizeof(uint16_t)) +
                          (sort_small_buckets<kMax>() + 32) * sizeof(int));
}

// One CTA per cell.  All threads gather the cell's particles (caller indices
// in orig) into cell order with coalesced writes: FP32 offsets from the cell
// centre (Section 3.2: shifted in FP64, then rounded) with the normalised
// mass, h, the copy kept for pv_update_positions and the wrapped FP64
// position; the cell's H_max is reduced on the way.  A cell of at most kMax
// particles is then sorted along the 13 axes from the staged copy, one warp
// per axis; larger cells are left to k_sort_big.
template <int kMax>
__global__ void __launch_bounds__(kSortThreads, 3) k_cell_sort(GridDev g,
                                                            const double* __restrict__ pos,
                                                            const float* __restrict__ h,
                                                            const float* __restrict__ m,
                                                            float m_uniform) {
  pdl_enter();
  constexpr int kB = sort_small_buckets<kMax>();
  extern __shared__ float4 smem4[];
  __shared__ unsigned int s_hmax;
  float4* s_x = smem4;                                           // [kMax]
  int* s_orig = reinterpret_cast<int*>(s_x + kMax);              // [kMax]
  float* s_key = reinterpret_cast<float*>(s_orig + kMax);        // [13][kMax]
  int* s_bkt = reinterpret_cast<int*>(s_key + kNDir * kMax);     // [13][kB + 32]
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_bkt + kNDir * (kB + 32));  // [13][kMax]
  uint16_t* s_tmp = s_out + kNDir * kMax;                        // [13][kMax]
  const int c = blockIdx.x;
  const int cnt = g.cell_count[c];
  if (cnt <= kSortTinyMax) return;  // k_cell_sort_tiny's
  const int cs = g.cell_start[c];
  const int bx = g.cell_box[c];
  const BoxDev B = g.boxes[bx];
  const int loc = c - B.cell_base;
  const double ctr[3] = {-((loc / (B.nc * B.nc)) + 0.5), -(((loc / B.nc) % B.nc) + 0.5),
                         -((loc % B.nc) + 0.5)};
  const float mmax = g.m_max[bx];
  if (threadIdx.x == 0) s_hmax = 0u;
  __syncthreads();
  float hmax = 0.0f;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int p = g.orig[cs + t];
    const size_t s = (size_t)cs + t;
    float off[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      double x = pos[3 * (size_t)p + k];
      if (!finite_bits(x)) x = 0.0;
      if (!in_box_bits(x, B.L)) x = wrap_coord(x, B.L);
      off[k] = (float)fma(ctr[k], B.edge, x);
      g.pos64[3 * s + k] = x;
    }
    const float mv = m ? m[p] : m_uniform;
    const float hv = h[p];
    const float4 xm = make_float4(off[0], off[1], off[2], mmax > 0.0f ? mv / mmax : 0.0f);
    g.xm[s] = xm;
    g.xm_ref[s] = xm;
    g.hs[s] = hv;
    if (valid_h_m(hv, mv)) hmax = fmaxf(hmax, g.gamma * hv);
    if (cnt <= kMax) {
      s_x[t] = xm;
      s_orig[t] = p;
    }
  }
  for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
  if ((threadIdx.x & 31) == 0 && hmax > 0.0f) atomicMax(&s_hmax, __float_as_uint(hmax));
  __syncthreads();
  if (threadIdx.x == 0) g.cell_Hmax[c] = __uint_as_float(s_hmax);
  if (cnt > kMax) return;
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float ux, uy, uz;
  axis_u(k, ux, uy, uz);
  float* key = s_key + k * kMax;
  uint16_t* out = s_out + k * kMax;
  uint16_t* tmp = s_tmp + k * kMax;
  int* bkt = s_bkt + k * (kB + 32);
  constexpr int kPer = kMax / 32;
  float kr[kPer];
  float kmin = 3.0e38f, kmax = -3.0e38f;
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    const int t = lane + 32 * j;
    kr[j] = 0.0f;
    if (t < cnt) {
      const float d = project(s_x[t], ux, uy, uz);
      key[t] = d;
      kr[j] = d;
      kmin = fminf(kmin, d);
      kmax = fmaxf(kmax, d);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  int nb = 32;
  while (nb < cnt) nb <<= 1;
  warp_sort_axis<kPer>(cnt, kr, key, s_orig, tmp, out, bkt, nb, lane, kmin, kmax);
  const size_t base = (size_t)k * g.n + cs;
#pragma unroll
  for (int j = 0; j < kPer; j++) {
    const int t = lane + 32 * j;
    if (t < cnt) {
      const int v = out[t];
      g.perm[base + t] = (uint16_t)v;
      g.dist[base + t] = key[v];
    }
  }
}

// One warp per cell of at most kSortTinyMax particles (a clustered box has
// tens of thousands of them, which k_cell_sort's one CTA per cell handles
// poorly): the same gather into cell order and H_max, then the 13 axes in
// turn with the same warp bucket sort, from a per-warp copy of the keys.
__global__ void __launch_bounds__(kSortTinyWarps * 32) k_cell_sort_tiny(
    GridDev g, const double* __restrict__ pos, const float* __restrict__ h,
    const float* __restrict__ m, float m_uniform) {
  pdl_enter();
  constexpr int kPer = kSortTinyMax / 32;
  __shared__ float4 s_x[kSortTinyWarps][kSortTinyMax];
  __shared__ float s_key[kSortTinyWarps][kSortTinyMax];
  __shared__ int s_orig[kSortTinyWarps][kSortTinyMax];
  __shared__ uint16_t s_tmp[kSortTinyWarps][kSortTinyMax];
  __shared__ uint16_t s_out[kSortTinyWarps][kSortTinyMax];
  __shared__ int s_bkt[kSortTinyWarps][kSortTinyMax + 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* wx = s_x[warp];
  float* key = s_key[warp];
  int* orig = s_orig[warp];
  for (int c = blockIdx.x * kSortTinyWarps + warp; c < g.ncell;
       c += gridDim.x * kSortTinyWarps) {
    const int cnt = g.cell_count[c];
    if (cnt > kSortTinyMax) continue;
    const int cs = g.cell_start[c];
    const int bx = g.cell_box[c];
    const BoxDev& B = g.boxes[bx];
    const int loc = c - B.cell_base;
    const double ctr[3] = {-((loc / (B.nc * B.nc)) + 0.5), -(((loc / B.nc) % B.nc) + 0.5),
                           -((loc % B.nc) + 0.5)};
    const float mmax = g.m_max[bx];
    float hmax = 0.0f;
    for (int t = lane; t < cnt; t += 32) {
      const int p = g.orig[cs + t];
      const size_t s = (size_t)cs + t;
      float off[3];
#pragma unroll
      for (int k = 0; k < 3; k++) {
        double x = pos[3 * (size_t)p + k];
        if (!finite_bits(x)) x = 0.0;
        if (!in_box_bits(x, B.L)) x = wrap_coord(x, B.L);
        off[k] = (float)fma(ctr[k], B.edge, x);
        g.pos64[3 * s + k] = x;
      }
      const float mv = m ? m[p] : m_uniform;
      const float hv = h[p];
      const float4 xm = make_float4(off[0], off[1], off[2], mmax > 0.0f ? mv / mmax : 0.0f);
      g.xm[s] = xm;
      g.xm_ref[s] = xm;
      g.hs[s] = hv;
      if (valid_h_m(hv, mv)) hmax = fmaxf(hmax, g.gamma * hv);
      wx[t] = xm;
      orig[t] = p;
    }
    for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    if (lane == 0) g.cell_Hmax[c] = hmax;
    if (cnt == 0) continue;
    __syncwarp();
    if (cnt <= 32) {
      // one key per lane: its rank is the number of keys before it in
      // (projection, caller index) order, counted over shuffles (the order
      // of the bucket sort below, without its buckets)
      const float4 xl = lane < cnt ? wx[lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const int ol = lane < cnt ? orig[lane] : 0;
      for (int k = 0; k < kNDir; k++) {
        float ux, uy, uz;
        axis_u(k, ux, uy, uz);
        const float kl = project(xl, ux, uy, uz);
        int r = 0;
        for (int u = 0; u < cnt; u++) {
          const float ku = __shfl_sync(0xffffffffu, kl, u);
          const int ou = __shfl_sync(0xffffffffu, ol, u);
          r += key_less(ku, ou, kl, ol) ? 1 : 0;
        }
        if (lane < cnt) {
          const size_t base = (size_t)k * g.n + cs;
          g.perm[base + r] = (uint16_t)lane;
          g.dist[base + r] = kl;
        }
      }
      continue;
    }
    int nb = 32;
    while (nb < cnt) nb <<= 1;
    for (int k = 0; k < kNDir; k++) {
      float ux, uy, uz;
      axis_u(k, ux, uy, uz);
      float kr[kPer];
      float kmin = 3.0e38f, kmax = -3.0e38f;
#pragma unroll
      for (int j = 0; j < kPer; j++) {
        const int t = lane + 32 * j;
        kr[j] = 0.0f;
        if (t < cnt) {
          const float d = project(wx[t], ux, uy, uz);
          key[t] = d;
          kr[j] = d;
          kmin = fminf(kmin, d);
          kmax = fmaxf(kmax, d);
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
      }
      __syncwarp();
      warp_sort_axis<kPer>(cnt, kr, key, orig, s_tmp[warp], s_out[warp], s_bkt[warp], nb, lane,
                           kmin, kmax);
      const size_t base = (size_t)k * g.n + cs;
#pragma unroll
      for (int j = 0; j < kPer; j++) {
        const int t = lane + 32 * j;
        if (t < cnt) {
          const int v = s_out[warp][t];
          g.perm[base + t] = (uint16_t)v;
          g.dist[base + t] = key[v];
        }
      }
      __syncwarp();  // key is rewritten by the next axis
    }
  }
}

// One CTA per (cell of more than kSortSmallMax particles, axis), the same
// bucket sort with the buckets in shared memory.  For a cell of at most
// kSortBigSmem particles the keys, caller indices and bucket-grouped indices
// are staged in shared memory too (keys computed once); larger cells need no
// scratch beyond the axis's own outputs: the bucket-grouped indices go into
// dist[k] (as int bits) until the exact ranks have been written to perm[k],
// then dist[k] receives the keys, which are recomputed from xm wherever they
// are needed (the same FP32 expression each time, so the same values).
constexpr int kSortBigThreads = 1024;
constexpr int kSortBigBuckets = 8192;
constexpr int kSortBigSmem = 6144;
constexpr size_t kSortBigDynSmem =
    (size_t)kSortBigSmem * (sizeof(float) + sizeof(int) + sizeof(uint16_t));

template <bool kStaged>
__global__ void __launch_bounds__(kSortBigThreads, kStaged ? 2 : 1) k_sort_big(GridDev g) {
  pdl_enter();
  __shared__ int s_bkt[kSortBigBuckets + kSortBigThreads];  // bucket b at bucket_slot(b, sh)
  __shared__ float s_red[2][32];
  __shared__ int s_scan[32];
  extern __shared__ float s_key[];                                  // [kSortBigSmem]
  int* s_org = reinterpret_cast<int*>(s_key + kSortBigSmem);        // [kSortBigSmem]
  uint16_t* s_grp = reinterpret_cast<uint16_t*>(s_org + kSortBigSmem);  // [kSortBigSmem]
  if (*g.flags) return;
  const int nbig = *g.n_big;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int idx = blockIdx.x; idx < nbig * kNDir; idx += gridDim.x) {
    const int c = g.big_cells[idx / kNDir], k = idx % kNDir;
    const int cnt = min(g.cell_count[c], PV_MAX_CELL_COUNT);
    // cells of at most kSortBigSmem particles go to the staged instance
    if ((cnt <= kSortBigSmem) != kStaged) continue;
    const int cs = g.cell_start[c];
    constexpr bool staged = kStaged;
    int B = kSortBigThreads;
    while (B < cnt && B < kSortBigBuckets) B <<= 1;
    float ux, uy, uz;
    axis_u(k, ux, uy, uz);
    const float4* X = g.xm + cs;
    const int* O = g.orig + cs;
    const size_t base = (size_t)k * g.n + cs;
    int* tmp = reinterpret_cast<int*>(g.dist + base);
    uint16_t* out = g.perm + base;
    auto key_of = [&](int t) { return staged ? s_key[t] : project(X[t], ux, uy, uz); };
    auto org_of = [&](int t) { return staged ? s_org[t] : O[t]; };
    float kmin = 3.0e38f, kmax = -3.0e38f;
    for (int t = tid; t < cnt; t += nthr) {
      const float d = project(X[t], ux, uy, uz);
      if (staged) {
        s_key[t] = d;
        s_org[t] = O[t];
      }
      kmin = fminf(kmin, d);
      kmax = fmaxf(kmax, d);
    }
    for (int o = 16; o > 0; o >>= 1) {
      kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
      kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if ((tid & 31) == 0) {
      s_red[0][tid >> 5] = kmin;
      s_red[1][tid >> 5] = kmax;
    }
    const int per = B / nthr, sh = __ffs(per) - 1;
    for (int b = tid; b < B + nthr; b += nthr) s_bkt[b] = 0;
    __syncthreads();
    kmin = s_red[0][0];
    kmax = s_red[1][0];
    for (int w = 1; w < (nthr >> 5); w++) {
      kmin = fminf(kmin, s_red[0][w]);
      kmax = fmaxf(kmax, s_red[1][w]);
    }
    const float scale = kmax > kmin ? (float)B / (kmax - kmin) : 0.0f;
    auto bucket_of = [&](float d) { return min(B - 1, max(0, (int)((d - kmin) * scale))); };
    for (int t = tid; t < cnt; t += nthr)
      atomicAdd(&s_bkt[bucket_slot(bucket_of(key_of(t)), sh)], 1);
    __syncthreads();
    // exclusive scan: each thread owns B / nthr consecutive buckets
    const int p0 = bucket_slot(tid * per, sh);
    int sum = 0;
    for (int b = p0; b < p0 + per; b++) sum += s_bkt[b];
    int run = group_exclusive_scan<true>(sum, tid, s_scan);
    for (int b = p0; b < p0 + per; b++) {
      const int v = s_bkt[b];
      s_bkt[b] = run;
      run += v;
    }
    __syncthreads();
    for (int t = tid; t < cnt; t += nthr) {
      const int at = atomicAdd(&s_bkt[bucket_slot(bucket_of(key_of(t)), sh)], 1);
      if (staged) s_grp[at] = (uint16_t)t; else tmp[at] = t;
    }
    __syncthreads();
    // s_bkt[b] is now the end of bucket b; rank each particle inside its bucket
    for (int t = tid; t < cnt; t += nthr) {
      const float kt = key_of(t);
      const int b = bucket_of(kt);
      const int s0 = b ? s_bkt[bucket_slot(b - 1, sh)] : 0, s1 = s_bkt[bucket_slot(b, sh)];
      const int ot = org_of(t);
      int r = 0;
      for (int u = s0; u < s1; u++) {
        const int v = staged ? (int)s_grp[u] : tmp[u];
        r += key_less(key_of(v), org_of(v), kt, ot) ? 1 : 0;
      }
      out[s0 + r] = (uint16_t)t;
    }
    __syncthreads();
    for (int t = tid; t < cnt; t += nthr) g.dist[base + t] = key_of(out[t]);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_bin(const GridDev& g, const double* pos, const float* h, const float* m,
                       float m_uniform, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  PV_LAUNCH(k_bin, (g.n + 255) / 256, 256, 0, st, g, pos, h, m, m_uniform);
  return cudaSuccess;
}

cudaError_t launch_scan(const GridDev& g, cudaStream_t st) {
  PV_LAUNCH(k_scan, 1, 1024, 0, st, g);
  return cudaSuccess;
}

cudaError_t launch_scatter(const GridDev& g, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  PV_LAUNCH(k_scatter, (g.n + 255) / 256, 256, 0, st, g);
  return cudaSuccess;
}

cudaError_t launch_update(const GridDev& g, const double* pos, const float* h, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  PV_LAUNCH(k_update, (g.n + 255) / 256, 256, 0, st, g, pos, h);
  PV_LAUNCH(k_update_check, (g.ncell + 255) / 256, 256, 0, st, g);
  return cudaSuccess;
}

cudaError_t launch_clear(const GridDev& g, cudaStream_t st) {
  const int n = g.ncell > g.n_boxes ? g.ncell : g.n_boxes;
  PV_LAUNCH(k_clear, (n + 255) / 256, 256, 0, st, g);
  return cudaSuccess;
}

cudaError_t launch_sort(const GridDev& g, const double* pos, const float* h, const float* m,
                        float m_uniform, cudaStream_t st) {
  constexpr int smem = (int)sort_small_smem<kSortSmallMax>();
  cudaError_t e =
      set_max_dynamic_smem(reinterpret_cast<const void*>(&k_cell_sort<kSortSmallMax>), smem, st);
  if (e != cudaSuccess) return e;
  PV_LAUNCH(k_cell_sort<kSortSmallMax>, g.ncell, kSortThreads, smem, st, g, pos, h, m,
            m_uniform);
  PV_LAUNCH(k_cell_sort_tiny, (g.ncell + kSortTinyWarps - 1) / kSortTinyWarps,
            kSortTinyWarps * 32, 0, st, g, pos, h, m, m_uniform);
  if (g.n == 0) return cudaSuccess;
  if ((e = set_max_dynamic_smem(reinterpret_cast<const void*>(&k_sort_big<true>),
                                (int)kSortBigDynSmem, st)) != cudaSuccess)
    return e;
  // persistent grids over (big cell, axis): two CTAs per SM for the staged
  // instance, one for the rare cells above kSortBigSmem
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  PV_LAUNCH_PLAIN(k_sort_big<true>, 2 * sms, kSortBigThreads, kSortBigDynSmem, st, g);
  PV_LAUNCH_PLAIN(k_sort_big<false>, sms, kSortBigThreads, 0, st, g);
  return cudaSuccess;
}

}  // namespace pv
