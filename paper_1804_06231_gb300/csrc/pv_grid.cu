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
//   k_clear    zeroes the occupancies, cell maxima and the per-sort scalars
//   k_bin      particle -> cell id, occupancy histogram, box m_max, input
//              checks (latched flags)
//   k_scan_tile, k_scan_add  exclusive scan of the occupancies (two passes
//              over tiles of cells), the cell lists of the sort paths
//   k_scatter  caller index of every cell-order slot
//   k_gather   one thread per cell-order slot: the particle's FP32 offset
//              from its cell centre + normalised mass, h, the wrapped FP64
//              position, and the cell's H_max
//   k_cell_sort_tiny  cells of <= 64 particles, one warp per cell: rank
//              counting over (axis, particle) pairs for <= 32, else the 13
//              axes in turn with a warp bucket (counting) sort, exact order
//              inside a bucket by (projection, caller index)
//   k_cell_sort   cells of 65..384 particles, one CTA per cell, one warp per
//              axis, the same warp bucket sort
//   k_sort_big    one CTA per (larger cell, axis), the same algorithm with
//              up to 16384 buckets in shared memory (three instances by size)
//   k_update, k_update_check  new positions on a kept sort (pv_update_positions)
#include <cuda_runtime.h>

#include "pv_internal.cuh"

namespace pv {

namespace {

// cells of up to kSortTinyMax particles are sorted by one warp, cells of up
// to kSortSmallMax particles by one CTA (74 KB of shared memory, three CTAs
// per SM, one warp per axis), larger ones with one CTA per (cell, axis)
constexpr int kSortTinyMax = 64;
constexpr int kSortSmallMax = 384;
constexpr int kSortMidMax = 1536;    // larger cells: one CTA per (cell, axis)
constexpr int kSortLargeMax = 6144;
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
  if (i < g.ncell) {
    g.cell_count[i] = 0;
    g.cell_Hmax[i] = 0.0f;
  }
  if (i < g.n_boxes) {
    g.m_max[i] = 0.0f;
    g.box_disp[i] = 0.0f;
  }
  if (i == 0) {
    *g.flags = 0u;
    *g.max_count = 0;
    *g.n_big = 0;
    *g.n_large = 0;
    *g.n_small = 0;
    *g.n_huge = 0;
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

__global__ void k_scatter(GridDev g) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < g.n) g.orig[g.cell_start[g.pcell[p]] + g.prank[p]] = p;
}

// Gathers the particle p of cell-order slot s of a cell of box B centred at
// -ctr (in units of the edge): the FP32 offset from the cell centre (Section
// 3.2: shifted in FP64, then rounded) with the normalised mass, h, the copy
// kept for pv_update_positions and the wrapped FP64 position.  Returns the
// staged record; hm is gamma h, or 0 for an invalid h or mass.
__device__ __forceinline__ float4 gather_slot(const GridDev& g, int s, int p, const BoxDev& B,
                                              const double (&ctr)[3], float mmax,
                                              const double* __restrict__ pos,
                                              const float* __restrict__ h,
                                              const float* __restrict__ m, float m_uniform,
                                              float& hm) {
  float off[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    double x = pos[3 * (size_t)p + k];
    if (!finite_bits(x)) x = 0.0;
    if (!in_box_bits(x, B.L)) x = wrap_coord(x, B.L);
    off[k] = (float)fma(ctr[k], B.edge, x);
    g.pos64[3 * (size_t)s + k] = x;
  }
  const float mv = m ? m[p] : m_uniform;
  const float hv = h[p];
  const float4 xm = make_float4(off[0], off[1], off[2], mmax > 0.0f ? mv / mmax : 0.0f);
  g.xm[s] = xm;
  g.xm_ref[s] = xm;
  g.hs[s] = hv;
  hm = valid_h_m(hv, mv) ? g.gamma * hv : 0.0f;
  return xm;
}

// The centre of cell c of box B, negated, in units of the edge.
__device__ __forceinline__ void cell_centre(const BoxDev& B, int c, double (&ctr)[3]) {
  const int loc = c - B.cell_base;
  ctr[0] = -((loc / (B.nc * B.nc)) + 0.5);
  ctr[1] = -(((loc / B.nc) % B.nc) + 0.5);
  ctr[2] = -((loc % B.nc) + 0.5);
}

// One thread per cell-order slot s: gathers the slot's particle and raises its
// cell's H_max (cleared by k_clear), one atomic per run of equal cells in the
// warp.  Every slot is independent, so the random reads of the caller's
// arrays all overlap.
__global__ void k_gather(GridDev g, const double* __restrict__ pos, const float* __restrict__ h,
                         const float* __restrict__ m, float m_uniform) {
  pdl_enter();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int cell = -1;
  float hm = 0.0f;
  if (s < g.n) {
    const int p = g.orig[s];
    cell = g.pcell[p];
    const int bx = g.cell_box[cell];
    const BoxDev& B = g.boxes[bx];
    double ctr[3];
    cell_centre(B, cell, ctr);
    gather_slot(g, s, p, B, ctr, g.m_max[bx], pos, h, m, m_uniform, hm);
  }
  // H_max >= 0: the float order is the order of the bit patterns
  const unsigned grp = __match_any_sync(0xffffffffu, cell);
  const unsigned hb = __reduce_max_sync(grp, __float_as_uint(hm));
  if (cell >= 0 && hb != 0u && (int)(threadIdx.x & 31) == __ffs(grp) - 1)
    atomicMax(reinterpret_cast<unsigned int*>(&g.cell_Hmax[cell]), hb);
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

// Appends val to list (at the front, or from the back when back) for every
// lane with pred: one atomic per warp.  All 32 lanes take part.
__device__ __forceinline__ void warp_push(bool pred, int32_t* list, int32_t* n, int val,
                                          bool back, int len) {
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if (!b) return;
  const int lane = threadIdx.x & 31, lead = __ffs(b) - 1;
  int base = 0;
  if (lane == lead) base = atomicAdd(n, __popc(b));
  base = __shfl_sync(0xffffffffu, base, lead);
  const int at = base + __popc(b & ((1u << lane) - 1u));
  if (pred) list[back ? len - 1 - at : at] = val;
}

// Exclusive scan of the cell occupancies in two passes over tiles of
// kScanTile cells.  k_scan_tile: the scan inside each tile (its total in
// tile_sum), the largest occupancy and the cell lists of the sort paths.
__global__ void __launch_bounds__(kScanTile) k_scan_tile(GridDev g) {
  pdl_enter();
  __shared__ int s_w[32];
  const int c = blockIdx.x * kScanTile + threadIdx.x;
  const int v = c < g.ncell ? g.cell_count[c] : 0;
  const int ex = group_exclusive_scan<true>(v, threadIdx.x, s_w);
  if (c < g.ncell) g.cell_start[c] = ex;
  if (threadIdx.x == kScanTile - 1) g.tile_sum[blockIdx.x] = ex + v;
  const int mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && mx > 0) {
    atomicMax(g.max_count, mx);
    if (mx > PV_MAX_CELL_COUNT) atomicOr(g.flags, PV_FLAG_CELL_OVERFLOW);
  }
  warp_push(v > kSortTinyMax && v <= kSortSmallMax, g.small_cells, g.n_small, c, false, g.ncell);
  warp_push(v > kSortLargeMax, g.small_cells, g.n_huge, c, true, g.ncell);
  warp_push(v > kSortSmallMax && v <= kSortMidMax, g.big_cells, g.n_big, c, false, g.ncell);
  warp_push(v > kSortMidMax && v <= kSortLargeMax, g.big_cells, g.n_large, c, true, g.ncell);
}

// k_scan_add: each tile adds the totals of the tiles before it; the last one
// also writes cell_start[C], the particle count.
__global__ void __launch_bounds__(kScanTile) k_scan_add(GridDev g) {
  pdl_enter();
  __shared__ int s_w[32];
  int p = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanTile) p += g.tile_sum[t];
  p = (int)__reduce_add_sync(0xffffffffu, (unsigned)p);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = p;
  __syncthreads();
  p = 0;
  for (int w = 0; w < kScanTile / 32; w++) p += s_w[w];
  const int c = blockIdx.x * kScanTile + threadIdx.x;
  if (c < g.ncell) g.cell_start[c] += p;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    g.cell_start[g.ncell] = p + g.tile_sum[blockIdx.x];
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

// (projection, caller index) as one unsigned integer of the same order: the
// FP32 order of d (-0 and +0 equal) in the high word, the index o >= 0 below
__device__ __forceinline__ unsigned long long sort_key64(float d, int o) {
  const unsigned b = __float_as_uint(d == 0.0f ? 0.0f : d);
  const unsigned u = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned)o;
}

// Cells of at most kSortTinyMax particles, one warp per cell (a clustered box
// has tens of thousands of them, which a CTA per cell handles poorly): the
// cell's staged offsets and caller indices are loaded into the warp's shared
// memory, then
// * cells of at most 32: the lanes take the 13 cnt (axis, particle) pairs in
//   turn; the rank of a key is the count of keys before it in (projection,
//   caller index) order, read from a row of 33 words per axis (broadcasts,
//   and lanes on different axes in different banks);
// * larger cells: the 13 axes in turn with the warp bucket sort.
constexpr int kTinyRow = 33;
struct TinyBuf {  // one warp's shared memory
  float4 x[kSortTinyMax];
  int orig[kSortTinyMax];
  // the 64-bit keys of the <= 32 path, or the bucket sort's arrays
  unsigned long long u[kNDir * kTinyRow];
};
static_assert(kSortTinyMax * (sizeof(float) + 2 * sizeof(uint16_t)) +
                      (kSortTinyMax + 32) * sizeof(int) <=
                  sizeof(TinyBuf::u),
              "the bucket sort's arrays fit the key rows");

// The warp with index w0 of nw takes cells w0, w0 + nw, ...
__device__ __forceinline__ void sort_tiny_cells(const GridDev& g, TinyBuf& tb, int lane, int w0,
                                                int nw) {
  constexpr int kPer = kSortTinyMax / 32;
  float4* wx = tb.x;
  int* orig = tb.orig;
  unsigned long long* kk = tb.u;
  float* key = reinterpret_cast<float*>(kk);
  uint16_t* tmp = reinterpret_cast<uint16_t*>(key + kSortTinyMax);
  uint16_t* out = tmp + kSortTinyMax;
  int* bkt = reinterpret_cast<int*>(out + kSortTinyMax);
  for (int c = w0; c < g.ncell; c += nw) {
    const int cnt = g.cell_count[c];
    if (cnt > kSortTinyMax || cnt == 0) continue;
    const int cs = g.cell_start[c];
    for (int t = lane; t < cnt; t += 32) {
      wx[t] = g.xm[cs + t];
      orig[t] = g.orig[cs + t];
    }
    __syncwarp();
    if (cnt <= 32) {
      const int npair = kNDir * cnt;
      // pair q = (axis k, particle t) with k = q / cnt: (q + 1/2) / cnt in
      // FP32 is at least 1 / (2 cnt) from an integer, far above its rounding
      const float inv = 1.0f / (float)cnt;
      float kf[kNDir];
#pragma unroll
      for (int j = 0; j < kNDir; j++) {
        const int q = lane + 32 * j;
        kf[j] = 0.0f;
        if (q < npair) {
          const int k = (int)(((float)q + 0.5f) * inv), t = q - k * cnt;
          float ux, uy, uz;
          axis_u(k, ux, uy, uz);
          kf[j] = project(wx[t], ux, uy, uz);
          kk[k * kTinyRow + t] = sort_key64(kf[j], orig[t]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kNDir; j++) {
        const int q = lane + 32 * j;
        if (q < npair) {
          const int k = (int)(((float)q + 0.5f) * inv), t = q - k * cnt;
          const unsigned long long* row = kk + k * kTinyRow;
          const unsigned long long me = row[t];
          int r = 0;
#pragma unroll 4
          for (int u = 0; u < cnt; u++) r += row[u] < me ? 1 : 0;
          const size_t base = (size_t)k * g.n + cs;
          g.perm[base + r] = (uint16_t)t;
          g.dist[base + r] = kf[j];
        }
      }
      __syncwarp();  // the rows are rewritten by the next cell
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
      kmin = warp_min_f(kmin);
      kmax = warp_max_f(kmax);
      __syncwarp();
      warp_sort_axis<kPer>(cnt, kr, key, orig, tmp, out, bkt, nb, lane, kmin, kmax);
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
      __syncwarp();  // key is rewritten by the next axis
    }
  }
}

// One warp's axis k of a staged cell of cnt <= 32 kPer particles (the keys,
// bucket sort and the axis's outputs).
template <int kPer>
__device__ __forceinline__ void cell_sort_axis(const GridDev& g, int k, int lane, int cnt, int cs,
                                               const float4* s_x, const int* s_orig, float* key,
                                               uint16_t* tmp, uint16_t* out, int* bkt) {
  float ux, uy, uz;
  axis_u(k, ux, uy, uz);
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
  kmin = warp_min_f(kmin);
  kmax = warp_max_f(kmax);
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

// One CTA per cell of kSortTinyMax < count <= kMax (entry blockIdx.x of the
// small_cells list; the grid covers every cell, the CTAs past the list's end
// exit at once): the cell's staged offsets and caller indices are loaded
// (coalesced) into shared memory, then the 13 axes are sorted one warp each.
template <int kMax>
__global__ void __launch_bounds__(kSortThreads, 3) k_cell_sort(GridDev g) {
  pdl_enter();
  constexpr int kB = sort_small_buckets<kMax>();
  extern __shared__ float4 smem4[];
  float4* s_x = smem4;                                           // [kMax]
  int* s_orig = reinterpret_cast<int*>(s_x + kMax);              // [kMax]
  float* s_key = reinterpret_cast<float*>(s_orig + kMax);        // [13][kMax]
  int* s_bkt = reinterpret_cast<int*>(s_key + kNDir * kMax);     // [13][kB + 32]
  uint16_t* s_out = reinterpret_cast<uint16_t*>(s_bkt + kNDir * (kB + 32));  // [13][kMax]
  uint16_t* s_tmp = s_out + kNDir * kMax;                        // [13][kMax]
  const int i = blockIdx.x;  // one CTA per listed cell (the grid covers every cell)
  if (i >= *g.n_small) return;
  const int c = g.small_cells[i];
  const int cnt = min(g.cell_count[c], kMax);
  const int cs = g.cell_start[c];
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    s_x[t] = g.xm[cs + t];
    s_orig[t] = g.orig[cs + t];
  }
  __syncthreads();
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cell_sort_axis<kMax / 32>(g, k, lane, cnt, cs, s_x, s_orig, s_key + k * kMax, s_tmp + k * kMax,
                            s_out + k * kMax, s_bkt + k * (kB + 32));
}

// One warp per cell of at most kSortTinyMax particles, over all cells.
constexpr int kSortTinyWarps = 4;  // (small CTAs: one retires when its four cells are done)
__global__ void __launch_bounds__(kSortTinyWarps * 32, 10) k_cell_sort_tiny(GridDev g) {
  pdl_enter();
  __shared__ TinyBuf s_tb[kSortTinyWarps];
  const int warp = threadIdx.x >> 5;
  sort_tiny_cells(g, s_tb[warp], threadIdx.x & 31, blockIdx.x * kSortTinyWarps + warp,
                  gridDim.x * kSortTinyWarps);
}

// One CTA per (cell of more than kSortSmallMax particles, axis), persistent:
// the same bucket sort with the buckets in shared memory and the keys
// computed once into shared memory.  Three instances over three cell lists:
//   mid   (<= kSortMidMax particles)   kSortMidThreads threads, six CTAs per SM
//   large (<= kSortLargeMax)           kSortLargeThreads threads, two per SM
//   huge  (the rest)                   kSortHugeThreads threads, one per SM
// The mid and large instances stage the caller indices and the ranks too,
// so that no phase waits on global memory.  The huge one stages only the
// keys and the bucket-grouped indices, and a cell above kStage needs no
// scratch beyond the axis's own outputs: the grouped indices go into dist[k]
// (as int bits) until the exact ranks have been written to perm[k], then
// dist[k] receives the keys, recomputed from xm wherever they are needed (the
// same FP32 expression each time, so the same values).  Caller indices are
// read only to order equal keys.
constexpr int kSortMidThreads = 256;
constexpr int kSortMidBuckets = 2048;  // >= kSortMidMax
constexpr int kSortLargeThreads = 512;
constexpr int kSortLargeBuckets = 8192;  // >= kSortLargeMax
constexpr int kSortHugeThreads = 1024;
constexpr int kSortHugeBuckets = 16384;
constexpr int kSortHugeStage = 24576;
enum SortList { kListMid = 0, kListLarge = 1, kListHuge = 2 };

template <int kThreads, int kMaxB, int kStage, int kList>
constexpr size_t sort_big_smem() {
  return (size_t)(kMaxB + kThreads) * sizeof(int) +
         (size_t)kStage * (kList == kListHuge ? sizeof(float) + sizeof(uint16_t)
                                              : sizeof(float) + sizeof(int) + 2 * sizeof(uint16_t));
}

template <int kThreads, int kMaxB, int kStage, int kList>
__global__ void __launch_bounds__(kThreads, kList == kListMid ? 6 : (kList == kListLarge ? 2 : 1))
    k_sort_big(GridDev g) {
  pdl_enter();
  static_assert(kMaxB % kThreads == 0, "whole buckets per thread in the scan");
  constexpr bool kFull = kList != kListHuge;  // every cell fits; indices and ranks staged
  constexpr int kWarps = kThreads / 32;
  extern __shared__ int s_dyn[];
  int* s_bkt = s_dyn;                                                 // [kMaxB + kThreads]
  float* s_key = reinterpret_cast<float*>(s_bkt + kMaxB + kThreads);  // [kStage]
  int* s_org = reinterpret_cast<int*>(s_key + kStage);                // [kStage] (kFull)
  uint16_t* s_grp = reinterpret_cast<uint16_t*>(kFull ? s_org + kStage : s_org);  // [kStage]
  uint16_t* s_out = s_grp + kStage;                                   // [kStage] (kFull)
  __shared__ float s_red[2][kWarps];
  __shared__ int s_scan[32];
  // huge instance: a list of at most kOrderMax cells is taken largest first,
  // so that the items of the last round are the shortest
  constexpr int kOrderMax = 256;
  __shared__ int s_order[kList == kListHuge ? kOrderMax : 1];
  if (*g.flags) return;
  const int nlist = kList == kListMid ? *g.n_big : (kList == kListLarge ? *g.n_large : *g.n_huge);
  const int nitem = nlist * kNDir;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool ordered = kList == kListHuge && nlist <= kOrderMax;  // (the same in every thread)
  if (ordered) {
    auto count_of = [&](int e) { return g.cell_count[g.small_cells[g.ncell - 1 - e]]; };
    for (int e = tid; e < nlist; e += kThreads) {
      const int ne = count_of(e);
      int r = 0;  // entries before e: larger, or as large and earlier in the list
      for (int f = 0; f < nlist; f++) {
        const int nf = count_of(f);
        r += (nf > ne || (nf == ne && f < e)) ? 1 : 0;
      }
      s_order[r] = e;
    }
    __syncthreads();
  }
  for (int idx = blockIdx.x; idx < nitem; idx += gridDim.x) {
    const int e0 = idx / kNDir, k = idx - e0 * kNDir;
    const int e = ordered ? s_order[e0] : e0;
    const int c = kList == kListMid     ? g.big_cells[e]
                  : kList == kListLarge ? g.big_cells[g.ncell - 1 - e]
                                        : g.small_cells[g.ncell - 1 - e];
    const int cnt = min(g.cell_count[c], kFull ? kStage : PV_MAX_CELL_COUNT);
    const bool staged = kFull || cnt <= kStage;
    const int cs = g.cell_start[c];
    int B = kThreads;
    while (B < cnt && B < kMaxB) B <<= 1;
    float ux, uy, uz;
    axis_u(k, ux, uy, uz);
    const float4* X = g.xm + cs;
    const int* O = g.orig + cs;
    const size_t base = (size_t)k * g.n + cs;
    int* tmp = reinterpret_cast<int*>(g.dist + base);
    uint16_t* out = g.perm + base;
    auto key_of = [&](int t) { return staged ? s_key[t] : project(X[t], ux, uy, uz); };
    auto org_of = [&](int t) { return kFull ? s_org[t] : O[t]; };
    float kmin = 3.0e38f, kmax = -3.0e38f;
    for (int t = tid; t < cnt; t += kThreads) {
      const float d = project(X[t], ux, uy, uz);
      if (staged) s_key[t] = d;
      if (kFull) s_org[t] = O[t];
      kmin = fminf(kmin, d);
      kmax = fmaxf(kmax, d);
    }
    kmin = warp_min_f(kmin);
    kmax = warp_max_f(kmax);
    if (lane == 0) {
      s_red[0][warp] = kmin;
      s_red[1][warp] = kmax;
    }
    const int per = B / kThreads, sh = __ffs(per) - 1;
    for (int b = tid; b < B + kThreads; b += kThreads) s_bkt[b] = 0;
    __syncthreads();
    kmin = warp_min_f(lane < kWarps ? s_red[0][lane] : 3.0e38f);
    kmax = warp_max_f(lane < kWarps ? s_red[1][lane] : -3.0e38f);
    const float scale = kmax > kmin ? (float)B / (kmax - kmin) : 0.0f;
    auto bucket_of = [&](float d) { return min(B - 1, max(0, (int)((d - kmin) * scale))); };
    for (int t = tid; t < cnt; t += kThreads)
      atomicAdd(&s_bkt[bucket_slot(bucket_of(key_of(t)), sh)], 1);
    __syncthreads();
    // exclusive scan: each thread owns B / kThreads consecutive buckets
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
    for (int t = tid; t < cnt; t += kThreads) {
      const int at = atomicAdd(&s_bkt[bucket_slot(bucket_of(key_of(t)), sh)], 1);
      if (staged) s_grp[at] = (uint16_t)t; else tmp[at] = t;
    }
    __syncthreads();
    // s_bkt[b] is now the end of bucket b; rank each particle inside its
    // bucket (caller indices only between equal keys)
    for (int t = tid; t < cnt; t += kThreads) {
      const float kt = key_of(t);
      const int b = bucket_of(kt);
      const int s0 = b ? s_bkt[bucket_slot(b - 1, sh)] : 0, s1 = s_bkt[bucket_slot(b, sh)];
      int r = 0;
      if (s1 - s0 > 1) {
        const int ot = org_of(t);
        for (int u = s0; u < s1; u++) {
          const int v = staged ? (int)s_grp[u] : tmp[u];
          const float kv = key_of(v);
          if (kv < kt) r++;
          else if (kv == kt && org_of(v) < ot) r++;
        }
      }
      if (kFull) s_out[s0 + r] = (uint16_t)t; else out[s0 + r] = (uint16_t)t;
    }
    __syncthreads();
    for (int t = tid; t < cnt; t += kThreads) {
      const int v = kFull ? (int)s_out[t] : (int)out[t];
      if (kFull) out[t] = (uint16_t)v;
      g.dist[base + t] = key_of(v);
    }
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
  const int tiles = scan_tiles(g.ncell);
  PV_LAUNCH(k_scan_tile, tiles, kScanTile, 0, st, g);
  PV_LAUNCH(k_scan_add, tiles, kScanTile, 0, st, g);
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
  if (g.n == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  PV_LAUNCH(k_gather, (g.n + 255) / 256, 256, 0, st, g, pos, h, m, m_uniform);
  PV_LAUNCH(k_cell_sort_tiny, (g.ncell + kSortTinyWarps - 1) / kSortTinyWarps,
            kSortTinyWarps * 32, 0, st, g);
  constexpr int smem = (int)sort_small_smem<kSortSmallMax>();
  if ((e = set_max_dynamic_smem(reinterpret_cast<const void*>(&k_cell_sort<kSortSmallMax>), smem,
                                st)) != cudaSuccess)
    return e;
  PV_LAUNCH(k_cell_sort<kSortSmallMax>, g.ncell, kSortThreads, smem, st, g);
  // persistent grids over the (cell, axis) items of the larger cells: six
  // CTAs per SM (mid), two (large) and one (huge)
  constexpr size_t mid_smem =
      sort_big_smem<kSortMidThreads, kSortMidBuckets, kSortMidMax, kListMid>();
  constexpr size_t large_smem =
      sort_big_smem<kSortLargeThreads, kSortLargeBuckets, kSortLargeMax, kListLarge>();
  constexpr size_t huge_smem =
      sort_big_smem<kSortHugeThreads, kSortHugeBuckets, kSortHugeStage, kListHuge>();
  auto* mid = &k_sort_big<kSortMidThreads, kSortMidBuckets, kSortMidMax, kListMid>;
  auto* large = &k_sort_big<kSortLargeThreads, kSortLargeBuckets, kSortLargeMax, kListLarge>;
  auto* huge = &k_sort_big<kSortHugeThreads, kSortHugeBuckets, kSortHugeStage, kListHuge>;
  if ((e = set_max_dynamic_smem(reinterpret_cast<const void*>(mid), (int)mid_smem, st)) !=
          cudaSuccess ||
      (e = set_max_dynamic_smem(reinterpret_cast<const void*>(large), (int)large_smem, st)) !=
          cudaSuccess ||
      (e = set_max_dynamic_smem(reinterpret_cast<const void*>(huge), (int)huge_smem, st)) !=
          cudaSuccess)
    return e;
  PV_LAUNCH_PLAIN(huge, sms, kSortHugeThreads, huge_smem, st, g);
  PV_LAUNCH_PLAIN(large, 2 * sms, kSortLargeThreads, large_smem, st, g);
  PV_LAUNCH_PLAIN(mid, 6 * sms, kSortMidThreads, mid_smem, st, g);
  return cudaSuccess;
}

}  // namespace pv
