/*
 * pv.h -- C ABI of the GB300 pseudo-Verlet SPH density loop.
 *
 * The operation (Willis et al., arXiv:1804.06231, Section 1 and Section 2):
 * particles in a periodic cube are binned into cells whose edge is at least
 * the largest interaction radius; for every pair of neighbouring cells the
 * particles of both cells are sorted by their projection on the axis joining
 * the cell centres (13 distinct axes by symmetry, Section 2), and each
 * particle i of cell a only computes distances to the particles j of cell b
 * whose projected distance is below its own radius (Section 2, Section 3.1).
 * The interaction gathered over those pairs is the SPH density of the 3D
 * cubic spline with support H = gamma h:
 *
 *   rho_i     = sum_j m_j W(r_ij, H_i)              (j = i included)
 *   drho_dh_i = sum_j m_j dW/dh(r_ij, h_i)
 *   n_i       = #{ j != i : r_ij < H_i }
 *   W(r, H)   = 8/(pi H^3) * { 1 - 6q^2 + 6q^3 (q < 1/2) | 2 (1-q)^3 (q < 1) | 0 },  q = r/H
 *
 * r_ij is the minimum-image distance in the periodic cube of the particle's
 * box.  All device pointers below are CUDA device (or managed) memory; "host"
 * pointers are ordinary host memory.  Every call is asynchronous on the given
 * stream (a cudaStream_t passed as void*, NULL = the legacy default stream)
 * unless stated otherwise; argument errors are returned synchronously and
 * nothing is launched.  Errors found by the kernels (a support larger than
 * the cell edge, a non-finite position, a cell above PV_MAX_CELL_COUNT, a
 * displacement beyond the skin of a kept sort) are latched in a device status
 * word; later kernels of the grid then leave their outputs untouched, and the
 * next call that synchronises (pv_grid_stats, pv_grid_sync) returns
 * PV_ERR_DEVICE.
 *
 * Thread safety: a pv_grid may be used by one host thread at a time.
 *
 * CUDA graphs: the launches of pv_sort_cells, pv_density and
 * pv_density_backward may be captured into a graph once each call has run
 * eagerly in the same CUDA context (the eager call sets the kernels'
 * shared-memory limits, which cannot be set inside a capture; a captured
 * call without it returns PV_ERR_CUDA).  After cudaDeviceReset, grids
 * created before it are invalid (their device memory is gone: destroy them);
 * new grids and pv_density_static work, the limits being set again by the
 * next eager call.
 */
#ifndef PV_H
#define PV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PV_OK = 0,
  PV_ERR_INVALID_ARGUMENT = 1, /* NULL pointer, negative size, bad box layout */
  PV_ERR_CELL_TOO_SMALL = 2,   /* nc < 3 (returned by pv_grid_create) */
  PV_ERR_OUT_OF_MEMORY = 3,    /* device or host allocation failed */
  PV_ERR_CUDA = 4,             /* a CUDA runtime call failed (see pv_last_cuda_error) */
  PV_ERR_NOT_SORTED = 5,       /* pv_density / pv_density_backward before pv_sort_cells */
  PV_ERR_DEVICE = 6,           /* a kernel latched an error; see pv_stats.device_flags */
  PV_ERR_TOO_LARGE = 7         /* more than 2^31 - 1 particles or cells */
} pv_status;

/* Bits of pv_stats.device_flags (set by the kernels of pv_sort_cells,
   pv_update_positions and pv_density_backward; cleared by pv_sort_cells). */
#define PV_FLAG_SUPPORT_EXCEEDS_CELL 1u /* gamma h_i > L/nc for some particle */
#define PV_FLAG_BAD_POSITION 2u         /* non-finite position coordinate */
#define PV_FLAG_BAD_SMOOTHING 4u        /* h_i not finite or not > 0, or m_i not finite */
#define PV_FLAG_CELL_OVERFLOW 8u        /* a cell holds more than PV_MAX_CELL_COUNT particles */
#define PV_FLAG_SKIN_EXCEEDED 16u       /* pv_update_positions: H_max + 2 x displacement > edge */
#define PV_FLAG_BAD_GRADIENT 32u        /* pv_density_backward: a non-finite upstream gradient */

/* Largest number of particles one cell may hold (cell-local indices are 16-bit). */
#define PV_MAX_CELL_COUNT 65535

/* One periodic box.  Boxes are independent: particles of different boxes
   never interact.  The particles of box b are the contiguous index range
   [first, first + n) of the arrays passed to pv_sort_cells. */
typedef struct {
  int64_t first; /* index of the box's first particle */
  int64_t n;     /* particles in the box (may be 0) */
  double L;      /* edge of the periodic cube [0, L)^3, > 0; positions are wrapped into it */
  int32_t nc;    /* cells per dimension, >= 3; the cell edge L/nc must be >= gamma * max h */
} pv_box_desc;

typedef struct {
  int32_t n_boxes;          /* >= 1 */
  const pv_box_desc* boxes; /* host array [n_boxes]; copied, the caller keeps ownership */
  double gamma;             /* H = gamma h; <= 0 or NaN selects 1.825742 */
  uint32_t flags;           /* must be 0 */
} pv_grid_desc;

typedef struct pv_grid pv_grid; /* opaque; owns all scratch device memory */

typedef struct {
  int64_t n_particles;      /* sum of the boxes' n */
  int64_t n_cells;          /* sum of nc^3 */
  int32_t max_cell_count;   /* largest cell occupancy seen by the last pv_sort_cells */
  uint32_t device_flags;    /* PV_FLAG_* bits latched since the last pv_sort_cells */
  int64_t interactions;     /* sum_i n_i of the last pv_density */
  int64_t guard_pairs;      /* pairs re-decided in FP64 near r = H_i by the last pv_density */
  int64_t candidates;       /* distance tests inside the sorted windows (pv_count_candidates) */
  int64_t device_bytes;     /* scratch device memory owned by the grid */
  int64_t kernel_launches;  /* kernels this grid has launched since it was created */
  int64_t candidates_adjoint; /* adjoint windows: j with projected distance < max(H_i, H_j) */
  int64_t pairs_adjoint;      /* pairs with r_ij < max(H_i, H_j), j = i included */
  int64_t orientation[4][2];  /* per class of neighbour (0 self, 1 face, 2 edge,
                                 3 corner): [0] window distance tests (self
                                 windows include j = i), [1] pairs j != i with
                                 r_ij < H_i (pv_count_candidates) */
} pv_stats;

/* Allocates a grid for the given boxes (cudaMalloc on the current device).
   Host-synchronous.  On success *out owns the grid; free it with
   pv_grid_destroy.  Returns PV_ERR_CELL_TOO_SMALL if a box has nc < 3. */
pv_status pv_grid_create(const pv_grid_desc* desc, pv_grid** out);

/* Frees the grid and its device memory (synchronises the device first).
   NULL is accepted. */
pv_status pv_grid_destroy(pv_grid* g);

/* Cell grid and sorted projections (Section 2; the dist/index arrays of the
   13 axes), built from the caller's particles:
     pos  device double [N][3]  positions (wrapped into [0, L) of their box)
     h    device float  [N]     smoothing lengths, > 0; support H = gamma h
     m    device float  [N]     masses, or NULL to use m_uniform for every particle
   N = sum of the boxes' n.  The grid copies what it needs: the caller may
   reuse pos, h and m once the work queued on `stream` has run.  Kernel-side
   input errors are latched (see PV_FLAG_*). */
pv_status pv_sort_cells(pv_grid* g, const double* pos, const float* h, const float* m,
                        float m_uniform, void* stream);

/* Density gather over the self cell and the 26 neighbour cells of every cell
   (Section 2 and Section 3: sorted sweep with early exit, trimmed to the
   particles that can reach the other cell), results in the caller's particle
   order:
     rho      device float   [N]
     drho_dh  device float   [N]   (NULL: not written)
     n_ngb    device int32_t [N]   (NULL: not written)
   Requires a prior pv_sort_cells on the same grid (else PV_ERR_NOT_SORTED).
   Deterministic: the result does not depend on scheduling. */
pv_status pv_density(pv_grid* g, float* rho, float* drho_dh, int32_t* n_ngb, void* stream);

/* The same rho, drho_dh and n_ngb as pv_density (same arguments, layout and
   requirements), computed with the paper's symmetric pair update (Section
   3.3, last paragraph): each pair of neighbouring cells is swept once, in one
   direction, with the window reaching the larger of the two particles'
   supports, and every pair (i, j) found in range is evaluated once and
   updates both particles (i when r < H_i, j when r < H_j).  The pairs of
   each cell pair are counted once instead of twice; the kernel terms are
   still evaluated per side.  Deterministic (64-bit fixed-point sums).  The
   gather form, pv_density, is the faster of the two on this GPU. */
pv_status pv_density_symmetric(pv_grid* g, float* rho, float* drho_dh, int32_t* n_ngb,
                               void* stream);

/* Adjoint of pv_density (not in the paper).  Given the upstream gradients
     g_rho      device float [N]   dL/drho_i
     g_drho_dh  device float [N]   dL/d(drho_dh)_i   (NULL: zero)
   writes
     g_pos      device float [N][3]  dL/dx_i
     g_h        device float [N]     dL/dh_i         (NULL: not written)
   with
     dL/dh_i = g_i drho_dh_i + k_i sum_j m_j d2W/dh2(r_ij, h_i)
     dL/dx_i = sum_{j != i} (x_i - x_j)/r_ij [ m_j (g_i dW/dr(r,H_i) + k_i d2W/dhdr(r,h_i)) [r < H_i]
                                             + m_i (g_j dW/dr(r,H_j) + k_j d2W/dhdr(r,h_j)) [r < H_j] ]
   (g = g_rho, k = g_drho_dh), computed by re-sweeping the same sorted cell
   pairs as a gather (the transposed term is a second gather, no atomics on
   the outputs).  Requires a prior pv_sort_cells.  Masses are constants.
   Deterministic: partial sums are combined in fixed point (scaled by bounds
   of the terms, per cell and per box), so the result does not depend on
   scheduling.  A non-finite g_rho or g_drho_dh latches PV_FLAG_BAD_GRADIENT
   and leaves g_pos and g_h untouched. */
pv_status pv_density_backward(pv_grid* g, const float* g_rho, const float* g_drho_dh,
                              float* g_pos, float* g_h, void* stream);

/* Re-uses the last pv_sort_cells for new positions and smoothing lengths of
   the same particles (the paper keeps the sorted lists while particles move
   little, Section 2).  Every particle keeps the cell, the slot and the 13
   sorted positions it had at that sort; its offset from that cell's centre
   (nearest periodic image) and its support are updated, and the largest
   displacement since the sort in each box, delta, widens every window by
   2 delta, so the sweeps still visit every pair in range.  That holds while
   H_max + 2 delta <= edge in every cell; otherwise PV_FLAG_SKIN_EXCEEDED is
   latched (later calls return PV_ERR_DEVICE without touching their outputs)
   and the caller must call pv_sort_cells again.  Masses are those of the
   sort.  pos: device double [N][3], h: device float [N], caller order.
   Asynchronous on `stream`.  Errors: PV_ERR_INVALID_ARGUMENT (g, pos or h
   NULL with N > 0), PV_ERR_NOT_SORTED, PV_ERR_CUDA. */
pv_status pv_update_positions(pv_grid* g, const double* pos, const float* h, void* stream);

/* Counts the distance tests of the sorted windows of the method (the
   "candidates": self-cell two-sided windows plus the pair windows of
   Section 2) for the particles sorted by the last pv_sort_cells, into
   pv_stats.candidates, and the corresponding counts of the adjoint sweep
   (window and cut-off max(H_i, H_j)) into pv_stats.candidates_adjoint and
   pv_stats.pairs_adjoint, and the per-orientation counts of the forward
   windows into pv_stats.orientation.  A diagnostic pass; not needed for the
   others. */
pv_status pv_count_candidates(pv_grid* g, void* stream);

/* Waits for the grid's work on `stream` and returns PV_ERR_DEVICE if a kernel
   latched an error flag, else PV_OK.  Host-synchronous. */
pv_status pv_grid_sync(pv_grid* g, void* stream);

/* Fills *out (host pointer).  Synchronises the device.  Returns
   PV_ERR_DEVICE when device_flags is non-zero (out is still filled). */
pv_status pv_grid_stats(pv_grid* g, pv_stats* out);

/* Launch shape of the sweeps (the paper has no counterpart; its method is
   the same for every value).  Per pass, two bins have a shape:
   - the cells whose 27 windows fit a cell-centric CTA's shared memory: the
     number of resident CTAs per SM sets each kernel's shared memory, and with
     it which cells fit; fewer CTAs = more shared memory per cell, more CTAs =
     more warps to hide latency;
   - the other (dense) cells, split into tasks (cell, slot, block of
     particles of a): the block size is the task's particle count and its
     CTA's thread count (64, 128 or 256: 2, 4 or 8 warps per task), with
     16, 8, 4 such CTAs per SM for the density and 14, 7, 3 for the adjoint.
   (Cells of at most 32 particles always go to one warp each.)  0 selects the
   default. */
typedef struct {
  int32_t density_ctas_per_sm;   /* 1..4 (default 3) */
  int32_t backward_ctas_per_sm;  /* 1..3 (default 3) */
  int32_t density_task_block;    /* 64, 128 or 256 (default 128) */
  int32_t backward_task_block;   /* 64, 128 or 256 (default 128) */
  int32_t reserved[4];           /* must be 0 */
} pv_tuning;

/* Sets the launch shape used by later pv_density / pv_density_backward calls
   of this grid.  Host-only, takes effect at the next call.  Errors:
   PV_ERR_INVALID_ARGUMENT for NULL pointers, values out of range or non-zero
   reserved fields (the grid is unchanged). */
pv_status pv_grid_set_tuning(pv_grid* g, const pv_tuning* t);

/* Writes the launch shape in use (defaults resolved) to *out (host). */
pv_status pv_grid_get_tuning(const pv_grid* g, pv_tuning* out);

/* Restricts later pv_density / pv_density_backward calls of this grid to the
   neighbour slots whose bit is set in `mask` (bit o for the neighbour at
   offset (ox, oy, oz) in {-1,0,1}^3, o = 9 (ox+1) + 3 (oy+1) + (oz+1); bit 13
   is the cell itself).  A measurement aid with no counterpart in the paper's
   method (it times the contribution of each neighbour orientation); with a
   partial mask the outputs are partial sums.  PV_SLOT_MASK_ALL restores the
   method.  Errors: PV_ERR_INVALID_ARGUMENT for g == NULL or bits above 26. */
#define PV_SLOT_MASK_ALL 0x7ffffffu
pv_status pv_grid_set_slot_mask(pv_grid* g, uint32_t mask);

/* Raw interaction throughput, the GPU counterpart of the paper's first
   experiment (Section 4: one particle against 2560, all SIMD lanes busy).
   For every i < n_i it sums over all j < n_j, `reps` times, m_j wh(q) and
   m_j th(q), q = |x_i - x_j| / H, the half-scaled kernel terms of pv_density
   (wh = (1-q)^3 - 4 max(1/2-q, 0)^3, th = (1-q)^2 (3-6q) - max(1/2-q, 0)^2
   (6-24q)), with no window, no mask and no cut-off test, so every pair must
   have |x_i - x_j| < H.  It is a measurement of the interaction arithmetic
   alone, not part of the method.
   xi: device float [n_i][4] {x, y, z, m}; xj: device float [n_j][4]; out:
   device float [n_i][2] {sum m wh, sum m th} (over all repetitions); all
   three 16-byte aligned.  Asynchronous on `stream`.  Errors:
   PV_ERR_INVALID_ARGUMENT (negative sizes, reps < 1, H not finite and > 0,
   NULL or misaligned pointers), PV_ERR_TOO_LARGE (sizes above 2^31 - 1),
   PV_ERR_CUDA (launch failure). */
pv_status pv_raw_interactions(const float* xi, int64_t n_i, const float* xj, int64_t n_j,
                              float H, int32_t reps, float* out, void* stream);

/* FP32 throughput probe (a measurement aid; the paper has no counterpart):
   queues one kernel of `threads` threads (a multiple of 256; the caller sizes
   it to fill the GPU), each running 8 independent dependent chains of
   4 x iters fused multiply-adds, as scalar FFMA (packed = 0) or as packed
   fma.rn.f32x2 pairs (packed != 0), and writing one float per thread to the
   device array sink[threads].  *flops (host) receives the FP32 operations of
   the launch (an FMA counts 2).  The caller times the launch on `stream`
   (CUDA events); flops / time is the FP32 peak that the sweep kernels' FP32
   work is compared with.  Errors: PV_ERR_INVALID_ARGUMENT (iters < 1,
   threads negative or not a multiple of 256, NULL flops, NULL sink with
   threads > 0), PV_ERR_TOO_LARGE, PV_ERR_CUDA (launch failure). */
pv_status pv_fp32_probe(int32_t packed, int32_t iters, float* sink, int64_t threads,
                        double* flops, void* stream);

/* Per-kernel timing of the two sweeps (a measurement aid; the paper has no
   counterpart).  With enable != 0, every later pv_density and
   pv_density_backward call records a pair of CUDA events on its stream
   around its cell-centric sweep kernel (the kernel that evaluates the pair
   windows of Section 2 for the cells that fit on chip), which adds no device
   work.  enable = 0 stops recording; both calls reset the totals.  Creates its
   events on the first call.  Errors: PV_ERR_INVALID_ARGUMENT for g == NULL,
   PV_ERR_CUDA if an event cannot be created. */
pv_status pv_grid_time_sweeps(pv_grid* g, int enable);

/* Waits for the recorded event pairs (host-synchronous) and returns, per
   sweep (index 0: density, 1: adjoint), the summed kernel time in
   milliseconds in ms[2] and the number of timed launches in launches[2]
   (host arrays; either may be NULL).  The totals then restart from zero. */
pv_status pv_grid_sweep_times(pv_grid* g, double* ms, int64_t* launches);

/* No-allocation variant of pv_sort_cells + pv_density for ONE periodic box.
   The paper has no counterpart; this exists for callers that may not
   allocate device memory while they run: an application whose memory pool
   owns all of the GPU's memory and forbids cudaMalloc behind its back, a
   plugin loaded into such a host, or a latency-critical loop that cannot take
   the device synchronisation and allocator locks of cudaMalloc/cudaFree.
   It computes the same rho, drho_dh and n_ngb as pv_sort_cells followed by
   pv_density on a one-box grid, with the same arguments' meaning and layout
   (pos device double [n][3], h device float [n], m device float [n] or NULL
   for m_uniform, outputs device float/int32 [n] in the caller's order; box
   [0, L)^3 with nc^3 cells; gamma <= 0 or NaN selects 1.825742).  flags_out, if not
   NULL, is a device uint32 that receives the PV_FLAG_* bits the kernels
   latched (0 = inputs valid; outputs are not written otherwise).
   Memory: every intermediate array lives in one fixed device array inside
   this library (about 15 MB, sized for the limits below) that each GPU
   loading the library keeps until the process exits; nothing is allocated
   or freed, by this library or by any library it calls.
   Limits: n <= PV_STATIC_MAX_PARTICLES and nc^3 <= PV_STATIC_MAX_CELLS;
   larger inputs return PV_ERR_TOO_LARGE before any work is queued.
   Every call looks up the current device's address of the array
   (cudaGetSymbolAddress, a host-side query: the address may change after
   cudaDeviceReset); the first call on a device may load the library's
   kernels there, so make it before any stream capture.  All calls share the one array: calls whose
   work overlaps on the GPU (other streams, other host threads) race and
   corrupt each other's results; serialise them. */
#define PV_STATIC_MAX_PARTICLES 65536
#define PV_STATIC_MAX_CELLS 4096
pv_status pv_density_static(const double* pos, const float* h, const float* m, float m_uniform,
                            int64_t n, double L, int32_t nc, double gamma, float* rho,
                            float* drho_dh, int32_t* n_ngb, uint32_t* flags_out, void* stream);

/* Static description of a status code (never NULL). */
const char* pv_status_str(pv_status s);

/* Text of the last CUDA error seen by this library on the calling thread. */
const char* pv_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PV_H */
