/*
 * pv_oracle.c -- plain, slow FP64 reference ("oracle") for the pseudo-Verlet
 * SPH density loop of Willis et al., "An Efficient SIMD Implementation of
 * Pseudo-Verlet Lists for Neighbour Interactions in Particle-Based Codes"
 * (arXiv:1804.06231).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * path.
 *
 * What is computed (all in double precision, periodic cube [0, L)^3,
 * minimum-image separations r_ij, support H_i = gamma * h_i):
 *
 *   rho_i      = sum_j m_j W(r_ij, H_i)                  (j runs over all, incl. i)
 *   drho_dh_i  = sum_j m_j dW/dh (r_ij, h_i)
 *   n_i        = #{ j != i : r_ij < H_i }
 *
 * with the 3D cubic spline of the workload,
 *   W(r, H) = H^-3 w(r/H),
 *   w(q) = (8/pi) * { 1 - 6 q^2 + 6 q^3    0 <= q < 1/2
 *                     2 (1 - q)^3          1/2 <= q < 1
 *                     0                    q >= 1 }.
 *
 * Three routes to the same sums (they agree up to summation order):
 *   or_density_brute  -- the plain O(N^2) definition;
 *   or_density_cells  -- the cell list of Section 1/2: every pair of particles
 *                        in neighbouring cells is tested (the naive pair loop
 *                        of Section 2, first listing);
 *   or_density_pv     -- the pseudo-Verlet list of Section 2 and Section 3.3:
 *                        per cell and per one of the 13 axes joining
 *                        neighbouring cell centres, particles are sorted by
 *                        their projection on the axis; a cell pair is swept
 *                        in sorted order and the inner loop over cell b stops
 *                        once the projected distance reaches the support of
 *                        the particle i of cell a.  Only the particles of a
 *                        that lie within the cell's largest support of b are
 *                        visited (the "first_a" trimming of Section 3.3).
 *
 * The adjoint of the density loop (not in the paper; it maps dL/drho and
 * dL/d(drho/dh) to dL/dx and dL/dh) comes by three routes as well:
 * or_backward_brute (definition), or_backward_cells (cell list) and
 * or_backward_pv (the pseudo-Verlet sweep with every reach widened to
 * max(H_i, Hmax_b), which the transposed term r < H_j needs).
 *
 * Readings of the paper that this file takes (the paper is silent on them):
 *   - the paper's cut-off "h" is the support H here; cells have edge >= H_max;
 *   - the interaction is the SPH density gather above;
 *   - cut-off test is strict: r < H_i;
 *   - n_i excludes j = i, rho_i and drho_dh_i include the self term;
 *   - gather form: particle i only collects from j with r_ij < H_i;
 *   - self-cell pairs use a two-sided window on the sorted axis (0,0,1);
 *   - the 13 axes are the vectors v in {-1,0,1}^3 that are lexicographically
 *     positive; a neighbour at -v uses the same sorted list read backwards;
 *   - particle offsets are taken from each cell's centre and the pair shift is
 *     the difference of the cell centres, which handles the periodic wrap
 *     (Section 3.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_NDIR 13
#define OR_BAND 1e-6 /* relative half-width of the cut-off band for n_i */

/* ------------------------------------------------------------------------ */
/* Cubic-spline kernel and its derivatives (functions of q = r/H).          */
/* ------------------------------------------------------------------------ */

double or_w(double q) {
  const double c = 8.0 / OR_PI;
  if (q < 0.5) return c * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
  if (q < 1.0) { double s = 1.0 - q; return c * 2.0 * s * s * s; }
  return 0.0;
}

double or_dw(double q) { /* dw/dq */
  const double c = 8.0 / OR_PI;
  if (q < 0.5) return c * (-12.0 * q + 18.0 * q * q);
  if (q < 1.0) { double s = 1.0 - q; return c * (-6.0 * s * s); }
  return 0.0;
}

double or_d2w(double q) { /* d2w/dq2 */
  const double c = 8.0 / OR_PI;
  if (q < 0.5) return c * (-12.0 + 36.0 * q);
  if (q < 1.0) return c * 12.0 * (1.0 - q);
  return 0.0;
}

/* w'(q)/q, written out so that q = 0 is finite. */
static double dw_over_q(double q) {
  const double c = 8.0 / OR_PI;
  if (q < 0.5) return c * (-12.0 + 18.0 * q);
  if (q < 1.0) { double s = 1.0 - q; return c * (-6.0 * s * s / q); }
  return 0.0;
}

/* (4 w'(q) + q w''(q)) / q, finite at q = 0. */
static double hr_over_q(double q) {
  const double c = 8.0 / OR_PI;
  if (q < 0.5) return c * (-60.0 + 108.0 * q);
  if (q < 1.0) { double s = 1.0 - q; return c * (-24.0 * s * s / q + 12.0 * s); }
  return 0.0;
}

/* W(r, H) */
double or_W(double r, double H) { return or_w(r / H) / (H * H * H); }

/* dW/dh at fixed r, with H = gamma h:  -(3 w + q w') / (h H^3) */
double or_W_h(double r, double h, double gamma) {
  double H = gamma * h, q = r / H;
  return -(3.0 * or_w(q) + q * or_dw(q)) / (h * H * H * H);
}

/* d2W/dh2:  (12 w + 8 q w' + q^2 w'') / (h^2 H^3) */
double or_W_hh(double r, double h, double gamma) {
  double H = gamma * h, q = r / H;
  return (12.0 * or_w(q) + 8.0 * q * or_dw(q) + q * q * or_d2w(q)) / (h * h * H * H * H);
}

/* dW/dr:  w' / H^4 */
double or_W_r(double r, double H) { double q = r / H; return or_dw(q) / (H * H * H * H); }

/* d/dr (dW/dh):  -(4 w' + q w'') / (h H^4) */
double or_W_hr(double r, double h, double gamma) {
  double H = gamma * h, q = r / H;
  return -(4.0 * or_dw(q) + q * or_d2w(q)) / (h * H * H * H * H);
}

/* ------------------------------------------------------------------------ */
/* Shared helpers                                                           */
/* ------------------------------------------------------------------------ */

static double wrap_coord(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y = 0.0;
  if (y < 0.0) y = 0.0;
  return y;
}

/* One gathered pair: accumulate i's sums for neighbour j at distance r. */
typedef struct {
  double rho, D, S;
  int32_t n, band;
} or_acc;

static void acc_pair(or_acc* a, double r, int same, double Hi, double hi, double mj,
                     double gamma) {
  if (!same && fabs(r - Hi) < OR_BAND * Hi) a->band++;
  if (r < Hi) {
    double wh = or_W_h(r, hi, gamma);
    a->rho += mj * or_W(r, Hi);
    a->D += mj * wh;
    a->S += mj * fabs(wh);
    if (!same) a->n++;
  }
}

static void store_acc(const or_acc* a, int64_t i, double* rho, double* D, int32_t* n,
                      double* S, int32_t* band) {
  rho[i] = a->rho;
  D[i] = a->D;
  n[i] = a->n;
  if (S) S[i] = a->S;
  if (band) band[i] = a->band;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

int or_max_threads(void) { return set_threads(0); }

/* ------------------------------------------------------------------------ */
/* 1. Brute force: the definition.                                          */
/* ------------------------------------------------------------------------ */

void or_density_brute(int64_t n, const double* pos, const double* h, const double* m,
                      double L, double gamma, double* rho, double* D, int32_t* nngb,
                      double* S, int32_t* band, int nthreads) {
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; i++) {
    or_acc a = {0, 0, 0, 0, 0};
    double Hi = gamma * h[i], hi = h[i];
    for (int64_t j = 0; j < n; j++) {
      double r2 = 0.0;
      for (int c = 0; c < 3; c++) {
        double d = pos[3 * i + c] - pos[3 * j + c];
        d -= L * nearbyint(d / L); /* minimum image */
        r2 += d * d;
      }
      acc_pair(&a, sqrt(r2), i == j, Hi, hi, m[j], gamma);
    }
    store_acc(&a, i, rho, D, nngb, S, band);
  }
}

/* ------------------------------------------------------------------------ */
/* 2. Cell grid (Section 1/2): cells of edge L/nc >= H_max, particles of a  */
/*    cell stored together, offsets from the cell centre.                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nc;
  double L, edge;
  int64_t ncell, n;
  int64_t* start;   /* [ncell+1] */
  int64_t* member;  /* [n]  original index, cell order, ascending within a cell */
  double* off;      /* [3n] offset from the cell centre, cell order */
  double* dist[OR_NDIR];   /* [n] per cell segment: sorted projections */
  int64_t* sidx[OR_NDIR];  /* [n] per cell segment: cell-order slot of each sorted entry */
  double* Hmax;     /* [ncell] largest support in the cell */
} or_grid;

/* The 13 axes: v in {-1,0,1}^3, lexicographically positive. */
static const int OR_V[OR_NDIR][3] = {
    {0, 0, 1}, {0, 1, -1}, {0, 1, 0}, {0, 1, 1}, {1, -1, -1}, {1, -1, 0}, {1, -1, 1},
    {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1}, {1, 1, 0}, {1, 1, 1}};

static int64_t cell_id(const or_grid* g, int cx, int cy, int cz) {
  int nc = g->nc;
  cx = ((cx % nc) + nc) % nc;
  cy = ((cy % nc) + nc) % nc;
  cz = ((cz % nc) + nc) % nc;
  return ((int64_t)cx * nc + cy) * nc + cz;
}

typedef struct { double d; int64_t orig; int64_t slot; } or_key;

static int key_cmp(const void* a, const void* b) {
  const or_key* x = (const or_key*)a;
  const or_key* y = (const or_key*)b;
  if (x->d < y->d) return -1;
  if (x->d > y->d) return 1;
  return (x->orig > y->orig) - (x->orig < y->orig);
}

static void grid_free(or_grid* g) {
  free(g->start); free(g->member); free(g->off); free(g->Hmax);
  for (int k = 0; k < OR_NDIR; k++) { free(g->dist[k]); free(g->sidx[k]); }
  memset(g, 0, sizeof(*g));
}

/* Bins the particles and, if with_sort, builds the 13 sorted projections. */
static int grid_build(or_grid* g, int64_t n, const double* pos, const double* h, double L,
                      int nc, double gamma, int with_sort) {
  memset(g, 0, sizeof(*g));
  g->nc = nc; g->L = L; g->edge = L / nc; g->n = n;
  g->ncell = (int64_t)nc * nc * nc;
  g->start = calloc((size_t)g->ncell + 1, sizeof(int64_t));
  g->member = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  g->off = malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
  g->Hmax = calloc((size_t)g->ncell, sizeof(double));
  int64_t* cid = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!g->start || !g->member || !g->off || !g->Hmax || !cid) { free(cid); grid_free(g); return -1; }

  for (int64_t i = 0; i < n; i++) {
    int c3[3];
    for (int c = 0; c < 3; c++) {
      double x = wrap_coord(pos[3 * i + c], L);
      int ci = (int)floor(x / g->edge);
      if (ci >= nc) ci = nc - 1;
      if (ci < 0) ci = 0;
      c3[c] = ci;
    }
    cid[i] = cell_id(g, c3[0], c3[1], c3[2]);
    g->start[cid[i] + 1]++;
  }
  for (int64_t c = 0; c < g->ncell; c++) g->start[c + 1] += g->start[c];
  int64_t* fill = calloc((size_t)g->ncell, sizeof(int64_t));
  if (!fill) { free(cid); grid_free(g); return -1; }
  for (int64_t i = 0; i < n; i++) { /* ascending original index within a cell */
    int64_t c = cid[i], s = g->start[c] + fill[c]++;
    g->member[s] = i;
    int cx = (int)(c / ((int64_t)nc * nc)), cy = (int)((c / nc) % nc), cz = (int)(c % nc);
    int c3[3] = {cx, cy, cz};
    for (int d = 0; d < 3; d++) {
      double centre = (c3[d] + 0.5) * g->edge;
      g->off[3 * s + d] = wrap_coord(pos[3 * i + d], L) - centre;
    }
    double Hi = gamma * h[i];
    if (Hi > g->Hmax[c]) g->Hmax[c] = Hi;
  }
  free(fill);
  free(cid);
  if (!with_sort) return 0;

  for (int k = 0; k < OR_NDIR; k++) {
    g->dist[k] = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    g->sidx[k] = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->dist[k] || !g->sidx[k]) { grid_free(g); return -1; }
  }
  int fail = 0;
#pragma omp parallel
  {
    int64_t cap = 0;
    or_key* keys = NULL;
#pragma omp for schedule(dynamic, 16)
    for (int64_t c = 0; c < g->ncell; c++) {
      int64_t s0 = g->start[c], cnt = g->start[c + 1] - s0;
      if (cnt > cap) {
        free(keys);
        cap = cnt;
        keys = malloc((size_t)cap * sizeof(or_key));
        if (!keys) { fail = 1; cap = 0; }
      }
      if (!keys) continue;
      for (int k = 0; k < OR_NDIR; k++) {
        double nv = sqrt((double)(OR_V[k][0] * OR_V[k][0] + OR_V[k][1] * OR_V[k][1] +
                                  OR_V[k][2] * OR_V[k][2]));
        for (int64_t t = 0; t < cnt; t++) {
          const double* o = g->off + 3 * (s0 + t);
          keys[t].d = (o[0] * OR_V[k][0] + o[1] * OR_V[k][1] + o[2] * OR_V[k][2]) / nv;
          keys[t].orig = g->member[s0 + t];
          keys[t].slot = s0 + t;
        }
        qsort(keys, (size_t)cnt, sizeof(or_key), key_cmp);
        for (int64_t t = 0; t < cnt; t++) {
          g->dist[k][s0 + t] = keys[t].d;
          g->sidx[k][s0 + t] = keys[t].slot;
        }
      }
    }
    free(keys);
  }
  return fail ? -1 : 0;
}

/* Distance between cell-order slots si (in cell a) and sj (in cell b), b = a + o. */
static double pair_r(const or_grid* g, int64_t si, int64_t sj, const int o[3]) {
  double r2 = 0.0;
  for (int c = 0; c < 3; c++) {
    double d = g->off[3 * si + c] - g->off[3 * sj + c] - o[c] * g->edge;
    r2 += d * d;
  }
  return sqrt(r2);
}

static void cell_coords(const or_grid* g, int64_t c, int c3[3]) {
  c3[0] = (int)(c / ((int64_t)g->nc * g->nc));
  c3[1] = (int)((c / g->nc) % g->nc);
  c3[2] = (int)(c % g->nc);
}

/* ------------------------------------------------------------------------ */
/* 3. Cell list: all pairs of particles in the 27 neighbouring cells.       */
/* ------------------------------------------------------------------------ */

int or_density_cells(int64_t n, const double* pos, const double* h, const double* m, double L,
                     int nc, double gamma, double* rho, double* D, int32_t* nngb, double* S,
                     int32_t* band, int nthreads) {
  if (nc < 3) return -2;
  set_threads(nthreads);
  or_grid g;
  if (grid_build(&g, n, pos, h, L, nc, gamma, 0)) return -1;
  for (int64_t c = 0; c < g.ncell; c++)
    if (g.Hmax[c] * (1.0 + OR_BAND) > g.edge) { grid_free(&g); return -3; }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t a = 0; a < g.ncell; a++) {
    int ca[3];
    cell_coords(&g, a, ca);
    for (int64_t si = g.start[a]; si < g.start[a + 1]; si++) {
      int64_t i = g.member[si];
      double Hi = gamma * h[i], hi = h[i];
      or_acc acc = {0, 0, 0, 0, 0};
      for (int ox = -1; ox <= 1; ox++)
        for (int oy = -1; oy <= 1; oy++)
          for (int oz = -1; oz <= 1; oz++) {
            int o[3] = {ox, oy, oz};
            int64_t b = cell_id(&g, ca[0] + ox, ca[1] + oy, ca[2] + oz);
            for (int64_t sj = g.start[b]; sj < g.start[b + 1]; sj++) {
              int64_t j = g.member[sj];
              acc_pair(&acc, pair_r(&g, si, sj, o), i == j, Hi, hi, m[j], gamma);
            }
          }
      store_acc(&acc, i, rho, D, nngb, S, band);
    }
  }
  grid_free(&g);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 4. Pseudo-Verlet list (Section 2 and Section 3.3).                        */
/*    counters[4][2]: per class (0 self, 1 face, 2 edge, 3 corner) the       */
/*    number of distance computations inside the sorted windows ("candidates")*/
/*    and the number of pairs j != i with r < H_i ("interactions").          */
/* ------------------------------------------------------------------------ */

int or_density_pv(int64_t n, const double* pos, const double* h, const double* m, double L,
                  int nc, double gamma, double* rho, double* D, int32_t* nngb, double* S,
                  int32_t* band, int64_t* counters, int nthreads) {
  if (nc < 3) return -2;
  set_threads(nthreads);
  or_grid g;
  if (grid_build(&g, n, pos, h, L, nc, gamma, 1)) return -1;
  for (int64_t c = 0; c < g.ncell; c++)
    if (g.Hmax[c] * (1.0 + OR_BAND) > g.edge) { grid_free(&g); return -3; }

  or_acc* acc = calloc((size_t)(n > 0 ? n : 1), sizeof(or_acc)); /* by cell-order slot */
  if (!acc) { grid_free(&g); return -1; }
  int64_t cnt_tot[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};

#pragma omp parallel
  {
    int64_t cnt[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma omp for schedule(dynamic, 4)
    for (int64_t a = 0; a < g.ncell; a++) {
      int ca[3];
      cell_coords(&g, a, ca);
      int64_t a0 = g.start[a], na = g.start[a + 1] - a0;

      /* Self interaction: two-sided window on the sorted axis (0,0,1). */
      {
        const double* dd = g.dist[0] + a0;
        const int64_t* ss = g.sidx[0] + a0;
        const int o[3] = {0, 0, 0};
        for (int64_t t = 0; t < na; t++) {
          int64_t si = ss[t], i = g.member[si];
          double Hi = gamma * h[i], hi = h[i];
          double Hb = Hi * (1.0 + OR_BAND); /* band pairs are looked at, not counted */
          or_acc* ai = &acc[si];
          for (int64_t u = t; u >= 0 && dd[u] > dd[t] - Hb; u--) {
            if (dd[u] > dd[t] - Hi) cnt[0][0]++;
            int64_t sj = ss[u], j = g.member[sj];
            double r = pair_r(&g, si, sj, o);
            if (r < Hi && j != i) cnt[0][1]++;
            acc_pair(ai, r, i == j, Hi, hi, m[j], gamma);
          }
          for (int64_t u = t + 1; u < na && dd[u] < dd[t] + Hb; u++) {
            if (dd[u] < dd[t] + Hi) cnt[0][0]++;
            int64_t sj = ss[u], j = g.member[sj];
            double r = pair_r(&g, si, sj, o);
            if (r < Hi && j != i) cnt[0][1]++;
            acc_pair(ai, r, i == j, Hi, hi, m[j], gamma);
          }
        }
      }

      /* Pair interactions: for each axis k and side s, cell b = a + s v_k
         gathers into a.  Projections along u = s v_k/|v_k| in a's frame:
           d_i = s dist_a[k][t],   d_j = s dist_b[k][t] + |v_k| edge,
         so b's particles all lie beyond a's along u; ascending order along u
         is the stored order for s = +1 and the reverse for s = -1. */
      for (int k = 0; k < OR_NDIR; k++) {
        int v2 = OR_V[k][0] * OR_V[k][0] + OR_V[k][1] * OR_V[k][1] + OR_V[k][2] * OR_V[k][2];
        int cls = v2; /* 1 face, 2 edge, 3 corner */
        double shift = sqrt((double)v2) * g.edge;
        for (int s = 1; s >= -1; s -= 2) {
          int o[3] = {s * OR_V[k][0], s * OR_V[k][1], s * OR_V[k][2]};
          int64_t b = cell_id(&g, ca[0] + o[0], ca[1] + o[1], ca[2] + o[2]);
          int64_t b0 = g.start[b], nb = g.start[b + 1] - b0;
          if (na == 0 || nb == 0) continue;
          /* t-th particle of a cell in ascending order along u */
#define A_POS(t) (s > 0 ? a0 + (t) : a0 + na - 1 - (t))
#define B_POS(t) (s > 0 ? b0 + (t) : b0 + nb - 1 - (t))
          double db_first = s * g.dist[k][B_POS(0)] + shift;
          /* first_a: particles of a beyond this one (in ascending order) can
             reach b with the cell's largest support; the ones before cannot. */
          int64_t first_a = na;
          while (first_a > 0 && s * g.dist[k][A_POS(first_a - 1)] + g.Hmax[a] > db_first)
            first_a--;
          for (int64_t t = first_a; t < na; t++) {
            int64_t si = g.sidx[k][A_POS(t)], i = g.member[si];
            double Hi = gamma * h[i], hi = h[i];
            double di = s * g.dist[k][A_POS(t)];
            double Hb = Hi * (1.0 + OR_BAND);
            or_acc* ai = &acc[si];
            /* sweep b from the interface; stop once the projected gap reaches H_i */
            for (int64_t u = 0; u < nb; u++) {
              double dj = s * g.dist[k][B_POS(u)] + shift;
              if (!(dj < di + Hb)) break;
              if (dj < di + Hi) cnt[cls][0]++;
              int64_t sj = g.sidx[k][B_POS(u)], j = g.member[sj];
              double r = pair_r(&g, si, sj, o);
              if (r < Hi) cnt[cls][1]++;
              acc_pair(ai, r, 0, Hi, hi, m[j], gamma);
            }
          }
#undef A_POS
#undef B_POS
        }
      }
    }
#pragma omp critical
    for (int c = 0; c < 4; c++) { cnt_tot[c][0] += cnt[c][0]; cnt_tot[c][1] += cnt[c][1]; }
  }
  for (int64_t s = 0; s < n; s++) store_acc(&acc[s], g.member[s], rho, D, nngb, S, band);
  if (counters)
    for (int c = 0; c < 4; c++) { counters[2 * c] = cnt_tot[c][0]; counters[2 * c + 1] = cnt_tot[c][1]; }
  free(acc);
  grid_free(&g);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 5. Adjoint.  With g_i = dL/drho_i and k_i = dL/d(drho/dh)_i:              */
/*   dL/dh_i = g_i drho_dh_i + k_i sum_j m_j d2W/dh2(r_ij, h_i)              */
/*   dL/dx_i = sum_{j != i} (x_i - x_j)/r_ij [ m_j (g_i W_r(r,H_i)           */
/*             + k_i W_hr(r,h_i)) [r < H_i] + m_i (g_j W_r(r,H_j)             */
/*             + k_j W_hr(r,h_j)) [r < H_j] ]                                 */
/* (x_i - x_j)/r is multiplied out analytically so r = 0 contributes 0.      */
/* ------------------------------------------------------------------------ */

typedef struct { double gx, gy, gz, gh; } or_gacc;

static void adj_pair(or_gacc* a, const double d[3], double r, int same, double hi, double hj,
                     double mi, double mj, double gi, double ki, double gj, double kj,
                     double gamma) {
  double Hi = gamma * hi, Hj = gamma * hj;
  if (r < Hi) {
    double q = r / Hi;
    double w = or_w(q), dw = or_dw(q), d2w = or_d2w(q);
    double Whh = (12.0 * w + 8.0 * q * dw + q * q * d2w) / (hi * hi * Hi * Hi * Hi);
    double Wh = -(3.0 * w + q * dw) / (hi * Hi * Hi * Hi);
    a->gh += gi * mj * Wh + ki * mj * Whh;
    if (!same) {
      double Wr_r = dw_over_q(q) / (Hi * Hi * Hi * Hi * Hi);
      double Whr_r = -hr_over_q(q) / (hi * Hi * Hi * Hi * Hi * Hi);
      double f = mj * (gi * Wr_r + ki * Whr_r);
      a->gx += f * d[0]; a->gy += f * d[1]; a->gz += f * d[2];
    }
  }
  if (!same && r < Hj) {
    double q = r / Hj;
    double Wr_r = dw_over_q(q) / (Hj * Hj * Hj * Hj * Hj);
    double Whr_r = -hr_over_q(q) / (hj * Hj * Hj * Hj * Hj * Hj);
    double f = mi * (gj * Wr_r + kj * Whr_r);
    a->gx += f * d[0]; a->gy += f * d[1]; a->gz += f * d[2];
  }
}

void or_backward_brute(int64_t n, const double* pos, const double* h, const double* m, double L,
                       double gamma, const double* g_rho, const double* g_D, double* g_pos,
                       double* g_h, int nthreads) {
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; i++) {
    or_gacc a = {0, 0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
      double d[3], r2 = 0.0;
      for (int c = 0; c < 3; c++) {
        d[c] = pos[3 * i + c] - pos[3 * j + c];
        d[c] -= L * nearbyint(d[c] / L);
        r2 += d[c] * d[c];
      }
      adj_pair(&a, d, sqrt(r2), i == j, h[i], h[j], m[i], m[j], g_rho[i], g_D[i], g_rho[j],
               g_D[j], gamma);
    }
    g_pos[3 * i] = a.gx; g_pos[3 * i + 1] = a.gy; g_pos[3 * i + 2] = a.gz;
    g_h[i] = a.gh;
  }
}

int or_backward_cells(int64_t n, const double* pos, const double* h, const double* m, double L,
                      int nc, double gamma, const double* g_rho, const double* g_D,
                      double* g_pos, double* g_h, int nthreads) {
  if (nc < 3) return -2;
  set_threads(nthreads);
  or_grid g;
  if (grid_build(&g, n, pos, h, L, nc, gamma, 0)) return -1;
  for (int64_t c = 0; c < g.ncell; c++)
    if (g.Hmax[c] > g.edge) { grid_free(&g); return -3; }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t a = 0; a < g.ncell; a++) {
    int ca[3];
    cell_coords(&g, a, ca);
    for (int64_t si = g.start[a]; si < g.start[a + 1]; si++) {
      int64_t i = g.member[si];
      or_gacc acc = {0, 0, 0, 0};
      for (int ox = -1; ox <= 1; ox++)
        for (int oy = -1; oy <= 1; oy++)
          for (int oz = -1; oz <= 1; oz++) {
            int o[3] = {ox, oy, oz};
            int64_t b = cell_id(&g, ca[0] + ox, ca[1] + oy, ca[2] + oz);
            for (int64_t sj = g.start[b]; sj < g.start[b + 1]; sj++) {
              int64_t j = g.member[sj];
              double d[3], r2 = 0.0;
              for (int c = 0; c < 3; c++) {
                d[c] = g.off[3 * si + c] - g.off[3 * sj + c] - o[c] * g.edge;
                r2 += d[c] * d[c];
              }
              adj_pair(&acc, d, sqrt(r2), i == j, h[i], h[j], m[i], m[j], g_rho[i], g_D[i],
                       g_rho[j], g_D[j], gamma);
            }
          }
      g_pos[3 * i] = acc.gx; g_pos[3 * i + 1] = acc.gy; g_pos[3 * i + 2] = acc.gz;
      g_h[i] = acc.gh;
    }
  }
  grid_free(&g);
  return 0;
}

/* The adjoint by the pseudo-Verlet sweep of the density (Section 2 second  */
/* listing, Section 3.3 trimming), with every reach widened to cover the    */
/* transposed term: a pair (i, j) contributes while r < max(H_i, H_j), and  */
/* its projected separation is at most r, so particle i of cell a sweeps    */
/* the sorted list of b up to max(H_i, Hmax_b) beyond d_i, and a is trimmed */
/* with max(Hmax_a, Hmax_b).  Each candidate is then decided exactly by     */
/* adj_pair (r < H_i own, r < H_j transposed).  Same result as the cell      */
/* list up to summation order, at the cost of the sweep's candidates.        */
int or_backward_pv(int64_t n, const double* pos, const double* h, const double* m, double L,
                   int nc, double gamma, const double* g_rho, const double* g_D,
                   double* g_pos, double* g_h, int nthreads) {
  if (nc < 3) return -2;
  set_threads(nthreads);
  or_grid g;
  if (grid_build(&g, n, pos, h, L, nc, gamma, 1)) return -1;
  for (int64_t c = 0; c < g.ncell; c++)
    if (g.Hmax[c] > g.edge) { grid_free(&g); return -3; }
  or_gacc* acc = calloc((size_t)(n > 0 ? n : 1), sizeof(or_gacc)); /* by cell-order slot */
  if (!acc) { grid_free(&g); return -1; }

#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t a = 0; a < g.ncell; a++) {
    int ca[3];
    cell_coords(&g, a, ca);
    const int64_t a0 = g.start[a], na = g.start[a + 1] - a0;
    if (na == 0) continue;
    /* one candidate pair: cell-order slots si (cell a) and sj (cell a + o) */
#define ADJ(si_, sj_, o_)                                                             \
    do {                                                                              \
      const int64_t i_ = g.member[si_], j_ = g.member[sj_];                           \
      double d_[3], r2_ = 0.0;                                                        \
      for (int c_ = 0; c_ < 3; c_++) {                                                \
        d_[c_] = g.off[3 * (si_) + c_] - g.off[3 * (sj_) + c_] - (o_)[c_] * g.edge;   \
        r2_ += d_[c_] * d_[c_];                                                       \
      }                                                                               \
      adj_pair(&acc[si_], d_, sqrt(r2_), i_ == j_, h[i_], h[j_], m[i_], m[j_],        \
               g_rho[i_], g_D[i_], g_rho[j_], g_D[j_], gamma);                        \
    } while (0)

    /* self: two-sided window on the sorted axis (0,0,1), reach max(H_i, Hmax_a) */
    {
      const double* dd = g.dist[0] + a0;
      const int64_t* ss = g.sidx[0] + a0;
      const int o[3] = {0, 0, 0};
      for (int64_t t = 0; t < na; t++) {
        const int64_t si = ss[t];
        const double R = fmax(gamma * h[g.member[si]], g.Hmax[a]);
        for (int64_t u = t; u >= 0 && dd[u] > dd[t] - R; u--) ADJ(si, ss[u], o);
        for (int64_t u = t + 1; u < na && dd[u] < dd[t] + R; u++) ADJ(si, ss[u], o);
      }
    }
    /* pairs: b = a + s v_k, projections as in or_density_pv */
    for (int k = 0; k < OR_NDIR; k++) {
      const int v2 = OR_V[k][0] * OR_V[k][0] + OR_V[k][1] * OR_V[k][1] + OR_V[k][2] * OR_V[k][2];
      const double shift = sqrt((double)v2) * g.edge;
      for (int s = 1; s >= -1; s -= 2) {
        const int o[3] = {s * OR_V[k][0], s * OR_V[k][1], s * OR_V[k][2]};
        const int64_t b = cell_id(&g, ca[0] + o[0], ca[1] + o[1], ca[2] + o[2]);
        const int64_t b0 = g.start[b], nb = g.start[b + 1] - b0;
        if (nb == 0) continue;
#define A_POS(t) (s > 0 ? a0 + (t) : a0 + na - 1 - (t))
#define B_POS(t) (s > 0 ? b0 + (t) : b0 + nb - 1 - (t))
        const double db_first = s * g.dist[k][B_POS(0)] + shift;
        const double reach_ab = fmax(g.Hmax[a], g.Hmax[b]);
        int64_t first_a = na;
        while (first_a > 0 && s * g.dist[k][A_POS(first_a - 1)] + reach_ab > db_first) first_a--;
        for (int64_t t = first_a; t < na; t++) {
          const int64_t si = g.sidx[k][A_POS(t)];
          const double R = fmax(gamma * h[g.member[si]], g.Hmax[b]);
          const double di = s * g.dist[k][A_POS(t)];
          for (int64_t u = 0; u < nb; u++) {
            const double dj = s * g.dist[k][B_POS(u)] + shift;
            if (!(dj < di + R)) break;
            ADJ(si, g.sidx[k][B_POS(u)], o);
          }
        }
#undef A_POS
#undef B_POS
      }
    }
#undef ADJ
  }
  for (int64_t sl = 0; sl < n; sl++) {
    const int64_t i = g.member[sl];
    g_pos[3 * i] = acc[sl].gx; g_pos[3 * i + 1] = acc[sl].gy; g_pos[3 * i + 2] = acc[sl].gz;
    g_h[i] = acc[sl].gh;
  }
  free(acc);
  grid_free(&g);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 6. Central finite difference of                                          */
/*      L = sum_i w_i (rho_i - 1)^2 + sum_i v_i drho_dh_i                    */
/*    with respect to x_p[comp] (comp = 0, 1, 2) or h_p (comp = 3).          */
/*    Only the sums that depend on the perturbed quantity are re-evaluated;  */
/*    every other term of L is identical in L(+) and L(-) and cancels.       */
/* ------------------------------------------------------------------------ */

static double min_image_r(const double* a, const double* b, double L) {
  double r2 = 0.0;
  for (int c = 0; c < 3; c++) {
    double d = a[c] - b[c];
    d -= L * nearbyint(d / L);
    r2 += d * d;
  }
  return sqrt(r2);
}

double or_fd_loss(int64_t n, const double* pos, const double* h, const double* m, double L,
                  double gamma, const double* wgt, const double* vgt, int64_t p, int comp,
                  double delta) {
  double Hmax = 0.0;
  for (int64_t i = 0; i < n; i++) Hmax = fmax(Hmax, gamma * h[i]);
  Hmax = fmax(Hmax, gamma * (h[p] + fabs(delta)));
  double reach = 2.0 * Hmax + 4.0 * fabs(delta);
  int64_t* J = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* A = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!J || !A) { free(J); free(A); return NAN; }
  int64_t nJ = 0, nA = 0;
  for (int64_t i = 0; i < n; i++) {
    double r = min_image_r(pos + 3 * i, pos + 3 * p, L);
    if (i == p || r < reach) J[nJ++] = i;
    /* sums of i that contain x_p: i = p, or p within i's support (either side) */
    if (comp < 3 && (i == p || r < gamma * h[i] + 2.0 * fabs(delta))) A[nA++] = i;
  }
  if (comp == 3) A[nA++] = p; /* h_p only enters rho_p and drho_dh_p */
  double f[2];
  for (int s = 0; s < 2; s++) {
    double sg = s == 0 ? 1.0 : -1.0;
    double xp[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
    double hp = h[p];
    if (comp < 3) xp[comp] += sg * delta; else hp += sg * delta;
    double acc = 0.0;
    for (int64_t t = 0; t < nA; t++) {
      int64_t i = A[t];
      const double* xi = (i == p) ? xp : pos + 3 * i;
      double hi = (i == p) ? hp : h[i];
      double Hi = gamma * hi, rho = 0.0, D = 0.0;
      for (int64_t u = 0; u < nJ; u++) {
        int64_t j = J[u];
        const double* xj = (j == p) ? xp : pos + 3 * j;
        double r = min_image_r(xi, xj, L);
        if (r < Hi) {
          rho += m[j] * or_W(r, Hi);
          D += m[j] * or_W_h(r, hi, gamma);
        }
      }
      acc += wgt[i] * (rho - 1.0) * (rho - 1.0) + vgt[i] * D;
    }
    f[s] = acc;
  }
  free(J);
  free(A);
  return (f[0] - f[1]) / (2.0 * delta);
}

/* ------------------------------------------------------------------------ */
/* 7. Counts of the adjoint sweep: per particle i and neighbour cell, the    */
/*    particles j of the sorted window with projected distance below         */
/*    max(H_i, H_j) ("candidates") and the pairs with r_ij < max(H_i, H_j)   */
/*    (j = i included).  out[0] = candidates, out[1] = pairs.                */
/* ------------------------------------------------------------------------ */

int or_adjoint_counts(int64_t n, const double* pos, const double* h, double L, int nc,
                      double gamma, int64_t* out, int nthreads) {
  if (nc < 3) return -2;
  set_threads(nthreads);
  or_grid g;
  if (grid_build(&g, n, pos, h, L, nc, gamma, 1)) return -1;
  for (int64_t c = 0; c < g.ncell; c++) /* the 27-cell stencil needs H <= edge */
    if (g.Hmax[c] * (1.0 + OR_BAND) > g.edge) { grid_free(&g); return -3; }
  int64_t cand = 0, pairs = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : cand, pairs)
  for (int64_t a = 0; a < g.ncell; a++) {
    int ca[3];
    cell_coords(&g, a, ca);
    int64_t a0 = g.start[a], na = g.start[a + 1] - a0;
    for (int k = 0; k < OR_NDIR; k++) {
      int v2 = OR_V[k][0] * OR_V[k][0] + OR_V[k][1] * OR_V[k][1] + OR_V[k][2] * OR_V[k][2];
      double shift = sqrt((double)v2) * g.edge;
      for (int s = 1; s >= -1; s -= 2) {
        int o[3] = {s * OR_V[k][0], s * OR_V[k][1], s * OR_V[k][2]};
        int64_t b = cell_id(&g, ca[0] + o[0], ca[1] + o[1], ca[2] + o[2]);
        int64_t b0 = g.start[b], nb = g.start[b + 1] - b0;
        for (int64_t t = 0; t < na; t++) {
          int64_t pa = s > 0 ? a0 + t : a0 + na - 1 - t;
          int64_t si = g.sidx[k][pa], i = g.member[si];
          double di = s * g.dist[k][pa], Hi = gamma * h[i];
          for (int64_t u = 0; u < nb; u++) {
            int64_t pb = s > 0 ? b0 + u : b0 + nb - 1 - u;
            double dj = s * g.dist[k][pb] + shift;
            if (dj - di >= g.Hmax[b] && dj - di >= Hi) break;
            int64_t sj = g.sidx[k][pb], j = g.member[sj];
            double R = fmax(Hi, gamma * h[j]);
            if (dj - di < R) {
              cand++;
              if (pair_r(&g, si, sj, o) < R) pairs++;
            }
          }
        }
      }
    }
    /* self cell: two-sided window on axis (0,0,1) */
    const int o0[3] = {0, 0, 0};
    for (int64_t t = 0; t < na; t++) {
      int64_t si = g.sidx[0][a0 + t], i = g.member[si];
      double di = g.dist[0][a0 + t], Hi = gamma * h[i];
      for (int64_t u = 0; u < na; u++) {
        int64_t sj = g.sidx[0][a0 + u], j = g.member[sj];
        double R = fmax(Hi, gamma * h[j]);
        if (fabs(g.dist[0][a0 + u] - di) < R) {
          cand++;
          if (pair_r(&g, si, sj, o0) < R) pairs++;
        }
      }
    }
  }
  out[0] = cand;
  out[1] = pairs;
  grid_free(&g);
  return 0;
}
