/*
 * Seeded synthetic EM-like image stacks (uint8), used as input by both the
 * CUDA solver's tests/benchmark and the CPU oracle's tests.  This file holds
 * no arithmetic of the gradient-domain method itself: it only draws pixels.
 *
 * The paper's own data (a registered serial-section EM stack, Sec. 5) is not
 * available, so this generator stands in for it with the structure that the
 * method reacts to (Sec. 1, Fig. 1):
 *   - a Voronoi cell mosaic per slice: bright cell interiors, dark 2-px-wide
 *     membranes along the bisectors of the two nearest seeds; the seeds drift
 *     smoothly from slice to slice, so structure is continuous along z;
 *   - per-slice photometric distortion (gain, offset, linear illumination
 *     ramp) that is independent from slice to slice: the inter-slice
 *     discontinuities the anisotropic diffusion step removes;
 *   - per-pixel Gaussian noise.
 *
 * Randomness: a counter-based generator, SplitMix64 (G. Steele, D. Lea,
 * C. Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
 * used as a hash of (seed, stream, counter).  Every value is a pure function of
 * the seeds and the global voxel / cell / slice index, so any window of a
 * stack can be generated on its own and agrees with the full stack.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GDS_OK 0
#define GDS_ERR_ARG 1
#define GDS_ERR_OOM 3

/* ---- SplitMix64 finaliser, used as a hash ---- */
static inline uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum { ST_CELL = 1, ST_SLICE = 2, ST_NOISE = 3 };

static inline uint64_t h3(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return sm64(sm64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + ctr);
}
/* uniform in [0,1) with 53 random bits */
static inline double u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }
/* uniform in (0,1] */
static inline double u01_open0(uint64_t h) { return ((double)(h >> 11) + 1.0) * 0x1.0p-53; }

static const double TWO_PI = 6.283185307179586476925286766559;

/* Standard normal from two counters (Box-Muller, cosine branch). */
static inline double gauss(uint64_t seed, uint64_t stream, uint64_t ctr) {
  double a = u01_open0(h3(seed, stream, 2 * ctr));
  double b = u01(h3(seed, stream, 2 * ctr + 1));
  return sqrt(-2.0 * log(a)) * cos(TWO_PI * b);
}

/* Per-cell parameters: 12 counters per cell in stream ST_CELL. */
typedef struct {
  double px, py;     /* position at z = 0 */
  double vx, vy;     /* linear drift, px per slice, |v| <= 0.3 */
  double ax, ay;     /* sinusoidal wobble amplitude vector, |a| <= 2 */
  double w, phi;     /* wobble angular frequency 2*pi/T (T ~ U(20,60)), phase */
  double inner, memb;/* interior ~ N(160,15), membrane ~ N(50,10) */
} cell_t;

static void make_cell(cell_t *c, uint64_t seed, int NX, int NY, uint64_t i) {
  uint64_t b = i * 16;
  c->px = u01(h3(seed, ST_CELL, b + 0)) * NX;
  c->py = u01(h3(seed, ST_CELL, b + 1)) * NY;
  double sa = TWO_PI * u01(h3(seed, ST_CELL, b + 2));
  double sr = 0.3 * sqrt(u01(h3(seed, ST_CELL, b + 3)));
  c->vx = sr * cos(sa);
  c->vy = sr * sin(sa);
  double wa = TWO_PI * u01(h3(seed, ST_CELL, b + 4));
  double wr = 2.0 * u01(h3(seed, ST_CELL, b + 5));
  c->ax = wr * cos(wa);
  c->ay = wr * sin(wa);
  double T = 20.0 + 40.0 * u01(h3(seed, ST_CELL, b + 6));
  c->w = TWO_PI / T;
  c->phi = TWO_PI * u01(h3(seed, ST_CELL, b + 7));
  c->inner = 160.0 + 15.0 * gauss(seed, ST_CELL, b / 2 + 4);
  c->memb = 50.0 + 10.0 * gauss(seed, ST_CELL, b / 2 + 5);
}

/* Per-slice photometric distortion in stream ST_SLICE. */
typedef struct { double gain, offset, ramp_amp, ct, st, umin, uinv; } slice_t;

static void make_slice(slice_t *s, uint64_t pseed, int NX, int NY, uint64_t z) {
  uint64_t b = z * 8;
  s->gain = 0.8 + 0.4 * u01(h3(pseed, ST_SLICE, b + 0));
  s->offset = -20.0 + 40.0 * u01(h3(pseed, ST_SLICE, b + 1));
  s->ramp_amp = -15.0 + 30.0 * u01(h3(pseed, ST_SLICE, b + 2));
  double th = TWO_PI * u01(h3(pseed, ST_SLICE, b + 3));
  s->ct = cos(th);
  s->st = sin(th);
  /* projection u = x cos + y sin over the pixel-centre corners of the slice */
  double u[4] = {0.0, (NX - 1) * s->ct, (NY - 1) * s->st, (NX - 1) * s->ct + (NY - 1) * s->st};
  double lo = u[0], hi = u[0];
  for (int k = 1; k < 4; ++k) { if (u[k] < lo) lo = u[k]; if (u[k] > hi) hi = u[k]; }
  s->umin = lo;
  s->uinv = (hi > lo) ? 1.0 / (hi - lo) : 0.0;
}

typedef struct {
  int nb_x, nb_y;     /* bucket grid */
  double bsz;         /* bucket edge, px */
  int *start;         /* nb_x*nb_y + 1 offsets */
  int *idx;           /* cell ids sorted by bucket */
  double *x, *y;      /* cell positions at this slice */
} grid_t;

static int grid_build(grid_t *g, const cell_t *cells, int ncells, int NX, int NY, double z) {
  double bsz = sqrt((double)NX * (double)NY / (double)ncells);
  if (bsz < 4.0) bsz = 4.0;
  g->bsz = bsz;
  g->nb_x = (int)ceil(NX / bsz);
  g->nb_y = (int)ceil(NY / bsz);
  if (g->nb_x < 1) g->nb_x = 1;
  if (g->nb_y < 1) g->nb_y = 1;
  int nb = g->nb_x * g->nb_y;
  g->start = (int *)calloc((size_t)nb + 1, sizeof(int));
  g->idx = (int *)malloc(sizeof(int) * (size_t)ncells);
  g->x = (double *)malloc(sizeof(double) * (size_t)ncells);
  g->y = (double *)malloc(sizeof(double) * (size_t)ncells);
  int *bk = (int *)malloc(sizeof(int) * (size_t)ncells);
  if (!g->start || !g->idx || !g->x || !g->y || !bk) { free(bk); return GDS_ERR_OOM; }
  for (int c = 0; c < ncells; ++c) {
    const cell_t *q = &cells[c];
    double s = sin(q->w * z + q->phi);
    double x = q->px + q->vx * z + q->ax * s;
    double y = q->py + q->vy * z + q->ay * s;
    g->x[c] = x;
    g->y[c] = y;
    int bx = (int)floor(x / bsz), by = (int)floor(y / bsz);
    if (bx < 0) bx = 0;
    if (bx >= g->nb_x) bx = g->nb_x - 1;
    if (by < 0) by = 0;
    if (by >= g->nb_y) by = g->nb_y - 1;
    bk[c] = by * g->nb_x + bx;
    g->start[bk[c] + 1]++;
  }
  for (int b = 0; b < nb; ++b) g->start[b + 1] += g->start[b];
  int *fill = (int *)malloc(sizeof(int) * (size_t)nb);
  if (!fill) { free(bk); return GDS_ERR_OOM; }
  memcpy(fill, g->start, sizeof(int) * (size_t)nb);
  for (int c = 0; c < ncells; ++c) g->idx[fill[bk[c]]++] = c;
  free(fill);
  free(bk);
  return GDS_OK;
}

static void grid_free(grid_t *g) {
  free(g->start); free(g->idx); free(g->x); free(g->y);
}

/* Two nearest cells of pixel centre (px,py): ring search over buckets.  A seed
 * clamped into an edge bucket lies at least as far as that bucket, so the
 * ring lower bound stays valid for it. */
static void nearest2(const grid_t *g, double px, double py, int *c1, double *d1, int *c2, double *d2) {
  int bx = (int)floor(px / g->bsz), by = (int)floor(py / g->bsz);
  if (bx < 0) bx = 0;
  if (bx >= g->nb_x) bx = g->nb_x - 1;
  if (by < 0) by = 0;
  if (by >= g->nb_y) by = g->nb_y - 1;
  double b1 = INFINITY, b2 = INFINITY;
  int i1 = -1, i2 = -1;
  int rmax = g->nb_x > g->nb_y ? g->nb_x : g->nb_y;
  for (int r = 0; r <= rmax; ++r) {
    /* every bucket at Chebyshev distance >= r from (bx,by) is at least
       (r-1)*bsz away from the pixel */
    double lb = (r - 1) * g->bsz;
    if (r >= 1 && lb > 0 && lb * lb > b2) break;
    for (int yy = by - r; yy <= by + r; ++yy) {
      if (yy < 0 || yy >= g->nb_y) continue;
      int on_edge_y = (yy == by - r) || (yy == by + r);
      for (int xx = bx - r; xx <= bx + r; ++xx) {
        if (xx < 0 || xx >= g->nb_x) continue;
        if (!on_edge_y && xx != bx - r && xx != bx + r) continue;
        int b = yy * g->nb_x + xx;
        for (int t = g->start[b]; t < g->start[b + 1]; ++t) {
          int c = g->idx[t];
          double dx = g->x[c] - px, dy = g->y[c] - py;
          double d = dx * dx + dy * dy;
          if (d < b1 || (d == b1 && c < i1)) {
            b2 = b1; i2 = i1; b1 = d; i1 = c;
          } else if (d < b2 || (d == b2 && c < i2)) {
            b2 = d; i2 = c;
          }
        }
      }
    }
  }
  *c1 = i1; *d1 = b1; *c2 = i2; *d2 = b2;
}

/*
 * Fill out[wz][wy][wx] (x fastest) with the window [x0,x0+wx) x [y0,y0+wy) x
 * [z0,z0+wz) of an NX x NY x NZ stack.
 *   ncells      Voronoi seeds per slice (>= 2)
 *   geom_seed   seeds the mosaic (cell positions, drift, values)
 *   photo_seed  seeds the per-slice gain / offset / ramp
 *   noise_seed  seeds the per-pixel noise; noise_sigma = 0 turns noise off
 * Returns 0 on success.
 */
int gds_em_window(uint8_t *out, int NX, int NY, int NZ, int ncells,
                  uint64_t geom_seed, uint64_t photo_seed, uint64_t noise_seed,
                  double noise_sigma, int x0, int y0, int z0, int wx, int wy, int wz) {
  if (!out || NX < 1 || NY < 1 || NZ < 1 || ncells < 2) return GDS_ERR_ARG;
  if (x0 < 0 || y0 < 0 || z0 < 0 || wx < 0 || wy < 0 || wz < 0) return GDS_ERR_ARG;
  if ((long)x0 + wx > NX || (long)y0 + wy > NY || (long)z0 + wz > NZ) return GDS_ERR_ARG;
  if (wx == 0 || wy == 0 || wz == 0) return GDS_OK;
  cell_t *cells = (cell_t *)malloc(sizeof(cell_t) * (size_t)ncells);
  if (!cells) return GDS_ERR_OOM;
  for (int c = 0; c < ncells; ++c) make_cell(&cells[c], geom_seed, NX, NY, (uint64_t)c);
  int err = GDS_OK;
  for (int zz = 0; zz < wz && err == GDS_OK; ++zz) {
    int z = z0 + zz;
    grid_t g;
    memset(&g, 0, sizeof(g));
    if (grid_build(&g, cells, ncells, NX, NY, (double)z) != GDS_OK) {
      grid_free(&g);
      err = GDS_ERR_OOM;
      break;
    }
    slice_t s;
    make_slice(&s, photo_seed, NX, NY, (uint64_t)z);
#pragma omp parallel for schedule(dynamic, 4)
    for (int yy = 0; yy < wy; ++yy) {
      int y = y0 + yy;
      uint8_t *row = out + ((size_t)zz * wy + yy) * (size_t)wx;
      for (int xx = 0; xx < wx; ++xx) {
        int x = x0 + xx;
        double px = x + 0.5, py = y + 0.5;
        int c1, c2;
        double d1, d2;
        nearest2(&g, px, py, &c1, &d1, &c2, &d2);
        double base = cells[c1].inner;
        if (c2 >= 0) {
          double sx = g.x[c2] - g.x[c1], sy = g.y[c2] - g.y[c1];
          double sep = sqrt(sx * sx + sy * sy);
          /* distance from the pixel centre to the bisector of the two seeds */
          double dist = sep > 0 ? (d2 - d1) / (2.0 * sep) : 0.0;
          if (dist < 1.0) base = cells[c1].memb;
        }
        double u = x * s.ct + y * s.st;
        double t = 2.0 * (u - s.umin) * s.uinv - 1.0;
        double v = s.gain * base + s.offset + s.ramp_amp * t;
        if (noise_sigma > 0) {
          uint64_t lin = ((uint64_t)z * (uint64_t)NY + (uint64_t)y) * (uint64_t)NX + (uint64_t)x;
          v += noise_sigma * gauss(noise_seed, ST_NOISE, lin);
        }
        if (v < 0.0) v = 0.0;
        if (v > 255.0) v = 255.0;
        row[xx] = (uint8_t)nearbyint(v); /* default rounding mode: half to even */
      }
    }
    grid_free(&g);
  }
  free(cells);
  return err;
}

int gds_version(void) { return 1; }
