/*
 * The synthetic EM-like stack generator of synth.c, evaluated on the GPU for
 * the large stacks (training pairs of the learned initial guess, the
 * 2048x2048x512 and 4096x4096x256 workloads).  Like synth.c it only draws
 * pixels and holds none of the gradient-domain method's arithmetic.
 *
 * The per-cell and per-slice parameters and the per-slice bucket grids are
 * built on the host by synth.c's own functions (included below), so they are
 * bit-identical; the per-pixel part (two nearest seeds, membrane test,
 * photometric distortion, SplitMix64 / Box-Muller noise, rounding) runs in a
 * kernel with the same double-precision formulas.  CUDA's log and cos may
 * differ from the host's libm in the last bit, which changes a byte only
 * when a value falls within ~1e-13 of a rounding boundary.
 */
#include "synth.c"

#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t d_sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t d_h3(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return d_sm64(d_sm64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + ctr);
}
__device__ __forceinline__ double d_u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }
__device__ __forceinline__ double d_u01_open0(uint64_t h) { return ((double)(h >> 11) + 1.0) * 0x1.0p-53; }
__device__ __forceinline__ double d_gauss(uint64_t seed, uint64_t stream, uint64_t ctr) {
  const double a = d_u01_open0(d_h3(seed, stream, 2 * ctr));
  const double b = d_u01(d_h3(seed, stream, 2 * ctr + 1));
  return sqrt(-2.0 * log(a)) * cos(6.283185307179586476925286766559 * b);  // 2 pi, as in synth.c
}

struct DevGrid {
  const double *x, *y;  // seed positions of every slice of the chunk, [slice][cell]
  const int *start;     // [slice][nb + 1]
  const int *idx;       // [slice][cell]
  int ncells, nb_x, nb_y;
  double bsz;
};

// two nearest seeds of (px, py) in slice s of the chunk: the same ring search
// and tie-breaking as nearest2 in synth.c
__device__ void d_nearest2(const DevGrid &g, int s, double px, double py, int *c1, double *d1, int *c2,
                           double *d2) {
  const int nb = g.nb_x * g.nb_y;
  const double *X = g.x + (size_t)s * g.ncells, *Y = g.y + (size_t)s * g.ncells;
  const int *start = g.start + (size_t)s * (nb + 1), *idx = g.idx + (size_t)s * g.ncells;
  int bx = (int)floor(px / g.bsz), by = (int)floor(py / g.bsz);
  if (bx < 0) bx = 0;
  if (bx >= g.nb_x) bx = g.nb_x - 1;
  if (by < 0) by = 0;
  if (by >= g.nb_y) by = g.nb_y - 1;
  double b1 = INFINITY, b2 = INFINITY;
  int i1 = -1, i2 = -1;
  const int rmax = g.nb_x > g.nb_y ? g.nb_x : g.nb_y;
  for (int r = 0; r <= rmax; ++r) {
    const double lb = (r - 1) * g.bsz;
    if (r >= 1 && lb > 0 && lb * lb > b2) break;
    for (int yy = by - r; yy <= by + r; ++yy) {
      if (yy < 0 || yy >= g.nb_y) continue;
      const int on_edge_y = (yy == by - r) || (yy == by + r);
      for (int xx = bx - r; xx <= bx + r; ++xx) {
        if (xx < 0 || xx >= g.nb_x) continue;
        if (!on_edge_y && xx != bx - r && xx != bx + r) continue;
        const int b = yy * g.nb_x + xx;
        for (int t = start[b]; t < start[b + 1]; ++t) {
          const int c = idx[t];
          const double dx = X[c] - px, dy = Y[c] - py;
          const double d = dx * dx + dy * dy;
          if (d < b1 || (d == b1 && c < i1)) {
            b2 = b1;
            i2 = i1;
            b1 = d;
            i1 = c;
          } else if (d < b2 || (d == b2 && c < i2)) {
            b2 = d;
            i2 = c;
          }
        }
      }
    }
  }
  *c1 = i1;
  *d1 = b1;
  *c2 = i2;
  *d2 = b2;
}

__global__ void k_em_window(uint8_t *out, DevGrid g, const double *inner, const double *memb, const slice_t *sl,
                            int NX, int NY, int x0, int y0, int z0, int wx, int wy, int nzc,
                            uint64_t noise_seed, double noise_sigma) {
  const size_t n = (size_t)wx * wy * nzc;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(e % wx);
    const size_t r = e / wx;
    const int yy = (int)(r % wy), s = (int)(r / wy);
    const int x = x0 + xx, y = y0 + yy, z = z0 + s;
    const double px = x + 0.5, py = y + 0.5;
    int c1, c2;
    double d1, d2;
    d_nearest2(g, s, px, py, &c1, &d1, &c2, &d2);
    double base = inner[c1];
    if (c2 >= 0) {
      const double *X = g.x + (size_t)s * g.ncells, *Y = g.y + (size_t)s * g.ncells;
      const double sx = X[c2] - X[c1], sy = Y[c2] - Y[c1];
      const double sep = sqrt(sx * sx + sy * sy);
      const double dist = sep > 0 ? (d2 - d1) / (2.0 * sep) : 0.0;
      if (dist < 1.0) base = memb[c1];
    }
    const slice_t S = sl[s];
    const double u = x * S.ct + y * S.st;
    const double t = 2.0 * (u - S.umin) * S.uinv - 1.0;
    double v = S.gain * base + S.offset + S.ramp_amp * t;
    if (noise_sigma > 0) {
      const uint64_t lin = ((uint64_t)z * (uint64_t)NY + (uint64_t)y) * (uint64_t)NX + (uint64_t)x;
      v += noise_sigma * d_gauss(noise_seed, ST_NOISE, lin);
    }
    if (v < 0.0) v = 0.0;
    if (v > 255.0) v = 255.0;
    out[e] = (uint8_t)rint(v);  // half to even, as nearbyint in the default mode
  }
}

template <typename T>
int dalloc(T **p, size_t n) {
  if (cudaMalloc((void **)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return GDS_ERR_OOM;
  }
  return GDS_OK;
}

}  // namespace

/*
 * gds_em_window_cuda -- gds_em_window into device memory `d_out`
 * ([wz][wy][wx], x fastest) on `stream` (a cudaStream_t or NULL).  Slices are
 * generated in chunks of up to 64; returns after the last chunk completes.
 * 0 on success, GDS_ERR_ARG for bad sizes, GDS_ERR_OOM, 4 for a CUDA error.
 */
extern "C" int gds_em_window_cuda(uint8_t *d_out, int NX, int NY, int NZ, int ncells, uint64_t geom_seed,
                                  uint64_t photo_seed, uint64_t noise_seed, double noise_sigma, int x0, int y0,
                                  int z0, int wx, int wy, int wz, void *stream) {
  if (!d_out || NX < 1 || NY < 1 || NZ < 1 || ncells < 2) return GDS_ERR_ARG;
  if (x0 < 0 || y0 < 0 || z0 < 0 || wx < 0 || wy < 0 || wz < 0) return GDS_ERR_ARG;
  if ((long)x0 + wx > NX || (long)y0 + wy > NY || (long)z0 + wz > NZ) return GDS_ERR_ARG;
  if (wx == 0 || wy == 0 || wz == 0) return GDS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cell_t *cells = (cell_t *)malloc(sizeof(cell_t) * (size_t)ncells);
  if (!cells) return GDS_ERR_OOM;
  for (int c = 0; c < ncells; ++c) make_cell(&cells[c], geom_seed, NX, NY, (uint64_t)c);
  const int CH = wz < 64 ? wz : 64;
  int err = GDS_OK;
  // geometry of the bucket grid (the same for every slice)
  grid_t g0;
  memset(&g0, 0, sizeof g0);
  if (grid_build(&g0, cells, ncells, NX, NY, 0.0) != GDS_OK) err = GDS_ERR_OOM;
  const int nb = g0.nb_x * g0.nb_y;
  const int nb_x = g0.nb_x, nb_y = g0.nb_y;
  const double bsz = g0.bsz;
  grid_free(&g0);
  double *h_x = nullptr, *h_y = nullptr, *h_in = nullptr, *h_mb = nullptr;
  int *h_start = nullptr, *h_idx = nullptr;
  slice_t *h_sl = nullptr;
  double *d_x = nullptr, *d_y = nullptr, *d_in = nullptr, *d_mb = nullptr;
  int *d_start = nullptr, *d_idx = nullptr;
  slice_t *d_sl = nullptr;
  if (err == GDS_OK) {
    h_x = (double *)malloc(sizeof(double) * (size_t)CH * ncells);
    h_y = (double *)malloc(sizeof(double) * (size_t)CH * ncells);
    h_start = (int *)malloc(sizeof(int) * (size_t)CH * (nb + 1));
    h_idx = (int *)malloc(sizeof(int) * (size_t)CH * ncells);
    h_sl = (slice_t *)malloc(sizeof(slice_t) * (size_t)CH);
    h_in = (double *)malloc(sizeof(double) * (size_t)ncells);
    h_mb = (double *)malloc(sizeof(double) * (size_t)ncells);
    if (!h_x || !h_y || !h_start || !h_idx || !h_sl || !h_in || !h_mb) err = GDS_ERR_OOM;
  }
  if (err == GDS_OK) {
    for (int c = 0; c < ncells; ++c) {
      h_in[c] = cells[c].inner;
      h_mb[c] = cells[c].memb;
    }
    if (dalloc(&d_x, (size_t)CH * ncells) || dalloc(&d_y, (size_t)CH * ncells) ||
        dalloc(&d_start, (size_t)CH * (nb + 1)) || dalloc(&d_idx, (size_t)CH * ncells) || dalloc(&d_sl, (size_t)CH) ||
        dalloc(&d_in, (size_t)ncells) || dalloc(&d_mb, (size_t)ncells))
      err = GDS_ERR_OOM;
  }
  if (err == GDS_OK && (cudaMemcpy(d_in, h_in, sizeof(double) * ncells, cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(d_mb, h_mb, sizeof(double) * ncells, cudaMemcpyHostToDevice) != cudaSuccess))
    err = 4;
  int dev = 0, sms = 132;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int zc = 0; zc < wz && err == GDS_OK; zc += CH) {
    const int nzc = wz - zc < CH ? wz - zc : CH;
    for (int s = 0; s < nzc && err == GDS_OK; ++s) {
      const int z = z0 + zc + s;
      grid_t g;
      memset(&g, 0, sizeof g);
      if (grid_build(&g, cells, ncells, NX, NY, (double)z) != GDS_OK) {
        grid_free(&g);
        err = GDS_ERR_OOM;
        break;
      }
      memcpy(h_x + (size_t)s * ncells, g.x, sizeof(double) * ncells);
      memcpy(h_y + (size_t)s * ncells, g.y, sizeof(double) * ncells);
      memcpy(h_start + (size_t)s * (nb + 1), g.start, sizeof(int) * (nb + 1));
      memcpy(h_idx + (size_t)s * ncells, g.idx, sizeof(int) * ncells);
      make_slice(&h_sl[s], photo_seed, NX, NY, (uint64_t)z);
      grid_free(&g);
    }
    if (err != GDS_OK) break;
    // the previous chunk's kernel reads these buffers: finish it first
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(d_x, h_x, sizeof(double) * (size_t)nzc * ncells, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_y, h_y, sizeof(double) * (size_t)nzc * ncells, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_start, h_start, sizeof(int) * (size_t)nzc * (nb + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_idx, h_idx, sizeof(int) * (size_t)nzc * ncells, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_sl, h_sl, sizeof(slice_t) * (size_t)nzc, cudaMemcpyHostToDevice) != cudaSuccess) {
      err = 4;
      break;
    }
    DevGrid dg{d_x, d_y, d_start, d_idx, ncells, nb_x, nb_y, bsz};
    const size_t n = (size_t)wx * wy * nzc;
    size_t blocks = (n + 255) / 256;
    if (blocks > (size_t)sms * 16) blocks = (size_t)sms * 16;
    k_em_window<<<(unsigned)blocks, 256, 0, st>>>(d_out + (size_t)zc * wx * wy, dg, d_in, d_mb, d_sl, NX, NY, x0,
                                                  y0, z0 + zc, wx, wy, nzc, noise_seed, noise_sigma);
    if (cudaGetLastError() != cudaSuccess) err = 4;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && err == GDS_OK) err = 4;
  cudaFree(d_x);
  cudaFree(d_y);
  cudaFree(d_start);
  cudaFree(d_idx);
  cudaFree(d_sl);
  cudaFree(d_in);
  cudaFree(d_mb);
  free(h_x);
  free(h_y);
  free(h_start);
  free(h_idx);
  free(h_sl);
  free(h_in);
  free(h_mb);
  free(cells);
  return err;
}
