/* Seeded-input generators for the synthetic parallel-beam CT workloads.
 *
 * This file builds the *operators* (input data) the solvers are run on; it
 * holds none of the solver arithmetic.  Geometry (fixed once, shared by every
 * consumer through the generated arrays, never through code):
 *   - N x N image of unit pixels centred at the origin, pixel (ix, iy) covers
 *     [ix - N/2, ix - N/2 + 1] x [iy - N/2, iy - N/2 + 1], column = iy*N + ix;
 *   - angles theta_a = a*pi/n_angles, a = 0..n_angles-1 (parallel beam over [0, pi));
 *   - n_bins unit-width detector bins centred at t_d = d - (n_bins-1)/2;
 *   - ray (a, d) is the line {p : p . (cos theta, sin theta) = t_d}, row a*n_bins + d.
 * siddon_*  : A[row, col] = exact chord length of the ray through the pixel
 *             (Siddon's ray-driven method), lengths < 1e-12 dropped, columns
 *             sorted ascending within each row.
 * pixel_*   : the pixel-driven linear-interpolation back-projector B (n x m):
 *             for each pixel centre c and angle a, t = c . (cos, sin) is split
 *             between the two nearest bin centres with weights summing to 1.
 * Both are deterministic (no RNG) and parallel over rows with OpenMP; the
 * output does not depend on the thread count.  Compiled with
 * -ffp-contract=off so x86-64 and aarch64 builds give identical arrays.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t col; double len; } seg_t;

/* Walk ray (a, d); write at most cap segments into out; return the count. */
static int64_t siddon_ray(int N, int n_angles, int n_bins, int64_t row, seg_t *out, int64_t cap) {
  const int a = (int)(row / n_bins), d = (int)(row % n_bins);
  const double th = (double)a * M_PI / (double)n_angles;
  const double c = cos(th), s = sin(th);
  const double t = (double)d - 0.5 * (double)(n_bins - 1);
  const double h = 0.5 * (double)N;
  const double px = t * c, py = t * s;   /* foot point */
  const double tiny = 1e-15;
  /* unit direction; a component below tiny (cos(pi/2) = 6e-17 in FP64) is
   * taken as exactly zero, so a ray that lies on a grid line belongs to the
   * pixel whose index is the floor of its coordinate along its whole length */
  const double dx = fabs(s) > tiny ? -s : 0.0, dy = fabs(c) > tiny ? c : 0.0;
  double lo = -INFINITY, hi = INFINITY;
  if (fabs(dx) > tiny) {
    double l0 = (-h - px) / dx, l1 = (h - px) / dx;
    lo = fmax(lo, fmin(l0, l1)); hi = fmin(hi, fmax(l0, l1));
  } else if (!(px > -h && px < h)) {
    return 0;
  }
  if (fabs(dy) > tiny) {
    double l0 = (-h - py) / dy, l1 = (h - py) / dy;
    lo = fmax(lo, fmin(l0, l1)); hi = fmin(hi, fmax(l0, l1));
  } else if (!(py > -h && py < h)) {
    return 0;
  }
  if (!(hi > lo)) return 0;
  /* crossings with the grid lines x = -h + kx and y = -h + ky, visited in
   * increasing lambda; each crossing is computed from its integer index */
  double kx = 0.0, ky = 0.0, lx = INFINITY, ly = INFINITY;
  const double sx = dx > 0 ? 1.0 : -1.0, sy = dy > 0 ? 1.0 : -1.0;
  const int use_x = fabs(dx) > tiny, use_y = fabs(dy) > tiny;
  if (use_x) {
    double xin = px + lo * dx + h;            /* entry point, in [0, N] */
    kx = dx > 0 ? floor(xin) + 1.0 : ceil(xin) - 1.0;
    lx = (kx - h - px) / dx;
  }
  if (use_y) {
    double yin = py + lo * dy + h;
    ky = dy > 0 ? floor(yin) + 1.0 : ceil(yin) - 1.0;
    ly = (ky - h - py) / dy;
  }
  int64_t cnt = 0;
  double prev = lo;
  for (int guard = 0; guard < 4 * N + 8; ++guard) {
    double next = fmin(fmin(lx, ly), hi);
    if (next - prev > 1e-12) {
      double lm = 0.5 * (prev + next);
      int ix = (int)floor(px + lm * dx + h), iy = (int)floor(py + lm * dy + h);
      if (ix < 0) ix = 0;
      if (ix > N - 1) ix = N - 1;
      if (iy < 0) iy = 0;
      if (iy > N - 1) iy = N - 1;
      if (out && cnt < cap) { out[cnt].col = iy * N + ix; out[cnt].len = next - prev; }
      cnt++;
    }
    if (next >= hi) break;
    if (use_x && lx == next) { kx += sx; lx = (kx - h - px) / dx; }
    if (use_y && ly == next) { ky += sy; ly = (ky - h - py) / dy; }
    prev = next;
  }
  return cnt;
}

/* Order the segments of one ray by column: iy and ix are each monotone along
 * the ray, so reverse the whole list if iy decreases, then reverse every run of
 * equal iy whose ix decreases. */
static void sort_ray(seg_t *v, int64_t n, int N) {
  if (n < 2) return;
  if (v[0].col / N > v[n - 1].col / N) {
    for (int64_t i = 0, j = n - 1; i < j; ++i, --j) { seg_t t = v[i]; v[i] = v[j]; v[j] = t; }
  }
  int64_t b = 0;
  while (b < n) {
    int64_t e = b + 1;
    while (e < n && v[e].col / N == v[b].col / N) ++e;
    if (e - b > 1 && v[b].col > v[e - 1].col) {
      for (int64_t i = b, j = e - 1; i < j; ++i, --j) { seg_t t = v[i]; v[i] = v[j]; v[j] = t; }
    }
    b = e;
  }
}

/* Pass 1: number of nonzeros per row (rowcnt has n_angles*n_bins entries). */
void siddon_count(int N, int n_angles, int n_bins, int64_t *rowcnt) {
  const int64_t m = (int64_t)n_angles * n_bins;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < m; ++r) rowcnt[r] = siddon_ray(N, n_angles, n_bins, r, NULL, 0);
}

/* Pass 2: fill CSR arrays given rowptr (m+1 entries, int64 prefix sums). */
void siddon_fill(int N, int n_angles, int n_bins, const int64_t *rowptr, int32_t *colidx, double *val) {
  const int64_t m = (int64_t)n_angles * n_bins;
#pragma omp parallel
  {
    seg_t *buf = (seg_t *)malloc(sizeof(seg_t) * (size_t)(4 * N + 8));
#pragma omp for schedule(dynamic, 64)
    for (int64_t r = 0; r < m; ++r) {
      int64_t cnt = siddon_ray(N, n_angles, n_bins, r, buf, 4 * N + 8);
      sort_ray(buf, cnt, N);
      for (int64_t i = 0; i < cnt; ++i) {
        colidx[rowptr[r] + i] = buf[i].col;
        val[rowptr[r] + i] = buf[i].len;
      }
    }
    free(buf);
  }
}

/* Pixel-driven back-projector B (n x m), two interpolation weights per
 * (pixel, angle).  Pass 1 counts, pass 2 fills; rows are pixels. */
static int pixel_row(int N, int n_angles, int n_bins, int64_t pix, int32_t *col, double *val) {
  const int ix = (int)(pix % N), iy = (int)(pix / N);
  const double h = 0.5 * (double)N;
  const double xc = (double)ix - h + 0.5, yc = (double)iy - h + 0.5;
  int cnt = 0;
  for (int a = 0; a < n_angles; ++a) {
    const double th = (double)a * M_PI / (double)n_angles;
    const double t = xc * cos(th) + yc * sin(th);
    const double u = t + 0.5 * (double)(n_bins - 1);
    const double d0 = floor(u);
    const double f = u - d0;
    const int i0 = (int)d0;
    if (i0 >= 0 && i0 < n_bins && 1.0 - f > 1e-12) {
      if (col) { col[cnt] = a * n_bins + i0; val[cnt] = 1.0 - f; }
      cnt++;
    }
    if (i0 + 1 >= 0 && i0 + 1 < n_bins && f > 1e-12) {
      if (col) { col[cnt] = a * n_bins + i0 + 1; val[cnt] = f; }
      cnt++;
    }
  }
  return cnt;
}

void pixel_count(int N, int n_angles, int n_bins, int64_t *rowcnt) {
  const int64_t n = (int64_t)N * N;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) rowcnt[p] = pixel_row(N, n_angles, n_bins, p, NULL, NULL);
}

void pixel_fill(int N, int n_angles, int n_bins, const int64_t *rowptr, int32_t *colidx, double *val) {
  const int64_t n = (int64_t)N * N;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) pixel_row(N, n_angles, n_bins, p, colidx + rowptr[p], val + rowptr[p]);
}

/* y = A x for a CSR matrix (used only to synthesise b = A x_true + e). */
void csr_matvec(int64_t m, const int64_t *rowptr, const int32_t *colidx, const double *val,
                const double *x, double *y) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < m; ++r) {
    double acc = 0.0;
    for (int64_t i = rowptr[r]; i < rowptr[r + 1]; ++i) acc += val[i] * x[colidx[i]];
    y[r] = acc;
  }
}
