// Matrix-free parallel-beam projectors: the operators of the CT experiments
// (Section 4.2) computed on the fly instead of read from a stored matrix.
//
// Geometry (the conventions of the synthetic workloads): N x N unit pixels
// centred at the origin (column iy*N + ix), angles a*pi/n_angles, unit bins
// centred at d - (n_bins-1)/2, ray (a, d) = {p : p.(cos, sin) = t_d} is row
// a*n_bins + d.  Three products, in RT arithmetic (the solve's vector type):
//   kProjRay        y = A x: Siddon's ray-driven walk, exact chord lengths;
//   kProjBackChord  y = A^T x, pixel-driven: the chord of ray (a, d) through a
//                   unit square is the square's trapezoid footprint;
//   kProjBackLinear y = B x, the unmatched pixel-driven back-projector: each
//                   pixel centre split linearly between its two nearest bins.
// A row's work is split over the 32 lanes of a warp (a ray's parameter range
// in 32 equal pieces, or a pixel's angles lane, lane + 32, ...); the product
// kernel adds the lanes' parts by a butterfly (a fixed order).
#pragma once

#include "common.cuh"

namespace sfl {

enum : int { kProjRay = 0, kProjBackChord = 1, kProjBackLinear = 2 };

// Per-angle table (kProjTab values per angle): cos, sin, the trapezoid's
// half-widths a1 = ||cos| - |sin||/2 <= a2 = (|cos| + |sin|)/2, its height
// H = 1/max(|cos|, |sin|), its ramp slope H/(a2 - a1) (0 when a1 = a2), and the
// axis flag (0: general; 1: |sin| < 1e-15, the rays are the lines x = const;
// 2: |cos| < 1e-15, the rays are y = const).
constexpr int kProjTab = 7;

// One lane's part of ray `row`: Siddon's walk over its piece of the ray.  The
// pixel indices start at the cell before the first grid line ahead on each
// axis (the same lines whose crossings the walk steps through) and step with
// the crossings (x line: ix += sign(dx), y line: iy += sign(dy), both at a
// corner).  Every segment then gets the pixel that contains it by the walk's
// own crossing order, without a floor per segment, and a start within
// rounding of a grid line cannot put the indices on the wrong side of it.
template <typename RT, typename XT>
__device__ __forceinline__ RT proj_ray_partial(int N, int nb, const RT *tab, const XT *__restrict__ x, int64_t row,
                                               int lane) {
  const int a = (int)(row / nb), d = (int)(row % nb);
  const RT c = tab[kProjTab * a], s = tab[kProjTab * a + 1];
  const RT t = (RT)d - RT(0.5) * (RT)(nb - 1);
  const RT h = RT(0.5) * (RT)N;
  const RT px = t * c, py = t * s;   // foot point
  const RT tiny = RT(1e-15);
  // unit direction; a component below tiny (cos(pi/2) in FP64) is exactly zero,
  // so a ray on a grid line belongs to the pixel with the floor index
  const RT dx = fabs(s) > tiny ? -s : RT(0), dy = fabs(c) > tiny ? c : RT(0);
  RT lo = -RT(1e30), hi = RT(1e30);
  const bool use_x = fabs(dx) > tiny, use_y = fabs(dy) > tiny;
  if (use_x) {
    const RT l0 = (-h - px) / dx, l1 = (h - px) / dx;
    lo = fmax(lo, fmin(l0, l1));
    hi = fmin(hi, fmax(l0, l1));
  } else if (!(px > -h && px < h)) {
    return RT(0);
  }
  if (use_y) {
    const RT l0 = (-h - py) / dy, l1 = (h - py) / dy;
    lo = fmax(lo, fmin(l0, l1));
    hi = fmin(hi, fmax(l0, l1));
  } else if (!(py > -h && py < h)) {
    return RT(0);
  }
  if (!(hi > lo)) return RT(0);
  // this lane's piece [a0, a0 + L] of the parameter range, walked in local parameters
  const RT span = hi - lo;
  const RT a0 = lo + span * (RT)lane / RT(32);
  const RT L = (lane == 31 ? hi : lo + span * (RT)(lane + 1) / RT(32)) - a0;
  const RT X0 = px + a0 * dx + h, Y0 = py + a0 * dy + h;   // grid coordinates in [0, N]
  RT lx = RT(1e30), ly = RT(1e30), lx0 = 0, ly0 = 0, ex = 0, ey = 0;
  int ix = (int)floor(X0), iy = (int)floor(Y0);   // kept on an axis without crossings
  if (use_x) {
    const RT kx = dx > 0 ? floor(X0) + RT(1) : ceil(X0) - RT(1);   // first x line ahead
    lx0 = lx = (kx - X0) / dx;
    ex = RT(1) / fabs(dx);
    ix = dx > 0 ? (int)kx - 1 : (int)kx;   // the column before that line
  }
  if (use_y) {
    const RT ky = dy > 0 ? floor(Y0) + RT(1) : ceil(Y0) - RT(1);
    ly0 = ly = (ky - Y0) / dy;
    ey = RT(1) / fabs(dy);
    iy = dy > 0 ? (int)ky - 1 : (int)ky;
  }
  const int sx = dx > 0 ? 1 : -1, sy = dy > 0 ? 1 : -1;
  RT acc = 0, prev = 0, jx = 0, jy = 0;
  for (int guard = 0; guard < 4 * N + 8; ++guard) {   // a piece crosses at most 2N + 2 grid lines
    const RT next = fmin(fmin(lx, ly), L);
    if (next - prev > RT(1e-12)) {
      const int cx = min(max(ix, 0), N - 1), cy = min(max(iy, 0), N - 1);
      acc += (next - prev) * (RT)x[(size_t)cy * N + cx];
    }
    if (next >= L) break;
    if (use_x && lx == next) { jx += RT(1); lx = lx0 + jx * ex; ix += sx; }
    if (use_y && ly == next) { jy += RT(1); ly = ly0 + jy * ey; iy += sy; }
    prev = next;
  }
  return acc;
}

// One lane's part of pixel `pix` of a back-projection (angles lane, lane + 32, ...).
template <typename RT, typename XT>
__device__ __forceinline__ RT proj_back_partial(int kind, int N, int na, int nb, const RT *tab,
                                                const XT *__restrict__ w, int64_t pix, int lane) {
  const int ix = (int)(pix % N), iy = (int)(pix / N);
  const RT h = RT(0.5) * (RT)N;
  const RT xc = (RT)ix - h + RT(0.5), yc = (RT)iy - h + RT(0.5);
  const RT off = RT(0.5) * (RT)(nb - 1);
  RT acc = 0;
  for (int a = lane; a < na; a += 32) {
    const RT *g = tab + kProjTab * a;
    const XT *wa = w + (size_t)a * nb;
    if (kind == kProjBackLinear) {
      const RT u = xc * g[0] + yc * g[1] + off;
      const RT d0 = floor(u);
      const RT f = u - d0;
      const int i0 = (int)d0;
      if (i0 >= 0 && i0 < nb && RT(1) - f > RT(1e-12)) acc += (RT(1) - f) * (RT)wa[i0];
      if (i0 + 1 >= 0 && i0 + 1 < nb && f > RT(1e-12)) acc += f * (RT)wa[i0 + 1];
      continue;
    }
    const int axis = (int)g[6];
    if (axis != 0) {
      // rays on grid lines: the walk gives a ray whose coordinate has floor =
      // the pixel index to that pixel (offset in [-1/2, 1/2) from its centre)
      // and never walks the image's lower boundary line
      const RT cen = axis == 1 ? xc : yc;
      const int idx = axis == 1 ? ix : iy;
      const int d = (int)ceil(cen + off - RT(0.5));   // the bin with d - off - cen in [-1/2, 1/2)
      if (d >= 0 && d < nb && !(idx == 0 && (RT)d - off - cen == RT(-0.5))) acc += (RT)wa[d];
      continue;
    }
    const RT u0 = xc * g[0] + yc * g[1] + off;   // bin coordinate of the pixel centre
    const RT a1 = g[2], a2 = g[3], H = g[4], slope = g[5];
    const int dlo = max(0, (int)ceil(u0 - a2)), dhi = min(nb - 1, (int)floor(u0 + a2));
    for (int d = dlo; d <= dhi; ++d) {
      const RT ad = fabs((RT)d - u0);
      if (!(ad < a2)) continue;
      const RT len = ad <= a1 ? H : H - slope * (ad - a1);
      if (len > RT(1e-12)) acc += len * (RT)wa[d];
    }
  }
  return acc;
}

}  // namespace sfl
