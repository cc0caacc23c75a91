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
// A ray of A x is walked by one thread (32 neighbouring rays per warp); a
// pixel of a back-projection is split over the 32 lanes of a warp (angles
// lane, lane + 32, ...), whose parts the product kernel adds by a butterfly
// (a fixed order).
#pragma once

#include "common.cuh"

namespace sfl {

enum : int { kProjRay = 0, kProjBackChord = 1, kProjBackLinear = 2 };

// Per-angle table (kProjTab values per angle): cos, sin, the trapezoid's
// half-widths a1 = ||cos| - |sin||/2 <= a2 = (|cos| + |sin|)/2, its height
// H = 1/max(|cos|, |sin|), its ramp slope H/(a2 - a1) (0 when a1 = a2), the
// axis flag (0: general; 1: |sin| < 1e-15, the rays are the lines x = const;
// 2: |cos| < 1e-15, the rays are y = const), and the reciprocals of the ray
// direction (dx, dy) = (-sin, cos): -1/sin and 1/cos (0 below 1e-15).
constexpr int kProjTab = 9;

// Fractional bits of a fixed-point bin coordinate in [-2, n_bins + 2]: |q| < 2^61.
__host__ __device__ inline int proj_bin_frac_bits(int nb) {
  int b = 0;
  for (unsigned v = (unsigned)nb + 2u; v; v >>= 1) ++b;
  return 61 - b;
}

template <typename RT> __device__ __forceinline__ RT proj_pow2(int e);
template <> __device__ __forceinline__ double proj_pow2<double>(int e) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}
template <> __device__ __forceinline__ float proj_pow2<float>(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ long long proj_to_fixed(double v) { return __double2ll_rn(v); }
__device__ __forceinline__ long long proj_to_fixed(float v) { return __float2ll_rn(v); }
template <typename RT> __device__ __forceinline__ RT proj_from_fixed(long long q);
template <> __device__ __forceinline__ double proj_from_fixed<double>(long long q) { return __ll2double_rn(q); }
template <> __device__ __forceinline__ float proj_from_fixed<float>(long long q) { return __ll2float_rn(q); }

// Ray `row` of A x, walked by one thread: Siddon's chords, column by column
// along the ray's major axis (the axis u with the larger direction component,
// |du| >= |dv|).  Between two major grid lines the ray rises by at most one
// unit along the minor axis v, so a column holds one pixel, or two split at
// one minor grid line.  The minor coordinate at the column ends is carried in
// 64-bit fixed point (F fractional bits, Q = round(v 2^F); inner columns add
// the per-column rise M = round(dv |1/du| 2^F)), which gives both pixels by
// shifts and the chord before the minor line as (its distance in v) |1/dv|.
// An inner column is |1/du| long, so its chords are |1/du| x2 + t (x1 - x2)
// (x1, x2 the pixels before and after the minor line, t the chord in x1); the
// walk adds x2 and t (x1 - x2) and scales the first sum by |1/du| once.  The
// two columns cut by the ray's entry and exit take their lengths from the
// parameters.  Pixels on a minor line count from the side the ray leaves, as
// the crossing order of a two-axis walk gives; a ray along a grid line takes
// the pixel with the floor index.  One thread per ray (the 32 rays of a warp
// are neighbouring bins of one angle) keeps the per-ray setup off the FP64
// pipe's critical count: it is issued once per 32 rays.
template <typename RT, typename XT>
__device__ __forceinline__ RT proj_ray(int N, int nb, const RT *tab, const XT *__restrict__ x, int64_t row) {
  const int a = (int)(row / nb), d = (int)(row % nb);
  const RT *g = tab + kProjTab * a;
  const RT c = g[0], s = g[1], inv_dx = g[7], inv_dy = g[8];
  const RT t = (RT)d - RT(0.5) * (RT)(nb - 1);
  const RT h = RT(0.5) * (RT)N;
  const RT px = t * c, py = t * s;   // foot point
  const RT tiny = RT(1e-15);
  // unit direction; a component below tiny (cos(pi/2) in FP64) is exactly zero,
  // so a ray on a grid line belongs to the pixel with the floor index
  const RT dx = fabs(s) > tiny ? -s : RT(0), dy = fabs(c) > tiny ? c : RT(0);
  RT lo = -RT(1e30), hi = RT(1e30);
  if (fabs(dx) > tiny) {
    const RT l0 = (-h - px) * inv_dx, l1 = (h - px) * inv_dx;
    lo = fmax(lo, fmin(l0, l1));
    hi = fmin(hi, fmax(l0, l1));
  } else if (!(px > -h && px < h)) {
    return RT(0);
  }
  if (fabs(dy) > tiny) {
    const RT l0 = (-h - py) * inv_dy, l1 = (h - py) * inv_dy;
    lo = fmax(lo, fmin(l0, l1));
    hi = fmin(hi, fmax(l0, l1));
  } else if (!(py > -h && py < h)) {
    return RT(0);
  }
  if (!(hi > lo)) return RT(0);
  const bool xmaj = fabs(dx) >= fabs(dy);
  const RT du = xmaj ? dx : dy, dv = xmaj ? dy : dx;
  const RT inv_du = xmaj ? inv_dx : inv_dy, inv_dv = xmaj ? inv_dy : inv_dx;
  const RT pu0 = (xmaj ? px : py) + h, pv0 = (xmaj ? py : px) + h;   // grid coordinates of the foot point
  const int64_t ustride = xmaj ? 1 : N, vstride = xmaj ? N : 1;
  // major grid lines strictly inside the ray: k1, k1 + su, ... (nl of them);
  // column i (0..nl) ends at line i (the ray's exit for i = nl)
  const bool fwd = du > RT(0);
  const int su = fwd ? 1 : -1;
  const RT ulo = pu0 + lo * du, uhi = pu0 + hi * du;
  const int k1 = fwd ? (int)floor(ulo) + 1 : (int)ceil(ulo) - 1;
  const int kl = fwd ? (int)ceil(uhi) - 1 : (int)floor(uhi) + 1;
  const int nl = min(max(fwd ? kl - k1 + 1 : k1 - kl + 1, 0), N + 1);
  const int F = proj_bin_frac_bits(N);   // |Q| < 2^61 for v in [-2, N + 2]
  const long long one = 1LL << F;
  const RT two_f = proj_pow2<RT>(F);
  const RT eu = fabs(inv_du), scale = proj_pow2<RT>(-F) * fabs(inv_dv);
  const RT nq = -pu0 * inv_du;
  const long long M = proj_to_fixed(dv * eu * two_f);
  // pixels x1 (after the column's start) and x2 (before its end) of column i,
  // and the chord t in x1 when they differ
  auto column = [&](int i, long long qs, long long qe, RT &x1, RT &x2) -> RT {
    int rs, re;
    if (dv > RT(0)) {
      rs = (int)(qs >> F);
      re = min(max(rs, (int)((qe - 1) >> F)), rs + 1);
    } else if (dv < RT(0)) {
      rs = (int)((qs - 1) >> F);
      re = max(min(rs, (int)(qe >> F)), rs - 1);
    } else {
      rs = re = (int)(qs >> F);
    }
    const long long vc = (long long)(dv > RT(0) ? rs + 1 : rs) * one;   // the minor line crossed
    const int cu = min(max(fwd ? k1 - 1 + i : k1 - i, 0), N - 1);
    x1 = (RT)x[cu * ustride + min(max(rs, 0), N - 1) * vstride];
    x2 = (RT)x[cu * ustride + min(max(re, 0), N - 1) * vstride];
    return re != rs ? proj_from_fixed<RT>(vc > qs ? vc - qs : qs - vc) * scale : RT(0);
  };
  RT S = RT(0), C, x1, x2;
  long long Qs = proj_to_fixed((pv0 + lo * dv) * two_f);
  {   // column 0: from the entry to line 0, or to the exit
    const RT le = nl == 0 ? hi : (RT)k1 * inv_du + nq;
    const long long Qe = proj_to_fixed((pv0 + le * dv) * two_f);
    const RT len = le - lo;
    const RT tc = fmin(column(0, Qs, Qe, x1, x2), len);
    C = len * x2 + tc * (x1 - x2);
    Qs = Qe;
  }
  for (int i = 1; i < nl; ++i) {   // inner columns, |1/du| long
    const long long Qe = Qs + M;
    const RT tc = column(i, Qs, Qe, x1, x2);
    S += x2;
    C += tc * (x1 - x2);
    Qs = Qe;
  }
  if (nl > 0) {   // column nl: from line nl - 1 to the exit
    const RT ls = (RT)(k1 + su * (nl - 1)) * inv_du + nq;
    const long long Qe = proj_to_fixed((pv0 + hi * dv) * two_f);
    const RT len = hi - ls;
    const RT tc = fmin(column(nl, Qs, Qe, x1, x2), len);
    C += len * x2 + tc * (x1 - x2);
  }
  return eu * S + C;
}

// The fraction f = fr 2^-F (0 <= fr < 2^F) as an FP64 value: the fraction's
// top 52 bits as the significand of a number in [1, 2), minus one (exact).
__device__ __forceinline__ double proj_frac(long long fr, int F) {
  const long long m = F >= 52 ? fr >> (F - 52) : fr << (52 - F);
  return __longlong_as_double(0x3FF0000000000000LL | m) - 1.0;
}

// Rows [row0, r1) of y = B x (pixel-driven linear interpolation), FP64, one
// 32-row block: lane l takes the angles l, l + 32, ... (kProjLinPass per lane
// and pass) and keeps each angle's bin coordinate u = xc cos + yc sin + off of
// the current pixel in fixed point (F = proj_bin_frac_bits(n_bins) fractional
// bits).  From one pixel to the next in an image row u grows by cos, a
// per-angle integer step round(cos 2^F) from the plan; a new block or image
// row starts from u itself.  The bins and weights then come from shifts and
// one FP64 subtraction, so a (pixel, angle) pair costs four FP64 instructions.
// Each pass's lane sums are added by a butterfly; lane r returns row r.
constexpr int kProjLinPass = 8;
template <typename XT>
__device__ __forceinline__ double proj_back_linear_block(int N, int na, int nb, const double *tab,
                                                         const long long *__restrict__ fix, const XT *__restrict__ w,
                                                         int64_t row0, int64_t r1, int lane) {
  const int F = proj_bin_frac_bits(nb);
  const long long one = 1LL << F, mask = one - 1;
  const double two_f = proj_pow2<double>(F);
  // weights below 1e-12 are dropped, as in the stored operator
  const long long thr_lo = (long long)(1e-12 * two_f), thr_hi = one - thr_lo;
  const double h = 0.5 * (double)N, off = 0.5 * (double)(nb - 1);
  double mine = 0.0;
  for (int a0 = 0; a0 < na; a0 += 32 * kProjLinPass) {
    long long U[kProjLinPass];
    for (int64_t row = row0; row < r1; ++row) {
      const int ix = (int)(row % N), iy = (int)(row / N);
      if (row == row0 || ix == 0) {
        const double xc = (double)ix - h + 0.5, yc = (double)iy - h + 0.5;
#pragma unroll
        for (int j = 0; j < kProjLinPass; ++j) {
          const int a = a0 + lane + 32 * j;
          if (a < na) U[j] = proj_to_fixed((xc * tab[kProjTab * a] + yc * tab[kProjTab * a + 1] + off) * two_f);
        }
      } else {
#pragma unroll
        for (int j = 0; j < kProjLinPass; ++j) {
          const int a = a0 + lane + 32 * j;
          if (a < na) U[j] += fix[a];
        }
      }
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < kProjLinPass; ++j) {
        const int a = a0 + lane + 32 * j;
        if (a < na) {
          const int i0 = (int)(U[j] >> F);
          const long long fr = U[j] & mask;
          const double f = proj_frac(fr, F);
          const XT *wa = w + (size_t)a * nb;
          const double w0 = i0 >= 0 && i0 < nb && fr < thr_hi ? (double)wa[i0] : 0.0;
          const double w1 = i0 + 1 >= 0 && i0 + 1 < nb && fr > thr_lo ? (double)wa[i0 + 1] : 0.0;
          acc = fma(1.0 - f, w0, acc);
          acc = fma(f, w1, acc);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == (int)(row - row0)) mine += acc;
    }
  }
  return mine;
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
