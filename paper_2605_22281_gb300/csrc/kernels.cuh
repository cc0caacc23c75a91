// Kernels of one sketched flexible Golub-Kahan step (Algorithms 1 and 2).
//
// Per step k the solver runs, on one stream, captured in a CUDA graph:
//   zorth   p~_k = z - sum_j c_j p_j (MGS coefficients c_j), z~_k = tau_k(p~_k)
//   fwd     w = A z_k (CSR SpMV) + window dots <w_j, w> + sketch S_m w
//   worth   w~_{k+1} = w - sum_j h_j w_j, ||w~_{k+1}||  (column k of H)
//   bwd     z = A^T w_{k+1} (CSR of A^T, or B) + dots <p_j, z> (+ S_n z, sFLSMR)
//   ls      append one column to the FP64 QR of the sketched problem, update
//           y_k and the stop ratio, set the graph's loop condition
// Every reduction is fixed-order, so results are bitwise reproducible.
#pragma once

#include <climits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "proj.cuh"

namespace cg = cooperative_groups;

namespace sfl {

// ---------------------------------------------------------------- sketch table

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the first output of a
// generator whose state is `state`.
__device__ __forceinline__ uint64_t splitmix64_first(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Column c of the sparse-sign sketch (Section 2.7): draws t = 0, 1, ... with
// h = splitmix64_first(seed ^ (c*2^32 + t)), row floor(h*s/2^64), sign from
// bit 0; duplicates rejected until zeta distinct rows.  Packed entry: row in
// bits 0..14, bit 15 set for a negative sign.  `zs` entries per column
// (zs >= zeta; unused entries are 0xFFFF).  Optional unpacked export.
// The seed is `seed` or, when seed_src is given, *seed_src (plus seed_add).
static __global__ void sketch_table_kernel(uint64_t seed, const uint64_t *seed_src, uint64_t seed_add, int s, int zeta,
                                    int64_t ncols, int zs, uint16_t *tab, int32_t *rows_out, int32_t *signs_out,
                                    int *err) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  if (seed_src) seed = *seed_src;
  seed += seed_add;
  int rows[kMaxZeta];
  int cnt = 0;
  for (uint32_t t = 0; cnt < zeta && t < 1000000u; ++t) {
    const uint64_t h = splitmix64_first(seed ^ (((uint64_t)c << 32) + t));
    const int r = (int)__umul64hi(h, (uint64_t)s);
    bool dup = false;
    for (int q = 0; q < cnt; ++q) dup |= (rows[q] == r);
    if (dup) continue;
    rows[cnt] = r;
    const int neg = (int)(h & 1ull);
    if (tab) tab[c * zs + cnt] = (uint16_t)(r | (neg << 15));
    if (rows_out) { rows_out[c * zeta + cnt] = r; signs_out[c * zeta + cnt] = neg ? -1 : 1; }
    ++cnt;
  }
  if (cnt < zeta) { atomicExch(err, 1); return; }
  if (tab) for (int q = cnt; q < zs; ++q) tab[c * zs + q] = 0xFFFFu;
}

// ---------------------------------------------------------------- step kernels

// Partial-sum buffers: each producing kernel stores one record per CTA; the
// next kernel on the stream reduces them (reduce_partials) and derives the
// scalars of the step identically in every CTA.  CTA 0 persists them.
struct Partials {
  double *b;     // init pass: ||b||^2                       -> init A^T w_1
  double *z;     // A^T w products: ||z||^2, <p_j, z>         -> z update of the next step
  double *p;     // z update: ||p~_k||^2, <p~_k, p~_j>        -> A z_k product
  double *w;     // A z_k product: ||w||^2, <w_j, w>          -> w update
  double *wn;    // w update: ||w~_{k+1}||^2, <w~_{k+1}, w~_j> -> A^T w_{k+1} product
};

enum SpmvMode : int {
  kModeApply = 0,    // plain y = A x
  kModeInitB = 1,    // row value = b_i: ||b||^2, w~_1 = b
  kModeInitBwd = 2,  // z = A^T w_1, ||z||^2
  kModeFwd = 3,      // w = A z_k, window dots with w_j, ||w||^2
  kModeBwd = 4       // z = A^T w_{k+1}, window dots with p_j, ||z||^2
};

template <typename VT, typename XT>
struct SpmvParams {
  const int32_t *rowptr;    // padded CSR (rows start at multiples of the load width)
  const int32_t *col;
  const VT *val;
  const int16_t *dcol;      // the 16-bit delta forms: column deltas along each lane's walk
  const int32_t *rbase;     //   and each stored row's base column
  int64_t rows;
  const int32_t *wrow;      // row range of every warp (nnz balanced), gridDim*kWarps + 1 entries
  const int32_t *orig;      // stored row i is operator row orig[i] (read by the kSpmvMatOrig form)
  int interleave;           // 1: the warps of a CTA take its 32-row blocks in turn (tiled operators)
  int mode;
  int method;
  int ell;
  int G_prev;               // CTAs of the kernel whose partials this one reduces
  const XT *x;              // kModeApply: input vector
  const double *b;          // kModeInitB
  XT *y;                    // output (kModeApply)
  SolveState *st;
  XT *wring; int64_t wstride; int RW;   // ring of w~ (m-vectors)
  XT *pring; int64_t pstride; int RP;   // ring of p~ (n-vectors)
  XT *Z; int64_t zstride;               // z~_j columns
  double *sigZ;
  int orth_z;                           // 1: the z window is Z's columns, not the p ring
  XT *wraw;                             // w = A z_k
  XT *zraw;                             // z = A^T w
  double *Hband;                        // columns of H, (hb_ell+2) entries per column (when want_h)
  int want_h;                           // H is recorded (sFLSMR, FLSQR)
  int hb_ell;                           // band width of Hband columns minus 2 (ell, or maxit when full)
  int full;                             // full orthogonalization: no window dots (block CGS2 kernels do it)
  XT *wfull;                            // full: every w~_j (column j - 1); the vector pass writes w~_1
  double *sigWall;                      // full: 1/||w~_j|| at index j - 1
  // fused sparse-sign sketch of the product output (sk_s > 0): every CTA adds
  // its rows' contributions into an s-vector record sk_rec[r * sk_cap + cta]
  int sk_s, sk_zeta;
  uint64_t sk_seed_add;                 // the sketch's seed is the solve's seed plus this
  double *sk_rec;
  int sk_cap;
  // matrix-free projector (the kSpmvProj form; the CSR arrays are unused)
  int proj;                             // kProjRay, kProjBackChord or kProjBackLinear
  int pN, pna, pnb;                     // image N x N, angles, bins
  const void *ptab;                     // per-angle constants, kProjTab values each, in the vectors' arithmetic
  const long long *pfix;                // FP64: per-angle bin-coordinate step round(cos 2^F) (proj.cuh)
  Partials part;
};

// Loads of P consecutive stored entries (P*4 bytes of indices, P*sizeof(VT) of values).
template <typename VT, int P> struct Chunk;
template <> struct Chunk<double, 4> {
  int c[4]; double v[4];
  __device__ __forceinline__ void load(const int32_t *col, const double *val, int off) {
    const int4 ci = __ldcs(reinterpret_cast<const int4 *>(col + off));
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(val + off));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(val + off + 2));
    c[0] = ci.x; c[1] = ci.y; c[2] = ci.z; c[3] = ci.w;
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <> struct Chunk<float, 4> {
  int c[4]; float v[4];
  __device__ __forceinline__ void load(const int32_t *col, const float *val, int off) {
    const int4 ci = __ldcs(reinterpret_cast<const int4 *>(col + off));
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(val + off));
    c[0] = ci.x; c[1] = ci.y; c[2] = ci.z; c[3] = ci.w;
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <> struct Chunk<__nv_bfloat16, 8> {
  int c[8]; float v[8];
  __device__ __forceinline__ void load(const int32_t *col, const __nv_bfloat16 *val, int off) {
    const int4 c0 = __ldcs(reinterpret_cast<const int4 *>(col + off));
    const int4 c1 = __ldcs(reinterpret_cast<const int4 *>(col + off + 4));
    const uint4 raw = __ldcs(reinterpret_cast<const uint4 *>(val + off));
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[2 * q] = __uint_as_float(w[q] << 16);
      v[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
    }
  }
};

// The same P entries with 16-bit column deltas (P*2 bytes) instead of indices.
__device__ __forceinline__ int lo16(int w) { return (w << 16) >> 16; }
__device__ __forceinline__ int hi16(int w) { return w >> 16; }
template <typename VT, int P> struct DChunk;
template <> struct DChunk<double, 4> {
  int d[4]; double v[4];
  __device__ __forceinline__ void load(const int16_t *dcol, const double *val, int off) {
    const int2 di = __ldcs(reinterpret_cast<const int2 *>(dcol + off));
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(val + off));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(val + off + 2));
    d[0] = lo16(di.x); d[1] = hi16(di.x); d[2] = lo16(di.y); d[3] = hi16(di.y);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <> struct DChunk<float, 4> {
  int d[4]; float v[4];
  __device__ __forceinline__ void load(const int16_t *dcol, const float *val, int off) {
    const int2 di = __ldcs(reinterpret_cast<const int2 *>(dcol + off));
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(val + off));
    d[0] = lo16(di.x); d[1] = hi16(di.x); d[2] = lo16(di.y); d[3] = hi16(di.y);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <> struct DChunk<__nv_bfloat16, 8> {
  int d[8]; float v[8];
  __device__ __forceinline__ void load(const int16_t *dcol, const __nv_bfloat16 *val, int off) {
    const int4 di = __ldcs(reinterpret_cast<const int4 *>(dcol + off));
    const uint4 raw = __ldcs(reinterpret_cast<const uint4 *>(val + off));
    const int wd[4] = {di.x, di.y, di.z, di.w};
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d[2 * q] = lo16(wd[q]);
      d[2 * q + 1] = hi16(wd[q]);
      v[2 * q] = __uint_as_float(w[q] << 16);
      v[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
    }
  }
};

template <typename VT> struct LoadWidth { static constexpr int P = 4; };
template <> struct LoadWidth<__nv_bfloat16> { static constexpr int P = 8; };

// Loads in flight per lane and resident CTAs per SM of the SpMV, per value
// type: 3 chunks (12 entries) per iteration at 3 CTAs per SM for FP64 values
// (measured at 1024^2 with the 16-bit column deltas: 9 % faster than 4 chunks
// at 2 CTAs, and than 2 chunks at 3 CTAs), 4 chunks for FP32 and 2 (16
// entries) for BF16 at 3 CTAs per SM.  The FP64 projector form keeps 2 CTAs per
// SM (its walks need the registers; see spmv_min_blocks).
template <typename VT> struct SpmvTune { static constexpr int NCH = 3, MINB = 3; };
template <> struct SpmvTune<float> { static constexpr int NCH = 4, MINB = 3; };
template <> struct SpmvTune<__nv_bfloat16> { static constexpr int NCH = 2, MINB = 3; };

template <typename XT> struct AccT { using T = XT; };

// Row sum of one row for a group of LPR lanes (lane gl of the group), P
// entries per lane per chunk load.  Every iteration issues NCH chunk loads per
// lane (those past the row end are predicated off and contribute zero), so a
// row costs ceil(chunks / NCH) memory round trips instead of one per leftover
// chunk.  With the plan's default slot layout every slot of LPR chunks is
// stored lane-interleaved, so the gathers of one q across the group's lanes
// read consecutive entries of the row.
template <typename VT, int P>
__device__ __forceinline__ void load_or_zero(Chunk<VT, P> &c, const int32_t *col, const VT *val, int off, bool ok) {
  if (ok) {
    c.load(col, val, off);
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q) { c.c[q] = 0; c.v[q] = 0; }
  }
}

template <typename VT, int P>
__device__ __forceinline__ void load_or_zero(DChunk<VT, P> &c, const int16_t *dcol, const VT *val, int off, bool ok) {
  if (ok) {
    c.load(dcol, val, off);
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q) { c.d[q] = 0; c.v[q] = 0; }
  }
}

// D16: the columns are the running sums of the lane's 16-bit deltas from the
// row's base column `cur` (the lane walks its chunks in slot order, so the sum
// passes every entry of the lane once, in order; chunks past the row end add
// zero).  The entries, their order and the gathers are those of the 32-bit
// form, so both forms give the same sums bit for bit.
template <typename VT, typename XT, int LPR, bool D16>
__device__ __forceinline__ typename AccT<XT>::T row_dot(const SpmvParams<VT, XT> &p, const XT *__restrict__ x,
                                                       int beg, int end, int gl, int cur) {
  constexpr int P = LoadWidth<VT>::P;
  constexpr int NCH = SpmvTune<VT>::NCH;
  constexpr int STR = LPR * P;
  using ACC = typename AccT<XT>::T;
  ACC s0 = (ACC)0, s1 = (ACC)0;
  // Chunk slots (LPR*P entries each) of this group's row and the largest over
  // the warp: FP64 instructions cost a full issue slot whatever the number of
  // active lanes, so chunks past every group's row end are skipped outright
  // (warp-uniform branches) rather than multiplied by zero.
  const int nslot = (end - beg + STR - 1) / STR;
  const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)nslot);
#pragma unroll 1
  for (int j = 0; j < nmax; j += NCH) {
    const int off = beg + gl * P + j * STR;
    if constexpr (D16) {
      DChunk<VT, P> c[NCH];
#pragma unroll
      for (int h = 0; h < NCH; ++h) load_or_zero(c[h], p.dcol, p.val, off + h * STR, off + h * STR < end);
#pragma unroll
      for (int h = 0; h < NCH; ++h) {
        if (h > 0 && j + h >= nmax) break;
        ACC &s = (h & 1) ? s1 : s0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
          cur += c[h].d[q];
          s += (ACC)c[h].v[q] * (ACC)__ldg(x + cur);
        }
      }
    } else {
      Chunk<VT, P> c[NCH];
#pragma unroll
      for (int h = 0; h < NCH; ++h) load_or_zero(c[h], p.col, p.val, off + h * STR, off + h * STR < end);
#pragma unroll
      for (int h = 0; h < NCH; ++h) {
        if (h > 0 && j + h >= nmax) break;
        ACC &s = (h & 1) ? s1 : s0;
#pragma unroll
        for (int q = 0; q < P; ++q) s += (ACC)c[h].v[q] * (ACC)__ldg(x + c[h].c[q]);
      }
    }
  }
  return s0 + s1;
}

// MGS coefficients of a window through its Gram matrix (unit vectors):
// c_a = d_a sig_a - sum_{b<a} c_b <v_a, v_b>, for window vectors lo..lo+nd-1.
__device__ __forceinline__ void mgs_coefficients(const double *dots, int nd, int lo, int R, const double *sig,
                                                 const double (*gram)[kRing], double *c) {
  for (int a = 0; a < nd; ++a) {
    const int sa = ring_slot(lo + a, R);
    double v = dots[a] * sig[sa];
    for (int q = 0; q < a; ++q) v -= c[q] * gram[sa][ring_slot(lo + q, R)];
    c[a] = v;
  }
}

// Storage slot of window vector j: its ring slot, or (R == 0) column j - 1 of
// a matrix that keeps every vector (Z).
__device__ __forceinline__ int window_slot(int j, int R) { return R > 0 ? ring_slot(j, R) : j - 1; }

// The 32-row blocks of one warp: row0 = first, first + stride, ... below
// end; a block holds rows [row0, min(row0 + 32, end)).
struct RowBlocks {
  int64_t first, stride, end;
};

// A warp's rows, in 32-row blocks: groups of LPR lanes run one row each in
// LPR substeps; per-lane partial sums are stashed in shared memory and lane r
// adds its row's partials in order, so the output and ||y||^2 run with lane r
// owning row r and every FP64 instruction on a full warp.  Stored row r goes
// to output index orig[r] (when the rows are stored in another order).  LPR = 1
// is the vector pass (no matrix; the row value is b_r).
template <typename VT, typename XT, int LPR, bool MAT, bool ORIG, bool D16>
__device__ __forceinline__ double spmv_rows(const SpmvParams<VT, XT> &p, RowBlocks rb,
                                            const XT *__restrict__ x, XT *y, typename AccT<XT>::T *stash) {
  constexpr int G = 32 / LPR;
  using ACC = typename AccT<XT>::T;
  const int lane = threadIdx.x & 31;
  const int gl = lane % LPR, grp = lane / LPR;
  double nrm = 0.0;
  for (int64_t row0 = rb.first; row0 < rb.end; row0 += rb.stride) {
    const int64_t r1 = min(row0 + 32, rb.end);
    const int64_t row = row0 + lane;
    const bool valid = row < r1;
    ACC yv = (ACC)0;
    if (MAT) {
      // lane r holds rowptr[row0 + r]; rows past the block read rowptr[r1] (empty ranges)
      const int rp = p.rowptr[valid ? row : r1];
      const int rp_last = p.rowptr[r1];
      int rp_next = __shfl_down_sync(0xffffffffu, rp, 1);
      if (lane == 31) rp_next = rp_last;
      const int cb = D16 && valid ? p.rbase[row] : 0;
#pragma unroll 1
      for (int t = 0; t < LPR; ++t) {
        const int r = t * G + grp;
        const int beg = __shfl_sync(0xffffffffu, rp, r);
        const int end = __shfl_sync(0xffffffffu, rp_next, r);
        const int base = D16 ? __shfl_sync(0xffffffffu, cb, r) : 0;
        stash[t * 32 + lane] = row_dot<VT, XT, LPR, D16>(p, x, beg, end, gl, base);
      }
      __syncwarp();
      const int t = lane / G, g = lane % G;
      ACC s = (ACC)0;
#pragma unroll
      for (int l = 0; l < LPR; ++l) s += stash[t * 32 + g * LPR + l];
      __syncwarp();
      yv = s;
    } else {
      if (valid) yv = (ACC)p.b[row];
    }
    if (valid) {
      y[ORIG ? p.orig[row] : row] = (XT)yv;
      if (!MAT && p.wfull) p.wfull[row] = (XT)yv;
    }
    const double yd = valid ? (double)yv : 0.0;
    nrm += yd * yd;
  }
  return nrm;
}

// Window dots <v_j, y> over the warp's rows, after the products: lane r
// re-reads the output of row r it stored itself, so the row loop above keeps
// no per-window registers.
template <typename XT, int ND, bool ORIG>
__device__ __forceinline__ void spmv_window_dots(RowBlocks rb, const int32_t *orig, const XT *y, const XT *win,
                                                 int64_t wst, int R, int lo, double (&acc)[ND + 1]) {
  const int lane = threadIdx.x & 31;
  const XT *wv[ND > 0 ? ND : 1];
#pragma unroll
  for (int a = 0; a < ND; ++a) wv[a] = win + (size_t)window_slot(lo + a, R) * wst;
  for (int64_t row0 = rb.first; row0 < rb.end; row0 += rb.stride) {
    const int64_t row = row0 + lane;
    if (row < min(row0 + 32, rb.end)) {
      const int64_t o = ORIG ? orig[row] : row;
      const double yd = (double)y[o];
#pragma unroll
      for (int a = 0; a < ND; ++a) acc[1 + a] += (double)wv[a][o] * yd;
    }
  }
}

template <typename XT, int ND, bool ORIG>
__device__ __forceinline__ void spmv_finish(RowBlocks rb, const int32_t *orig, const XT *y, const XT *win,
                                            int64_t wst, int R, int lo, double nrm, double *outpart, double *wsum) {
  double acc[ND + 1];
  acc[0] = nrm;
#pragma unroll
  for (int a = 1; a <= ND; ++a) acc[a] = 0.0;
  spmv_window_dots<XT, ND, ORIG>(rb, orig, y, win, wst, R, lo, acc);
  __syncthreads();
  store_partials<ND + 1>(acc, wsum, outpart);
}

__host__ __device__ inline size_t spmv_smem_bytes(int lpr, size_t acc_bytes) {
  return acc_bytes * kWarps * 32 * (lpr > 1 ? lpr : 1);
}

// Draws of sketch column c in registers: the generator of sketch_table_kernel
// (same rows, same signs, same order); rows[q] = -1 past a draw-cap miss.
template <int Z>
__device__ __forceinline__ void sketch_column_draws(uint64_t seed, int64_t c, int s, int zeta, int (&rows)[Z],
                                                    uint32_t &neg) {
  int cnt = 0;
  neg = 0;
#pragma unroll
  for (int q = 0; q < Z; ++q) rows[q] = -1;
  for (uint32_t t = 0; cnt < zeta && t < 1000000u; ++t) {
    const uint64_t h = splitmix64_first(seed ^ (((uint64_t)c << 32) + t));
    const int r = (int)__umul64hi(h, (uint64_t)s);
    bool dup = false;
#pragma unroll
    for (int q = 0; q < Z; ++q) dup |= (rows[q] == r);
    if (dup) continue;
#pragma unroll
    for (int q = 0; q < Z; ++q)
      if (q == cnt) rows[q] = r;
    neg |= (uint32_t)(h & 1ull) << cnt;
    ++cnt;
  }
}

// round(v * 2^E) as a two's-complement integer, from the bit pattern (no
// floating-point instruction); |v| * 2^E < 2^62 is the caller's guarantee.
__device__ __forceinline__ long long to_fixed(double v, int E) {
  const long long bits = __double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  const unsigned long long mant = (unsigned long long)(bits & 0xFFFFFFFFFFFFFll) | (ex ? (1ull << 52) : 0ull);
  const int e2 = (ex ? ex : 1) - 1075 + E;   // v * 2^E = mant * 2^e2
  unsigned long long mag;
  if (e2 >= 0) mag = mant << min(e2, 9);
  else if (e2 > -64) mag = (mant + (1ull << (-e2 - 1))) >> (-e2);   // half rounds up in magnitude
  else mag = 0;
  return bits < 0 ? -(long long)mag : (long long)mag;
}

// Fused sparse-sign sketch of the product output (Section 2.7 draws): this
// CTA's record rec[r * cap + blockIdx.x] = sum over the CTA's outputs y[o] of
// +-y[o] for the zeta rows r drawn for column o (the scale 1/sqrt(zeta) and
// the output's scale are applied where the records are reduced).
// The CTA's outputs are those of its rows [first, end) (through orig for
// pixel-tiled rows), taken in 32-row blocks round-robin over the warps, so
// the work is even whatever the warps' row counts.  The terms are fixed-point
// integers round(+-y[o] * 2^E) and the sums exact, so their order does not
// matter: shared-memory atomics into acc (s words, zeroed before the row loop),
// bitwise reproducible.  E is the CTA's, from its sum of squares (wn: the
// warps' totals of the lanes' nrm partials) and output count n: every entry
// is at most sqrt(n) * ||y_CTA|| in magnitude and 2^E times that is below
// 2^61.  One term's rounding is at most 2^-E / 2, about n * 2^-62 times the
// outputs' rms.  All threads call, after a barrier that follows the rows and
// the warps' writes of wn.
template <typename XT, bool ORIG, int Z>
__device__ __noinline__ void spmv_sketch(int s, int zeta, uint64_t seed, int64_t first, int64_t end,
                                         const int32_t *orig, const XT *y, const double *wn,
                                         unsigned long long *acc, double *rec, int cap) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double ss = 0.0;
  for (int w = 0; w < kWarps; ++w) ss += wn[w];
  const double bound = sqrt((double)(end - first)) * sqrt(ss);
  const bool live = bound > 0.0 && isfinite(bound);   // non-finite outputs stop the solve elsewhere
  int E = 0;
  if (live) {
    int ex;
    frexp(bound, &ex);   // bound < 2^ex
    E = 61 - ex;
    for (int64_t row = first + 32 * warp + lane; row < end; row += 32 * kWarps) {
      const int64_t o = ORIG ? orig[row] : row;
      const long long f = to_fixed((double)y[o], E);
      int rows[Z];
      uint32_t neg;
      sketch_column_draws<Z>(seed, o, s, zeta, rows, neg);
#pragma unroll
      for (int q = 0; q < Z; ++q)
        if (q < zeta && rows[q] >= 0) atomicAdd(acc + rows[q], (unsigned long long)(((neg >> q) & 1u) ? -f : f));
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < s; r += kThreads)
    rec[(size_t)r * cap + blockIdx.x] = live ? ldexp((double)(long long)acc[r], -E) : 0.0;
}

// Scalars booked by CTA 0 of a product (all its threads call): it stages the
// solve state, reduces the records of the kernel before the product and
// writes the step's scalars to the device state.  The other CTAs never need
// them: products store unscaled outputs and their consumers apply the scale.
template <typename VT, typename XT>
__device__ __noinline__ void spmv_bookkeeping(const SpmvParams<VT, XT> &p, int k, SolveState *sst, double *tot) {
  stage_state(p.st, sst);
  SolveState *st = p.st;
  const bool t0 = threadIdx.x == 0;
  if (p.mode == kModeInitBwd) {
    // beta_1 = ||b||, w_1 = b / beta_1
    reduce_partials_n<1>(p.part.b, p.G_prev, tot);
    if (!t0) return;
    const double beta = sqrt(tot[0]);
    st->beta0 = beta;
    st->sig_w[ring_slot(1, p.RW)] = 1.0 / beta;
    if (p.sigWall) p.sigWall[0] = 1.0 / beta;
    st->tol = (sst->noise_norm > 0.0) ? sst->eta * sst->noise_norm / beta : 0.0;
    if (!(beta > 0.0)) st->stop = SFL_STOP_BREAKDOWN;
    if (!isfinite(tot[0])) st->stop = kStopNonfinite;
  } else if (p.mode == kModeFwd) {
    // alpha_k = ||p~_k|| from the z update; breakdown test; Gram row of p_k (of z_k when the z window is Z)
    const int lz = max(1, k - p.ell), ndz = p.full ? 0 : k - lz;   // window of the z update
    reduce_partials(p.part.p, p.G_prev, 1 + ndz, nullptr, tot);
    if (!t0) return;
    const double alpha = sqrt(tot[0]);
    const bool bad = !(alpha > 1e-300) || !(alpha > 1e-14 * sqrt(sst->znorm_raw2)) || !isfinite(tot[0]);
    if (bad) {
      st->stop = isfinite(tot[0]) ? SFL_STOP_BREAKDOWN : kStopNonfinite;
      return;
    }
    const double ia = 1.0 / alpha;
    const int ns = ring_slot(k, p.RP);
    st->alpha = alpha;
    st->sig_p[ns] = ia;
    p.sigZ[k - 1] = ia;
    for (int a = 0; a < ndz; ++a) {
      const int sa = ring_slot(lz + a, p.RP);
      const double g = tot[1 + a] * sst->sig_p[sa] * ia;
      st->gram_p[ns][sa] = g; st->gram_p[sa][ns] = g;
    }
  } else {   // kModeBwd
    // beta_{k+1} = ||w~_{k+1}|| from the w update; lucky-breakdown test; Gram row of w_{k+1}
    const int lw = max(1, k - p.ell), ndw = p.full ? 0 : k - lw + 1;   // window of the w update
    reduce_partials(p.part.wn, p.G_prev, 1 + ndw, nullptr, tot);
    if (!t0) return;
    const double beta = sqrt(tot[0]);
    if (!isfinite(tot[0])) {
      st->stop = kStopNonfinite;
    } else if (!(beta > 1e-300) || !(beta > 1e-14 * sqrt(sst->wnorm_raw2))) {
      st->lucky = 1;                 // step k is still solved; there is no w_{k+1}
      st->betak = 0.0;
    } else {
      const double ib = 1.0 / beta;
      const int ns = ring_slot(k + 1, p.RW);
      st->betak = beta;
      st->sig_w[ns] = ib;
      if (p.want_h) p.Hband[(size_t)(k - 1) * (p.hb_ell + 2) + p.hb_ell + 1] = beta;
      if (p.sigWall) p.sigWall[k] = ib;
      for (int a = 0; a < ndw; ++a) {
        const int sa = ring_slot(lw + a, p.RW);
        const double g = tot[1 + a] * sst->sig_w[sa] * ib;
        st->gram_w[ns][sa] = g; st->gram_w[sa][ns] = g;
      }
    }
  }
}

// Forms of the product kernel: the vector pass (y = b), the matrix form, the
// matrix form writing through an original-row map (pixel-tiled rows; a
// compile-time form, so untiled operators carry no dependent index load), the
// matrix-free projector form (proj.cuh), and the two matrix forms reading
// 16-bit column deltas (StoredCsr::dcol) instead of 32-bit indices.
enum : int { kSpmvVec = 0, kSpmvMat = 1, kSpmvMatOrig = 2, kSpmvProj = 3, kSpmvMat16 = 4, kSpmvMatOrig16 = 5 };
// Lanes per row of the 16-bit delta forms (the only width they are built for).
constexpr int kDeltaLpr = 8;
// Resident CTAs per SM the product kernel is compiled for: the FP64 projector
// walks (fixed-point columns, stepped bin coordinates) keep 2.
template <typename VT> constexpr int spmv_min_blocks(int form) {
  return form == kSpmvProj && sizeof(VT) == 8 ? 2 : SpmvTune<VT>::MINB;
}

// The rows of a warp for the projector form, in 32-row blocks: lane r walks
// ray r of the block (A x), or, for a back-projection, the lanes' parts of
// each row are added by a butterfly and lane r keeps row r's value; lane r
// then writes it and its square as the stored form does.
template <typename VT, typename XT>
__device__ __forceinline__ double proj_rows(const SpmvParams<VT, XT> &p, RowBlocks rb, const XT *__restrict__ x, XT *y) {
  using RT = typename AccT<XT>::T;
  const int lane = threadIdx.x & 31;
  const RT *tab = reinterpret_cast<const RT *>(p.ptab);
  double nrm = 0.0;
  for (int64_t row0 = rb.first; row0 < rb.end; row0 += rb.stride) {
    const int64_t r1 = min(row0 + 32, rb.end);
    RT mine = RT(0);
    if (p.proj == kProjRay) {
      if (row0 + lane < r1) mine = proj_ray<RT, XT>(p.pN, p.pnb, tab, x, row0 + lane);
    } else if (std::is_same<RT, double>::value && p.proj == kProjBackLinear) {
      mine = (RT)proj_back_linear_block<XT>(p.pN, p.pna, p.pnb, reinterpret_cast<const double *>(p.ptab), p.pfix, x,
                                            row0, r1, lane);
    } else {
      for (int64_t row = row0; row < r1; ++row) {
        RT v = proj_back_partial<RT, XT>(p.proj, p.pN, p.pna, p.pnb, tab, x, row, lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == (int)(row - row0)) mine = v;
      }
    }
    const int64_t row = row0 + lane;
    if (row < r1) {
      y[row] = (XT)mine;
      const double yd = (double)(XT)mine;
      nrm += yd * yd;
    }
  }
  return nrm;
}

// Fused SpMV of one step.  In the solve modes past the first vector pass,
// CTA 0 books the step's scalars (above) while the other CTAs run the rows:
// outputs are stored unscaled (y = A x for the stored, unnormalised x), with
// ||y||^2 and the window dots <v_j, y> as per-CTA records (CTA 0's are zero).
template <typename VT, typename XT, int LPR, int FORM>
__global__ void __launch_bounds__(kThreads, spmv_min_blocks<VT>(FORM)) spmv_fused_kernel(SpmvParams<VT, XT> p) {
  constexpr bool MAT = FORM != kSpmvVec, ORIG = FORM == kSpmvMatOrig || FORM == kSpmvMatOrig16;
  constexpr bool D16 = FORM == kSpmvMat16 || FORM == kSpmvMatOrig16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SolveState sst;
  __shared__ double wsum[(kMaxWindow + 2) * kThreads];   // reduction scratch
  __shared__ double tot[kPartStride];
  // a launch with too little shared memory does nothing (never writes out of bounds)
  if (dynamic_smem_bytes() < spmv_smem_bytes(LPR, sizeof(typename AccT<XT>::T))) return;
  if (p.sk_s && dynamic_smem_bytes() < spmv_smem_bytes(LPR, sizeof(typename AccT<XT>::T)) +
                                        sizeof(unsigned long long) * (size_t)p.sk_s)
    return;
  griddep_wait();
  griddep_launch_dependents();
  int k = 0, lo = 1, nd = 0;
  const XT *x = p.x;
  XT *y = p.y;
  const XT *win = nullptr; int64_t wst = 0; int R = 1;
  double *outpart = nullptr;
  bool reduce = true;
  int rcta = blockIdx.x, ncta = gridDim.x;   // this CTA among the row CTAs
  if (p.mode == kModeApply) {
    reduce = false;
  } else {
    if (__ldcg(&p.st->stop)) return;
    k = __ldcg(&p.st->k) + 1;
    if (p.mode == kModeInitB) {
      y = p.wring + (size_t)ring_slot(1, p.RW) * p.wstride;
      outpart = p.part.b;
    } else if (p.mode == kModeInitBwd) {
      x = p.wring + (size_t)ring_slot(1, p.RW) * p.wstride;
      y = p.zraw;
      outpart = p.part.z;
    } else if (p.mode == kModeFwd) {
      x = p.Z + (size_t)(k - 1) * p.zstride;
      y = p.wraw;
      lo = max(1, k - p.ell); nd = p.full ? 0 : k - lo + 1;
      win = p.wring; wst = p.wstride; R = p.RW;
      outpart = p.part.w;
    } else {  // kModeBwd
      x = p.wring + (size_t)ring_slot(k + 1, p.RW) * p.wstride;
      y = p.zraw;
      lo = max(1, k + 1 - p.ell); nd = p.full ? 0 : k - lo + 1;
      if (p.orth_z) { win = p.Z; wst = p.zstride; R = 0; }   // column j - 1 holds z~_j
      else { win = p.pring; wst = p.pstride; R = p.RP; }
      outpart = p.part.z;
    }
    if (p.mode != kModeInitB) {
      if (blockIdx.x == 0) {
        if (threadIdx.x < kPartStride) outpart[(size_t)threadIdx.x * kPartCap] = 0.0;   // CTA 0's record
        if (p.sk_s)
          for (int r = threadIdx.x; r < p.sk_s; r += kThreads) p.sk_rec[(size_t)r * p.sk_cap] = 0.0;
        spmv_bookkeeping(p, k, &sst, tot);
        return;
      }
      rcta = blockIdx.x - 1;
      ncta = gridDim.x - 1;
    }
  }
  // this warp's rows: the products, then the window dots and the partial record
  using ACC = typename AccT<XT>::T;
  const int warp = threadIdx.x >> 5;
  ACC *stash = reinterpret_cast<ACC *>(smem_raw) + warp * 32 * (LPR > 1 ? LPR : 1);
  // fused sketch: the CTA's s-vector follows the stash
  unsigned long long *sk_acc = reinterpret_cast<unsigned long long *>(
      smem_raw + spmv_smem_bytes(LPR, sizeof(typename AccT<XT>::T)));
  if (p.sk_s)
    for (int r = threadIdx.x; r < p.sk_s; r += kThreads) sk_acc[r] = 0ull;
  // this warp's blocks: its own balanced range, or (tiled operators) every
  // kWarps-th block of the CTA's range, so the CTA's warps work on one tile
  const int gw = rcta * kWarps + warp;
  auto bound = [&](int64_t w) {
    return p.wrow ? (int64_t)p.wrow[w] : (p.rows * w) / ((int64_t)ncta * kWarps);
  };
  RowBlocks rb;
  if (FORM == kSpmvProj && p.proj == kProjRay && !p.sk_s) {
    // one thread per ray: whole 32-ray blocks, dealt warp-major so that a
    // CTA's warps take blocks from across the sinogram (a ray at the centre of
    // an angle's bins crosses up to N columns, one at its edge a few).  With
    // the fused sketch the CTA keeps its contiguous range, which the sketch
    // epilogue reads back.
    rb.first = 32 * ((int64_t)warp * ncta + rcta);
    rb.stride = 32 * (int64_t)ncta * kWarps;
    rb.end = p.rows;
  } else if (p.interleave) {
    rb.first = bound((int64_t)rcta * kWarps) + 32 * warp;
    rb.stride = 32 * kWarps;
    rb.end = bound((int64_t)(rcta + 1) * kWarps);
  } else {
    rb.first = bound(gw);
    rb.stride = 32;
    rb.end = bound(gw + 1);
  }
  double nrm;
  if constexpr (FORM == kSpmvProj) nrm = proj_rows<VT, XT>(p, rb, x, y);
  else nrm = spmv_rows<VT, XT, LPR, MAT, ORIG, D16>(p, rb, x, y, stash);
  if (!reduce) return;
  const int32_t *og = p.orig;
  if (p.sk_s) {   // the warps' sums of squares for the sketch's scale (tot is CTA 0's scratch)
    const double wn = warp_sum(nrm);
    if ((threadIdx.x & 31) == 0) tot[warp] = wn;
  }
  if (!MAT) {     // vector pass: no window dots
    spmv_finish<XT, 0, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum);
    return;
  }
  switch (nd) {   // the window size is a compile-time constant inside the tail
    case 0: spmv_finish<XT, 0, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 1: spmv_finish<XT, 1, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 2: spmv_finish<XT, 2, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 3: spmv_finish<XT, 3, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 4: spmv_finish<XT, 4, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 5: spmv_finish<XT, 5, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 6: spmv_finish<XT, 6, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 7: spmv_finish<XT, 7, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    case 8: spmv_finish<XT, 8, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
    default: spmv_finish<XT, 9, ORIG>(rb, og, y, win, wst, R, lo, nrm, outpart, wsum); break;
  }
  if (p.sk_s) {
    __syncthreads();   // every row done: the outputs and the warps' norms are visible
    const int64_t first = bound((int64_t)rcta * kWarps), last = bound((int64_t)(rcta + 1) * kWarps);
    const uint64_t sd = __ldcg(&p.st->seed) + p.sk_seed_add;
    if (p.sk_zeta <= 8)
      spmv_sketch<XT, ORIG, 8>(p.sk_s, p.sk_zeta, sd, first, last, og, y, tot, sk_acc, p.sk_rec, p.sk_cap);
    else
      spmv_sketch<XT, ORIG, kMaxZeta>(p.sk_s, p.sk_zeta, sd, first, last, og, y, tot, sk_acc, p.sk_rec, p.sk_cap);
  }
}

// Row cost for the warp partition of a product, in quarter iterations: the
// row's load iterations (ceil(len / unit), unit = entries one iteration of its
// lane group covers), plus, when slot > 0, its chunk slots (ceil(len / slot),
// the FMA instructions it issues: on this GPU an FP64 instruction costs a full
// issue slot whatever the number of active lanes), plus one quarter for the
// row's share of the per-row work.  Warps over short rows run more iterations
// per stored entry than warps over long rows, so entries alone do not balance.
// When cost_x is given it gets the cost plus `extra` quarters per row, the
// price of the fused sketch's per-output work (CTA ranges are balanced on it).
static __global__ void row_cost_kernel(const int32_t *rowptr, int64_t rows, int unit, int slot, int extra,
                                       int64_t *cost, int64_t *cost_x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > rows) return;
  if (i == rows) {
    cost[i] = 0;
    if (cost_x) cost_x[i] = 0;
    return;
  }
  const int len = rowptr[i + 1] - rowptr[i];
  int64_t c = 4 * (int64_t)((len + unit - 1) / unit) + 1;
  if (slot > 0) c += 4 * (int64_t)((len + slot - 1) / slot);
  cost[i] = c;
  if (cost_x) cost_x[i] = c + extra;
}

// First row in [lo, hi) whose prefix reaches target (hi when none does).
__device__ __forceinline__ int64_t first_at_least(const int64_t *prefix, int64_t lo, int64_t hi, int64_t target) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] < target) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Two-level row ranges for products whose CTAs also sketch their outputs:
// CTA c's range [B_c, B_{c+1}) splits the cost with the sketch's price
// (prefix_x) evenly over the nc CTAs, and the range's warps split its row-loop
// cost (prefix) evenly, since the CTA's sketch work is spread over all its
// warps.  wrow has nc * kWarps + 1 entries.
static __global__ void balance_rows2_kernel(const int64_t *prefix, const int64_t *prefix_x, int64_t rows, int nc,
                                            int32_t *wrow) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > nc) return;
  if (c == nc) { wrow[(size_t)nc * kWarps] = (int32_t)rows; return; }
  const int64_t tx = prefix_x[rows];
  const int64_t b0 = first_at_least(prefix_x, 0, rows, (int64_t)(((__int128)tx * c) / nc));
  const int64_t b1 = c + 1 == nc ? rows : first_at_least(prefix_x, 0, rows, (int64_t)(((__int128)tx * (c + 1)) / nc));
  const int64_t p0 = prefix[b0], p1 = prefix[b1];
  for (int j = 0; j < kWarps; ++j)
    wrow[(size_t)c * kWarps + j] =
        (int32_t)(j == 0 ? b0 : first_at_least(prefix, b0, b1, p0 + (int64_t)(((__int128)(p1 - p0) * j) / kWarps)));
}

// Row range of every warp: warp w starts at the first row whose cost prefix
// reaches w/W of the total (prefix[rows] = total).
static __global__ void balance_rows_kernel(const int64_t *prefix, int64_t rows, int W, int32_t *wrow) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > W) return;
  const int64_t total = prefix[rows];
  const int64_t target = (int64_t)(((__int128)total * w) / W);
  int64_t lo = 0, hi = rows;          // first row whose start is >= target
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] < target) lo = mid + 1; else hi = mid;
  }
  wrow[w] = (int32_t)(w == W ? rows : lo);
}

// ---------------------------------------------------------------- sketch (gather form)

// Draws of every column as (row, column | sign bit) pairs in column-major
// order, for the stable sort that builds the row-major sketch table.
static __global__ void sketch_pairs_kernel(uint64_t seed, int s, int zeta, int64_t ncols, uint32_t *keys,
                                           uint32_t *vals, int *err) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  int rows[kMaxZeta];
  int cnt = 0;
  for (uint32_t t = 0; cnt < zeta && t < 1000000u; ++t) {
    const uint64_t h = splitmix64_first(seed ^ (((uint64_t)c << 32) + t));
    const int r = (int)__umul64hi(h, (uint64_t)s);
    bool dup = false;
    for (int q = 0; q < cnt; ++q) dup |= (rows[q] == r);
    if (dup) continue;
    rows[cnt] = r;
    keys[c * zeta + cnt] = (uint32_t)r;
    vals[c * zeta + cnt] = (uint32_t)c | ((uint32_t)(h & 1ull) << 31);
    ++cnt;
  }
  if (cnt < zeta) {            // never expected; keep every entry in range and report it
    atomicExch(err, 1);
    for (; cnt < zeta; ++cnt) { keys[c * zeta + cnt] = 0u; vals[c * zeta + cnt] = (uint32_t)c; }
  }
}

// Row pointer of the sorted sketch table: first entry of each row.
static __global__ void sketch_rowptr_kernel(const uint32_t *keys, int64_t nent, int s, int32_t *rowptr) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r > s) return;
  int64_t lo = 0, hi = nent;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)keys[mid] < r) lo = mid + 1; else hi = mid;
  }
  rowptr[r] = (int32_t)lo;
}

enum SketchMode : int {
  kSkPlain = 0,    // sk_out = S v (v FP64)
  kSkInitB = 1,    // S_m b: sFLSQR right-hand side, or sFLSMR's residual-rule S_m b
  kSkInitBwd = 2,  // sFLSMR: S_n A^T w_1 -> first column of S A^T W, right-hand side beta * it
  kSkStep = 3      // S_m w (LS column / stop column) and, for sFLSMR, S_n z (new column of S A^T W)
};

template <typename XT>
struct SketchParams {
  int mode, method, s;
  double isz;                              // 1 / sqrt(zeta)
  SolveState *st;
  const double *v64;                       // kSkPlain / kSkInitB input
  const XT *wraw, *zraw;                   // kSkStep / kSkInitBwd inputs (unscaled product outputs)
  int RW, RP;                               // ring sizes (slots of the scales of wraw and zraw)
  const int32_t *rowM; const uint32_t *entM;   // m-side table (S_m)
  const int32_t *rowN; const uint32_t *entN;   // n-side table (S_n)
  const double *dM, *dN;                       // explicit sketches (row-major s x m, s x n) instead of the tables
  int64_t lenM, lenN;
  int gen;                                     // generated sketch (sfl_sketch_kind SRHT or GAUSSIAN), 0: none
  int bitsM, bitsN;                            // SRHT: log2 of the padded lengths
  int gen_m_add;                               // the m-side sketch's seed is the solve's seed plus this
  double *SAZ, *SAtW, *rhs, *e, *sbm, *sk_out;
};

// One CTA of kSkWarps warps per sketch row: sum of +-v[c] over the row's
// entries (threads strided, four independent accumulators, warp butterflies,
// warps added in order), times 1/sqrt(zeta).  The sign is applied to the bit
// pattern, so each entry costs one add.  Vectors held in FP64 accumulate in
// FP64; reduced-precision vectors accumulate in FP32.  Rows rows_total =
// (number of sketches) * s, one CTA each.
constexpr int kSkWarps = 4;

__device__ __forceinline__ double flip_sign(double v, uint32_t e) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(e >> 31) << 63));
}
__device__ __forceinline__ float flip_sign(float v, uint32_t e) {
  return __uint_as_float(__float_as_uint(v) ^ (e & 0x80000000u));
}

template <typename T, typename VT>
__device__ __forceinline__ T sketch_row_sum(const int32_t *rowptr, const uint32_t *ent, const VT *v, int r) {
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  constexpr int B = kSkWarps * 32;
  const int b0 = rowptr[r], b1 = rowptr[r + 1];
  int i = b0 + threadIdx.x;
  for (; i + 3 * B < b1; i += 4 * B) {
    const uint32_t e0 = __ldg(ent + i), e1 = __ldg(ent + i + B), e2 = __ldg(ent + i + 2 * B), e3 = __ldg(ent + i + 3 * B);
    a0 += flip_sign((T)v[e0 & 0x7FFFFFFFu], e0);
    a1 += flip_sign((T)v[e1 & 0x7FFFFFFFu], e1);
    a2 += flip_sign((T)v[e2 & 0x7FFFFFFFu], e2);
    a3 += flip_sign((T)v[e3 & 0x7FFFFFFFu], e3);
  }
  for (; i < b1; i += B) {
    const uint32_t e = __ldg(ent + i);
    a0 += flip_sign((T)v[e & 0x7FFFFFFFu], e);
  }
  return warp_sum((a0 + a1) + (a2 + a3));
}

// Row r of an explicit sketch times v: the row's len entries, threads
// strided, four independent accumulators, then a warp butterfly.
template <typename T, typename VT>
__device__ __forceinline__ T dense_row_sum(const double *Srow, const VT *v, int64_t len) {
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  constexpr int B = kSkWarps * 32;
  int64_t i = threadIdx.x;
  for (; i + 3 * B < len; i += 4 * B) {
    a0 += (T)Srow[i] * (T)v[i];
    a1 += (T)Srow[i + B] * (T)v[i + B];
    a2 += (T)Srow[i + 2 * B] * (T)v[i + 2 * B];
    a3 += (T)Srow[i + 3 * B] * (T)v[i + 3 * B];
  }
  for (; i < len; i += B) a0 += (T)Srow[i] * (T)v[i];
  return warp_sum((a0 + a1) + (a2 + a3));
}

// Generated sketches (sfl_opts.sketch_kind): every application regenerates
// the entries from the seed; nothing is stored.
//   SRHT: S[r, c] = (-1)^(popcount(rho(r) & c) + d_c) / sqrt(s), the sampled
//   rows rho(r) of the Sylvester-Hadamard matrix of order M = 2^b >= len
//   given by a seeded bijection of [0, M) (xor-shifts and an odd multiplier),
//   d_c a sign bit of the hash;
//   GAUSSIAN: S[r, c] = sqrt(-2 ln u1) cos(2 pi u2) / sqrt(s), u1 and u2 the
//   top 53 bits of two hash outputs of the counter r * len + c (Box-Muller).
// The factor 1/sqrt(s) is applied by the caller.
constexpr uint64_t kTagSrht = 0x5352485400000000ull, kTagSign = 0x5352485400000001ull,
                   kTagGauss = 0x4741555353000000ull;

__device__ __forceinline__ uint32_t srht_row(uint64_t seed, uint32_t r, int b) {
  const uint64_t k = splitmix64_first(seed ^ kTagSrht);
  const uint32_t mask = (uint32_t)((1ull << b) - 1ull), K = (uint32_t)(k >> 32) | 1u;
  const int h = max(1, b / 2);
  uint32_t x = (r ^ (uint32_t)k) & mask;
  for (int i = 0; i < 2; ++i) {
    x ^= x >> h;
    x = (x * K) & mask;
  }
  return x ^ (x >> h);
}

__device__ __forceinline__ double gaussian_entry(uint64_t seed, uint64_t key) {
  const uint64_t base = seed ^ kTagGauss;
  const uint64_t h1 = splitmix64_first(base ^ (2ull * key)), h2 = splitmix64_first(base ^ (2ull * key + 1ull));
  const double u1 = ((double)(h1 >> 11) + 1.0) * 0x1p-53, u2 = (double)(h2 >> 11) * 0x1p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Row r of a generated sketch (without the 1/sqrt(s)) times v: threads
// strided over the columns, two accumulators, then a warp butterfly.
template <typename T, typename VT>
__device__ __forceinline__ T gen_row_sum(int kind, uint64_t seed, int r, int b, const VT *v, int64_t len) {
  T a0 = 0, a1 = 0;
  constexpr int B = kSkWarps * 32;
  if (kind == SFL_SKETCH_SRHT) {
    const uint32_t rho = srht_row(seed, (uint32_t)r, b);
    const uint64_t sg = seed ^ kTagSign;
    int64_t c = threadIdx.x;
    for (; c + B < len; c += 2 * B) {
      const uint32_t p0 = (__popc(rho & (uint32_t)c) + (uint32_t)(splitmix64_first(sg ^ (uint64_t)c) >> 63)) & 1u;
      const uint32_t p1 =
          (__popc(rho & (uint32_t)(c + B)) + (uint32_t)(splitmix64_first(sg ^ (uint64_t)(c + B)) >> 63)) & 1u;
      const T x0 = (T)v[c], x1 = (T)v[c + B];
      a0 += p0 ? -x0 : x0;
      a1 += p1 ? -x1 : x1;
    }
    for (; c < len; c += B) {
      const uint32_t p0 = (__popc(rho & (uint32_t)c) + (uint32_t)(splitmix64_first(sg ^ (uint64_t)c) >> 63)) & 1u;
      const T x0 = (T)v[c];
      a0 += p0 ? -x0 : x0;
    }
  } else {
    const uint64_t row0 = (uint64_t)r * (uint64_t)len;
    for (int64_t c = threadIdx.x; c < len; c += B) a0 += (T)gaussian_entry(seed, row0 + (uint64_t)c) * (T)v[c];
  }
  return warp_sum(a0 + a1);
}

// This lane's parts of the sums of two rows of per-CTA sketch records
// (ra, and rb when rb is given), records lane, lane + 32, ... of each: loads
// in batches of 16 per row (one batch covers 512 records), all issued before
// the batch is added in a fixed order.
__device__ __forceinline__ void sum_records2(const double *ra, const double *rb, int cap, int lane, double &a,
                                             double &b) {
  a = 0.0;
  b = 0.0;
  for (int b0 = lane; b0 < cap; b0 += 16 * 32) {
    double va[16], vb[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const bool in = b0 + 32 * j < cap;
      va[j] = in ? __ldcg(ra + b0 + 32 * j) : 0.0;
      vb[j] = in && rb ? __ldcg(rb + b0 + 32 * j) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) { a += va[j]; b += vb[j]; }
  }
}

template <typename XT>
__global__ void __launch_bounds__(kSkWarps * 32) sketch_rows_kernel(SketchParams<XT> p, int rows_total) {
  __shared__ double wpart[kSkWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gr = blockIdx.x;
  if (gr >= rows_total) return;
  griddep_wait();
  griddep_launch_dependents();
  int k = 0;
  double beta = 1.0, vscale = 1.0;
  const int which = gr / p.s, r = gr % p.s;
  if (p.mode != kSkPlain) {
    const SolveState *st = p.st;
    if (__ldcg(&st->stop)) return;
    k = __ldcg(&st->k) + 1;
    if (p.mode == kSkStep && gr >= p.s && __ldcg(&st->lucky)) return;   // no z at a lucky breakdown
    if (p.mode == kSkInitBwd) beta = __ldcg(&st->beta0);
    // scale of the unscaled product output: 1/alpha_k for A z_k, 1/beta_{k+1} for A^T w_{k+1}
    if (p.mode == kSkInitBwd) vscale = __ldcg(&st->sig_w[ring_slot(1, p.RW)]);
    else if (p.mode == kSkStep) vscale = which == 0 ? __ldcg(&st->sig_p[ring_slot(k, p.RP)])
                                                    : __ldcg(&st->sig_w[ring_slot(k + 1, p.RW)]);
  }
  const bool nside = (p.mode == kSkInitBwd) || (p.mode == kSkStep && which == 1);
  const int32_t *rowptr = nside ? p.rowN : p.rowM;
  const uint32_t *ent = nside ? p.entN : p.entM;
  double t;
  const double *dmat = nside ? p.dN : p.dM;
  if (p.gen) {
    const int64_t len = nside ? p.lenN : p.lenM;
    const uint64_t seed = __ldcg(&p.st->seed) + (nside ? 0 : p.gen_m_add);
    const int b = nside ? p.bitsN : p.bitsM;
    if (p.mode == kSkInitB) t = gen_row_sum<double>(p.gen, seed, r, b, p.v64, len);
    else t = (double)gen_row_sum<typename AccT<XT>::T>(p.gen, seed, r, b, nside ? p.zraw : p.wraw, len);
  } else if (dmat) {
    const int64_t len = nside ? p.lenN : p.lenM;
    const double *Srow = dmat + (size_t)r * len;
    if (p.mode == kSkInitB) t = dense_row_sum<double>(Srow, p.v64, len);
    else t = (double)dense_row_sum<typename AccT<XT>::T>(Srow, nside ? p.zraw : p.wraw, len);
  } else if (p.mode == kSkPlain || p.mode == kSkInitB) {
    t = sketch_row_sum<double>(rowptr, ent, p.v64, r);
  } else {
    t = (double)sketch_row_sum<typename AccT<XT>::T>(rowptr, ent, nside ? p.zraw : p.wraw, r);
  }
  if (lane == 0) wpart[warp] = t;
  __syncthreads();
  if (threadIdx.x != 0) return;
  static_assert(kSkWarps == 4, "warp totals are added as a pair of pairs");
  const double v = ((wpart[0] + wpart[1]) + (wpart[2] + wpart[3])) * p.isz * vscale;
  if (p.mode == kSkPlain) {
    p.sk_out[r] = v;
  } else if (p.mode == kSkStep) {
    if (which == 0) p.SAZ[(size_t)(k - 1) * p.s + r] = v;
    else p.SAtW[(size_t)k * p.s + r] = v;
  } else if (p.mode == kSkInitB) {
    if (p.method == kSFLSQR) { p.rhs[r] = v; p.e[r] = v; }
    else p.sbm[r] = v;
  } else {   // kSkInitBwd
    p.SAtW[r] = v;
    p.rhs[r] = beta * v;
    p.e[r] = beta * v;
  }
}

// ---------------------------------------------------------------- orthogonalization updates

template <typename XT>
struct OrthParams {
  int scale_ring;     // size of the ring whose scale of slot k applies to raw (w ring for z, p ring for w)
  SolveState *st;
  int side;            // 0: z side (p ring, tau, Z), 1: w side (w ring)
  int orth_z;          // z side: the window is the stored z~_j (Z columns) instead of the p ring
  int ell;
  int method;
  int G_prev;          // CTAs of the product kernel whose partials this one reduces
  int64_t len;
  const XT *raw;       // z (n) or w (m) before orthogonalization
  XT *ring; int64_t stride; int R;
  XT *Z; int64_t zstride;   // z side: Z columns
  const double *sigZ;
  int precond;
  const double *diag_w;     // SFL_PRECOND_DIAG
  const double *y;          // LS solution y_{k-1} (SFL_PRECOND_REWEIGHT)
  double *Hband;            // column k of H (rows lo..k) when want_h
  int want_h;               // H is recorded (sFLSMR, FLSQR)
  int full;                 // full orthogonalization: the block CGS2 kernels already orthogonalized raw
  XT *vfull;                // full: every new vector is also stored at column newj - 1
  // w side, fused sketch: the A z_k product's per-CTA records (sk_cap per
  // sketch row) -> column k of S A Z (sk_col, s entries), scaled by
  // 1/sqrt(zeta) and the product output's scale
  const double *sk_rec;
  int sk_cap, sk_s;
  double *sk_col_base;      // S A Z; column k - 1 starts at (k - 1) * sk_s
  double sk_isz;
  Partials part;
};

// z side: p~_k = z - sum_{j=lo}^{k-1} c_j v_j, z~_k = tau_k(p~_k), with v_j = p_j
// (or z_j when orth_z);
// w side: w~_{k+1} = w - sum_{j=lo}^{k} h_j w_j.
// Stores this CTA's ||new||^2 and <new, v~_j> over the window (<z~_k, z~_j>
// when orth_z: the Gram row the next steps' coefficients need).  ND (the
// window size) is a compile-time constant, so no FP64 instruction is issued
// for an unused window slot.
template <typename XT, int ND>
__device__ __forceinline__ void orth_run(const OrthParams<XT> &p, const SolveState &sst, int k, int lo, int newj,
                                         const double *coefs, const double *s_c, bool reweight, double *wsum,
                                         double rs) {
  double coef[ND > 0 ? ND : 1];
  const XT *vj[ND > 0 ? ND : 1];
#pragma unroll
  for (int a = 0; a < ND; ++a) {
    const int slot = ring_slot(lo + a, p.R);
    const double sg = (p.side == 0) ? sst.sig_p[slot] : sst.sig_w[slot];   // z~_j shares p~_j's scale
    coef[a] = coefs[a] * sg;
    vj[a] = (p.side == 0 && p.orth_z) ? p.Z + (size_t)(lo + a - 1) * p.zstride : p.ring + (size_t)slot * p.stride;
  }
  XT *out = p.ring + (size_t)ring_slot(newj, p.R) * p.stride;
  XT *fout = p.vfull ? p.vfull + (size_t)(newj - 1) * p.stride : nullptr;
  XT *zout = (p.side == 0) ? p.Z + (size_t)(k - 1) * p.zstride : nullptr;
  double acc[ND + 1];
#pragma unroll
  for (int a = 0; a <= ND; ++a) acc[a] = 0.0;
  // one contiguous chunk of ceil(len / grid) elements per CTA: every CTA gets
  // the same work (a grid-stride loop leaves CTAs idle when len < grid * block)
  const int64_t chunk = (p.len + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = min(p.len, i0 + chunk);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double v = (double)p.raw[i] * rs;
    double old[ND > 0 ? ND : 1];
#pragma unroll
    for (int a = 0; a < ND; ++a) { old[a] = (double)vj[a][i]; v -= coef[a] * old[a]; }
    const XT vx = (XT)v;
    out[i] = vx;
    if (fout) fout[i] = vx;
    const double vd = (double)vx;
    acc[0] += vd * vd;
    if (!(p.side == 0 && p.orth_z)) {
#pragma unroll
      for (int a = 0; a < ND; ++a) acc[1 + a] += vd * old[a];
    }
    if (p.side == 0) {
      double zt = vd;
      if (p.precond == SFL_PRECOND_DIAG) {
        zt = p.diag_w[i] * vd;
      } else if (reweight) {
        // x_{k-1}[i] = sum_j z~_j[i] c_j, four independent partial sums
        const XT *zi = p.Z + i;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int j = 0;
        for (; j + 3 < k - 1; j += 4) {
          a0 += (double)zi[(size_t)j * p.zstride] * s_c[j];
          a1 += (double)zi[(size_t)(j + 1) * p.zstride] * s_c[j + 1];
          a2 += (double)zi[(size_t)(j + 2) * p.zstride] * s_c[j + 2];
          a3 += (double)zi[(size_t)(j + 3) * p.zstride] * s_c[j + 3];
        }
        for (; j < k - 1; ++j) a0 += (double)zi[(size_t)j * p.zstride] * s_c[j];
        const double xv = (a0 + a1) + (a2 + a3);
        zt = sqrt(sqrt(xv * xv + sst.irw_eps)) * vd;
      }
      const XT zx = (XT)zt;
      zout[i] = zx;
      if (p.orth_z) {
        const double zd = (double)zx;
#pragma unroll
        for (int a = 0; a < ND; ++a) acc[1 + a] += zd * old[a];
      }
    }
  }
  __syncthreads();
  store_partials<ND + 1>(acc, wsum, p.side == 0 ? p.part.p : p.part.wn);
}

template <typename XT>
__global__ void __launch_bounds__(kThreads) orth_update_kernel(OrthParams<XT> p) {
  extern __shared__ __align__(16) double s_c[];     // [maxit] reweighting coefficients
  __shared__ SolveState sst;
  __shared__ double wsum[(kMaxWindow + 2) * kThreads];   // reduction scratch
  __shared__ double tot[kPartStride];
  __shared__ double coefs[kMaxWindow + 2];
  griddep_wait();
  griddep_launch_dependents();
  stage_state(p.st, &sst);
  if (sst.stop) return;
  const int k = sst.k + 1;
  if (dynamic_smem_bytes() < sizeof(double) * (size_t)k) return;
  const bool cta0 = blockIdx.x == 0 && threadIdx.x == 0;
  // the product stored its output unscaled: raw * rs is the true vector
  const double rs = p.side == 0 ? sst.sig_w[ring_slot(k, p.scale_ring)] : sst.sig_p[ring_slot(k, p.scale_ring)];
  auto scale_dots = [&](int nq) {   // thread 0: products' records are of the unscaled output
    tot[0] *= rs * rs;
    for (int a = 1; a < nq; ++a) tot[a] *= rs;
  };
  int lo, nd, newj;
  if (p.side == 0) {
    // coefficients of z against p_lo..p_{k-1} from the A^T w product's dots
    lo = max(1, k - p.ell); nd = p.full ? 0 : k - lo; newj = k;
    reduce_partials(p.part.z, p.G_prev, 1 + nd, wsum, tot);
    if (threadIdx.x == 0) {
      scale_dots(1 + nd);
      mgs_coefficients(tot + 1, nd, lo, p.R, sst.sig_p, sst.gram_p, coefs);
    }
    if (cta0) p.st->znorm_raw2 = tot[0];
  } else {
    // coefficients of w against w_lo..w_k (column k of H) from the A z_k product's dots
    lo = max(1, k - p.ell); nd = p.full ? 0 : k - lo + 1; newj = k + 1;
    if (p.sk_rec) {
      // the fused sketch of A z_k -> column k of S A Z, by the warps the
      // reduction below leaves idle (all warps when none is): a warp per pair
      // of sketch rows over the grid
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      const int w0 = 1 + nd < kWarps ? 1 + nd : 0, nsk = kWarps - w0;
      if (warp >= w0) {
        const int gw = blockIdx.x * nsk + (warp - w0), nw = gridDim.x * nsk;
        double *col = p.sk_col_base + (size_t)(k - 1) * p.sk_s;
        const double sc = p.sk_isz * rs;
        for (int r = gw; r < p.sk_s; r += 2 * nw) {
          const int r2 = r + nw;
          double a, b;
          sum_records2(p.sk_rec + (size_t)r * p.sk_cap, r2 < p.sk_s ? p.sk_rec + (size_t)r2 * p.sk_cap : nullptr,
                       p.sk_cap, lane, a, b);
          a = warp_sum(a);
          b = warp_sum(b);
          if (lane == 0) {
            col[r] = a * sc;
            if (r2 < p.sk_s) col[r2] = b * sc;
          }
        }
      }
    }
    reduce_partials(p.part.w, p.G_prev, 1 + nd, wsum, tot);
    if (threadIdx.x == 0) {
      scale_dots(1 + nd);
      mgs_coefficients(tot + 1, nd, lo, p.R, sst.sig_w, sst.gram_w, coefs);
    }
    if (cta0) {
      p.st->wnorm_raw2 = tot[0];
      for (int a = 0; a < nd; ++a) p.st->hw[a] = coefs[a];
      if (p.want_h && !p.full) {   // full: the block CGS2 kernels wrote the column
        double *hb = p.Hband + (size_t)(k - 1) * (p.ell + 2);
        for (int q = 0; q < p.ell + 2; ++q) hb[q] = 0.0;
        for (int a = 0; a < nd; ++a) hb[(lo + a) - k + p.ell] = coefs[a];
      }
    }
  }
  // reweighting: coefficients c_j = sig_j y_j of x_{k-1} = sum_j z~_j c_j
  const bool reweight = p.side == 0 && p.precond == SFL_PRECOND_REWEIGHT;
  if (reweight)
    for (int j = threadIdx.x; j < k - 1; j += blockDim.x) s_c[j] = p.sigZ[j] * p.y[j];
  __syncthreads();
  switch (nd) {
    case 0: orth_run<XT, 0>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 1: orth_run<XT, 1>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 2: orth_run<XT, 2>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 3: orth_run<XT, 3>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 4: orth_run<XT, 4>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 5: orth_run<XT, 5>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 6: orth_run<XT, 6>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 7: orth_run<XT, 7>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    case 8: orth_run<XT, 8>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
    default: orth_run<XT, 9>(p, sst, k, lo, newj, coefs, s_c, reweight, wsum, rs); break;
  }
}

__host__ __device__ inline size_t orth_smem_bytes(int maxit) { return sizeof(double) * (size_t)(maxit + 1); }

// ---------------------------------------------------------------- small FP64 least squares

struct LsParams {
  SolveState *st;
  int method, s, maxit, ell, stop_rule;
  int stage_q;        // 1: each CTA copies its block of Q rows into shared memory first
  int stage_saz;      // 1: each CTA copies its block of SAZ rows into shared memory (residual rule)
  double *Q;          // s x maxit, row-major: orthonormal basis of the sketched columns
  double *Rinv;       // maxit x maxit, row-major: inverse of the triangular factor
  double *y;          // maxit
  double *e;          // s: residual of the small problem
  double *SAZ;        // sFLSQR: LS columns; sFLSMR: m-side columns for the residual rule
  double *SAtW;       // sFLSMR
  const double *Hband;
  const double *sbm;  // sFLSMR residual rule: S_m b
  const double *rhs;  // right-hand side of the small problem
  double *relres_hist;
  cudaGraphConditionalHandle cond;
  int use_cond;
  // fused sketch (single sFLSMR solves): the A^T w_{k+1} / B w_{k+1} product
  // left per-CTA records of its unscaled sketch; this step adds them (fixed
  // order) into column k+1 of S A^T W, scaled by 1/sqrt(zeta) and the
  // output's scale (the w update does the same for the A z_k product's)
  const double *skz_rec;
  int skz_cap;
  double sk_isz;
  int RW;
  // several independent problems (one cluster each, problem = cluster index):
  // st is an array of states and every buffer above advances by its stride
  int64_t bQ, bRinv, by, be, bSAZ, bSAtW, bHband, bvec, bhist;   // per-problem strides (0: one problem)
};

constexpr int kMaxCluster = 16;

// Shared-memory plan of the least-squares step (in doubles), identical on the
// host (launch size) and the device (guard): six vectors of maxit+2, three
// row blocks, slice partials, and optionally the staged Q and SAZ blocks with
// an odd row stride (no bank conflicts between rows).
__host__ __device__ inline int ls_rows_per_cta(int s, int cl) { return (s + cl - 1) / cl; }
__host__ __device__ inline int ls_qld(int maxit) { return maxit | 1; }
__host__ __device__ inline size_t ls_smem_doubles(int s, int maxit, int cl, int stage_q, int stage_saz) {
  const int RB = ls_rows_per_cta(s, cl);
  size_t n = 6 * (size_t)(maxit + 2) + 3 * (size_t)RB + (size_t)(RB > kThreads ? RB : kThreads);
  if (stage_q) n += (size_t)RB * ls_qld(maxit);
  if (stage_saz) n += (size_t)RB * ls_qld(maxit);
  return n;
}

// One thread-block cluster appends column k of the sketched matrix to an
// explicit-Q QR by classical Gram-Schmidt applied twice (CGS2), updates the
// residual e, the inverse triangular factor and y_k = y_{k-1} + gamma_k
// Rinv[:,k], and evaluates the stop test.  Rows of Q are split in blocks over
// the CTAs of the cluster.  Q^T c runs one thread per column (no per-column
// reductions); partial vectors are exchanged through distributed shared
// memory and every CTA adds the ranks' values as the same fixed tree, so all
// CTAs hold bitwise identical totals and take the same branches.
// Rows r0 .. r0 + nr - 1 of a sketched column from per-CTA records
// (cap per row), times sc.  Warp w takes rows w, w + kWarps, ...; lanes go
// over the records.  The loads of up to four rows (10 records per lane and
// row per pass) are all issued before any is added, so a warp's rows cost
// one L2 round trip for cap <= 320.  Each row adds its records in a fixed
// order.  Not inlined, so its loads in flight do not weigh on the small
// least-squares step's registers.
static __device__ __noinline__ void ls_sketch_rows(const double *rec, int cap, int r0, int nr, double sc,
                                                   double *col) {
  constexpr int kRows = 4, kPer = 10;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = warp; i0 < nr; i0 += kRows * kWarps) {
    double a[kRows];
#pragma unroll
    for (int j = 0; j < kRows; ++j) a[j] = 0.0;
    for (int b0 = lane; b0 < cap; b0 += kPer * 32) {
      double v[kRows][kPer];
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        const int i = i0 + j * kWarps;
        const double *rc = rec + (size_t)(r0 + (i < nr ? i : 0)) * cap;
#pragma unroll
        for (int t = 0; t < kPer; ++t) v[j][t] = (i < nr && b0 + 32 * t < cap) ? __ldcg(rc + b0 + 32 * t) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < kRows; ++j)
#pragma unroll
        for (int t = 0; t < kPer; ++t) a[j] += v[j][t];
    }
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const int i = i0 + j * kWarps;
      const double t = warp_sum(a[j]);
      if (lane == 0 && i < nr) col[r0 + i] = t * sc;
    }
  }
}

static __global__ void __launch_bounds__(kThreads) ls_step_kernel(LsParams pin) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this cluster's problem
  const int64_t prob = blockIdx.x / CL;
  LsParams p = pin;
  p.st += prob;
  p.Q += prob * p.bQ;
  p.Rinv += prob * p.bRinv;
  p.y += prob * p.by;
  p.e += prob * p.be;
  p.SAZ += prob * p.bSAZ;
  if (p.SAtW) p.SAtW += prob * p.bSAtW;
  if (p.Hband) p.Hband += prob * p.bHband;
  if (p.sbm) p.sbm += prob * p.bvec;
  p.rhs += prob * p.bvec;
  if (p.relres_hist) p.relres_hist += prob * p.bhist;
  SolveState *st = p.st;
  griddep_wait();
  griddep_launch_dependents();
  // Every CTA reads the flags before the first cluster barrier; rank 0 writes
  // them only after the last one, so all CTAs take the same branches.
  const int stop0 = st->stop, lucky = st->lucky;
  if (stop0 || CL > kMaxCluster) {
    if (rank == 0 && tid == 0 && p.use_cond) cudaGraphSetConditional(p.cond, 0u);
    return;
  }
  const int k = st->k + 1, kk = k - 1;
  // state that only this kernel's final block writes, read here so that no
  // later phase waits on a global load: the first diagonal of R (k > 1), the
  // stop-ratio denominator (k > 1) and the stop tolerance
  const double R11_prev = st->R11, den_prev = st->stop_den, tol = st->tol, cmax_prev = st->rinv_cmax;
  const double inv_den_prev = 1.0 / den_prev;   // used at the stop test (k > 1)
  const int s = p.s;
  const int RB = ls_rows_per_cta(s, CL);
  const int r0 = min(s, rank * RB), r1 = min(s, r0 + RB), nr = r1 - r0;
  const int KP = p.maxit + 2;
  const bool resid_rule = p.method == kSFLSMR && p.stop_rule == SFL_STOP_RULE_RESIDUAL;
  // every CTA of the cluster got the same shared memory: all leave together
  if (dynamic_smem_bytes() < sizeof(double) * ls_smem_doubles(s, p.maxit, CL, p.stage_q, p.stage_saz)) {
    if (rank == 0 && tid == 0 && p.use_cond) cudaGraphSetConditional(p.cond, 0u);
    return;
  }

  // ---- prefetch, consumed in step 7: this warp's rows of R^{-1} (columns < kk) and of y
  constexpr int kPR = 2, kPC = 8;   // rows per warp, values per lane per row held in registers
  double rin[kPR][kPC], yold[kPR];
#pragma unroll
  for (int t = 0; t < kPR; ++t) {
    const int i = rank * kWarps + warp + t * CL * kWarps;
    yold[t] = (i < kk) ? p.y[i] : 0.0;
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
      const int j = i + lane + 32 * c;
      rin[t][c] = (i < kk && j < kk) ? p.Rinv[(size_t)i * p.maxit + j] : 0.0;
    }
  }

  extern __shared__ __align__(16) double lsm[];
  double *part0 = lsm;              // [KP] partial vectors exchanged in the cluster (pass 1)
  double *part1 = part0 + KP;       // [KP] (pass 2 and its two scalars)
  double *red = part1 + KP;         // [KP] cluster-reduced vector
  double *rr = red + KP;            // [KP] R column above the diagonal
  double *ys = rr + KP;             // [KP] entries of y_k computed by this CTA (read by peers)
  double *yfull = ys + KP;          // [KP] y_k gathered from the cluster
  double *crow = yfull + KP;        // [RB] my rows of the working column
  double *ecur = crow + RB;         // [RB] my rows of e
  double *upd = ecur + RB;          // [RB] my rows of a matrix-vector product
  double *tmp = upd + RB;           // [max(kThreads, RB)] slice partials
  double *Qs = tmp + max(kThreads, RB);                        // [RB x ldq] staged Q block
  double *Ss = Qs + (p.stage_q ? (size_t)RB * ls_qld(p.maxit) : 0);   // [RB x ldq] staged SAZ block
  const int H = max(1, kThreads / max(RB, 1));   // column slices per row
  __shared__ double s_sc[2][4];     // scalar partials exchanged in the cluster
  __shared__ double s_res[2][4];
  __shared__ double s_r2n;
  __shared__ double s_u2[kWarps];   // per-warp sums of the new R^{-1} column's squares

  // my block of Q rows: staged copy or the global rows
  const double *Qb = p.stage_q ? Qs : p.Q + (size_t)r0 * p.maxit;
  const int64_t qld = p.stage_q ? ls_qld(p.maxit) : p.maxit;

  // Totals over the cluster of per-CTA vectors buf[0..cnt): every CTA sums
  // the ranks' entries as one fixed tree (ranks past CL add zero).
  auto cluster_allreduce_vec = [&](double *buf, int cnt, double *dst) {
    cl.sync();
    for (int j = tid; j < cnt; j += kThreads) {
      double v[kMaxCluster];
#pragma unroll
      for (int b = 0; b < kMaxCluster; ++b) v[b] = (b < CL) ? cl.map_shared_rank(buf, b)[j] : 0.0;
#pragma unroll
      for (int w = kMaxCluster / 2; w >= 1; w >>= 1)
#pragma unroll
        for (int b = 0; b < w; ++b) v[b] += v[b + w];
      dst[j] = v[0];
    }
    __syncthreads();
  };
  // Totals over the cluster of up to three scalars whose per-lane partials
  // are held by warp 0 (lane sums, then rank sums, both butterflies).
  auto cluster_allreduce_sc = [&](double a0, double a1, double a2, int nq, int slot) {
    if (warp == 0) {
      a0 = warp_sum(a0);
      a1 = nq > 1 ? warp_sum(a1) : 0.0;
      a2 = nq > 2 ? warp_sum(a2) : 0.0;
      if (lane == 0) { s_sc[slot][0] = a0; s_sc[slot][1] = a1; s_sc[slot][2] = a2; }
    }
    cl.sync();
    if (warp == 0) {
      double b0 = 0.0, b1 = 0.0, b2 = 0.0;
      if (lane < CL) {
        const double *r = cl.map_shared_rank(&s_sc[slot][0], lane);
        b0 = r[0]; b1 = r[1]; b2 = r[2];
      }
      b0 = warp_sum(b0);
      b1 = nq > 1 ? warp_sum(b1) : 0.0;
      b2 = nq > 2 ? warp_sum(b2) : 0.0;
      if (lane == 0) { s_res[slot][0] = b0; s_res[slot][1] = b1; s_res[slot][2] = b2; }
    }
    __syncthreads();
  };
  // buf[j] = sum_i Q[r0+i][j] crow[i] over my rows, one thread per column
  auto qt_partial = [&](double *buf) {
    for (int j = tid; j < kk; j += kThreads) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int i = 0;
      for (; i + 3 < nr; i += 4) {
        a0 += Qb[(size_t)i * qld + j] * crow[i];
        a1 += Qb[(size_t)(i + 1) * qld + j] * crow[i + 1];
        a2 += Qb[(size_t)(i + 2) * qld + j] * crow[i + 2];
        a3 += Qb[(size_t)(i + 3) * qld + j] * crow[i + 3];
      }
      for (; i < nr; ++i) a0 += Qb[(size_t)i * qld + j] * crow[i];
      buf[j] = (a0 + a1) + (a2 + a3);
    }
  };
  // out[i] = sum_{j < ncol} M(i, j) coef[j] for my rows, M(i, j) = M[i*rs + j*cs];
  // thread (row i, slice h) sums the columns j = h (mod H), slices added in order.
  auto rows_times_vec = [&](const double *M, int64_t rs, int64_t cs, const double *coef, int ncol, double *out) {
    for (int t = tid; t < H * RB; t += kThreads) {
      const int i = t % RB, h = t / RB;
      double a0 = 0.0, a1 = 0.0;
      if (i < nr) {
        const double *mi = M + (size_t)i * rs;
        int j = h;
        for (; j + H < ncol; j += 2 * H) {
          a0 += mi[(size_t)j * cs] * coef[j];
          a1 += mi[(size_t)(j + H) * cs] * coef[j + H];
        }
        if (j < ncol) a0 += mi[(size_t)j * cs] * coef[j];
      }
      tmp[t] = a0 + a1;
    }
    __syncthreads();
    for (int i = tid; i < nr; i += kThreads) {
      double a0 = 0.0, a1 = 0.0;
      int h = 0;
      for (; h + 1 < H; h += 2) { a0 += tmp[h * RB + i]; a1 += tmp[(h + 1) * RB + i]; }
      if (h < H) a0 += tmp[h * RB + i];
      out[i] = a0 + a1;
    }
    __syncthreads();
  };

  // ---- 0. the new column and e, my rows; the staged blocks
  if (p.skz_rec && !lucky) {   // the fused sketch of this step's A^T w_{k+1} / B w_{k+1} product, my rows
    ls_sketch_rows(p.skz_rec, p.skz_cap, r0, nr, p.sk_isz * __ldcg(&st->sig_w[ring_slot(k + 1, p.RW)]),
                   p.SAtW + (size_t)k * s);
    __syncthreads();
  }
  for (int i = tid; i < nr; i += kThreads) {
    const int row = r0 + i;
    double c;
    if (p.method == kSFLSQR) {
      c = p.SAZ[(size_t)kk * s + row];
    } else {
      // column k of [S A^T W, S z] H_{k+1,k}: a sum over the band of H
      const double *hb = p.Hband + (size_t)kk * (p.ell + 2);
      c = 0.0;
      const int lo = max(1, k - p.ell);
      for (int j = lo; j <= k + 1; ++j) {
        if (j == k + 1 && lucky) continue;
        c += p.SAtW[(size_t)(j - 1) * s + row] * hb[j - k + p.ell];
      }
    }
    crow[i] = c;
    ecur[i] = p.e[row];
  }
  const int ldq = ls_qld(p.maxit);
  if (p.stage_q && kk > 0)
    for (int t = tid; t < nr * kk; t += kThreads) {
      const int i = t / kk, j = t - i * kk;
      Qs[(size_t)i * ldq + j] = p.Q[(size_t)(r0 + i) * p.maxit + j];
    }
  if (p.stage_saz && resid_rule)
    for (int t = tid; t < nr * k; t += kThreads) {
      const int j = t / nr, i = t - j * nr;
      Ss[(size_t)i * ldq + j] = p.SAZ[(size_t)j * s + r0 + i];
    }
  __syncthreads();

  // ---- 1-5. classical Gram-Schmidt twice against the first kk columns; the
  // second pass also totals ||c'||^2 and <c', e>, so that
  // rho^2 = ||c'||^2 - ||Q^T c'||^2 and <c'', e> = <c', e> - (Q^T c').(Q^T e),
  // whose last term is a product of two rounding-level vectors and is dropped.
  double rho2, ce, den, inv_den;
  if (kk > 0) {
    qt_partial(part0);
    cluster_allreduce_vec(part0, kk, red);
    for (int j = tid; j < kk; j += kThreads) rr[j] = red[j];
    rows_times_vec(Qb, qld, 1, red, kk, upd);
    for (int i = tid; i < nr; i += kThreads) crow[i] -= upd[i];
    __syncthreads();
    qt_partial(part1);
    if (warp == kWarps - 1) {
      double a0 = 0.0, a1 = 0.0;
      for (int i = lane; i < nr; i += 32) {
        a0 += crow[i] * crow[i];
        a1 += crow[i] * ecur[i];
      }
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      if (lane == 0) { part1[kk] = a0; part1[kk + 1] = a1; }
    }
    cluster_allreduce_vec(part1, kk + 2, red);
    for (int j = tid; j < kk; j += kThreads) rr[j] += red[j];
    if (warp == 0) {
      double a = 0.0;
      for (int j = lane; j < kk; j += 32) a += red[j] * red[j];
      a = warp_sum(a);
      if (lane == 0) s_r2n = a;
    }
    rows_times_vec(Qb, qld, 1, red, kk, upd);   // synchronises: s_r2n is visible after it
    for (int i = tid; i < nr; i += kThreads) crow[i] -= upd[i];
    rho2 = red[kk] - s_r2n;
    ce = red[kk + 1];
    den = den_prev;
    inv_den = inv_den_prev;
  } else {
    // first step: ||c||^2, <c, e> and the stop-ratio denominator ||s_b||
    // (sFLSQR), ||S_m b|| (sFLSMR, residual rule) or ||s_{A^T b}|| (sFLSMR,
    // normal-equation rule)
    const double *dv = resid_rule ? p.sbm : p.rhs;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (warp == 0)
      for (int i = lane; i < nr; i += 32) {
        a0 += crow[i] * crow[i];
        a1 += crow[i] * ecur[i];
        a2 += dv[r0 + i] * dv[r0 + i];
      }
    cluster_allreduce_sc(a0, a1, a2, 3, 0);
    rho2 = s_res[0][0];
    ce = s_res[0][1];
    den = sqrt(s_res[0][2]);
    inv_den = 1.0 / den;
  }
  // rho^2 may round below zero for a dependent column (a breakdown); NaN stays
  // NaN (and +inf becomes NaN: 0 * inf).  1/rho is one reciprocal square root
  // and rho = rho^2 / rho, instead of a square root followed by a division.
  double rho, irho = 0.0;
  if (rho2 > 0.0) {
    irho = rsqrt(rho2);
    rho = rho2 * irho;
  } else {
    rho = rho2 < 0.0 ? 0.0 : rho2;
  }
  const double R11 = (k == 1) ? rho : R11_prev;
  if (!(rho > 1e-300) || !(rho > 1e-14 * R11) || !isfinite(rho)) {
    cl.sync();   // no CTA leaves while a peer may still read its shared memory
    if (rank == 0 && tid == 0) {
      st->stop = isfinite(rho) ? SFL_STOP_BREAKDOWN : kStopNonfinite;
      if (p.use_cond) cudaGraphSetConditional(p.cond, 0u);
    }
    return;
  }
  // ---- 6. q_k = c / rho, gamma_k = <q_k, e>, e -= gamma_k q_k
  const double gamma = ce * irho;
  __syncthreads();   // crow is final
  for (int i = tid; i < nr; i += kThreads) {
    const double q = crow[i] * irho;
    p.Q[(size_t)(r0 + i) * p.maxit + kk] = q;
    const double ei = ecur[i] - gamma * q;
    p.e[r0 + i] = ei;
    ecur[i] = ei;
  }
  // ---- 7. column kk of R^{-1} and y_k = [y_{k-1}; 0] + gamma_k R^{-1}[:, kk]
  double u2 = 0.0;   // lane 0: squares of this warp's entries of the new column
  auto rinv_row = [&](int i, double a, double y_prev) {
    a = warp_sum(a);
    if (lane == 0) {
      const double u = -a * irho;
      u2 += u * u;
      const double yn = y_prev + gamma * u;
      p.Rinv[(size_t)i * p.maxit + kk] = u;
      p.y[i] = yn;
      ys[i] = yn;
    }
  };
#pragma unroll
  for (int t = 0; t < kPR; ++t) {
    const int i = rank * kWarps + warp + t * CL * kWarps;
    if (i < kk) {
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int c = 0; c < kPC; ++c) {
        const int j = i + lane + 32 * c;
        if (j < kk) {
          if (c & 1) a1 += rin[t][c] * rr[j];
          else a0 += rin[t][c] * rr[j];
        }
      }
      for (int j = i + lane + 32 * kPC; j < kk; j += 32) a0 += p.Rinv[(size_t)i * p.maxit + j] * rr[j];
      rinv_row(i, a0 + a1, yold[t]);
    }
  }
  for (int t = kPR;; ++t) {   // rows past the prefetched ones (kk > kPR * CL * kWarps)
    const int i = rank * kWarps + warp + t * CL * kWarps;
    if (i >= kk) break;
    double a = 0.0;
    for (int j = i + lane; j < kk; j += 32) a += p.Rinv[(size_t)i * p.maxit + j] * rr[j];
    rinv_row(i, a, p.y[i]);
  }
  if (rank == 0 && tid == 0) {
    p.Rinv[(size_t)kk * p.maxit + kk] = irho;
    p.y[kk] = gamma * irho;
  }
  if (lane == 0) s_u2[warp] = u2;   // read after the barriers of step 8
  // ---- 8. residual of the stop test (and the norm of the new R^{-1} column)
  if (resid_rule) {
    // || S_m b - S_m A Z_k y_k ||, my rows; y_k is gathered from its owners'
    // shared memory after a cluster barrier
    cl.sync();
    for (int j = tid; j < kk; j += kThreads) {
      const int owner = (j % (CL * kWarps)) / kWarps;
      yfull[j] = cl.map_shared_rank(ys, owner)[j];
    }
    if (tid == 0) yfull[kk] = gamma * irho;
    __syncthreads();
    if (p.stage_saz) rows_times_vec(Ss, ldq, 1, yfull, k, upd);
    else rows_times_vec(p.SAZ + r0, 1, s, yfull, k, upd);
    double a0 = 0.0;
    if (warp == 0)
      for (int i = lane; i < nr; i += 32) {
        const double d = p.sbm[r0 + i] - upd[i];
        a0 += d * d;
      }
    cluster_allreduce_sc(a0, (warp == 0 && lane < kWarps) ? s_u2[lane] : 0.0, 0.0, 2, 1);
  } else {
    __syncthreads();   // ecur is final
    double a0 = 0.0;
    if (warp == 0)
      for (int i = lane; i < nr; i += 32) a0 += ecur[i] * ecur[i];
    cluster_allreduce_sc(a0, (warp == 0 && lane < kWarps) ? s_u2[lane] : 0.0, 0.0, 2, 1);
  }
  const double res2 = s_res[1][0];
  // condition estimate of the small triangular factor: R11 * (largest column
  // norm of R^{-1}), a lower bound on kappa(R).  Past 1e12 the problem is
  // numerically rank deficient and the explicit-inverse recurrence for y
  // loses accuracy: the step's iterate is returned and the solve stops
  // (breakdown).
  const double cmax = fmax(cmax_prev, sqrt(s_res[1][1] + irho * irho));
  cl.sync();   // no CTA leaves while a peer may still read its shared memory
  if (rank == 0 && tid == 0) {
    if (k == 1) st->stop_den = den;
    const double rel = sqrt(res2) * inv_den;
    st->relres = rel;
    if (p.relres_hist) p.relres_hist[kk] = rel;
    if (k == 1) st->R11 = rho;
    st->rinv_cmax = cmax;
    st->k = k;
    st->hist_pending = 1;
    int stop = 0;
    if (rel < tol) stop = SFL_STOP_DISCREPANCY;
    else if (lucky || R11 * cmax > 1e12) stop = SFL_STOP_BREAKDOWN;
    else if (k >= p.maxit) stop = SFL_STOP_MAXIT;
    if (!isfinite(rel)) stop = kStopNonfinite;
    st->stop = stop;
    if (p.use_cond) cudaGraphSetConditional(p.cond, stop ? 0u : 1u);
  }
}

// ---------------------------------------------------------------- full orthogonalization (window < 0)

// With window ell < 0 (full orthogonalization, eq. (FGK) with the band filled:
// FLSQR / FLSMR and their sketched forms) the product output is orthogonalized
// against every earlier basis vector by block classical Gram-Schmidt applied
// twice (CGS2) before the ordinary update kernel normalises it:
//   pass 1: c1 = V^T x;  x <- x - V c1;   pass 2: c2 = V^T x;  x <- x - V c2,
// with V the unit basis (p_1..p_{k-1} for z at step k, w_1..w_k for w), stored
// unnormalised with its scales.  Each pass is a tall-skinny product with the
// stored basis: one DFMA per basis entry, the basis streamed from HBM.  The
// coefficients are in the units of the raw (unscaled) product output; for the
// w side the column of H is rs (c1 + c2), rs the product's scale sig_p(k).
constexpr int kCgsChunk = 4096;   // most vector entries one CTA of the dot kernels holds in shared memory

template <typename XT>
struct CgsParams {
  SolveState *st;
  int side;                    // 0: z against p_1..p_{k-1}; 1: w against w_1..w_k
  int want_h;                  // w side: write column k of H
  int64_t len;
  const XT *x;                 // the raw product output (left as it is: the sketch still reads it)
  XT *xo;                      // the orthogonalized vector
  const XT *V; int64_t vstride;   // column j - 1: v~_j
  const double *sigV;          // 1/||v~_j|| at index j - 1
  const double *sigP;          // sig_p(k) at index k - 1 (the scale of the raw w)
  double *rec;                 // per-CTA dots, rec[(j - 1) * cap + cta]
  int cap;                     // record stride (>= the dot kernels' grid)
  double *coef;                // [2][kMaxIt + 2]: unit-basis coefficients of passes 1 and 2
  double *Hband; int hb_ell;   // H columns, hb_ell + 2 entries each
};

template <typename XT>
__device__ __forceinline__ int cgs_nbasis(const CgsParams<XT> &p, int &k) {
  if (__ldcg(&p.st->stop)) return 0;
  k = __ldcg(&p.st->k) + 1;
  return p.side == 0 ? k - 1 : k;
}

// Per-CTA dots <v~_j, x> over one contiguous chunk of the entries.  pass 2
// first applies pass 1's update to the chunk (xo = x - V c1) and takes the
// dots of the updated entries.  The chunk sits in shared memory;
// warp w sums the columns j = w, w + 8, ... with coalesced loads.
template <typename XT>
__global__ void __launch_bounds__(kThreads) cgs_dots_kernel(CgsParams<XT> p, int pass) {
  __shared__ double xs[kCgsChunk];
  __shared__ double cs[kMaxIt + 2];
  int k = 0;
  const int kv = cgs_nbasis(p, k);
  if (kv <= 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t chunk = (p.len + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int nloc = (int)max((int64_t)0, min(p.len, i0 + chunk) - i0);
  if (chunk > kCgsChunk) return;   // the host sizes the grid so this never happens
  if (pass == 2)
    for (int j = tid; j < kv; j += kThreads) cs[j] = __ldcg(p.coef + j) * p.sigV[j];
  __syncthreads();
  for (int i = tid; i < nloc; i += kThreads) {
    double v = (double)p.x[i0 + i];
    if (pass == 2) {
      const XT *vi = p.V + i0 + i;
      double a0 = 0.0, a1 = 0.0;
      int j = 0;
      for (; j + 1 < kv; j += 2) {
        a0 += (double)vi[(size_t)j * p.vstride] * cs[j];
        a1 += (double)vi[(size_t)(j + 1) * p.vstride] * cs[j + 1];
      }
      if (j < kv) a0 += (double)vi[(size_t)j * p.vstride] * cs[j];
      const XT nx = (XT)(v - (a0 + a1));
      p.xo[i0 + i] = nx;
      v = (double)nx;
    }
    xs[i] = v;
  }
  __syncthreads();
  for (int j = warp; j < kv; j += kWarps) {
    const XT *vj = p.V + (size_t)j * p.vstride + i0;
    double a0 = 0.0, a1 = 0.0;
    int i = lane;
    for (; i + 32 < nloc; i += 64) {
      a0 += (double)vj[i] * xs[i];
      a1 += (double)vj[i + 32] * xs[i + 32];
    }
    if (i < nloc) a0 += (double)vj[i] * xs[i];
    const double t = warp_sum(a0 + a1);
    if (lane == 0) p.rec[(size_t)j * p.cap + blockIdx.x] = t;
  }
}

// Coefficients of one pass: warp per basis vector, the G per-CTA records
// summed in a fixed order, times the vector's scale.  After pass 2 of the w
// side, column k of H (rows 1..k) when it is recorded.
template <typename XT>
__global__ void __launch_bounds__(kThreads) cgs_reduce_kernel(CgsParams<XT> p, int pass, int G) {
  int k = 0;
  const int kv = cgs_nbasis(p, k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * kWarps + warp;
  if (j >= kv) return;
  const double *r = p.rec + (size_t)j * p.cap;
  double a0 = 0.0, a1 = 0.0;
  int b = lane;
  for (; b + 32 < G; b += 64) { a0 += __ldcg(r + b); a1 += __ldcg(r + b + 32); }
  if (b < G) a0 += __ldcg(r + b);
  const double t = warp_sum(a0 + a1);
  if (lane != 0) return;
  const double c = t * p.sigV[j];
  p.coef[(pass - 1) * (kMaxIt + 2) + j] = c;
  if (pass == 2 && p.side == 1 && p.want_h) {
    const double rs = p.sigP[k - 1];
    // row j + 1 of column k: index (j + 1) - k + hb_ell in the band
    p.Hband[(size_t)(k - 1) * (p.hb_ell + 2) + (j + 1) - k + p.hb_ell] = rs * (__ldcg(p.coef + j) + c);
  }
}

// Pass 2's update: xo <- xo - V c2 (entries strided over the grid).
template <typename XT>
__global__ void __launch_bounds__(kThreads) cgs_update_kernel(CgsParams<XT> p) {
  __shared__ double cs[kMaxIt + 2];
  int k = 0;
  const int kv = cgs_nbasis(p, k);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (kv <= 0) {   // no basis yet (z at step 1): the vector passes through
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.len; i += stride) p.xo[i] = p.x[i];
    return;
  }
  for (int j = threadIdx.x; j < kv; j += kThreads) cs[j] = __ldcg(p.coef + (kMaxIt + 2) + j) * p.sigV[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.len; i += stride) {
    const XT *vi = p.V + i;
    double a0 = 0.0, a1 = 0.0;
    int j = 0;
    for (; j + 1 < kv; j += 2) {
      a0 += (double)vi[(size_t)j * p.vstride] * cs[j];
      a1 += (double)vi[(size_t)(j + 1) * p.vstride] * cs[j + 1];
    }
    if (j < kv) a0 += (double)vi[(size_t)j * p.vstride] * cs[j];
    p.xo[i] = (XT)((double)p.xo[i] - (a0 + a1));
  }
}

// FLSQR's small problem is min || beta e_1 - H_{k+1,k} y ||: right-hand side
// and initial residual beta e_1 (beta = ||b|| from the initial pass).
static __global__ void flsqr_rhs_kernel(const SolveState *st, double *rhs, double *e, int s) {
  const double beta = __ldcg(&st->beta0);
  for (int r = threadIdx.x; r < s; r += blockDim.x) {
    const double v = r == 0 ? beta : 0.0;
    rhs[r] = v;
    e[r] = v;
  }
}

// Columns 0..ncol-1 of the s x ncol identity, column-major (FLSQR's stand-in
// for the sketched columns S A^T W, so that [I] H is H itself).
static __global__ void identity_cols_kernel(double *M, int s, int ncol) {
  const int64_t tot = (int64_t)s * ncol;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x)
    M[t] = (t / s == t % s) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------- x = Z y

// x[i] = sum_{j<k} z~_j[i] sig_j y_j (FP64 accumulation).  history: writes x_k
// at row k-1 of `hist` when a step finished since the last call.
template <typename XT>
__global__ void __launch_bounds__(kThreads) solution_kernel(SolveState *st, const XT *Z, int64_t zstride,
                                                            const double *sigZ, const double *y, int64_t n,
                                                            double *x, double *hist) {
  const int k = st->k;
  double *out = x;
  if (hist) {
    if (!st->hist_pending) return;
    out = hist + (size_t)(k - 1) * n;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += (double)Z[(size_t)j * zstride + i] * (sigZ[j] * y[j]);
    out[i] = v;
  }
}

static __global__ void clear_hist_flag_kernel(SolveState *st) { st->hist_pending = 0; }

// Start-of-solve state: everything zero except the solve parameters.
static __global__ void reset_state_kernel(SolveState *st, uint64_t seed, double eta, double noise_norm, double irw_eps) {
  *st = SolveState();
  st->seed = seed;
  st->eta = eta;
  st->noise_norm = noise_norm;
  st->irw_eps = irw_eps;
}

}  // namespace sfl
