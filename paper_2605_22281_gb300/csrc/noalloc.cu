// Allocation-free variant of the sparse-sign sketch apply (sk = S v).
//
// sfl_sketch_apply allocates a draw table and its reduction scratch with
// cudaMalloc on every call.  Some callers cannot do that: code that runs on a
// device-memory budget fixed up front (a framework's caching allocator owns
// the memory and a foreign cudaMalloc either fails or fragments its pool), and
// latency-critical loops where a cudaMalloc/cudaFree pair would synchronise
// the device.  This variant allocates nothing: the sketch draws are
// regenerated inside the kernel, and the deterministic two-level reduction
// uses a fixed scratch array that lives in the library image (file-scope
// __device__ memory, about 2.2 MB, held by every GPU that loads the library
// until the process exits).
#include <mutex>

#include "engine.h"

namespace sfl {

constexpr int kNoAllocMaxS = 1024;                         // largest sketch size accepted
constexpr int kNoAllocGrid = 256;                          // most CTAs a launch may use
constexpr int kNoAllocStride = kNoAllocMaxS + 16;          // doubles per CTA partial
constexpr int kNoAllocGroups = kNoAllocGrid / kGroup;      // first-level reduction groups
constexpr size_t kNoAllocDoubles = (size_t)(kNoAllocGrid + kNoAllocGroups) * kNoAllocStride;
constexpr uint16_t kNoAllocUnused = 0xFFFFu;                 // marks a draw slot that holds no row

// Shared by every call on a device; a call leaves its partial sums behind.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocDoubles];
static __device__ __align__(256) unsigned int g_noalloc_tickets[kMaxGroups + 1];

// Each lane draws the zeta distinct rows of its own column (same generator
// and rejection rule as sketch_table_kernel), stages them in shared memory,
// and the warp then adds the columns into its private s-vector in index order.
__global__ void __launch_bounds__(kThreads) sketch_apply_inline_kernel(uint64_t seed, int s, int zeta,
                                                                      const double *__restrict__ v, int64_t len,
                                                                      double *sk_out, RedScratch red) {
  extern __shared__ __align__(16) double nsm[];
  double *acc = nsm;                                   // [kWarps][s]
  double *vals = acc + (size_t)kWarps * s;             // [s]
  __shared__ uint16_t stage[kWarps][32][kMaxZeta];
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kWarps * s; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  double *myacc = acc + (size_t)warp * s;
  const int64_t nblk = (len + 31) / 32;
  for (int64_t rb = (int64_t)blockIdx.x * kWarps + warp; rb < nblk; rb += (int64_t)gridDim.x * kWarps) {
    const int64_t c = rb * 32 + lane;
    double vc = 0.0;
    if (c < len) {
      vc = v[c];
      int rows[kMaxZeta];
      int cnt = 0;
      for (uint32_t t = 0; cnt < zeta && t < 1000000u; ++t) {
        const uint64_t h = splitmix64_first(seed ^ (((uint64_t)c << 32) + t));
        const int r = (int)__umul64hi(h, (uint64_t)s);
        bool dup = false;
        for (int q = 0; q < cnt; ++q) dup |= (rows[q] == r);
        if (dup) continue;
        rows[cnt] = r;
        stage[warp][lane][cnt] = (uint16_t)(r | ((int)(h & 1ull) << 15));
        ++cnt;
      }
      // a column whose draws hit the cap holds fewer than zeta rows (never
      // expected): its missing entries are marked and skipped below
      for (int q = cnt; q < zeta; ++q) stage[warp][lane][q] = kNoAllocUnused;
    }
    __syncwarp();
    const int nrow = (len - rb * 32) < 32 ? (int)(len - rb * 32) : 32;
    for (int L = 0; L < nrow; ++L) {
      const double x = __shfl_sync(0xffffffffu, vc, L);
      if (lane < zeta) {
        const uint16_t ent = stage[warp][L][lane];
        if (ent != kNoAllocUnused) myacc[ent & 0x7FFF] += (ent & 0x8000) ? -x : x;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = tid; i < s; i += blockDim.x) {
    double a = 0.0;
    for (int w = 0; w < kWarps; ++w) a += acc[(size_t)w * s + i];
    vals[i] = a;
  }
  __syncthreads();
  if (grid_reduce(vals, s, red, vals, &s_flag)) {
    const double isz = 1.0 / sqrt((double)zeta);
    for (int i = tid; i < s; i += blockDim.x) sk_out[i] = vals[i] * isz;
  }
}

struct NoAllocDevice {
  bool ready = false;
  double *partials = nullptr;
  unsigned int *tickets = nullptr;
  int grid = 0;
};

static std::mutex g_noalloc_mutex;
static NoAllocDevice g_noalloc_dev[64];

// Once per device, with that device current: host-side addresses of the
// scratch arrays (their names are host stand-ins, not device addresses).
static int noalloc_setup(int dev, NoAllocDevice **out) {
  if (dev < 0 || dev >= 64) return SFL_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocDevice &d = g_noalloc_dev[dev];
  if (!d.ready) {
    void *p = nullptr, *q = nullptr;
    SFL_CU(cudaGetSymbolAddress(&p, g_noalloc_partials));
    SFL_CU(cudaGetSymbolAddress(&q, g_noalloc_tickets));
    int sms = 0;
    SFL_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SFL_CU(cudaFuncSetAttribute(sketch_apply_inline_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * ((size_t)kWarps * kNoAllocMaxS + kNoAllocMaxS))));
    d.partials = (double *)p;
    d.tickets = (unsigned int *)q;
    d.grid = sms < kNoAllocGrid ? sms : kNoAllocGrid;
    d.ready = true;
  }
  *out = &d;
  return SFL_OK;
}

}  // namespace sfl

using namespace sfl;

extern "C" int sfl_sketch_apply_noalloc(uint64_t seed, int32_t s, int32_t zeta, const double *v, int64_t len,
                                        double *sk, sfl_stream stream) {
  if (!v || !sk || len < 1 || zeta < 1 || zeta > kMaxZeta || s < zeta) return SFL_EINVAL;
  if (s > kNoAllocMaxS) return SFL_EINVAL;   // the fixed scratch holds partial sums of at most 1024 rows
  int dev = 0;
  SFL_CU(cudaGetDevice(&dev));
  NoAllocDevice *d = nullptr;
  int r = noalloc_setup(dev, &d);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  // the tickets must start at zero; a call that stopped early could have left them set
  SFL_CU(cudaMemsetAsync(d->tickets, 0, sizeof(unsigned int) * (kMaxGroups + 1), st));
  RedScratch red;
  red.part = d->partials;
  red.gpart = d->partials + (size_t)kNoAllocGrid * kNoAllocStride;
  red.cnt = d->tickets;
  red.stride = kNoAllocStride;
  const size_t smem = sizeof(double) * ((size_t)kWarps * s + s);
  sketch_apply_inline_kernel<<<d->grid, kThreads, smem, st>>>(seed, s, zeta, v, len, sk, red);
  SFL_CU(cudaGetLastError());
  return SFL_OK;
}
