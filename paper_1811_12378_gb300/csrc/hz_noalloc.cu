// hz_residual_noalloc: the float64 residual r = fscale*f - A u and its squared norm, for
// callers that must not allocate device memory.
//
// Why it exists: some callers cannot call cudaMalloc at all -- code running while a CUDA
// graph is being captured on their stream, allocators that hand out one fixed arena and
// forbid further device allocations, or embedding hosts that own the GPU memory budget.  The
// rest of this library keeps its reduction scratch in buffers that hz_problem_create
// allocates; this entry point keeps its scratch (per-block partial sums and the "last
// block" tickets of the reduction) in the file-scope array below instead, so it needs no
// hz_problem and allocates nothing.  It computes the same residual as the cycle start of
// hz_solve, with the same reduction tree, so its norm equals the one hz_solve reports.
//
// Limits and sharing:
//  * kMaxPartials = 65536 block partials: nvec * ceil(n / 1024) must not exceed it (e.g. a
//    256^3 grid with up to 4 fields); kMaxVec = 64 fields per call.  Larger calls are
//    rejected with HZ_ERR_INVALID.  The array (1 MiB + 256 bytes) stays resident on every
//    device that loads the library until the process exits.
//  * Every call on a device uses the same array, and the array keeps the last call's
//    contents (each call clears the tickets it needs before its kernel starts).  Calls whose
//    kernels overlap on the GPU -- issued on two streams, or from two host threads -- race
//    on the array and give wrong results: serialise them, e.g. issue them on one stream.
//    Separate processes each have their own copy.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current, and caches it.  Make that first call
//    before any stream capture begins.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "hz.h"
#include "hz_internal.h"

namespace {

constexpr int kThreads = 256;                   // same reduction tree as hz_solve's residual
constexpr int kPpt = 4;
constexpr int kChunk = kThreads * kPpt;
constexpr long long kMaxPartials = 65536;       // double2 block partials
constexpr int kMaxVec = 64;                     // fields per call (one ticket each)
constexpr int kMaxDevices = 64;

// The scratch: kMaxPartials partial sums followed by kMaxVec 32-bit tickets (tickets must be
// zero when a reduction starts; each call clears its own before launching).
static __device__ __align__(256) double2 g_noalloc_scratch[kMaxPartials + kMaxVec / 4];

std::mutex g_mu;
double2* g_dev_addr[kMaxDevices] = {};

__device__ __forceinline__ int depth1(int i, int n, int L) {
  int e = min(i, n - 1 - i);
  return max(0, L - e);
}

__device__ __forceinline__ double2 block_sum(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sh[lane] : make_double2(0.0, 0.0);
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
  }
  __syncthreads();
  return v;
}

// r = fs*f - A u (u may be null), norm2[r] = ||r||^2.  partial/tickets point into the
// static scratch.
__global__ void __launch_bounds__(kThreads)
k_residual_noalloc(int nx, int ny, int nz, int layer, double cs, double sig, double cmin2,
                   const double* __restrict__ c, const double2* __restrict__ f, double fs,
                   const double2* __restrict__ u, double2* __restrict__ rout, double* norm2,
                   double2* partial, unsigned* tickets) {
  __shared__ double2 sh[32];
  __shared__ bool is_last;
  const int r = blockIdx.y;
  const long long n = (long long)nx * ny * nz;
  const long long sxy = (long long)nx * ny;
  const long long base = (long long)blockIdx.x * kChunk + threadIdx.x;
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < kPpt; ++e) {
    const long long p = base + (long long)e * kThreads;
    if (p >= n) continue;
    const double2 fv = f[r * n + p];
    double2 v = make_double2(fs * fv.x, fs * fv.y);
    if (u) {
      const int k = int(p / sxy);
      const long long rem = p - (long long)k * sxy;
      const int j = int(rem / nx);
      const int i = int(rem - (long long)j * nx);
      const double2* ur = u + r * n;
      const double cp = c[p];
      const double mp = cmin2 / (cp * cp);
      double ap = 0.0;
      if (layer > 0) {
        const int d = max(depth1(i, nx, layer), max(depth1(j, ny, layer), depth1(k, nz, layer)));
        const double t = double(d) / double(layer);
        ap = (sig * (t * t)) * mp;
      }
      double2 nb = make_double2(0.0, 0.0);
      auto add = [&](long long q) {
        const double2 w = ur[q];
        nb.x += w.x;
        nb.y += w.y;
      };
      if (i > 0) add(p - 1);
      if (i < nx - 1) add(p + 1);
      if (j > 0) add(p - nx);
      if (j < ny - 1) add(p + nx);
      if (k > 0) add(p - sxy);
      if (k < nz - 1) add(p + sxy);
      const double2 xc = ur[p];
      const double tx = 6.0 * xc.x - nb.x, ty = 6.0 * xc.y - nb.y;
      const double dr = -(mp + 0.0), di = -(ap + 0.0);
      const double ax = cs * tx + dr * xc.x - di * xc.y;
      const double ay = cs * ty + dr * xc.y + di * xc.x;
      v = make_double2(v.x - ax, v.y - ay);
    }
    if (rout) rout[r * n + p] = v;
    s += v.x * v.x + v.y * v.y;
  }
  double2* part = partial + (long long)r * gridDim.x;
  const double2 t = block_sum(make_double2(s, 0.0), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(tickets + r, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double2 acc = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double2 v = __ldcg(part + b);
    acc.x += v.x;
    acc.y += v.y;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    norm2[r] = acc.x;
    tickets[r] = 0;
  }
}

hz_status fail(hz_status s, const std::string& m) {
  hz::set_last_error(m);
  return s;
}

}  // namespace

extern "C" hz_status hz_residual_noalloc(const hz_grid* grid, const double* c, double c_min,
                                         const void* f, double fscale, const void* u, void* r,
                                         double* norm2, int nvec, void* stream) {
  if (!grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0) ||
      !(grid->omega > 0) || grid->layer_cells < 0 || !(grid->sigma_max >= 0) || !(c_min > 0) ||
      grid->discretization != HZ_DISC_FD7)
    return fail(HZ_ERR_INVALID, "hz_residual_noalloc: invalid grid or c_min (7-point grids only)");
  if (nvec < 0 || nvec > kMaxVec)
    return fail(HZ_ERR_INVALID, "hz_residual_noalloc: nvec must be in [0, 64]");
  if (nvec == 0) return HZ_OK;
  if (!f || !norm2 || (u && !c))
    return fail(HZ_ERR_INVALID, "hz_residual_noalloc: null f, norm2 or c");
  const long long n = (long long)grid->nx * grid->ny * grid->nz;
  const long long nblk = (n + kChunk - 1) / kChunk;
  if (nblk * nvec > kMaxPartials || nblk > 0x7fffffffLL)
    return fail(HZ_ERR_INVALID,
                "hz_residual_noalloc: nvec * ceil(n/1024) = " + std::to_string(nblk * nvec) +
                    " exceeds the static scratch of 65536 block partials");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(HZ_ERR_CUDA, std::string("hz_residual_noalloc: cudaGetDevice: ") +
                                 cudaGetErrorString(e));
  double2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_addr[dev]) {
      // the array's name is only a host-side stand-in: ask the runtime for the address of
      // this device's copy (the current device is `dev`)
      e = cudaGetSymbolAddress((void**)&g_dev_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_dev_addr[dev] = nullptr;
        return fail(HZ_ERR_CUDA, std::string("hz_residual_noalloc: cudaGetSymbolAddress: ") +
                                     cudaGetErrorString(e));
      }
    }
    scratch = g_dev_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* tickets = (unsigned*)(scratch + kMaxPartials);
  e = cudaMemsetAsync(tickets, 0, sizeof(unsigned) * nvec, st);
  if (e != cudaSuccess)
    return fail(HZ_ERR_CUDA, std::string("hz_residual_noalloc: clearing tickets: ") +
                                 cudaGetErrorString(e));
  const double s = c_min * c_min / (grid->omega * grid->omega);
  const double cs = s / (grid->h * grid->h);
  hz::count_launch();
  k_residual_noalloc<<<dim3((unsigned)nblk, nvec), kThreads, 0, st>>>(
      grid->nx, grid->ny, grid->nz, grid->layer_cells, cs, grid->sigma_max, c_min * c_min, c,
      (const double2*)f, fscale, (const double2*)u, (double2*)r, norm2, scratch, tickets);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(HZ_ERR_CUDA, std::string("hz_residual_noalloc: launch: ") + cudaGetErrorString(e));
  return HZ_OK;
}
