// Device helpers shared by the kernel translation units of libhz: complex arithmetic on
// float2/double2, deterministic block reductions with a "last block" ticket, and the Givens
// step of a (F)GMRES column.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "hz_internal.h"

namespace hz {
namespace {

// ---------------------------------------------------------------- complex helpers
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename T> __device__ __forceinline__ T czero() { T z; z.x = 0; z.y = 0; return z; }
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- reductions
// Sum of v over the block; the result is valid in thread 0.  sh holds >= 32 entries.
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

// Ticket of the last block of this rhs; true in every thread of that block.
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// In the last block: out[s] = sum over blocks of part[s][b], s < nslots, in block order.
__device__ void finish_slots(const double2* part, int nslots, double2* out, double2* sh) {
  for (int s = 0; s < nslots; ++s) {
    double2 acc = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      double2 v = __ldcg(part + (long long)s * gridDim.x + b);
      acc.x += v.x;
      acc.y += v.y;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[s] = acc;
  }
}

// Givens step for column k of rhs r (Saad's GMRES with complex rotations), called by every
// thread of one block.  The new Hessenberg column and the previous rotations are staged in
// shared memory first, so the sequential rotation sweep of thread 0 does not wait on a
// global-memory round trip per rotation.
constexpr int kGivMax = 130;  // restart lengths up to 128

__device__ void givens_column(const GmresDev& gs, int r, int k, double brk) {
  __shared__ double2 sR[kGivMax];
  __shared__ double scc[kGivMax];
  __shared__ double2 sss[kGivMax];
  const int M = gs.mmax;
  const double2* h1 = gs.h1 + (long long)r * (M + 2);
  const double2* h2 = gs.h2 + (long long)r * (M + 2);
  const double* cc = gs.cc + (long long)r * M;
  const double2* ss = gs.ss + (long long)r * M;
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    sR[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
    if (i < k) {
      scc[i] = cc[i];
      sss[i] = ss[i];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* sc = gs.scal + (long long)r * SC_COUNT;
  const double hn = sqrt(gs.nrm[2 * r].x);
  const double wn = sqrt(h1[k + 1].x);
  for (int i = 0; i < k; ++i) {
    const double c = scc[i];
    const double2 s = sss[i], a = sR[i], b = sR[i + 1];
    sR[i] = cadd(mk(c * a.x, c * a.y), cmul(s, b));
    sR[i + 1] = cadd(mk(-(s.x * a.x + s.y * a.y), -(s.x * a.y - s.y * a.x)), mk(c * b.x, c * b.y));
  }
  double c;
  double2 s;
  const double2 a = sR[k];
  if (hn == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (a.x == 0.0 && a.y == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    const double ra = hypot(a.x, a.y);
    const double rr = hypot(ra, hn);
    c = ra / rr;
    s = make_double2(a.x / ra * hn / rr, a.y / ra * hn / rr);
  }
  sR[k] = cadd(mk(c * a.x, c * a.y), mk(s.x * hn, s.y * hn));
  double2* R = gs.R + (long long)r * (M + 1) * M + (long long)k * (M + 1);
  for (int i = 0; i <= k; ++i) R[i] = sR[i];
  R[k + 1] = make_double2(0.0, 0.0);
  gs.cc[(long long)r * M + k] = c;
  gs.ss[(long long)r * M + k] = s;
  double2* gg = gs.g + (long long)r * (M + 1);
  const double2 gk = gg[k];
  gg[k] = mk(c * gk.x, c * gk.y);
  const double2 gk1 = mk(-(s.x * gk.x + s.y * gk.y), -(s.x * gk.y - s.y * gk.x));
  gg[k + 1] = gk1;
  const double est = hypot(gk1.x, gk1.y);
  const bool brk_now = hn <= brk * wn;
  sc[SC_EST] = est;
  sc[SC_HN] = hn;
  sc[SC_INV] = brk_now ? 0.0 : 1.0 / hn;
  gs.kend[r] = k + 1;
  if (brk_now || est <= sc[SC_TOL]) gs.stopped[r] = 1;
}

}  // namespace
}  // namespace hz
