// Device helpers shared by the kernel translation units of libhz: complex arithmetic on
// float2/double2, deterministic block reductions with a "last block" ticket, and the Givens
// step of a (F)GMRES column.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "hz_internal.h"

namespace hz {

// ---------------------------------------------------------------- programmatic dependent launch
// Every kernel launched with launch_pdl starts with pdl_enter(): wait until the kernel before
// it on the stream has completed and its writes are visible.  Programmatic stream
// serialization lets a dependent kernel's launch overlap the end of the one before it (the
// solver is a chain of short dependent kernels; CUDA graphs keep the programmatic edges).
// Nothing is read or written before the wait, so the ordering of the stream is unchanged.  No
// kernel triggers its dependents early (griddepcontrol.launch_dependents): measured on the
// 64^3 solve, a trigger right after the wait made it 38% slower.  Kernels without
// pdl_enter() are launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

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

// ---------------------------------------------------------------- float pairs
// Float pairs (hi + lo, |lo| <= half an ulp of hi) for sums that float32 alone would round
// too coarsely.  two_sum is Knuth's error-free sum; two_prod_ff(a, bh, bl) = a * (bh + bl) with
// the product a * bh split exactly by an FMA.  The _rn intrinsics keep the compiler from
// contracting or reordering these steps.
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  const float lo = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
  return two_sum(s.x, lo);
}

__device__ __forceinline__ float2 two_prod_ff(float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  const float e = __fmaf_rn(a, bh, -p);
  return two_sum(p, __fmaf_rn(a, bl, e));
}

// (hi, lo) -> the same value with |lo| <= half an ulp of hi, given |a| >= |b| (Dekker).
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// acc += a * b for float pairs, with acc.lo left unnormalised (it gathers the rounding errors
// of a few terms; ff_norm restores the pair): 1 multiply, 3 FMA, 1 two_sum, 2 adds.
__device__ __forceinline__ void ff_acc_mul(float2& acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float2 s = two_sum(acc.x, p);
  acc.x = s.x;
  acc.y = __fadd_rn(acc.y, __fadd_rn(s.y, e));
}

__device__ __forceinline__ float2 ff_norm(float2 a) { return two_sum(a.x, a.y); }

// float64 -> float pair (two float64-pipe conversions and one subtraction) and back.
__device__ __forceinline__ float2 ff_from_d(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - double(h)));
}
__device__ __forceinline__ double d_from_ff(float2 a) { return double(a.x) + double(a.y); }

// Complex float pairs: float4 (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ float4 ffc_add(float4 a, float4 b) {
  const float2 re = ff_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
  const float2 im = ff_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
  return make_float4(re.x, re.y, im.x, im.y);
}
__device__ __forceinline__ float4 ffc_of(float2 v) { return make_float4(v.x, 0.f, v.y, 0.f); }
__device__ __forceinline__ float4 shfl_xor4(float4 v, int m) {
  return make_float4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                     __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}
__device__ __forceinline__ double2 d_from_ffc(float4 v) {
  return make_double2(d_from_ff(make_float2(v.x, v.y)), d_from_ff(make_float2(v.z, v.w)));
}
__device__ __forceinline__ float2 f_from_ffc(float4 v) {
  return make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
}

// In the last block, one warp: the float-pair sum over the G block partials of slot sidx
// (part[sidx][b], float4), valid in every lane.  Float32 instructions only (on GB300 a
// float64 instruction issues at 1/64 of the float32 rate, which made float64 partial sums the
// longest part of the small reduction kernels); eight loads per lane in flight; fixed order.
__device__ __forceinline__ float4 warp_sum_partials_ff(const float4* part, int sidx, int G,
                                                       int lane) {
  const float4* ps = part + (long long)sidx * G;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int b0 = 0; b0 < G; b0 += 32 * 8) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < G ? __ldcg(ps + b) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = ffc_add(acc, v[u]);
  }
  for (int o = 16; o > 0; o >>= 1) acc = ffc_add(acc, shfl_xor4(acc, o));
  return acc;
}

// The same sum in compact code, for the cooperative kernels.  Their reductions run between long
// passes that have pushed them out of the instruction cache, and there an
// unrolled float-pair sequence costs several cycles per instruction in fetches (measured: the
// cooperative outer Arnoldi step 1.5% faster per solve with this form, while the short
// reduction kernels were 1.5% slower with it); one out-of-line add serves every step.
__device__ __noinline__ float4 ffc_add_n(float4 a, float4 b) { return ffc_add(a, b); }

__device__ __forceinline__ float4 warp_sum_partials_ffn(const float4* part, int sidx, int G,
                                                        int lane) {
  const float4* ps = part + (long long)sidx * G;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int b0 = 0; b0 < G; b0 += 32 * 8) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < G ? __ldcg(ps + b) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // a pairwise tree over the eight loads, then into the running sum
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = ffc_add_n(v[u], v[u + 4]);
    v[0] = ffc_add_n(v[0], v[2]);
    v[1] = ffc_add_n(v[1], v[3]);
    acc = ffc_add_n(acc, ffc_add_n(v[0], v[1]));
  }
#pragma unroll 1
  for (int o = 16; o > 0; o >>= 1) acc = ffc_add_n(acc, shfl_xor4(acc, o));
  return acc;
}

// ---------------------------------------------------------------- complex64 stencil
// y[t] = ((A - zI) x) at (i, j, k0 + t), t < ZC, from the precomputed complex64 diagonal
// (dg = 6 s/h^2 - m - i a):  (dg - z) x - (s/h^2) * (sum of the 6 neighbours), Dirichlet
// zeros outside.  All loads of the column are issued together and the z-neighbours of one
// point are the centres of the next.  Points beyond nz give 0.  (i, j) must be inside.
template <int ZC>
__device__ __forceinline__ void stencil32_column(const Geom& g, const float2* __restrict__ dg,
                                                 const float2* __restrict__ xr, int i, int j,
                                                 int k0, float zr, float zi, float2 (&y)[ZC]) {
  const long long sxy = (long long)g.nx * g.ny;
  const long long p0 = i + (long long)g.nx * j + sxy * k0;
  const float2 zero = make_float2(0.f, 0.f);
  float2 dv[ZC], xm[ZC], xp[ZC], ym[ZC], yp[ZC], c[ZC + 2];
#pragma unroll
  for (int t = 0; t < ZC; ++t) {
    const bool ok = k0 + t < g.nz;
    const long long pp = p0 + sxy * t;
    dv[t] = ok ? dg[pp] : zero;
    xm[t] = (ok && i > 0) ? xr[pp - 1] : zero;
    xp[t] = (ok && i < g.nx - 1) ? xr[pp + 1] : zero;
    ym[t] = (ok && j > 0) ? xr[pp - g.nx] : zero;
    yp[t] = (ok && j < g.ny - 1) ? xr[pp + g.nx] : zero;
  }
#pragma unroll
  for (int t = 0; t < ZC + 2; ++t) {
    const int kz = k0 + t - 1;
    c[t] = (kz >= 0 && kz < g.nz) ? xr[p0 + sxy * (t - 1)] : zero;
  }
  const float cs = g.csf;
#pragma unroll
  for (int t = 0; t < ZC; ++t) {
    const float2 xc = c[t + 1];
    const float nbx = ((xm[t].x + xp[t].x) + (ym[t].x + yp[t].x)) + (c[t].x + c[t + 2].x);
    const float nby = ((xm[t].y + xp[t].y) + (ym[t].y + yp[t].y)) + (c[t].y + c[t + 2].y);
    const float dr = dv[t].x - zr, di = dv[t].y - zi;
    y[t] = k0 + t < g.nz
               ? make_float2(dr * xc.x - di * xc.y - cs * nbx, dr * xc.y + di * xc.x - cs * nby)
               : zero;
  }
}

// Butterfly reduction of 8 per-lane complex partials over a warp: after the three exchange
// steps each lane holds one vector's partial (vector index bits = lane bits 4, 3, 2), and two
// more xor steps finish it.  18 float64 adds reduce 8 vectors, against 80 for 8 separate
// shuffle trees -- float64 is the scarce pipe.  Lane l with (l & 3) == 0 ends with the sum
// of vector ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1).
__device__ __forceinline__ double2 warp_reduce8(double2 (&a)[8], int lane) {
  double2 b4[4], b2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const double2 keep = h16 ? a[4 + t] : a[t];
    const double2 give = h16 ? a[t] : a[4 + t];
    b4[t] = make_double2(keep.x + __shfl_xor_sync(0xffffffffu, give.x, 16),
                         keep.y + __shfl_xor_sync(0xffffffffu, give.y, 16));
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const double2 keep = h8 ? b4[2 + t] : b4[t];
    const double2 give = h8 ? b4[t] : b4[2 + t];
    b2[t] = make_double2(keep.x + __shfl_xor_sync(0xffffffffu, give.x, 8),
                         keep.y + __shfl_xor_sync(0xffffffffu, give.y, 8));
  }
  const double2 keep = h4 ? b2[1] : b2[0];
  const double2 give = h4 ? b2[0] : b2[1];
  double x = keep.x + __shfl_xor_sync(0xffffffffu, give.x, 4);
  double y = keep.y + __shfl_xor_sync(0xffffffffu, give.y, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  return make_double2(x, y);
}

// ---------------------------------------------------------------- float-pair complex fields
__device__ __forceinline__ float2 re_of(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 im_of(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }

// Butterfly reduce-scatter of 8 complex float-pair partials over a warp (the lane map of
// warp_reduce8 above): lane l with (l & 3) == 0 ends with the sum of vector
// ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1).
__device__ __forceinline__ float4 warp_reduce8_ff(float4 (&a)[8], int lane) {
  float4 b4[4], b2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float4 keep = h16 ? a[4 + t] : a[t];
    const float4 give = h16 ? a[t] : a[4 + t];
    b4[t] = ffc_add(keep, shfl_xor4(give, 16));
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float4 keep = h8 ? b4[2 + t] : b4[t];
    const float4 give = h8 ? b4[t] : b4[2 + t];
    b2[t] = ffc_add(keep, shfl_xor4(give, 8));
  }
  const float4 keep = h4 ? b2[1] : b2[0];
  const float4 give = h4 ? b2[0] : b2[1];
  float4 x = ffc_add(keep, shfl_xor4(give, 4));
  x = ffc_add(x, shfl_xor4(x, 2));
  x = ffc_add(x, shfl_xor4(x, 1));
  return x;
}

// Butterfly reduction of 8 per-lane float2 partials over a warp (same lane map as the float64
// version above): lane l with (l & 3) == 0 ends with the sum of vector
// ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1).
__device__ __forceinline__ float2 warp_reduce8f(float2 (&a)[8], int lane) {
  float2 b4[4], b2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float2 keep = h16 ? a[4 + t] : a[t];
    const float2 give = h16 ? a[t] : a[4 + t];
    b4[t] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, give.x, 16),
                        keep.y + __shfl_xor_sync(0xffffffffu, give.y, 16));
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float2 keep = h8 ? b4[2 + t] : b4[t];
    const float2 give = h8 ? b4[t] : b4[2 + t];
    b2[t] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, give.x, 8),
                        keep.y + __shfl_xor_sync(0xffffffffu, give.y, 8));
  }
  const float2 keep = h4 ? b2[1] : b2[0];
  const float2 give = h4 ? b2[0] : b2[1];
  float x = keep.x + __shfl_xor_sync(0xffffffffu, give.x, 4);
  float y = keep.y + __shfl_xor_sync(0xffffffffu, give.y, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  return make_float2(x, y);
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- grid barrier
// Grid barrier over nblocks resident blocks: bar[0] counts arrivals, bar[1] is the generation,
// bar[3] the poll limit (set by the host; GRID_SPINS_DEFAULT unless changed).  Arrival is an
// acquire-release atomic (it publishes the block's writes, ordered before it by the block
// barrier, and the last arriver sees everyone's); the last arriver resets the count and
// releases the next generation; the others poll the generation with acquire loads, first back
// to back, then with a short sleep, at most bar[3] times.  false if this block gave up (or
// another already had): the caller returns.
__device__ bool grid_sync(unsigned* bar, unsigned nblocks, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen, old, spins;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(spins) : "l"(bar + 3) : "memory");
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    if (old == nblocks - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
      ok = 1;
    } else {
      ok = 0;
      for (unsigned it = 0; it < spins; ++it) {
        unsigned now;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(bar + 1) : "memory");
        if (now != gen) {
          ok = 1;
          break;
        }
        if (*(volatile int*)err) break;
        if (it >= 64) __nanosleep(32);
      }
      if (!ok) atomicExch(err, 1);
    }
  }
  __syncthreads();
  return ok != 0;
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
    for (int b0 = 0; b0 < (int)gridDim.x; b0 += 4 * blockDim.x) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u * blockDim.x + threadIdx.x;
        v[u] = b < (int)gridDim.x ? __ldcg(part + (long long)s * gridDim.x + b)
                                  : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc.x += v[u].x;
        acc.y += v[u].y;
      }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[s] = acc;
  }
}

// In the last block, one warp: the sum over the G block partials of slot sidx (part[sidx][b]),
// valid in lane 0.  Eight independent loads per lane are in flight at a time (a dependent
// chain of L2 round trips here would be the longest part of a small reduction kernel); the
// order of the additions is fixed, so results are bit-reproducible.
__device__ __forceinline__ double2 warp_sum_partials(const double2* part, int sidx, int G,
                                                     int lane) {
  const double2* ps = part + (long long)sidx * G;
  double ax = 0.0, ay = 0.0;
  for (int b0 = 0; b0 < G; b0 += 32 * 8) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = b0 + u * 32 + lane;
      v[u] = b < G ? __ldcg(ps + b) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ax += v[u].x;
      ay += v[u].y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, o);
    ay += __shfl_down_sync(0xffffffffu, ay, o);
  }
  return make_double2(ax, ay);
}

// Givens step for column k of rhs r (Saad's GMRES with complex rotations), called by every
// thread of one block; warp 0 does the work.
//
// Applying rotations 0..k-1 to the new column h is a chain through one value: with t_0 = h_0,
// rotation i leaves R_i = c_i t_i + s_i h_{i+1} and passes on t_{i+1} = -conj(s_i) t_i +
// c_i h_{i+1}.  That recurrence is affine in t, so the warp evaluates it as a prefix scan of
// the maps t -> a t + b (lane l composes a chunk of ceil(k/32) consecutive rotations, a
// Kogge-Stone scan over the lanes gives each chunk its incoming t, then the chunks produce
// their R_i): about 10 + 2 ceil(k/32) dependent float64 steps in place of 2k, which matters on
// a GPU whose float64 pipe spends 64 cycles on each warp instruction.  Since |a| = |s_i| <= 1
// the composed maps do not grow; the rounding differs from the sequential sweep only in order.
constexpr int kGivMax = 130;  // restart lengths up to 128

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ double2 shfl_up2(double2 v, int o) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o));
}

// The step itself, run by one whole warp (lane = threadIdx.x & 31) once h1, h2 and the norm of
// column k are in memory and visible to it.
__device__ void givens_column_warp(const GmresDev& gs, int r, int k, double brk) {
  const int lane = threadIdx.x & 31;
  const int M = gs.mmax;
  const double2* h1 = gs.h1 + (long long)r * (M + 2);
  const double2* h2 = gs.h2 + (long long)r * (M + 2);
  const double* cc = gs.cc + (long long)r * M;
  const double2* ss = gs.ss + (long long)r * M;
  double2* R = gs.R + (long long)r * (M + 1) * M + (long long)k * (M + 1);
  auto hcol = [&](int i) { return make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y); };
  const int q = (k + 31) / 32;  // rotations per lane
  const int i0 = min(lane * q, k), i1 = min(i0 + q, k);
  // this lane's maps composed: t -> A t + B
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
  for (int i = i0; i < i1; ++i) {
    const double c = cc[i];
    const double2 s = ss[i], al = make_double2(-s.x, s.y), hn1 = hcol(i + 1);
    B = cfma(al, B, make_double2(c * hn1.x, c * hn1.y));
    A = cmul(al, A);
  }
  // inclusive scan over the lanes (earlier lanes' maps applied first), then shifted by one
#pragma unroll 1
  for (int o = 1; o < 32; o <<= 1) {
    const double2 Ap = shfl_up2(A, o), Bp = shfl_up2(B, o);
    if (lane >= o) {
      B = cfma(A, Bp, B);
      A = cmul(A, Ap);
    }
  }
  double2 Ax = shfl_up2(A, 1), Bx = shfl_up2(B, 1);
  if (lane == 0) {
    Ax = make_double2(1.0, 0.0);
    Bx = make_double2(0.0, 0.0);
  }
  double2 t = cfma(Ax, hcol(0), Bx);  // t_{i0}
  for (int i = i0; i < i1; ++i) {
    const double c = cc[i];
    const double2 s = ss[i], hn1 = hcol(i + 1);
    R[i] = cfma(s, hn1, make_double2(c * t.x, c * t.y));
    t = cfma(make_double2(-s.x, s.y), t, make_double2(c * hn1.x, c * hn1.y));
  }
  // the lane holding t_k: the one whose chunk ends at rotation k - 1 (lane 0 when k = 0)
  const int last = k == 0 ? 0 : (k - 1) / q;
  if (lane != last) return;
  double* sc = gs.scal + (long long)r * SC_COUNT;
  const double hn = sqrt(gs.nrm[2 * r].x);
  const double wn = sqrt(h1[k + 1].x);
  double c;
  double2 s;
  const double2 a = t;
  if (hn == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (a.x == 0.0 && a.y == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    const double ra = hypot(a.x, a.y);
    const double irr = 1.0 / hypot(ra, hn);
    c = ra * irr;
    const double f = hn * irr / ra;
    s = make_double2(a.x * f, a.y * f);
  }
  R[k] = cadd(mk(c * a.x, c * a.y), mk(s.x * hn, s.y * hn));
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

__device__ void givens_column(const GmresDev& gs, int r, int k, double brk) {
  __syncthreads();  // the caller's stores of h1, h2 and the norm come first
  if (threadIdx.x < 32) givens_column_warp(gs, r, k, brk);
}

// ---------------------------------------------------------------- float-pair products
// Double-float product after Dekker (1971): hi from the float32 product, its rounding error
// exactly from an FMA, the cross terms added; about 48 significant bits.
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, neg(b)); }

}  // namespace
}  // namespace hz
