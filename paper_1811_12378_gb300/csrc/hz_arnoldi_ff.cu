// One step of the outer float-pair Arnoldi (HZ_MIXED_C64_FF form, one right-hand side) as one
// cooperative kernel: w = A z_k (float64 stencil, rounded to float pairs), the two classical
// Gram-Schmidt passes against v_0..v_k, ||w||, the Givens step of the new Hessenberg column
// and v_{k+1} = w / h_{k+1,k} with its complex64 rounding, the next FCI application's input
// (the Arnoldi process of FGMRES, Section 3, with the CGS2 orthogonalisation).  The Givens step
// and its least-squares state are float64 (givens_column, block 0).
//
// Per point the arithmetic is that of the multi-kernel form (k_stencil_diag<true>,
// k_cgs_ff<0..2>, k_scale_ff): the same float-pair products in the same order, the same
// float64 coefficients rounded to float pairs.  Only the grouping of the global sums differs.
// The five launches of that form spend much of their time in ramps, in a partial second wave
// and in the serial finish of each reduction by its last block.  Here the grid stays resident
// (one block of 512 threads on every SM), each block owns a contiguous range of points and
// keeps its part of w in shared memory through every pass, and the passes are separated by two
// grid barriers (three where the Pythagorean norm of the last pass would cancel, see below).
// After each barrier every block adds all blocks' float-pair partials in the same fixed order,
// so every block holds the same coefficients without a broadcast.  Block 0 alone writes the
// Hessenberg column, and its first warp runs the Givens step while the other warps, and every
// other block, run the last pass.
//
// The barrier spins with a bound (about a second); a block that gives up sets the error flag
// and returns, the others then skip their waits, and the host reports the flag after the solve.
#include <cuda_runtime.h>

#include <algorithm>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int AT = 512;  // threads per block, one block per SM
constexpr int AWARPS = AT / 32;

struct Arn {
  Geom g;
  const double2* dg;  // float64 diagonal 6 s/h^2 - m - i a
  const double2* z;   // z_k, the FCI output
  const float4* V;    // basis v_0..v_{nb-1}, float-pair fields of n points
  float4* vnext;      // v_nb
  float2* y32;        // complex64 rounding of v_nb
  GmresDev gs;
  float4* part;       // two halves of (mmax + 2) slots x G block partials
  unsigned* bar;
  int* err;
  long long n;
  int nb;
  int pyth;  // 0: always sum the norm of the last pass
  double brk;
};

// Partials of phase q live in half (q & 1): a block past barrier q + 1 may write phase q + 2
// while no block still reads phase q (each finished that reduction before arriving at q + 1).
__device__ __forceinline__ float4* arn_part(const Arn& a, int q) {
  return a.part + (long long)(q & 1) * (a.gs.mmax + 2) * gridDim.x;
}

// This thread's points are pbeg + threadIdx.x + e AT (e < ppt, below pend); w lives in shared
// memory at sw[e AT + threadIdx.x].  The loops over e are not unrolled (one copy of each pass's
// body keeps the kernel inside the instruction cache) and take two points per iteration, so 16
// loads of basis elements are in flight per thread.
struct Pts {
  long long t0, pend;
  int ppt;
};

__device__ __forceinline__ float4 ld_v(const Arn& a, int b, long long p, bool ok) {
  return ok ? __ldg(a.V + (long long)b * a.n + p) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Per-warp dots conj(v_b) w for b < nb, 8 fields at a time, reduced over the warp into
// wp[warp][b].
__device__ __forceinline__ void warp_dots(const Arn& a, const Pts& P, const float4* sw, float4* wp,
                                          int ldw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = a.nb;
  for (int b0 = 0; b0 < nb; b0 += 8) {
    float2 are[8], aim[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) are[t] = aim[t] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int e = 0; e < P.ppt; e += 2) {
      const long long p0 = P.t0 + (long long)e * AT, p1 = p0 + AT;
      const bool ok0 = p0 < P.pend, ok1 = e + 1 < P.ppt && p1 < P.pend;
      float4 v0[8], v1[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v0[t] = ld_v(a, b0 + t, p0, ok0 && b0 + t < nb);
        v1[t] = ld_v(a, b0 + t, p1, ok1 && b0 + t < nb);
      }
      const float4 w0 = ok0 ? sw[e * AT + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 w1 = ok1 ? sw[(e + 1) * AT + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          float2 vre = re_of(v0[t]), vim = im_of(v0[t]);
          ff_acc_mul(are[t], vre, re_of(w0));
          ff_acc_mul(are[t], vim, im_of(w0));
          ff_acc_mul(aim[t], vre, im_of(w0));
          ff_acc_mul(aim[t], neg(vim), re_of(w0));
          vre = re_of(v1[t]);
          vim = im_of(v1[t]);
          ff_acc_mul(are[t], vre, re_of(w1));
          ff_acc_mul(are[t], vim, im_of(w1));
          ff_acc_mul(aim[t], vre, im_of(w1));
          ff_acc_mul(aim[t], neg(vim), re_of(w1));
          are[t] = ff_norm(are[t]);
          aim[t] = ff_norm(aim[t]);
        }
      }
    }
    float4 acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = make_float4(are[t].x, are[t].y, aim[t].x, aim[t].y);
    const float4 red = warp_reduce8_ff(acc, lane);
    if ((lane & 3) == 0) {
      const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
      if (b0 + t < nb) wp[warp * ldw + b0 + t] = red;
    }
  }
}

// ||w||^2 over this thread's points, reduced over the warp into wp[warp][slot].
__device__ __forceinline__ void warp_norm(const Pts& P, const float4* sw, float4* wp, int ldw,
                                          int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 q = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int e = 0; e < P.ppt; ++e) {
    if (P.t0 + (long long)e * AT < P.pend) {
      const float4 w = sw[e * AT + threadIdx.x];
      ff_acc_mul(q, re_of(w), re_of(w));
      ff_acc_mul(q, im_of(w), im_of(w));
      q = ff_norm(q);
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    q = ff_add(q, make_float2(__shfl_xor_sync(0xffffffffu, q.x, o),
                              __shfl_xor_sync(0xffffffffu, q.y, o)));
  if (lane == 0) wp[warp * ldw + slot] = make_float4(q.x, q.y, 0.f, 0.f);
}

// w += V (-h) (hf: the negated coefficients as float pairs), then w renormalised; per point
// the products come in the order of k_cgs_ff.
__device__ __forceinline__ void update(const Arn& a, const Pts& P, float4* sw, const float4* hf) {
  const int nb = a.nb;
#pragma unroll 1
  for (int e = 0; e < P.ppt; e += 2) {
    const long long p0 = P.t0 + (long long)e * AT, p1 = p0 + AT;
    const bool ok0 = p0 < P.pend, ok1 = e + 1 < P.ppt && p1 < P.pend;
    float4 w0 = ok0 ? sw[e * AT + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 w1 = ok1 ? sw[(e + 1) * AT + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 r0 = re_of(w0), i0 = im_of(w0), r1 = re_of(w1), i1 = im_of(w1);
#pragma unroll 1
    for (int b0 = 0; b0 < nb; b0 += 8) {
      float4 v0[8], v1[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v0[t] = ld_v(a, b0 + t, p0, ok0 && b0 + t < nb);
        v1[t] = ld_v(a, b0 + t, p1, ok1 && b0 + t < nb);
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          const float4 nh = hf[b0 + t];
          const float2 nre = re_of(nh), nim = im_of(nh), mnim = neg(nim);
          float2 vre = re_of(v0[t]), vim = im_of(v0[t]);
          ff_acc_mul(r0, vre, nre);
          ff_acc_mul(r0, vim, mnim);
          ff_acc_mul(i0, vre, nim);
          ff_acc_mul(i0, vim, nre);
          vre = re_of(v1[t]);
          vim = im_of(v1[t]);
          ff_acc_mul(r1, vre, nre);
          ff_acc_mul(r1, vim, mnim);
          ff_acc_mul(i1, vre, nim);
          ff_acc_mul(i1, vim, nre);
        }
      }
    }
    r0 = ff_norm(r0);
    i0 = ff_norm(i0);
    r1 = ff_norm(r1);
    i1 = ff_norm(i1);
    if (ok0) sw[e * AT + threadIdx.x] = make_float4(r0.x, r0.y, i0.x, i0.y);
    if (ok1) sw[(e + 1) * AT + threadIdx.x] = make_float4(r1.x, r1.y, i1.x, i1.y);
  }
}

// The block's partials of ns slots (summed over its warps in order) to part[s][block].
__device__ __forceinline__ void block_partial(float4* part, const float4* wp, int ldw, int ns) {
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += AT) {
    float4 t = wp[s];
    for (int w = 1; w < AWARPS; ++w) t = ffc_add(t, wp[w * ldw + s]);
    part[(long long)s * gridDim.x + blockIdx.x] = t;
  }
}

// After the barrier, in every block: h[s] = the float-pair sum over all blocks of slot s
// (s < ns), in a fixed order, so the same bits in every block; hf[s] = -h[s] for s < nneg (the
// coefficients k_cgs_ff loads: its float64 round trip of a normalised pair is exact).
__device__ __forceinline__ void grid_reduce(const float4* part, int ns, float4* h, float4* hf,
                                            int nneg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = warp; s < ns; s += AWARPS) {
    const float4 v = warp_sum_partials_ffn(part, s, (int)gridDim.x, lane);
    if (lane == 0) {
      h[s] = v;
      if (s < nneg) hf[s] = make_float4(-v.x, -v.y, -v.z, -v.w);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(AT, 1) k_arnoldi_ff(Arn a, int ppt) {
  pdl_enter();
  // sw[ppt][AT] | wp[AWARPS][nb + 8] | hf, h1f, h2f[nb + 1] (float pairs)
  extern __shared__ float4 sm4[];
  __shared__ float2 s_inv, s_hn2;
  __shared__ int s_fast;
  if (a.gs.stopped[0]) return;  // uniform: no block of this grid writes it before barrier 1
  const int nb = a.nb, ldw = nb + 8;
  float4* sw = sm4;
  float4* wp = sw + ppt * AT;
  float4* hf = wp + AWARPS * ldw;
  float4* h1f = hf + nb + 1;
  float4* h2f = h1f + nb + 1;
  const unsigned G = gridDim.x;
  const long long n = a.n;
  Pts P;
  P.t0 = (long long)blockIdx.x * n / G + threadIdx.x;
  P.pend = (long long)(blockIdx.x + 1) * n / G;
  P.ppt = ppt;
  const Geom& g = a.g;

  // ---- w = A z_k at this thread's points (float64, as k_stencil_diag), as float pairs
  {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const double2 z0 = make_double2(0.0, 0.0);
    const double mcs = -g.cs;
#pragma unroll 1
    for (int e = 0; e < ppt; ++e) {
      const long long p = P.t0 + (long long)e * AT;
      if (p < P.pend) {
        const int pi = int(p);  // n < 2^31
        const int k = pi / int(sz);
        const int rem = pi - k * int(sz);
        const int j = rem / g.nx;
        const int i = rem - j * g.nx;
        const double2* x = a.z;
        const double2 xm = i > 0 ? __ldg(x + p - 1) : z0;
        const double2 xp = i < g.nx - 1 ? __ldg(x + p + 1) : z0;
        const double2 ym = j > 0 ? __ldg(x + p - sy) : z0;
        const double2 yp = j < g.ny - 1 ? __ldg(x + p + sy) : z0;
        const double2 zm = k > 0 ? __ldg(x + p - sz) : z0;
        const double2 zp = k < g.nz - 1 ? __ldg(x + p + sz) : z0;
        const double2 xc = __ldg(x + p);
        const double2 d = __ldg(a.dg + p);
        const double nbx = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
        const double nby = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
        const double yx = fma(d.x, xc.x, fma(-d.y, xc.y, mcs * nbx));
        const double yy = fma(d.x, xc.y, fma(d.y, xc.x, mcs * nby));
        const float2 re = ff_from_d(yx), im = ff_from_d(yy);
        sw[e * AT + threadIdx.x] = make_float4(re.x, re.y, im.x, im.y);
      }
    }
  }
  // (each thread reads back only its own elements of sw before the next __syncthreads)

  // ---- first pass: h1 = V^H w, and ||w||^2 in slot nb
  warp_dots(a, P, sw, wp, ldw);
  warp_norm(P, sw, wp, ldw, nb);
  block_partial(arn_part(a, 0), wp, ldw, nb + 1);
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce(arn_part(a, 0), nb + 1, h1f, hf, nb);

  // ---- second pass: w -= V h1, then h2 = V^H w and ||w||^2 (slot nb)
  update(a, P, sw, hf);
  warp_dots(a, P, sw, wp, ldw);
  warp_norm(P, sw, wp, ldw, nb);
  block_partial(arn_part(a, 1), wp, ldw, nb + 1);
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce(arn_part(a, 1), nb + 1, h2f, hf, nb);

  // ---- h_{k+1,k}^2 = ||w - V h2||^2 = ||w||^2 - ||h2||^2: V is orthonormal and w already
  // nearly orthogonal to it, so the second pass removes little and the difference keeps its
  // accuracy; then no further reduction is needed.  Where the second pass removed more than
  // three quarters of ||w||^2 (w close to the span of V, the subtraction would cancel), the
  // norm of w - V h2 is summed instead.  Every block sees the same sums: the branch is uniform.
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float2 q = make_float2(0.f, 0.f);
    for (int b = lane; b < nb; b += 32) {
      const float4 h = h2f[b];
      q = ff_add(q, ff_add(ff_mul(re_of(h), re_of(h)), ff_mul(im_of(h), im_of(h))));
    }
    for (int o = 16; o > 0; o >>= 1)
      q = ff_add(q, make_float2(__shfl_xor_sync(0xffffffffu, q.x, o),
                                __shfl_xor_sync(0xffffffffu, q.y, o)));
    if (lane == 0) {
      const float2 wq = re_of(h2f[nb]);
      const float2 hp = ff_sub(wq, q);
      s_fast = a.pyth && hp.x > 0.25f * wq.x ? 1 : 0;
      s_hn2 = hp;
    }
  }
  __syncthreads();
  const float2 wn2 = re_of(h1f[nb]);
  // v_{k+1} = w / h_{k+1,k} (zero at a breakdown): the float64 test and scale of the Givens
  // step (givens_column), from the same float64 values it reads
  auto set_inv = [&](float2 hn2) {
    const double hn = sqrt(d_from_ff(hn2)), wn = sqrt(d_from_ff(wn2));
    s_inv = ff_from_d(hn <= a.brk * wn ? 0.0 : 1.0 / hn);
  };
  // block 0: the Hessenberg column and the norms in float64 for the Givens step
  auto store_column = [&](float2 hn2) {
    for (int i = threadIdx.x; i <= nb; i += AT) {
      a.gs.h1[i] = d_from_ffc(h1f[i]);
      if (i < nb) a.gs.h2[i] = d_from_ffc(h2f[i]);
    }
    if (threadIdx.x == 0) a.gs.nrm[0] = make_double2(d_from_ff(hn2), 0.0);
  };
  bool givens_done = false;
  if (s_fast) {
    // h_{k+1,k} is known: block 0's first warp runs the Givens step (serial float64, about
    // 14 us) while the other warps start the last pass, and does its own points after it
    const float2 hn2 = s_hn2;
    if (threadIdx.x == 0) set_inv(hn2);
    if (blockIdx.x == 0) store_column(hn2);
    __syncthreads();  // uniform: s_fast is the same in every thread
    if (blockIdx.x == 0 && threadIdx.x < 32) givens_column_warp(a.gs, 0, nb - 1, a.brk);
    givens_done = true;
    update(a, P, sw, hf);  // w -= V h2
  } else {
    update(a, P, sw, hf);
    warp_norm(P, sw, wp, ldw, 0);
    block_partial(arn_part(a, 2), wp, ldw, 1);
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce(arn_part(a, 2), 1, wp, hf, 0);  // ||w||^2 to wp[0]
    const float2 hn2 = re_of(wp[0]);
    if (threadIdx.x == 0) set_inv(hn2);
    if (blockIdx.x == 0) store_column(hn2);
    __syncthreads();
  }
  {
    const float2 s = s_inv;
#pragma unroll 1
    for (int e = 0; e < ppt; ++e) {
      const long long p = P.t0 + (long long)e * AT;
      if (p < P.pend) {
        const float4 w = sw[e * AT + threadIdx.x];
        float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
        ff_acc_mul(re, re_of(w), s);
        ff_acc_mul(im, im_of(w), s);
        re = ff_norm(re);
        im = ff_norm(im);
        a.vnext[p] = make_float4(re.x, re.y, im.x, im.y);
        a.y32[p] = make_float2(re.x, im.x);
      }
    }
  }
  if (blockIdx.x == 0 && !givens_done && threadIdx.x < 32)
    givens_column_warp(a.gs, 0, nb - 1, a.brk);
}

constexpr int ARN_PPT_MAX = 16;

size_t arn_smem(int nb, int ppt) {
  return sizeof(float4) * ((size_t)ppt * AT + (size_t)AWARPS * (nb + 8) + 3 * (size_t)(nb + 1));
}

}  // namespace

cudaError_t arnoldi_ff_plan(long long n, int mmax, int* ppt, int* blocks) {
  *ppt = 0;
  *blocks = 0;
  if (n < 1 || n > 0x7fffffffLL || mmax < 1 || mmax > 128) return cudaSuccess;
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) return e;
  // the grid: one block on every SM (fewer where n is small), each a contiguous range of
  // about n / G points; more blocks make every barrier and all-blocks sum longer (measured at
  // 64^3: 152 blocks of 512 threads 0.9% faster per solve than 304 of 256)
  const long long g = std::min<long long>((long long)sms, (n + AT - 1) / AT);
  const int p = (int)(((n + g - 1) / g + AT - 1) / AT);
  if (p > ARN_PPT_MAX) return cudaSuccess;  // the multi-kernel form serves
  const size_t smem = arn_smem(mmax + 1, p);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_arnoldi_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi_ff, AT, smem);
  if (e != cudaSuccess) return e;
  if ((long long)per_sm * sms < g) return cudaSuccess;
  *ppt = p;
  *blocks = (int)g;
  return cudaSuccess;
}

cudaError_t launch_arnoldi_ff(const Geom& g, const double2* dg, const double2* z,
                              const float4* V, float4* vnext, float2* y32, const GmresDev& gs,
                              double2* partial, unsigned* bar, int* err, long long n, int nb,
                              double brk, int pyth, int ppt, int blocks, cudaStream_t st) {
  if (nb < 1 || nb > gs.mmax || blocks < 1 || ppt < 1 || ppt > ARN_PPT_MAX ||
      (long long)blocks * ppt * AT < n || n > 0x7fffffffLL)
    return cudaErrorInvalidValue;
  Arn a;
  a.g = g;
  a.dg = dg;
  a.z = z;
  a.V = V;
  a.vnext = vnext;
  a.y32 = y32;
  a.gs = gs;
  a.part = reinterpret_cast<float4*>(partial);
  a.bar = bar;
  a.err = err;
  a.n = n;
  a.nb = nb;
  a.pyth = pyth;
  a.brk = brk;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(AT);
  cfg.dynamicSmemBytes = arn_smem(nb, ppt);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_arnoldi_ff, a, ppt);
}

}  // namespace hz
