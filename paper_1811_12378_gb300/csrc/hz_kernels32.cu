// Complex64 kernels of the FCI internals for the HZ_MIXED_C64_FCI32 form: the step size d
// (Algorithm 1 step 3) and the inner GMRES (steps 4-5) run on float2 fields, with float32
// products, float64 partial sums across warps and blocks, and the float64 Hessenberg/Givens
// state of GmresDev.  The outer FGMRES that consumes FCI's output stays float64.
//
// On GB300 the float64 pipe delivers 1/58 of the float32 rate, so these kernels avoid every
// float64 instruction that is not a cross-warp accumulation: coefficients are converted to
// float32 once per block into shared memory.
#include <cuda_runtime.h>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int C_WARPS = 8;  // block: 8 warps x 32 lanes x 4 points
constexpr int C_PPL = 4;
constexpr int C_CHUNK = C_WARPS * 32 * C_PPL;

// Butterfly reduction of 8 per-lane float2 partials over a warp (same lane map as the float64
// version in hz_kernels.cu): lane l with (l & 3) == 0 ends with the sum of vector
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

// Classical Gram-Schmidt pieces on float2 fields (modes as in launch_cgs).
template <int MODE>
__global__ void __launch_bounds__(C_WARPS * 32)
k_cgs32(const float2* __restrict__ V, long long vis, long long vrs, int nb, float2* w,
        long long wrs, long long n, GmresDev gs, double2* partial, unsigned* counters, double brk) {
  extern __shared__ double2 sm[];  // wp[C_WARPS][nb + 8] (double2) | hs[nb] (float2)
  const int r = blockIdx.y;
  if (gs.stopped[r]) return;
  const int M = gs.mmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldw = nb + 8;
  const long long seg = (long long)blockIdx.x * C_CHUNK + (long long)warp * 32 * C_PPL + lane;
  float2* wr = w + r * wrs;
  const float2* Vr = V + r * vrs;
  double2* wp = sm;
  float2* hs = reinterpret_cast<float2*>(sm + C_WARPS * ldw);
  if (MODE != 0) {
    const double2* hp = (MODE == 1 ? gs.h1 : gs.h2) + (long long)r * (M + 2);
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      hs[b] = make_float2(float(hp[b].x), float(hp[b].y));
    __syncthreads();
  }
  float2 wv[C_PPL];
#pragma unroll
  for (int e = 0; e < C_PPL; ++e) {
    const long long p = seg + 32LL * e;
    wv[e] = p < n ? wr[p] : make_float2(0.f, 0.f);
  }
  if (MODE != 0) {
    for (int b = 0; b < nb; ++b) {
      const float2 h = hs[b];
      const float2* vb = Vr + b * vis;
#pragma unroll
      for (int e = 0; e < C_PPL; ++e) {
        const long long p = seg + 32LL * e;
        if (p < n) {
          const float2 v = vb[p];
          wv[e].x = fmaf(-h.x, v.x, fmaf(h.y, v.y, wv[e].x));
          wv[e].y = fmaf(-h.x, v.y, fmaf(-h.y, v.x, wv[e].y));
        }
      }
    }
#pragma unroll
    for (int e = 0; e < C_PPL; ++e) {
      const long long p = seg + 32LL * e;
      if (p < n) wr[p] = wv[e];
    }
  }
  if (MODE != 2) {
    for (int b0 = 0; b0 < nb; b0 += 8) {
      float2 acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          const float2* vb = Vr + (b0 + t) * vis;
#pragma unroll
          for (int e = 0; e < C_PPL; ++e) {
            const long long p = seg + 32LL * e;
            if (p < n) {
              const float2 v = vb[p];
              acc[t].x = fmaf(v.x, wv[e].x, fmaf(v.y, wv[e].y, acc[t].x));
              acc[t].y = fmaf(v.x, wv[e].y, fmaf(-v.y, wv[e].x, acc[t].y));
            }
          }
        }
      }
      const float2 red = warp_reduce8f(acc, lane);
      if ((lane & 3) == 0) {
        const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        wp[warp * ldw + b0 + t] = make_double2(double(red.x), double(red.y));
      }
    }
  }
  if (MODE != 1) {
    float q = 0.f;
#pragma unroll
    for (int e = 0; e < C_PPL; ++e) q = fmaf(wv[e].x, wv[e].x, fmaf(wv[e].y, wv[e].y, q));
    q = warp_sum(q);
    if (lane == 0) wp[warp * ldw + (MODE == 0 ? nb : 0)] = make_double2(double(q), 0.0);
  }
  __syncthreads();
  const int nslots = MODE == 0 ? nb + 1 : (MODE == 1 ? nb : 1);
  double2* part = partial + (long long)r * (M + 2) * gridDim.x;
  for (int sidx = threadIdx.x; sidx < nslots; sidx += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int ww = 0; ww < C_WARPS; ++ww) acc = cadd(acc, wp[ww * ldw + sidx]);
    part[(long long)sidx * gridDim.x + blockIdx.x] = acc;
  }
  if (!last_block(counters + r)) return;
  double2* out = MODE == 0 ? gs.h1 + (long long)r * (M + 2)
               : MODE == 1 ? gs.h2 + (long long)r * (M + 2) : gs.nrm + 2 * r;
  for (int sidx = warp; sidx < nslots; sidx += C_WARPS) {
    double ax = 0.0, ay = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double2 v = __ldcg(part + (long long)sidx * gridDim.x + b);
      ax += v.x;
      ay += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_down_sync(0xffffffffu, ax, o);
      ay += __shfl_down_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) out[sidx] = make_double2(ax, ay);
  }
  __syncthreads();
  if (threadIdx.x == 0) counters[r] = 0;
  if (MODE == 2) givens_column(gs, r, nb - 1, brk);  // whole block
}

__global__ void k_scale32(float2* __restrict__ dst, long long drs, const float2* __restrict__ src,
                          long long srs, long long n, GmresDev gs) {
  const int r = blockIdx.y;
  const float s = float(gs.scal[(long long)r * SC_COUNT + SC_INV]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float2 v = src[r * srs + p];
    dst[r * drs + p] = make_float2(v.x * s, v.y * s);
  }
}

// d = <Aw, r> / <Aw, Aw> with float32 products and float64 accumulation across warps/blocks.
__global__ void __launch_bounds__(C_WARPS * 32)
k_fci_dots32(const float2* __restrict__ Aw, long long ars, const float2* __restrict__ rv,
             long long rrs, long long n, GmresDev gs, double2* partial, unsigned* counters) {
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long seg = (long long)blockIdx.x * C_CHUNK + (long long)warp * 32 * C_PPL + lane;
  float nx = 0.f, ny = 0.f, dd = 0.f;
#pragma unroll
  for (int e = 0; e < C_PPL; ++e) {
    const long long p = seg + 32LL * e;
    if (p < n) {
      const float2 a = Aw[r * ars + p], b = rv[r * rrs + p];
      nx = fmaf(a.x, b.x, fmaf(a.y, b.y, nx));
      ny = fmaf(a.x, b.y, fmaf(-a.y, b.x, ny));
      dd = fmaf(a.x, a.x, fmaf(a.y, a.y, dd));
    }
  }
  nx = warp_sum(nx);
  ny = warp_sum(ny);
  dd = warp_sum(dd);
  __shared__ double2 wn[C_WARPS], wd[C_WARPS];
  if (lane == 0) {
    wn[warp] = make_double2(double(nx), double(ny));
    wd[warp] = make_double2(double(dd), 0.0);
  }
  __syncthreads();
  double2* part = partial + (long long)r * (gs.mmax + 2) * gridDim.x;
  if (threadIdx.x == 0) {
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    for (int ww = 0; ww < C_WARPS; ++ww) {
      a = cadd(a, wn[ww]);
      b = cadd(b, wd[ww]);
    }
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
  }
  if (!last_block(counters + r)) return;
  __shared__ double2 tot[2];
  finish_slots(part, 2, tot, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    double* sc = gs.scal + (long long)r * SC_COUNT;
    const double den = tot[1].x;
    sc[SC_DR] = den != 0.0 ? tot[0].x / den : 0.0;
    sc[SC_DI] = den != 0.0 ? tot[0].y / den : 0.0;
  }
}

// v0 = r - d Aw on float2 fields, ||v0||^2 -> inner cycle start.
__global__ void __launch_bounds__(C_WARPS * 32)
k_fci_start32(const float2* __restrict__ Aw, long long ars, const float2* __restrict__ rv,
              long long rrs, float2* __restrict__ v0, long long vrs, long long n, GmresDev gs,
              double2* partial, unsigned* counters) {
  __shared__ double2 sh[32];
  __shared__ float2 dsh;
  const int r = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    const double* sc = gs.scal + (long long)r * SC_COUNT;
    dsh = make_float2(float(sc[SC_DR]), float(sc[SC_DI]));
  }
  __syncthreads();
  const float2 d = dsh;
  const long long seg = (long long)blockIdx.x * C_CHUNK + (long long)warp * 32 * C_PPL + lane;
  float q = 0.f;
#pragma unroll
  for (int e = 0; e < C_PPL; ++e) {
    const long long p = seg + 32LL * e;
    if (p < n) {
      const float2 a = Aw[r * ars + p], b = rv[r * rrs + p];
      const float2 v = make_float2(b.x - (d.x * a.x - d.y * a.y), b.y - (d.x * a.y + d.y * a.x));
      v0[r * vrs + p] = v;
      q = fmaf(v.x, v.x, fmaf(v.y, v.y, q));
    }
  }
  q = warp_sum(q);
  __shared__ double wq[C_WARPS];
  if (lane == 0) wq[warp] = double(q);
  __syncthreads();
  double2* part = partial + (long long)r * (gs.mmax + 2) * gridDim.x;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int ww = 0; ww < C_WARPS; ++ww) s += wq[ww];
    part[blockIdx.x] = make_double2(s, 0.0);
  }
  if (!last_block(counters + r)) return;
  __shared__ double2 tot;
  finish_slots(part, 1, &tot, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    double* sc = gs.scal + (long long)r * SC_COUNT;
    const double beta = sqrt(tot.x);
    sc[SC_RES2] = tot.x;
    sc[SC_BETA] = beta;
    sc[SC_INV] = beta > 0.0 ? 1.0 / beta : 0.0;
    gs.g[(long long)r * (gs.mmax + 1)] = make_double2(beta, 0.0);
    gs.kend[r] = 0;
    gs.stopped[r] = beta > 0.0 ? 0 : 1;
  }
}

// out = double(sum_{i<kend} y_i B_i) + d * E: the inner correction summed in float32, the
// float64 quadrature sum E added in float64 (Algorithm 1 step 5, v + d w).
__global__ void k_combine_fci32(double2* __restrict__ out, long long ors,
                                const float2* __restrict__ B, long long bis, long long brs,
                                GmresDev gs, const double2* __restrict__ E, long long ers,
                                long long n) {
  __shared__ float2 ys[128];
  __shared__ double2 dsh;
  const int r = blockIdx.y;
  const int kk = gs.kend[r];
  if (threadIdx.x < kk) {
    const double2 yv = gs.y[(long long)r * gs.mmax + threadIdx.x];
    ys[threadIdx.x] = make_float2(float(yv.x), float(yv.y));
  }
  if (threadIdx.x == 0) {
    const double* sc = gs.scal + (long long)r * SC_COUNT;
    dsh = make_double2(sc[SC_DR], sc[SC_DI]);
  }
  __syncthreads();
  const double2 d = dsh;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    for (int b = 0; b < kk; ++b) v = cadd(v, cmul(ys[b], B[r * brs + b * bis + p]));
    const double2 e = E[r * ers + p];
    out[r * ors + p] = make_double2(double(v.x) + (d.x * e.x - d.y * e.y),
                                    double(v.y) + (d.x * e.y + d.y * e.x));
  }
}

inline unsigned blocks32(long long n) { return unsigned((n + C_CHUNK - 1) / C_CHUNK); }
inline unsigned ew_blocks32(long long n) {
  long long b = (n + 255) / 256;
  return unsigned(b < 4096 ? b : 4096);
}

}  // namespace

cudaError_t launch_cgs32(int mode, const float2* V, long long vis, long long vrs, int nb,
                         Buf<float2> w, long long n, const GmresDev& gs, double2* partial,
                         unsigned* counters, int nvec, double breakdown, cudaStream_t st) {
  dim3 grd(blocks32(n), nvec);
  const size_t smem = sizeof(double2) * (size_t)C_WARPS * (nb + 8) + sizeof(float2) * (size_t)nb;
  count_launch();
  if (mode == 0)
    k_cgs32<0><<<grd, C_WARPS * 32, smem, st>>>(V, vis, vrs, nb, w.p, w.rs, n, gs, partial,
                                                counters, breakdown);
  else if (mode == 1)
    k_cgs32<1><<<grd, C_WARPS * 32, smem, st>>>(V, vis, vrs, nb, w.p, w.rs, n, gs, partial,
                                                counters, breakdown);
  else
    k_cgs32<2><<<grd, C_WARPS * 32, smem, st>>>(V, vis, vrs, nb, w.p, w.rs, n, gs, partial,
                                                counters, breakdown);
  return cudaGetLastError();
}

cudaError_t launch_scale32(Buf<float2> dst, Buf<const float2> src, long long n, const GmresDev& gs,
                           int nvec, cudaStream_t st) {
  count_launch();
  k_scale32<<<dim3(ew_blocks32(n), nvec), 256, 0, st>>>(dst.p, dst.rs, src.p, src.rs, n, gs);
  return cudaGetLastError();
}

cudaError_t launch_fci_step32(Buf<const float2> Aw, Buf<const float2> r, Buf<float2> v0,
                              const GmresDev& gs, double2* partial, unsigned* counters,
                              long long n, int nvec, cudaStream_t st) {
  dim3 grd(blocks32(n), nvec);
  count_launch();
  k_fci_dots32<<<grd, C_WARPS * 32, 0, st>>>(Aw.p, Aw.rs, r.p, r.rs, n, gs, partial, counters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  k_fci_start32<<<grd, C_WARPS * 32, 0, st>>>(Aw.p, Aw.rs, r.p, r.rs, v0.p, v0.rs, n, gs, partial,
                                               counters);
  return cudaGetLastError();
}

cudaError_t launch_combine_fci32(Buf<double2> out, const float2* B, long long bis, long long brs,
                                 const GmresDev& gs, Buf<const double2> E, long long n, int nvec,
                                 cudaStream_t st) {
  if (gs.mmax > 128) return cudaErrorInvalidValue;
  count_launch();
  k_combine_fci32<<<dim3(ew_blocks32(n), nvec), 256, 0, st>>>(out.p, out.rs, B, bis, brs, gs, E.p,
                                                              E.rs, n);
  return cudaGetLastError();
}

}  // namespace hz
