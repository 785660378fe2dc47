// Float-pair kernels of the outer FGMRES Arnoldi for the HZ_MIXED_C64_FF form.
//
// GB300 delivers 627.6 G float64 FMA/s against 36.7 T float32 FMA/s, so the float64 CGS2 of the
// outer Arnoldi (4 FMA per element per basis field per pass) is bound by the float64 pipe.
// This form keeps the outer basis V, and the vector being orthogonalised, as float pairs
// (hi + lo, about 48 significant bits): a complex element is a float4 (re.hi, re.lo, im.hi,
// im.lo), 16 bytes like a double2.  Products are error-free float32 transformations (FMA),
// sums are two-sum chains, so the CGS2 passes run on the float32 pipes.  Dots are accumulated
// across warps and blocks as float pairs too and converted to float64 once per value; the
// Hessenberg/Givens least squares stays float64, as in the float64 form.
#include <cuda_runtime.h>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int F_WARPS = 8;  // block: 8 warps x 32 lanes x 2 points
constexpr int F_PPL = 2;
constexpr int F_CHUNK = F_WARPS * 32 * F_PPL;

// Classical Gram-Schmidt pieces on float-pair fields, modes as in the float64 k_cgs:
//   0: h1 = V^H w and ||w||^2;  1: w -= V h1, then h2 = V^H w;  2: w -= V h2, ||w||^2 and the
//   Givens step of the column.  Lane l of warp w owns the F_PPL points seg + l + 32 e.  Basis
//   fields are taken 8 at a time with every load of the group issued before its arithmetic, so
//   a warp keeps 8 * F_PPL 16-byte loads in flight (the kernels are bound by memory latency,
//   not by the float32 pipes).
template <int MODE>
__global__ void __launch_bounds__(F_WARPS * 32)
k_cgs_ff(const float4* __restrict__ V, long long vis, long long vrs, int nb, float4* w,
         long long wrs, long long n, GmresDev gs, double2* partial, unsigned* counters,
         double brk) {
  pdl_enter();
  extern __shared__ float4 sm4[];  // wp[F_WARPS][nb + 8] | hs[nb] (float-pair complex each)
  const int r = blockIdx.y;
  if (gs.stopped[r]) return;
  const int M = gs.mmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldw = nb + 8;
  const long long seg = (long long)blockIdx.x * F_CHUNK + (long long)warp * 32 * F_PPL + lane;
  float4* wr = w + r * wrs;
  const float4* Vr = V + r * vrs;
  float4* wp = sm4;
  float4* hs = sm4 + F_WARPS * ldw;
  if (MODE != 0) {
    // the coefficients, negated, as float pairs (float64 conversions once per block)
    const double2* hp = (MODE == 1 ? gs.h1 : gs.h2) + (long long)r * (M + 2);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const float2 a = ff_from_d(-hp[b].x), c = ff_from_d(-hp[b].y);
      hs[b] = make_float4(a.x, a.y, c.x, c.y);
    }
    __syncthreads();
  }
  float2 wre[F_PPL], wim[F_PPL];
#pragma unroll
  for (int e = 0; e < F_PPL; ++e) {
    const long long p = seg + 32LL * e;
    const float4 v = p < n ? wr[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    wre[e] = re_of(v);
    wim[e] = im_of(v);
  }
  if (MODE != 0) {
    for (int b0 = 0; b0 < nb; b0 += 8) {
      float4 vv[8][F_PPL];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int e = 0; e < F_PPL; ++e) {
          const long long p = seg + 32LL * e;
          vv[t][e] = (b0 + t < nb && p < n) ? Vr[(b0 + t) * vis + p]
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          const float4 nh = hs[b0 + t];
          const float2 nre = re_of(nh), nim = im_of(nh), mnim = neg(nim);
#pragma unroll
          for (int e = 0; e < F_PPL; ++e) {
            const float2 vre = re_of(vv[t][e]), vim = im_of(vv[t][e]);
            // w += v * (-h)
            ff_acc_mul(wre[e], vre, nre);
            ff_acc_mul(wre[e], vim, mnim);
            ff_acc_mul(wim[e], vre, nim);
            ff_acc_mul(wim[e], vim, nre);
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < F_PPL; ++e) {
      const long long p = seg + 32LL * e;
      wre[e] = ff_norm(wre[e]);
      wim[e] = ff_norm(wim[e]);
      if (p < n) wr[p] = make_float4(wre[e].x, wre[e].y, wim[e].x, wim[e].y);
    }
  }
  if (MODE != 2) {
    for (int b0 = 0; b0 < nb; b0 += 8) {
      float4 vv[8][F_PPL];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int e = 0; e < F_PPL; ++e) {
          const long long p = seg + 32LL * e;
          vv[t][e] = (b0 + t < nb && p < n) ? Vr[(b0 + t) * vis + p]
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      float4 acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          float2 are = make_float2(0.f, 0.f), aim = make_float2(0.f, 0.f);
#pragma unroll
          for (int e = 0; e < F_PPL; ++e) {
            const float2 vre = re_of(vv[t][e]), vim = im_of(vv[t][e]);
            // conj(v) * w
            ff_acc_mul(are, vre, wre[e]);
            ff_acc_mul(are, vim, wim[e]);
            ff_acc_mul(aim, vre, wim[e]);
            ff_acc_mul(aim, neg(vim), wre[e]);
          }
          are = ff_norm(are);
          aim = ff_norm(aim);
          acc[t] = make_float4(are.x, are.y, aim.x, aim.y);
        }
      }
      const float4 red = warp_reduce8_ff(acc, lane);
      if ((lane & 3) == 0) {
        const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (b0 + t < nb) wp[warp * ldw + b0 + t] = red;  // slot nb is the norm's (mode 0)
      }
    }
  }
  if (MODE != 1) {
    float2 q = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < F_PPL; ++e) {
      ff_acc_mul(q, wre[e], wre[e]);
      ff_acc_mul(q, wim[e], wim[e]);
    }
    q = ff_norm(q);
    for (int o = 16; o > 0; o >>= 1)
      q = ff_add(q, make_float2(__shfl_xor_sync(0xffffffffu, q.x, o),
                                __shfl_xor_sync(0xffffffffu, q.y, o)));
    if (lane == 0) wp[warp * ldw + (MODE == 0 ? nb : 0)] = make_float4(q.x, q.y, 0.f, 0.f);
  }
  __syncthreads();
  const int nslots = MODE == 0 ? nb + 1 : (MODE == 1 ? nb : 1);
  float4* part = reinterpret_cast<float4*>(partial) + (long long)r * (M + 2) * gridDim.x;
  for (int sidx = threadIdx.x; sidx < nslots; sidx += blockDim.x) {
    float4 a = wp[sidx];
    for (int ww = 1; ww < F_WARPS; ++ww) a = ffc_add(a, wp[ww * ldw + sidx]);
    part[(long long)sidx * gridDim.x + blockIdx.x] = a;
  }
  if (!last_block(counters + r)) return;
  double2* out = MODE == 0 ? gs.h1 + (long long)r * (M + 2)
               : MODE == 1 ? gs.h2 + (long long)r * (M + 2) : gs.nrm + 2 * r;
  for (int sidx = warp; sidx < nslots; sidx += F_WARPS) {
    const float4 t = warp_sum_partials_ff(part, sidx, (int)gridDim.x, lane);
    if (lane == 0) out[sidx] = d_from_ffc(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) counters[r] = 0;
  if (MODE == 2) givens_column(gs, r, nb - 1, brk);  // whole block; float64 least squares
}

// v = w * (1 / h_{k+1,k}) in place on float pairs; the float64 scale is split once per block.
// y32 (may be null): also the complex64 rounding of the result, the next FCI application's input.
__global__ void k_scale_ff(float4* v, long long vrs, long long n, GmresDev gs, float2* y32,
                           long long yrs) {
  pdl_enter();
  __shared__ float2 s_ff;
  const int r = blockIdx.y;
  if (threadIdx.x == 0) s_ff = ff_from_d(gs.scal[(long long)r * SC_COUNT + SC_INV]);
  __syncthreads();
  const float2 s = s_ff;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float4 x = v[r * vrs + p];
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    ff_acc_mul(a, re_of(x), s);
    ff_acc_mul(b, im_of(x), s);
    a = ff_norm(a);
    b = ff_norm(b);
    v[r * vrs + p] = make_float4(a.x, a.y, b.x, b.y);
    if (y32) y32[r * yrs + p] = make_float2(a.x, b.x);
  }
}

// v0 = r / beta from the float64 residual, written as float pairs over the same storage
// (each element is read and rewritten by one thread).
__global__ void k_scale_ff_from64(float4* dst, long long drs, const double2* src, long long srs,
                                  long long n, GmresDev gs, float2* y32, long long yrs) {
  pdl_enter();
  const int r = blockIdx.y;
  const double s = gs.scal[(long long)r * SC_COUNT + SC_INV];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 x = src[r * srs + p];
    const float2 a = ff_from_d(x.x * s), b = ff_from_d(x.y * s);
    dst[r * drs + p] = make_float4(a.x, a.y, b.x, b.y);
    if (y32) y32[r * yrs + p] = make_float2(a.x, b.x);
  }
}

inline unsigned ff_ew_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return unsigned(b < 4096 ? b : 4096);
}

}  // namespace

cudaError_t launch_cgs_ff(int mode, const float4* V, long long vis, long long vrs, int nb,
                          Buf<float4> w, long long n, const GmresDev& gs, double2* partial,
                          unsigned* counters, int nvec, double breakdown, cudaStream_t st) {
  dim3 grd(unsigned((n + F_CHUNK - 1) / F_CHUNK), nvec);
  const size_t smem = sizeof(float4) * ((size_t)F_WARPS * (nb + 8) + (size_t)nb);
  count_launch();
  if (mode == 0)
    return launch_pdl(k_cgs_ff<0>, grd, F_WARPS * 32, smem, st, V, vis, vrs, nb, w.p, w.rs, n, gs,
                      partial, counters, breakdown);
  if (mode == 1)
    return launch_pdl(k_cgs_ff<1>, grd, F_WARPS * 32, smem, st, V, vis, vrs, nb, w.p, w.rs, n, gs,
                      partial, counters, breakdown);
  return launch_pdl(k_cgs_ff<2>, grd, F_WARPS * 32, smem, st, V, vis, vrs, nb, w.p, w.rs, n, gs, partial,
                    counters, breakdown);
}

cudaError_t launch_scale_ff(Buf<float4> v, long long n, const GmresDev& gs, int nvec,
                            cudaStream_t st, Buf<float2> y32) {
  count_launch();
  return launch_pdl(k_scale_ff, dim3(ff_ew_blocks(n), nvec), 256, 0, st, v.p, v.rs, n, gs, y32.p,
                    y32.rs);
}

cudaError_t launch_scale_ff_from64(Buf<float4> dst, Buf<const double2> src, long long n,
                                   const GmresDev& gs, int nvec, cudaStream_t st,
                                   Buf<float2> y32) {
  count_launch();
  return launch_pdl(k_scale_ff_from64, dim3(ff_ew_blocks(n), nvec), 256, 0, st, dst.p, dst.rs,
                    src.p, src.rs, n, gs, y32.p, y32.rs);
}


}  // namespace hz
