// Complex64 kernels of the FCI internals for the HZ_MIXED_C64_FCI32 form: the step size d
// (Algorithm 1 step 3) and the inner GMRES (steps 4-5) run on float2 fields with float32
// products, float-pair (about 48-bit) sums across warps and blocks, and float32 scalar work
// (d, beta, the Givens step, the triangular solve); GmresDev keeps its float64 storage, filled
// by a few lane-parallel conversions.  The outer FGMRES that consumes FCI's output is not here.
//
// On GB300 a float64 instruction issues at 1/64 of the float32 rate per SM partition, so a
// serial float64 chain (a square root, a division, a Givens rotation in one thread) costs
// microseconds; these kernels keep float64 instructions off their critical paths.
#include <cuda_runtime.h>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int C_WARPS = 8;  // block: 8 warps x 32 lanes x 2 points
constexpr int C_PPL = 2;
constexpr int C_CHUNK = C_WARPS * 32 * C_PPL;

// Givens step for column k of rhs r in float32, by one warp: lanes stage the column
// h1 + h2 and the previous rotations (float64 storage, converted in parallel), lane 0 applies
// the rotations and forms the new one, lanes write the results back.  hn2 = ||w||^2 after the
// second pass.  Same steps as givens_column (Saad's GMRES with complex rotations).
__device__ void givens_column32(const GmresDev& gs, int r, int k, float hn2, float brk) {
  __shared__ float2 sR[kGivMax];
  __shared__ float scc[kGivMax];
  __shared__ float2 sss[kGivMax];
  __shared__ float2 out6[3];  // (c, 0), s, g[k+1]
  __shared__ float2 gk_new;
  __shared__ float est_s, hn_s, inv_s;
  __shared__ int stop_s;
  const int lane = threadIdx.x & 31;
  const int M = gs.mmax;
  const double2* h1 = gs.h1 + (long long)r * (M + 2);
  const double2* h2 = gs.h2 + (long long)r * (M + 2);
  const double* cc = gs.cc + (long long)r * M;
  const double2* ss = gs.ss + (long long)r * M;
  double2* gg = gs.g + (long long)r * (M + 1);
  for (int i = lane; i <= k; i += 32) {
    sR[i] = make_float2(float(h1[i].x + h2[i].x), float(h1[i].y + h2[i].y));
    if (i < k) {
      scc[i] = float(cc[i]);
      sss[i] = make_float2(float(ss[i].x), float(ss[i].y));
    }
  }
  float wn2 = 0.f;
  float2 gk = make_float2(0.f, 0.f);
  if (lane == 0) {
    wn2 = float(h1[k + 1].x);
    gk = make_float2(float(gg[k].x), float(gg[k].y));
  }
  __syncwarp();
  if (lane == 0) {
    const float hn = sqrtf(hn2), wn = sqrtf(wn2);
    for (int i = 0; i < k; ++i) {
      const float c = scc[i];
      const float2 s = sss[i], a = sR[i], b = sR[i + 1];
      sR[i] = make_float2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
      sR[i + 1] = make_float2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    float c;
    float2 s;
    const float2 a = sR[k];
    if (hn == 0.f) {
      c = 1.f;
      s = make_float2(0.f, 0.f);
    } else if (a.x == 0.f && a.y == 0.f) {
      c = 0.f;
      s = make_float2(1.f, 0.f);
    } else {
      const float ra = hypotf(a.x, a.y);
      const float rr = hypotf(ra, hn);
      c = ra / rr;
      s = make_float2(a.x / ra * hn / rr, a.y / ra * hn / rr);
    }
    sR[k] = make_float2(c * a.x + s.x * hn, c * a.y + s.y * hn);
    gk_new = make_float2(c * gk.x, c * gk.y);
    const float2 gk1 = make_float2(-(s.x * gk.x + s.y * gk.y), -(s.x * gk.y - s.y * gk.x));
    out6[0] = make_float2(c, 0.f);
    out6[1] = s;
    out6[2] = gk1;
    const bool brk_now = hn <= brk * wn;
    est_s = hypotf(gk1.x, gk1.y);
    hn_s = hn;
    inv_s = brk_now ? 0.f : 1.f / hn;
    stop_s = brk_now ? 1 : 0;
  }
  __syncwarp();
  double2* R = gs.R + (long long)r * (M + 1) * M + (long long)k * (M + 1);
  for (int i = lane; i <= k + 1; i += 32)
    R[i] = i <= k ? make_double2(double(sR[i].x), double(sR[i].y)) : make_double2(0.0, 0.0);
  double* sc = gs.scal + (long long)r * SC_COUNT;
  if (lane == 1) gs.cc[(long long)r * M + k] = double(out6[0].x);
  if (lane == 2) gs.ss[(long long)r * M + k] = make_double2(double(out6[1].x), double(out6[1].y));
  if (lane == 3) gg[k] = make_double2(double(gk_new.x), double(gk_new.y));
  if (lane == 4) gg[k + 1] = make_double2(double(out6[2].x), double(out6[2].y));
  if (lane == 5) sc[SC_EST] = double(est_s);
  if (lane == 6) sc[SC_HN] = double(hn_s);
  if (lane == 7) sc[SC_INV] = double(inv_s);
  if (lane == 8) {
    gs.kend[r] = k + 1;
    if (stop_s || double(est_s) <= sc[SC_TOL]) gs.stopped[r] = 1;
  }
}

// Classical Gram-Schmidt pieces on float2 fields (modes as in launch_cgs).  Basis fields are
// taken 8 at a time with every load of the group issued before its arithmetic: the kernel is
// bound by memory latency, so a warp keeps 8 * C_PPL loads in flight.
template <int MODE>
__global__ void __launch_bounds__(C_WARPS * 32)
k_cgs32(const float2* __restrict__ V, long long vis, long long vrs, int nb, float2* w,
        long long wrs, long long n, GmresDev gs, double2* partial, unsigned* counters, double brk) {
  pdl_enter();
  extern __shared__ double2 sm[];  // wp[C_WARPS][nb + 8] | hs[nb] (float2 each)
  const int r = blockIdx.y;
  if (gs.stopped[r]) return;
  const int M = gs.mmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldw = nb + 8;
  const long long seg = (long long)blockIdx.x * C_CHUNK + (long long)warp * 32 * C_PPL + lane;
  float2* wr = w + r * wrs;
  const float2* Vr = V + r * vrs;
  float2* wp = reinterpret_cast<float2*>(sm);
  float2* hs = wp + C_WARPS * ldw;
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
    for (int b0 = 0; b0 < nb; b0 += 8) {
      float2 vv[8][C_PPL];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int e = 0; e < C_PPL; ++e) {
          const long long p = seg + 32LL * e;
          vv[t][e] = (b0 + t < nb && p < n) ? Vr[(b0 + t) * vis + p] : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          const float2 h = hs[b0 + t];
#pragma unroll
          for (int e = 0; e < C_PPL; ++e) {
            const float2 v = vv[t][e];
            wv[e].x = fmaf(-h.x, v.x, fmaf(h.y, v.y, wv[e].x));
            wv[e].y = fmaf(-h.x, v.y, fmaf(-h.y, v.x, wv[e].y));
          }
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
      float2 vv[8][C_PPL];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int e = 0; e < C_PPL; ++e) {
          const long long p = seg + 32LL * e;
          vv[t][e] = (b0 + t < nb && p < n) ? Vr[(b0 + t) * vis + p] : make_float2(0.f, 0.f);
        }
      float2 acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
#pragma unroll
        for (int e = 0; e < C_PPL; ++e) {
          const float2 v = vv[t][e];
          acc[t].x = fmaf(v.x, wv[e].x, fmaf(v.y, wv[e].y, acc[t].x));
          acc[t].y = fmaf(v.x, wv[e].y, fmaf(-v.y, wv[e].x, acc[t].y));
        }
      }
      const float2 red = warp_reduce8f(acc, lane);
      if ((lane & 3) == 0) {
        const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (b0 + t < nb) wp[warp * ldw + b0 + t] = red;  // slot nb is the norm's (mode 0)
      }
    }
  }
  if (MODE != 1) {
    float q = 0.f;
#pragma unroll
    for (int e = 0; e < C_PPL; ++e) q = fmaf(wv[e].x, wv[e].x, fmaf(wv[e].y, wv[e].y, q));
    q = warp_sum(q);
    if (lane == 0) wp[warp * ldw + (MODE == 0 ? nb : 0)] = make_float2(q, 0.f);
  }
  __syncthreads();
  const int nslots = MODE == 0 ? nb + 1 : (MODE == 1 ? nb : 1);
  float4* part = reinterpret_cast<float4*>(partial) + (long long)r * (M + 2) * gridDim.x;
  for (int sidx = threadIdx.x; sidx < nslots; sidx += blockDim.x) {
    float4 acc = ffc_of(wp[sidx]);
    for (int ww = 1; ww < C_WARPS; ++ww) acc = ffc_add(acc, ffc_of(wp[ww * ldw + sidx]));
    part[(long long)sidx * gridDim.x + blockIdx.x] = acc;
  }
  if (!last_block(counters + r)) return;
  double2* out = MODE == 0 ? gs.h1 + (long long)r * (M + 2)
               : MODE == 1 ? gs.h2 + (long long)r * (M + 2) : gs.nrm + 2 * r;
  __shared__ float2 tot2;
  for (int sidx = warp; sidx < nslots; sidx += C_WARPS) {
    const float4 t = warp_sum_partials_ff(part, sidx, (int)gridDim.x, lane);
    if (lane == 0) {
      out[sidx] = d_from_ffc(t);
      if (MODE == 2) tot2 = f_from_ffc(t);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) counters[r] = 0;
  if (MODE == 2 && warp == 0) givens_column32(gs, r, nb - 1, tot2.x, float(brk));
}

// Ticket of the last of G blocks of this rhs (grids of any shape); true in every thread of it.
__device__ __forceinline__ bool last_of(unsigned* counter, unsigned G) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) is_last = (atomicAdd(counter, 1u) == G - 1);
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// The complex64 stencil y = A x fused with the reduction that consumes it (saves a launch and a
// re-read of y), block (32, rows), z-columns of ZC points:
//   KIND 0 (first CGS pass of an inner Arnoldi step): h1 = V^H y over nb basis fields and
//          ||y||^2 into slot nb, as k_cgs32<0>;
//   KIND 1 (Algorithm 1 step 3): d = (Aw)^H r / ||Aw||^2 with V = r (one field), as
//          k_fci_dots32.
// Float32 products, float-pair sums across warps and blocks.
template <int ZC, int KIND>
__global__ void __launch_bounds__(128)
k_stencil32_dots(Geom g, const float2* __restrict__ dg, const float2* __restrict__ x,
                 long long xrs, float2* __restrict__ y, long long yrs,
                 const float2* __restrict__ V, long long vis, long long vrs, int nb, GmresDev gs,
                 double2* partial, unsigned* counters) {
  pdl_enter();
  extern __shared__ float2 wsm[];  // [rows][nb + 8] per-warp sums
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const int zb = blockIdx.z % nzc;
  const int k0 = zb * ZC;
  const int r = blockIdx.z / nzc;
  const int lane = threadIdx.x, warp = threadIdx.y, rows = blockDim.y;
  const unsigned G = gridDim.x * gridDim.y * nzc;
  const unsigned bl = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zb);
  const bool inside = i < g.nx && j < g.ny;
  const long long sxy = (long long)g.nx * g.ny;
  const long long p0 = i + (long long)g.nx * j + sxy * k0;
  float2 yv[ZC];
#pragma unroll
  for (int t = 0; t < ZC; ++t) yv[t] = make_float2(0.f, 0.f);
  if (inside) {
    stencil32_column<ZC>(g, dg, x + r * xrs, i, j, k0, 0.f, 0.f, yv);
#pragma unroll
    for (int t = 0; t < ZC; ++t)
      if (k0 + t < g.nz) y[r * yrs + p0 + sxy * t] = yv[t];
  }
  if (KIND == 0 && gs.stopped[r]) return;  // uniform over the rhs: no reduction wanted
  const int nsl = KIND == 0 ? nb : 1;  // dot slots; the norm goes to slot nsl
  const int ldw = nsl + 8;
  const float2* Vr = V + r * vrs;
  for (int b0 = 0; b0 < nsl; b0 += 8) {
    float2 vv[8][ZC];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
      for (int e = 0; e < ZC; ++e)
        vv[t][e] = (inside && b0 + t < nsl && k0 + e < g.nz) ? Vr[(b0 + t) * vis + p0 + sxy * e]
                                                             : make_float2(0.f, 0.f);
    float2 acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      acc[t] = make_float2(0.f, 0.f);
#pragma unroll
      for (int e = 0; e < ZC; ++e) {
        const float2 v = vv[t][e], w = yv[e];
        if (KIND == 0) {  // conj(v) * y
          acc[t].x = fmaf(v.x, w.x, fmaf(v.y, w.y, acc[t].x));
          acc[t].y = fmaf(v.x, w.y, fmaf(-v.y, w.x, acc[t].y));
        } else {  // conj(y) * v
          acc[t].x = fmaf(w.x, v.x, fmaf(w.y, v.y, acc[t].x));
          acc[t].y = fmaf(w.x, v.y, fmaf(-w.y, v.x, acc[t].y));
        }
      }
    }
    const float2 red = warp_reduce8f(acc, lane);
    if ((lane & 3) == 0) {
      const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
      wsm[warp * ldw + b0 + t] = red;
    }
  }
  float q = 0.f;
#pragma unroll
  for (int e = 0; e < ZC; ++e) q = fmaf(yv[e].x, yv[e].x, fmaf(yv[e].y, yv[e].y, q));
  q = warp_sum(q);
  if (lane == 0) wsm[warp * ldw + nsl] = make_float2(q, 0.f);
  __syncthreads();
  const int nslots = nsl + 1;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  float4* part = reinterpret_cast<float4*>(partial) + (long long)r * (gs.mmax + 2) * G;
  for (int sidx = tid; sidx < nslots; sidx += 32 * rows) {
    float4 a = ffc_of(wsm[sidx]);
    for (int ww = 1; ww < rows; ++ww) a = ffc_add(a, ffc_of(wsm[ww * ldw + sidx]));
    part[(long long)sidx * G + bl] = a;
  }
  if (!last_of(counters + r, G)) return;
  if (KIND == 0) {
    double2* out = gs.h1 + (long long)r * (gs.mmax + 2);
    for (int sidx = warp; sidx < nslots; sidx += rows) {
      const float4 t = warp_sum_partials_ff(part, sidx, (int)G, lane);
      if (lane == 0) out[sidx] = d_from_ffc(t);
    }
    __syncthreads();
    if (tid == 0) counters[r] = 0;
  } else {
    __shared__ float4 tot[2];
    for (int sidx = warp; sidx < 2; sidx += rows) {
      const float4 t = warp_sum_partials_ff(part, sidx, (int)G, lane);
      if (lane == 0) tot[sidx] = t;
    }
    __syncthreads();
    if (tid == 0) {
      counters[r] = 0;
      double* sc = gs.scal + (long long)r * SC_COUNT;
      const float2 num = f_from_ffc(tot[0]);
      const float den = f_from_ffc(tot[1]).x;
      sc[SC_DR] = den != 0.f ? double(num.x / den) : 0.0;
      sc[SC_DI] = den != 0.f ? double(num.y / den) : 0.0;
    }
  }
}

__global__ void k_scale32(float2* __restrict__ dst, long long drs, const float2* __restrict__ src,
                          long long srs, long long n, GmresDev gs) {
  pdl_enter();
  const int r = blockIdx.y;
  const float s = float(gs.scal[(long long)r * SC_COUNT + SC_INV]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float2 v = src[r * srs + p];
    dst[r * drs + p] = make_float2(v.x * s, v.y * s);
  }
}

// d = <Aw, r> / <Aw, Aw> with float32 products, float-pair sums across warps and blocks and
// the quotient in float32 (Algorithm 1 step 3).
__global__ void __launch_bounds__(C_WARPS * 32)
k_fci_dots32(const float2* __restrict__ Aw, long long ars, const float2* __restrict__ rv,
             long long rrs, long long n, GmresDev gs, double2* partial, unsigned* counters) {
  pdl_enter();
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
  __shared__ float2 wn[C_WARPS], wd[C_WARPS];
  if (lane == 0) {
    wn[warp] = make_float2(nx, ny);
    wd[warp] = make_float2(dd, 0.f);
  }
  __syncthreads();
  float4* part = reinterpret_cast<float4*>(partial) + (long long)r * (gs.mmax + 2) * gridDim.x;
  if (threadIdx.x < 2) {
    const float2* src = threadIdx.x == 0 ? wn : wd;
    float4 a = ffc_of(src[0]);
    for (int ww = 1; ww < C_WARPS; ++ww) a = ffc_add(a, ffc_of(src[ww]));
    part[(long long)threadIdx.x * gridDim.x + blockIdx.x] = a;
  }
  if (!last_block(counters + r)) return;
  __shared__ float4 tot[2];
  if (warp < 2) {
    const float4 t = warp_sum_partials_ff(part, warp, (int)gridDim.x, lane);
    if (lane == 0) tot[warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    double* sc = gs.scal + (long long)r * SC_COUNT;
    const float2 num = f_from_ffc(tot[0]);
    const float den = f_from_ffc(tot[1]).x;
    sc[SC_DR] = den != 0.f ? double(num.x / den) : 0.0;
    sc[SC_DI] = den != 0.f ? double(num.y / den) : 0.0;
  }
}

// v0 = r - d Aw on float2 fields, ||v0||^2 -> inner cycle start.
__global__ void __launch_bounds__(C_WARPS * 32)
k_fci_start32(const float2* __restrict__ Aw, long long ars, const float2* __restrict__ rv,
              long long rrs, float2* __restrict__ v0, long long vrs, long long n, GmresDev gs,
              double2* partial, unsigned* counters) {
  pdl_enter();
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
  __shared__ float wq[C_WARPS];
  if (lane == 0) wq[warp] = q;
  __syncthreads();
  float4* part = reinterpret_cast<float4*>(partial) + (long long)r * (gs.mmax + 2) * gridDim.x;
  if (threadIdx.x == 0) {
    float4 a = ffc_of(make_float2(wq[0], 0.f));
    for (int ww = 1; ww < C_WARPS; ++ww) a = ffc_add(a, ffc_of(make_float2(wq[ww], 0.f)));
    part[blockIdx.x] = a;
  }
  if (!last_block(counters + r)) return;
  if (warp == 0) {
    const float4 t = warp_sum_partials_ff(part, 0, (int)gridDim.x, lane);
    if (lane == 0) {
      counters[r] = 0;
      double* sc = gs.scal + (long long)r * SC_COUNT;
      const float b2 = f_from_ffc(t).x;
      const float beta = sqrtf(b2);
      sc[SC_RES2] = double(b2);
      sc[SC_BETA] = double(beta);
      sc[SC_INV] = beta > 0.f ? double(1.f / beta) : 0.0;
      gs.g[(long long)r * (gs.mmax + 1)] = make_double2(double(beta), 0.0);
      gs.kend[r] = 0;
      gs.stopped[r] = beta > 0.f ? 0 : 1;
    }
  }
}

// y = R^{-1} g over the kend[r] leading columns in float32, one warp per rhs: the packed
// triangle and g are converted into shared memory by all lanes, lane 0 divides, the lanes
// update the remaining right-hand side (the float64 storage of GmresDev is kept).
__global__ void __launch_bounds__(32) k_backsolve32(GmresDev gs, int nvec) {
  pdl_enter();
  extern __shared__ float2 smt[];  // packed triangle (column i at i(i+1)/2) | right-hand side
  const int r = blockIdx.x;
  if (r >= nvec) return;
  const int lane = threadIdx.x;
  const int M = gs.mmax;
  float2* T = smt;
  float2* sv = smt + M * (M + 1) / 2;
  const int kk = gs.kend[r];
  const double2* R = gs.R + (long long)r * (M + 1) * M;
  const double2* g = gs.g + (long long)r * (M + 1);
  double2* y = gs.y + (long long)r * M;
  for (int i = 0; i < kk; ++i)
    for (int j = lane; j <= i; j += 32) {
      const double2 v = R[j + (long long)i * (M + 1)];
      T[i * (i + 1) / 2 + j] = make_float2(float(v.x), float(v.y));
    }
  for (int j = lane; j < kk; j += 32) sv[j] = make_float2(float(g[j].x), float(g[j].y));
  __syncwarp();
  for (int i = kk - 1; i >= 0; --i) {
    float yx = 0.f, yy = 0.f;
    if (lane == 0) {
      const float2 d = T[i * (i + 1) / 2 + i];
      const float2 si = sv[i];
      const float den = d.x * d.x + d.y * d.y;
      yx = (si.x * d.x + si.y * d.y) / den;
      yy = (si.y * d.x - si.x * d.y) / den;
    }
    yx = __shfl_sync(0xffffffffu, yx, 0);
    yy = __shfl_sync(0xffffffffu, yy, 0);
    if (lane == 0) y[i] = make_double2(double(yx), double(yy));
    for (int j = lane; j < i; j += 32) {
      const float2 t = T[i * (i + 1) / 2 + j];
      sv[j] = make_float2(sv[j].x - (t.x * yx - t.y * yy), sv[j].y - (t.x * yy + t.y * yx));
    }
    __syncwarp();
  }
}

// out = double(sum_{i<kend} y_i B_i) + d * E: the inner correction summed in float32, the
// float64 quadrature sum E added in float64 (Algorithm 1 step 5, v + d w).
__global__ void k_combine_fci32(double2* __restrict__ out, long long ors,
                                const float2* __restrict__ B, long long bis, long long brs,
                                GmresDev gs, const double2* __restrict__ E, long long ers,
                                long long n) {
  pdl_enter();
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
  const size_t smem = sizeof(float2) * ((size_t)C_WARPS * (nb + 8) + (size_t)nb);
  count_launch();
  if (mode == 0)
    return launch_pdl(k_cgs32<0>, grd, C_WARPS * 32, smem, st, V, vis, vrs, nb, w.p, w.rs, n, gs,
                      partial, counters, breakdown);
  if (mode == 1)
    return launch_pdl(k_cgs32<1>, grd, C_WARPS * 32, smem, st, V, vis, vrs, nb, w.p, w.rs, n, gs,
                      partial, counters, breakdown);
  return launch_pdl(k_cgs32<2>, grd, C_WARPS * 32, smem, st, V, vis, vrs, nb, w.p, w.rs, n, gs, partial,
                    counters, breakdown);
}

cudaError_t launch_scale32(Buf<float2> dst, Buf<const float2> src, long long n, const GmresDev& gs,
                           int nvec, cudaStream_t st) {
  count_launch();
  return launch_pdl(k_scale32, dim3(ew_blocks32(n), nvec), 256, 0, st, dst.p, dst.rs, src.p, src.rs,
                    n, gs);
}

cudaError_t launch_fci_start32(Buf<const float2> Aw, Buf<const float2> r, Buf<float2> v0,
                               const GmresDev& gs, double2* partial, unsigned* counters,
                               long long n, int nvec, cudaStream_t st) {
  dim3 grd(blocks32(n), nvec);
  count_launch();
  return launch_pdl(k_fci_start32, grd, C_WARPS * 32, 0, st, Aw.p, Aw.rs, r.p, r.rs, v0.p, v0.rs, n,
                    gs, partial, counters);
}

cudaError_t launch_fci_step32(Buf<const float2> Aw, Buf<const float2> r, Buf<float2> v0,
                              const GmresDev& gs, double2* partial, unsigned* counters,
                              long long n, int nvec, cudaStream_t st) {
  dim3 grd(blocks32(n), nvec);
  count_launch();
  const cudaError_t e = launch_pdl(k_fci_dots32, grd, C_WARPS * 32, 0, st, Aw.p, Aw.rs, r.p,
                                   r.rs, n, gs, partial, counters);
  if (e != cudaSuccess) return e;
  count_launch();
  return launch_pdl(k_fci_start32, grd, C_WARPS * 32, 0, st, Aw.p, Aw.rs, r.p, r.rs, v0.p, v0.rs, n,
                    gs, partial, counters);
}

cudaError_t launch_stencil32_dots(int kind, const Geom& g, const float2* dg, Buf<const float2> x,
                                  Buf<float2> y, const float2* V, long long vis, long long vrs,
                                  int nb, const GmresDev& gs, double2* partial,
                                  unsigned* counters, int nvec, cudaStream_t st) {
  constexpr int ZC = 4, ROWS = 4;  // 512 points per block: within the partial-sum buffer
  dim3 blk(32, ROWS, 1);
  dim3 grd((g.nx + 31) / 32, (g.ny + ROWS - 1) / ROWS, ((g.nz + ZC - 1) / ZC) * nvec);
  const int nsl = kind == 0 ? nb : 1;
  const size_t smem = sizeof(float2) * (size_t)ROWS * (nsl + 8);
  count_launch();
  if (kind == 0)
    return launch_pdl(k_stencil32_dots<ZC, 0>, grd, blk, smem, st, g, dg, x.p, x.rs, y.p, y.rs, V,
                      vis, vrs, nb, gs, partial, counters);
  return launch_pdl(k_stencil32_dots<ZC, 1>, grd, blk, smem, st, g, dg, x.p, x.rs, y.p, y.rs, V,
                    vis, vrs, 1, gs, partial, counters);
}

size_t backsolve32_smem(int mmax) { return sizeof(float2) * ((size_t)mmax * (mmax + 1) / 2 + mmax); }

cudaError_t prepare_kernels32(int mmax) {
  return cudaFuncSetAttribute(k_backsolve32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)backsolve32_smem(mmax));
}

cudaError_t launch_backsolve32(const GmresDev& gs, int nvec, cudaStream_t st) {
  if (gs.mmax > 128) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_backsolve32, nvec, 32, backsolve32_smem(gs.mmax), st, gs, nvec);
}

cudaError_t launch_combine_fci32(Buf<double2> out, const float2* B, long long bis, long long brs,
                                 const GmresDev& gs, Buf<const double2> E, long long n, int nvec,
                                 cudaStream_t st) {
  if (gs.mmax > 128) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_combine_fci32, dim3(ew_blocks32(n), nvec), 256, 0, st, out.p, out.rs, B, bis,
                    brs, gs, E.p, E.rs, n);
}

}  // namespace hz
