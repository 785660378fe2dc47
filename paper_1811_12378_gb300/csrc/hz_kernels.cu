// Device kernels of libhz: the shifted 7-point Helmholtz stencil, the batched stage of the
// polynomial fixed-point scheme with the fused quadrature sum, and the float64 Krylov
// reductions (CGS2 dots, norms, Givens, back substitution, combinations).
//
// Operator (§7.1 eq:stiff-mass, Case One of §3): in normalised units
//     (A - zI) x = (dg - z) x_p - cs * (sum of the 6 neighbours),
// dg = 6 cs - m_p - i a_p, cs = s/h^2, zero Dirichlet ghosts, a_p = sigma_max (depth_p /
// layer)^2 m_p in the sponge.  dg is precomputed once per problem (complex64 and complex128
// copies), so a stencil point reads its field and one diagonal value.
//
// Reductions are deterministic: each block writes its partial sums, the last block to finish
// (atomic ticket) adds them in block order and resets the ticket.
#include <cuda_runtime.h>

#include "hz_internal.h"
#include "hz_device.cuh"

namespace hz {

std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

constexpr int BX = 32;  // stencil block: 32 x 4 points of one z-plane
constexpr int BY = 4;
constexpr int CG_WARPS = 8;  // Gram-Schmidt block: 8 warps x 32 lanes x PPL points (PPL >= 4)

template <typename T> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

__device__ __forceinline__ int depth1(int i, int n, int L) {
  int e = min(i, n - 1 - i);
  return max(0, L - e);
}

// Sponge damping a_p = sigma_max * (d/L)^2 * m_p (0 without a layer).
__device__ __forceinline__ int sponge_depth(const Geom& g, int i, int j, int k) {
  return max(depth1(i, g.nx, g.layer), max(depth1(j, g.ny, g.layer), depth1(k, g.nz, g.layer)));
}
template <typename R>
__device__ __forceinline__ R sponge(const Geom& g, int i, int j, int k, R mp);
template <>
__device__ __forceinline__ double sponge<double>(const Geom& g, int i, int j, int k, double mp) {
  if (g.layer <= 0) return 0.0;
  const double t = double(sponge_depth(g, i, j, k)) / double(g.layer);
  return (g.sig * (t * t)) * mp;
}
template <typename R> __device__ __forceinline__ R lap_weight(const Geom& g);
template <> __device__ __forceinline__ double lap_weight<double>(const Geom& g) { return g.cs; }
template <> __device__ __forceinline__ float lap_weight<float>(const Geom& g) { return g.csf; }

// Sum of the six neighbours of point p = (i, j, k); zero beyond the boundary.
template <typename T>
__device__ __forceinline__ T nbsum(const T* __restrict__ x, long long p, int i, int j, int k,
                                   const Geom& g) {
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  T s = czero<T>();
  if (i > 0) s = cadd(s, x[p - 1]);
  if (i < g.nx - 1) s = cadd(s, x[p + 1]);
  if (j > 0) s = cadd(s, x[p - sy]);
  if (j < g.ny - 1) s = cadd(s, x[p + sy]);
  if (k > 0) s = cadd(s, x[p - sz]);
  if (k < g.nz - 1) s = cadd(s, x[p + sz]);
  return s;
}

// ((A - zI) x)_p from the centre value, the neighbour sum and the local coefficients.
template <typename T, typename R>
__device__ __forceinline__ T apply_point(T xc, T nb, R cs, R mp, R ap, R zr, R zi) {
  T t = mk(R(6) * xc.x - nb.x, R(6) * xc.y - nb.y);
  R dr = -(mp + zr), di = -(ap + zi);
  return mk(cs * t.x + dr * xc.x - di * xc.y, cs * t.y + dr * xc.y + di * xc.x);
}

// Complex64 shifted stencil from the precomputed diagonal, z-columns of ZC points per thread
// (stencil32_column in hz_device.cuh).
template <int ZC>
__global__ void __launch_bounds__(256)
k_stencil32(Geom g, const float2* __restrict__ dg, const float2* __restrict__ x, long long xrs,
            float2* __restrict__ y, long long yrs, float zr, float zi) {
  pdl_enter();
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const int k0 = (blockIdx.z % nzc) * ZC;
  const int r = blockIdx.z / nzc;
  if (i >= g.nx || j >= g.ny) return;
  const long long sxy = (long long)g.nx * g.ny;
  const long long p0 = i + (long long)g.nx * j + sxy * k0;
  float2 yv[ZC];
  stencil32_column<ZC>(g, dg, x + r * xrs, i, j, k0, zr, zi, yv);
#pragma unroll
  for (int t = 0; t < ZC; ++t)
    if (k0 + t < g.nz) y[r * yrs + p0 + sxy * t] = yv[t];
}

// ---------------------------------------------------------------- polynomial stage
// One stencil sweep of every active node of the scheme eq:fix-pt-exp.
//
// Block: 32 consecutive x-points of one grid row, times the active nodes (warp y works on
// node y, so a warp runs one node kind without divergence and the node warps hide each
// other's latency).  Each thread walks a column of ZC points along z: all loads of the column
// are issued together, the z-neighbours of one point are the centres of the next, and the
// operator's diagonal comes precomputed (dg = 6 s/h^2 - m - i a), so a point costs a few
// dozen instructions.  Fields of one node are distinct buffers, so the __restrict__
// qualifiers below hold.  On the final stage of an FCI application the block sums
// sigma_j/z_j y_j over its nodes in shared memory (float64) and writes the quadrature sum w.
template <typename T> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

template <typename T, int ZC>
__global__ void __launch_bounds__(512)
k_poly_stage(Geom g, const T* __restrict__ dg, const T* __restrict__ f, long long frs, T* ws,
             long long wrs, double2* __restrict__ w, long long wwrs, float2* __restrict__ w32,
             long long w32rs, const StageArgs<typename RealOf<T>::type> a) {
  pdl_enter();
  using R = typename RealOf<T>::type;
  extern __shared__ double2 qs[];  // [rows][nnodes][ZC][32] on the final stage only
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * blockDim.z + threadIdx.z;
  const int nzc = (g.nz + ZC - 1) / ZC;
  const int k0 = (blockIdx.z % nzc) * ZC;
  const int r = blockIdx.z / nzc;
  const int q = threadIdx.y;
  const bool inside = i < g.nx && j < g.ny;
  const long long sxy = (long long)g.nx * g.ny;
  const long long p0 = i + (long long)g.nx * j + sxy * k0;
  const StageNode<R>& nd = a.nd[q];
  const int kind = nd.kind;
  T yn[ZC];
#pragma unroll
  for (int t = 0; t < ZC; ++t) yn[t] = czero<T>();
  if (inside) {
    T* wsr = ws + r * wrs;
    const T* __restrict__ fr = f + r * frs;
    const T* __restrict__ in = wsr + nd.in;
    const T* accin = wsr + nd.acc;  // accin and accout alias: no __restrict__ on either
    T* __restrict__ kout = wsr + nd.kout;
    T* accout = wsr + nd.acc;
    T* __restrict__ yout = wsr + nd.yout;
    const bool first = kind == SK_FIRST || kind == SK_FIRST_LAST;
    const bool stencil = !(first && nd.yzero);
    const bool use_acc = kind == SK_MID || kind == SK_LAST;
    const T zero = czero<T>();
    T fv[ZC], dv[ZC], av[ZC], xm[ZC], xp[ZC], ym[ZC], yp[ZC], c[ZC + 2];
#pragma unroll
    for (int t = 0; t < ZC; ++t) {
      const bool ok = k0 + t < g.nz;
      const long long pp = p0 + sxy * t;
      fv[t] = ok ? fr[pp] : zero;
      dv[t] = ok ? dg[pp] : zero;
      av[t] = (ok && use_acc) ? accin[pp] : zero;
      xm[t] = (ok && stencil && i > 0) ? in[pp - 1] : zero;
      xp[t] = (ok && stencil && i < g.nx - 1) ? in[pp + 1] : zero;
      ym[t] = (ok && stencil && j > 0) ? in[pp - g.nx] : zero;
      yp[t] = (ok && stencil && j < g.ny - 1) ? in[pp + g.nx] : zero;
    }
#pragma unroll
    for (int t = 0; t < ZC + 2; ++t) {
      const int kz = k0 + t - 1;
      c[t] = (stencil && kz >= 0 && kz < g.nz) ? in[p0 + sxy * (t - 1)] : zero;
    }
    const R cs = lap_weight<R>(g);
    const T md = mk(nd.mdr, nd.mdi);
    const T cf = mk(nd.cfr, nd.cfi);
    const T ip = mk(nd.ipr, nd.ipi);
#pragma unroll
    for (int t = 0; t < ZC; ++t) {
      if (k0 + t >= g.nz) break;
      const long long pp = p0 + sxy * t;
      // (A - z0) x at this point, x = the node's input field
      const T xc = c[t + 1];
      const R nbx = ((xm[t].x + xp[t].x) + (ym[t].x + yp[t].x)) + (c[t].x + c[t + 2].x);
      const R nby = ((xm[t].y + xp[t].y) + (ym[t].y + yp[t].y)) + (c[t].y + c[t + 2].y);
      const R dr = dv[t].x - nd.z0r, di = dv[t].y - nd.z0i;
      const T Ax = mk(dr * xc.x - di * xc.y - cs * nbx, dr * xc.y + di * xc.x - cs * nby);
      if (first) {
        // k1 = -i delta ((A - z0) y - f), acc = y + k1; with y = 0: k1 = -i delta (-f)
        const T kv = cmul(md, csub(Ax, fv[t]));
        if (kind == SK_FIRST) {
          kout[pp] = kv;
          accout[pp] = cadd(xc, kv);
        } else {
          yn[t] = cmul(cadd(xc, kv), ip);
        }
      } else {
        const T kv = cmul(md, csub(Ax, cmul(cf, fv[t])));
        if (kind == SK_MID) {
          kout[pp] = kv;
          accout[pp] = cadd(av[t], kv);
        } else {
          yn[t] = cmul(cadd(av[t], kv), ip);
        }
      }
      if (!a.final_quad && (kind == SK_LAST || kind == SK_FIRST_LAST)) yout[pp] = yn[t];
    }
  }
  if (a.final_quad) {  // uniform over the launch; every node is LAST or FIRST_LAST here
    if (sizeof(T) == 8 && a.quad64) {
      // complex64 y, float64 sum: each y_j is exact in float64, so the terms and their sum
      // carry only float64 rounding (the quadrature accumulation of the float64-outer form)
      double2* qr = qs + (size_t)threadIdx.z * a.nnodes * ZC * 32;
#pragma unroll
      for (int t = 0; t < ZC; ++t) {
        const double yr = double(yn[t].x), yi = double(yn[t].y);
        qr[(q * ZC + t) * 32 + threadIdx.x] =
            make_double2(fma(nd.wqr, yr, -nd.wqi * yi), fma(nd.wqr, yi, nd.wqi * yr));
      }
      __syncthreads();
      if (inside) {
        for (int t = q; t < ZC; t += a.nnodes) {
          if (k0 + t >= g.nz) break;
          double sx = 0.0, sy = 0.0;
          for (int u = 0; u < a.nnodes; ++u) {
            const double2 v = qr[(u * ZC + t) * 32 + threadIdx.x];
            sx += v.x;
            sy += v.y;
          }
          w[r * wwrs + p0 + sxy * t] = make_double2(sx, sy);
          if (w32) w32[r * w32rs + p0 + sxy * t] = make_float2(float(sx), float(sy));
        }
      }
    } else if constexpr (sizeof(T) == 8) {
      // complex64 y: each node's term (sigma_j / z_j) y_j as float pairs (hi + lo) from
      // error-free products and sums, then a float-pair sum over the nodes (about 48 bits,
      // no float64 instruction until the final conversion)
      float4* qf = reinterpret_cast<float4*>(qs) + (size_t)threadIdx.z * a.nnodes * ZC * 32;
#pragma unroll
      for (int t = 0; t < ZC; ++t) {
        const float yr = yn[t].x, yi = yn[t].y;
        float2 tx = two_prod_ff(yr, nd.wrh, nd.wrl), tx2 = two_prod_ff(yi, nd.wih, nd.wil);
        float2 ty = two_prod_ff(yi, nd.wrh, nd.wrl), ty2 = two_prod_ff(yr, nd.wih, nd.wil);
        tx = ff_add(tx, make_float2(-tx2.x, -tx2.y));
        ty = ff_add(ty, ty2);
        qf[(q * ZC + t) * 32 + threadIdx.x] = make_float4(tx.x, tx.y, ty.x, ty.y);
      }
      __syncthreads();
      if (inside) {
        for (int t = q; t < ZC; t += a.nnodes) {  // warp q sums column points q, q + nnodes, ...
          if (k0 + t >= g.nz) break;
          float2 sx = make_float2(0.f, 0.f), sy = make_float2(0.f, 0.f);
          for (int u = 0; u < a.nnodes; ++u) {
            const float4 v = qf[(u * ZC + t) * 32 + threadIdx.x];
            sx = ff_add(sx, make_float2(v.x, v.y));
            sy = ff_add(sy, make_float2(v.z, v.w));
          }
          const long long pp = p0 + sxy * t;
          w[r * wwrs + pp] = make_double2(double(sx.x) + double(sx.y), double(sy.x) + double(sy.y));
          if (w32) w32[r * w32rs + pp] = make_float2(__fadd_rn(sx.x, sx.y), __fadd_rn(sy.x, sy.y));
        }
      }
    } else {
      double2* qr = qs + (size_t)threadIdx.z * a.nnodes * ZC * 32;
#pragma unroll
      for (int t = 0; t < ZC; ++t) {
        const double yr = double(yn[t].x), yi = double(yn[t].y);
        qr[(q * ZC + t) * 32 + threadIdx.x] =
            make_double2(nd.wqr * yr - nd.wqi * yi, nd.wqr * yi + nd.wqi * yr);
      }
      __syncthreads();
      if (inside) {
        for (int t = q; t < ZC; t += a.nnodes) {  // warp q sums column points q, q + nnodes, ...
          if (k0 + t >= g.nz) break;
          double sx = 0.0, sy = 0.0;
          for (int u = 0; u < a.nnodes; ++u) {
            const double2 v = qr[(u * ZC + t) * 32 + threadIdx.x];
            sx += v.x;
            sy += v.y;
          }
          w[r * wwrs + p0 + sxy * t] = make_double2(sx, sy);
          if (w32)
            w32[r * w32rs + p0 + sxy * t] = make_float2(float(sx), float(sy));
        }
      }
    }
  }
}

// ---------------------------------------------------------------- conversions
__global__ void k_c128_to_c64(const double2* __restrict__ x, long long xrs, float2* __restrict__ y,
                              long long yrs, long long n) {
  pdl_enter();
  const int r = blockIdx.y;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 v = x[r * xrs + p];
    y[r * yrs + p] = make_float2(float(v.x), float(v.y));
  }
}

__global__ void k_c64_to_c128(const float2* __restrict__ x, long long xrs, double2* __restrict__ y,
                              long long yrs, long long n) {
  pdl_enter();
  const int r = blockIdx.y;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float2 v = x[r * xrs + p];
    y[r * yrs + p] = make_double2(double(v.x), double(v.y));
  }
}

// Classical Gram-Schmidt pieces in float64.  A block of CG_WARPS warps owns 256 PPL points;
// lane l of warp w owns the PPL points seg + l + 32 e, kept in registers, so every basis
// field is read with coalesced 512-byte warp loads.  Dots are formed 8 basis fields at a time
// and reduced by warp_reduce8; per-warp sums go through shared memory to one partial per
// block, and the last block adds the partials in block order (warp per slot).
template <int MODE, int PPL>
__global__ void __launch_bounds__(CG_WARPS * 32)
k_cgs(const double2* __restrict__ V, long long vis, long long vrs, int nb, double2* w,
      long long wrs, long long n, GmresDev gs, double2* partial, unsigned* counters, double brk) {
  pdl_enter();
  extern __shared__ double2 sm[];  // hs[nb] | wp[CG_WARPS][nb + 8]
  const int r = blockIdx.y;
  if (gs.stopped[r]) return;
  const int M = gs.mmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldw = nb + 8;
  const long long seg =
      (long long)blockIdx.x * (CG_WARPS * 32 * PPL) + (long long)warp * 32 * PPL + lane;
  double2* wr = w + r * wrs;
  const double2* Vr = V + r * vrs;
  double2* hs = sm;
  double2* wp = sm + nb;
  if (MODE != 0) {
    const double2* hp = (MODE == 1 ? gs.h1 : gs.h2) + (long long)r * (M + 2);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hs[b] = hp[b];
    __syncthreads();
  }
  double2 wv[PPL];
#pragma unroll
  for (int e = 0; e < PPL; ++e) {
    const long long p = seg + 32LL * e;
    wv[e] = p < n ? wr[p] : make_double2(0.0, 0.0);
  }
  if (MODE != 0) {
    for (int b = 0; b < nb; ++b) {
      const double2 h = hs[b];
      const double2* vb = Vr + b * vis;
#pragma unroll
      for (int e = 0; e < PPL; ++e) {
        const long long p = seg + 32LL * e;
        if (p < n) {
          const double2 v = vb[p];
          wv[e].x = fma(-h.x, v.x, fma(h.y, v.y, wv[e].x));
          wv[e].y = fma(-h.x, v.y, fma(-h.y, v.x, wv[e].y));
        }
      }
    }
#pragma unroll
    for (int e = 0; e < PPL; ++e) {
      const long long p = seg + 32LL * e;
      if (p < n) wr[p] = wv[e];
    }
  }
  if (MODE != 2) {
    for (int b0 = 0; b0 < nb; b0 += 8) {
      double2 acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = make_double2(0.0, 0.0);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (b0 + t < nb) {
          const double2* vb = Vr + (b0 + t) * vis;
#pragma unroll
          for (int e = 0; e < PPL; ++e) {
            const long long p = seg + 32LL * e;
            if (p < n) {
              const double2 v = vb[p];
              acc[t].x = fma(v.x, wv[e].x, fma(v.y, wv[e].y, acc[t].x));
              acc[t].y = fma(v.x, wv[e].y, fma(-v.y, wv[e].x, acc[t].y));
            }
          }
        }
      }
      const double2 red = warp_reduce8(acc, lane);
      if ((lane & 3) == 0) {
        const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (b0 + t < nb) wp[warp * ldw + b0 + t] = red;  // slot nb is the norm's (mode 0)
      }
    }
  }
  if (MODE != 1) {
    double q = 0.0;
#pragma unroll
    for (int e = 0; e < PPL; ++e) q = fma(wv[e].x, wv[e].x, fma(wv[e].y, wv[e].y, q));
    for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
    if (lane == 0) wp[warp * ldw + (MODE == 0 ? nb : 0)] = make_double2(q, 0.0);
  }
  __syncthreads();
  const int nslots = MODE == 0 ? nb + 1 : (MODE == 1 ? nb : 1);
  double2* part = partial + (long long)r * (M + 2) * gridDim.x;
  for (int sidx = threadIdx.x; sidx < nslots; sidx += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int ww = 0; ww < CG_WARPS; ++ww) acc = cadd(acc, wp[ww * ldw + sidx]);
    part[(long long)sidx * gridDim.x + blockIdx.x] = acc;
  }
  if (!last_block(counters + r)) return;
  double2* out = MODE == 0 ? gs.h1 + (long long)r * (M + 2)
               : MODE == 1 ? gs.h2 + (long long)r * (M + 2) : gs.nrm + 2 * r;
  for (int sidx = warp; sidx < nslots; sidx += CG_WARPS) {
    const double2 t = warp_sum_partials(part, sidx, (int)gridDim.x, lane);
    if (lane == 0) out[sidx] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) counters[r] = 0;
  if (MODE == 2) givens_column(gs, r, nb - 1, brk);  // whole block
}

// A field value as float64 (complex64 input converts exactly).
__device__ __forceinline__ double2 as_d2(double2 v) { return v; }
__device__ __forceinline__ double2 as_d2(float2 v) { return make_double2(double(v.x), double(v.y)); }

// Float64 shifted stencil from the precomputed complex diagonal d = 6 s/h^2 - m - i a:
//     (A - zI) x = (d - z) x - (s/h^2) * (sum of the 6 neighbours).
// About 16 float64 operations a point (the float64 pipe is the scarce unit on GB300).
// FF: the result is stored as float pairs (float4 per complex point) for the float-pair
// Arnoldi of HZ_MIXED_C64_FF.  TX: the input field's type (double2, or float2 for FGMRES
// directions stored in complex64; the arithmetic is float64 either way).
template <bool FF, typename TX>
__global__ void __launch_bounds__(BX * BY)
k_stencil_diag(Geom g, const double2* __restrict__ dg, const TX* __restrict__ x,
               long long xrs, double2* __restrict__ y, long long yrs, double zr, double zi) {
  pdl_enter();
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z % g.nz;
  const int r = blockIdx.z / g.nz;
  if (i >= g.nx || j >= g.ny) return;
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  const long long p = i + sy * j + sz * k;
  const TX* xr = x + r * xrs;
  const double2 z0 = make_double2(0.0, 0.0);
  const double2 xm = i > 0 ? as_d2(xr[p - 1]) : z0, xp = i < g.nx - 1 ? as_d2(xr[p + 1]) : z0;
  const double2 ym = j > 0 ? as_d2(xr[p - sy]) : z0, yp = j < g.ny - 1 ? as_d2(xr[p + sy]) : z0;
  const double2 zm = k > 0 ? as_d2(xr[p - sz]) : z0, zp = k < g.nz - 1 ? as_d2(xr[p + sz]) : z0;
  const double2 xc = as_d2(xr[p]);
  const double2 d = dg[p];
  const double nbx = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
  const double nby = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
  const double dr = d.x - zr, di = d.y - zi;
  const double mcs = -g.cs;
  const double yx = fma(dr, xc.x, fma(-di, xc.y, mcs * nbx));
  const double yy = fma(dr, xc.y, fma(di, xc.x, mcs * nby));
  if constexpr (FF) {
    const float2 a = ff_from_d(yx), b = ff_from_d(yy);
    reinterpret_cast<float4*>(y)[r * yrs + p] = make_float4(a.x, a.y, b.x, b.y);
  } else {
    y[r * yrs + p] = make_double2(yx, yy);
  }
}

__global__ void k_scale(double2* __restrict__ dst, long long drs, const double2* __restrict__ src,
                        long long srs, long long n, GmresDev gs) {
  pdl_enter();
  const int r = blockIdx.y;
  const double s = gs.scal[(long long)r * SC_COUNT + SC_INV];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[r * srs + p];
    dst[r * drs + p] = make_double2(v.x * s, v.y * s);
  }
}

template <typename TB>
__global__ void k_combine(double2* out, long long ors, const TB* __restrict__ B, long long bis,
                          long long brs, GmresDev gs, const double2* __restrict__ E, long long ers,
                          int use_e, int accumulate, long long n) {
  pdl_enter();
  const int r = blockIdx.y;
  const int kk = gs.kend[r];
  const double2* y = gs.y + (long long)r * gs.mmax;
  const double* sc = gs.scal + (long long)r * SC_COUNT;
  const double2 d = make_double2(sc[SC_DR], sc[SC_DI]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 acc = accumulate ? out[r * ors + p] : make_double2(0.0, 0.0);
    for (int b = 0; b < kk; ++b) acc = cadd(acc, cmul(y[b], as_d2(B[r * brs + b * bis + p])));
    if (use_e) acc = cadd(acc, cmul(d, E[r * ers + p]));
    out[r * ors + p] = acc;
  }
}

// y = R^{-1} g over the kend[r] leading columns, one block per rhs.  The packed upper
// triangle is staged in shared memory; warp 0 then sweeps the columns from the last one,
// each lane updating its share of the remaining right-hand side.
__global__ void __launch_bounds__(256) k_backsolve(GmresDev gs, int nvec) {
  pdl_enter();
  extern __shared__ double2 smb[];
  const int r = blockIdx.x;
  if (r >= nvec) return;
  const int M = gs.mmax;
  const int kk = gs.kend[r];
  const double2* R = gs.R + (long long)r * (M + 1) * M;
  const double2* g = gs.g + (long long)r * (M + 1);
  double2* y = gs.y + (long long)r * M;
  double2* T = smb;                 // column i at i(i+1)/2, rows 0..i
  double2* s = smb + kk * (kk + 1) / 2;
  for (int i = 0; i < kk; ++i)
    for (int j = threadIdx.x; j <= i; j += blockDim.x)
      T[i * (i + 1) / 2 + j] = R[j + (long long)i * (M + 1)];
  for (int j = threadIdx.x; j < kk; j += blockDim.x) s[j] = g[j];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  for (int i = kk - 1; i >= 0; --i) {
    double yx = 0.0, yy = 0.0;
    if (lane == 0) {
      const double2 d = T[i * (i + 1) / 2 + i];
      const double2 si = s[i];
      const double den = d.x * d.x + d.y * d.y;
      yx = (si.x * d.x + si.y * d.y) / den;
      yy = (si.y * d.x - si.x * d.y) / den;
      y[i] = make_double2(yx, yy);
    }
    yx = __shfl_sync(0xffffffffu, yx, 0);
    yy = __shfl_sync(0xffffffffu, yy, 0);
    const double2 yi = make_double2(yx, yy);
    for (int j = lane; j < i; j += 32) s[j] = csub(s[j], cmul(T[i * (i + 1) / 2 + j], yi));
    __syncwarp();
  }
}

// Start of a cycle: v0 = fs*f - A x (x may be null), beta = ||v0||, g[0] = beta.
__device__ void start_cycle(const GmresDev& gs, int r, double2 nrm2) {
  double* sc = gs.scal + (long long)r * SC_COUNT;
  const double beta = sqrt(nrm2.x);
  sc[SC_RES2] = nrm2.x;
  sc[SC_BETA] = beta;
  sc[SC_INV] = beta > 0.0 ? 1.0 / beta : 0.0;
  gs.g[(long long)r * (gs.mmax + 1)] = make_double2(beta, 0.0);
  gs.kend[r] = 0;
  gs.stopped[r] = beta > 0.0 ? 0 : 1;
}

__global__ void __launch_bounds__(RED_THREADS)
k_residual_start(Geom g, const double* __restrict__ m, const double2* __restrict__ f,
                 long long frs, double fs, const double2* __restrict__ x, long long xrs,
                 double2* __restrict__ v0, long long vrs, GmresDev gs, double2* partial,
                 unsigned* counters) {
  pdl_enter();
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  const long long base = (long long)blockIdx.x * RED_CHUNK + threadIdx.x;
  const long long sxy = (long long)g.nx * g.ny;
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < RED_PPT; ++e) {
    const long long p = base + (long long)e * RED_THREADS;
    if (p >= g.n) continue;
    const double2 fv = f[r * frs + p];
    double2 v = make_double2(fs * fv.x, fs * fv.y);
    if (x) {
      const int k = int(p / sxy);
      const long long rem = p - (long long)k * sxy;
      const int j = int(rem / g.nx);
      const int i = int(rem - (long long)j * g.nx);
      const double2* xr = x + r * xrs;
      const double mp = m[p];
      const double ap = sponge<double>(g, i, j, k, mp);
      v = csub(v, apply_point<double2, double>(xr[p], nbsum(xr, p, i, j, k, g), g.cs, mp, ap,
                                               0.0, 0.0));
    }
    v0[r * vrs + p] = v;
    s += v.x * v.x + v.y * v.y;
  }
  double2* part = partial + (long long)r * (gs.mmax + 2) * gridDim.x;
  double2 t = block_sum(make_double2(s, 0.0), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (!last_block(counters + r)) return;
  __shared__ double2 tot;
  finish_slots(part, 1, &tot, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    start_cycle(gs, r, tot);
  }
}

// d = <Aw, r> / <Aw, Aw>  (Algorithm 1, step size; d = 0 when Aw = 0)
__global__ void __launch_bounds__(RED_THREADS)
k_fci_dots(const double2* __restrict__ Aw, long long ars, const double2* __restrict__ rv,
           long long rrs, long long n, GmresDev gs, double2* partial, unsigned* counters) {
  pdl_enter();
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  const long long base = (long long)blockIdx.x * RED_CHUNK + threadIdx.x;
  double2 num = make_double2(0.0, 0.0);
  double den = 0.0;
#pragma unroll
  for (int e = 0; e < RED_PPT; ++e) {
    const long long p = base + (long long)e * RED_THREADS;
    if (p >= n) continue;
    const double2 a = Aw[r * ars + p];
    num = cadd(num, cmulc(a, rv[r * rrs + p]));
    den += a.x * a.x + a.y * a.y;
  }
  double2* part = partial + (long long)r * (gs.mmax + 2) * gridDim.x;
  double2 t = block_sum(num, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  t = block_sum(make_double2(den, 0.0), sh);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t;
  if (!last_block(counters + r)) return;
  __shared__ double2 tot[2];
  finish_slots(part, 2, tot, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    double* sc = gs.scal + (long long)r * SC_COUNT;
    const double dd = tot[1].x;
    sc[SC_DR] = dd != 0.0 ? tot[0].x / dd : 0.0;
    sc[SC_DI] = dd != 0.0 ? tot[0].y / dd : 0.0;
  }
}

// v0 = r - d Aw, then the inner cycle start (||v0|| -> beta)
__global__ void __launch_bounds__(RED_THREADS)
k_fci_start(const double2* __restrict__ Aw, long long ars, const double2* __restrict__ rv,
            long long rrs, double2* __restrict__ v0, long long vrs, long long n, GmresDev gs,
            double2* partial, unsigned* counters) {
  pdl_enter();
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  const long long base = (long long)blockIdx.x * RED_CHUNK + threadIdx.x;
  const double* sc = gs.scal + (long long)r * SC_COUNT;
  const double2 d = make_double2(sc[SC_DR], sc[SC_DI]);
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < RED_PPT; ++e) {
    const long long p = base + (long long)e * RED_THREADS;
    if (p >= n) continue;
    const double2 v = csub(rv[r * rrs + p], cmul(d, Aw[r * ars + p]));
    v0[r * vrs + p] = v;
    s += v.x * v.x + v.y * v.y;
  }
  double2* part = partial + (long long)r * (gs.mmax + 2) * gridDim.x;
  double2 t = block_sum(make_double2(s, 0.0), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (!last_block(counters + r)) return;
  __shared__ double2 tot;
  finish_slots(part, 1, &tot, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    start_cycle(gs, r, tot);
  }
}

inline unsigned red_blocks(long long n) { return unsigned((n + RED_CHUNK - 1) / RED_CHUNK); }
inline unsigned ew_blocks(long long n) {
  long long b = (n + 255) / 256;
  return unsigned(b < 4096 ? b : 4096);
}

}  // namespace

// ---------------------------------------------------------------- wrappers
template <typename T, typename R>
cudaError_t launch_poly_stage(const Geom& g, const T* dg, Buf<const T> f, T* ws, long long wrs,
                              Buf<double2> w, Buf<float2> w32, int nvec, const StageArgs<R>& a,
                              cudaStream_t st) {
  const int cls = stage_class(a.nnodes);
  int zc = g.pzc[cls];
  if (sizeof(T) == 16 && zc > 2) zc = 2;  // float64 columns: register budget
  const int rows = g.prows[cls];
  dim3 blk(32, a.nnodes, rows);
  dim3 grd((g.nx + 31) / 32, (g.ny + rows - 1) / rows, ((g.nz + zc - 1) / zc) * nvec);
  const size_t smem = a.final_quad ? sizeof(double2) * 32 * zc * a.nnodes * rows : 0;
  count_launch();
  switch (zc) {
    case 1:
      return launch_pdl(k_poly_stage<T, 1>, grd, blk, smem, st, g, dg, f.p, f.rs, ws, wrs, w.p,
                        w.rs, w32.p, w32.rs, a);
    case 2:
      return launch_pdl(k_poly_stage<T, 2>, grd, blk, smem, st, g, dg, f.p, f.rs, ws, wrs, w.p,
                        w.rs, w32.p, w32.rs, a);
    default:
      if constexpr (sizeof(T) == 8)
        return launch_pdl(k_poly_stage<T, 4>, grd, blk, smem, st, g, dg, f.p, f.rs, ws, wrs, w.p,
                          w.rs, w32.p, w32.rs, a);
      return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_poly_stage<float2, float>(const Geom&, const float2*, Buf<const float2>,
                                                      float2*, long long, Buf<double2>,
                                                      Buf<float2>, int, const StageArgs<float>&,
                                                      cudaStream_t);
template cudaError_t launch_poly_stage<double2, double>(const Geom&, const double2*,
                                                        Buf<const double2>, double2*, long long,
                                                        Buf<double2>, Buf<float2>, int,
                                                        const StageArgs<double>&, cudaStream_t);

cudaError_t launch_convert_c128_c64(Buf<const double2> x, Buf<float2> y, long long n, int nvec,
                                    cudaStream_t st) {
  count_launch();
  return launch_pdl(k_c128_to_c64, dim3(ew_blocks(n), nvec), 256, 0, st, x.p, x.rs, y.p, y.rs, n);
}

cudaError_t launch_convert_c64_c128(Buf<const float2> x, Buf<double2> y, long long n, int nvec,
                                    cudaStream_t st) {
  count_launch();
  return launch_pdl(k_c64_to_c128, dim3(ew_blocks(n), nvec), 256, 0, st, x.p, x.rs, y.p, y.rs, n);
}

// Points per lane of the float64 Gram-Schmidt kernels.  They are bound by the float64 pipe,
// which the blocks resident on an SM share, so the time is set by the SM with the most work:
// ceil(blocks * nvec / SMs) * PPL.  The smallest such PPL wins (ties: the smaller PPL).
int cgs_ppl(long long n, int nvec) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  static const int cand[] = {4, 5, 6, 7, 8};
  int best = 4;
  long long best_cost = -1;
  for (int ppl : cand) {
    const long long blocks = (n + CG_WARPS * 32LL * ppl - 1) / (CG_WARPS * 32LL * ppl);
    const long long cost = (blocks * nvec + sms - 1) / sms * ppl;
    if (best_cost < 0 || cost < best_cost) {
      best = ppl;
      best_cost = cost;
    }
  }
  return best;
}

template <int MODE, int PPL>
cudaError_t launch_cgs_ppl(const double2* V, long long vis, long long vrs, int nb, Buf<double2> w,
                           long long n, const GmresDev& gs, double2* partial, unsigned* counters,
                           int nvec, double breakdown, cudaStream_t st) {
  const long long chunk = CG_WARPS * 32LL * PPL;
  dim3 grd(unsigned((n + chunk - 1) / chunk), nvec);
  const size_t smem = sizeof(double2) * (size_t)(nb + CG_WARPS * (nb + 8));
  return launch_pdl(k_cgs<MODE, PPL>, grd, dim3(CG_WARPS * 32), smem, st, V, vis, vrs, nb, w.p,
                    w.rs, n, gs, partial, counters, breakdown);
}

template <int MODE>
cudaError_t launch_cgs_mode(int ppl, const double2* V, long long vis, long long vrs, int nb,
                            Buf<double2> w, long long n, const GmresDev& gs, double2* partial,
                            unsigned* counters, int nvec, double breakdown, cudaStream_t st) {
  switch (ppl) {
    case 5: return launch_cgs_ppl<MODE, 5>(V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
    case 6: return launch_cgs_ppl<MODE, 6>(V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
    case 7: return launch_cgs_ppl<MODE, 7>(V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
    case 8: return launch_cgs_ppl<MODE, 8>(V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
    default: return launch_cgs_ppl<MODE, 4>(V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
  }
}

cudaError_t launch_cgs(int mode, const double2* V, long long vis, long long vrs, int nb,
                       Buf<double2> w, long long n, const GmresDev& gs, double2* partial,
                       unsigned* counters, int nvec, double breakdown, cudaStream_t st) {
  const int ppl = cgs_ppl(n, nvec);
  count_launch();
  if (mode == 0)
    return launch_cgs_mode<0>(ppl, V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
  if (mode == 1)
    return launch_cgs_mode<1>(ppl, V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
  return launch_cgs_mode<2>(ppl, V, vis, vrs, nb, w, n, gs, partial, counters, nvec, breakdown, st);
}

cudaError_t launch_stencil32(const Geom& g, const float2* dg, Buf<const float2> x, Buf<float2> y,
                             int nvec, double zr, double zi, cudaStream_t st) {
  const int zc = g.szc, rows = g.srows;
  dim3 blk(32, rows, 1);
  dim3 grd((g.nx + 31) / 32, (g.ny + rows - 1) / rows, ((g.nz + zc - 1) / zc) * nvec);
  count_launch();
  switch (zc) {
    case 2:
      return launch_pdl(k_stencil32<2>, grd, blk, 0, st, g, dg, x.p, x.rs, y.p, y.rs, float(zr),
                        float(zi));
    case 8:
      return launch_pdl(k_stencil32<8>, grd, blk, 0, st, g, dg, x.p, x.rs, y.p, y.rs, float(zr),
                        float(zi));
    default:
      return launch_pdl(k_stencil32<4>, grd, blk, 0, st, g, dg, x.p, x.rs, y.p, y.rs, float(zr),
                        float(zi));
  }
}

cudaError_t launch_stencil_diag(const Geom& g, const double2* dg, Buf<const double2> x,
                                Buf<double2> y, int nvec, double zr, double zi, cudaStream_t st) {
  dim3 blk(BX, BY, 1);
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz * nvec);
  count_launch();
  return launch_pdl(k_stencil_diag<false, double2>, grd, blk, 0, st, g, dg, x.p, x.rs, y.p, y.rs,
                    zr, zi);
}

cudaError_t launch_stencil_diag_x32(const Geom& g, const double2* dg, Buf<const float2> x,
                                    Buf<double2> y, int nvec, cudaStream_t st) {
  dim3 blk(BX, BY, 1);
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz * nvec);
  count_launch();
  return launch_pdl(k_stencil_diag<false, float2>, grd, blk, 0, st, g, dg, x.p, x.rs, y.p, y.rs,
                    0.0, 0.0);
}

cudaError_t launch_stencil_diag_ff(const Geom& g, const double2* dg, Buf<const double2> x,
                                   Buf<float4> y, int nvec, cudaStream_t st) {
  dim3 blk(BX, BY, 1);
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz * nvec);
  count_launch();
  return launch_pdl(k_stencil_diag<true, double2>, grd, blk, 0, st, g, dg, x.p, x.rs,
                    reinterpret_cast<double2*>(y.p), y.rs, 0.0, 0.0);
}

cudaError_t launch_scale(Buf<double2> dst, Buf<const double2> src, long long n, const GmresDev& gs,
                         int nvec, cudaStream_t st) {
  count_launch();
  return launch_pdl(k_scale, dim3(ew_blocks(n), nvec), 256, 0, st, dst.p, dst.rs, src.p, src.rs, n,
                    gs);
}

cudaError_t launch_combine(Buf<double2> out, const double2* B, long long bis, long long brs,
                           const GmresDev& gs, Buf<const double2> E, int e_slot, int accumulate,
                           long long n, int nvec, int kmax, cudaStream_t st) {
  (void)kmax;
  count_launch();
  return launch_pdl(k_combine<double2>, dim3(ew_blocks(n), nvec), 256, 0, st, out.p, out.rs, B, bis,
                    brs, gs, E.p, E.rs, e_slot >= 0 ? 1 : 0, accumulate, n);
}

cudaError_t launch_combine_b32(Buf<double2> out, const float2* B, long long bis, long long brs,
                               const GmresDev& gs, int accumulate, long long n, int nvec,
                               cudaStream_t st) {
  count_launch();
  return launch_pdl(k_combine<float2>, dim3(ew_blocks(n), nvec), 256, 0, st, out.p, out.rs, B, bis,
                    brs, gs, (const double2*)nullptr, 0LL, 0, accumulate, n);
}

cudaError_t prepare_kernels(int mmax) {
  const int M = mmax > 0 ? mmax : 1;
  const size_t smem = sizeof(double2) * ((size_t)M * (M + 1) / 2 + M);
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_backsolve(const GmresDev& gs, int nvec, cudaStream_t st) {
  const int M = gs.mmax > 0 ? gs.mmax : 1;
  const size_t smem = sizeof(double2) * ((size_t)M * (M + 1) / 2 + M);
  count_launch();
  return launch_pdl(k_backsolve, nvec, 256, smem, st, gs, nvec);
}

cudaError_t launch_residual_start(const Geom& g, const double* m, Buf<const double2> f, double fs,
                                  Buf<const double2> x, Buf<double2> v0, const GmresDev& gs,
                                  double2* partial, unsigned* counters, int nvec,
                                  cudaStream_t st) {
  count_launch();
  return launch_pdl(k_residual_start, dim3(red_blocks(g.n), nvec), RED_THREADS, 0, st, g, m, f.p,
                    f.rs, fs, x.p, x.rs, v0.p, v0.rs, gs, partial, counters);
}

cudaError_t launch_fci_step(Buf<const double2> Aw, Buf<const double2> r, Buf<double2> v0,
                            const GmresDev& gs, double2* partial, unsigned* counters,
                            long long n, int nvec, cudaStream_t st) {
  dim3 grd(red_blocks(n), nvec);
  count_launch();
  const cudaError_t e = launch_pdl(k_fci_dots, grd, RED_THREADS, 0, st, Aw.p, Aw.rs, r.p, r.rs, n,
                                   gs, partial, counters);
  if (e != cudaSuccess) return e;
  count_launch();
  return launch_pdl(k_fci_start, grd, RED_THREADS, 0, st, Aw.p, Aw.rs, r.p, r.rs, v0.p, v0.rs, n,
                    gs, partial, counters);
}

}  // namespace hz
