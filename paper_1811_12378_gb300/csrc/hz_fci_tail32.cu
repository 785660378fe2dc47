// The tail of one complex64 FCI application (Algorithm 1 steps 3-5) as one cooperative kernel:
// the step size d = (Aw)^H r / ||Aw||^2, g = r - d Aw, k_in steps of GMRES on A v = g (CGS2
// Arnoldi, Givens rotations), the triangular solve and out = V y + d w.
//
// At the grid sizes where the solver is launch- and latency-bound (64^3: every field in L2),
// the multi-kernel form of this tail is about 24 dependent launches whose time is mostly ramp
// and the serial finish of each reduction.  Here the grid stays resident: each block owns a
// contiguous range of points and each of its threads a fixed set in it, phases are separated
// by a grid barrier, and
// after each barrier every block reads all blocks' partial sums (float pairs) and computes the
// same scalars (d, beta, the Hessenberg column, the Givens rotation, y) redundantly in float32,
// so no scalar has to be broadcast through memory and no further barrier is spent on it.
// Fields written inside the kernel are read with ordinary loads (never the read-only path): the
// grid barrier's acquire makes the other blocks' writes visible to them.
// The next basis vector is published unnormalised (scratch field W) together with its norm's
// reduction, and the stencil of the next step scales A W by 1/h: that saves the barrier a
// normalised copy would need (3 barriers per Arnoldi step, 2 for step d and beta).
//
// The barrier spins with a bound (about a second); a block that gives up sets the error flag
// and returns, the others then skip their waits, and the host reports the flag after the
// solve.  One right-hand side, k_in <= TAIL_KMAX (instances for k_in <= 4 and <= 16).
#include <cuda_runtime.h>

#include <algorithm>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int TB = 256;  // threads per block

struct Tail {
  Geom g;
  const float2* dg;    // complex64 diagonal
  const float2* w32;   // quadrature sum rounded to complex64
  const float2* f32;   // r (the FCI input) in complex64
  const double2* w64;  // quadrature sum in float64
  float2* V;           // inner basis, kin + 1 fields of n
  float2* W;           // scratch field: the next basis vector before its normalisation
  double2* out;        // FCI output
  float4* part;        // [slots][gridDim.x] block partial sums
  unsigned* bar;       // barrier counter and generation
  int* err;
  long long n;
  int kin;
  int pyth;  // 0: always sum the norm after the second Gram-Schmidt pass
  float brk;
};

// The partial sums of phase q live in half (q & 1) of the partial buffer, (KC + 2) slots of G
// blocks each: a block that has passed barrier q + 1 writes phase q + 2 while no block can
// still be reading phase q (every block finished that reduction before arriving at q + 1),
// whereas one shared area would let a fast block overwrite sums a slow block is still adding.
template <int KC>
__device__ __forceinline__ float4* part_of(const Tail& a, int q) {
  return a.part + (long long)(q & 1) * (KC + 2) * gridDim.x;
}

// Block partial of ns complex slots: the threads' values in v[0..ns) are summed over the warp
// (butterfly, 8 at a time), over the block's warps as float pairs, and written to
// part[s * G + block].
// wsum has (TB / 32) rows of LDW entries.
template <int NS, int LDW>
__device__ __forceinline__ void block_partial(float4* part, float2 (&v)[NS], int ns,
                                              float2* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int b0 = 0; b0 < NS; b0 += 8) {
    if (b0 < ns) {  // uniform over the block
      float2 acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        acc[t] = (b0 + t < NS && b0 + t < ns) ? v[b0 + t < NS ? b0 + t : 0] : make_float2(0.f, 0.f);
      const float2 red = warp_reduce8f(acc, lane);
      if ((lane & 3) == 0) {
        const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (b0 + t < ns) wsum[warp * LDW + b0 + t] = red;
      }
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += TB) {
    float4 t = ffc_of(wsum[s]);
    for (int w = 1; w < TB / 32; ++w) t = ffc_add(t, ffc_of(wsum[w * LDW + s]));
    part[(long long)s * gridDim.x + blockIdx.x] = t;
  }
}

// After the barrier: every block sums all blocks' partials of ns slots into hs[] (float32).
__device__ __forceinline__ void grid_reduce(const float4* part, int ns, float2* hs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = warp; s < ns; s += TB / 32) {
    const float4 t = warp_sum_partials_ffn(part, s, (int)gridDim.x, lane);
    if (lane == 0) hs[s] = f_from_ffc(t);
  }
  __syncthreads();
}

template <int PPT, int KC>
__global__ void __launch_bounds__(TB) k_fci_tail32(Tail a) {
  pdl_enter();
  constexpr int LDW = KC + 8;
  __shared__ float2 wsum[(TB / 32) * LDW];
  __shared__ float2 hs[KC + 2], h1s[KC + 2];
  __shared__ float2 R[(KC + 1) * KC];  // rotated Hessenberg, column c at c * (KC + 1)
  __shared__ float csn[KC];
  __shared__ float2 snn[KC], gg[KC + 1], ys[KC];
  __shared__ float2 dsh;
  __shared__ float inv_s;
  __shared__ int kend_s, stop_s, fast_s;
  const Geom& g = a.g;
  const long long n = a.n;
  // block b owns the points [b n / G, (b + 1) n / G), its thread t the points begin + t + e * TB
  const long long T = TB;
  const long long pbeg = (long long)blockIdx.x * a.n / gridDim.x;
  const long long pend = (long long)(blockIdx.x + 1) * a.n / gridDim.x;
  const long long t0 = pbeg + threadIdx.x;
  const unsigned G = gridDim.x;
  const float2 zero = make_float2(0.f, 0.f);
  const float cs = g.csf;
  const long long sxy = (long long)g.nx * g.ny;

  // grid coordinates of this thread's points (n < 2^31)
  int ci[PPT], cj[PPT], ck[PPT];
#pragma unroll
  for (int e = 0; e < PPT; ++e) {
    const long long p = t0 + e * T;
    const int pi = p < pend ? int(p) : 0;
    const int nxy = g.nx * g.ny;
    ck[e] = pi / nxy;
    const int rem = pi - ck[e] * nxy;
    cj[e] = rem / g.nx;
    ci[e] = rem - cj[e] * g.nx;
  }

  // (A x)(p) for own point e, from a field x written earlier in this kernel or before it
  auto apply = [&](const float2* x, int e, long long p, bool in_kernel) -> float2 {
    const int i = ci[e], j = cj[e], k = ck[e];
    auto ld = [&](long long q) { return in_kernel ? x[q] : __ldg(x + q); };
    const float2 xc = ld(p);
    const float2 xm = i > 0 ? ld(p - 1) : zero, xp = i < g.nx - 1 ? ld(p + 1) : zero;
    const float2 ym = j > 0 ? ld(p - g.nx) : zero, yp = j < g.ny - 1 ? ld(p + g.nx) : zero;
    const float2 zm = k > 0 ? ld(p - sxy) : zero, zp = k < g.nz - 1 ? ld(p + sxy) : zero;
    const float2 d = __ldg(a.dg + p);
    const float nbx = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
    const float nby = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
    return make_float2(d.x * xc.x - d.y * xc.y - cs * nbx, d.x * xc.y + d.y * xc.x - cs * nby);
  };

  // ---- step 3: Aw and d = (Aw)^H r / ||Aw||^2
  float2 aw[PPT], rv[PPT], wv[PPT];
  {
    float2 v[2] = {zero, zero};
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      const long long p = t0 + e * T;
      aw[e] = zero;
      rv[e] = zero;
      if (p < pend) {
        aw[e] = apply(a.w32, e, p, false);
        rv[e] = __ldg(a.f32 + p);
        v[0].x = fmaf(aw[e].x, rv[e].x, fmaf(aw[e].y, rv[e].y, v[0].x));
        v[0].y = fmaf(aw[e].x, rv[e].y, fmaf(-aw[e].y, rv[e].x, v[0].y));
        v[1].x = fmaf(aw[e].x, aw[e].x, fmaf(aw[e].y, aw[e].y, v[1].x));
      }
    }
    block_partial<2, LDW>(part_of<KC>(a, 0), v, 2, wsum);
  }
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce(part_of<KC>(a, 0), 2, hs);
  if (threadIdx.x == 0) {
    const float den = hs[1].x;
    dsh = den != 0.f ? make_float2(hs[0].x / den, hs[0].y / den) : zero;
  }
  __syncthreads();
  const float2 d = dsh;

  // ---- v0 = (r - d Aw) / beta
  {
    float2 v[1] = {zero};
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      wv[e] = make_float2(rv[e].x - (d.x * aw[e].x - d.y * aw[e].y),
                          rv[e].y - (d.x * aw[e].y + d.y * aw[e].x));
      v[0].x = fmaf(wv[e].x, wv[e].x, fmaf(wv[e].y, wv[e].y, v[0].x));
    }
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      const long long p = t0 + e * T;
      if (p < pend) a.W[p] = wv[e];
    }
    block_partial<1, LDW>(part_of<KC>(a, 1), v, 1, wsum);
  }
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce(part_of<KC>(a, 1), 1, hs);
  if (threadIdx.x == 0) {
    const float beta = sqrtf(hs[0].x);
    gg[0] = make_float2(beta, 0.f);
    inv_s = beta > 0.f ? 1.f / beta : 0.f;
    kend_s = 0;
    stop_s = beta > 0.f ? 0 : 1;
  }
  __syncthreads();
  {
    const float inv = inv_s;
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      const long long p = t0 + e * T;
      if (p < pend) a.V[p] = make_float2(wv[e].x * inv, wv[e].y * inv);
    }
  }

  // Givens step for column j with h_{j+1,j} = hn (thread 0; the same arithmetic as the
  // multi-kernel float32 form)
  auto givens = [&](int j, float hn) {
    const float wn = sqrtf(h1s[j + 1].x);
    float2* col = R + j * (KC + 1);
    for (int i = 0; i <= j; ++i) col[i] = h1s[i];
    for (int i = 0; i < j; ++i) {
      const float c = csn[i];
      const float2 s = snn[i], x = col[i], y = col[i + 1];
      col[i] = make_float2(c * x.x + (s.x * y.x - s.y * y.y), c * x.y + (s.x * y.y + s.y * y.x));
      col[i + 1] = make_float2(-(s.x * x.x + s.y * x.y) + c * y.x, -(s.x * x.y - s.y * x.x) + c * y.y);
    }
    float c;
    float2 s;
    const float2 x = col[j];
    if (hn == 0.f) {
      c = 1.f;
      s = zero;
    } else if (x.x == 0.f && x.y == 0.f) {
      c = 0.f;
      s = make_float2(1.f, 0.f);
    } else {
      const float ra = hypotf(x.x, x.y);
      const float rr = hypotf(ra, hn);
      c = ra / rr;
      s = make_float2(x.x / ra * hn / rr, x.y / ra * hn / rr);
    }
    col[j] = make_float2(c * x.x + s.x * hn, c * x.y + s.y * hn);
    csn[j] = c;
    snn[j] = s;
    const float2 gk = gg[j];
    gg[j] = make_float2(c * gk.x, c * gk.y);
    gg[j + 1] = make_float2(-(s.x * gk.x + s.y * gk.y), -(s.x * gk.y - s.y * gk.x));
    const bool brk_now = hn <= a.brk * wn;
    inv_s = brk_now ? 0.f : 1.f / hn;
    kend_s = j + 1;
    stop_s = brk_now ? 1 : 0;
  };

  // ---- inner GMRES (Algorithm 1 step 4), CGS2 Arnoldi with Givens rotations
  for (int j = 0; j < a.kin && !stop_s; ++j) {
    const float invj = inv_s;  // v_j = W / h: W is complete since the last barrier
    const int nb = j + 1;
    // w = A v_j, first pass h1 = V^H w, ||w||^2
    {
      float2 v[KC + 2];
#pragma unroll
      for (int s = 0; s < KC + 2; ++s) v[s] = zero;
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + e * T;
        wv[e] = zero;
        if (p < pend) {
          const float2 aw_ = apply(a.W, e, p, true);
          wv[e] = make_float2(aw_.x * invj, aw_.y * invj);
#pragma unroll
          for (int b = 0; b < KC + 1; ++b) {
            if (b < nb) {
              const float2 vb = a.V[(long long)b * n + p];
              v[b].x = fmaf(vb.x, wv[e].x, fmaf(vb.y, wv[e].y, v[b].x));
              v[b].y = fmaf(vb.x, wv[e].y, fmaf(-vb.y, wv[e].x, v[b].y));
            }
          }
          v[KC + 1].x = fmaf(wv[e].x, wv[e].x, fmaf(wv[e].y, wv[e].y, v[KC + 1].x));
        }
      }
#pragma unroll
      for (int s = 0; s < KC + 1; ++s)
        if (s == nb) v[s] = v[KC + 1];  // the norm goes to slot nb
      block_partial<KC + 2, LDW>(part_of<KC>(a, 3 * j + 2), v, nb + 1, wsum);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce(part_of<KC>(a, 3 * j + 2), nb + 1, h1s);
    // w -= V h1, second pass h2 = V^H w and ||w||^2 (slot nb)
    {
      float2 v[KC + 2];
#pragma unroll
      for (int s = 0; s < KC + 2; ++s) v[s] = zero;
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + e * T;
        if (p < pend) {
          float2 vb[KC + 1];
#pragma unroll
          for (int b = 0; b < KC + 1; ++b)
            vb[b] = b < nb ? a.V[(long long)b * n + p] : zero;
#pragma unroll
          for (int b = 0; b < KC + 1; ++b) {
            if (b < nb) {
              const float2 h = h1s[b];
              wv[e].x = fmaf(-h.x, vb[b].x, fmaf(h.y, vb[b].y, wv[e].x));
              wv[e].y = fmaf(-h.x, vb[b].y, fmaf(-h.y, vb[b].x, wv[e].y));
            }
          }
#pragma unroll
          for (int b = 0; b < KC + 1; ++b) {
            if (b < nb) {
              v[b].x = fmaf(vb[b].x, wv[e].x, fmaf(vb[b].y, wv[e].y, v[b].x));
              v[b].y = fmaf(vb[b].x, wv[e].y, fmaf(-vb[b].y, wv[e].x, v[b].y));
            }
          }
          v[KC + 1].x = fmaf(wv[e].x, wv[e].x, fmaf(wv[e].y, wv[e].y, v[KC + 1].x));
        }
      }
#pragma unroll
      for (int s = 0; s < KC + 1; ++s)
        if (s == nb) v[s] = v[KC + 1];
      block_partial<KC + 2, LDW>(part_of<KC>(a, 3 * j + 3), v, nb + 1, wsum);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce(part_of<KC>(a, 3 * j + 3), nb + 1, hs);
    // the Hessenberg column h1 + h2 (hs keeps h2 for the last pass)
    if (threadIdx.x <= j) {
      const float2 h2 = hs[threadIdx.x];
      h1s[threadIdx.x] = make_float2(h1s[threadIdx.x].x + h2.x, h1s[threadIdx.x].y + h2.y);
    }
    __syncthreads();
    // h_{j+1,j}^2 = ||w||^2 - ||h2||^2 for the w of this pass: V is orthonormal and w already
    // nearly orthogonal to it, so the last pass removes little and the difference keeps its
    // accuracy, and no reduction of ||w - V h2||^2 is needed.  Where the last pass removes more
    // than three quarters of ||w||^2 (the difference would cancel) that norm is summed.  Every
    // block computes the same scalars, so the branch is uniform over the grid.
    if (threadIdx.x == 0) {
      float q = 0.f;
      for (int b = 0; b <= j; ++b) q = fmaf(hs[b].x, hs[b].x, fmaf(hs[b].y, hs[b].y, q));
      const float wq = hs[nb].x, hp = wq - q;
      fast_s = a.pyth && hp > 0.25f * wq ? 1 : 0;
      if (fast_s) givens(j, sqrtf(hp));
    }
    __syncthreads();
    const bool fast = fast_s;
    const bool more = j + 1 < a.kin;
    // w -= V h2 (and ||w||^2 where it is summed)
    {
      float2 v[1] = {zero};
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + e * T;
        if (p < pend) {
#pragma unroll
          for (int b = 0; b < KC + 1; ++b) {
            if (b < nb) {
              const float2 vb = a.V[(long long)b * n + p];
              const float2 h = hs[b];
              wv[e].x = fmaf(-h.x, vb.x, fmaf(h.y, vb.y, wv[e].x));
              wv[e].y = fmaf(-h.x, vb.y, fmaf(-h.y, vb.x, wv[e].y));
            }
          }
          v[0].x = fmaf(wv[e].x, wv[e].x, fmaf(wv[e].y, wv[e].y, v[0].x));
          // every read of W in this step came before the first barrier
          if (!fast || more) a.W[p] = wv[e];
        }
      }
      if (!fast) block_partial<1, LDW>(part_of<KC>(a, 3 * j + 4), v, 1, wsum);
    }
    if (fast) {
      // v_{j+1} now; the barrier only where a next step's stencil reads W
      if (!stop_s && more) {
        const float inv = inv_s;
        float2* vn = a.V + (long long)(j + 1) * n;
#pragma unroll
        for (int e = 0; e < PPT; ++e) {
          const long long p = t0 + e * T;
          if (p < pend) vn[p] = make_float2(wv[e].x * inv, wv[e].y * inv);
        }
        if (!grid_sync(a.bar, G, a.err)) return;
      }
      continue;
    }
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce(part_of<KC>(a, 3 * j + 4), 1, hs);
    if (threadIdx.x == 0) givens(j, sqrtf(hs[0].x));
    __syncthreads();
    if (!stop_s && more) {
      const float inv = inv_s;
      float2* vn = a.V + (long long)(j + 1) * n;
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + e * T;
        if (p < pend) vn[p] = make_float2(wv[e].x * inv, wv[e].y * inv);
      }
    }
  }

  // ---- y = R^{-1} g (float32, every block the same), out = V y + d w (Algorithm 1 step 5)
  if (threadIdx.x == 0) {
    const int kk = kend_s;
    for (int i = kk - 1; i >= 0; --i) {
      float2 sacc = gg[i];
      for (int c = i + 1; c < kk; ++c) {
        const float2 r = R[c * (KC + 1) + i], y = ys[c];
        sacc = make_float2(sacc.x - (r.x * y.x - r.y * y.y), sacc.y - (r.x * y.y + r.y * y.x));
      }
      const float2 dd = R[i * (KC + 1) + i];
      const float den = dd.x * dd.x + dd.y * dd.y;
      ys[i] = make_float2((sacc.x * dd.x + sacc.y * dd.y) / den, (sacc.y * dd.x - sacc.x * dd.y) / den);
    }
  }
  __syncthreads();
  const int kk = kend_s;
  const double2 dd = make_double2(double(d.x), double(d.y));
#pragma unroll
  for (int e = 0; e < PPT; ++e) {
    const long long p = t0 + e * T;
    if (p < pend) {
      float2 v = zero;
      for (int b = 0; b < kk; ++b) {
        const float2 vb = a.V[(long long)b * n + p], y = ys[b];
        v = make_float2(v.x + (y.x * vb.x - y.y * vb.y), v.y + (y.x * vb.y + y.y * vb.x));
      }
      const double2 ew = __ldg(a.w64 + p);
      a.out[p] = make_double2(double(v.x) + (dd.x * ew.x - dd.y * ew.y),
                              double(v.y) + (dd.x * ew.y + dd.y * ew.x));
    }
  }
}

template <int PPT, int KC>
cudaError_t occupancy_of(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fci_tail32<PPT, KC>, TB,
                                                       0);
}

template <int KC>
cudaError_t occupancy_kc(int p, int* per_sm) {
  switch (p) {
    case 1: return occupancy_of<1, KC>(per_sm);
    case 2: return occupancy_of<2, KC>(per_sm);
    case 4: return occupancy_of<4, KC>(per_sm);
    default: return occupancy_of<8, KC>(per_sm);
  }
}

template <int KC>
cudaError_t launch_kc(const cudaLaunchConfig_t& cfg, int ppt, const Tail& a) {
  switch (ppt) {
    case 1: return cudaLaunchKernelEx(&cfg, k_fci_tail32<1, KC>, a);
    case 2: return cudaLaunchKernelEx(&cfg, k_fci_tail32<2, KC>, a);
    case 4: return cudaLaunchKernelEx(&cfg, k_fci_tail32<4, KC>, a);
    case 8: return cudaLaunchKernelEx(&cfg, k_fci_tail32<8, KC>, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t fci_tail32_plan(long long n, int kin, int* ppt, int* blocks) {
  if (n > 0x7fffffffLL) {
    *ppt = 0;
    *blocks = 0;
    return cudaSuccess;
  }
  *ppt = 0;
  *blocks = 0;
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) return e;
  for (int p : {1, 2, 4, 8}) {
    int per_sm = 0;
    e = kin <= 4 ? occupancy_kc<4>(p, &per_sm) : occupancy_kc<TAIL_KMAX>(p, &per_sm);
    if (e != cudaSuccess) return e;
    // at most two blocks per SM: more blocks make every barrier and every reduction of the
    // block partial sums longer (measured at 64^3: 1024 blocks 227 us, 256 blocks 99 us,
    // 128 blocks 118 us per application)
    const long long need = (n + (long long)TB * p - 1) / ((long long)TB * p);
    if (need <= (long long)std::min(per_sm, 2) * sms) {
      *ppt = p;
      *blocks = (int)need;
      return cudaSuccess;
    }
  }
  return cudaSuccess;  // too large for one resident grid: the multi-kernel form serves
}

cudaError_t launch_fci_tail32(const Geom& g, const float2* dg, const float2* w32,
                              const float2* f32, const double2* w64, float2* V, float2* W,
                              double2* out,
                              double2* partial, unsigned* bar, int* err, long long n, int kin,
                              double brk, int pyth, int ppt, int blocks, cudaStream_t st) {
  if (kin > TAIL_KMAX || blocks < 1 || n > 0x7fffffffLL) return cudaErrorInvalidValue;
  Tail a;
  a.g = g;
  a.dg = dg;
  a.w32 = w32;
  a.f32 = f32;
  a.w64 = w64;
  a.V = V;
  a.W = W;
  a.out = out;
  a.part = reinterpret_cast<float4*>(partial);
  a.bar = bar;
  a.err = err;
  a.n = n;
  a.kin = kin;
  a.pyth = pyth;
  a.brk = float(brk);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(TB);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return kin <= 4 ? launch_kc<4>(cfg, ppt, a) : launch_kc<TAIL_KMAX>(cfg, ppt, a);
}

}  // namespace hz
