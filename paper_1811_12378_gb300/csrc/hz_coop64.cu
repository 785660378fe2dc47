// Float64 cooperative kernels of the float64-outer forms (HZ_C128, HZ_MIXED_C64) for one
// right-hand side:
//   * k_arnoldi64: one outer FGMRES Arnoldi step (Section 2, after Algorithm 1): w = A z_k,
//     the two classical Gram-Schmidt passes against v_0..v_k, the Givens step of the new
//     Hessenberg column and v_{k+1} = w / h_{k+1,k};
//   * k_fci_tail64: steps 3-5 of Algorithm 1: the step d = (Aw)^H r / ||Aw||^2, k_in GMRES steps
//     (CGS2, Givens) on A v = r - d A w from v = 0, the triangular solve and out = V y + d w.
// Every value, product and sum is float64: these are the Arnoldi orthogonalisation and the
// Hessenberg/Givens least squares of the float64-outer forms.
//
// At 64^3 the multi-kernel form of these steps is about 16 dependent launches per outer step,
// each a few microseconds of float64 work plus its ramp and the serial finish of its reduction
// by the last block.  Here the grid stays resident, each block owns a contiguous range of
// points (and keeps its part of w in registers or shared memory), and phases are separated by
// the bounded grid barrier of hz_device.cuh.  After each barrier every block adds all blocks'
// partial sums in the same fixed order, so all blocks hold the same scalars without a
// broadcast.  As in the complex64 and float-pair kernels, each h_{j+1,j} comes from
// ||w'||^2 - ||V^H w'||^2 after the second pass (w' the vector after the first) unless that
// difference would cancel, which saves a reduction and a barrier per step.
//
// The barrier gives up after its poll limit; the kernel then returns and the host reports
// HZ_ERR_TIMEOUT.  Partial sums of phase q live in half (q & 1) of the partial buffer: a block
// past barrier q + 1 may write phase q + 2 while no block still reads phase q.
#include <cuda_runtime.h>

#include <algorithm>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int AT = 512;  // outer step: threads per block, one block per SM
constexpr int AW = AT / 32;
constexpr int TT = 256;  // FCI tail: threads per block
constexpr int TW = TT / 32;
constexpr int TKC = 4;   // FCI tail: inner steps k_in <= 4

__device__ __forceinline__ double2 cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(double(v.x), double(v.y)); }

// ((A - 0 I) x)_p in float64 from the diagonal dg = 6 s/h^2 - m - i a (the arithmetic of
// k_stencil_diag); (i, j, k) the grid coordinates of p.
template <typename TX, bool LDG>
__device__ __forceinline__ double2 stencil64(const Geom& g, const double2* dg, const TX* x,
                                             long long p, int i, int j, int k) {
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  auto ld = [&](long long q) { return to_d2(LDG ? __ldg(x + q) : x[q]); };
  const double2 xm = i > 0 ? ld(p - 1) : cz(), xp = i < g.nx - 1 ? ld(p + 1) : cz();
  const double2 ym = j > 0 ? ld(p - sy) : cz(), yp = j < g.ny - 1 ? ld(p + sy) : cz();
  const double2 zm = k > 0 ? ld(p - sz) : cz(), zp = k < g.nz - 1 ? ld(p + sz) : cz();
  const double2 xc = ld(p);
  const double2 d = __ldg(dg + p);
  const double nbx = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
  const double nby = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
  const double mcs = -g.cs;
  return make_double2(fma(d.x, xc.x, fma(-d.y, xc.y, mcs * nbx)),
                      fma(d.x, xc.y, fma(d.y, xc.x, mcs * nby)));
}

__device__ __forceinline__ void coords_of(const Geom& g, long long p, int& i, int& j, int& k) {
  const int pi = int(p);  // n < 2^31
  const int nxy = g.nx * g.ny;
  k = pi / nxy;
  const int rem = pi - k * nxy;
  j = rem / g.nx;
  i = rem - j * g.nx;
}

// acc += conj(v) w
__device__ __forceinline__ void dot_acc(double2& acc, double2 v, double2 w) {
  acc.x = fma(v.x, w.x, fma(v.y, w.y, acc.x));
  acc.y = fma(v.x, w.y, fma(-v.y, w.x, acc.y));
}
// w -= h v
__device__ __forceinline__ void axpy_sub(double2& w, double2 h, double2 v) {
  w.x = fma(-h.x, v.x, fma(h.y, v.y, w.x));
  w.y = fma(-h.x, v.y, fma(-h.y, v.x, w.y));
}

// Every block: h[s] = sum over the G blocks of part[s][b] (fixed order), s < ns.
__device__ __forceinline__ void grid_reduce64(const double2* part, int ns, double2* h, int nwarps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = warp; s < ns; s += nwarps) {
    const double2 t = warp_sum_partials(part, s, (int)gridDim.x, lane);
    if (lane == 0) h[s] = t;
  }
  __syncthreads();
}

// The block's sums of ns slots from wp[warp][slot] (rows of ldw) to part[s][block].
__device__ __forceinline__ void block_partial64(double2* part, const double2* wp, int ldw, int ns,
                                                int nwarps) {
  __syncthreads();
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    double2 t = wp[s];
    for (int w = 1; w < nwarps; ++w) t = cadd(t, wp[w * ldw + s]);
    part[(long long)s * gridDim.x + blockIdx.x] = t;
  }
}

// Store the warp sum of one complex per-thread value into wp[warp][slot].
__device__ __forceinline__ void warp_store(double2 v, double2* wp, int ldw, int slot) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if ((threadIdx.x & 31) == 0) wp[(threadIdx.x >> 5) * ldw + slot] = v;
}

// ================================================================== outer Arnoldi step
struct Arn64 {
  Geom g;
  const double2* dg;
  const void* z;     // z_k: double2, or float2 when z32
  int z32;
  const double2* V;  // v_0..v_{nb-1}, fields of n points
  double2* vnext;    // v_nb
  GmresDev gs;
  double2* part;     // two halves of (mmax + 2) slots x G block partials
  unsigned* bar;
  int* err;
  long long n;
  int nb;
  int pyth;
  double brk;
};

struct Pts {
  long long t0, pend;
  int ppt;
};

// Per-warp sums conj(v_b) w for b < nb (8 fields at a time) into wp[warp][b]; the thread's w at
// sw[e AT + tid].
__device__ __forceinline__ void dots64(const Arn64& a, const Pts& P, const double2* sw,
                                       double2* wp, int ldw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = a.nb;
  for (int b0 = 0; b0 < nb; b0 += 8) {
    double2 acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = cz();
#pragma unroll 1
    for (int e = 0; e < P.ppt; ++e) {
      const long long p = P.t0 + (long long)e * AT;
      if (p >= P.pend) break;
      const double2 w = sw[e * AT + threadIdx.x];
      double2 v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        v[t] = b0 + t < nb ? __ldg(a.V + (long long)(b0 + t) * a.n + p) : cz();
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (b0 + t < nb) dot_acc(acc[t], v[t], w);  // uniform: nb is the same in every thread
    }
    const double2 red = warp_reduce8(acc, lane);
    if ((lane & 3) == 0) {
      const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
      if (b0 + t < nb) wp[warp * ldw + b0 + t] = red;
    }
  }
}

__device__ __forceinline__ void norm64(const Pts& P, const double2* sw, double2* wp, int ldw,
                                       int slot) {
  double q = 0.0;
#pragma unroll 1
  for (int e = 0; e < P.ppt; ++e) {
    if (P.t0 + (long long)e * AT >= P.pend) break;
    const double2 w = sw[e * AT + threadIdx.x];
    q = fma(w.x, w.x, fma(w.y, w.y, q));
  }
  warp_store(make_double2(q, 0.0), wp, ldw, slot);
}

// w -= V h (h[b], b < nb, in shared memory)
__device__ __forceinline__ void update64(const Arn64& a, const Pts& P, double2* sw,
                                         const double2* h) {
  const int nb = a.nb;
#pragma unroll 1
  for (int e = 0; e < P.ppt; ++e) {
    const long long p = P.t0 + (long long)e * AT;
    if (p >= P.pend) break;
    double2 w = sw[e * AT + threadIdx.x];
#pragma unroll 1
    for (int b0 = 0; b0 < nb; b0 += 8) {
      double2 v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        v[t] = b0 + t < nb ? __ldg(a.V + (long long)(b0 + t) * a.n + p) : cz();
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (b0 + t < nb) axpy_sub(w, h[b0 + t], v[t]);
    }
    sw[e * AT + threadIdx.x] = w;
  }
}

__global__ void __launch_bounds__(AT, 1) k_arnoldi64(Arn64 a, int ppt) {
  pdl_enter();
  // sw[ppt][AT] | wp[AW][nb + 8] | h1[nb + 1] | h2[nb + 1]
  extern __shared__ double2 smd[];
  __shared__ double s_inv, s_hn2;
  __shared__ int s_fast;
  if (a.gs.stopped[0]) return;  // uniform: no block of this grid writes it before barrier 1
  const int nb = a.nb, ldw = nb + 8;
  double2* sw = smd;
  double2* wp = sw + ppt * AT;
  double2* h1 = wp + AW * ldw;
  double2* h2 = h1 + nb + 1;
  const unsigned G = gridDim.x;
  const long long n = a.n;
  const long long half = (long long)(a.gs.mmax + 2) * G;
  Pts P;
  P.t0 = (long long)blockIdx.x * n / G + threadIdx.x;
  P.pend = (long long)(blockIdx.x + 1) * n / G;
  P.ppt = ppt;

  // ---- w = A z_k (float64)
#pragma unroll 1
  for (int e = 0; e < ppt; ++e) {
    const long long p = P.t0 + (long long)e * AT;
    if (p >= P.pend) break;
    int i, j, k;
    coords_of(a.g, p, i, j, k);
    sw[e * AT + threadIdx.x] =
        a.z32 ? stencil64<float2, true>(a.g, a.dg, (const float2*)a.z, p, i, j, k)
              : stencil64<double2, true>(a.g, a.dg, (const double2*)a.z, p, i, j, k);
  }
  // ---- first pass: h1 = V^H w, ||w||^2 in slot nb
  dots64(a, P, sw, wp, ldw);
  norm64(P, sw, wp, ldw, nb);
  block_partial64(a.part, wp, ldw, nb + 1, AW);
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce64(a.part, nb + 1, h1, AW);
  // ---- second pass: w -= V h1, then h2 = V^H w, ||w||^2 in slot nb
  update64(a, P, sw, h1);
  dots64(a, P, sw, wp, ldw);
  norm64(P, sw, wp, ldw, nb);
  block_partial64(a.part + half, wp, ldw, nb + 1, AW);
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce64(a.part + half, nb + 1, h2, AW);
  // ---- h_{k+1,k}^2 = ||w'||^2 - ||h2||^2 unless it would cancel (uniform over the grid)
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int b = 0; b < nb; ++b) q = fma(h2[b].x, h2[b].x, fma(h2[b].y, h2[b].y, q));
    const double wq = h2[nb].x, hp = wq - q;
    s_fast = a.pyth && hp > 0.25 * wq ? 1 : 0;
    s_hn2 = hp;
  }
  __syncthreads();
  const double wn2 = h1[nb].x;
  auto set_inv = [&](double hn2) {  // the test and scale of givens_column
    const double hn = sqrt(hn2), wn = sqrt(wn2);
    s_inv = hn <= a.brk * wn ? 0.0 : 1.0 / hn;
  };
  auto store_column = [&](double hn2) {  // block 0: the column for the Givens step
    for (int i = threadIdx.x; i <= nb; i += AT) {
      a.gs.h1[i] = h1[i];
      if (i < nb) a.gs.h2[i] = h2[i];
    }
    if (threadIdx.x == 0) a.gs.nrm[0] = make_double2(hn2, 0.0);
  };
  bool givens_done = false;
  if (s_fast) {
    const double hn2 = s_hn2;
    if (threadIdx.x == 0) set_inv(hn2);
    if (blockIdx.x == 0) store_column(hn2);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < 32) givens_column_warp(a.gs, 0, nb - 1, a.brk);
    givens_done = true;
    update64(a, P, sw, h2);
  } else {
    update64(a, P, sw, h2);
    norm64(P, sw, wp, ldw, 0);
    block_partial64(a.part, wp, ldw, 1, AW);
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce64(a.part, 1, wp, AW);
    const double hn2 = wp[0].x;
    if (threadIdx.x == 0) set_inv(hn2);
    if (blockIdx.x == 0) store_column(hn2);
    __syncthreads();
  }
  const double s = s_inv;
#pragma unroll 1
  for (int e = 0; e < ppt; ++e) {
    const long long p = P.t0 + (long long)e * AT;
    if (p >= P.pend) break;
    const double2 w = sw[e * AT + threadIdx.x];
    a.vnext[p] = make_double2(w.x * s, w.y * s);
  }
  if (blockIdx.x == 0 && !givens_done && threadIdx.x < 32)
    givens_column_warp(a.gs, 0, nb - 1, a.brk);
}

constexpr int ARN_PPT_MAX = 8;

size_t arn64_smem(int nb, int ppt) {
  return sizeof(double2) * ((size_t)ppt * AT + (size_t)AW * (nb + 8) + 2 * (size_t)(nb + 1));
}

// ================================================================== FCI tail
struct Tail64 {
  Geom g;
  const double2* dg;
  const double2* w;  // quadrature sum (float64)
  const double2* r;  // FCI input
  double2* V;        // inner basis, kin + 1 fields of n
  double2* W;        // scratch: the next basis vector before its normalisation
  double2* out;
  double2* part;     // two halves of (TKC + 2) slots x G
  unsigned* bar;
  int* err;
  long long n;
  int kin;
  int pyth;
  double brk;
};

template <int PPT>
__global__ void __launch_bounds__(TT) k_fci_tail64(Tail64 a) {
  pdl_enter();
  constexpr int LDW = TKC + 2;
  __shared__ double2 wsum[TW * LDW];
  __shared__ double2 hs[TKC + 2], h1s[TKC + 2];
  __shared__ double2 R[(TKC + 1) * TKC];
  __shared__ double csn[TKC];
  __shared__ double2 snn[TKC], gg[TKC + 1], ys[TKC];
  __shared__ double2 dsh;
  __shared__ double inv_s;
  __shared__ int kend_s, stop_s, fast_s;
  const Geom& g = a.g;
  const long long n = a.n;
  const long long pbeg = (long long)blockIdx.x * n / gridDim.x;
  const long long pend = (long long)(blockIdx.x + 1) * n / gridDim.x;
  const long long t0 = pbeg + threadIdx.x;
  const unsigned G = gridDim.x;
  const long long half = (long long)(TKC + 2) * G;
  auto part = [&](int q) { return a.part + (q & 1) * half; };
  int ci[PPT], cj[PPT], ck[PPT];
#pragma unroll
  for (int e = 0; e < PPT; ++e) {
    const long long p = t0 + (long long)e * TT;
    coords_of(g, p < pend ? p : 0, ci[e], cj[e], ck[e]);
  }
  // partial sums of ns slots v[0..ns) of this thread -> part(q): one or two slots by
  // shuffle trees, more by the butterfly of warp_reduce8 (18 float64 adds for up to 8 slots
  // against 10 per slot: float64 adds are the scarce instructions here)
  auto partial = [&](double2* v, int ns, int q) {
    if (ns <= 2) {
      for (int s = 0; s < ns; ++s) warp_store(v[s], wsum, LDW, s);
    } else {
      const int lane = threadIdx.x & 31;
      double2 acc[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] = t < ns ? v[t] : cz();
      const double2 red = warp_reduce8(acc, lane);
      if ((lane & 3) == 0) {
        const int t = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        if (t < ns) wsum[(threadIdx.x >> 5) * LDW + t] = red;
      }
    }
    block_partial64(part(q), wsum, LDW, ns, TW);
  };

  // ---- step 3: Aw and d = (Aw)^H r / ||Aw||^2
  double2 aw[PPT], rv[PPT], wv[PPT];
  {
    double2 v[2] = {cz(), cz()};
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      const long long p = t0 + (long long)e * TT;
      aw[e] = rv[e] = cz();
      if (p < pend) {
        aw[e] = stencil64<double2, true>(g, a.dg, a.w, p, ci[e], cj[e], ck[e]);
        rv[e] = __ldg(a.r + p);
        dot_acc(v[0], aw[e], rv[e]);
        v[1].x = fma(aw[e].x, aw[e].x, fma(aw[e].y, aw[e].y, v[1].x));
      }
    }
    partial(v, 2, 0);
  }
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce64(part(0), 2, hs, TW);
  if (threadIdx.x == 0) {
    const double den = hs[1].x;
    dsh = den != 0.0 ? make_double2(hs[0].x / den, hs[0].y / den) : cz();
  }
  __syncthreads();
  const double2 d = dsh;
  // ---- v0 = (r - d Aw) / beta
  {
    double2 v[1] = {cz()};
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      wv[e] = rv[e];
      axpy_sub(wv[e], d, aw[e]);
      v[0].x = fma(wv[e].x, wv[e].x, fma(wv[e].y, wv[e].y, v[0].x));
      const long long p = t0 + (long long)e * TT;
      if (p < pend) a.W[p] = wv[e];
    }
    partial(v, 1, 1);
  }
  if (!grid_sync(a.bar, G, a.err)) return;
  grid_reduce64(part(1), 1, hs, TW);
  if (threadIdx.x == 0) {
    const double beta = sqrt(hs[0].x);
    gg[0] = make_double2(beta, 0.0);
    inv_s = beta > 0.0 ? 1.0 / beta : 0.0;
    kend_s = 0;
    stop_s = beta > 0.0 ? 0 : 1;
  }
  __syncthreads();
  {
    const double inv = inv_s;
#pragma unroll
    for (int e = 0; e < PPT; ++e) {
      const long long p = t0 + (long long)e * TT;
      if (p < pend) a.V[p] = make_double2(wv[e].x * inv, wv[e].y * inv);
    }
  }
  // Givens step of column j with h_{j+1,j} = hn (thread 0; Saad's complex rotations)
  auto givens = [&](int j, double hn) {
    const double wn = sqrt(h1s[j + 1].x);
    double2* col = R + j * (TKC + 1);
    for (int i = 0; i <= j; ++i) col[i] = h1s[i];
    for (int i = 0; i < j; ++i) {
      const double c = csn[i];
      const double2 s = snn[i], x = col[i], y = col[i + 1];
      col[i] = make_double2(c * x.x + (s.x * y.x - s.y * y.y), c * x.y + (s.x * y.y + s.y * y.x));
      col[i + 1] = make_double2(-(s.x * x.x + s.y * x.y) + c * y.x,
                                -(s.x * x.y - s.y * x.x) + c * y.y);
    }
    double c;
    double2 s;
    const double2 x = col[j];
    if (hn == 0.0) {
      c = 1.0;
      s = cz();
    } else if (x.x == 0.0 && x.y == 0.0) {
      c = 0.0;
      s = make_double2(1.0, 0.0);
    } else {
      const double ra = hypot(x.x, x.y), rr = hypot(ra, hn);
      c = ra / rr;
      s = make_double2(x.x / ra * hn / rr, x.y / ra * hn / rr);
    }
    col[j] = make_double2(c * x.x + s.x * hn, c * x.y + s.y * hn);
    csn[j] = c;
    snn[j] = s;
    const double2 gk = gg[j];
    gg[j] = make_double2(c * gk.x, c * gk.y);
    gg[j + 1] = make_double2(-(s.x * gk.x + s.y * gk.y), -(s.x * gk.y - s.y * gk.x));
    const bool brk_now = hn <= a.brk * wn;
    inv_s = brk_now ? 0.0 : 1.0 / hn;
    kend_s = j + 1;
    stop_s = brk_now ? 1 : 0;
  };

  // ---- inner GMRES (Algorithm 1 step 4), CGS2 Arnoldi with Givens rotations
  for (int j = 0; j < a.kin && !stop_s; ++j) {
    const double invj = inv_s;  // v_j = W / h: W is complete since the last barrier
    const int nb = j + 1;
    {  // w = A v_j, first pass h1 = V^H w, ||w||^2 in slot nb
      double2 v[TKC + 2];
#pragma unroll
      for (int s = 0; s < TKC + 2; ++s) v[s] = cz();
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + (long long)e * TT;
        wv[e] = cz();
        if (p < pend) {
          const double2 t = stencil64<double2, false>(g, a.dg, a.W, p, ci[e], cj[e], ck[e]);
          wv[e] = make_double2(t.x * invj, t.y * invj);
#pragma unroll
          for (int b = 0; b < TKC + 1; ++b)
            if (b < nb) dot_acc(v[b], a.V[(long long)b * n + p], wv[e]);
          v[TKC + 1].x = fma(wv[e].x, wv[e].x, fma(wv[e].y, wv[e].y, v[TKC + 1].x));
        }
      }
      v[nb] = v[TKC + 1];
      partial(v, nb + 1, 3 * j + 2);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce64(part(3 * j + 2), nb + 1, h1s, TW);
    {  // w -= V h1, second pass h2 = V^H w, ||w||^2 in slot nb
      double2 v[TKC + 2];
#pragma unroll
      for (int s = 0; s < TKC + 2; ++s) v[s] = cz();
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + (long long)e * TT;
        if (p < pend) {
          double2 vb[TKC + 1];
#pragma unroll
          for (int b = 0; b < TKC + 1; ++b) vb[b] = b < nb ? a.V[(long long)b * n + p] : cz();
#pragma unroll
          for (int b = 0; b < TKC + 1; ++b)
            if (b < nb) axpy_sub(wv[e], h1s[b], vb[b]);
#pragma unroll
          for (int b = 0; b < TKC + 1; ++b)
            if (b < nb) dot_acc(v[b], vb[b], wv[e]);
          v[TKC + 1].x = fma(wv[e].x, wv[e].x, fma(wv[e].y, wv[e].y, v[TKC + 1].x));
        }
      }
      v[nb] = v[TKC + 1];
      partial(v, nb + 1, 3 * j + 3);
    }
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce64(part(3 * j + 3), nb + 1, hs, TW);
    if (threadIdx.x <= j) {  // the Hessenberg column h1 + h2
      const double2 t = hs[threadIdx.x];
      h1s[threadIdx.x] = make_double2(h1s[threadIdx.x].x + t.x, h1s[threadIdx.x].y + t.y);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double q = 0.0;
      for (int b = 0; b <= j; ++b) q = fma(hs[b].x, hs[b].x, fma(hs[b].y, hs[b].y, q));
      const double wq = hs[nb].x, hp = wq - q;
      fast_s = a.pyth && hp > 0.25 * wq ? 1 : 0;
      if (fast_s) givens(j, sqrt(hp));
    }
    __syncthreads();
    const bool fast = fast_s;
    const bool more = j + 1 < a.kin;
    {  // w -= V h2 (and ||w||^2 where it is summed)
      double2 v[1] = {cz()};
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + (long long)e * TT;
        if (p < pend) {
#pragma unroll
          for (int b = 0; b < TKC + 1; ++b)
            if (b < nb) axpy_sub(wv[e], hs[b], a.V[(long long)b * n + p]);
          v[0].x = fma(wv[e].x, wv[e].x, fma(wv[e].y, wv[e].y, v[0].x));
          // every read of W in this step came before the first barrier
          if (!fast || more) a.W[p] = wv[e];
        }
      }
      if (!fast) partial(v, 1, 3 * j + 4);
    }
    if (fast) {
      if (!stop_s && more) {
        const double inv = inv_s;
        double2* vn = a.V + (long long)(j + 1) * n;
#pragma unroll
        for (int e = 0; e < PPT; ++e) {
          const long long p = t0 + (long long)e * TT;
          if (p < pend) vn[p] = make_double2(wv[e].x * inv, wv[e].y * inv);
        }
        if (!grid_sync(a.bar, G, a.err)) return;
      }
      continue;
    }
    if (!grid_sync(a.bar, G, a.err)) return;
    grid_reduce64(part(3 * j + 4), 1, hs, TW);
    if (threadIdx.x == 0) givens(j, sqrt(hs[0].x));
    __syncthreads();
    if (!stop_s && more) {
      const double inv = inv_s;
      double2* vn = a.V + (long long)(j + 1) * n;
#pragma unroll
      for (int e = 0; e < PPT; ++e) {
        const long long p = t0 + (long long)e * TT;
        if (p < pend) vn[p] = make_double2(wv[e].x * inv, wv[e].y * inv);
      }
    }
  }

  // ---- y = R^{-1} g (every block the same), out = V y + d w (Algorithm 1 step 5)
  if (threadIdx.x == 0) {
    const int kk = kend_s;
    for (int i = kk - 1; i >= 0; --i) {
      double2 sacc = gg[i];
      for (int c = i + 1; c < kk; ++c) sacc = csub(sacc, cmul(R[c * (TKC + 1) + i], ys[c]));
      const double2 dd = R[i * (TKC + 1) + i];
      const double den = dd.x * dd.x + dd.y * dd.y;
      ys[i] = make_double2((sacc.x * dd.x + sacc.y * dd.y) / den,
                           (sacc.y * dd.x - sacc.x * dd.y) / den);
    }
  }
  __syncthreads();
  const int kk = kend_s;
#pragma unroll
  for (int e = 0; e < PPT; ++e) {
    const long long p = t0 + (long long)e * TT;
    if (p < pend) {
      double2 v = cmul(d, __ldg(a.w + p));
      for (int b = 0; b < kk; ++b) v = cadd(v, cmul(ys[b], a.V[(long long)b * n + p]));
      a.out[p] = v;
    }
  }
}

template <int PPT>
cudaError_t tail64_occ(int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_fci_tail64<PPT>, TT, 0);
}

}  // namespace

cudaError_t arnoldi64_plan(long long n, int mmax, int* ppt, int* blocks) {
  *ppt = 0;
  *blocks = 0;
  if (n < 1 || n > 0x7fffffffLL || mmax < 1 || mmax > 128) return cudaSuccess;
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) return e;
  const long long gsz = std::min<long long>((long long)sms, (n + AT - 1) / AT);
  const int p = (int)(((n + gsz - 1) / gsz + AT - 1) / AT);
  if (p > ARN_PPT_MAX) return cudaSuccess;  // the multi-kernel form serves
  const size_t smem = arn64_smem(mmax + 1, p);
  if (smem > 227 * 1024) return cudaSuccess;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_arnoldi64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi64, AT, smem);
  if (e != cudaSuccess) return e;
  if ((long long)per_sm * sms < gsz) return cudaSuccess;
  *ppt = p;
  *blocks = (int)gsz;
  return cudaSuccess;
}

cudaError_t launch_arnoldi64(const Geom& g, const double2* dg, const void* z, int z32,
                             const double2* V, double2* vnext, const GmresDev& gs,
                             double2* partial, unsigned* bar, int* err, long long n, int nb,
                             double brk, int pyth, int ppt, int blocks, cudaStream_t st) {
  if (nb < 1 || nb > gs.mmax || blocks < 1 || ppt < 1 || ppt > ARN_PPT_MAX ||
      (long long)blocks * ppt * AT < n || n > 0x7fffffffLL)
    return cudaErrorInvalidValue;
  Arn64 a;
  a.g = g;
  a.dg = dg;
  a.z = z;
  a.z32 = z32;
  a.V = V;
  a.vnext = vnext;
  a.gs = gs;
  a.part = partial;
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
  cfg.dynamicSmemBytes = arn64_smem(nb, ppt);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_arnoldi64, a, ppt);
}

cudaError_t fci_tail64_plan(long long n, int* ppt, int* blocks) {
  *ppt = 0;
  *blocks = 0;
  if (n > 0x7fffffffLL) return cudaSuccess;
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) return e;
  for (int p : {1, 2, 4, 8}) {
    int per_sm = 0;
    switch (p) {
      case 1: e = tail64_occ<1>(&per_sm); break;
      case 2: e = tail64_occ<2>(&per_sm); break;
      case 4: e = tail64_occ<4>(&per_sm); break;
      default: e = tail64_occ<8>(&per_sm); break;
    }
    if (e != cudaSuccess) return e;
    // at most two blocks per SM (more blocks lengthen every barrier and all-blocks sum), and
    // the same number on every SM (float64-bound: the busiest SM sets the time)
    const long long need = (n + (long long)TT * p - 1) / ((long long)TT * p);
    const long long cap = (long long)std::min(per_sm, 2) * sms;
    if (need <= cap) {
      *ppt = p;
      *blocks = (int)std::min<long long>(need <= sms ? need : cap, (n + TT - 1) / TT);
      // points per thread for that grid
      *ppt = (int)((n + (long long)(*blocks) * TT - 1) / ((long long)(*blocks) * TT));
      if (*ppt > 8) {
        *ppt = 0;
        *blocks = 0;
        continue;
      }
      *ppt = *ppt <= 1 ? 1 : (*ppt <= 2 ? 2 : (*ppt <= 4 ? 4 : 8));
      return cudaSuccess;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_fci_tail64(const Geom& g, const double2* dg, const double2* w,
                              const double2* r, double2* V, double2* W, double2* out,
                              double2* partial, unsigned* bar, int* err, long long n, int kin,
                              double brk, int pyth, int ppt, int blocks, cudaStream_t st) {
  if (kin > TKC || kin < 0 || blocks < 1 || n > 0x7fffffffLL ||
      (long long)blocks * ppt * TT < n)
    return cudaErrorInvalidValue;
  Tail64 a;
  a.g = g;
  a.dg = dg;
  a.w = w;
  a.r = r;
  a.V = V;
  a.W = W;
  a.out = out;
  a.part = partial;
  a.bar = bar;
  a.err = err;
  a.n = n;
  a.kin = kin;
  a.pyth = pyth;
  a.brk = brk;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(TT);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  switch (ppt) {
    case 1: return cudaLaunchKernelEx(&cfg, k_fci_tail64<1>, a);
    case 2: return cudaLaunchKernelEx(&cfg, k_fci_tail64<2>, a);
    case 4: return cudaLaunchKernelEx(&cfg, k_fci_tail64<4>, a);
    case 8: return cudaLaunchKernelEx(&cfg, k_fci_tail64<8>, a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hz
