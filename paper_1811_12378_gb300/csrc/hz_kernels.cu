// Device kernels of libhz: the shifted 7-point Helmholtz stencil, the batched stage of the
// polynomial fixed-point scheme with the fused quadrature sum, and the float64 Krylov
// reductions (CGS2 dots, norms, Givens, back substitution, combinations).
//
// Operator (§7.1 eq:stiff-mass, Case One of §3): in normalised units
//     (A - zI) x = cs * (6 x_p - sum of the 6 neighbours) - (m_p + z) x_p - i a_p x_p,
// cs = s/h^2, zero Dirichlet ghosts, a_p = sigma_max (depth_p / layer)^2 m_p in the sponge.
// The sponge depth is recomputed from the grid index, so the only coefficient field read
// from memory is m.
//
// Reductions are deterministic: each block writes its partial sums, the last block to finish
// (atomic ticket) adds them in block order and resets the ticket.
#include <cuda_runtime.h>

#include "hz_internal.h"

namespace hz {

std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

constexpr int BX = 32;  // stencil block: 32 x 4 points of one z-plane
constexpr int BY = 4;

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

template <typename T> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

__device__ __forceinline__ int depth1(int i, int n, int L) {
  int e = min(i, n - 1 - i);
  return max(0, L - e);
}

// Sponge damping a_p = sigma_max * (d/L)^2 * m_p (0 without a layer).
template <typename R>
__device__ __forceinline__ R sponge(const Geom& g, int i, int j, int k, R mp) {
  if (g.layer <= 0) return R(0);
  int d = max(depth1(i, g.nx, g.layer), max(depth1(j, g.ny, g.layer), depth1(k, g.nz, g.layer)));
  R t = R(d) / R(g.layer);
  return (R(g.sig) * (t * t)) * mp;
}

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

// ---------------------------------------------------------------- stencil
template <typename T, typename R>
__global__ void __launch_bounds__(BX * BY)
k_stencil(Geom g, const R* __restrict__ m, const T* __restrict__ x, long long xrs,
          T* __restrict__ y, long long yrs, R zr, R zi) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z % g.nz;
  const int r = blockIdx.z / g.nz;
  if (i >= g.nx || j >= g.ny) return;
  const long long p = i + (long long)g.nx * (j + (long long)g.ny * k);
  const T* xr = x + r * xrs;
  const R mp = m[p];
  const R ap = sponge<R>(g, i, j, k, mp);
  y[r * yrs + p] = apply_point<T, R>(xr[p], nbsum(xr, p, i, j, k, g), R(g.cs), mp, ap, zr, zi);
}

// ---------------------------------------------------------------- polynomial stage
// One stencil sweep of every active node of the scheme eq:fix-pt-exp, all nodes of one
// right-hand side handled by the same thread so that f and m are read once per point.
template <typename T, typename R>
__global__ void __launch_bounds__(BX * BY)
k_poly_stage(Geom g, const R* __restrict__ m, const T* __restrict__ f, long long frs, T* ws,
             long long wrs, double2* __restrict__ w, long long wwrs, const StageArgs a) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z % g.nz;
  const int r = blockIdx.z / g.nz;
  if (i >= g.nx || j >= g.ny) return;
  const long long p = i + (long long)g.nx * (j + (long long)g.ny * k);
  const T fp = f[r * frs + p];
  const R mp = m[p];
  const R ap = sponge<R>(g, i, j, k, mp);
  const R cs = R(g.cs);
  T* wsr = ws + r * wrs;
  double wsx = 0.0, wsy = 0.0;
  for (int q = 0; q < a.nnodes; ++q) {
    const StageNode& nd = a.nd[q];
    const int kind = nd.kind;
    if (kind == SK_NONE) continue;
    const T md = mk(R(nd.mdr), R(nd.mdi));
    const R z0r = R(nd.z0r), z0i = R(nd.z0i);
    T yn;
    bool have_y = false;
    if (kind == SK_FIRST || kind == SK_FIRST_LAST) {
      T yv, kv;
      if (nd.yzero) {
        yv = czero<T>();
        kv = cmul(md, mk(-fp.x, -fp.y));
      } else {
        const T* yin = wsr + nd.in;
        yv = yin[p];
        T Ay = apply_point<T, R>(yv, nbsum(yin, p, i, j, k, g), cs, mp, ap, z0r, z0i);
        kv = cmul(md, csub(Ay, fp));
      }
      if (kind == SK_FIRST) {
        wsr[nd.kout + p] = kv;
        wsr[nd.acc + p] = cadd(yv, kv);
      } else {
        yn = cmul(cadd(yv, kv), mk(R(nd.ipr), R(nd.ipi)));
        have_y = true;
      }
    } else {
      const T* kin = wsr + nd.in;
      T Ak = apply_point<T, R>(kin[p], nbsum(kin, p, i, j, k, g), cs, mp, ap, z0r, z0i);
      T kv = cmul(md, csub(Ak, cmul(mk(R(nd.cfr), R(nd.cfi)), fp)));
      T acc = wsr[nd.acc + p];
      if (kind == SK_MID) {
        wsr[nd.kout + p] = kv;
        wsr[nd.acc + p] = cadd(acc, kv);
      } else {
        yn = cmul(cadd(acc, kv), mk(R(nd.ipr), R(nd.ipi)));
        have_y = true;
      }
    }
    if (have_y) {
      if (a.final_quad) {
        const double yr = double(yn.x), yi = double(yn.y);
        wsx += nd.wqr * yr - nd.wqi * yi;
        wsy += nd.wqr * yi + nd.wqi * yr;
      } else {
        wsr[nd.yout + p] = yn;
      }
    }
  }
  if (a.final_quad) w[r * wwrs + p] = make_double2(wsx, wsy);
}

// ---------------------------------------------------------------- conversions
__global__ void k_c128_to_c64(const double2* __restrict__ x, long long xrs, float2* __restrict__ y,
                              long long yrs, long long n) {
  const int r = blockIdx.y;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 v = x[r * xrs + p];
    y[r * yrs + p] = make_float2(float(v.x), float(v.y));
  }
}

__global__ void k_c64_to_c128(const float2* __restrict__ x, long long xrs, double2* __restrict__ y,
                              long long yrs, long long n) {
  const int r = blockIdx.y;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float2 v = x[r * xrs + p];
    y[r * yrs + p] = make_double2(double(v.x), double(v.y));
  }
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

// Givens step for column k of rhs r (Saad's GMRES with complex rotations).
__device__ void givens_column(const GmresDev& gs, int r, int k, double brk) {
  const int M = gs.mmax;
  const double2* h1 = gs.h1 + (long long)r * (M + 2);
  const double2* h2 = gs.h2 + (long long)r * (M + 2);
  double* sc = gs.scal + (long long)r * SC_COUNT;
  const double hn = sqrt(gs.nrm[2 * r].x);
  const double wn = sqrt(h1[k + 1].x);
  double2* R = gs.R + (long long)r * (M + 1) * M + (long long)k * (M + 1);
  for (int i = 0; i <= k; ++i) R[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
  const double* cc = gs.cc + (long long)r * M;
  const double2* ss = gs.ss + (long long)r * M;
  for (int i = 0; i < k; ++i) {
    const double c = cc[i];
    const double2 s = ss[i], a = R[i], b = R[i + 1];
    R[i] = cadd(mk(c * a.x, c * a.y), cmul(s, b));
    R[i + 1] = cadd(mk(-(s.x * a.x + s.y * a.y), -(s.x * a.y - s.y * a.x)), mk(c * b.x, c * b.y));
  }
  double c;
  double2 s;
  const double2 a = R[k];
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
  R[k] = cadd(mk(c * a.x, c * a.y), mk(s.x * hn, s.y * hn));
  R[k + 1] = make_double2(0.0, 0.0);
  gs.cc[(long long)r * M + k] = c;
  gs.ss[(long long)r * M + k] = s;
  double2* gg = gs.g + (long long)r * (M + 1);
  const double2 gk = gg[k];
  gg[k] = mk(c * gk.x, c * gk.y);
  gg[k + 1] = mk(-(s.x * gk.x + s.y * gk.y), -(s.x * gk.y - s.y * gk.x));
  const double est = hypot(gg[k + 1].x, gg[k + 1].y);
  const bool brk_now = hn <= brk * wn;
  sc[SC_EST] = est;
  sc[SC_HN] = hn;
  sc[SC_INV] = brk_now ? 0.0 : 1.0 / hn;
  gs.kend[r] = k + 1;
  if (brk_now || est <= sc[SC_TOL]) gs.stopped[r] = 1;
}

template <int MODE>
__global__ void __launch_bounds__(RED_THREADS)
k_cgs(const double2* __restrict__ V, long long vis, long long vrs, int nb, double2* w,
      long long wrs, long long n, GmresDev gs, double2* partial, unsigned* counters, double brk) {
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  if (gs.stopped[r]) return;
  const int M = gs.mmax;
  const long long base = (long long)blockIdx.x * RED_CHUNK + threadIdx.x;
  double2* wr = w + r * wrs;
  const double2* Vr = V + r * vrs;
  double2 wv[RED_PPT];
#pragma unroll
  for (int e = 0; e < RED_PPT; ++e) {
    const long long p = base + (long long)e * RED_THREADS;
    wv[e] = p < n ? wr[p] : make_double2(0.0, 0.0);
  }
  if (MODE != 0) {
    const double2* hp = (MODE == 1 ? gs.h1 : gs.h2) + (long long)r * (M + 2);
    for (int b = 0; b < nb; ++b) {
      const double2 h = hp[b];
      const double2* vb = Vr + b * vis;
#pragma unroll
      for (int e = 0; e < RED_PPT; ++e) {
        const long long p = base + (long long)e * RED_THREADS;
        if (p < n) wv[e] = csub(wv[e], cmul(h, vb[p]));
      }
    }
#pragma unroll
    for (int e = 0; e < RED_PPT; ++e) {
      const long long p = base + (long long)e * RED_THREADS;
      if (p < n) wr[p] = wv[e];
    }
  }
  double2* part = partial + (long long)r * (M + 2) * gridDim.x;
  if (MODE != 2) {
    for (int b = 0; b < nb; ++b) {
      const double2* vb = Vr + b * vis;
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int e = 0; e < RED_PPT; ++e) {
        const long long p = base + (long long)e * RED_THREADS;
        if (p < n) s = cadd(s, cmulc(vb[p], wv[e]));
      }
      s = block_sum(s, sh);
      if (threadIdx.x == 0) part[(long long)b * gridDim.x + blockIdx.x] = s;
    }
  }
  if (MODE != 1) {
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < RED_PPT; ++e) s += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
    double2 t = block_sum(make_double2(s, 0.0), sh);
    const int slot = MODE == 0 ? nb : 0;
    if (threadIdx.x == 0) part[(long long)slot * gridDim.x + blockIdx.x] = t;
  }
  if (!last_block(counters + r)) return;
  const int nslots = MODE == 0 ? nb + 1 : (MODE == 1 ? nb : 1);
  double2* out = MODE == 0 ? gs.h1 + (long long)r * (M + 2)
               : MODE == 1 ? gs.h2 + (long long)r * (M + 2) : gs.nrm + 2 * r;
  finish_slots(part, nslots, out, sh);
  if (threadIdx.x == 0) {
    counters[r] = 0;
    if (MODE == 2) givens_column(gs, r, nb - 1, brk);
  }
}

__global__ void k_scale(double2* __restrict__ dst, long long drs, const double2* __restrict__ src,
                        long long srs, long long n, GmresDev gs) {
  const int r = blockIdx.y;
  const double s = gs.scal[(long long)r * SC_COUNT + SC_INV];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[r * srs + p];
    dst[r * drs + p] = make_double2(v.x * s, v.y * s);
  }
}

__global__ void k_combine(double2* out, long long ors, const double2* __restrict__ B, long long bis,
                          long long brs, GmresDev gs, const double2* __restrict__ E, long long ers,
                          int use_e, int accumulate, long long n) {
  const int r = blockIdx.y;
  const int kk = gs.kend[r];
  const double2* y = gs.y + (long long)r * gs.mmax;
  const double* sc = gs.scal + (long long)r * SC_COUNT;
  const double2 d = make_double2(sc[SC_DR], sc[SC_DI]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 acc = accumulate ? out[r * ors + p] : make_double2(0.0, 0.0);
    for (int b = 0; b < kk; ++b) acc = cadd(acc, cmul(y[b], B[r * brs + b * bis + p]));
    if (use_e) acc = cadd(acc, cmul(d, E[r * ers + p]));
    out[r * ors + p] = acc;
  }
}

__global__ void k_backsolve(GmresDev gs, int nvec) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nvec) return;
  const int M = gs.mmax;
  const int kk = gs.kend[r];
  const double2* R = gs.R + (long long)r * (M + 1) * M;
  const double2* g = gs.g + (long long)r * (M + 1);
  double2* y = gs.y + (long long)r * M;
  for (int i = kk - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int jj = i + 1; jj < kk; ++jj) s = csub(s, cmul(R[i + (long long)jj * (M + 1)], y[jj]));
    const double2 d = R[i + (long long)i * (M + 1)];
    const double den = d.x * d.x + d.y * d.y;
    y[i] = make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den);
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
cudaError_t launch_stencil(const Geom& g, const R* m, Buf<const T> x, Buf<T> y, int nvec,
                           double zr, double zi, cudaStream_t st) {
  dim3 blk(BX, BY, 1);
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz * nvec);
  count_launch();
  k_stencil<T, R><<<grd, blk, 0, st>>>(g, m, x.p, x.rs, y.p, y.rs, R(zr), R(zi));
  return cudaGetLastError();
}

template cudaError_t launch_stencil<float2, float>(const Geom&, const float*, Buf<const float2>,
                                                   Buf<float2>, int, double, double, cudaStream_t);
template cudaError_t launch_stencil<double2, double>(const Geom&, const double*,
                                                     Buf<const double2>, Buf<double2>, int,
                                                     double, double, cudaStream_t);

template <typename T, typename R>
cudaError_t launch_poly_stage(const Geom& g, const R* m, Buf<const T> f, T* ws, long long wrs,
                              Buf<double2> w, int nvec, const StageArgs& a, cudaStream_t st) {
  dim3 blk(BX, BY, 1);
  dim3 grd((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz * nvec);
  count_launch();
  k_poly_stage<T, R><<<grd, blk, 0, st>>>(g, m, f.p, f.rs, ws, wrs, w.p, w.rs, a);
  return cudaGetLastError();
}

template cudaError_t launch_poly_stage<float2, float>(const Geom&, const float*, Buf<const float2>,
                                                      float2*, long long, Buf<double2>, int,
                                                      const StageArgs&, cudaStream_t);
template cudaError_t launch_poly_stage<double2, double>(const Geom&, const double*,
                                                        Buf<const double2>, double2*, long long,
                                                        Buf<double2>, int, const StageArgs&,
                                                        cudaStream_t);

cudaError_t launch_convert_c128_c64(Buf<const double2> x, Buf<float2> y, long long n, int nvec,
                                    cudaStream_t st) {
  count_launch();
  k_c128_to_c64<<<dim3(ew_blocks(n), nvec), 256, 0, st>>>(x.p, x.rs, y.p, y.rs, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_c64_c128(Buf<const float2> x, Buf<double2> y, long long n, int nvec,
                                    cudaStream_t st) {
  count_launch();
  k_c64_to_c128<<<dim3(ew_blocks(n), nvec), 256, 0, st>>>(x.p, x.rs, y.p, y.rs, n);
  return cudaGetLastError();
}

cudaError_t launch_cgs(int mode, const double2* V, long long vis, long long vrs, int nb,
                       Buf<double2> w, long long n, const GmresDev& gs, double2* partial,
                       unsigned* counters, int nvec, double breakdown, cudaStream_t st) {
  dim3 grd(red_blocks(n), nvec);
  count_launch();
  if (mode == 0)
    k_cgs<0><<<grd, RED_THREADS, 0, st>>>(V, vis, vrs, nb, w.p, w.rs, n, gs, partial, counters,
                                          breakdown);
  else if (mode == 1)
    k_cgs<1><<<grd, RED_THREADS, 0, st>>>(V, vis, vrs, nb, w.p, w.rs, n, gs, partial, counters,
                                          breakdown);
  else
    k_cgs<2><<<grd, RED_THREADS, 0, st>>>(V, vis, vrs, nb, w.p, w.rs, n, gs, partial, counters,
                                          breakdown);
  return cudaGetLastError();
}

cudaError_t launch_scale(Buf<double2> dst, Buf<const double2> src, long long n, const GmresDev& gs,
                         int nvec, cudaStream_t st) {
  count_launch();
  k_scale<<<dim3(ew_blocks(n), nvec), 256, 0, st>>>(dst.p, dst.rs, src.p, src.rs, n, gs);
  return cudaGetLastError();
}

cudaError_t launch_combine(Buf<double2> out, const double2* B, long long bis, long long brs,
                           const GmresDev& gs, Buf<const double2> E, int e_slot, int accumulate,
                           long long n, int nvec, int kmax, cudaStream_t st) {
  (void)kmax;
  count_launch();
  k_combine<<<dim3(ew_blocks(n), nvec), 256, 0, st>>>(out.p, out.rs, B, bis, brs, gs, E.p, E.rs,
                                                      e_slot >= 0 ? 1 : 0, accumulate, n);
  return cudaGetLastError();
}

cudaError_t launch_backsolve(const GmresDev& gs, int nvec, cudaStream_t st) {
  count_launch();
  k_backsolve<<<(nvec + 31) / 32, 32, 0, st>>>(gs, nvec);
  return cudaGetLastError();
}

cudaError_t launch_residual_start(const Geom& g, const double* m, Buf<const double2> f, double fs,
                                  Buf<const double2> x, Buf<double2> v0, const GmresDev& gs,
                                  double2* partial, unsigned* counters, int nvec,
                                  cudaStream_t st) {
  count_launch();
  k_residual_start<<<dim3(red_blocks(g.n), nvec), RED_THREADS, 0, st>>>(
      g, m, f.p, f.rs, fs, x.p, x.rs, v0.p, v0.rs, gs, partial, counters);
  return cudaGetLastError();
}

cudaError_t launch_fci_step(Buf<const double2> Aw, Buf<const double2> r, Buf<double2> v0,
                            const GmresDev& gs, double2* partial, unsigned* counters,
                            long long n, int nvec, cudaStream_t st) {
  dim3 grd(red_blocks(n), nvec);
  count_launch();
  k_fci_dots<<<grd, RED_THREADS, 0, st>>>(Aw.p, Aw.rs, r.p, r.rs, n, gs, partial, counters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  k_fci_start<<<grd, RED_THREADS, 0, st>>>(Aw.p, Aw.rs, r.p, r.rs, v0.p, v0.rs, n, gs, partial,
                                           counters);
  return cudaGetLastError();
}

}  // namespace hz
