// Case Two of Section 3 (eq:mat-2x2): the double-size coefficient matrix iC - I acting on
// stacked fields x = (x1; x2), with C = [[0, I], [-(A1 + I), -A2]] and A = A1 - i A2 the
// normalised operator of Section 7.1.  From the diagonal dg = 6 s/h^2 - m - i a the two parts
// are A1 x1 = Re(dg) x1 - (s/h^2) (sum of the 6 neighbours of x1) and A2 = -Im(dg), so
//     y1 = i x2 - x1 - z x1,
//     y2 = -i (A1 x1 + x1) - i A2 x2 - x2 - z x2,
// and (iC - I)(iu; u) = (0; f) exactly when A u = f.  One thread per point, the neighbours of
// x1 read from memory.  The solver of this form (float64) runs the polynomial scheme
// eq:fix-pt-exp on iC - I at the Case Two contour's nodes (k_poly_stage_2x2, then the
// quadrature sum k_quad_2x2) and the generic float64 Krylov kernels on fields of 2n points.
#include <cuda_runtime.h>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

template <typename T, typename R>
__global__ void k_apply_2x2(Geom g, const T* __restrict__ dg, const T* __restrict__ x,
                            long long xrs, T* __restrict__ y, long long yrs, R zr, R zi, R cs) {
  pdl_enter();
  const long long n = g.n;
  const int r = blockIdx.y;
  const T* x1 = x + xrs * r;
  const T* x2 = x1 + n;
  T* y1 = y + yrs * r;
  T* y2 = y1 + n;
  const int nxy = g.nx * g.ny;
  const long long sy = g.nx, sz = nxy;
  const T zero = czero<T>();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int pi = int(p);  // n < 2^31 (checked by the launcher)
    const int k = pi / nxy;
    const int rem = pi - k * nxy;
    const int j = rem / g.nx;
    const int i = rem - j * g.nx;
    const T xm = i > 0 ? x1[p - 1] : zero, xp = i < g.nx - 1 ? x1[p + 1] : zero;
    const T ym = j > 0 ? x1[p - sy] : zero, yp = j < g.ny - 1 ? x1[p + sy] : zero;
    const T zm = k > 0 ? x1[p - sz] : zero, zp = k < g.nz - 1 ? x1[p + sz] : zero;
    const R nbr = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
    const R nbi = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
    const T d = dg[p], a = x1[p], b = x2[p];
    // u = A1 x1 + x1
    const R ur = d.x * a.x - cs * nbr + a.x, ui = d.x * a.y - cs * nbi + a.y;
    y1[p] = mk(-b.y - a.x - (zr * a.x - zi * a.y), b.x - a.y - (zr * a.y + zi * a.x));
    // y2 = -i u - i A2 x2 - (1 + z) x2 with -i u = (ui, -ur) and -i A2 x2 = i Im(dg) x2
    y2[p] = mk(ui - d.y * b.y - b.x - (zr * b.x - zi * b.y),
               -ur + d.y * b.x - b.y - (zr * b.y + zi * b.x));
  }
}

inline unsigned blocks_2x2(long long n) {
  const long long b = (n + 255) / 256;
  return unsigned(b < 4096 ? b : 4096);
}

// ((iC - I) - z I) x at point p of the stacked field x (x1 at x, x2 at x + n), both halves.
__device__ __forceinline__ void apply2x2_at(const Geom& g, const double2* __restrict__ dg,
                                            const double2* x, long long p, int i, int j, int k,
                                            double zr, double zi, double2& o1, double2& o2) {
  const long long n = g.n, sy = g.nx, sz = (long long)g.nx * g.ny;
  const double2* x1 = x;
  const double2* x2 = x + n;
  const double2 zero = make_double2(0.0, 0.0);
  const double2 xm = i > 0 ? x1[p - 1] : zero, xp = i < g.nx - 1 ? x1[p + 1] : zero;
  const double2 ym = j > 0 ? x1[p - sy] : zero, yp = j < g.ny - 1 ? x1[p + sy] : zero;
  const double2 zm = k > 0 ? x1[p - sz] : zero, zp = k < g.nz - 1 ? x1[p + sz] : zero;
  const double nbr = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
  const double nbi = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
  const double2 d = dg[p], a = x1[p], b = x2[p];
  const double cs = g.cs;
  const double ur = d.x * a.x - cs * nbr + a.x, ui = d.x * a.y - cs * nbi + a.y;
  o1 = make_double2(-b.y - a.x - (zr * a.x - zi * a.y), b.x - a.y - (zr * a.y + zi * a.x));
  o2 = make_double2(ui - d.y * b.y - b.x - (zr * b.x - zi * b.y),
                    -ur + d.y * b.x - b.y - (zr * b.y + zi * b.x));
}

// One stencil sweep of every active node of the scheme eq:fix-pt-exp on iC - I (Case Two),
// float64, one thread per grid point and node (blockIdx.y: the node slot, blockIdx.z: the
// right-hand side); each thread updates both halves of its point.  Node kinds and
// coefficients as k_poly_stage (the scheme is the same, only the operator differs); every
// node's final y is stored in its slot and summed by k_quad_2x2.
__global__ void k_poly_stage_2x2(Geom g, const double2* __restrict__ dg,
                                 const double2* __restrict__ f, long long frs, double2* ws,
                                 long long wrs, const StageArgs<double> a) {
  pdl_enter();
  const StageNode<double>& nd = a.nd[blockIdx.y];
  const long long n = g.n;
  const int r = blockIdx.z;
  double2* wsr = ws + r * wrs;
  const double2* fr = f + r * frs;  // (f1; f2), 2n values
  const int nxy = g.nx * g.ny;
  const double2 md = make_double2(nd.mdr, nd.mdi), cf = make_double2(nd.cfr, nd.cfi);
  const double2 ip = make_double2(nd.ipr, nd.ipi);
  const int kind = nd.kind;
  const bool first = kind == SK_FIRST || kind == SK_FIRST_LAST;
  const bool stencil = !(first && nd.yzero);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int pi = int(p);  // n < 2^31
    const int k = pi / nxy, rem = pi - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    const double2* in = wsr + nd.in;
    double2 b1 = make_double2(0.0, 0.0), b2 = b1;
    if (stencil) apply2x2_at(g, dg, in, p, i, j, k, nd.z0r, nd.z0i, b1, b2);
    const double2 f1 = fr[p], f2 = fr[n + p];
    for (int h = 0; h < 2; ++h) {
      const long long q = p + h * n;
      const double2 bx = h == 0 ? b1 : b2, fv = h == 0 ? f1 : f2;
      if (first) {
        const double2 kv = cmul(md, csub(bx, fv));
        const double2 xc = nd.yzero ? make_double2(0.0, 0.0) : in[q];
        if (kind == SK_FIRST) {
          wsr[nd.kout + q] = kv;
          wsr[nd.acc + q] = cadd(xc, kv);
        } else {
          wsr[nd.yout + q] = cmul(cadd(xc, kv), ip);
        }
      } else {
        const double2 kv = cmul(md, csub(bx, cmul(cf, fv)));
        const double2 av = wsr[nd.acc + q];
        if (kind == SK_MID) {
          wsr[nd.kout + q] = kv;
          wsr[nd.acc + q] = cadd(av, kv);
        } else {
          wsr[nd.yout + q] = cmul(cadd(av, kv), ip);
        }
      }
    }
  }
}

struct Quad2 {
  long long off[MAXJ];  // each node's final y in the workspace of a right-hand side
  double wr[MAXJ], wi[MAXJ];
  int nn;
};

// w = sum_j (sigma_j / z_j) y_j over the 2n values of each right-hand side.
__global__ void k_quad_2x2(const double2* __restrict__ ws, long long wrs, double2* __restrict__ w,
                           long long wwrs, long long nf, const Quad2 q) {
  pdl_enter();
  const int r = blockIdx.y;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nf;
       p += (long long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < q.nn; ++s) {
      const double2 y = ws[r * wrs + q.off[s] + p];
      sx += q.wr[s] * y.x - q.wi[s] * y.y;
      sy += q.wr[s] * y.y + q.wi[s] * y.x;
    }
    w[r * wwrs + p] = make_double2(sx, sy);
  }
}

// Start of a Case Two cycle: v0 = F - t with F = (0; fs f) and t = (iC - I) U already computed
// (t may be null: U = 0), ||v0||^2 -> beta (start_cycle).  Fields of 2n points.
__global__ void __launch_bounds__(RED_THREADS)
k_residual_2x2(const double2* __restrict__ f, long long frs, double fs,
               const double2* __restrict__ t, long long trs, double2* __restrict__ v0,
               long long vrs, long long n, GmresDev gs, double2* partial, unsigned* counters) {
  pdl_enter();
  __shared__ double2 sh[32];
  const int r = blockIdx.y;
  const long long nf = 2 * n;
  const long long base = (long long)blockIdx.x * RED_CHUNK + threadIdx.x;
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < RED_PPT; ++e) {
    const long long p = base + (long long)e * RED_THREADS;
    if (p >= nf) continue;
    double2 v = make_double2(0.0, 0.0);
    if (p >= n) {
      const double2 fv = f[r * frs + (p - n)];
      v = make_double2(fs * fv.x, fs * fv.y);
    }
    if (t) v = csub(v, t[r * trs + p]);
    v0[r * vrs + p] = v;
    s += v.x * v.x + v.y * v.y;
  }
  double2* part = partial + (long long)r * (gs.mmax + 2) * gridDim.x;
  double2 tot = block_sum(make_double2(s, 0.0), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
  if (!last_block(counters + r)) return;
  __shared__ double2 all;
  finish_slots(part, 1, &all, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    counters[r] = 0;
    double* sc = gs.scal + (long long)r * SC_COUNT;
    const double beta = sqrt(all.x);
    sc[SC_RES2] = all.x;
    sc[SC_BETA] = beta;
    sc[SC_INV] = beta > 0.0 ? 1.0 / beta : 0.0;
    gs.g[(long long)r * (gs.mmax + 1)] = make_double2(beta, 0.0);
    gs.kend[r] = 0;
    gs.stopped[r] = beta > 0.0 ? 0 : 1;
  }
}

}  // namespace

cudaError_t launch_apply_2x2(const Geom& g, const double2* dg, const double2* x, double2* y,
                             int nvec, double zr, double zi, cudaStream_t st) {
  return launch_apply_2x2_strided(g, dg, x, 2 * g.n, y, 2 * g.n, nvec, zr, zi, st);
}

cudaError_t launch_apply_2x2_strided(const Geom& g, const double2* dg, const double2* x,
                                     long long xrs, double2* y, long long yrs, int nvec,
                                     double zr, double zi, cudaStream_t st) {
  if (g.n > 0x7fffffffLL || nvec > 65535) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_apply_2x2<double2, double>, dim3(blocks_2x2(g.n), nvec), 256, 0, st, g,
                    dg, x, xrs, y, yrs, zr, zi, g.cs);
}

cudaError_t launch_poly_stage_2x2(const Geom& g, const double2* dg, Buf<const double2> f,
                                  double2* ws, long long wrs, int nvec, const StageArgs<double>& a,
                                  cudaStream_t st) {
  if (g.n > 0x7fffffffLL || a.nnodes < 1 || a.nnodes > MAXJ || nvec > 65535)
    return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_poly_stage_2x2, dim3(blocks_2x2(g.n), a.nnodes, nvec), 256, 0, st, g, dg,
                    f.p, f.rs, ws, wrs, a);
}

cudaError_t launch_quad_2x2(const double2* ws, long long wrs, Buf<double2> w, long long nf,
                            int nvec, const long long* off, const double* wr, const double* wi,
                            int nn, cudaStream_t st) {
  if (nn < 1 || nn > MAXJ) return cudaErrorInvalidValue;
  Quad2 q;
  for (int s = 0; s < nn; ++s) {
    q.off[s] = off[s];
    q.wr[s] = wr[s];
    q.wi[s] = wi[s];
  }
  q.nn = nn;
  count_launch();
  return launch_pdl(k_quad_2x2, dim3(blocks_2x2(nf), nvec), 256, 0, st, ws, wrs, w.p, w.rs, nf, q);
}

cudaError_t launch_residual_2x2(const double2* f, long long frs, double fs, Buf<const double2> t,
                                Buf<double2> v0, long long n, const GmresDev& gs,
                                double2* partial, unsigned* counters, int nvec, cudaStream_t st) {
  count_launch();
  const unsigned blocks = unsigned((2 * n + RED_CHUNK - 1) / RED_CHUNK);
  return launch_pdl(k_residual_2x2, dim3(blocks, nvec), RED_THREADS, 0, st, f, frs, fs, t.p,
                    t.rs, v0.p, v0.rs, n, gs, partial, counters);
}

cudaError_t launch_apply_2x2_32(const Geom& g, const float2* dg, const float2* x, float2* y,
                                int nvec, float zr, float zi, cudaStream_t st) {
  if (g.n > 0x7fffffffLL || nvec > 65535) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_apply_2x2<float2, float>, dim3(blocks_2x2(g.n), nvec), 256, 0, st, g, dg,
                    x, 2 * g.n, y, 2 * g.n, zr, zi, g.csf);
}

}  // namespace hz
