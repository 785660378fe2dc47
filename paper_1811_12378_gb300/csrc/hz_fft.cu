// The Fourier spectral discretisation of Section 7.1 on the GPU: S = F^H Lambda F on the
// periodic nx x ny x nz box, Lambda the squared wavenumbers 2 pi min(i, n - i) / (n h) summed
// over the axes (eq:eig-Laplacian-spectral), and the regularised inverse Laplacian
// F^H diag(1 / max(lambda_i, 1)) F of the spectral runs' inner preconditioner (Section 7.3).
//
// A 3D transform is a sequence of line transforms, one axis at a time.  One application of S
// (or of the preconditioner) to nvec fields takes five passes, each reading and writing every
// field once:
//   1. x lines, forward (input -> scratch)      4. y lines, inverse
//   2. y lines, forward                         5. x lines, inverse, then the epilogue
//   3. z lines: forward, multiply by the diagonal (lambda or 1 / max(lambda, 1), over the
//      number of points), inverse -- the last forward and the first inverse axis fused
// The epilogue of pass 5 stores s S x or adds the pointwise part (dg - z) x of the operator.
//
// A block owns a tile of TL whole lines: it loads them into shared memory (coalesced: along x
// the lines are contiguous, along y and z the tile is TL adjacent x-positions, so consecutive
// threads read consecutive addresses), transforms them there and writes them back to the same
// place, so passes 2-4 work in place.  The line transform is a Stockham autosort FFT: with L
// the length already combined and radix p, r = n / (L p), butterfly (m, j), j < L, m < r, takes
// a_q = w_{Lp}^{jq} X[(m + r q) L + j] (q < p) to Y[m L p + j + L k] = sum_q w_p^{kq} a_q, so
// the output is in natural order after the last stage; radix 4 and 2 butterflies are written
// out, 3 and 5 use the twiddle table.  Inverse transforms are conj(FFT(conj(x))), unnormalised;
// the 1/(nx ny nz) is folded into the diagonal of pass 3.  Twiddles and the per-axis
// eigenvalue shares are tables made on the host in float64 (rounded for the float32 kernels).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {

bool fft_factor(int n, int* rad, int* nst) {
  if (n < 1 || n > FFT_MAXN) return false;
  int k = 0;
  while (n % 4 == 0 && k < FFT_MAXST) { rad[k++] = 4; n /= 4; }
  while (n % 2 == 0 && k < FFT_MAXST) { rad[k++] = 2; n /= 2; }
  while (n % 3 == 0 && k < FFT_MAXST) { rad[k++] = 3; n /= 3; }
  while (n % 5 == 0 && k < FFT_MAXST) { rad[k++] = 5; n /= 5; }
  *nst = k;
  return n == 1;
}

namespace {

constexpr int FT = 256;  // threads of a line-transform block

enum PassKind { PASS_FWD = 0, PASS_MID = 1, PASS_INV = 2, PASS_LAST = 3 };

template <typename T> struct RealT;
template <> struct RealT<float2> { using type = float; };
template <> struct RealT<double2> { using type = double; };

struct PassArgs {
  VecMap src, dst, xin;
  int nx, ny, nz, nvec;
  int tl;           // lines per tile
  int kind;         // PassKind
  int invlap;       // PASS_MID: 1 / max(lambda, 1) instead of lambda
  int combine;      // PASS_LAST: add (dg - z) x
  double scale;     // 1 / (nx ny nz)
  double zr, zi;
  const void* dg;
  int n, nst;       // this pass's line length and stages
  int rad[FFT_MAXST];
  const void* tw;   // this axis's twiddle table (T)
  const void* ex;   // per-axis eigenvalue shares (real type of T)
  const void* ey;
  const void* ez;
};

template <typename T>
__device__ __forceinline__ T cconj(T a) { return mk(a.x, -a.y); }

template <typename T>
__device__ __forceinline__ T* field_ptr(const VecMap& m, int v) {
  return (T*)m.base + (long long)(v / m.nq) * m.rs + m.off[v % m.nq];
}

// One Stockham stage over all lines of the tile: X -> Y.
template <typename T>
__device__ __forceinline__ void fft_stage(const T* X, T* Y, int tl, int n, int ls, int L, int p,
                                          const T* __restrict__ tw) {
  const int nb = n / p;          // butterflies per line
  const int r = n / (L * p);
  const int ts = n / (L * p);    // twiddle index step: w_{Lp}^{jq} = tw[j q ts]
  for (int b = threadIdx.x; b < tl * nb; b += FT) {
    const int l = b / nb, u = b - l * nb;
    const int j = u % L, m = u / L;
    const T* x = X + l * ls;
    T* y = Y + l * ls;
    T a[5];
    a[0] = x[m * L + j];
    for (int q = 1; q < p; ++q) {
      const T v = x[(m + r * q) * L + j];
      a[q] = (j == 0) ? v : cmul(v, tw[j * q * ts]);
    }
    T* o = y + m * L * p + j;
    if (p == 2) {
      o[0] = cadd(a[0], a[1]);
      o[L] = csub(a[0], a[1]);
    } else if (p == 4) {
      const T s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
      const T s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
      // -i (a1 - a3) for output 1, +i for output 3
      const T mi = mk(d13.y, -d13.x);
      o[0] = cadd(s02, s13);
      o[L] = cadd(d02, mi);
      o[2 * L] = csub(s02, s13);
      o[3 * L] = csub(d02, mi);
    } else {
      const int wstep = n / p;  // w_p^m = tw[m n / p]
      for (int k = 0; k < p; ++k) {
        T acc = a[0];
        for (int q = 1; q < p; ++q) acc = cadd(acc, cmul(a[q], tw[((k * q) % p) * wstep]));
        o[k * L] = acc;
      }
    }
  }
}

// Runs the line FFT of the tile in shared memory; returns the buffer holding the result.
template <typename T>
__device__ T* fft_lines(T* A, T* B, int tl, int ls, const PassArgs& a, const T* __restrict__ tw) {
  int L = 1;
  for (int s = 0; s < a.nst; ++s) {
    const int p = a.rad[s];
    fft_stage<T>(A, B, tl, a.n, ls, L, p, tw);
    __syncthreads();
    T* t = A;
    A = B;
    B = t;
    L *= p;
  }
  return A;
}

template <typename T, int AXIS>
__global__ void __launch_bounds__(FT) k_fft_pass(const PassArgs a) {
  pdl_enter();
  using R = typename RealT<T>::type;
  extern __shared__ unsigned char fft_smem[];
  const int n = a.n, tl = a.tl;
  const int ls = n | 1;  // odd line stride in shared memory
  T* A = reinterpret_cast<T*>(fft_smem);
  T* B = A + (size_t)tl * ls;
  const long long sxy = (long long)a.nx * a.ny;
  const T* __restrict__ tw = (const T*)a.tw;
  // line l of the tile: its field, the offset of its first point and its point stride
  auto line = [&](int l, int& v, long long& off, long long& stride) -> bool {
    if (AXIS == 0) {
      const long long lg = (long long)blockIdx.x * tl + l;
      const long long per = (long long)a.ny * a.nz;
      if (lg >= per * a.nvec) return false;
      v = (int)(lg / per);
      off = (lg - (long long)v * per) * a.nx;
      stride = 1;
      return true;
    }
    const int i = blockIdx.x * tl + l;
    if (i >= a.nx) return false;
    v = blockIdx.z;
    off = (AXIS == 1 ? (long long)blockIdx.y * sxy : (long long)blockIdx.y * a.nx) + i;
    stride = AXIS == 1 ? a.nx : sxy;
    return true;
  };
  const bool conj_in = a.kind == PASS_INV || a.kind == PASS_LAST;
  // load
  for (int t = threadIdx.x; t < tl * n; t += FT) {
    const int l = AXIS == 0 ? t / n : t % tl;
    const int e = AXIS == 0 ? t % n : t / tl;
    int v;
    long long off, stride;
    T val = czero<T>();
    if (line(l, v, off, stride)) {
      val = field_ptr<const T>(a.src, v)[off + (long long)e * stride];
      if (conj_in) val = cconj(val);
    }
    A[l * ls + e] = val;
  }
  __syncthreads();
  T* X = fft_lines<T>(A, B, tl, ls, a, tw);
  if (a.kind == PASS_MID) {
    // z lines after the x and y transforms: point (l, e) holds wave numbers (i, j, e)
    const R* ex = (const R*)a.ex;
    const R* ey = (const R*)a.ey;
    const R* ez = (const R*)a.ez;
    const R sc = R(a.scale);
    const R lj = ey[blockIdx.y];
    for (int t = threadIdx.x; t < tl * n; t += FT) {
      const int l = t % tl, e = t / tl;
      const int i = blockIdx.x * tl + l;
      const R lam = (i < a.nx ? ex[i] : R(0)) + lj + ez[e];
      const R mlt = a.invlap ? sc / (lam > R(1) ? lam : R(1)) : sc * lam;
      const T x = X[l * ls + e];
      X[l * ls + e] = mk(mlt * x.x, -(mlt * x.y));  // conj: the inverse transform follows
    }
    __syncthreads();
    T* Y = (X == A) ? B : A;
    X = fft_lines<T>(X, Y, tl, ls, a, tw);
  }
  const bool conj_out = a.kind != PASS_FWD;
  const T* __restrict__ dg = (const T*)a.dg;
  const R zr = R(a.zr), zi = R(a.zi);
  for (int t = threadIdx.x; t < tl * n; t += FT) {
    const int l = AXIS == 0 ? t / n : t % tl;
    const int e = AXIS == 0 ? t % n : t / tl;
    int v;
    long long off, stride;
    if (!line(l, v, off, stride)) continue;
    const long long pp = off + (long long)e * stride;
    T val = X[l * ls + e];
    if (conj_out) val = cconj(val);
    if (a.kind == PASS_LAST && a.combine) {
      const T x = field_ptr<const T>(a.xin, v)[pp];
      const T d = dg[pp];
      const R dr = d.x - zr, di = d.y - zi;
      val = mk(val.x + dr * x.x - di * x.y, val.y + dr * x.y + di * x.x);
    }
    field_ptr<T>(a.dst, v)[pp] = val;
  }
}

template <typename T>
int tile_lines(int n, int axis) {
  const int target = sizeof(T) == 16 ? 1024 : 2048;  // points per tile: 32 KB of shared memory
  int tl = std::max(1, target / n);
  if (axis != 0) tl = std::min(tl, 32);
  return tl;
}

template <typename T>
const void* tw_of(const FftAxis& ax);
template <>
const void* tw_of<double2>(const FftAxis& ax) { return ax.tw64; }
template <>
const void* tw_of<float2>(const FftAxis& ax) { return ax.tw32; }
template <typename T>
const void* e_of(const FftAxis& ax);
template <>
const void* e_of<double2>(const FftAxis& ax) { return ax.e64; }
template <>
const void* e_of<float2>(const FftAxis& ax) { return ax.e32; }

template <typename T>
cudaError_t run_pass(int axis, PassArgs a, const SpecPlan& sp, cudaStream_t st) {
  const FftAxis& ax = sp.ax[axis];
  a.n = ax.n;
  a.nst = ax.nst;
  for (int s = 0; s < FFT_MAXST; ++s) a.rad[s] = s < ax.nst ? ax.rad[s] : 1;
  a.tw = tw_of<T>(ax);
  a.tl = tile_lines<T>(ax.n, axis);
  const size_t smem = 2 * sizeof(T) * (size_t)a.tl * (size_t)(ax.n | 1);
  count_launch();
  if (axis == 0) {
    const long long lines = (long long)a.ny * a.nz * a.nvec;
    const dim3 grid((unsigned)((lines + a.tl - 1) / a.tl));
    return launch_pdl(k_fft_pass<T, 0>, grid, dim3(FT), smem, st, a);
  }
  const dim3 grid((a.nx + a.tl - 1) / a.tl, axis == 1 ? a.nz : a.ny, a.nvec);
  if (axis == 1) return launch_pdl(k_fft_pass<T, 1>, grid, dim3(FT), smem, st, a);
  return launch_pdl(k_fft_pass<T, 2>, grid, dim3(FT), smem, st, a);
}

// ------------------------------------------------------------------ polynomial stage
// The stage of eq:fix-pt-exp with (A - z0) x = s S x + (dg - z0) x, s S x precomputed: one
// thread per point and right-hand side runs every active node (the stage's pointwise part),
// and on the final stage sums sigma_j / z_j y_j in float64 in node order.
template <typename T, typename R>
__global__ void __launch_bounds__(256)
k_poly_stage_spec(long long n, const T* __restrict__ dg, const T* __restrict__ f, long long frs,
                  T* ws, long long wrs, const T* __restrict__ lap, int nlap,
                  double2* __restrict__ w, long long wwrs, float2* __restrict__ w32,
                  long long w32rs, const StageArgs<R> a) {
  pdl_enter();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (p >= n) return;
  T* wsr = ws + r * wrs;
  const T fv = f[r * frs + p];
  const T dv = dg[p];
  double sx = 0.0, sy = 0.0;
  for (int q = 0; q < a.nnodes; ++q) {
    const StageNode<R>& nd = a.nd[q];
    const int kind = nd.kind;
    const bool first = kind == SK_FIRST || kind == SK_FIRST_LAST;
    const bool use_in = !(first && nd.yzero);
    const T xc = use_in ? wsr[nd.in + p] : czero<T>();
    T Ax = czero<T>();
    if (use_in) {
      const T lv = lap[((long long)r * nlap + nd.lapi) * n + p];
      const R dr = dv.x - nd.z0r, di = dv.y - nd.z0i;
      Ax = mk(lv.x + dr * xc.x - di * xc.y, lv.y + dr * xc.y + di * xc.x);
    }
    const T md = mk(nd.mdr, nd.mdi);
    T yn = czero<T>();
    if (first) {
      const T kv = cmul(md, csub(Ax, fv));
      if (kind == SK_FIRST) {
        wsr[nd.kout + p] = kv;
        wsr[nd.acc + p] = cadd(xc, kv);
      } else {
        yn = cmul(cadd(xc, kv), mk(nd.ipr, nd.ipi));
      }
    } else {
      const T kv = cmul(md, csub(Ax, cmul(mk(nd.cfr, nd.cfi), fv)));
      const T av = wsr[nd.acc + p];
      if (kind == SK_MID) {
        wsr[nd.kout + p] = kv;
        wsr[nd.acc + p] = cadd(av, kv);
      } else {
        yn = cmul(cadd(av, kv), mk(nd.ipr, nd.ipi));
      }
    }
    if (kind == SK_LAST || kind == SK_FIRST_LAST) {
      if (a.final_quad) {
        const double yr = double(yn.x), yi = double(yn.y);
        sx += fma(nd.wqr, yr, -nd.wqi * yi);
        sy += fma(nd.wqr, yi, nd.wqi * yr);
      } else {
        wsr[nd.yout + p] = yn;
      }
    }
  }
  if (a.final_quad) {
    w[r * wwrs + p] = make_double2(sx, sy);
    if (w32) w32[r * w32rs + p] = make_float2(float(sx), float(sy));
  }
}

__global__ void __launch_bounds__(256)
k_scaled_sub(const double2* __restrict__ f, long long frs, double sc,
             const double2* __restrict__ a, long long ars, double2* __restrict__ t,
             long long trs, long long n) {
  pdl_enter();
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (p >= n) return;
  const double2 x = f[r * frs + p], y = a[r * ars + p];
  t[r * trs + p] = make_double2(sc * x.x - y.x, sc * x.y - y.y);
}

}  // namespace

cudaError_t launch_scaled_sub(const double2* f, long long frs, double sc, const double2* a,
                              long long ars, double2* t, long long trs, long long n, int nvec,
                              cudaStream_t st) {
  count_launch();
  return launch_pdl(k_scaled_sub, dim3((unsigned)((n + 255) / 256), nvec), dim3(256), 0, st, f,
                    frs, sc, a, ars, t, trs, n);
}

template <typename T>
cudaError_t launch_spectral(const SpecPlan& sp, const Geom& g, int mode, const VecMap& in,
                            const VecMap& out, int nvec, const T* dg, double zr, double zi,
                            T* tmp, cudaStream_t st) {
  if (nvec <= 0 || g.n == 0) return cudaSuccess;
  PassArgs a{};
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.nvec = nvec;
  a.scale = 1.0 / double(g.n);
  a.zr = zr;
  a.zi = zi;
  a.dg = dg;
  a.ex = e_of<T>(sp.ax[0]);
  a.ey = e_of<T>(sp.ax[1]);
  a.ez = e_of<T>(sp.ax[2]);
  a.invlap = mode == SPEC_INVLAP ? 1 : 0;
  const VecMap tm = vec_map(tmp, g.n);
  cudaError_t e;
  a.src = in;
  a.dst = tm;
  a.kind = PASS_FWD;
  if ((e = run_pass<T>(0, a, sp, st)) != cudaSuccess) return e;
  a.src = tm;
  if ((e = run_pass<T>(1, a, sp, st)) != cudaSuccess) return e;
  a.kind = PASS_MID;
  if ((e = run_pass<T>(2, a, sp, st)) != cudaSuccess) return e;
  a.kind = PASS_INV;
  if ((e = run_pass<T>(1, a, sp, st)) != cudaSuccess) return e;
  a.kind = PASS_LAST;
  a.dst = out;
  a.xin = in;
  a.combine = mode == SPEC_APPLY ? 1 : 0;
  return run_pass<T>(0, a, sp, st);
}

template cudaError_t launch_spectral<double2>(const SpecPlan&, const Geom&, int, const VecMap&,
                                              const VecMap&, int, const double2*, double, double,
                                              double2*, cudaStream_t);
template cudaError_t launch_spectral<float2>(const SpecPlan&, const Geom&, int, const VecMap&,
                                             const VecMap&, int, const float2*, double, double,
                                             float2*, cudaStream_t);

template <typename T, typename R>
cudaError_t launch_poly_stage_spec(const Geom& g, const T* dg, Buf<const T> f, T* ws,
                                   long long wrs, const T* lap, int nlap, Buf<double2> w,
                                   Buf<float2> w32, int nvec, const StageArgs<R>& a,
                                   cudaStream_t st) {
  count_launch();
  const dim3 grid((unsigned)((g.n + 255) / 256), nvec);
  return launch_pdl(k_poly_stage_spec<T, R>, grid, dim3(256), 0, st, g.n, dg, f.p, f.rs, ws, wrs,
                    lap, nlap, w.p, w.rs, w32.p, w32.rs, a);
}

template cudaError_t launch_poly_stage_spec<float2, float>(const Geom&, const float2*,
                                                           Buf<const float2>, float2*, long long,
                                                           const float2*, int, Buf<double2>,
                                                           Buf<float2>, int,
                                                           const StageArgs<float>&, cudaStream_t);
template cudaError_t launch_poly_stage_spec<double2, double>(const Geom&, const double2*,
                                                             Buf<const double2>, double2*,
                                                             long long, const double2*, int,
                                                             Buf<double2>, Buf<float2>, int,
                                                             const StageArgs<double>&,
                                                             cudaStream_t);

}  // namespace hz
