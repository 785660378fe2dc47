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
//
// Compiled lengths 32, 128 and 256 run two register-resident stages (radix 8 x 4, 16 x 8,
// 16 x 16) on a padded shared layout.  The square lengths go further (k_fft_x_sq, k_fft_yz_sq:
// 64-point lines, and complex64 256-point lines): one thread a butterfly, the first stage read
// straight from global memory and the second written straight back, so each transform passes
// through shared memory once.
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

constexpr int FT = 128;       // threads of a k_fft_pass block
constexpr int FT_XLINES = 64;  // most lines of an x-pass tile (their pointers sit in shared memory)
constexpr int FU = 8;          // global loads a thread keeps in flight filling or draining an x tile

enum PassKind { PASS_FWD = 0, PASS_MID = 1, PASS_INV = 2, PASS_LAST = 3 };

template <typename T> struct RealT;
template <> struct RealT<float2> { using type = float; };
template <> struct RealT<double2> { using type = double; };

struct PassArgs {
  VecMap src, dst, xin;
  int nx, ny, nz, nvec;
  int tl;           // lines per tile (a power of two)
  int tlsh;         // log2(tl)
  int kind;         // PassKind
  int invlap;       // PASS_MID: 1 / max(lambda, 1) instead of lambda
  int combine;      // PASS_LAST: add (dg - z) x
  double scale;     // 1 / (nx ny nz)
  double zr, zi;
  const void* dg;
  int n, nst;       // this pass's line length and stages
  int nsh;          // log2(n), or -1 when n is not a power of two
  int rad[FFT_MAXST];
  int lsh[FFT_MAXST];   // log2 of the length L combined before stage s, or -1
  int nbsh[FFT_MAXST];  // log2(n / radix of stage s), or -1
  const void* tw;   // this axis's twiddle table (T)
  const void* ex;   // per-axis eigenvalue shares (real type of T)
  const void* ey;
  const void* ez;
};

// q = x / d, r = x - q d, by a shift where d = 2^sh
__device__ __forceinline__ void divmod(int x, int d, int sh, int& q, int& r) {
  if (sh >= 0) {
    q = x >> sh;
    r = x & ((1 << sh) - 1);
  } else {
    q = x / d;
    r = x - q * d;
  }
}

template <typename T>
__device__ __forceinline__ T cconj(T a) { return mk(a.x, -a.y); }

template <typename T>
__device__ __forceinline__ T* field_ptr(const VecMap& m, int v) {
  return (T*)m.base + (long long)(v / m.nq) * m.rs + m.off[v % m.nq];
}

// One Stockham stage of radix P over all lines of the tile: X -> Y.
template <typename T, int P>
__device__ __forceinline__ void fft_stage(const T* X, T* Y, int tl, int n, int ls, int L,
                                          int lsh, int nbsh, const T* __restrict__ tw) {
  const int nb = n / P;        // butterflies per line
  const int r = n / (L * P);   // also the twiddle index step: w_{LP}^{jq} = tw[j q r]
  for (int b = threadIdx.x; b < tl * nb; b += FT) {
    int l, u, m, j;
    divmod(b, nb, nbsh, l, u);
    divmod(u, L, lsh, m, j);
    const T* x = X + l * ls;
    T a[P];
    a[0] = x[m * L + j];
#pragma unroll
    for (int q = 1; q < P; ++q) {
      const T v = x[(m + r * q) * L + j];
      a[q] = (j == 0) ? v : cmul(v, tw[j * q * r]);
    }
    T* o = Y + l * ls + m * L * P + j;
    if constexpr (P == 2) {
      o[0] = cadd(a[0], a[1]);
      o[L] = csub(a[0], a[1]);
    } else if constexpr (P == 4) {
      const T s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
      const T s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
      const T mi = mk(d13.y, -d13.x);  // -i (a1 - a3): output 1 adds it, output 3 subtracts
      o[0] = cadd(s02, s13);
      o[L] = cadd(d02, mi);
      o[2 * L] = csub(s02, s13);
      o[3 * L] = csub(d02, mi);
    } else {
      const int wstep = n / P;  // w_P^m = tw[m n / P]
#pragma unroll
      for (int k = 0; k < P; ++k) {
        T acc = a[0];
#pragma unroll
        for (int q = 1; q < P; ++q) acc = cadd(acc, cmul(a[q], tw[((k * q) % P) * wstep]));
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
    if (p == 4) fft_stage<T, 4>(A, B, tl, a.n, ls, L, a.lsh[s], a.nbsh[s], tw);
    else if (p == 2) fft_stage<T, 2>(A, B, tl, a.n, ls, L, a.lsh[s], a.nbsh[s], tw);
    else if (p == 3) fft_stage<T, 3>(A, B, tl, a.n, ls, L, a.lsh[s], a.nbsh[s], tw);
    else fft_stage<T, 5>(A, B, tl, a.n, ls, L, a.lsh[s], a.nbsh[s], tw);
    __syncthreads();
    T* t = A;
    A = B;
    B = t;
    L *= p;
  }
  return A;
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// ---- compiled line lengths N = 32 .. 256: two register-radix stages (8 x 4, 16 x 4, 16 x 8,
// 16 x 16), so every element passes through shared memory twice per transform, and a padded
// shared layout (one spare element after every 16) so that the radix-strided accesses of a
// warp fall into different banks.
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
template <int N> __host__ __device__ constexpr int padded_stride() { return N + N / 16 + 1; }

// w_16^m = cos(2 pi m / 16) - i sin(2 pi m / 16) for the m = n2 k1 of a 16 = 4 x 4 split
template <typename R>
__device__ __forceinline__ void w16(int m, R& c, R& s) {
  const R c1 = R(0.92387953251128674), s1 = R(0.38268343236508977), h = R(0.70710678118654752);
  switch (m) {
    case 0: c = R(1); s = R(0); break;
    case 1: c = c1; s = -s1; break;
    case 2: c = h; s = -h; break;
    case 3: c = s1; s = -c1; break;
    case 4: c = R(0); s = R(-1); break;
    case 6: c = -h; s = -h; break;
    default: c = -c1; s = s1; break;  // m = 9
  }
}

template <typename T>
__device__ __forceinline__ void dft4(T& a0, T& a1, T& a2, T& a3) {
  const T s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const T s13 = cadd(a1, a3), d13 = csub(a1, a3);
  const T mi = mk(d13.y, -d13.x);  // -i (a1 - a3)
  a0 = cadd(s02, s13);
  a1 = cadd(d02, mi);
  a2 = csub(s02, s13);
  a3 = csub(d02, mi);
}

// In-register DFT of P = 4, 8 or 16 points, natural order in and out.
template <typename T, int P>
__device__ __forceinline__ void dft_reg(T (&a)[P]) {
  using R = decltype(a[0].x);
  if constexpr (P == 4) {
    dft4(a[0], a[1], a[2], a[3]);
  } else if constexpr (P == 8) {
    // 8 = 4 x 2: DFT4 over n1 of a[2 n1 + n2], twiddle w8^{n2 k1}, DFT2 over n2
    T b0[4] = {a[0], a[2], a[4], a[6]}, b1[4] = {a[1], a[3], a[5], a[7]};
    dft4(b0[0], b0[1], b0[2], b0[3]);
    dft4(b1[0], b1[1], b1[2], b1[3]);
    const R h = R(0.70710678118654752);
    b1[1] = mk(h * (b1[1].x + b1[1].y), h * (b1[1].y - b1[1].x));    // * (1 - i)/sqrt2
    b1[2] = mk(b1[2].y, -b1[2].x);                                     // * -i
    b1[3] = mk(h * (b1[3].y - b1[3].x), -h * (b1[3].x + b1[3].y));   // * (-1 - i)/sqrt2
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      a[k1] = cadd(b0[k1], b1[k1]);
      a[k1 + 4] = csub(b0[k1], b1[k1]);
    }
  } else {
    // 16 = 4 x 4: DFT4 over n1 of a[4 n1 + n2], twiddle w16^{n2 k1}, DFT4 over n2
    T b[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      b[n2][0] = a[n2];
      b[n2][1] = a[4 + n2];
      b[n2][2] = a[8 + n2];
      b[n2][3] = a[12 + n2];
      dft4(b[n2][0], b[n2][1], b[n2][2], b[n2][3]);
    }
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) {
        R c, sn;
        w16<R>(n2 * k1, c, sn);
        b[n2][k1] = cmul(b[n2][k1], mk(c, sn));
      }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      T c0 = b[0][k1], c1 = b[1][k1], c2 = b[2][k1], c3 = b[3][k1];
      dft4(c0, c1, c2, c3);
      a[k1] = c0;
      a[k1 + 4] = c1;
      a[k1 + 8] = c2;
      a[k1 + 12] = c3;
    }
  }
}

// One Stockham stage of radix P (4, 8, 16) with the combined length L before it, all constants,
// on the padded layout: butterfly (m, j) takes a_q = w_{LP}^{jq} X[(m + r q) L + j] to
// Y[m L P + j + L k].
template <typename T, int N, int L, int P, int NT>
__device__ __forceinline__ void fft_stage_ct(const T* X, T* Y, int tl, int ls,
                                             const T* __restrict__ tw) {
  constexpr int nb = N / P, r = N / (L * P);
  for (int b = threadIdx.x; b < tl * nb; b += NT) {
    const int l = b / nb, u = b % nb;
    const int j = u % L, m = u / L;
    const T* x = X + l * ls;
    T a[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const T v = x[padi((m + r * q) * L + j)];
      a[q] = (q == 0 || j == 0) ? v : cmul(v, tw[j * q * r]);
    }
    dft_reg<T, P>(a);
    T* y = Y + l * ls;
#pragma unroll
    for (int k = 0; k < P; ++k) y[padi(m * L * P + j + L * k)] = a[k];
  }
}

template <int N> struct Plan2;
template <> struct Plan2<32> { static constexpr int P1 = 8, P2 = 4; };
template <> struct Plan2<128> { static constexpr int P1 = 16, P2 = 8; };
template <> struct Plan2<256> { static constexpr int P1 = 16, P2 = 16; };

template <typename T, int N, int NT>
__device__ __forceinline__ T* fft_lines_ct(T* A, T* B, int tl, int ls, const T* __restrict__ tw) {
  constexpr int P1 = Plan2<N>::P1, P2 = Plan2<N>::P2;
  static_assert(P1 * P2 == N, "two stages");
  fft_stage_ct<T, N, 1, P1, NT>(A, B, tl, ls, tw);
  __syncthreads();
  fft_stage_ct<T, N, P1, P2, NT>(B, A, tl, ls, tw);
  __syncthreads();
  return A;
}

// NC: the line length when it is one of the compiled power-of-two sizes, else 0 (any length
// with the radix plan of the pass arguments).
template <typename T, int AXIS, int NC>
__global__ void __launch_bounds__(FT) k_fft_pass(const PassArgs a) {
  pdl_enter();
  constexpr int NT = FT;
  using R = typename RealT<T>::type;
  extern __shared__ __align__(16) unsigned char fft_smem[];
  __shared__ const T* s_src[FT_XLINES];  // x pass: each line's first point, per buffer
  __shared__ T* s_dst[FT_XLINES];
  __shared__ const T* s_xin[FT_XLINES];
  __shared__ long long s_off[FT_XLINES];  // x pass: each line's first point within its field
  const int n = NC > 0 ? NC : a.n, tl = a.tl;
  const int nsh = NC > 0 ? ilog2c(NC) : a.nsh;
  // line stride in shared memory (odd); compiled lengths use the padded layout
  const int ls = NC > 0 ? padded_stride<(NC > 0 ? NC : 16)>() : (n | 1);
  auto sx = [&](int l, int e) { return l * ls + (NC > 0 ? padi(e) : e); };
  T* A = reinterpret_cast<T*>(fft_smem);
  T* B = A + (size_t)tl * ls;
  const long long sxy = (long long)a.nx * a.ny;
  const T* __restrict__ tw = (const T*)a.tw;
  // lines of the tile: x pass, pointers per line; y and z passes, one base per buffer and
  // valid lines [0, nvalid), line l at base + l, point e at + e * stride
  int nvalid = 0;
  long long stride = 1;
  const T* srcb = nullptr;
  T* dstb = nullptr;
  if (AXIS == 0) {
    const long long per = (long long)a.ny * a.nz;
    const long long total = per * a.nvec;
    const long long l0 = (long long)blockIdx.x * tl;
    nvalid = (int)(total - l0 < tl ? total - l0 : (long long)tl);
    for (int l = threadIdx.x; l < nvalid; l += NT) {
      const long long lg = l0 + l;
      const int v = (int)(lg / per);
      const long long off = (lg - (long long)v * per) * a.nx;
      s_src[l] = field_ptr<const T>(a.src, v) + off;
      s_dst[l] = field_ptr<T>(a.dst, v) + off;
      s_xin[l] = a.combine ? field_ptr<const T>(a.xin, v) + off : nullptr;
      s_off[l] = off;
    }
    __syncthreads();
  } else {
    const int i0 = blockIdx.x * tl;
    nvalid = min(tl, a.nx - i0);
    const int v = blockIdx.z;
    const long long off = (AXIS == 1 ? (long long)blockIdx.y * sxy : (long long)blockIdx.y * a.nx)
                          + i0;
    stride = AXIS == 1 ? a.nx : sxy;
    srcb = field_ptr<const T>(a.src, v) + off;
    dstb = field_ptr<T>(a.dst, v) + off;
  }
  const bool conj_in = a.kind == PASS_INV || a.kind == PASS_LAST;
  const int tot = tl * n;
  // global loads a thread issues before storing any of them to shared memory: FU along x
  // (contiguous lines); one along y and z, whose rows are far apart (measured slower batched)
  constexpr int fu = AXIS == 0 ? FU : 1;
  // point t of the tile: x pass, consecutive threads walk a line; y, z, consecutive threads the
  // x positions
  auto point = [&](int t, int& l, int& e) {
    if (AXIS == 0) divmod(t, n, nsh, l, e);
    else divmod(t, tl, a.tlsh, e, l);
  };
  for (int t0 = threadIdx.x; t0 < tot; t0 += fu * NT) {
    T v[fu];
#pragma unroll
    for (int k = 0; k < fu; ++k) {
      int l, e;
      point(t0 + k * NT, l, e);
      v[k] = czero<T>();
      if (t0 + k * NT < tot && l < nvalid)
        v[k] = AXIS == 0 ? s_src[l][e] : srcb[l + (long long)e * stride];
    }
#pragma unroll
    for (int k = 0; k < fu; ++k) {
      int l, e;
      point(t0 + k * NT, l, e);
      if (t0 + k * NT < tot) A[sx(l, e)] = conj_in ? cconj(v[k]) : v[k];
    }
  }
  __syncthreads();
  T* X;
  if constexpr (NC > 0) X = fft_lines_ct<T, NC, NT>(A, B, tl, ls, tw);
  else X = fft_lines<T>(A, B, tl, ls, a, tw);
  if (a.kind == PASS_MID) {
    // z lines after the x and y transforms: point (l, e) holds wave numbers (i0 + l, j, e)
    const R* ex = (const R*)a.ex;
    const R* ez = (const R*)a.ez;
    const R sc = R(a.scale);
    const R lj = ((const R*)a.ey)[blockIdx.y];
    const int i0 = blockIdx.x * tl;
    for (int t = threadIdx.x; t < tot; t += NT) {
      int l, e;
      point(t, l, e);
      const R lam = (l < nvalid ? ex[i0 + l] : R(0)) + lj + ez[e];
      const R mlt = a.invlap ? sc / (lam > R(1) ? lam : R(1)) : sc * lam;
      const T x = X[sx(l, e)];
      X[sx(l, e)] = mk(mlt * x.x, -(mlt * x.y));  // conj: the inverse transform follows
    }
    __syncthreads();
    T* Y = (X == A) ? B : A;
    if constexpr (NC > 0) X = fft_lines_ct<T, NC, NT>(X, Y, tl, ls, tw);
    else X = fft_lines<T>(X, Y, tl, ls, a, tw);
  }
  const bool conj_out = a.kind != PASS_FWD;
  const T* __restrict__ dg = (const T*)a.dg;
  const R zr = R(a.zr), zi = R(a.zi);
  const bool comb = AXIS == 0 && a.kind == PASS_LAST && a.combine;
  for (int t0 = threadIdx.x; t0 < tot; t0 += fu * NT) {
    T xv[fu], dv[fu];
    if (comb) {  // the last pass runs along x: its pointwise part's loads, all in flight at once
#pragma unroll
      for (int k = 0; k < fu; ++k) {
        int l, e;
        point(t0 + k * NT, l, e);
        xv[k] = dv[k] = czero<T>();
        if (t0 + k * NT < tot && l < nvalid) {
          xv[k] = s_xin[l][e];
          dv[k] = dg[s_off[l] + e];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < fu; ++k) {
      int l, e;
      point(t0 + k * NT, l, e);
      if (t0 + k * NT >= tot || l >= nvalid) continue;
      T val = X[sx(l, e)];
      if (conj_out) val = cconj(val);
      if (comb) {  // add (dg - z) x at the point
        const T x = xv[k];
        const R dr = dv[k].x - zr, di = dv[k].y - zi;
        val = mk(val.x + dr * x.x - di * x.y, val.y + dr * x.y + di * x.x);
      }
      if (AXIS == 0) s_dst[l][e] = val;
      else dstb[l + (long long)e * stride] = val;
    }
  }
}

// Complex64 lines of a square length N = P^2 (64 = 8 x 8, 256 = 16 x 16), the sizes of the
// large grids: one thread a radix-P butterfly, TL = 256 / P lines a block of 256 threads.  The
// first stage reads its P inputs straight from global memory (P loads in flight a thread) and
// the second writes its P outputs straight back, so a transform passes through shared memory
// once, in one buffer of TL padded lines.  Stages as in fft_stage_ct: the first (L = 1) takes
// points u + P q of butterfly u to P u + k, the second (L = P) points P q + u, with twiddles
// w_N^{u q}, to u + P k.
template <int N> struct SqRadix;
template <> struct SqRadix<64> { static constexpr int P = 8; };
template <> struct SqRadix<256> { static constexpr int P = 16; };

// The two stages on the thread's butterfly u of its line's buffer Al: stage 1 from x (points
// u + P q) into the buffer, then stage 2 from the buffer into x (points u + P k).
template <typename T, int N>
__device__ __forceinline__ void sq_stages(T (&x)[SqRadix<N>::P], T* Al, int u,
                                          const T* __restrict__ tw) {
  constexpr int P = SqRadix<N>::P;
  dft_reg<T, P>(x);
#pragma unroll
  for (int k = 0; k < P; ++k) Al[padi(P * u + k)] = x[k];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const T val = Al[padi(P * q + u)];
    x[q] = (q == 0 || u == 0) ? val : cmul(val, tw[u * q]);
  }
  dft_reg<T, P>(x);
}

// y and z passes: a tile is TL adjacent x positions (a warp load covers 128-256 contiguous
// bytes of a row).  Pass 3 (z) runs the diagonal and the inverse transform in the same block.
template <typename T, int AXIS, int N>
__global__ void __launch_bounds__(256) k_fft_yz_sq(const PassArgs a) {
  pdl_enter();
  using R = typename RealT<T>::type;
  constexpr int P = SqRadix<N>::P, TL = 256 / P;
  constexpr int ls = padded_stride<N>();
  extern __shared__ __align__(16) unsigned char fft_smem[];
  const int l = threadIdx.x % TL;  // line of the tile: x position i0 + l
  const int u = threadIdx.x / TL;  // butterfly of the line
  const int i0 = blockIdx.x * TL;
  const bool valid = l < a.nx - i0;
  const long long sxy = (long long)a.nx * a.ny;
  const long long stride = AXIS == 1 ? a.nx : sxy;
  const long long off =
      (AXIS == 1 ? (long long)blockIdx.y * sxy : (long long)blockIdx.y * a.nx) + i0 + l;
  const T* __restrict__ src = field_ptr<const T>(a.src, blockIdx.z) + off;
  T* __restrict__ dst = field_ptr<T>(a.dst, blockIdx.z) + off;
  const T* __restrict__ tw = (const T*)a.tw;
  T* Al = reinterpret_cast<T*>(fft_smem) + l * ls;
  const bool conj_in = a.kind == PASS_INV || a.kind == PASS_LAST;
  T x[P];
#pragma unroll
  for (int q = 0; q < P; ++q) x[q] = valid ? src[(long long)(u + P * q) * stride] : czero<T>();
  if (conj_in) {
#pragma unroll
    for (int q = 0; q < P; ++q) x[q] = cconj(x[q]);
  }
  sq_stages<T, N>(x, Al, u, tw);
  if (a.kind == PASS_MID) {
    // z lines after the x and y transforms: point (l, e) holds wave numbers (i0 + l, j, e)
    const R* ez = (const R*)a.ez;
    const R sc = R(a.scale);
    const R lxy = (valid ? ((const R*)a.ex)[i0 + l] : R(0)) + ((const R*)a.ey)[blockIdx.y];
    // x[k] holds point u + P k: the inputs of butterfly u of the inverse transform's first
    // stage, so the diagonal is applied in registers
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const R lam = lxy + ez[u + P * k];
      const R mlt = a.invlap ? sc / (lam > R(1) ? lam : R(1)) : sc * lam;
      x[k] = mk(mlt * x[k].x, -(mlt * x[k].y));  // conj: the inverse transform follows
    }
    __syncthreads();  // every thread has read the buffer
    sq_stages<T, N>(x, Al, u, tw);
  }
  if (!valid) return;
  const bool conj_out = a.kind != PASS_FWD;
#pragma unroll
  for (int k = 0; k < P; ++k)
    dst[(long long)(u + P * k) * stride] = conj_out ? cconj(x[k]) : x[k];
}

// x passes: TL whole lines a block, the P lanes of a line's butterflies consecutive (a warp load
// covers 256 contiguous bytes).  The last pass adds the operator's pointwise part (dg - z) x,
// its loads issued eight points at a time.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_fft_x_sq(const PassArgs a) {
  pdl_enter();
  using R = typename RealT<T>::type;
  constexpr int P = SqRadix<N>::P, TL = 256 / P;
  constexpr int ls = padded_stride<N>();
  extern __shared__ __align__(16) unsigned char fft_smem[];
  const int u = threadIdx.x % P;  // butterfly of the line
  const int l = threadIdx.x / P;  // line of the tile
  const long long per = (long long)a.ny * a.nz;
  const long long lg = (long long)blockIdx.x * TL + l;
  const bool valid = lg < per * a.nvec;
  int v = 0;
  long long off = 0;  // the line's first point within its field
  if (valid) {
    v = (int)(lg / per);
    off = (lg - (long long)v * per) * N;
  }
  const T* __restrict__ src = field_ptr<const T>(a.src, v) + off;
  T* __restrict__ dst = field_ptr<T>(a.dst, v) + off;
  const T* __restrict__ tw = (const T*)a.tw;
  T* Al = reinterpret_cast<T*>(fft_smem) + l * ls;
  const bool conj_in = a.kind == PASS_INV || a.kind == PASS_LAST;
  T x[P];
#pragma unroll
  for (int q = 0; q < P; ++q) x[q] = valid ? src[u + P * q] : czero<T>();
  if (conj_in) {
#pragma unroll
    for (int q = 0; q < P; ++q) x[q] = cconj(x[q]);
  }
  sq_stages<T, N>(x, Al, u, tw);  // x[k] = point u + P k
  if (!valid) return;
  const bool conj_out = a.kind != PASS_FWD;
  if (a.kind == PASS_LAST && a.combine) {  // add (dg - z) x at the point
    const T* __restrict__ xin = field_ptr<const T>(a.xin, v) + off;
    const T* __restrict__ dg = (const T*)a.dg + off;
    const R zr = R(a.zr), zi = R(a.zi);
#pragma unroll
    for (int k0 = 0; k0 < P; k0 += 8) {
      T xv[8], dv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        xv[k] = xin[u + P * (k0 + k)];
        dv[k] = dg[u + P * (k0 + k)];
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const T val = conj_out ? cconj(x[k0 + k]) : x[k0 + k];
        const R dr = dv[k].x - zr, di = dv[k].y - zi;
        dst[u + P * (k0 + k)] = mk(val.x + dr * xv[k].x - di * xv[k].y,
                                   val.y + dr * xv[k].y + di * xv[k].x);
      }
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < P; ++k) dst[u + P * k] = conj_out ? cconj(x[k]) : x[k];
}

inline int ilog2_exact(long long v) {  // log2(v) for a power of two, else -1
  if (v <= 0 || (v & (v - 1)) != 0) return -1;
  int k = 0;
  while ((1LL << k) < v) ++k;
  return k;
}

// Lines per tile: x passes 512-1024 points (the lines are contiguous); y and z passes 16
// adjacent x positions (128-256 contiguous bytes per row, the DRAM-friendly width) as long as
// both buffers stay within kFftSmemMax, else 8 or fewer.
constexpr size_t kFftSmemMax = 96 * 1024;
int line_stride(int n) {
  const bool compiled = n == 32 || n == 64 || n == 128 || n == 256;
  return compiled ? n + n / 16 + 1 : (n | 1);  // as the kernel's line stride
}
int tile_lines(int n, int axis, size_t elem) {
  if (axis == 0) {
    int tl = 1;
    while (tl * 2 <= FT_XLINES && tl * 2 * n <= 512) tl *= 2;
    // compiled lengths: up to 1024 points while the first radix-16 (32: radix-8) stage has
    // fewer butterflies than the block has threads
    if (n == 32 || n == 64 || n == 128 || n == 256) {
      const int p1 = n == 32 ? 8 : 16;
      while (tl * 2 <= FT_XLINES && tl * (n / p1) < FT && tl * n < 1024) tl *= 2;
    }
    return tl;
  }
  int tl = 16;
  while (tl > 1 && 2 * elem * (size_t)tl * (size_t)line_stride(n) > kFftSmemMax) tl /= 2;
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

template <typename T, int NC>
cudaError_t launch_axis(int axis, dim3 grid, size_t smem, cudaStream_t st, const PassArgs& a) {
  if (axis == 0) return launch_pdl(k_fft_pass<T, 0, NC>, grid, dim3(FT), smem, st, a);
  if (axis == 1) return launch_pdl(k_fft_pass<T, 1, NC>, grid, dim3(FT), smem, st, a);
  return launch_pdl(k_fft_pass<T, 2, NC>, grid, dim3(FT), smem, st, a);
}

// One pass of lines of the square length N through k_fft_x_sq / k_fft_yz_sq: TL = 256 / sqrt(N)
// lines a block of 256 threads.
template <typename T, int N>
cudaError_t launch_sq(int axis, const PassArgs& a, cudaStream_t st) {
  constexpr int TL = 256 / SqRadix<N>::P;
  const size_t smem = sizeof(T) * (size_t)TL * (size_t)line_stride(N);
  if (axis == 0) {
    const dim3 grid((unsigned)(((long long)a.ny * a.nz * a.nvec + TL - 1) / TL));
    return launch_pdl(k_fft_x_sq<T, N>, grid, dim3(256), smem, st, a);
  }
  const dim3 grid((a.nx + TL - 1) / TL, axis == 1 ? a.nz : a.ny, a.nvec);
  if (axis == 1) return launch_pdl(k_fft_yz_sq<T, 1, N>, grid, dim3(256), smem, st, a);
  return launch_pdl(k_fft_yz_sq<T, 2, N>, grid, dim3(256), smem, st, a);
}

template <typename T>
cudaError_t run_pass(int axis, PassArgs a, const SpecPlan& sp, cudaStream_t st) {
  const FftAxis& ax = sp.ax[axis];
  a.n = ax.n;
  a.nst = ax.nst;
  a.nsh = ilog2_exact(ax.n);
  int L = 1;
  for (int s = 0; s < FFT_MAXST; ++s) {
    const int p = s < ax.nst ? ax.rad[s] : 1;
    a.rad[s] = p;
    a.lsh[s] = ilog2_exact(L);
    a.nbsh[s] = ilog2_exact(ax.n / p);
    L *= p;
  }
  a.tw = tw_of<T>(ax);
  a.tl = tile_lines(ax.n, axis, sizeof(T));
  a.tlsh = ilog2_exact(a.tl);
  const size_t smem = 2 * sizeof(T) * (size_t)a.tl * (size_t)line_stride(ax.n);
  count_launch();
  // lines of a square length run the register-staged kernels (their one shared buffer is at
  // most 35 KB: complex64 256-point, complex128 64-point lines)
  if (ax.n == 64) return launch_sq<T, 64>(axis, a, st);
  if constexpr (sizeof(T) == 8) {
    if (ax.n == 256) return launch_sq<T, 256>(axis, a, st);
  }
  dim3 grid;
  if (axis == 0) {
    const long long lines = (long long)a.ny * a.nz * a.nvec;
    grid = dim3((unsigned)((lines + a.tl - 1) / a.tl));
  } else {
    grid = dim3((a.nx + a.tl - 1) / a.tl, axis == 1 ? a.nz : a.ny, a.nvec);
  }
  switch (ax.n) {
    case 32: return launch_axis<T, 32>(axis, grid, smem, st, a);
    case 128: return launch_axis<T, 128>(axis, grid, smem, st, a);
    case 256: return launch_axis<T, 256>(axis, grid, smem, st, a);
    default: return launch_axis<T, 0>(axis, grid, smem, st, a);
  }
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

namespace {
template <typename T, int NC>
cudaError_t fft_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_fft_pass<T, 0, NC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_pass<T, 1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFftSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft_pass<T, 2, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFftSmemMax);
  return e;
}
template <typename T>
cudaError_t fft_attrs() {
  cudaError_t e = fft_attr<T, 0>();
  if (e == cudaSuccess) e = fft_attr<T, 32>();
  if (e == cudaSuccess) e = fft_attr<T, 128>();
  if (e == cudaSuccess) e = fft_attr<T, 256>();
  return e;
}
}  // namespace

cudaError_t fft_prepare() {
  cudaError_t e = fft_attrs<float2>();
  if (e == cudaSuccess) e = fft_attrs<double2>();
  return e;
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
