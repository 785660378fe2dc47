// ILU(0) of the 7-point Laplacian as the right preconditioner of the inner GMRES of FCI
// (Section 6.3: an incomplete factorisation without fill of the discrete Laplacian deflates
// the large eigenvalues; Section 7.3 uses it for the finite-difference runs).
//
// K = cs * (6 on the diagonal, -1 per neighbour), cs = s/h^2, is the Laplacian part of the
// normalised operator.  For the 7-point pattern ILU(0) is M = (D + L) D^{-1} (D + U), L and U
// the strict lower and upper parts of K in natural order (x fastest) and
//     d_p = 6 cs - cs^2 * (sum over the lower neighbours q of 1 / d_q),
// computed once on the host.  z = M^{-1} t is a forward sweep u_p = (t_p + cs * sum of u over
// the lower neighbours) / d_p and a backward sweep z_p = u_p + cs / d_p * (sum of z over the
// upper neighbours).  Each value depends on its three lower (upper) neighbours only, so the
// points of one hyperplane i + j + k = const are independent: one block per right-hand side
// walks the nx + ny + nz - 2 hyperplanes with a block barrier between them (no grid-wide wait);
// its threads take the (j, k) lines, each holding the one point of its line on the plane.
#include <cuda_runtime.h>

#include <vector>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int IT = 1024;  // threads of the sweep block

__global__ void __launch_bounds__(IT) k_ilu0_apply(Geom g, const double* __restrict__ invd,
                                                   double cs, const double2* __restrict__ t,
                                                   long long trs, double2* z, long long zrs) {
  pdl_enter();
  const int r = blockIdx.x;
  const double2* tr = t + r * trs;
  double2* zr = z + r * zrs;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  const int W = nx + ny + nz - 2;
  const int lines = ny * nz;
  // forward: (D + L) u = t, u stored in z
  for (int w = 0; w < W; ++w) {
    for (int l = threadIdx.x; l < lines; l += IT) {
      const int j = l % ny, k = l / ny, i = w - j - k;
      if (i < 0 || i >= nx) continue;
      const long long p = i + sy * j + sz * k;
      double2 acc = tr[p];
      if (i > 0) acc = cadd(acc, make_double2(cs * zr[p - 1].x, cs * zr[p - 1].y));
      if (j > 0) acc = cadd(acc, make_double2(cs * zr[p - sy].x, cs * zr[p - sy].y));
      if (k > 0) acc = cadd(acc, make_double2(cs * zr[p - sz].x, cs * zr[p - sz].y));
      const double iv = invd[p];
      zr[p] = make_double2(acc.x * iv, acc.y * iv);
    }
    __syncthreads();
  }
  // backward: (D + U) z = D u, in place
  for (int w = W - 1; w >= 0; --w) {
    for (int l = threadIdx.x; l < lines; l += IT) {
      const int j = l % ny, k = l / ny, i = w - j - k;
      if (i < 0 || i >= nx) continue;
      const long long p = i + sy * j + sz * k;
      double2 acc = make_double2(0.0, 0.0);
      if (i < nx - 1) acc = cadd(acc, zr[p + 1]);
      if (j < ny - 1) acc = cadd(acc, zr[p + sy]);
      if (k < nz - 1) acc = cadd(acc, zr[p + sz]);
      const double f = cs * invd[p];
      const double2 u = zr[p];
      zr[p] = make_double2(u.x + f * acc.x, u.y + f * acc.y);
    }
    __syncthreads();
  }
}

// The same sweeps with each (j, k) line's latest value held in shared memory: the three
// neighbours a point needs from the previous hyperplane are the previous values of its own
// line and of lines (j - 1, k) and (j, k - 1) (upper sweep: j + 1, k + 1), so a hyperplane
// step reads only shared memory besides its own t, 1/d (and u) values, which do not depend on
// the recurrence and are loaded ahead.  Two buffers alternate by hyperplane parity, since a
// line is overwritten in the same step in which its neighbour lines read its previous value.
__global__ void __launch_bounds__(IT) k_ilu0_apply_smem(Geom g, const double* __restrict__ invd,
                                                        double cs,
                                                        const double2* __restrict__ t,
                                                        long long trs, double2* z,
                                                        long long zrs) {
  pdl_enter();
  extern __shared__ double2 lv[];  // [2][ny * nz]
  const int r = blockIdx.x;
  const double2* tr = t + r * trs;
  double2* zr = z + r * zrs;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  const int W = nx + ny + nz - 2;
  const int lines = ny * nz;
  double2* buf[2] = {lv, lv + lines};
  // forward: u_p = (t_p + cs (u_{i-1} + u_{j-1} + u_{k-1})) / d_p
  for (int w = 0; w < W; ++w) {
    const double2* old = buf[(w + 1) & 1];
    double2* cur = buf[w & 1];
    for (int l = threadIdx.x; l < lines; l += IT) {
      const int j = l % ny, k = l / ny, i = w - j - k;
      if (i < 0 || i >= nx) continue;
      const long long p = i + sy * j + sz * k;
      const double2 tv = tr[p];
      const double iv = invd[p];
      double2 acc = make_double2(0.0, 0.0);
      if (i > 0) acc = cadd(acc, old[l]);
      if (j > 0) acc = cadd(acc, old[l - 1]);
      if (k > 0) acc = cadd(acc, old[l - ny]);
      const double2 u = make_double2((tv.x + cs * acc.x) * iv, (tv.y + cs * acc.y) * iv);
      cur[l] = u;
      zr[p] = u;
    }
    __syncthreads();
  }
  // backward: z_p = u_p + cs / d_p (z_{i+1} + z_{j+1} + z_{k+1}), each thread on its own lines
  for (int w = W - 1; w >= 0; --w) {
    const double2* old = buf[(w + 1) & 1];
    double2* cur = buf[w & 1];
    for (int l = threadIdx.x; l < lines; l += IT) {
      const int j = l % ny, k = l / ny, i = w - j - k;
      if (i < 0 || i >= nx) continue;
      const long long p = i + sy * j + sz * k;
      const double2 u = zr[p];
      const double f = cs * invd[p];
      double2 acc = make_double2(0.0, 0.0);
      if (i < nx - 1) acc = cadd(acc, old[l]);
      if (j < ny - 1) acc = cadd(acc, old[l + 1]);
      if (k < nz - 1) acc = cadd(acc, old[l + ny]);
      const double2 zv = make_double2(u.x + f * acc.x, u.y + f * acc.y);
      cur[l] = zv;
      zr[p] = zv;
    }
    __syncthreads();
  }
}

// The sweeps in float32 arithmetic for the complex64-sweep form (HZ_MIXED_C64): the result is
// a preconditioner application, like the complex64 polynomial sweeps, and one SM retires 64
// times more float32 than float64 operations on GB300, which is what bounds a sweep run by a
// single block.  t and z stay float64 fields (the inner basis is float64); the forward result
// goes to a complex64 scratch field u.
__global__ void __launch_bounds__(IT) k_ilu0_apply_smem32(Geom g, const float* __restrict__ invd,
                                                          float cs,
                                                          const double2* __restrict__ t,
                                                          long long trs, float2* u32,
                                                          long long urs, double2* z,
                                                          long long zrs) {
  pdl_enter();
  extern __shared__ float2 lv32[];  // [2][ny * nz]
  const int r = blockIdx.x;
  const double2* tr = t + r * trs;
  float2* ur = u32 + r * urs;
  double2* zr = z + r * zrs;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  const int W = nx + ny + nz - 2;
  const int lines = ny * nz;
  float2* b0 = lv32;
  float2* b1 = lv32 + lines;
  for (int w = 0; w < W; ++w) {
    const float2* old = (w & 1) ? b0 : b1;
    float2* cur = (w & 1) ? b1 : b0;
    for (int l = threadIdx.x; l < lines; l += IT) {
      const int j = l % ny, k = l / ny, i = w - j - k;
      if (i < 0 || i >= nx) continue;
      const long long p = i + sy * j + sz * k;
      const double2 tv = tr[p];
      const float iv = invd[p];
      float ax = 0.f, ay = 0.f;
      if (i > 0) { ax += old[l].x; ay += old[l].y; }
      if (j > 0) { ax += old[l - 1].x; ay += old[l - 1].y; }
      if (k > 0) { ax += old[l - ny].x; ay += old[l - ny].y; }
      const float2 u = make_float2((float(tv.x) + cs * ax) * iv, (float(tv.y) + cs * ay) * iv);
      cur[l] = u;
      ur[p] = u;
    }
    __syncthreads();
  }
  for (int w = W - 1; w >= 0; --w) {
    const float2* old = (w & 1) ? b0 : b1;
    float2* cur = (w & 1) ? b1 : b0;
    for (int l = threadIdx.x; l < lines; l += IT) {
      const int j = l % ny, k = l / ny, i = w - j - k;
      if (i < 0 || i >= nx) continue;
      const long long p = i + sy * j + sz * k;
      const float2 u = ur[p];
      const float f = cs * invd[p];
      float ax = 0.f, ay = 0.f;
      if (i < nx - 1) { ax += old[l].x; ay += old[l].y; }
      if (j < ny - 1) { ax += old[l + 1].x; ay += old[l + 1].y; }
      if (k < nz - 1) { ax += old[l + ny].x; ay += old[l + ny].y; }
      const float2 zv = make_float2(u.x + f * ax, u.y + f * ay);
      cur[l] = zv;
      zr[p] = make_double2(double(zv.x), double(zv.y));
    }
    __syncthreads();
  }
}

constexpr size_t kIluSmemMax = 200 * 1024;

// out[r] += d[r] w[r], d the FCI step size in the inner GMRES state
__global__ void k_add_dw(double2* __restrict__ out, long long ors, const double2* __restrict__ w,
                         long long wrs, long long n, GmresDev gs) {
  pdl_enter();
  const int r = blockIdx.y;
  const double* sc = gs.scal + (long long)r * SC_COUNT;
  const double2 d = make_double2(sc[SC_DR], sc[SC_DI]);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    out[r * ors + p] = cadd(out[r * ors + p], cmul(d, w[r * wrs + p]));
}

}  // namespace

cudaError_t ilu0_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_ilu0_apply_smem,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kIluSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ilu0_apply_smem32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kIluSmemMax);
  return e;
}

cudaError_t launch_ilu0_32(const Geom& g, const float* invd32, Buf<const double2> t,
                           Buf<float2> u32, Buf<double2> z, int nvec, cudaStream_t st) {
  if (nvec < 1 || nvec > 65535) return cudaErrorInvalidValue;
  const size_t smem = 2 * sizeof(float2) * (size_t)g.ny * g.nz;
  if (smem > kIluSmemMax) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_ilu0_apply_smem32, dim3(nvec), dim3(IT), smem, st, g, invd32,
                    float(g.cs), t.p, t.rs, u32.p, u32.rs, z.p, z.rs);
}

bool ilu0_fits32(const Geom& g) {
  return 2 * sizeof(float2) * (size_t)g.ny * g.nz <= kIluSmemMax;
}

void ilu0_inverse_pivots(int nx, int ny, int nz, double cs, std::vector<double>& invd) {
  const long long n = (long long)nx * ny * nz;
  std::vector<double> d(n);
  const long long sy = nx, sz = (long long)nx * ny;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long long p = i + sy * j + sz * k;
        double v = 6.0 * cs;
        if (i > 0) v -= cs * cs / d[p - 1];
        if (j > 0) v -= cs * cs / d[p - sy];
        if (k > 0) v -= cs * cs / d[p - sz];
        d[p] = v;
      }
  invd.resize(n);
  for (long long p = 0; p < n; ++p) invd[p] = 1.0 / d[p];
}

cudaError_t launch_ilu0(const Geom& g, const double* invd, Buf<const double2> t, Buf<double2> z,
                        int nvec, cudaStream_t st) {
  if (nvec < 1 || nvec > 65535) return cudaErrorInvalidValue;
  count_launch();
  const size_t smem = 2 * sizeof(double2) * (size_t)g.ny * g.nz;
  if (smem <= kIluSmemMax) {
    return launch_pdl(k_ilu0_apply_smem, dim3(nvec), dim3(IT), smem, st, g, invd, g.cs, t.p,
                      t.rs, z.p, z.rs);
  }
  return launch_pdl(k_ilu0_apply, dim3(nvec), dim3(IT), 0, st, g, invd, g.cs, t.p, t.rs, z.p,
                    z.rs);
}

cudaError_t launch_add_dw(Buf<double2> out, Buf<const double2> w, long long n, const GmresDev& gs,
                          int nvec, cudaStream_t st) {
  count_launch();
  const long long b = (n + 255) / 256;
  return launch_pdl(k_add_dw, dim3(unsigned(b < 4096 ? b : 4096), nvec), 256, 0, st, out.p,
                    out.rs, w.p, w.rs, n, gs);
}

}  // namespace hz
