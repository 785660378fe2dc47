// Case Two of Section 3 (eq:mat-2x2): the double-size coefficient matrix iC - I acting on
// stacked fields x = (x1; x2), with C = [[0, I], [-(A1 + I), -A2]] and A = A1 - i A2 the
// normalised operator of Section 7.1.  From the diagonal dg = 6 s/h^2 - m - i a the two parts
// are A1 x1 = Re(dg) x1 - (s/h^2) (sum of the 6 neighbours of x1) and A2 = -Im(dg), so
//     y1 = i x2 - x1 - z x1,
//     y2 = -i (A1 x1 + x1) - i A2 x2 - x2 - z x2,
// and (iC - I)(iu; u) = (0; f) exactly when A u = f.  One thread per point, the neighbours of
// x1 read from memory (the operator alone; the solver of this form is not on the GPU yet).
#include <cuda_runtime.h>

#include "hz_device.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

template <typename T, typename R>
__global__ void k_apply_2x2(Geom g, const T* __restrict__ dg, const T* __restrict__ x,
                            T* __restrict__ y, R zr, R zi, R cs) {
  pdl_enter();
  const long long n = g.n;
  const int r = blockIdx.y;
  const T* x1 = x + 2 * n * r;
  const T* x2 = x1 + n;
  T* y1 = y + 2 * n * r;
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

}  // namespace

cudaError_t launch_apply_2x2(const Geom& g, const double2* dg, const double2* x, double2* y,
                             int nvec, double zr, double zi, cudaStream_t st) {
  if (g.n > 0x7fffffffLL || nvec > 65535) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_apply_2x2<double2, double>, dim3(blocks_2x2(g.n), nvec), 256, 0, st, g,
                    dg, x, y, zr, zi, g.cs);
}

cudaError_t launch_apply_2x2_32(const Geom& g, const float2* dg, const float2* x, float2* y,
                                int nvec, float zr, float zi, cudaStream_t st) {
  if (g.n > 0x7fffffffLL || nvec > 65535) return cudaErrorInvalidValue;
  count_launch();
  return launch_pdl(k_apply_2x2<float2, float>, dim3(blocks_2x2(g.n), nvec), 256, 0, st, g, dg,
                    x, y, zr, zi, g.csf);
}

}  // namespace hz
