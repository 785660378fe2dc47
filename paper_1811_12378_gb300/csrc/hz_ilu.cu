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

#include <algorithm>
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

// ---------------------------------------------------------------- multi-block wavefront
// The same sweeps spread over the SMs: block K owns the TK z-planes k0 = K TK .. k0 + TK - 1
// (all their (j, k) lines) and walks the global hyperplanes w = i + j + k that cross them.  A
// point's lower neighbour in z across the slab boundary, (i, j, k0 - 1), lies on hyperplane
// w - 1 of block K - 1, so block K takes plane w once block K - 1 has published that it finished
// plane w - 1 (release stores of its progress every CHAIN_Q planes, acquire loads before); the
// backward sweep mirrors this with block K + 1.  Within a block the lines' latest values live in shared
// memory as in the one-block kernels, and a neighbour block's boundary values are read from the
// global field past L1.  The blocks wait on one another, so the grid is launched cooperatively
// (all blocks resident); each wait is bounded by the problem's poll limit, after which the
// block records the error, stops waiting and runs on (its results are then wrong and the solve
// reports HZ_ERR_TIMEOUT), so no block waits forever.
constexpr int CHAIN_Q = 4;  // planes between two published progress values
constexpr int CHAIN_D = 4;  // planes a line's loads run ahead of its computation

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <typename V>
__device__ __forceinline__ V ld_cg(const V* p);
template <>
__device__ __forceinline__ float2 ld_cg<float2>(const float2* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ double2 ld_cg<double2>(const double2* p) { return __ldcg(p); }

// Bounded wait of thread 0 until ready(*flag); false (error recorded) if the limit ran out.
template <typename Ready>
__device__ bool chain_wait(const int* flag, Ready ready, unsigned* bar) {
  const unsigned lim = *(volatile unsigned*)(bar + 3);
  for (unsigned it = 0;; ++it) {
    if (ready(ld_acquire(flag))) return true;
    if (it >= lim) {
      atomicExch(bar + 2, 1u);
      return false;
    }
    if (it > 64) __nanosleep(32);
  }
}

template <typename R>
__device__ __forceinline__ typename CplxOf<R>::type to_r(double2 v);
template <>
__device__ __forceinline__ float2 to_r<float>(double2 v) {
  return make_float2(float(v.x), float(v.y));
}
template <>
__device__ __forceinline__ double2 to_r<double>(double2 v) { return v; }

// Forward sweep (D + L) u = t: u into uo (complex of R).  One thread per (j, k) line of the
// slab (blockDim >= lines), software-pipelined: a line's t and 1/d run CHAIN_D planes ahead of
// its computation in registers, and the neighbour block's boundary value for plane w + 1 is
// loaded during plane w when its published progress already covers plane w.  The neighbour's progress
// is polled only when the last value seen is not far enough, and this block's is published
// every CHAIN_Q planes, after the block barrier that closes the planes before, by one release
// store (cumulative over the block's writes it has observed through that barrier).
template <typename R>
__global__ void k_ilu0_chain_fwd(Geom g, const R* __restrict__ invd, R cs,
                                 const typename CplxOf<R>::type* t, long long trs,
                                 typename CplxOf<R>::type* uo, long long urs, int TK, int* prog,
                                 unsigned* bar) {
  using V = typename CplxOf<R>::type;
  extern __shared__ unsigned char ch_smem[];
  __shared__ int s_seen;
  const int K = blockIdx.x, r = blockIdx.y, nK = gridDim.x;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  const int k0 = K * TK, tkc = min(TK, nz - k0);
  const int lines = ny * tkc;
  V* buf0 = reinterpret_cast<V*>(ch_smem);
  V* buf1 = buf0 + (size_t)ny * TK;
  const V* tr = t + r * trs;  // may be the field u is written to: each point is read first
  V* ur = uo + r * urs;
  int* mine = prog + (long long)r * nK + K;
  const int* prev = K > 0 ? mine - 1 : nullptr;
  bool waiting = prev != nullptr;
  int seen = 0;
  const int l = threadIdx.x;
  const bool has = l < lines;
  const int j = has ? l % ny : 0, kl = has ? l / ny : 0, k = k0 + kl;
  const bool edge = has && kl == 0 && K > 0;  // the lower z neighbour lies in block K - 1
  const long long pl = sy * j + sz * k;       // the line's first point
  const int wlo = k0, whi = k0 + tkc - 1 + nx - 1 + ny - 1;
  V tq[CHAIN_D], nb_n{};
  R iq[CHAIN_D];
  bool nb_ok = false;
#pragma unroll
  for (int d = 0; d < CHAIN_D; ++d) {  // the loads of planes wlo .. wlo + CHAIN_D - 1
    const int id = wlo + d - j - k;
    tq[d] = V{};
    iq[d] = 0;
    if (has && id >= 0 && id < nx) {
      tq[d] = tr[pl + id];
      iq[d] = invd[pl + id];
    }
  }
  for (int w0 = wlo; w0 <= whi; w0 += CHAIN_D) {
#pragma unroll
  for (int d = 0; d < CHAIN_D; ++d) {  // slot d of the register ring holds plane w0 + d
    const int w = w0 + d;
    if (w > whi) break;
    const int i = w - j - k;
    const bool act = has && i >= 0 && i < nx;
    const long long p = pl + i;
    const V tv = tq[d], nbp = nb_n;
    const R iv = iq[d];
    const bool have_nb = nb_ok;
    {
      const int ia = i + CHAIN_D;  // the slot's next plane, w + CHAIN_D
      if (has && ia >= 0 && ia < nx) {
        tq[d] = tr[pl + ia];
        iq[d] = invd[pl + ia];
      }
    }
    if (threadIdx.x == 0) {
      if (waiting && seen < w &&
          !chain_wait(prev, [&seen, w](int v) { seen = v; return v >= w; }, bar))
        waiting = false;
      s_seen = waiting ? seen : 0x7fffffff;
    }
    __syncthreads();  // planes < w of this block are complete
    if (threadIdx.x == 0 && w > wlo && (w - wlo) % CHAIN_Q == 0) st_release(mine, w);
    // the next plane's boundary value where block K - 1 has finished plane w
    nb_ok = false;
    if (edge && i + 1 >= 0 && i + 1 < nx && s_seen >= w + 1) {
      nb_n = ld_cg(ur + p + 1 - sz);
      nb_ok = true;
    }
    const V* old = (w & 1) ? buf0 : buf1;
    V* cur = (w & 1) ? buf1 : buf0;
    if (act) {
      R ax = 0, ay = 0;
      if (i > 0) { ax += old[l].x; ay += old[l].y; }
      if (j > 0) { ax += old[l - 1].x; ay += old[l - 1].y; }
      if (kl > 0) {
        ax += old[l - ny].x;
        ay += old[l - ny].y;
      } else if (K > 0) {
        const V nb = have_nb ? nbp : ld_cg(ur + p - sz);
        ax += nb.x;
        ay += nb.y;
      }
      V u;
      u.x = (tv.x + cs * ax) * iv;
      u.y = (tv.y + cs * ay) * iv;
      cur[l] = u;
      ur[p] = u;
    }
  }
  }
  __syncthreads();
  if (threadIdx.x == 0) st_release(mine, 0x7fffffff);  // finished: nothing more to wait for
}

// Backward sweep (D + U) z = D u: reads u (complex of R), writes z (double2); z may be the
// field u lives in (float64 form: each point's u is read before this block overwrites it).
// Pipelined and published like the forward sweep, towards decreasing planes.
template <typename R>
__global__ void k_ilu0_chain_bwd(Geom g, const R* __restrict__ invd, R cs,
                                 const typename CplxOf<R>::type* ui, long long urs,
                                 typename CplxOf<R>::type* z, long long zrs, int TK, int* prog,
                                 unsigned* bar) {
  using V = typename CplxOf<R>::type;
  extern __shared__ unsigned char ch_smem[];
  __shared__ int s_seen;
  const int K = blockIdx.x, r = blockIdx.y, nK = gridDim.x;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long sy = nx, sz = (long long)nx * ny;
  const int k0 = K * TK, tkc = min(TK, nz - k0);
  const int lines = ny * tkc;
  V* buf0 = reinterpret_cast<V*>(ch_smem);
  V* buf1 = buf0 + (size_t)ny * TK;
  const V* ur = ui + r * urs;
  V* zr = z + r * zrs;
  int* mine = prog + (long long)r * nK + K;
  const int* next = K + 1 < nK ? mine + 1 : nullptr;
  bool waiting = next != nullptr;
  int seen = 0x7fffffff;
  const int l = threadIdx.x;
  const bool has = l < lines;
  const int j = has ? l % ny : 0, kl = has ? l / ny : 0, k = k0 + kl;
  const bool edge = has && kl == tkc - 1 && K + 1 < nK;  // upper z neighbour in block K + 1
  const long long pl = sy * j + sz * k;
  const int wlo = k0, whi = k0 + tkc - 1 + nx - 1 + ny - 1;
  V uq[CHAIN_D], nb_n{};
  R fq[CHAIN_D];
  bool nb_ok = false;
#pragma unroll
  for (int d = 0; d < CHAIN_D; ++d) {  // the loads of planes whi .. whi - CHAIN_D + 1
    const int id = whi - d - j - k;
    uq[d] = V{};
    fq[d] = 0;
    if (has && id >= 0 && id < nx) {
      uq[d] = ur[pl + id];
      fq[d] = cs * invd[pl + id];
    }
  }
  for (int w0 = whi; w0 >= wlo; w0 -= CHAIN_D) {
#pragma unroll
  for (int d = 0; d < CHAIN_D; ++d) {  // slot d holds plane w0 - d
    const int w = w0 - d;
    if (w < wlo) break;
    const int i = w - j - k;
    const bool act = has && i >= 0 && i < nx;
    const long long p = pl + i;
    const V u = uq[d], nbp = nb_n;
    const R f = fq[d];
    const bool have_nb = nb_ok;
    {
      const int ia = i - CHAIN_D;  // the slot's next plane, w - CHAIN_D
      if (has && ia >= 0 && ia < nx) {
        uq[d] = ur[pl + ia];
        fq[d] = cs * invd[pl + ia];
      }
    }
    if (threadIdx.x == 0) {
      if (waiting && seen > w + 1 &&
          !chain_wait(next, [&seen, w](int v) { seen = v; return v <= w + 1; }, bar))
        waiting = false;
      s_seen = waiting ? seen : (int)0x80000000;
    }
    __syncthreads();  // planes > w of this block are complete
    if (threadIdx.x == 0 && w < whi && (whi - w) % CHAIN_Q == 0) st_release(mine, w + 1);
    nb_ok = false;
    if (edge && i - 1 >= 0 && i - 1 < nx && s_seen <= w) {  // block K + 1 finished plane w
      nb_n = ld_cg(zr + p - 1 + sz);
      nb_ok = true;
    }
    const V* old = (w & 1) ? buf0 : buf1;
    V* cur = (w & 1) ? buf1 : buf0;
    if (act) {
      R ax = 0, ay = 0;
      if (i < nx - 1) { ax += old[l].x; ay += old[l].y; }
      if (j < ny - 1) { ax += old[l + 1].x; ay += old[l + 1].y; }
      if (kl < tkc - 1) {
        ax += old[l + ny].x;
        ay += old[l + ny].y;
      } else if (K + 1 < nK) {
        const V nb = have_nb ? nbp : ld_cg(zr + p + sz);
        ax += nb.x;
        ay += nb.y;
      }
      V zv;
      zv.x = u.x + f * ax;
      zv.y = u.y + f * ay;
      cur[l] = zv;
      zr[p] = zv;
    }
  }
  }
  __syncthreads();
  if (threadIdx.x == 0) st_release(mine, (int)0x80000000);  // finished
}

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

// ---- multi-block wavefront sweeps
namespace {
int chain_tk(int ny) { return std::max(1, 512 / std::max(1, ny)); }
int chain_threads(int ny, int tk) { return (ny * tk + 31) / 32 * 32; }  // one per line

template <typename R>
bool chain_fits_r(const Geom& g, int nvec) {
  using V = typename CplxOf<R>::type;
  const int tk = chain_tk(g.ny), nk = (g.nz + tk - 1) / tk, nt = chain_threads(g.ny, tk);
  const size_t smem = 2 * sizeof(V) * (size_t)g.ny * tk;
  if (smem > 48 * 1024 || nk < 2 || nt > 1024) return false;
  int dev = 0, sms = 0, bf = 0, bb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_ilu0_chain_fwd<R>, nt, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_ilu0_chain_bwd<R>, nt, smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (long long)std::min(bf, bb) * sms >= (long long)nk * nvec;
}

template <typename K, typename... Args>
cudaError_t launch_coop(K kern, dim3 grid, int nt, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// t, u and z in the arithmetic's own type (the float32 sweeps run on complex64 copies made by
// the caller: a float64 <-> float32 conversion is a float64-pipe instruction, too slow for
// the sequential planes).
template <typename R>
cudaError_t launch_chain_r(const Geom& g, const R* invd, const typename CplxOf<R>::type* t,
                           long long trs, typename CplxOf<R>::type* u, long long urs,
                           typename CplxOf<R>::type* z, long long zrs, int nvec, int* prog,
                           unsigned* bar, cudaStream_t st) {
  using V = typename CplxOf<R>::type;
  const int tk = chain_tk(g.ny), nk = (g.nz + tk - 1) / tk, nt = chain_threads(g.ny, tk);
  const size_t smem = 2 * sizeof(V) * (size_t)g.ny * tk;
  const size_t np = (size_t)nk * nvec;
  int* pf = prog;
  int* pb = prog + np;
  cudaError_t e = cudaMemsetAsync(pf, 0, sizeof(int) * np, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pb, 0x7f, sizeof(int) * np, st);
  if (e != cudaSuccess) return e;
  const dim3 grid(nk, nvec);
  count_launch();
  e = launch_coop(k_ilu0_chain_fwd<R>, grid, nt, smem, st, g, invd, R(g.cs), t, trs, u, urs,
                  tk, pf, bar);
  if (e != cudaSuccess) return e;
  count_launch();
  return launch_coop(k_ilu0_chain_bwd<R>, grid, nt, smem, st, g, invd, R(g.cs),
                     (const V*)u, urs, z, zrs, tk, pb, bar);
}
}  // namespace

bool ilu0_chain_fits(const Geom& g, int nvec, bool f32) {
  return f32 ? chain_fits_r<float>(g, nvec) : chain_fits_r<double>(g, nvec);
}

long long ilu0_chain_prog_ints(const Geom& g, int nvec) {
  const int tk = chain_tk(g.ny);
  return 2LL * ((g.nz + tk - 1) / tk) * nvec;
}

cudaError_t launch_ilu0_chain(const Geom& g, const double* invd, Buf<const double2> t,
                              Buf<double2> z, int nvec, int* prog, unsigned* bar,
                              cudaStream_t st) {
  // the forward result lives in z itself, which the backward sweep overwrites point by point
  return launch_chain_r<double>(g, invd, t.p, t.rs, z.p, z.rs, z.p, z.rs, nvec, prog, bar, st);
}

cudaError_t launch_ilu0_chain32(const Geom& g, const float* invd32, Buf<const double2> t,
                                Buf<float2> u32, Buf<double2> z, int nvec, int* prog,
                                unsigned* bar, cudaStream_t st) {
  // t rounded to complex64 into u32, both sweeps in place there, then back to float64 in z
  cudaError_t e = launch_convert_c128_c64(t, u32, g.n, nvec, st);
  if (e == cudaSuccess)
    e = launch_chain_r<float>(g, invd32, u32.p, u32.rs, u32.p, u32.rs, u32.p, u32.rs, nvec, prog,
                              bar, st);
  if (e == cudaSuccess)
    e = launch_convert_c64_c128(Buf<const float2>{u32.p, u32.rs}, z, g.n, nvec, st);
  return e;
}

cudaError_t launch_add_dw(Buf<double2> out, Buf<const double2> w, long long n, const GmresDev& gs,
                          int nvec, cudaStream_t st) {
  count_launch();
  const long long b = (n + 255) / 256;
  return launch_pdl(k_add_dw, dim3(unsigned(b < 4096 ? b : 4096), nvec), 256, 0, st, out.p,
                    out.rs, w.p, w.rs, n, gs);
}

}  // namespace hz
