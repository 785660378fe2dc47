// The learned right preconditioner: a 4-level 3D U-Net (16 base channels, 3x3x3 kernels, BF16
// weights and activations with FP32 accumulation on the tensor cores) that maps a residual to
// an approximate error, trained on the GPU with the library's own forward and backward kernels.
//
// The paper's method has no network; flexible GMRES admits a right preconditioner that changes
// from step to step (Section 2, after Algorithm 1), which is what lets a network, or a network
// combined with FCI, serve as one.  The true residual still decides convergence.
//
// Architecture (channels last, "++" concatenation along channels, the upsampled map first):
//   x0 [8: Re r, Im r, m, 0...] -> e1a 16 -> e1b 16 = s1
//   pool -> e2a 32 -> e2b 32 = s2;  pool -> e3a 64 -> e3b 64 = s3;  pool -> ba 128 -> bb 128
//   up ++ s3 -> d3a 64 -> d3b 64;  up ++ s2 -> d2a 32 -> d2b 32;  up ++ s1 -> d1a 16 -> d1b 16
//   head: 1x1x1 16 -> 2 (Re e, Im e)
// every 3x3x3 convolution followed by ReLU; pool = 2x2x2 mean, up = nearest neighbour x2.
// Parameters are one flat fp32 array: per convolution w[Cout][27][Cin] then b[Cout], in the
// order above, then the head's w[2][16] and b[2].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "hz.h"
#include "hz_internal.h"
#include "hz_net_internal.h"

#define HZ_TRY_NET(call)          \
  do {                            \
    hz_status s_ = (call);        \
    if (s_ != HZ_OK) return s_;   \
  } while (0)

namespace hz {
namespace {

constexpr int NCONV = 14;
struct ConvSpec {
  int cin0, cin1, cout;
};
constexpr ConvSpec kConv[NCONV] = {{8, 0, 16},    {16, 0, 16},  {16, 0, 32},  {32, 0, 32},
                                   {32, 0, 64},   {64, 0, 64},  {64, 0, 128}, {128, 0, 128},
                                   {128, 64, 64}, {64, 0, 64},  {64, 32, 32}, {32, 0, 32},
                                   {32, 16, 16},  {16, 0, 16}};
enum { E1A, E1B, E2A, E2B, E3A, E3B, BA, BB, D3A, D3B, D2A, D2B, D1A, D1B };
constexpr int HEAD_IN = 16, OUT_CH = 2;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ---- elementwise kernels (grid-stride) ----
#define GRID_STRIDE(i, total) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (total); \
       i += (long long)gridDim.x * blockDim.x)

// dst [B][D/2][H/2][W/2][C] = mean of 2x2x2 blocks of src [B][D][H][W][C]
__global__ void k_pool(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                       int B, int D, int H, int W, int C) {
  const int d = D / 2, h = H / 2, w = W / 2;
  GRID_STRIDE(i, (long long)B * d * h * w * C) {
    const int c = (int)(i % C);
    long long v = i / C;
    const int x = (int)(v % w), y = (int)((v / w) % h), z = (int)((v / ((long long)w * h)) % d);
    const int b = (int)(v / ((long long)w * h * d));
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const long long u = ((((long long)b * D + 2 * z + (q >> 2)) * H + 2 * y + ((q >> 1) & 1)) * W +
                           2 * x + (q & 1)) * C + c;
      s += bf(src[u]);
    }
    dst[i] = __float2bfloat16_rn(s * 0.125f);
  }
}

// dst [B][2D][2H][2W][C] = nearest-neighbour upsampling of src [B][D][H][W][C]; a thread
// moves 8 channels (16 bytes)
__global__ void k_up(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                     int B, int D, int H, int W, int C) {
  const int D2 = 2 * D, H2 = 2 * H, W2 = 2 * W, C8 = C / 8;
  const uint4* s8 = reinterpret_cast<const uint4*>(src);
  uint4* d8 = reinterpret_cast<uint4*>(dst);
  GRID_STRIDE(i, (long long)B * D2 * H2 * W2 * C8) {
    const int c = (int)(i % C8);
    long long v = i / C8;
    const int x = (int)(v % W2), y = (int)((v / W2) % H2), z = (int)((v / ((long long)W2 * H2)) % D2);
    const int b = (int)(v / ((long long)W2 * H2 * D2));
    d8[i] = s8[((((long long)b * D + z / 2) * H + y / 2) * W + x / 2) * C8 + c];
  }
}

// dst [B][D][H][W][C] = sum of the 2x2x2 fine values of g [B][2D][2H][2W][C] (adjoint of k_up)
__global__ void k_up_back(const float* __restrict__ g, float* __restrict__ dst, int B, int D,
                          int H, int W, int C) {
  const int H2 = 2 * H, W2 = 2 * W;
  GRID_STRIDE(i, (long long)B * D * H * W * C) {
    const int c = (int)(i % C);
    long long v = i / C;
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)((v / ((long long)W * H)) % D);
    const int b = (int)(v / ((long long)W * H * D));
    float s = 0.f;
    for (int q = 0; q < 8; ++q)
      s += g[((((long long)b * 2 * D + 2 * z + (q >> 2)) * H2 + 2 * y + ((q >> 1) & 1)) * W2 +
              2 * x + (q & 1)) * C + c];
    dst[i] = s;
  }
}

// dst [B][2D][2H][2W][C] += g [B][D][H][W][C] / 8 at every fine voxel (adjoint of k_pool)
__global__ void k_pool_back_add(const float* __restrict__ g, float* __restrict__ dst, int B,
                                int D, int H, int W, int C) {
  const int D2 = 2 * D, H2 = 2 * H, W2 = 2 * W;
  GRID_STRIDE(i, (long long)B * D2 * H2 * W2 * C) {
    const int c = (int)(i % C);
    long long v = i / C;
    const int x = (int)(v % W2), y = (int)((v / W2) % H2), z = (int)((v / ((long long)W2 * H2)) % D2);
    const int b = (int)(v / ((long long)W2 * H2 * D2));
    dst[i] += 0.125f * g[((((long long)b * D + z / 2) * H + y / 2) * W + x / 2) * C + c];
  }
}

// Through the ReLU: dpre = g * (out > 0), rounded to bf16 for the tensor-core kernels; the bias
// gradient db[c] += sum over voxels of dpre (block sums, one atomic per block and channel).
__global__ void k_relu_back(const float* __restrict__ g, const __nv_bfloat16* __restrict__ out,
                            __nv_bfloat16* __restrict__ dpre, float* __restrict__ db,
                            long long nvox, int C) {
  extern __shared__ float sdb[];
  for (int c = threadIdx.x; c < C; c += blockDim.x) sdb[c] = 0.f;
  __syncthreads();
  // each thread keeps its channel fixed (blockDim is a multiple of C)
  const int c = threadIdx.x % C;
  float acc = 0.f;
  GRID_STRIDE(i, nvox * C) {
    const float v = bf(out[i]) > 0.f ? g[i] : 0.f;
    dpre[i] = __float2bfloat16_rn(v);
    acc += v;
  }
  atomicAdd(&sdb[c], acc);
  __syncthreads();
  for (int q = threadIdx.x; q < C; q += blockDim.x) atomicAdd(&db[q], sdb[q]);
}

// y[v][o] = sum_c d1[v][c] w[o][c] + b[o]  (head, fp32 out)
__global__ void k_head(const __nv_bfloat16* __restrict__ d1, const float* __restrict__ w,
                       const float* __restrict__ b, float* __restrict__ y, long long nvox) {
  GRID_STRIDE(v, nvox) {
    float s0 = b[0], s1 = b[1];
    for (int c = 0; c < HEAD_IN; ++c) {
      const float x = bf(d1[v * HEAD_IN + c]);
      s0 = fmaf(x, w[c], s0);
      s1 = fmaf(x, w[HEAD_IN + c], s1);
    }
    y[2 * v] = s0;
    y[2 * v + 1] = s1;
  }
}

// Loss L = sum (y - t)^2 / (2 nvox_per_sample) over the batch (each sample's term), dy = (y -
// t) / nvox_per_sample; the head's backward: g1[v][c] = sum_o dy[v][o] w[o][c], dW[o][c] +=
// sum_v dy[v][o] d1[v][c], db[o] += sum_v dy[v][o].
__global__ void k_loss_head_back(const float* __restrict__ y, const float* __restrict__ t,
                                 const __nv_bfloat16* __restrict__ d1, const float* __restrict__ w,
                                 float* __restrict__ g1, float* __restrict__ dw,
                                 float* __restrict__ dbias, double* __restrict__ loss,
                                 long long nvox, float inv_per_sample) {
  __shared__ float sw[OUT_CH * HEAD_IN + OUT_CH];
  __shared__ double sl;
  for (int q = threadIdx.x; q < OUT_CH * HEAD_IN + OUT_CH; q += blockDim.x) sw[q] = 0.f;
  if (threadIdx.x == 0) sl = 0.0;
  __syncthreads();
  float pw[OUT_CH * HEAD_IN + OUT_CH];
  for (int q = 0; q < OUT_CH * HEAD_IN + OUT_CH; ++q) pw[q] = 0.f;
  double pl = 0.0;
  GRID_STRIDE(v, nvox) {
    const float e0 = y[2 * v] - t[2 * v], e1 = y[2 * v + 1] - t[2 * v + 1];
    pl += 0.5 * ((double)e0 * e0 + (double)e1 * e1) * inv_per_sample;
    const float d0 = e0 * inv_per_sample, dd1 = e1 * inv_per_sample;
    for (int c = 0; c < HEAD_IN; ++c) {
      const float x = bf(d1[v * HEAD_IN + c]);
      g1[v * HEAD_IN + c] = d0 * w[c] + dd1 * w[HEAD_IN + c];
      pw[c] = fmaf(d0, x, pw[c]);
      pw[HEAD_IN + c] = fmaf(dd1, x, pw[HEAD_IN + c]);
    }
    pw[2 * HEAD_IN] += d0;
    pw[2 * HEAD_IN + 1] += dd1;
  }
  // per-warp sums first (shuffles), one shared atomic per warp and value
  for (int q = 0; q < OUT_CH * HEAD_IN + OUT_CH; ++q) {
    float v = pw[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sw[q], v);
  }
  for (int o = 16; o > 0; o >>= 1) pl += __shfl_xor_sync(0xffffffffu, pl, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&sl, pl);
  __syncthreads();
  for (int q = threadIdx.x; q < OUT_CH * HEAD_IN; q += blockDim.x) atomicAdd(&dw[q], sw[q]);
  if (threadIdx.x < OUT_CH) atomicAdd(&dbias[threadIdx.x], sw[OUT_CH * HEAD_IN + threadIdx.x]);
  if (threadIdx.x == 0) atomicAdd(loss, sl);
}

// Adam (Kingma and Ba, 2015) with bias correction: c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
  GRID_STRIDE(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                              long long n) {
  GRID_STRIDE(i, n) y[i] = __float2bfloat16_rn(x[i]);
}

// Sum of |r|^2 per field (double, block sums then atomics): ss[b].
__global__ void k_sumsq(const double2* __restrict__ r, long long rrs, long long n,
                        double* __restrict__ ss) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = r[b * rrs + i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(&ss[b], s);
  }
}

// Network input from a complex field: x0[b][v] = (Re r / rms, Im r / rms, m, 0, ..., 0) in
// bf16, rms = sqrt(ss[b] / n); optional target t[b][v] = (Re e, Im e) / rms in fp32.
__global__ void k_field_to_input(const double2* __restrict__ r, long long rrs,
                                 const double* __restrict__ m, const double* __restrict__ ss,
                                 const double2* __restrict__ e, long long ers,
                                 __nv_bfloat16* __restrict__ x0, float* __restrict__ t,
                                 long long n, int B) {
  GRID_STRIDE(i, (long long)B * n) {
    const int b = (int)(i / n);
    const long long v = i - (long long)b * n;
    const double inv = ss[b] > 0.0 ? rsqrt(ss[b] / (double)n) : 0.0;
    const double2 rv = r[b * rrs + v];
    uint4 pk;
    __nv_bfloat162 h0 = __floats2bfloat162_rn((float)(rv.x * inv), (float)(rv.y * inv));
    __nv_bfloat162 h1 = __floats2bfloat162_rn((float)m[v], 0.f);
    __nv_bfloat162 hz = __floats2bfloat162_rn(0.f, 0.f);
    pk.x = *reinterpret_cast<uint32_t*>(&h0);
    pk.y = *reinterpret_cast<uint32_t*>(&h1);
    pk.z = *reinterpret_cast<uint32_t*>(&hz);
    pk.w = pk.z;
    reinterpret_cast<uint4*>(x0)[i] = pk;
    if (t) {
      const double2 ev = e[b * ers + v];
      t[2 * i] = (float)(ev.x * inv);
      t[2 * i + 1] = (float)(ev.y * inv);
    }
  }
}

// z[b][v] = rms * (y0 + i y1) (+ z if accumulate)
__global__ void k_output_to_field(const float* __restrict__ y, const double* __restrict__ ss,
                                  double2* __restrict__ z, long long zrs, long long n, int B,
                                  int accumulate) {
  GRID_STRIDE(i, (long long)B * n) {
    const int b = (int)(i / n);
    const long long v = i - (long long)b * n;
    const double rms = sqrt(ss[b] / (double)n);
    double2 o = make_double2(rms * y[2 * i], rms * y[2 * i + 1]);
    double2* zp = z + b * zrs + v;
    if (accumulate) {
      const double2 zi = *zp;
      o.x += zi.x;
      o.y += zi.y;
    }
    *zp = o;
  }
}

// t = v - a (per field, strided), or dst += src with a = null semantics below
__global__ void k_field_sub(const double2* __restrict__ v, long long vrs,
                            const double2* __restrict__ a, long long ars, double2* __restrict__ t,
                            long long trs, long long n, int B) {
  GRID_STRIDE(i, (long long)B * n) {
    const int b = (int)(i / n);
    const long long q = i - (long long)b * n;
    const double2 x = v[b * vrs + q], y = a[b * ars + q];
    t[b * trs + q] = make_double2(x.x - y.x, x.y - y.y);
  }
}

__global__ void k_scale_by_step(double2* __restrict__ z, long long zrs, GmresDev gs, long long n) {
  const int r = blockIdx.y;
  const double* sc = gs.scal + (long long)r * SC_COUNT;
  const double dr = sc[SC_DR], di = sc[SC_DI];
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 v = z[r * zrs + p];
    z[r * zrs + p] = make_double2(dr * v.x - di * v.y, dr * v.y + di * v.x);
  }
}

__global__ void k_field_add(double2* __restrict__ dst, long long drs,
                            const double2* __restrict__ src, long long srs, long long n, int B) {
  GRID_STRIDE(i, (long long)B * n) {
    const int b = (int)(i / n);
    const long long q = i - (long long)b * n;
    const double2 x = dst[b * drs + q], y = src[b * srs + q];
    dst[b * drs + q] = make_double2(x.x + y.x, x.y + y.y);
  }
}

inline int gs_blocks(long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8192));
}

}  // namespace

long long net_param_count() {
  long long n = 0;
  for (const ConvSpec& c : kConv) n += 27LL * (c.cin0 + c.cin1) * c.cout + c.cout;
  return n + OUT_CH * HEAD_IN + OUT_CH;
}

}  // namespace hz

using hz::FMap;
using hz::kConv;
using hz::NCONV;

struct hz_net {
  int device = 0;
  int D = 0, H = 0, W = 0, Bmax = 0;
  int sms = 152;
  long long np = 0;
  float *par = nullptr, *grad = nullptr, *mom1 = nullptr, *mom2 = nullptr;
  long long woff[NCONV] = {}, boff[NCONV] = {}, hw = 0, hb = 0;
  __nv_bfloat16 *wp[NCONV] = {}, *wt[NCONV] = {};
  int adam_t = 0;
  // activations (bf16, channels last) and the output
  __nv_bfloat16 *x0 = nullptr, *act[NCONV] = {}, *pool1 = nullptr, *pool2 = nullptr,
                *pool3 = nullptr, *up3 = nullptr, *up2 = nullptr, *up1 = nullptr, *dpre = nullptr;
  float *y = nullptr, *tgt = nullptr;
  // gradients of activations (fp32)
  float *gA = nullptr, *gB = nullptr, *ds1 = nullptr, *ds2 = nullptr, *ds3 = nullptr;
  double* dscal = nullptr;  // [0] loss, [1..Bmax] per-sample sums of squares
  float* ksplit = nullptr;  // fp32 sums of the convolutions that split their K loop (levels >= 1)
  long long ksplit_floats = 0;
  int* err = nullptr;
  bool packed = false;
  std::vector<void*> allocs;
  ~hz_net() {
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

thread_local std::string t_net_err;

hz_status nfail(hz_status s, const std::string& m) {
  hz::set_last_error(m);
  return s;
}

#define NCHK(call)                                                                     \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return nfail(HZ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
hz_status nalloc(hz_net* n, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nfail(HZ_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  n->allocs.push_back(*p);
  return HZ_OK;
}

FMap fm(const void* p, int C, int W, int H, int D, int B) { return FMap{p, C, W, H, D, B}; }

// Pack both weight layouts of every convolution from the fp32 parameters.
hz_status repack(hz_net* n, cudaStream_t st) {
  for (int l = 0; l < NCONV; ++l) {
    const int cin = kConv[l].cin0 + kConv[l].cin1, cout = kConv[l].cout;
    NCHK(hz::launch_pack_weights(n->par + n->woff[l], n->wp[l], cin, cout, 0, st));
    if (l != 0) NCHK(hz::launch_pack_weights(n->par + n->woff[l], n->wt[l], cin, cout, 1, st));
  }
  n->packed = true;
  return HZ_OK;
}

hz_status check_err(hz_net* n) {
  int e = 0;
  NCHK(cudaMemcpy(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    cudaMemset(n->err, 0, sizeof(int));
    return nfail(HZ_ERR_TIMEOUT, "a bounded wait of a tensor-core convolution gave up");
  }
  return HZ_OK;
}

struct Dims {
  int B, D, H, W;
  long long vox(int level) const {
    return (long long)B * (D >> level) * (H >> level) * (W >> level);
  }
};

// Forward pass from n->x0 (already filled) to n->y.
hz_status net_forward(hz_net* n, const Dims& d, cudaStream_t st) {
  if (!n->packed) HZ_TRY_NET(repack(n, st));
  const int B = d.B;
  auto lv = [&](int l, int C, const void* p) {
    return fm(p, C, d.W >> l, d.H >> l, d.D >> l, B);
  };
  auto conv = [&](int l, const FMap& a, const FMap* b, __nv_bfloat16* out) -> hz_status {
    NCHK(hz::launch_conv_fwd(a, b, n->wp[l], n->par + n->boff[l], kConv[l].cout, 1, out, nullptr,
                             nullptr, nullptr, 0, 0, 0, n->err, st, n->ksplit, n->ksplit_floats,
                             n->sms));
    return HZ_OK;
  };
  auto pool = [&](const __nv_bfloat16* s, __nv_bfloat16* o, int l, int C) -> hz_status {
    hz::count_launch();
    hz::k_pool<<<hz::gs_blocks(d.vox(l + 1) * C), 256, 0, st>>>(s, o, B, d.D >> l, d.H >> l,
                                                                  d.W >> l, C);
    NCHK(cudaGetLastError());
    return HZ_OK;
  };
  auto up = [&](const __nv_bfloat16* s, __nv_bfloat16* o, int l, int C) -> hz_status {
    hz::count_launch();  // from level l to level l - 1
    hz::k_up<<<hz::gs_blocks(d.vox(l - 1) * C / 8), 256, 0, st>>>(s, o, B, d.D >> l, d.H >> l,
                                                                d.W >> l, C);
    NCHK(cudaGetLastError());
    return HZ_OK;
  };
  HZ_TRY_NET(conv(hz::E1A, lv(0, 8, n->x0), nullptr, n->act[hz::E1A]));
  HZ_TRY_NET(conv(hz::E1B, lv(0, 16, n->act[hz::E1A]), nullptr, n->act[hz::E1B]));
  HZ_TRY_NET(pool(n->act[hz::E1B], n->pool1, 0, 16));
  HZ_TRY_NET(conv(hz::E2A, lv(1, 16, n->pool1), nullptr, n->act[hz::E2A]));
  HZ_TRY_NET(conv(hz::E2B, lv(1, 32, n->act[hz::E2A]), nullptr, n->act[hz::E2B]));
  HZ_TRY_NET(pool(n->act[hz::E2B], n->pool2, 1, 32));
  HZ_TRY_NET(conv(hz::E3A, lv(2, 32, n->pool2), nullptr, n->act[hz::E3A]));
  HZ_TRY_NET(conv(hz::E3B, lv(2, 64, n->act[hz::E3A]), nullptr, n->act[hz::E3B]));
  HZ_TRY_NET(pool(n->act[hz::E3B], n->pool3, 2, 64));
  HZ_TRY_NET(conv(hz::BA, lv(3, 64, n->pool3), nullptr, n->act[hz::BA]));
  HZ_TRY_NET(conv(hz::BB, lv(3, 128, n->act[hz::BA]), nullptr, n->act[hz::BB]));
  HZ_TRY_NET(up(n->act[hz::BB], n->up3, 3, 128));
  FMap s3 = lv(2, 64, n->act[hz::E3B]);
  HZ_TRY_NET(conv(hz::D3A, lv(2, 128, n->up3), &s3, n->act[hz::D3A]));
  HZ_TRY_NET(conv(hz::D3B, lv(2, 64, n->act[hz::D3A]), nullptr, n->act[hz::D3B]));
  HZ_TRY_NET(up(n->act[hz::D3B], n->up2, 2, 64));
  FMap s2 = lv(1, 32, n->act[hz::E2B]);
  HZ_TRY_NET(conv(hz::D2A, lv(1, 64, n->up2), &s2, n->act[hz::D2A]));
  HZ_TRY_NET(conv(hz::D2B, lv(1, 32, n->act[hz::D2A]), nullptr, n->act[hz::D2B]));
  HZ_TRY_NET(up(n->act[hz::D2B], n->up1, 1, 32));
  FMap s1 = lv(0, 16, n->act[hz::E1B]);
  HZ_TRY_NET(conv(hz::D1A, lv(0, 32, n->up1), &s1, n->act[hz::D1A]));
  HZ_TRY_NET(conv(hz::D1B, lv(0, 16, n->act[hz::D1A]), nullptr, n->act[hz::D1B]));
  hz::count_launch();
  hz::k_head<<<hz::gs_blocks(d.vox(0)), 256, 0, st>>>(n->act[hz::D1B], n->par + n->hw,
                                                      n->par + n->hb, n->y, d.vox(0));
  NCHK(cudaGetLastError());
  return HZ_OK;
}

// Backward pass after net_forward, with n->tgt holding the targets: loss into dscal[0] (added),
// every parameter gradient into n->grad (zeroed here first).
hz_status net_backward(hz_net* n, const Dims& d, cudaStream_t st) {
  const int B = d.B;
  NCHK(cudaMemsetAsync(n->grad, 0, sizeof(float) * n->np, st));
  auto lv = [&](int l, int C, const void* p) {
    return fm(p, C, d.W >> l, d.H >> l, d.D >> l, B);
  };
  const long long per = (long long)(d.D) * d.H * d.W;
  hz::count_launch();
  hz::k_loss_head_back<<<(int)std::min<long long>(hz::gs_blocks(d.vox(0)), 2 * n->sms), 256, 0,
                          st>>>(
      n->y, n->tgt, n->act[hz::D1B], n->par + n->hw, n->gA, n->grad + n->hw, n->grad + n->hb,
      n->dscal, d.vox(0), 1.0f / (float)per);
  NCHK(cudaGetLastError());
  // one convolution + relu backward: g (fp32, d out) -> dpre; weight and bias gradients; the
  // input gradient into outa (first na channels) / outb (rest) unless outa is null
  auto layer = [&](int l, int lev, const FMap& in0, const FMap* in1, const float* g,
                   float* outa, float* outb, int na, int acc_b) -> hz_status {
    const int C = kConv[l].cout;
    const long long nv = d.vox(lev);
    hz::count_launch();
    const int threads = 256;  // a multiple of every channel count (16..128)
    hz::k_relu_back<<<hz::gs_blocks(nv * C), threads, sizeof(float) * C, st>>>(
        g, n->act[l], n->dpre, n->grad + n->boff[l], nv, C);
    NCHK(cudaGetLastError());
    const FMap gm = lv(lev, C, n->dpre);
    NCHK(hz::launch_conv_wgrad(in0, in1, gm, n->grad + n->woff[l], n->err, n->sms, st));
    if (outa) {
      const int cin = kConv[l].cin0 + kConv[l].cin1;
      NCHK(hz::launch_conv_fwd(gm, nullptr, n->wt[l], nullptr, cin, 0, nullptr, nullptr, outa,
                               outb, na, 0, acc_b, n->err, st, n->ksplit, n->ksplit_floats,
                               n->sms));
    }
    return HZ_OK;
  };
  auto upb = [&](const float* g, float* o, int l, int C) -> hz_status {  // level l-1 -> l
    hz::count_launch();
    hz::k_up_back<<<hz::gs_blocks(d.vox(l) * C), 256, 0, st>>>(g, o, B, d.D >> l, d.H >> l,
                                                               d.W >> l, C);
    NCHK(cudaGetLastError());
    return HZ_OK;
  };
  auto poolb = [&](const float* g, float* o, int l, int C) -> hz_status {  // level l -> l-1, add
    hz::count_launch();
    hz::k_pool_back_add<<<hz::gs_blocks(d.vox(l - 1) * C), 256, 0, st>>>(g, o, B, d.D >> l,
                                                                        d.H >> l, d.W >> l, C);
    NCHK(cudaGetLastError());
    return HZ_OK;
  };
  using namespace hz;
  FMap s1 = lv(0, 16, n->act[E1B]), s2 = lv(1, 32, n->act[E2B]), s3 = lv(2, 64, n->act[E3B]);
  HZ_TRY_NET(layer(D1B, 0, lv(0, 16, n->act[D1A]), nullptr, n->gA, n->gB, nullptr, 16, 0));
  HZ_TRY_NET(layer(D1A, 0, lv(0, 32, n->up1), &s1, n->gB, n->gA, n->ds1, 32, 0));
  HZ_TRY_NET(upb(n->gA, n->gB, 1, 32));
  HZ_TRY_NET(layer(D2B, 1, lv(1, 32, n->act[D2A]), nullptr, n->gB, n->gA, nullptr, 32, 0));
  HZ_TRY_NET(layer(D2A, 1, lv(1, 64, n->up2), &s2, n->gA, n->gB, n->ds2, 64, 0));
  HZ_TRY_NET(upb(n->gB, n->gA, 2, 64));
  HZ_TRY_NET(layer(D3B, 2, lv(2, 64, n->act[D3A]), nullptr, n->gA, n->gB, nullptr, 64, 0));
  HZ_TRY_NET(layer(D3A, 2, lv(2, 128, n->up3), &s3, n->gB, n->gA, n->ds3, 128, 0));
  HZ_TRY_NET(upb(n->gA, n->gB, 3, 128));
  HZ_TRY_NET(layer(BB, 3, lv(3, 128, n->act[BA]), nullptr, n->gB, n->gA, nullptr, 128, 0));
  HZ_TRY_NET(layer(BA, 3, lv(3, 64, n->pool3), nullptr, n->gA, n->gB, nullptr, 64, 0));
  HZ_TRY_NET(poolb(n->gB, n->ds3, 3, 64));
  HZ_TRY_NET(layer(E3B, 2, lv(2, 64, n->act[E3A]), nullptr, n->ds3, n->gA, nullptr, 64, 0));
  HZ_TRY_NET(layer(E3A, 2, lv(2, 32, n->pool2), nullptr, n->gA, n->gB, nullptr, 32, 0));
  HZ_TRY_NET(poolb(n->gB, n->ds2, 2, 32));
  HZ_TRY_NET(layer(E2B, 1, lv(1, 32, n->act[E2A]), nullptr, n->ds2, n->gA, nullptr, 32, 0));
  HZ_TRY_NET(layer(E2A, 1, lv(1, 16, n->pool1), nullptr, n->gA, n->gB, nullptr, 16, 0));
  HZ_TRY_NET(poolb(n->gB, n->ds1, 1, 16));
  HZ_TRY_NET(layer(E1B, 0, lv(0, 16, n->act[E1A]), nullptr, n->ds1, n->gA, nullptr, 16, 0));
  HZ_TRY_NET(layer(E1A, 0, lv(0, 8, n->x0), nullptr, n->gA, nullptr, nullptr, 0, 0));
  return HZ_OK;
}

hz_status net_adam(hz_net* n, float lr, cudaStream_t st) {
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
  hz::count_launch();
  hz::k_adam<<<hz::gs_blocks(n->np), 256, 0, st>>>(n->par, n->grad, n->mom1, n->mom2, n->np, lr,
                                                   b1, b2, c1, c2, 1e-8f);
  NCHK(cudaGetLastError());
  return repack(n, st);
}

bool dims_ok(const hz_net* n, int B, int D, int H, int W) {
  return B >= 1 && B <= n->Bmax && D >= 8 && H >= 8 && W >= 8 && D % 8 == 0 && H % 8 == 0 &&
         W % 8 == 0 && (long long)D * H * W <= (long long)n->D * n->H * n->W;
}

}  // namespace

namespace hz {

// The network's z = N(r) for nvec complex128 fields r of an nx x ny x nz grid (each scaled to
// unit RMS; the output scaled back), with the medium channel m; z is written (accumulate = 0)
// or added to.  Used by the solver as (part of) the right preconditioner.
hz_status net_apply_field(hz_net* n, const double2* r, long long rrs, const double* m, double2* z,
                          long long zrs, int nvec, int nx, int ny, int nz, int accumulate,
                          cudaStream_t st) {
  if (!dims_ok(n, nvec, nz, ny, nx)) return nfail(HZ_ERR_INVALID, "grid not usable by the network");
  const long long nn = (long long)nx * ny * nz;
  NCHK(cudaMemsetAsync(n->dscal + 1, 0, sizeof(double) * nvec, st));
  count_launch();
  k_sumsq<<<dim3((unsigned)std::min<long long>((nn + 255) / 256, 512), nvec), 256, 0, st>>>(
      r, rrs, nn, n->dscal + 1);
  NCHK(cudaGetLastError());
  count_launch();
  k_field_to_input<<<gs_blocks(nn * nvec), 256, 0, st>>>(r, rrs, m, n->dscal + 1, nullptr, 0,
                                                         n->x0, nullptr, nn, nvec);
  NCHK(cudaGetLastError());
  Dims d{nvec, nz, ny, nx};
  HZ_TRY_NET(net_forward(n, d, st));
  count_launch();
  k_output_to_field<<<gs_blocks(nn * nvec), 256, 0, st>>>(n->y, n->dscal + 1, z, zrs, nn, nvec,
                                                          accumulate);
  NCHK(cudaGetLastError());
  return HZ_OK;
}

// One training step on complex field pairs (r, e), A e = r: input (r / rms(r), m), target
// e / rms(r); loss into *loss (host, after a synchronisation).
hz_status net_train_fields(hz_net* n, const double2* r, const double* m, const double2* e,
                           int nvec, int nx, int ny, int nz, float lr, double* loss,
                           cudaStream_t st) {
  if (!dims_ok(n, nvec, nz, ny, nx)) return nfail(HZ_ERR_INVALID, "grid not usable by the network");
  if (!(lr >= 0.f)) return nfail(HZ_ERR_INVALID, "lr must be >= 0");
  const long long nn = (long long)nx * ny * nz;
  NCHK(cudaMemsetAsync(n->dscal, 0, sizeof(double) * (1 + nvec), st));
  count_launch();
  k_sumsq<<<dim3((unsigned)std::min<long long>((nn + 255) / 256, 512), nvec), 256, 0, st>>>(
      r, nn, nn, n->dscal + 1);
  NCHK(cudaGetLastError());
  count_launch();
  k_field_to_input<<<gs_blocks(nn * nvec), 256, 0, st>>>(r, nn, m, n->dscal + 1, e, nn, n->x0,
                                                         n->tgt, nn, nvec);
  NCHK(cudaGetLastError());
  const Dims d{nvec, nz, ny, nx};
  HZ_TRY_NET(net_forward(n, d, st));
  HZ_TRY_NET(net_backward(n, d, st));
  if (lr > 0.f) HZ_TRY_NET(net_adam(n, lr, st));
  double l = 0.0;
  NCHK(cudaMemcpyAsync(&l, n->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  NCHK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return check_err(n);
}

cudaError_t launch_field_sub(const double2* v, long long vrs, const double2* a, long long ars,
                             double2* t, long long trs, long long n, int nvec, cudaStream_t st) {
  count_launch();
  k_field_sub<<<gs_blocks(n * nvec), 256, 0, st>>>(v, vrs, a, ars, t, trs, n, nvec);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_step(double2* z, long long zrs, const GmresDev& gs, long long n,
                                 int nvec, cudaStream_t st) {
  count_launch();
  k_scale_by_step<<<dim3(gs_blocks(n), nvec), 256, 0, st>>>(z, zrs, gs, n);
  return cudaGetLastError();
}

cudaError_t launch_field_add(double2* dst, long long drs, const double2* src, long long srs,
                             long long n, int nvec, cudaStream_t st) {
  count_launch();
  k_field_add<<<gs_blocks(n * nvec), 256, 0, st>>>(dst, drs, src, srs, n, nvec);
  return cudaGetLastError();
}

bool net_fits(const hz_net* n, int nvec, int nx, int ny, int nz) {
  return n && dims_ok(n, nvec, nz, ny, nx);
}

hz_status net_check(hz_net* n) { return check_err(n); }

}  // namespace hz

extern "C" {

long long hz_net_param_count(void) { return hz::net_param_count(); }

hz_status hz_net_create(int D, int H, int W, int batch_max, hz_net** out) {
  if (!out) return nfail(HZ_ERR_INVALID, "out is null");
  *out = nullptr;
  if (batch_max < 1 || D < 8 || H < 8 || W < 8 || D % 8 || H % 8 || W % 8)
    return nfail(HZ_ERR_INVALID, "hz_net_create: D, H, W multiples of 8 (>= 8), batch_max >= 1");
  cudaError_t e = hz::tma_encoder_init();
  if (e != cudaSuccess) return nfail(HZ_ERR_CUDA, "tensor-map encoder unavailable");
  hz_net* n = new hz_net();
  auto bail = [&](hz_status s) {
    delete n;
    return s;
  };
  cudaGetDevice(&n->device);
  if (cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, n->device) != cudaSuccess)
    n->sms = 152;
  n->D = D;
  n->H = H;
  n->W = W;
  n->Bmax = batch_max;
  n->np = hz::net_param_count();
  long long off = 0;
  for (int l = 0; l < NCONV; ++l) {
    n->woff[l] = off;
    off += 27LL * (kConv[l].cin0 + kConv[l].cin1) * kConv[l].cout;
    n->boff[l] = off;
    off += kConv[l].cout;
  }
  n->hw = off;
  n->hb = off + hz::OUT_CH * hz::HEAD_IN;
  hz_status s;
  if ((s = nalloc(n, &n->par, n->np)) || (s = nalloc(n, &n->grad, n->np)) ||
      (s = nalloc(n, &n->mom1, n->np)) || (s = nalloc(n, &n->mom2, n->np)))
    return bail(s);
  for (int l = 0; l < NCONV; ++l) {
    const int cin = kConv[l].cin0 + kConv[l].cin1, cout = kConv[l].cout;
    if ((s = nalloc(n, &n->wp[l], (size_t)hz::conv_nchunk_pad(cin) * cout * 8))) return bail(s);
    if (l && (s = nalloc(n, &n->wt[l], (size_t)hz::conv_nchunk_pad(cout) * cin * 8)))
      return bail(s);
  }
  const long long v0 = (long long)batch_max * D * H * W;  // level-0 voxels
  const long long v1 = v0 / 8, v2 = v0 / 64, v3 = v0 / 512;
  const long long lvox[4] = {v0, v1, v2, v3};
  const int lev[NCONV] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
  if ((s = nalloc(n, &n->x0, v0 * 8))) return bail(s);
  for (int l = 0; l < NCONV; ++l)
    if ((s = nalloc(n, &n->act[l], lvox[lev[l]] * kConv[l].cout))) return bail(s);
  for (int l = 0; l < NCONV; ++l)  // forward (cout) and data-gradient (cin) outputs
    if (lev[l] >= 1)
      n->ksplit_floats = std::max(n->ksplit_floats,
                                  lvox[lev[l]] * std::max(kConv[l].cout,
                                                          kConv[l].cin0 + kConv[l].cin1));
  if ((s = nalloc(n, &n->ksplit, n->ksplit_floats))) return bail(s);
  if ((s = nalloc(n, &n->pool1, v1 * 16)) || (s = nalloc(n, &n->pool2, v2 * 32)) ||
      (s = nalloc(n, &n->pool3, v3 * 64)) || (s = nalloc(n, &n->up3, v2 * 128)) ||
      (s = nalloc(n, &n->up2, v1 * 64)) || (s = nalloc(n, &n->up1, v0 * 32)) ||
      (s = nalloc(n, &n->dpre, v0 * 16)) || (s = nalloc(n, &n->y, v0 * 2)) ||
      (s = nalloc(n, &n->tgt, v0 * 2)) || (s = nalloc(n, &n->gA, v0 * 32)) ||
      (s = nalloc(n, &n->gB, v0 * 32)) || (s = nalloc(n, &n->ds1, v0 * 16)) ||
      (s = nalloc(n, &n->ds2, v1 * 32)) || (s = nalloc(n, &n->ds3, v2 * 64)) ||
      (s = nalloc(n, &n->dscal, 1 + batch_max)) || (s = nalloc(n, &n->err, 1)))
    return bail(s);
  e = cudaMemset(n->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->par, 0, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMemset(n->mom1, 0, sizeof(float) * n->np);
  if (e == cudaSuccess) e = cudaMemset(n->mom2, 0, sizeof(float) * n->np);
  if (e != cudaSuccess) return bail(nfail(HZ_ERR_CUDA, "cudaMemset"));
  *out = n;
  return HZ_OK;
}

hz_status hz_net_destroy(hz_net* n) {
  if (!n) return HZ_OK;
  cudaDeviceSynchronize();
  delete n;
  return HZ_OK;
}

hz_status hz_net_set_params(hz_net* n, const float* host) {
  if (!n || !host) return nfail(HZ_ERR_INVALID, "null argument");
  NCHK(cudaMemcpy(n->par, host, sizeof(float) * n->np, cudaMemcpyHostToDevice));
  NCHK(cudaMemset(n->mom1, 0, sizeof(float) * n->np));
  NCHK(cudaMemset(n->mom2, 0, sizeof(float) * n->np));
  n->adam_t = 0;
  HZ_TRY_NET(repack(n, 0));
  NCHK(cudaDeviceSynchronize());
  return HZ_OK;
}

hz_status hz_net_get_params(const hz_net* n, float* host) {
  if (!n || !host) return nfail(HZ_ERR_INVALID, "null argument");
  NCHK(cudaMemcpy(host, n->par, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  return HZ_OK;
}

hz_status hz_net_forward(hz_net* n, const float* x, float* y, int batch, int D, int H, int W,
                         void* stream) {
  if (!n || !x || !y) return nfail(HZ_ERR_INVALID, "null argument");
  if (!dims_ok(n, batch, D, H, W)) return nfail(HZ_ERR_INVALID, "dims beyond the network's");
  const cudaStream_t st = (cudaStream_t)stream;
  const long long nv = (long long)batch * D * H * W;
  hz::count_launch();
  hz::k_f32_to_bf16<<<hz::gs_blocks(nv * 8), 256, 0, st>>>(x, n->x0, nv * 8);
  NCHK(cudaGetLastError());
  HZ_TRY_NET(net_forward(n, Dims{batch, D, H, W}, st));
  NCHK(cudaMemcpyAsync(y, n->y, sizeof(float) * nv * 2, cudaMemcpyDeviceToDevice, st));
  NCHK(cudaStreamSynchronize(st));
  return check_err(n);
}

hz_status hz_net_train_step(hz_net* n, const float* x, const float* target, int batch, int D,
                            int H, int W, float lr, float* grads, double* loss, void* stream) {
  if (!n || !x || !target) return nfail(HZ_ERR_INVALID, "null argument");
  if (!dims_ok(n, batch, D, H, W)) return nfail(HZ_ERR_INVALID, "dims beyond the network's");
  if (!(lr >= 0.f)) return nfail(HZ_ERR_INVALID, "lr must be >= 0");
  const cudaStream_t st = (cudaStream_t)stream;
  const long long nv = (long long)batch * D * H * W;
  hz::count_launch();
  hz::k_f32_to_bf16<<<hz::gs_blocks(nv * 8), 256, 0, st>>>(x, n->x0, nv * 8);
  NCHK(cudaGetLastError());
  NCHK(cudaMemcpyAsync(n->tgt, target, sizeof(float) * nv * 2, cudaMemcpyDeviceToDevice, st));
  NCHK(cudaMemsetAsync(n->dscal, 0, sizeof(double), st));
  const Dims d{batch, D, H, W};
  HZ_TRY_NET(net_forward(n, d, st));
  HZ_TRY_NET(net_backward(n, d, st));
  if (grads)
    NCHK(cudaMemcpyAsync(grads, n->grad, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, st));
  if (lr > 0.f) HZ_TRY_NET(net_adam(n, lr, st));
  double l = 0.0;
  NCHK(cudaMemcpyAsync(&l, n->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  NCHK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return check_err(n);
}

hz_status hz_conv3d(const void* x, int B, int D, int H, int W, int Cin, const float* w,
                    const float* bias, int Cout, int relu, float* y, void* workspace,
                    void* stream) {
  if (!x || !w || !y || !workspace) return nfail(HZ_ERR_INVALID, "null argument");
  if (Cin < 8 || Cin % 8 || Cout < 16 || Cout > 256 || Cout % 16)
    return nfail(HZ_ERR_INVALID, "Cin a multiple of 8, Cout a multiple of 16 in [16, 256]");
  cudaError_t e = hz::tma_encoder_init();
  if (e != cudaSuccess) return nfail(HZ_ERR_CUDA, "tensor-map encoder unavailable");
  const cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16* wp = (__nv_bfloat16*)workspace;
  int* err = (int*)((char*)workspace + (size_t)hz::conv_nchunk_pad(Cin) * Cout * 16);
  NCHK(cudaMemsetAsync(err, 0, sizeof(int), st));
  NCHK(hz::launch_pack_weights(w, wp, Cin, Cout, 0, st));
  NCHK(hz::launch_conv_fwd(fm(x, Cin, W, H, D, B), nullptr, wp, bias, Cout, relu, nullptr, y,
                           nullptr, nullptr, 0, 0, 0, err, st));
  int h = 0;
  NCHK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCHK(cudaStreamSynchronize(st));
  return h ? nfail(HZ_ERR_TIMEOUT, "a bounded wait gave up") : HZ_OK;
}

hz_status hz_conv3d_backward(const void* x, const void* g, int B, int D, int H, int W, int Cin,
                             const float* w, int Cout, float* dx, float* dw, void* workspace,
                             void* stream) {
  if (!x || !g || !w || !dw || !workspace) return nfail(HZ_ERR_INVALID, "null argument");
  if (Cin < 16 || Cin % 16 || Cout < 16 || Cout > 128 || Cout % 16)
    return nfail(HZ_ERR_INVALID, "Cin a multiple of 16, Cout a multiple of 16 in [16, 128]");
  cudaError_t e = hz::tma_encoder_init();
  if (e != cudaSuccess) return nfail(HZ_ERR_CUDA, "tensor-map encoder unavailable");
  const cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16* wt = (__nv_bfloat16*)workspace;
  int* err = (int*)((char*)workspace + (size_t)hz::conv_nchunk_pad(Cout) * Cin * 16);
  NCHK(cudaMemsetAsync(err, 0, sizeof(int), st));
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const FMap xm = fm(x, Cin, W, H, D, B), gm = fm(g, Cout, W, H, D, B);
  NCHK(cudaMemsetAsync(dw, 0, sizeof(float) * 27 * Cin * Cout, st));
  NCHK(hz::launch_conv_wgrad(xm, nullptr, gm, dw, err, sms, st));
  if (dx) {
    NCHK(hz::launch_pack_weights(w, wt, Cin, Cout, 1, st));
    NCHK(hz::launch_conv_fwd(gm, nullptr, wt, nullptr, Cin, 0, nullptr, nullptr, dx, nullptr, Cin,
                             0, 0, err, st));
  }
  int h = 0;
  NCHK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NCHK(cudaStreamSynchronize(st));
  return h ? nfail(HZ_ERR_TIMEOUT, "a bounded wait gave up") : HZ_OK;
}

long long hz_conv3d_workspace_bytes(int Cin, int Cout) {
  const long long a = (long long)hz::conv_nchunk_pad(Cin) * Cout * 16;
  const long long b = (long long)hz::conv_nchunk_pad(Cout) * Cin * 16;
  return std::max(a, b) + 256;
}

}  // extern "C"
