// BF16 tensor-core 3x3x3 convolutions of the learned preconditioner (the network of
// hz_net.cu): forward, data gradient and weight gradient as implicit GEMMs on tcgen05.mma with
// FP32 accumulation in tensor memory, operands staged by TMA.
//
// Feature maps are bf16, channels last: element (b, z, y, x, c) at ((((b D + z) H + y) W + x) C
// + c), C a multiple of 8.  A 3x3x3 convolution with zero padding is
//     out[v, n] = sum over taps t and input channels c of in[v + off_t, c] w[n, t, c],
// a GEMM with M = voxels, N = output channels and K = 27 C.  K is split into "chunks" of 8
// channels of one tap (chunk kc = t (C/8) + c8); one MMA (K = 16) takes two chunks.  For each
// chunk the producer loads a TMA box {8 channels, bx, by, bz voxels} of the input at the tap's
// offset: 128 voxel rows x 16 bytes, one K-major core-matrix column of the A operand, with the
// zero halo supplied by TMA's out-of-bounds fill.  Weights are packed once per update into the
// B operand's order (Wp[kc][n][8]) and fetched with one bulk copy per MMA.  A concatenated input
// (the U-Net's skip connections) is two source maps: chunks of the first C0 channels come from
// the first, the rest from the second.
//
// The data gradient of a convolution is a convolution of the output gradient with the weights
// flipped in space and transposed in channels (w'[c, 26 - t, n] = w[n, t, c]), so it runs on
// the same kernel with differently packed weights.  The weight gradient
//     dw[n, t, c] = sum over voxels v of g[v, n] in[v + off_t, c]
// is a GEMM with K = voxels: M = 128 rows of (tap, channel) pairs (16 chunks), N = output
// channels, both operands MN-major (channels contiguous), split over voxel ranges across blocks
// and added into dw with float atomics.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "hz_internal.h"
#include "hz_net_internal.h"
#include "hz_tc.cuh"

namespace hz {
namespace {

constexpr int CT = 128;        // threads of a convolution block (4 warps)
constexpr int FWD_STAGES = 4;  // pipeline depth of the forward kernel
constexpr int WG_STAGES = 3;   // of the weight-gradient kernel
constexpr int WG_ROWS = 64;    // voxels per weight-gradient K block

struct ChunkMap {
  int cpt;   // chunks per tap (input channels / 8)
  int c0;    // chunks of the first source (its channels / 8)
  int nchunk;
};

// Tap, source and the source's channel offset of chunk kc.
__device__ __forceinline__ void chunk_of(const ChunkMap& cm, int kc, int& dz, int& dy, int& dx,
                                         int& src, int& coff) {
  const int t = kc / cm.cpt, c8 = kc - t * cm.cpt;
  dz = t / 9 - 1;
  dy = (t / 3) % 3 - 1;
  dx = t % 3 - 1;
  src = c8 < cm.c0 ? 0 : 1;
  coff = 8 * (src == 0 ? c8 : c8 - cm.c0);
}

struct FwdArgs {
  CUtensorMap src[2];
  ChunkMap cm;
  const __nv_bfloat16* wp;  // [nchunk rounded up to even][N][8]
  const float* bias;        // [N] or null
  int N;
  int D, H, W;
  int bx, by, bz, tx, ty;   // tile box and tiles along x, y
  int stage_bytes;
  // epilogue
  int relu;
  __nv_bfloat16* out16;     // [vox][N] or null
  float* out32;             // [vox][N] (mode 0) or null
  float* outa;              // split fp32 outputs: channels [0, na) -> outa [vox][na]
  float* outb;              //                    channels [na, N) -> outb [vox][N - na]
  int na, acc_a, acc_b;
  int* err;
  // split over K (layers with few voxel tiles): blockIdx.z takes MMA steps [z ks, (z+1) ks) and
  // adds its raw sums into acc (fp32 [vox][N], zeroed first); k_conv_finalize then applies
  // the epilogue.  ks = 0: one block per tile does every step and the epilogue itself.
  int ks;
  float* acc;
};

// The epilogue of 16 output channels c0.. of voxel vox: bias, ReLU, then the stores asked for.
__device__ __forceinline__ void conv_epilogue16(const FwdArgs& a, long long vox, int c0,
                                                float* v) {
  const int N = a.N;
  if (a.bias) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += a.bias[c0 + j];
  }
  if (a.relu) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
  }
  if (a.out16) {
    uint4 pk[2];
    uint32_t* pw = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      pw[j] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    uint4* dst = reinterpret_cast<uint4*>(a.out16 + vox * N + c0);
    dst[0] = pk[0];
    dst[1] = pk[1];
  }
  if (a.out32) {
    float4* dst = reinterpret_cast<float4*>(a.out32 + vox * N + c0);
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  }
  if (a.outa) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = c0 + j;
      if (n < a.na) {
        float* d = a.outa + vox * a.na + n;
        *d = a.acc_a ? *d + v[j] : v[j];
      } else {
        float* d = a.outb + vox * (N - a.na) + (n - a.na);
        *d = a.acc_b ? *d + v[j] : v[j];
      }
    }
  }
}

__global__ void __launch_bounds__(CT) k_conv_fwd(const __grid_constant__ FwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[FWD_STAGES], empty[FWD_STAGES], done;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, b = blockIdx.y;
  const int x0 = (tile % a.tx) * a.bx;
  const int y0 = ((tile / a.tx) % a.ty) * a.by;
  const int z0 = (tile / (a.tx * a.ty)) * a.bz;
  const int N = a.N;
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  const int nsteps_all = (a.cm.nchunk + 1) / 2;
  const int s_first = a.ks > 0 ? (int)blockIdx.z * a.ks : 0;
  const int nsteps = a.ks > 0 ? min(a.ks, nsteps_all - s_first) : nsteps_all;
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 32) {
    for (int s = 0; s < FWD_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const uint32_t sbase = tc::su32(smem);

  if (threadIdx.x == 0) {
    // producer: two A chunks (TMA) and their B slice (bulk) per stage
    const uint32_t bbytes = 2u * N * 16u;
    int issued = 0;
    for (int s = 0; s < nsteps; ++s) {
      const int st = s % FWD_STAGES;
      const uint32_t ph = (uint32_t)(s / FWD_STAGES) & 1u;
      if (s >= FWD_STAGES && !tc::mbar_wait(&empty[st], ph ^ 1u)) {
        atomicExch(a.err, 1);
        break;
      }
      uint8_t* sa = smem + (size_t)st * a.stage_bytes;
      const int gs = s_first + s;  // the step's place in the whole K loop
      tc::mbar_expect_tx(&full[st], 2u * 2048u + bbytes);
      for (int h = 0; h < 2; ++h) {
        // a padding chunk past the last re-reads the last one (its weights are zero)
        const int kc = min(2 * gs + h, a.cm.nchunk - 1);
        int dz, dy, dx, src, coff;
        chunk_of(a.cm, kc, dz, dy, dx, src, coff);
        tc::tma_load5(sa + h * 2048, &a.src[src], &full[st], coff, x0 + dx, y0 + dy, z0 + dz, b);
      }
      tc::bulk_load(sa + 4096, a.wp + (size_t)2 * gs * N * 8, bbytes, &full[st]);
      issued = s + 1;
    }
    // no copy may still be in flight when the block exits
    for (int s = max(0, issued - FWD_STAGES); s < issued; ++s)
      if (!tc::mbar_wait(&full[s % FWD_STAGES], (uint32_t)(s / FWD_STAGES) & 1u))
        atomicExch(a.err, 1);
  } else if (threadIdx.x == 32) {
    // MMA issuer
    const uint32_t idesc = tc::idesc_bf16(128, N, 0, 0);
    for (int s = 0; s < nsteps; ++s) {
      const int st = s % FWD_STAGES;
      if (!tc::mbar_wait(&full[st], (uint32_t)(s / FWD_STAGES) & 1u)) {
        atomicExch(a.err, 1);
        break;
      }
      tc::fence_after();
      const uint32_t sa = sbase + (uint32_t)st * a.stage_bytes;
      const uint64_t ad = tc::sdesc(sa, 2048, 128);
      const uint64_t bd = tc::sdesc(sa + 4096, (uint32_t)N * 16u, 128);
      tc::mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
      tc::mma_commit(&empty[st]);
    }
    tc::mma_commit(&done);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&done, 0));
  tc::fence_after();
  if (ok) {
    const int r = warp * 32 + lane;
    const int x = x0 + r % a.bx, y = y0 + (r / a.bx) % a.by, z = z0 + r / (a.bx * a.by);
    const bool in = x < a.W && y < a.H && z < a.D;
    const long long vox = (((long long)b * a.D + z) * a.H + y) * a.W + x;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (!in) continue;
      if (a.ks > 0) {
        float* d = a.acc + vox * N + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(d + j, v[j]);
      } else {
        conv_epilogue16(a, vox, c0, v);
      }
    }
  } else if (lane == 0) {
    atomicExch(a.err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// The epilogue of a split convolution: acc holds the summed raw outputs.
__global__ void __launch_bounds__(256) k_conv_finalize(const __grid_constant__ FwdArgs a,
                                                       long long nvox) {
  const int groups = a.N / 16;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox * groups) return;
  const long long vox = i / groups;
  const int c0 = (int)(i - vox * groups) * 16;
  float v[16];
  const float4* src = reinterpret_cast<const float4*>(a.acc + vox * a.N + c0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 q = src[j];
    v[4 * j] = q.x;
    v[4 * j + 1] = q.y;
    v[4 * j + 2] = q.z;
    v[4 * j + 3] = q.w;
  }
  conv_epilogue16(a, vox, c0, v);
}

// ------------------------------------------------------------------ halo-tile forward kernel
// The same convolution for N <= 64 output channels and W a multiple of 8, with the input read
// once per tile instead of once per tap: the block's tile is 8 x 16 x 1 voxels (x, y, z), and
// for each 8-channel chunk one TMA box {8 channels, 10, 18, 3} -- the tile with a one-voxel halo
// on every side, 540 rows of 16 bytes in x-fastest order -- lands in shared memory.  The A
// operand of tap (dx, dy, dz) is then a window of that box: core matrix k (output rows 8k..8k+7,
// y = k, x = 0..7) starts at row (dz+1) 180 + (dy+1) 10 + (dx+1) + 10 k, so the descriptor takes
// the tap's start address and SBO = 10 rows (160 bytes); the second K core matrix of an MMA is the
// next chunk's box (LBO = the box spacing).  With 8 input channels (one chunk per tap) an MMA
// pairs taps t and t+1 of the same box instead (LBO = their row distance; the 28th tap is the
// zero-weight padding chunk).  Per chunk pair: two box loads, 27 bulk copies of the taps' weight
// slices, 27 MMAs.
constexpr int HX = 10, HY = 18, HZ = 3;
constexpr int HALO_BYTES = 8704;  // 540 rows x 16 bytes = 8640, to a multiple of 128
constexpr int HALO_STAGES = 2;

struct HaloArgs {
  CUtensorMap src[2];  // boxes {8, 10, 18, 3, 1}
  ChunkMap cm;
  const __nv_bfloat16* wp;  // [nchunk rounded up to even][N][8]
  int N, D, H, W, tx, ty;   // tiles: tx = W / 8 along x, ty along y (16 rows), D along z
  int ngroups;              // chunk pairs (cpt / 2), or 1 when cpt == 1
  int nh;                   // boxes per group: 2, or 1
  int nmma;                 // MMAs per group: 27, or 14
  int bbytes;               // weight bytes per group
  int stage_bytes;
  FwdArgs epi;              // the epilogue's fields (bias, relu, outputs; ks = 0)
};

__device__ __forceinline__ int tap_row(int t) { return (t / 9) * HX * HY + ((t / 3) % 3) * HX + t % 3; }

__global__ void __launch_bounds__(CT) k_conv_fwd_halo(const __grid_constant__ HaloArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[HALO_STAGES], empty[HALO_STAGES], done;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, b = blockIdx.y;
  const int x0 = (tile % a.tx) * 8;
  const int y0 = ((tile / a.tx) % a.ty) * 16;
  const int z0 = tile / (a.tx * a.ty);
  const int N = a.N;
  const uint32_t ncols = N <= 32 ? 32 : 64;
  int* err = a.epi.err;
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 32) {
    for (int s = 0; s < HALO_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
  }
  // the 64 bytes after each box are never loaded but read by the last tap pair of the 8-channel
  // case (times zero weights): zero them, so that no stale NaN of an earlier kernel gets in
  for (int i = threadIdx.x; i < HALO_STAGES * a.nh * 4; i += CT) {
    const int box = i >> 2, row = i & 3;
    uint8_t* p = smem + (size_t)(box / a.nh) * a.stage_bytes + (box % a.nh) * HALO_BYTES +
                 HX * HY * HZ * 16 + row * 16;
    *reinterpret_cast<uint4*>(p) = make_uint4(0u, 0u, 0u, 0u);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const uint32_t sbase = tc::su32(smem);
  const int cpt = a.cm.cpt;

  if (threadIdx.x == 0) {
    int issued = 0;
    for (int g = 0; g < a.ngroups; ++g) {
      const int st = g % HALO_STAGES;
      const uint32_t ph = (uint32_t)(g / HALO_STAGES) & 1u;
      if (g >= HALO_STAGES && !tc::mbar_wait(&empty[st], ph ^ 1u)) {
        atomicExch(err, 1);
        break;
      }
      uint8_t* sa = smem + (size_t)st * a.stage_bytes;
      uint8_t* sb = sa + a.nh * HALO_BYTES;
      tc::mbar_expect_tx(&full[st], (uint32_t)(a.nh * HX * HY * HZ * 16 + a.bbytes));
      for (int h = 0; h < a.nh; ++h) {
        const int c8 = a.nh == 2 ? 2 * g + h : 0;
        const int src = c8 < a.cm.c0 ? 0 : 1;
        const int coff = 8 * (src == 0 ? c8 : c8 - a.cm.c0);
        tc::tma_load5(sa + h * HALO_BYTES, &a.src[src], &full[st], coff, x0 - 1, y0 - 1, z0 - 1,
                      b);
      }
      if (a.nh == 2) {
        const uint32_t piece = 2u * N * 16u;  // chunks t cpt + 2g and + 1 of tap t
        for (int t = 0; t < 27; ++t)
          tc::bulk_load(sb + t * piece, a.wp + ((size_t)t * cpt + 2 * g) * N * 8, piece, &full[st]);
      } else {
        tc::bulk_load(sb, a.wp, (uint32_t)a.bbytes, &full[st]);  // all 28 chunks
      }
      issued = g + 1;
    }
    for (int g = max(0, issued - HALO_STAGES); g < issued; ++g)
      if (!tc::mbar_wait(&full[g % HALO_STAGES], (uint32_t)(g / HALO_STAGES) & 1u))
        atomicExch(err, 1);
  } else if (threadIdx.x == 32) {
    const uint32_t idesc = tc::idesc_bf16(128, N, 0, 0);
    for (int g = 0; g < a.ngroups; ++g) {
      const int st = g % HALO_STAGES;
      if (!tc::mbar_wait(&full[st], (uint32_t)(g / HALO_STAGES) & 1u)) {
        atomicExch(err, 1);
        break;
      }
      tc::fence_after();
      const uint32_t sa = sbase + (uint32_t)st * a.stage_bytes;
      const uint32_t sb = sa + (uint32_t)a.nh * HALO_BYTES;
      for (int i = 0; i < a.nmma; ++i) {
        uint32_t aaddr, lbo, baddr;
        if (a.nh == 2) {
          aaddr = sa + 16u * tap_row(i);
          lbo = HALO_BYTES;
          baddr = sb + (uint32_t)i * 2u * N * 16u;
        } else {
          const int t = 2 * i;
          aaddr = sa + 16u * tap_row(t);
          lbo = t + 1 < 27 ? 16u * (tap_row(t + 1) - tap_row(t)) : 16u;
          baddr = sb + (uint32_t)t * N * 16u;
        }
        const uint64_t ad = tc::sdesc(aaddr, lbo, HX * 16);
        const uint64_t bd = tc::sdesc(baddr, (uint32_t)N * 16u, 128);
        tc::mma_bf16(tmem, ad, bd, idesc, (g > 0 || i > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[st]);
    }
    tc::mma_commit(&done);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&done, 0));
  tc::fence_after();
  if (ok) {
    const int r = warp * 32 + lane;
    const int x = x0 + (r & 7), y = y0 + (r >> 3);
    const bool in = y < a.H;
    const long long vox = (((long long)b * a.D + z0) * a.H + y) * a.W + x;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (in) conv_epilogue16(a.epi, vox, c0, v);
    }
  } else if (lane == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

struct WgArgs {
  CUtensorMap src[2];  // inputs of the convolution (boxes of 64 voxels)
  CUtensorMap grad;    // output gradient g (boxes of 64 voxels)
  ChunkMap cm;
  int N;               // output channels of the convolution
  int Cin;
  int D, H, W;
  int bx, by, bz, tx, ty, tiles;  // 64-voxel boxes
  int per_block;       // boxes per block (split over voxels)
  int stage_bytes;
  float* dw;           // [N][27][Cin], added to
  int* err;
};

__global__ void __launch_bounds__(CT) k_conv_wgrad(const __grid_constant__ WgArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[WG_STAGES], empty[WG_STAGES], done;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, b = blockIdx.z;
  const int t0 = blockIdx.y * a.per_block, t1 = min(a.tiles, t0 + a.per_block);
  const int nsteps = max(0, t1 - t0);
  const int N = a.N;
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 32) {
    for (int s = 0; s < WG_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const uint32_t sbase = tc::su32(smem);
  const int abytes = 16 * 1024;  // 16 chunks x 64 rows x 16 bytes

  if (threadIdx.x == 0) {
    int issued = 0;
    for (int s = 0; s < nsteps; ++s) {
      const int st = s % WG_STAGES;
      const uint32_t ph = (uint32_t)(s / WG_STAGES) & 1u;
      if (s >= WG_STAGES && !tc::mbar_wait(&empty[st], ph ^ 1u)) {
        atomicExch(a.err, 1);
        break;
      }
      const int tile = t0 + s;
      const int x0 = (tile % a.tx) * a.bx;
      const int y0 = ((tile / a.tx) % a.ty) * a.by;
      const int z0 = (tile / (a.tx * a.ty)) * a.bz;
      uint8_t* sa = smem + (size_t)st * a.stage_bytes;
      tc::mbar_expect_tx(&full[st], (uint32_t)abytes + (uint32_t)N * 128u);
      for (int g = 0; g < 16; ++g) {
        const int kc = min(mt * 16 + g, a.cm.nchunk - 1);
        int dz, dy, dx, src, coff;
        chunk_of(a.cm, kc, dz, dy, dx, src, coff);
        tc::tma_load5(sa + g * 1024, &a.src[src], &full[st], coff, x0 + dx, y0 + dy, z0 + dz, b);
      }
      for (int g = 0; g < N / 8; ++g)
        tc::tma_load5(sa + abytes + g * 1024, &a.grad, &full[st], 8 * g, x0, y0, z0, b);
      issued = s + 1;
    }
    for (int s = max(0, issued - WG_STAGES); s < issued; ++s)
      if (!tc::mbar_wait(&full[s % WG_STAGES], (uint32_t)(s / WG_STAGES) & 1u))
        atomicExch(a.err, 1);
  } else if (threadIdx.x == 32) {
    const uint32_t idesc = tc::idesc_bf16(128, N, 1, 1);
    for (int s = 0; s < nsteps; ++s) {
      const int st = s % WG_STAGES;
      if (!tc::mbar_wait(&full[st], (uint32_t)(s / WG_STAGES) & 1u)) {
        atomicExch(a.err, 1);
        break;
      }
      tc::fence_after();
      const uint32_t sa = sbase + (uint32_t)st * a.stage_bytes;
#pragma unroll
      for (int i = 0; i < WG_ROWS / 16; ++i) {
        const uint64_t ad = tc::sdesc(sa + i * 256, 128, 1024);
        const uint64_t bd = tc::sdesc(sa + abytes + i * 256, 128, 1024);
        tc::mma_bf16(tmem, ad, bd, idesc, (s > 0 || i > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[st]);
    }
    tc::mma_commit(&done);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&done, 0));
  tc::fence_after();
  if (ok && nsteps > 0) {
    const int r = warp * 32 + lane;  // row m of the M tile: chunk mt*16 + r/8, channel r%8
    const int kc = mt * 16 + r / 8;
    const bool valid = kc < a.cm.nchunk;
    int t = 0, ci = 0;
    if (valid) {
      t = kc / a.cm.cpt;
      ci = 8 * (kc - t * a.cm.cpt) + (r & 7);
    }
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (!valid) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        atomicAdd(a.dw + ((long long)(c0 + j) * 27 + t) * a.Cin + ci, v[j]);
    }
  } else if (!ok && lane == 0) {
    atomicExch(a.err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// Packed forward weights: wp[kc][n][e] = w[n][t][8 c8 + e] for chunk kc = t cpt + c8 (zero for
// the padding chunk).  flip: the data-gradient packing of the same convolution, whose input
// channels are w's outputs: wp[kc][c][e] = w[8 c8 + e][26 - t][c].
__global__ void k_pack_weights(const float* __restrict__ w, __nv_bfloat16* __restrict__ wp,
                               int Cin, int Cout, int flip, int nchunk_pad) {
  const int Kc = flip ? Cout : Cin;   // channels the packed chunks run over
  const int Nn = flip ? Cin : Cout;   // rows of the packed operand
  const int cpt = Kc / 8;
  const long long total = (long long)nchunk_pad * Nn * 8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i % 8);
    const int n = (int)((i / 8) % Nn);
    const int kc = (int)(i / (8LL * Nn));
    float val = 0.f;
    if (kc < 27 * cpt) {
      const int t = kc / cpt, k = 8 * (kc % cpt) + e;
      val = flip ? w[((long long)k * 27 + (26 - t)) * Cin + n] : w[((long long)n * 27 + t) * Cin + k];
    }
    wp[i] = __float2bfloat16_rn(val);
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Resolves the tensor-map encoder and sets the kernels' shared-memory limits (once; before any
// launch, so that no attribute call happens while a stream is being captured).
cudaError_t tma_encoder_init() {
  if (g_encode) return cudaSuccess;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (!fn || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
  e = cudaFuncSetAttribute(k_conv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           FWD_STAGES * (4096 + 8192));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             WG_STAGES * (16 * 1024 + 128 * 128));
  if (e == cudaSuccess)  // N <= 64: two boxes and 27 x 2 x 64 x 16 bytes of weights per stage
    e = cudaFuncSetAttribute(k_conv_fwd_halo, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             HALO_STAGES * ((2 * HALO_BYTES + 27 * 2 * 64 * 16 + 1023) / 1024 *
                                            1024));
  if (e != cudaSuccess) return e;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// 5-d map {C, W, H, D, B} of a channels-last bf16 map, box {8, bx, by, bz, 1}.
static cudaError_t encode_map(CUtensorMap* m, const FMap& f, int bx, int by, int bz) {
  if (!g_encode) return cudaErrorNotSupported;
  cuuint64_t dims[5] = {(cuuint64_t)f.C, (cuuint64_t)f.W, (cuuint64_t)f.H, (cuuint64_t)f.D,
                        (cuuint64_t)f.B};
  cuuint64_t str[4] = {(cuuint64_t)f.C * 2, (cuuint64_t)f.C * 2 * f.W,
                       (cuuint64_t)f.C * 2 * f.W * f.H, (cuuint64_t)f.C * 2 * f.W * f.H * f.D};
  cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)f.p, dims, str, box,
                              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Box of n voxels (a power of two) for a W x H x D map: x first, up to 32 wide.
static void box_for(int n, int W, int H, int& bx, int& by, int& bz) {
  bx = 8;
  while (bx < 32 && bx < W) bx *= 2;
  if (bx > n) bx = n;
  by = 1;
  while (bx * by * 2 <= n && by < H) by *= 2;
  bz = n / (bx * by);
}

static bool map_ok(const FMap& f) {
  return f.p && f.C >= 8 && f.C % 8 == 0 && f.W >= 1 && f.H >= 1 && f.D >= 1 && f.B >= 1 &&
         (reinterpret_cast<uintptr_t>(f.p) & 15) == 0;
}

int conv_nchunk_pad(int Cin) { return (27 * (Cin / 8) + 1) / 2 * 2; }

cudaError_t launch_pack_weights(const float* w, __nv_bfloat16* wp, int Cin, int Cout, int flip,
                                cudaStream_t st) {
  const int Kc = flip ? Cout : Cin, Nn = flip ? Cin : Cout;
  const int ncp = conv_nchunk_pad(Kc);
  const long long total = (long long)ncp * Nn * 8;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  count_launch();
  k_pack_weights<<<blocks, 256, 0, st>>>(w, wp, Cin, Cout, flip, ncp);
  return cudaGetLastError();
}

cudaError_t launch_conv_fwd(const FMap& in0, const FMap* in1, const __nv_bfloat16* wp,
                            const float* bias, int N, int relu, __nv_bfloat16* out16,
                            float* out32, float* outa, float* outb, int na, int acc_a, int acc_b,
                            int* err, cudaStream_t st, float* scratch, long long scratch_floats,
                            int sms) {
  if (!map_ok(in0) || (in1 && (!map_ok(*in1) || in1->W != in0.W || in1->H != in0.H ||
                               in1->D != in0.D || in1->B != in0.B)))
    return cudaErrorInvalidValue;
  if (N < 16 || N > 256 || N % 16 != 0 || !wp || !err) return cudaErrorInvalidValue;
  if (outa && (!outb && na < N)) return cudaErrorInvalidValue;
  if ((out16 && (reinterpret_cast<uintptr_t>(out16) & 15)) ||
      (out32 && (reinterpret_cast<uintptr_t>(out32) & 15)))
    return cudaErrorInvalidValue;
  FwdArgs a;
  std::memset(&a, 0, sizeof(a));
  const int cin = in0.C + (in1 ? in1->C : 0);
  {
    // the halo-tile kernel where it applies: N <= 64 (two stages fit), W a multiple of 8, enough
    // tiles for the device (or no scratch to split the per-tap kernel's K loop with)
    const int cpt = cin / 8;
    const long long htiles = (long long)(in0.W / 8) * ((in0.H + 15) / 16) * in0.D * in0.B;
    const bool fits = N <= 64 && in0.W % 8 == 0 && (cpt == 1 || cpt % 2 == 0);
    if (fits && (htiles >= sms || !scratch)) {
      HaloArgs h;
      std::memset(&h, 0, sizeof(h));
      cudaError_t e = encode_map(&h.src[0], in0, HX, HY, HZ);
      if (e != cudaSuccess) return e;
      e = encode_map(&h.src[1], in1 ? *in1 : in0, HX, HY, HZ);
      if (e != cudaSuccess) return e;
      h.cm.cpt = cpt;
      h.cm.c0 = in0.C / 8;
      h.cm.nchunk = 27 * cpt;
      h.wp = wp;
      h.N = N;
      h.D = in0.D;
      h.H = in0.H;
      h.W = in0.W;
      h.tx = in0.W / 8;
      h.ty = (in0.H + 15) / 16;
      h.nh = cpt == 1 ? 1 : 2;
      h.ngroups = cpt == 1 ? 1 : cpt / 2;
      h.nmma = cpt == 1 ? 14 : 27;
      h.bbytes = cpt == 1 ? conv_nchunk_pad(8) * N * 16 : 27 * 2 * N * 16;
      h.stage_bytes = (h.nh * HALO_BYTES + h.bbytes + 1023) / 1024 * 1024;
      h.epi.bias = bias;
      h.epi.N = N;
      h.epi.relu = relu;
      h.epi.out16 = out16;
      h.epi.out32 = out32;
      h.epi.outa = outa;
      h.epi.outb = outb;
      h.epi.na = na;
      h.epi.acc_a = acc_a;
      h.epi.acc_b = acc_b;
      h.epi.err = err;
      const size_t smem = (size_t)HALO_STAGES * h.stage_bytes;
      count_launch();
      k_conv_fwd_halo<<<dim3((unsigned)(h.tx * h.ty * in0.D), (unsigned)in0.B), CT, smem, st>>>(
          h);
      return cudaGetLastError();
    }
  }
  box_for(128, in0.W, in0.H, a.bx, a.by, a.bz);
  cudaError_t e = encode_map(&a.src[0], in0, a.bx, a.by, a.bz);
  if (e != cudaSuccess) return e;
  e = encode_map(&a.src[1], in1 ? *in1 : in0, a.bx, a.by, a.bz);
  if (e != cudaSuccess) return e;
  a.cm.cpt = cin / 8;
  a.cm.c0 = in0.C / 8;
  a.cm.nchunk = 27 * a.cm.cpt;
  a.wp = wp;
  a.bias = bias;
  a.N = N;
  a.D = in0.D;
  a.H = in0.H;
  a.W = in0.W;
  a.tx = (in0.W + a.bx - 1) / a.bx;
  a.ty = (in0.H + a.by - 1) / a.by;
  const int tz = (in0.D + a.bz - 1) / a.bz;
  a.stage_bytes = 4096 + (2 * N * 16 + 1023) / 1024 * 1024;
  a.relu = relu;
  a.out16 = out16;
  a.out32 = out32;
  a.outa = outa;
  a.outb = outb;
  a.na = na;
  a.acc_a = acc_a;
  a.acc_b = acc_b;
  a.err = err;
  const size_t smem = (size_t)FWD_STAGES * a.stage_bytes;
  // layers with fewer voxel tiles than about two per SM split their K loop over blocks (at
  // least 4 MMA steps each) when a scratch of vox x N floats is given
  const long long tiles = (long long)a.tx * a.ty * tz * in0.B;
  const long long nvox = (long long)in0.W * in0.H * in0.D * in0.B;
  const int nsteps = (a.cm.nchunk + 1) / 2;
  int nsplit = 1;
  if (scratch && scratch_floats >= nvox * N && tiles < 2LL * sms) {
    nsplit = (int)std::min<long long>((2LL * sms + tiles - 1) / tiles, std::max(1, nsteps / 4));
    if (nsplit > 1) {
      a.ks = (nsteps + nsplit - 1) / nsplit;
      nsplit = (nsteps + a.ks - 1) / a.ks;
    }
  }
  if (nsplit > 1) {
    a.acc = scratch;
    cudaError_t me = cudaMemsetAsync(scratch, 0, sizeof(float) * (size_t)(nvox * N), st);
    if (me != cudaSuccess) return me;
  } else {
    a.ks = 0;
  }
  count_launch();
  k_conv_fwd<<<dim3((unsigned)(a.tx * a.ty * tz), (unsigned)in0.B, (unsigned)nsplit), CT, smem,
               st>>>(a);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess || nsplit == 1) return le;
  count_launch();
  const long long items = nvox * (N / 16);
  k_conv_finalize<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(a, nvox);
  return cudaGetLastError();
}

cudaError_t launch_conv_wgrad(const FMap& in0, const FMap* in1, const FMap& grad, float* dw,
                              int* err, int sms, cudaStream_t st) {
  if (!map_ok(in0) || !map_ok(grad) ||
      (in1 && (!map_ok(*in1) || in1->W != in0.W || in1->H != in0.H || in1->D != in0.D ||
               in1->B != in0.B)) ||
      grad.W != in0.W || grad.H != in0.H || grad.D != in0.D || grad.B != in0.B)
    return cudaErrorInvalidValue;
  const int N = grad.C;
  if (N < 16 || N > 128 || N % 16 != 0 || !dw || !err) return cudaErrorInvalidValue;
  WgArgs a;
  std::memset(&a, 0, sizeof(a));
  box_for(WG_ROWS, in0.W, in0.H, a.bx, a.by, a.bz);
  cudaError_t e = encode_map(&a.src[0], in0, a.bx, a.by, a.bz);
  if (e != cudaSuccess) return e;
  e = encode_map(&a.src[1], in1 ? *in1 : in0, a.bx, a.by, a.bz);
  if (e != cudaSuccess) return e;
  e = encode_map(&a.grad, grad, a.bx, a.by, a.bz);
  if (e != cudaSuccess) return e;
  const int cin = in0.C + (in1 ? in1->C : 0);
  a.cm.cpt = cin / 8;
  a.cm.c0 = in0.C / 8;
  a.cm.nchunk = 27 * a.cm.cpt;
  a.N = N;
  a.Cin = cin;
  a.D = in0.D;
  a.H = in0.H;
  a.W = in0.W;
  a.tx = (in0.W + a.bx - 1) / a.bx;
  a.ty = (in0.H + a.by - 1) / a.by;
  const int tz = (in0.D + a.bz - 1) / a.bz;
  a.tiles = a.tx * a.ty * tz;
  const int mtiles = (a.cm.nchunk + 15) / 16;
  // enough blocks for about two waves, each with at least 8 voxel boxes
  const long long want = 2LL * std::max(sms, 1);
  long long splits = std::max<long long>(1, want / std::max(1, mtiles * in0.B));
  splits = std::min<long long>(splits, std::max(1, a.tiles / 8));
  a.per_block = (int)((a.tiles + splits - 1) / splits);
  splits = (a.tiles + a.per_block - 1) / a.per_block;
  a.stage_bytes = 16 * 1024 + N * 128;
  a.dw = dw;
  a.err = err;
  const size_t smem = (size_t)WG_STAGES * a.stage_bytes;
  count_launch();
  k_conv_wgrad<<<dim3((unsigned)mtiles, (unsigned)splits, (unsigned)in0.B), CT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hz
