// Internal declarations of the learned preconditioner (hz_conv.cu, hz_net.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "hz.h"

namespace hz {

// A channels-last bf16 feature map: B samples of D x H x W voxels with C channels each.
struct FMap {
  const void* p;
  int C, W, H, D, B;
};

// Resolve the driver's tensor-map encoder (once per process).
cudaError_t tma_encoder_init();

// Chunks of 8 channels over the 27 taps for Cin input channels, rounded up to an even count
// (one MMA takes two).
int conv_nchunk_pad(int Cin);

// Pack fp32 weights w[Cout][27][Cin] into the bf16 B-operand order of the forward kernel
// (flip = 0: wp[kc][Cout][8]) or of the data-gradient convolution (flip = 1: wp[kc][Cin][8],
// taps mirrored, channels transposed).
cudaError_t launch_pack_weights(const float* w, __nv_bfloat16* wp, int Cin, int Cout, int flip,
                                cudaStream_t st);

// out = conv3(in0 ++ in1, wp) (+ bias, relu): bf16 [vox][N] into out16, fp32 into out32, or
// split fp32 outputs (channels [0, na) into outa, the rest into outb; acc_*: add instead of
// store).  N a multiple of 16 in [16, 256].  err: set if a bounded wait gave up.
// scratch (vox x N floats, may be null): lets layers with few voxel tiles split their K loop
// over blocks (sms: the device's SM count).
cudaError_t launch_conv_fwd(const FMap& in0, const FMap* in1, const __nv_bfloat16* wp,
                            const float* bias, int N, int relu, __nv_bfloat16* out16,
                            float* out32, float* outa, float* outb, int na, int acc_a, int acc_b,
                            int* err, cudaStream_t st, float* scratch = nullptr,
                            long long scratch_floats = 0, int sms = 152);

// dw[N][27][Cin] += sum over voxels of grad[v][n] (in0 ++ in1)[v + off_t][c]; N = grad.C a
// multiple of 16 in [16, 128].
cudaError_t launch_conv_wgrad(const FMap& in0, const FMap* in1, const FMap& grad, float* dw,
                              int* err, int sms, cudaStream_t st);

// The network's z = N(r) for nvec complex128 fields of an nx x ny x nz grid (field b of r at
// r + b rrs, of z at z + b zrs), m the medium channel (c_min^2 / c^2 per point); z is written,
// or added to when accumulate is set.
hz_status net_apply_field(hz_net* n, const double2* r, long long rrs, const double* m, double2* z,
                          long long zrs, int nvec, int nx, int ny, int nz, int accumulate,
                          cudaStream_t st);
// One Adam training step on (r, e) field pairs (contiguous, nvec of n each).
hz_status net_train_fields(hz_net* n, const double2* r, const double* m, const double2* e,
                           int nvec, int nx, int ny, int nz, float lr, double* loss,
                           cudaStream_t st);
// The network's bounded waits: HZ_ERR_TIMEOUT once if one gave up (after a synchronisation).
hz_status net_check(hz_net* n);
bool net_fits(const hz_net* n, int nvec, int nx, int ny, int nz);
// t = v - a, dst += src (strided fields)
cudaError_t launch_field_sub(const double2* v, long long vrs, const double2* a, long long ars,
                             double2* t, long long trs, long long n, int nvec, cudaStream_t st);
cudaError_t launch_field_add(double2* dst, long long drs, const double2* src, long long srs,
                             long long n, int nvec, cudaStream_t st);
// z *= d per field, d the step of the last step-d reduction in gs (scal[SC_DR], scal[SC_DI]).
cudaError_t launch_scale_by_step(double2* z, long long zrs, const GmresDev& gs, long long n,
                                 int nvec, cudaStream_t st);

}  // namespace hz
