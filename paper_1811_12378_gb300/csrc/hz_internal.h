// Internal declarations shared by the translation units of libhz (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "hz.h"

namespace hz {

constexpr int MAXJ = 16;          // contour nodes per problem
constexpr int RED_THREADS = 256;  // threads of a reduction block
constexpr int RED_PPT = 4;        // points per thread in a reduction block
constexpr int RED_CHUNK = RED_THREADS * RED_PPT;
constexpr unsigned GRID_SPINS_DEFAULT = 1u << 23;  // grid-barrier poll limit: about a second
constexpr int RED_MIN_CHUNK = 256;  // smallest points per block of any reduction kernel
                                    // (sizes the per-block partial sums)

// Grid geometry and the scalars of the normalised operator (A = s L_h - diag(m) - i diag(a)).
struct Geom {
  int nx, ny, nz;
  int layer;       // sponge cells
  long long n;     // nx*ny*nz
  double cs;       // s / h^2: weight of the 7-point Laplacian
  double sig;      // sigma_max of the sponge
  float csf;       // s / h^2 in float32, so float32 kernels convert nothing
  // tile shapes chosen by the autotuner at problem creation (kernel launch parameters only)
  int pzc[3];      // polynomial stage: z-column length for 1, 2-3, >= 4 active nodes
  int prows[3];    // polynomial stage: grid rows per block for the same classes
  int szc, srows;  // complex64 stencil: z-column length, rows per block
};

// Node-count class of a polynomial stage for the tile tables above.
inline int stage_class(int nnodes) { return nnodes >= 4 ? 2 : (nnodes >= 2 ? 1 : 0); }

// Per-node parameters of the polynomial scheme (eq:fix-pt-exp) and the quadrature (§6).
struct NodeParams {
  double zr, zi;     // node z_j
  double sr, si;     // weight sigma_j
  double z0r, z0i;   // Taylor centre z0 = (b1+b2)/2 + i Im z_j
  double delta;      // real step
  double nu;         // predicted rate (eq:fix-pt-conv)
  int q;             // polynomial order
  int sweeps;        // fixed-point sweeps per shifted solve
};

// A device buffer of one field per right-hand side: field r at p + r*rs (elements).
template <typename T>
struct Buf {
  T* p;
  long long rs;
};

enum StageKind { SK_NONE = 0, SK_FIRST = 1, SK_MID = 2, SK_LAST = 3, SK_FIRST_LAST = 4 };

// What one node does in one stage (one stencil sweep) of the batched polynomial solve.
//   FIRST      k = mdi((A - z0) y - f),   acc = y + k                (yzero: y = 0, no stencil)
//   MID        k = mdi((A - z0) kin - cf f),   acc += k
//   LAST       y = (acc + mdi((A - z0) kin - cf f)) * ip
//   FIRST_LAST y_out = (y + mdi((A - z0) y - f)) * ip                 (q = 1)
// With `final_quad` set, LAST / FIRST_LAST add wq * y_new into w instead of storing y.
// The coefficients are held in the kernel's own real type R (float32 sweeps must not spend
// the scarce float64 pipe on conversions); the quadrature weight is always float64.
template <typename R>
struct StageNode {
  R mdr, mdi;        // -i delta / j
  R cfr, cfi;        // coefficient of f
  R z0r, z0i;
  R ipr, ipi;        // 1 / ptilde(z)
  double wqr, wqi;   // sigma_j / z_j
  float wrh, wrl, wih, wil;  // the same split into float pairs (hi + lo) for the complex64 sum
  int kind, yzero;
  long long in, kout, acc, yout;  // element offsets of the node's fields in the rhs workspace
  int lapi;  // spectral problems: index of the node's input in the stage's Laplacian batch
};

template <typename R>
struct StageArgs {
  StageNode<R> nd[MAXJ];
  int nnodes;
  int final_quad;
  int quad64;  // complex64 sweeps: form the quadrature sum in float64 (0: float pairs)
};

// ---------------------------------------------------------------- Fourier spectral (hz_fft.cu)
// The spectral Laplacian S = F^H Lambda F of the periodic box (Section 7.1,
// eq:eig-Laplacian-spectral) and the regularised inverse Laplacian F^H diag(1/max(lambda, 1)) F
// (Section 7.3), applied by line FFTs of the project's own (radices 2, 3, 4, 5).
constexpr int FFT_MAXN = 1024;  // longest grid line of a spectral problem
constexpr int FFT_MAXST = 10;   // radix stages of one line

struct FftAxis {
  int n, nst;
  int rad[FFT_MAXST];
  const double2* tw64;  // exp(-2 pi i k / n), k < n
  const float2* tw32;
  const double* e64;    // s (2 pi min(k, n - k) / (n h))^2, k < n: this axis's share of lambda
  const float* e32;
};

struct SpecPlan {
  FftAxis ax[3];  // x, y, z
};

// nvec fields: field v at (T*)base + (v / nq) * rs + off[v % nq] (elements).
struct VecMap {
  const void* base;
  long long rs;
  int nq;
  long long off[MAXJ];
};

inline VecMap vec_map(const void* p, long long rs) {
  VecMap m{};
  m.base = p;
  m.rs = rs;
  m.nq = 1;
  return m;
}

enum SpecMode { SPEC_APPLY = 0, SPEC_LAP = 1, SPEC_INVLAP = 2 };

// Shared-memory limits of the line-FFT kernels (once per process, before any capture).
cudaError_t fft_prepare();
// Radices of an FFT of length n (false unless n = 2^a 3^b 5^c <= FFT_MAXN).
bool fft_factor(int n, int* rad, int* nst);
// out = (s S - diag(m) - i diag(a) - zI) in (SPEC_APPLY, dg = -m - i a), s S in (SPEC_LAP) or the
// regularised inverse Laplacian of in (SPEC_INVLAP), for nvec fields; tmp holds nvec fields.
template <typename T>
cudaError_t launch_spectral(const SpecPlan& sp, const Geom& g, int mode, const VecMap& in,
                            const VecMap& out, int nvec, const T* dg, double zr, double zi,
                            T* tmp, cudaStream_t st);
// t = sc f - a (nvec fields): the true residual from a precomputed A u.
cudaError_t launch_scaled_sub(const double2* f, long long frs, double sc, const double2* a,
                              long long ars, double2* t, long long trs, long long n, int nvec,
                              cudaStream_t st);
// One stage of the polynomial scheme on a spectral problem: the node inputs' s S x come
// precomputed in lap (field l of right-hand side r at lap + (r * nlap + l) * n).
template <typename T, typename R>
cudaError_t launch_poly_stage_spec(const Geom& g, const T* dg, Buf<const T> f, T* ws,
                                   long long wrs, const T* lap, int nlap, Buf<double2> w,
                                   Buf<float2> w32, int nvec, const StageArgs<R>& a,
                                   cudaStream_t st);

// Per-right-hand-side state of one GMRES / FGMRES cycle on the device.
struct GmresDev {
  int mmax;
  double2* R;      // [r][(mmax+1)*mmax] upper triangle after rotations, column-major
  double* cc;      // [r][mmax] rotation cosines
  double2* ss;     // [r][mmax] rotation sines
  double2* g;      // [r][mmax+1] rotated right-hand side beta e1
  double2* y;      // [r][mmax] least-squares solution
  double2* h1;     // [r][mmax+2] first Gram-Schmidt pass (+ ||w||^2 in slot k+1)
  double2* h2;     // [r][mmax+2] second pass
  double2* nrm;    // [r][2]
  double* scal;    // [r][SC_COUNT]
  int* kend;       // [r] columns of the least-squares problem
  int* stopped;    // [r] 1 once the cycle of this rhs has ended
};

enum { SC_EST = 0, SC_INV = 1, SC_BETA = 2, SC_TOL = 3, SC_HN = 4, SC_DR = 5, SC_DI = 6,
       SC_RES2 = 7, SC_COUNT = 8 };

// Launch counter shared by every kernel wrapper.
extern std::atomic<unsigned long long> g_launches;

// ---- kernel wrappers (hz_kernels.cu); each returns cudaGetLastError() after launch ----
// dg: the operator's diagonal 6 s/h^2 - m - i a per point, in the field's precision.
// On the final stage (a.final_quad) w receives the quadrature sum in float64 and, where w32.p
// is not null, also its complex64 rounding.
template <typename T, typename R>
cudaError_t launch_poly_stage(const Geom& g, const T* dg, Buf<const T> f, T* ws, long long wrs,
                              Buf<double2> w, Buf<float2> w32, int nvec, const StageArgs<R>& a,
                              cudaStream_t st);

// Complex64 (A - zI)x from the complex64 diagonal dg, z-columns of 4 points per thread.
cudaError_t launch_stencil32(const Geom& g, const float2* dg, Buf<const float2> x, Buf<float2> y,
                             int nvec, double zr, double zi, cudaStream_t st);

// Float64 (A - zI)x from the precomputed diagonal dg = 6 s/h^2 - m - i a (one per point).
cudaError_t launch_stencil_diag(const Geom& g, const double2* dg, Buf<const double2> x,
                                Buf<double2> y, int nvec, double zr, double zi, cudaStream_t st);

// The same with complex64 input (FGMRES directions stored in complex64), float64 arithmetic,
// z = 0.
cudaError_t launch_stencil_diag_x32(const Geom& g, const double2* dg, Buf<const float2> x,
                                    Buf<double2> y, int nvec, cudaStream_t st);

cudaError_t launch_convert_c128_c64(Buf<const double2> x, Buf<float2> y, long long n, int nvec,
                                    cudaStream_t st);
cudaError_t launch_convert_c64_c128(Buf<const float2> x, Buf<double2> y, long long n, int nvec,
                                    cudaStream_t st);

// Gram-Schmidt reductions over nb basis fields V_0..V_{nb-1} (V_i of rhs r at
// V + r*vrs + i*vis) and one field w.  mode 0: h1[i] = <V_i, w>, h1[nb] = ||w||^2;
// mode 1: w -= sum_i h1[i] V_i, then h2[i] = <V_i, w>;
// mode 2: w -= sum_i h2[i] V_i, then ||w||^2, then the Givens step of column nb-1.
cudaError_t launch_cgs(int mode, const double2* V, long long vis, long long vrs, int nb,
                       Buf<double2> w, long long n, const GmresDev& gs, double2* partial,
                       unsigned* counters, int nvec, double breakdown, cudaStream_t st);

// dst[r] = src[r] * gs.scal[r][SC_INV]
cudaError_t launch_scale(Buf<double2> dst, Buf<const double2> src, long long n, const GmresDev& gs,
                         int nvec, cudaStream_t st);

// out[r] = (accumulate ? out[r] : 0) + sum_{i<kend[r]} y[r][i] B_i + e_coef[r] * E[r]
cudaError_t launch_combine(Buf<double2> out, const double2* B, long long bis, long long brs,
                           const GmresDev& gs, Buf<const double2> E, int e_slot, int accumulate,
                           long long n, int nvec, int kmax, cudaStream_t st);

// out[r] = (accumulate ? out[r] : 0) + sum_{i<kend[r]} y[r][i] B_i with complex64 fields B.
cudaError_t launch_combine_b32(Buf<double2> out, const float2* B, long long bis, long long brs,
                               const GmresDev& gs, int accumulate, long long n, int nvec,
                               cudaStream_t st);

// y = R^{-1} g over kend[r] columns (one block per rhs)
cudaError_t launch_backsolve(const GmresDev& gs, int nvec, cudaStream_t st);

// ---- float-pair outer Arnoldi of HZ_MIXED_C64_FF (hz_kernels_ff.cu); a complex element is a
// float4 (re.hi, re.lo, im.hi, im.lo) in storage of the double2 layout ----
cudaError_t launch_stencil_diag_ff(const Geom& g, const double2* dg, Buf<const double2> x,
                                   Buf<float4> y, int nvec, cudaStream_t st);
cudaError_t launch_cgs_ff(int mode, const float4* V, long long vis, long long vrs, int nb,
                          Buf<float4> w, long long n, const GmresDev& gs, double2* partial,
                          unsigned* counters, int nvec, double breakdown, cudaStream_t st);
// v *= 1/h (float pairs), and y32 = its complex64 rounding where y32.p is not null.
cudaError_t launch_scale_ff(Buf<float4> v, long long n, const GmresDev& gs, int nvec,
                            cudaStream_t st, Buf<float2> y32);
// dst = src / beta as float pairs (src float64, may be dst's storage), and y32 as above.
cudaError_t launch_scale_ff_from64(Buf<float4> dst, Buf<const double2> src, long long n,
                                   const GmresDev& gs, int nvec, cudaStream_t st,
                                   Buf<float2> y32);

// One-time kernel attributes for restart lengths up to mmax (shared memory of k_backsolve).
cudaError_t prepare_kernels(int mmax);
// The same for the float32 triangular solve of the complex64 FCI form (inner lengths).
cudaError_t prepare_kernels32(int mmax);
// v0 = r - d Aw and the inner cycle start (the second half of launch_fci_step32).
cudaError_t launch_fci_start32(Buf<const float2> Aw, Buf<const float2> r, Buf<float2> v0,
                               const GmresDev& gs, double2* partial, unsigned* counters,
                               long long n, int nvec, cudaStream_t st);
// y = A x (complex64) fused with the reduction that consumes it: kind 0 = the first CGS pass
// (h1 = V^H y over nb fields, ||y||^2), kind 1 = the FCI step size d = (Ax)^H V0 / ||Ax||^2
// with V the single field V0.  Blocks of 512 points.
cudaError_t launch_stencil32_dots(int kind, const Geom& g, const float2* dg, Buf<const float2> x,
                                  Buf<float2> y, const float2* V, long long vis, long long vrs,
                                  int nb, const GmresDev& gs, double2* partial,
                                  unsigned* counters, int nvec, cudaStream_t st);
// ---- the complex64 FCI tail as one cooperative kernel (hz_fci_tail32.cu) ----
constexpr int TAIL_KMAX = 16;
// Points per thread and grid size for n points so that the grid is co-resident (kin inner
// steps); *ppt = 0 where it does not fit or cooperative launch is unavailable.
cudaError_t fci_tail32_plan(long long n, int kin, int* ppt, int* blocks);
// Steps 3-5 of Algorithm 1 for one right-hand side: d from A w32 and f32, inner GMRES(kin) on
// V (kin + 1 fields; W: one scratch field), out = V y + d w64.  bar: 2 zeroed counters; err:
// set on a barrier timeout.  partial: at least 2 (TAIL_KMAX + 2) blocks float4.  pyth: take
// each h_{j+1,j} from ||w||^2 - ||h2||^2 where that does not cancel (0: always sum the norm of
// the last Gram-Schmidt pass).  n < 2^31.
cudaError_t launch_fci_tail32(const Geom& g, const float2* dg, const float2* w32,
                              const float2* f32, const double2* w64, float2* V, float2* W,
                              double2* out,
                              double2* partial, unsigned* bar, int* err, long long n, int kin,
                              double brk, int pyth, int ppt, int blocks, cudaStream_t st);
// ---- Case Two (hz_case_two.cu): y = ((iC - I) - zI) x on stacked fields (x1; x2) per vector,
// C = [[0, I], [-(A1 + I), -A2]] (eq:mat-2x2), from the diagonal dg of A = A1 - i A2 ----
cudaError_t launch_apply_2x2(const Geom& g, const double2* dg, const double2* x, double2* y,
                             int nvec, double zr, double zi, cudaStream_t st);
cudaError_t launch_apply_2x2_32(const Geom& g, const float2* dg, const float2* x, float2* y,
                                int nvec, float zr, float zi, cudaStream_t st);
// the same (float64) with per-vector strides (fields of 2n points at x + r xrs)
cudaError_t launch_apply_2x2_strided(const Geom& g, const double2* dg, const double2* x,
                                     long long xrs, double2* y, long long yrs, int nvec,
                                     double zr, double zi, cudaStream_t st);
// One sweep of eq:fix-pt-exp on iC - I for the active nodes of a stage (float64); f holds
// (f1; f2) per right-hand side, workspace slots are 2n-point fields; every node's final y is
// stored (no fused quadrature).
cudaError_t launch_poly_stage_2x2(const Geom& g, const double2* dg, Buf<const double2> f,
                                  double2* ws, long long wrs, int nvec, const StageArgs<double>& a,
                                  cudaStream_t st);
// w = sum_s (wr_s + i wi_s) y_s with y_s at ws + r wrs + off[s] (nf values per field).
cudaError_t launch_quad_2x2(const double2* ws, long long wrs, Buf<double2> w, long long nf,
                            int nvec, const long long* off, const double* wr, const double* wi,
                            int nn, cudaStream_t st);
// Case Two cycle start: v0 = (0; fs f) - t (t = (iC - I) U, or null for U = 0), beta.
cudaError_t launch_residual_2x2(const double2* f, long long frs, double fs, Buf<const double2> t,
                                Buf<double2> v0, long long n, const GmresDev& gs,
                                double2* partial, unsigned* counters, int nvec, cudaStream_t st);
// ---- one outer float-pair Arnoldi step as one cooperative kernel (hz_arnoldi_ff.cu) ----
// Points per thread and grid size for n points and restart length mmax; *ppt = 0 where the
// grid cannot be co-resident or cooperative launch is unavailable.
cudaError_t arnoldi_ff_plan(long long n, int mmax, int* ppt, int* blocks);
// For one right-hand side and nb = k + 1 basis fields V (float pairs): w = A z (dg: float64
// diagonal), CGS2 against V into gs.h1, gs.h2, gs.nrm, the Givens step of column k, and
// vnext = w / h_{k+1,k} with its complex64 rounding y32.  Does nothing once gs.stopped[0] is
// set.  pyth: take h_{k+1,k} from ||w||^2 - ||h2||^2 where that does not cancel (0: always
// sum the norm of the last pass).  partial: at least 2 (gs.mmax + 2) blocks float4; bar, err
// as launch_fci_tail32.
cudaError_t launch_arnoldi_ff(const Geom& g, const double2* dg, const double2* z,
                              const float4* V, float4* vnext, float2* y32, const GmresDev& gs,
                              double2* partial, unsigned* bar, int* err, long long n, int nb,
                              double brk, int pyth, int ppt, int blocks, cudaStream_t st);
// ---- float64 cooperative kernels of the float64-outer forms (hz_coop64.cu), one right-hand side
// Grid plans (ppt 0: the multi-kernel forms serve).
cudaError_t arnoldi64_plan(long long n, int mmax, int* ppt, int* blocks);
cudaError_t fci_tail64_plan(long long n, int* ppt, int* blocks);
constexpr int TAIL64_KMAX = 4;
// One outer Arnoldi step in float64: w = A z (z double2, or float2 if z32), CGS2 against the nb
// fields V, the Givens step of column nb - 1 and vnext = w / h; partial: 2 (mmax + 2) blocks.
cudaError_t launch_arnoldi64(const Geom& g, const double2* dg, const void* z, int z32,
                             const double2* V, double2* vnext, const GmresDev& gs,
                             double2* partial, unsigned* bar, int* err, long long n, int nb,
                             double brk, int pyth, int ppt, int blocks, cudaStream_t st);
// Algorithm 1 steps 3-5 in float64 (kin <= 4): w the quadrature sum, r the FCI input, V kin + 1
// fields, W one scratch field; partial: 2 (TAIL64_KMAX + 2) blocks.
cudaError_t launch_fci_tail64(const Geom& g, const double2* dg, const double2* w,
                              const double2* r, double2* V, double2* W, double2* out,
                              double2* partial, unsigned* bar, int* err, long long n, int kin,
                              double brk, int pyth, int ppt, int blocks, cudaStream_t st);

// ---- ILU(0) of the 7-point Laplacian, the inner GMRES's right preconditioner (hz_ilu.cu)
// 1 / d_p of M = (D + L) D^{-1} (D + U), K = cs * (7-point stencil), natural order (host).
void ilu0_inverse_pivots(int nx, int ny, int nz, double cs, std::vector<double>& invd);
// Kernel attributes of the sweeps (once, outside any stream capture).
cudaError_t ilu0_prepare();
// The same in float32 arithmetic (float64 fields t and z, complex64 scratch u32), where the
// y-z lines fit in shared memory (ilu0_fits32).
cudaError_t launch_ilu0_32(const Geom& g, const float* invd32, Buf<const double2> t,
                           Buf<float2> u32, Buf<double2> z, int nvec, cudaStream_t st);
bool ilu0_fits32(const Geom& g);
// The same sweeps as a multi-block wavefront over z-slabs (cooperative launches; every wait on
// a neighbouring block bounded by bar[3] polls, giving up sets bar[2]).  prog: scratch of
// ilu0_chain_prog_ints ints.  ilu0_chain_fits: the grid can be co-resident.
bool ilu0_chain_fits(const Geom& g, int nvec, bool f32);
long long ilu0_chain_prog_ints(const Geom& g, int nvec);
cudaError_t launch_ilu0_chain(const Geom& g, const double* invd, Buf<const double2> t,
                              Buf<double2> z, int nvec, int* prog, unsigned* bar,
                              cudaStream_t st);
cudaError_t launch_ilu0_chain32(const Geom& g, const float* invd32, Buf<const double2> t,
                                Buf<float2> u32, Buf<double2> z, int nvec, int* prog,
                                unsigned* bar, cudaStream_t st);
// z = M^{-1} t for nvec fields (t and z must not overlap).
cudaError_t launch_ilu0(const Geom& g, const double* invd, Buf<const double2> t, Buf<double2> z,
                        int nvec, cudaStream_t st);
// out += d w, d = the FCI step size of each right-hand side (gs.scal).
cudaError_t launch_add_dw(Buf<double2> out, Buf<const double2> w, long long n, const GmresDev& gs,
                          int nvec, cudaStream_t st);

// y = R^{-1} g in float32 for the complex64 FCI form's inner GMRES (GmresDev storage float64).
cudaError_t launch_backsolve32(const GmresDev& gs, int nvec, cudaStream_t st);

// Starting vector of a cycle.  v0[r] = f[r] - fscale*A x[r] (x may be null = 0; A applied
// in float64), then ||v0||^2 -> beta, inv, g[0] = beta, kend = 0, stopped = (beta == 0).
cudaError_t launch_residual_start(const Geom& g, const double* m, Buf<const double2> f, double fs,
                                  Buf<const double2> x, Buf<double2> v0, const GmresDev& gs,
                                  double2* partial, unsigned* counters, int nvec, cudaStream_t st);

// FCI step size: d = <Aw, r> / <Aw, Aw> into scal[SC_DR/SC_DI]; then v0 = r - d Aw and the
// inner cycle start as in launch_residual_start.
cudaError_t launch_fci_step(Buf<const double2> Aw, Buf<const double2> r, Buf<double2> v0,
                            const GmresDev& gs, double2* partial, unsigned* counters,
                            long long n, int nvec, cudaStream_t st);

// ---- complex64 FCI internals (hz_kernels32.cu), for HZ_MIXED_C64_FCI32 ----
cudaError_t launch_cgs32(int mode, const float2* V, long long vis, long long vrs, int nb,
                         Buf<float2> w, long long n, const GmresDev& gs, double2* partial,
                         unsigned* counters, int nvec, double breakdown, cudaStream_t st);
cudaError_t launch_scale32(Buf<float2> dst, Buf<const float2> src, long long n, const GmresDev& gs,
                           int nvec, cudaStream_t st);
cudaError_t launch_fci_step32(Buf<const float2> Aw, Buf<const float2> r, Buf<float2> v0,
                              const GmresDev& gs, double2* partial, unsigned* counters,
                              long long n, int nvec, cudaStream_t st);
cudaError_t launch_combine_fci32(Buf<double2> out, const float2* B, long long bis, long long brs,
                                 const GmresDev& gs, Buf<const double2> E, long long n, int nvec,
                                 cudaStream_t st);

void count_launch();

// Message returned by hz_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// ---- host set-up (hz_setup.cpp) ----
struct Setup {
  double c_min, s, b1, b2, rho2;
  std::vector<double> m;  // c_min^2 / c^2
};

// Coefficients and spectrum rectangle of a problem (Lemma 3.1 with exact Weyl bounds).
void setup_operator(const hz_grid& g, const double* c, Setup& out);

// Nodes and weights of eq:quad-points, then per node (z0, delta, q, nu, sweeps) by the delta
// search of eq:fix-pt-conv.  Returns false if some node has no converging order <= qmax.
bool setup_nodes(const Setup& su, const hz_contour_opts& co, std::vector<NodeParams>& nodes,
                 std::string& err);

}  // namespace hz
