// C ABI of libhz and the host orchestration of the solver:
//   * the batched polynomial solve of all contour nodes (§4.2 eq:fix-pt-exp), right-aligned so
//     that every node ends on the same stencil sweep, where the quadrature sum
//     w = sum_j sigma_j/z_j y_j of Algorithm 1 is formed without storing the y_j;
//   * FCI (§2 Algorithm 1): w, the step d, a few float64 GMRES steps on A v = r - d A w;
//   * flexible GMRES(m) with FCI as the variable right preconditioner (§2, after Algorithm 1),
//     float64 CGS2 Arnoldi and Givens on the device, restarts on the float64 true residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hz.h"
#include "hz_internal.h"
#include "hz_net_internal.h"

using hz::Buf;
using hz::GmresDev;
using hz::NodeParams;

namespace {

thread_local std::string t_err;

hz_status fail(hz_status s, const std::string& msg) {
  t_err = msg;
  return s;
}

hz_status cuda_fail(cudaError_t e, const char* where) {
  t_err = std::string(where) + ": " + cudaGetErrorString(e);
  return HZ_ERR_CUDA;
}

#define HZ_CUDA(call)                                    \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

#define HZ_TRY(call)                  \
  do {                                \
    hz_status s_ = (call);            \
    if (s_ != HZ_OK) return s_;       \
  } while (0)

constexpr double kBreakdown = 1e-14;
constexpr int kProfPool = 1024;  // event pairs per kernel class before a flush

// CUDA-event timing of one kernel class (see hz_profile_enable).
struct ProfClass {
  std::vector<cudaEvent_t> ev;  // 2 * kProfPool
  int used = 0;
  long long launches = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
};

}  // namespace

struct hz_problem {
  int device = 0;
  hz_grid grid{};
  hz_contour_opts copt{};
  hz_limits lim{};
  hz::Geom g{};
  hz::Setup su;
  std::vector<NodeParams> nodes;
  int J = 0;

  // device memory
  double* m64 = nullptr;
  double2* d64 = nullptr;    // [n] float64 diagonal 6 s/h^2 - m - i a
  float2* d32 = nullptr;     // [n] the same diagonal rounded to complex64
  void* poly = nullptr;      // [nrhs][4 J][n] fields (double2 or float2)
  float2* f32 = nullptr;     // [nrhs][n]
  double2* w = nullptr;      // [nrhs][n] quadrature sum
  double2* Aw = nullptr;     // [nrhs][n]
  double2* Vin = nullptr;    // [nrhs][kin+1][n] inner basis
  float2* Vin32 = nullptr;   // [nrhs][kin+1][n] inner basis of the complex64 FCI form
  float2* w32 = nullptr;     // [nrhs][n] quadrature sum rounded to complex64
  float2* Aw32 = nullptr;    // [nrhs][n]
  double2* V = nullptr;      // [nrhs][m+1][n] outer basis
  double2* Z = nullptr;      // [nrhs][m][n] preconditioned directions (float64)
  float2* Z32 = nullptr;     // [nrhs][m][n] the same stored in complex64 (HZ_LIMIT_Z_C64)
  bool case2 = false;        // HZ_LIMIT_CASE_TWO: the solver runs on iC - I (eq:mat-2x2)
  bool spectral = false;     // HZ_DISC_SPECTRAL: Fourier spectral Laplacian, periodic box
  hz::SpecPlan spec{};       // its line-FFT tables
  void* spec_tmp = nullptr;  // [J nrhs][n] double2: the FFT scratch and a stage's s S x batch
  bool invlap_on = false;    // hz_problem_set_inner_invlap: 1/max(lambda, 1) right-preconditions
                             // the inner GMRES (spectral problems)
  bool ilu_on = false;       // hz_problem_set_inner_ilu: ILU(0) right-preconditions inner GMRES
  double* invd = nullptr;    // [n] 1 / ILU(0) pivots
  float* invd32 = nullptr;   // [n] the same in float32 (the sweeps of HZ_MIXED_C64)
  float2* ilu_u32 = nullptr; // [nrhs][n] complex64 scratch of those sweeps
  double2* ilu_t = nullptr;  // [nrhs][n] scratch field of the preconditioned inner GMRES
  int* ilu_prog = nullptr;   // progress words of the multi-block wavefront sweeps
  bool ilu_chain64 = false, ilu_chain32 = false;  // those sweeps fit (all blocks resident)
  long long nf = 0;          // points of a solver field: n, or 2n for Case Two
  bool z32 = false;          // HZ_LIMIT_Z_C64
  bool sweeps32 = false;     // HZ_LIMIT_SWEEPS_C64
  double2* partial = nullptr;
  unsigned* counters = nullptr;
  void* gmem = nullptr;      // all GmresDev arrays
  GmresDev gin{}, gout{};

  // pinned host mirrors
  double* h_scal = nullptr;  // [nrhs][SC_COUNT]   device -> host
  int* h_stopped = nullptr;  // [nrhs]             both directions, always after a sync
  double* h_tol = nullptr;   // [nrhs]             host -> device

  std::vector<void*> allocs;

  bool prof_on = false;
  ProfClass prof[3];

  // CUDA graphs of the outer FGMRES steps, one per step index k, valid for graph_key
  // (right-hand sides, precision, inner steps); the solve runs on the library's own stream
  // because the legacy default stream cannot be captured.
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaGraphExec_t> step_graphs;
  std::vector<unsigned long long> step_kernels;  // kernels captured in each step graph
  long long graph_key = -1;
  bool graphs_on = true;

  // the complex64 FCI tail as one cooperative kernel (hz_fci_tail32.cu): grid plans for
  // k_in <= 4 and k_in <= TAIL_KMAX (ppt 0: does not fit), its barrier words and error flag
  int tail_mode = 1;         // hz_problem_fused_tail: 0 per piece, 1 cooperative, 2 summed norm
  bool tail_solo = true;     // false while several problems run concurrently (batched solve)
  bool tail_used = false;
  int tail_ppt[2] = {0, 0}, tail_blocks[2] = {0, 0};
  unsigned* tail_bar = nullptr;  // [0] arrivals, [1] generation, [2] error flag, [3] poll limit
  unsigned* h_bar = nullptr;     // pinned copy of the error flag, read after each outer step
  // the outer float-pair Arnoldi step as one cooperative kernel (hz_arnoldi_ff.cu), sharing
  // the barrier words and the error flag of the FCI tail (the two never run concurrently)
  int arn_mode = 1;  // hz_problem_fused_arnoldi: 0 five kernels, 1 cooperative, 2 summed norm
  int arn_ppt = 0, arn_blocks = 0;
  // the float64 cooperative FCI tail and outer step (hz_coop64.cu), same modes and barrier
  int t64_ppt = 0, t64_blocks = 0;
  int a64_ppt = 0, a64_blocks = 0;

  // the learned right preconditioner (hz_problem_set_preconditioner): the network, how it
  // combines with FCI, and two float64 fields per right-hand side for the combinations
  hz_net* net = nullptr;
  int net_mode = 0;
  double2* pre_t = nullptr;
  double2* pre_z = nullptr;

  void drop_graphs() {
    for (cudaGraphExec_t g : step_graphs)
      if (g) cudaGraphExecDestroy(g);
    step_graphs.clear();
    step_kernels.clear();
    graph_key = -1;
  }

  ~hz_problem() {
    drop_graphs();
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (own) cudaStreamDestroy(own);
    for (auto& c : prof)
      for (cudaEvent_t e : c.ev) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    if (h_scal) cudaFreeHost(h_scal);
    if (h_stopped) cudaFreeHost(h_stopped);
    if (h_tol) cudaFreeHost(h_tol);
    if (h_bar) cudaFreeHost(h_bar);
  }
};

namespace {

hz_status dalloc(hz_problem* p, void** out, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HZ_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                cudaGetErrorString(e));
  }
  p->allocs.push_back(*out);
  return HZ_OK;
}

char* carve(char*& cur, size_t bytes) {
  char* r = cur;
  cur += (bytes + 255) / 256 * 256;
  return r;
}

// Device arrays of a GmresDev for nrhs right-hand sides and M columns, carved from `cur`.
void gmres_layout(GmresDev& gs, char*& cur, int nrhs, int M) {
  const int Mc = std::max(M, 1);
  gs.mmax = M;
  gs.R = (double2*)carve(cur, sizeof(double2) * nrhs * (size_t)(M + 1) * Mc);
  gs.cc = (double*)carve(cur, sizeof(double) * nrhs * Mc);
  gs.ss = (double2*)carve(cur, sizeof(double2) * nrhs * Mc);
  gs.g = (double2*)carve(cur, sizeof(double2) * nrhs * (M + 1));
  gs.y = (double2*)carve(cur, sizeof(double2) * nrhs * Mc);
  gs.h1 = (double2*)carve(cur, sizeof(double2) * nrhs * (M + 2));
  gs.h2 = (double2*)carve(cur, sizeof(double2) * nrhs * (M + 2));
  gs.nrm = (double2*)carve(cur, sizeof(double2) * 2 * nrhs);
  gs.scal = (double*)carve(cur, sizeof(double) * nrhs * hz::SC_COUNT);
  gs.kend = (int*)carve(cur, sizeof(int) * nrhs);
  gs.stopped = (int*)carve(cur, sizeof(int) * nrhs);
}

size_t gmres_carved_bytes(int nrhs, int M) {
  const int Mc = std::max(M, 1);
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  return r(sizeof(double2) * nrhs * (size_t)(M + 1) * Mc) + r(sizeof(double) * nrhs * Mc) +
         r(sizeof(double2) * nrhs * Mc) + r(sizeof(double2) * nrhs * (M + 1)) +
         r(sizeof(double2) * nrhs * Mc) + 2 * r(sizeof(double2) * nrhs * (M + 2)) +
         r(sizeof(double2) * 2 * nrhs) + r(sizeof(double) * nrhs * hz::SC_COUNT) +
         2 * r(sizeof(int) * nrhs);
}

bool valid_grid(const hz_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->h > 0 && std::isfinite(g->h) &&
         g->omega > 0 && std::isfinite(g->omega) && g->layer_cells >= 0 && g->sigma_max >= 0 &&
         std::isfinite(g->sigma_max) && g->ny <= 65535 && g->nz <= 65535 &&
         (g->discretization == HZ_DISC_FD7 || g->discretization == HZ_DISC_SPECTRAL);
}

// ------------------------------------------------------------------ kernel timing

hz_status prof_flush(ProfClass& c) {
  for (int i = 0; i < c.used; ++i) {
    HZ_CUDA(cudaEventSynchronize(c.ev[2 * i + 1]));
    float ms = 0.f;
    HZ_CUDA(cudaEventElapsedTime(&ms, c.ev[2 * i], c.ev[2 * i + 1]));
    c.ms += ms;
  }
  c.used = 0;
  return HZ_OK;
}

// Brackets one launch of class `cls` with events when timing is on.
struct ProfScope {
  hz_problem* p;
  int cls, slot = -1;
  cudaStream_t st;
  double bytes;
  double flops = 0.0;
  hz_status begin() {
    if (!p->prof_on) return HZ_OK;
    ProfClass& c = p->prof[cls];
    if (c.used == kProfPool) HZ_TRY(prof_flush(c));
    slot = c.used++;
    HZ_CUDA(cudaEventRecord(c.ev[2 * slot], st));
    return HZ_OK;
  }
  hz_status end() {
    if (slot < 0) return HZ_OK;
    ProfClass& c = p->prof[cls];
    HZ_CUDA(cudaEventRecord(c.ev[2 * slot + 1], st));
    c.launches++;
    c.bytes += bytes;
    c.flops += flops;
    return HZ_OK;
  }
};

#define HZ_TIMED(P, CLS, ST, BYTES, CALL)        \
  do {                                           \
    ProfScope ps_{(P), (CLS), -1, (ST), (BYTES)}; \
    HZ_TRY(ps_.begin());                         \
    HZ_CUDA(CALL);                               \
    HZ_TRY(ps_.end());                           \
  } while (0)

// The same for a float64 kernel, also adding its algorithmic float64 flops (an FMA counts 2).
#define HZ_TIMED_F(P, CLS, ST, BYTES, FLOPS, CALL)            \
  do {                                                        \
    ProfScope ps_{(P), (CLS), -1, (ST), (BYTES), (FLOPS)};    \
    HZ_TRY(ps_.begin());                                      \
    HZ_CUDA(CALL);                                            \
    HZ_TRY(ps_.end());                                        \
  } while (0)

// Algorithmic bytes of one stencil launch: x read and y written once per field, m once.
template <typename T, typename R>
double stencil_bytes(long long n, int nvec) {
  return double(n) * (2.0 * sizeof(T) * nvec + sizeof(R));
}

// Algorithmic bytes of one Gram-Schmidt launch over nb basis fields (V read once, w read,
// and written back in the update modes).
double cgs_bytes(int mode, long long n, int nb, int nvec) {
  const double fld = 16.0 * double(n) * nvec;
  return mode == 0 ? fld * (nb + 1) : fld * (nb + 2);
}

// Float64 flops of one Gram-Schmidt launch per point and field: a complex dot or update term
// is 4 FMA (8 flops), a squared norm 2 FMA.  Mode 0: nb dots + the norm; mode 1: nb updates
// and nb dots; mode 2: nb updates + the norm.
double cgs_flops(int mode, long long n, int nb, int nvec) {
  const double pts = double(n) * nvec;
  return mode == 1 ? pts * 16.0 * nb : pts * (8.0 * nb + 4.0);
}

// Float64 flops of the float64 stencil per point: 10 neighbour additions, the shifted diagonal
// (2), and two complex multiply-adds with the Laplacian weight (10).
constexpr double kStencil64Flops = 22.0;

// ------------------------------------------------------------------ polynomial solves

// Buffer slots of node slot `s` in one rhs workspace of 4*nn fields.
struct Slots {
  long long Y, ACC, KA, KB;
};

Slots slots_of(int s, long long n) {
  const long long b = 4LL * s * n;
  return {b, b + n, b + 2 * n, b + 3 * n};
}

// The stage schedule of the batched scheme eq:fix-pt-exp for the nodes in `which` from y = 0:
// schedules are right-aligned, so every node's last sweep ends on the last stage; stage t
// lists its active nodes (compacted) with their step kind, coefficients and workspace slots.
// With `quad` the last stage is marked to form the quadrature sum instead of writing y.
// ycur returns each node slot's final y offset.
template <typename R>
void build_schedule(const hz_problem* p, const std::vector<int>& which, bool quad,
                    std::vector<hz::StageArgs<R>>& out, std::vector<long long>& ycur) {
  const long long n = p->nf;
  const int nn = (int)which.size();
  int T_total = 0;
  for (int node : which) T_total = std::max(T_total, p->nodes[node].q * p->nodes[node].sweeps);
  ycur.assign(nn, 0);
  for (int s = 0; s < nn; ++s) ycur[s] = slots_of(s, n).Y;
  out.assign(T_total, hz::StageArgs<R>{});
  for (int t = 0; t < T_total; ++t) {
    hz::StageArgs<R>& a = out[t];
    std::memset(&a, 0, sizeof(a));
    a.nnodes = 0;
    a.final_quad = (quad && t == T_total - 1) ? 1 : 0;
    for (int s = 0; s < nn; ++s) {
      const NodeParams& np = p->nodes[which[s]];
      const int Tj = np.q * np.sweeps;
      const int start = T_total - Tj;
      if (t < start) continue;
      hz::StageNode<R>& sn = a.nd[a.nnodes++];
      const int tl = t - start;
      const int sweep = tl / np.q;
      const int jj = tl % np.q + 1;
      const Slots sl = slots_of(s, n);
      // c_{j} = (-i delta (z - z0))^j / j!,  ptilde(z) = sum_{j<=q} c_j
      const std::complex<double> zz(np.zr, np.zi), z0(np.z0r, np.z0i);
      const std::complex<double> u = std::complex<double>(0.0, -np.delta) * (zz - z0);
      std::vector<std::complex<double>> c(np.q + 1);
      c[0] = 1.0;
      for (int k = 1; k <= np.q; ++k) c[k] = c[k - 1] * u / double(k);
      std::complex<double> pz = 0.0;
      for (int k = 0; k <= np.q; ++k) pz += c[k];
      const std::complex<double> ip = 1.0 / pz;
      const std::complex<double> md = std::complex<double>(0.0, -np.delta) / double(jj);
      const std::complex<double> wq = std::complex<double>(np.sr, np.si) / zz;
      sn.mdr = R(md.real());
      sn.mdi = R(md.imag());
      sn.cfr = R(c[jj - 1].real());
      sn.cfi = R(c[jj - 1].imag());
      sn.z0r = R(np.z0r);
      sn.z0i = R(np.z0i);
      sn.ipr = R(ip.real());
      sn.ipi = R(ip.imag());
      sn.wqr = wq.real();
      sn.wqi = wq.imag();
      sn.wrh = float(wq.real());
      sn.wrl = float(wq.real() - double(sn.wrh));
      sn.wih = float(wq.imag());
      sn.wil = float(wq.imag() - double(sn.wih));
      sn.acc = sl.ACC;
      auto kbuf = [&](int step) { return (step % 2 == 1) ? sl.KA : sl.KB; };
      if (jj == 1) {
        sn.yzero = sweep == 0 ? 1 : 0;
        sn.in = ycur[s];
        if (np.q == 1) {
          sn.kind = hz::SK_FIRST_LAST;
          sn.yout = (ycur[s] == sl.Y) ? sl.ACC : sl.Y;
          ycur[s] = sn.yout;
        } else {
          sn.kind = hz::SK_FIRST;
          sn.kout = kbuf(1);
        }
      } else if (jj < np.q) {
        sn.kind = hz::SK_MID;
        sn.in = kbuf(jj - 1);
        sn.kout = kbuf(jj);
      } else {
        sn.kind = hz::SK_LAST;
        sn.in = kbuf(jj - 1);
        sn.yout = sl.Y;
        ycur[s] = sl.Y;
      }
    }
  }
}

// Algorithmic bytes per point of one stage: f and the diagonal once; per node FIRST y?(r) k(w)
// acc(w), MID k(r) acc(r/w) k(w), LAST k(r) acc(r) y(w, or the float64 sum w once at the
// final stage).
template <typename T, typename R>
double stage_bytes_per_point(const hz::StageArgs<R>& a, int nvec, bool w32) {
  double bpp = double(sizeof(T)) * 1 + double(sizeof(R)) / nvec;
  for (int s = 0; s < a.nnodes; ++s) {
    const hz::StageNode<R>& sn = a.nd[s];
    const double e = sizeof(T);
    if (sn.kind == hz::SK_FIRST) bpp += (sn.yzero ? 2 : 3) * e;
    else if (sn.kind == hz::SK_MID) bpp += 4 * e;
    else if (sn.kind == hz::SK_LAST) bpp += (a.final_quad ? 2 : 3) * e;
    else if (sn.kind == hz::SK_FIRST_LAST) bpp += ((sn.yzero ? 0 : 1) + (a.final_quad ? 0 : 1)) * e;
  }
  if (a.final_quad) bpp += sizeof(double2) + (w32 ? sizeof(float2) : 0);
  return bpp;
}

// Runs the batched scheme eq:fix-pt-exp for the nodes in `which` from y = 0, one launch per
// stage.  With `quad` the last stage writes w = sum sigma_j/z_j y_j (double2, wbuf; and its
// complex64 rounding into w32buf where that is given); otherwise node slot s ends with its y
// in the returned offset yfinal[s] of the workspace.
template <typename T, typename R>
hz_status run_poly(hz_problem* p, const T* dg, Buf<const T> f, int nvec,
                   const std::vector<int>& which, bool quad, Buf<double2> wbuf,
                   std::vector<long long>* yfinal, cudaStream_t st,
                   Buf<float2> w32buf = Buf<float2>{nullptr, 0}, bool quad64 = false) {
  const long long n = p->nf;
  T* ws = (T*)p->poly;
  const long long wrs = 4LL * p->J * n;  // elements of T per rhs
  std::vector<hz::StageArgs<R>> sched;
  std::vector<long long> ycur;
  if constexpr (sizeof(T) == sizeof(double2)) {
    if (p->case2) {
      // Case Two: the scheme on iC - I, every node's y stored, then the quadrature sum
      build_schedule<R>(p, which, false, sched, ycur);
      ProfScope seq{p, 0, -1, st, 0.0};
      HZ_TRY(seq.begin());
      for (const auto& a : sched)
        HZ_CUDA(hz::launch_poly_stage_2x2(p->g, p->d64, Buf<const double2>{f.p, f.rs},
                                          (double2*)ws, wrs, nvec, a, st));
      if (quad) {
        std::vector<double> wr(which.size()), wi(which.size());
        for (size_t s = 0; s < which.size(); ++s) {
          const NodeParams& np = p->nodes[which[s]];
          const std::complex<double> wq = std::complex<double>(np.sr, np.si) /
                                          std::complex<double>(np.zr, np.zi);
          wr[s] = wq.real();
          wi[s] = wq.imag();
        }
        HZ_CUDA(hz::launch_quad_2x2((const double2*)ws, wrs, wbuf, n, nvec, ycur.data(),
                                    wr.data(), wi.data(), (int)which.size(), st));
      }
      seq.bytes = 0.0;
      HZ_TRY(seq.end());
      if (seq.slot >= 0) p->prof[0].launches += (long long)sched.size() - 1;
      if (yfinal) *yfinal = ycur;
      return HZ_OK;
    }
  }
  build_schedule<R>(p, which, quad, sched, ycur);
  const int T_total = (int)sched.size();
  if (quad && T_total > 0) sched.back().quad64 = quad64 ? 1 : 0;
  if (p->spectral) {
    // each stage: s S x of every node input it reads (line FFTs), then the pointwise stage
    ProfScope seq{p, 0, -1, st, 0.0};
    HZ_TRY(seq.begin());
    double seq_bytes = 0.0;
    int launches = 0;
    for (int t = 0; t < T_total; ++t) {
      hz::StageArgs<R>& a = sched[t];
      hz::VecMap in = hz::vec_map(ws, wrs);
      in.nq = 0;
      for (int q = 0; q < a.nnodes; ++q) {
        hz::StageNode<R>& nd = a.nd[q];
        const bool first = nd.kind == hz::SK_FIRST || nd.kind == hz::SK_FIRST_LAST;
        nd.lapi = -1;
        if (first && nd.yzero) continue;
        nd.lapi = in.nq;
        in.off[in.nq++] = nd.in;
      }
      T* lap = (T*)p->spec_tmp;
      if (in.nq > 0) {
        HZ_CUDA(hz::launch_spectral<T>(p->spec, p->g, hz::SPEC_LAP, in, hz::vec_map(lap, n),
                                       in.nq * nvec, dg, 0.0, 0.0, lap, st));
        launches += 5;
        seq_bytes += 10.0 * sizeof(T) * double(n) * in.nq * nvec;
      }
      HZ_CUDA((hz::launch_poly_stage_spec<T, R>(p->g, dg, f, ws, wrs, lap, in.nq, wbuf, w32buf,
                                                nvec, a, st)));
      ++launches;
      seq_bytes += (stage_bytes_per_point<T, R>(a, nvec, w32buf.p != nullptr) +
                    double(sizeof(T)) * in.nq) * double(n) * nvec;
    }
    seq.bytes = seq_bytes;
    HZ_TRY(seq.end());
    if (seq.slot >= 0) p->prof[0].launches += launches - 1;
    if (yfinal) *yfinal = ycur;
    return HZ_OK;
  }
  // one event pair around the whole stage sequence (per-launch events would cost more than
  // a 64^3 stage); launches and bytes are added per stage
  ProfScope seq{p, 0, -1, st, 0.0};
  HZ_TRY(seq.begin());
  double seq_bytes = 0.0;
  for (int t = 0; t < T_total; ++t) {
    HZ_CUDA((hz::launch_poly_stage<T, R>(p->g, dg, f, ws, wrs, wbuf, w32buf, nvec, sched[t], st)));
    seq_bytes += stage_bytes_per_point<T, R>(sched[t], nvec, w32buf.p != nullptr) * double(n) * nvec;
  }
  seq.bytes = seq_bytes;
  HZ_TRY(seq.end());
  if (seq.slot >= 0) p->prof[0].launches += T_total - 1;  // end() counted one
  if (yfinal) *yfinal = ycur;
  return HZ_OK;
}

// After a synchronisation: a grid barrier of a cooperative kernel that gave up leaves its
// flag set; report it once and reset the barrier words (not the poll limit) for the next launch.
hz_status check_tail_fault(hz_problem* p) {
  if (!p->tail_used) return HZ_OK;
  unsigned w[3] = {0, 0, 0};
  HZ_CUDA(cudaMemcpy(w, p->tail_bar, sizeof(w), cudaMemcpyDeviceToHost));
  if (w[2] == 0) return HZ_OK;
  HZ_CUDA(cudaMemset(p->tail_bar, 0, sizeof(unsigned) * 3));
  return fail(HZ_ERR_TIMEOUT, "a grid barrier of a cooperative kernel gave up waiting");
}

// FCI (Algorithm 1) on nvec double-complex fields r -> out.

bool tail_fits(const hz_problem* p, int nvec, int kin) {
  const int c = kin <= 4 ? 0 : 1;
  return p->tail_mode != 0 && p->tail_solo && nvec == 1 && kin <= hz::TAIL_KMAX &&
         p->tail_ppt[c] > 0;
}

bool arnoldi_fits(const hz_problem* p, int nvec) {
  return p->arn_mode != 0 && p->tail_solo && nvec == 1 && p->arn_ppt > 0;
}

// The float64 cooperative kernels pay off where the float64 Krylov work is latency-bound, not
// where it is float64-throughput-bound (measured on GB300, HZ_MIXED_C64, one right-hand side:
// 32^3 10.9 ms per solve against 13.7 ms for the multi-kernel form; 64^3 60.6 against 54.0 ms,
// where the multi-kernel Gram-Schmidt kernels, sized so the busiest SM has the least work, keep
// the float64 pipes busier than one resident grid with barriers and serial Givens steps).
constexpr long long kCoop64MaxPoints = 1LL << 17;

bool tail64_fits(const hz_problem* p, int nvec, int kin) {
  return p->tail_mode != 0 && p->tail_solo && nvec == 1 && kin <= hz::TAIL64_KMAX &&
         p->t64_ppt > 0 && p->g.n <= kCoop64MaxPoints && !p->ilu_on;
}

bool arnoldi64_fits(const hz_problem* p, int nvec) {
  return p->arn_mode != 0 && p->tail_solo && nvec == 1 && p->a64_ppt > 0 &&
         p->g.n <= kCoop64MaxPoints;
}

// Algorithmic bytes of the complex64 FCI tail (steps 3-5, one cooperative launch): step d
// reads w, r and the diagonal and writes v_0; inner step j (basis of j fields) reads v_{j-1}
// for A v, the basis twice per CGS2 pass pair (dot, update) with w read and written alongside,
// and writes v_j: 4j + 7 fields; the combine reads the k_in + 1 basis fields and the float64 w
// and writes the float64 result.  Every field counted once per pass, 8 bytes a point.
double fci_tail32_bytes(long long n, int kin) {
  double f = 4.0;
  for (int j = 1; j <= kin; ++j) f += 4.0 * j + 7.0;
  f += kin + 1.0;
  return 8.0 * double(n) * f + 32.0 * double(n);
}

// Algorithmic bytes and float64 flops per point of the float64 FCI tail (step d, kin CGS2
// steps, v + d w) and of one float64 outer Arnoldi step with nb basis fields: every field read
// or written once per pass, 8 flops per complex multiply-add, 22 per stencil point.
double tail64_bytes(long long n, int kin) {
  double f = 3.0 + 2.0;  // step d: w, r, diagonal; W and v_0 written
  for (int nb = 1; nb <= kin; ++nb) f += 2.0 + 3.0 * nb + 2.0;
  return 16.0 * n * (f + kin + 1.0);
}
double tail64_flops(long long n, int kin) {
  double f = 22.0 + 12.0 + 12.0;
  for (int nb = 1; nb <= kin; ++nb) f += 24.0 + 32.0 * nb + 8.0;
  return double(n) * (f + 8.0 * kin + 8.0);
}
double arn64_bytes(long long n, int nb) { return 16.0 * n * (3.0 + 3.0 * nb + 1.0); }
double arn64_flops(long long n, int nb) { return double(n) * (22.0 + 32.0 * nb + 10.0); }

// Algorithmic bytes and float64 flops of apply_op64 on nvec fields: the 7-point stencil, or
// the five line-FFT passes of the spectral operator (every field read and written once per
// pass, the input and diagonal read again by the last; 5 log2(n_a) flops per point and
// transform direction along each axis, 10 for the diagonal and the pointwise part).
double op64_bytes(const hz_problem* p, int nvec) {
  const double n = double(p->nf);
  if (!p->spectral) return stencil_bytes<double2, double2>(p->nf, nvec);
  return 16.0 * n * (11.0 * nvec + 1.0);
}
double op64_flops(const hz_problem* p, int nvec) {
  const double n = double(p->nf);
  if (!p->spectral) return kStencil64Flops * n * nvec;
  double f = 10.0;
  for (int a = 0; a < 3; ++a) f += 10.0 * std::log2(double(p->spec.ax[a].n));
  return f * n * nvec;
}

// y = (B - 0 I) x in float64 for solver fields: B = A (Case One) or iC - I (Case Two).
cudaError_t apply_op64(const hz_problem* p, Buf<const double2> x, Buf<double2> y, int nvec,
                       cudaStream_t st) {
  if (p->case2)
    return hz::launch_apply_2x2_strided(p->g, p->d64, x.p, x.rs, y.p, y.rs, nvec, 0.0, 0.0, st);
  if (p->spectral)
    return hz::launch_spectral<double2>(p->spec, p->g, hz::SPEC_APPLY, hz::vec_map(x.p, x.rs),
                                        hz::vec_map(y.p, y.rs), nvec, p->d64, 0.0, 0.0,
                                        (double2*)p->spec_tmp, st);
  return hz::launch_stencil_diag(p->g, p->d64, x, y, nvec, 0.0, 0.0, st);
}

// r_ff: r holds float pairs (the outer basis of HZ_MIXED_C64_FF) whose complex64 rounding the
// normalisation kernel already wrote into p->f32; otherwise r is complex128.
hz_status run_fci(hz_problem* p, Buf<const double2> r, Buf<double2> out, int nvec, int kin,
                  int precision, cudaStream_t st, bool r_ff = false) {
  const long long n = p->nf;
  const bool fci32 = precision == HZ_MIXED_C64_FCI32 || precision == HZ_MIXED_C64_FF;
  std::vector<int> all(p->J);
  for (int j = 0; j < p->J; ++j) all[j] = j;
  Buf<double2> wb{p->w, n};
  if (precision != HZ_C128) {
    // the complex64 form of the FCI internals also takes w rounded to complex64
    const Buf<float2> w32b{fci32 ? p->w32 : nullptr, n};
    // (float-pair input: the normalisation that made r already wrote its complex64 rounding)
    if (!r_ff) HZ_CUDA(hz::launch_convert_c128_c64(r, Buf<float2>{p->f32, n}, n, nvec, st));
    // HZ_MIXED_C64 keeps the quadrature accumulation in float64; the complex64-FCI forms sum
    // the terms in float pairs
    HZ_TRY((run_poly<float2, float>(p, p->d32, Buf<const float2>{p->f32, n}, nvec, all, true,
                                    wb, nullptr, st, w32b, precision == HZ_MIXED_C64)));
  } else {
    HZ_TRY((run_poly<double2, double>(p, p->d64, r, nvec, all, true, wb, nullptr, st)));
  }
  if (!fci32 && tail64_fits(p, nvec, kin)) {
    // steps 3-5 in float64 as one cooperative launch (Aw serves as its scratch field)
    HZ_TIMED_F(p, 2, st, tail64_bytes(n, kin), tail64_flops(n, kin),
               hz::launch_fci_tail64(p->g, p->d64, p->w, r.p, p->Vin, p->Aw, out.p, p->partial,
                                     p->tail_bar, (int*)(p->tail_bar + 2), n, kin, kBreakdown,
                                     p->tail_mode == 1 ? 1 : 0, p->t64_ppt, p->t64_blocks, st));
    p->tail_used = true;
    return HZ_OK;
  }
  if (fci32 && tail_fits(p, nvec, kin)) {
    // steps 3-5 in one cooperative launch
    const int c = kin <= 4 ? 0 : 1;
    HZ_TIMED(p, 2, st, fci_tail32_bytes(n, kin),
             hz::launch_fci_tail32(p->g, p->d32, p->w32, p->f32, p->w, p->Vin32, p->Aw32, out.p,
                                   p->partial, p->tail_bar, (int*)(p->tail_bar + 2), n, kin,
                                   kBreakdown, p->tail_mode == 1 ? 1 : 0, p->tail_ppt[c],
                                   p->tail_blocks[c], st));
    p->tail_used = true;
    return HZ_OK;
  }
  if (fci32) {
    // step d and the inner GMRES on complex64 fields; w itself stays float64 for v + d w
    const long long vrs = (long long)(p->lim.inner_k_max + 1) * n;
    // Aw and d = (Aw)^H r / ||Aw||^2 in one launch, then v0 = r - d Aw and beta
    HZ_TIMED(p, 1, st, (stencil_bytes<float2, float2>(n, nvec)) + 8.0 * n * nvec,
             (hz::launch_stencil32_dots(1, p->g, p->d32, Buf<const float2>{p->w32, n},
                                        Buf<float2>{p->Aw32, n}, p->f32, n, n, 1, p->gin,
                                        p->partial, p->counters, nvec, st)));
    HZ_TIMED(p, 2, st, 8.0 * n * nvec * 3,
             hz::launch_fci_start32(Buf<const float2>{p->Aw32, n}, Buf<const float2>{p->f32, n},
                                    Buf<float2>{p->Vin32, vrs}, p->gin, p->partial, p->counters,
                                    n, nvec, st));
    HZ_CUDA(hz::launch_scale32(Buf<float2>{p->Vin32, vrs}, Buf<const float2>{p->Vin32, vrs}, n,
                               p->gin, nvec, st));
    for (int j = 0; j < kin; ++j) {
      Buf<float2> wj{p->Vin32 + (long long)(j + 1) * n, vrs};
      // w = A v_j and the first CGS pass in one launch, then the second pass and Givens
      HZ_TIMED(p, 1, st,
               (stencil_bytes<float2, float2>(n, nvec)) + 0.5 * cgs_bytes(0, n, j + 1, nvec),
               (hz::launch_stencil32_dots(
                   0, p->g, p->d32, Buf<const float2>{p->Vin32 + (long long)j * n, vrs}, wj,
                   p->Vin32, n, vrs, j + 1, p->gin, p->partial, p->counters, nvec, st)));
      for (int mode = 1; mode < 3; ++mode)
        HZ_TIMED(p, 2, st, 0.5 * cgs_bytes(mode, n, j + 1, nvec),
                 hz::launch_cgs32(mode, p->Vin32, n, vrs, j + 1, wj, n, p->gin, p->partial,
                                  p->counters, nvec, kBreakdown, st));
      HZ_CUDA(hz::launch_scale32(wj, Buf<const float2>{wj.p, vrs}, n, p->gin, nvec, st));
    }
    HZ_CUDA(hz::launch_backsolve32(p->gin, nvec, st));
    HZ_CUDA(hz::launch_combine_fci32(out, p->Vin32, n, vrs, p->gin, Buf<const double2>{p->w, n},
                                     n, nvec, st));
    return HZ_OK;
  }
  // Aw, step d, inner start v0 = (r - d Aw)/||r - d Aw||
  HZ_TIMED_F(p, 1, st, op64_bytes(p, nvec), op64_flops(p, nvec),
             apply_op64(p, Buf<const double2>{p->w, n}, Buf<double2>{p->Aw, n}, nvec, st));
  const long long vrs = (long long)(p->lim.inner_k_max + 1) * n;
  // two launches: d (reads Aw, r) and v0 = r - d Aw with its norm (reads Aw, r; writes v0)
  HZ_TIMED_F(p, 2, st, 16.0 * n * nvec * 5, 24.0 * n * nvec,
             hz::launch_fci_step(Buf<const double2>{p->Aw, n}, r, Buf<double2>{p->Vin, vrs},
                                 p->gin, p->partial, p->counters, n, nvec, st));
  HZ_CUDA(hz::launch_scale(Buf<double2>{p->Vin, vrs}, Buf<const double2>{p->Vin, vrs}, n, p->gin,
                           nvec, st));
  // with ILU(0) (Section 6.3) the inner GMRES runs right-preconditioned on A M^{-1}; its sweeps
  // in float32 arithmetic in the complex64-sweep form, float64 in the all-float64 form
  const bool ilu = p->ilu_on || p->invlap_on;
  const bool ilu32 = p->ilu_on && precision == HZ_MIXED_C64 && hz::ilu0_fits32(p->g);
  auto ilu_apply = [&](Buf<const double2> t, Buf<double2> z) -> cudaError_t {
    if (p->ilu_on && (ilu32 ? p->ilu_chain32 : p->ilu_chain64) && nvec <= p->lim.nrhs_max) {
      p->tail_used = true;  // its bounded waits report through the barrier words
      if (ilu32)
        return hz::launch_ilu0_chain32(p->g, p->invd32, t, Buf<float2>{p->ilu_u32, p->g.n}, z,
                                       nvec, p->ilu_prog, p->tail_bar, st);
      return hz::launch_ilu0_chain(p->g, p->invd, t, z, nvec, p->ilu_prog, p->tail_bar, st);
    }
    if (p->invlap_on)
      return hz::launch_spectral<double2>(p->spec, p->g, hz::SPEC_INVLAP, hz::vec_map(t.p, t.rs),
                                          hz::vec_map(z.p, z.rs), nvec, p->d64, 0.0, 0.0,
                                          (double2*)p->spec_tmp, st);
    if (ilu32)
      return hz::launch_ilu0_32(p->g, p->invd32, t, Buf<float2>{p->ilu_u32, p->g.n}, z, nvec,
                                st);
    return hz::launch_ilu0(p->g, p->invd, t, z, nvec, st);
  };
  for (int j = 0; j < kin; ++j) {
    Buf<double2> wj{p->Vin + (long long)(j + 1) * n, vrs};
    Buf<const double2> src{p->Vin + (long long)j * n, vrs};
    if (ilu) {
      HZ_CUDA(ilu_apply(src, Buf<double2>{p->ilu_t, n}));
      src = Buf<const double2>{p->ilu_t, n};
    }
    HZ_TIMED_F(p, 1, st, op64_bytes(p, nvec), op64_flops(p, nvec),
               apply_op64(p, src, wj, nvec, st));
    for (int mode = 0; mode < 3; ++mode)
      HZ_TIMED_F(p, 2, st, cgs_bytes(mode, n, j + 1, nvec), cgs_flops(mode, n, j + 1, nvec),
                 hz::launch_cgs(mode, p->Vin, n, vrs, j + 1, wj, n, p->gin, p->partial,
                                p->counters, nvec, kBreakdown, st));
    HZ_CUDA(hz::launch_scale(wj, Buf<const double2>{wj.p, vrs}, n, p->gin, nvec, st));
  }
  HZ_CUDA(hz::launch_backsolve(p->gin, nvec, st));
  if (ilu) {
    // out = M^{-1} (V y) + d w
    HZ_CUDA(hz::launch_combine(Buf<double2>{p->ilu_t, n}, p->Vin, n, vrs, p->gin,
                               Buf<const double2>{nullptr, 0}, -1, 0, n, nvec, kin, st));
    HZ_CUDA(ilu_apply(Buf<const double2>{p->ilu_t, n}, out));
    HZ_CUDA(hz::launch_add_dw(out, Buf<const double2>{p->w, n}, n, p->gin, nvec, st));
    return HZ_OK;
  }
  HZ_CUDA(hz::launch_combine(out, p->Vin, n, vrs, p->gin, Buf<const double2>{p->w, n}, 0, 0, n,
                             nvec, kin, st));
  return HZ_OK;
}

// The right preconditioner z = M(v) of one outer step (v field r at v.p + r v.rs, z likewise).
// net_mode 0: FCI (Algorithm 1); 1: the network alone; 2: z = N(v) + FCI(v - A N(v)); 3: z =
// FCI(v) + N(v - A FCI(v)).  The corrections use the float64 stencil for the residual.
hz_status run_precond(hz_problem* p, Buf<const double2> v, Buf<double2> z, int nrhs, int K,
                      int precision, cudaStream_t st, bool r_ff) {
  if (p->net_mode == 0 || !p->net) return run_fci(p, v, z, nrhs, K, precision, st, r_ff);
  const long long n = p->g.n;
  const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
  auto net = [&](Buf<const double2> in, Buf<double2> out, int acc) {
    return hz::net_apply_field(p->net, in.p, in.rs, p->m64, out.p, out.rs, nrhs, nx, ny, nz, acc,
                               st);
  };
  // t = v - A z (A z into pre_z as scratch)
  auto residual = [&]() -> hz_status {
    HZ_TIMED_F(p, 1, st, (stencil_bytes<double2, double2>(n, nrhs)), kStencil64Flops * n * nrhs,
               (hz::launch_stencil_diag(p->g, p->d64, Buf<const double2>{z.p, z.rs},
                                        Buf<double2>{p->pre_z, n}, nrhs, 0.0, 0.0, st)));
    HZ_CUDA(hz::launch_field_sub(v.p, v.rs, p->pre_z, n, p->pre_t, n, n, nrhs, st));
    return HZ_OK;
  };
  if (p->net_mode == 1) return net(v, z, 0);
  if (p->net_mode == 2) {
    // z = d N(v) + FCI(v - d A N(v)), d = (A N v)^H v / ||A N v||^2: the network's correction
    // with the step that minimises the residual it leaves (as step d does for w in Algorithm 1),
    // so a poor network output cannot raise the residual FCI then works on
    HZ_TRY(net(v, z, 0));
    HZ_TIMED_F(p, 1, st, (stencil_bytes<double2, double2>(n, nrhs)), kStencil64Flops * n * nrhs,
               (hz::launch_stencil_diag(p->g, p->d64, Buf<const double2>{z.p, z.rs},
                                        Buf<double2>{p->pre_z, n}, nrhs, 0.0, 0.0, st)));
    HZ_CUDA(hz::launch_fci_step(Buf<const double2>{p->pre_z, n}, v, Buf<double2>{p->pre_t, n},
                                p->gin, p->partial, p->counters, n, nrhs, st));
    HZ_CUDA(hz::launch_scale_by_step(z.p, z.rs, p->gin, n, nrhs, st));
    HZ_TRY(run_fci(p, Buf<const double2>{p->pre_t, n}, Buf<double2>{p->pre_z, n}, nrhs, K,
                   precision, st, false));
    HZ_CUDA(hz::launch_field_add(z.p, z.rs, p->pre_z, n, n, nrhs, st));
    return HZ_OK;
  }
  HZ_TRY(run_fci(p, v, z, nrhs, K, precision, st, r_ff));
  HZ_TRY(residual());
  return net(Buf<const double2>{p->pre_t, n}, z, 1);
}

// One outer FGMRES step k on all right-hand sides: z_k = M(v_k) (FCI, or the network), w = A z_k,
// CGS2 against v_0..v_k with the Givens update of column k, v_{k+1} = w / h_{k+1,k}.
hz_status outer_step_launches(hz_problem* p, int k, int nrhs, int K, int precision,
                              cudaStream_t st) {
  const long long n = p->nf;
  const long long vrs = (long long)(p->lim.restart_max + 1) * n;
  const long long zrs = (long long)p->lim.restart_max * n;
  GmresDev& go = p->gout;
  Buf<const double2> vk{p->V + (long long)k * n, vrs};
  const bool ff = precision == HZ_MIXED_C64_FF;
  if (p->z32) {
    // z_k = FCI(v_k) into a float64 scratch field (Aw is free once FCI has returned), stored
    // rounded to complex64; the matvec then reads the stored value
    HZ_TRY(run_precond(p, vk, Buf<double2>{p->Aw, n}, nrhs, K, precision, st, false));
    Buf<float2> z32k{p->Z32 + (long long)k * n, zrs};
    HZ_CUDA(hz::launch_convert_c128_c64(Buf<const double2>{p->Aw, n}, z32k, n, nrhs, st));
    Buf<double2> wk{p->V + (long long)(k + 1) * n, vrs};
    if (arnoldi64_fits(p, nrhs)) {
      HZ_TIMED_F(p, 2, st, arn64_bytes(n, k + 1) - 8.0 * n, arn64_flops(n, k + 1),
                 hz::launch_arnoldi64(p->g, p->d64, z32k.p, 1, p->V, wk.p, go, p->partial,
                                      p->tail_bar, (int*)(p->tail_bar + 2), n, k + 1, kBreakdown,
                                      p->arn_mode == 1 ? 1 : 0, p->a64_ppt, p->a64_blocks, st));
      p->tail_used = true;
      return HZ_OK;
    }
    HZ_TIMED_F(p, 1, st, double(n) * nrhs * (8.0 + 16.0 + 16.0), kStencil64Flops * n * nrhs,
               (hz::launch_stencil_diag_x32(p->g, p->d64, Buf<const float2>{z32k.p, zrs}, wk,
                                            nrhs, st)));
    for (int mode = 0; mode < 3; ++mode)
      HZ_TIMED_F(p, 2, st, cgs_bytes(mode, n, k + 1, nrhs), cgs_flops(mode, n, k + 1, nrhs),
                 hz::launch_cgs(mode, p->V, n, vrs, k + 1, wk, n, go, p->partial, p->counters,
                                nrhs, kBreakdown, st));
    HZ_CUDA(hz::launch_scale(wk, Buf<const double2>{wk.p, vrs}, n, go, nrhs, st));
    return HZ_OK;
  }
  Buf<double2> zk{p->Z + (long long)k * n, zrs};
  HZ_TRY(run_precond(p, vk, zk, nrhs, K, precision, st, ff));
  if (ff) {
    // the float-pair Arnoldi: w = A z_k stored as float pairs in v_{k+1}'s slot
    Buf<float4> wf{(float4*)(p->V + (long long)(k + 1) * n), vrs};
    if (arnoldi_fits(p, nrhs)) {
      // one cooperative launch: stencil, CGS2 (V read once per pass), Givens, normalisation
      HZ_TIMED(p, 2, st, 16.0 * n * (3.0 + 3.0 * (k + 1)) + 8.0 * n,
               hz::launch_arnoldi_ff(p->g, p->d64, zk.p, (const float4*)p->V, wf.p, p->f32, go,
                                     p->partial, p->tail_bar, (int*)(p->tail_bar + 2), n, k + 1,
                                     kBreakdown, p->arn_mode == 1 ? 1 : 0, p->arn_ppt,
                                     p->arn_blocks, st));
      p->tail_used = true;
      return HZ_OK;
    }
    HZ_TIMED(p, 1, st, 16.0 * 3 * n * nrhs,
             (hz::launch_stencil_diag_ff(p->g, p->d64, Buf<const double2>{zk.p, zrs}, wf, nrhs,
                                         st)));
    for (int mode = 0; mode < 3; ++mode)
      HZ_TIMED(p, 2, st, cgs_bytes(mode, n, k + 1, nrhs),
               hz::launch_cgs_ff(mode, (const float4*)p->V, n, vrs, k + 1, wf, n, go, p->partial,
                                 p->counters, nrhs, kBreakdown, st));
    // v_{k+1}, and its complex64 rounding: the next FCI application's input
    HZ_CUDA(hz::launch_scale_ff(wf, n, go, nrhs, st, Buf<float2>{p->f32, n}));
    return HZ_OK;
  }
  Buf<double2> wk{p->V + (long long)(k + 1) * n, vrs};
  if (arnoldi64_fits(p, nrhs)) {
    HZ_TIMED_F(p, 2, st, arn64_bytes(n, k + 1), arn64_flops(n, k + 1),
               hz::launch_arnoldi64(p->g, p->d64, zk.p, 0, p->V, wk.p, go, p->partial,
                                    p->tail_bar, (int*)(p->tail_bar + 2), n, k + 1, kBreakdown,
                                    p->arn_mode == 1 ? 1 : 0, p->a64_ppt, p->a64_blocks, st));
    p->tail_used = true;
    return HZ_OK;
  }
  HZ_TIMED_F(p, 1, st, op64_bytes(p, nrhs), op64_flops(p, nrhs),
             apply_op64(p, Buf<const double2>{zk.p, zrs}, wk, nrhs, st));
  for (int mode = 0; mode < 3; ++mode)
    HZ_TIMED_F(p, 2, st, cgs_bytes(mode, n, k + 1, nrhs), cgs_flops(mode, n, k + 1, nrhs),
               hz::launch_cgs(mode, p->V, n, vrs, k + 1, wk, n, go, p->partial, p->counters, nrhs,
                              kBreakdown, st));
  HZ_CUDA(hz::launch_scale(wk, Buf<const double2>{wk.p, vrs}, n, go, nrhs, st));
  return HZ_OK;
}

// The same step replayed from a CUDA graph captured on first use (the ~60 launches of a
// step then cost one graph launch); plain launches while kernel timing is on.
hz_status outer_step(hz_problem* p, int k, int nrhs, int K, int precision, cudaStream_t st) {
  if (p->prof_on || !p->graphs_on) return outer_step_launches(p, k, nrhs, K, precision, st);
  const long long key =
      ((((long long)nrhs * 4 + precision) * 1024 + K) * 2 + (tail_fits(p, nrhs, K) ? 1 : 0)) * 2 +
      (arnoldi_fits(p, nrhs) ? 1 : 0) + 2 * (p->arn_mode == 2 ? 1 : 0) +
      4 * (p->tail_mode == 2 ? 1 : 0) + 8 * p->net_mode + 32 * (tail64_fits(p, nrhs, K) ? 1 : 0) +
      64 * (arnoldi64_fits(p, nrhs) ? 1 : 0);
  if (p->graph_key != key) {
    p->drop_graphs();
    p->graph_key = key;
    p->step_graphs.assign(p->lim.restart_max, nullptr);
    p->step_kernels.assign(p->lim.restart_max, 0);
  }
  if (!p->step_graphs[k]) {
    cudaGraph_t g = nullptr;
    HZ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const unsigned long long before = hz::g_launches.load();
    const hz_status s = outer_step_launches(p, k, nrhs, K, precision, st);
    // captured kernels did not run: take them off the launch count, add them per replay
    p->step_kernels[k] = hz::g_launches.load() - before;
    hz::g_launches.fetch_sub(p->step_kernels[k]);
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (s != HZ_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate");
    p->step_graphs[k] = ex;
  }
  HZ_CUDA(cudaGraphLaunch(p->step_graphs[k], st));
  hz::g_launches.fetch_add(p->step_kernels[k]);
  return HZ_OK;
}

// Times the candidate tile shapes of the polynomial stage (per node-count class) and of the
// complex64 stencil on this problem's grid and keeps the fastest (fields zeroed first; every
// candidate computes the same values, only the launch shape differs).
hz_status autotune(hz_problem* p) {
  const cudaStream_t st = p->own;
  const long long n = p->g.n;
  const long long wrs = 4LL * p->J * n;
  HZ_CUDA(cudaMemsetAsync(p->f32, 0, sizeof(float2) * n, st));
  HZ_CUDA(cudaMemsetAsync(p->w32, 0, sizeof(float2) * n, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HZ_CUDA(cudaEventCreate(&e0));
  HZ_CUDA(cudaEventCreate(&e1));
  // best of 3 trials of 8 back-to-back launches (one trial is noisy at a few microseconds)
  auto timed = [&](auto launch) -> float {
    float best = 1e30f;
    if (launch() != cudaSuccess) return best;
    for (int trial = 0; trial < 3; ++trial) {
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 8; ++rep)
        if (launch() != cudaSuccess) return 1e30f;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  const int J = p->J;
  // classes with several active nodes: time the whole stage sequence of one complex64 FCI
  // application (dependent launches, as a solve runs them); a stage timed alone, back to back
  // with copies of itself, ranked the tiles differently from the chained sequence
  std::vector<int> all(J);
  for (int j = 0; j < J; ++j) all[j] = j;
  auto sequence = [&] {
    const hz_status rs = run_poly<float2, float>(p, p->d32, Buf<const float2>{p->f32, n}, 1, all,
                                                 true, Buf<double2>{p->w, n}, nullptr, st,
                                                 Buf<float2>{p->w32, n});
    return rs == HZ_OK ? cudaSuccess : cudaErrorUnknown;
  };
  // (only where a sequence is short: L2-resident grids; larger grids are bandwidth-bound and
  // their stages time reliably alone)
  const bool chained = n <= (1LL << 21);
  for (int cls : {1, 2}) {
    if (!chained || (cls == 1 && J < 2) || (cls == 2 && J < 4)) continue;
    float best = timed(sequence);
    int bz = p->g.pzc[cls], br = p->g.prows[cls];
    const int nn = cls == 1 ? 3 : J;  // the largest block of the class
    for (int zc : {1, 2, 4})
      for (int rows : {1, 2, 4}) {
        if (32 * nn * rows > 512) continue;
        if (sizeof(double2) * 32 * zc * J * rows > 48 * 1024) continue;
        p->g.pzc[cls] = zc;
        p->g.prows[cls] = rows;
        const float t = timed(sequence);
        if (t < 0.98f * best) {
          best = t;
          bz = zc;
          br = rows;
        }
      }
    p->g.pzc[cls] = bz;
    p->g.prows[cls] = br;
  }
  for (int cls = 0; cls < 3; ++cls) {
    if (chained && cls > 0) continue;
    const int nn = cls == 0 ? 1 : (cls == 1 ? 2 : J);
    if (nn > J || (cls == 2 && J < 4)) continue;
    hz::StageArgs<float> a;
    std::memset(&a, 0, sizeof(a));
    a.nnodes = nn;
    for (int s = 0; s < nn; ++s) {
      const Slots sl = slots_of(s, n);
      hz::StageNode<float>& sn = a.nd[s];
      sn.kind = hz::SK_MID;
      sn.mdr = 0.f;
      sn.mdi = -0.1f;
      sn.cfr = 1.f;
      sn.ipr = 1.f;
      sn.in = sl.KA;
      sn.kout = sl.KB;
      sn.acc = sl.ACC;
    }
    float best = 1e30f;
    int bz = p->g.pzc[cls], br = p->g.prows[cls];
    for (int zc : {1, 2, 4})
      for (int rows : {1, 2, 4}) {
        if (32 * nn * rows > 512) continue;
        if (cls == 2 && sizeof(double2) * 32 * zc * J * rows > 48 * 1024) continue;
        p->g.pzc[cls] = zc;
        p->g.prows[cls] = rows;
        const float t = timed([&] {
          return hz::launch_poly_stage<float2, float>(p->g, p->d32,
                                                      Buf<const float2>{p->f32, n},
                                                      (float2*)p->poly, wrs,
                                                      Buf<double2>{p->w, n},
                                                      Buf<float2>{nullptr, 0}, 1, a, st);
        });
        if (t < best) {
          best = t;
          bz = zc;
          br = rows;
        }
      }
    p->g.pzc[cls] = bz;
    p->g.prows[cls] = br;
  }
  float best = 1e30f;
  int bz = p->g.szc, br = p->g.srows;
  for (int zc : {2, 4, 8})
    for (int rows : {2, 4, 8}) {
      p->g.szc = zc;
      p->g.srows = rows;
      const float t = timed([&] {
        return hz::launch_stencil32(p->g, p->d32, Buf<const float2>{p->w32, n},
                                    Buf<float2>{p->Aw32, n}, 1, 0.0, 0.0, st);
      });
      if (t < best) {
        best = t;
        bz = zc;
        br = rows;
      }
    }
  p->g.szc = bz;
  p->g.srows = br;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  return HZ_OK;
}

hz_status check_problem(const hz_problem* p) {
  if (!p) return fail(HZ_ERR_INVALID, "null problem");
  return HZ_OK;
}

hz_status set_device(const hz_problem* p) {
  int cur = -1;
  HZ_CUDA(cudaGetDevice(&cur));
  if (cur != p->device) HZ_CUDA(cudaSetDevice(p->device));
  return HZ_OK;
}

// Early-stop tolerance of the outer cycle per rhs (scal[r][SC_TOL]; < 0: never).  The pinned
// staging buffer is only rewritten after a stream synchronisation, so no copy from it is
// still pending.
hz_status fill_scal_tol(hz_problem* p, GmresDev& gs, const std::vector<double>& tol, int nvec,
                        cudaStream_t st) {
  for (int r = 0; r < nvec; ++r) p->h_tol[r] = tol[r];
  HZ_CUDA(cudaMemcpy2DAsync(gs.scal + hz::SC_TOL, sizeof(double) * hz::SC_COUNT, p->h_tol,
                            sizeof(double), sizeof(double), nvec, cudaMemcpyHostToDevice, st));
  return HZ_OK;
}

}  // namespace

namespace hz {
void set_last_error(const std::string& msg) { t_err = msg; }
}  // namespace hz

namespace {
struct SolveState;
hz_status solve_on(hz_problem* p, const void* f, void* u, int nrhs, const hz_solve_opts* opts,
                   hz_solve_stats* stats, cudaStream_t st);
hz_status solve_batched_on(hz_problem* const* probs, int nprob, const void* const* f,
                           void* const* u, const int* nrhs, const hz_solve_opts* opts,
                           hz_solve_stats* stats);

// Argument checks shared by hz_solve and hz_solve_batched.
hz_status check_solve_args(const hz_problem* p, int nrhs, const hz_solve_opts* opts) {
  if (!p) return fail(HZ_ERR_INVALID, "null problem");
  if (!opts) return fail(HZ_ERR_INVALID, "opts is null");
  if (nrhs < 0 || nrhs > p->lim.nrhs_max) return fail(HZ_ERR_INVALID, "nrhs out of range");
  if (opts->restart_m < 1 || opts->restart_m > p->lim.restart_max)
    return fail(HZ_ERR_INVALID, "restart_m out of range");
  if (opts->inner_k < 0 || opts->inner_k > p->lim.inner_k_max)
    return fail(HZ_ERR_INVALID, "inner_k out of range");
  if (opts->max_cycles < 0 || opts->fixed_its < 0 || !(opts->rtol >= 0))
    return fail(HZ_ERR_INVALID, "invalid max_cycles / fixed_its / rtol");
  if (opts->precision != HZ_C128 && opts->precision != HZ_MIXED_C64 &&
      opts->precision != HZ_MIXED_C64_FCI32 && opts->precision != HZ_MIXED_C64_FF)
    return fail(HZ_ERR_INVALID, "unknown precision");
  if (p->sweeps32 && opts->precision == HZ_C128)
    return fail(HZ_ERR_INVALID, "HZ_C128 needs a problem created without HZ_LIMIT_SWEEPS_C64");
  if (p->z32 && opts->precision != HZ_MIXED_C64 && opts->precision != HZ_MIXED_C64_FCI32)
    return fail(HZ_ERR_INVALID, "a problem created with HZ_LIMIT_Z_C64 solves in HZ_MIXED_C64 or "
                                "HZ_MIXED_C64_FCI32 only");
  if (p->case2 && opts->precision != HZ_C128)
    return fail(HZ_ERR_INVALID, "Case Two problems solve in HZ_C128");
  if (p->spectral && opts->precision != HZ_C128 && opts->precision != HZ_MIXED_C64)
    return fail(HZ_ERR_INVALID, "spectral problems solve in HZ_C128 or HZ_MIXED_C64");
  if (p->ilu_on && opts->precision != HZ_C128 && opts->precision != HZ_MIXED_C64)
    return fail(HZ_ERR_INVALID, "ILU(0) preconditions the float64 inner GMRES (HZ_C128, "
                                "HZ_MIXED_C64)");
  if (p->net_mode != 0 && opts->precision == HZ_MIXED_C64_FF)
    return fail(HZ_ERR_INVALID, "the learned preconditioner needs a float64 outer basis");
  if (p->net_mode != 0 && !hz::net_fits(p->net, nrhs, p->g.nx, p->g.ny, p->g.nz))
    return fail(HZ_ERR_INVALID, "right-hand sides or grid beyond the network's capacity");
  return HZ_OK;
}
}  // namespace

extern "C" {

const char* hz_status_string(hz_status s) {
  switch (s) {
    case HZ_OK: return "ok";
    case HZ_ERR_INVALID: return "invalid argument";
    case HZ_ERR_CUDA: return "CUDA error";
    case HZ_ERR_OOM: return "out of memory";
    case HZ_ERR_NOT_CONVERGED: return "not converged";
    case HZ_ERR_BREAKDOWN: return "breakdown";
    case HZ_ERR_DIVERGED: return "diverged";
    case HZ_ERR_SETUP: return "set-up failed";
    case HZ_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

const char* hz_last_error(void) { return t_err.c_str(); }

unsigned long long hz_launch_count(void) { return hz::g_launches.load(); }

hz_status hz_problem_create(const hz_grid* grid, const double* c_host,
                            const hz_contour_opts* contour, const hz_limits* limits,
                            hz_problem** out) {
  if (!out) return fail(HZ_ERR_INVALID, "out is null");
  *out = nullptr;
  if (!valid_grid(grid)) return fail(HZ_ERR_INVALID, "invalid grid");
  if (!c_host) return fail(HZ_ERR_INVALID, "c_host is null");
  if (!contour || contour->J < 1 || contour->J > hz::MAXJ || !(contour->t > 0) ||
      !(contour->eps > 0) || contour->qmax < 1 || contour->qmax > 12 ||
      !(contour->reduction > 1.0))
    return fail(HZ_ERR_INVALID, "invalid contour options (1 <= J <= 16, t > 0, eps > 0, "
                                "1 <= qmax <= 12, reduction > 1)");
  if (!limits || limits->nrhs_max < 1 || limits->restart_max < 1 || limits->inner_k_max < 0 ||
      limits->restart_max > 128 || limits->inner_k_max > 128 ||
      (limits->flags & ~(HZ_LIMIT_SWEEPS_C64 | HZ_LIMIT_Z_C64 | HZ_LIMIT_CASE_TWO)) != 0 ||
      ((limits->flags & HZ_LIMIT_CASE_TWO) &&
       (limits->flags & (HZ_LIMIT_SWEEPS_C64 | HZ_LIMIT_Z_C64))))
    return fail(HZ_ERR_INVALID, "invalid limits (1 <= restart_max <= 128, 0 <= inner_k_max <= 128, "
                                "known flags only; HZ_LIMIT_CASE_TWO alone)");
  const long long n = (long long)grid->nx * grid->ny * grid->nz;
  for (long long i = 0; i < n; ++i)
    if (!(c_host[i] > 0) || !std::isfinite(c_host[i]))
      return fail(HZ_ERR_INVALID, "wavespeed must be positive and finite");
  if ((long long)grid->nz * limits->nrhs_max > 65535)
    return fail(HZ_ERR_INVALID, "nz * nrhs_max must not exceed 65535");
  hz::SpecPlan spec{};
  if (grid->discretization == HZ_DISC_SPECTRAL) {
    if (limits->flags & (HZ_LIMIT_CASE_TWO | HZ_LIMIT_Z_C64))
      return fail(HZ_ERR_INVALID, "spectral problems: HZ_LIMIT_SWEEPS_C64 is the only flag");
    const int dims[3] = {grid->nx, grid->ny, grid->nz};
    for (int a = 0; a < 3; ++a) {
      spec.ax[a].n = dims[a];
      if (!hz::fft_factor(dims[a], spec.ax[a].rad, &spec.ax[a].nst))
        return fail(HZ_ERR_INVALID, "spectral grid sizes must be products of 2, 3 and 5, at "
                                    "most 1024");
    }
  }

  hz_problem* p = new hz_problem();
  auto bail = [&](hz_status s) {
    delete p;
    return s;
  };
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  p->grid = *grid;
  p->copt = *contour;
  p->lim = *limits;
  p->J = contour->J;
  hz::setup_operator(*grid, c_host, p->su);
  p->g.nx = grid->nx;
  p->g.ny = grid->ny;
  p->g.nz = grid->nz;
  p->g.n = n;
  p->g.layer = grid->layer_cells;
  p->g.cs = p->su.s / (grid->h * grid->h);
  p->g.sig = grid->sigma_max;
  p->g.csf = float(p->g.cs);
  for (int c = 0; c < 3; ++c) p->g.pzc[c] = 4;
  p->g.prows[0] = 4;
  p->g.prows[1] = 2;
  p->g.prows[2] = 1;
  p->g.szc = 4;
  p->g.srows = 4;
  std::string err;
  p->case2 = (limits->flags & HZ_LIMIT_CASE_TWO) != 0;
  p->spectral = grid->discretization == HZ_DISC_SPECTRAL;
  p->spec = spec;
  p->nf = p->case2 ? 2 * n : n;
  bool nodes_ok;
  if (p->case2) {
    // Case Two: the rectangle of the Remark after Theorem thm:spectrum-2x2 for iC - I,
    // |mu + 1| <= R = rho2/2 + sqrt(rho2^2/4 + rho1), rho1 = rho(A1 + I) <= b2 + 1 (Weyl)
    hz::Setup s2 = p->su;
    const double rho1 = p->su.b2 + 1.0, rho2 = p->su.rho2;
    const double Rr = 0.5 * rho2 + std::sqrt(0.25 * rho2 * rho2 + rho1);
    s2.b1 = -1.0 - Rr;
    s2.b2 = -1.0 + Rr;
    nodes_ok = hz::setup_nodes(s2, *contour, p->nodes, err);
  } else {
    nodes_ok = hz::setup_nodes(p->su, *contour, p->nodes, err);
  }
  if (!nodes_ok) {
    delete p;
    return fail(HZ_ERR_SETUP, err);
  }
  const long long nf = p->nf;

  const int R = limits->nrhs_max, M = limits->restart_max, K = limits->inner_k_max;
  hz_status s;
  if ((s = dalloc(p, (void**)&p->m64, sizeof(double) * n)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->d64, sizeof(double2) * n)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->d32, sizeof(float2) * n)) != HZ_OK) return bail(s);
  p->sweeps32 = (limits->flags & HZ_LIMIT_SWEEPS_C64) != 0;
  p->z32 = (limits->flags & HZ_LIMIT_Z_C64) != 0;
  const size_t poly_es = p->sweeps32 ? sizeof(float2) : sizeof(double2);
  if ((s = dalloc(p, &p->poly, poly_es * 4 * (size_t)p->J * nf * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->f32, sizeof(float2) * (size_t)n * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->w, sizeof(double2) * (size_t)nf * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->Aw, sizeof(double2) * (size_t)nf * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->Vin, sizeof(double2) * (size_t)nf * (K + 1) * R)) != HZ_OK)
    return bail(s);
  if ((s = dalloc(p, (void**)&p->Vin32, sizeof(float2) * (size_t)n * (K + 1) * R)) != HZ_OK)
    return bail(s);
  if ((s = dalloc(p, (void**)&p->w32, sizeof(float2) * (size_t)n * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->Aw32, sizeof(float2) * (size_t)n * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->V, sizeof(double2) * (size_t)nf * (M + 1) * R)) != HZ_OK)
    return bail(s);
  if (p->z32) {
    if ((s = dalloc(p, (void**)&p->Z32, sizeof(float2) * (size_t)n * M * R)) != HZ_OK) return bail(s);
  } else {
    if ((s = dalloc(p, (void**)&p->Z, sizeof(double2) * (size_t)nf * M * R)) != HZ_OK) return bail(s);
  }
  // grids of the cooperative kernels (whole numbers of blocks per SM)
  {
    cudaError_t pe = hz::fci_tail32_plan(n, std::min(K, 4), &p->tail_ppt[0], &p->tail_blocks[0]);
    if (pe == cudaSuccess && K > 4)
      pe = hz::fci_tail32_plan(n, hz::TAIL_KMAX, &p->tail_ppt[1], &p->tail_blocks[1]);
    if (pe == cudaSuccess) pe = hz::arnoldi_ff_plan(n, M, &p->arn_ppt, &p->arn_blocks);
    if (pe == cudaSuccess) pe = hz::arnoldi64_plan(n, M, &p->a64_ppt, &p->a64_blocks);
    if (pe == cudaSuccess) pe = hz::fci_tail64_plan(n, &p->t64_ppt, &p->t64_blocks);
    if (pe != cudaSuccess) {
      delete p;
      return cuda_fail(pe, "cooperative kernel plans");
    }
    if (p->case2 || p->spectral) {
      // the cooperative kernels apply the 7-point operator of Case One only
      p->tail_ppt[0] = p->tail_ppt[1] = p->arn_ppt = p->a64_ppt = p->t64_ppt = 0;
    }
  }
  // block partial sums (16 bytes each): linear reduction kernels (>= 256 points a block) and
  // the fused stencil reductions (32 x 4 x 4 tiles, ragged at the edges), (slots x blocks) per
  // rhs; the cooperative kernels, two alternating areas of their slots x blocks
  const long long nblk = std::max<long long>(
      (nf + hz::RED_MIN_CHUNK - 1) / hz::RED_MIN_CHUNK,
      (long long)((grid->nx + 31) / 32) * ((grid->ny + 3) / 4) * ((grid->nz + 3) / 4));
  const int slots = std::max(M, K) + 2;
  const long long npart = std::max(
      {nblk * slots * R,
       2LL * (hz::TAIL_KMAX + 2) * std::max(p->tail_blocks[0], p->tail_blocks[1]),
       2LL * (M + 2) * p->arn_blocks, 2LL * (M + 2) * p->a64_blocks,
       2LL * (hz::TAIL64_KMAX + 2) * p->t64_blocks});
  if ((s = dalloc(p, (void**)&p->partial, sizeof(double2) * (size_t)npart)) != HZ_OK)
    return bail(s);
  if ((s = dalloc(p, (void**)&p->counters, sizeof(unsigned) * R)) != HZ_OK) return bail(s);
  if ((s = dalloc(p, (void**)&p->tail_bar, sizeof(unsigned) * 4)) != HZ_OK) return bail(s);
  const size_t gb = gmres_carved_bytes(R, M) + gmres_carved_bytes(R, K) + 1024;
  if ((s = dalloc(p, &p->gmem, gb)) != HZ_OK) return bail(s);
  char* cur = (char*)p->gmem;
  gmres_layout(p->gout, cur, R, M);
  gmres_layout(p->gin, cur, R, K);
  e = cudaMemset(p->gmem, 0, gb);
  if (e == cudaSuccess) e = cudaMemset(p->counters, 0, sizeof(unsigned) * R);
  if (e == cudaSuccess) e = cudaMemset(p->poly, 0, poly_es * 4 * (size_t)p->J * nf * R);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaMemset");
  }
  if (cudaMallocHost(&p->h_scal, sizeof(double) * hz::SC_COUNT * R) != cudaSuccess ||
      cudaMallocHost(&p->h_stopped, sizeof(int) * R) != cudaSuccess ||
      cudaMallocHost(&p->h_tol, sizeof(double) * R) != cudaSuccess ||
      cudaMallocHost(&p->h_bar, sizeof(unsigned) * 4) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(HZ_ERR_OOM, "pinned host allocation failed");
  }
  std::memset(p->h_bar, 0, sizeof(unsigned) * 4);
  // the inner GMRES of FCI never stops on a tolerance (SC_TOL < 0), fixed once here
  {
    std::vector<double> sc(hz::SC_COUNT * (size_t)R, 0.0);
    for (int r = 0; r < R; ++r) sc[r * hz::SC_COUNT + hz::SC_TOL] = -1.0;
    e = cudaMemcpy(p->gin.scal, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaMemcpy of inner tolerances");
    }
  }
  if (cudaStreamCreateWithFlags(&p->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    e = cudaGetLastError();
    delete p;
    return cuda_fail(e, "stream/event creation");
  }
  e = hz::prepare_kernels(std::max(M, K));
  if (e == cudaSuccess) e = hz::prepare_kernels32(std::max(K, 1));
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "kernel attributes");
  }
  e = cudaMemcpy(p->m64, p->su.m.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // diagonal of the float64 stencil: 6 s/h^2 - m - i a, a = sigma_max (depth/L)^2 m
    std::vector<double2> dg(n);
    const int L = grid->layer_cells;
    auto dep = [L](int idx, int nn) { return std::max(0, L - std::min(idx, nn - 1 - idx)); };
    for (int k = 0; k < grid->nz; ++k)
      for (int j = 0; j < grid->ny; ++j)
        for (int i = 0; i < grid->nx; ++i) {
          const long long q = i + (long long)grid->nx * (j + (long long)grid->ny * k);
          const double mp = p->su.m[q];
          double ap = 0.0;
          if (L > 0) {
            const int d = std::max(dep(i, grid->nx), std::max(dep(j, grid->ny), dep(k, grid->nz)));
            const double t = double(d) / double(L);
            ap = (grid->sigma_max * (t * t)) * mp;
          }
          dg[q] = make_double2((p->spectral ? 0.0 : 6.0 * p->g.cs) - mp, -ap);
        }
    e = cudaMemcpy(p->d64, dg.data(), sizeof(double2) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      std::vector<float2> dg32(n);
      for (long long q = 0; q < n; ++q) dg32[q] = make_float2(float(dg[q].x), float(dg[q].y));
      e = cudaMemcpy(p->d32, dg32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaMemcpy of coefficients");
  }
  e = cudaMemset(p->tail_bar, 0, sizeof(unsigned) * 3);
  if (e == cudaSuccess) {
    const unsigned lim = hz::GRID_SPINS_DEFAULT;
    e = cudaMemcpy(p->tail_bar + 3, &lim, sizeof(unsigned), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cooperative FCI tail set-up");
  }
  if (p->spectral) {
    e = hz::fft_prepare();
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "line-FFT kernel attributes");
    }
    // line-FFT tables of every axis: twiddles exp(-2 pi i k / n) and the eigenvalue shares
    // s (2 pi min(k, n - k) / (n h))^2, float64 on the host, rounded for the float32 kernels
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
      hz::FftAxis& ax = p->spec.ax[a];
      const int na = ax.n;
      std::vector<double2> tw(na);
      std::vector<float2> tw32(na);
      std::vector<double> ev(na);
      std::vector<float> ev32(na);
      for (int k = 0; k < na; ++k) {
        const double ang = 2.0 * std::acos(-1.0) * double(k) / double(na);
        tw[k] = make_double2(std::cos(ang), -std::sin(ang));
        tw32[k] = make_float2(float(tw[k].x), float(tw[k].y));
        const double kw = 2.0 * std::acos(-1.0) * double(std::min(k, na - k)) /
                          (double(na) * grid->h);
        ev[k] = p->su.s * kw * kw;
        ev32[k] = float(ev[k]);
      }
      void* d[4];
      const size_t sz[4] = {sizeof(double2) * na, sizeof(float2) * na, sizeof(double) * na,
                            sizeof(float) * na};
      const void* h[4] = {tw.data(), tw32.data(), ev.data(), ev32.data()};
      for (int b = 0; b < 4; ++b) {
        if ((s = dalloc(p, &d[b], sz[b])) != HZ_OK) return bail(s);
        e = cudaMemcpy(d[b], h[b], sz[b], cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
      }
      ax.tw64 = (const double2*)d[0];
      ax.tw32 = (const float2*)d[1];
      ax.e64 = (const double*)d[2];
      ax.e32 = (const float*)d[3];
    }
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "spectral tables");
    }
    // FFT scratch: a stage's batch of J x nrhs node inputs in double2 covers every use
    if ((s = dalloc(p, &p->spec_tmp, sizeof(double2) * (size_t)p->J * R * n)) != HZ_OK)
      return bail(s);
  }
  if (limits->autotune && !p->case2 && !p->spectral) {
    const hz_status ts = autotune(p);
    if (ts != HZ_OK) {
      delete p;
      return ts;
    }
  }
  *out = p;
  return HZ_OK;
}

hz_status hz_plan(const hz_grid* grid, const double* c_host, const hz_contour_opts* contour,
                  hz_problem_info* info, double* z_ri, double* sigma_ri, double* z0_ri,
                  double* delta, int* q, double* nu, int* sweeps) {
  if (!valid_grid(grid)) return fail(HZ_ERR_INVALID, "invalid grid");
  if (!c_host) return fail(HZ_ERR_INVALID, "c_host is null");
  if (!contour || contour->J < 1 || contour->J > hz::MAXJ || !(contour->t > 0) ||
      !(contour->eps > 0) || contour->qmax < 1 || contour->qmax > 12 ||
      !(contour->reduction > 1.0))
    return fail(HZ_ERR_INVALID, "invalid contour options");
  const long long n = (long long)grid->nx * grid->ny * grid->nz;
  for (long long i = 0; i < n; ++i)
    if (!(c_host[i] > 0) || !std::isfinite(c_host[i]))
      return fail(HZ_ERR_INVALID, "wavespeed must be positive and finite");
  hz::Setup su;
  hz::setup_operator(*grid, c_host, su);
  std::vector<NodeParams> nodes;
  std::string err;
  if (!hz::setup_nodes(su, *contour, nodes, err)) return fail(HZ_ERR_SETUP, err);
  if (info) {
    info->s = su.s;
    info->b1 = su.b1;
    info->b2 = su.b2;
    info->rho2 = su.rho2;
    info->J = contour->J;
    int T = 0;
    for (const auto& nd : nodes) T = std::max(T, nd.q * nd.sweeps);
    info->stages = T;
    info->n = n;
  }
  for (int j = 0; j < contour->J; ++j) {
    const NodeParams& nd = nodes[j];
    if (z_ri) { z_ri[2 * j] = nd.zr; z_ri[2 * j + 1] = nd.zi; }
    if (sigma_ri) { sigma_ri[2 * j] = nd.sr; sigma_ri[2 * j + 1] = nd.si; }
    if (z0_ri) { z0_ri[2 * j] = nd.z0r; z0_ri[2 * j + 1] = nd.z0i; }
    if (delta) delta[j] = nd.delta;
    if (q) q[j] = nd.q;
    if (nu) nu[j] = nd.nu;
    if (sweeps) sweeps[j] = nd.sweeps;
  }
  return HZ_OK;
}

hz_status hz_problem_fused_tail(hz_problem* p, int mode) {
  HZ_TRY(check_problem(p));
  if (mode < 0 || mode > 2) return fail(HZ_ERR_INVALID, "hz_problem_fused_tail: mode 0, 1 or 2");
  if (p->tail_mode != mode) p->drop_graphs();
  p->tail_mode = mode;
  return HZ_OK;
}

hz_status hz_problem_fused_arnoldi(hz_problem* p, int mode) {
  HZ_TRY(check_problem(p));
  if (mode < 0 || mode > 2) return fail(HZ_ERR_INVALID, "hz_problem_fused_arnoldi: mode 0, 1 or 2");
  if (p->arn_mode != mode) p->drop_graphs();
  p->arn_mode = mode;
  return HZ_OK;
}

hz_status hz_problem_set_spin_limit(hz_problem* p, long long polls) {
  HZ_TRY(check_problem(p));
  HZ_TRY(set_device(p));
  if (polls > 0xffffffffLL) return fail(HZ_ERR_INVALID, "poll limit above 2^32 - 1");
  const unsigned lim = polls < 0 ? hz::GRID_SPINS_DEFAULT : (unsigned)polls;
  // the problem's kernels run on its own stream: let them finish before the word changes
  HZ_CUDA(cudaStreamSynchronize(p->own));
  HZ_CUDA(cudaMemcpy(p->tail_bar + 3, &lim, sizeof(unsigned), cudaMemcpyHostToDevice));
  return HZ_OK;
}

hz_status hz_problem_set_preconditioner(hz_problem* p, hz_net* net, int mode) {
  HZ_TRY(check_problem(p));
  if (mode < 0 || mode > 3) return fail(HZ_ERR_INVALID, "preconditioner mode 0..3");
  if (mode != 0 && !net) return fail(HZ_ERR_INVALID, "modes 1..3 need a network");
  if (mode != 0 && p->spectral)
    return fail(HZ_ERR_INVALID, "the network preconditions 7-point problems only");
  if (mode != 0 && p->case2)
    return fail(HZ_ERR_INVALID, "the network preconditions Case One problems only");
  if (mode != 0 && !hz::net_fits(net, 1, p->g.nx, p->g.ny, p->g.nz))
    return fail(HZ_ERR_INVALID, "grid sizes must be multiples of 8 within the network's volume");
  HZ_TRY(set_device(p));
  if (mode != 0 && !p->pre_t) {
    const size_t bytes = sizeof(double2) * (size_t)p->g.n * p->lim.nrhs_max;
    HZ_TRY(dalloc(p, (void**)&p->pre_t, bytes));
    HZ_TRY(dalloc(p, (void**)&p->pre_z, bytes));
  }
  if (mode != p->net_mode || net != p->net) p->drop_graphs();
  p->net = mode != 0 ? net : nullptr;
  p->net_mode = mode;
  return HZ_OK;
}

hz_status hz_problem_set_inner_ilu(hz_problem* p, int on) {
  HZ_TRY(check_problem(p));
  if (on && p->case2) return fail(HZ_ERR_INVALID, "ILU(0) applies to Case One problems");
  if (on && p->spectral)
    return fail(HZ_ERR_INVALID, "ILU(0) applies to 7-point problems (spectral problems: "
                                "hz_problem_set_inner_invlap)");
  HZ_TRY(set_device(p));
  if (on && !p->invd) {
    HZ_CUDA(hz::ilu0_prepare());
    std::vector<double> invd;
    hz::ilu0_inverse_pivots(p->g.nx, p->g.ny, p->g.nz, p->g.cs, invd);
    HZ_TRY(dalloc(p, (void**)&p->invd, sizeof(double) * invd.size()));
    HZ_TRY(dalloc(p, (void**)&p->ilu_t, sizeof(double2) * (size_t)p->nf * p->lim.nrhs_max));
    HZ_CUDA(cudaMemcpy(p->invd, invd.data(), sizeof(double) * invd.size(),
                       cudaMemcpyHostToDevice));
    std::vector<float> invd32(invd.size());
    for (size_t q = 0; q < invd.size(); ++q) invd32[q] = float(invd[q]);
    HZ_TRY(dalloc(p, (void**)&p->invd32, sizeof(float) * invd32.size()));
    HZ_TRY(dalloc(p, (void**)&p->ilu_u32, sizeof(float2) * (size_t)p->g.n * p->lim.nrhs_max));
    HZ_CUDA(cudaMemcpy(p->invd32, invd32.data(), sizeof(float) * invd32.size(),
                       cudaMemcpyHostToDevice));
    HZ_TRY(dalloc(p, (void**)&p->ilu_prog,
                  sizeof(int) * (size_t)hz::ilu0_chain_prog_ints(p->g, p->lim.nrhs_max)));
    p->ilu_chain64 = hz::ilu0_chain_fits(p->g, p->lim.nrhs_max, false);
    p->ilu_chain32 = hz::ilu0_chain_fits(p->g, p->lim.nrhs_max, true);
  }
  if ((on != 0) != p->ilu_on) p->drop_graphs();
  p->ilu_on = on != 0;
  return HZ_OK;
}

hz_status hz_problem_set_inner_invlap(hz_problem* p, int on) {
  HZ_TRY(check_problem(p));
  if (on && !p->spectral)
    return fail(HZ_ERR_INVALID, "the inverse-Laplacian preconditioner needs a spectral problem");
  HZ_TRY(set_device(p));
  if (on && !p->ilu_t)  // the preconditioned inner GMRES's scratch field per right-hand side
    HZ_TRY(dalloc(p, (void**)&p->ilu_t, sizeof(double2) * (size_t)p->nf * p->lim.nrhs_max));
  if ((on != 0) != p->invlap_on) p->drop_graphs();
  p->invlap_on = on != 0;
  return HZ_OK;
}

hz_status hz_invlap_apply(hz_problem* p, const void* t, void* z, int nvec, void* stream) {
  HZ_TRY(check_problem(p));
  if (!p->spectral) return fail(HZ_ERR_INVALID, "hz_invlap_apply needs a spectral problem");
  if (nvec < 0 || nvec > p->lim.nrhs_max * p->J) return fail(HZ_ERR_INVALID, "nvec out of range");
  if (nvec == 0) return HZ_OK;
  if (!t || !z) return fail(HZ_ERR_INVALID, "null field");
  HZ_TRY(set_device(p));
  const long long n = p->g.n;
  HZ_CUDA(hz::launch_spectral<double2>(p->spec, p->g, hz::SPEC_INVLAP, hz::vec_map(t, n),
                                       hz::vec_map(z, n), nvec, p->d64, 0.0, 0.0,
                                       (double2*)p->spec_tmp, (cudaStream_t)stream));
  return HZ_OK;
}

hz_status hz_ilu0_apply(hz_problem* p, const void* t, void* z, int nvec, void* stream) {
  HZ_TRY(check_problem(p));
  if (!p->ilu_on) return fail(HZ_ERR_INVALID, "enable ILU(0) with hz_problem_set_inner_ilu first");
  if (nvec < 0 || nvec > 65535) return fail(HZ_ERR_INVALID, "nvec out of range");
  if (nvec == 0) return HZ_OK;
  if (!t || !z || t == z) return fail(HZ_ERR_INVALID, "null or overlapping fields");
  HZ_TRY(set_device(p));
  const long long n = p->g.n;
  if (p->ilu_chain64 && nvec <= p->lim.nrhs_max) {
    // the multi-block sweeps; a bounded wait that gave up is reported here (after a sync)
    HZ_CUDA(hz::launch_ilu0_chain(p->g, p->invd, Buf<const double2>{(const double2*)t, n},
                                  Buf<double2>{(double2*)z, n}, nvec, p->ilu_prog, p->tail_bar,
                                  (cudaStream_t)stream));
    p->tail_used = true;
    HZ_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return check_tail_fault(p);
  }
  HZ_CUDA(hz::launch_ilu0(p->g, p->invd, Buf<const double2>{(const double2*)t, n},
                          Buf<double2>{(double2*)z, n}, nvec, (cudaStream_t)stream));
  return HZ_OK;
}

hz_status hz_net_train_fields(hz_net* net, hz_problem* p, const void* r, const void* e, int nvec,
                              float lr, double* loss, void* stream) {
  HZ_TRY(check_problem(p));
  if (!net || !r || !e) return fail(HZ_ERR_INVALID, "null argument");
  if (nvec < 1) return fail(HZ_ERR_INVALID, "nvec < 1");
  HZ_TRY(set_device(p));
  return hz::net_train_fields(net, (const double2*)r, p->m64, (const double2*)e, nvec, p->g.nx,
                              p->g.ny, p->g.nz, lr, loss, (cudaStream_t)stream);
}

hz_status hz_profile_enable(hz_problem* p, int on) {
  HZ_TRY(check_problem(p));
  HZ_TRY(set_device(p));
  for (ProfClass& c : p->prof) {
    if (c.ev.empty()) {
      c.ev.resize(2 * kProfPool);
      for (cudaEvent_t& e : c.ev) HZ_CUDA(cudaEventCreate(&e));
    }
    HZ_TRY(prof_flush(c));
    c.launches = 0;
    c.ms = 0.0;
    c.bytes = 0.0;
    c.flops = 0.0;
  }
  p->prof_on = on != 0;
  return HZ_OK;
}

hz_status hz_profile_read(hz_problem* p, int cls, long long* launches, double* ms,
                          double* bytes, double* flops) {
  HZ_TRY(check_problem(p));
  if (cls < 0 || cls > 2) return fail(HZ_ERR_INVALID, "kernel class must be 0, 1 or 2");
  ProfClass& c = p->prof[cls];
  HZ_TRY(prof_flush(c));
  if (launches) *launches = c.launches;
  if (ms) *ms = c.ms;
  if (bytes) *bytes = c.bytes;
  if (flops) *flops = c.flops;
  return HZ_OK;
}

hz_status hz_problem_destroy(hz_problem* p) {
  if (!p) return HZ_OK;
  int cur = -1;
  cudaGetDevice(&cur);
  const int dev = p->device;
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  delete p;
  if (cur >= 0 && cur != dev) cudaSetDevice(cur);
  return HZ_OK;
}

hz_status hz_problem_get_info(const hz_problem* p, hz_problem_info* info) {
  HZ_TRY(check_problem(p));
  if (!info) return fail(HZ_ERR_INVALID, "info is null");
  info->s = p->su.s;
  info->b1 = p->su.b1;
  info->b2 = p->su.b2;
  info->rho2 = p->su.rho2;
  info->J = p->J;
  int T = 0;
  for (const auto& nd : p->nodes) T = std::max(T, nd.q * nd.sweeps);
  info->stages = T;
  info->n = p->g.n;
  for (int c = 0; c < 3; ++c) {
    info->tile_poly_zc[c] = p->g.pzc[c];
    info->tile_poly_rows[c] = p->g.prows[c];
  }
  info->tile_stencil_zc = p->g.szc;
  info->tile_stencil_rows = p->g.srows;
  return HZ_OK;
}

hz_status hz_problem_nodes(const hz_problem* p, double* z_ri, double* sigma_ri, double* z0_ri,
                           double* delta, int* q, double* nu, int* sweeps) {
  HZ_TRY(check_problem(p));
  for (int j = 0; j < p->J; ++j) {
    const NodeParams& nd = p->nodes[j];
    if (z_ri) { z_ri[2 * j] = nd.zr; z_ri[2 * j + 1] = nd.zi; }
    if (sigma_ri) { sigma_ri[2 * j] = nd.sr; sigma_ri[2 * j + 1] = nd.si; }
    if (z0_ri) { z0_ri[2 * j] = nd.z0r; z0_ri[2 * j + 1] = nd.z0i; }
    if (delta) delta[j] = nd.delta;
    if (q) q[j] = nd.q;
    if (nu) nu[j] = nd.nu;
    if (sweeps) sweeps[j] = nd.sweeps;
  }
  return HZ_OK;
}

hz_status hz_problem_set_nodes(hz_problem* p, int J, const double* z_ri, const double* sigma_ri,
                               const double* z0_ri, const double* delta, const int* q,
                               const int* sweeps) {
  HZ_TRY(check_problem(p));
  if (J < 1 || J > p->copt.J) return fail(HZ_ERR_INVALID, "J must be in [1, J at creation]");
  if (!z_ri || !sigma_ri || !z0_ri || !delta || !q || !sweeps)
    return fail(HZ_ERR_INVALID, "null node table");
  std::vector<NodeParams> nodes(J);
  for (int j = 0; j < J; ++j) {
    NodeParams& nd = nodes[j];
    nd.zr = z_ri[2 * j];
    nd.zi = z_ri[2 * j + 1];
    nd.sr = sigma_ri[2 * j];
    nd.si = sigma_ri[2 * j + 1];
    nd.z0r = z0_ri[2 * j];
    nd.z0i = z0_ri[2 * j + 1];
    nd.delta = delta[j];
    nd.q = q[j];
    nd.sweeps = sweeps[j];
    nd.nu = std::nan("");
    if (nd.q < 1 || nd.q > 64 || nd.sweeps < 1 || nd.sweeps > 100000 || (nd.zr == 0 && nd.zi == 0))
      return fail(HZ_ERR_INVALID, "node " + std::to_string(j) + ": need 1 <= q <= 64, "
                                  "1 <= sweeps <= 100000, z != 0");
  }
  p->nodes = nodes;
  p->J = J;
  p->drop_graphs();  // captured steps hold the old node parameters
  return HZ_OK;
}

hz_status hz_apply_shifted(hz_problem* p, double zr, double zi, const void* x, void* y, int nvec,
                           int precision, void* stream) {
  HZ_TRY(check_problem(p));
  if (nvec < 0) return fail(HZ_ERR_INVALID, "nvec < 0");
  if (nvec == 0) return HZ_OK;
  if (!x || !y) return fail(HZ_ERR_INVALID, "null field");
  if ((long long)p->g.nz * nvec > 65535) return fail(HZ_ERR_INVALID, "nz * nvec > 65535");
  HZ_TRY(set_device(p));
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = p->g.n;
  if (p->spectral) {
    if (nvec > p->lim.nrhs_max * p->J)
      return fail(HZ_ERR_INVALID, "spectral problems: nvec <= nrhs_max * J");
    if (precision == HZ_C128) {
      HZ_TIMED(p, 1, st, op64_bytes(p, nvec),
               (hz::launch_spectral<double2>(p->spec, p->g, hz::SPEC_APPLY,
                                             hz::vec_map(x, n), hz::vec_map(y, n), nvec, p->d64,
                                             zr, zi, (double2*)p->spec_tmp, st)));
    } else if (precision == HZ_MIXED_C64) {
      HZ_TIMED(p, 1, st, 0.5 * op64_bytes(p, nvec),
               (hz::launch_spectral<float2>(p->spec, p->g, hz::SPEC_APPLY, hz::vec_map(x, n),
                                            hz::vec_map(y, n), nvec, p->d32, zr, zi,
                                            (float2*)p->spec_tmp, st)));
    } else {
      return fail(HZ_ERR_INVALID, "unknown precision");
    }
    return HZ_OK;
  }
  if (precision == HZ_C128) {
    HZ_TIMED(p, 1, st, (stencil_bytes<double2, double2>(n, nvec)),
             (hz::launch_stencil_diag(p->g, p->d64,
                                                  Buf<const double2>{(const double2*)x, n},
                                                  Buf<double2>{(double2*)y, n}, nvec, zr, zi, st)));
  } else if (precision == HZ_MIXED_C64) {
    HZ_TIMED(p, 1, st, (stencil_bytes<float2, float2>(n, nvec)),
             (hz::launch_stencil32(p->g, p->d32,
                                                Buf<const float2>{(const float2*)x, n},
                                                Buf<float2>{(float2*)y, n}, nvec, zr, zi, st)));
  } else {
    return fail(HZ_ERR_INVALID, "unknown precision");
  }
  return HZ_OK;
}

hz_status hz_apply_2x2(hz_problem* p, double zr, double zi, const void* x, void* y, int nvec,
                       int precision, void* stream) {
  HZ_TRY(check_problem(p));
  if (nvec < 0) return fail(HZ_ERR_INVALID, "nvec < 0");
  if (nvec == 0) return HZ_OK;
  if (!x || !y) return fail(HZ_ERR_INVALID, "null field");
  if (nvec > 65535) return fail(HZ_ERR_INVALID, "nvec > 65535");
  if (p->g.n > 0x7fffffffLL) return fail(HZ_ERR_INVALID, "grid of 2^31 points or more");
  HZ_TRY(set_device(p));
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == HZ_C128) {
    HZ_CUDA(hz::launch_apply_2x2(p->g, p->d64, (const double2*)x, (double2*)y, nvec, zr, zi, st));
  } else if (precision == HZ_MIXED_C64) {
    HZ_CUDA(hz::launch_apply_2x2_32(p->g, p->d32, (const float2*)x, (float2*)y, nvec, float(zr),
                                    float(zi), st));
  } else {
    return fail(HZ_ERR_INVALID, "unknown precision");
  }
  return HZ_OK;
}

hz_status hz_shifted_solve(hz_problem* p, int node, const void* f, void* y, int nvec,
                           int precision, void* stream) {
  HZ_TRY(check_problem(p));
  if (node < 0 || node >= p->J) return fail(HZ_ERR_INVALID, "node out of range");
  if (nvec < 0 || nvec > p->lim.nrhs_max) return fail(HZ_ERR_INVALID, "nvec out of range");
  if (nvec == 0) return HZ_OK;
  if (!f || !y) return fail(HZ_ERR_INVALID, "null field");
  HZ_TRY(set_device(p));
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = p->nf;
  std::vector<int> which{node};
  std::vector<long long> yfin;
  Buf<double2> nob{nullptr, 0};
  size_t es;
  if (p->case2 && precision != HZ_C128)
    return fail(HZ_ERR_INVALID, "Case Two problems solve in HZ_C128");
  if (precision == HZ_C128 && p->sweeps32)
    return fail(HZ_ERR_INVALID, "HZ_C128 needs a problem created without HZ_LIMIT_SWEEPS_C64");
  if (precision == HZ_C128) {
    HZ_TRY((run_poly<double2, double>(p, p->d64, Buf<const double2>{(const double2*)f, n}, nvec,
                                      which, false, nob, &yfin, st)));
    es = sizeof(double2);
  } else if (precision == HZ_MIXED_C64) {
    HZ_TRY((run_poly<float2, float>(p, p->d32, Buf<const float2>{(const float2*)f, n}, nvec, which,
                                    false, nob, &yfin, st)));
    es = sizeof(float2);
  } else {
    return fail(HZ_ERR_INVALID, "unknown precision");
  }
  const long long wrs = 4LL * p->J * n;
  HZ_CUDA(cudaMemcpy2DAsync(y, es * n, (const char*)p->poly + es * yfin[0], es * wrs, es * n, nvec,
                            cudaMemcpyDeviceToDevice, st));
  return HZ_OK;
}

hz_status hz_fci(hz_problem* p, const void* r, void* out, int nvec, int inner_k, int precision,
                 void* stream) {
  HZ_TRY(check_problem(p));
  if (nvec < 0 || nvec > p->lim.nrhs_max) return fail(HZ_ERR_INVALID, "nvec out of range");
  if (inner_k < 0 || inner_k > p->lim.inner_k_max)
    return fail(HZ_ERR_INVALID, "inner_k out of range");
  if (precision != HZ_C128 && precision != HZ_MIXED_C64 && precision != HZ_MIXED_C64_FCI32 &&
      precision != HZ_MIXED_C64_FF)
    return fail(HZ_ERR_INVALID, "unknown precision");
  if (p->sweeps32 && precision == HZ_C128)
    return fail(HZ_ERR_INVALID, "HZ_C128 needs a problem created without HZ_LIMIT_SWEEPS_C64");
  if (p->case2 && precision != HZ_C128)
    return fail(HZ_ERR_INVALID, "Case Two problems solve in HZ_C128");
  if (p->ilu_on && precision != HZ_C128 && precision != HZ_MIXED_C64)
    return fail(HZ_ERR_INVALID, "ILU(0) preconditions the float64 inner GMRES (HZ_C128, "
                                "HZ_MIXED_C64)");
  if (p->spectral && precision != HZ_C128 && precision != HZ_MIXED_C64)
    return fail(HZ_ERR_INVALID, "spectral problems run HZ_C128 or HZ_MIXED_C64");
  if (nvec == 0) return HZ_OK;
  if (!r || !out) return fail(HZ_ERR_INVALID, "null field");
  HZ_TRY(set_device(p));
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = p->nf;
  return run_fci(p, Buf<const double2>{(const double2*)r, n}, Buf<double2>{(double2*)out, n}, nvec,
                 inner_k, precision, st);
}

hz_status hz_solve(hz_problem* p, const void* f, void* u, int nrhs, const hz_solve_opts* opts,
                   hz_solve_stats* stats, void* stream) {
  HZ_TRY(check_solve_args(p, nrhs, opts));
  if (nrhs == 0) return HZ_OK;
  if (!f || !u) return fail(HZ_ERR_INVALID, "null field");
  HZ_TRY(set_device(p));
  // run on the library's stream, ordered after the caller's stream
  const cudaStream_t user = (cudaStream_t)stream;
  HZ_CUDA(cudaEventRecord(p->ev_in, user));
  HZ_CUDA(cudaStreamWaitEvent(p->own, p->ev_in, 0));
  const cudaStream_t st = p->own;
  const hz_status status = solve_on(p, f, u, nrhs, opts, stats, st);
  cudaEventRecord(p->ev_out, st);
  cudaStreamWaitEvent(user, p->ev_out, 0);
  return status;
}

hz_status hz_solve_batched(hz_problem* const* probs, int nprob, const void* const* f,
                           void* const* u, const int* nrhs, const hz_solve_opts* opts,
                           hz_solve_stats* stats, void* stream) {
  if (nprob < 0 || (nprob > 0 && (!probs || !f || !u || !nrhs)))
    return fail(HZ_ERR_INVALID, "null argument array");
  if (nprob == 0) return HZ_OK;
  int dev = -1;
  HZ_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < nprob; ++i) {
    HZ_TRY(check_solve_args(probs[i], nrhs[i], opts));
    if (nrhs[i] > 0 && (!f[i] || !u[i])) return fail(HZ_ERR_INVALID, "null field");
    if (probs[i]->device != dev)
      return fail(HZ_ERR_INVALID, "all problems must live on the current device");
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) return fail(HZ_ERR_INVALID, "a problem appears twice");
  }
  const cudaStream_t user = (cudaStream_t)stream;
  HZ_CUDA(cudaEventRecord(probs[0]->ev_in, user));
  for (int i = 0; i < nprob; ++i) HZ_CUDA(cudaStreamWaitEvent(probs[i]->own, probs[0]->ev_in, 0));
  const hz_status status = solve_batched_on(probs, nprob, f, u, nrhs, opts, stats);
  for (int i = 0; i < nprob; ++i) {
    cudaEventRecord(probs[i]->ev_out, probs[i]->own);
    cudaStreamWaitEvent(user, probs[i]->ev_out, 0);
  }
  return status;
}

}  // extern "C"

namespace {

// One FGMRES(m) solve with FCI as the right preconditioner, split into enqueue and host phases
// so that several problems can advance in lockstep on their own streams (hz_solve_batched):
// the host waits once per outer step for all of them, while their kernels overlap on the GPU.
struct SolveState {
  hz_problem* p;
  const void* f;
  void* u;
  int nrhs;
  const hz_solve_opts* o;
  hz_solve_stats* stats;
  cudaStream_t st;
  int M = 0, K = 0;
  long long n = 0, vrs = 0, zrs = 0, mv_fci = 0;
  bool fixed = false;
  std::vector<double> fnorm, rel;
  std::vector<int> its, cycles, done, active;
  std::vector<long long> mvs;
  int cycle = 0, k = 0;
  bool diverged = false, finished = false, in_cycle = false;

  hz_status init() {
    M = o->restart_m;
    K = o->inner_k;
    n = p->nf;
    vrs = (long long)(p->lim.restart_max + 1) * n;
    zrs = (long long)p->lim.restart_max * n;
    fixed = o->fixed_its > 0;
    mv_fci = 1 + K;
    for (const auto& nd : p->nodes) mv_fci += nd.q * nd.sweeps - 1;
    fnorm.assign(nrhs, 0.0);
    rel.assign(nrhs, 1.0);
    its.assign(nrhs, 0);
    cycles.assign(nrhs, 0);
    done.assign(nrhs, 0);
    active.assign(nrhs, 0);
    mvs.assign(nrhs, 0);
    HZ_CUDA(cudaMemsetAsync(u, 0, sizeof(double2) * n * nrhs, st));
    return HZ_OK;
  }

  hz_status enqueue_flags() {
    GmresDev& go = p->gout;
    HZ_CUDA(cudaMemcpyAsync(p->h_scal, go.scal, sizeof(double) * hz::SC_COUNT * nrhs,
                            cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(p->h_stopped, go.stopped, sizeof(int) * nrhs, cudaMemcpyDeviceToHost,
                            st));
    if (p->tail_used)
      HZ_CUDA(cudaMemcpyAsync(p->h_bar, p->tail_bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost,
                              st));
    return HZ_OK;
  }

  // after the stream synchronised: a cooperative kernel's barrier gave up during this step
  // (the solve stops; drive() reports HZ_ERR_TIMEOUT)
  bool barrier_gave_up() {
    if (!p->tail_used || p->h_bar[0] == 0) return false;
    finished = true;
    in_cycle = false;
    return true;
  }

  // true residual r = s f - A u, v0 = r / ||r||
  hz_status enqueue_cycle_start() {
    GmresDev& go = p->gout;
    if (p->case2) {
      // Case Two: r = (0; s f) - (iC - I) U, U = (iu; u) the 2n-point iterate
      if (cycle > 0)
        HZ_CUDA(apply_op64(p, Buf<const double2>{(const double2*)u, n}, Buf<double2>{p->Aw, n},
                           nrhs, st));
      HZ_CUDA(hz::launch_residual_2x2((const double2*)f, p->g.n, p->su.s,
                                      cycle == 0 ? Buf<const double2>{nullptr, 0}
                                                 : Buf<const double2>{p->Aw, n},
                                      Buf<double2>{p->V, vrs}, p->g.n, go, p->partial,
                                      p->counters, nrhs, st));
      for (int r = 0; r < nrhs; ++r) mvs[r] += cycle == 0 ? 0 : 1;
      HZ_CUDA(hz::launch_scale(Buf<double2>{p->V, vrs}, Buf<const double2>{p->V, vrs}, n, go,
                               nrhs, st));
      return enqueue_flags();
    }
    if (p->spectral && cycle > 0) {
      // spectral: A u by the line FFTs, s f - A u in Aw, then the start from that field
      HZ_CUDA(apply_op64(p, Buf<const double2>{(const double2*)u, n}, Buf<double2>{p->Aw, n},
                         nrhs, st));
      HZ_CUDA(hz::launch_scaled_sub((const double2*)f, n, p->su.s, p->Aw, n, p->Aw, n, n, nrhs,
                                    st));
      HZ_CUDA(hz::launch_residual_start(p->g, p->m64, Buf<const double2>{p->Aw, n}, 1.0,
                                        Buf<const double2>{nullptr, 0}, Buf<double2>{p->V, vrs},
                                        go, p->partial, p->counters, nrhs, st));
    } else {
      HZ_CUDA(hz::launch_residual_start(p->g, p->m64, Buf<const double2>{(const double2*)f, n},
                                        p->su.s,
                                        cycle == 0 ? Buf<const double2>{nullptr, 0}
                                                   : Buf<const double2>{(const double2*)u, n},
                                        Buf<double2>{p->V, vrs}, go, p->partial, p->counters,
                                        nrhs, st));
    }
    for (int r = 0; r < nrhs; ++r) mvs[r] += cycle == 0 ? 0 : 1;
    if (o->precision == HZ_MIXED_C64_FF)
      HZ_CUDA(hz::launch_scale_ff_from64(Buf<float4>{(float4*)p->V, vrs},
                                         Buf<const double2>{p->V, vrs}, n, go, nrhs, st,
                                         Buf<float2>{p->f32, n}));
    else
      HZ_CUDA(hz::launch_scale(Buf<double2>{p->V, vrs}, Buf<const double2>{p->V, vrs}, n, go,
                               nrhs, st));
    return enqueue_flags();
  }

  // after the stream synchronised: convergence per rhs; start the next cycle or finish
  hz_status after_cycle_start() {
    GmresDev& go = p->gout;
    if (barrier_gave_up()) return HZ_OK;
    bool all_done = true;
    for (int r = 0; r < nrhs; ++r) {
      const double beta = p->h_scal[r * hz::SC_COUNT + hz::SC_BETA];
      if (cycle == 0) fnorm[r] = beta;
      rel[r] = fnorm[r] > 0 ? beta / fnorm[r] : 0.0;
      if (!std::isfinite(beta)) {
        diverged = true;
        done[r] = 1;
      } else if (fnorm[r] == 0.0) {
        done[r] = 1;
      } else if (fixed) {
        done[r] = its[r] >= o->fixed_its ? 1 : 0;
      } else {
        done[r] = rel[r] <= o->rtol ? 1 : 0;
      }
      all_done = all_done && done[r];
    }
    if (all_done || cycle >= o->max_cycles || diverged) {
      finished = true;
      return HZ_OK;
    }
    ++cycle;
    std::vector<double> tol(nrhs);
    for (int r = 0; r < nrhs; ++r) {
      tol[r] = fixed ? -1.0 : o->rtol * fnorm[r];
      p->h_stopped[r] = done[r];
      if (!done[r]) cycles[r]++;
      active[r] = !done[r];
    }
    HZ_TRY(fill_scal_tol(p, go, tol, nrhs, st));
    HZ_CUDA(cudaMemcpyAsync(go.stopped, p->h_stopped, sizeof(int) * nrhs, cudaMemcpyHostToDevice,
                            st));
    k = 0;
    in_cycle = true;
    return HZ_OK;
  }

  hz_status enqueue_step() {
    HZ_TRY(outer_step(p, k, nrhs, K, o->precision, st));
    for (int r = 0; r < nrhs; ++r)
      if (active[r]) {
        its[r]++;
        mvs[r] += mv_fci + 1;
      }
    return enqueue_flags();
  }

  // after the stream synchronised: stop flags; end the cycle when no rhs is left or m steps
  hz_status after_step() {
    GmresDev& go = p->gout;
    if (barrier_gave_up()) return HZ_OK;
    bool any_active = false, push = false;
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r]) continue;
      if (!std::isfinite(p->h_scal[r * hz::SC_COUNT + hz::SC_EST])) {
        diverged = true;
        p->h_stopped[r] = 1;
        push = true;
      }
      if (p->h_stopped[r]) {
        active[r] = 0;
        continue;
      }
      if (fixed && its[r] >= o->fixed_its) {
        p->h_stopped[r] = 1;
        active[r] = 0;
        push = true;
        continue;
      }
      any_active = true;
    }
    if (push)
      HZ_CUDA(cudaMemcpyAsync(go.stopped, p->h_stopped, sizeof(int) * nrhs, cudaMemcpyHostToDevice,
                              st));
    ++k;
    if (!any_active || k >= M) {
      // u += Z y (rhs done at the cycle start have kend = 0)
      in_cycle = false;
      HZ_CUDA(hz::launch_backsolve(go, nrhs, st));
      if (p->z32)
        HZ_CUDA(hz::launch_combine_b32(Buf<double2>{(double2*)u, n}, p->Z32, n, zrs, go, 1, n,
                                       nrhs, st));
      else
        HZ_CUDA(hz::launch_combine(Buf<double2>{(double2*)u, n}, p->Z, n, zrs, go,
                                   Buf<const double2>{nullptr, 0}, -1, 1, n, nrhs, M, st));
      if (diverged) finished = true;
    }
    return HZ_OK;
  }

  hz_status result() {
    hz_status ret = HZ_OK;
    for (int r = 0; r < nrhs; ++r) {
      const bool conv = std::isfinite(rel[r]) && rel[r] <= o->rtol;
      if (stats) {
        stats[r].cycles = cycles[r];
        stats[r].its = its[r];
        stats[r].matvecs = mvs[r];
        stats[r].converged = conv ? 1 : 0;
        stats[r].rel_res_true = rel[r];
      }
      if (!conv && !fixed && ret == HZ_OK) ret = HZ_ERR_NOT_CONVERGED;
    }
    if (diverged) return fail(HZ_ERR_DIVERGED, "a residual became NaN or Inf");
    if (ret == HZ_ERR_NOT_CONVERGED) t_err = "max_cycles reached above rtol";
    return ret;
  }
};

// Advances every state to the end in lockstep: a cycle start for all, then outer steps for all
// that are inside a cycle, one host synchronisation per round.
hz_status drive(std::vector<SolveState>& ss) {
  for (auto& s : ss) HZ_TRY(s.init());
  for (;;) {
    bool any = false;
    for (auto& s : ss)
      if (!s.finished) {
        HZ_TRY(s.enqueue_cycle_start());
        any = true;
      }
    if (!any) break;
    for (auto& s : ss)
      if (!s.finished) HZ_CUDA(cudaStreamSynchronize(s.st));
    for (auto& s : ss)
      if (!s.finished) HZ_TRY(s.after_cycle_start());
    for (;;) {
      bool stepping = false;
      for (auto& s : ss)
        if (!s.finished && s.in_cycle) {
          HZ_TRY(s.enqueue_step());
          stepping = true;
        }
      if (!stepping) break;
      for (auto& s : ss)
        if (!s.finished && s.in_cycle) HZ_CUDA(cudaStreamSynchronize(s.st));
      for (auto& s : ss)
        if (!s.finished && s.in_cycle) HZ_TRY(s.after_step());
    }
  }
  // the loop ends right after a residual evaluation, so rel[] is the final true residual
  for (auto& s : ss) HZ_CUDA(cudaStreamSynchronize(s.st));
  for (auto& s : ss) HZ_TRY(check_tail_fault(s.p));
  for (auto& s : ss)
    if (s.p->net_mode != 0 && s.p->net) HZ_TRY(hz::net_check(s.p->net));
  hz_status ret = HZ_OK;
  for (auto& s : ss) {
    const hz_status r = s.result();
    if (r != HZ_OK && (ret == HZ_OK || ret == HZ_ERR_NOT_CONVERGED)) ret = r;
  }
  return ret;
}

hz_status solve_batched_on(hz_problem* const* probs, int nprob, const void* const* f,
                           void* const* u, const int* nrhs, const hz_solve_opts* opts,
                           hz_solve_stats* stats) {
  // grid-wide barriers of cooperative kernels on concurrent streams could wait on each other's
  // resources: problems solved together use the multi-kernel FCI tail
  struct Solo {
    hz_problem* const* pr;
    int np;
    Solo(hz_problem* const* a, int b) : pr(a), np(b) {
      if (np > 1)
        for (int i = 0; i < np; ++i) pr[i]->tail_solo = false;
    }
    ~Solo() {
      for (int i = 0; i < np; ++i) pr[i]->tail_solo = true;
    }
  } solo(probs, nprob);
  std::vector<SolveState> ss;
  long long off = 0;
  for (int i = 0; i < nprob; ++i) {
    if (nrhs[i] == 0) continue;
    SolveState s;
    s.p = probs[i];
    s.f = f[i];
    s.u = u[i];
    s.nrhs = nrhs[i];
    s.o = opts;
    s.stats = stats ? stats + off : nullptr;
    s.st = probs[i]->own;
    ss.push_back(s);
    off += nrhs[i];
  }
  return drive(ss);
}

hz_status solve_on(hz_problem* p, const void* f, void* u, int nrhs, const hz_solve_opts* opts,
                   hz_solve_stats* stats, cudaStream_t st) {
  std::vector<SolveState> ss(1);
  ss[0].p = p;
  ss[0].f = f;
  ss[0].u = u;
  ss[0].nrhs = nrhs;
  ss[0].o = opts;
  ss[0].stats = stats;
  ss[0].st = st;
  return drive(ss);
}

}  // namespace

