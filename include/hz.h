/*
 * hz.h -- C ABI of the GB300 contour-integral Helmholtz solver.
 *
 * The library solves A u = f for the discretised 3D Helmholtz operator -Delta - omega^2/c^2(x)
 * (Section 1, eq:helmholtz-op and eq:lin-sys) with a 7-point finite-difference Laplacian,
 * zero Dirichlet ghosts and a diagonal absorbing sponge (Section 7.1, eq:stiff-mass).
 * It uses the fast contour-integration preconditioner FCI of Algorithm 1 (Section 2) inside
 * flexible GMRES: every shifted system (A - z_j I) y = f at the contour nodes z_j of
 * eq:quad-points (Section 6.2) is solved by the polynomial fixed-point scheme eq:fix-pt-exp
 * (Section 4.2), with parameters chosen by eq:fix-pt-conv.
 *
 * Units.  Internally the operator is normalised as in Section 7.1:
 *     A = s * L_h - diag(m) - i * diag(a),   s = c_min^2 / omega^2,   m = c_min^2 / c^2,
 * L_h = 7-point -Delta_h, a = sigma_max * (depth/layer)^2 * m in the sponge (0 in the core),
 * so that the real part of the spectrum lies in [-1, rho1 - 1] and the imaginary part in
 * [-rho2, 0] (Lemma 3.1).  hz_apply_shifted, hz_shifted_solve and hz_fci work in these
 * normalised units.  hz_solve takes the physical right-hand side f of
 * -Delta u - omega^2/c^2 u = f and scales it by s internally, so u is in physical units.
 *
 * Layout.  A field is nx*ny*nz complex values, x fastest: point (i, j, k) at linear index
 * i + nx*(j + ny*k), interleaved (re, im).  HZ_C128 fields are double complex (16 bytes a
 * point), HZ_MIXED_C64 fields of hz_apply_shifted / hz_shifted_solve are float complex
 * (8 bytes a point).  A batch of nvec fields is stored one field after another.
 *
 * Memory.  Pointers named x, y, f, r, out, u are DEVICE pointers owned by the caller
 * (cudaMalloc / torch).  hz_problem_create copies the wavespeed from host memory and
 * allocates every workspace of the problem on the current device; no later call allocates.
 * Calls taking a stream enqueue their work on it (0 = legacy default stream); hz_solve
 * synchronises that stream to read convergence flags and returns when u is final.
 *
 * Errors.  Every call returns an hz_status and never aborts.  On HZ_ERR_CUDA the problem
 * should be destroyed.  hz_last_error() gives a message for the last failure on the
 * calling thread.
 */
#ifndef HZ_H
#define HZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hz_problem hz_problem;

typedef enum {
  HZ_OK = 0,
  HZ_ERR_INVALID = 1,        /* bad argument (null pointer, size, option) */
  HZ_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  HZ_ERR_OOM = 3,            /* device or pinned allocation failed */
  HZ_ERR_NOT_CONVERGED = 4,  /* hz_solve: max_cycles reached above rtol; u is the last iterate */
  HZ_ERR_BREAKDOWN = 5,      /* reserved */
  HZ_ERR_DIVERGED = 6,       /* hz_solve: a residual became NaN or Inf */
  HZ_ERR_SETUP = 7,          /* no polynomial order <= qmax converges at some node */
  HZ_ERR_TIMEOUT = 8         /* a grid-wide barrier of a cooperative kernel gave up waiting
                                (hz_problem_set_spin_limit); the solve stopped at that step */
} hz_status;

typedef enum {
  HZ_C128 = 0,        /* everything complex128 / float64 ("plain" form) */
  HZ_MIXED_C64 = 1,   /* polynomial sweeps in complex64; the quadrature-weighted sum of their
                         results accumulated in float64; step d, the inner and outer Arnoldi
                         (CGS2), Givens least squares and the true residual in float64 */
  HZ_MIXED_C64_FCI32 = 2, /* the whole FCI preconditioner in complex64 (sweeps, step d, inner
                         GMRES with float32 scalars), except its quadrature sum, accumulated in
                         float pairs (about 48 bits) and returned as float64; the outer
                         FGMRES (CGS2 Arnoldi, Givens, updates) and the true residual in
                         float64.  FGMRES admits a variable preconditioner, so the solution
                         still reaches the float64 residual target. */
  HZ_MIXED_C64_FF = 3  /* as HZ_MIXED_C64_FCI32, with the outer Arnoldi basis and its CGS2
                         passes in float pairs (two float32 per value, about 48 significant
                         bits, error-free float32 products and two-sum additions) instead of
                         float64; Hessenberg, Givens, the solution update and the true
                         residual stay float64.  Only hz_solve / hz_solve_batched distinguish
                         it; hz_fci treats it as HZ_MIXED_C64_FCI32. */
} hz_precision;

/* Discretisation of the Laplacian (Section 7.1). */
typedef enum {
  HZ_DISC_FD7 = 0,      /* 7-point finite differences, zero Dirichlet values outside the grid */
  HZ_DISC_SPECTRAL = 1  /* Fourier spectral S = F^H Lambda F on the periodic box of nx*ny*nz
                           points (eq:eig-Laplacian-spectral): Lambda_i = sum over the axes of
                           (2 pi min(i_a, n_a - i_a) / (n_a h))^2.  Each n_a must be a product of
                           2, 3 and 5 and at most 1024.  Spectral problems run HZ_C128 and
                           HZ_MIXED_C64, Case One, without the network or ILU(0) (their inner
                           preconditioner is hz_problem_set_inner_invlap). */
} hz_discretization;

/* Grid and medium.  Interior points nx*ny*nz with spacing h; omega the angular frequency;
 * layer_cells the sponge thickness in cells (0 = none); sigma_max its peak strength in
 * normalised units (Section 7.1: a diagonal damping, positive near the boundary, zero inside);
 * discretization an hz_discretization (0, the 7-point stencil, when zero-initialised). */
typedef struct {
  int nx, ny, nz;
  double h;
  double omega;
  int layer_cells;
  double sigma_max;
  int discretization;
} hz_grid;

/* Contour and polynomial-scheme settings (Sections 4.2, 6.1, 6.2).  J nodes on the ellipse
 * with axis ratio t and margin eps (eq:quad-points, eq:quad-radius); polynomial orders
 * 1..qmax are tried and each shifted solve runs the sweeps that reduce its error bound by
 * `reduction` (Table tab:param uses 5). */
typedef struct {
  int J;
  double t;
  double eps;
  int qmax;
  double reduction;
} hz_contour_opts;

/* Workspace limits fixed at creation: right-hand sides per call (nz * nrhs_max <= 65535),
 * outer restart length (1..128), inner GMRES steps (0..128).  autotune != 0 times the
 * candidate tile shapes of the polynomial-stage and complex64 stencil kernels on this grid
 * at creation (a few milliseconds) and keeps the fastest; 0 keeps fixed defaults.  Tiling
 * changes no result: every candidate performs the same arithmetic per point.  flags: an OR of
 * hz_limit_flags (0 for none), which trade precision forms for device memory. */
typedef struct {
  int nrhs_max;
  int restart_max;
  int inner_k_max;
  int autotune;
  int flags;
} hz_limits;

typedef enum {
  /* the polynomial workspace (4 J fields per right-hand side) sized for complex64 sweeps only:
     half the memory; HZ_C128 in hz_solve, hz_fci and hz_shifted_solve returns HZ_ERR_INVALID */
  HZ_LIMIT_SWEEPS_C64 = 1,
  /* FGMRES stores its directions z_k = FCI(v_k) rounded to complex64 (half the memory of the
     m direction fields).  The outer matvec A z_k is taken in float64 from the stored value, so
     the Arnoldi relation holds for the directions as stored and the solution update u += Z y
     (float64) stays consistent with the Krylov residual; this is FGMRES with a preconditioner
     whose output is rounded (Section 2, after Algorithm 1: any right preconditioner may vary
     from step to step).  hz_solve accepts only HZ_MIXED_C64 and HZ_MIXED_C64_FCI32 then. */
  HZ_LIMIT_Z_C64 = 2,
  /* Case Two of Section 3: the solver runs on the double-size matrix iC - I of eq:mat-2x2
     (float64, HZ_C128 only; not combined with the other flags).  The contour and the
     polynomial parameters come from the rectangle of the Remark after Theorem
     thm:spectrum-2x2: Re mu in [-1 - R, -1 + R], Im mu in [-rho2, 0], R = rho2/2 +
     sqrt(rho2^2/4 + rho1), rho1 = rho(A1 + I) bounded by Weyl's inequality.  Fields of the
     solver are 2n points (x1; x2): hz_fci takes and returns such fields, hz_shifted_solve
     returns them, and hz_solve takes the physical f (n points per right-hand side) and
     returns Y = (i u; u) (2n points per right-hand side; u is its second half), solving
     (iC - I) Y = (0; s f); its stats report the residual of that system.  The workspace is
     twice that of a Case One problem. */
  HZ_LIMIT_CASE_TWO = 4
} hz_limit_flags;

/* hz_solve settings.  restart_m <= restart_max, inner_k <= inner_k_max.  precision is an
 * hz_precision.  fixed_its > 0 takes exactly that many outer Arnoldi steps (cycles of
 * restart_m) ignoring rtol, for run-to-run comparison of iterates. */
typedef struct {
  int restart_m;
  int inner_k;
  double rtol;
  int max_cycles;
  int precision;
  int fixed_its;
} hz_solve_opts;

/* Per right-hand side results of hz_solve. */
typedef struct {
  int cycles;           /* FGMRES restarts begun */
  int its;              /* outer Arnoldi steps */
  long long matvecs;    /* stencil applications charged to this right-hand side */
  int converged;        /* 1 if the true relative residual <= rtol */
  double rel_res_true;  /* ||f - A u|| / ||f|| recomputed at the end, float64 */
} hz_solve_stats;

/* Scalars of a problem after set-up. */
typedef struct {
  double s;        /* c_min^2 / omega^2 */
  double b1, b2;   /* real extent of the spectrum rectangle B (Lemma 3.1 with Weyl bounds) */
  double rho2;     /* largest damping = height of B */
  int J;           /* contour nodes */
  int stages;      /* stencil sweeps of one FCI application (max over nodes of q*sweeps) */
  long long n;     /* grid points */
  int tile_poly_zc[3];    /* polynomial stage z-column length for 1, 2-3, >= 4 active nodes */
  int tile_poly_rows[3];  /* polynomial stage grid rows per block, same classes */
  int tile_stencil_zc;    /* complex64 stencil z-column length */
  int tile_stencil_rows;  /* complex64 stencil rows per block */
} hz_problem_info;

/* Create a problem: copy the wavespeed c_host (nx*ny*nz doubles, x fastest, host memory),
 * build m and the sponge, bound the spectrum (Lemma 3.1), place the J contour nodes
 * (eq:quad-points), pick (z0, delta, q, sweeps) per node (eq:fix-pt-conv) and allocate all
 * device workspace for `limits`.  Uses the current CUDA device.  *out receives the handle. */
hz_status hz_problem_create(const hz_grid* grid, const double* c_host,
                            const hz_contour_opts* contour, const hz_limits* limits,
                            hz_problem** out);

/* Host-only planning: the scalars of hz_problem_get_info (info->n, s, b1, b2, rho2, J,
 * stages) and the node tables of hz_problem_nodes that hz_problem_create would compute for
 * this grid, wavespeed (host array as in hz_problem_create) and contour.  Touches no GPU and
 * allocates no device memory.  Table pointers may be null; non-null ones take J entries. */
hz_status hz_plan(const hz_grid* grid, const double* c_host, const hz_contour_opts* contour,
                  hz_problem_info* info, double* z_ri, double* sigma_ri, double* z0_ri,
                  double* delta, int* q, double* nu, int* sweeps);

/* Free the problem and all its device memory.  Null is accepted. */
hz_status hz_problem_destroy(hz_problem* p);

hz_status hz_problem_get_info(const hz_problem* p, hz_problem_info* info);

/* Copy the node tables out (host arrays, J entries each; complex values as (re, im) pairs):
 * nodes z_j, weights sigma_j (Section 6.1), expansion centres z0_j, step delta_j, order q_j,
 * rate nu_j (eq:fix-pt-conv) and sweeps_j.  Any pointer may be null. */
hz_status hz_problem_nodes(const hz_problem* p, double* z_ri, double* sigma_ri, double* z0_ri,
                           double* delta, int* q, double* nu, int* sweeps);

/* Replace the node tables (J <= the J given at creation; host arrays as in
 * hz_problem_nodes; nu is not needed).  Lets a caller run the method with externally
 * chosen nodes and parameters. */
hz_status hz_problem_set_nodes(hz_problem* p, int J, const double* z_ri, const double* sigma_ri,
                               const double* z0_ri, const double* delta, const int* q,
                               const int* sweeps);

/* y = (A - z I) x for nvec fields (normalised operator; Section 7.1).  x and y must not
 * overlap.  precision HZ_C128: double complex fields; HZ_MIXED_C64: float complex fields,
 * computed in float32. */
hz_status hz_apply_shifted(hz_problem* p, double zr, double zi, const void* x, void* y,
                           int nvec, int precision, void* stream);

/* Case Two of Section 3 (eq:mat-2x2): y = ((iC - I) - z I) x for the double-size matrix with
 * C = [[0, I], [-(A1 + I), -A2]], where A = A1 - i A2 is the normalised operator split into its
 * Hermitian part A1 = s L_h - diag(m) and A2 = diag(a).  Each of the nvec vectors is two
 * fields stored one after the other, x = (x1; x2) (2*nx*ny*nz values), so (iC - I)(iu; u) =
 * (0; f) exactly when A u = f.  For Hermitian A (layer_cells = 0 or sigma_max = 0) the shift
 * z = s gives the shifted form eq:shifted-2x2; with a sponge the lower blocks are -i(A1 + I)
 * and -i A2 - (s + 1) I instead.  x and y must
 * not overlap.  precision HZ_C128: double complex; HZ_MIXED_C64: float complex, computed in
 * float32.  HZ_ERR_INVALID for nvec > 65535 or grids of 2^31 points or more. */
hz_status hz_apply_2x2(hz_problem* p, double zr, double zi, const void* x, void* y, int nvec,
                       int precision, void* stream);

/* y ~ (A - z_node I)^{-1} f for nvec fields by sweeps_node steps of eq:fix-pt-exp from
 * y = 0 (Section 4.2).  Field type as in hz_apply_shifted.  nvec <= nrhs_max. */
hz_status hz_shifted_solve(hz_problem* p, int node, const void* f, void* y, int nvec,
                           int precision, void* stream);

/* out = FCI(r) (Algorithm 1) for nvec double-complex fields: the J shifted solves, the
 * quadrature w = sum_j sigma_j/z_j y_j, the step d = argmin ||r - d A w||, inner_k GMRES
 * steps on A v = r - d A w, out = v + d w.  precision (an hz_precision) selects where the
 * work runs in complex64; r and out are always double complex.  nvec <= nrhs_max. */
hz_status hz_fci(hz_problem* p, const void* r, void* out, int nvec, int inner_k, int precision,
                 void* stream);

/* Solve -Delta u - omega^2/c^2 u = f for nrhs double-complex right-hand sides (physical
 * units) by FGMRES(restart_m) with FCI as the right preconditioner, x0 = 0.  Convergence is
 * declared on the float64 true residual ||f - A u|| <= rtol ||f||.  stats: nrhs entries
 * (may be null).  Returns HZ_ERR_NOT_CONVERGED if any right-hand side missed rtol. */
hz_status hz_solve(hz_problem* p, const void* f, void* u, int nrhs, const hz_solve_opts* opts,
                   hz_solve_stats* stats, void* stream);

/* Solve several problems at once (instances of different grid sizes, media and contours,
 * each with its own right-hand sides): the FGMRES cycles of all problems advance in lockstep,
 * each problem's kernels on its own stream so that they overlap on the GPU, with one host
 * synchronisation per outer step for all of them.  probs: nprob distinct problems on the
 * current device; f[i], u[i]: device fields of problem i (nrhs[i] each, physical units as in
 * hz_solve); stats: sum of nrhs[i] entries in problem order (may be null).  Results equal
 * separate hz_solve calls.  Returns the first failure, else HZ_ERR_NOT_CONVERGED if any
 * right-hand side missed rtol. */
hz_status hz_solve_batched(hz_problem* const* probs, int nprob, const void* const* f,
                           void* const* u, const int* nrhs, const hz_solve_opts* opts,
                           hz_solve_stats* stats, void* stream);

/* Kernel timing for roofline reports.  While enabled on a problem, each launch of a kernel
 * class is bracketed by CUDA events on its stream, and the algorithmic bytes it must move
 * (fields read and written once, neighbours not counted again) are added up.  Classes:
 * 0 = batched polynomial stage (eq:fix-pt-exp sweeps + quadrature; timed as whole stage
 * sequences, so its time includes the short gaps between stages), 1 = shifted stencil,
 * 2 = Krylov reductions (CGS2, norms, step d).  hz_profile_read synchronises the recorded
 * events and returns, per class, launches, total milliseconds, total algorithmic bytes and
 * the algorithmic float64 flops of the float64 kernels among them (an FMA counts 2; float32
 * kernels add none) since the last enable; any output pointer may be null. */
hz_status hz_profile_enable(hz_problem* p, int on);

/* ILU(0) of the 7-point discrete Laplacian (Section 6.3, used for the finite-difference runs of
 * Section 7.3) as the right preconditioner of the inner GMRES of FCI (Algorithm 1 step 4):
 * the inner GMRES minimises ||g - A M^{-1} x|| and returns v = M^{-1} x.  M = (D + L) D^{-1}
 * (D + U) is the incomplete factorisation without fill of the normalised operator's Laplacian
 * part s L_h in natural order (x fastest): L, U its strict lower and upper parts, d_p =
 * 6 s/h^2 - (s/h^2)^2 * (sum of 1/d_q over the lower neighbours q).  on != 0 enables it (the
 * first time it computes the pivots on the host and allocates one float64 field per
 * right-hand side); it applies to the float64 inner GMRES of HZ_C128 and HZ_MIXED_C64, and
 * hz_solve / hz_fci refuse the complex64-FCI forms while it is on.  Case One problems only. */
hz_status hz_problem_set_inner_ilu(hz_problem* p, int on);

/* z = M^{-1} t with the ILU(0) factors above, for nvec double-complex fields of n points
 * (device; t and z must not overlap).  Needs hz_problem_set_inner_ilu(p, 1).  The sweeps run as
 * a wavefront over z-slabs, one block per slab, where all blocks fit on the device at once
 * (then the call synchronises the stream and returns HZ_ERR_TIMEOUT if a bounded wait between
 * blocks gave up), else in one block per field (asynchronous). */
hz_status hz_ilu0_apply(hz_problem* p, const void* t, void* z, int nvec, void* stream);

/* Spectral problems (HZ_DISC_SPECTRAL): right-precondition the inner GMRES of FCI (step 4 of
 * Algorithm 1) with the regularised inverse Laplacian M^{-1} = F^H diag(1 / max(lambda_i, 1)) F,
 * lambda_i = s Lambda_i the normalised eigenvalues of the spectral Laplacian (Section 7.3: the
 * spectral runs' preconditioner; Section 6.3: an approximate Laplacian deflates the large
 * eigenvalues).  The inner GMRES then runs on A M^{-1} and FCI returns M^{-1} x + d w.  on = 0
 * turns it off.  HZ_ERR_INVALID for a 7-point problem.  Applies to HZ_C128 and HZ_MIXED_C64
 * (the float64 inner GMRES). */
hz_status hz_problem_set_inner_invlap(hz_problem* p, int on);

/* z = M^{-1} t with the regularised inverse Laplacian above, for nvec double-complex fields
 * of n points (device; t and z may be the same buffer).  nvec <= nrhs_max * J.  Any spectral
 * problem (it need not be switched on).  Asynchronous on `stream`. */
hz_status hz_invlap_apply(hz_problem* p, const void* t, void* z, int nvec, void* stream);

/* Poll limit of the grid-wide barriers inside the cooperative kernels (hz_problem_fused_tail,
 * hz_problem_fused_arnoldi): a block polls the barrier at most `polls` times (back to back,
 * then about 32 ns apart) before it gives up; polls < 0 restores the default (2^23, about a
 * second).  A barrier that gives up makes its kernel return early, hz_solve stops after that
 * outer step and returns HZ_ERR_TIMEOUT (u is then not a solution), and the next call starts
 * clean.  With polls = 0 every barrier wait that is not already satisfied gives up at once.
 * Waits for the problem's queued work first.  Not in the paper: a guard for shared devices. */
hz_status hz_problem_set_spin_limit(hz_problem* p, long long polls);

/* Selects how the complex64 forms run steps 3-5 of Algorithm 1 (step d, the inner GMRES,
 * v + d w) for a single right-hand side.  mode = 1 (the default): one cooperative kernel whose
 * phases are separated by grid-wide barriers, where the grid fits on the device and
 * k_in <= 16; each h_{j+1,j} comes from ||w'||^2 - ||V^H w'||^2 after the second Gram-Schmidt
 * pass (w' the vector after the first), or, where that difference would cancel, from a summed
 * norm.  mode = 2: the same kernel, always summing the norm.  mode = 0: one kernel per Arnoldi
 * piece.  The modes differ only in float32 rounding.  Several right-hand sides per call, and
 * problems solved together by hz_solve_batched, always use mode 0.  Other modes:
 * HZ_ERR_INVALID.  A barrier that waits longer than about a second gives up, and the next
 * hz_solve on the problem returns HZ_ERR_CUDA. */
hz_status hz_problem_fused_tail(hz_problem* p, int mode);

/* Selects how HZ_MIXED_C64_FF runs each outer Arnoldi step of FGMRES (Section 3: w = A z_k,
 * the two classical Gram-Schmidt passes against v_0..v_k, the Givens rotation of the new
 * Hessenberg column, v_{k+1} = w / h_{k+1,k}) for a single right-hand side.  mode = 1 (the
 * default): one cooperative kernel with two grid-wide barriers, where the grid fits on the
 * device; h_{k+1,k} comes from ||w'||^2 - ||V^H w'||^2 after the second pass (w' the vector
 * after the first), or, where that difference would cancel, from a third summed norm.
 * mode = 2: the same kernel, always summing the norm.  mode = 0: five kernels (stencil, three
 * Gram-Schmidt passes, normalisation).  The modes differ only in rounding.  Several right-hand
 * sides per call, and hz_solve_batched, always use mode 0.  Other modes: HZ_ERR_INVALID.  A
 * barrier timeout is reported as for hz_problem_fused_tail. */
hz_status hz_problem_fused_arnoldi(hz_problem* p, int mode);
hz_status hz_profile_read(hz_problem* p, int cls, long long* launches, double* ms,
                          double* bytes, double* flops);

/* Residual without any device allocation, for callers that cannot call cudaMalloc (code
 * running while their stream is being captured into a CUDA graph, allocators that own a
 * fixed arena, hosts that control the GPU memory budget).  Needs no hz_problem.  For nvec
 * double-complex fields (device, x fastest) computes r = fscale*f - A u with A the
 * normalised operator of this header built from the device wavespeed c (nx*ny*nz doubles)
 * and c_min = min c: m = c_min^2/c^2, s = c_min^2/omega^2; u may be null (r = fscale*f), r may
 * be null (not stored).  norm2 (device, nvec doubles) receives ||r||^2; with
 * fscale = c_min^2/omega^2 this is the residual hz_solve reports for u.  The paper has no
 * counterpart: this is a deployment aid.
 * Scratch lives in one static device array of 1 MiB (+256 bytes) that every device loading
 * the library keeps until exit: nvec <= 64 and nvec * ceil(nx*ny*nz / 1024) <= 65536, else
 * HZ_ERR_INVALID.  All calls share it: calls that overlap on the GPU race, so serialise
 * them (one stream).  The first call on a device looks up the array's device address (with
 * that device current); make it before any stream capture.  Asynchronous on `stream`. */
/* (7-point grids only: HZ_ERR_INVALID for grid->discretization != HZ_DISC_FD7.) */
hz_status hz_residual_noalloc(const hz_grid* grid, const double* c, double c_min, const void* f,
                              double fscale, const void* u, void* r, double* norm2, int nvec,
                              void* stream);

/* ---- The learned right preconditioner ----
 * The paper has no network: flexible GMRES admits a right preconditioner that changes from
 * step to step (Section 2, the remark after Algorithm 1), so a learned map from a residual to
 * an approximate error can serve as one, alone or combined with FCI, while the float64 true
 * residual still decides convergence.  The network is a 4-level 3D U-Net with 16 base channels
 * and 3x3x3 kernels; its convolutions run on the tensor cores in BF16 with FP32 accumulation,
 * its training (forward, backward, Adam) on the GPU.  Input per voxel: 8 channels (Re r, Im r,
 * the medium m = c_min^2/c^2, five zeros) with r scaled to unit RMS; output: 2 channels
 * (Re e, Im e), scaled back.  Volumes are multiples of 8 in each direction.
 * Parameters: one flat float32 array of hz_net_param_count() values: for each of the 14
 * convolutions in the order e1a (8->16), e1b (16->16), e2a (16->32), e2b, e3a (32->64), e3b,
 * ba (64->128), bb, d3a (192->64), d3b, d2a (96->32), d2b, d1a (48->16), d1b, the weights
 * w[Cout][27][Cin] (tap t = 9 dz + 3 dy + dx for offsets dz - 1, dy - 1, dx - 1) then the bias
 * b[Cout]; then the head's w[2][16] and b[2].  The decoder's inputs are the upsampled map
 * followed by the skip map. */
typedef struct hz_net hz_net;

long long hz_net_param_count(void);

/* Allocate a network (parameters zero) with activation and gradient storage for up to
 * batch_max volumes of D x H x W voxels (multiples of 8, >= 8) on the current device. */
hz_status hz_net_create(int D, int H, int W, int batch_max, hz_net** out);
hz_status hz_net_destroy(hz_net* net);

/* Copy the parameters in from host memory (and reset Adam's moments) or out to host memory. */
hz_status hz_net_set_params(hz_net* net, const float* host);
hz_status hz_net_get_params(const hz_net* net, float* host);

/* y = N(x): x device float32 [batch][D][H][W][8] (rounded to bf16 on entry), y device float32
 * [batch][D][H][W][2].  Synchronises the stream.  HZ_ERR_TIMEOUT if a bounded wait inside a
 * tensor-core kernel gave up. */
hz_status hz_net_forward(hz_net* net, const float* x, float* y, int batch, int D, int H, int W,
                         void* stream);

/* One training step on device float32 inputs x [batch][D][H][W][8] and targets
 * [batch][D][H][W][2]: forward, loss L = sum over samples of sum |y - t|^2 / (2 D H W) into
 * *loss (host), every parameter gradient (into grads, device float32, the parameter layout, if
 * not null), and an Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr (none
 * for lr = 0).  Synchronises the stream. */
hz_status hz_net_train_step(hz_net* net, const float* x, const float* target, int batch, int D,
                            int H, int W, float lr, float* grads, double* loss, void* stream);

/* The same on nvec pairs of complex128 device fields (residual r, error e with A e = r) of
 * problem p's grid: the input is built from r / rms(r) and p's medium, the target is
 * e / rms(r). */
hz_status hz_net_train_fields(hz_net* net, hz_problem* p, const void* r, const void* e, int nvec,
                              float lr, double* loss, void* stream);

/* Right preconditioner of hz_solve: mode 0 FCI (Algorithm 1, the default; net may be null);
 * 1 the network alone, z = N(v); 2 z = d N(v) + FCI(v - d A N(v)) with the least-squares step
 * d = (A N v)^H v / ||A N v||^2 (the step of Algorithm 1's step 3 applied to the network's
 * output, so that v - d A N(v) is never larger than v); 3 z = FCI(v) + N(v - A FCI(v)).
 * The network must hold the grid (multiples of 8) and nrhs_max volumes; allocates two float64
 * fields per right-hand side on first use.  HZ_MIXED_C64_FF is refused with a network. */
hz_status hz_problem_set_preconditioner(hz_problem* p, hz_net* net, int mode);

/* Single 3x3x3 convolutions on the tensor cores, for checking the network's kernels.
 * hz_conv3d: y = conv3(x, w) + bias (ReLU if relu), x device bf16 [B][D][H][W][Cin] (Cin a
 * multiple of 8), w device float32 [Cout][27][Cin] (Cout a multiple of 16, <= 256), bias
 * float32 [Cout] or null, y device float32 [B][D][H][W][Cout].  hz_conv3d_backward: for the
 * output gradient g (device bf16 [B][D][H][W][Cout], Cout <= 128) dw = sum over voxels of
 * g (x) shifted x (device float32 [Cout][27][Cin]) and, if dx is not null, dx = the input
 * gradient (device float32 [B][D][H][W][Cin], Cin a multiple of 16).  workspace: device,
 * hz_conv3d_workspace_bytes(Cin, Cout) bytes, 16-byte aligned.  Both synchronise the stream. */
hz_status hz_conv3d(const void* x, int B, int D, int H, int W, int Cin, const float* w,
                    const float* bias, int Cout, int relu, float* y, void* workspace,
                    void* stream);
hz_status hz_conv3d_backward(const void* x, const void* g, int B, int D, int H, int W, int Cin,
                             const float* w, int Cout, float* dx, float* dw, void* workspace,
                             void* stream);
long long hz_conv3d_workspace_bytes(int Cin, int Cout);

/* Name of a status code. */
const char* hz_status_string(hz_status s);

/* Message of the last failure on the calling thread ("" if none). */
const char* hz_last_error(void);

/* Kernels this library has launched since it was loaded (all problems, all threads;
 * kernels replayed from the solver's CUDA graphs count once per replay). */
unsigned long long hz_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
