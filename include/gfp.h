/*
 * gfp.h -- C ABI of the GB300 Green-function-preconditioned (GFP) fixed-point solver for the
 * periodic linear-elastic unit-cell problem (Khorrami, Mianroodi, Shanthraj, Svendsen,
 * "Development and comparison of spectral algorithms for numerical modeling of the
 * quasi-static mechanical behavior of inhomogeneous materials").
 *
 * One iteration (Sec. 5.2 Algorithm T-3D, Sec. 5.4 Algorithms P-3D and D-3D, in strain form):
 *   sigma = C(x) : eps                       (isotropic C, Sec. 5.1)
 *   T_check = forward 3D DFT of sigma         (eq. DisFouMat3D)
 *   eta = ||T_check q^b|| / ||T_check(0)||_F  (equilibrium residual; stop when eta < tol)
 *   Delta E_check = -Gamma(k) T_check         (Gamma from eq. EquMecFunGre3D, or Gamma^c of Alg. D)
 *   eps += inverse 3D DFT of Delta E_check    (the mean strain stays the prescribed E_bar)
 *
 * Conventions
 *   - Grids are n1 x n2 x n3 voxels, spacing h; every n_r must factor as 2^a 3^b, n_r <= 1024.
 *   - Fields are structure-of-arrays in C order with x1 fastest: field[c][i3][i2][i1].
 *   - Symmetric tensors use the six tensor components (11, 22, 33, 23, 13, 12) with no factor 2;
 *     only C_eff uses the Voigt (engineering shear) convention: for load J the mean strain is the
 *     Voigt unit vector e_J (tensor shear 1/2) and column J of C_eff is the mean stress.
 *   - "where" = 0 means a host pointer, 1 a device pointer (read or written in stream order on the
 *     grid's stream).  Output buffers are owned by the caller; the grid owns every device
 *     allocation it makes.  No pointer is kept beyond the call.
 *   - Every call returns a gfp_status.  Nothing is thrown across the ABI.  Calls on one grid are
 *     not thread-safe; distinct grids are independent.
 */
#ifndef GFP_H
#define GFP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfp_grid_s* gfp_grid;
typedef struct gfp_batch_s* gfp_batch;

typedef enum {
  GFP_OK = 0,
  GFP_ERR_ARG = -1,              /* bad argument (null pointer, negative size, NaN/non-positive mu, ...) */
  GFP_ERR_UNSUPPORTED_SIZE = -2, /* a grid size is not 2^a 3^b or exceeds the limit */
  GFP_ERR_OOM = -3,              /* device allocation failed */
  GFP_ERR_NOT_CONVERGED = -4,    /* maxit reached; the result is still filled */
  GFP_ERR_DIVERGED = -5,         /* eta is NaN/Inf or grew over a long window */
  GFP_ERR_DEVICE_TIMEOUT = -6,   /* a bounded device-side wait gave up */
  GFP_ERR_CUDA = -7,             /* a CUDA runtime call failed */
  GFP_ERR_UNSUPPORTED = -8       /* combination not implemented (e.g. mixed precision with DGO) */
} gfp_status;

/* Discretization of Sec. 3 (TD: trapezoidal, material sampled at x_i = (i-1)h; PCD: piecewise
 * constant, sampled at x_i^c = (i-1/2)h).  For the finite-difference schemes the half-cell phases of
 * the PCD transforms cancel (Sec. 3.2, "independent of s"), so both run the same iteration on the
 * given samples; the field tells which sampling the caller used.  DGO is PCD by definition. */
typedef enum { GFP_TD = 0, GFP_PCD = 1 } gfp_disc;

/* Effective wave vectors (Sec. 5.3, eqs. FreDifFinFBDF3D, FreDifFinFBDFR3D, EffNumWavConWil3D):
 *   GFP_F     plain Fourier q = i k, conjugate pairing
 *   GFP_CD    central differences, conjugate pairing
 *   GFP_ACD   averaged central differences, conjugate pairing
 *   GFP_HC    half-central differences, conjugate pairing
 *   GFP_AHC   averaged half-central differences, conjugate pairing
 *   GFP_AFB_R (AFD, AhC) average forward-backward / Willot's rotated scheme R
 *   GFP_DGO   discrete Green operator of Algorithm D-3D (alias sum over nu in [-m, m-1]^3)
 * For every pairing except DGO, q^a = e^{i phi} i kt and q^b = +-e^{-i phi'} i kt with one real vector
 * kt(k), and the strain increment is -Gamma0_iso(lambda_H, mu_H; kt) T_check, so AHC and AFB_R give
 * identical iterates. */
typedef enum { GFP_F = 0, GFP_CD = 1, GFP_ACD = 2, GFP_HC = 3, GFP_AHC = 4, GFP_AFB_R = 5, GFP_DGO = 6 } gfp_op;

typedef enum { GFP_FP64 = 0, GFP_MIXED = 1 } gfp_prec;

typedef struct {
  int disc;       /* gfp_disc */
  int op;         /* gfp_op */
  int dgo_m;      /* DGO alias half-range m (<= 0: n_r / 2 per axis, at least 1) */
  int prec;       /* gfp_prec: FP64 throughout, or FP32 FFT/Gamma/stress inner iterations inside an
                     FP64 outer loop (FP64 residual, mean strain and refinement correction) */
  int stop_rule;  /* 0: equilibrium residual eta (default); DGO uses the strain increment norm.
                     1: the stopping rule of Algorithms T-3D / P-3D (Sec. 5.2, 5.4): stop when
                     sum_mu |du^(it) - du^(it-1)| < tol, the L1 norm over the modes of the unitary
                     transform of the change of the displacement increment (the first iteration never
                     stops).  FP64 with CD, ACD, AHC or AFB_R only (GFP_ERR_UNSUPPORTED otherwise); not
                     with gfp_set_state resumes. */
  /* Variants of the discrete Green operator (GFP_DGO only; zero selects the defaults).  Algorithm D-3D
   * prints the weights s_j = sinc(pi j / n) and the update E_check += Gamma^c T_check; with them
   * -Gamma^c C_H has eigenvalues of both signs and the iteration can grow (on a two-phase cube at
   * contrast 10 it does).  The defaults are the squared weights and the polarization form
   * E = E_bar + F+ Gamma^c F- [(C - C_H) E] (the form the footnote to Algorithm D-1D names). */
  int dgo_power;  /* 0 or 2: weights s^2 (default); 1: the printed weights s */
  int dgo_form;   /* 0: polarization form (default); 1: the printed stress form, E_check += Gamma^c T_check */
  int dgo_range;  /* 0: alias range nu_r in [-m, m-1] as printed; 1: [-m, m], applied as its Hermitian part
                     1/2 (Gamma^c(omega) + Gamma^c(-omega)) since the strain is real */
} gfp_scheme;

typedef struct {
  int iters;              /* iterations (stress evaluations); a homogeneous cell reports 1 */
  int outer;              /* mixed precision: FP64 outer passes (0 in FP64 mode) */
  double residual;        /* final eta (stop_rule 1: the final increment criterion) */
  double sigma_mean[6];   /* mean stress, tensor components (11,22,33,23,13,12); FP64 solves form it by a
                             compensated real-space sum of C : (eps - estar) over the final strain */
  int status;             /* gfp_status of the solve */
  double* residual_history; /* caller-owned host array of history_cap doubles, or NULL: eta (stop_rule 1:
                               the criterion, infinite at the first iteration) per iteration, FP64 solves */
  int history_cap;
  int launches;           /* GPU kernels this call launched (iterations are launched in chunks between
                             convergence checks, so a few after convergence run as no-ops) */
} gfp_result;

/* Create a grid of n1 x n2 x n3 voxels with spacing h on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream).  Allocates every device buffer the solver needs (about (6*8 + 6*16*(n1/2+1)/n1 + 16)
 * bytes per voxel in FP64 mode).  On success *out receives the handle. */
int gfp_create_grid(int n1, int n2, int n3, double h, void* cuda_stream, gfp_grid* out);

/* Per-voxel Lame fields lambda, mu ([n3][n2][n1] float64; where = 0 host, 1 device).  They are the
 * samples C_i = C(x_i) (TD) or C(x_i^c) (PCD) of Algorithms T/P/D.  ref_lambda_mu may give the
 * reference medium (lambda_H, mu_H); NULL selects 1/2 (min + max) of each constant over the grid
 * (Sec. 4: C_H = 1/2 (C_M + C_I)).  mu must be > 0 and finite, lambda finite. */
int gfp_set_phases(gfp_grid g, const double* lambda, const double* mu, int where, const double* ref_lambda_mu);

/* Eigenstrain field E_* (the generalization stated at the end of Sec. 6: T = C[E - E_*], so that the
 * initial stress becomes T^(0) = C_i[E_bar - E_*i]): [6][n3][n2][n1] float64 tensor components
 * (11,22,33,23,13,12, no factor 2) sampled like lambda and mu; where = 0 host, 1 device (copied; the
 * caller keeps ownership).  NULL removes it.  It applies to gfp_solve in FP64 and mixed precision (the
 * FP64 stress of every outer pass; the FP32 correction equation does not involve it); the strain
 * returned stays the total strain.  While one is set, the DGO scheme, gfp_effective_stiffness,
 * gfp_grad and gfp_solve_batch return GFP_ERR_UNSUPPORTED (their results are defined for the
 * stiffness-only problem). */
int gfp_set_eigenstrain(gfp_grid g, const double* estar, int where);

/* Periodic displacement of the last solve, u^p = F^+ u_check, the primary unknown of Algorithms T/P
 * (Sec. 5.2, 5.4): recovered mode by mode from the strain fluctuation E~ = sym(u_check (x) q^a) with
 * the scheme's q^a (pass the scheme of the solve): u_check = (2 E~ kt - kt (kt.E~ kt)/|kt|^2) / (c i |kt|^2),
 * c = 1 except for AFB/R (c = e^{i(theta1+theta2+theta3)/2}, the forward difference's half-voxel
 * shift), 0 where kt = 0.  dst: [3][n3][n2][n1] float64 (where = 0 host, 1 device), zero mean; the
 * total displacement is E_bar x + u^p.  On Nyquist planes of even axes the schemes without the phase
 * (F, CD, ACD, HC, AHC) have a purely imaginary q^a, whose real displacement vanishes there: those
 * strain modes are not represented.  GFP_ERR_ARG before any solve; DGO returns GFP_ERR_UNSUPPORTED.
 * The grid's spectrum buffer is used as scratch; the strain is not changed. */
int gfp_get_displacement(gfp_grid g, const gfp_scheme* scheme, double* dst, int where);

/* Solve for the strain with prescribed mean E_macro (6 tensor components) until eta < tol or
 * maxit iterations.  The result's fields are filled even when the status is NOT_CONVERGED. */
int gfp_solve(gfp_grid g, const gfp_scheme* scheme, const double E_macro[6], double tol, int maxit,
              gfp_result* out);

/* Copy the current strain field (6 x [n3][n2][n1] float64, tensor components) to dst. */
int gfp_get_strain(gfp_grid g, double* dst, int where);

/* Effective stiffness: six solves with the Voigt unit loads; C_eff is 6x6 row-major (Voigt),
 * iters[6] receives the iteration count of each load (may be NULL). */
int gfp_effective_stiffness(gfp_grid g, const gfp_scheme* scheme, double tol, int maxit, double C_eff[36],
                            int iters[6]);

/* Sensitivities of C_eff,IJ (0 <= I, J < 6) to the per-voxel Lame constants:
 * dC_dlambda[i] = (1/N) tr eps^I_i tr eps^J_i,  dC_dmu[i] = (2/N) eps^I_i : eps^J_i,
 * where eps^I is the converged forward field of load I and eps^J the adjoint field, which for the
 * symmetric Gamma of every scheme here is the forward field of load J.  Outputs [n3][n2][n1]
 * float64 (where = 0 host, 1 device). */
int gfp_grad(gfp_grid g, const gfp_scheme* scheme, int I, int J, double tol, int maxit, double* dC_dlambda,
             double* dC_dmu, int where);

/* Batched homogenization (no counterpart in the paper): the six Voigt load cases of `count` cells of
 * possibly different sizes, mixed precision only (FP32 inner iterations, FP64 residual, mean strain and
 * refinement; schemes CD, ACD, AHC, AFB_R).  Every (cell, load) pair is a slot with its own device
 * buffers and state.  The batch is one CUDA graph holding one while-node per slot: the loop body is a
 * window of the slot's solve (an FP64 residual pass when its inner solve has reached its target, then
 * 32 FP32 inner iterations), and its last kernel decides on the device whether the slot runs another
 * window (outer residual still >= tol and fewer than ceil(maxit / 32) windows run).  A solve is one
 * graph launch; slots run concurrently and a finished slot stops launching.  The iterates and results
 * equal those of gfp_effective_stiffness.
 *
 * gfp_batch_create: validates the cells (phases set, no eigenstrain), allocates the slot buffers
 *   (about 230 bytes per voxel per load, owned by the handle) and builds the graph.  The grids must
 *   outlive the handle.  Errors: GFP_ERR_ARG, GFP_ERR_UNSUPPORTED (precision, scheme, stop rule or
 *   eigenstrain), GFP_ERR_OOM, GFP_ERR_CUDA; *out is NULL on error.
 * gfp_batch_solve: runs the batch from eps = E_J in every slot.  C_eff_out: count x 36 (row-major Voigt
 *   per cell); iters_out (may be NULL): count x 6 inner iterations per load.  A grid's new phases or
 *   tiles (gfp_set_phases, gfp_set_tiles) since the last build make it build the graph again.  Returns
 *   GFP_ERR_NOT_CONVERGED (results still filled) when a slot ran out of windows.  Calls on one handle
 *   must not overlap.
 * gfp_batch_destroy: waits for the handle's work and frees it.
 * gfp_solve_batch: create, solve and destroy in one call. */
int gfp_batch_create(int count, gfp_grid* grids, const gfp_scheme* scheme, gfp_batch* out);
int gfp_batch_solve(gfp_batch batch, double tol, int maxit, double* C_eff_out, int* iters_out);
int gfp_batch_destroy(gfp_batch batch);
int gfp_solve_batch(int count, gfp_grid* grids, const gfp_scheme* scheme, double tol, int maxit, double* C_eff_out,
                    int* iters_out);

/* Checkpoint/resume: the strain field and the iteration count fully determine a solve's state. */
int gfp_get_state(gfp_grid g, double* eps_dst, int* iters);
int gfp_set_state(gfp_grid g, const double* eps_src, int iters);

/* Measurement hook: runs `iters` iterations of the hot path on the grid's current strain (the
 * convergence test is disabled) with CUDA events around each kernel on the grid's stream, and returns
 * the mean duration in milliseconds of pass_x, pass_y (forward), pass_z_gamma, the residual reduction
 * and pass_y (inverse) in pass_ms[0..4].  With scheme->prec = GFP_MIXED it first runs one FP64
 * residual pass and then times the FP32 inner iterations.  The strain state is modified. */
int gfp_time_passes(gfp_grid g, const gfp_scheme* scheme, int iters, double pass_ms[5]);

/* Autotuner (no counterpart in the paper): times candidate tile shapes of each pass on this grid for
 * the scheme's precision -- lines per CTA of the register-FFT x-pass, k1 columns per CTA of the y and
 * z passes, and whether the z-pass loads its tiles with TMA -- and keeps the fastest; then, on every
 * axis whose length has no compile-time register-FFT plan (lengths other than 32, 64, 96, 128, 192,
 * 256, 512), it times candidate radix schedules of the shared-memory Stockham pass (the power of two
 * as radix-16, -8 or -4 stages, the radix-3 stages first or last) and keeps the fastest
 * (gfp_get_plans reads them).  tiles_out (may be
 * NULL) receives {x lines, y columns, z columns}, the x entry negated when the x-pass stages its loads
 * with cp.async and the z entry negated when the TMA z-pass is chosen.
 * The strain state is modified; call before a solve. */
int gfp_tune(gfp_grid g, const gfp_scheme* scheme, int iters, int tiles_out[3]);

/* Apply tile shapes for one precision (GFP_FP64 or GFP_MIXED), e.g. read from a tuning cache, in the
 * format gfp_tune returns; invalid shapes return GFP_ERR_ARG. */
int gfp_set_tiles(gfp_grid g, int prec, const int tiles[3]);

/* Radix schedules of the shared-memory Stockham passes for one precision (GFP_FP64 or GFP_MIXED), one per
 * axis: nst[r] stages with radices radix[12 r .. 12 r + nst[r] - 1], each in {2, 3, 4, 8, 16}, their
 * product n_r (unused entries 0).  gfp_set_plans applies schedules read back from gfp_get_plans (e.g. a
 * tuning cache); a schedule whose product is not n_r, with another radix or more than 12 stages returns
 * GFP_ERR_ARG.  Lengths with a register-FFT plan use these schedules only in the FP32 transforms of the
 * mixed solve's FP64 residual. */
int gfp_get_plans(gfp_grid g, int prec, int radix_out[36], int nst_out[3]);
int gfp_set_plans(gfp_grid g, int prec, const int radix[36], const int nst[3]);

int gfp_destroy_grid(gfp_grid g);

/* Allocation-free solve, for callers that cannot allocate GPU memory themselves, e.g. code that runs
 * where device memory is owned and pre-reserved by a host framework or pool, or where the device-wide
 * synchronisation of cudaMalloc/cudaFree would stall other work.  The paper has no counterpart: this
 * is gfp_solve (FP64, finite-difference schemes, residual stopping rule) without a grid handle.
 *   lambda, mu  device pointers, [n3][n2][n1] float64 (read);
 *   eps         device pointer, 6 x [n3][n2][n1] float64: the solver state and the output strain;
 *   ref_lambda_mu  host pointer to (lambda_H, mu_H), or NULL for 1/2 (min + max) of each constant;
 *   cuda_stream    stream for all work (NULL = legacy default stream).
 * It allocates nothing: its scratch (spectrum, tables, residual partials, state) lives in one
 * file-scope device array of 8 MiB (8388608 bytes) that every GPU loading the library holds until the
 * process exits.  A grid whose scratch does not fit (about 6 x 16 x (n1/2 + 1) x n2 x n3 bytes plus
 * a few KB; 48^3 fits, 64^3 does not) is rejected with GFP_ERR_UNSUPPORTED_SIZE and a message in
 * gfp_last_error_detail().  The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.  All calls share the array
 * and the previous call's contents stay in it (the solve clears what it needs), so calls that overlap
 * on the GPU -- concurrent streams, or threads -- race and must be serialised by the caller.
 * DGO and mixed precision return GFP_ERR_UNSUPPORTED. */
int gfp_solve_noalloc(int n1, int n2, int n3, double h, const double* lambda, const double* mu,
                      const double* ref_lambda_mu, const gfp_scheme* scheme, const double E_macro[6], double tol,
                      int maxit, double* eps, gfp_result* out, void* cuda_stream);

/* Measurement hook (no counterpart in the paper): the peak fused multiply-add rate of the current GPU,
 * in TFLOP/s (2 flops per FMA), from eight independent FMA chains per thread over 8 CTAs of 256 threads
 * per SM, best of three timed launches after one warm-up, on the legacy default stream.
 *   dtype   0: FP64, 1: FP32
 *   tflops  out: the measured rate
 * Used as the denominator of the FP64 path's arithmetic roofline (its transforms are bound by the FP64
 * units on this GPU).  Returns GFP_ERR_ARG for other dtypes or a null pointer, GFP_ERR_CUDA on a CUDA
 * error; allocates and frees a small device buffer. */
int gfp_measure_fma_peak(int dtype, double* tflops);

/* Static message for a status code. */
const char* gfp_error_string(int status);

/* Fault injection for tests of failure detection (no counterpart in the paper).  kind 1, value 1: every
 * later TMA-fed z-pass makes its first tile wait poll, with a short budget (2^22 cycles), a barrier that
 * nothing arrives at, so the wait runs out as a real one would after about a second: the kernel marks
 * the solve timed out, waits (bounded) until the tile loads it has issued have landed, and returns, and
 * the solve returns GFP_ERR_DEVICE_TIMEOUT with the CUDA context intact.  Value 0 turns it off.  No GPU
 * fault is involved and the tile barriers' byte counts stay those of the loads.  Other kinds or values
 * return GFP_ERR_ARG.  Not thread-safe. */
int gfp_set_fault_injection(int kind, int value);

/* Detail of the last CUDA runtime failure seen by this thread (CUDA's message, code and source line),
 * or an empty string.  The pointer stays valid until the thread's next failing call. */
const char* gfp_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* GFP_H */
