/*
 * gpe.h -- C ABI of libgpe: GB300 (sm_103a) kernels for the regularized Newton
 * ground-state method of Wu, Wen & Bao, "A Regularized Newton Method for
 * Computing Ground States of Bose-Einstein Condensates" (arXiv:1504.02891).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grids (paper §2).  For GPE_FOURIER, n[a] is the number of periodic points N_a
 * on [lo, hi) with x_j = lo + j h, h = (hi-lo)/N_a, j = 0..N_a-1 (§2.3).  For
 * GPE_SINE and GPE_FD, n[a] is the number of intervals N_a and the unknowns are
 * the N_a - 1 interior nodes x_j = lo + j h, j = 1..N_a-1 (§2.1, §2.2).
 *
 * Layout.  A grid function ("psi buffer") is a DEVICE array, row-major
 * [batch][nz][ny][nx] with x fastest, of the plan's precision: float/double when
 * the plan is real (is_complex = 0), interleaved complex float2/double2 when it
 * is complex.  Values are physical grid values psi_j with the discrete norm
 * ||psi||_h^2 = h_vol * sum |psi_j|^2, h_vol = prod h_a.
 *
 * Units.  E and mu are the paper's E_h and mu_h (Eq. energy-discrete-FD,
 * energy-discrete-SP-34, energy-discrete-FP, chemical-potential).  H psi is
 * (-1/2 Delta_h + V + beta |psi|^2 - Omega L_z,h) psi, so the paper's gradient
 * G_h = nabla E_h equals 2 h_vol H psi.
 *
 * Ownership.  The caller owns every psi/direction/output buffer and keeps it
 * alive until the work queued on the plan's stream has finished.  The plan owns
 * its tables (potential, symbols, twiddles), workspace and reduction scratch.
 *
 * Execution.  Work is queued on the CUDA stream given at plan creation (NULL:
 * the legacy default stream).  Entry points that return host scalars
 * synchronise that stream; the others are asynchronous.  Buffers must not
 * alias unless an entry point says so.
 *
 * Errors.  Every call returns a gpe_status; nothing aborts or throws across the
 * ABI.  gpe_last_error() returns a message for the last failure on the calling
 * thread.  Invalid arguments return GPE_EINVAL before any work is queued.
 */
#ifndef GPE_H
#define GPE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpe_plan_s* gpe_plan;

typedef enum {
  GPE_OK = 0,
  GPE_EINVAL = 1,      /* bad argument (shape, pointer, option)                */
  GPE_ECUDA = 2,       /* a CUDA runtime call failed                            */
  GPE_ENOMEM = 3,      /* device allocation failed                              */
  GPE_ENONFINITE = 4,  /* a reduction produced NaN/Inf                          */
  GPE_ENOCONV = 5,     /* iteration cap reached; outputs are still written      */
  GPE_ETIMEOUT = 6     /* a bounded device wait expired                         */
} gpe_status;

typedef enum { GPE_FOURIER = 0, GPE_SINE = 1, GPE_FD = 2 } gpe_disc;
typedef enum { GPE_F32 = 0, GPE_F64 = 1 } gpe_prec;

/* External trap V (Eq. harmpen, optic98/asypon, §4.2 Case II):
 *   GPE_V_HARMONIC: V = 1/2 sum_a g_a^2 x_a^2,           v_param[0..2] = g_x, g_y, g_z
 *   GPE_V_LATTICE : harmonic + A sum_a sin^2(k x_a),      v_param[3] = A, v_param[4] = k
 *   GPE_V_STIRRER : harmonic + w0 exp(-d((x-r0)^2+y^2)),  v_param[3] = w0, [4] = d, [5] = r0
 *   GPE_V_ARRAY   : v_host points to the potential on the grid (host, float64,
 *                   one instance's unknowns in the layout above); copied.      */
typedef enum { GPE_V_HARMONIC = 0, GPE_V_LATTICE = 1, GPE_V_STIRRER = 2, GPE_V_ARRAY = 3 } gpe_vkind;

typedef struct {
  int dim;               /* 1, 2 or 3                                           */
  int n[3];              /* N_a per axis (see Grids); unused axes ignored       */
  double lo[3], hi[3];   /* computational box U                                 */
  int disc;              /* gpe_disc                                            */
  double beta;           /* interaction constant                                */
  double omega;          /* rotation speed; nonzero needs is_complex, dim >= 2,
                            and GPE_FOURIER or GPE_FD (§2.2 uses sine for
                            Omega = 0 only)                                      */
  int is_complex;        /* 0: real psi (Omega = 0), 1: complex psi             */
  int v_kind;            /* gpe_vkind                                           */
  double v_param[8];
  const double* v_host;  /* GPE_V_ARRAY only                                    */
} gpe_problem;

/* Create a plan for `nbatch` >= 1 instances of problem *p on one device.
 * Fourier grids need every n[a] to be a power of two in [4, 1024]; sine grids
 * need n[a] a power of two in [4, 512] (the DST-I runs as a 2N-point FFT of
 * the odd extension); FD grids need n[a] >= 3.  prec is gpe_prec.  stream is
 * a cudaStream_t (may be NULL).  On success *out receives the plan.
 * Errors: GPE_EINVAL (shape/option), GPE_ENOMEM, GPE_ECUDA. */
gpe_status gpe_plan_create(const gpe_problem* p, int nbatch, int prec, void* stream,
                           gpe_plan* out);

/* Release the plan and everything it owns (synchronises its stream). */
gpe_status gpe_plan_destroy(gpe_plan plan);

/* Text of the last failure on this thread ("" if none).  Never NULL. */
const char* gpe_last_error(void);

/* Number of unknowns of one instance and the cell volume h_vol. */
gpe_status gpe_plan_size(gpe_plan plan, int64_t* n_unknowns, double* h_vol);

/* Discrete energy of each instance: E[b] = E_h(psi_b), mu[b] = mu_h(psi_b),
 * norm2[b] = ||psi_b||_h^2 (Eq. energy-discrete-*, chemical-potential, §2).
 * Each output is a host array of nbatch doubles, or NULL.  Synchronises.
 * Reductions are accumulated in float64 whatever the plan precision. */
gpe_status gpe_energy(gpe_plan plan, const void* psi, double* E, double* mu, double* norm2);

/* hpsi = H(psi) psi = (-1/2 Delta_h + V + beta|psi|^2 - Omega L_z,h) psi, i.e.
 * G_h / (2 h_vol) with G_h of Eq. Gh1dsin and its Fourier/FD analogues.  If E or
 * mu is non-NULL it also returns E_h and mu_h per instance (host arrays;
 * synchronises); otherwise the call is asynchronous.  hpsi must not alias psi. */
gpe_status gpe_grad(gpe_plan plan, const void* psi, void* hpsi, double* E, double* mu);

/* out = H_psi[d] + shift * d, the Hessian of Lemma 3.1 in grid units:
 * H_psi[d] = (-1/2 Delta_h + V - Omega L_z,h) d + beta (|psi|^2 d + 2 Re(conj(psi) d) psi).
 * In the unified variables X = sqrt(h_vol) psi of Eq. prob this is
 * nabla^2 F(X)[D] / 2.  Asynchronous.  out must not alias psi or d. */
gpe_status gpe_hessvec(gpe_plan plan, const void* psi, const void* d, double shift, void* out);

/* One sphere-preserving Cayley step (Eq. eq-Y, Theorem 3.3) in the unified
 * variables X = sqrt(h_vol) psi, G = 2 sqrt(h_vol) hpsi, for every instance:
 *   Y(tau) = a(tau) X + b(tau) G, then scaled to ||Y||_2 = 1 (the §4
 *   renormalisation), written back in grid units to psi_out.
 * psi must satisfy ||psi||_h ~ 1 and hpsi must be H(psi) psi (gpe_grad).
 * tau >= 0 is the step of Theorem 3.3 in the unified variables.  If E_out is
 * non-NULL, E_h(psi_out) per instance is returned (synchronises).
 * psi_out must not alias psi or hpsi. */
gpe_status gpe_feasible_step(gpe_plan plan, const void* psi, const void* hpsi, double tau,
                             void* psi_out, double* E_out);

/* Cascadic transfer (Algorithm 3): interpolate psi_c from the coarse plan's
 * grid to the fine plan's grid and renormalise to ||psi_f||_h = 1.  Both plans
 * must have the same dim, box, discretisation, complexity, batch and precision,
 * and fine->n[a] = 2 * coarse->n[a].  Fourier: zero-padding of the centred
 * spectrum with the Nyquist coefficient split evenly; sine: zero-padding of the
 * DST-I coefficients; FD: linear interpolation.  Runs on the fine plan's stream. */
gpe_status gpe_prolong(gpe_plan coarse, gpe_plan fine, const void* psi_c, void* psi_f);

/* Options of gpe_rnewton_solve.  gpe_solve_opts_default() fills the values
 * given in brackets. */
typedef struct {
  int levels;         /* cascade levels of Algorithm 3, >= 1 (coarsest = n >> (levels-1)) [1] */
  int mode;           /* 0: float64 throughout; 1: float32 bulk (Algorithm 1 on
                         every level) then float64 regularized Newton on the
                         finest level; 2: float32 only                         [1] */
  int method;         /* 0: Algorithm 2 (regularized Newton); 1: Algorithm 1    [0] */
  int k_init;         /* Algorithm 1 warm-start iterations in Algorithm 2       [100] */
  int k_sub;          /* Algorithm 1 iterations per subproblem (Eq. tr-sub)     [200] */
  int max_outer;      /* regularized Newton iterations per level and precision  [200] */
  int max_iter;       /* Algorithm 1 iterations when method = 1                 [2000] */
  double eps0;        /* Eq. crit1 tolerance (Algorithm 1)                      [1e-6] */
  double delta_stop;  /* Eq. crit2 tolerance on accepted steps (Algorithm 2)    [1e-8] */
  double res_tol;     /* stop when ||H psi - mu psi||_h <= res_tol (0 = off)    [1e-9] */
  double delta0;      /* initial regularisation (unified variables)             [1.0] */
  double switch_rel;  /* modes 1, 2: the float32 bulk (Algorithm 1 on every
                         level) stops once ||A(X)X|| <= switch_rel * |X^*G|, or
                         when 40 steps bring no new smallest residual          [1e-6] */
  int chunk;          /* Algorithm 1 iterations queued between host checks      [16] */
  int use_graphs;     /* capture the queued iterations in CUDA graphs           [1] */
  int persistent;     /* spectral grids: run each Algorithm 1 run as one
                         cooperative persistent launch (grid barriers with
                         bounded waits; GPE_ETIMEOUT if one expires)            [1] */
  int cluster;        /* float32 Algorithm 1 on 2D Fourier grids: one thread-block
                         cluster holds the whole state in distributed shared
                         memory (grids up to 256^2 complex)                      [1] */
  int search;         /* line search of every Algorithm 1 run: 0 the nonmonotone
                         search of Eq. NMLS-Armijo from half a BB step (Eq. bb-1);
                         1 the monotone Armijo search of the Remark after
                         Theorem 3.4 (Eq. Armijo1): tau = alpha_hat 2^-m, m the
                         smallest integer (<= 60) with F(Y(tau)) <=
                         F(X) - rho1 tau ||A(X)X||^2                          [0] */
  double alpha_hat;   /* search 1: first trial step, > 0 (unified units)      [1e-3] */
  double eta;         /* search 0: weight of the reference value C^(k) in
                         Eq. NMLS-Armijo, 0 <= eta < 1 (0: C^(k) = F(X^(k)),
                         a monotone test from BB steps)                        [0.85] */
} gpe_solve_opts;

typedef struct {
  double E, mu;       /* E_h, mu_h of the result (float64 evaluation)           */
  double res;         /* ||H psi - mu psi||_h of the result                     */
  int status;         /* gpe_status of the solve                               */
  int outer_f32, outer_f64;   /* regularized Newton iterations on the finest level */
  int inner_f32, inner_f64;   /* Algorithm 1 iterations on the finest level         */
  int nfe;                    /* operator applications, all levels              */
  double ms_f32, ms_f64;      /* wall time of the float32 / float64 phases       */
} gpe_solve_report;

gpe_status gpe_solve_opts_default(gpe_solve_opts* opts);

/* Ground state by Algorithm 3 (cascade) around Algorithm 2 (or 1), for a plan
 * with nbatch = 1.  psi_inout holds the initial guess on the plan's (finest)
 * grid; the coarsest level starts from its values at the coarse nodes
 * (injection), normalised.  On return psi_inout holds the computed state,
 * normalised, in the plan's precision.  report may be NULL.  Synchronises.
 * Returns GPE_ENOCONV if an iteration cap ended the finest level before the
 * stopping rules (the state is still written). */
gpe_status gpe_rnewton_solve(gpe_plan plan, void* psi_inout, const gpe_solve_opts* opts,
                             gpe_solve_report* report);

/* Second-order certificate of a stationary state (Lemma 3.2, Eq. sec-opt):
 * the smallest value of grad^2 F(X)[D, D] - theta D^*D over unit D in the
 * tangent set T_X = {D : X^*D = 0} (Eq. tangent-St), in the unified units of
 * Eq. prob (X = sqrt(h_vol) psi, theta = 2 mu; equal to twice the smallest
 * eigenvalue of P (H'' - mu) P in grid units, H'' as in gpe_hessvec and P the
 * projector onto the complement of psi and, for complex data, i psi).  A
 * negative value shows a saddle (not a minimiser); a local minimiser has a
 * value >= 0, and for complex data the phase direction i psi is excluded.
 * psi: device grid function of the plan (nbatch = 1), a stationary state for
 * the test to be meaningful (any state is accepted).  Lanczos with full
 * reorthogonalisation from a fixed pseudo-random start vector, at most
 * max_iter (2..1000) steps, until the Ritz residual estimate is below
 * tol * max(1, |value|).  lambda_min receives the value; residual (may be
 * NULL) the true residual norm of the Ritz pair in the same units; iters (may
 * be NULL) the Lanczos steps taken.  Allocates its Lanczos vectors per call
 * (max_iter + 3 grid functions) and synchronises the plan's stream. */
gpe_status gpe_hess_min_eig(gpe_plan plan, const void* psi, int max_iter, double tol, double* lambda_min,
                            double* residual, int* iters);

/* Many independent ground-state problems in one call: the mixed schedule,
 * batched.  First Algorithm 1 (Theorem 3.3 step, Eq. bb-1 BB step, Eq.
 * NMLS-Armijo search) in float32 with float64 reductions and device-side
 * control for every instance at once; then (opts->mode 1, the default) for
 * every instance that has not reached res_tol, the float64 refinement of the
 * mixed schedule: Algorithm 2 (Eq. TR-ratio, update-X, tau-up) with float64
 * outer quantities and float32 difference-form subproblems, at most
 * max_outer outer steps (k_sub, delta0 as in gpe_rnewton_solve; Eq. crit2 is
 * not used: an instance stops at res_tol or max_outer).  mode 2: the float32
 * stage only.  Other modes: GPE_EINVAL.  problems[i] (i < n): 2D
 * Fourier grids whose state fits one thread-block cluster (n[0], n[1] powers
 * of two, up to 256^2; real with omega = 0, or complex); each instance has
 * its own beta, omega and potential.  Instances with the same grid (extents,
 * box, complexity) run in one cluster launch, clusters taking the next
 * unstarted instance when one finishes, each instance stopping on its own
 * criteria.  psi[i]: device buffer of problems[i]'s grid in float32 (complex64
 * interleaved when complex), the initial guess in physical units on entry
 * (normalised on the grid), the state on return.  opts (NULL = defaults):
 * max_iter bounds the iterations per instance; an instance stops when
 * ||H psi - mu psi||_h <= res_tol, or ||A(X)X|| <= switch_rel |X^*G|, or after
 * 40 accepted steps without a new smallest residual (the float32 floor).
 * The states are returned in float32 (after a refinement: the float64 state
 * rounded to float32).  reports[i] receives E, mu and res of the final
 * evaluation (float32 stage: float64 sums of float32 values; refined: the
 * float64 state), inner_f32 / outer_f64 / inner_f64 (iterations), nfe,
 * ms_f32 (the float32 stage's time per instance of its group), ms_f64 (the
 * refinement of that instance), and status GPE_OK when res <= res_tol,
 * GPE_ENOCONV when an instance stopped short of it (max_iter, the float32
 * floor or switch_rel in mode 2, max_outer after a refinement), or
 * GPE_ENONFINITE.  Runs on cuda_stream (NULL = legacy
 * default stream) and synchronises; allocates its own scratch per call.
 * Returns GPE_EINVAL for a grid outside the above and GPE_ENONFINITE if any
 * instance went non-finite (the other states are still written). */
gpe_status gpe_solve_batch(const gpe_problem* problems, int n, void* const* psi, const gpe_solve_opts* opts,
                           gpe_solve_report* reports, void* cuda_stream);

/* Measured launch shapes (the paper has no counterpart: an implementation
 * choice).  For a plan on a 2D Fourier grid, times on the plan's stream:
 *   - the register-FFT line kernels of the H-apply (gpe_grad) of this grid and
 *     batch, for 1, 2, 4 and 8 resident waves of CTAs per kernel;
 *   - the cluster engine of single float32 solves (Algorithm 1, 24 iterations
 *     from a Gaussian) on this grid and on the `levels` - 1 coarser cascade
 *     grids, for each per-CTA share of a state vector in {2,...,32} KiB that
 *     gives a distinct cluster size;
 * and records the fastest choices in a process-wide table keyed by grid (and
 * batch), which every later launch on those shapes uses (without an entry:
 * 4 waves, 4 KiB).  Launch shapes do not change computed values (reductions
 * may differ by rounding order); the fused-or-two-kernel choice changes the
 * FFT factorisation, so operator values agree to rounding.  Other grids: nothing to tune, GPE_OK.  Allocates scratch
 * of two plan vectors and one solver level per grid; synchronises.  Not
 * thread-safe with concurrent launches on the tuned shapes.
 *   - float32 square grids: the fused one-launch operator kernel against the
 *     two line kernels, for this grid and batch;
 * Errors: GPE_EINVAL (NULL plan, levels outside [1, 8]), GPE_ENOMEM, GPE_ECUDA. */
gpe_status gpe_plan_autotune(gpe_plan plan, int levels);

/* Text of the choices made by gpe_plan_autotune so far in this process
 * (NUL-terminated, truncated to buflen).  GPE_EINVAL if buf is NULL or buflen 0. */
gpe_status gpe_autotune_report(char* buf, size_t buflen);

/* Allocation-free Cayley step (the paper has no counterpart: this is a
 * packaging variant of gpe_feasible_step for callers that cannot call
 * cudaMalloc -- e.g. code running inside an allocator or memory-pool callback,
 * which must not re-enter the allocator, a loop whose device memory budget was
 * fixed up front, or a host framework that owns all device memory and passes
 * the library only its own buffers -- and so cannot create a plan).
 * Computes the same result as gpe_feasible_step(..., E_out = NULL) for
 * `nbatch` instances of `n_unknowns` values each: psi and hpsi are device
 * buffers in the layout above (prec = gpe_prec, is_complex as in the problem),
 * h_vol the cell volume, tau >= 0.  psi_out (device, same layout) must not
 * alias psi or hpsi.  stream is a cudaStream_t (NULL = legacy default stream);
 * the call is asynchronous.
 * Scratch: a fixed 512 KiB array in device memory, part of the library image,
 * held by every GPU that loads the library until the process exits.  Limits:
 * 1 <= nbatch <= 64 and nbatch * min(ceil(n_unknowns / 256), 512) <= 4096;
 * larger requests return GPE_EINVAL and do nothing.
 * The first call on each device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress and caches it with the
 * identity of the device's CUDA context; the first call after a
 * cudaDeviceReset (a new context) looks it up again.  Make that first call
 * before any stream capture.  Every call reuses the same array, so
 * calls whose work overlaps on the GPU (other streams, other threads) race;
 * serialise them.  The call allocates nothing. */
gpe_status gpe_feasible_step_noalloc(int prec, int is_complex, int64_t n_unknowns, int nbatch, double h_vol,
                                     const void* psi, const void* hpsi, double tau, void* psi_out,
                                     void* stream);

/* Instrumentation (the paper has no counterpart; used by the benchmark).
 * gpe_kernel_launches: kernels this process has launched through libgpe so far
 *   (a CUDA-graph launch counts each of its kernel nodes).
 * gpe_profile_enable(1): from now on record a pair of CUDA events on the
 *   launching stream around every kernel libgpe launches outside stream
 *   capture; gpe_rnewton_solve then runs without CUDA graphs so that every
 *   launch is recorded.  gpe_profile_enable(0) stops and discards the records.
 * gpe_profile_summary: synchronises the recorded events and writes a JSON
 *   object {"kernel-name": [launches, total_ms], ...} into buf (NUL
 *   terminated, truncated to buflen).  GPE_EINVAL if buf is NULL. */
int64_t gpe_kernel_launches(void);

/* Operator implementation on float32 square 2D Fourier grids (the paper has
 * no counterpart: an implementation choice that never changes the operator's
 * values beyond rounding order).  path 0: automatic -- the choice
 * gpe_plan_autotune measured for the grid and batch, else the fused kernel
 * for batches of at least 16 instances on grids up to 256^2; 1: always the
 * fused one-launch kernel;
 * 2: always the two line kernels.  Process-wide, for later launches; a
 * diagnostic and test knob.  Errors: GPE_EINVAL (path outside 0..2). */
gpe_status gpe_set_operator_path(int path);

/* Bounded device waits (the paper has no counterpart: failure handling).  The
 * persistent Algorithm 1 launch waits at grid barriers and the fused 2D
 * operator kernel's x-tasks wait for the y-tasks of their instance; each wait
 * polls at most a fixed number of times (2^22 barrier polls, 2^24 task polls,
 * about a second) and then gives up: gpe_rnewton_solve returns GPE_ETIMEOUT,
 * and so do gpe_energy and gpe_grad with energies requested (the outputs of
 * that call are not valid).  gpe_set_wait_limit(n), n > 0, replaces both
 * limits by n polls for every later launch in this process (a diagnostic
 * and test knob: a limit of 1 makes a wait give up almost at once); n = 0
 * restores the defaults.  Not thread-safe with concurrent launches.
 * Errors: GPE_EINVAL (n < 0). */
gpe_status gpe_set_wait_limit(int64_t polls);

/* Arithmetic peak of the current device, measured (the paper has no
 * counterpart: instrumentation for the roofline of the operator kernels).
 * kind 0: float32 fused multiply-add; 1: packed two-lane float32 multiply-add
 * (one instruction, two results); 2: float64 fused multiply-add.  Runs six
 * launches of independent multiply-add chains on every SM at full occupancy
 * on `stream` (a cudaStream_t, NULL = legacy default stream), times the last
 * five with CUDA events, synchronises, and writes the rate in TFLOP/s
 * (2 flops per multiply-add) to *tflops.  Allocates nothing.
 * Errors: GPE_EINVAL (kind, NULL tflops), GPE_ECUDA. */
gpe_status gpe_probe_peak(int kind, void* stream, double* tflops);
gpe_status gpe_profile_enable(int on);
gpe_status gpe_profile_summary(char* buf, int buflen);

#ifdef __cplusplus
}
#endif
#endif /* GPE_H */
