// solver.cu -- gpe_rnewton_solve: Algorithm 3 (cascade) around Algorithm 2
// (regularized Newton with the trust-region ratio test) and Algorithm 1
// (feasible gradient with BB steps and the nonmonotone curvilinear search).
//
// Every numerical step runs on the device: an Algorithm 1 iteration is the
// operator passes with the Cayley step formed while loading the first pass and
// the step-size logic executed by the last CTA of the final pass (alg1_control).
// The host only queues fixed chunks of iterations (captured once in a CUDA
// graph per level and objective) and reads the small control block between
// chunks to learn whether the run has stopped.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <chrono>
#include <memory>
#include <type_traits>
#include <vector>
#include "gpe_internal.h"

namespace gpe {

template <typename T>
struct Level {
  GridHost g;
  GridDev<T> d;
  Scratch sc;
  long long M = 0;
  size_t bytes = 0;
  void* acc = nullptr;
  void* xs[3] = {nullptr, nullptr, nullptr};
  void* gs[3] = {nullptr, nullptr, nullptr};
  void* xk = nullptr;
  void* gk = nullptr;
  void** d_xs = nullptr;
  void** d_gs = nullptr;
  Alg1Ctl* ctl = nullptr;
  RNCtl* rn = nullptr;
  Alg1Ctl* h_ctl = nullptr;
  RNCtl* h_rn = nullptr;
  cudaGraphExec_t chunk_exec[3] = {nullptr, nullptr, nullptr};   // objective F, W, W difference form
  size_t chunk_nodes[3] = {0, 0, 0};
  int chunk_len = 0;
  // persistent Algorithm 1 launch (spectral grids): barrier words, error flag,
  // launch shape per objective (grid 0 = not available)
  unsigned int* bar = nullptr;
  int* err = nullptr;
  int* h_err = nullptr;
  int p_grid[2] = {-1, -1};
  size_t p_smem[2] = {0, 0};
  float* d_omega = nullptr;   // Omega as float32 for the cluster engine

  gpe_status create(const GridHost& gh) {
    g = gh;
    M = g.M;
    bytes = sizeof(T) * (g.is_complex ? 2 : 1) * M;
    gpe_status s = d.create(g);
    if (s != GPE_OK) return s;
    s = sc.create(d.max_blocks, 1);
    if (s != GPE_OK) return s;
    GPE_CUDA(cudaMalloc(&acc, bytes));
    for (int i = 0; i < 3; ++i) {
      GPE_CUDA(cudaMalloc(&xs[i], bytes));
      GPE_CUDA(cudaMalloc(&gs[i], bytes));
    }
    GPE_CUDA(cudaMalloc(&xk, bytes));
    GPE_CUDA(cudaMalloc(&gk, bytes));
    GPE_CUDA(cudaMalloc(&d_xs, sizeof(void*) * 3));
    GPE_CUDA(cudaMalloc(&d_gs, sizeof(void*) * 3));
    GPE_CUDA(cudaMemcpy(d_xs, xs, sizeof(void*) * 3, cudaMemcpyHostToDevice));
    GPE_CUDA(cudaMemcpy(d_gs, gs, sizeof(void*) * 3, cudaMemcpyHostToDevice));
    GPE_CUDA(cudaMalloc(&ctl, sizeof(Alg1Ctl)));
    GPE_CUDA(cudaMalloc(&rn, sizeof(RNCtl)));
    GPE_CUDA(cudaMalloc(&bar, 2 * sizeof(unsigned int)));
    {
      const float om = (float)g.omega;
      GPE_CUDA(cudaMalloc(&d_omega, sizeof(float)));
      GPE_CUDA(cudaMemcpy(d_omega, &om, sizeof(float), cudaMemcpyHostToDevice));
    }
    GPE_CUDA(cudaMalloc(&err, sizeof(int)));
    GPE_CUDA(cudaMallocHost(&h_err, sizeof(int)));
    GPE_CUDA(cudaMallocHost(&h_ctl, sizeof(Alg1Ctl)));
    GPE_CUDA(cudaMallocHost(&h_rn, sizeof(RNCtl)));
    memset(h_ctl, 0, sizeof(Alg1Ctl));
    memset(h_rn, 0, sizeof(RNCtl));
    return GPE_OK;
  }
  void destroy() {
    for (int i = 0; i < 3; ++i)
      if (chunk_exec[i]) cudaGraphExecDestroy(chunk_exec[i]);
    d.destroy();
    sc.destroy();
    cudaFree(acc);
    for (int i = 0; i < 3; ++i) {
      cudaFree(xs[i]);
      cudaFree(gs[i]);
    }
    cudaFree(xk);
    cudaFree(gk);
    cudaFree(d_xs);
    cudaFree(d_gs);
    cudaFree(ctl);
    cudaFree(rn);
    cudaFree(bar);
    cudaFree(err);
    cudaFree(d_omega);
    cudaFreeHost(h_err);
    cudaFreeHost(h_ctl);
    cudaFreeHost(h_rn);
  }
  PassData<T> solver_data(int objective) const {
    PassData<T> D{};
    D.xs = d_xs;
    D.gs = d_gs;
    D.ctl = ctl;
    D.use_slots = 1;
    D.V = d.V;
    D.lin_scale = 2.0;
    D.base = objective >= 1 ? xk : nullptr;   // W: X^k; difference form: X^k (and gk = P_k)
    D.gk = objective == 2 ? gk : nullptr;
    D.partials = sc.partials;
    D.results = sc.results;
    D.ticket = sc.ticket;
    D.nq = NQ;
    D.control = 1;
    return D;
  }
};

// GPE_TRACE=1 in the environment prints one line per regularized Newton
// iteration (and per Algorithm 1 run) to stderr.
static bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("GPE_TRACE");
    on = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return on == 1;
}

static unsigned long long* g_pdbg = nullptr;
static unsigned long long* g_pdbg_h = nullptr;
static const int PDBG_N = 256;

unsigned long long* persist_debug_buffer(int* n) {
  const char* e = getenv("GPE_PERSIST_TRACE");
  *n = 0;
  if (!(e && e[0] && e[0] != '0')) return nullptr;
  if (!g_pdbg) {
    if (cudaMalloc(&g_pdbg, sizeof(unsigned long long) * 4 * PDBG_N) != cudaSuccess) return nullptr;
    if (cudaMallocHost(&g_pdbg_h, sizeof(unsigned long long) * 4 * PDBG_N) != cudaSuccess) return nullptr;
  }
  cudaMemset(g_pdbg, 0, sizeof(unsigned long long) * 4 * PDBG_N);
  *n = PDBG_N;
  return g_pdbg;
}

void persist_debug_report(cudaStream_t st, long long M, int f64) {
  if (!g_pdbg) return;
  cudaMemcpyAsync(g_pdbg_h, g_pdbg, sizeof(unsigned long long) * 4 * PDBG_N, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double s[3] = {0, 0, 0};
  int n = 0;
  for (int i = 0; i < PDBG_N; ++i) {
    const unsigned long long* t = g_pdbg_h + 4 * i;
    if (!t[0] || !t[3]) break;
    s[0] += (double)(t[1] - t[0]);
    s[1] += (double)(t[2] - t[1]);
    s[2] += (double)(t[3] - t[2]);
    ++n;
  }
  if (n)
    fprintf(stderr, "[gpe] persist %s M=%lld loops=%d  pass0 %.2f us  pass1 %.2f us  fold+control %.2f us\n",
            f64 ? "f64" : "f32", M, n, s[0] / n / 1e3, s[1] / n / 1e3, s[2] / n / 1e3);
}

static void cluster_debug_report(cudaStream_t st, int nloops) {
  if (!g_pdbg) return;
  cudaMemcpyAsync(g_pdbg_h, g_pdbg, sizeof(unsigned long long) * 4 * PDBG_N, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  // stamp slots in time order (the kernel's slot numbers)
  static const int order[12] = {0, 1, 2, 3, 4, 5, 8, 9, 6, 10, 11, 7};
  // line passes: x, barrier, y, barrier (shared-memory stages) or barrier, y,
  // barrier, x (register line FFTs)
  static const char* name[11] = {"step", "lines1", "lines2", "lines3", "lines4", "points", "block-sum", "push",
                                 "sync", "fold", "ctl"};
  double s[11] = {0};
  int n = 0;
  for (int i = 0; i < nloops; ++i) {
    const unsigned long long* t = g_pdbg_h + 16 * i;
    if (!t[0] || !t[7]) break;
    for (int k = 0; k < 11; ++k) s[k] += (double)(t[order[k + 1]] - t[order[k]]);
    ++n;
  }
  if (n) {
    fprintf(stderr, "[gpe] cluster phases (us, %d loops):", n);
    for (int k = 0; k < 11; ++k) fprintf(stderr, " %s %.2f", name[k], s[k] / n / 1e3);
    fprintf(stderr, "\n");
  }
}

struct RunStats {
  int iters = 0, nfe = 0, status = 0;
  double F = 0, res = 0, theta = 0;
};

struct SolveParams {
  int k_init, k_sub, max_outer, max_iter, method, chunk, use_graphs, persistent, cluster, search;
  int refine = 0;      // gpe_solve_batch: float64 refinement after the float32 bulk
  double eps0, delta_stop, res_tol_X, delta0, switch_rel, alpha_hat, eta;
};

// Options of the line search: search 0 or 1, alpha_hat > 0, 0 <= eta < 1.
static bool search_opts_ok(const gpe_solve_opts& o) {
  return (o.search == 0 || o.search == 1) && o.alpha_hat > 0.0 && o.alpha_hat < 1e20 && o.eta >= 0.0 &&
         o.eta < 1.0;
}

// Line search of an Algorithm 1 run: Eq. NMLS-Armijo with weight eta and BB
// first steps (search 0), or the monotone Armijo search of the Remark after
// Theorem 3.4 (search 1: tau = alpha_hat 2^-m, at most 60 halvings).
static void set_search(Alg1Ctl& c, const SolveParams& P) {
  c.eta = P.eta;
  if (P.search == 1) {
    c.monotone = 1;
    c.alpha_hat = P.alpha_hat;
    c.delta_bt = 0.5;
    c.max_bt = 60;
  }
}

template <typename T>
static gpe_status read_ctl(Level<T>& L, cudaStream_t st) {
  GPE_CUDA(cudaMemcpyAsync(L.h_ctl, L.ctl, sizeof(Alg1Ctl), cudaMemcpyDeviceToHost, st));
  GPE_CUDA(cudaStreamSynchronize(st));
  return GPE_OK;
}

// Epilogue of an Algorithm 1 objective: 0 F, 1 W^(k), 2 W^(k) in difference form.
static int objective_epi(int objective) { return objective == 0 ? EPI_F : (objective == 1 ? EPI_W : EPI_WS); }

// Queue `n` Algorithm 1 iterations (each: Cayley step formed on load, the
// operator passes, control in the last CTA).
template <typename T>
static gpe_status queue_iters(Level<T>& L, int objective, int n, cudaStream_t st) {
  const PassData<T> D = L.solver_data(objective);
  const int epi = objective_epi(objective);
  const long long n_all = L.M * L.g.nbatch;   // elements (complex or real)
  for (int i = 0; i < n; ++i) {
    gpe_status s;
    if (objective == 2) {
      // difference form: the step needs X^k, so it runs as its own kernel
      s = launch_step<T>(D.xs, D.gs, D.ctl, n_all, L.g.is_complex, st, L.xk);
      if (s != GPE_OK) return s;
      s = apply_op<T>(L.g, L.d, D, epi, L.acc, false, st);
    } else {
      s = apply_op<T>(L.g, L.d, D, epi, L.acc, true, st);
    }
    if (s != GPE_OK) return s;
  }
  return GPE_OK;
}

template <typename T>
static gpe_status run_chunk(Level<T>& L, int objective, const SolveParams& P, cudaStream_t st) {
  if (!P.use_graphs || prof_enabled()) return queue_iters<T>(L, objective, P.chunk, st);
  cudaGraphExec_t& ex = L.chunk_exec[objective];
  if (!ex || L.chunk_len != P.chunk) {
    if (ex) {
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
    cudaGraph_t graph;
    GPE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    gpe_status s = queue_iters<T>(L, objective, P.chunk, st);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != GPE_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    L.chunk_nodes[objective] = nn;
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    L.chunk_len = P.chunk;
  }
  GPE_CUDA(cudaGraphLaunch(ex, st));
  instr_count((long long)L.chunk_nodes[objective]);
  return GPE_OK;
}

// Algorithm 1 on objective F (0) or W^(k) (1) from the point in xs[first_slot]
// (unit norm).  Returns the state of the control block in L.h_ctl.
template <typename T>
static gpe_status alg1_run(Level<T>& L, int objective, int first_slot, int max_iter, double res_tol, double eps0,
                           double delta, const SolveParams& P, cudaStream_t st, RunStats& out, double res_rel = 0.0,
                           double theta_hint = 0.0, int stall_iters = 0, double theta_ref = 0.0) {
  Alg1Ctl& c = *L.h_ctl;
  memset(&c, 0, sizeof(c));
  c.alpha = L.g.beta / (2.0 * L.g.hvol);
  c.delta = delta;
  c.rho1 = 1e-4;
  c.eta = 0.85;
  c.delta_bt = 0.1;
  c.eps0 = eps0;
  c.res_tol = res_tol;
  c.res_rel = res_rel;
  c.tau0 = 1e-3;
  c.renorm_tol = 1e-14;
  c.max_bt = 10;
  c.max_iter = max_iter;
  c.objective = objective;
  c.always_renorm = sizeof(T) == 4 ? 1 : 0;
  c.cur = 0;
  c.prev = 1;
  c.trial = first_slot;
  c.has_cur = 0;
  c.done = 0;
  c.phase = 0;
  c.theta_hint = theta_hint;
  c.stall_iters = stall_iters;
  if (objective == 2) {
    // difference form: the Cayley curve keeps ||X^k + D||, no rescaling
    c.always_renorm = 0;
    c.renorm_tol = 1e300;
    c.theta_ref = theta_ref;
  }
  set_search(c, P);
  GPE_CUDA(cudaMemcpyAsync(L.ctl, &c, sizeof(Alg1Ctl), cudaMemcpyHostToDevice, st));
  // first evaluation (no step)
  gpe_status s = apply_op<T>(L.g, L.d, L.solver_data(objective), objective_epi(objective), L.acc, false, st);
  if (s != GPE_OK) return s;
  // bounded: every queued iteration either accepts or backtracks (<= max_bt times)
  const long long max_launch = (long long)(max_iter + 1) * (c.max_bt + 1) + 1;
  long long launched = 0;
  s = read_ctl<T>(L, st);
  if (s != GPE_OK) return s;
  if (!L.h_ctl->done && P.persistent && objective < 2 && !prof_enabled()) {
    if (L.p_grid[objective] < 0) {
      s = persist_config<T>(L.g, L.d, objective == 1 ? EPI_W : EPI_F, &L.p_grid[objective], &L.p_smem[objective]);
      if (s != GPE_OK) return s;
    }
    if (L.p_grid[objective] > 0) {
      s = launch_alg1_persist<T>(L.g, L.d, L.solver_data(objective), L.acc, L.bar, L.err, (int)max_launch,
                                 objective == 1 ? EPI_W : EPI_F, L.p_grid[objective], L.p_smem[objective], st);
      if (s != GPE_OK) return s;
      GPE_CUDA(cudaMemcpyAsync(L.h_err, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
      persist_debug_report(st, L.M, sizeof(T) == 8);
      s = read_ctl<T>(L, st);
      if (s != GPE_OK) return s;
      if (*L.h_err) return fail(GPE_ETIMEOUT, "a grid barrier wait of the persistent Algorithm 1 launch expired");
      launched = max_launch;
    }
  }
  while (!L.h_ctl->done && launched < max_launch) {
    s = run_chunk<T>(L, objective, P, st);
    if (s != GPE_OK) return s;
    launched += P.chunk;
    s = read_ctl<T>(L, st);
    if (s != GPE_OK) return s;
  }
  out.iters = L.h_ctl->k;
  out.nfe = L.h_ctl->nfe;
  out.status = L.h_ctl->status;
  out.F = L.h_ctl->F_cur;
  out.res = L.h_ctl->res;
  out.theta = L.h_ctl->theta_c;
  if (trace_on())
    fprintf(stderr, "[gpe] alg1 %s M=%lld obj=%d iters=%d nfe=%d status=%d F=%.15g res=%.3e tau=%.3e th=%.10g\n",
            sizeof(T) == 8 ? "f64" : "f32", L.M, objective, out.iters, out.nfe, out.status, out.F, out.res,
            L.h_ctl->tau, out.theta);
  if (L.h_ctl->status == GPE_ENONFINITE) return fail(GPE_ENONFINITE, "non-finite energy during Algorithm 1");
  return GPE_OK;
}

// X in xs[slot] scaled to unit 2-norm.
template <typename T>
static gpe_status normalise_slot(Level<T>& L, int slot, cudaStream_t st) {
  gpe_status s = launch_moments<T>(L.xs[slot], nullptr, L.M, 1, L.g.is_complex, L.sc, st);
  if (s != GPE_OK) return s;
  s = launch_norm_coef(L.sc.results, 1, 1.0, L.sc.coef, st);
  if (s != GPE_OK) return s;
  return launch_axpby<T>(L.xs[slot], nullptr, L.sc.coef, 1, L.M, 1, L.xs[slot], L.g.is_complex, st);
}
template <typename T>
static gpe_status normalise_slot0(Level<T>& L, cudaStream_t st) {
  return normalise_slot<T>(L, 0, st);
}

struct LevelStats {
  int outer = 0, inner = 0, inner32 = 0, nfe = 0;
  double F = 0, res = 0, theta = 0;
  bool converged = false;
};

// Algorithm 2 on one level, starting from xs[0]; result in xk/gk.
// mode_f32: stop on the float32 criteria (relative residual or stagnation).
static gpe_status sub_run_cluster(Level<float>& Lf, const SolveParams& P, double thk, double delta, double sub_tol,
                                  cudaStream_t st, RunStats& out, bool* used);

template <typename T>
static gpe_status rn_run(Level<T>& L, const SolveParams& P, int k_init, bool stop_f32, cudaStream_t st,
                         LevelStats& ls, double theta_start, Level<float>* Lf32 = nullptr) {
  RunStats r;
  const double res_tol = P.res_tol_X;
  // warm start (Algorithm 1, <= k_init iterations; k_init = 0 is one evaluation)
  gpe_status s = alg1_run<T>(L, 0, 0, k_init, res_tol, P.eps0, 0.0, P, st, r, 0.0, theta_start);
  if (s != GPE_OK) return s;
  ls.inner += r.iters;
  ls.nfe += r.nfe;
  double Fk = r.F, resk = r.res, thk = r.theta;
  const int cur = L.h_ctl->cur;
  GPE_CUDA(cudaMemcpyAsync(L.xk, L.xs[cur], L.bytes, cudaMemcpyDeviceToDevice, st));
  GPE_CUDA(cudaMemcpyAsync(L.gk, L.gs[cur], L.bytes, cudaMemcpyDeviceToDevice, st));
  double delta = P.delta0;
  double best_res = resk;
  int stall = 0, rejects = 0;
  // GPE_TRACE: device time of each outer step's subproblem, ratio pass and
  // evaluation at the accepted point (events on the solver's stream)
  struct TraceEvents {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    TraceEvents() {
      if (trace_on())
        for (auto& x : e) cudaEventCreate(&x);
    }
    ~TraceEvents() {
      for (auto& x : e)
        if (x) cudaEventDestroy(x);
    }
  } trace_ev;
  cudaEvent_t* tev = trace_ev.e;
  for (int outer = 0; outer < P.max_outer; ++outer) {
    if (res_tol > 0.0 && resk <= res_tol) { ls.converged = true; break; }
    if (stop_f32 && resk <= P.switch_rel * fabs(thk)) break;
    // subproblem (Eq. tr-sub) by Algorithm 1 on W^(k) from X^k
    const double sub_tol = fmax(1e-2 * resk, 1e-14);
    if (tev[0]) cudaEventRecord(tev[0], st);
    int zc = 0;
    bool done32 = false;
    if constexpr (std::is_same<T, double>::value) {
      if (Lf32) {
        // float32 inner solve in difference form around the float64 outer iterate
        const long long nreal = L.M * (L.g.is_complex ? 2 : 1);
        s = launch_to_shifted_f32((const double*)L.xk, (const double*)L.gk, thk, (float*)Lf32->xk,
                                  (float*)Lf32->gk, nreal, st);
        if (s != GPE_OK) return s;
        s = sub_run_cluster(*Lf32, P, thk, delta, sub_tol, st, r, &done32);
        if (s != GPE_OK) return s;
        int dslot = 0;
        if (!done32 && L.g.disc != GPE_FD) {
          // grids the cluster does not hold: the same difference form with the
          // per-launch passes (D = 0 at the start)
          GPE_CUDA(cudaMemsetAsync(Lf32->xs[0], 0, Lf32->bytes, st));
          s = alg1_run<float>(*Lf32, 2, 0, P.k_sub, sub_tol, 0.0, delta, P, st, r, 0.0, 0.0, 0, thk);
          if (s != GPE_OK) return s;
          dslot = Lf32->h_ctl->cur;
          done32 = true;
        }
        if (done32) {
          s = launch_add_f32_to_f64((const double*)L.xk, (const float*)Lf32->xs[dslot], (double*)L.xs[1], nreal,
                                    st);
          if (s != GPE_OK) return s;
          // Z = X^k + D back on the unit sphere in float64 (D carries float32 rounding)
          s = normalise_slot<T>(L, 1, st);
          if (s != GPE_OK) return s;
          zc = 1;
          ls.inner32 += r.iters;
          ls.nfe += r.nfe;
        }
      }
    }
    if (!done32) {
      GPE_CUDA(cudaMemcpyAsync(L.xs[0], L.xk, L.bytes, cudaMemcpyDeviceToDevice, st));
      s = alg1_run<T>(L, 1, 0, P.k_sub, sub_tol, 0.0, delta, P, st, r, 0.0, thk);
      if (s != GPE_OK) return s;
      ls.inner += r.iters;
      ls.nfe += r.nfe;
      zc = L.h_ctl->cur;
    }
    if (tev[1]) cudaEventRecord(tev[1], st);
    // ratio test (Eq. TR-ratio) and delta update (Eq. tau-up)
    RNCtl& rc = *L.h_rn;
    memset(&rc, 0, sizeof(rc));
    rc.alpha = L.g.beta / (2.0 * L.g.hvol);
    rc.delta = delta;
    rc.eta1 = 0.01;
    rc.eta2 = 0.9;
    rc.gamma1 = 2.0;
    rc.gamma2 = 4.0;
    rc.delta_min = 1e-12;
    rc.delta_max = 1e12;
    rc.F_k = Fk;
    GPE_CUDA(cudaMemcpyAsync(L.rn, &rc, sizeof(RNCtl), cudaMemcpyHostToDevice, st));
    PassData<T> D{};
    D.x = L.xs[zc];
    D.xsub = L.xk;
    D.base = L.xk;
    D.gk = L.gk;
    D.rn = L.rn;
    D.V = L.d.V;
    D.lin_scale = 2.0;
    D.partials = L.sc.partials;
    D.results = L.sc.results;
    D.ticket = L.sc.ticket;
    D.nq = NQ;
    D.control = 2;
    s = apply_op<T>(L.g, L.d, D, EPI_RATIO, L.acc, false, st);
    if (s != GPE_OK) return s;
    if (tev[2]) cudaEventRecord(tev[2], st);
    GPE_CUDA(cudaMemcpyAsync(L.h_rn, L.rn, sizeof(RNCtl), cudaMemcpyDeviceToHost, st));
    GPE_CUDA(cudaStreamSynchronize(st));
    ls.nfe += 1;
    ls.outer += 1;
    const bool accepted = L.h_rn->accepted != 0;
    const double dmax = L.h_rn->dmax;
    delta = L.h_rn->delta;
    if (trace_on())
      fprintf(stderr, "[gpe] rn %s M=%lld outer=%d res=%.3e sub_tol=%.3e inner=%d rho=%.6f ared=%.6e pred=%.6e delta=%.3e dmax=%.3e acc=%d\n",
              sizeof(T) == 8 ? "f64" : "f32", L.M, outer, resk, sub_tol, r.iters, L.h_rn->rho, L.h_rn->ared,
              L.h_rn->pred, delta, dmax, (int)accepted);
    if (!isfinite(L.h_rn->rho)) return fail(GPE_ENONFINITE, "non-finite ratio in the regularized Newton step");
    if (accepted) {
      rejects = 0;
      // gradient at the accepted point (Eq. update-X): one evaluation
      s = alg1_run<T>(L, 0, zc, 0, 0.0, 0.0, 0.0, P, st, r, 0.0, thk);
      if (s != GPE_OK) return s;
      ls.nfe += r.nfe;
      const int c2 = L.h_ctl->cur;
      GPE_CUDA(cudaMemcpyAsync(L.xk, L.xs[c2], L.bytes, cudaMemcpyDeviceToDevice, st));
      GPE_CUDA(cudaMemcpyAsync(L.gk, L.gs[c2], L.bytes, cudaMemcpyDeviceToDevice, st));
      Fk = r.F;
      resk = r.res;
      thk = r.theta;
      if (tev[3]) {
        cudaEventRecord(tev[3], st);
        cudaEventSynchronize(tev[3]);
        float t1 = 0, t2 = 0, t3 = 0;
        cudaEventElapsedTime(&t1, tev[0], tev[1]);
        cudaEventElapsedTime(&t2, tev[1], tev[2]);
        cudaEventElapsedTime(&t3, tev[2], tev[3]);
        fprintf(stderr, "[gpe] rn outer %d: subproblem %.1f us, ratio pass %.1f us, evaluation %.1f us\n", outer,
                1e3 * t1, 1e3 * t2, 1e3 * t3);
      }
      if (!stop_f32 && dmax <= P.delta_stop) { ls.converged = true; break; }   // Eq. crit2
    } else {
      ++rejects;
    }
    if (stop_f32) {
      // float32 stagnation: three accepted steps in a row without halving the
      // best residual, or four rejections in a row
      if (accepted) {
        if (resk < 0.5 * best_res) {
          best_res = resk;
          stall = 0;
        } else if (++stall >= 3) {
          break;
        }
      }
      if (rejects >= 4) break;
    }
  }
  // the last allowed outer step may itself have reached the tolerance
  if (res_tol > 0.0 && resk <= res_tol) ls.converged = true;
  ls.F = Fk;
  ls.res = resk;
  ls.theta = thk;
  return GPE_OK;
}

// Algorithm 1 only (method = 1, and the float32 bulk of the mixed schedule):
// result in xk/gk.  In float32 the run stops at the relative residual
// switch_rel or when the residual stops improving (the float32 floor).
template <typename T>
static gpe_status fg_run(Level<T>& L, const SolveParams& P, bool stop_f32, cudaStream_t st, LevelStats& ls,
                         double theta_start) {
  RunStats r;
  const double eps0 = stop_f32 ? 0.0 : P.eps0;
  gpe_status s = alg1_run<T>(L, 0, 0, P.max_iter, P.res_tol_X, eps0, 0.0, P, st, r, stop_f32 ? P.switch_rel : 0.0,
                             theta_start, stop_f32 ? 40 : 0);
  if (s != GPE_OK) return s;
  const int cur = L.h_ctl->cur;
  GPE_CUDA(cudaMemcpyAsync(L.xk, L.xs[cur], L.bytes, cudaMemcpyDeviceToDevice, st));
  GPE_CUDA(cudaMemcpyAsync(L.gk, L.gs[cur], L.bytes, cudaMemcpyDeviceToDevice, st));
  ls.inner += r.iters;
  ls.nfe += r.nfe;
  ls.F = r.F;
  ls.res = r.res;
  ls.theta = r.theta;
  ls.converged = (r.status == 0);
  return GPE_OK;
}

// Control block of a float32 Algorithm 1 run on F in the cluster engine
// (readings S3-S5: constants; two slots; the float32 floor ends the run).
static void init_cluster_ctl(Alg1Ctl& c, double alpha, const SolveParams& P, bool stop_f32, double theta_start) {
  memset(&c, 0, sizeof(c));
  c.alpha = alpha;
  c.rho1 = 1e-4;
  c.eta = 0.85;
  c.delta_bt = 0.1;
  c.eps0 = stop_f32 ? 0.0 : P.eps0;
  c.res_tol = P.res_tol_X;
  c.res_rel = stop_f32 ? P.switch_rel : 0.0;
  c.tau0 = 1e-3;
  c.renorm_tol = 1e-14;
  c.max_bt = 10;
  c.max_iter = P.max_iter;
  c.objective = 0;
  c.always_renorm = 1;
  c.cur = 1;
  c.trial = 0;
  c.theta_hint = theta_start;
  c.stall_iters = stop_f32 ? 40 : 0;
  c.two_slots = 1;
  set_search(c, P);
}

// Algorithm 1 on F in float32 by the cluster engine (2D Fourier grids whose
// state fits in one cluster's shared memory); the start point is xs[0].
// Returns false in *used if the grid is not eligible.
static gpe_status fg_run_cluster(Level<float>& L, const SolveParams& P, bool stop_f32, cudaStream_t st,
                                 LevelStats& ls, double theta_start, bool* used) {
  *used = false;
  const GridHost& g = L.g;
  if (!P.cluster || g.disc != GPE_FOURIER || g.dim != 2 || prof_enabled()) return GPE_OK;
  int cs, lch, P0, P1;
  size_t smem;
  unsigned int vb, vp;
  if (!cluster_shape(g.ext[0], g.ext[1], g.is_complex, 5, &cs, &lch, &P0, &P1, &smem, &vb, &vp)) return GPE_OK;
  const int share_kb = tuned_share_kb(g.ext[0], g.ext[1], g.is_complex);   // single solve: 4 KiB or the measured choice
  cluster_shape(g.ext[0], g.ext[1], g.is_complex, 5, &cs, &lch, &P0, &P1, &smem, &vb, &vp, (size_t)share_kb * 1024);
  Alg1Ctl& c = *L.h_ctl;
  init_cluster_ctl(c, g.beta / (2.0 * g.hvol), P, stop_f32, theta_start);
  GPE_CUDA(cudaMemcpyAsync(L.ctl, &c, sizeof(Alg1Ctl), cudaMemcpyHostToDevice, st));
  ClusterArgs A{};
  A.n0 = g.ext[0];
  A.n1 = g.ext[1];
  A.ninst = 1;
  A.max_loops = (P.max_iter + 1) * (c.max_bt + 1) + 1;
  A.dlam0 = (float)(2.0 * M_PI / (g.hi[0] - g.lo[0]));
  A.dlam1 = (float)(2.0 * M_PI / (g.hi[1] - g.lo[1]));
  A.V = L.d.V;
  A.vstride = 0;
  A.xn = L.d.coord[0];
  A.yn = L.d.coord[1];
  A.omega = g.omega != 0.0 ? L.d_omega : nullptr;
  A.tw0 = L.d.tw[0];
  A.tw1 = L.d.tw[1];
  A.x = L.xs[0];
  A.g = L.gs[0];
  A.ctl = L.ctl;
  A.results = L.sc.results;
  A.dbg = persist_debug_buffer(&A.dbg_n);
  if (A.dbg) A.dbg_n = A.dbg_n / 4;     // 16 stamp slots per loop in a buffer of 4 x n
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (trace_on()) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  A.share_kb = share_kb;
  gpe_status s = launch_cluster_alg1(A, g.is_complex, st);
  if (s != GPE_OK) return s;
  if (A.dbg) cluster_debug_report(st, A.dbg_n);
  float ms = 0.f;
  if (e0) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  GPE_CUDA(cudaMemcpyAsync(L.xk, L.xs[0], L.bytes, cudaMemcpyDeviceToDevice, st));
  GPE_CUDA(cudaMemcpyAsync(L.gk, L.gs[0], L.bytes, cudaMemcpyDeviceToDevice, st));
  s = read_ctl<float>(L, st);
  if (s != GPE_OK) return s;
  const Alg1Ctl& h = *L.h_ctl;
  if (trace_on())
    fprintf(stderr, "[gpe] cluster f32 M=%lld cs=%d iters=%d nfe=%d status=%d F=%.15g res=%.3e  %.3f ms (%.2f us/trial)\n",
            L.M, cs, h.k, h.nfe, h.status, h.F_cur, h.res, ms, 1e3 * ms / (h.nfe > 0 ? h.nfe : 1));
  if (h.status == GPE_ENONFINITE) return fail(GPE_ENONFINITE, "non-finite energy during Algorithm 1");
  ls.inner += h.k;
  ls.nfe += h.nfe;
  ls.F = h.F_cur;
  ls.res = h.res;
  ls.theta = h.theta_c;
  ls.converged = (h.status == 0);
  *used = true;
  return GPE_OK;
}

// The regularized Newton subproblem in float32 by the cluster engine, shifted
// difference form: X^k and P_k = G_k - theta_k X^k already in Lf.xk / Lf.gk
// (float32).  Result D in Lf.xs[0].  *used = false if not eligible.
static gpe_status sub_run_cluster(Level<float>& Lf, const SolveParams& P, double thk, double delta, double sub_tol,
                                  cudaStream_t st, RunStats& out, bool* used) {
  *used = false;
  const GridHost& g = Lf.g;
  if (!P.cluster || g.disc != GPE_FOURIER || g.dim != 2 || prof_enabled()) return GPE_OK;
  int cs, lch, P0, P1;
  size_t smem;
  unsigned int vb, vp;
  if (!cluster_shape(g.ext[0], g.ext[1], g.is_complex, 7, &cs, &lch, &P0, &P1, &smem, &vb, &vp)) return GPE_OK;
  Alg1Ctl& c = *Lf.h_ctl;
  memset(&c, 0, sizeof(c));
  c.alpha = g.beta / (2.0 * g.hvol);
  c.delta = delta;
  c.theta_ref = thk;
  c.rho1 = 1e-4;
  c.eta = 0.85;
  c.delta_bt = 0.1;
  c.eps0 = 0.0;
  c.res_tol = sub_tol;
  c.tau0 = 1e-3;
  c.renorm_tol = 1e300;    // the Cayley step keeps the norm; no rescaling in difference form
  c.max_bt = 10;
  c.max_iter = P.k_sub;
  c.objective = 1;
  c.always_renorm = 0;
  c.cur = 1;
  c.trial = 0;
  c.theta_hint = 0.0;
  c.two_slots = 1;
  c.stall_iters = 0;       // sub_tol is relative to ||P_k||: above the float32 floor
  set_search(c, P);
  GPE_CUDA(cudaMemcpyAsync(Lf.ctl, &c, sizeof(Alg1Ctl), cudaMemcpyHostToDevice, st));
  ClusterArgs A{};
  A.n0 = g.ext[0];
  A.n1 = g.ext[1];
  A.ninst = 1;
  A.max_loops = (P.k_sub + 1) * (c.max_bt + 1) + 1;
  A.dlam0 = (float)(2.0 * M_PI / (g.hi[0] - g.lo[0]));
  A.dlam1 = (float)(2.0 * M_PI / (g.hi[1] - g.lo[1]));
  A.V = Lf.d.V;
  A.vstride = 0;
  A.xn = Lf.d.coord[0];
  A.yn = Lf.d.coord[1];
  A.omega = g.omega != 0.0 ? Lf.d_omega : nullptr;
  A.tw0 = Lf.d.tw[0];
  A.tw1 = Lf.d.tw[1];
  A.x = Lf.xs[0];
  A.g = Lf.gs[0];
  A.ctl = Lf.ctl;
  A.results = Lf.sc.results;
  A.shifted = 1;
  A.xk = Lf.xk;
  A.pk = Lf.gk;
  A.share_kb = tuned_share_kb(g.ext[0], g.ext[1], g.is_complex);   // single solve: 4 KiB or the measured choice
  gpe_status s = launch_cluster_alg1(A, g.is_complex, st);
  if (s != GPE_OK) return s;
  s = read_ctl<float>(Lf, st);
  if (s != GPE_OK) return s;
  const Alg1Ctl& h = *Lf.h_ctl;
  if (h.status == GPE_ENONFINITE) return fail(GPE_ENONFINITE, "non-finite model value in the subproblem");
  out.iters = h.k;
  out.nfe = h.nfe;
  out.status = h.status;
  out.F = h.F_cur;
  out.res = h.res;
  out.theta = h.theta_c;
  *used = true;
  return GPE_OK;
}


template <typename Ti, typename To>
static gpe_status convert_vec(const void* in, void* out, long long n_real, double scale, cudaStream_t st) {
  return launch_convert<Ti, To>((const Ti*)in, (To*)out, n_real, scale, st);
}

// Cache of solver levels kept in the plan between calls.
struct SolverCache {
  int levels = 0, mode = -1;
  std::vector<std::unique_ptr<Level<float>>> lf;
  std::vector<std::unique_ptr<Level<double>>> ld;
  std::unique_ptr<Level<double>> fine64;   // float64 refinement/report level (modes 1, 2)
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  void* inj = nullptr;                     // injected initial guess (plan precision, coarse grid)
  ~SolverCache() {
    for (auto& l : lf) l->destroy();
    for (auto& l : ld) l->destroy();
    if (fine64) fine64->destroy();
    if (st) cudaStreamDestroy(st);
    if (ev) cudaEventDestroy(ev);
    cudaFree(inj);
  }
};

void destroy_solver_cache(void* p) { delete static_cast<SolverCache*>(p); }

template <typename T>
static gpe_status make_levels(const GridHost& fine, int levels, std::vector<std::unique_ptr<Level<T>>>& out) {
  out.clear();
  for (int l = 0; l < levels; ++l) {
    GridHost g = grid_coarsen(fine, levels - 1 - l);
    g.nbatch = 1;
    std::unique_ptr<Level<T>> L(new Level<T>());
    gpe_status s = L->create(g);
    if (s != GPE_OK) {
      L->destroy();
      return s;
    }
    out.push_back(std::move(L));
  }
  return GPE_OK;
}

// Initial guess (plan precision, finest grid) -> xs[0] of the coarsest level (X units, unit norm).
template <typename Tp, typename T>
static gpe_status load_initial(gpe_plan plan, SolverCache& C, Level<T>& L0, const void* psi, bool inject) {
  const long long nreal = L0.M * (L0.g.is_complex ? 2 : 1);
  const void* src = psi;
  if (inject) {
    gpe_status s = launch_inject<Tp>(plan->g, L0.g, psi, C.inj, C.st);
    if (s != GPE_OK) return s;
    src = C.inj;
  }
  gpe_status s = convert_vec<Tp, T>(src, L0.xs[0], nreal, sqrt(L0.g.hvol), C.st);
  if (s != GPE_OK) return s;
  return normalise_slot0<T>(L0, C.st);
}

template <typename T>
static gpe_status prolong_into(Level<T>& Lc, Level<T>& Lf, cudaStream_t st) {
  gpe_status s = launch_prolong<T>(Lc.g, Lf.g, Lc.d, Lf.d, Lc.xk, Lf.xs[0], Lf.acc, Lf.gs[0], st);
  if (s != GPE_OK) return s;
  return normalise_slot0<T>(Lf, st);
}

template <typename T>
static gpe_status solve_levels(std::vector<std::unique_ptr<Level<T>>>& lv, const SolveParams& P, bool f32,
                               cudaStream_t st, LevelStats& fine_stats, int& nfe_total) {
  double theta = 0.0;   // theta of the previous level: a nearby value for the first evaluation
  for (size_t l = 0; l < lv.size(); ++l) {
    if (l > 0) {
      gpe_status s = prolong_into<T>(*lv[l - 1], *lv[l], st);
      if (s != GPE_OK) return s;
    }
    LevelStats ls;
    // float32 bulk of the mixed schedule: Algorithm 1 down to the float32
    // floor on every level (the regularized Newton steps run in float64)
    gpe_status s = GPE_OK;
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (P.method == 1 || f32) {
        s = fg_run_cluster(*lv[l], P, f32, st, ls, theta, &done);
        if (s != GPE_OK) return s;
      }
    }
    if (!done)
      s = (P.method == 1 || f32) ? fg_run<T>(*lv[l], P, f32, st, ls, theta)
                                 : rn_run<T>(*lv[l], P, P.k_init, f32, st, ls, theta);
    if (s != GPE_OK) return s;
    theta = ls.theta;
    nfe_total += ls.nfe;
    if (l + 1 == lv.size()) fine_stats = ls;
  }
  return GPE_OK;
}

// Mixed schedule (mode 1), level by level of the cascade: float32 Algorithm 1
// from the prolonged state to the float32 floor; then, on the finest level and
// on any level where the float32 run stopped short of switch_rel (stagnation,
// as in rotating problems), Algorithm 2 with float64 outer quantities and
// float32 subproblems in difference form.  A level that ended in float64 is
// prolonged in float64.  Result in C.ld.back()->xk.
static gpe_status solve_mixed(SolverCache& C, const SolveParams& P, cudaStream_t st, LevelStats& fs, int& nfe,
                              gpe_solve_report& rep) {
  double theta = 0.0;
  bool prev_double = false;
  double ms32 = 0.0, ms64 = 0.0;
  for (size_t l = 0; l < C.lf.size(); ++l) {
    Level<float>& Lf = *C.lf[l];
    Level<double>& Ld = *C.ld[l];
    const long long nreal = Lf.M * (Lf.g.is_complex ? 2 : 1);
    const bool fine = l + 1 == C.lf.size();
    gpe_status s = GPE_OK;
    auto t0 = std::chrono::steady_clock::now();
    if (l > 0) {
      if (prev_double) {
        s = prolong_into<double>(*C.ld[l - 1], Ld, st);
        if (s == GPE_OK) s = convert_vec<double, float>(Ld.xs[0], Lf.xs[0], nreal, 1.0, st);
        if (s == GPE_OK) s = normalise_slot0<float>(Lf, st);
      } else {
        s = prolong_into<float>(*C.lf[l - 1], Lf, st);
      }
      if (s != GPE_OK) return s;
    }
    LevelStats ls;
    bool done = false;
    s = fg_run_cluster(Lf, P, true, st, ls, theta, &done);
    if (s != GPE_OK) return s;
    if (!done) s = fg_run<float>(Lf, P, true, st, ls, theta);
    if (s != GPE_OK) return s;
    nfe += ls.nfe;
    theta = ls.theta;
    GPE_CUDA(cudaStreamSynchronize(st));
    auto t1 = std::chrono::steady_clock::now();
    ms32 += std::chrono::duration<double, std::milli>(t1 - t0).count();
    if (fine) {
      rep.inner_f32 = ls.inner;
      rep.outer_f32 = 0;
    }
    const bool at_floor = ls.res <= P.switch_rel * fabs(ls.theta);
    prev_double = false;
    if (!fine && at_floor) continue;
    if (P.method == 1 && !fine) continue;
    s = convert_vec<float, double>(Lf.xk, Ld.xs[0], nreal, 1.0, st);
    if (s == GPE_OK) s = normalise_slot0<double>(Ld, st);
    if (s != GPE_OK) return s;
    LevelStats l2;
    s = rn_run<double>(Ld, P, 0, false, st, l2, theta, &Lf);
    if (s != GPE_OK) return s;
    nfe += l2.nfe;
    theta = l2.theta;
    prev_double = true;
    GPE_CUDA(cudaStreamSynchronize(st));
    ms64 += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    if (fine) {
      fs = l2;
      rep.outer_f64 = l2.outer;
      rep.inner_f64 = l2.inner;
      rep.inner_f32 += l2.inner32;
    }
  }
  rep.ms_f32 = ms32;
  rep.ms_f64 = ms64;
  return GPE_OK;
}

template <typename Tp>
static gpe_status solve_impl(gpe_plan plan, void* psi, const gpe_solve_opts& o, gpe_solve_report& rep) {
  auto t0 = std::chrono::steady_clock::now();
  SolverCache*& C = reinterpret_cast<SolverCache*&>(plan->solver_cache);
  if (C && (C->levels != o.levels || C->mode != o.mode)) {
    cudaStreamSynchronize(C->st);
    delete C;
    C = nullptr;
  }
  if (!C) {
    C = new SolverCache();
    C->levels = o.levels;
    C->mode = o.mode;
    GPE_CUDA(cudaStreamCreateWithFlags(&C->st, cudaStreamNonBlocking));
    GPE_CUDA(cudaEventCreateWithFlags(&C->ev, cudaEventDisableTiming));
    gpe_status s = GPE_OK;
    if (o.mode != 2) s = make_levels<double>(plan->g, o.levels, C->ld);
    if (s == GPE_OK && o.mode != 0) s = make_levels<float>(plan->g, o.levels, C->lf);
    if (s == GPE_OK && o.mode == 2) {
      GridHost g = plan->g;
      g.nbatch = 1;
      C->fine64.reset(new Level<double>());
      s = C->fine64->create(g);
    }
    if (s == GPE_OK) {
      cudaError_t e = cudaMalloc(&C->inj, elem_size(plan->prec, plan->g.is_complex) * plan->g.M);
      if (e != cudaSuccess) s = cuda_fail(e, "cudaMalloc(injection)");
    }
    if (s != GPE_OK) {
      delete C;
      C = nullptr;
      return s;
    }
  }
  cudaStream_t st = C->st;
  // order after the caller's stream
  GPE_CUDA(cudaEventRecord(C->ev, plan->stream));
  GPE_CUDA(cudaStreamWaitEvent(st, C->ev, 0));

  SolveParams P;
  P.k_init = o.k_init;
  P.k_sub = o.k_sub;
  P.max_outer = o.max_outer;
  P.max_iter = o.max_iter;
  P.method = o.method;
  P.chunk = o.chunk;
  P.use_graphs = o.use_graphs;
  P.persistent = o.persistent;
  P.cluster = o.cluster;
  P.search = o.search;
  P.alpha_hat = o.alpha_hat;
  P.eta = o.eta;
  P.eps0 = o.eps0;
  P.delta_stop = o.delta_stop;
  P.res_tol_X = 2.0 * o.res_tol;     // ||A(X)X||_2 = 2 ||H psi - mu psi||_h
  P.delta0 = o.delta0;
  P.switch_rel = o.switch_rel;

  const bool inject = o.levels > 1;
  LevelStats fs;
  int nfe = 0;
  gpe_status s;
  Level<double>* fin = nullptr;
  if (o.mode == 0) {
    s = load_initial<Tp, double>(plan, *C, *C->ld[0], psi, inject);
    if (s != GPE_OK) return s;
    s = solve_levels<double>(C->ld, P, false, st, fs, nfe);
    if (s != GPE_OK) return s;
    fin = C->ld.back().get();
    rep.outer_f64 = fs.outer;
    rep.inner_f64 = fs.inner;
    GPE_CUDA(cudaStreamSynchronize(st));
    rep.ms_f64 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  } else if (o.mode == 1) {
    s = load_initial<Tp, float>(plan, *C, *C->lf[0], psi, inject);
    if (s != GPE_OK) return s;
    s = solve_mixed(*C, P, st, fs, nfe, rep);
    if (s != GPE_OK) return s;
    fin = C->ld.back().get();
  } else {
    s = load_initial<Tp, float>(plan, *C, *C->lf[0], psi, inject);
    if (s != GPE_OK) return s;
    s = solve_levels<float>(C->lf, P, true, st, fs, nfe);
    if (s != GPE_OK) return s;
    rep.outer_f32 = fs.outer;
    rep.inner_f32 = fs.inner;
    GPE_CUDA(cudaStreamSynchronize(st));
    auto t1 = std::chrono::steady_clock::now();
    rep.ms_f32 = std::chrono::duration<double, std::milli>(t1 - t0).count();
    // float64 refinement (mode 1) or float64 evaluation of the result (mode 2)
    Level<float>& Lf = *C->lf.back();
    fin = C->fine64.get();
    const long long nreal = Lf.M * (Lf.g.is_complex ? 2 : 1);
    s = convert_vec<float, double>(Lf.xk, fin->xs[0], nreal, 1.0, st);
    if (s != GPE_OK) return s;
    s = normalise_slot0<double>(*fin, st);
    if (s != GPE_OK) return s;
    LevelStats ls;
    {
      // mode 2: one float64 evaluation of the float32 result
      SolveParams P64 = P;
      P64.max_outer = 0;
      s = rn_run<double>(*fin, P64, 0, false, st, ls, fs.theta);
    }
    if (s != GPE_OK) return s;
    nfe += ls.nfe;
    fs = ls;
    GPE_CUDA(cudaStreamSynchronize(st));
    rep.ms_f64 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  }
  // result: X (float64 or bulk precision) -> psi in plan precision
  const long long nreal = fin->M * (fin->g.is_complex ? 2 : 1);
  const double inv_s = 1.0 / sqrt(fin->g.hvol);
  if (plan->prec == GPE_F64) s = convert_vec<double, double>(fin->xk, psi, nreal, inv_s, st);
  else s = convert_vec<double, float>(fin->xk, psi, nreal, inv_s, st);
  if (s != GPE_OK) return s;
  GPE_CUDA(cudaEventRecord(C->ev, st));
  GPE_CUDA(cudaStreamWaitEvent(plan->stream, C->ev, 0));
  GPE_CUDA(cudaStreamSynchronize(st));
  rep.E = fs.F;
  rep.mu = 0.5 * fs.theta;
  rep.res = 0.5 * fs.res;
  rep.nfe = nfe;
  rep.status = fs.converged ? GPE_OK : GPE_ENOCONV;
  if (o.mode == 2) rep.status = GPE_OK;
  return GPE_OK;
}

// Autotuning of the cluster engine's per-CTA share for single solves on grid
// gh: a float32 Algorithm 1 run of 24 iterations from the trap's Gaussian (unit
// norm) for every share of {2, 4, 8, 16, 32} KiB that gives a distinct
// cluster size; the fastest time per trial wins and is recorded.
gpe_status tune_cluster_share(const GridHost& gh, cudaStream_t st, int* best_kb, double* best_us) {
  *best_kb = 0;
  *best_us = 0.0;
  if (gh.disc != GPE_FOURIER || gh.dim != 2 || gh.v_kind == GPE_V_ARRAY) return GPE_OK;
  GridHost g = gh;
  g.nbatch = 1;
  const int n0 = g.ext[0], n1 = g.ext[1], cplx = g.is_complex;
  int cs, lch, P0, P1;
  size_t smem;
  unsigned int vb, vp;
  if (!cluster_shape(n0, n1, cplx, 5, &cs, &lch, &P0, &P1, &smem, &vb, &vp)) return GPE_OK;
  // start point: exp(-(x^2 + y^2)/2), unit 2-norm, float32 (complex: zero imaginary part)
  const int per = cplx ? 2 : 1;
  std::vector<float> h((size_t)g.M * per, 0.f);
  double nrm = 0.0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      const double x = g.nodes[0][i], y = g.nodes[1][j];
      const double v = exp(-0.5 * (x * x + y * y));
      h[((size_t)j * n0 + i) * per] = (float)v;
      nrm += v * v;
    }
  const float sc = (float)(1.0 / sqrt(nrm));
  for (size_t k = 0; k < h.size(); ++k) h[k] *= sc;
  Level<float> L;
  gpe_status s = L.create(g);
  SolveParams P{};
  P.max_iter = 24;
  P.cluster = 1;
  P.search = 0;
  P.eta = 0.85;
  P.alpha_hat = 1e-3;
  const int saved = tuned_share_kb(n0, n1, cplx);
  int last_cs = -1, pick = saved;
  double best = 1e300;
  const int cand[5] = {2, 4, 8, 16, 32};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (s == GPE_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    s = fail(GPE_ECUDA, "cudaEventCreate");
  for (int ci = 0; ci < 5 && s == GPE_OK; ++ci) {
    if (!cluster_shape(n0, n1, cplx, 5, &cs, &lch, &P0, &P1, &smem, &vb, &vp, (size_t)cand[ci] * 1024)) continue;
    if (cs == last_cs) continue;
    last_cs = cs;
    set_tuned_share_kb(n0, n1, cplx, cand[ci]);
    double ms_sum = 0.0;
    int nfe_sum = 0;
    for (int rep = 0; rep < 3 && s == GPE_OK; ++rep) {
      if (cudaStreamSynchronize(st) != cudaSuccess ||
          cudaMemcpy(L.xs[0], h.data(), L.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        s = fail(GPE_ECUDA, "autotune start point");
        break;
      }
      LevelStats ls;
      bool used = false;
      cudaEventRecord(e0, st);
      s = fg_run_cluster(L, P, false, st, ls, 0.0, &used);
      cudaEventRecord(e1, st);
      if (s != GPE_OK || !used) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) {
        ms_sum += ms;
        nfe_sum += ls.nfe;
      }
    }
    if (s == GPE_OK && nfe_sum > 0) {
      const double us = 1e3 * ms_sum / nfe_sum;
      if (us < best) {
        best = us;
        pick = cand[ci];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  L.destroy();
  set_tuned_share_kb(n0, n1, cplx, s == GPE_OK ? pick : saved);
  if (s != GPE_OK) return s;
  if (best < 1e300) {
    *best_kb = pick;
    *best_us = best;
  }
  return GPE_OK;
}

}  // namespace gpe

using namespace gpe;

extern "C" gpe_status gpe_rnewton_solve(gpe_plan plan, void* psi_inout, const gpe_solve_opts* opts,
                                        gpe_solve_report* report) {
  if (!plan || !psi_inout) return fail(GPE_EINVAL, "plan or psi is NULL");
  if (plan->g.nbatch != 1) return fail(GPE_EINVAL, "gpe_rnewton_solve needs a plan with nbatch = 1");
  gpe_solve_opts o;
  if (opts) o = *opts;
  else gpe_solve_opts_default(&o);
  if (o.levels < 1 || o.mode < 0 || o.mode > 2 || o.method < 0 || o.method > 1 || o.chunk < 1 || o.k_init < 0 ||
      o.k_sub < 1 || o.max_outer < 0 || o.max_iter < 0 || !(o.res_tol >= 0) || !(o.delta0 > 0) ||
      !search_opts_ok(o))
    return fail(GPE_EINVAL, "invalid solve options");
  for (int a = 0; a < plan->g.dim; ++a) {
    const int nc = plan->g.N[a] >> (o.levels - 1);
    if ((nc << (o.levels - 1)) != plan->g.N[a] || nc < 4)
      return fail(GPE_EINVAL, "too many cascade levels for this grid (coarsest n must be >= 4)");
  }
  gpe_solve_report rep;
  memset(&rep, 0, sizeof(rep));
  gpe_status s = plan->prec == GPE_F64 ? solve_impl<double>(plan, psi_inout, o, rep)
                                       : solve_impl<float>(plan, psi_inout, o, rep);
  if (report) *report = rep;
  if (s != GPE_OK) return s;
  return rep.status == GPE_ENOCONV ? GPE_ENOCONV : GPE_OK;
}

// ----------------------------------------------------------------- batched solves
namespace gpe {

// Device buffers of one group of same-grid instances.
struct BatchGroup {
  std::vector<int> idx;
  GridHost g;
  GridDev<float> d;
  Scratch sc;
  void* x = nullptr;
  void* gr = nullptr;
  float* V = nullptr;
  float* omega = nullptr;
  Alg1Ctl* ctl = nullptr;
  unsigned int* next = nullptr;
  ~BatchGroup() {
    d.destroy();
    sc.destroy();
    cudaFree(x);
    cudaFree(gr);
    cudaFree(V);
    cudaFree(omega);
    cudaFree(ctl);
    cudaFree(next);
  }
};

// Point a level built for one problem of a group at another problem on the
// same grid (extents, box, complexity): its potential, beta and Omega.  The
// level's cached CUDA graphs captured the old operator and are dropped.
template <typename T>
static gpe_status level_set_problem(Level<T>& L, const GridHost& gi) {
  L.g.beta = gi.beta;
  L.g.omega = gi.omega;
  std::vector<T> hv((size_t)L.M);
  for (long long i = 0; i < L.M; ++i) hv[(size_t)i] = (T)gi.V[(size_t)i];
  GPE_CUDA(cudaMemcpy(L.d.V, hv.data(), sizeof(T) * hv.size(), cudaMemcpyHostToDevice));
  if (L.g.disc != GPE_FD) {
    for (int a = 0; a < 2 && a < L.g.dim; ++a) {
      PassGeom<T>& G = L.d.geom[a];
      if (gi.omega != 0.0) {
        G.c1 = (T)((a == 0 ? gi.omega : -gi.omega) / G.F);
        G.rcoord = L.d.coord[a == 0 ? 1 : 0];
      } else {
        G.c1 = (T)0;
        G.rcoord = nullptr;
      }
    }
  }
  L.d.fd.omega = gi.omega;
  const float om = (float)gi.omega;
  GPE_CUDA(cudaMemcpy(L.d_omega, &om, sizeof(float), cudaMemcpyHostToDevice));
  for (int i = 0; i < 3; ++i)
    if (L.chunk_exec[i]) {
      cudaGraphExecDestroy(L.chunk_exec[i]);
      L.chunk_exec[i] = nullptr;
    }
  return GPE_OK;
}

static bool same_grid(const GridHost& a, const GridHost& b) {
  return a.ext[0] == b.ext[0] && a.ext[1] == b.ext[1] && a.is_complex == b.is_complex && a.lo[0] == b.lo[0] &&
         a.lo[1] == b.lo[1] && a.hi[0] == b.hi[0] && a.hi[1] == b.hi[1];
}

static gpe_status run_batch_group(BatchGroup& B, const std::vector<GridHost>& gh, void* const* psi,
                                  const SolveParams& P, gpe_solve_report* reports, cudaStream_t st) {
  const int n = (int)B.idx.size();
  const GridHost& g = B.g;
  const long long M = g.M;
  const int cplx = g.is_complex;
  const long long nreal = M * (cplx ? 2 : 1);
  const size_t vbytes = sizeof(float) * (size_t)nreal;
  gpe_status s = B.d.create(g);
  if (s != GPE_OK) return s;
  const long long tiles = std::max<long long>(1, std::min<long long>((M + NTHREADS - 1) / NTHREADS, 512));
  s = B.sc.create((size_t)tiles * n, n);
  if (s != GPE_OK) return s;
  GPE_CUDA(cudaMalloc(&B.x, vbytes * n));
  GPE_CUDA(cudaMalloc(&B.gr, vbytes * n));
  GPE_CUDA(cudaMalloc(&B.V, sizeof(float) * (size_t)M * n));
  GPE_CUDA(cudaMalloc(&B.omega, sizeof(float) * n));
  GPE_CUDA(cudaMalloc(&B.ctl, sizeof(Alg1Ctl) * n));
  GPE_CUDA(cudaMalloc(&B.next, sizeof(unsigned int)));
  // per-instance potential, Omega and control (alpha = beta / (2 h_vol))
  std::vector<float> hv((size_t)M * n), hom(n);
  std::vector<Alg1Ctl> hc(n);
  for (int k = 0; k < n; ++k) {
    const GridHost& gi = gh[B.idx[k]];
    for (long long i = 0; i < M; ++i) hv[(size_t)k * M + i] = (float)gi.V[i];
    hom[k] = (float)gi.omega;
    init_cluster_ctl(hc[k], gi.beta / (2.0 * gi.hvol), P, true, 0.0);
  }
  GPE_CUDA(cudaMemcpyAsync(B.V, hv.data(), sizeof(float) * hv.size(), cudaMemcpyHostToDevice, st));
  GPE_CUDA(cudaMemcpyAsync(B.omega, hom.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
  GPE_CUDA(cudaMemcpyAsync(B.ctl, hc.data(), sizeof(Alg1Ctl) * n, cudaMemcpyHostToDevice, st));
  GPE_CUDA(cudaMemsetAsync(B.next, 0, sizeof(unsigned int), st));
  // initial data: psi -> X = sqrt(h_vol) psi, then unit 2-norm per instance
  const double sh = sqrt(g.hvol);
  for (int k = 0; k < n; ++k) {
    s = launch_convert<float, float>((const float*)psi[B.idx[k]], (float*)((char*)B.x + vbytes * k), nreal, sh, st);
    if (s != GPE_OK) return s;
  }
  s = launch_moments<float>(B.x, nullptr, M, n, cplx, B.sc, st);
  if (s != GPE_OK) return s;
  s = launch_norm_coef(B.sc.results, n, 1.0, B.sc.coef, st);
  if (s != GPE_OK) return s;
  s = launch_axpby<float>(B.x, nullptr, B.sc.coef, 1, M, n, B.x, cplx, st);
  if (s != GPE_OK) return s;
  // all instances of the group in one cluster launch
  ClusterArgs A{};
  A.n0 = g.ext[0];
  A.n1 = g.ext[1];
  A.ninst = n;
  A.max_loops = (P.max_iter + 1) * (hc[0].max_bt + 1) + 1;
  A.dlam0 = (float)(2.0 * M_PI / (g.hi[0] - g.lo[0]));
  A.dlam1 = (float)(2.0 * M_PI / (g.hi[1] - g.lo[1]));
  A.V = B.V;
  A.vstride = M;
  A.xn = B.d.coord[0];
  A.yn = B.d.coord[1];
  A.omega = cplx ? B.omega : nullptr;
  A.tw0 = B.d.tw[0];
  A.tw1 = B.d.tw[1];
  A.x = B.x;
  A.g = B.gr;
  A.ctl = B.ctl;
  A.results = B.sc.results;
  A.next = B.next;
  auto t0 = std::chrono::steady_clock::now();
  s = launch_cluster_alg1(A, cplx, st);
  if (s != GPE_OK) return s;
  // results back to psi (physical units) and the reports
  for (int k = 0; k < n; ++k) {
    s = launch_convert<float, float>((const float*)((char*)B.x + vbytes * k), (float*)psi[B.idx[k]], nreal, 1.0 / sh,
                                     st);
    if (s != GPE_OK) return s;
  }
  GPE_CUDA(cudaMemcpyAsync(hc.data(), B.ctl, sizeof(Alg1Ctl) * n, cudaMemcpyDeviceToHost, st));
  GPE_CUDA(cudaStreamSynchronize(st));
  const double ms32 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() / n;
  for (int k = 0; k < n; ++k) {
    const Alg1Ctl& c = hc[k];
    gpe_solve_report& r = reports[B.idx[k]];
    memset(&r, 0, sizeof(r));
    r.E = c.F_cur;
    r.mu = 0.5 * c.theta_c;
    r.res = 0.5 * c.res;
    // an instance that met res_tol converged; one that stopped at switch_rel
    // or at the float32 floor did not reach the stated tolerance
    r.status = c.status == 4 ? GPE_ENONFINITE : ((c.status == 5 || r.res > 0.5 * P.res_tol_X) ? GPE_ENOCONV : GPE_OK);
    r.inner_f32 = c.k;
    r.nfe = c.nfe;
    r.ms_f32 = ms32;
  }
  if (!P.refine) return GPE_OK;
  // float64 refinement (the mixed schedule's finest level, per instance):
  // Algorithm 2 with float64 outer quantities and float32 difference-form
  // subproblems in the cluster engine, from the float32 state, for every
  // instance that did not reach res_tol
  struct LevelPair {
    Level<double> d;
    Level<float> f;
    ~LevelPair() {
      d.destroy();
      f.destroy();
    }
  };
  std::unique_ptr<LevelPair> LP(new LevelPair());
  Level<double>* Ld = &LP->d;
  Level<float>* Lf = &LP->f;
  s = Ld->create(g);
  if (s == GPE_OK) s = Lf->create(g);
  if (s != GPE_OK) return s;
  // the refinement captures CUDA graphs, which the caller's stream may not
  // allow (the legacy default stream cannot be captured): it runs on a
  // private stream, after the work queued so far and before anything queued
  // on the caller's stream later
  struct PrivStream {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ~PrivStream() {
      if (e) cudaEventDestroy(e);
      if (s) cudaStreamDestroy(s);
    }
  } ps;
  GPE_CUDA(cudaStreamCreateWithFlags(&ps.s, cudaStreamNonBlocking));
  GPE_CUDA(cudaEventCreateWithFlags(&ps.e, cudaEventDisableTiming));
  GPE_CUDA(cudaEventRecord(ps.e, st));
  GPE_CUDA(cudaStreamWaitEvent(ps.s, ps.e, 0));
  const cudaStream_t caller = st;
  st = ps.s;
  for (int k = 0; k < n; ++k) {
    gpe_solve_report& r = reports[B.idx[k]];
    if (r.status == GPE_ENONFINITE || r.status == GPE_OK) continue;
    const GridHost& gi = gh[B.idx[k]];
    auto t1 = std::chrono::steady_clock::now();
    s = level_set_problem<double>(*Ld, gi);
    if (s == GPE_OK) s = level_set_problem<float>(*Lf, gi);
    if (s != GPE_OK) return s;
    s = launch_convert<float, double>((const float*)((char*)B.x + vbytes * k), (double*)Ld->xs[0], nreal, 1.0, st);
    if (s == GPE_OK) s = normalise_slot0<double>(*Ld, st);
    if (s != GPE_OK) return s;
    LevelStats l2;
    s = rn_run<double>(*Ld, P, 0, false, st, l2, 2.0 * r.mu, Lf);
    if (s != GPE_OK) return s;
    s = launch_convert<double, float>((const double*)Ld->xk, (float*)psi[B.idx[k]], nreal, 1.0 / sh, st);
    if (s != GPE_OK) return s;
    GPE_CUDA(cudaStreamSynchronize(st));
    r.E = l2.F;
    r.mu = 0.5 * l2.theta;
    r.res = 0.5 * l2.res;
    r.status = l2.converged ? GPE_OK : GPE_ENOCONV;
    r.outer_f64 = l2.outer;
    r.inner_f64 = l2.inner;
    r.inner_f32 += l2.inner32;
    r.nfe += l2.nfe;
    r.ms_f64 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  }
  GPE_CUDA(cudaEventRecord(ps.e, st));
  GPE_CUDA(cudaStreamWaitEvent(caller, ps.e, 0));
  GPE_CUDA(cudaStreamSynchronize(st));
  return GPE_OK;
}

}  // namespace gpe

extern "C" gpe_status gpe_solve_batch(const gpe_problem* problems, int n, void* const* psi,
                                      const gpe_solve_opts* opts, gpe_solve_report* reports, void* cuda_stream) {
  if (!problems || !psi || !reports || n < 1) return fail(GPE_EINVAL, "NULL argument or n < 1");
  gpe_solve_opts o;
  if (opts) o = *opts;
  else gpe_solve_opts_default(&o);
  if (o.max_iter < 1 || !(o.res_tol >= 0) || !search_opts_ok(o)) return fail(GPE_EINVAL, "invalid solve options");
  std::vector<GridHost> gh(n);
  for (int i = 0; i < n; ++i) {
    if (!psi[i]) return fail(GPE_EINVAL, "psi[i] is NULL");
    gpe_status s = grid_from_problem(&problems[i], 1, gh[i]);
    if (s != GPE_OK) return s;
    const GridHost& g = gh[i];
    int cs, lch, P0, P1;
    size_t smem;
    unsigned int vb, vp;
    if (g.disc != GPE_FOURIER || g.dim != 2 ||
        !cluster_shape(g.ext[0], g.ext[1], g.is_complex, 5, &cs, &lch, &P0, &P1, &smem, &vb, &vp))
      return fail(GPE_EINVAL, "gpe_solve_batch takes 2D Fourier grids whose state fits one cluster (<= 256^2)");
  }
  if (o.mode != 1 && o.mode != 2) return fail(GPE_EINVAL, "gpe_solve_batch: mode must be 1 (mixed) or 2 (float32)");
  SolveParams P{};
  P.max_iter = o.max_iter;
  P.search = o.search;
  P.alpha_hat = o.alpha_hat;
  P.eta = o.eta;
  P.eps0 = o.eps0;
  P.res_tol_X = 2.0 * o.res_tol;
  P.switch_rel = o.switch_rel;
  // the float64 refinement (mode 1) runs Algorithm 2 with these
  P.refine = o.mode == 1 && o.res_tol > 0.0;
  P.k_init = 0;
  P.k_sub = o.k_sub;
  P.max_outer = o.max_outer;
  P.chunk = o.chunk;
  P.use_graphs = o.use_graphs;
  P.persistent = o.persistent;
  P.cluster = o.cluster;
  P.delta_stop = 0.0;        // stop on res_tol (or max_outer), not on Eq. crit2
  P.delta0 = o.delta0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // group the instances by grid; one cluster launch per group
  std::vector<std::unique_ptr<BatchGroup>> groups;
  for (int i = 0; i < n; ++i) {
    BatchGroup* grp = nullptr;
    for (auto& b : groups)
      if (same_grid(b->g, gh[i])) grp = b.get();
    if (!grp) {
      groups.emplace_back(new BatchGroup());
      grp = groups.back().get();
      grp->g = gh[i];
      grp->g.nbatch = 1;
    }
    grp->idx.push_back(i);
  }
  for (auto& b : groups) {
    gpe_status s = run_batch_group(*b, gh, psi, P, reports, st);
    if (s != GPE_OK) return s;
  }
  for (int i = 0; i < n; ++i)
    if (reports[i].status == GPE_ENONFINITE) return fail(GPE_ENONFINITE, "non-finite energy in a batched instance");
  return GPE_OK;
}
