// gpe_kernels.cuh -- device code of libgpe (sm_103a).
//
// The discretised GP operator of the paper (§2) is applied matrix-free as a sum
// of per-axis line operators: along every axis, each grid line is transformed
// (Fourier: an N-point DFT, Eq. fftp36; sine: the DST-I of Eq. tpll computed as
// the 2N-point DFT of the odd extension), multiplied by the line's symbol
// (lam^2/2, plus the folded rotation term +Omega*y*lam on x-lines and
// -Omega*x*eta on y-lines, Eq. energy-discrete-FP), and transformed back
// (Eq. fftp35 / spdo1).  One CTA owns a tile of lines in shared memory for the
// whole forward-multiply-inverse sequence, so a pass reads its input once and
// writes its output once.  The last pass of an application fuses the pointwise
// terms (V, the cubic term, Lemma 3.1's Hessian terms) and float64 block
// reductions; the last CTA to finish folds the per-CTA partials in a fixed
// order (deterministic) and, in the solver, runs Algorithm 1's step-size logic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpe {

template <typename T> struct C2t;
template <> struct C2t<float> { using type = float2; };
template <> struct C2t<double> { using type = double2; };

constexpr int NTHREADS = 256;  // largest block size
constexpr int MAXLB = 128;     // data lines per tile
constexpr int NQ = 15;         // reduction slots per launch and instance

// Reduction slots of the solver's evaluation passes (EPI_F / EPI_W).
enum {
  Q_E2 = 0,    // Re sum conj(y) (H_lin y)          -> 1/2 Y^*AY
  Q_E4 = 1,    // sum |y|^4
  Q_NY = 2,    // sum |y|^2
  Q_YG = 3,    // Re sum conj(y) g
  Q_GG = 4,    // sum |g|^2
  Q_Q = 5,     // sum |g - th_c y|^2
  Q_QY = 6,    // Re sum conj(g - th_c y) y
  Q_SS = 7,    // sum |s|^2,     s = y - x_c
  Q_SV = 8,    // Re sum conj(s) v,  v = g - g_c - th_c s
  Q_VV = 9,    // sum |v|^2
  Q_VY = 10,   // Re sum conj(v) y
  Q_SY = 11,   // Re sum conj(s) y
  Q_WX = 12,   // W objective: non-quadratic part of W^(k)
  Q_DF = 13,   // objective(y) - objective(x_c) in difference form
  Q_MAX = 14   // max |s_j| (max-reduction)
};
// Slots of the ratio pass (EPI_RATIO), d = Z - X^k.
enum { R_AXD = 0, R_DAD = 1, R_QD = 2, R_X2D2 = 3, R_R2 = 4, R_DD = 5, R_GD = 6 };

// EPI_WS: the regularized Newton model in difference form (unknown D = X - X^k,
// gradient G^ = P_k + H_k D + (delta - theta_k) D; base = X^k, gk = P_k).
enum Epi { EPI_ACC = 0, EPI_GRAD = 1, EPI_HESS = 2, EPI_F = 3, EPI_W = 4, EPI_RATIO = 5, EPI_WS = 6 };

// Device-resident state of one Algorithm 1 run (one instance).  The passes read
// the slot indices and scalars at their start; the last CTA of the final pass
// updates them (see alg1_control).
// S: storage type of the real-valued fields (double in global memory; the
// cluster engine's float32 runs keep a float copy in shared memory, whose
// control then runs without float64 conversions).  The objective values stay
// double (reported, never tested).
template <typename S>
struct Alg1CtlT {
  // configuration (host-written before the run)
  double alpha;        // beta / (2 h_vol)
  S delta;             // W objective: regularisation delta^(k)
  S rho1, eta, delta_bt, eps0, res_tol, res_rel, tau0, renorm_tol;
  int max_bt, max_iter, objective, always_renorm;
  // slot state
  int cur, prev, trial, has_cur, done, status, phase, pad0;
  S theta_c;           // theta of the current point (used by the passes)
  S theta_hint;        // before the first point is accepted: a nearby theta
                       // (the projected-gradient norm is formed relative to it)
  // iteration state
  int k, m, nfe, accepted_last;
  S tau, Cg, Q;        // Cg = C - F_cur
  double F_cur;
  S nX, XG, GG, PP, smax;
  double obj_last;
  S tau_last;
  S a, b, s;           // Cayley step coefficients of the next trial
  S am1;               // a - 1 without cancellation (shifted subproblem form)
  S theta_ref;         // shifted form: theta_k of the outer iterate
  S res;               // ||A(X)X||_2 of the current point
  S best_res;          // smallest res seen (stagnation test)
  int k_best, stall_iters;   // stop after stall_iters accepted steps without a new best (0 = off)
  int two_slots;       // 1: slots cur/trial swap on acceptance (no third slot)
  int monotone;        // 1: monotone Armijo search, tau = alpha_hat delta_bt^m, C = F(X_cur)
  S alpha_hat;         // first trial step of every monotone search
};
using Alg1Ctl = Alg1CtlT<double>;

// Field-by-field copy between storage types.
template <typename D, typename S>
__host__ __device__ inline void ctl_copy(Alg1CtlT<D>& d, const Alg1CtlT<S>& s) {
  d.alpha = s.alpha;
  d.delta = (D)s.delta;
  d.rho1 = (D)s.rho1;
  d.eta = (D)s.eta;
  d.delta_bt = (D)s.delta_bt;
  d.eps0 = (D)s.eps0;
  d.res_tol = (D)s.res_tol;
  d.res_rel = (D)s.res_rel;
  d.tau0 = (D)s.tau0;
  d.renorm_tol = (D)s.renorm_tol;
  d.max_bt = s.max_bt;
  d.max_iter = s.max_iter;
  d.objective = s.objective;
  d.always_renorm = s.always_renorm;
  d.cur = s.cur;
  d.prev = s.prev;
  d.trial = s.trial;
  d.has_cur = s.has_cur;
  d.done = s.done;
  d.status = s.status;
  d.phase = s.phase;
  d.pad0 = s.pad0;
  d.theta_c = (D)s.theta_c;
  d.theta_hint = (D)s.theta_hint;
  d.k = s.k;
  d.m = s.m;
  d.nfe = s.nfe;
  d.accepted_last = s.accepted_last;
  d.tau = (D)s.tau;
  d.Cg = (D)s.Cg;
  d.Q = (D)s.Q;
  d.F_cur = s.F_cur;
  d.nX = (D)s.nX;
  d.XG = (D)s.XG;
  d.GG = (D)s.GG;
  d.PP = (D)s.PP;
  d.smax = (D)s.smax;
  d.obj_last = s.obj_last;
  d.tau_last = (D)s.tau_last;
  d.a = (D)s.a;
  d.b = (D)s.b;
  d.s = (D)s.s;
  d.am1 = (D)s.am1;
  d.theta_ref = (D)s.theta_ref;
  d.res = (D)s.res;
  d.best_res = (D)s.best_res;
  d.k_best = s.k_best;
  d.stall_iters = s.stall_iters;
  d.two_slots = s.two_slots;
  d.monotone = s.monotone;
  d.alpha_hat = (D)s.alpha_hat;
}

// Outer state of Algorithm 2 (ratio test), written by the ratio pass.
struct RNCtl {
  double alpha, delta, eta1, eta2, gamma1, gamma2, delta_min, delta_max, F_k;
  double ared, pred, rho, dmax;
  int accepted, pad;
};

template <typename T>
struct PassGeom {
  int axis;             // 0 (x), 1 (y), 2 (z)
  int n0, n1, n2;       // extents of one instance
  long long M;          // unknowns per instance
  int len;              // extent along the axis
  long long stride;     // element stride along the axis
  long long ostride;    // axes 1,2: stride of the outer index
  int F, logF;          // FFT length
  int P;                // row pitch of the shared-memory FFT buffers (padded, see pidx)
  int odd_ext;          // sine grid: odd extension to 2N
  int LB;               // data lines per tile (power of two, <= MAXLB)
  int logLB;
  int LC;               // complex lines per tile
  int tpl, ltpl;        // axis 0: threads per line (power of two) and its log2
  int nthreads;         // block size
  int tiles;            // tiles per instance
  int xt;               // axes 1,2: tiles along x
  const typename C2t<T>::type* tw;  // e^{-2 pi i k / F}
  const T* lam;         // wavenumber of FFT index m
  T c2, c1;             // symbol = c2*lam^2 + c1*coord*lam  (1/F folded in)
  T dlam;               // lam of FFT index m = dlam * p(m), p(m) = m or m - F
  const T* rcoord;      // rotation coordinate table (x or y nodes) or null
};

struct FDGeom {
  int dim, n0, n1, n2;
  long long M;
  double ih2[3];        // 1/h_a^2
  double ih2c[3];       // 1/(2 h_a) for the central differences
  double omega;
  int tiles;            // blocks per instance
};

template <typename T>
struct PassData {
  const void* x;        // input vector (ABI modes); solver: resolved from slots
  const void* xsub;     // optional: input = x - xsub
  const void* acc_in;   // kinetic part of earlier passes (or null)
  void* out;            // EPI_ACC: accumulator; final: output vector (or null)
  // solver slots
  void* const* xs;      // 3 X slots
  void* const* gs;      // 3 G slots
  Alg1Ctl* ctl;         // non-null in solver mode
  RNCtl* rn;            // ratio pass
  int step_on_load;     // Y = s(a X_cur + b G_cur) formed on load, stored to xs[trial]
  int use_slots;        // x = xs[trial], out = gs[trial] (final), xc/gc from slots
  // pointwise data
  const T* V;
  const void* base;     // HESS: psi; W, RATIO: X^k
  const void* gk;       // RATIO: G_k
  double nl;            // ABI: beta; solver: alpha (read from ctl when null)
  double shift;         // HESS shift
  double lin_scale;     // 1 (ABI) or 2 (unified A = 2 H_lin)
  // reductions
  double* partials;     // [gridDim.x][NQ]
  double* results;      // [nbatch][NQ]
  unsigned int* ticket;
  int nq;               // active slots (0: none)
  int control;          // 0: none, 1: Algorithm 1 control, 2: ratio control
};

// Arguments of the cluster engine (float32 Algorithm 1, 2D Fourier grids, one
// thread-block cluster per instance).
struct ClusterArgs {
  int n0, n1;              // x extent (row length) and y extent (rows), powers of two
  int logn0, logn1;
  int cs, logcs;           // cluster size
  int ninst;               // instances
  int max_loops;           // bound on Algorithm 1 trials per instance
  int lch;                 // complex lines per FFT chunk (power of two)
  int P0, P1;              // padded row pitches of the FFT buffers (n0 and n1 lines)
  float dlam0, dlam1;      // 2 pi / L per axis
  const float* V;          // potential [ninst or 1][n1][n0]
  long long vstride;       // instance stride of V (0 = shared)
  const float* xn;         // x nodes [n0]
  const float* yn;         // y nodes [n1]
  const float* omega;      // Omega per instance (null: 0)
  const float2* tw0;       // e^{-2 pi i k / n0}
  const float2* tw1;       // e^{-2 pi i k / n1}
  void* x;                 // [ninst][n1][n0]: X0 in (unit norm), final X out
  void* g;                 // [ninst][n1][n0]: final G out (may be null)
  Alg1Ctl* ctl;            // [ninst], phase 0 prepared by the host
  double* results;         // [ninst][NQ] sums of the final evaluation
  unsigned int vec_bytes;  // bytes of one CTA's share of a vector (16-byte multiple)
  unsigned int vpot_bytes; // bytes of the CTA's rows of the potential (float32, 16-byte multiple)
  unsigned long long* dbg; // optional phase timestamps (CTA 0, first instance): [loop][8]
  int dbg_n;
  int shifted;             // 1: regularized Newton subproblem in difference form (see cluster.cu)
  const void* xk;          // shifted: X^k (float32) [ninst][n1][n0]
  const void* pk;          // shifted: P_k = G_k - theta_k X^k (float32)
  int share_kb;            // cluster size: smallest with a per-CTA vector share <= this (KiB; 0: 16)
  unsigned int* next;      // instance counter (zero at launch): clusters take the next
                           // unstarted instance when they finish one; null: round robin
};

// Arguments of the persistent Algorithm 1 kernel.
template <typename T>
struct PersistArgs {
  PassGeom<T> G[3];
  int blocks[3];        // tiles (x instances) of each axis pass
  int dim;
  PassData<T> D;        // solver data (slots, control block, reduction scratch)
  void* acc;            // kinetic accumulator
  unsigned int* bar;    // grid barrier: [0] arrivals, [1] generation
  int* err;             // set when a barrier wait gave up
  long long max_polls;  // polls of one barrier wait before it gives up
  int max_loops;        // bound on the iterations (accepted + rejected trials)
  size_t tw_bytes;      // twiddle tables of all axes at the front of shared memory (16-byte multiple)
  unsigned long long* dbg;   // optional phase timestamps (globaltimer, CTA 0): [loop][4]
  int dbg_n;
};

}  // namespace gpe
