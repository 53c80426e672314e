// ops_impl.cuh -- kernel templates of libgpe, instantiated per precision by
// ops_f32.cu and ops_f64.cu.  See gpe_kernels.cuh for the design summary.
#pragma once
#include <math.h>
#include "gpe_kernels.cuh"
#include "gpe_internal.h"

namespace gpe {

// ----------------------------------------------------------------- value helpers
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

template <typename T, bool CPLX> struct VT { using V = T; };
template <typename T> struct VT<T, true> { using V = typename C2t<T>::type; };

// Re(conj(a) b), |a|^2 in the working precision
__device__ __forceinline__ float tre(float a, float b) { return a * b; }
__device__ __forceinline__ double tre(double a, double b) { return a * b; }
__device__ __forceinline__ float tre(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ double tre(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
// the same products accumulated in float64
__device__ __forceinline__ double dre(float a, float b) { return (double)a * (double)b; }
__device__ __forceinline__ double dre(double a, double b) { return a * b; }
__device__ __forceinline__ double dre(float2 a, float2 b) { return (double)a.x * b.x + (double)a.y * b.y; }
__device__ __forceinline__ double dre(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }
template <> __device__ __forceinline__ double vzero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C mk(double re, double im);
template <> __device__ __forceinline__ float2 mk<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ double2 mk<double2>(double re, double im) { return make_double2(re, im); }

// ----------------------------------------------------------------- tile geometry
// Base offset of data line l of a tile; false if the line lies outside the grid.
// ri receives the index into the rotation coordinate table.
template <typename T>
__device__ __forceinline__ bool line_base(const PassGeom<T>& G, int inst, int tile, int l,
                                          long long& base, int& ri) {
  if (G.axis == 0) {
    long long r = (long long)tile * G.LB + l;
    if (r >= (long long)G.n1 * G.n2) return false;
    base = inst * G.M + r * G.n0;
    ri = (int)(r % G.n1);
    return true;
  }
  int o = tile / G.xt;
  int x = (tile - o * G.xt) * G.LB + l;
  if (x >= G.n0) return false;
  base = inst * G.M + (long long)o * G.ostride + x;
  ri = x;
  return true;
}

// ----------------------------------------------------------------- FFT in shared memory
// Stockham autosort, radix 4 (and one radix-2 stage when log2 F is odd),
// forward sign e^{-2 pi i j p / F}, unnormalised.  nl lines of length F stored
// contiguously in `a`; `b` is scratch of the same size.  Returns the buffer that
// holds the result.  Ends with a barrier.
template <typename C>
__device__ C* fft_lines(C* a, C* b, int F, int nl, const C* __restrict__ tw) {
  C* src = a;
  C* dst = b;
  for (int Ns = 1; Ns < F;) {
    const int R = ((F / Ns) & 3) == 0 ? 4 : 2;
    const int nb = F / R;
    const int tot = nl * nb;
    const int twstep = F / (Ns * R);
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int line = t / nb;
      const int j = t - line * nb;
      const int k = j & (Ns - 1);
      const C* s = src + line * F + j;
      C* d = dst + line * F + (j - k) * R + k;
      if (R == 4) {
        C v0 = s[0], v1 = s[nb], v2 = s[2 * nb], v3 = s[3 * nb];
        if (Ns > 1) {
          const int e = k * twstep;
          v1 = cmul(v1, tw[e]);
          v2 = cmul(v2, tw[2 * e]);
          v3 = cmul(v3, tw[3 * e]);
        }
        C s02 = v0 + v2, d02 = v0 - v2, s13 = v1 + v3, d13 = v1 - v3;
        d[0] = s02 + s13;
        d[Ns].x = d02.x + d13.y;  d[Ns].y = d02.y - d13.x;      // d02 - i d13
        d[2 * Ns] = s02 - s13;
        d[3 * Ns].x = d02.x - d13.y; d[3 * Ns].y = d02.y + d13.x;  // d02 + i d13
      } else {
        C v0 = s[0], v1 = s[nb];
        if (Ns > 1) v1 = cmul(v1, tw[k * twstep]);
        d[0] = v0 + v1;
        d[Ns] = v0 - v1;
      }
    }
    __syncthreads();
    C* t = src; src = dst; dst = t;
    Ns *= R;
  }
  return src;
}

// ----------------------------------------------------------------- block reductions
// Reduce acc[0..NQ) over the block (slot Q_MAX is a max), write this CTA's
// partials, and let the last CTA fold all partials per instance in a fixed order
// into results[inst][q].  Returns true in the last CTA (all threads).
static __device__ bool reduce_partials(double (&acc)[NQ], int nq, double* partials, double* results,
                                unsigned int* ticket, int tiles_per_inst) {
  __shared__ double red[NTHREADS / 32][NQ];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  (void)nq;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      double w = __shfl_down_sync(0xffffffffu, v, o);
      v = (q == Q_MAX) ? fmax(v, w) : v + w;
    }
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v = (q == Q_MAX) ? fmax(v, red[w][q]) : v + red[w][q];
    partials[(size_t)blockIdx.x * NQ + q] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const int ninst = gridDim.x / tiles_per_inst;
  for (int b = 0; b < ninst; ++b) {
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int i = threadIdx.x; i < tiles_per_inst; i += blockDim.x) {
      const double* p = partials + ((size_t)b * tiles_per_inst + i) * NQ;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double w = __ldcg(p + q);
        v[q] = (q == Q_MAX) ? fmax(v[q], w) : v[q] + w;
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = v[q];
      for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_down_sync(0xffffffffu, x, o);
        x = (q == Q_MAX) ? fmax(x, w) : x + w;
      }
      if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
      const int q = threadIdx.x;
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x = (q == Q_MAX) ? fmax(x, red[w][q]) : x + red[w][q];
      results[(size_t)b * NQ + q] = x;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence();
  __syncthreads();
  return true;
}

// ----------------------------------------------------------------- solver control
// Cayley coefficients of Theorem 3.3 for the current point and step tau, with
// the §4 renormalisation folded in as the scale s.
static __device__ void set_coef(Alg1Ctl* c) {
  const double t = c->tau, nX = c->nX, XG = c->XG, GG = c->GG, PP = c->PP;
  const double nxpp = nX * PP;                       // nX*GG - XG^2, cancellation-free
  const double den = 1.0 + t * t * nxpp;
  const double a = (1.0 + 2.0 * t * XG - t * t * nxpp) / den;
  const double b = -2.0 * t * nX / den;
  const double ny = a * a * nX + 2.0 * a * b * XG + b * b * GG;
  double s = 1.0 / sqrt(ny);
  if (!c->always_renorm && fabs(ny - 1.0) <= c->renorm_tol) s = 1.0;
  c->a = a;
  c->b = b;
  c->s = s;
}

// Algorithm 1 after an evaluation at the trial point: the nonmonotone test of
// Eq. NMLS-Armijo, backtracking, the reference value update (C, Q), Eq. crit1,
// and the next Barzilai-Borwein step of Eq. bb-1 (alternating tau^{k,1} on even
// k and tau^{k,2} on odd k; projected-gradient differences formed with the
// theta shift so that no large terms cancel).
static __device__ void alg1_control(Alg1Ctl* c, const double* r) {
  const double obj = (c->objective == 0) ? r[Q_E2] + c->alpha * r[Q_E4] : r[Q_E2] + r[Q_WX];
  const double nY = r[Q_NY], YG = r[Q_YG];
  c->obj_last = obj;
  c->nfe += 1;
  if (!isfinite(obj) || !isfinite(r[Q_GG]) || !(nY > 0.0)) {
    c->done = 1;
    c->status = 4;  // GPE_ENONFINITE
    return;
  }
  bool accept = true;
  if (c->phase != 0) {
    const double thr = c->C - c->rho1 * c->tau * c->res * c->res;
    accept = (obj <= thr) || (c->m >= c->max_bt);
  }
  if (!accept) {
    c->tau *= c->delta_bt;
    c->m += 1;
    c->accepted_last = 0;
    set_coef(c);
    return;
  }
  const double thY = YG / nY;
  const double dth = thY - (c->has_cur ? c->theta_c : c->theta_hint);
  double PPn = r[Q_Q] - 2.0 * dth * r[Q_QY] + dth * dth * nY;
  if (PPn < 0.0) PPn = 0.0;
  const double SS = r[Q_SS];
  const double SW = r[Q_SV] - dth * r[Q_SY];
  const double WW = r[Q_VV] - 2.0 * dth * r[Q_VY] + dth * dth * nY;
  if (c->has_cur) {
    const int oc = c->cur, op = c->prev, tr = c->trial;
    c->prev = oc;
    c->cur = tr;
    c->trial = op;
  } else {
    const int tr = c->trial;
    c->cur = tr;
    c->prev = (tr + 1) % 3;
    c->trial = (tr + 2) % 3;
  }
  c->F_cur = obj;
  c->theta_c = thY;
  c->nX = nY;
  c->XG = YG;
  c->GG = r[Q_GG];
  c->PP = PPn;
  c->res = nY * sqrt(PPn);
  c->smax = r[Q_MAX];
  if (c->phase == 0) {
    c->C = obj;
    c->Q = 1.0;
    c->k = 0;
    c->tau = c->tau0;
    c->phase = 1;
    c->has_cur = 1;
  } else {
    const double Qn = c->eta * c->Q + 1.0;
    c->C = (c->eta * c->Q * c->C + obj) / Qn;
    c->Q = Qn;
    c->k += 1;
    c->tau_last = c->tau;
    if (c->eps0 > 0.0 && r[Q_MAX] / c->tau <= c->eps0) { c->done = 1; c->status = 0; }
    double tb;
    if ((c->k & 1) == 0) tb = fabs(SW) > 0.0 ? SS / fabs(SW) : 1e20;
    else tb = WW > 0.0 ? fabs(SW) / WW : 1e20;
    if (!isfinite(tb)) tb = 1e20;
    tb = fmin(fmax(tb, 1e-20), 1e20);
    c->tau = 0.5 * tb;
  }
  c->m = 0;
  c->accepted_last = 1;
  if (c->res_tol > 0.0 && c->res <= c->res_tol) { c->done = 1; c->status = 0; }
  if (c->res_rel > 0.0 && c->res <= c->res_rel * fabs(thY)) { c->done = 1; c->status = 0; }
  // precision floor: no new smallest residual (by 10%) for stall_iters steps
  if (c->phase == 1 && (c->k == 0 || c->res < 0.9 * c->best_res)) {
    c->best_res = c->res;
    c->k_best = c->k;
  } else if (c->stall_iters > 0 && c->k - c->k_best >= c->stall_iters) {
    c->done = 1;
    c->status = 0;
  }
  if (!c->done && c->k >= c->max_iter) { c->done = 1; c->status = 5; }
  set_coef(c);
}

// Eq. TR-ratio with both reductions in difference form, Eq. update-X and
// Eq. tau-up (gamma1, gamma2 factors), on the ratio pass's sums.
static __device__ void rn_control(RNCtl* c, const double* r) {
  const double a = c->alpha, d = c->delta;
  const double ared = r[R_AXD] + 0.5 * r[R_DAD] + a * r[R_QD];
  const double pred = r[R_GD] + 0.5 * (r[R_DAD] + 4.0 * a * (r[R_X2D2] + 2.0 * r[R_R2])) + 0.5 * d * r[R_DD];
  double rho;
  if (fabs(pred) <= 1e-15 * fmax(fabs(c->F_k), 1.0)) rho = 1.0;
  else rho = ared / pred;
  c->ared = ared;
  c->pred = pred;
  c->rho = rho;
  c->dmax = r[Q_MAX];
  c->accepted = (rho >= c->eta1) ? 1 : 0;
  double nd = d;
  if (rho > c->eta2) nd = d / c->gamma1;
  else if (rho >= c->eta1) nd = d;
  else nd = d * c->gamma2;
  c->delta = fmin(fmax(nd, c->delta_min), c->delta_max);
}

// ----------------------------------------------------------------- pointwise epilogue
template <typename T, bool CPLX>
struct EpiCtx {
  using V = typename VT<T, CPLX>::V;
  V* out;
  const V* xc;
  const V* gc;
  const V* base;
  const V* gk;
  T nl, shift, lin_scale, th_c, delta;
};

template <typename T, bool CPLX, int EPI>
__device__ __forceinline__ void epilogue_point(const EpiCtx<T, CPLX>& E, long long gi,
                                               typename VT<T, CPLX>::V x,
                                               typename VT<T, CPLX>::V lin, double (&acc)[NQ]) {
  using V = typename VT<T, CPLX>::V;
  if (EPI == EPI_GRAD) {
    const T x2 = tre(x, x);
    if (E.out) E.out[gi] = lin + (E.nl * x2) * x;
    const double dx2 = dre(x, x);
    acc[0] += dre(x, lin);
    acc[1] += dx2 * dx2;
    acc[2] += dx2;
  } else if (EPI == EPI_HESS) {
    const V p = E.base[gi];
    const T p2 = tre(p, p);
    const T R = tre(p, x);
    E.out[gi] = lin + E.nl * (p2 * x + (T(2) * R) * p) + E.shift * x;
  } else if (EPI == EPI_F || EPI == EPI_W) {
    const V y = x;
    V g;
    if (EPI == EPI_F) {
      g = E.lin_scale * lin + (T(4) * E.nl * tre(y, y)) * y;
    } else {
      const V xk = E.base[gi];
      const V dd = y - xk;
      const T x2 = tre(xk, xk);
      const T R = tre(xk, dd);
      g = E.lin_scale * lin + (T(4) * E.nl * x2) * y + (T(8) * E.nl * R) * xk + E.delta * dd;
      const double dx2 = (double)x2, dR = dre(xk, dd), dd2 = dre(dd, dd);
      acc[Q_WX] += 4.0 * (double)E.nl * dx2 * dR + 2.0 * (double)E.nl * (dx2 * dd2 + 2.0 * dR * dR)
                   + 0.5 * (double)E.delta * dd2;
    }
    E.out[gi] = g;
    const double y2 = dre(y, y);
    acc[Q_E2] += dre(y, lin);
    acc[Q_E4] += y2 * y2;
    acc[Q_NY] += y2;
    acc[Q_YG] += dre(y, g);
    acc[Q_GG] += dre(g, g);
    const V q = g - E.th_c * y;
    acc[Q_Q] += dre(q, q);
    acc[Q_QY] += dre(q, y);
    const V xc = E.xc ? E.xc[gi] : vzero<V>();
    const V gc = E.gc ? E.gc[gi] : vzero<V>();
    const V s = y - xc;
    const V v = (g - gc) - E.th_c * s;
    const double s2 = dre(s, s);
    acc[Q_SS] += s2;
    acc[Q_SV] += dre(s, v);
    acc[Q_VV] += dre(v, v);
    acc[Q_VY] += dre(v, y);
    acc[Q_SY] += dre(s, y);
    acc[Q_MAX] = fmax(acc[Q_MAX], sqrt(s2));
  } else if (EPI == EPI_RATIO) {
    const V d = x;
    const V xk = E.base[gi];
    const V gk = E.gk[gi];
    const T x2 = tre(xk, xk);
    const V ax = gk - (T(4) * E.nl * x2) * xk;
    const V z = xk + d;
    const double dx2 = (double)x2, dR = dre(xk, d), dd2 = dre(d, d);
    acc[R_AXD] += dre(ax, d);
    acc[R_DAD] += 2.0 * dre(d, lin);
    acc[R_QD] += (2.0 * dR + dd2) * (dre(z, z) + dx2);
    acc[R_X2D2] += dx2 * dd2;
    acc[R_R2] += dR * dR;
    acc[R_DD] += dd2;
    acc[R_GD] += dre(gk, d);
    acc[Q_MAX] = fmax(acc[Q_MAX], sqrt(dd2));
  }
}

template <typename T, bool CPLX, int EPI>
__device__ __forceinline__ void make_ctx(EpiCtx<T, CPLX>& E, const PassData<T>& D) {
  using V = typename VT<T, CPLX>::V;
  E.out = (V*)D.out;
  E.xc = nullptr;
  E.gc = nullptr;
  E.base = (const V*)D.base;
  E.gk = (const V*)D.gk;
  E.nl = (T)D.nl;
  E.shift = (T)D.shift;
  E.lin_scale = (T)D.lin_scale;
  E.th_c = T(0);
  E.delta = T(0);
  if (D.ctl) {
    const Alg1Ctl* c = D.ctl;
    E.nl = (T)c->alpha;
    E.delta = (T)c->delta;
    if (D.use_slots) {
      E.out = (V*)D.gs[c->trial];
      if (c->has_cur) {
        E.xc = (const V*)D.xs[c->cur];
        E.gc = (const V*)D.gs[c->cur];
        E.th_c = (T)c->theta_c;
      } else {
        E.th_c = (T)c->theta_hint;
      }
    }
  }
  if (D.rn) E.nl = (T)D.rn->alpha;
}

template <typename T>
__device__ __forceinline__ void run_control(const PassData<T>& D) {
  if (threadIdx.x == 0) {
    if (D.control == 1) alg1_control(D.ctl, D.results);
    else if (D.control == 2) rn_control(D.rn, D.results);
  }
}

// ----------------------------------------------------------------- the axis pass
// Visit the data elements (line l, position j, global offset) of this CTA's
// tile with a coalesced thread mapping and no integer division: axis-0 lines
// are contiguous (tpl threads per line); strided lines are read as LB
// consecutive x positions per row.
template <typename T, typename Fn>
__device__ __forceinline__ void visit_tile(const PassGeom<T>& G, const long long* s_off, Fn&& fn) {
  const int nt = blockDim.x, tid = threadIdx.x;
  if (G.axis == 0) {
    const int lps = nt >> G.ltpl;
    for (int l = tid >> G.ltpl; l < G.LB; l += lps) {
      const long long off = s_off[l];
      if (off < 0) continue;
      for (int j = tid & (G.tpl - 1); j < G.len; j += G.tpl) fn(l, j, off + j);
    }
  } else {
    const int nval = G.LB * G.len;
    for (int f = tid; f < nval; f += nt) {
      const int l = f & (G.LB - 1);
      const int j = f >> G.logLB;
      const long long off = s_off[l];
      if (off < 0) continue;
      fn(l, j, off + (long long)j * G.stride);
    }
  }
}

template <typename T, bool CPLX, int EPI>
__global__ void __launch_bounds__(NTHREADS) k_pass(PassGeom<T> G, PassData<T> D) {
  using C = typename C2t<T>::type;
  using V = typename VT<T, CPLX>::V;
  if (D.ctl && D.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_off[MAXLB];
  __shared__ T s_rc[MAXLB];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + G.LC * G.F;
  const int inst = blockIdx.x / G.tiles;
  const int tile = blockIdx.x - inst * G.tiles;
  const int F = G.F;
  const int nt = blockDim.x, tid = threadIdx.x;

  const V* xin = (const V*)D.x;
  V* yst = nullptr;
  const V* xcur = nullptr;
  const V* gcur = nullptr;
  T sa = 0, sb = 0;
  if (D.use_slots) {
    const Alg1Ctl* c = D.ctl;
    xin = (const V*)D.xs[c->trial];
    if (D.step_on_load) {
      yst = (V*)D.xs[c->trial];
      xcur = (const V*)D.xs[c->cur];
      gcur = (const V*)D.gs[c->cur];
      sa = (T)(c->s * c->a);
      sb = (T)(c->s * c->b);
    }
  }
  const V* xsub = (const V*)D.xsub;

  for (int l = tid; l < G.LB; l += nt) {
    long long b;
    int ri;
    const bool ok = line_base(G, inst, tile, l, b, ri);
    s_off[l] = ok ? b : -1;
    if (G.rcoord) s_rc[l] = G.rcoord[ok ? ri : 0];
  }
  for (int i = tid; i < G.LC * F; i += nt) buf0[i] = mk<C>(0.0, 0.0);
  __syncthreads();

  visit_tile(G, s_off, [&](int l, int j, long long gi) {
    V v;
    if (yst) {
      v = sa * xcur[gi] + sb * gcur[gi];
      yst[gi] = v;
    } else {
      v = xin[gi];
      if (xsub) v = v - xsub[gi];
    }
    const int m = G.odd_ext ? j + 1 : j;
    if constexpr (CPLX) {
      C* row = buf0 + l * F;
      row[m] = v;
      if (G.odd_ext) row[F - m] = -v;
    } else {
      T* row = reinterpret_cast<T*>(buf0 + (l >> 1) * F);
      const int comp = l & 1;
      row[2 * m + comp] = v;
      if (G.odd_ext) row[2 * (F - m) + comp] = -v;
    }
  });
  __syncthreads();

  C* r = fft_lines<C>(buf0, buf1, F, G.LC, G.tw);
  // symbol multiply; the conjugation turns the next forward FFT into the inverse
  for (int t = tid; t < G.LC * F; t += nt) {
    const int c = t >> G.logF;
    const int m = t & (F - 1);
    const T lm = G.lam[m];
    T sym = G.c2 * lm * lm;
    if (G.rcoord) sym += G.c1 * s_rc[c] * lm;
    C v = r[t];
    v.x = sym * v.x;
    v.y = -sym * v.y;
    r[t] = v;
  }
  __syncthreads();
  C* o = fft_lines<C>(r, r == buf0 ? buf1 : buf0, F, G.LC, G.tw);

  EpiCtx<T, CPLX> E;
  if (EPI != EPI_ACC) make_ctx<T, CPLX, EPI>(E, D);
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  const V* accin = (const V*)D.acc_in;
  const long long ibase = inst * G.M;
  visit_tile(G, s_off, [&](int l, int j, long long gi) {
    const int m = G.odd_ext ? j + 1 : j;
    V kin;
    if constexpr (CPLX) {
      const C ov = o[l * F + m];
      kin.x = ov.x;
      kin.y = -ov.y;
    } else {
      const C ov = o[(l >> 1) * F + m];
      kin = (l & 1) ? -ov.y : ov.x;
    }
    if (EPI == EPI_ACC) {
      V a = kin;
      if (accin) a = accin[gi] + a;
      ((V*)D.out)[gi] = a;
      return;
    }
    V x;
    if (yst) x = yst[gi];
    else {
      x = xin[gi];
      if (xsub) x = x - xsub[gi];
    }
    V lin = kin + D.V[gi - ibase] * x;
    if (accin) lin = lin + accin[gi];
    epilogue_point<T, CPLX, EPI>(E, gi, x, lin, acc);
  });
  if (EPI == EPI_ACC || EPI == EPI_HESS || D.nq == 0) return;
  if (reduce_partials(acc, D.nq, D.partials, D.results, D.ticket, G.tiles)) run_control<T>(D);
}

// ----------------------------------------------------------------- finite differences
// H_lin of §2.1 per axis (3/5/7-point, zero Dirichlet values outside) with the
// central-difference rotation term, then the same epilogue as the spectral pass.
template <typename T, bool CPLX, int EPI>
__global__ void __launch_bounds__(NTHREADS) k_fd(FDGeom G, const T* __restrict__ rx, const T* __restrict__ ry,
                                                PassData<T> D) {
  using V = typename VT<T, CPLX>::V;
  if (D.ctl && D.ctl->done) return;
  const int inst = blockIdx.x / G.tiles;
  const int tb = blockIdx.x - inst * G.tiles;
  const V* xin = (const V*)D.x;
  if (D.use_slots) xin = (const V*)D.xs[D.ctl->trial];
  const V* xsub = (const V*)D.xsub;
  EpiCtx<T, CPLX> E;
  make_ctx<T, CPLX, EPI>(E, D);
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  const long long base = inst * G.M;
  const T a0 = (T)G.ih2[0], a1 = (T)G.ih2[1], a2 = (T)G.ih2[2];
  for (long long li = (long long)tb * blockDim.x + threadIdx.x; li < G.M; li += (long long)G.tiles * blockDim.x) {
    const int i0 = (int)(li % G.n0);
    const long long rest = li / G.n0;
    const int i1 = (int)(rest % G.n1);
    const int i2 = (int)(rest / G.n1);
    auto ld = [&](long long k) -> V {
      V v = xin[base + k];
      if (xsub) v = v - xsub[base + k];
      return v;
    };
    const V x = ld(li);
    V xm = i0 > 0 ? ld(li - 1) : vzero<V>();
    V xp = i0 < G.n0 - 1 ? ld(li + 1) : vzero<V>();
    V lin = (a0) * x - (T(0.5) * a0) * (xm + xp);
    V dx = xp - xm;
    V dy = vzero<V>();
    if (G.dim >= 2) {
      V ym = i1 > 0 ? ld(li - G.n0) : vzero<V>();
      V yp = i1 < G.n1 - 1 ? ld(li + G.n0) : vzero<V>();
      lin = lin + (a1) * x - (T(0.5) * a1) * (ym + yp);
      dy = yp - ym;
    }
    if (G.dim >= 3) {
      const long long s2 = (long long)G.n0 * G.n1;
      V zm = i2 > 0 ? ld(li - s2) : vzero<V>();
      V zp = i2 < G.n2 - 1 ? ld(li + s2) : vzero<V>();
      lin = lin + (a2) * x - (T(0.5) * a2) * (zm + zp);
    }
    if constexpr (CPLX) {
      if (G.omega != 0.0) {
        // -Omega L_z psi = i Omega (x d_y psi - y d_x psi)
        const T cx = (T)(G.omega * G.ih2c[0]), cy = (T)(G.omega * G.ih2c[1]);
        const T xv = rx[i0], yv = ry[i1];
        const V w = (xv * cy) * dy - (yv * cx) * dx;
        V iw;
        iw.x = -w.y;
        iw.y = w.x;
        lin = lin + iw;
      }
    }
    lin = lin + D.V[li] * x;
    epilogue_point<T, CPLX, EPI>(E, base + li, x, lin, acc);
  }
  if (EPI == EPI_HESS || D.nq == 0) return;
  if (reduce_partials(acc, D.nq, D.partials, D.results, D.ticket, G.tiles)) run_control<T>(D);
}

// ----------------------------------------------------------------- elementwise kernels
// Cayley step of Theorem 3.3 into the trial slot (FD path; the spectral path
// forms it while loading the first pass).
template <typename T, bool CPLX>
__global__ void k_step(void* const* xs, void* const* gs, const Alg1Ctl* c, long long n) {
  using V = typename VT<T, CPLX>::V;
  if (c->done) return;
  const V* X = (const V*)xs[c->cur];
  const V* Gv = (const V*)gs[c->cur];
  V* Y = (V*)xs[c->trial];
  const T a = (T)(c->s * c->a), b = (T)(c->s * c->b);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    Y[i] = a * X[i] + b * Gv[i];
}

// Per-instance sums |x|^2, Re conj(x) g, |g|^2 (g may be null).
template <typename T, bool CPLX>
__global__ void __launch_bounds__(NTHREADS) k_moments(const void* xv, const void* gv, long long M, int tiles,
                                                      double* partials, double* results, unsigned int* ticket) {
  using V = typename VT<T, CPLX>::V;
  const V* x = (const V*)xv;
  const V* g = (const V*)gv;
  const int inst = blockIdx.x / tiles;
  const int tb = blockIdx.x - inst * tiles;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  const long long base = inst * M;
  for (long long i = (long long)tb * blockDim.x + threadIdx.x; i < M; i += (long long)tiles * blockDim.x) {
    const V xi = x[base + i];
    acc[0] += dre(xi, xi);
    if (g) {
      const V gi = g[base + i];
      acc[1] += dre(xi, gi);
      acc[2] += dre(gi, gi);
    }
  }
  reduce_partials(acc, 3, partials, results, ticket, tiles);
}

// out_b = ca[b] * x_b + cb[b] * g_b  (g may be null)
template <typename T, bool CPLX>
__global__ void k_axpby(const void* xv, const void* gv, const double* coef, int stride_coef, long long M,
                        int nbatch, void* outv) {
  using V = typename VT<T, CPLX>::V;
  const V* x = (const V*)xv;
  const V* g = (const V*)gv;
  V* out = (V*)outv;
  const long long n = M * nbatch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / M);
    const T ca = (T)coef[(size_t)b * stride_coef + 0];
    V v = ca * x[i];
    if (g) v = v + (T)coef[(size_t)b * stride_coef + 1] * g[i];
    out[i] = v;
  }
}

// Coefficients for gpe_feasible_step from the moments (grid units in, unified
// units inside): X = sqrt(h) psi, G = 2 sqrt(h) hpsi.
static __global__ void k_step_coef(const double* mom, int nbatch, double h, double tau, double* coef) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbatch) return;
  const double* r = mom + (size_t)b * NQ;
  const double nX = h * r[0], XG = 2.0 * h * r[1], GG = 4.0 * h * r[2];
  double PP = GG - XG * XG / nX;
  if (PP < 0.0) PP = 0.0;
  const double t = tau, nxpp = nX * PP, den = 1.0 + t * t * nxpp;
  const double a = (1.0 + 2.0 * t * XG - t * t * nxpp) / den;
  const double bb = -2.0 * t * nX / den;
  const double ny = a * a * nX + 2.0 * a * bb * XG + bb * bb * GG;
  const double s = 1.0 / sqrt(ny);
  // psi_out = (s a X + s b G) / sqrt(h) = s a psi + 2 s b hpsi
  coef[(size_t)b * 2 + 0] = s * a;
  coef[(size_t)b * 2 + 1] = 2.0 * s * bb;
}

// scale to unit discrete norm: coef[b] = 1/sqrt(h * sum|x|^2)
static __global__ void k_norm_coef(const double* mom, int nbatch, double h, double* coef) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbatch) return;
  coef[b] = 1.0 / sqrt(h * mom[(size_t)b * NQ + 0]);
}

template <typename Ti, typename To>
__global__ void k_convert(const Ti* in, To* out, long long n, double scale) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (To)((double)in[i] * scale);
}

// fine -> coarse: values at the coarse nodes (Algorithm 3 initial guess).  The
// fine mesh is r = 2^k times finer; coarse index i sits at fine index r*i
// (periodic grids, node 0 shared) or r*(i+1)-1 (interior nodes of Dirichlet
// grids).
template <typename T, bool CPLX>
__global__ void k_inject(const void* fv, void* cv, int dim, int f0, int f1, int c0, int c1, int r, int dirichlet,
                         long long Mf, long long Mc, int nbatch) {
  using V = typename VT<T, CPLX>::V;
  const V* f = (const V*)fv;
  V* c = (V*)cv;
  const long long n = Mc * nbatch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / Mc);
    const long long li = i - b * Mc;
    const int i0 = (int)(li % c0);
    const long long rr = li / c0;
    const int i1 = (int)(rr % c1);
    const int i2 = (int)(rr / c1);
    auto fine = [&](int ic) -> long long { return dirichlet ? (long long)r * (ic + 1) - 1 : (long long)r * ic; };
    const long long j0 = fine(i0);
    const long long j1 = dim >= 2 ? fine(i1) : 0;
    const long long j2 = dim >= 3 ? fine(i2) : 0;
    c[i] = f[b * Mf + (j2 * f1 + j1) * f0 + j0];
  }
}

// Spectral prolongation along one axis (Algorithm 3 transfer): each line of
// length Nc (Fourier) or Nc-1 (sine, odd extension to 2Nc) is transformed,
// zero-padded to Ff = 2 Fc with the Fourier Nyquist coefficient split evenly
// between +-Nc/2, and transformed back on the fine line.  Lines are enumerated
// like the axis pass (coarse extents along this axis, current extents along the
// others).
template <typename T, bool CPLX>
__global__ void __launch_bounds__(NTHREADS) k_prolong_axis(PassGeom<T> G, int Ff, int logFf, const typename C2t<T>::type* twf,
                                                           int len_f, long long stride_f, long long ostride_f,
                                                           long long Mf, const void* inv, void* outv) {
  using C = typename C2t<T>::type;
  using V = typename VT<T, CPLX>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Fc = G.F;
  C* b0 = reinterpret_cast<C*>(smem_raw);
  C* b1 = b0 + G.LC * Ff;
  const int inst = blockIdx.x / G.tiles;
  const int tile = blockIdx.x - inst * G.tiles;
  const V* in = (const V*)inv;
  V* out = (V*)outv;
  for (int i = threadIdx.x; i < 2 * G.LC * Ff; i += blockDim.x) b0[i] = mk<C>(0.0, 0.0);
  __syncthreads();
  const int nval = G.LB * G.len;
  for (int f = threadIdx.x; f < nval; f += blockDim.x) {
    int l, j;
    if (G.axis == 0) { l = f / G.len; j = f - l * G.len; }
    else { j = f / G.LB; l = f - j * G.LB; }
    long long b;
    int ri;
    if (!line_base(G, inst, tile, l, b, ri)) continue;
    const V v = in[b + (long long)j * G.stride];
    const int m = G.odd_ext ? j + 1 : j;
    if constexpr (CPLX) {
      C* row = b0 + l * Fc;
      row[m] = v;
      if (G.odd_ext) row[Fc - m] = -v;
    } else {
      T* row = reinterpret_cast<T*>(b0 + (l >> 1) * Fc);
      row[2 * m + (l & 1)] = v;
      if (G.odd_ext) row[2 * (Fc - m) + (l & 1)] = -v;
    }
  }
  __syncthreads();
  // coarse forward FFTs use the first LC*Fc entries of b0/b1
  C* r = fft_lines<C>(b0, b1, Fc, G.LC, G.tw);
  C* dst = (r == b0) ? b1 : b0;
  for (int i = threadIdx.x; i < G.LC * Ff; i += blockDim.x) dst[i] = mk<C>(0.0, 0.0);
  __syncthreads();
  const T inv_n = T(1) / T(Fc);
  for (int t = threadIdx.x; t < G.LC * Fc; t += blockDim.x) {
    const int c = t / Fc;
    const int m = t - c * Fc;
    C v = r[t];
    v.x *= inv_n;
    v.y *= inv_n;
    // conjugate now so that the forward FFT below acts as the inverse
    v.y = -v.y;
    C* row = dst + c * Ff;
    if (m < Fc / 2) {
      row[m] = v;
    } else if (m > Fc / 2) {
      row[Ff - (Fc - m)] = v;
    } else {
      // Nyquist p = -Fc/2: zero for the sine extension; split for Fourier
      v.x *= T(0.5);
      v.y *= T(0.5);
      row[Fc / 2] = v;
      row[Ff - Fc / 2] = v;
    }
  }
  __syncthreads();
  C* o = fft_lines<C>(dst, r, Ff, G.LC, twf);
  const int nvf = G.LB * len_f;
  for (int f = threadIdx.x; f < nvf; f += blockDim.x) {
    int l, j;
    if (G.axis == 0) { l = f / len_f; j = f - l * len_f; }
    else { j = f / G.LB; l = f - j * G.LB; }
    // output line base on the fine-along-axis array
    long long bo;
    if (G.axis == 0) {
      long long rr = (long long)tile * G.LB + l;
      if (rr >= (long long)G.n1 * G.n2) continue;
      bo = inst * Mf + rr * len_f;
    } else {
      int oo = tile / G.xt;
      int x = (tile - oo * G.xt) * G.LB + l;
      if (x >= G.n0) continue;
      bo = inst * Mf + (long long)oo * ostride_f + x;
    }
    const int m = G.odd_ext ? j + 1 : j;
    V val;
    if constexpr (CPLX) {
      const C ov = o[l * Ff + m];
      val.x = ov.x;
      val.y = -ov.y;
    } else {
      const C ov = o[(l >> 1) * Ff + m];
      val = (l & 1) ? -ov.y : ov.x;
    }
    out[bo + (long long)j * stride_f] = val;
  }
  (void)logFf;
}

// FD prolongation along one axis: linear interpolation with zero Dirichlet ends.
template <typename T, bool CPLX>
__global__ void k_prolong_fd_axis(const void* inv, void* outv, int axis, int e0, int e1, int e2, int lc, int lf,
                                  long long Mc, long long Mf, int nbatch) {
  using V = typename VT<T, CPLX>::V;
  const V* in = (const V*)inv;
  V* out = (V*)outv;
  // output extents: along `axis` lf, others e*
  int o0 = e0, o1 = e1, o2 = e2;
  if (axis == 0) o0 = lf; else if (axis == 1) o1 = lf; else o2 = lf;
  const long long n = Mf * nbatch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / Mf);
    const long long li = i - b * Mf;
    int idx[3];
    idx[0] = (int)(li % o0);
    const long long r = li / o0;
    idx[1] = (int)(r % o1);
    idx[2] = (int)(r / o1);
    const int jf = idx[axis] + 1;                     // fine node number 1..lf
    const int jc = jf >> 1;                            // coarse node left of it
    const bool odd = jf & 1;
    auto at = [&](int node) -> V {                     // coarse node value (0 at the ends)
      if (node < 1 || node > lc) return vzero<V>();
      int id[3] = {idx[0], idx[1], idx[2]};
      id[axis] = node - 1;
      int c0 = e0, c1 = e1;
      if (axis == 0) c0 = lc; else if (axis == 1) c1 = lc;
      return in[b * Mc + ((long long)id[2] * c1 + id[1]) * c0 + id[0]];
    };
    V v;
    if (!odd) v = at(jc);
    else v = T(0.5) * (at(jc) + at(jc + 1));
    out[i] = v;
  }
}

}  // namespace gpe
