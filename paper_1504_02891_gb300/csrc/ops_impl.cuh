// ops_impl.cuh -- kernel templates of libgpe, instantiated per precision by
// ops_f32.cu and ops_f64.cu.  See gpe_kernels.cuh for the design summary.
#pragma once
#include <math.h>
#include <type_traits>
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

// ----------------------------------------------------------------- accumulators
// Per-thread sums of the float64 reductions.  In float32 kernels they are kept
// as unevaluated float pairs (hi + lo, Knuth two-sum), so no float64 unit is
// touched per element (GB300's float64 rate is a small fraction of float32);
// the pairs become float64 once per warp.  Float64 kernels accumulate in
// double.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void acc_zero(DF& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void acc_add(DF& a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b - bb);
  a.hi = s;
  a.lo += err;
}
__device__ __forceinline__ void acc_add(double& a, double b) { a += b; }
__device__ __forceinline__ void acc_add(float& a, float b) { a += b; }   // short float partials
__device__ __forceinline__ void acc_merge(DF& a, const DF& b) {
  acc_add(a, b.hi);
  a.lo += b.lo;
}
__device__ __forceinline__ void acc_merge(double& a, double b) { a += b; }
__device__ __forceinline__ double acc_value(const DF& a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ DF shfl_down(const DF& a, int o) {
  DF r;
  r.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
  r.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
  return r;
}
__device__ __forceinline__ double shfl_down(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
template <typename T> struct AccT { using type = double; };
template <> struct AccT<float> { using type = DF; };

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
__device__ C* fft_lines(C* a, C* b, int F, int nl, const C* __restrict__ tw, int P = 0) {
  if (P == 0) P = F;     // row pitch (>= F; padded rows avoid bank conflicts)
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
      const C* s = src + line * P + j;
      C* d = dst + line * P + (j - k) * R + k;
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

// ----------------------------------------------------------------- register-radix FFT
// Mixed-radix Stockham FFT (radix 16/8/4/2 butterflies in registers, 2-3
// shared-memory stages for F <= 1024) on nl lines of length F with row pitch P
// and padded indexing pidx(i) = i + i/16 (one spare slot every 16 elements),
// which keeps the stride-16 scatter of the first stage free of bank conflicts.
// Forward sign, unnormalised.  `post(line, m, v)` is applied to every output of
// the last stage (m = frequency index), e.g. the spectral symbol.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

template <typename C> __device__ __forceinline__ C cmulc(C v, double wr, double wi) {
  using T = decltype(v.x);
  C r;
  r.x = v.x * (T)wr - v.y * (T)wi;
  r.y = v.x * (T)wi + v.y * (T)wr;
  return r;
}
template <typename C> __device__ __forceinline__ C mul_mi(C v) {   // -i v
  C r;
  r.x = v.y;
  r.y = -v.x;
  return r;
}

// Complex sum and difference of the butterflies.  PK: in float32 one packed
// two-lane instruction each (a - b as fma(b, -1, a), exactly rounded); it
// trades issue slots for FMA-pipe throughput, which pays in the latency-bound
// cluster engine and not in the register-FFT line kernels (measured).
template <bool PK, typename C> __device__ __forceinline__ C cadd(C a, C b) {
  if constexpr (PK && std::is_same<C, float2>::value) return __fadd2_rn(a, b);
  else return a + b;
}
template <bool PK, typename C> __device__ __forceinline__ C csub(C a, C b) {
  if constexpr (PK && std::is_same<C, float2>::value) return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
  else return a - b;
}

template <typename C, bool PK = true> __device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd<PK>(t, b);
  b = csub<PK>(t, b);
}
template <typename C, bool PK = true> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C s02 = cadd<PK>(v0, v2), d02 = csub<PK>(v0, v2), s13 = cadd<PK>(v1, v3), d13 = csub<PK>(v1, v3);
  v0 = cadd<PK>(s02, s13);
  v2 = csub<PK>(s02, s13);
  v1 = d02 + mul_mi(d13);
  v3 = d02 - mul_mi(d13);
}
// cos(pi/8), sin(pi/8), sqrt(2)/2
#define GPE_C8 0.92387953251128675613
#define GPE_S8 0.38268343236508977173
#define GPE_R2 0.70710678118654752440
template <typename C, bool PK = true> __device__ __forceinline__ void dft8(C* v) {
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<C, PK>(e0, e1, e2, e3);
  dft4<C, PK>(o0, o1, o2, o3);
  o1 = cmulc(o1, GPE_R2, -GPE_R2);
  o2 = mul_mi(o2);
  o3 = cmulc(o3, -GPE_R2, -GPE_R2);
  v[0] = cadd<PK>(e0, o0); v[4] = csub<PK>(e0, o0);
  v[1] = cadd<PK>(e1, o1); v[5] = csub<PK>(e1, o1);
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = cadd<PK>(e3, o3); v[7] = csub<PK>(e3, o3);
}
template <typename C> __device__ __forceinline__ void dft16(C* v) {
  C e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft8(e);
  dft8(o);
  o[1] = cmulc(o[1], GPE_C8, -GPE_S8);
  o[2] = cmulc(o[2], GPE_R2, -GPE_R2);
  o[3] = cmulc(o[3], GPE_S8, -GPE_C8);
  o[4] = mul_mi(o[4]);
  o[5] = cmulc(o[5], -GPE_S8, -GPE_C8);
  o[6] = cmulc(o[6], -GPE_R2, -GPE_R2);
  o[7] = cmulc(o[7], -GPE_C8, -GPE_S8);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = cadd<true>(e[i], o[i]);
    v[i + 8] = csub<true>(e[i], o[i]);
  }
}
template <typename C, int R> __device__ __forceinline__ void dft_r(C* v) {
  if constexpr (R == 2) dft2(v[0], v[1]);
  else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8(v);
  else dft16(v);
}

// One Stockham stage of radix R = 2^LR.
template <typename C, int LR, typename Post>
__device__ __forceinline__ void fft_stage(const C* __restrict__ src, C* __restrict__ dst, int logF, int logNs, int nl,
                                          int P, const C* __restrict__ tw, bool last, Post& post) {
  constexpr int R = 1 << LR;
  const int lognb = logF - LR;
  const int nb = 1 << lognb;
  const int Ns = 1 << logNs;
  const int tot = nl << lognb;
  const int logtw = logF - logNs - LR;        // twiddle step F / (Ns R)
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int line = t >> lognb;
    const int j = t & (nb - 1);
    const int k = j & (Ns - 1);
    const C* s = src + line * P;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[pidx(j + (r << lognb))];
    if (Ns > 1) {
      // twiddles w^r, w = e^{-2 pi i k / (Ns R)}, from w, w^2, w^4, w^8 of the table
      const int e = k << logtw;
      C w[R];
      w[1] = tw[e];
      if constexpr (R >= 4) {
        w[2] = tw[2 * e];
        w[3] = cmul(w[1], w[2]);
      }
      if constexpr (R >= 8) {
        w[4] = tw[4 * e];
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
      }
      if constexpr (R >= 16) {
        w[8] = tw[8 * e];
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r]);
    }
    dft_r<C, R>(v);
    C* d = dst + line * P;
    const int mb = ((j - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = mb + (r << logNs);
      d[pidx(m)] = last ? post(line, m, v[r]) : v[r];
    }
  }
}

struct PostNone {
  template <typename C> __device__ __forceinline__ C operator()(int, int, C v) const { return v; }
};

// Radix schedule: ceil(logF/4) stages with the bits spread evenly (16x16 for
// 256, 8x8x8 for 512, 16x8x8 for 1024, ...).  Ends with a barrier.
template <typename C, typename Post>
__device__ C* fft_run(C* a, C* b, int logF, int nl, int P, const C* tw, Post post) {
  const int S = (logF + 3) >> 2;
  const int base = S ? logF / S : 0, extra = S ? logF % S : 0;
  C* src = a;
  C* dst = b;
  int logNs = 0;
  for (int st = 0; st < S; ++st) {
    const int lr = base + (st < extra ? 1 : 0);
    const bool last = st == S - 1;
    switch (lr) {
      case 1: fft_stage<C, 1>(src, dst, logF, logNs, nl, P, tw, last, post); break;
      case 2: fft_stage<C, 2>(src, dst, logF, logNs, nl, P, tw, last, post); break;
      case 3: fft_stage<C, 3>(src, dst, logF, logNs, nl, P, tw, last, post); break;
      default: fft_stage<C, 4>(src, dst, logF, logNs, nl, P, tw, last, post); break;
    }
    __syncthreads();
    C* t = src;
    src = dst;
    dst = t;
    logNs += lr;
  }
  return src;
}

// Asynchronous global -> shared copies (cp.async, sm_80+): the whole tile is in
// flight at once instead of one dependent load per thread and iteration.
template <typename V>
__device__ __forceinline__ void cp_async(V* dst_smem, const V* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(V) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
  } else if constexpr (sizeof(V) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ----------------------------------------------------------------- block reductions
// Partials are NQ slots of 8 bytes per CTA: float64 in float64 kernels, float
// pairs (hi, lo) in float32 kernels, so that a float32 reduction never touches
// the float64 pipe until its final NQ values.
__device__ __forceinline__ void df_max(DF& a, const DF& b) { a.hi = fmaxf(a.hi, b.hi); }

// Reduce the per-thread sums acc[0..nq) and the max slot over the block and
// write this CTA's partials to out[0..NQ) (slots >= nq other than Q_MAX as 0).
// Ends with a barrier.
template <typename A, typename M>
static __device__ void block_partial(A (&acc)[NQ], M amax2, int nq, double* out) {
  // amax2 is the largest |.|^2 of the CTA's points; a float32 run takes the
  // root in float32 (correctly rounded, the same value as the float64 root
  // rounded to float32; a float64 root costs ~0.3 us and the FP64 pipe)
  constexpr bool F32ACC = sizeof(A) == sizeof(DF) && !std::is_same<A, double>::value;
  const double acc_max = F32ACC ? 0.0 : sqrt((double)amax2);
  const float acc_max_f = F32ACC ? sqrtf((float)amax2) : 0.f;
  __shared__ A red[NTHREADS / 32][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    A v;
    if (q == Q_MAX) {
      if constexpr (F32ACC) {
        v.hi = acc_max_f;
        v.lo = 0.f;
        for (int o = 16; o > 0; o >>= 1) v.hi = fmaxf(v.hi, __shfl_down_sync(0xffffffffu, v.hi, o));
      } else {
        v = acc_max;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
      }
    } else if (q < nq) {
      v = acc[q];
      for (int o = 16; o > 0; o >>= 1) acc_merge(v, shfl_down(v, o));
    } else {
      acc_zero(v);
    }
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    A v = red[0][q];
    for (int w = 1; w < nw; ++w) {
      if constexpr (std::is_same<A, double>::value) v = (q == Q_MAX) ? fmax(v, red[w][q]) : v + red[w][q];
      else {
        if (q == Q_MAX) df_max(v, red[w][q]);
        else acc_merge(v, red[w][q]);
      }
    }
    reinterpret_cast<A*>(out)[q] = v;
  }
  __syncthreads();
}

// Fold the partials of `tiles` consecutive CTAs (fixed order) into float64
// out[0..NQ).  Called by one whole CTA.  Ends with a barrier.
template <typename A>
static __device__ void fold_partials(const double* partials, int tiles, int nq, double* out) {
  __shared__ A red[NTHREADS / 32][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  A v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc_zero(v[q]);
  const A* pp = reinterpret_cast<const A*>(partials);
  for (int i = threadIdx.x; i < tiles; i += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (q >= nq && q != Q_MAX) continue;
      A w;
      if constexpr (std::is_same<A, double>::value) {
        w = __ldcg(pp + (size_t)i * NQ + q);
        v[q] = (q == Q_MAX) ? fmax(v[q], w) : v[q] + w;
      } else {
        const float2 f = __ldcg(reinterpret_cast<const float2*>(pp + (size_t)i * NQ + q));
        w.hi = f.x;
        w.lo = f.y;
        if (q == Q_MAX) df_max(v[q], w);
        else acc_merge(v[q], w);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    A x = v[q];
    if (q < nq || q == Q_MAX) {
      for (int o = 16; o > 0; o >>= 1) {
        if constexpr (std::is_same<A, double>::value) {
          const double w = __shfl_down_sync(0xffffffffu, x, o);
          x = (q == Q_MAX) ? fmax(x, w) : x + w;
        } else {
          const DF w = shfl_down(x, o);
          if (q == Q_MAX) df_max(x, w);
          else acc_merge(x, w);
        }
      }
    } else {
      acc_zero(x);
    }
    if (lane == 0) red[warp][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    A x = red[0][q];
    for (int w = 1; w < nw; ++w) {
      if constexpr (std::is_same<A, double>::value) x = (q == Q_MAX) ? fmax(x, red[w][q]) : x + red[w][q];
      else {
        if (q == Q_MAX) df_max(x, red[w][q]);
        else acc_merge(x, red[w][q]);
      }
    }
    out[q] = acc_value(x);
  }
  __syncthreads();
}

// Several instances: warp w folds instances w, w + nwarps, ... (lanes stride
// over the tiles in a fixed order, then a fixed shuffle tree), so the final
// fold of a large batch is spread over the CTA's warps.  Ends with a barrier.
template <typename A>
static __device__ void fold_partials_warps(const double* partials, int tiles, int nq, double* results, int ninst) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const A* pp = reinterpret_cast<const A*>(partials);
  for (int b = warp; b < ninst; b += nw) {
    for (int q = 0; q < NQ; ++q) {
      if (q >= nq && q != Q_MAX) {
        if (lane == 0) results[(size_t)b * NQ + q] = 0.0;
        continue;
      }
      A x;
      acc_zero(x);
      for (int i = lane; i < tiles; i += 32) {
        const size_t o = ((size_t)b * tiles + i) * NQ + q;
        if constexpr (std::is_same<A, double>::value) {
          const double w = __ldcg(pp + o);
          x = (q == Q_MAX) ? fmax(x, w) : x + w;
        } else {
          const float2 f = __ldcg(reinterpret_cast<const float2*>(pp + o));
          A w;
          w.hi = f.x;
          w.lo = f.y;
          if (q == Q_MAX) df_max(x, w);
          else acc_merge(x, w);
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        if constexpr (std::is_same<A, double>::value) {
          const double w = __shfl_down_sync(0xffffffffu, x, o);
          x = (q == Q_MAX) ? fmax(x, w) : x + w;
        } else {
          const DF w = shfl_down(x, o);
          if (q == Q_MAX) df_max(x, w);
          else acc_merge(x, w);
        }
      }
      if (lane == 0) results[(size_t)b * NQ + q] = acc_value(x);
    }
  }
  __syncthreads();
}

// Block partial, then the last CTA to finish (atomic ticket) folds all
// partials per instance into results[inst][q].  Returns true in the last CTA.
template <typename A, typename M>
static __device__ bool reduce_partials(A (&acc)[NQ], M amax2, int nq, double* partials, double* results,
                                       unsigned int* ticket, int tiles_per_inst) {
  __shared__ int s_last;
  block_partial(acc, amax2, nq, partials + (size_t)blockIdx.x * NQ);
  __threadfence();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const int ninst = gridDim.x / tiles_per_inst;
  if (ninst == 1) fold_partials<A>(partials, tiles_per_inst, nq, results);
  else fold_partials_warps<A>(partials, tiles_per_inst, nq, results, ninst);
  if (threadIdx.x == 0) *ticket = 0u;
  __threadfence();
  __syncthreads();
  return true;
}

// Grid-wide barrier for a cooperative (co-resident) launch: arrival counter
// bar[0] and generation bar[1].  Every wait is bounded: after max_polls polls
// (2^22 by default, about a second) the CTA sets *err and returns false, and
// so does every CTA that later sees *err set.
static __device__ bool grid_barrier(unsigned int* bar, int* err, long long max_polls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = bar + 1;
    volatile int* verr = err;
    const unsigned int gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*vgen == gen) {
        if (*verr) { ok = 0; break; }
        if (++polls > max_polls) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (*verr) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ----------------------------------------------------------------- solver control
// The control of Algorithm 1 is one thread's serial chain of scalar
// operations once per trial; it runs in the arithmetic type R of the run.
// Float64 runs keep float64 (R = double).  Float32 runs (R = float) take their
// sums from float32 data, and use the step coefficients, theta and tau as
// float32 values, so float32 arithmetic loses nothing they can use, and on
// this hardware a float64 division or square root has a latency of hundreds
// of nanoseconds against tens for float32.  The block keeps float64 storage.

// Cayley coefficients of Theorem 3.3 for the current point and step tau, with
// the §4 renormalisation folded in as the scale s.
template <typename R, typename CT>
static __device__ __forceinline__ void set_coef(CT* c) {
  const R t = (R)c->tau, nX = (R)c->nX, XG = (R)c->XG, GG = (R)c->GG, PP = (R)c->PP;
  const R nxpp = nX * PP;                            // nX*GG - XG^2, cancellation-free
  R a, b, am1;
  if (sizeof(R) == 4 && t > R(1) && !(nxpp > R(0))) {
    // float32, A(X)X = 0 to float32 accuracy: the curve stays at X
    a = R(1);
    b = R(0);
    am1 = R(0);
  } else if (sizeof(R) == 4 && t > R(1)) {
    // float32: numerator and denominator divided by tau^2 (u = 1/tau), so
    // that steps up to the 1e20 clamp do not overflow
    const R u = R(1) / t;
    const R inv = R(1) / (u * u + nxpp);
    a = (u * u + R(2) * u * XG - nxpp) * inv;
    b = R(-2) * u * nX * inv;
    am1 = (R(2) * u * XG - R(2) * nxpp) * inv;
  } else {
    const R inv = R(1) / (R(1) + t * t * nxpp);      // one division for a, b and a - 1
    a = (R(1) + R(2) * t * XG - t * t * nxpp) * inv;
    b = R(-2) * t * nX * inv;
    am1 = (R(2) * t * XG - R(2) * t * t * nxpp) * inv;
  }
  // |Y|^2: float64 evaluates a^2 nX + 2ab XG + b^2 GG; in float32 those terms
  // cancel to rounding noise for large tau, so the identity |Y|^2 = |X|^2 of
  // Theorem 3.3 (the Cayley curve keeps the norm) is used instead
  const R ny = sizeof(R) == 4 ? nX : a * a * nX + R(2) * a * b * XG + b * b * GG;
  R s = R(1) / sqrt(ny);
  if (!c->always_renorm && fabs(ny - R(1)) <= (R)c->renorm_tol) s = R(1);
  c->a = a;
  c->b = b;
  c->s = s;
  c->am1 = am1;   // a - 1
}

// Algorithm 1 after an evaluation at the trial point: the nonmonotone test of
// Eq. NMLS-Armijo, backtracking, the reference value update (C, Q), Eq. crit1,
// and the next Barzilai-Borwein step of Eq. bb-1 (alternating tau^{k,1} on even
// k and tau^{k,2} on odd k, clamped), then the coefficients of the next trial.
// The objective value itself is kept in float64 (reported, never tested).
template <typename R, typename CT>
static __device__ __forceinline__ void alg1_control_impl(CT* c, const double* r) {
  const double obj = (c->objective == 0) ? r[Q_E2] + c->alpha * r[Q_E4] : r[Q_E2] + r[Q_WX];
  const R nY = (R)r[Q_NY], YG = (R)r[Q_YG];
  c->obj_last = obj;
  c->nfe += 1;
  if (!isfinite(obj) || !isfinite(r[Q_GG]) || !(nY > R(0))) {
    c->done = 1;
    c->status = 4;  // GPE_ENONFINITE
    return;
  }
  // Eq. NMLS-Armijo relative to the current point: with Cg = C - F(X_cur),
  // F(Y) <= C - rho1 tau res^2 reads dF <= Cg - rho1 tau res^2, dF formed
  // pointwise (no cancellation of two nearly equal objective values)
  const R dF = (R)r[Q_DF];
  const R tau = (R)c->tau, res = (R)c->res;
  bool accept = true;
  if (c->phase != 0) {
    const R thr = (R)c->Cg - (R)c->rho1 * tau * res * res;
    accept = (dF <= thr) || (c->m >= c->max_bt);
  }
  if (!accept) {
    c->tau = tau * (R)c->delta_bt;
    c->m += 1;
    c->accepted_last = 0;
    set_coef<R>(c);
    return;
  }
  const R thY = YG / nY;
  const R dth = thY - (R)(c->has_cur ? c->theta_c : c->theta_hint);
  R PPn = (R)r[Q_Q] - R(2) * dth * (R)r[Q_QY] + dth * dth * nY;
  if (PPn < R(0)) PPn = R(0);
  const R SS = (R)r[Q_SS];
  const R SW = (R)r[Q_SV] - dth * (R)r[Q_SY];
  const R WW = (R)r[Q_VV] - R(2) * dth * (R)r[Q_VY] + dth * dth * nY;
  if (c->two_slots) {
    const int oc = c->has_cur ? c->cur : 1 - c->trial;
    c->cur = c->trial;
    c->trial = oc;
    c->prev = oc;
  } else if (c->has_cur) {
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
  const R resn = nY * sqrt(PPn);
  c->F_cur = obj;
  c->theta_c = thY;
  c->nX = nY;
  c->XG = YG;
  c->GG = r[Q_GG];
  c->PP = PPn;
  c->res = resn;
  c->smax = r[Q_MAX];
  if (c->phase == 0) {
    c->Cg = 0.0;
    c->Q = 1.0;
    c->k = 0;
    c->tau = c->monotone ? c->alpha_hat : c->tau0;
    c->phase = 1;
    c->has_cur = 1;
  } else {
    if (c->monotone) {
      // Eq. Armijo1: the reference value is F(X^(k+1)) itself
      c->Cg = 0.0;
    } else {
      // C+ = (eta Q C + F(Y)) / Q+  =>  C+ - F(Y) = eta Q (Cg - dF) / Q+
      const R eta = (R)c->eta, Q = (R)c->Q;
      const R Qn = eta * Q + R(1);
      c->Cg = eta * Q * ((R)c->Cg - dF) / Qn;
      c->Q = Qn;
    }
    c->k += 1;
    c->tau_last = c->tau;
    if (c->eps0 > 0.0 && (R)r[Q_MAX] <= (R)c->eps0 * tau) { c->done = 1; c->status = 0; }   // Eq. crit1, tau > 0
    if (c->monotone) {
      c->tau = c->alpha_hat;   // Remark after Theorem 3.4: every search starts at alpha_hat
    } else {
      R tb;
      if ((c->k & 1) == 0) tb = fabs(SW) > R(0) ? SS / fabs(SW) : R(1e20);
      else tb = WW > R(0) ? fabs(SW) / WW : R(1e20);
      if (!isfinite(tb)) tb = R(1e20);
      tb = fmin(fmax(tb, R(1e-20)), R(1e20));
      c->tau = R(0.5) * tb;
    }
  }
  c->m = 0;
  c->accepted_last = 1;
  if (c->res_tol > 0.0 && resn <= (R)c->res_tol) { c->done = 1; c->status = 0; }
  if (c->res_rel > 0.0 && resn <= (R)c->res_rel * fabs(thY)) { c->done = 1; c->status = 0; }
  // precision floor: no new smallest residual (by 10%) for stall_iters steps
  if (c->phase == 1 && (c->k == 0 || resn < R(0.9) * (R)c->best_res)) {
    c->best_res = resn;
    c->k_best = c->k;
  } else if (c->stall_iters > 0 && c->k - c->k_best >= c->stall_iters) {
    // the precision floor: stopped, not converged (GPE_ENOCONV)
    c->done = 1;
    c->status = 5;
  }
  if (!c->done && c->k >= c->max_iter) { c->done = 1; c->status = 5; }
  set_coef<R>(c);
}

// The control on a register copy of the block and of the sums: the fields are
// read and written back once instead of one dependent shared- or global-memory
// access per use (the control is a single thread's serial chain).
template <typename R, typename CT>
static __device__ void alg1_control(CT* cp, const double* rp) {
  CT c = *cp;
  double r[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) r[q] = rp[q];
  alg1_control_impl<R>(&c, r);
  *cp = c;
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

// ----------------------------------------------------------------- coherent loads
// Inside a persistent launch, data written by other CTAs during the same launch
// must bypass the (non-coherent) L1: ld.global.cg.
// COH = 2: data that no thread writes during the launch, loaded through the
// read-only path (the compiler may then issue the loads ahead of earlier
// stores, which it must not do for plain loads of possibly aliasing arrays).
template <int COH, typename X> __device__ __forceinline__ X ldv(const X* p) {
  if constexpr (COH == 1) return __ldcg(p);
  else if constexpr (COH == 2) return __ldg(p);
  else return *p;
}
template <int COH, typename X> __device__ __forceinline__ X rdc(const X& r) {
  if constexpr (COH == 1) return *(const volatile X*)&r;
  else return r;
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
  T nl, shift, lin_scale, th_c, delta, thk;
};

template <typename T, bool CPLX, int EPI, int COH = 0, typename A>
__device__ __forceinline__ void epilogue_point(const EpiCtx<T, CPLX>& E, long long gi,
                                               typename VT<T, CPLX>::V x,
                                               typename VT<T, CPLX>::V lin, A (&acc)[NQ], T& amax) {
  using V = typename VT<T, CPLX>::V;
  if (EPI == EPI_GRAD) {
    const T x2 = tre(x, x);
    if (E.out) E.out[gi] = lin + (E.nl * x2) * x;
    acc_add(acc[0], tre(x, lin));
    acc_add(acc[1], x2 * x2);
    acc_add(acc[2], x2);
  } else if (EPI == EPI_HESS) {
    const V p = ldv<COH>(E.base + gi);
    const T p2 = tre(p, p);
    const T R = tre(p, x);
    E.out[gi] = lin + E.nl * (p2 * x + (T(2) * R) * p) + E.shift * x;
  } else if (EPI == EPI_F || EPI == EPI_W) {
    const V y = x;
    V g;
    if (EPI == EPI_F) {
      g = E.lin_scale * lin + (T(4) * E.nl * tre(y, y)) * y;
    } else {
      const V xk = ldv<COH>(E.base + gi);
      const V dd = y - xk;
      const T x2 = tre(xk, xk);
      const T R = tre(xk, dd);
      g = E.lin_scale * lin + (T(4) * E.nl * x2) * y + (T(8) * E.nl * R) * xk + E.delta * dd;
      const T d2 = tre(dd, dd);
      acc_add(acc[Q_WX], T(4) * E.nl * x2 * R + T(2) * E.nl * (x2 * d2 + T(2) * R * R) + T(0.5) * E.delta * d2);
    }
    E.out[gi] = g;
    const T y2 = tre(y, y);
    acc_add(acc[Q_E2], tre(y, lin));
    acc_add(acc[Q_E4], y2 * y2);
    acc_add(acc[Q_NY], y2);
    acc_add(acc[Q_YG], tre(y, g));
    acc_add(acc[Q_GG], tre(g, g));
    const V q = g - E.th_c * y;
    acc_add(acc[Q_Q], tre(q, q));
    acc_add(acc[Q_QY], tre(q, y));
    const V xc = E.xc ? ldv<COH>(E.xc + gi) : vzero<V>();
    const V gc = E.gc ? ldv<COH>(E.gc + gi) : vzero<V>();
    const V s = y - xc;
    const V v = (g - gc) - E.th_c * s;
    const T s2 = tre(s, s);
    acc_add(acc[Q_SS], s2);
    acc_add(acc[Q_SV], tre(s, v));
    acc_add(acc[Q_VV], tre(v, v));
    acc_add(acc[Q_VY], tre(v, y));
    acc_add(acc[Q_SY], tre(s, y));
    // objective(y) - objective(x_c) by the trapezoid rule on the theta-shifted
    // gradients (q + q_c = 2q - v); exact for the quadratic part, the quartic
    // term of F adds -alpha Re<s, y + x_c> |s|^2.  The dropped real multiple
    // of y + x_c changes the objective only off the unit sphere.
    T df = tre(s, q) - T(0.5) * tre(s, v);
    if (EPI == EPI_F) df -= E.nl * tre(s, y + xc) * s2;
    acc_add(acc[Q_DF], df);
    amax = fmax(amax, s2);
  } else if (EPI == EPI_WS) {
    // difference form (the unknown y is D = X - X^k): G^ = P_k + H_k D +
    // (delta - theta_k) D, objective Re<P_k, D> + theta_k Re<X^k, D> +
    // 1/2 Re<D, H_k D> + delta/2 |D|^2, moments of X = X^k + D
    const V y = x;
    const V xk = ldv<COH>(E.base + gi);
    const V pk = ldv<COH>(E.gk + gi);
    const T x2 = tre(xk, xk), R = tre(xk, y);
    const V hD = E.lin_scale * lin + (T(4) * E.nl) * (x2 * y + (T(2) * R) * xk);
    const V gh = pk + hD + (E.delta - E.thk) * y;
    E.out[gi] = gh;
    const V X = xk + y;
    acc_add(acc[Q_WX], tre(pk, y) + E.thk * R + T(0.5) * tre(y, hD) + T(0.5) * E.delta * tre(y, y));
    acc_add(acc[Q_NY], tre(X, X));
    acc_add(acc[Q_YG], tre(X, gh));
    acc_add(acc[Q_GG], tre(gh, gh));
    const V q = gh - E.th_c * X;
    acc_add(acc[Q_Q], tre(q, q));
    acc_add(acc[Q_QY], tre(q, X));
    const V yc = E.xc ? ldv<COH>(E.xc + gi) : vzero<V>();
    const V gc = E.gc ? ldv<COH>(E.gc + gi) : vzero<V>();
    const V s = y - yc;
    const V v = (gh - gc) - E.th_c * s;
    const T s2 = tre(s, s);
    acc_add(acc[Q_SS], s2);
    acc_add(acc[Q_SV], tre(s, v));
    acc_add(acc[Q_VV], tre(v, v));
    acc_add(acc[Q_VY], tre(v, X));
    acc_add(acc[Q_SY], tre(s, X));
    acc_add(acc[Q_DF], tre(s, q) - T(0.5) * tre(s, v));   // the model is quadratic: trapezoid exact
    amax = fmax(amax, s2);
  } else if (EPI == EPI_RATIO) {
    const V d = x;
    const V xk = ldv<COH>(E.base + gi);
    const V gk = ldv<COH>(E.gk + gi);
    const T x2 = tre(xk, xk);
    const V ax = gk - (T(4) * E.nl * x2) * xk;
    const V z = xk + d;
    const T R = tre(xk, d), d2 = tre(d, d);
    acc_add(acc[R_AXD], tre(ax, d));
    acc_add(acc[R_DAD], T(2) * tre(d, lin));
    acc_add(acc[R_QD], (T(2) * R + d2) * (tre(z, z) + x2));
    acc_add(acc[R_X2D2], x2 * d2);
    acc_add(acc[R_R2], R * R);
    acc_add(acc[R_DD], d2);
    acc_add(acc[R_GD], tre(gk, d));
    amax = fmax(amax, d2);
  }
}

template <typename T, bool CPLX, int EPI, int COH = 0>
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
    E.nl = (T)rdc<COH>(c->alpha);
    E.delta = (T)rdc<COH>(c->delta);
    if (D.use_slots) {
      E.out = (V*)D.gs[rdc<COH>(c->trial)];
      if (rdc<COH>(c->has_cur)) {
        E.xc = (const V*)D.xs[rdc<COH>(c->cur)];
        E.gc = (const V*)D.gs[rdc<COH>(c->cur)];
        E.th_c = (T)rdc<COH>(c->theta_c);
      } else {
        E.th_c = (T)rdc<COH>(c->theta_hint);
      }
    }
  }
  E.thk = D.ctl ? (T)rdc<COH>(D.ctl->theta_ref) : T(0);
  if (D.rn) E.nl = (T)D.rn->alpha;
}

template <typename T>
__device__ __forceinline__ void run_control(const PassData<T>& D) {
  if (threadIdx.x == 0) {
    if (D.control == 1) alg1_control<T>(D.ctl, D.results);
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

// One tile of one axis pass: load (asynchronous copies, or L2-coherent loads
// inside a persistent launch), forward FFT with the fused symbol, inverse FFT,
// epilogue into acc/amax.  blk = instance * tiles + tile.  Ends with a barrier.
template <typename T, bool CPLX, int EPI, bool COH, typename A>
__device__ __forceinline__ void pass_tile(const PassGeom<T>& G, const PassData<T>& D, int blk,
                                          unsigned char* smem_raw, long long* s_off, T* s_rc, A (&acc)[NQ],
                                          T& amax,
                                          const typename C2t<T>::type* tw_pre = nullptr) {
  using C = typename C2t<T>::type;
  using V = typename VT<T, CPLX>::V;
  const int F = G.F, Pt = G.P;
  const int nt = blockDim.x, tid = threadIdx.x;
  const int inst = blk / G.tiles;
  const int tile = blk - inst * G.tiles;

  // operands: src0 (input, or X_cur for the Cayley step), src1 (x_sub or G_cur), acc_in
  const V* xin = (const V*)D.x;
  V* yst = nullptr;
  const V* src1 = (const V*)D.xsub;
  T sa = 0, sb = 0;
  if (D.use_slots) {
    const Alg1Ctl* c = D.ctl;
    const int trial = rdc<COH>(c->trial);
    xin = (const V*)D.xs[trial];
    if (D.step_on_load) {
      const int cur = rdc<COH>(c->cur);
      yst = (V*)D.xs[trial];
      xin = (const V*)D.xs[cur];
      src1 = (const V*)D.gs[cur];
      const double cs = rdc<COH>(c->s);
      sa = (T)(cs * rdc<COH>(c->a));
      sb = (T)(cs * rdc<COH>(c->b));
    }
  }
  const V* accin = (const V*)D.acc_in;
  const int tile_n = G.LB * G.len;
  C* tw_s = reinterpret_cast<C*>(smem_raw);
  C* buf0 = tw_s + F;
  C* buf1 = buf0 + G.LC * Pt;
  V* st0 = reinterpret_cast<V*>(buf1 + G.LC * Pt);
  V* st1 = st0 + tile_n;
  V* st2 = st1 + (src1 ? tile_n : 0);
  // potential of the tile (final passes only), staged with the other operands
  T* stv = reinterpret_cast<T*>(st2 + (accin ? tile_n : 0));
  const bool want_v = EPI != EPI_ACC;
  const long long vbase = (long long)inst * G.M;

  for (int l = tid; l < G.LB; l += nt) {
    long long b;
    int ri;
    const bool ok = line_base(G, inst, tile, l, b, ri);
    s_off[l] = ok ? b : -1;
    if (G.rcoord) s_rc[l] = G.rcoord[ok ? ri : 0];
  }
  // twiddle table (read-only): preloaded by the caller, or an asynchronous
  // copy, or plain loads when the tile loads below are not asynchronous
  if (!tw_pre) {
    for (int i = tid; i < F; i += nt) {
      if constexpr (COH) tw_s[i] = G.tw[i];
      else cp_async(tw_s + i, G.tw + i);
    }
  }
  const C* twx = tw_pre ? tw_pre : tw_s;
  __syncthreads();
  // the whole tile (and the operands the epilogue needs) in flight at once
  visit_tile(G, s_off, [&](int l, int j, long long gi) {
    const int q = G.axis == 0 ? l * G.len + j : j * G.LB + l;
    if constexpr (COH) {
      st0[q] = __ldcg(xin + gi);
      if (src1) st1[q] = __ldcg(src1 + gi);
      if (accin) st2[q] = __ldcg(accin + gi);
      if (want_v) stv[q] = D.V[gi - vbase];
    } else {
      cp_async(st0 + q, xin + gi);
      if (src1) cp_async(st1 + q, src1 + gi);
      if (accin) cp_async(st2 + q, accin + gi);
      if (want_v) cp_async(stv + q, D.V + (gi - vbase));
    }
  });
  for (int i = tid; i < G.LC * Pt; i += nt) buf0[i] = mk<C>(0.0, 0.0);
  if constexpr (!COH) cp_async_wait_all();
  __syncthreads();

  visit_tile(G, s_off, [&](int l, int j, long long gi) {
    const int q = G.axis == 0 ? l * G.len + j : j * G.LB + l;
    V v = st0[q];
    if (src1) {
      v = yst ? sa * v + sb * st1[q] : v - st1[q];
      st0[q] = v;
      if (yst) yst[gi] = v;
    }
    const int m = G.odd_ext ? j + 1 : j;
    if constexpr (CPLX) {
      C* row = buf0 + l * Pt;
      row[pidx(m)] = v;
      if (G.odd_ext) row[pidx(F - m)] = -v;
    } else {
      T* row = reinterpret_cast<T*>(buf0 + (l >> 1) * Pt);
      const int comp = l & 1;
      row[2 * pidx(m) + comp] = v;
      if (G.odd_ext) row[2 * pidx(F - m) + comp] = -v;
    }
  });
  __syncthreads();

  // forward FFT with the line symbol (and the conjugation that turns the
  // next forward FFT into the inverse) fused into its last stage
  const T c2 = G.c2, c1 = G.c1, dlam = G.dlam;
  const bool rot = G.rcoord != nullptr;
  auto symbol = [&](int line, int m, C v) -> C {
    const T lm = dlam * (T)(m < (F >> 1) ? m : m - F);
    T sym = c2 * lm * lm;
    if (rot) sym += c1 * s_rc[line] * lm;
    C r;
    r.x = sym * v.x;
    r.y = -sym * v.y;
    return r;
  };
  C* r = fft_run<C>(buf0, buf1, G.logF, G.LC, Pt, twx, symbol);
  C* o = fft_run<C>(r, r == buf0 ? buf1 : buf0, G.logF, G.LC, Pt, twx, PostNone());

  EpiCtx<T, CPLX> E;
  if (EPI != EPI_ACC) make_ctx<T, CPLX, EPI, COH>(E, D);
  const long long ibase = inst * G.M;
  visit_tile(G, s_off, [&](int l, int j, long long gi) {
    const int q = G.axis == 0 ? l * G.len + j : j * G.LB + l;
    const int m = G.odd_ext ? j + 1 : j;
    V kin;
    if constexpr (CPLX) {
      const C ov = o[l * Pt + pidx(m)];
      kin.x = ov.x;
      kin.y = -ov.y;
    } else {
      const C ov = o[(l >> 1) * Pt + pidx(m)];
      kin = (l & 1) ? -ov.y : ov.x;
    }
    if (accin) kin = kin + st2[q];
    if (EPI == EPI_ACC) {
      ((V*)D.out)[gi] = kin;
      return;
    }
    const V x = st0[q];
    const V lin = kin + stv[q] * x;
    epilogue_point<T, CPLX, EPI, COH>(E, gi, x, lin, acc, amax);
  });
  __syncthreads();
}

template <typename T, bool CPLX, int EPI>
__global__ void __launch_bounds__(NTHREADS) k_pass(PassGeom<T> G, PassData<T> D) {
  if (D.ctl && D.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_off[MAXLB];
  __shared__ T s_rc[MAXLB];
  using A = typename AccT<T>::type;
  A acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
  T amax = T(0);
  pass_tile<T, CPLX, EPI, false>(G, D, blockIdx.x, smem_raw, s_off, s_rc, acc, amax);
  if (EPI == EPI_ACC || EPI == EPI_HESS || D.nq == 0) return;
  if (reduce_partials(acc, amax, D.nq, D.partials, D.results, D.ticket, G.tiles)) run_control<T>(D);
}

// One launch runs a whole Algorithm 1 run (until the control block says done).
// Every iteration executes the axis passes over all tiles (CTAs loop over
// tiles) separated by bounded grid barriers; then EVERY CTA folds the last
// pass's tile partials in the same fixed order and runs the step-size control
// on its own shared-memory copy of the control block, so all CTAs hold
// bit-identical state without a third barrier.  CTA 0 writes the state back.
// The slot pointers and the twiddle tables stay in shared memory for the whole
// launch.  Must be launched cooperatively (all CTAs co-resident).
template <typename T, bool CPLX, int EPI>
__global__ void __launch_bounds__(NTHREADS) k_alg1_persist(PersistArgs<T> P) {
  using C = typename C2t<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_off[MAXLB];
  __shared__ T s_rc[MAXLB];
  __shared__ Alg1Ctl s_ctl;
  __shared__ void* s_xs[3];
  __shared__ void* s_gs[3];
  __shared__ double s_res[NQ];
  using A = typename AccT<T>::type;
  // twiddle tables of all axes at the front of dynamic shared memory
  C* s_tw[3] = {nullptr, nullptr, nullptr};
  {
    C* tp = reinterpret_cast<C*>(smem_raw);
    for (int a = 0; a < P.dim; ++a) {
      s_tw[a] = tp;
      for (int i = threadIdx.x; i < P.G[a].F; i += blockDim.x) tp[i] = P.G[a].tw[i];
      tp += P.G[a].F;
    }
  }
  unsigned char* work = smem_raw + P.tw_bytes;
  if (threadIdx.x == 0) {
    s_ctl = *P.D.ctl;
    for (int i = 0; i < 3; ++i) {
      s_xs[i] = P.D.xs[i];
      s_gs[i] = P.D.gs[i];
    }
  }
  __syncthreads();
  PassData<T> D0 = P.D;
  D0.ctl = &s_ctl;
  D0.xs = s_xs;
  D0.gs = s_gs;
  auto stamp = [&](int loop, int k) {
    if (P.dbg && blockIdx.x == 0 && threadIdx.x == 0 && loop < P.dbg_n) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      P.dbg[loop * 4 + k] = t;
    }
  };
  auto writeback = [&]() {
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.D.ctl = s_ctl;
  };
  for (int loop = 0; loop < P.max_loops; ++loop) {
    if (s_ctl.done) {
      writeback();
      return;
    }
    stamp(loop, 0);
    for (int a = 0; a < P.dim; ++a) {
      const bool last = a == P.dim - 1;
      PassData<T> Da = D0;
      Da.step_on_load = a == 0 ? 1 : 0;
      Da.acc_in = a > 0 ? P.acc : nullptr;
      if (!last) {
        Da.out = P.acc;
        Da.nq = 0;
      }
      for (int blk = blockIdx.x; blk < P.blocks[a]; blk += gridDim.x) {
        A acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
        T amax = T(0);
        if (!last) {
          pass_tile<T, CPLX, EPI_ACC, true>(P.G[a], Da, blk, work, s_off, s_rc, acc, amax, s_tw[a]);
        } else {
          pass_tile<T, CPLX, EPI, true>(P.G[a], Da, blk, work, s_off, s_rc, acc, amax, s_tw[a]);
          block_partial(acc, amax, NQ, P.D.partials + (size_t)blk * NQ);
        }
      }
      if (!grid_barrier(P.bar, P.err, P.max_polls)) {
        writeback();
        return;
      }
      stamp(loop, 1 + (a < 1 ? a : 1));
    }
    fold_partials<A>(P.D.partials, P.blocks[P.dim - 1], NQ, s_res);
    if (threadIdx.x == 0) alg1_control<T>(&s_ctl, s_res);
    __syncthreads();
    stamp(loop, 3);
  }
  writeback();
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
  using A = typename AccT<T>::type;
  A acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
  T amax = T(0);
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
    epilogue_point<T, CPLX, EPI>(E, base + li, x, lin, acc, amax);
  }
  if (EPI == EPI_HESS || D.nq == 0) return;
  if (reduce_partials(acc, amax, D.nq, D.partials, D.results, D.ticket, G.tiles)) run_control<T>(D);
}

// ----------------------------------------------------------------- elementwise kernels
// Cayley step of Theorem 3.3 into the trial slot (FD path; the spectral path
// forms it while loading the first pass).
template <typename T, bool CPLX>
__global__ void k_step(void* const* xs, void* const* gs, const Alg1Ctl* c, long long n, const void* xkv) {
  using V = typename VT<T, CPLX>::V;
  if (c->done) return;
  const V* X = (const V*)xs[c->cur];
  const V* Gv = (const V*)gs[c->cur];
  V* Y = (V*)xs[c->trial];
  const T a = (T)(c->s * c->a), b = (T)(c->s * c->b);
  if (xkv) {
    // difference form: D+ = (a - 1) X^k + a D + b G^ (no renormalisation)
    const V* xk = (const V*)xkv;
    const T am1 = (T)c->am1, a1 = (T)c->a, b1 = (T)c->b;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      Y[i] = am1 * xk[i] + a1 * X[i] + b1 * Gv[i];
    return;
  }
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
  using A = typename AccT<T>::type;
  A acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
  const long long base = inst * M;
  for (long long i = (long long)tb * blockDim.x + threadIdx.x; i < M; i += (long long)tiles * blockDim.x) {
    const V xi = x[base + i];
    acc_add(acc[0], tre(xi, xi));
    if (g) {
      const V gi = g[base + i];
      acc_add(acc[1], tre(xi, gi));
      acc_add(acc[2], tre(gi, gi));
    }
  }
  reduce_partials(acc, T(0), 3, partials, results, ticket, tiles);
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

// Shifted subproblem inputs in float32: X^k and P_k = G_k - theta_k X^k
// (interleaved real components; theta_k is real).
static __global__ void k_to_shifted_f32(const double* xk, const double* gk, double th, float* xk32, float* pk32,
                                 long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = xk[i];
    xk32[i] = (float)x;
    pk32[i] = (float)(gk[i] - th * x);
  }
}

// Z = X^k + D (D from the float32 subproblem), float64.
static __global__ void k_add_f32_to_f64(const double* xk, const float* d, double* z, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = xk[i] + (double)d[i];
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
