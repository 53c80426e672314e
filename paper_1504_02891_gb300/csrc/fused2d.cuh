// fused2d.cuh -- the operator on square 2D Fourier grids in float32 as ONE
// persistent kernel of independent warps (the paper's Eq. fftp36 / fftp35
// transforms with the line symbols of Eq. energy-discrete-FP, then the
// pointwise terms and reductions of Lemma 3.1).
//
// Line transform.  A line of F = TPL x PPT points belongs to TPL lanes of one
// warp (TPL = 8, 16 or 32; 32 / TPL lines per warp); lane j holds the points
// j + TPL s, s = 0..PPT-1.  With n = j + TPL s and k = k2 + PPT k1,
//   X[k2 + PPT k1] = sum_j W_TPL^{j k1} ( W_F^{j k2} sum_s x[j + TPL s] W_PPT^{s k2} ),
// so a transform is: a PPT-point DFT in each lane's registers, the twiddles
// W_F^{j k2} (a k2-major table in shared memory: one conflict-free load each),
// one exchange through the warp's shared-memory rows (lane j's value k2 to
// slot k2 TPL + (j ^ (k2 mod TPL)), conflict-free on both sides), and
// PPT / TPL TPL-point DFTs per lane.  Lane u then holds X[u + TPL s'] -- the
// same register order as the input -- so loads, the symbol multiply and
// stores need no further exchange, and a line waits only for its own warp.
// The inverse transform is the forward one applied to the conjugate.
//
// Scheduling.  The x-part of a point needs T_y psi of its whole row, so each
// instance is done in two kinds of tasks: y-tasks (32 / TPL columns each:
// T_y into the output array) and x-tasks (32 / TPL rows each: T_x, the
// pointwise epilogue, per-task partial sums).  Warps take tasks in a fixed
// order from an atomic counter -- the y-tasks of instance b, then the y-tasks
// of b + 1 and the x-tasks of b, and so on -- and an x-task of b starts once
// every y-task of b has finished (a per-instance counter; the wait is
// bounded).  Every task a warp waits for was handed out earlier to a running
// warp, so the waits always end.  A few instances are in flight at a time,
// so T_y psi is read back from L2 and psi is read from DRAM once: the DRAM
// traffic of an application is its algorithmic bytes (read psi, write the
// output).  The last x-task of an instance folds that instance's task
// partials in task order (deterministic) and, in the solver, runs the
// control; the last warp to leave resets the counters for the next launch.
#pragma once
#include "ops_launch.cuh"

namespace gpe {

constexpr int FUSED_THREADS = 128;   // 4 independent warps per CTA
#ifndef FUSED_SKEW
#define FUSED_SKEW 2
#endif
// resident CTAs per SM the register budget is sized for: 128 registers per
// lane up to 256-point lines; 255 at 512 and 1024 (32 complex values per
// lane; measured: faster than 168 registers with three CTAs per SM)
__host__ __device__ constexpr int fused_minb(int lf) { return lf <= 8 ? 4 : 2; }

// cos(pi/16), sin(pi/16), cos(3 pi/16), sin(3 pi/16)
#define GPE_C16 0.98078528040323044913
#define GPE_S16 0.19509032201612826785
#define GPE_C316 0.83146961230254523708
#define GPE_S316 0.55557023301960222474

// 32-point DFT in registers, natural order in and out (two 16-point DFTs of
// the even and odd samples, twiddles W_32^k = e^{-2 pi i k / 32}).
template <typename C, bool PK> __device__ __forceinline__ void dft32(C* v) {
  C e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16(e);
  dft16(o);
  o[1] = cmulc(o[1], GPE_C16, -GPE_S16);
  o[2] = cmulc(o[2], GPE_C8, -GPE_S8);
  o[3] = cmulc(o[3], GPE_C316, -GPE_S316);
  o[4] = cmulc(o[4], GPE_R2, -GPE_R2);
  o[5] = cmulc(o[5], GPE_S316, -GPE_C316);
  o[6] = cmulc(o[6], GPE_S8, -GPE_C8);
  o[7] = cmulc(o[7], GPE_S16, -GPE_C16);
  o[8] = mul_mi(o[8]);
  o[9] = cmulc(o[9], -GPE_S16, -GPE_C16);
  o[10] = cmulc(o[10], -GPE_S8, -GPE_C8);
  o[11] = cmulc(o[11], -GPE_S316, -GPE_C316);
  o[12] = cmulc(o[12], -GPE_R2, -GPE_R2);
  o[13] = cmulc(o[13], -GPE_C316, -GPE_S316);
  o[14] = cmulc(o[14], -GPE_C8, -GPE_S8);
  o[15] = cmulc(o[15], -GPE_C16, -GPE_S16);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = cadd<PK>(e[i], o[i]);
    v[i + 16] = csub<PK>(e[i], o[i]);
  }
}

template <typename C, int N, bool PK> __device__ __forceinline__ void dft_n(C* v) {
  if constexpr (N == 8) dft8<C, PK>(v);
  else if constexpr (N == 16) dft16(v);
  else dft32<C, PK>(v);
}

template <typename T, int LF, bool PK>
struct WarpLineFFT {
  using C = typename C2t<T>::type;
  static constexpr int F = 1 << LF;
  static constexpr int TPL = F <= 128 ? 8 : (F <= 512 ? 16 : 32);
  static constexpr int PPT = F / TPL;
  static constexpr int R = PPT / TPL;           // TPL-point DFTs per lane in stage 2
  static constexpr int LPW = 32 / TPL;          // lines per warp
  // exchange row pitch: with 8 lanes per line two lines share a half-warp
  // wavefront, and a pitch of 8 (mod 16) complex values keeps them on
  // different banks
  static constexpr int P = F + (TPL == 8 ? 8 : 0);
  static_assert(PPT % TPL == 0 && (PPT == 8 || PPT == 16 || PPT == 32), "line split");

  // Forward DFT (unnormalised) of the line: v[s] = x[j + TPL s] in,
  // X[j + TPL s] out.  ex: this line's exchange row; tw2: k2-major twiddles.
  static __device__ __forceinline__ void forward(C (&v)[PPT], C* ex, const C* tw2, int j) {
    dft_n<C, PPT, PK>(v);
    // twiddles in groups of 8: loaded as they are needed (hoisting all of
    // them ahead of the DFT would hold 2 (PPT - 1) more registers)
#pragma unroll
    for (int k2 = 1; k2 < PPT; ++k2) {
      if (k2 % 8 == 0) asm volatile("" ::: "memory");
      v[k2] = cmul(v[k2], tw2[k2 * TPL + j]);
    }
#pragma unroll
    for (int k2 = 0; k2 < PPT; ++k2) ex[k2 * TPL + (j ^ (k2 & (TPL - 1)))] = v[k2];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C w[TPL];
#pragma unroll
      for (int jj = 0; jj < TPL; ++jj) w[jj] = ex[(j + TPL * r) * TPL + (jj ^ j)];
      dft_n<C, TPL, PK>(w);
#pragma unroll
      for (int k1 = 0; k1 < TPL; ++k1) v[r + R * k1] = w[k1];
    }
    // the row is rewritten by the next transform only after every lane has read it
    __syncwarp();
  }

  // T applied to the line: forward DFT, symbol and conjugation, forward DFT,
  // conjugation (the inverse DFT of the symbol times the spectrum).
  template <typename Sym>
  static __device__ __forceinline__ void apply(C (&v)[PPT], C* ex, const C* tw2, int j, const Sym& sym) {
    forward(v, ex, tw2, j);
#pragma unroll
    for (int s = 0; s < PPT; ++s) {
      const T sy = sym(j + s * TPL);
      v[s].x = sy * v[s].x;
      v[s].y = -sy * v[s].y;
    }
    forward(v, ex, tw2, j);
#pragma unroll
    for (int s = 0; s < PPT; ++s) v[s].y = -v[s].y;
  }
};

// The line symbol c2 lam^2 + c1c lam with lam = dl * (m, or m - F above F/2):
// the x-line symbol lambda_p^2/2 + Omega y lambda_p and the y-line symbol
// eta_q^2/2 - Omega x eta_q of Eq. energy-discrete-FP (1/F folded into c2, c1).
template <typename T, int F>
struct FusedSym {
  T c2, c1c, dl;
  __device__ __forceinline__ T operator()(int m) const {
    const T lm = dl * (T)(m < (F >> 1) ? m : m - F);
    return (c2 * lm + c1c) * lm;
  }
};

struct FusedArgs {
  void* ty;                 // T_y of the y-tasks (the output array when every point is written)
  unsigned int* sync;       // [0] tasks handed out, [1] warps done, [2, 2+nb) y-tasks done,
                            // [2+nb, 2+2nb) x-tasks done, [2+2nb] error flag
  int nbatch, NY, NX;       // instances, y-tasks and x-tasks per instance
  long long max_polls;      // polls of one task wait before it gives up
  int skew;                 // instances whose y-tasks precede the first x-task
  const void* tw2x;         // k2-major twiddles of the x- and y-lines
  const void* tw2y;
};

// Completion counters with release/acquire semantics at GPU scope: a warp's
// stores are ordered before its lane 0's release by the warp barrier that
// precedes it (a release is cumulative), so no lane needs a full fence.
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_add_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int atom_add_acqrel_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;\n" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Task t of the fixed order with skew S (1 <= S <= nb instances):
//   Y_0 ... Y_{S-1}, (Y_S, X_0), (Y_{S+1}, X_1), ..., (Y_{nb-1}, X_{nb-1-S}), X_{nb-S} ... X_{nb-1}
// kind 0 = y-task, 1 = x-task; b = instance; i = task within the instance.
// With S about the warps in flight over NY, the y-tasks of an instance are
// done by the time its x-tasks are handed out.
__device__ __forceinline__ void decode_task(int t, int nb, int NY, int NX, int S, int& kind, int& b, int& i) {
  if (t < S * NY) {
    kind = 0;
    b = t / NY;
    i = t - b * NY;
    return;
  }
  const int u = t - S * NY;
  const int pairs = nb - S;
  if (u < pairs * (NY + NX)) {
    const int p = u / (NY + NX);
    const int o = u - p * (NY + NX);
    if (o < NY) {
      kind = 0;
      b = S + p;
      i = o;
    } else {
      kind = 1;
      b = p;
      i = o - NY;
    }
    return;
  }
  const int w = u - pairs * (NY + NX);
  kind = 1;
  b = pairs + w / NX;
  i = w - (w / NX) * NX;
}

template <typename T, bool CPLX, int EPI, int LF, bool PK>
__global__ void __launch_bounds__(FUSED_THREADS, fused_minb(LF)) k_fused2d(PassGeom<T> gx, PassGeom<T> gy, PassData<T> D, FusedArgs FA) {
  static_assert(std::is_same<T, float>::value, "float32 only");
  using FFT = WarpLineFFT<T, LF, PK>;
  using C = typename FFT::C;
  using V = typename VT<T, CPLX>::V;
  using A = typename AccT<T>::type;
  constexpr int F = FFT::F, TPL = FFT::TPL, PPT = FFT::PPT, LPW = FFT::LPW;
  constexpr int NV = CPLX ? PPT : 2 * PPT;     // values per lane and x-task (real: two rows)
  constexpr unsigned FULL = 0xffffffffu;
  // a finished solver run (control block done) takes no tasks; the warps still
  // count themselves out below, so the counters are reset all the same
  const bool idle = D.ctl && D.ctl->done;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* twx = reinterpret_cast<C*>(smem_raw);
  C* twy = twx + F;
  C* exb = twy + F;
  C* stb = exb + (FUSED_THREADS / 32) * LPW * FFT::P;   // x-tasks: the input of each line
  for (int i = threadIdx.x; i < F; i += blockDim.x) {
    twx[i] = reinterpret_cast<const C*>(FA.tw2x)[i];
    twy[i] = reinterpret_cast<const C*>(FA.tw2y)[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = lane / TPL, j = lane & (TPL - 1);
  C* ex = exb + (warp * LPW + h) * FFT::P;
  const int nb = FA.nbatch, NY = FA.NY, NX = FA.NX;
  unsigned int* cnt = FA.sync;
  unsigned int* ydone = cnt + 2;
  unsigned int* xdone = cnt + 2 + nb;
  const int n0 = gx.n0;                          // row length (points)
  const int n0c = CPLX ? n0 : n0 >> 1;           // complex columns of the y-lines
  const long long M = gx.M;

  // operands (as in the two-kernel path): input, optional second operand,
  // optional trial point formed on load (solver)
  const V* xin = (const V*)D.x;
  const V* xsub = (const V*)D.xsub;
  const C* ysrc0 = nullptr;      // y-tasks: X_cur (step on load)
  const C* ysrc1 = nullptr;      // y-tasks: G_cur (step on load)
  C* yst = nullptr;
  T sa = 0, sb = 0;
  if (D.use_slots) {
    const Alg1Ctl* c = D.ctl;
    xin = (const V*)D.xs[c->trial];
    if (D.step_on_load) {
      yst = (C*)D.xs[c->trial];
      ysrc0 = (const C*)D.xs[c->cur];
      ysrc1 = (const C*)D.gs[c->cur];
      sa = (T)(c->s * c->a);
      sb = (T)(c->s * c->b);
    }
  }
  C* tyc = (C*)FA.ty;                            // T_y in complex units (y view)
  const V* tyv = (const V*)FA.ty;                // the same array per point (x view)
  EpiCtx<T, CPLX> E;
  make_ctx<T, CPLX, EPI, false>(E, D);
  const T* Vp = D.V;
  const bool reduce = EPI != EPI_HESS && D.nq > 0;
  constexpr bool FPART = EPI == EPI_GRAD;
  const int ntask = nb * (NY + NX);

  while (!idle) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(cnt, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= ntask) break;
    int kind, b, ti;
    decode_task(t, nb, NY, NX, FA.skew, kind, b, ti);
    // Both kinds of task share one copy of the line transform below: four
    // unrolled copies of it (y and x, forward and inverse) overflow the
    // instruction cache.  Every load of a task is issued before its first
    // store (a store in between would hold the later loads back); read-only
    // operands go through the non-coherent path.
    C v[PPT];
    int ok = 1;
    long long cb = 0, rb = 0, ib = 0;
    int row0 = 0;
    FusedSym<T, F> sym;
    if (kind == 0) {
      // ---------------- y-task: columns ti*LPW + h (complex view)
      const int ccol = ti * LPW + h;
      cb = (long long)b * (CPLX ? M : M >> 1) + ccol;
      if (yst) {
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
          const long long e = cb + (long long)(j + TPL * s) * n0c;
          v[s] = sa * __ldg(ysrc0 + e) + sb * __ldg(ysrc1 + e);
        }
#pragma unroll
        for (int s = 0; s < PPT; ++s) yst[cb + (long long)(j + TPL * s) * n0c] = v[s];
      } else {
        const C* xc = (const C*)xin;
        const C* sc = (const C*)xsub;
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
          const long long e = cb + (long long)(j + TPL * s) * n0c;
          C a = __ldg(xc + e);
          if (sc) a = a - __ldg(sc + e);
          v[s] = a;
        }
      }
      sym.c2 = gy.c2;
      sym.dl = gy.dlam;
      sym.c1c = (CPLX && gy.rcoord) ? gy.c1 * gy.rcoord[ccol] : T(0);
    } else {
      // ---------------- x-task: complex lines ti*LPW + h (rows; real: row pairs)
      if (lane == 0) {
        long long polls = 0;
        while (ld_acquire_u32(ydone + b) < (unsigned)NY) {
          if (++polls > FA.max_polls) {
            atomicExch(cnt + 2 + 2 * nb, 1u);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      ok = __shfl_sync(FULL, ok, 0);
      __syncwarp();   // every lane's reads of T_y come after lane 0's acquire
      const int line = ti * LPW + h;
      row0 = CPLX ? line : 2 * line;
      ib = (long long)b * M;
      rb = ib + (long long)row0 * n0 + j;
      // the input: the trial point written by this launch's y-tasks (step
      // on load), else read-only data
#pragma unroll
      for (int s = 0; s < PPT; ++s) {
        if constexpr (CPLX) {
          const long long e = rb + TPL * s;
          V a = yst ? __ldcg(xin + e) : __ldg(xin + e);
          if (xsub) a = a - __ldg(xsub + e);
          v[s] = a;
        } else {
          const long long e = rb + TPL * s;
          T a = yst ? __ldcg(xin + e) : __ldg(xin + e);
          T c = yst ? __ldcg(xin + e + n0) : __ldg(xin + e + n0);
          if (xsub) {
            a -= __ldg(xsub + e);
            c -= __ldg(xsub + e + n0);
          }
          v[s].x = a;
          v[s].y = c;
        }
      }
      // the epilogue needs the input again: kept in this lane's stash slots
      C* stash = stb + (warp * LPW + h) * FFT::P;
#pragma unroll
      for (int s = 0; s < PPT; ++s) stash[j + TPL * s] = v[s];
      sym.c2 = gx.c2;
      sym.dl = gx.dlam;
      sym.c1c = (CPLX && gx.rcoord) ? gx.c1 * gx.rcoord[row0] : T(0);
    }
    // ---------------- the line operator: forward DFT, symbol and conjugation,
    // forward DFT, conjugation (the inverse DFT of symbol x spectrum)
    {
      const C* tw = kind == 0 ? twy : twx;
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        FFT::forward(v, ex, tw, j);
        if (pass == 0) {
#pragma unroll
          for (int s = 0; s < PPT; ++s) {
            const T sy = sym(j + s * TPL);
            v[s].x = sy * v[s].x;
            v[s].y = -sy * v[s].y;
          }
        }
      }
#pragma unroll
      for (int s = 0; s < PPT; ++s) v[s].y = -v[s].y;
    }
    if (kind == 0) {
#pragma unroll
      for (int s = 0; s < PPT; ++s) tyc[cb + (long long)(j + TPL * s) * n0c] = v[s];
      __syncwarp();
      if (lane == 0) red_add_release_u32(ydone + b, 1u);
      continue;
    }
    {
      A acc[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
      T amax = T(0);
      if (ok) {
        const C* stash = stb + (warp * LPW + h) * FFT::P;
        // + T_y of the row(s): all these loads precede the epilogue's stores
#pragma unroll
        for (int s = 0; s < PPT; ++s) {
          if constexpr (CPLX) {
            v[s] = v[s] + __ldcg(tyv + rb + TPL * s);
          } else {
            v[s].x += __ldcg(tyv + rb + TPL * s);
            v[s].y += __ldcg(tyv + rb + n0 + TPL * s);
          }
        }
        T pacc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) pacc[q] = T(0);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const long long gi = rb + (long long)(q / PPT) * n0 + TPL * (q % PPT);
          const C xs = stash[j + TPL * (q % PPT)];
          V x, kin;
          if constexpr (CPLX) {
            x = xs;
            kin = v[q];
          } else {
            x = (q < PPT) ? xs.x : xs.y;
            kin = (q < PPT) ? v[q].x : v[q - PPT].y;
          }
          const V lin = kin + __ldg(Vp + (gi - ib)) * x;
          if constexpr (FPART) epilogue_point<T, CPLX, EPI, 2>(E, gi, x, lin, pacc, amax);
          else epilogue_point<T, CPLX, EPI, 2>(E, gi, x, lin, acc, amax);
        }
        if constexpr (FPART) {
#pragma unroll
          for (int q = 0; q < 3; ++q) acc_add(acc[q], pacc[q]);
        }
      }
      if (reduce) {
        // the task's partial sums: fixed shuffle tree, slot b * NX + ti
        double* part = D.partials + ((size_t)b * NX + ti) * NQ;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          if (q == Q_MAX) {
            float m = sqrtf(amax);   // correctly rounded: the float64 root rounded to float32
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(FULL, m, o));
            if (lane == 0) reinterpret_cast<float2*>(part)[q] = make_float2(ok ? m : __int_as_float(0x7fc00000), 0.f);
          } else if (q < D.nq) {
            A w = acc[q];
            for (int o = 16; o > 0; o >>= 1) acc_merge(w, shfl_down(w, o));
            if (lane == 0)
              reinterpret_cast<float2*>(part)[q] = make_float2(ok ? w.hi : __int_as_float(0x7fc00000), w.lo);
          } else if (lane == 0) {
            reinterpret_cast<float2*>(part)[q] = make_float2(0.f, 0.f);
          }
        }
        // lane 0 wrote the partials; its acquire-release count orders them
        // before the count and, for the last task, every other task's
        // partials before the fold
        int last = 0;
        if (lane == 0) last = atom_add_acqrel_u32(xdone + b, 1u) == (unsigned)(NX - 1);
        last = __shfl_sync(FULL, last, 0);
        __syncwarp();
        if (last) {
          // fold instance b's NX partials in task order
          const float2* pp = reinterpret_cast<const float2*>(D.partials + (size_t)b * NX * NQ);
          for (int q = 0; q < NQ; ++q) {
            double val = 0.0;
            if (q < D.nq || q == Q_MAX) {
              DF x;
              acc_zero(x);
              for (int i = lane; i < NX; i += 32) {
                const float2 f = __ldcg(pp + (size_t)i * NQ + q);
                DF w;
                w.hi = f.x;
                w.lo = f.y;
                if (q == Q_MAX) df_max(x, w);
                else acc_merge(x, w);
              }
              for (int o = 16; o > 0; o >>= 1) {
                const DF w = shfl_down(x, o);
                if (q == Q_MAX) df_max(x, w);
                else acc_merge(x, w);
              }
              val = acc_value(x);
            }
            if (lane == 0) D.results[(size_t)b * NQ + q] = val;
          }
          if (lane == 0 && D.control) {
            if (D.control == 1) alg1_control<T>(D.ctl, D.results);
            else if (D.control == 2) rn_control(D.rn, D.results);
          }
        }
      }
    }
  }
  // the last warp to finish resets the counters for the next launch (every
  // warp has stopped taking tasks by then); the error flag stays set
  __syncwarp();
  int lastw = 0;
  if (lane == 0) lastw = atom_add_acqrel_u32(cnt + 1, 1u) == gridDim.x * (blockDim.x >> 5) - 1;
  lastw = __shfl_sync(FULL, lastw, 0);
  __syncwarp();
  if (lastw) {
    for (int i = lane; i < 2 + 2 * nb; i += 32) cnt[i] = 0u;
  }
}

// Dynamic shared memory of the fused kernel: two twiddle tables, and for every
// line of the CTA's warps an exchange row and a stash row (the x-task input).
template <typename T, int LF>
static size_t fused_smem() {
  using FFT = WarpLineFFT<T, LF, true>;
  return (2 * (size_t)FFT::F + 2 * (size_t)(FUSED_THREADS / 32) * FFT::LPW * FFT::P) * sizeof(typename FFT::C);
}

template <typename T, bool CPLX, int EPI, int LF, bool PK>
static gpe_status launch_fused2d_t(const GridHost& g, const GridDev<T>& d, const PassData<T>& D, void* acc,
                                   bool step_first, cudaStream_t st) {
  using FFT = WarpLineFFT<T, LF, PK>;
  const int nb = g.nbatch;
  const int n0c = g.is_complex ? g.ext[0] : g.ext[0] / 2;
  const int lines = g.is_complex ? g.ext[1] : g.ext[1] / 2;
  FusedArgs FA;
  FA.nbatch = nb;
  FA.NY = n0c / FFT::LPW;
  FA.NX = lines / FFT::LPW;
  FA.sync = d.fsync;
  FA.max_polls = wait_limit(1LL << 24);
  FA.tw2x = d.tw2[0];
  FA.tw2y = d.tw2[1];
  // T_y goes into the output array when the epilogue writes every point of it
  // (gradient, Hessian-vector, objective passes), else into the accumulator
  FA.ty = acc;
  if ((EPI == EPI_GRAD || EPI == EPI_HESS) && D.out) FA.ty = D.out;
  if ((size_t)FA.NX * nb > (size_t)d.max_blocks) return fail(GPE_EINVAL, "reduction scratch too small");
  PassData<T> Df = D;
  Df.step_on_load = step_first ? 1 : 0;
  const size_t smem = fused_smem<T, LF>();
  static int occ = -1;
  if (occ < 0) {
    GPE_CUDA(cudaFuncSetAttribute(k_fused2d<T, CPLX, EPI, LF, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    GPE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused2d<T, CPLX, EPI, LF, PK>, FUSED_THREADS,
                                                           smem));
    if (occ < 1) occ = 1;
  }
  int dev = 0, nsm = 0;
  GPE_CUDA(cudaGetDevice(&dev));
  GPE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const long long ntask = (long long)nb * (FA.NY + FA.NX);
  const long long wpc = FUSED_THREADS / 32;
  const int grid = (int)std::max<long long>(1, std::min<long long>((ntask + wpc - 1) / wpc, (long long)occ * nsm));
  // S: about twice the warps in flight over the y-tasks per instance
  // (measured: 64 x 256^2 complex 87 -> 76 us per apply against once)
  FA.skew = (int)std::min<long long>(nb, (FUSED_SKEW * (long long)grid * wpc + FA.NY - 1) / FA.NY + 1);
  ProfScope ps(kernel_name("fused2d", 0, CPLX, EPI, g.M * nb), st);
  k_fused2d<T, CPLX, EPI, LF, PK><<<grid, FUSED_THREADS, smem, st>>>(d.geom[0], d.geom[1], Df, FA);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

// Square float32 Fourier grids n x n, n = 64 ... 1024 (the line split needs
// n0 = n1 so that both kinds of task share one transform shape).
template <typename T>
static bool fused2d_ok(const GridHost& g) {
  if (!std::is_same<T, float>::value) return false;
  if (g.disc != GPE_FOURIER || g.dim != 2 || g.ext[0] != g.ext[1]) return false;
  const int n = g.ext[0];
  return n >= 64 && n <= 1024 && (n & (n - 1)) == 0;
}

// GPE_FUSED2D=0 in the environment selects the two-kernel line path instead
// (for comparisons); read once.
static bool fused2d_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("GPE_FUSED2D");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on != 0;
}

template <typename T, bool CPLX, int EPI>
static gpe_status fused2d_dispatch(const GridHost& g, const GridDev<T>& d, const PassData<T>& D, void* acc,
                                   bool step_first, cudaStream_t st) {
  switch (ilog2(g.ext[0])) {
    case 6: return launch_fused2d_t<T, CPLX, EPI, 6, true>(g, d, D, acc, step_first, st);
    case 7: return launch_fused2d_t<T, CPLX, EPI, 7, true>(g, d, D, acc, step_first, st);
    case 8: return launch_fused2d_t<T, CPLX, EPI, 8, true>(g, d, D, acc, step_first, st);
    case 9: return launch_fused2d_t<T, CPLX, EPI, 9, true>(g, d, D, acc, step_first, st);
    case 10: return launch_fused2d_t<T, CPLX, EPI, 10, true>(g, d, D, acc, step_first, st);
  }
  return fail(GPE_EINVAL, "unsupported line length");
}

}  // namespace gpe
