// cluster.cu -- float32 Algorithm 1 on 2D Fourier grids with one thread-block
// cluster per instance, the whole state in distributed shared memory.
//
// Why: at the cascade's grid sizes (<= 256^2 points) an operator application
// is a latency chain, not a bandwidth problem.  A cluster of CS CTAs (2..16)
// keeps X_cur, G_cur, the trial point, its gradient and the kinetic sum of
// its rows in shared memory: each CTA owns n1/CS consecutive rows.  Per
// Algorithm 1 iteration:
//   1. Cayley step on the local rows (Theorem 3.3 coefficients);
//   2. x-lines (local rows): FFT, line symbol, inverse FFT -> T_x Y;
//   3. cluster barrier;
//   4. y-lines (n0/CS columns per CTA): gather the columns of Y from every
//      CTA's shared memory (DSMEM), FFT, symbol, inverse FFT -> T_y Y at the
//      owners of the rows;
//   5. cluster barrier;
//   6. epilogue on the local rows (G = 2(T_x Y + T_y Y + V Y) + 4 alpha |Y|^2 Y
//      and the float64 reduction terms, float pairs per thread), CTA partials;
//   7. cluster barrier; every CTA folds the CS partials (a fixed shuffle tree
//      over the ranks) and runs the step-size control (alg1_control) on its
//      own copy of the control block -- identical inputs, identical state, no
//      further barrier.
// Square grids of 64, 128 and 256 points per side (LF = log2 n > 0) hold each
// line in registers (the line FFT of the 2D line kernels: F/8 threads per
// line, 8 points each, exchanges within the line's warp), so the line passes
// wait at no CTA barrier: T_x goes into the trial slot's G (dead until the
// epilogue overwrites it), T_y is stored into the owners' K with plain remote
// stores.  Other grids stage lines through shared memory (Stockham stages
// with a CTA barrier each, LF = 0), K = T_x and the y-lines add T_y into the
// owners' K (remote read-modify-write, one writer per element).
// Nothing goes to global memory until the run ends.  Cluster barriers are
// hardware barriers; every CTA executes the same sequence of them because the
// control decisions are bit-identical across the cluster.
#include <cooperative_groups.h>
#include "ops_impl.cuh"
#include "linefft.cuh"

namespace cg = cooperative_groups;

namespace gpe {

// SHIFT = true: Algorithm 1 on the regularized Newton model W^(k) in
// difference form.  The unknown is D = X - X^k, the gradient is kept as
// G^ = grad W - theta_k X = P_k + H_k D + (delta - theta_k) D with
// P_k = G_k - theta_k X^k (float64 on the host side, passed in float32), so
// every float32 vector is small and nothing cancels.  The Cayley curve is the
// same for G^ as for grad W (A(X) = G X^* - X G^* does not change when a real
// multiple of X is added to G), so Theorem 3.3's coefficients apply to G^;
// the step is D' = (a - 1) X^k + a D + b G^ with a - 1 formed without
// cancellation.  The objective is the model decrease
// Re<P_k, D> + theta_k Re<X^k, D> + 1/2 Re<D, H_k D> + delta/2 ||D||^2.
// Distributed-shared-memory access by shared::cluster addresses (mapa of a
// local shared address to the CTA of cluster rank `rank`).
__device__ __forceinline__ unsigned dsmem_addr(const void* local, int rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 dsmem_ld2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void dsmem_st2(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// The CTA's partial sums of the NQ quantities into out[0..NQ) (float pairs).
// Within a warp a reduce-scatter: at offsets 16, 8, 4, 2 a lane keeps one half
// of its quantities (chosen by its lane bit) and adds its partner's copy of
// that half, so after four steps lane l holds quantity (l >> 1) & 15 summed
// over the 16 lanes of its parity, and offset 1 adds the other parity: 16
// merges and 32 shuffles per lane instead of a 5-level tree per quantity.  The
// max-norm slot is reduced by its own shuffle tree.  Then NQ threads fold the
// warps' sums in warp order.  Every CTA and every run folds in the same order.
__device__ __forceinline__ void cluster_block_partial(const DF (&acc)[NQ], float amax2, double* out) {
  static_assert(NQ <= 16, "16 reduce-scatter slots");
  __shared__ DF red[NTHREADS / 32][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DF v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (q < NQ && q != Q_MAX) v[q] = acc[q];
    else acc_zero(v[q]);
  }
#pragma unroll
  for (int o = 16, H = 8; o >= 2; o >>= 1, H >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const DF keep = up ? v[i + H] : v[i];
      const DF send = up ? v[i] : v[i + H];
      DF w;
      w.hi = __shfl_xor_sync(0xffffffffu, send.hi, o);
      w.lo = __shfl_xor_sync(0xffffffffu, send.lo, o);
      v[i] = keep;
      acc_merge(v[i], w);
    }
  }
  {
    DF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v[0].hi, 1);
    w.lo = __shfl_xor_sync(0xffffffffu, v[0].lo, 1);
    // the two parities in a fixed order (even lane's sum first)
    if (lane & 1) {
      DF t = w;
      acc_merge(t, v[0]);
      v[0] = t;
    } else {
      acc_merge(v[0], w);
    }
  }
  float m = sqrtf(amax2);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int q = (lane >> 1) & 15;
  if ((lane & 1) == 0 && q < NQ) {
    if (q == Q_MAX) {
      red[warp][q].hi = m;
      red[warp][q].lo = 0.f;
    } else {
      red[warp][q] = v[0];
    }
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int qq = threadIdx.x;
    DF a = red[0][qq];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      if (qq == Q_MAX) a.hi = fmaxf(a.hi, red[w][qq].hi);
      else acc_merge(a, red[w][qq]);
    }
    reinterpret_cast<DF*>(out)[qq] = a;
  }
  __syncthreads();
}

// Register line FFT of the cluster engine for a square grid of 2^LF points per
// side, or 0 (shared-memory stages).
__host__ __device__ constexpr int cluster_lf(int n0, int n1) {
  return (n0 == n1 && (n0 == 64 || n0 == 128 || n0 == 256)) ? (n0 == 64 ? 6 : (n0 == 128 ? 7 : 8)) : 0;
}
// Complex values of one exchange buffer of the register path (every line the
// CTA's threads hold at once, row pitch of the line FFT).
template <int LF> __host__ __device__ constexpr int cluster_exbuf() {
  return (NTHREADS / ((1 << LF) / 8)) * LineFFT<float, LF>::P;
}

template <bool CPLX, bool SHIFT, int LF>
__global__ void __launch_bounds__(NTHREADS) k_cluster_alg1(ClusterArgs A) {
  using V = typename VT<float, CPLX>::V;
  using C = float2;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cs = A.cs;
  const int cid = blockIdx.x >> A.logcs;
  const int ncl = gridDim.x >> A.logcs;
  const int logR = A.logn1 - A.logcs;      // rows per CTA = n1 / cs
  const int R = 1 << logR;
  const int Cc = A.n0 >> A.logcs;          // columns per CTA in the y-pass
  const int n0 = A.n0, n1 = A.n1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int Pm = A.P0 > A.P1 ? A.P0 : A.P1;

  extern __shared__ __align__(16) unsigned char sm[];
  C* tw0 = reinterpret_cast<C*>(sm);
  C* tw1 = tw0 + n0;
  unsigned char* vb = reinterpret_cast<unsigned char*>(tw1 + n1);
  constexpr int NVEC = SHIFT ? 7 : 5;
  V* vec[NVEC];
#pragma unroll
  for (int i = 0; i < NVEC; ++i) vec[i] = reinterpret_cast<V*>(vb + (size_t)i * A.vec_bytes);  // X0 X1 G0 G1 K [Xk Pk]
  float* Vs = reinterpret_cast<float*>(vb + (size_t)NVEC * A.vec_bytes);      // potential of the local rows
  C* f0 = reinterpret_cast<C*>(vb + (size_t)NVEC * A.vec_bytes + A.vpot_bytes);
  const int fbuf = LF > 0 ? cluster_exbuf<(LF > 0 ? LF : 6)>() : A.lch * Pm;
  C* f1 = f0 + fbuf;
  double* part = reinterpret_cast<double*>(f1 + fbuf);
  // the control block in float32 storage (its arithmetic is float32 anyway):
  // the one-thread control then needs no float64 conversion
  __shared__ Alg1CtlT<float> s_ctl;
  __shared__ double s_res[NQ];
  __shared__ float2 s_gath[16 * NQ];   // every CTA's partials, pushed by their owners
  using Acc = DF;

  for (int i = tid; i < n0; i += nt) tw0[i] = A.tw0[i];
  for (int i = tid; i < n1; i += nt) tw1[i] = A.tw1[i];
  // register path: one line transform object (square grid: both axes share
  // the twiddle table), threads tid / TPL of a line, lane jq within it
  using RFFT = LineFFT<float, (LF > 0 ? LF : 6)>;
  constexpr int RTPL = RFFT::TPL, RLPC = NTHREADS / RTPL;
  const int lq = tid / RTPL, jq = tid & (RTPL - 1);
  RFFT rfft;
  int rpar = 0;
  // Storage index of element (local row r, column c) of a vector.  The
  // register path's y-lines read one column from 32 rows per warp access; with
  // rows n0 words apart those would all fall into one bank, so a row's
  // columns are XOR-permuted by its row bits (pairs of real columns stay
  // adjacent).  Elementwise phases see the same permutation in every vector.
  auto sidx = [&](int r, int c) -> int {
    if constexpr (LF > 0) return r * n0 + (c ^ (CPLX ? (r & 15) : 2 * (r & 15)));
    return r * n0 + c;
  };
  if constexpr (LF > 0) {
    __syncthreads();
    rfft.init(jq, tw0);
  }

  const int nloc = R * n0;                 // local elements per vector
  auto stamp = [&](int inst, int loop, int k) {
    if (A.dbg && blockIdx.x == 0 && tid == 0 && inst == 0 && loop < A.dbg_n) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      A.dbg[loop * 16 + k] = t;
    }
  };
  __shared__ int s_inst;
  for (int it = 0;; ++it) {
    // the next instance: rank 0 draws it, the cluster reads rank 0's copy
    if (rank == 0 && tid == 0) s_inst = A.next ? (int)atomicAdd(A.next, 1u) : cid + it * ncl;
    cl.sync();
    const int inst = *cl.map_shared_rank(&s_inst, 0);
    cl.sync();
    if (inst >= A.ninst) break;
    const long long gbase = (long long)inst * n0 * n1 + (long long)rank * nloc;
    const V* xin = reinterpret_cast<const V*>(A.x) + gbase;
    const float* Vp = A.V + inst * A.vstride + (long long)rank * nloc;
    const float om = A.omega ? A.omega[inst] : 0.f;
    if (tid == 0) ctl_copy(s_ctl, A.ctl[inst]);
    __syncthreads();
    for (int i = tid; i < nloc; i += nt) {
      if constexpr (SHIFT) {
        const int si = sidx(i >> A.logn0, i & (n0 - 1));
        vec[s_ctl.trial][i] = vzero<V>();           // D = 0: the trial point is X^k
        vec[5][si] = reinterpret_cast<const V*>(A.xk)[gbase + i];
        vec[6][si] = reinterpret_cast<const V*>(A.pk)[gbase + i];
      } else {
        vec[s_ctl.trial][sidx(i >> A.logn0, i & (n0 - 1))] = xin[i];
      }
      Vs[sidx(i >> A.logn0, i & (n0 - 1))] = Vp[i];
    }
    __syncthreads();

    for (int loop = 0; loop < A.max_loops; ++loop) {
      if (s_ctl.done) break;
      stamp(inst, loop, 0);
      const int trial = s_ctl.trial, cur = s_ctl.cur;
      V* Xt = vec[trial];
      V* Gt = vec[2 + trial];
      V* K = vec[4];
      const bool hc = s_ctl.has_cur != 0;
      // 1. Cayley step on the local rows
      if (hc) {
        const V* Xc = vec[cur];
        const V* Gc = vec[2 + cur];
        if constexpr (SHIFT) {
          const V* Xk = vec[5];
          const float am1 = (float)s_ctl.am1, sa = (float)s_ctl.a, sb = (float)s_ctl.b;
          for (int i = tid; i < nloc; i += nt) Xt[i] = am1 * Xk[i] + sa * Xc[i] + sb * Gc[i];
        } else {
          const float sa = (float)(s_ctl.s * s_ctl.a), sb = (float)(s_ctl.s * s_ctl.b);
          for (int i = tid; i < nloc; i += nt) Xt[i] = sa * Xc[i] + sb * Gc[i];
        }
        __syncthreads();
      }
      stamp(inst, loop, 1);
      if constexpr (LF > 0) {
        // register path: every thread arrives at the cluster barrier once
        // its part of the trial rows is formed (release), runs the x-lines
        // of the local rows while the other CTAs finish their steps, then
        // waits (acquire); the y-lines (they gather the trial rows of every
        // CTA) write K = T_y at the owners; the barrier.  The epilogue adds
        // T_x from G.
        asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
        // 2. x-lines of the local rows: T_x Y into the trial slot's G (dead
        // until the epilogue, which adds it and then overwrites it)
        {
        const int nlines = CPLX ? R : R / 2;
        const float c1 = om / n0;
        LineSym<float, RFFT::F> sym;
        sym.c2 = 0.5f / n0;
        sym.dl = A.dlam0;
        ExRow<C, RFFT::P> ex{f0 + lq * RFFT::P, fbuf, 1 + lq, RTPL};
        for (int lb = 0; lb < nlines; lb += RLPC) {
          // every lane of a warp runs the transform (its exchanges are warp
          // barriers); lines past the CTA's rows carry zeros and store nothing
          const int line = lb + lq;
          const bool act = line < nlines;
          C v[8];
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const int m = jq + s * RTPL;
            v[s] = make_float2(0.f, 0.f);
            if (act) {
              if constexpr (CPLX) v[s] = Xt[sidx(line, m)];
              else v[s] = make_float2(Xt[sidx(2 * line, m)], Xt[sidx(2 * line + 1, m)]);
            }
          }
          sym.c1c = (CPLX && act) ? c1 * A.yn[rank * R + line] : 0.f;
          ex.sync();   // the rows are rewritten only after every lane has read them
          rfft.apply(v, ex, rpar, sym);
          if (act) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
              const int m = jq + s * RTPL;
              if constexpr (CPLX) {
                Gt[sidx(line, m)] = v[s];
              } else {
                Gt[sidx(2 * line, m)] = v[s].x;
                Gt[sidx(2 * line + 1, m)] = v[s].y;
              }
            }
          }
        }
        }
        stamp(inst, loop, 2);
        asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
        stamp(inst, loop, 3);
        // 4. y-lines of this CTA's columns: gather from every CTA, T_y Y into the owners' K
        {
        const int nlines = CPLX ? Cc : Cc / 2;
        const int colbase = rank * Cc;
        const float c1 = -om / n1;
        // Point p of every line of this CTA is row p + rank R (mod n1): T_y is
        // circulant along a line (a diagonal symbol on the periodic grid), so
        // transforming the rotated line and writing back at the rotated rows
        // gives T_y itself, and at each register slot the CTAs of the cluster
        // read and write distinct owners instead of all the same two.
        const int ysh = rank * R;
        LineSym<float, RFFT::F> sym;
        sym.c2 = 0.5f / n1;
        sym.dl = A.dlam1;
        ExRow<C, RFFT::P> ex{f0 + lq * RFFT::P, fbuf, 1 + lq, RTPL};
        for (int lb = 0; lb < nlines; lb += RLPC) {
          const int line = lb + lq;
          const bool act = line < nlines;
          // column `line` (complex) or the column pair 2 line, 2 line + 1 (real)
          const int col = CPLX ? colbase + line : colbase + 2 * line;
          C v[8];
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const int y = (jq + s * RTPL + ysh) & (n1 - 1);
            v[s] = make_float2(0.f, 0.f);
            if (act) {
              v[s] = dsmem_ld2(dsmem_addr(Xt + sidx(y & (R - 1), col), y >> logR));
            }
          }
          sym.c1c = (CPLX && act) ? c1 * A.xn[col] : 0.f;
          ex.sync();
          rfft.apply(v, ex, rpar, sym);
          if (act) {
            // K = T_y at the owners (plain remote stores)
#pragma unroll
            for (int s = 0; s < 8; ++s) {
              const int y = (jq + s * RTPL + ysh) & (n1 - 1);
              dsmem_st2(dsmem_addr(K + sidx(y & (R - 1), col), y >> logR), v[s]);
            }
          }
        }
        }
        stamp(inst, loop, 4);
        cl.sync();
        stamp(inst, loop, 5);
      } else {
      {
        const int nlines = CPLX ? R : R / 2;
        const float c2 = 0.5f / n0, c1 = om / n0, dl = A.dlam0;
        for (int c0 = 0; c0 < nlines; c0 += A.lch) {
          const int nl = min(A.lch, nlines - c0);
          const int ndata = CPLX ? nl : 2 * nl;
          for (int f = tid; f < ndata * n0; f += nt) {
            const int l = f >> A.logn0, j = f & (n0 - 1);
            const int row = (CPLX ? c0 : 2 * c0) + l;
            const V v = Xt[row * n0 + j];
            if constexpr (CPLX) f0[l * A.P0 + pidx(j)] = v;
            else reinterpret_cast<float*>(f0 + (l >> 1) * A.P0)[2 * pidx(j) + (l & 1)] = v;
          }
          __syncthreads();
          const int rowbase = rank * R + (CPLX ? c0 : 2 * c0);
          auto sym = [&](int line, int m, C v) -> C {
            const float lm = dl * (float)(m < (n0 >> 1) ? m : m - n0);
            float sy = c2 * lm * lm;
            if (CPLX) sy += c1 * A.yn[rowbase + line] * lm;
            C r;
            r.x = sy * v.x;
            r.y = -sy * v.y;
            return r;
          };
          C* r = fft_run<C>(f0, f1, A.logn0, nl, A.P0, tw0, sym);
          C* o = fft_run<C>(r, r == f0 ? f1 : f0, A.logn0, nl, A.P0, tw0, PostNone());
          for (int f = tid; f < ndata * n0; f += nt) {
            const int l = f >> A.logn0, j = f & (n0 - 1);
            const int row = (CPLX ? c0 : 2 * c0) + l;
            V kv;
            if constexpr (CPLX) {
              const C ov = o[l * A.P0 + pidx(j)];
              kv.x = ov.x;
              kv.y = -ov.y;
            } else {
              const C ov = o[(l >> 1) * A.P0 + pidx(j)];
              kv = (l & 1) ? -ov.y : ov.x;
            }
            K[row * n0 + j] = kv;
          }
          __syncthreads();
        }
      }
      stamp(inst, loop, 2);
      cl.sync();
      stamp(inst, loop, 3);
      {
        const int nlines = CPLX ? Cc : Cc / 2;
        const float c2 = 0.5f / n1, c1 = -om / n1, dl = A.dlam1;
        for (int c0 = 0; c0 < nlines; c0 += A.lch) {
          const int nl = min(A.lch, nlines - c0);
          const int ndata = CPLX ? nl : 2 * nl;
          const int logd = 31 - __clz(ndata);          // ndata is a power of two
          const int colbase = rank * Cc + (CPLX ? c0 : 2 * c0);
          for (int f = tid; f < ndata * n1; f += nt) {
            const int l = f & (ndata - 1), y = f >> logd;
            const int owner = y >> logR, lr = y & (R - 1);
            const V* rem = cl.map_shared_rank(Xt, owner);
            const V v = rem[lr * n0 + colbase + l];
            if constexpr (CPLX) f0[l * A.P1 + pidx(y)] = v;
            else reinterpret_cast<float*>(f0 + (l >> 1) * A.P1)[2 * pidx(y) + (l & 1)] = v;
          }
          __syncthreads();
          auto sym = [&](int line, int m, C v) -> C {
            const float lm = dl * (float)(m < (n1 >> 1) ? m : m - n1);
            float sy = c2 * lm * lm;
            if (CPLX) sy += c1 * A.xn[colbase + line] * lm;
            C r;
            r.x = sy * v.x;
            r.y = -sy * v.y;
            return r;
          };
          C* r = fft_run<C>(f0, f1, A.logn1, nl, A.P1, tw1, sym);
          C* o = fft_run<C>(r, r == f0 ? f1 : f0, A.logn1, nl, A.P1, tw1, PostNone());
          for (int f = tid; f < ndata * n1; f += nt) {
            const int l = f & (ndata - 1), y = f >> logd;
            const int owner = y >> logR, lr = y & (R - 1);
            V kv;
            if constexpr (CPLX) {
              const C ov = o[l * A.P1 + pidx(y)];
              kv.x = ov.x;
              kv.y = -ov.y;
            } else {
              const C ov = o[(l >> 1) * A.P1 + pidx(y)];
              kv = (l & 1) ? -ov.y : ov.x;
            }
            V* remk = cl.map_shared_rank(K, owner);
            V* pk = remk + lr * n0 + colbase + l;
            *pk = *pk + kv;
          }
          __syncthreads();
        }
      }
      stamp(inst, loop, 4);
      cl.sync();
      stamp(inst, loop, 5);
      }
      // 6. epilogue on the local rows
      Acc acc[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
      float amax = 0.f;
      // per-thread sums: up to 8 points in float, then into the float pairs
      float pacc[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) pacc[q] = 0.f;
      int npart = 0;
      auto merge = [&]() {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          acc_add(acc[q], pacc[q]);
          pacc[q] = 0.f;
        }
        npart = 0;
      };
      if constexpr (SHIFT) {
        const float al = (float)s_ctl.alpha, de = (float)s_ctl.delta, thk = (float)s_ctl.theta_ref;
        const float thc = (float)(hc ? s_ctl.theta_c : s_ctl.theta_hint);
        const V* Xk = vec[5];
        const V* Pk = vec[6];
        const V* Xc = hc ? vec[cur] : nullptr;
        const V* Gc = hc ? vec[2 + cur] : nullptr;
        for (int i = tid; i < nloc; i += nt) {
          const V y = Xt[i], xk = Xk[i], pk = Pk[i];
          const V lin = (LF > 0 ? K[i] + Gt[i] : K[i]) + Vs[i] * y;
          const float x2 = tre(xk, xk), R = tre(xk, y);
          const V hD = 2.f * lin + (4.f * al) * (x2 * y + (2.f * R) * xk);
          const V gh = pk + hD + (de - thk) * y;
          Gt[i] = gh;
          const V x = xk + y;
          acc_add(pacc[Q_WX], tre(pk, y) + thk * R + 0.5f * tre(y, hD) + 0.5f * de * tre(y, y));
          acc_add(pacc[Q_NY], tre(x, x));
          acc_add(pacc[Q_YG], tre(x, gh));
          acc_add(pacc[Q_GG], tre(gh, gh));
          const V q = gh - thc * x;
          acc_add(pacc[Q_Q], tre(q, q));
          acc_add(pacc[Q_QY], tre(q, x));
          const V yc = Xc ? Xc[i] : vzero<V>();
          const V gc = Gc ? Gc[i] : vzero<V>();
          const V sv = y - yc;
          const V vv = (gh - gc) - thc * sv;
          const float s2 = tre(sv, sv);
          acc_add(pacc[Q_SS], s2);
          acc_add(pacc[Q_SV], tre(sv, vv));
          acc_add(pacc[Q_VV], tre(vv, vv));
          acc_add(pacc[Q_VY], tre(vv, x));
          acc_add(pacc[Q_SY], tre(sv, x));
          acc_add(pacc[Q_DF], tre(sv, q) - 0.5f * tre(sv, vv));   // W quadratic: trapezoid exact
          amax = fmaxf(amax, s2);
          if (++npart == 8) merge();
        }
      } else {
        EpiCtx<float, CPLX> E;
        E.out = Gt;
        E.xc = hc ? vec[cur] : nullptr;
        E.gc = hc ? vec[2 + cur] : nullptr;
        E.base = nullptr;
        E.gk = nullptr;
        E.nl = (float)s_ctl.alpha;
        E.shift = 0.f;
        E.lin_scale = 2.f;
        E.th_c = (float)(hc ? s_ctl.theta_c : s_ctl.theta_hint);
        E.delta = 0.f;
        for (int i = tid; i < nloc; i += nt) {
          const V y = Xt[i];
          const V lin = (LF > 0 ? K[i] + Gt[i] : K[i]) + Vs[i] * y;
          epilogue_point<float, CPLX, EPI_F, false>(E, i, y, lin, pacc, amax);
          if (++npart == 8) merge();
        }
      }
      stamp(inst, loop, 8);
      merge();
      cluster_block_partial(acc, amax, part);
      stamp(inst, loop, 9);
      // push this CTA's partials into every CTA's gather array (remote stores
      // do not wait; the barrier below makes them visible), so that the fold
      // reads local shared memory only.  The previous iteration's reads of
      // s_gath are separated from these writes by the two barriers of this
      // iteration's line passes.
      for (int idx = tid; idx < cs * NQ; idx += nt) {
        const int r = idx / NQ, q = idx - r * NQ;
        float2* dst = cl.map_shared_rank(s_gath, r);
        dst[rank * NQ + q] = reinterpret_cast<const float2*>(part)[q];
      }
      stamp(inst, loop, 6);
      cl.sync();
      stamp(inst, loop, 10);
      // 7. fold the cluster's partials (a fixed shuffle tree over the ranks:
      // warp w folds quantities 2w and 2w + 1, one half-warp each; every CTA
      // folds the same values in the same order), then the control on the
      // local copy
      static_assert(2 * (NTHREADS / 32) >= NQ, "two quantities per warp");
      {
        const int lane = tid & 31, q = 2 * (tid >> 5) + (lane >> 4), r = lane & 15;
        DF v;
        acc_zero(v);
        if (q < NQ && r < cs) {
          const float2 f = s_gath[r * NQ + q];
          v.hi = f.x;
          v.lo = f.y;
        }
        for (int o = 8; o > 0; o >>= 1) {
          DF w;
          w.hi = __shfl_down_sync(0xffffffffu, v.hi, o, 16);
          w.lo = __shfl_down_sync(0xffffffffu, v.lo, o, 16);
          if (q == Q_MAX) v.hi = fmaxf(v.hi, w.hi);
          else acc_merge(v, w);
        }
        if (r == 0 && q < NQ) s_res[q] = acc_value(v);
      }
      __syncthreads();
      stamp(inst, loop, 11);
      if (tid == 0) alg1_control<float>(&s_ctl, s_res);
      __syncthreads();
      stamp(inst, loop, 7);
    }
    // write back the current point and its gradient, the control block and the sums
    {
      V* xo = reinterpret_cast<V*>(A.x) + gbase;
      V* go = A.g ? reinterpret_cast<V*>(A.g) + gbase : nullptr;
      const V* Xc = vec[s_ctl.cur];
      const V* Gc = vec[2 + s_ctl.cur];
      for (int i = tid; i < nloc; i += nt) {
        const int si = sidx(i >> A.logn0, i & (n0 - 1));
        xo[i] = Xc[si];
        if (go) go[i] = Gc[si];
      }
      if (rank == 0 && tid == 0) ctl_copy(A.ctl[inst], s_ctl);
      if (rank == 0 && tid < NQ) A.results[(size_t)inst * NQ + tid] = s_res[tid];
    }
    cl.sync();   // no CTA reuses or leaves its shared memory while others may read it
  }
}

// Cluster size, chunk and shared memory for an n0 x n1 grid; false if the
// state does not fit in a 16-CTA cluster.
bool cluster_shape(int n0, int n1, int cplx, int nvec, int* cs_out, int* lch_out, int* P0, int* P1, size_t* smem_out,
                   unsigned int* vec_bytes, unsigned int* vpot_bytes, size_t share, int* lf_out) {
  const size_t vsz = cplx ? 8 : 4;
  const size_t total = (size_t)n0 * n1 * vsz;
  // smallest cluster whose per-CTA share of a vector is <= share (more CTAs
  // share the work of one instance: 4 KiB for a single solve, where latency
  // counts; 16 KiB for a batch, where SMs are better spent on more instances),
  // else the largest that fits
  int pick = -1;
  for (int cs = 1; cs <= 16; cs *= 2) {
    if (n1 / cs < (cplx ? 1 : 2) || n0 / cs < (cplx ? 1 : 2)) break;
    if (total / cs <= share) { pick = cs; break; }
    if (total / cs <= 48 * 1024) pick = cs;
  }
  if (pick < 0) return false;
  const int cs = pick;
  const int R = n1 / cs, Cc = n0 / cs;
  const int lines = std::max(cplx ? R : R / 2, cplx ? Cc : Cc / 2);
  const int Fm = std::max(n0, n1);
  int lch = 1;
  while (lch * 2 <= lines && lch * 2 * Fm <= 4096) lch *= 2;
  const int p0 = n0 + n0 / 16 + 1, p1 = n1 + n1 / 16 + 1;
  const size_t vb = ((size_t)R * n0 * vsz + 15) & ~(size_t)15;
  const size_t vp = ((size_t)R * n0 * 4 + 15) & ~(size_t)15;
  // the register path (square 64^2 ... 256^2) when its exchange rows fit
  // (up to 220 KiB of the 227 KiB a CTA may have), else the shared-memory
  // stages with lc lines per chunk (up to 200 KiB)
  int lf = cluster_lf(n0, n1);
  auto need = [&](int lc) {
    const size_t fb = lf == 6   ? (size_t)cluster_exbuf<6>()
                      : lf == 7 ? (size_t)cluster_exbuf<7>()
                      : lf == 8 ? (size_t)cluster_exbuf<8>()
                                : (size_t)lc * std::max(p0, p1);
    return (size_t)(n0 + n1) * 8 + nvec * vb + vp + 2 * fb * 8 + NQ * 8;
  };
  if (lf > 0 && need(lch) > 220 * 1024) lf = 0;
  if (lf == 0)
    while (lch > 1 && need(lch) > 200 * 1024) lch /= 2;
  const size_t smem = need(lch);
  if (smem > (lf > 0 ? 220 : 200) * 1024) return false;
  if (lf_out) *lf_out = lf;
  *cs_out = cs;
  *lch_out = lch;
  *P0 = p0;
  *P1 = p1;
  *smem_out = smem;
  *vec_bytes = (unsigned int)vb;
  *vpot_bytes = (unsigned int)vp;
  return true;
}

template <bool CPLX, bool SHIFT>
static const void* cluster_fn(int lf) {
  switch (lf) {
    case 6: return (const void*)k_cluster_alg1<CPLX, SHIFT, 6>;
    case 7: return (const void*)k_cluster_alg1<CPLX, SHIFT, 7>;
    case 8: return (const void*)k_cluster_alg1<CPLX, SHIFT, 8>;
  }
  return (const void*)k_cluster_alg1<CPLX, SHIFT, 0>;
}

static int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Launch the cluster engine for `ninst` instances of one grid; clusters loop
// over instances.  Returns GPE_EINVAL if the grid does not fit (callers then
// use the CTA-grid path).
gpe_status launch_cluster_alg1(ClusterArgs A, int cplx, cudaStream_t st) {
  int cs, lch, P0, P1;
  size_t smem;
  unsigned int vb, vp;
  int lf = 0;
  if (!cluster_shape(A.n0, A.n1, cplx, A.shifted ? 7 : 5, &cs, &lch, &P0, &P1, &smem, &vb, &vp,
                     (size_t)(A.share_kb > 0 ? A.share_kb : 16) * 1024, &lf))
    return fail(GPE_EINVAL, "grid too large for the cluster engine");
  A.cs = cs;
  A.logcs = ilog2i(cs);
  A.logn0 = ilog2i(A.n0);
  A.logn1 = ilog2i(A.n1);
  A.lch = lch;
  A.P0 = P0;
  A.P1 = P1;
  A.vec_bytes = vb;
  A.vpot_bytes = vp;
  const void* fn = A.shifted ? (cplx ? cluster_fn<true, true>(lf) : cluster_fn<false, true>(lf))
                             : (cplx ? cluster_fn<true, false>(lf) : cluster_fn<false, false>(lf));
  GPE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (cs > 8) GPE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int maxc = 0;
  cfg.gridDim = dim3(cs);
  GPE_CUDA(cudaOccupancyMaxActiveClusters(&maxc, fn, &cfg));
  if (maxc < 1) return fail(GPE_EINVAL, "no cluster of this shape fits on the device");
  const int ncl = std::min(A.ninst, maxc);
  cfg.gridDim = dim3(cs * ncl);
  ProfScope ps(kernel_name("cluster_alg1", 0, cplx, -1, (long long)A.n0 * A.n1), st);
  void* args[] = {&A};
  GPE_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  return GPE_OK;
}

}  // namespace gpe
