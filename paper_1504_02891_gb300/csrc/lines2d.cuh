// lines2d.cuh -- the operator on 2D Fourier grids as two kernels, one per axis,
// with every line FFT held in registers.
//
// A line of F = 2^LF points is owned by F/8 threads, 8 points each: thread j
// holds the points j + s F/8 (s = 0..7).  The transform is a Stockham autosort
// FFT of radix-8 stages and, when LF is not a multiple of 3, one radix-4 or
// radix-2 tail stage; every stage reads the points j + s F/8, so the natural
// order of the input (coalesced global loads), of the spectrum (symbol
// multiply) and of the output (coalesced stores) is the register order, and
// shared memory is touched only by the exchanges between stages (two
// alternating buffers, one barrier per exchange).  Twiddles are per thread and
// per stage, computed once per launch.
//
//   y-kernel: lines are columns (complex columns; real fields pack two real
//     columns into one complex line); an optional Cayley step on load
//     (Theorem 3.3) writes the trial point; output T_y X into the accumulator.
//   x-kernel: lines are rows (real fields: two rows per complex line); the
//     epilogue adds the y-kernel's T_y X and V X and runs the pointwise
//     epilogue of the pass kernels (gradient, Hessian-vector, Algorithm 1 and
//     ratio-test sums), then the deterministic reduction and control.
//
// Spectral operator of both kernels: the x-line symbol lambda_p^2/2 + Omega y
// lambda_p and the y-line symbol eta_q^2/2 - Omega x eta_q (Eq. fftp36 /
// Eq. energy-discrete-FP with the rotation term folded per line), 1/F folded
// into the coefficients, the inverse transform taken as a conjugated forward
// transform.
#pragma once
#include <stdlib.h>
#include "ops_launch.cuh"
#include "linefft.cuh"
#include "fused2d.cuh"

namespace gpe {

// Threads of the x-kernel's CTA: 256 in float32.  In float64 a CTA holds as
// few lines as it can (64 threads, or one line of F/8 threads): the float64
// stages run on small grids (256^2: 16 CTAs of 256 threads), and the float64
// FMA rate of one SM is 1/64 of its float32 rate, so spreading the lines over
// more SMs is what shortens them.  At most 128 registers per thread.
template <typename T> __host__ __device__ constexpr int lines_x_threads(int lf) {
  return sizeof(T) == 4 ? 256 : ((1 << lf) / 8 > 64 ? (1 << lf) / 8 : 64);
}
template <typename T> __host__ __device__ constexpr int lines_x_minb(int lf) {
  return 65536 / (lines_x_threads<T>(lf) * 128);
}

// Exchange slots of CW lines stored interleaved (point-major, the CW lines of
// a point side by side): the y-kernel, where a warp holds 32/CW points of CW
// lines.  The low bits of the point index are XORed with bits 3.. so that the
// stride-8 scatter of a radix-8 stage spreads over the bank rows.
template <typename C, int CW>
struct ExCols {
  C* base;          // buffer 0 + column
  int pstride;
  static constexpr int G = (128 / int(sizeof(C))) / CW;   // points per 128-byte bank row
  static constexpr int MASK = G > 1 ? (G > 8 ? 7 : G - 1) : 0;
  __device__ __forceinline__ C* operator()(int par, int m) const {
    const int ms = m ^ ((m >> 3) & MASK);
    return base + par * pstride + ms * CW;
  }
  // a column's points are spread over all warps of the CTA
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};


// Threads of the y-kernel's CTA: 512 in float32 (8 columns of 512 points, 64 B
// row segments); in float64 as few columns as a line allows, as for the
// x-kernel.
template <typename T> __host__ __device__ constexpr int lines_y_threads(int lf) {
  return sizeof(T) == 4 ? 512 : lines_x_threads<T>(lf);
}

// Copy of the twiddle table e^{-2 pi i n / F} into shared memory.
template <typename C>
__device__ __forceinline__ void load_table(C* dst, const C* src, int F) {
  for (int i = threadIdx.x; i < F; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// y-kernel: T_y of columns into D.out; groups of CW complex columns, the CTAs
// stride over the groups of all instances.  The next group's operands are
// fetched (cp.async, each thread its own 8 points) while this group's
// transforms run.
template <typename T, bool CPLX, int LF>
__global__ void __launch_bounds__(lines_y_threads<T>(LF)) k_lines_y(PassGeom<T> G, PassData<T> D, int colgroups,
                                                                  int total) {
  using FFT = LineFFT<T, LF>;
  using C = typename FFT::C;
  constexpr int NT = lines_y_threads<T>(LF);
  constexpr int TPL = FFT::TPL;
  constexpr int CW = NT / TPL;
  constexpr int F = FFT::F;
  if (D.ctl && D.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tws = reinterpret_cast<C*>(smem_raw);
  C* xb = tws + F;                            // [2][F][CW], swizzled points
  C* pf0 = xb + 2 * F * CW;                   // [8][NT]: next group's input
  C* pf1 = pf0 + 8 * NT;                      // [8][NT]: next group's second operand
  load_table(tws, G.tw, F);
  const int tid = threadIdx.x;
  const int cl = tid & (CW - 1), j = tid / CW;
  FFT fft;
  fft.init(j, tws);
  int par = 0;
  const int n0c = CPLX ? G.n0 : G.n0 >> 1;    // complex columns per row
  const C* xin = (const C*)D.x;
  const C* src1 = (const C*)D.xsub;
  C* yst = nullptr;
  T sa = 0, sb = 0;
  if (D.use_slots) {
    const Alg1Ctl* c = D.ctl;
    xin = (const C*)D.xs[c->trial];
    if (D.step_on_load) {
      yst = (C*)D.xs[c->trial];
      xin = (const C*)D.xs[c->cur];
      src1 = (const C*)D.gs[c->cur];
      sa = (T)(c->s * c->a);
      sb = (T)(c->s * c->b);
    }
  }
  C* out = (C*)D.out;
  LineSym<T, F> sym;
  sym.c2 = G.c2;
  sym.dl = G.dlam;
  ExCols<C, CW> ex{xb + cl, F * CW};
  auto ebase = [&](int gidx) {
    const int inst = gidx / colgroups;
    const int ccol = (gidx - inst * colgroups) * CW + cl;
    return (long long)inst * (CPLX ? G.M : G.M >> 1) + ccol;
  };
  auto fetch = [&](int gidx) {
    const long long base = ebase(gidx);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const long long e = base + (long long)(j + s * TPL) * n0c;
      cp_async(pf0 + s * NT + tid, xin + e);
      if (src1) cp_async(pf1 + s * NT + tid, src1 + e);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (blockIdx.x < total) fetch(blockIdx.x);
  for (int gidx = blockIdx.x; gidx < total; gidx += gridDim.x) {
    const long long base = ebase(gidx);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    C v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      C a = pf0[s * NT + tid];
      if (src1) {
        const C b = pf1[s * NT + tid];
        a = yst ? sa * a + sb * b : a - b;
        if (yst) yst[base + (long long)(j + s * TPL) * n0c] = a;
      }
      v[s] = a;
    }
    // every read of the prefetch buffers is done before they are refilled
    __syncthreads();
    if (gidx + (int)gridDim.x < total) fetch(gidx + gridDim.x);
    const int ccol = (int)(base % n0c);
    sym.c1c = (CPLX && G.rcoord) ? G.c1 * G.rcoord[ccol] : T(0);
    fft.apply(v, ex, par, sym);
#pragma unroll
    for (int s = 0; s < 8; ++s) out[base + (long long)(j + s * TPL) * n0c] = v[s];
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// x-kernel: T_x of rows, + T_y X (D.acc_in) + V X, then the epilogue, the
// reduction and the control.  CTA `tile` of an instance takes the line groups
// tile, tile + tiles_per_inst, ...; the next group's input and this group's
// epilogue operands are fetched with cp.async (each thread its own points)
// while the transforms run.
// (at most 128 registers per thread)
template <typename T, bool CPLX, int EPI, int LF>
__global__ void __launch_bounds__(lines_x_threads<T>(LF), lines_x_minb<T>(LF)) k_lines_x(PassGeom<T> G, PassData<T> D, int tiles_per_inst,
                                                              int groups) {
  using FFT = LineFFT<T, LF>;
  using C = typename FFT::C;
  using V = typename VT<T, CPLX>::V;
  using A = typename AccT<T>::type;
  constexpr int NT = lines_x_threads<T>(LF);
  constexpr int TPL = FFT::TPL;
  constexpr int NL = NT / TPL;
  constexpr int F = FFT::F;
  constexpr int NV = CPLX ? 8 : 16;           // values per thread and group (real: two rows)
  if (D.ctl && D.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tws = reinterpret_cast<C*>(smem_raw);
  C* xb = tws + F;                            // [2][NL][P]
  V* xs = reinterpret_cast<V*>(xb + 2 * NL * FFT::P);   // [2][NV][NT] input, double-buffered
  V* ea = xs + 2 * NV * NT;                   // [NV][NT] T_y X of this group
  T* ev = reinterpret_cast<T*>(ea + NV * NT); // [NV][NT] potential of this group
  load_table(tws, G.tw, F);
  const int tid = threadIdx.x;
  const int l = tid / TPL, j = tid & (TPL - 1);
  FFT fft;
  fft.init(j, tws);
  int par = 0;
  const int inst = blockIdx.x / tiles_per_inst;
  const int tile = blockIdx.x - inst * tiles_per_inst;
  const V* xin = (const V*)D.x;
  if (D.use_slots) xin = (const V*)D.xs[D.ctl->trial];
  const V* xsub = (const V*)D.xsub;
  const V* accin = (const V*)D.acc_in;
  EpiCtx<T, CPLX> E;
  make_ctx<T, CPLX, EPI, false>(E, D);
  A acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc_zero(acc[q]);
  T amax = T(0);
  // H psi sums in float32: each group's 8 (16) points are summed in float and
  // the group sum enters the float-pair accumulator (float32 data carry no
  // more digits than that)
  constexpr bool FPART = EPI == EPI_GRAD && std::is_same<T, float>::value;
  T pacc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) pacc[q] = T(0);
  const long long ibase = (long long)inst * G.M;
  const T* Vp = D.V;
  LineSym<T, F> sym;
  sym.c2 = G.c2;
  sym.dl = G.dlam;
  // lines of F >= 256 points occupy whole warps (TPL >= 32 threads); the
  // CTA's NL <= 8 lines take named barriers 1..NL
  static_assert(TPL < 32 || (TPL % 32 == 0 && NL <= 15), "named barriers per line");
  ExRow<C, FFT::P> ex{xb + l * FFT::P, NL * FFT::P, 1 + l, TPL};
  // element of value q (q = s, or s + 8 for the second row of a real pair)
  auto gidx = [&](int grp, int q) -> long long {
    const int line = grp * NL + l;
    const int row = (CPLX ? line : 2 * line) + (q >> 3);
    return ibase + (long long)row * G.n0 + j + (q & 7) * TPL;
  };
  auto fetch_x = [&](int grp, int b) {
#pragma unroll
    for (int q = 0; q < NV; ++q) cp_async(xs + (b * NV + q) * NT + tid, xin + gidx(grp, q));
  };
  int b = 0;
  if (tile < groups) {
    fetch_x(tile, 0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int grp = tile; grp < groups; grp += tiles_per_inst) {
    // the prefetch slots are per thread; the line's exchange rows are reused
    // by the next group only after the line's own barrier
    ex.sync();
    const bool more = grp + tiles_per_inst < groups;
    if (more) fetch_x(grp + tiles_per_inst, b ^ 1);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const long long gi = gidx(grp, q);
      if (accin) cp_async(ea + q * NT + tid, accin + gi);
      cp_async(ev + q * NT + tid, Vp + (gi - ibase));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // this group's input (committed one group earlier)
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    C v[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      if constexpr (CPLX) {
        V a = xs[(b * NV + s) * NT + tid];
        if (xsub) a = a - xsub[gidx(grp, s)];
        v[s] = a;
      } else {
        T a = xs[(b * NV + s) * NT + tid], c = xs[(b * NV + s + 8) * NT + tid];
        if (xsub) {
          a -= xsub[gidx(grp, s)];
          c -= xsub[gidx(grp, s + 8)];
        }
        v[s].x = a;
        v[s].y = c;
      }
    }
    const int row0 = CPLX ? grp * NL + l : 2 * (grp * NL + l);
    sym.c1c = (CPLX && G.rcoord) ? G.c1 * G.rcoord[row0] : T(0);
    fft.apply(v, ex, par, sym);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(0) : "memory");
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const long long gi = gidx(grp, q);
      V x = xs[(b * NV + q) * NT + tid];
      if (xsub) x = x - xsub[gi];
      V kin;
      if constexpr (CPLX) kin = v[q];
      else kin = (q < 8) ? v[q].x : v[q - 8].y;
      if (accin) kin = kin + ea[q * NT + tid];
      const V lin = kin + ev[q * NT + tid] * x;
      if constexpr (FPART) epilogue_point<T, CPLX, EPI, false>(E, gi, x, lin, pacc, amax);
      else epilogue_point<T, CPLX, EPI, false>(E, gi, x, lin, acc, amax);
    }
    if constexpr (FPART) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        acc_add(acc[q], pacc[q]);
        pacc[q] = T(0);
      }
    }
    b ^= 1;
  }
  if (EPI == EPI_HESS || D.nq == 0) return;
  if (reduce_partials(acc, amax, D.nq, D.partials, D.results, D.ticket, tiles_per_inst)) run_control<T>(D);
}

static int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

template <typename T, bool CPLX, int EPI, int LF0>
static gpe_status launch_lines_x(const GridDev<T>& d, const PassData<T>& Dx, int nbatch, int groups,
                                 cudaStream_t st) {
  using C = typename C2t<T>::type;
  const PassGeom<T>& gx = d.geom[0];
  constexpr int NTX = lines_x_threads<T>(LF0);
  constexpr int NL = NTX / ((1 << LF0) / 8);
  constexpr int NV = CPLX ? 8 : 16;
  const size_t vsz = sizeof(T) * (CPLX ? 2 : 1);
  const size_t smem = ((size_t)(1 << LF0) + 2 * (size_t)NL * LineFFT<T, LF0>::P) * sizeof(C) +
                      3 * (size_t)NV * NTX * vsz + (size_t)NV * NTX * sizeof(T);
  static int occ = -1;
  if (occ < 0) {
    GPE_CUDA(cudaFuncSetAttribute(k_lines_x<T, CPLX, EPI, LF0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    GPE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lines_x<T, CPLX, EPI, LF0>, NTX, smem));
    if (occ < 1) occ = 1;
  }
  // a few resident waves in all (4, or the measured choice), at most the
  // reduction scratch's capacity
  const long long want = (long long)tuned_waves(0, sizeof(T) == 8, CPLX, gx.n0, gx.n1, nbatch) * occ * num_sms();
  int tiles = groups;
  while (tiles > 1 && (long long)tiles * nbatch > want) tiles = (tiles + 1) / 2;
  while (tiles > 1 && (long long)tiles * nbatch > d.max_blocks) tiles = (tiles + 1) / 2;
  if ((long long)tiles * nbatch > d.max_blocks) return fail(GPE_EINVAL, "reduction scratch too small");
  ProfScope ps(kernel_name("linesx", sizeof(T) == 8, CPLX, EPI, gx.M * nbatch), st);
  k_lines_x<T, CPLX, EPI, LF0><<<nbatch * tiles, NTX, smem, st>>>(gx, Dx, tiles, groups);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

template <typename T, bool CPLX, int EPI, int LF0, int LF1>
static gpe_status launch_lines2d_t(const GridDev<T>& d, const PassData<T>& D, int nbatch, void* acc, bool step_first,
                                   cudaStream_t st) {
  using C = typename C2t<T>::type;
  const PassGeom<T>& gx = d.geom[0];
  const PassGeom<T>& gy = d.geom[1];
  constexpr int YT = lines_y_threads<T>(LF1);
  constexpr int CW = YT / ((1 << LF1) / 8);
  constexpr int NL = lines_x_threads<T>(LF0) / ((1 << LF0) / 8);
  const int n0c = CPLX ? gx.n0 : gx.n0 / 2;
  const int colgroups = n0c / CW;
  const int lines = CPLX ? gx.n1 : gx.n1 / 2;
  const int groups = lines / NL;
  // y pass (first: it also forms the trial point)
  {
    PassData<T> Dy = D;
    Dy.step_on_load = step_first ? 1 : 0;
    Dy.acc_in = nullptr;
    Dy.out = acc;
    Dy.nq = 0;
    Dy.control = 0;
    const size_t smem = ((size_t)(1 << LF1) * (1 + 2 * CW) + 16 * (size_t)YT) * sizeof(C);
    static int occ = -1;
    if (occ < 0) {
      GPE_CUDA(cudaFuncSetAttribute(k_lines_y<T, CPLX, LF1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      GPE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lines_y<T, CPLX, LF1>, YT, smem));
      if (occ < 1) occ = 1;
    }
    const int total = nbatch * colgroups;
    const int grid = std::min(total, tuned_waves(1, sizeof(T) == 8, CPLX, gx.n0, gx.n1, nbatch) * occ * num_sms());
    ProfScope ps(kernel_name("linesy", sizeof(T) == 8, CPLX, EPI_ACC, gx.M * nbatch), st);
    k_lines_y<T, CPLX, LF1><<<grid, YT, smem, st>>>(gy, Dy, colgroups, total);
    GPE_CUDA(cudaGetLastError());
  }
  // x pass with the epilogue
  {
    PassData<T> Dx = D;
    Dx.step_on_load = 0;
    Dx.acc_in = acc;
    gpe_status s = launch_lines_x<T, CPLX, EPI, LF0>(d, Dx, nbatch, groups, st);
    if (s != GPE_OK) return s;
  }
  return GPE_OK;
}

// The supported shapes: n0, n1 in {64, ..., 1024}; the column groups and line
// groups must tile the grid.
template <typename T>
static bool lines2d_ok(const GridHost& g) {
  if (g.disc != GPE_FOURIER || g.dim != 2) return false;
  const int n0 = g.ext[0], n1 = g.ext[1];
  auto pow2 = [](int n) { return n >= 64 && n <= 1024 && (n & (n - 1)) == 0; };
  if (!pow2(n0) || !pow2(n1)) return false;
  const int cw = lines_y_threads<T>(ilog2(n1)) / (n1 / 8), nl = lines_x_threads<T>(ilog2(n0)) / (n0 / 8);
  const int n0c = g.is_complex ? n0 : n0 / 2;
  const int lines = g.is_complex ? n1 : n1 / 2;
  return n0c % cw == 0 && lines % nl == 0;
}

template <typename T, bool CPLX, int EPI, int LF0>
static gpe_status lines2d_dispatch1(const GridDev<T>& d, const PassData<T>& D, int nbatch, void* acc, bool step_first,
                                    int lf1, cudaStream_t st) {
  switch (lf1) {
    case 6: return launch_lines2d_t<T, CPLX, EPI, LF0, 6>(d, D, nbatch, acc, step_first, st);
    case 7: return launch_lines2d_t<T, CPLX, EPI, LF0, 7>(d, D, nbatch, acc, step_first, st);
    case 8: return launch_lines2d_t<T, CPLX, EPI, LF0, 8>(d, D, nbatch, acc, step_first, st);
    case 9: return launch_lines2d_t<T, CPLX, EPI, LF0, 9>(d, D, nbatch, acc, step_first, st);
    case 10: return launch_lines2d_t<T, CPLX, EPI, LF0, 10>(d, D, nbatch, acc, step_first, st);
  }
  return fail(GPE_EINVAL, "unsupported line length");
}

template <typename T, bool CPLX, int EPI>
static gpe_status lines2d_dispatch0(const GridDev<T>& d, const PassData<T>& D, int nbatch, void* acc, bool step_first,
                                    int lf0, int lf1, cudaStream_t st) {
  switch (lf0) {
    case 6: return lines2d_dispatch1<T, CPLX, EPI, 6>(d, D, nbatch, acc, step_first, lf1, st);
    case 7: return lines2d_dispatch1<T, CPLX, EPI, 7>(d, D, nbatch, acc, step_first, lf1, st);
    case 8: return lines2d_dispatch1<T, CPLX, EPI, 8>(d, D, nbatch, acc, step_first, lf1, st);
    case 9: return lines2d_dispatch1<T, CPLX, EPI, 9>(d, D, nbatch, acc, step_first, lf1, st);
    case 10: return lines2d_dispatch1<T, CPLX, EPI, 10>(d, D, nbatch, acc, step_first, lf1, st);
  }
  return fail(GPE_EINVAL, "unsupported line length");
}

// GPE_LINES2D=0 in the environment selects the general axis-pass kernels
// instead (for comparisons); read once.
static bool lines2d_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("GPE_LINES2D");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on != 0;
}

template <typename T>
gpe_status launch_lines2d(const GridHost& g, const GridDev<T>& d, const PassData<T>& D, int epi, void* acc,
                          bool step_first, cudaStream_t st, bool* handled) {
  *handled = false;
  gpe_status s;
  if constexpr (std::is_same<T, float>::value) {
    const int path = operator_path();
    const bool fused = path == 1 || (path == 0 && tuned_fused(g.is_complex, g.ext[0], g.nbatch));
    if (fused2d_ok<T>(g) && fused && fused2d_enabled() && lines2d_enabled()) {
#define GPE_F2D_CASE(E)                                                                    \
  case E:                                                                                  \
    s = g.is_complex ? fused2d_dispatch<T, true, E>(g, d, D, acc, step_first, st)           \
                     : fused2d_dispatch<T, false, E>(g, d, D, acc, step_first, st);         \
    break;
      switch (epi) {
        GPE_F2D_CASE(EPI_GRAD)
        GPE_F2D_CASE(EPI_HESS)
        GPE_F2D_CASE(EPI_F)
        GPE_F2D_CASE(EPI_W)
        GPE_F2D_CASE(EPI_RATIO)
        GPE_F2D_CASE(EPI_WS)
        default:
          return GPE_OK;
      }
#undef GPE_F2D_CASE
      if (s == GPE_OK) *handled = true;
      return s;
    }
  }
  if (!lines2d_ok<T>(g) || !lines2d_enabled()) return GPE_OK;
  const int lf0 = ilog2(g.ext[0]), lf1 = ilog2(g.ext[1]);
  const int nb = g.nbatch;
#define GPE_L2D_CASE(E)                                                                           \
  case E:                                                                                         \
    s = g.is_complex ? lines2d_dispatch0<T, true, E>(d, D, nb, acc, step_first, lf0, lf1, st)     \
                     : lines2d_dispatch0<T, false, E>(d, D, nb, acc, step_first, lf0, lf1, st);   \
    break;
  switch (epi) {
    GPE_L2D_CASE(EPI_GRAD)
    GPE_L2D_CASE(EPI_HESS)
    GPE_L2D_CASE(EPI_F)
    GPE_L2D_CASE(EPI_W)
    GPE_L2D_CASE(EPI_RATIO)
    GPE_L2D_CASE(EPI_WS)
    default:
      return GPE_OK;
  }
#undef GPE_L2D_CASE
  if (s == GPE_OK) *handled = true;
  return s;
}

}  // namespace gpe
