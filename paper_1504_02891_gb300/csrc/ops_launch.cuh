// ops_launch.cuh -- host launch wrappers and device tables, instantiated per
// precision by ops_f32.cu / ops_f64.cu.
#pragma once
#include <math.h>
#include <algorithm>
#include "ops_impl.cuh"

namespace gpe {

static inline int pow2floor(long long v) {
  int p = 1;
  while ((long long)p * 2 <= v) p *= 2;
  return p;
}
static inline int pow2ceil(long long v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}
static inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

constexpr int TARGET_CTAS = 2 * 152;

// Threads per line of the fused warp-line FFT (fused2d.cuh) for a line of F
// points: F = TPL x PPT with PPT >= TPL points per thread.
static inline int fused_tpl(int F) { return F <= 128 ? 8 : (F <= 512 ? 16 : 32); }

// Tile shape of a line pass along `axis` of an array with extents ext, lines of
// FFT length Fbuf in shared memory (Fbuf >= F when the lines grow, prolongation).
template <typename T>
static PassGeom<T> make_geom(int axis, const int ext[3], int F, int Fbuf, int odd_ext, int cplx, int nbatch,
                             int* blocks, size_t* smem) {
  using C = typename C2t<T>::type;
  PassGeom<T> G{};
  G.axis = axis;
  G.n0 = ext[0];
  G.n1 = ext[1];
  G.n2 = ext[2];
  G.M = (long long)ext[0] * ext[1] * ext[2];
  G.len = ext[axis];
  G.stride = axis == 0 ? 1 : (axis == 1 ? (long long)ext[0] : (long long)ext[0] * ext[1]);
  G.ostride = axis == 1 ? (long long)ext[0] * ext[1] : (long long)ext[0];
  G.F = F;
  G.logF = ilog2(F);
  G.odd_ext = odd_ext;
  // shared memory per complex line: two padded FFT rows + two staged operand
  // rows (input and accumulator); budget ~96 KiB per CTA
  const size_t vsz = sizeof(T) * (cplx ? 2 : 1);
  const size_t per_cline = 2 * (size_t)(Fbuf + Fbuf / 16 + 1) * sizeof(C) + 2 * (size_t)(cplx ? 1 : 2) * ext[axis] * vsz;
  const size_t budget = 96 * 1024 - (size_t)Fbuf * sizeof(C);
  const int lc_cap = cplx ? MAXLB : MAXLB / 2;
  const int lc_max = std::max(1, std::min((int)(budget / per_cline), lc_cap));
  long long lines = axis == 0 ? (long long)ext[1] * ext[2] : (long long)ext[0] * (axis == 1 ? ext[2] : ext[1]);
  long long tot = lines * nbatch;
  long long tot_c = cplx ? tot : (tot + 1) / 2;
  // as many CTAs as there are SMs x 2 when the grid allows, else one line (pair) per CTA
  long long want = std::max<long long>(1, tot_c / TARGET_CTAS);
  int lc = pow2floor(std::min<long long>(want, lc_max));
  if (axis != 0) {
    const int x2 = pow2ceil(ext[0]);
    // strided lines: read rows of >= 32 bytes when there is work for the whole GPU
    const int want_lb = std::min((int)std::max<size_t>(1, 32 / vsz), x2);
    const int want_lc = cplx ? want_lb : std::max(1, want_lb / 2);
    if (tot_c >= (long long)want_lc * TARGET_CTAS) lc = std::max(lc, std::min(want_lc, pow2floor(lc_max)));
    lc = std::min(lc, cplx ? x2 : std::max(1, x2 / 2));
  }
  G.LC = lc;
  G.LB = cplx ? lc : 2 * lc;
  G.logLB = ilog2(G.LB);
  if (axis == 0) {
    G.tiles = (int)((lines + G.LB - 1) / G.LB);
    G.xt = 1;
  } else {
    G.xt = (ext[0] + G.LB - 1) / G.LB;
    G.tiles = (axis == 1 ? ext[2] : ext[1]) * G.xt;
  }
  const int work = std::max(G.LC * Fbuf / 4, G.LB * G.len);
  G.nthreads = std::min(NTHREADS, std::max(64, pow2ceil(std::min(work, NTHREADS))));
  G.tpl = std::min(pow2ceil(G.len), G.nthreads);
  G.ltpl = ilog2(G.tpl);
  G.P = Fbuf + Fbuf / 16 + 1;   // padded rows (pidx) + 1 to stagger consecutive rows
  *blocks = G.tiles * nbatch;
  // FFT part only; launch_pass adds the twiddle table and staged operands
  *smem = 2 * (size_t)G.LC * Fbuf * sizeof(C);
  return G;
}

template <typename T>
gpe_status GridDev<T>::create(const GridHost& g) {
  using Cx = typename C2t<T>::type;
  std::vector<T> hv(g.M);
  for (long long i = 0; i < g.M; ++i) hv[i] = (T)g.V[i];
  GPE_CUDA(cudaMalloc(&V, sizeof(T) * g.M));
  GPE_CUDA(cudaMemcpy(V, hv.data(), sizeof(T) * g.M, cudaMemcpyHostToDevice));
  max_blocks = 1;
  for (int a = 0; a < g.dim; ++a) {
    std::vector<T> hc(g.ext[a]);
    for (int i = 0; i < g.ext[a]; ++i) hc[i] = (T)g.nodes[a][i];
    GPE_CUDA(cudaMalloc(&coord[a], sizeof(T) * g.ext[a]));
    GPE_CUDA(cudaMemcpy(coord[a], hc.data(), sizeof(T) * g.ext[a], cudaMemcpyHostToDevice));
  }
  if (g.disc != GPE_FD) {
    for (int a = 0; a < g.dim; ++a) {
      const int F = g.F[a];
      std::vector<Cx> ht(F);
      std::vector<T> hl(F);
      // Sine grids: the odd extension lives on a box of length 2L.
      const double L = (g.hi[a] - g.lo[a]) * (g.disc == GPE_SINE ? 2.0 : 1.0);
      for (int k = 0; k < F; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)F;
        ht[k].x = (T)cos(ang);
        ht[k].y = (T)sin(ang);
        const int p = k < F / 2 ? k : k - F;
        hl[k] = (T)(2.0 * M_PI * (double)p / L);
      }
      GPE_CUDA(cudaMalloc(&tw[a], sizeof(Cx) * F));
      GPE_CUDA(cudaMemcpy(tw[a], ht.data(), sizeof(Cx) * F, cudaMemcpyHostToDevice));
      GPE_CUDA(cudaMalloc(&lam[a], sizeof(T) * F));
      GPE_CUDA(cudaMemcpy(lam[a], hl.data(), sizeof(T) * F, cudaMemcpyHostToDevice));
      PassGeom<T> G = make_geom<T>(a, g.ext, F, F, g.disc == GPE_SINE, g.is_complex, g.nbatch, &blocks[a], &smem[a]);
      G.tw = tw[a];
      G.lam = lam[a];
      G.dlam = (T)(2.0 * M_PI / L);
      G.c2 = (T)(0.5 / F);
      G.c1 = (T)0;
      G.rcoord = nullptr;
      if (g.omega != 0.0 && g.dim >= 2 && a <= 1) {
        // x-lines: +Omega*y*lam ; y-lines: -Omega*x*eta  (Eq. energy-discrete-FP)
        G.c1 = (T)((a == 0 ? g.omega : -g.omega) / F);
        G.rcoord = coord[a == 0 ? 1 : 0];
      }
      geom[a] = G;
      max_blocks = std::max(max_blocks, blocks[a]);
      if (g.dim == 2 && F >= 64 && F <= 1024) {
        // k2-major twiddles of the fused kernel's line FFT (F = TPL x PPT)
        const int tpl = fused_tpl(F), ppt = F / tpl;
        std::vector<Cx> h2(F);
        for (int k2 = 0; k2 < ppt; ++k2)
          for (int j = 0; j < tpl; ++j) {
            const double ang = -2.0 * M_PI * (double)((j * k2) % F) / (double)F;
            h2[k2 * tpl + j].x = (T)cos(ang);
            h2[k2 * tpl + j].y = (T)sin(ang);
          }
        GPE_CUDA(cudaMalloc(&tw2[a], sizeof(Cx) * F));
        GPE_CUDA(cudaMemcpy(tw2[a], h2.data(), sizeof(Cx) * F, cudaMemcpyHostToDevice));
      }
    }
    if (g.dim == 2) {
      // per-task partial sums of the fused kernel: one slot per x-task
      if (g.disc == GPE_FOURIER && g.ext[0] >= 64 && g.ext[0] <= 1024) {
        const int lines = g.is_complex ? g.ext[1] : g.ext[1] / 2;
        const int lpw = 32 / fused_tpl(g.ext[0]);
        max_blocks = std::max(max_blocks, std::max(1, lines / lpw) * g.nbatch);
      }
      const size_t nsync = 3 + 2 * (size_t)g.nbatch;
      GPE_CUDA(cudaMalloc(&fsync, sizeof(unsigned int) * nsync));
      GPE_CUDA(cudaMemset(fsync, 0, sizeof(unsigned int) * nsync));
    }
  } else {
    fd.dim = g.dim;
    fd.n0 = g.ext[0];
    fd.n1 = g.ext[1];
    fd.n2 = g.ext[2];
    fd.M = g.M;
    for (int a = 0; a < 3; ++a) {
      fd.ih2[a] = a < g.dim ? 1.0 / (g.h[a] * g.h[a]) : 0.0;
      fd.ih2c[a] = a < g.dim ? 0.5 / g.h[a] : 0.0;
    }
    fd.omega = g.omega;
    fd.tiles = (int)std::max<long long>(1, std::min<long long>((g.M + NTHREADS - 1) / NTHREADS, 1024));
    fd_blocks = fd.tiles * g.nbatch;
    max_blocks = std::max(max_blocks, fd_blocks);
  }
  max_blocks = std::max(max_blocks, 512 * g.nbatch);   // moments kernels
  return GPE_OK;
}

template <typename T>
void GridDev<T>::destroy() {
  cudaFree(V);
  V = nullptr;
  for (int a = 0; a < 3; ++a) {
    cudaFree(tw[a]);
    cudaFree(lam[a]);
    cudaFree(coord[a]);
    tw[a] = nullptr;
    lam[a] = nullptr;
    coord[a] = nullptr;
  }
  for (int a = 0; a < 2; ++a) {
    cudaFree(tw2[a]);
    tw2[a] = nullptr;
  }
  cudaFree(fsync);
  fsync = nullptr;
}

// Opt in to `bytes` of dynamic shared memory (static shared memory counts
// against the 48 KiB default too, so the opt-in is requested for any size).
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, bool CPLX, int EPI>
static gpe_status launch_pass_t(const PassGeom<T>& G, int blocks, const PassData<T>& D, cudaStream_t st) {
  using C = typename C2t<T>::type;
  const size_t vsz = sizeof(T) * (CPLX ? 2 : 1);
  const int nst = 1 + ((D.xsub || D.step_on_load) ? 1 : 0) + (D.acc_in ? 1 : 0);
  const size_t smem = (size_t)G.F * sizeof(C) + 2 * (size_t)G.LC * G.P * sizeof(C) +
                      (size_t)nst * G.LB * G.len * vsz + (EPI != EPI_ACC ? (size_t)G.LB * G.len * sizeof(T) : 0);
  static size_t allowed = 0;
  if (smem > allowed) {
    GPE_CUDA(allow_smem(k_pass<T, CPLX, EPI>, smem));
    allowed = smem;
  }
  ProfScope ps(kernel_name("pass", sizeof(T) == 8, CPLX, EPI, G.M * (blocks / G.tiles)), st);
  k_pass<T, CPLX, EPI><<<blocks, G.nthreads, smem, st>>>(G, D);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

template <typename T>
gpe_status launch_pass(const GridDev<T>& d, int axis, const PassData<T>& D, int cplx, int epi, cudaStream_t st) {
  const PassGeom<T>& G = d.geom[axis];
  const int nb = d.blocks[axis];
#define GPE_PASS_CASE(E)                                                            \
  case E:                                                                           \
    return cplx ? launch_pass_t<T, true, E>(G, nb, D, st) : launch_pass_t<T, false, E>(G, nb, D, st);
  switch (epi) {
    GPE_PASS_CASE(EPI_ACC)
    GPE_PASS_CASE(EPI_GRAD)
    GPE_PASS_CASE(EPI_HESS)
    GPE_PASS_CASE(EPI_F)
    GPE_PASS_CASE(EPI_W)
    GPE_PASS_CASE(EPI_RATIO)
    GPE_PASS_CASE(EPI_WS)
  }
#undef GPE_PASS_CASE
  return fail(GPE_EINVAL, "unknown epilogue");
}

template <typename T>
gpe_status launch_fd(const GridDev<T>& d, const PassData<T>& D, int cplx, int epi, cudaStream_t st) {
  const T* rx = d.coord[0];
  const T* ry = d.coord[1] ? d.coord[1] : d.coord[0];
  ProfScope ps(kernel_name("fd", sizeof(T) == 8, cplx, epi, d.fd.M * (d.fd_blocks / d.fd.tiles)), st);
#define GPE_FD_CASE(E)                                                                                   \
  case E:                                                                                                \
    if (cplx) k_fd<T, true, E><<<d.fd_blocks, NTHREADS, 0, st>>>(d.fd, rx, ry, D);                        \
    else k_fd<T, false, E><<<d.fd_blocks, NTHREADS, 0, st>>>(d.fd, rx, ry, D);                            \
    break;
  switch (epi) {
    GPE_FD_CASE(EPI_GRAD)
    GPE_FD_CASE(EPI_HESS)
    GPE_FD_CASE(EPI_F)
    GPE_FD_CASE(EPI_W)
    GPE_FD_CASE(EPI_RATIO)
    default:
      return fail(GPE_EINVAL, "unknown FD epilogue");
  }
#undef GPE_FD_CASE
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

static inline int ew_blocks(long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + NTHREADS - 1) / NTHREADS, 152 * 8));
}

template <typename T>
gpe_status launch_step(void* const* xs, void* const* gs, const Alg1Ctl* ctl, long long n, int cplx, cudaStream_t st,
                       const void* xk) {
  ProfScope ps(kernel_name("step", sizeof(T) == 8, cplx, -1, n), st);
  if (cplx) k_step<T, true><<<ew_blocks(n), NTHREADS, 0, st>>>(xs, gs, ctl, n, xk);
  else k_step<T, false><<<ew_blocks(n), NTHREADS, 0, st>>>(xs, gs, ctl, n, xk);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

template <typename T>
gpe_status launch_moments(const void* x, const void* g, long long M, int nbatch, int cplx, Scratch& sc,
                          cudaStream_t st) {
  const int tiles = (int)std::max<long long>(1, std::min<long long>((M + NTHREADS - 1) / NTHREADS, 512));
  if ((size_t)tiles * nbatch > sc.cap_blocks) return fail(GPE_EINVAL, "reduction scratch too small");
  ProfScope ps(kernel_name("moments", sizeof(T) == 8, cplx, -1), st);
  if (cplx) k_moments<T, true><<<tiles * nbatch, NTHREADS, 0, st>>>(x, g, M, tiles, sc.partials, sc.results, sc.ticket);
  else k_moments<T, false><<<tiles * nbatch, NTHREADS, 0, st>>>(x, g, M, tiles, sc.partials, sc.results, sc.ticket);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

template <typename T>
gpe_status launch_axpby(const void* x, const void* g, const double* coef, int stride_coef, long long M, int nbatch,
                        void* out, int cplx, cudaStream_t st) {
  const long long n = M * nbatch;
  ProfScope ps(kernel_name("axpby", sizeof(T) == 8, cplx, -1), st);
  if (cplx) k_axpby<T, true><<<ew_blocks(n), NTHREADS, 0, st>>>(x, g, coef, stride_coef, M, nbatch, out);
  else k_axpby<T, false><<<ew_blocks(n), NTHREADS, 0, st>>>(x, g, coef, stride_coef, M, nbatch, out);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

template <typename T>
gpe_status launch_inject(const GridHost& gf, const GridHost& gc, const void* f, void* c, cudaStream_t st) {
  const int dirichlet = gf.disc == GPE_FOURIER ? 0 : 1;
  const int r = gf.N[0] / gc.N[0];
  for (int a = 0; a < gf.dim; ++a)
    if (gf.N[a] != r * gc.N[a]) return fail(GPE_EINVAL, "injection needs the same refinement on every axis");
  const long long n = gc.M * gc.nbatch;
  ProfScope ps(kernel_name("inject", sizeof(T) == 8, gf.is_complex, -1), st);
  if (gf.is_complex)
    k_inject<T, true><<<ew_blocks(n), NTHREADS, 0, st>>>(f, c, gf.dim, gf.ext[0], gf.ext[1], gc.ext[0], gc.ext[1], r,
                                                         dirichlet, gf.M, gc.M, gc.nbatch);
  else
    k_inject<T, false><<<ew_blocks(n), NTHREADS, 0, st>>>(f, c, gf.dim, gf.ext[0], gf.ext[1], gc.ext[0], gc.ext[1], r,
                                                          dirichlet, gf.M, gc.M, gc.nbatch);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

template <typename T>
gpe_status launch_prolong(const GridHost& gc, const GridHost& gf, const GridDev<T>& dc, const GridDev<T>& df,
                          const void* in, void* out, void* tmp1, void* tmp2, cudaStream_t st) {
  int ext[3] = {gc.ext[0], gc.ext[1], gc.ext[2]};
  const void* src = in;
  for (int a = 0; a < gc.dim; ++a) {
    void* dst = (a == gc.dim - 1) ? out : ((a & 1) ? tmp2 : tmp1);
    int oext[3] = {ext[0], ext[1], ext[2]};
    oext[a] = gf.ext[a];
    const long long Mc = (long long)ext[0] * ext[1] * ext[2];
    const long long Mf = (long long)oext[0] * oext[1] * oext[2];
    ProfScope ps(kernel_name("prolong", sizeof(T) == 8, gc.is_complex, -1), st);
    if (gc.disc == GPE_FD) {
      const long long n = Mf * gc.nbatch;
      if (gc.is_complex)
        k_prolong_fd_axis<T, true><<<ew_blocks(n), NTHREADS, 0, st>>>(src, dst, a, ext[0], ext[1], ext[2], gc.ext[a],
                                                                      gf.ext[a], Mc, Mf, gc.nbatch);
      else
        k_prolong_fd_axis<T, false><<<ew_blocks(n), NTHREADS, 0, st>>>(src, dst, a, ext[0], ext[1], ext[2], gc.ext[a],
                                                                       gf.ext[a], Mc, Mf, gc.nbatch);
    } else {
      int blocks;
      size_t smem;
      PassGeom<T> G = make_geom<T>(a, ext, gc.F[a], gf.F[a], gc.disc == GPE_SINE, gc.is_complex, gc.nbatch, &blocks,
                                   &smem);
      G.tw = dc.tw[a];
      G.lam = dc.lam[a];
      const long long stride_f = a == 0 ? 1 : (a == 1 ? (long long)oext[0] : (long long)oext[0] * oext[1]);
      const long long ostride_f = a == 1 ? (long long)oext[0] * oext[1] : (long long)oext[0];
      const int Ff = gf.F[a];
      if (gc.is_complex) {
        static size_t allowed_c = 0;
        if (smem > allowed_c) { GPE_CUDA(allow_smem(k_prolong_axis<T, true>, smem)); allowed_c = smem; }
        k_prolong_axis<T, true><<<blocks, NTHREADS, smem, st>>>(G, Ff, ilog2(Ff), df.tw[a], gf.ext[a], stride_f,
                                                                ostride_f, Mf, src, dst);
      } else {
        static size_t allowed_r = 0;
        if (smem > allowed_r) { GPE_CUDA(allow_smem(k_prolong_axis<T, false>, smem)); allowed_r = smem; }
        k_prolong_axis<T, false><<<blocks, NTHREADS, smem, st>>>(G, Ff, ilog2(Ff), df.tw[a], gf.ext[a], stride_f,
                                                                 ostride_f, Mf, src, dst);
      }
    }
    GPE_CUDA(cudaGetLastError());
    ext[a] = gf.ext[a];
    src = dst;
  }
  return GPE_OK;
}

// 2D Fourier grids: the register-FFT line kernels (lines2d.cuh); *handled is
// false for shapes they do not cover.
template <typename T>
gpe_status launch_lines2d(const GridHost& g, const GridDev<T>& d, const PassData<T>& D, int epi, void* acc,
                          bool step_first, cudaStream_t st, bool* handled);

template <typename T>
gpe_status apply_op(const GridHost& g, const GridDev<T>& d, PassData<T> D, int epi, void* acc, bool step_first,
                    cudaStream_t st) {
  if (g.disc == GPE_FOURIER && g.dim == 2) {
    bool handled = false;
    gpe_status s = launch_lines2d<T>(g, d, D, epi, acc, step_first, st, &handled);
    if (s != GPE_OK || handled) return s;
  }
  if (g.disc == GPE_FD) {
    if (step_first) {
      gpe_status s = launch_step<T>(D.xs, D.gs, D.ctl, g.M * g.nbatch, g.is_complex, st, nullptr);
      if (s != GPE_OK) return s;
    }
    return launch_fd<T>(d, D, g.is_complex, epi, st);
  }
  for (int a = 0; a < g.dim; ++a) {
    PassData<T> Da = D;
    Da.step_on_load = (step_first && a == 0) ? 1 : 0;
    Da.acc_in = a > 0 ? acc : nullptr;
    gpe_status s;
    if (a < g.dim - 1) {
      Da.out = acc;
      Da.nq = 0;
      Da.control = 0;
      s = launch_pass<T>(d, a, Da, g.is_complex, EPI_ACC, st);
    } else {
      s = launch_pass<T>(d, a, Da, g.is_complex, epi, st);
    }
    if (s != GPE_OK) return s;
  }
  return GPE_OK;
}

// Launch shape of the persistent Algorithm 1 kernel: dynamic shared memory for
// the largest axis pass and as many CTAs as fit co-resident (<= the largest
// pass's tile count).  grid = 0 if the grid is not spectral.
template <typename T>
gpe_status persist_config(const GridHost& g, const GridDev<T>& d, int epi, int* grid, size_t* smem_out) {
  using C = typename C2t<T>::type;
  *grid = 0;
  *smem_out = 0;
  if (g.disc == GPE_FD) return GPE_OK;
  const size_t vsz = sizeof(T) * (g.is_complex ? 2 : 1);
  size_t smem = 0, twb = 0;
  int maxb = 1;
  for (int a = 0; a < g.dim; ++a) {
    const PassGeom<T>& G = d.geom[a];
    const size_t b = (size_t)G.F * sizeof(C) + 2 * (size_t)G.LC * G.P * sizeof(C) + 2 * (size_t)G.LB * G.len * vsz +
                     (size_t)G.LB * G.len * sizeof(T);
    smem = std::max(smem, b);
    twb += (size_t)G.F * sizeof(C);
    maxb = std::max(maxb, d.blocks[a]);
  }
  twb = (twb + 15) & ~(size_t)15;
  smem += twb;
  int dev = 0, nsm = 0, occ = 0;
  GPE_CUDA(cudaGetDevice(&dev));
  GPE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  GPE_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return GPE_OK;
  const void* fn = nullptr;
  if (epi == EPI_F) fn = g.is_complex ? (const void*)k_alg1_persist<T, true, EPI_F> : (const void*)k_alg1_persist<T, false, EPI_F>;
  else fn = g.is_complex ? (const void*)k_alg1_persist<T, true, EPI_W> : (const void*)k_alg1_persist<T, false, EPI_W>;
  GPE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GPE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NTHREADS, smem));
  if (occ < 1) return GPE_OK;
  *grid = std::min(maxb, occ * nsm);
  *smem_out = smem;
  return GPE_OK;
}

template <typename T>
gpe_status launch_alg1_persist(const GridHost& g, const GridDev<T>& d, const PassData<T>& D, void* acc,
                               unsigned int* bar, int* err, int max_loops, int epi, int grid, size_t smem,
                               cudaStream_t st) {
  PersistArgs<T> P{};
  for (int a = 0; a < g.dim; ++a) {
    P.G[a] = d.geom[a];
    P.blocks[a] = d.blocks[a];
  }
  P.dim = g.dim;
  P.D = D;
  P.acc = acc;
  P.bar = bar;
  P.err = err;
  P.max_loops = max_loops;
  P.max_polls = wait_limit(1LL << 22);
  size_t twb = 0;
  for (int a = 0; a < g.dim; ++a) twb += (size_t)d.geom[a].F * sizeof(typename C2t<T>::type);
  P.tw_bytes = (twb + 15) & ~(size_t)15;
  P.dbg = persist_debug_buffer(&P.dbg_n);
  GPE_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), st));
  GPE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  void* args[] = {&P};
  const void* fn = nullptr;
  if (epi == EPI_F) fn = g.is_complex ? (const void*)k_alg1_persist<T, true, EPI_F> : (const void*)k_alg1_persist<T, false, EPI_F>;
  else fn = g.is_complex ? (const void*)k_alg1_persist<T, true, EPI_W> : (const void*)k_alg1_persist<T, false, EPI_W>;
  ProfScope ps(kernel_name("persist", sizeof(T) == 8, g.is_complex, epi, g.M), st);
  GPE_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(NTHREADS), args, smem, st));
  return GPE_OK;
}

#define GPE_INSTANTIATE(T)                                                                                         \
  template struct GridDev<T>;                                                                                      \
  template gpe_status launch_pass<T>(const GridDev<T>&, int, const PassData<T>&, int, int, cudaStream_t);          \
  template gpe_status launch_fd<T>(const GridDev<T>&, const PassData<T>&, int, int, cudaStream_t);                  \
  template gpe_status launch_step<T>(void* const*, void* const*, const Alg1Ctl*, long long, int, cudaStream_t,      \
                                     const void*);                                                                 \
  template gpe_status launch_moments<T>(const void*, const void*, long long, int, int, Scratch&, cudaStream_t);     \
  template gpe_status launch_axpby<T>(const void*, const void*, const double*, int, long long, int, void*, int,     \
                                      cudaStream_t);                                                               \
  template gpe_status launch_inject<T>(const GridHost&, const GridHost&, const void*, void*, cudaStream_t);         \
  template gpe_status launch_prolong<T>(const GridHost&, const GridHost&, const GridDev<T>&, const GridDev<T>&,     \
                                        const void*, void*, void*, void*, cudaStream_t);                           \
  template gpe_status apply_op<T>(const GridHost&, const GridDev<T>&, PassData<T>, int, void*, bool, cudaStream_t); \
  template gpe_status persist_config<T>(const GridHost&, const GridDev<T>&, int, int*, size_t*);                      \
  template gpe_status launch_alg1_persist<T>(const GridHost&, const GridDev<T>&, const PassData<T>&, void*,         \
                                             unsigned int*, int*, int, int, int, size_t, cudaStream_t);

}  // namespace gpe
