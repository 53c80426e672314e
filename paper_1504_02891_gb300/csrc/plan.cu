// plan.cu -- plans, grids and the operator entry points of the C ABI.
#include <math.h>
#include <string.h>
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include "gpe_internal.h"

namespace gpe {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

gpe_status fail(gpe_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

gpe_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? GPE_ENOMEM : GPE_ECUDA;
}

// ---------------------------------------------------------------- instrumentation
static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
struct ProfRec {
  std::string name;
  cudaEvent_t a = nullptr, b = nullptr;
};
static std::vector<ProfRec> g_recs;

void instr_count(long long n) { g_launches += n; }
bool prof_enabled() { return g_prof.load(); }

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

ProfScope::ProfScope(const char* name, cudaStream_t s) {
  st = s;
  if (capturing(s)) return;   // counted when the graph is launched
  g_launches += 1;
  if (!g_prof.load()) return;
  ProfRec r;
  r.name = name;
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
  cudaEventRecord(r.a, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  slot = (int)g_recs.size();
  g_recs.push_back(r);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < (int)g_recs.size()) cudaEventRecord(g_recs[slot].b, st);
}

const char* kernel_name(const char* base, int f64, int cplx, int epi, long long points) {
  static const char* epis[] = {"acc", "grad", "hess", "F", "W", "ratio", "WS"};
  static std::mutex mu;
  static std::map<std::string, std::string> names;
  std::string k = std::string(base) + (f64 ? "_f64" : "_f32") + (cplx ? "_c" : "_r");
  if (epi >= 0 && epi < 7) k += std::string("_") + epis[epi];
  if (points >= 0) k += "@" + std::to_string(points);
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(k);
  if (it == names.end()) it = names.emplace(k, k).first;
  return it->second.c_str();
}

static void prof_clear() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_recs) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  g_recs.clear();
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Grid, nodes and potential of §2 from the ABI problem (float64 on the host).
gpe_status grid_from_problem(const gpe_problem* p, int nbatch, GridHost& g) {
  if (!p) return fail(GPE_EINVAL, "problem is NULL");
  if (p->dim < 1 || p->dim > 3) return fail(GPE_EINVAL, "dim must be 1, 2 or 3");
  if (nbatch < 1) return fail(GPE_EINVAL, "nbatch must be >= 1");
  if (p->disc < GPE_FOURIER || p->disc > GPE_FD) return fail(GPE_EINVAL, "unknown discretisation");
  if (p->omega != 0.0) {
    if (!p->is_complex) return fail(GPE_EINVAL, "Omega != 0 needs a complex field");
    if (p->dim < 2) return fail(GPE_EINVAL, "Omega != 0 needs dim >= 2");
    if (p->disc == GPE_SINE) return fail(GPE_EINVAL, "the sine discretisation is for Omega = 0 only");
  }
  if (!(isfinite(p->beta) && isfinite(p->omega))) return fail(GPE_EINVAL, "beta/omega not finite");
  g = GridHost();
  g.dim = p->dim;
  g.disc = p->disc;
  g.is_complex = p->is_complex ? 1 : 0;
  g.nbatch = nbatch;
  g.beta = p->beta;
  g.omega = p->omega;
  g.v_kind = p->v_kind;
  memcpy(g.v_param, p->v_param, sizeof(g.v_param));
  g.M = 1;
  g.hvol = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (a >= p->dim) {
      g.N[a] = 1;
      g.ext[a] = 1;
      g.F[a] = 0;
      continue;
    }
    const int n = p->n[a];
    if (!(p->hi[a] > p->lo[a]) || !isfinite(p->lo[a]) || !isfinite(p->hi[a]))
      return fail(GPE_EINVAL, "box must satisfy lo < hi");
    if (p->disc == GPE_FOURIER) {
      if (!is_pow2(n) || n < 4 || n > 1024) return fail(GPE_EINVAL, "Fourier n must be a power of two in [4, 1024]");
      g.ext[a] = n;
      g.F[a] = n;
    } else if (p->disc == GPE_SINE) {
      if (!is_pow2(n) || n < 4 || n > 512) return fail(GPE_EINVAL, "sine n must be a power of two in [4, 512]");
      g.ext[a] = n - 1;
      g.F[a] = 2 * n;
    } else {
      if (n < 3) return fail(GPE_EINVAL, "FD n must be >= 3");
      g.ext[a] = n - 1;
      g.F[a] = 0;
    }
    g.N[a] = n;
    g.lo[a] = p->lo[a];
    g.hi[a] = p->hi[a];
    g.h[a] = (p->hi[a] - p->lo[a]) / n;
    g.hvol *= g.h[a];
    g.M *= g.ext[a];
    g.nodes[a].resize(g.ext[a]);
    const int j0 = p->disc == GPE_FOURIER ? 0 : 1;
    for (int i = 0; i < g.ext[a]; ++i) g.nodes[a][i] = p->lo[a] + (double)(i + j0) * g.h[a];
  }
  if (g.M > (1LL << 31)) return fail(GPE_EINVAL, "grid too large");
  g.V.resize(g.M);
  if (p->v_kind == GPE_V_ARRAY) {
    if (!p->v_host) return fail(GPE_EINVAL, "GPE_V_ARRAY needs v_host");
    for (long long i = 0; i < g.M; ++i) g.V[i] = p->v_host[i];
  } else if (p->v_kind < GPE_V_HARMONIC || p->v_kind > GPE_V_STIRRER) {
    return fail(GPE_EINVAL, "unknown potential kind");
  } else {
    const double* q = p->v_param;
    for (long long i = 0; i < g.M; ++i) {
      const int i0 = (int)(i % g.ext[0]);
      const int i1 = (int)((i / g.ext[0]) % g.ext[1]);
      const int i2 = (int)(i / ((long long)g.ext[0] * g.ext[1]));
      const int idx[3] = {i0, i1, i2};
      double x[3] = {0, 0, 0};
      for (int a = 0; a < g.dim; ++a) x[a] = g.nodes[a][idx[a]];
      double v = 0.0;
      for (int a = 0; a < g.dim; ++a) v += 0.5 * q[a] * q[a] * x[a] * x[a];
      if (p->v_kind == GPE_V_LATTICE) {
        for (int a = 0; a < g.dim; ++a) {
          const double s = sin(q[4] * x[a]);
          v += q[3] * s * s;
        }
      } else if (p->v_kind == GPE_V_STIRRER) {
        const double dx = x[0] - q[5];
        v += q[3] * exp(-q[4] * (dx * dx + x[1] * x[1]));
      }
      g.V[i] = v;
    }
    for (long long i = 0; i < g.M; ++i)
      if (!isfinite(g.V[i])) return fail(GPE_EINVAL, "potential not finite");
  }
  return GPE_OK;
}

// The same problem on a mesh coarsened `levels_down` times (N halved per level).
GridHost grid_coarsen(const GridHost& f, int levels_down) {
  gpe_problem p{};
  p.dim = f.dim;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = a < f.dim ? (f.N[a] >> levels_down) : 1;
    p.lo[a] = f.lo[a];
    p.hi[a] = f.hi[a];
  }
  p.disc = f.disc;
  p.beta = f.beta;
  p.omega = f.omega;
  p.is_complex = f.is_complex;
  p.v_kind = f.v_kind;
  memcpy(p.v_param, f.v_param, sizeof(p.v_param));
  GridHost g;
  grid_from_problem(&p, f.nbatch, g);
  return g;
}

gpe_status Scratch::create(size_t blocks, int nb) {
  cap_blocks = blocks;
  nbatch = nb;
  GPE_CUDA(cudaMalloc(&partials, sizeof(double) * NQ * blocks));
  GPE_CUDA(cudaMalloc(&results, sizeof(double) * NQ * nb));
  GPE_CUDA(cudaMalloc(&coef, sizeof(double) * 4 * nb));
  GPE_CUDA(cudaMalloc(&ticket, sizeof(unsigned int)));
  GPE_CUDA(cudaMemset(ticket, 0, sizeof(unsigned int)));
  GPE_CUDA(cudaMemset(results, 0, sizeof(double) * NQ * nb));
  GPE_CUDA(cudaMallocHost(&h_results, sizeof(double) * NQ * nb));
  return GPE_OK;
}

void Scratch::destroy() {
  cudaFree(partials);
  cudaFree(results);
  cudaFree(coef);
  cudaFree(ticket);
  cudaFreeHost(h_results);
  partials = results = coef = nullptr;
  ticket = nullptr;
  h_results = nullptr;
}

}  // namespace gpe

using namespace gpe;

static void plan_free(gpe_plan p) {
  if (!p) return;
  if (p->d32) { p->d32->destroy(); delete p->d32; }
  if (p->d64) { p->d64->destroy(); delete p->d64; }
  if (p->solver_cache) destroy_solver_cache(p->solver_cache);
  p->sc.destroy();
  cudaFree(p->acc);
  cudaFree(p->tmp);
  delete p;
}

extern "C" const char* gpe_last_error(void) { return gpe::g_last_error.c_str(); }

extern "C" gpe_status gpe_plan_create(const gpe_problem* prob, int nbatch, int prec, void* stream, gpe_plan* out) {
  if (!out) return fail(GPE_EINVAL, "out is NULL");
  *out = nullptr;
  if (prec != GPE_F32 && prec != GPE_F64) return fail(GPE_EINVAL, "prec must be GPE_F32 or GPE_F64");
  gpe_plan p = new gpe_plan_s();
  gpe_status s = grid_from_problem(prob, nbatch, p->g);
  if (s != GPE_OK) { delete p; return s; }
  p->prec = prec;
  p->stream = (cudaStream_t)stream;
  cudaGetDevice(&p->device);
  int max_blocks = 0;
  if (prec == GPE_F32) {
    p->d32 = new GridDev<float>();
    s = p->d32->create(p->g);
    max_blocks = p->d32->max_blocks;
  } else {
    p->d64 = new GridDev<double>();
    s = p->d64->create(p->g);
    max_blocks = p->d64->max_blocks;
  }
  if (s == GPE_OK) s = p->sc.create(max_blocks, nbatch);
  const size_t bytes = elem_size(prec, p->g.is_complex) * p->g.M * nbatch;
  if (s == GPE_OK) {
    cudaError_t e = cudaMalloc(&p->acc, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->tmp, bytes);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMalloc(workspace)");
  }
  if (s != GPE_OK) { plan_free(p); return s; }
  *out = p;
  return GPE_OK;
}

extern "C" gpe_status gpe_plan_destroy(gpe_plan plan) {
  if (!plan) return GPE_OK;
  cudaStreamSynchronize(plan->stream);
  plan_free(plan);
  return GPE_OK;
}

extern "C" gpe_status gpe_plan_size(gpe_plan plan, int64_t* n_unknowns, double* h_vol) {
  if (!plan) return fail(GPE_EINVAL, "plan is NULL");
  if (n_unknowns) *n_unknowns = plan->g.M;
  if (h_vol) *h_vol = plan->g.hvol;
  return GPE_OK;
}

template <typename T>
static PassData<T> abi_data(gpe_plan p, const GridDev<T>& d) {
  PassData<T> D{};
  D.V = d.V;
  D.nl = p->g.beta;
  D.lin_scale = 1.0;
  D.partials = p->sc.partials;
  D.results = p->sc.results;
  D.ticket = p->sc.ticket;
  return D;
}

// E, mu, norm2 from the GRAD-epilogue sums of each instance.
static gpe_status read_energy(gpe_plan p, double* E, double* mu, double* norm2) {
  const int nb = p->g.nbatch;
  GPE_CUDA(cudaMemcpyAsync(p->sc.h_results, p->sc.results, sizeof(double) * NQ * nb, cudaMemcpyDeviceToHost, p->stream));
  GPE_CUDA(cudaStreamSynchronize(p->stream));
  gpe_status st = GPE_OK;
  // a bounded task wait of the fused 2D kernel that gave up leaves its flag set
  // (and NaN partial sums): report it as the expired wait it was, then clear it
  unsigned int* fs = p->prec == GPE_F32 ? p->d32->fsync : p->d64->fsync;
  if (fs) {
    unsigned int flag = 0;
    GPE_CUDA(cudaMemcpy(&flag, fs + 2 + 2 * (size_t)nb, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) {
      GPE_CUDA(cudaMemset(fs + 2 + 2 * (size_t)nb, 0, sizeof(flag)));
      return fail(GPE_ETIMEOUT, "a bounded task wait of the fused 2D operator kernel expired");
    }
  }
  for (int b = 0; b < nb; ++b) {
    const double* r = p->sc.h_results + (size_t)b * NQ;
    const double e2 = r[0], e4 = r[1], n2 = r[2];
    const double h = p->g.hvol;
    if (E) E[b] = h * (e2 + 0.5 * p->g.beta * e4);
    if (mu) mu[b] = h * (e2 + p->g.beta * e4);
    if (norm2) norm2[b] = h * n2;
    if (!isfinite(e2) || !isfinite(e4)) st = fail(GPE_ENONFINITE, "energy reduction is not finite");
  }
  return st;
}

template <typename T>
static gpe_status do_grad(gpe_plan p, const GridDev<T>& d, const void* psi, void* hpsi) {
  PassData<T> D = abi_data<T>(p, d);
  D.x = psi;
  D.out = hpsi;
  D.nq = 3;
  return apply_op<T>(p->g, d, D, EPI_GRAD, p->acc, false, p->stream);
}

extern "C" gpe_status gpe_energy(gpe_plan p, const void* psi, double* E, double* mu, double* norm2) {
  if (!p || !psi) return fail(GPE_EINVAL, "plan or psi is NULL");
  gpe_status s = p->prec == GPE_F32 ? do_grad<float>(p, *p->d32, psi, nullptr) : do_grad<double>(p, *p->d64, psi, nullptr);
  if (s != GPE_OK) return s;
  return read_energy(p, E, mu, norm2);
}

extern "C" gpe_status gpe_grad(gpe_plan p, const void* psi, void* hpsi, double* E, double* mu) {
  if (!p || !psi || !hpsi) return fail(GPE_EINVAL, "plan, psi or hpsi is NULL");
  if (psi == hpsi) return fail(GPE_EINVAL, "hpsi must not alias psi");
  gpe_status s = p->prec == GPE_F32 ? do_grad<float>(p, *p->d32, psi, hpsi) : do_grad<double>(p, *p->d64, psi, hpsi);
  if (s != GPE_OK) return s;
  if (E || mu) return read_energy(p, E, mu, nullptr);
  return GPE_OK;
}

template <typename T>
static gpe_status do_hess(gpe_plan p, const GridDev<T>& d, const void* psi, const void* dir, double shift, void* out) {
  PassData<T> D = abi_data<T>(p, d);
  D.x = dir;
  D.base = psi;
  D.shift = shift;
  D.out = out;
  D.nq = 0;
  return apply_op<T>(p->g, d, D, EPI_HESS, p->acc, false, p->stream);
}

extern "C" gpe_status gpe_hessvec(gpe_plan p, const void* psi, const void* dir, double shift, void* out) {
  if (!p || !psi || !dir || !out) return fail(GPE_EINVAL, "NULL argument");
  if (out == psi || out == dir) return fail(GPE_EINVAL, "out must not alias psi or d");
  if (!isfinite(shift)) return fail(GPE_EINVAL, "shift not finite");
  return p->prec == GPE_F32 ? do_hess<float>(p, *p->d32, psi, dir, shift, out)
                            : do_hess<double>(p, *p->d64, psi, dir, shift, out);
}

template <typename T>
static gpe_status do_step(gpe_plan p, const void* psi, const void* hpsi, double tau, void* out) {
  gpe_status s = launch_moments<T>(psi, hpsi, p->g.M, p->g.nbatch, p->g.is_complex, p->sc, p->stream);
  if (s != GPE_OK) return s;
  s = launch_step_coef(p->sc.results, p->g.nbatch, p->g.hvol, tau, p->sc.coef, p->stream);
  if (s != GPE_OK) return s;
  return launch_axpby<T>(psi, hpsi, p->sc.coef, 2, p->g.M, p->g.nbatch, out, p->g.is_complex, p->stream);
}

extern "C" gpe_status gpe_feasible_step(gpe_plan p, const void* psi, const void* hpsi, double tau, void* psi_out,
                                        double* E_out) {
  if (!p || !psi || !hpsi || !psi_out) return fail(GPE_EINVAL, "NULL argument");
  if (psi_out == psi || psi_out == hpsi) return fail(GPE_EINVAL, "psi_out must not alias psi or hpsi");
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(GPE_EINVAL, "tau must be finite and >= 0");
  gpe_status s = p->prec == GPE_F32 ? do_step<float>(p, psi, hpsi, tau, psi_out) : do_step<double>(p, psi, hpsi, tau, psi_out);
  if (s != GPE_OK) return s;
  if (E_out) return gpe_energy(p, psi_out, E_out, nullptr, nullptr);
  return GPE_OK;
}

template <typename T>
static gpe_status do_prolong(gpe_plan c, gpe_plan f, const GridDev<T>& dc, const GridDev<T>& df, const void* in, void* out) {
  gpe_status s = launch_prolong<T>(c->g, f->g, dc, df, in, out, f->acc, f->tmp, f->stream);
  if (s != GPE_OK) return s;
  s = launch_moments<T>(out, nullptr, f->g.M, f->g.nbatch, f->g.is_complex, f->sc, f->stream);
  if (s != GPE_OK) return s;
  s = launch_norm_coef(f->sc.results, f->g.nbatch, f->g.hvol, f->sc.coef, f->stream);
  if (s != GPE_OK) return s;
  return launch_axpby<T>(out, nullptr, f->sc.coef, 1, f->g.M, f->g.nbatch, out, f->g.is_complex, f->stream);
}

extern "C" gpe_status gpe_prolong(gpe_plan c, gpe_plan f, const void* psi_c, void* psi_f) {
  if (!c || !f || !psi_c || !psi_f) return fail(GPE_EINVAL, "NULL argument");
  const GridHost &gc = c->g, &gf = f->g;
  if (gc.dim != gf.dim || gc.disc != gf.disc || gc.is_complex != gf.is_complex || gc.nbatch != gf.nbatch ||
      c->prec != f->prec)
    return fail(GPE_EINVAL, "coarse and fine plans differ in dim/disc/complexity/batch/precision");
  for (int a = 0; a < gc.dim; ++a) {
    if (gf.N[a] != 2 * gc.N[a]) return fail(GPE_EINVAL, "fine n must be twice the coarse n on every axis");
    if (gc.lo[a] != gf.lo[a] || gc.hi[a] != gf.hi[a]) return fail(GPE_EINVAL, "boxes differ");
  }
  if (c->stream != f->stream) {
    cudaStreamSynchronize(c->stream);
  }
  return c->prec == GPE_F32 ? do_prolong<float>(c, f, *c->d32, *f->d32, psi_c, psi_f)
                            : do_prolong<double>(c, f, *c->d64, *f->d64, psi_c, psi_f);
}

extern "C" int64_t gpe_kernel_launches(void) { return (int64_t)g_launches.load(); }

namespace gpe {
static std::atomic<long long> g_wait_limit{0};
long long wait_limit(long long default_polls) {
  const long long v = g_wait_limit.load();
  return v > 0 ? v : default_polls;
}
}  // namespace gpe

namespace gpe {
static std::atomic<int> g_op_path{0};
int operator_path() { return g_op_path.load(); }
}  // namespace gpe

extern "C" gpe_status gpe_set_operator_path(int path) {
  if (path < 0 || path > 2) return fail(GPE_EINVAL, "path must be 0, 1 or 2");
  gpe::g_op_path.store(path);
  return GPE_OK;
}

extern "C" gpe_status gpe_set_wait_limit(int64_t polls) {
  if (polls < 0) return fail(GPE_EINVAL, "polls must be >= 0");
  gpe::g_wait_limit.store((long long)polls);
  return GPE_OK;
}

extern "C" gpe_status gpe_profile_enable(int on) {
  if (!on) prof_clear();
  g_prof = on != 0;
  return GPE_OK;
}

extern "C" gpe_status gpe_profile_summary(char* buf, int buflen) {
  if (!buf || buflen <= 0) return fail(GPE_EINVAL, "buffer is NULL");
  std::map<std::string, std::pair<long long, double>> agg;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_recs) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess) continue;
      if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
      auto& e = agg[r.name];
      e.first += 1;
      e.second += ms;
    }
  }
  std::string out = "{";
  bool first = true;
  char tmp[256];
  for (auto& kv : agg) {
    snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(), kv.second.first,
             kv.second.second);
    out += tmp;
    first = false;
  }
  out += "}";
  snprintf(buf, buflen, "%s", out.c_str());
  return GPE_OK;
}

extern "C" gpe_status gpe_solve_opts_default(gpe_solve_opts* o) {
  if (!o) return fail(GPE_EINVAL, "opts is NULL");
  memset(o, 0, sizeof(*o));
  o->levels = 1;
  o->mode = 1;
  o->method = 0;
  o->k_init = 100;
  o->k_sub = 200;
  o->max_outer = 200;
  o->max_iter = 2000;
  o->eps0 = 1e-6;
  o->delta_stop = 1e-8;
  o->res_tol = 1e-9;
  o->delta0 = 1.0;
  o->switch_rel = 1e-6;
  o->chunk = 16;
  o->use_graphs = 1;
  o->persistent = 1;
  o->cluster = 1;
  o->search = 0;
  o->alpha_hat = 1e-3;
  o->eta = 0.85;
  return GPE_OK;
}
