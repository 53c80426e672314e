// autotune.cu -- measured launch shapes.
//
// Two choices are made by timing candidates on the device instead of by a fixed
// rule, and kept in a process-wide table keyed by the grid (and batch):
//   * the register-FFT line kernels of 2D Fourier grids: how many resident
//     waves of CTAs the y-kernel (columns) and the x-kernel (rows, epilogue,
//     reduction) are launched with (1, 2, 4 or 8; the CTAs stride over the
//     remaining line groups);
//   * the cluster engine of single float32 solves on 2D Fourier grids: the
//     per-CTA share of one state vector (2-32 KiB), which sets the cluster
//     size (smaller share: more CTAs per instance, shorter line passes, more
//     cluster-wide synchronisation).
//   * float32 square 2D Fourier grids: the fused one-launch operator kernel
//     (fused2d.cuh) or the two line kernels, whichever applies the operator
//     faster for the grid and batch.
// Launches with no table entry use the fixed rule (4 waves; 4 KiB; the fused
// kernel for batches of >= 16 instances on grids up to 256^2).  The
// choice never changes what is computed, only how the work is spread: the
// operator values are identical, reductions may differ by rounding order.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gpe_internal.h"

namespace gpe {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_waves;   // (prec, cplx, n0, n1, nbatch)
std::map<std::tuple<int, int, int>, int> g_share;                            // (n0, n1, cplx)
std::map<std::tuple<int, int, int>, int> g_fused;                            // (cplx, n, nbatch)
}  // namespace

bool tuned_fused(int cplx, int n, int nbatch) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_fused.find(std::make_tuple(cplx, n, nbatch));
  // without a measurement: the fused kernel for batches on grids up to 256^2
  // (faster there on GB300; a single instance waits for its own y-tasks and
  // is faster with the two line kernels, and so are 512^2 and 1024^2 lines)
  if (it == g_fused.end()) return n <= 256 && nbatch >= 16;
  return it->second != 0;
}

void set_tuned_fused(int cplx, int n, int nbatch, int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_fused[std::make_tuple(cplx, n, nbatch)] = on;
}

int tuned_waves(int axis, int prec64, int cplx, int n0, int n1, int nbatch) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_waves.find(std::make_tuple(prec64, cplx, n0, n1, nbatch));
  if (it == g_waves.end()) return 4;
  return axis == 0 ? it->second.first : it->second.second;
}

void set_tuned_waves(int prec64, int cplx, int n0, int n1, int nbatch, int wx, int wy) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_waves[std::make_tuple(prec64, cplx, n0, n1, nbatch)] = std::make_pair(wx, wy);
}

int tuned_share_kb(int n0, int n1, int cplx) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_share.find(std::make_tuple(n0, n1, cplx));
  return it == g_share.end() ? 4 : it->second;
}

void set_tuned_share_kb(int n0, int n1, int cplx, int kb) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_share[std::make_tuple(n0, n1, cplx)] = kb;
}

// Mean time of `reps` H-applies (gpe_grad, no host read-back) on the plan's stream.
static gpe_status time_grad(gpe_plan p, const void* x, void* y, int reps, float* us) {
  cudaEvent_t e0, e1;
  GPE_CUDA(cudaEventCreate(&e0));
  GPE_CUDA(cudaEventCreate(&e1));
  gpe_status s = GPE_OK;
  for (int i = 0; i < 2 && s == GPE_OK; ++i) s = gpe_grad(p, x, y, nullptr, nullptr);
  if (s == GPE_OK) {
    cudaEventRecord(e0, p->stream);
    for (int i = 0; i < reps && s == GPE_OK; ++i) s = gpe_grad(p, x, y, nullptr, nullptr);
    cudaEventRecord(e1, p->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *us = 1e3f * ms / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == GPE_OK) GPE_CUDA(cudaGetLastError());
  return s;
}

static gpe_status tune_lines(gpe_plan p, std::string& rep) {
  const GridHost& g = p->g;
  const bool f64 = p->prec == GPE_F64;
  auto pow2 = [](int n) { return n >= 64 && n <= 1024 && (n & (n - 1)) == 0; };
  if (g.disc != GPE_FOURIER || g.dim != 2 || !pow2(g.ext[0]) || !pow2(g.ext[1])) return GPE_OK;
  const size_t bytes = (f64 ? 8 : 4) * (g.is_complex ? 2 : 1) * (size_t)g.M * g.nbatch;
  void* x = nullptr;
  void* y = nullptr;
  GPE_CUDA(cudaMalloc(&x, bytes));
  gpe_status s = GPE_OK;
  if (cudaMalloc(&y, bytes) != cudaSuccess) {
    cudaFree(x);
    return fail(GPE_ENOMEM, "autotune scratch");
  }
  // finite data: bytes 0x3c give float32 0.0115 and float64 1.6e-19 everywhere
  cudaMemsetAsync(x, 0x3c, bytes, p->stream);
  const int n0 = g.ext[0], n1 = g.ext[1], nb = g.nbatch, c = g.is_complex, pr = f64 ? 1 : 0;
  const int wx0 = tuned_waves(0, pr, c, n0, n1, nb), wy0 = tuned_waves(1, pr, c, n0, n1, nb);
  // the waves are those of the two line kernels: time them, not the fused kernel
  const bool sq = !f64 && n0 == n1;
  const bool fused0 = sq && tuned_fused(c, n0, nb);
  if (sq) set_tuned_fused(c, n0, nb, 0);
  const int cand[4] = {1, 2, 4, 8};
  int wx = 4, wy = 4;
  float best = 1e30f, t = 0.f;
  const int reps = 5;
  // columns first with the rows at the fixed rule, then the rows
  for (int i = 0; i < 4 && s == GPE_OK; ++i) {
    set_tuned_waves(pr, c, n0, n1, nb, 4, cand[i]);
    s = time_grad(p, x, y, reps, &t);
    if (s == GPE_OK && t < best) { best = t; wy = cand[i]; }
  }
  best = 1e30f;
  for (int i = 0; i < 4 && s == GPE_OK; ++i) {
    set_tuned_waves(pr, c, n0, n1, nb, cand[i], wy);
    s = time_grad(p, x, y, reps, &t);
    if (s == GPE_OK && t < best) { best = t; wx = cand[i]; }
  }
  cudaStreamSynchronize(p->stream);
  cudaFree(x);
  cudaFree(y);
  if (sq) set_tuned_fused(c, n0, nb, fused0 ? 1 : 0);
  if (s != GPE_OK) {
    set_tuned_waves(pr, c, n0, n1, nb, wx0, wy0);   // leave the table as it was
    return s;
  }
  set_tuned_waves(pr, c, n0, n1, nb, wx, wy);
  char buf[200];
  snprintf(buf, sizeof(buf), "lines %s%s %dx%d nbatch %d: waves x %d y %d (%.1f us/apply); ", f64 ? "f64" : "f32",
           c ? " complex" : "", n0, n1, nb, wx, wy, best);
  rep += buf;
  return GPE_OK;
}

// Float32 square grids: the fused kernel against the two line kernels (with
// their tuned waves); the faster is recorded for the grid and batch.
static gpe_status tune_fused(gpe_plan p, std::string& rep) {
  const GridHost& g = p->g;
  if (p->prec != GPE_F32 || g.disc != GPE_FOURIER || g.dim != 2 || g.ext[0] != g.ext[1]) return GPE_OK;
  const int n = g.ext[0];
  if (n < 64 || n > 1024 || (n & (n - 1)) != 0 || operator_path() != 0) return GPE_OK;
  const size_t bytes = 4 * (g.is_complex ? 2 : 1) * (size_t)g.M * g.nbatch;
  void* x = nullptr;
  void* y = nullptr;
  GPE_CUDA(cudaMalloc(&x, bytes));
  if (cudaMalloc(&y, bytes) != cudaSuccess) {
    cudaFree(x);
    return fail(GPE_ENOMEM, "autotune scratch");
  }
  cudaMemsetAsync(x, 0x3c, bytes, p->stream);
  const int c = g.is_complex, nb = g.nbatch;
  const bool was = tuned_fused(c, n, nb);
  float t[2] = {0.f, 0.f};
  gpe_status s = GPE_OK;
  for (int on = 0; on < 2 && s == GPE_OK; ++on) {
    set_tuned_fused(c, n, nb, on);
    s = time_grad(p, x, y, 5, &t[on]);
  }
  cudaStreamSynchronize(p->stream);
  cudaFree(x);
  cudaFree(y);
  if (s != GPE_OK) {
    set_tuned_fused(c, n, nb, was ? 1 : 0);
    return s;
  }
  const int best = t[1] < t[0] ? 1 : 0;
  set_tuned_fused(c, n, nb, best);
  char buf[200];
  snprintf(buf, sizeof(buf), "operator f32%s %dx%d nbatch %d: %s (fused %.1f us, two kernels %.1f us); ",
           c ? " complex" : "", n, n, nb, best ? "fused kernel" : "two line kernels", t[1], t[0]);
  rep += buf;
  return GPE_OK;
}

}  // namespace gpe

using namespace gpe;

namespace {
std::string g_report;
std::mutex g_rep_mu;
}  // namespace

extern "C" gpe_status gpe_plan_autotune(gpe_plan plan, int levels) {
  if (!plan) return fail(GPE_EINVAL, "plan is NULL");
  if (levels < 1 || levels > 8) return fail(GPE_EINVAL, "levels must be in [1, 8]");
  std::string rep;
  gpe_status s = tune_lines(plan, rep);
  if (s != GPE_OK) return s;
  s = tune_fused(plan, rep);
  if (s != GPE_OK) return s;
  const GridHost& g = plan->g;
  if (g.disc == GPE_FOURIER && g.dim == 2 && g.v_kind != GPE_V_ARRAY) {
    for (int l = 0; l < levels; ++l) {
      const int n0 = g.N[0] >> l, n1 = g.N[1] >> l;
      if ((n0 << l) != g.N[0] || (n1 << l) != g.N[1] || n0 < 4 || n1 < 4) break;
      int kb = 0;
      double us = 0.0;
      s = tune_cluster_share(grid_coarsen(g, l), plan->stream, &kb, &us);
      if (s != GPE_OK) return s;
      if (kb > 0) {
        char buf[128];
        snprintf(buf, sizeof(buf), "cluster %dx%d%s: share %d KiB (%.2f us/trial); ", n0, n1,
                 g.is_complex ? " complex" : "", kb, us);
        rep += buf;
      }
    }
  }
  std::lock_guard<std::mutex> lk(g_rep_mu);
  g_report += rep;
  return GPE_OK;
}

extern "C" gpe_status gpe_autotune_report(char* buf, size_t buflen) {
  if (!buf || buflen == 0) return fail(GPE_EINVAL, "buf is NULL");
  std::lock_guard<std::mutex> lk(g_rep_mu);
  snprintf(buf, buflen, "%s", g_report.c_str());
  return GPE_OK;
}
