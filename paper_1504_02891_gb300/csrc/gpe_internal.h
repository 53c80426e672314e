// gpe_internal.h -- host-side internals of libgpe (grids, device tables,
// launch wrappers).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include "gpe_kernels.cuh"
#include "../../include/gpe.h"

namespace gpe {

// Thread-local error text behind gpe_last_error().
void set_error(const std::string& msg);
gpe_status fail(gpe_status st, const std::string& msg);
gpe_status cuda_fail(cudaError_t e, const char* what);

#define GPE_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Host description of one grid (FP64 tables, §2).
struct GridHost {
  int dim = 1;
  int N[3] = {1, 1, 1};     // paper's N per axis
  int ext[3] = {1, 1, 1};   // array extents (unknowns per axis)
  int F[3] = {0, 0, 0};     // FFT length per axis (0 for FD)
  int disc = 0, is_complex = 0, nbatch = 1;
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
  double hvol = 1.0, beta = 0.0, omega = 0.0;
  long long M = 1;
  int v_kind = 0;
  double v_param[8] = {0};
  std::vector<double> nodes[3];
  std::vector<double> V;
};

gpe_status grid_from_problem(const gpe_problem* p, int nbatch, GridHost& g);
GridHost grid_coarsen(const GridHost& g, int levels_down);

// Measured launch shapes (autotune.cu): resident waves of the line kernels
// (axis 0: x-kernel, 1: y-kernel; 4 without an entry) and the cluster
// engine's per-CTA share for single solves (4 KiB without an entry).
int tuned_waves(int axis, int prec64, int cplx, int n0, int n1, int nbatch);
void set_tuned_waves(int prec64, int cplx, int n0, int n1, int nbatch, int wx, int wy);
// Fused 2D operator kernel or two line kernels for a float32 square grid n x n
// (default without a measurement: fused for batches of >= 16 instances, n <= 256).
bool tuned_fused(int cplx, int n, int nbatch);
void set_tuned_fused(int cplx, int n, int nbatch, int on);
// gpe_set_operator_path: 0 automatic (measured or default choice), 1 the fused
// kernel wherever it applies, 2 the two line kernels.
int operator_path();
int tuned_share_kb(int n0, int n1, int cplx);
void set_tuned_share_kb(int n0, int n1, int cplx, int kb);
// Time the cluster engine's float32 Algorithm 1 on grid g for each distinct
// cluster size and record the fastest share (solver.cu); *kb = 0 if the grid
// does not run in the cluster engine.
gpe_status tune_cluster_share(const GridHost& g, cudaStream_t st, int* kb, double* us_per_trial);

// Device tables and launch geometry of one grid in precision T.
template <typename T>
struct GridDev {
  using C = typename C2t<T>::type;
  T* V = nullptr;
  C* tw[3] = {nullptr, nullptr, nullptr};
  T* lam[3] = {nullptr, nullptr, nullptr};
  T* coord[3] = {nullptr, nullptr, nullptr};
  PassGeom<T> geom[3];
  int blocks[3] = {0, 0, 0};
  size_t smem[3] = {0, 0, 0};
  FDGeom fd;
  int fd_blocks = 0;
  int max_blocks = 0;
  // 2D Fourier grids (fused warp-line kernel, fused2d.cuh): per axis the
  // twiddles e^{-2 pi i j k2 / F} in k2-major order (entry k2 * TPL + j, TPL
  // the threads per line), and the launch's counters: task counter, exited
  // warps, per-instance finished y- and x-tasks, error flag (zero between
  // launches; the last warp of a launch resets them)
  C* tw2[2] = {nullptr, nullptr};
  unsigned int* fsync = nullptr;
  gpe_status create(const GridHost& g);
  void destroy();
};

// Reduction scratch shared by the launches of one plan/level.
struct Scratch {
  double* partials = nullptr;
  double* results = nullptr;     // [nbatch][NQ]
  double* coef = nullptr;        // [nbatch][4]
  unsigned int* ticket = nullptr;
  double* h_results = nullptr;   // pinned mirror
  size_t cap_blocks = 0;
  int nbatch = 0;
  gpe_status create(size_t blocks, int nbatch);
  void destroy();
};

// Launch wrappers (explicitly instantiated for float and double).
template <typename T>
gpe_status launch_pass(const GridDev<T>& d, int axis, const PassData<T>& D, int cplx, int epi, cudaStream_t st);
template <typename T>
gpe_status launch_fd(const GridDev<T>& d, const PassData<T>& D, int cplx, int epi, cudaStream_t st);
template <typename T>
gpe_status launch_step(void* const* xs, void* const* gs, const Alg1Ctl* ctl, long long n, int cplx, cudaStream_t st,
                       const void* xk = nullptr);
template <typename T>
gpe_status launch_moments(const void* x, const void* g, long long M, int nbatch, int cplx, Scratch& sc,
                          cudaStream_t st);
template <typename T>
gpe_status launch_axpby(const void* x, const void* g, const double* coef, int stride_coef, long long M, int nbatch,
                        void* out, int cplx, cudaStream_t st);
template <typename T>
gpe_status launch_inject(const GridHost& gf, const GridHost& gc, const void* f, void* c, cudaStream_t st);
template <typename T>
gpe_status launch_prolong(const GridHost& gc, const GridHost& gf, const GridDev<T>& dc, const GridDev<T>& df,
                          const void* in, void* out, void* tmp1, void* tmp2, cudaStream_t st);
template <typename Ti, typename To>
gpe_status launch_convert(const Ti* in, To* out, long long n, double scale, cudaStream_t st);
gpe_status launch_step_coef(const double* mom, int nbatch, double h, double tau, double* coef, cudaStream_t st);
gpe_status launch_norm_coef(const double* mom, int nbatch, double h, double* coef, cudaStream_t st);
gpe_status launch_to_shifted_f32(const double* xk, const double* gk, double th, float* xk32, float* pk32, long long n,
                                 cudaStream_t st);
gpe_status launch_add_f32_to_f64(const double* xk, const float* d, double* z, long long n, cudaStream_t st);

// One operator application: the per-axis passes (or the FD stencil) with the
// epilogue `epi` on the last pass.  acc is a scratch vector of the grid's size.
template <typename T>
gpe_status apply_op(const GridHost& g, const GridDev<T>& d, PassData<T> D, int epi, void* acc, bool step_first,
                    cudaStream_t st);

template <typename T>
gpe_status persist_config(const GridHost& g, const GridDev<T>& d, int epi, int* grid, size_t* smem);
template <typename T>
gpe_status launch_alg1_persist(const GridHost& g, const GridDev<T>& d, const PassData<T>& D, void* acc,
                               unsigned int* bar, int* err, int max_loops, int epi, int grid, size_t smem,
                               cudaStream_t st);

// GPE_PERSIST_TRACE=1: phase timestamps of persistent launches (debug aid).
unsigned long long* persist_debug_buffer(int* n);
void persist_debug_report(cudaStream_t st, long long M, int f64);

gpe_status launch_cluster_alg1(ClusterArgs A, int cplx, cudaStream_t st);
// lf (optional): the line path the shape uses, log2 n of the register line
// FFT or 0 (shared-memory stages).
bool cluster_shape(int n0, int n1, int cplx, int nvec, int* cs, int* lch, int* P0, int* P1, size_t* smem,
                   unsigned int* vec_bytes, unsigned int* vpot_bytes, size_t share = 16 * 1024, int* lf = nullptr);

void destroy_solver_cache(void* cache);

// Polls after which a bounded device wait gives up (gpe_set_wait_limit;
// 2^22 by default for grid barriers, 2^24 for the fused kernel's task waits,
// whose polls are shorter).
long long wait_limit(long long default_polls);

// Instrumentation: launch counting and optional per-kernel CUDA-event timing.
void instr_count(long long n);
bool prof_enabled();
struct ProfScope {
  int slot = -1;
  cudaStream_t st = nullptr;
  ProfScope(const char* name, cudaStream_t s);   // counts the launch unless the stream is capturing
  ~ProfScope();
};
const char* kernel_name(const char* base, int f64, int cplx, int epi, long long points = -1);

inline size_t elem_size(int prec, int cplx) { return (prec == GPE_F64 ? 8 : 4) * (cplx ? 2 : 1); }

}  // namespace gpe

struct gpe_plan_s {
  gpe::GridHost g;
  int prec = 0;
  cudaStream_t stream = nullptr;
  gpe::GridDev<float>* d32 = nullptr;
  gpe::GridDev<double>* d64 = nullptr;
  gpe::Scratch sc;
  void* acc = nullptr;     // kinetic accumulator, plan precision
  void* tmp = nullptr;     // second work vector (prolongation, solver)
  void* solver_cache = nullptr;   // levels, buffers and graphs of gpe_rnewton_solve
  int device = 0;
};
