// noalloc.cu -- gpe_feasible_step_noalloc: the sphere-preserving Cayley step of
// gpe_feasible_step for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// inside a custom allocator or memory-pool callback (which must not re-enter
// the allocator), in a real-time loop whose device memory budget was fixed up
// front, or in a host framework that owns all device memory and hands the
// library only caller-owned buffers.  gpe_feasible_step needs a plan, and
// creating a plan allocates tables and reduction scratch; this entry point
// takes no plan.
//
// Where its scratch lives: one file-scope device array (g_noalloc_scratch),
// 512 KiB, placed in every GPU's memory when the library is loaded on it and
// kept until the process exits.  Host code cannot use the array's name as a
// device address (it names a host-side shadow), so the device address is
// looked up with cudaGetSymbolAddress on the first call made while a device is
// current, and cached together with the identity of that device's CUDA
// context: after a cudaDeviceReset the context (and the array's address) is
// new, and the next call looks the address up again.
#include <cuda.h>
#include <mutex>
#include "ops_impl.cuh"

namespace {

constexpr int NOALLOC_MAX_BLOCKS = 4096;   // reduction CTAs per call (all instances)
constexpr int NOALLOC_MAX_BATCH = 64;      // instances per call
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr size_t NOALLOC_PARTIALS = (size_t)NOALLOC_MAX_BLOCKS * gpe::NQ;   // doubles
constexpr size_t NOALLOC_RESULTS = (size_t)NOALLOC_MAX_BATCH * gpe::NQ;     // doubles
constexpr size_t NOALLOC_COEF = (size_t)NOALLOC_MAX_BATCH * 2;              // doubles
constexpr size_t NOALLOC_BYTES = 512 * 1024;
static_assert((NOALLOC_PARTIALS + NOALLOC_RESULTS + NOALLOC_COEF) * sizeof(double) + 256 <= NOALLOC_BYTES,
              "scratch layout exceeds the array");

// partials | results | coef | ticket (unsigned int), each 256-byte aligned
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
struct CachedAddr {
  unsigned long long ctx_id;   // 0: nothing cached
  void* addr;
};
CachedAddr g_addr[NOALLOC_MAX_DEVICES] = {};

// Driver entry points for the identity of the current context, resolved
// through the runtime (the library does not link the driver library itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

gpe_status resolve_driver_calls() {
  if (g_ctx_current && g_ctx_id) return GPE_OK;
  void* f1 = nullptr;
  void* f2 = nullptr;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
  if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1)
    return gpe::cuda_fail(e != cudaSuccess ? e : cudaErrorSymbolNotFound, "driver entry point cuCtxGetCurrent");
  e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
  if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !f2)
    return gpe::cuda_fail(e != cudaSuccess ? e : cudaErrorSymbolNotFound, "driver entry point cuCtxGetId");
  g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
  g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  return GPE_OK;
}

// Unique id of the context current on this thread (0 if none yet).
gpe_status current_ctx_id(unsigned long long* id) {
  *id = 0;
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS) return gpe::fail(GPE_ECUDA, "cuCtxGetCurrent failed");
  if (!ctx) return GPE_OK;
  if (g_ctx_id(ctx, id) != CUDA_SUCCESS) return gpe::fail(GPE_ECUDA, "cuCtxGetId failed");
  return GPE_OK;
}

gpe_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gpe::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return gpe::fail(GPE_EINVAL, "device index beyond the supported range");
  std::lock_guard<std::mutex> lk(g_mu);
  gpe_status s = resolve_driver_calls();
  if (s != GPE_OK) return s;
  unsigned long long id = 0;
  s = current_ctx_id(&id);
  if (s != GPE_OK) return s;
  CachedAddr& c = g_addr[dev];
  if (id == 0 || c.ctx_id != id) {
    // first call on this device, or its context was replaced (device reset):
    // the lookup also makes the device's primary context current if needed
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return gpe::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    s = current_ctx_id(&id);
    if (s != GPE_OK) return s;
    if (id == 0) return gpe::fail(GPE_ECUDA, "no CUDA context current after cudaGetSymbolAddress");
    c.ctx_id = id;
    c.addr = p;
  }
  *out = static_cast<unsigned char*>(c.addr);
  return GPE_OK;
}

template <typename T, bool CPLX>
gpe_status run(const void* psi, const void* hpsi, long long M, int nbatch, double h, double tau, void* out,
               cudaStream_t st, unsigned char* base, int tiles) {
  double* partials = reinterpret_cast<double*>(base);
  double* results = partials + NOALLOC_PARTIALS;
  double* coef = results + NOALLOC_RESULTS;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(coef + NOALLOC_COEF);
  // the array keeps the previous call's contents: the ticket must start at zero
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return gpe::cuda_fail(e, "cudaMemsetAsync(ticket)");
  gpe::k_moments<T, CPLX><<<tiles * nbatch, gpe::NTHREADS, 0, st>>>(psi, hpsi, M, tiles, partials, results, ticket);
  gpe::k_step_coef<<<(nbatch + 127) / 128, 128, 0, st>>>(results, nbatch, h, tau, coef);
  const long long n = M * nbatch;
  const int eb = (int)std::max<long long>(1, std::min<long long>((n + gpe::NTHREADS - 1) / gpe::NTHREADS, 152 * 8));
  gpe::k_axpby<T, CPLX><<<eb, gpe::NTHREADS, 0, st>>>(psi, hpsi, coef, 2, M, nbatch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gpe::cuda_fail(e, "gpe_feasible_step_noalloc launch");
  return GPE_OK;
}

}  // namespace

extern "C" gpe_status gpe_feasible_step_noalloc(int prec, int is_complex, int64_t n_unknowns, int nbatch, double h_vol,
                                                const void* psi, const void* hpsi, double tau, void* psi_out,
                                                void* stream) {
  if (prec != GPE_F32 && prec != GPE_F64) return gpe::fail(GPE_EINVAL, "prec must be GPE_F32 or GPE_F64");
  if (!psi || !hpsi || !psi_out) return gpe::fail(GPE_EINVAL, "NULL buffer");
  if (psi_out == psi || psi_out == hpsi) return gpe::fail(GPE_EINVAL, "psi_out must not alias psi or hpsi");
  if (n_unknowns < 1) return gpe::fail(GPE_EINVAL, "n_unknowns must be >= 1");
  if (nbatch < 1 || nbatch > NOALLOC_MAX_BATCH)
    return gpe::fail(GPE_EINVAL, "nbatch must be in [1, 64] for gpe_feasible_step_noalloc");
  if (!(h_vol > 0.0) || !isfinite(h_vol)) return gpe::fail(GPE_EINVAL, "h_vol must be finite and > 0");
  if (!(tau >= 0.0) || !isfinite(tau)) return gpe::fail(GPE_EINVAL, "tau must be finite and >= 0");
  const int tiles = (int)std::max<long long>(1, std::min<long long>((n_unknowns + gpe::NTHREADS - 1) / gpe::NTHREADS, 512));
  if ((long long)tiles * nbatch > NOALLOC_MAX_BLOCKS)
    return gpe::fail(GPE_EINVAL,
                     "gpe_feasible_step_noalloc: nbatch * min(ceil(n_unknowns/256), 512) exceeds its 4096 reduction "
                     "blocks (512 KiB fixed scratch); use gpe_feasible_step");
  unsigned char* base = nullptr;
  gpe_status s = scratch_address(&base);
  if (s != GPE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == GPE_F32)
    return is_complex ? run<float, true>(psi, hpsi, n_unknowns, nbatch, h_vol, tau, psi_out, st, base, tiles)
                      : run<float, false>(psi, hpsi, n_unknowns, nbatch, h_vol, tau, psi_out, st, base, tiles);
  return is_complex ? run<double, true>(psi, hpsi, n_unknowns, nbatch, h_vol, tau, psi_out, st, base, tiles)
                    : run<double, false>(psi, hpsi, n_unknowns, nbatch, h_vol, tau, psi_out, st, base, tiles);
}
