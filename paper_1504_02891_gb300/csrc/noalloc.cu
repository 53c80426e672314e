// noalloc.cu -- gpe_feasible_step_noalloc: the sphere-preserving Cayley step of
// gpe_feasible_step for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// inside a CUDA stream capture that must not contain allocation calls, inside a
// custom allocator or memory-pool callback, in a real-time loop whose memory
// budget was fixed up front, or in a host that gives the library only
// caller-owned buffers.  gpe_feasible_step needs a plan, and creating a plan
// allocates tables and reduction scratch; this entry point takes no plan.
//
// Where its scratch lives: one file-scope device array (g_noalloc_scratch),
// 512 KiB, placed in every GPU's memory when the library is loaded on it and
// kept until the process exits.  Host code cannot use the array's name as a
// device address (it names a host-side shadow), so the device address is
// looked up with cudaGetSymbolAddress once per device, on the first call made
// while that device is current, and cached.
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
void* g_addr[NOALLOC_MAX_DEVICES] = {nullptr};

gpe_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gpe::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return gpe::fail(GPE_EINVAL, "device index beyond the supported range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return gpe::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
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
