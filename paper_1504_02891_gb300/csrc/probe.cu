// probe.cu -- measured arithmetic peaks of the GPU the library runs on (the
// paper has no counterpart: instrumentation).  The H-apply and the solver's
// transforms issue mostly float32 FMAs and adds; whether a kernel is bound by
// HBM or by the arithmetic pipes depends on these rates, which are measured
// here instead of taken from a data sheet.
//
// Each thread runs CH independent multiply-add chains x <- x * m + c for
// `iters` steps (enough independent work to hide the pipe latency at full
// occupancy); the result is written only if it takes an impossible value, so
// nothing can be optimised away and nothing is stored in practice.
#include "gpe_internal.h"

using namespace gpe;

namespace {

constexpr int PROBE_CH = 8;
constexpr int PROBE_THREADS = 256;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, float m, float c, double* sink) {
  if constexpr (KIND == 0) {
    float x[PROBE_CH];
#pragma unroll
    for (int i = 0; i < PROBE_CH; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 16; ++u)
#pragma unroll
        for (int i = 0; i < PROBE_CH; ++i) x[i] = fmaf(x[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CH; ++i) s += x[i];
    if (s == -1.2345f) sink[0] = s;
  } else if constexpr (KIND == 1) {
    float2 x[PROBE_CH];
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < PROBE_CH; ++i) x[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 16; ++u)
#pragma unroll
        for (int i = 0; i < PROBE_CH; ++i) x[i] = __ffma2_rn(x[i], m2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CH; ++i) s += x[i].x + x[i].y;
    if (s == -1.2345f) sink[0] = s;
  } else {
    double x[PROBE_CH];
    const double md = m, cd = c;
#pragma unroll
    for (int i = 0; i < PROBE_CH; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < 16; ++u)
#pragma unroll
        for (int i = 0; i < PROBE_CH; ++i) x[i] = fma(x[i], md, cd);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CH; ++i) s += x[i];
    if (s == -1.2345) sink[0] = s;
  }
}

template <int KIND>
gpe_status run_probe(cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0, occ = 0;
  GPE_CUDA(cudaGetDevice(&dev));
  GPE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GPE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_probe<KIND>, PROBE_THREADS, 0));
  if (occ < 1) occ = 1;
  const int blocks = sms * occ;
  // about 10 ms of float32 work per launch at the nominal rate (fewer steps
  // for float64, whose rate is far lower)
  const int iters = KIND == 2 ? 64 : 2048;
  cudaEvent_t a, b;
  GPE_CUDA(cudaEventCreate(&a));
  GPE_CUDA(cudaEventCreate(&b));
  k_fma_probe<KIND><<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999f, 1e-3f, nullptr);   // warm-up
  cudaEventRecord(a, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) k_fma_probe<KIND><<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999f, 1e-3f, nullptr);
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "arithmetic probe");
  instr_count(reps + 1);
  const double fl_per_fma = KIND == 1 ? 4.0 : 2.0;     // FFMA2: two lanes of a * b + c
  const double flops = (double)reps * blocks * PROBE_THREADS * (double)iters * 16.0 * PROBE_CH * fl_per_fma;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return GPE_OK;
}

}  // namespace

extern "C" gpe_status gpe_probe_peak(int kind, void* stream, double* tflops) {
  if (!tflops) return fail(GPE_EINVAL, "tflops is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  switch (kind) {
    case 0: return run_probe<0>(st, tflops);
    case 1: return run_probe<1>(st, tflops);
    case 2: return run_probe<2>(st, tflops);
  }
  return fail(GPE_EINVAL, "kind must be 0 (float32 FMA), 1 (packed float32 FMA) or 2 (float64 FMA)");
}
