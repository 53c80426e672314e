// Float64 instantiation of the libgpe kernels and launch wrappers.
#include "ops_launch.cuh"
namespace gpe {
GPE_INSTANTIATE(double)
}  // namespace gpe

namespace gpe {
template <typename Ti, typename To>
gpe_status launch_convert(const Ti* in, To* out, long long n, double scale, cudaStream_t st) {
  ProfScope ps(kernel_name("convert", sizeof(To) == 8, 0, -1), st);
  k_convert<Ti, To><<<ew_blocks(n), NTHREADS, 0, st>>>(in, out, n, scale);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}
template gpe_status launch_convert<float, double>(const float*, double*, long long, double, cudaStream_t);
template gpe_status launch_convert<double, float>(const double*, float*, long long, double, cudaStream_t);
template gpe_status launch_convert<float, float>(const float*, float*, long long, double, cudaStream_t);
template gpe_status launch_convert<double, double>(const double*, double*, long long, double, cudaStream_t);

gpe_status launch_step_coef(const double* mom, int nbatch, double h, double tau, double* coef, cudaStream_t st) {
  ProfScope ps("step_coef", st);
  k_step_coef<<<(nbatch + 127) / 128, 128, 0, st>>>(mom, nbatch, h, tau, coef);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}

gpe_status launch_norm_coef(const double* mom, int nbatch, double h, double* coef, cudaStream_t st) {
  ProfScope ps("norm_coef", st);
  k_norm_coef<<<(nbatch + 127) / 128, 128, 0, st>>>(mom, nbatch, h, coef);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}
}  // namespace gpe

namespace gpe {
gpe_status launch_to_shifted_f32(const double* xk, const double* gk, double th, float* xk32, float* pk32, long long n,
                                 cudaStream_t st) {
  ProfScope ps("to_shifted_f32", st);
  k_to_shifted_f32<<<ew_blocks(n), NTHREADS, 0, st>>>(xk, gk, th, xk32, pk32, n);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}
gpe_status launch_add_f32_to_f64(const double* xk, const float* d, double* z, long long n, cudaStream_t st) {
  ProfScope ps("add_f32_to_f64", st);
  k_add_f32_to_f64<<<ew_blocks(n), NTHREADS, 0, st>>>(xk, d, z, n);
  GPE_CUDA(cudaGetLastError());
  return GPE_OK;
}
}  // namespace gpe
