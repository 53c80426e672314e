// Float32 instantiation of the libgpe kernels and launch wrappers.
#include "ops_launch.cuh"
namespace gpe {
GPE_INSTANTIATE(float)
}  // namespace gpe
