// lines2d_f64.cu -- double instantiation of the register-FFT 2D line kernels.
#include "lines2d.cuh"

namespace gpe {
template gpe_status launch_lines2d<double>(const GridHost&, const GridDev<double>&, const PassData<double>&, int, void*, bool,
                                       cudaStream_t, bool*);
}  // namespace gpe
