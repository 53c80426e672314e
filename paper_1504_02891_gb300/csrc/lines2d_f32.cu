// lines2d_f32.cu -- float instantiation of the register-FFT 2D line kernels.
#include "lines2d.cuh"

namespace gpe {
template gpe_status launch_lines2d<float>(const GridHost&, const GridDev<float>&, const PassData<float>&, int, void*, bool,
                                       cudaStream_t, bool*);
}  // namespace gpe
