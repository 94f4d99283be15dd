// sweep_f32.cu -- sweep kernels instantiated for the f32 precision policy.
#include "sweep.cuh"

namespace hy {
cudaError_t launch_sweep_f32(const SweepLaunch &a) { return launch_sweep_prec<float, PREC_F32>(a); }
}  // namespace hy
