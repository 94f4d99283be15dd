// sweep_mixed.cu -- sweep kernels instantiated for the mixed precision policy.
#include "sweep.cuh"

namespace hy {
cudaError_t launch_sweep_mixed(const SweepLaunch &a) { return launch_sweep_prec<float, PREC_MIXED>(a); }
}  // namespace hy
