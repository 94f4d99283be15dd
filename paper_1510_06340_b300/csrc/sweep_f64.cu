// sweep_f64.cu -- sweep kernels instantiated for the f64 precision policy.
#include "sweep.cuh"

namespace hy {
cudaError_t launch_sweep_f64(const SweepLaunch &a) { return launch_sweep_prec<double, PREC_F64>(a); }
}  // namespace hy
