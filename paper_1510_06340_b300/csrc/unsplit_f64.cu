// unsplit_f64.cu -- unsplit-scheme kernels instantiated for the f64 policy.
#include "unsplit.cuh"

namespace hy {
cudaError_t launch_unsplit_f64(const UnsplitLaunch &a) {
    return launch_unsplit_prec<double, PREC_F64>(a);
}
}  // namespace hy
