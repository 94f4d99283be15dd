// unsplit_mixed.cu -- unsplit-scheme kernels instantiated for the mixed precision policy.
#include "unsplit.cuh"

namespace hy {
cudaError_t launch_unsplit_mixed(const UnsplitLaunch &a) {
    return launch_unsplit_prec<float, PREC_MIXED>(a);
}
}  // namespace hy
