// unsplit_f32.cu -- unsplit-scheme kernels instantiated for the f32 policy.
#include "unsplit.cuh"

namespace hy {
cudaError_t launch_unsplit_f32(const UnsplitLaunch &a) {
    return launch_unsplit_prec<float, PREC_F32>(a);
}
}  // namespace hy
