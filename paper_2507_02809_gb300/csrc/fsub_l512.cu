// Instantiations of the persistent forward substitution for L in {512}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_512(const FsubBatch& b, cudaStream_t st) { return launch_L<512>(b, st); }
int fsub_max_grid_512(int sms) { return max_grid_L<512>(sms); }

}  // namespace tsfde
