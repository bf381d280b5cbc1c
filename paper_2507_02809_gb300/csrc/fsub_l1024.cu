// Instantiations of the persistent forward substitution for L in {1024}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_1024(const FsubBatch& b, cudaStream_t st) { return launch_L<1024>(b, st); }
int fsub_max_grid_1024(int sms) { return max_grid_L<1024>(sms); }

}  // namespace tsfde
