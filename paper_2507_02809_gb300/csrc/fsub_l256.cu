// Instantiations of the persistent forward substitution for L in {256}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_256(const FsubBatch& b, cudaStream_t st) { return launch_L<256>(b, st); }
int fsub_max_grid_256(int sms) { return max_grid_L<256>(sms); }

}  // namespace tsfde
