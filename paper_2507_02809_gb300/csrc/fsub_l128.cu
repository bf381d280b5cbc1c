// Instantiations of the persistent forward substitution for L in {128}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_128(const FsubBatch& b, cudaStream_t st) { return launch_L<128>(b, st); }
int fsub_max_grid_128(int sms) { return max_grid_L<128>(sms); }

}  // namespace tsfde
