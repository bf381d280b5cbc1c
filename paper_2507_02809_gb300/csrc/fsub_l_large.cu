// Instantiations of the persistent forward substitution for L in {2048, 4096}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_2048(const FsubBatch& b, cudaStream_t st) { return launch_L<2048>(b, st); }
int fsub_max_grid_2048(int sms) { return max_grid_L<2048>(sms); }

cudaError_t fsub_launch_4096(const FsubBatch& b, cudaStream_t st) { return launch_L<4096>(b, st); }
int fsub_max_grid_4096(int sms) { return max_grid_L<4096>(sms); }

}  // namespace tsfde
