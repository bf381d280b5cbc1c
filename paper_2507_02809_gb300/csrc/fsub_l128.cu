// Instantiations of the persistent forward substitution for L in {128}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_128(const FsubArgs& a, int grid, cudaStream_t st) { return launch_L<128>(a, grid, st); }
int fsub_max_grid_128(int sms) { return max_grid_L<128>(sms); }

}  // namespace tsfde
