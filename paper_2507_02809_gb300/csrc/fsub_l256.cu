// Instantiations of the persistent forward substitution for L in {256}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_256(const FsubArgs& a, int grid, cudaStream_t st) { return launch_L<256>(a, grid, st); }
int fsub_max_grid_256(int sms) { return max_grid_L<256>(sms); }

}  // namespace tsfde
