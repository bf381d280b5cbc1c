// Instantiations of the persistent forward substitution for L in {8, 16, 32, 64}.
#include "fsub_impl.cuh"

namespace tsfde {

cudaError_t fsub_launch_8(const FsubBatch& b, cudaStream_t st) { return launch_L<8>(b, st); }
int fsub_max_grid_8(int sms) { return max_grid_L<8>(sms); }

cudaError_t fsub_launch_16(const FsubBatch& b, cudaStream_t st) { return launch_L<16>(b, st); }
int fsub_max_grid_16(int sms) { return max_grid_L<16>(sms); }

cudaError_t fsub_launch_32(const FsubBatch& b, cudaStream_t st) { return launch_L<32>(b, st); }
int fsub_max_grid_32(int sms) { return max_grid_L<32>(sms); }

cudaError_t fsub_launch_64(const FsubBatch& b, cudaStream_t st) { return launch_L<64>(b, st); }
int fsub_max_grid_64(int sms) { return max_grid_L<64>(sms); }

}  // namespace tsfde
