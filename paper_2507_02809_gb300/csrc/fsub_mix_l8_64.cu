// Bodies of the mixed-length persistent kernel (fsub_mix.cu) for L in {8, 16, 32, 64}: relocatable
// device code compiled with at most 128 registers per thread, so that the kernel calling them
// can run CTAs of 512 threads.
#include "fsub_impl.cuh"

namespace tsfde {

__device__ void fsub_mixed_body_8(const FsubArgs* a, int G, int bid) { fsub_body<8>(a, G, bid); }
__device__ void fsub_mixed_body_16(const FsubArgs* a, int G, int bid) { fsub_body<16>(a, G, bid); }
__device__ void fsub_mixed_body_32(const FsubArgs* a, int G, int bid) { fsub_body<32>(a, G, bid); }
__device__ void fsub_mixed_body_64(const FsubArgs* a, int G, int bid) { fsub_body<64>(a, G, bid); }

}  // namespace tsfde
