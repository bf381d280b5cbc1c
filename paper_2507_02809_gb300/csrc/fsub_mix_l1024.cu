// Bodies of the mixed-length persistent kernel (fsub_mix.cu) for L in {1024}: relocatable
// device code compiled with at most 128 registers per thread, so that the kernel calling them
// can run CTAs of 512 threads.
#include "fsub_impl.cuh"

namespace tsfde {

__device__ void fsub_mixed_body_1024(const FsubArgs* a, int G, int bid) { fsub_body<1024>(a, G, bid); }

}  // namespace tsfde
