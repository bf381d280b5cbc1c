// Bodies of the mixed-length persistent kernel (fsub_mix.cu) for L in {256}: relocatable
// device code compiled with at most 128 registers per thread, so that the kernel calling them
// can run CTAs of 512 threads.
#include "fsub_impl.cuh"

namespace tsfde {

__device__ void fsub_mixed_body_256(const FsubArgs* a, int G, int bid) { fsub_body<256>(a, G, bid); }

}  // namespace tsfde
