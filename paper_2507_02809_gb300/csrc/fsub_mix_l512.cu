// Bodies of the mixed-length persistent kernel (fsub_mix.cu) for L in {512}: relocatable
// device code compiled with at most 128 registers per thread, so that the kernel calling them
// can run CTAs of 512 threads.
#include "fsub_impl.cuh"

namespace tsfde {

__device__ void fsub_mixed_body_512(const FsubArgs* a, int G, int bid) { fsub_body<512>(a, G, bid); }

}  // namespace tsfde
