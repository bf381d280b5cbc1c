// The mixed-length persistent kernel: one cooperative launch runs the forward (or backward)
// substitution of instances with DIFFERENT transform lengths and dimensions.  Each CTA looks up
// its instance and calls the body compiled for that instance's length (fsub_mix_l*.cu, separate
// relocatable device code, at most 128 registers per thread); all bodies run in CTAs of 512
// threads (the length-4096 body needs them, the shorter ones hold more line groups).  Each
// instance keeps its own sub-grid, barrier counter and partial sums, so the instances proceed
// independently and give the results they give alone on a sub-grid of the same size.
#include "fft.cuh"
#include "fsub.h"

namespace tsfde {

#define TSFDE_MIXED_LENGTHS(X) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

#define TSFDE_DECL_BODY(LL) __device__ void fsub_mixed_body_##LL(const FsubArgs* a, int G, int bid);
TSFDE_MIXED_LENGTHS(TSFDE_DECL_BODY)
#undef TSFDE_DECL_BODY

__global__ void __launch_bounds__(kMixedThreads) k_fsub_mixed(FsubMixed m) {
  const int inst = m.cta_inst[blockIdx.x];
  const FsubArgs* a = m.args + inst;
  const int L = a->L, G = a->gper, bid = (int)blockIdx.x - a->cta0;
  switch (L) {
#define TSFDE_CASE_BODY(LL) \
  case LL:                  \
    fsub_mixed_body_##LL(a, G, bid); \
    break;
    TSFDE_MIXED_LENGTHS(TSFDE_CASE_BODY)
#undef TSFDE_CASE_BODY
    default:
      break;
  }
}

// Line buffers of kMixedThreads / (L / 8) groups, then the twiddle tables (as fsub_body lays them out).
size_t fsub_mixed_smem(int L) {
  if (L < 8 || L > 4096 || (L & (L - 1)) != 0) return 0;
  const int groups = kMixedThreads / (L / 8);
  return (size_t)groups * line_stride(L) * sizeof(double2) + (size_t)L * (sizeof(double2) + sizeof(float2));
}

int fsub_mixed_max_grid(size_t smem, int sms) {
  if (cudaFuncSetAttribute(k_fsub_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fsub_mixed, kMixedThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per * sms;
}

// (fsub_mixed_max_grid with the same smem has set the kernel's shared-memory limit; no attribute
// call here, so that the launch can be captured into a graph)
cudaError_t fsub_mixed_launch(const FsubMixed& m, int grid, size_t smem, cudaStream_t st) {
  FsubMixed args = m;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)k_fsub_mixed, dim3(grid), dim3(kMixedThreads), params, smem, st);
}

}  // namespace tsfde
