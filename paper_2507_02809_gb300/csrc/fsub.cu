// Dispatch of the persistent forward substitution over the transform length L.
#include "fsub.h"

namespace tsfde {

#define TSFDE_FSUB_DECL(LL)                                          \
  cudaError_t fsub_launch_##LL(const FsubBatch& b, cudaStream_t st); \
  int fsub_max_grid_##LL(int sms);
TSFDE_FSUB_DECL(8)
TSFDE_FSUB_DECL(16)
TSFDE_FSUB_DECL(32)
TSFDE_FSUB_DECL(64)
TSFDE_FSUB_DECL(128)
TSFDE_FSUB_DECL(256)
TSFDE_FSUB_DECL(512)
TSFDE_FSUB_DECL(1024)
TSFDE_FSUB_DECL(2048)
TSFDE_FSUB_DECL(4096)
#undef TSFDE_FSUB_DECL

#define TSFDE_FSUB_SWITCH(L, CALL) \
  switch (L) {                     \
    case 8: CALL(8); break;        \
    case 16: CALL(16); break;      \
    case 32: CALL(32); break;      \
    case 64: CALL(64); break;      \
    case 128: CALL(128); break;    \
    case 256: CALL(256); break;    \
    case 512: CALL(512); break;    \
    case 1024: CALL(1024); break;  \
    case 2048: CALL(2048); break;  \
    case 4096: CALL(4096); break;  \
    default: break;                \
  }

int fsub_max_grid(int L, int sms) {
  int g = 0;
#define TSFDE_CALL_G(LL) g = fsub_max_grid_##LL(sms)
  TSFDE_FSUB_SWITCH(L, TSFDE_CALL_G)
#undef TSFDE_CALL_G
  return g;
}

cudaError_t fsub_launch(int L, const FsubBatch& b, cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
#define TSFDE_CALL_F(LL) e = fsub_launch_##LL(b, st)
  TSFDE_FSUB_SWITCH(L, TSFDE_CALL_F)
#undef TSFDE_CALL_F
  return e;
}

}  // namespace tsfde
