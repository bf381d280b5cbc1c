// Persistent forward-substitution kernel (fsub.cu): arguments and host entry points.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace tsfde {

struct FsubBarrier {
  unsigned int* count;  // arrivals since the launch began (zeroed by the host before each launch)
  int* err;             // set when a wait exceeded its cap
};

struct FsubArgs {
  int d, n, L, S;
  long long N;
  int mode;  // 0: FP64 refinement around FP32 CG corrections; 1: one FP32 CG solve per block
  int refine_max, pcg_iters, pcg_max;
  int warm;  // initial guess of each block solve, extrapolated in processing order from the levels
             // already solved: 0 zero; k >= 1 the polynomial of degree k - 1 through the last k (<= 8)
  int trans;  // 1: backward substitution for P^T (f block first, then levels S..1); y = P^-T r
  double tol2_outer, tol2_inner, tol2_mixed;
  double cs, cf;
  const double* r;  // right-hand side [S+1][N]
  double* y;        // result [S+1][N]
  const double *g1, *g2, *ew;
  const double* dvec64;
  const float* dvec32;
  const float* dbar32;
  const double2* tw64;
  const float2* tw32;
  const double *lam64, *mu64;
  const float *lam32, *mu32;
  double2 *w64a, *w64b;
  float2 *w32a, *w32b;
  double* lb;
  double* lBx;  // FP64 mode, warm start: [8][N], slot p mod 8 holds B_n x of position p's final x
                // (from its last refinement residual), so that B_n x0 of an extrapolated x0 is the
                // same combination of the slots
  double* hfar; // [16][N]: far part of the history sums of the current group of 16 levels
  float *lb32, *lx32, *lr32, *lz32, *lp32, *lq32;
  int fused;              // d >= 2: the four-pass inner CG (row sine transforms / spectra carried)
  int block_solver;       // 0: inner CG to tolerance; 1: one (dbar I + c tau(B_n))^-1 solve per block
                          // (T_{n,S}); 2: one (dbar I + c s(B_n))^-1 Fourier solve (S_{n,S})
  const double* dbar64;   // [S] level means of e_0 gamma1 / gamma2
  float *ltr32, *ltq32;   // row sine transforms of r and q [N / n][np], np = L/2 - 1
  double *t1_64, *t2_64;  // tau solves' intermediates: [N / n][np], and [n][np][np] for d = 3
  float *t1_32, *t2_32;
  float2 *w32z, *w32p;    // row half spectra of z and p [N / n][L / 2 + 1]
  const double* zero64;
  const float* zero32;
  // S_{n,S}: Bluestein tables for DFTs of length n (chirp [n], FFT of the conjugate chirp [L] / L)
  // and the eigenvalues of s(B_n) [n]^d in DFT order
  const double2 *sch64, *sbh64;
  const float2 *sch32, *sbh32;
  const double* slam64;
  const float* slam32;
  double* part;  // >= 8 * grid doubles
  FsubBarrier bar;
  long long spin_limit;  // polls of one grid-barrier wait before it gives up (error flag, TSFDE_ETIMEOUT)
  int gper, cta0;        // mixed-length launch: CTAs of this instance's sub-grid and its first CTA
  Scalars* stats;  // [2]: counters accumulated by the launch (fails, sweeps, iters)
  // optional timeline: CTA 0 records (globaltimer, phase kind) at every grid barrier
  unsigned long long* trace;  // [2 * trace_cap] or nullptr
  int trace_cap;
  int* trace_len;             // entries written
};

// phase kinds of the timeline
enum FsubPhase : int {
  PH_RHS = 0, PH_B64_ROWFWD, PH_B64_COLS, PH_B64_ROWINV, PH_TAU_ROWS_IN, PH_TAU_COLS, PH_TAU_ROWS_OUT,
  PH_B32_ROWFWD, PH_B32_COLS, PH_B32_ROWINV, PH_CAST, PH_COUNT
};

// A batch of instances with the same transform length in one launch: args is a device array of
// `count` FsubArgs; instance i runs on CTAs [i gper, (i+1) gper) as its own sub-grid.
struct FsubBatch {
  const FsubArgs* args;
  int count;
  int gper;
};
constexpr int kMaxBatch = 64;

// A batch of instances of DIFFERENT transform lengths (and dimensions) in one launch of the
// mixed-length kernel: CTAs of kMixedThreads threads; CTA c runs instance cta_inst[c] as block
// c - args[i].cta0 of its sub-grid of args[i].gper CTAs, through the body compiled for args[i].L.
struct FsubMixed {
  const FsubArgs* args;
  const int* cta_inst;
  int count;
};
constexpr int kMixedThreads = 512;
constexpr int kMaxMixedGrid = 1024;
// Dynamic shared memory the mixed-length kernel needs for a transform of length L.
size_t fsub_mixed_smem(int L);
// Largest co-resident grid of the mixed-length kernel with `smem` bytes of dynamic shared memory.
int fsub_mixed_max_grid(size_t smem, int sms);
cudaError_t fsub_mixed_launch(const FsubMixed& m, int grid, size_t smem, cudaStream_t st);

// Largest co-resident grid for transforms of length L on `sms` SMs (0 if unsupported).
int fsub_max_grid(int L, int sms);
// Cooperative launch of the whole forward (or backward) substitution of a batch.
cudaError_t fsub_launch(int L, const FsubBatch& b, cudaStream_t st);

}  // namespace tsfde
