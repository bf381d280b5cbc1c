// C ABI of libtsfde: setup of one instance, the matvec of Eq. 11, the forward substitution of
// Sec. 5.1 and restarted GMRES (Sec. 5 "Implementation", Sec. 6.1.2), all on one GPU.
#include "../../include/tsfde.h"

#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fsub.h"
#include "internal.h"
#include "kernels.h"
#include "rowio.cuh"

namespace tsfde {

static thread_local std::string g_last_error;
void set_error(const std::string& s) { g_last_error = s; }

}  // namespace tsfde

using namespace tsfde;

struct BatchCoord;

struct tsfde_ctx {
  // sizes and scalars of Sec. 4-5
  int d = 0, n = 0, S = 0;
  int np = 0;  // transform grid of the tau solves (np + 1 a power of two, >= n + 1)
  long long N = 0, U = 0;
  double length = 1, h = 0, T = 1, dt = 0, beta = 0, omega = 0, alpha = 0, eta = 0, cs = 0, cf = 0;
  tsfde_opts opts{};
  cudaStream_t st = nullptr;

  // owned inputs and tables (device)
  double *g1 = nullptr, *g2 = nullptr, *q = nullptr, *rho = nullptr, *mu = nullptr;
  double *bw = nullptr, *ew = nullptr;  // L1 weights b_m, e_m (m < S)
  double *a_tab = nullptr;              // a_l, 0 <= l_i < n
  double *lam64 = nullptr, *mu64 = nullptr;
  float *lam32 = nullptr, *mu32 = nullptr;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  double* dvec64 = nullptr;  // e_0 gamma1 / gamma2, [S][N]
  float* dvec32 = nullptr;
  double* dbar64 = nullptr;  // per-level mean of dvec
  double* a_tau = nullptr;   // coefficients a_l, l < np per axis (tau(B_np) of the padded grid)
  double *t1_64 = nullptr, *t2_64 = nullptr;  // tau intermediates (persistent kernel)
  float *t1_32 = nullptr, *t2_32 = nullptr;
  float* dbar32 = nullptr;
  double* zero64 = nullptr;  // [N] zeros (the f block has no diagonal term)
  float* zero32 = nullptr;
  // S_{n,S} (block_solver = 2), built on first use: Bluestein tables of the length-n DFT and the
  // eigenvalues of the Strang circulant s(B_n)
  bool strang_ready = false;
  double2 *str_chirp64 = nullptr, *str_bhat64 = nullptr;
  float2 *str_chirp32 = nullptr, *str_bhat32 = nullptr;
  double* str_lam64 = nullptr;
  float* str_lam32 = nullptr;

  SpatialPlan<double> sp64_all;  // batch of S + 1 fields (matvec)
  SpatialPlan<double> sp64_one;  // one field (block solves)
  SpatialPlan<float> sp32_one;

  // matvec / preconditioner workspaces
  double* By = nullptr;      // [(S+1) N]
  double* adj_u = nullptr;   // [(S+1) N] D_2 lam for the transposed matvec (allocated on first use)
  double* lb = nullptr;      // [N] symmetrised block right-hand side
  double* lBx = nullptr;     // [8][N]
  double* lr64 = nullptr;    // [N] FP64 PCG vectors
  double* lz64 = nullptr;
  double* lp64 = nullptr;
  double* lq64 = nullptr;
  float* lx32 = nullptr;     // FP32 PCG vectors
  float* lr32 = nullptr;
  float* lz32 = nullptr;
  float* lp32 = nullptr;
  float* lq32 = nullptr;
  float* lBp32 = nullptr;
  float* lb32 = nullptr;
  float* ltr32 = nullptr;    // fused inner CG: row sine transforms of r and q
  float* ltq32 = nullptr;
  float2* w32z = nullptr;    // fused inner CG: row spectra of z and p
  float2* w32p = nullptr;
  Scalars* sc = nullptr;     // [2]: outer (refinement / FP64 PCG), inner (FP32 PCG)
  RedWork rw{};

  // GMRES workspaces
  int m_alloc = 0;
  bool flex_alloc = false;
  double *V = nullptr, *Zf = nullptr, *x = nullptr, *z = nullptr, *r = nullptr, *w = nullptr, *tmp = nullptr;
  long long ldV = 0;  // leading dimension of the bases V and Zf: U rounded up to 32 doubles (256 B rows)
  double *H = nullptr, *gcs = nullptr, *gsn = nullptr, *gg = nullptr, *h1 = nullptr, *h2 = nullptr, *yk = nullptr;
  double *dnrm = nullptr, *dest = nullptr;
  double* host_scal = nullptr;  // pinned [4]

  // CUDA graph of the preconditioner application (internal stream, fixed in/out buffers)
  double* pin = nullptr;
  double* pout = nullptr;
  cudaStream_t gst = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_prec = -1;
  long long graph_key = 0;

  // event profiler of the preconditioner application and of the matvec (tsfde_profile)
  struct Prof {
    long long count = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> pool;
  };
  bool prof_on = false;
  bool timeline_on = false;
  Prof prof[3];                  // [0] preconditioner, [1] matvec, [2] CGS2 orthogonalisation
  double orth_bytes = 0.0;       // algorithmic HBM bytes of the profiled orthogonalisations
  long long launches = 0;        // kernels enqueued by this handle (graph replays add their kernel nodes)
  long long graph_kernels = 0;   // kernel nodes in the preconditioner graph
  long long apps_total = 0;      // preconditioner applications since set-up

  // persistent forward substitution (fsub.cu)
  int fsub_grid = 0;
  int fsub_maxg = 0;                  // largest co-resident grid of the persistent kernel
  int fsub_sms = 0;
  FsubArgs* fsub_args_dev = nullptr;  // [kMaxBatch] device copy of the launch's arguments
  int* fsub_cta_dev = nullptr;        // [kMaxMixedGrid] instance of each CTA of a mixed-length launch
  // Mixed-length batch rounds led by this handle, replayed from a CUDA graph (opts.graphs): the
  // captured launch sequence (barrier resets, argument copies from pinned staging, the cooperative
  // launch) of the last configuration, keyed by the instances' barrier buffers, sub-grid sizes
  // and shared memory; the staging buffers are rewritten before each replay.
  cudaGraphExec_t mix_exec = nullptr;
  std::vector<const void*> mix_key_bar;
  std::vector<int> mix_key_g;
  size_t mix_key_smem = 0;
  FsubArgs* mix_args_pin = nullptr;
  int* mix_cta_pin = nullptr;
  cudaEvent_t mix_done = nullptr;
  bool mix_done_valid = false;
  bool mix_graph_failed = false;
  std::string mix_graph_error;  // why the capture was unavailable (empty when it worked)
  long long mix_graph_builds = 0, mix_graph_replays = 0;
  BatchCoord* coord = nullptr;        // set while a batched solve runs this handle
  double* fsub_part = nullptr;
  double* fsub_hfar = nullptr;        // [16][N] far history sums (persistent kernel)
  unsigned int* fsub_bar = nullptr;   // [0] arrival counter, [1] unused, [2] error flag
  unsigned long long* trace = nullptr; // timeline of the persistent kernel (profiling only)
  int* trace_len = nullptr;
  int trace_cap = 0;
  double phase_ms[PH_COUNT] = {0};
  long long phase_n[PH_COUNT] = {0};

  std::vector<void*> allocs;
  size_t bytes = 0;
};

namespace {

#define TSFDE_CU(call)                                                                               \
  do {                                                                                               \
    cudaError_t _e = (call);                                                                         \
    if (_e != cudaSuccess) {                                                                         \
      set_error(std::string(#call) + ": " + cudaGetErrorString(_e));                                 \
      return _e == cudaErrorMemoryAllocation ? TSFDE_ENOMEM : TSFDE_ECUDA;                           \
    }                                                                                                \
  } while (0)

template <typename T>
tsfde_status dalloc(tsfde_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc(") + std::to_string(sizeof(T) * count) + "): " + cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? TSFDE_ENOMEM : TSFDE_ECUDA;
  }
  c->allocs.push_back(*p);
  c->bytes += sizeof(T) * count;
  return TSFDE_OK;
}

#define TSFDE_TRY(x)                      \
  do {                                    \
    tsfde_status _s = (x);                \
    if (_s != TSFDE_OK) return _s;        \
  } while (0)

tsfde_status validate_opts(const tsfde_opts* o) {
  if (o->precision != TSFDE_PREC_FP64 && o->precision != TSFDE_PREC_MIXED) return TSFDE_EINVAL;
  if (o->side < 0 || o->side > 2) return TSFDE_EINVAL;
  if (o->restart < 1 || o->restart > 64) return TSFDE_EINVAL;
  if (o->max_iters < 1) return TSFDE_EINVAL;
  if (!(o->tol > 0) || !(o->inner_tol > 0) || !(o->inner_tol_mixed > 0)) return TSFDE_EINVAL;
  if (o->pcg_iters < 1 || o->pcg_max < 1 || o->refine_max < 1) return TSFDE_EINVAL;
  if (o->coeff_K < 0) return TSFDE_EINVAL;
  if (o->graphs != 0 && o->graphs != 1) return TSFDE_EINVAL;
  if (o->persistent != 0 && o->persistent != 1) return TSFDE_EINVAL;
  if (o->warm_start < 0 || o->warm_start > 8) return TSFDE_EINVAL;
  if (o->spin_limit < 1) return TSFDE_EINVAL;
  if (o->warm_start_mixed < 0 || o->warm_start_mixed > 8) return TSFDE_EINVAL;
  if (o->grid_ctas < 0) return TSFDE_EINVAL;
  if (o->fused_cg != 0 && o->fused_cg != 1) return TSFDE_EINVAL;
  if (o->block_solver < 0 || o->block_solver > 2) return TSFDE_EINVAL;
  if (!(o->inner_tol_corr > 0) || !(o->inner_tol_corr < 1)) return TSFDE_EINVAL;
  return TSFDE_OK;
}

tsfde_status check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return TSFDE_ECUDA;
  }
  return TSFDE_OK;
}

long long opts_key(const tsfde_opts& o) {
  return (long long)o.pcg_iters + 100LL * o.pcg_max + 10000LL * o.refine_max + 100000LL * o.warm_start +
         1000000LL * (long long)llround(-log10(o.inner_tol) * 16) + 1000000000LL * (long long)llround(-log10(o.inner_tol_mixed) * 16) +
         100000000000LL * (long long)llround(-log10(o.inner_tol_corr) * 16);
}

int default_K(int d, int n) {
  int base = 1;
  while (base < 2 * n) base <<= 1;
  return (d <= 2 ? 8 : 2) * base;
}

void free_all(tsfde_ctx* c) {
  for (auto& P : c->prof) {
    for (auto& pr : P.pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    for (auto e : P.pool) cudaEventDestroy(e);
    P.pending.clear();
    P.pool.clear();
  }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  if (c->mix_exec) cudaGraphExecDestroy(c->mix_exec);
  c->mix_exec = nullptr;
  if (c->mix_args_pin) cudaFreeHost(c->mix_args_pin);
  if (c->mix_cta_pin) cudaFreeHost(c->mix_cta_pin);
  c->mix_args_pin = nullptr;
  c->mix_cta_pin = nullptr;
  if (c->mix_done) cudaEventDestroy(c->mix_done);
  c->mix_done = nullptr;
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->gst) cudaStreamDestroy(c->gst);
  c->ev_in = c->ev_out = nullptr;
  c->gst = nullptr;
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->host_scal) cudaFreeHost(c->host_scal);
  c->host_scal = nullptr;
  if (c->tw64) cudaFree(c->tw64);
  if (c->tw32) cudaFree(c->tw32);
  c->tw64 = nullptr;
  c->tw32 = nullptr;
}

// CTAs of one instance's persistent substitution: one CTA for d = 1 (a line fits it); else one per
// SM, or opts.grid_ctas when set (at most the co-resident limit)
int persistent_grid(const tsfde_ctx* c, const tsfde_opts& o) {
  if (c->fsub_maxg <= 0) return 0;
  if (c->d == 1) return 1;
  const int g = o.grid_ctas > 0 ? o.grid_ctas : c->fsub_sms;
  return g < c->fsub_maxg ? g : c->fsub_maxg;
}

tsfde_status alloc_gmres(tsfde_ctx* c) {
  const int m = c->opts.restart;
  const bool flex = (c->opts.side == TSFDE_SIDE_FLEXIBLE);
  if (c->V && m <= c->m_alloc && (!flex || c->flex_alloc)) return TSFDE_OK;
  if (c->V) {
    // grow: release the old GMRES buffers (they were allocated last and are tracked too)
    auto rel = [&](double*& p) {
      if (!p) return;
      for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
        if (*it == p) { c->allocs.erase(it); break; }
      cudaFree(p);
      p = nullptr;
    };
    rel(c->V);
    rel(c->Zf);
  }
  c->ldV = (c->U + 31) / 32 * 32;
  TSFDE_TRY(dalloc(c, &c->V, (size_t)(m + 1) * c->ldV));
  if (flex) TSFDE_TRY(dalloc(c, &c->Zf, (size_t)m * c->ldV));
  c->m_alloc = m;
  c->flex_alloc = flex;
  return TSFDE_OK;
}

// ---------------------------------------------------------------------------------------
// Diagonal-block solves of the forward substitution
// ---------------------------------------------------------------------------------------

// Solve (diag(dvec) + c B) x = b (FP64 result) to the FP64 inner tolerance: FP32 tau-PCG
// corrections inside FP64 iterative refinement.  x holds the initial guess on entry.
// Per sweep: [B_n x in FP64 + residual] then [tau solve + r.z] then pcg_iters x
// ([B_n p + q, alpha] [x, r update + tau solve + beta]); every launch returns at once when
// the block solve has converged.
void block_solve_fp64(tsfde_ctx* C, cudaStream_t st, const double* b, double* x, const double* dvec64,
                      const float* dvec32, const float* dbar32, int dbar_off, double cc) {
  Scalars* outer = C->sc;
  Scalars* inner = C->sc + 1;
  const float c32 = (float)cc;
  const double pcg_tol = C->opts.inner_tol_corr;
  scalars_reset_solve(outer, C->opts.inner_tol, st);
  for (int sweep = 0; sweep <= C->opts.refine_max; ++sweep) {
    RowIO<double> r64;
    r64.ld = (sweep == 0) ? LD_PLAIN : LD_X_UPDATE;
    r64.src = x;
    r64.x = x;
    r64.dx32 = C->lx32;
    r64.st = ST_RESID_REFINE;
    r64.b = b;
    r64.dvec = dvec64;
    r64.c = cc;
    r64.r32 = C->lr32;
    r64.first = (sweep == 0);
    r64.inner_tol2 = pcg_tol * pcg_tol;
    r64.sc = outer;
    r64.sc2 = inner;
    r64.rw = C->rw;
    r64.skip = &outer->done;
    bapply_io<double>(C->sp64_one, 1, r64, st);
    if (sweep == C->opts.refine_max) break;
    RowIO<float> t0;
    t0.src = C->lr32;
    t0.st = ST_RZ_FIRST;
    t0.dst = C->lz32;
    t0.p = C->lp32;
    t0.x = C->lx32;
    t0.r = C->lr32;
    t0.sc = inner;
    t0.rw = C->rw;
    t0.skip = &inner->done;
    tau_io<float>(C->sp32_one, 1, dbar32, dbar_off, c32, t0, st);
    for (int k = 0; k < C->opts.pcg_iters; ++k) {
      RowIO<float> b1;
      b1.ld = (k == 0) ? LD_PLAIN : LD_P_UPDATE;
      b1.src = (k == 0) ? C->lp32 : C->lz32;
      b1.p = C->lp32;
      b1.st = ST_PCG_Q;
      b1.dvec = dvec32;
      b1.c = c32;
      b1.qout = C->lq32;
      b1.sc = inner;
      b1.rw = C->rw;
      b1.skip = &inner->done;
      bapply_io<float>(C->sp32_one, 1, b1, st);
      RowIO<float> t1;
      t1.ld = LD_PCG_UPDATE;
      t1.x = C->lx32;
      t1.p = C->lp32;
      t1.r = C->lr32;
      t1.q = C->lq32;
      t1.st = ST_RZ_BETA;
      t1.dst = C->lz32;
      t1.sc = inner;
      t1.rw = C->rw;
      t1.skip = &inner->done;
      tau_io<float>(C->sp32_one, 1, dbar32, dbar_off, c32, t1, st);
    }
  }
  scalars_count_fail(outer, st);
}

// Mixed precision: one FP32 tau-PCG solve to inner_tol_mixed, started from x (FP64, cast).
void block_solve_fp32(tsfde_ctx* C, cudaStream_t st, const double* b, double* x, const float* dvec32,
                      const float* dbar32, int dbar_off, double cc) {
  const long long N = C->N;
  Scalars* sc = C->sc + 1;
  const float c32 = (float)cc;
  cast_d2f(b, C->lb32, N, st);
  cast_d2f(x, C->lx32, N, st);
  scalars_reset_solve(sc, C->opts.inner_tol_mixed, st);
  RowIO<float> r0;
  r0.src = C->lx32;
  r0.st = ST_RESID;
  r0.b = C->lb32;
  r0.x = C->lx32;
  r0.dvec = dvec32;
  r0.c = c32;
  r0.r = C->lr32;
  r0.sc = sc;
  r0.rw = C->rw;
  r0.skip = &sc->done;
  bapply_io<float>(C->sp32_one, 1, r0, st);
  RowIO<float> t0;
  t0.src = C->lr32;
  t0.st = ST_RZ_FIRST;
  t0.dst = C->lz32;
  t0.p = C->lp32;
  t0.r = C->lr32;
  t0.sc = sc;
  t0.rw = C->rw;
  t0.skip = &sc->done;
  tau_io<float>(C->sp32_one, 1, dbar32, dbar_off, c32, t0, st);
  for (int k = 0; k < C->opts.pcg_max; ++k) {
    RowIO<float> b1;
    b1.ld = (k == 0) ? LD_PLAIN : LD_P_UPDATE;
    b1.src = (k == 0) ? C->lp32 : C->lz32;
    b1.p = C->lp32;
    b1.st = ST_PCG_Q;
    b1.dvec = dvec32;
    b1.c = c32;
    b1.qout = C->lq32;
    b1.sc = sc;
    b1.rw = C->rw;
    b1.skip = &sc->done;
    bapply_io<float>(C->sp32_one, 1, b1, st);
    RowIO<float> t1;
    t1.ld = LD_PCG_UPDATE;
    t1.x = C->lx32;
    t1.p = C->lp32;
    t1.r = C->lr32;
    t1.q = C->lq32;
    t1.st = ST_RZ_BETA;
    t1.dst = C->lz32;
    t1.sc = sc;
    t1.rw = C->rw;
    t1.skip = &sc->done;
    tau_io<float>(C->sp32_one, 1, dbar32, dbar_off, c32, t1, st);
  }
  scalars_count_fail(sc, st);
  cast_f2d(C->lx32, x, N, st);
}

void block_solve(tsfde_ctx* C, cudaStream_t st, const double* b, double* x,
                 int level /* 0..S-1, or S for the f block */) {
  const long long N = C->N;
  const bool fblock = (level == C->S);
  const double cc = fblock ? 1.0 : C->cs;
  const double* d64 = fblock ? C->zero64 : C->dvec64 + (long long)level * N;
  const float* d32 = fblock ? C->zero32 : C->dvec32 + (long long)level * N;
  const float* db32 = fblock ? nullptr : C->dbar32;
  const int off = fblock ? 0 : level;
  if (C->opts.precision == TSFDE_PREC_FP64)
    block_solve_fp64(C, st, b, x, d64, d32, db32, off, cc);
  else
    block_solve_fp32(C, st, b, x, d32, db32, off, cc);
}

// y = P^-1 r (forward substitution, Sec. 5.1), enqueued on `st`.
void precond_enqueue(tsfde_ctx* C, cudaStream_t st, const double* r, double* y) {
  const long long N = C->N;
  const int S = C->S;
  for (int sl = 0; sl < S; ++sl) {
    history_rhs(r, y, C->g1, C->g2, C->ew, C->lb, sl, N, st);
    double* xs = y + (long long)sl * N;
    if (sl == 0 || !C->opts.warm_start)
      cudaMemsetAsync(xs, 0, sizeof(double) * N, st);
    else
      cudaMemcpyAsync(xs, xs - N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    block_solve(C, st, C->lb, xs, sl);
  }
  // f block: (alpha/h^omega) D_2^(S) B f = r^(S+1) - y^(S)  <=>  B f = (r^(S+1) - y^(S)) / (cf gamma2^(S))
  fblock_rhs(r + (long long)S * N, y + (long long)(S - 1) * N, C->g2 + (long long)(S - 1) * N, C->cf, C->lb, N, st);
  double* xf = y + (long long)S * N;
  cudaMemsetAsync(xf, 0, sizeof(double) * N, st);
  block_solve(C, st, C->lb, xf, S);
}

cudaEvent_t prof_event(tsfde_ctx::Prof& P) {
  if (!P.pool.empty()) {
    cudaEvent_t e = P.pool.back();
    P.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// begin/end of a profiled unit on stream st (no-op when profiling is off)
void prof_begin(tsfde_ctx* C, int which, cudaStream_t st) {
  if (!C->prof_on) return;
  auto& P = C->prof[which];
  cudaEvent_t a = prof_event(P), b = prof_event(P);
  cudaEventRecord(a, st);
  P.pending.push_back({a, b});
}
void prof_end(tsfde_ctx* C, int which, cudaStream_t st) {
  if (!C->prof_on) return;
  auto& P = C->prof[which];
  if (!P.pending.empty()) cudaEventRecord(P.pending.back().second, st);
}
void prof_resolve(tsfde_ctx* C) {
  for (auto& P : C->prof) {
    for (auto& pr : P.pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
        P.ms += ms;
        P.count += 1;
      }
      P.pool.push_back(pr.first);
      P.pool.push_back(pr.second);
    }
    P.pending.clear();
  }
}

void drop_graph(tsfde_ctx* C) {
  if (C->gexec) cudaGraphExecDestroy(C->gexec);
  C->gexec = nullptr;
  C->graph_prec = -1;
}

// Tables of S_{n,S} (block_solver = 2), built once per handle on first use.
tsfde_status ensure_strang(tsfde_ctx* C) {
  if (C->strang_ready) return TSFDE_OK;
  const int L = 2 * (C->np + 1);
  TSFDE_TRY(dalloc(C, &C->str_chirp64, C->n));
  TSFDE_TRY(dalloc(C, &C->str_chirp32, C->n));
  TSFDE_TRY(dalloc(C, &C->str_bhat64, L));
  TSFDE_TRY(dalloc(C, &C->str_bhat32, L));
  TSFDE_TRY(dalloc(C, &C->str_lam64, (size_t)C->N));
  TSFDE_TRY(dalloc(C, &C->str_lam32, (size_t)C->N));
  TSFDE_CU(build_strang(C->d, C->n, L, C->a_tab, C->str_chirp64, C->str_chirp32, C->str_bhat64, C->str_bhat32,
                        C->str_lam64, C->st));
  cast_d2f(C->str_lam64, C->str_lam32, C->N, C->st);
  TSFDE_TRY(check_launch("S_{n,S} tables"));
  C->strang_ready = true;
  return TSFDE_OK;
}

// One cooperative launch of the persistent forward substitution (fsub.cu).
// Arguments of one instance's persistent forward (trans = 0) or backward (trans = 1) substitution.
void fill_fsub_args(tsfde_ctx* C, const double* r, double* y, int trans, FsubArgs& a) {
  a = FsubArgs{};
  a.trans = trans;
  a.d = C->d;
  a.n = C->n;
  a.L = 2 * (C->np + 1);
  a.t1_64 = C->t1_64;
  a.t2_64 = C->t2_64;
  a.t1_32 = C->t1_32;
  a.t2_32 = C->t2_32;
  a.S = C->S;
  a.N = C->N;
  a.mode = (C->opts.precision == TSFDE_PREC_FP64) ? 0 : 1;
  a.refine_max = C->opts.refine_max;
  // the zero-padded tau preconditioner of grids with n + 1 not a power of two is weaker: twice the cap
  a.pcg_iters = C->opts.pcg_iters * (C->np != C->n ? 2 : 1);
  a.pcg_max = C->opts.pcg_max;
  a.warm = (C->opts.precision == TSFDE_PREC_FP64) ? C->opts.warm_start : C->opts.warm_start_mixed;
  a.spin_limit = C->opts.spin_limit;
  a.tol2_outer = C->opts.inner_tol * C->opts.inner_tol;
  a.tol2_inner = C->opts.inner_tol_corr * C->opts.inner_tol_corr;
  a.tol2_mixed = C->opts.inner_tol_mixed * C->opts.inner_tol_mixed;
  a.cs = C->cs;
  a.cf = C->cf;
  a.r = r;
  a.y = y;
  a.g1 = C->g1;
  a.g2 = C->g2;
  a.ew = C->ew;
  a.dvec64 = C->dvec64;
  a.dvec32 = C->dvec32;
  a.dbar32 = C->dbar32;
  a.tw64 = C->tw64;
  a.tw32 = C->tw32;
  a.lam64 = C->lam64;
  a.mu64 = C->mu64;
  a.lam32 = C->lam32;
  a.mu32 = C->mu32;
  a.w64a = C->sp64_one.work0;
  a.w64b = C->sp64_one.work1;
  a.w32a = C->sp32_one.work0;
  a.w32b = C->sp32_one.work1;
  a.lb = C->lb;
  a.lBx = C->lBx;
  a.hfar = C->fsub_hfar;
  a.lb32 = C->lb32;
  a.lx32 = C->lx32;
  a.lr32 = C->lr32;
  a.lz32 = C->lz32;
  a.lp32 = C->lp32;
  a.lq32 = C->lq32;
  a.fused = (C->opts.fused_cg && C->d >= 2) ? 1 : 0;
  a.block_solver = C->opts.block_solver;
  a.sch64 = C->str_chirp64;
  a.sbh64 = C->str_bhat64;
  a.sch32 = C->str_chirp32;
  a.sbh32 = C->str_bhat32;
  a.slam64 = C->str_lam64;
  a.slam32 = C->str_lam32;
  a.dbar64 = C->dbar64;
  a.ltr32 = C->ltr32;
  a.ltq32 = C->ltq32;
  a.w32z = C->w32z;
  a.w32p = C->w32p;
  a.zero64 = C->zero64;
  a.zero32 = C->zero32;
  a.part = C->fsub_part;
  a.bar.count = C->fsub_bar;
  a.bar.err = reinterpret_cast<int*>(C->fsub_bar + 2);
  a.stats = C->sc;
  a.trace = C->timeline_on ? C->trace : nullptr;
  a.trace_cap = C->trace_cap;
  a.trace_len = C->timeline_on ? C->trace_len : nullptr;
}

// One cooperative launch of the persistent substitution for `count` instances with the same
// transform length, on the stream of the first.  Each instance gets a sub-grid of gper CTAs with
// its own barrier counter and partials; the other instances' streams are ordered with events.
// One cooperative launch of the mixed-length kernel for instances whose transform lengths (or
// dimensions) differ.  CTAs (one per SM, 512 threads): a one-dimensional instance runs on one CTA;
// the others share the rest in proportion to their unknowns, at least one each.
tsfde_status fsub_mixed_batch_launch(tsfde_ctx* const* Cs, const double* const* rs, double* const* ys,
                                     const int* trans, int count) {
  tsfde_ctx* C0 = Cs[0];
  cudaStream_t st = C0->st;
  for (int i = 0; i < count; ++i) {
    if (Cs[i]->opts.block_solver == 2 && !Cs[i]->strang_ready) {
      set_error("S_{n,S}: the Strang tables of an instance are missing");
      return TSFDE_EINVAL;
    }
  }
  size_t smem = 0;
  for (int i = 0; i < count; ++i) smem = std::max(smem, fsub_mixed_smem(2 * (Cs[i]->np + 1)));
  int dev = 0, sms = 0;
  TSFDE_CU(cudaGetDevice(&dev));
  TSFDE_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int gmax = std::min(fsub_mixed_max_grid(smem, sms), kMaxMixedGrid);
  if (gmax < count) {
    set_error("batch: " + std::to_string(count) + " instances of different transform lengths do not fit one "
              "co-resident launch of the mixed-length kernel (" + std::to_string(gmax) + " CTAs)");
    return TSFDE_EINVAL;
  }
  std::vector<int> gper(count, 1);
  double wsum = 0.0;
  int n1 = 0;
  for (int i = 0; i < count; ++i) {
    if (Cs[i]->d == 1) ++n1;
    else wsum += (double)Cs[i]->U;
  }
  const int rest = gmax - n1;
  int used = n1;
  for (int i = 0; i < count; ++i) {
    if (Cs[i]->d == 1) continue;
    int g = (int)((double)rest * (double)Cs[i]->U / wsum);
    g = std::max(1, std::min(g, Cs[i]->fsub_grid));
    gper[i] = g;
    used += g;
  }
  while (used > gmax) {  // rounding up to one CTA each can overshoot: take from the largest
    int k = 0;
    for (int i = 1; i < count; ++i)
      if (gper[i] > gper[k]) k = i;
    if (gper[k] <= 1) break;
    --gper[k];
    --used;
  }
  FsubArgs host[kMaxBatch];
  std::vector<int> cta;
  cta.reserve(used);
  std::vector<const void*> key_bar(count);
  for (int i = 0; i < count; ++i) {
    tsfde_ctx* C = Cs[i];
    fill_fsub_args(C, rs[i], ys[i], trans[i], host[i]);
    host[i].gper = gper[i];
    host[i].cta0 = (int)cta.size();
    for (int b = 0; b < gper[i]; ++b) cta.push_back(i);
    key_bar[i] = C->fsub_bar;
    if (i > 0) {
      TSFDE_CU(cudaEventRecord(C->ev_in, C->st));
      TSFDE_CU(cudaStreamWaitEvent(st, C->ev_in, 0));
    }
    prof_begin(C, 0, st);
  }
  const int grid = (int)cta.size();
  FsubMixed m{C0->fsub_args_dev, C0->fsub_cta_dev, count};
  // the launch sequence on stream q: barrier resets of every instance, arguments, the cooperative launch
  auto enqueue = [&](const FsubArgs* args_src, const int* cta_src, cudaStream_t q) -> cudaError_t {
    for (int i = 0; i < count; ++i) {
      cudaError_t e1 = cudaMemsetAsync(Cs[i]->fsub_bar, 0, sizeof(unsigned int), q);
      if (e1 == cudaSuccess) e1 = cudaMemsetAsync(Cs[i]->fsub_bar + 2, 0, sizeof(unsigned int), q);
      if (e1 != cudaSuccess) return e1;
    }
    cudaError_t e1 = cudaMemcpyAsync(C0->fsub_args_dev, args_src, sizeof(FsubArgs) * count, cudaMemcpyHostToDevice, q);
    if (e1 == cudaSuccess)
      e1 = cudaMemcpyAsync(C0->fsub_cta_dev, cta_src, sizeof(int) * grid, cudaMemcpyHostToDevice, q);
    if (e1 == cudaSuccess) e1 = fsub_mixed_launch(m, grid, smem, q);
    return e1;
  };
  cudaError_t e = cudaSuccess;
  bool done = false;
  if (C0->opts.graphs && !C0->mix_graph_failed) {
    if (!C0->mix_args_pin) {
      TSFDE_CU(cudaMallocHost((void**)&C0->mix_args_pin, sizeof(FsubArgs) * kMaxBatch));
      TSFDE_CU(cudaMallocHost((void**)&C0->mix_cta_pin, sizeof(int) * kMaxMixedGrid));
      TSFDE_CU(cudaEventCreateWithFlags(&C0->mix_done, cudaEventDisableTiming));
    }
    // the previous replay has read the staging buffers before they are rewritten
    if (C0->mix_done_valid) TSFDE_CU(cudaEventSynchronize(C0->mix_done));
    memcpy(C0->mix_args_pin, host, sizeof(FsubArgs) * count);
    memcpy(C0->mix_cta_pin, cta.data(), sizeof(int) * grid);
    // captured and replayed on the handle's internal stream (the caller's stream may be the legacy
    // default stream, which cannot be captured), ordered with the caller's stream by events
    cudaStream_t q = C0->gst;
    if (!(C0->mix_exec && C0->mix_key_bar == key_bar && C0->mix_key_g == gper && C0->mix_key_smem == smem)) {
      if (C0->mix_exec) cudaGraphExecDestroy(C0->mix_exec);
      C0->mix_exec = nullptr;
      cudaGraph_t g = nullptr;
      cudaError_t ec = cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal);
      if (ec == cudaSuccess) {
        const cudaError_t eq = enqueue(C0->mix_args_pin, C0->mix_cta_pin, q);
        ec = cudaStreamEndCapture(q, &g);
        if (eq != cudaSuccess) ec = eq;
      }
      if (ec == cudaSuccess) ec = cudaGraphInstantiate(&C0->mix_exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (ec != cudaSuccess) {
        // capture unavailable (for instance a cooperative launch it does not take): launch directly
        C0->mix_graph_error = cudaGetErrorString(ec);
        cudaGetLastError();
        if (C0->mix_exec) cudaGraphExecDestroy(C0->mix_exec);
        C0->mix_exec = nullptr;
        C0->mix_graph_failed = true;
      } else {
        C0->mix_key_bar = key_bar;
        C0->mix_key_g = gper;
        C0->mix_key_smem = smem;
        C0->mix_graph_builds += 1;
      }
    }
    if (C0->mix_exec) {
      e = cudaEventRecord(C0->ev_in, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(q, C0->ev_in, 0);
      if (e == cudaSuccess) e = cudaGraphLaunch(C0->mix_exec, q);
      if (e == cudaSuccess) e = cudaEventRecord(C0->mix_done, q);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, C0->mix_done, 0);
      C0->mix_done_valid = true;
      C0->mix_graph_replays += 1;
      done = true;
    }
  }
  if (!done) e = enqueue(host, cta.data(), st);
  for (int i = 0; i < count; ++i) prof_end(Cs[i], 0, st);
  if (e != cudaSuccess) {
    set_error(std::string("mixed-length persistent substitution launch: ") + cudaGetErrorString(e));
    return TSFDE_ECUDA;
  }
  C0->launches += 1;
  TSFDE_CU(cudaEventRecord(C0->ev_out, st));
  for (int i = 1; i < count; ++i) TSFDE_CU(cudaStreamWaitEvent(Cs[i]->st, C0->ev_out, 0));
  for (int i = 0; i < count; ++i) Cs[i]->apps_total += 1;
  return TSFDE_OK;
}

tsfde_status fsub_batch_launch(tsfde_ctx* const* Cs, const double* const* rs, double* const* ys, const int* trans,
                               int count) {
  tsfde_ctx* C0 = Cs[0];
  for (int i = 1; i < count; ++i)
    if (Cs[i]->d != C0->d || Cs[i]->np != C0->np) return fsub_mixed_batch_launch(Cs, rs, ys, trans, count);
  cudaStream_t st = C0->st;
  int gmin = C0->fsub_grid;
  for (int i = 1; i < count; ++i) gmin = std::min(gmin, Cs[i]->fsub_grid);
  const int gper = (C0->d == 1) ? 1 : std::max(1, gmin / count);
  if (count * gper > C0->fsub_maxg) {
    set_error("batch: " + std::to_string(count) + " instances do not fit one co-resident launch");
    return TSFDE_EINVAL;
  }
  FsubArgs host[kMaxBatch];
  for (int i = 0; i < count; ++i) {
    if (Cs[i]->opts.block_solver == 2 && !Cs[i]->strang_ready) {
      set_error("S_{n,S}: the Strang tables of an instance are missing");
      return TSFDE_EINVAL;
    }
  }
  for (int i = 0; i < count; ++i) {
    tsfde_ctx* C = Cs[i];
    fill_fsub_args(C, rs[i], ys[i], trans[i], host[i]);
    if (i > 0) {
      TSFDE_CU(cudaEventRecord(C->ev_in, C->st));
      TSFDE_CU(cudaStreamWaitEvent(st, C->ev_in, 0));
    }
    // a previous time-out may have left the arrival counter and the flag set
    TSFDE_CU(cudaMemsetAsync(C->fsub_bar, 0, sizeof(unsigned int), st));
    TSFDE_CU(cudaMemsetAsync(C->fsub_bar + 2, 0, sizeof(unsigned int), st));
    prof_begin(C, 0, st);
  }
  TSFDE_CU(cudaMemcpyAsync(C0->fsub_args_dev, host, sizeof(FsubArgs) * count, cudaMemcpyHostToDevice, st));
  FsubBatch b{C0->fsub_args_dev, count, gper};
  cudaError_t e = fsub_launch(2 * (C0->np + 1), b, st);
  for (int i = 0; i < count; ++i) prof_end(Cs[i], 0, st);
  if (e != cudaSuccess) {
    set_error(std::string("persistent substitution launch: ") + cudaGetErrorString(e));
    return TSFDE_ECUDA;
  }
  C0->launches += 1;
  if (count > 1) {
    TSFDE_CU(cudaEventRecord(C0->ev_out, st));
    for (int i = 1; i < count; ++i) TSFDE_CU(cudaStreamWaitEvent(Cs[i]->st, C0->ev_out, 0));
  }
  for (int i = 0; i < count; ++i) Cs[i]->apps_total += 1;
  if (count == 1 && C0->timeline_on && C0->trace) {
    tsfde_ctx* C = C0;
    int len = 0;
    TSFDE_CU(cudaMemcpyAsync(&len, C->trace_len, sizeof(int), cudaMemcpyDeviceToHost, C->st));
    TSFDE_CU(cudaStreamSynchronize(C->st));
    if (len > 0) {
      std::vector<unsigned long long> tr(2 * (size_t)len);
      TSFDE_CU(cudaMemcpy(tr.data(), C->trace, sizeof(unsigned long long) * 2 * len, cudaMemcpyDeviceToHost));
      for (int i = 1; i < len; ++i) {
        const int kind = (int)tr[2 * i + 1];
        if (kind >= 0 && kind < PH_COUNT) {
          C->phase_ms[kind] += (double)(tr[2 * i] - tr[2 * i - 2]) * 1e-6;
          C->phase_n[kind] += 1;
        }
      }
    }
  }
  return TSFDE_OK;
}

}  // namespace

// The preconditioner calls of several handles' solves, gathered into batched launches: each
// solve runs on its own host thread; a call blocks until every solve still running has made its
// call, and the last one to arrive launches them all at once.
struct BatchCoord {
  std::mutex m;
  std::condition_variable cv;
  int active = 0;
  long long gen = 0;
  tsfde_status status = TSFDE_OK;
  std::vector<tsfde_ctx*> Cs;
  std::vector<const double*> rs;
  std::vector<double*> ys;
  std::vector<int> tr;

  std::vector<tsfde_ctx*> order;  // the batch's handles in the caller's order

  void launch_locked() {
    // requests in the caller's order (not arrival order): the same batch always gets the same
    // leading handle, sub-grid layout and hence the same results and the same replayed graph
    const int c = (int)Cs.size();
    std::vector<int> idx(c);
    for (int i = 0; i < c; ++i) idx[i] = i;
    auto rank = [&](tsfde_ctx* C) {
      for (int k = 0; k < (int)order.size(); ++k)
        if (order[k] == C) return k;
      return (int)order.size();
    };
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return rank(Cs[a]) < rank(Cs[b]); });
    std::vector<tsfde_ctx*> Cs2(c);
    std::vector<const double*> rs2(c);
    std::vector<double*> ys2(c);
    std::vector<int> tr2(c);
    for (int i = 0; i < c; ++i) {
      Cs2[i] = Cs[idx[i]];
      rs2[i] = rs[idx[i]];
      ys2[i] = ys[idx[i]];
      tr2[i] = tr[idx[i]];
    }
    status = fsub_batch_launch(Cs2.data(), rs2.data(), ys2.data(), tr2.data(), c);
    Cs.clear();
    rs.clear();
    ys.clear();
    tr.clear();
    ++gen;
    cv.notify_all();
  }
  tsfde_status request(tsfde_ctx* C, const double* r, double* y, int trans) {
    std::unique_lock<std::mutex> lk(m);
    Cs.push_back(C);
    rs.push_back(r);
    ys.push_back(y);
    tr.push_back(trans);
    const long long g = gen;
    if ((int)Cs.size() == active) {
      launch_locked();
    } else {
      cv.wait(lk, [&] { return gen != g; });
    }
    return status;
  }
  void leave() {
    std::lock_guard<std::mutex> lk(m);
    --active;
    if (active > 0 && (int)Cs.size() == active) launch_locked();
  }
};

namespace {

tsfde_status precond_persistent(tsfde_ctx* C, const double* r, double* y, int trans = 0) {
  if (C->coord) return C->coord->request(C, r, y, trans);
  tsfde_ctx* Cs[1] = {C};
  const double* rs[1] = {r};
  double* ys[1] = {y};
  int tr[1] = {trans};
  return fsub_batch_launch(Cs, rs, ys, tr, 1);
}

// Forward substitution.  With graphs enabled the whole application (every level, sweep and
// PCG step) is captured once into a CUDA graph on an internal stream, reading C->pin and
// writing C->pout, and replayed on later calls; the caller's stream is ordered with events.
tsfde_status precond_apply(tsfde_ctx* C, const double* r, double* y) {
  const long long U = C->U;
  if (C->coord) return precond_persistent(C, r, y);
  if (C->opts.block_solver != 0 || C->np != C->n) {
    // T_{n,S}, S_{n,S}, and grids with n + 1 not a power of two, run in the persistent kernel only
    if (C->fsub_grid <= 0) {
      set_error("this preconditioner needs the persistent kernel (cooperative launch unavailable)");
      return TSFDE_EUNSUPPORTED;
    }
    return precond_persistent(C, r, y);
  }
  if (C->opts.persistent && C->fsub_grid > 0) return precond_persistent(C, r, y);
  if (!C->opts.graphs) {
    prof_begin(C, 0, C->st);
    precond_enqueue(C, C->st, r, y);
    prof_end(C, 0, C->st);
    return check_launch("precond_apply");
  }
  if (!C->gexec || C->graph_prec != C->opts.precision || C->graph_key != opts_key(C->opts)) {
    drop_graph(C);
    // one eager run first (sets kernel attributes), then capture
    if (r != C->pin) TSFDE_CU(cudaMemcpyAsync(C->pin, r, sizeof(double) * U, cudaMemcpyDeviceToDevice, C->st));
    precond_enqueue(C, C->st, C->pin, C->pout);
    TSFDE_TRY(check_launch("precond_apply (eager)"));
    TSFDE_CU(cudaStreamSynchronize(C->st));
    cudaGraph_t g = nullptr;
    TSFDE_CU(cudaStreamBeginCapture(C->gst, cudaStreamCaptureModeRelaxed));
    precond_enqueue(C, C->gst, C->pin, C->pout);
    cudaError_t ce = cudaStreamEndCapture(C->gst, &g);
    if (ce != cudaSuccess) {
      set_error(std::string("graph capture: ") + cudaGetErrorString(ce));
      cudaGetLastError();
      return TSFDE_ECUDA;
    }
    {
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
      long long kcount = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kcount;
      }
      C->graph_kernels = kcount;
      C->launches += kcount;   // the eager run above launched the same kernels
    }
    ce = cudaGraphInstantiate(&C->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      C->gexec = nullptr;
      set_error(std::string("graph instantiate: ") + cudaGetErrorString(ce));
      return TSFDE_ECUDA;
    }
    C->graph_prec = C->opts.precision;
    C->graph_key = opts_key(C->opts);
    if (y != C->pout) TSFDE_CU(cudaMemcpyAsync(y, C->pout, sizeof(double) * U, cudaMemcpyDeviceToDevice, C->st));
    return check_launch("precond_apply");
  }
  if (r != C->pin) TSFDE_CU(cudaMemcpyAsync(C->pin, r, sizeof(double) * U, cudaMemcpyDeviceToDevice, C->st));
  TSFDE_CU(cudaEventRecord(C->ev_in, C->st));
  TSFDE_CU(cudaStreamWaitEvent(C->gst, C->ev_in, 0));
  prof_begin(C, 0, C->gst);
  TSFDE_CU(cudaGraphLaunch(C->gexec, C->gst));
  prof_end(C, 0, C->gst);
  C->launches += C->graph_kernels;
  C->apps_total += 1;
  TSFDE_CU(cudaEventRecord(C->ev_out, C->gst));
  TSFDE_CU(cudaStreamWaitEvent(C->st, C->ev_out, 0));
  if (y != C->pout) TSFDE_CU(cudaMemcpyAsync(y, C->pout, sizeof(double) * U, cudaMemcpyDeviceToDevice, C->st));
  return check_launch("precond_apply");
}

tsfde_status matvec(tsfde_ctx* C, const double* y, double* z) {
  prof_begin(C, 1, C->st);
  bapply<double>(C->sp64_all, y, C->By, C->S + 1, nullptr, C->st);
  matvec_time(y, C->By, C->g1, C->g2, C->q, C->ew, z, C->S, C->N, C->cs, C->cf, C->eta, C->st);
  prof_end(C, 1, C->st);
  C->launches += (C->d == 1 ? 1 : (C->d == 2 ? 3 : 5)) + 1;
  return check_launch("matvec");
}

// z = A^T lam: u = D_2 lam, B_n u for all S + 1 fields, then the transposed time sum and coupling.
tsfde_status matvec_T(tsfde_ctx* C, const double* lam, double* z) {
  if (!C->adj_u) TSFDE_TRY(dalloc(C, &C->adj_u, (size_t)C->U));
  prof_begin(C, 1, C->st);
  scale_gamma2(lam, C->g2, C->adj_u, C->S, C->N, C->st);
  bapply<double>(C->sp64_all, C->adj_u, C->By, C->S + 1, nullptr, C->st);
  matvec_time_T(lam, C->By, C->g1, C->q, C->ew, z, C->S, C->N, C->cs, C->cf, C->eta, C->st);
  prof_end(C, 1, C->st);
  C->launches += (C->d == 1 ? 1 : (C->d == 2 ? 3 : 5)) + 2;
  return check_launch("matvec_T");
}

// y = P^-T r: the backward substitution always runs as the persistent kernel.
tsfde_status precond_apply_T(tsfde_ctx* C, const double* r, double* y) {
  if (C->fsub_grid <= 0) {
    set_error("P^-T needs the persistent kernel (cooperative launch unavailable)");
    return TSFDE_EUNSUPPORTED;
  }
  return precond_persistent(C, r, y, 1);
}

double read_scalar(tsfde_ctx* C, const double* dev) {
  cudaMemcpyAsync(C->host_scal, dev, sizeof(double), cudaMemcpyDeviceToHost, C->st);
  cudaStreamSynchronize(C->st);
  return C->host_scal[0];
}

}  // namespace

// =======================================================================================
// ABI
// =======================================================================================
extern "C" {

void tsfde_default_opts(tsfde_opts* o) {
  if (!o) return;
  o->precision = TSFDE_PREC_FP64;
  o->side = TSFDE_SIDE_LEFT;
  o->restart = 30;
  o->max_iters = 3000;
  o->tol = 1e-10;
  o->inner_tol = 1e-11;
  o->inner_tol_mixed = 1e-5;
  o->pcg_iters = 6;
  o->pcg_max = 20;
  o->refine_max = 6;
  o->coeff_K = 0;
  o->graphs = 1;
  o->persistent = 1;
  o->warm_start = 6;
  o->fused_cg = 1;
  o->inner_tol_corr = 3e-6;
  o->block_solver = 0;
  o->spin_limit = 1LL << 24;
  o->warm_start_mixed = 3;
  o->grid_ctas = 0;
}

const char* tsfde_status_string(tsfde_status s) {
  switch (s) {
    case TSFDE_OK: return "ok";
    case TSFDE_NOT_CONVERGED: return "not converged";
    case TSFDE_EINVAL: return "invalid argument";
    case TSFDE_ENOMEM: return "out of device memory";
    case TSFDE_ECUDA: return "CUDA error";
    case TSFDE_EBREAKDOWN: return "breakdown (NaN/Inf or zero pivot)";
    case TSFDE_EUNSUPPORTED: return "unsupported size or option";
    case TSFDE_ETIMEOUT: return "a bounded device wait expired";
  }
  return "unknown status";
}

const char* tsfde_last_error(void) { return tsfde::g_last_error.c_str(); }

size_t tsfde_device_bytes(tsfde_handle h) { return h ? h->bytes : 0; }

static tsfde_status setup_impl(tsfde_ctx* C, const tsfde_grid* g, double beta, double omega, double alpha,
                               const double* gamma1, const double* gamma2, const double* q, const double* rho,
                               const double* mu) {
  const int d = g->d, n = g->n, S = g->S;
  C->d = d;
  C->n = n;
  C->S = S;
  long long N = 1;
  for (int i = 0; i < d; ++i) N *= n;
  C->N = N;
  C->U = (long long)(S + 1) * N;
  C->length = g->length;
  C->T = g->T;
  C->h = g->length / (n + 1);
  C->dt = g->T / S;
  C->beta = beta;
  C->omega = omega;
  C->alpha = alpha;
  C->eta = pow(C->dt, beta) * tgamma(2.0 - beta);
  C->cs = C->eta / pow(C->h, omega);
  C->cf = alpha / pow(C->h, omega);
  cudaStream_t st = C->st;
  // transform grid: L = 2 (np + 1) with np + 1 the smallest power of two >= n + 1 (np = n when n + 1
  // is a power of two); B_n is embedded in a circulant of size L >= 2 n - 1, and the tau solves of
  // the inner CG work on the zero-padded np grid
  int p2 = 1;
  while (p2 < n + 1) p2 <<= 1;
  const int np = p2 - 1;
  C->np = np;
  const int L = 2 * (np + 1), H = L / 2 + 1;
  long long Np = 1;
  for (int i = 0; i < d; ++i) Np *= np;

  // inputs (host or device; cudaMemcpyDefault resolves the direction through unified addressing)
  TSFDE_TRY(dalloc(C, &C->g1, (size_t)S * N));
  TSFDE_TRY(dalloc(C, &C->g2, (size_t)S * N));
  TSFDE_TRY(dalloc(C, &C->q, S));
  TSFDE_TRY(dalloc(C, &C->rho, N));
  TSFDE_TRY(dalloc(C, &C->mu, N));
  TSFDE_CU(cudaMemcpyAsync(C->g1, gamma1, sizeof(double) * S * N, cudaMemcpyDefault, st));
  TSFDE_CU(cudaMemcpyAsync(C->g2, gamma2, sizeof(double) * S * N, cudaMemcpyDefault, st));
  TSFDE_CU(cudaMemcpyAsync(C->q, q, sizeof(double) * S, cudaMemcpyDefault, st));
  TSFDE_CU(cudaMemcpyAsync(C->rho, rho, sizeof(double) * N, cudaMemcpyDefault, st));
  TSFDE_CU(cudaMemcpyAsync(C->mu, mu, sizeof(double) * N, cudaMemcpyDefault, st));
  {
    // gamma2 > 0 everywhere: the symmetrised block solves divide by it and need D_2 B_n SPD
    unsigned int* bad_dev = nullptr;
    TSFDE_TRY(dalloc(C, &bad_dev, 1));
    TSFDE_CU(cudaMemsetAsync(bad_dev, 0, sizeof(unsigned int), st));
    count_nonpositive(C->g2, (long long)S * N, bad_dev, st);
    unsigned int bad = 0;
    TSFDE_CU(cudaMemcpyAsync(&bad, bad_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    TSFDE_CU(cudaStreamSynchronize(st));
    if (bad) {
      set_error("tsfde_setup: gamma2 must be finite and positive (" + std::to_string(bad) + " entries are not)");
      return TSFDE_EINVAL;
    }
  }

  // L1 weights (Sec. 4): b_m = (m+1)^(1-beta) - m^(1-beta), e_0 = b_0, e_m = b_m - b_{m-1}
  {
    std::vector<double> bh(S), eh(S);
    for (int m = 0; m < S; ++m) bh[m] = pow(m + 1.0, 1.0 - beta) - pow((double)m, 1.0 - beta);
    eh[0] = bh[0];
    for (int m = 1; m < S; ++m) eh[m] = bh[m] - bh[m - 1];
    TSFDE_TRY(dalloc(C, &C->bw, S));
    TSFDE_TRY(dalloc(C, &C->ew, S));
    TSFDE_CU(cudaMemcpyAsync(C->bw, bh.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st));
    TSFDE_CU(cudaMemcpyAsync(C->ew, eh.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st));
    TSFDE_CU(cudaStreamSynchronize(st));
  }

  // fractional coefficients a_l: d = 1 by the recursion of Lemma 1(b) from a_0 of Lemma 1(a);
  // d >= 2 by the K-point trapezoid rule for Eq. 8
  // (a_tab: l < n per axis, the entries of B_n; a_tau: l < np, for tau(B_np) on the padded grid)
  TSFDE_TRY(dalloc(C, &C->a_tab, N));
  TSFDE_TRY(dalloc(C, &C->a_tau, Np));
  if (d == 1) {
    std::vector<double> a(np);
    a[0] = tgamma(omega + 1.0) / (tgamma(omega / 2.0 + 1.0) * tgamma(omega / 2.0 + 1.0));
    for (int l = 0; l + 1 < np; ++l) a[l + 1] = (1.0 - (omega + 1.0) / (omega / 2.0 + l + 1.0)) * a[l];
    TSFDE_CU(cudaMemcpy(C->a_tab, a.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    TSFDE_CU(cudaMemcpy(C->a_tau, a.data(), sizeof(double) * np, cudaMemcpyHostToDevice));
  } else {
    const int K = C->opts.coeff_K > 0 ? C->opts.coeff_K : default_K(d, n);
    TSFDE_CU(build_coeffs_dft(d, n, omega, K, C->a_tab, st));
    if (np == n) TSFDE_CU(cudaMemcpyAsync(C->a_tau, C->a_tab, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    else TSFDE_CU(build_coeffs_dft(d, np, omega, K, C->a_tau, st));
  }

  // circulant symbol and tau eigenvalues
  long long lam_sz = H;
  for (int i = 1; i < d; ++i) lam_sz *= L;
  TSFDE_TRY(dalloc(C, &C->lam64, lam_sz));
  TSFDE_TRY(dalloc(C, &C->mu64, Np));
  TSFDE_TRY(dalloc(C, &C->lam32, lam_sz));
  TSFDE_TRY(dalloc(C, &C->mu32, Np));
  TSFDE_CU(build_symbols(d, n, np, C->a_tab, C->a_tau, C->lam64, C->mu64, st));
  cast_d2f(C->lam64, C->lam32, lam_sz, st);
  cast_d2f(C->mu64, C->mu32, Np, st);
  {
    void *t64 = nullptr, *t32 = nullptr;
    TSFDE_CU(make_twiddles(L, &t64, &t32, st));
    C->tw64 = (double2*)t64;
    C->tw32 = (float2*)t32;
  }

  // symmetrised block diagonals e_0 gamma1 / gamma2 and their per-level means
  TSFDE_TRY(dalloc(C, &C->dvec64, (size_t)S * N));
  TSFDE_TRY(dalloc(C, &C->dvec32, (size_t)S * N));
  TSFDE_TRY(dalloc(C, &C->dbar64, S));
  TSFDE_TRY(dalloc(C, &C->dbar32, S));
  block_diag(C->g1, C->g2, 1.0 /* e_0 = b_0 = 1 */, C->dvec64, C->dvec32, (long long)S * N, st);
  level_mean(C->dvec64, C->dbar64, C->dbar32, S, N, st);
  TSFDE_TRY(dalloc(C, &C->zero64, N));
  TSFDE_TRY(dalloc(C, &C->zero32, N));
  TSFDE_CU(cudaMemsetAsync(C->zero64, 0, sizeof(double) * N, st));
  TSFDE_CU(cudaMemsetAsync(C->zero32, 0, sizeof(float) * N, st));

  // spatial plans
  auto fill = [&](auto& P, auto* tw, auto* lam, auto* muv, int F) -> tsfde_status {
    P.d = d;
    P.n = n;
    P.L = L;
    P.H = H;
    P.N = N;
    P.max_fields = F;
    P.tw = tw;
    P.lam = lam;
    P.mu = muv;
    P.work_elems = spatial_work_elems(d, n, L, F);
    if (d >= 2) TSFDE_TRY(dalloc(C, &P.work0, P.work_elems));
    if (d == 3) TSFDE_TRY(dalloc(C, &P.work1, P.work_elems));
    return TSFDE_OK;
  };
  TSFDE_TRY(fill(C->sp64_all, C->tw64, C->lam64, C->mu64, S + 1));
  TSFDE_TRY(fill(C->sp64_one, C->tw64, C->lam64, C->mu64, 1));
  TSFDE_TRY(fill(C->sp32_one, C->tw32, C->lam32, C->mu32, 1));

  // workspaces
  TSFDE_TRY(dalloc(C, &C->By, (size_t)C->U));
  for (double** p : {&C->lb, &C->lr64, &C->lz64, &C->lp64, &C->lq64}) TSFDE_TRY(dalloc(C, p, N));
  TSFDE_TRY(dalloc(C, &C->lBx, 8 * (size_t)N));
  for (float** p : {&C->lx32, &C->lr32, &C->lz32, &C->lp32, &C->lq32, &C->lBp32, &C->lb32}) TSFDE_TRY(dalloc(C, p, N));
  {
    // tau intermediates on the padded coefficient grid: [N / n][np], and [n][np][np] for d = 3
    const size_t t1 = (size_t)(N / n) * np, t2 = (d == 3) ? (size_t)n * np * np : 1;
    for (float** p : {&C->ltr32, &C->ltq32, &C->t1_32}) TSFDE_TRY(dalloc(C, p, t1));
    TSFDE_TRY(dalloc(C, &C->t2_32, t2));
    TSFDE_TRY(dalloc(C, &C->t1_64, t1));
    TSFDE_TRY(dalloc(C, &C->t2_64, t2));
  }
  if (d >= 2) {
    const size_t spec = (size_t)(N / n) * H;  // half spectra of the rows of one field
    TSFDE_TRY(dalloc(C, &C->w32z, spec));
    TSFDE_TRY(dalloc(C, &C->w32p, spec));
  }
  TSFDE_TRY(dalloc(C, &C->sc, 2));
  TSFDE_CU(cudaMemsetAsync(C->sc, 0, sizeof(Scalars) * 2, st));
  TSFDE_TRY(dalloc(C, &C->rw.part, (size_t)kMaxRedBlocks * kMaxRedVals));
  TSFDE_TRY(dalloc(C, &C->rw.ticket, 1));
  TSFDE_CU(cudaMemsetAsync(C->rw.ticket, 0, sizeof(unsigned int), st));
  for (double** p : {&C->x, &C->z, &C->r, &C->w, &C->tmp}) TSFDE_TRY(dalloc(C, p, (size_t)C->U));
  TSFDE_TRY(dalloc(C, &C->H, (size_t)65 * 64));
  for (double** p : {&C->gcs, &C->gsn, &C->gg, &C->h1, &C->h2, &C->yk}) TSFDE_TRY(dalloc(C, p, 65));
  TSFDE_TRY(dalloc(C, &C->dnrm, 4));
  TSFDE_TRY(dalloc(C, &C->dest, 4));
  TSFDE_CU(cudaMallocHost((void**)&C->host_scal, sizeof(double) * 4));
  {
    int dev = 0, sms = 0;
    TSFDE_CU(cudaGetDevice(&dev));
    TSFDE_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int coop = 0;
    TSFDE_CU(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    const int maxg = coop ? fsub_max_grid(L, sms) : 0;
    // one CTA per SM for d >= 2 (fewer CTAs make the grid barrier cheaper); d = 1 fits one CTA
    C->fsub_sms = sms;
    C->fsub_maxg = maxg;
    if (C->opts.grid_ctas > 0 && maxg > 0 && C->opts.grid_ctas > maxg) {
      set_error("grid_ctas above the co-resident limit of the persistent kernel (" + std::to_string(maxg) + ")");
      return TSFDE_EINVAL;
    }
    C->fsub_grid = persistent_grid(C, C->opts);
    TSFDE_TRY(dalloc(C, &C->fsub_args_dev, kMaxBatch));
    TSFDE_TRY(dalloc(C, &C->fsub_cta_dev, kMaxMixedGrid));
    TSFDE_TRY(dalloc(C, &C->fsub_part, (size_t)8 * (maxg > 0 ? maxg : 1)));
    TSFDE_TRY(dalloc(C, &C->fsub_bar, 4));
    TSFDE_TRY(dalloc(C, &C->fsub_hfar, (size_t)16 * N));
    TSFDE_CU(cudaMemsetAsync(C->fsub_bar, 0, sizeof(unsigned int) * 4, st));
  }
  TSFDE_TRY(dalloc(C, &C->pin, (size_t)C->U));
  TSFDE_TRY(dalloc(C, &C->pout, (size_t)C->U));
  TSFDE_CU(cudaStreamCreateWithFlags(&C->gst, cudaStreamNonBlocking));
  TSFDE_CU(cudaEventCreateWithFlags(&C->ev_in, cudaEventDisableTiming));
  TSFDE_CU(cudaEventCreateWithFlags(&C->ev_out, cudaEventDisableTiming));
  TSFDE_TRY(alloc_gmres(C));
  if (C->opts.block_solver == 2) TSFDE_TRY(ensure_strang(C));
  TSFDE_CU(cudaStreamSynchronize(st));
  return check_launch("tsfde_setup");
}

tsfde_status tsfde_setup(tsfde_handle* out, const tsfde_grid* g, double beta, double omega, double alpha,
                         const double* gamma1, const double* gamma2, const double* q, const double* rho,
                         const double* mu, const tsfde_opts* opts, void* stream) {
  if (!out) return TSFDE_EINVAL;
  *out = nullptr;
  set_error("");
  if (!g || !gamma1 || !gamma2 || !q || !rho || !mu) {
    set_error("null argument");
    return TSFDE_EINVAL;
  }
  if (g->d < 1 || g->d > 3 || g->S < 1 || !(g->length > 0) || !(g->T > 0)) {
    set_error("grid: need 1 <= d <= 3, S >= 1, length > 0, T > 0");
    return TSFDE_EINVAL;
  }
  // transforms of length L = 2 p2, p2 the smallest power of two >= n + 1
  const int maxL = (g->d == 1) ? 4096 : (g->d == 2 ? 2048 : 512);
  int p2 = 1;
  while (g->n >= 3 && p2 < g->n + 1) p2 <<= 1;
  if (g->n < 3 || 2 * p2 > maxL) {
    set_error("grid: need 3 <= n <= " + std::to_string(maxL / 2 - 1) + " for d = " + std::to_string(g->d));
    return TSFDE_EUNSUPPORTED;
  }
  if (p2 != g->n + 1 && opts && opts->block_solver == 1) {
    set_error("block_solver = 1 (T_{n,S}) needs n + 1 a power of two (tau(B_n) on the grid itself)");
    return TSFDE_EUNSUPPORTED;
  }
  if (!(beta > 0 && beta < 1) || !(omega > 1 && omega < 2) || !(alpha > 0)) {
    set_error("need 0 < beta < 1, 1 < omega < 2, alpha > 0");
    return TSFDE_EINVAL;
  }
  tsfde_ctx* C = new (std::nothrow) tsfde_ctx();
  if (!C) return TSFDE_ENOMEM;
  if (opts) C->opts = *opts;
  else tsfde_default_opts(&C->opts);
  if (validate_opts(&C->opts) != TSFDE_OK) {
    delete C;
    set_error("invalid options");
    return TSFDE_EINVAL;
  }
  C->st = (cudaStream_t)stream;
  tsfde_status s = setup_impl(C, g, beta, omega, alpha, gamma1, gamma2, q, rho, mu);
  if (s != TSFDE_OK) {
    cudaStreamSynchronize(C->st);
    free_all(C);
    delete C;
    return s;
  }
  *out = C;
  return TSFDE_OK;
}

tsfde_status tsfde_set_opts(tsfde_handle h, const tsfde_opts* opts) {
  if (!h || !opts) return TSFDE_EINVAL;
  if (validate_opts(opts) != TSFDE_OK) return TSFDE_EINVAL;
  if (opts->block_solver == 1 && h->np != h->n) {
    set_error("block_solver = 1 (T_{n,S}) needs n + 1 a power of two (tau(B_n) on the grid itself)");
    return TSFDE_EUNSUPPORTED;
  }
  if (opts->coeff_K != h->opts.coeff_K && h->d >= 2) {
    set_error("coeff_K can only be chosen at setup");
    return TSFDE_EINVAL;
  }
  if (opts->grid_ctas > 0 && h->fsub_maxg > 0 && opts->grid_ctas > h->fsub_maxg) {
    set_error("grid_ctas above the co-resident limit of the persistent kernel (" + std::to_string(h->fsub_maxg) + ")");
    return TSFDE_EINVAL;
  }
  // tables first: the handle keeps its old options if they cannot be built
  if (opts->block_solver == 2) TSFDE_TRY(ensure_strang(h));
  h->opts = *opts;
  if (h->fsub_maxg > 0) h->fsub_grid = persistent_grid(h, h->opts);
  drop_graph(h);
  return alloc_gmres(h);
}

tsfde_status tsfde_rhs(tsfde_handle h, double* z) {
  if (!h || !z) return TSFDE_EINVAL;
  build_rhs(h->g1, h->rho, h->mu, h->bw, z, h->S, h->N, h->st);
  return check_launch("tsfde_rhs");
}

tsfde_status tsfde_matvec(tsfde_handle h, const double* y, double* z) {
  if (!h || !y || !z || y == z) return TSFDE_EINVAL;
  return matvec(h, y, z);
}

tsfde_status tsfde_precond_apply(tsfde_handle h, const double* r, double* y) {
  if (!h || !r || !y || r == y) return TSFDE_EINVAL;
  TSFDE_CU(cudaMemsetAsync(&h->sc[0].fails, 0, sizeof(int), h->st));
  TSFDE_CU(cudaMemsetAsync(&h->sc[1].fails, 0, sizeof(int), h->st));
  TSFDE_TRY(precond_apply(h, r, y));
  int fails[2] = {0, 0};
  unsigned int barerr = 0;
  TSFDE_CU(cudaMemcpyAsync(&fails[0], &h->sc[0].fails, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  TSFDE_CU(cudaMemcpyAsync(&fails[1], &h->sc[1].fails, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  TSFDE_CU(cudaMemcpyAsync(&barerr, h->fsub_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->st));
  TSFDE_CU(cudaStreamSynchronize(h->st));
  if (h->opts.graphs) TSFDE_CU(cudaStreamSynchronize(h->gst));
  if (barerr) {
    set_error("persistent forward substitution: a grid barrier wait expired");
    return TSFDE_ETIMEOUT;
  }
  const int f = (h->opts.precision == TSFDE_PREC_FP64) ? fails[0] : fails[1];
  return f > 0 ? TSFDE_NOT_CONVERGED : TSFDE_OK;
}

}  // extern "C"

namespace tsfde {
namespace {

// Restarted GMRES on A x = z (trans = false) or A^T x = z (trans = true, preconditioned with
// P^T), from the right-hand side in C->z and the initial guess in C->x; the result is copied to
// y (host or device) when y is not null.
tsfde_status gmres_run(tsfde_ctx* C, bool trans, double* y, tsfde_info* info,
                       std::chrono::steady_clock::time_point t0) {
  cudaStream_t st = C->st;
  const long long U = C->U;
  const int m = C->opts.restart;
  const int side = C->opts.side;
  const double tol = C->opts.tol;
  auto MV = [&](const double* in, double* out) { return trans ? matvec_T(C, in, out) : matvec(C, in, out); };
  auto PC = [&](const double* in, double* out) {
    return trans ? precond_apply_T(C, in, out) : precond_apply(C, in, out);
  };

  // reference norm: ||P^-1 z|| (left) or ||z|| (right, flexible)
  double refnorm;
  if (side == TSFDE_SIDE_LEFT) {
    TSFDE_TRY(PC(C->z, C->tmp));
    norm2(C->tmp, U, C->dnrm, C->rw, st);
  } else {
    norm2(C->z, U, C->dnrm, C->rw, st);
  }
  refnorm = sqrt(read_scalar(C, C->dnrm));
  C->launches += 1;
  TSFDE_TRY(check_launch("gmres: reference norm"));
  {
    // NaN / Inf in the data (z) or met by the preconditioner: nothing can be solved
    double zn0 = refnorm;
    if (side == TSFDE_SIDE_LEFT) {
      norm2(C->z, U, C->dnrm, C->rw, st);
      zn0 = sqrt(read_scalar(C, C->dnrm));
      C->launches += 1;
    }
    if (!std::isfinite(refnorm) || !std::isfinite(zn0)) {
      set_error("gmres: the right-hand side or its preconditioned image is not finite");
      return TSFDE_EBREAKDOWN;
    }
  }

  int total = 0, restarts = 0, hist = 0;
  bool converged = false;
  double est_rel = 1.0;
  auto residual = [&]() -> tsfde_status {
    // r = z - A x; left: r <- P^-1 r
    TSFDE_TRY(MV(C->x, C->tmp));
    cudaMemcpyAsync(C->r, C->z, sizeof(double) * U, cudaMemcpyDeviceToDevice, st);
    axpby(-1.0, C->tmp, 1.0, C->r, U, st);
    C->launches += 1;
    if (side == TSFDE_SIDE_LEFT) {
      TSFDE_TRY(PC(C->r, C->tmp));
      cudaMemcpyAsync(C->r, C->tmp, sizeof(double) * U, cudaMemcpyDeviceToDevice, st);
    }
    return TSFDE_OK;
  };
  if (refnorm == 0.0) {
    cudaMemsetAsync(C->x, 0, sizeof(double) * U, st);
    converged = true;
    est_rel = 0.0;
  } else {
    TSFDE_TRY(residual());
  }
  const int ld = m + 1;
  // stagnation: three consecutive restart cycles that each reduce the residual by less than 0.1 %
  // end the solve (not converged): the target lies below the attainable accuracy
  double prev_beta = -1.0;
  int stalled = 0;
  while (!converged && total < C->opts.max_iters) {
    norm2(C->r, U, C->dnrm, C->rw, st);
    double beta0 = sqrt(read_scalar(C, C->dnrm));
    est_rel = beta0 / refnorm;
    if (prev_beta > 0.0 && beta0 > 0.999 * prev_beta) {
      if (++stalled >= 3) break;
    } else {
      stalled = 0;
    }
    prev_beta = beta0;
    if (info && info->history && hist < info->history_cap) info->history[hist++] = est_rel;
    if (!(beta0 == beta0)) {
      set_error("gmres: NaN residual");
      return TSFDE_EBREAKDOWN;
    }
    if (beta0 <= tol * refnorm) {
      converged = true;
      break;
    }
    scale_by_invnorm(C->r, C->V, U, C->dnrm, st);
    init_g(C->gg, m + 1, C->dnrm, st);
    C->launches += 3;
    int k = 0;
    bool cyc_conv = false;
    for (int j = 0; j < m && total < C->opts.max_iters; ++j) {
      double* vj = C->V + (long long)j * C->ldV;
      double* w = C->w;
      if (side == TSFDE_SIDE_LEFT) {
        TSFDE_TRY(MV(vj, C->tmp));
        TSFDE_TRY(PC(C->tmp, w));
      } else if (side == TSFDE_SIDE_RIGHT) {
        TSFDE_TRY(PC(vj, C->tmp));
        TSFDE_TRY(MV(C->tmp, w));
      } else {
        double* zj = C->Zf + (long long)j * C->ldV;
        TSFDE_TRY(PC(vj, zj));
        TSFDE_TRY(MV(zj, w));
      }
      // classical Gram-Schmidt with one reorthogonalisation; per pass the k = j + 1 basis vectors
      // and w are read by the dot products, then the basis and w read and w written by the update:
      // 16 U (2k + 3) algorithmic bytes for the two passes
      prof_begin(C, 2, st);
      multidot(C->V, C->ldV, j + 1, U, w, C->h1, C->rw, st);
      multiaxpy(C->V, C->ldV, j + 1, U, C->h1, -1.0, w, st);
      multidot(C->V, C->ldV, j + 1, U, w, C->h2, C->rw, st);
      multiaxpy(C->V, C->ldV, j + 1, U, C->h2, -1.0, w, st);
      prof_end(C, 2, st);
      if (C->prof_on) C->orth_bytes += 16.0 * (double)U * (2.0 * (j + 1) + 3.0);
      double* Hcol = C->H + (long long)j * ld;
      add_vec(C->h1, C->h2, Hcol, j + 1, st);
      norm2(w, U, C->dnrm, C->rw, st);
      givens_step(Hcol, C->gcs, C->gsn, C->gg, j, C->dnrm, C->dest, st);
      scale_by_invnorm(w, C->V + (long long)(j + 1) * C->ldV, U, C->dnrm, st);
      double est = read_scalar(C, C->dest);
      C->launches += 8;
      TSFDE_TRY(check_launch("gmres: arnoldi step"));
      ++total;
      k = j + 1;
      est_rel = est / refnorm;
      if (info && info->history && hist < info->history_cap) info->history[hist++] = est_rel;
      if (!(est == est)) {
        set_error("gmres: NaN in the Arnoldi process");
        return TSFDE_EBREAKDOWN;
      }
      if (est <= tol * refnorm) {
        cyc_conv = true;
        break;
      }
    }
    // x += Z y_k with y_k = R^-1 g
    tri_solve(C->H, ld, C->gg, k, C->yk, st);
    C->launches += (side == TSFDE_SIDE_RIGHT) ? 4 : 2;
    if (side == TSFDE_SIDE_LEFT) {
      multiaxpy(C->V, C->ldV, k, U, C->yk, 1.0, C->x, st);
    } else if (side == TSFDE_SIDE_RIGHT) {
      cudaMemsetAsync(C->w, 0, sizeof(double) * U, st);
      multiaxpy(C->V, C->ldV, k, U, C->yk, 1.0, C->w, st);
      TSFDE_TRY(PC(C->w, C->tmp));
      axpby(1.0, C->tmp, 1.0, C->x, U, st);
    } else {
      multiaxpy(C->Zf, C->ldV, k, U, C->yk, 1.0, C->x, st);
    }
    ++restarts;
    TSFDE_TRY(residual());
    if (cyc_conv) {
      C->launches += 1;
      norm2(C->r, U, C->dnrm, C->rw, st);
      double rr = sqrt(read_scalar(C, C->dnrm));
      est_rel = rr / refnorm;
      // accept when the recomputed residual also meets the test (tiny slack for rounding)
      if (rr <= 1.5 * tol * refnorm) converged = true;
    }
  }
  // true relative residual ||z - A x|| / ||z||
  TSFDE_TRY(MV(C->x, C->tmp));
  cudaMemcpyAsync(C->w, C->z, sizeof(double) * U, cudaMemcpyDeviceToDevice, st);
  axpby(-1.0, C->tmp, 1.0, C->w, U, st);
  norm2(C->w, U, C->dnrm, C->rw, st);
  double rtrue = sqrt(read_scalar(C, C->dnrm));
  norm2(C->z, U, C->dnrm, C->rw, st);
  double zn = sqrt(read_scalar(C, C->dnrm));
  C->launches += 3;
  if (y) TSFDE_CU(cudaMemcpyAsync(y, C->x, sizeof(double) * U, cudaMemcpyDefault, st));
  int fails[2] = {0, 0};
  unsigned int barerr = 0;
  TSFDE_CU(cudaMemcpyAsync(&fails[0], &C->sc[0].fails, sizeof(int), cudaMemcpyDeviceToHost, st));
  TSFDE_CU(cudaMemcpyAsync(&fails[1], &C->sc[1].fails, sizeof(int), cudaMemcpyDeviceToHost, st));
  TSFDE_CU(cudaMemcpyAsync(&barerr, C->fsub_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  TSFDE_CU(cudaStreamSynchronize(st));
  if (barerr) {
    set_error("persistent forward substitution: a grid barrier wait expired");
    return TSFDE_ETIMEOUT;
  }
  TSFDE_TRY(check_launch("gmres: final"));
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->iters = total;
    info->restarts = restarts;
    info->converged = converged ? 1 : 0;
    info->relres_est = est_rel;
    info->relres_true = zn > 0 ? rtrue / zn : rtrue;
    info->seconds = std::chrono::duration<double>(t1 - t0).count();
    info->precond_failures = (C->opts.precision == TSFDE_PREC_FP64) ? fails[0] : fails[1];
    info->history_len = hist;
  }
  return converged ? TSFDE_OK : TSFDE_NOT_CONVERGED;
}

// M = A (which = 0) or P^-1 A (which = 1), and its transpose A^T P^-T, applied to in -> out.
tsfde_status spec_apply(tsfde_ctx* C, int which, bool transpose, const double* in, double* out) {
  if (which == 0) return transpose ? matvec_T(C, in, out) : matvec(C, in, out);
  if (!transpose) {
    TSFDE_TRY(matvec(C, in, C->tmp));
    return precond_apply(C, C->tmp, out);
  }
  TSFDE_TRY(precond_apply_T(C, in, C->tmp));
  return matvec_T(C, C->tmp, out);
}

// w -= Q Q^T w for the j vectors of Q (stride U), twice (classical Gram-Schmidt with one
// reorthogonalisation), in chunks of 64 vectors; the coefficients of both passes are added into
// hcol[0..j) when hcol is not null (device).
void reorth(tsfde_ctx* C, const double* Q, int j, double* w, double* hcol) {
  for (int pass = 0; pass < 2; ++pass)
    for (int c0 = 0; c0 < j; c0 += 64) {
      const int cnt = std::min(64, j - c0);
      const double* Qc = Q + (long long)c0 * C->U;
      multidot(Qc, C->U, cnt, C->U, w, C->h1, C->rw, C->st);
      multiaxpy(Qc, C->U, cnt, C->U, C->h1, -1.0, w, C->st);
      if (hcol) add_vec(hcol + c0, C->h1, hcol + c0, cnt, C->st);
      C->launches += hcol ? 3 : 2;
    }
}

struct DevBuf {
  double* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace
}  // namespace tsfde

extern "C" {

tsfde_status tsfde_gmres_solve(tsfde_handle C, double* y, tsfde_info* info) {
  if (!C || !y) return TSFDE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = C->st;
  TSFDE_TRY(alloc_gmres(C));
  TSFDE_CU(cudaMemsetAsync(&C->sc[0].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemsetAsync(&C->sc[1].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemcpyAsync(C->x, y, sizeof(double) * C->U, cudaMemcpyDefault, st));
  build_rhs(C->g1, C->rho, C->mu, C->bw, C->z, C->S, C->N, st);
  C->launches += 1;
  return gmres_run(C, false, y, info, t0);
}

tsfde_status tsfde_solve(tsfde_handle C, const double* z, double* y, tsfde_info* info) {
  if (!C || !z || !y) return TSFDE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = C->st;
  TSFDE_TRY(alloc_gmres(C));
  TSFDE_CU(cudaMemsetAsync(&C->sc[0].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemsetAsync(&C->sc[1].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemcpyAsync(C->x, y, sizeof(double) * C->U, cudaMemcpyDefault, st));
  TSFDE_CU(cudaMemcpyAsync(C->z, z, sizeof(double) * C->U, cudaMemcpyDefault, st));
  return gmres_run(C, false, y, info, t0);
}

tsfde_status tsfde_matvec_transpose(tsfde_handle h, const double* lam, double* z) {
  if (!h || !lam || !z || lam == z) return TSFDE_EINVAL;
  return matvec_T(h, lam, z);
}

tsfde_status tsfde_precond_apply_transpose(tsfde_handle h, const double* r, double* y) {
  if (!h || !r || !y || r == y) return TSFDE_EINVAL;
  TSFDE_CU(cudaMemsetAsync(&h->sc[0].fails, 0, sizeof(int), h->st));
  TSFDE_CU(cudaMemsetAsync(&h->sc[1].fails, 0, sizeof(int), h->st));
  TSFDE_TRY(precond_apply_T(h, r, y));
  int fails[2] = {0, 0};
  unsigned int barerr = 0;
  TSFDE_CU(cudaMemcpyAsync(&fails[0], &h->sc[0].fails, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  TSFDE_CU(cudaMemcpyAsync(&fails[1], &h->sc[1].fails, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  TSFDE_CU(cudaMemcpyAsync(&barerr, h->fsub_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->st));
  TSFDE_CU(cudaStreamSynchronize(h->st));
  if (barerr) {
    set_error("persistent backward substitution: a grid barrier wait expired");
    return TSFDE_ETIMEOUT;
  }
  const int f = (h->opts.precision == TSFDE_PREC_FP64) ? fails[0] : fails[1];
  return f > 0 ? TSFDE_NOT_CONVERGED : TSFDE_OK;
}

tsfde_status tsfde_adjoint(tsfde_handle C, const double* y, const double* ybar, double* lam, double* dJ_dalpha,
                           double* dJ_dmu, double* dJ_dgamma2, tsfde_info* info) {
  if (!C || !ybar) return TSFDE_EINVAL;
  const bool grads = dJ_dalpha || dJ_dmu || dJ_dgamma2;
  if (grads && !y) return TSFDE_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = C->st;
  const long long U = C->U, N = C->N;
  const int S = C->S;
  TSFDE_TRY(alloc_gmres(C));
  TSFDE_CU(cudaMemsetAsync(&C->sc[0].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemsetAsync(&C->sc[1].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemsetAsync(C->x, 0, sizeof(double) * U, st));
  TSFDE_CU(cudaMemcpyAsync(C->z, ybar, sizeof(double) * U, cudaMemcpyDefault, st));
  const tsfde_status sv = gmres_run(C, true, lam, info, t0);
  if (sv < 0) return sv;
  if (grads) {
    // B_n y for the forward solution, then the gradient formulas (C->x holds lam)
    TSFDE_CU(cudaMemcpyAsync(C->tmp, y, sizeof(double) * U, cudaMemcpyDefault, st));
    bapply<double>(C->sp64_all, C->tmp, C->By, S + 1, nullptr, st);
    adjoint_grads(C->x, C->By, C->g2, C->w, C->r, C->r + N, S, N, C->cs, C->cf, st);
    multidot(C->x + (long long)S * N, N, 1, N, C->r + N, C->dnrm, C->rw, st);
    C->launches += (C->d == 1 ? 1 : (C->d == 2 ? 3 : 5)) + 2;
    TSFDE_TRY(check_launch("tsfde_adjoint: gradients"));
    const double dot = read_scalar(C, C->dnrm);
    if (dJ_dalpha) *dJ_dalpha = -dot / pow(C->h, C->omega);
    if (dJ_dmu) TSFDE_CU(cudaMemcpyAsync(dJ_dmu, C->r, sizeof(double) * N, cudaMemcpyDefault, st));
    if (dJ_dgamma2) TSFDE_CU(cudaMemcpyAsync(dJ_dgamma2, C->w, sizeof(double) * S * N, cudaMemcpyDefault, st));
    TSFDE_CU(cudaStreamSynchronize(st));
  }
  if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return sv;
}

tsfde_status tsfde_direct_solve(tsfde_handle C, const double* f, const double* F, double* v) {
  if (!C || !v || (f == nullptr) == (F == nullptr)) return TSFDE_EINVAL;
  cudaStream_t st = C->st;
  const long long N = C->N;
  const int S = C->S;
  TSFDE_CU(cudaMemsetAsync(&C->sc[0].fails, 0, sizeof(int), st));
  TSFDE_CU(cudaMemsetAsync(&C->sc[1].fails, 0, sizeof(int), st));
  // the source on the device (host or device input), in C->w
  TSFDE_CU(cudaMemcpyAsync(C->w, f ? f : F, sizeof(double) * (f ? N : (long long)S * N), cudaMemcpyDefault, st));
  direct_rhs(C->g1, C->rho, C->bw, C->q, f ? C->w : nullptr, F ? C->w : nullptr, C->eta, C->tmp, S, N, st);
  C->launches += 1;
  TSFDE_TRY(check_launch("tsfde_direct_solve: right-hand side"));
  // the first S stages of the forward substitution solve the direct problem
  TSFDE_TRY(precond_apply(C, C->tmp, C->z));
  TSFDE_CU(cudaMemcpyAsync(v, C->z, sizeof(double) * (long long)S * N, cudaMemcpyDefault, st));
  int fails[2] = {0, 0};
  unsigned int barerr = 0;
  TSFDE_CU(cudaMemcpyAsync(&fails[0], &C->sc[0].fails, sizeof(int), cudaMemcpyDeviceToHost, st));
  TSFDE_CU(cudaMemcpyAsync(&fails[1], &C->sc[1].fails, sizeof(int), cudaMemcpyDeviceToHost, st));
  TSFDE_CU(cudaMemcpyAsync(&barerr, C->fsub_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  TSFDE_CU(cudaStreamSynchronize(st));
  if (C->opts.graphs) TSFDE_CU(cudaStreamSynchronize(C->gst));
  if (barerr) {
    set_error("persistent forward substitution: a grid barrier wait expired");
    return TSFDE_ETIMEOUT;
  }
  const int fl = (C->opts.precision == TSFDE_PREC_FP64) ? fails[0] : fails[1];
  return fl > 0 ? TSFDE_NOT_CONVERGED : TSFDE_OK;
}

tsfde_status tsfde_spectral_bidiag(tsfde_handle C, int which, int k, const double* u0, double* alpha, double* beta) {
  if (!C || !u0 || !alpha || !beta || k < 1 || (which != 0 && which != 1)) return TSFDE_EINVAL;
  cudaStream_t st = C->st;
  const long long U = C->U;
  TSFDE_TRY(alloc_gmres(C));
  DevBuf Ub, Vb;
  TSFDE_CU(cudaMalloc((void**)&Ub.p, sizeof(double) * (size_t)(k + 1) * U));
  TSFDE_CU(cudaMalloc((void**)&Vb.p, sizeof(double) * (size_t)(k + 1) * U));
  // beta_1 u_1 = u0; alpha_1 v_1 = M^T u_1
  TSFDE_CU(cudaMemcpyAsync(C->w, u0, sizeof(double) * U, cudaMemcpyDefault, st));
  norm2(C->w, U, C->dnrm, C->rw, st);
  if (!(read_scalar(C, C->dnrm) > 0.0)) return TSFDE_EINVAL;
  scale_by_invnorm(C->w, Ub.p, U, C->dnrm, st);
  TSFDE_TRY(spec_apply(C, which, true, Ub.p, C->w));
  norm2(C->w, U, C->dnrm, C->rw, st);
  double a = sqrt(read_scalar(C, C->dnrm));
  scale_by_invnorm(C->w, Vb.p, U, C->dnrm, st);
  for (int j = 1; j <= k; ++j) {
    alpha[j - 1] = a;
    // beta_{j+1} u_{j+1} = M v_j - alpha_j u_j
    TSFDE_TRY(spec_apply(C, which, false, Vb.p + (long long)(j - 1) * U, C->w));
    axpby(-a, Ub.p + (long long)(j - 1) * U, 1.0, C->w, U, st);
    reorth(C, Ub.p, j, C->w, nullptr);
    norm2(C->w, U, C->dnrm, C->rw, st);
    const double b = sqrt(read_scalar(C, C->dnrm));
    beta[j - 1] = b;
    if (j == k || !(b > 0.0)) {
      for (int i = j; i < k; ++i) alpha[i] = beta[i] = 0.0;
      break;
    }
    scale_by_invnorm(C->w, Ub.p + (long long)j * U, U, C->dnrm, st);
    // alpha_{j+1} v_{j+1} = M^T u_{j+1} - beta_{j+1} v_j
    TSFDE_TRY(spec_apply(C, which, true, Ub.p + (long long)j * U, C->w));
    axpby(-b, Vb.p + (long long)(j - 1) * U, 1.0, C->w, U, st);
    reorth(C, Vb.p, j, C->w, nullptr);
    norm2(C->w, U, C->dnrm, C->rw, st);
    a = sqrt(read_scalar(C, C->dnrm));
    if (!(a > 0.0)) {
      for (int i = j; i < k; ++i) alpha[i] = beta[i] = 0.0;
      break;
    }
    scale_by_invnorm(C->w, Vb.p + (long long)j * U, U, C->dnrm, st);
    TSFDE_TRY(check_launch("tsfde_spectral_bidiag"));
  }
  TSFDE_CU(cudaStreamSynchronize(st));
  return TSFDE_OK;
}

tsfde_status tsfde_spectral_arnoldi(tsfde_handle C, int which, int k, const double* v0, double* H, int* steps) {
  if (!C || !v0 || !H || k < 1 || (which != 0 && which != 1)) return TSFDE_EINVAL;
  cudaStream_t st = C->st;
  const long long U = C->U;
  const int ld = k + 1;
  TSFDE_TRY(alloc_gmres(C));
  DevBuf Vb, Hd;
  TSFDE_CU(cudaMalloc((void**)&Vb.p, sizeof(double) * (size_t)(k + 1) * U));
  TSFDE_CU(cudaMalloc((void**)&Hd.p, sizeof(double) * (size_t)ld * k));
  TSFDE_CU(cudaMemsetAsync(Hd.p, 0, sizeof(double) * (size_t)ld * k, st));
  for (int i = 0; i < ld * k; ++i) H[i] = 0.0;
  TSFDE_CU(cudaMemcpyAsync(C->w, v0, sizeof(double) * U, cudaMemcpyDefault, st));
  norm2(C->w, U, C->dnrm, C->rw, st);
  if (!(read_scalar(C, C->dnrm) > 0.0)) return TSFDE_EINVAL;
  scale_by_invnorm(C->w, Vb.p, U, C->dnrm, st);
  int done = 0;
  for (int j = 0; j < k; ++j) {
    TSFDE_TRY(spec_apply(C, which, false, Vb.p + (long long)j * U, C->w));
    norm2(C->w, U, C->dnrm, C->rw, st);
    const double wn = sqrt(read_scalar(C, C->dnrm));
    reorth(C, Vb.p, j + 1, C->w, Hd.p + (long long)j * ld);
    norm2(C->w, U, C->dnrm, C->rw, st);
    const double hn = sqrt(read_scalar(C, C->dnrm));
    TSFDE_CU(cudaMemcpyAsync(H + (long long)j * ld, Hd.p + (long long)j * ld, sizeof(double) * (j + 1),
                             cudaMemcpyDeviceToHost, st));
    TSFDE_CU(cudaStreamSynchronize(st));
    H[(long long)j * ld + j + 1] = hn;
    done = j + 1;
    // an invariant subspace: the new direction is rounding noise
    if (!(hn > 1e-12 * wn)) break;
    scale_by_invnorm(C->w, Vb.p + (long long)(j + 1) * U, U, C->dnrm, st);
    TSFDE_TRY(check_launch("tsfde_spectral_arnoldi"));
  }
  if (steps) *steps = done;
  return TSFDE_OK;
}

static tsfde_status batch_check(int count, const tsfde_handle* hs) {
  if (count < 1 || count > kMaxBatch || !hs) {
    set_error("batch: need 1 <= count <= " + std::to_string(kMaxBatch));
    return TSFDE_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return TSFDE_EINVAL;
    if (hs[i]->fsub_grid <= 0) {
      set_error("batch: the persistent kernel is unavailable (cooperative launch)");
      return TSFDE_EUNSUPPORTED;
    }
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) {
        set_error("batch: a handle appears twice");
        return TSFDE_EINVAL;
      }
  }
  return TSFDE_OK;
}

tsfde_status tsfde_precond_apply_batch(int count, const tsfde_handle* hs, const double* const* rs, double* const* ys) {
  TSFDE_TRY(batch_check(count, hs));
  if (!rs || !ys) return TSFDE_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!rs[i] || !ys[i] || rs[i] == ys[i]) return TSFDE_EINVAL;
  for (int i = 0; i < count; ++i) {
    TSFDE_CU(cudaMemsetAsync(&hs[i]->sc[0].fails, 0, sizeof(int), hs[i]->st));
    TSFDE_CU(cudaMemsetAsync(&hs[i]->sc[1].fails, 0, sizeof(int), hs[i]->st));
  }
  std::vector<int> tr(count, 0);
  TSFDE_TRY(fsub_batch_launch(hs, rs, ys, tr.data(), count));
  tsfde_status worst = TSFDE_OK;
  for (int i = 0; i < count; ++i) {
    tsfde_ctx* h = hs[i];
    int fails[2] = {0, 0};
    unsigned int barerr = 0;
    TSFDE_CU(cudaMemcpyAsync(&fails[0], &h->sc[0].fails, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    TSFDE_CU(cudaMemcpyAsync(&fails[1], &h->sc[1].fails, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    TSFDE_CU(cudaMemcpyAsync(&barerr, h->fsub_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->st));
    TSFDE_CU(cudaStreamSynchronize(h->st));
    if (barerr) {
      set_error("persistent forward substitution: a grid barrier wait expired");
      worst = TSFDE_ETIMEOUT;
    } else if (worst == TSFDE_OK && ((h->opts.precision == TSFDE_PREC_FP64) ? fails[0] : fails[1]) > 0) {
      worst = TSFDE_NOT_CONVERGED;
    }
  }
  return worst;
}

tsfde_status tsfde_gmres_solve_batch(int count, const tsfde_handle* hs, double* const* ys, tsfde_info* infos) {
  TSFDE_TRY(batch_check(count, hs));
  if (!ys) return TSFDE_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!ys[i]) return TSFDE_EINVAL;
  int dev = 0;
  TSFDE_CU(cudaGetDevice(&dev));
  BatchCoord coord;
  coord.active = count;
  coord.order.assign(hs, hs + count);
  for (int i = 0; i < count; ++i) hs[i]->coord = &coord;
  std::vector<tsfde_status> st(count, TSFDE_OK);
  std::vector<std::string> msg(count);
  auto run = [&](int i) {
    cudaSetDevice(dev);
    st[i] = tsfde_gmres_solve(hs[i], ys[i], infos ? &infos[i] : nullptr);
    if (st[i] < 0) msg[i] = tsfde_last_error();
    coord.leave();
  };
  std::vector<std::thread> th;
  for (int i = 1; i < count; ++i) th.emplace_back(run, i);
  run(0);
  for (auto& t : th) t.join();
  for (int i = 0; i < count; ++i) hs[i]->coord = nullptr;
  tsfde_status worst = TSFDE_OK;
  for (int i = 0; i < count; ++i) {
    if (st[i] < 0 && (worst >= 0 || st[i] < worst)) {
      worst = st[i];
      set_error("batch instance " + std::to_string(i) + ": " + msg[i]);
    } else if (worst == TSFDE_OK && st[i] > 0) {
      worst = st[i];
    }
  }
  return worst;
}

tsfde_status tsfde_profile(tsfde_handle h, int enable) {
  if (!h) return TSFDE_EINVAL;
  TSFDE_CU(cudaStreamSynchronize(h->st));
  TSFDE_CU(cudaStreamSynchronize(h->gst));
  prof_resolve(h);
  for (auto& P : h->prof) {
    P.count = 0;
    P.ms = 0.0;
  }
  h->orth_bytes = 0.0;
  h->prof_on = enable != 0;
  h->timeline_on = enable == 2;
  for (int i = 0; i < PH_COUNT; ++i) {
    h->phase_ms[i] = 0.0;
    h->phase_n[i] = 0;
  }
  if (h->timeline_on && !h->trace && h->fsub_grid > 0) {
    h->trace_cap = 1 << 20;
    TSFDE_TRY(dalloc(h, &h->trace, (size_t)2 * h->trace_cap));
    TSFDE_TRY(dalloc(h, &h->trace_len, 1));
  }
  return TSFDE_OK;
}

tsfde_status tsfde_profile_read(tsfde_handle h, tsfde_profile_stats* out) {
  if (!h || !out) return TSFDE_EINVAL;
  TSFDE_CU(cudaStreamSynchronize(h->st));
  TSFDE_CU(cudaStreamSynchronize(h->gst));
  prof_resolve(h);
  Scalars sc[2];
  TSFDE_CU(cudaMemcpy(sc, h->sc, sizeof(Scalars) * 2, cudaMemcpyDeviceToHost));
  out->precond_count = h->prof[0].count;
  out->precond_ms = h->prof[0].ms;
  out->matvec_count = h->prof[1].count;
  out->matvec_ms = h->prof[1].ms;
  out->orth_count = h->prof[2].count;
  out->orth_ms = h->prof[2].ms;
  out->orth_bytes = h->orth_bytes;
  out->fp64_block_residuals = (long long)sc[0].sweeps + (h->opts.precision == TSFDE_PREC_MIXED ? (long long)sc[1].sweeps : 0);
  out->pcg_iterations = (long long)sc[1].iters;
  out->guess_fallbacks = (long long)sc[0].fallbacks;
  out->batch_graph_builds = h->mix_graph_builds;
  out->batch_graph_replays = h->mix_graph_replays;
  snprintf(out->batch_graph_error, sizeof(out->batch_graph_error), "%s", h->mix_graph_error.c_str());
  // algorithmic FLOPs of one B_n apply of one field on the pruned embedding (complex FFT of
  // length L costs 5 L log2 L; the last axis runs two real rows per complex line)
  const double L = 2.0 * (h->np + 1), lg = log2(L);
  const double fft = 5.0 * L * lg;
  double lines_b = 0, lines_t = 0;
  if (h->d == 1) { lines_b = 1.0; lines_t = 1.0; }   // per field: fwd + inv folded into one line pair
  else if (h->d == 2) {
    lines_b = h->n / 2.0 * 2 + (L / 2 + 1) * 2;       // rows fwd + inv (pairs), columns fwd + inv
    lines_t = h->n / 2.0 * 2 + h->n;                  // DST rows fwd + inv (pairs), columns (pairs, two transforms)
  } else {
    const double n = h->n;
    lines_b = n * n / 2.0 * 2 + n * (L / 2 + 1) * 2 + L * (L / 2 + 1) * 2;
    lines_t = n * n / 2.0 * 2 + n * n + n * n / 2.0 * 2;
  }
  out->flops_bapply = (h->d == 1 ? 2.0 * fft / 2.0 : lines_b * fft);
  out->flops_tau = (h->d == 1 ? 2.0 * fft / 2.0 : lines_t * fft);
  out->flops_timesum = (double)h->N * h->S * (h->S + 1);
  out->bytes_matvec = 8.0 * (2.0 * h->U + 2.0 * h->S * h->N);
  for (int i = 0; i < PH_COUNT && i < 12; ++i) {
    out->phase_ms[i] = h->phase_ms[i];
    out->phase_count[i] = h->phase_n[i];
  }
  out->launches = h->launches;
  out->precond_apps_total = h->apps_total;
  out->graph_kernels = h->graph_kernels;
  return TSFDE_OK;
}

void tsfde_destroy(tsfde_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  free_all(h);
  delete h;
}

}  // extern "C"
