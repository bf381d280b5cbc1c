// Host launchers of the time-direction and Krylov kernels (internal).
#pragma once

#include <cuda_runtime.h>

namespace tsfde {

// ---- time direction (timesum.cu) -------------------------------------------------
void matvec_time(const double* y, const double* By, const double* g1, const double* g2, const double* q,
                 const double* e, double* z, int S, long long N, double cs, double cf, double eta,
                 cudaStream_t st);
void history_rhs(const double* r, const double* y, const double* g1, const double* g2, const double* e,
                 double* out, int sl, long long N, cudaStream_t st);
void build_rhs(const double* g1, const double* rho, const double* mu, const double* b, double* z, int S,
               long long N, cudaStream_t st);
// direct problem: out = [b_{s-1} gamma1^(s) rho + eta (q^(s) f or F^(s)); 0]
void direct_rhs(const double* g1, const double* rho, const double* b, const double* q, const double* f,
                const double* F, double eta, double* out, int S, long long N, cudaStream_t st);
void block_diag(const double* g1, const double* g2, double e0, double* d64, float* d32, long long total,
                cudaStream_t st);
void level_mean(const double* d64, double* dbar64, float* dbar32, int S, long long N, cudaStream_t st);
// *bad += number of entries of x[total] that are not finite and positive (*bad zeroed by the caller)
void count_nonpositive(const double* x, long long total, unsigned int* bad, cudaStream_t st);
// transpose of the operator: u = D_2 lam (S + 1 fields), then z = A^T lam from lam and Bu = B_n u
void scale_gamma2(const double* lam, const double* g2, double* u, int S, long long N, cudaStream_t st);
void matvec_time_T(const double* lam, const double* Bu, const double* g1, const double* q, const double* e,
                   double* z, int S, long long N, double cs, double cf, double eta, cudaStream_t st);
// misfit gradients: dg2 [S][N], dmu [N], w = D_2^(S) B_n f [N] (for dJ/dalpha = -h^-omega lam_f . w)
void adjoint_grads(const double* lam, const double* By, const double* g2, double* dg2, double* dmu, double* w,
                   int S, long long N, double cs, double cf, cudaStream_t st);

// ---- reductions / PCG / GMRES (krylov.cu) -----------------------------------------
// Device scalar block used by the iterative kernels (all FP64, one per solver).
struct Scalars {
  double rho;      // PCG r.z
  double alpha;    // PCG step
  double beta;     // PCG direction update
  double bnorm2;   // ||b||^2 of the current block solve
  double rnorm2;   // ||r||^2 of the current block solve
  double tol2;     // squared relative tolerance of the current block solve
  int done;        // current block solve converged (later kernels of the solve return at once)
  int breakdown;   // NaN / Inf or non-positive curvature met
  int fails;       // block solves that stopped at their iteration cap
  int fallbacks;   // levels whose extrapolated guess was replaced by a better lower-order one
  unsigned long long sweeps;  // FP64 residual evaluations (B_n applies in FP64) executed
  unsigned long long iters;   // PCG iterations executed
};

// Workspace for deterministic grid reductions: per-block partials + a ticket counter.
struct RedWork {
  double* part;           // >= kMaxRedBlocks * kMaxRedVals doubles
  unsigned int* ticket;   // one counter (zero between uses)
};
constexpr int kMaxRedBlocks = 1024;
constexpr int kMaxRedVals = 64;

template <typename R>
struct PcgVecs {
  R *x, *r, *z, *p, *q, *Bp;
};

// PCG (K = diag(dvec) + c B, M = dbar I + c tau(B)) kernels; all skip when sc->done.
// rho = r.z, p = z, and x = 0 when x != nullptr
template <typename R>
void pcg_rz_first(const R* r, const R* z, R* p, R* x, long long N, Scalars* sc, RedWork rw, cudaStream_t st);
template <typename R>
void pcg_q_alpha(const R* p, const R* Bp, const R* dvec, R c, R* q, long long N, Scalars* sc, RedWork rw,
                 cudaStream_t st);
template <typename R>
void pcg_update(R* x, R* r, const R* p, const R* q, long long N, Scalars* sc, RedWork rw, cudaStream_t st);
template <typename R>
void pcg_rz_beta(const R* r, const R* z, long long N, Scalars* sc, RedWork rw, cudaStream_t st);
template <typename R>
void pcg_p(const R* z, R* p, long long N, Scalars* sc, cudaStream_t st);
template <typename R>
void pcg_residual(const R* b, const R* x, const R* Bx, const R* dvec, R c, R* r, long long N, Scalars* sc,
                  RedWork rw, cudaStream_t st);

// FP64 refinement around an FP32 correction solve: r32 = (float)(b - (dvec x + c Bx)); outer done
// test on ||r|| <= tol ||b||; resets the inner (FP32 PCG) scalars for the correction solve.
void refine_residual_ex(const double* b, const double* x, const double* Bx, const double* dvec, double c,
                        float* r32, long long N, Scalars* outer, Scalars* inner, RedWork rw, bool first,
                        double inner_tol, cudaStream_t st);
void refine_update(double* x, const float* dx, long long N, Scalars* sc, cudaStream_t st);
void scalars_reset_solve(Scalars* sc, double tol, cudaStream_t st);
void scalars_count_fail(Scalars* sc, cudaStream_t st);

// f block: out = (r_f - y^(S)) / (cf * gamma2^(S))
void fblock_rhs(const double* rf, const double* yS, const double* g2S, double cf, double* out, long long N,
                cudaStream_t st);

// ---- GMRES (FP64) -----------------------------------------------------------------
// h[i] = V_i . w, i < k (V_i = V + i ld, rows of length U; k <= 64).  Rows are read as double2
// when ld is even and V, w are 16-byte aligned, element by element otherwise.
void multidot(const double* V, long long ld, int k, long long U, const double* w, double* h, RedWork rw,
              cudaStream_t st);
// w -= sum_{i<k} h[i] V_i  (sign = -1) or w += ... (sign = +1); same layout and vector rule
void multiaxpy(const double* V, long long ld, int k, long long U, const double* h, double sign, double* w,
               cudaStream_t st);
// out = ||w||^2
void norm2(const double* w, long long U, double* out, RedWork rw, cudaStream_t st);
// y = x / sqrt(*nrm2) (or 0 when *nrm2 == 0)
void scale_by_invnorm(const double* x, double* y, long long U, const double* nrm2, cudaStream_t st);
// y = a x + b y
void axpby(double a, const double* x, double b, double* y, long long U, cudaStream_t st);
// Givens update of Hessenberg column j; see krylov.cu
void givens_step(double* Hcol, double* cs, double* sn, double* g, int j, const double* hnew2, double* est,
                 cudaStream_t st);
// back substitution with the m x m upper triangle stored column-major with leading dim ld
void tri_solve(const double* Hmat, int ld, const double* g, int k, double* yk, cudaStream_t st);
// g[0] = sqrt(*nrm2), g[1..len-1] = 0
void init_g(double* g, int len, const double* nrm2, cudaStream_t st);
// Hcol[0..k-1] = h1 + h2 (CGS2)
void add_vec(const double* a, const double* b, double* out, int k, cudaStream_t st);

}  // namespace tsfde
