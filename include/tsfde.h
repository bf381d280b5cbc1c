/*
 * tsfde.h -- C ABI of the GB300 (sm_103a) solver for the all-at-once system of
 * the quasi-boundary-value regularised time-space fractional inverse source
 * problem (Majumdar, Serra-Capizzano, Sormani, arXiv 2507.02809).
 *
 * Problem (Sec. 1, Eq. 1; regularised form Eq. 4): find u(x,t) and f(x) with
 *   gamma1 D_t^beta u + gamma2 (-Delta)^(omega/2) u = f(x) q(t)   in Omega x (0,T),
 *   u = 0 outside Omega, u(.,0) = rho, u(.,T) = mu_eps - alpha gamma2(.,T) (-Delta)^(omega/2) f.
 * Discretisation (Sec. 4): L1 formula in time (Eq. 5), fractional centred
 * differences in space (Eq. 6-9), giving the block system A y = z of Eq. 11
 * with y = [v^(1); ...; v^(S); f] and z = [b_{s-1} D_1^(s) rho; mu_eps].
 * The regularisation parameter the paper writes lambda is called alpha here.
 *
 * Conventions shared by every entry point
 *   - Omega = (0, length)^d, n interior points per direction (the paper's unique
 *     step size), h = length / (n + 1); d in {1, 2, 3}; N = n^d; U = (S + 1) N.
 *     Node order is lexicographic with the last index fastest (Sec. 2).
 *   - Level-major layout: a field over time levels is [S][N] doubles (level s = 1..S
 *     at offset (s-1) N); a full vector y, z or r is [S+1][N], the last block being f
 *     (for y) or the final-condition row (for z).
 *   - Vectors passed to tsfde_matvec / tsfde_precond_apply are DEVICE pointers, owned
 *     by the caller, 16-byte aligned.  tsfde_setup and tsfde_gmres_solve accept host
 *     or device memory; both are copied with cudaMemcpyAsync(cudaMemcpyDefault) on the
 *     handle's stream (unified addressing tells the direction).
 *   - The library owns all workspace (allocated in tsfde_setup, freed in
 *     tsfde_destroy); it never frees caller memory.  setup copies what it keeps.
 *   - Work is enqueued on the CUDA stream given to tsfde_setup (NULL = legacy default
 *     stream).  tsfde_gmres_solve synchronises that stream to fill its info.
 *   - No exceptions cross the ABI and there is no CPU fallback: without a usable GPU
 *     every call returns TSFDE_ECUDA.
 *   - Supported sizes: 3 <= n <= 2047 for d = 1, <= 1023 for d = 2, <= 255 for d = 3; S >= 1.
 *     Transforms have the power-of-two length L = 2 p, p the smallest power of two >= n + 1: B_n
 *     is embedded in a circulant of size L >= 2 n - 1, and the tau preconditioner of the inner CG
 *     works on the grid of p - 1 points (zero-padded when n + 1 is not a power of two; then the
 *     preconditioner runs in the persistent kernel only, and block_solver = 1 is refused;
 *     block_solver = 2 works on every grid).
 */
#ifndef TSFDE_H
#define TSFDE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsfde_ctx* tsfde_handle;

typedef enum {
  TSFDE_OK = 0,
  TSFDE_NOT_CONVERGED = 1,   /* result returned, but the tolerance was not reached */
  TSFDE_EINVAL = -1,         /* bad argument (null pointer, size out of range, ...) */
  TSFDE_ENOMEM = -2,         /* device allocation failed */
  TSFDE_ECUDA = -3,          /* a CUDA call failed; see tsfde_last_error() */
  TSFDE_EBREAKDOWN = -4,     /* NaN/Inf met in a reduction, or a zero pivot */
  TSFDE_EUNSUPPORTED = -5,   /* valid request outside what this build implements */
  TSFDE_ETIMEOUT = -6        /* a bounded device wait (grid barrier) expired; results invalid */
} tsfde_status;

typedef struct {
  int d;          /* spatial dimension, 1..3 */
  int n;          /* interior points per direction */
  double length;  /* side of the hypercube domain */
  int S;          /* number of time steps (Sec. 4: Delta t = T / S) */
  double T;       /* final time */
} tsfde_grid;

enum { TSFDE_PREC_FP64 = 0, TSFDE_PREC_MIXED = 1 };
enum { TSFDE_SIDE_LEFT = 0, TSFDE_SIDE_RIGHT = 1, TSFDE_SIDE_FLEXIBLE = 2 };
/* values of tsfde_opts.block_solver: P_{n,S} (Sec. 5.1), T_{n,S} and S_{n,S} (Remark 1) */
enum { TSFDE_BLOCK_SOLVE = 0, TSFDE_BLOCK_TAU = 1, TSFDE_BLOCK_STRANG = 2 };

typedef struct {
  int precision;     /* TSFDE_PREC_FP64: each diagonal-block solve of the forward substitution
                        is converged to inner_tol (FP32 tau-PCG corrections inside FP64
                        iterative refinement), so P^-1 is applied to FP64 accuracy;
                        TSFDE_PREC_MIXED: one FP32 tau-PCG solve per block, to inner_tol_mixed */
  int side;          /* TSFDE_SIDE_LEFT (the paper's choice, stopping test on ||P^-1 r||),
                        _RIGHT or _FLEXIBLE (stopping test on the true residual) */
  int restart;       /* GMRES restart length m, 1..64 */
  int max_iters;     /* maximum number of Arnoldi steps over all restart cycles */
  double tol;        /* relative residual target */
  double inner_tol;  /* FP64 mode: relative residual of each block solve (default 1e-11) */
  double inner_tol_mixed; /* mixed mode: relative residual of each FP32 block solve (default 1e-5) */
  int pcg_iters;     /* FP32 PCG iterations per refinement sweep (FP64 mode); doubled on grids with
                        n + 1 not a power of two, whose zero-padded tau preconditioner is weaker */
  int pcg_max;       /* cap on FP32 PCG iterations per block (mixed mode) */
  int refine_max;    /* FP64 mode: maximum refinement sweeps per block */
  int coeff_K;       /* d >= 2: trapezoid size for the coefficient table a_l; 0 = default */
  int graphs;        /* when persistent = 0: 1 captures the preconditioner application once into a
                        CUDA graph on an internal stream and replays it (ordered with the handle's
                        stream by events); 0 launches its kernels one by one.  In a batch of
                        instances of different transform lengths led by this handle (first in the
                        list), 1 also captures each round's launch sequence of the mixed-length
                        kernel into a CUDA graph, replayed while the batch stays the same */
  int persistent;    /* 1: the whole forward substitution runs as one persistent cooperative kernel
                        (one launch per application, bounded grid barriers); 0: separate kernels */
  int warm_start;    /* initial guess of each block solve: 0 zero (its first residual is then the
                        right-hand side, no operator application); 1 the previous level's solution;
                        k = 2..8 the polynomial of degree k - 1 through the last k levels, evaluated
                        at this one (k = 2 linear, 3 quadratic, ...; the p-th level processed uses
                        at most 1 + p / 4 levels, the solution being least smooth near t = 0;
                        persistent kernel; the
                        separate-kernel form treats k >= 2 as 1).  The guess changes the work of a
                        block solve, not the tolerance it meets */
  int fused_cg;      /* persistent kernel, d >= 2: 1 runs each inner CG step as four passes over
                        the field in 2-D (eight in 3-D) by carrying the row spectra of the search
                        direction and the row sine transforms of the residual from step to step;
                        0 recomputes them (six / ten passes).  Same iteration, different rounding. */
  double inner_tol_corr; /* FP64 mode: relative residual each FP32 CG correction aims at within a
                        refinement sweep (default 3e-6); with pcg_iters it sets how the work of a block
                        solve splits between FP32 CG steps and FP64 residual sweeps, not its result */
  int block_solver;  /* 0: the diagonal blocks of P are solved to inner_tol (P_{n,S} of Sec. 5.1);
                        1: every B_n in the diagonal blocks is replaced by tau(B_n) (T_{n,S} of
                        Remark 1), each block solved by one sine-transform solve, the variable
                        diagonal e_0 gamma1 / gamma2 by its level mean (exact T_{n,S} for constant
                        coefficients); cheaper applications, more GMRES steps.  Needs n + 1 a
                        power of two.
                        2: the same with the Strang circulant s(B_n) (S_{n,S} of Remark 1: per
                        level the central diagonals a_l, |l| <= n/2, wrapped around), each block
                        solved in the Fourier basis by DFTs of length n (Bluestein's chirp-z
                        transform on the length-L FFTs, so any n); the Remark expects more GMRES
                        steps than with 1.  Persistent kernel only. */
  long long spin_limit; /* persistent kernel: polls of one grid-barrier wait before the launch gives up
                        (every CTA leaves at its next barrier and the call returns TSFDE_ETIMEOUT with
                        invalid results; the handle stays usable); default 2^24, at least 1 */
  int warm_start_mixed; /* the same for the mixed mode (0..8): its levels are solved to inner_tol_mixed
                        only, whose errors the extrapolation amplifies by 2^k - 1, so a low order
                        is best there */
  int grid_ctas;     /* persistent kernel, d >= 2: CTAs of the instance's grid (its launch shape: more
                        CTAs spread a pass's lines wider, fewer make its grid barrier cheaper);
                        0 = one per SM; at most the co-resident limit (TSFDE_EINVAL above it) */
} tsfde_opts;

typedef struct {
  int iters;          /* Arnoldi steps in total */
  int restarts;       /* completed restart cycles */
  int converged;      /* 1 if the stopping test was met */
  double relres_est;  /* last residual estimate relative to the reference norm */
  double relres_true; /* ||z - A y|| / ||z|| recomputed at the end */
  double seconds;     /* wall time of the solve (host clock around the whole call) */
  int precond_failures; /* block solves that hit refine_max / pcg_max without converging */
  double* history;    /* optional host array for the residual estimates, or NULL */
  int history_cap;    /* capacity of history */
  int history_len;    /* entries written */
} tsfde_info;

/* Fill *o with the defaults: FP64, left, restart 30, max_iters 3000, tol 1e-10,
 * inner_tol 1e-11, inner_tol_mixed 1e-5, pcg_iters 6, pcg_max 20, refine_max 6,
 * coeff_K 0, graphs 1, persistent 1, warm_start 6, fused_cg 1, inner_tol_corr 3e-6,
 * block_solver 0, spin_limit 2^24, warm_start_mixed 3, grid_ctas 0. */
void tsfde_default_opts(tsfde_opts* o);

/* Create a solver for one instance of Eq. 10 / Eq. 11.
 *   grid            sizes (see the conventions above)
 *   beta in (0,1)   Caputo order; omega in (1,2) fractional Laplacian order
 *   alpha > 0       regularisation parameter (lambda in Eq. 4)
 *   gamma1, gamma2  [S][N] values gamma_i(x_j, t_s), s = 1..S; gamma2 > 0 (needed by the
 *                   symmetrised block solves); host or device
 *   q               [S] values q(t_s); host or device
 *   rho, mu         [N] initial state and noisy final data mu_eps; host or device
 *   opts            NULL for the defaults
 *   stream          cudaStream_t (as void*) on which all later work of the handle runs
 * Builds the tables of Sec. 4-5 on the GPU: b_m, e_m, eta, the coefficients a_l
 * (Eq. 9 / Lemma 1(b) for d = 1, K-point trapezoid rule of Eq. 8 for d >= 2), the
 * circulant-embedding symbol of B_n and the tau(B_n) eigenvalues; with block_solver = 2 also the
 * tables of S_{n,S} (Bluestein chirp of the length-n DFT and its FFT, the eigenvalues of the Strang
 * circulant s(B_n)).  On error *out is NULL and nothing is leaked. */
tsfde_status tsfde_setup(tsfde_handle* out, const tsfde_grid* grid, double beta, double omega,
                         double alpha, const double* gamma1, const double* gamma2, const double* q,
                         const double* rho, const double* mu, const tsfde_opts* opts, void* stream);

/* Replace the options of an existing handle (validated as in tsfde_setup).  coeff_K cannot change
 * after setup (TSFDE_EINVAL); block_solver = 1 on a grid with n + 1 not a power of two is
 * TSFDE_EUNSUPPORTED.  Switching to block_solver = 2 builds the S_{n,S} tables first, once per
 * handle; if that fails the handle keeps its previous options.  Synchronises. */
tsfde_status tsfde_set_opts(tsfde_handle h, const tsfde_opts* opts);

/* z = [b_0 D_1^(1) rho; ...; b_{S-1} D_1^(S) rho; mu_eps] (Eq. 11); z: device [U]. */
tsfde_status tsfde_rhs(tsfde_handle h, double* z);

/* z = A_{n,S} y (Eq. 11) without assembly, in the steps of Sec. 5 "Implementation":
 * time sums sum_m e_{s-m} y^(m), B_n y^(s) by circulant embedding + FFT, the D_1, D_2
 * scalings, the -eta q^(s) f coupling and the last row y^(S) + (alpha/h^omega) D_2^(S) B_n f.
 * y, z: device [U], distinct. FP64 throughout. */
tsfde_status tsfde_matvec(tsfde_handle h, const double* y, double* z);

/* y = P_{n,S}^-1 r by the forward substitution of Sec. 5.1 ("Implementation"):
 * for s = 1..S, rhat = r^(s) - D_1^(s) sum_{m<s} e_{s-m} y^(m), then solve
 * (e_0 D_1^(s) + (eta/h^omega) D_2^(s) B_n) y^(s) = rhat; finally solve
 * (alpha/h^omega) D_2^(S) B_n f = r^(S+1) - y^(S).  The paper's dense backslash solves are
 * replaced by tau-preconditioned CG on the D_2-symmetrised blocks (tau from Remark 1),
 * converged to opts.inner_tol (FP64 mode) or inner_tol_mixed (mixed mode).  With
 * opts.block_solver = 1 or 2 the same substitution applies T_{n,S} or S_{n,S} of Remark 1
 * instead: each block one sine-transform (tau) or Fourier (Strang) solve, no iteration.
 * r, y: device [U], distinct.  Synchronises the stream; returns TSFDE_NOT_CONVERGED if a
 * block solve stopped at its iteration cap (the result is still written) and TSFDE_ETIMEOUT
 * if a grid barrier of the persistent kernel expired. */
tsfde_status tsfde_precond_apply(tsfde_handle h, const double* r, double* y);

/* Solve A y = z (z from tsfde_rhs) with restarted GMRES preconditioned by P_{n,S}:
 * classical Gram-Schmidt with one reorthogonalisation, Givens rotations for the
 * least-squares update (Sec. 5 "Implementation", Sec. 6.1.2).  y: [U], host or device;
 * on entry the initial guess (the paper uses zero), on exit [v^(1..S); f].  Stops at tol, at
 * max_iters Arnoldi steps, or after three consecutive restart cycles that each reduce the residual
 * by less than 0.1 % (stagnation: the target lies below the attainable accuracy); the last two
 * return TSFDE_NOT_CONVERGED with the iterate written.  Synchronises the stream; fills *info if not
 * NULL. */
tsfde_status tsfde_gmres_solve(tsfde_handle h, double* y, tsfde_info* info);

/* As tsfde_gmres_solve for a right-hand side z given by the caller instead of Eq. 11's (z, y: [U],
 * host or device; y is the initial guess on entry). */
tsfde_status tsfde_solve(tsfde_handle h, const double* z, double* y, tsfde_info* info);

/* z = A_{n,S}^T lam, the transpose of the matrix of Eq. 11 (B_n is symmetric):
 * (A^T lam)^(m) = sum_{s>=m} e_{s-m} D_1^(s) lam^(s) + (eta/h^omega) B_n D_2^(m) lam^(m)
 *                 + [m = S] lam_f,
 * (A^T lam)_f   = -eta sum_s q^(s) lam^(s) + (alpha/h^omega) B_n D_2^(S) lam_f.
 * lam, z: device [U], distinct.  FP64.  Asynchronous on the handle's stream. */
tsfde_status tsfde_matvec_transpose(tsfde_handle h, const double* lam, double* z);

/* lam = P_{n,S}^-T r.  P^T is block upper triangular (P is A without its last block column,
 * Sec. 5.1), so this is a backward substitution, the f block first:
 * (alpha/h^omega) B_n D_2^(S) lam_f = r_f, then for s = S..1
 * (e_0 D_1^(s) + (eta/h^omega) B_n D_2^(s)) lam^(s) = r^(s) - sum_{m>s} e_{m-s} D_1^(m) lam^(m)
 * - [s = S] lam_f.  Each block is solved for w = D_2^(s) lam^(s) with the same symmetric
 * system and tau-preconditioned CG as the forward substitution, at the same tolerances;
 * it always runs as the persistent kernel (TSFDE_EUNSUPPORTED without cooperative launch).
 * r, lam: device [U], distinct.  Synchronises; statuses as tsfde_precond_apply. */
tsfde_status tsfde_precond_apply_transpose(tsfde_handle h, const double* r, double* lam);

/* Adjoint solve and gradients of a misfit J(y) of the solution y of Eq. 11.
 * Solves A^T lam = ybar (ybar = dJ/dy) by restarted GMRES preconditioned with P^T (the same
 * options as tsfde_gmres_solve: side, restart, tol, precision), from lam = 0, and then, with
 * y the forward solution, forms
 *   dJ/dalpha        = -lam_f . (h^-omega D_2^(S) B_n f)                  (host scalar)
 *   dJ/dmu           =  lam_f                                             [N]
 *   dJ/dgamma2^(s)_j = -lam^(s)_j (eta/h^omega) (B_n v^(s))_j
 *                      - [s = S] lam_{f,j} (alpha/h^omega) (B_n f)_j      [S][N]
 * (alpha and D_2^(S) enter the last block row of Eq. 11, D_2^(s) the diagonal blocks, mu the
 * last block of z; for J = 1/2 ||f - f_true||^2, ybar = [0; f - f_true]).  Only the forward
 * solution y is needed, not the forward Krylov basis: the adjoint GMRES reuses the handle's
 * workspace of restart + 1 vectors.
 * y, ybar: [U]; lam: [U] or NULL; dJ_dmu: [N] or NULL; dJ_dgamma2: [S][N] or NULL;
 * dJ_dalpha: host double or NULL.  Arrays may be host or device memory (cudaMemcpyDefault);
 * y may be NULL when no gradient is requested.  Synchronises; fills *info (the adjoint
 * solve's iterations and residuals) if not NULL.  Returns TSFDE_NOT_CONVERGED (results
 * written) if the adjoint GMRES stopped at max_iters. */
tsfde_status tsfde_adjoint(tsfde_handle h, const double* y, const double* ybar, double* lam, double* dJ_dalpha,
                           double* dJ_dmu, double* dJ_dgamma2, tsfde_info* info);

/* The direct problem of Sec. 6.1: v = [v^(1); ...; v^(S)] with Ahat v = zhat, Ahat the leading
 * S x S block part of P_{n,S} and zhat^(s) = b_{s-1} D_1^(s) rho + eta q^(s) f (the source known).
 * Solved by the first S stages of the forward substitution, with the handle's options (block
 * solver, precision, tolerances); v^(S) is the final state mu = u(., T).  Exactly one of f [N] (the
 * separable source q(t) f(x)) or F [S][N] (a general source F(x_j, t_s), replacing q^(s) f) is
 * given; f, F, v may be host or device memory.  Synchronises; statuses as tsfde_precond_apply. */
tsfde_status tsfde_direct_solve(tsfde_handle h, const double* f, const double* F, double* v);

/* Spectral diagnostics of M = A_{n,S} (which = 0) or M = P_{n,S}^-1 A_{n,S} (which = 1), as in the
 * spectral analyses of Sec. 6.1.1 and 6.2.1 (condition numbers, eigenvalue clustering), at sizes
 * where the matrices cannot be assembled.
 *
 * tsfde_spectral_bidiag: k steps of Golub-Kahan bidiagonalisation started from u0 (host or device
 * [U]), using M and M^T (A^T, P^-T from the transposed calls), with full reorthogonalisation of
 * both bases (classical Gram-Schmidt, two passes).  Returns the lower bidiagonal B_k
 * ((k+1) x k): alpha[i] = B[i][i], beta[i] = B[i+1][i], i < k (host arrays); its singular values
 * approximate those of M, the largest first (cond_2(M) ~ sigma_max(B_k) / sigma_min(B_k) once
 * sigma_min has converged).  A zero alpha or beta (invariant subspace) ends the process; the
 * remaining entries are 0.
 *
 * tsfde_spectral_arnoldi: up to k Arnoldi steps on M from v0, full reorthogonalisation; H (host,
 * (k+1) x k, column-major, leading dimension k+1) receives the Hessenberg matrix, *steps the number
 * of steps done (fewer than k when the Krylov space became invariant: for M = P^-1 A, whose
 * difference from I has rank at most N (Sec. 5.1), after at most N + 1 steps).  The eigenvalues of
 * the leading steps x steps block are the Ritz values.
 *
 * Both keep (k+1) vectors of U doubles per basis on the device (allocated per call) and
 * synchronise. */
tsfde_status tsfde_spectral_bidiag(tsfde_handle h, int which, int k, const double* u0, double* alpha, double* beta);
tsfde_status tsfde_spectral_arnoldi(tsfde_handle h, int which, int k, const double* v0, double* H, int* steps);

/* Batched forms: several instances (handles) with the same d and the same transform length (n + 1
 * rounded up to a power of two, so n may differ) share each launch of the persistent kernel.  The cooperative grid is split into
 * one sub-grid per instance (its own barrier counter, partial sums and counters), so the instances
 * run independently inside the launch; their passes fill SMs that one instance leaves idle.
 * Instances may differ in S, beta, omega, alpha, gamma1, gamma2, q, rho, mu and options.
 * count: 1..64; the handles must be distinct.  TSFDE_EINVAL if d or the transform length differ or
 * the instances do not fit one co-resident launch; TSFDE_EUNSUPPORTED without cooperative launch. */

/* y_i = P_i^-1 r_i for every instance in one launch (on the first handle's stream, ordered with
 * the others by events).  rs[i], ys[i]: device [U_i], distinct.  Synchronises every handle's
 * stream; returns the worst status over the instances (statuses as tsfde_precond_apply). */
tsfde_status tsfde_precond_apply_batch(int count, const tsfde_handle* hs, const double* const* rs,
                                       double* const* ys);

/* tsfde_gmres_solve for every instance, in lockstep: each solve runs on its own host thread with
 * its handle's options and stream, and every preconditioner application of the solves still
 * running is gathered into one batched launch.  ys[i]: [U_i], host or device (initial guess in,
 * solution out); infos: array of count (or NULL).  Returns the worst status over the instances. */
tsfde_status tsfde_gmres_solve_batch(int count, const tsfde_handle* hs, double* const* ys, tsfde_info* infos);

/* Counters of the event profiler (see tsfde_profile). */
typedef struct {
  long long precond_count;       /* preconditioner applications timed */
  double precond_ms;             /* their summed duration (CUDA events on the stream they ran on) */
  long long matvec_count;        /* matvecs timed */
  double matvec_ms;
  long long fp64_block_residuals;/* FP64 block residuals B_n x evaluated since setup (all applications) */
  long long pcg_iterations;      /* FP32 PCG iterations executed since setup */
  double flops_bapply;           /* algorithmic FLOPs of one B_n apply of one field (5 L log2 L per
                                    complex line of length L, pruned embedding) */
  double flops_tau;              /* same for one tau solve of one field */
  double flops_timesum;          /* FLOPs of the time sums of one matvec: N S (S + 1) */
  double bytes_matvec;           /* algorithmic HBM bytes of one matvec: 8 (2 U + 2 S N) */
  long long launches;            /* kernels launched by the handle since setup (graph replays count
                                    their kernel nodes) */
  long long graph_kernels;       /* kernel nodes in the captured preconditioner graph */
  long long precond_apps_total;  /* preconditioner applications since set-up (the work counters above
                                    count over the same span) */
  /* timeline of the persistent forward substitution (profiling on): time and count of the
   * passes closed by its grid barriers, by kind: 0 block right-hand side, 1-3 FP64 B_n apply
   * (rows forward, columns, rows inverse + residual), 4-6 tau solve (first rows, columns, last
   * rows), 7-9 FP32 B_n apply, 10 FP32 -> FP64 copy; 11 unused */
  double phase_ms[12];
  long long phase_count[12];
  long long orth_count;          /* GMRES Arnoldi orthogonalisations timed (classical Gram-Schmidt with one
                                    reorthogonalisation: two dot-product and two update launches each) */
  double orth_ms;                /* their summed duration (CUDA events on the handle's stream) */
  double orth_bytes;             /* their algorithmic HBM bytes, 16 U (2k + 3) for k basis vectors */
  long long batch_graph_builds;  /* batches of different transform lengths led by this handle (first in
                                    the list): launch sequences captured into a CUDA graph, and */
  long long batch_graph_replays; /* rounds launched by replaying that graph (0 when graphs = 0 or capture
                                    is unavailable: then each round is launched directly) */
  char batch_graph_error[96];    /* why the capture was unavailable ("" when it worked or was not tried) */
  long long guess_fallbacks;     /* FP64-mode block solves since set-up whose extrapolated initial guess
                                    left a larger first residual than the previous level or zero, and
                                    started from that instead */
} tsfde_profile_stats;

/* Turn the event profiler on (1), on with the timeline (2), or off (0), and reset its
 * counters.  When on, every preconditioner application, matvec and Arnoldi orthogonalisation of
 * the GMRES solve is bracketed by two CUDA events on the stream it runs on (the internal graph stream for the preconditioner).  With
 * the timeline, the persistent forward substitution also records a timestamp at each grid
 * barrier, read back after each application (which then synchronises); the first call with
 * enable = 2 allocates the 16 MB timeline buffer.  Synchronises. */
tsfde_status tsfde_profile(tsfde_handle h, int enable);

/* Read the profiler counters (synchronises the handle's streams). */
tsfde_status tsfde_profile_read(tsfde_handle h, tsfde_profile_stats* out);

/* z = A_{n,S} y for a one-dimensional instance (d = 1), without allocating any device memory.
 * The paper has no counterpart: it is an addition for callers that cannot allocate device
 * memory (a process whose device memory is owned by a pool or arena, an application that must
 * not trigger cudaMalloc and its implicit synchronisation while other work runs, a plug-in
 * whose host forbids allocation after start-up); such callers cannot use tsfde_setup.
 *   n, S, length, T, beta, omega, alpha   as in tsfde_setup (grid with d = 1)
 *   gamma1, gamma2 [S][n], q [S], y [(S+1) n], z [(S+1) n]: DEVICE pointers, caller-owned;
 *   y and z distinct.  Work is enqueued on `stream` (cudaStream_t as void*, NULL = legacy).
 * The operator, the layout and the FP64 arithmetic are those of tsfde_matvec.  All tables and
 * the work buffer live in one fixed __device__ array of 16.9 MB that every GPU loading the
 * library holds until exit; sizes beyond it are rejected with TSFDE_EUNSUPPORTED: n + 1 must
 * be a power of two with 4 <= n + 1 <= 2048, S <= 4096 and (S + 1) n <= 2^21.  The first call
 * on a device looks the array's address up once (cudaGetSymbolAddress); with CUDA's lazy module
 * loading (the default) that first call is also when the library's device code is loaded and
 * the array is reserved on that device, which can synchronise.  Make the first call once during
 * initialisation, before any stream capture and outside any window in which the caller may not
 * allocate.  The address is kept per device ordinal for the life of the process, for the
 * device's primary context: after cudaDeviceReset, or from a non-primary context, it is not
 * valid, and such callers must not use this entry point.
 * Calls share the array: calls that overlap on the GPU (other streams,
 * other host threads on the same device) race and must be serialised by the caller.  Every
 * call rebuilds the tables it reads, so no state carries over between calls.  Calls no
 * cudaMalloc, cudaFree or allocating library routine. */
tsfde_status tsfde_matvec_1d_noalloc(int n, int S, double length, double T, double beta, double omega,
                                     double alpha, const double* gamma1, const double* gamma2,
                                     const double* q, const double* y, double* z, void* stream);

/* Bytes of device memory owned by the handle. */
size_t tsfde_device_bytes(tsfde_handle h);

/* Release the handle and its device memory (NULL is ignored).  Synchronises the stream. */
void tsfde_destroy(tsfde_handle h);

/* Static description of a status code. */
const char* tsfde_status_string(tsfde_status s);

/* Text of the last CUDA or validation error seen by this thread ("" if none). */
const char* tsfde_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TSFDE_H */
