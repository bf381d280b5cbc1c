// Time direction of the all-at-once operator (FP64):
//   * matvec rows 1..S of Eq. 11: z^(s) = D_1^(s) sum_{m<=s} e_{s-m} y^(m) + (eta/h^omega) D_2^(s) (B y^(s))
//     - eta q^(s) f, and the last row z^(S+1) = y^(S) + (alpha/h^omega) D_2^(S) (B f)
//     (Sec. 5 "Implementation", steps 1(a)-(c) and 2(a)-(b); step 1(c) subtracts the f block).
//   * the history term of the forward substitution (Sec. 5.1 step 2(b)):
//     rhat = r^(s) - D_1^(s) sum_{m<s} e_{s-m} y^(m), returned symmetrised as rhat / gamma2^(s).
//   * the right-hand side z of Eq. 11.
//   * the transposed operator A^T (adjoint solves) and the gradients of a misfit.
// The lower-triangular Toeplitz time sum is computed directly: each thread owns one node and
// TS consecutive levels, streams y^(m) once for all of them and keeps the TS sums in registers
// (the transpose streams the levels above the tile the same way).
#include <algorithm>

#include "internal.h"
#include "kernels.h"

namespace tsfde {

constexpr int TS = 16;

// grid: x over nodes (256 per block), y over level blocks of TS, plus one extra y for the last row.
__global__ void __launch_bounds__(256)
k_matvec_time(const double* __restrict__ y, const double* __restrict__ By, const double* __restrict__ g1,
              const double* __restrict__ g2, const double* __restrict__ q, const double* __restrict__ e,
              double* __restrict__ z, int S, long long N, double cs, double cf, double eta) {
  extern __shared__ double e_s[];   // S + TS entries, zero beyond S
  for (int i = threadIdx.x; i < S + TS; i += blockDim.x) e_s[i] = (i < S) ? e[i] : 0.0;
  __syncthreads();
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int nblk = (S + TS - 1) / TS;
  if ((int)blockIdx.y == nblk) {
    // last block row: z^(S+1) = y^(S) + cf * gamma2^(S) * (B f)
    z[(long long)S * N + j] = y[(long long)(S - 1) * N + j] + cf * g2[(long long)(S - 1) * N + j] * By[(long long)S * N + j];
    return;
  }
  const int s0 = blockIdx.y * TS;
  double acc[TS];
#pragma unroll
  for (int t = 0; t < TS; ++t) acc[t] = 0.0;
  // levels m < s0 contribute to every s in the tile
  for (int m = 0; m < s0; ++m) {
    const double v = y[(long long)m * N + j];
#pragma unroll
    for (int t = 0; t < TS; ++t) acc[t] = fma(e_s[s0 + t - m], v, acc[t]);
  }
  // the triangular part m in [s0, s0 + TS)
#pragma unroll
  for (int dm = 0; dm < TS; ++dm) {
    const int m = s0 + dm;
    if (m >= S) break;
    const double v = y[(long long)m * N + j];
#pragma unroll
    for (int t = 0; t < TS; ++t)
      if (t >= dm) acc[t] = fma(e_s[t - dm], v, acc[t]);
  }
  const double f = y[(long long)S * N + j];
#pragma unroll
  for (int t = 0; t < TS; ++t) {
    const int s = s0 + t;
    if (s >= S) break;
    const long long o = (long long)s * N + j;
    z[o] = g1[o] * acc[t] + cs * g2[o] * By[o] - eta * q[s] * f;
  }
}

void matvec_time(const double* y, const double* By, const double* g1, const double* g2, const double* q,
                 const double* e, double* z, int S, long long N, double cs, double cf, double eta,
                 cudaStream_t st) {
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)((S + TS - 1) / TS + 1));
  const size_t smem = sizeof(double) * (S + TS);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_matvec_time, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_matvec_time<<<grid, 256, smem, st>>>(y, By, g1, g2, q, e, z, S, N, cs, cf, eta);
}

// ---- transpose of Eq. 11 -------------------------------------------------------------------
// A^T lam, lam = [lam^(1); ...; lam^(S); lam_f] (B_n symmetric, the D's diagonal):
//   (A^T lam)^(m) = sum_{s >= m} e_{s-m} D_1^(s) lam^(s) + (eta/h^omega) B_n D_2^(m) lam^(m) + [m = S] lam_f
//   (A^T lam)_f   = -eta sum_s q^(s) lam^(s) + (alpha/h^omega) B_n D_2^(S) lam_f
// u = D_2 lam (the last field with D_2^(S)) is formed first and B_n applied to all S + 1 fields;
// k_matvec_time_T then forms the upper-triangular time sum, the coupling and the f row.

__global__ void k_scale_gamma2(const double* __restrict__ lam, const double* __restrict__ g2,
                               double* __restrict__ u, int S, long long N) {
  const long long total = (long long)(S + 1) * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / N, j = i - s * N;
    u[i] = g2[(s < S ? s : S - 1) * N + j] * lam[i];
  }
}

void scale_gamma2(const double* lam, const double* g2, double* u, int S, long long N, cudaStream_t st) {
  const long long total = (long long)(S + 1) * N;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_scale_gamma2<<<blocks, 256, 0, st>>>(lam, g2, u, S, N);
}

// grid: x over nodes (256 per block), y over level blocks of TS, plus one extra y for the f row.
__global__ void __launch_bounds__(256)
k_matvec_time_T(const double* __restrict__ lam, const double* __restrict__ Bu, const double* __restrict__ g1,
                const double* __restrict__ q, const double* __restrict__ e, double* __restrict__ z, int S,
                long long N, double cs, double cf, double eta) {
  extern __shared__ double e_s[];   // S + TS entries, zero beyond S
  for (int i = threadIdx.x; i < S + TS; i += blockDim.x) e_s[i] = (i < S) ? e[i] : 0.0;
  __syncthreads();
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int nblk = (S + TS - 1) / TS;
  if ((int)blockIdx.y == nblk) {
    // f row: -eta sum_s q^(s) lam^(s) + cf B_n D_2^(S) lam_f
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int m = 0;
    for (; m + 3 < S; m += 4) {
      a0 = fma(q[m], lam[(long long)m * N + j], a0);
      a1 = fma(q[m + 1], lam[(long long)(m + 1) * N + j], a1);
      a2 = fma(q[m + 2], lam[(long long)(m + 2) * N + j], a2);
      a3 = fma(q[m + 3], lam[(long long)(m + 3) * N + j], a3);
    }
    for (; m < S; ++m) a0 = fma(q[m], lam[(long long)m * N + j], a0);
    z[(long long)S * N + j] = -eta * ((a0 + a1) + (a2 + a3)) + cf * Bu[(long long)S * N + j];
    return;
  }
  const int s0 = blockIdx.y * TS;
  double acc[TS];
#pragma unroll
  for (int t = 0; t < TS; ++t) acc[t] = 0.0;
  // levels m >= s0 + TS contribute to every s in the tile, with weight e_{m-s}
  for (int m = s0 + TS; m < S; ++m) {
    const long long o = (long long)m * N + j;
    const double v = g1[o] * lam[o];
#pragma unroll
    for (int t = 0; t < TS; ++t) acc[t] = fma(e_s[m - s0 - t], v, acc[t]);
  }
  // the triangular part m in [s0, s0 + TS): m >= s
#pragma unroll
  for (int dm = 0; dm < TS; ++dm) {
    const int m = s0 + dm;
    if (m >= S) break;
    const long long o = (long long)m * N + j;
    const double v = g1[o] * lam[o];
#pragma unroll
    for (int t = 0; t < TS; ++t)
      if (t <= dm) acc[t] = fma(e_s[dm - t], v, acc[t]);
  }
  const double lf = lam[(long long)S * N + j];
#pragma unroll
  for (int t = 0; t < TS; ++t) {
    const int s = s0 + t;
    if (s >= S) break;
    const long long o = (long long)s * N + j;
    z[o] = acc[t] + cs * Bu[o] + (s == S - 1 ? lf : 0.0);
  }
}

void matvec_time_T(const double* lam, const double* Bu, const double* g1, const double* q, const double* e,
                   double* z, int S, long long N, double cs, double cf, double eta, cudaStream_t st) {
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)((S + TS - 1) / TS + 1));
  const size_t smem = sizeof(double) * (S + TS);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_matvec_time_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_matvec_time_T<<<grid, 256, smem, st>>>(lam, Bu, g1, q, e, z, S, N, cs, cf, eta);
}

// Gradients of a misfit J from y (forward solution), lam (A^T lam = dJ/dy) and By = B_n y (all
// S + 1 fields):  dJ/dgamma2^(s) = -lam^(s) c_s (B_n v^(s)) - [s = S] lam_f c_f (B_n f),
// dJ/dmu = lam_f, and w = D_2^(S) (B_n f) for dJ/dalpha = -h^-omega lam_f . w.
__global__ void k_adjoint_grads(const double* __restrict__ lam, const double* __restrict__ By,
                                const double* __restrict__ g2, double* __restrict__ dg2, double* __restrict__ dmu,
                                double* __restrict__ w, int S, long long N, double cs, double cf) {
  const long long total = (long long)S * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    double v = -lam[i] * cs * By[i];
    if (i >= (long long)(S - 1) * N) {
      const long long j = i - (long long)(S - 1) * N;
      const long long f = (long long)S * N + j;
      v -= lam[f] * cf * By[f];
      dmu[j] = lam[f];
      w[j] = g2[i] * By[f];
    }
    dg2[i] = v;
  }
}

void adjoint_grads(const double* lam, const double* By, const double* g2, double* dg2, double* dmu, double* w,
                   int S, long long N, double cs, double cf, cudaStream_t st) {
  const long long total = (long long)S * N;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_adjoint_grads<<<blocks, 256, 0, st>>>(lam, By, g2, dg2, dmu, w, S, N, cs, cf);
}

// Right-hand side of the direct problem (Sec. 6.1): zhat^(s) = b_{s-1} D_1^(s) rho + eta q^(s) f
// (or eta F^(s) for a general source F [S][N]); the last block (f row of Eq. 11) is set to 0.
__global__ void k_direct_rhs(const double* __restrict__ g1, const double* __restrict__ rho,
                             const double* __restrict__ b, const double* __restrict__ q,
                             const double* __restrict__ f, const double* __restrict__ F, double eta,
                             double* __restrict__ out, int S, long long N) {
  const long long total = (long long)(S + 1) * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / N, j = i - s * N;
    if (s == S) {
      out[i] = 0.0;
    } else {
      const double src = F ? F[i] : q[s] * f[j];
      out[i] = b[s] * g1[i] * rho[j] + eta * src;
    }
  }
}

void direct_rhs(const double* g1, const double* rho, const double* b, const double* q, const double* f,
                const double* F, double eta, double* out, int S, long long N, cudaStream_t st) {
  const long long total = (long long)(S + 1) * N;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_direct_rhs<<<blocks, 256, 0, st>>>(g1, rho, b, q, f, F, eta, out, S, N);
}

// rhs_sym[j] = (r^(s)_j - gamma1^(s)_j sum_{m<s} e_{s-m} y^(m)_j) / gamma2^(s)_j, level s = sl + 1.
__global__ void __launch_bounds__(256)
k_history(const double* __restrict__ r, const double* __restrict__ y, const double* __restrict__ g1,
          const double* __restrict__ g2, const double* __restrict__ e, double* __restrict__ out, int sl,
          long long N) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int m = 0;
  for (; m + 3 < sl; m += 4) {
    a0 = fma(e[sl - m], y[(long long)m * N + j], a0);
    a1 = fma(e[sl - m - 1], y[(long long)(m + 1) * N + j], a1);
    a2 = fma(e[sl - m - 2], y[(long long)(m + 2) * N + j], a2);
    a3 = fma(e[sl - m - 3], y[(long long)(m + 3) * N + j], a3);
  }
  for (; m < sl; ++m) a0 = fma(e[sl - m], y[(long long)m * N + j], a0);
  const long long o = (long long)sl * N + j;
  out[j] = (r[o] - g1[o] * ((a0 + a1) + (a2 + a3))) / g2[o];
}

void history_rhs(const double* r, const double* y, const double* g1, const double* g2, const double* e,
                 double* out, int sl, long long N, cudaStream_t st) {
  k_history<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(r, y, g1, g2, e, out, sl, N);
}

// z = [b_{s-1} gamma1^(s) rho ; mu]
__global__ void k_rhs(const double* __restrict__ g1, const double* __restrict__ rho, const double* __restrict__ mu,
                      const double* __restrict__ b, double* __restrict__ z, int S, long long N) {
  const long long total = (long long)(S + 1) * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / N, j = i % N;
    z[i] = (s < S) ? b[s] * g1[i] * rho[j] : mu[j];
  }
}

void build_rhs(const double* g1, const double* rho, const double* mu, const double* b, double* z, int S,
               long long N, cudaStream_t st) {
  const long long total = (long long)(S + 1) * N;
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_rhs<<<blocks, 256, 0, st>>>(g1, rho, mu, b, z, S, N);
}

// dvec[s][j] = e_0 gamma1 / gamma2 (diagonal of the symmetrised block), in FP64 and FP32.
__global__ void k_block_diag(const double* __restrict__ g1, const double* __restrict__ g2, double e0,
                             double* __restrict__ d64, float* __restrict__ d32, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = e0 * g1[i] / g2[i];
    d64[i] = v;
    d32[i] = (float)v;
  }
}

// dbar[s] = mean_j d64[s][j]: one block per level, fixed-order reduction.
__global__ void k_level_mean(const double* __restrict__ d64, double* __restrict__ dbar64, float* __restrict__ dbar32,
                             long long N) {
  __shared__ double scratch[32];
  const double* row = d64 + (long long)blockIdx.x * N;
  double acc = 0.0;
  for (long long j = threadIdx.x; j < N; j += blockDim.x) acc += row[j];
  acc = block_sum(acc, scratch);
  if (threadIdx.x == 0) {
    dbar64[blockIdx.x] = acc / (double)N;
    dbar32[blockIdx.x] = (float)(acc / (double)N);
  }
}

void level_mean(const double* d64, double* dbar64, float* dbar32, int S, long long N, cudaStream_t st) {
  k_level_mean<<<S, 256, 0, st>>>(d64, dbar64, dbar32, N);
}

// *bad += the number of entries that are not finite and positive (an integer count: any order).
__global__ void k_count_nonpositive(const double* __restrict__ x, long long total, unsigned int* bad) {
  unsigned int c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (!(v > 0.0) || !isfinite(v)) ++c;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

void count_nonpositive(const double* x, long long total, unsigned int* bad, cudaStream_t st) {
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  if (blocks < 1) blocks = 1;
  k_count_nonpositive<<<blocks, 256, 0, st>>>(x, total, bad);
}

void block_diag(const double* g1, const double* g2, double e0, double* d64, float* d32, long long total,
                cudaStream_t st) {
  int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_block_diag<<<blocks, 256, 0, st>>>(g1, g2, e0, d64, d32, total);
}

}  // namespace tsfde
