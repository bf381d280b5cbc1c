// Krylov kernels: the inner preconditioned CG of the diagonal-block solves (FP64 or FP32),
// the FP64 refinement around an FP32 correction solve, and the GMRES building blocks
// (batched dot products and updates for classical Gram-Schmidt with one
// reorthogonalisation, Givens rotations, back substitution).
//
// Reductions are deterministic: every block reduces its values with a fixed tree and writes
// one partial per value; the last block to finish (ticket counter) adds the partials in block
// order and updates the scalars.  Kernels of a block solve return at once when its `done`
// flag is set, so a solve that has converged costs only empty launches.
#include <math.h>

#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "kernels.h"

namespace tsfde {

namespace {

constexpr int kThreads = 256;

inline int red_blocks(long long N) {
  long long b = (N + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min<long long>(b, 2 * 152));
}

// Grid reduction of NV per-thread values; returns true in the last block, with the totals.
template <int NV>
__device__ bool grid_reduce(const double (&v)[NV], RedWork rw, double (&tot)[NV]) {
  __shared__ double scratch[32];
  __shared__ int am_last;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = block_sum(v[k], scratch);
    if (threadIdx.x == 0) rw.part[k * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(rw.ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(&rw.part[k * gridDim.x + i]);
    tot[k] = block_sum(acc, scratch);
  }
  if (threadIdx.x == 0) *rw.ticket = 0u;
  return true;
}

TSFDE_D bool finite(double v) { return isfinite(v); }

}  // namespace

// ------------------------------------------------------------------------------------
// PCG for (diag(dvec) + c B) x = b with preconditioner (dbar I + c tau(B))^-1
// ------------------------------------------------------------------------------------

// r = b - (dvec x + c Bx); reduce ||b||^2 and ||r||^2; done when ||r|| <= tol ||b||.
template <typename R>
__global__ void k_pcg_residual(const R* __restrict__ b, const R* __restrict__ x, const R* __restrict__ Bx,
                               const R* __restrict__ dvec, R c, R* __restrict__ r, long long N, Scalars* sc,
                               RedWork rw) {
  if (sc->done) return;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    R bi = b[i];
    R ri = bi - (dvec[i] * x[i] + c * Bx[i]);
    r[i] = ri;
    v[0] += (double)bi * bi;
    v[1] += (double)ri * ri;
  }
  double tot[2];
  if (grid_reduce<2>(v, rw, tot) && threadIdx.x == 0) {
    sc->bnorm2 = tot[0];
    sc->rnorm2 = tot[1];
    if (!finite(tot[0]) || !finite(tot[1])) { sc->breakdown = 1; sc->done = 1; }
    else if (tot[1] <= sc->tol2 * tot[0]) sc->done = 1;
  }
}

// rho = r.z ; p = z ; x = 0 (if given)
template <typename R>
__global__ void k_pcg_rz_first(const R* __restrict__ r, const R* __restrict__ z, R* __restrict__ p, R* __restrict__ x,
                               long long N, Scalars* sc, RedWork rw) {
  if (sc->done) return;
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    R zi = z[i];
    p[i] = zi;
    if (x) x[i] = R(0);
    v[0] += (double)r[i] * zi;
  }
  double tot[1];
  if (grid_reduce<1>(v, rw, tot) && threadIdx.x == 0) {
    sc->rho = tot[0];
    if (!finite(tot[0])) { sc->breakdown = 1; sc->done = 1; }
  }
}

// q = dvec p + c Bp ; alpha = rho / (p.q)
template <typename R>
__global__ void k_pcg_q_alpha(const R* __restrict__ p, const R* __restrict__ Bp, const R* __restrict__ dvec, R c,
                              R* __restrict__ q, long long N, Scalars* sc, RedWork rw) {
  if (sc->done) return;
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    R pi = p[i];
    R qi = dvec[i] * pi + c * Bp[i];
    q[i] = qi;
    v[0] += (double)pi * qi;
  }
  double tot[1];
  if (grid_reduce<1>(v, rw, tot) && threadIdx.x == 0) {
    if (!(tot[0] > 0.0) || !finite(tot[0])) {
      // p.q <= 0 happens only at an exact solution (p = 0) or from rounding garbage: stop
      sc->alpha = 0.0;
      if (!finite(tot[0])) sc->breakdown = 1;
      sc->done = 1;
    } else {
      sc->alpha = sc->rho / tot[0];
    }
  }
}

// x += alpha p ; r -= alpha q ; done when ||r|| <= tol ||b||
template <typename R>
__global__ void k_pcg_update(R* __restrict__ x, R* __restrict__ r, const R* __restrict__ p, const R* __restrict__ q,
                             long long N, Scalars* sc, RedWork rw) {
  if (sc->done) return;
  const R a = (R)sc->alpha;
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    R ri = r[i] - a * q[i];
    r[i] = ri;
    v[0] += (double)ri * ri;
  }
  double tot[1];
  if (grid_reduce<1>(v, rw, tot) && threadIdx.x == 0) {
    sc->rnorm2 = tot[0];
    if (!finite(tot[0])) { sc->breakdown = 1; sc->done = 1; }
    else if (tot[0] <= sc->tol2 * sc->bnorm2) sc->done = 1;
  }
}

// beta = (r.z) / rho ; rho = r.z
template <typename R>
__global__ void k_pcg_rz_beta(const R* __restrict__ r, const R* __restrict__ z, long long N, Scalars* sc, RedWork rw) {
  if (sc->done) return;
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    v[0] += (double)r[i] * z[i];
  double tot[1];
  if (grid_reduce<1>(v, rw, tot) && threadIdx.x == 0) {
    if (!finite(tot[0]) || sc->rho == 0.0) { sc->breakdown = !finite(tot[0]); sc->done = 1; }
    else {
      sc->beta = tot[0] / sc->rho;
      sc->rho = tot[0];
    }
  }
}

// p = z + beta p
template <typename R>
__global__ void k_pcg_p(const R* __restrict__ z, R* __restrict__ p, long long N, const Scalars* sc) {
  if (sc->done) return;
  const R bt = (R)sc->beta;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + bt * p[i];
}

template <typename R>
void pcg_residual(const R* b, const R* x, const R* Bx, const R* dvec, R c, R* r, long long N, Scalars* sc, RedWork rw,
                  cudaStream_t st) {
  k_pcg_residual<R><<<red_blocks(N), kThreads, 0, st>>>(b, x, Bx, dvec, c, r, N, sc, rw);
}
template <typename R>
void pcg_rz_first(const R* r, const R* z, R* p, R* x, long long N, Scalars* sc, RedWork rw, cudaStream_t st) {
  k_pcg_rz_first<R><<<red_blocks(N), kThreads, 0, st>>>(r, z, p, x, N, sc, rw);
}
template <typename R>
void pcg_q_alpha(const R* p, const R* Bp, const R* dvec, R c, R* q, long long N, Scalars* sc, RedWork rw,
                 cudaStream_t st) {
  k_pcg_q_alpha<R><<<red_blocks(N), kThreads, 0, st>>>(p, Bp, dvec, c, q, N, sc, rw);
}
template <typename R>
void pcg_update(R* x, R* r, const R* p, const R* q, long long N, Scalars* sc, RedWork rw, cudaStream_t st) {
  k_pcg_update<R><<<red_blocks(N), kThreads, 0, st>>>(x, r, p, q, N, sc, rw);
}
template <typename R>
void pcg_rz_beta(const R* r, const R* z, long long N, Scalars* sc, RedWork rw, cudaStream_t st) {
  k_pcg_rz_beta<R><<<red_blocks(N), kThreads, 0, st>>>(r, z, N, sc, rw);
}
template <typename R>
void pcg_p(const R* z, R* p, long long N, Scalars* sc, cudaStream_t st) {
  k_pcg_p<R><<<red_blocks(N), kThreads, 0, st>>>(z, p, N, sc);
}

#define TSFDE_INST_PCG(R)                                                                                        \
  template void pcg_residual<R>(const R*, const R*, const R*, const R*, R, R*, long long, Scalars*, RedWork,    \
                                cudaStream_t);                                                                   \
  template void pcg_rz_first<R>(const R*, const R*, R*, R*, long long, Scalars*, RedWork, cudaStream_t);       \
  template void pcg_q_alpha<R>(const R*, const R*, const R*, R, R*, long long, Scalars*, RedWork, cudaStream_t); \
  template void pcg_update<R>(R*, R*, const R*, const R*, long long, Scalars*, RedWork, cudaStream_t);          \
  template void pcg_rz_beta<R>(const R*, const R*, long long, Scalars*, RedWork, cudaStream_t);                 \
  template void pcg_p<R>(const R*, R*, long long, Scalars*, cudaStream_t);
TSFDE_INST_PCG(double)
TSFDE_INST_PCG(float)

// ------------------------------------------------------------------------------------
// FP64 refinement around an FP32 correction solve
// ------------------------------------------------------------------------------------

// r = b - (dvec x + c Bx) in FP64, r32 = (float) r; outer scalars: ||b||^2 (first sweep) and
// ||r||^2, done test; the inner (FP32 PCG) scalars are reset for the next correction solve.
__global__ void k_refine_residual(const double* __restrict__ b, const double* __restrict__ x,
                                  const double* __restrict__ Bx, const double* __restrict__ dvec, double c,
                                  float* __restrict__ r32, long long N, Scalars* outer, Scalars* inner, RedWork rw,
                                  int first, double inner_tol2) {
  if (outer->done) return;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double bi = b[i];
    double ri = bi - (dvec[i] * x[i] + c * Bx[i]);
    r32[i] = (float)ri;
    v[0] += bi * bi;
    v[1] += ri * ri;
  }
  double tot[2];
  if (grid_reduce<2>(v, rw, tot) && threadIdx.x == 0) {
    if (first) outer->bnorm2 = tot[0];
    outer->rnorm2 = tot[1];
    int done = 0;
    if (!finite(tot[0]) || !finite(tot[1])) { outer->breakdown = 1; done = 1; }
    else if (tot[1] <= outer->tol2 * outer->bnorm2) done = 1;
    outer->done = done;
    inner->done = done;
    inner->bnorm2 = tot[1];
    inner->tol2 = inner_tol2;
  }
}

void refine_residual_ex(const double* b, const double* x, const double* Bx, const double* dvec, double c,
                        float* r32, long long N, Scalars* outer, Scalars* inner, RedWork rw, bool first,
                        double inner_tol, cudaStream_t st) {
  k_refine_residual<<<red_blocks(N), kThreads, 0, st>>>(b, x, Bx, dvec, c, r32, N, outer, inner, rw, first ? 1 : 0,
                                                        inner_tol * inner_tol);
}

__global__ void k_refine_update(double* __restrict__ x, const float* __restrict__ dx, long long N,
                                const Scalars* outer) {
  if (outer->done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)dx[i];
}

void refine_update(double* x, const float* dx, long long N, Scalars* sc, cudaStream_t st) {
  k_refine_update<<<red_blocks(N), kThreads, 0, st>>>(x, dx, N, sc);
}

__global__ void k_reset_solve(Scalars* sc, double tol2) {
  sc->done = 0;
  sc->tol2 = tol2;
  sc->rho = sc->alpha = sc->beta = 0.0;
}
void scalars_reset_solve(Scalars* sc, double tol, cudaStream_t st) { k_reset_solve<<<1, 1, 0, st>>>(sc, tol * tol); }

__global__ void k_count_fail(Scalars* sc) {
  if (!sc->done) sc->fails += 1;
}
void scalars_count_fail(Scalars* sc, cudaStream_t st) { k_count_fail<<<1, 1, 0, st>>>(sc); }

__global__ void k_fblock_rhs(const double* __restrict__ rf, const double* __restrict__ yS,
                             const double* __restrict__ g2S, double cf, double* __restrict__ out, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    out[i] = (rf[i] - yS[i]) / (cf * g2S[i]);
}
void fblock_rhs(const double* rf, const double* yS, const double* g2S, double cf, double* out, long long N,
                cudaStream_t st) {
  k_fblock_rhs<<<red_blocks(N), kThreads, 0, st>>>(rf, yS, g2S, cf, out, N);
}

// ------------------------------------------------------------------------------------
// GMRES building blocks (FP64)
// ------------------------------------------------------------------------------------
// The orthogonalisation kernels of classical Gram-Schmidt stream the k basis vectors once per
// call and are bound by HBM bandwidth.  Both run a grid of exactly the resident CTAs (a grid-stride
// loop over the rows, one CTA wave), read the rows as double2 (16-byte loads, all of a thread's
// rows issued before their products are used), and handle a last odd element separately.
constexpr int kOrthThreads = 256;

template <typename K>
int resident_grid(K kern, int threads, long long work_items) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess || per < 1) per = 1;
  const long long need = (work_items + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(need, (long long)per * sms));
}

// Dot products h[t] = V_t . w for t < k.  A CTA of kDotThreads threads is kDotParts warp groups of
// four warps.  A pass over w takes up to kDotParts kDotVec vectors: with vg = 1, 2 or 4 vector
// groups (as many as the pass's vectors need), group q works on vectors (q mod vg) kDotVec + t (t <
// kDotVec) and on the share q div vg of the rows, so a thread holds kDotVec accumulators and loads
// (few registers, many warps), no group idles when k is small, and w comes from DRAM once per pass
// (the groups' loads of the same w entries meet in L1).  Per CTA and vector one partial,
// part[t nb + blockIdx], in a fixed order; the last CTA adds them (one warp per vector, lanes
// strided over the CTAs).
// VEC: V rows (leading dimension ld, even) and w 16-byte aligned, read as double2.
constexpr int kDotVec = 8;
constexpr int kDotParts = 4;
constexpr int kDotThreads = 128 * kDotParts;
template <bool VEC>
__global__ void __launch_bounds__(kDotThreads, 2)
k_multidot(const double* __restrict__ V, long long ld, int k, long long U, const double* __restrict__ w,
           double* __restrict__ h, RedWork rw) {
  __shared__ double red[kDotThreads / 32][kDotVec];
  __shared__ int am_last;
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int part = threadIdx.x / 128, tg = threadIdx.x % 128;  // warp group, thread in group
  for (int g0 = 0; g0 < k; g0 += kDotVec * kDotParts) {
    const int need = (k - g0 + kDotVec - 1) / kDotVec;       // vector groups this pass needs
    const int vg = need >= 3 ? 4 : need;                     // 1, 2 or 4
    const int es = kDotParts / vg;                           // row shares
    const int vp = part % vg, ep = part / vg;
    const long long tid = ((long long)blockIdx.x * es + ep) * 128 + tg;
    const long long stride = (long long)nb * es * 128;
    const int v0 = g0 + vp * kDotVec;
    const int cnt = max(0, min(kDotVec, k - v0));
    const double* Vg = V + (long long)v0 * ld;
    double acc[kDotVec];
#pragma unroll
    for (int t = 0; t < kDotVec; ++t) acc[t] = 0.0;
    if (cnt > 0) {
      if (VEC) {
        const double2* w2 = reinterpret_cast<const double2*>(w);
        const double2* V2 = reinterpret_cast<const double2*>(Vg);
        const long long ld2 = ld / 2, U2 = U / 2;
        for (long long i = tid; i < U2; i += stride) {
          const double2 wi = __ldg(w2 + i);
          // the vectors in two halves of four loads each (register budget of two CTAs per SM)
#pragma unroll
          for (int h = 0; h < kDotVec; h += 4) {
            double2 v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (h + t < cnt) v[t] = __ldcs(V2 + (h + t) * ld2 + i);
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (h + t < cnt) acc[h + t] = fma(v[t].y, wi.y, fma(v[t].x, wi.x, acc[h + t]));
          }
        }
        if ((U & 1) && tid == stride - 1) {
          const double wl = w[U - 1];
#pragma unroll
          for (int t = 0; t < kDotVec; ++t)
            if (t < cnt) acc[t] = fma(Vg[t * ld + U - 1], wl, acc[t]);
        }
      } else {
        for (long long i = tid; i < U; i += stride) {
          const double wi = __ldg(w + i);
          double v[kDotVec];
#pragma unroll
          for (int t = 0; t < kDotVec; ++t)
            if (t < cnt) v[t] = Vg[t * ld + i];
#pragma unroll
          for (int t = 0; t < kDotVec; ++t)
            if (t < cnt) acc[t] = fma(v[t], wi, acc[t]);
        }
      }
    }
    // CTA sums in a fixed order: warp butterflies, then the four warps of the group in order
#pragma unroll
    for (int t = 0; t < kDotVec; ++t) {
      const double a = warp_sum(acc[t]);
      if (lane == 0) red[wid][t] = a;
    }
    __syncthreads();
    if (threadIdx.x < kDotVec * vg) {
      // vector (q, t): the warps of the groups q, q + vg, ... in order
      const int q = threadIdx.x / kDotVec, t = threadIdx.x % kDotVec;
      if (g0 + q * kDotVec + t < k) {
        double sum = 0.0;
        for (int e = 0; e < es; ++e) {
          const int grp = e * vg + q;
#pragma unroll
          for (int u = 0; u < 4; ++u) sum += red[grp * 4 + u][t];
        }
        rw.part[(long long)(g0 + q * kDotVec + t) * nb + blockIdx.x] = sum;
      }
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(rw.ticket, 1u) == (unsigned)nb - 1);
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  for (int t = wid; t < k; t += kDotThreads / 32) {
    const double* pt = rw.part + (long long)t * nb;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nb; b += 128) {
      a0 += __ldcg(pt + b);
      a1 += __ldcg(pt + b + 32);
      a2 += __ldcg(pt + b + 64);
      a3 += __ldcg(pt + b + 96);
    }
    for (; b < nb; b += 32) a0 += __ldcg(pt + b);
    const double tot = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) h[t] = tot;
  }
  if (threadIdx.x == 0) *rw.ticket = 0u;
}

void multidot(const double* V, long long ld, int k, long long U, const double* w, double* h, RedWork rw,
              cudaStream_t st) {
  const bool vec = (ld % 2 == 0) && ((uintptr_t)V % 16 == 0) && ((uintptr_t)w % 16 == 0);
  // rows are walked by 128 threads per CTA (every warp group walks them)
  if (vec) {
    const int g = std::min(resident_grid(k_multidot<true>, kDotThreads, (U / 2 + 1) * kDotParts), kMaxRedBlocks);
    k_multidot<true><<<g, kDotThreads, 0, st>>>(V, ld, k, U, w, h, rw);
  } else {
    const int g = std::min(resident_grid(k_multidot<false>, kDotThreads, U * kDotParts), kMaxRedBlocks);
    k_multidot<false><<<g, kDotThreads, 0, st>>>(V, ld, k, U, w, h, rw);
  }
}

// w += sign * sum_{i<k} h[i] V_i
template <bool VEC>
__global__ void __launch_bounds__(kOrthThreads)
k_multiaxpy(const double* __restrict__ V, long long ld, int k, long long U, const double* __restrict__ h, double sign,
            double* __restrict__ w) {
  __shared__ double hs[64];
  for (int t = threadIdx.x; t < k; t += blockDim.x) hs[t] = sign * h[t];
  __syncthreads();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (VEC) {
    double2* w2 = reinterpret_cast<double2*>(w);
    const double2* V2 = reinterpret_cast<const double2*>(V);
    const long long ld2 = ld / 2, U2 = U / 2;
    for (long long i = tid; i < U2; i += stride) {
      double2 acc = w2[i];
      int t = 0;
      for (; t + 8 <= k; t += 8) {
        const double2* Vt = V2 + t * ld2 + i;
        const double2 v0 = __ldcs(Vt), v1 = __ldcs(Vt + ld2), v2 = __ldcs(Vt + 2 * ld2), v3 = __ldcs(Vt + 3 * ld2);
        const double2 v4 = __ldcs(Vt + 4 * ld2), v5 = __ldcs(Vt + 5 * ld2), v6 = __ldcs(Vt + 6 * ld2),
                      v7 = __ldcs(Vt + 7 * ld2);
        acc.x = fma(hs[t], v0.x, acc.x);
        acc.y = fma(hs[t], v0.y, acc.y);
        acc.x = fma(hs[t + 1], v1.x, acc.x);
        acc.y = fma(hs[t + 1], v1.y, acc.y);
        acc.x = fma(hs[t + 2], v2.x, acc.x);
        acc.y = fma(hs[t + 2], v2.y, acc.y);
        acc.x = fma(hs[t + 3], v3.x, acc.x);
        acc.y = fma(hs[t + 3], v3.y, acc.y);
        acc.x = fma(hs[t + 4], v4.x, acc.x);
        acc.y = fma(hs[t + 4], v4.y, acc.y);
        acc.x = fma(hs[t + 5], v5.x, acc.x);
        acc.y = fma(hs[t + 5], v5.y, acc.y);
        acc.x = fma(hs[t + 6], v6.x, acc.x);
        acc.y = fma(hs[t + 6], v6.y, acc.y);
        acc.x = fma(hs[t + 7], v7.x, acc.x);
        acc.y = fma(hs[t + 7], v7.y, acc.y);
      }
      for (; t < k; ++t) {
        const double2 v = __ldcs(V2 + t * ld2 + i);
        acc.x = fma(hs[t], v.x, acc.x);
        acc.y = fma(hs[t], v.y, acc.y);
      }
      w2[i] = acc;
    }
    if ((U & 1) && tid == stride - 1) {
      double acc = w[U - 1];
      for (int t = 0; t < k; ++t) acc = fma(hs[t], V[t * ld + U - 1], acc);
      w[U - 1] = acc;
    }
  } else {
    for (long long i = tid; i < U; i += stride) {
      double acc = w[i];
      for (int t = 0; t < k; ++t) acc = fma(hs[t], V[(long long)t * ld + i], acc);
      w[i] = acc;
    }
  }
}

void multiaxpy(const double* V, long long ld, int k, long long U, const double* h, double sign, double* w,
               cudaStream_t st) {
  const bool vec = (ld % 2 == 0) && ((uintptr_t)V % 16 == 0) && ((uintptr_t)w % 16 == 0);
  if (vec) {
    const int g = resident_grid(k_multiaxpy<true>, kOrthThreads, U / 2 + 1);
    k_multiaxpy<true><<<g, kOrthThreads, 0, st>>>(V, ld, k, U, h, sign, w);
  } else {
    const int g = resident_grid(k_multiaxpy<false>, kOrthThreads, U);
    k_multiaxpy<false><<<g, kOrthThreads, 0, st>>>(V, ld, k, U, h, sign, w);
  }
}

__global__ void k_norm2(const double* __restrict__ w, long long U, double* out, RedWork rw) {
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < U; i += (long long)gridDim.x * blockDim.x) {
    double a = w[i];
    v[0] = fma(a, a, v[0]);
  }
  double tot[1];
  if (grid_reduce<1>(v, rw, tot) && threadIdx.x == 0) *out = tot[0];
}
void norm2(const double* w, long long U, double* out, RedWork rw, cudaStream_t st) {
  k_norm2<<<red_blocks(U), kThreads, 0, st>>>(w, U, out, rw);
}

__global__ void k_scale_invnorm(const double* __restrict__ x, double* __restrict__ y, long long U,
                                const double* __restrict__ nrm2) {
  const double n2 = *nrm2;
  const double s = (n2 > 0.0) ? 1.0 / sqrt(n2) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < U; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}
void scale_by_invnorm(const double* x, double* y, long long U, const double* nrm2, cudaStream_t st) {
  int blocks = (int)std::min<long long>((U + kThreads - 1) / kThreads, 152 * 16);
  k_scale_invnorm<<<blocks, kThreads, 0, st>>>(x, y, U, nrm2);
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long long U) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < U; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
void axpby(double a, const double* x, double b, double* y, long long U, cudaStream_t st) {
  int blocks = (int)std::min<long long>((U + kThreads - 1) / kThreads, 152 * 16);
  k_axpby<<<blocks, kThreads, 0, st>>>(a, x, b, y, U);
}

// Column j of the Hessenberg matrix: Hcol[0..j] already holds V^T w, Hcol[j+1] = ||w||.
// Apply the j earlier rotations, form rotation j, update g; est = |g[j+1]|.
__global__ void k_givens(double* Hcol, double* cs, double* sn, double* g, int j, const double* hnew2, double* est) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Hcol[j + 1] = sqrt(*hnew2);
  for (int i = 0; i < j; ++i) {
    double a = Hcol[i], b = Hcol[i + 1];
    Hcol[i] = cs[i] * a + sn[i] * b;
    Hcol[i + 1] = -sn[i] * a + cs[i] * b;
  }
  double a = Hcol[j], b = Hcol[j + 1];
  double c = 1.0, s = 0.0, r = a;
  if (b != 0.0) {
    r = hypot(a, b);
    c = a / r;
    s = b / r;
  }
  cs[j] = c;
  sn[j] = s;
  Hcol[j] = r;
  Hcol[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  *est = fabs(g[j + 1]);
}
void givens_step(double* Hcol, double* cs, double* sn, double* g, int j, const double* hnew2, double* est,
                 cudaStream_t st) {
  k_givens<<<1, 32, 0, st>>>(Hcol, cs, sn, g, j, hnew2, est);
}

// Solve R y = g, R upper triangular k x k, column j of R at Hmat + j * ld.
__global__ void k_tri_solve(const double* Hmat, int ld, const double* g, int k, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int j = i + 1; j < k; ++j) acc -= Hmat[(long long)j * ld + i] * y[j];
    double d = Hmat[(long long)i * ld + i];
    y[i] = (d != 0.0) ? acc / d : 0.0;
  }
}
void tri_solve(const double* Hmat, int ld, const double* g, int k, double* yk, cudaStream_t st) {
  k_tri_solve<<<1, 32, 0, st>>>(Hmat, ld, g, k, yk);
}

__global__ void k_init_g(double* g, int len, const double* nrm2) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = (i == 0) ? sqrt(*nrm2) : 0.0;
}
void init_g(double* g, int len, const double* nrm2, cudaStream_t st) { k_init_g<<<1, 128, 0, st>>>(g, len, nrm2); }

__global__ void k_add_vec(const double* a, const double* b, double* out, int k) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) out[i] = a[i] + b[i];
}
void add_vec(const double* a, const double* b, double* out, int k, cudaStream_t st) {
  k_add_vec<<<1, 64, 0, st>>>(a, b, out, k);
}

}  // namespace tsfde
