// Fused element-wise work around the row passes of the spatial transforms.
//
// The first row pass of a transform (forward FFT of B_n x, first DST of a tau solve) can
// compute its input from the state of a CG / refinement iteration (load modes), and the
// last row pass can consume the transform's output (store modes).  Reductions of the
// fused work are deterministic grid reductions; the last block updates the scalars.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace tsfde {

enum LoadMode : int {
  LD_PLAIN = 0,       // v = src[i]
  LD_P_UPDATE = 1,    // p[i] = z[i] + beta p[i] (first: p = z); v = p[i]       (src = z)
  LD_X_UPDATE = 2,    // x[i] += dx32[i] (FP64 refinement); v = x[i]
  LD_PCG_UPDATE = 3,  // x[i] += alpha p[i]; r[i] -= alpha q[i]; v = r[i]; ||r||^2 -> done test
};

enum StoreMode : int {
  ST_PLAIN = 0,         // dst[i] = v
  ST_PCG_Q = 1,         // q[i] = dvec p + c v; p.q -> alpha = rho / p.q
  ST_RESID_REFINE = 2,  // r = b - (dvec x + c v) in FP64, r32[i] = (float) r (bx[i] = v if bx); outer done
                        // test, inner reset
  ST_RESID = 3,         // r[i] = b - (dvec x + c v); done test on ||r|| <= tol ||b||
  ST_RZ_FIRST = 4,      // dst[i] = v; p[i] = v; x[i] = 0 (if x); rho = r.z
  ST_RZ_BETA = 5,       // dst[i] = v; beta = r.z / rho; rho = r.z
};

template <typename R>
struct RowIO {
  int ld = LD_PLAIN, st = ST_PLAIN;
  const R* src = nullptr;   // LD_PLAIN input, LD_P_UPDATE z
  R* dst = nullptr;         // ST_PLAIN / ST_RZ_* output
  R* p = nullptr;
  R* x = nullptr;
  R* r = nullptr;
  const R* q = nullptr;
  R* qout = nullptr;
  const R* dvec = nullptr;
  const R* b = nullptr;
  R c = 0;
  int first = 0;
  const float* dx32 = nullptr;  // LD_X_UPDATE
  float* r32 = nullptr;         // ST_RESID_REFINE
  R* bx = nullptr;              // ST_RESID_REFINE: optional copy of v = (B_n x)_i
  double inner_tol2 = 0;
  Scalars* sc = nullptr;        // scalars of this solve
  Scalars* sc2 = nullptr;       // ST_RESID_REFINE: the inner solve's scalars
  RedWork rw{};
  const int* skip = nullptr;    // return at once when *skip != 0
  TSFDE_HD bool reduces_load() const { return ld == LD_PCG_UPDATE; }
  TSFDE_HD bool reduces_store() const { return st != ST_PLAIN; }
};

template <typename R>
TSFDE_D R io_load(const RowIO<R>& io, long long i, double* acc) {
  switch (io.ld) {
    case LD_P_UPDATE: {
      R v = io.first ? io.src[i] : io.src[i] + (R)io.sc->beta * io.p[i];
      io.p[i] = v;
      return v;
    }
    case LD_X_UPDATE: {
      R v = io.x[i] + (R)io.dx32[i];
      io.x[i] = v;
      return v;
    }
    case LD_PCG_UPDATE: {
      const R a = (R)io.sc->alpha;
      io.x[i] += a * io.p[i];
      R rv = io.r[i] - a * io.q[i];
      io.r[i] = rv;
      acc[0] += (double)rv * rv;
      return rv;
    }
    default:
      return io.src[i];
  }
}

template <typename R>
TSFDE_D void io_store(const RowIO<R>& io, long long i, R v, double* acc) {
  switch (io.st) {
    case ST_PCG_Q: {
      R pi = io.p[i];
      R qi = io.dvec[i] * pi + io.c * v;
      io.qout[i] = qi;
      acc[1] += (double)pi * qi;
      break;
    }
    case ST_RESID_REFINE: {
      R bi = io.b[i];
      R ri = bi - fma(io.dvec[i], io.x[i], io.c * v);
      io.r32[i] = (float)ri;
      if (io.bx) io.bx[i] = v;
      acc[0] += (double)bi * bi;
      acc[1] += (double)ri * ri;
      break;
    }
    case ST_RESID: {
      R bi = io.b[i];
      R ri = bi - fma(io.dvec[i], io.x[i], io.c * v);
      io.r[i] = ri;
      acc[0] += (double)bi * bi;
      acc[1] += (double)ri * ri;
      break;
    }
    case ST_RZ_FIRST: {
      io.dst[i] = v;
      io.p[i] = v;
      if (io.x) io.x[i] = R(0);
      acc[1] += (double)io.r[i] * v;
      break;
    }
    case ST_RZ_BETA: {
      io.dst[i] = v;
      acc[1] += (double)io.r[i] * v;
      break;
    }
    default:
      io.dst[i] = v;
  }
}

// Batched forms of io_load / io_store for J elements with indices idx[j] (valid when ok[j]):
// the mode is switched on once, every global load of the batch is issued before any value is
// used, so one memory latency is paid per batch instead of one per element.
template <typename R, int J>
TSFDE_D void io_load_batch(const RowIO<R>& io, const long long (&idx)[J], const bool (&ok)[J], R (&v)[J],
                           double* acc) {
  switch (io.ld) {
    case LD_P_UPDATE: {
      R z[J], p[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        z[j] = ok[j] ? io.src[idx[j]] : R(0);
        p[j] = (ok[j] && !io.first) ? io.p[idx[j]] : R(0);
      }
      const R bt = (R)io.sc->beta;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        v[j] = io.first ? z[j] : z[j] + bt * p[j];
        if (ok[j]) io.p[idx[j]] = v[j];
      }
      break;
    }
    case LD_X_UPDATE: {
      R x[J];
      float d[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        x[j] = ok[j] ? io.x[idx[j]] : R(0);
        d[j] = ok[j] ? io.dx32[idx[j]] : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        v[j] = x[j] + (R)d[j];
        if (ok[j]) io.x[idx[j]] = v[j];
      }
      break;
    }
    case LD_PCG_UPDATE: {
      R x[J], p[J], r[J], q[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        x[j] = ok[j] ? io.x[idx[j]] : R(0);
        p[j] = ok[j] ? io.p[idx[j]] : R(0);
        r[j] = ok[j] ? io.r[idx[j]] : R(0);
        q[j] = ok[j] ? io.q[idx[j]] : R(0);
      }
      const R a = (R)io.sc->alpha;
      R s0 = 0;  // per-thread partial in the working precision (FP64 only for the block sum)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const R rv = r[j] - a * q[j];
        v[j] = rv;
        if (ok[j]) {
          io.x[idx[j]] = x[j] + a * p[j];
          io.r[idx[j]] = rv;
          s0 += rv * rv;
        }
      }
      acc[0] += (double)s0;
      break;
    }
    default:
#pragma unroll
      for (int j = 0; j < J; ++j) v[j] = ok[j] ? io.src[idx[j]] : R(0);
  }
}

template <typename R, int J>
TSFDE_D void io_store_batch(const RowIO<R>& io, const long long (&idx)[J], const bool (&ok)[J], const R (&v)[J],
                            double* acc) {
  switch (io.st) {
    case ST_PCG_Q: {
      R p[J], d[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        p[j] = ok[j] ? io.p[idx[j]] : R(0);
        d[j] = ok[j] ? io.dvec[idx[j]] : R(0);
      }
      R s1 = 0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        if (ok[j]) {
          const R qi = d[j] * p[j] + io.c * v[j];
          io.qout[idx[j]] = qi;
          s1 += p[j] * qi;
        }
      }
      acc[1] += (double)s1;
      break;
    }
    case ST_RESID_REFINE:
    case ST_RESID: {
      R b[J], d[J], x[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        b[j] = ok[j] ? io.b[idx[j]] : R(0);
        d[j] = ok[j] ? io.dvec[idx[j]] : R(0);
        x[j] = ok[j] ? io.x[idx[j]] : R(0);
      }
      R s0 = 0, s1 = 0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        if (ok[j]) {
          const R ri = b[j] - fma(d[j], x[j], io.c * v[j]);
          if (io.st == ST_RESID_REFINE) {
            io.r32[idx[j]] = (float)ri;
            if (io.bx) io.bx[idx[j]] = v[j];
          } else {
            io.r[idx[j]] = ri;
          }
          s0 += b[j] * b[j];
          s1 += ri * ri;
        }
      }
      acc[0] += (double)s0;
      acc[1] += (double)s1;
      break;
    }
    case ST_RZ_FIRST:
    case ST_RZ_BETA: {
      R r[J];
#pragma unroll
      for (int j = 0; j < J; ++j) r[j] = ok[j] ? io.r[idx[j]] : R(0);
      R s1 = 0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        if (ok[j]) {
          io.dst[idx[j]] = v[j];
          if (io.st == ST_RZ_FIRST) {
            io.p[idx[j]] = v[j];
            if (io.x) io.x[idx[j]] = R(0);
          }
          s1 += r[j] * v[j];
        }
      }
      acc[1] += (double)s1;
      break;
    }
    default:
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (ok[j]) io.dst[idx[j]] = v[j];
  }
}

// Deterministic grid reduction of two values; true in the last block (totals valid there).
TSFDE_D bool io_grid_reduce2(double a0, double a1, RedWork rw, double* tot) {
  __shared__ double scratch[32];
  __shared__ int am_last;
  double s0 = block_sum(a0, scratch);
  double s1 = block_sum(a1, scratch);
  if (threadIdx.x == 0) {
    rw.part[blockIdx.x] = s0;
    rw.part[gridDim.x + blockIdx.x] = s1;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(rw.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double t0 = 0.0, t1 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    t0 += __ldcg(&rw.part[b]);
    t1 += __ldcg(&rw.part[gridDim.x + b]);
  }
  tot[0] = block_sum(t0, scratch);
  tot[1] = block_sum(t1, scratch);
  if (threadIdx.x == 0) *rw.ticket = 0u;
  return true;
}

// Scalar updates after the reduction (one thread of the last block).  `do_load` and
// `do_store` select which fused parts ran in this kernel.
template <typename R>
TSFDE_D void io_finalize(const RowIO<R>& io, bool do_load, bool do_store, const double* tot) {
  Scalars* sc = io.sc;
  if (do_load && io.ld == LD_PCG_UPDATE) {
    sc->iters += 1;
    sc->rnorm2 = tot[0];
    if (!isfinite(tot[0])) {
      sc->breakdown = 1;
      sc->done = 1;
    } else if (tot[0] <= sc->tol2 * sc->bnorm2) {
      sc->done = 1;
    }
    if (sc->done) return;
  }
  if (!do_store) return;
  switch (io.st) {
    case ST_PCG_Q:
      if (!(tot[1] > 0.0) || !isfinite(tot[1])) {
        sc->alpha = 0.0;
        if (!isfinite(tot[1])) sc->breakdown = 1;
        sc->done = 1;
      } else {
        sc->alpha = sc->rho / tot[1];
      }
      break;
    case ST_RESID_REFINE: {
      sc->sweeps += 1;
      if (io.first) sc->bnorm2 = tot[0];
      sc->rnorm2 = tot[1];
      int done = 0;
      if (!isfinite(tot[0]) || !isfinite(tot[1])) {
        sc->breakdown = 1;
        done = 1;
      } else if (tot[1] <= sc->tol2 * sc->bnorm2) {
        done = 1;
      }
      sc->done = done;
      io.sc2->done = done;
      io.sc2->bnorm2 = tot[1];
      io.sc2->rnorm2 = tot[1];
      // The FP32 correction aims at inner_tol2 relative to this residual, or, if that is looser,
      // at a tenth of what the block tolerance still asks (a last sweep stops there instead of
      // overshooting); at least a tenfold reduction either way.
      double t2 = io.inner_tol2;
      if (!done && tot[1] > 0.0) {
        double need = 0.01 * sc->tol2 * sc->bnorm2 / tot[1];
        if (need > 0.01) need = 0.01;
        if (need > t2) t2 = need;
      }
      io.sc2->tol2 = t2;
      break;
    }
    case ST_RESID:
      sc->sweeps += 1;
      sc->bnorm2 = tot[0];
      sc->rnorm2 = tot[1];
      if (!isfinite(tot[0]) || !isfinite(tot[1])) {
        sc->breakdown = 1;
        sc->done = 1;
      } else if (tot[1] <= sc->tol2 * tot[0]) {
        sc->done = 1;
      }
      break;
    case ST_RZ_FIRST:
      sc->rho = tot[1];
      if (!isfinite(tot[1])) {
        sc->breakdown = 1;
        sc->done = 1;
      }
      break;
    case ST_RZ_BETA:
      if (!isfinite(tot[1]) || sc->rho == 0.0) {
        sc->breakdown = !isfinite(tot[1]);
        sc->done = 1;
      } else {
        sc->beta = tot[1] / sc->rho;
        sc->rho = tot[1];
      }
      break;
    default:
      break;
  }
}

}  // namespace tsfde
