// Implementation of the persistent forward substitution (instantiated per transform length
// in fsub_l*.cu).
//
// Forward substitution for P_{n,S} y = r (Sec. 5.1 "Implementation"), or backward substitution
// for P^T, as ONE persistent cooperative kernel: every time level's history term, every
// refinement sweep of its block solve and every step of the inner tau-preconditioned CG run inside
// a single launch, with grid barriers between dependent passes.  One launch can serve a batch of
// instances with the same transform length, each on its own sub-grid of CTAs.  Control flow is decided on the device: every CTA reduces
// the same per-CTA partials in the same order, so all CTAs hold identical scalars and take the
// same branches; converged block solves cost nothing.
//
// Work decomposition.  A CTA of BLOCK threads holds NG line groups of NT = L / 8 threads; one
// group transforms one line (a pair of real rows, one complex column, or a pair of real
// columns for a DST) with its values in registers and shared memory for the exchanges.  Item i of
// a pass runs on CTA i mod G, group (i div G) mod NG of the instance's sub-grid of G CTAs, so the
// lines of a pass are spread over all SMs first.  Fields have n points per axis; the tau solves
// work on the np = L/2 - 1 grid (zero-padded when n + 1 is not a power of two).
//
// Grid barrier: arrive with a release add on a launch-wide counter, wait until it has counted
// every CTA; every wait is capped (FsubArgs::spin_limit polls, 2^24 by default); on expiry
// the kernel sets an error flag, every CTA leaves at its next barrier, and the host reports
// TSFDE_ETIMEOUT.
#pragma once

#include <math.h>

#include "fft.cuh"
#include "fsub.h"
#include "internal.h"
#include "kernels.h"
#include "rowio.cuh"

namespace tsfde {
namespace {

// positions per group of the blocked history sums
constexpr int kHB = 16;

template <int L>
struct LG {
  static constexpr int NT = L / 8;
  static constexpr int BLOCK = NT >= 256 ? NT : 256;
  static constexpr int NG = BLOCK / NT;
  static constexpr int LS = line_stride(L);
};

// Synchronisation of one line group: the whole CTA when the group is the CTA, a named barrier
// (id 1 + group) for groups of two or more warps, the warp itself for groups of one warp or less
// (every group of such a warp runs the same stages).  The CTA may hold LG<L>::NG groups (the
// kernel of one transform length) or more (512-thread CTAs of the mixed-length kernel); at most
// eight groups of two or more warps fit a CTA of 512 threads, so named barrier ids stay <= 8.
template <int L>
struct GSync {
  int id;
  TSFDE_D void operator()() const {
    if (LG<L>::NT == (int)blockDim.x) {
      __syncthreads();
    } else if constexpr (LG<L>::NT >= 64) {
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(LG<L>::NT) : "memory");
    } else {
      __syncwarp();
    }
  }
};

// Per-CTA state shared by all threads (kept in shared memory so that reading it after a
// barrier costs a shared-memory load, not a reload from local memory).
struct KShared {
  int G;         // CTAs of this instance's sub-grid
  int bid;       // this CTA's index in the sub-grid
  FsubBarrier bar;
  double* part;  // [2 parity][2 values][G]
  int parity;
  int phase;     // kind of the pass that the next barrier closes (timeline)
  int tn;        // timeline entries written by this launch (CTA 0)
  unsigned long long* trace;
  int trace_cap;
  int ok;        // 0 after a barrier time-out
  unsigned int epoch;  // grid barriers passed by this CTA in this launch
  long long spin_limit;  // polls of one barrier wait before it gives up
  int ng;        // line groups in this CTA (blockDim.x / NT)
  double scratch[64];
  double red[4];
};

// Passed by value: a pointer to the shared state and this thread's place in its line group.
struct KCtx {
  KShared* s;
  int grp, t;
};

TSFDE_D void set_phase(const KCtx& k, int ph) {
  if (threadIdx.x == 0) k.s->phase = ph;
}

TSFDE_D unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid barrier; returns false (in every thread) after a time-out anywhere.  The
// counter only grows during a launch (the host zeroes it before each launch): the k-th barrier
// is passed once it reaches k G.  Arrival is one release add (no reply needed); waiting is a
// poll with acquire loads, so the last arrival releases everyone after a single trip through
// L2 (a generation counter bumped by the last arriver costs two more).  The comparison is
// modulo 2^32 and stays valid while no CTA is 2^31 arrivals behind.
TSFDE_D unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
TSFDE_D void red_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Arrival and bounded wait of thread 0 (the caller synchronises the CTA before and after).  The
// fast path is one release add and polls of the counter alone: the error flag (set by a CTA whose
// wait ran out) is read every 32 polls, so a CTA leaves at most one barrier after the flag is set
// (the CTA that timed out arrives no more, and a wait that cannot finish sees the flag).
TSFDE_D int barrier_arrive_wait(KShared* s) {
  int ok = 1;
  s->epoch += 1;
  const unsigned int target = (unsigned int)s->G * s->epoch;
  red_release(s->bar.count, 1u);
  long long spins = 0;
  while ((int)(ld_acquire(s->bar.count) - target) < 0) {
    ++spins;
    if ((spins & 31) == 0) {
      volatile int* verr = s->bar.err;
      if (*verr) { ok = 0; break; }
    }
    if (spins > s->spin_limit) {
      atomicExch(s->bar.err, 1);
      ok = 0;
      break;
    }
  }
  if (s->trace && s->bid == 0 && s->tn < s->trace_cap) {
    s->trace[2 * s->tn] = global_ns();
    s->trace[2 * s->tn + 1] = (unsigned long long)s->phase;
    ++s->tn;
  }
  return ok;
}

TSFDE_D bool grid_sync(const KCtx& k) {
  KShared* s = k.s;
  __syncthreads();
  if (threadIdx.x == 0) s->ok = barrier_arrive_wait(s);
  __syncthreads();
  return s->ok != 0;
}

// Reduce NV (<= 4) per-thread values of type T (double, or float for the FP32 inner CG) over the
// grid; every CTA gets the same totals (fixed order: warp butterflies, then a butterfly over the
// warps' sums in warp 0, then the CTAs strided over the lanes of warp 0 and a butterfly).  All the
// adds run on full warps: a chain of adds on one thread would cost a full-warp issue per add on
// the FP64 pipe.  Partials are double-buffered by parity ([2 parity][4 values][G] doubles, a float
// partial in the first half of its slot), so a CTA that runs ahead cannot overwrite totals still
// being read.
template <typename T, int NV>
TSFDE_D bool reduce_syncT(const KCtx& k, const T (&a)[NV], double* tot) {
  static_assert(NV >= 1 && NV <= 4, "up to four values");
  KShared* s = k.s;
  const int G = s->G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* buf = reinterpret_cast<T*>(s->part + (size_t)s->parity * 4 * G);
  T* scr = reinterpret_cast<T*>(s->scratch);
  T v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(a[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) scr[NV * wid + i] = v[i];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(lane < nw ? scr[NV * lane + i] : T(0));
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) buf[(size_t)i * G + s->bid] = v[i];
      s->ok = barrier_arrive_wait(s);
      s->parity ^= 1;  // every thread read the parity before the first __syncthreads
    }
  }
  __syncthreads();
  if (wid == 0) {
    T t[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) t[i] = T(0);
    if (G <= 256) {
      // every partial load in flight at once, summed in the order of the loop below
      T x[8][NV];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int b = lane + 32 * q;
#pragma unroll
        for (int i = 0; i < NV; ++i) x[q][i] = b < G ? __ldcg(&buf[(size_t)i * G + b]) : T(0);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int i = 0; i < NV; ++i) t[i] += x[q][i];
      }
    } else {
      for (int b = lane; b < G; b += 32) {
#pragma unroll
        for (int i = 0; i < NV; ++i) t[i] += __ldcg(&buf[(size_t)i * G + b]);
      }
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) t[i] = warp_sum(t[i]);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) s->red[i] = (double)t[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) tot[i] = s->red[i];
  return s->ok != 0;
}

template <int NV>
TSFDE_D bool reduce_syncN(const KCtx& k, const double (&a)[NV], double* tot) {
  return reduce_syncT<double, NV>(k, a, tot);
}

// Two values: the FP64 passes (double) and the FP32 inner CG (float).
TSFDE_D bool reduce_sync(const KCtx& k, double a0, double a1, double* tot) {
  const double a[2] = {a0, a1};
  return reduce_syncT<double, 2>(k, a, tot);
}
TSFDE_D bool reduce_sync(const KCtx& k, float a0, float a1, double* tot) {
  const float a[2] = {a0, a1};
  return reduce_syncT<float, 2>(k, a, tot);
}

// Groups of at least a warp own their barrier, so a group without an item skips the pass;
// smaller groups share __syncwarp with the rest of their warp and always run.
template <int L>
TSFDE_D bool group_runs(bool act) {
  return act || LG<L>::NT < 32;
}

template <int L>
TSFDE_D long long rounds_for(const KCtx& k, long long items) {
  const long long per = (long long)k.s->G * k.s->ng;
  return (items + per - 1) / per;
}
template <int L>
TSFDE_D long long item_of(const KCtx& k, long long rd) {
  return rd * (long long)k.s->G * k.s->ng + (long long)k.grp * k.s->G + k.s->bid;
}

// ---- passes (one line per group per round) ----------------------------------------------

// Every thread of a group owns the 8 line positions t + j NT (j < 8); all of its global loads
// are issued before any is used, and the transforms keep the values in registers (fft_regs).

// d = 1 fused B_n apply of one field: load, FFT, symbol, inverse FFT, store.
template <typename R, int L>
TSFDE_D void pass_b1d(const KCtx& k, const RowIO<R>& io, int n, const R* lam, const cx<R>* tw, PBuf<R> buf,
                      double* acc) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const bool act = (k.s->bid == 0 && k.grp == 0);
  if (!group_runs<L>(act)) return;
  long long idx[8];
  bool ok[8];
  R a[8], lm[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = k.t + j * NT;
    idx[j] = p;
    ok[j] = act && p < n;
    lm[j] = lam[p <= L / 2 ? p : L - p];
  }
  io_load_batch<R, 8>(io, idx, ok, a, acc);
  cx<R> v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = mk<R>(a[j], R(0));
  fft_regs<R, L, -1>(v, buf, tw, k.t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = cscale<R>(v[j], lm[j]);
  fft_regs<R, L, 1>(v, buf, tw, k.t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = v[j].x;
  io_store_batch<R, 8>(io, idx, ok, a, acc);
}

// Last axis forward: pairs of real rows -> half spectra.
template <typename R, int L>
TSFDE_D void pass_rowfwd(const KCtx& k, const RowIO<R>& io, long long NR, int n, int H, cx<R>* out,
                         const cx<R>* tw, PBuf<R> buf, double* acc) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    long long idx[16];
    bool ok[16];
    R a[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      idx[j] = r0 * n + p;
      ok[j] = act && p < n && r0 < NR;
      idx[8 + j] = r1 * n + p;
      ok[8 + j] = act && p < n && r1 < NR;
    }
    io_load_batch<R, 16>(io, idx, ok, a, acc);
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = mk<R>(a[j], a[8 + j]);
    fft_regs<R, L, -1>(v, buf, tw, k.t, sync);
    // X_q = (Z_q + conj Z_{-q}) / 2, Y_q = (Z_q - conj Z_{-q}) / (2i): Z_{-q} is another thread's
#pragma unroll
    for (int j = 0; j < 8; ++j) buf[k.t + j * NT] = v[j];
    sync();
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = k.t + j * NT;
        if (q < H) {
          cx<R> zk = v[j], zm = buf[(L - q) & (L - 1)];
          if (r0 < NR) out[r0 * H + q] = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
          if (r1 < NR) out[r1 * H + q] = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
        }
      }
    }
    sync();
  }
}

// Last axis inverse: half spectra of two rows -> two real rows (first n), store mode.
template <typename R, int L>
TSFDE_D void pass_rowinv(const KCtx& k, const RowIO<R>& io, long long NR, int n, int H, const cx<R>* in,
                         const cx<R>* tw, PBuf<R> buf, double* acc) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    // Z_p = X_p + i Y_p for p <= L/2 and conj X_{L-p} + i conj Y_{L-p} above
    cx<R> X[8], Y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      const int q = p <= L / 2 ? p : L - p;
      X[j] = (act && r0 < NR) ? in[r0 * H + q] : mk<R>(0, 0);
      Y[j] = (act && r1 < NR) ? in[r1 * H + q] : mk<R>(0, 0);
    }
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      v[j] = (p <= L / 2) ? mk<R>(X[j].x - Y[j].y, X[j].y + Y[j].x) : mk<R>(X[j].x + Y[j].y, Y[j].x - X[j].y);
    }
    fft_regs<R, L, 1>(v, buf, tw, k.t, sync);
    long long idx[16];
    bool ok[16];
    R a[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      idx[j] = r0 * n + p;
      ok[j] = act && p < n && r0 < NR;
      a[j] = v[j].x;
      idx[8 + j] = r1 * n + p;
      ok[8 + j] = act && p < n && r1 < NR;
      a[8 + j] = v[j].y;
    }
    io_store_batch<R, 16>(io, idx, ok, a, acc);
  }
}

// ---- FP64 row passes on wide line groups (two groups, L / 4 threads, four values a thread) ----
// A pass over row pairs has about half as many lines as a pass over columns, so on groups of L / 8
// threads it keeps only half of the SM sub-partitions' FP64 pipes busy; each FP64 instruction of a
// warp holds its sub-partition's narrow FP64 pipe for many cycles, and the line's time is that of
// its busiest warps.  Pairs of groups (2g, 2g + 1) therefore run each line on L / 4 threads with
// fft_regs4: half the FP64 work per thread.  Items (row pairs) go to wide group w of CTA b as
// w G + b, as for the groups of one pass.  Usable when the CTA holds an even number of groups of at
// least a warp each (wide_rows<L>).
template <int L>
TSFDE_D bool wide_rows(const KCtx& k) {
  return LG<L>::NT >= 32 && (k.s->ng & 1) == 0;
}

// Synchronisation of a wide group: the CTA when the group is the CTA, else a named barrier
// (id 1 + wide group index, ids distinct from those the pass's other wide groups use).
struct WideSync {
  int id, n;
  TSFDE_D void operator()() const {
    if (n == (int)blockDim.x) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
};

// pass_rowfwd<double> on wide groups: two rows (load mode of io) -> their half spectra in out.
template <int L>
TSFDE_D void pass_rowfwd_w(const KCtx& k, const RowIO<double>& io, long long NR, int n, int H, cx<double>* out,
                           const cx<double>* tw, PBuf<double> buf, double* acc) {
  constexpr int NT = LG<L>::NT, NW = 2 * NT;
  const KShared* s = k.s;
  const int g2 = k.grp >> 1, t = (k.grp & 1) * NT + k.t;
  PBuf<double> wb{buf.p - (k.grp & 1) * LG<L>::LS};  // the line buffer of group 2 g2
  WideSync sync{1 + g2, NW};
  const long long per = (long long)s->G * (s->ng >> 1);
  const long long items = (NR + 1) / 2;
  const long long rounds = (items + per - 1) / per;
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = rd * per + (long long)g2 * s->G + s->bid;
    if (it >= items) continue;  // uniform in the wide group, which owns its barrier
    const long long r0 = 2 * it, r1 = r0 + 1;
    long long idx[8];
    bool ok[8];
    double a[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = t + j * NW;
      idx[j] = r0 * n + p;
      ok[j] = p < n && r0 < NR;
      idx[4 + j] = r1 * n + p;
      ok[4 + j] = p < n && r1 < NR;
    }
    io_load_batch<double, 8>(io, idx, ok, a, acc);
    cx<double> v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = mk<double>(a[j], a[4 + j]);
    fft_regs4<double, L, -1>(v, wb, tw, t, sync);
    // X_q = (Z_q + conj Z_{-q}) / 2, Y_q = (Z_q - conj Z_{-q}) / (2i): Z_{-q} is another thread's
#pragma unroll
    for (int j = 0; j < 4; ++j) wb[t + j * NW] = v[j];
    sync();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = t + j * NW;
      if (q < H) {
        const cx<double> zk = v[j], zm = wb[(L - q) & (L - 1)];
        if (r0 < NR) out[r0 * H + q] = mk<double>(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
        if (r1 < NR) out[r1 * H + q] = mk<double>(0.5 * (zk.y + zm.y), -0.5 * (zk.x - zm.x));
      }
    }
    sync();
  }
}

// pass_rowinv<double> on wide groups: half spectra of two rows -> the rows (first n), store mode.
template <int L>
TSFDE_D void pass_rowinv_w(const KCtx& k, const RowIO<double>& io, long long NR, int n, int H,
                           const cx<double>* in, const cx<double>* tw, PBuf<double> buf, double* acc) {
  constexpr int NT = LG<L>::NT, NW = 2 * NT;
  const KShared* s = k.s;
  const int g2 = k.grp >> 1, t = (k.grp & 1) * NT + k.t;
  PBuf<double> wb{buf.p - (k.grp & 1) * LG<L>::LS};
  WideSync sync{1 + g2, NW};
  const long long per = (long long)s->G * (s->ng >> 1);
  const long long items = (NR + 1) / 2;
  const long long rounds = (items + per - 1) / per;
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = rd * per + (long long)g2 * s->G + s->bid;
    if (it >= items) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    // Z_p = X_p + i Y_p for p <= L/2 and conj X_{L-p} + i conj Y_{L-p} above
    cx<double> v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = t + j * NW;
      const int q = p <= L / 2 ? p : L - p;
      const cx<double> X = (r0 < NR) ? in[r0 * H + q] : mk<double>(0, 0);
      const cx<double> Y = (r1 < NR) ? in[r1 * H + q] : mk<double>(0, 0);
      v[j] = (p <= L / 2) ? mk<double>(X.x - Y.y, X.y + Y.x) : mk<double>(X.x + Y.y, Y.x - X.y);
    }
    fft_regs4<double, L, 1>(v, wb, tw, t, sync);
    long long idx[8];
    bool ok[8];
    double a[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = t + j * NW;
      idx[j] = r0 * n + p;
      ok[j] = p < n && r0 < NR;
      a[j] = v[j].x;
      idx[4 + j] = r1 * n + p;
      ok[4 + j] = p < n && r1 < NR;
      a[4 + j] = v[j].y;
    }
    io_store_batch<double, 8>(io, idx, ok, a, acc);
  }
}

// Strided complex lines (o, i), element p at o*os + i + p*es.  MODE 0 forward, 1 forward +
// symbol lam[k*NI + i] + inverse, 2 inverse.
template <typename R, int L, int MODE>
TSFDE_D void pass_cline(const KCtx& k, const cx<R>* in, cx<R>* out, int NI, long long NO, long long in_os,
                        long long in_es, long long out_os, long long out_es, int n_load, int n_store, const R* lam,
                        const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (long long)NI * NO;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long o = act ? it / NI : 0;
    const int i = act ? (int)(it % NI) : 0;
    cx<R> v[8];
    R lm[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      v[j] = (act && p < n_load) ? in[o * in_os + i + (long long)p * in_es] : mk<R>(0, 0);
      if constexpr (MODE == 1) lm[j] = lam[(long long)p * NI + i];
    }
    if constexpr (MODE == 2) {
      fft_regs<R, L, 1>(v, buf, tw, k.t, sync);
    } else {
      fft_regs<R, L, -1>(v, buf, tw, k.t, sync);
    }
    if constexpr (MODE == 1) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = cscale<R>(v[j], lm[j]);
      fft_regs<R, L, 1>(v, buf, tw, k.t, sync);
    }
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = k.t + j * NT;
        if (p < n_store) out[o * out_os + i + (long long)p * out_es] = v[j];
      }
    }
  }
}

// Odd extension of two real lines held as the values of positions 1..n (slots j < 4, since
// n + 1 = L / 2 and slot j < 4 covers positions below L / 2): the slots j >= 4 receive the
// negated mirror -u_{L-p} through shared memory; positions 0 and L/2 are zero.
template <typename R, int L>
TSFDE_D void odd_extend(cx<R> (&v)[8], PBuf<R> buf, int t, GSync<L> sync) {
  constexpr int NT = LG<L>::NT;
#pragma unroll
  for (int j = 0; j < 4; ++j) buf[t + j * NT] = v[j];
  sync();
#pragma unroll
  for (int j = 4; j < 8; ++j) {
    const int p = t + j * NT;
    cx<R> m = (p == L / 2) ? mk<R>(0, 0) : buf[L - p];
    v[j] = mk<R>(-m.x, -m.y);
  }
  if (t == 0) v[0] = mk<R>(0, 0);
  sync();
}

// DST-I of two real lines (values of positions 1..n in slots j < 4 of v): on return slot j < 4
// holds (DST of line a, DST of line b) at k = t + j NT.  SCALE: the coefficients are scaled by
// norm / (dbar + c mu) and transformed again (the first axis of a tau solve).
template <typename R, int L, bool SCALE>
TSFDE_D void dst_regs(cx<R> (&v)[8], PBuf<R> buf, int n, const cx<R>* tw, int t, GSync<L> sync, const R* mu,
                      long long mstride, long long m0, long long m1, R dbar, R c, R norm, bool has1) {
  constexpr int NT = LG<L>::NT;
  R mu0[4], mu1[4];
  if constexpr (SCALE) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = t + j * NT;
      const bool in = q >= 1 && q <= n;
      mu0[j] = in ? mu[(long long)(q - 1) * mstride + m0] : R(1);
      mu1[j] = (in && has1) ? mu[(long long)(q - 1) * mstride + m1] : R(1);
    }
  }
  odd_extend<R, L>(v, buf, t, sync);
  fft_regs<R, L, -1>(v, buf, tw, t, sync);
  // DST(a)_k = -Im Z_k / 2, DST(b)_k = Re Z_k / 2
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = mk<R>(R(-0.5) * v[j].y, R(0.5) * v[j].x);
  if constexpr (SCALE) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j].x *= norm / (dbar + c * mu0[j]);
      v[j].y = has1 ? v[j].y * (norm / (dbar + c * mu1[j])) : R(0);
    }
    odd_extend<R, L>(v, buf, t, sync);
    fft_regs<R, L, -1>(v, buf, tw, t, sync);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = mk<R>(R(-0.5) * v[j].y, R(0.5) * v[j].x);
  }
}

// Contiguous rows (last axis) of the tau solve.  A pair of rows is loaded at positions 1..n_in:
// from the fused load mode of io (USE_LD: data rows, row stride n_in) or from tin (row stride
// tin_rs); sine-transformed with length np = L/2 - 1 (positions above n_in are zero: the data is
// zero-padded to the transform grid); and stored at positions 1..n_out: to the fused store mode
// of io (USE_ST: data rows, row stride n_out) or to tout (row stride tout_rs).  SCALE: d = 1, the
// whole solve (transform, scale, transform) in one pass.
template <typename R, int L, bool SCALE, bool USE_LD, bool USE_ST>
TSFDE_D void pass_dst_rows(const KCtx& k, const RowIO<R>& io, const R* tin, long long tin_rs, R* tout,
                           long long tout_rs, long long NR, int n_in, int n_out, int np, const R* mu, R dbar, R c,
                           R norm, const cx<R>* tw, PBuf<R> buf, double* acc) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  const long long in_rs = USE_LD ? n_in : tin_rs;
  const long long out_rs = USE_ST ? n_out : tout_rs;
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    long long idx[8];
    bool ok[8];
    R a[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;  // positions 0 .. L/2 - 1; data at 1..n_in
      const bool in = act && p >= 1 && p <= n_in;
      idx[j] = r0 * in_rs + p - 1;
      ok[j] = in && r0 < NR;
      idx[4 + j] = r1 * in_rs + p - 1;
      ok[4 + j] = in && r1 < NR;
    }
    if (USE_LD) {
      io_load_batch<R, 8>(io, idx, ok, a, acc);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = ok[j] ? tin[idx[j]] : R(0);
    }
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = mk<R>(a[j], a[4 + j]);
    dst_regs<R, L, SCALE>(v, buf, np, tw, k.t, sync, mu, 1, 0, 0, dbar, c, norm, r1 < NR);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = k.t + j * NT;
      const bool in = act && q >= 1 && q <= n_out;
      a[j] = v[j].x;
      a[4 + j] = v[j].y;
      idx[j] = r0 * out_rs + q - 1;
      ok[j] = in && r0 < NR;
      idx[4 + j] = r1 * out_rs + q - 1;
      ok[4 + j] = in && r1 < NR;
    }
    if (USE_ST) {
      io_store_batch<R, 8>(io, idx, ok, a, acc);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (ok[j]) tout[idx[j]] = a[j];
    }
  }
}

// Strided real lines (o, i), paired (i, i+1): n_in values loaded from in[o in_os + i + (p-1) in_es],
// p = 1..n_in, zero-padded to the transform length np = L/2 - 1, sine-transformed, and n_out values
// stored to out[o out_os + i + (q-1) out_es] (in place when in == out).  SCALE: the first axis of
// the tau solve, eigenvalue index (k-1) NI + i.
template <typename R, int L, bool SCALE>
TSFDE_D void pass_dst_strided(const KCtx& k, const R* in, R* out, int NI, long long NO, long long in_os,
                              long long in_es, long long out_os, long long out_es, int n_in, int n_out, int np,
                              const R* mu, R dbar, R c, R norm, const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const int npair = (NI + 1) / 2;
  const long long items = (long long)npair * NO;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long o = act ? it / npair : 0;
    const int i0 = act ? 2 * (int)(it % npair) : 0, i1 = i0 + 1;
    const bool has1 = act && i1 < NI;
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;
      const bool ld = act && p >= 1 && p <= n_in;
      const long long base = o * in_os + (long long)(p - 1) * in_es;
      R a = ld ? in[base + i0] : R(0);
      R b = (ld && has1) ? in[base + i1] : R(0);
      v[j] = mk<R>(a, b);
    }
    dst_regs<R, L, SCALE>(v, buf, np, tw, k.t, sync, mu, NI, i0, has1 ? i1 : i0, dbar, c, norm, has1);
    if (act) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = k.t + j * NT;
        if (q >= 1 && q <= n_out) {
          const long long base = o * out_os + (long long)(q - 1) * out_es;
          out[base + i0] = v[j].x;
          if (has1) out[base + i1] = v[j].y;
        }
      }
    }
  }
}

// ---- Fourier passes of the Strang solve: DFTs of length n by Bluestein's chirp-z transform ----
// s(B_n) is a d-level circulant of size n, diagonalised by DFTs of length n, which need not be a
// power of two.  A DFT of length n becomes a circular convolution of length L >= 2 n - 1:
// jk = (j^2 + k^2 - (k - j)^2) / 2 gives X_k = c_k sum_j (x_j c_j) conj(c_{k-j}) with the chirp
// c_j = exp(-i pi j^2 / n).  chirp holds c_j (j < n); bhat the length-L FFT of the conjugate chirp
// placed at m and L - m (|m| < n), divided by L.  Two FFTs of length L per DFT.

// In-place forward DFT X_k = sum_j x_j exp(-2 pi i jk / n) of the values in the slots
// p = t + j NT < n of v; slots p >= n are ignored on input and zero on output.
template <typename R, int L>
TSFDE_D void czt_regs(cx<R> (&v)[8], PBuf<R> buf, int n, const cx<R>* chirp, const cx<R>* bhat, const cx<R>* tw,
                      int t, GSync<L> sync) {
  constexpr int NT = LG<L>::NT;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = t + j * NT;
    v[j] = p < n ? cmul<R>(v[j], chirp[p]) : mk<R>(0, 0);
  }
  fft_regs<R, L, -1>(v, buf, tw, t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = cmul<R>(v[j], bhat[t + j * NT]);
  fft_regs<R, L, 1>(v, buf, tw, t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = t + j * NT;
    v[j] = p < n ? cmul<R>(v[j], chirp[p]) : mk<R>(0, 0);
  }
}

// Unnormalised inverse DFT x_j = sum_k X_k exp(+2 pi i jk / n) = conj(DFT(conj X))_j.
template <typename R, int L>
TSFDE_D void iczt_regs(cx<R> (&v)[8], PBuf<R> buf, int n, const cx<R>* chirp, const cx<R>* bhat, const cx<R>* tw,
                       int t, GSync<L> sync) {
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = cconj<R>(v[j]);
  czt_regs<R, L>(v, buf, n, chirp, bhat, tw, t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = cconj<R>(v[j]);
}

// d = 1: the whole solve dst = (dbar I + c s(B_n))^-1 src in one line (CTA 0, group 0).
template <typename R, int L>
TSFDE_D void pass_czt_1d(const KCtx& k, const R* src, R* dst, int n, const R* slam, R dbar, R c, R norm,
                         const cx<R>* chirp, const cx<R>* bhat, const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const bool act = (k.s->bid == 0 && k.grp == 0);
  if (!group_runs<L>(act)) return;
  cx<R> v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = k.t + j * NT;
    v[j] = mk<R>((act && p < n) ? src[p] : R(0), R(0));
  }
  czt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = k.t + j * NT;
    if (p < n) v[j] = cscale<R>(v[j], norm / (dbar + c * slam[p]));
  }
  iczt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
  if (act) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      if (p < n) dst[p] = v[j].x;
    }
  }
}

// Last axis forward: pairs of real rows of src (row stride n) -> half spectra out [NR][Hn],
// Hn = n / 2 + 1, through one complex DFT per pair.
template <typename R, int L>
TSFDE_D void pass_czt_rows_fwd(const KCtx& k, const R* src, long long NR, int n, int Hn, cx<R>* out,
                               const cx<R>* chirp, const cx<R>* bhat, const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      const bool in = act && p < n;
      v[j] = mk<R>((in && r0 < NR) ? src[r0 * n + p] : R(0), (in && r1 < NR) ? src[r1 * n + p] : R(0));
    }
    czt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
    // X_q = (Z_q + conj Z_{n-q}) / 2, Y_q = (Z_q - conj Z_{n-q}) / (2i): Z_{n-q} is another thread's
#pragma unroll
    for (int j = 0; j < 8; ++j) buf[k.t + j * NT] = v[j];
    sync();
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = k.t + j * NT;
        if (q < Hn) {
          const cx<R> zk = v[j], zm = buf[q == 0 ? 0 : n - q];
          if (r0 < NR) out[r0 * Hn + q] = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
          if (r1 < NR) out[r1 * Hn + q] = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
        }
      }
    }
    sync();
  }
}

// Last axis inverse: half spectra of two rows (in [NR][Hn], extended by Hermitian symmetry) ->
// two real rows of dst (row stride n).
template <typename R, int L>
TSFDE_D void pass_czt_rows_inv(const KCtx& k, const cx<R>* in, long long NR, int n, int Hn, R* dst,
                               const cx<R>* chirp, const cx<R>* bhat, const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      cx<R> X = mk<R>(0, 0), Y = mk<R>(0, 0);
      if (act && p < n) {
        const int q = p < Hn ? p : n - p;
        if (r0 < NR) X = in[r0 * Hn + q];
        if (r1 < NR) Y = in[r1 * Hn + q];
        if (p >= Hn) {
          X = cconj<R>(X);
          Y = cconj<R>(Y);
        }
      }
      v[j] = mk<R>(X.x - Y.y, X.y + Y.x);  // X + i Y
    }
    iczt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = k.t + j * NT;
        if (p < n) {
          if (r0 < NR) dst[r0 * n + p] = v[j].x;
          if (r1 < NR) dst[r1 * n + p] = v[j].y;
        }
      }
    }
  }
}

// Complex lines (o, i), o < NO, i < NI, element p < n at w[o os + i + p es], transformed in place.
// MODE 0 forward DFT; 2 inverse; 1 forward, division by dbar + c lambda (eigenvalue index
// p nd1 + (i / Hn) n + i mod Hn: this axis first, the half-spectrum axis last) times norm, inverse.
template <typename R, int L, int MODE>
TSFDE_D void pass_czt_lines(const KCtx& k, cx<R>* w, int NI, long long NO, long long os, long long es, int n, int Hn,
                            long long nd1, const R* slam, R dbar, R c, R norm, const cx<R>* chirp, const cx<R>* bhat,
                            const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (long long)NI * NO;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long o = act ? it / NI : 0;
    const int i = act ? (int)(it % NI) : 0;
    const long long base = o * os + i;
    cx<R> v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      v[j] = (act && p < n) ? w[base + (long long)p * es] : mk<R>(0, 0);
    }
    if constexpr (MODE == 2) {
      iczt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
    } else {
      czt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
    }
    if constexpr (MODE == 1) {
      const long long e0 = (long long)(i / Hn) * n + (i % Hn);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = k.t + j * NT;
        if (p < n) v[j] = cscale<R>(v[j], norm / (dbar + c * slam[(long long)p * nd1 + e0]));
      }
      iczt_regs<R, L>(v, buf, n, chirp, bhat, tw, k.t, sync);
    }
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = k.t + j * NT;
        if (p < n) w[base + (long long)p * es] = v[j];
      }
    }
  }
}

// ---- passes of the fused inner CG (d >= 2) ------------------------------------------------
// One CG step on  (diag(dvec) + c B) x = r  with preconditioner (dbar I + c tau(B))^-1 is
// four passes in 2-D (eight in 3-D) instead of six (ten): by linearity, the row spectra of
// p = z + beta p_old are Wz + beta Wp_old and the row DSTs of r = r_old - alpha q are
// Tr_old - alpha Tq, so the search-direction and residual updates ride on the passes that
// produce z and q:
//   cols   W = Wz + beta Wp (kept as the new Wp), column transforms of B          (no reduction)
//   rowsq  rows of B p; p = z + beta p_old; q = dvec p + c B p; Tq = DST_rows(q)   (p.q -> alpha)
//   tcols  T = Tr - alpha Tq (kept as the new Tr), column transforms of the tau solve
//   rowsz  z = DST_rows(T); x += alpha p; r -= alpha q; Wz = FFT_rows(z)            (r.r, r.z -> beta)

// Complex strided lines with the combination W = Wz + beta Wp (first: W = Wz) stored back to Wp
// (positions < n_load), then transformed like pass_cline.
template <typename R, int L, int MODE>
TSFDE_D void pass_cg_cols(const KCtx& k, const cx<R>* wz, cx<R>* wp, R beta, bool first, cx<R>* out, int NI,
                          long long NO, long long in_os, long long in_es, long long out_os, long long out_es,
                          int n_load, int n_store, const R* lam, const cx<R>* tw, PBuf<R> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (long long)NI * NO;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long o = act ? it / NI : 0;
    const int i = act ? (int)(it % NI) : 0;
    cx<R> v[8], u[8];
    R lm[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      const bool in = act && p < n_load;
      const long long a = o * in_os + i + (long long)p * in_es;
      v[j] = in ? wz[a] : mk<R>(0, 0);
      u[j] = (in && !first) ? wp[a] : mk<R>(0, 0);
      if constexpr (MODE == 1) lm[j] = lam[(long long)p * NI + i];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      if (!first) v[j] = mk<R>(v[j].x + beta * u[j].x, v[j].y + beta * u[j].y);
      if (act && p < n_load) wp[o * in_os + i + (long long)p * in_es] = v[j];
    }
    fft_regs<R, L, -1>(v, buf, tw, k.t, sync);
    if constexpr (MODE == 1) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = cscale<R>(v[j], lm[j]);
      fft_regs<R, L, 1>(v, buf, tw, k.t, sync);
    }
    if (act) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = k.t + j * NT;
        if (p < n_store) out[o * out_os + i + (long long)p * out_es] = v[j];
      }
    }
  }
}

// Two rows of values (index p at slot t + j NT, p < n) -> DST-I of both rows on the transform grid
// (length L/2 - 1 >= n, the data zero-padded): returns the coefficients k = 1..L/2-1 in slots j < 4
// (k = t + j NT), through one shared-memory exchange that shifts the values to positions 1..n and
// builds the odd extension.
template <typename R, int L>
TSFDE_D void rows_to_dst(cx<R> (&v)[8], PBuf<R> buf, int n, const cx<R>* tw, int t, GSync<L> sync) {
  constexpr int NT = LG<L>::NT;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = t + j * NT;
    if (p < n) buf[p + 1] = v[j];
  }
  sync();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int p = t + j * NT;
    v[j] = (p >= 1 && p <= n) ? buf[p] : mk<R>(0, 0);
  }
#pragma unroll
  for (int j = 4; j < 8; ++j) {
    const int p = t + j * NT;
    const cx<R> m = (p == L / 2 || L - p > n) ? mk<R>(0, 0) : buf[L - p];
    v[j] = mk<R>(-m.x, -m.y);
  }
  sync();
  fft_regs<R, L, -1>(v, buf, tw, t, sync);
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = mk<R>(R(-0.5) * v[j].y, R(0.5) * v[j].x);
}

// DST coefficients k = 1..n in slots j < 4 -> the same two rows as values at index k - 1
// placed in slots t + j NT (index p < n), then the forward row FFT and its half spectra.
template <typename R, int L>
TSFDE_D void dst_to_row_spectra(const cx<R> (&zv)[4], cx<R>* out, long long r0, long long r1, long long NR, int n,
                                int H, bool act, PBuf<R> buf, const cx<R>* tw, int t, GSync<L> sync) {
  constexpr int NT = LG<L>::NT;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = t + j * NT;
    if (q >= 1 && q <= n) buf[q - 1] = zv[j];
  }
  sync();
  cx<R> v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = t + j * NT;
    v[j] = (p < n) ? buf[p] : mk<R>(0, 0);
  }
  sync();
  fft_regs<R, L, -1>(v, buf, tw, t, sync);
#pragma unroll
  for (int j = 0; j < 8; ++j) buf[t + j * NT] = v[j];
  sync();
  if (act) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int q = t + j * NT;
      if (q < H) {
        const cx<R> zk = v[j], zm = buf[(L - q) & (L - 1)];
        if (r0 < NR) out[r0 * H + q] = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
        if (r1 < NR) out[r1 * H + q] = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
      }
    }
  }
  sync();
}

// The vectors of the fused inner CG.  x, r, p, q, z: node values [N]; tr, tq: row sine transforms of
// r and q, and tt: the tau solve's intermediate in the same layout, [N / n rows][np coefficients];
// tt2: the 3-D solve's second intermediate [n][np][np]; wz, wp: row half spectra of z and p; w0, w1:
// the B_n work buffers.
struct CgVec {
  float *x, *r, *p, *q, *z;
  float *tt, *tr, *tq, *tt2;
  float2 *wz, *wp, *w0, *w1;
  const float* dvec;
};

// rows of B p (inverse row FFT of w0) -> p, q, p.q, Tq
template <int L>
TSFDE_D void pass_cg_rowsq(const KCtx& k, const CgVec& V, long long NR, int n, int np, int H, float c, float beta,
                           bool first, const cx<float>* tw, PBuf<float> buf, float* acc) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    cx<float> X[8], Y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      const int q = p <= L / 2 ? p : L - p;
      X[j] = (act && r0 < NR) ? V.w0[r0 * H + q] : mk<float>(0, 0);
      Y[j] = (act && r1 < NR) ? V.w0[r1 * H + q] : mk<float>(0, 0);
    }
    // node operands of the two rows
    float z0[8], z1[8], po0[8], po1[8], d0[8], d1[8];
    bool ok0[8], ok1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      ok0[j] = act && p < n && r0 < NR;
      ok1[j] = act && p < n && r1 < NR;
      const long long a0 = r0 * n + p, a1 = r1 * n + p;
      z0[j] = ok0[j] ? V.z[a0] : 0.f;
      z1[j] = ok1[j] ? V.z[a1] : 0.f;
      po0[j] = (ok0[j] && !first) ? V.p[a0] : 0.f;
      po1[j] = (ok1[j] && !first) ? V.p[a1] : 0.f;
      d0[j] = ok0[j] ? V.dvec[a0] : 0.f;
      d1[j] = ok1[j] ? V.dvec[a1] : 0.f;
    }
    cx<float> v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      v[j] = (p <= L / 2) ? mk<float>(X[j].x - Y[j].y, X[j].y + Y[j].x)
                          : mk<float>(X[j].x + Y[j].y, Y[j].x - X[j].y);
    }
    fft_regs<float, L, 1>(v, buf, tw, k.t, sync);
    float s1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int p = k.t + j * NT;
      const float pn0 = first ? z0[j] : z0[j] + beta * po0[j];
      const float pn1 = first ? z1[j] : z1[j] + beta * po1[j];
      const float q0 = d0[j] * pn0 + c * v[j].x;
      const float q1 = d1[j] * pn1 + c * v[j].y;
      if (ok0[j]) {
        V.p[r0 * n + p] = pn0;
        V.q[r0 * n + p] = q0;
        s1 += pn0 * q0;
      }
      if (ok1[j]) {
        V.p[r1 * n + p] = pn1;
        V.q[r1 * n + p] = q1;
        s1 += pn1 * q1;
      }
      v[j] = mk<float>(ok0[j] ? q0 : 0.f, ok1[j] ? q1 : 0.f);
    }
    acc[1] += s1;
    rows_to_dst<float, L>(v, buf, n, tw, k.t, sync);
    if (act) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = k.t + j * NT;
        if (q >= 1 && q <= np) {
          if (r0 < NR) V.tq[r0 * np + q - 1] = v[j].x;
          if (r1 < NR) V.tq[r1 * np + q - 1] = v[j].y;
        }
      }
    }
  }
}

// Strided real lines of the tau solve (its first strided pass), loading T = Tr - alpha Tq
// (positions 1..n_in at o in_os + i + (p-1) in_es) and keeping it as the new Tr; INIT: T = Tr as it
// is (Tq is not read, Tr not rewritten).  The sine transform has length np; n_out values are
// stored to out (layout out_os, out_es).  SCALE: this pass is the first axis (d = 2), eigenvalue
// index (k-1) NI + i.
template <int L, bool SCALE>
TSFDE_D void pass_cg_tcols(const KCtx& k, const CgVec& V, float alpha, bool init, int NI, long long NO,
                           long long in_os, long long in_es, float* out, long long out_os, long long out_es, int n_in,
                           int n_out, int np, const float* mu, float dbar, float c, float norm, const cx<float>* tw,
                           PBuf<float> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const int npair = (NI + 1) / 2;
  const long long items = (long long)npair * NO;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long o = act ? it / npair : 0;
    const int i0 = act ? 2 * (int)(it % npair) : 0, i1 = i0 + 1;
    const bool has1 = act && i1 < NI;
    float ra[4], rb[4], qa[4], qb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;
      const bool in = act && p >= 1 && p <= n_in;
      const long long base = o * in_os + (long long)(p - 1) * in_es;
      ra[j] = in ? V.tr[base + i0] : 0.f;
      rb[j] = (in && has1) ? V.tr[base + i1] : 0.f;
      qa[j] = (in && !init) ? V.tq[base + i0] : 0.f;
      qb[j] = (in && has1 && !init) ? V.tq[base + i1] : 0.f;
    }
    cx<float> v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;
      const bool in = act && p >= 1 && p <= n_in;
      const float ta = init ? ra[j] : ra[j] - alpha * qa[j];
      const float tb = init ? rb[j] : rb[j] - alpha * qb[j];
      if (in && !init) {
        const long long base = o * in_os + (long long)(p - 1) * in_es;
        V.tr[base + i0] = ta;
        if (has1) V.tr[base + i1] = tb;
      }
      v[j] = mk<float>(ta, has1 ? tb : 0.f);
    }
    dst_regs<float, L, SCALE>(v, buf, np, tw, k.t, sync, mu, NI, i0, has1 ? i1 : i0, dbar, c, norm, has1);
    if (act) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = k.t + j * NT;
        if (q >= 1 && q <= n_out) {
          const long long base = o * out_os + (long long)(q - 1) * out_es;
          out[base + i0] = v[j].x;
          if (has1) out[base + i1] = v[j].y;
        }
      }
    }
  }
}

// first pass of the initial tau solve: Tr = DST_rows(r)
template <int L>
TSFDE_D void pass_cg_rows_init(const KCtx& k, const CgVec& V, long long NR, int n, int np, const cx<float>* tw,
                               PBuf<float> buf) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    cx<float> v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;
      const bool in = act && p >= 1 && p <= n;
      v[j] = mk<float>((in && r0 < NR) ? V.r[r0 * n + p - 1] : 0.f, (in && r1 < NR) ? V.r[r1 * n + p - 1] : 0.f);
    }
    dst_regs<float, L, false>(v, buf, np, tw, k.t, sync, nullptr, 0, 0, 0, 0.f, 0.f, 1.f, r1 < NR);
    if (act) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = k.t + j * NT;
        if (q >= 1 && q <= np) {
          if (r0 < NR) V.tr[r0 * np + q - 1] = v[j].x;
          if (r1 < NR) V.tr[r1 * np + q - 1] = v[j].y;
        }
      }
    }
  }
}

// Last pass of a tau solve: z = DST_rows(T) (T in tt, rows of np coefficients); INIT: r.z only
// (x set to 0 when zero_x); else x += alpha p, r -= alpha q and the new r's r.r and r.z; then
// Wz = FFT_rows(z).
template <int L>
TSFDE_D void pass_cg_rowsz(const KCtx& k, const CgVec& V, long long NR, int n, int np, int H, float alpha,
                           bool init, bool zero_x, const cx<float>* tw, PBuf<float> buf, float* acc) {
  constexpr int NT = LG<L>::NT;
  GSync<L> sync{1 + k.grp};
  const long long items = (NR + 1) / 2;
  const long long rounds = rounds_for<L>(k, items);
  for (long long rd = 0; rd < rounds; ++rd) {
    const long long it = item_of<L>(k, rd);
    const bool act = it < items;
    if (!group_runs<L>(act)) continue;
    const long long r0 = 2 * it, r1 = r0 + 1;
    // tau-solve rows and the node operands (index q - 1 for coefficient q = t + j NT)
    cx<float> v[8];
    float xa[4], xb[4], pa[4], pb[4], ra[4], rb[4], qa[4], qb[4];
    bool oka[4], okb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;
      const bool in = act && p >= 1 && p <= n;
      const bool inc = act && p >= 1 && p <= np;
      oka[j] = in && r0 < NR;
      okb[j] = in && r1 < NR;
      const long long a0 = r0 * n + p - 1, a1 = r1 * n + p - 1;
      v[j] = mk<float>((inc && r0 < NR) ? V.tt[r0 * np + p - 1] : 0.f, (inc && r1 < NR) ? V.tt[r1 * np + p - 1] : 0.f);
      ra[j] = oka[j] ? V.r[a0] : 0.f;
      rb[j] = okb[j] ? V.r[a1] : 0.f;
      xa[j] = (oka[j] && !init) ? V.x[a0] : 0.f;
      xb[j] = (okb[j] && !init) ? V.x[a1] : 0.f;
      pa[j] = (oka[j] && !init) ? V.p[a0] : 0.f;
      pb[j] = (okb[j] && !init) ? V.p[a1] : 0.f;
      qa[j] = (oka[j] && !init) ? V.q[a0] : 0.f;
      qb[j] = (okb[j] && !init) ? V.q[a1] : 0.f;
    }
    dst_regs<float, L, false>(v, buf, np, tw, k.t, sync, nullptr, 0, 0, 0, 0.f, 0.f, 1.f, r1 < NR);
    float s0 = 0.f, s1 = 0.f;
    cx<float> zv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = k.t + j * NT;
      const long long a0 = r0 * n + p - 1, a1 = r1 * n + p - 1;
      const float rna = init ? ra[j] : ra[j] - alpha * qa[j];
      const float rnb = init ? rb[j] : rb[j] - alpha * qb[j];
      zv[j] = v[j];
      if (oka[j]) {
        V.z[a0] = v[j].x;
        if (!init) V.x[a0] = xa[j] + alpha * pa[j];
        else if (zero_x) V.x[a0] = 0.f;
        if (!init) V.r[a0] = rna;
        s0 += rna * rna;
        s1 += rna * v[j].x;
      }
      if (okb[j]) {
        V.z[a1] = v[j].y;
        if (!init) V.x[a1] = xb[j] + alpha * pb[j];
        else if (zero_x) V.x[a1] = 0.f;
        if (!init) V.r[a1] = rnb;
        s0 += rnb * rnb;
        s1 += rnb * v[j].y;
      }
    }
    acc[0] += s0;
    acc[1] += s1;
    dst_to_row_spectra<float, L>(zv, V.wz, r0, r1, NR, n, H, act, buf, tw, k.t, sync);
  }
}

// ---- whole transforms of one field --------------------------------------------------------

template <typename R>
// One field's transforms: n points per axis, N = n^d; the FFT length L >= 2 (n + 1) and the
// tau solve's grid np = L/2 - 1 >= n (the data zero-padded to it when n + 1 is not a power of
// two); lam the circulant symbol of B_n on the L grid, mu the tau(B_np) eigenvalues [np]^d; w0, w1
// the B_n work buffers; t1 [N / n][np] and t2 [n][np][np] (d = 3) the tau solve's intermediates.
struct FPlan {
  int d, n, np, L, H;
  long long N;
  const cx<R>* tw;
  const R* lam;
  const R* mu;
  cx<R>* w0;
  cx<R>* w1;
  R* t1;
  R* t2;
};

// Tables of the Strang solve: Bluestein chirp [n] and FFT of the conjugate chirp [L] / L, the
// eigenvalues of s(B_n) [n]^d in DFT order.
template <typename R>
struct SPlan {
  const cx<R>* chirp;
  const cx<R>* bhat;
  const R* slam;
};

// B_n applied to one field with fused load / store; ends with a grid reduction whose totals
// are finalised into io.sc (and io.sc2).  Returns false after a barrier time-out.
template <typename R, int L>
__device__ __noinline__ bool bapply_field(const KCtx k, const RowIO<R> io_in, const FPlan<R> P_in, PBuf<R> buf) {
  __shared__ RowIO<R> s_io;
  __shared__ FPlan<R> s_P;
  if (threadIdx.x == 0) {
    s_io = io_in;
    s_P = P_in;
  }
  __syncthreads();
  const RowIO<R>& io = s_io;
  const FPlan<R>& P = s_P;
  double acc[2] = {0.0, 0.0};
  const int n = P.n, H = P.H;
  if (P.d == 1) {
    pass_b1d<R, L>(k, io, n, P.lam, P.tw, buf, acc);
  } else {
    const long long NR = P.N / n;
    const int base = sizeof(R) == 8 ? PH_B64_ROWFWD : PH_B32_ROWFWD;
    set_phase(k, base);
    if constexpr (sizeof(R) == 8) {
      if (wide_rows<L>(k)) pass_rowfwd_w<L>(k, io, NR, n, H, P.w0, P.tw, buf, acc);
      else pass_rowfwd<R, L>(k, io, NR, n, H, P.w0, P.tw, buf, acc);
    } else {
      pass_rowfwd<R, L>(k, io, NR, n, H, P.w0, P.tw, buf, acc);
    }
    if (!grid_sync(k)) return false;
    set_phase(k, base + 1);
    if (P.d == 2) {
      pass_cline<R, L, 1>(k, P.w0, P.w0, H, 1, (long long)n * H, H, (long long)n * H, H, n, n, P.lam, P.tw, buf);
      if (!grid_sync(k)) return false;
    } else {
      pass_cline<R, L, 0>(k, P.w0, P.w1, H, n, (long long)n * H, H, (long long)L * H, H, n, L, nullptr, P.tw, buf);
      if (!grid_sync(k)) return false;
      pass_cline<R, L, 1>(k, P.w1, P.w1, L * H, 1, (long long)n * L * H, (long long)L * H, (long long)n * L * H,
                          (long long)L * H, n, n, P.lam, P.tw, buf);
      if (!grid_sync(k)) return false;
      pass_cline<R, L, 2>(k, P.w1, P.w0, H, n, (long long)L * H, H, (long long)n * H, H, L, n, nullptr, P.tw, buf);
      if (!grid_sync(k)) return false;
    }
    set_phase(k, base + 2);
    if constexpr (sizeof(R) == 8) {
      if (wide_rows<L>(k)) pass_rowinv_w<L>(k, io, NR, n, H, P.w0, P.tw, buf, acc);
      else pass_rowinv<R, L>(k, io, NR, n, H, P.w0, P.tw, buf, acc);
    } else {
      pass_rowinv<R, L>(k, io, NR, n, H, P.w0, P.tw, buf, acc);
    }
  }
  if (P.d == 1) set_phase(k, sizeof(R) == 8 ? PH_B64_ROWINV : PH_B32_ROWINV);
  double tot[2];
  bool ok = reduce_sync(k, acc[0], acc[1], tot);
  if (threadIdx.x == 0) io_finalize(io, false, true, tot);
  __syncthreads();
  return ok;
}

// (dbar I + c tau(B_np))^-1 applied to one field: the first pass loads with io's load mode (and
// its reduction), the last stores with its store mode (io.dst the output); the intermediates live
// in P.t1 / P.t2 on the padded coefficient grid.  When the load-side test finishes the CG, the
// remaining passes are skipped.
template <typename R, int L>
__device__ __noinline__ bool tau_field(const KCtx k, const RowIO<R> io_in, const FPlan<R> P_in, R dbar, R c,
                                       PBuf<R> buf) {
  __shared__ RowIO<R> s_io;
  __shared__ FPlan<R> s_P;
  if (threadIdx.x == 0) {
    s_io = io_in;
    s_P = P_in;
  }
  __syncthreads();
  const RowIO<R>& io = s_io;
  const FPlan<R>& P = s_P;
  const int n = P.n, np = P.np;
  R norm = 1;
  for (int i = 0; i < P.d; ++i) norm *= R(2.0 / (np + 1));
  double acc[2] = {0.0, 0.0};
  double tot[2];
  if (P.d == 1) {
    set_phase(k, PH_TAU_ROWS_OUT);
    if (k.s->bid == 0)
      pass_dst_rows<R, L, true, true, true>(k, io, nullptr, 0, nullptr, 0, 1, n, n, np, P.mu, dbar, c, norm, P.tw, buf,
                                           acc);
    bool ok = reduce_sync(k, acc[0], acc[1], tot);
    if (threadIdx.x == 0) io_finalize(io, true, true, tot);
    __syncthreads();
    return ok;
  }
  const long long NR = P.N / n;
  set_phase(k, PH_TAU_ROWS_IN);
  pass_dst_rows<R, L, false, true, false>(k, io, nullptr, 0, P.t1, np, NR, n, np, np, nullptr, dbar, c, norm, P.tw,
                                         buf, acc);
  if (io.reduces_load()) {
    bool ok = reduce_sync(k, acc[0], acc[1], tot);
    if (threadIdx.x == 0) io_finalize(io, true, false, tot);
    __syncthreads();
    if (!ok) return false;
    if (io.sc->done) return true;
  } else if (!grid_sync(k)) {
    return false;
  }
  set_phase(k, PH_TAU_COLS);
  if (P.d == 2) {
    // columns k1 of t1 [n][np]: n values at stride np, scaled on the [np][np] grid
    pass_dst_strided<R, L, true>(k, P.t1, P.t1, np, 1, 0, np, 0, np, n, n, np, P.mu, dbar, c, norm, P.tw, buf);
    if (!grid_sync(k)) return false;
  } else {
    const long long np2 = (long long)np * np;
    // axis 1: t1 [n][n][np] -> t2 [n][np][np]; axis 0 scaled on [np]^3; axis 1 back to t1
    pass_dst_strided<R, L, false>(k, P.t1, P.t2, np, n, (long long)n * np, np, np2, np, n, np, np, nullptr, dbar, c,
                                  norm, P.tw, buf);
    if (!grid_sync(k)) return false;
    pass_dst_strided<R, L, true>(k, P.t2, P.t2, (int)np2, 1, 0, np2, 0, np2, n, n, np, P.mu, dbar, c, norm, P.tw,
                                 buf);
    if (!grid_sync(k)) return false;
    pass_dst_strided<R, L, false>(k, P.t2, P.t1, np, n, np2, np, (long long)n * np, np, np, n, np, nullptr, dbar, c,
                                  norm, P.tw, buf);
    if (!grid_sync(k)) return false;
  }
  acc[0] = acc[1] = 0.0;
  set_phase(k, PH_TAU_ROWS_OUT);
  pass_dst_rows<R, L, false, false, true>(k, io, P.t1, np, nullptr, 0, NR, np, n, np, nullptr, dbar, c, norm, P.tw,
                                         buf, acc);
  bool ok = reduce_sync(k, acc[0], acc[1], tot);
  if (threadIdx.x == 0) io_finalize(io, false, true, tot);
  __syncthreads();
  return ok;
}

// dst = (dbar I + c s(B_n))^-1 src for one field (S_{n,S} of Remark 1): forward DFTs of length n
// along every axis, division by the eigenvalues of the Strang circulant, inverse DFTs.  The row
// half spectra live in P.w0 ([N / n][n / 2 + 1] complex).  Ends with a grid barrier.  Timeline
// phases are those of the tau solve (rows in, columns, rows out).
template <typename R, int L>
__device__ __noinline__ bool strang_field(const KCtx k, const R* src, R* dst, const FPlan<R> P_in,
                                          const SPlan<R> Q_in, R dbar, R c, PBuf<R> buf) {
  __shared__ FPlan<R> s_P;
  __shared__ SPlan<R> s_Q;
  if (threadIdx.x == 0) {
    s_P = P_in;
    s_Q = Q_in;
  }
  __syncthreads();
  const FPlan<R>& P = s_P;
  const SPlan<R>& Q = s_Q;
  const int n = P.n, Hn = n / 2 + 1;
  R norm = 1;
  for (int i = 0; i < P.d; ++i) norm /= R(n);
  if (P.d == 1) {
    set_phase(k, PH_TAU_ROWS_OUT);
    pass_czt_1d<R, L>(k, src, dst, n, Q.slam, dbar, c, norm, Q.chirp, Q.bhat, P.tw, buf);
    return grid_sync(k);
  }
  const long long NR = P.N / n;
  cx<R>* w = P.w0;
  set_phase(k, PH_TAU_ROWS_IN);
  pass_czt_rows_fwd<R, L>(k, src, NR, n, Hn, w, Q.chirp, Q.bhat, P.tw, buf);
  if (!grid_sync(k)) return false;
  set_phase(k, PH_TAU_COLS);
  if (P.d == 2) {
    // columns k2 < Hn: n values at stride Hn
    pass_czt_lines<R, L, 1>(k, w, Hn, 1, 0, Hn, n, Hn, n, Q.slam, dbar, c, norm, Q.chirp, Q.bhat, P.tw, buf);
    if (!grid_sync(k)) return false;
  } else {
    const long long nH = (long long)n * Hn, n2 = (long long)n * n;
    // w [n][n][Hn]: axis 1 forward; axis 0 forward, divide, inverse; axis 1 inverse
    pass_czt_lines<R, L, 0>(k, w, Hn, n, nH, Hn, n, Hn, n2, Q.slam, dbar, c, norm, Q.chirp, Q.bhat, P.tw, buf);
    if (!grid_sync(k)) return false;
    pass_czt_lines<R, L, 1>(k, w, (int)nH, 1, 0, nH, n, Hn, n2, Q.slam, dbar, c, norm, Q.chirp, Q.bhat, P.tw, buf);
    if (!grid_sync(k)) return false;
    pass_czt_lines<R, L, 2>(k, w, Hn, n, nH, Hn, n, Hn, n2, Q.slam, dbar, c, norm, Q.chirp, Q.bhat, P.tw, buf);
    if (!grid_sync(k)) return false;
  }
  set_phase(k, PH_TAU_ROWS_OUT);
  pass_czt_rows_inv<R, L>(k, w, NR, n, Hn, dst, Q.chirp, Q.bhat, P.tw, buf);
  return grid_sync(k);
}

// ---- history term of the right-hand side, blocked in time ------------------------------------
// Position p in processing order holds level lev(p) (forward: p; transposed: S - 1 - p); the
// history of position p is sum_{p' < p} e_{p-p'} u(p') with u(p') = y^(lev p') (forward) or
// dvec^(lev p') y^(lev p') (transposed: D_1 lam = dvec w), since |level difference| = p - p'.
TSFDE_D double hist_u(const FsubArgs& a, int pp, long long j) {
  const int lev = a.trans ? a.S - 1 - pp : pp;
  const long long o = (long long)lev * a.N + j;
  return a.trans ? a.dvec64[o] * a.y[o] : a.y[o];
}

// Inner tau-preconditioned CG on (diag(dvec) + c B_n) x = r for d >= 2, with the fused passes
// above.  Starts from x = 0 (zero_x; r is the right-hand side) or from the x in place (r its
// residual), and runs at most max_steps steps or until ||r||^2 <= tol2 ||b||^2 (sc).  The
// iteration is the one of tau_field / bapply_field (same alpha, beta and stopping test); only
// the row transforms of p and r are formed by recurrence instead of from p and r.
template <int L>
__device__ __noinline__ bool cg_fused(const KCtx k, const CgVec V_in, const FPlan<float> P_in, float dbar, float c,
                                      int max_steps, bool zero_x, Scalars* sc, PBuf<float> buf) {
  __shared__ CgVec s_V;
  __shared__ FPlan<float> s_P;
  if (threadIdx.x == 0) {
    s_V = V_in;
    s_P = P_in;
  }
  __syncthreads();
  const CgVec& V = s_V;
  const FPlan<float>& P = s_P;
  const int n = P.n, np = P.np, H = P.H, L_ = P.L;
  const long long NR = P.N / n;
  const long long np2 = (long long)np * np;
  float norm = 1.f;
  for (int i = 0; i < P.d; ++i) norm *= 2.0f / (float)(np + 1);
  float acc[2];
  double tot[2];
  RowIO<float> fin;
  fin.sc = sc;

  // tau solve of a field whose row transforms are in tr (combined with tq unless init);
  // leaves the column-transformed field in tt for pass_cg_rowsz
  auto tau_cols = [&](bool init, float alpha) -> bool {
    set_phase(k, PH_TAU_COLS);
    if (P.d == 2) {
      // columns k1 of Tr, Tq [n][np]: n values at stride np, scaled on [np][np], into tt [n][np]
      pass_cg_tcols<L, true>(k, V, alpha, init, np, 1, 0, np, V.tt, 0, np, n, n, np, P.mu, dbar, c, norm, P.tw, buf);
      return grid_sync(k);
    }
    // axis 1: Tr, Tq [n][n][np] -> tt2 [n][np][np]; axis 0 scaled on [np]^3; axis 1 back into tt
    pass_cg_tcols<L, false>(k, V, alpha, init, np, n, (long long)n * np, np, V.tt2, np2, np, n, np, np, nullptr,
                            dbar, c, norm, P.tw, buf);
    if (!grid_sync(k)) return false;
    pass_dst_strided<float, L, true>(k, V.tt2, V.tt2, (int)np2, 1, 0, np2, 0, np2, n, n, np, P.mu, dbar, c, norm,
                                     P.tw, buf);
    if (!grid_sync(k)) return false;
    pass_dst_strided<float, L, false>(k, V.tt2, V.tt, np, n, np2, np, (long long)n * np, np, np, n, np, nullptr,
                                      dbar, c, norm, P.tw, buf);
    return grid_sync(k);
  };

  // z = tau^-1 r, p = z, rho = r.z
  set_phase(k, PH_TAU_ROWS_IN);
  pass_cg_rows_init<L>(k, V, NR, n, np, P.tw, buf);
  if (!grid_sync(k)) return false;
  if (!tau_cols(true, 0.f)) return false;
  set_phase(k, PH_TAU_ROWS_OUT);
  acc[0] = acc[1] = 0.f;
  pass_cg_rowsz<L>(k, V, NR, n, np, H, 0.f, true, zero_x, P.tw, buf, acc);
  if (!reduce_sync(k, acc[0], acc[1], tot)) return false;
  if (threadIdx.x == 0) {
    fin.ld = LD_PLAIN;
    fin.st = ST_RZ_FIRST;
    io_finalize(fin, false, true, tot);
  }
  __syncthreads();
  for (int it = 0; it < max_steps && !sc->done; ++it) {
    const bool first = (it == 0);
    const float beta = (float)sc->beta;
    // columns of B p from the row spectra Wp = Wz + beta Wp
    set_phase(k, PH_B32_COLS);
    if (P.d == 2) {
      pass_cg_cols<float, L, 1>(k, V.wz, V.wp, beta, first, V.w0, H, 1, (long long)n * H, H, (long long)n * H, H, n,
                                n, P.lam, P.tw, buf);
      if (!grid_sync(k)) return false;
    } else {
      pass_cg_cols<float, L, 0>(k, V.wz, V.wp, beta, first, V.w1, H, n, (long long)n * H, H, (long long)L_ * H, H, n,
                                L_, nullptr, P.tw, buf);
      if (!grid_sync(k)) return false;
      pass_cline<float, L, 1>(k, V.w1, V.w1, L_ * H, 1, (long long)n * L_ * H, (long long)L_ * H,
                              (long long)n * L_ * H, (long long)L_ * H, n, n, P.lam, P.tw, buf);
      if (!grid_sync(k)) return false;
      pass_cline<float, L, 2>(k, V.w1, V.w0, H, n, (long long)L_ * H, H, (long long)n * H, H, L_, n, nullptr, P.tw,
                              buf);
      if (!grid_sync(k)) return false;
    }
    // rows of B p; p, q, p.q -> alpha; Tq
    set_phase(k, PH_B32_ROWINV);
    acc[0] = acc[1] = 0.f;
    pass_cg_rowsq<L>(k, V, NR, n, np, H, c, beta, first, P.tw, buf, acc);
    if (!reduce_sync(k, acc[0], acc[1], tot)) return false;
    if (threadIdx.x == 0) {
      fin.ld = LD_PLAIN;
      fin.st = ST_PCG_Q;
      io_finalize(fin, false, true, tot);
    }
    __syncthreads();
    if (sc->done) break;
    const float alpha = (float)sc->alpha;
    if (!tau_cols(false, alpha)) return false;
    // z of the new residual; x, r updated; r.r (stopping test) and r.z -> beta
    set_phase(k, PH_TAU_ROWS_OUT);
    acc[0] = acc[1] = 0.f;
    pass_cg_rowsz<L>(k, V, NR, n, np, H, alpha, false, false, P.tw, buf, acc);
    if (!reduce_sync(k, acc[0], acc[1], tot)) return false;
    if (threadIdx.x == 0) {
      fin.ld = LD_PCG_UPDATE;
      fin.st = ST_RZ_BETA;
      io_finalize(fin, true, true, tot);
    }
    __syncthreads();
  }
  return true;
}

// Positions come in groups of kHB: at the first position `base` of a group every thread streams
// the finished positions p' < base once and keeps kHB sums, F_t = sum_{p'<base} e_{base+t-p'} u(p'),
// stored in hfar[t][j]; position base + t then adds only its near terms base <= p' < p.  Every
// thread handles the same nodes j in every phase, so hfar needs no barrier of its own.  (Run
// concurrently with the FP32 CG passes by idle line groups, these FP64 sums slowed the passes by
// about as much as they saved: the sums stay at the group start.)
// highest order of the extrapolated initial guess of a block solve (slots of B_n x kept)
constexpr int kMaxWarm = 8;

// Weights of the extrapolated guess: c[ord][k-1] = (-1)^(k+1) C(ord, k), zero for k > ord, built in
// integers at compile time (C(ord, k) = C(ord, k-1) (ord-k+1) / k divides exactly) and read from
// constant memory with the level's uniform ord.
struct ExtrapWeights {
  double c[kMaxWarm + 1][kMaxWarm];
};
constexpr ExtrapWeights make_extrap_weights() {
  ExtrapWeights t{};
  for (int ord = 0; ord <= kMaxWarm; ++ord) {
    long long b = 1;
    for (int q = 1; q <= kMaxWarm; ++q) {
      b = b * (ord - q + 1) / q;
      t.c[ord][q - 1] = (q & 1) ? (double)b : -(double)b;
    }
  }
  return t;
}
static __constant__ ExtrapWeights kExtrap = make_extrap_weights();

__device__ __noinline__ double hist_far(const FsubArgs& a, int base, long long j) {
  double F[kHB];
#pragma unroll
  for (int t = 0; t < kHB; ++t) F[t] = 0.0;
  const int S = a.S;
  int pp = 0;
  for (; pp + 4 <= base; pp += 4) {
    double u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = hist_u(a, pp + k, j);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int t = 0; t < kHB; ++t) {
        const int m = base + t - (pp + k);  // >= 1
        if (m < S) F[t] = fma(__ldg(&a.ew[m]), u[k], F[t]);
      }
    }
  }
  for (; pp < base; ++pp) {
    const double u = hist_u(a, pp, j);
#pragma unroll
    for (int t = 0; t < kHB; ++t) {
      const int m = base + t - pp;
      if (m < S) F[t] = fma(__ldg(&a.ew[m]), u, F[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < kHB; ++t)
    if (base + t < S) a.hfar[(long long)t * a.N + j] = F[t];
  return F[0];
}

// The near terms base <= p' < p (at most kHB - 1): every load is issued before any product, so one
// memory latency is paid for all of them; the products stop at the p - base terms that exist (a
// uniform bound: FP64 instructions are the scarce resource here, each costs a full-warp issue).
TSFDE_D double history(const FsubArgs& a, int p, long long j) {
  const int base = (p / kHB) * kHB;
  const int cnt = p - base;
  double far = 0.0;
  if (base > 0) far = (p == base) ? hist_far(a, base, j) : a.hfar[(long long)cnt * a.N + j];
  double u[kHB - 1], w[kHB - 1];
#pragma unroll
  for (int t = 0; t < kHB - 1; ++t) {
    const bool in = t < cnt;
    u[t] = in ? hist_u(a, base + t, j) : 0.0;
    w[t] = in ? __ldg(&a.ew[cnt - t]) : 0.0;
  }
  double h[4] = {far, 0.0, 0.0, 0.0};
#pragma unroll
  for (int t = 0; t < kHB - 1; ++t) {
    if (t >= cnt) break;
    h[t & 3] = fma(w[t], u[t], h[t & 3]);
  }
  return (h[0] + h[1]) + (h[2] + h[3]);
}

// ---- the kernel ----------------------------------------------------------------------------

// The whole substitution of one instance, run by block `bid` of the instance's own sub-grid of G
// CTAs (its own barrier counter, partial sums and counters), so instances sharing a launch run
// independently.  The CTA may have LG<L>::BLOCK threads or more (the mixed-length kernel).
template <int L>
__device__ __forceinline__ void fsub_body(const FsubArgs* argp, int G, int bid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ KShared s_k;
  __shared__ Scalars s_sc[2];  // [0] outer (refinement), [1] inner (CG); identical in every CTA
  __shared__ int s_fails[2];
  __shared__ int s_fix;       // guess of this level replaced: 1 previous level, 2 zero
  __shared__ int s_fixes;     // levels whose guess was replaced (statistics)
  __shared__ double s_red[1];
  __shared__ FsubArgs s_a;
  {
    static_assert(sizeof(FsubArgs) % sizeof(long long) == 0, "FsubArgs copied in 8-byte words");
    const long long* src = reinterpret_cast<const long long*>(argp);
    long long* dst = reinterpret_cast<long long*>(&s_a);
    for (int i = threadIdx.x; i < (int)(sizeof(FsubArgs) / sizeof(long long)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const FsubArgs& a = s_a;
  const int ng = (int)blockDim.x / LG<L>::NT;
  if (threadIdx.x == 0) {
    s_k.G = G;
    s_k.bid = bid;
    s_k.ng = ng;
    s_k.bar = a.bar;
    s_k.part = a.part;
    s_k.parity = 0;
    s_k.phase = PH_RHS;
    s_k.tn = 0;
    s_k.trace = a.trace;
    s_k.trace_cap = a.trace_cap;
    s_k.ok = 1;
    s_k.epoch = 0;
    s_k.spin_limit = a.spin_limit;
  }
  KCtx k;
  k.s = &s_k;
  k.grp = threadIdx.x / LG<L>::NT;
  k.t = threadIdx.x % LG<L>::NT;
  PBuf<double> buf64{reinterpret_cast<cx<double>*>(smem_raw) + (size_t)k.grp * LG<L>::LS};
  PBuf<float> buf32{reinterpret_cast<cx<float>*>(smem_raw) + (size_t)k.grp * LG<L>::LS};
  // twiddle tables in shared memory for the whole launch (after the line buffers)
  cx<double>* tw64s = reinterpret_cast<cx<double>*>(smem_raw) + (size_t)ng * LG<L>::LS;
  cx<float>* tw32s = reinterpret_cast<cx<float>*>(tw64s + L);
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    tw64s[i] = a.tw64[i];
    tw32s[i] = a.tw32[i];
  }
  if (threadIdx.x == 0) {
    s_sc[0] = Scalars{};
    s_sc[1] = Scalars{};
    s_fails[0] = s_fails[1] = 0;
    s_fix = 0;
    s_fixes = 0;
  }
  __syncthreads();
  Scalars* outer = &s_sc[0];
  Scalars* inner = &s_sc[1];
  const long long N = a.N;
  const int S = a.S;
  FPlan<double> P64{a.d, a.n, L / 2 - 1, L, L / 2 + 1, N, tw64s, a.lam64, a.mu64, a.w64a, a.w64b, a.t1_64, a.t2_64};
  FPlan<float> P32{a.d, a.n, L / 2 - 1, L, L / 2 + 1, N, tw32s, a.lam32, a.mu32, a.w32a, a.w32b, a.t1_32, a.t2_32};
  const long long gtid = (long long)s_k.bid * blockDim.x + threadIdx.x;
  const long long gstride = (long long)s_k.G * blockDim.x;
  bool ok = true;

  for (int step = 0; step <= S && ok; ++step) {
    // forward: levels 0..S-1, then the f block; transposed: the f block, then levels S-1..0
    const int sl = a.trans ? S - step : step;
    const bool fblock = (sl == S);
    double* x64 = a.y + (long long)sl * N;
    // ---- right-hand side of the block and the initial guess -----------------------------
    // The initial guess x0 of a level extrapolates the levels solved before it, in processing
    // order: the previous one (warm = 1), linearly from two (2 y1 - y2, warm = 2), and so on up
    // to the polynomial of degree warm - 1 through the last warm levels (warm <= kMaxWarm), with
    // as many as exist.  The level solutions vary smoothly in time, so each order lowers the
    // initial block residual by one to two decades (relative residuals about 1e-3, 5e-6, 1e-7,
    // 3e-9, 1e-10 for orders 1..5 on the vectors GMRES applies P^-1 to), until the rounding of
    // the earlier levels, amplified by sum |c_k| = 2^warm - 1, takes over.  With a zero initial guess the first
    // residual is the right-hand side itself: it is written here (FP32 copy) and its norm reduced
    // at this phase's barrier.  In FP64 mode with a warm start, the first residual
    // b - (D x0 + c B_n x0) is formed here as well, from B_n x0 = the same combination of the
    // B_n x that the earlier positions' last refinement residuals stored (slots of lBx, position
    // p in slot p mod kMaxWarm): B_n is linear, so no B_n apply is needed.  Every slot must hold
    // B_n x of its position's final x to FP64 rounding: a combination of slots carries their
    // rounding times sum |c_k| = 2^ord - 1, and used again in later combinations that error would
    // grow like a polynomial of degree ord - 1 in the number of levels.  So a position that converges
    // here (|r0| within the block tolerance, which the exact slots make an exact test) still gets
    // one FP64 residual pass, which writes its slot from B_n x itself.
    //
    // Forward substitution (Sec. 5.1): level sl solves (e_0 D_1 + c_s D_2 B_n) v = rhat, i.e.
    // (dvec + c_s B_n) v = rhat / gamma2 with rhat = r^(sl) - D_1 sum_{m<sl} e_{sl-m} v^(m); the
    // f block solves c_f D_2^(S) B_n f = r_f - v^(S).  Transposed: with w = D_2 lam, level sl
    // solves (dvec + c_s B_n) w = r^(sl) - sum_{m>sl} e_{m-sl} dvec^(m) w^(m) - [last level] lam_f
    // (D_1 lam = dvec w since e_0 = 1) and the f block B_n w_f = r_f / c_f; lam = w / gamma2 at
    // the end.
    const double cc = fblock ? 1.0 : a.cs;
    const double* d64 = fblock ? a.zero64 : a.dvec64 + (long long)sl * N;
    const bool r0_here = (a.mode == 0 && a.warm && a.block_solver == 0);
    const int pos = fblock ? S : (a.trans ? S - 1 - sl : sl);  // position in processing order
    // levels the guess combines: at most warm, and 1 + pos / 4 near the start of the substitution,
    // where the solution of a fractional problem is least smooth in time (about t^beta at t = 0)
    const int ord = fblock ? 0 : min(min(a.warm, pos), 1 + pos / 4);
    const int dl = a.trans ? 1 : -1;  // level of the previous position: sl + dl
    // x0 = sum_{k=1..ord} c_k y(position p - k), c_k = (-1)^(k+1) C(ord, k): the polynomial of
    // degree ord - 1 through the last ord levels, evaluated one step further
    double cw[kMaxWarm];
#pragma unroll
    for (int q = 0; q < kMaxWarm; ++q) cw[q] = kExtrap.c[ord][q];
    double* bxs = a.lBx + (long long)(pos % kMaxWarm) * N;  // this position's slot
    double bb = 0.0, rr = 0.0, rr1 = 0.0;
    for (long long j = gtid; j < N; j += gstride) {
      double bj;
      if (fblock) {
        bj = a.trans ? a.r[(long long)S * N + j] / a.cf
                     : (a.r[(long long)S * N + j] - a.y[(long long)(S - 1) * N + j]) /
                           (a.cf * a.g2[(long long)(S - 1) * N + j]);
      } else if (!a.trans) {
        // rhat / gamma2 with rhat = r^(sl) - D_1 sum_{m<sl} e_{sl-m} y^(m)
        const long long o = (long long)sl * N + j;
        bj = (a.r[o] - a.g1[o] * history(a, sl, j)) / a.g2[o];
      } else {
        // r^(sl) - sum_{m>sl} e_{m-sl} dvec^(m) w^(m) - [sl = S-1] lam_f
        bj = a.r[(long long)sl * N + j] - history(a, S - 1 - sl, j);
        if (sl == S - 1) bj -= a.y[(long long)S * N + j] / a.g2[(long long)(S - 1) * N + j];
      }
      // the extrapolation's loads first (independent), then the sums in a fixed order
      double yv[kMaxWarm], bv[kMaxWarm];
#pragma unroll
      for (int q = 1; q <= kMaxWarm; ++q) {
        const bool in = q <= ord;
        yv[q - 1] = in ? a.y[(long long)(sl + q * dl) * N + j] : 0.0;
        bv[q - 1] = (in && r0_here) ? a.lBx[(long long)((pos - q) % kMaxWarm) * N + j] : 0.0;
      }
      double x0 = 0.0, bx = 0.0;
#pragma unroll
      for (int q = 0; q < kMaxWarm; ++q) {
        if (q >= ord) break;
        x0 = fma(cw[q], yv[q], x0);
        if (r0_here) bx = fma(cw[q], bv[q], bx);
      }
      a.lb[j] = bj;
      x64[j] = x0;
      if (a.mode != 0) {
        // FP32 right-hand side and initial guess of the mixed-mode CG (the FP64 mode's CG solves
        // for a correction from x = 0 with r = the FP64 residual)
        a.lb32[j] = (float)bj;
        a.lx32[j] = (float)x0;
      }
      if (!a.warm) a.lr32[j] = (float)bj;
      if (r0_here) {
        bxs[j] = bx;
        const double dj = d64[j];
        const double rj = bj - fma(dj, x0, cc * bx);
        a.lr32[j] = (float)rj;
        rr = fma(rj, rj, rr);
        if (ord >= 2) {
          // residual of the previous level as the guess (order 1), to fall back on
          const double r1 = bj - fma(dj, yv[0], cc * bv[0]);
          rr1 = fma(r1, r1, rr1);
        }
      }
      bb = fma(bj, bj, bb);
    }
    set_phase(k, PH_RHS);
    int ord_used = ord;
    {
      double tot[3];
      const double sums[3] = {bb, rr, rr1};
      if (!reduce_syncN<3>(k, sums, tot)) { ok = false; break; }
      // The extrapolated guess is kept unless the previous level (order 1) or zero leaves a smaller
      // first residual: a level whose solution breaks the smooth trend (a sign change, a level far
      // smaller than its neighbours) would otherwise start far off, and an x0 much larger than the
      // solution would also leave FP64 rounding of |x0| in its residual.
      if (threadIdx.x == 0) {
        s_fix = 0;
        if (r0_here && ord >= 2) {
          if (tot[0] < tot[1] && tot[0] <= tot[2]) s_fix = 2;
          else if (tot[2] < tot[1]) s_fix = 1;
          if (s_fix) tot[1] = (s_fix == 1) ? tot[2] : tot[0];
          s_red[0] = tot[1];
        }
      }
      __syncthreads();
      if (r0_here && ord >= 2 && s_fix) {
        // rewrite the guess (same nodes, same threads): x0 = y(p - 1) or 0 with its slot and residual
        const int fx = s_fix;
        const double* yp = a.y + (long long)(sl + dl) * N;
        const double* bp = a.lBx + (long long)((pos - 1) % kMaxWarm) * N;
        for (long long j = gtid; j < N; j += gstride) {
          const double x0 = (fx == 1) ? yp[j] : 0.0;
          const double bx = (fx == 1) ? bp[j] : 0.0;
          x64[j] = x0;
          bxs[j] = bx;
          a.lr32[j] = (float)(a.lb[j] - fma(d64[j], x0, cc * bx));
        }
        ord_used = (fx == 1) ? 1 : 0;
        if (threadIdx.x == 0) s_fixes += 1;
        if (!grid_sync(k)) { ok = false; break; }
        tot[1] = s_red[0];
      }
      if (threadIdx.x == 0 && !a.warm) {
        // residual of the zero initial guess
        const double tol2 = (a.mode == 0) ? a.tol2_outer : a.tol2_mixed;
        Scalars* s0 = (a.mode == 0) ? outer : inner;
        s0->bnorm2 = tot[0];
        s0->rnorm2 = tot[0];
        s0->tol2 = tol2;
        s0->done = (tot[0] == 0.0);
        if (a.mode == 0) {
          inner->done = outer->done;
          inner->bnorm2 = tot[0];
          inner->tol2 = a.tol2_inner;
        }
      }
      if (threadIdx.x == 0 && r0_here) {
        // first refinement residual: the finalisation of a residual pass (first sweep)
        outer->tol2 = a.tol2_outer;
        RowIO<double> f;
        f.st = ST_RESID_REFINE;
        f.first = 1;
        f.sc = outer;
        f.sc2 = inner;
        f.inner_tol2 = a.tol2_inner;
        io_finalize(f, false, true, tot);
        outer->sweeps -= 1;  // the counter counts FP64 B_n applies; this residual needed none
      }
      __syncthreads();
    }
    const float c32 = (float)cc;
    const float* d32 = fblock ? a.zero32 : a.dvec32 + (long long)sl * N;
    const float dbar = fblock ? 0.0f : a.dbar32[sl];
    const CgVec V32{a.lx32, a.lr32, a.lp32, a.lq32, a.lz32, a.t1_32, a.ltr32, a.ltq32, a.t2_32,
                    a.w32z, a.w32p, a.w32a, a.w32b, d32};

    if (a.block_solver == 2) {
      // ---- S_{n,S} (Remark 1): one Fourier solve with (dbar I + c s(B_n)) -------------------
      if (a.mode == 0) {
        const SPlan<double> Q64{a.sch64, a.sbh64, a.slam64};
        if (!strang_field<double, L>(k, a.lb, x64, P64, Q64, fblock ? 0.0 : a.dbar64[sl], cc, buf64)) {
          ok = false;
          break;
        }
      } else {
        const SPlan<float> Q32{a.sch32, a.sbh32, a.slam32};
        if (!strang_field<float, L>(k, a.lb32, a.lx32, P32, Q32, dbar, c32, buf32)) { ok = false; break; }
        for (long long j = gtid; j < N; j += gstride) x64[j] = (double)a.lx32[j];
        set_phase(k, PH_CAST);
        if (!grid_sync(k)) { ok = false; break; }
      }
      continue;
    }
    if (a.block_solver == 1) {
      // ---- T_{n,S} (Remark 1): one sine-transform solve with (dbar I + c tau(B_n)) ----------
      if (a.mode == 0) {
        RowIO<double> t;
        t.src = a.lb;
        t.dst = x64;
        if (!tau_field<double, L>(k, t, P64, fblock ? 0.0 : a.dbar64[sl], cc, buf64)) { ok = false; break; }
      } else {
        RowIO<float> t;
        t.src = a.lb32;
        t.dst = a.lx32;
        if (!tau_field<float, L>(k, t, P32, dbar, c32, buf32)) { ok = false; break; }
        for (long long j = gtid; j < N; j += gstride) x64[j] = (double)a.lx32[j];
        set_phase(k, PH_CAST);
        if (!grid_sync(k)) { ok = false; break; }
      }
      continue;
    }

    if (a.mode == 0) {
      // ---- FP64 block solve: FP32 tau-CG corrections inside FP64 refinement -------------
      // a block that converged at its first residual still refreshes its B_n x slot (see above)
      const bool verify = r0_here && ord_used >= 2 && outer->done;
      for (int sweep = 0; sweep <= a.refine_max && ok; ++sweep) {
        if (sweep > 0 || verify) {
        RowIO<double> r64;
        r64.ld = (sweep > 0) ? LD_X_UPDATE : LD_PLAIN;
        r64.src = x64;
        r64.x = x64;
        r64.dx32 = a.lx32;
        r64.st = ST_RESID_REFINE;
        r64.b = a.lb;
        r64.dvec = d64;
        r64.c = cc;
        r64.r32 = a.lr32;
        r64.bx = bxs;
        r64.inner_tol2 = a.tol2_inner;
        r64.sc = outer;
        r64.sc2 = inner;
        if (!bapply_field<double, L>(k, r64, P64, buf64)) { ok = false; break; }
        }
        if (outer->done || sweep == a.refine_max) break;
        if (a.fused) {
          if (!cg_fused<L>(k, V32, P32, dbar, c32, a.pcg_iters, true, inner, buf32)) { ok = false; break; }
        } else {
        RowIO<float> t0;
        t0.src = a.lr32;
        t0.st = ST_RZ_FIRST;
        t0.dst = a.lz32;
        t0.p = a.lp32;
        t0.x = a.lx32;
        t0.r = a.lr32;
        t0.sc = inner;
        if (!tau_field<float, L>(k, t0, P32, dbar, c32, buf32)) { ok = false; break; }
        for (int it = 0; it < a.pcg_iters && !inner->done; ++it) {
          RowIO<float> b1;
          b1.ld = (it == 0) ? LD_PLAIN : LD_P_UPDATE;
          b1.src = (it == 0) ? a.lp32 : a.lz32;
          b1.p = a.lp32;
          b1.st = ST_PCG_Q;
          b1.dvec = d32;
          b1.c = c32;
          b1.qout = a.lq32;
          b1.sc = inner;
          if (!bapply_field<float, L>(k, b1, P32, buf32)) { ok = false; break; }
          if (inner->done) break;
          RowIO<float> t1;
          t1.ld = LD_PCG_UPDATE;
          t1.x = a.lx32;
          t1.p = a.lp32;
          t1.r = a.lr32;
          t1.q = a.lq32;
          t1.st = ST_RZ_BETA;
          t1.dst = a.lz32;
          t1.sc = inner;
          if (!tau_field<float, L>(k, t1, P32, dbar, c32, buf32)) { ok = false; break; }
        }
        if (!ok) break;
        }
      }
      if (threadIdx.x == 0 && !outer->done) s_fails[0] += 1;
    } else {
      // ---- mixed precision: one FP32 tau-CG solve -----------------------------------------
      if (threadIdx.x == 0 && a.warm) {
        inner->done = 0;
        inner->tol2 = a.tol2_mixed;
      }
      __syncthreads();
      if (a.warm) {
      RowIO<float> r0;
      r0.src = a.lx32;
      r0.st = ST_RESID;
      r0.b = a.lb32;
      r0.x = a.lx32;
      r0.dvec = d32;
      r0.c = c32;
      r0.r = a.lr32;
      r0.sc = inner;
      if (!bapply_field<float, L>(k, r0, P32, buf32)) { ok = false; break; }
      }
      if (!inner->done && a.fused) {
        if (!cg_fused<L>(k, V32, P32, dbar, c32, a.pcg_max, false, inner, buf32)) { ok = false; break; }
      } else if (!inner->done) {
        RowIO<float> t0;
        t0.src = a.lr32;
        t0.st = ST_RZ_FIRST;
        t0.dst = a.lz32;
        t0.p = a.lp32;
        t0.r = a.lr32;
        t0.sc = inner;
        if (!tau_field<float, L>(k, t0, P32, dbar, c32, buf32)) { ok = false; break; }
        for (int it = 0; it < a.pcg_max && !inner->done; ++it) {
          RowIO<float> b1;
          b1.ld = (it == 0) ? LD_PLAIN : LD_P_UPDATE;
          b1.src = (it == 0) ? a.lp32 : a.lz32;
          b1.p = a.lp32;
          b1.st = ST_PCG_Q;
          b1.dvec = d32;
          b1.c = c32;
          b1.qout = a.lq32;
          b1.sc = inner;
          if (!bapply_field<float, L>(k, b1, P32, buf32)) { ok = false; break; }
          if (inner->done) break;
          RowIO<float> t1;
          t1.ld = LD_PCG_UPDATE;
          t1.x = a.lx32;
          t1.p = a.lp32;
          t1.r = a.lr32;
          t1.q = a.lq32;
          t1.st = ST_RZ_BETA;
          t1.dst = a.lz32;
          t1.sc = inner;
          if (!tau_field<float, L>(k, t1, P32, dbar, c32, buf32)) { ok = false; break; }
        }
      }
      if (!ok) break;
      if (threadIdx.x == 0 && !inner->done) s_fails[1] += 1;
      for (long long j = gtid; j < N; j += gstride) x64[j] = (double)a.lx32[j];
      set_phase(k, PH_CAST);
      if (!grid_sync(k)) { ok = false; break; }
    }
  }
  if (ok && a.trans) {
    // lam = w / gamma2 (every level's w is final and visible after the last barrier)
    const long long U = (long long)(S + 1) * N;
    for (long long i = gtid; i < U; i += gstride) {
      const long long s = i / N;
      a.y[i] /= a.g2[(s < S ? s : S - 1) * N + (i - s * N)];
    }
  }
  if (s_k.bid == 0 && threadIdx.x == 0) {
    if (a.trace_len) *a.trace_len = s_k.tn;
    a.stats[0].fails += s_fails[0];
    a.stats[0].fallbacks += s_fixes;
    a.stats[1].fails += s_fails[1];
    a.stats[0].sweeps += outer->sweeps;
    a.stats[1].sweeps += inner->sweeps;
    a.stats[0].iters += outer->iters;
    a.stats[1].iters += inner->iters;
  }
}

// One launch serves a batch of instances with the same transform length: CTA blockIdx.x works
// on instance blockIdx.x / gper, as block blockIdx.x mod gper of that instance's sub-grid.
template <int L>
__global__ void __launch_bounds__(LG<L>::BLOCK) k_fsub(FsubBatch batch) {
  const int inst = blockIdx.x / batch.gper;
  fsub_body<L>(batch.args + inst, batch.gper, (int)blockIdx.x - inst * batch.gper);
}

// Dynamic shared memory of fsub_body<L> in a CTA of `threads` threads: the line buffers of its
// groups, then the twiddle tables.
template <int L>
constexpr size_t fsub_smem(int threads) {
  return (size_t)(threads / LG<L>::NT) * LG<L>::LS * sizeof(double2) + (size_t)L * (sizeof(double2) + sizeof(float2));
}

template <int L>
cudaError_t launch_L(const FsubBatch& b, cudaStream_t st) {
  constexpr int BLOCK = LG<L>::BLOCK;
  const size_t smem = fsub_smem<L>(BLOCK);
  auto kern = k_fsub<L>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  FsubBatch args = b;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(b.count * b.gper), dim3(BLOCK), params, smem, st);
}

template <int L>
int max_grid_L(int sms) {
  constexpr int BLOCK = LG<L>::BLOCK;
  const size_t smem = fsub_smem<L>(BLOCK);
  auto kern = k_fsub<L>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BLOCK, smem) != cudaSuccess) return 0;
  return per * sms;
}

}  // namespace

}  // namespace tsfde
