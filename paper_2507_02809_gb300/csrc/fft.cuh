// Shared-memory Stockham FFT for one line of power-of-two length L (8 <= L <= 4096).
//
// A line lives in shared memory as L complex values (padded, see PBuf).  NT = L / 8 threads work on it;
// every stage reads each thread's butterfly inputs into registers, synchronises,
// then writes the outputs in Stockham (self-sorting) order, so no bit reversal is
// needed.  Stage radices are 8 while at least 8 remain, then one radix-4 or radix-2
// stage.  For a stage of radix R after sub-transforms of size Ns, butterfly j takes
// x[j + r L/R] (r < R), multiplies input r by W_{Ns R}^{r (j mod Ns)}, does a length-R
// DFT and writes output q to (j div Ns) Ns R + (j mod Ns) + q Ns.
//
// DIR = -1 is the forward transform X_k = sum_j x_j exp(-2 pi i jk / L); DIR = +1 the
// unnormalised inverse.  Twiddles come from a table tw[k] = exp(-2 pi i k / L), k < L,
// built on the host in long double: a butterfly loads W^(j mod Ns) once and forms the
// other powers it needs by complex products (at most 3 products deep, an error of a few
// units in the last place); the inverse uses the conjugates.
//
// All threads of the CTA must call these routines together (they contain
// __syncthreads), also threads whose line is a padding line.
#pragma once

#include "common.cuh"

namespace tsfde {

// Synchronisation used between FFT stages: the whole CTA, one named barrier per line group
// (groups of NT >= 32 threads aligned to warps), or the warp (groups smaller than a warp,
// where every group of the warp runs the same stages).
struct SyncCTA {
  TSFDE_D void operator()() const { __syncthreads(); }
};
struct SyncNamed {
  int id, nthreads;
  TSFDE_D void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory"); }
};
struct SyncWarp {
  TSFDE_D void operator()() const { __syncwarp(); }
};

// A line of L complex values in shared memory with one padding slot after every 8 entries, so
// that the strided writes of the Stockham stages (stride 8 and 64 entries) fall in distinct
// banks.  line_stride(L) is the number of complex slots a padded line occupies.
__host__ __device__ constexpr int line_stride(int L) { return L + (L >> 3) + 1; }
template <typename R>
struct PBuf {
  cx<R>* p;
  TSFDE_D cx<R>& operator[](int i) const { return p[i + (i >> 3)]; }
};

template <typename R, int DIR>
TSFDE_D void dft2(cx<R>& a, cx<R>& b) {
  cx<R> t = a;
  a = cadd<R>(t, b);
  b = csub<R>(t, b);
}

// In-place length-4 DFT: (v0, v1, v2, v3) -> (X0, X1, X2, X3).
template <typename R, int DIR>
TSFDE_D void dft4(cx<R>& v0, cx<R>& v1, cx<R>& v2, cx<R>& v3) {
  cx<R> t0 = cadd<R>(v0, v2), t1 = csub<R>(v0, v2);
  cx<R> t2 = cadd<R>(v1, v3), t3 = mul_i<R, DIR>(csub<R>(v1, v3));
  v0 = cadd<R>(t0, t2);
  v2 = csub<R>(t0, t2);
  v1 = cadd<R>(t1, t3);
  v3 = csub<R>(t1, t3);
}

// In-place length-8 DFT, natural order in and out.
template <typename R, int DIR>
TSFDE_D void dft8(cx<R>* v) {
  const R s = R(0.70710678118654752440084436210484903928483593768847);
  cx<R> a0 = cadd<R>(v[0], v[4]), b0 = csub<R>(v[0], v[4]);
  cx<R> a1 = cadd<R>(v[1], v[5]), b1 = csub<R>(v[1], v[5]);
  cx<R> a2 = cadd<R>(v[2], v[6]), b2 = csub<R>(v[2], v[6]);
  cx<R> a3 = cadd<R>(v[3], v[7]), b3 = csub<R>(v[3], v[7]);
  // b_r *= W8^r  (W8 = exp(DIR i pi / 4))
  if (DIR < 0) {
    b1 = mk<R>((b1.x + b1.y) * s, (b1.y - b1.x) * s);
    b3 = mk<R>((b3.y - b3.x) * s, -(b3.x + b3.y) * s);
  } else {
    b1 = mk<R>((b1.x - b1.y) * s, (b1.x + b1.y) * s);
    b3 = mk<R>(-(b3.x + b3.y) * s, (b3.x - b3.y) * s);
  }
  b2 = mul_i<R, DIR>(b2);
  dft4<R, DIR>(a0, a1, a2, a3);
  dft4<R, DIR>(b0, b1, b2, b3);
  v[0] = a0; v[2] = a1; v[4] = a2; v[6] = a3;
  v[1] = b0; v[3] = b1; v[5] = b2; v[7] = b3;
}

template <typename R, int RAD, int DIR>
TSFDE_D void dft_rad(cx<R>* v) {
  if constexpr (RAD == 8) dft8<R, DIR>(v);
  else if constexpr (RAD == 4) dft4<R, DIR>(v[0], v[1], v[2], v[3]);
  else dft2<R, DIR>(v[0], v[1]);
}

template <typename R, int L, int DIR, int NS, int RAD, class SYNC>
TSFDE_D void fft_stage(PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  constexpr int NT = L / 8;
  constexpr int NB = L / RAD;
  constexpr int PER = NB / NT;
  constexpr int TWS = L / (NS * RAD);
  cx<R> v[PER][RAD];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * NT;
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[b][r] = buf[j + r * NB];
  }
  sync();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * NT;
    const int k = j & (NS - 1);
    if constexpr (NS > 1) {
      // one table load (W^k, from global or shared memory), the other powers by products
      cx<R> w[RAD];
      w[1] = tw[k * TWS];
      if constexpr (RAD >= 4) {
        w[2] = cmul<R>(w[1], w[1]);
        w[3] = cmul<R>(w[2], w[1]);
      }
      if constexpr (RAD == 8) {
        w[4] = cmul<R>(w[2], w[2]);
        w[5] = cmul<R>(w[4], w[1]);
        w[6] = cmul<R>(w[3], w[3]);
        w[7] = cmul<R>(w[4], w[3]);
      }
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[b][r] = (DIR < 0) ? cmul<R>(v[b][r], w[r]) : cmulc<R>(v[b][r], w[r]);
    }
    dft_rad<R, RAD, DIR>(v[b]);
    const int base = (j / NS) * NS * RAD + k;
#pragma unroll
    for (int q = 0; q < RAD; ++q) buf[base + q * NS] = v[b][q];
  }
  sync();
}

template <typename R, int L, int DIR, int NS, class SYNC>
TSFDE_D void fft_stages(PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  if constexpr (NS < L) {
    constexpr int REM = L / NS;
    constexpr int RAD = REM >= 8 ? 8 : REM;
    fft_stage<R, L, DIR, NS, RAD>(buf, tw, t, sync);
    fft_stages<R, L, DIR, NS * RAD>(buf, tw, t, sync);
  }
}

// Transform the line in `buf` (L entries) in place.  t in [0, L/8).
template <typename R, int L, int DIR, class SYNC = SyncCTA>
TSFDE_D void fft_line(PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync = SYNC()) {
  static_assert(L >= 8 && (L & (L - 1)) == 0, "power-of-two length >= 8");
  fft_stages<R, L, DIR, 1>(buf, tw, t, sync);
}

// ---- register-resident form -----------------------------------------------------------------
// Thread t of a line group owns the 8 positions t + m NT (m < 8).  A Stockham transform whose
// first stage has radix 8 reads exactly these positions in its first butterfly, and its last
// stage writes its outputs to these positions again (output q of butterfly b lands at
// t + (b + q PER) NT).  fft_regs therefore takes and returns the 8 values in registers and uses
// shared memory only for the exchanges between stages.

template <typename R, int L, int DIR, int NS, class SYNC>
TSFDE_D void fft_mid_stages(PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  constexpr int REM = L / NS;
  constexpr int RAD = REM >= 8 ? 8 : REM;
  if constexpr (NS * RAD < L) {
    fft_stage<R, L, DIR, NS, RAD>(buf, tw, t, sync);
    fft_mid_stages<R, L, DIR, NS * RAD>(buf, tw, t, sync);
  }
}

template <int L>
__host__ __device__ constexpr int last_stage_ns() {
  int ns = 1;
  while (true) {
    const int rem = L / ns, rad = rem >= 8 ? 8 : rem;
    if (ns * rad >= L) return ns;
    ns *= rad;
  }
}

// In-place transform of the thread's 8 values (positions t + m NT).  Ends with a
// synchronisation, so the caller may reuse `buf` at once.
template <typename R, int L, int DIR, class SYNC>
TSFDE_D void fft_regs(cx<R> (&v)[8], PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  static_assert(L >= 8 && (L & (L - 1)) == 0, "power-of-two length >= 8");
  dft8<R, DIR>(v);  // first stage: Ns = 1, butterfly t, no twiddles
  if constexpr (L > 8) {
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[8 * t + q] = v[q];
    sync();
    fft_mid_stages<R, L, DIR, 8>(buf, tw, t, sync);
    constexpr int NS = last_stage_ns<L>();
    constexpr int RAD = L / NS, NT = L / 8, NB = L / RAD, PER = NB / NT, TWS = L / (NS * RAD);
    cx<R> u[PER][RAD];
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int j = t + b * NT;
#pragma unroll
      for (int r = 0; r < RAD; ++r) u[b][r] = buf[j + r * NB];
    }
    sync();
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int j = t + b * NT;
      const int k = j & (NS - 1);
      cx<R> w[RAD];
      w[1] = tw[k * TWS];
      if constexpr (RAD >= 4) {
        w[2] = cmul<R>(w[1], w[1]);
        w[3] = cmul<R>(w[2], w[1]);
      }
      if constexpr (RAD == 8) {
        w[4] = cmul<R>(w[2], w[2]);
        w[5] = cmul<R>(w[4], w[1]);
        w[6] = cmul<R>(w[3], w[3]);
        w[7] = cmul<R>(w[4], w[3]);
      }
#pragma unroll
      for (int r = 1; r < RAD; ++r) u[b][r] = (DIR < 0) ? cmul<R>(u[b][r], w[r]) : cmulc<R>(u[b][r], w[r]);
      dft_rad<R, RAD, DIR>(u[b]);
#pragma unroll
      for (int q = 0; q < RAD; ++q) v[b + q * PER] = u[b][q];
    }
  }
}

// ---- register-resident form on L / 4 threads (four values per thread) ----------------------
// The same Stockham transform with radix-4 stages (one radix-2 stage last when log2 L is odd), run
// by L / 4 threads that own the 4 positions t + m (L/4) each.  Every thread does half the arithmetic
// of the eight-value form, at the price of more exchanges: for FP64 lines, whose instructions each
// hold an SM sub-partition's narrow FP64 pipe for many cycles, spreading a line over twice the warps
// halves its time when the lines of a pass leave sub-partitions idle.

template <typename R, int L, int DIR, int NS, int RAD, int NTH, class SYNC>
TSFDE_D void fft_stage_nt(PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  constexpr int NB = L / RAD;
  constexpr int PER = NB / NTH;
  static_assert(PER >= 1 && NB % NTH == 0, "butterflies spread evenly over the threads");
  constexpr int TWS = L / (NS * RAD);
  cx<R> v[PER][RAD];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * NTH;
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[b][r] = buf[j + r * NB];
  }
  sync();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * NTH;
    const int k = j & (NS - 1);
    cx<R> w[RAD];
    w[1] = tw[k * TWS];
    if constexpr (RAD >= 4) {
      w[2] = cmul<R>(w[1], w[1]);
      w[3] = cmul<R>(w[2], w[1]);
    }
#pragma unroll
    for (int r = 1; r < RAD; ++r) v[b][r] = (DIR < 0) ? cmul<R>(v[b][r], w[r]) : cmulc<R>(v[b][r], w[r]);
    dft_rad<R, RAD, DIR>(v[b]);
    const int base = (j / NS) * NS * RAD + k;
#pragma unroll
    for (int q = 0; q < RAD; ++q) buf[base + q * NS] = v[b][q];
  }
  sync();
}

template <typename R, int L, int DIR, int NS, class SYNC>
TSFDE_D void fft_mid_stages4(PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  constexpr int REM = L / NS;
  constexpr int RAD = REM >= 4 ? 4 : REM;
  if constexpr (NS * RAD < L) {
    fft_stage_nt<R, L, DIR, NS, RAD, L / 4>(buf, tw, t, sync);
    fft_mid_stages4<R, L, DIR, NS * RAD>(buf, tw, t, sync);
  }
}

template <int L>
__host__ __device__ constexpr int last_stage_ns4() {
  int ns = 1;
  while (true) {
    const int rem = L / ns, rad = rem >= 4 ? 4 : rem;
    if (ns * rad >= L) return ns;
    ns *= rad;
  }
}

// In-place transform of the thread's 4 values (positions t + m L/4, t < L/4).  Ends with a
// synchronisation, so the caller may reuse `buf` at once.
template <typename R, int L, int DIR, class SYNC>
TSFDE_D void fft_regs4(cx<R> (&v)[4], PBuf<R> buf, const cx<R>* __restrict__ tw, int t, SYNC sync) {
  static_assert(L >= 8 && (L & (L - 1)) == 0, "power-of-two length >= 8");
  dft4<R, DIR>(v[0], v[1], v[2], v[3]);  // first stage: Ns = 1, butterfly t, no twiddles
#pragma unroll
  for (int q = 0; q < 4; ++q) buf[4 * t + q] = v[q];
  sync();
  fft_mid_stages4<R, L, DIR, 4>(buf, tw, t, sync);
  constexpr int NS = last_stage_ns4<L>();
  constexpr int RAD = L / NS, NT = L / 4, NB = L / RAD, PER = NB / NT, TWS = L / (NS * RAD);
  cx<R> u[PER][RAD];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * NT;
#pragma unroll
    for (int r = 0; r < RAD; ++r) u[b][r] = buf[j + r * NB];
  }
  sync();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * NT;
    const int k = j & (NS - 1);
    cx<R> w[RAD];
    w[1] = tw[k * TWS];
    if constexpr (RAD >= 4) {
      w[2] = cmul<R>(w[1], w[1]);
      w[3] = cmul<R>(w[2], w[1]);
    }
#pragma unroll
    for (int r = 1; r < RAD; ++r) u[b][r] = (DIR < 0) ? cmul<R>(u[b][r], w[r]) : cmulc<R>(u[b][r], w[r]);
    dft_rad<R, RAD, DIR>(u[b]);
#pragma unroll
    for (int q = 0; q < RAD; ++q) v[b + q * PER] = u[b][q];
  }
}

}  // namespace tsfde
