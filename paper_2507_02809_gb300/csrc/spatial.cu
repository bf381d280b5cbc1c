// Spatial operators of the all-at-once system on a power-of-two transform grid L >= 2 (n + 1)
// (the tau kernels below need L = 2 (n + 1); the persistent kernel handles padded grids):
//   * B_n x for a batch of fields: B_n is the d-level symmetric Toeplitz matrix with
//     entries a_{i-j} (Sec. 5 after Eq. 10), applied by embedding each level in a
//     circulant of size L and using the FFT (Sec. 5, matvec step 1(b)).  Real rows are
//     transformed two at a time as one complex line; the last axis keeps the half
//     spectrum (L/2 + 1 values); the first axis does forward FFT, symbol multiply and
//     inverse FFT in one pass; all-zero padding lines are never transformed.
//   * tau(B_n)^-1-type solves (dbar I + c tau(B_n))^-1 x, where tau(B_n) = S diag(mu) S
//     with the orthonormal DST-I matrix S (Bini-Di Benedetto tau matrix, Remark 1).  The
//     DST-I of two real lines is the imaginary / real part of one complex FFT of length
//     2 (n + 1) of their odd extensions.
//   * setup transforms: the circulant symbol and the tau eigenvalues from the coefficient
//     table a_l, and the d >= 2 coefficient table itself (K-point trapezoid rule of Eq. 8).
#include <math.h>
#include <stdio.h>

#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "rowio.cuh"

namespace tsfde {

// ----------------------------------------------------------------------------------
// Row kernels.  A block handles LPB line groups (NT = L/8 threads each), and loops over
// groups of row pairs with a grid stride; the fused load / store work of RowIO and its
// reductions are done in the same pass.
// ----------------------------------------------------------------------------------
template <typename R>
TSFDE_D void io_reduce_finalize(const RowIO<R>& io, bool do_load, bool do_store, const double* acc) {
  if ((do_load && io.reduces_load()) || (do_store && io.reduces_store())) {
    double tot[2];
    if (io_grid_reduce2(acc[0], acc[1], io.rw, tot) && threadIdx.x == 0) io_finalize(io, do_load, do_store, tot);
  }
}

// d = 1: fused forward FFT, symbol multiply, inverse FFT for pairs of fields.
template <typename R, int L, int LPB>
__global__ void __launch_bounds__(LPB * (L / 8))
k_bapply_1d(int F, int n, const R* __restrict__ lam, const cx<R>* __restrict__ tw, RowIO<R> io) {
  if (io.skip && *io.skip) return;
  constexpr int NT = L / 8, LS = line_stride(L);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PBuf<R> buf{reinterpret_cast<cx<R>*>(smem_raw) + (threadIdx.x / NT) * LS};
  const int t = threadIdx.x % NT;
  double acc[2] = {0.0, 0.0};
  const long long ngroups = ((long long)(F + 1) / 2 + LPB - 1) / LPB;
  for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const long long pair = g * LPB + threadIdx.x / NT;
    const long long f0 = 2 * pair, f1 = f0 + 1;
    for (int p = t; p < L; p += NT) {
      R a = (p < n && f0 < F) ? io_load(io, f0 * n + p, acc) : R(0);
      R b = (p < n && f1 < F) ? io_load(io, f1 * n + p, acc) : R(0);
      buf[p] = mk<R>(a, b);
    }
    __syncthreads();
    fft_line<R, L, -1>(buf, tw, t);
    for (int p = t; p < L; p += NT) buf[p] = cscale<R>(buf[p], lam[p <= L / 2 ? p : L - p]);
    __syncthreads();
    fft_line<R, L, 1>(buf, tw, t);
    for (int p = t; p < n; p += NT) {
      cx<R> v = buf[p];
      if (f0 < F) io_store(io, f0 * n + p, v.x, acc);
      if (f1 < F) io_store(io, f1 * n + p, v.y, acc);
    }
    __syncthreads();
  }
  io_reduce_finalize(io, true, true, acc);
}

// Last axis (contiguous rows of n reals), forward: half spectra of two rows per line.
template <typename R, int L, int LPB>
__global__ void __launch_bounds__(LPB * (L / 8))
k_rowfwd(cx<R>* __restrict__ out, long long NR, int n, int H, const cx<R>* __restrict__ tw, RowIO<R> io) {
  if (io.skip && *io.skip) return;
  constexpr int NT = L / 8, LS = line_stride(L);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PBuf<R> buf{reinterpret_cast<cx<R>*>(smem_raw) + (threadIdx.x / NT) * LS};
  const int t = threadIdx.x % NT;
  double acc[2] = {0.0, 0.0};
  const long long ngroups = ((NR + 1) / 2 + LPB - 1) / LPB;
  for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const long long pair = g * LPB + threadIdx.x / NT;
    const long long r0 = 2 * pair, r1 = r0 + 1;
    for (int p = t; p < L; p += NT) {
      R a = (p < n && r0 < NR) ? io_load(io, r0 * n + p, acc) : R(0);
      R b = (p < n && r1 < NR) ? io_load(io, r1 * n + p, acc) : R(0);
      buf[p] = mk<R>(a, b);
    }
    __syncthreads();
    fft_line<R, L, -1>(buf, tw, t);
    for (int k = t; k < H; k += NT) {
      cx<R> zk = buf[k], zm = buf[(L - k) & (L - 1)];
      // X = (Z_k + conj Z_{-k}) / 2,  Y = (Z_k - conj Z_{-k}) / (2 i)
      cx<R> X = mk<R>(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
      cx<R> Y = mk<R>(R(0.5) * (zk.y + zm.y), R(-0.5) * (zk.x - zm.x));
      if (r0 < NR) out[r0 * H + k] = X;
      if (r1 < NR) out[r1 * H + k] = Y;
    }
    __syncthreads();
  }
  io_reduce_finalize(io, true, false, acc);
}

// Last axis, inverse: two half spectra -> one complex line -> two real rows (first n).
template <typename R, int L, int LPB>
__global__ void __launch_bounds__(LPB * (L / 8))
k_rowinv(const cx<R>* __restrict__ in, long long NR, int n, int H, const cx<R>* __restrict__ tw, RowIO<R> io) {
  if (io.skip && *io.skip) return;
  constexpr int NT = L / 8, LS = line_stride(L);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PBuf<R> buf{reinterpret_cast<cx<R>*>(smem_raw) + (threadIdx.x / NT) * LS};
  const int t = threadIdx.x % NT;
  double acc[2] = {0.0, 0.0};
  const long long ngroups = ((NR + 1) / 2 + LPB - 1) / LPB;
  for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const long long pair = g * LPB + threadIdx.x / NT;
    const long long r0 = 2 * pair, r1 = r0 + 1;
    for (int k = t; k < H; k += NT) {
      cx<R> X = (r0 < NR) ? in[r0 * H + k] : mk<R>(0, 0);
      cx<R> Y = (r1 < NR) ? in[r1 * H + k] : mk<R>(0, 0);
      buf[k] = mk<R>(X.x - Y.y, X.y + Y.x);
      if (k != 0 && k != L / 2) buf[L - k] = mk<R>(X.x + Y.y, Y.x - X.y);
    }
    __syncthreads();
    fft_line<R, L, 1>(buf, tw, t);
    for (int p = t; p < n; p += NT) {
      cx<R> v = buf[p];
      if (r0 < NR) io_store(io, r0 * n + p, v.x, acc);
      if (r1 < NR) io_store(io, r1 * n + p, v.y, acc);
    }
    __syncthreads();
  }
  io_reduce_finalize(io, false, true, acc);
}

// ----------------------------------------------------------------------------------
// Strided complex lines: line (o, i), element p at base + o*os + i + p*es.  A block takes
// TI consecutive i (adjacent in memory) of one o, so loads and stores are coalesced.
// MODE 0: load n_load (zero padded to L), forward FFT, store n_store.
// MODE 1: load n_load, forward FFT, multiply by lam[k * NI + i], inverse FFT, store n_store.
// MODE 2: load n_load, inverse FFT, store n_store.
// ----------------------------------------------------------------------------------
template <typename R, int L, int TI, int MODE>
__global__ void __launch_bounds__(TI * (L / 8))
k_cline(const cx<R>* in, cx<R>* out, int NI, long long NO, long long in_os, long long in_es,
        long long out_os, long long out_es, int n_load, int n_store, const R* __restrict__ lam,
        const cx<R>* __restrict__ tw, const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int NT = L / 8, LS = line_stride(L);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* sm = reinterpret_cast<cx<R>*>(smem_raw);
  const int tiles = (NI + TI - 1) / TI;
  const long long o = blockIdx.x / tiles;
  const int i0 = (int)(blockIdx.x % tiles) * TI;
  const int nthr = TI * NT;
  for (int idx = threadIdx.x; idx < L * TI; idx += nthr) {
    const int p = idx / TI, li = idx % TI, i = i0 + li;
    cx<R> v = mk<R>(0, 0);
    if (p < n_load && i < NI && o < NO) v = in[o * in_os + i + (long long)p * in_es];
    PBuf<R>{sm + li * LS}[p] = v;
  }
  __syncthreads();
  const int line = threadIdx.x / NT, t = threadIdx.x % NT;
  PBuf<R> buf{sm + line * LS};
  if constexpr (MODE == 2) {
    fft_line<R, L, 1>(buf, tw, t);
  } else {
    fft_line<R, L, -1>(buf, tw, t);
  }
  if constexpr (MODE == 1) {
    const int i = i0 + line;
    const int ic = i < NI ? i : NI - 1;
    for (int k = t; k < L; k += NT) buf[k] = cscale<R>(buf[k], lam[(long long)k * NI + ic]);
    __syncthreads();
    fft_line<R, L, 1>(buf, tw, t);
  }
  for (int idx = threadIdx.x; idx < n_store * TI; idx += nthr) {
    const int p = idx / TI, li = idx % TI, i = i0 + li;
    if (i < NI && o < NO) out[o * out_os + i + (long long)p * out_es] = PBuf<R>{sm + li * LS}[p];
  }
}

// ----------------------------------------------------------------------------------
// DST-I helpers.  For two real lines u, v of length n, z = odd(u) + i odd(v) with
// odd(u)_p = u_p (1 <= p <= n), -u_{L-p} (n+2 <= p < L), 0 at p = 0, n + 1.  Then
// DST(u)_k = sum_j u_j sin(pi j k / (n+1)) = -Im Z_k / 2 and DST(v)_k = Re Z_k / 2.
// ----------------------------------------------------------------------------------
template <typename R>
TSFDE_D R dst_scale(const R* mu, long long midx, const R* dbar, int field, R c, R norm) {
  R db = dbar ? dbar[field] : R(0);
  return norm / (db + c * mu[midx]);
}

// Contiguous rows (last axis).  USE_LD: the input comes from the RowIO load mode (else
// io.dst is read, in place); USE_ST: the output goes through the store mode (else io.dst).
// SCALE: forward DST, scale, DST again (d = 1 tau solve: one row per field; mu index k - 1).
template <typename R, int L, int LPB, bool SCALE, bool USE_LD, bool USE_ST>
__global__ void __launch_bounds__(LPB * (L / 8))
k_dst_rows(long long NR, int n, const R* __restrict__ mu, const R* __restrict__ dbar, R c, R norm,
           const cx<R>* __restrict__ tw, RowIO<R> io) {
  if (io.skip && *io.skip) return;
  constexpr int NT = L / 8, LS = line_stride(L);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PBuf<R> buf{reinterpret_cast<cx<R>*>(smem_raw) + (threadIdx.x / NT) * LS};
  const int t = threadIdx.x % NT;
  double acc[2] = {0.0, 0.0};
  const long long ngroups = ((NR + 1) / 2 + LPB - 1) / LPB;
  for (long long g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const long long pair = g * LPB + threadIdx.x / NT;
    const long long r0 = 2 * pair, r1 = r0 + 1;
    // odd extension: positions 1..n hold the row, L-1..n+2 its negative, 0 and n+1 zero
    for (int p = 1 + t; p <= n; p += NT) {
      R a = 0, b = 0;
      if (r0 < NR) a = USE_LD ? io_load(io, r0 * n + p - 1, acc) : io.dst[r0 * n + p - 1];
      if (r1 < NR) b = USE_LD ? io_load(io, r1 * n + p - 1, acc) : io.dst[r1 * n + p - 1];
      buf[p] = mk<R>(a, b);
      buf[L - p] = mk<R>(-a, -b);
    }
    if (t == 0) {
      buf[0] = mk<R>(0, 0);
      buf[n + 1] = mk<R>(0, 0);
    }
    __syncthreads();
    fft_line<R, L, -1>(buf, tw, t);
    if constexpr (SCALE) {
      R su[4], sv[4];
      int cnt = 0;
      for (int k = 1 + t; k <= n; k += NT, ++cnt) {
        cx<R> z = buf[k];
        R s0 = (r0 < NR) ? dst_scale<R>(mu, k - 1, dbar, (int)r0, c, norm) : R(0);
        R s1 = (r1 < NR) ? dst_scale<R>(mu, k - 1, dbar, (int)r1, c, norm) : R(0);
        su[cnt] = R(-0.5) * z.y * s0;
        sv[cnt] = R(0.5) * z.x * s1;
      }
      __syncthreads();
      cnt = 0;
      for (int k = 1 + t; k <= n; k += NT, ++cnt) {
        buf[k] = mk<R>(su[cnt], sv[cnt]);
        buf[L - k] = mk<R>(-su[cnt], -sv[cnt]);
      }
      if (t == 0) {
        buf[0] = mk<R>(0, 0);
        buf[n + 1] = mk<R>(0, 0);
      }
      __syncthreads();
      fft_line<R, L, -1>(buf, tw, t);
    }
    for (int k = 1 + t; k <= n; k += NT) {
      cx<R> z = buf[k];
      if (r0 < NR) {
        if (USE_ST) io_store(io, r0 * n + k - 1, R(-0.5) * z.y, acc);
        else io.dst[r0 * n + k - 1] = R(-0.5) * z.y;
      }
      if (r1 < NR) {
        if (USE_ST) io_store(io, r1 * n + k - 1, R(0.5) * z.x, acc);
        else io.dst[r1 * n + k - 1] = R(0.5) * z.x;
      }
    }
    __syncthreads();
  }
  io_reduce_finalize(io, USE_LD, USE_ST, acc);
}

// Strided real lines: line (o, i), element p at o*os + i + p*es; TI real lines (TI/2
// complex FFTs) per block.  SCALE: first-axis pass of a tau solve (field = o, mu index
// (k-1)*NI + i).
template <typename R, int L, int TI, bool SCALE>
__global__ void __launch_bounds__((TI / 2) * (L / 8))
k_dst_strided(const R* x, R* y, int NI, long long NO, long long os, long long es, int n,
              const R* __restrict__ mu, const R* __restrict__ dbar, R c, R norm,
              const cx<R>* __restrict__ tw, const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int NT = L / 8, LS = line_stride(L), NL = TI / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* sm = reinterpret_cast<cx<R>*>(smem_raw);
  const int tiles = (NI + TI - 1) / TI;
  const long long o = blockIdx.x / tiles;
  const int i0 = (int)(blockIdx.x % tiles) * TI;
  const int nthr = NL * NT;
  // zero the two fixed points of every line
  for (int l = threadIdx.x; l < NL; l += nthr) {
    PBuf<R> b{sm + l * LS};
    b[0] = mk<R>(0, 0);
    b[n + 1] = mk<R>(0, 0);
  }
  for (int idx = threadIdx.x; idx < n * TI; idx += nthr) {
    const int p = idx / TI + 1, li = idx % TI, i = i0 + li;
    R v = 0;
    if (i < NI && o < NO) v = x[o * os + i + (long long)(p - 1) * es];
    const int line = li >> 1, part = li & 1;
    PBuf<R> b{sm + line * LS};
    if (part) {
      b[p].y = v;
      b[L - p].y = -v;
    } else {
      b[p].x = v;
      b[L - p].x = -v;
    }
  }
  __syncthreads();
  const int line = threadIdx.x / NT, t = threadIdx.x % NT;
  PBuf<R> buf{sm + line * LS};
  fft_line<R, L, -1>(buf, tw, t);
  if constexpr (SCALE) {
    const int ia = i0 + 2 * line, ib = ia + 1;
    R su[4], sv[4];
    int cnt = 0;
    for (int k = 1 + t; k <= n; k += NT, ++cnt) {
      cx<R> z = buf[k];
      R s0 = (ia < NI) ? dst_scale<R>(mu, (long long)(k - 1) * NI + ia, dbar, (int)o, c, norm) : R(0);
      R s1 = (ib < NI) ? dst_scale<R>(mu, (long long)(k - 1) * NI + ib, dbar, (int)o, c, norm) : R(0);
      su[cnt] = R(-0.5) * z.y * s0;
      sv[cnt] = R(0.5) * z.x * s1;
    }
    __syncthreads();
    cnt = 0;
    for (int k = 1 + t; k <= n; k += NT, ++cnt) {
      buf[k] = mk<R>(su[cnt], sv[cnt]);
      buf[L - k] = mk<R>(-su[cnt], -sv[cnt]);
    }
    if (t == 0) {
      buf[0] = mk<R>(0, 0);
      buf[n + 1] = mk<R>(0, 0);
    }
    __syncthreads();
    fft_line<R, L, -1>(buf, tw, t);
  }
  for (int idx = threadIdx.x; idx < n * TI; idx += nthr) {
    const int k = idx / TI + 1, li = idx % TI, i = i0 + li;
    if (i < NI && o < NO) {
      cx<R> z = PBuf<R>{sm + (li >> 1) * LS}[k];
      y[o * os + i + (long long)(k - 1) * es] = (li & 1) ? R(0.5) * z.x : R(-0.5) * z.y;
    }
  }
}

// ----------------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------------
namespace {

template <int L> constexpr int lpb_rows() { return (L / 8) >= 32 ? 1 : 32 / (L / 8); }
// lines per block of the strided passes: 64-byte coalesced segments, at most 1024 threads
template <typename R, int L> constexpr int ti_cplx() {
  return (64 / (int)sizeof(cx<R>)) * (L / 8) <= 1024 ? 64 / (int)sizeof(cx<R>) : 1024 / (L / 8);
}
template <typename R, int L> constexpr int ti_real() {
  return (64 / (int)sizeof(R) / 2) * (L / 8) <= 1024 ? 64 / (int)sizeof(R) : 2 * (1024 / (L / 8));
}

template <typename K>
void set_smem(K kern, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R>
unsigned row_grid(long long NR, int LPB, const RowIO<R>& io, bool load_side, bool store_side) {
  long long groups = ((NR + 1) / 2 + LPB - 1) / LPB;
  const bool red = (load_side && io.reduces_load()) || (store_side && io.reduces_store());
  long long cap = red ? 4 * 152 : (1LL << 30);
  if (groups > cap) groups = cap;
  return (unsigned)(groups < 1 ? 1 : groups);
}

template <typename R, int L>
void bapply_L(const SpatialPlan<R>& P, int F, const RowIO<R>& io, cudaStream_t st) {
  constexpr int LPB = lpb_rows<L>();
  constexpr int NT = L / 8;
  constexpr int LS = line_stride(L);
  const int n = P.n, H = P.H;
  const int* skip = io.skip;
  const size_t smem_rows = (size_t)LPB * LS * sizeof(cx<R>);
  if (P.d == 1) {
    auto kern = k_bapply_1d<R, L, LPB>;
    set_smem(kern, smem_rows);
    kern<<<row_grid<R>(F, LPB, io, true, true), LPB * NT, smem_rows, st>>>(F, n, P.lam, P.tw, io);
    return;
  }
  if constexpr (L <= 2048) {
  constexpr int TI = ti_cplx<R, L>();
  const size_t smem_cl = (size_t)TI * LS * sizeof(cx<R>);
  const long long NR = (long long)F * (P.N / n);
  {
    auto kern = k_rowfwd<R, L, LPB>;
    set_smem(kern, smem_rows);
    kern<<<row_grid<R>(NR, LPB, io, true, false), LPB * NT, smem_rows, st>>>(P.work0, NR, n, H, P.tw, io);
  }
  if (P.d == 2) {
    auto kern = k_cline<R, L, TI, 1>;
    set_smem(kern, smem_cl);
    const int NI = H;
    long long blocks = (long long)F * ceil_div(NI, TI);
    kern<<<(unsigned)blocks, TI * NT, smem_cl, st>>>(P.work0, P.work0, NI, F, (long long)n * H, H,
                                                     (long long)n * H, H, n, n, P.lam, P.tw, skip);
  } else {
    // axis 1 forward: [F][n][n][H] -> [F][n][L][H]
    {
      auto kern = k_cline<R, L, TI, 0>;
      set_smem(kern, smem_cl);
      const int NI = H;
      const long long NO = (long long)F * n;
      long long blocks = NO * ceil_div(NI, TI);
      kern<<<(unsigned)blocks, TI * NT, smem_cl, st>>>(P.work0, P.work1, NI, NO, (long long)n * H, H,
                                                       (long long)L * H, H, n, L, nullptr, P.tw, skip);
    }
    // axis 0: forward, symbol, inverse, in place on [F][n][L][H]
    {
      auto kern = k_cline<R, L, TI, 1>;
      set_smem(kern, smem_cl);
      const int NI = L * H;
      long long blocks = (long long)F * ceil_div(NI, TI);
      kern<<<(unsigned)blocks, TI * NT, smem_cl, st>>>(P.work1, P.work1, NI, F, (long long)n * L * H,
                                                       (long long)L * H, (long long)n * L * H,
                                                       (long long)L * H, n, n, P.lam, P.tw, skip);
    }
    // axis 1 inverse: [F][n][L][H] -> [F][n][n][H]
    {
      auto kern = k_cline<R, L, TI, 2>;
      set_smem(kern, smem_cl);
      const int NI = H;
      const long long NO = (long long)F * n;
      long long blocks = NO * ceil_div(NI, TI);
      kern<<<(unsigned)blocks, TI * NT, smem_cl, st>>>(P.work1, P.work0, NI, NO, (long long)L * H, H,
                                                       (long long)n * H, H, L, n, nullptr, P.tw, skip);
    }
  }
  {
    auto kern = k_rowinv<R, L, LPB>;
    set_smem(kern, smem_rows);
    kern<<<row_grid<R>(NR, LPB, io, false, true), LPB * NT, smem_rows, st>>>(P.work0, NR, n, H, P.tw, io);
  }
  }
}

template <typename R, int L>
void tau_L(const SpatialPlan<R>& P, int F, const R* dbar, R c, const RowIO<R>& io, cudaStream_t st) {
  constexpr int LPB = lpb_rows<L>();
  constexpr int NT = L / 8;
  constexpr int LS = line_stride(L);
  const int n = P.n;
  const int* skip = io.skip;
  R norm = 1;
  for (int i = 0; i < P.d; ++i) norm *= R(2.0 / (n + 1));
  const size_t smem_rows = (size_t)LPB * LS * sizeof(cx<R>);
  if (P.d == 1) {
    auto kern = k_dst_rows<R, L, LPB, true, true, true>;
    set_smem(kern, smem_rows);
    kern<<<row_grid<R>(F, LPB, io, true, true), LPB * NT, smem_rows, st>>>(F, n, P.mu, dbar, c, norm, P.tw, io);
    return;
  }
  if constexpr (L <= 2048) {
  const long long NR = (long long)F * (P.N / n);
  {
    auto kern = k_dst_rows<R, L, LPB, false, true, false>;
    set_smem(kern, smem_rows);
    kern<<<row_grid<R>(NR, LPB, io, true, false), LPB * NT, smem_rows, st>>>(NR, n, nullptr, nullptr, c, norm,
                                                                          P.tw, io);
  }
  constexpr int TI = ti_real<R, L>();
  const size_t smem_s = (size_t)(TI / 2) * LS * sizeof(cx<R>);
  auto kfree = k_dst_strided<R, L, TI, false>;
  auto kscale = k_dst_strided<R, L, TI, true>;
  set_smem(kfree, smem_s);
  set_smem(kscale, smem_s);
  R* y = io.dst;
  const long long n2 = (long long)n * n;
  if (P.d == 3) {
    // axis 1: lines (o = (f, i0), i = i2)
    const long long NO = (long long)F * n;
    kfree<<<(unsigned)(NO * ceil_div(n, TI)), (TI / 2) * NT, smem_s, st>>>(y, y, n, NO, n2, n, n, nullptr,
                                                                           nullptr, c, norm, P.tw, skip);
  }
  {
    const int NI = (int)(P.N / n);
    const long long es = NI;
    kscale<<<(unsigned)((long long)F * ceil_div(NI, TI)), (TI / 2) * NT, smem_s, st>>>(
        y, y, NI, F, P.N, es, n, P.mu, dbar, c, norm, P.tw, skip);
  }
  if (P.d == 3) {
    const long long NO = (long long)F * n;
    kfree<<<(unsigned)(NO * ceil_div(n, TI)), (TI / 2) * NT, smem_s, st>>>(y, y, n, NO, n2, n, n, nullptr,
                                                                           nullptr, c, norm, P.tw, skip);
  }
  {
    auto kern = k_dst_rows<R, L, LPB, false, false, true>;
    set_smem(kern, smem_rows);
    kern<<<row_grid<R>(NR, LPB, io, false, true), LPB * NT, smem_rows, st>>>(NR, n, nullptr, nullptr, c, norm,
                                                                          P.tw, io);
  }
  }
}

}  // namespace

#define TSFDE_L_SWITCH(L, CALL)            \
  switch (L) {                             \
    case 8: CALL(8); break;                \
    case 16: CALL(16); break;              \
    case 32: CALL(32); break;              \
    case 64: CALL(64); break;              \
    case 128: CALL(128); break;            \
    case 256: CALL(256); break;            \
    case 512: CALL(512); break;            \
    case 1024: CALL(1024); break;          \
    case 2048: CALL(2048); break;          \
    case 4096: CALL(4096); break;          \
    default: break;                        \
  }

template <typename R>
void bapply_io(const SpatialPlan<R>& p, int F, const RowIO<R>& io, cudaStream_t st) {
#define TSFDE_CALL_B(LL) bapply_L<R, LL>(p, F, io, st)
  TSFDE_L_SWITCH(p.L, TSFDE_CALL_B)
#undef TSFDE_CALL_B
}

template <typename R>
void tau_io(const SpatialPlan<R>& p, int F, const R* dbar, int dbar_off, R c, const RowIO<R>& io,
            cudaStream_t st) {
  const R* db = dbar ? dbar + dbar_off : nullptr;
#define TSFDE_CALL_T(LL) tau_L<R, LL>(p, F, db, c, io, st)
  TSFDE_L_SWITCH(p.L, TSFDE_CALL_T)
#undef TSFDE_CALL_T
}

template <typename R>
void bapply(const SpatialPlan<R>& p, const R* x, R* y, int F, const int* skip, cudaStream_t st) {
  RowIO<R> io;
  io.src = x;
  io.dst = y;
  io.skip = skip;
  bapply_io<R>(p, F, io, st);
}

template <typename R>
void tau_solve(const SpatialPlan<R>& p, const R* x, R* y, int F, const R* dbar, int dbar_off, R c,
               const int* skip, cudaStream_t st) {
  RowIO<R> io;
  io.src = x;
  io.dst = y;
  io.skip = skip;
  tau_io<R>(p, F, dbar, dbar_off, c, io, st);
}

template void bapply_io<double>(const SpatialPlan<double>&, int, const RowIO<double>&, cudaStream_t);
template void bapply_io<float>(const SpatialPlan<float>&, int, const RowIO<float>&, cudaStream_t);
template void tau_io<double>(const SpatialPlan<double>&, int, const double*, int, double, const RowIO<double>&,
                             cudaStream_t);
template void tau_io<float>(const SpatialPlan<float>&, int, const float*, int, float, const RowIO<float>&,
                            cudaStream_t);
template void bapply<double>(const SpatialPlan<double>&, const double*, double*, int, const int*, cudaStream_t);
template void bapply<float>(const SpatialPlan<float>&, const float*, float*, int, const int*, cudaStream_t);
template void tau_solve<double>(const SpatialPlan<double>&, const double*, double*, int, const double*, int,
                                double, const int*, cudaStream_t);
template void tau_solve<float>(const SpatialPlan<float>&, const float*, float*, int, const float*, int, float,
                               const int*, cudaStream_t);

size_t spatial_work_elems(int d, int n, int L_in, int F) {
  const long long L = L_in, H = L / 2 + 1;
  if (d == 1) return 0;
  if (d == 2) return (size_t)F * n * H;
  return (size_t)F * n * L * H;   // the larger of the two d = 3 buffers
}

// ----------------------------------------------------------------------------------
// Setup kernels
// ----------------------------------------------------------------------------------

// out[a][k][b] = scale * sum_{j < J} w_j in[a][j][b] cos(2 pi ((j (k + k0)) mod M) / M),
// w_j = 1 for j = 0 and (half-range trapezoid, wmode 1) j = J - 1, else 2.
__global__ void k_cos_axis(const double* __restrict__ in, double* __restrict__ out, long long A, int J,
                           long long B, int Kout, int k0, int M, const double* __restrict__ cosM, int wmode,
                           double scale) {
  const long long total = A * Kout * B;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx % B;
    const long long ak = idx / B;
    const int k = (int)(ak % Kout);
    const long long a = ak / Kout;
    const long long kk = k + k0;
    const double* src = in + a * J * B + b;
    double acc = 0.0;
    long long m = 0;   // (j * kk) mod M, advanced incrementally
    const long long step = kk % M;
    for (int j = 0; j < J; ++j) {
      double w = (j == 0 || (wmode == 1 && j == J - 1)) ? 1.0 : 2.0;
      acc += w * src[(long long)j * B] * cosM[m];
      m += step;
      if (m >= M) m -= M;
    }
    out[idx] = scale * acc;
  }
}

// g on the half grid [0, K/2]^d: g = (sum_i 4 sin^2(pi k_i / K))^(omega/2)   (Eq. 7)
__global__ void k_g_grid(double* __restrict__ g, int d, int Kh, const double* __restrict__ sin2,
                         double half_omega) {
  long long total = 1;
  for (int i = 0; i < d; ++i) total *= Kh;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
      s += 4.0 * sin2[r % Kh];
      r /= Kh;
    }
    g[idx] = (s > 0.0) ? pow(s, half_omega) : 0.0;
  }
}

namespace {

cudaError_t upload_cos_table(int M, double** dev) {
  std::vector<double> h(M);
  const long double twopi = 6.283185307179586476925286766559005768L;
  for (int m = 0; m < M; ++m) h[m] = (double)cosl(twopi * (long double)m / (long double)M);
  cudaError_t e = cudaMalloc(dev, sizeof(double) * M);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dev, h.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
}

void launch_cos_axis(const double* in, double* out, long long A, int J, long long B, int Kout, int k0, int M,
                     const double* cosM, int wmode, double scale, cudaStream_t st) {
  long long total = A * Kout * B;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_cos_axis<<<blocks, 256, 0, st>>>(in, out, A, J, B, Kout, k0, M, cosM, wmode, scale);
}

long long ipow(long long b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

}  // namespace

cudaError_t build_coeffs_dft(int d, int n, double omega, int K, double* a_out, cudaStream_t st) {
  const int Kh = K / 2 + 1;
  double *sin2 = nullptr, *cosK = nullptr, *bufA = nullptr, *bufB = nullptr;
  cudaError_t e;
  {
    std::vector<double> h(Kh);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < Kh; ++k) {
      long double s = sinl(pi * (long double)k / (long double)K);
      h[k] = (double)(s * s);
    }
    e = cudaMalloc(&sin2, sizeof(double) * Kh);
    if (e == cudaSuccess) e = cudaMemcpy(sin2, h.data(), sizeof(double) * Kh, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = upload_cos_table(K, &cosK);
  const long long gsz = ipow(Kh, d);
  if (e == cudaSuccess) e = cudaMalloc(&bufA, sizeof(double) * gsz);
  if (e == cudaSuccess) e = cudaMalloc(&bufB, sizeof(double) * gsz);
  if (e == cudaSuccess) {
    k_g_grid<<<(int)std::min<long long>((gsz + 255) / 256, 152 * 64), 256, 0, st>>>(bufA, d, Kh, sin2,
                                                                                      omega / 2.0);
    // transform axis by axis, last axis first; shape [Kh or n]... with n on finished axes
    double* src = bufA;
    double* dst = bufB;
    for (int ax = d - 1; ax >= 0; --ax) {
      const long long A = ipow(Kh, ax);           // axes before: still untransformed
      const long long B = ipow(n, d - 1 - ax);    // axes after: already transformed
      const double scale = 1.0 / (double)K;
      double* target = (ax == 0) ? a_out : dst;
      launch_cos_axis(src, target, A, Kh, B, n, 0, K, cosK, 1, scale, st);
      std::swap(src, dst);
    }
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(sin2);
  cudaFree(cosK);
  cudaFree(bufA);
  cudaFree(bufB);
  return e;
}

cudaError_t build_symbols(int d, int n, int np, const double* a_dev, const double* a_tau, double* lam_out,
                          double* mu_out, cudaStream_t st) {
  const int L = 2 * (np + 1), H = L / 2 + 1;
  double *cosL = nullptr, *bufA = nullptr, *bufB = nullptr;
  cudaError_t e = upload_cos_table(L, &cosL);
  const long long big = ipow(L, d);
  if (e == cudaSuccess) e = cudaMalloc(&bufA, sizeof(double) * big);
  if (e == cudaSuccess) e = cudaMalloc(&bufB, sizeof(double) * big);
  if (e == cudaSuccess) {
    // circulant symbol of B_n embedded in size L >= 2 n - 1: per axis
    // lam_k = sum_{l<n} w_l a_l cos(2 pi l k / L), w = (1, 2, 2, ...)
    const double* src = a_dev;
    double* bufs[2] = {bufA, bufB};
    int which = 0;
    for (int ax = d - 1; ax >= 0; --ax) {
      const int Kout = (ax == d - 1) ? H : L;
      const long long A = ipow(n, ax);
      const long long B = (ax == d - 1) ? 1 : ipow(L, d - 2 - ax) * H;
      double scale = 1.0 / (double)L;
      double* target = (ax == 0) ? lam_out : bufs[which];
      launch_cos_axis(src, target, A, n, B, Kout, 0, L, cosL, 0, scale, st);
      src = target;
      which ^= 1;
    }
    // eigenvalues of tau(B_np): mu_k = sum_{l<np} w_l a_l prod cos(pi l_i k_i / (np+1)), k_i = 1..np
    src = a_tau;
    which = 0;
    for (int ax = d - 1; ax >= 0; --ax) {
      const long long A = ipow(np, ax);
      const long long B = ipow(np, d - 1 - ax);
      double* target = (ax == 0) ? mu_out : bufs[which];
      launch_cos_axis(src, target, A, np, B, np, 1, L, cosL, 0, 1.0, st);
      src = target;
      which ^= 1;
    }
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(cosL);
  cudaFree(bufA);
  cudaFree(bufB);
  return e;
}

// Box [J]^d of a ([n]^d, J <= n): out[i] = a[the same multi-index], last axis fastest.
__global__ void k_box(const double* __restrict__ a, double* __restrict__ out, int d, int n, int J) {
  long long total = 1;
  for (int i = 0; i < d; ++i) total *= J;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx, src = 0, mul = 1;
    for (int i = 0; i < d; ++i) {
      src += (r % J) * mul;
      r /= J;
      mul *= n;
    }
    out[idx] = a[src];
  }
}

cudaError_t build_strang(int d, int n, int L, const double* a_dev, double2* chirp64, float2* chirp32, double2* bhat64,
                         float2* bhat32, double* lam_out, cudaStream_t st) {
  if (2 * n - 1 > L) return cudaErrorInvalidValue;
  // chirp c_j = exp(-i pi j^2 / n), the angle reduced with j^2 mod 2n
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> cr(n), ci(n);
  std::vector<double2> c64(n), b64(L);
  std::vector<float2> c32(n), b32(L);
  for (int j = 0; j < n; ++j) {
    const long long m = ((long long)j * j) % (2LL * n);
    const long double ang = pi * (long double)m / (long double)n;
    cr[j] = cosl(ang);
    ci[j] = -sinl(ang);
    c64[j] = make_double2((double)cr[j], (double)ci[j]);
    c32[j] = make_float2((float)cr[j], (float)ci[j]);
  }
  // bhat_k = (1/L) sum_{|m| < n} conj(c_|m|) exp(-2 pi i k m / L)
  //        = (1/L) [conj(c_0) + 2 sum_{m=1}^{n-1} conj(c_m) cos(2 pi k m / L)]
  std::vector<long double> cosL(L);
  for (int i = 0; i < L; ++i) cosL[i] = cosl(2.0L * pi * (long double)i / (long double)L);
  for (int k = 0; k < L; ++k) {
    long double sr = cr[0], si = -ci[0];
    for (int m = 1; m < n; ++m) {
      const long double w = 2.0L * cosL[(int)(((long long)k * m) % L)];
      sr += cr[m] * w;
      si -= ci[m] * w;
    }
    sr /= (long double)L;
    si /= (long double)L;
    b64[k] = make_double2((double)sr, (double)si);
    b32[k] = make_float2((float)sr, (float)si);
  }
  cudaError_t e = cudaMemcpyAsync(chirp64, c64.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(chirp32, c32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bhat64, b64.data(), sizeof(double2) * L, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bhat32, b32.data(), sizeof(float2) * L, cudaMemcpyHostToDevice, st);
  // eigenvalues of s(B_n): per axis lam_k = sum_{l <= n/2} w_l a_l cos(2 pi l k / n), w_0 = 1, w_l = 2,
  // and w_{n/2} = 1 for even n (the first column keeps a_l for l <= n/2 and wraps a_{n-l} above)
  const int J = n / 2 + 1;
  double *cosN = nullptr, *bufA = nullptr, *bufB = nullptr;
  const long long big = ipow(n, d);
  if (e == cudaSuccess) e = upload_cos_table(n, &cosN);
  if (e == cudaSuccess) e = cudaMalloc(&bufA, sizeof(double) * big);
  if (e == cudaSuccess) e = cudaMalloc(&bufB, sizeof(double) * big);
  if (e == cudaSuccess) {
    const long long box = ipow(J, d);
    k_box<<<(int)std::min<long long>((box + 255) / 256, 152 * 16), 256, 0, st>>>(a_dev, bufA, d, n, J);
    const double* src = bufA;
    double* bufs[2] = {bufB, bufA};
    int which = 0;
    for (int ax = d - 1; ax >= 0; --ax) {
      const long long A = ipow(J, ax);
      const long long B = ipow(n, d - 1 - ax);
      double* target = (ax == 0) ? lam_out : bufs[which];
      launch_cos_axis(src, target, A, J, B, n, 0, n, cosN, (n % 2 == 0) ? 1 : 0, 1.0, st);
      src = target;
      which ^= 1;
    }
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(cosN);
  cudaFree(bufA);
  cudaFree(bufB);
  return e;
}

cudaError_t make_twiddles(int L, void** out_d, void** out_f, cudaStream_t st) {
  std::vector<double2> hd(L);
  std::vector<float2> hf(L);
  const long double twopi = 6.283185307179586476925286766559005768L;
  for (int k = 0; k < L; ++k) {
    long double a = twopi * (long double)k / (long double)L;
    hd[k].x = (double)cosl(a);
    hd[k].y = (double)(-sinl(a));
    hf[k].x = (float)cosl(a);
    hf[k].y = (float)(-sinl(a));
  }
  cudaError_t e = cudaMalloc(out_d, sizeof(double2) * L);
  if (e == cudaSuccess) e = cudaMalloc(out_f, sizeof(float2) * L);
  if (e == cudaSuccess) e = cudaMemcpyAsync(*out_d, hd.data(), sizeof(double2) * L, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(*out_f, hf.data(), sizeof(float2) * L, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

__global__ void k_cast_d2f(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void k_cast_f2d(const float* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
void cast_d2f(const double* x, float* y, long long n, cudaStream_t st) {
  int b = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  if (b > 0) k_cast_d2f<<<b, 256, 0, st>>>(x, y, n);
}
void cast_f2d(const float* x, double* y, long long n, cudaStream_t st) {
  int b = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  if (b > 0) k_cast_f2d<<<b, 256, 0, st>>>(x, y, n);
}

}  // namespace tsfde
