// z = A y for a one-dimensional instance without any device allocation.
//
// Some callers of this library cannot allocate device memory themselves or let a library do
// it: code running inside a memory pool or arena that owns all device memory of the process,
// a host application that must not trigger cudaMalloc (and its implicit device-wide
// synchronisation) while other work is in flight, or a plug-in whose host framework forbids
// allocation after initialisation.  For them this file provides tsfde_matvec_1d_noalloc: the
// same operator as tsfde_matvec for d = 1, but every table and the work buffer live in one
// file-scope __device__ array of fixed size (kScratchDoubles doubles, about 16.9 MB), which
// every GPU that loads the library holds until the process exits.
//
// Set-up: on the first call on a device (with that device current) the address of the array
// is looked up once with cudaGetSymbolAddress; that first call should therefore come before
// any stream capture.  Under lazy module loading (CUDA's default) the same first call loads the
// module on that device and reserves the array there, so callers make it once during
// initialisation.  The address is cached per device ordinal and belongs to the device's primary
// context: it is not valid after cudaDeviceReset or from another context.  All calls share the
// array and it keeps the last call's contents; every
// call rebuilds the tables it reads and overwrites the work buffer before reading it, so
// nothing needs to start at zero.  Calls whose work overlaps on the GPU (different streams, or
// host threads on the same device) race on the array and must be serialised by the caller.
#include <math.h>

#include <mutex>
#include <string>

#include "../../include/tsfde.h"
#include "internal.h"
#include "kernels.h"
#include "rowio.cuh"

namespace tsfde {
namespace {

// Layout of the scratch array, in doubles (every offset a multiple of 32 doubles = 256 bytes)
constexpr long long kMaxS = 4096;
constexpr long long kMaxN = 2047;            // n + 1 <= 2048, transforms of length L <= 4096
constexpr long long kMaxL = 2 * (kMaxN + 1);
constexpr long long kOffE = 0;                                  // e_m, m < S
constexpr long long kOffA = kOffE + kMaxS;                      // a_l, l < n
constexpr long long kOffLam = kOffA + 2048;                     // symbol / L, k <= L/2
constexpr long long kOffTw = kOffLam + 2080;                    // twiddles, L double2
constexpr long long kOffBy = kOffTw + 2 * kMaxL;                // B_n y for S+1 fields
constexpr long long kMaxU = 1LL << 21;                          // (S + 1) n <= 2^21
constexpr long long kScratchDoubles = kOffBy + kMaxU;
static_assert(kOffA % 32 == 0 && kOffLam % 32 == 0 && kOffTw % 32 == 0 && kOffBy % 32 == 0, "alignment");

}  // namespace
}  // namespace tsfde

// The scratch array (device memory reserved by the module, not by an allocation call).
static __device__ __align__(256) double g_tsfde_noalloc_scratch[tsfde::kScratchDoubles];

namespace tsfde {
namespace {

std::mutex g_scratch_mutex;
double* g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tsfde_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// e_m of the L1 formula (Sec. 4): e_0 = b_0 = 1, e_m = b_m - b_{m-1}, b_m = (m+1)^(1-beta) - m^(1-beta)
__global__ void k_na_weights(double* e, int S, double beta) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < S; m += gridDim.x * blockDim.x) {
    const double g = 1.0 - beta;
    if (m == 0) {
      e[0] = 1.0;
    } else {
      double bm = pow(m + 1.0, g) - pow((double)m, g);
      double bm1 = pow((double)m, g) - pow(m - 1.0, g);
      e[m] = bm - bm1;
    }
  }
}

// a_l by the recursion of Lemma 1(b) from a_0 of Lemma 1(a) (one thread: sequential)
__global__ void k_na_coeffs(double* a, int n, double omega) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double h = tgamma(omega / 2.0 + 1.0);
  double v = tgamma(omega + 1.0) / (h * h);
  for (int l = 0; l < n; ++l) {
    a[l] = v;
    v *= 1.0 - (omega + 1.0) / (omega / 2.0 + l + 1.0);
  }
}

// twiddles exp(-2 pi i k / L)
__global__ void k_na_twiddles(double2* tw, int L) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * k / (double)L, &s, &c);
    tw[k] = make_double2(c, -s);
  }
}

// circulant symbol / L: lam_k = (a_0 + 2 sum_{l=1}^{n-1} a_l cos(2 pi l k / L)) / L, k <= L/2
__global__ void k_na_symbol(const double* a, const double2* tw, double* lam, int n, int L) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= L / 2; k += gridDim.x * blockDim.x) {
    double acc = a[0];
    long long m = 0;
    for (int l = 1; l < n; ++l) {
      m += k;
      if (m >= L) m -= L;
      acc += 2.0 * a[l] * tw[m].x;
    }
    lam[k] = acc / (double)L;
  }
}

}  // namespace
}  // namespace tsfde

using namespace tsfde;

extern "C" tsfde_status tsfde_matvec_1d_noalloc(int n, int S, double length, double T, double beta, double omega,
                                                double alpha, const double* gamma1, const double* gamma2,
                                                const double* q, const double* y, double* z, void* stream) {
  set_error("");
  if (!gamma1 || !gamma2 || !q || !y || !z || y == z) {
    set_error("tsfde_matvec_1d_noalloc: null or aliased pointer");
    return TSFDE_EINVAL;
  }
  if (!(beta > 0 && beta < 1) || !(omega > 1 && omega < 2) || !(alpha > 0) || !(length > 0) || !(T > 0) || S < 1) {
    set_error("tsfde_matvec_1d_noalloc: need 0 < beta < 1, 1 < omega < 2, alpha > 0, length > 0, T > 0, S >= 1");
    return TSFDE_EINVAL;
  }
  const int np1 = n + 1;
  if (n < 3 || (np1 & (np1 - 1)) != 0 || n > kMaxN || S > kMaxS || (long long)(S + 1) * n > kMaxU) {
    set_error("tsfde_matvec_1d_noalloc: needs n + 1 a power of two, 4 <= n + 1 <= 2048, S <= 4096 and "
              "(S + 1) n <= 2097152 (the fixed scratch array holds 16.9 MB)");
    return TSFDE_EUNSUPPORTED;
  }
  double* scratch = nullptr;
  cudaError_t ce = scratch_address(&scratch);
  if (ce != cudaSuccess) {
    set_error(std::string("tsfde_matvec_1d_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
    return TSFDE_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int L = 2 * np1;
  const long long N = n;
  const double h = length / (n + 1), dt = T / S;
  const double eta = pow(dt, beta) * tgamma(2.0 - beta);
  const double cs = eta / pow(h, omega), cf = alpha / pow(h, omega);
  double* e = scratch + kOffE;
  double* a = scratch + kOffA;
  double* lam = scratch + kOffLam;
  double2* tw = reinterpret_cast<double2*>(scratch + kOffTw);
  double* By = scratch + kOffBy;

  k_na_weights<<<(S + 255) / 256, 256, 0, st>>>(e, S, beta);
  k_na_coeffs<<<1, 1, 0, st>>>(a, n, omega);
  k_na_twiddles<<<(L + 255) / 256, 256, 0, st>>>(tw, L);
  k_na_symbol<<<(L / 2 + 1 + 127) / 128, 128, 0, st>>>(a, tw, lam, n, L);

  SpatialPlan<double> P;
  P.d = 1;
  P.n = n;
  P.L = L;
  P.H = L / 2 + 1;
  P.N = N;
  P.max_fields = S + 1;
  P.tw = tw;
  P.lam = lam;
  bapply<double>(P, y, By, S + 1, nullptr, st);
  matvec_time(y, By, gamma1, gamma2, q, e, z, S, N, cs, cf, eta, st);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    set_error(std::string("tsfde_matvec_1d_noalloc: launch: ") + cudaGetErrorString(ce));
    return TSFDE_ECUDA;
  }
  return TSFDE_OK;
}
