// Declarations shared by the translation units of libtsfde (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "common.cuh"

namespace tsfde {

// Spatial operator data for one instance: B_n (d-level Toeplitz, Sec. 5) applied by circulant
// embedding of size L per direction (L = 2 p, p the smallest power of two >= n + 1), and
// tau(B_{p-1}) (Remark 1) diagonalised by the DST-I on the grid of p - 1 points (the standalone tau
// kernels of the graph form need p - 1 = n).  All arrays are device memory.
template <typename R>
struct SpatialPlan {
  int d = 0, n = 0, L = 0, H = 0;  // H = L / 2 + 1 (half spectrum of the last axis)
  long long N = 0;                 // n^d
  int max_fields = 0;              // fields one B apply may process at once
  const cx<R>* tw = nullptr;       // twiddles exp(-2 pi i k / L), k < L
  const R* lam = nullptr;          // circulant symbol / L^d, [L]^(d-1) x [H]
  const R* mu = nullptr;           // tau eigenvalues, [p - 1]^d
  cx<R>* work0 = nullptr;          // complex workspace for d >= 2
  cx<R>* work1 = nullptr;          // second workspace for d = 3
  size_t work_elems = 0;           // complex elements in each workspace
};

// y[f] = B_n x[f] for fields f < F (x, y: [F][N]; may alias only if x == y is not used).
// `skip` (may be nullptr): when *skip != 0 at kernel start the call does nothing.
template <typename R>
void bapply(const SpatialPlan<R>& p, const R* x, R* y, int F, const int* skip, cudaStream_t st);

// y[f] = (dbar_f I + c tau(B_n))^-1 x[f]; dbar == nullptr means dbar_f = 0.
// dbar is indexed dbar[dbar_off + f].
template <typename R>
void tau_solve(const SpatialPlan<R>& p, const R* x, R* y, int F, const R* dbar, int dbar_off, R c,
               const int* skip, cudaStream_t st);

template <typename R> struct RowIO;
// B_n applied with fused load / store work (rowio.cuh): the input of the first row pass comes
// from io's load mode and the output of the last row pass goes through io's store mode.
template <typename R>
void bapply_io(const SpatialPlan<R>& p, int F, const RowIO<R>& io, cudaStream_t st);
// tau solve with fused load (first DST pass) and store (last DST pass); io.dst is the work /
// output buffer of the solve.
template <typename R>
void tau_io(const SpatialPlan<R>& p, int F, const R* dbar, int dbar_off, R c, const RowIO<R>& io,
            cudaStream_t st);

// Workspace size (complex elements per buffer) for a B apply of F fields.
size_t spatial_work_elems(int d, int n, int L, int F);

// Setup, on the transform grid L = 2 (np + 1): the circulant symbol of B_n from a_dev ([n]^d,
// a_l for 0 <= l_i < n), lam_out [L]^(d-1) x [H] (scaled by 1 / L^d); the eigenvalues of tau(B_np)
// from a_tau ([np]^d), mu_out [np]^d.
cudaError_t build_symbols(int d, int n, int np, const double* a_dev, const double* a_tau, double* lam_out,
                          double* mu_out, cudaStream_t st);

// Setup of S_{n,S} (Remark 1) for transforms of length L >= 2 n - 1: the Bluestein tables of the
// length-n DFT (chirp [n]: exp(-i pi j^2 / n); bhat [L]: FFT of the conjugate chirp placed at m
// and L - m, |m| < n, divided by L; built in long double on the host) and the eigenvalues of the
// Strang circulant s(B_n) from a_dev ([n]^d), lam_out [n]^d in DFT order.  All outputs device memory.
cudaError_t build_strang(int d, int n, int L, const double* a_dev, double2* chirp64, float2* chirp32, double2* bhat64,
                         float2* bhat32, double* lam_out, cudaStream_t st);

// Setup, d >= 2: a_l = K^-d sum_k g(2 pi k / K) prod_i cos(2 pi l_i k_i / K) for 0 <= l_i < n
// (K-point trapezoid rule for Eq. 8).  a_out: device [n]^d.
cudaError_t build_coeffs_dft(int d, int n, double omega, int K, double* a_out, cudaStream_t st);

// Twiddle table exp(-2 pi i k / L) on the device.
cudaError_t make_twiddles(int L, void** out_dev_double2, void** out_dev_float2, cudaStream_t st);

// Element-wise conversion.
void cast_d2f(const double* x, float* y, long long n, cudaStream_t st);
void cast_f2d(const float* x, double* y, long long n, cudaStream_t st);

void set_error(const std::string& s);

}  // namespace tsfde
