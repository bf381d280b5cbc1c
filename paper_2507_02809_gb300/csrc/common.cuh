// Shared device helpers: complex types, warp/block reductions, launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define TSFDE_HD __host__ __device__ __forceinline__
#define TSFDE_D __device__ __forceinline__

namespace tsfde {

template <typename R> struct CplxT;
template <> struct CplxT<double> { using T = double2; };
template <> struct CplxT<float> { using T = float2; };
template <typename R> using cx = typename CplxT<R>::T;

template <typename R> TSFDE_HD cx<R> mk(R a, R b) { cx<R> z; z.x = a; z.y = b; return z; }
template <typename R> TSFDE_HD cx<R> cadd(cx<R> a, cx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> TSFDE_HD cx<R> csub(cx<R> a, cx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> TSFDE_HD cx<R> cmul(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename R> TSFDE_HD cx<R> cmulc(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename R> TSFDE_HD cx<R> cconj(cx<R> a) { return mk<R>(a.x, -a.y); }
template <typename R> TSFDE_HD cx<R> cscale(cx<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
// multiply by -i (DIR = -1) or +i (DIR = +1)
template <typename R, int DIR> TSFDE_HD cx<R> mul_i(cx<R> a) {
  return DIR < 0 ? mk<R>(a.y, -a.x) : mk<R>(-a.y, a.x);
}

template <typename R> TSFDE_D R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed tree); result valid in every thread.
// `scratch` must hold blockDim.x / 32 values; blockDim.x a multiple of 32, <= 1024.
template <typename R> TSFDE_D R block_sum(R v, R* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  R t = (threadIdx.x < (unsigned)nw) ? scratch[threadIdx.x] : R(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  t = scratch[0];
  __syncthreads();
  return t;
}

// Sum of `count` partials in a fixed order by one block (all threads get it).
template <typename R> TSFDE_D R block_reduce_partials(const R* __restrict__ part, int count, R* scratch) {
  R v = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += part[i];
  return block_sum(v, scratch);
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace tsfde
