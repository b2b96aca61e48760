// Vector kernels of the biconjugate gradient solver (csrc_bicg): BiCG as written in Saad,
// Iterative Methods for Sparse Linear Systems (2nd ed.), Algorithm 7.3, the oblique-projection
// use that Section 1 gives for CSRC's implicit transpose. The products are the library's
// own csrc_spmv / csrc_spmv_t; these kernels do the rest of an iteration in two fused passes.
//
// Inner products are deterministic: every block sums a fixed grid-stride slice in FP64 and
// reduces it in shared memory in a fixed tree order, then one block adds the block sums in
// index order. FP32 vectors (FP32 / BF16 storage) are accumulated in FP64 as well.
#include <cstdint>

#include "internal.h"

namespace csrc {

namespace {

constexpr int kDotThreads = 256;

// Sums v[0..K) over the block in a fixed order; thread 0 gets the totals.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < K; ++k) sh[k * kDotThreads + t] = v[k];
  __syncthreads();
  for (int o = kDotThreads / 2; o > 0; o >>= 1) {
    if (t < o) {
#pragma unroll
      for (int k = 0; k < K; ++k) sh[k * kDotThreads + t] += sh[k * kDotThreads + t + o];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k * kDotThreads];
}

// partial[block] = sum over the block's slice of a[i] * b[i]
template <typename X>
__global__ void __launch_bounds__(kDotThreads) dot_kernel(int64_t n, const X* __restrict__ a,
                                                          const X* __restrict__ b, double* __restrict__ partial) {
  __shared__ double sh[kDotThreads];
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads)
    v[0] = fma((double)a[i], (double)b[i], v[0]);
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

// r = b - q; r* = r; p = r; p* = r; partials of (r, r) and (b, b)
template <typename X>
__global__ void __launch_bounds__(kDotThreads) bicg_init_kernel(int64_t n, const X* __restrict__ b,
                                                                const X* __restrict__ q, X* __restrict__ r,
                                                                X* __restrict__ rs, X* __restrict__ p,
                                                                X* __restrict__ ps, double* __restrict__ partial) {
  __shared__ double sh[2 * kDotThreads];
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads) {
    const X bi = b[i];
    const X ri = bi - q[i];
    r[i] = ri;
    rs[i] = ri;
    p[i] = ri;
    ps[i] = ri;
    v[0] = fma((double)ri, (double)ri, v[0]);
    v[1] = fma((double)bi, (double)bi, v[1]);
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = v[0];
    partial[2 * blockIdx.x + 1] = v[1];
  }
}

// x += alpha p; r -= alpha q; r* -= alpha q*; partials of (r, r) and (r, r*)
template <typename X>
__global__ void __launch_bounds__(kDotThreads) bicg_update1_kernel(int64_t n, double alpha, const X* __restrict__ p,
                                                                   const X* __restrict__ q, const X* __restrict__ qs,
                                                                   X* __restrict__ x, X* __restrict__ r,
                                                                   X* __restrict__ rs, double* __restrict__ partial) {
  __shared__ double sh[2 * kDotThreads];
  const X al = (X)alpha;
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads) {
    x[i] = fma(al, p[i], x[i]);
    const X ri = fma(-al, q[i], r[i]);
    const X rsi = fma(-al, qs[i], rs[i]);
    r[i] = ri;
    rs[i] = rsi;
    v[0] = fma((double)ri, (double)ri, v[0]);
    v[1] = fma((double)ri, (double)rsi, v[1]);
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = v[0];
    partial[2 * blockIdx.x + 1] = v[1];
  }
}

// p = r + beta p; p* = r* + beta p*
template <typename X>
__global__ void __launch_bounds__(kDotThreads) bicg_update2_kernel(int64_t n, double beta, const X* __restrict__ r,
                                                                   const X* __restrict__ rs, X* __restrict__ p,
                                                                   X* __restrict__ ps) {
  const X be = (X)beta;
  for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads) {
    p[i] = fma(be, p[i], r[i]);
    ps[i] = fma(be, ps[i], rs[i]);
  }
}

// out[k] = sum over blocks of partial[block * K + k], blocks in index order (one block)
__global__ void __launch_bounds__(kDotThreads) sum_partials_kernel(int nblocks, int K, const double* __restrict__ partial,
                                                                   double* __restrict__ out) {
  __shared__ double sh[kDotThreads];
  for (int k = 0; k < K; ++k) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nblocks; b += kDotThreads) v[0] += partial[(int64_t)b * K + k];
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) out[k] = v[0];
    __syncthreads();
  }
}

}  // namespace

int solver_blocks(int sms) { return sms > 0 ? 2 * sms : 304; }

cudaError_t launch_solver_op(int op, bool fp64, int64_t n, int nblocks, double scalar, const void* v0, const void* v1,
                             const void* v2, void* w0, void* w1, void* w2, void* w3, double* partial, double* out,
                             cudaStream_t s) {
  if (n < 0 || nblocks <= 0) return cudaErrorInvalidValue;
  int K = 0;
#define CSRC_OP(X)                                                                                                 \
  switch (op) {                                                                                                    \
    case SOLVER_DOT:                                                                                               \
      dot_kernel<X><<<nblocks, kDotThreads, 0, s>>>(n, static_cast<const X*>(v0), static_cast<const X*>(v1),        \
                                                    partial);                                                      \
      K = 1;                                                                                                       \
      break;                                                                                                       \
    case SOLVER_INIT:                                                                                              \
      bicg_init_kernel<X><<<nblocks, kDotThreads, 0, s>>>(n, static_cast<const X*>(v0), static_cast<const X*>(v1),  \
                                                          static_cast<X*>(w0), static_cast<X*>(w1),                \
                                                          static_cast<X*>(w2), static_cast<X*>(w3), partial);      \
      K = 2;                                                                                                       \
      break;                                                                                                       \
    case SOLVER_UPDATE1:                                                                                           \
      bicg_update1_kernel<X><<<nblocks, kDotThreads, 0, s>>>(n, scalar, static_cast<const X*>(v0),                 \
                                                             static_cast<const X*>(v1), static_cast<const X*>(v2), \
                                                             static_cast<X*>(w0), static_cast<X*>(w1),             \
                                                             static_cast<X*>(w2), partial);                        \
      K = 2;                                                                                                       \
      break;                                                                                                       \
    default:                                                                                                       \
      bicg_update2_kernel<X><<<nblocks, kDotThreads, 0, s>>>(n, scalar, static_cast<const X*>(v0),                 \
                                                             static_cast<const X*>(v1), static_cast<X*>(w0),       \
                                                             static_cast<X*>(w1));                                 \
      break;                                                                                                       \
  }
  if (fp64) {
    CSRC_OP(double)
  } else {
    CSRC_OP(float)
  }
#undef CSRC_OP
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || K == 0) return e;
  sum_partials_kernel<<<1, kDotThreads, 0, s>>>(nblocks, K, partial, out);
  return cudaGetLastError();
}

}  // namespace csrc
