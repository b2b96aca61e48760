// The auxiliary CSR of a rectangular CSRC matrix (Section 2.1, Fig. 2(b)).
//
// An n-by-m matrix (m >= n) is A_S + A_R: A_S is the n-by-n structurally symmetric part,
// run by the band kernels like any square matrix, and A_R holds the columns n..m-1. A_R
// only gathers: in Fig. 2(b) row i adds sum_k ar(k) x(jar(k)) to its sum before y(i) is
// assigned. Here that loop is its own kernel, run after the square product has written y:
//  - rect_rows_kernel: y[i] += sum over row i of A_R, for the rows that have A_R entries
//    (a compact list), one thread per row, entries in column order (deterministic).
//  - rect_cols_kernel: the transpose's last m - n entries, y[n + c] = sum over column c of
//    A_R of ar * x[row], from a column-major copy of A_R built at creation (a gather, so
//    no atomics and a fixed order).
// FP64 storage sums in FP64 (a few operations per auxiliary entry), FP32 and BF16
// storage in FP32, as the square part does.
#include <cstdint>

#include "internal.h"

namespace csrc {

template <typename V>
__device__ __forceinline__ float rect_f32(V v);
template <>
__device__ __forceinline__ float rect_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float rect_f32<uint16_t>(uint16_t v) { return __uint_as_float((unsigned)v << 16); }

template <typename V, typename X>
__global__ void rect_rows_kernel(int32_t nrows, const int32_t* __restrict__ rows, const int32_t* __restrict__ ptr,
                                 const int32_t* __restrict__ col, const V* __restrict__ val, const X* __restrict__ x,
                                 X* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows) return;
  const int k1 = ptr[t + 1];
  X s = X(0);
  for (int k = ptr[t]; k < k1; ++k) {
    if constexpr (sizeof(X) == 8) {
      s = fma((double)val[k], x[col[k]], s);
    } else {
      s = __fmaf_rn(rect_f32<V>(val[k]), x[col[k]], s);
    }
  }
  const int i = rows[t];
  y[i] = y[i] + s;
}

template <typename V, typename X>
__global__ void rect_cols_kernel(int32_t ncols, int32_t n, const int32_t* __restrict__ ptr,
                                 const int32_t* __restrict__ row, const V* __restrict__ val, const X* __restrict__ x,
                                 X* __restrict__ y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  const int k1 = ptr[c + 1];
  X s = X(0);
  for (int k = ptr[c]; k < k1; ++k) {
    if constexpr (sizeof(X) == 8) {
      s = fma((double)val[k], x[row[k]], s);
    } else {
      s = __fmaf_rn(rect_f32<V>(val[k]), x[row[k]], s);
    }
  }
  y[(int64_t)n + c] = s;
}

cudaError_t launch_rect_rows(int storage, int32_t nrows, const int32_t* rows, const int32_t* ptr, const int32_t* col,
                             const void* val, const void* x, void* y, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int bs = 128;
  const unsigned grid = (unsigned)((nrows + bs - 1) / bs);
  if (storage == CSRC_F64) {
    rect_rows_kernel<double, double><<<grid, bs, 0, s>>>(nrows, rows, ptr, col, static_cast<const double*>(val),
                                                         static_cast<const double*>(x), static_cast<double*>(y));
  } else if (storage == CSRC_F32) {
    rect_rows_kernel<float, float><<<grid, bs, 0, s>>>(nrows, rows, ptr, col, static_cast<const float*>(val),
                                                       static_cast<const float*>(x), static_cast<float*>(y));
  } else {
    rect_rows_kernel<uint16_t, float><<<grid, bs, 0, s>>>(nrows, rows, ptr, col, static_cast<const uint16_t*>(val),
                                                          static_cast<const float*>(x), static_cast<float*>(y));
  }
  return cudaGetLastError();
}

cudaError_t launch_rect_cols(int storage, int32_t ncols, int32_t n, const int32_t* ptr, const int32_t* row,
                             const void* val, const void* x, void* y, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const int bs = 128;
  const unsigned grid = (unsigned)((ncols + bs - 1) / bs);
  if (storage == CSRC_F64) {
    rect_cols_kernel<double, double><<<grid, bs, 0, s>>>(ncols, n, ptr, row, static_cast<const double*>(val),
                                                         static_cast<const double*>(x), static_cast<double*>(y));
  } else if (storage == CSRC_F32) {
    rect_cols_kernel<float, float><<<grid, bs, 0, s>>>(ncols, n, ptr, row, static_cast<const float*>(val),
                                                       static_cast<const float*>(x), static_cast<float*>(y));
  } else {
    rect_cols_kernel<uint16_t, float><<<grid, bs, 0, s>>>(ncols, n, ptr, row, static_cast<const uint16_t*>(val),
                                                          static_cast<const float*>(x), static_cast<float*>(y));
  }
  return cudaGetLastError();
}

}  // namespace csrc
