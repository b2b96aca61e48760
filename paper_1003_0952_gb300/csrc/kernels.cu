// Stream-order band kernels (single vectors) and the accumulation kernel of the CSRC
// products. The band kernel itself is in band.cuh.
#include "band.cuh"

namespace csrc {

// ---------------------------------------------------------------------------- accumulation
// y[row, c] += sum of the row's spilled partial sums, in band order (deterministic).
// One thread per (receiving row, column); spill entries hold rk columns each. Row i's sums
// are spill entries acc_src[e] for e in [acc_ptr[i], acc_ptr[i+1]), or the entries e
// themselves when acc_src is null (a spill buffer already ordered by receiving row).
template <typename T>
__global__ void accumulate_kernel(int64_t nacc, int rk, int ldx, const int32_t* __restrict__ acc_row,
                                  const int32_t* __restrict__ acc_ptr, const int32_t* __restrict__ acc_src,
                                  const T* __restrict__ spill, T* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nacc * rk) return;
  const int64_t i = t / rk;
  const int c = (int)(t % rk);
  const int row = acc_row[i];
  T s = y[(size_t)row * ldx + c];
  const int e1 = acc_ptr[i + 1];
  if (acc_src) {
    for (int e = acc_ptr[i]; e < e1; ++e) s += spill[(size_t)acc_src[e] * rk + c];
  } else {
    for (int e = acc_ptr[i]; e < e1; ++e) s += spill[(size_t)e * rk + c];
  }
  y[(size_t)row * ldx + c] = s;
}

// ---------------------------------------------------------------------------- bounded-wait self-test
// One CTA waits, with the band kernels' bounded wait, on an mbarrier that nothing arrives at:
// the wait must give up after `limit` cycles and record DEV_TIMEOUT in *status.
__global__ void wait_probe_kernel(long long limit, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1u);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(b, 0u, limit)) atomicOr(status, DEV_TIMEOUT);
    mbar_inval(b);
  }
}

cudaError_t launch_wait_probe(long long limit, int32_t* status, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(limit, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- double-float split
__global__ void split_df_kernel(const double* __restrict__ v, df32* __restrict__ out, int64_t count) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = df_split<false>(v[k], nullptr);
}

cudaError_t launch_split_df(const double* v, void* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)std::max(sms, 1) * 32);
  split_df_kernel<<<(unsigned)blocks, 256, 0, s>>>(v, static_cast<df32*>(out), count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- launchers
template <int MODE>
static cudaError_t set_smem_mode() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_band_smem<MODE, 1, false, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 1, true, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 2, false, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 2, true, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 4, false, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 4, true, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 8, false, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 8, true, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 16, false, 1>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 16, true, 1>()) != cudaSuccess) e = r;
  return e;
}

cudaError_t prepare_band_kernels() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_smem_mode<MODE_DF>()) != cudaSuccess) e = r;
  if ((r = set_smem_mode<MODE_F64>()) != cudaSuccess) e = r;
  if ((r = set_smem_mode<MODE_F32>()) != cudaSuccess) e = r;
  if ((r = set_smem_mode<MODE_BF16>()) != cudaSuccess) e = r;
  if ((r = prepare_band_kernels_block()) != cudaSuccess) e = r;
  return e;
}

template <int MODE>
static void launch_mode(int group, bool atomic, const BandArgs& a, dim3 grid, int smem, cudaStream_t s) {
#define CSRC_G(GV)                                                                        \
  if (atomic) band_kernel<MODE, GV, true, 1><<<grid, band_threads(GV, 1, 1), smem, s>>>(a); \
  else band_kernel<MODE, GV, false, 1><<<grid, band_threads(GV, 1, 1), smem, s>>>(a);
  switch (group) {
    case 1: CSRC_G(1) break;
    case 2: CSRC_G(2) break;
    case 4: CSRC_G(4) break;
    case 8: CSRC_G(8) break;
    default: CSRC_G(16) break;
  }
#undef CSRC_G
}

cudaError_t launch_band(Arith arith, int storage, bool atomic_flush, const BandArgs& a, int nbands, int smem,
                        cudaStream_t s) {
  if (nbands <= 0) return cudaSuccess;
  if (a.block > 1) return launch_band_block(arith, storage, a, nbands, smem, s);
  const int mode = mode_of(arith, storage);
  dim3 grid(nbands);
  switch (mode) {
    case MODE_DF: launch_mode<MODE_DF>(a.group, atomic_flush, a, grid, smem, s); break;
    case MODE_F64: launch_mode<MODE_F64>(a.group, atomic_flush, a, grid, smem, s); break;
    case MODE_F32: launch_mode<MODE_F32>(a.group, atomic_flush, a, grid, smem, s); break;
    default: launch_mode<MODE_BF16>(a.group, atomic_flush, a, grid, smem, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_accumulate(Arith arith, int storage, int64_t nacc, int rk, int ldx, const int32_t* acc_row,
                              const int32_t* acc_ptr, const int32_t* acc_src, const void* spill, void* y,
                              cudaStream_t s) {
  if (nacc <= 0) return cudaSuccess;
  const int bs = 256;
  const unsigned grid = (unsigned)((nacc * rk + bs - 1) / bs);
  if (storage == CSRC_F64) {
    accumulate_kernel<double><<<grid, bs, 0, s>>>(nacc, rk, ldx, acc_row, acc_ptr, acc_src,
                                                  static_cast<const double*>(spill), static_cast<double*>(y));
  } else {
    accumulate_kernel<float><<<grid, bs, 0, s>>>(nacc, rk, ldx, acc_row, acc_ptr, acc_src,
                                                 static_cast<const float*>(spill), static_cast<float*>(y));
  }
  (void)arith;
  return cudaGetLastError();
}

}  // namespace csrc
