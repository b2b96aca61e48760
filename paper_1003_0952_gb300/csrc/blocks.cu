// Band kernels for matrices with node blocks (2 or 3 consecutive rows that share their
// columns below the diagonal block): single vectors, window strategy. The kernel is in
// band.cuh (block_unit); this unit only instantiates and launches it.
#include "band.cuh"

namespace csrc {

template <int MODE, int B>
static cudaError_t set_smem_block() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_band_smem<MODE, 1, false, 1, B>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 2, false, 1, B>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 4, false, 1, B>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 8, false, 1, B>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 16, false, 1, B>()) != cudaSuccess) e = r;
  return e;
}

cudaError_t prepare_band_kernels_block() {
  cudaError_t e = cudaSuccess, r;
#define CSRC_M(M)                                                   \
  if ((r = set_smem_block<M, 2>()) != cudaSuccess) e = r;          \
  if ((r = set_smem_block<M, 3>()) != cudaSuccess) e = r;
  CSRC_M(MODE_DF) CSRC_M(MODE_F64) CSRC_M(MODE_F32) CSRC_M(MODE_BF16)
#undef CSRC_M
  return e;
}

template <int MODE, int B>
static void launch_b(int group, const BandArgs& a, dim3 grid, int smem, cudaStream_t s) {
  constexpr int T = BandShape<MODE>::T;
  switch (group) {
    case 1: band_kernel<MODE, 1, false, 1, B><<<grid, T, smem, s>>>(a); break;
    case 2: band_kernel<MODE, 2, false, 1, B><<<grid, T, smem, s>>>(a); break;
    case 4: band_kernel<MODE, 4, false, 1, B><<<grid, T, smem, s>>>(a); break;
    case 8: band_kernel<MODE, 8, false, 1, B><<<grid, T, smem, s>>>(a); break;
    default: band_kernel<MODE, 16, false, 1, B><<<grid, T, smem, s>>>(a); break;
  }
}

template <int MODE>
static void launch_mode_block(const BandArgs& a, dim3 grid, int smem, cudaStream_t s) {
  if (a.block == 2) launch_b<MODE, 2>(a.group, a, grid, smem, s);
  else launch_b<MODE, 3>(a.group, a, grid, smem, s);
}

cudaError_t launch_band_block(Arith arith, int storage, const BandArgs& a, int nbands, int smem, cudaStream_t s) {
  if (nbands <= 0) return cudaSuccess;
  if (a.block != 2 && a.block != 3) return cudaErrorInvalidValue;
  dim3 grid(nbands);
  switch (mode_of(arith, storage)) {
    case MODE_DF: launch_mode_block<MODE_DF>(a, grid, smem, s); break;
    case MODE_F64: launch_mode_block<MODE_F64>(a, grid, smem, s); break;
    case MODE_F32: launch_mode_block<MODE_F32>(a, grid, smem, s); break;
    default: launch_mode_block<MODE_BF16>(a, grid, smem, s); break;
  }
  return cudaGetLastError();
}

}  // namespace csrc
