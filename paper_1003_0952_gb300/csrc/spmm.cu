// Band kernels for several right-hand sides: RK = 2, 4 or 8 columns of a row-major
// block X per pass (window strategy). The kernel is in band.cuh; this unit only
// instantiates and launches it, so that it compiles in parallel with kernels.cu.
#include "band.cuh"

namespace csrc {

template <int MODE, int RK>
static cudaError_t set_smem_rk() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_band_smem<MODE, 1, false, RK>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 2, false, RK>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 4, false, RK>()) != cudaSuccess) e = r;
  if ((r = set_band_smem<MODE, 8, false, RK>()) != cudaSuccess) e = r;
  return e;
}

template <int MODE>
static cudaError_t set_smem_mode_rk() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_smem_rk<MODE, 2>()) != cudaSuccess) e = r;
  if ((r = set_smem_rk<MODE, 4>()) != cudaSuccess) e = r;
  if ((r = set_smem_rk<MODE, 8>()) != cudaSuccess) e = r;
  return e;
}

cudaError_t prepare_band_kernels_rk() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_smem_mode_rk<MODE_DF>()) != cudaSuccess) e = r;
  if ((r = set_smem_mode_rk<MODE_F64>()) != cudaSuccess) e = r;
  if ((r = set_smem_mode_rk<MODE_F32>()) != cudaSuccess) e = r;
  if ((r = set_smem_mode_rk<MODE_BF16>()) != cudaSuccess) e = r;
  return e;
}

template <int MODE, int RK>
static void launch_rk(int group, const BandArgs& a, dim3 grid, int smem, cudaStream_t s) {
  constexpr int T = BandShape<MODE>::T;
  switch (group) {
    case 1: band_kernel<MODE, 1, false, RK><<<grid, T, smem, s>>>(a); break;
    case 2: band_kernel<MODE, 2, false, RK><<<grid, T, smem, s>>>(a); break;
    case 4: band_kernel<MODE, 4, false, RK><<<grid, T, smem, s>>>(a); break;
    default: band_kernel<MODE, 8, false, RK><<<grid, T, smem, s>>>(a); break;
  }
}

template <int MODE>
static void launch_mode_rk(const BandArgs& a, dim3 grid, int smem, cudaStream_t s) {
  switch (a.rk) {
    case 2: launch_rk<MODE, 2>(a.group, a, grid, smem, s); break;
    case 4: launch_rk<MODE, 4>(a.group, a, grid, smem, s); break;
    default: launch_rk<MODE, 8>(a.group, a, grid, smem, s); break;
  }
}

cudaError_t launch_band_rk(Arith arith, int storage, const BandArgs& a, int nbands, int smem, cudaStream_t s) {
  if (nbands <= 0) return cudaSuccess;
  if (a.rk != 2 && a.rk != 4 && a.rk != 8) return cudaErrorInvalidValue;
  dim3 grid(nbands);
  switch (mode_of(arith, storage)) {
    case MODE_DF: launch_mode_rk<MODE_DF>(a, grid, smem, s); break;
    case MODE_F64: launch_mode_rk<MODE_F64>(a, grid, smem, s); break;
    case MODE_F32: launch_mode_rk<MODE_F32>(a, grid, smem, s); break;
    default: launch_mode_rk<MODE_BF16>(a, grid, smem, s); break;
  }
  return cudaGetLastError();
}

}  // namespace csrc
