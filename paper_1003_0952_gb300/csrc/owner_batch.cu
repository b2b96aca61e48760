// Batched products on the owner kernel: one launch over the (member, band, column tile)
// tiles of many matrices of one mode. Each CTA takes one tile, reads that member's
// arguments and runs the band (owner.cuh) on the tile's columns, so small and large
// matrices share the GPU in one launch; the hardware block scheduler balances the tiles.
#include "owner.cuh"

namespace csrc {

template <int MODE, int RK>
__global__ void __launch_bounds__(owner_threads(RK), owner_ctas_per_sm(RK))
    owner_batch_kernel(const OwnerArgs* __restrict__ members, const OwnerTile* __restrict__ tiles) {
  const OwnerTile t = tiles[blockIdx.x];
  OwnerArgs a = members[t.member];
  using X = typename OwnerTypes<MODE>::X;
  using A = typename OwnerTypes<MODE>::A;
  a.x = static_cast<const X*>(a.x) + t.col0;
  a.y = static_cast<X*>(a.y) + t.col0;
  a.spill = static_cast<A*>(a.spill) + t.col0;
  owner_body<MODE, RK>(a, t.band);
}

template <int MODE>
static cudaError_t prepare_batch_mode() {
  cudaError_t e = cudaSuccess, r;
#define CSRC_P(RKV)                                                                                  \
  r = cudaFuncSetAttribute(owner_batch_kernel<MODE, RKV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           owner_smem_budget(RKV));                                                  \
  if (r != cudaSuccess) e = r;
  CSRC_P(1) CSRC_P(2) CSRC_P(4) CSRC_P(8)
#undef CSRC_P
  return e;
}

cudaError_t prepare_owner_batch_kernels() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_batch_mode<OM_F64>()) != cudaSuccess) e = r;
  if ((r = prepare_batch_mode<OM_F32>()) != cudaSuccess) e = r;
  if ((r = prepare_batch_mode<OM_BF16>()) != cudaSuccess) e = r;
  if ((r = prepare_batch_mode<OM_F32_X64>()) != cudaSuccess) e = r;
  if ((r = prepare_batch_mode<OM_BF16_X64>()) != cudaSuccess) e = r;
  return e;
}

template <int MODE>
static void launch_batch_mode(int rk, const OwnerArgs* members, const OwnerTile* tiles, dim3 grid, int smem,
                              cudaStream_t s) {
  switch (rk) {
    case 1: owner_batch_kernel<MODE, 1><<<grid, owner_threads(1), smem, s>>>(members, tiles); break;
    case 2: owner_batch_kernel<MODE, 2><<<grid, owner_threads(2), smem, s>>>(members, tiles); break;
    case 4: owner_batch_kernel<MODE, 4><<<grid, owner_threads(4), smem, s>>>(members, tiles); break;
    default: owner_batch_kernel<MODE, 8><<<grid, owner_threads(8), smem, s>>>(members, tiles); break;
  }
}

cudaError_t launch_owner_batch(int mode, int rk, const OwnerArgs* members, const OwnerTile* tiles, int ntiles,
                               int smem, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const dim3 grid((unsigned)ntiles);
  switch (mode) {
    case OM_F64: launch_batch_mode<OM_F64>(rk, members, tiles, grid, smem, s); break;
    case OM_F32: launch_batch_mode<OM_F32>(rk, members, tiles, grid, smem, s); break;
    case OM_BF16: launch_batch_mode<OM_BF16>(rk, members, tiles, grid, smem, s); break;
    case OM_F32_X64: launch_batch_mode<OM_F32_X64>(rk, members, tiles, grid, smem, s); break;
    default: launch_batch_mode<OM_BF16_X64>(rk, members, tiles, grid, smem, s); break;
  }
  return cudaGetLastError();
}

}  // namespace csrc
