// Batched products: one persistent launch over the bands of many matrices.
//
// The host lists every (member, band) tile of a batch, grouped by lanes per row G
// and by strategy, largest bands first. Each CTA of the persistent kernel takes the
// next tile from a device counter and runs it with the member's arguments (its arrays,
// plan, x and y), so small and large matrices share the GPU in one launch. A second
// kernel then folds every member's spilled partial sums into its y. The host captures
// the sequence in a CUDA graph (batch executor in api.cpp).
#include "band.cuh"

namespace csrc {

template <int MODE, int G, bool ATOMIC>
__global__ void __launch_bounds__(BandShape<MODE>::T, BandShape<MODE>::kCtasPerSm)
    batch_band_kernel(const BandArgs* __restrict__ members, const int2* __restrict__ tiles, int ntiles,
                      int* __restrict__ next_tile) {
  __shared__ int tile;
  while (true) {
    if (threadIdx.x == 0) tile = atomicAdd(next_tile, 1);
    __syncthreads();
    const int t = tile;
    __syncthreads();
    if (t >= ntiles) break;
    const int2 mt = tiles[t];  // (member, band)
    const BandArgs a = members[mt.x];
    if (!band_body<MODE, G, ATOMIC, 1>(a, mt.y)) break;
  }
}

// y_m[row] += spilled partial sums of member m, for every receiving row of every member.
// offs[m] = first global index of member m (offs[nmembers] = total).
template <typename T>
__global__ void batch_accumulate_kernel(const AccArgs* __restrict__ members, const int64_t* __restrict__ offs,
                                        int nmembers, int64_t total) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nmembers - 1;  // member m with offs[m] <= g < offs[m+1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const AccArgs& m = members[lo];
  const int64_t i = g - offs[lo];
  const int row = m.acc_row[i];
  const T* spill = static_cast<const T*>(m.spill);
  T* y = static_cast<T*>(m.y);
  T s = y[row];
  const int e1 = m.acc_ptr[i + 1];
  for (int e = m.acc_ptr[i]; e < e1; ++e) s += spill[m.acc_src[e]];
  y[row] = s;
}

template <int MODE>
static cudaError_t set_batch_smem_mode() {
  cudaError_t e = cudaSuccess, r;
#define CSRC_B(GV, A)                                                                                         \
  r = cudaFuncSetAttribute(batch_band_kernel<MODE, GV, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                           band_smem_limit(MODE));                                                            \
  if (r != cudaSuccess) e = r;
  CSRC_B(1, false) CSRC_B(2, false) CSRC_B(4, false) CSRC_B(8, false)
  CSRC_B(1, true) CSRC_B(2, true) CSRC_B(4, true) CSRC_B(8, true)
#undef CSRC_B
  return e;
}

cudaError_t prepare_batch_kernels() {
  cudaError_t e = cudaSuccess, r;
  if ((r = set_batch_smem_mode<MODE_DF>()) != cudaSuccess) e = r;
  if ((r = set_batch_smem_mode<MODE_F64>()) != cudaSuccess) e = r;
  if ((r = set_batch_smem_mode<MODE_F32>()) != cudaSuccess) e = r;
  if ((r = set_batch_smem_mode<MODE_BF16>()) != cudaSuccess) e = r;
  return e;
}

template <int MODE>
static void launch_batch_mode(int group, bool atomic, dim3 grid, int smem, cudaStream_t s, const BandArgs* members,
                              const int2* tiles, int ntiles, int* next_tile) {
  constexpr int T = BandShape<MODE>::T;
#define CSRC_G(GV)                                                                                \
  if (atomic) batch_band_kernel<MODE, GV, true><<<grid, T, smem, s>>>(members, tiles, ntiles, next_tile); \
  else batch_band_kernel<MODE, GV, false><<<grid, T, smem, s>>>(members, tiles, ntiles, next_tile);
  switch (group) {
    case 1: CSRC_G(1) break;
    case 2: CSRC_G(2) break;
    case 4: CSRC_G(4) break;
    default: CSRC_G(8) break;
  }
#undef CSRC_G
}

cudaError_t launch_batch_band(Arith arith, int storage, int group, bool atomic, int grid, int smem, cudaStream_t s,
                              const BandArgs* members, const int2* tiles, int ntiles, int* next_tile) {
  if (ntiles <= 0 || grid <= 0) return cudaSuccess;
  switch (mode_of(arith, storage)) {
    case MODE_DF: launch_batch_mode<MODE_DF>(group, atomic, grid, smem, s, members, tiles, ntiles, next_tile); break;
    case MODE_F64: launch_batch_mode<MODE_F64>(group, atomic, grid, smem, s, members, tiles, ntiles, next_tile); break;
    case MODE_F32: launch_batch_mode<MODE_F32>(group, atomic, grid, smem, s, members, tiles, ntiles, next_tile); break;
    default: launch_batch_mode<MODE_BF16>(group, atomic, grid, smem, s, members, tiles, ntiles, next_tile); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_accumulate(int storage, const AccArgs* members, const int64_t* offs, int nmembers,
                                    int64_t total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int bs = 256;
  const unsigned grid = (unsigned)((total + bs - 1) / bs);
  if (storage == CSRC_F64) batch_accumulate_kernel<double><<<grid, bs, 0, s>>>(members, offs, nmembers, total);
  else batch_accumulate_kernel<float><<<grid, bs, 0, s>>>(members, offs, nmembers, total);
  return cudaGetLastError();
}

}  // namespace csrc
