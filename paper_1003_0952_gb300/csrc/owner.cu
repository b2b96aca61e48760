// Launchers of the window strategy's owner kernel (owner.cuh) and the set-up kernel
// that lays the values out in list order.
#include "owner.cuh"

namespace csrc {

template <int ST, int RK>
__global__ void __launch_bounds__(kOwnerThreads, (RK <= 1 ? 4 : (RK <= 2 ? 2 : 1))) owner_kernel(OwnerArgs a) {
  owner_body<ST, RK>(a, blockIdx.x + a.band_offset);
}

// out_a[e], out_t[e]: the value of list entry e for A x and for A^T x (al and au exchanged,
// Section 5). code = k << 2 | kind: kind 0 = ad[k], 1 = al[k], 2 = au[k].
template <typename T>
__global__ void owner_gather_kernel(const int64_t* __restrict__ code, int64_t count, const T* __restrict__ al,
                                    const T* __restrict__ au, const T* __restrict__ ad, T* __restrict__ out_a,
                                    T* __restrict__ out_t) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = code[e];
    const int64_t k = c >> 2;
    const int kind = (int)(c & 3);
    const T lo = kind == 1 ? al[k] : (kind == 2 ? au[k] : ad[k]);
    out_a[e] = lo;
    if (out_t) out_t[e] = kind == 1 ? au[k] : (kind == 2 ? al[k] : lo);
  }
}

cudaError_t launch_owner_gather(int vbytes, const int64_t* code, int64_t count, const void* al, const void* au,
                                const void* ad, void* out_a, void* out_t, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)std::max(sms, 1) * 16);
#define CSRC_GATHER(T)                                                                                         \
  owner_gather_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(code, count, static_cast<const T*>(al),            \
                                                         static_cast<const T*>(au), static_cast<const T*>(ad), \
                                                         static_cast<T*>(out_a), static_cast<T*>(out_t))
  if (vbytes == 8) CSRC_GATHER(double);
  else if (vbytes == 4) CSRC_GATHER(float);
  else CSRC_GATHER(uint16_t);
#undef CSRC_GATHER
  return cudaGetLastError();
}

template <int ST>
static cudaError_t prepare_owner_storage() {
  cudaError_t e = cudaSuccess, r;
#define CSRC_P(RKV)                                                                                  \
  r = cudaFuncSetAttribute(owner_kernel<ST, RKV>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                           owner_smem_budget(RKV));                                                  \
  if (r != cudaSuccess) e = r;
  CSRC_P(1) CSRC_P(2) CSRC_P(4) CSRC_P(8)
#undef CSRC_P
  return e;
}

cudaError_t prepare_owner_kernels() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_owner_storage<CSRC_F64>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_storage<CSRC_F32>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_storage<CSRC_BF16>()) != cudaSuccess) e = r;
  return e;
}

template <int ST>
static void launch_owner_storage(int rk, const OwnerArgs& a, dim3 grid, int smem, cudaStream_t s) {
  switch (rk) {
    case 1: owner_kernel<ST, 1><<<grid, kOwnerThreads, smem, s>>>(a); break;
    case 2: owner_kernel<ST, 2><<<grid, kOwnerThreads, smem, s>>>(a); break;
    case 4: owner_kernel<ST, 4><<<grid, kOwnerThreads, smem, s>>>(a); break;
    default: owner_kernel<ST, 8><<<grid, kOwnerThreads, smem, s>>>(a); break;
  }
}

cudaError_t launch_owner(int storage, int rk, const OwnerArgs& a, int nbands, int smem, cudaStream_t s) {
  if (nbands <= 0) return cudaSuccess;
  const dim3 grid((unsigned)nbands);
  switch (storage) {
    case CSRC_F64: launch_owner_storage<CSRC_F64>(rk, a, grid, smem, s); break;
    case CSRC_F32: launch_owner_storage<CSRC_F32>(rk, a, grid, smem, s); break;
    default: launch_owner_storage<CSRC_BF16>(rk, a, grid, smem, s); break;
  }
  return cudaGetLastError();
}

}  // namespace csrc
