// Launchers of the window strategy's owner kernel (owner.cuh), the set-up kernel that
// lays the values out in list order, and the accumulation of the row-ordered spills.
#include "owner.cuh"

namespace csrc {

template <int MODE, int RK>
__global__ void __launch_bounds__(owner_threads(RK), owner_ctas_per_sm(RK)) owner_kernel(OwnerArgs a) {
  owner_body<MODE, RK>(a, blockIdx.x + a.band_offset);
}

// ---------------------------------------------------------------------------- value layout
// FP64 -> BF16 rounded to nearest, ties to even, from the double's bits in one step (no
// intermediate FP32 rounding). Subnormal BF16 results are produced; NaN stays NaN.
__device__ __forceinline__ uint16_t f64_to_bf16_rne(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 63);
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned long long mant = b & ((1ULL << 52) - 1);
  if (E == 0x7ff) return (uint16_t)((sign << 15) | 0x7f80u | (mant ? 0x40u : 0u));
  if (E == 0) return (uint16_t)(sign << 15);  // FP64 subnormals lie far below BF16's range
  const int e = E - 1023;                     // v = 1.m * 2^e
  const int keep = e >= -126 ? 7 : 7 - (-126 - e);  // fraction bits kept
  if (keep < -1) return (uint16_t)(sign << 15);
  const unsigned long long sig = (1ULL << 52) | mant;
  const int drop = 52 - keep;
  unsigned long long q = drop >= 64 ? 0ULL : (sig >> drop);
  const unsigned long long rem = drop >= 64 ? sig : (sig & ((1ULL << drop) - 1));
  const unsigned long long half = 1ULL << (drop - 1);
  if (rem > half || (rem == half && (q & 1ULL))) ++q;
  unsigned out;
  if (e >= -126) {
    int eb = e + 127;
    if (q >> 8) {  // the rounding carried into the next binade
      q >>= 1;
      ++eb;
    }
    if (eb >= 255) return (uint16_t)((sign << 15) | 0x7f80u);
    out = ((unsigned)eb << 7) | (unsigned)(q & 0x7f);
  } else {
    out = (unsigned)q;  // subnormal (q == 128 is the smallest normal)
  }
  return (uint16_t)((sign << 15) | out);
}

template <typename TI, typename TO>
__device__ __forceinline__ TO owner_convert(TI v) {
  if constexpr (std::is_same<TI, TO>::value) {
    return v;
  } else if constexpr (std::is_same<TO, float>::value) {
    return __double2float_rn(v);
  } else {
    return f64_to_bf16_rne(v);
  }
}

// out_a[e], out_t[e]: the value of list entry e for A x and for A^T x (al and au exchanged,
// Section 5). code = k << 2 | kind: kind 0 = ad[k], 1 = al[k], 2 = au[k].
template <typename TI, typename TO>
__global__ void owner_gather_kernel(const int64_t* __restrict__ code, int64_t count, const TI* __restrict__ al,
                                    const TI* __restrict__ au, const TI* __restrict__ ad, TO* __restrict__ out_a,
                                    TO* __restrict__ out_t) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = code[e];
    const int64_t k = c >> 2;
    const int kind = (int)(c & 3);
    const TI lo = kind == 1 ? al[k] : (kind == 2 ? au[k] : ad[k]);
    out_a[e] = owner_convert<TI, TO>(lo);
    if (out_t) out_t[e] = owner_convert<TI, TO>(kind == 1 ? au[k] : (kind == 2 ? al[k] : lo));
  }
}

cudaError_t launch_owner_gather(int in_bytes, int out_bytes, const int64_t* code, int64_t count, const void* al,
                                const void* au, const void* ad, void* out_a, void* out_t, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)std::max(sms, 1) * 16);
#define CSRC_GATHER(TI, TO)                                                                                    \
  owner_gather_kernel<TI, TO><<<(unsigned)blocks, 256, 0, s>>>(code, count, static_cast<const TI*>(al),       \
                                                              static_cast<const TI*>(au),                     \
                                                              static_cast<const TI*>(ad), static_cast<TO*>(out_a), \
                                                              static_cast<TO*>(out_t))
  if (in_bytes == 8 && out_bytes == 8) CSRC_GATHER(double, double);
  else if (in_bytes == 8 && out_bytes == 4) CSRC_GATHER(double, float);
  else if (in_bytes == 8 && out_bytes == 2) CSRC_GATHER(double, uint16_t);
  else if (in_bytes == 4 && out_bytes == 4) CSRC_GATHER(float, float);
  else if (in_bytes == 2 && out_bytes == 2) CSRC_GATHER(uint16_t, uint16_t);
  else return cudaErrorInvalidValue;
#undef CSRC_GATHER
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- accumulation
// y[row, c] += the row's spilled sums, in band order: the owner plans store them contiguously
// by receiving row (entries acc_ptr[i] .. acc_ptr[i+1] of the spill buffer, rk columns each).
template <typename TY, typename TS>
__global__ void owner_accumulate_kernel(int64_t nacc, int rk, int ldx, const int32_t* __restrict__ acc_row,
                                        const int32_t* __restrict__ acc_ptr, const TS* __restrict__ spill,
                                        TY* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nacc * rk) return;
  const int64_t i = t / rk;
  const int c = (int)(t % rk);
  TY* yp = y + (size_t)acc_row[i] * ldx + c;
  TY v = *yp;
  const int e1 = acc_ptr[i + 1];
  for (int e = acc_ptr[i]; e < e1; ++e) v += (TY)spill[(size_t)e * rk + c];
  *yp = v;
}

// The same over the members of a batch (one mode): item g is (member, row, column).
template <typename TY, typename TS>
__global__ void owner_batch_accumulate_kernel(const OwnerAccArgs* __restrict__ members,
                                              const int64_t* __restrict__ offs, int nmembers, int64_t total) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nmembers - 1;  // member m with offs[m] <= g < offs[m+1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const OwnerAccArgs& m = members[lo];
  const int64_t t = g - offs[lo];
  const int64_t i = t / m.rk;
  const int c = (int)(t % m.rk);
  TY* yp = static_cast<TY*>(m.y) + (size_t)m.acc_row[i] * m.ldx + c;
  const TS* spill = static_cast<const TS*>(m.spill);
  TY v = *yp;
  const int e1 = m.acc_ptr[i + 1];
  for (int e = m.acc_ptr[i]; e < e1; ++e) v += (TY)spill[(size_t)e * m.rk + c];
  *yp = v;
}

cudaError_t launch_owner_accumulate(int mode, int64_t nacc, int rk, int ldx, const int32_t* acc_row,
                                    const int32_t* acc_ptr, const void* spill, void* y, cudaStream_t s) {
  if (nacc <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((nacc * rk + 255) / 256);
  if (mode == OM_F64)
    owner_accumulate_kernel<double, double><<<grid, 256, 0, s>>>(nacc, rk, ldx, acc_row, acc_ptr,
                                                                 static_cast<const double*>(spill),
                                                                 static_cast<double*>(y));
  else if (mode == OM_F32 || mode == OM_BF16)
    owner_accumulate_kernel<float, float><<<grid, 256, 0, s>>>(nacc, rk, ldx, acc_row, acc_ptr,
                                                               static_cast<const float*>(spill),
                                                               static_cast<float*>(y));
  else
    owner_accumulate_kernel<double, float><<<grid, 256, 0, s>>>(nacc, rk, ldx, acc_row, acc_ptr,
                                                                static_cast<const float*>(spill),
                                                                static_cast<double*>(y));
  return cudaGetLastError();
}

cudaError_t launch_owner_batch_accumulate(int mode, const OwnerAccArgs* members, const int64_t* offs,
                                          int nmembers, int64_t total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (mode == OM_F64)
    owner_batch_accumulate_kernel<double, double><<<grid, 256, 0, s>>>(members, offs, nmembers, total);
  else if (mode == OM_F32 || mode == OM_BF16)
    owner_batch_accumulate_kernel<float, float><<<grid, 256, 0, s>>>(members, offs, nmembers, total);
  else
    owner_batch_accumulate_kernel<double, float><<<grid, 256, 0, s>>>(members, offs, nmembers, total);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- launchers
template <int MODE>
static cudaError_t prepare_owner_mode() {
  cudaError_t e = cudaSuccess, r;
#define CSRC_P(RKV)                                                                                  \
  r = cudaFuncSetAttribute(owner_kernel<MODE, RKV>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                           owner_smem_budget(RKV));                                                  \
  if (r != cudaSuccess) e = r;
  CSRC_P(1) CSRC_P(2) CSRC_P(4) CSRC_P(8)
#undef CSRC_P
  return e;
}

cudaError_t prepare_owner_kernels() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_owner_mode<OM_F64>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_mode<OM_F32>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_mode<OM_BF16>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_mode<OM_F32_X64>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_mode<OM_BF16_X64>()) != cudaSuccess) e = r;
  if ((r = prepare_owner_batch_kernels()) != cudaSuccess) e = r;
  return e;
}

template <int MODE>
static void launch_owner_mode(int rk, const OwnerArgs& a, dim3 grid, int smem, cudaStream_t s) {
  switch (rk) {
    case 1: owner_kernel<MODE, 1><<<grid, owner_threads(1), smem, s>>>(a); break;
    case 2: owner_kernel<MODE, 2><<<grid, owner_threads(2), smem, s>>>(a); break;
    case 4: owner_kernel<MODE, 4><<<grid, owner_threads(4), smem, s>>>(a); break;
    default: owner_kernel<MODE, 8><<<grid, owner_threads(8), smem, s>>>(a); break;
  }
}

cudaError_t launch_owner(int mode, int rk, const OwnerArgs& a, int nbands, int smem, cudaStream_t s) {
  if (nbands <= 0) return cudaSuccess;
  const dim3 grid((unsigned)nbands);
  switch (mode) {
    case OM_F64: launch_owner_mode<OM_F64>(rk, a, grid, smem, s); break;
    case OM_F32: launch_owner_mode<OM_F32>(rk, a, grid, smem, s); break;
    case OM_BF16: launch_owner_mode<OM_BF16>(rk, a, grid, smem, s); break;
    case OM_F32_X64: launch_owner_mode<OM_F32_X64>(rk, a, grid, smem, s); break;
    default: launch_owner_mode<OM_BF16_X64>(rk, a, grid, smem, s); break;
  }
  return cudaGetLastError();
}

}  // namespace csrc
