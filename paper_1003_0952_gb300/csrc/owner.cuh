// The window strategy's product kernel for sm_103a: one CTA per band, one lane per
// window row (the owner-list layout of internal.h).
//
// Section 3.1 gives each thread a private buffer over its band's effective range and
// adds the buffers afterwards. Here the private buffer is the band's window: the x of
// every row the band touches sits in shared memory, and the partial sum of every row
// the band writes lives in one lane's registers. The plan has sorted the band's scatter
// (au[k] * x[i] into row ja[k], Fig. 2(a)) by target, so a window row's sum is one
// multiply-add chain over its list: the diagonal, its own lower pairs (the gather of
// Fig. 2(a)) and the pairs that scatter into it. No two lanes add into the same row,
// so there are no atomics and the result is the same in every run. Own rows are stored
// to y; rows below the band go to the spill buffer, which the accumulation kernel
// folds into y in band order (the "effective" accumulation of Section 3.1).
//
// A warp takes a slice of 32 window rows at a time; step m of the slice is the m-th
// entry of every lane whose list is longer than m, stored contiguously, so each load of
// a step is coalesced. Per entry the kernel does one multiply-add per column, in the
// storage's accumulation type (FP64 for FP64 storage, FP32 otherwise): the FP64 path
// spends exactly one FP64 instruction per stored value, which is what GB300's FP64
// pipe can sustain at HBM speed.
#pragma once

#include <cstdint>

#include "internal.h"

namespace csrc {

template <int ST>
struct OwnerTypes;
template <>
struct OwnerTypes<CSRC_F64> {
  using V = double;  // stored value
  using X = double;  // x and y
  using A = double;  // window x and accumulation
};
template <>
struct OwnerTypes<CSRC_F32> {
  using V = float;
  using X = float;
  using A = float;
};
template <>
struct OwnerTypes<CSRC_BF16> {
  using V = uint16_t;  // BF16 bits
  using X = float;
  using A = float;
};

__device__ __forceinline__ double owner_widen(double v) { return v; }
__device__ __forceinline__ float owner_widen(float v) { return v; }
__device__ __forceinline__ float owner_widen(uint16_t v) { return __uint_as_float((unsigned)v << 16); }

__device__ __forceinline__ double owner_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float owner_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Entries are read once: streaming loads through the non-coherent path.
__device__ __forceinline__ uint32_t owner_ld(const uint16_t* p) { return (uint32_t)__ldg(p); }
__device__ __forceinline__ double owner_ldv(const double* p) { return __ldg(p); }
__device__ __forceinline__ float owner_ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ uint16_t owner_ldv(const uint16_t* p) { return __ldg(p); }

// Entries loaded per lane before their multiply-adds (their load latencies overlap).
constexpr int owner_unroll(int rk) { return rk == 1 ? 8 : (rk == 2 ? 4 : 2); }

// Band b of the product described by a, run by the whole CTA.
template <int ST, int RK>
__device__ __forceinline__ void owner_body(const OwnerArgs& a, const int b) {
  using V = typename OwnerTypes<ST>::V;
  using X = typename OwnerTypes<ST>::X;
  using A = typename OwnerTypes<ST>::A;
  constexpr int U = owner_unroll(RK);
  extern __shared__ __align__(16) unsigned char owner_smem[];
  A* xs = reinterpret_cast<A*>(owner_smem);  // window: x of slot s, column c at s * RK + c
  const int4 bd = __ldg(a.band + b);
  const int r0 = bd.x, nown = bd.y, nsp = bd.z, sbase = bd.w;
  const X* __restrict__ x = static_cast<const X*>(a.x);
  const int ldx = a.ldx;
  const int tid = threadIdx.x;
  const int T = blockDim.x;

  // ---- the window's x: spill rows (gathered through their row list), then own rows
  for (int i = tid; i < nsp * RK; i += T) {
    const int s = i / RK, c = i % RK;
    xs[i] = (A)__ldg(x + (size_t)__ldg(a.spill_row + sbase + s) * ldx + c);
  }
  for (int i = tid; i < nown * RK; i += T) {
    const int s = i / RK, c = i % RK;
    xs[nsp * RK + i] = (A)__ldg(x + (size_t)(r0 + s) * ldx + c);
  }
  __syncthreads();

  // ---- the lists, one slice of 32 window rows per warp at a time
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int W = T >> 5;
  const uint16_t* __restrict__ S = a.S;
  const V* __restrict__ Vv = static_cast<const V*>(a.V);
  const int q1 = __ldg(a.band_slice + b + 1);
  for (int q = __ldg(a.band_slice + b) + warp; q < q1; q += W) {
    const uint32_t w = __ldg(a.lane + (size_t)q * kOwnerLanes + lane);
    const int len = (int)(w >> 16);
    const int slot = (int)(w & 0xffffu);
    const int maxlen = __shfl_sync(0xffffffffu, len, 0);  // lengths descend across the slice
    int64_t off = __ldg(a.slice_off + q);                  // first entry of the current step
    A acc[RK];
#pragma unroll
    for (int c = 0; c < RK; ++c) acc[c] = A(0);
    for (int m0 = 0; m0 < maxlen; m0 += U) {
      uint32_t sv[U];
      V vv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool act = m0 + u < len;
        const unsigned bal = __ballot_sync(0xffffffffu, act);
        sv[u] = 0u;
        vv[u] = V(0);
        if (act) {
          sv[u] = owner_ld(S + off + lane);
          vv[u] = owner_ldv(Vv + off + lane);
        }
        off += __popc(bal);
      }
      A xv[U][RK];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < RK; ++c) xv[u][c] = xs[sv[u] * RK + c];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (m0 + u < len) {
          const A v = owner_widen(vv[u]);
#pragma unroll
          for (int c = 0; c < RK; ++c) acc[c] = owner_fma(v, xv[u][c], acc[c]);
        }
      }
    }
    if (slot < nsp) {
      A* sp = static_cast<A*>(a.spill) + (size_t)(sbase + slot) * RK;
#pragma unroll
      for (int c = 0; c < RK; ++c) sp[c] = acc[c];
    } else if (slot != (int)kOwnerPadSlot) {
      X* yr = static_cast<X*>(a.y) + (size_t)(r0 + (slot - nsp)) * ldx;
#pragma unroll
      for (int c = 0; c < RK; ++c) yr[c] = (X)acc[c];
    }
  }
}

}  // namespace csrc
