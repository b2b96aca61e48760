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
#include <type_traits>

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
template <>
struct OwnerTypes<OM_F32_X64> {  // reduced precision on double vectors
  using V = float;
  using X = double;
  using A = float;
};
template <>
struct OwnerTypes<OM_BF16_X64> {
  using V = uint16_t;
  using X = double;
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

// The RK columns of x of window slot s, with 16-byte shared-memory loads where they fit.
template <typename A, int RK>
__device__ __forceinline__ void owner_window_x(const A* xs, uint32_t s, A (&xv)[RK]) {
  constexpr int kVec = 16 / (int)sizeof(A);  // elements per 16-byte load
  if constexpr (RK % kVec == 0) {
    const uint4* p = reinterpret_cast<const uint4*>(xs + (size_t)s * RK);
#pragma unroll
    for (int q = 0; q < RK / kVec; ++q) {
      const uint4 w = p[q];
      A t[kVec];
      static_assert(sizeof(t) == sizeof(uint4), "16-byte vector");
      __builtin_memcpy(t, &w, sizeof(w));
#pragma unroll
      for (int c = 0; c < kVec; ++c) xv[q * kVec + c] = t[c];
    }
  } else {
#pragma unroll
    for (int c = 0; c < RK; ++c) xv[c] = xs[(size_t)s * RK + c];
  }
}

// Loads of steps m0 .. m0 + U - 1 of a slice for this lane (slot and value; 0 past the lane's
// list). off is the first entry of step m0 and is advanced past the batch: step m holds one
// entry for every lane whose list is longer than m, and those lanes come first.
template <typename V, int U>
__device__ __forceinline__ void owner_load_batch(const uint16_t* __restrict__ S, const V* __restrict__ Vv, int m0,
                                                 int len, int lane, int64_t& off, uint32_t (&sv)[U], V (&vv)[U]) {
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
}

// The multiply-adds of steps m0 .. m0 + U - 1 of this lane: x of each entry's slot from the
// window, one multiply-add per column.
template <typename A, typename V, int U, int RK>
__device__ __forceinline__ void owner_fma_batch(const A* xs, int m0, int len, const uint32_t (&sv)[U],
                                                const V (&vv)[U], A (&acc)[RK]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    A xv[RK];
    owner_window_x<A, RK>(xs, sv[u], xv);
    if (m0 + u < len) {
      const A v = owner_widen(vv[u]);
#pragma unroll
      for (int c = 0; c < RK; ++c) acc[c] = owner_fma(v, xv[c], acc[c]);
    }
  }
}

// Block loads: the 4 or 8 consecutive slots / values of one lane's block, with vector loads
// (the block starts on a multiple of its length in entries).
__device__ __forceinline__ void owner_ld_block(const uint16_t* p, uint32_t (&s)[4]) {
  const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
  s[0] = w.x & 0xffffu;
  s[1] = w.x >> 16;
  s[2] = w.y & 0xffffu;
  s[3] = w.y >> 16;
}
__device__ __forceinline__ void owner_ld_block(const uint16_t* p, uint32_t (&s)[8]) {
  const uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
  const unsigned q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    s[2 * i] = q[i] & 0xffffu;
    s[2 * i + 1] = q[i] >> 16;
  }
}
__device__ __forceinline__ void owner_ldv_block(const double* p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void owner_ldv_block(const float* p, float (&v)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void owner_ldv_block(const uint16_t* p, uint16_t (&v)[4]) {
  const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
  v[0] = (uint16_t)(w.x & 0xffffu);
  v[1] = (uint16_t)(w.x >> 16);
  v[2] = (uint16_t)(w.y & 0xffffu);
  v[3] = (uint16_t)(w.y >> 16);
}
__device__ __forceinline__ void owner_ldv_block(const uint16_t* p, uint16_t (&v)[8]) {
  const uint4 w = __ldg(reinterpret_cast<const uint4*>(p));
  const unsigned q[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = (uint16_t)(q[i] & 0xffffu);
    v[2 * i + 1] = (uint16_t)(q[i] >> 16);
  }
}

// Loads of block bi of a slice's regular part (every lane active): the lane's U steps lie
// side by side at pS / pV + 32 * U * bi, pS and pV pointing at the lane's first block.
template <typename V, int U>
__device__ __forceinline__ void owner_load_full(const uint16_t* __restrict__ pS, const V* __restrict__ pV, int bi,
                                                uint32_t (&sv)[U], V (&vv)[U]) {
  const size_t o = (size_t)kOwnerLanes * U * bi;
  owner_ld_block(pS + o, sv);
  owner_ldv_block(pV + o, vv);
}

// The multiply-adds of a full batch (every step active for this lane).
template <typename A, typename V, int U, int RK>
__device__ __forceinline__ void owner_fma_full(const A* xs, const uint32_t (&sv)[U], const V (&vv)[U],
                                               A (&acc)[RK]) {
  if constexpr (RK == 1) {
    // single columns: all U window loads first, so that their latencies overlap
    A xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = xs[sv[u]];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[0] = owner_fma(owner_widen(vv[u]), xv[u], acc[0]);
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      A xv[RK];
      owner_window_x<A, RK>(xs, sv[u], xv);
      const A v = owner_widen(vv[u]);
#pragma unroll
      for (int c = 0; c < RK; ++c) acc[c] = owner_fma(v, xv[c], acc[c]);
    }
  }
}

// The multiply-adds of a packed block of 8 steps with 2-byte (BF16) values: slot and value of
// step 2i + h are the low (h = 0) or high (h = 1) half of word i of s and v.
template <typename A, int RK>
__device__ __forceinline__ void owner_fma_packed(const A* xs, const uint4& s, const uint4& v, A (&acc)[RK]) {
  const unsigned sw[4] = {s.x, s.y, s.z, s.w};
  const unsigned vw[4] = {v.x, v.y, v.z, v.w};
  if constexpr (RK == 1) {
    A xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = xs[(sw[u >> 1] >> (16 * (u & 1))) & 0xffffu];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const A a = __uint_as_float((u & 1) ? (vw[u >> 1] & 0xffff0000u) : (vw[u >> 1] << 16));
      acc[0] = owner_fma(a, xv[u], acc[0]);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      A xv[RK];
      owner_window_x<A, RK>(xs, (sw[u >> 1] >> (16 * (u & 1))) & 0xffffu, xv);
      const A a = __uint_as_float((u & 1) ? (vw[u >> 1] & 0xffff0000u) : (vw[u >> 1] << 16));
#pragma unroll
      for (int c = 0; c < RK; ++c) acc[c] = owner_fma(a, xv[c], acc[c]);
    }
  }
}

// Steps of a ragged-tail batch (the regular part's batches are blocks of owner_block(ST, RK)).
constexpr int kOwnerRaggedBatch = 4;

// Band b of the product described by a, run by the whole CTA.
template <int ST, int RK>
__device__ __forceinline__ void owner_body(const OwnerArgs& a, const int b) {
  using V = typename OwnerTypes<ST>::V;
  using X = typename OwnerTypes<ST>::X;
  using A = typename OwnerTypes<ST>::A;
  constexpr int U = owner_block(ST, RK);  // steps per block of the regular part
  constexpr int R = kOwnerRaggedBatch;
  extern __shared__ __align__(16) unsigned char owner_smem[];
  A* xs = reinterpret_cast<A*>(owner_smem);  // window: x of slot s, column c at s * RK + c
  const int4 bd = __ldg(a.band + b);
  const int r0 = bd.x, nown = bd.y, nsp = bd.z, sbase = bd.w;
  const X* __restrict__ x = static_cast<const X*>(a.x);
  const int ldx = a.ldx;
  const int tid = threadIdx.x;
  const int T = blockDim.x;

  // ---- the window's x: spill rows (gathered through their row list), then own rows; each
  // thread issues kWin loads before it stores any, so that their latencies overlap
  constexpr int kWin = 8;
  const int nsx = nsp * RK, nox = nown * RK;
  for (int i0 = tid; i0 < nsx + nox; i0 += kWin * T) {
    A v[kWin];
    int row[kWin];
#pragma unroll
    for (int u = 0; u < kWin; ++u) {
      const int i = i0 + u * T;
      row[u] = i < nsx ? __ldg(a.spill_row + sbase + i / RK) : r0 + (i - nsx) / RK;
    }
#pragma unroll
    for (int u = 0; u < kWin; ++u) {
      const int i = i0 + u * T;
      const int c = (i < nsx ? i : i - nsx) % RK;
      v[u] = i < nsx + nox ? (A)__ldg(x + (size_t)row[u] * ldx + c) : A(0);
    }
#pragma unroll
    for (int u = 0; u < kWin; ++u) {
      const int i = i0 + u * T;
      if (i < nsx + nox) xs[i] = v[u];
    }
  }
  __syncthreads();

  // ---- the lists, one slice of 32 window rows per warp at a time
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int W = T >> 5;
  const uint16_t* __restrict__ S = a.S;
  const V* __restrict__ Vv = static_cast<const V*>(a.V);
  const int q1 = __ldg(a.band_slice + b + 1);
  // a slice's lane word and list offset are loaded one slice ahead, so that a warp's next
  // slice starts with its list loads (short lists, as in wide-bandwidth orderings, make
  // many slices of a few steps each)
  int q = __ldg(a.band_slice + b) + warp;
  uint32_t wn = 0;
  int64_t basen = 0;
  if (q < q1) {
    wn = __ldg(a.lane + (size_t)q * kOwnerLanes + lane);
    basen = __ldg(a.slice_off + q);
  }
  for (; q < q1; q += W) {
    const uint32_t w = wn;
    const int64_t base = basen;
    if (q + W < q1) {
      wn = __ldg(a.lane + (size_t)(q + W) * kOwnerLanes + lane);
      basen = __ldg(a.slice_off + q + W);
    }
    const int len = (int)(w >> 16);
    const int slot = (int)(w & 0xffffu);
    // a spill row's position in the spill buffer, read now and used after the list
    const int spos = slot < nsp ? __ldg(a.spill_pos + sbase + slot) : 0;
    // lengths descend across the slice: lane 0 has the longest list, lane 31 the shortest
    const int maxlen = __shfl_sync(0xffffffffu, len, 0);
    const int minlen = __shfl_sync(0xffffffffu, len, 31);
    A acc[RK];
#pragma unroll
    for (int c = 0; c < RK; ++c) acc[c] = A(0);
    // Regular part: the steps of whole blocks below minlen hold all 32 lanes, each lane's U
    // steps of a block side by side, so each lane reads a block with vector loads. Two blocks
    // are in flight in a ring of registers: a block's loads are issued two compute phases before
    // its multiply-adds, so that memory latency overlaps this and other warps' arithmetic.
    const uint16_t* __restrict__ pS = S + base + U * lane;
    const V* __restrict__ pV = Vv + base + U * lane;
    const int nfull = minlen / U;  // batches of U steps with every lane active
    if constexpr (sizeof(V) == 2 && U == 8) {
      // 2-byte values: a block is one 16-byte word of slots and one of values, kept packed in
      // the ring (8 registers per block) and unpacked at the multiply-adds
      uint4 s0 = make_uint4(0, 0, 0, 0), s1 = s0, v0 = s0, v1 = s0;
      const uint4* __restrict__ qS = reinterpret_cast<const uint4*>(pS);
      const uint4* __restrict__ qV = reinterpret_cast<const uint4*>(pV);
      if (nfull > 0) {
        s0 = __ldg(qS);
        v0 = __ldg(qV);
      }
      if (nfull > 1) {
        s1 = __ldg(qS + kOwnerLanes);
        v1 = __ldg(qV + kOwnerLanes);
      }
      int bi = 0;
      for (; bi + 1 < nfull; bi += 2) {
        owner_fma_packed<A, RK>(xs, s0, v0, acc);
        if (bi + 2 < nfull) {
          s0 = __ldg(qS + (size_t)kOwnerLanes * (bi + 2));
          v0 = __ldg(qV + (size_t)kOwnerLanes * (bi + 2));
        }
        owner_fma_packed<A, RK>(xs, s1, v1, acc);
        if (bi + 3 < nfull) {
          s1 = __ldg(qS + (size_t)kOwnerLanes * (bi + 3));
          v1 = __ldg(qV + (size_t)kOwnerLanes * (bi + 3));
        }
      }
      if (bi < nfull) owner_fma_packed<A, RK>(xs, s0, v0, acc);
    } else {
      uint32_t s0[U], s1[U];
      V v0[U], v1[U];
      if (nfull > 0) owner_load_full<V, U>(pS, pV, 0, s0, v0);
      if (nfull > 1) owner_load_full<V, U>(pS, pV, 1, s1, v1);
      int bi = 0;
      for (; bi + 1 < nfull; bi += 2) {
        owner_fma_full<A, V, U, RK>(xs, s0, v0, acc);
        if (bi + 2 < nfull) owner_load_full<V, U>(pS, pV, bi + 2, s0, v0);
        owner_fma_full<A, V, U, RK>(xs, s1, v1, acc);
        if (bi + 3 < nfull) owner_load_full<V, U>(pS, pV, bi + 3, s1, v1);
      }
      if (bi < nfull) owner_fma_full<A, V, U, RK>(xs, s0, v0, acc);
    }
    // Ragged tail: steps m >= nfull * U, where lanes whose list has ended drop out; step m
    // holds one entry for each lane whose list is longer than m (those lanes come first).
    int64_t off = base + (int64_t)kOwnerLanes * nfull * U;
    for (int m0 = nfull * U; m0 < maxlen; m0 += R) {
      uint32_t sv[R];
      V vv[R];
      owner_load_batch<V, R>(S, Vv, m0, len, lane, off, sv, vv);
      owner_fma_batch<A, V, R, RK>(xs, m0, len, sv, vv, acc);
    }
    if (slot < nsp) {
      A* sp = static_cast<A*>(a.spill) + (size_t)spos * a.lds;
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
