// The band kernel of the CSRC products (Fig. 2(a)) for sm_103a, shared by the
// single-vector product (kernels.cu, RK = 1) and the several-right-hand-side
// product (spmm.cu, RK = 2, 4 or 8 columns per pass).
//
// One CTA runs one row band [r0, r1) of the window plan. The band's stored
// pairs are the contiguous slice [ia[r0], ia[r1]) of ja / al / au. They are
// streamed into a ring of shared-memory stages by TMA bulk copies
// (cp.async.bulk, completion counted on an mbarrier per stage), issued by one
// thread while the others compute. A stage holds whole consecutive rows (the
// host cuts the band into stages; a row longer than a stage is cut too). Each
// row of a stage is taken by a group of G lanes that stride through its pairs,
// so a row's gathered sum stays in registers until the row ends.
//
// Every pair k of row i gathers al[k]*x[ja[k]] into row i and scatters
// au[k]*x[i] into row ja[k]. Both land in a private window in shared memory,
// the GPU form of the local buffers of Section 3.1: it holds the rows this
// band writes, its own rows and every row below r0 that ja reaches (its
// "effective range"), kept at 64-row page granularity behind a page table.
// x for those rows (RK columns of them) is staged in the same window, so
// gathers read shared memory too. When the stream ends:
//  - window strategy: own rows are stored to y, and rows below r0 go to a
//    compact spill buffer. A separate accumulation kernel folds the spills into
//    y, in band order, like the "effective" accumulation of Section 3.1.
//  - atomic strategy (RK = 1): y was zeroed, and every window row is added to y
//    with a global atomic (executed in L2). Pages outside the window (plans with
//    overflow) scatter straight to y with the same atomics.
//
// Arithmetic by mode:
//  - MODE_DF: FP64 storage and vectors. The gather runs on the FP64 pipe (one
//    FMA per pair and column, the row sum in a double register). The scatter
//    product and the window sums use double-float arithmetic on the FP32 pipes
//    (df32.cuh): GB300 runs FP64 at a small fraction of its FP32 rate, so one FP64
//    operation per pair is what that pipe can take at HBM speed.
//  - MODE_F64: FP64 storage, every operation on the FP64 pipe.
//  - MODE_F32: FP32 storage, FP32 vectors and accumulation.
//  - MODE_BF16: BF16 storage, FP32 vectors and accumulation.
#pragma once

#include <cstdint>
#include <type_traits>

#include "df32.cuh"
#include "internal.h"

namespace csrc {


// ---------------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0u;
}

// Bounded wait for the phase with the given parity: gives up after `limit` SM clock
// cycles (by default about two seconds at ~2 GHz) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = 4000000000LL) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Shared-memory reads by the generic proxy before async-proxy (TMA) writes to the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// TMA bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completion signalled on the mbarrier as transaction bytes.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// ---------------------------------------------------------------------------- per-mode types
template <int MODE>
struct Traits;

template <>
struct Traits<MODE_DF> {
  using V = double;  // stored value
  using X = double;  // vector element
};
template <>
struct Traits<MODE_F64> {
  using V = double;
  using X = double;
};
template <>
struct Traits<MODE_F32> {
  using V = float;
  using X = float;
};
template <>
struct Traits<MODE_BF16> {
  using V = uint16_t;
  using X = float;
};

__device__ __forceinline__ float bf16_to_f32(uint16_t v) { return __uint_as_float((unsigned)v << 16); }

template <int MODE>
__device__ __forceinline__ float as_f32(typename Traits<MODE>::V v) {
  if constexpr (MODE == MODE_BF16) {
    return bf16_to_f32(v);
  } else {
    return static_cast<float>(v);
  }
}

// Window of a band in shared memory: x of every slot, then the accumulators.
template <int MODE>
struct Window;

template <>
struct Window<MODE_DF> {
  double* xs;
  float* whi;
  float* wlo;
  __device__ void bind(unsigned char* s, int nslots) {
    xs = reinterpret_cast<double*>(s);
    whi = reinterpret_cast<float*>(xs + nslots);
    wlo = whi + nslots;
  }
  __device__ void zero(int s) {
    whi[s] = 0.f;
    wlo[s] = 0.f;
  }
  __device__ double value(int s) const { return (double)whi[s] + (double)wlo[s]; }
};
template <>
struct Window<MODE_F64> {
  double* xs;
  double* w;
  __device__ void bind(unsigned char* s, int nslots) {
    xs = reinterpret_cast<double*>(s);
    w = xs + nslots;
  }
  __device__ void zero(int s) { w[s] = 0.0; }
  __device__ double value(int s) const { return w[s]; }
};
template <int MODE>
struct Window {  // MODE_F32 and MODE_BF16
  float* xs;
  float* w;
  __device__ void bind(unsigned char* s, int nslots) {
    xs = reinterpret_cast<float*>(s);
    w = xs + nslots;
  }
  __device__ void zero(int s) { w[s] = 0.f; }
  __device__ float value(int s) const { return w[s]; }
};

// Scatter factor x[i] of the current row, as the mode multiplies with it.
template <int MODE>
struct RowX {
  using type = typename Traits<MODE>::X;
};
template <>
struct RowX<MODE_DF> {
  using type = df32;
};


// ---------------------------------------------------------------------------- the band kernel
// One unit of B consecutive rows r .. r+B-1 of a node block (B degrees of freedom per
// node, dense B-by-B node blocks): row r+t holds the L0 pairs of row r's columns (all
// below r), in the same order, then t pairs for columns r .. r+t-1. The host checked that
// structure for every unit of the matrix. A group of G lanes takes the unit: per shared
// column it looks up the window slot and loads x once, gathers into the B row sums, and
// scatters the sum of the B products with one window update. The unit's pairs are whole
// in the ring stage (s* point at the stage, indexed by pair number).
template <int MODE, int G, int B>
__device__ __forceinline__ void block_unit(int r, const int32_t* s_ia, const int32_t* sja,
                                           const typename Traits<MODE>::V* sal, const typename Traits<MODE>::V* sau,
                                           Window<MODE>& win, const int32_t* tab, int plo, int ntab, int gl,
                                           unsigned gmask, unsigned& bad) {
  using V = typename Traits<MODE>::V;
  using X = typename Traits<MODE>::X;
  using XR = typename RowX<MODE>::type;
  auto lookup = [&](int j) -> int {
    const int t = (j >> kPageShift) - plo;
    const int pb = (unsigned)t < (unsigned)ntab ? tab[t] : -1;
    bad |= pb < 0 ? 4u : 0u;
    return max(pb, 0) + (j & (kPageRows - 1));
  };
  int kbt[B], rs[B];
  XR xr[B];
  X acc[B];
#pragma unroll
  for (int t = 0; t < B; ++t) {
    kbt[t] = s_ia[r + t];
    rs[t] = lookup(r + t);
    if constexpr (MODE == MODE_DF) {
      xr[t] = df_split<true>(win.xs[rs[t]], &bad);
    } else {
      xr[t] = win.xs[rs[t]];
    }
    acc[t] = X(0);
  }
  const int L0 = s_ia[r + 1] - kbt[0];
  // shared columns
  for (int m = gl; m < L0; m += G) {
    const int sv = lookup(sja[kbt[0] + m]);
    const X xj = win.xs[sv];
    if constexpr (MODE == MODE_DF) {
      df32 p;
#pragma unroll
      for (int t = 0; t < B; ++t) {
        acc[t] = fma(sal[kbt[t] + m], xj, acc[t]);
        const df32 q = df_mul(df_split<false>(sau[kbt[t] + m], nullptr), xr[t]);
        if (t == 0) p = q; else df_acc(p, q);
      }
      df_atomic_add(win.whi + sv, win.wlo + sv, p);
    } else if constexpr (MODE == MODE_F64) {
      double p = 0.0;
#pragma unroll
      for (int t = 0; t < B; ++t) {
        acc[t] = fma(sal[kbt[t] + m], xj, acc[t]);
        p = fma(sau[kbt[t] + m], xr[t], p);
      }
      atomicAdd(win.w + sv, p);
    } else {
      float p = 0.f;
#pragma unroll
      for (int t = 0; t < B; ++t) {
        acc[t] = __fmaf_rn(as_f32<MODE>(sal[kbt[t] + m]), xj, acc[t]);
        p = __fmaf_rn(as_f32<MODE>(sau[kbt[t] + m]), xr[t], p);
      }
      atomicAdd(win.w + sv, p);
    }
  }
  // the unit's own block: pair q of row r+t's tail couples rows r+t and r+q (q < t)
#pragma unroll
  for (int t = 1; t < B; ++t) {
#pragma unroll
    for (int q = 0; q < t; ++q) {
      if (gl == ((t * (t - 1) / 2 + q) % G)) {
        const int k = kbt[t] + L0 + q;
        const int sv = lookup(sja[k]);
        if constexpr (MODE == MODE_DF) {
          acc[t] = fma(sal[k], win.xs[sv], acc[t]);
          df_atomic_add(win.whi + sv, win.wlo + sv, df_mul(df_split<false>(sau[k], nullptr), xr[t]));
        } else if constexpr (MODE == MODE_F64) {
          acc[t] = fma(sal[k], win.xs[sv], acc[t]);
          atomicAdd(win.w + sv, sau[k] * xr[t]);
        } else {
          acc[t] = __fmaf_rn(as_f32<MODE>(sal[k]), win.xs[sv], acc[t]);
          atomicAdd(win.w + sv, __fmul_rn(as_f32<MODE>(sau[k]), xr[t]));
        }
      }
    }
  }
  // the B row sums, reduced across the group and added once each
#pragma unroll
  for (int t = 0; t < B; ++t) {
    if constexpr (MODE == MODE_DF) {
      df32 v = df_split<false>(acc[t], nullptr);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        df32 u;
        u.hi = __shfl_xor_sync(gmask, v.hi, o, G);
        u.lo = __shfl_xor_sync(gmask, v.lo, o, G);
        df_acc(v, u);
      }
      if (gl == 0) df_atomic_add(win.whi + rs[t], win.wlo + rs[t], v);
    } else {
      X v = acc[t];
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, G);
      if (gl == 0) atomicAdd(win.w + rs[t], v);
    }
  }
}

// One band b of the product described by a, run by the whole CTA. The CTA may run
// several bands one after another (the batched kernel): its mbarriers are initialised at
// the start and invalidated at the end. Returns false when a bounded wait ran out (the
// status word says so and the CTA must not run further bands).
template <int MODE, int G, bool ATOMIC, int RK, int B = 1>
__device__ __forceinline__ bool band_body(const BandArgs& a, const int b) {
  using Sh = BandShape<MODE>;
  using V = typename Traits<MODE>::V;
  using X = typename Traits<MODE>::X;
  using XR = typename RowX<MODE>::type;
  constexpr int T = band_threads(G, B, RK);
  constexpr int NS = Sh::NS;
  constexpr int SP = Sh::kSlotPairs;  // pairs per ring slot
  constexpr int VB = (int)sizeof(V);
  constexpr int XB = (int)sizeof(X);
  static_assert(!ATOMIC || RK == 1, "the atomic strategy runs single vectors");
  static_assert(B == 1 || (RK == 1 && !ATOMIC), "row blocks run single vectors with the window strategy");
  // plain rows with the window strategy (any number of columns) read window slots from the ring
  constexpr bool LOCAL = B == 1 && !ATOMIC;
  using SV = std::conditional_t<LOCAL && MODE == MODE_DF, df32, V>;  // scatter operand as streamed

  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int r0 = a.band_row[b];
  const int r1 = a.band_row[b + 1];
  const int plo = a.band_plo[b];
  const int ntab = a.band_ntab[b];
  const int wp0 = a.band_wp[b];
  const int np = a.band_wp[b + 1] - wp0;
  const int nslots = np << kPageShift;
  const int st0 = a.band_stage[b];
  const int st1 = a.band_stage[b + 1] - 1;  // index of the band's end entry
  const int nstages = st1 - st0;
  const int ldx = a.ldx;                    // row stride of x and y (elements)
  // numerically symmetric storage (Section 2.2): al is also the scatter operand, so the ring
  // carries no au (the host passes the same array for both)
  const bool sym = a.au == a.al;

  // ---- shared memory: [mbarriers][ring slots][x][sums][page table][ia][stage_k][stage_r]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);  // full[NS], empty[NS], setup
  unsigned char* ring = smem + kRingOffset;
  int32_t* ring_ja = reinterpret_cast<int32_t*>(ring);                    // [NS][SP]
  V* ring_al = reinterpret_cast<V*>(ring + (size_t)NS * SP * 4);          // [NS][SP]
  V* ring_au = reinterpret_cast<V*>(ring + (size_t)NS * SP * (4 + VB));   // [NS][SP]
  unsigned char* rest = ring + Sh::ring_bytes();
  const BandLayout L = BandLayout::make(nslots, RK * window_x_bytes(MODE), RK * window_acc_bytes(MODE), ntab, r0,
                                        r1, st0, st1);
  Window<MODE> win;  // element (slot, column c) at slot * RK + c
  win.bind(rest + L.xs, nslots * RK);
  int32_t* tab = reinterpret_cast<int32_t*>(rest + L.tab);
  const int ia_base = r0 & ~3;
  const int st_base = st0 & ~3;
  const int32_t* s_ia = reinterpret_cast<const int32_t*>(rest + L.ia) - ia_base;  // s_ia[r] = ia[r]
  const int32_t* s_sk = reinterpret_cast<const int32_t*>(rest + L.sk) - st_base;  // s_sk[st] = stage_k[st]
  const int32_t* s_sr = reinterpret_cast<const int32_t*>(rest + L.sr) - st_base;

  const uint32_t bar_full = smem_addr(bars);
  const uint32_t bar_empty = smem_addr(bars + NS);
  const uint32_t bar_setup = smem_addr(bars + 2 * NS);
  // ring stage s: pairs [ks & ~7, ceil8(ke)) (16-byte aligned for every value type; the
  // stored arrays are padded so the rounded-up end stays inside them)
  auto issue = [&](int s, int ks, int ke) {
    const int slot = s % NS;
    ks &= ~(kPairAlign - 1);
    ke = (ke + kPairAlign - 1) & ~(kPairAlign - 1);
    const int cnt = ke - ks;  // <= kStageCap + 16 (the host caps a stage's pairs)
    const uint32_t bar = bar_full + 8u * slot;
    const uint32_t ib = a.ja16 ? 2u : 4u;  // index bytes per pair
    mbar_arrive_expect_tx(bar, (uint32_t)cnt * (ib + (uint32_t)((sym ? 1 : 2) * VB)));
    if (a.ja16)
      bulk_copy_g2s(smem_addr(ring_ja + (size_t)slot * SP), a.ja16 + ks, (uint32_t)cnt * 2u, bar);
    else
      bulk_copy_g2s(smem_addr(ring_ja + (size_t)slot * SP), a.ja + ks, (uint32_t)cnt * 4u, bar);
    bulk_copy_g2s(smem_addr(ring_al + (size_t)slot * SP), static_cast<const V*>(a.al) + ks, (uint32_t)cnt * VB, bar);
    if (!sym)
      bulk_copy_g2s(smem_addr(ring_au + (size_t)slot * SP), static_cast<const V*>(a.au) + ks, (uint32_t)cnt * VB, bar);
  };

  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(bar_full + 8u * i, 1u);
      mbar_init(bar_empty + 8u * i, (uint32_t)(T / 32));
    }
    mbar_init(bar_setup, 1u);
    mbar_init_fence();
  }
  __syncthreads();

  // ---- phase 1: warp 0 starts the copies (first ring stages, the band's ia slice and
  // stage table, x of every full window page when its rows are contiguous in memory);
  // the other warps clear the sums and build the page table meanwhile.
  unsigned bad = 0u;
  int issued = 0;
  const bool x_pages_bulk = a.x_bulk && ldx == RK;
  if (warp == 0) {
    if (lane == 0) {
      for (; issued < NS && issued < nstages; ++issued)
        issue(issued, __ldg(a.stage_k + st0 + issued), __ldg(a.stage_k + st0 + issued + 1));
    }
    uint32_t bytes = 0;
    if (lane == 0) {
      const uint32_t nia = (uint32_t)(L.sk - L.ia), nst = (uint32_t)(L.sr - L.sk);
      bulk_copy_g2s(smem_addr(rest + L.ia), a.ia + ia_base, nia, bar_setup);
      bulk_copy_g2s(smem_addr(rest + L.sk), a.stage_k + st_base, nst, bar_setup);
      bulk_copy_g2s(smem_addr(rest + L.sr), a.stage_r + st_base, nst, bar_setup);
      bytes += nia + 2 * nst;
    }
    if (x_pages_bulk) {
      for (int q = lane; q < np; q += 32) {
        const int page = __ldg(a.wpage + wp0 + q);
        if ((page + 1) * kPageRows <= a.n) {
          bulk_copy_g2s(smem_addr(win.xs + (size_t)(q << kPageShift) * RK),
                        static_cast<const X*>(a.x) + (size_t)(page << kPageShift) * RK,
                        (uint32_t)(kPageRows * RK * XB), bar_setup);
          bytes += (uint32_t)(kPageRows * RK * XB);
        }
      }
    }
    // every copy is issued before the one arrival that closes the phase
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(bar_setup, bytes);
  }
  for (int t = tid; t < ntab; t += T) tab[t] = -1;
  for (int s = tid; s < nslots * RK; s += T) win.zero(s);
  __syncthreads();
  for (int q = tid; q < np; q += T) {
    const int page = __ldg(a.wpage + wp0 + q);
    const int t = page - plo;
    if ((unsigned)t < (unsigned)ntab) {
      tab[t] = q << kPageShift;
    } else {
      bad |= 4u;
    }
    // pages without a bulk copy (strided or unaligned x, or a page running past n)
    if (!x_pages_bulk || (page + 1) * kPageRows > a.n) {
      for (int e = 0; e < kPageRows; ++e) {
        const int j = (page << kPageShift) + e;
#pragma unroll
        for (int c = 0; c < RK; ++c)
          win.xs[(size_t)((q << kPageShift) + e) * RK + c] =
              j < a.n ? __ldg(static_cast<const X*>(a.x) + (size_t)j * ldx + c) : X(0);
      }
    }
  }
  bool timed_out = !mbar_wait(bar_setup, 0u);
  __syncthreads();

  // slot of row j in the window, or -1 (page outside the window)
  auto slot_of = [&](int j) -> int {
    const int t = (j >> kPageShift) - plo;
    if ((unsigned)t >= (unsigned)ntab) return -1;
    const int base = tab[t];
    return base < 0 ? -1 : base + (j & (kPageRows - 1));
  };

  // ---- phase 2: stream the band's pairs, one row per group of G lanes. The groups of a
  // warp take rows D = G apart: warp w's groups g take rows (w / G) * 32 + g * G + w % G, so
  // the 32 rows that warps w0..w0+G-1 share form one block of consecutive rows. Their ring
  // slices, x entries and window slots fall on nearby addresses while a warp's rows stay far
  // enough apart not to share a node (and its targets) in 3-DOF meshes. Measured against
  // spreading rows one warp apart (rows g * W + w): band kernel 15-57 % faster for 1-4 lanes
  // per row (Q1 scalar, P1 and tetrahedral meshes), 7-10 % for q1v_96 (16 lanes).
  constexpr int W = T / 32, GPW = 32 / G;
  constexpr int D = G;
  static_assert(W % D == 0, "the row spacing divides the warp count");
  const int rowoff = (warp / D) * (D * GPW) + ((lane / G) % GPW) * D + (warp % D);
  const int gl = lane % G;  // lane within the group
  // lanes of this group, for the shuffles that sum a row over the group
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  for (int s = 0; s < nstages && !timed_out; ++s) {
    const int slot = s % NS;
    const uint32_t parity = (uint32_t)((s / NS) & 1);
    const int ks = s_sk[st0 + s];
    const int ke = s_sk[st0 + s + 1];
    const int r = s_sr[st0 + s] + rowoff * B;  // first row of this group's unit (B rows)
    int kb = 0, kx = 0;  // this group's pairs [kb, kx) of row r inside the stage
    if (r < r1) {
      kb = max(s_ia[r], ks);
      kx = min(s_ia[r + 1], ke);
    }
    if (!mbar_wait(bar_full + 8u * slot, parity)) {
      timed_out = true;
      break;
    }
    if constexpr (B > 1) {
      // stages hold whole units: this group's unit is in stage s when it starts before its end
      if (r < r1 && s_ia[r] < ke) block_unit<MODE, G, B>(r, s_ia, ring_ja + (size_t)slot * SP - (ks & ~(kPairAlign - 1)),
                                         ring_al + (size_t)slot * SP - (ks & ~(kPairAlign - 1)),
                                         (sym ? ring_al : ring_au) + (size_t)slot * SP - (ks & ~(kPairAlign - 1)),
                                         win, tab, plo,
                                         ntab, gl, gmask, bad);
    } else if (kb < kx) {  // the whole group enters (its lanes meet in the shuffles below)
      const int base = ks & ~(kPairAlign - 1);
      const int32_t* sja = ring_ja + (size_t)slot * SP - base;
      const V* sal = ring_al + (size_t)slot * SP - base;
      const V* sau = (sym ? ring_al : ring_au) + (size_t)slot * SP - base;
      int rslot = slot_of(r);
      if (rslot < 0) {
        bad |= 4u;
        rslot = 0;
      }
      XR xr[RK];
#pragma unroll
      for (int c = 0; c < RK; ++c) {
        if constexpr (MODE == MODE_DF) {
          xr[c] = df_split<true>(win.xs[rslot * RK + c], &bad);
        } else {
          xr[c] = win.xs[rslot * RK + c];
        }
      }
      X acc[RK];
#pragma unroll
      for (int c = 0; c < RK; ++c) acc[c] = X(0);
      if constexpr (LOCAL) {
        // Plain rows, window strategy: the ring carries each pair's window slot (the host
        // wrote it in place of the column), so no page lookup is needed; slots are clamped
        // to the window all the same. With MODE_DF the scatter operand arrives pre-split
        // into double-float pairs. A pair's slot and split serve all RK columns. The U
        // unrolled loads may run past the row's last pair (up to (U-1)*G pairs past the
        // stage): they stay inside shared memory (the ring's next slot or array, or the
        // window after the last one) and their values are never used.
        constexpr int U = RK == 1 ? (G == 16 ? 3 : 4) : (RK >= 4 ? 1 : 4 / RK);
        const unsigned smax = (unsigned)(nslots - 1);
        const SV* ssc = reinterpret_cast<const SV*>(ring_au + (size_t)slot * SP) - (ks & ~(kPairAlign - 1));
        const uint16_t* s16 = reinterpret_cast<const uint16_t*>(ring_ja + (size_t)slot * SP) - (ks & ~(kPairAlign - 1));
        const bool narrow = a.ja16 != nullptr;
        for (int k0 = kb + gl; k0 < kx; k0 += U * G) {
          unsigned sv[U];
          V gv[U];
          SV vv[U];
          X xv[U][RK];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int k = k0 + u * G;
            sv[u] = min(narrow ? (unsigned)s16[k] : (unsigned)sja[k], smax) * RK;
            gv[u] = sal[k];
            if constexpr (MODE == MODE_DF) {
              vv[u] = sym ? df_split<false>(gv[u], nullptr) : ssc[k];
            } else {
              vv[u] = sym ? gv[u] : ssc[k];
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < RK; ++c) xv[u][c] = win.xs[sv[u] + c];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (k0 + u * G < kx) {
#pragma unroll
              for (int c = 0; c < RK; ++c) {
                if constexpr (MODE == MODE_DF) {
                  acc[c] = fma(gv[u], xv[u][c], acc[c]);
                  df_atomic_add(win.whi + sv[u] + c, win.wlo + sv[u] + c, df_mul(vv[u], xr[c]));
                } else if constexpr (MODE == MODE_F64) {
                  acc[c] = fma(gv[u], xv[u][c], acc[c]);
                  atomicAdd(win.w + sv[u] + c, vv[u] * xr[c]);
                } else {
                  acc[c] = __fmaf_rn(as_f32<MODE>(gv[u]), xv[u][c], acc[c]);
                  atomicAdd(win.w + sv[u] + c, __fmul_rn(as_f32<MODE>(vv[u]), xr[c]));
                }
              }
            }
          }
        }
      } else if constexpr (!ATOMIC) {
        // Window strategy: the plan puts every target of the band in its window, so the
        // slot lookup needs no branch (a page missing from the table would be a plan error:
        // it is flagged, and its value goes to an in-range slot). U pairs per lane are
        // loaded before any of them is scattered, so their shared-memory latencies overlap.
        constexpr int U = RK >= 4 ? 1 : (RK == 1 && G == 16 ? 3 : 4 / RK);
        for (int k0 = kb + gl; k0 < kx; k0 += U * G) {
          int jv[U], sv[U];
          V gv[U], vv[U];
          X xv[U][RK];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            // past the row's end, re-read its first pair (an in-bounds address; the value is unused)
            const int k = k0 + u * G < kx ? k0 + u * G : kb;
            jv[u] = sja[k];
            gv[u] = sal[k];
            vv[u] = sau[k];
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int t = (jv[u] >> kPageShift) - plo;
            const int pb = (unsigned)t < (unsigned)ntab ? tab[t] : -1;
            bad |= pb < 0 ? 4u : 0u;
            sv[u] = max(pb, 0) + (jv[u] & (kPageRows - 1));
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < RK; ++c) xv[u][c] = win.xs[sv[u] * RK + c];
          if constexpr (MODE == MODE_DF) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              if (k0 + u * G < kx) {
                const df32 vs = df_split<false>(vv[u], nullptr);
#pragma unroll
                for (int c = 0; c < RK; ++c) {
                  acc[c] = fma(gv[u], xv[u][c], acc[c]);
                  df_atomic_add(win.whi + sv[u] * RK + c, win.wlo + sv[u] * RK + c, df_mul(vs, xr[c]));
                }
              }
            }
          } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              if (k0 + u * G < kx) {
                if constexpr (MODE == MODE_F64) {
#pragma unroll
                  for (int c = 0; c < RK; ++c) {
                    acc[c] = fma(gv[u], xv[u][c], acc[c]);
                    atomicAdd(win.w + sv[u] * RK + c, vv[u] * xr[c]);
                  }
                } else {
                  const float g32 = as_f32<MODE>(gv[u]), v32 = as_f32<MODE>(vv[u]);
#pragma unroll
                  for (int c = 0; c < RK; ++c) {
                    acc[c] = __fmaf_rn(g32, xv[u][c], acc[c]);
                    atomicAdd(win.w + sv[u] * RK + c, __fmul_rn(v32, xr[c]));
                  }
                }
              }
            }
          }
        }
      } else {
        // Atomic strategy: targets outside the window (plans with overflow) go to y in L2.
        for (int k = kb + gl; k < kx; k += G) {
          const int j = sja[k];
          const int js = slot_of(j);
          if constexpr (MODE == MODE_DF) {
            const double xj = js >= 0 ? win.xs[js] : __ldg(static_cast<const double*>(a.x) + (size_t)j * ldx);
            acc[0] = fma(sal[k], xj, acc[0]);
            const df32 p = df_mul(df_split<false>(sau[k], nullptr), xr[0]);
            if (js >= 0) {
              df_atomic_add(win.whi + js, win.wlo + js, p);
            } else {
              atomicAdd(static_cast<double*>(a.y) + (size_t)j * ldx, (double)p.hi + (double)p.lo);
            }
          } else if constexpr (MODE == MODE_F64) {
            const double xj = js >= 0 ? win.xs[js] : __ldg(static_cast<const double*>(a.x) + (size_t)j * ldx);
            acc[0] = fma(sal[k], xj, acc[0]);
            const double p = sau[k] * xr[0];
            if (js >= 0) {
              atomicAdd(win.w + js, p);
            } else {
              atomicAdd(static_cast<double*>(a.y) + (size_t)j * ldx, p);
            }
          } else {
            const float xj = js >= 0 ? win.xs[js] : __ldg(static_cast<const float*>(a.x) + (size_t)j * ldx);
            acc[0] = __fmaf_rn(as_f32<MODE>(sal[k]), xj, acc[0]);
            const float p = __fmul_rn(as_f32<MODE>(sau[k]), xr[0]);
            if (js >= 0) {
              atomicAdd(win.w + js, p);
            } else {
              atomicAdd(static_cast<float*>(a.y) + (size_t)j * ldx, p);
            }
          }
        }
      }
      // the group's gathered sums of row r: reduced across its G lanes, added once. The
      // double-float tree keeps each level's high-word error exactly and sums the low words
      // without renormalising (at most four levels: the low word stays within 2^-20 of the
      // sum); the atomic flush renormalises the high word.
#pragma unroll
      for (int c = 0; c < RK; ++c) {
        if constexpr (MODE == MODE_DF) {
          df32 t = df_split<false>(acc[c], nullptr);
#pragma unroll
          for (int o = G / 2; o > 0; o >>= 1) {
            df32 u;
            u.hi = __shfl_xor_sync(gmask, t.hi, o, G);
            u.lo = __shfl_xor_sync(gmask, t.lo, o, G);
            df_acc_short(t, u);
          }
          if (gl == 0) df_atomic_add(win.whi + rslot * RK + c, win.wlo + rslot * RK + c, t);
        } else {
          X v = acc[c];
#pragma unroll
          for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, G);
          if (gl == 0) atomicAdd(win.w + rslot * RK + c, v);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_empty + 8u * slot);
    if (tid == 0 && issued < nstages) {
      // every warp is done with stage s: refill its ring slot with stage s + NS
      if (!mbar_wait(bar_empty + 8u * slot, parity)) {
        timed_out = true;
        break;
      }
      fence_proxy_async_smem();
      issue(issued, s_sk[st0 + issued], s_sk[st0 + issued + 1]);
      ++issued;
    }
  }

  // ---- a wait ran out (should not happen): let this CTA's copies land, then stop
  __shared__ int abort_flag;
  __syncthreads();
  if (tid == 0) abort_flag = 0;
  __syncthreads();
  if (timed_out) abort_flag = 1;
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) {
      mbar_wait(bar_setup, 0u);
      for (int s = 0; s < issued; ++s) mbar_wait(bar_full + 8u * (s % NS), (uint32_t)((s / NS) & 1));
      atomicOr(a.status, DEV_TIMEOUT);
    }
    return false;
  }
  // every copy has landed and every wait has completed: the barriers can be retired
  if (tid == 0) {
    for (int i = 0; i < 2 * NS + 1; ++i) mbar_inval(smem_addr(bars + i));
  }

  // ---- phase 3: own rows (the diagonal term is added here, so rows without pairs are covered)
  for (int e = tid; e < (r1 - r0) * RK; e += T) {
    const int r = r0 + e / RK, c = e % RK;
    const int s = slot_of(r);
    if (s < 0) {
      bad |= 4u;
      continue;
    }
    const size_t yi = (size_t)r * ldx + c;
    if constexpr (MODE == MODE_DF || MODE == MODE_F64) {
      const double out = fma(__ldg(static_cast<const double*>(a.ad) + r), win.xs[s * RK + c], win.value(s * RK + c));
      if (ATOMIC) atomicAdd(static_cast<double*>(a.y) + yi, out);
      else static_cast<double*>(a.y)[yi] = out;
    } else {
      const float out = __fmaf_rn(as_f32<MODE>(__ldg(static_cast<const V*>(a.ad) + r)), win.xs[s * RK + c],
                                  win.value(s * RK + c));
      if (ATOMIC) atomicAdd(static_cast<float*>(a.y) + yi, out);
      else static_cast<float*>(a.y)[yi] = out;
    }
  }

  // ---- phase 4: rows below r0 (one warp per window page)
  for (int q = warp; q < np; q += T / 32) {
    const uint64_t mask = __ldg(reinterpret_cast<const unsigned long long*>(a.wmask) + wp0 + q);
    if (mask == 0ull) continue;
    const int base = __ldg(a.wbase + wp0 + q);
    const int page = __ldg(a.wpage + wp0 + q);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int e = half * 32 + lane;
      if (!((mask >> e) & 1ull)) continue;
      const int s = (q << kPageShift) | e;
      const int row = (page << kPageShift) | e;
      const int pos = base + __popcll(mask & ((1ull << e) - 1ull));
#pragma unroll
      for (int c = 0; c < RK; ++c) {
        const X v = win.value(s * RK + c);
        if (ATOMIC) atomicAdd(static_cast<X*>(a.y) + (size_t)row * ldx + c, v);
        else static_cast<X*>(a.spill)[(size_t)pos * RK + c] = v;
      }
    }
  }
  if (bad) atomicOr(a.status, (int)((bad & 1u) ? DEV_RANGE : 0) | (int)((bad & 4u) ? DEV_BOUNDS : 0));
  __syncthreads();  // the next band of this CTA reuses the shared memory
  return true;
}

template <int MODE, int G, bool ATOMIC, int RK, int B = 1>
__global__ void __launch_bounds__(band_threads(G, B, RK), BandShape<MODE>::kCtasPerSm) band_kernel(BandArgs a) {
  band_body<MODE, G, ATOMIC, RK, B>(a, blockIdx.x + a.band_offset);
}

// Dynamic shared memory limit of one instantiation.
template <int MODE, int G, bool ATOMIC, int RK, int B = 1>
cudaError_t set_band_smem() {
  return cudaFuncSetAttribute(band_kernel<MODE, G, ATOMIC, RK, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              band_smem_limit(MODE));
}

}  // namespace csrc
