// Band kernels of the CSRC product y = A x (Fig. 2(a)) for sm_103a.
//
// One CTA runs one row band [r0, r1) of the window plan. It streams the band's
// contiguous slice [ia[r0], ia[r1]) of ja / al / au with coalesced 16-byte
// loads, four pairs per thread per step. Every pair gathers al*x[j] into its
// row's register accumulator and scatters au*x[i] into y[j].
//
// The scatter goes to a private window in shared memory, the GPU form of the
// local buffers of Section 3.1. The window holds the rows this band writes: its
// own rows and every row ja reaches below r0 (the band's "effective range"),
// kept at 64-row page granularity and found through a page table. x for those
// rows is staged in the same window, so gathers read shared memory too. When
// the stream ends:
//  - window strategy: own rows are stored to y, and rows below r0 go to a
//    compact spill buffer. A separate accumulation kernel folds the spills into
//    y in fixed band order (deterministic), like the "effective" accumulation
//    of Section 3.1.
//  - atomic strategy: y was zeroed, and every window row is added to y with a
//    global atomic (red.global.add, executed in L2). Pages outside the window
//    (plans with overflow) scatter straight to y with the same atomics.
//
// Arithmetic by mode:
//  - MODE_DF: FP64 storage and vectors, double-float accumulation (df32.cuh).
//  - MODE_F64: FP64 storage, FP64-pipe arithmetic (bit-for-bit IEEE products).
//  - MODE_F32: FP32 storage, FP32 vectors and accumulation.
//  - MODE_BF16: BF16 storage, FP32 vectors and accumulation.
#include <cstdint>

#include "df32.cuh"
#include "internal.h"

namespace csrc {

enum { MODE_DF = 0, MODE_F64 = 1, MODE_F32 = 2, MODE_BF16 = 3 };

// ---------------------------------------------------------------------------- loads
__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }

// The 4 stored values starting at k (k % 4 == 0), kept in their storage format.
template <int MODE>
struct Raw4 {  // MODE_DF / MODE_F64: 32 bytes
  double2 a, b;
};
template <>
struct Raw4<MODE_F32> {
  float4 a;
};
template <>
struct Raw4<MODE_BF16> {
  uint2 a;
};

template <int MODE>
__device__ __forceinline__ Raw4<MODE> raw_load(const void* base, int k) {
  Raw4<MODE> r;
  if constexpr (MODE == MODE_DF || MODE == MODE_F64) {
    const double2* p = reinterpret_cast<const double2*>(static_cast<const double*>(base) + k);
    r.a = __ldcs(p);
    r.b = __ldcs(p + 1);
  } else if constexpr (MODE == MODE_F32) {
    r.a = __ldcs(reinterpret_cast<const float4*>(static_cast<const float*>(base) + k));
  } else {
    r.a = __ldcs(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(base) + k));
  }
  return r;
}

template <int MODE>
__device__ __forceinline__ double raw_d(const Raw4<MODE>& r, int q) {
  return q == 0 ? r.a.x : q == 1 ? r.a.y : q == 2 ? r.b.x : r.b.y;
}

template <int MODE>
__device__ __forceinline__ float raw_f(const Raw4<MODE>& r, int q) {
  if constexpr (MODE == MODE_F32) {
    return q == 0 ? r.a.x : q == 1 ? r.a.y : q == 2 ? r.a.z : r.a.w;
  } else {
    const unsigned w = q < 2 ? r.a.x : r.a.y;
    return __uint_as_float((q & 1) ? (w & 0xffff0000u) : (w << 16));
  }
}

// One stored diagonal value as the mode's element.
template <int MODE>
__device__ __forceinline__ float load_one_f(const void* base, int i) {
  if constexpr (MODE == MODE_F32) {
    return __ldg(static_cast<const float*>(base) + i);
  } else {
    const unsigned short v = __ldg(static_cast<const unsigned short*>(base) + i);
    return __uint_as_float((unsigned)v << 16);
  }
}

// ---------------------------------------------------------------------------- window views
// Shared memory of a band: [x window][accumulator window][page table (int16)].
template <int MODE>
struct Window;

template <>
struct Window<MODE_DF> {
  df32* xs;
  float* whi;
  float* wlo;
  static constexpr int kBytesPerSlot = 16;
  __device__ void bind(unsigned char* s, int nslots) {
    xs = reinterpret_cast<df32*>(s);
    whi = reinterpret_cast<float*>(xs + nslots);
    wlo = whi + nslots;
  }
};
template <>
struct Window<MODE_F64> {
  double* xs;
  double* w;
  static constexpr int kBytesPerSlot = 16;
  __device__ void bind(unsigned char* s, int nslots) {
    xs = reinterpret_cast<double*>(s);
    w = xs + nslots;
  }
};
template <int MODE>
struct Window {  // MODE_F32 and MODE_BF16
  float* xs;
  float* w;
  static constexpr int kBytesPerSlot = 8;
  __device__ void bind(unsigned char* s, int nslots) {
    xs = reinterpret_cast<float*>(s);
    w = xs + nslots;
  }
};

// Accumulator type and operations per mode.
template <int MODE>
struct Acc;

template <>
struct Acc<MODE_DF> {
  using X = df32;  // x element as held in registers/shared memory
  df32 v;
  __device__ void zero() { v.hi = 0.f; v.lo = 0.f; }
};
template <>
struct Acc<MODE_F64> {
  using X = double;
  double v;
  __device__ void zero() { v = 0.0; }
};
template <int MODE>
struct Acc {
  using X = float;
  float v;
  __device__ void zero() { v = 0.f; }
};

// ---------------------------------------------------------------------------- the band kernel
template <int MODE, bool ATOMIC>
__global__ void __launch_bounds__(kBandThreads, 2) band_kernel(BandArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x + a.band_offset;
  const int r0 = a.band_row[b];
  const int r1 = a.band_row[b + 1];
  const int plo = a.band_plo[b];
  const int ntab = a.band_ntab[b];
  const int wp0 = a.band_wp[b];
  const int np = a.band_wp[b + 1] - wp0;
  const int nslots = np << kPageShift;
  const int tid = threadIdx.x;
  Window<MODE> win;
  win.bind(smem, nslots);
  short* tab = reinterpret_cast<short*>(smem + (size_t)nslots * Window<MODE>::kBytesPerSlot);
  unsigned bad = 0u;

  // ---- phase 1: clear the page table, stage x into the window, clear the accumulators
  for (int t = tid; t < ntab; t += kBandThreads) tab[t] = (short)-1;
  for (int s = tid; s < nslots; s += kBandThreads) {
    const int page = __ldg(a.wpage + wp0 + (s >> kPageShift));
    const int j = (page << kPageShift) | (s & (kPageRows - 1));
    if constexpr (MODE == MODE_DF) {
      const double xv = j < a.n ? __ldg(static_cast<const double*>(a.x) + j) : 0.0;
      win.xs[s] = df_split<true>(xv, &bad);
      win.whi[s] = 0.f;
      win.wlo[s] = 0.f;
    } else if constexpr (MODE == MODE_F64) {
      win.xs[s] = j < a.n ? __ldg(static_cast<const double*>(a.x) + j) : 0.0;
      win.w[s] = 0.0;
    } else {
      win.xs[s] = j < a.n ? __ldg(static_cast<const float*>(a.x) + j) : 0.f;
      win.w[s] = 0.f;
    }
  }
  __syncthreads();
  for (int q = tid; q < np; q += kBandThreads) {
    const int t = __ldg(a.wpage + wp0 + q) - plo;
    if ((unsigned)t < (unsigned)ntab) {
      tab[t] = (short)q;
    } else {
      bad |= 4u;
    }
  }
  __syncthreads();

  // slot of row j in the window, or -1 (page outside the window)
  auto slot_of = [&](int j) -> int {
    const int t = (j >> kPageShift) - plo;
    if ((unsigned)t >= (unsigned)ntab) return -1;
    const int q = tab[t];
    return q < 0 ? -1 : ((q << kPageShift) | (j & (kPageRows - 1)));
  };

  // ---- phase 2: stream the band's pairs
  // Each thread takes 4 consecutive pairs per step (one 16-byte ja load, 16/8-byte value
  // loads), and the loads of the next step are issued before the current step is
  // processed. The row of a pair is searched between the rows that start the pair's
  // 128-pair block and the next one (blk_row, precomputed), a few rows at most.
  const int kbeg = __ldg(a.ia + r0);
  const int kend = __ldg(a.ia + r1);
  using XT = typename Acc<MODE>::X;
  constexpr int kStep = 4 * kBandThreads;
  int k0 = (kbeg & ~3) + 4 * tid;
  int4 cj = make_int4(0, 0, 0, 0);
  Raw4<MODE> cg{}, cv{};
  if (k0 < kend) {
    cj = ld_stream(reinterpret_cast<const int4*>(a.ja + k0));
    cg = raw_load<MODE>(a.al, k0);
    cv = raw_load<MODE>(a.au, k0);
  }
  for (; k0 < kend; k0 += kStep) {
    const int kn = k0 + kStep;
    int4 nj = make_int4(0, 0, 0, 0);
    Raw4<MODE> ng{}, nv{};
    if (kn < kend) {
      nj = ld_stream(reinterpret_cast<const int4*>(a.ja + kn));
      ng = raw_load<MODE>(a.al, kn);
      nv = raw_load<MODE>(a.au, kn);
    }
    const int jj[4] = {cj.x, cj.y, cj.z, cj.w};
    // row of the first pair of this thread that lies inside the band
    const int kf = k0 > kbeg ? k0 : kbeg;
    const int blk = k0 >> kBlockShift;
    int lo = max(__ldg(a.blk_row + blk), r0);
    int hi = min(__ldg(a.blk_row + blk + 1), r1 - 1);
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.ia + mid) <= kf) lo = mid; else hi = mid - 1;
    }
    int r = lo;
    int rend = __ldg(a.ia + r + 1);
    int rslot = slot_of(r);
    if (rslot < 0) { bad |= 4u; rslot = 0; }
    XT xr = win.xs[rslot];
    Acc<MODE> acc;
    acc.zero();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q;
      if (k < kbeg || k >= kend) continue;
      while (k >= rend) {  // row change: hand the finished row segment to the window
        if constexpr (MODE == MODE_DF) {
          df_atomic_add(win.whi + rslot, win.wlo + rslot, acc.v);
        } else {
          atomicAdd(win.w + rslot, acc.v);
        }
        acc.zero();
        ++r;
        rend = __ldg(a.ia + r + 1);
        rslot = slot_of(r);
        if (rslot < 0) { bad |= 4u; rslot = 0; }
        xr = win.xs[rslot];
      }
      const int j = jj[q];
      const int js = slot_of(j);
      if constexpr (MODE == MODE_DF) {
        df32 xj;
        if (js >= 0) {
          xj = win.xs[js];
        } else {
          xj = df_split<true>(__ldg(static_cast<const double*>(a.x) + j), &bad);
        }
        const df32 g = df_split<false>(raw_d(cg, q), nullptr);
        const df32 sv = df_split<false>(raw_d(cv, q), nullptr);
        df_acc_short(acc.v, df_mul(g, xj));
        const df32 p = df_mul(sv, xr);
        if (js >= 0) {
          df_atomic_add(win.whi + js, win.wlo + js, p);
        } else if (ATOMIC) {
          atomicAdd(static_cast<double*>(a.y) + j, df_to_f64(p));
        } else {
          bad |= 4u;
        }
      } else if constexpr (MODE == MODE_F64) {
        const double xj = js >= 0 ? win.xs[js] : __ldg(static_cast<const double*>(a.x) + j);
        acc.v = fma(raw_d(cg, q), xj, acc.v);
        const double p = raw_d(cv, q) * xr;
        if (js >= 0) {
          atomicAdd(win.w + js, p);
        } else if (ATOMIC) {
          atomicAdd(static_cast<double*>(a.y) + j, p);
        } else {
          bad |= 4u;
        }
      } else {
        const float xj = js >= 0 ? win.xs[js] : __ldg(static_cast<const float*>(a.x) + j);
        acc.v = __fmaf_rn(raw_f<MODE>(cg, q), xj, acc.v);
        const float p = __fmul_rn(raw_f<MODE>(cv, q), xr);
        if (js >= 0) {
          atomicAdd(win.w + js, p);
        } else if (ATOMIC) {
          atomicAdd(static_cast<float*>(a.y) + j, p);
        } else {
          bad |= 4u;
        }
      }
    }
    if constexpr (MODE == MODE_DF) {
      df_atomic_add(win.whi + rslot, win.wlo + rslot, acc.v);
    } else {
      atomicAdd(win.w + rslot, acc.v);
    }
    cj = nj;
    cg = ng;
    cv = nv;
  }
  __syncthreads();

  // ---- phase 3: own rows (diagonal term added here, so empty rows are covered)
  for (int r = r0 + tid; r < r1; r += kBandThreads) {
    int s = slot_of(r);
    if (s < 0) { bad |= 4u; continue; }
    if constexpr (MODE == MODE_DF) {
      df32 v;
      v.hi = win.whi[s];
      v.lo = win.wlo[s];
      const df32 dd = df_split<false>(__ldg(static_cast<const double*>(a.ad) + r), nullptr);
      df_acc(v, df_mul(dd, win.xs[s]));
      const double out = df_to_f64(v);
      if (ATOMIC) atomicAdd(static_cast<double*>(a.y) + r, out);
      else static_cast<double*>(a.y)[r] = out;
    } else if constexpr (MODE == MODE_F64) {
      const double out = fma(__ldg(static_cast<const double*>(a.ad) + r), win.xs[s], win.w[s]);
      if (ATOMIC) atomicAdd(static_cast<double*>(a.y) + r, out);
      else static_cast<double*>(a.y)[r] = out;
    } else {
      const float out = __fmaf_rn(load_one_f<MODE>(a.ad, r), win.xs[s], win.w[s]);
      if (ATOMIC) atomicAdd(static_cast<float*>(a.y) + r, out);
      else static_cast<float*>(a.y)[r] = out;
    }
  }

  // ---- phase 4: rows below r0 (one warp per window page)
  const int lane = tid & 31;
  const int warp = tid >> 5;
  for (int q = warp; q < np; q += kBandThreads / 32) {
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
      if constexpr (MODE == MODE_DF) {
        df32 v;
        v.hi = win.whi[s];
        v.lo = win.wlo[s];
        const double out = df_to_f64(v);
        if (ATOMIC) atomicAdd(static_cast<double*>(a.y) + row, out);
        else static_cast<double*>(a.spill)[pos] = out;
      } else if constexpr (MODE == MODE_F64) {
        if (ATOMIC) atomicAdd(static_cast<double*>(a.y) + row, win.w[s]);
        else static_cast<double*>(a.spill)[pos] = win.w[s];
      } else {
        if (ATOMIC) atomicAdd(static_cast<float*>(a.y) + row, win.w[s]);
        else static_cast<float*>(a.spill)[pos] = win.w[s];
      }
    }
  }
  if (bad) atomicOr(a.status, (int)((bad & 1u) ? DEV_RANGE : 0) | (int)((bad & 4u) ? DEV_BOUNDS : 0));
}

// ---------------------------------------------------------------------------- accumulation
// y[row] += sum of the row's spilled partial sums, in band order (deterministic).
template <typename T>
__global__ void accumulate_kernel(int64_t nacc, const int32_t* __restrict__ acc_row,
                                  const int32_t* __restrict__ acc_ptr, const int32_t* __restrict__ acc_src,
                                  const T* __restrict__ spill, T* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nacc) return;
  const int row = acc_row[i];
  T s = y[row];
  const int e1 = acc_ptr[i + 1];
  for (int e = acc_ptr[i]; e < e1; ++e) s += spill[acc_src[e]];
  y[row] = s;
}

// ---------------------------------------------------------------------------- launchers
static int mode_of(Arith arith, int storage) {
  if (storage == CSRC_F32) return MODE_F32;
  if (storage == CSRC_BF16) return MODE_BF16;
  return arith == ARITH_F64 ? MODE_F64 : MODE_DF;
}

template <int MODE, bool ATOMIC>
static cudaError_t set_smem(int bytes) {
  return cudaFuncSetAttribute(band_kernel<MODE, ATOMIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t prepare_band_kernels(int max_smem_bytes) {
  cudaError_t e = cudaSuccess;
  cudaError_t r;
#define CSRC_SET(M, A) r = set_smem<M, A>(max_smem_bytes); if (r != cudaSuccess) e = r;
  CSRC_SET(MODE_DF, false) CSRC_SET(MODE_DF, true) CSRC_SET(MODE_F64, false) CSRC_SET(MODE_F64, true)
  CSRC_SET(MODE_F32, false) CSRC_SET(MODE_F32, true) CSRC_SET(MODE_BF16, false) CSRC_SET(MODE_BF16, true)
#undef CSRC_SET
  return e;
}

cudaError_t launch_band(Arith arith, int storage, bool atomic_flush, const BandArgs& a, int nbands, int smem,
                        cudaStream_t s) {
  if (nbands <= 0) return cudaSuccess;
  const int mode = mode_of(arith, storage);
  dim3 grid(nbands), block(kBandThreads);
#define CSRC_LAUNCH(M)                                                        \
  if (atomic_flush) band_kernel<M, true><<<grid, block, smem, s>>>(a);        \
  else band_kernel<M, false><<<grid, block, smem, s>>>(a);
  switch (mode) {
    case MODE_DF: CSRC_LAUNCH(MODE_DF) break;
    case MODE_F64: CSRC_LAUNCH(MODE_F64) break;
    case MODE_F32: CSRC_LAUNCH(MODE_F32) break;
    default: CSRC_LAUNCH(MODE_BF16) break;
  }
#undef CSRC_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_accumulate(Arith arith, int storage, int64_t nacc, const int32_t* acc_row, const int32_t* acc_ptr,
                              const int32_t* acc_src, const void* spill, void* y, cudaStream_t s) {
  if (nacc <= 0) return cudaSuccess;
  const int bs = 256;
  const unsigned grid = (unsigned)((nacc + bs - 1) / bs);
  if (storage == CSRC_F64) {
    accumulate_kernel<double><<<grid, bs, 0, s>>>(nacc, acc_row, acc_ptr, acc_src,
                                                  static_cast<const double*>(spill), static_cast<double*>(y));
  } else {
    accumulate_kernel<float><<<grid, bs, 0, s>>>(nacc, acc_row, acc_ptr, acc_src, static_cast<const float*>(spill),
                                                 static_cast<float*>(y));
  }
  (void)arith;
  return cudaGetLastError();
}

}  // namespace csrc
