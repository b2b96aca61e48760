// Colouring of the write-conflict graph and the colour-ordered product (Section 3.2).
//
// Rows u and v conflict when their write sets intersect, where
// W(i) = {i} U {ja[k] : k in row i} is the set of y entries that row i updates in
// Fig. 2(a). The graph is never materialised. The neighbours of u are found by
// walking t in W(u) and, for each t, the row t itself and the rows of A_U's
// column t: the rows v > t with t in their ja, listed in (up_ptr, up).
//
// uncolored[0] counts the rows left uncoloured by a round; uncolored[1] is set when a
// row would need more than 65536 colours.
//
// Jones-Plassmann: in every round, each uncoloured row that outranks all its
// uncoloured neighbours (priority SplitMix64(seed ^ row)) takes the smallest
// colour unused by its coloured neighbours. Adjacent rows are never both local
// maxima, so a row's choice depends only on its higher-priority neighbours,
// all coloured in earlier rounds. The result therefore equals sequential greedy
// colouring in decreasing priority order. A row's state packs
// (round << 16) | colour, so rows coloured during the current round still
// count as uncoloured.
#include <cstdint>

#include "internal.h"

namespace csrc {

// SplitMix64 (Steele, Lea, Flood 2014): mix(z + 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

template <typename F>
__device__ __forceinline__ bool for_each_neighbour(int u, const int32_t* __restrict__ ia,
                                                   const int32_t* __restrict__ ja,
                                                   const int32_t* __restrict__ up_ptr,
                                                   const int32_t* __restrict__ up, F&& f) {
  const int k0 = ia[u], k1 = ia[u + 1];
  for (int q = k0 - 1; q < k1; ++q) {
    const int t = q < k0 ? u : ja[q];
    if (t != u && !f(t)) return false;
    const int p1 = up_ptr[t + 1];
    for (int p = up_ptr[t]; p < p1; ++p) {
      const int v = up[p];
      if (v != u && !f(v)) return false;
    }
  }
  return true;
}

__global__ void jp_round_kernel(int32_t n, const int32_t* __restrict__ ia, const int32_t* __restrict__ ja,
                                const int32_t* __restrict__ up_ptr, const int32_t* __restrict__ up, uint64_t seed,
                                int32_t round, int32_t* state, int32_t* uncolored) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  if (state[u] >= 0) return;
  const uint64_t pu = splitmix64(seed ^ (uint64_t)u);
  // local maximum among the rows still uncoloured at the start of this round
  const bool is_max = for_each_neighbour(u, ia, ja, up_ptr, up, [&](int v) {
    const int st = state[v];
    if (st < 0 || (st >> 16) == round) return !(splitmix64(seed ^ (uint64_t)v) > pu);
    return true;
  });
  if (!is_max) {
    atomicAdd(uncolored, 1);
    return;
  }
  // smallest colour not used by neighbours coloured in earlier rounds, 64 colours at a time
  for (int base = 0; base < 65536; base += 64) {
    unsigned long long used = 0ull;
    for_each_neighbour(u, ia, ja, up_ptr, up, [&](int v) {
      const int st = state[v];
      if (st >= 0 && (st >> 16) < round) {
        const unsigned c = (unsigned)(st & 0xffff) - (unsigned)base;
        if (c < 64u) used |= 1ull << c;
      }
      return true;
    });
    if (~used != 0ull) {
      const int c = base + __ffsll((long long)~used) - 1;
      state[u] = (round << 16) | c;
      return;
    }
  }
  atomicAdd(uncolored, 1);
  atomicOr(uncolored + 1, 1);  // more than 65536 colours: the host reports a failure
}

cudaError_t launch_jp_round(int32_t n, const int32_t* ia, const int32_t* ja, const int32_t* up_ptr, const int32_t* up,
                            uint64_t seed, int32_t round, int32_t* state, int32_t* uncolored, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int bs = 256;
  jp_round_kernel<<<(n + bs - 1) / bs, bs, 0, s>>>(n, ia, ja, up_ptr, up, seed, round, state, uncolored);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- colour-ordered product
// All colour classes in one persistent, cooperative launch (every CTA resident): class c's
// rows are spread over groups of G lanes grid-wide, then a grid barrier, then class c + 1.
// y was zeroed. Rows of one class write disjoint entries of y, so plain read-modify-write
// updates are race-free; they go through L2 (ld.global.cg / st.global.cg) so that the next
// class, run by other CTAs after the barrier, sees them. A group streams its row's ja / al /
// au slices with G lanes side by side (coalesced) and sums the row's gather with shuffles.
// FP64 storage computes in FP64, FP32 / BF16 storage in FP32.
template <typename V, typename X>
__device__ __forceinline__ X to_x(V v);
template <>
__device__ __forceinline__ double to_x<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_x<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_x<uint16_t, float>(uint16_t v) { return __uint_as_float((unsigned)v << 16); }

// Grid barrier of a cooperative launch: every CTA adds one to *bar and waits, with a bound of
// about two seconds of SM clock, until it reaches target. Returns false when the wait ran out.
__device__ __forceinline__ bool color_grid_sync(unsigned* bar, unsigned target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const long long t0 = clock64();
    bool good = true;
    while (atomicAdd(bar, 0u) < target) {
      if (clock64() - t0 > 4000000000LL) {
        good = false;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    ok = good ? 1 : 0;
  }
  __syncthreads();
  return ok != 0;
}

// Threads per CTA of the colour product.
constexpr int kColorThreads = 256;

struct ColorArgs {
  int32_t ncolors;
  const int32_t* color_ptr;  // ncolors + 1: rows of class c are rows[color_ptr[c] .. color_ptr[c+1])
  const int32_t* rows;
  const int32_t* ia;
  const int32_t* ja;
  const void* al;  // gathered values (au for the transpose)
  const void* au;  // scattered values
  const void* ad;
  const void* x;
  void* y;
  unsigned* barrier;  // zero at launch
  int32_t* status;
};

template <typename V, typename X, int G>
__global__ void __launch_bounds__(kColorThreads) color_persistent_kernel(ColorArgs a) {
  const V* __restrict__ al = static_cast<const V*>(a.al);
  const V* __restrict__ au = static_cast<const V*>(a.au);
  const V* __restrict__ ad = static_cast<const V*>(a.ad);
  const X* __restrict__ x = static_cast<const X*>(a.x);
  X* y = static_cast<X*>(a.y);
  const int gpb = blockDim.x / G;
  const int ngroups = gridDim.x * gpb;
  const int gid = blockIdx.x * gpb + threadIdx.x / G;
  const int gl = threadIdx.x % G;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  for (int c = 0; c < a.ncolors; ++c) {
    const int p1 = __ldg(a.color_ptr + c + 1);
    for (int idx = __ldg(a.color_ptr + c) + gid; idx < p1; idx += ngroups) {
      const int i = __ldg(a.rows + idx);
      const X xi = __ldg(x + i);
      X s = X(0);
      const int k1 = __ldg(a.ia + i + 1);
      // four pairs per lane at a time: their loads (slices, x and y through L2) overlap
      constexpr int U = 4;
      for (int k0 = __ldg(a.ia + i) + gl; k0 < k1; k0 += U * G) {
        int j[U];
        V g[U], v[U];
        X xj[U], yj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u * G;
          j[u] = k < k1 ? __ldg(a.ja + k) : -1;
          g[u] = k < k1 ? __ldg(al + k) : V(0);
          v[u] = k < k1 ? __ldg(au + k) : V(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          xj[u] = j[u] >= 0 ? __ldg(x + j[u]) : X(0);
          yj[u] = j[u] >= 0 ? __ldcg(y + j[u]) : X(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (j[u] >= 0) {
            s = fma(to_x<V, X>(g[u]), xj[u], s);
            __stcg(y + j[u], fma(to_x<V, X>(v[u]), xi, yj[u]));
          }
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
      if (gl == 0) {
        X* yp = y + i;
        __stcg(yp, __ldcg(yp) + fma(to_x<V, X>(__ldg(ad + i)), xi, s));
      }
    }
    if (c + 1 < a.ncolors && !color_grid_sync(a.barrier, (unsigned)(c + 1) * gridDim.x)) {
      if (threadIdx.x == 0) atomicOr(a.status, DEV_TIMEOUT);
      return;
    }
  }
}

// Lanes per row: about a quarter of the mean row length, a power of two in [1, 32] (measured
// against an eighth and a sixteenth on the Q1 matrices: 4 lanes for q1s_96, 16 for q1v_96).
int color_group(double mean_pairs) {
  int g = 1;
  while (g < 32 && 4.0 * g < mean_pairs) g *= 2;
  return g;
}

template <typename V, typename X>
static cudaError_t launch_color_typed(int group, const ColorArgs& a, cudaStream_t s) {
  void* fn = nullptr;
  switch (group) {
    case 1: fn = (void*)color_persistent_kernel<V, X, 1>; break;
    case 2: fn = (void*)color_persistent_kernel<V, X, 2>; break;
    case 4: fn = (void*)color_persistent_kernel<V, X, 4>; break;
    case 8: fn = (void*)color_persistent_kernel<V, X, 8>; break;
    case 16: fn = (void*)color_persistent_kernel<V, X, 16>; break;
    default: fn = (void*)color_persistent_kernel<V, X, 32>; break;
  }
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kColorThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm <= 0) return cudaErrorLaunchOutOfResources;
  const int grid = sms * per_sm;  // every CTA resident at once: the grid barrier needs it
  ColorArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kColorThreads), params, 0, s);
}

cudaError_t launch_color_spmv(int storage, int group, int32_t ncolors, const int32_t* color_ptr, const int32_t* rows,
                              const int32_t* ia, const int32_t* ja, const void* al, const void* au, const void* ad,
                              const void* x, void* y, unsigned* barrier, int32_t* status, cudaStream_t s) {
  if (ncolors <= 0) return cudaSuccess;
  ColorArgs a{ncolors, color_ptr, rows, ia, ja, al, au, ad, x, y, barrier, status};
  if (storage == CSRC_F64) return launch_color_typed<double, double>(group, a, s);
  if (storage == CSRC_F32) return launch_color_typed<float, float>(group, a, s);
  return launch_color_typed<uint16_t, float>(group, a, s);
}

}  // namespace csrc
