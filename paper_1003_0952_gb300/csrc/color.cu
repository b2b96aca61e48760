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
// One colour class per launch, one thread per row. y was zeroed. Rows of one colour
// write disjoint entries of y, so plain read-modify-write updates are race-free.
// FP64 storage uses FP64-pipe arithmetic here, FP32/BF16 storage uses FP32.
template <typename V, typename X>
__device__ __forceinline__ X to_x(V v);
template <>
__device__ __forceinline__ double to_x<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_x<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_x<uint16_t, float>(uint16_t v) { return __uint_as_float((unsigned)v << 16); }

template <typename V, typename X>
__global__ void color_rows_kernel(int32_t nrows, const int32_t* __restrict__ rows, const int32_t* __restrict__ ia,
                                  const int32_t* __restrict__ ja, const V* __restrict__ al, const V* __restrict__ au,
                                  const V* __restrict__ ad, const X* __restrict__ x, X* y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows) return;
  const int i = rows[t];
  const X xi = x[i];
  X s = to_x<V, X>(ad[i]) * xi;
  const int k1 = ia[i + 1];
  for (int k = ia[i]; k < k1; ++k) {
    const int j = ja[k];
    s = fma(to_x<V, X>(al[k]), x[j], s);
    y[j] = fma(to_x<V, X>(au[k]), xi, y[j]);
  }
  y[i] += s;
}

cudaError_t launch_color_spmv(Arith arith, int storage, int32_t nrows, const int32_t* rows, const int32_t* ia,
                              const int32_t* ja, const void* al, const void* au, const void* ad, const void* x, void* y,
                              cudaStream_t s) {
  (void)arith;
  if (nrows <= 0) return cudaSuccess;
  const int bs = 128;
  const int grid = (nrows + bs - 1) / bs;
  if (storage == CSRC_F64) {
    color_rows_kernel<double, double><<<grid, bs, 0, s>>>(
        nrows, rows, ia, ja, static_cast<const double*>(al), static_cast<const double*>(au),
        static_cast<const double*>(ad), static_cast<const double*>(x), static_cast<double*>(y));
  } else if (storage == CSRC_F32) {
    color_rows_kernel<float, float><<<grid, bs, 0, s>>>(
        nrows, rows, ia, ja, static_cast<const float*>(al), static_cast<const float*>(au),
        static_cast<const float*>(ad), static_cast<const float*>(x), static_cast<float*>(y));
  } else {
    color_rows_kernel<uint16_t, float><<<grid, bs, 0, s>>>(
        nrows, rows, ia, ja, static_cast<const uint16_t*>(al), static_cast<const uint16_t*>(au),
        static_cast<const uint16_t*>(ad), static_cast<const float*>(x), static_cast<float*>(y));
  }
  return cudaGetLastError();
}

}  // namespace csrc
