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

__device__ __forceinline__ unsigned color_ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch, in two halves so that read-only loads can be issued
// between them: color_arrive after the CTA's last store of a class, color_wait before its
// first access to y in the next. Every CTA adds one to *bar (a release at GPU scope: the
// CTA's stores of y, ordered before it by __syncthreads, are visible to the CTAs that see the
// count) and waits until the count reaches target, polling with plain loads (no
// read-modify-write traffic on the counter's word) and an acquire fence once it has. The wait
// gives up after about two seconds of SM clock and returns false.
__device__ __forceinline__ void color_arrive(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" : : "l"(bar) : "memory");
}

__device__ __forceinline__ bool color_wait(unsigned* bar, unsigned target) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    bool good = true;
    while (color_ld_relaxed(bar) < target) {
      if (clock64() - t0 > 4000000000LL) {
        good = false;
        break;
      }
    }
    asm volatile("fence.acq_rel.gpu;" : : : "memory");
    ok = good ? 1 : 0;
  }
  __syncthreads();
  return ok != 0;
}

// Threads per CTA of the colour product.
constexpr int kColorThreads = 256;

struct ColorArgs {
  int32_t ncolors;
  const int32_t* color_ptr;  // ncolors + 1: rows of class c are desc[color_ptr[c] .. color_ptr[c+1])
  const int4* desc;          // per row of a class: {row, k0, k1, -}: its pairs are k0 .. k1 - 1
  const int32_t* ja;         // ja, al, au in class order (the colouring's copy)
  const void* al;  // gathered values (au for the transpose)
  const void* au;  // scattered values
  const void* ad;
  const void* x;
  void* y;
  unsigned* barrier;  // zero at launch
  int32_t* status;
};

// Pairs per lane per chunk of a row: their loads (slices, then x and y through L2) overlap.
constexpr int kColorU = 2;

// The first chunk of a row: each lane's kColorU pairs (slot -1 where the row has none). These
// are read-only loads, so a group issues them for its first row of the next class before the
// grid barrier, and they land while it waits.
template <typename V>
struct ColorChunk {
  int j[kColorU];
  V g[kColorU], v[kColorU];
};

template <typename V>
__device__ __forceinline__ void color_load_chunk(const ColorArgs& a, int k0, int k1, ColorChunk<V>& ch) {
  const V* __restrict__ al = static_cast<const V*>(a.al);
  const V* __restrict__ au = static_cast<const V*>(a.au);
#pragma unroll
  for (int u = 0; u < kColorU; ++u) {
    const int k = k0 + u;
    ch.j[u] = k < k1 ? __ldg(a.ja + k) : -1;
    ch.g[u] = k < k1 ? __ldg(al + k) : V(0);
    ch.v[u] = k < k1 ? __ldg(au + k) : V(0);
  }
}

// y[j] += v x_i for the chunk's pairs, and their gather into s.
template <typename V, typename X>
__device__ __forceinline__ void color_apply_chunk(const ColorChunk<V>& ch, const X* __restrict__ x, X* y, X xi,
                                                  X& s) {
  X xj[kColorU], yj[kColorU];
#pragma unroll
  for (int u = 0; u < kColorU; ++u) {
    xj[u] = ch.j[u] >= 0 ? __ldg(x + ch.j[u]) : X(0);
    yj[u] = ch.j[u] >= 0 ? __ldcg(y + ch.j[u]) : X(0);
  }
#pragma unroll
  for (int u = 0; u < kColorU; ++u) {
    if (ch.j[u] >= 0) {
      s = fma(to_x<V, X>(ch.g[u]), xj[u], s);
      __stcg(y + ch.j[u], fma(to_x<V, X>(ch.v[u]), xi, yj[u]));
    }
  }
}

// Row d = {i, ia[i], ia[i+1]} of the current class, run by a group of G lanes: lane gl takes
// the kColorU consecutive pairs at d.y + kColorU * (gl + G * t) for t = 0, 1, ..., with the
// chunk t = 0 already loaded in first.
template <typename V, typename X, int G>
__device__ __forceinline__ void color_row(const ColorArgs& a, int4 d, const ColorChunk<V>& first, int gl,
                                          unsigned gmask) {
  const V* __restrict__ ad = static_cast<const V*>(a.ad);
  const X* __restrict__ x = static_cast<const X*>(a.x);
  X* y = static_cast<X*>(a.y);
  const int i = d.x;
  const X xi = __ldg(x + i);
  // y[i] and ad[i] are read before the row's pairs: only this row writes y[i] in this class
  // (its scatter targets lie below i), so the read overlaps the pair loads
  X yi = X(0);
  V di = V(0);
  if (gl == 0) {
    yi = __ldcg(y + i);
    di = __ldg(ad + i);
  }
  X s = X(0);
  // chunk t + 1's slice loads are issued before chunk t's x and y accesses
  ColorChunk<V> cur = first;
  for (int k0 = d.y + kColorU * (gl + G); k0 < d.z; k0 += kColorU * G) {
    ColorChunk<V> nxt;
    color_load_chunk<V>(a, k0, d.z, nxt);
    color_apply_chunk<V, X>(cur, x, y, xi, s);
    cur = nxt;
  }
  color_apply_chunk<V, X>(cur, x, y, xi, s);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
  if (gl == 0) __stcg(y + i, yi + fma(to_x<V, X>(di), xi, s));
}

template <typename V, typename X, int G>
__global__ void __launch_bounds__(kColorThreads, 4) color_persistent_kernel(ColorArgs a) {
  const int gpb = blockDim.x / G;
  const int ngroups = gridDim.x * gpb;
  const int gid = blockIdx.x * gpb + threadIdx.x / G;
  const int gl = threadIdx.x % G;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  // the group's first row of class c and its first chunk, loaded ahead
  int4 nd = make_int4(-1, 0, 0, 0);
  ColorChunk<V> nch;
  // the group's second and third rows of the class: their descriptors too (q1v_96 with the JP
  // colouring: 1.33 -> 1.23 ms)
  int4 nd2 = make_int4(-1, 0, 0, 0), nd3 = make_int4(-1, 0, 0, 0);
  auto load_first = [&](int c) {
    const int idx = __ldg(a.color_ptr + c) + gid;
    const int pe = __ldg(a.color_ptr + c + 1);
    nd = idx < pe ? __ldg(a.desc + idx) : make_int4(-1, 0, 0, 0);
    nd2 = idx + ngroups < pe ? __ldg(a.desc + idx + ngroups) : make_int4(-1, 0, 0, 0);
    nd3 = idx + 2 * ngroups < pe ? __ldg(a.desc + idx + 2 * ngroups) : make_int4(-1, 0, 0, 0);
    color_load_chunk<V>(a, nd.x >= 0 ? nd.y + kColorU * gl : 0, nd.x >= 0 ? nd.z : 0, nch);
  };
  load_first(0);
  for (int c = 0; c < a.ncolors; ++c) {
    const int p1 = __ldg(a.color_ptr + c + 1);
    if (nd.x >= 0) color_row<V, X, G>(a, nd, nch, gl, gmask);
    for (int idx = __ldg(a.color_ptr + c) + gid + ngroups; idx < p1; idx += ngroups) {
      const int i0 = __ldg(a.color_ptr + c) + gid;
      const int4 d = idx == i0 + ngroups ? nd2 : (idx == i0 + 2 * ngroups ? nd3 : __ldg(a.desc + idx));
      ColorChunk<V> ch;
      color_load_chunk<V>(a, d.y + kColorU * gl, d.z, ch);
      color_row<V, X, G>(a, d, ch, gl, gmask);
    }
    if (c + 1 < a.ncolors) {
      color_arrive(a.barrier);
      load_first(c + 1);  // read-only: it overlaps the wait
      if (!color_wait(a.barrier, (unsigned)(c + 1) * gridDim.x)) {
        if (threadIdx.x == 0) atomicOr(a.status, DEV_TIMEOUT);
        return;
      }
    }
  }
}

// Lanes per row: the power of two in [1, 32] nearest (in ratio) to a quarter of the mean row
// length, so that a row takes about two chunks of kColorU pairs per lane (timed against
// halving and doubling it: 4 lanes for q1s_96, 8 for q1v_96).
int color_group(double mean_pairs) {
  int g = 1;
  while (g < 32 && 1.41421356 * g < mean_pairs / 4.0) g *= 2;
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

// The class-ordered copy of the lists: row t of the class order (desc[t] = {i, k0, k1, ia[i]})
// gets its pairs ja / al / au[ia[i] ..] at k0 .. k1 - 1, one warp per row. The colour product
// then streams each class's slices contiguously instead of gathering rows spread over the
// whole matrix.
template <typename V>
__global__ void color_copy_kernel(const int4* __restrict__ desc, int32_t n, const int32_t* __restrict__ ja,
                                  const V* __restrict__ al, const V* __restrict__ au, int32_t* __restrict__ cja,
                                  V* __restrict__ cal, V* __restrict__ cau) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = w0; t < n; t += nw) {
    const int4 d = desc[t];
    for (int k = d.y + lane; k < d.z; k += 32) {
      const int src = d.w + (k - d.y);
      cja[k] = ja[src];
      cal[k] = al[src];
      if (cau) cau[k] = au[src];
    }
  }
}

cudaError_t launch_color_copy(int vbytes, const int4* desc, int32_t n, const int32_t* ja, const void* al,
                              const void* au, int32_t* cja, void* cal, void* cau, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, (int64_t)std::max(sms, 1) * 16);
#define CSRC_COPY(T)                                                                                         \
  color_copy_kernel<T><<<grid, 256, 0, s>>>(desc, n, ja, static_cast<const T*>(al), static_cast<const T*>(au), \
                                            cja, static_cast<T*>(cal), static_cast<T*>(cau))
  if (vbytes == 8) CSRC_COPY(double);
  else if (vbytes == 4) CSRC_COPY(float);
  else if (vbytes == 2) CSRC_COPY(uint16_t);
  else return cudaErrorInvalidValue;
#undef CSRC_COPY
  return cudaGetLastError();
}

cudaError_t launch_color_spmv(int storage, int group, int32_t ncolors, const int32_t* color_ptr, const int4* desc,
                              const int32_t* ja, const void* al, const void* au, const void* ad, const void* x,
                              void* y, unsigned* barrier, int32_t* status, cudaStream_t s) {
  if (ncolors <= 0) return cudaSuccess;
  ColorArgs a{ncolors, color_ptr, desc, ja, al, au, ad, x, y, barrier, status};
  if (storage == CSRC_F64) return launch_color_typed<double, double>(group, a, s);
  if (storage == CSRC_F32) return launch_color_typed<float, float>(group, a, s);
  return launch_color_typed<uint16_t, float>(group, a, s);
}

}  // namespace csrc
