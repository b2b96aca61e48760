// Host side of the C ABI declared in include/csrc.h.
//
// Set-up (conversion, partition, window planning, colouring driver) runs here on
// the host or through setup kernels. Every product runs in the CUDA kernels of
// kernels.cu and color.cu. There is no CPU compute path: without a usable CUDA
// device every compute call returns CSRC_ERR_CUDA.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "internal.h"

using namespace csrc;

struct csrc_matrix_s {
  int32_t n = 0;
  int64_t h = 0;
  csrc_dtype storage = CSRC_F64;
  uint32_t flags = 0;
  Arith arith = ARITH_DF32;
  int device = 0;
  int sms = 0;
  std::vector<int32_t> ia, ja;  // host copy of the structure (planning, colouring)
  int32_t* d_ia = nullptr;
  int32_t* d_ja = nullptr;
  void* d_al = nullptr;
  void* d_au = nullptr;        // null for numerically symmetric storage (al serves both)
  void* d_ad = nullptr;
  bool sym = false;            // CSRC_FLAG_SYMMETRIC_VALUES: au is al (Section 2.2)
  void* au_ptr() const { return sym ? d_al : d_au; }
  // double-float arithmetic: al and au split into (hi, lo) FP32 pairs once, the scatter
  // operand of the window kernels (the split they would otherwise repeat per pair)
  void* d_al_df = nullptr;
  void* d_au_df = nullptr;
  int32_t* d_status = nullptr;
  // rectangular matrices (Section 2.1): m columns, the auxiliary CSR of columns n..m-1 for
  // the rows that have any (d_rrow, d_rptr, d_rcol, d_rval) and its column-major copy
  int32_t m = 0;
  int64_t rnnz = 0;
  int32_t nrrows = 0;
  int32_t* d_rrow = nullptr;
  int32_t* d_rptr = nullptr;
  int32_t* d_rcol = nullptr;
  void* d_rval = nullptr;
  // BiCG scratch (csrc_bicg): r, r*, p, p*, q, q* and the partial inner products
  void* d_solve = nullptr;
  double* d_partial = nullptr;
  int32_t* d_tptr = nullptr;
  int32_t* d_trow = nullptr;
  void* d_tval = nullptr;
  bool rect() const { return m != n; }
  // partition (Section 3.1 rule) and the plans built from it
  std::vector<int32_t> part;
  // owner lists of the window strategy: single vectors, and rk = 2, 4, 8 columns per pass
  OwnerPlan oplan;
  bool have_oplan = false;
  OwnerPlan oplan_rk[3];
  bool have_orp[3] = {false, false, false};
  bool fits_orp[3] = {false, false, false};
  // owner lists sized for batches (bands of about kOwnerBandNnz non-zeros), rk = 1, 2, 4, 8
  OwnerPlan oplan_bt[4];
  bool have_obt[4] = {false, false, false, false};
  bool fits_obt[4] = {false, false, false, false};
  int64_t obt_target[4] = {0, 0, 0, 0};  // non-zeros per band the batch plans were built for
  // stream-order plan of the window-atomic and atomic strategies
  DevPlan plan;
  bool have_plan = false;
  bool plan_covers = false;   // every scatter target lies in its band's window
  int32_t part_nbands = 0;    // band count requested for the partition (0 = automatic)
  int32_t owner_nbands = 0;   // band count of the owner plans (0 = automatic; set by the autotuner)
  // precision of the window strategy's values (csrc_set_precision): the storage type, or FP32 /
  // BF16 for a CSRC_F64 handle that runs its window products at reduced precision on double vectors
  int32_t precision = CSRC_F64;
  int32_t owner_mode() const {
    if (storage != CSRC_F64) return storage;
    return precision == CSRC_F32 ? OM_F32_X64 : (precision == CSRC_BF16 ? OM_BF16_X64 : OM_F64);
  }
  int64_t max_row_nnz = 0;    // longest row of A (diagonal, lower and upper entries)
  uint64_t phash = 0;         // pattern hash (tuning cache key)
  char devname[64] = {0};     // device name and SM count (tuning cache key)
  int32_t block = 1;          // rows per node block found at creation (1 = none)
  DevPlan plan_b1;            // plain-row plan when the main plan uses node blocks
  bool have_b1 = false;
  bool covers_b1 = false;
  // colouring
  int32_t ncolors = 0;
  int4* d_color_desc = nullptr;    // class-ordered rows {row, k0, k1, ia[row]}: pairs k0 .. k1 - 1 of the copy
  int32_t* d_cja = nullptr;        // ja, al, au in class order (au not copied for symmetric values)
  void* d_cal = nullptr;
  void* d_cau = nullptr;
  int32_t* d_color_ptr = nullptr;  // device copy of color_ptr
  unsigned* d_barrier = nullptr;   // grid barrier counter of the colour product
  std::vector<int32_t> color_ptr;
  // staging for host vectors
  void* d_xs = nullptr;
  void* d_ys = nullptr;
  int32_t tuned = 0;
  int32_t tuned_rk = 0;       // columns per pass for several right-hand sides (0 = up to 8)
  uint64_t generation = 0;    // bumped whenever plans or the tuned strategy change
  // kernel timing (csrc_set_profiling): CUDA events around every launch of this handle
  bool profiling = false;
  struct TimedLaunch {
    int32_t kind;
    int32_t kernels;  // kernel launches the record covers (a graph replay covers several)
    cudaEvent_t start, stop;
  };
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  size_t vbytes() const { return storage == CSRC_F64 ? 8 : (storage == CSRC_F32 ? 4 : 2); }
  size_t xbytes() const { return storage == CSRC_F64 ? 8 : 4; }
};

namespace {

std::mutex g_setup_mutex;  // serialises one-time kernel attribute set-up
bool g_prepared = false;

csrc_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CSRC_OK;
  if (e == cudaErrorMemoryAllocation) return CSRC_ERR_OUT_OF_MEMORY;
  return CSRC_ERR_CUDA;
}

#define CSRC_TRY(expr)                         \
  do {                                         \
    cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) return from_cuda(e_); \
  } while (0)

#define CSRC_TRY_S(expr)            \
  do {                              \
    csrc_status s_ = (expr);        \
    if (s_ != CSRC_OK) return s_;   \
  } while (0)

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

void free_plan(DevPlan& p) {
  dfree(p.band_row); dfree(p.band_plo); dfree(p.band_ntab); dfree(p.band_wp);
  dfree(p.wpage); dfree(p.wbase); dfree(p.wmask);
  dfree(p.acc_row); dfree(p.acc_ptr); dfree(p.acc_src); dfree(p.spill_buf);
  dfree(p.band_stage); dfree(p.stage_k); dfree(p.stage_r); dfree(p.jslot); dfree(p.jslot16);
  p = DevPlan();
}

// FP64 -> BF16, nearest with ties to even, straight from the double's bits (one rounding).
uint16_t f64_to_bf16(double v) {
  uint64_t b;
  std::memcpy(&b, &v, 8);
  const uint64_t sign = b >> 63;
  const int E = (int)((b >> 52) & 0x7ff);
  const uint64_t mant = b & ((1ULL << 52) - 1);
  if (E == 0x7ff) return (uint16_t)((sign << 15) | 0x7f80u | (mant ? 0x40u : 0u));  // inf / NaN
  if (E == 0) return (uint16_t)(sign << 15);  // zero / FP64 subnormal (far below BF16's range)
  const int e = E - 1023;                     // v = 1.m * 2^e
  // number of fraction bits kept: 7 for normal BF16 (e >= -126), fewer below
  const int keep = e >= -126 ? 7 : 7 - (-126 - e);
  if (keep < -1) return (uint16_t)(sign << 15);  // below half the smallest subnormal
  // significand with the implicit bit: 53 bits; keep (1 + keep) of them
  const uint64_t sig = (1ULL << 52) | mant;
  const int drop = 52 - keep;                  // 45 .. 53
  uint64_t q = drop >= 64 ? 0 : (sig >> drop);
  const uint64_t rem = drop >= 64 ? sig : (sig & ((1ULL << drop) - 1));
  const uint64_t half = 1ULL << (drop - 1);
  if (rem > half || (rem == half && (q & 1ULL))) ++q;
  // q now holds the rounded significand in units of 2^(e - keep)
  uint32_t out;
  if (e >= -126) {
    int eb = e + 127;
    if (q >> 8) {  // carried into a new binade
      q >>= 1;
      ++eb;
    }
    if (eb >= 255) return (uint16_t)((sign << 15) | 0x7f80u);
    out = ((uint32_t)eb << 7) | (uint32_t)(q & 0x7f);
  } else {
    // subnormal: value = q * 2^(e - keep) = q * 2^-133
    out = (uint32_t)q;  // q <= 128; q == 128 is the smallest normal (exponent field 1)
  }
  return (uint16_t)((sign << 15) | out);
}

// Section 3.1: smallest r with P(r) * B >= t * nnz, w_i = 1 + 2 * pairs(i), over rows [a, b).
void nnz_partition(const std::vector<int32_t>& ia, int32_t a, int32_t b, int32_t nb, std::vector<int32_t>& out) {
  out.assign((size_t)nb + 1, a);
  const int64_t tot = (int64_t)(b - a) + 2 * ((int64_t)ia[b] - ia[a]);
  int64_t P = 0;
  int32_t r = a;
  for (int32_t t = 1; t <= nb; ++t) {
    const unsigned __int128 goal = (unsigned __int128)t * (unsigned __int128)tot;
    while (r < b && (unsigned __int128)P * (unsigned __int128)nb < goal) {
      P += 1 + 2 * ((int64_t)ia[r + 1] - ia[r]);
      ++r;
    }
    out[t] = r;
  }
}

struct HostPlan {
  std::vector<int32_t> band_row{0}, band_plo, band_ntab, band_wp{0}, wpage, wbase;
  std::vector<int32_t> band_stage{0}, stage_k, stage_r;
  std::vector<uint64_t> wmask;
  int32_t max_slots = 0, max_tab = 0, smem = 0;
  int64_t spill = 0;
  bool covers = true;
};

// Ring stages of band [r0, r1) for the band kernel: consecutive units of B rows (B = 1:
// single rows; B > 1: node blocks, which are never cut), at most `units` of them and at
// most `cap` pairs per stage. A single row that does not fit in what is left of a stage
// is cut there and continues in the next one. With `out` null, only counts. Otherwise
// appends each stage's first pair and first row, then the band's end (ia[r1], r1), and
// closes the band in band_stage. Returns the number of stages, or -1 when a node block
// alone holds more than `cap` pairs.
int32_t build_stages(const std::vector<int32_t>& ia, int32_t r0, int32_t r1, int32_t units, int32_t cap, int32_t B,
                     HostPlan* out) {
  int64_t k = ia[r0];
  int32_t r = r0;
  const int64_t kend = ia[r1];
  int32_t count = 0;
  while (k < kend) {
    if (B == 1) {
      while (ia[(size_t)r + 1] <= k) ++r;  // the row holding pair k
    } else {
      while (ia[(size_t)r + B] <= k) r += B;  // the unit holding pair k
    }
    const int64_t ks = k;
    if (out) {
      out->stage_k.push_back((int32_t)ks);
      out->stage_r.push_back(r);
    }
    ++count;
    int32_t used = 0;
    while (k < kend && used < units) {
      const int64_t end = ia[(size_t)r + B];
      if (B > 1) {
        if (end - ks > cap) {
          if (used == 0) return -1;  // a node block larger than a stage
          break;
        }
        k = end;
        ++used;
        r += B;
        continue;
      }
      const int64_t take = std::min<int64_t>(end - k, ks + cap - k);
      if (take <= 0) break;
      k += take;
      ++used;
      if (k < end) break;  // the row continues in the next stage
      ++r;
    }
  }
  if (out) {
    out->stage_k.push_back((int32_t)kend);
    out->stage_r.push_back(r1);
    out->band_stage.push_back((int32_t)out->stage_k.size());
  }
  return count;
}

// Build the window plan: each partition band becomes one or more execution bands
// whose shared memory (window of np pages, page table, ia slice and stage table, as laid
// out by BandLayout) fits `budget` bytes. A band that does not fit is split at its
// non-zero midpoint. A single row that still does not fit gets a capped window when
// allow_overflow (targets outside it take the global-atomic path); otherwise planning fails.
bool build_host_plan(const csrc_matrix_s* h, const std::vector<int32_t>& part, int32_t budget, int mode, int rk,
                     bool allow_overflow, int32_t stage_units, int32_t stage_cap, int32_t B, HostPlan& hp) {
  const int32_t n = h->n;
  const std::vector<int32_t>& ia = h->ia;
  const std::vector<int32_t>& ja = h->ja;
  const int32_t npages = (n + kPageRows - 1) / kPageRows;
  std::vector<int32_t> page_stamp((size_t)npages + 1, -1), row_stamp((size_t)n + 1, -1);
  int32_t stamp = 0;
  std::vector<int32_t> pages;
  const int xb = rk * window_x_bytes(mode), ab = rk * window_acc_bytes(mode);
  auto bytes_of = [&](int64_t np, int64_t ntab, int32_t r0, int32_t r1, int32_t nst) -> int64_t {
    if (np > 32767 || ntab > (1 << 24)) return INT64_MAX;
    const int32_t st0 = (int32_t)hp.stage_k.size();
    return BandLayout::make((int)(np * kPageRows), xb, ab, (int)ntab, r0, r1, st0, st0 + nst).end;
  };
  struct Range { int32_t a, b; };
  std::vector<Range> stack;
  for (size_t t = 0; t + 1 < part.size(); ++t) {
    if (part[t + 1] <= part[t]) continue;  // empty band
    stack.push_back({part[t], part[t + 1]});
    while (!stack.empty()) {
      Range rg = stack.back();
      stack.pop_back();
      const int32_t r0 = rg.a, r1 = rg.b;
      ++stamp;
      pages.clear();
      for (int32_t p = r0 >> kPageShift; p <= (r1 - 1) >> kPageShift; ++p) {
        page_stamp[p] = stamp;
        pages.push_back(p);
      }
      int32_t minpage = r0 >> kPageShift;
      for (int32_t k = ia[r0]; k < ia[r1]; ++k) {
        const int32_t p = ja[k] >> kPageShift;
        if (page_stamp[p] != stamp) {
          page_stamp[p] = stamp;
          pages.push_back(p);
          if (p < minpage) minpage = p;
        }
      }
      const int32_t phi = (r1 - 1) >> kPageShift;
      int64_t ntab = (int64_t)phi - minpage + 1;
      const int32_t nst = build_stages(ia, r0, r1, stage_units, stage_cap, B, nullptr);
      if (nst < 0) return false;
      bool fits = bytes_of((int64_t)pages.size(), ntab, r0, r1, nst) <= budget;
      if (!fits && r1 - r0 > B) {
        std::vector<int32_t> half;
        nnz_partition(ia, r0, r1, 2, half);
        int32_t mid = half[1] / B * B;  // bands hold whole node blocks
        if (mid <= r0 || mid >= r1) mid = r0 + (r1 - r0) / (2 * B) * B;
        stack.push_back({mid, r1});  // processed after the left half
        stack.push_back({r0, mid});
        continue;
      }
      std::sort(pages.begin(), pages.end());
      if (!fits) {
        if (!allow_overflow || B > 1) return false;
        hp.covers = false;
        // keep the band's own pages and the nearest target pages that fit
        const int64_t own = phi - (r0 >> kPageShift) + 1;
        if (bytes_of(own, own, r0, r1, nst) > budget) return false;
        int64_t keep = own;
        int32_t lowest = r0 >> kPageShift;
        for (int64_t q = (int64_t)pages.size() - own - 1; q >= 0; --q) {
          const int32_t p = pages[(size_t)q];
          if (bytes_of(keep + 1, (int64_t)phi - p + 1, r0, r1, nst) > budget) break;
          ++keep;
          lowest = p;
        }
        pages.erase(pages.begin(), pages.end() - keep);
        minpage = lowest;
        ntab = (int64_t)phi - minpage + 1;
      }
      const int64_t used_bytes = bytes_of((int64_t)pages.size(), ntab, r0, r1, nst);
      // rows below r0 that this band writes (spill rows)
      for (int32_t k = ia[r0]; k < ia[r1]; ++k) {
        const int32_t j = ja[k];
        if (j < r0) row_stamp[j] = stamp;
      }
      hp.band_plo.push_back(minpage);
      hp.band_ntab.push_back((int32_t)ntab);
      for (int32_t p : pages) {
        uint64_t mask = 0;
        const int32_t rbase = p << kPageShift;
        for (int e = 0; e < kPageRows; ++e) {
          const int32_t j = rbase + e;
          if (j < r0 && j < n && row_stamp[j] == stamp) mask |= 1ULL << e;
        }
        hp.wpage.push_back(p);
        hp.wbase.push_back((int32_t)hp.spill);
        hp.wmask.push_back(mask);
        hp.spill += __builtin_popcountll(mask);
      }
      hp.band_wp.push_back((int32_t)hp.wpage.size());
      hp.band_row.push_back(r1);
      build_stages(ia, r0, r1, stage_units, stage_cap, B, &hp);
      hp.max_slots = std::max(hp.max_slots, (int32_t)pages.size() * kPageRows);
      hp.max_tab = std::max(hp.max_tab, (int32_t)ntab);
      hp.smem = std::max(hp.smem, (int32_t)used_bytes);
    }
  }
  if (hp.band_row.size() == 1) hp.band_row.push_back(0);  // n == 0
  return true;
}

template <typename T>
cudaError_t upload(T** d, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = dmalloc(d, v.size());
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  return e;
}

// Window plan for rk columns per pass into p (freed first). Sets covers when every
// scatter target of every band lies in its window.
csrc_status build_plan(csrc_matrix_s* h, int32_t nbands, int rk, int B, DevPlan& p, bool& covers,
                       std::vector<int32_t>* part_out) {
  // paper-rule partition
  int32_t nb = nbands;
  if (nb <= 0) {
    const int64_t nnz = (int64_t)h->n + 2 * h->h;
    const int64_t target = 160000;  // non-zeros per band before window splitting
    int64_t k = (nnz + (int64_t)h->sms * target - 1) / ((int64_t)h->sms * target);
    if (k < 1) k = 1;
    nb = (int32_t)std::min<int64_t>((int64_t)h->sms * k, std::max<int32_t>(1, h->n));
  }
  std::vector<int32_t> part;
  nnz_partition(h->ia, 0, h->n, nb, part);
  // execution bands start at node-block boundaries
  std::vector<int32_t> epart(part);
  if (B > 1)
    for (auto& v : epart) v = v == h->n ? v : v / B * B;
  const int mode = mode_of(h->arith, h->storage);
  const int32_t budget = band_smem_limit(mode) - band_ring_bytes(mode);  // everything after the ring
  // lanes per unit: the smallest G whose T/G units of average size fill at most one stage
  const double avg = h->n > 0 ? (double)B * (double)h->h / (double)h->n : 0.0;
  int32_t group = 1;
  const int32_t gmax = B > 1 ? 16 : 8;
  while (group < gmax && (double)(kBandThreads / group) * avg > (double)kStageCap) group *= 2;
  // long single-vector rows (32 or more pairs on average): 16 lanes per row in a CTA of
  // twice the threads; a stage still holds 64 rows
  if (B == 1 && rk == 1 && group == 8 && avg >= 32.0) group = 16;
  const int32_t units = band_threads(group, B, rk) / group;
  HostPlan hp;
  bool ok = build_host_plan(h, epart, budget, mode, rk, false, units, kStageCap, B, hp);
  if (!ok && rk == 1 && B == 1) {
    hp = HostPlan();
    ok = build_host_plan(h, epart, budget, mode, rk, true, units, kStageCap, B, hp);
  }
  if (!ok) return CSRC_ERR_NOT_PARTITIONED;
  // accumulation map: group spill entries by row (stable: band order)
  std::vector<int32_t> cnt((size_t)h->n + 1, 0);
  for (size_t q = 0; q < hp.wpage.size(); ++q) {
    uint64_t m = hp.wmask[q];
    while (m) {
      const int e = __builtin_ctzll(m);
      m &= m - 1;
      cnt[(size_t)(hp.wpage[q] << kPageShift) + e + 1]++;
    }
  }
  std::vector<int32_t> acc_row, acc_ptr{0};
  std::vector<int32_t> start((size_t)h->n + 1, 0);
  for (int32_t r = 0; r < h->n; ++r) start[r + 1] = start[r] + cnt[r + 1];
  for (int32_t r = 0; r < h->n; ++r)
    if (cnt[r + 1]) {
      acc_row.push_back(r);
      acc_ptr.push_back(start[r + 1]);
    }
  std::vector<int32_t> acc_src((size_t)hp.spill);
  std::vector<int32_t> fill(start.begin(), start.end() - 1);
  for (size_t q = 0; q < hp.wpage.size(); ++q) {
    uint64_t m = hp.wmask[q];
    int32_t pos = hp.wbase[q];
    while (m) {
      const int e = __builtin_ctzll(m);
      m &= m - 1;
      const int32_t row = (hp.wpage[q] << kPageShift) + e;
      acc_src[(size_t)fill[row]++] = pos++;
    }
  }
  // upload
  free_plan(p);
  cudaStream_t s = 0;
  p.nb = (int32_t)hp.band_row.size() - 1;
  if (h->n == 0) p.nb = 0;
  CSRC_TRY(upload(&p.band_row, hp.band_row, s));
  CSRC_TRY(upload(&p.band_plo, hp.band_plo, s));
  CSRC_TRY(upload(&p.band_ntab, hp.band_ntab, s));
  CSRC_TRY(upload(&p.band_wp, hp.band_wp, s));
  CSRC_TRY(upload(&p.wpage, hp.wpage, s));
  CSRC_TRY(upload(&p.wbase, hp.wbase, s));
  CSRC_TRY(upload(&p.wmask, hp.wmask, s));
  CSRC_TRY(upload(&p.acc_row, acc_row, s));
  CSRC_TRY(upload(&p.acc_ptr, acc_ptr, s));
  CSRC_TRY(upload(&p.acc_src, acc_src, s));
  hp.stage_k.resize(hp.stage_k.size() + kMetaPad, 0);  // rounded-up bulk copies read past the end
  hp.stage_r.resize(hp.stage_r.size() + kMetaPad, 0);
  CSRC_TRY(upload(&p.band_stage, hp.band_stage, s));
  CSRC_TRY(upload(&p.stage_k, hp.stage_k, s));
  CSRC_TRY(upload(&p.stage_r, hp.stage_r, s));
  CSRC_TRY(cudaMalloc(&p.spill_buf, std::max<size_t>(1, (size_t)hp.spill * rk * h->xbytes())));
  if (B == 1) {
    // window slot of every stored pair: page q of band b's window holds slots q*64 .. q*64+63.
    // Pairs whose page is outside the window (plans with overflow, which only the atomic
    // strategy runs) get slot 0.
    const size_t hcap = ((size_t)h->h + kPairAlign - 1) / kPairAlign * kPairAlign + kPairAlign;
    std::vector<int32_t> jslot(hcap, 0);
    std::vector<int32_t> qmap;
    for (size_t b = 0; b + 1 < hp.band_row.size(); ++b) {
      const int32_t plo = hp.band_plo[b], ntab = hp.band_ntab[b];
      qmap.assign((size_t)std::max(ntab, 0), -1);
      for (int32_t q = hp.band_wp[b]; q < hp.band_wp[b + 1]; ++q) {
        const int32_t t = hp.wpage[(size_t)q] - plo;
        if (t >= 0 && t < ntab) qmap[(size_t)t] = q - hp.band_wp[b];
      }
      const int64_t k0 = h->ia[(size_t)hp.band_row[b]], k1 = h->ia[(size_t)hp.band_row[b + 1]];
      for (int64_t k = k0; k < k1; ++k) {
        const int32_t j = h->ja[(size_t)k];
        const int32_t t = (j >> kPageShift) - plo;
        const int32_t q = (t >= 0 && t < ntab) ? qmap[(size_t)t] : -1;
        jslot[(size_t)k] = q < 0 ? 0 : (q << kPageShift) | (j & (kPageRows - 1));
      }
    }
    bool narrow = (h->flags & CSRC_FLAG_COMPRESS_INDICES) != 0;
    for (size_t b = 0; narrow && b + 1 < hp.band_row.size(); ++b)
      narrow = (int64_t)(hp.band_wp[b + 1] - hp.band_wp[b]) * kPageRows <= 65536;
    if (narrow) {
      std::vector<uint16_t> j16(jslot.size());
      for (size_t k = 0; k < jslot.size(); ++k) j16[k] = (uint16_t)jslot[k];
      CSRC_TRY(upload(&p.jslot16, j16, s));
    } else {
      CSRC_TRY(upload(&p.jslot, jslot, s));
    }
  }
  CSRC_TRY(cudaStreamSynchronize(s));
  p.spill = hp.spill;
  p.group = group;
  p.block = B;
  p.nstages = (int64_t)hp.stage_k.size() - kMetaPad - (int64_t)(hp.band_stage.size() - 1);
  p.nacc = (int64_t)acc_row.size();
  p.max_slots = hp.max_slots;
  p.max_tab = hp.max_tab;
  p.smem_bytes = band_ring_bytes(mode) + hp.smem;
  p.total_pages = (int64_t)hp.wpage.size();
  p.band_pairs.resize((size_t)p.nb);
  for (int32_t b = 0; b < p.nb; ++b)
    p.band_pairs[(size_t)b] = (int64_t)h->ia[(size_t)hp.band_row[(size_t)b + 1]] - h->ia[(size_t)hp.band_row[(size_t)b]];
  covers = hp.covers;
  if (part_out) part_out->swap(part);
  return CSRC_OK;
}

// ---------------------------------------------------------------------------- owner plans
// Automatic band count of an owner plan: a multiple of the CTAs the GPU holds at once
// (SMs x resident CTAs for rk columns), with about kOwnerBandNnz non-zeros per band, so
// that the bands of equal weight finish in whole waves.
constexpr int64_t kOwnerBandNnz = 100000;
int32_t owner_auto_bands(const csrc_matrix_s* h, int rk) {
  const int64_t nnz = (int64_t)h->n + 2 * h->h;
  if (rk > 1) {
    // wider passes: the window size splits the bands much further anyway; start from bands of
    // kOwnerBandNnz non-zeros and let the splits decide (measured faster than whole waves here)
    return (int32_t)std::min<int64_t>(std::max<int64_t>(1, (nnz + kOwnerBandNnz - 1) / kOwnerBandNnz),
                                      std::max<int32_t>(1, h->n));
  }
  // FP32 / BF16 values leave room for larger bands (fewer spills; measured on q1v_96: 1,216
  // bands against 2,432 for FP64, whose product the FP64 pipe bounds)
  const int64_t target = h->owner_mode() == OM_F64 ? kOwnerBandNnz : kOwnerBandNnz * 9 / 5;
  const int64_t slots = (int64_t)h->sms * owner_ctas_per_sm(rk);
  int64_t waves = (nnz + slots * target - 1) / (slots * target);
  if (waves < 1) waves = 1;
  return (int32_t)std::min<int64_t>(slots * waves, std::max<int32_t>(1, h->n));
}

// Owner lists for rk columns per pass from the Section 3.1 partition into nbands bands
// (0 = automatic); bands whose windows exceed shared memory are split further.
csrc_status build_owner(csrc_matrix_s* h, int rk, int32_t nbands, OwnerPlan& p, std::vector<int32_t>* part_out) {
  int32_t nb = nbands > 0 ? std::min<int32_t>(nbands, std::max<int32_t>(1, h->n)) : owner_auto_bands(h, rk);
  std::vector<int32_t> part;
  nnz_partition(h->ia, 0, h->n, nb, part);
  CSRC_TRY_S(build_owner_plan(h->n, h->h, h->ia, h->ja, part, rk, h->owner_mode(), owner_smem_budget(rk),
                              (int)h->vbytes(), h->d_al, h->au_ptr(), h->d_ad, h->sym, p));
  // An automatic single-column count whose windows did not fit was split band by band, which
  // leaves halves beside whole bands (uneven work in the last wave). Partition again into the
  // next whole number of waves at or above the split count, so that every band is about equal
  // (Delaunay 2M in FP64: 608 bands split into 1,202, then 1,216 equal bands: 0.143 -> 0.110 ms).
  const int64_t slots = (int64_t)h->sms * owner_ctas_per_sm(rk);
  for (int it = 0; nbands <= 0 && rk == 1 && it < 3 && p.nb > nb; ++it) {
    const int32_t nb2 = (int32_t)std::min<int64_t>((p.nb + slots - 1) / slots * slots, std::max<int32_t>(1, h->n));
    if (nb2 <= nb) break;
    OwnerPlan q;
    std::vector<int32_t> part2;
    nnz_partition(h->ia, 0, h->n, nb2, part2);
    CSRC_TRY_S(build_owner_plan(h->n, h->h, h->ia, h->ja, part2, rk, h->owner_mode(), owner_smem_budget(rk),
                                (int)h->vbytes(), h->d_al, h->au_ptr(), h->d_ad, h->sym, q));
    free_owner_plan(p);
    p = std::move(q);
    part.swap(part2);
    nb = nb2;
  }
  if (part_out) part_out->swap(part);
  return CSRC_OK;
}

void drop_owner_plans(csrc_matrix_s* h) {
  free_owner_plan(h->oplan);
  h->have_oplan = false;
  for (int i = 0; i < 3; ++i) {
    free_owner_plan(h->oplan_rk[i]);
    h->have_orp[i] = h->fits_orp[i] = false;
  }
  for (int i = 0; i < 4; ++i) {
    free_owner_plan(h->oplan_bt[i]);
    h->have_obt[i] = h->fits_obt[i] = false;
  }
}

// The owner plan of a batch member for rk columns per pass: bands of about band_nnz non-zeros
// whatever the SM count (the batch's other members fill the GPU; a single product's automatic
// count would cut each small member into many tiny bands). Rebuilt when band_nnz changes.
csrc_status owner_batch_for(csrc_matrix_s* h, int rk, int64_t band_nnz, OwnerPlan** out) {
  const int i = rk == 1 ? 0 : (rk == 2 ? 1 : (rk == 4 ? 2 : 3));
  if (h->have_obt[i] && h->obt_target[i] != band_nnz) {
    free_owner_plan(h->oplan_bt[i]);
    h->have_obt[i] = false;
  }
  if (!h->have_obt[i]) {
    h->obt_target[i] = band_nnz;
    const int64_t nnz = (int64_t)h->n + 2 * h->h;
    const int64_t nb = std::min<int64_t>(std::max<int64_t>(1, (nnz + band_nnz - 1) / band_nnz),
                                         std::max<int32_t>(1, h->n));
    const csrc_status st = build_owner(h, rk, (int32_t)nb, h->oplan_bt[i], nullptr);
    if (st != CSRC_OK && st != CSRC_ERR_NOT_PARTITIONED) return st;
    h->have_obt[i] = true;
    h->fits_obt[i] = st == CSRC_OK;
    ++h->generation;
  }
  if (!h->fits_obt[i]) return CSRC_ERR_NOT_PARTITIONED;
  *out = &h->oplan_bt[i];
  return CSRC_OK;
}

// The owner plan for rk = 1, 2, 4 or 8 columns per pass, built on first use. Single vectors
// use the band count of csrc_partition (or the autotuner's); wider passes pick their own.
csrc_status owner_for(csrc_matrix_s* h, int rk, OwnerPlan** out) {
  if (rk == 1) {
    if (!h->have_oplan) {
      CSRC_TRY_S(build_owner(h, 1, h->owner_nbands, h->oplan, &h->part));
      h->have_oplan = true;
      ++h->generation;
    }
    *out = &h->oplan;
    return CSRC_OK;
  }
  const int i = rk == 2 ? 0 : (rk == 4 ? 1 : 2);
  if (!h->have_orp[i]) {
    const csrc_status st = build_owner(h, rk, 0, h->oplan_rk[i], nullptr);
    if (st != CSRC_OK && st != CSRC_ERR_NOT_PARTITIONED) return st;
    h->have_orp[i] = true;  // remembered either way: a window of rk columns may not fit
    h->fits_orp[i] = st == CSRC_OK;
  }
  if (!h->fits_orp[i]) return CSRC_ERR_NOT_PARTITIONED;
  *out = &h->oplan_rk[i];
  return CSRC_OK;
}

// Componentwise error bound of the window strategy at the handle's precision (relative to
// sum_j |a_ij||x_j|): u_v + u_x + (L + P - 1) u_a, L the longest row, P the most partial sums of
// a row (its own band's and the spilled ones), u_v / u_x / u_a the unit roundoffs of the values,
// of x in the window and of the multiply-adds. Builds the single-vector lists if needed.
csrc_status owner_error_bound(csrc_matrix_s* h, double* out) {
  *out = 0.0;
  if (h->n == 0) return CSRC_OK;
  OwnerPlan* p = nullptr;
  CSRC_TRY_S(owner_for(h, 1, &p));
  const double u53 = std::ldexp(1.0, -53), u24 = std::ldexp(1.0, -24), u8 = std::ldexp(1.0, -8);
  double uv = 0.0, ux = 0.0, ua = u53;
  switch (p->mode) {
    case OM_F64: break;
    case OM_F32: uv = u24; ua = u24; break;          // x is given as float
    case OM_BF16: uv = u8; ua = u24; break;
    case OM_F32_X64: uv = u24; ux = u24; ua = u24; break;
    default: uv = u8; ux = u24; ua = u24; break;     // OM_BF16_X64
  }
  const double terms = (double)h->max_row_nnz + (double)p->max_parts - 1.0;
  const double g = terms * ua / (1.0 - terms * ua);  // gamma_terms
  *out = uv + ux + uv * ux + g * (1.0 + uv) * (1.0 + ux);
  return CSRC_OK;
}

// ---------------------------------------------------------------------------- stream-order plans
// The stream-order plan of the window-atomic and atomic strategies, from the band count of
// csrc_partition (0 = automatic); built on first use.
csrc_status make_plan(csrc_matrix_s* h) {
  h->have_plan = false;
  free_plan(h->plan_b1);
  h->have_b1 = false;
  csrc_status st = CSRC_ERR_NOT_PARTITIONED;
  if (h->block > 1) {
    st = build_plan(h, h->part_nbands, 1, h->block, h->plan, h->plan_covers, nullptr);
    if (st != CSRC_OK && st != CSRC_ERR_NOT_PARTITIONED) return st;
    if (st == CSRC_OK && !h->plan_covers) st = CSRC_ERR_NOT_PARTITIONED;
  }
  if (st != CSRC_OK) CSRC_TRY_S(build_plan(h, h->part_nbands, 1, 1, h->plan, h->plan_covers, nullptr));
  h->have_plan = true;
  ++h->generation;
  return CSRC_OK;
}

// A single-vector stream-order plan of plain rows (the atomic strategy and the batched kernel
// run rows one at a time): the main plan, or, when that one uses node blocks, a second plan.
csrc_status plan_b1_for(csrc_matrix_s* h, DevPlan** out, bool* covers) {
  if (!h->have_plan) CSRC_TRY_S(make_plan(h));
  if (h->plan.block == 1) {
    *out = &h->plan;
    *covers = h->plan_covers;
    return CSRC_OK;
  }
  if (!h->have_b1) {
    CSRC_TRY_S(build_plan(h, h->part_nbands, 1, 1, h->plan_b1, h->covers_b1, nullptr));
    h->have_b1 = true;
  }
  *out = &h->plan_b1;
  *covers = h->covers_b1;
  return CSRC_OK;
}

cudaEvent_t pooled_event(csrc_matrix_s* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Runs `launch` on stream s; with profiling on, brackets it with a pair of events.
template <typename F>
cudaError_t timed_launch(csrc_matrix_s* h, int32_t kind, cudaStream_t s, F&& launch, int32_t kernels = 1) {
  if (!h->profiling) return launch();
  cudaEvent_t a = pooled_event(h), b = pooled_event(h);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, s);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e != cudaSuccess) return e;
  h->timed.push_back({kind, kernels, a, b});
  return cudaSuccess;
}

void release_timing(csrc_matrix_s* h) {
  for (auto& t : h->timed) {
    h->event_pool.push_back(t.start);
    h->event_pool.push_back(t.stop);
  }
  h->timed.clear();
}

// Makes the handle's device current for the duration of an entry point and gives the
// caller's current device back when the entry point returns (nested entries that find the
// handle's device already current change nothing).
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  csrc_status enter(const csrc_matrix_s* h) {
    if (cudaGetDevice(&prev) != cudaSuccess) return CSRC_ERR_CUDA;
    if (prev != h->device) {
      if (cudaSetDevice(h->device) != cudaSuccess) return CSRC_ERR_CUDA;
      switched = true;
    }
    return CSRC_OK;
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Arguments of one band-kernel launch: the handle's arrays and plan p, al and au swapped
// for the transpose (Section 5); x and y point at the pass's first column, ldx is their
// row stride and rk the columns per pass.
BandArgs band_args(const csrc_matrix_s* h, const DevPlan& p, bool transpose, const void* x, void* y, void* spill,
                   int ldx, int rk, bool atomic) {
  BandArgs a;
  // the window strategy's plain-row kernels read window slots, and with double-float
  // arithmetic pre-split scatter operands
  const bool local = !atomic && p.block == 1;
  (void)rk;
  a.n = h->n;
  a.ia = h->d_ia;
  a.ja = local && p.jslot ? p.jslot : h->d_ja;
  a.ja16 = local ? p.jslot16 : nullptr;
  a.band_stage = p.band_stage;
  a.stage_k = p.stage_k;
  a.stage_r = p.stage_r;
  a.group = p.group;
  a.al = transpose ? h->au_ptr() : h->d_al;  // gathered values
  a.au = transpose ? h->d_al : h->au_ptr();  // scattered values (the same array when symmetric)
  if (local && h->arith == ARITH_DF32 && !h->sym) a.au = transpose ? h->d_al_df : h->d_au_df;
  a.ad = h->d_ad;
  a.x = x;
  a.y = y;
  a.band_row = p.band_row;
  a.band_plo = p.band_plo;
  a.band_ntab = p.band_ntab;
  a.band_wp = p.band_wp;
  a.wpage = p.wpage;
  a.wbase = p.wbase;
  a.wmask = p.wmask;
  a.spill = spill;
  a.status = h->d_status;
  a.band_offset = 0;
  a.x_bulk = (reinterpret_cast<uintptr_t>(x) & 15u) == 0u;
  a.ldx = ldx;
  a.rk = rk;
  a.block = p.block;
  return a;
}

// Arguments of one owner-kernel launch on plan p: A x, or A^T x with the exchanged values
// (Section 5); x and y point at the pass's first column, ldx is their row stride.
OwnerArgs owner_args(const OwnerPlan& p, bool transpose, const void* x, void* y, void* spill, int ldx, int lds) {
  OwnerArgs a;
  a.band = p.band;
  a.band_slice = p.band_slice;
  a.slice_off = p.slice_off;
  a.lane = p.lane;
  a.spill_row = p.spill_row;
  a.spill_pos = p.spill_pos;
  a.S = p.S;
  a.V = transpose ? p.VT : p.VA;
  a.x = x;
  a.y = y;
  a.spill = spill;
  a.ldx = ldx;
  a.lds = lds;
  a.band_offset = 0;
  return a;
}

// The window strategy on owner plan p: the owner kernel, then the accumulation of spills.
csrc_status run_owner(csrc_matrix_s* h, const OwnerPlan& p, bool transpose, const void* x, void* y, void* spill,
                      int ldx, int rk, cudaStream_t s) {
  const OwnerArgs a = owner_args(p, transpose, x, y, spill, ldx, rk);
  CSRC_TRY(timed_launch(h, CSRC_KERNEL_PRODUCT, s,
                        [&] { return launch_owner(p.mode, rk, a, p.nb, p.smem_bytes, s); }));
  if (p.nacc > 0)
    CSRC_TRY(timed_launch(h, CSRC_KERNEL_ACCUMULATE, s, [&] {
      return launch_owner_accumulate(p.mode, p.nacc, rk, ldx, p.acc_row, p.acc_ptr, spill, y, s);
    }));
  return CSRC_OK;
}

csrc_status run_spmv(csrc_matrix_s* h, const void* x, void* y, csrc_strategy st, cudaStream_t s, bool transpose) {
  if (!h || !x || !y) return CSRC_ERR_INVALID_ARG;
  if (st < CSRC_STRAT_AUTO || st > CSRC_STRAT_WINDOW_ATOMIC) return CSRC_ERR_INVALID_ARG;
  if (h->m == 0) return CSRC_OK;
  // x and y lengths: n each, or m and n (A x) / n and m (A^T x) for a rectangular matrix
  const size_t vb = (size_t)h->n * h->xbytes();
  const size_t xb = (size_t)(transpose ? h->n : h->m) * h->xbytes();
  const size_t yb = (size_t)(transpose ? h->m : h->n) * h->xbytes();
  const char* xa = static_cast<const char*>(x);
  const char* ya = static_cast<const char*>(y);
  if (xa < ya + yb && ya < xa + xb) return CSRC_ERR_ALIAS;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  csrc_strategy strat = st;
  if (strat == CSRC_STRAT_AUTO) strat = h->tuned ? (csrc_strategy)h->tuned : CSRC_STRAT_WINDOW;
  OwnerPlan* op = nullptr;
  if (h->n > 0 && strat == CSRC_STRAT_WINDOW) {
    const csrc_status ps = owner_for(h, 1, &op);
    if (ps == CSRC_ERR_NOT_PARTITIONED && st == CSRC_STRAT_AUTO) strat = CSRC_STRAT_ATOMIC;  // no window fits
    else if (ps != CSRC_OK) return ps;
  }
  if (h->n > 0 && (strat == CSRC_STRAT_WINDOW_ATOMIC || strat == CSRC_STRAT_ATOMIC) && !h->have_plan)
    CSRC_TRY_S(make_plan(h));
  if (h->n > 0 && strat == CSRC_STRAT_WINDOW_ATOMIC && !h->plan_covers) return CSRC_ERR_NOT_PARTITIONED;
  if (h->n > 0 && strat == CSRC_STRAT_COLOR && h->ncolors == 0) return CSRC_ERR_NOT_COLORED;
  // host vectors are staged through handle-owned device buffers (m entries: room for either)
  const size_t sb = (size_t)h->m * h->xbytes();
  const bool xdev = is_device_ptr(x), ydev = is_device_ptr(y);
  const void* dx = x;
  void* dy = y;
  if (!xdev) {
    if (!h->d_xs) CSRC_TRY(cudaMalloc(&h->d_xs, sb));
    CSRC_TRY(cudaMemcpyAsync(h->d_xs, x, xb, cudaMemcpyHostToDevice, s));
    dx = h->d_xs;
  }
  if (!ydev) {
    if (!h->d_ys) CSRC_TRY(cudaMalloc(&h->d_ys, sb));
    dy = h->d_ys;
  }
  const void* g = transpose ? h->au_ptr() : h->d_al;  // gathered values
  const void* sc = transpose ? h->d_al : h->au_ptr(); // scattered values
  if (h->n == 0) {
    // nothing to do for A_S
  } else if (strat == CSRC_STRAT_WINDOW) {
    CSRC_TRY_S(run_owner(h, *op, transpose, dx, dy, op->spill_buf, 1, 1, s));
  } else if (strat == CSRC_STRAT_COLOR) {
    CSRC_TRY(cudaMemsetAsync(dy, 0, vb, s));
    CSRC_TRY(cudaMemsetAsync(h->d_barrier, 0, sizeof(unsigned), s));
    const int group = color_group(h->n > 0 ? (double)h->h / (double)h->n : 0.0);
    CSRC_TRY(timed_launch(h, CSRC_KERNEL_PRODUCT, s, [&] {
      const void* cau = h->sym ? h->d_cal : h->d_cau;
      return launch_color_spmv(h->storage, group, h->ncolors, h->d_color_ptr, h->d_color_desc, h->d_cja,
                               transpose ? cau : h->d_cal, transpose ? h->d_cal : cau, h->d_ad, dx, dy, h->d_barrier,
                               h->d_status, s);
    }));
  } else {
    const bool atomic = strat == CSRC_STRAT_ATOMIC;
    DevPlan* p = &h->plan;  // the atomic strategy runs plain rows
    bool covers = h->plan_covers;
    if (atomic) CSRC_TRY_S(plan_b1_for(h, &p, &covers));
    const BandArgs a = band_args(h, *p, transpose, dx, dy, p->spill_buf, 1, 1, atomic);
    if (atomic) CSRC_TRY(cudaMemsetAsync(dy, 0, vb, s));
    CSRC_TRY(timed_launch(h, CSRC_KERNEL_PRODUCT, s,
                          [&] { return launch_band(h->arith, h->storage, atomic, a, p->nb, p->smem_bytes, s); }));
    if (!atomic && p->nacc > 0)
      CSRC_TRY(timed_launch(h, CSRC_KERNEL_ACCUMULATE, s, [&] {
        return launch_accumulate(h->arith, h->storage, p->nacc, 1, 1, p->acc_row, p->acc_ptr, p->acc_src,
                                 p->spill_buf, dy, s);
      }));
  }
  // the auxiliary CSR of a rectangular matrix: A_R x added to y[0..n), or A_R^T x into y[n..m)
  if (h->rect()) {
    if (!transpose) {
      CSRC_TRY(timed_launch(h, CSRC_KERNEL_OTHER, s, [&] {
        return launch_rect_rows(h->storage, h->nrrows, h->d_rrow, h->d_rptr, h->d_rcol, h->d_rval, dx, dy, s);
      }));
    } else {
      CSRC_TRY(timed_launch(h, CSRC_KERNEL_OTHER, s, [&] {
        return launch_rect_cols(h->storage, h->m - h->n, h->n, h->d_tptr, h->d_trow, h->d_tval, dx, dy, s);
      }));
    }
  }
  if (!ydev) CSRC_TRY(cudaMemcpyAsync(y, dy, yb, cudaMemcpyDeviceToHost, s));
  return CSRC_OK;
}

// ---------------------------------------------------------------------------- batched products
// A batch executor. Each member runs at its own mode (storage and precision): members whose
// strategy is the window strategy become units (member, column chunk of rk columns), whose
// bands are tiles of one owner-kernel launch per (mode, rk) group, followed by one
// accumulation launch per mode over all units; members tuned to another strategy run their
// own launches. The whole sequence is captured in a CUDA graph, cached by its arguments and
// replayed while the members' plans are unchanged.
struct BatchExec {
  int device = 0;
  std::vector<csrc_matrix_s*> hs;
  std::vector<uint64_t> gens;
  std::vector<const void*> xs;
  std::vector<void*> ys;
  int transpose = 0;
  int32_t nrhs = 1;
  OwnerArgs* d_units = nullptr;
  OwnerTile* d_tiles = nullptr;
  OwnerAccArgs* d_acc = nullptr;
  int64_t* d_offs = nullptr;
  std::vector<void*> spills;  // spill buffers the executor owns (chunks of several columns)
  std::vector<int32_t> others;  // members that run their own launches after the graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;  // kernel launches per replay
  ~BatchExec() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    dfree(d_units); dfree(d_tiles); dfree(d_acc); dfree(d_offs);
    for (void* p : spills) dfree(p);
  }
};

std::mutex g_batch_mutex;
std::vector<BatchExec*> g_batches;  // most recently used last
constexpr size_t kMaxBatches = 8;

void drop_batches_of(const csrc_matrix_s* h) {
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  for (size_t i = 0; i < g_batches.size();) {
    BatchExec* e = g_batches[i];
    if (std::find(e->hs.begin(), e->hs.end(), h) != e->hs.end()) {
      delete e;
      g_batches.erase(g_batches.begin() + (long)i);
    } else {
      ++i;
    }
  }
}

bool batch_matches(const BatchExec* e, const csrc_handle* hs, int32_t batch, const void* const* X, void* const* Y,
                   int32_t nrhs, int transpose, int device) {
  if (e->device != device || e->transpose != transpose || e->nrhs != nrhs || (int32_t)e->hs.size() != batch)
    return false;
  for (int32_t b = 0; b < batch; ++b)
    if (e->hs[(size_t)b] != hs[b] || e->gens[(size_t)b] != hs[b]->generation || e->xs[(size_t)b] != X[b] ||
        e->ys[(size_t)b] != Y[b])
      return false;
  return true;
}

// The column chunks of nrhs columns: the widest pass first (rk = 8, 4, 2, 1, capped by the
// handle's tuned k-tile), then narrower ones for the remainder.
std::vector<std::pair<int32_t, int>> column_chunks(const csrc_matrix_s* h, int32_t nrhs) {
  std::vector<std::pair<int32_t, int>> out;
  const int cap = h->tuned_rk > 0 ? h->tuned_rk : 8;
  for (int32_t c0 = 0; c0 < nrhs;) {
    int rk = 8;
    while (rk > 1 && (rk > cap || c0 + rk > nrhs)) rk /= 2;
    out.push_back({c0, rk});
    c0 += rk;
  }
  return out;
}
csrc_status build_batch(const csrc_handle* hs, int32_t batch, const void* const* X, void* const* Y, int32_t nrhs,
                        int transpose, int device, BatchExec** out) {
  BatchExec* e = new BatchExec();
  auto fail = [&](csrc_status st) {
    delete e;
    return st;
  };
  e->device = device;
  e->transpose = transpose;
  e->nrhs = nrhs;
  std::vector<int32_t>& others = e->others;
  struct Unit {
    const OwnerPlan* p;
    int mode, rk;
  };
  std::vector<Unit> units;
  std::vector<OwnerArgs> uargs;
  std::vector<OwnerAccArgs> uacc;
  // non-zeros per band: kOwnerBandNnz, or less when the whole batch would not fill four waves
  // of the GPU's resident CTAs
  int64_t total_nnz = 0;  // non-zeros of all the column chunks of all members
  int sms = 1;
  for (int32_t b = 0; b < batch; ++b) {
    total_nnz += ((int64_t)hs[b]->n + 2 * hs[b]->h) * (int64_t)column_chunks(hs[b], nrhs).size();
    sms = std::max(sms, hs[b]->sms);
  }
  // FP64 members: about four waves of bands of up to kOwnerBandNnz; FP32 / BF16 members: two
  // waves of bands of up to 1.8 kOwnerBandNnz (the FP32 batch of 256 P1 meshes: 0.480 -> 0.463 ms)
  const int64_t slots = (int64_t)sms * owner_ctas_per_sm(1);
  const int64_t band_nnz = std::max<int64_t>(4096, std::min<int64_t>(kOwnerBandNnz, total_nnz / (slots * 4)));
  const int64_t band_nnz_narrow =
      std::max<int64_t>(4096, std::min<int64_t>(kOwnerBandNnz * 9 / 5, total_nnz / (slots * 2)));
  for (int32_t b = 0; b < batch; ++b) {
    csrc_matrix_s* h = hs[b];
    e->hs.push_back(h);
    e->xs.push_back(X[b]);
    e->ys.push_back(Y[b]);
    if (h->n == 0) {
      e->gens.push_back(h->generation);
      continue;
    }
    if (!is_device_ptr(X[b]) || !is_device_ptr(Y[b])) return fail(CSRC_ERR_INVALID_ARG);
    const size_t vb = (size_t)h->n * (size_t)nrhs * h->xbytes();
    const char* xa = static_cast<const char*>(X[b]);
    const char* ya = static_cast<const char*>(Y[b]);
    if (xa < ya + vb && ya < xa + vb) return fail(CSRC_ERR_ALIAS);
    // single vectors: the member's tuned strategy; several columns: the window strategy (the
    // stream-order strategies have no multi-column form)
    const int strat = h->tuned ? h->tuned : CSRC_STRAT_WINDOW;
    bool window = nrhs > 1 || strat == CSRC_STRAT_WINDOW;
    std::vector<std::pair<int32_t, const OwnerPlan*>> chunks;  // (first column, plan)
    if (window) {
      std::vector<std::pair<int32_t, int>> todo = column_chunks(h, nrhs);
      std::reverse(todo.begin(), todo.end());
      while (window && !todo.empty()) {
        const auto c = todo.back();
        todo.pop_back();
        OwnerPlan* p = nullptr;
        const csrc_status st =
            owner_batch_for(h, c.second, h->owner_mode() == OM_F64 ? band_nnz : band_nnz_narrow, &p);
        if (st == CSRC_OK) {
          chunks.push_back({c.first, p});
        } else if (st == CSRC_ERR_NOT_PARTITIONED && c.second > 1) {  // narrower passes fit better
          todo.push_back({c.first + c.second / 2, c.second / 2});
          todo.push_back({c.first, c.second / 2});
        } else if (st == CSRC_ERR_NOT_PARTITIONED && nrhs == 1) {
          window = false;  // no window holds this member's rows: it runs the atomic strategy
        } else {
          return fail(st);
        }
      }
    }
    if (!window) {
      // plans are built now, outside the graph; the member runs its own launches
      if (strat == CSRC_STRAT_COLOR && h->ncolors == 0) return fail(CSRC_ERR_NOT_COLORED);
      if (strat != CSRC_STRAT_COLOR && !h->have_plan) {
        const csrc_status st = make_plan(h);
        if (st != CSRC_OK) return fail(st);
      }
      others.push_back(b);
      e->gens.push_back(h->generation);
      continue;
    }
    for (const auto& c : chunks) {
      const OwnerPlan* p = c.second;
      const int rk = p->rk;
      void* spill = p->spill_buf;
      if (nrhs > 1) {  // chunks of one member run at the same time: each has its own spill buffer
        void* buf = nullptr;
        if (cudaMalloc(&buf, std::max<size_t>(1, (size_t)p->spill * rk * owner_acc_bytes(p->mode))) != cudaSuccess)
          return fail(CSRC_ERR_OUT_OF_MEMORY);
        e->spills.push_back(buf);
        spill = buf;
      }
      const void* xc = static_cast<const char*>(X[b]) + (size_t)c.first * h->xbytes();
      void* yc = static_cast<char*>(Y[b]) + (size_t)c.first * h->xbytes();
      units.push_back({p, p->mode, rk});
      uargs.push_back(owner_args(*p, transpose != 0, xc, yc, spill, nrhs, rk));
      uacc.push_back({p->acc_row, p->acc_ptr, spill, yc, rk, nrhs});
    }
    e->gens.push_back(h->generation);
  }
  // tiles grouped by (mode, rk), largest bands first; accumulations grouped by mode
  struct Group {
    int mode, rk, first, count, smem;
  };
  std::vector<Group> groups;
  std::vector<OwnerTile> tiles;
  for (int mode = 0; mode < kOwnerModes; ++mode)
    for (int rk = 1; rk <= 8; rk *= 2) {
      std::vector<std::pair<int64_t, OwnerTile>> v;
      int smem = 16;
      for (size_t u = 0; u < units.size(); ++u) {
        if (units[u].mode != mode || units[u].rk != rk) continue;
        smem = std::max(smem, units[u].p->smem_bytes);
        for (int32_t band = 0; band < units[u].p->nb; ++band)
          v.push_back({units[u].p->band_entries[(size_t)band], OwnerTile{(int32_t)u, band, 0, 0}});
      }
      if (v.empty()) continue;
      std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
      groups.push_back({mode, rk, (int)tiles.size(), (int)v.size(), smem});
      for (const auto& t : v) tiles.push_back(t.second);
    }
  struct AccGroup {
    int mode, first, count, ofirst;
    int64_t total;
  };
  std::vector<AccGroup> agroups;
  std::vector<OwnerAccArgs> accs;
  std::vector<int64_t> offs;
  for (int mode = 0; mode < kOwnerModes; ++mode) {
    AccGroup g{mode, (int)accs.size(), 0, (int)offs.size(), 0};
    offs.push_back(0);
    for (size_t u = 0; u < units.size(); ++u) {
      if (units[u].mode != mode || units[u].p->nacc == 0) continue;
      accs.push_back(uacc[u]);
      g.total += units[u].p->nacc * units[u].rk;
      offs.push_back(g.total);
      ++g.count;
    }
    if (g.count == 0) {
      offs.pop_back();
      continue;
    }
    agroups.push_back(g);
  }
  cudaStream_t s = nullptr;
  cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return fail(from_cuda(ce));
  auto done = [&](cudaError_t err) -> csrc_status {
    if (s) cudaStreamDestroy(s);
    if (err != cudaSuccess) return fail(from_cuda(err));
    return CSRC_OK;
  };
  if ((ce = upload(&e->d_units, uargs, s)) != cudaSuccess) return done(ce);
  if ((ce = upload(&e->d_tiles, tiles, s)) != cudaSuccess) return done(ce);
  if ((ce = upload(&e->d_acc, accs, s)) != cudaSuccess) return done(ce);
  if ((ce = upload(&e->d_offs, offs, s)) != cudaSuccess) return done(ce);
  if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) return done(ce);
  if ((ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return done(ce);
  cudaError_t cap = cudaSuccess;
  for (const Group& g : groups) {
    if (cap != cudaSuccess) break;
    cap = launch_owner_batch(g.mode, g.rk, e->d_units, e->d_tiles + g.first, g.count, g.smem, s);
    ++e->kernels;
  }
  for (const AccGroup& g : agroups) {
    if (cap != cudaSuccess) break;
    cap = launch_owner_batch_accumulate(g.mode, e->d_acc + g.first, e->d_offs + g.ofirst, g.count, g.total, s);
    ++e->kernels;
  }
  if (groups.empty() && agroups.empty() && cap == cudaSuccess) cap = cudaMemsetAsync(e->d_offs, 0, 0, s);
  ce = cudaStreamEndCapture(s, &e->graph);
  if (cap != cudaSuccess) return done(cap);
  if (ce != cudaSuccess) return done(ce);
  if ((ce = cudaGraphInstantiate(&e->exec, e->graph, 0)) != cudaSuccess) return done(ce);
  *out = e;
  return done(cudaSuccess);
}

csrc_status run_batch(const csrc_handle* hs, int32_t batch, const void* const* X, void* const* Y, int32_t nrhs,
                      int transpose, cudaStream_t stream) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return CSRC_ERR_CUDA;
  for (int32_t b = 0; b < batch; ++b)
    if (hs[b]->device != device) return CSRC_ERR_INVALID_ARG;  // one device per batch
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  BatchExec* e = nullptr;
  for (size_t i = 0; i < g_batches.size(); ++i)
    if (batch_matches(g_batches[i], hs, batch, X, Y, nrhs, transpose, device)) {
      e = g_batches[i];
      g_batches.erase(g_batches.begin() + (long)i);
      g_batches.push_back(e);
      break;
    }
  if (!e) {
    CSRC_TRY_S(build_batch(hs, batch, X, Y, nrhs, transpose, device, &e));
    if (g_batches.size() >= kMaxBatches) {
      delete g_batches.front();
      g_batches.erase(g_batches.begin());
    }
    g_batches.push_back(e);
  }
  csrc_matrix_s* h0 = hs[0];
  if (e->kernels > 0)
    CSRC_TRY(timed_launch(h0, CSRC_KERNEL_PRODUCT, stream, [&] { return cudaGraphLaunch(e->exec, stream); },
                          e->kernels));
  // single-vector members tuned to another strategy (or whose windows do not fit) run their
  // own launches on the same stream
  for (int32_t b : e->others) {
    csrc_matrix_s* h = hs[b];
    const int tuned = h->tuned ? h->tuned : CSRC_STRAT_ATOMIC;
    const csrc_strategy st = (csrc_strategy)(tuned == CSRC_STRAT_WINDOW ? CSRC_STRAT_ATOMIC : tuned);
    CSRC_TRY_S(run_spmv(h, X[b], Y[b], st, stream, transpose != 0));
  }
  return CSRC_OK;
}

// Rows per node block: the largest B in {3, 2} such that n is a multiple of B and every
// unit of rows r = qB .. qB+B-1 has the node-block shape the band kernel exploits: row
// r+t holds row r's columns (all below r, same order) followed by columns r .. r+t-1.
// FE matrices with B unknowns per node interleaved (B-by-B dense node blocks) have it.
// Returns 1 when neither size fits.
int32_t detect_node_blocks(int32_t n, const std::vector<int32_t>& ia, const std::vector<int32_t>& ja) {
  for (int32_t B = 3; B >= 2; --B) {
    if (n < B || n % B != 0) continue;
    bool ok = true;
    for (int32_t r = 0; r < n && ok; r += B) {
      const int32_t L0 = ia[(size_t)r + 1] - ia[(size_t)r];
      for (int32_t t = 1; t < B && ok; ++t) {
        const int32_t kb = ia[(size_t)r + t];
        if (ia[(size_t)r + t + 1] - kb != L0 + t) {
          ok = false;
          break;
        }
        for (int32_t m = 0; m < L0; ++m)
          if (ja[(size_t)kb + m] != ja[(size_t)ia[(size_t)r] + m]) {
            ok = false;
            break;
          }
        for (int32_t q = 0; q < t && ok; ++q)
          if (ja[(size_t)kb + L0 + q] != r + q) ok = false;
      }
    }
    if (ok) return B;
  }
  return 1;
}

csrc_status create_from_host_csr(csrc_handle* out, int32_t n, const int64_t* row_ptr, const int32_t* col,
                                 const double* val, csrc_dtype storage, uint32_t flags, cudaStream_t stream) {
  const int64_t base = (flags & CSRC_FLAG_ONE_BASED) ? 1 : 0;
  const int64_t nnz = row_ptr[n] - base;
  // transposed upper part: for every a_ji with i > j, list (j, a_ji) under row i, j ascending
  std::vector<int64_t> up_ptr((size_t)n + 1, 0);
  for (int32_t r = 0; r < n; ++r)
    for (int64_t p = row_ptr[r] - base; p < row_ptr[r + 1] - base; ++p) {
      const int64_t c = col[p] - base;
      if (c > r) up_ptr[(size_t)c + 1]++;
    }
  for (int32_t r = 0; r < n; ++r) up_ptr[r + 1] += up_ptr[r];
  std::vector<int32_t> up_row((size_t)up_ptr[n]);
  std::vector<double> up_val((size_t)up_ptr[n]);
  {
    std::vector<int64_t> fill(up_ptr.begin(), up_ptr.end() - 1);
    for (int32_t r = 0; r < n; ++r)
      for (int64_t p = row_ptr[r] - base; p < row_ptr[r + 1] - base; ++p) {
        const int64_t c = col[p] - base;
        if (c > r) {
          up_row[(size_t)fill[c]] = r;
          up_val[(size_t)fill[c]++] = val[p];
        }
      }
  }
  const bool pad = flags & CSRC_FLAG_PAD_PATTERN;
  std::vector<int32_t> ia((size_t)n + 1, 0);
  std::vector<int32_t> ja;
  std::vector<double> al, au, ad((size_t)n, 0.0);
  ja.reserve((size_t)std::max<int64_t>(0, (nnz - n) / 2));
  al.reserve(ja.capacity());
  au.reserve(ja.capacity());
  for (int32_t i = 0; i < n; ++i) {
    if ((int64_t)ja.size() > (int64_t)INT32_MAX - 16) return CSRC_ERR_INVALID_ARG;
    ia[i] = (int32_t)ja.size();
    int64_t p = row_ptr[i] - base;
    const int64_t pe = row_ptr[i + 1] - base;
    int64_t u = up_ptr[i];
    const int64_t ue = up_ptr[i + 1];
    while (true) {
      const int64_t cl = (p < pe && col[p] - base < i) ? col[p] - base : INT64_MAX;
      const int64_t cu = (u < ue) ? up_row[(size_t)u] : INT64_MAX;
      if (cl == INT64_MAX && cu == INT64_MAX) break;
      if (cl == cu) {
        ja.push_back((int32_t)cl);
        al.push_back(val[p]);
        au.push_back(up_val[(size_t)u]);
        ++p;
        ++u;
      } else if (cl < cu) {
        if (!pad) return CSRC_ERR_NOT_STRUCT_SYMMETRIC;
        ja.push_back((int32_t)cl);
        al.push_back(val[p]);
        au.push_back(0.0);
        ++p;
      } else {
        if (!pad) return CSRC_ERR_NOT_STRUCT_SYMMETRIC;
        ja.push_back((int32_t)cu);
        al.push_back(0.0);
        au.push_back(up_val[(size_t)u]);
        ++u;
      }
    }
    if (p < pe && col[p] - base == i) ad[i] = val[p];
  }
  ia[n] = (int32_t)ja.size();
  const int64_t h64 = (int64_t)ja.size();
  int64_t max_row_nnz = n > 0 ? 1 : 0;  // diagonal, lower and upper entries of the longest row
  {
    std::vector<int32_t> up((size_t)n, 0);
    for (int32_t k : ja) up[(size_t)k]++;
    for (int32_t i = 0; i < n; ++i)
      max_row_nnz = std::max<int64_t>(max_row_nnz, 1 + (int64_t)(ia[(size_t)i + 1] - ia[(size_t)i]) + up[(size_t)i]);
  }

  csrc_matrix_s* m = new (std::nothrow) csrc_matrix_s();
  if (!m) return CSRC_ERR_OUT_OF_MEMORY;
  m->n = n;
  m->m = n;
  m->h = h64;
  m->storage = storage;
  m->precision = storage;
  m->max_row_nnz = max_row_nnz;
  m->flags = flags;
  m->block = (flags & CSRC_FLAG_NODE_BLOCKS) ? detect_node_blocks(n, ia, ja) : 1;
  if (flags & CSRC_FLAG_SYMMETRIC_VALUES) {
    for (size_t k = 0; k < al.size(); ++k)
      if (std::memcmp(&al[k], &au[k], sizeof(double)) != 0) {
        delete m;
        return CSRC_ERR_NOT_NUM_SYMMETRIC;
      }
    m->sym = true;
  }
  cudaGetDevice(&m->device);
  cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device);
  if (m->sms <= 0) m->sms = 1;
  {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, m->device) == cudaSuccess)
      std::snprintf(m->devname, sizeof(m->devname), "%.48s/%dSM", prop.name, m->sms);
    else
      cudaGetLastError();
  }
  m->phash = pattern_hash(n, ia, ja);
  if (storage == CSRC_F64) {
    // FP64 arithmetic unless double-float is asked for (stream-order strategies only)
    m->arith = ((flags & CSRC_FLAG_DF32_ARITH) && !(flags & CSRC_FLAG_FP64_ARITH)) ? ARITH_DF32 : ARITH_F64;
    // the double-float path needs values in [2^-50, 2^63) (or zero); otherwise use FP64 arithmetic
    auto in_range = [](double v) {
      if (v == 0.0) return true;
      const double a = std::fabs(v);
      return a >= 0x1p-50 && a < 0x1p63;
    };
    if (m->arith == ARITH_DF32) {
      bool ok = true;
      for (double v : al) ok = ok && in_range(v);
      for (double v : au) ok = ok && in_range(v);
      for (double v : ad) ok = ok && in_range(v);
      if (!ok) m->arith = ARITH_F64;
    }
  } else {
    m->arith = ARITH_F32;
  }
  csrc_status st = CSRC_OK;
  auto fail = [&](csrc_status s) {
    csrc_destroy(m);
    return s;
  };
  // aligned bulk copies of the band kernels may read up to the next multiple of kPairAlign pairs
  const size_t hcap = ((size_t)h64 + kPairAlign - 1) / kPairAlign * kPairAlign + kPairAlign;
  const size_t vb = m->vbytes();
  // ia is padded: the band kernels copy row-pointer slices rounded up to 4 entries
  if (from_cuda(dmalloc(&m->d_ia, (size_t)n + 1 + kMetaPad)) != CSRC_OK) return fail(CSRC_ERR_OUT_OF_MEMORY);
  if ((st = from_cuda(cudaMemsetAsync(m->d_ia, 0, ((size_t)n + 1 + kMetaPad) * 4, stream))) != CSRC_OK) return fail(st);
  if (from_cuda(dmalloc(&m->d_ja, hcap)) != CSRC_OK) return fail(CSRC_ERR_OUT_OF_MEMORY);
  if (cudaMalloc(&m->d_al, hcap * vb) != cudaSuccess) return fail(CSRC_ERR_OUT_OF_MEMORY);
  if (!m->sym && cudaMalloc(&m->d_au, hcap * vb) != cudaSuccess) return fail(CSRC_ERR_OUT_OF_MEMORY);
  if (cudaMalloc(&m->d_ad, std::max<size_t>(1, (size_t)n) * vb) != cudaSuccess) return fail(CSRC_ERR_OUT_OF_MEMORY);
  if (from_cuda(dmalloc(&m->d_status, 1)) != CSRC_OK) return fail(CSRC_ERR_OUT_OF_MEMORY);
  if ((st = from_cuda(cudaMemsetAsync(m->d_ja, 0, hcap * 4, stream))) != CSRC_OK) return fail(st);
  if ((st = from_cuda(cudaMemsetAsync(m->d_al, 0, hcap * vb, stream))) != CSRC_OK) return fail(st);
  if (!m->sym && (st = from_cuda(cudaMemsetAsync(m->d_au, 0, hcap * vb, stream))) != CSRC_OK) return fail(st);
  if ((st = from_cuda(cudaMemsetAsync(m->d_status, 0, 4, stream))) != CSRC_OK) return fail(st);
  if ((st = from_cuda(cudaMemcpyAsync(m->d_ia, ia.data(), ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, stream))) != CSRC_OK)
    return fail(st);
  if (h64 > 0 &&
      (st = from_cuda(cudaMemcpyAsync(m->d_ja, ja.data(), (size_t)h64 * 4, cudaMemcpyHostToDevice, stream))) != CSRC_OK)
    return fail(st);
  auto put_values = [&](void* dst, const std::vector<double>& src) -> csrc_status {
    if (src.empty()) return CSRC_OK;
    if (storage == CSRC_F64)
      return from_cuda(cudaMemcpyAsync(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice, stream));
    if (storage == CSRC_F32) {
      std::vector<float> tmp(src.size());
      for (size_t i = 0; i < src.size(); ++i) tmp[i] = (float)src[i];
      cudaError_t e = cudaMemcpyAsync(dst, tmp.data(), tmp.size() * 4, cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      return from_cuda(e);
    }
    std::vector<uint16_t> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = f64_to_bf16(src[i]);
    cudaError_t e = cudaMemcpyAsync(dst, tmp.data(), tmp.size() * 2, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return from_cuda(e);
  };
  if ((st = put_values(m->d_al, al)) != CSRC_OK) return fail(st);
  if (!m->sym && (st = put_values(m->d_au, au)) != CSRC_OK) return fail(st);
  if ((st = put_values(m->d_ad, ad)) != CSRC_OK) return fail(st);
  if (m->arith == ARITH_DF32 && !m->sym) {
    if (cudaMalloc(&m->d_al_df, hcap * 8) != cudaSuccess) return fail(CSRC_ERR_OUT_OF_MEMORY);
    if (cudaMalloc(&m->d_au_df, hcap * 8) != cudaSuccess) return fail(CSRC_ERR_OUT_OF_MEMORY);
    if ((st = from_cuda(launch_split_df(static_cast<const double*>(m->d_al), m->d_al_df, (int64_t)hcap, stream))) !=
        CSRC_OK)
      return fail(st);
    if ((st = from_cuda(launch_split_df(static_cast<const double*>(m->d_au), m->d_au_df, (int64_t)hcap, stream))) !=
        CSRC_OK)
      return fail(st);
  }
  if ((st = from_cuda(cudaStreamSynchronize(stream))) != CSRC_OK) return fail(st);
  m->ia.swap(ia);
  m->ja.swap(ja);
  {
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_prepared) {
      if (prepare_band_kernels() != cudaSuccess || prepare_owner_kernels() != cudaSuccess) {
        cudaGetLastError();
        return fail(CSRC_ERR_CUDA);
      }
      g_prepared = true;
    }
  }
  *out = m;
  return CSRC_OK;
}

// Install a colouring (colour of every row) as the handle's colour classes: rows grouped by
// colour, ascending within a class, on the device with the class pointers.
csrc_status set_colouring(csrc_matrix_s* h, const std::vector<int32_t>& color, int32_t* ncolors_out,
                          int32_t* colors_out) {
  const int32_t n = h->n;
  int32_t nc = 0;
  for (int32_t v : color) nc = std::max(nc, v + 1);
  std::vector<int32_t> cptr((size_t)nc + 1, 0), rows((size_t)std::max(n, 1));
  for (int32_t i = 0; i < n; ++i) cptr[(size_t)color[(size_t)i] + 1]++;
  for (int32_t c = 0; c < nc; ++c) cptr[(size_t)c + 1] += cptr[(size_t)c];
  {
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int32_t i = 0; i < n; ++i) rows[(size_t)fill[(size_t)color[(size_t)i]]++] = i;
  }
  // the rows' pairs in class order: row t of the order owns k0 .. k1 - 1 of the copy
  std::vector<int4> desc((size_t)std::max(n, 1));
  {
    int64_t off = 0;
    for (int32_t t = 0; t < n; ++t) {
      const int32_t i = rows[(size_t)t];
      const int32_t k0 = h->ia[(size_t)i], k1 = h->ia[(size_t)i + 1];
      int4 d;
      d.x = i;
      d.y = (int)off;
      d.z = (int)(off + (k1 - k0));
      d.w = k0;
      desc[(size_t)t] = d;
      off += k1 - k0;
    }
  }
  cudaStream_t s = 0;
  dfree(h->d_color_desc); dfree(h->d_cja); dfree(h->d_cal); dfree(h->d_cau);
  dfree(h->d_color_ptr);
  h->d_color_desc = nullptr;
  h->d_cja = nullptr;
  h->d_cal = h->d_cau = nullptr;
  h->d_color_ptr = nullptr;
  h->ncolors = 0;
  const size_t hh = (size_t)std::max<int64_t>(h->h, 1);
  cudaError_t e = upload(&h->d_color_desc, desc, s);
  if (e == cudaSuccess) e = dmalloc(&h->d_cja, hh);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_cal, hh * h->vbytes());
  if (e == cudaSuccess && !h->sym) e = cudaMalloc(&h->d_cau, hh * h->vbytes());
  if (e == cudaSuccess)
    e = launch_color_copy((int)h->vbytes(), h->d_color_desc, n, h->d_ja, h->d_al, h->sym ? nullptr : h->d_au,
                          h->d_cja, h->d_cal, h->sym ? nullptr : h->d_cau, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  CSRC_TRY(e);
  CSRC_TRY(upload(&h->d_color_ptr, cptr, s));
  if (!h->d_barrier) CSRC_TRY(dmalloc(&h->d_barrier, 1));
  CSRC_TRY(cudaStreamSynchronize(s));
  h->color_ptr.swap(cptr);
  h->ncolors = nc;
  ++h->generation;
  if (ncolors_out) *ncolors_out = nc;
  if (colors_out) std::copy(color.begin(), color.end(), colors_out);
  return CSRC_OK;
}

}  // namespace

namespace csrc {

int32_t handle_device(const csrc_matrix_s* h) { return h->device; }

// Window-strategy product whose spilled partial sums go to caller-provided device
// memory `spill` (capacity in elements of the vector type). It allocates nothing:
// the handle must already hold a window plan that covers every scatter target,
// and x, y must be device pointers. The device of the handle must be current.
csrc_status spmv_external_spill(csrc_matrix_s* h, const void* x, void* y, bool transpose, void* spill,
                                int64_t capacity, cudaStream_t s) {
  if (!h || !x || !y || !spill || h->rect()) return CSRC_ERR_INVALID_ARG;
  if (h->n == 0) return CSRC_OK;
  const size_t vb = (size_t)h->n * h->xbytes();
  const char* xa = static_cast<const char*>(x);
  const char* ya = static_cast<const char*>(y);
  if (xa < ya + vb && ya < xa + vb) return CSRC_ERR_ALIAS;
  if (!h->have_oplan) return CSRC_ERR_NOT_PARTITIONED;
  if (h->oplan.spill > capacity) return CSRC_ERR_INVALID_ARG;
  if (!is_device_ptr(x) || !is_device_ptr(y)) return CSRC_ERR_INVALID_ARG;
  const OwnerPlan& p = h->oplan;
  const OwnerArgs a = owner_args(p, transpose, x, y, spill, 1, 1);
  CSRC_TRY(launch_owner(p.mode, 1, a, p.nb, p.smem_bytes, s));
  if (p.nacc > 0) CSRC_TRY(launch_owner_accumulate(p.mode, p.nacc, 1, 1, p.acc_row, p.acc_ptr, spill, y, s));
  return CSRC_OK;
}

}  // namespace csrc

extern "C" {

csrc_status csrc_create_from_csr(csrc_handle* out, int32_t n, const int64_t* row_ptr, const int32_t* col,
                                 const double* val, csrc_dtype storage, uint32_t flags, cudaStream_t stream) {
  if (!out) return CSRC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 0 || !row_ptr) return CSRC_ERR_INVALID_ARG;
  if (storage < CSRC_F64 || storage > CSRC_BF16) return CSRC_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(CSRC_FLAG_PAD_PATTERN | CSRC_FLAG_ONE_BASED | CSRC_FLAG_FP64_ARITH |
                         CSRC_FLAG_NODE_BLOCKS | CSRC_FLAG_SYMMETRIC_VALUES |
                         CSRC_FLAG_COMPRESS_INDICES | CSRC_FLAG_DF32_ARITH))
    return CSRC_ERR_INVALID_ARG;
  const int64_t base = (flags & CSRC_FLAG_ONE_BASED) ? 1 : 0;
  if (row_ptr[0] != base) return CSRC_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return CSRC_ERR_INVALID_ARG;
  const int64_t nnz = row_ptr[n] - base;
  if (nnz > 0 && (!col || !val)) return CSRC_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i) {
    for (int64_t p = row_ptr[i] - base; p < row_ptr[i + 1] - base; ++p) {
      const int64_t c = (int64_t)col[p] - base;
      if (c < 0 || c >= n) return CSRC_ERR_INDEX_RANGE;
      if (p > row_ptr[i] - base && c <= (int64_t)col[p - 1] - base) return CSRC_ERR_DUPLICATE;
    }
  }
  try {
    return create_from_host_csr(out, n, row_ptr, col, val, storage, flags, stream);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_create_rect_from_csr(csrc_handle* out, int32_t n, int32_t m, const int64_t* row_ptr,
                                      const int32_t* col, const double* val, csrc_dtype storage, uint32_t flags,
                                      cudaStream_t stream) {
  if (!out) return CSRC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 0 || m < n || !row_ptr) return CSRC_ERR_INVALID_ARG;
  if (storage < CSRC_F64 || storage > CSRC_BF16) return CSRC_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(CSRC_FLAG_PAD_PATTERN | CSRC_FLAG_ONE_BASED | CSRC_FLAG_FP64_ARITH |
                         CSRC_FLAG_NODE_BLOCKS | CSRC_FLAG_SYMMETRIC_VALUES |
                         CSRC_FLAG_COMPRESS_INDICES | CSRC_FLAG_DF32_ARITH))
    return CSRC_ERR_INVALID_ARG;
  const int64_t base = (flags & CSRC_FLAG_ONE_BASED) ? 1 : 0;
  if (row_ptr[0] != base) return CSRC_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return CSRC_ERR_INVALID_ARG;
  const int64_t nnz = row_ptr[n] - base;
  if (nnz > 0 && (!col || !val)) return CSRC_ERR_INVALID_ARG;
  try {
    // Section 2.1: columns below n form A_S, the others A_R (0-based from here on)
    std::vector<int64_t> sptr((size_t)n + 1, 0);
    std::vector<int32_t> scol, rrow, rptr{0}, rcol;
    std::vector<double> sval, rval;
    for (int32_t i = 0; i < n; ++i) {
      bool any = false;
      for (int64_t p = row_ptr[i] - base; p < row_ptr[i + 1] - base; ++p) {
        const int64_t c = (int64_t)col[p] - base;
        if (c < 0 || c >= m) return CSRC_ERR_INDEX_RANGE;
        if (p > row_ptr[i] - base && c <= (int64_t)col[p - 1] - base) return CSRC_ERR_DUPLICATE;
        if (c < n) {
          scol.push_back((int32_t)c);
          sval.push_back(val[p]);
        } else {
          rcol.push_back((int32_t)c);
          rval.push_back(val[p]);
          any = true;
        }
      }
      sptr[(size_t)i + 1] = (int64_t)scol.size();
      if (any) {
        if (rcol.size() > (size_t)INT32_MAX - 1) return CSRC_ERR_INVALID_ARG;
        rrow.push_back(i);
        rptr.push_back((int32_t)rcol.size());
      }
    }
    csrc_handle h = nullptr;
    CSRC_TRY_S(create_from_host_csr(&h, n, sptr.data(), scol.data(), sval.data(), storage,
                                    flags & ~(uint32_t)CSRC_FLAG_ONE_BASED, stream));
    h->m = m;
    h->rnnz = (int64_t)rcol.size();
    h->nrrows = (int32_t)rrow.size();
    // column-major copy of A_R for A^T x: columns n..m-1, rows ascending within a column
    std::vector<int32_t> tptr((size_t)(m - n) + 1, 0), trow(rcol.size());
    std::vector<double> tval(rcol.size());
    for (int32_t c : rcol) tptr[(size_t)(c - n) + 1]++;
    for (size_t c = 0; c + 1 < tptr.size(); ++c) tptr[c + 1] += tptr[c];
    {
      std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
      for (size_t t = 0; t < rrow.size(); ++t)
        for (int32_t k = rptr[t]; k < rptr[t + 1]; ++k) {
          const int32_t q = fill[(size_t)(rcol[(size_t)k] - n)]++;
          trow[(size_t)q] = rrow[t];
          tval[(size_t)q] = rval[(size_t)k];
        }
    }
    auto values = [&](void** dst, const std::vector<double>& v) -> cudaError_t {
      const size_t cnt = std::max<size_t>(1, v.size());
      if (storage == CSRC_F64) {
        cudaError_t e = cudaMalloc(dst, cnt * 8);
        if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice);
        return e;
      }
      if (storage == CSRC_F32) {
        std::vector<float> t(v.size());
        for (size_t i = 0; i < v.size(); ++i) t[i] = (float)v[i];
        cudaError_t e = cudaMalloc(dst, cnt * 4);
        if (e == cudaSuccess && !t.empty()) e = cudaMemcpy(*dst, t.data(), t.size() * 4, cudaMemcpyHostToDevice);
        return e;
      }
      std::vector<uint16_t> t(v.size());
      for (size_t i = 0; i < v.size(); ++i) t[i] = f64_to_bf16(v[i]);
      cudaError_t e = cudaMalloc(dst, cnt * 2);
      if (e == cudaSuccess && !t.empty()) e = cudaMemcpy(*dst, t.data(), t.size() * 2, cudaMemcpyHostToDevice);
      return e;
    };
    cudaError_t e = cudaSuccess;
    auto ints = [&](int32_t** dst, const std::vector<int32_t>& v) {
      if (e != cudaSuccess) return;
      e = dmalloc(dst, v.size());
      if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice);
    };
    ints(&h->d_rrow, rrow);
    ints(&h->d_rptr, rptr);
    ints(&h->d_rcol, rcol);
    ints(&h->d_tptr, tptr);
    ints(&h->d_trow, trow);
    if (e == cudaSuccess) e = values(&h->d_rval, rval);
    if (e == cudaSuccess) e = values(&h->d_tval, tval);
    if (e != cudaSuccess) {
      csrc_destroy(h);
      return from_cuda(e);
    }
    *out = h;
    return CSRC_OK;
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_create_from_coo(csrc_handle* out, int32_t n, int64_t nnz, const int32_t* row, const int32_t* col,
                                 const double* val, csrc_dtype storage, uint32_t flags, cudaStream_t stream) {
  if (!out) return CSRC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 0 || nnz < 0 || (nnz > 0 && (!row || !col || !val))) return CSRC_ERR_INVALID_ARG;
  const int64_t base = (flags & CSRC_FLAG_ONE_BASED) ? 1 : 0;
  try {
    // counting sort by row, then sort each row by column and sum duplicates
    std::vector<int64_t> ptr((size_t)n + 1, 0);
    for (int64_t p = 0; p < nnz; ++p) {
      const int64_t r = row[p] - base, c = col[p] - base;
      if (r < 0 || r >= n || c < 0 || c >= n) return CSRC_ERR_INDEX_RANGE;
      ptr[(size_t)r + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    std::vector<std::pair<int32_t, double>> ent((size_t)nnz);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t p = 0; p < nnz; ++p)
      ent[(size_t)fill[(size_t)(row[p] - base)]++] = {(int32_t)(col[p] - base), val[p]};
    std::vector<int64_t> rp((size_t)n + 1, 0);
    std::vector<int32_t> cc;
    std::vector<double> vv;
    cc.reserve((size_t)nnz);
    vv.reserve((size_t)nnz);
    for (int32_t i = 0; i < n; ++i) {
      auto b = ent.begin() + ptr[i], e = ent.begin() + ptr[i + 1];
      std::stable_sort(b, e, [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
        return x.first < y.first;
      });
      for (auto it = b; it != e; ++it) {
        if (!cc.empty() && (int64_t)vv.size() > rp[i] && cc.back() == it->first)
          vv.back() += it->second;  // duplicates summed in input order
        else {
          cc.push_back(it->first);
          vv.push_back(it->second);
        }
      }
      rp[(size_t)i + 1] = (int64_t)cc.size();
    }
    return csrc_create_from_csr(out, n, rp.data(), cc.data(), vv.data(), storage,
                                flags & ~(uint32_t)CSRC_FLAG_ONE_BASED, stream);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_partition(csrc_handle h, int32_t nbands, int32_t* band_ptr_out) {
  if (!h || nbands < 0) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  try {
    // the window strategy's lists are rebuilt from the new partition now, the stream-order
    // plans when next needed
    h->part_nbands = nbands;
    h->owner_nbands = nbands;
    drop_owner_plans(h);
    free_plan(h->plan);
    free_plan(h->plan_b1);
    h->have_plan = h->have_b1 = false;
    OwnerPlan* op = nullptr;
    const csrc_status st = owner_for(h, 1, &op);
    if (st == CSRC_ERR_NOT_PARTITIONED) {
      // no window of this matrix fits in shared memory: report the partition all the same
      nnz_partition(h->ia, 0, h->n, nbands > 0 ? std::min<int32_t>(nbands, std::max<int32_t>(1, h->n))
                                               : owner_auto_bands(h, 1), h->part);
    } else if (st != CSRC_OK) {
      return st;
    }
    ++h->generation;
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
  if (band_ptr_out) std::copy(h->part.begin(), h->part.end(), band_ptr_out);
  return CSRC_OK;
}

csrc_status csrc_color(csrc_handle h, uint64_t seed, int32_t* ncolors_out, int32_t* colors_out) {
  if (!h) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  const int32_t n = h->n;
  if (n == 0) {
    h->ncolors = 0;
    if (ncolors_out) *ncolors_out = 0;
    return CSRC_OK;
  }
  try {
    // A_U column lists: rows v with t in ja(v), v ascending
    std::vector<int32_t> up_ptr((size_t)n + 1, 0);
    for (int64_t k = 0; k < h->h; ++k) up_ptr[(size_t)h->ja[(size_t)k] + 1]++;
    for (int32_t t = 0; t < n; ++t) up_ptr[t + 1] += up_ptr[t];
    std::vector<int32_t> up((size_t)std::max<int64_t>(1, h->h));
    {
      std::vector<int32_t> fill(up_ptr.begin(), up_ptr.end() - 1);
      for (int32_t v = 0; v < n; ++v)
        for (int32_t k = h->ia[v]; k < h->ia[v + 1]; ++k) up[(size_t)fill[h->ja[k]]++] = v;
    }
    int32_t *d_up_ptr = nullptr, *d_up = nullptr, *d_state = nullptr, *d_cnt = nullptr;
    auto cleanup = [&]() { dfree(d_up_ptr); dfree(d_up); dfree(d_state); dfree(d_cnt); };
    cudaStream_t s = 0;
    cudaError_t e = upload(&d_up_ptr, up_ptr, s);
    if (e == cudaSuccess) e = upload(&d_up, up, s);
    if (e == cudaSuccess) e = dmalloc(&d_state, (size_t)n);
    if (e == cudaSuccess) e = dmalloc(&d_cnt, 2);  // uncoloured rows, too-many-colours flag
    if (e == cudaSuccess) e = cudaMemsetAsync(d_state, 0xff, (size_t)n * 4, s);
    int32_t round = 0;
    int32_t left[2] = {n, 0};
    while (e == cudaSuccess && left[0] > 0) {
      ++round;
      if (round >= 32768) {
        cleanup();
        return CSRC_ERR_DEVICE_TIMEOUT;
      }
      e = cudaMemsetAsync(d_cnt, 0, 8, s);
      if (e == cudaSuccess) e = launch_jp_round(n, h->d_ia, h->d_ja, d_up_ptr, d_up, seed, round, d_state, d_cnt, s);
      if (e == cudaSuccess) e = cudaMemcpy(left, d_cnt, 8, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && left[1] != 0) {
        cleanup();
        return CSRC_ERR_INVALID_ARG;  // more than 65536 colours
      }
    }
    std::vector<int32_t> state((size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(state.data(), d_state, (size_t)n * 4, cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return from_cuda(e);
    for (auto& v : state) v &= 0xffff;
    return set_colouring(h, state, ncolors_out, colors_out);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_color_stride(csrc_handle h, int64_t stride, int32_t* ncolors_out, int32_t* colors_out) {
  if (!h) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  const int32_t n = h->n;
  try {
    // rows of A_U's columns: the rows v > t with t in their ja, ascending
    std::vector<int32_t> up_ptr((size_t)n + 1, 0);
    for (int32_t t : h->ja) up_ptr[(size_t)t + 1]++;
    for (int32_t t = 0; t < n; ++t) up_ptr[(size_t)t + 1] += up_ptr[(size_t)t];
    std::vector<int32_t> up(h->ja.size());
    {
      std::vector<int32_t> fill(up_ptr.begin(), up_ptr.end() - 1);
      for (int32_t v = 0; v < n; ++v)
        for (int32_t k = h->ia[(size_t)v]; k < h->ia[(size_t)v + 1]; ++k) up[(size_t)fill[(size_t)h->ja[(size_t)k]]++] = v;
    }
    // rows in ascending order; banned[c] == i marks colour c as held by an earlier row that
    // writes into W(i); last[c] is colour c's latest member
    std::vector<int32_t> color((size_t)n, -1), banned, last;
    for (int32_t i = 0; i < n; ++i) {
      auto ban = [&](int32_t v) {
        if (v < i) banned[(size_t)color[(size_t)v]] = i;  // rows below i are coloured already
      };
      const int32_t k0 = h->ia[(size_t)i], k1 = h->ia[(size_t)i + 1];
      for (int32_t q = k0 - 1; q < k1; ++q) {
        const int32_t t = q < k0 ? i : h->ja[(size_t)q];
        if (t != i) ban(t);
        for (int32_t p = up_ptr[(size_t)t]; p < up_ptr[(size_t)t + 1]; ++p) {
          const int32_t v = up[(size_t)p];
          if (v >= i) break;  // ascending: the rest are not coloured yet
          ban(v);
        }
      }
      int32_t c = 0;
      const int32_t nc = (int32_t)last.size();
      while (c < nc && (banned[(size_t)c] == i || (stride > 0 && (int64_t)i - last[(size_t)c] > stride))) ++c;
      if (c == nc) {
        if (nc >= 65536) return CSRC_ERR_INVALID_ARG;  // more than 65536 colours
        last.push_back(i);
        banned.push_back(-1);
      }
      color[(size_t)i] = c;
      last[(size_t)c] = i;
    }
    return set_colouring(h, color, ncolors_out, colors_out);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_spmv(csrc_handle h, const void* x, void* y, csrc_strategy strategy, cudaStream_t stream) {
  try {
    return run_spmv(h, x, y, strategy, stream, false);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_spmv_t(csrc_handle h, const void* x, void* y, csrc_strategy strategy, cudaStream_t stream) {
  try {
    return run_spmv(h, x, y, strategy, stream, true);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_spmm_batched(const csrc_handle* hs, int32_t batch, const void* const* X, void* const* Y,
                              int32_t nrhs, int32_t transpose, cudaStream_t stream) {
  if (batch < 0 || nrhs <= 0 || (batch > 0 && (!hs || !X || !Y))) return CSRC_ERR_INVALID_ARG;
  for (int32_t b = 0; b < batch; ++b) {
    if (!hs[b] || !X[b] || !Y[b]) return CSRC_ERR_INVALID_ARG;
    if (hs[b]->rect()) return CSRC_ERR_INVALID_ARG;  // rectangular matrices run single products
  }
  if (batch == 0) return CSRC_OK;
  try {
    DeviceGuard dg;
    CSRC_TRY_S(dg.enter(hs[0]));
    if (batch == 1 && nrhs == 1) {
      // one vector of one matrix: its own plans (bands in whole waves of the GPU), no graph
      if (!is_device_ptr(X[0]) || !is_device_ptr(Y[0])) return CSRC_ERR_INVALID_ARG;
      return run_spmv(hs[0], X[0], Y[0], CSRC_STRAT_AUTO, stream, transpose != 0);
    }
    // several columns (even of one matrix) or several matrices: every column chunk's bands are
    // tiles of one launch per group, with one accumulation, replayed as a graph
    return run_batch(hs, batch, X, Y, nrhs, transpose != 0 ? 1 : 0, stream);
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_autotune(csrc_handle h, const void* x, void* y, cudaStream_t stream) {
  if (!h || !x || !y) return CSRC_ERR_INVALID_ARG;
  if (!is_device_ptr(x) || !is_device_ptr(y)) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  if (h->n == 0) {
    h->tuned = CSRC_STRAT_WINDOW;
    return CSRC_OK;
  }
  const int mode = tune_mode();
  if (mode == TUNE_OFF) return CSRC_OK;
  csrc_tune_key key;
  csrc_get_tune_key(h, &key);
  int32_t cached[4] = {0, 0, 0, 0};
  if (mode == TUNE_CACHE && csrc_tune_cache_lookup(&key, CSRC_TUNE_STRATEGY, 0.0, cached) == CSRC_OK &&
      cached[0] >= CSRC_STRAT_WINDOW && cached[0] <= CSRC_STRAT_WINDOW_ATOMIC && cached[1] >= 0 &&
      (cached[0] != CSRC_STRAT_COLOR || h->ncolors > 0)) {
    if (h->owner_nbands != cached[1]) {
      h->owner_nbands = cached[1];
      drop_owner_plans(h);
    }
    h->tuned = cached[0];
    ++h->generation;
    return CSRC_OK;
  }
  try {
    const bool prof = h->profiling;
    h->profiling = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CSRC_TRY(cudaEventCreate(&e0));
    CSRC_TRY(cudaEventCreate(&e1));
    auto time_it = [&](csrc_strategy st, float* ms) -> csrc_status {
      CSRC_TRY_S(run_spmv(h, x, y, st, stream, false));  // warm-up
      CSRC_TRY(cudaEventRecord(e0, stream));
      for (int i = 0; i < 3; ++i) CSRC_TRY_S(run_spmv(h, x, y, st, stream, false));
      CSRC_TRY(cudaEventRecord(e1, stream));
      CSRC_TRY(cudaEventSynchronize(e1));
      CSRC_TRY(cudaEventElapsedTime(ms, e0, e1));
      return CSRC_OK;
    };
    // the window strategy with the automatic band count (0; or the partition's count), one
    // wave of bands fewer and one more; then the stream-order strategies, and the colour
    // strategy when the rows are coloured
    float best = 1e30f;
    int32_t best_nb = 0, best_st = CSRC_STRAT_WINDOW;
    csrc_status st = CSRC_OK;
    const int32_t nb0 = h->part_nbands > 0 ? h->part_nbands : owner_auto_bands(h, 1);
    const int32_t wave = std::max<int32_t>(1, h->sms * owner_ctas_per_sm(1));
    const int32_t counts[3] = {h->part_nbands > 0 ? nb0 : 0, nb0 > wave ? nb0 - wave : std::max(1, nb0 / 2),
                               nb0 + wave};
    for (int32_t nb : counts) {
      if (nb > h->n) continue;
      h->owner_nbands = nb;
      drop_owner_plans(h);
      OwnerPlan* op = nullptr;
      const csrc_status ps = owner_for(h, 1, &op);
      if (ps == CSRC_ERR_NOT_PARTITIONED) continue;
      if ((st = ps) != CSRC_OK) break;
      float ms = 0.f;
      if ((st = time_it(CSRC_STRAT_WINDOW, &ms)) != CSRC_OK) break;
      if (ms < best) {
        best = ms;
        best_nb = nb;
        best_st = CSRC_STRAT_WINDOW;
      }
    }
    if (st == CSRC_OK) {
      const csrc_strategy cands[3] = {CSRC_STRAT_WINDOW_ATOMIC, CSRC_STRAT_ATOMIC, CSRC_STRAT_COLOR};
      for (csrc_strategy c : cands) {
        if (c == CSRC_STRAT_COLOR && h->ncolors == 0) continue;
        if (c != CSRC_STRAT_COLOR && !h->have_plan && (st = make_plan(h)) != CSRC_OK) break;
        if (c == CSRC_STRAT_WINDOW_ATOMIC && !h->plan_covers) continue;
        float ms = 0.f;
        if ((st = time_it(c, &ms)) != CSRC_OK) break;
        if (ms < best) {
          best = ms;
          best_st = c;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->profiling = prof;
    if (st != CSRC_OK) return st;
    if (h->owner_nbands != best_nb) {
      h->owner_nbands = best_nb;
      drop_owner_plans(h);
    }
    h->tuned = best_st;
    ++h->generation;
    const int32_t v[4] = {best_st, best_nb, 0, 0};
    csrc_tune_cache_store(&key, CSRC_TUNE_STRATEGY, 0.0, v);
    return CSRC_OK;
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_autotune_spmm(csrc_handle h, const void* X, void* Y, int32_t nrhs, cudaStream_t stream) {
  if (!h || !X || !Y || nrhs <= 0 || h->rect()) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  if (h->n == 0 || nrhs == 1) return CSRC_OK;
  const int mode = tune_mode();
  if (mode == TUNE_OFF) return CSRC_OK;
  csrc_tune_key key;
  csrc_get_tune_key(h, &key);
  int32_t cached[4] = {0, 0, 0, 0};
  if (mode == TUNE_CACHE && csrc_tune_cache_lookup(&key, CSRC_TUNE_KTILE, (double)nrhs, cached) == CSRC_OK &&
      (cached[0] == 1 || cached[0] == 2 || cached[0] == 4 || cached[0] == 8)) {
    h->tuned_rk = cached[0];
    ++h->generation;
    return CSRC_OK;
  }
  try {
    const bool prof = h->profiling;
    h->profiling = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CSRC_TRY(cudaEventCreate(&e0));
    CSRC_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int32_t best_rk = 0;
    csrc_status st = CSRC_OK;
    for (int32_t rk = 1; rk <= 8 && st == CSRC_OK; rk *= 2) {
      if (rk > nrhs) break;
      h->tuned_rk = rk;
      ++h->generation;
      const csrc_handle one[1] = {h};
      const void* const xs1[1] = {X};
      void* const ys1[1] = {Y};
      if ((st = run_batch(one, 1, xs1, ys1, nrhs, 0, stream)) != CSRC_OK) break;  // warm-up
      float ms = 0.f;
      cudaError_t ce = cudaEventRecord(e0, stream);
      for (int i = 0; i < 3 && st == CSRC_OK && ce == cudaSuccess; ++i) st = run_batch(one, 1, xs1, ys1, nrhs, 0, stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, stream);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) st = from_cuda(ce);
      if (st == CSRC_OK && ms < best) {
        best = ms;
        best_rk = rk;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->profiling = prof;
    h->tuned_rk = best_rk;
    ++h->generation;
    if (st == CSRC_OK && best_rk > 0) {
      const int32_t v[4] = {best_rk, 0, 0, 0};
      csrc_tune_cache_store(&key, CSRC_TUNE_KTILE, (double)nrhs, v);
    }
    return st;
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_get_tune_key(csrc_handle h, csrc_tune_key* key) {
  if (!h || !key) return CSRC_ERR_INVALID_ARG;
  std::memset(key, 0, sizeof(*key));
  key->pattern_hash = h->phash;
  key->n = h->n;
  key->nnz = (int64_t)h->n + 2 * h->h;
  key->storage = h->storage;
  key->flags = h->flags;
  std::memcpy(key->device, h->devname, sizeof(key->device));
  key->device[sizeof(key->device) - 1] = 0;
  return CSRC_OK;
}

csrc_status csrc_set_precision(csrc_handle h, csrc_dtype precision) {
  if (!h) return CSRC_ERR_INVALID_ARG;
  if (precision < CSRC_F64 || precision > CSRC_BF16) return CSRC_ERR_INVALID_ARG;
  if (h->storage != CSRC_F64 && precision != h->storage) return CSRC_ERR_INVALID_ARG;
  if (h->precision == precision) return CSRC_OK;
  drop_batches_of(h);
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  cudaDeviceSynchronize();  // products in flight may still read the lists being replaced
  h->precision = precision;
  drop_owner_plans(h);
  ++h->generation;
  return CSRC_OK;
}

csrc_status csrc_autotune_precision(csrc_handle h, const void* x, void* y, double max_rel_err, int32_t* chosen_out,
                                    double* bound_out, cudaStream_t stream) {
  if (!h || !x || !y || !(max_rel_err > 0.0) || h->rect()) return CSRC_ERR_INVALID_ARG;
  if (!is_device_ptr(x) || !is_device_ptr(y)) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  try {
    const int mode = tune_mode();
    csrc_tune_key key;
    csrc_get_tune_key(h, &key);
    int32_t cached[4] = {0, 0, 0, 0};
    if (mode == TUNE_CACHE && csrc_tune_cache_lookup(&key, CSRC_TUNE_PRECISION, max_rel_err, cached) == CSRC_OK &&
        cached[0] >= CSRC_F64 && cached[0] <= CSRC_BF16 && (h->storage == CSRC_F64 || cached[0] == h->storage)) {
      CSRC_TRY_S(csrc_set_precision(h, (csrc_dtype)cached[0]));
    } else if (mode != TUNE_OFF) {
      // candidates in the handle's reach, cheapest bytes first
      std::vector<csrc_dtype> cands;
      if (h->storage == CSRC_F64) cands = {CSRC_BF16, CSRC_F32, CSRC_F64};
      else cands = {h->storage};
      const bool prof = h->profiling;
      h->profiling = false;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      CSRC_TRY(cudaEventCreate(&e0));
      CSRC_TRY(cudaEventCreate(&e1));
      float best = 1e30f;
      int32_t best_p = -1;
      csrc_status st = CSRC_OK;
      for (csrc_dtype p : cands) {
        if ((st = csrc_set_precision(h, p)) != CSRC_OK) break;
        double bound = 0.0;
        if ((st = owner_error_bound(h, &bound)) != CSRC_OK) break;
        if (bound > max_rel_err) continue;
        if ((st = run_spmv(h, x, y, CSRC_STRAT_WINDOW, stream, false)) != CSRC_OK) break;  // warm-up
        cudaError_t ce = cudaEventRecord(e0, stream);
        for (int i = 0; i < 5 && st == CSRC_OK && ce == cudaSuccess; ++i)
          st = run_spmv(h, x, y, CSRC_STRAT_WINDOW, stream, false);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) st = from_cuda(ce);
        if (st != CSRC_OK) break;
        // narrower precisions come first and keep their place unless a wider one is more than
        // 3 % faster: a near-tie (a launch-bound small matrix) goes to the fewer bytes, which is
        // what counts once the matrix runs inside a batch
        if (best_p < 0 || ms < 0.97f * best) {
          best = ms;
          best_p = p;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      h->profiling = prof;
      if (st != CSRC_OK) return st;
      if (best_p < 0) return CSRC_ERR_INVALID_ARG;  // not even FP64 meets the budget
      CSRC_TRY_S(csrc_set_precision(h, (csrc_dtype)best_p));
      const int32_t v[4] = {best_p, 0, 0, 0};
      csrc_tune_cache_store(&key, CSRC_TUNE_PRECISION, max_rel_err, v);
    }
    double bound = 0.0;
    CSRC_TRY_S(owner_error_bound(h, &bound));
    if (chosen_out) *chosen_out = h->precision;
    if (bound_out) *bound_out = bound;
    return CSRC_OK;
  } catch (const std::bad_alloc&) {
    return CSRC_ERR_OUT_OF_MEMORY;
  }
}

csrc_status csrc_set_profiling(csrc_handle h, int32_t enable) {
  if (!h) return CSRC_ERR_INVALID_ARG;
  release_timing(h);
  h->profiling = enable != 0;
  return CSRC_OK;
}

csrc_status csrc_get_kernel_times(csrc_handle h, csrc_kernel_times* out) {
  if (!h || !out) return CSRC_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  csrc_status st = CSRC_OK;
  for (auto& t : h->timed) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(t.stop);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.start, t.stop);
    if (e != cudaSuccess) {
      st = from_cuda(e);
      break;
    }
    if (t.kind >= 0 && t.kind < CSRC_KERNEL_KINDS) {
      out->launches[t.kind] += t.kernels;
      out->ms[t.kind] += ms;
    }
  }
  release_timing(h);
  return st;
}

csrc_status csrc_bicg(csrc_handle h, const void* b, void* x, double rtol, int32_t maxit, csrc_strategy strategy,
                      int32_t* iters_out, double* relres_out, cudaStream_t stream) {
  if (iters_out) *iters_out = 0;
  if (relres_out) *relres_out = 0.0;
  if (!h || !b || !x || !(rtol >= 0.0) || maxit < 0 || h->rect()) return CSRC_ERR_INVALID_ARG;
  if (!is_device_ptr(b) || !is_device_ptr(x)) return CSRC_ERR_INVALID_ARG;
  const int64_t n = h->n;
  const size_t vb = (size_t)n * h->xbytes();
  const char* ba = static_cast<const char*>(b);
  const char* xa = static_cast<const char*>(x);
  if (ba < xa + vb && xa < ba + vb) return CSRC_ERR_ALIAS;
  if (n == 0) return CSRC_OK;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  const bool fp64 = h->xbytes() == 8;
  const int nb = solver_blocks(h->sms);
  if (!h->d_solve) CSRC_TRY(cudaMalloc(&h->d_solve, 6 * vb));
  if (!h->d_partial) CSRC_TRY(dmalloc(&h->d_partial, (size_t)2 * nb + 2));
  char* base = static_cast<char*>(h->d_solve);
  void *r = base, *rs = base + vb, *p = base + 2 * vb, *ps = base + 3 * vb, *q = base + 4 * vb, *qs = base + 5 * vb;
  double* out = h->d_partial + 2 * nb;
  double hv[2] = {0.0, 0.0};
  auto pass = [&](int op, double sc, const void* v0, const void* v1, const void* v2, void* w0, void* w1, void* w2,
                  void* w3) -> csrc_status {
    CSRC_TRY(timed_launch(h, CSRC_KERNEL_OTHER, stream, [&] {
      return launch_solver_op(op, fp64, n, nb, sc, v0, v1, v2, w0, w1, w2, w3, h->d_partial, out, stream);
    }, op == SOLVER_UPDATE2 ? 1 : 2));
    if (op != SOLVER_UPDATE2) {
      CSRC_TRY(cudaMemcpyAsync(hv, out, (op == SOLVER_DOT ? 1 : 2) * sizeof(double), cudaMemcpyDeviceToHost, stream));
      CSRC_TRY(cudaStreamSynchronize(stream));
    }
    return CSRC_OK;
  };
  // r = b - A x; r* = p = p* = r
  CSRC_TRY_S(run_spmv(h, x, q, strategy, stream, false));
  CSRC_TRY_S(pass(SOLVER_INIT, 0.0, b, q, nullptr, r, rs, p, ps));
  double nrm2 = hv[0];
  const double bb = hv[1];
  const double tol2 = rtol * rtol * bb;
  double rho = nrm2;  // (r, r*) with r* = r
  auto finish = [&](int32_t it, csrc_status st) {
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = bb > 0.0 ? std::sqrt(nrm2 / bb) : 0.0;
    // the products' device status word: an error raised during the solve is returned here
    // (and cleared) rather than left for a later call to find
    int32_t w = 0;
    if (cudaMemcpy(&w, h->d_status, 4, cudaMemcpyDeviceToHost) == cudaSuccess && w != 0) {
      cudaMemset(h->d_status, 0, 4);
      if (w & DEV_TIMEOUT) return CSRC_ERR_DEVICE_TIMEOUT;
      if (w & DEV_BOUNDS) return CSRC_ERR_DEVICE_BOUNDS;
      if (w & DEV_RANGE) return CSRC_ERR_RANGE;
    }
    return st;
  };
  if (nrm2 <= tol2) return finish(0, CSRC_OK);
  for (int32_t it = 1; it <= maxit; ++it) {
    CSRC_TRY_S(run_spmv(h, p, q, strategy, stream, false));
    CSRC_TRY_S(run_spmv(h, ps, qs, strategy, stream, true));
    CSRC_TRY_S(pass(SOLVER_DOT, 0.0, q, ps, nullptr, nullptr, nullptr, nullptr, nullptr));
    const double sigma = hv[0];
    if (rho == 0.0 || sigma == 0.0 || !std::isfinite(sigma)) return finish(it - 1, CSRC_ERR_BREAKDOWN);
    const double alpha = rho / sigma;
    CSRC_TRY_S(pass(SOLVER_UPDATE1, alpha, p, q, qs, x, r, rs, nullptr));
    nrm2 = hv[0];
    if (nrm2 <= tol2) return finish(it, CSRC_OK);
    const double rho_new = hv[1];
    const double beta = rho_new / rho;
    rho = rho_new;
    CSRC_TRY_S(pass(SOLVER_UPDATE2, beta, r, rs, nullptr, p, ps, nullptr, nullptr));
  }
  return finish(maxit, CSRC_ERR_NOT_CONVERGED);
}

csrc_status csrc_selftest_bounded_wait(int64_t cycles) {
  const long long limit = (long long)std::min<int64_t>(std::max<int64_t>(cycles, 1000), 2000000000LL);
  int32_t* status = nullptr;
  CSRC_TRY(dmalloc(&status, 1));
  int32_t w = 0;
  cudaError_t e = cudaMemset(status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = launch_wait_probe(limit, status, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&w, status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(status);
  CSRC_TRY(e);
  return (w & DEV_TIMEOUT) ? CSRC_ERR_DEVICE_TIMEOUT : CSRC_OK;
}

csrc_status csrc_get_info(csrc_handle h, csrc_info* info) {
  if (!h || !info) return CSRC_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n = h->n;
  info->pairs = h->h;
  info->nnz = (int64_t)h->n + 2 * h->h;
  info->storage = h->storage;
  info->arith = h->arith;
  const int64_t vb = (int64_t)h->vbytes(), xb = (int64_t)h->xbytes();
  // index bytes per pair: 2 with index compression (unless a stream-order plan had to keep
  // 32-bit slots because a window exceeds 65,536 rows)
  const int64_t ib = (h->flags & CSRC_FLAG_COMPRESS_INDICES) && (!h->have_plan || h->plan.jslot16) ? 2 : 4;
  info->model_bytes = 4 * ((int64_t)h->n + 1) + ib * h->h + (h->sym ? 1 : 2) * vb * h->h + vb * h->n + 2 * xb * h->n;
  if (h->have_plan) {
    info->nbands = h->plan.nb;
    info->page_rows = kPageRows;
    info->spill_entries = h->plan.spill;
    info->spill_rows = h->plan.nacc;
    // spill write + read + source index; row list and pointers; y read + write
    info->accum_bytes = h->plan.spill * (2 * xb + 4) + h->plan.nacc * (8 + 2 * xb);
    info->max_window_slots = h->plan.max_slots;
    info->smem_bytes = h->plan.smem_bytes;
    info->stream_nbands = h->plan.nb;
    info->stream_spill_entries = h->plan.spill;
  }
  if (h->have_oplan) {  // the window strategy's plan: its figures take precedence
    const OwnerPlan& p = h->oplan;
    info->nbands = p.nb;
    info->page_rows = 0;
    info->spill_entries = p.spill;
    info->spill_rows = p.nacc;
    info->accum_bytes = p.spill * (2 * xb + 4) + p.nacc * (8 + 2 * xb);
    info->max_window_slots = p.max_slots;
    info->smem_bytes = p.smem_bytes;
    info->list_entries = p.entries;
    info->list_slices = p.nslices;
    info->list_lane_steps = p.lane_steps;
    // what the owner kernel moves: slots and values of the entries, lane words and slice
    // offsets, band records, spill row list, x of every window slot, y and the spill writes
    info->list_bytes = (2 + vb) * p.entries + (4 * kOwnerLanes + 8) * p.nslices + 20 * (int64_t)p.nb +
                       4 * p.spill + xb * ((int64_t)h->n + p.spill) + xb * h->n + xb * p.spill;
  }
  info->ncolors = h->ncolors;
  info->precision = h->precision;
  if (h->have_oplan) owner_error_bound(h, &info->error_bound);
  info->tuned_strategy = h->tuned;
  info->tuned_rk = h->tuned_rk;
  info->group = h->have_plan ? h->plan.group : 0;
  info->block = h->have_plan ? h->plan.block : h->block;
  info->nstages = h->have_plan ? h->plan.nstages : 0;
  info->m = h->m;
  info->rect_nnz = h->rnnz;
  if (h->rect())  // the auxiliary CSR: compact row list and pointers, columns, values, x of the overlap
    info->model_bytes += 8 * (int64_t)h->nrrows + 4 + (4 + vb) * h->rnnz + xb * ((int64_t)h->m - h->n);
  return CSRC_OK;
}

csrc_status csrc_get_last_device_error(csrc_handle h) {
  if (!h) return CSRC_ERR_INVALID_ARG;
  DeviceGuard dg;
  CSRC_TRY_S(dg.enter(h));
  CSRC_TRY(cudaDeviceSynchronize());
  int32_t w = 0;
  CSRC_TRY(cudaMemcpy(&w, h->d_status, 4, cudaMemcpyDeviceToHost));
  CSRC_TRY(cudaMemset(h->d_status, 0, 4));
  if (w & DEV_TIMEOUT) return CSRC_ERR_DEVICE_TIMEOUT;
  if (w & DEV_BOUNDS) return CSRC_ERR_DEVICE_BOUNDS;
  if (w & DEV_RANGE) return CSRC_ERR_RANGE;
  return CSRC_OK;
}

csrc_status csrc_destroy(csrc_handle h) {
  if (!h) return CSRC_OK;
  drop_batches_of(h);
  DeviceGuard dg;
  dg.enter(h);
  cudaDeviceSynchronize();
  free_plan(h->plan);
  drop_owner_plans(h);
  free_plan(h->plan_b1);
  dfree(h->d_ia); dfree(h->d_ja); dfree(h->d_al); dfree(h->d_au); dfree(h->d_ad);
  dfree(h->d_al_df); dfree(h->d_au_df);
  dfree(h->d_rrow); dfree(h->d_rptr); dfree(h->d_rcol); dfree(h->d_rval);
  dfree(h->d_tptr); dfree(h->d_trow); dfree(h->d_tval);
  dfree(h->d_solve); dfree(h->d_partial);
  dfree(h->d_status); dfree(h->d_color_desc); dfree(h->d_cja); dfree(h->d_cal); dfree(h->d_cau);
  dfree(h->d_color_ptr); dfree(h->d_barrier); dfree(h->d_xs);
  dfree(h->d_ys);
  release_timing(h);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  delete h;
  return CSRC_OK;
}

const char* csrc_status_string(csrc_status st) {
  switch (st) {
    case CSRC_OK: return "success";
    case CSRC_ERR_INVALID_ARG: return "invalid argument";
    case CSRC_ERR_NOT_STRUCT_SYMMETRIC: return "pattern is not structurally symmetric";
    case CSRC_ERR_INDEX_RANGE: return "index out of range";
    case CSRC_ERR_DUPLICATE: return "duplicate or unsorted column in a CSR row";
    case CSRC_ERR_ALIAS: return "x and y overlap";
    case CSRC_ERR_NOT_PARTITIONED: return "no window plan fits this matrix for the requested strategy";
    case CSRC_ERR_NOT_COLORED: return "colour strategy requested before csrc_color";
    case CSRC_ERR_OUT_OF_MEMORY: return "out of memory";
    case CSRC_ERR_CUDA: return "CUDA runtime error";
    case CSRC_ERR_DEVICE_TIMEOUT: return "bounded device wait ran out";
    case CSRC_ERR_DEVICE_BOUNDS: return "device index check failed";
    case CSRC_ERR_RANGE: return "x value outside the double-float range";
    case CSRC_ERR_MISMATCH: return "storage type mismatch";
    case CSRC_ERR_NOT_NUM_SYMMETRIC: return "symmetric-value storage requested but a_ij != a_ji";
    case CSRC_ERR_NOT_CONVERGED: return "iteration limit reached above the tolerance";
    case CSRC_ERR_BREAKDOWN: return "BiCG breakdown: a zero inner product";
    case CSRC_ERR_NOT_FOUND: return "no tuning cache entry for this key";
    case CSRC_ERR_IO: return "the tuning cache file cannot be written";
  }
  return "unknown status";
}

}  // extern "C"
