// Host side of the window strategy's owner lists (layout described in internal.h).
//
// For each band of the Section 3.1 partition the builder finds the band's effective
// range (its own rows and the rows below it that its pairs scatter into), numbers
// those rows as window slots, sorts the band's scatter by target (a counting sort of
// its pairs by ja), and writes every slot's entry list in jagged-diagonal order. Bands
// are independent, so both passes run on several host threads. The values are then
// gathered on the device from the handle's al / au / ad.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"

namespace csrc {
namespace {

struct PlanBand {
  int32_t r0, r1, nspill;
};

// Per-thread scratch. stamp[j] == cur marks row j as a spill row of the band being built,
// with slot[j] its slot.
struct Scratch {
  std::vector<int32_t> stamp, slot, sp, ptr, fill, order, upk, upr, len;
  int32_t cur = 0;
  explicit Scratch(int32_t n) : stamp((size_t)n, 0), slot((size_t)n, 0) {}
};

// Distinct columns below r0 of the pairs of rows [r0, r1), ascending (the band's spill rows);
// afterwards sc.slot[j] is the slot of spill row j.
void collect_spill_rows(const std::vector<int32_t>& ia, const std::vector<int32_t>& ja, int32_t r0, int32_t r1,
                        Scratch& sc) {
  ++sc.cur;
  sc.sp.clear();
  for (int64_t k = ia[(size_t)r0]; k < ia[(size_t)r1]; ++k) {
    const int32_t j = ja[(size_t)k];
    if (j < r0 && sc.stamp[(size_t)j] != sc.cur) {
      sc.stamp[(size_t)j] = sc.cur;
      sc.sp.push_back(j);
    }
  }
  std::sort(sc.sp.begin(), sc.sp.end());
  for (size_t s = 0; s < sc.sp.size(); ++s) sc.slot[(size_t)sc.sp[s]] = (int32_t)s;
}

// First pass: the bands of partition bands [t0, t1), each split at its non-zero midpoint
// while its window (own + spill rows, rk columns of slot_bytes each) does not fit.
// Returns false when a single row's window does not fit.
bool plan_bands(const std::vector<int32_t>& ia, const std::vector<int32_t>& ja, const std::vector<int32_t>& part,
                size_t t0, size_t t1, int64_t slot_bytes, int64_t budget, Scratch& sc, std::vector<PlanBand>& out) {
  std::vector<std::pair<int32_t, int32_t>> stack;
  for (size_t t = t0; t < t1; ++t) {
    if (part[t + 1] <= part[t]) continue;
    stack.push_back({part[t], part[t + 1]});
    while (!stack.empty()) {
      const auto rg = stack.back();
      stack.pop_back();
      const int32_t r0 = rg.first, r1 = rg.second;
      collect_spill_rows(ia, ja, r0, r1, sc);
      const int64_t nslots = (int64_t)sc.sp.size() + (r1 - r0);
      if (nslots <= kOwnerMaxSlots && nslots * slot_bytes <= budget) {
        out.push_back({r0, r1, (int32_t)sc.sp.size()});
        continue;
      }
      if (r1 - r0 <= 1) return false;
      // split where the prefix weight (w_i = 1 + 2 pairs(i)) reaches half of the band's
      const int64_t tot = (int64_t)(r1 - r0) + 2 * ((int64_t)ia[(size_t)r1] - ia[(size_t)r0]);
      int64_t P = 0;
      int32_t mid = r0;
      while (mid < r1 && 2 * P < tot) {
        P += 1 + 2 * ((int64_t)ia[(size_t)mid + 1] - ia[(size_t)mid]);
        ++mid;
      }
      if (mid <= r0 || mid >= r1) mid = r0 + (r1 - r0) / 2;
      stack.push_back({mid, r1});  // processed after the left half
      stack.push_back({r0, mid});
    }
  }
  return true;
}

struct Layout {
  std::vector<int4> band;
  std::vector<int32_t> band_slice;
  std::vector<int64_t> band_entry;  // first entry of each band (nb + 1)
};

// Second pass: the lists of band b, written in its region [e0, e_end) of the entry arrays.
// Returns false when a list is longer than kOwnerMaxLength.
bool fill_band(const std::vector<int32_t>& ia, const std::vector<int32_t>& ja, const PlanBand& pb, const int4& bd,
               int32_t q0, int64_t e0, int64_t e_end, int blk, Scratch& sc, int64_t* slice_off, uint32_t* lane,
               uint16_t* S, int64_t* code, int32_t* spill_row, int64_t* lane_steps) {
  const int32_t r0 = pb.r0, r1 = pb.r1;
  collect_spill_rows(ia, ja, r0, r1, sc);
  const int32_t nsp = (int32_t)sc.sp.size();
  const int32_t nown = r1 - r0, nslots = nsp + nown;
  for (int32_t s = 0; s < nsp; ++s) spill_row[(size_t)bd.w + s] = sc.sp[(size_t)s];
  auto slot_of = [&](int32_t j) -> int32_t { return j >= r0 ? nsp + (j - r0) : sc.slot[(size_t)j]; };
  // the band's scatter sorted by target slot (counting sort, pairs in k order within a target)
  const int64_t k0 = ia[(size_t)r0], k1 = ia[(size_t)r1];
  sc.ptr.assign((size_t)nslots + 1, 0);
  for (int64_t k = k0; k < k1; ++k) sc.ptr[(size_t)slot_of(ja[(size_t)k]) + 1]++;
  for (int32_t t = 0; t < nslots; ++t) sc.ptr[(size_t)t + 1] += sc.ptr[(size_t)t];
  sc.fill.assign(sc.ptr.begin(), sc.ptr.end() - 1);
  sc.upk.resize((size_t)(k1 - k0));
  sc.upr.resize((size_t)(k1 - k0));
  for (int32_t r = r0; r < r1; ++r)
    for (int64_t k = ia[(size_t)r]; k < ia[(size_t)r + 1]; ++k) {
      const int32_t q = sc.fill[(size_t)slot_of(ja[(size_t)k])]++;
      sc.upk[(size_t)q] = (int32_t)(k - k0);
      sc.upr[(size_t)q] = r;
    }
  // list lengths, and slots by length (descending; ties in slot order)
  sc.len.resize((size_t)nslots);
  for (int32_t t = 0; t < nslots; ++t) {
    int64_t L = sc.ptr[(size_t)t + 1] - sc.ptr[(size_t)t];
    if (t >= nsp) {
      const int32_t r = r0 + (t - nsp);
      L += 1 + ((int64_t)ia[(size_t)r + 1] - ia[(size_t)r]);
    }
    if (L > kOwnerMaxLength) return false;
    sc.len[(size_t)t] = (int32_t)L;
  }
  sc.order.resize((size_t)nslots);
  for (int32_t t = 0; t < nslots; ++t) sc.order[(size_t)t] = t;
  std::stable_sort(sc.order.begin(), sc.order.end(),
                   [&](int32_t a, int32_t b) { return sc.len[(size_t)a] > sc.len[(size_t)b]; });
  // slices of 32 slots in jagged-diagonal order
  int64_t E = e0;
  const int32_t nsl = (nslots + kOwnerLanes - 1) / kOwnerLanes;
  for (int32_t q = 0; q < nsl; ++q) {
    const int32_t a = q * kOwnerLanes;
    const int32_t cnt = std::min(kOwnerLanes, nslots - a);
    uint32_t* lw = lane + (size_t)(q0 + q) * kOwnerLanes;
    for (int32_t l = 0; l < kOwnerLanes; ++l) {
      if (l < cnt) {
        const int32_t t = sc.order[(size_t)a + l];
        lw[l] = ((uint32_t)sc.len[(size_t)t] << 16) | (uint32_t)t;
      } else {
        lw[l] = kOwnerPadSlot;  // length 0
      }
    }
    E = (E + blk - 1) / blk * blk;  // slices start on a block boundary
    slice_off[(size_t)q0 + q] = E;
    const int64_t base = E;
    const int32_t maxlen = sc.len[(size_t)sc.order[(size_t)a]];
    // regular part: the steps below the shortest list (lane 31's; 0 when lanes are unused), in
    // whole blocks of blk steps, each lane's steps of a block side by side
    const int32_t minlen = cnt == kOwnerLanes ? sc.len[(size_t)sc.order[(size_t)a + cnt - 1]] : 0;
    const int32_t regular = minlen / blk * blk;
    *lane_steps += (int64_t)kOwnerLanes * maxlen;
    int32_t active = cnt;  // lanes whose list is longer than m (a prefix: lengths descend)
    for (int32_t m = 0; m < maxlen; ++m) {
      if (m == regular) E = base + (int64_t)kOwnerLanes * regular;  // the ragged tail follows
      while (active > 0 && sc.len[(size_t)sc.order[(size_t)a + active - 1]] <= m) --active;
      for (int32_t l = 0; l < active; ++l) {
        const int32_t t = sc.order[(size_t)a + l];
        int64_t c = 0;
        int32_t s = 0;
        int32_t u = m;  // index into the slot's upper entries
        if (t >= nsp) {
          const int32_t r = r0 + (t - nsp);
          const int32_t L = ia[(size_t)r + 1] - ia[(size_t)r];
          if (m == 0) {
            c = (int64_t)r << 2;  // diagonal
            s = t;
            u = -1;
          } else if (m <= L) {
            const int64_t k = ia[(size_t)r] + (m - 1);
            c = (k << 2) | 1;  // lower pair: al[k] with x[ja[k]]
            s = slot_of(ja[(size_t)k]);
            u = -1;
          } else {
            u = m - 1 - L;
          }
        }
        if (u >= 0) {
          const int32_t qq = sc.ptr[(size_t)t] + u;
          c = ((int64_t)(k0 + sc.upk[(size_t)qq]) << 2) | 2;  // scattered pair: au[k] with x of its row
          s = nsp + (sc.upr[(size_t)qq] - r0);
        }
        const int64_t pos = m < regular ? base + (int64_t)kOwnerLanes * blk * (m / blk) + (int64_t)blk * l + m % blk
                                        : E + l;
        S[(size_t)pos] = (uint16_t)s;
        code[(size_t)pos] = c;
      }
      if (m >= regular) E += active;
    }
    if (regular == maxlen) E = base + (int64_t)kOwnerLanes * regular;
  }
  return E <= e_end;
}

template <typename T>
cudaError_t upload_vec(T** d, const std::vector<T>& v) {
  *d = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), std::max<size_t>(1, v.size()) * sizeof(T));
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

int worker_count() {
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(16u, hc == 0 ? 4u : hc));
}

// Runs fn(w) for w < workers on host threads (fn(0) on the caller's thread).
template <typename F>
void run_workers(int workers, F&& fn) {
  std::vector<std::thread> th;
  for (int w = 1; w < workers; ++w) th.emplace_back([&, w] { fn(w); });
  fn(0);
  for (auto& t : th) t.join();
}

}  // namespace

void free_owner_plan(OwnerPlan& p) {
  void* ptrs[] = {p.band, p.band_slice, p.slice_off, p.lane, p.spill_row, p.spill_pos, p.S, p.VA,
                  p.VT == p.VA ? nullptr : p.VT, p.acc_row, p.acc_ptr, p.spill_buf};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p = OwnerPlan();
}

csrc_status build_owner_plan(int32_t n, int64_t h, const std::vector<int32_t>& ia, const std::vector<int32_t>& ja,
                             const std::vector<int32_t>& part, int rk, int mode, int budget, int in_bytes,
                             const void* al, const void* au, const void* ad, bool sym, OwnerPlan& out) {
  (void)h;
  const int slot_bytes = owner_acc_bytes(mode), spill_bytes = owner_acc_bytes(mode);
  const int blk = owner_block(mode, rk);
  const int vbytes = owner_value_bytes(mode);
  free_owner_plan(out);
  const int workers = std::max(1, std::min<int>(worker_count(), n / 4096 + 1));
  // ---- pass 1: bands whose windows fit (in partition order)
  const size_t nparts = part.size() > 0 ? part.size() - 1 : 0;
  std::vector<std::vector<PlanBand>> chunks((size_t)workers);
  std::vector<char> ok((size_t)workers, 1);
  {
    run_workers(workers, [&](int w) {
      Scratch sc(n);
      const size_t t0 = nparts * (size_t)w / (size_t)workers, t1 = nparts * (size_t)(w + 1) / (size_t)workers;
      ok[(size_t)w] = plan_bands(ia, ja, part, t0, t1, (int64_t)slot_bytes * rk, budget, sc, chunks[(size_t)w]);
    });
  }
  for (char c : ok)
    if (!c) return CSRC_ERR_NOT_PARTITIONED;
  std::vector<PlanBand> bands;
  for (auto& c : chunks) bands.insert(bands.end(), c.begin(), c.end());
  chunks.clear();
  const int32_t nb = (int32_t)bands.size();
  // ---- offsets
  Layout L;
  L.band.resize((size_t)nb);
  L.band_slice.assign((size_t)nb + 1, 0);
  L.band_entry.assign((size_t)nb + 1, 0);
  int64_t spill = 0, entries_used = 0;
  int32_t max_slots = 0;
  for (int32_t b = 0; b < nb; ++b) {
    const PlanBand& pb = bands[(size_t)b];
    const int32_t nown = pb.r1 - pb.r0, nslots = pb.nspill + nown;
    int4& bd = L.band[(size_t)b];
    bd.x = pb.r0;
    bd.y = nown;
    bd.z = pb.nspill;
    bd.w = (int)spill;
    spill += pb.nspill;
    if (spill > (int64_t)INT32_MAX - 1) return CSRC_ERR_NOT_PARTITIONED;
    max_slots = std::max(max_slots, nslots);
    L.band_slice[(size_t)b + 1] = L.band_slice[(size_t)b] + (nslots + kOwnerLanes - 1) / kOwnerLanes;
    // the band's region: its entries plus room to start every slice on a block boundary
    const int64_t need = nown + 2 * ((int64_t)ia[(size_t)pb.r1] - ia[(size_t)pb.r0]) +
                         (int64_t)(blk - 1) * ((nslots + kOwnerLanes - 1) / kOwnerLanes);
    L.band_entry[(size_t)b + 1] = L.band_entry[(size_t)b] + (need + blk - 1) / blk * blk;
    entries_used += nown + 2 * ((int64_t)ia[(size_t)pb.r1] - ia[(size_t)pb.r0]);
  }
  const int64_t nslices = L.band_slice[(size_t)nb];
  const int64_t entries = L.band_entry[(size_t)nb];
  // ---- pass 2: the lists
  std::vector<int64_t> slice_off((size_t)std::max<int64_t>(1, nslices));
  std::vector<uint32_t> lane((size_t)std::max<int64_t>(1, nslices * kOwnerLanes));
  std::vector<uint16_t> S((size_t)std::max<int64_t>(1, entries));
  std::vector<int64_t> code((size_t)std::max<int64_t>(1, entries));
  std::vector<int32_t> spill_row((size_t)std::max<int64_t>(1, spill));
  std::vector<int64_t> steps((size_t)workers, 0);
  std::atomic<int32_t> next{0};
  std::atomic<bool> fits{true};
  run_workers(workers, [&](int w) {
    Scratch sc(n);
    while (true) {
      const int32_t b = next.fetch_add(1);
      if (b >= nb) break;
      if (!fill_band(ia, ja, bands[(size_t)b], L.band[(size_t)b], L.band_slice[(size_t)b],
                     L.band_entry[(size_t)b], L.band_entry[(size_t)b + 1], blk, sc, slice_off.data(), lane.data(),
                     S.data(), code.data(), spill_row.data(), &steps[(size_t)w]))
        fits = false;
    }
  });
  if (!fits) return CSRC_ERR_NOT_PARTITIONED;
  // ---- accumulation map: spill slots grouped by row (ascending), in band order within a row
  std::vector<int32_t> cnt((size_t)n + 1, 0);
  for (int64_t g = 0; g < spill; ++g) cnt[(size_t)spill_row[(size_t)g] + 1]++;
  std::vector<int32_t> acc_row, acc_ptr{0};
  for (int32_t r = 0; r < n; ++r)
    if (cnt[(size_t)r + 1]) {
      acc_row.push_back(r);
      acc_ptr.push_back(acc_ptr.back() + cnt[(size_t)r + 1]);
    }
  std::vector<int32_t> first((size_t)n + 1, 0);
  for (int32_t r = 0; r < n; ++r) first[(size_t)r + 1] = first[(size_t)r] + cnt[(size_t)r + 1];
  std::vector<int32_t> spill_pos((size_t)std::max<int64_t>(1, spill));
  for (int64_t g = 0; g < spill; ++g) spill_pos[(size_t)g] = first[(size_t)spill_row[(size_t)g]]++;
  // ---- upload
  OwnerPlan p;
  p.nb = nb;
  p.rk = rk;
  p.mode = mode;
  for (int64_t q = 0; q < nslices; ++q) p.max_len = std::max<int32_t>(p.max_len, (int32_t)(lane[(size_t)q * kOwnerLanes] >> 16));
  p.entries = entries_used;
  p.capacity = entries;
  p.nslices = nslices;
  p.spill = spill;
  p.max_slots = max_slots;
  p.smem_bytes = std::max(16, max_slots * slot_bytes * rk);
  for (int64_t v : steps) p.lane_steps += v;
  p.nacc = (int64_t)acc_row.size();
  for (size_t i = 0; i + 1 < acc_ptr.size(); ++i) p.max_parts = std::max(p.max_parts, 1 + acc_ptr[i + 1] - acc_ptr[i]);
  p.band_entries.resize((size_t)nb);
  for (int32_t b = 0; b < nb; ++b)
    p.band_entries[(size_t)b] = L.band_entry[(size_t)b + 1] - L.band_entry[(size_t)b];
  cudaError_t e = cudaSuccess;
  auto up = [&](auto** d, const auto& v) {
    if (e == cudaSuccess) e = upload_vec(d, v);
  };
  up(&p.band, L.band);
  up(&p.band_slice, L.band_slice);
  up(&p.slice_off, slice_off);
  up(&p.lane, lane);
  up(&p.spill_row, spill_row);
  up(&p.S, S);
  up(&p.acc_row, acc_row);
  up(&p.acc_ptr, acc_ptr);
  up(&p.spill_pos, spill_pos);
  if (e == cudaSuccess)
    e = cudaMalloc(&p.spill_buf, std::max<size_t>(1, (size_t)spill * (size_t)rk * (size_t)spill_bytes));
  int64_t* dcode = nullptr;
  if (e == cudaSuccess) e = upload_vec(&dcode, code);
  code.clear();
  code.shrink_to_fit();
  if (e == cudaSuccess) e = cudaMalloc(&p.VA, std::max<size_t>(1, (size_t)entries * (size_t)vbytes));
  if (e == cudaSuccess && !sym) e = cudaMalloc(&p.VT, std::max<size_t>(1, (size_t)entries * (size_t)vbytes));
  if (e == cudaSuccess && sym) p.VT = p.VA;
  if (e == cudaSuccess)
    e = launch_owner_gather(in_bytes, vbytes, dcode, entries, al, sym ? al : au, ad, p.VA, sym ? nullptr : p.VT, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (dcode) cudaFree(dcode);
  if (e != cudaSuccess) {
    free_owner_plan(p);
    return e == cudaErrorMemoryAllocation ? CSRC_ERR_OUT_OF_MEMORY : CSRC_ERR_CUDA;
  }
  out = std::move(p);
  return CSRC_OK;
}

}  // namespace csrc
