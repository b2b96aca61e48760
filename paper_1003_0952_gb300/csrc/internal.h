// Internal declarations shared by the host library (api.cpp) and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime_api.h>

#include "../../include/csrc.h"

namespace csrc {

// Rows per window page (page table granularity, one 64-bit spill mask per page).
constexpr int kPageShift = 6;
constexpr int kPageRows = 1 << kPageShift;


// Stored arrays (ja, al, au) are padded so that 8-pair aligned bulk copies stay inside them.
constexpr int kPairAlign = 8;

// Kernel modes (storage x arithmetic).
enum { MODE_DF = 0, MODE_F64 = 1, MODE_F32 = 2, MODE_BF16 = 3 };

// Shape of the band kernel per mode: T threads, ring stages of up to kStageCap pairs
// (plus 16 for alignment), NS stages, CTAs per SM. A stage holds whole rows (a row longer
// than a stage is cut), at most T/G of them, G = lanes per row (a per-matrix choice).
// kSlotBytes = shared bytes per window row (x plus its accumulator).
template <int MODE>
struct BandShape {
  static constexpr int T = 512;
  static constexpr int kStageCap = 2560;
  static constexpr int NS = 3;
  static constexpr int kCtasPerSm = 1;
  static constexpr int kValueBytes = MODE == MODE_BF16 ? 2 : (MODE == MODE_F32 ? 4 : 8);
  static constexpr int kSlotBytes = (MODE == MODE_DF || MODE == MODE_F64) ? 16 : 8;
  static constexpr int kSlotPairs = kStageCap + 16;
  static constexpr int ring_bytes() { return NS * kSlotPairs * (4 + 2 * kValueBytes); }
};
constexpr int kBandThreads = 512;
// Threads of a band CTA: 512, or 1024 when single-vector rows are taken by 16 lanes each
// (rows of 32 or more pairs): twice the warps hide more shared-memory latency, and the
// kernel then fits in 64 registers per thread.
__host__ __device__ constexpr int band_threads(int G, int B, int RK) {
  return (G == 16 && B == 1 && RK == 1) ? 1024 : kBandThreads;
}
constexpr int kStageCap = 2560;

// Shared memory ahead of the ring (mbarriers: NS full, NS empty, one for the band's set-up copies).
constexpr int kRingOffset = 128;

// Dynamic shared memory a band CTA may use, per mode (a little below the per-CTA maximum
// for its CTAs-per-SM target, leaving room for static shared variables).
constexpr int kSmemPerSm = 233472;   // 228 KB on sm_103
constexpr int kSmemPerCtaMax = 232448;  // 227 KB opt-in maximum
constexpr int smem_limit_for(int ctas_per_sm) {
  return (ctas_per_sm <= 1 ? kSmemPerCtaMax : kSmemPerSm / ctas_per_sm - 1024) - 256;
}
inline int band_smem_limit(int mode) {
  switch (mode) {
    case MODE_DF: return smem_limit_for(BandShape<MODE_DF>::kCtasPerSm);
    case MODE_F64: return smem_limit_for(BandShape<MODE_F64>::kCtasPerSm);
    case MODE_F32: return smem_limit_for(BandShape<MODE_F32>::kCtasPerSm);
    default: return smem_limit_for(BandShape<MODE_BF16>::kCtasPerSm);
  }
}
inline int band_ring_bytes(int mode) {
  switch (mode) {
    case MODE_DF: return kRingOffset + BandShape<MODE_DF>::ring_bytes();
    case MODE_F64: return kRingOffset + BandShape<MODE_F64>::ring_bytes();
    case MODE_F32: return kRingOffset + BandShape<MODE_F32>::ring_bytes();
    default: return kRingOffset + BandShape<MODE_BF16>::ring_bytes();
  }
}

// Layout of a band's shared memory after the ring, identical on host and device:
// [x of the window slots][window sums][page table][ia slice][stage_k slice][stage_r slice].
// The ia slice covers rows [r0 & ~3, (r1 + 4) & ~3), the stage slices cover stage entries
// [st0 & ~3, (st1 + 4) & ~3) where st1 = index of the band's end entry; each part is a
// multiple of 16 bytes so that it can be filled by bulk copies.
struct BandLayout {
  int xs, acc, tab, ia, sk, sr, end;  // byte offsets from the ring's end
  static constexpr int up16(int v) { return (v + 15) & ~15; }
  __host__ __device__ static BandLayout make(int nslots, int x_bytes, int acc_bytes, int ntab, int r0, int r1,
                                             int st0, int st1) {
    BandLayout l;
    l.xs = 0;
    l.acc = nslots * x_bytes;
    l.tab = l.acc + nslots * acc_bytes;
    l.ia = l.tab + up16(4 * ntab);
    const int nia = ((r1 + 4) & ~3) - (r0 & ~3);
    l.sk = l.ia + 4 * nia;
    const int nst = ((st1 + 4) & ~3) - (st0 & ~3);
    l.sr = l.sk + 4 * nst;
    l.end = l.sr + 4 * nst;
    return l;
  }
};
// Bytes per window slot of x and of the sums, per mode.
constexpr int window_x_bytes(int mode) { return (mode == MODE_DF || mode == MODE_F64) ? 8 : 4; }
constexpr int window_acc_bytes(int mode) { return (mode == MODE_DF || mode == MODE_F64) ? 8 : 4; }
// Padding (in entries) after ia and the stage arrays, so the rounded-up slices stay inside.
constexpr int kMetaPad = 8;

inline int band_slot_bytes(int mode) { return (mode == MODE_DF || mode == MODE_F64) ? 16 : 8; }

// Arithmetic of a product.
enum Arith : int32_t { ARITH_DF32 = 0, ARITH_F64 = 1, ARITH_F32 = 2 };

inline int mode_of(Arith arith, int storage) {
  if (storage == CSRC_F32) return MODE_F32;
  if (storage == CSRC_BF16) return MODE_BF16;
  return arith == ARITH_F64 ? MODE_F64 : MODE_DF;
}

// Device arrays of one execution plan of the window / atomic strategies.
// A plan is a list of row bands. Band b covers rows [band_row[b], band_row[b+1]).
// Its shared-memory window is a set of pages of kPageRows rows (wpage[band_wp[b]..band_wp[b+1])),
// indexed through a page table that spans pages [band_plo[b], band_plo[b] + band_ntab[b]).
struct DevPlan {
  int32_t nb = 0;
  int32_t group = 1;             // lanes per row unit (1, 2, 4, 8 or 16)
  int32_t block = 1;             // rows per unit: node blocks of 2 or 3 rows, else 1
  int64_t nstages = 0;           // ring stages over all bands
  int32_t* band_stage = nullptr; // nb+1: stages of band b are [band_stage[b], band_stage[b+1]-1)
  int32_t* stage_k = nullptr;    // first pair of each stage (the band's last entry is its end)
  int32_t* stage_r = nullptr;    // first row of each stage
  int32_t* band_row = nullptr;   // nb+1
  int32_t* band_plo = nullptr;   // nb
  int32_t* band_ntab = nullptr;  // nb
  int32_t* band_wp = nullptr;    // nb+1
  int32_t* wpage = nullptr;      // total window pages
  int32_t* wbase = nullptr;      // per window page: first spill index of the page
  uint64_t* wmask = nullptr;     // per window page: rows (bit = row & 63) that spill (row < band start)
  // accumulation (spill -> y) map, rows ascending, sources in band order
  int64_t spill = 0;             // spill entries
  int64_t nacc = 0;              // rows that receive spills
  int32_t* acc_row = nullptr;    // nacc
  int32_t* acc_ptr = nullptr;    // nacc+1
  int32_t* acc_src = nullptr;    // spill
  void* spill_buf = nullptr;     // spill values (double or float)
  int32_t max_slots = 0;
  int32_t max_tab = 0;
  int32_t smem_bytes = 0;      // dynamic shared memory of a band CTA (ring + window + table)
  std::vector<int64_t> band_pairs;  // host copy: stored pairs of each band (batched scheduling)
  int64_t total_pages = 0;
  // plans of plain rows: the window slot of every stored pair, written in place of its
  // column for the window strategy (h entries, padded like ja)
  int32_t* jslot = nullptr;
  uint16_t* jslot16 = nullptr;   // the same slots as 16 bits (index compression); jslot is then null
};

// ---------------------------------------------------------------------------- owner lists
// The window strategy's plan (owner.cu, owner_plan.cpp). Each band [r0, r1) of the
// Section 3.1 partition writes the rows of its effective range: its own rows and the
// rows below r0 that its pairs scatter into ("spill rows"). Window slots number them:
// slots [0, nspill) are the spill rows in ascending order, slots [nspill, nspill + nown)
// the own rows. Every slot has an entry list, each entry a (value, slot) couple whose
// product value * x[slot] belongs to the slot's row:
//   own row r:  the diagonal ad[r] (with x of r), the row's lower pairs al[k] (with x of
//               ja[k]) in column order, then the pairs of later rows i of the band with
//               ja[k] = r, au[k] (with x of i), in row order;
//   spill row:  the pairs of the band that scatter into it, au[k] with x of their row.
// A^T x uses the same lists with al and au exchanged (Section 5). The scatter of Fig. 2(a)
// is thereby sorted by target when the plan is built, and each slot's sum is formed by one
// lane in registers: no two lanes ever add into the same window row.
// The lists of a band are stored in jagged-diagonal order: slots are sorted by list length
// (descending), cut into slices of 32 (one lane each), and step m of a slice holds entry m
// of every lane whose list is longer than m, contiguously, so that a warp's loads of one
// step are coalesced.
constexpr int kOwnerLanes = 32;
// The regular part of a slice (the steps below its shortest list, where all 32 lanes are
// active) is stored in blocks of B steps with each lane's steps side by side: entry (m, lane)
// at slice start + 32 * B * (m / B) + B * lane + m % B, so that a lane reads a block with
// vector loads; slices start on a block boundary, and the ragged tail (jagged-diagonal order)
// follows the regular part. B = owner_block(mode, rk): 8 steps for 2-byte values in single-
// column passes (one 16-byte load of slots and one of values; measured 9 % faster on q1v_96 in
// BF16, 3-4 % slower for rk > 1 and for the short lists of a Delaunay mesh), 4 otherwise.
constexpr int kOwnerBlock = 4;
constexpr uint32_t kOwnerPadSlot = 0xffffu;  // lane word slot of an unused lane (length 0)
constexpr int kOwnerMaxSlots = 65535;         // slots are 16-bit; 0xffff marks unused lanes
constexpr int kOwnerMaxLength = 65535;        // list lengths are 16-bit

// Arithmetic modes of the owner kernel: the storage of the listed values and the type of x
// and y. Modes 0-2 are the handle's storage types (FP64: FP64 arithmetic; FP32 / BF16: FP32
// arithmetic on float vectors). Modes 3-4 serve a CSRC_F64 handle whose window strategy runs at
// a reduced precision (csrc_set_precision): values rounded to FP32 / BF16, x rounded to FP32 in
// the window, FP32 multiply-adds, y written as double.
enum OwnerMode : int { OM_F64 = 0, OM_F32 = 1, OM_BF16 = 2, OM_F32_X64 = 3, OM_BF16_X64 = 4 };
constexpr int kOwnerModes = 5;
inline int owner_value_bytes(int mode) { return mode == OM_F64 ? 8 : ((mode == OM_F32 || mode == OM_F32_X64) ? 4 : 2); }
inline int owner_acc_bytes(int mode) { return mode == OM_F64 ? 8 : 4; }   // window x, sums, spill
inline int owner_vec_bytes(int mode) { return (mode == OM_F64 || mode >= OM_F32_X64) ? 8 : 4; }  // x, y
__host__ __device__ constexpr int owner_block(int mode, int rk) {
  return (mode == OM_BF16 || mode == OM_BF16_X64) && rk == 1 ? 8 : 4;
}
constexpr int kOwnerMaxBlock = 8;

// Kernel shape: threads per CTA and CTAs per SM the window budget is sized for.
// Four CTAs of 256 threads per SM for every column count: wider passes get smaller bands (a
// window holds rk columns of x) rather than fewer warps, which measured faster for rk = 2..8.
__host__ __device__ constexpr int owner_threads(int rk) { return rk > 0 ? 256 : 256; }
__host__ __device__ constexpr int owner_ctas_per_sm(int rk) { return rk > 0 ? 4 : 4; }
inline int owner_smem_budget(int rk) { return smem_limit_for(owner_ctas_per_sm(rk)); }

struct OwnerPlan {
  int32_t nb = 0;            // bands
  int32_t rk = 1;            // columns per pass the windows are sized for
  int32_t mode = OM_F64;     // OwnerMode of the values
  int32_t max_len = 0;       // longest entry list
  int32_t max_parts = 1;     // most partial sums of one row (its own band's and the spilled ones)
  int64_t entries = 0;       // list entries of all bands (n + 2h)
  int64_t capacity = 0;      // length of the entry arrays (entries plus block-alignment gaps)
  int64_t lane_steps = 0;    // sum over slices of 32 * longest list (FMA lanes issued)
  int64_t nslices = 0;
  int64_t spill = 0;         // spill slots of all bands
  int32_t max_slots = 0;
  int32_t smem_bytes = 0;    // window bytes of the largest band (rk columns)
  int4* band = nullptr;          // nb: {r0, own rows, spill rows, first spill slot}
  int32_t* band_slice = nullptr; // nb+1: slices of band b are [band_slice[b], band_slice[b+1])
  int64_t* slice_off = nullptr;  // nslices: first entry of each slice
  uint32_t* lane = nullptr;      // nslices*32: (list length << 16) | slot
  int32_t* spill_row = nullptr;  // spill: the row of every spill slot
  int32_t* spill_pos = nullptr;  // spill: where the slot's sum goes in the spill buffer, which is
                                 // ordered by receiving row (and by band within a row)
  uint16_t* S = nullptr;         // entries: the slot whose x the entry multiplies
  void* VA = nullptr;            // entries: values for A x (storage type)
  void* VT = nullptr;            // entries: values for A^T x (VA itself when al = au)
  // accumulation (spill -> y): receiving rows ascending; the sums of row acc_row[i] are
  // spill entries [acc_ptr[i], acc_ptr[i+1]), in band order
  int64_t nacc = 0;
  int32_t* acc_row = nullptr;
  int32_t* acc_ptr = nullptr;
  void* spill_buf = nullptr;     // spill values (rk per slot; double or float)
  std::vector<int64_t> band_entries;  // host copy: list entries of each band (batched scheduling)
};

// Arguments of one owner-kernel launch (passed by value).
struct OwnerArgs {
  const int4* band;
  const int32_t* band_slice;
  const int64_t* slice_off;
  const uint32_t* lane;
  const int32_t* spill_row;
  const int32_t* spill_pos;
  const uint16_t* S;
  const void* V;
  const void* x;
  void* y;
  void* spill;
  int32_t ldx;        // row stride of x and y in elements (the pass's columns start at x, y)
  int32_t lds;        // row stride of the spill buffer in elements (the pass's columns start at spill)
  int32_t band_offset;
};

// One tile of a batched launch: band `band` of member `member`, columns [col0, col0 + RK).
struct OwnerTile {
  int32_t member, band, col0, pad;
};

// Host side of the owner plan (owner_plan.cpp). Builds the lists of the bands of `part`
// (split further while a window of rk columns of `slot_bytes` bytes each would exceed
// `budget` bytes or 65,535 slots), the accumulation map, and uploads them; values are
// gathered on the device from al / au / ad (storage type of vbytes bytes per value).
// Returns CSRC_ERR_NOT_PARTITIONED when a list is longer than 65,535 entries or a single
// row's window does not fit.
// The handle's al / au / ad are of `in_bytes` bytes per value (8 = double, 4 = float, 2 = BF16);
// the lists hold the values of `mode` (a double is rounded to nearest-even when the mode's
// values are narrower).
csrc_status build_owner_plan(int32_t n, int64_t h, const std::vector<int32_t>& ia, const std::vector<int32_t>& ja,
                             const std::vector<int32_t>& part, int rk, int mode, int budget, int in_bytes,
                             const void* al, const void* au, const void* ad, bool sym, OwnerPlan& out);
void free_owner_plan(OwnerPlan& p);

// Launchers (owner.cu, owner_batch.cu).
cudaError_t prepare_owner_kernels();
// out_a[e] / out_t[e] = the value of entry e for A x / A^T x, from its source code
// (k << 2 | kind, kind 0 = ad[k], 1 = al[k], 2 = au[k]); sources of in_bytes bytes per value,
// outputs of out_bytes (8 -> 4: round to nearest FP32; 8 -> 2: round to nearest-even BF16 directly).
cudaError_t launch_owner_gather(int in_bytes, int out_bytes, const int64_t* code, int64_t count, const void* al,
                                const void* au, const void* ad, void* out_a, void* out_t, cudaStream_t s);
cudaError_t launch_owner(int mode, int rk, const OwnerArgs& a, int nbands, int smem, cudaStream_t s);
// Batched: one CTA per tile, member arguments on the device.
cudaError_t prepare_owner_batch_kernels();
cudaError_t launch_owner_batch(int mode, int rk, const OwnerArgs* members, const OwnerTile* tiles, int ntiles,
                               int smem, cudaStream_t s);
// y[row, c] += the row's spilled sums, for the owner plans' row-ordered spill buffers: y of the
// mode's vector type, spill of its accumulation type (rk columns, row stride ldx in y and rk in spill).
cudaError_t launch_owner_accumulate(int mode, int64_t nacc, int rk, int ldx, const int32_t* acc_row,
                                    const int32_t* acc_ptr, const void* spill, void* y, cudaStream_t s);
// Accumulation arguments of one member of a batch (row-ordered spill buffer, rk columns).
struct OwnerAccArgs {
  const int32_t* acc_row;
  const int32_t* acc_ptr;
  const void* spill;
  void* y;
  int32_t rk;
  int32_t ldx;
};
// Every member's accumulation in one launch: members of one mode; offs[m] = first (row, column)
// item of member m (offs[nmembers] = total items).
cudaError_t launch_owner_batch_accumulate(int mode, const OwnerAccArgs* members, const int64_t* offs,
                                          int nmembers, int64_t total, cudaStream_t s);

// Arguments of the band kernels (passed by value).
struct BandArgs {
  int32_t n;
  const int32_t* ia;
  const int32_t* ja;  // columns; window slots (DevPlan::jslot) for the window strategy's
                      // plain-row kernels
  const uint16_t* ja16;  // 16-bit window slots in place of ja for those kernels (index
                         // compression), else null
  const int32_t* band_stage;
  const int32_t* stage_k;
  const int32_t* stage_r;
  int32_t group;  // lanes per row
  int32_t x_bulk; // x is 16-byte aligned: window pages of x are fetched with bulk copies
  int32_t ldx;    // row stride of x and y in elements (1 for a single vector)
  int32_t rk;     // columns per pass (1, 2, 4 or 8); x and y point at the pass's first column
  int32_t block;  // rows per unit (node blocks), 1 for plain rows
  const void* al;  // gathered values  (au for the transpose)
  const void* au;  // scattered values (al for the transpose); pre-split double-float
                   // pairs for the MODE_DF kernels that read window slots
  const void* ad;
  const void* x;
  void* y;
  const int32_t* band_row;
  const int32_t* band_plo;
  const int32_t* band_ntab;
  const int32_t* band_wp;
  const int32_t* wpage;
  const int32_t* wbase;
  const uint64_t* wmask;
  void* spill;
  int32_t* status;  // device status word (bit flags)
  int32_t band_offset;
};

// Tuning cache (tune.cpp): CSRC_TUNE = off / cache (default) / full, the cache file, and the
// pattern hash of a matrix.
enum { TUNE_OFF = 0, TUNE_CACHE = 1, TUNE_FULL = 2 };
int tune_mode();
std::string tune_cache_path();
uint64_t pattern_hash(int32_t n, const std::vector<int32_t>& ia, const std::vector<int32_t>& ja);

// Device status bits (OR-ed by kernels, read by csrc_get_last_device_error).
enum : int32_t { DEV_RANGE = 1, DEV_TIMEOUT = 2, DEV_BOUNDS = 4 };

// Launchers (kernels.cu). All return cudaGetLastError() of their launch.
cudaError_t launch_band(Arith arith, int storage, bool atomic_flush, const BandArgs& a, int nbands,
                        int smem_bytes, cudaStream_t s);
cudaError_t launch_accumulate(Arith arith, int storage, int64_t nacc, int rk, int ldx, const int32_t* acc_row,
                              const int32_t* acc_ptr, const int32_t* acc_src, const void* spill, void* y,
                              cudaStream_t s);
// out[k] = the double-float split (df32.cuh) of v[k], k < count: the scatter operand of the
// MODE_DF window kernels, split once when the handle is created.
cudaError_t launch_split_df(const double* v, void* out, int64_t count, cudaStream_t s);
// The auxiliary CSR of a rectangular matrix (rect.cu): y[rows[t]] += row t of A_R times x,
// and y[n + c] = column c of A_R times x (column-major copy), FP64 for FP64 storage.
cudaError_t launch_rect_rows(int storage, int32_t nrows, const int32_t* rows, const int32_t* ptr, const int32_t* col,
                             const void* val, const void* x, void* y, cudaStream_t s);
cudaError_t launch_rect_cols(int storage, int32_t ncols, int32_t n, const int32_t* ptr, const int32_t* row,
                             const void* val, const void* x, void* y, cudaStream_t s);
// Vector passes of the BiCG solver (solver.cu). SOLVER_DOT: out[0] = (v0, v1).
// SOLVER_INIT: w0 = w1 = w2 = w3 = v0 - v1, out = {(w0, w0), (v0, v0)}.
// SOLVER_UPDATE1: w0 += s v0; w1 -= s v1; w2 -= s v2; out = {(w1, w1), (w1, w2)}.
// SOLVER_UPDATE2: w0 = v0 + s w0; w1 = v1 + s w1. Vectors of n doubles (fp64) or floats;
// partial holds 2 * nblocks doubles, out 2; sums are FP64 and in a fixed order.
enum SolverOp : int { SOLVER_DOT = 0, SOLVER_INIT = 1, SOLVER_UPDATE1 = 2, SOLVER_UPDATE2 = 3 };
int solver_blocks(int sms);
cudaError_t launch_solver_op(int op, bool fp64, int64_t n, int nblocks, double scalar, const void* v0, const void* v1,
                             const void* v2, void* w0, void* w1, void* w2, void* w3, double* partial, double* out,
                             cudaStream_t s);
// Bounded-wait self-test (kernels.cu): one CTA waits `limit` cycles on an mbarrier that
// nothing arrives at and ORs DEV_TIMEOUT into *status.
cudaError_t launch_wait_probe(long long limit, int32_t* status, cudaStream_t s);
cudaError_t prepare_band_kernels();
cudaError_t prepare_band_kernels_block();
cudaError_t launch_band_block(Arith arith, int storage, const BandArgs& a, int nbands, int smem, cudaStream_t s);

// Product into caller-provided spill memory, allocating nothing (api.cpp; used by noalloc.cu).
int32_t handle_device(const csrc_matrix_s* h);
csrc_status spmv_external_spill(csrc_matrix_s* h, const void* x, void* y, bool transpose, void* spill,
                                int64_t capacity, cudaStream_t s);

// Colouring (color.cu).
cudaError_t launch_jp_round(int32_t n, const int32_t* ia, const int32_t* ja, const int32_t* up_ptr,
                            const int32_t* up, uint64_t seed, int32_t round, int32_t* state,
                            int32_t* uncolored, cudaStream_t s);
// Colour-ordered product (color.cu): every class in one cooperative launch with grid barriers
// (barrier: a zeroed counter), `group` lanes per row. A barrier wait that runs out sets
// DEV_TIMEOUT in *status.
int color_group(double mean_pairs);
// The class-ordered copy of the lists: for the n rows of the class order, desc[t] = {i, k0, k1,
// ia[i]}; pairs ia[i] .. ia[i+1] - 1 of ja, al and au (au may be null) go to k0 .. k1 - 1 of
// cja, cal and cau. vbytes: 8, 4 or 2.
cudaError_t launch_color_copy(int vbytes, const int4* desc, int32_t n, const int32_t* ja, const void* al,
                              const void* au, int32_t* cja, void* cal, void* cau, cudaStream_t s);
// The colour-ordered product over the class-ordered copy (desc, ja, al = gathered values, au =
// scattered values).
cudaError_t launch_color_spmv(int storage, int group, int32_t ncolors, const int32_t* color_ptr, const int4* desc,
                              const int32_t* ja, const void* al, const void* au, const void* ad, const void* x,
                              void* y, unsigned* barrier, int32_t* status, cudaStream_t s);

}  // namespace csrc
