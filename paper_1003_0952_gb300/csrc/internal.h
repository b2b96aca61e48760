// Internal declarations shared by the host library (api.cpp) and the kernels.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime_api.h>

#include "../../include/csrc.h"

namespace csrc {

// Rows per window page (page table granularity, one 64-bit spill mask per page).
constexpr int kPageShift = 6;
constexpr int kPageRows = 1 << kPageShift;
constexpr int kBandThreads = 512;
// Pairs per block of the row-start metadata (blk_row[g] = row holding pair g << kBlockShift).
constexpr int kBlockShift = 7;

// Arithmetic of a product.
enum Arith : int32_t { ARITH_DF32 = 0, ARITH_F64 = 1, ARITH_F32 = 2 };

// Device arrays of one execution plan of the window / atomic strategies.
// A plan is a list of row bands. Band b covers rows [band_row[b], band_row[b+1]).
// Its shared-memory window is a set of pages of kPageRows rows (wpage[band_wp[b]..band_wp[b+1])),
// indexed through a page table that spans pages [band_plo[b], band_plo[b] + band_ntab[b]).
struct DevPlan {
  int32_t nb = 0;
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
  int32_t smem_bytes = 0;
  int64_t total_pages = 0;
};

// Arguments of the band kernels (passed by value).
struct BandArgs {
  int32_t n;
  const int32_t* ia;
  const int32_t* ja;
  const int32_t* blk_row;  // ceil(h / 128) + 1 entries
  const void* al;  // gathered values  (au for the transpose)
  const void* au;  // scattered values (al for the transpose)
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

// Device status bits (OR-ed by kernels, read by csrc_get_last_device_error).
enum : int32_t { DEV_RANGE = 1, DEV_TIMEOUT = 2, DEV_BOUNDS = 4 };

// Launchers (kernels.cu). All return cudaGetLastError() of their launch.
cudaError_t launch_band(Arith arith, int storage, bool atomic_flush, const BandArgs& a, int nbands,
                        int smem_bytes, cudaStream_t s);
cudaError_t launch_accumulate(Arith arith, int storage, int64_t nacc, const int32_t* acc_row,
                              const int32_t* acc_ptr, const int32_t* acc_src, const void* spill, void* y,
                              cudaStream_t s);
cudaError_t prepare_band_kernels(int max_smem_bytes);

// Product into caller-provided spill memory, allocating nothing (api.cpp; used by noalloc.cu).
int32_t handle_device(const csrc_matrix_s* h);
csrc_status spmv_external_spill(csrc_matrix_s* h, const void* x, void* y, bool transpose, void* spill,
                                int64_t capacity, cudaStream_t s);

// Colouring (color.cu).
cudaError_t launch_jp_round(int32_t n, const int32_t* ia, const int32_t* ja, const int32_t* up_ptr,
                            const int32_t* up, uint64_t seed, int32_t round, int32_t* state,
                            int32_t* uncolored, cudaStream_t s);
cudaError_t launch_color_spmv(Arith arith, int storage, int32_t nrows, const int32_t* rows, const int32_t* ia,
                              const int32_t* ja, const void* al, const void* au, const void* ad, const void* x,
                              void* y, cudaStream_t s);

}  // namespace csrc
