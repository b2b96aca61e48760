// csrc_spmv_noalloc: the window-strategy product with its spill buffer in a
// fixed, statically allocated device array instead of memory the handle
// allocates.
//
// Who needs it: callers that may not allocate device memory while they run
// products. Examples are code whose device memory is owned by another
// allocator (a framework's caching pool that has reserved the GPU), and host
// threads that must not block, since cudaMalloc and cudaFree can synchronise
// the device. Such a caller creates and partitions its handles once at
// set-up, and from then on calls only this entry point.
//
// The scratch array lives in this file. Host code cannot use its name as a
// device address (on the host it names a stand-in object), so the address is
// taken once per device with cudaGetSymbolAddress while that device is
// current, and passed to the kernels as a pointer.
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace {

// Spilled partial sums of one product: CSRC_NOALLOC_MAX_SPILL_ENTRIES values
// (doubles for FP64 storage; floats otherwise, which use the first half of the
// array). 16 MiB, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_spill[CSRC_NOALLOC_MAX_SPILL_ENTRIES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_spill on the current device (set up on first use).
csrc_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return CSRC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_spill);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return CSRC_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CSRC_OK;
}

}  // namespace

extern "C" csrc_status csrc_spmv_noalloc(csrc_handle h, const void* x, void* y, int32_t transpose,
                                         cudaStream_t stream) {
  if (!h || !x || !y) return CSRC_ERR_INVALID_ARG;
  const int dev = csrc::handle_device(h);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return CSRC_ERR_CUDA;
  if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return CSRC_ERR_CUDA;
  void* spill = nullptr;
  csrc_status st = scratch_address(dev, &spill);
  // Every spill slot that the accumulation kernel reads is written by the product
  // kernel of the same call, so nothing in the array has to start at zero.
  if (st == CSRC_OK)
    st = csrc::spmv_external_spill(h, x, y, transpose != 0, spill, CSRC_NOALLOC_MAX_SPILL_ENTRIES, stream);
  if (cur != dev) cudaSetDevice(cur);  // the caller's current device, as it was
  return st;
}
