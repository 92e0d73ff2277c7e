// pdq_sort_keys_noalloc: the keys-only sort for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or ask anyone else to): code that lives inside a
// framework whose device memory is owned entirely by its own caching allocator, plug-ins that
// are handed a fixed memory budget, and latency-sensitive loops where cudaMalloc / cudaFree
// would synchronise the whole device.  They pass only their keys; the sort's scratch (its
// temporary key buffer, counters and work lists) comes from one file-scope device array.
//
// The array is a fixed 64 MiB per GPU and lives as long as the process: every GPU that loads
// this part of the library holds it until exit.  The entry point takes at most 2^20 keys of any
// key type (their workspace fits the array); larger calls are rejected with PDQ_ERR_ARG.  All
// calls on a device share the one array, which keeps the last call's contents; the sort resets
// every counter and list length it reads before using it, so stale contents are harmless, but
// calls that overlap on the GPU (two streams, or two host threads) race on the array and must
// not be issued.
//
// Set-up: every call, with the target device current, asks the runtime for the device address
// of the array (cudaGetSymbolAddress) and checks the result.  The first call on a device loads
// the module there, so issue it before any stream capture.  Looking the address up on every call
// (it is cheap once the module is loaded) keeps it valid after a device reset, which may place
// the array elsewhere.  In host code the array's name is only a host-side stand-in, so the
// kernels always receive the looked-up device address.

#include <cstring>
#include <string>

#include "sort_api.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int64_t kNoAllocMaxKeys = int64_t(1) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace

using pdq::set_error;

extern "C" int pdq_sort_keys_noalloc(void* d_keys, int64_t n, pdq_dtype key_dtype, void* cuda_stream,
                                     pdq_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const size_t need = pdq_workspace_bytes(n < 0 ? 0 : n, 0, key_dtype, 0);
  if (need == 0) return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  if (n < 0) return set_error(PDQ_ERR_ARG, "n must be >= 0");
  if (n <= 1) return pdq_sort_keys(d_keys, n, key_dtype, nullptr, 0, cuda_stream, nullptr, stats);
  if (n > kNoAllocMaxKeys || need > kNoAllocScratchBytes) {
    return set_error(PDQ_ERR_ARG, "pdq_sort_keys_noalloc: n = " + std::to_string(n) +
                                      " is above its limit of 2^20 keys (fixed " +
                                      std::to_string(kNoAllocScratchBytes) +
                                      "-byte scratch array); use pdq_sort_keys with a workspace");
  }
  void* scratch = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
  if (e != cudaSuccess || scratch == nullptr)
    return set_error(PDQ_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  return pdq_sort_keys(d_keys, n, key_dtype, scratch, kNoAllocScratchBytes, cuda_stream, nullptr, stats);
}
