// pdq_sort_keys_noalloc: the keys-only sort for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or ask anyone else to): code that lives inside a
// framework whose device memory is owned entirely by its own caching allocator, plug-ins that
// are handed a fixed memory budget, and latency-sensitive loops where cudaMalloc / cudaFree
// would synchronise the whole device.  They pass only their keys; the sort's scratch (its
// temporary key buffer, counters and work lists) comes from one file-scope device array.
//
// The array is a fixed 64 MiB per GPU and lives as long as the process: every GPU that loads
// this part of the library holds it until exit.  64 MiB covers the workspace of up to 2^20
// keys of any key type; larger calls are rejected with PDQ_ERR_ARG.  All calls on a device
// share the one array, which keeps the last call's contents; the sort resets every counter it
// reads at the start of each pass, so stale contents are harmless, but calls that overlap on
// the GPU (two streams, or two host threads) race on the array and must not be issued.
//
// Set-up: the first call on each device, with that device current, asks the runtime for the
// device address of the array (cudaGetSymbolAddress) and caches it; issue that first call
// before any stream capture.  In host code the array's name is only a host-side stand-in, so
// the kernels always receive the looked-up device address.

#include <cstring>
#include <mutex>
#include <string>

#include "sort_api.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

using pdq::set_error;

extern "C" int pdq_sort_keys_noalloc(void* d_keys, int64_t n, pdq_dtype key_dtype, void* cuda_stream,
                                     pdq_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const size_t need = pdq_workspace_bytes(n < 0 ? 0 : n, 0, key_dtype, 0);
  if (need == 0) return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  if (n < 0) return set_error(PDQ_ERR_ARG, "n must be >= 0");
  if (n <= 1) return pdq_sort_keys(d_keys, n, key_dtype, nullptr, 0, cuda_stream, nullptr, stats);
  if (need > kNoAllocScratchBytes) {
    return set_error(PDQ_ERR_ARG, "pdq_sort_keys_noalloc: n = " + std::to_string(n) + " needs " +
                                      std::to_string(need) + " bytes of scratch, above its fixed " +
                                      std::to_string(kNoAllocScratchBytes) +
                                      " (enough for up to 2^20 keys); use pdq_sort_keys with a workspace");
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(PDQ_ERR_ARG, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr)
        return set_error(PDQ_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  return pdq_sort_keys(d_keys, n, key_dtype, scratch, kNoAllocScratchBytes, cuda_stream, nullptr, stats);
}
