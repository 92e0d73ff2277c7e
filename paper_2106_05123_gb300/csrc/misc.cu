// Small stand-alone entry points: the in-place reversal exposed through the C ABI.
#include <string>

#include "kernels.cuh"
#include "sort_api.h"

using namespace pdq;

extern "C" int pdq_reverse(void* d_data, int64_t n, int elem_bytes, void* cuda_stream) {
  if (n < 0 || (elem_bytes != 4 && elem_bytes != 8)) return set_error(PDQ_ERR_ARG, "bad n or elem_bytes");
  if (n < 2) return PDQ_OK;
  if (!d_data || ((uintptr_t)d_data % elem_bytes)) return set_error(PDQ_ERR_ARG, "data null or misaligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int threads = 256;
  const int64_t want = (n / 2 + threads - 1) / threads;
  const unsigned blocks = (unsigned)(want < 8192 ? (want < 1 ? 1 : want) : 8192);
  {
    LaunchScope ls("reverse", s, 2.0 * n * elem_bytes);
    if (elem_bytes == 4) reverse_kernel<uint32_t><<<blocks, threads, 0, s>>>(static_cast<uint32_t*>(d_data), n);
    else reverse_kernel<uint64_t><<<blocks, threads, 0, s>>>(static_cast<uint64_t*>(d_data), n);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("reverse: ") + cudaGetErrorString(e));
  return PDQ_OK;
}
