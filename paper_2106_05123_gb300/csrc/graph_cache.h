// Cache of instantiated CUDA graphs of the segmented path, one per distinct call shape.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

namespace pdq {

struct GraphKey {
  int kt, vb, block, logb, oversample, bad0, inject;
  uint64_t wait_ns;
  const void *keys, *vals, *offsets, *ws;
  int64_t nseg, n;
  bool operator<(const GraphKey& o) const {
    return std::tie(kt, vb, block, logb, oversample, bad0, inject, wait_ns, keys, vals, offsets, ws, nseg, n) <
           std::tie(o.kt, o.vb, o.block, o.logb, o.oversample, o.bad0, o.inject, o.wait_ns, o.keys, o.vals,
                    o.offsets, o.ws, o.nseg, o.n);
  }
};

struct GraphCache {
  std::mutex mu;
  std::map<GraphKey, cudaGraphExec_t> execs;
  cudaStream_t capture_stream = nullptr;
};

GraphCache& graph_cache();

}  // namespace pdq
