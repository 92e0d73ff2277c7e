// C ABI of the library (see include/pdq.h): argument checks, dtype dispatch, error strings,
// launch counting and the optional per-kernel event timing used for measurement.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "graph_cache.h"
#include "sort_api.h"

namespace pdq {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

// ------------------------------------------------------------------ launch accounting
static std::atomic<int64_t> g_launches{0};
static std::atomic<bool> g_profile{false};

struct ProfEntry {
  double ms = 0.0;
  int64_t launches = 0;
  double bytes = 0.0;
};
struct Pending {
  std::string name;
  cudaEvent_t e0, e1;
  double bytes;
};
static std::mutex g_prof_mu;
static std::map<std::string, ProfEntry> g_prof;
static std::vector<Pending> g_pending;
static thread_local std::vector<Pending> t_open;

void note_launch(const char* name, cudaStream_t s, double bytes) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  nvtxRangePushA(name);  // a named range per launch for timeline tools (no-op when none attached)
  if (!g_profile.load(std::memory_order_relaxed)) return;
  Pending p;
  p.name = name;
  p.bytes = bytes;
  cudaEventCreate(&p.e0);
  cudaEventCreate(&p.e1);
  cudaEventRecord(p.e0, s);
  t_open.push_back(p);
}

void note_launch_end(const char* name, cudaStream_t s) {
  nvtxRangePop();
  if (t_open.empty()) return;
  Pending p = t_open.back();
  t_open.pop_back();
  (void)name;
  cudaEventRecord(p.e1, s);
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_pending.push_back(p);
}

int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void note_launch_count(int extra) { g_launches.fetch_add(extra, std::memory_order_relaxed); }

bool profiling_enabled() { return g_profile.load(std::memory_order_relaxed); }

AuxStreams* aux_streams() {
  constexpr int kMaxDev = 64;
  thread_local AuxStreams* sets[kMaxDev] = {};
  thread_local bool failed[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || failed[dev]) return nullptr;
  if (!sets[dev]) {
    AuxStreams* a = new AuxStreams();
    bool ok = cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&a->ready, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&a->copied, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&a->copy, cudaStreamNonBlocking) == cudaSuccess;
    for (int c = 0; c < kBaseClasses && ok; ++c) {
      ok = cudaStreamCreateWithFlags(&a->s[c], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&a->join[c], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      failed[dev] = true;
      return nullptr;  // (the partial set is left to the context's teardown)
    }
    sets[dev] = a;
  }
  return sets[dev];
}

void* host_staging(int which, size_t bytes) {
  struct Buf {  // kept until exit, like the auxiliary streams
    void* p = nullptr;
    size_t n = 0;
  };
  thread_local Buf bufs[2];
  if (which < 0 || which > 1) return nullptr;
  Buf& b = bufs[which];
  if (b.n < bytes) {
    // grow geometrically: each reallocation frees pinned memory, which synchronises the device
    const size_t want = std::max<size_t>(bytes, std::max<size_t>(64 * 1024, 2 * b.n));
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.n = 0;
    if (cudaHostAlloc(&b.p, want, cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return nullptr;
    }
    b.n = want;
  }
  return b.p;
}

GraphCache& graph_cache() {
  static GraphCache* gc = new GraphCache();  // lives until exit (graph objects are host-side)
  return *gc;
}

static void resolve_pending() {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (Pending& p : g_pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.e1);
    cudaEventElapsedTime(&ms, p.e0, p.e1);
    ProfEntry& e = g_prof[p.name];
    e.ms += ms;
    e.launches += 1;
    e.bytes += p.bytes;
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  g_pending.clear();
}

// ------------------------------------------------------------------ dispatch helpers
static int key_bytes(int dt) {
  switch (dt) {
    case PDQ_I32: case PDQ_U32: case PDQ_F32: return 4;
    case PDQ_I64: case PDQ_U64: case PDQ_I32I32: case PDQ_F32U32: return 8;
    default: return 0;
  }
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 148;
  }
  return sms;
}

static int make_tuning(const pdq_tuning* t, Tuning* out) {
  Tuning d;
  d.logb = kDefaultLogB;
  d.oversample = kDefaultOversample;
  d.base_cap = kBaseCapMax;
  d.bad_allowed = 0;
  d.probe = true;
  d.wait_us = 0;
  d.inject_wait = 0;
  d.seg_block = 512;
  d.fixup = true;
  if (t) {
    if (t->log2_buckets) {
      if (t->log2_buckets < 1 || t->log2_buckets > kLogBMax)
        return set_error(PDQ_ERR_ARG, "tuning.log2_buckets out of range 1..9");
      d.logb = t->log2_buckets;
    }
    if (t->oversample) {
      if (t->oversample < 1 || t->oversample > kMaxSamples || (t->oversample & (t->oversample - 1)))
        return set_error(PDQ_ERR_ARG, "tuning.oversample must be a power of two <= 4096");
      d.oversample = t->oversample;
    }
    if (t->base_capacity) {
      const int c = t->base_capacity;
      if (c < kBaseCapMin || c > kBaseCapMax || (c & (c - 1)))
        return set_error(PDQ_ERR_ARG, "tuning.base_capacity must be a power of two in 256..16384");
      d.base_cap = c;
    }
    if (t->bad_allowed) d.bad_allowed = t->bad_allowed;
    if (t->probe < 0) d.probe = false;
    if (t->wait_limit_us < 0) return set_error(PDQ_ERR_ARG, "tuning.wait_limit_us must be >= 0");
    d.wait_us = t->wait_limit_us;
    d.inject_wait = t->inject_wait != 0;
    if (t->seg_block && t->seg_block != 256 && t->seg_block != 512)
      return set_error(PDQ_ERR_ARG, "tuning.seg_block must be 256 or 512");
    if (t->seg_block) d.seg_block = t->seg_block;
    if (t->fixup) d.fixup = t->fixup > 0;
  }
  *out = d;
  return PDQ_OK;
}

template <int VB>
static int dispatch_sort(int dt, const SortArgs& a, pdq_stats* st) {
  switch (dt) {
    case PDQ_I32: return sort_impl<PDQ_I32, VB>(a, st);
    case PDQ_U32: return sort_impl<PDQ_U32, VB>(a, st);
    case PDQ_I64: return sort_impl<PDQ_I64, VB>(a, st);
    case PDQ_U64: return sort_impl<PDQ_U64, VB>(a, st);
    case PDQ_F32: return sort_impl<PDQ_F32, VB>(a, st);
    case PDQ_I32I32: return sort_impl<PDQ_I32I32, VB>(a, st);
    case PDQ_F32U32: return sort_impl<PDQ_F32U32, VB>(a, st);
    default: return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  }
}

template <int VB>
static int dispatch_seg(int dt, const SegArgs& a, pdq_stats* st) {
  switch (dt) {
    case PDQ_I32: return seg_sort_impl<PDQ_I32, VB>(a, st);
    case PDQ_U32: return seg_sort_impl<PDQ_U32, VB>(a, st);
    case PDQ_I64: return seg_sort_impl<PDQ_I64, VB>(a, st);
    case PDQ_U64: return seg_sort_impl<PDQ_U64, VB>(a, st);
    case PDQ_F32: return seg_sort_impl<PDQ_F32, VB>(a, st);
    case PDQ_I32I32: return seg_sort_impl<PDQ_I32I32, VB>(a, st);
    case PDQ_F32U32: return seg_sort_impl<PDQ_F32U32, VB>(a, st);
    default: return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  }
}

template <int VB>
static size_t dispatch_seg_ws(int dt, int64_t n, int64_t nseg) {
  switch (dt) {
    case PDQ_I32: return seg_workspace_bytes_impl<PDQ_I32, VB>(n, nseg);
    case PDQ_U32: return seg_workspace_bytes_impl<PDQ_U32, VB>(n, nseg);
    case PDQ_I64: return seg_workspace_bytes_impl<PDQ_I64, VB>(n, nseg);
    case PDQ_U64: return seg_workspace_bytes_impl<PDQ_U64, VB>(n, nseg);
    case PDQ_F32: return seg_workspace_bytes_impl<PDQ_F32, VB>(n, nseg);
    case PDQ_I32I32: return seg_workspace_bytes_impl<PDQ_I32I32, VB>(n, nseg);
    case PDQ_F32U32: return seg_workspace_bytes_impl<PDQ_F32U32, VB>(n, nseg);
    default: return 0;
  }
}

template <int VB>
static size_t dispatch_ws(int dt, int64_t n) {
  switch (dt) {
    case PDQ_I32: return workspace_bytes_impl<PDQ_I32, VB>(n);
    case PDQ_U32: return workspace_bytes_impl<PDQ_U32, VB>(n);
    case PDQ_I64: return workspace_bytes_impl<PDQ_I64, VB>(n);
    case PDQ_U64: return workspace_bytes_impl<PDQ_U64, VB>(n);
    case PDQ_F32: return workspace_bytes_impl<PDQ_F32, VB>(n);
    case PDQ_I32I32: return workspace_bytes_impl<PDQ_I32I32, VB>(n);
    case PDQ_F32U32: return workspace_bytes_impl<PDQ_F32U32, VB>(n);
    default: return 0;
  }
}

static int sort_common(void* keys, void* vals, int value_bytes, int64_t n, int dt, void* ws,
                       size_t ws_bytes, void* stream, const pdq_tuning* tuning, pdq_stats* stats,
                       void* host_keys = nullptr, void* host_vals = nullptr) {
  g_last_error.clear();
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const int kb = key_bytes(dt);
  if (!kb) return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  if (n < 0 || n >= (int64_t(1) << 32)) return set_error(PDQ_ERR_ARG, "n must be in [0, 2^32)");
  if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8)
    return set_error(PDQ_ERR_ARG, "value_bytes must be 4 or 8");
  if (n <= 1) return PDQ_OK;
  if (!keys || ((uintptr_t)keys % kb)) return set_error(PDQ_ERR_ARG, "keys pointer null or misaligned");
  if (value_bytes && (!vals || ((uintptr_t)vals % value_bytes)))
    return set_error(PDQ_ERR_ARG, "values pointer null or misaligned");
  if (!ws || ((uintptr_t)ws % 256)) return set_error(PDQ_ERR_WORKSPACE, "workspace null or not 256-byte aligned");
  SortArgs a;
  a.keys = keys;
  a.vals = vals;
  a.n = n;
  a.ws = ws;
  a.ws_bytes = ws_bytes;
  a.stream = static_cast<cudaStream_t>(stream);
  a.num_sms = num_sms();
  a.host_keys = host_keys;
  a.host_vals = value_bytes ? host_vals : nullptr;
  pdq_tuning tuned;
  if (!tuning && autotune_lookup(false, dt, value_bytes, n, 0, &tuned)) tuning = &tuned;
  int rc = make_tuning(tuning, &a.tune);
  if (rc) return rc;
  switch (value_bytes) {
    case 0: return dispatch_sort<0>(dt, a, stats);
    case 4: return dispatch_sort<4>(dt, a, stats);
    default: return dispatch_sort<8>(dt, a, stats);
  }
}

}  // namespace pdq

using namespace pdq;

extern "C" {

size_t pdq_workspace_bytes(int64_t n, int64_t num_segments, pdq_dtype key_dtype, int value_bytes) {
  if (n < 0 || num_segments < 0) return 0;
  if (num_segments > 0) {
    switch (value_bytes) {
      case 0: return dispatch_seg_ws<0>(key_dtype, n, num_segments);
      case 4: return dispatch_seg_ws<4>(key_dtype, n, num_segments);
      case 8: return dispatch_seg_ws<8>(key_dtype, n, num_segments);
      default: return 0;
    }
  }
  switch (value_bytes) {
    case 0: return dispatch_ws<0>(key_dtype, n);
    case 4: return dispatch_ws<4>(key_dtype, n);
    case 8: return dispatch_ws<8>(key_dtype, n);
    default: return 0;
  }
}

int pdq_sort_keys(void* d_keys, int64_t n, pdq_dtype key_dtype, void* d_ws, size_t ws_bytes,
                  void* cuda_stream, const pdq_tuning* tuning, pdq_stats* stats) {
  return sort_common(d_keys, nullptr, 0, n, key_dtype, d_ws, ws_bytes, cuda_stream, tuning, stats);
}

int pdq_sort_pairs(void* d_keys, void* d_vals, int value_bytes, int64_t n, pdq_dtype key_dtype,
                   void* d_ws, size_t ws_bytes, void* cuda_stream, const pdq_tuning* tuning,
                   pdq_stats* stats) {
  if (value_bytes != 4 && value_bytes != 8) return set_error(PDQ_ERR_ARG, "value_bytes must be 4 or 8");
  return sort_common(d_keys, d_vals, value_bytes, n, key_dtype, d_ws, ws_bytes, cuda_stream, tuning, stats);
}

int pdq_sort_host(void* h_keys, void* h_vals, int value_bytes, int64_t n, pdq_dtype key_dtype,
                  void* d_keys, void* d_vals, void* d_ws, size_t ws_bytes, void* cuda_stream,
                  const pdq_tuning* tuning, pdq_stats* stats) {
  g_last_error.clear();
  const int kb = key_bytes(key_dtype);
  if (!kb) return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  if (n < 0) return set_error(PDQ_ERR_ARG, "n must be >= 0");
  if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8)
    return set_error(PDQ_ERR_ARG, "value_bytes must be 0, 4 or 8");
  if (n == 0) return PDQ_OK;
  if (!h_keys || !d_keys || (value_bytes && (!h_vals || !d_vals)))
    return set_error(PDQ_ERR_ARG, "null buffer");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemcpyAsync(d_keys, h_keys, (size_t)n * kb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && value_bytes)
    e = cudaMemcpyAsync(d_vals, h_vals, (size_t)n * value_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("H2D: ") + cudaGetErrorString(e));
  // the sort itself copies every range of the result into the host arrays once it is final
  // (n <= 1: nothing to sort, the arrays come back as they went)
  int rc = n <= 1 ? PDQ_OK
                  : sort_common(d_keys, d_vals, value_bytes, n, key_dtype, d_ws, ws_bytes, cuda_stream, tuning,
                                stats, h_keys, h_vals);
  if (rc) return rc;
  if (n <= 1) {
    e = cudaMemcpyAsync(h_keys, d_keys, (size_t)n * kb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && value_bytes)
      e = cudaMemcpyAsync(h_vals, d_vals, (size_t)n * value_bytes, cudaMemcpyDeviceToHost, s);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("D2H: ") + cudaGetErrorString(e));
  return PDQ_OK;
}

int pdq_sort_segmented(void* d_keys, void* d_vals, int value_bytes, const int64_t* d_offsets,
                       int64_t num_segments, int64_t n, pdq_dtype key_dtype, void* d_ws, size_t ws_bytes,
                       void* cuda_stream, const pdq_tuning* tuning, pdq_stats* stats) {
  g_last_error.clear();
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const int kb = key_bytes(key_dtype);
  if (!kb) return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  if (n < 0 || n >= (int64_t(1) << 32) || num_segments < 0)
    return set_error(PDQ_ERR_ARG, "n must be in [0, 2^32) and num_segments >= 0");
  if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8)
    return set_error(PDQ_ERR_ARG, "value_bytes must be 0, 4 or 8");
  if (num_segments == 0 || n <= 1) return PDQ_OK;
  if (!d_offsets || ((uintptr_t)d_offsets % 8)) return set_error(PDQ_ERR_ARG, "offsets pointer null or misaligned");
  if (!d_keys || ((uintptr_t)d_keys % kb)) return set_error(PDQ_ERR_ARG, "keys pointer null or misaligned");
  if (value_bytes && (!d_vals || ((uintptr_t)d_vals % value_bytes)))
    return set_error(PDQ_ERR_ARG, "values pointer null or misaligned");
  if (!d_ws || ((uintptr_t)d_ws % 256)) return set_error(PDQ_ERR_WORKSPACE, "workspace null or not 256-byte aligned");
  SegArgs a;
  a.keys = d_keys;
  a.vals = d_vals;
  a.offsets = d_offsets;
  a.nseg = num_segments;
  a.n = n;
  a.ws = d_ws;
  a.ws_bytes = ws_bytes;
  a.stream = static_cast<cudaStream_t>(cuda_stream);
  a.num_sms = num_sms();
  pdq_tuning tuned;
  if (!tuning && autotune_lookup(true, key_dtype, value_bytes, n, num_segments, &tuned)) tuning = &tuned;
  int rc = make_tuning(tuning, &a.tune);
  if (rc) return rc;
  switch (value_bytes) {
    case 0: return dispatch_seg<0>(key_dtype, a, stats);
    case 4: return dispatch_seg<4>(key_dtype, a, stats);
    default: return dispatch_seg<8>(key_dtype, a, stats);
  }
}

int pdq_sort_keys_learned(void* d_keys, int64_t n, pdq_dtype key_dtype, void* d_ws, size_t ws_bytes,
                          void* cuda_stream, const pdq_tuning* tuning, pdq_stats* stats) {
  g_last_error.clear();
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (key_dtype != PDQ_F32) return set_error(PDQ_ERR_DTYPE, "the learned path sorts float32 keys");
  if (n < 0 || n >= (int64_t(1) << 32)) return set_error(PDQ_ERR_ARG, "n must be in [0, 2^32)");
  if (n <= 1) return PDQ_OK;
  if (!d_keys || ((uintptr_t)d_keys % 4)) return set_error(PDQ_ERR_ARG, "keys pointer null or misaligned");
  if (!d_ws || ((uintptr_t)d_ws % 256)) return set_error(PDQ_ERR_WORKSPACE, "workspace null or not 256-byte aligned");
  if (ws_bytes < learned_workspace_bytes(n)) return set_error(PDQ_ERR_WORKSPACE, "workspace too small");
  SortArgs a;
  a.keys = d_keys;
  a.vals = nullptr;
  a.n = n;
  a.ws = d_ws;
  a.ws_bytes = ws_bytes;
  a.stream = static_cast<cudaStream_t>(cuda_stream);
  a.num_sms = num_sms();
  int rc = make_tuning(tuning, &a.tune);
  if (rc) return rc;
  return learned_sort_f32(a, stats);
}

const char* pdq_last_error(void) { return g_last_error.c_str(); }

int64_t pdq_launch_count(void) { return launches_so_far(); }

void pdq_profile_enable(int on) { g_profile.store(on != 0); }

int pdq_profile_read(char* names, double* total_ms, int64_t* launches, double* bytes, int cap) {
  cudaDeviceSynchronize();
  resolve_pending();
  std::lock_guard<std::mutex> g(g_prof_mu);
  int i = 0;
  for (const auto& kv : g_prof) {
    if (i >= cap) break;
    if (names) {
      std::strncpy(names + 64 * i, kv.first.c_str(), 63);
      names[64 * i + 63] = 0;
    }
    if (total_ms) total_ms[i] = kv.second.ms;
    if (launches) launches[i] = kv.second.launches;
    if (bytes) bytes[i] = kv.second.bytes;
    ++i;
  }
  return (int)g_prof.size();
}

void pdq_profile_reset(void) {
  cudaDeviceSynchronize();
  resolve_pending();
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof.clear();
}

}  // extern "C"
