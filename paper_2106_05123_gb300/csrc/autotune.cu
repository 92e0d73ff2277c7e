// Autotuner: picks the tile shape, bucket count per level and base-case size of a call shape by
// timing candidates on a scratch copy of the caller's input, and records the winner so that
// later calls of the same shape class that pass no tuning use it.
//
// Shape class: (segmented or not, key type, payload width, ceil(log2 n), ceil(log2 segments)).
// Candidates:
//   plain path     : log2_buckets in {6, 7, 8, 9} x base_capacity in {4096, 8192, 16384}
//   segmented path : seg_block (persistent CTA size, which is also the size up to which a
//                    segment is sorted in shared memory: 256 -> 4096 keys, 512 -> 8192 keys for
//                    4-byte keys) in {256, 512} x log2_buckets of its one-CTA partitions in
//                    {4, 5, 6, 7, 8}
// Each candidate runs once untimed (this also captures the segmented path's CUDA graph), then
// twice timed with CUDA events on the caller's stream; the candidate's time is the faster run.
// The input is copied into the scratch area before every run and is never modified.

#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sort_api.h"

namespace {

using ShapeKey = std::array<int64_t, 5>;

std::mutex g_tune_mu;
std::map<ShapeKey, pdq_tuning>& tune_table() {
  static std::map<ShapeKey, pdq_tuning> t;
  return t;
}

int ceil_log2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

ShapeKey shape_of(bool seg, int dt, int vb, int64_t n, int64_t nseg) {
  return ShapeKey{seg ? 1 : 0, dt, vb, ceil_log2(n < 1 ? 1 : n), seg ? ceil_log2(nseg < 1 ? 1 : nseg) : 0};
}

int key_bytes_of(int dt) {
  switch (dt) {
    case PDQ_I32: case PDQ_U32: case PDQ_F32: return 4;
    case PDQ_I64: case PDQ_U64: case PDQ_I32I32: case PDQ_F32U32: return 8;
    default: return 0;
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

namespace pdq {

bool autotune_lookup(bool seg, int dt, int vb, int64_t n, int64_t nseg, pdq_tuning* out) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto& t = tune_table();
  auto it = t.find(shape_of(seg, dt, vb, n, nseg));
  if (it == t.end()) return false;
  *out = it->second;
  return true;
}

}  // namespace pdq

using pdq::set_error;

extern "C" {

size_t pdq_autotune_scratch_bytes(int64_t n, int64_t num_segments, pdq_dtype key_dtype, int value_bytes) {
  const int kb = key_bytes_of(key_dtype);
  if (!kb || n < 0 || num_segments < 0 || (value_bytes != 0 && value_bytes != 4 && value_bytes != 8)) return 0;
  const size_t ws = pdq_workspace_bytes(n, num_segments, key_dtype, value_bytes);
  if (!ws) return 0;
  return align256((size_t)n * kb) + align256((size_t)n * value_bytes) + ws;
}

int pdq_autotune(const void* d_keys, const void* d_vals, int value_bytes, const int64_t* d_offsets,
                 int64_t num_segments, int64_t n, pdq_dtype key_dtype, void* d_scratch, size_t scratch_bytes,
                 void* cuda_stream, pdq_tuning* best, float* best_ms) {
  const int kb = key_bytes_of(key_dtype);
  if (!kb) return set_error(PDQ_ERR_DTYPE, "unknown key dtype");
  if (n < 2 || n >= (int64_t(1) << 32)) return set_error(PDQ_ERR_ARG, "autotune needs 2 <= n < 2^32");
  if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8)
    return set_error(PDQ_ERR_ARG, "value_bytes must be 0, 4 or 8");
  if (!d_keys || (value_bytes && !d_vals)) return set_error(PDQ_ERR_ARG, "null key or value pointer");
  const bool seg = num_segments > 0;
  if (seg && !d_offsets) return set_error(PDQ_ERR_ARG, "segmented autotune needs offsets");
  const size_t need = pdq_autotune_scratch_bytes(n, seg ? num_segments : 0, key_dtype, value_bytes);
  if (!d_scratch || ((uintptr_t)d_scratch % 256) || scratch_bytes < need)
    return set_error(PDQ_ERR_WORKSPACE, "autotune scratch null, misaligned or smaller than pdq_autotune_scratch_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  char* base = static_cast<char*>(d_scratch);
  void* keys = base;
  void* vals = value_bytes ? base + align256((size_t)n * kb) : nullptr;
  void* ws = base + align256((size_t)n * kb) + align256((size_t)n * value_bytes);
  const size_t ws_bytes = scratch_bytes - (size_t)((char*)ws - base);

  std::vector<pdq_tuning> cands;
  if (seg) {
    for (int blk : {256, 512})
      for (int lb : {4, 5, 6, 7, 8}) {
        pdq_tuning t;
        std::memset(&t, 0, sizeof(t));
        t.seg_block = blk;
        t.log2_buckets = lb;
        cands.push_back(t);
      }
  } else {
    for (int lb : {6, 7, 8, 9})
      for (int cap : {4096, 8192, 16384}) {
        pdq_tuning t;
        std::memset(&t, 0, sizeof(t));
        t.log2_buckets = lb;
        t.base_capacity = cap;
        cands.push_back(t);
      }
  }

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_error(PDQ_ERR_CUDA, "autotune: cudaEventCreate failed");
  }
  auto run_once = [&](const pdq_tuning& t, float* ms) -> int {
    cudaError_t e = cudaMemcpyAsync(keys, d_keys, (size_t)n * kb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && value_bytes)
      e = cudaMemcpyAsync(vals, d_vals, (size_t)n * value_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("autotune copy: ") + cudaGetErrorString(e));
    cudaEventRecord(e0, s);
    int rc;
    if (seg)
      rc = pdq_sort_segmented(keys, vals, value_bytes, d_offsets, num_segments, n, key_dtype, ws, ws_bytes, s, &t,
                              nullptr);
    else if (value_bytes)
      rc = pdq_sort_pairs(keys, vals, value_bytes, n, key_dtype, ws, ws_bytes, s, &t, nullptr);
    else
      rc = pdq_sort_keys(keys, n, key_dtype, ws, ws_bytes, s, &t, nullptr);
    if (rc) return rc;
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("autotune sync: ") + cudaGetErrorString(e));
    cudaEventElapsedTime(ms, e0, e1);
    return PDQ_OK;
  };
  int rc = PDQ_OK;
  int best_i = -1;
  float best_t = 0.f;
  for (size_t i = 0; i < cands.size() && !rc; ++i) {
    float warm = 0.f, t1 = 0.f, t2 = 0.f;
    rc = run_once(cands[i], &warm);
    if (!rc) rc = run_once(cands[i], &t1);
    if (!rc) rc = run_once(cands[i], &t2);
    if (rc) break;
    const float t = t1 < t2 ? t1 : t2;
    if (best_i < 0 || t < best_t) {
      best_i = (int)i;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_table()[shape_of(seg, key_dtype, value_bytes, n, num_segments)] = cands[best_i];
  }
  if (best) *best = cands[best_i];
  if (best_ms) *best_ms = best_t;
  return PDQ_OK;
}

int pdq_autotune_lookup(int64_t n, int64_t num_segments, pdq_dtype key_dtype, int value_bytes, pdq_tuning* out) {
  pdq_tuning t;
  if (!pdq::autotune_lookup(num_segments > 0, key_dtype, value_bytes, n, num_segments, &t)) return 0;
  if (out) *out = t;
  return 1;
}

void pdq_autotune_reset(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  tune_table().clear();
}

}  // extern "C"
