// Shared definitions of the GB300 sort library: key encoding, descriptors, launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pdq.h"

namespace pdq {

// ------------------------------------------------------------------ limits and defaults
constexpr int kLogBMax = 9;                  // at most 512 buckets (+ equality buckets) a level
constexpr int kBMax = 1 << kLogBMax;
constexpr int kBinsMax = 2 * kBMax;          // bin 2b: keys strictly inside bucket b; 2b+1: == splitter b
constexpr int kDefaultLogB = 8;
constexpr int kDefaultOversample = 16;
constexpr int kMaxSamples = 4096;            // samples sorted in one CTA for splitter selection
constexpr int kBaseCapMax = 16384;           // largest bucket the shared-memory base sort takes
constexpr int kBaseCapMin = 256;             // smallest base capacity a caller may ask for
constexpr int kChunkMin = 1 << 14;           // smallest chunk of a task one CTA classifies
constexpr int kTaskRound = 512;              // tasks split per launch round
constexpr int kBaseClasses = 5;              // base-sort size classes: 1K, 2K, 4K, 8K, 16K elements

enum Buf : int { kBufKeys = 0, kBufTmp = 1 };

// A bucket that still has to be split (one distribution level).
struct Task {
  int64_t begin;      // first element (same index in the key buffer and the temp buffer)
  int64_t size;
  int32_t buf;        // where the elements are now (kBufKeys / kBufTmp)
  int32_t enc;        // 1: stored as ordered-unsigned codes; 0: raw user keys
  int32_t bad_left;   // bad-split budget of this subtree (Sec. 4.1)
  int32_t attempt;    // how many times this range was split already (sampling seed)
};

// A finished-or-final piece of work: base sort, copy to the key buffer, or fallback.
struct Item {
  int64_t begin;
  uint32_t size;
  uint16_t buf;
  uint16_t enc;
};

// One chunk of a task, classified by one CTA.
struct Chunk {
  int64_t begin;      // absolute first element
  int32_t size;
  int32_t task;       // index of the task in the round
};

// Base-sort lists can be split by position into this many groups (host-buffer sorts of large
// arrays: each group's range goes back to the host as soon as its base sorts are done).
constexpr int kOutGroups = 8;

// Device-side counters written by the bookkeeping kernel.
struct Counters {
  unsigned long long n_next;        // tasks for the next level
  unsigned long long n_base[kOutGroups][kBaseClasses];  // base-sort items per position group and size class
  unsigned long long n_copy;        // items to copy temp -> keys
  unsigned long long n_fallback;    // items for the merge-path fallback
  unsigned long long equal_buckets;
  unsigned long long bad_splits;
  unsigned long long overflow;      // a list would have exceeded its capacity
  unsigned long long base_elems;    // elements in the base-sort list
  unsigned long long copy_elems;    // elements in the copy list
  unsigned long long timeout;       // a bounded device-side wait gave up
  unsigned long long probe[8];      // probe results: descents, ascents, min code, max code
};

// Capacities of the bookkeeping lists (passed by value to the bookkeeping kernel).
struct ListCaps {
  int64_t base_off[kBaseClasses];
  int64_t base_cap[kBaseClasses];
  int64_t task_cap, copy_cap, fb_cap;
  // position groups of the base lists: an item starting at element b belongs to group
  // floor((b - group_first) * groups / group_n); group g's lists start group_stride items after
  // group g - 1's
  int groups;
  int64_t group_stride, group_first, group_n;
};

// ------------------------------------------------------------------ key encoding (ordered unsigned)
// Every supported key maps bijectively to an unsigned integer whose unsigned order is the key
// order: signed integers flip the sign bit; float32 flips the sign bit of positive numbers and
// all bits of negative ones (this realises IEEE 754 totalOrder on bit patterns); unsigned keys
// are unchanged.  Kernels compare codes only and decode on the final store.
template <int KT> struct Key;
template <> struct Key<PDQ_U32> {
  using U = uint32_t;
  static __host__ __device__ __forceinline__ U enc(U x) { return x; }
  static __host__ __device__ __forceinline__ U dec(U x) { return x; }
};
template <> struct Key<PDQ_I32> {
  using U = uint32_t;
  static __host__ __device__ __forceinline__ U enc(U x) { return x ^ 0x80000000u; }
  static __host__ __device__ __forceinline__ U dec(U x) { return x ^ 0x80000000u; }
};
template <> struct Key<PDQ_F32> {
  using U = uint32_t;
  static __host__ __device__ __forceinline__ U enc(U x) {
    return x ^ ((uint32_t)((int32_t)x >> 31) | 0x80000000u);
  }
  static __host__ __device__ __forceinline__ U dec(U x) {
    return x ^ (((x >> 31) - 1u) | 0x80000000u);
  }
};
template <> struct Key<PDQ_U64> {
  using U = uint64_t;
  static __host__ __device__ __forceinline__ U enc(U x) { return x; }
  static __host__ __device__ __forceinline__ U dec(U x) { return x; }
};
template <> struct Key<PDQ_I64> {
  using U = uint64_t;
  static __host__ __device__ __forceinline__ U enc(U x) { return x ^ 0x8000000000000000ull; }
  static __host__ __device__ __forceinline__ U dec(U x) { return x ^ 0x8000000000000000ull; }
};
// Composite keys: an 8-byte record {field 0, field 1} read as one little-endian word (field 0 in
// the low half).  The code puts field 0's code in the high half and field 1's in the low half, so
// the unsigned order of codes is the lexicographic order of the records.
template <> struct Key<PDQ_I32I32> {
  using U = uint64_t;
  static __host__ __device__ __forceinline__ U enc(U x) {
    return ((U)(Key<PDQ_I32>::enc((uint32_t)x)) << 32) | Key<PDQ_I32>::enc((uint32_t)(x >> 32));
  }
  static __host__ __device__ __forceinline__ U dec(U c) {
    return (U)Key<PDQ_I32>::dec((uint32_t)(c >> 32)) | ((U)Key<PDQ_I32>::dec((uint32_t)c) << 32);
  }
};
template <> struct Key<PDQ_F32U32> {
  using U = uint64_t;
  static __host__ __device__ __forceinline__ U enc(U x) {
    return ((U)(Key<PDQ_F32>::enc((uint32_t)x)) << 32) | (x >> 32);
  }
  static __host__ __device__ __forceinline__ U dec(U c) {
    return (U)Key<PDQ_F32>::dec((uint32_t)(c >> 32)) | ((c & 0xFFFFFFFFull) << 32);
  }
};

// Value payload: VB = 0 (none), 4 or 8 bytes.
template <int VB> struct Val { using T = uint32_t; };
template <> struct Val<8> { using T = uint64_t; };

// ------------------------------------------------------------------ small device helpers
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014): a counter-based hash for sample positions.
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ int ilog2_floor(uint64_t x) {
  int r = 0;
  while (x > 1) { x >>= 1; ++r; }
  return r;
}

// ------------------------------------------------------------------ host-side launch bookkeeping
void note_launch(const char* name, cudaStream_t s, double bytes);    // before a launch
void note_launch_end(const char* name, cudaStream_t s);              // after a launch
int64_t launches_so_far();
void note_launch_count(int extra);                                   // kernels inside a graph launch

// Streams and events that let the base-sort size classes of one level run concurrently: the
// calling stream forks to one auxiliary stream per class and joins them again.  One set per host
// thread and device, created on first use (nullptr if creation failed: run serially).
struct AuxStreams {
  cudaStream_t s[kBaseClasses];
  cudaEvent_t fork;
  cudaEvent_t join[kBaseClasses];
  cudaStream_t copy;        // device-to-host copies of final ranges (host-buffer form)
  cudaEvent_t ready, copied;
};
AuxStreams* aux_streams();
// Pinned host staging of the calling thread (portable across devices), at least `bytes` long;
// `which` selects one of two independent buffers (0: uploads, 1: counter read-backs).  A
// caller must not reuse a buffer before the copies from or into it have completed.  Null if
// pinned memory cannot be had (callers then use pageable memory).
void* host_staging(int which, size_t bytes);
bool profiling_enabled();  // per-kernel event timing is on: launches stay serial on their stream

struct LaunchScope {
  const char* name;
  cudaStream_t s;
  LaunchScope(const char* n, cudaStream_t st, double bytes) : name(n), s(st) {
    note_launch(n, st, bytes);
  }
  ~LaunchScope() { note_launch_end(name, s); }
};

}  // namespace pdq
