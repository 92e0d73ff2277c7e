// Device kernels of the sort (templates; instantiated per key dtype and payload width).
//
// Data-parallel form of pattern-defeating quicksort (Peters, arXiv 2106.05123):
//   probe_kernel      - descents / ascents / min / max over neighbours: the sorted and
//                       reverse-sorted exits (Sec. 5.2)
//   reverse_kernel    - in-place reversal for non-increasing input (Sec. 5.2)
//   sample_kernel     - splitter selection from a hashed sample, sorted on chip; a
//                       multi-way generalisation of median-of-k pivots (Sec. 2) with fresh
//                       samples per attempt (Sec. 4.2)
//   count_kernel      - branchless classification of every key into 2B bins: bin 2b holds keys
//                       strictly between splitters b-1 and b, bin 2b+1 keys equal to splitter b
//                       (the equal-key rule of Sec. 3); stores every key's bin slot
//   scan_bookkeep_kernel - per task: bucket starts, per-bin cursors the scatter reserves runs
//                       from, then the bookkeeping of the task's children: equal bins are
//                       final; small bins go to the base sort; a bin keeping more than 7/8 of
//                       its parent's non-equal keys is a bad split and decrements the subtree's
//                       counter; at 0 the bin goes to the fallback (Sec. 4.1)
//   scatter_kernel    - streams a tile with its stored bin slots, ranks keys per bin with shared
//                       atomics, stages the tile in shared memory grouped by bin and writes
//                       contiguous runs (the GPU form of block partitioning, Sec. 5.3)
//   base_sort_kernel  - shared-memory sort of a small bucket (Sec. 5.1): all-equal buckets are
//                       copied, narrow code ranges take stable LSD counting passes, wide ones a
//                       register-blocked merge sort
//   copy_plan_kernel, copy_kernel - final buckets left in the temp buffer go home, decoded, in
//                       tiles spread over all such buckets
//   merge_tile_kernel - tiled merge-path merge (the O(n log n) fallback's passes, Sec. 4.1, and
//                       the nearly-sorted fix-up's final merge); merge_pass_kernel serves
//                       passes whose run pairs are shorter than a tile
//   fix_*_kernel      - the nearly-sorted fix-up: mark descents, repair, split (Sec. 5.2's aim)
#pragma once

#include "common.cuh"
#include "tile_pipe.cuh"

namespace pdq {

template <int N>
struct IntC {
  static constexpr int value = N;
};

// ================================================================== reductions
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Identity placement of counters in shared memory.
struct SlotIdentity {
  __device__ __forceinline__ int operator()(int b) const { return b; }
};

// Exclusive scan of nbins counters held in shared memory `in`, result in `out` (may alias);
// counter b lives at in[slot(b)] and its prefix goes to out[slot(b)].  All threads of the block
// must call it.
template <int THREADS, class Slot = SlotIdentity>
__device__ void block_exclusive_scan(const uint32_t* in, uint32_t* out, int nbins,
                                     uint32_t* warp_tmp /* >= THREADS/32 + 1 */, Slot slot = Slot()) {
  const int tid = threadIdx.x;
  const int per = (nbins + THREADS - 1) / THREADS;
  const int lo = tid * per;
  uint32_t sum = 0;
  for (int i = 0; i < per; ++i) {
    const int b = lo + i;
    if (b < nbins) sum += in[slot(b)];
  }
  // inclusive scan of per-thread sums across the block
  const int lane = tid & 31, warp = tid >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = THREADS / 32;
    uint32_t w = lane < NW ? warp_tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) warp_tmp[lane] = w;  // inclusive warp totals
    if (lane == NW - 1) warp_tmp[NW] = w;
  }
  __syncthreads();
  uint32_t run = x - sum + (warp > 0 ? warp_tmp[warp - 1] : 0);  // exclusive prefix of thread
  for (int i = 0; i < per; ++i) {
    const int b = lo + i;
    if (b < nbins) {
      const uint32_t c = in[slot(b)];
      out[slot(b)] = run;
      run += c;
    }
  }
  __syncthreads();
}

// Exclusive block scan of one 32-bit value per thread; *total receives the sum (all threads).
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t* wtmp /* >= THREADS/32 */,
                                                        uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = THREADS / 32;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (NW == 1) {
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
  }
  if (lane == 31) wtmp[warp] = x;
  __syncthreads();
  uint32_t w = lane < NW ? wtmp[lane] : 0u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
    if (lane >= o) w += y;
  }
  *total = __shfl_sync(0xffffffffu, w, NW - 1);
  const uint32_t before = __shfl_sync(0xffffffffu, w, warp > 0 ? warp - 1 : 0);
  __syncthreads();  // wtmp may be reused by the caller
  return x - v + (warp > 0 ? before : 0u);
}

// ================================================================== probe (Sec. 5.2)
// out[0] += #descents (a[i] > a[i+1]), out[1] += #ascents, out[2] = min code, out[3] = max code.
// stride == 1: every neighbour pair of a[0..n).  stride > 1: the sample a[j*stride], j < m.
template <int KT>
__global__ void probe_kernel(const typename Key<KT>::U* __restrict__ a, int64_t n, int64_t stride,
                             int64_t m, unsigned long long* out) {
  using U = typename Key<KT>::U;
  unsigned long long desc = 0, asc = 0;
  U mn = ~U(0), mx = U(0);
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  // eight consecutive sample points per thread and step: nine independent loads in flight
  constexpr int G = 8;
  for (int64_t j0 = gt * G; j0 < m; j0 += gs * G) {
    U v[G + 1];
#pragma unroll
    for (int e = 0; e <= G; ++e) {
      const int64_t j = j0 + e;
      v[e] = j < m ? Key<KT>::enc(__ldg(a + j * stride)) : U(0);
    }
#pragma unroll
    for (int e = 0; e < G; ++e) {
      const int64_t j = j0 + e;
      if (j < m) {
        mn = v[e] < mn ? v[e] : mn;
        mx = v[e] > mx ? v[e] : mx;
        if (j + 1 < m) {
          desc += v[e] > v[e + 1];
          asc += v[e] < v[e + 1];
        }
      }
    }
  }
  (void)n;
  __shared__ unsigned long long s_d[32], s_a[32];
  __shared__ U s_mn[32], s_mx[32];
  desc = warp_sum(desc);
  asc = warp_sum(asc);
  mn = warp_min(mn);
  mx = warp_max(mx);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_d[warp] = desc; s_a[warp] = asc; s_mn[warp] = mn; s_mx[warp] = mx; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    desc = lane < nw ? s_d[lane] : 0;
    asc = lane < nw ? s_a[lane] : 0;
    mn = lane < nw ? s_mn[lane] : ~U(0);
    mx = lane < nw ? s_mx[lane] : U(0);
    desc = warp_sum(desc);
    asc = warp_sum(asc);
    mn = warp_min(mn);
    mx = warp_max(mx);
    if (lane == 0) {
      if (desc) atomicAdd(out + 0, desc);
      if (asc) atomicAdd(out + 1, asc);
      atomicMin(out + 2, (unsigned long long)mn);
      atomicMax(out + 3, (unsigned long long)mx);
    }
  }
}

// ================================================================== reverse (Sec. 5.2)
template <class T>
__global__ void reverse_kernel(T* __restrict__ a, int64_t n) {
  const int64_t half = n / 2;
  constexpr int G = 4;  // swaps per thread and step, loaded before any is stored
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < half; i0 += G * step) {
    T x[G], y[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t i = i0 + g * step;
      if (i < half) {
        x[g] = a[i];
        y[g] = a[n - 1 - i];
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t i = i0 + g * step;
      if (i < half) {
        a[i] = y[g];
        a[n - 1 - i] = x[g];
      }
    }
  }
}

// ================================================================== classification
// Eytzinger tree over the B-1 sorted splitters: tree[1..B-1], node j has children 2j and 2j+1.
// Descent "go right when code > node" ends at leaf B + b where b = #splitters < code.  The key
// then belongs to bin 2b+1 if it equals splitter b (an equality bucket, Sec. 3), else bin 2b.
// The depth is known at compile time (fully unrolled descent).
template <int LOGB, class U>
__device__ __forceinline__ int classify_t(U code, const U* __restrict__ tree, const U* __restrict__ spl) {
  int j = 1;
#pragma unroll
  for (int l = 0; l < LOGB; ++l) j = 2 * j + (code > tree[j] ? 1 : 0);
  constexpr int B = 1 << LOGB;
  const int b = j - B;
  const int sb = b < B - 1 ? b : B - 2;
  return 2 * b + (code == spl[sb] ? 1 : 0);
}

// Exact rank prefilter over the splitter range [lo, hi] = [spl[0], spl[B-2]]: entry k of `tab`
// covers the codes lo + [k << shift, (k + 1) << shift).  With b_lo = #splitters < first code and
// b_hi = #splitters <= last code of the slice, every code of the slice has rank
// (#splitters < code) in [b_lo, b_hi].  Codes outside [lo, hi] are clamped into the first or last
// slice, whose bounds still hold for them.  The 32-bit entry holds b_lo (bits 0-15), a flag for
// one candidate (bit 30: b_hi == b_lo + 1) and a flag for several (bit 31: b_hi > b_lo + 1).
// The one candidate s0 = spl[b_lo] settles both the rank (b_lo + [s0 < code]) and the equality
// test (code == s0), as splitter b_lo + 1, if any, lies above the slice and cannot equal a code
// in it; with no candidate the rank is b_lo.  Only lanes whose slice holds a candidate read spl,
// so most lookups cost one 4-byte shared load; slices with several candidates take the tree.
// 4096 entries of 4 bytes (16 KB) for both key widths.
template <class U>
__host__ __device__ constexpr int pref_bits() { return 12; }
template <class U>
__host__ __device__ constexpr int pref_entries() { return 1 << pref_bits<U>(); }

// One slice: b_lo | one-candidate flag << 30 | several-candidates flag << 31.
using PrefEnt = uint32_t;
constexpr uint32_t kPrefOne = 1u << 30, kPrefMany = 1u << 31;
// Bytes of one task's prefilter table, the same for both key widths.
constexpr size_t kPrefTableBytes = 16384;
static_assert(pref_entries<uint32_t>() * sizeof(PrefEnt) == kPrefTableBytes &&
                  pref_entries<uint64_t>() * sizeof(PrefEnt) == kPrefTableBytes,
              "prefilter table size");

template <class U>
struct Pref {
  U lo, hi;
  int shift;
  int nent;
};

// Histogram slot of a code: rank b (#splitters < code) for a key inside bucket b, B + b for a key
// equal to splitter b (its equality bin).  The slot is the bin's place in the per-CTA shared
// histograms (BinSlot below: bin 2b at slot b, bin 2b+1 at slot B + b).  A prefilter slice with
// at most one candidate splitter settles it with one predicated comparison (branch-free); a
// wider slice falls back to the Eytzinger descent.
template <int LOGB, class U>
__device__ __forceinline__ int classify_fast(U code, const U* __restrict__ tree, const U* __restrict__ spl,
                                             const PrefEnt* __restrict__ tab, const Pref<U>& pf) {
  constexpr int B = 1 << LOGB;
  const U y = code < pf.lo ? pf.lo : (code > pf.hi ? pf.hi : code);
  const uint32_t e = tab[(uint32_t)((y - pf.lo) >> pf.shift)];
  if (!(e & kPrefMany)) {
    const int blo = (int)(e & 0xFFFFu);
    const bool cand = (e & kPrefOne) != 0u;
    U s0 = U(0);
    if (cand) s0 = spl[blo];
    return blo + ((cand && s0 < code) ? 1 : 0) + ((cand && code == s0) ? B : 0);
  }
  int j = 1;
#pragma unroll
  for (int l = 0; l < LOGB; ++l) j = 2 * j + (code > tree[j] ? 1 : 0);
  const int b = j - B;
  const int sb = b < B - 1 ? b : B - 2;
  return b + (code == spl[sb] ? B : 0);
}

// Splitter classifier of a task with 2^LOGB buckets (returns histogram slots, see
// classify_fast): one code at a time, or N codes at once
// (all prefilter lookups, then all candidate-splitter loads, then the comparisons, so the N
// dependency chains of shared loads overlap; the tree runs only when some code's slice holds
// several candidates).
template <int LOGB, class U>
struct SplitterClassifier {
  const U* tree;
  const U* spl;
  const PrefEnt* tab;
  Pref<U> pf;
  __device__ __forceinline__ int operator()(U code) const { return classify_fast<LOGB>(code, tree, spl, tab, pf); }
  template <int N>
  __device__ __forceinline__ void vec(const U (&code)[N], int (&slot)[N]) const {
    constexpr int B = 1 << LOGB;
    uint32_t e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const U y = code[i] < pf.lo ? pf.lo : (code[i] > pf.hi ? pf.hi : code[i]);
      e[i] = tab[(uint32_t)((y - pf.lo) >> pf.shift)];
    }
    U s0[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {  // candidate splitters, read only where the slice has one
      s0[i] = U(0);
      if (e[i] & kPrefOne) s0[i] = spl[e[i] & 0xFFFFu];
    }
    uint32_t any = 0u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int blo = (int)(e[i] & 0xFFFFu);
      const bool cand = (e[i] & kPrefOne) != 0u;
      slot[i] = blo + ((cand && s0[i] < code[i]) ? 1 : 0) + ((cand && code[i] == s0[i]) ? B : 0);
      any |= e[i];
    }
    if (any & kPrefMany) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if (e[i] & kPrefMany) {
          int j = 1;
#pragma unroll
          for (int l = 0; l < LOGB; ++l) j = 2 * j + (code[i] > tree[j] ? 1 : 0);
          const int b = j - B;
          const int sb = b < B - 1 ? b : B - 2;
          slot[i] = b + (code[i] == spl[sb] ? B : 0);
        }
      }
    }
  }
};

// Calls f(std::integral_constant<int, LOGB>) for the runtime depth (uniform per CTA).
template <class F>
__device__ __forceinline__ void with_logb(int logb, F&& f) {
  switch (logb) {
    case 1: f(IntC<1>()); break;
    case 2: f(IntC<2>()); break;
    case 3: f(IntC<3>()); break;
    case 4: f(IntC<4>()); break;
    case 5: f(IntC<5>()); break;
    case 6: f(IntC<6>()); break;
    case 7: f(IntC<7>()); break;
    case 8: f(IntC<8>()); break;
    default: f(IntC<9>()); break;
  }
}

// In-order index of Eytzinger node j in a complete tree with B-1 nodes.
__device__ __forceinline__ int eytz_inorder(int j, int logb) {
  const int d = 31 - __clz(j);
  const int p = j - (1 << d);
  return (2 * p + 1) * (1 << (logb - d - 1)) - 1;
}

// ================================================================== splitter selection
// One CTA per task.  Draws ns = min(oversample * B, kMaxSamples) keys at hashed positions
// (SplitMix64 of a seed derived from the task's range and attempt), sorts them with a bitonic
// network in shared memory and takes every (ns/B)-th as a splitter.  A value drawn many times
// repeats as a splitter: its keys all go to its equality bin.  It also clears what the round's
// later kernels accumulate into: the task's bin totals, and (CTA 0) the round's counters up to
// the probe results.
template <int KT, int THREADS>
__global__ void __launch_bounds__(THREADS)
sample_kernel(const Task* __restrict__ tasks, const int32_t* __restrict__ task_logb, int oversample,
              const typename Key<KT>::U* __restrict__ keys, const typename Key<KT>::U* __restrict__ tmp,
              typename Key<KT>::U* __restrict__ tree_out, typename Key<KT>::U* __restrict__ spl_out,
              Pref<typename Key<KT>::U>* __restrict__ pref_out, PrefEnt* __restrict__ tab_out,
              Counters* __restrict__ ctr, uint32_t* __restrict__ totals, int bin_stride) {
  using U = typename Key<KT>::U;
  __shared__ U s[kMaxSamples];
  const Task t = tasks[blockIdx.x];
  const int logb = task_logb[blockIdx.x];
  const int B = 1 << logb;
  for (int b = threadIdx.x; b < 2 * B; b += THREADS) totals[(size_t)blockIdx.x * bin_stride + b] = 0u;
  if (blockIdx.x == 0) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(ctr);
    for (int i = threadIdx.x; i < (int)(offsetof(Counters, probe) / 8); i += THREADS) w[i] = 0ull;
  }
  int ns = oversample * B;
  if (ns > kMaxSamples) ns = kMaxSamples;
  if (ns < B) ns = B;
  const U* src = (t.buf == kBufKeys ? keys : tmp) + t.begin;
  const uint64_t seed = mix64((uint64_t)t.begin * 0x9E3779B97F4A7C15ull ^ mix64((uint64_t)t.size) ^
                              ((uint64_t)t.attempt << 48));
  static_assert(THREADS * 4 == kMaxSamples, "four samples per thread");
  const int tid = threadIdx.x, lane = tid & 31;
  // thread tid holds sample slots 4 tid .. 4 tid + 3; slots at or past ns hold the largest code,
  // so the first ns slots of the sorted 4096 are the sorted sample
  U v[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int j = 4 * tid + e;
    v[e] = ~U(0);
    if (j < ns) {
      const uint64_t h = mix64(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull);
      v[e] = src[(int64_t)__umulhi((uint32_t)(h >> 32), (uint32_t)t.size)];  // uniform in [0, size)
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (4 * tid + e < ns && !t.enc) v[e] = Key<KT>::enc(v[e]);
  }
  // Bitonic network over 4096 slots: slot i meets i ^ j; the lower slot keeps the smaller code
  // when (i & k) == 0, the larger otherwise.  Distances below 4 stay in a thread's registers,
  // below 128 they cross lanes of a warp by shuffle, and from 128 up they go through shared
  // memory (15 of the 78 layers).
  auto keep = [](U mine, U other, bool lower, bool up) {
    const U lo = mine < other ? mine : other, hi = mine < other ? other : mine;
    return lower == up ? lo : hi;
  };
#pragma unroll
  for (int k = 2; k <= kMaxSamples; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < 4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p = e ^ j;
          if (p > e) {
            const bool up = ((4 * tid + e) & k) == 0;
            const U a = v[e], b = v[p];
            const bool sw = (a > b) == up;
            v[e] = sw ? b : a;
            v[p] = sw ? a : b;
          }
        }
      } else if (j < 128) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * tid + e;
          const U o = __shfl_xor_sync(0xffffffffu, v[e], j >> 2);
          v[e] = keep(v[e], o, (i & j) == 0, (i & k) == 0);
        }
      } else {
        __syncthreads();  // the previous exchange's reads are done
#pragma unroll
        for (int e = 0; e < 4; ++e) s[4 * tid + e] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * tid + e;
          v[e] = keep(v[e], s[i ^ j], (i & j) == 0, (i & k) == 0);
        }
      }
    }
  }
  (void)lane;
  __syncthreads();
#pragma unroll
  for (int e = 0; e < 4; ++e) s[4 * tid + e] = v[e];
  __syncthreads();
  U* tree = tree_out + (size_t)blockIdx.x * kBMax;
  U* spl = spl_out + (size_t)blockIdx.x * kBMax;
  const int step = ns / B;
  __shared__ U s_spl[kBMax];
  for (int i = tid; i < B - 1; i += THREADS) {
    const U x = s[(i + 1) * step - 1];
    spl[i] = x;
    s_spl[i] = x;
  }
  for (int j = 1 + tid; j < B; j += THREADS) tree[j] = s[(eytz_inorder(j, logb) + 1) * step - 1];
  // prefilter table over [spl[0], spl[B-2]]
  const U lo = s[step - 1], hi = s[(B - 1) * step - 1];
  const U range = hi - lo;
  const int bits = range == 0 ? 0 : (int)(8 * sizeof(U)) - (sizeof(U) == 4 ? __clz((uint32_t)range) : __clzll((uint64_t)range));
  const int shift = bits > pref_bits<U>() ? bits - pref_bits<U>() : 0;
  const int nent = (int)(range >> shift) + 1;
  if (tid == 0) {
    Pref<U> pf;
    pf.lo = lo;
    pf.hi = hi;
    pf.shift = shift;
    pf.nent = nent;
    pref_out[blockIdx.x] = pf;
  }
  // Slice k covers the codes lo + [k << shift, (k + 1) << shift) (the last one ends at hi).  A
  // splitter lies below every code of slice k exactly when its own slice is below k, so with
  // hist[k] = #splitters in slice k, b_lo(k) = #splitters < first code of k = sum of hist below
  // k, and hist[k] is the number of candidates inside the slice.
  __syncthreads();  // every read of the sorted sample is done: its array becomes the histogram
  uint32_t* hist = reinterpret_cast<uint32_t*>(s);
  static_assert(sizeof(s) >= sizeof(uint32_t) * 4096, "histogram fits the sample array");
#pragma unroll
  for (int e = 0; e < 4; ++e) hist[4 * tid + e] = 0u;
  __syncthreads();
  for (int i = tid; i < B - 1; i += THREADS) atomicAdd(&hist[(uint32_t)((s_spl[i] - lo) >> shift)], 1u);
  __syncthreads();
  uint32_t c[4], sum = 0u;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    c[e] = hist[4 * tid + e];
    sum += c[e];
  }
  __shared__ uint32_t s_wtmp[THREADS / 32];
  uint32_t total;
  uint32_t run = block_exclusive_sum<THREADS>(sum, s_wtmp, &total);
  PrefEnt* tab = tab_out + (size_t)blockIdx.x * pref_entries<U>();
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = 4 * tid + e;
    if (k < nent) tab[k] = run | (c[e] == 1u ? kPrefOne : 0u) | (c[e] > 1u ? kPrefMany : 0u);
    run += c[e];
  }
}

// Loads the task's tree and splitters into shared memory.
template <class U>
__device__ __forceinline__ void load_splitters(U* s_tree, U* s_spl, const U* tree, const U* spl, int B) {
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    s_tree[j] = tree[j];
    s_spl[j] = spl[j];
  }
}

// ================================================================== classifier policies
// The distribution kernels are generic over how a code is mapped to its bin.
//   SplitterCls: bins of sampled splitters (2B bins, odd bins hold keys equal to a splitter),
//                prefilter table + Eytzinger tree, one splitter set per task.
//   (the learned CDF model of the learned path is another policy, see learned.cuh)
template <class U>
struct SplitterCls {
  static constexpr int kMaxBins = kBinsMax;
  static constexpr bool kEqualBins = true;
  struct Params {
    const int32_t* task_logb;
    const U* tree;
    const U* spl;
    const Pref<U>* pref;
    const PrefEnt* tab;
  };
  struct Shared {
    U tree[kBMax], spl[kBMax];
    PrefEnt tab[pref_entries<U>()];
    Pref<U> pf;
    int logb;
  };
  // Fills the shared state of `task` (all threads); returns the task's number of bins.
  __device__ static int setup(Shared& sh, const Params& p, int task) {
    const int logb = p.task_logb[task];
    const int B = 1 << logb;
    load_splitters(sh.tree, sh.spl, p.tree + (size_t)task * kBMax, p.spl + (size_t)task * kBMax, B);
    const Pref<U> pf = p.pref[task];
    for (int k = threadIdx.x; k < pf.nent; k += blockDim.x) sh.tab[k] = p.tab[(size_t)task * pref_entries<U>() + k];
    if (threadIdx.x == 0) {
      sh.pf = pf;
      sh.logb = logb;
    }
    return 2 * B;
  }
  // The task's number of bins, without the shared state.
  __device__ static int nbins(const Params& p, int task) { return 2 << p.task_logb[task]; }
  // Calls f(classifier) with a classifier specialised for the task's depth.
  template <class F>
  __device__ static void with(const Shared& sh, const Params&, F&& f) {
    with_logb(sh.logb, [&](auto LB) {
      constexpr int L = decltype(LB)::value;
      const Pref<U> pf = sh.pf;
      f(SplitterClassifier<L, U>{sh.tree, sh.spl, sh.tab, pf});
    });
  }
};

// Shared-memory slot of a bin in the per-CTA histograms.  With equality bins nearly every key
// of distinct data lands in an even bin (2b), so an identity layout would leave the odd banks
// idle and double the bank conflicts of the histogram atomics and lookups; bucket bin 2b lives
// at slot b and equality bin 2b+1 at slot B + b instead.  Without equality bins: identity.
// Classifiers return slots; this map serves the loops that walk the bins in key order.
template <bool EQ>
struct BinSlot {
  int lb;  // log2 of the bucket count B = nbins / 2 (EQ only)
  __device__ __forceinline__ int operator()(int bin) const { return EQ ? (bin >> 1) | ((bin & 1) << lb) : bin; }
  // the slot holds an equality bin
  __device__ __forceinline__ bool equal(int sl) const { return EQ && (sl >> lb) != 0; }
};

// ================================================================== count
// One CTA per chunk.  The chunk is cut into 16-byte-aligned windows of TILE codes that stream
// into STAGES shared buffers by bulk copy; elements of a window outside the chunk are masked
// (only the first and last window have any), and the last window's sub-16-byte tail is
// classified straight from global memory.  Every code is classified and counted in a shared
// histogram, written to counts[chunk][bin] at the end and added to the task's bin totals.  Every
// key's histogram slot is also stored (2 bytes, at the key's element index in `slots`), so that
// the scatter reads the classification instead of repeating it.
template <int KT, class CLS, int THREADS, int TILE, int STAGES>
__global__ void __launch_bounds__(THREADS)
count_kernel(const Chunk* __restrict__ chunks, const Task* __restrict__ tasks,
             const typename Key<KT>::U* __restrict__ keys, const typename Key<KT>::U* __restrict__ tmp,
             typename CLS::Params cp, uint32_t* __restrict__ counts, int bin_stride,
             uint32_t* __restrict__ totals, uint16_t* __restrict__ slots, Counters* ctr) {
  using U = typename Key<KT>::U;
  constexpr int KS = sizeof(U);
  constexpr int VEC = 16 / KS;                // codes per 16-byte vector
  constexpr int NV = TILE / VEC / THREADS;    // vectors per thread per window
  static_assert(TILE % (VEC * THREADS) == 0, "window must split evenly into vectors");
  constexpr int BUF_BYTES = TILE * KS;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[STAGES];
  __shared__ typename CLS::Shared cs;
  __shared__ uint32_t hist[CLS::kMaxBins];

  const Chunk c = chunks[blockIdx.x];
  const Task t = tasks[c.task];
  const int nb = CLS::setup(cs, cp, c.task);
  const BinSlot<CLS::kEqualBins> slot{__ffs(nb) - 2};
  for (int b = threadIdx.x; b < nb; b += THREADS) hist[b] = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(&bars[i], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  const U* src = t.buf == kBufKeys ? keys : tmp;
  const bool enc = t.enc != 0;
  const int64_t cb = c.begin, ce = c.begin + c.size;
  const int64_t a0 = cb - cb % VEC;  // first window starts 16-byte aligned
  const int ntiles = (int)((ce - a0 + TILE - 1) / TILE);
  auto buf = [&](int stg) { return reinterpret_cast<U*>(smem + (size_t)stg * BUF_BYTES); };
  auto issue = [&](int tile) {
    const int64_t ws = a0 + (int64_t)tile * TILE;
    const int64_t we = ws + TILE < ce ? ws + TILE : ce;
    const int64_t wa = we - we % VEC;
    const int stg = tile % STAGES;
    const uint32_t bytes = (uint32_t)((wa - ws) * KS);
    mbar_arrive_expect_tx(&bars[stg], bytes);
    if (bytes) bulk_g2s(buf(stg), src + ws, bytes, &bars[stg]);
  };
  if (threadIdx.x == 0)
    for (int i = 0; i < STAGES && i < ntiles; ++i) issue(i);
  uint32_t parity = 0;
  bool failed = false;
  CLS::with(cs, cp, [&](auto classify) {
    auto count_one = [&](U x, int64_t pos) {
      const int sl = classify(enc ? x : Key<KT>::enc(x));
      atomicAdd(&hist[sl], 1u);
      slots[pos] = (uint16_t)sl;
    };
    for (int tile = 0; tile < ntiles; ++tile) {
      const int stg = tile % STAGES;
      const int64_t ws = a0 + (int64_t)tile * TILE;
      const int64_t we = ws + TILE < ce ? ws + TILE : ce;
      const int64_t wa = we - we % VEC;
      const bool ok = mbar_wait_bounded(&bars[stg], (parity >> stg) & 1u);
      parity ^= 1u << stg;
      if (!__syncthreads_and(ok)) { failed = true; break; }
      const uint4* bp = reinterpret_cast<const uint4*>(buf(stg));
      if (ws >= cb && ws + TILE <= ce) {  // interior window: every element valid
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          U v[VEC];
          *reinterpret_cast<uint4*>(v) = bp[threadIdx.x + q * THREADS];
          if (!enc) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) v[i] = Key<KT>::enc(v[i]);
          }
          int sl[VEC];
          classify.vec(v, sl);
          uint16_t s16[VEC];
#pragma unroll
          for (int i = 0; i < VEC; ++i) {
            atomicAdd(&hist[sl[i]], 1u);
            s16[i] = (uint16_t)sl[i];
          }
          // the window starts on a 16-byte boundary of the keys, so these VEC slots are aligned
          const int64_t pos = ws + (int64_t)(threadIdx.x + q * THREADS) * VEC;
          if constexpr (VEC == 4) *reinterpret_cast<uint2*>(slots + pos) = *reinterpret_cast<const uint2*>(s16);
          else *reinterpret_cast<uint32_t*>(slots + pos) = *reinterpret_cast<const uint32_t*>(s16);
        }
      } else {
        const int k0 = (int)((cb > ws ? cb : ws) - ws), k1 = (int)(wa - ws);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int vi = threadIdx.x + q * THREADS;
          if (vi * VEC >= k1) break;
          U v[VEC];
          *reinterpret_cast<uint4*>(v) = bp[vi];
#pragma unroll
          for (int i = 0; i < VEC; ++i) {
            const int k = vi * VEC + i;
            if (k >= k0 && k < k1) count_one(v[i], ws + k);
          }
        }
        // sub-16-byte tail of the chunk, straight from global memory
        const int64_t g = (wa > cb ? wa : cb) + threadIdx.x;
        if (g < we) count_one(src[g], g);
      }
      __syncthreads();  // this stage's buffer is consumed
      if (threadIdx.x == 0 && tile + STAGES < ntiles) {
        fence_proxy_async_smem();
        issue(tile + STAGES);
      }
    }
  });
  if (failed) {
    // a bulk copy did not complete in time: report, then give in-flight copies a bounded wait
    if (threadIdx.x == 0) {
      atomicAdd(&ctr->timeout, 1ull);
      for (int i = 0; i < STAGES; ++i) mbar_wait_bounded(&bars[i], (parity >> i) & 1u);
    }
    return;
  }
  __syncthreads();
  uint32_t* out = counts + (size_t)blockIdx.x * bin_stride;
  uint32_t* tot = totals + (size_t)c.task * bin_stride;
  for (int b = threadIdx.x; b < nb; b += THREADS) {
    const uint32_t v = hist[slot(b)];
    out[b] = v;
    if (v) atomicAdd(tot + b, v);
  }
}

// ================================================================== scatter
// One CTA per chunk.  The chunk is cut into 16-byte-aligned windows of TILE elements,
// double-buffered in shared memory by bulk copy (the last window's sub-16-byte tail is fetched
// with plain loads a tile ahead and stored before use); elements outside the chunk are masked.
// Every key's bin slot comes from the count pass (`slots`, streamed in beside the keys), so the
// scatter does no classification.  Per window: rank every code inside its bin with a shared
// atomic, scan the bin counts, stage the window in place grouped by bin (codes and values), then
// write each bin's run to its next free slots in the destination buffer (coalesced within runs).
// Keys of an equality bin written to the key buffer are final and are decoded on the way out.
template <int KT, int VB, class CLS, int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS, 2)  // two resident CTAs per SM: at most 64 registers
scatter_kernel(const Chunk* __restrict__ chunks, const Task* __restrict__ tasks,
               typename Key<KT>::U* __restrict__ keys, typename Val<VB>::T* __restrict__ vals,
               typename Key<KT>::U* __restrict__ tmpk, typename Val<VB>::T* __restrict__ tmpv,
               typename CLS::Params cp, const uint32_t* __restrict__ counts, int bin_stride,
               uint32_t* __restrict__ cursors, const uint16_t* __restrict__ slots, Counters* ctr) {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  constexpr int KS = sizeof(U);
  constexpr int VS = VB ? VB : KS;
  constexpr int VK = 16 / KS;                       // codes per 16-byte vector
  constexpr int VV = 16 / VS;                       // values per 16-byte vector
  constexpr int VA = VK > VV ? VK : VV;             // window alignment (elements)
  constexpr int NV = TILE / VK / THREADS;           // code vectors per thread
  constexpr int ITEMS = NV * VK;
  static_assert(TILE % (VK * THREADS) == 0 && TILE % VA == 0, "window must split evenly");
  static_assert(TILE <= 65536 && CLS::kMaxBins <= 65536, "rank and bin share one 32-bit word");
  constexpr int KBUF = TILE * KS;
  constexpr int VBUF = VB ? TILE * VS : 0;
  constexpr int NBMAX = CLS::kMaxBins;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + 2 * (KBUF + VBUF));  // per-window counts, then starts
  uint32_t* cursor = hist + NBMAX;                                         // next write offset per bin
  uint32_t* gbase = cursor + NBMAX;                                        // cursor - window start
  // two slot tiles, each the window widened to 8-element boundaries; a window's staged bin tags
  // overwrite its own slot tile once every thread holds its slots
  constexpr int SBUF = TILE + 16;
  uint16_t* sbuf0 = reinterpret_cast<uint16_t*>(gbase + NBMAX);
  auto sbuf = [&](int stg) { return sbuf0 + (size_t)stg * SBUF; };
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t wtmp[THREADS / 32 + 1];

  const Chunk c = chunks[blockIdx.x];
  const Task t = tasks[c.task];
  const int nb = CLS::nbins(cp, c.task);
  const BinSlot<CLS::kEqualBins> slot{__ffs(nb) - 2};  // hist, cursor, gbase and stage_b hold slots
  for (int b = threadIdx.x; b < nb; b += THREADS) {  // reserve this chunk's run in every bin
    const uint32_t cnt = counts[(size_t)blockIdx.x * bin_stride + b];
    cursor[slot(b)] = cnt ? atomicAdd(cursors + (size_t)c.task * bin_stride + b, cnt) : 0u;
    hist[b] = 0;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();

  const bool from_keys = t.buf == kBufKeys;
  const U* srck = from_keys ? keys : tmpk;
  const V* srcv = VB ? (from_keys ? vals : tmpv) : nullptr;
  U* dstk = (from_keys ? tmpk : keys) + t.begin;
  V* dstv = VB ? (from_keys ? tmpv : vals) + t.begin : nullptr;
  const bool dst_is_keys = !from_keys;
  const bool enc = t.enc != 0;
  const int64_t cb = c.begin, ce = c.begin + c.size;
  const int64_t a0 = cb - cb % VA;
  const int ntiles = (int)((ce - a0 + TILE - 1) / TILE);
  auto kbuf = [&](int stg) { return reinterpret_cast<U*>(smem + (size_t)stg * KBUF); };
  auto vbuf = [&](int stg) { return reinterpret_cast<V*>(smem + 2 * (size_t)KBUF + (size_t)stg * VBUF); };

  // sub-16-byte tails (fewer than VK codes / VV values) are fetched at issue time into
  // registers of threads 0..VK-2 (codes) and 32..32+VV-2 (values), stored before use
  U pend_k0 = U(0), pend_k1 = U(0);
  V pend_v0 = V(0), pend_v1 = V(0);
  auto issue = [&](int tile) {
    const int stg = tile & 1;
    const int64_t ws = a0 + (int64_t)tile * TILE;
    const int64_t we = ws + TILE < ce ? ws + TILE : ce;
    const int64_t wk = we - we % VK, wv = we - we % VV;
    if (threadIdx.x == 0) {
      const uint32_t kb = (uint32_t)((wk - ws) * KS), vb = VB ? (uint32_t)((wv - ws) * VS) : 0u;
      // slots [ws rounded down to 8, we rounded up to 8): 16-byte aligned, inside the slot array
      const int64_t s0 = ws & ~(int64_t)7, s1 = (we + 7) & ~(int64_t)7;
      const uint32_t sbytes = (uint32_t)((s1 - s0) * 2);
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bars[stg], kb + vb + sbytes);
      if (kb) bulk_g2s(kbuf(stg), srck + ws, kb, &bars[stg]);
      if (VB && vb) bulk_g2s(vbuf(stg), srcv + ws, vb, &bars[stg]);
      if (sbytes) bulk_g2s(sbuf(stg), slots + s0, sbytes, &bars[stg]);
    }
    const int tid = threadIdx.x;
    if (tid < VK && wk + tid < we) {
      const U x = srck[wk + tid];
      if (stg) pend_k1 = x; else pend_k0 = x;
    }
    if (VB && tid >= 32 && tid < 32 + VV && wv + (tid - 32) < we) {
      const V x = srcv[wv + (tid - 32)];
      if (stg) pend_v1 = x; else pend_v0 = x;
    }
  };
  issue(0);
  if (ntiles > 1) issue(1);

  uint32_t parity = 0;
  bool failed = false;
  for (int tile = 0; tile < ntiles; ++tile) {
    const int stg = tile & 1;
    const int64_t ws = a0 + (int64_t)tile * TILE;
    const int64_t we = ws + TILE < ce ? ws + TILE : ce;
    const int64_t wk = we - we % VK, wv = we - we % VV;
    const int k0 = (int)((cb > ws ? cb : ws) - ws), k1 = (int)(we - ws);  // valid buffer range
    const int cnt = k1 - k0;
    const bool full = k0 == 0 && k1 == TILE;
    U* bk = kbuf(stg);
    V* bv = VB ? vbuf(stg) : nullptr;
    {
      const int tid = threadIdx.x;
      if (tid < VK && wk + tid < we) bk[wk - ws + tid] = stg ? pend_k1 : pend_k0;
      if (VB && tid >= 32 && tid < 32 + VV && wv + (tid - 32) < we) bv[wv - ws + (tid - 32)] = stg ? pend_v1 : pend_v0;
    }
    const bool ok = mbar_wait_bounded(&bars[stg], (parity >> stg) & 1u);
    parity ^= 1u << stg;
    if (!__syncthreads_and(ok)) { failed = true; break; }

    U code[ITEMS];
    V val[ITEMS];
    uint32_t packed[ITEMS];  // slot << 16 | rank inside the bin; 0xFFFFFFFF for masked elements
    const uint16_t* sw = sbuf(stg) + (ws & 7);  // slot of window element 0
    uint16_t* stage_b = sbuf(stg);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int vi = threadIdx.x + q * THREADS;
      U v[VK];
      *reinterpret_cast<uint4*>(v) = reinterpret_cast<const uint4*>(bk)[vi];
#pragma unroll
      for (int i = 0; i < VK; ++i) {
        v[i] = enc ? v[i] : Key<KT>::enc(v[i]);
        code[q * VK + i] = v[i];
        if (VB) val[q * VK + i] = bv[vi * VK + i];
      }
      // the window starts on a multiple of VA >= VK elements: the VK slots are aligned
      uint16_t s16[VK];
      if constexpr (VK == 4) *reinterpret_cast<uint2*>(s16) = *reinterpret_cast<const uint2*>(sw + vi * VK);
      else *reinterpret_cast<uint32_t*>(s16) = *reinterpret_cast<const uint32_t*>(sw + vi * VK);
#pragma unroll
      for (int i = 0; i < VK; ++i) {
        const int k = vi * VK + i;
        const uint32_t sl = s16[i];
        packed[q * VK + i] = (full || (k >= k0 && k < k1)) ? ((sl << 16) | atomicAdd(&hist[sl], 1u)) : 0xFFFFFFFFu;
      }
    }
    __syncthreads();
    block_exclusive_scan<THREADS>(hist, hist, nb, wtmp, slot);  // hist := window start of each bin
    for (int b = threadIdx.x; b < nb; b += THREADS) {
      const int sl = slot(b);
      const uint32_t start = hist[sl];
      const uint32_t next = (b + 1 < nb) ? hist[slot(b + 1)] : (uint32_t)cnt;
      gbase[sl] = cursor[sl] - start;
      cursor[sl] += next - start;
    }
    // stage in place: every thread has read its codes from the buffer (scan barriers above)
#pragma unroll
    for (int e = 0; e < ITEMS; ++e) {
      if (packed[e] != 0xFFFFFFFFu) {
        const uint32_t sl = packed[e] >> 16;
        const uint32_t p = hist[sl] + (packed[e] & 0xFFFFu);
        bk[p] = code[e];
        if (VB) bv[p] = val[e];
        stage_b[p] = (uint16_t)sl;
      }
    }
    __syncthreads();
    auto write_one = [&](int i) {
      const int b = stage_b[i];
      const uint32_t o = gbase[b] + (uint32_t)i;
      const U k = bk[i];
      dstk[o] = (dst_is_keys && slot.equal(b)) ? Key<KT>::dec(k) : k;  // equality bin: final
      if (VB) dstv[o] = bv[i];
    };
    if (full) {
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) write_one(r * THREADS + threadIdx.x);
    } else {
      for (int i = threadIdx.x; i < cnt; i += THREADS) write_one(i);
    }
    __syncthreads();  // buffer, stage_b and hist are free again
    for (int b = threadIdx.x; b < nb; b += THREADS) hist[b] = 0;
    if (tile + 2 < ntiles) issue(tile + 2);
  }
  if (failed && threadIdx.x == 0) {
    atomicAdd(&ctr->timeout, 1ull);
    for (int i = 0; i < 2; ++i) mbar_wait_bounded(&bars[i], (parity >> i) & 1u);
  }
}

// ================================================================== bookkeeping (Sec. 4.1, Sec. 3)
// One thread per child bin.  Every warp stays whole until its counters are updated: list slots
// and counter increments are aggregated per warp (one atomic per warp and list), because at
// the second level tens of thousands of children hit the same few counters.
// Reserves `want`-many slots of a list for the lanes that want one; returns the lane's slot.
__device__ __forceinline__ unsigned long long warp_reserve(bool want, unsigned long long* counter) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (m == 0u) return 0ull;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0ull;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
}

// Adds the warp's sum of v to *counter (one atomic per warp, none when the sum is zero).
__device__ __forceinline__ void warp_add(unsigned long long v, unsigned long long* counter) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(counter, v);
}

// What becomes of child bin b = (start, size) of task t; every lane of the calling warp takes
// part (list slots and counters are aggregated per warp).  nonequal: the parent's keys outside
// its equality bins.
struct BookLists {
  Counters* ctr;
  Task* next;
  Item* base_items;
  Item* copy_items;
  Item* fb_items;
  ListCaps caps;
};

__device__ __forceinline__ void bookkeep_child(const Task& t, int b, uint2 ch, int64_t nonequal, int equal_bins,
                                               int base_cap, const BookLists& L) {
  Counters* ctr = L.ctr;
  const int dst = t.buf == kBufKeys ? kBufTmp : kBufKeys;
  Item it;
  it.begin = t.begin + ch.x;
  it.size = ch.y;
  it.buf = (uint16_t)dst;
  it.enc = 1;
  // what becomes of this child
  const bool live = ch.y != 0u;
  const bool equal = live && equal_bins && (b & 1);  // every key equals the splitter: final (Sec. 3)
  const bool base = live && !equal && (int64_t)ch.y <= base_cap;
  const bool split = live && !equal && !base;
  // bad split (Sec. 4.1, p = 1/8): the child kept more than floor(7/8) of the parent's keys
  // that are not in an equality bin (those are final and are not split further)
  const bool bad = split && (int64_t)ch.y > ((7 * nonequal) >> 3);
  const int left = t.bad_left - (bad ? 1 : 0);
  const bool fallback = split && left <= 0;
  const bool recurse = split && left > 0;
  const bool copy = equal && dst == kBufTmp;
  const int cls = ch.y <= 1024u ? 0 : (ch.y <= 2048u ? 1 : (ch.y <= 4096u ? 2 : (ch.y <= 8192u ? 3 : 4)));

  warp_add(equal ? 1ull : 0ull, &ctr->equal_buckets);
  warp_add(bad ? 1ull : 0ull, &ctr->bad_splits);
  warp_add(copy ? (unsigned long long)ch.y : 0ull, &ctr->copy_elems);
  warp_add(base ? (unsigned long long)ch.y : 0ull, &ctr->base_elems);
  auto put = [&](bool want, Item* list, unsigned long long* counter, int64_t cap) {
    const unsigned long long k = warp_reserve(want, counter);
    if (want) {
      if ((int64_t)k < cap) list[k] = it;
      else atomicAdd(&ctr->overflow, 1ull);
    }
  };
  put(copy, L.copy_items, &ctr->n_copy, L.caps.copy_cap);
  int grp = 0;
  if (L.caps.groups > 1) {
    grp = (int)(((it.begin - L.caps.group_first) * L.caps.groups) / L.caps.group_n);
    grp = grp < 0 ? 0 : (grp >= L.caps.groups ? L.caps.groups - 1 : grp);
  }
  for (int g = 0; g < L.caps.groups; ++g) {
    Item* lists = L.base_items + (size_t)g * L.caps.group_stride;
#pragma unroll
    for (int c = 0; c < kBaseClasses; ++c)
      put(base && cls == c && grp == g, lists + L.caps.base_off[c], &ctr->n_base[g][c], L.caps.base_cap[c]);
  }
  put(fallback, L.fb_items, &ctr->n_fallback, L.caps.fb_cap);
  const unsigned long long k = warp_reserve(recurse, &ctr->n_next);
  if (recurse) {
    Task nt;
    nt.begin = it.begin;
    nt.size = it.size;
    nt.buf = dst;
    nt.enc = 1;
    nt.bad_left = left;
    nt.attempt = t.attempt + 1;
    if ((int64_t)k < L.caps.task_cap) L.next[k] = nt;
    else atomicAdd(&ctr->overflow, 1ull);
  }
}

// One CTA per task: the exclusive scan of the task's bin totals gives every bin's first element
// (relative to the task's first element); the totals become the bins' write cursors, from which
// every scatter CTA reserves the run of its chunk with one atomic per bin (runs of different
// chunks land in a bin in the order of their reservations: the sort is unstable, so any order is
// correct); children[task * bin_stride + bin] = (start, size).  The same CTA then does the
// task's bookkeeping (bookkeep_child for every bin), so a level needs one launch for both.
template <int THREADS, int MAXBINS>
__global__ void __launch_bounds__(THREADS)
scan_bookkeep_kernel(const Task* __restrict__ tasks, const int32_t* __restrict__ task_nbins,
                     uint32_t* __restrict__ totals, int bin_stride, uint2* __restrict__ children, int equal_bins,
                     int base_cap, BookLists L) {
  __shared__ uint32_t tot[MAXBINS];
  __shared__ uint32_t start[MAXBINS];
  __shared__ uint32_t wtmp[THREADS / 32 + 1];
  __shared__ unsigned long long s_equal;
  const int task = blockIdx.x;
  const int nb = task_nbins[task];
  uint32_t* tt = totals + (size_t)task * bin_stride;
  for (int b = threadIdx.x; b < nb; b += THREADS) tot[b] = tt[b];
  if (threadIdx.x == 0) s_equal = 0ull;
  __syncthreads();
  block_exclusive_scan<THREADS>(tot, start, nb, wtmp);
  unsigned long long e = 0ull;
  for (int b = threadIdx.x; b < nb; b += THREADS) {
    children[(size_t)task * bin_stride + b] = make_uint2(start[b], tot[b]);
    tt[b] = start[b];
    if (equal_bins && (b & 1)) e += tot[b];
  }
  e = warp_sum(e);
  if ((threadIdx.x & 31) == 0 && e) atomicAdd(&s_equal, e);
  __syncthreads();
  const Task t = tasks[task];
  const int64_t nonequal = t.size - (int64_t)s_equal;
  for (int b0 = 0; b0 < nb; b0 += THREADS) {  // whole warps: the lists are reserved per warp
    const int b = b0 + (int)threadIdx.x;
    const uint2 ch = b < nb ? make_uint2(start[b], tot[b]) : make_uint2(0u, 0u);
    bookkeep_child(t, b, ch, nonequal, equal_bins, base_cap, L);
  }
}

// ================================================================== base sort (Sec. 5.1)
// One CTA per bucket of at most CAP = THREADS * ITEMS elements, sorted in shared memory by a
// register-blocked merge sort: every thread sorts ITEMS consecutive codes in registers with a
// compile-time bitonic network, then log2(active threads) merge-path rounds double the sorted
// runs.  Shared-memory indices are padded (one word per 32) so the blocked per-thread accesses
// are free of bank conflicts.  With a payload the sort key is (code, original position), which
// also orders the padding (largest code, positions >= m) after real keys; values are gathered
// through the positions at the end.  Without a payload, padding and real largest-code keys are
// identical bit patterns, so the first m outputs are correct whatever their order.
// Padded capacity of the shared arrays: CAP plus one pad element per 32 (4-byte codes) or per
// 16 (8-byte codes), rounded up to a multiple of 4 so that each array that follows (positions,
// values) starts 16-byte aligned.
template <int KS>
__host__ __device__ constexpr int base_sort_pcap(int cap, int items) {
  // cap elements, one sentinel slot per run of the first merge round (runs of `items`), and
  // 32 slack elements (read-ahead and the padding of the last thread); then the bank padding
  return (cap + cap / items + 32 + (cap + cap / items + 32) / (KS == 4 ? 32 : 16) + 1 + 3) / 4 * 4;
}

template <class U>
__device__ __forceinline__ int pad_idx(int x) {
  return sizeof(U) == 4 ? x + (x >> 5) : x + (x >> 4);
}

// (a, ia) precedes (b, ib): by code, then by position when WITH_IDX
template <bool WITH_IDX, class U>
__device__ __forceinline__ bool precedes(U a, uint32_t ia, U b, uint32_t ib) {
  if (WITH_IDX) return a < b || (a == b && ia < ib);
  return a < b;
}

// Compile-time bitonic network over N registers.  CARRY: the index array x moves with its keys;
// CMPIDX: ties between equal codes are broken by x (otherwise equal codes are left in any order).
template <bool CARRY, bool CMPIDX, int N, class U>
__device__ __forceinline__ void register_sort(U (&k)[N], uint32_t (&x)[N]) {
#pragma unroll
  for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & kk) == 0;  // compile-time direction
          if (CARRY) {
            const bool gt = precedes<CMPIDX>(k[l], x[l], k[i], x[i]);
            const bool sw = gt == up;
            const U a = k[i], b = k[l];
            const uint32_t ya = x[i], yb = x[l];
            k[i] = sw ? b : a;
            k[l] = sw ? a : b;
            x[i] = sw ? yb : ya;
            x[l] = sw ? ya : yb;
          } else {
            const U a = k[i], b = k[l];
            const U lo = a < b ? a : b, hi = a < b ? b : a;
            k[i] = up ? lo : hi;
            k[l] = up ? hi : lo;
          }
        }
      }
    }
  }
}

// Shared bytes of the base sort's key, position and value arrays (the radix counters follow).
template <int KS, int VB, int THREADS, int ITEMS>
__host__ __device__ constexpr size_t base_sort_core_smem() {
  return ((size_t)base_sort_pcap<KS>(THREADS * ITEMS, ITEMS) * (KS + (VB ? 4 : 0)) + (size_t)THREADS * ITEMS * VB +
          15) / 16 * 16;
}

// ------------------------------------------------------------------ range-aware radix base case
// After the distribution levels a bucket holds the keys between two neighbouring splitters, so
// its codes usually span a narrow range [mn, mx].  Such a bucket is sorted by a stable LSD
// counting sort on r = code - mn (at most kRadixMaxBits bits): ceil(bits / kRadixDigitBits)
// passes over equal-width digits, every pass ranking the keys in shared memory.
//
// Ranking (one pass): thread t holds ITEMS consecutive keys (blocked).  Each thread counts its
// own keys per digit in 16-bit counters, two digits packed in one 32-bit word: digit d counts
// in word (d mod LW) * THREADS + t, low half for d < LW, high half above (LW = half the digit
// count).  A thread's counters all sit in the bank of its lane, so the counting is free of
// bank conflicts.  The words are then scanned in their linear order (digit-major, thread-minor),
// which is exactly the order of the stable ranks: each thread rakes LW + 1 consecutive words (an
// odd stride: conflict-free), a block scan joins the rakes, and one packed scan gives the
// prefixes of the low digits in the low halves and of the high digits in the high halves; the
// high digits then add the count of all low digits.  A key's destination is its digit-thread
// prefix plus the number of the thread's earlier keys with that digit.  The (LW+1)-th word of
// every raking segment is padding that is never counted.
constexpr int kRadixDigitBits = 6;                 // at most 64 digits per pass
constexpr int kRadixLanes = 1 << (kRadixDigitBits - 1);
constexpr int kRadixMaxBits = 24;                  // wider ranges use the merge-path base sort

template <int THREADS>
__host__ __device__ constexpr size_t radix_counter_bytes() {
  return (size_t)(kRadixLanes + 1) * THREADS * sizeof(uint32_t);
}

// The radix path is compiled in where its counters fit next to the base sort's arrays in the
// 227 KiB a CTA may use (all classes but the largest ones with values).
template <int KS, int VB, int THREADS, int ITEMS>
__host__ __device__ constexpr bool radix_fits() {
  return base_sort_core_smem<KS, VB, THREADS, ITEMS>() + radix_counter_bytes<THREADS>() <= (size_t)227 * 1024;
}

// Sorts the active threads' keys r[0..ITEMS) (and positions x, when W) by LSD passes over
// `nbits` <= 24 bits.  Real keys are below 2^24; padding keys are 0xFFFFFF and stay behind every
// real key (stable ranks, padding last in the input).  Bits 24-31 of r carry, within a pass, the
// key's rank among its thread's earlier keys of the same digit.  On return arr[pad(i)] (and
// idx[pad(i)]) hold the sorted sequence for i < P.  ctr: radix_counter_bytes<THREADS>().
template <int THREADS, int ITEMS, bool W>
__device__ __forceinline__ void radix_block_sort(uint32_t (&r)[ITEMS], uint32_t (&x)[ITEMS], bool active,
                                                 int nbits, uint32_t* __restrict__ arr, uint32_t* __restrict__ idx,
                                                 uint32_t* __restrict__ ctr, uint32_t* wtmp) {
  constexpr int LW = kRadixLanes;
  constexpr int SEG = LW + 1;
  const int tid = threadIdx.x;
  const int passes = (nbits + kRadixDigitBits - 1) / kRadixDigitBits;
  const int w = (nbits + passes - 1) / passes;
  const uint32_t dmask = (1u << w) - 1u;
  auto pad = [](int i) { return i + (i >> 5); };
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * w;
#pragma unroll
    for (int j = 0; j < SEG; ++j) ctr[tid * SEG + j] = 0u;
    __syncthreads();
    if (active) {
#pragma unroll
      for (int e = 0; e < ITEMS; ++e) {
        const uint32_t d = (r[e] >> shift) & dmask;
        const uint32_t sh = (d & LW) ? 16u : 0u;
        uint32_t* c = ctr + (d & (LW - 1)) * THREADS + tid;
        const uint32_t v = *c;
        r[e] = (r[e] & 0xFFFFFFu) | (((v >> sh) & 0xFFu) << 24);
        *c = v + (1u << sh);
      }
    }
    __syncthreads();
    uint32_t sum = 0u;  // the raking segment is read twice rather than held in registers
#pragma unroll
    for (int j = 0; j < SEG; ++j) sum += ctr[tid * SEG + j];
    uint32_t total;
    uint32_t run = block_exclusive_sum<THREADS>(sum, wtmp, &total);
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const uint32_t v = ctr[tid * SEG + j];
      ctr[tid * SEG + j] = run;
      run += v;
    }
    const uint32_t low_total = total & 0xFFFFu;  // keys whose digit is below LW
    __syncthreads();
    // every thread's keys are in its registers, so the array can be overwritten at once
    if (active) {
#pragma unroll
      for (int e = 0; e < ITEMS; ++e) {
        const uint32_t d = (r[e] >> shift) & dmask;
        const uint32_t v = ctr[(d & (LW - 1)) * THREADS + tid];
        const int dst = (int)(((d & LW) ? (v >> 16) + low_total : (v & 0xFFFFu)) + (r[e] >> 24));
        arr[pad(dst)] = r[e] & 0xFFFFFFu;
        if (W) idx[pad(dst)] = x[e];
      }
    }
    __syncthreads();  // the array is complete and every counter read before the next clear
    if (active && pass + 1 < passes) {
#pragma unroll
      for (int e = 0; e < ITEMS; ++e) {
        r[e] = arr[pad(tid * ITEMS + e)];
        if (W) x[e] = idx[pad(tid * ITEMS + e)];
      }
    }
  }
}

// The whole sort of one item by one CTA (blockDim.x == THREADS); `smem` holds
// base_sort_smem<KS, VB, THREADS, ITEMS>() bytes, 16-byte aligned (base_sort_core_smem when
// RADIX is false: callers whose buckets rarely have a narrow code range, or that need the
// shared memory for other work, keep the merge path only and a smaller footprint).
template <int KT, int VB, int THREADS, int ITEMS, bool RADIX = true>
__device__ __forceinline__ void base_sort_block(const Item& it, typename Key<KT>::U* __restrict__ keys,
                                                typename Val<VB>::T* __restrict__ vals,
                                                typename Key<KT>::U* __restrict__ tmpk,
                                                typename Val<VB>::T* __restrict__ tmpv, int out_buf, int decode,
                                                unsigned char* smem) {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  constexpr bool W = VB > 0;
  constexpr int CAP = THREADS * ITEMS;
  constexpr int PCAP = base_sort_pcap<sizeof(U)>(CAP, ITEMS);
  static_assert(PCAP % 4 == 0, "padded arrays must keep 16-byte alignment of the next array");
  U* sk = reinterpret_cast<U*>(smem);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + PCAP);
  V* sv = reinterpret_cast<V*>(si + (W ? PCAP : 0));

  const int m = (int)it.size;
  const int tid = threadIdx.x;
  // P: m rounded up to whole threads (at most ITEMS-1 padding elements); runs may be ragged
  const int na = (m + ITEMS - 1) / ITEMS;
  const int P = na * ITEMS;
  const U* srck = (it.buf == kBufKeys ? keys : tmpk) + it.begin;
  const V* srcv = W ? (it.buf == kBufKeys ? vals : tmpv) + it.begin : nullptr;
  bool max_code = false;  // a real code equal to the sentinel value (all ones)
  U mn = ~U(0), mx = U(0);  // range of the real codes
  // Staging of slots [0, P + ITEMS) (ITEMS slack slots: harmless read-ahead of the merge).
  // Merge-only callers stage with a plain strided loop (fewer live registers, more resident
  // CTAs); with the radix path every thread covers ITEMS + 1 strided slots (CAP + THREADS >=
  // P + ITEMS) and issues all of its global loads before using any, so their latency is paid once.
  if constexpr (!RADIX) {
    for (int i = tid; i < P + ITEMS; i += THREADS) {
      U c = ~U(0);
      if (i < m) {
        const U x = srck[i];
        c = it.enc ? x : Key<KT>::enc(x);
        max_code |= c == ~U(0);
        mn = c < mn ? c : mn;
        mx = c > mx ? c : mx;
        if (W) sv[i] = srcv[i];
      }
      sk[pad_idx<U>(i)] = c;
      if (W) si[pad_idx<U>(i)] = (uint32_t)i;
    }
  } else {
    U xk[ITEMS + 1];
    V xv[W ? ITEMS + 1 : 1];
#pragma unroll
    for (int e = 0; e <= ITEMS; ++e) {
      const int i = tid + e * THREADS;
      xk[e] = ~U(0);
      if (i < m) {
        xk[e] = srck[i];
        if (W) xv[W ? e : 0] = srcv[i];
      }
    }
#pragma unroll
    for (int e = 0; e <= ITEMS; ++e) {
      const int i = tid + e * THREADS;
      U c = ~U(0);
      if (i < m) {
        c = it.enc ? xk[e] : Key<KT>::enc(xk[e]);
        max_code |= c == ~U(0);
        mn = c < mn ? c : mn;
        mx = c > mx ? c : mx;
        if (W) sv[i] = xv[W ? e : 0];
      }
      if (i < P + ITEMS) {
        sk[pad_idx<U>(i)] = c;
        if (W) si[pad_idx<U>(i)] = (uint32_t)i;
      }
    }
  }
  __shared__ U s_wmn[THREADS / 32], s_wmx[THREADS / 32];
  __shared__ uint32_t s_wtmp[THREADS / 32];
  mn = warp_min(mn);
  mx = warp_max(mx);
  if ((tid & 31) == 0) {
    s_wmn[tid >> 5] = mn;
    s_wmx[tid >> 5] = mx;
  }
  // Without a real all-ones code every real key is below the padding and the sentinels, and
  // equal real keys may end in any order (the sort is unstable), so codes alone are compared
  // (CMPIDX false).  A real all-ones code ties with the sentinels and the padding: keys only,
  // such a bucket merges with bounds tests (`checked`); with values, ties are broken by the
  // original position (CMPIDX true: padding positions are >= m, sentinel indices all ones).
  // (the block-wide OR is also the barrier after the staging writes: always executed)
  const bool any_max = __syncthreads_or(max_code) != 0;
#pragma unroll 1
  for (int w = 0; w < THREADS / 32; ++w) {
    mn = s_wmn[w] < mn ? s_wmn[w] : mn;
    mx = s_wmx[w] > mx ? s_wmx[w] : mx;
  }
  U* dstk = (out_buf == kBufKeys ? keys : tmpk) + it.begin;
  V* dstv = W ? (out_buf == kBufKeys ? vals : tmpv) + it.begin : nullptr;
  if (mn == mx) {  // every key is equal: the order is the input order (values keep theirs)
    const U c = decode ? Key<KT>::dec(mn) : mn;
    for (int i = tid; i < m; i += THREADS) {
      dstk[i] = c;
      if (W) dstv[i] = sv[i];
    }
    return;
  }
  const U span = mx - mn;
  const int nbits = (int)(8 * sizeof(U)) - (sizeof(U) == 4 ? __clz((uint32_t)span) : __clzll((uint64_t)span));
  if constexpr (RADIX && radix_fits<sizeof(U), VB, THREADS, ITEMS>()) {
   if (nbits <= kRadixMaxBits) {
    // narrow range: LSD counting passes on r = code - mn (padding r = 0xFFFFFF sorts last)
    uint32_t* arr = reinterpret_cast<uint32_t*>(sk);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(smem + base_sort_core_smem<sizeof(U), VB, THREADS, ITEMS>());
    uint32_t r[ITEMS], xp[ITEMS];
    const bool act = tid < na;
    if (act) {
#pragma unroll
      for (int e = 0; e < ITEMS; ++e) {
        const int i = tid * ITEMS + e;
        r[e] = i < m ? (uint32_t)(sk[pad_idx<U>(i)] - mn) : 0xFFFFFFu;
        xp[e] = (uint32_t)i;
      }
    }
    __syncthreads();  // the code array is rewritten as 32-bit ranks
    radix_block_sort<THREADS, ITEMS, W>(r, xp, act, nbits, arr, si, ctr, s_wtmp);
    for (int i = tid; i < m; i += THREADS) {
      const int p = i + (i >> 5);
      const U c = mn + (U)arr[p];
      dstk[i] = decode ? Key<KT>::dec(c) : c;
      if (W) dstv[i] = sv[si[p]];
    }
    return;
   }
  }
  const bool checked = !W && any_max;
  U k[ITEMS];
  uint32_t x[ITEMS];
  const bool active = tid < na;
  auto sort_runs = [&](auto CMP) {
    constexpr bool C = decltype(CMP)::value;
    if (active) {
#pragma unroll
      for (int e = 0; e < ITEMS; ++e) {
        const int p = pad_idx<U>(tid * ITEMS + e);
        k[e] = sk[p];
        x[e] = W ? si[p] : 0u;
      }
      register_sort<W, C>(k, x);
    }
    // Merge rounds.  Before round R the registers go back to shared memory with runs of R
    // elements, each followed by one sentinel slot (all-ones code, all-ones index).  While a pair of
    // runs (2R elements) lies inside one warp's WSPAN = 32 * ITEMS elements, each warp keeps a fixed
    // region of WSPAN + 32 slots (its runs and their sentinels), so the round reads only what its
    // own warp wrote and a warp barrier suffices; wider rounds use one array-wide layout (run r at
    // slot r * (R + 1)) and block barriers.  A thread's ITEMS elements never straddle runs.
    constexpr int WSPAN = 32 * ITEMS;
    constexpr int WSTRIDE = WSPAN + 32;
    constexpr int LG_WSPAN = ITEMS == 32 ? 10 : (ITEMS == 16 ? 9 : 8);
    static_assert((1 << LG_WSPAN) == WSPAN, "ITEMS must be 8, 16 or 32");
    auto slot_of = [&](int pos, int lgR, bool wl) {
      if (wl) {
        const int lp = pos & (WSPAN - 1);
        return (pos >> LG_WSPAN) * WSTRIDE + lp + (lp >> lgR);
      }
      return pos + (pos >> lgR);
    };
    int lg = 0;
    while ((ITEMS << lg) < P) ++lg;
    int R = ITEMS;
    for (int round = 0; round < lg; ++round, R <<= 1) {
      const int lgR = __ffs(R) - 1;
      const bool warp_local = 2 * R <= WSPAN;
      // the first round's layout differs from the staging layout across warps: block barrier
      if (warp_local && round > 0) __syncwarp(); else __syncthreads();
      if (active) {
        const int pos0 = tid * ITEMS;
        const int slot0 = slot_of(pos0, lgR, warp_local);
#pragma unroll
        for (int e = 0; e < ITEMS; ++e) {
          const int p = pad_idx<U>(slot0 + e);
          sk[p] = k[e];
          if (W) si[p] = x[e];
        }
        if (((pos0 + ITEMS) & (R - 1)) == 0 || pos0 + ITEMS == P) {  // last thread of its run
          const int p = pad_idx<U>(slot0 + ITEMS);
          sk[p] = ~U(0);
          if (W) si[p] = 0xFFFFFFFFu;
        }
      }
      if (warp_local) __syncwarp(); else __syncthreads();
      if (active) {
        const int pos = tid * ITEMS;
        const int g = pos & ~(2 * R - 1);             // first element of the pair of runs
        const int d = pos - g;                        // this thread's diagonal inside the pair
        const int a0 = slot_of(g, lgR, warp_local);   // slot of run A's first element
        const int b0 = a0 + R + 1;                    // slot of run B's first element
        const int la = min(R, P - g);                  // run A (may be the ragged last run)
        const int lb = max(0, min(R, P - g - R));      // run B (may be short or empty)
        // merge-path split: the number of A elements among the first d outputs (ties take A)
        int lo = d > lb ? d - lb : 0;
        int hi = d < la ? d : la;
        for (int span = R; span > 0; span >>= 1) {  // log2(R) + 1 halvings suffice
          if (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int pa = pad_idx<U>(a0 + mid), pb = pad_idx<U>(b0 + d - 1 - mid);
            if (!precedes<C>(sk[pb], C ? si[pb] : 0u, sk[pa], C ? si[pa] : 0u)) lo = mid + 1;
            else hi = mid;
          }
        }
        int ia = a0 + lo, ib = b0 + (d - lo);  // slots of the next A and B elements
        U ka = lo < la ? sk[pad_idx<U>(ia)] : ~U(0), kb = d - lo < lb ? sk[pad_idx<U>(ib)] : ~U(0);
        uint32_t xa = 0xFFFFFFFFu, xb = 0xFFFFFFFFu;
        if (W) {
          if (lo < la) xa = si[pad_idx<U>(ia)];
          if (d - lo < lb) xb = si[pad_idx<U>(ib)];
        }
        if (!checked) {
          // Sentinels end both runs, so an exhausted run is never chosen while the other still
          // holds a smaller element.  Comparing codes only, padding codes (all ones) tie with A's
          // sentinel and ties take A, so A's index stops at its sentinel (those outputs land on
          // positions >= m, which are padding either way); with positions compared, the
          // sentinel's all-ones index breaks every tie.
          const int ea = a0 + la;
#pragma unroll
          for (int e = 0; e < ITEMS; ++e) {
            const bool take_a = !precedes<C>(kb, xb, ka, xa);
            if (W) {
              k[e] = take_a ? ka : kb;
              x[e] = take_a ? xa : xb;
            } else {
              k[e] = ka < kb ? ka : kb;
            }
            ia += take_a ? 1 : 0;
            if (!C) ia = min(ia, ea);
            ib += take_a ? 0 : 1;
            const int p = pad_idx<U>(take_a ? ia : ib);
            const U nk = sk[p];
            ka = take_a ? nk : ka;
            kb = take_a ? kb : nk;
            if (W) {
              const uint32_t nx = si[p];
              xa = take_a ? nx : xa;
              xb = take_a ? xb : nx;
            }
          }
        } else {
          // keys only with a real all-ones code: the same merge with explicit run ends
          const int ea = a0 + la, eb = b0 + lb;
#pragma unroll
          for (int e = 0; e < ITEMS; ++e) {
            const bool take_a = ia < ea && (ib >= eb || !(kb < ka));
            k[e] = take_a ? ka : kb;
            ia += take_a ? 1 : 0;
            ib += take_a ? 0 : 1;
            const U nk = sk[pad_idx<U>(take_a ? ia : ib)];
            ka = take_a ? nk : ka;
            kb = take_a ? kb : nk;
          }
        }
      }
    }
  };
  if (W && any_max) sort_runs(IntC<1>());
  else sort_runs(IntC<0>());
  __syncthreads();
  if (active) {
#pragma unroll
    for (int e = 0; e < ITEMS; ++e) {
      const int p = pad_idx<U>(tid * ITEMS + e);
      sk[p] = k[e];
      if (W) si[p] = x[e];
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += THREADS) {
    const int p = pad_idx<U>(i);
    const U c = sk[p];
    dstk[i] = decode ? Key<KT>::dec(c) : c;
    if (W) dstv[i] = sv[si[p]];
  }
}

// 24 resident warps per SM (at most 80 registers a thread): measured faster than both the
// unbounded allocation (16 warps) and 32 warps (64 registers with spills).
template <int THREADS>
constexpr int base_sort_min_blocks() { return 768 / THREADS > 0 ? 768 / THREADS : 1; }

template <int KT, int VB, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, base_sort_min_blocks<THREADS>())
base_sort_kernel(const Item* __restrict__ items, typename Key<KT>::U* __restrict__ keys,
                 typename Val<VB>::T* __restrict__ vals, typename Key<KT>::U* __restrict__ tmpk,
                 typename Val<VB>::T* __restrict__ tmpv, int out_buf, int decode) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Item it = items[blockIdx.x];
  base_sort_block<KT, VB, THREADS, ITEMS>(it, keys, vals, tmpk, tmpv, out_buf, decode, smem);
}

template <int KS, int VB, int THREADS, int ITEMS>
constexpr size_t base_sort_smem() {
  return base_sort_core_smem<KS, VB, THREADS, ITEMS>() +
         (radix_fits<KS, VB, THREADS, ITEMS>() ? radix_counter_bytes<THREADS>() : 0);
}

// ================================================================== copy temp -> keys (decode)
// Final buckets left in the temp buffer (equality buckets of odd levels) go home, decoded.  Their
// sizes are skewed (one duplicated value can hold most of the array), so the work is cut into
// tiles of TILE elements over all items: copy_plan_kernel numbers the tiles (one CTA; tile0[k] =
// first tile of item k, tile0[n] = total), and every CTA of copy_kernel takes tiles grid-strided.
// When every item fits one tile (tile0 == nullptr) tile k is item k and no numbering is needed.
template <int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS)
copy_plan_kernel(const Item* __restrict__ items, int n, uint32_t* __restrict__ tile0) {
  __shared__ uint32_t wtmp[THREADS / 32 + 1];
  const int tid = threadIdx.x;
  const int per = (n + THREADS - 1) / THREADS;
  const int lo = tid * per;
  uint32_t sum = 0;
  for (int i = 0; i < per && lo + i < n; ++i) sum += (items[lo + i].size + TILE - 1) / TILE;
  const int lane = tid & 31, warp = tid >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    constexpr int NW = THREADS / 32;
    uint32_t w = lane < NW ? wtmp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) wtmp[lane] = w;
  }
  __syncthreads();
  uint32_t run = x - sum + (warp > 0 ? wtmp[warp - 1] : 0u);
  for (int i = 0; i < per && lo + i < n; ++i) {
    tile0[lo + i] = run;
    run += (items[lo + i].size + TILE - 1) / TILE;
  }
  if (tid == THREADS - 1) tile0[n] = run;
}

template <int KT, int VB, int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS)
copy_kernel(const Item* __restrict__ items, int n, const uint32_t* __restrict__ tile0,
            typename Key<KT>::U* __restrict__ keys, typename Val<VB>::T* __restrict__ vals,
            const typename Key<KT>::U* __restrict__ tmpk, const typename Val<VB>::T* __restrict__ tmpv) {
  static_assert(TILE % THREADS == 0, "tile shape");
  const uint32_t total = tile0 ? tile0[n] : (uint32_t)n;  // no numbering: one tile per item
  for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
    int a = tile0 ? 0 : (int)t, b = tile0 ? n - 1 : (int)t;  // the item holding tile t: last k with tile0[k] <= t
    while (a < b) {
      const int m = (a + b + 1) >> 1;
      if (tile0[m] <= t) a = m; else b = m - 1;
    }
    const Item it = items[a];
    const int64_t e0 = tile0 ? (int64_t)(t - tile0[a]) * TILE : 0;
    const int64_t len = (int64_t)it.size - e0 < TILE ? (int64_t)it.size - e0 : TILE;
    const int64_t base = it.begin + e0;
#pragma unroll 8
    for (int r = 0; r < TILE / THREADS; ++r) {
      const int i = r * THREADS + threadIdx.x;
      if (i < len) {
        keys[base + i] = Key<KT>::dec(tmpk[base + i]);
        if (VB) vals[base + i] = tmpv[base + i];
      }
    }
  }
}

// ================================================================== nearly-sorted fix-up
// For input with few scattered descents (Sec. 5.2's partial insertion sort has the same aim:
// finish an almost sorted range in linear time).  Both elements of every descent are marked,
// repair rounds extend the marks until the unmarked elements R are ascending, one split moves R
// and the marked elements E apart, E is sorted on its own, and R and E are merged.  Comparisons
// are of the encoded codes.

// Marks both elements of every descent of src[0..len) in the bit mask (bit i of word i / 32):
// each warp takes four consecutive 32-element words per step, one load per element (the
// neighbours come by shuffle, the two across the ends by extra loads); *marked receives the
// number of marked elements.
template <int KT>
__global__ void fix_mark_kernel(const typename Key<KT>::U* __restrict__ src, int64_t len, uint32_t* __restrict__ mask,
                                unsigned long long* __restrict__ marked) {
  using U = typename Key<KT>::U;
  constexpr int WPS = 4;  // words per warp step
  const int lane = threadIdx.x & 31;
  const int64_t nwords = (len + 31) / 32;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  unsigned long long cnt = 0;
  for (int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * WPS; w0 < nwords;
       w0 += warps * WPS) {
    U x[WPS];
#pragma unroll
    for (int k = 0; k < WPS; ++k) {
      const int64_t i = (w0 + k) * 32 + lane;
      x[k] = i < len ? Key<KT>::enc(__ldg(src + i)) : U(0);
    }
    const int64_t e0 = w0 * 32 - 1, e1 = (w0 + WPS) * 32;  // neighbours across the step's ends
    const U before = (e0 >= 0 && e0 < len) ? Key<KT>::enc(__ldg(src + e0)) : U(0);
    const U after = e1 < len ? Key<KT>::enc(__ldg(src + e1)) : U(0);
#pragma unroll
    for (int k = 0; k < WPS; ++k) {
      const int64_t i = (w0 + k) * 32 + lane;
      U prev = __shfl_up_sync(0xffffffffu, x[k], 1);
      U next = __shfl_down_sync(0xffffffffu, x[k], 1);
      const U last_prev = __shfl_sync(0xffffffffu, k > 0 ? x[k > 0 ? k - 1 : 0] : before, 31);
      const U first_next = __shfl_sync(0xffffffffu, k + 1 < WPS ? x[k + 1 < WPS ? k + 1 : k] : after, 0);
      if (lane == 0) prev = k > 0 ? last_prev : before;
      if (lane == 31) next = k + 1 < WPS ? first_next : after;
      const bool left = i > 0 && i < len && prev > x[k];
      const bool right = i + 1 < len && x[k] > next;
      const uint32_t bits = __ballot_sync(0xffffffffu, left || right);
      if (w0 + k < nwords && lane == 0) {
        mask[w0 + k] = bits;
        cnt += (unsigned long long)__popc(bits);
      }
    }
  }
  if (lane == 0 && cnt) atomicAdd(marked, cnt);
}

__device__ __forceinline__ uint32_t fix_word(const uint32_t* mask, int64_t w) { return __ldcg(mask + w); }

// One repair round: for every run of marked elements, its kept neighbours p (before) and q
// (after) become adjacent once the run is removed; if src[p] > src[q] both are marked.  p is
// found a word at a time; a run whose kept predecessor lies more than 64 words back marks the
// round as given up.  Sets *changed when it marked anything; *added counts the marks.
template <int KT>
__global__ void fix_repair_kernel(const typename Key<KT>::U* __restrict__ src, int64_t len, uint32_t* __restrict__ mask,
                                  unsigned int* __restrict__ changed, unsigned int* __restrict__ added) {
  const int64_t nwords = (len + 31) / 32;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t m = fix_word(mask, w);
    if (!m) continue;
    // run ends in this word: marked bits whose successor is unmarked
    const uint32_t nxt = w + 1 < nwords ? fix_word(mask, w + 1) : ~0u;
    uint32_t ends = m & ~((m >> 1) | (nxt << 31));
    while (ends) {
      const int b = __ffs(ends) - 1;
      ends &= ends - 1;
      const int64_t q = w * 32 + b + 1;
      if (q >= len) continue;
      // kept predecessor: the highest unmarked bit below the run
      int64_t pw = w;
      uint32_t below = ~m & ((1u << b) - 1u);  // unmarked bits below position b
      int hops = 0;
      while (!below && pw > 0 && hops < 64) {
        --pw;
        ++hops;
        below = ~fix_word(mask, pw);
      }
      if (!below) {
        if (hops >= 64) atomicOr(changed, 2u);
        continue;  // no kept predecessor (the run starts the array), or too far
      }
      const int64_t p = pw * 32 + (31 - __clz(below));
      if (Key<KT>::enc(src[p]) > Key<KT>::enc(src[q])) {
        atomicOr(&mask[p >> 5], 1u << (p & 31));
        atomicOr(&mask[q >> 5], 1u << (q & 31));
        atomicOr(changed, 1u);
        atomicAdd(added, 2u);
      }
    }
  }
}

// Marked elements per tile of TILE elements (TILE a multiple of 32).
template <int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS)
fix_tile_count_kernel(const uint32_t* __restrict__ mask, int64_t len, uint32_t* __restrict__ tile_cnt) {
  __shared__ uint32_t wsum[THREADS / 32];
  const int64_t w0 = (int64_t)blockIdx.x * (TILE / 32);
  const int64_t nwords = (len + 31) / 32;
  uint32_t c = 0;
  for (int j = threadIdx.x; j < TILE / 32; j += THREADS) {
    const int64_t w = w0 + j;
    if (w < nwords) c += (uint32_t)__popc(mask[w]);
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < THREADS / 32; ++w) t += wsum[w];
    tile_cnt[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile counts in place (one CTA); *total receives the sum.
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
fix_scan_kernel(uint32_t* __restrict__ tile_cnt, int ntiles, unsigned long long* __restrict__ total) {
  __shared__ uint32_t wtmp[THREADS / 32 + 1];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += THREADS) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < ntiles ? tile_cnt[i] : 0u;
    // inclusive warp scan, then across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wtmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < THREADS / 32 ? wtmp[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < THREADS / 32) wtmp[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = carry + (warp ? wtmp[warp - 1] : 0u) + x - v;
    if (i < ntiles) tile_cnt[i] = excl;
    __syncthreads();
    if (threadIdx.x == THREADS - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Elements whose mask bit is clear go to dst (in order), marked ones to pe[e_off + ...] (in
// order).  Warp w of a tile owns the 32 * PER consecutive elements from t0 + w * 32 * PER; row e
// of the warp is the 32 consecutive elements base + 32 e + lane (coalesced) and one mask word.
template <int KT, int VB, int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS)
fix_compact_kernel(const typename Key<KT>::U* __restrict__ src, const typename Val<VB>::T* __restrict__ srcv,
                   int64_t len, const uint32_t* __restrict__ bits, typename Key<KT>::U* __restrict__ dst,
                   typename Val<VB>::T* __restrict__ dstv, typename Key<KT>::U* __restrict__ pe,
                   typename Val<VB>::T* __restrict__ pev, int64_t e_off, const uint32_t* __restrict__ tile_pre) {
  constexpr int NW = THREADS / 32;
  constexpr int PER = TILE / THREADS;  // rows per warp
  static_assert(TILE % THREADS == 0 && PER <= 32, "tile shape");
  __shared__ uint32_t wcnt[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)warp * 32 * PER;
  uint32_t mask[PER];
  uint32_t peeled = 0;
#pragma unroll
  for (int e = 0; e < PER; ++e) {
    const int64_t i = base + 32 * e + lane;
    const int64_t r0 = base + 32 * e;  // rows are 32-aligned: one mask word each (warp-uniform)
    mask[e] = r0 < len ? bits[r0 >> 5] : 0u;
    (void)i;
    peeled += (uint32_t)__popc(mask[e]);
  }
  if (lane == 0) wcnt[warp] = peeled;
  __syncthreads();
  uint32_t before = tile_pre[blockIdx.x];  // peeled elements before this warp's range
  for (int w = 0; w < warp; ++w) before += wcnt[w];
  const uint32_t lt = (1u << lane) - 1u;
  constexpr int G = 8;  // rows loaded ahead: G independent loads in flight per thread
#pragma unroll
  for (int e0 = 0; e0 < PER; e0 += G) {
    typename Key<KT>::U kx[G];
    typename Val<VB>::T vx[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int64_t i = base + 32 * (e0 + g) + lane;
      if (e0 + g < PER && i < len) {
        kx[g] = src[i];
        if (VB) vx[g] = srcv[i];
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int e = e0 + g;
      if (e < PER) {
        const int64_t i = base + 32 * e + lane;
        const uint32_t p = before + (uint32_t)__popc(mask[e] & lt);  // marked before element i
        if (i < len) {
          if ((mask[e] >> lane) & 1u) {
            pe[e_off + p] = kx[g];
            if (VB) pev[e_off + p] = vx[g];
          } else {
            dst[i - p] = kx[g];
            if (VB) dstv[i - p] = vx[g];
          }
        }
        before += (uint32_t)__popc(mask[e]);
      }
    }
  }
}

// ================================================================== tiled merge
// Merges ascending runs by tiles of TILE = THREADS * ITEMS outputs per CTA (merge path, Odeh et
// al. 2012): the CTA finds where its tile starts and ends on the merge path of its pair by two
// binary searches in global memory, loads both input ranges into shared memory with coalesced
// reads, every thread merges ITEMS outputs from shared memory, and the tile is stored coalesced.
// Pairs: with w > 0 the runs of width w of one array a[0..n) are merged pairwise (2w a multiple
// of TILE); with w == 0 the single pair is a[0..la) and b[0..lb).  raw: inputs are keys (compared
// by their codes, and written back as keys); otherwise they are codes, written decoded when
// `decode` is set.  Ties take A.
template <int KT, int VB>
struct MergeArgs {
  const typename Key<KT>::U* a;
  const typename Val<VB>::T* av;
  int64_t la;
  const typename Key<KT>::U* b;
  const typename Val<VB>::T* bv;
  int64_t lb;
  typename Key<KT>::U* out;
  typename Val<VB>::T* outv;
  int64_t w;  // 0: one pair (a, b); > 0: pairwise runs of a[0..n)
  int64_t n;
  int raw;
  int decode;
};

template <int KS, int VB, int THREADS, int ITEMS>
constexpr size_t merge_tile_smem() {
  return (size_t)2 * THREADS * ITEMS * (KS + VB);
}

// The pair a tile of the merge belongs to: its runs A, B and its first output p0.
template <int KT, int VB>
struct MergePair {
  const typename Key<KT>::U* A;
  const typename Val<VB>::T* Av;
  const typename Key<KT>::U* B;
  const typename Val<VB>::T* Bv;
  int64_t la, lb, p0;
};
template <int KT, int VB>
__device__ __forceinline__ MergePair<KT, VB> merge_pair_of(const MergeArgs<KT, VB>& m, int64_t t0) {
  MergePair<KT, VB> q;
  if (m.w > 0) {
    q.p0 = t0 / (2 * m.w) * (2 * m.w);
    q.la = m.n - q.p0 < m.w ? m.n - q.p0 : m.w;
    q.lb = m.n - q.p0 - q.la < m.w ? m.n - q.p0 - q.la : m.w;
    if (q.lb < 0) q.lb = 0;
    q.A = m.a + q.p0;
    q.Av = VB ? m.av + q.p0 : nullptr;
    q.B = q.A + q.la;
    q.Bv = VB ? q.Av + q.la : nullptr;
  } else {
    q.p0 = 0;
    q.la = m.la;
    q.lb = m.lb;
    q.A = m.a;
    q.Av = m.av;
    q.B = m.b;
    q.Bv = m.bv;
  }
  return q;
}

// Merge-path split (A elements among the first d outputs of the tile's pair) at the start of
// every tile, one thread per tile, all searches in parallel.
template <int KT, int VB, int TILE>
__global__ void merge_split_kernel(MergeArgs<KT, VB> m, int64_t ntiles, int64_t* __restrict__ splits) {
  using U = typename Key<KT>::U;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const MergePair<KT, VB> q = merge_pair_of(m, t * TILE);
  auto code = [&](U x) { return m.raw ? Key<KT>::enc(x) : x; };
  const int64_t d = t * TILE - q.p0;
  int64_t lo = d > q.lb ? d - q.lb : 0, hi = d < q.la ? d : q.la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (!(code(q.B[d - 1 - mid]) < code(q.A[mid]))) lo = mid + 1;
    else hi = mid;
  }
  splits[t] = lo;
}

template <int KT, int VB, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
merge_tile_kernel(MergeArgs<KT, VB> m, const int64_t* __restrict__ splits) {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  constexpr int TILE = THREADS * ITEMS;
  extern __shared__ __align__(16) unsigned char smem[];
  U* sin = reinterpret_cast<U*>(smem);          // A range then B range (codes)
  U* sout = sin + TILE;                         // merged tile (codes)
  V* sinv = reinterpret_cast<V*>(sout + TILE);
  V* soutv = sinv + TILE;

  const int64_t t0 = (int64_t)blockIdx.x * TILE;
  const MergePair<KT, VB> q = merge_pair_of(m, t0);
  const U* A = q.A;
  const V* Av = q.Av;
  const U* B = q.B;
  const V* Bv = q.Bv;
  const int64_t la = q.la, lb = q.lb, p0 = q.p0;
  auto code = [&](U x) { return m.raw ? Key<KT>::enc(x) : x; };
  const int64_t d0 = t0 - p0;
  const int64_t d1 = d0 + TILE < la + lb ? d0 + TILE : la + lb;
  // the tile ends where the next one starts, or at the end of its pair (all of A consumed)
  const int64_t a_lo = splits[blockIdx.x], a_hi = d1 == la + lb ? la : splits[blockIdx.x + 1];
  const int na = (int)(a_hi - a_lo), nb = (int)((d1 - a_hi) - (d0 - a_lo));
  const int64_t b_lo = d0 - a_lo;
  for (int j = threadIdx.x; j < na; j += THREADS) {
    sin[j] = code(A[a_lo + j]);
    if (VB) sinv[j] = Av[a_lo + j];
  }
  for (int j = threadIdx.x; j < nb; j += THREADS) {
    sin[na + j] = code(B[b_lo + j]);
    if (VB) sinv[na + j] = Bv[b_lo + j];
  }
  __syncthreads();
  const int total = na + nb;
  const int d = threadIdx.x * ITEMS;
  if (d < total) {
    const U* sa = sin;
    const U* sb = sin + na;
    int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (!(sb[d - 1 - mid] < sa[mid])) lo = mid + 1;
      else hi = mid;
    }
    int ia = lo, ib = d - lo;
    const int cnt = total - d < ITEMS ? total - d : ITEMS;
#pragma unroll
    for (int e = 0; e < ITEMS; ++e) {
      if (e < cnt) {
        const bool take_a = ia < na && (ib >= nb || !(sb[ib] < sa[ia]));
        const int src = take_a ? ia : na + ib;
        sout[d + e] = sin[src];
        if (VB) soutv[d + e] = sinv[src];
        ia += take_a ? 1 : 0;
        ib += take_a ? 0 : 1;
      }
    }
  }
  __syncthreads();
  U* out = m.out + p0 + d0;
  V* outv = VB ? m.outv + p0 + d0 : nullptr;
  const bool dec = m.raw || m.decode;
  for (int j = threadIdx.x; j < total; j += THREADS) {
    const U c = sout[j];
    out[j] = dec ? Key<KT>::dec(c) : c;
    if (VB) outv[j] = soutv[j];
  }
}

// ================================================================== merge-path pass (fallback)
// Merges consecutive sorted runs of `width` codes of one bucket (n elements, src -> dst), one
// output element per thread: the element at output position d of a pair (A, B) is found by a
// binary search on the merge path (Odeh, Green, Mwassi, Shmueli, Birk, "Merge Path", IPDPSW
// 2012).  Ties take A first.
template <int KT, int VB>
__global__ void merge_pass_kernel(const typename Key<KT>::U* __restrict__ srck,
                                  const typename Val<VB>::T* __restrict__ srcv,
                                  typename Key<KT>::U* __restrict__ dstk, typename Val<VB>::T* __restrict__ dstv,
                                  int64_t n, int64_t width, int decode) {
  using U = typename Key<KT>::U;
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int64_t pair0 = (o / (2 * width)) * (2 * width);
  const int64_t a0 = pair0;
  const int64_t la = min(width, n - a0);
  const int64_t b0 = a0 + la;
  const int64_t lb = min(width, n - b0 < 0 ? 0 : n - b0);
  const int64_t d = o - pair0;
  int64_t lo = d - lb > 0 ? d - lb : 0;
  int64_t hi = d < la ? d : la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (srck[a0 + mid] <= srck[b0 + d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  const int64_t i = lo, j = d - lo;
  int64_t src;
  if (i < la && (j >= lb || srck[a0 + i] <= srck[b0 + j])) src = a0 + i;
  else src = b0 + j;
  const U k = srck[src];
  dstk[o] = decode ? Key<KT>::dec(k) : k;
  if (VB) dstv[o] = srcv[src];
}

}  // namespace pdq
