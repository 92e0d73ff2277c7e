// Device kernels of the sort (templates; instantiated per key dtype and payload width).
//
// Data-parallel form of pattern-defeating quicksort (Peters, arXiv 2106.05123):
//   probe_kernel      - descents / ascents / min / max over neighbours: the sorted and
//                       reverse-sorted exits (Sec. 5.2)
//   reverse_kernel    - in-place reversal for non-increasing input (Sec. 5.2)
//   sample_kernel     - splitter selection from a hashed sample, sorted in shared memory; a
//                       multi-way generalisation of median-of-k pivots (Sec. 2) with fresh
//                       samples per attempt (Sec. 4.2)
//   count_kernel      - branchless classification of every key into 2B bins: bin 2b holds keys
//                       strictly between splitters b-1 and b, bin 2b+1 keys equal to splitter b
//                       (the equal-key rule of Sec. 3)
//   scan_kernel       - bucket offsets per (chunk, bin)
//   scatter_kernel    - re-classifies a tile, ranks keys per bin with shared atomics, stages the
//                       tile in shared memory grouped by bin and writes contiguous runs
//                       (the GPU form of block partitioning, Sec. 5.3)
//   bookkeep_kernel   - equal bins are final; small bins go to the base sort; a bin keeping
//                       more than 7/8 of its parent is a bad split and decrements the subtree's
//                       counter; at 0 the bin goes to the fallback (Sec. 4.1)
//   base_sort_kernel  - shared-memory sort of a small bucket (Sec. 5.1)
//   merge_pass_kernel - merge-path merge pass of the O(n log n) fallback (Sec. 4.1)
#pragma once

#include "common.cuh"

namespace pdq {

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

// Exclusive scan of nbins counters held in shared memory `in`, result in `out` (may alias).
// Returns the total in *total (shared).  All threads of the block must call it.
template <int THREADS>
__device__ void block_exclusive_scan(const uint32_t* in, uint32_t* out, int nbins,
                                     uint32_t* warp_tmp /* >= THREADS/32 + 1 */) {
  const int tid = threadIdx.x;
  const int per = (nbins + THREADS - 1) / THREADS;
  const int lo = tid * per;
  uint32_t sum = 0;
  for (int i = 0; i < per; ++i) {
    const int b = lo + i;
    if (b < nbins) sum += in[b];
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
      const uint32_t c = in[b];
      out[b] = run;
      run += c;
    }
  }
  __syncthreads();
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
  for (int64_t j = gt; j < m; j += gs) {
    const U x = Key<KT>::enc(__ldg(a + j * stride));
    mn = x < mn ? x : mn;
    mx = x > mx ? x : mx;
    if (j + 1 < m) {
      const U y = Key<KT>::enc(__ldg(a + (j + 1) * stride));
      desc += x > y;
      asc += x < y;
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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < half;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = n - 1 - i;
    const T x = a[i], y = a[j];
    a[i] = y;
    a[j] = x;
  }
}

// ================================================================== classification
// Eytzinger tree over the B-1 sorted splitters: tree[1..B-1], node j has children 2j and 2j+1.
// Descent "go right when code > node" ends at leaf B + b where b = #splitters < code.  The key
// then belongs to bin 2b+1 if it equals splitter b (an equality bucket, Sec. 3), else bin 2b.
template <class U>
__device__ __forceinline__ int classify(U code, const U* __restrict__ tree,
                                        const U* __restrict__ spl, int logb) {
  int j = 1;
  for (int l = 0; l < logb; ++l) j = 2 * j + (code > tree[j] ? 1 : 0);
  const int B = 1 << logb;
  const int b = j - B;
  const int sb = b < B - 1 ? b : B - 2;
  return 2 * b + (code == spl[sb] ? 1 : 0);
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
// repeats as a splitter: its keys all go to its equality bin.
template <int KT, int THREADS>
__global__ void __launch_bounds__(THREADS)
sample_kernel(const Task* __restrict__ tasks, const int32_t* __restrict__ task_logb, int oversample,
              const typename Key<KT>::U* __restrict__ keys, const typename Key<KT>::U* __restrict__ tmp,
              typename Key<KT>::U* __restrict__ tree_out, typename Key<KT>::U* __restrict__ spl_out) {
  using U = typename Key<KT>::U;
  __shared__ U s[kMaxSamples];
  const Task t = tasks[blockIdx.x];
  const int logb = task_logb[blockIdx.x];
  const int B = 1 << logb;
  int ns = oversample * B;
  if (ns > kMaxSamples) ns = kMaxSamples;
  if (ns < B) ns = B;
  const U* src = (t.buf == kBufKeys ? keys : tmp) + t.begin;
  const uint64_t seed = mix64((uint64_t)t.begin * 0x9E3779B97F4A7C15ull ^ mix64((uint64_t)t.size) ^
                              ((uint64_t)t.attempt << 48));
  for (int j = threadIdx.x; j < ns; j += THREADS) {
    const uint64_t r = mix64(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull);
    const int64_t pos = (int64_t)(r % (uint64_t)t.size);
    const U x = src[pos];
    s[j] = t.enc ? x : Key<KT>::enc(x);
  }
  __syncthreads();
  // bitonic sort of s[0..ns), ns a power of two
  for (int k = 2; k <= ns; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = threadIdx.x; q < ns / 2; q += THREADS) {
        const int i = (q / j) * 2 * j + (q % j);
        const int l = i + j;
        const bool up = (i & k) == 0;
        const U a = s[i], b = s[l];
        if ((a > b) == up) { s[i] = b; s[l] = a; }
      }
      __syncthreads();
    }
  }
  U* tree = tree_out + (size_t)blockIdx.x * kBMax;
  U* spl = spl_out + (size_t)blockIdx.x * kBMax;
  const int step = ns / B;
  for (int i = threadIdx.x; i < B - 1; i += THREADS) spl[i] = s[(i + 1) * step - 1];
  for (int j = 1 + threadIdx.x; j < B; j += THREADS) tree[j] = s[(eytz_inorder(j, logb) + 1) * step - 1];
}

// Loads the task's tree and splitters into shared memory.
template <class U>
__device__ __forceinline__ void load_splitters(U* s_tree, U* s_spl, const U* tree, const U* spl, int B) {
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    s_tree[j] = tree[j];
    s_spl[j] = spl[j];
  }
}

// ================================================================== count
template <int KT, int THREADS>
__global__ void __launch_bounds__(THREADS)
count_kernel(const Chunk* __restrict__ chunks, const Task* __restrict__ tasks,
             const int32_t* __restrict__ task_logb, const typename Key<KT>::U* __restrict__ keys,
             const typename Key<KT>::U* __restrict__ tmp, const typename Key<KT>::U* __restrict__ tree_g,
             const typename Key<KT>::U* __restrict__ spl_g, uint32_t* __restrict__ counts) {
  using U = typename Key<KT>::U;
  __shared__ U s_tree[kBMax], s_spl[kBMax];
  __shared__ uint32_t hist[kBinsMax];
  const Chunk c = chunks[blockIdx.x];
  const Task t = tasks[c.task];
  const int logb = task_logb[c.task];
  const int B = 1 << logb;
  const int nb = 2 * B;
  load_splitters(s_tree, s_spl, tree_g + (size_t)c.task * kBMax, spl_g + (size_t)c.task * kBMax, B);
  for (int b = threadIdx.x; b < nb; b += THREADS) hist[b] = 0;
  __syncthreads();
  const U* src = (t.buf == kBufKeys ? keys : tmp) + c.begin;
  if (t.enc) {
    for (int i = threadIdx.x; i < c.size; i += THREADS)
      atomicAdd(&hist[classify(src[i], s_tree, s_spl, logb)], 1u);
  } else {
    for (int i = threadIdx.x; i < c.size; i += THREADS)
      atomicAdd(&hist[classify(Key<KT>::enc(src[i]), s_tree, s_spl, logb)], 1u);
  }
  __syncthreads();
  uint32_t* out = counts + (size_t)blockIdx.x * kBinsMax;
  for (int b = threadIdx.x; b < nb; b += THREADS) out[b] = hist[b];
}

// ================================================================== scan
// One CTA per task: bin totals over the task's chunks, bin starts, and per-chunk write offsets
// (relative to the task's first element), written over the counts.  Child (start, size) pairs
// go to children[task][bin].
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
scan_kernel(const int32_t* __restrict__ task_logb, const int32_t* __restrict__ task_chunk0,
            const int32_t* __restrict__ task_nchunks, uint32_t* __restrict__ counts,
            uint2* __restrict__ children) {
  __shared__ uint32_t tot[kBinsMax];
  __shared__ uint32_t start[kBinsMax];
  __shared__ uint32_t wtmp[THREADS / 32 + 1];
  const int task = blockIdx.x;
  const int nb = 2 << task_logb[task];
  const int c0 = task_chunk0[task], nc = task_nchunks[task];
  for (int b = threadIdx.x; b < nb; b += THREADS) {
    uint32_t s = 0;
    for (int c = 0; c < nc; ++c) s += counts[(size_t)(c0 + c) * kBinsMax + b];
    tot[b] = s;
  }
  __syncthreads();
  block_exclusive_scan<THREADS>(tot, start, nb, wtmp);
  for (int b = threadIdx.x; b < nb; b += THREADS) {
    uint32_t run = start[b];
    for (int c = 0; c < nc; ++c) {
      uint32_t* p = counts + (size_t)(c0 + c) * kBinsMax + b;
      const uint32_t v = *p;
      *p = run;
      run += v;
    }
    children[(size_t)task * kBinsMax + b] = make_uint2(start[b], tot[b]);
  }
}

// ================================================================== scatter
// One CTA per chunk; the chunk is processed in tiles of TILE = ITEMS * THREADS elements.
template <int KT, int VB, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
scatter_kernel(const Chunk* __restrict__ chunks, const Task* __restrict__ tasks,
               const int32_t* __restrict__ task_logb, typename Key<KT>::U* __restrict__ keys,
               typename Val<VB>::T* __restrict__ vals, typename Key<KT>::U* __restrict__ tmpk,
               typename Val<VB>::T* __restrict__ tmpv, const typename Key<KT>::U* __restrict__ tree_g,
               const typename Key<KT>::U* __restrict__ spl_g, const uint32_t* __restrict__ offsets) {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  constexpr int TILE = THREADS * ITEMS;
  extern __shared__ __align__(16) unsigned char smem[];
  U* stage_k = reinterpret_cast<U*>(smem);
  V* stage_v = reinterpret_cast<V*>(stage_k + TILE);
  uint16_t* stage_b = reinterpret_cast<uint16_t*>(VB ? (unsigned char*)(stage_v + TILE) : (unsigned char*)(stage_k + TILE));
  __shared__ U s_tree[kBMax], s_spl[kBMax];
  __shared__ uint32_t hist[kBinsMax];     // per-tile counts, then tile bin starts
  __shared__ uint32_t cursor[kBinsMax];   // next write offset per bin (task-relative)
  __shared__ uint32_t gbase[kBinsMax];    // cursor - tile start, per bin
  __shared__ uint32_t wtmp[THREADS / 32 + 1];

  const Chunk c = chunks[blockIdx.x];
  const Task t = tasks[c.task];
  const int logb = task_logb[c.task];
  const int B = 1 << logb;
  const int nb = 2 * B;
  load_splitters(s_tree, s_spl, tree_g + (size_t)c.task * kBMax, spl_g + (size_t)c.task * kBMax, B);
  for (int b = threadIdx.x; b < nb; b += THREADS) cursor[b] = offsets[(size_t)blockIdx.x * kBinsMax + b];

  const bool from_keys = t.buf == kBufKeys;
  const U* srck = (from_keys ? keys : tmpk) + c.begin;
  const V* srcv = VB ? (from_keys ? vals : tmpv) + c.begin : nullptr;
  U* dstk = (from_keys ? tmpk : keys) + t.begin;
  V* dstv = VB ? (from_keys ? tmpv : vals) + t.begin : nullptr;
  const bool dst_is_keys = !from_keys;

  for (int tile0 = 0; tile0 < c.size; tile0 += TILE) {
    const int cnt = min(TILE, c.size - tile0);
    for (int b = threadIdx.x; b < nb; b += THREADS) hist[b] = 0;
    __syncthreads();
    U code[ITEMS];
    V val[ITEMS];
    int bin[ITEMS];
    uint32_t rank[ITEMS];
#pragma unroll
    for (int e = 0; e < ITEMS; ++e) {
      const int i = e * THREADS + threadIdx.x;
      if (i < cnt) {
        const U x = srck[tile0 + i];
        code[e] = t.enc ? x : Key<KT>::enc(x);
        if (VB) val[e] = srcv[tile0 + i];
        bin[e] = classify(code[e], s_tree, s_spl, logb);
        rank[e] = atomicAdd(&hist[bin[e]], 1u);
      }
    }
    __syncthreads();
    block_exclusive_scan<THREADS>(hist, hist, nb, wtmp);  // hist := tile start of each bin
    for (int b = threadIdx.x; b < nb; b += THREADS) {
      const uint32_t next = (b + 1 < nb) ? hist[b + 1] : (uint32_t)cnt;
      gbase[b] = cursor[b] - hist[b];
      cursor[b] += next - hist[b];
    }
#pragma unroll
    for (int e = 0; e < ITEMS; ++e) {
      const int i = e * THREADS + threadIdx.x;
      if (i < cnt) {
        const uint32_t p = hist[bin[e]] + rank[e];
        stage_k[p] = code[e];
        if (VB) stage_v[p] = val[e];
        stage_b[p] = (uint16_t)bin[e];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += THREADS) {
      const int b = stage_b[i];
      const uint32_t o = gbase[b] + (uint32_t)i;
      U k = stage_k[i];
      if (dst_is_keys && (b & 1)) k = Key<KT>::dec(k);  // equality bin: final, decode now
      dstk[o] = k;
      if (VB) dstv[o] = stage_v[i];
    }
    __syncthreads();
  }
}

// ================================================================== bookkeeping (Sec. 4.1, Sec. 3)
static __global__ void bookkeep_kernel(const Task* __restrict__ tasks, const int32_t* __restrict__ task_logb,
                                const uint2* __restrict__ children, int base_cap, Counters* ctr,
                                Task* __restrict__ next, Item* __restrict__ base_items,
                                Item* __restrict__ copy_items, Item* __restrict__ fb_items,
                                int64_t task_cap, int64_t item_cap) {
  const int task = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = 2 << task_logb[task];
  if (b >= nb) return;
  const uint2 ch = children[(size_t)task * kBinsMax + b];
  if (ch.y == 0) return;
  const Task t = tasks[task];
  const int dst = t.buf == kBufKeys ? kBufTmp : kBufKeys;
  Item it;
  it.begin = t.begin + ch.x;
  it.size = ch.y;
  it.buf = (uint16_t)dst;
  it.enc = 1;
  auto push = [&](Item* list, unsigned long long* counter) {
    const unsigned long long k = atomicAdd(counter, 1ull);
    if ((int64_t)k < item_cap) list[k] = it;
    else atomicAdd(&ctr->overflow, 1ull);
  };
  if (b & 1) {  // equality bucket: every key equals the splitter, final (Sec. 3)
    atomicAdd(&ctr->equal_buckets, 1ull);
    if (dst == kBufTmp) {
      push(copy_items, &ctr->n_copy);
      atomicAdd(&ctr->copy_elems, (unsigned long long)ch.y);
    }
    return;
  }
  if ((int64_t)ch.y <= base_cap) {
    push(base_items, &ctr->n_base[0]);
    atomicAdd(&ctr->base_elems, (unsigned long long)ch.y);
    return;
  }
  // bad split: the child kept more than 7/8 of its parent (p = 1/8, a shift; Sec. 4.1)
  const bool bad = (int64_t)ch.y > t.size - (t.size >> 3);
  if (bad) atomicAdd(&ctr->bad_splits, 1ull);
  const int left = t.bad_left - (bad ? 1 : 0);
  if (left <= 0) {
    push(fb_items, &ctr->n_fallback);
    return;
  }
  Task nt;
  nt.begin = it.begin;
  nt.size = it.size;
  nt.buf = dst;
  nt.enc = 1;
  nt.bad_left = left;
  nt.attempt = t.attempt + 1;
  const unsigned long long k = atomicAdd(&ctr->n_next, 1ull);
  if ((int64_t)k < task_cap) next[k] = nt;
  else atomicAdd(&ctr->overflow, 1ull);
}

// ================================================================== base sort (Sec. 5.1)
// One CTA per item of at most CAP elements: load into shared memory (encoding raw keys), pad to
// a power of two with the largest code, bitonic-sort, write to the output buffer (decoded when
// `decode`).  With a payload, the sort key is (code, index) so padding sorts after real keys and
// values are gathered through the index.
template <int KT, int VB, int THREADS>
__global__ void __launch_bounds__(THREADS)
base_sort_kernel(const Item* __restrict__ items, int cap, typename Key<KT>::U* __restrict__ keys,
                 typename Val<VB>::T* __restrict__ vals, typename Key<KT>::U* __restrict__ tmpk,
                 typename Val<VB>::T* __restrict__ tmpv, int out_buf, int decode) {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  U* sk = reinterpret_cast<U*>(smem);
  V* sv = reinterpret_cast<V*>(sk + cap);
  uint32_t* si = reinterpret_cast<uint32_t*>(VB ? (unsigned char*)(sv + cap) : (unsigned char*)(sk + cap));
  const Item it = items[blockIdx.x];
  const int m = (int)it.size;
  const int P = (int)next_pow2_u32(m < 2 ? 2 : (uint32_t)m);
  const U* srck = (it.buf == kBufKeys ? keys : tmpk) + it.begin;
  const V* srcv = VB ? (it.buf == kBufKeys ? vals : tmpv) + it.begin : nullptr;
  for (int i = threadIdx.x; i < P; i += THREADS) {
    if (i < m) {
      const U x = srck[i];
      sk[i] = it.enc ? x : Key<KT>::enc(x);
      if (VB) sv[i] = srcv[i];
    } else {
      sk[i] = ~U(0);
    }
    if (VB) si[i] = i;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = threadIdx.x; q < P / 2; q += THREADS) {
        const int i = (q / j) * 2 * j + (q % j);
        const int l = i + j;
        const bool up = (i & k) == 0;
        const U a = sk[i], b = sk[l];
        bool gt;
        if (VB) gt = a > b || (a == b && si[i] > si[l]);
        else gt = a > b;
        if (gt == up) {
          sk[i] = b;
          sk[l] = a;
          if (VB) { const uint32_t x = si[i]; si[i] = si[l]; si[l] = x; }
        }
      }
      __syncthreads();
    }
  }
  U* dstk = (out_buf == kBufKeys ? keys : tmpk) + it.begin;
  V* dstv = VB ? (out_buf == kBufKeys ? vals : tmpv) + it.begin : nullptr;
  for (int i = threadIdx.x; i < m; i += THREADS) {
    const U k = sk[i];
    dstk[i] = decode ? Key<KT>::dec(k) : k;
    if (VB) dstv[i] = sv[si[i]];
  }
}

// ================================================================== copy temp -> keys (decode)
template <int KT, int VB>
__global__ void copy_kernel(const Item* __restrict__ items, typename Key<KT>::U* __restrict__ keys,
                            typename Val<VB>::T* __restrict__ vals, const typename Key<KT>::U* __restrict__ tmpk,
                            const typename Val<VB>::T* __restrict__ tmpv) {
  const Item it = items[blockIdx.x];
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < it.size;
       i += (int64_t)gridDim.y * blockDim.x) {
    const int64_t p = it.begin + i;
    keys[p] = Key<KT>::dec(tmpk[p]);
    if (VB) vals[p] = tmpv[p];
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
