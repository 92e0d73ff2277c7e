// Batched segmented sort: many independent segments in one persistent launch.
//
// Every segment is a task.  A binning kernel puts each segment into a size-binned device queue:
// segments that fit the shared-memory base sort go to the base queue, larger ones (up to a
// limit) to the partition queue, and very large ones to a list the host sorts with the plain
// multi-CTA path.  The persistent kernel's CTAs then pull tasks (partition queue first):
//   base task      - the CTA sorts the bucket in shared memory (Sec. 5.1) into the key buffer;
//   partition task - the CTA runs one distribution level on its own: hashed sample, splitters,
//                    count, scan, scatter into the other buffer (Sec. 3 equal-key bins are
//                    finished on the spot), and pushes the children; a child that keeps more
//                    than 7/8 of its parent's non-equal keys costs one unit of the subtree's
//                    bad-split budget,
//                    and at 0 it goes to the host's O(n log n) fallback (Sec. 4.1).
// Queue slots carry ready flags; every wait is bounded in time.  If a wait gives up, the
// kernel records a timeout and switches to salvage mode: remaining tasks only move their data
// back to the key buffer, so the arrays always end as a permutation of the input.
#pragma once

#include "kernels.cuh"

namespace pdq {

enum SegKind : uint8_t { kSegBase = 0, kSegPart = 2 };

struct __align__(8) SegTask {
  int64_t begin;
  uint32_t size;
  uint8_t buf, enc, kind, bad_left;
  uint32_t attempt;
  uint32_t depth;
};
static_assert(sizeof(SegTask) == 24, "a queue slot is three 8-byte words");

struct SegQueue {
  unsigned long long head, tail;
};

struct SegState {
  SegQueue q[2];                    // 0: partition tasks, 1: base tasks
  unsigned long long outstanding;   // tasks published and not yet finished
  unsigned long long error;         // bit 0: a bounded wait expired, bit 1: list overflow, bit 2: bad offsets
  unsigned long long n_fallback;
  unsigned long long n_huge;
  unsigned long long equal_buckets;
  unsigned long long base_buckets;
  unsigned long long partitions;
  unsigned long long bad_splits;
  unsigned long long max_depth;
  unsigned long long never_set;     // written by nobody: the wait-injection hook waits on it
  unsigned long long n_blist[kBaseClasses];  // entries appended to each base-size class list
};

struct SegLists {
  SegTask* slots[2];
  uint32_t* ready[2];
  int64_t cap[2];
  Item* fallback;
  int64_t fb_cap;
  Item* huge;
  int64_t huge_cap;
  // buckets of at most max_base elements, binned by size class (1024 << c) for the
  // class-shaped base-sort kernels that run after the persistent kernel
  Item* blist[kBaseClasses];
  int64_t bcap[kBaseClasses];
  int64_t max_base;
};

struct SegParams {
  int max_logb;
  int oversample;
  int bad0;            // >0 forced budget, -1 start at 0, 0 floor(log2 size)
  int inject_wait;     // test hook: CTA 0 first waits on a flag nobody sets
  int64_t persist_max; // largest segment handled inside the persistent kernel
  uint64_t wait_ns;    // bound of every wait
};

__device__ __forceinline__ uint64_t seg_now() { return global_ns(); }

__device__ __forceinline__ bool seg_push(SegState* st, const SegLists& L, int qi, const SegTask& t) {
  const unsigned long long slot = atomicAdd(&st->q[qi].tail, 1ull);
  if ((int64_t)slot >= L.cap[qi]) return false;  // consumers never claim slots >= cap
  atomicAdd(&st->outstanding, 1ull);              // counted before it can be claimed
  L.slots[qi][slot] = t;
  __threadfence();
  atomicExch(&L.ready[qi][slot], 1u);
  return true;
}

__device__ __forceinline__ bool list_push(unsigned long long* counter, Item* list, int64_t cap, const Item& it) {
  const unsigned long long k = atomicAdd(counter, 1ull);
  if ((int64_t)k >= cap) return false;
  list[k] = it;
  return true;
}

__device__ __forceinline__ int seg_base_class(int64_t m) {
  return m <= 1024 ? 0 : (m <= 2048 ? 1 : (m <= 4096 ? 2 : (m <= 8192 ? 3 : 4)));
}

// Appends a base-size bucket to its size-class list; false when that list is full.
__device__ __forceinline__ bool seg_base_push(SegState* st, const SegLists& L, const Item& it) {
  const int c = seg_base_class(it.size);
  return list_push(&st->n_blist[c], L.blist[c], L.bcap[c], it);
}

// Claims the next published slot of queue qi (thread 0 only).  0: got a task, 1: empty,
// 2: a claimed slot's ready flag did not appear in time.
static __device__ int seg_try_pop(SegState* st, const SegLists& L, int qi, SegTask* out, uint64_t wait_ns) {
  volatile unsigned long long* vh = &st->q[qi].head;
  volatile unsigned long long* vt = &st->q[qi].tail;
  for (int tries = 0; tries < 64; ++tries) {
    const unsigned long long h = *vh;
    unsigned long long t = *vt;
    if (t > (unsigned long long)L.cap[qi]) t = (unsigned long long)L.cap[qi];
    if (h >= t) return 1;
    if (atomicCAS((unsigned long long*)vh, h, h + 1) != h) continue;
    volatile uint32_t* rf = &L.ready[qi][h];
    if (*rf == 0) {
      const uint64_t t0 = seg_now();
      while (*rf == 0)
        if (seg_now() - t0 > wait_ns) return 2;
    }
    __threadfence();
    // the slot was written after this SM may have cached its line: read it from L2
    const unsigned long long* w = reinterpret_cast<const unsigned long long*>(&L.slots[qi][h]);
    unsigned long long* o = reinterpret_cast<unsigned long long*>(out);
    o[0] = __ldcg(w);
    o[1] = __ldcg(w + 1);
    o[2] = __ldcg(w + 2);
    return 0;
  }
  return 1;
}

// ------------------------------------------------------------------ binning
template <int KT>
__global__ void seg_bin_kernel(const int64_t* __restrict__ offsets, int64_t nseg, int64_t n, int cap,
                               SegParams prm, SegState* st, SegLists L) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = offsets[s], e = offsets[s + 1];
    if (b < 0 || e < b || e > n) {
      atomicOr(&st->error, 4ull);
      continue;
    }
    const int64_t size = e - b;
    if (size <= 1) continue;
    const int bad0 = prm.bad0 > 0 ? prm.bad0 : (prm.bad0 < 0 ? 0 : ilog2_floor((uint64_t)size));
    SegTask t;
    t.begin = b;
    t.size = (uint32_t)size;
    t.buf = kBufKeys;
    t.enc = 0;
    t.bad_left = (uint8_t)(bad0 > 255 ? 255 : bad0);
    t.attempt = 0;
    t.depth = 0;
    Item it{b, (uint32_t)size, (uint16_t)kBufKeys, 0};
    if (size <= L.max_base && seg_base_push(st, L, it)) continue;
    if (size <= cap) {  // its class list is full: the persistent kernel sorts it
      t.kind = kSegBase;
      if (!seg_push(st, L, 1, t) && !list_push(&st->n_fallback, L.fallback, L.fb_cap, it))
        atomicOr(&st->error, 2ull);
    } else if (size > prm.persist_max) {
      if (!list_push(&st->n_huge, L.huge, L.huge_cap, it)) atomicOr(&st->error, 2ull);
    } else if (bad0 == 0) {
      if (!list_push(&st->n_fallback, L.fallback, L.fb_cap, it)) atomicOr(&st->error, 2ull);
    } else {
      t.kind = kSegPart;
      if (!seg_push(st, L, 0, t) && !list_push(&st->n_fallback, L.fallback, L.fb_cap, it))
        atomicOr(&st->error, 2ull);
    }
  }
}

// ------------------------------------------------------------------ one-CTA distribution level
// Elements per streamed tile of the one-CTA partition (two slots of it hold the 4096 samples).
constexpr int kSegTile = 2048;

template <int KT, int VB, int THREADS>
__device__ void seg_partition(const SegTask& t, const SegParams& prm, int cap, typename Key<KT>::U* keys,
                              typename Val<VB>::T* vals, typename Key<KT>::U* tmpk, typename Val<VB>::T* tmpv,
                              unsigned char* smem, uint32_t* wtmp, SegState* st, const SegLists& L) {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  constexpr int T = kSegTile;      // elements per streamed tile
  constexpr int ITP = T / THREADS;  // elements per thread per tile
  static_assert(T % THREADS == 0 && 2 * T >= kMaxSamples, "tile shape");
  // shared memory: two stream slots (keys, then values; the samples live there first), tree,
  // splitters, staged tile (keys, values), per-bin totals / cursors / tile counts, staged bins
  U* kslot = reinterpret_cast<U*>(smem);
  V* vslot = reinterpret_cast<V*>(kslot + 2 * T);
  U* s = kslot;
  U* s_tree = reinterpret_cast<U*>(reinterpret_cast<unsigned char*>(vslot) + (size_t)2 * T * VB);
  U* s_spl = s_tree + kBMax;
  U* sk = s_spl + kBMax;
  V* sv = reinterpret_cast<V*>(sk + T);
  uint32_t* hist = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(sv) + (size_t)T * VB);
  uint32_t* curs = hist + kBinsMax;  // global write cursor per bin
  uint32_t* th = curs + kBinsMax;    // tile count, then tile start, per bin
  uint16_t* sb = reinterpret_cast<uint16_t*>(th + kBinsMax);
  const int tid = threadIdx.x;
  const int64_t size = t.size;
  // buckets: expected child a quarter of the largest base-size bucket
  int logb = 1;
  {
    const int64_t q = L.max_base / 4;
    const int64_t want = (size + q - 1) / q;
    while ((int64_t(1) << logb) < want && logb < prm.max_logb) ++logb;
  }
  const int B = 1 << logb;
  const int nb = 2 * B;
  const BinSlot<true> slot{logb};  // hist, curs and th are indexed by bin slot (bank spread)
  int ns = prm.oversample * B;
  if (ns > kMaxSamples) ns = kMaxSamples;
  if (ns < B) ns = B;
  const bool from_keys = t.buf == kBufKeys;
  const U* srck = (from_keys ? keys : tmpk) + t.begin;
  const V* srcv = VB ? (from_keys ? vals : tmpv) + t.begin : nullptr;
  U* dstk = (from_keys ? tmpk : keys) + t.begin;
  V* dstv = VB ? (from_keys ? tmpv : vals) + t.begin : nullptr;
  const bool enc = t.enc != 0;

  // hashed sample, sorted in shared memory (fresh per attempt, Sec. 4.2)
  const uint64_t seed = mix64((uint64_t)t.begin * 0x9E3779B97F4A7C15ull ^ mix64((uint64_t)t.size) ^
                              ((uint64_t)t.attempt << 48));
  for (int j = tid; j < ns; j += THREADS) {
    const uint64_t r = mix64(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull);
    const U x = srck[(int64_t)(r % (uint64_t)size)];
    s[j] = enc ? x : Key<KT>::enc(x);
  }
  __syncthreads();
  for (int k = 2; k <= ns; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int q = tid; q < ns / 2; q += THREADS) {
        const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));  // j is a power of two
        const int l = i + j;
        const bool up = (i & k) == 0;
        const U a = s[i], b = s[l];
        if ((a > b) == up) { s[i] = b; s[l] = a; }
      }
      __syncthreads();
    }
  }
  const int step = ns / B;
  for (int i = tid; i < B - 1; i += THREADS) s_spl[i] = s[(i + 1) * step - 1];
  for (int j = 1 + tid; j < B; j += THREADS) s_tree[j] = s[(eytz_inorder(j, logb) + 1) * step - 1];
  for (int b = tid; b < nb; b += THREADS) hist[b] = 0;
  __syncthreads();
  // Both passes stream the segment through the two slots with cp.async: tile k+1 is in flight
  // while tile k is processed (every thread commits one group per tile, possibly empty).
  auto fetch = [&](int64_t t0, int slot, bool with_vals) {
#pragma unroll
    for (int e = 0; e < ITP; ++e) {
      const int j = e * THREADS + tid;
      const int64_t i = t0 + j;
      if (i < size) {
        cp_async<sizeof(U)>(&kslot[slot * T + j], &srck[i]);
        if constexpr (VB > 0) {
          if (with_vals) cp_async<VB>(&vslot[slot * T + j], &srcv[i]);
        }
      }
    }
    cp_async_commit();
  };
  // count
  with_logb(logb, [&](auto LB) {
    constexpr int LL = decltype(LB)::value;
    fetch(0, 0, false);
    int k = 0;
    for (int64_t t0 = 0; t0 < size; t0 += T, ++k) {
      if (t0 + T < size) fetch(t0 + T, (k + 1) & 1, false);
      else cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      const U* kb = kslot + (k & 1) * T;
#pragma unroll
      for (int e = 0; e < ITP; ++e) {
        const int j = e * THREADS + tid;
        if (t0 + j < size) {
          const U x = kb[j];
          atomicAdd(&hist[slot(classify_t<LL>(enc ? x : Key<KT>::enc(x), s_tree, s_spl))], 1u);
        }
      }
      __syncthreads();
    }
    cp_async_wait<0>();
  });
  __syncthreads();
  block_exclusive_scan<THREADS>(hist, curs, nb, wtmp, slot);  // curs := bin starts
  // scatter, one tile at a time: rank inside the tile per bin, stage grouped by bin in shared
  // memory, then write each bin's run of the tile at its cursor (contiguous stores); equality
  // bins written to the key buffer are final, so they are decoded on the way
  const bool dst_is_keys = !from_keys;
  with_logb(logb, [&](auto LB) {
    constexpr int LL = decltype(LB)::value;
    fetch(0, 0, true);
    int k = 0;
    for (int64_t t0 = 0; t0 < size; t0 += T, ++k) {
      const int cnt = (int)(size - t0 < T ? size - t0 : T);
      for (int b = tid; b < nb; b += THREADS) th[b] = 0;
      if (t0 + T < size) fetch(t0 + T, (k + 1) & 1, true);
      else cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      const U* kb = kslot + (k & 1) * T;
      const V* vb = vslot + (k & 1) * T;
      int bin[ITP];  // bin slots
      uint32_t rk[ITP];
#pragma unroll
      for (int e = 0; e < ITP; ++e) {
        const int j = e * THREADS + tid;
        if (j < cnt) {
          const U x = kb[j];
          bin[e] = slot(classify_t<LL>(enc ? x : Key<KT>::enc(x), s_tree, s_spl));
          rk[e] = atomicAdd(&th[bin[e]], 1u);
        }
      }
      __syncthreads();
      block_exclusive_scan<THREADS>(th, th, nb, wtmp, slot);  // th := tile starts
#pragma unroll
      for (int e = 0; e < ITP; ++e) {
        const int j = e * THREADS + tid;
        if (j < cnt) {
          const U x = kb[j];
          const U code = enc ? x : Key<KT>::enc(x);
          const uint32_t p = th[bin[e]] + rk[e];
          sk[p] = (dst_is_keys && slot.equal(bin[e])) ? Key<KT>::dec(code) : code;
          sb[p] = (uint16_t)bin[e];
          if (VB) sv[p] = vb[j];
        }
      }
      __syncthreads();
      for (int j = tid; j < cnt; j += THREADS) {
        const int b = sb[j];
        const uint32_t g = curs[b] + (uint32_t)j - th[b];
        dstk[g] = sk[j];
        if (VB) dstv[g] = sv[j];
      }
      __syncthreads();
      for (int b = tid; b < nb; b += THREADS) {
        const int sl = slot(b);
        curs[sl] += (b + 1 < nb ? th[slot(b + 1)] : (uint32_t)cnt) - th[sl];
      }
      __syncthreads();
    }
    cp_async_wait<0>();
  });
  __syncthreads();
  // the parent's keys outside its equality bins, for the bad-split rule (Sec. 4.1)
  __shared__ unsigned long long s_equal;
  if (tid == 0) s_equal = 0ull;
  __syncthreads();
  {
    unsigned long long e = 0ull;
    for (int b = 2 * tid + 1; b < nb; b += 2 * THREADS) e += hist[slot(b)];
    e = warp_sum(e);
    if ((tid & 31) == 0 && e) atomicAdd(&s_equal, e);
  }
  __syncthreads();
  const int64_t nonequal = size - (int64_t)s_equal;
  // children
  for (int b = tid; b < nb; b += THREADS) {
    const uint32_t cnt = hist[slot(b)];
    if (cnt == 0) continue;
    const uint32_t start = curs[slot(b)] - cnt;
    Item it{t.begin + start, cnt, (uint16_t)(from_keys ? kBufTmp : kBufKeys), 1};
    if (b & 1) {
      atomicAdd(&st->equal_buckets, 1ull);
      continue;  // copied below when it sits in the temp buffer
    }
    SegTask c;
    c.begin = it.begin;
    c.size = cnt;
    c.buf = (uint8_t)it.buf;
    c.enc = 1;
    c.attempt = t.attempt + 1;
    c.depth = t.depth + 1;
    if ((int64_t)cnt <= L.max_base && seg_base_push(st, L, it)) continue;
    if ((int64_t)cnt <= cap) {  // its class list is full: the persistent kernel sorts it
      c.kind = kSegBase;
      c.bad_left = t.bad_left;
      if (!seg_push(st, L, 1, c) && !list_push(&st->n_fallback, L.fallback, L.fb_cap, it))
        atomicOr(&st->error, 2ull);
      continue;
    }
    // bad: kept more than floor(7/8) of the parent's non-equal keys (Sec. 4.1)
    const bool bad = (int64_t)cnt > ((7 * nonequal) >> 3);
    if (bad) atomicAdd(&st->bad_splits, 1ull);
    const int left = (int)t.bad_left - (bad ? 1 : 0);
    c.kind = kSegPart;
    c.bad_left = (uint8_t)(left < 0 ? 0 : left);
    if (left <= 0 || (int64_t)cnt > prm.persist_max || !seg_push(st, L, 0, c)) {
      if (!list_push(&st->n_fallback, L.fallback, L.fb_cap, it)) atomicOr(&st->error, 2ull);
    }
  }
  // equality buckets left in the temp buffer go home now, decoded
  if (!dst_is_keys) {
    for (int b = 1; b < nb; b += 2) {
      const uint32_t cnt = hist[slot(b)];
      if (cnt == 0) continue;
      const int64_t start = curs[slot(b)] - cnt;
      for (int64_t i = tid; i < cnt; i += THREADS) {
        keys[t.begin + start + i] = Key<KT>::dec(tmpk[t.begin + start + i]);
        if (VB) vals[t.begin + start + i] = tmpv[t.begin + start + i];
      }
    }
  }
  if (tid == 0) {
    atomicAdd(&st->partitions, 1ull);
    atomicMax(&st->max_depth, (unsigned long long)(t.depth + 1));
  }
}

// ------------------------------------------------------------------ persistent kernel
template <int KT, int VB, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 512 / THREADS)
seg_persistent_kernel(typename Key<KT>::U* __restrict__ keys, typename Val<VB>::T* __restrict__ vals,
                      typename Key<KT>::U* __restrict__ tmpk, typename Val<VB>::T* __restrict__ tmpv,
                      SegState* st, SegLists L, SegParams prm) {
  using U = typename Key<KT>::U;
  constexpr int CAP = THREADS * ITEMS;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SegTask cur;
  __shared__ int action;  // 0: work, 1: exit
  __shared__ int salvage;
  __shared__ uint32_t wtmp[THREADS / 32 + 1];
  const int tid = threadIdx.x;
  bool injected = false;
  for (;;) {
    if (tid == 0) {
      if (prm.inject_wait && blockIdx.x == 0 && !injected) {
        // test hook: wait (bounded) on a word nothing writes, as a lost producer would look
        injected = true;
        volatile unsigned long long* f = &st->never_set;
        const uint64_t t0 = seg_now();
        while (*f == 0)
          if (seg_now() - t0 > prm.wait_ns) { atomicOr(&st->error, 1ull); break; }
      }
      action = 1;
      const uint64_t t0 = seg_now();
      for (;;) {
        int r = seg_try_pop(st, L, 0, &cur, prm.wait_ns);
        if (r == 1) r = seg_try_pop(st, L, 1, &cur, prm.wait_ns);
        if (r == 0) { action = 0; break; }
        if (r == 2) atomicOr(&st->error, 1ull);
        if (*(volatile unsigned long long*)&st->outstanding == 0) break;
        const uint64_t waited = seg_now() - t0;
        // a normal wait is bounded by wait_ns; in salvage mode the drain gets ten times that
        const bool err = (*(volatile unsigned long long*)&st->error & 1ull) != 0;
        if (!err && waited > prm.wait_ns) atomicOr(&st->error, 1ull);
        if (err && waited > 10 * prm.wait_ns) break;
        __nanosleep(128);
      }
      salvage = (*(volatile unsigned long long*)&st->error & 1ull) != 0;
    }
    __syncthreads();
    if (action != 0) break;
    const SegTask t = cur;
    if (salvage) {
      // keep the arrays a permutation of the input: data in the temp buffer moves back
      if (t.buf == kBufTmp) {
        for (int64_t i = tid; i < t.size; i += THREADS) {
          const U x = tmpk[t.begin + i];
          keys[t.begin + i] = t.enc ? Key<KT>::dec(x) : x;
          if (VB) vals[t.begin + i] = tmpv[t.begin + i];
        }
      } else if (t.enc) {
        for (int64_t i = tid; i < t.size; i += THREADS) keys[t.begin + i] = Key<KT>::dec(keys[t.begin + i]);
      }
    } else if (t.kind == kSegBase) {
      const Item it{t.begin, t.size, (uint16_t)t.buf, (uint16_t)t.enc};
      // (rare: the bucket's size-class list was full) the merge path only, so that the base
      // sort needs no more shared memory than the partition
      base_sort_block<KT, VB, THREADS, ITEMS, false>(it, keys, vals, tmpk, tmpv, kBufKeys, 1, smem);
      if (tid == 0) atomicAdd(&st->base_buckets, 1ull);
    } else {
      seg_partition<KT, VB, THREADS>(t, prm, CAP, keys, vals, tmpk, tmpv, smem, wtmp, st, L);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(&st->outstanding, ~0ull);  // minus one
    }
  }
}

// ------------------------------------------------------------------ class-shaped base sorts
// After the persistent kernel: every CTA sorts list entries blockIdx.x, blockIdx.x + gridDim.x,
// ... of one size class in shared memory, decoding into the key buffer.  The entry count is read
// on the device, so the launch needs no host round trip and is captured with the rest.
template <int KT, int VB, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS)
seg_base_list_kernel(const Item* __restrict__ list, const unsigned long long* __restrict__ count, int64_t cap,
                     typename Key<KT>::U* __restrict__ keys, typename Val<VB>::T* __restrict__ vals,
                     typename Key<KT>::U* __restrict__ tmpk, typename Val<VB>::T* __restrict__ tmpv) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t c = (int64_t)*count;
  const int64_t m = c < cap ? c : cap;
  for (int64_t k = blockIdx.x; k < m; k += gridDim.x) {
    const Item it = list[k];
    // segments hold raw keys whose codes span nearly the whole key width, so the radix path
    // would rarely apply; without it the kernel keeps a smaller footprint and more CTAs per SM
    base_sort_block<KT, VB, THREADS, ITEMS, false>(it, keys, vals, tmpk, tmpv, kBufKeys, 1, smem);
    __syncthreads();
  }
}

template <int KS, int VB, int THREADS, int ITEMS>
constexpr size_t seg_smem() {
  constexpr size_t base = base_sort_core_smem<KS, VB, THREADS, ITEMS>();
  constexpr size_t part = (size_t)(3 * kSegTile + 2 * kBMax) * KS + (size_t)3 * kSegTile * VB +
                         3 * kBinsMax * sizeof(uint32_t) + (size_t)kSegTile * 2;
  return base > part ? base : part;
}

}  // namespace pdq
