// Host driver of the plain path: probe, distribution levels, base sorts, fallback.
#pragma once

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "learned.cuh"
#include "sort_api.h"

namespace pdq {

// ------------------------------------------------------------------ workspace layout
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int64_t chunk_min_for(int64_t n) {
  const int64_t c = (n + 4095) / 4096;
  return c > 8192 ? c : 8192;
}

constexpr int kTrainSteps = 24;       // Adam steps of the learned model
constexpr int kTrainBatch = 32768;    // points per step, drawn from the 1% sample
constexpr float kTrainLr = 0.05f;

constexpr int64_t kFixMin = int64_t(1) << 16;  // smallest array given the nearly-sorted fix-up
constexpr int kFixTile = 8192;                 // elements per tile of the fix-up's peel pass
constexpr int kCopyTile = 8192;                // elements per tile of the copy of final buckets home

// A round's upload: nt tasks, then 4 int32 of metadata per task, then the chunks (16-byte
// aligned parts).
inline size_t round_in_meta_off(int64_t nt) { return align_up((size_t)nt * sizeof(Task), 16); }
inline size_t round_in_chunks_off(int64_t nt) { return align_up(round_in_meta_off(nt) + (size_t)nt * 16, 16); }
inline size_t round_in_bytes(int64_t nt, int64_t nchunks) {
  return round_in_chunks_off(nt) + (size_t)nchunks * sizeof(Chunk);
}

inline Layout make_layout(int64_t n, int ks, int vb, bool learned = false, bool fixup = true) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  const int64_t cmin = kBaseCapMin;
  L.task_cap = n / (cmin + 1) + 2;
  L.round_cap = std::min<int64_t>(kTaskRound, L.task_cap);
  L.chunk_cap = n / chunk_min_for(n) + 1 + L.round_cap;
  L.item_cap = std::min<int64_t>(L.round_cap * kBMax, n + 1);
  L.fb_cap = n / (cmin + 1) + 2;
  // base-sort lists: class 0 (<= 1024 elements) may hold item_cap entries; an item of class
  // c >= 1 has more than 512 << c elements, so that list needs at most n / (512 << c) + 1.
  int64_t base_total = 0;
  for (int c = 0; c < kBaseClasses; ++c) {
    L.base_cap[c] = c == 0 ? L.item_cap : std::min<int64_t>(L.item_cap, n / ((int64_t)512 << c) + 1);
    L.base_off[c] = base_total;
    base_total += L.base_cap[c];
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  // temp buffers index like the (aligned-down) key buffer: up to 16 bytes of shift
  L.tmpk = take((size_t)(n + 16 / ks) * ks);
  L.tmpv = take((size_t)(n + (vb ? 16 / vb : 0)) * vb);
  // every key's bin slot of the current level (2 bytes, indexed like the key buffer; the
  // scatter's slot copies round out to 8-element boundaries past the last key)
  L.slots = take((size_t)(n + 64) * sizeof(uint16_t));
  L.ctr = take(sizeof(Counters));
  L.round_in = take(round_in_bytes(L.round_cap, L.chunk_cap));
  L.tasks_next = take((size_t)L.task_cap * sizeof(Task));
  L.counts = take((size_t)L.chunk_cap * kBinsMax * sizeof(uint32_t));
  // per-(task, bin) totals, then write cursors (the learned level has one task of 4096 bins)
  L.totals = take((size_t)std::max<int64_t>(L.round_cap * kBinsMax, 4096) * sizeof(uint32_t));
  L.tree = take((size_t)L.round_cap * kBMax * ks);
  L.spl = take((size_t)L.round_cap * kBMax * ks);
  L.children = take((size_t)L.round_cap * kBinsMax * sizeof(uint2));
  L.pref = take((size_t)L.round_cap * 32);
  L.tab = take((size_t)L.round_cap * kPrefTableBytes);
  // large arrays keep one set of base lists per position group (host-buffer sorts stream each
  // group's range back as soon as it is sorted); 2^26 keys and up, where the lists are small
  // beside the temp buffer
  L.base_total = base_total;
  L.base_groups = n >= (int64_t(1) << 26) ? kOutGroups : 1;
  L.base_items = take((size_t)base_total * L.base_groups * sizeof(Item));
  L.copy_items = take((size_t)L.item_cap * sizeof(Item));
  L.fb_items = take((size_t)L.fb_cap * sizeof(Item));
  L.msplit = take((size_t)(n / 2048 + 2) * sizeof(int64_t));  // merge-path splits, one per 2048-output tile
  if (learned) {  // 1% training sample and the trained model (learned path, float32 keys)
    L.learned_m = std::min<int64_t>(n, std::max<int64_t>(4096, n / 100));
    L.learned_xs = take((size_t)L.learned_m * sizeof(float));
    L.learned_out = take(sizeof(TrainOut));
    L.learned_sync = take(sizeof(TrainSync));
  }
  if (fixup && n >= kFixMin) {
    L.fix_m = n / 16;
    L.fix_e = take((size_t)(L.fix_m + 16) * ks);
    L.fix_ev = take((size_t)(L.fix_m + 16) * vb);
    L.fix_cnt = take((size_t)(n / kFixTile + 2) * sizeof(uint32_t));
    L.fix_mask = take((size_t)(n / 32 + 2) * sizeof(uint32_t));
    L.fix_ws_bytes = make_layout(L.fix_m, ks, vb, false, false).total;
    L.fix_ws = take(L.fix_ws_bytes);
  }
  L.total = off;
  return L;
}

// ------------------------------------------------------------------ tile shapes
template <int KS, int VB>
struct Shape {
  // scatter: 512 threads, a 32 KiB tile of codes+values (power-of-two element count), double
  // buffered with its 2-byte bin slots (from the count pass), staged in place
  static constexpr int kScatterThreads = 512;
  static constexpr int kScatterTile = (KS + VB) <= 4 ? 8192 : ((KS + VB) <= 8 ? 4096 : 2048);
  static constexpr size_t kScatterSmem = 2 * ((size_t)kScatterTile * KS + (size_t)kScatterTile * VB) +
                                         3 * (size_t)kBinsMax * 4 + 2 * ((size_t)kScatterTile + 16) * 2;
  // count: 512 threads, three 16 KiB tiles in flight
  static constexpr int kCountThreads = 512;
  static constexpr int kCountTile = 16384 / KS;
  static constexpr int kCountStages = 3;
  static constexpr size_t kCountSmem = (size_t)kCountStages * kCountTile * KS;
  static constexpr int kSampleThreads = 1024;
  // base sort: CAP = THREADS * ITEMS for the size classes 1024, 2048, 4096, 8192 (, 16384 for
  // 4-byte keys with at most 4-byte values: 1024 threads, and the shared memory fits); ITEMS =
  // 32 keys per thread for 4-byte keys alone, 16 otherwise (54-79 registers, no spills)
  static constexpr int kBaseItems = VB == 0 && KS == 4 ? 32 : 16;
  static constexpr int base_threads(int cls) { return (1024 << cls) / kBaseItems; }
  static constexpr int kMaxClass = (KS == 4 && VB <= 4) ? 4 : 3;
  static constexpr int kMaxCap = 1024 << kMaxClass;
};

inline int base_class_of(int64_t m) {
  return m <= 1024 ? 0 : (m <= 2048 ? 1 : (m <= 4096 ? 2 : (m <= 8192 ? 3 : 4)));
}

#define PDQ_CUDA(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e__ = (expr);                                                           \
    if (e__ != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string(#expr) + ": " + \
                                             cudaGetErrorString(e__));                  \
  } while (0)

#define PDQ_LAUNCHED(name)                                                                   \
  do {                                                                                       \
    cudaError_t e__ = cudaGetLastError();                                                    \
    if (e__ != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("launch ") + (name) + \
                                             ": " + cudaGetErrorString(e__));                \
  } while (0)

template <int KT, int VB>
class PlainSorter {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  static constexpr int KS = sizeof(U);
  using S = Shape<KS, VB>;

 public:
  explicit PlainSorter(const SortArgs& a, bool learned = false, bool nested = false) : a_(a) {
    cap_ = std::min(a.tune.base_cap, S::kMaxCap);
    L_ = make_layout(a.n, KS, VB, learned, !nested);
    char* ws = static_cast<char*>(a.ws);
    // The tile kernels need 16-byte-aligned buffers: a key array that starts off a 16-byte
    // boundary is addressed from the boundary below it, and every index is shifted by off_
    // elements (reads of those leading elements are masked; nothing outside [off_, off_ + n) is
    // written).  Values must share the same shift.
    off_ = (int64_t)(((uintptr_t)a.keys % 16) / KS);
    keys_ = static_cast<U*>(a.keys) - off_;
    vals_ = VB ? static_cast<V*>(a.vals) - off_ : static_cast<V*>(a.vals);
    vals_misaligned_ = VB && ((uintptr_t)vals_ % 16) != 0;
    tmpk_ = reinterpret_cast<U*>(ws + L_.tmpk);
    tmpv_ = reinterpret_cast<V*>(ws + L_.tmpv);
    slots_ = reinterpret_cast<uint16_t*>(ws + L_.slots);
    ctr_ = reinterpret_cast<Counters*>(ws + L_.ctr);
    round_in_ = ws + L_.round_in;
    set_round_in(L_.round_cap);
    next_ = reinterpret_cast<Task*>(ws + L_.tasks_next);
    counts_ = reinterpret_cast<uint32_t*>(ws + L_.counts);
    totals_ = reinterpret_cast<uint32_t*>(ws + L_.totals);
    tree_ = reinterpret_cast<U*>(ws + L_.tree);
    spl_ = reinterpret_cast<U*>(ws + L_.spl);
    children_ = reinterpret_cast<uint2*>(ws + L_.children);
    pref_ = reinterpret_cast<Pref<U>*>(ws + L_.pref);
    tab_ = reinterpret_cast<PrefEnt*>(ws + L_.tab);
    base_items_ = reinterpret_cast<Item*>(ws + L_.base_items);
    copy_items_ = reinterpret_cast<Item*>(ws + L_.copy_items);
    fb_items_ = reinterpret_cast<Item*>(ws + L_.fb_items);
    st_ = a.stream;
    groups_ = a.host_keys && L_.base_groups > 1 ? (int)L_.base_groups : 1;
  }

  int run() {
    bool done = false;
    int bad0 = 0;
    int rc = prologue(&done, &bad0);
    if (rc) return rc;
    if (done) return a_.host_keys ? stream_out(off_ + a_.n, true) : PDQ_OK;
    std::vector<Task> cur;
    if (spec_ready_) {  // the first level already ran with the probe: finish it
      ++stats_.passes;
      rc = finish_round(&cur, &spec_h_, true, true);
      if (rc) return rc;
    } else {
      cur.push_back(Task{off_, a_.n, kBufKeys, 0, bad0, 0});
    }
    rc = level_loop(std::move(cur));
    if (rc || !a_.host_keys) return rc;
    return stream_out(off_ + a_.n, true);  // whatever the rounds did not send yet
  }

  // Copies [frontier_, end) of the keys (and values) to the host arrays after everything queued
  // on the call's stream; `last`: the call's stream then waits for every copy.
  int64_t frontier_ = -1;
  int stream_out(int64_t end, bool last) {
    if (frontier_ < 0) frontier_ = off_;
    AuxStreams* aux = aux_streams();
    cudaStream_t cs = st_;
    if (aux) {
      cs = aux->copy;
      PDQ_CUDA(cudaEventRecord(aux->ready, st_));
      PDQ_CUDA(cudaStreamWaitEvent(cs, aux->ready, 0));
    }
    if (end > frontier_) {
      const int64_t e0 = frontier_ - off_, len = end - frontier_;
      PDQ_CUDA(cudaMemcpyAsync(static_cast<U*>(a_.host_keys) + e0, keys_ + frontier_, (size_t)len * KS,
                               cudaMemcpyDeviceToHost, cs));
      if (VB)
        PDQ_CUDA(cudaMemcpyAsync(static_cast<V*>(a_.host_vals) + e0, vals_ + frontier_, (size_t)len * VB,
                                 cudaMemcpyDeviceToHost, cs));
      frontier_ = end;
    }
    if (last && aux) {
      PDQ_CUDA(cudaEventRecord(aux->copied, cs));
      PDQ_CUDA(cudaStreamWaitEvent(st_, aux->copied, 0));
    }
    return PDQ_OK;
  }

  // Learned path (float32 keys): a trained monotone CDF model cuts the array into 4096
  // buckets in place of the first sampled-splitter level; buckets above the base capacity
  // continue through the exact splitter levels (the overflow repair).
  int run_learned() {
    bool done = false;
    int bad0 = 0;
    allow_spec_ = false;
    int rc = prologue(&done, &bad0);
    if (rc || done) return rc;
    std::vector<Task> nxt;
    if constexpr (KT == PDQ_F32 && VB == 0) {
      ++stats_.passes;
      rc = learned_round(bad0, &nxt);
      if (rc) return rc;
    } else {
      return set_error(PDQ_ERR_DTYPE, "the learned path sorts float32 keys without values");
    }
    return level_loop(std::move(nxt));
  }

  TrainOut train_out_{};

  pdq_stats stats_{};

  // entry points used by the segmented path's host side
  int configure_public() { return configure(); }
  int fallback_public(const Item& it) { return fallback(it); }

 private:
  SortArgs a_;
  Layout L_;
  int cap_;  // base capacity for this key/value width
  int groups_ = 1;  // position groups of the base lists (host-buffer sorts of large arrays)
  int64_t off_ = 0;  // element shift of the key buffer from its 16-byte boundary
  bool vals_misaligned_ = false;
  U *keys_, *tmpk_, *tree_, *spl_;
  V *vals_, *tmpv_;
  Counters* ctr_;
  Task *tasks_, *next_;  // tasks_, meta_ and chunks_ point into round_in_ (set_round_in)
  int32_t* meta_;
  Chunk* chunks_;
  char* round_in_;
  // Points tasks_, meta_ and chunks_ at their parts of the upload region for nt tasks.
  void set_round_in(int64_t nt) {
    tasks_ = reinterpret_cast<Task*>(round_in_);
    meta_ = reinterpret_cast<int32_t*>(round_in_ + round_in_meta_off(nt));
    chunks_ = reinterpret_cast<Chunk*>(round_in_ + round_in_chunks_off(nt));
  }
  uint16_t* slots_;
  uint32_t* counts_;
  uint32_t* totals_;  // per-(task, bin) key totals, turned into write cursors by the scan
  uint2* children_;
  Pref<U>* pref_;
  PrefEnt* tab_;
  Item *base_items_, *copy_items_, *fb_items_;
  cudaStream_t st_;

  // Checks, the single-bucket case, the sorted / reverse probe and the zero-budget fallback.
  // Sets *done when nothing more is needed, else the root's bad-split budget.
  int prologue(bool* done, int* bad0_out) {
    *done = true;
    if (a_.ws_bytes < L_.total) return set_error(PDQ_ERR_WORKSPACE, "workspace too small");
    if (vals_misaligned_)
      return set_error(PDQ_ERR_ARG, "keys and values must sit at the same offset from a 16-byte boundary");
    int rc = configure();
    if (rc) return rc;
    const int64_t n = a_.n;
    if (n <= 1) return PDQ_OK;
    const int cap = cap_;
    if (n <= cap) {
      Item it{off_, (uint32_t)n, kBufKeys, 0};
      const int cls = base_class_of(n);
      PDQ_CUDA(cudaMemcpyAsync(base_items_ + L_.base_off[cls], &it, sizeof(it),
                               cudaMemcpyHostToDevice, st_));
      return base_sort(cls, 1, kBufKeys, 1, n);
    }
    const int bad0 = a_.tune.bad_allowed > 0 ? a_.tune.bad_allowed
                                              : (a_.tune.bad_allowed < 0 ? 0 : ilog2_floor((uint64_t)n));
    if (a_.tune.probe) {
      bool sorted = false, nearly = false;
      rc = speculate(bad0);
      if (rc) return rc;
      if (spec_ready_) {
        *done = false;
        *bad0_out = bad0;
        return PDQ_OK;
      }
      rc = probe(&sorted, &nearly);
      if (rc || sorted) return rc;
      if (nearly) {
        bool fixed = false;
        rc = fixup(&fixed);
        if (rc || fixed) return rc;
      }
    }
    if (bad0 == 0) {
      Item it{off_, (uint32_t)n, kBufKeys, 0};
      ++stats_.fallback_buckets;
      return fallback(it);
    }
    *done = false;
    *bad0_out = bad0;
    return PDQ_OK;
  }

  int level_loop(std::vector<Task> cur) {
    while (!cur.empty()) {
      std::vector<Task> nxt;
      ++stats_.passes;
      for (size_t r0 = 0; r0 < cur.size(); r0 += (size_t)L_.round_cap) {
        const size_t r1 = std::min(cur.size(), r0 + (size_t)L_.round_cap);
        const int rc = level_round(cur.data() + r0, (int)(r1 - r0), &nxt, r1 == cur.size());
        if (rc) return rc;
      }
      cur.swap(nxt);
    }
    return PDQ_OK;
  }

  // The learned level over the whole array (one task).
  int learned_round(int bad0, std::vector<Task>* nxt) {
    if constexpr (KT == PDQ_F32 && VB == 0) {
      constexpr int kLTile = 4096;
      constexpr size_t kLScatterSmem =
          2 * (size_t)kLTile * 4 + 3 * (size_t)kLearnedBuckets * 4 + 2 * ((size_t)kLTile + 16) * 2;
      static bool configured = false;
      if (!configured) {
        PDQ_CUDA(cudaFuncSetAttribute(count_kernel<KT, ModelCls, S::kCountThreads, S::kCountTile, S::kCountStages>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kCountSmem));
        PDQ_CUDA(cudaFuncSetAttribute(scatter_kernel<KT, 0, ModelCls, 512, kLTile>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLScatterSmem));
        configured = true;
      }
      const int64_t n = a_.n, m = L_.learned_m;
      char* ws = static_cast<char*>(a_.ws);
      float* xs = reinterpret_cast<float*>(ws + L_.learned_xs);
      TrainOut* tout = reinterpret_cast<TrainOut*>(ws + L_.learned_out);
      const uint64_t seed = mix64((uint64_t)n ^ 0x5EEDull);
      {  // 1% sample at hashed positions
        LaunchScope ls("learned_gather", st_, (double)m * 8);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, a_.num_sms * 8));
        learned_gather_kernel<<<blocks, 256, 0, st_>>>(reinterpret_cast<const float*>(keys_ + off_), n, xs, m, seed);
      }
      PDQ_LAUNCHED("learned_gather");
      {  // sort the sample with the plain path (its workspace is the part before the sample)
        SortArgs sa = a_;
        sa.host_keys = sa.host_vals = nullptr;
        sa.keys = xs;
        sa.vals = nullptr;
        sa.n = m;
        sa.ws_bytes = L_.learned_xs;
        PlainSorter<PDQ_F32, 0> sub(sa);
        const int rc = sub.run();
        if (rc) return rc;
      }
      {
        LaunchScope ls("learned_train", st_, 0.0);
        TrainSync* sy = reinterpret_cast<TrainSync*>(ws + L_.learned_sync);
        PDQ_CUDA(launch_learned_train(xs, m, kTrainSteps, kTrainBatch, kTrainLr, seed ^ 0x7A11ull, tout, sy,
                                      a_.num_sms, st_));
      }
      PDQ_LAUNCHED("learned_train");
      PDQ_CUDA(cudaMemcpyAsync(&train_out_, tout, sizeof(TrainOut), cudaMemcpyDeviceToHost, st_));
      PDQ_CUDA(cudaStreamSynchronize(st_));
      if (train_out_.status) return set_error(PDQ_ERR_TIMEOUT, "learned_train: a grid barrier gave up");
      const LearnedModel model = train_out_.model;
      // one task in about one large chunk per SM (keeps the 4096-bin scan short); chunks x 4096
      // bins must fit the count array
      int64_t ch = std::max<int64_t>(chunk_min_for(n), (n + a_.num_sms - 1) / a_.num_sms);
      const int64_t max_chunks = std::max<int64_t>(1, L_.chunk_cap * kBinsMax / kLearnedBuckets);
      ch = std::max<int64_t>(ch, (n + max_chunks - 1) / max_chunks);
      std::vector<Chunk> chunks;
      for (int64_t o = 0; o < n; o += ch) chunks.push_back(Chunk{off_ + o, (int32_t)std::min<int64_t>(ch, n - o), 0});
      const int nchunks = (int)chunks.size();
      const Task root{off_, n, kBufKeys, 0, bad0, 0};
      const int32_t meta[4] = {0, 0, nchunks, kLearnedBuckets};  // logb (unused), chunk0, nchunks, nbins
      set_round_in(L_.round_cap);  // (the chunk part then has room for chunk_cap chunks)
      PDQ_CUDA(cudaMemcpyAsync(tasks_, &root, sizeof(Task), cudaMemcpyHostToDevice, st_));
      PDQ_CUDA(cudaMemcpyAsync(meta_, meta, sizeof(meta), cudaMemcpyHostToDevice, st_));
      PDQ_CUDA(cudaMemcpyAsync(chunks_, chunks.data(), sizeof(Chunk) * nchunks, cudaMemcpyHostToDevice, st_));
      PDQ_CUDA(cudaMemsetAsync(ctr_, 0, offsetof(Counters, probe), st_));
      PDQ_CUDA(cudaMemsetAsync(totals_, 0, sizeof(uint32_t) * kLearnedBuckets, st_));
      const int32_t* d_nb = meta_ + 3;
      {
        LaunchScope ls("learned_count", st_, (double)n * KS);
        count_kernel<KT, ModelCls, S::kCountThreads, S::kCountTile, S::kCountStages>
            <<<nchunks, S::kCountThreads, S::kCountSmem, st_>>>(chunks_, tasks_, keys_, tmpk_, model, counts_,
                                                                kLearnedBuckets, totals_, slots_, ctr_);
      }
      PDQ_LAUNCHED("learned_count");
      {
        LaunchScope ls("learned_scan", st_, 0.0);
        scan_bookkeep_kernel<1024, kLearnedBuckets><<<1, 1024, 0, st_>>>(tasks_, d_nb, totals_, kLearnedBuckets,
                                                                         children_, 0, cap_, book_lists());
      }
      PDQ_LAUNCHED("learned_scan");
      {
        LaunchScope ls("learned_scatter", st_, 2.0 * (double)n * KS);
        scatter_kernel<KT, 0, ModelCls, 512, kLTile><<<nchunks, 512, kLScatterSmem, st_>>>(
            chunks_, tasks_, keys_, vals_, tmpk_, tmpv_, model, counts_, kLearnedBuckets, totals_, slots_,
            ctr_);
      }
      PDQ_LAUNCHED("learned_scatter");
      Counters h;
      const int rc = finish_round(nxt, &h);
      stats_.learned_overflow = (int64_t)(h.n_next + h.n_fallback);
      return rc;
    } else {
      (void)bad0;
      (void)nxt;
      return set_error(PDQ_ERR_DTYPE, "the learned path sorts float32 keys without values");
    }
  }

  template <int CLS>
  int configure_base() {
    constexpr int T = S::base_threads(CLS);
    PDQ_CUDA(cudaFuncSetAttribute(base_sort_kernel<KT, VB, T, S::kBaseItems>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)base_sort_smem<KS, VB, T, S::kBaseItems>()));
    // as many resident CTAs as shared memory allows (the L1 share is of no use to this kernel)
    PDQ_CUDA(cudaFuncSetAttribute(base_sort_kernel<KT, VB, T, S::kBaseItems>,
                                  cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared));
    return PDQ_OK;
  }

  int configure() {
    static bool done = false;  // per template instantiation
    if (done) return PDQ_OK;
    PDQ_CUDA(cudaFuncSetAttribute(scatter_kernel<KT, VB, SplitterCls<U>, S::kScatterThreads, S::kScatterTile>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kScatterSmem));
    PDQ_CUDA(cudaFuncSetAttribute(count_kernel<KT, SplitterCls<U>, S::kCountThreads, S::kCountTile, S::kCountStages>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kCountSmem));
    PDQ_CUDA(cudaFuncSetAttribute(merge_tile_kernel<KT, VB, kMergeThreads, kMergeItems>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)merge_tile_smem<KS, VB, kMergeThreads, kMergeItems>()));
    int rc = configure_base<0>();
    if (!rc) rc = configure_base<1>();
    if (!rc) rc = configure_base<2>();
    if (!rc) rc = configure_base<3>();
    if constexpr (S::kMaxClass >= 4) {
      if (!rc) rc = configure_base<4>();
    }
    if (rc) return rc;
    done = true;
    return PDQ_OK;
  }

  // Queues the probe over every stride-th key (results in ctr_->probe: descents, ascents, ...).
  int launch_probe(int64_t stride) {
    const int64_t n = a_.n;
    const unsigned long long init[4] = {0, 0, ~0ull, 0};
    PDQ_CUDA(cudaMemcpyAsync(ctr_->probe, init, sizeof(init), cudaMemcpyHostToDevice, st_));
    const int64_t m = (n - 1) / stride + 1;
    const int threads = 256;
    int blocks = (int)std::min<int64_t>((m + threads - 1) / threads, (int64_t)a_.num_sms * 8);
    if (blocks < 1) blocks = 1;
    {
      LaunchScope ls("probe", st_, (double)m * KS);
      probe_kernel<KT><<<blocks, threads, 0, st_>>>(keys_ + off_, n, stride, m, ctr_->probe);
    }
    PDQ_LAUNCHED("probe");
    return PDQ_OK;
  }

  static int64_t probe_stride(int64_t n) { return std::max<int64_t>(1, n / 65536); }

  // Whether the sampled probe's descents h0 and ascents h1 (over m_sample strided pairs) send the
  // array to the ordinary sort: the sample is neither monotone, and its descents are not few (at
  // most 1/16 of its pairs) yet scattered (at least 1/256: not a handful of long ascending runs,
  // whose boundaries the fix-up cannot repair) -- such an array is probed in full for the fix-up.
  bool sample_says_sort(unsigned long long h0, unsigned long long h1, int64_t m_sample) const {
    const bool can_fix = a_.tune.fixup && L_.fix_m > 0;
    return h0 != 0 && h1 != 0 && !(can_fix && (int64_t)h0 * 16 <= m_sample && (int64_t)h0 * 256 >= m_sample);
  }

  // Small arrays (up to kSpecMax keys, with a sampled probe): the probe's sample and the whole
  // first level are queued back to back, and one read-back of the counters (which hold the probe
  // results too) serves both, instead of one synchronisation after each.  The first level only
  // reads the keys and writes the temporary buffers, lists and counters, so when the probe asks
  // for anything but the ordinary sort (sorted, reversed, the fix-up), its work is dropped and
  // the usual path runs from the probe on.  Sets spec_ready_ (with spec_h_) when it was kept.
  static constexpr int64_t kSpecMax = int64_t(1) << 22;
  bool allow_spec_ = true;  // (the learned path replaces the first level: no speculation)
  bool spec_ready_ = false;
  Counters spec_h_{};
  int speculate(int bad0) {
    const int64_t n = a_.n;
    const int64_t stride = probe_stride(n);
    if (!allow_spec_ || n > kSpecMax || stride < 2 || bad0 <= 0) return PDQ_OK;
    int rc = launch_probe(stride);
    if (rc) return rc;
    const Task root{off_, n, kBufKeys, 0, bad0, 0};
    rc = launch_round(&root, 1);
    if (rc) return rc;
    rc = read_counters(&spec_h_);
    if (rc) return rc;
    if (sample_says_sort(spec_h_.probe[0], spec_h_.probe[1], (n - 1) / stride + 1)) spec_ready_ = true;
    return PDQ_OK;
  }

  // Sorted / reverse probe (Sec. 5.2): a sample first, the full pass only when the sample is
  // monotone or has few scattered descents.  Sets *done when the array needs nothing more.
  int probe(bool* done, bool* nearly) {
    const int64_t n = a_.n;
    const bool can_fix = a_.tune.fixup && L_.fix_m > 0;
    unsigned long long h[4];
    auto run_probe = [&](int64_t stride) -> int {
      const int rc = launch_probe(stride);
      if (rc) return rc;
      PDQ_CUDA(cudaMemcpyAsync(h, ctr_->probe, sizeof(h), cudaMemcpyDeviceToHost, st_));
      PDQ_CUDA(cudaStreamSynchronize(st_));
      return PDQ_OK;
    };
    const int64_t stride = probe_stride(n);
    int rc = run_probe(stride);
    if (rc) return rc;
    const int64_t m_sample = (n - 1) / stride + 1;
    if (stride > 1 && sample_says_sort(h[0], h[1], m_sample)) return PDQ_OK;
    if (stride > 1) {
      rc = run_probe(1);
      if (rc) return rc;
    }
    if (h[0] == 0) {  // no descent: sorted (all-equal included)
      stats_.sorted_exit = 1;
      *done = true;
      return PDQ_OK;
    }
    if (h[1] == 0) {  // no ascent: non-increasing, reverse in place
      stats_.reversed = 1;
      *done = true;
      const int threads = 256;
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n / 2 + threads - 1) / threads,
                                                                       (int64_t)a_.num_sms * 16));
      {
        LaunchScope ls("reverse", st_, 2.0 * n * (KS + VB));
        reverse_kernel<U><<<blocks, threads, 0, st_>>>(keys_ + off_, n);
        if (VB) reverse_kernel<V><<<blocks, threads, 0, st_>>>(vals_ + off_, n);
      }
      PDQ_LAUNCHED("reverse");
      return PDQ_OK;
    }
    // Few descents, but not so few that the input is a handful of long ascending runs (whose
    // boundaries peeling cannot repair): the fix-up.
    if (can_fix && (int64_t)h[0] <= n / 32 && (int64_t)h[0] >= n / 4096) *nearly = true;
    return PDQ_OK;
  }

  // Nearly-sorted fix-up: mark both elements of every descent; then, in repair rounds that
  // only look at the kept neighbours of each marked run, mark them too while they are out of
  // order, until the unmarked elements are ascending (at most 16 rounds, at most fix_m marked).
  // Only then is anything moved: one compaction splits the array into the ascending remainder R
  // and the marked elements E, E is sorted on its own, and R and E are merged into the key
  // buffer.  *fixed is false when a bound is hit: nothing has moved, the caller sorts as usual.
  int fixup(bool* fixed) {
    *fixed = false;
    const int64_t n = a_.n;
    char* ws = static_cast<char*>(a_.ws);
    U* E = reinterpret_cast<U*>(ws + L_.fix_e);
    V* Ev = reinterpret_cast<V*>(ws + L_.fix_ev);
    uint32_t* tc = reinterpret_cast<uint32_t*>(ws + L_.fix_cnt);
    uint32_t* mask = reinterpret_cast<uint32_t*>(ws + L_.fix_mask);
    U* src = keys_ + off_;
    V* srcv = VB ? vals_ + off_ : nullptr;
    unsigned long long* marked = &ctr_->probe[4];
    unsigned int* changed = reinterpret_cast<unsigned int*>(&ctr_->probe[5]);
    PDQ_CUDA(cudaMemsetAsync(marked, 0, sizeof(unsigned long long), st_));
    {
      LaunchScope ls("fixup_mark", st_, (double)n * KS);
      const int64_t words = (n + 31) / 32;
      const unsigned blocks = (unsigned)std::min<int64_t>((words + 7) / 8, (int64_t)a_.num_sms * 16);
      fix_mark_kernel<KT><<<blocks, 256, 0, st_>>>(src, n, mask, marked);
    }
    PDQ_LAUNCHED("fixup_mark");
    unsigned long long h[2] = {0, 0};
    PDQ_CUDA(cudaMemcpyAsync(h, marked, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st_));
    PDQ_CUDA(cudaStreamSynchronize(st_));
    if ((int64_t)h[0] > L_.fix_m) return PDQ_OK;
    bool clean = false;
    unsigned int* added = changed + 1;
    unsigned int prev_added = 0;
    for (int round = 0; round < 16; ++round) {
      PDQ_CUDA(cudaMemsetAsync(changed, 0, 2 * sizeof(unsigned int), st_));
      {
        LaunchScope ls("fixup_repair", st_, 0.0);
        const int64_t words = (n + 31) / 32;
        const unsigned blocks = (unsigned)std::min<int64_t>((words + 255) / 256, (int64_t)a_.num_sms * 8);
        fix_repair_kernel<KT><<<blocks, 256, 0, st_>>>(src, n, mask, changed, added);
      }
      PDQ_LAUNCHED("fixup_repair");
      unsigned int c[2] = {0, 0};
      PDQ_CUDA(cudaMemcpyAsync(c, changed, sizeof(c), cudaMemcpyDeviceToHost, st_));
      PDQ_CUDA(cudaStreamSynchronize(st_));
      if (c[0] & 2u) break;  // a marked run too long to repair locally
      if (c[0] == 0) {
        clean = true;
        break;
      }
      // a first repair that marks more than an eighth again (a shuffled stretch), or rounds
      // that stop shrinking (long ascending runs grow their junctions steadily): give up
      if (round == 0 && (uint64_t)c[1] * 8 > (uint64_t)h[0]) break;
      if (round >= 1 && (uint64_t)c[1] * 10 >= (uint64_t)prev_added * 9) break;
      prev_added = c[1];
    }
    if (!clean) return PDQ_OK;
    // marked elements per tile, their exclusive prefix (total = |E|), then the split
    const int ntiles = (int)((n + kFixTile - 1) / kFixTile);
    {
      LaunchScope ls("fixup_split", st_, 2.0 * (double)n * (KS + VB));
      fix_tile_count_kernel<256, kFixTile><<<ntiles, 256, 0, st_>>>(mask, n, tc);
      fix_scan_kernel<1024><<<1, 1024, 0, st_>>>(tc, ntiles, marked);
      note_launch_count(1);
    }
    PDQ_LAUNCHED("fixup_split");
    PDQ_CUDA(cudaMemcpyAsync(h, marked, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st_));
    PDQ_CUDA(cudaStreamSynchronize(st_));
    const int64_t e_len = (int64_t)h[0];
    if (e_len > L_.fix_m) return PDQ_OK;
    U* R = tmpk_ + off_;
    V* Rv = VB ? tmpv_ + off_ : nullptr;
    const int64_t len = n - e_len;
    {
      LaunchScope ls("fixup_compact", st_, 2.0 * (double)n * (KS + VB));
      fix_compact_kernel<KT, VB, 256, kFixTile><<<ntiles, 256, 0, st_>>>(src, srcv, n, mask, R, Rv, E, Ev, 0, tc);
    }
    PDQ_LAUNCHED("fixup_compact");
    stats_.fixup_peeled = e_len;
    if (e_len > 1) {  // the marked keys' own sort (no fix-up inside it)
      SortArgs sa = a_;
      sa.host_keys = sa.host_vals = nullptr;
      sa.keys = E;
      sa.vals = VB ? static_cast<void*>(Ev) : nullptr;
      sa.n = e_len;
      sa.ws = ws + L_.fix_ws;
      sa.ws_bytes = L_.fix_ws_bytes;
      PlainSorter<KT, VB> sub(sa, false, true);
      const int rc = sub.run();
      if (rc) return rc;
      stats_.passes = sub.stats_.passes;
      stats_.base_buckets += sub.stats_.base_buckets;
      stats_.equal_buckets += sub.stats_.equal_buckets;
      stats_.fallback_buckets += sub.stats_.fallback_buckets;
    }
    {
      MergeArgs<KT, VB> ma;
      ma.a = R;
      ma.av = Rv;
      ma.la = len;
      ma.b = E;
      ma.bv = Ev;
      ma.lb = e_len;
      ma.out = keys_ + off_;
      ma.outv = VB ? vals_ + off_ : nullptr;
      ma.w = 0;
      ma.n = n;
      ma.raw = 1;
      ma.decode = 0;
      LaunchScope ls("fixup_merge", st_, 2.0 * (double)n * (KS + VB));
      launch_merge_tiles(ma, n);
    }
    PDQ_LAUNCHED("fixup_merge");
    *fixed = true;
    return PDQ_OK;
  }

  // The bookkeeping's work lists and their capacities.
  BookLists book_lists() const {
    BookLists b;
    b.ctr = ctr_;
    b.next = next_;
    b.base_items = base_items_;
    b.copy_items = copy_items_;
    b.fb_items = fb_items_;
    for (int c = 0; c < kBaseClasses; ++c) {
      b.caps.base_off[c] = L_.base_off[c];
      b.caps.base_cap[c] = L_.base_cap[c];
    }
    b.caps.task_cap = L_.task_cap;
    b.caps.copy_cap = L_.item_cap;
    b.caps.fb_cap = L_.fb_cap;
    b.caps.groups = groups_;
    b.caps.group_stride = L_.base_total;
    b.caps.group_first = off_;
    b.caps.group_n = a_.n;
    return b;
  }

  // Buckets per level: enough that the expected bucket is a quarter of the base capacity (so
  // that, with sampling noise, almost every bucket fits the base sort after this level).
  typename SplitterCls<U>::Params cls_params(const int32_t* d_logb) const {
    typename SplitterCls<U>::Params p;
    p.task_logb = d_logb;
    p.tree = tree_;
    p.spl = spl_;
    p.pref = pref_;
    p.tab = tab_;
    return p;
  }

  int choose_logb(int64_t size) const {
    const int64_t quarter = std::max<int64_t>(1, cap_ / 4);
    const int64_t want = (size + quarter - 1) / quarter;
    int lb = 1;
    while ((int64_t(1) << lb) < want && lb < a_.tune.logb) ++lb;
    // Headroom on the last level: when the tuned width leaves buckets that fit the base sort on
    // average but average above a third of its capacity (a parent well above the mean size),
    // sampling noise can push one of them past the capacity and cost a whole further level; one
    // more bit of buckets keeps the pass count of the sort the same from run to run.
    if (lb == a_.tune.logb && lb < kLogBMax && size > ((int64_t)cap_ / 3 << lb) && size <= ((int64_t)cap_ << lb))
      ++lb;
    return lb;
  }

  // The host-built part of a distribution round and its sample kernel: chunks, uploads of the
  // task and chunk lists, counter resets, splitter selection.
  struct Head {
    int nchunks = 0;
    int64_t total = 0;
  };

  int round_head(const Task* tasks, int nt, Head* hd) {
    const int64_t n = a_.n;
    int64_t total = 0;
    for (int i = 0; i < nt; ++i) total += tasks[i].size;
    // Chunks: one task is cut into 6 chunks per SM, whole waves of both the count (3 resident
    // CTAs per SM with 4-byte keys, 2 with 8-byte keys) and the scatter (2 per SM).  Several
    // tasks cannot share chunks, so each task is cut into equal parts of at most about total /
    // (2 x 6 per SM) elements: near-full waves instead of full ones and a ragged tail.
    const int64_t slots = (int64_t)a_.num_sms * 6;
    const int64_t want = nt == 1 ? slots : 2 * slots;
    const int64_t ch = std::max<int64_t>(chunk_min_for(n), (total + want - 1) / want);
    std::vector<int32_t> meta(4 * (size_t)nt);
    std::vector<Chunk> chunks;
    chunks.reserve((size_t)(total / ch + nt + 1));
    for (int i = 0; i < nt; ++i) {
      const int lb = choose_logb(tasks[i].size);
      meta[i] = lb;
      meta[nt + i] = (int32_t)chunks.size();
      const int64_t size = tasks[i].size;
      const int64_t parts = std::max<int64_t>(1, (size + ch - 1) / ch);
      for (int64_t j = 0; j < parts; ++j) {
        const int64_t o0 = size * j / parts, o1 = size * (j + 1) / parts;
        chunks.push_back(Chunk{tasks[i].begin + o0, (int32_t)(o1 - o0), i});
      }
      meta[2 * nt + i] = (int32_t)parts;
      meta[3 * nt + i] = 2 << lb;
    }
    const int nchunks = (int)chunks.size();
    if (nchunks > L_.chunk_cap) return set_error(PDQ_ERR_INTERNAL, "chunk capacity exceeded");
    // one upload of tasks, metadata (logb, first chunk, chunk count, bin count per task) and
    // chunks, from pinned staging when there is some (every round ends with a synchronisation
    // of the call's stream, so the staging is free again when the next round fills it)
    set_round_in(nt);
    const size_t bytes = round_in_bytes(nt, nchunks);
    char* stage = static_cast<char*>(host_staging(0, bytes));
    std::vector<char> pageable;
    if (!stage) {
      pageable.resize(bytes);
      stage = pageable.data();
    }
    std::memcpy(stage, tasks, sizeof(Task) * nt);
    std::memcpy(stage + round_in_meta_off(nt), meta.data(), sizeof(int32_t) * meta.size());
    std::memcpy(stage + round_in_chunks_off(nt), chunks.data(), sizeof(Chunk) * nchunks);
    PDQ_CUDA(cudaMemcpyAsync(round_in_, stage, bytes, cudaMemcpyHostToDevice, st_));
    int32_t* d_logb = meta_;
    int32_t* d_nb = meta_ + 3 * nt;

    int oversample = a_.tune.oversample;
    {  // (it also clears the round's counters and bin totals)
      LaunchScope ls("sample", st_, 0.0);
      sample_kernel<KT, S::kSampleThreads><<<nt, S::kSampleThreads, 0, st_>>>(
          tasks_, d_logb, oversample, keys_, tmpk_, tree_, spl_, pref_, tab_, ctr_, totals_, kBinsMax);
    }
    PDQ_LAUNCHED("sample");
    (void)d_nb;
    hd->nchunks = nchunks;
    hd->total = total;
    return PDQ_OK;
  }

  // One distribution level over tasks[0..nt): sample, count, scan and bookkeeping, scatter, then
  // base sorts / copies / fallbacks of the children that finished.  Next tasks are appended.
  int level_round(const Task* tasks, int nt, std::vector<Task>* nxt, bool last_round = false) {
    const int rc = launch_round(tasks, nt);
    if (rc) return rc;
    Counters h;
    return finish_round(nxt, &h, last_round);
  }

  // Queues one distribution level over tasks[0..nt): sample, count, scan and bookkeeping, scatter.
  int launch_round(const Task* tasks, int nt) {
    Head hd;
    const int rc0 = round_head(tasks, nt, &hd);
    if (rc0) return rc0;
    const int nchunks = hd.nchunks;
    const int64_t total = hd.total;
    int32_t* d_logb = meta_;
    int32_t* d_nb = meta_ + 3 * nt;
    {
      LaunchScope ls("count", st_, (double)total * KS);
      count_kernel<KT, SplitterCls<U>, S::kCountThreads, S::kCountTile, S::kCountStages>
          <<<nchunks, S::kCountThreads, S::kCountSmem, st_>>>(chunks_, tasks_, keys_, tmpk_, cls_params(d_logb),
                                                              counts_, kBinsMax, totals_, slots_, ctr_);
    }
    PDQ_LAUNCHED("count");
    {
      LaunchScope ls("scan_bookkeep", st_, 0.0);
      scan_bookkeep_kernel<512, kBinsMax><<<nt, 512, 0, st_>>>(tasks_, d_nb, totals_, kBinsMax, children_, 1,
                                                               cap_, book_lists());
    }
    PDQ_LAUNCHED("scan_bookkeep");
    {
      LaunchScope ls("scatter", st_, 2.0 * (double)total * (KS + VB));
      scatter_kernel<KT, VB, SplitterCls<U>, S::kScatterThreads, S::kScatterTile>
          <<<nchunks, S::kScatterThreads, S::kScatterSmem, st_>>>(
              chunks_, tasks_, keys_, vals_, tmpk_, tmpv_, cls_params(d_logb), counts_, kBinsMax, totals_,
              slots_, ctr_);
    }
    PDQ_LAUNCHED("scatter");
    return PDQ_OK;
  }

  // Reads the round's counters back (through pinned staging when there is some) and waits for
  // the call's stream.
  int read_counters(Counters* h) {
    Counters* hc = static_cast<Counters*>(host_staging(1, sizeof(Counters)));
    PDQ_CUDA(cudaMemcpyAsync(hc ? hc : h, ctr_, sizeof(Counters), cudaMemcpyDeviceToHost, st_));
    PDQ_CUDA(cudaStreamSynchronize(st_));
    if (hc) *h = *hc;
    return PDQ_OK;
  }

  // After a round's bookkeeping: read the counters, sort finished buckets, copy final buckets
  // home, run fallbacks, and collect the next level's tasks.
  // have_counters: *hout already holds them.
  int finish_round(std::vector<Task>* nxt, Counters* hout, bool last_round = false, bool have_counters = false) {
    Counters& h = *hout;
    if (!have_counters) {
      const int rc = read_counters(&h);
      if (rc) return rc;
    }
    if (h.timeout) return set_error(PDQ_ERR_TIMEOUT, "a tile copy did not complete within its bounded wait");
    if (h.overflow) return set_error(PDQ_ERR_INTERNAL, "bookkeeping list capacity exceeded");
    stats_.equal_buckets += (int64_t)h.equal_buckets;
    stats_.bad_splits += (int64_t)h.bad_splits;
    // The size classes run concurrently on auxiliary streams forked from the call's stream and
    // joined back before anything later on it (the next level's bookkeeping rewrites the lists);
    // the copy of final buckets home runs meanwhile on the call's stream.  With position groups
    // (host-buffer sorts of large arrays) the groups follow one another on each class's stream,
    // and when this round finishes the sort, every group's range is copied to the host once its
    // base sorts are done, while the later groups sort.  The level's base elements are counted
    // once, on the first launch.
    int64_t base_elems = (int64_t)h.base_elems;
    int nlaunch = 0;
    for (int g = 0; g < groups_; ++g)
      for (int cls = 0; cls < kBaseClasses; ++cls) nlaunch += h.n_base[g][cls] ? 1 : 0;
    const bool stream_now = a_.host_keys && groups_ > 1 && last_round && nxt->empty() && h.n_next == 0 &&
                            h.n_fallback == 0;
    // (with per-kernel timing on they stay serial, so that each launch's time is its own)
    AuxStreams* aux = nlaunch > 1 && !profiling_enabled() ? aux_streams() : nullptr;
    if (aux && cudaEventRecord(aux->fork, st_) != cudaSuccess) aux = nullptr;
    bool joined[kBaseClasses] = {};
    auto join_all = [&]() {  // the call's stream waits for every class launched so far
      for (int cls = 0; cls < kBaseClasses; ++cls)
        if (joined[cls]) cudaStreamWaitEvent(st_, aux->join[cls], 0);
    };
    bool forked[kBaseClasses] = {};
    if (h.n_copy) {
      // The tile numbering lives in the counts region, free between a level's scatter and the
      // next level's count (item_cap + 1 words always fit: it holds at least 4096 bytes per task).
      // With at most one tile's elements in total every item fits one tile: no numbering.
      LaunchScope ls("copy", st_, 2.0 * (double)h.copy_elems * (KS + VB));
      uint32_t* tile0 = h.copy_elems > (unsigned long long)kCopyTile ? counts_ : nullptr;
      if (tile0) {
        copy_plan_kernel<1024, kCopyTile><<<1, 1024, 0, st_>>>(copy_items_, (int)h.n_copy, tile0);
        note_launch_count(1);
      }
      const int64_t blocks = std::min<int64_t>(a_.num_sms * 8, tile0 ? INT32_MAX : (int64_t)h.n_copy);
      copy_kernel<KT, VB, 256, kCopyTile><<<(unsigned)blocks, 256, 0, st_>>>(
          copy_items_, (int)h.n_copy, tile0, keys_, vals_, tmpk_, tmpv_);
    }
    PDQ_LAUNCHED("copy");
    for (int g = 0; g < groups_; ++g) {
      for (int cls = 0; cls < kBaseClasses; ++cls) {
        if (!h.n_base[g][cls]) continue;
        cudaStream_t s = st_;
        if (aux) {
          s = aux->s[cls];
          if (!forked[cls]) {
            if (cudaStreamWaitEvent(s, aux->fork, 0) != cudaSuccess) s = st_;
            else forked[cls] = true;
          }
        }
        const int rc = base_sort(cls, (int64_t)h.n_base[g][cls], kBufKeys, 1, base_elems, s, g);
        if (s != st_ && cudaEventRecord(aux->join[cls], s) == cudaSuccess) joined[cls] = true;
        if (rc) {
          if (aux) join_all();
          return rc;
        }
        base_elems = 0;
      }
      if (stream_now) {  // everything before the next group's first element is final
        if (aux) join_all();
        const int rc = stream_out(off_ + (((int64_t)(g + 1) * a_.n + groups_ - 1) / groups_), false);
        if (rc) return rc;
      }
    }
    if (aux) join_all();
    if (h.n_fallback) {
      std::vector<Item> fb(h.n_fallback);
      PDQ_CUDA(cudaMemcpyAsync(fb.data(), fb_items_, sizeof(Item) * fb.size(), cudaMemcpyDeviceToHost, st_));
      PDQ_CUDA(cudaStreamSynchronize(st_));
      stats_.fallback_buckets += (int64_t)fb.size();
      for (const Item& it : fb) {
        int rc = fallback(it);
        if (rc) return rc;
      }
    }
    if (h.n_next) {
      const size_t off = nxt->size();
      nxt->resize(off + h.n_next);
      PDQ_CUDA(cudaMemcpyAsync(nxt->data() + off, next_, sizeof(Task) * h.n_next, cudaMemcpyDeviceToHost, st_));
      PDQ_CUDA(cudaStreamSynchronize(st_));
    }
    return PDQ_OK;
  }

  // Base sort of `count` items of size class `cls` (holding `elems` elements for the byte
  // accounting) already in that class's list.
  template <int CLS>
  int base_sort_cls(int64_t count, int out_buf, int decode, int64_t elems, cudaStream_t st, int group) {
    constexpr int T = S::base_threads(CLS);
    constexpr size_t smem = base_sort_smem<KS, VB, T, S::kBaseItems>();
    const Item* list = base_items_ + (size_t)group * L_.base_total + L_.base_off[CLS];
    for (int64_t done = 0; done < count;) {
      const int64_t g = std::min<int64_t>(count - done, 1 << 30);
      LaunchScope ls("base_sort", st, done == 0 ? 2.0 * (double)elems * (KS + VB) : 0.0);
      base_sort_kernel<KT, VB, T, S::kBaseItems><<<(unsigned)g, T, smem, st>>>(
          list + done, keys_, vals_, tmpk_, tmpv_, out_buf, decode);
      done += g;
    }
    PDQ_LAUNCHED("base_sort");
    return PDQ_OK;
  }

  static constexpr int kMergeThreads = 256, kMergeItems = 8, kMergeTile = kMergeThreads * kMergeItems;
  void launch_merge_tiles(const MergeArgs<KT, VB>& ma, int64_t total) {
    constexpr size_t smem = merge_tile_smem<KS, VB, kMergeThreads, kMergeItems>();
    const int64_t blocks = (total + kMergeTile - 1) / kMergeTile;
    int64_t* splits = reinterpret_cast<int64_t*>(static_cast<char*>(a_.ws) + L_.msplit);
    merge_split_kernel<KT, VB, kMergeTile><<<(unsigned)((blocks + 255) / 256), 256, 0, st_>>>(ma, blocks, splits);
    merge_tile_kernel<KT, VB, kMergeThreads, kMergeItems><<<(unsigned)blocks, kMergeThreads, smem, st_>>>(ma, splits);
    note_launch_count(1);
  }

  int base_sort(int cls, int64_t count, int out_buf, int decode, int64_t elems, cudaStream_t st = nullptr,
                int group = 0) {
    stats_.base_buckets += count;
    if (!st) st = st_;
    switch (cls) {
      case 0: return base_sort_cls<0>(count, out_buf, decode, elems, st, group);
      case 1: return base_sort_cls<1>(count, out_buf, decode, elems, st, group);
      case 2: return base_sort_cls<2>(count, out_buf, decode, elems, st, group);
      case 3: return base_sort_cls<3>(count, out_buf, decode, elems, st, group);
      default:
        if constexpr (S::kMaxClass >= 4) return base_sort_cls<4>(count, out_buf, decode, elems, st, group);
        return set_error(PDQ_ERR_INTERNAL, "base class out of range");
    }
  }

  // O(n log n) fallback for one bucket (Sec. 4.1): shared-memory sorts of runs of base_cap
  // elements, then merge-path passes, ping-ponging between the key and temp buffers so that
  // the last pass lands decoded in the key buffer.
  int fallback(const Item& it) {
    const int64_t run = cap_;
    int passes = 0;
    while ((run << passes) < (int64_t)it.size) ++passes;
    const int x = (passes % 2 == 0) ? kBufKeys : kBufTmp;
    const int64_t ntiles = ((int64_t)it.size + run - 1) / run;
    std::vector<Item> tiles;
    for (int64_t t0 = 0; t0 < ntiles;) {
      const int64_t t1 = std::min<int64_t>(ntiles, t0 + L_.base_cap[base_class_of(run)]);
      tiles.clear();
      for (int64_t t = t0; t < t1; ++t) {
        const int64_t b = t * run;
        tiles.push_back(Item{it.begin + b, (uint32_t)std::min<int64_t>(run, (int64_t)it.size - b), it.buf, it.enc});
      }
      const int cls = base_class_of(run);
      PDQ_CUDA(cudaMemcpyAsync(base_items_ + L_.base_off[cls], tiles.data(), sizeof(Item) * tiles.size(),
                               cudaMemcpyHostToDevice, st_));
      const int64_t tile_elems = std::min<int64_t>((int64_t)it.size - t0 * run, (t1 - t0) * run);
      int rc = base_sort(cls, (int64_t)tiles.size(), x, passes == 0 ? 1 : 0, tile_elems);
      if (rc) return rc;
      stats_.base_buckets -= (int64_t)tiles.size();  // tiles are not buckets
      PDQ_CUDA(cudaStreamSynchronize(st_));  // tiles buffer is reused by the next batch
      t0 = t1;
    }
    int cur = x;
    for (int p = 1; p <= passes; ++p) {
      const int64_t w = run << (p - 1);
      U* sk = (cur == kBufKeys ? keys_ : tmpk_) + it.begin;
      V* sv = VB ? (cur == kBufKeys ? vals_ : tmpv_) + it.begin : nullptr;
      U* dk = (cur == kBufKeys ? tmpk_ : keys_) + it.begin;
      V* dv = VB ? (cur == kBufKeys ? tmpv_ : vals_) + it.begin : nullptr;
      {
        LaunchScope ls("merge_pass", st_, 2.0 * (double)it.size * (KS + VB));
        if (2 * w >= kMergeTile) {  // pairs span whole tiles: the tiled merge
          MergeArgs<KT, VB> ma;
          ma.a = sk;
          ma.av = sv;
          ma.la = 0;
          ma.b = nullptr;
          ma.bv = nullptr;
          ma.lb = 0;
          ma.out = dk;
          ma.outv = dv;
          ma.w = w;
          ma.n = (int64_t)it.size;
          ma.raw = 0;
          ma.decode = p == passes ? 1 : 0;
          launch_merge_tiles(ma, (int64_t)it.size);
        } else {
          const unsigned blocks = (unsigned)(((int64_t)it.size + 255) / 256);
          merge_pass_kernel<KT, VB><<<blocks, 256, 0, st_>>>(sk, sv, dk, dv, (int64_t)it.size, w, p == passes ? 1 : 0);
        }
      }
      PDQ_LAUNCHED("merge_pass");
      cur = 1 - cur;
    }
    if (cur != kBufKeys) return set_error(PDQ_ERR_INTERNAL, "fallback ended outside the key buffer");
    return PDQ_OK;
  }
};

template <int KT, int VB>
int sort_impl(const SortArgs& a, pdq_stats* stats) {
  const int64_t l0 = launches_so_far();
  PlainSorter<KT, VB> s(a);
  const int rc = s.run();
  if (stats) {
    *stats = s.stats_;
    stats->kernel_launches = launches_so_far() - l0;
  }
  return rc;
}

template <int KT, int VB>
size_t workspace_bytes_impl(int64_t n) {
  return make_layout(n, (int)sizeof(typename Key<KT>::U), VB).total;
}

}  // namespace pdq

#define PDQ_INSTANTIATE(KT)                                                      \
  template int pdq::sort_impl<KT, 0>(const pdq::SortArgs&, pdq_stats*);         \
  template int pdq::sort_impl<KT, 4>(const pdq::SortArgs&, pdq_stats*);         \
  template int pdq::sort_impl<KT, 8>(const pdq::SortArgs&, pdq_stats*);         \
  template size_t pdq::workspace_bytes_impl<KT, 0>(int64_t);                     \
  template size_t pdq::workspace_bytes_impl<KT, 4>(int64_t);                     \
  template size_t pdq::workspace_bytes_impl<KT, 8>(int64_t);
