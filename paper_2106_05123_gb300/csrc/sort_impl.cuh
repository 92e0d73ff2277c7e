// Host driver of the plain path: probe, distribution levels, base sorts, fallback.
#pragma once

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "sort_api.h"

namespace pdq {

// ------------------------------------------------------------------ workspace layout
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline int64_t chunk_min_for(int64_t n) {
  const int64_t c = (n + 4095) / 4096;
  return c > 8192 ? c : 8192;
}

inline Layout make_layout(int64_t n, int ks, int vb) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  const int64_t cmin = kBaseCapMin;
  L.task_cap = n / (cmin + 1) + 2;
  L.round_cap = std::min<int64_t>(kTaskRound, L.task_cap);
  L.chunk_cap = n / chunk_min_for(n) + 1 + L.round_cap;
  L.item_cap = std::min<int64_t>(L.round_cap * kBMax, n + 1);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.tmpk = take((size_t)n * ks);
  L.tmpv = take((size_t)n * vb);
  L.ctr = take(sizeof(Counters));
  L.tasks_cur = take((size_t)L.round_cap * sizeof(Task));
  L.tasks_next = take((size_t)L.task_cap * sizeof(Task));
  L.task_meta = take((size_t)L.round_cap * 3 * sizeof(int32_t));
  L.chunks = take((size_t)L.chunk_cap * sizeof(Chunk));
  L.counts = take((size_t)L.chunk_cap * kBinsMax * sizeof(uint32_t));
  L.tree = take((size_t)L.round_cap * kBMax * ks);
  L.spl = take((size_t)L.round_cap * kBMax * ks);
  L.children = take((size_t)L.round_cap * kBinsMax * sizeof(uint2));
  L.base_items = take((size_t)L.item_cap * sizeof(Item));
  L.copy_items = take((size_t)L.item_cap * sizeof(Item));
  L.fb_items = take((size_t)L.item_cap * sizeof(Item));
  L.total = off;
  return L;
}

// ------------------------------------------------------------------ tile shapes
template <int KS, int VB>
struct Shape {
  static constexpr int kScatterThreads = 512;
  static constexpr int kBytes = KS + VB;
  static constexpr int kItems = kBytes <= 4 ? 16 : (kBytes <= 8 ? 8 : 4);
  static constexpr int kTile = kScatterThreads * kItems;
  static constexpr size_t kScatterSmem = (size_t)kTile * (KS + VB + 2);
  static constexpr int kCountThreads = 512;
  static constexpr int kSampleThreads = 512;
  static constexpr int kBaseThreads = 256;
  static constexpr size_t base_smem(int cap) { return (size_t)cap * (KS + VB + (VB ? 4 : 0)); }
};

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
  PlainSorter(const SortArgs& a) : a_(a) {
    L_ = make_layout(a.n, KS, VB);
    char* ws = static_cast<char*>(a.ws);
    keys_ = static_cast<U*>(a.keys);
    vals_ = static_cast<V*>(a.vals);
    tmpk_ = reinterpret_cast<U*>(ws + L_.tmpk);
    tmpv_ = reinterpret_cast<V*>(ws + L_.tmpv);
    ctr_ = reinterpret_cast<Counters*>(ws + L_.ctr);
    tasks_ = reinterpret_cast<Task*>(ws + L_.tasks_cur);
    next_ = reinterpret_cast<Task*>(ws + L_.tasks_next);
    meta_ = reinterpret_cast<int32_t*>(ws + L_.task_meta);
    chunks_ = reinterpret_cast<Chunk*>(ws + L_.chunks);
    counts_ = reinterpret_cast<uint32_t*>(ws + L_.counts);
    tree_ = reinterpret_cast<U*>(ws + L_.tree);
    spl_ = reinterpret_cast<U*>(ws + L_.spl);
    children_ = reinterpret_cast<uint2*>(ws + L_.children);
    base_items_ = reinterpret_cast<Item*>(ws + L_.base_items);
    copy_items_ = reinterpret_cast<Item*>(ws + L_.copy_items);
    fb_items_ = reinterpret_cast<Item*>(ws + L_.fb_items);
    st_ = a.stream;
  }

  int run() {
    if (a_.ws_bytes < L_.total) return set_error(PDQ_ERR_WORKSPACE, "workspace too small");
    int rc = configure();
    if (rc) return rc;
    const int64_t n = a_.n;
    if (n <= 1) return PDQ_OK;
    const int cap = a_.tune.base_cap;
    if (n <= cap) {
      Item it{0, (uint32_t)n, kBufKeys, 0};
      PDQ_CUDA(cudaMemcpyAsync(base_items_, &it, sizeof(it), cudaMemcpyHostToDevice, st_));
      return base_sort(1, kBufKeys, 1, n);
    }
    if (a_.tune.probe) {
      bool done = false;
      rc = probe(&done);
      if (rc || done) return rc;
    }
    const int bad0 = a_.tune.bad_allowed > 0 ? a_.tune.bad_allowed
                                              : (a_.tune.bad_allowed < 0 ? 0 : ilog2_floor((uint64_t)n));
    if (bad0 == 0) {
      Item it{0, (uint32_t)n, kBufKeys, 0};
      ++stats_.fallback_buckets;
      return fallback(it);
    }
    std::vector<Task> cur(1);
    cur[0] = Task{0, n, kBufKeys, 0, bad0, 0};
    while (!cur.empty()) {
      std::vector<Task> nxt;
      ++stats_.passes;
      for (size_t r0 = 0; r0 < cur.size(); r0 += (size_t)L_.round_cap) {
        const size_t r1 = std::min(cur.size(), r0 + (size_t)L_.round_cap);
        rc = level_round(cur.data() + r0, (int)(r1 - r0), &nxt);
        if (rc) return rc;
      }
      cur.swap(nxt);
    }
    return PDQ_OK;
  }

  pdq_stats stats_{};

 private:
  SortArgs a_;
  Layout L_;
  U *keys_, *tmpk_, *tree_, *spl_;
  V *vals_, *tmpv_;
  Counters* ctr_;
  Task *tasks_, *next_;
  int32_t* meta_;
  Chunk* chunks_;
  uint32_t* counts_;
  uint2* children_;
  Item *base_items_, *copy_items_, *fb_items_;
  cudaStream_t st_;

  int configure() {
    static bool done = false;  // per template instantiation
    if (done) return PDQ_OK;
    PDQ_CUDA(cudaFuncSetAttribute(scatter_kernel<KT, VB, S::kScatterThreads, S::kItems>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kScatterSmem));
    PDQ_CUDA(cudaFuncSetAttribute(base_sort_kernel<KT, VB, S::kBaseThreads>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)S::base_smem(kBaseCapMax)));
    done = true;
    return PDQ_OK;
  }

  // Sorted / reverse probe (Sec. 5.2): a sample first, the full pass only when the sample is
  // monotone.  Sets *done when the array needs nothing more.
  int probe(bool* done) {
    const int64_t n = a_.n;
    unsigned long long h[4];
    auto run_probe = [&](int64_t stride) -> int {
      const unsigned long long init[4] = {0, 0, ~0ull, 0};
      PDQ_CUDA(cudaMemcpyAsync(ctr_->probe, init, sizeof(init), cudaMemcpyHostToDevice, st_));
      const int64_t m = (n - 1) / stride + 1;
      const int threads = 256;
      int blocks = (int)std::min<int64_t>((m + threads - 1) / threads, (int64_t)a_.num_sms * 8);
      if (blocks < 1) blocks = 1;
      {
        LaunchScope ls("probe", st_, (double)m * KS);
        probe_kernel<KT><<<blocks, threads, 0, st_>>>(keys_, n, stride, m, ctr_->probe);
      }
      PDQ_LAUNCHED("probe");
      PDQ_CUDA(cudaMemcpyAsync(h, ctr_->probe, sizeof(h), cudaMemcpyDeviceToHost, st_));
      PDQ_CUDA(cudaStreamSynchronize(st_));
      return PDQ_OK;
    };
    const int64_t stride = std::max<int64_t>(1, n / 65536);
    int rc = run_probe(stride);
    if (rc) return rc;
    if (stride > 1 && h[0] != 0 && h[1] != 0) return PDQ_OK;  // sample is neither monotone
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
        reverse_kernel<U><<<blocks, threads, 0, st_>>>(keys_, n);
        if (VB) reverse_kernel<V><<<blocks, threads, 0, st_>>>(vals_, n);
      }
      PDQ_LAUNCHED("reverse");
      return PDQ_OK;
    }
    return PDQ_OK;
  }

  int choose_logb(int64_t size) const {
    const int64_t half = std::max<int64_t>(1, a_.tune.base_cap / 2);
    const int64_t want = (size + half - 1) / half;
    int lb = 1;
    while ((int64_t(1) << lb) < want && lb < a_.tune.logb) ++lb;
    return lb;
  }

  // One distribution level over tasks[0..nt): sample, count, scan, scatter, bookkeeping, then
  // base sorts / copies / fallbacks of the children that finished.  Next tasks are appended.
  int level_round(const Task* tasks, int nt, std::vector<Task>* nxt) {
    const int64_t n = a_.n;
    int64_t total = 0;
    for (int i = 0; i < nt; ++i) total += tasks[i].size;
    int64_t ch = std::max<int64_t>(chunk_min_for(n), (total + a_.num_sms * 4 - 1) / (a_.num_sms * 4));
    std::vector<int32_t> meta(3 * (size_t)nt);
    std::vector<Chunk> chunks;
    chunks.reserve((size_t)(total / ch + nt + 1));
    int max_logb = 1;
    for (int i = 0; i < nt; ++i) {
      const int lb = choose_logb(tasks[i].size);
      max_logb = std::max(max_logb, lb);
      meta[i] = lb;
      meta[nt + i] = (int32_t)chunks.size();
      int32_t nc = 0;
      for (int64_t o = 0; o < tasks[i].size; o += ch, ++nc)
        chunks.push_back(Chunk{tasks[i].begin + o, (int32_t)std::min<int64_t>(ch, tasks[i].size - o), i});
      meta[2 * nt + i] = nc;
    }
    const int nchunks = (int)chunks.size();
    if (nchunks > L_.chunk_cap) return set_error(PDQ_ERR_INTERNAL, "chunk capacity exceeded");
    int32_t* d_logb = meta_;
    int32_t* d_c0 = meta_ + nt;
    int32_t* d_nc = meta_ + 2 * nt;
    PDQ_CUDA(cudaMemcpyAsync(tasks_, tasks, sizeof(Task) * nt, cudaMemcpyHostToDevice, st_));
    PDQ_CUDA(cudaMemcpyAsync(meta_, meta.data(), sizeof(int32_t) * meta.size(), cudaMemcpyHostToDevice, st_));
    PDQ_CUDA(cudaMemcpyAsync(chunks_, chunks.data(), sizeof(Chunk) * nchunks, cudaMemcpyHostToDevice, st_));
    PDQ_CUDA(cudaMemsetAsync(ctr_, 0, offsetof(Counters, probe), st_));

    int oversample = a_.tune.oversample;
    {
      LaunchScope ls("sample", st_, 0.0);
      sample_kernel<KT, S::kSampleThreads><<<nt, S::kSampleThreads, 0, st_>>>(
          tasks_, d_logb, oversample, keys_, tmpk_, tree_, spl_);
    }
    PDQ_LAUNCHED("sample");
    {
      LaunchScope ls("count", st_, (double)total * KS);
      count_kernel<KT, S::kCountThreads><<<nchunks, S::kCountThreads, 0, st_>>>(
          chunks_, tasks_, d_logb, keys_, tmpk_, tree_, spl_, counts_);
    }
    PDQ_LAUNCHED("count");
    {
      LaunchScope ls("scan", st_, 0.0);
      scan_kernel<256><<<nt, 256, 0, st_>>>(d_logb, d_c0, d_nc, counts_, children_);
    }
    PDQ_LAUNCHED("scan");
    {
      LaunchScope ls("scatter", st_, 2.0 * (double)total * (KS + VB));
      scatter_kernel<KT, VB, S::kScatterThreads, S::kItems>
          <<<nchunks, S::kScatterThreads, S::kScatterSmem, st_>>>(
              chunks_, tasks_, d_logb, keys_, vals_, tmpk_, tmpv_, tree_, spl_, counts_);
    }
    PDQ_LAUNCHED("scatter");
    {
      LaunchScope ls("bookkeep", st_, 0.0);
      dim3 grid((unsigned)((2 << max_logb) + 255) / 256, (unsigned)nt);
      bookkeep_kernel<<<grid, 256, 0, st_>>>(tasks_, d_logb, children_, a_.tune.base_cap, ctr_, next_,
                                               base_items_, copy_items_, fb_items_, L_.task_cap,
                                               L_.item_cap);
    }
    PDQ_LAUNCHED("bookkeep");
    Counters h;
    PDQ_CUDA(cudaMemcpyAsync(&h, ctr_, sizeof(Counters), cudaMemcpyDeviceToHost, st_));
    PDQ_CUDA(cudaStreamSynchronize(st_));
    if (h.overflow) return set_error(PDQ_ERR_INTERNAL, "bookkeeping list capacity exceeded");
    stats_.equal_buckets += (int64_t)h.equal_buckets;
    stats_.bad_splits += (int64_t)h.bad_splits;
    if (h.n_base[0]) {
      int rc = base_sort((int64_t)h.n_base[0], kBufKeys, 1, (int64_t)h.base_elems);
      if (rc) return rc;
    }
    if (h.n_copy) {
      LaunchScope ls("copy", st_, 2.0 * (double)h.copy_elems * (KS + VB));
      dim3 grid((unsigned)h.n_copy, 16);
      copy_kernel<KT, VB><<<grid, 256, 0, st_>>>(copy_items_, keys_, vals_, tmpk_, tmpv_);
    }
    PDQ_LAUNCHED("copy");
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

  // Base sort of `count` items (holding `elems` elements) already in base_items_.
  int base_sort(int64_t count, int out_buf, int decode, int64_t elems) {
    const int cap = a_.tune.base_cap;
    stats_.base_buckets += count;
    for (int64_t done = 0; done < count;) {
      const int64_t g = std::min<int64_t>(count - done, 1 << 30);
      LaunchScope ls("base_sort", st_, done == 0 ? 2.0 * (double)elems * (KS + VB) : 0.0);
      base_sort_kernel<KT, VB, S::kBaseThreads><<<(unsigned)g, S::kBaseThreads, S::base_smem(cap), st_>>>(
          base_items_ + done, cap, keys_, vals_, tmpk_, tmpv_, out_buf, decode);
      done += g;
    }
    PDQ_LAUNCHED("base_sort");
    return PDQ_OK;
  }

  // O(n log n) fallback for one bucket (Sec. 4.1): shared-memory sorts of runs of base_cap
  // elements, then merge-path passes, ping-ponging between the key and temp buffers so that
  // the last pass lands decoded in the key buffer.
  int fallback(const Item& it) {
    const int64_t run = a_.tune.base_cap;
    int passes = 0;
    while ((run << passes) < (int64_t)it.size) ++passes;
    const int x = (passes % 2 == 0) ? kBufKeys : kBufTmp;
    const int64_t ntiles = ((int64_t)it.size + run - 1) / run;
    std::vector<Item> tiles;
    for (int64_t t0 = 0; t0 < ntiles;) {
      const int64_t t1 = std::min<int64_t>(ntiles, t0 + L_.item_cap);
      tiles.clear();
      for (int64_t t = t0; t < t1; ++t) {
        const int64_t b = t * run;
        tiles.push_back(Item{it.begin + b, (uint32_t)std::min<int64_t>(run, (int64_t)it.size - b), it.buf, it.enc});
      }
      PDQ_CUDA(cudaMemcpyAsync(base_items_, tiles.data(), sizeof(Item) * tiles.size(), cudaMemcpyHostToDevice, st_));
      const int64_t tile_elems = std::min<int64_t>((int64_t)it.size - t0 * run, (t1 - t0) * run);
      int rc = base_sort((int64_t)tiles.size(), x, passes == 0 ? 1 : 0, tile_elems);
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
      const unsigned blocks = (unsigned)(((int64_t)it.size + 255) / 256);
      {
        LaunchScope ls("merge_pass", st_, 2.0 * (double)it.size * (KS + VB));
        merge_pass_kernel<KT, VB><<<blocks, 256, 0, st_>>>(sk, sv, dk, dv, (int64_t)it.size, w, p == passes ? 1 : 0);
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
