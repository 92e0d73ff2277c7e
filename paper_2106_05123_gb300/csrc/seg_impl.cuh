// Host driver of the batched segmented sort (one persistent launch, captured in a CUDA graph).
#pragma once

#include <map>
#include <mutex>
#include <tuple>

#include "graph_cache.h"
#include "seg.cuh"
#include "sort_impl.cuh"

namespace pdq {

constexpr int64_t kSegPersistMax = int64_t(1) << 20;  // larger segments use the multi-CTA path

struct SegLayout {
  size_t tmpk, tmpv, state, slots0, ready0, slots1, ready1, fb, huge, total;
  int64_t cap0, cap1, fb_cap, huge_cap;
  size_t blist[kBaseClasses];
  int64_t bcap[kBaseClasses];
};

inline SegLayout make_seg_layout(int64_t n, int64_t nseg, int ks, int vb) {
  SegLayout L;
  std::memset(&L, 0, sizeof(L));
  const int64_t cmin = 2048;  // smallest base capacity of the persistent kernel
  L.cap0 = 4 * (n / (cmin + 1) + 1) + nseg + 64;
  L.cap1 = std::min<int64_t>(n + 1, nseg + 16 * (n / cmin + 1) + 4096);
  L.fb_cap = n / (cmin + 1) + nseg + 64;
  L.huge_cap = n / (kSegPersistMax + 1) + 2;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.tmpk = take((size_t)n * ks);  // same place as the plain path's temp buffers
  L.tmpv = take((size_t)n * vb);
  L.state = take(sizeof(SegState));
  L.slots0 = take((size_t)L.cap0 * sizeof(SegTask));
  L.ready0 = take((size_t)L.cap0 * sizeof(uint32_t));
  L.slots1 = take((size_t)L.cap1 * sizeof(SegTask));
  L.ready1 = take((size_t)L.cap1 * sizeof(uint32_t));
  L.fb = take((size_t)L.fb_cap * sizeof(Item));
  L.huge = take((size_t)L.huge_cap * sizeof(Item));
  // size-class lists: an entry of class c >= 1 has more than 512 << c elements, so at most
  // n / (512 << c) of them exist; class 0 gets one entry per segment plus n / 256 (a full list
  // sends further buckets to the persistent kernel's own base queue)
  for (int c = 0; c < kBaseClasses; ++c) {
    L.bcap[c] = c == 0 ? nseg + n / 256 + 1024 : n / ((int64_t)512 << c) + 1;
    L.blist[c] = take((size_t)L.bcap[c] * sizeof(Item));
  }
  L.total = off;
  return L;
}

template <int KT, int VB>
size_t seg_workspace_bytes_impl(int64_t n, int64_t nseg) {
  const int ks = (int)sizeof(typename Key<KT>::U);
  return std::max(make_seg_layout(n, nseg, ks, VB).total, make_layout(n, ks, VB).total);
}

template <int KT, int VB>
class SegSorter {
  using U = typename Key<KT>::U;
  using V = typename Val<VB>::T;
  static constexpr int KS = sizeof(U);
  static constexpr int ITEMS = KS == 4 ? 16 : 8;

 public:
  explicit SegSorter(const SegArgs& a) : a_(a) {}

  int run(pdq_stats* stats) {
    const int64_t n = a_.n, nseg = a_.nseg;
    SegLayout L = make_seg_layout(n, nseg, KS, VB);
    if (a_.ws_bytes < seg_workspace_bytes_impl<KT, VB>(n, nseg))
      return set_error(PDQ_ERR_WORKSPACE, "workspace too small");
    if (nseg == 0 || n <= 1) return PDQ_OK;
    char* ws = static_cast<char*>(a_.ws);
    SegState* st = reinterpret_cast<SegState*>(ws + L.state);
    SegLists lists;
    lists.slots[0] = reinterpret_cast<SegTask*>(ws + L.slots0);
    lists.slots[1] = reinterpret_cast<SegTask*>(ws + L.slots1);
    lists.ready[0] = reinterpret_cast<uint32_t*>(ws + L.ready0);
    lists.ready[1] = reinterpret_cast<uint32_t*>(ws + L.ready1);
    lists.cap[0] = L.cap0;
    lists.cap[1] = L.cap1;
    lists.fallback = reinterpret_cast<Item*>(ws + L.fb);
    lists.fb_cap = L.fb_cap;
    lists.huge = reinterpret_cast<Item*>(ws + L.huge);
    lists.huge_cap = L.huge_cap;
    for (int c = 0; c < kBaseClasses; ++c) {
      lists.blist[c] = reinterpret_cast<Item*>(ws + L.blist[c]);
      lists.bcap[c] = c <= S::kMaxClass ? L.bcap[c] : 0;
    }
    lists.max_base = S::kMaxCap;
    SegParams prm;
    prm.max_logb = a_.tune.logb;
    prm.oversample = a_.tune.oversample;
    prm.bad0 = a_.tune.bad_allowed;
    prm.inject_wait = a_.tune.inject_wait;
    prm.persist_max = kSegPersistMax;
    prm.wait_ns = a_.tune.wait_us > 0 ? (uint64_t)a_.tune.wait_us * 1000ull : 2000000000ull;
    const int block = a_.tune.seg_block == 256 ? 256 : 512;
    int rc = block == 256 ? launch<256>(L, st, lists, prm) : launch<512>(L, st, lists, prm);
    if (rc) return rc;
    SegState h;
    PDQ_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, a_.stream));
    PDQ_CUDA(cudaStreamSynchronize(a_.stream));
    std::vector<Item> huge((size_t)std::min<int64_t>((int64_t)h.n_huge, L.huge_cap));
    std::vector<Item> fb((size_t)std::min<int64_t>((int64_t)h.n_fallback, L.fb_cap));
    if (!huge.empty())
      PDQ_CUDA(cudaMemcpyAsync(huge.data(), lists.huge, sizeof(Item) * huge.size(), cudaMemcpyDeviceToHost, a_.stream));
    if (!fb.empty())
      PDQ_CUDA(cudaMemcpyAsync(fb.data(), lists.fallback, sizeof(Item) * fb.size(), cudaMemcpyDeviceToHost, a_.stream));
    PDQ_CUDA(cudaStreamSynchronize(a_.stream));
    stats_.equal_buckets = (int64_t)h.equal_buckets;
    stats_.base_buckets = (int64_t)h.base_buckets;
    for (int c = 0; c <= S::kMaxClass; ++c)
      stats_.base_buckets += (int64_t)std::min<unsigned long long>(h.n_blist[c], (unsigned long long)L.bcap[c]);
    stats_.bad_splits = (int64_t)h.bad_splits;
    stats_.passes = (int64_t)h.max_depth;
    stats_.fallback_buckets = (int64_t)fb.size();
    int status = PDQ_OK;
    if (h.error & 4ull) status = set_error(PDQ_ERR_ARG, "offsets are not non-decreasing within [0, n]");
    else if (h.error & 2ull) status = set_error(PDQ_ERR_INTERNAL, "a segmented work list overflowed");
    else if (h.error & 1ull) status = set_error(PDQ_ERR_TIMEOUT, "a bounded wait of the persistent kernel expired");
    // very large segments: the plain multi-CTA path, one segment at a time (workspace reused)
    for (const Item& it : huge) {
      if (status) break;
      SortArgs sa;
      sa.keys = static_cast<U*>(a_.keys) + it.begin;
      sa.vals = VB ? static_cast<void*>(static_cast<V*>(a_.vals) + it.begin) : nullptr;
      sa.n = it.size;
      sa.ws = a_.ws;
      sa.ws_bytes = a_.ws_bytes;
      sa.stream = a_.stream;
      sa.tune = a_.tune;
      sa.num_sms = a_.num_sms;
      PlainSorter<KT, VB> ps(sa);
      const int r = ps.run();
      if (r) return r;
      stats_.passes = std::max(stats_.passes, ps.stats_.passes);
      stats_.base_buckets += ps.stats_.base_buckets;
      stats_.equal_buckets += ps.stats_.equal_buckets;
      stats_.fallback_buckets += ps.stats_.fallback_buckets;
    }
    // buckets whose bad-split budget ran out (or that did not fit a queue): O(n log n) fallback
    if (!fb.empty()) {
      SortArgs sa;
      sa.keys = a_.keys;
      sa.vals = a_.vals;
      sa.n = n;
      sa.ws = a_.ws;
      sa.ws_bytes = a_.ws_bytes;
      sa.stream = a_.stream;
      sa.tune = a_.tune;
      sa.num_sms = a_.num_sms;
      PlainSorter<KT, VB> ps(sa);
      int r = ps.configure_public();
      for (size_t i = 0; !r && i < fb.size(); ++i) r = ps.fallback_public(fb[i]);
      if (r) return r;
    }
    if (stats) *stats = stats_;
    return status;
  }

  pdq_stats stats_{};

 private:
  SegArgs a_;

  using S = Shape<KS, VB>;

  // Class c of the size-class base sorts: the plain path's base-sort shape for that class.
  template <int CLS>
  int configure_class(int* grid) {
    constexpr int T = S::base_threads(CLS);
    constexpr size_t smem = base_sort_core_smem<KS, VB, T, S::kBaseItems>();
    static bool configured = false;
    if (!configured) {
      PDQ_CUDA(cudaFuncSetAttribute(seg_base_list_kernel<KT, VB, T, S::kBaseItems>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      PDQ_CUDA(cudaFuncSetAttribute(seg_base_list_kernel<KT, VB, T, S::kBaseItems>,
                                    cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
      configured = true;
    }
    int per_sm = 0;
    PDQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_base_list_kernel<KT, VB, T, S::kBaseItems>,
                                                           T, smem));
    *grid = a_.num_sms * (per_sm < 1 ? 1 : per_sm);
    return PDQ_OK;
  }
  template <int CLS>
  int launch_class(int grid, const SegLists& lists, SegState* st, U* keys, V* vals, U* tmpk, V* tmpv,
                   cudaStream_t s) {
    constexpr int T = S::base_threads(CLS);
    constexpr size_t smem = base_sort_core_smem<KS, VB, T, S::kBaseItems>();
    seg_base_list_kernel<KT, VB, T, S::kBaseItems><<<grid, T, smem, s>>>(
        lists.blist[CLS], &st->n_blist[CLS], lists.bcap[CLS], keys, vals, tmpk, tmpv);
    PDQ_LAUNCHED("seg_base_list");
    return PDQ_OK;
  }

  template <int T>
  int launch(const SegLayout& L, SegState* st, const SegLists& lists, const SegParams& prm) {
    constexpr size_t smem = seg_smem<KS, VB, T, ITEMS>();
    static bool configured = false;
    if (!configured) {
      PDQ_CUDA(cudaFuncSetAttribute(seg_persistent_kernel<KT, VB, T, ITEMS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      configured = true;
    }
    int cls_grid[kBaseClasses] = {0, 0, 0, 0, 0};
    {
      int rc = configure_class<0>(&cls_grid[0]);
      if (!rc) rc = configure_class<1>(&cls_grid[1]);
      if (!rc) rc = configure_class<2>(&cls_grid[2]);
      if (!rc) rc = configure_class<3>(&cls_grid[3]);
      if constexpr (S::kMaxClass >= 4) {
        if (!rc) rc = configure_class<4>(&cls_grid[4]);
      }
      if (rc) return rc;
    }
    int per_sm = 0;
    PDQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, seg_persistent_kernel<KT, VB, T, ITEMS>, T, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = a_.num_sms * per_sm;
    const int bin_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((a_.nseg + 255) / 256, 4096));
    char* ws = static_cast<char*>(a_.ws);
    U* keys = static_cast<U*>(a_.keys);
    V* vals = static_cast<V*>(a_.vals);
    U* tmpk = reinterpret_cast<U*>(ws + L.tmpk);
    V* tmpv = reinterpret_cast<V*>(ws + L.tmpv);
    auto enqueue = [&](cudaStream_t s) -> int {
      PDQ_CUDA(cudaMemsetAsync(st, 0, sizeof(SegState), s));
      PDQ_CUDA(cudaMemsetAsync(lists.ready[0], 0, (size_t)L.cap0 * sizeof(uint32_t), s));
      PDQ_CUDA(cudaMemsetAsync(lists.ready[1], 0, (size_t)L.cap1 * sizeof(uint32_t), s));
      seg_bin_kernel<KT><<<bin_blocks, 256, 0, s>>>(a_.offsets, a_.nseg, a_.n, T * ITEMS, prm, st, lists);
      PDQ_LAUNCHED("seg_bin");
      seg_persistent_kernel<KT, VB, T, ITEMS><<<grid, T, smem, s>>>(keys, vals, tmpk, tmpv, st, lists, prm);
      PDQ_LAUNCHED("seg_persistent");
      int rc = launch_class<0>(cls_grid[0], lists, st, keys, vals, tmpk, tmpv, s);
      if (!rc) rc = launch_class<1>(cls_grid[1], lists, st, keys, vals, tmpk, tmpv, s);
      if (!rc) rc = launch_class<2>(cls_grid[2], lists, st, keys, vals, tmpk, tmpv, s);
      if (!rc) rc = launch_class<3>(cls_grid[3], lists, st, keys, vals, tmpk, tmpv, s);
      if constexpr (S::kMaxClass >= 4) {
        if (!rc) rc = launch_class<4>(cls_grid[4], lists, st, keys, vals, tmpk, tmpv, s);
      }
      if (rc) return rc;
      return PDQ_OK;
    };
    GraphKey key{KT, VB, T, prm.max_logb, prm.oversample, prm.bad0, prm.inject_wait, prm.wait_ns,
                 a_.keys, a_.vals, a_.offsets, a_.ws, a_.nseg, a_.n};
    GraphCache& gc = graph_cache();
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> g(gc.mu);
      auto itg = gc.execs.find(key);
      if (itg != gc.execs.end()) exec = itg->second;
    }
    if (!exec) {
      std::lock_guard<std::mutex> g(gc.mu);
      if (!gc.capture_stream) PDQ_CUDA(cudaStreamCreateWithFlags(&gc.capture_stream, cudaStreamNonBlocking));
      PDQ_CUDA(cudaStreamBeginCapture(gc.capture_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = enqueue(gc.capture_stream);
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(gc.capture_stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (ee != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) return set_error(PDQ_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
      if (gc.execs.size() >= 16) {  // small bounded cache
        cudaGraphExecDestroy(gc.execs.begin()->second);
        gc.execs.erase(gc.execs.begin());
      }
      gc.execs[key] = exec;
    }
    {
      LaunchScope ls("seg_graph", a_.stream, 2.0 * (double)a_.n * (KS + VB));
      note_launch_count(1);  // the graph holds two kernels: binning and the persistent kernel
      PDQ_CUDA(cudaGraphLaunch(exec, a_.stream));
    }
    return PDQ_OK;
  }
};

template <int KT, int VB>
int seg_sort_impl(const SegArgs& a, pdq_stats* stats) {
  const int64_t l0 = launches_so_far();
  SegSorter<KT, VB> s(a);
  const int rc = s.run(stats);
  if (stats) stats->kernel_launches = launches_so_far() - l0;
  return rc;
}

}  // namespace pdq

#define PDQ_INSTANTIATE_SEG(KT)                                                     \
  template int pdq::seg_sort_impl<KT, 0>(const pdq::SegArgs&, pdq_stats*);         \
  template int pdq::seg_sort_impl<KT, 4>(const pdq::SegArgs&, pdq_stats*);         \
  template int pdq::seg_sort_impl<KT, 8>(const pdq::SegArgs&, pdq_stats*);         \
  template size_t pdq::seg_workspace_bytes_impl<KT, 0>(int64_t, int64_t);           \
  template size_t pdq::seg_workspace_bytes_impl<KT, 4>(int64_t, int64_t);           \
  template size_t pdq::seg_workspace_bytes_impl<KT, 8>(int64_t, int64_t);
