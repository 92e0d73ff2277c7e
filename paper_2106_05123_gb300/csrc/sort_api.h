// Internal interface between the C ABI (api.cu) and the per-dtype sort instantiations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pdq.h"

namespace pdq {

struct Tuning {
  int logb;          // log2 of the largest bucket count per level
  int oversample;    // samples per bucket (power of two)
  int base_cap;      // largest bucket for the shared-memory base sort (power of two)
  int bad_allowed;   // >0 forced start of the bad-split counter, -1 start at 0, 0 floor(log2 n)
  bool probe;        // run the sorted / reverse probe
  int wait_us;       // bound of the persistent kernel's waits (0: 2 s)
  int inject_wait;   // test hook: the persistent kernel first waits on a flag nobody sets
  int seg_block;     // persistent kernel block size (256 or 512)
  bool fixup;        // try the nearly-sorted fix-up
};

struct SortArgs {
  void* keys;
  void* vals;
  int64_t n;
  void* ws;
  size_t ws_bytes;
  cudaStream_t stream;
  Tuning tune;
  int num_sms;
  // host-buffer form (pdq_sort_host): the sorted keys / values are copied here, each range as
  // soon as it is final, while later ranges are still sorting (null: device result only)
  void* host_keys = nullptr;
  void* host_vals = nullptr;
};

// Byte offsets of the workspace regions.
struct Layout {
  // round_in: one round's task list, per-task metadata and chunk list, uploaded in one copy
  size_t tmpk, tmpv, slots, ctr, round_in, tasks_next, counts, totals, tree, spl, children, pref, tab,
      base_items, copy_items, fb_items, msplit, total;
  int64_t task_cap, round_cap, chunk_cap, item_cap, fb_cap;
  int64_t base_off[5];  // first entry of each base-sort size class's list (in items)
  int64_t base_cap[5];  // capacity of each class's list
  int64_t base_total;   // items of one position group's lists
  int64_t base_groups;  // position groups of the base lists (1, or kOutGroups for large arrays)
  size_t learned_xs, learned_out, learned_sync;  // learned path only
  int64_t learned_m;
  // nearly-sorted fix-up (absent in nested sorts and below kFixMin elements): peeled keys and
  // values (up to fix_m), per-tile counts, and the workspace of the peeled keys' own sort
  size_t fix_e, fix_ev, fix_cnt, fix_mask, fix_ws, fix_ws_bytes;
  int64_t fix_m;
};

// Arguments of the segmented sort.
struct SegArgs {
  void* keys;
  void* vals;
  const int64_t* offsets;
  int64_t nseg;
  int64_t n;
  void* ws;
  size_t ws_bytes;
  cudaStream_t stream;
  Tuning tune;
  int num_sms;
};

int set_error(int code, const std::string& msg);

template <int KT, int VB>
int sort_impl(const SortArgs& a, pdq_stats* stats);
template <int KT, int VB>
size_t workspace_bytes_impl(int64_t n);
template <int KT, int VB>
int seg_sort_impl(const SegArgs& a, pdq_stats* stats);
int learned_sort_f32(const SortArgs& a, pdq_stats* stats);
size_t learned_workspace_bytes(int64_t n);
template <int KT, int VB>
size_t seg_workspace_bytes_impl(int64_t n, int64_t nseg);

// Tuning recorded by pdq_autotune for a call shape (autotune.cu); false when none was recorded.
bool autotune_lookup(bool seg, int dt, int vb, int64_t n, int64_t nseg, pdq_tuning* out);

}  // namespace pdq
