// Instantiation of the plain sort path for PDQ_F32 keys (keys only, 4-byte and 8-byte payloads; plain and segmented).
#include "seg_impl.cuh"
#include "sort_impl.cuh"
PDQ_INSTANTIATE(PDQ_F32)
PDQ_INSTANTIATE_SEG(PDQ_F32)

namespace pdq {

size_t learned_workspace_bytes(int64_t n) { return make_layout(n, 4, 0, true).total; }

// The learned-CDF path (float32 keys, no values) shares this unit's kernels and their
// shared-memory attributes with the plain float32 path.
int learned_sort_f32(const SortArgs& a, pdq_stats* stats) {
  const int64_t l0 = launches_so_far();
  PlainSorter<PDQ_F32, 0> s(a, true);
  const int rc = s.run_learned();
  if (stats) {
    *stats = s.stats_;
    stats->kernel_launches = launches_so_far() - l0;
  }
  return rc;
}

}  // namespace pdq
