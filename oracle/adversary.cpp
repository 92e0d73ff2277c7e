// McIlroy's adaptive "killer adversary" for quicksort-like sorts (M. D. McIlroy, "A Killer
// Adversary for Quicksort", Software: Practice and Experience 29(4), 1999), restated here.
//
// TEST INFRASTRUCTURE ONLY (see pdq_oracle.cpp).  Used to pin the oracle's O(n log n) worst
// case (Theorem 2) and its heapsort fallback (Sec. 4.1): the adversary decides the outcome of
// each comparison lazily so as to make every partition as unbalanced as it can.
//
// Every item starts as "gas" (value not yet decided; gas compares above every decided value).
// When two gas items meet, one of them is frozen to the next "solid" value; the adversary
// freezes the one it believes is the pivot (the last gas item that was compared against a
// solid one).  Once the sort finishes, the remaining gas items get fresh values above all
// solid ones; re-running the sort on those concrete values repeats the same comparisons.

#include <cstdint>
#include <vector>

extern "C" {
typedef struct {
  int64_t insertion_threshold, ninther_threshold, partial_limit, bad_allowed_override;
} oracle_params;
typedef struct {
  int64_t comparisons, heapsort_calls, bad_partitions, partition_right_calls, partition_left_calls,
      partial_insertion_successes, insertion_sort_calls, max_depth;
} oracle_stats;
void oracle_pdqsort_callback(int64_t* items, int64_t n, int (*less)(int64_t, int64_t, void*),
                             void* ctx, const oracle_params* p, oracle_stats* st);
}

namespace {

struct Adversary {
  std::vector<int64_t> val;
  int64_t gas;
  int64_t nsolid = 0;
  int64_t candidate = -1;

  void freeze(int64_t x) { val[x] = nsolid++; }

  bool less(int64_t x, int64_t y) {
    if (val[x] == gas && val[y] == gas) {
      if (x == candidate) freeze(x);
      else freeze(y);
    }
    if (val[x] == gas) candidate = x;
    else if (val[y] == gas) candidate = y;
    return val[x] < val[y];
  }
};

int adversary_less(int64_t x, int64_t y, void* ctx) {
  return static_cast<Adversary*>(ctx)->less(x, y) ? 1 : 0;
}

}  // namespace

extern "C" {
// Runs the oracle against the adversary on n items.  Writes the concrete killer input
// (values[i] = final value of item i) and the oracle's statistics for that run.
void oracle_killer_adversary(int64_t n, const oracle_params* p, oracle_stats* st, int64_t* values) {
  Adversary adv;
  adv.gas = n;  // above every solid value 0..n-1
  adv.val.assign(n, adv.gas);
  std::vector<int64_t> items(n);
  for (int64_t i = 0; i < n; ++i) items[i] = i;
  oracle_pdqsort_callback(items.data(), n, adversary_less, &adv, p, st);
  for (int64_t i = 0; i < n; ++i) {
    if (adv.val[i] == adv.gas) adv.val[i] = adv.nsolid++;
    values[i] = adv.val[i];
  }
}
}
