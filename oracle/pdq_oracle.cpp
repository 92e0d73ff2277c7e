// Oracle: plain, single-threaded pattern-defeating quicksort (Peters, arXiv 2106.05123).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
// and reference legs may load this library.  The GPU product path never calls it.  It shares
// no code with the CUDA sources (no headers, helpers, tables or key transforms).
//
// What it computes: the unstable ascending sort of an array under a strict weak order
// (Sec. 1, Sec. 3).  The result for keys is unique: the ascending arrangement of the multiset.
// For key/value pairs the order of values inside a run of equal keys is unspecified.
//
// How (paper's steps, in the paper's order):
//   * driver: each call either falls back, runs insertion sort, or partitions and recurses;
//     recursion on the left part, iteration on the right part (Sec. 2).
//   * pivot: median of 3 (first, middle, last), Tukey's ninther above a size threshold; the
//     candidates are sorted in place and the median is moved to the front (Sec. 2; Sec. 5.2
//     footnote on linear time for descending input).
//   * partition_right / partition_left with one comparison per element; partition_left is used
//     when the predecessor compares equal to the pivot, and its left part is final (Sec. 3,
//     Fig. 3 semantics; Lemmas 1-4, Theorem 1).
//   * bad partitions: a part smaller than size/8 (p = 1/8, a shift) decrements a per-subtree
//     counter that starts at floor(log2 n); a call that starts with the counter at 0 uses
//     heapsort (Sec. 4.1, Theorem 2).
//   * fresh pivot candidates after a bad partition: swap the first and last candidates with
//     elements at about 25% and 75% of each part, and the ninther candidates too (Sec. 4.2).
//   * insertion sort with moves for small parts, unguarded when not leftmost (Sec. 5.1).
//   * optimistic partial insertion sort after a swapless, not-bad partition (Sec. 5.2).
//
// Readings where the paper leaves a constant open (Sec. 5.1 "16-32", Sec. 2 "sufficiently
// large", Sec. 5.2 "tiny number of corrections") are parameters with defaults 24 / 128 / 8.
// Block partitioning (Sec. 5.3) changes speed, not results, and is not part of the oracle.
//
// Float32 keys are ordered by IEEE 754-2008 totalOrder (Sec. 5.10 of that standard), with the
// order among NaNs of one sign fixed by their payload bits.  Composite keys (two 4-byte fields)
// are ordered lexicographically by their fields' orders.

#include <cstdint>
#include <cstring>
#include <utility>

namespace {

struct Params {
  int64_t insertion_threshold;  // parts smaller than this use insertion sort (Sec. 5.1)
  int64_t ninther_threshold;    // parts larger than this use Tukey's ninther (Sec. 2)
  int64_t partial_limit;        // element moves before a partial insertion sort gives up (Sec. 5.2)
  int64_t bad_allowed_override; // < 0: floor(log2 n) (Sec. 4.1); >= 0: forced start value
};

struct Stats {
  int64_t comparisons;
  int64_t heapsort_calls;
  int64_t bad_partitions;
  int64_t partition_right_calls;
  int64_t partition_left_calls;
  int64_t partial_insertion_successes;
  int64_t insertion_sort_calls;
  int64_t max_depth;
};

int floor_log2(int64_t n) {
  int r = 0;
  while (n > 1) { n >>= 1; ++r; }
  return r;
}

// ---------------------------------------------------------------- comparators
// Integers: numeric order, the native `<`.
template <class T>
struct NumericLess {
  bool operator()(const T& a, const T& b) const { return a < b; }
};

// Float32 totalOrder, stated from the IEEE 754-2008 definition: every negative-signed datum
// (including -NaN and -0) is below every positive-signed one; among positive data a larger
// magnitude is higher (finite < +inf < +NaN, NaNs by payload); among negative data a larger
// magnitude is lower.  The magnitude of a binary32 datum is monotone in its low 31 bits.
struct TotalOrderLess {
  bool operator()(const float& a, const float& b) const {
    uint32_t ua, ub;
    std::memcpy(&ua, &a, 4);
    std::memcpy(&ub, &b, 4);
    const bool neg_a = (ua >> 31) != 0, neg_b = (ub >> 31) != 0;
    if (neg_a != neg_b) return neg_a;  // the negative one is below
    const uint32_t mag_a = ua & 0x7FFFFFFFu, mag_b = ub & 0x7FFFFFFFu;
    return neg_a ? (mag_a > mag_b) : (mag_a < mag_b);
  }
};

// Composite keys (the "small tuples" of Sec. 5.3): records of two 4-byte fields compared
// lexicographically, which is a strict weak order whenever each field's order is one: the first
// field decides unless the two first fields are equivalent (neither below the other), then the
// second field decides.
struct TupleI32I32 {
  int32_t first;
  int32_t second;
};
struct TupleF32U32 {
  float first;      // IEEE 754 totalOrder
  uint32_t second;  // numeric order
};
template <class T, class FirstLess, class SecondLess>
struct LexLess {
  bool operator()(const T& a, const T& b) const {
    const FirstLess f;
    if (f(a.first, b.first)) return true;
    if (f(b.first, a.first)) return false;
    return SecondLess{}(a.second, b.second);
  }
};
using LexLessI32I32 = LexLess<TupleI32I32, NumericLess<int32_t>, NumericLess<int32_t>>;
using LexLessF32U32 = LexLess<TupleF32U32, TotalOrderLess, NumericLess<uint32_t>>;
static_assert(sizeof(TupleI32I32) == 8 && sizeof(TupleF32U32) == 8, "8-byte records");

// A key/value record; ordering looks at the key only (values ride along).
template <class K, class V>
struct Rec {
  K key;
  V val;
};

template <class K, class V, class KeyLess>
struct RecLess {
  KeyLess kl;
  bool operator()(const Rec<K, V>& a, const Rec<K, V>& b) const { return kl(a.key, b.key); }
};

// Comparator given as a C callback over int64 items (used by the adversary harness).
struct CallbackLess {
  int (*fn)(int64_t, int64_t, void*);
  void* ctx;
  bool operator()(const int64_t& a, const int64_t& b) const { return fn(a, b, ctx) != 0; }
};

// ---------------------------------------------------------------- the sort
template <class T, class Less>
class Pdq {
 public:
  Pdq(Less less, const Params& p, Stats* st) : less_(less), p_(p), st_(st) {}

  void sort(T* a, int64_t n) {
    if (n < 2) return;
    const int bad0 = p_.bad_allowed_override >= 0 ? (int)p_.bad_allowed_override : floor_log2(n);
    recurse(a, a + n, bad0, true, 1);
  }

 private:
  Less less_;
  Params p_;
  Stats* st_;

  bool lt(const T& x, const T& y) {
    ++st_->comparisons;
    return less_(x, y);
  }

  // Sort the three elements at x, y, z in place (so that *x <= *y <= *z), using compare-swaps.
  void sort3(T* x, T* y, T* z) {
    if (lt(*y, *x)) std::swap(*x, *y);
    if (lt(*z, *y)) {
      std::swap(*y, *z);
      if (lt(*y, *x)) std::swap(*x, *y);
    }
  }

  // Pivot selection (Sec. 2 and the Sec. 5.2 footnote): candidates are sorted in place and the
  // median ends at the middle position, which is then moved to *begin.  Median of 3 uses the
  // first, middle and last element; the ninther takes the medians of three such triples (each
  // spanning the part) and the median of those three.
  void choose_pivot(T* begin, T* end) {
    const int64_t size = end - begin;
    const int64_t mid = size / 2;
    if (size > p_.ninther_threshold) {
      sort3(begin, begin + mid, end - 1);
      sort3(begin + 1, begin + mid - 1, end - 2);
      sort3(begin + 2, begin + mid + 1, end - 3);
      sort3(begin + mid - 1, begin + mid, begin + mid + 1);
    } else {
      sort3(begin, begin + mid, end - 1);
    }
    std::swap(*begin, begin[mid]);
  }

  // Insertion sort by moves (Sec. 5.1), bounds-checked: for a leftmost part.
  void insertion_sort(T* begin, T* end) {
    ++st_->insertion_sort_calls;
    for (T* cur = begin + 1; cur < end; ++cur) {
      if (!lt(*cur, cur[-1])) continue;
      T held = std::move(*cur);
      T* hole = cur;
      do {
        *hole = std::move(hole[-1]);
        --hole;
      } while (hole > begin && lt(held, hole[-1]));
      *hole = std::move(held);
    }
  }

  // Insertion sort without the lower bound check (Sec. 5.1): valid only when the element just
  // before `begin` (the predecessor) is <= every element of the part, which holds for every
  // part that is not leftmost, because its predecessor is an ancestor's pivot (Lemma 1).
  void unguarded_insertion_sort(T* begin, T* end) {
    ++st_->insertion_sort_calls;
    for (T* cur = begin + 1; cur < end; ++cur) {
      if (!lt(*cur, cur[-1])) continue;
      T held = std::move(*cur);
      T* hole = cur;
      do {
        *hole = std::move(hole[-1]);
        --hole;
      } while (lt(held, hole[-1]));
      *hole = std::move(held);
    }
  }

  // Partial insertion sort (Sec. 5.2): as insertion sort, but gives up (returns false) once the
  // number of element moves exceeds the limit.  The element being inserted is always placed
  // first, so the array stays a permutation of its input.
  bool partial_insertion_sort(T* begin, T* end) {
    int64_t moves = 0;
    for (T* cur = begin + 1; cur < end; ++cur) {
      if (!lt(*cur, cur[-1])) continue;
      T held = std::move(*cur);
      T* hole = cur;
      do {
        *hole = std::move(hole[-1]);
        --hole;
        ++moves;
      } while (hole > begin && lt(held, hole[-1]));
      *hole = std::move(held);
      if (moves > p_.partial_limit) return false;
    }
    return true;
  }

  // partition_right (Sec. 3): pivot p = *begin.  Afterwards [begin, r) < p, *r == p and
  // (r, end) >= p; elements equal to p go right.  Approaching pointers i (from the left, skips
  // elements < p) and j (from the right, skips elements >= p); a pair that violates both
  // invariants is swapped.  `no_swaps` reports that no pair had to be swapped.
  std::pair<T*, bool> partition_right(T* begin, T* end) {
    ++st_->partition_right_calls;
    const T pivot = *begin;
    T* i = begin + 1;  // first element not yet known to be < p
    T* j = end - 1;    // last element not yet known to be >= p
    bool swapped = false;
    for (;;) {
      while (i <= j && lt(*i, pivot)) ++i;
      while (j >= i && !lt(*j, pivot)) --j;
      if (i >= j) break;
      std::swap(*i, *j);
      swapped = true;
      ++i;
      --j;
    }
    T* r = i - 1;  // last element < p (or begin itself when there is none)
    std::swap(*begin, *r);
    return {r, !swapped};
  }

  // partition_left (Sec. 3): pivot p = *begin.  Afterwards [begin, r) <= p, *r == p and
  // (r, end) > p; elements equal to p go left.  Only called when the predecessor equals p, so
  // nothing is < p and the whole left part equals p.
  T* partition_left(T* begin, T* end) {
    ++st_->partition_left_calls;
    const T pivot = *begin;
    T* i = begin + 1;  // first element not yet known to be <= p
    T* j = end - 1;    // last element not yet known to be > p
    for (;;) {
      while (i <= j && !lt(pivot, *i)) ++i;
      while (j >= i && lt(pivot, *j)) --j;
      if (i >= j) break;
      std::swap(*i, *j);
      ++i;
      --j;
    }
    T* r = i - 1;
    std::swap(*begin, *r);
    return r;
  }

  // Textbook binary-heap sort (Williams 1964), the O(n log n) fallback (Sec. 2, Sec. 4.1).
  void sift_down(T* a, int64_t root, int64_t n) {
    for (;;) {
      int64_t child = 2 * root + 1;
      if (child >= n) return;
      if (child + 1 < n && lt(a[child], a[child + 1])) ++child;
      if (!lt(a[root], a[child])) return;
      std::swap(a[root], a[child]);
      root = child;
    }
  }
  void heapsort(T* begin, T* end) {
    ++st_->heapsort_calls;
    const int64_t n = end - begin;
    for (int64_t i = n / 2 - 1; i >= 0; --i) sift_down(begin, i, n);
    for (int64_t last = n - 1; last > 0; --last) {
      std::swap(begin[0], begin[last]);
      sift_down(begin, 0, last);
    }
  }

  // Fresh pivot candidates for one part [b, e) after a bad partition (Sec. 4.2): the first and
  // last candidate are exchanged with elements at about 25% and 75% of the part; when the part
  // is large enough for the ninther, its other outer candidates are exchanged too.
  void refresh_candidates(T* b, T* e) {
    const int64_t m = e - b;
    const int64_t q = m / 4;
    if (m < p_.insertion_threshold || q == 0) return;
    std::swap(b[0], b[q]);
    std::swap(e[-1], e[-q]);
    if (m > p_.ninther_threshold) {
      std::swap(b[1], b[q + 1]);
      std::swap(b[2], b[q + 2]);
      std::swap(e[-2], e[-q - 1]);
      std::swap(e[-3], e[-q - 2]);
    }
  }

  // The driver (Sec. 2, Sec. 4.1): one call sorts [begin, end).  `leftmost` is false when the
  // element before begin (the predecessor) belongs to the same array and is <= the part.
  void recurse(T* begin, T* end, int bad_allowed, bool leftmost, int64_t depth) {
    if (depth > st_->max_depth) st_->max_depth = depth;
    for (;;) {
      const int64_t size = end - begin;
      if (size < p_.insertion_threshold) {
        if (leftmost) insertion_sort(begin, end);
        else unguarded_insertion_sort(begin, end);
        return;
      }
      if (bad_allowed == 0) {
        heapsort(begin, end);
        return;
      }
      choose_pivot(begin, end);

      // Predecessor compares equal to the pivot (it is never greater): partition_left, and the
      // left part (all equal to the pivot) is final (Sec. 3, Lemma 4).
      if (!leftmost && !lt(begin[-1], *begin)) {
        T* r = partition_left(begin, end);
        begin = r + 1;
        continue;
      }

      std::pair<T*, bool> res = partition_right(begin, end);
      T* pos = res.first;
      const bool no_swaps = res.second;
      const int64_t l = pos - begin;
      const int64_t r = end - (pos + 1);
      const int64_t cut = size >> 3;  // p = 1/8 (Sec. 4.1)
      const bool bad = l < cut || r < cut;
      if (bad) {
        ++st_->bad_partitions;
        --bad_allowed;
        refresh_candidates(begin, pos);
        refresh_candidates(pos + 1, end);
      } else if (no_swaps) {
        if (partial_insertion_sort(begin, pos) && partial_insertion_sort(pos + 1, end)) {
          ++st_->partial_insertion_successes;
          return;
        }
      }
      recurse(begin, pos, bad_allowed, leftmost, depth + 1);
      begin = pos + 1;
      leftmost = false;
    }
  }
};

Params params_or_default(const Params* p) {
  if (p) return *p;
  Params d;
  d.insertion_threshold = 24;
  d.ninther_threshold = 128;
  d.partial_limit = 8;
  d.bad_allowed_override = -1;
  return d;
}

template <class T, class Less>
void run(T* a, int64_t n, Less less, const Params* p, Stats* st) {
  Stats local;
  std::memset(&local, 0, sizeof(local));
  Pdq<T, Less> s(less, params_or_default(p), st ? st : &local);
  if (st) std::memset(st, 0, sizeof(Stats));
  s.sort(a, n);
}

template <class K, class V, class KeyLess>
void run_pairs(K* keys, V* vals, int64_t n, const Params* p, Stats* st) {
  Rec<K, V>* recs = new Rec<K, V>[n > 0 ? n : 1];
  for (int64_t i = 0; i < n; ++i) { recs[i].key = keys[i]; recs[i].val = vals[i]; }
  run(recs, n, RecLess<K, V, KeyLess>{KeyLess{}}, p, st);
  for (int64_t i = 0; i < n; ++i) { keys[i] = recs[i].key; vals[i] = recs[i].val; }
  delete[] recs;
}

}  // namespace

// ---------------------------------------------------------------- C entry points
extern "C" {

typedef Params oracle_params;
typedef Stats oracle_stats;

void oracle_default_params(oracle_params* p) { *p = params_or_default(nullptr); }

void oracle_pdqsort_i32(int32_t* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, NumericLess<int32_t>{}, p, st);
}
void oracle_pdqsort_u32(uint32_t* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, NumericLess<uint32_t>{}, p, st);
}
void oracle_pdqsort_i64(int64_t* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, NumericLess<int64_t>{}, p, st);
}
void oracle_pdqsort_u64(uint64_t* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, NumericLess<uint64_t>{}, p, st);
}
void oracle_pdqsort_f32(float* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, TotalOrderLess{}, p, st);
}
void oracle_pdqsort_i32i32(TupleI32I32* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, LexLessI32I32{}, p, st);
}
void oracle_pdqsort_f32u32(TupleF32U32* a, int64_t n, const oracle_params* p, oracle_stats* st) {
  run(a, n, LexLessF32U32{}, p, st);
}

#define ORACLE_PAIRS(NAME, K, LESS)                                                           \
  void oracle_pdqsort_pairs_##NAME##_v32(K* k, uint32_t* v, int64_t n, const oracle_params* p, \
                                          oracle_stats* st) {                                 \
    run_pairs<K, uint32_t, LESS>(k, v, n, p, st);                                             \
  }                                                                                           \
  void oracle_pdqsort_pairs_##NAME##_v64(K* k, uint64_t* v, int64_t n, const oracle_params* p, \
                                          oracle_stats* st) {                                 \
    run_pairs<K, uint64_t, LESS>(k, v, n, p, st);                                             \
  }
ORACLE_PAIRS(i32, int32_t, NumericLess<int32_t>)
ORACLE_PAIRS(u32, uint32_t, NumericLess<uint32_t>)
ORACLE_PAIRS(i64, int64_t, NumericLess<int64_t>)
ORACLE_PAIRS(u64, uint64_t, NumericLess<uint64_t>)
ORACLE_PAIRS(f32, float, TotalOrderLess)
ORACLE_PAIRS(i32i32, TupleI32I32, LexLessI32I32)
ORACLE_PAIRS(f32u32, TupleF32U32, LexLessF32U32)
#undef ORACLE_PAIRS

// Sort int64 items with a caller-supplied strict-weak-order callback (returns nonzero for
// "a < b").  Used to run the sort against an adaptive adversary.
void oracle_pdqsort_callback(int64_t* items, int64_t n, int (*less)(int64_t, int64_t, void*),
                             void* ctx, const oracle_params* p, oracle_stats* st) {
  run(items, n, CallbackLess{less, ctx}, p, st);
}

// Segmented: sort each [offsets[s], offsets[s+1]) independently.
#define ORACLE_SEG(NAME, T, LESS)                                                          \
  void oracle_pdqsort_segmented_##NAME(T* a, const int64_t* offsets, int64_t num_segments, \
                                       const oracle_params* p) {                          \
    for (int64_t s = 0; s < num_segments; ++s)                                            \
      run(a + offsets[s], offsets[s + 1] - offsets[s], LESS{}, p, (oracle_stats*)nullptr); \
  }
ORACLE_SEG(i32, int32_t, NumericLess<int32_t>)
ORACLE_SEG(u32, uint32_t, NumericLess<uint32_t>)
ORACLE_SEG(i64, int64_t, NumericLess<int64_t>)
ORACLE_SEG(u64, uint64_t, NumericLess<uint64_t>)
ORACLE_SEG(f32, float, TotalOrderLess)
ORACLE_SEG(i32i32, TupleI32I32, LexLessI32I32)
ORACLE_SEG(f32u32, TupleF32U32, LexLessF32U32)
#undef ORACLE_SEG

}  // extern "C"
