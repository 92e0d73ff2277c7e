// Independent checker for the oracle: a naive top-down merge sort.
//
// TEST INFRASTRUCTURE ONLY (see pdq_oracle.cpp).  It deliberately shares no code with the
// pdqsort oracle: its own recursion, its own merge, and its own statement of the float order.
// Keys are compared through an exact integer rank:
//   * integers: the value itself widened to a signed 128-bit-safe pair (sign, magnitude) via
//     plain comparisons of the native type;
//   * float32: IEEE 754-2008 totalOrder expressed as a signed 64-bit rank: a positive-signed
//     datum ranks by its 31 magnitude bits (0 .. 2^31-1), a negative-signed one by
//     -(magnitude bits) - 1, so -0 ranks -1 < +0 at 0, -NaN lowest, +NaN highest;
//   * composite records: the pair (rank of field 0, rank of field 1), compared first by field 0.
// The sort is stable, so for pairs it yields one particular valid order (ties by input order).

#include <cstdint>
#include <cstring>
#include <vector>

namespace {

inline int64_t float_rank(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const int64_t mag = (int64_t)(u & 0x7FFFFFFFu);
  return (u >> 31) ? -mag - 1 : mag;
}

template <class K>
inline bool key_before(const K& a, const K& b) { return a < b; }
template <>
inline bool key_before<float>(const float& a, const float& b) { return float_rank(a) < float_rank(b); }

// Composite records (two 4-byte fields), ordered by the pair of exact ranks (first, second).
struct RecI32I32 {
  int32_t first, second;
};
struct RecF32U32 {
  float first;
  uint32_t second;
};
template <>
inline bool key_before<RecI32I32>(const RecI32I32& a, const RecI32I32& b) {
  const int64_t a1 = a.first, b1 = b.first, a2 = a.second, b2 = b.second;
  return a1 != b1 ? a1 < b1 : a2 < b2;
}
template <>
inline bool key_before<RecF32U32>(const RecF32U32& a, const RecF32U32& b) {
  const int64_t a1 = float_rank(a.first), b1 = float_rank(b.first);
  const int64_t a2 = a.second, b2 = b.second;
  return a1 != b1 ? a1 < b1 : a2 < b2;
}

template <class K, class V>
void merge_rec(K* k, V* v, K* tk, V* tv, int64_t lo, int64_t hi, bool with_vals) {
  if (hi - lo < 2) return;
  const int64_t mid = lo + (hi - lo) / 2;
  merge_rec(k, v, tk, tv, lo, mid, with_vals);
  merge_rec(k, v, tk, tv, mid, hi, with_vals);
  int64_t a = lo, b = mid, o = lo;
  while (a < mid && b < hi) {
    // take from the right run only when strictly smaller: stable
    if (key_before(k[b], k[a])) {
      tk[o] = k[b];
      if (with_vals) tv[o] = v[b];
      ++b;
    } else {
      tk[o] = k[a];
      if (with_vals) tv[o] = v[a];
      ++a;
    }
    ++o;
  }
  while (a < mid) { tk[o] = k[a]; if (with_vals) tv[o] = v[a]; ++a; ++o; }
  while (b < hi) { tk[o] = k[b]; if (with_vals) tv[o] = v[b]; ++b; ++o; }
  for (int64_t i = lo; i < hi; ++i) {
    k[i] = tk[i];
    if (with_vals) v[i] = tv[i];
  }
}

template <class K, class V>
void msort(K* k, V* v, int64_t n) {
  if (n < 2) return;
  std::vector<K> tk(n);
  std::vector<V> tv(v ? n : 1);
  merge_rec(k, v ? v : tv.data(), tk.data(), tv.data(), 0, n, v != nullptr);
}

}  // namespace

extern "C" {
void check_mergesort_i32(int32_t* k, uint32_t* v, int64_t n) { msort<int32_t, uint32_t>(k, v, n); }
void check_mergesort_u32(uint32_t* k, uint32_t* v, int64_t n) { msort<uint32_t, uint32_t>(k, v, n); }
void check_mergesort_i64(int64_t* k, uint32_t* v, int64_t n) { msort<int64_t, uint32_t>(k, v, n); }
void check_mergesort_u64(uint64_t* k, uint32_t* v, int64_t n) { msort<uint64_t, uint32_t>(k, v, n); }
void check_mergesort_f32(float* k, uint32_t* v, int64_t n) { msort<float, uint32_t>(k, v, n); }
void check_mergesort_i32i32(RecI32I32* k, uint32_t* v, int64_t n) { msort<RecI32I32, uint32_t>(k, v, n); }
void check_mergesort_f32u32(RecF32U32* k, uint32_t* v, int64_t n) { msort<RecF32U32, uint32_t>(k, v, n); }
}
