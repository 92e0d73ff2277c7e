/*
 * pdq.h -- C ABI of the GB300 (sm_103a) pattern-defeating sort library.
 *
 * Operation (Peters, "Pattern-defeating Quicksort", arXiv 2106.05123, Sec. 1 and Sec. 3):
 * sort a contiguous array in place, ascending, unstable, under a strict weak order.  Here the
 * order is numeric for int32/uint32/int64/uint64 keys and IEEE 754-2008 totalOrder for float32
 * keys (a total order on bit patterns: -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN).  The
 * sorted key array is therefore unique and every call produces it bit for bit.  With a value
 * payload, each value stays with its key; the order of values inside a run of equal keys is
 * unspecified (the sort is unstable, Sec. 1).
 *
 * The GPU method keeps the paper's heuristics in data-parallel form:
 *   - equal keys: a splitter that repeats, or any key equal to a splitter, lands in an equality
 *     bucket that is final at once (Sec. 3, Lemma 4 / Theorem 1: O(nk) for k distinct keys);
 *   - sorted / reverse-sorted input exits after a probe, reversing in place when descending
 *     (Sec. 5.2);
 *   - a bucket that keeps more than 7/8 of its parent's keys outside the parent's equality
 *     buckets is a bad split; each subtree has a counter starting at floor(log2 n), and a
 *     bucket whose counter reaches 0 is sorted by a merge-path merge sort, the O(n log n)
 *     fallback (Sec. 4.1, Theorem 2);
 *   - fresh splitter samples after a bad split (Sec. 4.2);
 *   - small buckets are sorted in shared memory (Sec. 5.1).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are HOST pointers.
 *   - Calls are asynchronous on `cuda_stream` (a cudaStream_t; NULL = legacy default stream)
 *     except that the plain paths read a few small counters back from the device between
 *     distribution levels, which synchronises the stream.  Host-side argument errors return at
 *     once without touching the device.
 *   - Workspace: caller-provided device memory of at least pdq_workspace_bytes(...) bytes,
 *     256-byte aligned.  The library allocates no device memory of its own, except the
 *     segmented path's CUDA-graph cache (see pdq_sort_segmented).  On host memory it keeps,
 *     per calling thread and until exit, two small pinned staging buffers (64 KiB or the size
 *     of one level's task and chunk lists) for its uploads and counter read-backs; without
 *     pinned memory it falls back to pageable copies.
 *   - n must be < 2^32.  n = 0 and n = 1 are no-ops.  value_bytes is 4 or 8.
 *   - d_keys and d_vals need their natural alignment.  Internally tiles are staged by 16-byte
 *     bulk copies from the 16-byte boundary at or below d_keys (up to 12 bytes before d_keys are
 *     read, never written); with a payload, d_vals must sit at the same element offset from a
 *     16-byte boundary as d_keys (true for any two arrays from cudaMalloc or PyTorch).
 *   - Return value: PDQ_OK or a negative pdq_status; pdq_last_error() gives a message (per
 *     host thread).  After PDQ_ERR_CUDA / PDQ_ERR_TIMEOUT / PDQ_ERR_INTERNAL the arrays hold
 *     an unspecified permutation of their input pairs.
 *   - stats (nullable): filled on return with counters of the work done.
 */
#ifndef PDQ_H_
#define PDQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key types.  The two composite types are 8-byte records of two 4-byte fields, field 0 at the
 * lower address (offset 0) and field 1 at offset 4, ordered lexicographically: by field 0, then
 * by field 1 (the "small tuples" a branchless comparison sort handles, Sec. 5.3):
 *   PDQ_I32I32: field 0 int32, field 1 int32 (both numeric order);
 *   PDQ_F32U32: field 0 float32 in IEEE 754 totalOrder, field 1 uint32 (e.g. a score and an id).
 * Their key pointer needs 8-byte alignment, like int64 keys. */
typedef enum {
  PDQ_I32 = 0,
  PDQ_U32 = 1,
  PDQ_I64 = 2,
  PDQ_U64 = 3,
  PDQ_F32 = 4,
  PDQ_I32I32 = 5,
  PDQ_F32U32 = 6
} pdq_dtype;

typedef enum {
  PDQ_OK = 0,
  PDQ_ERR_ARG = -1,        /* bad pointer, size, alignment or value_bytes */
  PDQ_ERR_DTYPE = -2,      /* unknown key dtype */
  PDQ_ERR_WORKSPACE = -3,  /* workspace too small or misaligned */
  PDQ_ERR_CUDA = -4,       /* a CUDA call failed (message has the CUDA error string) */
  PDQ_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up (persistent segmented path) */
  PDQ_ERR_INTERNAL = -6    /* a device-side consistency check failed */
} pdq_status;

typedef struct {
  int64_t passes;            /* distribution passes (levels) executed over any bucket */
  int64_t equal_buckets;     /* non-empty equality buckets finished by a splitter (Sec. 3) */
  int64_t fallback_buckets;  /* buckets sorted by the merge-path fallback (Sec. 4.1) */
  int64_t reversed;          /* 1 if the input was strictly non-increasing and was reversed */
  int64_t sorted_exit;       /* 1 if the probe found the input sorted (or all equal) */
  int64_t learned_overflow;  /* learned path: buckets re-partitioned by the exact repair */
  int64_t bad_splits;        /* children that kept more than 7/8 of their parent's non-equal
                                keys (Sec. 4.1) */
  int64_t base_buckets;      /* buckets finished by the shared-memory base sort (Sec. 5.1) */
  int64_t kernel_launches;   /* kernels launched by the call */
  int64_t fixup_peeled;      /* nearly-sorted fix-up: keys peeled off descents and merged back
                                (0 when the fix-up did not run) */
} pdq_stats;

/* Tuning knobs.  Zero in a field means "library default".  Used by tests to force rare paths
 * (tiny bucket counts and base-case sizes, a zero bad-split budget) on small inputs. */
typedef struct {
  int32_t log2_buckets;     /* log2 of buckets per distribution level, 1..9 (default 8) */
  int32_t oversample;       /* samples per bucket for splitter selection (default 16) */
  int32_t base_capacity;    /* largest bucket sorted in shared memory, 256..16384, power of 2 */
  int32_t bad_allowed;      /* >0: start value of the bad-split counter; -1: start at 0 */
  int32_t probe;            /* 0: default (probe on); -1: skip the sorted/reverse probe */
  int32_t wait_limit_us;    /* segmented path: bound of every device-side wait (0: 2 s) */
  int32_t inject_wait;      /* test hook, segmented path: one CTA first waits on a flag nothing
                               sets; with a short wait_limit_us the call returns PDQ_ERR_TIMEOUT */
  int32_t seg_block;        /* segmented path: persistent kernel block size, 256 or 512 (default) */
  int32_t fixup;            /* nearly-sorted fix-up when the probe finds few scattered descents
                               (mark the keys of every descent, repair, sort them apart, merge):
                               0 default (on), -1 off, 1 on */
} pdq_tuning;

/* Bytes of workspace the sort of n keys (and a payload of value_bytes, 0 for keys only) needs.
 * num_segments: 0 for the single-array calls; the segment count (>= 1) for pdq_sort_segmented.
 * Returns 0 for an unknown dtype or value_bytes. */
size_t pdq_workspace_bytes(int64_t n, int64_t num_segments, pdq_dtype key_dtype, int value_bytes);

/* Sort n keys in place (Sec. 1 problem statement).
 *   d_keys   : device array of n keys of key_dtype (4- or 8-byte elements, naturally aligned)
 *   d_ws     : device workspace of ws_bytes >= pdq_workspace_bytes(n, 1, key_dtype, 0)
 *   tuning   : NULL for defaults                                                          */
int pdq_sort_keys(void* d_keys, int64_t n, pdq_dtype key_dtype, void* d_ws, size_t ws_bytes,
                  void* cuda_stream, const pdq_tuning* tuning, pdq_stats* stats);

/* Sort n (key, value) pairs in place by key; values (value_bytes = 4 or 8) move with their key.
 *   d_vals   : device array of n values                                                   */
int pdq_sort_pairs(void* d_keys, void* d_vals, int value_bytes, int64_t n, pdq_dtype key_dtype,
                   void* d_ws, size_t ws_bytes, void* cuda_stream, const pdq_tuning* tuning,
                   pdq_stats* stats);

/* Sort num_segments independent segments [offsets[s], offsets[s+1]) of one array in a single
 * call: segments go to size-binned device work queues served by one persistent kernel (each
 * CTA sorts small segments in shared memory and partitions larger ones, pushing the parts back);
 * the launch is captured in a CUDA graph that is reused while pointers and sizes repeat (this
 * graph cache is the only memory the library allocates; host-side graph objects).  Segments
 * above 2^20 keys use the plain multi-CTA path.
 *   d_offsets: device int64 array of num_segments + 1 non-decreasing entries in [0, n]
 *   n        : number of keys (offsets[num_segments] at most)
 *   d_vals   : NULL with value_bytes 0, else the payload array
 * Offsets outside [0, n] or decreasing give PDQ_ERR_ARG (detected on the device).
 * A bounded wait that expires gives PDQ_ERR_TIMEOUT; the arrays then still hold a permutation
 * of the input pairs. */
int pdq_sort_segmented(void* d_keys, void* d_vals, int value_bytes, const int64_t* d_offsets,
                       int64_t num_segments, int64_t n, pdq_dtype key_dtype, void* d_ws, size_t ws_bytes,
                       void* cuda_stream, const pdq_tuning* tuning, pdq_stats* stats);

/* Learned-CDF proposal (float32 keys only, no payload).  A 1% sample of the keys is sorted and a
 * monotone model F(x) = sum_j a_j sat(w_j (x - t_j)) (16 hidden units, a_j > 0, w_j > 0; a 2-layer
 * MLP) is trained on it on the device by Adam on the squared error to the sample's empirical CDF.
 * The model then maps every key straight to one of 4096 buckets (min(4095, trunc(4096 F(x))),
 * NaNs by sign to the first or last bucket) in place of the first sampled-splitter level; every
 * bucket larger than the base capacity is re-partitioned exactly by the splitter levels
 * (stats.learned_overflow counts them).  The result is bit-identical to pdq_sort_keys.
 *   d_ws: workspace of at least pdq_workspace_bytes_learned(n) bytes.  Other arguments as
 *   pdq_sort_keys. */
int pdq_sort_keys_learned(void* d_keys, int64_t n, pdq_dtype key_dtype, void* d_ws, size_t ws_bytes,
                          void* cuda_stream, const pdq_tuning* tuning, pdq_stats* stats);
size_t pdq_workspace_bytes_learned(int64_t n);

/* Autotuner.  Picks, for the shape of one call, the bucket count per distribution level
 * (log2_buckets), the shared-memory base-case size (base_capacity; on the segmented path the
 * persistent CTA size seg_block, which fixes the size up to which a segment is sorted in shared
 * memory) by timing a fixed candidate grid on a scratch copy of the caller's input with CUDA
 * events, and records the fastest for the call's shape class: (plain or segmented, key type,
 * value_bytes, ceil(log2 n), ceil(log2 num_segments)).  Later pdq_sort_keys / pdq_sort_pairs /
 * pdq_sort_segmented / pdq_sort_host calls of that class that pass tuning = NULL use the recorded
 * tuning (an explicit tuning always wins).  The table is per process and lives until exit or
 * pdq_autotune_reset().
 *   d_keys, d_vals, value_bytes, d_offsets, num_segments (0 = plain path), n, key_dtype: the input
 *                as it would be passed to the sort; it is only read (never modified).
 *   d_scratch  : device memory of scratch_bytes >= pdq_autotune_scratch_bytes(...) bytes, 256-byte
 *                aligned (a copy of the keys and values plus a sort workspace).
 *   best       : nullable; receives the chosen tuning.  best_ms: nullable; its time in ms.
 * The call synchronises cuda_stream after every candidate; it takes a few dozen sorts' time.
 * Errors as for the sorts; on error nothing is recorded. */
size_t pdq_autotune_scratch_bytes(int64_t n, int64_t num_segments, pdq_dtype key_dtype, int value_bytes);
int pdq_autotune(const void* d_keys, const void* d_vals, int value_bytes, const int64_t* d_offsets,
                 int64_t num_segments, int64_t n, pdq_dtype key_dtype, void* d_scratch, size_t scratch_bytes,
                 void* cuda_stream, pdq_tuning* best, float* best_ms);
/* 1 and *out = the recorded tuning if pdq_autotune recorded one for this shape class, else 0. */
int pdq_autotune_lookup(int64_t n, int64_t num_segments, pdq_dtype key_dtype, int value_bytes, pdq_tuning* out);
/* Forget every recorded tuning. */
void pdq_autotune_reset(void);

/* Test probes of the learned model (parity of the hand-written forward/backward with a CPU
 * reference).  theta = [alpha(16), omega(16), c(16)]: a = softmax(alpha), w = exp(omega),
 * F(x) = sum_j a_j sat(w_j ((x - mu) / sigma - c_j)).
 * pdq_learned_loss_grad: h_out[0..48) = sum over points of d/dtheta of 0.5 (F(x_i) - t_i)^2,
 *   h_out[48] = sum of 0.5 (F(x_i) - t_i)^2; d_ws: >= 512 bytes of device scratch.
 * pdq_learned_train: trains on the sorted sample d_xs[0..m) (targets (i + 0.5) / m) for `steps`
 *   Adam steps of `batch` points; returns theta, [mu, sigma, first loss, last loss] and the
 *   folded model's w, t, a (3 x 16 floats: h_j = sat(w_j (x - t_j))); d_ws: >= 4096 bytes of
 *   device scratch, 256-byte aligned.  The training runs as one cooperative launch of one CTA
 *   per SM whose grid barriers are bounded (1 s): PDQ_ERR_TIMEOUT if one gives up. */
int pdq_learned_loss_grad(const float* d_x, const float* d_targets, int64_t m, const float* h_theta,
                          float mu, float sigma, float* h_out, void* d_ws, void* cuda_stream);
int pdq_learned_train(const float* d_xs, int64_t m, int steps, int batch, float lr, void* d_ws,
                      float* h_theta, float* h_norm_loss, float* h_wba, void* cuda_stream);

/* Host-buffer form of pdq_sort_keys / pdq_sort_pairs: copies h_keys (and h_vals when
 * value_bytes > 0) into the caller's device buffers d_keys / d_vals, sorts them there and copies
 * the result back into the host arrays, ordered on cuda_stream; returns after every copy has
 * finished.  For 2^26 keys and more the result goes back range by range: the last round's base
 * sorts run in position-ordered groups, and each group's range is copied to the host (on a
 * library-owned copy stream, ordered by events) while the later groups sort.  Host arrays should
 * be page-locked for full copy speed; they must not be touched until the call returns. */
int pdq_sort_host(void* h_keys, void* h_vals, int value_bytes, int64_t n, pdq_dtype key_dtype,
                  void* d_keys, void* d_vals, void* d_ws, size_t ws_bytes, void* cuda_stream,
                  const pdq_tuning* tuning, pdq_stats* stats);

/* Keys-only sort that allocates nothing, for callers that cannot call cudaMalloc (code whose
 * device memory is owned by a framework's allocator, fixed-budget plug-ins, latency-sensitive
 * loops where cudaMalloc/cudaFree would synchronise the device).  The paper has no counterpart:
 * this is a memory-ownership variant of pdq_sort_keys.  Its scratch is one file-scope device
 * array of 64 MiB per GPU, held until the process exits.  It takes at most 2^20 keys of any key
 * type; larger n returns PDQ_ERR_ARG with the limit in the message.  Every call looks up the
 * array's device address on the current device (cudaGetSymbolAddress, checked); the first call
 * on a device loads the module there, so make it before any stream capture.  All calls on a
 * device share the array, which keeps the last call's contents (the sort re-initialises every
 * counter and list length it reads): calls that overlap on the GPU race and must not be issued.
 * d_keys, n, key_dtype, cuda_stream, stats: as pdq_sort_keys. */
int pdq_sort_keys_noalloc(void* d_keys, int64_t n, pdq_dtype key_dtype, void* cuda_stream,
                          pdq_stats* stats);

/* Reverse n elements of elem_bytes (4 or 8) in place on the device (the descending-input exit
 * of Sec. 5.2, exposed for testing). */
int pdq_reverse(void* d_data, int64_t n, int elem_bytes, void* cuda_stream);

/* Message for the last error returned on this host thread ("" if none). */
const char* pdq_last_error(void);

/* Number of kernels this library has launched in this process (all threads). */
int64_t pdq_launch_count(void);

/* Per-kernel device time, for measurement: when enabled, each kernel launch of the library is
 * bracketed by CUDA events on its stream and its time is accumulated per kernel name. */
void pdq_profile_enable(int on);
/* Copies up to cap entries: names (each up to 63 chars + NUL, 64 bytes per entry), total
 * milliseconds, launch counts and the kernels' algorithmic bytes.  Synchronises the device.
 * Returns the number of kernel names recorded. */
int pdq_profile_read(char* names, double* total_ms, int64_t* launches, double* bytes, int cap);
void pdq_profile_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* PDQ_H_ */
