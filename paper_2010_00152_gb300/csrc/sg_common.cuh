// sg_common.cuh -- shared device definitions of the grouping path.
//
// Row formats (Sec. 3.3: the row format inside runs may differ from input and
// output rows):
//   raw rows    key + the payload columns the aggregates read;
//   state rows  key + one int64 partial aggregate per output aggregate.
// A FoldDesc says how to derive every state column from a source row: from a
// source column (or the constant 1 for count(*) of raw rows) combined with
// SUM, MIN or MAX ("row-plus-row accumulation", Sec. 6.1).
#pragma once
#include <cstdint>
#include <cuda/atomic>

namespace sg {

constexpr int kMaxKeyCols = 8;
constexpr int kMaxCols = 32;

enum : int8_t { OP_SUM = 0, OP_MIN = 1, OP_MAX = 2 };

// Error codes written to the device error word (host maps them to statuses).
enum : int { ERR_NONE = 0, ERR_TIMEOUT = 1, ERR_CAPACITY = 2, ERR_INTERNAL = 3 };

// ---------------------------------------------------------------------------
// Keys.  Normalized key (Sec. 2.4): unsigned key columns concatenated with
// column 0 most significant, right-aligned in a uint64.
// ---------------------------------------------------------------------------
struct KeyCols {
  int n_cols;
  int bytes[kMaxKeyCols];
  int shift[kMaxKeyCols];        // bits below column c in the normalized key
  const void* cols[kMaxKeyCols];
};

struct KeyOut {
  int n_cols;
  int bytes[kMaxKeyCols];
  int shift[kMaxKeyCols];
  void* cols[kMaxKeyCols];
};

__device__ __forceinline__ uint64_t load_col(const void* p, int bytes, int64_t i) {
  switch (bytes) {
    case 1: return __ldg(reinterpret_cast<const uint8_t*>(p) + i);
    case 2: return __ldg(reinterpret_cast<const uint16_t*>(p) + i);
    case 4: return __ldg(reinterpret_cast<const uint32_t*>(p) + i);
    default: return __ldg(reinterpret_cast<const unsigned long long*>(p) + i);
  }
}

__device__ __forceinline__ uint64_t load_key(const KeyCols& k, int64_t i) {
  if (k.n_cols == 1) return load_col(k.cols[0], k.bytes[0], i);
  uint64_t v = 0;
  for (int c = 0; c < k.n_cols; ++c) v |= load_col(k.cols[c], k.bytes[c], i) << k.shift[c];
  return v;
}

__device__ __forceinline__ void store_key(const KeyOut& k, int64_t j, uint64_t key) {
  for (int c = 0; c < k.n_cols; ++c) {
    uint64_t v = k.shift[c] >= 64 ? 0 : (key >> k.shift[c]);
    switch (k.bytes[c]) {
      case 1: reinterpret_cast<uint8_t*>(k.cols[c])[j] = (uint8_t)v; break;
      case 2: reinterpret_cast<uint16_t*>(k.cols[c])[j] = (uint16_t)v; break;
      case 4: reinterpret_cast<uint32_t*>(k.cols[c])[j] = (uint32_t)v; break;
      default: reinterpret_cast<unsigned long long*>(k.cols[c])[j] = v; break;
    }
  }
}

// ---------------------------------------------------------------------------
// Row sources.
// ---------------------------------------------------------------------------
enum : int { SRC_RAW = 0, SRC_SOA = 1, SRC_AOS = 2 };

struct RowSrc {
  int kind;
  int ncols;                        // columns carried (payload or state)
  int64_t offset;                   // added to every row index
  unsigned long long key_or;        // SRC_RAW: OR-ed into every key (instance id of a batch)
  KeyCols key;                          // SRC_RAW
  const unsigned long long* keys;       // SRC_SOA
  const long long* cols[kMaxCols];      // SRC_RAW payload / SRC_SOA state columns
  const long long* aos;                 // SRC_AOS: rows of (1 + ncols) words
};

__device__ __forceinline__ uint64_t src_key(const RowSrc& s, int64_t i) {
  int64_t r = s.offset + i;
  if (s.kind == SRC_AOS) return (uint64_t)s.aos[r * (1 + s.ncols)];
  if (s.kind == SRC_SOA) return __ldg(s.keys + r);
  return load_key(s.key, r) | s.key_or;
}

__device__ __forceinline__ long long src_col(const RowSrc& s, int c, int64_t i) {
  int64_t r = s.offset + i;
  if (s.kind == SRC_AOS) return s.aos[r * (1 + s.ncols) + 1 + c];
  return __ldg(s.cols[c] + r);
}

// 8-byte asynchronous copy, global to shared (completion: cp_async_wait;
// the copied words are visible to the issuing thread after it, to the
// others after a barrier).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Whether a source's keys are one column of 8-byte words (copied as is).
__host__ __device__ inline bool src_keys_direct(const RowSrc& s) {
  return s.kind == SRC_SOA || s.kind == SRC_AOS ||
         (s.kind == SRC_RAW && s.key.n_cols == 1 && s.key.bytes[0] == 8 && s.key_or == 0);
}

// Address of row i's key for such a source.
__device__ __forceinline__ const unsigned long long* src_key_ptr(const RowSrc& s, int64_t i) {
  const int64_t r = s.offset + i;
  if (s.kind == SRC_AOS) return reinterpret_cast<const unsigned long long*>(s.aos + r * (1 + s.ncols));
  if (s.kind == SRC_SOA) return s.keys + r;
  return reinterpret_cast<const unsigned long long*>(s.key.cols[0]) + r;
}

struct FoldDesc {
  int n_state;
  int8_t src[kMaxCols];   // source column of state column s, -1 = constant 1
  int8_t op[kMaxCols];    // OP_SUM / OP_MIN / OP_MAX
};

__device__ __forceinline__ int64_t op_identity(int op) {
  return op == OP_SUM ? 0 : (op == OP_MIN ? INT64_MAX : INT64_MIN);
}

__device__ __forceinline__ int64_t op_combine(int op, int64_t a, int64_t b) {
  if (op == OP_SUM) return (int64_t)((unsigned long long)a + (unsigned long long)b);
  if (op == OP_MIN) return b < a ? b : a;
  return b > a ? b : a;
}

// ---------------------------------------------------------------------------
// Partitioning digit.  fine(k) = clamp((k - base) >> fshift, 0, 2^fbits - 1)
// is monotone in k, so buckets of equal fine digit are key ranges in key
// order; the coarse digit is fine >> ebits.  Keys below base go to bucket 0,
// keys above the sampled range to the last bucket.
// ---------------------------------------------------------------------------
// One segment of a segmented digit: the keys whose bits above seg_shift
// equal the segment's index (one instance of a batched call) map to buckets
// base + ((low bits - kmin) >> shift), clamped to base + span.
struct SegEntry {
  unsigned long long kmin;
  unsigned base;
  unsigned info;  // shift in bits 0-7, span (buckets - 1) in bits 8-31
};

struct Digit {
  unsigned long long base;
  int fshift;
  int fbits;
  int ebits;
  int seg_shift;            // with seg: segment index = key >> seg_shift
  int seg_n;                // segments in the table
  const SegEntry* seg;      // null: one linear digit over the whole key range
  // Several batches partitioned in one launch (brows > 0): launch tile t is
  // tile t % btiles of batch t / btiles (rows [b * brows, (b + 1) * brows)),
  // and its buckets are b << bbits plus the digit, so every batch keeps
  // buckets of its own.
  long long brows;
  int btiles;
  int bbits;
};

// SEG: the digit has a segment table (kernels are compiled for either form,
// so the common linear digit carries no table lookup).
template <bool SEG = false>
__device__ __forceinline__ uint32_t fine_digit(const Digit& d, uint64_t k) {
  if (SEG) {
    uint64_t i = k >> d.seg_shift;
    i = i < (uint64_t)d.seg_n ? i : (uint64_t)d.seg_n - 1;
    const SegEntry e = d.seg[i];
    const uint64_t low = k & ((1ull << d.seg_shift) - 1);
    uint64_t x = low < e.kmin ? 0 : ((low - e.kmin) >> (e.info & 255u));
    const uint64_t span = e.info >> 8;
    x = x > span ? span : x;
    const uint64_t f = e.base + x, lim = (1ull << d.fbits) - 1;
    return (uint32_t)(f > lim ? lim : f);
  }
  if (d.fbits == 0 || k < d.base) return 0;
  uint64_t x = d.fshift >= 64 ? 0 : ((k - d.base) >> d.fshift);
  uint64_t lim = (1ull << d.fbits) - 1;
  return (uint32_t)(x > lim ? lim : x);
}

template <bool SEG = false>
__device__ __forceinline__ uint32_t coarse_digit(const Digit& d, uint64_t k) {
  return fine_digit<SEG>(d, k) >> d.ebits;
}

// ---------------------------------------------------------------------------
// Decoupled look-back across chunks processed in ticket order (the chained
// scan of Merrill and Garland, "Single-pass parallel prefix scan with
// decoupled look-back", 2016): each chunk publishes its row count as soon as
// it is known, then sums its predecessors' counts until it meets a published
// inclusive prefix.  Every wait is bounded; on timeout the chunk raises the
// error word and returns, and every other waiter sees the word and stops.
// ---------------------------------------------------------------------------
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

struct LookBack {
  unsigned long long* status;   // one word per chunk, zeroed before the launch
  unsigned int* ticket;         // zeroed before the launch
  const long long* base_in;     // exclusive prefix of chunk 0 (nullptr = 0)
  long long* total_out;         // inclusive prefix of the last chunk (nullptr = none)
  int* err;                     // device error word
  long long spin_limit;
  int n_chunks;
  int stall;                    // test hook: chunk 0 never publishes
};

__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
  a.store(v, cuda::memory_order_release);
}

__device__ __forceinline__ unsigned long long lb_load(unsigned long long* p) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
  return a.load(cuda::memory_order_acquire);
}

__device__ __forceinline__ int err_load(int* p) {
  cuda::atomic_ref<int, cuda::thread_scope_device> a(*p);
  return a.load(cuda::memory_order_relaxed);
}

__device__ __forceinline__ void err_raise(int* p, int code) {
  atomicCAS(p, 0, code);
}

// Publishes chunk `id`'s row count (lane 0 of the calling warp stores):
// chunk 0 its inclusive prefix (base + count), every other chunk its
// aggregate.  Returns chunk 0's base (0 for other chunks), read here once:
// base_in may be the same word as total_out, which the last chunk writes as
// soon as chunk 0's prefix is out.
__device__ __forceinline__ long long lookback_publish(const LookBack& lb, int id, long long count) {
  const long long b0 = (id == 0 && lb.base_in) ? *lb.base_in : 0;
  if ((threadIdx.x & 31) != 0) return b0;
  if (id == 0) {
    if (!lb.stall) lb_store(&lb.status[0], kFlagPre | (unsigned long long)(b0 + count));
  } else {
    lb_store(&lb.status[id], kFlagAgg | (unsigned long long)count);
  }
  return b0;
}

// Called by one full warp after lookback_publish (b0: what it returned).
// Returns the exclusive prefix of chunk `id` and publishes its inclusive
// prefix, or returns -1 after raising ERR_TIMEOUT (or seeing another error).
// Each round trip reads the status of up to 4 x 32 predecessors (windows of
// 32, nearest first) and folds windows in order while they are complete.
__device__ long long lookback_resolve(const LookBack& lb, int id, long long count, long long b0) {
  constexpr int NW = 4;
  const int lane = threadIdx.x & 31;
  long long excl = 0;
  if (id == 0) return b0;
  int j = id - 1;  // highest predecessor not yet folded into excl
  long long spins = 0;
  while (true) {
    unsigned long long sv[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      const int p = j - 32 * q - lane;
      sv[q] = p >= 0 ? lb_load(&lb.status[p]) : kFlagPre;
    }
    bool done = false, moved = false, past = false;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      const int p = j - lane;  // the window read for round q (j moved by whole windows so far)
      const unsigned long long s = sv[q];
      const bool ready = (s >> 62) != 0;
      const unsigned all_ready = __ballot_sync(0xffffffffu, ready);
      // lanes 0..(first not-ready - 1) are usable only if contiguous from lane 0
      const unsigned not_ready = ~all_ready;
      const int usable = not_ready ? __ffs(not_ready) - 1 : 32;
      const unsigned pre = __ballot_sync(0xffffffffu, ready && ((s >> 62) == 2) && lane < usable);
      if (pre) {
        const int stop = __ffs(pre) - 1;  // nearest inclusive prefix
        long long v = (lane <= stop) ? (long long)(s & kValMask) : 0;
        if (p < 0) v = 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        excl += __shfl_sync(0xffffffffu, v, 0);
        done = true;
        break;
      }
      if (usable == 0) break;
      long long v = (lane < usable && p >= 0) ? (long long)(s & kValMask) : 0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      excl += __shfl_sync(0xffffffffu, v, 0);
      j -= usable;
      moved = true;
      if (j < 0) {  // walked past chunk 0 without a prefix: chunk 0 always publishes one
        past = true;
        break;
      }
      if (usable < 32) break;  // the next windows were read for other positions
    }
    if (done) break;
    if (past) {
      excl += lb.base_in ? *lb.base_in : 0;
      break;
    }
    if (moved) continue;
    // warp-uniform exit: the error word is read by lane 0 only
    int e = __shfl_sync(0xffffffffu, lane == 0 ? err_load(lb.err) : 0, 0);
    if (++spins > lb.spin_limit || e) {
      if (lane == 0) err_raise(lb.err, ERR_TIMEOUT);
      return -1;
    }
    __nanosleep(spins < 4 ? 64u : 512u);  // back off once a wait is not short
  }
  if (lane == 0) lb_store(&lb.status[id], kFlagPre | (unsigned long long)(excl + count));
  return excl;
}

// Called by one full warp.  Publishes `count` for chunk `id` and returns the
// exclusive prefix, or -1 after raising ERR_TIMEOUT (or seeing another error).
__device__ __forceinline__ long long lookback_warp(const LookBack& lb, int id, long long count) {
  const long long b0 = lookback_publish(lb, id, count);
  return lookback_resolve(lb, id, count, b0);
}

}  // namespace sg
