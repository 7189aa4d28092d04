// sgagg.cu -- host side of the grouping path: C ABI, planner, run store.
//
// Pipeline of one sgagg_aggregate call (Sec. 3, Sec. 4, Sec. 6.1):
//   probe      sample keys once: key range for the partitioning digit and an
//              estimate of the duplicate rate (decides tile pre-aggregation);
//   per batch  (read-sort-write cycle of M rows) run generation with early
//              aggregation: optional tile pre-fold, partition by key range,
//              sort+fold every chunk -> one sorted run of distinct keys, with
//              per-fine-bucket offsets (the run's sparse index);
//   merge      one wide merge over all runs: merge tiles are key ranges
//              (groups of fine buckets) whose rows from every run fit one
//              CTA; each tile folds equal keys across runs and writes the
//              final rows in key order.
// With a single batch the run is written straight to the output (no spill,
// the in-memory case of Sec. 5.2.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sgagg.h"
#include "sg_part.cuh"
#include "sg_merge.cuh"
#include "sg_lowcard.cuh"
#include "sg_hybrid.cuh"

using namespace sg;

namespace {

// Planner: a chunk starts every kChunkTarget rows of buckets of at most
// kBigBucket rows, so such chunks stay below kChunkTarget + kBigBucket =
// kTileCap rows; a bigger bucket is a chunk of its own, solved apart when it
// holds more than kTileCap rows.  Coarse buckets average
// kBucketRows rows (32 standard deviations below kBigBucket for uniform keys).
constexpr long long kBigBucket = 2048;
constexpr long long kChunkTarget = kTileCap - kBigBucket;
constexpr long long kBucketRows = 1024;
constexpr int kClasses = SGAGG_K_STREAM + 1;
// The streaming fold of few keys (k_lowcard) is taken for one batch of at
// least this many rows.
constexpr long long kLowCardMinRows = 1ll << 16;
// Merge tiles (k_merge): at most kMergeTile rows over all runs; fine buckets
// of the runs' sparse indexes average at most kMergeFineRows rows, so tiles
// are packed close to the cap.
constexpr long long kMergeFineRows = 256;
// Runs are allocated with this many bytes past their last row: a merge
// tile's bulk copy of a slice may read one row past the slice.
constexpr size_t kRunSlack = 16;
constexpr int kMaxDepth = 70;
constexpr long long kMaxBatch = 1ll << 30;
constexpr int kSample = 16384;
constexpr long long kBatchGroupRows = 1ll << 25;   // rows per group of a batched call (default)

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  size_t used = 0;   // bytes requested by the current call
  int gen = -1;      // call that last requested this buffer
  bool arena = false;  // run storage: counted as run bytes, not scratch
};

struct Run {
  long long start;   // absolute row in its arena (host copy, filled after sync)
  long long rows;
  int host;          // 1: pinned host arena
};

// A sorted run of state rows as the merge sees it (device-accessible pointers).
struct RunRef {
  const long long* keys;
  const long long* cols[sg::kMaxCols];
  long long* offs;   // nf + 1 fine-bucket offsets (absolute rows of its arrays)
  long long rows;
  int host = 0;      // arrays in pinned host memory (no bulk copies from them)
};

}  // namespace

// A host-buffer call (sgagg_aggregate_host): inputs are copied batch by
// batch on a copy stream, batch b + 1 while batch b is grouped; the final
// merge runs in parts and each part's output is copied back while the next
// parts merge.
constexpr int kMergeParts = 8;
struct HostIO {
  cudaStream_t copy = nullptr;
  int nk = 0;
  const void* hkeys[kMaxKeyCols];
  int kb[kMaxKeyCols];
  void* dkeys[kMaxKeyCols];
  int np = 0;
  const int64_t* const* hpay = nullptr;  // host payload columns
  const bool* used = nullptr;            // payload columns the aggregates read
  int64_t* const* dpay = nullptr;        // their device copies
  void* hout_keys[kMaxKeyCols];
  void* dout_keys[kMaxKeyCols];
  int S = 0;
  int64_t* const* hout_aggs = nullptr;
  int64_t* const* dout_aggs = nullptr;
  long long capacity = 0;
  long long copied_out = 0;  // output rows whose copy back is enqueued
};

struct sgagg_ctx {
  long long M = 1;
  std::vector<unsigned long long> sset_key;  // host hash set of a key sample
  std::vector<unsigned> sset_stamp;          // slot in use when == sset_gen
  unsigned sset_gen = 0;
  int prefold_opt = -1;
  long long arena_cap = -1;
  int radix_bits = 0;
  long long spin_limit = 1ll << 26;
  int fanin_cap = 0;
  int fault_alloc = 0;
  int alloc_count = 0;
  int timing = 0;
  long long timing_mask = -1;    // SGAGG_OPT_TIMING_CLASSES
  bool timer_open = false;       // kbegin recorded the start event of the open launch
  int test_stall = 0;
  int policy = 0;                // 0: a run per batch, 1: absorbing index
  long long absorb_batch = 0;    // rows per batch of the absorbing policy (0: auto)
  int lowcard = -1;              // streaming fold of few keys: -1 auto, 0 off
  int merge_threads = 0;         // threads of a merge CTA (128, 256, 512; 0 = default)
  int merge_copy = 0;            // merge staging: 0 bulk copies by the workers, 1 16-byte cp.async,
                                 // 2 bulk copies by the control warp
  int prefold_bins = 0;          // tile pre-aggregation binning: 0 key range, 1 hash of the key
  int one_pass = 1;              // small batches: every run in one pass per step (0: a batch at a time)
  int part_levels = 0;           // partition levels: 0 auto (two above 2^7 buckets), 1 always one
  long long batch_group_rows = kBatchGroupRows;  // batched call: rows of the instances grouped at once
  long long prefold_rows = kTileCap;  // rows per pre-aggregation tile of a batched call
  int hybrid_fanin = 10;         // hybrid run generation (policy 2): F
  int hybrid_f = -1;             // f (-1: from the estimated output size)
  bool hybrid_last_given = false;
  unsigned long long hybrid_last = 0;   // last key of the resident range, when given
  std::vector<long long> run_sizes;     // rows of each run of the last call, in the order written
  DevBuf hsplit_keys[2];               // hybrid: resident / spilled rows (SoA)
  std::vector<DevBuf> hsplit_cols[2];
  std::string err;
  // per-launch event pairs (SGAGG_OPT_TIMING)
  struct KT { cudaEvent_t a = nullptr, b = nullptr; int cls = 0; };
  std::vector<KT> timers;
  int ntimers = 0;
  bool timers_read = true;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int device = -1;

  // workspace (grown on demand, freed by destroy)
  // per recursion depth (fixed arrays: pointers stay valid for accounting)
  DevBuf scatter[kMaxDepth + 1];  // rows of 1 + ncols words
  DevBuf thist[kMaxDepth + 1], btot[kMaxDepth + 1], bstart[kMaxDepth + 1];
  DevBuf chunks[kMaxDepth + 1], biglist[kMaxDepth + 1];
  DevBuf copykeys[kMaxDepth + 1];  // solved big buckets (SoA)
  // two-level partition: level-1 output (SoA), tables
  DevBuf akeys[kMaxDepth + 1], acolptr[kMaxDepth + 1], thist1[kMaxDepth + 1], btot1[kMaxDepth + 1];
  DevBuf bstart1[kMaxDepth + 1], tiles2[kMaxDepth + 1], tfirst[kMaxDepth + 1], thist2[kMaxDepth + 1];
  std::vector<DevBuf> acols[kMaxDepth + 1];
  std::vector<DevBuf> copycols[kMaxDepth + 1];
  DevBuf pf[2];                  // pre-fold ping-pong: keys
  std::vector<DevBuf> pfcols[2];
  DevBuf status;                 // look-back status words + ticket
  DevBuf small;                  // error word, counters, plan info, min/max
  DevBuf sample;
  DevBuf arena_keys;
  std::vector<DevBuf> arena_cols;
  DevBuf offs;                   // runs x (nf + 1)
  DevBuf runptrs;
  DevBuf fsizes;
  DevBuf gather_keys;
  std::vector<DevBuf> gather_cols;
  DevBuf gather_ptrs;
  DevBuf runstarts;              // batches + 1 device scalars
  DevBuf binst, bchunks, bkeys, bout_keys;   // batched call: instances, tiles, partial rows, output
  DevBuf bseg, brange, bstartb;              // batched call: segmented digit, key ranges, row starts
  DevBuf bdirect;                            // batched call: chunks of the one-chunk instances
  std::vector<DevBuf> bcols, bout_cols;
  DevBuf ab_keys[3], ab_offs[3], ab_tmp;   // absorbing policy: index, batch, merged index
  DevBuf dk_keys, rg_heads;                // count(distinct): (g, u) rows, regroup block heads
  DevBuf plan_tmp;                         // chunk planner: per-block sums and starts
  DevBuf lc_part;                          // streaming fold of few keys: per-block partials
  DevBuf tslo;                             // wide merge: every tile's slice start in every run
  DevBuf tcount, tbase;                    // wide merge: every tile's distinct keys, output base
  std::vector<DevBuf> dk_cols;
  std::vector<DevBuf> ab_cols[3];
  DevBuf marena_keys;            // runs written by preliminary merges
  std::vector<DevBuf> marena_cols;
  DevBuf moffs;
  // host arena (pinned, mapped)
  void* harena_keys = nullptr;
  std::vector<void*> harena_cols;
  size_t harena_rows = 0;
  // host-side input staging for sgagg_aggregate_host
  DevBuf in_keys[kMaxKeyCols];
  std::vector<DevBuf> in_pay;
  DevBuf out_keys[kMaxKeyCols];
  std::vector<DevBuf> out_cols;

  // pinned host scratch for small read-backs
  void* hsmall = nullptr;
  // host-buffer calls: the copy stream and its events
  HostIO* hio = nullptr;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> io_events;       // input batches staged
  cudaEvent_t part_events[kMergeParts] = {};  // parts of the final merge done

  // buffers requested by the current call (scratch accounting)
  int gen = 0;
  std::vector<DevBuf*> touched;
  bool top_prefold = false;
  int key_bytes = 0;
  int spec_aggs = 0;

  // last call
  bool have_call = false;
  long long last_rows = 0;
  sgagg_stats_t st{};
  long long scratch_bytes = 0;
  int pending_err = 0;
};

namespace {

// small device block layout
struct Small {
  int err;
  int pad;
  unsigned long long mm[2];
  PlanInfo info;
  long long total;              // total_out of the final sort+fold
  long long pftot;              // total_out of a pre-fold pass
  long long dsum;               // rows of the one-chunk instances of a batched call
  int lc_over;                  // streaming fold of few keys: a key outside the sample
  int lc_pad;
  long long part_tot[kMergeParts];  // final merge in parts: output end of every part
  long long hy_rows;            // hybrid: resident rows (split total)
  long long hy_keys;            // hybrid: resident groups = output base of the merged runs
  long long dtot[kMaxDepth + 2];  // base/total of the sub-solves under depth d
};

struct HostSmall {
  PlanInfo info;
  int err;
  int pad;
  unsigned long long mm[2];
  long long v[8];
  unsigned long long sample[kSample];
  Chunk ch[4];
  long long part_end[kMergeParts];   // final merge: output end of every part
};

sgagg_status fail(sgagg_t h, sgagg_status s, const char* fmt, const char* a = "") {
  char buf[512];
  snprintf(buf, sizeof buf, fmt, a);
  if (h) h->err = buf;
  return s;
}

#define CU(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      return fail(h, e_ == cudaErrorMemoryAllocation ? SGAGG_ENOMEM : SGAGG_ECUDA, \
                  "%s", cudaGetErrorString(e_));                              \
    }                                                                         \
  } while (0)

#define TRY(x)                          \
  do {                                  \
    sgagg_status s_ = (x);              \
    if (s_ != SGAGG_OK) return s_;      \
  } while (0)

// Partition kernels come in two forms, with and without a segmented digit;
// the staged scatter also in two, copying by cp.async or through registers.
#define PART_CFG(...) __VA_ARGS__
#define PART_LAUNCH(kern, cfg, args)                             \
  do {                                                           \
    if (dig.seg) kern<true><<<PART_CFG cfg>>>(PART_CFG args);    \
    else kern<false><<<PART_CFG cfg>>>(PART_CFG args);           \
  } while (0)
#define HIST_LAUNCH(kern, srcv, cfg, args)                                                        \
  do {                                                                                            \
    const bool dir_ = staged_direct(srcv);                                                        \
    if (dig.seg) {                                                                                \
      if (dir_) kern<true, true><<<PART_CFG cfg>>>(PART_CFG args);                                 \
      else kern<true, false><<<PART_CFG cfg>>>(PART_CFG args);                                     \
    } else {                                                                                      \
      if (dir_) kern<false, true><<<PART_CFG cfg>>>(PART_CFG args);                                \
      else kern<false, false><<<PART_CFG cfg>>>(PART_CFG args);                                    \
    }                                                                                             \
  } while (0)
#define STAGED_LAUNCH(srcv, cfg, args)                                                            \
  do {                                                                                            \
    const bool dir_ = staged_direct(srcv);                                                        \
    if (dig.seg) {                                                                                \
      if (dir_) k_scatter_staged<true, true><<<PART_CFG cfg>>>(PART_CFG args);                     \
      else k_scatter_staged<true, false><<<PART_CFG cfg>>>(PART_CFG args);                         \
    } else {                                                                                      \
      if (dir_) k_scatter_staged<false, true><<<PART_CFG cfg>>>(PART_CFG args);                    \
      else k_scatter_staged<false, false><<<PART_CFG cfg>>>(PART_CFG args);                        \
    }                                                                                             \
  } while (0)

// Kernel-class bookkeeping: launches, compulsory bytes, optional event time.
void kbegin(sgagg_t h, int cls) {
  ++h->st.class_launches[cls];
  ++h->st.kernel_launches;
  h->timer_open = h->timing && ((h->timing_mask >> cls) & 1);
  if (!h->timer_open) return;
  if (h->ntimers == (int)h->timers.size()) {
    sgagg_ctx::KT t;
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
    h->timers.push_back(t);
  }
  auto& t = h->timers[h->ntimers];
  t.cls = cls;
  cudaEventRecord(t.a, h->stream);
}

void kend(sgagg_t h) {
  if (!h->timer_open) return;
  h->timer_open = false;
  cudaEventRecord(h->timers[h->ntimers].b, h->stream);
  ++h->ntimers;
  h->timers_read = false;
}

void kbytes(sgagg_t h, int cls, long long bytes) { h->st.class_bytes[cls] += bytes; }

long long src_row_bytes(const RowSrc& s) {
  if (s.kind == SRC_RAW) {
    long long kb = 0;
    for (int c = 0; c < s.key.n_cols; ++c) kb += s.key.bytes[c];
    return kb + 8ll * s.ncols;
  }
  return 8ll * (1 + s.ncols);
}

sgagg_status grow(sgagg_t h, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.gen != h->gen) {
    b.gen = h->gen;
    b.used = 0;
    h->touched.push_back(&b);
  }
  b.used = std::max(b.used, bytes);
  if (b.cap >= bytes) return SGAGG_OK;
  ++h->alloc_count;
  if (h->fault_alloc > 0 && h->alloc_count == h->fault_alloc)
    return fail(h, SGAGG_ENOMEM, "injected allocation failure");
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(h, SGAGG_ENOMEM, "device allocation of %s bytes failed",
                std::to_string(want).c_str());
  }
  b.cap = want;
  return SGAGG_OK;
}

template <class T>
T* P(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

Small* dsmall(sgagg_t h) { return reinterpret_cast<Small*>(h->small.p); }
HostSmall* hsmall(sgagg_t h) { return reinterpret_cast<HostSmall*>(h->hsmall); }

// ---- host-buffer calls: staged copies (see HostIO) ----
sgagg_status io_event(sgagg_t h, size_t i, cudaEvent_t* e) {
  while (h->io_events.size() <= i) {
    cudaEvent_t x;
    CU(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    h->io_events.push_back(x);
  }
  *e = h->io_events[i];
  return SGAGG_OK;
}

// Enqueue the copies of input rows [lo, hi) on the copy stream; event i
// fires when they are done.
sgagg_status stage_rows(sgagg_t h, long long lo, long long hi, size_t i) {
  HostIO& io = *h->hio;
  if (hi > lo) {
    for (int c = 0; c < io.nk; ++c)
      CU(cudaMemcpyAsync(static_cast<char*>(io.dkeys[c]) + lo * io.kb[c],
                         static_cast<const char*>(io.hkeys[c]) + lo * io.kb[c], (size_t)(hi - lo) * io.kb[c],
                         cudaMemcpyHostToDevice, io.copy));
    for (int c = 0; c < io.np; ++c)
      if (io.used[c])
        CU(cudaMemcpyAsync(io.dpay[c] + lo, io.hpay[c] + lo, (size_t)(hi - lo) * 8, cudaMemcpyHostToDevice, io.copy));
  }
  cudaEvent_t e;
  TRY(io_event(h, i, &e));
  CU(cudaEventRecord(e, io.copy));
  return SGAGG_OK;
}

// The compute stream waits for the copies of event i.
sgagg_status wait_rows(sgagg_t h, size_t i) {
  CU(cudaStreamWaitEvent(h->stream, h->io_events[i], 0));
  return SGAGG_OK;
}

// Enqueue the copy back of output rows [lo, hi) on the copy stream, after
// event `after` (recorded on the compute stream).
sgagg_status unstage_rows(sgagg_t h, long long lo, long long hi, cudaEvent_t after) {
  HostIO& io = *h->hio;
  hi = std::min(hi, io.capacity);
  if (hi <= lo) return SGAGG_OK;
  CU(cudaStreamWaitEvent(io.copy, after, 0));
  for (int c = 0; c < io.nk; ++c)
    CU(cudaMemcpyAsync(static_cast<char*>(io.hout_keys[c]) + lo * io.kb[c],
                       static_cast<const char*>(io.dout_keys[c]) + lo * io.kb[c], (size_t)(hi - lo) * io.kb[c],
                       cudaMemcpyDeviceToHost, io.copy));
  for (int a = 0; a < io.S; ++a)
    CU(cudaMemcpyAsync(io.hout_aggs[a] + lo, io.dout_aggs[a] + lo, (size_t)(hi - lo) * 8, cudaMemcpyDeviceToHost,
                       io.copy));
  return SGAGG_OK;
}

// The planner's key sample taken from the host columns (the same rows the
// device probe reads), so that no input copy has to finish first.
void host_sample(const HostIO& io, const sg::KeyCols& kc, long long n, int count, unsigned long long* out) {
  for (int i = 0; i < count; ++i) {
    const long long r = (long long)((__int128)i * n / count);
    unsigned long long v = 0;
    for (int c = 0; c < io.nk; ++c) {
      const char* p = static_cast<const char*>(io.hkeys[c]) + r * io.kb[c];
      unsigned long long x = 0;
      switch (io.kb[c]) {
        case 1: x = *reinterpret_cast<const uint8_t*>(p); break;
        case 2: x = *reinterpret_cast<const uint16_t*>(p); break;
        case 4: x = *reinterpret_cast<const uint32_t*>(p); break;
        default: x = *reinterpret_cast<const unsigned long long*>(p); break;
      }
      v |= kc.n_cols == 1 ? x : (x << kc.shift[c]);
    }
    out[i] = v;
  }
}

int ilog2_ceil(long long x) {
  int b = 0;
  while ((1ll << b) < x) ++b;
  return b;
}

int bitlen(unsigned long long x) { return x ? 64 - __builtin_clzll(x) : 0; }

// Estimated distinct values D of a domain from `dist` distinct among `s`
// uniform draws (inverse of D (1 - exp(-s/D))), by bisection.
double estimate_domain(double s, double dist) {
  if (dist >= s) return 1e18;
  double lo = dist, hi = 1e18;
  for (int it = 0; it < 200; ++it) {
    double mid = std::sqrt(lo * hi);
    double e = mid * (1.0 - std::exp(-s / mid));
    if (e < dist) lo = mid; else hi = mid;
  }
  return lo;
}

// The distinct keys of a sample, in place: v[0 .. return value) holds them
// in order of first appearance; *mn / *mx get the sample's minimum and
// maximum.  An open-addressed hash set (load factor <= 1/2, slots stamped
// with a generation so nothing is cleared between calls) keeps this linear
// in the sample: sorting 16,384 keys first measured ten times slower, and
// the host does this before the first launch of a call.
long long sample_distinct(sgagg_t h, unsigned long long* v, int n, unsigned long long* mn, unsigned long long* mx) {
  constexpr int kBits = 15;  // 2^15 slots for up to kSample keys
  static_assert(kSample <= (1 << (kBits - 1)), "sample set too small");
  if (h->sset_key.empty()) {
    h->sset_key.assign(1u << kBits, 0);
    h->sset_stamp.assign(1u << kBits, 0);
  }
  if (++h->sset_gen == 0) {
    std::fill(h->sset_stamp.begin(), h->sset_stamp.end(), 0u);
    h->sset_gen = 1;
  }
  unsigned long long* key = h->sset_key.data();
  unsigned* stamp = h->sset_stamp.data();
  const unsigned gen = h->sset_gen;
  unsigned long long lo = ~0ull, hi = 0;
  long long d = 0;
  for (int i = 0; i < n; ++i) {
    const unsigned long long k = v[i];
    lo = std::min(lo, k);
    hi = std::max(hi, k);
    // multiplicative hashing: the product's top bits depend on every key bit
    unsigned s = (unsigned)((k * 0x9E3779B97F4A7C15ull) >> (64 - kBits));
    bool seen = false;
    while (stamp[s] == gen) {
      if (key[s] == k) {
        seen = true;
        break;
      }
      s = (s + 1) & ((1u << kBits) - 1);
    }
    if (seen) continue;
    stamp[s] = gen;
    key[s] = k;
    v[d++] = k;
  }
  *mn = lo;
  *mx = hi;
  return d;
}

bool want_prefold(sgagg_t h, long long sample_n, long long distinct) {
  if (h->prefold_opt >= 0) return h->prefold_opt == 1;
  if (sample_n < 64) return false;
  double D = estimate_domain((double)sample_n, (double)distinct);
  double per_tile = D * (1.0 - std::exp(-(double)kTileCap / D));
  return per_tile * 2.0 <= (double)kTileCap;
}

// Kernel attributes belong to one device's context: each kind of setup
// keeps a bit per device index (set once the attributes are in place; two
// threads racing on a new device both set them, which is harmless).
struct DeviceOnce {
  std::atomic<unsigned long long> mask{0};
  bool need(int* dev) {
    if (cudaGetDevice(dev) != cudaSuccess) *dev = 0;
    return *dev >= 64 || !((mask.load(std::memory_order_acquire) >> *dev) & 1ull);
  }
  void done(int dev) {
    if (dev < 64) mask.fetch_or(1ull << dev, std::memory_order_release);
  }
};

template <int MODE, int KS>
void set_smem_attr() {
  static DeviceOnce once;
  int dev = 0;
  if (once.need(&dev)) {
    cudaFuncSetAttribute(k_sortfold<MODE, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSortSmemBytes);
    once.done(dev);
  }
}

// Launch the sort+fold kernel specialized for the number of aggregates.
template <int MODE, int KS>
void launch_ks(int grid, cudaStream_t st, const Chunk* dchunks, const RowSrc& src,
               const CopySrc& copy, const FoldDesc& fd, const OutSink& out, const LookBack& lb,
               long long tile_n, int tile_f_hi, const InstSet& is = InstSet{}) {
  set_smem_attr<MODE, KS>();
  k_sortfold<MODE, KS><<<grid, kThreads, kSortSmemBytes, st>>>(dchunks, src, copy, fd, out, lb, tile_n,
                                                              tile_f_hi, is);
}

constexpr int kMaxCoarseBits = 15;  // per-tile histogram / cursors: 2^15 x 4 B of shared memory

void set_part_attrs() {
  static DeviceOnce once;
  int dev = 0;
  if (once.need(&dev)) {
    cudaFuncSetAttribute(k_hist<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << kMaxCoarseBits) * 4);
    cudaFuncSetAttribute(k_hist<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << kMaxCoarseBits) * 4);
    cudaFuncSetAttribute(k_hist<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << kMaxCoarseBits) * 4);
    cudaFuncSetAttribute(k_hist<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << kMaxCoarseBits) * 4);
    cudaFuncSetAttribute(k_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << kMaxCoarseBits) * 4);
    cudaFuncSetAttribute(k_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (1 << kMaxCoarseBits) * 4);
    cudaFuncSetAttribute(k_scatter_staged<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)staged_smem_bytes(1 << kMaxCoarseBits > 1024 ? 1024 : 1 << kMaxCoarseBits, kStageCols));
    cudaFuncSetAttribute(k_scatter_staged<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)staged_smem_bytes(1 << kMaxCoarseBits > 1024 ? 1024 : 1 << kMaxCoarseBits, kStageCols));
    cudaFuncSetAttribute(k_scatter_staged<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)staged_smem_bytes(1 << kMaxCoarseBits > 1024 ? 1024 : 1 << kMaxCoarseBits, kStageCols));
    cudaFuncSetAttribute(k_hist2<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_hist2<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_scatter_staged<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)staged_smem_bytes(1 << kMaxCoarseBits > 1024 ? 1024 : 1 << kMaxCoarseBits, kStageCols));
    cudaFuncSetAttribute(k_hist2<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_hist2<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    once.done(dev);
  }
}

// Buckets of the first partitioning level: few enough that a staged sub-tile
// (kStage rows) leaves >= 32 rows per bucket, i.e. runs of >= 256 bytes per
// column, so no write leaves a partial sector behind.
constexpr int kLevel1Bits = 7;

// Everything a sort+fold launch writes into.
struct Sink {
  OutSink o;
  int n_state;
};

FoldDesc identity_fold(const FoldDesc& raw) {
  FoldDesc f = raw;
  for (int s = 0; s < raw.n_state; ++s) f.src[s] = (int8_t)s;
  return f;
}

// Launch the sort+fold kernel over n_chunks chunks.
template <int MODE>
sgagg_status launch_sortfold(sgagg_t h, int cls, const Chunk* dchunks, int n_chunks, long long tile_n,
                             const RowSrc& src, const CopySrc& copy,
                             const FoldDesc& fd, const OutSink& out, const long long* base_in,
                             long long* total_out, int tile_f_hi = 0, const InstSet& is = InstSet{}) {
  if (n_chunks <= 0) {
    // still publish the running total
    if (total_out) {
      if (base_in) CU(cudaMemcpyAsync(total_out, base_in, 8, cudaMemcpyDeviceToDevice, h->stream));
      else CU(cudaMemsetAsync(total_out, 0, 8, h->stream));
    }
    return SGAGG_OK;
  }
  TRY(grow(h, h->status, (size_t)(n_chunks + 2) * 8));
  CU(cudaMemsetAsync(h->status.p, 0, (size_t)(n_chunks + 2) * 8, h->stream));
  LookBack lb;
  lb.ticket = reinterpret_cast<unsigned int*>(P<unsigned long long>(h->status));
  lb.status = P<unsigned long long>(h->status) + 2;
  lb.base_in = reinterpret_cast<const long long*>(base_in);
  lb.total_out = reinterpret_cast<long long*>(total_out);
  lb.err = &dsmall(h)->err;
  lb.spin_limit = h->spin_limit;
  lb.n_chunks = n_chunks;
  lb.stall = h->test_stall == 1 ? 1 : 0;  // 2 waits for the next merge launch
  if (h->test_stall == 1) h->test_stall = 0;
  kbegin(h, cls);
  if (fd.n_state <= 2)
    launch_ks<MODE, 2>(n_chunks, h->stream, dchunks, src, copy, fd, out, lb, tile_n, tile_f_hi, is);
  else if (fd.n_state <= 4)
    launch_ks<MODE, 4>(n_chunks, h->stream, dchunks, src, copy, fd, out, lb, tile_n, tile_f_hi, is);
  else if (fd.n_state <= 8)
    launch_ks<MODE, 8>(n_chunks, h->stream, dchunks, src, copy, fd, out, lb, tile_n, tile_f_hi, is);
  else if (fd.n_state <= 16)
    launch_ks<MODE, 16>(n_chunks, h->stream, dchunks, src, copy, fd, out, lb, tile_n, tile_f_hi, is);
  else
    launch_ks<MODE, 32>(n_chunks, h->stream, dchunks, src, copy, fd, out, lb, tile_n, tile_f_hi, is);
  kend(h);
  CU(cudaGetLastError());
  return SGAGG_OK;
}

// Launch the wide-merge kernel over n_chunks merge tiles of at most
// kMergeTile rows.  bulk: every run array is device memory with a 16-byte
// aligned start and kRunSlack bytes past its rows (slices are bulk-copied).
sgagg_status launch_merge(sgagg_t h, const Chunk* dchunks, int n_chunks, const long long* tslo, const RunSet& runs,
                          bool bulk, const CopySrc& copy, const FoldDesc& fd, const OutSink& out,
                          const long long* base_in, long long* total_out) {
  if (n_chunks <= 0) {
    if (total_out) {
      if (base_in) CU(cudaMemcpyAsync(total_out, base_in, 8, cudaMemcpyDeviceToDevice, h->stream));
      else CU(cudaMemsetAsync(total_out, 0, 8, h->stream));
    }
    return SGAGG_OK;
  }
  // every tile's distinct keys (a count pass), their scan: the tiles' output bases
  const int sblocks = (n_chunks + kScanThreads - 1) / kScanThreads;
  TRY(grow(h, h->status, (size_t)(sblocks + 2) * 8));
  TRY(grow(h, h->tcount, (size_t)n_chunks * 8));
  TRY(grow(h, h->tbase, (size_t)n_chunks * 8));
  CU(cudaMemsetAsync(h->status.p, 0, (size_t)(sblocks + 2) * 8, h->stream));
  MergeArgs a{};
  a.lb.ticket = reinterpret_cast<unsigned int*>(P<unsigned long long>(h->status));
  a.lb.status = P<unsigned long long>(h->status) + 2;
  a.lb.base_in = reinterpret_cast<const long long*>(base_in);
  a.lb.total_out = reinterpret_cast<long long*>(total_out);
  a.lb.err = &dsmall(h)->err;
  a.lb.spin_limit = h->spin_limit;
  a.lb.n_chunks = sblocks;
  a.lb.stall = h->test_stall != 0 ? 1 : 0;
  h->test_stall = 0;
  kbegin(h, SGAGG_K_MERGE);
  k_merge_count<<<n_chunks, kCountThreads, 0, h->stream>>>(dchunks, tslo, runs, P<long long>(h->tcount),
                                                           &dsmall(h)->err);
  k_merge_scan<<<sblocks, kScanThreads, 0, h->stream>>>(P<long long>(h->tcount), n_chunks, P<long long>(h->tbase),
                                                        a.lb, out.capacity);
  kend(h);
  CU(cudaGetLastError());
  h->st.class_launches[SGAGG_K_MERGE] += 1;  // kbegin counted one of the two
  h->st.kernel_launches += 1;
  a.chunks = dchunks;
  a.tbase = P<long long>(h->tbase);
  a.tslo = tslo;
  a.runs = runs;
  a.copy = copy;
  a.fd = fd;
  a.out = out;
  a.bulk = bulk ? (h->merge_copy == 1 ? 2 : (h->merge_copy == 2 ? 1 : 3)) : 0;
  const int k = runs.k, S = runs.ncols;
  a.capk = (int)(((kMergeTile + 2ll * k) + 15) / 16 * 16);
  constexpr int threads = 256;
  if (a.capk > kMergeCapMax) return fail(h, SGAGG_ECUDA, "merge fan-in exceeds the tile layout");
  // state columns staged at once: all of them (at least two buffers) within
  // three CTAs per SM, else all within two, else as many as fit two
  constexpr size_t kBudget3 = 74 * 1024, kBudget2 = 112 * 1024;
  const int want = std::max(2, S);
  int scol;
  if (merge_smem_bytes(a.capk, want, k, threads) <= kBudget3) {
    scol = want;
  } else if (merge_smem_bytes(a.capk, want, k, threads) <= kBudget2) {
    scol = want;
  } else {
    scol = 2;
    while (scol + 1 < want && merge_smem_bytes(a.capk, scol + 1, k, threads) <= kBudget2) ++scol;
  }
  a.scol = scol;
  const size_t smem = merge_smem_bytes(a.capk, a.scol, k, threads);
  if (smem > 200 * 1024) return fail(h, SGAGG_ECUDA, "merge tile does not fit shared memory");
  static DeviceOnce once;
  int dev = 0;
  if (once.need(&dev)) {
    CU(cudaFuncSetAttribute(k_merge<256, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    once.done(dev);
  }
  kbegin(h, SGAGG_K_MERGE);
  k_merge<256, 8><<<n_chunks, threads + 32, smem, h->stream>>>(a);
  kend(h);
  CU(cudaGetLastError());
  return SGAGG_OK;
}

sgagg_status sync_read(sgagg_t h, void* dst, const void* src, size_t bytes) {
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return SGAGG_OK;
}

// Host -> device copy ordered on the call's stream, complete on return.
sgagg_status sync_write(sgagg_t h, void* dst, const void* src, size_t bytes) {
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return SGAGG_OK;
}

sgagg_status device_err_status(sgagg_t h, int err) {
  if (err == ERR_TIMEOUT) return fail(h, SGAGG_ETIMEOUT, "device-side wait exceeded the spin limit");
  if (err == ERR_CAPACITY) return fail(h, SGAGG_ECAPACITY, "out_capacity is smaller than the number of distinct keys");
  if (err) return fail(h, SGAGG_ECUDA, "internal device error");
  return SGAGG_OK;
}

// Device -> host copy ordered on the call's stream, together with the
// device error word (one wait for both); a set error word fails the call.
sgagg_status sync_read_checked(sgagg_t h, void* dst, const void* src, size_t bytes) {
  HostSmall* hs = hsmall(h);
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(&hs->err, &dsmall(h)->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return device_err_status(h, hs->err);
}

struct Solver {
  sgagg_t h;
  FoldDesc fd_src;     // how state columns derive from the source's columns
  int n_state;
};

// The chunk planner over nb bucket counts w: up to kPlanSmallMax buckets one
// launch of one block (k_plan_small, which with thist given also turns the
// per-tile histograms into per-tile offsets and fills w), else six small
// launches over up to 1024 blocks (k_plan_*), one bucket per thread up to
// 2^18 buckets (after k_tilescan when thist is given).
sgagg_status run_plan(sgagg_t h, long long* w, int nb, int fine_shift, long long* bstart, Chunk* chunks,
                      int* biglist, PlanInfo* info, long long cap = kTileCap, long long target = kChunkTarget,
                      long long big = kBigBucket, unsigned int* thist = nullptr, int ntiles = 0,
                      int seg_bits = 0) {
  cudaStream_t st = h->stream;
  if (seg_bits > 0 && nb > kPlanSmallMax) return fail(h, SGAGG_ECUDA, "batched plan over too many buckets");
  if (nb <= kPlanSmallMax) {
    k_plan_small<<<1, kPlanSmallThreads, 0, st>>>(thist, ntiles, w, nb, fine_shift, target, big, cap, bstart, chunks,
                                                  biglist, info, seg_bits);
    CU(cudaGetLastError());
    return SGAGG_OK;
  }
  if (thist) {
    k_tilescan<<<(nb * 32 + 255) / 256, 256, 0, st>>>(thist, nb, ntiles, w);
    h->st.class_launches[SGAGG_K_PLAN] += 1;
    h->st.kernel_launches += 1;
  }
  const int sub = std::max(1, (nb + kPlanThreads * 1024 - 1) / (kPlanThreads * 1024));
  const int per = sub * kPlanThreads;
  const int g = (nb + per - 1) / per;
  TRY(grow(h, h->plan_tmp, (size_t)(4 * g + 4) * 8));
  long long* part = P<long long>(h->plan_tmp);
  long long* starts = part + 3 * g;
  k_plan_sums<<<g, kPlanThreads, 0, st>>>(w, nb, per, sub, big, cap, part);
  k_plan_scan3<<<1, 1024, 0, st>>>(part, g, nb, bstart, info);
  k_plan_starts<<<g, kPlanThreads, 0, st>>>(w, nb, per, sub, target, big, part, starts);
  k_plan_scan1<<<1, 1024, 0, st>>>(starts, g, info);
  k_plan_apply<<<g, kPlanThreads, 0, st>>>(w, nb, per, sub, target, big, cap, part, starts,
                                           bstart, chunks, biglist);
  k_plan_finish<<<std::max(1, std::min(4 * h->num_sms, (nb + 255) / 256)), 256, 0, st>>>(nb, fine_shift, bstart,
                                                                                        chunks, info);
  CU(cudaGetLastError());
  h->st.class_launches[SGAGG_K_PLAN] += 5;  // kbegin counted one
  h->st.kernel_launches += 5;
  return SGAGG_OK;
}

sgagg_status ensure_depth(sgagg_t h, int depth) {
  if (depth >= kMaxDepth) return fail(h, SGAGG_ECUDA, "recursion too deep");
  return SGAGG_OK;
}

sgagg_status grow_cols(sgagg_t h, std::vector<DevBuf>& v, int S, size_t bytes) {
  if ((int)v.size() < kMaxCols) v.resize(kMaxCols);  // never reallocated afterwards
  for (int s = 0; s < S; ++s) TRY(grow(h, v[s], bytes));
  return SGAGG_OK;
}

sgagg_status solve(sgagg_t h, const RowSrc& src0, long long n, const FoldDesc& fd0, const OutSink& out,
                   const long long* base_in, long long* total_out, const Digit* gdig, int depth);

// Tile pre-aggregation passes while they shrink the rows at least by half.
// On return *src / *n / *fd describe the (possibly) reduced rows.
sgagg_status prefold(sgagg_t h, RowSrc* src, long long* n, FoldDesc* fd, int force_until_fit) {
  const int S = fd->n_state;
  int which = 0;
  while (*n > kTileCap) {
    DevBuf& kb = h->pf[which];
    auto& cb = h->pfcols[which];
    long long ntile = (*n + kTileCap - 1) / kTileCap;
    TRY(grow(h, kb, (size_t)(*n) * 8));
    TRY(grow_cols(h, cb, S, (size_t)(*n) * 8));
    OutSink o{};
    o.user = 0;
    o.keys = P<unsigned long long>(kb);
    for (int s = 0; s < S; ++s) o.cols[s] = P<long long>(cb[s]);
    o.capacity = *n;
    o.offs = nullptr;
    CopySrc cs{};
    long long* tot = &dsmall(h)->pftot;
    InstSet grp{};
    grp.grouped = h->prefold_bins;
    TRY(launch_sortfold<MODE_TILES>(h, SGAGG_K_PREFOLD, nullptr, (int)ntile, *n, *src, cs, *fd, o,
                                    nullptr, tot, 0, grp));
    HostSmall* hs = hsmall(h);
    TRY(sync_read_checked(h, &hs->v[0], tot, 8));
    ++h->st.prefold_passes;
    long long n2 = hs->v[0];
    kbytes(h, SGAGG_K_PREFOLD, *n * src_row_bytes(*src) + n2 * 8ll * (1 + S));
    RowSrc r{};
    r.kind = SRC_SOA;
    r.ncols = S;
    r.offset = 0;
    r.keys = o.keys;
    for (int s = 0; s < S; ++s) r.cols[s] = o.cols[s];
    bool shrank = n2 * 2 <= *n;
    *src = r;
    *fd = identity_fold(*fd);
    *n = n2;
    which ^= 1;
    if (!shrank && !force_until_fit) break;
  }
  return SGAGG_OK;
}

// Sort and fold n resident rows of src into `out` at *base_in (device),
// writing the end position to *total_out.  gdig: digit whose fine buckets the
// run's offsets use (top level of run generation), else computed here.
sgagg_status solve(sgagg_t h, const RowSrc& src0, long long n, const FoldDesc& fd0, const OutSink& out,
                   const long long* base_in, long long* total_out, const Digit* gdig, int depth) {
  TRY(ensure_depth(h, depth));
  RowSrc src = src0;
  FoldDesc fd = fd0;
  HostSmall* hs = hsmall(h);
  CopySrc nocopy{};

  // keys all equal / small: pre-fold decision from a sample (depth > 0 or
  // when the top level asked for it through prefold_opt)
  bool do_pf = false;
  if (n > kTileCap) {
    if (depth == 0) {
      do_pf = h->top_prefold;
    } else {
      int cnt = (int)std::min<long long>(n, 4096);
      TRY(grow(h, h->sample, (size_t)kSample * 8));
      kbegin(h, SGAGG_K_PROBE);
      k_sample<<<std::max(1, (cnt + 255) / 256), 256, 0, h->stream>>>(src, n, cnt, P<unsigned long long>(h->sample));
      kend(h);
      TRY(sync_read(h, hs->sample, h->sample.p, (size_t)cnt * 8));
      unsigned long long mn, mx;
      const long long dist = sample_distinct(h, hs->sample, cnt, &mn, &mx);
      do_pf = want_prefold(h, cnt, dist);
    }
  }
  if (do_pf) TRY(prefold(h, &src, &n, &fd, 0));

  Digit dig{};
  int nb = 1;
  if (gdig) {
    dig = *gdig;
  }
  if (n > kTileCap && !gdig) {
    // exact key range of these rows
    Small* ds = dsmall(h);
    unsigned long long init[2] = {~0ull, 0ull};
    memcpy(hs->mm, init, sizeof init);
    CU(cudaMemcpyAsync(ds->mm, hs->mm, 16, cudaMemcpyHostToDevice, h->stream));
    kbegin(h, SGAGG_K_PROBE);
    k_minmax<<<std::max(1, std::min(h->num_sms * 4, (int)((n + 1023) / 1024))), 256, 0, h->stream>>>(src, n, ds->mm);
    kend(h);
    kbytes(h, SGAGG_K_PROBE, n * 8);
    TRY(sync_read(h, hs->mm, ds->mm, 16));
    unsigned long long kmin = hs->mm[0], kmax = hs->mm[1];
    if (kmin == kmax) {
      // one key value: tile folds shrink it by kTileCap per pass
      TRY(prefold(h, &src, &n, &fd, 1));
    } else {
      int L = bitlen(kmax - kmin);
      int Db = std::min(kMaxCoarseBits, std::max(1, ilog2_ceil((n + kBucketRows - 1) / kBucketRows)));
      Db = std::min(Db, L);
      dig.base = kmin;
      dig.fbits = Db;
      dig.fshift = L - Db;
      dig.ebits = 0;
    }
  }
  const int W = 1 + src.ncols;

  if (n <= kTileCap) {
    // one chunk, straight from the source (one tile covering the fine range)
    TRY(launch_sortfold<MODE_TILES>(h, SGAGG_K_RUNGEN, nullptr, 1, n, src, nocopy, fd, out, base_in,
                                    total_out, out.offs ? (1 << dig.fbits) : 0));
    kbytes(h, SGAGG_K_RUNGEN, n * src_row_bytes(src));
    return SGAGG_OK;
  }

  // ---- partition by the coarse digit ----
  const int Db = dig.fbits - dig.ebits;
  nb = 1 << Db;
  int ntiles = (int)std::max(1ll, std::min<long long>((n + 8191) / 8192, (long long)h->num_sms * 2));
  set_part_attrs();
  const long long srb = src_row_bytes(src);
  const int C = src.ncols;
  const bool staged = C <= kStageCols;
  Small* ds = dsmall(h);
  TRY(grow(h, h->scatter[depth], (size_t)n * W * 8));
  TRY(grow(h, h->btot[depth], (size_t)nb * 8));
  TRY(grow(h, h->bstart[depth], (size_t)(nb + 1) * 8));
  TRY(grow(h, h->chunks[depth], (size_t)nb * sizeof(Chunk)));
  TRY(grow(h, h->biglist[depth], (size_t)nb * 4));
  if (staged && Db > kLevel1Bits && h->part_levels != 1) {
    // two levels: 2^kLevel1Bits buckets, then the remaining D2 digit bits
    const int D2 = Db - kLevel1Bits, nb1 = 1 << kLevel1Bits, nb2 = 1 << D2;
    const long long nt2max = (n + kTile2 - 1) / kTile2 + nb1;
    TRY(grow(h, h->thist1[depth], (size_t)nb1 * ntiles * 4));
    TRY(grow(h, h->btot1[depth], (size_t)nb1 * 8));
    TRY(grow(h, h->bstart1[depth], (size_t)(nb1 + 1) * 8));
    TRY(grow(h, h->akeys[depth], (size_t)n * 8));
    TRY(grow_cols(h, h->acols[depth], C, (size_t)n * 8));
    TRY(grow(h, h->tiles2[depth], (size_t)nt2max * sizeof(Tile2)));
    TRY(grow(h, h->tfirst[depth], (size_t)(nb1 + 1) * 4));
    TRY(grow(h, h->thist2[depth], (size_t)nt2max * nb2 * 4));
    long long* acp[kMaxCols];
    StageCols acs{};
    for (int c = 0; c < C; ++c) acp[c] = acs.c[c] = P<long long>(h->acols[depth][c]);
    kbegin(h, SGAGG_K_HIST);
    HIST_LAUNCH(k_hist, src, (ntiles, kPartThreads, hist_smem_bytes(nb1, kPartThreads), h->stream),
                (src, n, dig, D2, nb1, ntiles, P<unsigned>(h->thist1[depth])));
    kend(h);
    kbytes(h, SGAGG_K_HIST, n * (srb - 8ll * C) + (long long)nb1 * ntiles * 4);
    kbegin(h, SGAGG_K_PLAN);
    k_tilescan<<<(nb1 * 32 + 255) / 256, 256, 0, h->stream>>>(P<unsigned>(h->thist1[depth]), nb1, ntiles,
                                                            P<long long>(h->btot1[depth]));
    k_scan_tiles2<<<1, kPartThreads, 0, h->stream>>>(P<long long>(h->btot1[depth]), nb1, P<long long>(h->bstart1[depth]),
                                                     P<Tile2>(h->tiles2[depth]), P<int>(h->tfirst[depth]));
    kend(h);
    ++h->st.class_launches[SGAGG_K_PLAN];
    ++h->st.kernel_launches;
    kbegin(h, SGAGG_K_SCATTER);
    STAGED_LAUNCH(src, (ntiles, kPartThreads, staged_smem_bytes(nb1, C), h->stream),
                (src, n, dig, D2, nb1, ntiles, nullptr, nullptr, P<unsigned>(h->thist1[depth]),
                 P<long long>(h->bstart1[depth]), P<unsigned long long>(h->akeys[depth]),
                 acs, nullptr));
    kend(h);
    kbytes(h, SGAGG_K_SCATTER, n * (srb + 8ll * W));
    RowSrc a{};
    a.kind = SRC_SOA;
    a.ncols = C;
    a.keys = P<unsigned long long>(h->akeys[depth]);
    for (int c = 0; c < C; ++c) a.cols[c] = acp[c];
    int* ntd = P<int>(h->tfirst[depth]) + nb1;
    kbegin(h, SGAGG_K_HIST);
    HIST_LAUNCH(k_hist2, a, ((int)nt2max, kPartThreads, hist2_smem_bytes(nb2), h->stream),
                (a, dig, nb2, P<Tile2>(h->tiles2[depth]), ntd, P<unsigned>(h->thist2[depth])));
    kend(h);
    kbytes(h, SGAGG_K_HIST, n * 8ll + nt2max * nb2 * 4);
    kbegin(h, SGAGG_K_PLAN);
    k_scan2<<<nb1, kPartThreads, 0, h->stream>>>(P<long long>(h->bstart1[depth]), nb2, P<int>(h->tfirst[depth]),
                                                P<unsigned>(h->thist2[depth]), P<long long>(h->btot[depth]));
    kend(h);
    kbegin(h, SGAGG_K_SCATTER);
    STAGED_LAUNCH(a, ((int)nt2max, kPartThreads, staged_smem_bytes(nb2, C), h->stream),
                (a, n, dig, 0, nb2, 0, P<Tile2>(h->tiles2[depth]), ntd, P<unsigned>(h->thist2[depth]), nullptr,
                 nullptr, StageCols{}, P<long long>(h->scatter[depth])));
    kend(h);
    kbytes(h, SGAGG_K_SCATTER, n * 16ll * W);
    kbegin(h, SGAGG_K_PLAN);
    TRY(run_plan(h, P<long long>(h->btot[depth]), nb, dig.ebits, P<long long>(h->bstart[depth]),
                 P<Chunk>(h->chunks[depth]), P<int>(h->biglist[depth]), &ds->info));
    kend(h);
    CU(cudaGetLastError());
  } else {
    TRY(grow(h, h->thist[depth], (size_t)nb * ntiles * 4));
    kbegin(h, SGAGG_K_HIST);
    HIST_LAUNCH(k_hist, src, (ntiles, kPartThreads, hist_smem_bytes(nb, kPartThreads), h->stream),
                (src, n, dig, 0, nb, ntiles, P<unsigned int>(h->thist[depth])));
    kend(h);
    kbytes(h, SGAGG_K_HIST, n * (srb - 8ll * C) + (long long)nb * ntiles * 4);
    kbegin(h, SGAGG_K_PLAN);
    TRY(run_plan(h, P<long long>(h->btot[depth]), nb, dig.ebits, P<long long>(h->bstart[depth]),
                 P<Chunk>(h->chunks[depth]), P<int>(h->biglist[depth]), &ds->info, kTileCap, kChunkTarget,
                 kBigBucket, P<unsigned int>(h->thist[depth]), ntiles));
    kend(h);
    kbytes(h, SGAGG_K_PLAN, (long long)nb * ntiles * 8 + (long long)nb * (8 + 8 + sizeof(Chunk)));
    kbegin(h, SGAGG_K_SCATTER);
    if (staged && Db <= kLevel1Bits)
      STAGED_LAUNCH(src, (ntiles, kPartThreads, staged_smem_bytes(nb, C), h->stream),
                  (src, n, dig, 0, nb, ntiles, nullptr, nullptr, P<unsigned>(h->thist[depth]),
                   P<long long>(h->bstart[depth]), nullptr, StageCols{}, P<long long>(h->scatter[depth])));
    else
      PART_LAUNCH(k_scatter, (ntiles, kPartThreads, nb * 4, h->stream),
                  (src, n, dig, nb, ntiles, P<unsigned int>(h->thist[depth]), P<long long>(h->bstart[depth]),
                   P<long long>(h->scatter[depth])));
    kend(h);
    kbytes(h, SGAGG_K_SCATTER, n * (srb + 8ll * W) + (long long)nb * ntiles * 4);
    CU(cudaGetLastError());
  }
  TRY(sync_read(h, &hs->info, &ds->info, sizeof(PlanInfo)));
  PlanInfo info = hs->info;
  if (info.max_chunk > kTileCap) return fail(h, SGAGG_ECUDA, "planner produced an oversized chunk");

  RowSrc aos{};
  aos.kind = SRC_AOS;
  aos.ncols = src.ncols;
  aos.offset = 0;
  aos.aos = P<long long>(h->scatter[depth]);

  CopySrc copy{};
  if (info.n_big > 0) {
    // solve every big bucket on its own, into this depth's copy buffer
    std::vector<int> big(info.n_big);
    TRY(sync_read(h, big.data(), h->biglist[depth].p, (size_t)info.n_big * 4));
    std::vector<Chunk> bch(info.n_big);
    long long tot = 0;
    for (int i = 0; i < info.n_big; ++i) {
      TRY(sync_read(h, &bch[i], P<Chunk>(h->chunks[depth]) + big[i], sizeof(Chunk)));
      tot += bch[i].hi - bch[i].lo;
    }
    const int S = fd.n_state;
    TRY(grow(h, h->copykeys[depth], (size_t)tot * 8));
    TRY(grow_cols(h, h->copycols[depth], S, (size_t)tot * 8));
    OutSink co{};
    co.user = 0;
    co.keys = P<unsigned long long>(h->copykeys[depth]);
    for (int s = 0; s < S; ++s) co.cols[s] = P<long long>(h->copycols[depth][s]);
    co.capacity = tot;
    co.offs = nullptr;
    long long at = 0;
    for (int i = 0; i < info.n_big; ++i) {
      RowSrc sub = aos;
      sub.offset = bch[i].lo;
      long long m = bch[i].hi - bch[i].lo;
      long long* tdev = &ds->dtot[depth];
      hs->v[0] = at;
      CU(cudaMemcpyAsync(tdev, &hs->v[0], 8, cudaMemcpyHostToDevice, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      // base and total share one word: chunk 0 reads it before the last chunk writes it
      TRY(solve(h, sub, m, fd, co, tdev, tdev, nullptr, depth + 1));
      ++h->st.split_segments;
      TRY(sync_read_checked(h, &hs->v[1], tdev, 8));
      long long end = hs->v[1];
      bch[i].lo = at;
      bch[i].hi = end;
      at = end;
      TRY(sync_write(h, P<Chunk>(h->chunks[depth]) + big[i], &bch[i], sizeof(Chunk)));
    }
    copy.keys = co.keys;
    for (int s = 0; s < S; ++s) copy.cols[s] = co.cols[s];
  }
  TRY(launch_sortfold<MODE_RANGE>(h, SGAGG_K_RUNGEN, P<Chunk>(h->chunks[depth]), info.n_chunks, 0, aos,
                                  copy, fd, out, base_in, total_out));
  kbytes(h, SGAGG_K_RUNGEN, n * 8ll * W);
  return SGAGG_OK;
}

void build_keycols(const sgagg_keys* keys, KeyCols* kc, KeyOut* ko, void* const* out_keys) {
  kc->n_cols = keys->n_cols;
  ko->n_cols = keys->n_cols;
  int below = 0;
  for (int c = keys->n_cols - 1; c >= 0; --c) {
    kc->bytes[c] = keys->bytes[c];
    kc->shift[c] = below;
    kc->cols[c] = keys->cols[c];
    ko->bytes[c] = keys->bytes[c];
    ko->shift[c] = below;
    ko->cols[c] = out_keys ? out_keys[c] : nullptr;
    below += 8 * keys->bytes[c];
  }
}

// Argument checks shared by every entry point; *msg gets a static message.
sgagg_status check_args(const sgagg_keys* keys, const int64_t* const* payload, int32_t n_payload, int64_t n,
                        const sgagg_spec* spec, void* const* out_keys, int64_t* const* out_aggs,
                        int64_t out_capacity, const char** msg) {
#define BAD(m) do { *msg = m; return SGAGG_EINVAL; } while (0)
  if (!keys || !spec) BAD("null keys or spec");
  if (n < 0) BAD("n < 0");
  if (out_capacity < 0) BAD("out_capacity < 0");
  if (keys->n_cols < 1 || keys->n_cols > kMaxKeyCols || !keys->bytes || !keys->cols)
    BAD("bad key columns");
  int bits = 0;
  for (int c = 0; c < keys->n_cols; ++c) {
    int b = keys->bytes[c];
    if (b != 1 && b != 2 && b != 4 && b != 8) BAD("key column width must be 1, 2, 4 or 8 bytes");
    bits += 8 * b;
    if (n > 0 && !keys->cols[c]) BAD("null key column");
  }
  if (bits > 64) BAD("key columns wider than 64 bits");
  if (spec->n_aggs < 0 || spec->n_aggs > kMaxCols || (spec->n_aggs > 0 && !spec->aggs))
    BAD("bad aggregate spec");
  if (n_payload < 0 || n_payload > 1024 || (n_payload > 0 && !payload))
    BAD("bad payload columns");
  for (int a = 0; a < spec->n_aggs; ++a) {
    int op = spec->aggs[a].op;
    if (op < SGAGG_COUNT || op > SGAGG_MAX) BAD("bad aggregate op");
    if (op != SGAGG_COUNT) {
      int c = spec->aggs[a].col;
      if (c < 0 || c >= n_payload) BAD("aggregate column out of range");
      if (n > 0 && !payload[c]) BAD("null payload column");
    }
  }
  if (out_capacity > 0 || n > 0) {
    if (!out_keys) BAD("null out_keys");
    for (int c = 0; c < keys->n_cols; ++c)
      if (!out_keys[c] && out_capacity > 0) BAD("null output key column");
    if (spec->n_aggs > 0 && !out_aggs) BAD("null out_aggs");
    for (int a = 0; a < spec->n_aggs; ++a)
      if (!out_aggs[a] && out_capacity > 0) BAD("null output aggregate column");
  }
  *msg = "";
  return SGAGG_OK;
#undef BAD
}

sgagg_status validate(sgagg_t h, const sgagg_keys* keys, const int64_t* const* payload, int32_t n_payload,
                      int64_t n, const sgagg_spec* spec, void* const* out_keys, int64_t* const* out_aggs,
                      int64_t out_capacity) {
  if (!h) return SGAGG_EINVAL;
  const char* msg = "";
  sgagg_status st = check_args(keys, payload, n_payload, n, spec, out_keys, out_aggs, out_capacity, &msg);
  if (st != SGAGG_OK) return fail(h, st, "%s", msg);
  return SGAGG_OK;
}

sgagg_status ensure_ctx_device(sgagg_t h) {
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (h->device != dev) {
    h->device = dev;
    CU(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  TRY(grow(h, h->small, sizeof(Small)));
  if (!h->hsmall) CU(cudaHostAlloc(&h->hsmall, sizeof(HostSmall), cudaHostAllocDefault));
  return SGAGG_OK;
}

sgagg_status alloc_host_arena(sgagg_t h, size_t rows, int S) {
  if (h->harena_rows >= rows && (int)h->harena_cols.size() >= S) return SGAGG_OK;
  if (h->harena_keys) cudaFreeHost(h->harena_keys);
  for (void* p : h->harena_cols) cudaFreeHost(p);
  h->harena_keys = nullptr;
  h->harena_cols.clear();
  h->harena_rows = 0;
  ++h->alloc_count;
  if (h->fault_alloc > 0 && h->alloc_count == h->fault_alloc)
    return fail(h, SGAGG_ENOMEM, "injected allocation failure");
  CU(cudaHostAlloc(&h->harena_keys, rows * 8 + 16, cudaHostAllocMapped));
  h->harena_cols.resize(S, nullptr);
  for (int s = 0; s < S; ++s) CU(cudaHostAlloc(&h->harena_cols[s], rows * 8 + 16, cudaHostAllocMapped));
  h->harena_rows = rows;
  return SGAGG_OK;
}

template <class T>
T* host_dev_ptr(sgagg_t h, void* p) {
  void* d = nullptr;
  cudaHostGetDevicePointer(&d, p, 0);
  return reinterpret_cast<T*>(d);
}

// One wide merge (Sec. 4): every run is cut by the same fine-bucket
// boundaries (their sparse indexes); the planner groups fine buckets into
// merge tiles of at most kTileCap rows over all runs, and one CTA per tile
// folds equal keys across runs.  A tile bigger than that (a key range dense
// in many runs) is gathered and solved on its own first, then copied.
sgagg_status merge_runs(sgagg_t h, const std::vector<RunRef>& rr, int S, const FoldDesc& fid, int nf,
                        const OutSink& out, const long long* base_in, long long* total_out, long long* end,
                        bool final_merge) {
  cudaStream_t stream = h->stream;
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  const int K = (int)rr.size();
  const long long row_bytes = 8ll * (1 + S);
  std::vector<const long long*> hp((size_t)K * (1 + S) + K);
  long long in_rows = 0;
  for (int r = 0; r < K; ++r) {
    hp[(size_t)r * (1 + S)] = rr[r].keys;
    for (int s = 0; s < S; ++s) hp[(size_t)r * (1 + S) + 1 + s] = rr[r].cols[s];
    hp[(size_t)K * (1 + S) + r] = rr[r].offs;
    in_rows += rr[r].rows;
  }
  TRY(grow(h, h->runptrs, hp.size() * 8));
  CU(cudaMemcpyAsync(h->runptrs.p, hp.data(), hp.size() * 8, cudaMemcpyHostToDevice, stream));
  RunSet rset{};
  rset.k = K;
  rset.ncols = S;
  rset.ptrs = reinterpret_cast<const long long* const*>(h->runptrs.p);
  rset.offs = reinterpret_cast<const long long* const*>(h->runptrs.p) + (size_t)K * (1 + S);

  TRY(grow(h, h->fsizes, (size_t)nf * 8));
  kbegin(h, SGAGG_K_PLAN);
  k_fine_sizes<<<std::max(1, std::min(4 * h->num_sms, (nf + 255) / 256)), 256, 0, stream>>>(
      rset.offs, K, nf, P<long long>(h->fsizes));
  kend(h);
  kbytes(h, SGAGG_K_PLAN, (long long)K * (nf + 1) * 8 + nf * 8ll);
  TRY(grow(h, h->bstart[0], (size_t)(nf + 1) * 8));
  TRY(grow(h, h->chunks[0], (size_t)nf * sizeof(Chunk)));
  TRY(grow(h, h->biglist[0], (size_t)nf * 4));
  kbegin(h, SGAGG_K_PLAN);
  TRY(run_plan(h, P<long long>(h->fsizes), nf, 0, P<long long>(h->bstart[0]), P<Chunk>(h->chunks[0]),
               P<int>(h->biglist[0]), &ds->info, kMergeTile, kMergeTile - kMergeTile / 4, kMergeTile / 4));
  kend(h);
  CU(cudaGetLastError());
  TRY(sync_read(h, &hs->info, &ds->info, sizeof(PlanInfo)));
  PlanInfo info = hs->info;
  if (final_merge) h->st.merge_tiles = info.n_chunks;
  // every tile's slice of every run (the merge kernel reads one row of it)
  TRY(grow(h, h->tslo, (size_t)(info.n_chunks + 1) * K * 8));
  if (info.n_chunks > 0) {
    kbegin(h, SGAGG_K_PLAN);
    const long long tot = (long long)(info.n_chunks + 1) * K;
    k_tile_slices<<<(int)std::max(1ll, std::min<long long>((tot + 255) / 256, 8ll * h->num_sms)), 256, 0, stream>>>(
        P<Chunk>(h->chunks[0]), info.n_chunks, rset.offs, K, P<long long>(h->tslo));
    kend(h);
    CU(cudaGetLastError());
    kbytes(h, SGAGG_K_PLAN, tot * 16);
  }
  CopySrc copy{};
  if (info.n_big > 0) {
    std::vector<int> big(info.n_big);
    TRY(sync_read(h, big.data(), h->biglist[0].p, (size_t)info.n_big * 4));
    std::vector<Chunk> bch(info.n_big);
    long long tot = 0;
    for (int i = 0; i < info.n_big; ++i) {
      TRY(sync_read(h, &bch[i], P<Chunk>(h->chunks[0]) + big[i], sizeof(Chunk)));
      tot += bch[i].hi - bch[i].lo;
    }
    TRY(grow(h, h->copykeys[0], (size_t)tot * 8));
    TRY(grow_cols(h, h->copycols[0], S, (size_t)tot * 8));
    OutSink co{};
    co.user = 0;
    co.keys = P<unsigned long long>(h->copykeys[0]);
    for (int s = 0; s < S; ++s) co.cols[s] = P<long long>(h->copycols[0][s]);
    co.capacity = tot;
    long long at = 0;
    for (int i = 0; i < info.n_big; ++i) {
      // gather the tile's rows from every run into one SoA buffer
      long long m = bch[i].hi - bch[i].lo;
      std::vector<long long> lo(K), hi(K), pre(K + 1, 0);
      for (int r = 0; r < K; ++r) {
        TRY(sync_read(h, &lo[r], rr[r].offs + bch[i].f_lo, 8));
        TRY(sync_read(h, &hi[r], rr[r].offs + bch[i].f_hi, 8));
        pre[r + 1] = pre[r] + (hi[r] - lo[r]);
      }
      TRY(grow(h, h->gather_keys, (size_t)m * 8));
      TRY(grow_cols(h, h->gather_cols, S, (size_t)m * 8));
      std::vector<long long*> gcols(std::max(1, S));
      for (int s = 0; s < S; ++s) gcols[s] = P<long long>(h->gather_cols[s]);
      TRY(grow(h, h->gather_ptrs, (size_t)(std::max(1, S) + K + 1) * 8));
      long long* dpre = P<long long>(h->gather_ptrs);
      long long** dcols = reinterpret_cast<long long**>(dpre + K + 1);
      TRY(sync_write(h, dpre, pre.data(), (size_t)(K + 1) * 8));
      TRY(sync_write(h, dcols, gcols.data(), (size_t)std::max(1, S) * 8));
      dim3 grid(std::max(1, std::min(64, (int)((m / K + 255) / 256))), K);
      kbegin(h, SGAGG_K_OTHER);
      k_gather_runs<<<grid, 256, 0, stream>>>(rset, bch[i].f_lo, bch[i].f_hi, dpre,
                                              P<unsigned long long>(h->gather_keys), dcols);
      kend(h);
      kbytes(h, SGAGG_K_OTHER, m * 16ll * (1 + S));
      RowSrc gs{};
      gs.kind = SRC_SOA;
      gs.ncols = S;
      gs.keys = P<unsigned long long>(h->gather_keys);
      for (int s = 0; s < S; ++s) gs.cols[s] = gcols[s];
      long long* tdev = &ds->dtot[kMaxDepth + 1];
      hs->v[0] = at;
      CU(cudaMemcpyAsync(tdev, &hs->v[0], 8, cudaMemcpyHostToDevice, stream));
      CU(cudaStreamSynchronize(stream));
      TRY(solve(h, gs, m, fid, co, tdev, tdev, nullptr, 1));
      ++h->st.split_segments;
      TRY(sync_read_checked(h, &hs->v[1], tdev, 8));
      long long e = hs->v[1];
      bch[i].lo = at;
      bch[i].hi = e;
      at = e;
      TRY(sync_write(h, P<Chunk>(h->chunks[0]) + big[i], &bch[i], sizeof(Chunk)));
    }
    copy.keys = co.keys;
    for (int s = 0; s < S; ++s) copy.cols[s] = co.cols[s];
  }
  bool bulk = true;
  for (const RunRef& r : rr) {
    bulk = bulk && !r.host && (reinterpret_cast<unsigned long long>(r.keys) & 15ull) == 0;
    for (int s = 0; s < S; ++s) bulk = bulk && (reinterpret_cast<unsigned long long>(r.cols[s]) & 15ull) == 0;
  }
  if (final_merge && h->hio && info.n_chunks >= 2) {
    // host buffers: merge in parts; each part's output is copied back while
    // the following parts merge
    const int parts = std::min(kMergeParts, info.n_chunks);
    for (int p = 0; p < parts; ++p) {
      const int c0 = (int)((long long)info.n_chunks * p / parts), c1 = (int)((long long)info.n_chunks * (p + 1) / parts);
      TRY(launch_merge(h, P<Chunk>(h->chunks[0]) + c0, c1 - c0, P<long long>(h->tslo) + (long long)c0 * K, rset,
                       bulk, copy, fid, out, p ? &ds->part_tot[p - 1] : base_in, &ds->part_tot[p]));
      CU(cudaMemcpyAsync(&hs->part_end[p], &ds->part_tot[p], 8, cudaMemcpyDeviceToHost, stream));
      if (!h->part_events[p]) CU(cudaEventCreateWithFlags(&h->part_events[p], cudaEventDisableTiming));
      CU(cudaEventRecord(h->part_events[p], stream));
    }
    long long prev = 0;
    for (int p = 0; p < parts; ++p) {
      CU(cudaEventSynchronize(h->part_events[p]));
      const long long e = hs->part_end[p];
      TRY(unstage_rows(h, prev, e, h->part_events[p]));
      prev = std::max(prev, e);
    }
    h->hio->copied_out = prev;
    CU(cudaMemcpyAsync(total_out, &ds->part_tot[parts - 1], 8, cudaMemcpyDeviceToDevice, stream));
  } else {
    TRY(launch_merge(h, P<Chunk>(h->chunks[0]), info.n_chunks, P<long long>(h->tslo), rset, bulk, copy, fid, out,
                     base_in, total_out));
  }
  TRY(sync_read_checked(h, &hs->v[0], total_out, 8));
  *end = hs->v[0];
  const long long out_row_bytes = out.user ? (h->key_bytes + 8ll * S) : row_bytes;
  kbytes(h, SGAGG_K_MERGE, in_rows * row_bytes);
  kbytes(h, SGAGG_K_MERGE, (final_merge ? *end : 0) * out_row_bytes);
  return SGAGG_OK;
}

// Wide merge of all runs into the caller's output (Sec. 4), after
// preliminary merges of the smallest runs when they exceed the fan-in
// (Sec. 4.3).
sgagg_status merge_all(sgagg_t h, std::vector<RunRef> rr, int S, const FoldDesc& fd, int nf, long long stride,
                       const Digit& gd, const OutSink& user, const long long* base_in = nullptr) {
  cudaStream_t stream = h->stream;
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  const long long row_bytes = 8ll * (1 + S);
  FoldDesc fid = identity_fold(fd);
  const int cap = (h->fanin_cap > 0) ? std::min(h->fanin_cap, kMaxFanIn) : kMaxFanIn;
  if ((int)rr.size() > cap) {
    // preliminary merges of the smallest runs until one wide merge can take
    // every run (Sec. 4.3); each writes a new run into the merge arena
    // rows all preliminary merges may write: replay the schedule with each
    // merged run as large as its inputs (an upper bound)
    long long need = 0;
    int extra = 0;
    {
      std::vector<long long> sz;
      for (auto& r : rr) sz.push_back(r.rows);
      while ((int)sz.size() > cap) {
        const int g = std::min<int>(cap, (int)sz.size() - cap + 1);
        std::stable_sort(sz.begin(), sz.end());
        long long m = 0;
        for (int i = 0; i < g; ++i) m += sz[i];
        sz.erase(sz.begin(), sz.begin() + g);
        sz.push_back(m);
        need += m;
        ++extra;
      }
    }
    TRY(grow(h, h->marena_keys, (size_t)std::max(1ll, need) * 8 + kRunSlack));
    TRY(grow_cols(h, h->marena_cols, S, (size_t)std::max(1ll, need) * 8 + kRunSlack));
    TRY(grow(h, h->moffs, (size_t)extra * stride * 8));
    long long used = 0;
    int made = 0;
    while ((int)rr.size() > cap) {
      const int g = std::min<int>(cap, (int)rr.size() - cap + 1);
      std::stable_sort(rr.begin(), rr.end(), [](const RunRef& x, const RunRef& y) { return x.rows < y.rows; });
      std::vector<RunRef> part(rr.begin(), rr.begin() + g);
      OutSink o{};
      o.user = 0;
      o.keys = P<unsigned long long>(h->marena_keys);
      for (int s = 0; s < S; ++s) o.cols[s] = P<long long>(h->marena_cols[s]);
      o.capacity = need;
      o.offs = P<long long>(h->moffs) + (long long)made * stride;
      o.dig = gd;
      long long* slot = &ds->dtot[kMaxDepth];
      hs->v[0] = used;
      CU(cudaMemcpyAsync(slot, &hs->v[0], 8, cudaMemcpyHostToDevice, stream));
      long long end = 0;
      TRY(merge_runs(h, part, S, fid, nf, o, slot, slot, &end, false));
      RunRef nr;
      nr.keys = P<long long>(h->marena_keys);
      for (int s = 0; s < S; ++s) nr.cols[s] = P<long long>(h->marena_cols[s]);
      nr.offs = o.offs;
      nr.rows = end - used;
      used = end;
      ++made;
      h->st.run_rows += nr.rows;
      h->run_sizes.push_back(nr.rows);
      h->st.run_bytes_device += nr.rows * row_bytes;
      ++h->st.runs;
      rr.erase(rr.begin(), rr.begin() + g);
      rr.push_back(nr);
    }
  }
  long long rows = 0;
  TRY(merge_runs(h, rr, S, fid, nf, user, base_in, &ds->total, &rows, true));
  h->last_rows = rows;
  h->st.out_rows = rows;
  return SGAGG_OK;
}

// Run generation with an absorbing index (SGAGG_OPT_POLICY = 1; Sec. 3 on
// early aggregation absorbing equal keys in the in-memory index, Sec. 6.1 on
// the in-sort algorithm: each batch sorted first, only its distinct keys
// looked up in the ordered index, the index written as a run when memory
// runs out).  The index is a sorted, folded array of at most M keys with an
// extra flag column (0 for rows of the index).  Per batch:
//   1. the batch is grouped (sorted, folded) with flag 1 on every key;
//   2. it is merged into the index (wide-merge kernel, two runs; flags
//      combine by min, so a merged row's flag says "not in the index");
//   3. if the new keys fit, the merged rows are the index; else, taking new
//      keys in ascending order, the index is full at the (q+1)-th new key t,
//      q = M - |index|: the merged rows below t and the index rows from t on
//      are written as a run of M keys, and the batch's keys from t on fill the
//      emptied index, M at a time (every full index but the last becomes a
//      run).
// No run at all when the output fits M keys; else the index is the last run
// and all runs go through the wide merge.
sgagg_status absorb_device(sgagg_t h, const RowSrc& raw, long long n, const FoldDesc& fd, int S,
                           const OutSink& user, const Digit& gd) {
  cudaStream_t stream = h->stream;
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  const long long M = h->M;
  const long long Bz = h->absorb_batch > 0 ? h->absorb_batch : std::min<long long>(M, 1ll << 22);
  const long long nb = (n + Bz - 1) / Bz;
  h->st.batches = nb;
  const int S1 = S + 1;
  if (S1 > kMaxCols) return fail(h, SGAGG_EINVAL, "too many aggregates for the absorbing policy");
  FoldDesc fdx = fd;  // the batch: the aggregates, then the flag (1)
  fdx.n_state = S1;
  fdx.src[S] = -1;
  fdx.op[S] = OP_MAX;
  FoldDesc fmx = identity_fold(fdx);  // the merge: flags by min
  fmx.op[S] = OP_MIN;
  const int nf = 1 << gd.fbits;
  const long long stride = nf + 1;
  const long long cap3 = M + std::min(Bz, n);
  for (int i = 0; i < 3; ++i) {
    TRY(grow(h, h->ab_keys[i], (size_t)cap3 * 8 + kRunSlack));
    TRY(grow_cols(h, h->ab_cols[i], S1, (size_t)cap3 * 8 + kRunSlack));
    TRY(grow(h, h->ab_offs[i], (size_t)stride * 8));
  }
  TRY(grow(h, h->ab_tmp, (size_t)(1024 + 8) * 8));
  const long long max_runs = n / M + 2;  // every run but the last holds M rows
  TRY(grow(h, h->arena_keys, (size_t)n * 8 + kRunSlack));
  TRY(grow_cols(h, h->arena_cols, S, (size_t)n * 8 + kRunSlack));
  h->arena_keys.arena = true;
  for (auto& b : h->arena_cols) b.arena = true;
  TRY(grow(h, h->offs, (size_t)max_runs * stride * 8));

  auto soa = [&](int i) {
    SoaRef r{};
    r.keys = P<unsigned long long>(h->ab_keys[i]);
    for (int c = 0; c < S1; ++c) r.cols[c] = P<long long>(h->ab_cols[i][c]);
    return r;
  };
  SoaRef arena{};
  arena.keys = P<unsigned long long>(h->arena_keys);
  for (int c = 0; c < S; ++c) arena.cols[c] = P<long long>(h->arena_cols[c]);
  auto grid = [&](long long m) {
    return (int)std::max(1ll, std::min<long long>((m + 255) / 256, (long long)h->num_sms * 8));
  };
  std::vector<Run> runs;
  long long acur = 0, rstart = 0;  // arena cursor, start of the run being written
  const long long row_bytes = 8ll * (1 + S);
  auto append = [&](int src, long long off, long long m) {
    if (m <= 0) return;
    kbegin(h, SGAGG_K_OTHER);
    k_copy_soa<<<grid(m), 256, 0, stream>>>(soa(src), off, arena, acur, m, S, -1);
    kend(h);
    kbytes(h, SGAGG_K_OTHER, m * 2 * row_bytes);
    acur += m;
  };
  auto close_run = [&]() -> sgagg_status {
    const long long m = acur - rstart;
    if ((long long)runs.size() >= max_runs) return fail(h, SGAGG_ECUDA, "absorbing policy: run table overflow");
    kbegin(h, SGAGG_K_PLAN);
    k_offsets_by_search<<<std::max(1, std::min(4 * h->num_sms, (nf + 256) / 256)), 256, 0, stream>>>(
        arena.keys + rstart, m, gd, nf, rstart, P<long long>(h->offs) + (long long)runs.size() * stride);
    kend(h);
    CU(cudaGetLastError());
    runs.push_back(Run{rstart, m, 0});
    h->st.run_rows += m;
    h->run_sizes.push_back(m);
    h->st.run_bytes_device += m * row_bytes;
    rstart = acur;
    return SGAGG_OK;
  };

  int iR = 0, iD = 1, iT = 2;
  long long r = 0;  // keys in the index
  for (long long b = 0; b < nb; ++b) {
    const long long m = std::min(Bz, n - b * Bz);
    RowSrc bs = raw;
    bs.offset = b * Bz;
    OutSink od{};
    od.user = 0;
    SoaRef d = soa(iD);
    od.keys = d.keys;
    for (int c = 0; c < S1; ++c) od.cols[c] = d.cols[c];
    od.capacity = cap3;
    od.offs = P<long long>(h->ab_offs[iD]);
    od.dig = gd;
    TRY(solve(h, bs, m, fdx, od, nullptr, &ds->total, &gd, 0));
    TRY(sync_read_checked(h, &hs->v[0], &ds->total, 8));
    const long long dn = hs->v[0];
    int iM = iD;  // buffer of the merged rows
    long long tn = dn;
    if (r > 0) {
      RunRef a{}, c{};
      SoaRef x = soa(iR);
      a.keys = reinterpret_cast<const long long*>(x.keys);
      for (int k = 0; k < S1; ++k) a.cols[k] = x.cols[k];
      a.offs = P<long long>(h->ab_offs[iR]);
      a.rows = r;
      c.keys = reinterpret_cast<const long long*>(d.keys);
      for (int k = 0; k < S1; ++k) c.cols[k] = d.cols[k];
      c.offs = P<long long>(h->ab_offs[iD]);
      c.rows = dn;
      OutSink ot{};
      ot.user = 0;
      SoaRef t = soa(iT);
      ot.keys = t.keys;
      for (int k = 0; k < S1; ++k) ot.cols[k] = t.cols[k];
      ot.capacity = cap3;
      ot.offs = P<long long>(h->ab_offs[iT]);
      ot.dig = gd;
      TRY(merge_runs(h, std::vector<RunRef>{a, c}, S1, fmx, nf, ot, nullptr, &ds->total, &tn, false));
      iM = iT;
    }
    const long long fresh = tn - r;  // batch keys not in the index
    if (r + fresh <= M) {
      std::swap(iR, iM == iT ? iT : iD);
      r = tn;
      CU(cudaMemsetAsync(P<long long>(h->ab_cols[iR][S]), 0, (size_t)r * 8, stream));
      continue;
    }
    const long long q = M - r;
    long long p = q, pr = 0, pd = q;
    if (r > 0) {
      long long* tmp = P<long long>(h->ab_tmp);
      const long long* flag = P<long long>(h->ab_cols[iT][S]);
      const int nbk = (int)std::max(1ll, std::min<long long>(1024, (tn + 4095) / 4096));
      const long long per = (tn + nbk - 1) / nbk;
      kbegin(h, SGAGG_K_PLAN);
      k_flag_counts<<<nbk, 256, 0, stream>>>(flag, tn, per, tmp);
      k_nth_flag<<<1, 1024, 0, stream>>>(flag, tn, per, tmp, nbk, q + 1, tmp + 1024);
      k_split_at<<<1, 32, 0, stream>>>(soa(iT).keys, tmp + 1024, soa(iR).keys, r, d.keys, dn, tmp + 1025);
      kend(h);
      CU(cudaGetLastError());
      TRY(sync_read(h, &hs->v[0], tmp + 1024, 24));
      p = hs->v[0];
      pr = hs->v[1];
      pd = hs->v[2];
      if (p >= tn || p + (r - pr) != M) return fail(h, SGAGG_ECUDA, "absorbing policy: inconsistent split");
    }
    // the full index: merged rows below t, then the index rows from t on
    append(iM, 0, p);
    append(iR, pr, r - pr);
    TRY(close_run());
    // the batch keys from t on refill the emptied index, M at a time
    long long off = pd, left = dn - pd;
    while (left > M) {
      append(iD, off, M);
      TRY(close_run());
      off += M;
      left -= M;
    }
    kbegin(h, SGAGG_K_OTHER);
    k_copy_soa<<<grid(std::max(1ll, left)), 256, 0, stream>>>(d, off, soa(iR), 0, left, S1, S);
    k_offsets_by_search<<<std::max(1, std::min(4 * h->num_sms, (nf + 256) / 256)), 256, 0, stream>>>(
        soa(iR).keys, left, gd, nf, 0, P<long long>(h->ab_offs[iR]));
    kend(h);
    CU(cudaGetLastError());
    r = left;
  }
  h->st.runs = (long long)runs.size();
  if (runs.empty()) {
    // the whole input was absorbed: the index is the output (Sec. 3)
    if (r > user.capacity) return fail(h, SGAGG_ECAPACITY, "out_capacity is smaller than the number of distinct keys");
    kbegin(h, SGAGG_K_OTHER);
    k_emit_soa<<<grid(std::max(1ll, r)), 256, 0, stream>>>(soa(iR), r, S, user);
    kend(h);
    CU(cudaGetLastError());
    kbytes(h, SGAGG_K_OTHER, r * (row_bytes + h->key_bytes + 8ll * S));
    h->last_rows = r;
    h->st.out_rows = r;
    return SGAGG_OK;
  }
  append(iR, 0, r);
  TRY(close_run());
  h->st.runs = (long long)runs.size();
  std::vector<RunRef> rr(runs.size());
  for (size_t i = 0; i < runs.size(); ++i) {
    rr[i].keys = reinterpret_cast<const long long*>(arena.keys);
    for (int c = 0; c < S; ++c) rr[i].cols[c] = arena.cols[c];
    rr[i].offs = P<long long>(h->offs) + (long long)i * stride;
    rr[i].rows = runs[i].rows;
  }
  return merge_all(h, rr, S, fd, nf, stride, gd, user);
}

// One batch whose keys take few values (Example 1, Sec. 3.2): one streaming
// pass folds every row into accumulators of the sampled distinct keys
// (kd <= kLowCardKeys, ascending).  *done is false when some row's key is
// not among them; the caller then groups the input by the general path.
sgagg_status lowcard_device(sgagg_t h, const RowSrc& raw, long long n, const FoldDesc& fd,
                            const unsigned long long* keys, int kd, const OutSink& user, bool* done) {
  *done = false;
  const int S = fd.n_state;
  LowCardArgs a{};
  a.src = raw;
  a.n = n;
  a.kd = kd;
  for (int g = 0; g < kd; ++g) a.keys[g] = keys[g];
  a.fd = fd;
  // aggregates by source column: count(*) first, then column 0, 1, ...
  int q = 0;
  for (int ag = 0; ag < S; ++ag)
    if (fd.src[ag] < 0) a.order[q++] = (int8_t)ag;
  a.col_end[0] = (int8_t)q;
  for (int c = 0; c < raw.ncols; ++c) {
    for (int ag = 0; ag < S; ++ag)
      if (fd.src[ag] == c) a.order[q++] = (int8_t)ag;
    a.col_end[c + 1] = (int8_t)q;
  }
  a.n_col = raw.ncols;
  const int T = (size_t)kd * S * 8 * 256 <= 110 * 1024 ? 256 : 128;
  // the report pattern: count(*), then sum / min / max of every payload
  // column in column order
  int cp = (S >= 1 && (S - 1) % 3 == 0 && fd.src[0] < 0) ? (S - 1) / 3 : 0;
  for (int c = 0; c < cp; ++c)
    if (fd.src[1 + 3 * c] != c || fd.src[2 + 3 * c] != c || fd.src[3 + 3 * c] != c || fd.op[1 + 3 * c] != OP_SUM ||
        fd.op[2 + 3 * c] != OP_MIN || fd.op[3 + 3 * c] != OP_MAX || raw.ncols != cp)
      cp = 0;
  if (cp > 4 || T != 256) cp = 0;
  // the report kernel keeps one set of accumulators per lane pair (128 per
  // block, three CTAs per SM); the general kernel one per thread
  const size_t smem = (size_t)kd * S * 8 * (cp >= 1 ? 128 : T);
  // the general kernel: as many blocks per SM as their accumulators fit (at
  // most 4, 227 KB of shared memory per SM)
  const int blocks = h->num_sms * (cp >= 1 ? 3 : (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (smem + 1024))));
  TRY(grow(h, h->lc_part, (size_t)blocks * kd * std::max(1, S) * 8));
  a.partial = P<long long>(h->lc_part);
  Small* ds = dsmall(h);
  a.overflow = &ds->lc_over;
  static DeviceOnce once;
  int dev = 0;
  if (once.need(&dev)) {
    CU(cudaFuncSetAttribute(k_lowcard<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024));
    CU(cudaFuncSetAttribute(k_lowcard<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024));
    CU(cudaFuncSetAttribute(k_lowcard<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024));
    CU(cudaFuncSetAttribute(k_lowcard<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024));
    CU(cudaFuncSetAttribute(k_lowcard<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024));
    once.done(dev);
  }
  const int kl = raw.key.n_cols == 1 && raw.key.bytes[0] == 8 ? 1
                 : (raw.key.n_cols == 2 && raw.key.bytes[0] == 1 && raw.key.bytes[1] == 1 ? 2 : 0);
  static DeviceOnce once_r;
  if (once_r.need(&dev)) {
#define LCR_ATTR(C)                                                                                     \
  CU(cudaFuncSetAttribute(k_lowcard_report<C, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024)); \
  CU(cudaFuncSetAttribute(k_lowcard_report<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024)); \
  CU(cudaFuncSetAttribute(k_lowcard_report<C, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024));
    LCR_ATTR(1) LCR_ATTR(2) LCR_ATTR(3) LCR_ATTR(4)
#undef LCR_ATTR
    once_r.done(dev);
  }
  CU(cudaMemsetAsync(&ds->lc_over, 0, sizeof(int), h->stream));
  kbegin(h, SGAGG_K_STREAM);
#define LCR_LAUNCH(C)                                                                 \
  do {                                                                                \
    if (kl == 1) k_lowcard_report<C, 1><<<blocks, T, smem, h->stream>>>(a);           \
    else if (kl == 2) k_lowcard_report<C, 2><<<blocks, T, smem, h->stream>>>(a);      \
    else k_lowcard_report<C, 0><<<blocks, T, smem, h->stream>>>(a);                   \
  } while (0)
  if (cp == 1) LCR_LAUNCH(1);
  else if (cp == 2) LCR_LAUNCH(2);
  else if (cp == 3) LCR_LAUNCH(3);
  else if (cp == 4) LCR_LAUNCH(4);
#undef LCR_LAUNCH
  else if (S <= 2) k_lowcard<2><<<blocks, T, smem, h->stream>>>(a);
  else if (S <= 4) k_lowcard<4><<<blocks, T, smem, h->stream>>>(a);
  else if (S <= 8) k_lowcard<8><<<blocks, T, smem, h->stream>>>(a);
  else if (S <= 16) k_lowcard<16><<<blocks, T, smem, h->stream>>>(a);
  else k_lowcard<32><<<blocks, T, smem, h->stream>>>(a);
  OutSinkLite ol{};
  ol.kout = user.kout;
  for (int s = 0; s < S; ++s) ol.cols[s] = user.cols[s];
  ol.capacity = user.capacity;
  k_lowcard_finish<<<1, 256, 0, h->stream>>>(a, blocks, ol, &ds->total);
  kend(h);
  ++h->st.class_launches[SGAGG_K_STREAM];
  ++h->st.kernel_launches;
  CU(cudaGetLastError());
  HostSmall* hs = hsmall(h);
  TRY(sync_read(h, hs->v, &ds->total, 8));
  int over = 0;
  TRY(sync_read(h, &over, &ds->lc_over, sizeof(int)));
  long long rb = 0;
  for (int c = 0; c < raw.key.n_cols; ++c) rb += raw.key.bytes[c];
  kbytes(h, SGAGG_K_STREAM, n * (rb + 8ll * raw.ncols));
  if (over) return SGAGG_OK;  // not done: the general path takes the input
  if (kd > user.capacity) return fail(h, SGAGG_ECAPACITY, "out_capacity is smaller than the number of distinct keys");
  kbytes(h, SGAGG_K_STREAM, kd * (h->key_bytes + 8ll * S));
  h->last_rows = kd;
  h->st.out_rows = kd;
  *done = true;
  return SGAGG_OK;
}

// Run generation in read-sort-write cycles of M rows of src (one run per
// batch, Sec. 3 and Sec. 6.1), then one wide merge of all runs into the
// caller's output at *base_in (Sec. 4; nullptr: 0).  stage_io: src is the
// host-buffer call's staged input, copied batch by batch.
// Every batch's run in one pass per step, for small batches (where the
// launches and host round trips of a batch, not its rows, would set the
// time): the digit gives each batch buckets of its own (batch << Db plus the
// key digit), the planner never lets a chunk span two batches, and one
// sort+fold launch writes the runs back to back, each chunk into its batch's
// sparse index.  The runs are exactly those a batch at a time would write
// (each is its batch's distinct keys in key order, folded).  *done stays
// false, with nothing the caller relies on written, when some bucket is
// bigger than a chunk; the caller then takes the batches one at a time.
constexpr long long kOnePassRows = 1ll << 24;

sgagg_status runs_one_pass(sgagg_t h, const RowSrc& src, long long n, long long M, long long B, const FoldDesc& fd,
                           const Digit& gd, const OutSink& o, long long stride, long long* rs_dev, bool* done) {
  *done = false;
  cudaStream_t stream = h->stream;
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  const int Db = gd.fbits - gd.ebits;
  const int nb = (int)(B << Db);
  const int T = (int)std::max(1ll, std::min((M + 8191) / 8192, (2ll * h->num_sms + B - 1) / B));
  const int ntiles = (int)(B * T);
  Digit dig = gd;
  dig.brows = M;
  dig.btiles = T;
  dig.bbits = Db;
  set_part_attrs();
  const int W = 1 + src.ncols;
  const long long srb = src_row_bytes(src);
  TRY(grow(h, h->scatter[0], (size_t)n * W * 8));
  TRY(grow(h, h->btot[0], (size_t)nb * 8));
  TRY(grow(h, h->bstart[0], (size_t)(nb + 1) * 8));
  TRY(grow(h, h->chunks[0], (size_t)nb * sizeof(Chunk)));
  TRY(grow(h, h->biglist[0], (size_t)nb * 4));
  TRY(grow(h, h->thist[0], (size_t)nb * ntiles * 4));
  kbegin(h, SGAGG_K_HIST);
  HIST_LAUNCH(k_hist, src, (ntiles, kPartThreads, hist_smem_bytes(nb, kPartThreads), stream),
              (src, n, dig, 0, nb, ntiles, P<unsigned>(h->thist[0])));
  kend(h);
  kbytes(h, SGAGG_K_HIST, n * (srb - 8ll * src.ncols) + (long long)nb * ntiles * 4);
  kbegin(h, SGAGG_K_PLAN);
  TRY(run_plan(h, P<long long>(h->btot[0]), nb, dig.ebits, P<long long>(h->bstart[0]), P<Chunk>(h->chunks[0]),
               P<int>(h->biglist[0]), &ds->info, kTileCap, kChunkTarget, kBigBucket, P<unsigned>(h->thist[0]),
               ntiles, Db));
  kend(h);
  kbytes(h, SGAGG_K_PLAN, (long long)nb * ntiles * 8 + (long long)nb * (8 + 8 + sizeof(Chunk)));
  TRY(sync_read(h, &hs->info, &ds->info, sizeof(PlanInfo)));
  const PlanInfo info = hs->info;
  if (info.n_big > 0 || info.max_chunk > kTileCap) return SGAGG_OK;
  kbegin(h, SGAGG_K_SCATTER);
  PART_LAUNCH(k_scatter, (ntiles, kPartThreads, nb * 4, stream),
              (src, n, dig, nb, ntiles, P<unsigned int>(h->thist[0]), P<long long>(h->bstart[0]),
               P<long long>(h->scatter[0])));
  kend(h);
  kbytes(h, SGAGG_K_SCATTER, n * (srb + 8ll * W) + (long long)nb * ntiles * 4);
  CU(cudaGetLastError());
  RowSrc aos{};
  aos.kind = SRC_AOS;
  aos.ncols = src.ncols;
  aos.offset = 0;
  aos.aos = P<long long>(h->scatter[0]);
  OutSink oo = o;
  oo.offs_stride = stride;
  oo.offs_bbits = Db;
  CopySrc nocopy{};
  TRY(launch_sortfold<MODE_RANGE>(h, SGAGG_K_RUNGEN, P<Chunk>(h->chunks[0]), info.n_chunks, 0, aos, nocopy,
                                  fd, oo, rs_dev, &ds->total));
  kbytes(h, SGAGG_K_RUNGEN, n * 8ll * W);
  kbegin(h, SGAGG_K_OTHER);
  k_run_bounds<<<(int)((B + 255) / 256), 256, 0, stream>>>(o.offs, stride, 1 << gd.fbits, (int)B, rs_dev);
  kend(h);
  CU(cudaGetLastError());
  ++h->st.one_pass;
  *done = true;
  return SGAGG_OK;
}

sgagg_status batch_runs(sgagg_t h, const RowSrc& src, long long n, long long M, const FoldDesc& fd, int S,
                        const OutSink& user, const Digit& gd, const long long* base_in, bool stage_io) {
  cudaStream_t stream = h->stream;
  const long long B = (n + M - 1) / M;
  const int nf = 1 << gd.fbits;
  const long long stride = nf + 1;
  const long long row_bytes = 8ll * (1 + S);
  long long dev_rows_cap = n;
  if (h->arena_cap >= 0) dev_rows_cap = std::min<long long>(n, h->arena_cap / row_bytes);
  TRY(grow(h, h->arena_keys, (size_t)std::max(1ll, dev_rows_cap) * 8 + kRunSlack));
  TRY(grow_cols(h, h->arena_cols, S, (size_t)std::max(1ll, dev_rows_cap) * 8 + kRunSlack));
  h->arena_keys.arena = true;
  for (auto& b : h->arena_cols) b.arena = true;
  TRY(grow(h, h->offs, (size_t)B * stride * 8));
  TRY(grow(h, h->runstarts, (size_t)(2 * (B + 1)) * 8));
  long long* rs_dev = P<long long>(h->runstarts);          // device arena cursor per batch
  long long* rs_host = rs_dev + (B + 1);                   // host arena cursor per batch
  CU(cudaMemsetAsync(rs_dev, 0, (size_t)(2 * (B + 1)) * 8, stream));
  bool any_host = false;
  std::vector<int> run_host(B, 0);
  {
    long long ub = 0;  // upper bound of device rows so far
    for (long long b = 0; b < B; ++b) {
      long long m = std::min(M, n - b * M);
      if (ub + m > dev_rows_cap) { run_host[b] = 1; any_host = true; }
      else ub += m;
    }
  }
  if (any_host) TRY(alloc_host_arena(h, (size_t)n, S));

  long long dev_cursor_idx = 0, host_cursor_idx = 0;
  // run b reads its base from the previous run of the same arena
  std::vector<long long*> base_ptr(B), end_ptr(B);
  {
    long long* last_dev = rs_dev;      // rs_dev[0] = 0
    long long* last_host = rs_host;    // rs_host[0] = 0
    for (long long b = 0; b < B; ++b) {
      if (run_host[b]) {
        base_ptr[b] = last_host;
        end_ptr[b] = rs_host + 1 + (++host_cursor_idx) - 1;
        last_host = end_ptr[b];
      } else {
        base_ptr[b] = last_dev;
        end_ptr[b] = rs_dev + 1 + (++dev_cursor_idx) - 1;
        last_dev = end_ptr[b];
      }
    }
  }
  bool one_pass = false;
  if (h->one_pass && !any_host && !stage_io && B > 1 && M > kTileCap && n <= kOnePassRows && !h->top_prefold &&
      gd.fbits - gd.ebits >= 1 && (B << (gd.fbits - gd.ebits)) <= kPlanSmallMax) {
    OutSink o{};
    o.user = 0;
    o.keys = P<unsigned long long>(h->arena_keys);
    for (int s = 0; s < S; ++s) o.cols[s] = P<long long>(h->arena_cols[s]);
    o.capacity = dev_rows_cap;
    o.offs = P<long long>(h->offs);
    o.dig = gd;
    TRY(runs_one_pass(h, src, n, M, B, fd, gd, o, stride, rs_dev, &one_pass));
  }
  if (stage_io) TRY(stage_rows(h, 0, std::min<long long>(M, n), 0));
  for (long long b = 0; b < B && !one_pass; ++b) {
    long long m = std::min(M, n - b * M);
    if (stage_io) {  // copy batch b + 1 while batch b is grouped
      if (b + 1 < B) TRY(stage_rows(h, (b + 1) * M, std::min<long long>(n, (b + 2) * M), (size_t)b + 1));
      TRY(wait_rows(h, (size_t)b));
    }
    RowSrc bs = src;
    // shift the source to the batch: offset applies to every column
    bs.offset = src.offset + b * M;
    OutSink o{};
    o.user = 0;
    if (run_host[b]) {
      o.keys = host_dev_ptr<unsigned long long>(h, h->harena_keys);
      for (int s = 0; s < S; ++s) o.cols[s] = host_dev_ptr<long long>(h, h->harena_cols[s]);
      o.capacity = (long long)h->harena_rows;
    } else {
      o.keys = P<unsigned long long>(h->arena_keys);
      for (int s = 0; s < S; ++s) o.cols[s] = P<long long>(h->arena_cols[s]);
      o.capacity = dev_rows_cap;
    }
    o.offs = P<long long>(h->offs) + b * stride;
    o.dig = gd;
    TRY(solve(h, bs, m, fd, o, base_ptr[b], end_ptr[b], &gd, 0));
  }

  // run bookkeeping (the paper's spill volume)
  std::vector<long long> rsd(2 * (B + 1));
  TRY(sync_read_checked(h, rsd.data(), rs_dev, rsd.size() * 8));
  std::vector<Run> runs(B);
  {
    long long di = 0, hi = 0;
    for (long long b = 0; b < B; ++b) {
      if (run_host[b]) {
        runs[b] = Run{rsd[(B + 1) + hi], rsd[(B + 1) + hi + 1] - rsd[(B + 1) + hi], 1};
        ++hi;
      } else {
        runs[b] = Run{rsd[di], rsd[di + 1] - rsd[di], 0};
        ++di;
      }
      h->st.run_rows += runs[b].rows;
      h->run_sizes.push_back(runs[b].rows);
      kbytes(h, SGAGG_K_RUNGEN, runs[b].rows * row_bytes);
      if (runs[b].host) h->st.run_bytes_host += runs[b].rows * row_bytes;
      else h->st.run_bytes_device += runs[b].rows * row_bytes;
    }
  }
  h->st.runs = B;

  // ---- wide merge ----
  std::vector<RunRef> rr(B);
  for (long long b2 = 0; b2 < B; ++b2) {
    RunRef& r = rr[b2];
    r.host = runs[b2].host;
    if (runs[b2].host) {
      r.keys = host_dev_ptr<long long>(h, h->harena_keys);
      for (int s = 0; s < S; ++s) r.cols[s] = host_dev_ptr<long long>(h, h->harena_cols[s]);
    } else {
      r.keys = P<long long>(h->arena_keys);
      for (int s = 0; s < S; ++s) r.cols[s] = P<long long>(h->arena_cols[s]);
    }
    r.offs = P<long long>(h->offs) + b2 * stride;
    r.rows = runs[b2].rows;
  }
  return merge_all(h, rr, S, fd, nf, stride, gd, user, base_in);
}

// Hybrid run generation (SGAGG_OPT_POLICY 2, Sec. 5.2.3): memory fraction
// 1 - f/F is an in-memory index for the lowest keys, which absorbs their rows
// without spilling; fraction f/F runs read-sort-write cycles of f/F * M rows
// over the other rows, and one wide merge folds those runs.  F is
// SGAGG_OPT_HYBRID_FANIN; f is SGAGG_OPT_HYBRID_F, or, as the paper sizes the
// fan-out of hybrid hashing, f = ceil((O - M) / (M - 1)) (page of one row)
// from the output size O estimated on the key sample, at most F.  The index
// holds the (1 - f/F) * M lowest distinct keys: the resident range ends at
// the key given by SGAGG_OPT_HYBRID_LAST, or else at the sampled distinct
// key whose estimated rank among all distinct keys is that count.  The
// resident groups lead the output (their keys are the lowest); the merged
// runs follow them.
sgagg_status hybrid_device(sgagg_t h, const RowSrc& raw, long long n, const FoldDesc& fd, int S, const OutSink& user,
                           const Digit& gd, double O_est, unsigned long long* sdist_keys, long long sdist) {
  cudaStream_t stream = h->stream;
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  const long long M = h->M;
  const int F = std::max(1, h->hybrid_fanin);
  int f = h->hybrid_f;
  if (f < 0) f = O_est <= (double)M ? 0 : (int)std::min<double>(F, std::ceil((O_est - M) / std::max(1.0, M - 1.0)));
  f = std::min(std::max(f, 0), F);
  const long long R = f < F ? (long long)((1.0 - (double)f / F) * M) : 0;
  const long long m_run = f > 0 ? std::max(1ll, (long long)((double)f / F * M)) : std::max(1ll, n);
  bool has_last = false;
  unsigned long long last = 0;
  if (R > 0) {
    if (h->hybrid_last_given) {
      has_last = true;
      last = h->hybrid_last;
    } else {
      const double q = O_est > 0 ? (double)R / O_est : 1.0;
      if (q >= 1.0) {
        has_last = true;
        last = ~0ull;
      } else {
        const long long i = (long long)(q * (double)sdist) - 1;
        if (i >= 0) {
          has_last = true;
          // the sample's i-th smallest distinct key (they are in no order)
          const long long j = std::min(i, sdist - 1);
          std::nth_element(sdist_keys, sdist_keys + j, sdist_keys + sdist);
          last = sdist_keys[j];
        }
      }
    }
  }
  h->st.hybrid_f = f;
  // split the rows by the resident range, each side in input order
  const int C = raw.ncols;
  SplitOut so{};
  for (int side = 0; side < 2; ++side) {
    TRY(grow(h, h->hsplit_keys[side], (size_t)n * 8));
    TRY(grow_cols(h, h->hsplit_cols[side], C, (size_t)n * 8));
    so.keys[side] = P<unsigned long long>(h->hsplit_keys[side]);
    for (int c = 0; c < C; ++c) so.cols[side][c] = P<long long>(h->hsplit_cols[side][c]);
  }
  const int tiles = (int)((n + kSplitTile - 1) / kSplitTile);
  TRY(grow(h, h->status, (size_t)(tiles + 2) * 8));
  CU(cudaMemsetAsync(h->status.p, 0, (size_t)(tiles + 2) * 8, stream));
  LookBack lb{};
  lb.ticket = reinterpret_cast<unsigned int*>(P<unsigned long long>(h->status));
  lb.status = P<unsigned long long>(h->status) + 2;
  lb.base_in = nullptr;
  lb.total_out = &ds->hy_rows;
  lb.err = &ds->err;
  lb.spin_limit = h->spin_limit;
  lb.n_chunks = tiles;
  kbegin(h, SGAGG_K_SCATTER);
  k_split_range<<<tiles, kSplitThreads, 0, stream>>>(raw, n, last, has_last ? 1 : 0, so, lb);
  kend(h);
  CU(cudaGetLastError());
  kbytes(h, SGAGG_K_SCATTER, n * (src_row_bytes(raw) + 8ll * (1 + C)));
  TRY(sync_read_checked(h, &hs->v[0], &ds->hy_rows, 8));
  const long long Rn = hs->v[0], Sn = n - Rn;
  RowSrc part[2];
  for (int side = 0; side < 2; ++side) {
    part[side] = RowSrc{};
    part[side].kind = SRC_SOA;
    part[side].ncols = C;
    part[side].keys = so.keys[side];
    for (int c = 0; c < C; ++c) part[side].cols[c] = so.cols[side][c];
  }
  // the index: the resident rows grouped in memory, written first
  long long Rk = 0;
  if (Rn > 0) {
    TRY(solve(h, part[0], Rn, fd, user, nullptr, &ds->hy_keys, nullptr, 0));
    TRY(sync_read_checked(h, &hs->v[0], &ds->hy_keys, 8));
    Rk = hs->v[0];
  } else {
    CU(cudaMemsetAsync(&ds->hy_keys, 0, 8, stream));
  }
  h->st.resident_rows = Rn;
  h->st.resident_keys = Rk;
  h->st.batches = Sn > 0 ? (Sn + m_run - 1) / m_run : 0;
  if (Sn == 0) {
    h->last_rows = Rk;
    h->st.out_rows = Rk;
    return SGAGG_OK;
  }
  // the other rows: runs of f/F * M rows, one wide merge after the index's groups
  TRY(batch_runs(h, part[1], Sn, m_run, fd, S, user, gd, &ds->hy_keys, false));
  h->st.batches = (Sn + m_run - 1) / m_run;
  return SGAGG_OK;
}

// The whole operation on device-resident inputs.
sgagg_status aggregate_device(sgagg_t h, const sgagg_keys* keys, const int64_t* const* payload_cols,
                              int32_t n_payload, int64_t n, const sgagg_spec* spec, void* const* out_keys,
                              int64_t* const* out_aggs, int64_t out_capacity, cudaStream_t stream,
                              const KeyOut* kout_override = nullptr) {
  h->stream = stream;
  h->have_call = true;
  h->st = sgagg_stats_t{};
  h->run_sizes.clear();
  h->scratch_bytes = 0;
  h->last_rows = 0;
  h->st.n_rows = n;
  ++h->gen;
  h->touched.clear();
  h->ntimers = 0;
  h->timers_read = true;
  h->key_bytes = 0;
  for (int c = 0; c < keys->n_cols; ++c) h->key_bytes += keys->bytes[c];
  h->spec_aggs = spec->n_aggs;
  TRY(ensure_ctx_device(h));
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  CU(cudaMemsetAsync(ds, 0, sizeof(Small), stream));

  // raw source: key columns + the payload columns the aggregates read
  RowSrc raw{};
  raw.kind = SRC_RAW;
  KeyOut kout{};
  build_keycols(keys, &raw.key, &kout, out_keys);
  std::vector<int> colmap(std::max(1, (int)n_payload), -1);
  int C = 0;
  FoldDesc fd{};
  fd.n_state = spec->n_aggs;
  for (int a = 0; a < spec->n_aggs; ++a) {
    int op = spec->aggs[a].op;
    if (op == SGAGG_COUNT) {
      fd.src[a] = -1;
      fd.op[a] = OP_SUM;
    } else {
      int c = spec->aggs[a].col;
      if (colmap[c] < 0) {
        colmap[c] = C;
        raw.cols[C] = reinterpret_cast<const long long*>(payload_cols[c]);
        ++C;
      }
      fd.src[a] = (int8_t)colmap[c];
      fd.op[a] = op == SGAGG_SUM ? OP_SUM : (op == SGAGG_MIN ? OP_MIN : OP_MAX);
    }
  }
  raw.ncols = C;
  const int S = spec->n_aggs;

  OutSink user{};
  user.user = 1;
  user.kout = kout_override ? *kout_override : kout;
  for (int a = 0; a < S; ++a) user.cols[a] = reinterpret_cast<long long*>(out_aggs[a]);
  user.capacity = out_capacity;
  user.offs = nullptr;

  if (n == 0) {
    h->last_rows = 0;
    return SGAGG_OK;
  }

  const long long M = std::min<long long>(h->M, kMaxBatch);
  const long long B = (n + M - 1) / M;
  h->st.batches = B;

  // ---- probe: sampled key range and duplicate rate ----
  int scount = (int)std::min<long long>(n, kSample);
  TRY(grow(h, h->sample, (size_t)kSample * 8));
  if (h->hio) {
    host_sample(*h->hio, raw.key, n, scount, hs->sample);
  } else {
    kbegin(h, SGAGG_K_PROBE);
    k_sample<<<std::max(1, (scount + 255) / 256), 256, 0, stream>>>(raw, n, scount, P<unsigned long long>(h->sample));
    kend(h);
    TRY(sync_read(h, hs->sample, h->sample.p, (size_t)scount * 8));
  }
  unsigned long long smin, smax;
  const long long sdist = sample_distinct(h, hs->sample, scount, &smin, &smax);
  // the streaming fold of few keys searches them in order
  if (sdist <= kLowCardKeys) std::sort(hs->sample, hs->sample + sdist);
  h->top_prefold = n > kTileCap && want_prefold(h, scount, sdist);

  // ---- global partitioning digit ----
  const long long mb = std::min<long long>(M, n);
  int Db = 0;
  if (mb > kTileCap) Db = std::min(kMaxCoarseBits, std::max(1, ilog2_ceil((mb + kBucketRows - 1) / kBucketRows)));
  if (h->radix_bits > 0 && mb > kTileCap) Db = std::min(kMaxCoarseBits, h->radix_bits);
  int Fb = Db;
  if (B > 1) Fb = std::max(Db, std::min(22, ilog2_ceil((n + kMergeFineRows - 1) / kMergeFineRows)));
  int L = bitlen(smax - smin);
  Digit gd{};
  gd.base = smin;
  gd.fbits = std::min(Fb, L);
  gd.fshift = L - gd.fbits;
  gd.ebits = std::max(0, gd.fbits - Db);

  if (h->hio && (h->policy != 0 || B == 1)) {  // host buffers: the whole input first
    TRY(stage_rows(h, 0, n, 0));
    TRY(wait_rows(h, 0));
  }
  if (h->policy == 1) {
    // absorbing index: the digit's fine buckets index the index, the
    // batches and the runs (sized by n, as for several batches)
    Digit ad = gd;
    const int afb = std::max(Db, std::min(22, ilog2_ceil((n + kMergeFineRows - 1) / kMergeFineRows)));
    ad.fbits = std::min(afb, L);
    ad.fshift = L - ad.fbits;
    ad.ebits = std::max(0, ad.fbits - Db);
    return absorb_device(h, raw, n, fd, S, user, ad);
  }
  if (h->policy == 2) {
    Digit hd = gd;  // runs of the spilled rows: fine buckets sized by n
    const int hfb = std::max(Db, std::min(22, ilog2_ceil((n + kMergeFineRows - 1) / kMergeFineRows)));
    hd.fbits = std::min(hfb, L);
    hd.fshift = L - hd.fbits;
    hd.ebits = std::max(0, hd.fbits - Db);
    const double O_est = std::min<double>((double)n, estimate_domain((double)scount, (double)sdist));
    return hybrid_device(h, raw, n, fd, S, user, hd, O_est, hs->sample, sdist);
  }

  if (B == 1 && sdist <= kLowCardKeys && n >= kLowCardMinRows && h->lowcard != 0 &&
      sdist * std::max(1, S) <= kLowCardMaxSlots && raw.ncols <= kMaxCols) {
    bool done = false;
    TRY(lowcard_device(h, raw, n, fd, hs->sample, (int)sdist, user, &done));
    if (done) return SGAGG_OK;
    ++h->st.split_segments;  // the sample missed a key: the general path regroups the input
  }
  if (B == 1) {
    long long* tot = &ds->total;
    TRY(solve(h, raw, n, fd, user, nullptr, tot, &gd, 0));
    TRY(sync_read_checked(h, &hs->v[0], tot, 8));
    h->last_rows = hs->v[0];
    h->st.out_rows = h->last_rows;
    kbytes(h, SGAGG_K_RUNGEN, h->last_rows * (h->key_bytes + 8ll * S));
    return SGAGG_OK;
  }

  return batch_runs(h, raw, n, M, fd, S, user, gd, nullptr, h->hio != nullptr);
}

}  // namespace

// ===========================================================================
// Batched call: many independent instances as one grouping on the composite
// normalized key (instance, key) -- instance id in the bits above the widest
// key.  Three steps, whatever the instance count:
//   1. one launch pre-aggregates instance-aligned tiles (a tile never spans
//      two instances) straight from every instance's columns;
//   2. the partial-aggregate rows are grouped by the ordinary path (partition,
//      chunk sort+fold; several batches and a wide merge when they are many);
//   3. one launch copies each instance's rows -- contiguous, since the output
//      is sorted by instance first -- into that instance's outputs.
// Composite keys need key bits + instance bits <= 64; beyond that the
// instances are grouped one by one.
// ===========================================================================
namespace {

// adds the CUDA-event times of the call's launches to the class totals
// (the call's stream must have completed)
void read_timers(sgagg_t h) {
  if (h->timers_read) return;
  for (int i = 0; i < h->ntimers; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->timers[i].a, h->timers[i].b) == cudaSuccess)
      h->st.class_ms[h->timers[i].cls] += ms;
  }
  h->timers_read = true;
}

sgagg_status aggregate_batched(sgagg_t h, const sgagg_instance* inst, int32_t count, const sgagg_spec* spec,
                               cudaStream_t stream) {
  if (count < 0 || (count > 0 && !inst) || !spec) return fail(h, SGAGG_EINVAL, "bad batched arguments");
  if (spec->n_aggs < 0 || spec->n_aggs > kMaxCols || (spec->n_aggs > 0 && !spec->aggs))
    return fail(h, SGAGG_EINVAL, "bad aggregate spec");
  int maxkb = 1, maxcol = -1, bigkb = 1;  // bigkb: widest key of the instances above one chunk
  long long total = 0;
  for (int i = 0; i < count; ++i) {
    const sgagg_instance& d = inst[i];
    const int kb = d.key_bytes;
    if (kb != 1 && kb != 2 && kb != 4 && kb != 8) return fail(h, SGAGG_EINVAL, "instance key width must be 1, 2, 4 or 8");
    if (d.n < 0 || d.out_capacity < 0 || !d.out_rows) return fail(h, SGAGG_EINVAL, "bad instance sizes or null out_rows");
    if (d.n > 0 && !d.keys) return fail(h, SGAGG_EINVAL, "null instance keys");
    if (d.n_payload < 0 || d.n_payload > 1024) return fail(h, SGAGG_EINVAL, "bad instance payload count");
    maxkb = std::max(maxkb, kb);
    if (d.n > kTileCap) bigkb = std::max(bigkb, kb);
    total += d.n;
  }
  for (int a = 0; a < spec->n_aggs; ++a) {
    const int op = spec->aggs[a].op;
    if (op < SGAGG_COUNT || op > SGAGG_MAX) return fail(h, SGAGG_EINVAL, "bad aggregate op");
    if (op != SGAGG_COUNT) {
      maxcol = std::max(maxcol, (int)spec->aggs[a].col);
      if (spec->aggs[a].col < 0) return fail(h, SGAGG_EINVAL, "aggregate column out of range");
    }
  }
  for (int i = 0; i < count; ++i)
    if (maxcol >= inst[i].n_payload || (maxcol >= 0 && inst[i].n > 0 && !inst[i].payload))
      return fail(h, SGAGG_EINVAL, "aggregate column out of range for an instance");
  const int S = spec->n_aggs;
  const int key_bits = 8 * bigkb;  // one-chunk instances never use the composite key
  const int inst_bits = std::max(1, ilog2_ceil(std::max(1, count)));  // >= 1: key_bits stays below 64
  h->stream = stream;
  h->have_call = true;
  h->st = sgagg_stats_t{};
  h->run_sizes.clear();
  h->st.n_rows = total;
  ++h->gen;
  h->touched.clear();
  h->ntimers = 0;
  h->timers_read = true;
  h->key_bytes = maxkb;
  h->spec_aggs = S;
  h->last_rows = 0;
  TRY(ensure_ctx_device(h));
  Small* ds = dsmall(h);
  HostSmall* hs = hsmall(h);
  CU(cudaMemsetAsync(ds, 0, sizeof(Small), stream));
  if (count == 0) return SGAGG_OK;

  // instance table (all instances); groups of consecutive instances of at
  // most h->batch_group_rows rows bound the scratch
  TRY(grow(h, h->binst, (size_t)count * sizeof(InstDesc)));
  TRY(grow(h, h->bseg, (size_t)count * sizeof(SegEntry)));
  TRY(grow(h, h->brange, (size_t)count * 16));
  TRY(grow(h, h->bstartb, (size_t)(count + 1) * 8));
  std::vector<SegEntry> seg(count);
  std::vector<unsigned long long> rng((size_t)count * 2);
  std::vector<long long> cnt1((size_t)count + 1);
  unsigned long long* kmin_d = P<unsigned long long>(h->brange);
  unsigned long long* kmax_d = kmin_d + count;
  CU(cudaMemsetAsync(kmin_d, 0xFF, (size_t)count * 8, stream));
  CU(cudaMemsetAsync(kmax_d, 0, (size_t)count * 8, stream));
  static_assert(sizeof(InstDesc) == sizeof(sgagg_instance), "instance layouts differ");
  CU(cudaMemcpyAsync(h->binst.p, inst, (size_t)count * sizeof(InstDesc), cudaMemcpyHostToDevice, stream));
  InstSet is{};
  is.inst = P<InstDesc>(h->binst);
  is.key_bits = key_bits;
  is.kmin = kmin_d;
  is.kmax = kmax_d;
  is.grouped = h->prefold_bins;
  FoldDesc fd{};
  fd.n_state = S;
  int colmap[1024];
  for (int c = 0; c < 1024; ++c) colmap[c] = -1;
  int C = 0;
  for (int a = 0; a < S; ++a) {
    const int op = spec->aggs[a].op;
    if (op == SGAGG_COUNT) {
      fd.src[a] = -1;
      fd.op[a] = OP_SUM;
    } else {
      const int c = spec->aggs[a].col;
      if (colmap[c] < 0) {
        colmap[c] = C;
        is.colsel[C] = (int8_t)c;
        ++C;
      }
      fd.src[a] = (int8_t)colmap[c];
      fd.op[a] = op == SGAGG_SUM ? OP_SUM : (op == SGAGG_MIN ? OP_MIN : OP_MAX);
    }
  }
  RowSrc raw{};
  raw.kind = SRC_RAW;
  raw.ncols = C;
  const FoldDesc fid = identity_fold(fd);
  long long rows_all = 0;

  // 1. instances of at most one chunk: one launch, a CTA each, written
  //    straight to their own outputs (any key width)
  {
    std::vector<Chunk> dch;
    for (int i = 0; i < count; ++i)
      if (inst[i].n <= kTileCap) {
        Chunk c{};
        c.lo = 0;
        c.hi = inst[i].n;
        c.kind = CH_NORMAL;
        c.pad = i;
        dch.push_back(c);
      }
    if (!dch.empty()) {
      TRY(grow(h, h->bdirect, dch.size() * sizeof(Chunk)));
      CU(cudaMemcpyAsync(h->bdirect.p, dch.data(), dch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, stream));
      OutSink o{};
      o.rows_sum = reinterpret_cast<unsigned long long*>(&ds->dsum);
      CopySrc nocopy{};
      TRY(launch_sortfold<MODE_DIRECT>(h, SGAGG_K_RUNGEN, P<Chunk>(h->bdirect), (int)dch.size(), 0, raw,
                                       nocopy, fd, o, nullptr, nullptr, 0, is));
      long long dn = 0;
      for (const Chunk& c : dch) dn += c.hi;
      kbytes(h, SGAGG_K_RUNGEN, dn * (maxkb + 8ll * C));
      TRY(sync_read_checked(h, &hs->v[2], &ds->dsum, 8));
      rows_all += hs->v[2];
      kbytes(h, SGAGG_K_RUNGEN, hs->v[2] * (maxkb + 8ll * S));
    }
  }
  if (key_bits + inst_bits > 64) {
    // composite key too wide: the bigger instances one at a time through
    // the ordinary path; the counters of the calls are added
    read_timers(h);
    sgagg_stats_t acc = h->st;
    for (int i = 0; i < count; ++i) {
      const sgagg_instance& d = inst[i];
      if (d.n <= kTileCap) continue;
      std::vector<const int64_t*> pay(std::max(1, d.n_payload), nullptr);
      std::vector<int64_t*> oa(std::max(1, S), nullptr);
      if (d.n_payload > 0) TRY(sync_read(h, pay.data(), d.payload, (size_t)d.n_payload * 8));
      if (S > 0) TRY(sync_read(h, oa.data(), d.out_aggs, (size_t)S * 8));
      int32_t kb = d.key_bytes;
      const void* kc = d.keys;
      sgagg_keys k{1, &kb, &kc};
      void* ok = d.out_keys;
      sgagg_status st = aggregate_device(h, &k, pay.data(), d.n_payload, d.n, spec, &ok, oa.data(),
                                         d.out_capacity, stream);
      long long r = st == SGAGG_OK ? h->last_rows : -1;
      if (st != SGAGG_OK && st != SGAGG_ECAPACITY) return st;
      CU(cudaMemcpyAsync(d.out_rows, &r, 8, cudaMemcpyHostToDevice, stream));
      CU(cudaStreamSynchronize(stream));
      rows_all += std::max(0ll, r);
      read_timers(h);
      const sgagg_stats_t& c = h->st;
      acc.batches += c.batches; acc.runs += c.runs; acc.run_rows += c.run_rows;
      acc.run_bytes_device += c.run_bytes_device; acc.run_bytes_host += c.run_bytes_host;
      acc.out_rows += c.out_rows; acc.prefold_passes += c.prefold_passes;
      acc.split_segments += c.split_segments; acc.merge_tiles += c.merge_tiles;
      acc.kernel_launches += c.kernel_launches;
      for (int k = 0; k < kClasses; ++k) {
        acc.class_launches[k] += c.class_launches[k];
        acc.class_bytes[k] += c.class_bytes[k];
        acc.class_ms[k] += c.class_ms[k];
      }
    }
    acc.n_rows = total;
    acc.out_rows = rows_all;
    h->st = acc;
    h->key_bytes = maxkb;
    h->last_rows = rows_all;
    return SGAGG_OK;
  }

  int i0 = 0;
  while (i0 < count) {
    int i1 = i0;
    long long grows = 0;
    auto big_rows = [&](int i) { return inst[i].n > kTileCap ? inst[i].n : 0ll; };
    while (i1 < count && (i1 == i0 || grows + big_rows(i1) <= h->batch_group_rows)) grows += big_rows(i1++);
    if (grows == 0) {  // only instances of the direct launch
      i0 = i1;
      continue;
    }
    std::vector<Chunk> tiles;
    for (int i = i0; i < i1; ++i)
      for (long long lo = 0; inst[i].n > kTileCap && lo < inst[i].n; lo += h->prefold_rows) {
        Chunk c{};
        c.lo = lo;
        c.hi = std::min<long long>(inst[i].n, lo + h->prefold_rows);
        c.kind = CH_NORMAL;
        c.pad = i;
        tiles.push_back(c);
      }
    const long long ntiles = (long long)tiles.size();
    TRY(grow(h, h->bchunks, (size_t)std::max(1ll, ntiles) * sizeof(Chunk)));
    if (ntiles)
      CU(cudaMemcpyAsync(h->bchunks.p, tiles.data(), tiles.size() * sizeof(Chunk), cudaMemcpyHostToDevice, stream));
    // 1. tile pre-aggregation over the group's instances
    TRY(grow(h, h->bkeys, (size_t)std::max(1ll, grows) * 8));
    TRY(grow_cols(h, h->bcols, S, (size_t)std::max(1ll, grows) * 8));
    OutSink o{};
    o.user = 0;
    o.keys = P<unsigned long long>(h->bkeys);
    for (int a = 0; a < S; ++a) o.cols[a] = P<long long>(h->bcols[a]);
    o.capacity = grows;
    CopySrc nocopy{};
    long long n1 = 0;
    if (ntiles) {
      TRY(launch_sortfold<MODE_INST>(h, SGAGG_K_PREFOLD, P<Chunk>(h->bchunks), (int)ntiles, 0, raw, nocopy,
                                     fd, o, nullptr, &ds->pftot, 0, is));
      TRY(sync_read_checked(h, &hs->v[0], &ds->pftot, 8));
      n1 = hs->v[0];
    }
    ++h->st.prefold_passes;
    kbytes(h, SGAGG_K_PREFOLD, grows * (maxkb + 8ll * C) + n1 * 8ll * (1 + S));
    // 2. group the partial rows on (instance, key)
    RowSrc part{};
    part.kind = SRC_SOA;
    part.ncols = S;
    part.keys = P<unsigned long long>(h->bkeys);
    for (int a = 0; a < S; ++a) part.cols[a] = P<long long>(h->bcols[a]);
    TRY(grow(h, h->bout_keys, (size_t)std::max(1ll, n1) * 8));
    TRY(grow_cols(h, h->bout_cols, S, (size_t)std::max(1ll, n1) * 8));
    OutSink g{};
    g.user = 0;
    g.keys = P<unsigned long long>(h->bout_keys);
    for (int a = 0; a < S; ++a) g.cols[a] = P<long long>(h->bout_cols[a]);
    g.capacity = n1;
    long long rows = 0;
    Digit sdig{};
    if (n1 > kTileCap) {
      // segmented digit: every instance gets buckets in proportion to its
      // partial rows over its own key range
      const int gi = i1 - i0;
      kbegin(h, SGAGG_K_PROBE);
      k_inst_bounds<<<(gi + 256) / 256, 256, 0, stream>>>(P<unsigned long long>(h->bkeys), n1, P<InstDesc>(h->binst),
                                                          key_bits, i0, gi, P<long long>(h->bstartb), 0,
                                                          kTileCap);
      kend(h);
      TRY(sync_read(h, cnt1.data(), h->bstartb.p, (size_t)(gi + 1) * 8));
      TRY(sync_read(h, rng.data(), kmin_d + i0, (size_t)gi * 8));
      TRY(sync_read(h, rng.data() + count, kmax_d + i0, (size_t)gi * 8));
      int Db = 0;
      for (long long per = kBucketRows;; per *= 2) {
        long long tot = 0;
        for (int j = 0; j < gi; ++j) {
          const long long m = cnt1[j + 1] - cnt1[j];
          SegEntry e{};
          e.base = (unsigned)tot;
          if (m > 0) {
            const unsigned long long lo = rng[j], hi = rng[count + j];
            const unsigned long long range = hi - lo;
            const long long F = std::min(1ll << 20, std::max(1ll, m / per));
            int sh = range < (unsigned long long)F ? 0 : bitlen(range) - (bitlen((unsigned long long)F) - 1);
            sh = std::max(0, sh);
            const long long span = (long long)(range >> sh);  // buckets - 1, below F
            e.kmin = lo;
            e.info = (unsigned)sh | ((unsigned)span << 8);
            tot += span + 1;
          }
          seg[i0 + j] = e;
        }
        Db = std::max(1, ilog2_ceil(tot));
        if (Db <= kMaxCoarseBits) break;
      }
      CU(cudaMemcpyAsync(P<SegEntry>(h->bseg) + i0, seg.data() + i0, (size_t)gi * sizeof(SegEntry),
                         cudaMemcpyHostToDevice, stream));
      sdig.fbits = Db;
      sdig.seg = P<SegEntry>(h->bseg);
      sdig.seg_shift = key_bits;
      sdig.seg_n = count;
    }
    if (n1 > 0) {
      h->top_prefold = false;
      if (n1 > kTileCap) {
        int cnt = (int)std::min<long long>(n1, 4096);
        TRY(grow(h, h->sample, (size_t)kSample * 8));
        kbegin(h, SGAGG_K_PROBE);
        k_sample<<<std::max(1, (cnt + 255) / 256), 256, 0, stream>>>(part, n1, cnt, P<unsigned long long>(h->sample));
        kend(h);
        TRY(sync_read(h, hs->sample, h->sample.p, (size_t)cnt * 8));
        unsigned long long mn, mx;
        const long long dist = sample_distinct(h, hs->sample, cnt, &mn, &mx);
        h->top_prefold = want_prefold(h, cnt, dist);
      }
      CU(cudaMemsetAsync(&ds->total, 0, 8, stream));
      TRY(solve(h, part, n1, fid, g, nullptr, &ds->total, sdig.seg ? &sdig : nullptr, 0));
      TRY(sync_read_checked(h, &hs->v[1], &ds->total, 8));
      rows = hs->v[1];
    }
    // 3. every instance's rows to its outputs
    CopySrc gs{};
    gs.keys = g.keys;
    for (int a = 0; a < S; ++a) gs.cols[a] = g.cols[a];
    kbegin(h, SGAGG_K_OTHER);
    k_inst_bounds<<<(i1 - i0 + 256) / 256, 256, 0, stream>>>(g.keys, rows, P<InstDesc>(h->binst), key_bits, i0,
                                                             i1 - i0, P<long long>(h->bstartb), 1, kTileCap);
    if (rows > 0)
      k_distribute<<<(int)((rows + kDistRows - 1) / kDistRows), 256, 0, stream>>>(
          g.keys, gs, rows, S, P<InstDesc>(h->binst), key_bits, i0, i1 - i0, P<long long>(h->bstartb));
    kend(h);
    if (rows > 0) {
      ++h->st.class_launches[SGAGG_K_OTHER];
      ++h->st.kernel_launches;
    }
    kbytes(h, SGAGG_K_OTHER, rows * (8ll * (1 + S) + maxkb + 8ll * S));
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(stream));  // the group's scratch is reused by the next group
    rows_all += rows;
    i0 = i1;
  }
  const long long rows = rows_all;
  h->last_rows = rows;
  h->st.out_rows = rows;
  return SGAGG_OK;
}

}  // namespace

// ===========================================================================
// Grouping without allocation (sgagg_aggregate_noalloc).
//
// One chunk of at most kTileCap rows is sorted and folded by the same kernel
// as every other chunk; its look-back status, ticket, error word and row
// count live in this fixed array instead of handle-owned buffers.  Host code
// must not pass the symbol itself to a kernel (on the host it names a
// stand-in, not device memory): the device address is looked up once per
// device with cudaGetSymbolAddress.
// ===========================================================================
static __device__ __align__(256) unsigned char g_noalloc_scratch[SGAGG_NOALLOC_SCRATCH_BYTES];

namespace {

// byte offsets inside g_noalloc_scratch
constexpr int kNaTicket = 0, kNaStatus = 8, kNaErr = 16, kNaTotal = 24, kNaZeroBytes = 24;

constexpr int kNaMaxDevices = 64;
std::atomic<unsigned char*> g_na_ptr[kNaMaxDevices];   // device address of the array, per device
thread_local char g_na_msg[256];

__global__ void k_noalloc_finish(const int* err, const long long* total, long long* out_rows) {
  *out_rows = *err ? -1 : *total;
}

sgagg_status na_fail(sgagg_status st, const char* msg) {
  snprintf(g_na_msg, sizeof g_na_msg, "%s", msg);
  return st;
}

}  // namespace

extern "C" sgagg_status sgagg_aggregate_noalloc(const sgagg_keys* keys, const int64_t* const* payload_cols,
                                                int32_t n_payload, int64_t n, const sgagg_spec* spec,
                                                void* const* out_keys, int64_t* const* out_aggs,
                                                int64_t out_capacity, int64_t* out_rows, void* stream) {
  g_na_msg[0] = 0;
  if (n > SGAGG_NOALLOC_MAX_ROWS)
    return na_fail(SGAGG_EINVAL, "sgagg_aggregate_noalloc: n exceeds SGAGG_NOALLOC_MAX_ROWS (8192)");
  if (!out_rows) return na_fail(SGAGG_EINVAL, "sgagg_aggregate_noalloc: null out_rows");
  const char* msg = "";
  sgagg_status vs = check_args(keys, payload_cols, n_payload, n, spec, out_keys, out_aggs, out_capacity, &msg);
  if (vs != SGAGG_OK) return na_fail(vs, msg);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
    return na_fail(SGAGG_ECUDA, "sgagg_aggregate_noalloc: no usable current device");
  if (!g_na_ptr[dev].load(std::memory_order_acquire)) {
    // set-up, once per device: the array's device address, and every kernel
    // this entry point launches loaded now (with lazy module loading a
    // kernel's first launch may load its module, which allocates), with its
    // shared-memory limit set
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return na_fail(SGAGG_ECUDA, cudaGetErrorString(e));
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_noalloc_finish);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sortfold<MODE_TILES, 2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sortfold<MODE_TILES, 4>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sortfold<MODE_TILES, 8>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sortfold<MODE_TILES, 16>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_sortfold<MODE_TILES, 32>);
    if (e != cudaSuccess) return na_fail(SGAGG_ECUDA, cudaGetErrorString(e));
    set_smem_attr<MODE_TILES, 2>();
    set_smem_attr<MODE_TILES, 4>();
    set_smem_attr<MODE_TILES, 8>();
    set_smem_attr<MODE_TILES, 16>();
    set_smem_attr<MODE_TILES, 32>();
    g_na_ptr[dev].store(reinterpret_cast<unsigned char*>(p), std::memory_order_release);
  }
  unsigned char* base = g_na_ptr[dev].load(std::memory_order_acquire);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // ticket, status word and error word must start at zero; the count is written
  if (cudaMemsetAsync(base, 0, kNaZeroBytes, st) != cudaSuccess)
    return na_fail(SGAGG_ECUDA, "sgagg_aggregate_noalloc: cudaMemsetAsync failed");
  if (n == 0) {
    if (cudaMemsetAsync(base + kNaTotal, 0, 8, st) != cudaSuccess)
      return na_fail(SGAGG_ECUDA, "sgagg_aggregate_noalloc: cudaMemsetAsync failed");
  } else {
    RowSrc raw{};
    raw.kind = SRC_RAW;
    KeyOut kout{};
    build_keycols(keys, &raw.key, &kout, out_keys);
    FoldDesc fd{};
    fd.n_state = spec->n_aggs;
    int colmap[1024];
    for (int c = 0; c < n_payload && c < 1024; ++c) colmap[c] = -1;
    int C = 0;
    for (int a = 0; a < spec->n_aggs; ++a) {
      const int op = spec->aggs[a].op;
      if (op == SGAGG_COUNT) {
        fd.src[a] = -1;
        fd.op[a] = OP_SUM;
      } else {
        const int c = spec->aggs[a].col;
        if (colmap[c] < 0) {
          if (C >= kMaxCols) return na_fail(SGAGG_EINVAL, "sgagg_aggregate_noalloc: too many payload columns");
          colmap[c] = C;
          raw.cols[C++] = reinterpret_cast<const long long*>(payload_cols[c]);
        }
        fd.src[a] = (int8_t)colmap[c];
        fd.op[a] = op == SGAGG_SUM ? OP_SUM : (op == SGAGG_MIN ? OP_MIN : OP_MAX);
      }
    }
    raw.ncols = C;
    OutSink o{};
    o.user = 1;
    o.kout = kout;
    for (int a = 0; a < spec->n_aggs; ++a) o.cols[a] = reinterpret_cast<long long*>(out_aggs[a]);
    o.capacity = out_capacity;
    LookBack lb{};
    lb.ticket = reinterpret_cast<unsigned int*>(base + kNaTicket);
    lb.status = reinterpret_cast<unsigned long long*>(base + kNaStatus);
    lb.err = reinterpret_cast<int*>(base + kNaErr);
    lb.total_out = reinterpret_cast<long long*>(base + kNaTotal);
    lb.base_in = nullptr;
    lb.spin_limit = 1ll << 26;
    lb.n_chunks = 1;
    CopySrc nocopy{};
    if (fd.n_state <= 2)
      launch_ks<MODE_TILES, 2>(1, st, nullptr, raw, nocopy, fd, o, lb, n, 0);
    else if (fd.n_state <= 4)
      launch_ks<MODE_TILES, 4>(1, st, nullptr, raw, nocopy, fd, o, lb, n, 0);
    else if (fd.n_state <= 8)
      launch_ks<MODE_TILES, 8>(1, st, nullptr, raw, nocopy, fd, o, lb, n, 0);
    else if (fd.n_state <= 16)
      launch_ks<MODE_TILES, 16>(1, st, nullptr, raw, nocopy, fd, o, lb, n, 0);
    else
      launch_ks<MODE_TILES, 32>(1, st, nullptr, raw, nocopy, fd, o, lb, n, 0);
    if (cudaGetLastError() != cudaSuccess) return na_fail(SGAGG_ECUDA, "sgagg_aggregate_noalloc: launch failed");
  }
  k_noalloc_finish<<<1, 1, 0, st>>>(reinterpret_cast<const int*>(base + kNaErr),
                                    reinterpret_cast<const long long*>(base + kNaTotal),
                                    reinterpret_cast<long long*>(out_rows));
  if (cudaGetLastError() != cudaSuccess) return na_fail(SGAGG_ECUDA, "sgagg_aggregate_noalloc: launch failed");
  return SGAGG_OK;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

sgagg_status sgagg_create(int64_t memory_budget_rows, sgagg_t* out) {
  if (!out || memory_budget_rows < 1) return SGAGG_EINVAL;
  sgagg_t h = new (std::nothrow) sgagg_ctx();
  if (!h) return SGAGG_ENOMEM;
  h->M = memory_budget_rows;
  *out = h;
  return SGAGG_OK;
}

sgagg_status sgagg_set_option(sgagg_t h, int32_t key, int64_t value) {
  if (!h) return SGAGG_EINVAL;
  switch (key) {
    case SGAGG_OPT_PREFOLD:
      if (value < -1 || value > 1) return fail(h, SGAGG_EINVAL, "prefold must be -1, 0 or 1");
      h->prefold_opt = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_ARENA_CAP: h->arena_cap = value; return SGAGG_OK;
    case SGAGG_OPT_RADIX_BITS:
      if (value < 0 || value > 15) return fail(h, SGAGG_EINVAL, "radix bits must be 0..15");
      h->radix_bits = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_SPIN_LIMIT:
      if (value < 1) return fail(h, SGAGG_EINVAL, "spin limit must be >= 1");
      h->spin_limit = value;
      return SGAGG_OK;
    case SGAGG_OPT_FANIN_CAP:
      if (value < 0) return fail(h, SGAGG_EINVAL, "fan-in cap must be >= 0");
      h->fanin_cap = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_FAULT_ALLOC:
      h->fault_alloc = (int)value;
      h->alloc_count = 0;
      return SGAGG_OK;
    case SGAGG_OPT_TIMING: h->timing = (int)value; return SGAGG_OK;
    case SGAGG_OPT_TEST_STALL: h->test_stall = value == 2 ? 2 : (value ? 1 : 0); return SGAGG_OK;
    case SGAGG_OPT_POLICY:
      if (value < 0 || value > 2) return fail(h, SGAGG_EINVAL, "policy must be 0, 1 or 2");
      h->policy = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_ABSORB_BATCH:
      if (value < 0) return fail(h, SGAGG_EINVAL, "absorbing batch must be >= 0");
      h->absorb_batch = value;
      return SGAGG_OK;
    case SGAGG_OPT_LOWCARD:
      h->lowcard = value == 0 ? 0 : -1;
      return SGAGG_OK;
    case SGAGG_OPT_HYBRID_FANIN:
      if (value < 1) return fail(h, SGAGG_EINVAL, "hybrid fan-in must be >= 1");
      h->hybrid_fanin = (int)std::min<int64_t>(value, 1 << 20);
      return SGAGG_OK;
    case SGAGG_OPT_HYBRID_F:
      h->hybrid_f = value < 0 ? -1 : (int)std::min<int64_t>(value, 1 << 20);
      return SGAGG_OK;
    case SGAGG_OPT_HYBRID_LAST:
      h->hybrid_last_given = true;
      h->hybrid_last = (unsigned long long)value;
      return SGAGG_OK;
    case SGAGG_OPT_HYBRID_LAST_AUTO:
      h->hybrid_last_given = false;
      return SGAGG_OK;
    case SGAGG_OPT_MERGE_COPY:
      h->merge_copy = (value == 1 || value == 2) ? (int)value : 0;
      return SGAGG_OK;
    case SGAGG_OPT_MERGE_THREADS:
      if (value != 0 && value != 256) return fail(h, SGAGG_EINVAL, "merge threads must be 0 or 256");
      h->merge_threads = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_PREFOLD_BINS:
      if (value != 0 && value != 1) return fail(h, SGAGG_EINVAL, "prefold bins must be 0 or 1");
      h->prefold_bins = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_PREFOLD_ROWS:
      if (value < 1024 || value > kTileCap) return fail(h, SGAGG_EINVAL, "prefold rows must be 1024..8192");
      h->prefold_rows = value;
      return SGAGG_OK;
    case SGAGG_OPT_ONE_PASS:
      h->one_pass = value ? 1 : 0;
      return SGAGG_OK;
    case SGAGG_OPT_PART_LEVELS:
      if (value != 0 && value != 1) return fail(h, SGAGG_EINVAL, "partition levels must be 0 or 1");
      h->part_levels = (int)value;
      return SGAGG_OK;
    case SGAGG_OPT_BATCH_GROUP_ROWS:
      if (value < (1 << 16) || value > (1ll << 31)) return fail(h, SGAGG_EINVAL, "batch group rows must be 2^16..2^31");
      h->batch_group_rows = value;
      return SGAGG_OK;
    case SGAGG_OPT_TIMING_CLASSES:
      h->timing_mask = value;
      return SGAGG_OK;
    default: return fail(h, SGAGG_EINVAL, "unknown option");
  }
}

sgagg_status sgagg_aggregate(sgagg_t h, const sgagg_keys* keys, const int64_t* const* payload_cols,
                             int32_t n_payload, int64_t n, const sgagg_spec* spec, void* const* out_keys,
                             int64_t* const* out_aggs, int64_t out_capacity, void* stream) {
  sgagg_status s = validate(h, keys, payload_cols, n_payload, n, spec, out_keys, out_aggs, out_capacity);
  if (s != SGAGG_OK) return s;
  h->err.clear();
  s = aggregate_device(h, keys, payload_cols, n_payload, n, spec, out_keys, out_aggs, out_capacity,
                       reinterpret_cast<cudaStream_t>(stream));
  h->pending_err = (int)s;
  return s;
}

sgagg_status sgagg_aggregate_host(sgagg_t h, const sgagg_keys* keys, const int64_t* const* payload_cols,
                                  int32_t n_payload, int64_t n, const sgagg_spec* spec, void* const* out_keys,
                                  int64_t* const* out_aggs, int64_t out_capacity, int64_t* rows, void* stream) {
  sgagg_status s = validate(h, keys, payload_cols, n_payload, n, spec, out_keys, out_aggs, out_capacity);
  if (s != SGAGG_OK) return s;
  if (!rows) return fail(h, SGAGG_EINVAL, "null rows");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  h->err.clear();
  TRY(ensure_ctx_device(h));
  if (!h->copy_stream) CU(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  // device buffers for the inputs (filled batch by batch) and the output
  HostIO io;
  io.copy = h->copy_stream;
  io.nk = keys->n_cols;
  sgagg_keys dk = *keys;
  const void* dkc[kMaxKeyCols];
  for (int c = 0; c < keys->n_cols; ++c) {
    TRY(grow(h, h->in_keys[c], (size_t)std::max(1ll, (long long)n) * keys->bytes[c]));
    dkc[c] = h->in_keys[c].p;
    io.hkeys[c] = keys->cols[c];
    io.kb[c] = keys->bytes[c];
    io.dkeys[c] = h->in_keys[c].p;
  }
  dk.cols = dkc;
  if ((int)h->in_pay.size() < n_payload) h->in_pay.resize(n_payload);
  std::unique_ptr<bool[]> used(new bool[std::max(1, (int)n_payload)]());
  for (int a = 0; a < spec->n_aggs; ++a)
    if (spec->aggs[a].op != SGAGG_COUNT) used[spec->aggs[a].col] = true;
  std::vector<int64_t*> dp(std::max(1, (int)n_payload), nullptr);
  for (int c = 0; c < n_payload; ++c) {
    if (!used[c]) continue;
    TRY(grow(h, h->in_pay[c], (size_t)std::max(1ll, (long long)n) * 8));
    dp[c] = P<int64_t>(h->in_pay[c]);
  }
  io.np = n_payload;
  io.hpay = payload_cols;
  io.used = used.get();
  io.dpay = dp.data();
  long long cap = std::min<long long>(out_capacity, n);
  void* dok[kMaxKeyCols];
  for (int c = 0; c < keys->n_cols; ++c) {
    TRY(grow(h, h->out_keys[c], (size_t)std::max(1ll, cap) * keys->bytes[c]));
    dok[c] = h->out_keys[c].p;
    io.hout_keys[c] = out_keys[c];
    io.dout_keys[c] = dok[c];
  }
  if ((int)h->out_cols.size() < spec->n_aggs) h->out_cols.resize(spec->n_aggs);
  std::vector<int64_t*> doa(std::max(1, spec->n_aggs), nullptr);
  for (int a = 0; a < spec->n_aggs; ++a) {
    TRY(grow(h, h->out_cols[a], (size_t)std::max(1ll, cap) * 8));
    doa[a] = P<int64_t>(h->out_cols[a]);
  }
  io.S = spec->n_aggs;
  io.hout_aggs = out_aggs;
  io.dout_aggs = doa.data();
  io.capacity = cap;
  // the copy stream starts after the caller's earlier work on `st`
  cudaEvent_t start;
  TRY(io_event(h, 0, &start));
  CU(cudaEventRecord(start, st));
  CU(cudaStreamWaitEvent(io.copy, start, 0));
  h->hio = &io;
  std::vector<const int64_t*> dpc(dp.begin(), dp.end());
  s = aggregate_device(h, &dk, dpc.data(), n_payload, n, spec, dok, doa.data(), cap, st);
  if (s == SGAGG_OK) {
    // the rows not copied back yet (all of them unless the final merge ran in parts)
    cudaEvent_t done;
    s = io_event(h, 0, &done);
    if (s == SGAGG_OK && cudaEventRecord(done, st) != cudaSuccess) s = fail(h, SGAGG_ECUDA, "event record failed");
    if (s == SGAGG_OK) s = unstage_rows(h, io.copied_out, h->last_rows, done);
  }
  h->hio = nullptr;
  cudaError_t e1 = cudaStreamSynchronize(io.copy);
  cudaError_t e2 = cudaStreamSynchronize(st);
  h->pending_err = (int)s;
  if (s != SGAGG_OK) return s;
  if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(h, SGAGG_ECUDA, "%s", cudaGetErrorString(e1 ? e1 : e2));
  *rows = h->last_rows;
  return SGAGG_OK;
}

// count(distinct u) per g (Sec. 7, Hypothesis 6): one grouping on the
// composite key (g, u) removes duplicate pairs and leaves them sorted by g,
// then one in-stream pass regroups on g.
sgagg_status aggregate_distinct(sgagg_t h, const sgagg_keys* keys, const void* dcol, int32_t dbytes,
                                const int64_t* const* payload_cols, int32_t n_payload, int64_t n,
                                const sgagg_spec* spec, void* const* out_keys, int64_t* out_distinct,
                                int64_t* const* out_aggs, int64_t out_capacity, cudaStream_t stream) {
  if (!keys || keys->n_cols < 1 || keys->n_cols + 1 > kMaxKeyCols)
    return fail(h, SGAGG_EINVAL, "bad group key columns");
  if (dbytes != 1 && dbytes != 2 && dbytes != 4 && dbytes != 8) return fail(h, SGAGG_EINVAL, "distinct column width must be 1, 2, 4 or 8");
  if (n > 0 && !dcol) return fail(h, SGAGG_EINVAL, "null distinct column");
  if (!out_distinct) return fail(h, SGAGG_EINVAL, "null out_distinct");
  int gbytes = 0;
  for (int c = 0; c < keys->n_cols; ++c) gbytes += keys->bytes[c];
  if (gbytes + dbytes > 8) return fail(h, SGAGG_EINVAL, "group key plus distinct column wider than 8 bytes");
  int32_t cb[kMaxKeyCols];
  const void* cc[kMaxKeyCols];
  for (int c = 0; c < keys->n_cols; ++c) {
    cb[c] = keys->bytes[c];
    cc[c] = keys->cols[c];
  }
  cb[keys->n_cols] = dbytes;
  cc[keys->n_cols] = dcol;
  sgagg_keys ck{keys->n_cols + 1, cb, cc};
  const int S = spec->n_aggs;
  TRY(ensure_ctx_device(h));
  TRY(grow(h, h->dk_keys, (size_t)std::max(1ll, (long long)n) * 8));
  TRY(grow_cols(h, h->dk_cols, S, (size_t)std::max(1ll, (long long)n) * 8));
  std::vector<int64_t*> dka(std::max(1, S), nullptr);
  for (int a = 0; a < S; ++a) dka[a] = P<int64_t>(h->dk_cols[a]);
  KeyOut canon{};
  canon.n_cols = 1;
  canon.bytes[0] = 8;
  canon.shift[0] = 0;
  canon.cols[0] = h->dk_keys.p;
  // 1. group on (g, u): duplicate (g, u) pairs removed, rows sorted by g
  TRY(aggregate_device(h, &ck, payload_cols, n_payload, n, spec, nullptr, dka.data(), n, stream, &canon));
  const long long rows1 = h->last_rows;
  h->key_bytes = gbytes;
  h->last_rows = 0;
  h->st.out_rows = 0;
  if (rows1 == 0) return SGAGG_OK;
  // 2. regroup on g in one pass over the sorted rows
  const int ubits = 8 * dbytes;
  const long long nblk = (rows1 + kRegroupRows - 1) / kRegroupRows;
  TRY(grow(h, h->rg_heads, (size_t)(2 * nblk + 1) * 8));
  long long* heads = P<long long>(h->rg_heads);
  long long* base = heads + nblk;
  kbegin(h, SGAGG_K_OTHER);
  k_regroup_count<<<(unsigned)nblk, 256, 0, stream>>>(P<unsigned long long>(h->dk_keys), rows1, ubits, heads);
  k_excl_scan<<<1, kPartThreads, 0, stream>>>(heads, (int)nblk, base);
  kend(h);
  CU(cudaGetLastError());
  HostSmall* hs = hsmall(h);
  TRY(sync_read(h, &hs->v[0], base + nblk, 8));
  const long long groups = hs->v[0];
  if (groups > out_capacity)
    return fail(h, SGAGG_ECAPACITY, "out_capacity is smaller than the number of distinct keys");
  FoldDesc fd{};  // the (g, u) rows' aggregates fold like runs do: counts and sums add
  fd.n_state = S;
  for (int a = 0; a < S; ++a) {
    const int op = spec->aggs[a].op;
    fd.src[a] = (int8_t)a;
    fd.op[a] = (op == SGAGG_COUNT || op == SGAGG_SUM) ? OP_SUM : (op == SGAGG_MIN ? OP_MIN : OP_MAX);
  }
  OutSink user{};
  user.user = 1;
  KeyCols gk;
  build_keycols(keys, &gk, &user.kout, out_keys);
  for (int a = 0; a < S; ++a) user.cols[a] = reinterpret_cast<long long*>(out_aggs[a]);
  user.capacity = out_capacity;
  CopySrc states{};
  states.keys = P<unsigned long long>(h->dk_keys);
  for (int a = 0; a < S; ++a) states.cols[a] = P<long long>(h->dk_cols[a]);
  kbegin(h, SGAGG_K_OTHER);
  k_regroup_init<<<std::max(1, std::min(h->num_sms * 4, (int)((groups + 255) / 256))), 256, 0, stream>>>(
      reinterpret_cast<long long*>(out_distinct), user, fd, groups);
  k_regroup_fold<<<(unsigned)nblk, 256, 0, stream>>>(P<unsigned long long>(h->dk_keys), states, rows1, ubits, fd,
                                                    base, user, reinterpret_cast<long long*>(out_distinct));
  kend(h);
  CU(cudaGetLastError());
  h->st.class_launches[SGAGG_K_OTHER] += 2;
  h->st.kernel_launches += 2;
  kbytes(h, SGAGG_K_OTHER, rows1 * 8ll * (2 + S) + groups * (gbytes + 8ll * (1 + S)));
  h->last_rows = groups;
  h->st.out_rows = groups;
  return SGAGG_OK;
}

sgagg_status sgagg_aggregate_distinct(sgagg_t h, const sgagg_keys* keys, const void* distinct_col,
                                      int32_t distinct_bytes, const int64_t* const* payload_cols,
                                      int32_t n_payload, int64_t n, const sgagg_spec* spec, void* const* out_keys,
                                      int64_t* out_distinct, int64_t* const* out_aggs, int64_t out_capacity,
                                      void* stream) {
  sgagg_status s = validate(h, keys, payload_cols, n_payload, n, spec, out_keys, out_aggs, out_capacity);
  if (s != SGAGG_OK) return s;
  h->err.clear();
  s = aggregate_distinct(h, keys, distinct_col, distinct_bytes, payload_cols, n_payload, n, spec, out_keys,
                         out_distinct, out_aggs, out_capacity, reinterpret_cast<cudaStream_t>(stream));
  h->pending_err = (int)s;
  return s;
}

sgagg_status sgagg_result_rows(sgagg_t h, int64_t* rows) {
  if (!h || !rows) return SGAGG_EINVAL;
  if (!h->have_call) return fail(h, SGAGG_ESTATE, "no aggregate call yet");
  if (h->pending_err) return (sgagg_status)h->pending_err;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, SGAGG_ECUDA, "%s", cudaGetErrorString(e));
  *rows = h->last_rows;
  return SGAGG_OK;
}

static long long scratch_in_use(sgagg_t h) {
  long long s = 0;
  for (DevBuf* b : h->touched)
    if (b->gen == h->gen && !b->arena) s += (long long)b->used;
  return s;
}

int64_t sgagg_temp_bytes(sgagg_t h) {
  if (!h) return -1;
  return h->st.run_bytes_device + h->st.run_bytes_host + scratch_in_use(h);
}

sgagg_status sgagg_stats(sgagg_t h, sgagg_stats_t* out) {
  if (!h || !out) return SGAGG_EINVAL;
  if (h->have_call) cudaStreamSynchronize(h->stream);
  read_timers(h);
  *out = h->st;
  out->peak_scratch_bytes = scratch_in_use(h);
  out->out_bytes = h->st.out_rows * (h->key_bytes + 8ll * h->spec_aggs);
  return SGAGG_OK;
}

sgagg_status sgagg_run_sizes(sgagg_t h, int64_t* rows, int64_t max_runs, int64_t* count) {
  if (!h || !count || max_runs < 0 || (max_runs > 0 && !rows)) return SGAGG_EINVAL;
  if (h->have_call) cudaStreamSynchronize(h->stream);
  *count = (int64_t)h->run_sizes.size();
  for (int64_t i = 0; i < max_runs && i < *count; ++i) rows[i] = h->run_sizes[(size_t)i];
  return SGAGG_OK;
}

sgagg_status sgagg_aggregate_batched(sgagg_t h, const sgagg_instance* inst, int32_t count, const sgagg_spec* spec,
                                     void* stream) {
  if (!h) return SGAGG_EINVAL;
  h->err.clear();
  sgagg_status s = aggregate_batched(h, inst, count, spec, reinterpret_cast<cudaStream_t>(stream));
  h->pending_err = (int)s;
  return s;
}

void sgagg_destroy(sgagg_t h) {
  if (!h) return;
  auto fv = [](std::vector<DevBuf>& v) { for (auto& b : v) free_buf(b); };
  for (int d = 0; d <= kMaxDepth; ++d) {
    free_buf(h->scatter[d]); free_buf(h->thist[d]); free_buf(h->btot[d]); free_buf(h->bstart[d]);
    free_buf(h->chunks[d]); free_buf(h->biglist[d]); free_buf(h->copykeys[d]); fv(h->copycols[d]);
    free_buf(h->akeys[d]); free_buf(h->acolptr[d]); free_buf(h->thist1[d]); free_buf(h->btot1[d]);
    free_buf(h->bstart1[d]); free_buf(h->tiles2[d]); free_buf(h->tfirst[d]); free_buf(h->thist2[d]);
    fv(h->acols[d]);
  }
  free_buf(h->pf[0]); free_buf(h->pf[1]); fv(h->pfcols[0]); fv(h->pfcols[1]);
  free_buf(h->status); free_buf(h->small); free_buf(h->sample); free_buf(h->arena_keys); fv(h->arena_cols);
  free_buf(h->offs); free_buf(h->runptrs); free_buf(h->fsizes); free_buf(h->gather_keys); fv(h->gather_cols);
  free_buf(h->gather_ptrs); free_buf(h->runstarts);
  free_buf(h->marena_keys); fv(h->marena_cols); free_buf(h->moffs);
  for (int i = 0; i < 3; ++i) {
    free_buf(h->ab_keys[i]); free_buf(h->ab_offs[i]); fv(h->ab_cols[i]);
  }
  free_buf(h->ab_tmp);
  free_buf(h->dk_keys); free_buf(h->rg_heads); fv(h->dk_cols); free_buf(h->plan_tmp); free_buf(h->lc_part); free_buf(h->tslo); free_buf(h->tcount); free_buf(h->tbase);
  for (int i = 0; i < 2; ++i) { free_buf(h->hsplit_keys[i]); fv(h->hsplit_cols[i]); }
  free_buf(h->binst); free_buf(h->bchunks); free_buf(h->bkeys); free_buf(h->bout_keys);
  free_buf(h->bseg); free_buf(h->brange); free_buf(h->bstartb); free_buf(h->bdirect);
  fv(h->bcols); fv(h->bout_cols);
  for (auto& b : h->in_keys) free_buf(b);
  fv(h->in_pay);
  for (auto& b : h->out_keys) free_buf(b);
  fv(h->out_cols);
  if (h->harena_keys) cudaFreeHost(h->harena_keys);
  for (void* p : h->harena_cols) cudaFreeHost(p);
  if (h->hsmall) cudaFreeHost(h->hsmall);
  for (auto& t : h->timers) {
    if (t.a) cudaEventDestroy(t.a);
    if (t.b) cudaEventDestroy(t.b);
  }
  delete h;
}

const char* sgagg_last_error(sgagg_t h) {
  if (!h) return g_na_msg;
  return h->err.c_str();
}

}  // extern "C"
