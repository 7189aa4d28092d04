// sg_sortfold.cuh -- sort a chunk of rows in shared memory and fold equal
// keys (the in-cache batch sort + duplicate detection of Sec. 6.1, and the
// absorbing of equal keys from many runs in the wide merge of Sec. 4).
//
// One CTA takes one chunk (ticket order) of at most kTileCap rows:
//   1. load the chunk's keys into shared memory (a row range of one source,
//      or one slice from each of k sorted runs);
//   2. sort a permutation of the chunk by key: a counting sort on the top
//      kBinBits bits of (key - chunk min); bins are then finished by insertion
//      sort, or -- when some bin is large -- the chunk is sorted by a stable
//      LSD radix sort (8-bit digits, warp-ballot ranking) over all bits that
//      vary inside the chunk;
//   3. mark segment heads (first row of every distinct key) and number the
//      segments; the segment count is the chunk's output row count;
//   4. get the chunk's output offset by decoupled look-back;
//   5. write the distinct keys and, per aggregate, the segmented reduction of
//      its source column, staged in shared memory so every global store is
//      coalesced.
#pragma once
#include "sg_common.cuh"

namespace sg {

constexpr int kTileCap = 8192;          // rows per chunk
constexpr int kThreads = 512;
constexpr int kEPT = kTileCap / kThreads;  // rows per thread (16)
constexpr int kBinBits = 12;
constexpr int kBins = 1 << kBinBits;
constexpr int kMaxFanIn = 512;          // runs one merge chunk can read
constexpr int kWarps = kThreads / 32;

enum : int { CH_NORMAL = 0, CH_COPY = 1 };
enum : int { MODE_RANGE = 0, MODE_RUNS = 1, MODE_TILES = 2 };

struct Chunk {
  long long lo, hi;   // MODE_RANGE: source rows; CH_COPY: rows of the copy source
  int f_lo, f_hi;     // fine buckets covered (offsets of runs; MODE_RUNS slices)
  int kind;
  int pad;
};

// k sorted runs of state rows in SoA form, for the wide merge.  Run r's rows
// with fine digit in [f_lo, f_hi) are rows offs[r*stride + f_lo] ..
// offs[r*stride + f_hi] - 1 of its arrays.
struct RunSet {
  int k;
  int ncols;
  const long long* const* ptrs;   // [k * (1 + ncols)]: keys, then state columns
  const long long* offs;
  long long stride;
};

// Sorted, folded state rows to copy verbatim (key ranges solved elsewhere).
struct CopySrc {
  const unsigned long long* keys;
  const long long* cols[kMaxCols];
};

struct OutSink {
  int user;                         // 1: key columns per kout, else canonical keys
  KeyOut kout;
  unsigned long long* keys;         // canonical keys
  long long* cols[kMaxCols];        // one per state column
  long long capacity;               // rows writable (absolute positions < capacity)
  long long* offs;                  // fine-bucket offsets of the run written, or null
  Digit dig;
};

struct SortSmem {
  unsigned long long* keys;   // [kTileCap]
  long long* work;            // [kTileCap] column buffer / output staging
  uint16_t* idxA;             // [kTileCap]
  uint16_t* idxB;             // [kTileCap]
  uint32_t* bins;             // [kBins / 2] packed 16-bit counters
  long long* slo;             // [kMaxFanIn] merge: slice start per run
  long long* spre;            // [kMaxFanIn + 1] merge: slice prefix
};

constexpr size_t kSortSmemBytes =
    kTileCap * 8 * 2 + kTileCap * 2 * 2 + (kBins / 2) * 4 + kMaxFanIn * 8 + (kMaxFanIn + 1) * 8 + 64;

__device__ __forceinline__ SortSmem carve(unsigned char* base) {
  SortSmem s;
  s.keys = reinterpret_cast<unsigned long long*>(base);
  s.work = reinterpret_cast<long long*>(base + kTileCap * 8);
  s.idxA = reinterpret_cast<uint16_t*>(base + kTileCap * 16);
  s.idxB = reinterpret_cast<uint16_t*>(base + kTileCap * 18);
  s.bins = reinterpret_cast<uint32_t*>(base + kTileCap * 20);
  s.slo = reinterpret_cast<long long*>(base + kTileCap * 20 + (kBins / 2) * 4);
  s.spre = s.slo + kMaxFanIn;
  return s;
}

// ---------------------------------------------------------------------------
// Block-wide helpers (kThreads threads).
// ---------------------------------------------------------------------------
__shared__ long long g_red[kWarps + 1];
__shared__ unsigned long long g_redu[2 * kWarps + 2];

// Exclusive sum over threads; returns the thread's exclusive prefix, *total.
__device__ __forceinline__ int block_excl_sum(int v, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) g_red[w] = x;
  __syncthreads();
  if (w == 0) {
    long long s = lane < kWarps ? g_red[lane] : 0;
    long long t = s;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) g_red[lane] = t - s;
    if (lane == kWarps - 1) g_red[kWarps] = t;
  }
  __syncthreads();
  int r = (int)g_red[w] + x - v;
  *total = (int)g_red[kWarps];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void block_minmax(unsigned long long vmin, unsigned long long vmax,
                                             unsigned long long* omin, unsigned long long* omax) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long a = __shfl_xor_sync(0xffffffffu, vmin, o);
    unsigned long long b = __shfl_xor_sync(0xffffffffu, vmax, o);
    vmin = a < vmin ? a : vmin;
    vmax = b > vmax ? b : vmax;
  }
  __syncthreads();
  if (lane == 0) { g_redu[w] = vmin; g_redu[kWarps + w] = vmax; }
  __syncthreads();
  if (w == 0) {
    unsigned long long a = lane < kWarps ? g_redu[lane] : ~0ull;
    unsigned long long b = lane < kWarps ? g_redu[kWarps + lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long x = __shfl_xor_sync(0xffffffffu, a, o);
      unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
      a = x < a ? x : a;
      b = y > b ? y : b;
    }
    if (lane == 0) { g_redu[2 * kWarps] = a; g_redu[2 * kWarps + 1] = b; }
  }
  __syncthreads();
  *omin = g_redu[2 * kWarps];
  *omax = g_redu[2 * kWarps + 1];
  __syncthreads();
}

__device__ __forceinline__ int block_max_int(int v) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) g_red[w] = v;
  __syncthreads();
  if (w == 0) {
    long long a = lane < kWarps ? g_red[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (lane == 0) g_red[kWarps] = a;
  }
  __syncthreads();
  int r = (int)g_red[kWarps];
  __syncthreads();
  return r;
}

// Inclusive segmented scan over threads of (flag, value): a set flag starts a
// new segment.  Returns the exclusive result (the combined value of the
// thread's segment over all earlier threads), valid when the earlier threads
// carry part of that segment.
__device__ __forceinline__ long long block_seg_carry(int op, bool flag, long long val) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  bool f = flag;
  long long a = val;
  for (int o = 1; o < 32; o <<= 1) {
    long long ya = __shfl_up_sync(0xffffffffu, a, o);
    int yf = __shfl_up_sync(0xffffffffu, (int)f, o);
    if (lane >= o) {
      if (!f) a = op_combine(op, ya, a);
      f = f || yf;
    }
  }
  // a, f: inclusive within the warp
  __syncthreads();
  if (lane == 31) { g_red[w] = a; g_redu[w] = f; }
  __syncthreads();
  if (w == 0) {
    long long ta = lane < kWarps ? g_red[lane] : op_identity(op);
    bool tf = lane < kWarps ? (g_redu[lane] != 0) : false;
    long long sa = ta;
    bool sf = tf;
    for (int o = 1; o < 32; o <<= 1) {
      long long ya = __shfl_up_sync(0xffffffffu, sa, o);
      int yf = __shfl_up_sync(0xffffffffu, (int)sf, o);
      if (lane >= o) {
        if (!sf) sa = op_combine(op, ya, sa);
        sf = sf || yf;
      }
    }
    // exclusive across warps
    long long ea = __shfl_up_sync(0xffffffffu, sa, 1);
    if (lane == 0) ea = op_identity(op);
    if (lane < kWarps) g_red[lane] = ea;
  }
  __syncthreads();
  long long wcarry = g_red[w];
  // exclusive within warp: previous lane's inclusive
  long long pa = __shfl_up_sync(0xffffffffu, a, 1);
  int pf = __shfl_up_sync(0xffffffffu, (int)f, 1);
  long long carry;
  if (lane == 0) carry = wcarry;
  else carry = pf ? pa : op_combine(op, wcarry, pa);
  __syncthreads();
  return carry;
}

// ---------------------------------------------------------------------------
// Sort helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bin_get(const uint32_t* bins, int b) {
  return (bins[b >> 1] >> ((b & 1) * 16)) & 0xFFFFu;
}

// Stable LSD radix sort of idx by (keys[idx] - kmin) over bits [0, vb).
// Positions are warp-striped so that ranking in (step, lane) order is the
// input order.  Returns the buffer that holds the result.
__device__ uint16_t* lsd_sort(const SortSmem& s, int n, unsigned long long kmin, int vb) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint16_t* in = s.idxA;
  uint16_t* out = s.idxB;
  for (int i = threadIdx.x; i < n; i += kThreads) in[i] = (uint16_t)i;
  uint16_t* whist = reinterpret_cast<uint16_t*>(s.bins);  // [kWarps][256]
  const unsigned lt = (1u << lane) - 1;
  for (int p = 0; p < vb; p += 8) {
    for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) whist[i] = 0;
    __syncthreads();
    uint16_t myidx[kEPT];
    uint16_t rank[kEPT];
    uint8_t dg[kEPT];
#pragma unroll
    for (int j = 0; j < kEPT; ++j) {
      int pos = w * (kEPT * 32) + j * 32 + lane;
      bool act = pos < n;
      uint16_t id = act ? in[pos] : 0;
      unsigned d = act ? (unsigned)(((s.keys[id] - kmin) >> p) & 0xFFu) : 0u;
      unsigned peers = __ballot_sync(0xffffffffu, act);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bb : ~bb;
      }
      unsigned base = 0;
      if (act) {
        int leader = __ffs(peers) - 1;
        if (lane == leader) {
          base = whist[w * 256 + d];
          whist[w * 256 + d] = (uint16_t)(base + __popc(peers));
        }
      }
      unsigned srcl = act ? (unsigned)(__ffs(peers) - 1) : (unsigned)lane;
      base = __shfl_sync(0xffffffffu, base, srcl);
      myidx[j] = id;
      rank[j] = (uint16_t)(base + __popc(peers & lt));
      dg[j] = (uint8_t)d;
    }
    __syncthreads();
    // exclusive scan over (digit, warp)
    {
      int d = threadIdx.x;  // kThreads >= 256
      int tot = 0;
      if (d < 256)
        for (int ww = 0; ww < kWarps; ++ww) tot += whist[ww * 256 + d];
      int total;
      int start = block_excl_sum(d < 256 ? tot : 0, &total);
      if (d < 256) {
        int run = start;
        for (int ww = 0; ww < kWarps; ++ww) {
          int c = whist[ww * 256 + d];
          whist[ww * 256 + d] = (uint16_t)run;
          run += c;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kEPT; ++j) {
      int pos = w * (kEPT * 32) + j * 32 + lane;
      if (pos < n) out[whist[w * 256 + dg[j]] + rank[j]] = myidx[j];
    }
    __syncthreads();
    uint16_t* t = in; in = out; out = t;
  }
  return in;
}

// Sort s.idx by key.  Returns the buffer holding the sorted permutation.
__device__ uint16_t* chunk_sort(const SortSmem& s, int n) {
  unsigned long long lmin = ~0ull, lmax = 0ull;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    unsigned long long k = s.keys[i];
    lmin = k < lmin ? k : lmin;
    lmax = k > lmax ? k : lmax;
  }
  unsigned long long kmin, kmax;
  block_minmax(lmin, lmax, &kmin, &kmax);
  if (n == 0) return s.idxA;
  const unsigned long long range = kmax - kmin;
  const int vb = range == 0 ? 0 : 64 - __clzll((long long)range);
  const int sh = vb > kBinBits ? vb - kBinBits : 0;
  // counting sort on the top bits
  for (int i = threadIdx.x; i < kBins / 2; i += kThreads) s.bins[i] = 0;
  __syncthreads();
  uint16_t rb[kEPT], rr[kEPT];
#pragma unroll
  for (int j = 0; j < kEPT; ++j) {
    int i = threadIdx.x + j * kThreads;
    if (i < n) {
      int b = (int)((s.keys[i] - kmin) >> sh);
      unsigned sft = (b & 1) * 16;
      unsigned old = atomicAdd(&s.bins[b >> 1], 1u << sft);
      rb[j] = (uint16_t)b;
      rr[j] = (uint16_t)((old >> sft) & 0xFFFFu);
    }
  }
  __syncthreads();
  // exclusive scan of the bin counts (kBins / kThreads = 8 per thread)
  constexpr int BPT = kBins / kThreads;
  int cnt[BPT];
  int loc = 0, mx = 0;
#pragma unroll
  for (int q = 0; q < BPT; ++q) {
    cnt[q] = (int)bin_get(s.bins, threadIdx.x * BPT + q);
    loc += cnt[q];
    mx = max(mx, cnt[q]);
  }
  int total;
  int start = block_excl_sum(loc, &total);
  int maxbin = block_max_int(mx);
  // write starts back (packed 16-bit; starts <= kTileCap fit)
#pragma unroll
  for (int q = 0; q < BPT; q += 2) {
    unsigned lo = (unsigned)start;
    start += cnt[q];
    unsigned hi = (unsigned)start;
    start += cnt[q + 1];
    s.bins[(threadIdx.x * BPT + q) >> 1] = lo | (hi << 16);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kEPT; ++j) {
    int i = threadIdx.x + j * kThreads;
    if (i < n) s.idxA[bin_get(s.bins, rb[j]) + rr[j]] = (uint16_t)i;
  }
  __syncthreads();
  if (sh == 0) return s.idxA;  // every bin holds one key value
  if (maxbin <= 32) {
    for (int b = threadIdx.x; b < kBins; b += kThreads) {
      int st = (int)bin_get(s.bins, b);
      int en = (b + 1 < kBins) ? (int)bin_get(s.bins, b + 1) : n;
      for (int i = st + 1; i < en; ++i) {
        uint16_t v = s.idxA[i];
        unsigned long long kv = s.keys[v];
        int j = i - 1;
        while (j >= st && s.keys[s.idxA[j]] > kv) {
          s.idxA[j + 1] = s.idxA[j];
          --j;
        }
        s.idxA[j + 1] = v;
      }
    }
    __syncthreads();
    return s.idxA;
  }
  return lsd_sort(s, n, kmin, vb);
}

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void load_chunk_column(const SortSmem& s, const RowSrc& src,
                                                  const RunSet& runs, const Chunk& ch, int n,
                                                  int col, long long* dst_ll,
                                                  unsigned long long* dst_key) {
  if (MODE == MODE_RUNS) {
    for (int r = 0; r < runs.k; ++r) {
      long long lo = s.slo[r], pre = s.spre[r];
      int len = (int)(s.spre[r + 1] - pre);
      const long long* p = runs.ptrs[(long long)r * (1 + runs.ncols) + (col < 0 ? 0 : 1 + col)];
      for (int i = threadIdx.x; i < len; i += kThreads) {
        long long v = __ldg(p + lo + i);
        if (col < 0) dst_key[pre + i] = (unsigned long long)v;
        else dst_ll[pre + i] = v;
      }
    }
  } else {
    for (int i = threadIdx.x; i < n; i += kThreads) {
      if (col < 0) dst_key[i] = src_key(src, ch.lo + i);
      else dst_ll[i] = src_col(src, col, ch.lo + i);
    }
  }
}

__device__ __forceinline__ void write_fine_offsets(const OutSink& out, const Chunk& ch, long long base,
                                                   long long g, long long count, unsigned long long key,
                                                   unsigned long long prev_key) {
  // offs[f] = absolute position of the first row with fine digit >= f; the
  // entry at f_hi (start of the next chunk's range) is written by both
  // neighbours with the same value.
  int f = (int)fine_digit(out.dig, key);
  int fp = (g == 0) ? ch.f_lo - 1 : (int)fine_digit(out.dig, prev_key);
  for (int ff = fp + 1; ff <= f; ++ff) out.offs[ff] = base + g;
  if (g == count - 1)
    for (int ff = f + 1; ff <= ch.f_hi; ++ff) out.offs[ff] = base + count;
}

__device__ __forceinline__ void sink_key(const OutSink& out, long long pos, unsigned long long key) {
  if (pos >= out.capacity) return;
  if (out.user) store_key(out.kout, pos, key);
  else out.keys[pos] = key;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_sortfold(const Chunk* __restrict__ chunks, RowSrc src, RunSet runs, CopySrc copy, FoldDesc fd,
           OutSink out, LookBack lb, long long tile_n, int tile_f_hi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem s = carve(smem_raw);
  __shared__ int s_cid;
  __shared__ long long s_base;
  __shared__ int s_n;
  __shared__ int s_count;

  __shared__ int s_err;
  if (threadIdx.x == 0) {
    s_cid = (int)atomicAdd(lb.ticket, 1u);
    s_err = err_load(lb.err);
  }
  __syncthreads();
  const int cid = s_cid;
  if (cid >= lb.n_chunks || s_err) return;  // block-uniform

  Chunk ch;
  if (MODE == MODE_TILES) {
    ch.lo = (long long)cid * kTileCap;
    ch.hi = min(tile_n, ch.lo + kTileCap);
    ch.f_lo = 0; ch.f_hi = tile_f_hi; ch.kind = CH_NORMAL; ch.pad = 0;
  } else {
    ch = chunks[cid];
  }

  if (ch.kind == CH_COPY) {
    const long long n = ch.hi - ch.lo;
    if (threadIdx.x < 32) {
      long long b = lookback_warp(lb, cid, n);
      if (threadIdx.x == 0) {
        s_base = b;
        if (b >= 0 && lb.total_out && cid == lb.n_chunks - 1) *lb.total_out = b + n;
        if (b >= 0 && b + n > out.capacity) err_raise(lb.err, ERR_CAPACITY);
      }
    }
    __syncthreads();
    const long long base = s_base;
    if (base < 0) return;
    for (long long g = threadIdx.x; g < n; g += kThreads) {
      unsigned long long key = copy.keys[ch.lo + g];
      sink_key(out, base + g, key);
      if (out.offs) {
        unsigned long long pk = g > 0 ? copy.keys[ch.lo + g - 1] : 0ull;
        write_fine_offsets(out, ch, base, g, n, key, pk);
      }
      if (base + g < out.capacity)
        for (int st = 0; st < fd.n_state; ++st) out.cols[st][base + g] = copy.cols[st][ch.lo + g];
    }
    if (out.offs && n == 0 && threadIdx.x == 0)
      for (int ff = ch.f_lo; ff <= ch.f_hi; ++ff) out.offs[ff] = base;
    return;
  }

  // ---- 1. keys ----
  if (MODE == MODE_RUNS) {
    const int k = runs.k;
    for (int r = threadIdx.x; r < k; r += kThreads) {
      long long lo = runs.offs[(long long)r * runs.stride + ch.f_lo];
      long long hi = runs.offs[(long long)r * runs.stride + ch.f_hi];
      s.slo[r] = lo;
      s.spre[r + 1] = hi - lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long acc = 0;
      s.spre[0] = 0;
      for (int r = 0; r < k; ++r) { acc += s.spre[r + 1]; s.spre[r + 1] = acc; }
      s_n = (int)min(acc, (long long)kTileCap + 1);
    }
    __syncthreads();
  } else {
    if (threadIdx.x == 0) s_n = (int)(ch.hi - ch.lo);
    __syncthreads();
  }
  const int n = s_n;
  if (n > kTileCap) {  // the planner never makes such chunks
    if (threadIdx.x == 0) err_raise(lb.err, ERR_INTERNAL);
    return;
  }
  load_chunk_column<MODE>(s, src, runs, ch, n, -1, nullptr, s.keys);
  __syncthreads();

  // ---- 2. sort ----
  uint16_t* sidx = chunk_sort(s, n);
  uint16_t* segid = (sidx == s.idxA) ? s.idxB : s.idxA;

  // ---- 3. segment heads / ids over contiguous strips ----
  const int s0 = threadIdx.x * kEPT;
  unsigned hmask = 0;
  int hc = 0;
#pragma unroll
  for (int j = 0; j < kEPT; ++j) {
    int p = s0 + j;
    if (p < n) {
      bool h = (p == 0) || (s.keys[sidx[p]] != s.keys[sidx[p - 1]]);
      hmask |= (unsigned)h << j;
      hc += h;
    }
  }
  int count;
  int g0 = block_excl_sum(hc, &count);
  {
    int g = g0 - 1;
#pragma unroll
    for (int j = 0; j < kEPT; ++j) {
      int p = s0 + j;
      if (p < n) {
        g += (hmask >> j) & 1u;
        segid[p] = (uint16_t)g;
      }
    }
  }
  // is the first row of the next strip a head (ends my last segment)?
  const bool next_head = (s0 + kEPT >= n) || (s0 + kEPT < n && (s.keys[sidx[s0 + kEPT]] != s.keys[sidx[s0 + kEPT - 1]]));

  // ---- 4. output offset ----
  if (threadIdx.x < 32) {
    long long b = lookback_warp(lb, cid, count);
    if (threadIdx.x == 0) {
      s_base = b;
      s_count = count;
      if (b >= 0 && lb.total_out && cid == lb.n_chunks - 1) *lb.total_out = b + count;
      if (b >= 0 && b + count > out.capacity) err_raise(lb.err, ERR_CAPACITY);
    }
  }
  __syncthreads();
  const long long base = s_base;
  if (base < 0) return;

  // ---- 5a. distinct keys, staged in work[] ----
  {
    unsigned long long kr[kEPT];
#pragma unroll
    for (int j = 0; j < kEPT; ++j) {
      int p = s0 + j;
      kr[j] = p < n ? s.keys[sidx[p]] : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kEPT; ++j) {
      int p = s0 + j;
      if (p < n && ((hmask >> j) & 1u)) s.work[segid[p]] = (long long)kr[j];
    }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < count; g += kThreads) {
    unsigned long long key = (unsigned long long)s.work[g];
    sink_key(out, base + g, key);
    if (out.offs) write_fine_offsets(out, ch, base, g, count,
                                     key, g > 0 ? (unsigned long long)s.work[g - 1] : 0ull);
  }
  if (out.offs && count == 0 && threadIdx.x == 0)
    for (int ff = ch.f_lo; ff <= ch.f_hi; ++ff) out.offs[ff] = base;
  __syncthreads();

  // ---- 5b. aggregates, one source column at a time ----
  const int ncols_src = (MODE == MODE_RUNS) ? runs.ncols : src.ncols;
  for (int c = -1; c < ncols_src; ++c) {
    bool used = false;
    for (int st = 0; st < fd.n_state; ++st) used |= (fd.src[st] == c);
    if (!used) continue;
    long long v[kEPT];
    if (c >= 0) {
      load_chunk_column<MODE>(s, src, runs, ch, n, c, s.work, nullptr);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kEPT; ++j) {
        int p = s0 + j;
        v[j] = p < n ? s.work[sidx[p]] : 0;
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int j = 0; j < kEPT; ++j) v[j] = 1;
    }
    for (int st = 0; st < fd.n_state; ++st) {
      if (fd.src[st] != c) continue;
      const int op = fd.op[st];
      // pass 1: partial of the strip's last segment
      long long acc = op_identity(op);
      bool hh = false;
#pragma unroll
      for (int j = 0; j < kEPT; ++j) {
        int p = s0 + j;
        if (p < n) {
          if ((hmask >> j) & 1u) { acc = v[j]; hh = true; }
          else acc = op_combine(op, acc, v[j]);
        }
      }
      long long carry = block_seg_carry(op, hh, acc);
      // pass 2: complete segments, staged by segment id (a strip that starts
      // with a head overwrites the carry at once)
      acc = carry;
#pragma unroll
      for (int j = 0; j < kEPT; ++j) {
        int p = s0 + j;
        if (p < n) {
          if ((hmask >> j) & 1u) acc = v[j];
          else acc = op_combine(op, acc, v[j]);
          bool ends = (j == kEPT - 1) ? next_head : (((hmask >> (j + 1)) & 1u) != 0 || p + 1 >= n);
          if (ends) s.work[segid[p]] = acc;
        }
      }
      __syncthreads();
      for (int g = threadIdx.x; g < count; g += kThreads)
        if (base + g < out.capacity) out.cols[st][base + g] = s.work[g];
      __syncthreads();
    }
  }
}

}  // namespace sg
