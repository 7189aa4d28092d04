// sg_sortfold.cuh -- sort a chunk of rows in shared memory and fold equal
// keys (the in-cache batch sort + duplicate detection of Sec. 6.1): the
// run-generation leaf, tile pre-aggregation, one-chunk inputs and the
// one-chunk instances of a batched call.  (The wide merge of Sec. 4 has a
// kernel of its own, sg_merge.cuh.)
//
// One CTA takes one chunk (ticket order) of at most kTileCap rows:
//   1. load the chunk's keys into shared memory (a row range of one source,
//      all loads in flight at once);
//   2. sort a permutation of the chunk by key: a counting sort on the top
//      kBinBits bits of (key - chunk min); one pass over adjacent positions
//      flags the bins still out of key order, and only those are finished:
//      by insertion sort up to 32 rows, a bigger bin (a repeated key, as a
//      rule) by a warp that ranks the bin's distinct keys; a bin of more
//      than 32 distinct keys sends the chunk to a stable LSD radix sort
//      (8-bit digits, warp-ballot ranking) over every bit that varies inside
//      the chunk;
//   3. fold equal keys: the chunk's distinct-key count gives its output
//      offset by decoupled look-back; each aggregate source column is staged
//      once into shared memory in sorted order (where the keys were) and
//      folded from there by segmented warp scans over head bits, or -- with
//      at most kFewGroups groups -- by the whole CTA one group at a time.
#pragma once
#include "sg_common.cuh"

namespace sg {

constexpr int kTileCap = 8192;             // rows per chunk
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kBinBits = 13;
constexpr int kBins = 1 << kBinBits;
constexpr int kBinsPerThread = kBins / kThreads;  // 16
constexpr int kMaxFanIn = 256;             // runs one wide-merge tile can read
constexpr int kFewGroups = 16;             // CTA-per-group fold below this many keys
constexpr int kAccBlock = 8;               // state columns folded per pass

enum : int { CH_NORMAL = 0, CH_COPY = 1 };
enum : int { MODE_RANGE = 0, MODE_TILES = 2, MODE_INST = 3, MODE_DIRECT = 4 };

// One instance of a batched call (same layout as sgagg_instance).
struct InstDesc {
  const void* keys;
  int key_bytes;
  int n_payload;
  const long long* const* payload;   // device array of n_payload device pointers
  long long n;
  void* out_keys;
  long long* const* out_aggs;        // device array
  long long out_capacity;
  long long* out_rows;               // device
};

// Batched tiles: chunk.pad = instance; the tile's rows are read from that
// instance's columns, its keys OR-ed with instance << key_bits.
struct InstSet {
  const InstDesc* inst;
  int key_bits;
  int8_t colsel[kMaxCols];   // carried column c -> the instance's payload column
  unsigned long long* kmin;  // per instance: least key (preset ~0), or null
  unsigned long long* kmax;  // per instance: greatest key (preset 0)
  int grouped;               // MODE_TILES / MODE_INST tile pre-aggregation: equal keys
                             // need only be adjacent (partial rows are sorted later),
                             // so the chunk is binned by a hash of the key
};

struct Chunk {
  long long lo, hi;   // MODE_RANGE: source rows; CH_COPY: rows of the copy source
  int f_lo, f_hi;     // fine buckets covered (the run's sparse index; merge tiles' slices)
  int kind;
  int pad;
};

// k sorted runs of state rows in SoA form, for the wide merge.  Run r's rows
// with fine digit in [f_lo, f_hi) are rows offs[r][f_lo] .. offs[r][f_hi] - 1
// of its arrays (offs[r] is the run's sparse index over fine buckets).
struct RunSet {
  int k;
  int ncols;
  const long long* const* ptrs;   // [k * (1 + ncols)]: keys, then state columns
  const long long* const* offs;   // [k] fine-bucket offsets of each run
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
  long long offs_stride;            // > 0: several runs at once (MODE_RANGE); the chunk whose
  int offs_bbits;                   // first bucket is d writes the offsets of run
                                    // d >> offs_bbits at offs + run * offs_stride
  Digit dig;
  long long* rows_out;              // MODE_DIRECT: the instance's row count (-1: over capacity)
  unsigned long long* rows_sum;     // MODE_DIRECT: rows of all instances (added), or null
};

struct SortSmem {
  unsigned long long* keys;   // [kTileCap]
  uint16_t* idx;              // [kTileCap] sorted permutation
  uint32_t* bins;             // [kBins / 2] packed 16-bit bin starts; LSD ping-pong buffer;
                              // then the inverse permutation (sorted position of each row)
  uint16_t* whist;            // [kWarps * 256] LSD per-warp digit counts; or the bin flags,
                              // big-bin and flagged-bin lists; then the head bitmask and
                              // its word prefix
};

constexpr size_t kSortSmemBytes = kTileCap * 8 + kTileCap * 2 + (kBins / 2) * 4 + kWarps * 256 * 2 + 64;
static_assert(kBins >= kTileCap, "the LSD ping-pong buffer lives in the bins area");
// two CTAs per SM: 2 x (dynamic + static (< 2.5 KB) + 1 KB reserved) within 228 KB
static_assert(kSortSmemBytes <= 113000, "k_sortfold must keep two CTAs per SM");

__device__ __forceinline__ SortSmem carve(unsigned char* base) {
  SortSmem s;
  s.keys = reinterpret_cast<unsigned long long*>(base);
  s.idx = reinterpret_cast<uint16_t*>(base + kTileCap * 8);
  s.bins = reinterpret_cast<uint32_t*>(base + kTileCap * 10);
  s.whist = reinterpret_cast<uint16_t*>(base + kTileCap * 10 + (kBins / 2) * 4);
  return s;
}

// ---------------------------------------------------------------------------
// Block-wide helpers (kThreads threads).
// ---------------------------------------------------------------------------
__shared__ long long g_red[kWarps + 1];
__shared__ int g_wmax[kWarps];

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

__device__ __forceinline__ long long warp_reduce(int op, long long v) {
  for (int o = 16; o > 0; o >>= 1) v = op_combine(op, v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Row access.
// ---------------------------------------------------------------------------
struct ChunkView {
  long long lo;     // first source row
  int n;
};

template <int MODE>
__device__ __forceinline__ void load_keys(const SortSmem& s, const RowSrc& src, const ChunkView& cv,
                                          unsigned long long* lmin, unsigned long long* lmax) {
  if (src_keys_direct(src)) {
    // 8-byte keys: copied global to shared by cp.async, all in flight at once
    for (int i = threadIdx.x; i < cv.n; i += kThreads) {
      const unsigned long long* p;
      if (MODE == MODE_RANGE) {
        p = reinterpret_cast<const unsigned long long*>(src.aos + (cv.lo + i) * (1 + src.ncols));
      } else {
        p = src_key_ptr(src, cv.lo + i);
      }
      cp_async8(&s.keys[i], p);
    }
    cp_async_wait();
    for (int i = threadIdx.x; i < cv.n; i += kThreads) {  // the thread's own copies
      const unsigned long long v = s.keys[i];
      *lmin = v < *lmin ? v : *lmin;
      *lmax = v > *lmax ? v : *lmax;
    }
    return;
  }
  constexpr int U = 8;  // loads in flight per thread
  for (int base = threadIdx.x; base < cv.n; base += U * kThreads) {
    unsigned long long v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int i = base + u * kThreads;
      if (i < cv.n) {
        v[u] = src_key(src, cv.lo + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int i = base + u * kThreads;
      if (i < cv.n) {
        s.keys[i] = v[u];
        *lmin = v[u] < *lmin ? v[u] : *lmin;
        *lmax = v[u] > *lmax ? v[u] : *lmax;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Sort.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bin_get(const uint32_t* bins, int b) {
  return (bins[b >> 1] >> ((b & 1) * 16)) & 0xFFFFu;
}

// Stable LSD radix sort of s.idx by (keys[idx] - kmin) over bits [0, vb);
// positions are warp-striped so that ranking in (step, lane) order is the
// input order.  The result is left in s.idx.
__device__ void lsd_sort(const SortSmem& s, int n, unsigned long long kmin, int vb) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int EPT = kTileCap / kThreads;
  uint16_t* in = s.idx;
  uint16_t* out = reinterpret_cast<uint16_t*>(s.bins);  // ping-pong in the bins area
  for (int i = threadIdx.x; i < n; i += kThreads) in[i] = (uint16_t)i;
  uint16_t* whist = s.whist;  // [kWarps][256]
  const unsigned lt = (1u << lane) - 1;
  for (int p = 0; p < vb; p += 8) {
    for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) whist[i] = 0;
    __syncthreads();
    uint32_t packed[EPT];  // rank (16 bits) | digit (8 bits) << 16
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      int pos = w * (EPT * 32) + j * 32 + lane;
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
      packed[j] = ((base + __popc(peers & lt)) & 0xFFFFu) | (d << 16);
    }
    __syncthreads();
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
    for (int j = 0; j < EPT; ++j) {
      int pos = w * (EPT * 32) + j * 32 + lane;
      if (pos < n) out[whist[w * 256 + (packed[j] >> 16)] + (packed[j] & 0xFFFFu)] = in[pos];
    }
    __syncthreads();
    uint16_t* t = in; in = out; out = t;
  }
  if (in != s.idx) {
    for (int i = threadIdx.x; i < n; i += kThreads) s.idx[i] = in[i];
    __syncthreads();
  }
}

// Insertion sort of positions [st, en) of s.idx by key (one thread).
__device__ __forceinline__ void insertion_sort_bin(const SortSmem& s, int st, int en) {
  for (int i = st + 1; i < en; ++i) {
    const uint16_t v = s.idx[i];
    const unsigned long long kv = s.keys[v];
    int j = i - 1;
    while (j >= st) {
      const uint16_t u = s.idx[j];
      if (s.keys[u] <= kv) break;
      s.idx[j + 1] = u;
      --j;
    }
    s.idx[j + 1] = v;
  }
}

// Sort s.idx by key; returns whether a key group may hold more than 32 rows.
// Block key range: each warp's least and greatest loaded key, combined by
// shared-memory atomics (g_kmin / g_kmax are preset when the CTA starts).
__shared__ unsigned long long g_kmin, g_kmax;
__shared__ int g_maxbin;

// Multiplicative (Fibonacci) hashing of a key to one of kBins bins.
__device__ __forceinline__ int hash_bin(unsigned long long key) {
  return (int)((key * 0x9E3779B97F4A7C15ull) >> (64 - kBinBits));
}

// Sort s.idx by key (the keys just loaded; lmin / lmax: the thread's least
// and greatest); returns whether a key group may hold more than 32 rows.
// hashed: bin by hash_bin instead of key range -- equal keys still end up
// adjacent (each bin is sorted), but bins are not in key order; a skewed key
// distribution then spreads over the bins instead of crowding a few.
__device__ bool chunk_sort(const SortSmem& s, int n, unsigned long long lmin, unsigned long long lmax,
                           bool hashed = false) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // zero the bins while the key range is combined: one barrier for the
  // loaded keys, the range and the bins
  for (int i = threadIdx.x; i < kBins / 2; i += kThreads) s.bins[i] = 0;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lmin, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, lmax, o);
    lmin = a < lmin ? a : lmin;
    lmax = b > lmax ? b : lmax;
  }
  if (lane == 0 && lmin <= lmax) {
    atomicMin(&g_kmin, lmin);
    atomicMax(&g_kmax, lmax);
  }
  __syncthreads();
  if (n == 0) return false;
  const unsigned long long kmin = g_kmin, kmax = g_kmax;
  const unsigned long long range = kmax - kmin;
  const int vb = range == 0 ? 0 : 64 - __clzll((long long)range);
  const int sh = vb > kBinBits ? vb - kBinBits : 0;
  // counting sort on the top bits: rank inside the bin from the atomic, kept
  // in registers (a thread's rows are i = threadIdx.x + j * kThreads)
  constexpr int EPT = kTileCap / kThreads;
  uint32_t br[EPT];  // bin << 16 | rank in bin
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int i = threadIdx.x + j * kThreads;
    if (i < n) {
      const int b = hashed ? hash_bin(s.keys[i]) : (int)((s.keys[i] - kmin) >> sh);
      const unsigned sft = (b & 1) * 16;
      const unsigned old = atomicAdd(&s.bins[b >> 1], 1u << sft);
      br[j] = ((unsigned)b << 16) | ((old >> sft) & 0xFFFFu);
    }
  }
  __syncthreads();
  int cnt[kBinsPerThread];
  int loc = 0, mx = 0;
#pragma unroll
  for (int q = 0; q < kBinsPerThread; ++q) {
    cnt[q] = (int)bin_get(s.bins, threadIdx.x * kBinsPerThread + q);
    loc += cnt[q];
    mx = max(mx, cnt[q]);
  }
  // exclusive scan of the thread counts and the largest bin, two barriers
  int x = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 31) {
    g_red[w] = x;
    g_wmax[w] = mx;
  }
  __syncthreads();
  if (w == 0) {
    const long long v = lane < kWarps ? g_red[lane] : 0;
    long long t = v;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) g_red[lane] = t - v;
    int m = lane < kWarps ? g_wmax[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) g_maxbin = m;
  }
  __syncthreads();
  int start = (int)g_red[w] + x - loc;
  const int maxbin = g_maxbin;
#pragma unroll
  for (int q = 0; q < kBinsPerThread; q += 2) {
    unsigned lo = (unsigned)start;
    start += cnt[q];
    unsigned hi = (unsigned)start;
    start += cnt[q + 1];
    s.bins[(threadIdx.x * kBinsPerThread + q) >> 1] = lo | (hi << 16);
  }
  __syncthreads();
  // place; the bin flags (below) and the big-bin list live in the LSD
  // histogram area, which is free until an LSD sort
  uint32_t* flag = reinterpret_cast<uint32_t*>(s.whist);  // [kBins / 32]: bin holds an inversion
  uint32_t* blist = flag + kBins / 32;                    // start | end << 16; fewer than n / 32 bins
  uint16_t* flist = s.whist + kBins / 16 * 2;             // [kFlagList] the flagged bins
  constexpr int kFlagList = kWarps * 256 - kBins / 16 * 2;
  __shared__ int s_nbig, s_over, s_nflag;
  if (hashed || sh != 0) {  // block-uniform
    for (int i = threadIdx.x; i < kBins / 32; i += kThreads) flag[i] = 0;
    if (threadIdx.x == 0) {
      s_nbig = 0;
      s_over = 0;
      s_nflag = 0;
    }
  }
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int i = threadIdx.x + j * kThreads;
    if (i < n) s.idx[(int)bin_get(s.bins, (int)(br[j] >> 16)) + (int)(br[j] & 0xFFFFu)] = (uint16_t)i;
  }
  __syncthreads();
  if (!hashed && sh == 0) return maxbin > 32;  // every bin is one key value
  // Bins are key ranges in key order, so two adjacent positions out of key
  // order lie in one bin: only the bins holding such an inversion need
  // sorting.  One pass over adjacent positions flags them (a bit per bin)
  // and lists them (first flag of a bin only).
  for (int p0 = threadIdx.x - lane; p0 < n; p0 += kThreads) {  // warp-uniform
    const int p = p0 + lane;
    const unsigned long long a = p < n ? s.keys[s.idx[p]] : ~0ull;
    unsigned long long b = __shfl_down_sync(0xffffffffu, a, 1);
    if (lane == 31 && p + 1 < n) b = s.keys[s.idx[p + 1]];
    // (range bins are in key order: an inversion lies inside one bin; hash
    // bins are compared as well)
    if (p + 1 < n && a > b && (!hashed || hash_bin(a) == hash_bin(b))) {
      const int bin = hashed ? hash_bin(a) : (int)((a - kmin) >> sh);
      const unsigned bit = 1u << (bin & 31);
      if (!(atomicOr(&flag[bin >> 5], bit) & bit)) {
        const int q = atomicAdd(&s_nflag, 1);
        if (q < kFlagList) flist[q] = (uint16_t)bin;
      }
    }
  }
  __syncthreads();
  if (maxbin <= 32) {
    // flagged bins are sorted by insertion: a thread per listed bin, or (list
    // overflow) a thread per kBinsPerThread consecutive bins
    const int nfl = s_nflag;
    if (nfl <= kFlagList) {  // block-uniform
      for (int q = threadIdx.x; q < nfl; q += kThreads) {
        const int b = flist[q];
        insertion_sort_bin(s, (int)bin_get(s.bins, b), b + 1 < kBins ? (int)bin_get(s.bins, b + 1) : n);
      }
    } else {
      const int b0 = threadIdx.x * kBinsPerThread;
      unsigned m = (flag[b0 >> 5] >> (b0 & 31)) & ((1u << kBinsPerThread) - 1u);
      while (m) {
        const int b = b0 + __ffs(m) - 1;
        m &= m - 1;
        insertion_sort_bin(s, (int)bin_get(s.bins, b), b + 1 < kBins ? (int)bin_get(s.bins, b + 1) : n);
      }
    }
    __syncthreads();
    return false;
  }
  // Some bin holds more than 32 rows -- usually a key repeated many times.
  // Flagged bins of up to 32 rows are finished by insertion as above.  A warp
  // takes each bigger flagged bin: it collects the bin's distinct keys (at
  // most 32, one per lane, with their row counts), ranks them, and places
  // every row at its key's position.  A bin with more distinct keys sends the
  // chunk to the LSD sort.
  for (int b = threadIdx.x; b < kBins; b += kThreads) {
    if (!((flag[b >> 5] >> (b & 31)) & 1u)) continue;
    const int st = (int)bin_get(s.bins, b);
    const int en = (b + 1 < kBins) ? (int)bin_get(s.bins, b + 1) : n;
    if (en - st > 32) blist[atomicAdd(&s_nbig, 1)] = (unsigned)st | ((unsigned)en << 16);
    else insertion_sort_bin(s, st, en);
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1;
    uint16_t* tmp = reinterpret_cast<uint16_t*>(s.bins);  // bin starts are no longer needed
    const int nbig = s_nbig;
    for (int q = w; q < nbig; q += kWarps) {
      const int st = (int)(blist[q] & 0xFFFFu), en = (int)(blist[q] >> 16);
      unsigned long long dkey = 0;  // lane e: distinct key e of the bin
      int dcnt = 0, nd = 0;         // lane e: its rows; nd: keys found (warp-uniform)
      bool over = false;
      for (int base = st; base < en && !over; base += 32) {
        const int i = base + lane;
        const bool act = i < en;
        const unsigned long long key = act ? s.keys[s.idx[i]] : 0ull;
        bool known = false;
        for (int e = 0; e < nd; ++e) {
          const unsigned long long ke = __shfl_sync(0xffffffffu, dkey, e);
          const unsigned m = __ballot_sync(0xffffffffu, act && key == ke);
          known |= (m >> lane) & 1u;
          if (lane == e) dcnt += __popc(m);
        }
        unsigned nf = __ballot_sync(0xffffffffu, act && !known);
        while (nf) {
          if (nd == 32) {
            over = true;
            break;
          }
          const int l = __ffs(nf) - 1;
          const unsigned long long kl = __shfl_sync(0xffffffffu, key, l);
          const unsigned m = __ballot_sync(0xffffffffu, act && !known && key == kl);
          if (lane == nd) {
            dkey = kl;
            dcnt = __popc(m);
          }
          ++nd;
          nf &= ~m;
        }
      }
      if (over) {  // warp-uniform
        if (lane == 0) s_over = 1;
        continue;
      }
      // lane e: first position of key e = st + rows of the smaller keys
      int cur = st;
      for (int e = 0; e < nd; ++e) {
        const unsigned long long ke = __shfl_sync(0xffffffffu, dkey, e);
        const int ce = __shfl_sync(0xffffffffu, dcnt, e);
        if (lane < nd && ke < dkey) cur += ce;
      }
      for (int base = st; base < en; base += 32) {
        const int i = base + lane;
        const bool act = i < en;
        const uint16_t v = act ? s.idx[i] : (uint16_t)0;
        const unsigned long long key = act ? s.keys[v] : 0ull;
        int pos = -1;
        for (int e = 0; e < nd; ++e) {
          const unsigned long long ke = __shfl_sync(0xffffffffu, dkey, e);
          const unsigned m = __ballot_sync(0xffffffffu, act && key == ke);
          const int c0 = __shfl_sync(0xffffffffu, cur, e);
          if ((m >> lane) & 1u) pos = c0 + __popc(m & lt);
          if (lane == e) cur += __popc(m);
        }
        if (act && pos >= st && pos < en) tmp[pos] = v;
      }
      __syncwarp();
      for (int i = st + lane; i < en; i += 32) s.idx[i] = tmp[i];
      __syncwarp();
    }
  }
  __syncthreads();
  if (s_over) lsd_sort(s, n, kmin, vb);  // block-uniform
  return true;
}

// ---------------------------------------------------------------------------
// Output helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void write_fine_offsets(const OutSink& out, const Chunk& ch, long long base,
                                                   long long g, long long count, unsigned long long key,
                                                   bool has_prev, unsigned long long prev_key) {
  // offs[f] = absolute position of the first row with fine digit >= f; the
  // entry at f_hi (start of the next chunk's range) is written by both
  // neighbours with the same value.
  int f = (int)fine_digit(out.dig, key);
  int fp = has_prev ? (int)fine_digit(out.dig, prev_key) : ch.f_lo - 1;
  for (int ff = fp + 1; ff <= f; ++ff) out.offs[ff] = base + g;
  if (g == count - 1)
    for (int ff = f + 1; ff <= ch.f_hi; ++ff) out.offs[ff] = base + count;
}

__device__ __forceinline__ void sink_key(const OutSink& out, long long pos, unsigned long long key) {
  if (pos >= out.capacity) return;
  if (!out.user) out.keys[pos] = key;
  else if (out.kout.n_cols == 1 && out.kout.bytes[0] == 8)  // one 8-byte column: the key as is
    reinterpret_cast<unsigned long long*>(out.kout.cols[0])[pos] = key;
  else store_key(out.kout, pos, key);
}

__device__ __forceinline__ void sink_val(const OutSink& out, int st, long long pos, long long v) {
  if (pos < out.capacity) out.cols[st][pos] = v;
}

// MODE_DIRECT: the chunk is a whole instance with outputs of its own: base
// 0, and the instance's row count (or -1 when it exceeds out_capacity; then
// nothing is written and the other instances go on).
__device__ __forceinline__ long long direct_base(const OutSink& out, long long count, long long* s_base) {
  if (threadIdx.x == 0) {
    const bool fits = count <= out.capacity;
    *out.rows_out = fits ? count : -1;
    if (fits && out.rows_sum) atomicAdd(out.rows_sum, (unsigned long long)count);
    *s_base = fits ? 0 : -1;
  }
  __syncthreads();
  return *s_base;
}

// Publishes `count` for the chunk and returns its base (or -1: stop).
__device__ __forceinline__ long long chunk_base(const LookBack& lb, const OutSink& out, int cid,
                                                long long count, long long* s_base) {
  if (threadIdx.x < 32) {
    long long b = lookback_warp(lb, cid, count);
    if (threadIdx.x == 0) {
      *s_base = b;
      if (b >= 0 && lb.total_out && cid == lb.n_chunks - 1) *lb.total_out = b + count;
      if (b >= 0 && b + count > out.capacity) err_raise(lb.err, ERR_CAPACITY);
    }
  }
  __syncthreads();
  return *s_base;
}

// ---------------------------------------------------------------------------
// Fold.  Each warp takes a contiguous, 32-aligned range of sorted positions,
// a lane per position; heads (first rows of key groups) come from a ballot,
// output positions from popc and one scan over warps, so consecutive lanes
// write consecutive rows.  The warp folds the groups whose heads lie in its
// range, by a lane per group or by segmented scans (fold_scan).
// ---------------------------------------------------------------------------
__shared__ int g_lcnt[kWarps + 1];

// Stage source column c of every chunk row into dst in sorted order (row i
// to dst[inv[i]]): 8-byte cp.async copies, global to shared, read in chunk
// order and all in flight at once; complete when it returns (visible to the
// other threads after a barrier).
template <int MODE>
__device__ __forceinline__ void stage_column(const RowSrc& src, const ChunkView& cv, int c, const uint16_t* inv,
                                             long long* dst) {
  for (int i = threadIdx.x; i < cv.n; i += kThreads) {
    const long long* p;
    if (MODE == MODE_RANGE) {
      p = src.aos + (cv.lo + i) * (1 + src.ncols) + 1 + c;
    } else {
      const int64_t row = src.offset + cv.lo + i;
      p = src.kind == SRC_AOS ? src.aos + row * (1 + src.ncols) + 1 + c : src.cols[c] + row;
    }
    cp_async8(&dst[inv[i]], p);
  }
  cp_async_wait();
}

__device__ __forceinline__ bool head_bit(const uint32_t* hm, int p) { return (hm[p >> 5] >> (p & 31)) & 1u; }

// End (exclusive) of the key group starting at head position p.
__device__ __forceinline__ int group_end(const uint32_t* hm, int p, int n) {
  int q = p + 1;
  while (q < n) {
    const uint32_t w = hm[q >> 5] >> (q & 31);
    if (w) return q + __ffs(w) - 1;
    q = (q | 31) + 1;
  }
  return n;
}

__shared__ int g_gstart[kFewGroups + 1];
__shared__ long long g_gacc[kWarps * kAccBlock];

// Few key groups: the CTA reduces one group at a time (positions in
// g_gstart), kAccBlock aggregates of source column c per sweep.
__device__ void fold_few(const SortSmem& s, const FoldDesc& fd, const OutSink& out,
                                      const long long* col, int c, int count, long long base) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ns = fd.n_state;
  for (int g = 0; g < count; ++g) {
    const int gs = g_gstart[g], ge = g_gstart[g + 1];
    for (int s0 = 0; s0 < ns; s0 += kAccBlock) {
      bool any = false;
      for (int a = 0; a < kAccBlock && s0 + a < ns; ++a) any |= (fd.src[s0 + a] == c);
      if (!any) continue;  // block-uniform
      long long acc[kAccBlock];
#pragma unroll
      for (int a = 0; a < kAccBlock; ++a)
        if (s0 + a < ns) acc[a] = op_identity(fd.op[s0 + a]);
      for (int p = gs + threadIdx.x; p < ge; p += kThreads) {
        const long long v = col[p];
#pragma unroll
        for (int a = 0; a < kAccBlock; ++a)
          if (s0 + a < ns && fd.src[s0 + a] == c) acc[a] = op_combine(fd.op[s0 + a], acc[a], v);
      }
#pragma unroll
      for (int a = 0; a < kAccBlock; ++a)
        if (s0 + a < ns && fd.src[s0 + a] == c) {
          const long long v = warp_reduce(fd.op[s0 + a], acc[a]);
          if (lane == 0) g_gacc[w * kAccBlock + a] = v;
        }
      __syncthreads();
      if (threadIdx.x < kAccBlock && s0 + (int)threadIdx.x < ns && fd.src[s0 + threadIdx.x] == c) {
        const int a = threadIdx.x, op = fd.op[s0 + a];
        long long v = op_identity(op);
        for (int ww = 0; ww < kWarps; ++ww) v = op_combine(op, v, g_gacc[ww * kAccBlock + a]);
        sink_val(out, s0 + a, base + g, v);
      }
      __syncthreads();
    }
  }
}

template <int OP>
__device__ __forceinline__ long long op_id() {
  return OP == OP_SUM ? 0 : (OP == OP_MIN ? INT64_MAX : INT64_MIN);
}

template <int OP>
__device__ __forceinline__ long long op_do(long long a, long long b) {
  if (OP == OP_SUM) return (long long)((unsigned long long)a + (unsigned long long)b);
  if (OP == OP_MIN) return b < a ? b : a;
  return b > a ? b : a;
}

// A warp's key groups (those whose heads lie in its position range), folded
// over their sorted positions [fh, xe) of col: per 32-position window a
// segmented inclusive scan (a segment starts at a head bit), the open
// group's value carried from window to window (a window inside one group
// only adds lane partials); the lane at a group's last position writes the
// group's value to dst[base + group ordinal].
template <int OP>
__device__ void fold_scan(const uint32_t* hm, const uint16_t* hpre, const long long* col, int n, int fh, int xe,
                          long long* dst, long long cap, long long base) {
  const int lane = threadIdx.x & 31;
  const unsigned below = 0xffffffffu >> (31 - lane);  // lanes 0..lane
  long long carry = op_id<OP>(), lacc = op_id<OP>();
  bool pend = false;  // warp-uniform: lane partials not yet in carry
  for (int b = fh & ~31; b < xe; b += 32) {
    const unsigned hb = hm[b >> 5];
    const unsigned hn = b + 32 < n ? hm[(b >> 5) + 1] : 1u;  // next window's heads (past n: a head)
    const int p = b + lane;
    const bool own = p >= fh && p < xe;
    const long long v0 = own ? col[p] : op_id<OP>();
    if (hb == 0 && b >= fh && !(hn & 1u) && b + 32 < xe) {
      // warp-uniform: the window lies inside one group, which goes on after it
      lacc = op_do<OP>(lacc, v0);
      pend = true;
      continue;
    }
    if (pend) {
      for (int o = 16; o > 0; o >>= 1) lacc = op_do<OP>(lacc, __shfl_xor_sync(0xffffffffu, lacc, o));
      carry = op_do<OP>(carry, lacc);
      lacc = op_id<OP>();
      pend = false;
    }
    const unsigned le = hb & below;  // heads at or below the lane
    const int ss = 31 - __clz(le);   // its group's head lane; -1: an earlier window
    const int d = lane - max(ss, 0); // earlier lanes of its group in this window
    const int dmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)d);
    long long v = v0;
    for (int o = 1; o <= dmax; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (o <= d) v = op_do<OP>(v, u);
    }
    if (ss < 0) v = op_do<OP>(v, carry);
    carry = __shfl_sync(0xffffffffu, v, 31);
    // the last position of a group: the next one is a head (or the range ends)
    const unsigned lastm = (hb >> 1) | (hn << 31);
    if (own && (((lastm >> lane) & 1u) || p + 1 == xe)) {
      const long long pos = base + (long long)hpre[b >> 5] + __popc(le) - 1;
      if (pos < cap) dst[pos] = v;
    }
  }
}

// fold_scan for the report pattern of one column -- its sum, min and max --
// in one pass: the windows, head masks, segment lengths and value loads are
// shared and the three scans interleaved; same results as fold_scan once per
// aggregate.
__device__ void fold_scan_smm(const uint32_t* hm, const uint16_t* hpre, const long long* col, int n, int fh, int xe,
                              long long* dsum, long long* dmin, long long* dmax_, long long cap, long long base) {
  const int lane = threadIdx.x & 31;
  const unsigned below = 0xffffffffu >> (31 - lane);
  long long cs = op_id<OP_SUM>(), cn = op_id<OP_MIN>(), cx = op_id<OP_MAX>();
  long long ls = cs, ln = cn, lx = cx;
  bool pend = false;  // warp-uniform: lane partials not yet in the carries
  for (int b = fh & ~31; b < xe; b += 32) {
    const unsigned hb = hm[b >> 5];
    const unsigned hn = b + 32 < n ? hm[(b >> 5) + 1] : 1u;  // next window's heads (past n: a head)
    const int p = b + lane;
    const bool own = p >= fh && p < xe;
    const long long raw = own ? col[p] : 0;
    const long long vs = own ? raw : op_id<OP_SUM>(), vn = own ? raw : op_id<OP_MIN>(),
                    vx = own ? raw : op_id<OP_MAX>();
    if (hb == 0 && b >= fh && !(hn & 1u) && b + 32 < xe) {
      // warp-uniform: the window lies inside one group, which goes on after it
      ls = op_do<OP_SUM>(ls, vs);
      ln = op_do<OP_MIN>(ln, vn);
      lx = op_do<OP_MAX>(lx, vx);
      pend = true;
      continue;
    }
    if (pend) {
      for (int o = 16; o > 0; o >>= 1) {
        ls = op_do<OP_SUM>(ls, __shfl_xor_sync(0xffffffffu, ls, o));
        ln = op_do<OP_MIN>(ln, __shfl_xor_sync(0xffffffffu, ln, o));
        lx = op_do<OP_MAX>(lx, __shfl_xor_sync(0xffffffffu, lx, o));
      }
      cs = op_do<OP_SUM>(cs, ls);
      cn = op_do<OP_MIN>(cn, ln);
      cx = op_do<OP_MAX>(cx, lx);
      ls = op_id<OP_SUM>();
      ln = op_id<OP_MIN>();
      lx = op_id<OP_MAX>();
      pend = false;
    }
    const unsigned le = hb & below;  // heads at or below the lane
    const int ss = 31 - __clz(le);   // its group's head lane; -1: an earlier window
    const int d = lane - max(ss, 0); // earlier lanes of its group in this window
    const int dm = (int)__reduce_max_sync(0xffffffffu, (unsigned)d);
    long long xs = vs, xn = vn, xx = vx;
    for (int o = 1; o <= dm; o <<= 1) {
      const long long us = __shfl_up_sync(0xffffffffu, xs, o);
      const long long un = __shfl_up_sync(0xffffffffu, xn, o);
      const long long ux = __shfl_up_sync(0xffffffffu, xx, o);
      if (o <= d) {
        xs = op_do<OP_SUM>(xs, us);
        xn = op_do<OP_MIN>(xn, un);
        xx = op_do<OP_MAX>(xx, ux);
      }
    }
    if (ss < 0) {
      xs = op_do<OP_SUM>(xs, cs);
      xn = op_do<OP_MIN>(xn, cn);
      xx = op_do<OP_MAX>(xx, cx);
    }
    cs = __shfl_sync(0xffffffffu, xs, 31);
    cn = __shfl_sync(0xffffffffu, xn, 31);
    cx = __shfl_sync(0xffffffffu, xx, 31);
    // the last position of a group: the next one is a head (or the range ends)
    const unsigned lastm = (hb >> 1) | (hn << 31);
    if (own && (((lastm >> lane) & 1u) || p + 1 == xe)) {
      const long long pos = base + (long long)hpre[b >> 5] + __popc(le) - 1;
      if (pos < cap) {
        dsum[pos] = xs;
        dmin[pos] = xn;
        dmax_[pos] = xx;
      }
    }
  }
}

// Fold the sorted chunk: heads (first rows of key groups) into a bitmask and
// the chunk's distinct-key count -> its output offset by look-back; keys and
// count(*) per head; then the aggregates one source column at a time, the
// column staged in sorted order in shared memory where the keys were.  Each
// warp folds the groups whose heads lie in its position range: a lane per
// group where nearly every row is a group of its own, else by segmented
// scans (fold_scan); with at most kFewGroups groups (possible only when the
// sort says that groups may exceed 32 rows) the whole CTA folds one group at
// a time.
template <int MODE, int KS, bool BIGS>
__device__ void fold_sorted(const SortSmem& s, const RowSrc& src, const ChunkView& cv,
                            const FoldDesc& fd, const OutSink& out, const LookBack& lb, const Chunk& ch,
                            int cid, long long* s_base) {
  const int n = cv.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1;
  const int Q = ((n + kWarps - 1) / kWarps + 31) & ~31;
  const int wb = min(n, w * Q), we = min(n, wb + Q);
  // the sort is done with the bins and the histogram area
  uint32_t* hm = reinterpret_cast<uint32_t*>(s.whist);                   // head bitmask
  uint16_t* hpre = s.whist + kTileCap / 32 * 2;                           // heads before each word
  uint16_t* inv = reinterpret_cast<uint16_t*>(s.bins);                    // sorted position of row i
  // pass 1: heads -> bitmask, per-warp counts (warp ranges are 32-aligned);
  // the inverse permutation
  int hc = 0;
  for (int b = wb; b < we; b += 32) {
    const int p = b + lane;
    const int ip = p < we ? s.idx[p] : 0;
    const unsigned long long kp = s.keys[ip];
    unsigned long long kq = __shfl_up_sync(0xffffffffu, kp, 1);
    if (lane == 0 && p > 0) kq = s.keys[s.idx[p - 1]];
    bool h = false;
    if (p < we) {
      h = (p == 0) || kp != kq;
      inv[ip] = (uint16_t)p;
    }
    const unsigned hb = __ballot_sync(0xffffffffu, h);
    if (lane == 0) {
      hm[b >> 5] = hb;
      hpre[b >> 5] = (uint16_t)hc;  // warp-local; the warp's prefix is added below
    }
    hc += __popc(hb);
  }
  if (lane == 0) g_lcnt[w] = hc;
  __syncthreads();
  if (w == 0) {
    int v = lane < kWarps ? g_lcnt[lane] : 0, x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < kWarps) g_lcnt[lane] = x - v;
    if (lane == kWarps - 1) g_lcnt[kWarps] = x;
  }
  __syncthreads();
  const int count = g_lcnt[kWarps];
  const bool few = BIGS && count <= kFewGroups;
  for (int b = wb + 32 * lane; b < we; b += 32 * 32) hpre[b >> 5] += (uint16_t)g_lcnt[w];
  // mostly one-row groups (three heads in four positions or more, each group
  // within 32 rows): a lane folds each group; otherwise segmented scans
  const bool lanefold = !BIGS && 4 * hc >= 3 * (we - wb);
  // the warp's groups for the scans: heads in [wb, we), positions [fh, xe)
  // (a word of hm lies inside one warp's range)
  int fh = n, xe = 0;
  if (!few && !lanefold) {
    int lh = -1;
    for (int b0 = wb; b0 < we; b0 += 32 * 32) {
      const int b = b0 + 32 * lane;
      const unsigned x = b < we ? hm[b >> 5] : 0u;
      const unsigned nz = __ballot_sync(0xffffffffu, x != 0);
      if (nz) {  // warp-uniform
        const int l0 = __ffs(nz) - 1, l1 = 31 - __clz(nz);
        const unsigned x0 = __shfl_sync(0xffffffffu, x, l0), x1 = __shfl_sync(0xffffffffu, x, l1);
        fh = min(fh, b0 + 32 * l0 + __ffs(x0) - 1);
        lh = b0 + 32 * l1 + 31 - __clz(x1);
      }
    }
    if (lh >= 0) xe = group_end(hm, lh, n);
  }
  const long long base =
      MODE == MODE_DIRECT ? direct_base(out, count, s_base) : chunk_base(lb, out, cid, count, s_base);
  if (base < 0) return;
  // the run's sparse index (several runs at once: the chunk's own run's)
  long long* const offs =
      (MODE == MODE_RANGE && out.offs && out.offs_stride > 0)
          ? out.offs + (long long)(ch.pad >> out.offs_bbits) * out.offs_stride : out.offs;
  if (offs && count == 0 && threadIdx.x == 0)
    for (int ff = ch.f_lo; ff <= ch.f_hi; ++ff) offs[ff] = base;
  const int ns = fd.n_state;
  // keys, count(*) of raw rows
  {
    int run = g_lcnt[w];
    for (int b = wb; b < we; b += 32) {
      const int p = b + lane;
      const unsigned hb = hm[b >> 5];
      if ((hb >> lane) & 1u) {
        const int g = run + __popc(hb & lt);
        const long long pos = base + g;
        sink_key(out, pos, s.keys[s.idx[p]]);
        int e = -1;
#pragma unroll(KS <= 8 ? KS : 1)
        for (int a = 0; a < KS; ++a)
          if (a < ns && fd.src[a] < 0) {
            if (e < 0) e = group_end(hm, p, n);
            sink_val(out, a, pos, fd.op[a] == OP_SUM ? (long long)(e - p) : 1);
          }
        if (few) g_gstart[g] = p;
      }
      run += __popc(hb);
    }
  }
  // the run's sparse index: offs[f] = rows of this run before the first key
  // with fine digit >= f, for every fine bucket of the chunk's key range (a
  // thread per fine bucket, by binary search over the sorted rows)
  if (offs) {
    for (int f = ch.f_lo + (int)threadIdx.x; f <= ch.f_hi; f += kThreads) {
      int lo = 0, hi = n;  // first sorted position whose fine digit is >= f
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)fine_digit(out.dig, s.keys[s.idx[mid]]) < f) lo = mid + 1; else hi = mid;
      }
      const int heads = lo >= n ? count
                                : (int)hpre[lo >> 5] + __popc(hm[lo >> 5] & ((1u << (lo & 31)) - 1u));
      offs[f] = base + heads;
    }
  }
  if (few && threadIdx.x == 0) g_gstart[count] = n;
  // aggregates, one source column at a time
  long long* col = reinterpret_cast<long long*>(s.keys);
  const int ncols = src.ncols;
  for (int c = 0; c < ncols; ++c) {
    bool used = false;
    for (int a = 0; a < ns; ++a) used |= (fd.src[a] == c);
    if (!used) continue;  // block-uniform
    __syncthreads();      // everyone is done with the previous contents (keys, offsets, column)
    stage_column<MODE>(src, cv, c, inv, col);
    __syncthreads();
    if (few) {
      fold_few(s, fd, out, col, c, count, base);
      continue;
    }
    // the report pattern on this column (exactly a sum, a min and a max):
    // folded in one pass (block-uniform)
    int a_sum = -1, a_min = -1, a_max = -1, n_on = 0;
    for (int a = 0; a < ns; ++a) {
      if (fd.src[a] != c) continue;
      ++n_on;
      if (fd.op[a] == OP_SUM) a_sum = a; else if (fd.op[a] == OP_MIN) a_min = a; else a_max = a;
    }
    // (compiled only where three aggregates fit: KS >= 3)
    const bool smm = KS >= 3 && n_on == 3 && a_sum >= 0 && a_min >= 0 && a_max >= 0;
    if (lanefold && smm) {
      int run = g_lcnt[w];
      for (int b = wb; b < we; b += 32) {
        const int p = b + lane;
        const unsigned hb = hm[b >> 5];
        if ((hb >> lane) & 1u) {
          const long long pos = base + run + __popc(hb & lt);
          const int e = group_end(hm, p, n);
          long long as = col[p], an = as, ax = as;
          for (int q = p + 1; q < e; ++q) {
            const long long v = col[q];
            as = op_do<OP_SUM>(as, v);
            an = op_do<OP_MIN>(an, v);
            ax = op_do<OP_MAX>(ax, v);
          }
          sink_val(out, a_sum, pos, as);
          sink_val(out, a_min, pos, an);
          sink_val(out, a_max, pos, ax);
        }
        run += __popc(hb);
      }
      continue;
    }
    if (lanefold) {
      // a lane per group (every group has at most 32 rows)
      int run = g_lcnt[w];
      for (int b = wb; b < we; b += 32) {
        const int p = b + lane;
        const unsigned hb = hm[b >> 5];
        if ((hb >> lane) & 1u) {
          const long long pos = base + run + __popc(hb & lt);
          const int e = group_end(hm, p, n);
#pragma unroll(KS <= 8 ? KS : 1)
          for (int a = 0; a < KS; ++a) {
            if (a < ns && fd.src[a] == c) {
              const int op = fd.op[a];
              long long acc = col[p];
              for (int q = p + 1; q < e; ++q) acc = op_combine(op, acc, col[q]);
              sink_val(out, a, pos, acc);
            }
          }
        }
        run += __popc(hb);
      }
      continue;
    }
    if (fh >= xe) continue;  // warp-uniform: no group of this warp
    if (smm) {
      fold_scan_smm(hm, hpre, col, n, fh, xe, out.cols[a_sum], out.cols[a_min], out.cols[a_max], out.capacity,
                    base);
      continue;
    }
#pragma unroll(KS <= 8 ? KS : 1)
    for (int a = 0; a < KS; ++a) {
      if (a < ns && fd.src[a] == c) {
        const int op = fd.op[a];
        if (op == OP_SUM) fold_scan<OP_SUM>(hm, hpre, col, n, fh, xe, out.cols[a], out.capacity, base);
        else if (op == OP_MIN) fold_scan<OP_MIN>(hm, hpre, col, n, fh, xe, out.cols[a], out.capacity, base);
        else fold_scan<OP_MAX>(hm, hpre, col, n, fh, xe, out.cols[a], out.capacity, base);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <int MODE, int KS>
__global__ void __launch_bounds__(kThreads, 2)
k_sortfold(const Chunk* __restrict__ chunks, RowSrc src_param, CopySrc copy, FoldDesc fd,
           OutSink out, LookBack lb, long long tile_n, int tile_f_hi, InstSet is) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem s = carve(smem_raw);
  __shared__ RowSrc s_src;   // MODE_INST / MODE_DIRECT: the chunk's instance as a source
  __shared__ OutSink s_out;  // MODE_DIRECT: the instance's outputs
  __shared__ int s_cid;
  __shared__ int s_err;
  __shared__ long long s_base;
  __shared__ int s_n;

  if (threadIdx.x == 0) {
    s_cid = (int)atomicAdd(lb.ticket, 1u);
    s_err = err_load(lb.err);
    g_kmin = ~0ull;
    g_kmax = 0ull;
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
  if (MODE == MODE_INST || MODE == MODE_DIRECT) {
    if (threadIdx.x == 0) {
      const InstDesc d = is.inst[ch.pad];
      s_src = src_param;
      s_src.kind = SRC_RAW;
      s_src.offset = 0;
      s_src.key.n_cols = 1;
      s_src.key.bytes[0] = d.key_bytes;
      s_src.key.shift[0] = 0;
      s_src.key.cols[0] = d.keys;
      s_src.key_or = MODE == MODE_INST ? (unsigned long long)ch.pad << is.key_bits : 0ull;
      for (int c = 0; c < src_param.ncols; ++c) s_src.cols[c] = d.payload[is.colsel[c]];
      if (MODE == MODE_DIRECT) {
        // the instance's own outputs, its key width
        s_out = out;
        s_out.user = 1;
        s_out.kout.n_cols = 1;
        s_out.kout.bytes[0] = d.key_bytes;
        s_out.kout.shift[0] = 0;
        s_out.kout.cols[0] = d.out_keys;
        for (int a = 0; a < fd.n_state; ++a) s_out.cols[a] = d.out_aggs[a];
        s_out.capacity = d.out_capacity;
        s_out.offs = nullptr;
        s_out.rows_out = d.out_rows;
      }
    }
    __syncthreads();
  }
  const RowSrc& src = (MODE == MODE_INST || MODE == MODE_DIRECT) ? s_src : src_param;
  const OutSink& dst = (MODE == MODE_DIRECT) ? s_out : out;

  if (ch.kind == CH_COPY) {
    const long long n = ch.hi - ch.lo;
    const long long base = chunk_base(lb, out, cid, n, &s_base);
    if (base < 0) return;
    for (long long g = threadIdx.x; g < n; g += kThreads) {
      unsigned long long key = copy.keys[ch.lo + g];
      sink_key(out, base + g, key);
      if (out.offs)
        write_fine_offsets(out, ch, base, g, n, key, g > 0, g > 0 ? copy.keys[ch.lo + g - 1] : 0ull);
      for (int st = 0; st < fd.n_state; ++st) sink_val(out, st, base + g, copy.cols[st][ch.lo + g]);
    }
    if (out.offs && n == 0 && threadIdx.x == 0)
      for (int ff = ch.f_lo; ff <= ch.f_hi; ++ff) out.offs[ff] = base;
    return;
  }

  ChunkView cv;
  cv.lo = ch.lo;
  if (threadIdx.x == 0) s_n = (int)(ch.hi - ch.lo);
  __syncthreads();
  cv.n = s_n;
  if (cv.n > kTileCap) {  // the planner never makes such chunks
    if (threadIdx.x == 0) err_raise(lb.err, ERR_INTERNAL);
    return;
  }
  unsigned long long lmin = ~0ull, lmax = 0ull;
  load_keys<MODE>(s, src, cv, &lmin, &lmax);
  // its first barrier completes the load
  const bool bigs = chunk_sort(s, cv.n, lmin, lmax, (MODE == MODE_TILES || MODE == MODE_INST) && is.grouped);
  if (MODE == MODE_INST && is.kmin && threadIdx.x == 0 && cv.n > 0) {
    // key range of the instance (the tile's least and greatest keys, all
    // of one instance), for the digit that partitions the partial rows
    const unsigned long long m = (1ull << is.key_bits) - 1;
    atomicMin(is.kmin + ch.pad, g_kmin & m);
    atomicMax(is.kmax + ch.pad, g_kmax & m);
  }
  if (bigs) fold_sorted<MODE, KS, true>(s, src, cv, fd, dst, lb, ch, cid, &s_base);
  else fold_sorted<MODE, KS, false>(s, src, cv, fd, dst, lb, ch, cid, &s_base);
}

}  // namespace sg
