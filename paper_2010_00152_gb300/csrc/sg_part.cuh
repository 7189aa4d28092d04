// sg_part.cuh -- partitioning a batch by key range before the per-chunk sort.
//
// A batch of up to M rows (one read-sort-write cycle, Sec. 3 / Sec. 6.1) is
// too large for one CTA, so it is first split by a most-significant digit of
// the key into buckets that are key ranges in key order:
//   k_hist     per-tile histogram of the coarse digit (one read of the keys);
//   k_tilescan per bucket, exclusive scan over tiles -> each tile's write
//              offset inside the bucket; bucket totals;
//   k_plan_*   bucket starts, and a grouping of consecutive buckets into
//              chunks of at most kTileCap rows; a bucket of more than a
//              chunk is set apart (solved separately, then copied in);
//   k_scatter  every row written once to its bucket (rows of 1 + ncols words).
// The same planner groups the fine buckets of the wide merge into merge
// tiles (k_fine_sizes gives each fine bucket's row count over all runs).
#pragma once
#include "sg_sortfold.cuh"

namespace sg {

constexpr int kPartThreads = 512;
constexpr int kPrivBuckets = 256;   // per-warp private histograms up to this many buckets

// Keys of `count` rows spread evenly over [0, n), for the planner's probe.
// Row floor(i * n / count) for sample i, in 64-bit arithmetic: with
// n = q * count + rem, it is i * q + floor(i * rem / count) (i, rem < count).
__global__ void k_sample(RowSrc src, long long n, int count, unsigned long long* out) {
  const long long q = n / count, rem = n % count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const long long r = (long long)i * q + ((long long)i * rem) / count;
    out[i] = src_key(src, r);
  }
}

// mm[0] = min key, mm[1] = max key over n rows (mm preset to {~0, 0}).
__global__ void k_minmax(RowSrc src, long long n, unsigned long long* mm) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long k = src_key(src, i);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
    unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
}

__device__ __forceinline__ void tile_range(long long n, int ntiles, int t, long long* lo, long long* hi) {
  long long per = (n + ntiles - 1) / ntiles;
  *lo = min(n, (long long)t * per);
  *hi = min(n, *lo + per);
}

// Rows [lo, hi) of launch tile t, and the bucket offset of its batch (0
// unless the digit partitions several batches at once).
__device__ __forceinline__ unsigned tile_rows(long long n, int ntiles, const Digit& dig, int t, long long* lo,
                                              long long* hi) {
  if (dig.brows == 0) {
    tile_range(n, ntiles, t, lo, hi);
    return 0u;
  }
  const int b = t / dig.btiles;
  const long long b0 = (long long)b * dig.brows;
  tile_range(max(0ll, min(n, b0 + dig.brows) - b0), dig.btiles, t % dig.btiles, lo, hi);
  *lo += b0;
  *hi += b0;
  return (unsigned)b << dig.bbits;
}

// Digit of one partitioning level: bits [dshift, dshift + log2(nb)) of the
// coarse digit.
template <bool SEG>
__device__ __forceinline__ unsigned level_digit(const Digit& dig, unsigned long long k, int dshift, int nb) {
  return (coarse_digit<SEG>(dig, k) >> dshift) & (unsigned)(nb - 1);
}

// thist[d * ntiles + t] = rows of tile t with level digit d.
template <bool SEG, bool DIRECT>
__global__ void __launch_bounds__(kPartThreads)
k_hist(RowSrc src, long long n, Digit dig, int dshift, int nb, int ntiles, unsigned int* thist) {
  extern __shared__ unsigned int sh_hist[];
  // up to 256 buckets: one private histogram per warp (no cross-warp atomic
  // contention), summed at the end; more buckets: one shared histogram
  const bool priv = nb <= kPrivBuckets;
  unsigned* mine = priv ? sh_hist + (threadIdx.x >> 5) * nb : sh_hist;
  const int nh = priv ? nb * (blockDim.x >> 5) : nb;
  for (int d = threadIdx.x; d < nh; d += blockDim.x) sh_hist[d] = 0;
  __syncthreads();
  long long lo, hi;
  const unsigned boff = tile_rows(n, ntiles, dig, blockIdx.x, &lo, &hi);
  const int nlev = dig.brows ? (1 << dig.bbits) : nb;  // buckets of one batch
  // independent loads in flight per thread: the grid is two CTAs per SM (the
  // scatter's tiles), so each thread keeps 16 keys (128 B) coming
  constexpr int U = 16;
  for (long long i0 = lo + threadIdx.x; i0 < hi; i0 += (long long)U * blockDim.x) {
    unsigned long long k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long i = i0 + (long long)u * blockDim.x;
      if (i < hi) k[u] = DIRECT ? __ldg(src_key_ptr(src, i)) : src_key(src, i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long i = i0 + (long long)u * blockDim.x;
      if (i < hi) atomicAdd(&mine[boff + level_digit<SEG>(dig, k[u], dshift, nlev)], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nb; d += blockDim.x) {
    unsigned v = sh_hist[d];
    if (priv)
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v += sh_hist[w * nb + d];
    thist[(long long)d * ntiles + blockIdx.x] = v;
  }
}

inline size_t hist_smem_bytes(int nb, int threads) {
  return (size_t)(nb <= 256 ? nb * (threads / 32) : nb) * 4;
}

// One warp per bucket: exclusive scan of thist over tiles (in place), total.
__global__ void k_tilescan(unsigned int* thist, int nb, int ntiles, long long* btot) {
  int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (wid >= nb) return;
  unsigned int* row = thist + (long long)wid * ntiles;
  unsigned int run = 0;
  for (int b = 0; b < ntiles; b += 32) {
    int t = b + lane;
    unsigned int v = t < ntiles ? row[t] : 0u;
    unsigned int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (t < ntiles) row[t] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) btot[wid] = run;
}

// Planner result read back by the host.
struct PlanInfo {
  int n_chunks;
  int n_big;
  long long total;
  long long max_chunk;
};

// The chunk plan (k_plan_* below).  w[0..nb) are bucket row counts in key
// order.  It writes bstart (exclusive prefix, nb + 1 entries), the chunk list
// and the indices of big chunks.  A bucket with more than `big` rows is a
// chunk of its own: kind
// CH_NORMAL up to `cap` rows, else CH_COPY (solved separately, listed in
// big_list).  Other buckets are grouped while their exclusive prefix over
// buckets of at most `big` rows stays in one multiple of `target`, so such a
// chunk holds fewer than target + big rows.  Chunk c covers buckets
// [d_lo, d_hi), i.e. fine range [d_lo << fine_shift, d_hi << fine_shift).
__device__ __forceinline__ bool plan_is_start(long long x, long long big, long long pB, long long target,
                                              bool* prev_big, long long* prev_q) {
  bool isbig = x > big;
  bool st;
  if (isbig) {
    st = true;
  } else {
    long long q = pB / target;
    st = *prev_big || q != *prev_q;
    *prev_q = q;
  }
  *prev_big = isbig;
  return st;
}


// ---------------------------------------------------------------------------
// The same plan computed by several blocks (k_plan_*): block b owns buckets
// [b * per, (b + 1) * per), a thread `sub` consecutive ones of them.
//   sums:   per-block rows of all / small buckets and big-bucket count;
//   scan3:  exclusive prefixes of the three (one block), totals into info;
//   starts: chunk starts per block (they need the global small-row prefix);
//   scan1:  exclusive prefix of the starts (one block), chunk count;
//   apply:  bucket starts, chunk first buckets and kinds, the big list;
//   finish: chunk ends, row ranges, fine ranges, the largest chunk.
// ---------------------------------------------------------------------------
constexpr int kPlanThreads = 256;

__device__ __forceinline__ long long block_sum_ll(long long v, long long* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
  return t;
}

// exclusive prefix of v over the block (blockDim.x <= 1024)
__device__ __forceinline__ long long block_excl_ll(long long v, long long* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[w] = x;
  __syncthreads();
  long long before = 0;
  for (int k = 0; k < w; ++k) before += red[k];
  return before + x - v;
}

__global__ void __launch_bounds__(kPlanThreads)
k_plan_sums(const long long* __restrict__ w, int nb, int per, int sub, long long big, long long cap, long long* part) {
  __shared__ long long red[32];
  const int d0 = min(nb, blockIdx.x * per + (int)threadIdx.x * sub), d1 = min(min(nb, (blockIdx.x + 1) * per), d0 + sub);
  long long ta = 0, tb = 0, tc = 0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    ta += x;
    if (x > cap) tc += 1;
    if (x <= big) tb += x;
  }
  ta = block_sum_ll(ta, red);
  tb = block_sum_ll(tb, red);
  tc = block_sum_ll(tc, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = ta;
    part[3 * blockIdx.x + 1] = tb;
    part[3 * blockIdx.x + 2] = tc;
  }
}

// exclusive prefix over g entries of stride `stride` (one block of 1024)
__device__ void scan_column(long long* v, int g, int stride, long long* total) {
  __shared__ long long red[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < g; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    const long long x = b < g ? v[(long long)b * stride] : 0;
    const long long ex = block_excl_ll(x, red);
    const long long c = carry;
    __syncthreads();
    if (b < g) v[(long long)b * stride] = c + ex;
    if (threadIdx.x == blockDim.x - 1) carry = c + ex + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(1024)
k_plan_scan3(long long* part, int g, int nb, long long* bstart, PlanInfo* info) {
  __shared__ long long tot[3];
  for (int k = 0; k < 3; ++k) {
    scan_column(part + k, g, 3, &tot[k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    info->total = tot[0];
    info->n_big = (int)tot[2];
    info->max_chunk = 0;
    bstart[nb] = tot[0];
  }
}

// state of bucket d0 - 1 (the one before a thread's range) from the small-row
// prefix B0 at d0, as k_plan computes it
__device__ __forceinline__ void plan_prev(const long long* w, int d0, long long B0, long long big, long long target,
                                          bool* pb, long long* pq) {
  *pb = true;
  *pq = -1;
  if (d0 > 0) {
    const long long x = w[d0 - 1];
    *pb = x > big;
    *pq = *pb ? -1 : (B0 - x) / target;
  }
}

__global__ void __launch_bounds__(kPlanThreads)
k_plan_starts(const long long* __restrict__ w, int nb, int per, int sub, long long target, long long big,
              const long long* part, long long* starts) {
  __shared__ long long red[32];
  const int d0 = min(nb, blockIdx.x * per + (int)threadIdx.x * sub), d1 = min(min(nb, (blockIdx.x + 1) * per), d0 + sub);
  long long tb = 0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    if (x <= big) tb += x;
  }
  const long long B0 = part[3 * blockIdx.x + 1] + block_excl_ll(tb, red);
  bool pbig;
  long long pq, pB = B0;
  plan_prev(w, d0, B0, big, target, &pbig, &pq);
  long long st = 0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    st += plan_is_start(x, big, pB, target, &pbig, &pq);
    if (x <= big) pB += x;
  }
  st = block_sum_ll(st, red);
  if (threadIdx.x == 0) starts[blockIdx.x] = st;
}

__global__ void __launch_bounds__(1024) k_plan_scan1(long long* starts, int g, PlanInfo* info) {
  __shared__ long long tot;
  scan_column(starts, g, 1, &tot);
  __syncthreads();
  if (threadIdx.x == 0) info->n_chunks = (int)tot;
}

__global__ void __launch_bounds__(kPlanThreads)
k_plan_apply(const long long* __restrict__ w, int nb, int per, int sub, long long target, long long big,
             long long cap, const long long* part, const long long* starts, long long* bstart, Chunk* chunks,
             int* big_list) {
  __shared__ long long red[32];
  const int d0 = min(nb, blockIdx.x * per + (int)threadIdx.x * sub), d1 = min(min(nb, (blockIdx.x + 1) * per), d0 + sub);
  long long ta = 0, tb = 0, tc = 0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    ta += x;
    if (x > cap) tc += 1;
    if (x <= big) tb += x;
  }
  const long long A0 = part[3 * blockIdx.x] + block_excl_ll(ta, red);
  const long long B0 = part[3 * blockIdx.x + 1] + block_excl_ll(tb, red);
  long long nbig = part[3 * blockIdx.x + 2] + block_excl_ll(tc, red);
  bool pbig;
  long long pq, pB = B0;
  plan_prev(w, d0, B0, big, target, &pbig, &pq);
  long long st = 0;
  {
    bool pb2 = pbig;
    long long pq2 = pq, pB2 = B0;
    for (int d = d0; d < d1; ++d) {
      const long long x = w[d];
      st += plan_is_start(x, big, pB2, target, &pb2, &pq2);
      if (x <= big) pB2 += x;
    }
  }
  long long cidx = starts[blockIdx.x] + block_excl_ll(st, red) - 1;
  long long pA = A0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    bstart[d] = pA;
    if (plan_is_start(x, big, pB, target, &pbig, &pq)) {
      ++cidx;
      chunks[cidx].pad = d;  // first bucket (its fine range is set by k_plan_finish)
      chunks[cidx].kind = x > cap ? CH_COPY : CH_NORMAL;
      if (x > cap) big_list[nbig++] = (int)cidx;
    }
    if (x <= big) pB += x;
    pA += x;
  }
}

__global__ void k_plan_finish(int nb, int fine_shift, const long long* bstart, Chunk* chunks, PlanInfo* info) {
  const int nc = info->n_chunks;
  long long mx = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const int dlo = chunks[c].pad;
    const int dhi = (c + 1 < nc) ? chunks[c + 1].pad : nb;
    Chunk& ch = chunks[c];
    ch.lo = bstart[dlo];
    ch.hi = bstart[dhi];
    ch.f_lo = dlo << fine_shift;
    ch.f_hi = dhi << fine_shift;
    if (ch.kind == CH_NORMAL) mx = max(mx, ch.hi - ch.lo);
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0)
    atomicMax(reinterpret_cast<unsigned long long*>(&info->max_chunk), (unsigned long long)mx);
}

// The same plan in one launch of one block, for at most kPlanSmallMax
// buckets (small batches and merges, where launches, not rows, cost).  With
// thist given it first does k_tilescan's work (per-tile offsets in place,
// bucket totals into w); then the sums and their prefixes, the chunk starts,
// the chunk list and the finishing pass, separated by barriers.
constexpr int kPlanSmallThreads = 1024;
constexpr int kPlanSmallMax = 8192;

__global__ void __launch_bounds__(kPlanSmallThreads)
k_plan_small(unsigned int* thist, int ntiles, long long* w, int nb, int fine_shift, long long target, long long big,
             long long cap, long long* bstart, Chunk* chunks, int* big_list, PlanInfo* info, int seg_bits) {
  // seg_bits > 0: buckets come in batches of 2^seg_bits (a digit over several
  // batches); a chunk never spans two, and its fine range is its batch's
  const int segm = seg_bits ? (1 << seg_bits) - 1 : 0;
  __shared__ long long red[32];
  __shared__ long long s_tot[3];
  const int lane = threadIdx.x & 31;
  if (thist) {  // a warp per bucket
    for (int d = threadIdx.x >> 5; d < nb; d += kPlanSmallThreads / 32) {
      unsigned int* row = thist + (long long)d * ntiles;
      unsigned int run = 0;
      for (int b = 0; b < ntiles; b += 32) {
        const int t = b + lane;
        const unsigned int v = t < ntiles ? row[t] : 0u;
        unsigned int x = v;
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (t < ntiles) row[t] = run + x - v;
        run += __shfl_sync(0xffffffffu, x, 31);
      }
      if (lane == 0) w[d] = run;
    }
    __syncthreads();
  }
  const int sub = (nb + kPlanSmallThreads - 1) / kPlanSmallThreads;
  const int d0 = min(nb, (int)threadIdx.x * sub), d1 = min(nb, d0 + sub);
  long long ta = 0, tb = 0, tc = 0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    ta += x;
    if (x > cap) tc += 1;
    if (x <= big) tb += x;
  }
  const long long A0 = block_excl_ll(ta, red);
  const long long B0 = block_excl_ll(tb, red);
  long long nbig = block_excl_ll(tc, red);
  bool pbig;
  long long pq;
  plan_prev(w, d0, B0, big, target, &pbig, &pq);
  long long st = 0;
  {
    bool pb2 = pbig;
    long long pq2 = pq, pB2 = B0;
    for (int d = d0; d < d1; ++d) {
      const long long x = w[d];
      const bool s0 = plan_is_start(x, big, pB2, target, &pb2, &pq2);
      st += (s0 || (segm && d > 0 && (d & segm) == 0)) ? 1 : 0;
      if (x <= big) pB2 += x;
    }
  }
  const long long cex = block_excl_ll(st, red);
  if (threadIdx.x == kPlanSmallThreads - 1) {
    s_tot[0] = A0 + ta;
    s_tot[1] = nbig + tc;
    s_tot[2] = cex + st;
  }
  long long cidx = cex - 1, pA = A0, pB = B0;
  for (int d = d0; d < d1; ++d) {
    const long long x = w[d];
    bstart[d] = pA;
    const bool s0 = plan_is_start(x, big, pB, target, &pbig, &pq);
    if (s0 || (segm && d > 0 && (d & segm) == 0)) {
      ++cidx;
      chunks[cidx].pad = d;
      chunks[cidx].kind = x > cap ? CH_COPY : CH_NORMAL;
      if (x > cap) big_list[nbig++] = (int)cidx;
    }
    if (x <= big) pB += x;
    pA += x;
  }
  __syncthreads();  // every chunk's first bucket and every bucket start is written
  const int nc = (int)s_tot[2];
  if (threadIdx.x == 0) {
    bstart[nb] = s_tot[0];
    info->total = s_tot[0];
    info->n_big = (int)s_tot[1];
    info->n_chunks = nc;
  }
  long long mx = 0;
  for (int c = threadIdx.x; c < nc; c += kPlanSmallThreads) {
    const int dlo = chunks[c].pad;
    const int dhi = (c + 1 < nc) ? chunks[c + 1].pad : nb;
    Chunk& ch = chunks[c];
    ch.lo = bstart[dlo];
    ch.hi = dhi == nb ? s_tot[0] : bstart[dhi];
    const int seg0 = segm ? (dlo & ~segm) : 0;  // the batch's first bucket (0 without batches)
    ch.f_lo = (dlo - seg0) << fine_shift;
    ch.f_hi = (dhi - seg0) << fine_shift;
    if (ch.kind == CH_NORMAL) mx = max(mx, ch.hi - ch.lo);
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if (lane == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int k = 0; k < kPlanSmallThreads / 32; ++k) m = max(m, red[k]);
    info->max_chunk = m;
  }
}

// Scatter rows [0, n) of src into buckets: row i goes to
// bstart[d] + (its tile's offset in bucket d) + (rank inside the tile).
// Output rows are 1 + ncols int64 words: key, then the carried columns.
template <bool SEG>
__global__ void __launch_bounds__(kPartThreads)
k_scatter(RowSrc src, long long n, Digit dig, int nb, int ntiles, const unsigned int* thist,
          const long long* bstart, long long* aos) {
  // positions inside one batch (< 2^30 rows) fit 32 bits; nb x 4 bytes of shared memory
  extern __shared__ unsigned int cursor[];
  for (int d = threadIdx.x; d < nb; d += blockDim.x)
    cursor[d] = (unsigned int)(bstart[d] + thist[(long long)d * ntiles + blockIdx.x]);
  __syncthreads();
  long long lo, hi;
  const unsigned boff = tile_rows(n, ntiles, dig, blockIdx.x, &lo, &hi);
  const int W = 1 + src.ncols;
  constexpr int U = 8;  // independent loads in flight per thread
  if (W == 2) {
    for (long long i0 = lo + threadIdx.x; i0 < hi; i0 += (long long)U * blockDim.x) {
      unsigned long long k[U];
      long long v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        long long i = i0 + (long long)u * blockDim.x;
        if (i < hi) { k[u] = src_key(src, i); v[u] = src_col(src, 0, i); }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        long long i = i0 + (long long)u * blockDim.x;
        if (i < hi) {
          unsigned pos = atomicAdd(&cursor[boff + coarse_digit<SEG>(dig, k[u])], 1u);
          // one 16-byte store: key + the one carried column
          longlong2 r;
          r.x = (long long)k[u];
          r.y = v[u];
          *reinterpret_cast<longlong2*>(aos + (long long)pos * 2) = r;
        }
      }
    }
    return;
  }
  for (long long i0 = lo + threadIdx.x; i0 < hi; i0 += (long long)U * blockDim.x) {
    unsigned long long k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long i = i0 + (long long)u * blockDim.x;
      if (i < hi) k[u] = src_key(src, i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long i = i0 + (long long)u * blockDim.x;
      if (i < hi) {
        unsigned pos = atomicAdd(&cursor[boff + coarse_digit<SEG>(dig, k[u])], 1u);
        long long* row = aos + (long long)pos * W;
        row[0] = (long long)k[u];
        for (int c = 0; c < src.ncols; ++c) row[1 + c] = src_col(src, c, i);
      }
    }
  }
}

// Runs generated in one pass lie back to back; run b ends where its sparse
// index ends: rs[1 + b] = offs[b * stride + nf] (rs[0] = 0, the first start).
__global__ void k_run_bounds(const long long* offs, long long stride, int nf, int B, long long* rs) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
    rs[1 + b] = offs[(long long)b * stride + nf];
}

// Rows of all runs in each fine bucket: sizes[f] = sum_r offs[r][f+1] - offs[r][f].
__global__ void k_fine_sizes(const long long* const* offs, int k, int nf, long long* sizes) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    long long s = 0;
    for (int r = 0; r < k; ++r) s += offs[r][f + 1] - offs[r][f];
    sizes[f] = s;
  }
}

// Copy rows [lo, hi) of k runs' fine range into one SoA buffer (state rows).
__global__ void k_gather_runs(RunSet runs, int f_lo, int f_hi, const long long* dst_pre,
                              unsigned long long* dkeys, long long* const* dcols) {
  const int r = blockIdx.y;
  long long lo = runs.offs[r][f_lo];
  long long hi = runs.offs[r][f_hi];
  long long pre = dst_pre[r];
  const long long* const* p = runs.ptrs + (long long)r * (1 + runs.ncols);
  for (long long i = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hi;
       i += (long long)gridDim.x * blockDim.x) {
    dkeys[pre + i - lo] = (unsigned long long)p[0][i];
    for (int c = 0; c < runs.ncols; ++c) dcols[c][pre + i - lo] = p[1 + c][i];
  }
}

// Fine-bucket offsets of a sorted run held elsewhere: offs[f] = base + number
// of rows whose fine digit is below f (binary search), f in [0, nf].
__global__ void k_offsets_by_search(const unsigned long long* keys, long long n, Digit dig, int nf,
                                    long long base, long long* offs) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f <= nf; f += gridDim.x * blockDim.x) {
    long long lo = 0, hi = n;
    while (lo < hi) {
      long long mid = (lo + hi) >> 1;
      if ((int)fine_digit(dig, keys[mid]) < f) lo = mid + 1; else hi = mid;
    }
    offs[f] = base + lo;
  }
}


// ---------------------------------------------------------------------------
// Two-level partitioning.  Level 1 splits the batch into at most 1024 buckets;
// level 2 splits every level-1 bucket by the remaining digit bits.  Both
// levels scatter through a shared-memory stage: a sub-tile of kStage rows is
// counting-sorted by digit first, so each bucket's rows leave as one
// contiguous run and every store is coalesced (no partially written sectors
// for the memory system to read back).
// ---------------------------------------------------------------------------
constexpr int kStage = 4096;
constexpr int kStageCols = 4;        // carried columns the staged scatter handles
constexpr int kTile2 = 8192;         // rows per level-2 tile

// Exclusive prefix of w[0..nb) into out[0..nb] (single CTA of kPartThreads).
__device__ __forceinline__ void excl_scan_block(const long long* w, int nb, long long* out) {
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kPartThreads) {
    int d = b0 + threadIdx.x;
    long long v = d < nb ? w[d] : 0;
    int tot;
    // values fit int (rows of one batch < 2^31)
    int ex = block_excl_sum((int)v, &tot);
    if (d < nb) out[d] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[nb] = carry;
}

__global__ void __launch_bounds__(kPartThreads) k_excl_scan(const long long* w, int nb, long long* out) {
  excl_scan_block(w, nb, out);
}

struct Tile2 {
  long long lo, hi;   // rows of the level-1 output
  int bucket;         // level-1 bucket
  int pad;
};

// Level-2 tiles: bucket b of the level-1 output is cut into ceil(size/kTile2)
// tiles; tfirst[b] = index of its first tile, tfirst[nb1] = tile count.
__device__ __forceinline__ void tiles2_block(const long long* bstart1, int nb1, Tile2* tiles, int* tfirst) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb1; b0 += kPartThreads) {
    int b = b0 + threadIdx.x;
    long long lo = 0, hi = 0;
    int nt = 0;
    if (b < nb1) {
      lo = bstart1[b];
      hi = bstart1[b + 1];
      nt = (int)((hi - lo + kTile2 - 1) / kTile2);
    }
    int tot;
    int ex = block_excl_sum(nt, &tot) + carry;
    if (b < nb1) {
      tfirst[b] = ex;
      for (int j = 0; j < nt; ++j) {
        Tile2 t;
        t.lo = lo + (long long)j * kTile2;
        t.hi = min(hi, t.lo + kTile2);
        t.bucket = b;
        t.pad = 0;
        tiles[ex + j] = t;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) tfirst[nb1] = carry;
}

// Level-1 bucket starts from their totals, then the level-2 tiles over them
// (one CTA; the tiles depend only on the starts, so they are cut before the
// level-1 scatter runs, in the same launch).
__global__ void __launch_bounds__(kPartThreads)
k_scan_tiles2(const long long* btot1, int nb1, long long* bstart1, Tile2* tiles, int* tfirst) {
  excl_scan_block(btot1, nb1, bstart1);
  __syncthreads();  // bstart1 (global, written by this CTA) is read below
  tiles2_block(bstart1, nb1, tiles, tfirst);
}

// Level-2 histograms: thist2[t * nb2 + d] = rows of tile t with digit d.
// A tile is only kTile2 rows (16 per thread), so the private histograms are
// shared by groups of warps (warp w adds to copy w % kHist2Copies): a copy
// per warp (16 x 256 counters zeroed, then summed) is as many shared-memory
// operations as the tile's rows take to count.
constexpr int kHist2Copies = 4;

inline size_t hist2_smem_bytes(int nb2) {
  return (size_t)(nb2 <= kPrivBuckets ? nb2 * kHist2Copies : nb2) * 4;
}

template <bool SEG, bool DIRECT>
__global__ void __launch_bounds__(kPartThreads)
k_hist2(RowSrc src, Digit dig, int nb2, const Tile2* tiles, const int* ntiles, unsigned* thist2) {
  extern __shared__ unsigned sh2[];
  const int t = blockIdx.x;
  if (t >= *ntiles) return;
  const bool priv = nb2 <= kPrivBuckets;
  unsigned* mine = priv ? sh2 + ((threadIdx.x >> 5) % kHist2Copies) * nb2 : sh2;
  const int nh = priv ? nb2 * kHist2Copies : nb2;
  for (int d = threadIdx.x; d < nh; d += blockDim.x) sh2[d] = 0;
  __syncthreads();
  const Tile2 tl = tiles[t];
  constexpr int U = 8;
  for (long long i0 = tl.lo + threadIdx.x; i0 < tl.hi; i0 += (long long)U * blockDim.x) {
    unsigned long long k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long i = i0 + (long long)u * blockDim.x;
      if (i < tl.hi) k[u] = DIRECT ? __ldg(src_key_ptr(src, i)) : src_key(src, i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      long long i = i0 + (long long)u * blockDim.x;
      if (i < tl.hi) atomicAdd(&mine[level_digit<SEG>(dig, k[u], 0, nb2)], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < nb2; d += blockDim.x) {
    unsigned v = sh2[d];
    if (priv)
      for (int w = 1; w < kHist2Copies; ++w) v += sh2[w * nb2 + d];
    thist2[(long long)t * nb2 + d] = v;
  }
}

// One CTA per level-1 bucket: turns the bucket's tile histograms into absolute
// write positions (thist2, in place) and writes the final bucket totals
// btot[b * nb2 + d] (fine-grained buckets in key order).
// A thread walks its digit's column of tile counts kScan2Batch tiles at a
// time: the batch's loads are issued before its stores, so a bucket of T
// tiles waits on about T / kScan2Batch memory latencies instead of T.
constexpr int kScan2Batch = 8;

__global__ void __launch_bounds__(kPartThreads)
k_scan2(const long long* bstart1, int nb2, const int* tfirst, unsigned* thist2, long long* btot) {
  const int b = blockIdx.x;
  const int t0 = tfirst[b], t1 = tfirst[b + 1];
  const int d = threadIdx.x;
  int tot = 0;
  if (d < nb2)
    for (int t = t0; t < t1; t += kScan2Batch) {
      unsigned c[kScan2Batch];
#pragma unroll
      for (int u = 0; u < kScan2Batch; ++u) c[u] = t + u < t1 ? thist2[(long long)(t + u) * nb2 + d] : 0u;
#pragma unroll
      for (int u = 0; u < kScan2Batch; ++u)
        if (t + u < t1) {
          thist2[(long long)(t + u) * nb2 + d] = (unsigned)tot;
          tot += (int)c[u];
        }
    }
  int all;
  int ex = block_excl_sum(d < nb2 ? tot : 0, &all);
  if (d < nb2) {
    const unsigned start = (unsigned)(bstart1[b] + ex);
    for (int t = t0; t < t1; t += kScan2Batch) {
      unsigned c[kScan2Batch];
#pragma unroll
      for (int u = 0; u < kScan2Batch; ++u) c[u] = t + u < t1 ? thist2[(long long)(t + u) * nb2 + d] : 0u;
#pragma unroll
      for (int u = 0; u < kScan2Batch; ++u)
        if (t + u < t1) thist2[(long long)(t + u) * nb2 + d] = c[u] + start;
    }
    btot[(long long)b * nb2 + d] = tot;
  }
}

// Staged scatter (both levels).  Level 1 (tiles == nullptr): tile t is an even
// share of rows [0, n) and bucket d's write cursor starts at
// bstart[d] + table[d * ntiles + t].  Level 2: tile t is tiles[t] and the
// cursor starts at table[t * nb + d].  Output: SoA (okeys/ocols) or rows of
// 1 + ncols words (oaos).
// SoA output columns of a staged scatter, passed by value (no pointer table
// to copy to the device before the launch).
struct StageCols {
  long long* c[kStageCols];
};

// Whether k_scatter_staged can copy the source with cp.async (DIRECT).
__host__ __device__ inline bool staged_direct(const RowSrc& src) {
  return src.kind != SRC_AOS && src_keys_direct(src);
}

template <bool SEG, bool DIRECT>
__global__ void __launch_bounds__(kPartThreads, 2)
k_scatter_staged(RowSrc src, long long n, Digit dig, int dshift, int nb, int ntiles, const Tile2* tiles,
                 const int* ntiles_dev, const unsigned* table, const long long* bstart,
                 unsigned long long* okeys, StageCols ocols, long long* oaos) {
  extern __shared__ __align__(16) unsigned char st_raw[];
  unsigned* cursor = reinterpret_cast<unsigned*>(st_raw);
  unsigned* lst = cursor + nb;
  const int C = src.ncols;
  // header (cursor, lst) padded to 16 bytes so the 8-byte stage stays aligned
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(st_raw + (((size_t)2 * nb * 4 + 15) & ~(size_t)15));
  long long* scol = reinterpret_cast<long long*>(skey + kStage);
  uint16_t* sperm = reinterpret_cast<uint16_t*>(scol + (long long)C * kStage);
  const int t = blockIdx.x;
  long long lo, hi;
  if (tiles) {
    if (t >= *ntiles_dev) return;
    lo = tiles[t].lo;
    hi = tiles[t].hi;
    for (int d = threadIdx.x; d < nb; d += blockDim.x) cursor[d] = table[(long long)t * nb + d];
  } else {
    tile_range(n, ntiles, t, &lo, &hi);
    for (int d = threadIdx.x; d < nb; d += blockDim.x)
      cursor[d] = (unsigned)(bstart[d] + table[(long long)d * ntiles + t]);
  }
  const int dsh = tiles ? 0 : dshift;
  constexpr int U = kStage / kPartThreads;  // 8
  // 8-byte keys in one column (SoA, or raw uint64 keys): the sub-tile is
  // copied into the stage by cp.async, global to shared without passing
  // through registers, all of it in flight at once
  constexpr bool direct = DIRECT;  // the host checked staged_direct(src)
  const unsigned long long* dkeys =
      src.kind == SRC_SOA ? src.keys : reinterpret_cast<const unsigned long long*>(src.key.cols[0]);
  for (long long s0 = lo; s0 < hi; s0 += kStage) {
    const int m = (int)min((long long)kStage, hi - s0);
    unsigned dr[U];  // digit << 16 | rank
    unsigned long long kk[U];
    if constexpr (direct) {
      const long long r0 = src.offset + s0;
      for (int i = threadIdx.x; i < m; i += kPartThreads) {
        cp_async8(&skey[i], dkeys + r0 + i);
        for (int c = 0; c < C; ++c) cp_async8(&scol[c * kStage + i], src.cols[c] + r0 + i);
      }
    }
    for (int d = threadIdx.x; d < nb; d += blockDim.x) lst[d] = 0;
    if constexpr (direct) {
      cp_async_wait();
      __syncthreads();
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = threadIdx.x + u * kPartThreads;
        if (i < m) {
          kk[u] = skey[i];
          const unsigned d = level_digit<SEG>(dig, kk[u], dsh, nb);
          dr[u] = (d << 16) | atomicAdd(&lst[d], 1u);
        }
      }
    } else {
    __syncthreads();
    // all loads of the sub-tile first (independent, in flight together) ...
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = threadIdx.x + u * kPartThreads;
      if (i < m) kk[u] = src_key(src, s0 + i);
    }
    if (C == 1) {
      long long cv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = threadIdx.x + u * kPartThreads;
        if (i < m) cv[u] = src_col(src, 0, s0 + i);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = threadIdx.x + u * kPartThreads;
        if (i < m) scol[i] = cv[u];
      }
    } else {
      for (int c = 0; c < C; ++c) {
        long long cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = threadIdx.x + u * kPartThreads;
          if (i < m) cv[u] = src_col(src, c, s0 + i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = threadIdx.x + u * kPartThreads;
          if (i < m) scol[c * kStage + i] = cv[u];
        }
      }
    }
    // ... then the stage writes and the per-digit ranks
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = threadIdx.x + u * kPartThreads;
      if (i < m) {
        skey[i] = kk[u];
        unsigned d = level_digit<SEG>(dig, kk[u], dsh, nb);
        unsigned r = atomicAdd(&lst[d], 1u);
        dr[u] = (d << 16) | r;
      }
    }
    }
    __syncthreads();
    // local starts: exclusive scan of the per-digit counts, two digits per
    // thread (nb <= 2 * kPartThreads)
    {
      const int d0 = 2 * threadIdx.x;
      const int c0 = d0 < nb ? (int)lst[d0] : 0;
      const int c1 = d0 + 1 < nb ? (int)lst[d0 + 1] : 0;
      int tot;
      const int ex = block_excl_sum(c0 + c1, &tot);
      if (d0 < nb) lst[d0] = (unsigned)ex;
      if (d0 + 1 < nb) lst[d0 + 1] = (unsigned)(ex + c0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = threadIdx.x + u * kPartThreads;
      if (i < m) sperm[lst[dr[u] >> 16] + (dr[u] & 0xFFFFu)] = (uint16_t)i;
    }
    __syncthreads();
    for (int lp = threadIdx.x; lp < m; lp += kPartThreads) {
      const int i = sperm[lp];
      const unsigned long long k = skey[i];
      const unsigned d = level_digit<SEG>(dig, k, dsh, nb);
      const long long gp = (long long)cursor[d] + (lp - (int)lst[d]);
      if (oaos) {
        long long* row = oaos + gp * (1 + C);
        if (C == 1) {
          longlong2 v;
          v.x = (long long)k;
          v.y = scol[i];
          *reinterpret_cast<longlong2*>(row) = v;
        } else {
          row[0] = (long long)k;
          for (int c = 0; c < C; ++c) row[1 + c] = scol[c * kStage + i];
        }
      } else {
        okeys[gp] = k;
        for (int c = 0; c < C; ++c) ocols.c[c][gp] = scol[c * kStage + i];
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += blockDim.x) {
      const unsigned next = (d + 1 < nb) ? lst[d + 1] : (unsigned)m;
      cursor[d] += next - lst[d];
    }
    __syncthreads();
  }
}

inline size_t staged_smem_bytes(int nb, int ncols) {
  return (((size_t)2 * nb * 4 + 15) & ~(size_t)15) + (size_t)kStage * 8 * (1 + ncols) + (size_t)kStage * 2 + 16;
}


// start[j] = first row of instance first + j, for j in [0, count], in rows
// whose keys carry the instance id above key_bits and come grouped by
// instance in ascending order (sorted within an instance's rows or not).
// With write_rows (the grouped output, step 1 of the batched output), each
// instance of more than skip_n rows gets *out_rows = its row count, or -1
// when that exceeds its out_capacity (then nothing is written for it).
__global__ void k_inst_bounds(const unsigned long long* keys, long long total, const InstDesc* inst,
                              int key_bits, int first, int count, long long* start, int write_rows,
                              long long skip_n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > count) return;
  auto lower = [&](int i) {
    const unsigned long long target = (unsigned long long)i << key_bits;
    long long lo = 0, hi = total;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (keys[mid] < target) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const long long a = lower(first + j);
  start[j] = a;
  if (write_rows && j < count && inst[first + j].n > skip_n) {
    const long long rows = lower(first + j + 1) - a;
    *inst[first + j].out_rows = rows > inst[first + j].out_capacity ? -1 : rows;
  }
}

// Batched output, step 2: row r of the grouped rows goes to row
// r - start[i] of instance i's outputs (key without the instance bits).
// A CTA copies kDistRows consecutive rows.
constexpr int kDistRows = 2048;
__global__ void __launch_bounds__(256)
k_distribute(const unsigned long long* keys, CopySrc states, long long total, int n_state,
             const InstDesc* inst, int key_bits, int first, int count, const long long* start) {
  const long long r0 = (long long)blockIdx.x * kDistRows;
  const long long r1 = min(total, r0 + kDistRows);
  const unsigned long long mask = (1ull << key_bits) - 1;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const unsigned long long key = keys[r];
    const long long j = (long long)(key >> key_bits) - first;
    if (j < 0 || j >= count) continue;  // not this group's row (never: rows are built so)
    const InstDesc& d = inst[first + j];
    const long long at = r - start[j];
    if (start[j + 1] - start[j] > d.out_capacity) continue;
    const unsigned long long k = key & mask;
    switch (d.key_bytes) {
      case 1: reinterpret_cast<uint8_t*>(d.out_keys)[at] = (uint8_t)k; break;
      case 2: reinterpret_cast<uint16_t*>(d.out_keys)[at] = (uint16_t)k; break;
      case 4: reinterpret_cast<uint32_t*>(d.out_keys)[at] = (uint32_t)k; break;
      default: reinterpret_cast<unsigned long long*>(d.out_keys)[at] = k; break;
    }
    for (int a = 0; a < n_state; ++a) d.out_aggs[a][at] = states.cols[a][r];
  }
}

// ---------------------------------------------------------------------------
// Absorbing-index run generation (host side in sgagg.cu): copies of sorted
// state rows between the index, the batch, the merged index and the runs,
// and the searches that split them.
// ---------------------------------------------------------------------------
struct SoaRef {
  unsigned long long* keys;
  long long* cols[kMaxCols];
};

// dst rows [dst_off, dst_off + n) = src rows [src_off, src_off + n), columns
// 0 .. ncols-1; column zero_col (if >= 0) is written as 0 instead.
__global__ void k_copy_soa(SoaRef src, long long src_off, SoaRef dst, long long dst_off, long long n, int ncols,
                           int zero_col) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    dst.keys[dst_off + i] = src.keys[src_off + i];
    for (int c = 0; c < ncols; ++c) dst.cols[c][dst_off + i] = c == zero_col ? 0 : src.cols[c][src_off + i];
  }
}

// The n rows of src to the caller's output (keys unpacked to its columns).
__global__ void k_emit_soa(SoaRef src, long long n, int ncols, OutSink out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    sink_key(out, i, src.keys[i]);
    for (int c = 0; c < ncols; ++c) sink_val(out, c, i, src.cols[c][i]);
  }
}

// counts[b] = nonzero entries of flag in block b's range (ranges of `per`).
__global__ void k_flag_counts(const long long* flag, long long n, long long per, long long* counts) {
  __shared__ long long part[32];
  const long long lo = blockIdx.x * per, hi = min(n, lo + per);
  long long c = 0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) c += flag[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    counts[blockIdx.x] = t;
  }
}

// *pos = index of the j-th (1-based) nonzero entry of flag, or n if there
// are fewer; one block of 1024 threads after k_flag_counts over nb ranges.
__global__ void __launch_bounds__(1024)
k_nth_flag(const long long* flag, long long n, long long per, const long long* counts, int nb, long long j,
           long long* pos) {
  __shared__ long long s_before;
  __shared__ int s_block;
  if (threadIdx.x == 0) {
    long long acc = 0;
    int b = 0;
    while (b < nb && acc + counts[b] < j) acc += counts[b++];
    s_before = acc;
    s_block = b;
  }
  __syncthreads();
  if (s_block >= nb) {
    if (threadIdx.x == 0) *pos = n;
    return;
  }
  const long long lo = s_block * per, hi = min(n, lo + per);
  long long need = j - s_before;  // >= 1, and the block holds at least that many
  __shared__ long long wsum[32];
  for (long long base = lo; base < hi; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const int f = (i < hi && flag[i] != 0) ? 1 : 0;
    // block inclusive scan of f
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = f;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      long long v = wsum[lane], t = v;
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wsum[lane] = t - v;
    }
    __syncthreads();
    const long long incl = wsum[w] + x;
    if (f && incl == need) *pos = i;
    const long long tot = wsum[31] + __shfl_sync(0xffffffffu, x, 31);  // valid in warp 31 only
    __shared__ long long s_tot;
    if (threadIdx.x == blockDim.x - 1) s_tot = tot;
    __syncthreads();
    need -= s_tot;
    if (need <= 0) return;
    __syncthreads();
  }
}

// With x = tkeys[*p]: out[0] = keys of a[0 .. na) below x, out[1] = keys of
// b[0 .. nb) below x (both ascending).  One thread.
__global__ void k_split_at(const unsigned long long* tkeys, const long long* p, const unsigned long long* a,
                           long long na, const unsigned long long* b, long long nb, long long* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long x = tkeys[*p];
  for (int w = 0; w < 2; ++w) {
    const unsigned long long* k = w ? b : a;
    long long lo = 0, hi = w ? nb : na;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (k[mid] < x) lo = mid + 1; else hi = mid;
    }
    out[w] = lo;
  }
}

// ---------------------------------------------------------------------------
// count(distinct u) per g: rows sorted by the composite key (g, u), each
// (g, u) once, are regrouped on g = key >> ubits in one pass, without a sort
// (the interesting ordering of Sec. 7).  A block takes kRegroupRows rows, a
// thread kRegroupRows / 256 consecutive ones; output slots are group ranks
// (heads before the block + heads before the row), and every thread folds
// its piece of each group it touches into the slot with integer atomics.
// ---------------------------------------------------------------------------
constexpr int kRegroupRows = 4096;

__device__ __forceinline__ bool regroup_head(const unsigned long long* keys, long long i, int ubits) {
  return i == 0 || (keys[i] >> ubits) != (keys[i - 1] >> ubits);
}

// heads[b] = rows of block b that open a group
__global__ void __launch_bounds__(256)
k_regroup_count(const unsigned long long* keys, long long n, int ubits, long long* heads) {
  __shared__ int s_c;
  if (threadIdx.x == 0) s_c = 0;
  __syncthreads();
  const long long r0 = blockIdx.x * (long long)kRegroupRows, r1 = min(n, r0 + kRegroupRows);
  int c = 0;
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) c += regroup_head(keys, i, ubits);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_c, c);
  __syncthreads();
  if (threadIdx.x == 0) heads[blockIdx.x] = s_c;
}

// Output slots [0, groups): distinct counts 0, aggregates at their identity.
__global__ void k_regroup_init(long long* distinct, OutSink out, FoldDesc fd, long long groups) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
    distinct[g] = 0;
    for (int a = 0; a < fd.n_state; ++a) out.cols[a][g] = op_identity(fd.op[a]);
  }
}

__device__ __forceinline__ void regroup_flush(long long slot, long long cnt, const long long* acc, OutSink& out,
                                              const FoldDesc& fd, long long* distinct) {
  atomicAdd(reinterpret_cast<unsigned long long*>(distinct + slot), (unsigned long long)cnt);
  for (int a = 0; a < fd.n_state; ++a) {
    long long* p = out.cols[a] + slot;
    if (fd.op[a] == OP_SUM) atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)acc[a]);
    else if (fd.op[a] == OP_MIN) atomicMin(p, acc[a]);
    else atomicMax(p, acc[a]);
  }
}

__global__ void __launch_bounds__(256)
k_regroup_fold(const unsigned long long* keys, CopySrc states, long long n, int ubits, FoldDesc fd,
               const long long* base, OutSink out, long long* distinct) {
  constexpr int R = kRegroupRows / 256;
  __shared__ int ws[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = min(n, blockIdx.x * (long long)kRegroupRows + threadIdx.x * R), r1 = min(n, r0 + R);
  int mine = 0;
  for (long long i = r0; i < r1; ++i) mine += regroup_head(keys, i, ubits);
  // block exclusive scan of the heads per thread
  int x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < w; ++k) before += ws[k];
  long long slot = base[blockIdx.x] + before + x - mine - 1;  // the group open at r0 (-1: none)
  long long acc[kMaxCols];
  long long cnt = 0;
  for (long long i = r0; i < r1; ++i) {
    if (regroup_head(keys, i, ubits)) {
      if (cnt > 0 && slot >= 0 && slot < out.capacity) regroup_flush(slot, cnt, acc, out, fd, distinct);
      ++slot;
      cnt = 0;
      if (slot < out.capacity) sink_key(out, slot, keys[i] >> ubits);
    }
    for (int a = 0; a < fd.n_state; ++a) {
      const long long v = states.cols[a][i];
      acc[a] = cnt == 0 ? v : op_combine(fd.op[a], acc[a], v);
    }
    ++cnt;
  }
  if (cnt > 0 && slot >= 0 && slot < out.capacity) regroup_flush(slot, cnt, acc, out, fd, distinct);
}

}  // namespace sg
