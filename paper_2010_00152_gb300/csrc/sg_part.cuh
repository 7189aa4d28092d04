// sg_part.cuh -- partitioning a batch by key range before the per-chunk sort.
//
// A batch of up to M rows (one read-sort-write cycle, Sec. 3 / Sec. 6.1) is
// too large for one CTA, so it is first split by a most-significant digit of
// the key into buckets that are key ranges in key order:
//   k_hist     per-tile histogram of the coarse digit (one read of the keys);
//   k_tilescan per bucket, exclusive scan over tiles -> each tile's write
//              offset inside the bucket; bucket totals;
//   k_plan     bucket starts, and a grouping of consecutive buckets into
//              chunks of at most kTileCap rows; a bucket bigger than half a
//              chunk is set apart (solved separately, then copied in);
//   k_scatter  every row written once to its bucket (rows of 1 + ncols words).
// The same planner groups the fine buckets of the wide merge into merge
// tiles (k_fine_sizes gives each fine bucket's row count over all runs).
#pragma once
#include "sg_sortfold.cuh"

namespace sg {

constexpr int kPartThreads = 512;

// Keys of `count` rows spread evenly over [0, n), for the planner's probe.
__global__ void k_sample(RowSrc src, long long n, int count, unsigned long long* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    long long r = (long long)((__int128)i * n / count);
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

// thist[d * ntiles + t] = rows of tile t with coarse digit d.
__global__ void __launch_bounds__(kPartThreads)
k_hist(RowSrc src, long long n, Digit dig, int nb, int ntiles, unsigned int* thist) {
  extern __shared__ unsigned int sh_hist[];
  for (int d = threadIdx.x; d < nb; d += blockDim.x) sh_hist[d] = 0;
  __syncthreads();
  long long lo, hi;
  tile_range(n, ntiles, blockIdx.x, &lo, &hi);
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&sh_hist[coarse_digit(dig, src_key(src, i))], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < nb; d += blockDim.x) thist[(long long)d * ntiles + blockIdx.x] = sh_hist[d];
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

// Single CTA.  w[0..nb) are bucket row counts in key order.  Writes bstart
// (exclusive prefix, nb + 1 entries), the chunk list and the indices of big
// chunks.  A bucket with more than `big` rows is a chunk of its own (kind
// CH_COPY: solved separately).  Other buckets are grouped while their
// exclusive prefix over non-big buckets stays in one multiple of `target`,
// so a chunk holds fewer than target + big rows.  Chunk c covers buckets
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

__global__ void __launch_bounds__(1024)
k_plan(const long long* __restrict__ w, int nb, long long target, long long big, int fine_shift,
       long long* bstart, Chunk* chunks, int* big_list, PlanInfo* info) {
  const int T = blockDim.x;
  const int per = (nb + T - 1) / T;
  const int d0 = min(nb, (int)threadIdx.x * per), d1 = min(nb, d0 + per);
  __shared__ long long sa[1024], sb[1024], sc[1024], sd[1024];
  __shared__ int s_nc;
  long long ta = 0, tb = 0, tc = 0;
  for (int d = d0; d < d1; ++d) {
    long long x = w[d];
    ta += x;
    if (x > big) tc += 1; else tb += x;
  }
  sa[threadIdx.x] = ta; sb[threadIdx.x] = tb; sc[threadIdx.x] = tc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long A = 0, B = 0, C = 0;
    for (int t = 0; t < T; ++t) {
      long long a = sa[t], b = sb[t], c = sc[t];
      sa[t] = A; sb[t] = B; sc[t] = C;
      A += a; B += b; C += c;
    }
    info->total = A;
    info->n_big = (int)C;
    bstart[nb] = A;
  }
  __syncthreads();
  const long long A0 = sa[threadIdx.x], B0 = sb[threadIdx.x], C0 = sc[threadIdx.x];
  // state just before d0 (the previous bucket)
  bool pb0 = true;
  long long pq0 = -1;
  if (d0 > 0 && d0 < nb) {
    long long x = w[d0 - 1];
    pb0 = x > big;
    pq0 = pb0 ? -1 : (B0 - x) / target;
  }
  int starts = 0;
  {
    bool pbig = pb0;
    long long pq = pq0, pB = B0;
    for (int d = d0; d < d1; ++d) {
      long long x = w[d];
      starts += plan_is_start(x, big, pB, target, &pbig, &pq);
      if (x <= big) pB += x;
    }
  }
  sd[threadIdx.x] = starts;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long S = 0;
    for (int t = 0; t < T; ++t) { long long c = sd[t]; sd[t] = S; S += c; }
    s_nc = (int)S;
    info->n_chunks = (int)S;
  }
  __syncthreads();
  {
    bool pbig = pb0;
    long long pq = pq0, pB = B0, pA = A0, nbig = C0;
    long long cidx = sd[threadIdx.x] - 1;
    for (int d = d0; d < d1; ++d) {
      long long x = w[d];
      bstart[d] = pA;
      if (plan_is_start(x, big, pB, target, &pbig, &pq)) {
        ++cidx;
        chunks[cidx].f_lo = d;  // bucket index for now
        chunks[cidx].kind = x > big ? CH_COPY : CH_NORMAL;
        if (x > big) big_list[nbig++] = (int)cidx;
      }
      if (x <= big) pB += x;
      pA += x;
    }
  }
  __syncthreads();
  const int nc = s_nc;
  long long mx = 0;
  // chunk c ends where chunk c + 1 starts: stash the end bucket in pad
  for (int c = threadIdx.x; c < nc; c += T) {
    int dhi = (c + 1 < nc) ? chunks[c + 1].f_lo : nb;
    chunks[c].pad = dhi;
    chunks[c].lo = bstart[chunks[c].f_lo];
    chunks[c].hi = bstart[dhi];
    if (chunks[c].kind == CH_NORMAL) mx = max(mx, chunks[c].hi - chunks[c].lo);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += T) {
    chunks[c].f_lo = chunks[c].f_lo << fine_shift;
    chunks[c].f_hi = chunks[c].pad << fine_shift;
    chunks[c].pad = 0;
  }
  sa[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int t = 0; t < T; ++t) m = max(m, sa[t]);
    info->max_chunk = m;
  }
}

// Scatter rows [0, n) of src into buckets: row i goes to
// bstart[d] + (its tile's offset in bucket d) + (rank inside the tile).
// Output rows are 1 + ncols int64 words: key, then the carried columns.
__global__ void __launch_bounds__(kPartThreads)
k_scatter(RowSrc src, long long n, Digit dig, int nb, int ntiles, const unsigned int* thist,
          const long long* bstart, long long* aos) {
  // positions inside one batch (< 2^30 rows) fit 32 bits; nb x 4 bytes of shared memory
  extern __shared__ unsigned int cursor[];
  for (int d = threadIdx.x; d < nb; d += blockDim.x)
    cursor[d] = (unsigned int)(bstart[d] + thist[(long long)d * ntiles + blockIdx.x]);
  __syncthreads();
  long long lo, hi;
  tile_range(n, ntiles, blockIdx.x, &lo, &hi);
  const int W = 1 + src.ncols;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    unsigned long long k = src_key(src, i);
    unsigned long long pos = atomicAdd(&cursor[coarse_digit(dig, k)], 1u);
    long long* row = aos + (long long)pos * W;
    if (W == 2) {
      // one 16-byte store when the row is key + one column
      longlong2 v;
      v.x = (long long)k;
      v.y = src_col(src, 0, i);
      *reinterpret_cast<longlong2*>(row) = v;
    } else {
      row[0] = (long long)k;
      for (int c = 0; c < src.ncols; ++c) row[1 + c] = src_col(src, c, i);
    }
  }
}

// Rows of all runs in each fine bucket: sizes[f] = sum_r offs[r][f+1] - offs[r][f].
__global__ void k_fine_sizes(const long long* offs, int k, long long stride, int nf, long long* sizes) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    long long s = 0;
    for (int r = 0; r < k; ++r) s += offs[(long long)r * stride + f + 1] - offs[(long long)r * stride + f];
    sizes[f] = s;
  }
}

// Copy rows [lo, hi) of k runs' fine range into one SoA buffer (state rows).
__global__ void k_gather_runs(RunSet runs, int f_lo, int f_hi, const long long* dst_pre,
                              unsigned long long* dkeys, long long* const* dcols) {
  const int r = blockIdx.y;
  long long lo = runs.offs[(long long)r * runs.stride + f_lo];
  long long hi = runs.offs[(long long)r * runs.stride + f_hi];
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

}  // namespace sg
