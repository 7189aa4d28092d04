// sg_hybrid.cuh -- the input split of hybrid run generation (Sec. 5.2.3):
// memory is divided between an in-memory index that absorbs the rows of a
// resident key range (no spill) and read-sort-write run generation for the
// other rows, followed by one wide merge.  On the GPU the resident range is
// the keys at or below a last resident key; one pass splits the input rows
// by it into two row sets, each keeping input order (the runs are batches
// of consecutive spilled rows, as the read-sort-write cycles read them).
#pragma once
#include "sg_common.cuh"

namespace sg {

constexpr int kSplitThreads = 512;
constexpr int kSplitPer = 8;                        // consecutive rows per thread
constexpr int kSplitTile = kSplitThreads * kSplitPer;

// Two SoA row sets: 0 the resident rows, 1 the spilled rows (normalized
// uint64 key, then the carried columns).
struct SplitOut {
  unsigned long long* keys[2];
  long long* cols[2][kMaxCols];
};

// Tiles of kSplitTile rows in ticket order: a tile's resident count gives
// its resident prefix by decoupled look-back (lb.total_out: all resident
// rows); its spilled prefix is the rest of the rows before it.
__global__ void __launch_bounds__(kSplitThreads)
k_split_range(RowSrc src, long long n, unsigned long long last, int has_last, SplitOut out, LookBack lb) {
  constexpr int W = kSplitThreads / 32;
  __shared__ int s_cid, s_err;
  __shared__ int s_w[W];
  __shared__ long long s_pre;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_cid = (int)atomicAdd(lb.ticket, 1u);
    s_err = err_load(lb.err);
  }
  __syncthreads();
  const int cid = s_cid;
  if (cid >= lb.n_chunks || s_err) return;
  const long long lo = (long long)cid * kSplitTile;
  const long long r0 = lo + (long long)tid * kSplitPer;
  const int valid = (int)max(0ll, min((long long)kSplitPer, n - r0));
  unsigned long long key[kSplitPer];
  unsigned fl = 0;
#pragma unroll
  for (int j = 0; j < kSplitPer; ++j) {
    key[j] = 0;
    if (j < valid) {
      key[j] = load_key(src.key, src.offset + r0 + j) | src.key_or;
      if (has_last && key[j] <= last) fl |= 1u << j;
    }
  }
  const int c = __popc(fl);
  int x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    before += q < w ? s_w[q] : 0;
    total += s_w[q];
  }
  const int rank = before + x - c;  // resident rows of the tile before this thread's
  if (tid < 32) {
    const long long b = lookback_warp(lb, cid, total);
    if (tid == 0) {
      s_pre = b;
      if (b >= 0 && lb.total_out && cid == lb.n_chunks - 1) *lb.total_out = b + total;
    }
  }
  __syncthreads();
  const long long pre = s_pre;
  if (pre < 0) return;
  long long pr = pre + rank;                                   // next resident position
  long long ps = (lo - pre) + ((long long)tid * kSplitPer - rank);  // next spilled position
#pragma unroll
  for (int j = 0; j < kSplitPer; ++j) {
    if (j < valid) {
      const int side = ((fl >> j) & 1u) ? 0 : 1;
      const long long at = side == 0 ? pr++ : ps++;
      out.keys[side][at] = key[j];
      for (int cc = 0; cc < src.ncols; ++cc) out.cols[side][cc][at] = src_col(src, cc, r0 + j);
    }
  }
}

}  // namespace sg
