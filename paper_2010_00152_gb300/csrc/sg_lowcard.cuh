// sg_lowcard.cuh -- grouping when the keys take few values: the report shape
// of Example 1 (Sec. 3.2), whose output is a handful of rows however large
// the input.  With one batch covering the input (no run is written, the
// in-memory case of Sec. 5.2.1) and at most kLowCardKeys distinct keys in the
// planner's key sample, sorting the rows is not needed to bring equal keys
// together: one streaming pass folds every row straight into accumulators of
// its key ("row-plus-row accumulation", Sec. 6.1), and the accumulators
// leave in key order.
//
//   k_lowcard         every thread folds its rows (coalesced, several rows
//                     in flight) into private shared-memory accumulators,
//                     one per (sampled key, aggregate); the block combines
//                     its threads' accumulators into one partial per key and
//                     aggregate;
//   k_lowcard_report  the same for the report pattern (count(*), then sum,
//                     min and max per payload column): accumulators at
//                     compile-time offsets, one set per pair of lanes;
//   k_lowcard_finish  one block combines the partials of all blocks and
//                     writes the keys (ascending) and the aggregates.
// A row whose key is not in the sample raises a flag; the host then groups
// the input by the general path instead (the result is the same, only the
// work differs).
#pragma once
#include "sg_common.cuh"

namespace sg {

constexpr int kLowCardKeys = 16;        // sampled distinct keys the pass takes at most
constexpr int kLowCardUnroll = 4;       // rows per thread per step
constexpr int kLowCardMaxSlots = 104;   // keys x aggregates accumulators per thread at most

// The caller's output columns (passed by value).
struct OutSinkLite {
  KeyOut kout;
  long long* cols[kMaxCols];
  long long capacity;
};

struct LowCardArgs {
  RowSrc src;                               // raw rows (key columns + payload columns)
  long long n;
  int kd;                                   // sampled distinct keys, ascending in keys[]
  int n_col;                                // source columns the aggregates read
  unsigned long long keys[kLowCardKeys];
  FoldDesc fd;
  int8_t order[kMaxCols];                   // aggregates ordered by source column
  int8_t col_end[kMaxCols + 1];             // order[col_end[c] .. col_end[c+1]) read column c;
                                            // order[0 .. col_end[0]) are count(*)
  long long* partial;                       // [gridDim.x][kd * n_state]
  int* overflow;                            // set when some row's key is not in keys[]
};

// Accumulator q = slot * n_state + aggregate of thread t at acc[q * T + t]:
// a warp's accesses hit 32 consecutive words whatever the rows' keys.  Per
// row, every accumulator of its key is loaded first, then combined, then
// stored (KS >= n_state aggregates unrolled), so a row costs one shared-
// memory round trip, not one per aggregate.
template <int KS>
__global__ void __launch_bounds__(256) k_lowcard(LowCardArgs a) {
  extern __shared__ long long lc_acc[];
  __shared__ unsigned long long sk[kLowCardKeys];
  const int T = blockDim.x, tid = threadIdx.x;
  const int S = a.fd.n_state, kd = a.kd, Q = kd * S;
  for (int q = 0; q < Q; ++q) lc_acc[q * T + tid] = op_identity(a.fd.op[q % S]);
  if (tid < kd) sk[tid] = a.keys[tid];
  __syncthreads();
  bool miss = false;
  constexpr int U = kLowCardUnroll;
  const long long step = (long long)gridDim.x * T * U;
  for (long long base = (long long)blockIdx.x * T * U; base < a.n; base += step) {
    int slot[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = base + (long long)u * T + tid;
      slot[u] = -1;
      if (i < a.n) {
        const unsigned long long key = load_key(a.src.key, a.src.offset + i);
        int lo = 0, hi = kd - 1;  // the key's position among the sampled keys
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sk[mid] < key) lo = mid + 1; else hi = mid;
        }
        if (sk[lo] == key) slot[u] = lo; else miss = true;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (slot[u] < 0) continue;
      const long long i = base + (long long)u * T + tid;
      // the row's value for every aggregate, each source column read once
      // (aggregates in column order)
      long long val[KS];
      long long cv = 0;
      int cprev = -2;
#pragma unroll
      for (int q = 0; q < KS; ++q) {
        if (q < S) {
          const int c = a.fd.src[a.order[q]];
          if (c != cprev) {
            cv = c < 0 ? 1 : src_col(a.src, c, i);
            cprev = c;
          }
          val[q] = cv;
        }
      }
      long long* acc = lc_acc + (long long)slot[u] * S * T + tid;
      long long cur[KS];
#pragma unroll
      for (int q = 0; q < KS; ++q)
        if (q < S) cur[q] = acc[a.order[q] * T];
#pragma unroll
      for (int q = 0; q < KS; ++q)
        if (q < S) cur[q] = op_combine(a.fd.op[a.order[q]], cur[q], val[q]);
#pragma unroll
      for (int q = 0; q < KS; ++q)
        if (q < S) acc[a.order[q] * T] = cur[q];
    }
  }
  if (miss) atomicOr(a.overflow, 1);
  __syncthreads();
  // combine the block's threads: warp w takes accumulators w, w + warps, ...
  const int lane = tid & 31, nw = T >> 5;
  for (int q = tid >> 5; q < Q; q += nw) {
    const int op = a.fd.op[q % S];
    long long v = op_identity(op);
    for (int t = lane; t < T; t += 32) v = op_combine(op, v, lc_acc[q * T + t]);
    for (int o = 16; o > 0; o >>= 1) v = op_combine(op, v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) a.partial[(long long)blockIdx.x * Q + q] = v;
  }
}

// KL: how the key columns are read -- 0 any (load_key), 1 one 8-byte column,
// 2 two 1-byte columns -- so that the loads of a step batch across rows.
template <int KL>
__device__ __forceinline__ unsigned long long lc_key(const KeyCols& k, long long i) {
  if (KL == 1) return __ldg(reinterpret_cast<const unsigned long long*>(k.cols[0]) + i);
  if (KL == 2)
    return ((unsigned long long)__ldg(reinterpret_cast<const uint8_t*>(k.cols[0]) + i) << 8) |
           (unsigned long long)__ldg(reinterpret_cast<const uint8_t*>(k.cols[1]) + i);
  return load_key(k, i);
}

// The report pattern of aggregates (count(*), then sum, min and max of each
// of CP payload columns in order -- the shape of Example 1's query): every
// accumulator sits at a compile-time offset and each column is read once
// per row.  Lanes l and l + 16 of a warp share one set of accumulators and
// update it in turns (the lower half-warp, then the upper), so a thread
// needs half the shared memory of a set of its own and three CTAs fit an SM
// (the accumulators of 256 threads each would allow two: measured on 2^28
// rows, 2.69 ms against 3.01).  U rows per thread per step, loaded at once.
// Partials as k_lowcard's, over the 128 lane pairs of the block.
template <int CP, int KL>
__global__ void __launch_bounds__(256, 3) k_lowcard_report(LowCardArgs a) {
  constexpr int T = 256, P = T / 2, S = 1 + 3 * CP, U = 4;
  extern __shared__ long long lc_acc[];
  __shared__ unsigned long long sk[kLowCardKeys];
  const int tid = threadIdx.x, lane = tid & 31, half = lane >> 4;
  const int pid = (tid >> 5) * 16 + (lane & 15);  // the accumulator set of this lane pair
  const int kd = a.kd, Q = kd * S;
  if (half == 0)
    for (int q = 0; q < Q; ++q) {
      const int ag = q % S;
      lc_acc[q * P + pid] = ag == 0 ? 0 : ((ag - 1) % 3 == 0 ? 0 : ((ag - 1) % 3 == 1 ? INT64_MAX : INT64_MIN));
    }
  if (tid < kd) sk[tid] = a.keys[tid];
  __syncthreads();
  bool miss = false;
  const long long step = (long long)gridDim.x * T * U;
  for (long long base = (long long)blockIdx.x * T * U; base < a.n; base += step) {
    int slot[U];
    unsigned long long key[U];
    long long v[U][CP];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = base + (long long)u * T + tid;
      key[u] = 0;
#pragma unroll
      for (int c = 0; c < CP; ++c) v[u][c] = 0;
      if (i < a.n) {
        key[u] = lc_key<KL>(a.src.key, a.src.offset + i);
#pragma unroll
        for (int c = 0; c < CP; ++c) v[u][c] = __ldg(a.src.cols[c] + a.src.offset + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      slot[u] = -1;
      if (base + (long long)u * T + tid < a.n) {
        int lo = 0, hi = kd - 1;  // the key's position among the sampled keys
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sk[mid] < key[u]) lo = mid + 1; else hi = mid;
        }
        if (sk[lo] == key[u]) slot[u] = lo; else miss = true;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (half == h && slot[u] >= 0) {
          long long* acc = lc_acc + slot[u] * (S * P) + pid;
          long long cur[S];
#pragma unroll
          for (int q = 0; q < S; ++q) cur[q] = acc[q * P];
          cur[0] += 1;
#pragma unroll
          for (int c = 0; c < CP; ++c) {
            const long long x = v[u][c];
            cur[1 + 3 * c] = (long long)((unsigned long long)cur[1 + 3 * c] + (unsigned long long)x);
            cur[2 + 3 * c] = x < cur[2 + 3 * c] ? x : cur[2 + 3 * c];
            cur[3 + 3 * c] = x > cur[3 + 3 * c] ? x : cur[3 + 3 * c];
          }
#pragma unroll
          for (int q = 0; q < S; ++q) acc[q * P] = cur[q];
        }
        __syncwarp();  // the other half-warp's turn sees these stores
      }
    }
  }
  if (miss) atomicOr(a.overflow, 1);
  __syncthreads();
  const int nw = T >> 5;
  for (int q = tid >> 5; q < Q; q += nw) {
    const int op = a.fd.op[q % S];
    long long x = op_identity(op);
    for (int t = lane; t < P; t += 32) x = op_combine(op, x, lc_acc[q * P + t]);
    for (int o = 16; o > 0; o >>= 1) x = op_combine(op, x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) a.partial[(long long)blockIdx.x * Q + q] = x;
  }
}

// One block: the blocks' partials combined, the kd keys and their
// aggregates written (when they fit out.capacity), *rows = kd.
__global__ void k_lowcard_finish(LowCardArgs a, int blocks, OutSinkLite out, long long* rows) {
  const int S = a.fd.n_state, Q = a.kd * S;
  const bool fits = a.kd <= out.capacity;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = threadIdx.x >> 5; q < Q; q += nw) {  // a warp per accumulator, lanes over blocks
    const int op = a.fd.op[q % S];
    long long v = op_identity(op);
    for (int b = lane; b < blocks; b += 32) v = op_combine(op, v, a.partial[(long long)b * Q + q]);
    for (int o = 16; o > 0; o >>= 1) v = op_combine(op, v, __shfl_xor_sync(0xffffffffu, v, o));
    if (fits && lane == 0) out.cols[q % S][q / S] = v;
  }
  for (int g = threadIdx.x; g < a.kd; g += blockDim.x)
    if (fits) store_key(out.kout, g, a.keys[g]);
  if (threadIdx.x == 0) *rows = a.kd;
}

}  // namespace sg
