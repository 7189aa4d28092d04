// sg_merge.cuh -- the wide merge of sorted runs (Sec. 4, wide merging): all
// runs are consumed in one step and equal keys keep folding across runs, so
// the output leaves sorted and fully aggregated.
//
// Every run is sorted and holds each key at most once (runs are folded when
// written).  The planner cuts every run at the same fine-bucket boundaries
// (the runs' sparse indexes), so a merge tile is a key range owned outright
// by one CTA, and its k slices, one per run, are sorted lists.  Per tile:
//   1. a control warp reads the k slice bounds (a table the planner fills),
//      lays the slices out in shared memory and issues one bulk copy
//      (cp.async.bulk, global -> shared, completion on an mbarrier) per
//      slice and column: keys and state columns arrive in slice order;
//   2. the tile's rows are put in key order: a counting sort on the key bits
//      below the tile's common prefix (2^12 buckets, about two per row), then
//      only buckets holding an inversion (different keys out of order) are
//      finished by insertion.  A tile whose keys crowd a few buckets (a
//      bucket of more than 32 rows out of order) is merged instead: ceil(log2
//      k) levels of pairwise merges of the sorted slices, split across
//      threads by merge-path diagonals;
//   3. each worker thread takes IPT consecutive sorted rows into registers;
//      heads (first rows of equal keys) and their ranks come from one scan;
//   4. every state column is folded from registers (segmented by the heads;
//      the group open at a thread's end takes the leading partials of the
//      next threads) and staged in output order in its own column buffer;
//   5. every output column leaves in coalesced 16-byte stores at the tile's
//      output base, which a count pass before the merge (k_merge_count: each
//      tile's distinct keys through a shared-memory hash set) and a scan of
//      the counts (k_merge_scan) fixed: no tile waits on another.
#pragma once
#include "sg_sortfold.cuh"

namespace sg {

constexpr int kMergeTile = 2048;                           // rows of one merge tile at most
constexpr int kMergeCapMax = kMergeTile + 2 * kMaxFanIn;   // slice-order elements (rows + pads)
constexpr int kMergeBucketBits = 12;
constexpr int kMergeBuckets = 1 << kMergeBucketBits;
constexpr int kMergeFlagList = 1024;                       // buckets with an inversion listed
constexpr int kMergeFixMax = 32;                           // rows of a bucket sorted by insertion

// One merge launch.  fd is the identity fold of the state columns: output
// column s folds run column s by fd.op[s].
struct MergeArgs {
  const Chunk* chunks;
  const long long* tbase;  // [tiles]: output row of every tile's first group (k_merge_scan)
  const long long* tslo;   // [(tiles + 1) * k]: tile t's slice of run r starts at row tslo[t * k + r]
                           // and ends where tile t + 1's starts
  RunSet runs;
  CopySrc copy;
  FoldDesc fd;
  OutSink out;
  LookBack lb;   // the error word and the wait limit (tiles do not wait on one another)
  int capk;     // elements of the key buffer and of every column buffer (a multiple
                // of 16, at least tile rows + 2k, at most kMergeCapMax)
  int scol;     // state-column buffers (at least 2)
  int bulk;     // how slices reach shared memory: 1 one bulk copy per slice
                //    and column (cp.async.bulk) issued by the control warp, 3
                //    the same bulk copies issued by the worker warps (a slice
                //    per warp, an array per lane), 2 16-byte cp.async copies
                //    by every worker -- all need every run array in device
                //    memory, 16-byte aligned, with one readable row past its
                //    last run row; 0 plain loads
};

// Position p of a dense ping-pong buffer, swizzled inside its 16-element
// block so that a warp's writes of consecutive items per thread (stride
// IPT) spread over all banks.
__device__ __forceinline__ int mswz(int p) { return p ^ ((p >> 4) & 15); }

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// is parked by the hardware for up to `ns` nanoseconds (woken when the phase
// completes) instead of polling.
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long* bar, unsigned parity, unsigned ns) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Bounded wait for an mbarrier phase: at most spin_limit / 16 + 1 parked
// waits of 2 us each; false (and ERR_TIMEOUT raised) when the limit runs out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, const LookBack& lb) {
  const long long lim = lb.spin_limit / 16 + 1;
  for (long long i = 0; i <= lim; ++i)
    if (mbar_try_wait_sleep(bar, parity, 2000u)) return true;
  err_raise(lb.err, ERR_TIMEOUT);
  return false;
}

// Bulk copy of `bytes` (a positive multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory layout of one merge CTA (dynamic part).
struct MergeSmem {
  unsigned long long* A;   // [capk] slice-order keys; then the output keys
  long long* C;            // [scol][capk] slice-order state columns, each then its staged
                           // output; a crowded tile first merges in this area
  uint16_t* sidx;          // [capk] slice-order index of each sorted position
  uint32_t* cnt;           // [kMergeBuckets / 2] packed 16-bit bucket counts, then starts
  uint32_t* vm;            // [capk / 32] slice-order positions holding a row (not a pad)
  uint32_t* fbits;         // [kMergeBuckets / 32] buckets holding an inversion
  uint16_t* flist;         // [kMergeFlagList] those buckets
  int* D;                  // [k + 1] dense prefix of the slice lengths
  int* RS;                 // [k + 1] start of each slice's region in slice order (even)
  int* DS;                 // [k]     first element of each slice's rows in slice order
  long long* LO;           // [k]     first run row of each slice
  long long* lead;         // [2][threads] leading partial of every thread (column parity)
  unsigned char* hh;       // [threads] thread holds a head
  unsigned long long* bar; // [2] mbarriers: keys, state columns
};

__host__ __device__ inline size_t merge_smem_bytes(int capk, int scol, int k, int threads) {
  size_t b = (size_t)capk * 8 * (1 + scol) + (size_t)capk * 2 + (size_t)kMergeBuckets / 2 * 4 +
             (size_t)capk / 32 * 4 + (size_t)kMergeBuckets / 32 * 4 + (size_t)kMergeFlagList * 2;
  b += (size_t)(k + 1) * 4 * 2 + (size_t)k * 4;
  b = (b + 7) & ~(size_t)7;
  b += (size_t)k * 8 + (size_t)2 * threads * 8 + 16;  // LO, lead, bar
  b += (size_t)threads;                               // hh
  return (b + 127) & ~(size_t)127;
}

__device__ __forceinline__ MergeSmem merge_carve(unsigned char* base, int capk, int scol, int k, int threads) {
  MergeSmem m;
  unsigned char* p = base;
  m.A = reinterpret_cast<unsigned long long*>(p); p += (size_t)capk * 8;
  m.C = reinterpret_cast<long long*>(p); p += (size_t)capk * 8 * scol;
  m.sidx = reinterpret_cast<uint16_t*>(p); p += (size_t)capk * 2;
  m.cnt = reinterpret_cast<uint32_t*>(p); p += (size_t)kMergeBuckets / 2 * 4;
  m.vm = reinterpret_cast<uint32_t*>(p); p += (size_t)capk / 32 * 4;
  m.fbits = reinterpret_cast<uint32_t*>(p); p += (size_t)kMergeBuckets / 32 * 4;
  m.flist = reinterpret_cast<uint16_t*>(p); p += (size_t)kMergeFlagList * 2;
  m.D = reinterpret_cast<int*>(p); p += (size_t)(k + 1) * 4;
  m.RS = reinterpret_cast<int*>(p); p += (size_t)(k + 1) * 4;
  m.DS = reinterpret_cast<int*>(p); p += (size_t)k * 4;
  p = base + ((size_t)(p - base + 7) & ~(size_t)7);
  m.LO = reinterpret_cast<long long*>(p); p += (size_t)k * 8;
  m.lead = reinterpret_cast<long long*>(p); p += (size_t)2 * threads * 8;
  m.bar = reinterpret_cast<unsigned long long*>(p); p += 16;
  m.hh = p;
  return m;
}

// One level of pairwise merges.  At level `span` (2, 4, 8, ...) output list
// i is the merge of input lists 2i and 2i+1, i.e. of slices
// [i*span, i*span + span/2) and [i*span + span/2, (i+1)*span); its outputs
// are dense positions [D[i*span], D[min((i+1)*span, k)]).  FIRST: the input
// lists are the slices themselves, in slice order (DS); otherwise they are
// dense ranges of the previous level's swizzled buffer.  FINAL: the thread's
// IPT outputs (positions d0 .. d0 + IPT - 1) stay in K / X; otherwise they
// are written to kout / xout.  Equal keys may come out in either order: the
// fold that follows is order-free.
template <bool FIRST, bool FINAL, int IPT>
__device__ __forceinline__ void merge_level(const MergeSmem& m, int span, int k, int n,
                                            const unsigned long long* kin, const uint16_t* xin,
                                            unsigned long long* kout, uint16_t* xout, int d0,
                                            unsigned long long (&K)[IPT], int (&X)[IPT]) {
  if (d0 >= n) return;
  const int half = span >> 1;
  const int nl = (k + span - 1) / span;
  // output list holding position d0: the last list starting at or before it
  int li;
  {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (m.D[mid * span] <= d0) lo = mid; else hi = mid - 1;
    }
    li = lo;
  }
  int abase, bbase, la, lb, ostart;
  auto setup = [&](int i) {
    const int sa = i * span, sb = min(sa + half, k), se = min(sa + span, k);
    ostart = m.D[sa];
    la = m.D[sb] - ostart;
    lb = m.D[se] - m.D[sb];
    if (FIRST) {
      abase = m.DS[sa];
      bbase = sb < k ? m.DS[sb] : 0;
    } else {
      abase = ostart;
      bbase = m.D[sb];
    }
  };
  auto key_at = [&](int base, int x) -> unsigned long long {
    return FIRST ? kin[base + x] : kin[mswz(base + x)];
  };
  auto idx_at = [&](int base, int x) -> int { return FIRST ? base + x : (int)xin[mswz(base + x)]; };
  setup(li);
  // merge path: ia outputs of the first d0 - ostart come from list a
  int ia, ib;
  {
    const int dl = d0 - ostart;
    int plo = max(0, dl - lb), phi = min(dl, la);
    while (plo < phi) {
      const int mid = (plo + phi) >> 1;
      if (key_at(abase, mid) <= key_at(bbase, dl - 1 - mid)) plo = mid + 1; else phi = mid;
    }
    ia = plo;
    ib = dl - plo;
  }
  unsigned long long ka = 0, kb = 0;
  int xa = 0, xb = 0;
  if (ia < la) { ka = key_at(abase, ia); xa = idx_at(abase, ia); }
  if (ib < lb) { kb = key_at(bbase, ib); xb = idx_at(bbase, ib); }
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const int p = d0 + j;
    if (p < n) {
      // the list is exhausted: the next non-empty list starts here
      while (ia == la && ib == lb && li + 1 < nl) {
        setup(++li);
        ia = 0;
        ib = 0;
        if (la > 0) { ka = key_at(abase, 0); xa = idx_at(abase, 0); }
        if (lb > 0) { kb = key_at(bbase, 0); xb = idx_at(bbase, 0); }
      }
      const bool ta = ia < la && (ib >= lb || ka <= kb);
      const unsigned long long key = ta ? ka : kb;
      const int idx = ta ? xa : xb;
      if (FINAL) {
        K[j] = key;
        X[j] = idx;
      } else {
        kout[mswz(p)] = key;
        xout[mswz(p)] = (uint16_t)idx;
      }
      const int nxt = (ta ? ia : ib) + 1;
      const int lim = ta ? la : lb;
      const int bs = ta ? abase : bbase;
      unsigned long long v = 0;
      int vx = 0;
      if (nxt < lim) {
        v = key_at(bs, nxt);
        vx = idx_at(bs, nxt);
      }
      if (ta) { ia = nxt; ka = v; xa = vx; } else { ib = nxt; kb = v; xb = vx; }
    }
  }
}

template <int OP>
__device__ __forceinline__ long long mop_id() {
  return OP == OP_SUM ? 0 : (OP == OP_MIN ? INT64_MAX : INT64_MIN);
}

template <int OP>
__device__ __forceinline__ long long mop(long long a, long long b) {
  if (OP == OP_SUM) return (long long)((unsigned long long)a + (unsigned long long)b);
  if (OP == OP_MIN) return b < a ? b : a;
  return b > a ? b : a;
}

// Named barrier 1 of a merge CTA: the worker threads (threads 0 .. THREADS
// - 1) among themselves (the control warp, the last warp, leaves after the
// prologue).
template <int NT>
__device__ __forceinline__ void wsync() { asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory"); }

// Fold one state column over the IPT sorted rows a thread holds (slice-
// order indexes X, heads hm): R[j] is the fold from the row's group head (or
// the thread's first row) to row j.  A group that closes inside the thread
// is written at once; the rows before the thread's first head are its
// leading partial, taken by the thread holding that group's head, which
// walks the following threads until one holds a head.  col is read before
// the barrier and written (staged output, rank order) after it.
template <int OP, int THREADS, int IPT>
__device__ __forceinline__ void fold_column(const MergeSmem& m, long long* col, const int (&X)[IPT], unsigned hm,
                                            int n, int nv, int g0, int par) {
  long long R[IPT];
  long long run = mop_id<OP>(), lead = mop_id<OP>();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if (j < nv) {
      const long long v = col[X[j]];
      run = ((hm >> j) & 1u) ? v : mop<OP>(run, v);
      if ((hm & ((2u << j) - 1u)) == 0) lead = run;  // no head yet: the leading partial
    }
    R[j] = run;
  }
  long long* ld = m.lead + par * THREADS;
  ld[threadIdx.x] = lead;
  wsync<THREADS>();
#pragma unroll
  for (int j = 0; j + 1 < IPT; ++j) {
    const unsigned upto = hm & ((2u << j) - 1u);
    if (j + 1 < nv && upto && ((hm >> (j + 1)) & 1u)) col[g0 + __popc(upto) - 1] = R[j];
  }
  if (hm) {  // the group open at the thread's end
    long long acc = R[0];
#pragma unroll
    for (int j = 1; j < IPT; ++j)
      if (j == nv - 1) acc = R[j];
    for (int t2 = threadIdx.x + 1; t2 < THREADS && t2 * IPT < n; ++t2) {
      acc = mop<OP>(acc, ld[t2]);
      if (m.hh[t2]) break;
    }
    col[g0 + __popc(hm) - 1] = acc;
  }
}

// Rows [0, count) of a staged column to dst[base ...], positions below cap
// only: 16-byte stores from an aligned position, single words at the ends.
template <int THREADS>
__device__ __forceinline__ void store_staged(long long* dst, const long long* src, int count, long long base,
                                             long long cap) {
  const long long room = cap - base;
  const int mcount = room <= 0 ? 0 : (int)min((long long)count, room);
  if (mcount <= 0) return;
  long long* d = dst + base;
  const int head = (reinterpret_cast<unsigned long long>(d) & 15ull) ? 1 : 0;
  if (head && threadIdx.x == 0) d[0] = src[0];
  const int pairs = (mcount - head) >> 1;
  for (int q = threadIdx.x; q < pairs; q += THREADS) {
    const int i = head + 2 * q;
    longlong2 v;
    v.x = src[i];
    v.y = src[i + 1];
    *reinterpret_cast<longlong2*>(d + i) = v;
  }
  if (((mcount - head) & 1) && threadIdx.x == THREADS - 1) d[mcount - 1] = src[mcount - 1];
}

__device__ __forceinline__ int mbin(const uint32_t* cnt, int b) { return (int)((cnt[b >> 1] >> ((b & 1) * 16)) & 0xFFFFu); }

// Bulk (or plain) copies of state columns [c0, c0 + gc) of every slice into
// the column buffers, completing on bar[1].  Called by one full warp.
__device__ __forceinline__ void stage_columns(const MergeArgs& a, const MergeSmem& m, int k, int E, int c0, int gc) {
  const int lane = threadIdx.x & 31;
  const int S = a.runs.ncols;
  if (lane == 0) mbar_arrive_tx(&m.bar[1], (a.bulk == 1 || a.bulk == 3) ? (unsigned)E * 8u * (unsigned)gc : 0u);
  __syncwarp();
  if (a.bulk != 1 && a.bulk != 3) return;
  for (int r = lane; r < k; r += 32) {
    const int cnt = m.RS[r + 1] - m.RS[r];
    if (cnt == 0) continue;
    const long long row0 = m.LO[r] - (m.DS[r] - m.RS[r]);
    const long long* const* pr = a.runs.ptrs + (long long)r * (1 + S);
    for (int c = 0; c < gc; ++c)
      bulk_g2s(m.C + (size_t)c * a.capk + m.RS[r], pr[1 + c0 + c] + row0, (unsigned)cnt * 8u, &m.bar[1]);
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

// 16-byte asynchronous copies (cp.async) of the slices of the keys (keys)
// and of state columns [c0, c0 + gc), issued by all workers, a warp per
// slice; complete and visible to every worker when it returns.
template <int THREADS>
__device__ __forceinline__ void copy_async16(const MergeArgs& a, const MergeSmem& m, int k, int c0, int gc,
                                             bool keys) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int S = a.runs.ncols;
  for (int r = w; r < k; r += THREADS / 32) {
    const int cnt = m.RS[r + 1] - m.RS[r];
    if (cnt == 0) continue;
    const long long row0 = m.LO[r] - (m.DS[r] - m.RS[r]);
    const long long* const* pr = a.runs.ptrs + (long long)r * (1 + S);
    const int chunks = cnt >> 1;
    for (int q = keys ? -1 : 0; q < gc; ++q) {
      const long long* src = (q < 0 ? pr[0] : pr[1 + c0 + q]) + row0;
      long long* dst = (q < 0 ? reinterpret_cast<long long*>(m.A) : m.C + (size_t)q * a.capk) + m.RS[r];
      for (int c = lane; c < chunks; c += 32) cp_async16(dst + 2 * c, src + 2 * c);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  wsync<THREADS>();
}

// The first staging of a tile (keys and the first gc state columns) as bulk
// copies issued by the worker warps: warp w takes slices w, w + W, ...; lane
// 0 copies the slice's keys, lane 1 + c its column c.  The mbarriers are
// armed by the control warp.
template <int THREADS>
__device__ __forceinline__ void bulk_by_workers(const MergeArgs& a, const MergeSmem& m, int k, int gc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int S = a.runs.ncols;
  for (int r = w; r < k; r += THREADS / 32) {
    const int cnt = m.RS[r + 1] - m.RS[r];
    if (cnt == 0 || lane > gc) continue;
    const long long row0 = m.LO[r] - (m.DS[r] - m.RS[r]);
    const long long* const* pr = a.runs.ptrs + (long long)r * (1 + S);
    if (lane == 0) bulk_g2s(m.A + m.RS[r], pr[0] + row0, (unsigned)cnt * 8u, &m.bar[0]);
    else bulk_g2s(m.C + (size_t)(lane - 1) * a.capk + m.RS[r], pr[lane] + row0, (unsigned)cnt * 8u, &m.bar[1]);
  }
}

// Plain loads of the same (runs in host memory or not aligned): all threads.
template <int THREADS>
__device__ __forceinline__ void load_columns_plain(const MergeArgs& a, const MergeSmem& m, int k, int n, int c0,
                                                   int gc, bool keys) {
  const int S = a.runs.ncols;
  for (int p = threadIdx.x; p < n; p += THREADS) {
    int lo = 0, hi = k - 1;  // slice holding dense position p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (m.D[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const long long row = m.LO[lo] + (p - m.D[lo]);
    const int e = m.DS[lo] + (p - m.D[lo]);
    const long long* const* pr = a.runs.ptrs + (long long)lo * (1 + S);
    if (keys) m.A[e] = (unsigned long long)pr[0][row];
    for (int c = 0; c < gc; ++c) m.C[(size_t)c * a.capk + e] = pr[1 + c0 + c][row];
  }
}

// Worker 0 waits (bounded) for phase `parity` of bar; false, for every
// worker alike, after a timeout (the error word is raised; worker 0 has
// waited a second time for the copies in flight).  Every worker then
// acquires the completed phase itself.
template <int THREADS>
__device__ __forceinline__ bool workers_wait(unsigned long long* bar, unsigned parity, const LookBack& lb,
                                             int* s_flag) {
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait(bar, parity, lb);
    if (!ok) mbar_wait(bar, parity, lb);
    *s_flag = ok ? 1 : 0;
  }
  wsync<THREADS>();
  if (!*s_flag) return false;
  mbar_try_wait(bar, parity);
  return true;
}


// The planner's slice table: tslo[t * k + r] = offs[r][f_lo of tile t] (the
// first row of run r in tile t), and one more row for the end of the last
// tile, offs[r][f_hi of the last tile].
__global__ void k_tile_slices(const Chunk* chunks, int n_chunks, const long long* const* offs, int k,
                              long long* tslo) {
  const long long total = (long long)(n_chunks + 1) * k;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / k), r = (int)(i % k);
    const int f = t < n_chunks ? chunks[t].f_lo : chunks[n_chunks - 1].f_hi;
    tslo[i] = offs[r][f];
  }
}

// ---------------------------------------------------------------------------
// Every tile's output rows before the merge: a tile's distinct keys are
// counted by inserting its keys into an open-addressing hash set in shared
// memory (no sort), and a scan of the counts gives every tile its output
// base -- so merge tiles never wait on one another.
// ---------------------------------------------------------------------------
constexpr int kCountThreads = 256;
constexpr int kCountSlotBits = 12;   // 4,096 slots for at most 2,048 keys
constexpr int kCountSlots = 1 << kCountSlotBits;

// count[t] = distinct keys of tile t (its rows, for a tile solved apart).
// Warp w takes slices w, w + 8, ...: their bounds and key addresses go to
// shared memory, and the warp walks its slices' rows as one array (lane +
// 32 u, kCountUnroll loads in flight per lane), a row's slice found by a
// short scan of the warp's slice starts.  The keys go into an
// open-addressing hash set in shared memory (at most kMergeTile keys in
// twice as many slots, so a free slot is near); the set's size is the count.
constexpr int kCountWarps = kCountThreads / 32;
constexpr int kCountWarpSlices = kMaxFanIn / kCountWarps;  // slices of one warp at most
constexpr int kCountUnroll = 8;

__device__ __forceinline__ unsigned count_hash(unsigned long long key) {
  const unsigned x = (unsigned)key ^ (unsigned)(key >> 32);
  return (x * 0x9E3779B1u) >> (32 - kCountSlotBits);
}

__global__ void __launch_bounds__(kCountThreads) k_merge_count(const Chunk* __restrict__ chunks,
                                                               const long long* __restrict__ tslo, RunSet runs,
                                                               long long* count, int* err) {
  __shared__ __align__(16) unsigned long long tab[kCountSlots];
  __shared__ const long long* wadr[kCountWarps][kCountWarpSlices];  // key address of a slice's first row
  __shared__ int wst[kCountWarps][kCountWarpSlices + 1];           // warp rows before each slice
  __shared__ int s_cnt, s_top;
  const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const Chunk ch = chunks[t];
  if (ch.kind == CH_COPY) {
    if (tid == 0) count[t] = ch.hi - ch.lo;
    return;
  }
  ulonglong2* t2 = reinterpret_cast<ulonglong2*>(tab);
  for (int i = tid; i < kCountSlots / 2; i += kCountThreads) t2[i] = make_ulonglong2(~0ull, ~0ull);  // empty
  if (tid == 0) {
    s_cnt = 0;
    s_top = 0;
  }
  const int k = runs.k;
  const int ns = k > w ? (k - w + kCountWarps - 1) / kCountWarps : 0;  // this warp's slices
  int run = 0;
  for (int q0 = 0; q0 < ns; q0 += 32) {
    const int q = q0 + lane;
    int len = 0;
    if (q < ns) {
      const int r = w + kCountWarps * q;
      const long long lo = tslo[(long long)t * k + r], hi = tslo[(long long)(t + 1) * k + r];
      len = (int)min(max(hi - lo, 0ll), (long long)kMergeTile);
      wadr[w][q] = runs.ptrs[(long long)r * (1 + runs.ncols)] + lo;
    }
    int x = len;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (q < ns) wst[w][q] = run + x - len;
    run = min(run + __shfl_sync(0xffffffffu, x, 31), kMergeTile);
  }
  if (lane == 0) wst[w][ns] = run;
  __syncthreads();  // the table is empty; every warp's slices are laid out
  int mine = 0;
  for (int b = 0; b < run; b += 32 * kCountUnroll) {
    unsigned long long key[kCountUnroll];
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      const int p = b + lane + 32 * u;
      key[u] = 0;
      if (p < run) {
        int q = 0;
        while (q + 1 < ns && wst[w][q + 1] <= p) ++q;
        key[u] = (unsigned long long)__ldg(wadr[w][q] + (p - wst[w][q]));
      }
    }
#pragma unroll
    for (int u = 0; u < kCountUnroll; ++u) {
      if (b + lane + 32 * u >= run) continue;
      const unsigned long long kk = key[u];
      if (kk == ~0ull) {  // the empty mark as a key: counted apart
        if (atomicExch(&s_top, 1) == 0) ++mine;
        continue;
      }
      unsigned slot = count_hash(kk);
      int probes = 0;
      while (true) {
        const unsigned long long old = atomicCAS(&tab[slot], ~0ull, kk);
        if (old == ~0ull) { ++mine; break; }
        if (old == kk) break;
        slot = (slot + 1) & (kCountSlots - 1);
        if (++probes == kCountSlots) {  // cannot happen with at most half the slots taken
          err_raise(err, ERR_INTERNAL);
          break;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (lane == 0) atomicAdd(&s_cnt, mine);
  __syncthreads();
  if (tid == 0) count[t] = s_cnt;
}

// base[t] = *base_in + count[0] + ... + count[t - 1]; *total_out = the end;
// ERR_CAPACITY when the end exceeds the output capacity.  Blocks of 1,024
// tiles in ticket order, chained by decoupled look-back.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_merge_scan(const long long* count, int n, long long* base,
                                                             LookBack lb, long long capacity) {
  __shared__ int s_id;
  __shared__ long long s_w[kScanThreads / 32];
  __shared__ long long s_pre;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) s_id = (int)atomicAdd(lb.ticket, 1u);
  __syncthreads();
  const int b = s_id;
  const int i = b * kScanThreads + tid;
  const long long v = i < n ? count[i] : 0;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  long long before = 0, total = 0;
  for (int q = 0; q < kScanThreads / 32; ++q) {
    before += q < w ? s_w[q] : 0;
    total += s_w[q];
  }
  if (tid < 32) {
    const long long pre = lookback_warp(lb, b, total);
    if (tid == 0) {
      s_pre = pre;
      if (pre >= 0 && b == lb.n_chunks - 1) {
        if (lb.total_out) *lb.total_out = pre + total;
        if (pre + total > capacity) err_raise(lb.err, ERR_CAPACITY);
      }
    }
  }
  __syncthreads();
  if (s_pre >= 0 && i < n) base[i] = s_pre + before + x - v;
}

// One CTA per merge tile: THREADS worker threads and one control warp.
template <int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS + 32, (THREADS <= 256 ? 3 : 2)) k_merge(MergeArgs a) {
  constexpr int W = THREADS / 32;               // worker warps
  constexpr int NALL = THREADS + 32;
  constexpr int EPT = (kMergeCapMax + THREADS - 1) / THREADS;
  constexpr int BPT = kMergeBuckets / THREADS;  // buckets per worker in the scan
  static_assert(BPT % 2 == 0 && BPT * THREADS == kMergeBuckets, "bucket scan layout");
  static_assert(IPT * THREADS == kMergeTile, "tile layout");
  extern __shared__ __align__(128) unsigned char msmem[];
  __shared__ int s_err, s_ok, s_n, s_E, s_flag, s_crowd, s_nflag;
  __shared__ unsigned long long s_kmin, s_kmax, s_wlast[W];
  __shared__ int s_wcnt[W];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const bool control = w == W;
  const LookBack& lb = a.lb;
  const OutSink& out = a.out;

  const int cid = blockIdx.x;
  // the control warp's first 32 slice bounds and everyone's chunk are read
  // before the barrier, so their latency overlaps it (tslo holds
  // (n_chunks + 1) x k entries and every tile, copy chunks too, has a row)
  long long lo0 = 0, hi0 = 0;
  if (control && lane < a.runs.k) {
    lo0 = a.tslo[(long long)cid * a.runs.k + lane];
    hi0 = a.tslo[(long long)(cid + 1) * a.runs.k + lane];
  }
  const Chunk ch = a.chunks[cid];
  if (tid == THREADS) s_err = err_load(lb.err);
  __syncthreads();
  if (s_err) return;  // block-uniform

  if (ch.kind == CH_COPY) {  // a key range solved apart: its rows are copied verbatim
    const long long n = ch.hi - ch.lo;
    const long long base = a.tbase[cid];
    for (long long g = tid; g < n; g += NALL) {
      const unsigned long long key = a.copy.keys[ch.lo + g];
      sink_key(out, base + g, key);
      if (out.offs)
        write_fine_offsets(out, ch, base, g, n, key, g > 0, g > 0 ? a.copy.keys[ch.lo + g - 1] : 0ull);
      for (int st = 0; st < a.fd.n_state; ++st) sink_val(out, st, base + g, a.copy.cols[st][ch.lo + g]);
    }
    if (out.offs && n == 0 && tid == 0)
      for (int ff = ch.f_lo; ff <= ch.f_hi; ++ff) out.offs[ff] = base;
    return;
  }

  const int k = a.runs.k;
  const int S = a.runs.ncols;
  const int capk = a.capk, scol = a.scol;
  const MergeSmem m = merge_carve(msmem, capk, scol, k, THREADS);
  const int g0cols = min(S, scol);

  // ---- control warp: slice bounds, layout, mbarriers, bulk copies ----
  if (control) {
    if (lane == 0) {
      mbar_init(&m.bar[0], 1);
      mbar_init(&m.bar[1], 1);
      mbar_fence_init();
    }
    int cd = 0, cr = 0;
    for (int b = 0; b < k; b += 32) {
      const int r = b + lane;
      long long lo = 0;
      int len = 0, ph = 0, cnt = 0;
      if (r < k) {
        lo = b == 0 ? lo0 : a.tslo[(long long)cid * k + r];
        const long long hi = b == 0 ? hi0 : a.tslo[(long long)(cid + 1) * k + r];
        len = (int)min(max(hi - lo, 0ll), (long long)capk);  // oversized tiles are refused below
        ph = (a.bulk != 0 && len > 0) ? (int)(lo & 1) : 0;
        cnt = len == 0 ? 0 : ((len + ph + 1) & ~1);
      }
      int xd = len, xr = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int yd = __shfl_up_sync(0xffffffffu, xd, o), yr = __shfl_up_sync(0xffffffffu, xr, o);
        if (lane >= o) { xd += yd; xr += yr; }
      }
      if (r < k) {
        m.LO[r] = lo;
        m.D[r + 1] = cd + xd;
        m.RS[r + 1] = cr + xr;
        m.DS[r] = cr + xr - cnt + ph;
      }
      cd += __shfl_sync(0xffffffffu, xd, 31);
      cr += __shfl_sync(0xffffffffu, xr, 31);
    }
    if (lane == 0) {
      m.D[0] = 0;
      m.RS[0] = 0;
    }
    const bool ok = cr <= capk && cd <= kMergeTile;
    __syncwarp();
    if (ok) {
      if (lane == 0) mbar_arrive_tx(&m.bar[0], (a.bulk == 1 || a.bulk == 3) ? (unsigned)cr * 8u : 0u);
      __syncwarp();
      if (a.bulk == 1) {
        for (int r = lane; r < k; r += 32) {
          const int cnt = m.RS[r + 1] - m.RS[r];
          if (cnt == 0) continue;
          const long long row0 = m.LO[r] - (m.DS[r] - m.RS[r]);
          bulk_g2s(m.A + m.RS[r], a.runs.ptrs[(long long)r * (1 + S)] + row0, (unsigned)cnt * 8u, &m.bar[0]);
        }
      }
      if (a.bulk == 3) {  // arm only: the workers copy
        if (lane == 0) mbar_arrive_tx(&m.bar[1], (unsigned)cr * 8u * (unsigned)g0cols);
        __syncwarp();
      } else {
        stage_columns(a, m, k, cr, 0, g0cols);
      }
      // slice-order positions holding a row: all of [0, cr) but the pads
      for (int q = lane; q < (cr + 31) / 32; q += 32) {
        const int left = cr - 32 * q;
        m.vm[q] = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
      }
      __syncwarp();
      for (int r = lane; r < k; r += 32) {
        const int rs = m.RS[r], re = m.RS[r + 1], ds = m.DS[r], de = ds + (m.D[r + 1] - m.D[r]);
        for (int e = rs; e < ds; ++e) atomicAnd(&m.vm[e >> 5], ~(1u << (e & 31)));
        for (int e = de; e < re; ++e) atomicAnd(&m.vm[e >> 5], ~(1u << (e & 31)));
      }
    }
    if (lane == 0) {
      s_ok = ok ? 1 : 0;
      s_n = cd;
      s_E = cr;
      s_kmin = ~0ull;
      s_kmax = 0ull;
      s_crowd = 0;
      s_nflag = 0;
    }
  } else {
    // meanwhile: the bucket counts and the inversion flags start at zero
    for (int i = tid; i < kMergeBuckets / 2; i += THREADS) m.cnt[i] = 0;
    for (int i = tid; i < kMergeBuckets / 32; i += THREADS) m.fbits[i] = 0;
  }
  __syncthreads();
  if (!s_ok) {  // the planner never makes such tiles; no copy was issued
    if (tid == 0) err_raise(lb.err, ERR_INTERNAL);
    return;
  }

  if (control) return;  // the control warp's part is done

  // ---- workers ----
  const int n = s_n, E = s_E;
  if (a.bulk == 0) {
    load_columns_plain<THREADS>(a, m, k, n, 0, g0cols, true);
    wsync<THREADS>();
  } else if (a.bulk == 2) {
    copy_async16<THREADS>(a, m, k, 0, g0cols, true);
  } else if (a.bulk == 3) {
    bulk_by_workers<THREADS>(a, m, k, g0cols);
  }
  if (!workers_wait<THREADS>(&m.bar[0], 0, lb, &s_flag)) return;

  // the tile's key range: slices are sorted
  if (tid < 32) {
    unsigned long long lmin = ~0ull, lmax = 0ull;
    for (int r = lane; r < k; r += 32) {
      const int len = m.D[r + 1] - m.D[r];
      if (len > 0) {
        lmin = min(lmin, m.A[m.DS[r]]);
        lmax = max(lmax, m.A[m.DS[r] + len - 1]);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if (lane == 0) {
      s_kmin = lmin;
      s_kmax = lmax;
    }
  }
  wsync<THREADS>();
  const unsigned long long kmin = s_kmin;
  const unsigned long long range = n > 0 ? s_kmax - kmin : 0ull;
  const int vb = range == 0 ? 0 : 64 - __clzll((long long)range);
  const int sh = vb > kMergeBucketBits ? vb - kMergeBucketBits : 0;

  // ---- counting sort on (key - kmin) >> sh; rank inside the bucket from the atomic ----
  uint32_t br[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = tid + j * THREADS;
    br[j] = 0xffffffffu;
    if (e < E && ((m.vm[e >> 5] >> (e & 31)) & 1u)) {
      const unsigned b = (unsigned)((m.A[e] - kmin) >> sh);
      const unsigned sft = (b & 1u) * 16u;
      const unsigned old = atomicAdd(&m.cnt[b >> 1], 1u << sft);
      br[j] = (b << 16) | ((old >> sft) & 0xFFFFu);
    }
  }
  wsync<THREADS>();
  {  // bucket starts: exclusive scan, BPT buckets per worker
    int c[BPT];
    int loc = 0;
#pragma unroll
    for (int q = 0; q < BPT; q += 2) {
      const uint32_t v = m.cnt[(tid * BPT + q) >> 1];
      c[q] = (int)(v & 0xFFFFu);
      c[q + 1] = (int)(v >> 16);
      loc += c[q] + c[q + 1];
    }
    int x = loc;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wcnt[w] = x;
    wsync<THREADS>();
    int start = x - loc;
#pragma unroll
    for (int q = 0; q < W; ++q) start += q < w ? s_wcnt[q] : 0;
#pragma unroll
    for (int q = 0; q < BPT; q += 2) {
      const unsigned lo = (unsigned)start;
      start += c[q];
      const unsigned hi = (unsigned)start;
      start += c[q + 1];
      m.cnt[(tid * BPT + q) >> 1] = lo | (hi << 16);
    }
  }
  wsync<THREADS>();
#pragma unroll
  for (int j = 0; j < EPT; ++j)
    if (br[j] != 0xffffffffu)
      m.sidx[mbin(m.cnt, (int)(br[j] >> 16)) + (int)(br[j] & 0xFFFFu)] = (uint16_t)(tid + j * THREADS);
  wsync<THREADS>();
  if (sh > 0) {  // uniform: a bucket may hold several keys
    // bucket b holds positions [start(b), start(b + 1)); an adjacent pair out
    // of key order lies inside one bucket, which is flagged and listed once
    for (int p0 = tid - lane; p0 < n; p0 += THREADS) {  // warp-uniform
      const int p = p0 + lane;
      const unsigned long long x = p < n ? m.A[m.sidx[p]] : ~0ull;
      unsigned long long y = __shfl_down_sync(0xffffffffu, x, 1);
      if (lane == 31 && p + 1 < n) y = m.A[m.sidx[p + 1]];
      if (p + 1 < n && x > y) {
        const int b = (int)((x - kmin) >> sh);
        const unsigned bit = 1u << (b & 31);
        if (!(atomicOr(&m.fbits[b >> 5], bit) & bit)) {
          const int q = atomicAdd(&s_nflag, 1);
          if (q < kMergeFlagList) m.flist[q] = (uint16_t)b;
        }
      }
    }
    wsync<THREADS>();
    const int nfl = s_nflag;
    if (nfl > kMergeFlagList) {
      if (tid == 0) s_crowd = 1;
    } else {
      // a warp per flagged bucket: lane l holds row l and ranks it by key
      // against the bucket's other rows (equal keys by lane)
      for (int q = w; q < nfl; q += W) {  // warp-uniform
        const int b = m.flist[q];
        const int st = mbin(m.cnt, b), en = b + 1 < kMergeBuckets ? mbin(m.cnt, b + 1) : n;
        const int cntb = en - st;
        if (cntb > kMergeFixMax) {
          if (lane == 0) s_crowd = 1;
          continue;
        }
        const bool act = lane < cntb;
        const uint16_t v = act ? m.sidx[st + lane] : (uint16_t)0;
        const unsigned long long kv = act ? m.A[v] : ~0ull;
        int rk = 0;
        for (int jj = 0; jj < cntb; ++jj) {
          const unsigned long long kj = __shfl_sync(0xffffffffu, kv, jj);
          rk += (kj < kv || (kj == kv && jj < lane)) ? 1 : 0;
        }
        __syncwarp();
        if (act) m.sidx[st + rk] = v;
        __syncwarp();
      }
    }
    wsync<THREADS>();
  }

  // ---- every worker: IPT consecutive sorted rows ----
  const int d0 = tid * IPT;
  const int nv = max(0, min(IPT, n - d0));
  unsigned long long K[IPT];
  int X[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) { K[j] = 0; X[j] = 0; }
  unsigned bphase = 0;  // next phase of the column mbarrier
  if (s_crowd) {
    // crowded buckets: merge the sorted slices instead (pairwise levels,
    // merge-path split), in the column area once its copies have landed
    if (!workers_wait<THREADS>(&m.bar[1], 0, lb, &s_flag)) return;
    unsigned long long* B = reinterpret_cast<unsigned long long*>(m.C);
    uint16_t* IA = reinterpret_cast<uint16_t*>(m.C + capk);
    uint16_t* IB = IA + capk;
    int levels = 1;
    while ((1 << levels) < k) ++levels;
    if (levels == 1) {
      merge_level<true, true, IPT>(m, 2, k, n, m.A, nullptr, nullptr, nullptr, d0, K, X);
    } else {
      merge_level<true, false, IPT>(m, 2, k, n, m.A, nullptr, B, IB, d0, K, X);
      wsync<THREADS>();
      for (int l = 2; l < levels; ++l) {
        const bool odd = (l & 1) != 0;  // level l reads the output of level l - 1
        merge_level<false, false, IPT>(m, 1 << l, k, n, odd ? m.A : B, odd ? IA : IB, odd ? B : m.A,
                                       odd ? IB : IA, d0, K, X);
        wsync<THREADS>();
      }
      const bool odd = (levels & 1) != 0;
      merge_level<false, true, IPT>(m, 1 << levels, k, n, odd ? m.A : B, odd ? IA : IB, nullptr, nullptr, d0, K,
                                    X);
    }
    wsync<THREADS>();  // the column area is free again: stage the columns anew
    if (w == 0) stage_columns(a, m, k, E, 0, g0cols);
    if (a.bulk == 0) {
      load_columns_plain<THREADS>(a, m, k, n, 0, g0cols, false);
      wsync<THREADS>();
    } else if (a.bulk == 2) {
      copy_async16<THREADS>(a, m, k, 0, g0cols, false);
    }
    bphase = 1;
  } else {
#pragma unroll
    for (int j = 0; j < IPT; ++j)
      if (j < nv) {
        X[j] = m.sidx[d0 + j];
        K[j] = m.A[X[j]];
      }
  }

  // ---- heads, ranks, the tile's count ----
  if (lane == 31) s_wlast[w] = K[IPT - 1];
  wsync<THREADS>();  // every worker holds its rows: A is free from here on
  unsigned long long prevk = __shfl_up_sync(0xffffffffu, K[IPT - 1], 1);
  if (lane == 0) prevk = w > 0 ? s_wlast[w - 1] : 0ull;
  unsigned hm = 0;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const unsigned long long pk = j == 0 ? prevk : K[j - 1];
    if (j < nv && (d0 + j == 0 || K[j] != pk)) hm |= 1u << j;
  }
  const int hc = __popc(hm);
  int x = hc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wcnt[w] = x;
  m.hh[tid] = hm != 0;
  wsync<THREADS>();
  int wpre = 0, count = 0;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    const int c = s_wcnt[q];
    wpre += q < w ? c : 0;
    count += c;
  }
  const int g0 = wpre + x - hc;
  {  // output keys, staged in A
    int r = g0;
#pragma unroll
    for (int j = 0; j < IPT; ++j)
      if ((hm >> j) & 1u) m.A[r++] = K[j];
  }

  // ---- fold the state columns, a group of scol at a time ----
  bool resolved = false;
  int par = 0;
  for (int c0 = 0; c0 < S || (c0 == 0 && !resolved); c0 += scol) {
    const int gc = min(scol, S - c0);
    if (gc > 0) {
      if (!workers_wait<THREADS>(&m.bar[1], bphase, lb, &s_flag)) return;
      bphase ^= 1u;
      for (int cl = 0; cl < gc; ++cl) {
        long long* col = m.C + (size_t)cl * capk;
        const int op = a.fd.op[c0 + cl];
        if (op == OP_SUM) fold_column<OP_SUM, THREADS, IPT>(m, col, X, hm, n, nv, g0, par);
        else if (op == OP_MIN) fold_column<OP_MIN, THREADS, IPT>(m, col, X, hm, n, nv, g0, par);
        else fold_column<OP_MAX, THREADS, IPT>(m, col, X, hm, n, nv, g0, par);
        par ^= 1;
      }
    }
    wsync<THREADS>();  // staged outputs complete
    const long long base = a.tbase[cid];
    if (!resolved) {
      resolved = true;
      // keys
      if (!out.user) {
        store_staged<THREADS>(reinterpret_cast<long long*>(out.keys), reinterpret_cast<const long long*>(m.A),
                              count, base, out.capacity);
      } else if (out.kout.n_cols == 1 && out.kout.bytes[0] == 8) {
        store_staged<THREADS>(reinterpret_cast<long long*>(out.kout.cols[0]),
                              reinterpret_cast<const long long*>(m.A), count, base, out.capacity);
      } else {
        for (int g = tid; g < count; g += THREADS)
          if (base + g < out.capacity) store_key(out.kout, base + g, m.A[g]);
      }
      // the written run's sparse index: offs[f] = first output row whose
      // fine digit is >= f, for every fine bucket of the tile's key range
      if (out.offs) {
        for (int f = ch.f_lo + tid; f <= ch.f_hi; f += THREADS) {
          int lo = 0, hi = count;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int)fine_digit(out.dig, m.A[mid]) < f) lo = mid + 1; else hi = mid;
          }
          out.offs[f] = base + lo;
        }
      }
    }
    for (int cl = 0; cl < gc; ++cl)
      store_staged<THREADS>(out.cols[c0 + cl], m.C + (size_t)cl * capk, count, base, out.capacity);
    if (c0 + scol < S) {
      wsync<THREADS>();  // the column buffers are read: stage the next group
      if (w == 0) stage_columns(a, m, k, E, c0 + scol, min(scol, S - c0 - scol));
      if (a.bulk == 0) {
        load_columns_plain<THREADS>(a, m, k, n, c0 + scol, min(scol, S - c0 - scol), false);
        wsync<THREADS>();
      } else if (a.bulk == 2) {
        copy_async16<THREADS>(a, m, k, c0 + scol, min(scol, S - c0 - scol), false);
      }
    }
  }
}

}  // namespace sg
