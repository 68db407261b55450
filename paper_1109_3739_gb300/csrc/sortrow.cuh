// sortrow.cuh -- one row of C by one warp, by sorting its products.
//
// Rows whose products seldom share a column (output count close to the
// product count, as in products of random sparse matrices) gain little from
// a hash table: every product still claims a slot, and the table must be
// sorted afterwards.  Here the warp lays the row's products (column, value)
// out in shared memory in product order, sorts packed keys
// (column - kmin) << PB | product index in registers with Batcher's bitonic
// network (32*K keys, K per lane), and folds runs of equal columns with a
// segmented scan over the sorted order: Algorithm 1's row-wise accumulation
// done as expand, sort, compress.  The row leaves in ascending column order,
// its values summed (or minimised, or-ed) with the semiring's add.  A row
// whose column span does not fit the packed key sorts 64-bit keys
// column << 32 | product index instead (WIDE; the host keeps rows of more
// than 256 products out of the sort tiers when the matrix is that wide, so
// the larger tiers need not hold 64-bit keys in registers).
#pragma once
#include "common.cuh"

namespace hs {

// padded shared-memory index: one spare word per 32, so that a lane reading
// its K consecutive elements and 32 lanes reading consecutive elements both
// hit 32 distinct banks
__device__ __forceinline__ int sr_pad(int e) { return e + (e >> 5); }
__host__ __device__ constexpr int sr_pad_len(int n) { return n + (n >> 5); }

template <int N> struct ILog2 {
  static constexpr int v = 1 + ILog2<N / 2>::v;
};
template <> struct ILog2<1> {
  static constexpr int v = 0;
};

// the semiring's identity, or nothing for structure-only products
template <class SR> __device__ __forceinline__ typename SR::val_t sr_identity() {
  if constexpr (SR::has_val) return SR::identity();
  else return typename SR::val_t{};
}

template <typename T> __device__ __forceinline__ T shfl_up_val(T x, int d) { return __shfl_up_sync(FULL, x, d); }
template <> __device__ __forceinline__ NoVal shfl_up_val<NoVal>(NoVal x, int) { return x; }
template <typename T> __device__ __forceinline__ T shfl_down_val(T x, int d) { return __shfl_down_sync(FULL, x, d); }
template <> __device__ __forceinline__ NoVal shfl_down_val<NoVal>(NoVal x, int) { return x; }

// compare-exchange: a takes the smaller key, b the larger
template <typename KT> __device__ __forceinline__ void ce_up(KT &a, KT &b) {
  const KT lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}

// bitonic stages of sizes 2 .. K/2 inside each lane (directions fixed by i)
template <int K, typename KT> __device__ __forceinline__ void bitonic_in_lane(KT (&key)[K]) {
#pragma unroll
  for (int size = 2; size < K; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
      for (int i = 0; i < K; ++i)
        if ((i & stride) == 0) {
          if ((i & size) == 0) ce_up(key[i], key[i | stride]);
          else ce_up(key[i | stride], key[i]);
        }
}

// the in-lane strides K/2 .. 1 of an ascending bitonic merge
template <int K, typename KT> __device__ __forceinline__ void merge_in_lane(KT (&key)[K]) {
#pragma unroll
  for (int stride = K >> 1; stride > 0; stride >>= 1)
#pragma unroll
    for (int i = 0; i < K; ++i)
      if ((i & stride) == 0) ce_up(key[i], key[i | stride]);
}

// Ascending bitonic sort of the warp's 32*K keys, element e = lane*K + i held
// in key[i] of lane `lane` (blocked layout).  Merges of blocks of K or more
// elements run as a loop over the block size: a block that the network
// sorts descending holds its keys complemented for that merge, so every
// comparator takes the smaller key to the lower element; comparator pairs
// closer than K elements sit in one lane's registers, the others are one
// shuffle apart.  The loop keeps the code small (a fully unrolled network of
// 1024 keys would not fit the instruction cache).
template <int K, typename KT> __device__ __forceinline__ void warp_bitonic(KT (&key)[K]) {
  constexpr int N = 32 * K;
  const int lane = lane_id();
  bitonic_in_lane<K>(key);
#pragma unroll 1
  for (int size = K; size <= N; size <<= 1) {
    const KT flip = ((lane * K) & size) ? ~KT(0) : KT(0);
#pragma unroll
    for (int i = 0; i < K; ++i) key[i] ^= flip;
#pragma unroll 1
    for (int stride = size >> 1; stride >= K; stride >>= 1) {
      const int lm = stride / K;
      const bool lower = (lane & lm) == 0;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const KT o = __shfl_xor_sync(FULL, key[i], lm);
        const KT x = key[i];
        key[i] = (lower == (o < x)) ? o : x;
      }
    }
    merge_in_lane<K>(key);
#pragma unroll
    for (int i = 0; i < K; ++i) key[i] ^= flip;
  }
}

// The products of A entries [q0, q1) by one warp, in product order, to
// shared memory (columns at s_col[sr_pad(p)], values at s_val[p], at most
// nmax of them); returns their number (warp-uniform) and the least and
// greatest column in *kmn, *kmx.  Shared by every register width, so a kernel
// that sorts rows of several widths holds one copy of the expansion.
template <class SR>
__device__ __forceinline__ int sort_expand(const DevCsr &A, const DevCsr &B, int64_t q0, int64_t q1, int nmax,
                                           int *s_col, typename SR::val_t *s_val, int *kmn_out, int *kmx_out) {
  using T = typename SR::val_t;
  const int lane = lane_id();
  int base = 0, kmn = 0x7fffffff, kmx = -1;
  for (int64_t qb = q0; qb < q1; qb += 32) {
    const int64_t q = qb + lane;
    int64_t s = 0, e = 0;
    T av{};
    if (q < q1) {
      entry_segment(A, B, q, false, 0, 0, s, e);
      if constexpr (SR::needs_a) av = load_val<T>(A.v, q);
    }
    auto put = [&](int col, T v, int p) {
      const int at = base + p;
      if (HS_G(A.dbg, at >= 0 && at < nmax, 90, at)) {
        s_col[sr_pad(at)] = col;
        if constexpr (SR::has_val) s_val[at] = v;
      }
      kmn = min(kmn, col);
      kmx = max(kmx, col);
    };
    base += warp_expand<SR>(B, s, (int)(e - s), av, put);
  }
  __syncwarp();
  *kmn_out = warp_min(kmn);
  *kmx_out = warp_max(kmx);
  return base;
}

// Sort and fold a row whose F products (F <= 32*K) sort_expand laid out,
// writing its c outputs at out_j / out_v.  An output count other than c
// sets *err (the structure disagrees with the symbolic pass).
template <class SR, int K, bool WIDE>
__device__ __forceinline__ void sort_finish(int F, int c, int kmn, int kmx, int *s_col,
                                            const typename SR::val_t *s_val, int32_t *out_j,
                                            typename SR::val_t *out_v, int *err, long long *dbg) {
  using T = typename SR::val_t;
  constexpr int N = 32 * K;
  constexpr int PB = ILog2<N>::v;
  const int lane = lane_id();
  if (F <= 0) return;
  const unsigned span = (unsigned)kmx - (unsigned)kmn;
  if (span < (1u << (32 - PB)) - 1u) {
    // 2. packed keys, sorted
    uint32_t key[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int e = lane * K + i;
      key[i] = e < F ? (((uint32_t)(s_col[sr_pad(e)] - kmn)) << PB) | (uint32_t)e : 0xffffffffu;
    }
    warp_bitonic<K>(key);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < K; ++i) s_col[sr_pad(lane * K + i)] = (int)key[i];
    __syncwarp();
    // 3. runs of equal columns folded in sorted order, 32 elements a round
    // (lane l takes element 32*i + l): a run's sum is complete at its last
    // element, which writes it at the run's rank among the row's columns
    const unsigned le = 0xffffffffu >> (31 - lane);  // lanes <= this one
    int outb = 0;
    T carry = sr_identity<SR>();
    for (int i = 0; i * 32 < F; ++i) {
      const int e = i * 32 + lane;
      const bool valid = e < F;
      const uint32_t kk = valid ? (uint32_t)s_col[sr_pad(e)] : 0xffffffffu;
      const uint32_t kp = (valid && e > 0) ? (uint32_t)s_col[sr_pad(e - 1)] : 0xffffffffu;
      const uint32_t kn = (e + 1 < F) ? (uint32_t)s_col[sr_pad(e + 1)] : 0xffffffffu;
      const bool head = valid && (e == 0 || (kk >> PB) != (kp >> PB));
      const bool tail = valid && (e + 1 >= F || (kn >> PB) != (kk >> PB));
      const unsigned hm = __ballot_sync(FULL, head);
      const int pos = outb + __popc(hm & le) - 1;
      T v{};
      if constexpr (SR::has_val) {
        v = valid ? s_val[kk & (N - 1)] : SR::identity();
        bool fl = head;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const T y = shfl_up_val<T>(v, d);
          const bool g = __shfl_up_sync(FULL, (int)fl, d) != 0;
          if (lane >= d) {
            if (!fl) v = SR::add(y, v);
            fl = fl || g;
          }
        }
        if (!fl && valid) v = SR::add(carry, v);  // continues the previous round's last run
        carry = shfl_val<T>(v, 31);
      }
      if (tail && HS_G(dbg, pos >= 0 && pos < c, 91, pos)) {
        __stcs(out_j + pos, (int)(kk >> PB) + kmn);
        if constexpr (SR::has_val) __stcs(out_v + pos, v);
      }
      outb += __popc(hm);
    }
    if (outb != c && lane == 0) atomicExch(err, 13);
    return;
  }
  if constexpr (!WIDE) {
    if (lane == 0) atomicExch(err, 14);  // a span the host should have kept out of this tier
    return;
  }
  // wide rows: 64-bit keys column << 32 | product index, sorted, then folded
  // in the blocked layout (lane l holds sorted elements l*K .. l*K+K-1)
  unsigned long long key[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = lane * K + i;
    key[i] = e < F ? (((unsigned long long)(unsigned)s_col[sr_pad(e)]) << 32) | (unsigned)e : ~0ull;
  }
  warp_bitonic<K>(key);
  const unsigned long long before = __shfl_up_sync(FULL, key[K - 1], 1);  // element lane*K - 1
  int nh = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const bool valid = key[i] != ~0ull;
    const unsigned long long pk = i ? key[i - 1] : before;
    nh += (valid && ((lane == 0 && i == 0) || (pk >> 32) != (key[i] >> 32))) ? 1 : 0;
  }
  const int hincl = warp_incl_scan(nh);
  const int total = __shfl_sync(FULL, hincl, 31);
  int outi = hincl - nh - 1;  // index of the run being summed
  T acc = sr_identity<SR>();
  T pre = acc;         // elements before this lane's first head (a run begun in an earlier lane)
  bool seen = false;   // a head in this lane
  int curcol = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const bool valid = key[i] != ~0ull;
    if (!valid) continue;
    const unsigned long long pk = i ? key[i - 1] : before;
    const bool head = (lane == 0 && i == 0) || (pk >> 32) != (key[i] >> 32);
    T v{};
    if constexpr (SR::has_val) v = s_val[(unsigned)(key[i] & 0xffffffffull)];
    if (head) {
      if (seen && HS_G(dbg, outi >= 0 && outi < c, 92, outi)) {  // the previous run of this lane is complete
        __stcs(out_j + outi, curcol);
        if constexpr (SR::has_val) __stcs(out_v + outi, acc);
      }
      ++outi;
      seen = true;
      curcol = (int)(key[i] >> 32);
      acc = v;
    } else if (seen) {
      if constexpr (SR::has_val) acc = SR::add(acc, v);
    } else {
      if constexpr (SR::has_val) pre = SR::add(pre, v);
    }
  }
  // the lane's last run continues into the next lanes up to the first lane
  // with a head of its own
  bool open = seen;
  for (int d = 1; d < 32; ++d) {
    const T pd = shfl_down_val<T>(pre, d);
    const bool hd = __shfl_down_sync(FULL, (int)seen, d) != 0;
    if (open && lane + d < 32) {
      if constexpr (SR::has_val) acc = SR::add(acc, pd);
      if (hd) open = false;
    }
  }
  if (seen && HS_G(dbg, outi >= 0 && outi < c, 93, outi)) {
    __stcs(out_j + outi, curcol);
    if constexpr (SR::has_val) __stcs(out_v + outi, acc);
  }
  if (total != c && lane == 0) atomicExch(err, 13);
}

// Row r of C (A entries [q0, q1), F products, c outputs) by one warp, for
// F <= 32*K.  s_col holds sr_pad_len(32*K) ints, s_val 32*K values.  A
// product count other than F sets *err.
template <class SR, int K, bool WIDE>
__device__ __forceinline__ void sort_row(const DevCsr &A, const DevCsr &B, int64_t q0, int64_t q1, int F, int c,
                                         int *s_col, typename SR::val_t *s_val, int32_t *out_j,
                                         typename SR::val_t *out_v, int *err) {
  int kmn = 0, kmx = 0;
  const int got = sort_expand<SR>(A, B, q0, q1, 32 * K, s_col, s_val, &kmn, &kmx);
  if (got != F || F < 0 || F > 32 * K) {
    if (lane_id() == 0) atomicExch(err, 12);
    return;
  }
  sort_finish<SR, K, WIDE>(F, c, kmn, kmx, s_col, s_val, out_j, out_v, err, A.dbg);
}

}  // namespace hs
