// common.cuh -- device building blocks shared by the SpGEMM kernels.
//
// Contents
//   * semiring traits (Section 1: SpGEMM over a semiring; Section 3.1 selector
//     products), each a mul and an add that may run as a shared-memory atomic;
//   * warp/CTA "groups" so one routine serves a warp-per-row and a CTA-per-row
//     kernel;
//   * the product iterator: the row-wise form of Algorithm 1, C(i,:) +=
//     A(i,k) * B(k,:), with products spread one per lane (a warp-level
//     load-balanced expansion, so short and long rows of B keep every lane busy);
//   * shared-memory hash tables (symbolic: keys; numeric: keys + values);
//   * sorted emission: compaction of a table, a monotone bucket sort in shared
//     memory and coalesced stores of the finished row.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace hs {

// Checked accesses: indices that come from data (row ids read from bin
// lists, column ids, offsets, hash/bucket positions, output ranks) are tested
// before the load or store they address.  A failed check records (code,
// index) in a device word pair that the host reads, and the access is
// skipped, so corrupt or inconsistent input can never turn into an
// out-of-range access on the GPU.
__device__ __forceinline__ bool hs_guard_fail(long long *dbg, int code, long long idx) {
  if (dbg && atomicCAS(reinterpret_cast<unsigned long long *>(dbg), 0ull, (unsigned long long)code) == 0ull)
    dbg[1] = idx;
  return false;
}
#define HS_G(dbg, cond, code, idx) ((cond) ? true : ::hs::hs_guard_fail((dbg), (code), (long long)(idx)))

constexpr unsigned FULL = 0xffffffffu;
constexpr int EMPTY = -1;

// ----------------------------------------------------------------- semirings
enum SrKind { PLUS_TIMES = 0, OR_AND = 1, MIN_PLUS = 2, SELECT2ND = 3, SELECT1ST = 4 };

__device__ __forceinline__ void atomic_min_f32(float *p, float v) {
  unsigned *ip = reinterpret_cast<unsigned *>(p);
  unsigned old = *reinterpret_cast<volatile unsigned *>(ip);
  while (__uint_as_float(old) > v) {
    unsigned prev = atomicCAS(ip, old, __float_as_uint(v));
    if (prev == old) break;
    old = prev;
  }
}

// A semiring over value type T.  mul() is applied to one stored pair,
// add_atomic() folds a product into an accumulator slot that was initialised
// to identity() (the identity is only ever a slot's starting content: every
// slot that is emitted received at least one product, and identity (+) x == x
// exactly for each semiring below).
template <int KIND, typename T> struct Semiring;

template <typename T> struct Semiring<PLUS_TIMES, T> {
  using val_t = T;
  static constexpr bool has_val = true, needs_a = true, needs_b = true;
  __device__ static T identity() { return T(0); }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T add(T x, T y) { return x + y; }
  __device__ static void add_atomic(T *p, T v) { atomicAdd(p, v); }
};
template <> struct Semiring<PLUS_TIMES, int64_t> {
  using val_t = int64_t;
  static constexpr bool has_val = true, needs_a = true, needs_b = true;
  __device__ static int64_t identity() { return 0; }
  // two's complement products and sums, wrapping modulo 2^64
  __device__ static int64_t mul(int64_t a, int64_t b) {
    return (int64_t)((unsigned long long)a * (unsigned long long)b);
  }
  __device__ static int64_t add(int64_t x, int64_t y) {
    return (int64_t)((unsigned long long)x + (unsigned long long)y);
  }
  __device__ static void add_atomic(int64_t *p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
  }
};
template <> struct Semiring<MIN_PLUS, float> {
  using val_t = float;
  static constexpr bool has_val = true, needs_a = true, needs_b = true;
  __device__ static float identity() { return __int_as_float(0x7f800000); }  // +inf
  __device__ static float mul(float a, float b) { return __fadd_rn(a, b); }
  __device__ static float add(float x, float y) { return y < x ? y : x; }
  __device__ static void add_atomic(float *p, float v) { atomic_min_f32(p, v); }
};
template <> struct Semiring<MIN_PLUS, int32_t> {
  using val_t = int32_t;
  static constexpr bool has_val = true, needs_a = true, needs_b = true;
  __device__ static int32_t identity() { return 0x7fffffff; }
  __device__ static int32_t mul(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
  __device__ static int32_t add(int32_t x, int32_t y) { return y < x ? y : x; }
  __device__ static void add_atomic(int32_t *p, int32_t v) { atomicMin(p, v); }
};
// structure only: no values at all
struct NoVal {};
template <> struct Semiring<OR_AND, NoVal> {
  using val_t = NoVal;
  static constexpr bool has_val = false, needs_a = false, needs_b = false;
};
// selectors: the value of the non-selector operand is copied; T is a bit
// container of the value's width (uint32_t or unsigned long long)
template <typename T> struct Semiring<SELECT2ND, T> {
  using val_t = T;
  static constexpr bool has_val = true, needs_a = false, needs_b = true;
  __device__ static T identity() { return T(0); }
  __device__ static T mul(T, T b) { return b; }
  __device__ static T add(T x, T) { return x; }
  __device__ static void add_atomic(T *p, T v) { *reinterpret_cast<volatile T *>(p) = v; }
};
template <typename T> struct Semiring<SELECT1ST, T> {
  using val_t = T;
  static constexpr bool has_val = true, needs_a = true, needs_b = false;
  __device__ static T identity() { return T(0); }
  __device__ static T mul(T a, T) { return a; }
  __device__ static T add(T x, T) { return x; }
  __device__ static void add_atomic(T *p, T v) { *reinterpret_cast<volatile T *>(p) = v; }
};

// ------------------------------------------------------------------ groups
struct WarpGroup {
  __device__ __forceinline__ static int size() { return 32; }
  __device__ __forceinline__ static int rank() { return threadIdx.x & 31; }
  __device__ __forceinline__ static int nwarps() { return 1; }
  __device__ __forceinline__ static int warp() { return 0; }
  __device__ __forceinline__ static void sync() { __syncwarp(); }
};
struct CtaGroup {
  __device__ __forceinline__ static int size() { return blockDim.x; }
  __device__ __forceinline__ static int rank() { return threadIdx.x; }
  __device__ __forceinline__ static int nwarps() { return blockDim.x >> 5; }
  __device__ __forceinline__ static int warp() { return threadIdx.x >> 5; }
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T> __device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T u = __shfl_up_sync(FULL, v, d);
    if (lane_id() >= d) v += u;
  }
  return v;
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}
__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = min(v, __shfl_xor_sync(FULL, v, d));
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = max(v, __shfl_xor_sync(FULL, v, d));
  return v;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = max(v, __shfl_xor_sync(FULL, v, d));
  return v;
}

// Exclusive scan of a[0..n) in shared memory by a whole group; returns the
// total.  tmp needs 32 ints (CTA groups only); the closing barrier also ends
// every read of tmp.
template <class G> __device__ int group_excl_scan(int *a, int n, int *tmp) {
  const int gs = G::size(), r = G::rank();
  const int per = (n + gs - 1) / gs;
  const int b = min(n, r * per), e = min(n, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += a[i];
  int incl = warp_incl_scan(s);
  int total;
  if (G::nwarps() == 1) {
    total = __shfl_sync(FULL, incl, 31);
  } else {
    // the warp totals are published once and every warp scans them itself
    // (nwarps <= 32), so one barrier separates the two levels
    if (lane_id() == 31) tmp[G::warp()] = incl;
    G::sync();
    const int w = lane_id() < G::nwarps() ? tmp[lane_id()] : 0;
    const int wi = warp_incl_scan(w);
    total = __shfl_sync(FULL, wi, 31);
    incl += __shfl_sync(FULL, wi - w, G::warp());
  }
  int run = incl - s;
  for (int i = b; i < e; ++i) {
    int x = a[i];
    a[i] = run;
    run += x;
  }
  G::sync();
  return total;
}

// ---------------------------------------------------------------- operands
struct DevCsr {
  const int64_t *p;  // row offsets (indexed by row slot)
  const int32_t *j;  // column ids
  const void *v;     // values (may be null)
  int64_t rows;      // row slots
  int64_t nnz;       // entries
  long long *dbg;    // guard record (guarded builds)
};

// lower_bound of x in j[s..e) (first position with j >= x)
__device__ __forceinline__ int64_t lower_bound_col(const int32_t *j, int64_t s, int64_t e, int x) {
  while (s < e) {
    int64_t mid = s + ((e - s) >> 1);
    if (__ldg(j + mid) < x) s = mid + 1;
    else e = mid;
  }
  return s;
}

template <typename T> __device__ __forceinline__ T load_val(const void *v, int64_t q) {
  return __ldg(reinterpret_cast<const T *>(v) + q);
}
template <> __device__ __forceinline__ NoVal load_val<NoVal>(const void *, int64_t) { return NoVal{}; }

// A visitor may split its work in two: prep(col) does the reads (and any
// atomic whose result it needs) and returns a state; commit(state, value)
// does the final write.  The long-segment loop then preps all of a step's
// products before committing any, so their shared-memory round trips overlap
// instead of queueing behind each other's atomics.
template <class V, class = void> struct two_stage : std::false_type {};
template <class V> struct two_stage<V, std::void_t<decltype(V::kTwoStage)>> : std::bool_constant<V::kTwoStage> {};

template <typename T> __device__ __forceinline__ T shfl_val(T x, int src) { return __shfl_sync(FULL, x, src); }
template <> __device__ __forceinline__ NoVal shfl_val<NoVal>(NoVal x, int) { return x; }

// Visit the products of up to 32 B-row segments (one per lane: start s,
// length len, left value a).  Segments of at least 32 products are walked by
// the whole warp, one segment at a time, with consecutive lanes on
// consecutive entries of B (coalesced, no search).  The remaining short
// segments are dealt one product per lane: lane l takes product base+l of
// their concatenation and finds its segment by a binary search over the
// inclusive length scan (shuffles only).  SB such rounds are taken at once,
// their B loads all issued before the first visit, so a lane has SB
// independent reads in flight instead of one round trip per round.
// visit(col, prod, p) runs on every lane that holds a product, p being the
// product's index in the order of the segments (as if they were walked lane
// by lane).  Returns the number of products.  All 32 lanes must call this
// together.
template <class SR, int U = 2, int SB = 4, class Visit>
__device__ __forceinline__ int warp_expand(const DevCsr &B, int64_t s, int len, typename SR::val_t a,
                                            Visit &visit) {
  using T = typename SR::val_t;
  using VisitT = std::decay_t<Visit>;
  const int lane = lane_id();
  const int incl = warp_incl_scan(len);
  const int total = __shfl_sync(FULL, incl, 31);
  const int ex_full = incl - len;
  // long segments: the whole warp on one segment, U entries per lane per
  // step (all loads of a step issued before the first visit)
  unsigned longm = __ballot_sync(FULL, len >= 32);
  while (longm) {
    const int l = __ffs(longm) - 1;
    longm &= longm - 1;
    const int64_t sl = __shfl_sync(FULL, s, l);
    const int ll = __shfl_sync(FULL, len, l);
    const int el = __shfl_sync(FULL, ex_full, l);
    const T al = shfl_val<T>(a, l);
    if (!HS_G(B.dbg, sl >= 0 && sl + ll <= B.nnz, 4, sl)) continue;
    const int32_t *bj = B.j + sl;
    const T *bv = reinterpret_cast<const T *>(B.v) + sl;
    for (int off = lane; off < ll; off += 32 * U) {
      int c[U];
      T b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool ok = off + 32 * u < ll;
        c[u] = ok ? __ldg(bj + off + 32 * u) : 0;
        b[u] = T{};
        if constexpr (SR::needs_b)
          if (ok) b[u] = __ldg(bv + off + 32 * u);
      }
      if constexpr (two_stage<VisitT>::value) {
        typename VisitT::State st[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (off + 32 * u < ll) st[u] = visit.prep(c[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (off + 32 * u >= ll) break;
          if constexpr (SR::has_val) visit.commit(st[u], SR::mul(al, b[u]));
          else visit.commit(st[u], NoVal{});
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (off + 32 * u >= ll) break;
          if constexpr (SR::has_val) visit(c[u], SR::mul(al, b[u]), el + off + 32 * u);
          else visit(c[u], NoVal{}, el + off + 32 * u);
        }
      }
    }
  }
  // short segments: one product per lane, SB rounds of 32 at a time
  const int slen = len < 32 ? len : 0;
  const int sincl = warp_incl_scan(slen);
  const int stotal = __shfl_sync(FULL, sincl, 31);
  const int sexcl = sincl - slen;
  for (int base = 0; base < stotal; base += 32 * SB) {
    int col[SB], pidx[SB];
    T pv[SB];
    bool ok[SB];
#pragma unroll
    for (int u = 0; u < SB; ++u) {
      ok[u] = false;
      col[u] = 0;
      pidx[u] = 0;
      pv[u] = T{};
      if (base + 32 * u < stotal) {  // warp-uniform: the shuffles below see every lane
        const int p = base + 32 * u + lane;
        int src = 0;  // number of lanes whose inclusive end is <= p
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int v = __shfl_sync(FULL, sincl, src + step - 1);
          if (v <= p) src += step;
        }
        const int64_t ss = __shfl_sync(FULL, s, src);
        const int sex = __shfl_sync(FULL, sexcl, src);
        const int fex = __shfl_sync(FULL, ex_full, src);
        const T aa = shfl_val<T>(a, src);
        if (p < stotal) {
          const int64_t pos = ss + (p - sex);
          if (HS_G(B.dbg, pos >= 0 && pos < B.nnz, 4, pos)) {
            ok[u] = true;
            col[u] = __ldg(B.j + pos);
            pidx[u] = fex + (p - sex);
            if constexpr (SR::has_val) {
              T b{};
              if constexpr (SR::needs_b) b = load_val<T>(B.v, pos);
              pv[u] = SR::mul(aa, b);
            }
          }
        }
      }
    }
    if constexpr (two_stage<VisitT>::value) {
      typename VisitT::State st[SB];
#pragma unroll
      for (int u = 0; u < SB; ++u)
        if (ok[u]) st[u] = visit.prep(col[u]);
#pragma unroll
      for (int u = 0; u < SB; ++u)
        if (ok[u]) visit.commit(st[u], pv[u]);
    } else {
#pragma unroll
      for (int u = 0; u < SB; ++u)
        if (ok[u]) visit(col[u], pv[u], pidx[u]);
    }
  }
  return total;
}

// B-row segment of A entry q: [s, e) of B(k,:), restricted to columns
// [lo, hi) when restrict_cols.
__device__ __forceinline__ void entry_segment(const DevCsr &A, const DevCsr &B, int64_t q, bool restrict_cols,
                                              int lo, int hi, int64_t &s, int64_t &e) {
  s = e = 0;
  if (!HS_G(A.dbg, q >= 0 && q < A.nnz, 1, q)) return;
  const int k = __ldg(A.j + q);
  if (!HS_G(A.dbg, k >= 0 && k < B.rows, 2, k)) return;
  s = __ldg(B.p + k);
  e = __ldg(B.p + k + 1);
  if (!HS_G(A.dbg, s >= 0 && s <= e && e <= B.nnz, 3, e)) {
    s = e = 0;
    return;
  }
  if (restrict_cols && s < e) {
    s = lower_bound_col(B.j, s, e, lo);
    e = lower_bound_col(B.j, s, e, hi);
  }
}

// Every product of one row, by one warp: A entries [q0, q1) in chunks of 32.
template <class SR, class Visit>
__device__ __forceinline__ void warp_products(const DevCsr &A, const DevCsr &B, int64_t q0, int64_t q1,
                                              Visit &&visit) {
  using T = typename SR::val_t;
  for (int64_t qb = q0; qb < q1; qb += 32) {
    const int64_t q = qb + lane_id();
    int64_t s = 0, e = 0;
    T a{};
    if (q < q1) {
      entry_segment(A, B, q, false, 0, 0, s, e);
      if constexpr (SR::needs_a) a = load_val<T>(A.v, q);
    }
    warp_expand<SR>(B, s, (int)(e - s), a, visit);
  }
}

// Ask for [p, p + bytes) to be brought into L2 ahead of its reads (bulk
// prefetch, no completion to wait for).  The range is narrowed to 16-byte
// boundaries, so it never leaves the buffer, and issued in pieces of at most
// 64 KB.
__device__ __forceinline__ void prefetch_l2(const void *p, int64_t bytes) {
  if (bytes <= 0) return;
  uint64_t a = (uint64_t)__cvta_generic_to_global(p);
  const uint64_t e = (a + (uint64_t)bytes) & ~(uint64_t)15;
  a = (a + 15) & ~(uint64_t)15;
  while (a < e) {
    const uint64_t len = e - a < 65536 ? e - a : 65536;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)len) : "memory");
    a += len;
  }
}

// Asynchronous copy (cp.async, 16-byte pieces, completed by cp.async.wait_all
// and a barrier) of the global bytes [src, src + bytes) into shared memory at
// dst + off, off = src mod 16: the copy runs from the 16-byte boundary at or
// below src to the one at or above src + bytes, so dst needs bytes + 32 bytes
// of room and the source buffer 16 bytes of slack past its end.  Every
// thread of the group calls it with its rank.
__device__ __forceinline__ int async_copy16(void *dst, const void *src, int64_t bytes, int rank, int nthreads) {
  const uint64_t s = (uint64_t)src;
  const uint64_t s0 = s & ~(uint64_t)15;
  const int64_t chunks = (int64_t)((s + (uint64_t)bytes + 15 - s0) >> 4);
  const unsigned d0 = (unsigned)__cvta_generic_to_shared(dst);
  for (int64_t c = rank; c < chunks; c += nthreads)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + (unsigned)(c << 4)),
                 "l"(__cvta_generic_to_global((const void *)(s0 + (uint64_t)(c << 4))))
                 : "memory");
  return (int)(s - s0);
}
__device__ __forceinline__ void async_copy_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__host__ __device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Shared-memory arrays for cta_products (CH A entries per round).
template <typename T, int CH> struct CtaExpandSmem {
  int excl[CH + 1];
  int64_t sbeg[CH];
  T aval[CH];
};

// The products of n staged B-row segments (start sbeg[e], exclusive length
// prefix excl[e], excl[n] = total, left values aval[e]) spread evenly over
// the warps of the CTA: each warp takes one contiguous range of the products
// and deals it one product per lane (warp_expand).  Reads the staged arrays
// only; all threads of the CTA must call it together.
// Each segment may also be charged K units of fixed cost (its setup in the
// warp loop): warps then split the cost, not just the products, so a warp
// whose range holds many short segments gets fewer products.  excl may hold
// a running prefix that starts at ebase instead of 0 (a batch of a longer
// list).
template <class SR, int U = 2, int K = 0, class Visit>
__device__ __forceinline__ void cta_expand_staged(const DevCsr &B, const int64_t *sbeg, const int *excl,
                                                  const typename SR::val_t *aval, int n, int total,
                                                  Visit &visit, int ebase = 0) {
  using T = typename SR::val_t;
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // entry e occupies [X_e, X_e+1) with X_e = excl[e] + K*e: K units of its
  // fixed cost, then its products
  const int64_t tcost = (int64_t)total + (int64_t)K * n;
  const int64_t pb = tcost * warp / nw, pe = tcost * (warp + 1) / nw;
  if (pb >= pe) return;
  // last entry whose start is <= pb (entry 0 starts at 0, so l >= 1)
  int l = 0, h = n;
  while (l < h) {
    const int mid = (l + h) >> 1;
    if (excl[mid] - ebase + (int64_t)K * mid <= pb) l = mid + 1;
    else h = mid;
  }
  for (int eb = l - 1; eb < n; eb += 32) {
    const int e = eb + lane;
    int64_t s = 0;
    int len = 0;
    T a{};
    if (e < n) {
      const int64_t x0 = excl[e] - ebase + (int64_t)K * e + K, x1 = excl[e + 1] - ebase + (int64_t)K * (e + 1);
      const int64_t cb = max(x0, pb), ce = min(x1, pe);
      if (ce > cb) {
        len = (int)(ce - cb);
        s = sbeg[e] + (cb - x0);
        if constexpr (SR::needs_a) a = aval[e];
      }
    }
    warp_expand<SR, U>(B, s, len, a, visit);
    if (eb + 32 >= n || excl[eb + 32] - ebase + (int64_t)K * (eb + 32) >= pe) break;
  }
}

// First position in [s, e) whose column is >= x.  Long ranges start with one
// interpolation probe (column ids of a row are close to uniform after a
// random relabelling) and narrow the bracket around it; then, as for short
// ranges, probe lo, lo+1, lo+3, lo+7, ... (galloping) and finish with a
// binary search, so the cost stays logarithmic for any distribution.
__device__ __forceinline__ int64_t gallop_lower_bound(const int32_t *j, int64_t s, int64_t e, int x);
__device__ __forceinline__ int64_t interp_lower_bound(const int32_t *j, int64_t s, int64_t e, int x) {
  if (e - s > 64) {
    const int c0 = __ldg(j + s), c1 = __ldg(j + e - 1);
    if (c0 >= x) return s;
    if (c1 < x) return e;
    // c0 < x <= c1: the answer is in (s, e-1]
    int64_t g = s + 1 + (int64_t)(((double)(x - c0) / (double)(c1 - c0 + 1)) * (double)(e - 2 - s));
    if (g > e - 1) g = e - 1;
    if (g <= s) g = s + 1;
    if (__ldg(j + g) >= x) {
      // answer in (s, g]: gallop leftwards from g
      int64_t hi = g, step = 1, lo = g - 1;
      while (lo > s && __ldg(j + lo) >= x) {
        hi = lo;
        step <<= 1;
        lo = g - step;
        if (lo < s) lo = s;
      }
      // j[lo] < x (or lo == s), j[hi] >= x
      int64_t a = lo + 1, b = hi;
      while (a < b) {
        const int64_t mid = a + ((b - a) >> 1);
        if (__ldg(j + mid) < x) a = mid + 1;
        else b = mid;
      }
      return a;
    }
    return gallop_lower_bound(j, g + 1, e, x);
  }
  return gallop_lower_bound(j, s, e, x);
}

// First position in [s, e) whose column is >= x: probe s, s+1, s+3, s+7, ...
// (galloping) and finish with a binary search, so a short distance costs few
// loads whatever the row's length.
__device__ __forceinline__ int64_t gallop_lower_bound(const int32_t *j, int64_t s, int64_t e, int x) {
  if (s >= e || __ldg(j + s) >= x) return s;
  int64_t lo = s + 1, step = 1, hi = s + 1;
  while (hi < e && __ldg(j + hi) < x) {
    lo = hi + 1;
    step <<= 1;
    hi = s + step;
  }
  if (hi > e) hi = e;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(j + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Every product of one row (or of the part of it inside columns [lo, hi)),
// spread evenly over the warps of the CTA.  A entries are taken CH at a time;
// their B segments' lengths are scanned across the CTA, the products of the
// round are cut into one contiguous range per warp, and each warp deals its
// range one product per lane (warp_expand).  Per-row product counts must stay
// below 2^31.  All threads of the CTA must call this together.
template <class SR, int CH, int U = 2, class Visit>
__device__ __forceinline__ void cta_products(const DevCsr &A, const DevCsr &B, int64_t q0, int64_t q1, bool restrict_cols,
                             int lo, int hi, CtaExpandSmem<typename SR::val_t, CH> &sm, int *wtmp,
                             Visit &&visit) {
  using T = typename SR::val_t;
  const int tid = threadIdx.x;
  for (int64_t c0 = q0; c0 < q1; c0 += CH) {
    const int n = (int)min((int64_t)CH, q1 - c0);
    for (int e = tid; e < n; e += blockDim.x) {
      int64_t s = 0, en = 0;
      entry_segment(A, B, c0 + e, restrict_cols, lo, hi, s, en);
      if constexpr (SR::needs_a) sm.aval[e] = load_val<T>(A.v, c0 + e);
      sm.excl[e] = (int)(en - s);
      sm.sbeg[e] = s;
    }
    if (tid == 0) sm.excl[n] = 0;  // scanned with the entries, it becomes the round's total
    __syncthreads();
    // only the staged entries are scanned (a short row costs what it holds)
    const int total = group_excl_scan<CtaGroup>(sm.excl, n + 1, wtmp);
    cta_expand_staged<SR, U, 32>(B, sm.sbeg, sm.excl, sm.aval, n, total, visit);
    __syncthreads();
  }
}

// ------------------------------------------------------------ hash tables
__device__ __forceinline__ unsigned hash_slot(int key, unsigned mask) {
  return (unsigned)(key * 2654435761u) & mask;  // Knuth multiplicative hash
}

// Symbolic insert: returns 1 if the key was new.  The table holds at least
// twice the row's product count, so it cannot fill; the probe count is still
// bounded (a full table would return 0 after visiting every slot).
__device__ __forceinline__ int hash_insert_key(int *keys, unsigned mask, int key) {
  unsigned h = hash_slot(key, mask);
  for (unsigned probes = 0; probes <= mask; ++probes) {
    int k = reinterpret_cast<volatile int *>(keys)[h];
    if (k == key) return 0;
    if (k == EMPTY) {
      int old = atomicCAS(keys + h, EMPTY, key);
      if (old == EMPTY) return 1;
      if (old == key) return 0;
    }
    h = (h + 1) & mask;
  }
  return 0;
}

// Numeric insert: fold v into the slot of key.  The table is sized from the
// symbolic count (at least twice the row's distinct keys), so it cannot fill;
// should it ever, the probe gives up after visiting every slot and raises
// *err instead of spinning.
template <class SR, typename T>
__device__ __forceinline__ void hash_insert_val(int *keys, T *vals, unsigned mask, int key, T v, int *err) {
  unsigned h = hash_slot(key, mask);
  for (unsigned probes = 0;; ++probes) {
    if (probes > mask) {
      atomicExch(err, 7);
      return;
    }
    int k = reinterpret_cast<volatile int *>(keys)[h];
    if (k == key) break;
    if (k == EMPTY) {
      int old = atomicCAS(keys + h, EMPTY, key);
      if (old == EMPTY || old == key) break;
    }
    h = (h + 1) & mask;
  }
  if constexpr (SR::has_val) SR::add_atomic(vals + h, v);
}

// ----------------------------------------------------------- sorted emit
// Shared-memory layout used by group_sort_emit (all offsets in bytes):
//   ck[cap] int32 | cv[cap] T           (compacted entries, arbitrary order)
//   work: bcnt[nb] int32 | order[c] int32 | sk[c] int32 | sv[c] T
// `work` may alias the hash table (it is free once compacted).
//
// Steps: (1) every occupied slot of the table is appended to ck/cv, and the
// key range [kmin, kmax] is found; (2) keys are distributed over nb buckets
// by the monotone map b = (key-kmin)*nb/(kmax-kmin+1); a histogram and an
// exclusive scan give every bucket its start; (3) entry e's final position
// is its bucket's start plus the number of keys in the same bucket that are
// smaller (keys are distinct), so the row leaves in ascending column order;
// (4) the sorted row is written to global memory with coalesced stores.
struct EmitScratch {
  int kmin, kmax, count;
};

// number of buckets for c entries: the largest power of two <= c
__host__ __device__ __forceinline__ int emit_buckets(int c) {
  int nb = 1;
  while (nb * 2 <= c) nb <<= 1;
  return nb;
}
// bytes of the `work` region for c entries with values of `vbytes` bytes
__host__ __device__ __forceinline__ size_t emit_work_bytes(int c, int vbytes) {
  return ((((size_t)(emit_buckets(c) + 2 * c) * 4 + 7) & ~(size_t)7)) + (size_t)c * vbytes;
}

template <class G, typename T, bool HAS_VAL>
__device__ void group_sort_emit(const int *keys, const T *vals, int slots, int c, int *ck, T *cv,
                                void *work, int *wtmp, EmitScratch *es, int32_t *out_j, T *out_v,
                                int *err, int cap, long long *dbg, bool unsorted = false) {
  constexpr int EU = 4;  // entries per thread per step: their shared-memory chains overlap
  const int gs = G::size(), r = G::rank(), lane = lane_id();
  if (!HS_G(dbg, c >= 0 && c <= cap, 20, c)) {
    if (r == 0) atomicExch(err, 8);
    return;
  }
  if (r == 0) {
    es->kmin = 0x7fffffff;
    es->kmax = -1;
    es->count = 0;
  }
  G::sync();
  // (1) compaction: each warp counts its run of slots, reserves room once,
  // then copies the run's entries in order
  {
    const int nw = G::nwarps(), w = G::warp();
    const int per = ((slots + nw - 1) / nw + 31) & ~31;
    const int s0 = min(slots, w * per), s1 = min(slots, s0 + per);
    int n = 0;
    for (int sb = s0; sb < s1; sb += 32) n += __popc(__ballot_sync(FULL, sb + lane < s1 && keys[sb + lane] != EMPTY));
    int base = 0;
    if (lane == 0 && n) base = atomicAdd(&es->count, n);
    base = __shfl_sync(FULL, base, 0);
    int lmin = 0x7fffffff, lmax = -1;
    for (int sb = s0; sb < s1; sb += 32) {
      const int sl = sb + lane;
      const int k = sl < s1 ? keys[sl] : EMPTY;
      const bool occ = k != EMPTY;
      const unsigned m = __ballot_sync(FULL, occ);
      if (occ) {
        const int at = base + __popc(m & ((1u << lane) - 1));
        if (at < c) {
          ck[at] = k;
          if constexpr (HAS_VAL) cv[at] = vals[sl];
        }
        lmin = min(lmin, k);
        lmax = max(lmax, k);
      }
      base += __popc(m);
    }
    lmin = warp_min(lmin);
    lmax = warp_max(lmax);
    if (lane == 0) {
      atomicMin(&es->kmin, lmin);
      atomicMax(&es->kmax, lmax);
    }
  }
  G::sync();
  if (es->count != c) {  // structure disagrees with the symbolic count
    if (r == 0) atomicExch(err, 1);
    return;
  }
  if (c == 0) return;
  if (unsorted) {  // the caller takes the row in table order
    for (int e = r; e < c; e += gs) {
      __stcs(out_j + e, ck[e]);
      if constexpr (HAS_VAL) __stcs(out_v + e, cv[e]);
    }
    return;
  }
  // (2) buckets
  const int nb = emit_buckets(c);
  int *bcnt = reinterpret_cast<int *>(work);
  int *order = bcnt + nb;
  int *sk = order + c;
  T *sv = reinterpret_cast<T *>(reinterpret_cast<char *>(work) + (((size_t)(nb + 2 * c) * 4 + 7) & ~(size_t)7));
  const int kmin = es->kmin;
  const uint64_t range = (uint64_t)(es->kmax - kmin) + 1;
  // monotone bucket map b = floor((key-kmin) * scale / 2^32), scale = floor(nb*2^32/range) < 2^32*nb/range
  const uint64_t scale = (((uint64_t)nb) << 32) / range;
  auto bucket = [&](int key) { return (int)(((uint64_t)(unsigned)(key - kmin) * scale) >> 32); };
  for (int b = r; b < nb; b += gs) bcnt[b] = 0;
  G::sync();
  for (int e = r; e < c; e += gs) {
    const int b = bucket(ck[e]);
    if (HS_G(dbg, b >= 0 && b < nb, 21, b)) atomicAdd(bcnt + b, 1);
  }
  G::sync();
  group_excl_scan<G>(bcnt, nb, wtmp);
  // scatter entry ids into their buckets (arbitrary order inside a bucket);
  // bcnt[b] advances to the bucket's end, so the start is bcnt[b] - size
  for (int e0 = r; e0 < c; e0 += EU * gs) {
    int b[EU], at[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const int e = e0 + u * gs;
      b[u] = e < c ? bucket(ck[e]) : -1;
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      at[u] = -1;
      if (b[u] >= 0 && HS_G(dbg, b[u] < nb, 22, b[u])) at[u] = atomicAdd(bcnt + b[u], 1);
    }
#pragma unroll
    for (int u = 0; u < EU; ++u)
      if (at[u] >= 0 && HS_G(dbg, at[u] < c, 23, at[u])) order[at[u]] = e0 + u * gs;
  }
  G::sync();
  // (3) rank inside the bucket: bucket b spans [end(b-1), end(b))
  for (int e0 = r; e0 < c; e0 += EU * gs) {
    int key[EU], bs[EU], be[EU], rank[EU];
    T v[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const int e = e0 + u * gs;
      key[u] = e < c ? ck[e] : 0;
      if constexpr (HAS_VAL) v[u] = e < c ? cv[e] : T{};
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const int b = e0 + u * gs < c ? bucket(key[u]) : 0;
      bs[u] = b ? bcnt[b - 1] : 0;
      be[u] = e0 + u * gs < c ? bcnt[b] : 0;
      rank[u] = bs[u];
    }
#pragma unroll
    for (int u = 0; u < EU; ++u)
      for (int t = bs[u]; t < be[u]; ++t)
        if (HS_G(dbg, t >= 0 && t < c && order[t] >= 0 && order[t] < c, 24, t)) rank[u] += ck[order[t]] < key[u];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      if (e0 + u * gs >= c || !HS_G(dbg, rank[u] >= 0 && rank[u] < c, 25, rank[u])) continue;
      sk[rank[u]] = key[u];
      if constexpr (HAS_VAL) sv[rank[u]] = v[u];
    }
  }
  G::sync();
  // (4) coalesced stores, evict-first: C is not read again here, B is
  for (int e = r; e < c; e += gs) {
    __stcs(out_j + e, sk[e]);
    if constexpr (HAS_VAL) __stcs(out_v + e, sv[e]);
  }
  G::sync();
}

}  // namespace hs
