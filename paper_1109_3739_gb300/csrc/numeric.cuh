// numeric.cuh -- values of C = A*B, rows emitted in ascending column order.
//
// Each bin runs the row-wise form of Algorithm 1 (C(i,:) += A(i,k)*B(k,:))
// into the accumulator that fits its rows:
//   tiny  (f <= 32)        one warp; products sit one per lane; lanes with
//                          equal columns (__match_any_sync) are folded by the
//                          lowest lane in product order, and each distinct
//                          column's rank among the row's columns is its output
//                          position;
//   warp  (f <= 512)       one warp; private shared hash table of <= 1024
//                          slots, then sorted emission;
//   mid   (c <= 2048)      one CTA of 256; shared hash table of 2c slots;
//   large (c <= CAP)       one CTA of 1024; shared hash table of 2c slots;
//   heavy (c > CAP)        one CTA of 512 per row (two per SM), rows handed
//                          out largest first; column parts accumulated with
//                          a bitmap + rank-indexed value array (see
//                          k_num_heavy).
// The shared hash table is the sparse accumulator of Figure 1 with the dense
// value array replaced by open addressing (keys + values), so its size
// follows the row's output, not the matrix dimension (Section 2.1's argument
// against dimension-dependent work).
#pragma once
#include "common.cuh"
#include "internal.h"
#include "sortrow.cuh"

namespace hs {

__device__ __forceinline__ DevCsr ndev_a(const RowSet &A) { return DevCsr{A.p, A.j, A.v, A.nslots, A.nnz, A.dbg}; }
__device__ __forceinline__ DevCsr ndev_b(const RightOp &B) { return DevCsr{B.p, B.j, B.v, B.m, B.nnz, B.dbg}; }
__device__ __forceinline__ int64_t nout_row(const RowSet &A, int r) {
  return A.ids ? (int64_t)A.ids[r] : (int64_t)r;
}

template <typename T> constexpr int vbytes() { return sizeof(T); }
template <> constexpr int vbytes<NoVal>() { return 0; }

template <typename T> constexpr int cap_large() { return vbytes<T>() == 8 ? 4096 : 8192; }

// the structure-only view of a semiring (same iteration, no values)
template <class SR> using StructOf = Semiring<OR_AND, NoVal>;

// --------------------------------------------------------------- tiny
constexpr int NTINY_WPB = 8;
template <class SR>
__global__ void __launch_bounds__(NTINY_WPB * 32, 4) k_num_tiny(NumArgs a) {
  using T = typename SR::val_t;
  __shared__ int scol[NTINY_WPB][32];
  __shared__ T sval[NTINY_WPB][32];
  const int w = threadIdx.x >> 5, lane = lane_id();
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  for (int idx = blockIdx.x * NTINY_WPB + w; idx < a.count; idx += gridDim.x * NTINY_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int64_t q0 = A.p[r], q1 = A.p[r + 1];
    int nprod = 0;
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane;
      int64_t s = 0, e = 0;
      T av{};
      if (q < q1) {
        entry_segment(A, B, q, false, 0, 0, s, e);
        if constexpr (SR::needs_a) av = load_val<T>(A.v, q);
      }
      auto put = [&](int col, T v, int p) {
        if (HS_G(a.A.dbg, nprod + p < 32, 40, nprod + p)) {
          scol[w][nprod + p] = col;
          if constexpr (SR::has_val) sval[w][nprod + p] = v;
        }
      };
      nprod += warp_expand<SR>(B, s, (int)(e - s), av, put);
    }
    __syncwarp();
    const bool have = lane < nprod;
    const int col = have ? scol[w][lane] : 0;
    const unsigned act = __ballot_sync(FULL, have);
    unsigned grp = 0;
    if (have) grp = __match_any_sync(act, col);
    const bool lead = have && lane == __ffs(grp) - 1;
    T acc{};
    if (lead) {
      if constexpr (SR::has_val) {
        acc = sval[w][lane];
        for (unsigned m = grp & (grp - 1); m; m &= m - 1) acc = SR::add(acc, sval[w][__ffs(m) - 1]);
      }
    }
    const unsigned leaders = __ballot_sync(FULL, lead);
    const int64_t o = nout_row(a.A, r);
    const int64_t base = a.Cp[o];
    if (lead) {
      int rank = 0;
      for (unsigned m = leaders; m; m &= m - 1) rank += scol[w][__ffs(m) - 1] < col;
      if (HS_G(a.A.dbg, base + rank < a.Cp[o + 1], 41, base + rank)) {
        a.Cj[base + rank] = col;
        if constexpr (SR::has_val) Cv[base + rank] = acc;
      }
    }
    if (lane == 0 && (int64_t)__popc(leaders) != a.Cp[o + 1] - base) atomicExch(a.err, 3);
    __syncwarp();
  }
}

// --------------------------------------------------------------- warp
constexpr int NWARP_WPB = 4;

// a warp's table (SLOTS), its compacted entries (at most CAP) and sort scratch
template <typename T, int SLOTS, int CAP> struct WarpNumSmem {
  static constexpr size_t table_bytes = (size_t)SLOTS * (4 + vbytes<T>());
  static constexpr size_t work_bytes = ((((size_t)(CAP / 1 + 2 * CAP) * 4 + 7) & ~(size_t)7)) +
                                       (size_t)CAP * vbytes<T>();
  static constexpr size_t region0 = ((table_bytes > work_bytes ? table_bytes : work_bytes) + 15) & ~(size_t)15;
  static constexpr size_t compact = (((size_t)CAP * (4 + vbytes<T>())) + 15) & ~(size_t)15;
  static constexpr size_t per_warp = region0 + compact + 16;
};

template <class SR, int NWARP_SLOTS, int NWARP_CAP>
__global__ void __launch_bounds__(NWARP_WPB * 32, 4) k_num_warp(NumArgs a) {
  using T = typename SR::val_t;
  using L = WarpNumSmem<T, NWARP_SLOTS, NWARP_CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = lane_id();
  unsigned char *base = smem_raw + (size_t)w * L::per_warp;
  int *keys = reinterpret_cast<int *>(base);
  T *vals = reinterpret_cast<T *>(base + (size_t)NWARP_SLOTS * 4);
  int *ck = reinterpret_cast<int *>(base + L::region0);
  T *cv = reinterpret_cast<T *>(base + L::region0 + (size_t)NWARP_CAP * 4);
  EmitScratch *es = reinterpret_cast<EmitScratch *>(base + L::region0 + L::compact);
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  for (int idx = blockIdx.x * NWARP_WPB + w; idx < a.count; idx += gridDim.x * NWARP_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int64_t o = nout_row(a.A, r);
    const int64_t cb = a.Cp[o];
    const int c = (int)(a.Cp[o + 1] - cb);
    const int slots = max(64, min(NWARP_SLOTS, next_pow2(2 * min(c, NWARP_CAP))));
    const unsigned mask = slots - 1;
    for (int s = lane; s < slots; s += 32) {
      keys[s] = EMPTY;
      if constexpr (SR::has_val) vals[s] = SR::identity();
    }
    __syncwarp();
    warp_products<SR>(A, B, A.p[r], A.p[r + 1],
                      [&](int col, T v, int) { hash_insert_val<SR>(keys, vals, mask, col, v, a.err); });
    __syncwarp();
    group_sort_emit<WarpGroup, T, SR::has_val>(keys, vals, slots, c, ck, cv, base, nullptr, es, a.Cj + cb,
                                               SR::has_val ? Cv + cb : nullptr, a.err, NWARP_CAP, a.A.dbg,
                                               a.unsorted);
    __syncwarp();
  }
}

// ---------------------------------------------------- mid / large / heavy
// A entries per expansion round: the mid kernel stages fewer so that more of
// its CTAs fit an SM (rows in flight hide each other's latency)
template <int CAP> constexpr int nch() { return CAP >= 8192 ? 1024 : 256; }

template <typename T, int SLOTS, int CAP> struct CtaNumLayout {
  static constexpr size_t table_bytes = (size_t)SLOTS * (4 + vbytes<T>());
  static constexpr size_t work_bytes =
      ((((size_t)(CAP + 2 * CAP) * 4 + 7) & ~(size_t)7)) + (size_t)CAP * vbytes<T>();
  static constexpr size_t region0 = ((table_bytes > work_bytes ? table_bytes : work_bytes) + 15) & ~(size_t)15;
  static constexpr size_t compact = (((size_t)CAP * (4 + vbytes<T>())) + 15) & ~(size_t)15;
  static constexpr size_t ex_off = region0 + compact;
  static constexpr size_t tail_off = ex_off + ((sizeof(CtaExpandSmem<T, nch<CAP>()>) + 15) & ~(size_t)15);
  struct Tail {
    EmitScratch es;
    int wtmp[33];
    int row;
    int part_end;
    int part_cnt;
  };
  static constexpr size_t bytes = tail_off + sizeof(Tail);
};

template <class SR, int SLOTS, int CAP, int NT>
__global__ void __launch_bounds__(NT, 1) k_num_cta(NumArgs a) {
  using T = typename SR::val_t;
  using L = CtaNumLayout<T, SLOTS, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int *keys = reinterpret_cast<int *>(smem_raw);
  T *vals = reinterpret_cast<T *>(smem_raw + (size_t)SLOTS * 4);
  int *ck = reinterpret_cast<int *>(smem_raw + L::region0);
  T *cv = reinterpret_cast<T *>(smem_raw + L::region0 + (size_t)CAP * 4);
  auto &ex = *reinterpret_cast<CtaExpandSmem<T, nch<CAP>()> *>(smem_raw + L::ex_off);
  auto &tl = *reinterpret_cast<typename L::Tail *>(smem_raw + L::tail_off);
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  for (int idx = blockIdx.x; idx < a.count; idx += gridDim.x) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 36, r)) continue;  // uniform: every thread skips
    const int64_t o = nout_row(a.A, r);
    const int64_t cb = a.Cp[o];
    const int c = (int)(a.Cp[o + 1] - cb);
    const int slots = max(64, min(SLOTS, next_pow2(2 * min(c, CAP))));
    const unsigned mask = slots - 1;
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      keys[s] = EMPTY;
      if constexpr (SR::has_val) vals[s] = SR::identity();
    }
    __syncthreads();
    cta_products<SR, nch<CAP>()>(A, B, A.p[r], A.p[r + 1], false, 0, 0, ex, tl.wtmp,
                          [&](int col, T v, int) { hash_insert_val<SR>(keys, vals, mask, col, v, a.err); });
    const int64_t lofs = (a.loff && a.glist) ? a.loff[r] : -1;
    if (lofs >= 0) {
      // the symbolic pass left the row's sorted columns: no sort, each
      // column's value is looked up in the table
      const int32_t *Lr = a.glist + lofs;
      for (int i = threadIdx.x; i < c; i += blockDim.x) {
        const int col = __ldg(Lr + i);
        unsigned hh = hash_slot(col, mask);
        int probes = 0;
        while (keys[hh] != col && probes <= (int)mask) {
          hh = (hh + 1) & mask;
          ++probes;
        }
        if (probes > (int)mask) {  // a listed column the products never reached
          atomicExch(a.err, 11);
          continue;
        }
        __stcs(a.Cj + cb + i, col);
        if constexpr (SR::has_val) __stcs(Cv + cb + i, vals[hh]);
      }
    } else {
      group_sort_emit<CtaGroup, T, SR::has_val>(keys, vals, slots, c, ck, cv, smem_raw, tl.wtmp, &tl.es,
                                                a.Cj + cb, SR::has_val ? Cv + cb : nullptr, a.err, CAP, a.A.dbg,
                                                a.unsorted);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ heavy
// Rows whose output exceeds one shared table.  The row's columns are cut into
// parts (consecutive 4096-column segments, planned from the symbolic pass's
// segment counts) holding at most HEAVY_CAP outputs and spanning at most
// HV_WMAX columns.  Each part is accumulated with the sparse accumulator of
// Figure 1 split in two: its occupancy as a bitmap over the part's columns,
// its values as a compact array indexed by the column's rank among the
// part's set bits, rank(col) = wpre[word] + popcount(bits of the word below
// col).  When the symbolic pass left the row's sorted column list, the part's
// slice of it gives the bits and the word ranks directly (work in proportion
// to the part's outputs), the products are visited once (values added at
// their rank) and the slice is copied out as the part's columns.  Without a
// list the kernel builds the bitmap from the products (pass 1), ranks the
// words by prefix sums, adds the values (pass 2) and walks the bitmap to
// write the columns.  No hashing and no sorting either way.
//
// The B-row segment of each A entry for a part continues where the previous
// part's ended (a cursor per entry; in shared memory for rows of at most
// HV_CH entries, else in global scratch indexed like A's entries).  The end
// comes from the B segment index when the B row has one (its offset at the
// part's last segment), else from a search from the cursor.
constexpr int HV_NT = 512;          // threads per CTA; two CTAs share an SM
constexpr int HV_WMAX = HV_SPAN_SEGS * SEG_W;  // columns per part: a 32 KB bitmap
constexpr int HV_WORDS = HV_WMAX / 32;
constexpr int HV_CH = 512;          // A entries staged per expansion round

template <typename T> constexpr int heavy_cap() {
  return vbytes<T>() == 8 ? 4096 : (vbytes<T>() == 0 ? 16384 : 8192);  // as heavy_part_cap()
}

template <typename T> struct HeavySmem {
  unsigned bitmap[HV_WORDS];        // all zero at every part's start
  uint16_t wpre[HV_WORDS];          // set bits before word w within the part
  int wtot[HV_NT / 32 + 1];         // per-warp totals, then their exclusive scan
  int excl[HV_CH + 1];
  int64_t sbeg[HV_CH];
  int64_t ebase[HV_CH];             // rows of at most HV_CH entries: per entry its B row's start,
  int elen[HV_CH];                  //   length,
  int et[HV_CH];                    //   segment-index row (-1 none),
  int ecur[HV_CH];                  //   and cursor (offset of the next part's first entry)
  T aval[HV_CH];
  T vals[heavy_cap<T>()];
  int wtmp[33];
  int row, total;
  int part_end2[2], part_cnt2[2];   // this part's and the next part's plan
  int pre[SEG_SMEM + 1];            // exclusive prefix of the row's segment counts
};

// Pass 2's visitor: prep finds the product's rank in the part (bitmap word
// and word rank), commit adds the value there.  A product whose column is not
// in the part's structure raises error 10 instead.
template <class SR> struct HeavyAdd {
  using T = typename SR::val_t;
  static constexpr bool kTwoStage = true;
  struct State {
    int rank;  // -1: outside the structure; -2: failed guard (already recorded)
  };
  const unsigned *bitmap;
  const uint16_t *wpre;
  T *vals;
  int lo;
  unsigned span;
  int pc;
  int *err;
  long long *dbg;
  __device__ __forceinline__ State prep(int col) const {
    const unsigned x = (unsigned)(col - lo);
    if (!HS_G(dbg, x < span, 60, col)) return State{-2};
    const int w = (int)(x >> 5);
    const unsigned bits = bitmap[w];
    const unsigned bit = 1u << (x & 31);
    const int rank = wpre[w] + __popc(bits & (bit - 1u));
    return State{(!(bits & bit) || rank >= pc) ? -1 : rank};
  }
  __device__ __forceinline__ void commit(const State &s, T v) const {
    if (s.rank >= 0) SR::add_atomic(vals + s.rank, v);
    else if (s.rank == -1) atomicExch(err, 10);
  }
  __device__ __forceinline__ void operator()(int col, T v, int) const { commit(prep(col), v); }
};

template <class SR>
__global__ void __launch_bounds__(HV_NT, 2) k_num_heavy(NumArgs a) {
  using T = typename SR::val_t;
  constexpr int CAPH = heavy_cap<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &sm = *reinterpret_cast<HeavySmem<T> *>(smem_raw);
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  int32_t *gcur = a.gcur, *gend = a.gend;
  const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nw = HV_NT / 32;
  const int64_t n = a.B.n;
  const int nseg = (int)((n + SEG_W - 1) / SEG_W);
  const int64_t bstride = (int64_t)nseg + 1;
  long long *dbg = a.A.dbg;
  for (int w = tid; w < HV_WORDS; w += HV_NT) sm.bitmap[w] = 0u;

  while (true) {
    if (tid == 0) sm.row = atomicAdd(a.dyn, 1);
    __syncthreads();
    const int idx = sm.row;
    if (idx >= a.count) break;
    const int r0 = a.list[idx];
    // a bad row id is processed as an empty row so the loop reaches its barriers;
    // so is a row that the unit kernel takes (it has a sorted column list)
    const bool r_ok = HS_G(dbg, r0 >= 0 && r0 < a.A.nslots, 36, r0) &&
                      !(a.units && a.loff && a.loff[r0] >= 0 && a.hslot[r0] >= 0);
    const int r = r_ok ? r0 : 0;
    const int64_t o = nout_row(a.A, r);
    const int64_t cb = a.Cp[o];
    const int64_t c = r_ok ? a.Cp[o + 1] - cb : 0;
    const int h = r_ok ? a.hslot[r] : -1;
    if (r_ok && h < 0 && tid == 0) atomicExch(a.err, 4);
    const uint32_t *hist = a.hist + (int64_t)(h < 0 ? 0 : h) * a.nseg;
    const int64_t q0 = A.p[r], q1 = r_ok ? A.p[r + 1] : q0;
    const int nrounds = (int)((q1 - q0 + HV_CH - 1) / HV_CH);
    const bool cached = nrounds == 1;
    // the row's sorted column list left by the symbolic pass, if any
    const int64_t lofs = (r_ok && a.loff && a.glist) ? a.loff[r] : -1;
    const int32_t *L = lofs >= 0 ? a.glist + lofs : nullptr;
    if (L && tid == 0) prefetch_l2(L, c * 4);  // the row's parts read it in order
    if (cached) {
      const int cnt = (int)(q1 - q0);
      for (int e = tid; e < cnt; e += HV_NT) {
        const int64_t q = q0 + e;
        const int k = __ldg(A.j + q);
        int64_t base = 0;
        int len = 0, t = -1;
        if (HS_G(dbg, k >= 0 && k < B.rows, 2, k)) {
          base = __ldg(B.p + k);
          len = (int)(__ldg(B.p + k + 1) - base);
          if (a.bci_id) t = __ldg(a.bci_id + k);
        }
        sm.ebase[e] = base;
        sm.elen[e] = len;
        sm.et[e] = t;
        sm.ecur[e] = 0;
        if constexpr (SR::needs_a) sm.aval[e] = load_val<T>(A.v, q);
      }
    } else {
      for (int64_t q = q0 + tid; q < q1; q += HV_NT) gcur[q] = 0;
    }
    // the row's parts, chosen greedily from its segment counts: at most CAPH
    // outputs and HV_WMAX columns each
    const bool plan = h >= 0 && nseg <= SEG_SMEM;
    if (plan) {
      for (int g = tid; g < nseg; g += HV_NT) sm.pre[g] = (int)hist[g];
      __syncthreads();
      const int tot = group_excl_scan<CtaGroup>(sm.pre, nseg, sm.wtmp);
      if (tid == 0) sm.pre[nseg] = tot;
    }
    // part planning (thread 0): the part starting at segment sg ends at the
    // last segment end in (sg, sg + HV_WMAX/SEG_W] that keeps at most CAPH
    // outputs; the next part is planned during the current one into the
    // other of two slots, so parts need no barrier of their own
    auto plan_part = [&](int sg, int slot) {
      const int emax = min(nseg, sg + HV_WMAX / SEG_W);
      int e = sg, sum = 0;
      if (plan) {
        const int base = sm.pre[sg];
        int lo_e = sg + 1, hi_e = emax;
        while (lo_e < hi_e) {
          const int mid = (lo_e + hi_e + 1) >> 1;
          if (sm.pre[mid] - base <= CAPH) lo_e = mid;
          else hi_e = mid - 1;
        }
        e = lo_e;
        sum = sm.pre[e] - base;
        if (sum > CAPH) e = sg;  // cannot happen: a segment holds at most SEG_W <= CAPH outputs
      } else {
        while (e < emax && sum + (int)hist[e] <= CAPH) sum += (int)hist[e++];
      }
      if (e == sg) {
        atomicExch(a.err, 5);
        e = nseg;
        sum = 0;
      }
      sm.part_end2[slot] = e;
      sm.part_cnt2[slot] = sum;
    };
    int64_t done = 0;
    int seg = 0, slot = 0;
    if (tid == 0 && h >= 0 && nseg > 0) plan_part(0, 0);
    __syncthreads();  // also orders the row set-up before the first part's reads
    while (seg < nseg && h >= 0) {
      const int pe = sm.part_end2[slot], pc = sm.part_cnt2[slot];
      if (tid == 0 && pe < nseg) plan_part(pe, slot ^ 1);
      if (pc > 0) {
        const int lo = seg * SEG_W;
        const int hi = (int)min((int64_t)pe * SEG_W, n);
        const int words = (hi - lo + 31) >> 5;
        const int32_t *Lp = (L && HS_G(dbg, done + pc <= c, 64, done + pc)) ? L + done : nullptr;
        // ---- occupancy and word ranks from the list: one bit per column and
        // one rank store per nonempty word
        // rows on the fast path below write their columns here, straight from
        // the list (they are C's columns of this part, in order)
        const bool cols_now = cached && Lp;
        const int64_t out = cb + done;
        if (Lp) {
          constexpr int U = 4;  // loads in flight per thread
          for (int i0 = tid; i0 < pc; i0 += U * HV_NT) {
            int x[U], xp[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int i = i0 + u * HV_NT;
              x[u] = i < pc ? __ldg(Lp + i) - lo : -1;
              xp[u] = (i < pc && i > 0) ? __ldg(Lp + i - 1) - lo : -1;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int i = i0 + u * HV_NT;
              if (i >= pc) continue;
              if (cols_now) __stcs(a.Cj + out + i, x[u] + lo);
              if (!HS_G(dbg, x[u] >= 0 && x[u] < hi - lo, 63, x[u])) continue;
              const int w = x[u] >> 5;
              atomicOr(sm.bitmap + w, 1u << (x[u] & 31));
              if (i == 0 || (xp[u] >> 5) != w) sm.wpre[w] = (uint16_t)i;
            }
          }
        }
        // segment [s, s + len) of cached entry e in this part; advances its cursor
        auto seg_end = [&](int e, int64_t &s) -> int {
          const int64_t base = sm.ebase[e];
          const int cur = sm.ecur[e], t = sm.et[e], rl = sm.elen[e];
          int eo = t >= 0 ? __ldg(a.bci + (int64_t)t * bstride + pe)
                          : (int)(interp_lower_bound(B.j, base + cur, base + rl, hi) - base);
          if (!HS_G(dbg, eo >= cur && eo <= rl, 65, eo)) eo = cur;
          s = base + cur;
          sm.ecur[e] = eo;
          return eo - cur;
        };
        bool consistent = true;
        if (cached && Lp) {
          // nearly every heavy row: its entries are cached and its columns
          // listed, so the segment ends, the value reset and the list's bitmap
          // share one phase; rows of at most 32 entries scan in one warp
          const int cnt = (int)(q1 - q0);
          if constexpr (SR::has_val)
            for (int i = tid; i < pc; i += HV_NT) sm.vals[i] = SR::identity();
          if (cnt <= 32) {
            if (warp == 0) {
              int64_t s = 0;
              const int len = lane < cnt ? seg_end(lane, s) : 0;
              const int incl = warp_incl_scan(len);
              if (lane < cnt) {
                sm.excl[lane] = incl - len;
                sm.sbeg[lane] = s;
              }
              if (lane == 31) sm.excl[cnt] = incl;
            }
            __syncthreads();
          } else {
            for (int e = tid; e < cnt; e += HV_NT) {
              int64_t s = 0;
              sm.excl[e] = seg_end(e, s);
              sm.sbeg[e] = s;
            }
            __syncthreads();
            const int t = group_excl_scan<CtaGroup>(sm.excl, cnt, sm.wtmp);
            if (tid == 0) sm.excl[cnt] = t;
            __syncthreads();
          }
          if constexpr (SR::has_val) {
            HeavyAdd<SR> add_val{sm.bitmap, sm.wpre, sm.vals, lo, (unsigned)(hi - lo), pc, a.err, dbg};
            cta_expand_staged<SR, 4, 32>(B, sm.sbeg, sm.excl, sm.aval, cnt, sm.excl[cnt], add_val);
          }
          __syncthreads();
        } else {
          // ---- B segments of the part (and, without a list, pass 1)
          int total = 0;
          for (int rd = 0; rd < nrounds; ++rd) {
            const int64_t rq0 = q0 + (int64_t)rd * HV_CH;
            const int cnt = (int)min((int64_t)HV_CH, q1 - rq0);
            __syncthreads();
            for (int e = tid; e < cnt; e += HV_NT) {
              int64_t s = 0;
              int len = 0;
              if (cached) {
                len = seg_end(e, s);
              } else {
                const int64_t q = rq0 + e;
                const int k = __ldg(A.j + q);
                if (HS_G(dbg, k >= 0 && k < B.rows, 2, k)) {
                  const int64_t base = __ldg(B.p + k), end = __ldg(B.p + k + 1);
                  const int t = a.bci_id ? __ldg(a.bci_id + k) : -1;
                  s = base + gcur[q];
                  int64_t se = t >= 0 ? base + __ldg(a.bci + (int64_t)t * bstride + pe)
                                      : interp_lower_bound(B.j, s, end, hi);
                  if (!HS_G(dbg, se >= s && se <= end, 65, se)) se = s;
                  len = (int)(se - s);
                  gend[q] = (int32_t)(se - base);
                }
              }
              sm.excl[e] = len;
              sm.sbeg[e] = s;
            }
            if (!cached && Lp) continue;  // only the part ends are needed (pass 2 restages)
            __syncthreads();
            total = group_excl_scan<CtaGroup>(sm.excl, cnt, sm.wtmp);
            if (tid == 0) sm.excl[cnt] = total;
            __syncthreads();
            if (!Lp) {
              auto set_bit = [&](int col, NoVal, int) {
                const int x = col - lo;
                if (HS_G(dbg, x >= 0 && x < hi - lo, 60, col)) atomicOr(sm.bitmap + (x >> 5), 1u << (x & 31));
              };
              cta_expand_staged<StructOf<SR>>(B, sm.sbeg, sm.excl, reinterpret_cast<const NoVal *>(sm.aval), cnt,
                                              total, set_bit);
            }
          }
          __syncthreads();
          if (!Lp) {
            // ---- rank: prefix of set bits per word, in runs of 32 words per warp
            const int wpw = ((words + nw - 1) / nw + 31) & ~31;
            const int w0 = warp * wpw, w1 = min(words, w0 + wpw);
            int carry = 0;
            for (int wb = w0; wb < w1; wb += 32) {
              const int w = wb + lane;
              const int pc_w = w < w1 ? __popc(sm.bitmap[w]) : 0;
              const int incl = warp_incl_scan(pc_w);
              if (w < w1) sm.wpre[w] = (uint16_t)(carry + incl - pc_w);
              carry += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) sm.wtot[warp] = carry;
            __syncthreads();
            if (warp == 0) {
              const int t = lane < nw ? sm.wtot[lane] : 0;
              const int ti = warp_incl_scan(t);
              if (lane < nw) sm.wtot[lane] = ti - t;
              if (lane == nw - 1) sm.total = ti;
            }
            __syncthreads();
            const int add = sm.wtot[warp];
            for (int w = w0 + lane; w < w1; w += 32) sm.wpre[w] = (uint16_t)(sm.wpre[w] + add);
          } else if (tid == 0) {
            sm.total = pc;
          }
          if constexpr (SR::has_val)
            for (int i = tid; i < pc; i += HV_NT) sm.vals[i] = SR::identity();
          __syncthreads();
          consistent = sm.total == pc;
          if (!consistent && tid == 0) atomicExch(a.err, 9);
          // ---- pass 2: values at their rank
          if constexpr (SR::has_val) {
            HeavyAdd<SR> add_val{sm.bitmap, sm.wpre, sm.vals, lo, (unsigned)(hi - lo), pc, a.err, dbg};
            if (!cached) {
              for (int rd = 0; rd < nrounds; ++rd) {
                const int64_t rq0 = q0 + (int64_t)rd * HV_CH;
                const int cnt = (int)min((int64_t)HV_CH, q1 - rq0);
                __syncthreads();
                for (int e = tid; e < cnt; e += HV_NT) {
                  int64_t s = 0;
                  int len = 0;
                  const int64_t q = rq0 + e;
                  const int k = __ldg(A.j + q);
                  if (HS_G(dbg, k >= 0 && k < B.rows, 2, k)) {
                    const int64_t base = __ldg(B.p + k);
                    s = base + gcur[q];
                    len = gend[q] - gcur[q];
                    gcur[q] = gend[q];
                    if constexpr (SR::needs_a) sm.aval[e] = load_val<T>(A.v, q);
                  }
                  sm.excl[e] = len;
                  sm.sbeg[e] = s;
                }
                __syncthreads();
                total = group_excl_scan<CtaGroup>(sm.excl, cnt, sm.wtmp);
                if (tid == 0) sm.excl[cnt] = total;
                __syncthreads();
                cta_expand_staged<SR, 4, 32>(B, sm.sbeg, sm.excl, sm.aval, cnt, total, add_val);
              }
            } else {
              cta_expand_staged<SR, 4, 32>(B, sm.sbeg, sm.excl, sm.aval, (int)(q1 - q0), total, add_val);
            }
            __syncthreads();
          } else if (!cached) {
            // structure only: still advance the cursors past this part
            for (int64_t q = q0 + tid; q < q1; q += HV_NT) gcur[q] = gend[q];
          }
        }
        // ---- emit (columns ascending, values in rank order), then clear the bitmap
        const bool fits = consistent && HS_G(dbg, done + pc <= c, 62, done + pc);
        if (cols_now) {
          // columns already written; clear the part's words
          for (int w = tid; w < words; w += HV_NT) sm.bitmap[w] = 0u;
        } else if (Lp) {
          constexpr int U = 4;
          for (int i0 = tid; i0 < pc; i0 += U * HV_NT) {
            int col[U];
#pragma unroll
            for (int u = 0; u < U; ++u) col[u] = i0 + u * HV_NT < pc ? __ldg(Lp + i0 + u * HV_NT) : lo - 1;
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int i = i0 + u * HV_NT;
              if (i >= pc) continue;
              if (fits) __stcs(a.Cj + out + i, col[u]);
              const int x = col[u] - lo;
              if (x >= 0 && x < hi - lo) sm.bitmap[x >> 5] = 0u;
            }
          }
        } else {
          for (int w = tid; w < words; w += HV_NT) {
            unsigned bits = sm.bitmap[w];
            int pos = sm.wpre[w];
            if (fits)
              while (bits) {
                const int b = __ffs(bits) - 1;
                a.Cj[out + pos] = lo + (w << 5) + b;
                ++pos;
                bits &= bits - 1;
              }
            sm.bitmap[w] = 0u;
          }
        }
        if constexpr (SR::has_val)
          if (fits)
            for (int i = tid; i < pc; i += HV_NT) __stcs(Cv + out + i, sm.vals[i]);
        done += pc;
      }
      seg = pe;
      slot ^= 1;
      __syncthreads();
    }
    if (tid == 0 && r_ok && done != c) atomicExch(a.err, 6);
    __syncthreads();
  }
}

// ------------------------------------------------------------ heavy units
// The heavy bin's rows that have a sorted column list, by units: one column
// part of one row per unit, handed out to CTAs by an atomic counter, so a hub
// row's parts run on many SMs at once and no row's length sets the kernel's
// tail.  Everything a unit reads that depends on other data has been laid out
// before the kernel runs: the part's slice of the row's sorted column list
// (written by the symbolic pass) and the part's B segments with their product
// prefix and left value (launch_build_pairs, which does the segment searches
// for all units in bulk).  A unit copies both into shared memory with
// cp.async, then: the list slice is written as C's columns and gives the
// part's occupancy bitmap and word ranks; the products add their value at
// rank(col) = wpre[word] + popcount(bits below col), spread evenly over the
// warps by their prefix; the values leave in column order.  Parts span at
// most 2^17 columns and hold KB kilobytes of values (16 or 32, at least a
// whole segment's 4096 outputs), so five CTAs of 256 threads share an SM
// with 16 KB parts (48 registers; three for 8-byte values or 32 KB parts).
constexpr int HU_NT = 256;
constexpr int HU_WMAX = HU_SPAN_SEGS * SEG_W;
constexpr int HU_WORDS = HU_WMAX / 32;
constexpr int HU_PB = 256;  // B segments copied per batch
// as unit_part_cap(): KB kilobytes of values, at least one segment's SEG_W outputs
template <typename T, int KB> constexpr int unit_cap() {
  return vbytes<T>() == 0 ? 65536 : (KB * 1024 / vbytes<T>() > SEG_W ? KB * 1024 / vbytes<T>() : SEG_W);
}

template <typename T, int KB> struct UnitSmem {
  static constexpr int CAP = vbytes<T>() ? unit_cap<T, KB>() : 1;
  // the part's values; first the list slice lands here (4-byte column ids
  // plus the copy's 32 bytes of alignment room)
  static constexpr size_t VBYTES = ((size_t)CAP * (vbytes<T>() > 4 ? vbytes<T>() : 4) + 32 + 15) & ~(size_t)15;
  alignas(16) unsigned char vals_raw[VBYTES];
  alignas(16) unsigned bitmap[HU_WORDS];  // all zero at every unit's start
  alignas(16) int64_t sbeg[HU_PB + 4];   // B segment starts (+ copy room)
  alignas(16) int excl[HU_PB + 8];       // their product prefix, then the batch's end
  alignas(16) unsigned char aval_raw[(HU_PB + 4) * (vbytes<T>() > 4 ? 8 : 4) + 16];
  uint16_t wpre[HU_WORDS];                // set bits before word w within the part
  int wtmp[33];
  int unit;
};

template <class SR, int KB>
__global__ void __launch_bounds__(HU_NT, (KB > 16 || vbytes<typename SR::val_t>() == 8) ? 3 : 5) k_num_units(NumArgs a) {
  using T = typename SR::val_t;
  using L = UnitSmem<T, KB>;
  constexpr int CAP = unit_cap<T, KB>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &sm = *reinterpret_cast<L *>(smem_raw);
  const DevCsr B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  T *vals = reinterpret_cast<T *>(sm.vals_raw);
  const int tid = threadIdx.x, lane = lane_id();
  const int64_t n = a.B.n;
  const int nseg = (int)((n + SEG_W - 1) / SEG_W);
  long long *dbg = a.A.dbg;
  if constexpr (SR::has_val)
    for (int w = tid; w < HU_WORDS; w += HU_NT) sm.bitmap[w] = 0u;
  if (tid == 0) sm.unit = atomicAdd(a.udyn, 1);
  __syncthreads();
  while (true) {
    const int64_t ui = sm.unit;
    if (ui >= a.nunits) break;
    const HeavyUnit u = a.units[ui];
    // the next unit is claimed now; its descriptor is brought into L2 once
    // the counter answers, so neither round trip waits at the unit's end
    int nxt = 0;
    if (tid == 0) nxt = atomicAdd(a.udyn, 1);
    // every thread reads the same words, so a failed check skips the unit in
    // every thread alike and the barriers below stay matched (the planner
    // checked that the part lies inside its row)
    const bool ok = HS_G(dbg, u.seg_lo >= 0 && u.seg_lo < u.seg_hi && u.seg_hi <= nseg &&
                                  u.seg_hi - u.seg_lo <= HU_SPAN_SEGS, 72, u.seg_lo) &&
                    HS_G(dbg, u.pc > 0 && u.pc <= CAP, 73, u.pc) &&
                    HS_G(dbg, u.npairs >= 0 && u.nprod >= 0 && u.out >= 0 && u.lofs >= 0, 77, u.npairs);
    if (ok) {
      const int lo = u.seg_lo * SEG_W;
      const int hi = (int)min((int64_t)u.seg_hi * SEG_W, n);
      const int pc = u.pc;
      const int32_t *Lp = a.glist + u.lofs;
      const int64_t out = u.out;
      if constexpr (SR::has_val) {
        // the list slice and the first batch of B segments, copied at once
        const int nb0 = u.npairs < HU_PB ? u.npairs : HU_PB;
        const int lofb = async_copy16(sm.vals_raw, Lp, (int64_t)pc * 4, tid, HU_NT) >> 2;
        const int sofb = async_copy16(sm.sbeg, a.pstart + u.poff, (int64_t)nb0 * 8, tid, HU_NT) >> 3;
        const int eofb = async_copy16(sm.excl, a.ppre + u.poff, (int64_t)nb0 * 4, tid, HU_NT) >> 2;
        int aofb = 0;
        if constexpr (SR::needs_a)
          aofb = async_copy16(sm.aval_raw, reinterpret_cast<const T *>(a.paval) + u.poff,
                              (int64_t)nb0 * sizeof(T), tid, HU_NT) / (int)sizeof(T);
        async_copy_wait();
        __syncthreads();
        // columns out, bits and word ranks in (entry i starts word w when
        // entry i-1 lies in another word)
        const int32_t *Ls = reinterpret_cast<const int32_t *>(sm.vals_raw) + lofb;
        for (int i = tid; i < pc; i += HU_NT) {
          const int col = Ls[i];
          __stcs(a.Cj + out + i, col);
          const int xx = col - lo;
          if (!HS_G(dbg, xx >= 0 && xx < hi - lo, 63, col)) continue;
          const int w = xx >> 5;
          atomicOr(sm.bitmap + w, 1u << (xx & 31));
          if (i == 0 || ((Ls[i - 1] - lo) >> 5) != w) sm.wpre[w] = (uint16_t)i;
        }
        if (tid == 0 && nxt < a.nunits) prefetch_l2(a.units + nxt, sizeof(HeavyUnit));
        __syncthreads();  // the list slice is read: its room becomes the values
        for (int i = tid; i < pc; i += HU_NT) vals[i] = SR::identity();
        HeavyAdd<SR> add_val{sm.bitmap, sm.wpre, vals, lo, (unsigned)(hi - lo), pc, a.err, dbg};
        for (int pb = 0; pb < u.npairs; pb += HU_PB) {
          const int nb = min(HU_PB, u.npairs - pb);
          int so = sofb, eo = eofb, ao = aofb;
          if (pb > 0) {  // the next batch (rows with many A entries)
            __syncthreads();
            so = async_copy16(sm.sbeg, a.pstart + u.poff + pb, (int64_t)nb * 8, tid, HU_NT) >> 3;
            eo = async_copy16(sm.excl, a.ppre + u.poff + pb, (int64_t)nb * 4, tid, HU_NT) >> 2;
            if constexpr (SR::needs_a)
              ao = async_copy16(sm.aval_raw, reinterpret_cast<const T *>(a.paval) + u.poff + pb,
                                (int64_t)nb * sizeof(T), tid, HU_NT) / (int)sizeof(T);
            async_copy_wait();
            __syncthreads();  // every copy has landed (the batch end below may share a copied piece)
          }
          int *ex = sm.excl + eo;
          if (tid == 0) ex[nb] = pb + nb < u.npairs ? __ldg(a.ppre + u.poff + pb + nb) : u.nprod;
          __syncthreads();
          const int base = ex[0];
          cta_expand_staged<SR, 4, 32>(B, sm.sbeg + so, ex, reinterpret_cast<const T *>(sm.aval_raw) + ao, nb,
                                       ex[nb] - base, add_val, base);
        }
        __syncthreads();
        // values in column order; the part's bitmap words cleared for the next unit
        for (int i = tid; i < pc; i += HU_NT) __stcs(Cv + out + i, vals[i]);
        const int words = (hi - lo + 31) >> 5;
        for (int w = tid; w < words; w += HU_NT) sm.bitmap[w] = 0u;
      } else {
        // structure only: the list slice is the part's columns
        for (int i = tid; i < pc; i += HU_NT) __stcs(a.Cj + out + i, __ldg(Lp + i));
      }
    }
    (void)lane;
    __syncthreads();  // every thread has read sm.unit; the part's buffers are free
    if (tid == 0) sm.unit = nxt;
    __syncthreads();
  }
}

// ------------------------------------------------------------ launchers
inline int ngrid_cap(int items, int per_block, int per_sm) {
  int g = (items + per_block - 1) / per_block;
  int cap = sm_count() * per_sm;
  return g < cap ? (g < 1 ? 1 : g) : cap;
}
// CTAs that fit one SM for this kernel, block size and dynamic shared memory
template <class K> int fit_per_sm(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return n < 1 ? 1 : n;
}

// ------------------------------------------------------------- sort tiers
// Rows with 32 < f <= F_SORT whose output count is close to their product
// count: one warp per row sorts the row's products (sort_row), one kernel
// per register width K (32*K products), so each kernel's code stays small.
// Only the tiers of at most 32*SORT_WIDE_K products sort 64-bit keys for
// rows spanning too many columns.
constexpr int NSORT_WPB = 4;
static_assert(SORT_WIDE_K * 32 == F_SORT_S, "the wide-key tiers are those of at most 256 products");
template <typename T, int K> struct SortSmemLayout {
  static constexpr size_t col_bytes = ((size_t)sr_pad_len(32 * K) * 4 + 15) & ~(size_t)15;
  static constexpr size_t per_warp = col_bytes + (((size_t)32 * K * vbytes<T>() + 15) & ~(size_t)15);
};
template <class SR, int K>
__global__ void __launch_bounds__(NSORT_WPB * 32, K >= 32 ? 6 : 8) k_num_sort(NumArgs a) {
  using T = typename SR::val_t;
  using L = SortSmemLayout<T, K>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5;
  int *s_col = reinterpret_cast<int *>(smem_raw + (size_t)w * L::per_warp);
  T *s_val = reinterpret_cast<T *>(smem_raw + (size_t)w * L::per_warp + L::col_bytes);
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  for (int idx = blockIdx.x * NSORT_WPB + w; idx < a.count; idx += gridDim.x * NSORT_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int64_t o = nout_row(a.A, r);
    const int64_t cb = a.Cp[o];
    const int c = (int)(a.Cp[o + 1] - cb);
    const int64_t F = a.f[r];
    T *out_v = SR::has_val ? Cv + cb : nullptr;
    sort_row<SR, K, (K <= SORT_WIDE_K)>(A, B, A.p[r], A.p[r + 1], F <= 32 * K ? (int)F : -1, c, s_col, s_val,
                                        a.Cj + cb, out_v, a.err);
    __syncwarp();
  }
}

template <class SR, int K> void launch_num_sort(const NumArgs &a, cudaStream_t st) {
  using T = typename SR::val_t;
  const size_t bytes = SortSmemLayout<T, K>::per_warp * NSORT_WPB;
  auto k = k_num_sort<SR, K>;
  set_smem_attr(k, bytes);
  count_launch();
  k<<<ngrid_cap(a.count, NSORT_WPB, fit_per_sm(k, NSORT_WPB * 32, bytes)), NSORT_WPB * 32, bytes, st>>>(a);
}

// ------------------------------------------------------------- dense SPA
// Products whose B has at most spa_cols() columns (Figure 1's sparse
// accumulator as it stands): one warp per row keeps a value for every column
// and an occupancy flag per column (a byte, set by a plain store, so lanes
// that hit one column do not queue on an atomic); lanes whose products share
// a column fold their values first (__match_any_sync) and one of them adds
// the sum.  The row leaves in column order by walking the flags (a lane owns
// a run of consecutive flag words; an exclusive scan of their counts gives
// each run's start).  Every value is reset to the identity and every flag
// cleared as it is written out, so the arrays are cleared once per kernel.
constexpr int NSPA_WPB = 4;
template <typename T> struct SpaLayout {
  static constexpr int COLS = spa_cols(vbytes<T>());
  static constexpr size_t flag_bytes = (size_t)COLS;
  static constexpr size_t per_warp = flag_bytes + (((size_t)COLS * vbytes<T>() + 15) & ~(size_t)15);
};
// the semiring's add folded over the lanes of `grp` (lanes with one column);
// every lane of the group returns the fold, in lane order
template <class SR>
__device__ __forceinline__ typename SR::val_t group_fold(unsigned grp, typename SR::val_t v) {
  using T = typename SR::val_t;
  T acc = v;
  bool first = true;
  for (unsigned m = grp; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
    const T x = __shfl_sync(grp, v, src);
    acc = first ? x : SR::add(acc, x);
    first = false;
  }
  return acc;
}
template <class SR>
__global__ void __launch_bounds__(NSPA_WPB * 32, 8) k_num_spa(NumArgs a) {
  using T = typename SR::val_t;
  using L = SpaLayout<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = lane_id();
  unsigned char *flag = smem_raw + (size_t)w * L::per_warp;
  T *vals = reinterpret_cast<T *>(smem_raw + (size_t)w * L::per_warp + L::flag_bytes);
  unsigned *flag4 = reinterpret_cast<unsigned *>(flag);
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  const int n = (int)a.B.n;
  const int fwords = (n + 3) >> 2;         // flag words of 4 columns
  const int wpl = (fwords + 31) >> 5;      // flag words a lane walks
  for (int i = lane; i < (L::COLS >> 2); i += 32) flag4[i] = 0u;
  if constexpr (SR::has_val)
    for (int i = lane; i < n; i += 32) vals[i] = SR::identity();
  __syncwarp();
  for (int idx = blockIdx.x * NSPA_WPB + w; idx < a.count; idx += gridDim.x * NSPA_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int64_t o = nout_row(a.A, r);
    const int64_t cb = a.Cp[o];
    const int c = (int)(a.Cp[o + 1] - cb);
    warp_products<SR>(A, B, A.p[r], A.p[r + 1], [&](int col, T v, int) {
      const bool ok = HS_G(a.A.dbg, col >= 0 && col < n, 85, col);
      if (ok) flag[col] = 1;
      if constexpr (SR::has_val) {
        const unsigned grp = __match_any_sync(__activemask(), ok ? col : -1);
        if (ok) {
          const T sum = (grp & (grp - 1)) ? group_fold<SR>(grp, v) : v;
          if (lane == __ffs(grp) - 1) SR::add_atomic(vals + col, sum);
        }
      }
    });
    __syncwarp();
    const int w0 = lane * wpl, w1 = min(fwords, w0 + wpl);
    int cnt = 0;
    for (int i = w0; i < w1; ++i) cnt += __popc(flag4[i] & 0x01010101u);
    const int incl = warp_incl_scan(cnt);
    const int total = __shfl_sync(FULL, incl, 31);
    if (total != c) {
      if (lane == 0) atomicExch(a.err, 1);
    } else {
      int pos = incl - cnt;
      for (int i = w0; i < w1; ++i) {
        const unsigned fw = flag4[i];
        if (!fw) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!((fw >> (8 * k)) & 0xffu)) continue;
          const int col = (i << 2) + k;
          __stcs(a.Cj + cb + pos, col);
          if constexpr (SR::has_val) {
            __stcs(Cv + cb + pos, vals[col]);
            vals[col] = SR::identity();
          }
          ++pos;
        }
      }
    }
    for (int i = w0; i < w1; ++i) flag4[i] = 0u;
    if constexpr (SR::has_val)
      if (total != c)  // values left behind by a row that failed its check
        for (int i = lane; i < n; i += 32) vals[i] = SR::identity();
    __syncwarp();
  }
}

template <class SR> void launch_num_spa(const NumArgs &a, cudaStream_t st) {
  using T = typename SR::val_t;
  const size_t bytes = SpaLayout<T>::per_warp * NSPA_WPB;
  auto k = k_num_spa<SR>;
  set_smem_attr(k, bytes);
  count_launch();
  k<<<ngrid_cap(a.count, NSPA_WPB, fit_per_sm(k, NSPA_WPB * 32, bytes)), NSPA_WPB * 32, bytes, st>>>(a);
}

template <class SR, int SLOTS, int CAP> void launch_num_warp(const NumArgs &a, cudaStream_t st) {
  using T = typename SR::val_t;
  const size_t bytes = WarpNumSmem<T, SLOTS, CAP>::per_warp * NWARP_WPB;
  auto k = k_num_warp<SR, SLOTS, CAP>;
  set_smem_attr(k, bytes);
  count_launch();
  k<<<ngrid_cap(a.count, NWARP_WPB, fit_per_sm(k, NWARP_WPB * 32, bytes)), NWARP_WPB * 32, bytes, st>>>(a);
}

template <class SR, int SLOTS, int CAP, int NT> void launch_num_cta(const NumArgs &a, cudaStream_t st) {
  using T = typename SR::val_t;
  using L = CtaNumLayout<T, SLOTS, CAP>;
  auto k = k_num_cta<SR, SLOTS, CAP, NT>;
  set_smem_attr(k, L::bytes);
  count_launch();
  k<<<ngrid_cap(a.count, 1, fit_per_sm(k, NT, L::bytes)), NT, L::bytes, st>>>(a);
}

template <class SR, int KB> void launch_num_units(const NumArgs &a, cudaStream_t st) {
  using T = typename SR::val_t;
  const size_t ub = sizeof(UnitSmem<T, KB>);
  auto ku = k_num_units<SR, KB>;
  set_smem_attr(ku, ub);
  count_launch();
  const int items = a.nunits < (1 << 30) ? (int)a.nunits : (1 << 30);
  ku<<<ngrid_cap(items, 1, fit_per_sm(ku, HU_NT, ub)), HU_NT, ub, st>>>(a);
}

template <class SR> void launch_numeric_sr(int kind, const NumArgs &a, cudaStream_t st) {
  using T = typename SR::val_t;
  if (a.count <= 0) return;
  constexpr int CAPL = cap_large<T>();
  switch (kind) {
    case 0:
      count_launch();
      k_num_tiny<SR><<<ngrid_cap(a.count, NTINY_WPB, 8), NTINY_WPB * 32, 0, st>>>(a);
      break;
    case 1: launch_num_warp<SR, 2 * F_WARP_S, F_WARP_S>(a, st); break;
    case 2: launch_num_warp<SR, 2 * F_WARP, F_WARP>(a, st); break;
    case 3: launch_num_cta<SR, 2 * CAP_MID_S, CAP_MID_S, 256>(a, st); break;
    case 4: launch_num_cta<SR, 2 * CAP_MID, CAP_MID, 256>(a, st); break;
    case 5:
      if constexpr (CAPL / 2 > CAP_MID) launch_num_cta<SR, CAPL, CAPL / 2, 512>(a, st);
      break;
    case 6: launch_num_cta<SR, 2 * CAPL, CAPL, 1024>(a, st); break;
    case 7: launch_num_sort<SR, 4>(a, st); break;
    case 8: launch_num_sort<SR, 8>(a, st); break;
    case 9: launch_num_sort<SR, 16>(a, st); break;
    case 10: launch_num_sort<SR, 32>(a, st); break;
    case 11: launch_num_spa<SR>(a, st); break;
    case 12: {
      if (a.units && a.nunits > 0) {
        if (a.unit_kb > 16) launch_num_units<SR, 32>(a, st);
        else launch_num_units<SR, 16>(a, st);
      }
      if (!a.units || a.lists_partial) {  // rows without a list: one CTA per row
        const size_t bytes = sizeof(HeavySmem<T>);
        set_smem_attr(k_num_heavy<SR>, bytes);
        count_launch();
        k_num_heavy<SR><<<ngrid_cap(a.count, 1, 2), HV_NT, bytes, st>>>(a);
      }
      break;
    }
  }
}

}  // namespace hs
