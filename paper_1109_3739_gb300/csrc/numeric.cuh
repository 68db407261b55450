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
//   heavy (c > CAP)        one CTA of 1024 per row, rows handed out largest
//                          first; the row's columns are cut into parts of at
//                          most CAP outputs using the per-segment counts of
//                          the symbolic pass, and each part runs the large
//                          kernel's accumulator over the products that fall
//                          in its column range.
// The shared hash table is the sparse accumulator of Figure 1 with the dense
// value array replaced by open addressing (keys + values), so its size
// follows the row's output, not the matrix dimension (Section 2.1's argument
// against dimension-dependent work).
#pragma once
#include "common.cuh"
#include "internal.h"

namespace hs {

__device__ __forceinline__ DevCsr ndev_a(const RowSet &A) { return DevCsr{A.p, A.j, A.v, A.nslots, A.nnz, A.dbg}; }
__device__ __forceinline__ DevCsr ndev_b(const RightOp &B) { return DevCsr{B.p, B.j, B.v, B.m, B.nnz, B.dbg}; }
__device__ __forceinline__ int64_t nout_row(const RowSet &A, int r) {
  return A.ids ? (int64_t)A.ids[r] : (int64_t)r;
}

template <typename T> constexpr int vbytes() { return sizeof(T); }
template <> constexpr int vbytes<NoVal>() { return 0; }

template <typename T> constexpr int cap_large() { return vbytes<T>() == 8 ? 4096 : 8192; }

// --------------------------------------------------------------- tiny
constexpr int NTINY_WPB = 8;
template <class SR>
__global__ void __launch_bounds__(NTINY_WPB * 32) k_num_tiny(NumArgs a) {
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
constexpr int NWARP_WPB = 4, NWARP_SLOTS = 1024, NWARP_CAP = 512;

template <typename T> struct WarpNumSmem {
  static constexpr size_t table_bytes = (size_t)NWARP_SLOTS * (4 + vbytes<T>());
  static constexpr size_t work_bytes = ((((size_t)(NWARP_CAP / 1 + 2 * NWARP_CAP) * 4 + 7) & ~(size_t)7)) +
                                       (size_t)NWARP_CAP * vbytes<T>();
  static constexpr size_t region0 = ((table_bytes > work_bytes ? table_bytes : work_bytes) + 15) & ~(size_t)15;
  static constexpr size_t compact = (((size_t)NWARP_CAP * (4 + vbytes<T>())) + 15) & ~(size_t)15;
  static constexpr size_t per_warp = region0 + compact + 16;
};

template <class SR>
__global__ void __launch_bounds__(NWARP_WPB * 32) k_num_warp(NumArgs a) {
  using T = typename SR::val_t;
  using L = WarpNumSmem<T>;
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
                                               SR::has_val ? Cv + cb : nullptr, a.err, NWARP_CAP, a.A.dbg);
    __syncwarp();
  }
}

// ---------------------------------------------------- mid / large / heavy
constexpr int NCH = 1024;  // A entries per expansion round

template <typename T, int SLOTS, int CAP> struct CtaNumLayout {
  static constexpr size_t table_bytes = (size_t)SLOTS * (4 + vbytes<T>());
  static constexpr size_t work_bytes =
      ((((size_t)(CAP + 2 * CAP) * 4 + 7) & ~(size_t)7)) + (size_t)CAP * vbytes<T>();
  static constexpr size_t region0 = ((table_bytes > work_bytes ? table_bytes : work_bytes) + 15) & ~(size_t)15;
  static constexpr size_t compact = (((size_t)CAP * (4 + vbytes<T>())) + 15) & ~(size_t)15;
  static constexpr size_t ex_off = region0 + compact;
  static constexpr size_t tail_off = ex_off + ((sizeof(CtaExpandSmem<T, NCH>) + 15) & ~(size_t)15);
  struct Tail {
    EmitScratch es;
    int wtmp[33];
    int row;
    int part_end;
    int part_cnt;
  };
  static constexpr size_t bytes = tail_off + sizeof(Tail);
};

template <class SR, int SLOTS, int CAP, bool PARTS>
__global__ void __launch_bounds__(PARTS || CAP > 2048 ? 1024 : 256) k_num_cta(NumArgs a) {
  using T = typename SR::val_t;
  using L = CtaNumLayout<T, SLOTS, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int *keys = reinterpret_cast<int *>(smem_raw);
  T *vals = reinterpret_cast<T *>(smem_raw + (size_t)SLOTS * 4);
  int *ck = reinterpret_cast<int *>(smem_raw + L::region0);
  T *cv = reinterpret_cast<T *>(smem_raw + L::region0 + (size_t)CAP * 4);
  auto &ex = *reinterpret_cast<CtaExpandSmem<T, NCH> *>(smem_raw + L::ex_off);
  auto &tl = *reinterpret_cast<typename L::Tail *>(smem_raw + L::tail_off);
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  T *Cv = reinterpret_cast<T *>(a.Cv);
  const int64_t n = a.B.n;

  // one part: columns [lo, hi) of row r holding pc outputs, written at out
  auto run_part = [&](int r, bool restrict_cols, int lo, int hi, int pc, int64_t out) {
    const int slots = max(64, min(SLOTS, next_pow2(2 * min(pc, CAP))));
    const unsigned mask = slots - 1;
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      keys[s] = EMPTY;
      if constexpr (SR::has_val) vals[s] = SR::identity();
    }
    __syncthreads();
    cta_products<SR, NCH>(A, B, A.p[r], A.p[r + 1], restrict_cols, lo, hi, ex, tl.wtmp,
                          [&](int col, T v, int) { hash_insert_val<SR>(keys, vals, mask, col, v, a.err); });
    group_sort_emit<CtaGroup, T, SR::has_val>(keys, vals, slots, pc, ck, cv, smem_raw, tl.wtmp, &tl.es,
                                              a.Cj + out, SR::has_val ? Cv + out : nullptr, a.err, CAP, a.A.dbg);
  };

  if constexpr (!PARTS) {
    for (int idx = blockIdx.x; idx < a.count; idx += gridDim.x) {
      const int r = a.list[idx];
      if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 36, r)) continue;  // uniform: every thread skips
      const int64_t o = nout_row(a.A, r);
      const int64_t cb = a.Cp[o];
      const int c = (int)(a.Cp[o + 1] - cb);
      run_part(r, false, 0, 0, c, cb);
      __syncthreads();
    }
  } else {
    const int nseg = (int)((n + SEG_W - 1) / SEG_W);
    while (true) {
      if (threadIdx.x == 0) tl.row = atomicAdd(a.dyn, 1);
      __syncthreads();
      const int idx = tl.row;
      if (idx >= a.count) break;
      const int r0 = a.list[idx];
      // a bad row id (guarded builds) is processed as an empty row so that the
      // loop still reaches its closing barrier
      const bool r_ok = HS_G(a.A.dbg, r0 >= 0 && r0 < a.A.nslots, 36, r0);
      const int r = r_ok ? r0 : 0;
      const int64_t o = nout_row(a.A, r);
      const int64_t cb = a.Cp[o];
      const int64_t c = r_ok ? a.Cp[o + 1] - cb : 0;
      const int h = r_ok ? a.hslot[r] : -1;
      const uint32_t *hist = a.hist + (int64_t)(h < 0 ? 0 : h) * a.nseg;
      if (r_ok && h < 0 && threadIdx.x == 0) atomicExch(a.err, 4);
      int64_t done = 0;
      int seg = 0;
      while (seg < nseg && h >= 0) {
        if (threadIdx.x == 0) {
          // greedy: extend the part while it stays within CAP outputs
          int e = seg, sum = 0;
          while (e < nseg && sum + (int)hist[e] <= CAP) sum += (int)hist[e++];
          if (e == seg) {  // a single over-full segment cannot happen (SEG_W <= CAP)
            atomicExch(a.err, 5);
            e = nseg;
          }
          tl.part_end = e;
          tl.part_cnt = sum;
        }
        __syncthreads();
        const int pe = tl.part_end, pc = tl.part_cnt;
        if (pc > 0) {
          const int lo = seg * SEG_W;
          const int hi = (int)min((int64_t)pe * SEG_W, n);
          run_part(r, true, lo, hi, pc, cb + done);
          done += pc;
        }
        seg = pe;
        __syncthreads();
      }
      if (threadIdx.x == 0 && done != c) atomicExch(a.err, 6);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------ launchers
inline int ngrid_cap(int items, int per_block, int per_sm) {
  int g = (items + per_block - 1) / per_block;
  int cap = sm_count() * per_sm;
  return g < cap ? (g < 1 ? 1 : g) : cap;
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
    case 1: {
      const size_t bytes = WarpNumSmem<T>::per_warp * NWARP_WPB;
      set_smem_attr(k_num_warp<SR>, bytes);
      count_launch();
      k_num_warp<SR><<<ngrid_cap(a.count, NWARP_WPB, 3), NWARP_WPB * 32, bytes, st>>>(a);
      break;
    }
    case 2: {
      using L = CtaNumLayout<T, 2 * CAP_MID, CAP_MID>;
      set_smem_attr(k_num_cta<SR, 2 * CAP_MID, CAP_MID, false>, L::bytes);
      count_launch();
      k_num_cta<SR, 2 * CAP_MID, CAP_MID, false><<<ngrid_cap(a.count, 1, 3), 256, L::bytes, st>>>(a);
      break;
    }
    case 3: {
      using L = CtaNumLayout<T, 2 * CAPL, CAPL>;
      set_smem_attr(k_num_cta<SR, 2 * CAPL, CAPL, false>, L::bytes);
      count_launch();
      k_num_cta<SR, 2 * CAPL, CAPL, false><<<ngrid_cap(a.count, 1, 1), 1024, L::bytes, st>>>(a);
      break;
    }
    case 4: {
      using L = CtaNumLayout<T, 2 * CAPL, CAPL>;
      set_smem_attr(k_num_cta<SR, 2 * CAPL, CAPL, true>, L::bytes);
      count_launch();
      k_num_cta<SR, 2 * CAPL, CAPL, true><<<ngrid_cap(a.count, 1, 1), 1024, L::bytes, st>>>(a);
      break;
    }
  }
}

}  // namespace hs
