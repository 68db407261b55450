// batch_persist.cu -- many independent products C_i = A_i * B_i in one
// persistent launch (hs_batch_plan_*).
//
// The problems are stacked once, at plan creation, into one block-diagonal
// product (hs_batch_stack), and C is allocated there with room for the flop
// bound sum_r min(f_r, n) (one host synchronisation, at creation only).  Each
// execution is then one memset of the work counters and one cooperative
// kernel whose CTAs stay resident and pull their work from atomic counters,
// the phases separated by grid-wide barriers (bounded waits):
//   1. products per row f_r (Algorithm 1's row-wise work), and the rows'
//      tiers: f_r <= 1024 to a warp (256 when a problem has 2^22 columns or
//      more), larger rows to the whole CTA;
//   2. distinct columns per row (the occupancy half of Figure 1's sparse
//      accumulator, as a shared hash set: a warp's 2048 slots, or the CTA's
//      8192), a CTA row's outputs also counted in 16 column buckets when they
//      exceed one CTA table (2048 values);
//   3. the row counts scanned into C's row offsets (each CTA scans a block of
//      rows, then adds the totals of the blocks before it);
//   4. the values, written in ascending column order at the row's offset: a
//      warp row by sorting its products (128, 256, 512 or 1024 keys) in the warp's
//      registers and folding equal columns (sort_row), a CTA row in a shared hash table of keys and
//      values (with more than 2048 outputs column range by column range,
//      ranges cut from its buckets).
// No allocation and no host synchronisation happen in an execution, so it
// can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/hspgemm.h"
#include "internal.h"
#include "numeric.cuh"

namespace hs {

constexpr int BP_NT = 256, BP_NW = BP_NT / 32;
constexpr int BPW_SYM = 2048;                    // warp tier symbolic set: f <= 1024
constexpr int BPW_FS = 256, BPW_F = 1024;        // warp tier values: 32*K sorted products, K = 4 .. 32
constexpr int BPW_G = 4;                         // warp groups: rows of at most 128, 256, 512, 1024 products
constexpr int BPC_SYM = 8192;                    // CTA tier symbolic set: f <= 4096
constexpr int BPC_SLOTS = 4096, BPC_CAP = 1536;  // CTA tier values: at most 1536 per column range
constexpr int BP_FMAX = 4096;                    // rows with more products are not taken
constexpr int BP_NBUCK = 16;                     // column buckets of a row with more than BPC_CAP outputs
constexpr int BP_REC = BP_NBUCK + 2;             // a bucket record: the counts, then the row's least and greatest column
constexpr int BP_CH = 256;                       // A entries staged per round (CTA tier)
constexpr int BP_CLAIM = 4;                      // warp rows a warp claims per atomic

// counters, zeroed before every execution
struct BpCounters {
  unsigned bar[2];  // grid barrier: arrivals, generation
  int nwarp[BPW_G], ncta;  // rows of each tier (warp rows by the keys they sort: 128 .. 1024)
  int sym_w, sym_c, num_w[BPW_G], num_c;  // work handed out per phase and tier
  int nbig;                         // CTA rows that need column ranges
  int err;   // bit 0: a row outside the tiers; 1: a barrier wait expired; 2: a column range too full
  int kerr;  // consistency codes of the row routines (hash table full, count mismatch)
  int pad[4];
  unsigned long long tns[6];  // global timer: start, after phases 1, 2, 3 (CTA 0), -, last CTA's exit
};

__device__ __forceinline__ unsigned long long bp_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// CTA 0 stamps phase boundaries (profiling only: the host reads them with
// hs_batch_plan_phase_ms)
__device__ __forceinline__ void bp_stamp(BpCounters *c, int i) {
  if (blockIdx.x == 0 && threadIdx.x == 0) c->tns[i] = bp_now();
}

struct BpArgs {
  RowSet A;
  RightOp B;
  int64_t m;           // stacked rows
  int32_t *wlist[BPW_G];  // warp-tier rows of at most 128, 256, 512 and wf_max products
  int wf_max;          // products of a warp-tier row at most (BPW_F, or BPW_FS for very wide problems)
  int32_t *clist;      // CTA-tier rows
  int32_t *fw;         // products per row (phase 1), read by the later phases
  int32_t *cbig;       // per CTA-tier row: its bucket record, or -1
  int32_t *buckets;    // BP_REC ints per CTA row with more than BPC_CAP outputs
  void *wscratch;      // per warp: the values of its row's products (BPW_F of them), in global memory
  int nbig_cap;        // records available
  int64_t *Cp;         // m + 1 row offsets (counts first)
  int32_t *Cj;
  void *Cv;
  int64_t cap;         // entries C's arrays hold
  int64_t *blk;        // per-CTA row-block totals
  BpCounters *ctr;
  long long spin_limit;
};

// bytes of a warp's shared region: its symbolic set, or its sort keys (the
// products' values wait in global scratch, which keeps the region small and
// three CTAs on an SM)
template <typename T> __host__ __device__ constexpr size_t bp_warp_bytes() {
  return SortSmemLayout<T, BPW_F / 32>::col_bytes > (size_t)BPW_SYM * 4 ? SortSmemLayout<T, BPW_F / 32>::col_bytes
                                                                        : (size_t)BPW_SYM * 4;
}

// Grid-wide barrier for co-resident CTAs (cooperative launch): the last CTA to
// arrive opens the next generation.  Waits are bounded: a CTA that gives up
// records it and goes on (the host reports HS_ETIMEDOUT).
__device__ __forceinline__ void bp_grid_sync(BpCounters *c, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = c->bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(c->bar, 1u) == gridDim.x - 1) {
      atomicExch(c->bar, 0u);
      __threadfence();
      atomicAdd(c->bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > limit) {
          atomicOr(&c->err, 2);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// append `want` lanes' rows to a list with one atomic per warp
__device__ __forceinline__ void bp_append(bool want, int r, int *count, int32_t *list) {
  const unsigned m = __ballot_sync(FULL, want);
  if (!m) return;
  const int lane = lane_id();
  int base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(FULL, base, __ffs(m) - 1);
  if (want) list[base + __popc(m & ((1u << lane) - 1u))] = r;
}

template <class SR>
__global__ void __launch_bounds__(BP_NT, 3) k_batch_persist(BpArgs a) {
  using T = typename SR::val_t;
  using Struct = Semiring<OR_AND, NoVal>;
  using LC = CtaNumLayout<T, BPC_SLOTS, BPC_CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item, s_count, s_cnt_b[BP_NBUCK], s_wtmp[33], s_kmin, s_kmax;
  const DevCsr A = ndev_a(a.A), B = ndev_b(a.B);
  const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  BpCounters *ctr = a.ctr;
  long long *dbg = a.A.dbg;
  const int64_t n = a.B.n;

  bp_stamp(ctr, 0);
  // ---- 1. products per row, tiers
  for (int64_t r0 = (int64_t)blockIdx.x * BP_NT; r0 < a.m; r0 += (int64_t)gridDim.x * BP_NT) {
    const int64_t r = r0 + tid;
    int64_t fr = 0;
    if (r < a.m) {
      for (int64_t q = A.p[r]; q < A.p[r + 1]; ++q) {
        if (!HS_G(dbg, q >= 0 && q < A.nnz, 50, q)) break;
        const int k = __ldg(A.j + q);
        if (HS_G(dbg, k >= 0 && k < B.rows, 51, k)) fr += __ldg(B.p + k + 1) - __ldg(B.p + k);
      }
      a.Cp[r + 1] = 0;
      a.fw[r] = (int32_t)(fr < 0x7fffffff ? fr : 0x7fffffff);
      if (fr > BP_FMAX) atomicOr(&ctr->err, 1);
    }
    bp_append(r < a.m && fr > 0 && fr <= BPW_FS / 2, (int)r, &ctr->nwarp[0], a.wlist[0]);
    bp_append(r < a.m && fr > BPW_FS / 2 && fr <= BPW_FS, (int)r, &ctr->nwarp[1], a.wlist[1]);
    bp_append(r < a.m && fr > BPW_FS && fr <= 2 * BPW_FS && fr <= a.wf_max, (int)r, &ctr->nwarp[2], a.wlist[2]);
    bp_append(r < a.m && fr > 2 * BPW_FS && fr <= a.wf_max, (int)r, &ctr->nwarp[3], a.wlist[3]);
    bp_append(r < a.m && fr > a.wf_max && fr <= BP_FMAX, (int)r, &ctr->ncta, a.clist);
  }
  if (blockIdx.x == 0 && tid == 0) a.Cp[0] = 0;
  bp_grid_sync(ctr, a.spin_limit);
  bp_stamp(ctr, 1);
  int nw_pre[BPW_G + 1];  // exclusive prefix of the warp groups' sizes
  nw_pre[0] = 0;
#pragma unroll
  for (int g = 0; g < BPW_G; ++g) nw_pre[g + 1] = nw_pre[g] + *(volatile int *)&ctr->nwarp[g];
  const int nw_rows = nw_pre[BPW_G], nc_rows = *(volatile int *)&ctr->ncta;

  // ---- 2. distinct columns per row
  {
    int *ckeys = reinterpret_cast<int *>(smem_raw);  // CTA set
    auto &cex = *reinterpret_cast<CtaExpandSmem<NoVal, BP_CH> *>(smem_raw + BPC_SYM * 4);
    while (true) {
      if (tid == 0) s_item = atomicAdd(&ctr->sym_c, 1);
      __syncthreads();
      const int i = s_item;
      if (i >= nc_rows) break;
      const int r = a.clist[i];
      const int cslots = max(64, min(BPC_SYM, next_pow2(2 * a.fw[r])));  // load at most one half
      for (int s = tid; s < cslots; s += BP_NT) ckeys[s] = EMPTY;
      if (tid < BP_NBUCK) s_cnt_b[tid] = 0;
      if (tid == 0) {
        s_count = 0;
        s_kmin = 0x7fffffff;
        s_kmax = -1;
      }
      __syncthreads();
      {  // the row's column range: first and last column of each of its B rows
        int lmin = 0x7fffffff, lmax = -1;
        for (int64_t q = A.p[r] + tid; q < A.p[r + 1]; q += BP_NT) {
          const int k = __ldg(A.j + q);
          if (!HS_G(dbg, k >= 0 && k < B.rows, 51, k)) continue;
          const int64_t b0 = __ldg(B.p + k), b1 = __ldg(B.p + k + 1);
          if (b0 < b1) {
            lmin = min(lmin, __ldg(B.j + b0));
            lmax = max(lmax, __ldg(B.j + b1 - 1));
          }
        }
        lmin = warp_min(lmin);
        lmax = warp_max(lmax);
        if (lane == 0) {
          atomicMin(&s_kmin, lmin);
          atomicMax(&s_kmax, lmax);
        }
      }
      __syncthreads();
      const int kmin = s_kmin;
      const int64_t span = (int64_t)s_kmax - kmin + 1;
      int cnt = 0;
      cta_products<Struct, BP_CH>(A, B, A.p[r], A.p[r + 1], false, 0, 0, cex, s_wtmp, [&](int col, NoVal, int) {
        if (hash_insert_key(ckeys, cslots - 1, col)) {
          ++cnt;
          const int bkt = (int)(((int64_t)(col - kmin) * BP_NBUCK) / span);
          if (HS_G(dbg, bkt >= 0 && bkt < BP_NBUCK, 82, col)) atomicAdd(&s_cnt_b[bkt], 1);
        }
      });
      cnt = warp_sum(cnt);
      if (lane == 0 && cnt) atomicAdd(&s_count, cnt);
      __syncthreads();
      if (tid == 0) {
        a.Cp[r + 1] = s_count;
        int rec = -1;
        if (s_count > BPC_CAP) {  // its values need column ranges: keep its buckets
          rec = atomicAdd(&ctr->nbig, 1);
          if (rec < a.nbig_cap) {
            int32_t *rb = a.buckets + (int64_t)rec * BP_REC;
            for (int b = 0; b < BP_NBUCK; ++b) rb[b] = s_cnt_b[b];
            rb[BP_NBUCK] = s_kmin;
            rb[BP_NBUCK + 1] = s_kmax;
          } else {
            atomicOr(&ctr->err, 4);
            rec = -1;
          }
        }
        a.cbig[i] = rec;
      }
      __syncthreads();
    }
    int *wkeys = reinterpret_cast<int *>(smem_raw + (size_t)warp * bp_warp_bytes<T>());  // a warp's set
    for (int i = 0, iend = 0;; ++i) {
      if (i >= iend) {
        int i0 = 0;
        if (lane == 0) i0 = atomicAdd(&ctr->sym_w, BP_CLAIM);
        i = __shfl_sync(FULL, i0, 0);
        iend = min(i + BP_CLAIM, nw_rows);
        if (i >= iend) break;
      }
      const int32_t *wl = a.wlist[0];
      int off = 0;
#pragma unroll
      for (int t = 1; t < BPW_G; ++t)
        if (i >= nw_pre[t]) {  // (unrolled: the prefix stays in registers)
          wl = a.wlist[t];
          off = nw_pre[t];
        }
      const int r = wl[i - off];
      const int slots = max(64, min(BPW_SYM, next_pow2(2 * a.fw[r])));  // load at most one half
      for (int s = lane; s < slots; s += 32) wkeys[s] = EMPTY;
      __syncwarp();
      int cnt = 0;
      warp_products<Struct>(A, B, A.p[r], A.p[r + 1],
                            [&](int col, NoVal, int) { cnt += hash_insert_key(wkeys, slots - 1, col); });
      cnt = warp_sum(cnt);
      if (lane == 0) a.Cp[r + 1] = cnt;
      __syncwarp();
    }
  }
  bp_grid_sync(ctr, a.spin_limit);
  bp_stamp(ctr, 2);

  // ---- 3. row offsets: block b of rows is scanned by CTA b, after the totals of the blocks before it
  {
    const int64_t per = (a.m + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = min(a.m, (int64_t)blockIdx.x * per), b1 = min(a.m, b0 + per);
    long long s = 0;
    for (int64_t r = b0 + tid; r < b1; r += BP_NT) s += a.Cp[r + 1];
    s = warp_sum(s);
    __shared__ long long s_sum[BP_NW];
    if (lane == 0) s_sum[warp] = s;
    __syncthreads();
    if (tid == 0) {
      long long t = 0;
      for (int w = 0; w < BP_NW; ++w) t += s_sum[w];
      a.blk[blockIdx.x] = t;
    }
    bp_grid_sync(ctr, a.spin_limit);
    __shared__ long long s_off;
    if (tid == 0) {
      long long o = 0;
      for (int b = 0; b < (int)blockIdx.x; ++b) o += a.blk[b];
      s_off = o;
    }
    __syncthreads();
    long long run = s_off;
    for (int64_t c0 = b0; c0 < b1; c0 += BP_NT) {
      const int64_t r = c0 + tid;
      const long long v = r < b1 ? a.Cp[r + 1] : 0;
      long long incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long u = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += u;
      }
      if (lane == 31) s_sum[warp] = incl;
      __syncthreads();
      long long before = 0, all = 0;
      for (int w = 0; w < BP_NW; ++w) {
        before += w < warp ? s_sum[w] : 0;
        all += s_sum[w];
      }
      if (r < b1) a.Cp[r + 1] = run + before + incl;
      run += all;
      __syncthreads();
    }
  }
  bp_grid_sync(ctr, a.spin_limit);
  bp_stamp(ctr, 3);

  // ---- 4. values, in ascending column order at the row offsets
  T *Cv = reinterpret_cast<T *>(a.Cv);
  {
    auto &tl = *reinterpret_cast<typename LC::Tail *>(smem_raw + LC::tail_off);
    int *keys = reinterpret_cast<int *>(smem_raw);
    T *vals = reinterpret_cast<T *>(smem_raw + (size_t)BPC_SLOTS * 4);
    int *ck = reinterpret_cast<int *>(smem_raw + LC::region0);
    T *cv = reinterpret_cast<T *>(smem_raw + LC::region0 + (size_t)BPC_CAP * 4);
    auto &ex = *reinterpret_cast<CtaExpandSmem<T, nch<BPC_CAP>()> *>(smem_raw + LC::ex_off);
    while (true) {
      if (tid == 0) s_item = atomicAdd(&ctr->num_c, 1);
      __syncthreads();
      const int i = s_item;
      if (i >= nc_rows) break;
      const int r = a.clist[i];
      const int64_t cb = a.Cp[r];
      const int c = (int)(a.Cp[r + 1] - cb);
      const int rec = a.cbig[i];
      // column ranges of at most BPC_CAP outputs, cut at bucket boundaries
      int done = 0, bk = 0;
      while (done < c) {
        int lo = 0, hi = (int)n, part = c;
        if (rec >= 0) {  // bucket b holds columns kmin + [ceil(b*span/16), ceil((b+1)*span/16))
          const int32_t *bc = a.buckets + (int64_t)rec * BP_REC;
          const int rkmin = bc[BP_NBUCK];
          const int64_t rspan = (int64_t)bc[BP_NBUCK + 1] - rkmin + 1;
          const int b0 = bk;
          part = 0;
          while (bk < BP_NBUCK && part + bc[bk] <= BPC_CAP) part += bc[bk++];
          if (bk == b0) {  // one bucket alone is too full: the row cannot be taken
            if (tid == 0) atomicOr(&ctr->err, 4);
            break;
          }
          lo = rkmin + (int)(((int64_t)b0 * rspan + BP_NBUCK - 1) / BP_NBUCK);
          hi = rkmin + (int)(((int64_t)bk * rspan + BP_NBUCK - 1) / BP_NBUCK);
        } else if (!HS_G(dbg, c <= BPC_CAP, 80, c)) {
          break;
        }
        const int slots = max(64, min(BPC_SLOTS, next_pow2(2 * max(part, 1))));
        const unsigned mask = slots - 1;
        for (int s = tid; s < slots; s += BP_NT) {
          keys[s] = EMPTY;
          if constexpr (SR::has_val) vals[s] = SR::identity();
        }
        __syncthreads();
        cta_products<SR, nch<BPC_CAP>()>(A, B, A.p[r], A.p[r + 1], rec >= 0, lo, hi, ex, tl.wtmp,
                                         [&](int col, T v, int) { hash_insert_val<SR>(keys, vals, mask, col, v, &ctr->kerr); });
        if (HS_G(dbg, cb + done + part <= a.cap, 81, cb + done + part))
          group_sort_emit<CtaGroup, T, SR::has_val>(keys, vals, slots, part, ck, cv, smem_raw, tl.wtmp, &tl.es,
                                                    a.Cj + cb + done, SR::has_val ? Cv + cb + done : nullptr,
                                                    &ctr->kerr, BPC_CAP, dbg);
        __syncthreads();
        done += part;
      }
      __syncthreads();
    }
    unsigned char *wb = smem_raw + (size_t)warp * bp_warp_bytes<T>();
    int *s_col = reinterpret_cast<int *>(wb);
    T *s_val = reinterpret_cast<T *>(a.wscratch) + ((size_t)blockIdx.x * BP_NW + warp) * BPW_F;
    // rows of 1024, then 512, then 256 keys: the warps of an SM mostly run the
    // same width at a time, and the expansion has one call site for all three
    int g = BPW_G - 1, i = 0, iend = 0;  // rows [i, iend) of group g claimed by this warp
    while (g >= 0) {
      if (i >= iend) {
        int i0 = 0;
        if (lane == 0) i0 = atomicAdd(&ctr->num_w[g], BP_CLAIM);
        i = __shfl_sync(FULL, i0, 0);
        iend = min(i + BP_CLAIM, *(volatile int *)&ctr->nwarp[g]);
        if (i >= iend) {
          --g;
          continue;
        }
      }
      const int r = a.wlist[g][i++];
      const int64_t cb = a.Cp[r];
      const int c = (int)(a.Cp[r + 1] - cb);
      const int fr = a.fw[r];
      int kmn = 0, kmx = 0;
      const int got = sort_expand<SR>(A, B, A.p[r], A.p[r + 1], BPW_F, s_col, s_val, &kmn, &kmx);
      if (got != fr || fr > ((BPW_FS / 2) << g)) {
        if (lane == 0) atomicExch(&ctr->kerr, 12);
      } else if (HS_G(dbg, cb + c <= a.cap, 81, cb + c)) {
        T *out_v = SR::has_val ? Cv + cb : nullptr;
        if (g == 0)
          sort_finish<SR, BPW_FS / 64, true>(fr, c, kmn, kmx, s_col, s_val, a.Cj + cb, out_v, &ctr->kerr, dbg);
        else if (g == 1)
          sort_finish<SR, BPW_FS / 32, true>(fr, c, kmn, kmx, s_col, s_val, a.Cj + cb, out_v, &ctr->kerr, dbg);
        else if (g == 2)
          sort_finish<SR, 2 * BPW_FS / 32, false>(fr, c, kmn, kmx, s_col, s_val, a.Cj + cb, out_v, &ctr->kerr, dbg);
        else
          sort_finish<SR, BPW_F / 32, false>(fr, c, kmn, kmx, s_col, s_val, a.Cj + cb, out_v, &ctr->kerr, dbg);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&ctr->tns[5], bp_now());
}

template <class SR> size_t bp_smem() {
  using T = typename SR::val_t;
  const size_t w = (size_t)BP_NW * bp_warp_bytes<T>();
  const size_t c = CtaNumLayout<T, BPC_SLOTS, BPC_CAP>::bytes;
  const size_t s = (size_t)BPC_SYM * 4 + sizeof(CtaExpandSmem<NoVal, BP_CH>);
  return std::max(w, std::max(c, s));
}

template <class SR> static int bp_launch(BpArgs &a, int grid, cudaStream_t st) {
  auto k = k_batch_persist<SR>;
  set_smem_attr(k, bp_smem<SR>());
  count_launch();
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(BP_NT);
  cfg.dynamicSmemBytes = bp_smem<SR>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a) == cudaSuccess ? HS_OK : HS_ECUDA;
}

template <class SR> static int bp_grid() {
  int per = 0;
  auto k = k_batch_persist<SR>;
  set_smem_attr(k, bp_smem<SR>());
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BP_NT, bp_smem<SR>()) != cudaSuccess || per < 1) {
    cudaGetLastError();
    return 0;
  }
  return per * sm_count();
}

// (semiring, value type) of a plan: the semirings hs_spgemm computes with values
enum BpKind { BP_PT64, BP_PT32, BP_PTI64, BP_MP32, BP_MPI32, BP_OA };

static int bp_dispatch(int kind, BpArgs *a, int grid, cudaStream_t st, bool launch) {
  switch (kind) {
    case BP_PT64: return launch ? bp_launch<Semiring<PLUS_TIMES, double>>(*a, grid, st) : bp_grid<Semiring<PLUS_TIMES, double>>();
    case BP_PT32: return launch ? bp_launch<Semiring<PLUS_TIMES, float>>(*a, grid, st) : bp_grid<Semiring<PLUS_TIMES, float>>();
    case BP_PTI64: return launch ? bp_launch<Semiring<PLUS_TIMES, int64_t>>(*a, grid, st) : bp_grid<Semiring<PLUS_TIMES, int64_t>>();
    case BP_MP32: return launch ? bp_launch<Semiring<MIN_PLUS, float>>(*a, grid, st) : bp_grid<Semiring<MIN_PLUS, float>>();
    case BP_MPI32: return launch ? bp_launch<Semiring<MIN_PLUS, int32_t>>(*a, grid, st) : bp_grid<Semiring<MIN_PLUS, int32_t>>();
    case BP_OA: return launch ? bp_launch<Semiring<OR_AND, NoVal>>(*a, grid, st) : bp_grid<Semiring<OR_AND, NoVal>>();
  }
  return launch ? HS_EINVAL : 0;
}

// products per row of the stacked A, their bounded sum and maximum (plan creation)
__global__ void k_bp_bound(RowSet A, RightOp B, int64_t m, unsigned long long *stats) {
  unsigned long long sb = 0, mx = 0, big = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t fr = 0;
    for (int64_t q = A.p[r]; q < A.p[r + 1]; ++q) {
      if (!HS_G(A.dbg, q >= 0 && q < A.nnz, 50, q)) break;
      const int k = A.j[q];
      if (HS_G(A.dbg, k >= 0 && k < B.m, 51, k)) fr += B.p[k + 1] - B.p[k];
    }
    sb += (unsigned long long)min(fr, B.n);
    mx = max(mx, (unsigned long long)fr);
    big += fr > BPC_CAP ? 1 : 0;  // rows that may need column ranges (a bucket record each)
  }
  sb = warp_sum(sb);
  mx = warp_max(mx);
  big = warp_sum(big);
  if (lane_id() == 0) {
    atomicAdd(stats, sb);
    atomicMax(stats + 1, mx);
    atomicAdd(stats + 2, big);
  }
}

}  // namespace hs

using namespace hs;

struct hs_batch_plan {
  int kind = 0, dtype = 0, vb = 0, grid = 0;
  int64_t count = 0, m = 0, cap = 0;
  hs_mat SA{}, SB{};
  std::vector<int64_t> row_offsets;
  const hs_allocator *al = nullptr;
  struct Blk {
    void *p;
    size_t n;
  };
  std::vector<Blk> blocks;
  BpArgs args{};
  long long *dbg = nullptr;
};

static void *bp_alloc(hs_batch_plan *P, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (P->al && P->al->alloc) p = P->al->alloc(bytes, (void *)st, P->al->ctx);
  else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) P->blocks.push_back({p, bytes});
  return p;
}

extern "C" void hs_batch_plan_destroy(hs_batch_plan *P, void *stream) {
  if (!P) return;
  cudaStream_t st = (cudaStream_t)stream;
  for (auto &b : P->blocks) {
    if (P->al && P->al->free) P->al->free(b.p, b.n, stream, P->al->ctx);
    else if (!P->al || !P->al->alloc) cudaFreeAsync(b.p, st);
  }
  hs_mat_free(&P->SA, P->al, stream);
  hs_mat_free(&P->SB, P->al, stream);
  delete P;
}

extern "C" int hs_batch_plan_create(int semiring, int64_t count, const hs_mat *A, const hs_mat *B,
                                    hs_batch_plan **plan, const hs_allocator *al, void *stream, uint32_t) {
  if (!plan) return HS_EINVAL;
  *plan = nullptr;
  if (count < 0 || (count > 0 && (!A || !B))) return HS_EINVAL;
  const int adt = count ? A[0].dtype : HS_F64, bdt = count ? B[0].dtype : HS_F64;
  int kind = -1, odt = adt;
  if (semiring == HS_PLUS_TIMES && adt == bdt)
    kind = adt == HS_F64 ? BP_PT64 : adt == HS_F32 ? BP_PT32 : adt == HS_I64 ? BP_PTI64 : -1;
  else if (semiring == HS_MIN_PLUS && adt == bdt)
    kind = adt == HS_F32 ? BP_MP32 : adt == HS_I32 ? BP_MPI32 : -1;
  else if (semiring == HS_OR_AND) {
    kind = BP_OA;
    odt = HS_BOOL;
  }
  if (kind < 0) return HS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  auto *P = new hs_batch_plan();
  P->kind = kind;
  P->dtype = odt;
  P->vb = odt == HS_F64 || odt == HS_I64 ? 8 : (odt == HS_BOOL ? 0 : 4);
  P->count = count;
  P->al = al;
  P->row_offsets.assign((size_t)count + 1, 0);
  int e = hs_batch_stack(count, A, B, &P->SA, &P->SB, P->row_offsets.data(), al, stream);
  if (e != HS_OK) {
    hs_batch_plan_destroy(P, stream);
    return e;
  }
  P->m = P->SA.m;
  const int64_t m = P->m;
  // the flop bound of C, the largest row and the rows that may need column ranges, once
  unsigned long long *stats = (unsigned long long *)bp_alloc(P, 16 + 16, st);
  long long *dbg = (long long *)bp_alloc(P, 16, st);
  unsigned long long *h = nullptr;
  if (!stats || !dbg || cudaMallocHost(&h, 32) != cudaSuccess) {
    cudaGetLastError();
    hs_batch_plan_destroy(P, stream);
    return HS_ENOMEM;
  }
  cudaMemsetAsync(stats, 0, 24, st);
  cudaMemsetAsync(dbg, 0, 16, st);
  P->dbg = dbg;
  RowSet rs{P->SA.ptr, P->SA.idx, P->SA.val, nullptr, m, P->SA.nnz, m, dbg};
  RightOp rb{P->SB.ptr, P->SB.idx, P->SB.val, P->SB.n, P->SB.m, P->SB.nnz, dbg};
  if (m > 0) {
    count_launch();
    int64_t g = (m + 255) / 256, gc = (int64_t)sm_count() * 8;
    k_bp_bound<<<(int)(g < gc ? g : gc), 256, 0, st>>>(rs, rb, m, stats);
  }
  cudaMemcpyAsync(h, stats, 24, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    hs_batch_plan_destroy(P, stream);
    return HS_ECUDA;
  }
  const unsigned long long bound = h[0], fmax = h[1], nbig = h[2];
  cudaFreeHost(h);
  if (fmax > (unsigned long long)BP_FMAX || m > 0x7fffffffLL) {  // rows this kernel does not take
    hs_batch_plan_destroy(P, stream);
    return HS_EUNSUPPORTED;
  }
  P->grid = bp_dispatch(kind, nullptr, 0, st, false);
  if (P->grid <= 0) {
    hs_batch_plan_destroy(P, stream);
    return HS_ECUDA;
  }
  P->cap = (int64_t)bound;
  const int nbig_cap = nbig < 1 ? 1 : (nbig > 0x7fffffffULL ? 0x7fffffff : (int)nbig);
  BpArgs &a = P->args;
  a.A = rs;
  a.B = rb;
  a.m = m;
  // the sorted warp rows pack (column - the row's least column) into 32-bit
  // keys with 10 bits of product index: problems of 2^22 columns or more
  // send rows above 256 products to the CTA tier
  int64_t nmax = 0;
  for (int64_t i = 0; i < count; ++i) nmax = B[i].n > nmax ? B[i].n : nmax;
  a.wf_max = nmax >= SORT_PACKED_COLS ? BPW_FS : BPW_F;
  a.wlist[0] = (int32_t *)bp_alloc(P, 4 * (size_t)BPW_G * (size_t)(m > 0 ? m : 1), st);
  for (int g = 1; g < BPW_G; ++g) a.wlist[g] = a.wlist[0] ? a.wlist[g - 1] + (m > 0 ? m : 1) : nullptr;
  a.clist = (int32_t *)bp_alloc(P, 4 * (size_t)(m > 0 ? m : 1), st);
  a.fw = (int32_t *)bp_alloc(P, 4 * (size_t)(m > 0 ? m : 1), st);
  a.cbig = (int32_t *)bp_alloc(P, 4 * (size_t)(m > 0 ? m : 1), st);
  a.buckets = (int32_t *)bp_alloc(P, 4 * (size_t)nbig_cap * BP_REC, st);
  a.wscratch = P->vb ? bp_alloc(P, (size_t)P->grid * BP_NW * BPW_F * (size_t)P->vb, st) : nullptr;
  a.nbig_cap = nbig_cap;
  a.Cp = (int64_t *)bp_alloc(P, 8 * (size_t)(m + 1), st);
  a.Cj = (int32_t *)bp_alloc(P, 4 * (size_t)(P->cap > 0 ? P->cap : 1), st);
  a.Cv = P->vb ? bp_alloc(P, (size_t)P->vb * (size_t)(P->cap > 0 ? P->cap : 1), st) : nullptr;
  a.cap = P->cap;
  a.blk = (int64_t *)bp_alloc(P, 8 * (size_t)P->grid, st);
  a.ctr = (BpCounters *)bp_alloc(P, sizeof(BpCounters), st);
  a.spin_limit = 1LL << 24;  // polls of a barrier word (64 ns naps): about a second
  if (!a.wlist[0] || !a.clist || !a.fw || !a.cbig || !a.buckets || !a.Cp || !a.Cj || (P->vb && (!a.Cv || !a.wscratch)) || !a.blk || !a.ctr) {
    hs_batch_plan_destroy(P, stream);
    return HS_ENOMEM;
  }
  *plan = P;
  return HS_OK;
}

extern "C" int hs_batch_plan_execute(hs_batch_plan *P, void *stream) {
  if (!P) return HS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(P->args.ctr, 0, sizeof(BpCounters), st) != cudaSuccess) {
    cudaGetLastError();
    return HS_ECUDA;
  }
  if (P->m == 0) return cudaMemsetAsync(P->args.Cp, 0, 8, st) == cudaSuccess ? HS_OK : HS_ECUDA;
  const int e = bp_dispatch(P->kind, &P->args, P->grid, st, true);
  if (e != HS_OK) cudaGetLastError();
  return e;
}

extern "C" int hs_batch_plan_phase_ms(hs_batch_plan *P, double *ms, void *stream) {
  if (!P || !ms) return HS_EINVAL;
  unsigned long long *h = nullptr;
  if (cudaMallocHost(&h, sizeof(unsigned long long) * 6) != cudaSuccess) {
    cudaGetLastError();
    return HS_ENOMEM;
  }
  cudaMemcpyAsync(h, P->args.ctr->tns, sizeof(unsigned long long) * 6, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  const cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
  if (ce == cudaSuccess) {
    auto span = [&](int a, int b) { return h[b] >= h[a] ? (double)(h[b] - h[a]) * 1e-6 : 0.0; };
    ms[0] = span(0, 1);  // products per row, tiers
    ms[1] = span(1, 2);  // distinct columns per row
    ms[2] = span(2, 3);  // row offsets
    ms[3] = span(3, 5);  // values
    ms[4] = span(0, 5);  // the whole execution
  }
  cudaFreeHost(h);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return HS_ECUDA;
  }
  return HS_OK;
}

extern "C" int hs_batch_plan_result(hs_batch_plan *P, hs_mat *C, int64_t *row_offsets, void *stream) {
  if (!P || !C) return HS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  long long *h = nullptr;
  if (cudaMallocHost(&h, 32) != cudaSuccess) {
    cudaGetLastError();
    return HS_ENOMEM;
  }
  cudaMemcpyAsync(h, P->args.Cp + P->m, 8, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(h + 1, &P->args.ctr->err, 8, cudaMemcpyDeviceToHost, st);  // err, kerr
  cudaMemcpyAsync(h + 2, P->dbg, 16, cudaMemcpyDeviceToHost, st);
  const cudaError_t ce = cudaStreamSynchronize(st);
  const long long nnz = h[0];
  const int err = (int)(h[1] & 0xffffffff), kerr = (int)(h[1] >> 32);
  const long long d0 = h[2];
  cudaFreeHost(h);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return HS_ECUDA;
  }
  if (err & 2) return HS_ETIMEDOUT;
  if (err & 5) return HS_EUNSUPPORTED;
  if (err || kerr || d0) return HS_EINTERNAL;
  if (nnz < 0 || nnz > P->cap) return HS_EINTERNAL;
  *C = hs_mat{HS_CSR, P->dtype, P->m, P->SB.n, nnz, 0, P->args.Cp, P->args.Cj, nullptr, P->args.Cv};
  if (row_offsets) memcpy(row_offsets, P->row_offsets.data(), sizeof(int64_t) * (size_t)(P->count + 1));
  return HS_OK;
}
