// symbolic.cu -- output nonzeros per row of C = A*B (structure only).
//
// The row-wise form of Algorithm 1 with the sparse accumulator of Figure 1
// reduced to its occupancy part: each row's distinct output columns are
// counted by the accumulator its bin selects.
//   tiny  (f <= 32)    one warp, one product per lane, equal columns found
//                      with __match_any_sync;
//   warp  (f <= 512)   one warp, private shared-memory hash set;
//   mid   (f <= 1024, and f <= 4096)
//                      one CTA, shared hash set of 2f slots (at most 2048,
//                      and 8192: the smaller tier keeps more CTAs per SM);
//   large (f <= min(16384, cap_large), so f <= 8192)
//                      one CTA, shared hash set of up to 16384 slots;
//   heavy (larger f)   one CTA, a bitmap over 2^20 columns (occupancy SPA in
//                      shared memory), rows handed out largest first.  The
//                      bitmap is read out in column order, so the kernel also
//                      writes the row's sorted column list for the numeric
//                      pass, which then only has to place values.
// Rows with more than cap_large products also get per-column-segment counts
// (4096-column segments) from which the numeric pass plans its column parts.
// Counts go to cnt[row + 1] so an inclusive scan turns them into row offsets.
#include "common.cuh"
#include "internal.h"

namespace hs {

using StructSR = Semiring<OR_AND, NoVal>;

__device__ __forceinline__ DevCsr dev_a(const RowSet &A) { return DevCsr{A.p, A.j, A.v, A.nslots, A.nnz, A.dbg}; }
__device__ __forceinline__ DevCsr dev_b(const RightOp &B) { return DevCsr{B.p, B.j, B.v, B.m, B.nnz, B.dbg}; }
// count of output row o goes to cnt[o + 1]
__device__ __forceinline__ void put_count(const SymArgs &a, int64_t o, int64_t v) {
  if (HS_G(a.A.dbg, o >= 0 && o < a.A.m, 30, o)) a.cnt[o + 1] = v;
}
__device__ __forceinline__ int64_t out_row(const RowSet &A, int r) { return A.ids ? (int64_t)A.ids[r] : (int64_t)r; }

// --------------------------------------------------------------- tiny
constexpr int TINY_WPB = 8;
__global__ void __launch_bounds__(TINY_WPB * 32, 4) k_sym_tiny(SymArgs a) {
  __shared__ int scol[TINY_WPB][32];
  const int w = threadIdx.x >> 5, lane = lane_id();
  const DevCsr A = dev_a(a.A), B = dev_b(a.B);
  for (int idx = blockIdx.x * TINY_WPB + w; idx < a.count; idx += gridDim.x * TINY_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int64_t q0 = A.p[r], q1 = A.p[r + 1];
    int nprod = 0;
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane;
      int64_t s = 0, e = 0;
      if (q < q1) entry_segment(A, B, q, false, 0, 0, s, e);
      auto put = [&](int col, NoVal, int p) {
        if (HS_G(a.A.dbg, nprod + p < 32, 34, nprod + p)) scol[w][nprod + p] = col;
      };
      nprod += warp_expand<StructSR>(B, s, (int)(e - s), NoVal{}, put);
    }
    __syncwarp();
    const bool have = lane < nprod && lane < 32;
    const int col = have ? scol[w][lane] : 0;
    const unsigned act = __ballot_sync(FULL, have);
    bool first = false;
    if (have) {
      const unsigned grp = __match_any_sync(act, col);
      first = lane == __ffs(grp) - 1;
    }
    const int cnt = __popc(__ballot_sync(FULL, first));
    if (lane == 0) {
      put_count(a, out_row(a.A, r), cnt);
      if (nprod > 32) atomicExch(a.err, 2);
    }
    __syncwarp();
  }
}

// --------------------------------------------------------------- warp
// one warp per row, a private table of 2f slots (at most SLOTS): rows of at
// most 512 products (1024 slots) and, in their own launch, of 513..1024
// products (2048 slots)
constexpr int WARP_WPB = 8;
template <int SLOTS>
__global__ void __launch_bounds__(WARP_WPB * 32, 4) k_sym_warp(SymArgs a) {
  extern __shared__ __align__(16) int tables[];
  const int w = threadIdx.x >> 5, lane = lane_id();
  int *keys = tables + w * SLOTS;
  const DevCsr A = dev_a(a.A), B = dev_b(a.B);
  for (int idx = blockIdx.x * WARP_WPB + w; idx < a.count; idx += gridDim.x * WARP_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int slots = max(64, min(SLOTS, next_pow2(2 * (int)a.f[r])));
    for (int s = lane; s < slots; s += 32) keys[s] = EMPTY;
    __syncwarp();
    int cnt = 0;
    const unsigned mask = slots - 1;
    warp_products<StructSR>(A, B, A.p[r], A.p[r + 1],
                            [&](int col, NoVal, int) { cnt += hash_insert_key(keys, mask, col); });
    cnt = warp_sum(cnt);
    if (lane == 0) put_count(a, out_row(a.A, r), cnt);
    __syncwarp();
  }
}

// ------------------------------------------------------------- dense SPA
// Products whose B has at most SPA_COLS_4 columns: one warp per row sets an
// occupancy flag per product (a byte per column of all n columns, plain
// stores: lanes that hit one column do not queue on an atomic) and counts
// the flags (the occupancy half of Figure 1's sparse accumulator).
constexpr int SPA_WPB = 8;
__global__ void __launch_bounds__(SPA_WPB * 32) k_sym_spa(SymArgs a) {
  __shared__ unsigned flags_all[SPA_WPB][SPA_COLS_4 / 4];
  const int w = threadIdx.x >> 5, lane = lane_id();
  unsigned *flag4 = flags_all[w];
  unsigned char *flag = reinterpret_cast<unsigned char *>(flag4);
  const DevCsr A = dev_a(a.A), B = dev_b(a.B);
  const int n = (int)a.B.n;
  const int fwords = (n + 3) >> 2;
  for (int i = lane; i < fwords; i += 32) flag4[i] = 0u;
  __syncwarp();
  for (int idx = blockIdx.x * SPA_WPB + w; idx < a.count; idx += gridDim.x * SPA_WPB) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    warp_products<StructSR>(A, B, A.p[r], A.p[r + 1], [&](int col, NoVal, int) {
      if (HS_G(a.A.dbg, col >= 0 && col < n, 84, col)) flag[col] = 1;
    });
    __syncwarp();
    int cnt = 0;
    for (int i = lane; i < fwords; i += 32) {
      cnt += __popc(flag4[i] & 0x01010101u);
      flag4[i] = 0u;
    }
    cnt = warp_sum(cnt);
    if (lane == 0) put_count(a, out_row(a.A, r), cnt);
    __syncwarp();
  }
}

// ----------------------------------------------------------- mid / large
constexpr int CH = 1024;   // A entries per expansion round (heavy)
constexpr int CHM = 256;   // the same for the hash kernels: smaller staging, more CTAs per SM

template <int SLOTS> struct SymCtaSmem {
  int keys[SLOTS];
  CtaExpandSmem<NoVal, CHM> ex;
  int wtmp[33];
  int total;
};

template <int SLOTS, int NT>
__global__ void __launch_bounds__(NT) k_sym_cta(SymArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &sm = *reinterpret_cast<SymCtaSmem<SLOTS> *>(smem_raw);
  const DevCsr A = dev_a(a.A), B = dev_b(a.B);
  for (int idx = blockIdx.x; idx < a.count; idx += gridDim.x) {
    const int r = a.list[idx];
    if (!HS_G(a.A.dbg, r >= 0 && r < a.A.nslots, 35, r)) continue;
    const int slots = max(64, min(SLOTS, next_pow2(2 * (int)a.f[r])));
    const unsigned mask = slots - 1;
    for (int s = threadIdx.x; s < slots; s += blockDim.x) sm.keys[s] = EMPTY;
    if (threadIdx.x == 0) sm.total = 0;
    __syncthreads();
    int cnt = 0;
    cta_products<StructSR, CHM>(A, B, A.p[r], A.p[r + 1], false, 0, 0, sm.ex, sm.wtmp,
                                [&](int col, NoVal, int) { cnt += hash_insert_key(sm.keys, mask, col); });
    cnt = warp_sum(cnt);
    if (lane_id() == 0 && cnt) atomicAdd(&sm.total, cnt);
    __syncthreads();
    if (threadIdx.x == 0) put_count(a, out_row(a.A, r), sm.total);
    __syncthreads();
  }
}

// --------------------------------------------------------------- heavy
// Per row and per chunk of 2^20 columns: the products set their bits (an OR
// whose old value nobody waits for), then each 4096-column segment's bits are
// counted by popcount.  The segment counts give the chunk's histogram and,
// scanned, each segment's place in the row's sorted column list.  Each warp then walks pairs of
// segments, every lane eight consecutive words: the lanes' bit counts are
// scanned across the warp, the columns go to a per-warp staging buffer in
// ascending order and leave it in coalesced stores.  A pair with more columns
// than the buffer holds is read again as eight steps of 1024 columns, lane l
// on the step's word l, so each step's columns also run in lane order and
// gather in the buffer (per-lane stores of the long runs measured 2.3 ms
// slower on R-MAT scale 20).
constexpr int SH_COLS = BITMAP_COLS;          // columns per chunk (one bitmap)
constexpr int SH_SEGS = SH_COLS / SEG_W;      // segments per chunk (256)
constexpr int SH_NT = 1024;                   // threads of the heavy symbolic CTA
constexpr int SH_WARPS = SH_NT / 32;
constexpr int SH_PPW = SH_SEGS / 2 / SH_WARPS;  // segment pairs per warp (4)
constexpr int SH_MINB = 1;                    // CTAs per SM the registers are sized for
static_assert(SH_PPW * SH_WARPS * 2 == SH_SEGS, "the warps' pairs cover a chunk's segments");
constexpr int SH_BUF = 384;                   // per-warp list staging entries
static_assert(SEG_W == 4096, "two segments are 256 words: eight per lane");

// Product visitor: sets the column's bit; the old word is not needed (the
// segment counts come from the finished bitmap), so no lane waits for it.
// (Reading the word first and skipping the atomic when the bit is already set
// measured slower on R-MAT scale 20: 27.7 against 24.3 ms.)
struct SymHeavyBit {
  unsigned *bitmap;
  int lo;
  unsigned span;
  long long *dbg;
  __device__ __forceinline__ void operator()(int col, NoVal, int) const {
    const unsigned x = (unsigned)(col - lo);
    if (HS_G(dbg, x < span, 33, col)) atomicOr(bitmap + (x >> 5), 1u << (x & 31));
  }
};

struct SymHeavySmem {
  CtaExpandSmem<NoVal, CH> ex;
  int wtmp[33];
  int row;
  long long loff;        // the row's list in the pool, or -1
  int scnt[SH_SEGS + 1];  // new columns per segment of the chunk, then their exclusive scan and total
  int wbuf[SH_WARPS][SH_BUF];
  alignas(16) unsigned bitmap[SH_COLS / 32];
};


// The eight bitmap words of a lane in a segment pair (words w0 .. w0 + 7),
// zero past the chunk's last word.
__device__ __forceinline__ void sh_load8(const unsigned *bitmap, int w0, int words, unsigned long long (&b)[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int w = w0 + 4 * h;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (w + 3 < words) v = *reinterpret_cast<const uint4 *>(bitmap + w);
    else if (w < words) {
      v.x = bitmap[w];
      if (w + 1 < words) v.y = bitmap[w + 1];
      if (w + 2 < words) v.z = bitmap[w + 2];
    }
    b[2 * h] = ((unsigned long long)v.y << 32) | v.x;
    b[2 * h + 1] = ((unsigned long long)v.w << 32) | v.z;
  }
}
// Clears the same eight words (the bitmap is left empty for the next row).
__device__ __forceinline__ void sh_clear8(unsigned *bitmap, int w0, int words) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int w = w0 + 4 * h;
    if (w + 3 < words) *reinterpret_cast<uint4 *>(bitmap + w) = make_uint4(0u, 0u, 0u, 0u);
    else
      for (int k = w; k < words && k < w + 4; ++k) bitmap[k] = 0u;
  }
}

__global__ void __launch_bounds__(SH_NT, SH_MINB) k_sym_heavy(SymArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto &sm = *reinterpret_cast<SymHeavySmem *>(smem_raw);
  const DevCsr A = dev_a(a.A), B = dev_b(a.B);
  const int64_t n = a.B.n;
  const int nchunk = (int)((n + SH_COLS - 1) / SH_COLS);
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = SH_WARPS;
  int *buf = sm.wbuf[warp];
  // the first chunk is the widest: clearing its words once leaves the whole
  // bitmap empty, and every chunk clears the words it read afterwards
  {
    const int words0 = (int)((min(n, (int64_t)SH_COLS) + 31) >> 5);
    for (int wd = threadIdx.x; wd < words0; wd += SH_NT) sm.bitmap[wd] = 0u;
  }
  while (true) {
    if (threadIdx.x == 0) sm.row = atomicAdd(a.dyn, 1);
    __syncthreads();
    const int idx = sm.row;
    if (idx >= a.count) break;
    const int r0 = a.list[idx];
    // a bad row id (guarded builds) runs no chunk, so the loop still reaches its closing barriers
    const bool r_ok = HS_G(a.A.dbg, r0 >= 0 && r0 < a.A.nslots, 35, r0);
    const int r = r_ok ? r0 : 0;
    const int h = r_ok ? a.hslot[r] : -1;
    uint32_t *hist = h >= 0 ? a.hist + (int64_t)h * a.nseg : nullptr;
    int32_t *lst = nullptr;  // the row's list, once its room is taken (first chunk)
    const int64_t lmax = r_ok ? min(a.f[r], n) : 0;  // the list's room: min(f, n) entries bound its output
    int64_t written = 0;  // columns of the earlier chunks
    for (int ch = 0; ch < (r_ok ? nchunk : 0); ++ch) {
      const int lo = ch * SH_COLS;
      const int hi = (int)min((int64_t)lo + SH_COLS, n);
      const int words = (hi - lo + 31) >> 5;
      const int nsc = (hi - lo + SEG_W - 1) / SEG_W;
      cta_products<StructSR, CH, 4>(A, B, A.p[r], A.p[r + 1], nchunk > 1, lo, hi, sm.ex, sm.wtmp,
                                    SymHeavyBit{sm.bitmap, lo, (unsigned)(hi - lo), a.A.dbg});
      // columns per segment, by pairs of segments (8192 columns, eight words
      // per lane; warp w takes pairs w, w + 32, ...): each lane's count and
      // its inclusive scan over the warp are kept for the list pass.  The
      // row's list room is taken from the pool meanwhile (thread 0 issues the
      // atomic first and reads its answer after its counts)
      unsigned long long at_l = 0ull;
      const bool take = threadIdx.x == 0 && ch == 0 && a.glist;
      if (take) at_l = atomicAdd(a.lpool, (unsigned long long)lmax);
      int keep[SH_PPW];  // (inclusive scan << 16) | lane count
#pragma unroll
      for (int i = 0; i < SH_PPW; ++i) {
        const int g = 2 * (warp + nw * i);
        keep[i] = 0;
        if (g < nsc) {  // warp-uniform
          const int wb = g * (SEG_W / 32) + 8 * lane;
          unsigned long long b[4];
          sh_load8(sm.bitmap, wb, words, b);
          const int pcl = __popcll(b[0]) + __popcll(b[1]) + __popcll(b[2]) + __popcll(b[3]);
          const int incl = warp_incl_scan(pcl);
          const int first = __shfl_sync(FULL, incl, 15);  // lanes 0..15 hold segment g
          const int tot = __shfl_sync(FULL, incl, 31);
          if (lane == 0) {
            sm.scnt[g] = first;
            if (g + 1 < nsc) sm.scnt[g + 1] = tot - first;
          }
          keep[i] = (incl << 16) | pcl;
          if (!a.glist) sh_clear8(sm.bitmap, wb, words);  // no list pass reads them again
        }
      }
      if (threadIdx.x == 0 && ch == 0) sm.loff = (take && (long long)at_l + lmax <= a.lcap) ? (long long)at_l : -1;
      __syncthreads();
      if (ch == 0 && sm.loff >= 0) lst = a.glist + sm.loff;
      // one warp: the counts out to the segment histogram, then their
      // exclusive scan (at most eight per lane), the chunk's total in the last slot
      if (warp == 0) {
        const int per = (nsc + 31) / 32;
        const int gb = min(nsc, lane * per), ge = min(nsc, gb + per);
        int cs = 0;
        for (int g = gb; g < ge; ++g) {
          const int c = sm.scnt[g];
          cs += c;
          if (hist && HS_G(a.A.dbg, lo / SEG_W + g < a.nseg, 32, g)) hist[lo / SEG_W + g] = (uint32_t)c;
        }
        const int ci = warp_incl_scan(cs);
        int run = ci - cs;
        for (int g = gb; g < ge; ++g) {
          const int c = sm.scnt[g];
          sm.scnt[g] = run;
          run += c;
        }
        if (lane == 31) sm.scnt[SH_SEGS] = ci;
      }
      __syncthreads();
      const int ctotal = sm.scnt[SH_SEGS];
      // list: the same pairs, read again (a row that found no room in the
      // pool only clears them)
      if (!lst && a.glist) {
#pragma unroll
        for (int i = 0; i < SH_PPW; ++i) {
          const int g = 2 * (warp + nw * i);
          if (g < nsc) sh_clear8(sm.bitmap, g * (SEG_W / 32) + 8 * lane, words);
        }
      }
      if (lst) {
#pragma unroll
        for (int i = 0; i < SH_PPW; ++i) {
          const int g = 2 * (warp + nw * i);
          if (g >= nsc) break;  // warp-uniform
          const int wb = g * (SEG_W / 32) + 8 * lane;
          unsigned long long b[4];
          sh_load8(sm.bitmap, wb, words, b);
          const int pcl = keep[i] & 0xffff, incl = keep[i] >> 16;
          const int tot = __shfl_sync(FULL, incl, 31);
          // the pair's columns start where segment g's do (g + 1 follows it)
          const int64_t at0 = written + sm.scnt[g];
          const int cbase = lo + (wb << 5);
          if (!HS_G(a.A.dbg, at0 + tot <= lmax, 34, at0 + tot)) {
            // nothing is written; the words are still cleared below
          } else if (tot <= SH_BUF) {
            // the lane's columns one per iteration over all eight words (the
            // warp runs as many iterations as its fullest lane has columns);
            // the next non-empty word is read again when the current one is spent
            unsigned m = 0u;  // the lane's non-empty words
#pragma unroll
            for (int q = 0; q < 4; ++q)
              m |= ((unsigned)((unsigned)b[q] != 0u) << (2 * q)) | ((unsigned)((unsigned)(b[q] >> 32) != 0u) << (2 * q + 1));
            int p = incl - pcl;
            unsigned cur = 0u;
            int cw = 0;
            for (int k = 0; k < pcl; ++k) {
              if (cur == 0u) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                cur = sm.bitmap[wb + j];
                cw = cbase + 32 * j;
              }
              buf[p++] = cw + __ffs(cur) - 1;
              cur &= cur - 1;
            }
            __syncwarp();
            for (int i2 = lane; i2 < tot; i2 += 32) __stcs(lst + at0 + i2, buf[i2]);  // evict-first: B stays in L2
          } else {
            // dense pair: re-read as eight steps of 1024 columns, lane l on the
            // step's word l, so a step's columns run in lane order; the steps
            // gather in the staging buffer and leave it in coalesced stores
            const int gw = g * (SEG_W / 32);
            int fill = 0;       // staged entries
            int64_t at = at0;   // list position of buf[0]
            for (int s2 = 0; s2 < 8; ++s2) {
              const int wd = gw + 32 * s2 + lane;
              unsigned bb = wd < words ? sm.bitmap[wd] : 0u;
              const int pc = __popc(bb);
              const int inc = warp_incl_scan(pc);
              const int st = __shfl_sync(FULL, inc, 31);
              if (fill + st > SH_BUF) {  // warp-uniform
                __syncwarp();
                for (int i2 = lane; i2 < fill; i2 += 32) __stcs(lst + at + i2, buf[i2]);
                __syncwarp();
                at += fill;
                fill = 0;
              }
              const int c0 = lo + (wd << 5);
              if (st <= SH_BUF) {
                int p = fill + inc - pc;
                while (bb) {
                  buf[p++] = c0 + __ffs(bb) - 1;
                  bb &= bb - 1;
                }
                fill += st;
              } else {  // more than SH_BUF columns in 1024: each lane's few go straight out
                int64_t q = at + inc - pc;
                while (bb) {
                  __stcs(lst + q++, c0 + __ffs(bb) - 1);
                  bb &= bb - 1;
                }
                at += st;
              }
            }
            __syncwarp();
            for (int i2 = lane; i2 < fill; i2 += 32) __stcs(lst + at + i2, buf[i2]);
          }
          __syncwarp();  // every lane's reads of the pair's words (and of buf) are done
          sh_clear8(sm.bitmap, wb, words);
        }
      }
      written += ctotal;
      __syncthreads();
    }
    if (threadIdx.x == 0 && r_ok) {
      put_count(a, out_row(a.A, r), written);
      if (a.loff) a.loff[r] = lst ? sm.loff : -1;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- launchers
static int grid_cap(int items, int per_block, int per_sm) {
  int g = (items + per_block - 1) / per_block;
  int cap = sm_count() * per_sm;
  return g < cap ? (g < 1 ? 1 : g) : cap;
}

void launch_sym_tiny(const SymArgs &a, cudaStream_t st) {
  if (a.count <= 0) return;
  count_launch();
  k_sym_tiny<<<grid_cap(a.count, TINY_WPB, 8), TINY_WPB * 32, 0, st>>>(a);
}
// CTAs that fit one SM for this kernel, block size and dynamic shared memory
template <class K> static int fit_per_sm(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return n < 1 ? 1 : n;
}

template <int SLOTS> static void launch_sym_warp_slots(const SymArgs &a, cudaStream_t st) {
  if (a.count <= 0) return;
  const size_t bytes = sizeof(int) * WARP_WPB * SLOTS;
  set_smem_attr(k_sym_warp<SLOTS>, bytes);
  count_launch();
  k_sym_warp<SLOTS><<<grid_cap(a.count, WARP_WPB, fit_per_sm(k_sym_warp<SLOTS>, WARP_WPB * 32, bytes)),
                      WARP_WPB * 32, bytes, st>>>(a);
}
void launch_sym_warp(const SymArgs &a, cudaStream_t st) { launch_sym_warp_slots<2 * F_WARP>(a, st); }
void launch_sym_spa(const SymArgs &a, cudaStream_t st) {
  if (a.count <= 0) return;
  count_launch();
  k_sym_spa<<<grid_cap(a.count, SPA_WPB, fit_per_sm(k_sym_spa, SPA_WPB * 32, 0)), SPA_WPB * 32, 0, st>>>(a);
}

template <int SLOTS, int NT> static void launch_sym_cta(const SymArgs &a, cudaStream_t st) {
  if (a.count <= 0) return;
  const size_t bytes = sizeof(SymCtaSmem<SLOTS>);
  set_smem_attr(k_sym_cta<SLOTS, NT>, bytes);
  count_launch();
  k_sym_cta<SLOTS, NT><<<grid_cap(a.count, 1, fit_per_sm(k_sym_cta<SLOTS, NT>, NT, bytes)), NT, bytes, st>>>(a);
}
// table capacity 2f: mid rows have f <= 4096, large rows f <= min(16384, cap_large) = 8192 at most
void launch_sym_mid_s(const SymArgs &a, cudaStream_t st) { launch_sym_warp_slots<2 * F_MID_S>(a, st); }
void launch_sym_mid(const SymArgs &a, cudaStream_t st) { launch_sym_cta<2 * F_MID, 256>(a, st); }
void launch_sym_large(const SymArgs &a, cudaStream_t st) { launch_sym_cta<16384, 512>(a, st); }

void launch_sym_heavy(const SymArgs &a, cudaStream_t st) {
  if (a.count <= 0) return;
  const int64_t words = (a.B.n + 31) / 32;
  const size_t bytes = offsetof(SymHeavySmem, bitmap) +
                       sizeof(unsigned) * (size_t)(words < SH_COLS / 32 ? words : SH_COLS / 32);
  set_smem_attr(k_sym_heavy, sizeof(SymHeavySmem));
  count_launch();
  k_sym_heavy<<<grid_cap(a.count, 1, fit_per_sm(k_sym_heavy, SH_NT, bytes)), SH_NT, bytes, st>>>(a);
}

}  // namespace hs
