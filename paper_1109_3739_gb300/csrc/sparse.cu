// sparse.cu -- the constructor sparse(i, j, v, m, n) of Section 2's notation:
// the m x n matrix with entry (i[k], j[k]) = v[k], tuples that name one
// position combined with the semiring's add.
//
// Each tuple becomes one key, row i in the high bits and column j in the low
// bits, so the keys' order is CSR order.  A stable least-significant-digit
// radix sort (8-bit digits, as many passes as the key has bytes of
// information) carries the values along; stability keeps the tuples of one
// position in their input order.  k_sp_allhist reads i and j once and counts
// the digits of every pass (and checks the index ranges).  Each pass is then
// one kernel, k_sp_onesweep: a tile of 4096 tuples is ranked stably in
// shared memory, publishes its per-digit counts, learns the counts of the
// tiles before it by decoupled look-back (Merrill & Garland's single-pass
// prefix scan, as in the Onesweep radix sort of Adinets & Merrill), and writes
// its tuples out digit run by digit run.  Then runs of equal keys are the
// entries of C: k_sp_heads counts run heads per tile, and k_sp_emit writes
// one column id and one combined value per run and counts the entries of
// each row; runs longer than SP_SHORT are combined by a warp each
// (k_sp_long).  A pass moves 24 bytes per tuple with 4-byte values.
#include "common.cuh"
#include "internal.h"

namespace hs {

constexpr int SP_NT = 256, SP_IPT = 16, SP_TILE = SP_NT * SP_IPT, SP_RADIX = 256;
constexpr int SP_WARPS = SP_NT / 32;
constexpr int SP_SHORT = 32;  // longer runs of one position go to k_sp_long
constexpr int SP_MAX_PASSES = 8;
// look-back status words: bit 63 inclusive prefix, bit 62 tile aggregate,
// bits 32..47 pass tag (pass + 1, so that one zeroed array serves every
// pass), bits 0..31 the count
constexpr unsigned long long SP_INCL = 1ull << 63, SP_AGG = 1ull << 62;
constexpr int SP_SPIN_LIMIT = 1 << 18;  // polls of one status word before giving up (well under a second)
int sp_spin_limit() { return SP_SPIN_LIMIT; }
static_assert(SP_NT == SP_RADIX, "one thread per digit in the per-tile digit scan");

template <bool FIRST>
__device__ __forceinline__ uint64_t sp_key(const uint64_t *K, const int32_t *I, const int32_t *J, int64_t t,
                                           int nbj, int64_t m, int64_t n, int *flag) {
  if (!FIRST) return K[t];
  const int32_t i = I[t], j = J[t];
  if (i < 0 || i >= m || j < 0 || j >= n) {  // the host reports HS_EINVAL; the key only has to be some digit
    atomicOr(flag, 1);
    return 0;
  }
  return ((uint64_t)(uint32_t)i << nbj) | (uint64_t)(uint32_t)j;
}

// digit counts of every pass in one read of i and j: ghist[p * 256 + d]
__global__ void __launch_bounds__(SP_NT) k_sp_allhist(const int32_t *I, const int32_t *J, int64_t nnz, int nbj,
                                                      int64_t m, int64_t n, int passes, unsigned long long *ghist,
                                                      int *flag) {
  __shared__ int h[SP_MAX_PASSES][SP_RADIX];
  for (int x = threadIdx.x; x < SP_MAX_PASSES * SP_RADIX; x += SP_NT) (&h[0][0])[x] = 0;
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * SP_NT + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * SP_NT) {
    const uint64_t key = sp_key<true>(nullptr, I, J, t, nbj, m, n, flag);
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(int)((key >> (8 * p)) & (SP_RADIX - 1))], 1);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < passes * SP_RADIX; x += SP_NT) {
    const int c = (&h[0][0])[x];
    if (c) atomicAdd(ghist + x, (unsigned long long)c);
  }
}

template <int VB> struct SpVal { using T = uint32_t; };
template <> struct SpVal<8> { using T = uint64_t; };

template <int VB> constexpr size_t sp_scatter_smem() {
  return (size_t)SP_TILE * 8 + (size_t)SP_TILE * (VB ? VB : 0) + sizeof(int) * SP_WARPS * SP_RADIX +
         sizeof(int) * SP_RADIX + sizeof(long long) * SP_RADIX;
}

__device__ __forceinline__ unsigned long long sp_ld(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void sp_st(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// one stable pass.  ghist: this pass's 256 digit totals; status: tiles x 256
// look-back words (zeroed once per call); ticket: tiles are numbered in the
// order the CTAs start, so every tile a CTA waits for has started before it.
template <bool FIRST, int VB>
__global__ void __launch_bounds__(SP_NT, 3) k_sp_onesweep(const uint64_t *Kin, const int32_t *I, const int32_t *J,
                                                       const void *Vin, int64_t nnz, int nbj, int64_t m,
                                                       int64_t n, int pass, const unsigned long long *ghist,
                                                       unsigned long long *status, int *ticket, uint64_t *Kout,
                                                       void *Vout, int *flag, int spin_limit, long long withhold) {
  using VT = typename SpVal<VB>::T;
  extern __shared__ __align__(16) unsigned char sp_smem[];
  uint64_t *skey = reinterpret_cast<uint64_t *>(sp_smem);
  VT *sval = reinterpret_cast<VT *>(sp_smem + (size_t)SP_TILE * 8);
  int *wcnt = reinterpret_cast<int *>(sp_smem + (size_t)SP_TILE * 8 + (size_t)SP_TILE * VB);  // [warp][digit]
  int *start = wcnt + SP_WARPS * SP_RADIX;
  long long *goff = reinterpret_cast<long long *>(start + SP_RADIX);
  __shared__ int wsum[SP_WARPS];
  __shared__ int tile_s;

  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int shift = 8 * pass;
  for (int x = threadIdx.x; x < SP_WARPS * SP_RADIX; x += SP_NT) wcnt[x] = 0;
  if (threadIdx.x == 0) tile_s = atomicAdd(ticket, 1);
  __syncthreads();
  const int64_t tile = tile_s;
  const int64_t t0 = tile * SP_TILE;
  const int nt = (int)(nnz - t0 < SP_TILE ? nnz - t0 : SP_TILE);
  const unsigned lt = (1u << lane) - 1u;
  uint64_t k[SP_IPT];
  VT v[SP_IPT];
  unsigned r2[SP_IPT / 2];  // ranks inside the warp's digit group (< 512), two per register
  // warp w ranks the tile's items w*512 .. w*512+511 in order, 32 at a time;
  // every load is issued before the first ranking step
#pragma unroll
  for (int it = 0; it < SP_IPT; ++it) {
    const int e = w * (SP_IPT * 32) + it * 32 + lane;
    k[it] = 0;
    v[it] = 0;
    if (e < nt) {
      k[it] = sp_key<FIRST>(Kin, I, J, t0 + e, nbj, m, n, flag);
      if (VB) v[it] = reinterpret_cast<const VT *>(Vin)[t0 + e];
    }
  }
#pragma unroll
  for (int it = 0; it < SP_IPT; ++it) {
    const int e = w * (SP_IPT * 32) + it * 32 + lane;
    const bool ok = e < nt;
    if (!(it & 1)) r2[it >> 1] = 0;
    const unsigned act = __ballot_sync(FULL, ok);
    if (ok) {
      const int d = (int)((k[it] >> shift) & (SP_RADIX - 1));
      const unsigned peers = __match_any_sync(act, d);
      const int base = wcnt[w * SP_RADIX + d];
      r2[it >> 1] |= (unsigned)(base + __popc(peers & lt)) << (16 * (it & 1));
      __syncwarp(act);
      if (lane == 31 - __clz(peers)) wcnt[w * SP_RADIX + d] = base + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // thread d: the warps' offsets inside the tile's run of digit d, the tile's
  // count of d, published at once so that later tiles can go on
  const int d = threadIdx.x;
  int tot = 0;
#pragma unroll
  for (int ww = 0; ww < SP_WARPS; ++ww) {
    const int c = wcnt[ww * SP_RADIX + d];
    wcnt[ww * SP_RADIX + d] = tot;
    tot += c;
  }
  const unsigned long long tag = (unsigned long long)(pass + 1) << 32;
  unsigned long long *my = status + tile * SP_RADIX + d;
  // (a tile equal to `withhold` never publishes: the failure-detection
  // tests use it so that the next tile's bounded wait runs out)
  const bool publish = tile != withhold;
  if (publish) {
    if (tile == 0) sp_st(my, SP_INCL | tag | (unsigned)tot);
    else sp_st(my, SP_AGG | tag | (unsigned)tot);
  }
  // tile start of each digit (exclusive scan over the digits) and the digit's
  // start in the whole output (exclusive scan of this pass's totals)
  const int incl = warp_incl_scan(tot);
  const long long gh = (long long)ghist[d];
  const long long gincl = warp_incl_scan(gh);
  __shared__ long long gsum[SP_WARPS];
  if (lane == 31) {
    wsum[w] = incl;
    gsum[w] = gincl;
  }
  __syncthreads();
  int before = 0;
  long long gbefore = 0;
#pragma unroll
  for (int ww = 0; ww < SP_WARPS; ++ww) {
    before += ww < w ? wsum[ww] : 0;
    gbefore += ww < w ? gsum[ww] : 0;
  }
  start[d] = before + incl - tot;
  // decoupled look-back over the tiles before this one
  long long excl = 0;
  if (tile > 0) {
    for (int64_t j = tile - 1; j >= 0; --j) {
      const unsigned long long *q = status + j * SP_RADIX + d;
      unsigned long long x = 0;
      int spin = 0;
      for (;;) {
        x = sp_ld(q);
        if ((x & (0xffffull << 32)) == tag && (x & (SP_INCL | SP_AGG))) break;
        if (++spin > spin_limit) {  // never expected: the host reports HS_ETIMEDOUT
          atomicOr(flag, 2);
          x = SP_INCL | tag;
          break;
        }
        if (spin > 32) __nanosleep(64);
      }
      excl += (long long)(x & 0xffffffffull);
      if (x & SP_INCL) break;
    }
    if (publish) sp_st(my, SP_INCL | tag | (unsigned)(excl + tot));
  }
  goff[d] = gbefore + gincl - gh + excl;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < SP_IPT; ++it) {
    const int e = w * (SP_IPT * 32) + it * 32 + lane;
    if (e < nt) {
      const int dd = (int)((k[it] >> shift) & (SP_RADIX - 1));
      const int pos = start[dd] + wcnt[w * SP_RADIX + dd] + (int)((r2[it >> 1] >> (16 * (it & 1))) & 0xffffu);
      skey[pos] = k[it];
      if (VB) sval[pos] = v[it];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nt; e += SP_NT) {
    const uint64_t key = skey[e];
    const int dd = (int)((key >> shift) & (SP_RADIX - 1));
    const long long out = goff[dd] + (e - start[dd]);
    if (out < 0 || out >= nnz) continue;  // only after an expired wait
    Kout[out] = key;
    if (VB) reinterpret_cast<VT *>(Vout)[out] = sval[e];
  }
}

// number of runs of equal keys starting in each tile
__global__ void __launch_bounds__(SP_NT) k_sp_heads(const uint64_t *K, int64_t nnz, int64_t *theads) {
  __shared__ int ws[SP_WARPS];
  const int64_t t0 = (int64_t)blockIdx.x * SP_TILE;
  int c = 0;
  for (int e = threadIdx.x; e < SP_TILE; e += SP_NT) {
    const int64_t t = t0 + e;
    if (t < nnz && (t == 0 || K[t] != K[t - 1])) ++c;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int ww = 0; ww < SP_WARPS; ++ww) s += ws[ww];
    theads[blockIdx.x] = s;
  }
}

// combine operations: 0 (+) on f64, 1 (+) on f32, 2 (+) on i64 (mod 2^64),
// 3 min on f32, 4 min on i32, 5 none (bool)
template <int OP> struct SpOp;
template <> struct SpOp<0> {
  using T = double;
  static __device__ T add(T a, T b) { return a + b; }
};
template <> struct SpOp<1> {
  using T = float;
  static __device__ T add(T a, T b) { return a + b; }
};
template <> struct SpOp<2> {
  using T = int64_t;
  static __device__ T add(T a, T b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
};
template <> struct SpOp<3> {
  using T = float;
  static __device__ T add(T a, T b) { return b < a ? b : a; }  // earlier value kept on ties
};
template <> struct SpOp<4> {
  using T = int32_t;
  static __device__ T add(T a, T b) { return b < a ? b : a; }
};
template <> struct SpOp<5> {
  using T = int32_t;  // unused
  static __device__ T add(T a, T) { return a; }
};

// one column id and one value per run; row counts into rowcnt[row + 1].
// Thread x owns the 16 sorted tuples x*16 .. x*16+15 of the tile and every
// run that starts among them; keys and values are loaded once, runs are
// folded in registers, and only a run that continues past the thread's last
// tuple reads further (up to SP_SHORT tuples, longer ones go to k_sp_long,
// which runs afterwards and overwrites their values).  The tile's entries of
// C are consecutive: they are assembled in shared memory and written out
// with coalesced stores.
template <int OP>
__global__ void __launch_bounds__(SP_NT) k_sp_emit(const uint64_t *K, const void *Vs, int64_t nnz, int nbj,
                                                   const int64_t *theads_incl, int32_t *Cidx, void *Cval,
                                                   int64_t *rowcnt, int64_t *longlist, int *nlong) {
  using T = typename SpOp<OP>::T;
  constexpr bool HAS_VAL = OP != 5;
  __shared__ int ws[SP_WARPS];
  extern __shared__ __align__(16) unsigned char sp_smem[];
  int32_t *scol = reinterpret_cast<int32_t *>(sp_smem);
  T *sv = reinterpret_cast<T *>(sp_smem + sizeof(int32_t) * SP_TILE);
  const T *V = reinterpret_cast<const T *>(Vs);
  const int64_t t0 = (int64_t)blockIdx.x * SP_TILE + (int64_t)threadIdx.x * SP_IPT;
  const uint64_t maskj = nbj ? ((1ull << nbj) - 1ull) : 0ull;
  uint64_t k[SP_IPT];
  T v[SP_IPT];
  const bool full = t0 + SP_IPT <= nnz;
  if (full) {  // 128 contiguous key bytes per thread
    const uint4 *src = reinterpret_cast<const uint4 *>(K + t0);
#pragma unroll
    for (int q = 0; q < SP_IPT / 2; ++q) {
      const uint4 x = src[q];
      k[2 * q] = ((uint64_t)x.y << 32) | x.x;
      k[2 * q + 1] = ((uint64_t)x.w << 32) | x.z;
    }
  } else {
#pragma unroll
    for (int e = 0; e < SP_IPT; ++e) k[e] = t0 + e < nnz ? K[t0 + e] : 0;
  }
  if (HAS_VAL) {
#pragma unroll
    for (int e = 0; e < SP_IPT; ++e) v[e] = t0 + e < nnz ? V[t0 + e] : T{};
  }
  const uint64_t prev = (t0 > 0 && t0 <= nnz) ? K[t0 - 1] : 0;
  unsigned heads = 0;
#pragma unroll
  for (int e = 0; e < SP_IPT; ++e) {
    const int64_t t = t0 + e;
    const bool h = t < nnz && (t == 0 || k[e] != (e ? k[e - 1] : prev));
    heads |= (unsigned)h << e;
  }
  const int c = __popc(heads);
  const int incl = warp_incl_scan(c);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 31) ws[w] = incl;
  __syncthreads();
  const int64_t base = blockIdx.x ? theads_incl[blockIdx.x - 1] : 0;
  const int in_tile = (int)(theads_incl[blockIdx.x] - base);
  int64_t p = 0;  // slot inside the tile's entries
  for (int ww = 0; ww < SP_WARPS; ++ww) p += ww < w ? ws[ww] : 0;
  p += incl - c;
  const int nv = full ? SP_IPT : (int)(nnz - t0);
  int64_t cur_row = -1;
  int rc = 0;
  T acc{};
  int run_len = 0;     // tuples folded into acc
  int64_t run_p = -1;  // output slot of the open run
  uint64_t last = 0;   // key of the thread's last tuple
#pragma unroll
  for (int e = 0; e < SP_IPT; ++e) {
    if (heads && e < nv) {
      last = k[e];
      if ((heads >> e) & 1u) {
        if (HAS_VAL && run_p >= 0) sv[run_p] = acc;
        const int64_t row = (int64_t)(k[e] >> nbj);
        scol[p] = (int32_t)(k[e] & maskj);
        if (row != cur_row) {
          if (rc) atomicAdd(reinterpret_cast<unsigned long long *>(rowcnt + cur_row + 1), (unsigned long long)rc);
          cur_row = row;
          rc = 0;
        }
        ++rc;
        if (HAS_VAL) {
          acc = v[e];
          run_len = 1;
          run_p = p;
        }
        ++p;
      } else if (HAS_VAL && run_p >= 0) {
        acc = SpOp<OP>::add(acc, v[e]);
        ++run_len;
      }
    }
  }
  if (rc) atomicAdd(reinterpret_cast<unsigned long long *>(rowcnt + cur_row + 1), (unsigned long long)rc);
  if (HAS_VAL && heads) {
    // the last run may continue into the next threads' tuples
    const uint64_t key = last;
    const int64_t start = t0 + nv - run_len;
    int64_t q = t0 + nv;
    while (q < nnz && q - start < SP_SHORT && K[q] == key) acc = SpOp<OP>::add(acc, V[q++]);
    if (q < nnz && q - start == SP_SHORT && K[q] == key) {
      const int at = atomicAdd(nlong, 1);  // at most nnz / (SP_SHORT + 1) runs qualify
      longlist[2 * at] = start;
      longlist[2 * at + 1] = base + run_p;
    }
    sv[run_p] = acc;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < in_tile; x += SP_NT) {
    __stcs(Cidx + base + x, scol[x]);
    if (HAS_VAL) __stcs(reinterpret_cast<T *>(Cval) + base + x, sv[x]);
  }
}

// runs longer than SP_SHORT: one warp each; lane l folds the l-th of 32
// consecutive slices in order, lane 0 folds the slices' results in order
template <int OP>
__global__ void __launch_bounds__(SP_NT) k_sp_long(const uint64_t *K, const void *Vs, int64_t nnz,
                                                   const int64_t *longlist, const int *nlong, void *Cval) {
  using T = typename SpOp<OP>::T;
  const T *V = reinterpret_cast<const T *>(Vs);
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * SP_NT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * SP_NT) >> 5;
  const int cnt = *nlong;
  for (int64_t x = gw; x < cnt; x += nw) {
    const int64_t t = longlist[2 * x], p = longlist[2 * x + 1];
    const uint64_t key = K[t];
    // end of the run: first q > t with a different key
    int64_t e = t + SP_SHORT;
    for (;;) {
      const int64_t q = e + lane;
      const bool diff = q >= nnz || K[q] != key;
      const unsigned b = __ballot_sync(FULL, diff);
      if (b) {
        e += __ffs(b) - 1;
        break;
      }
      e += 32;
    }
    const int64_t len = e - t, per = (len + 31) / 32;
    const int64_t a = t + lane * per, z = a + per < e ? a + per : e;
    T acc{};
    bool has = a < z;
    if (has) {
      acc = V[a];
      for (int64_t q = a + 1; q < z; ++q) acc = SpOp<OP>::add(acc, V[q]);
    }
    T tot{};
    bool any = false;
    for (int l = 0; l < 32; ++l) {
      const T x2 = __shfl_sync(FULL, acc, l);
      const bool h2 = __shfl_sync(FULL, (int)has, l);
      if (h2) {
        tot = any ? SpOp<OP>::add(tot, x2) : x2;
        any = true;
      }
    }
    if (lane == 0) reinterpret_cast<T *>(Cval)[p] = tot;
  }
}

static int sp_grid(int64_t tiles) { return (int)tiles; }
template <int OP> static constexpr size_t sp_emit_smem() {
  return sizeof(int32_t) * SP_TILE + (OP == 5 ? 0 : sizeof(typename SpOp<OP>::T) * SP_TILE);
}

void launch_sp_allhist(const int32_t *I, const int32_t *J, int64_t nnz, int nbj, int64_t m, int64_t n, int passes,
                       unsigned long long *ghist, int *flag, cudaStream_t st) {
  if (nnz <= 0) return;
  int64_t g = (nnz + SP_NT - 1) / SP_NT, cap = (int64_t)sm_count() * 8;
  count_launch();
  k_sp_allhist<<<(int)(g < cap ? g : cap), SP_NT, 0, st>>>(I, J, nnz, nbj, m, n, passes, ghist, flag);
}

template <bool FIRST, int VB>
static void sp_pass_one(const uint64_t *Kin, const int32_t *I, const int32_t *J, const void *Vin, int64_t nnz,
                        int nbj, int64_t m, int64_t n, int pass, const unsigned long long *ghist,
                        unsigned long long *status, int *ticket, int64_t ntiles, uint64_t *Kout, void *Vout,
                        int *flag, int spin_limit, long long withhold, cudaStream_t st) {
  constexpr size_t smem = sp_scatter_smem<VB>();
  set_smem_attr(k_sp_onesweep<FIRST, VB>, smem);
  count_launch();
  k_sp_onesweep<FIRST, VB><<<sp_grid(ntiles), SP_NT, smem, st>>>(Kin, I, J, Vin, nnz, nbj, m, n, pass, ghist,
                                                                 status, ticket, Kout, Vout, flag, spin_limit,
                                                                 withhold);
}

void launch_sp_pass(int vb, const uint64_t *Kin, const int32_t *I, const int32_t *J, const void *Vin, int64_t nnz,
                    int nbj, int64_t m, int64_t n, int pass, const unsigned long long *ghist,
                    unsigned long long *status, int *ticket, int64_t ntiles, uint64_t *Kout, void *Vout, int *flag,
                    int spin_limit, long long withhold, cudaStream_t st) {
  if (ntiles <= 0) return;
  if (spin_limit < 1) spin_limit = 1;
#define SP_PS(F, B)                                                                                              \
  sp_pass_one<F, B>(Kin, I, J, Vin, nnz, nbj, m, n, pass, ghist, status, ticket, ntiles, Kout, Vout, flag, \
                    spin_limit, withhold, st)
  if (pass == 0) {
    if (vb == 8) SP_PS(true, 8);
    else if (vb == 4) SP_PS(true, 4);
    else SP_PS(true, 0);
  } else {
    if (vb == 8) SP_PS(false, 8);
    else if (vb == 4) SP_PS(false, 4);
    else SP_PS(false, 0);
  }
#undef SP_PS
}

void launch_sp_heads(const uint64_t *K, int64_t nnz, int64_t *theads, int64_t ntiles, cudaStream_t st) {
  if (ntiles <= 0) return;
  count_launch();
  k_sp_heads<<<sp_grid(ntiles), SP_NT, 0, st>>>(K, nnz, theads);
}

void launch_sp_emit(int op, const uint64_t *K, const void *V, int64_t nnz, int nbj, const int64_t *theads_incl,
                    int64_t ntiles, int32_t *Cidx, void *Cval, int64_t *rowcnt, int64_t *longlist, int *nlong,
                    cudaStream_t st) {
  if (ntiles <= 0) return;
  count_launch();
#define SP_EM(O)                                                                                       \
  set_smem_attr(k_sp_emit<O>, sp_emit_smem<O>());                                                      \
  k_sp_emit<O><<<sp_grid(ntiles), SP_NT, sp_emit_smem<O>(), st>>>(K, V, nnz, nbj, theads_incl, Cidx, Cval, \
                                                                  rowcnt, longlist, nlong)
  switch (op) {
    case 0: SP_EM(0); break;
    case 1: SP_EM(1); break;
    case 2: SP_EM(2); break;
    case 3: SP_EM(3); break;
    case 4: SP_EM(4); break;
    default: SP_EM(5); break;
  }
#undef SP_EM
  if (op == 5) return;
  count_launch();
  const int grid = sm_count() * 4;
#define SP_LG(O) k_sp_long<O><<<grid, SP_NT, 0, st>>>(K, V, nnz, longlist, nlong, Cval)
  switch (op) {
    case 0: SP_LG(0); break;
    case 1: SP_LG(1); break;
    case 2: SP_LG(2); break;
    case 3: SP_LG(3); break;
    default: SP_LG(4); break;
  }
#undef SP_LG
}

int64_t sp_tiles(int64_t nnz) { return (nnz + SP_TILE - 1) / SP_TILE; }
int sp_radix_bits() { return 8; }
int sp_max_passes() { return SP_MAX_PASSES; }
int64_t sp_long_capacity(int64_t nnz) { return nnz / (SP_SHORT + 1) + 1; }

}  // namespace hs
