// analysis.cu -- integer work ahead of the products: per-row flop counts,
// binning of rows, prefix sums and input validation.
//
// flops(A*B) for row i is the number of nonzero multiplications of that row
// (Section 2 notation): sum over stored A(i,k) of nnz(B(k,:)).  Rows with no
// products are left out of every bin, so no later kernel does work for empty
// rows: the dimension-independent work list of the doubly compressed format
// (Section 2.2), built on the fly.
#include "common.cuh"
#include "internal.h"

namespace hs {

static int g_sms = 0;
static unsigned long long g_launches = 0;
void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
unsigned long long launch_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
cudaError_t &attr_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}
void launch_sm_count_init() {
  if (g_sms) return;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (g_sms <= 0) g_sms = 1;
}
int sm_count() {
  launch_sm_count_init();
  return g_sms;
}

static int grid_for(int64_t items, int per_block, int max_per_sm) {
  int64_t g = (items + per_block - 1) / per_block;
  int64_t cap = (int64_t)sm_count() * max_per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ flops
// stats[0] += total flops, stats[1] = max row flops, stats[2] = max row nnz
// of A, stats[3] += min(f, n) over rows of the symbolic heavy bin
__global__ void k_flops(RowSet A, RightOp B, int64_t *f, int *key_cnt, unsigned long long *stats, BinCfg bins) {
  __shared__ int hist[NKEYS];
  __shared__ unsigned long long blk_tot, blk_max, blk_amax, blk_heavy;
  for (int i = threadIdx.x; i < NKEYS; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) blk_tot = blk_max = blk_amax = blk_heavy = 0;
  __syncthreads();
  const int lane = lane_id();
  const int64_t wpb = blockDim.x >> 5;
  unsigned long long my_tot = 0, my_max = 0, my_amax = 0, my_heavy = 0;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < A.nslots; r += (int64_t)gridDim.x * wpb) {
    const int64_t q0 = A.p[r], q1 = A.p[r + 1];
    long long s = 0;
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      if (!HS_G(A.dbg, q >= 0 && q < A.nnz, 50, q)) break;
      const int k = A.j[q];
      if (HS_G(A.dbg, k >= 0 && k < B.m, 51, k)) s += B.p[k + 1] - B.p[k];
    }
    s = warp_sum(s);
    if (lane == 0) {
      f[r] = s;
      const int key = sym_key(s, bins);
      if (key) atomicAdd(hist + key, 1);
      if (key >= KEY_HEAVY) my_heavy += (unsigned long long)min((int64_t)s, B.n);
      my_tot += (unsigned long long)s;
      my_max = max(my_max, (unsigned long long)s);
      my_amax = max(my_amax, (unsigned long long)(q1 - q0));
    }
  }
  if (lane == 0) {
    atomicAdd(&blk_tot, my_tot);
    atomicMax(&blk_max, my_max);
    atomicMax(&blk_amax, my_amax);
    atomicAdd(&blk_heavy, my_heavy);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NKEYS; i += blockDim.x)
    if (hist[i]) atomicAdd(key_cnt + i, hist[i]);
  if (threadIdx.x == 0) {
    atomicAdd(stats + 0, blk_tot);
    atomicMax(stats + 1, blk_max);
    atomicMax(stats + 2, blk_amax);
    atomicAdd(stats + 3, blk_heavy);
  }
}

void launch_flops(const RowSet &A, const RightOp &B, int64_t *f, int *key_cnt, unsigned long long *stats,
                  const BinCfg &bins, cudaStream_t st) {
  if (A.nslots == 0) return;
  count_launch();
  k_flops<<<grid_for(A.nslots, 8, 16), 256, 0, st>>>(A, B, f, key_cnt, stats, bins);
}

// ------------------------------------------------ flat products per entry
// The same counts, computed per A entry instead of per row, so that no row
// is walked by one warp: s[q - lo] = nnz(B(A.j[q], :)) for q in [lo, hi) =
// [A.p[0], A.p[nslots]); zeros[0] counts the entries whose B row is empty
// (they make no product).  After an inclusive scan S of s, a row's count is
// S[q1 - 1 - lo] - S[q0 - 1 - lo].
__global__ void k_entry_flops(RowSet A, RightOp B, int64_t *s, unsigned long long *zeros) {
  // offsets are trusted only as far as s's length (A.nnz entries)
  const int64_t lo = A.p[0], hi = min(A.p[A.nslots], lo + A.nnz);
  int z = 0;
  for (int64_t q = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < hi;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int k = A.j[q];
    const int64_t v = HS_G(A.dbg, k >= 0 && k < B.m, 52, k) ? B.p[k + 1] - B.p[k] : 0;
    s[q - lo] = v;
    z += v == 0;
  }
  z = warp_sum(z);
  if (lane_id() == 0 && z) atomicAdd(zeros, (unsigned long long)z);
}

// thread per row: f from the scanned entry counts, then the row's key and
// the statistics k_flops gathers
__global__ void k_row_flops(RowSet A, const int64_t *S, int64_t *f, int *key_cnt, unsigned long long *stats,
                            BinCfg bins, int64_t bn) {
  __shared__ int hist[NKEYS];
  for (int i = threadIdx.x; i < NKEYS; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int64_t lo = A.p[0], len = min(A.p[A.nslots] - lo, A.nnz);
  unsigned long long my_tot = 0, my_max = 0, my_amax = 0, my_heavy = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.nslots;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q0 = min(max(A.p[r] - lo, (int64_t)0), len), q1 = min(max(A.p[r + 1] - lo, (int64_t)0), len);
    const int64_t fr = q1 > q0 ? S[q1 - 1] - (q0 > 0 ? S[q0 - 1] : 0) : 0;
    f[r] = fr;
    const int key = sym_key(fr, bins);
    if (key) atomicAdd(hist + key, 1);
    if (key >= KEY_HEAVY) my_heavy += (unsigned long long)min(fr, bn);
    my_tot += (unsigned long long)fr;
    my_max = max(my_max, (unsigned long long)fr);
    my_amax = max(my_amax, (unsigned long long)(q1 - q0));
  }
  my_tot = warp_sum(my_tot);
  my_heavy = warp_sum(my_heavy);
  my_max = warp_max(my_max);
  my_amax = warp_max(my_amax);
  if (lane_id() == 0) {
    if (my_tot) atomicAdd(stats + 0, my_tot);
    atomicMax(stats + 1, my_max);
    atomicMax(stats + 2, my_amax);
    if (my_heavy) atomicAdd(stats + 3, my_heavy);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NKEYS; i += blockDim.x)
    if (hist[i]) atomicAdd(key_cnt + i, hist[i]);
}

void launch_entry_flops(const RowSet &A, const RightOp &B, int64_t *s, unsigned long long *zeros,
                        cudaStream_t st) {
  if (A.nslots == 0 || A.nnz == 0) return;
  count_launch();
  k_entry_flops<<<grid_for(A.nnz, 256, 8), 256, 0, st>>>(A, B, s, zeros);
}
void launch_row_flops(const RowSet &A, const int64_t *S, int64_t *f, int *key_cnt, unsigned long long *stats,
                      const BinCfg &bins, int64_t bn, cudaStream_t st) {
  if (A.nslots == 0) return;
  count_launch();
  k_row_flops<<<grid_for(A.nslots, 256, 8), 256, 0, st>>>(A, S, f, key_cnt, stats, bins, bn);
}

// Dropping the A entries whose B row is empty (their products are none, so
// C is unchanged): keep[q - lo] = 1 where s > 0, recovered from the scanned
// counts; after an inclusive scan K of keep, entry q goes to K[q - lo] - 1
// and row r starts at K[A.p[r] - 1 - lo].
__global__ void k_keep_flags(RowSet A, const int64_t *S, int64_t *keep) {
  const int64_t n = min(A.p[A.nslots] - A.p[0], A.nnz);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    keep[x] = (S[x] - (x > 0 ? S[x - 1] : 0)) > 0;
}
__global__ void k_compact_entries(RowSet A, const int64_t *K, int32_t *j2, void *v2, int vb) {
  const int64_t lo = A.p[0], n = min(A.p[A.nslots] - lo, A.nnz);
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t before = x > 0 ? K[x - 1] : 0;
    if (K[x] == before) continue;
    j2[before] = A.j[lo + x];
    if (vb == 8) reinterpret_cast<uint64_t *>(v2)[before] = reinterpret_cast<const uint64_t *>(A.v)[lo + x];
    else if (vb == 4) reinterpret_cast<uint32_t *>(v2)[before] = reinterpret_cast<const uint32_t *>(A.v)[lo + x];
  }
}
__global__ void k_compact_offsets(RowSet A, const int64_t *K, int64_t *p2) {
  const int64_t lo = A.p[0], n = min(A.p[A.nslots] - lo, A.nnz);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= A.nslots;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = min(max(A.p[r] - lo, (int64_t)0), n);
    p2[r] = x > 0 ? K[x - 1] : 0;
  }
}
void launch_compact_by_keep(const RowSet &A, const int64_t *K, int32_t *j2, void *v2, int vb, int64_t *p2,
                            cudaStream_t st) {
  count_launch();
  k_compact_entries<<<grid_for(A.nnz, 256, 8), 256, 0, st>>>(A, K, j2, v2, vb);
  count_launch();
  k_compact_offsets<<<grid_for(A.nslots + 1, 256, 8), 256, 0, st>>>(A, K, p2);
}
void launch_compact_a(const RowSet &A, const int64_t *S, int64_t *keep, int64_t *scan_tmp, int32_t *j2, void *v2,
                      int vb, int64_t *p2, cudaStream_t st) {
  count_launch();
  k_keep_flags<<<grid_for(A.nnz, 256, 8), 256, 0, st>>>(A, S, keep);
  launch_scan_i64(keep, A.nnz, scan_tmp, st);
  launch_compact_by_keep(A, keep, j2, v2, vb, p2, st);
}

// explicit zeros (value == 0; for floats +0 and -0 alike)
template <typename T> __global__ void k_keep_nonzero(const T *v, int64_t n, int64_t *keep) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    keep[x] = v[x] != T(0);
}
void launch_keep_nonzero(const void *v, int dtype, int64_t n, int64_t *keep, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  const int g = grid_for(n, 256, 8);
  switch (dtype) {
    case 0: k_keep_nonzero<<<g, 256, 0, st>>>(reinterpret_cast<const double *>(v), n, keep); break;
    case 1: k_keep_nonzero<<<g, 256, 0, st>>>(reinterpret_cast<const float *>(v), n, keep); break;
    case 2: k_keep_nonzero<<<g, 256, 0, st>>>(reinterpret_cast<const int32_t *>(v), n, keep); break;
    default: k_keep_nonzero<<<g, 256, 0, st>>>(reinterpret_cast<const int64_t *>(v), n, keep); break;
  }
}

// ---------------------------------------------------- B segment index
// One warp per B row.  Rows longer than min_len take the next table row and
// record, for every segment g = 0..nseg, the offset of their first entry with
// column >= g*SEG_W (nseg gives the row length).  Entry p fills the segments
// after its predecessor's up to its own; the last entry fills the rest.
__global__ void k_build_bci(RightOp B, int nseg, int min_len, int64_t max_rows, int32_t *bci_id, int32_t *bci,
                            int *counter) {
  const int lane = lane_id();
  const int64_t wpb = blockDim.x >> 5;
  const int64_t stride = (int64_t)nseg + 1;
  for (int64_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < B.m; k += (int64_t)gridDim.x * wpb) {
    const int64_t b0 = B.p[k], b1 = B.p[k + 1];
    const int64_t len = b1 - b0;
    int t = -1;
    if (len > min_len && lane == 0) {
      t = atomicAdd(counter, 1);
      if (t >= max_rows) t = -1;
    }
    t = __shfl_sync(FULL, t, 0);
    if (lane == 0) bci_id[k] = t;
    if (t < 0) continue;
    int32_t *row = bci + (int64_t)t * stride;
    for (int64_t q = lane; q < len; q += 32) {
      if (!HS_G(B.dbg, b0 + q < B.nnz, 53, b0 + q)) break;
      const int c = B.j[b0 + q];
      if (!HS_G(B.dbg, c >= 0 && c < B.n, 54, c)) break;
      const int g = c / SEG_W;
      const int gp = q ? B.j[b0 + q - 1] / SEG_W : -1;
      for (int x = gp + 1; x <= g && x <= nseg; ++x) row[x] = (int32_t)q;
      if (q == len - 1)
        for (int x = g + 1; x <= nseg; ++x) row[x] = (int32_t)len;
    }
  }
}

void launch_build_bci(const RightOp &B, int nseg, int min_len, int64_t max_rows, int32_t *bci_id, int32_t *bci,
                      int *counter, cudaStream_t st) {
  if (B.m <= 0) return;
  count_launch();
  k_build_bci<<<grid_for(B.m, 8, 16), 256, 0, st>>>(B, nseg, min_len, max_rows, bci_id, bci, counter);
}

// one warp: exclusive scan of the NKEYS counters into offsets and cursors
__global__ void k_key_offsets(const int *cnt, int *off, int *cur) {
  const int lane = lane_id();
  const int a = cnt[2 * lane], b = cnt[2 * lane + 1];
  const int incl = warp_incl_scan(a + b);
  const int ex = incl - a - b;
  off[2 * lane] = ex;
  off[2 * lane + 1] = ex + a;
  cur[2 * lane] = ex;
  cur[2 * lane + 1] = ex + a;
  if (lane == 31) off[NKEYS] = incl;
}
static_assert(NKEYS == 64, "k_key_offsets assumes 64 keys");

void launch_key_offsets(const int *key_cnt, int *key_off, int *key_cur, cudaStream_t st) {
  count_launch();
  k_key_offsets<<<1, 32, 0, st>>>(key_cnt, key_off, key_cur);
}

// append row r to the list of its key; lanes with equal keys share one atomic
__device__ __forceinline__ void append_row(int key, int r, int *key_cur, int *list, int64_t cap, long long *dbg) {
  const unsigned act = __activemask();
  const unsigned grp = __match_any_sync(act, key);
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if (lane_id() == leader) base = atomicAdd(key_cur + key, __popc(grp));
  base = __shfl_sync(grp, base, leader);
  const int64_t at = base + __popc(grp & ((1u << lane_id()) - 1));
  if (HS_G(dbg, at >= 0 && at < cap, 52, at)) list[at] = r;
}

__global__ void k_scatter_sym(RowSet A, const int64_t *f, int *key_cur, int *list, int32_t *hslot, int *nhist,
                              BinCfg bins) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.nslots;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fr = f[r];
    const int key = sym_key(fr, bins);
    if (key) append_row(key, (int)r, key_cur, list, A.nslots, A.dbg);
    // rows that may need column parts in the numeric pass (every row of the
    // bitmap kernel) get a histogram slot
    const bool h = fr > bins.sym_heavy_from;
    const unsigned act = __activemask();
    const unsigned hm = __ballot_sync(act, h);
    int base = 0;
    const int leader = __ffs(act) - 1;
    if (lane_id() == leader && hm) base = atomicAdd(nhist, __popc(hm));
    base = __shfl_sync(act, base, leader);
    hslot[r] = h ? base + __popc(hm & ((1u << lane_id()) - 1)) : -1;
  }
}

void launch_scatter_sym(const RowSet &A, const int64_t *f, int *key_cur, int *list, int32_t *hslot, int *nhist,
                        const BinCfg &bins, cudaStream_t st) {
  if (A.nslots == 0) return;
  count_launch();
  k_scatter_sym<<<grid_for(A.nslots, 256, 8), 256, 0, st>>>(A, f, key_cur, list, hslot, nhist, bins);
}

__device__ __forceinline__ int64_t out_count(const RowSet &A, const int64_t *Cp, int64_t r) {
  const int64_t o = A.ids ? A.ids[r] : r;
  return Cp[o + 1] - Cp[o];
}

__global__ void k_num_count(RowSet A, const int64_t *f, const int64_t *Cp, BinCfg bins, int *key_cnt) {
  __shared__ int hist[NKEYS];
  for (int i = threadIdx.x; i < NKEYS; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.nslots;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int key = num_key(f[r], out_count(A, Cp, r), bins);
    if (key) atomicAdd(hist + key, 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NKEYS; i += blockDim.x)
    if (hist[i]) atomicAdd(key_cnt + i, hist[i]);
}

void launch_num_count(const RowSet &A, const int64_t *f, const int64_t *Cp, const BinCfg &bins, int *key_cnt,
                      cudaStream_t st) {
  if (A.nslots == 0) return;
  count_launch();
  k_num_count<<<grid_for(A.nslots, 256, 8), 256, 0, st>>>(A, f, Cp, bins, key_cnt);
}

__global__ void k_scatter_num(RowSet A, const int64_t *f, const int64_t *Cp, BinCfg bins, int *key_cur,
                              int *list) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.nslots;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int key = num_key(f[r], out_count(A, Cp, r), bins);
    if (key) append_row(key, (int)r, key_cur, list, A.nslots, A.dbg);
  }
}

void launch_scatter_num(const RowSet &A, const int64_t *f, const int64_t *Cp, const BinCfg &bins, int *key_cur,
                        int *list, cudaStream_t st) {
  if (A.nslots == 0) return;
  count_launch();
  k_scatter_num<<<grid_for(A.nslots, 256, 8), 256, 0, st>>>(A, f, Cp, bins, key_cur, list);
}

// ------------------------------------------------------------------- scan
// Inclusive prefix sum of an int64 array, in place: tiles of SCAN_TILE
// elements are scanned by one CTA each; the tile totals are scanned
// recursively and added back.
constexpr int SCAN_NT = 256, SCAN_PER = 8, SCAN_TILE = SCAN_NT * SCAN_PER;

__global__ void k_scan_tiles(int64_t *a, int64_t n, int64_t *tot) {
  __shared__ long long wsum[SCAN_NT / 32 + 1];
  const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + threadIdx.x * SCAN_PER;
  long long v[SCAN_PER];
  long long s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_PER; ++i) {
    v[i] = (base + i < n) ? a[base + i] : 0;
    s += v[i];
  }
  long long incl = warp_incl_scan(s);
  if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long w = threadIdx.x < SCAN_NT / 32 ? wsum[threadIdx.x] : 0;
    long long wi = warp_incl_scan(w);
    if (threadIdx.x < SCAN_NT / 32) wsum[threadIdx.x] = wi - w;
    if (threadIdx.x == 31) wsum[SCAN_NT / 32] = wi;
  }
  __syncthreads();
  long long run = incl - s + wsum[threadIdx.x >> 5];
#pragma unroll
  for (int i = 0; i < SCAN_PER; ++i) {
    run += v[i];
    if (base + i < n) a[base + i] = run;
  }
  if (threadIdx.x == 0 && tot) tot[blockIdx.x] = wsum[SCAN_NT / 32];
}

__global__ void k_scan_add(int64_t *a, int64_t n, const int64_t *tot) {
  if (blockIdx.x == 0) return;
  const int64_t add = tot[blockIdx.x - 1];
  const int64_t base = blockIdx.x * (int64_t)SCAN_TILE;
  for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
    if (base + i < n) a[base + i] += add;
}

int64_t scan_tmp_elems(int64_t n) {
  int64_t t = 0;
  while (n > SCAN_TILE) {
    n = (n + SCAN_TILE - 1) / SCAN_TILE;
    t += n;
  }
  return t + 1;
}

void launch_scan_i64(int64_t *a, int64_t n, int64_t *tmp, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    count_launch();
    k_scan_tiles<<<1, SCAN_NT, 0, st>>>(a, n, nullptr);
    return;
  }
  count_launch();
  k_scan_tiles<<<(unsigned)tiles, SCAN_NT, 0, st>>>(a, n, tmp);
  launch_scan_i64(tmp, tiles, tmp + tiles, st);
  count_launch();
  k_scan_add<<<(unsigned)tiles, SCAN_NT, 0, st>>>(a, n, tmp);
}

// -------------------------------------------------------------- validation
// flag bit 1: a column id outside [0, ncols); bit 2: a row not strictly
// increasing; bit 4: row offsets decreasing.
__global__ void k_validate(const int64_t *p, const int32_t *j, int64_t rows, int64_t ncols, int *flag) {
  const int lane = lane_id();
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
    const int64_t q0 = p[r], q1 = p[r + 1];
    if (q1 < q0) {
      if (lane == 0) atomicOr(flag, 4);
      continue;
    }
    int bad = 0;
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const int c = j[q];
      if (c < 0 || c >= ncols) bad |= 1;
      if (q > q0 && j[q - 1] >= c) bad |= 2;
    }
    bad = __reduce_or_sync(FULL, bad);
    if (lane == 0 && bad) atomicOr(flag, bad);
  }
}

void launch_validate(const int64_t *p, const int32_t *j, int64_t rows, int64_t ncols, int *flag, cudaStream_t st) {
  if (rows <= 0) return;
  count_launch();
  k_validate<<<grid_for(rows, 8, 16), 256, 0, st>>>(p, j, rows, ncols, flag);
}

// ------------------------------------------------------- heavy row parts
// A heavy row's columns are cut into parts of whole SEG_W-column segments:
// a part takes segments in order while its outputs stay within caph and its
// span within `span` segments (a segment holds at most SEG_W <= caph
// outputs, so every segment fits a part of its own; were one to hold more,
// its part would carry its true count, which the numeric kernel rejects);
// parts without outputs are dropped.  One warp per row: the warp stages the
// row's segment counts in shared memory, WP_STAGE at a time, and lane 0 walks
// them (the greedy cut is sequential; plain shared loads keep its chain
// short); `emit(part, seg_lo, seg_hi, pc, done)` runs on lane 0 (done: the
// row's outputs before the part).  Every lane returns the part count.
constexpr int WP_NT = 256;     // threads of the planning kernels
constexpr int WP_STAGE = 256;  // segment counts staged per warp at a time
template <class Emit>
__device__ __forceinline__ int walk_parts(const uint32_t *hist, int nseg, int caph, int span, uint32_t *stage,
                                          Emit &&emit) {
  const int lane = lane_id();
  int start = 0, sum = 0, parts = 0;
  long long done = 0;
  for (int g0 = 0; g0 < nseg; g0 += WP_STAGE) {
    const int lim = min(WP_STAGE, nseg - g0);
    __syncwarp();  // lane 0 is done with the previous counts
    for (int j = lane; j < lim; j += 32) stage[j] = hist[g0 + j];
    __syncwarp();
    if (lane == 0) {
#pragma unroll 8
      for (int j = 0; j < lim; ++j) {
        const int x = (int)stage[j];
        const int g = g0 + j;
        if (g - start >= span || sum + x > caph) {
          if (sum > 0) {
            emit(parts, start, g, sum, done);
            ++parts;
            done += sum;
          }
          start = g;
          sum = 0;
        }
        sum += x;
      }
    }
  }
  if (lane == 0 && sum > 0) {
    emit(parts, start, nseg, sum, done);
    ++parts;
  }
  return __shfl_sync(FULL, parts, 0);
}

__global__ void k_count_parts(RowSet A, const int *list, const int *key_off, int key_lo, const int32_t *hslot,
                              const uint32_t *hist, const int64_t *loff, int nseg, int caph, int span, int64_t nmax,
                              int64_t *cnt, int64_t *cap) {
  const int lane = lane_id();
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lo = key_off[key_lo];
  const int64_t count = key_off[NKEYS] - lo;
  __shared__ uint32_t s_stage[WP_NT / 32][WP_STAGE];
  uint32_t *stage = s_stage[threadIdx.x >> 5];
  for (int64_t w = wid; w < nmax; w += nw) {
    int64_t parts = 0, room = 0;
    if (w < count) {
      const int r = list[lo + w];
      const int h = (r >= 0 && r < A.nslots) ? hslot[r] : -1;
      if (h >= 0 && loff[r] >= 0) {
        parts = walk_parts(hist + (int64_t)h * nseg, nseg, caph, span, stage, [](int, int, int, int, long long) {});
        room = parts * (A.p[r + 1] - A.p[r]);
      }
    }
    if (lane == 0) {
      cnt[w] = parts;
      cap[w] = room;
    }
  }
}

void launch_count_parts(const RowSet &A, const int *list, const int *key_off, int key_lo, const int32_t *hslot,
                        const uint32_t *hist, const int64_t *loff, int nseg, int caph, int span, int64_t nmax,
                        int64_t *cnt, int64_t *cap, cudaStream_t st) {
  if (nmax <= 0) return;
  count_launch();
  k_count_parts<<<grid_for(nmax, WP_NT / 32, 16), WP_NT, 0, st>>>(A, list, key_off, key_lo, hslot, hist, loff, nseg, caph,
                                                       span, nmax, cnt, cap);
}

__global__ void k_plan_parts(RowSet A, const int *list, int count, const int32_t *hslot, const uint32_t *hist,
                             const int64_t *loff, const int64_t *Cp, int nseg, int caph, int span,
                             const int64_t *off, const int64_t *poff, HeavyUnit *units) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ uint32_t s_stage[WP_NT / 32][WP_STAGE];
  uint32_t *stage = s_stage[threadIdx.x >> 5];
  for (int64_t w = wid; w < count; w += nw) {
    const int r = list[w];
    const int h = (r >= 0 && r < A.nslots) ? hslot[r] : -1;
    if (h < 0 || loff[r] < 0) continue;
    const int64_t base = w ? off[w - 1] : 0;
    const int64_t end = off[w];
    const int64_t pbase = w ? poff[w - 1] : 0;
    const int64_t nq = A.p[r + 1] - A.p[r];
    const int64_t o = A.ids ? (int64_t)A.ids[r] : (int64_t)r;
    const int64_t cb = Cp[o], c = Cp[o + 1] - cb, lb = loff[r];
    walk_parts(hist + (int64_t)h * nseg, nseg, caph, span, stage, [&](int p, int s0, int s1, int pc, long long done) {
      // a part must lie inside its row (else pc 0: the numeric kernel rejects the unit)
      const bool fits = HS_G(A.dbg, done + pc <= c, 74, done);
      if (base + p < end)
        units[base + p] = HeavyUnit{r, s0, s1, fits ? pc : 0, done, pbase + p * nq, 0, 0, cb + done, lb + done};
    });
  }
}

void launch_plan_parts(const RowSet &A, const int *list, int count, const int32_t *hslot, const uint32_t *hist,
                       const int64_t *loff, const int64_t *Cp, int nseg, int caph, int span, const int64_t *off,
                       const int64_t *poff, HeavyUnit *units, cudaStream_t st) {
  if (count <= 0) return;
  count_launch();
  k_plan_parts<<<grid_for(count, WP_NT / 32, 16), WP_NT, 0, st>>>(A, list, count, hslot, hist, loff, Cp, nseg, caph, span, off,
                                                       poff, units);
}

// One warp per unit: its row's A entries 32 at a time, each entry's B
// segment inside the part from the segment index (or a binary search of a B
// row without one), the non-empty ones compacted by ballot into the unit's
// slice with the running product count as their exclusive prefix.  The
// searches of many units run at once, so their latency is hidden here
// instead of sitting on the numeric kernel's path.
template <int AB>
__global__ void k_build_pairs(RowSet A, RightOp B, HeavyUnit *units, int64_t nunits, const int32_t *bci_id,
                              const int32_t *bci, int nseg, int64_t *pstart, int32_t *ppre, void *paval) {
  using VT = typename std::conditional<AB == 8, unsigned long long, unsigned>::type;
  const int lane = lane_id();
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t bstride = (int64_t)nseg + 1;
  for (int64_t ui = wid; ui < nunits; ui += nw) {
    const HeavyUnit u = units[ui];
    if (!HS_G(A.dbg, u.row >= 0 && u.row < A.nslots && u.seg_lo >= 0 && u.seg_lo < u.seg_hi && u.seg_hi <= nseg,
              75, ui))
      continue;
    const int64_t lo = (int64_t)u.seg_lo * SEG_W, hi = (int64_t)u.seg_hi * SEG_W;
    const int64_t q0 = A.p[u.row], q1 = A.p[u.row + 1];
    int out = 0;
    long long prod = 0;
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane;
      int64_t s0 = 0, s1 = 0;
      VT av = 0;
      if (q < q1 && HS_G(A.dbg, q >= 0 && q < A.nnz, 1, q)) {
        const int k = __ldg(A.j + q);
        if (HS_G(A.dbg, k >= 0 && k < B.m, 2, k)) {
          const int64_t base = __ldg(B.p + k), end = __ldg(B.p + k + 1);
          const int t = bci_id ? __ldg(bci_id + k) : -1;
          s0 = s1 = base;  // an empty B row: an empty segment at its start
          if (t >= 0) {
            s0 = base + __ldg(bci + (int64_t)t * bstride + u.seg_lo);
            s1 = base + __ldg(bci + (int64_t)t * bstride + u.seg_hi);
          } else if (end > base) {
            s0 = lower_bound_col(B.j, base, end, (int)lo);
            s1 = hi > 0x7fffffffLL ? end : lower_bound_col(B.j, s0, end, (int)hi);
          }
          if (!HS_G(A.dbg, base <= s0 && s0 <= s1 && s1 <= end, 65, s1)) s0 = s1 = 0;
          if constexpr (AB > 0)
            if (s1 > s0) av = __ldg(reinterpret_cast<const VT *>(A.v) + q);
        }
      }
      const int len = (int)(s1 - s0);
      const unsigned m = __ballot_sync(FULL, len > 0);
      const int incl = warp_incl_scan(len);
      if (len > 0) {
        const int64_t at = u.poff + out + __popc(m & ((1u << lane) - 1u));
        // evict-first: the pairs are read once, later; B and the segment
        // index stay in L2 for this kernel and the unit kernel after it
        __stcs(reinterpret_cast<long long *>(pstart) + at, (long long)s0);
        __stcs(ppre + at, (int32_t)(prod + incl - len));
        if constexpr (AB > 0) __stcs(reinterpret_cast<VT *>(paval) + at, av);
      }
      out += __popc(m);
      prod += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) {
      units[ui].npairs = out;
      units[ui].nprod = HS_G(A.dbg, prod < 0x7fffffffLL, 76, ui) ? (int32_t)prod : 0;
    }
  }
}

void launch_build_pairs(const RowSet &A, const RightOp &B, HeavyUnit *units, int64_t nunits, const int32_t *bci_id,
                        const int32_t *bci, int nseg, int a_bytes, int64_t *pstart, int32_t *ppre, void *paval,
                        cudaStream_t st) {
  if (nunits <= 0) return;
  count_launch();
  const int g = grid_for(nunits, 8, 16);
  if (a_bytes == 8)
    k_build_pairs<8><<<g, 256, 0, st>>>(A, B, units, nunits, bci_id, bci, nseg, pstart, ppre, paval);
  else if (a_bytes == 4)
    k_build_pairs<4><<<g, 256, 0, st>>>(A, B, units, nunits, bci_id, bci, nseg, pstart, ppre, paval);
  else
    k_build_pairs<0><<<g, 256, 0, st>>>(A, B, units, nunits, bci_id, bci, nseg, pstart, ppre, paval);
}

}  // namespace hs
