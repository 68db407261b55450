// internal.h -- declarations shared by the library's translation units
// (host launchers of the kernels and the bin layout).  Not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hs {

// ---------------------------------------------------------------- bins
// Rows are binned by their product count f (flops) before the symbolic pass
// and by (f, output count c) before the numeric pass.  A bin "key" orders the
// concatenated row lists; heavy rows get one key per power of two of f,
// largest first, so dynamic scheduling hands out the longest rows first.
constexpr int NKEYS = 64;
constexpr int KEY_TINY = 1;     // f <= 32: warp, one product per lane
constexpr int KEY_WARP_S = 2;   // numeric: f <= 128: warp, 256-slot table
constexpr int KEY_WARP = 3;     // f <= 512: warp, private shared hash table
constexpr int KEY_MID_S = 4;    // symbolic: f <= 1024;  numeric: c <= 1024
constexpr int KEY_MID = 5;      // symbolic: f <= 4096;  numeric: c <= CAP_MID
constexpr int KEY_LARGE_S = 6;  // numeric: c <= cap_large / 2
constexpr int KEY_LARGE = 7;    // symbolic: f <= min(16384, cap_large); numeric: c <= cap_large
// numeric rows with little compression, one warp sorting 32*K products:
constexpr int KEY_SORT_XS = 8;  // f <= 128 (K = 4)
constexpr int KEY_SORT_S = 9;   // f <= 256 (K = 8)
constexpr int KEY_SORT_M = 10;  // f <= 512 (K = 16)
constexpr int KEY_SORT = 11;    // f <= 1024 (K = 32)
constexpr int KEY_SPA = 12;     // products with few columns (BinCfg::spa): f > 32, a warp's dense accumulator
constexpr int KEY_HEAVY = 13;   // 13 + min(50, 62 - floor(log2 f)): symbolic bitmap / numeric column parts
constexpr int F_TINY = 32, F_WARP_S = 128, F_WARP = 512, F_MID_S = 1024, F_MID = 4096, F_LARGE = 16384;
constexpr int F_SORT_XS = 128, F_SORT_S = 256, F_SORT_M = 512, F_SORT = 1024;
// Sort tiers pack (column - min column) << log2(32K) | product index into 32
// bits for 32*K-product rows; the tiers above 256 products hold no 64-bit
// fallback, so a matrix with at least SORT_PACKED_COLS columns keeps rows
// of more than 256 products out of them (numeric_bins).
constexpr int SORT_WIDE_K = 8;
constexpr int64_t SORT_PACKED_COLS = (1 << 22) - 1;
// Products whose B has at most spa_cols(value bytes) columns may take (tuning
// spa_max), for every row of more than 32 products, one warp's dense
// accumulator of all n columns (Figure 1's SPA as it stands: a value per
// column and an occupancy flag).
constexpr int SPA_COLS_8 = 1024, SPA_COLS_4 = 2048;
__host__ __device__ constexpr int spa_cols(int value_bytes) { return value_bytes == 8 ? SPA_COLS_8 : SPA_COLS_4; }
constexpr int CAP_MID_S = 1024, CAP_MID = 2048;
// Column segments recorded for rows that may need column parts: width SEG_W
// (a multiple of 1024, at most every numeric table's capacity).
constexpr int SEG_W = 4096;
constexpr int HV_SPAN_SEGS = 64;      // segments a heavy column part spans at most (2^18 columns)
constexpr int HU_SPAN_SEGS = 32;      // the same for the parts of the unit kernel (2^17 columns)
constexpr int BITMAP_COLS = 1 << 20;  // columns covered by the heavy symbolic bitmap
constexpr int SEG_SMEM = 1024;        // segment counters kept in shared memory when nseg <= this

__host__ __device__ inline int floor_log2_u64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return 63 - __clzll((long long)x);
#else
  return 63 - __builtin_clzll(x);
#endif
}
// Largest rows first: one key per power of two of f down to 2^12; smaller
// heavy rows (a bitmap threshold below 4096) share the last key, so every key
// stays below NKEYS.
__host__ __device__ inline int heavy_key(int64_t f) {
  const int k = 62 - floor_log2_u64((uint64_t)f);
  return KEY_HEAVY + (k < NKEYS - 1 - KEY_HEAVY ? k : NKEYS - 1 - KEY_HEAVY);
}
// Bin thresholds.  The tier capacities (table sizes) are fixed by the
// kernels; which rows take which tier is set here, at run time (defaults
// below, or a tuning chosen by measurement), within those capacities.
struct BinCfg {
  int cap_large;       // numeric large capacity: 8192 (4-byte values, bool) or 4096 (8-byte)
  int warp_s_max;      // numeric: rows with 32 < f <= this take the 256-slot warp tier (32..128)
  int mid_s_max;       // numeric: rows with c <= this take the 1024-capacity CTA tier (0..1024)
  int large_s_max;     // numeric: rows with CAP_MID < c <= this take the half-capacity large tier
  int sym_mid_s_max;   // symbolic: rows with 512 < f <= this take the warp's 2048-slot tier (512..1024)
  int sym_heavy_from;  // symbolic: rows with f > this take the bitmap kernel (2048..cap_large)
  int sort_max;        // numeric: rows with 32 < f <= this and 100*c >= sort_pct*f sort their products (32..1024)
  int sort_pct;        // (0..101; 101 switches the sort tiers off)
  int spa_max;         // products whose B has at most min(this, spa_cols()) columns take the dense tier (0: none)
  int unit_kb;         // numeric heavy units hold this many KB of values (16 or 32)
  int num_heavy_from;  // numeric: rows with c > this that took the bitmap kernel go to the units (2048..cap_large)
  int spa;             // set per product: rows of more than 32 products take KEY_SPA
};
// Symbolic bins.  Every row that may end in the numeric heavy bin (c >
// cap_large needs f > cap_large) takes the bitmap kernel, which also writes
// the row's sorted column list for the numeric pass.
__host__ __device__ inline int sym_key(int64_t f, const BinCfg &b) {
  if (f <= 0) return 0;
  if (f <= F_TINY) return KEY_TINY;
  if (b.spa) return KEY_SPA;
  if (f <= F_WARP) return KEY_WARP;
  if (f <= b.sym_mid_s_max) return KEY_MID_S;
  if (f <= F_MID && f <= b.sym_heavy_from) return KEY_MID;
  if (f <= F_LARGE && f <= b.sym_heavy_from) return KEY_LARGE;
  return heavy_key(f);
}
// Numeric bins: the smaller tiers take smaller tables, so more of their rows
// are in flight on an SM at once.
__host__ __device__ inline int num_key(int64_t f, int64_t c, const BinCfg &b) {
  if (c <= 0) return 0;
  if (f <= F_TINY) return KEY_TINY;
  if (b.spa) return KEY_SPA;
  if (f <= b.sort_max && c * 100 >= f * b.sort_pct)
    return f <= F_SORT_XS ? KEY_SORT_XS : (f <= F_SORT_S ? KEY_SORT_S : (f <= F_SORT_M ? KEY_SORT_M : KEY_SORT));
  if (f <= b.warp_s_max) return KEY_WARP_S;
  if (f <= F_WARP) return KEY_WARP;
  if (c > b.num_heavy_from && f > b.sym_heavy_from) return heavy_key(f);  // a sorted list exists
  if (c <= b.mid_s_max) return KEY_MID_S;
  if (c <= CAP_MID) return KEY_MID;
  if (c <= b.large_s_max) return KEY_LARGE_S;
  if (c <= b.cap_large) return KEY_LARGE;
  return heavy_key(f);
}
// the default thresholds for a value width, clamped tuning values otherwise
BinCfg bin_config(int value_bytes);
// the thresholds of a product whose B has ncols columns (value_bytes: C's
// value width): the dense-accumulator tier for narrow products, and the sort
// tiers' 64-bit limit for very wide ones
inline BinCfg product_bins(BinCfg b, int64_t ncols, int value_bytes) {
  const int lim = b.spa_max < spa_cols(value_bytes) ? b.spa_max : spa_cols(value_bytes);
  b.spa = (ncols > 0 && ncols <= lim) ? 1 : 0;
  return b;
}
inline BinCfg numeric_bins(BinCfg b, int64_t ncols) {
  if (ncols >= SORT_PACKED_COLS && b.sort_max > F_SORT_S) b.sort_max = F_SORT_S;
  return b;
}

// ---------------------------------------------------------- device views
struct RowSet {          // the left operand's stored rows
  const int64_t *p;      // offsets, nslots+1
  const int32_t *j;      // column ids
  const void *v;         // values or null
  const int32_t *ids;    // DCSR row ids (null for CSR: slot == row)
  int64_t nslots;
  int64_t nnz;
  int64_t m;             // rows of A (and of C)
  long long *dbg;        // guard record (guarded builds)
};
struct RightOp {
  const int64_t *p;
  const int32_t *j;
  const void *v;
  int64_t n;    // columns
  int64_t m;    // rows
  int64_t nnz;
  long long *dbg;
};

// kernel launches issued by this library (all threads), for benchmarks
void count_launch();
unsigned long long launch_total();

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) with the failure kept for
// the driver to report (launchers return void)
cudaError_t &attr_error();
template <class K> inline void set_smem_attr(K kernel, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) attr_error() = e;
}

// --------------------------------------------------------------- launchers
// analysis.cu
// stats[0] total flops, [1] max row flops, [2] max row nnz of A, [3] sum of
// min(f, n) over the rows of the symbolic heavy bin (their list pool bound)
void launch_flops(const RowSet &A, const RightOp &B, int64_t *f, int *key_cnt, unsigned long long *stats,
                  const BinCfg &bins, cudaStream_t st);
// per-entry product counts (s over A's entries, zeros: entries with an
// empty B row), the row counts and keys from their inclusive scan S, and the
// copy of A without the zero entries (p2: nslots+1 offsets from 0)
void launch_entry_flops(const RowSet &A, const RightOp &B, int64_t *s, unsigned long long *zeros, cudaStream_t st);
void launch_row_flops(const RowSet &A, const int64_t *S, int64_t *f, int *key_cnt, unsigned long long *stats,
                      const BinCfg &bins, int64_t bn, cudaStream_t st);
void launch_compact_a(const RowSet &A, const int64_t *S, int64_t *keep, int64_t *scan_tmp, int32_t *j2, void *v2,
                      int vb, int64_t *p2, cudaStream_t st);
// entries of a CSR whose value is not zero (dtype F64, F32, I32 or I64):
// keep flags, then (after their inclusive scan) the compacted copy
void launch_keep_nonzero(const void *v, int dtype, int64_t n, int64_t *keep, cudaStream_t st);
void launch_compact_by_keep(const RowSet &A, const int64_t *K, int32_t *j2, void *v2, int vb, int64_t *p2,
                            cudaStream_t st);
void launch_key_offsets(const int *key_cnt, int *key_off, int *key_cur, cudaStream_t st);
// rows with more than cap_large products get a column-segment histogram slot
void launch_scatter_sym(const RowSet &A, const int64_t *f, int *key_cur, int *list, int32_t *hslot,
                        int *nhist, const BinCfg &bins, cudaStream_t st);
void launch_num_count(const RowSet &A, const int64_t *f, const int64_t *Cp, const BinCfg &bins, int *key_cnt,
                      cudaStream_t st);
void launch_scatter_num(const RowSet &A, const int64_t *f, const int64_t *Cp, const BinCfg &bins, int *key_cur,
                        int *list, cudaStream_t st);
void launch_scan_i64(int64_t *a, int64_t n, int64_t *tmp, cudaStream_t st);  // inclusive, in place
int64_t scan_tmp_elems(int64_t n);
// B segment index: for every B row longer than `min_len`, the offset (within
// the row) of its first entry in each SEG_W-column segment, nseg+1 values
// (the last is the row length).  Rows get consecutive table rows through
// *counter; at most max_rows of them are indexed.
void launch_build_bci(const RightOp &B, int nseg, int min_len, int64_t max_rows, int32_t *bci_id, int32_t *bci,
                      int *counter, cudaStream_t st);
void launch_validate(const int64_t *p, const int32_t *j, int64_t rows, int64_t ncols, int *flag, cudaStream_t st);
void launch_sm_count_init();
int sm_count();

// symbolic.cu: counts go to cnt[out_row + 1] (int64)
struct SymArgs {
  RowSet A;
  RightOp B;
  const int64_t *f;        // flops per row slot
  const int *list;         // rows of the bin
  int count;               // rows in the bin
  int64_t *cnt;            // per output row
  const int32_t *hslot;    // segment-histogram slot per row (-1 none)
  uint32_t *hist;          // nhist x nseg
  int nseg;
  int *dyn;                // dynamic row counter (heavy)
  int *err;
  int32_t *glist;          // heavy rows' sorted column lists (pool of lcap entries), or null
  int64_t *loff;           // per row slot: start of its list in the pool (-1 none)
  unsigned long long *lpool;  // pool cursor (entries handed out)
  int64_t lcap;
};
void launch_sym_tiny(const SymArgs &a, cudaStream_t st);
void launch_sym_warp(const SymArgs &a, cudaStream_t st);
void launch_sym_mid_s(const SymArgs &a, cudaStream_t st);
void launch_sym_mid(const SymArgs &a, cudaStream_t st);
void launch_sym_large(const SymArgs &a, cudaStream_t st);
void launch_sym_heavy(const SymArgs &a, cudaStream_t st);
void launch_sym_spa(const SymArgs &a, cudaStream_t st);


// A unit of the numeric heavy pass: one column part of one heavy row.  The
// part spans segments [seg_lo, seg_hi) of SEG_W columns, holds pc outputs,
// and its outputs start `done` entries into the row (and into the row's
// sorted column list).  Units of one row are independent: they write
// disjoint ranges of C, so any CTA may take any unit.
struct alignas(16) HeavyUnit {
  int32_t row;     // row slot
  int32_t seg_lo;
  int32_t seg_hi;
  int32_t pc;
  int64_t done;
  int64_t poff;    // the unit's slice of the pair arrays (room for every A entry of its row)
  int32_t npairs;  // A entries with products in the part (the slice's used length)
  int32_t nprod;   // products in the part
  int64_t out;     // position in C of the part's first entry (C's row offset + done)
  int64_t lofs;    // position of the part's first column in the sorted-list pool
};
// outputs a heavy column part holds at most, by value width (the part's
// values live in shared memory)
inline int heavy_part_cap(int value_bytes) { return value_bytes == 8 ? 4096 : (value_bytes == 0 ? 16384 : 8192); }
// the same for the unit kernel: kb KB of values (16 or 32, the tuning's
// heavy_part_kb), and never less than one segment's SEG_W columns (structure
// only: 2^16 outputs)
inline int unit_part_cap(int value_bytes, int kb = 16) {
  return value_bytes == 0 ? 65536 : (kb * 1024 / value_bytes > SEG_W ? kb * 1024 / value_bytes : SEG_W);
}
// parts per heavy row (numeric heavy bin, in list order) into cnt[0..nmax),
// 0 for rows without a sorted column list (loff < 0), and the room the row's
// units need in the pair arrays (parts x A entries) into cap[0..nmax); then
// the units themselves at the scanned offsets (off, poff: inclusive scans of
// cnt and cap)
void launch_count_parts(const RowSet &A, const int *list, const int *key_off, int key_lo, const int32_t *hslot,
                        const uint32_t *hist, const int64_t *loff, int nseg, int caph, int span, int64_t nmax,
                        int64_t *cnt, int64_t *cap, cudaStream_t st);
void launch_plan_parts(const RowSet &A, const int *list, int count, const int32_t *hslot, const uint32_t *hist,
                       const int64_t *loff, const int64_t *Cp, int nseg, int caph, int span, const int64_t *off,
                       const int64_t *poff, HeavyUnit *units, cudaStream_t st);
// Each unit's B segments: for every A entry of its row whose B row has
// entries inside the part's columns, (segment start, exclusive prefix of the
// products, the entry's value when the semiring reads it), compacted into the
// unit's slice; sets npairs and nprod.  a_bytes: width of A's values to copy
// (0: none).
void launch_build_pairs(const RowSet &A, const RightOp &B, HeavyUnit *units, int64_t nunits, const int32_t *bci_id,
                        const int32_t *bci, int nseg, int a_bytes, int64_t *pstart, int32_t *ppre, void *paval,
                        cudaStream_t st);

// numeric_*.cu
struct NumArgs {
  RowSet A;
  RightOp B;
  const int64_t *f;
  const int *list;
  int count;
  const int64_t *Cp;
  int32_t *Cj;
  void *Cv;
  const int32_t *hslot;
  const uint32_t *hist;
  int nseg;
  int *dyn;
  int *err;
  int32_t *gcur;  // heavy bin: per-A-entry cursor into its B row (nnz(A) entries)
  int32_t *gend;  // heavy bin: end of the current part's segment
  const int32_t *glist;   // sorted column lists written by the symbolic heavy pass, or null
  const int64_t *loff;    // per row slot: its list (-1 none)
  const int32_t *bci_id;  // per B row: its row of the segment index (-1 none), or null
  const int32_t *bci;     // segment index: nseg+1 offsets per indexed B row
  int unsorted;           // hash bins write their entries in table order (no sort)
  const HeavyUnit *units; // heavy bin by units (rows with sorted lists), or null: one CTA per row
  int64_t nunits;
  int *udyn;              // the unit kernel's work counter
  int lists_partial;      // with units: some heavy rows have no list (the row kernel takes them)
  const int64_t *pstart;  // units' B segments (launch_build_pairs)
  const int32_t *ppre;
  const void *paval;
  int pair_abytes;        // width of the left values the pairs carry (0: none)
  int unit_kb;            // the units' value capacity in KB (16 or 32): which unit kernel runs
};
// kind: 0 tiny, 1 warp_s, 2 warp, 3 mid_s, 4 mid, 5 large_s, 6 large,
// 7 sort_xs, 8 sort_s, 9 sort_m, 10 sort, 11 spa, 12 heavy (bin key
// KEY_TINY + kind; heavy takes every key from KEY_HEAVY on).  dtype codes as
// in the ABI.
constexpr int NUM_KINDS = 13;
bool launch_numeric_pt(int dtype, int kind, const NumArgs &a, cudaStream_t st);
bool launch_numeric_mp(int dtype, int kind, const NumArgs &a, cudaStream_t st);
bool launch_numeric_oa(int kind, const NumArgs &a, cudaStream_t st);
bool launch_numeric_sel(int second, int vbytes, int kind, const NumArgs &a, cudaStream_t st);

// index.cu: selection matrices and the SpAsgn merge
void launch_build_Q_count(const int32_t *J, int64_t nJ, int64_t bound, int64_t *Qp_counts, cudaStream_t st);
void launch_max_count(const int64_t *cnt, int64_t n, unsigned long long *out, cudaStream_t st);
void launch_iota_i32(int32_t *p, int64_t n, cudaStream_t st);
void launch_build_Q_fill(const int32_t *J, int64_t nJ, int64_t *Qcur, int32_t *Qj, cudaStream_t st);
void launch_sort_short_rows(const int64_t *ptr, int32_t *j, int64_t rows, cudaStream_t st);
void launch_check_range(const int32_t *X, int64_t n, int64_t bound, int *flag, cudaStream_t st);
// pos[X[i]] = i for in-range X[i] (bit 1 of flag: out of range; bit 2: repeated)
void launch_mark_positions(const int32_t *X, int64_t n, int64_t bound, int32_t *pos, int *flag, cudaStream_t st);
void launch_fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t st);
// SpRef by gathering the selected rows (index.cu)
struct GatherArgs {
  const int64_t *Ap;
  const int32_t *Aj;
  const void *Av;
  int vb;
  const int32_t *I;
  const int64_t *G;    // nI + 1 gathered offsets
  const int64_t *row;  // scanned row starts: row of g = row[g] - 1
  const int64_t *Qp;   // n + 1
  const int32_t *Qj;
  int64_t total;       // gathered entries
  int64_t ncols;       // columns of A: a column id outside [0, ncols) makes no tuple
};
void launch_gather_len(const int64_t *Ap, const int32_t *I, int64_t nI, int64_t *G, cudaStream_t st);
void launch_row_starts(const int64_t *G, int64_t nI, int64_t total, int64_t *inc, cudaStream_t st);
void launch_gather_w(const GatherArgs &a, int64_t *W, cudaStream_t st);
void launch_gather_fill(const GatherArgs &a, const int64_t *W, int32_t *ti, int32_t *pj, void *tv, cudaStream_t st);
void launch_gather_direct(const GatherArgs &a, const int64_t *W, int32_t *Bj, void *Bv, cudaStream_t st);
void launch_gather_offsets(const int64_t *G, int64_t nI, const int64_t *W, int64_t *Bp, cudaStream_t st);
void launch_check_increasing(const int32_t *X, int64_t n, int *flag, cudaStream_t st);

// sparse.cu: sparse(i, j, v, m, n) by a stable radix sort of (row, column)
// keys.  Tiles of sp_tiles(nnz); look-back status of 256 words per tile.
int64_t sp_tiles(int64_t nnz);
int sp_radix_bits();
int64_t sp_long_capacity(int64_t nnz);  // runs longer than the emit kernel folds alone
int sp_max_passes();
// flag bit 1: an index out of range; bit 2: a look-back wait expired.
// spin_limit: polls of one look-back word before giving up (sp_spin_limit()
// in production); withhold: a tile that never publishes its counts (-1: none;
// failure-detection tests only)
int sp_spin_limit();
void launch_sp_allhist(const int32_t *I, const int32_t *J, int64_t nnz, int nbj, int64_t m, int64_t n, int passes,
                       unsigned long long *ghist, int *flag, cudaStream_t st);
void launch_sp_pass(int vb, const uint64_t *Kin, const int32_t *I, const int32_t *J, const void *Vin, int64_t nnz,
                    int nbj, int64_t m, int64_t n, int pass, const unsigned long long *ghist,
                    unsigned long long *status, int *ticket, int64_t ntiles, uint64_t *Kout, void *Vout, int *flag,
                    int spin_limit, long long withhold, cudaStream_t st);
void launch_sp_heads(const uint64_t *K, int64_t nnz, int64_t *theads, int64_t ntiles, cudaStream_t st);
// op: 0 (+) f64, 1 (+) f32, 2 (+) i64, 3 min f32, 4 min i32, 5 structure only
void launch_sp_emit(int op, const uint64_t *K, const void *V, int64_t nnz, int nbj, const int64_t *theads_incl,
                    int64_t ntiles, int32_t *Cidx, void *Cval, int64_t *rowcnt, int64_t *longlist, int *nlong,
                    cudaStream_t st);
void launch_rows_from_pos(const int32_t *pos, int64_t m, int64_t *cnt, cudaStream_t st);
void launch_fill_from_pos(const int32_t *pos, int64_t m, const int64_t *ptr, int32_t *out, cudaStream_t st);
void launch_iota_i64(int64_t *p, int64_t n, cudaStream_t st);
void launch_add_i64(int64_t *p, int64_t n, int64_t add, cudaStream_t st);  // p[i] += add
struct AsgnArgs {
  const int64_t *Ap; const int32_t *Aj; const void *Av;   // A (m x n)
  const int64_t *Xp; const int32_t *Xj; const void *Xv;   // X = R*B*Q (m x n)
  const int32_t *rpos;  // m: row in I or -1
  const int32_t *cpos;  // n: column in J or -1
  int64_t m;
  int vbytes;           // value width (0 for bool)
  int accumulate;
  int add_kind;         // semiring for extend-add collisions
  int dtype;
  int64_t *Cp;          // counts then offsets
  int32_t *Cj;
  void *Cv;
};
void launch_asgn_count(const AsgnArgs &a, cudaStream_t st);
void launch_asgn_fill(const AsgnArgs &a, cudaStream_t st);

}  // namespace hs
