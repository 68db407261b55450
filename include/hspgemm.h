/*
 * hspgemm.h -- C ABI of libhspgemm: sparse matrix-matrix multiplication over a
 * semiring (SpGEMM), sparse indexing (SpRef) and sparse assignment (SpAsgn)
 * on one NVIDIA GB300 GPU.
 *
 * The operations are those of Buluc & Gilbert, "Parallel Sparse Matrix-Matrix
 * Multiplication and Indexing: Implementation and Experiments" (SIAM J. Sci.
 * Comput. 2012):
 *   - SpGEMM C = A*B over a semiring (Section 1; Algorithm 1; Section 2.1),
 *   - SpRef  B = A(I,J) computed as the triple product R*A*Q with 0/1
 *     selection matrices (Section 3.1, SpRef listing and Figure "spref"),
 *   - SpAsgn A(I,J) = B computed as A + R*B*Q - S*A*T, the subtraction being
 *     an elementwise product with the structural negation of S*A*T
 *     (Section 3.1, SpAsgn listing and the theorem after it),
 *   - Liu's extend-add A(I,J) = A(I,J) + B (Section 3),
 *   - the constructor sparse(i, j, v, m, n) with repeated positions combined
 *     (Section 2's notation).
 *
 * Conventions shared by every entry point
 *   - Indices are 0-based (the paper is 1-based).  Column ids are int32, row
 *     offsets int64, so nnz may exceed 2^31.
 *   - Matrices are canonical: within a row, column ids strictly increase.
 *     Outputs are always canonical.  Inputs are checked only when
 *     HS_FLAG_VALIDATE is passed (then a violation returns HS_ENONCANON).
 *   - All matrix arrays are DEVICE pointers on the current CUDA device.  The
 *     library never modifies its inputs.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream ordered.  Each product performs two small
 *     device->host reads of sizes and therefore two host synchronisations
 *     with `stream` (after binning and after the symbolic pass).
 *   - Outputs and temporaries are allocated through `alloc` (see
 *     hs_allocator); with alloc == NULL the library uses cudaMallocAsync /
 *     cudaFreeAsync on `stream`.  Output arrays are owned by the caller and
 *     released with hs_mat_free (or by the caller's own allocator).
 *   - Every call returns HS_OK (0) or a negative status; on failure no output
 *     memory is left allocated.
 */
#ifndef HSPGEMM_H
#define HSPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Semirings (Section 1: the product is defined over any semiring; Section
 * 3.1: SpRef and SpAsgn multiply a 0/1 selection matrix with a matrix of any
 * value type, here the two selector semirings). */
typedef enum {
  HS_PLUS_TIMES = 0, /* (+, x): F64, F32, I64                                  */
  HS_OR_AND = 1,     /* (or, and): structure only; output dtype HS_BOOL         */
  HS_MIN_PLUS = 2,   /* (min, +): F32, I32                                      */
  HS_SELECT2ND = 3,  /* mul(a,b) = b: A is a 0/1 selector (any dtype, values
                        ignored); every output entry must receive exactly one
                        contribution, else which one is kept is unspecified   */
  HS_SELECT1ST = 4   /* mul(a,b) = a: B is the selector; same rule            */
} hs_semiring;

/* Value types; HS_BOOL matrices carry no value array (val == NULL). */
typedef enum { HS_F64 = 0, HS_F32 = 1, HS_I32 = 2, HS_I64 = 3, HS_BOOL = 4 } hs_dtype;

/* Storage formats (Section 2.2).  HS_DCSR is the row analogue of DCSC: only
 * non-empty rows are stored; ids[r] is the id of the r-th stored row and
 * ptr has nzr+1 entries.  Accepted for the left operand A of hs_spgemm; all
 * other operands and every output are HS_CSR. */
typedef enum { HS_CSR = 0, HS_DCSR = 1 } hs_format;

typedef struct hs_mat {
  int32_t fmt;   /* hs_format                                           */
  int32_t dtype; /* hs_dtype                                            */
  int64_t m, n;  /* shape                                               */
  int64_t nnz;   /* stored entries (== ptr[rows])                       */
  int64_t nzr;   /* HS_DCSR: number of stored rows; ignored for HS_CSR  */
  int64_t *ptr;  /* row offsets: m+1 (CSR) or nzr+1 (DCSR), int64       */
  int32_t *idx;  /* column ids, nnz                                     */
  int32_t *ids;  /* HS_DCSR: stored row ids, nzr, increasing; else NULL */
  void *val;     /* values, nnz * sizeof(dtype); NULL for HS_BOOL       */
} hs_mat;

/* Stream-ordered device allocator.  alloc returns device memory usable on
 * `stream` (NULL on failure -> HS_ENOMEM); free releases it on `stream`. */
typedef struct hs_allocator {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
  void *ctx;
} hs_allocator;

/* Status codes. */
#define HS_OK 0
#define HS_EINVAL -1       /* bad shape, dtype/semiring pair, pointer or index */
#define HS_ENONCANON -2    /* input row not strictly increasing (validation)   */
#define HS_EDUP -3         /* duplicate index in SpAsgn I or J                 */
#define HS_ENOMEM -4       /* allocator returned NULL                          */
#define HS_ETIMEDOUT -5    /* a bounded device-side wait expired               */
#define HS_ECUDA -6        /* CUDA runtime error (see hs_last_cuda_error)      */
#define HS_EUNSUPPORTED -7 /* valid request this build does not implement    */
#define HS_EINTERNAL -8    /* device-side consistency check failed            */
#define HS_ESCRATCH -9     /* hs_spgemm_noalloc: the product needs more scratch
                              than HS_NOALLOC_SCRATCH_MAX bytes                */
#define HS_ECAPACITY -10   /* hs_spgemm_noalloc / hs_spgemm_to_host: output
                              capacity too small                               */

/* Flags. */
#define HS_FLAG_VALIDATE 1u      /* check canonical inputs and index ranges */
#define HS_FLAG_STAGE_ON_DEVICE 2u /* hs_spgemm_to_host: compute C in device memory and
                                      copy it, even into host memory the GPU maps */
#define HS_FLAG_UNSORTED 4u    /* hs_spgemm, hs_spgemm_batched, hs_spgemm_to_host,
                                  hs_plan_create: rows of C may
                                  come out in any column order (the hash bins skip their
                                  sort); such a C is not canonical and must not be passed
                                  where a canonical operand is expected */
#define HS_FLAG_PRUNE_ZEROS 8u /* hs_spgemm and hs_spgemm_batched with HS_PLUS_TIMES: remove
                                  the entries of C whose
                                  sum is exactly zero (+0 or -0) by one compaction of C (one
                                  more host synchronisation; C's arrays are reallocated, so
                                  two copies of C are live for a moment); other semirings and
                                  entry points ignore it */

/* C = A*B over `semiring` (Section 1; Algorithm 1 and Section 2.1).
 * A: m x k, CSR or DCSR.  B: k x n, CSR.  C: m x n CSR, filled in by the
 * call (C->ptr, C->idx, C->val allocated through `al`).  For HS_PLUS_TIMES
 * and HS_MIN_PLUS, A and B share one dtype, which C gets; HS_OR_AND gives
 * an HS_BOOL C; HS_SELECT2ND gives B's dtype, HS_SELECT1ST A's.
 * Floating-point sums are formed in the input precision, in an unspecified
 * order.  Explicit entries are never dropped: C's structure is the symbolic
 * product of A's and B's structures.  Errors: HS_EINVAL (shapes, dtypes,
 * NULL pointers), HS_ENONCANON (with HS_FLAG_VALIDATE), HS_ENOMEM, HS_ECUDA,
 * HS_EINTERNAL. */
int hs_spgemm(int semiring, const hs_mat *A, const hs_mat *B, hs_mat *C,
              const hs_allocator *al, void *stream, uint32_t flags);

/* B = A(I,J) (Section 3; SpRef listing of Section 3.1): B is len(I) x len(J),
 * row t of B is row I[t] of A and column p of B is column J[p] of A.  I and J
 * are int32 device arrays, any order, duplicates allowed (they repeat
 * rows/columns).  This is the product R*A*Q with R = sparse(1:len(I), I, 1)
 * and Q = sparse(J, 1:len(J), 1), evaluated without forming R*A: the rows
 * I[t] are gathered, each entry (I[t], c) becomes (t, p) for every p with
 * J[p] == c, and the entries are ordered by a stable radix sort (none when J
 * is strictly increasing).  Values are copied bit for bit.  Index ranges are
 * always checked; with HS_FLAG_VALIDATE, A is checked to be canonical too.
 * At most 2^31-1 entries of B unless J is strictly increasing; three or four
 * host synchronisations with `stream`.  Errors: HS_EINVAL (an index out of
 * range, bad shapes, NULL pointers), HS_ENONCANON (with HS_FLAG_VALIDATE),
 * HS_EUNSUPPORTED, HS_ENOMEM, HS_ECUDA. */
int hs_spref(const hs_mat *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ,
             hs_mat *B, const hs_allocator *al, void *stream, uint32_t flags);

/* C = A with A(I,J) = B (accumulate == 0; SpAsgn listing of Section 3.1) or
 * A(I,J) = A(I,J) + B (accumulate != 0; extend-add).  A: m x n CSR,
 * B: len(I) x len(J) CSR of A's dtype.  I and J: int32 device arrays without
 * duplicates (HS_EDUP otherwise).  Assignment removes every entry of A inside
 * the I x J block (the structural negation of S*A*T) and inserts B's entries
 * (R*B*Q); extend-add combines colliding entries with `add_semiring`'s add
 * (HS_PLUS_TIMES or HS_MIN_PLUS; HS_OR_AND for HS_BOOL).  Values are copied
 * bit for bit except where extend-add combines two.  Errors: HS_EINVAL,
 * HS_EDUP, HS_ENOMEM, HS_ECUDA. */
int hs_spasgn(const hs_mat *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ,
              const hs_mat *B, int accumulate, int add_semiring, hs_mat *C,
              const hs_allocator *al, void *stream, uint32_t flags);

/* C = sparse(i, j, v, m, n) (Section 2's constructor): the m x n CSR matrix
 * with C(i[k], j[k]) = v[k] for k < nnz.  Tuples that name the same position
 * are combined with `add_semiring`'s add: HS_PLUS_TIMES sums (dtype HS_F64,
 * HS_F32 or HS_I64), HS_MIN_PLUS keeps the minimum (HS_F32, HS_I32), HS_OR_AND
 * builds the structure only (HS_BOOL; v is ignored and may be NULL).  i, j:
 * int32 device arrays of nnz indices in [0,m) and [0,n), any order; v: device
 * array of nnz values of `dtype`.  Every position named by a tuple is stored,
 * even where its values sum to zero.  Integer sums wrap modulo 2^64;
 * floating-point sums are formed in the value type.  Computed by a stable
 * radix sort of the keys (i, j) that carries v, so the tuples of a position
 * are folded in input order (runs of more than 32 tuples: in 32 consecutive
 * slices, folded in order) and results are deterministic.  Temporaries: two
 * key arrays (8 bytes per tuple) and two value arrays; one host
 * synchronisation with `stream`.  Errors: HS_EINVAL (an index out of range --
 * always checked --, a dtype/semiring pair not listed, NULL pointers),
 * HS_EUNSUPPORTED (nnz, m or n above 2^31-1), HS_ENOMEM, HS_ECUDA. */
int hs_sparse(const int32_t *i, const int32_t *j, const void *v, int64_t nnz, int64_t m, int64_t n,
              int dtype, int add_semiring, hs_mat *C, const hs_allocator *al, void *stream,
              uint32_t flags);

/* Many independent products C_i = A_i * B_i, i < count, in one pass of the
 * pipeline (the batched form; Section 1's SpGEMM applied to a batch): the
 * problems are stacked into one block-diagonal product, so rows of every
 * problem share the same bins and launches, and the batch costs one launch
 * per phase and two host synchronisations.  A[i], B[i]: CSR descriptors of
 * device arrays (A[i].n == B[i].m; one dtype for all A, one for all B).  On
 * return C is the stacked result (sum of A[i].m rows, max B[i].n columns,
 * local column ids) allocated through `al`, and row_offsets (host array of
 * count+1) gives problem i's rows [row_offsets[i], row_offsets[i+1]) of C.
 * Semirings and dtypes as for hs_spgemm.  Errors: HS_EINVAL (shapes, mixed
 * dtypes, NULL pointers), HS_EUNSUPPORTED (more than 2^31-1 stacked rows of
 * B), HS_ENOMEM, HS_ECUDA, and those of hs_spgemm. */
int hs_spgemm_batched(int semiring, int64_t count, const hs_mat *A, const hs_mat *B, hs_mat *C,
                      int64_t *row_offsets, const hs_allocator *al, void *stream, uint32_t flags);

/* C = A*B delivered to host memory, with the copies overlapped: A's rows are
 * cut into nblocks consecutive blocks; each block's product is computed on
 * `stream` while the previous block's rows travel to the host on a stream of
 * the call's own.  A must be CSR.  h_ptr (A->m + 1 int64), h_idx (capacity
 * int32) and h_val (capacity values of C's dtype; unused for bool) are host
 * arrays, best page-locked (cudaHostAlloc) for full copy bandwidth.  On
 * success they hold C in CSR (offsets from 0) and *nnz_out = nnz(C).  If
 * nnz(C) > capacity the call returns HS_ECAPACITY with *nnz_out the size
 * needed (blocks that fit were copied; call again with larger arrays).
 * With nblocks = 1 and arrays in page-locked host memory that the GPU maps
 * (cudaHostAlloc / cudaHostRegister under unified addressing), the numeric
 * kernels store C's columns and values straight into h_idx / h_val while
 * they run (over NVLink-C2C on Grace systems; C then needs no device memory)
 * and only the row offsets are copied afterwards, unless
 * HS_FLAG_STAGE_ON_DEVICE is set; otherwise each block is computed in device
 * memory and copied.  Temporaries come from a memory pool of the library's own on the
 * current device, which keeps its memory for later calls until
 * hs_trim_memory().
 * Same semirings, dtypes, results and errors as hs_spgemm; the call returns
 * when everything is on the host. */
int hs_spgemm_to_host(int semiring, const hs_mat *A, const hs_mat *B, int64_t nblocks, int64_t *h_ptr,
                      int32_t *h_idx, void *h_val, int64_t capacity, int64_t *nnz_out, void *stream,
                      uint32_t flags);
/* Waits for the current device and returns the memory the library's own pool
 * keeps (see hs_spgemm_to_host) to the system.  HS_OK or HS_ECUDA. */
int hs_trim_memory(void);

/* Row-bin thresholds (process-wide; every later call on any thread uses
 * them).  Rows are binned by their product count f and output count c, and
 * each bin runs the accumulator sized for it (Sections 2.1-2.2: work follows
 * the row, not the dimension).  The tables' capacities are fixed; these
 * thresholds decide which rows take the smaller tiers, whose smaller tables
 * leave room for more rows in flight per SM.  Values are clamped to what the
 * tiers hold:
 *   warp_s_max      numeric rows with 32 < f <= warp_s_max take 256-slot warp
 *                   tables, the others up to f = 512 take 1024 (32..128; 128)
 *   mid_s_max       numeric rows with f > 512 and c <= mid_s_max take the
 *                   1024-output CTA tier, the others up to 2048 the next (0..1024; 1024)
 *   large_s_max     numeric rows with 2048 < c <= large_s_max take the tier
 *                   of half the large capacity (2048..4096 for 4-byte values
 *                   and bool; that tier is empty for 8-byte values; 4096)
 *   sym_mid_s_max   symbolic rows with 512 < f <= sym_mid_s_max take one
 *                   warp's 2048-slot table, the others up to f = 4096 a CTA's
 *                   8192 (512..1024; 1024)
 *   sym_heavy_from  symbolic rows with f > sym_heavy_from take the bitmap
 *                   kernel that also writes their sorted column lists
 *                   (2048..large capacity; 0 = automatic: 4096 for 4-byte
 *                   values and bool, the large capacity for 8-byte)
 *   sort_max        numeric rows with 32 < f <= sort_max whose output count
 *   sort_pct        c is at least sort_pct percent of f sort their products
 *                   in a warp's registers (expand, sort, compress) instead of
 *                   hashing them (sort_max 32..1024, 1024; sort_pct 0..101,
 *                   50; 101 switches the sort tiers off)
 *   spa_max         products whose B has at most spa_max columns (at most
 *                   2048, 1024 for 8-byte values) give every row of more
 *                   than 32 products one warp's dense accumulator of all the
 *                   columns (Figure 1's SPA) instead of the tiers above
 *                   (0..2048; 0 = never)
 *   heavy_part_kb   shared memory of values a column part of a heavy row
 *                   holds: 16 (four CTAs per SM) or 32 (half the parts,
 *                   three CTAs per SM); 16
 *   num_heavy_from  numeric rows with more than num_heavy_from outputs whose
 *                   structure came from the bitmap kernel (f > sym_heavy_from)
 *                   take the column-part units instead of a CTA hash table
 *                   (2048..large capacity; 0 = automatic: 2048 for 4-byte
 *                   values and bool, the large capacity for 8-byte)
 * Results do not depend on the thresholds.  hs_set_tuning(NULL) restores the
 * defaults (given last above).  Both calls return HS_OK (hs_get_tuning:
 * HS_EINVAL for NULL). */
typedef struct hs_tuning {
  int32_t warp_s_max, mid_s_max, large_s_max, sym_mid_s_max, sym_heavy_from;
  int32_t sort_max, sort_pct;
  int32_t spa_max;
  int32_t heavy_part_kb;
  int32_t num_heavy_from;
} hs_tuning;
int hs_set_tuning(const hs_tuning *t);
int hs_get_tuning(hs_tuning *t);

/* Symbolic once, numeric many times.  In a multigrid setup the Galerkin
 * product R*A*R^T of Section 4.3.2 is recomputed whenever A's values change
 * while every structure stays the same; a batch of products can be rerun the
 * same way.  hs_plan_create computes C = A*B exactly as hs_spgemm does (same
 * arguments, results, errors and allocations of C) and keeps, in a plan,
 * everything its numeric pass needs: the row bins, the heavy rows' column
 * lists, the B segment index and the scratch, allocated through `al` (which
 * must stay valid until hs_plan_destroy).
 *
 * hs_plan_execute recomputes C's values from new value arrays of A and B
 * (device pointers, same dtypes and entry order as at creation) into C_val
 * (c->nnz values of C's dtype; may be C->val).  It rewrites C->idx with the
 * same column ids, so C->ptr and C->idx, and A's and B's ptr/idx/ids arrays,
 * must stay allocated and unchanged while the plan is used.  A_val (B_val) may
 * be NULL where the semiring ignores that operand's values.  The call only
 * enqueues kernels (and one 4-byte memset) on `stream`: it allocates nothing
 * and never waits for the GPU, so it can be captured in a CUDA graph and
 * replayed.  Executions of one plan must not overlap (they share its scratch).
 * Device-side checks raised during executes are reported by hs_plan_status,
 * which synchronises with `stream`: HS_OK or HS_EINTERNAL.
 *
 * hs_plan_destroy releases the plan's scratch on `stream` (C is the caller's
 * and is released with hs_mat_free). */
typedef struct hs_plan hs_plan;
int hs_plan_create(int semiring, const hs_mat *A, const hs_mat *B, hs_mat *C, hs_plan **plan,
                   const hs_allocator *al, void *stream, uint32_t flags);
int hs_plan_execute(const hs_plan *plan, const void *A_val, const void *B_val, void *C_val, void *stream);
int hs_plan_status(const hs_plan *plan, void *stream);
void hs_plan_destroy(hs_plan *plan, void *stream);

/* The stacked operands of a batch: SA holds A_0..A_{count-1} one after the
 * other (rows concatenated, column ids shifted to the stacked rows of SB), SB
 * holds B_0..B_{count-1} likewise (local column ids), so SA*SB is the block
 * diagonal product whose rows row_offsets[i]..row_offsets[i+1] are A_i*B_i.
 * Same requirements on the inputs as hs_spgemm_batched; SA and SB are
 * allocated through `al`, owned by the caller and released with hs_mat_free.
 * hs_spgemm_batched is this call, one hs_spgemm and the release of SA, SB. */
int hs_batch_stack(int64_t count, const hs_mat *A, const hs_mat *B, hs_mat *SA, hs_mat *SB,
                   int64_t *row_offsets, const hs_allocator *al, void *stream);

/* Batched products in one persistent launch (the paper has no counterpart:
 * many independent products C_i = A_i * B_i, uneven in size, served at once).
 * hs_batch_plan_create stacks the problems as hs_batch_stack does (A_i and B_i
 * are read only here), finds each row's products once (one host
 * synchronisation) and allocates C with room for the flop bound
 * sum_r min(f_r, n); nothing is computed yet.  Semirings and dtypes as
 * hs_spgemm: (+,x) F64/F32/I64, (min,+) F32/I32, (or,and) BOOL.  Rows with
 * more than 4096 products are not taken (HS_EUNSUPPORTED: use
 * hs_spgemm_batched).
 * hs_batch_plan_execute computes C: one memset of the plan's work counters
 * and one cooperative kernel whose resident CTAs take rows from atomic
 * counters through four phases (products per row, distinct columns per row,
 * row offsets, values) separated by grid-wide barriers with bounded waits.
 * It allocates nothing and does not synchronise with the host, so it can be
 * captured in a CUDA graph and replayed; each execution recomputes C from the
 * stacked inputs.
 * hs_batch_plan_result (one host synchronisation) describes the last
 * execution's C: the stacked product whose rows row_offsets[i] ..
 * row_offsets[i+1] are C_i (local column ids), with arrays owned by the plan
 * (valid until the next execution or hs_batch_plan_destroy), and returns
 * HS_ETIMEDOUT if a barrier wait expired, HS_EUNSUPPORTED if a row did not fit
 * the kernel's tables, HS_EINTERNAL after a failed device check.
 * row_offsets (host, count + 1 entries) may be null. */
typedef struct hs_batch_plan hs_batch_plan;
int hs_batch_plan_create(int semiring, int64_t count, const hs_mat *A, const hs_mat *B, hs_batch_plan **plan,
                         const hs_allocator *al, void *stream, uint32_t flags);
int hs_batch_plan_execute(hs_batch_plan *plan, void *stream);
int hs_batch_plan_result(hs_batch_plan *plan, hs_mat *C, int64_t *row_offsets, void *stream);
void hs_batch_plan_destroy(hs_batch_plan *plan, void *stream);
/* Profiling: the last execution's phase times in milliseconds, from the GPU's
 * global timer read by the first CTA at the grid barriers (ms[0] products per
 * row, ms[1] distinct columns, ms[2] row offsets, ms[3] values, ms[4] the
 * whole kernel, ending when the last CTA leaves).  One host synchronisation.
 * HS_EINVAL for NULL arguments. */
int hs_batch_plan_phase_ms(hs_batch_plan *plan, double *ms, void *stream);

/* SpGEMM for callers that cannot allocate device memory while they run (the
 * paper has no counterpart): for example code that has given the GPU's memory
 * to its own pool and must keep its footprint fixed, or code running where a
 * cudaMalloc is not allowed.  Same operation, semirings, dtypes and results
 * as hs_spgemm, but this call allocates nothing: the caller passes C with
 * C->ptr (A->m + 1 int64), C->idx (capacity int32) and, for typed results,
 * C->val (capacity values) already allocated on the device.  The call fills
 * C->ptr, C->idx, C->val and sets C's shape, dtype and nnz.  Temporaries come
 * from one fixed device array of HS_NOALLOC_SCRATCH_MAX bytes inside the
 * library, which every GPU that loads the library holds until the process
 * exits; host-side readbacks use ordinary host memory.
 *   - HS_ESCRATCH: the product needs more scratch than the maximum (roughly
 *     16 bytes per row of A, plus 4 bytes per 4096 columns for every row of
 *     the symbolic bitmap kernel (more than sym_heavy_from products: 4096 by
 *     default) and 8 bytes per entry of A when such rows exist); nothing is
 *     written but
 *     C->ptr, and C->nnz is 0.
 *   - HS_EINVAL: besides the checks of hs_spgemm, a missing A->ptr or B->ptr
 *     (operand with rows), A->idx or B->idx (operand with entries), C->ptr,
 *     or C->idx / C->val with capacity > 0; found before any CUDA call.
 *   - HS_ECAPACITY: nnz(C) > capacity; C->ptr is complete and C->nnz holds
 *     the capacity needed, so the caller can provide larger arrays and call
 *     again.  C->idx and C->val are not touched.
 * The first call on a device looks up the fixed array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the array and leaves its
 * contents behind; each call clears what must start at zero.  Calls that
 * overlap on the GPU (two streams or two host threads on one device) race on
 * the array and must be serialised by the caller.  The call synchronises
 * with `stream` three times (sizes, nnz(C), final error check). */
#define HS_NOALLOC_SCRATCH_MAX (32u * 1024u * 1024u)
int hs_spgemm_noalloc(int semiring, const hs_mat *A, const hs_mat *B, hs_mat *C, int64_t capacity,
                      void *stream);

/* Releases the arrays of a matrix produced by this library through `al` (the
 * allocator it was produced with) and zeroes the descriptor. */
void hs_mat_free(hs_mat *M, const hs_allocator *al, void *stream);

/* Human-readable name of a status code (static storage). */
const char *hs_strerror(int status);

/* The cudaError_t value behind the last HS_ECUDA on this host thread. */
int hs_last_cuda_error(void);

/* A one-line description of the last failure on this host thread (the phase
 * and the CUDA error or failed check), or "" (static thread-local storage). */
const char *hs_last_error_detail(void);

/* Library version as major*10000 + minor*100 + patch. */
int hs_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices); differences around a region count its launches. */
int64_t hs_launch_count(void);

/* Failure-detection test hook (the paper has no counterpart; not part of any
 * operation).  The next radix sort on this host thread (an hs_sparse call
 * with at least one tuple, or an hs_spref that sorts) runs its passes with a
 * look-back poll limit of
 * `spin_limit` (at least 1) and with tile `withhold_tile` (0-based, tiles of
 * 4096 tuples) never publishing its digit counts, so the bounded wait of a
 * later tile runs out: the call then returns HS_ETIMEDOUT, every store of
 * the pass stays inside its buffers (they are bounds-checked) and nothing is
 * left allocated.  The setting is consumed by that one call.  Returns HS_OK,
 * or HS_EINVAL for spin_limit < 1 or withhold_tile < 0. */
int hs_test_lookback_expiry(int spin_limit, int64_t withhold_tile);

/* Phase timing.  With hs_profile_enable(1) every later call records CUDA
 * events on its stream around each phase; hs_profile_read copies the
 * accumulated milliseconds, launch counts and names of up to `cap` phases
 * and returns the number of phases.  hs_profile_reset clears the totals.
 * Intended for benchmarking; adds event records, no synchronisation beyond
 * the product's own. */
void hs_profile_enable(int on);
void hs_profile_reset(void);
int hs_profile_read(double *ms, int64_t *launches, const char **names, int cap);

#ifdef __cplusplus
}
#endif
#endif /* HSPGEMM_H */
